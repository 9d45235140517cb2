"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No GPU.  Each test cites the passage of arXiv 2304.05505 it follows."""
import json
import os

import numpy as np
import pytest

from oracle import thc_oracle as O
from paper_2304_05505_gb300 import cells

import pins

FULL_GRID_CASES = [((2, 2, 2), (10, 10, 10)), ((3, 3, 3), (8, 8, 8)), ((3, 2, 4), (8, 8, 8))]


@pytest.mark.parametrize("mesh,grid", FULL_GRID_CASES)
def test_full_grid_identity(mesh, grid):
    """Every grid point an interpolation point: the THC-oo-K energy and K C
    (Eq. thcoccrik, Algorithm 2) equal brute-force periodic exchange
    (Eq. pbcexchange) on the grid.  The 3x3x3 and 3x2x4 meshes detect a wrong
    sign of q = k' - k (on 2x2x2 every q is its own inverse)."""
    r = pins.check_full_grid(mesh, grid)
    assert r["ex_rel"] < 1e-10
    assert r["kc_rel"] < 1e-10
    assert r["ex"] < 0


def test_full_grid_golden():
    """Stored brute-force energies (written by tests/golden/make_golden.py,
    which calls only oracle/ and the input generator) still reproduce."""
    path = os.path.join(os.path.dirname(__file__), "golden", "full_grid_c0.json")
    gold = json.load(open(path))
    for case in gold["cases"]:
        c, Xg, C, V, bf = pins.full_grid_case(tuple(case["mesh"]), tuple(case["grid"]))
        assert abs(bf["Ex"] - case["Ex_bruteforce"]) < 1e-10 * abs(case["Ex_bruteforce"])
        out = O.build(Xg, C, V, c.mesh, route="fft")
        assert abs(out["Ex"] - case["Ex_bruteforce"]) < 1e-10 * abs(case["Ex_bruteforce"])


@pytest.mark.parametrize("mesh", [(2, 2, 2), (3, 3, 3), (4, 4, 4), (3, 4, 2), (1, 1, 1), (5, 1, 1)])
def test_direct_sum_equals_fft(mesh):
    """Sec. 2.2: the q sum is a convolution in k space, so the O(N_k^2) double
    sum equals the FFT route (cross-correlation theorem)."""
    assert pins.check_conv_routes(mesh) < 1e-12


def test_convolution_index_map():
    """q = k' - k (Sec. 2.2): a single D term and a single V term land at
    k = k' - q, wrapped on a non-cubic mesh."""
    assert pins.check_conv_single_term() < 1e-12


@pytest.mark.parametrize("mesh", [(2, 2, 2), (3, 3, 3)])
def test_hermitian(mesh):
    """K^k and M^k are Hermitian: a Hadamard product of Hermitian D^k' and V^q
    summed over k'."""
    p = pins.model_case(mesh)
    assert pins.check_hermitian(p.X, p.C, p.V, p.cell.mesh) < 1e-13


@pytest.mark.parametrize("mesh", [(2, 2, 2), (3, 3, 3)])
def test_psd_and_sign(mesh):
    """V^q PSD => M^k PSD (Schur product theorem) => K^k PSD and E_x <= 0."""
    p = pins.model_case(mesh)
    r = pins.check_psd(p.X, p.C, p.V, p.cell.mesh)
    assert r["mineig_M"] > -1e-12
    assert r["mineig_K"] > -1e-12
    assert r["ex"] < 0
    assert abs(r["ex_imag"]) < 1e-13 * abs(r["ex"])


@pytest.mark.parametrize("mesh", [(3, 3, 3), (4, 4, 4), (3, 2, 4)])
def test_time_reversal(mesh):
    """X^{-k} = conj X^k, C^{-k} = conj C^k, V^{-q} = conj V^q give
    K^{-k} = conj(K^k)."""
    p = pins.model_case(mesh, nisdf=24)
    assert pins.check_time_reversal(p.X, p.C, p.V, p.cell.mesh) < 1e-12


def test_gauge_covariance():
    """C^k -> C^k U^k (unitary) gives KC -> KC U and leaves E_x unchanged."""
    p = pins.model_case((3, 3, 3))
    r = pins.check_gauge(p.X, p.C, p.V, p.cell.mesh)
    assert r["kc"] < 1e-12 and r["ex"] < 1e-12


def test_energy_trace():
    """E_x = -(1/N_k) sum_k Tr(C^kH (K C)^k) equals the point-space route of
    Eq. thcoccrik."""
    p = pins.model_case((3, 3, 3))
    assert pins.check_energy_trace(p.X, p.C, p.V, p.cell.mesh) < 1e-12


def test_gamma_point_formula():
    """N_k = 1 reduces to the Gamma-point THC exchange, Eq. thcexchange,
    summed literally with the AO density matrix."""
    p = pins.model_case((1, 1, 1), nisdf=30)
    assert pins.check_gamma(p.X, p.C, p.V) < 1e-12


def test_scalar_closed_form():
    """n = 1 and N_P = 1: every step is a scalar, done with explicit loops."""
    assert pins.check_scalar() < 1e-13


def test_linear_in_kernel():
    """K C is linear in V."""
    p = pins.model_case((2, 2, 2))
    assert pins.check_linear_in_V(p.X, p.C, p.V, p.cell.mesh) < 1e-12


def test_random_inputs_symmetries():
    """The unstructured random generator keeps the symmetries the pins use."""
    r = cells.random_problem((3, 2, 2), nbas=6, nocc=2, nisdf=7)
    assert pins.check_hermitian(r["X"], r["C"], r["V"], r["mesh"]) < 1e-12
    assert pins.check_time_reversal(r["X"], r["C"], r["V"], r["mesh"]) < 1e-12


# ---------------------------------------------------------------------------
# the Coulomb kernel, G set and q representatives of the setup oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L", [8.0, 9.0])
def test_gaussian_self_energy_closed_form(L):
    """The oracle's ISDF kernel of a repeated unit Gaussian charge gives its
    Coulomb energy with the G = 0 term dropped: the Gaussian self-energy plus
    the simple-cubic Madelung term and the background term (Ewald)."""
    r = pins.check_gaussian_self_energy(L)
    assert r["rel"] < 1e-12, r
    assert r["imag"] < 1e-14


@pytest.mark.parametrize("mesh", [(2, 2, 2), (3, 3, 3), (3, 2, 4)])
@pytest.mark.parametrize("G0", [(0, 0, 0), (1, 0, 0), (0, -1, 2)])
def test_plane_wave_kernel_closed_form(mesh, G0):
    """A plane-wave interpolation vector gives 4 pi / |G0 + q|^2 (Omega / N_k)
    at every q of the mesh, with q the shortest vector of its coset found by
    brute force (orthorhombic cell; zone-boundary q averaged over its ties)."""
    lattice = np.diag([6.95, 8.9, 6.45])
    assert pins.check_plane_wave_kernel(lattice, (8, 8, 8), mesh, G0) < 1e-13


@pytest.mark.parametrize("grid", [(8, 7, 6), (5, 5, 5), (16, 16, 16)])
def test_gset_is_the_symmetric_fft_set(grid):
    assert pins.check_gset_symmetric(grid) == 0.0


def test_rowblock_build_equals_build():
    """Running steps 2-4a a block of rows at a time (for cells too large to
    hold D and M) gives the build itself: the (P, Q) elements are independent."""
    r = cells.random_problem((3, 2, 2), nbas=9, nocc=3, nisdf=37, seed=4)
    a = O.build(r["X"], r["C"], r["V"], r["mesh"], route="direct")
    b = O.build_rowblocks(r["X"], r["C"], r["V"], r["mesh"], block=8)
    assert np.abs(a["KC"] - b["KC"]).max() <= 1e-13 * np.abs(a["KC"]).max()
    assert abs(a["Ex"] - b["Ex"]) <= 1e-13 * abs(a["Ex"])
