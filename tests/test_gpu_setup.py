"""GPU FP64 pivoted-Cholesky interpolation points vs the oracle, through the C ABI.

Pivot indices are compared exactly (integer output); the residual diagonal
within 1e-10 of the Gram scale (FP64 with a different summation order)."""
import numpy as np
import pytest

from oracle import setup_oracle as S
from paper_2304_05505_gb300 import cells

pytestmark = pytest.mark.gpu


def rand_u(nf, nr, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(nf, nr)) + 1j * rng.normal(size=(nf, nr))


@pytest.fixture(scope="module")
def thc_mod(cuda_required):
    import os

    from paper_2304_05505_gb300 import build_lib, thc
    if not os.path.exists(thc.LIB_PATH):
        build_lib.build()
    thc.load()
    return thc


@pytest.mark.parametrize("nf,nr,npts,seed", [(6, 40, 40, 3), (8, 300, 48, 4), (12, 1000, 100, 5), (3, 17, 5, 6)])
def test_pivots_match_oracle(thc_mod, nf, nr, npts, seed):
    import torch
    U = rand_u(nf, nr, seed)
    ref = S.pivoted_cholesky(U, npts)
    pts, resid = thc_mod.thc_select_points(torch.from_numpy(U).cuda(), npts)
    assert np.array_equal(pts, ref["points"])
    scale = float(np.max(np.sum(np.abs(U) ** 2, axis=0) ** 2))
    assert np.abs(resid.cpu().numpy() - ref["resid"]).max() <= 1e-10 * scale


def test_toy_cell_orbitals(thc_mod):
    """Points of the toy cubic cell (48 from the 16^3 grid, 2x2x2 k, 4 orbitals):
    the occupied orbitals' periodic parts on the grid as candidates."""
    import torch
    c = cells.make_cell("C0")
    pts = cells.grid_points(c, 1)
    kf = cells.kmesh_frac(c.mesh)
    Xg = cells.bloch_collocation(c, pts, kf)
    C = cells.occupied_coefficients(c)
    psi = np.einsum("kmr,kmi->kir", Xg, C)
    phase = np.exp(-1j * (pts @ (kf @ c.recip).T)).T            # exp(-i k.r), [k][r]
    U = (psi * phase[:, None, :]).reshape(-1, pts.shape[0])     # u^k_i(r), f = (k, i)
    ref = S.pivoted_cholesky(U, 48)
    got, _ = thc_mod.thc_select_points(torch.from_numpy(np.ascontiguousarray(U)).cuda(), 48)
    assert np.array_equal(got, ref["points"])


def test_rank_termination(thc_mod):
    import torch
    U = rand_u(4, 200, 11)
    got, resid = thc_mod.thc_select_points(torch.from_numpy(U).cuda(), 100)
    assert len(got) == 16                                       # rank of the pair Gram matrix
    assert float(resid.sum()) <= 1e-12 * float(np.sum(np.sum(np.abs(U) ** 2, axis=0) ** 2))
