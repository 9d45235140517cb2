"""The generator's torch route (set_accelerator) makes the same inputs as its
numpy route: run here with torch on the CPU, to rounding."""
import numpy as np
import pytest

from paper_2304_05505_gb300 import cells


def _both(fn):
    ref = fn()
    cells.set_accelerator("cpu")
    try:
        got = fn()
    finally:
        cells.set_accelerator(None)
    return ref, got


@pytest.mark.parametrize("name,over", [("C0", {}), ("C1", dict(grid=(12, 16, 12), mesh=(2, 1, 2), nocc=6))])
def test_bloch_collocation_routes_agree(name, over):
    c = cells.make_cell(name, **over)
    rng = np.random.default_rng(3)
    pts = rng.uniform(size=(257, 3)) @ c.lattice
    kf = cells.kmesh_frac(c.mesh)
    ref, got = _both(lambda: cells.bloch_collocation(c, pts, kf))
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_orbitals_routes_agree():
    c = cells.make_cell("C0", mesh=(3, 1, 2))
    (C0, U0), (C1, U1) = _both(lambda: (lambda C: (C, cells.grid_orbitals(c, C)))(cells.occupied_coefficients(c)))
    # eigenvectors are fixed up to a phase per column; the products they make
    # (the density matrix per k) are not
    P0 = np.einsum("kmi,kni->kmn", C0, C0.conj())
    P1 = np.einsum("kmi,kni->kmn", C1, C1.conj())
    assert np.abs(P1 - P0).max() <= 1e-9 * np.abs(P0).max()
    Ug = cells.grid_orbitals(c, C0)
    cells.set_accelerator("cpu")
    try:
        Ut = cells.grid_orbitals(c, C0, as_tensor=True)
    finally:
        cells.set_accelerator(None)
    assert np.abs(Ut.numpy() - Ug).max() <= 1e-12 * np.abs(Ug).max()


def test_virtual_orbitals_complete_an_orthonormal_set():
    """orbital_coefficients(cell, nvir): the occupied part spans what
    occupied_coefficients gives, the occupied and virtual orbitals together
    are orthonormal in the overlap metric of the generator's quadrature
    (S^k = (Omega/N_q) sum_r conj(phi_mu(r)) phi_nu(r)), and the virtual ones
    keep C^{-k} = conj(C^k).  These are the inputs of the orbital gradient."""
    c = cells.make_cell("C0", mesh=(3, 1, 2))
    C, Cv = cells.orbital_coefficients(c, 4)
    C0 = cells.occupied_coefficients(c)
    P = np.einsum("kmi,kni->kmn", C, C.conj())
    P0 = np.einsum("kmi,kni->kmn", C0, C0.conj())
    assert np.abs(P - P0).max() <= 1e-9 * np.abs(P0).max()
    pts = cells.grid_points(c, c.quad_stride)
    kf = cells.kmesh_frac(c.mesh)
    phi = cells.bloch_collocation(c, pts, kf)                      # [k][mu][r]
    Sk = (c.volume / pts.shape[0]) * np.einsum("kmr,knr->kmn", phi.conj(), phi)
    Call = np.concatenate([C, Cv], axis=2)
    G = np.einsum("kma,kmn,knb->kab", Call.conj(), Sk, Call)
    assert np.abs(G - np.eye(Call.shape[2])[None]).max() <= 1e-9
    mk = cells.minus_k_index(c.mesh)
    assert np.abs(Cv[mk] - Cv.conj()).max() <= 1e-12 * np.abs(Cv).max()
