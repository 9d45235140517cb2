"""Pins of the FP64 oracle of interpolation-point selection and the ISDF fit.

No GPU.  The points are the pivots of a greedy pivoted Cholesky of the Gram
matrix of occupied pair products (the metric of the least-squares fit of
Eq. pbcinterpvec, restricted to occupied orbitals as in Eq. orbprodoo);
pivoted Cholesky is the QR-with-column-pivoting selection of Sec. 2.1 in
exact arithmetic."""
import numpy as np
import pytest
import scipy.linalg.lapack as lapack

from oracle import setup_oracle as S


def rand_u(nf, nr, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(nf, nr)) + 1j * rng.normal(size=(nf, nr))


@pytest.mark.parametrize("nf,nr,seed", [(6, 40, 3), (4, 60, 4), (8, 90, 5)])
def test_pivots_equal_lapack(nf, nr, seed):
    """The greedy rule (largest residual diagonal) is LAPACK dpstrf's; on the
    explicitly formed Gram matrix both give the same pivots and rank."""
    U = rand_u(nf, nr, seed)
    A = S.pair_gram(U)
    r = S.pivoted_cholesky(U, nr)
    _, piv, rank, info = lapack.dpstrf(A.copy(), tol=-1)
    assert rank == len(r["points"]) == min(nf * nf, nr)
    assert np.array_equal(r["points"], piv[:rank] - 1)


def test_rank_terminated_fit_is_exact():
    """With as many points as the Gram rank every occupied pair product
    conj(u_f) u_g is interpolated exactly (Eq. orbprodoo holds with equality)."""
    U = rand_u(5, 70, 7)
    r = S.pivoted_cholesky(U, 70)
    assert len(r["points"]) == 25
    assert r["resid"].sum() <= 1e-12 * np.sum(np.abs(U) ** 2, axis=0).dot(np.sum(np.abs(U) ** 2, axis=0))
    xi = S.isdf_fit(U, r["points"])
    for f in range(5):
        for g in range(5):
            pair = U[f].conj() * U[g]
            approx = pair[r["points"]] @ xi
            assert np.abs(approx - pair).max() < 1e-8 * np.abs(pair).max()


def test_fit_error_never_increases():
    """Systematically improvable (Sec. 4.1): more points never raise the error."""
    U = rand_u(6, 120, 8)
    r = S.pivoted_cholesky(U, 36)
    errs = [S.fit_error(U, r["points"][:m]) for m in range(1, 37)]
    assert all(b <= a * (1 + 1e-9) + 1e-12 for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6


def test_residual_diagonal_is_schur_complement():
    """The residual diagonal after m pivots equals diag(A - A_:P A_PP^-1 A_P:)."""
    U = rand_u(4, 50, 9)
    A = S.pair_gram(U)
    r = S.pivoted_cholesky(U, 10)
    P = r["points"]
    schur = np.diag(A) - np.einsum("rp,pq,rq->r", A[:, P], np.linalg.inv(A[np.ix_(P, P)]), A[:, P])
    assert np.abs(r["resid"] - np.maximum(schur, 0)).max() < 1e-9 * np.abs(np.diag(A)).max()


# ---------------------------------------------------------------------------
# the kernel built from interpolation vectors
# ---------------------------------------------------------------------------

from paper_2304_05505_gb300 import cells  # noqa: E402
from oracle import thc_oracle as O  # noqa: E402


@pytest.mark.parametrize("mesh", [(2, 2, 2), (3, 3, 3)])
def test_delta_vectors_give_the_full_grid_kernel(mesh):
    """With every grid point a point and xi = delta (an exact interpolation),
    the reciprocal-space kernel of the vectors is the closed-form full-grid
    kernel, which is itself pinned against the brute-force grid exchange."""
    c = cells.make_cell("C0", mesh=mesh, grid=(6, 6, 6))
    ng = 216
    V = S.kernel_from_xi(c.lattice, c.grid, c.mesh, np.eye(ng), np.arange(ng))
    ref = S.full_grid_kernel(c.lattice, c.grid, c.mesh)
    assert np.abs(V - ref).max() <= 1e-12 * np.abs(ref).max()


def _toy_u(mesh, grid):
    c = cells.make_cell("C0", mesh=mesh, grid=grid)
    pts = cells.grid_points(c, 1)
    kf = cells.kmesh_frac(c.mesh)
    Xg = cells.bloch_collocation(c, pts, kf)
    C = cells.occupied_coefficients(c)
    psi = np.einsum("kmr,kmi->kir", Xg, C)
    phase = np.exp(-1j * (pts @ (kf @ c.recip).T)).T
    U = (psi * phase[:, None, :]).reshape(-1, pts.shape[0])
    return c, Xg, C, U


def test_fitted_kernel_symmetries():
    """V^q Hermitian and positive semidefinite, V^{-q} = conj(V^q), and the
    vectors interpolate exactly at the points (xi_P(r_Q) = delta_PQ)."""
    c, _, _, U = _toy_u((3, 3, 3), (8, 8, 8))
    r = S.pivoted_cholesky(U, 40)
    xi = S.isdf_fit(U, r["points"])
    assert np.abs(xi[:, r["points"]] - np.eye(40)).max() < 1e-9
    V = S.fit_kernel(c.lattice, c.grid, c.mesh, U, r["points"])
    scale = np.abs(V).max()
    mk = cells.minus_k_index(c.mesh)
    for q in range(V.shape[0]):
        assert np.abs(V[q] - V[q].conj().T).max() <= 1e-13 * scale
        assert np.linalg.eigvalsh(V[q]).min() >= -1e-12 * scale
        assert np.abs(V[mk[q]] - V[q].conj()).max() <= 1e-13 * scale


def test_gamma_exchange_of_an_exact_fit_is_the_grid_exchange():
    """Gamma only: with rank-terminated points the fit reproduces every
    occupied pair product, so the build's E_x with the fitted kernel equals the
    brute-force grid exchange (Eq. orbprodoo with equality)."""
    c, Xg, C, U = _toy_u((1, 1, 1), (8, 8, 8))
    r = S.pivoted_cholesky(U, 512)
    P = r["points"]
    assert len(P) < 512
    V = S.fit_kernel(c.lattice, c.grid, c.mesh, U, P)
    got = O.build(Xg[:, :, P], C, V, c.mesh)
    bf = S.brute_force_exchange(c.lattice, c.grid, c.mesh, Xg, C)
    assert abs(got["Ex"] - bf["Ex"]) <= 1e-10 * abs(bf["Ex"])
