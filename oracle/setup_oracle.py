"""FP64 CPU oracle of the exchange on a real-space grid and of the ISDF kernel.

TEST INFRASTRUCTURE (see ``oracle/thc_oracle.py`` for who may import it).

Two objects the build is pinned against:

* ``full_grid_kernel``: the ISDF kernel when every grid point is an
  interpolation point and the interpolation vectors are grid deltas, so the
  fit of Eq. orbprodoo is exact.  Then the GPW form of ``M^q`` (Sec. 2.2)
  has the closed form
  ``V^q[P, Q] = Omega / (N_k N_g^2) sum_G v(G + q) exp(-i (G + q).(r_P - r_Q))``.
* ``brute_force_exchange``: the periodic exchange of Eq. pbcexchange for the
  occupied orbitals on the grid, from the FFT of every pair density:
  ``E_x = -(Omega / N_k^2) sum_{k k' i j} sum_G v(G + q) |g_G|^2`` with
  ``g(r) = exp(-i q.r) conj(psi^k_i(r)) psi^{k'}_j(r)``, ``q = k' - k``.

Conventions where the paper is silent (each is listed with the other
readings of the paper in the design notes):

* ``v(K) = 4 pi / |K|^2`` with ``K = 0`` left out; no Madelung correction.
* The G set is the grid's FFT frequencies with the Nyquist planes of even
  dimensions dropped, so it is symmetric under G -> -G.
* A wrapped q whose fractional component is exactly 1/2 has two minimum-image
  representatives along that axis; the kernel (and the brute-force sum) is
  the mean over all representatives.  Then ``V^{-q} = conj(V^q)`` exactly and
  the result does not depend on a choice of sign.
"""
from __future__ import annotations

import itertools

import numpy as np

from .thc_oracle import mesh_coords, q_index


def recip_vectors(lattice: np.ndarray) -> np.ndarray:
    return 2.0 * np.pi * np.linalg.inv(lattice).T


def representatives(qco, mesh) -> list:
    """Minimum-image fractional representatives of q = qco / mesh."""
    opts = []
    for a in range(3):
        f = (int(qco[a]) % mesh[a]) / mesh[a]
        if abs(f - 0.5) < 1e-12:
            opts.append([0.5, -0.5])
        elif f > 0.5:
            opts.append([f - 1.0])
        else:
            opts.append([f])
    return [np.array(t) for t in itertools.product(*opts)]


def symmetric_gset(grid) -> np.ndarray:
    """Integer G triples of the grid without the Nyquist planes."""
    rng = []
    for g in grid:
        h = (g - 1) // 2
        rng.append(np.arange(-h, h + 1))
    m = np.stack(np.meshgrid(*rng, indexing="ij"), axis=-1).reshape(-1, 3)
    return m


def grid_frac(grid) -> np.ndarray:
    axes = [np.arange(g) / g for g in grid]
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)


def coulomb(K: np.ndarray) -> np.ndarray:
    K2 = np.einsum("gi,gi->g", K, K)
    out = np.zeros_like(K2)
    nz = K2 > 1e-12
    out[nz] = 4.0 * np.pi / K2[nz]
    return out


def full_grid_kernel(lattice, grid, mesh) -> np.ndarray:
    """V[q, P, Q] with every grid point an interpolation point (xi = delta)."""
    B = recip_vectors(lattice)
    vol = abs(np.linalg.det(lattice))
    r = grid_frac(grid) @ lattice                 # (N_g, 3)
    ng = r.shape[0]
    nk = int(np.prod(mesh))
    gm = symmetric_gset(grid)
    V = np.zeros((nk, ng, ng), dtype=np.complex128)
    for q, qco in enumerate(mesh_coords(mesh)):
        reps = representatives(qco, mesh)
        for qr in reps:
            K = (gm + qr[None, :]) @ B
            v = coulomb(K)
            A = np.exp(-1j * (r @ K.T)) * np.sqrt(v)[None, :]
            V[q] += (A @ A.conj().T) / len(reps)
    V *= vol / (nk * ng * ng)
    return V


def brute_force_exchange(lattice, grid, mesh, Xgrid, C) -> dict:
    """E_x and (K C)^k from the FFT of every occupied (and AO-occupied) pair.

    Xgrid: (N_k, N, N_g) Bloch basis on the grid (phase included); C: (N_k, N, n).
    (K C)^k[mu, i] = (Omega/N_k) sum_{k' j} sum_G v(G+q) h_G conj(g_G) with
    h(r) = exp(-i q.r) conj(X^k_mu(r)) psi^{k'}_j(r)."""
    B = recip_vectors(lattice)
    vol = abs(np.linalg.det(lattice))
    f = grid_frac(grid)
    r = f @ lattice
    ng = r.shape[0]
    nk, nb, n = C.shape
    gm = symmetric_gset(grid)
    flat = np.ravel_multi_index(tuple((gm % np.array(grid)).T), grid)
    psi = np.einsum("kmr,kmi->kir", Xgrid, C)     # psi^k_i(r), phase included
    Ex = 0.0 + 0.0j
    KC = np.zeros((nk, nb, n), dtype=np.complex128)
    co = mesh_coords(mesh)
    for k in range(nk):
        for kp in range(nk):
            q = q_index(mesh, k, kp)
            reps = representatives(co[q], mesh)
            for qr in reps:
                w = 1.0 / len(reps)
                K = (gm + qr[None, :]) @ B
                v = coulomb(K)
                ph = np.exp(-1j * (r @ (qr @ B)))
                g = ph[None, None, :] * psi[k].conj()[:, None, :] * psi[kp][None, :, :]
                gh = np.fft.fftn(g.reshape((n, n) + tuple(grid)), axes=(2, 3, 4))
                gh = gh.reshape(n, n, ng)[:, :, flat] / ng
                Ex += -(vol / nk ** 2) * w * np.sum(v[None, None, :] * np.abs(gh) ** 2)
                h = ph[None, None, :] * Xgrid[k].conj()[:, None, :] * psi[kp][None, :, :]
                hh = np.fft.fftn(h.reshape((nb, n) + tuple(grid)), axes=(2, 3, 4))
                hh = hh.reshape(nb, n, ng)[:, :, flat] / ng
                KC[k] += (vol / nk) * w * np.einsum("mjg,g,ijg->mi", hh, v, gh.conj())
    return dict(Ex=float(Ex.real), Ex_imag=float(Ex.imag), KC=KC)


# ----------------------------------------------------------------------------
# interpolation points: pivoted Cholesky of the occupied-pair Gram matrix
# ----------------------------------------------------------------------------

def pair_gram(U: np.ndarray) -> np.ndarray:
    """A(r, r') = |sum_f conj(U[f, r]) U[f, r']|^2 for U[f, r] = u^k_i(r),
    f = (k, i): the Gram matrix of all occupied pair products
    conj(u^k_i) u^k'_j (the metric of the fit in Eq. pbcinterpvec, restricted
    to occupied orbitals as in Eq. orbprodoo)."""
    B = U.conj().T @ U
    return np.abs(B) ** 2


def pivoted_cholesky(U: np.ndarray, npts: int, rel_tol: float = 1e-14) -> dict:
    """Greedy pivoted Cholesky of pair_gram(U) without forming it: the pivot
    is the largest residual diagonal (the lowest index among equal ones); stop
    after npts pivots or when the residual trace falls to rel_tol times the
    trace of A.  Returns pivots, the residual diagonal and the factor columns."""
    rho = np.sum(np.abs(U) ** 2, axis=0)
    d = rho ** 2                                   # A(r, r)
    tr0 = d.sum()
    cols, piv = [], []
    for _ in range(npts):
        if d.sum() <= rel_tol * tr0:
            break
        p = int(np.argmax(d))
        a = np.abs(U.conj().T @ U[:, p]) ** 2      # column A(:, p)
        for L in cols:
            a = a - L * L[p]
        ell = a / np.sqrt(d[p])
        d = np.maximum(d - ell ** 2, 0.0)
        d[p] = 0.0
        cols.append(ell)
        piv.append(p)
    return dict(points=np.array(piv, dtype=np.int64), resid=d, L=np.array(cols))


def isdf_fit(U: np.ndarray, points: np.ndarray) -> np.ndarray:
    """Interpolation vectors xi[P, r] = sum_Q S^-1[P, Q] A(r_Q, r), S = A[points,
    points] (the least-squares fit of Eq. orbprodoo; S is the ISDF metric)."""
    A = pair_gram(U)
    S = A[np.ix_(points, points)]
    return np.linalg.solve(S, A[points, :])


def fit_error(U: np.ndarray, points: np.ndarray) -> float:
    """Relative residual sqrt(sum_r d_r / sum_r A_rr) of the pivoted-Cholesky
    (Schur complement) diagonal after selecting `points`."""
    A = pair_gram(U)
    S = A[np.ix_(points, points)]
    Ar = A[:, points]
    d = np.diag(A) - np.einsum("rp,pq,rq->r", Ar, np.linalg.inv(S), Ar)
    return float(np.sqrt(max(d.sum(), 0.0) / np.trace(A)))


# ----------------------------------------------------------------------------
# the ISDF kernel from the interpolation vectors
# ----------------------------------------------------------------------------

def kernel_from_xi(lattice, grid, mesh, xi: np.ndarray, points: np.ndarray) -> np.ndarray:
    """V[q, P, Q] of the interpolation vectors xi[P, r] (Sec. 2.2, the Coulomb
    kernel between two interpolation vectors taken in reciprocal space):

        V^q[P, Q] = 1/(N_k Omega) exp(-i q.(r_P - r_Q))
                    sum_G v(G + q) xh_P(G) conj(xh_Q(G)),
        xh_P(G) = (Omega / N_g) sum_r xi_P(r) exp(-i G.r),

    with the pair phase folded in as for every kernel of the build, the
    symmetric G set, and the mean over the minimum-image representatives of a
    q on the zone boundary (as in full_grid_kernel)."""
    B = recip_vectors(lattice)
    vol = abs(np.linalg.det(lattice))
    ng = int(np.prod(grid))
    nk = int(np.prod(mesh))
    npts = len(points)
    rP = (grid_frac(grid) @ lattice)[points]
    gm = symmetric_gset(grid)
    flat = np.ravel_multi_index(tuple((gm % np.array(grid)).T), grid)
    xh = np.fft.fftn(np.asarray(xi, dtype=np.complex128).reshape((npts,) + tuple(grid)), axes=(1, 2, 3))
    xh = xh.reshape(npts, ng)[:, flat] * (vol / ng)
    V = np.zeros((nk, npts, npts), dtype=np.complex128)
    for q, qco in enumerate(mesh_coords(mesh)):
        reps = representatives(qco, mesh)
        for qr in reps:
            qc = qr @ B
            v = coulomb((gm + qr[None, :]) @ B)
            A = xh * np.sqrt(v)[None, :] * np.exp(-1j * (rP @ qc))[:, None]
            V[q] += (A @ A.conj().T) / len(reps)
    return V / (nk * vol)


def fit_kernel(lattice, grid, mesh, U: np.ndarray, points: np.ndarray) -> np.ndarray:
    """The ISDF kernel of the occupied-pair fit: kernel_from_xi of isdf_fit."""
    return kernel_from_xi(lattice, grid, mesh, isdf_fit(U, points), points)
