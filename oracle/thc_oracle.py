"""FP64 CPU oracle of the THC-oo-K exchange build (arXiv 2304.05505).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The CUDA library
shares no code with it, and it imports nothing of the library.

It is the plain definition of what one build computes, step by step, in
complex128, in the most obvious order.  Only numpy matmul (and, for the
second route of step 3, numpy's FFT) serve as library primitives.  Notation
(the paper's symbols in brackets):

* ``X[k, mu, P]`` basis function mu at point P, Bloch phase included
  [``u^k_mu(r_P)`` times ``exp(i k.r_P)``].
* ``C[k, mu, i]`` occupied coefficients.
* ``V[q, P, Q]`` ISDF Coulomb kernel with the pair phase folded in
  [``M^q_PQ`` times ``exp(-i q.(r_P - r_Q))``].
* ``Psi[k, P, i]`` occupied orbitals at the points [``u^k_i(r_P)`` with phase].
* ``D[k, P, Q]`` point-space density, ``M[k, P, Q]`` the k-convolved
  intermediate [``X^k_PQ`` of Algorithms 1 and 2].

k and q share one mesh index ``(n1 * N2 + n2) * N3 + n3`` on the
Gamma-centred mesh, and ``q = k' - k`` wraps onto the mesh (the paper defines
q that way in Sec. 2.2).

Parity pins for every function here live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# mesh helpers
# ----------------------------------------------------------------------------

def mesh_coords(mesh) -> np.ndarray:
    """(N_k, 3) integer coordinates (n1, n2, n3) in mesh index order."""
    n1, n2, n3 = mesh
    a, b, c = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    return np.stack([a.ravel(), b.ravel(), c.ravel()], axis=1)


def mesh_index(mesh, coord) -> int:
    n1, n2, n3 = mesh
    a, b, c = (int(coord[0]) % n1, int(coord[1]) % n2, int(coord[2]) % n3)
    return (a * n2 + b) * n3 + c


def q_index(mesh, k: int, kp: int) -> int:
    """Mesh index of q = k' - k, wrapped (Sec. 2.2: q = k' - k)."""
    co = mesh_coords(mesh)
    return mesh_index(mesh, co[kp] - co[k])


# ----------------------------------------------------------------------------
# the five steps
# ----------------------------------------------------------------------------

def collocate(X: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Step 1: Psi^k[P, i] = sum_mu X^k[mu, P] C^k[mu, i].

    The occupied orbitals at the interpolation points, u^k_i(r_P) of
    Eq. thcoccrik; a transpose of X, no conjugate."""
    nk = X.shape[0]
    return np.stack([X[k].T @ C[k] for k in range(nk)])


def density(Psi: np.ndarray) -> np.ndarray:
    """Step 2: D^k[P, Q] = sum_i Psi^k[P, i] conj(Psi^k[Q, i]).

    The inner sum over i in the convolution step of Algorithm 2."""
    nk = Psi.shape[0]
    return np.stack([Psi[k] @ Psi[k].conj().T for k in range(nk)])


def density_rows(Psi: np.ndarray, rows) -> np.ndarray:
    """Step 2 for the rows P in ``rows`` only: D^k[P, Q] for all k and Q.

    Every (P, Q) element of steps 2 and 3 is independent of the others, so
    the build on the largest cells runs them a block of rows at a time
    (D and M for all rows do not fit in memory at once)."""
    nk = Psi.shape[0]
    return np.stack([Psi[k][rows] @ Psi[k].conj().T for k in range(nk)])


def kconv_direct(D: np.ndarray, V: np.ndarray, mesh) -> np.ndarray:
    """Step 3, defining form: M^k = sum_{k'} D^{k'} o V^{q(k, k')}, q = k' - k.

    The O(N_k^2) double sum over k and k' of Eq. kpointthck / Algorithm 2
    (with k' = k + q), element by element (Hadamard) in P, Q."""
    nk = D.shape[0]
    M = np.zeros_like(D)
    for k in range(nk):
        for kp in range(nk):
            M[k] += D[kp] * V[q_index(mesh, k, kp)]
    return M


def kconv_fft(D: np.ndarray, V: np.ndarray, mesh) -> np.ndarray:
    """Step 3, the paper's route (Sec. 2.2: the q sum is a convolution in k
    space, done by FFT in O(N_k log N_k)).

    Per (P, Q): forward DFT of D over the mesh, multiply by the DFT of V taken
    with the opposite sign (the q sum is a cross-correlation because
    q = k' - k), inverse DFT."""
    nk, npt = D.shape[0], D.shape[1]
    shp = tuple(mesh) + D.shape[1:]
    Dh = np.fft.fftn(D.reshape(shp), axes=(0, 1, 2))
    Vc = np.fft.ifftn(V.reshape(shp), axes=(0, 1, 2)) * nk
    M = np.fft.ifftn(Dh * Vc, axes=(0, 1, 2))
    return M.reshape(D.shape)


def apply_M(M: np.ndarray, Psi: np.ndarray) -> np.ndarray:
    """Step 4a: Y^k = M^k Psi^k (first half of the K_ij step of Algorithm 2)."""
    return np.stack([M[k] @ Psi[k] for k in range(M.shape[0])])


def backproject(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Step 4b: (K C)^k[mu, i] = sum_P conj(X^k[mu, P]) Y^k[P, i].

    With K^k = conj(X^k) M^k X^{kT} (the K step of Algorithm 1), this is K^k C^k."""
    return np.stack([X[k].conj() @ Y[k] for k in range(X.shape[0])])


def exchange_energy(Psi: np.ndarray, Y: np.ndarray) -> complex:
    """Step 5, Eq. thcoccrik: E_x = -(1/N_k) sum_k sum_{P,i} conj(Psi^k[P,i]) Y^k[P,i].

    Closed-shell exchange per cell.  Returned complex; the imaginary part is
    a residual that vanishes for Hermitian V."""
    nk = Psi.shape[0]
    return -np.sum(Psi.conj() * Y) / nk


def build(X, C, V, mesh, route: str = "direct", keep: bool = False) -> dict:
    """One exchange build: KC = K^k C^k for every k and E_x.

    ``route`` picks the defining double sum ("direct") or the FFT route
    ("fft") for step 3."""
    Psi = collocate(X, C)
    D = density(Psi)
    if route == "direct":
        M = kconv_direct(D, V, mesh)
    elif route == "fft":
        M = kconv_fft(D, V, mesh)
    else:
        raise ValueError(route)
    Y = apply_M(M, Psi)
    KC = backproject(X, Y)
    ex = exchange_energy(Psi, Y)
    out = dict(KC=KC, Ex=float(ex.real), Ex_imag=float(ex.imag))
    if keep:
        out.update(Psi=Psi, D=D, M=M, Y=Y)
    return out


def build_rowblocks(X, C, V, mesh, block: int = 200) -> dict:
    """The same build with steps 2-4a run on blocks of ``block`` rows P (the
    FFT route of step 3 on each block), for cells whose D and M do not fit in
    memory whole.  Steps 1, 4b and 5 are those of ``build``."""
    Psi = collocate(X, C)
    npt = Psi.shape[1]
    Y = np.zeros_like(Psi)
    for r0 in range(0, npt, block):
        rows = slice(r0, min(npt, r0 + block))
        M = kconv_fft(density_rows(Psi, rows), V[:, rows, :], mesh)
        Y[:, rows, :] = apply_M(M, Psi)
    KC = backproject(X, Y)
    ex = exchange_energy(Psi, Y)
    return dict(KC=KC, Ex=float(ex.real), Ex_imag=float(ex.imag))


def exchange_matrix(X: np.ndarray, M: np.ndarray) -> np.ndarray:
    """K^k = conj(X^k) M^k X^{kT}, the AO exchange matrix (used by pins)."""
    return np.stack([X[k].conj() @ M[k] @ X[k].T for k in range(X.shape[0])])


# ----------------------------------------------------------------------------
# sampled outputs for full-size parity checks
# ----------------------------------------------------------------------------

def build_sampled(X, C, V, mesh, ks, route: str = "fft") -> dict:
    """KC^k for the k in ``ks`` only, and the full E_x.

    Step 3 needs D at every k', so steps 1-2 run for all k; steps 3-4 run for
    the sampled k (direct route) or for all k (FFT route)."""
    Psi = collocate(X, C)
    D = density(Psi)
    if route == "fft":
        M = kconv_fft(D, V, mesh)
        Y = apply_M(M, Psi)
        ex = exchange_energy(Psi, Y)
        KC = {k: X[k].conj() @ Y[k] for k in ks}
        return dict(KC=KC, Ex=float(ex.real), Ex_imag=float(ex.imag))
    nk = X.shape[0]
    KC = {}
    for k in ks:
        Mk = np.zeros_like(D[0])
        for kp in range(nk):
            Mk += D[kp] * V[q_index(mesh, k, kp)]
        KC[k] = X[k].conj() @ (Mk @ Psi[k])
    return dict(KC=KC)
