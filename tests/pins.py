"""Checks that pin the FP64 oracle to what the paper and the mathematics fix.

Each check returns the measured discrepancy, so that the pin tests can
assert on it and the mutation tests can show that a planted mistake in the
oracle makes at least one check fail.  None of these retypes the oracle's
own formulas: each compares against an independent object (brute-force grid
exchange, a symmetry, a literal Gamma-point formula, a scalar closed form).
"""
from __future__ import annotations

import functools

import numpy as np

from oracle import setup_oracle as S
from oracle import thc_oracle as O
from paper_2304_05505_gb300 import cells


@functools.lru_cache(maxsize=None)
def full_grid_case(mesh, grid):
    c = cells.make_cell("C0", mesh=mesh, grid=grid)
    pts = cells.grid_points(c, 1)
    Xg = cells.bloch_collocation(c, pts, cells.kmesh_frac(c.mesh))
    C = cells.occupied_coefficients(c)
    V = S.full_grid_kernel(c.lattice, c.grid, c.mesh)
    bf = S.brute_force_exchange(c.lattice, c.grid, c.mesh, Xg, C)
    return c, Xg, C, V, bf


@functools.lru_cache(maxsize=None)
def model_case(mesh=(3, 3, 3), nisdf=40, seed=None):
    """C0 cell with density-sampled points and the model kernel."""
    p = cells.make_problem("C0", seed=seed, mesh=mesh, nisdf=nisdf)
    return p


def check_full_grid(mesh, grid) -> dict:
    """Oracle build with every grid point as a point vs brute-force exchange."""
    c, Xg, C, V, bf = full_grid_case(mesh, grid)
    out = O.build(Xg, C, V, c.mesh, route="direct")
    return dict(
        ex_rel=abs(out["Ex"] - bf["Ex"]) / abs(bf["Ex"]),
        kc_rel=float(np.abs(out["KC"] - bf["KC"]).max() / np.abs(bf["KC"]).max()),
        ex=out["Ex"], ex_bf=bf["Ex"])


def check_hermitian(X, C, V, mesh) -> float:
    out = O.build(X, C, V, mesh, keep=True)
    K = O.exchange_matrix(X, out["M"])
    M = out["M"]
    e1 = np.abs(K - K.conj().transpose(0, 2, 1)).max() / np.abs(K).max()
    e2 = np.abs(M - M.conj().transpose(0, 2, 1)).max() / np.abs(M).max()
    return float(max(e1, e2))


def check_psd(X, C, V, mesh) -> dict:
    out = O.build(X, C, V, mesh, keep=True)
    M = out["M"]
    K = O.exchange_matrix(X, M)
    mineig_M = min(np.linalg.eigvalsh(0.5 * (m + m.conj().T)).min() / np.abs(m).max() for m in M)
    mineig_K = min(np.linalg.eigvalsh(0.5 * (k + k.conj().T)).min() / np.abs(k).max() for k in K)
    return dict(mineig_M=float(mineig_M), mineig_K=float(mineig_K), ex=out["Ex"],
                ex_imag=out["Ex_imag"])


def check_time_reversal(X, C, V, mesh) -> float:
    out = O.build(X, C, V, mesh, keep=True)
    K = O.exchange_matrix(X, out["M"])
    mk = cells.minus_k_index(mesh)
    return float(np.abs(K[mk] - K.conj()).max() / np.abs(K).max())


def check_gauge(X, C, V, mesh, seed=5) -> dict:
    rng = np.random.default_rng(seed)
    nk, nb, n = C.shape
    U = np.zeros((nk, n, n), dtype=np.complex128)
    for k in range(nk):
        q, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
        U[k] = q
    a = O.build(X, C, V, mesh)
    b = O.build(X, np.einsum("kmi,kij->kmj", C, U), V, mesh)
    kc_rot = np.einsum("kmi,kij->kmj", a["KC"], U)
    return dict(kc=float(np.abs(b["KC"] - kc_rot).max() / np.abs(a["KC"]).max()),
                ex=abs(a["Ex"] - b["Ex"]) / abs(a["Ex"]))


def check_energy_trace(X, C, V, mesh) -> float:
    out = O.build(X, C, V, mesh)
    nk = X.shape[0]
    tr = -sum(np.trace(C[k].conj().T @ out["KC"][k]) for k in range(nk)) / nk
    return abs(tr.real - out["Ex"]) / abs(out["Ex"])


def gamma_literal(X, C, V) -> dict:
    """Eq. thcexchange at one k-point, summed literally over lambda, sigma, P, Q
    with the AO density matrix P_ls = sum_i C_li conj(C_si)."""
    x = X[0]
    c = C[0]
    v = V[0]
    nb, npt = x.shape
    P = c @ c.conj().T
    K = np.zeros((nb, nb), dtype=np.complex128)
    for l in range(nb):
        for s in range(nb):
            if P[l, s] == 0:
                continue
            # phi_mu(r_P)^* phi_l(r_P) M_PQ phi_s(r_Q)^* phi_nu(r_Q) P_ls
            a = x.conj() * x[l][None, :]           # (mu, P)
            b = x.conj()[s][:, None] * x.T          # (Q, nu)... phi_s(r_Q)^* phi_nu(r_Q)
            K += P[l, s] * (a @ v @ b)
    return dict(K=K, KC=K @ c, Ex=float(-np.trace(c.conj().T @ K @ c).real))


def check_gamma(X, C, V) -> float:
    out = O.build(X, C, V, (1, 1, 1), keep=True)
    ref = gamma_literal(X, C, V)
    K = O.exchange_matrix(X, out["M"])[0]
    return float(max(np.abs(K - ref["K"]).max() / np.abs(ref["K"]).max(),
                     abs(out["Ex"] - ref["Ex"]) / abs(ref["Ex"])))


def check_scalar(mesh=(3, 1, 2), seed=11) -> float:
    """n = 1, N_P = 1: Psi^k is a number, M^k = sum_k' |Psi^k'|^2 V^(k'-k)."""
    rng = np.random.default_rng(seed)
    nk = int(np.prod(mesh))
    nb = 3
    X = rng.normal(size=(nk, nb, 1)) + 1j * rng.normal(size=(nk, nb, 1))
    C = rng.normal(size=(nk, nb, 1)) + 1j * rng.normal(size=(nk, nb, 1))
    v = rng.uniform(0.1, 1.0, size=nk)      # real positive kernel, one per q
    V = v.reshape(nk, 1, 1).astype(np.complex128)
    out = O.build(X, C, V, mesh)
    co = np.array([[a, b, c] for a in range(mesh[0]) for b in range(mesh[1]) for c in range(mesh[2])])
    psi = np.array([sum(X[k, m, 0] * C[k, m, 0] for m in range(nb)) for k in range(nk)])
    ex = 0.0
    kc = np.zeros((nk, nb), dtype=np.complex128)
    for k in range(nk):
        m = 0.0
        for kp in range(nk):
            d = (co[kp] - co[k]) % np.array(mesh)
            q = (d[0] * mesh[1] + d[1]) * mesh[2] + d[2]
            m += abs(psi[kp]) ** 2 * v[q]
        ex += -abs(psi[k]) ** 2 * m / nk
        kc[k] = X[k, :, 0].conj() * m * psi[k]
    return float(max(abs(out["Ex"] - ex) / abs(ex), np.abs(out["KC"][:, :, 0] - kc).max() / np.abs(kc).max()))


def check_linear_in_V(X, C, V, mesh, seed=3) -> float:
    rng = np.random.default_rng(seed)
    V2 = V * rng.uniform(0.5, 1.5)
    V2 = V2 + 0.3 * V.conj()
    a = O.build(X, C, V, mesh)
    b = O.build(X, C, V2, mesh)
    s = O.build(X, C, V + V2, mesh)
    return float(np.abs(s["KC"] - a["KC"] - b["KC"]).max() / np.abs(s["KC"]).max())


def check_conv_routes(mesh, seed=2) -> float:
    """Direct double sum vs the FFT route on random (non-Hermitian) data."""
    rng = np.random.default_rng(seed)
    nk = int(np.prod(mesh))
    D = rng.normal(size=(nk, 5, 4)) + 1j * rng.normal(size=(nk, 5, 4))
    V = rng.normal(size=(nk, 5, 4)) + 1j * rng.normal(size=(nk, 5, 4))
    a = O.kconv_direct(D, V, mesh)
    b = O.kconv_fft(D, V, mesh)
    return float(np.abs(a - b).max() / np.abs(a).max())


def check_conv_single_term(mesh=(3, 4, 2)) -> float:
    """A delta density at k' = k0 and a delta kernel at q = q0 give M nonzero
    only at k = k0 - q0 (wrapped): the index map of Sec. 2.2, q = k' - k."""
    nk = int(np.prod(mesh))
    worst = 0.0
    for k0 in [0, 5, nk - 1]:
        for q0 in [1, 7, nk - 2]:
            D = np.zeros((nk, 1, 1), dtype=np.complex128)
            V = np.zeros_like(D)
            D[k0] = 2.0
            V[q0] = 3.0
            co = np.array([[a, b, c] for a in range(mesh[0]) for b in range(mesh[1]) for c in range(mesh[2])])
            d = (co[k0] - co[q0]) % np.array(mesh)
            kt = (d[0] * mesh[1] + d[1]) * mesh[2] + d[2]
            expect = np.zeros((nk, 1, 1), dtype=np.complex128)
            expect[kt] = 6.0
            for route in (O.kconv_direct, O.kconv_fft):
                worst = max(worst, float(np.abs(route(D, V, mesh) - expect).max()))
    return worst
