"""Checks that pin the FP64 oracle to what the paper and the mathematics fix.

Each check returns the measured discrepancy, so that the pin tests can
assert on it and the mutation tests can show that a planted mistake in the
oracle makes at least one check fail.  None of these retypes the oracle's
own formulas: each compares against an independent object (brute-force grid
exchange, a symmetry, a literal Gamma-point formula, a scalar closed form).
"""
from __future__ import annotations

import functools
import itertools

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


# ---------------------------------------------------------------------------
# the Coulomb kernel of the setup oracle, pinned to closed forms
# ---------------------------------------------------------------------------

# Energy per cell of a simple cubic lattice of unit point charges in a
# neutralising uniform background is MADELUNG_SC / (2 L) (Nijboer and de
# Wette's lattice constant, 2.8372974794806...).
MADELUNG_SC = -2.8372974794806196


def _grid_cart(lattice, grid):
    axes = [np.arange(g) / g for g in grid]
    f = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    return f @ np.asarray(lattice)


def check_gaussian_self_energy(L: float, alpha: float = 1.0, g: int = 24) -> dict:
    """Coulomb energy of a unit Gaussian charge (alpha/pi)^{3/2} exp(-alpha r^2)
    repeated in a cubic box of side L, with the G = 0 term left out (a
    neutralising background), from the oracle's ISDF kernel of that charge
    taken as a single interpolation vector at Gamma: E = V^0[P, P] / 2.

    Closed form (Ewald split with eta^2 = alpha / 2, whose reciprocal sum is
    exactly this G sum): E = sqrt(alpha / (2 pi)) + MADELUNG_SC / (2 L)
    + pi / (alpha L^3), up to a real-space tail below erfc(sqrt(alpha/2) L)."""
    lattice = L * np.eye(3)
    grid = (g, g, g)
    r = _grid_cart(lattice, grid)
    xi = np.zeros(len(r))
    for n in itertools.product((-1, 0, 1), repeat=3):
        d = r - np.array(n, dtype=float) * L
        xi += (alpha / np.pi) ** 1.5 * np.exp(-alpha * np.einsum("ri,ri->r", d, d))
    V = S.kernel_from_xi(lattice, grid, (1, 1, 1), xi[None, :], np.array([0]))
    e = 0.5 * V[0, 0, 0].real
    exact = np.sqrt(alpha / (2 * np.pi)) + MADELUNG_SC / (2 * L) + np.pi / (alpha * L ** 3)
    return dict(rel=abs(e - exact) / abs(exact), e=e, exact=exact, imag=abs(V[0, 0, 0].imag))


def check_plane_wave_kernel(lattice, grid, mesh, G0) -> float:
    """A plane-wave interpolation vector xi(r) = exp(i G0.r) has the single
    Fourier coefficient Omega at G0, so its kernel at q is the Coulomb energy
    of the Bloch pair density exp(i (G0 + q).r) over the cell:
        V^q[P, P] = (Omega / N_k) 4 pi / |G0 + q|^2     (0 where G0 + q = 0),
    with q the shortest vector of its coset on the reciprocal lattice (the mean
    over ties for a q on the zone boundary).  The shortest vector is found here
    by brute force over the neighbouring cosets.  Returns the largest relative
    deviation over the q of the mesh."""
    lattice = np.asarray(lattice, dtype=float)
    B = 2.0 * np.pi * np.linalg.inv(lattice).T
    vol = abs(np.linalg.det(lattice))
    nk = int(np.prod(mesh))
    r = _grid_cart(lattice, grid)
    G0 = np.asarray(G0, dtype=float)
    xi = np.exp(1j * (r @ (G0 @ B)))
    V = S.kernel_from_xi(lattice, grid, mesh, xi[None, :], np.array([0]))
    worst = 0.0
    for q in range(nk):
        co = np.array(np.unravel_index(q, mesh), dtype=float) / np.array(mesh)
        cands = [co + np.array(n, dtype=float) for n in itertools.product((-1, 0, 1), repeat=3)]
        lens = np.array([np.linalg.norm(c @ B) for c in cands])
        ties = [c for c, ln in zip(cands, lens) if ln <= lens.min() * (1 + 1e-12) + 1e-14]
        vals = []
        for c in ties:
            K = (G0 + c) @ B
            k2 = float(K @ K)
            vals.append(0.0 if k2 < 1e-12 else 4.0 * np.pi / k2)
        expect = vol / nk * float(np.mean(vals))
        scale = max(abs(expect), vol / nk * 4.0 * np.pi / float(np.sum(B * B)))
        worst = max(worst, abs(V[q, 0, 0] - expect) / scale)
    return float(worst)


def check_gset_symmetric(grid) -> float:
    """The G set is the grid's FFT frequencies without the unpaired Nyquist
    plane of an even size: every frequency whose negative is also one."""
    got = {tuple(int(x) for x in t) for t in S.symmetric_gset(grid)}
    axes = []
    for g in grid:
        f = set(int(x) for x in np.rint(np.fft.fftfreq(g) * g))
        axes.append(sorted(x for x in f if -x in f))
    want = set(itertools.product(*axes))
    return float(len(got ^ want))
