"""Seeded synthetic inputs for the THC-oo-K exchange build.

This module only *makes inputs*.  It builds a periodic cell, a Bloch-summed
Gaussian basis, occupied coefficients from a model Hamiltonian, interpolation
points and a model ISDF Coulomb kernel, all from a seed.  It holds none of the
build's arithmetic: no orbital collocation at the points, no point-space
density, no k-convolution, no back-projection and no energy.  The CUDA
library, the tests, the bench and the CPU oracle all draw their inputs from
here, and this module imports neither of the two implementations.

Objects and where the paper defines them (arXiv 2304.05505):

* Bloch basis, Sec. 1 (the crystalline GTO equation):
  ``X^k[mu, p] = sum_R exp(i k.R) phi_mu(r_p - R)``.  It is normalised per cell
  (no 1/sqrt(N_k)) and carries the Bloch phase, so ``X^{k+G} = X^k`` and
  ``X^{-k} = conj(X^k)``.
* k-mesh: Gamma-centred, ``k_n = sum_a (n_a / N_a) b_a``, k index
  ``(n1 * N2 + n2) * N3 + n3``.
* Occupied coefficients ``C^k``: the lowest ``n_occ`` solutions of
  ``H^k C = S^k C e`` for a model Hamiltonian (grid kinetic energy plus
  Gaussian wells) by grid quadrature, ``C^H S C = 1``.  They stand in for the
  SCF orbitals of Algorithm 2 and satisfy ``C^{-k} = conj(C^k)``.
* Model ISDF kernel ``V^q[P, Q]``: the GPW form of ``M^q`` (Sec. 2.2, the
  M^q equation) for interpolation vectors that are Gaussian-smeared deltas of
  weight ``Omega / N_P`` at the points, with the Bloch phase of the pair folded
  in.  The G sum runs over ``K = G + q`` in a sphere, with ``K = 0`` left out.
  The result is Hermitian positive semidefinite per q, and ``V^{-q} =
  conj(V^q)`` exactly.

The configurations C0..C3 follow the synthetic workload recipe: a toy cubic
cell, and orthorhombic cells shaped like the benzene crystal of Sec. 4.3.
"""
from __future__ import annotations

import dataclasses
import math
import os

import numpy as np

# ----------------------------------------------------------------------------
# cell and basis
# ----------------------------------------------------------------------------

# Image cutoff for Bloch sums (bohr); terms with exp(-alpha r^2) < exp(-36.8)
# (about 1e-16 of the peak) are also dropped, which does not change a double.
IMAGE_CUTOFF = 20.0
GAUSS_DROP = 36.8

# Optional torch device for the large complex matrix products of input
# generation (the quadrature matrices S, T, V of the model Hamiltonian and the
# Gram products of the model kernel), in FP64 as on the CPU.  None: numpy.
# Only these products move; the inputs stay numpy arrays that the library and
# the oracle both consume.
_ACCEL = None


def set_accelerator(device) -> None:
    """Route the generator's large matrix products through torch on `device`
    (e.g. "cuda"), or back to numpy with None.  Used to make the largest
    synthetic cell in reasonable time; results agree with numpy to rounding."""
    global _ACCEL
    _ACCEL = device


def _mm_h(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """a @ b^H (complex, FP64)."""
    if _ACCEL is None:
        return a @ b.conj().T
    import torch
    ta = torch.from_numpy(np.ascontiguousarray(a)).to(_ACCEL)
    tb = torch.from_numpy(np.ascontiguousarray(b)).to(_ACCEL)
    return (ta @ tb.conj().T).cpu().numpy()


@dataclasses.dataclass
class Cell:
    name: str
    lattice: np.ndarray          # (3, 3) rows a1, a2, a3, bohr
    centres: np.ndarray          # (Na, 3) cartesian, bohr
    kinds: list                  # per centre: 'C', 'H' or 'S'
    grid: tuple                  # real-space grid (g1, g2, g3)
    mesh: tuple                  # k mesh (n1, n2, n3)
    nocc: int
    nisdf: int
    quad_stride: int             # quadrature grid = every stride-th grid point
    seed: int
    # expanded basis, one entry per function
    fn_centre: np.ndarray = None  # (N,) int
    fn_l: np.ndarray = None       # (N,) int
    fn_m: np.ndarray = None       # (N,) int
    fn_alpha: np.ndarray = None   # (N,) float

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))

    @property
    def recip(self) -> np.ndarray:
        """Rows b1, b2, b3 with a_i . b_j = 2 pi delta_ij."""
        return 2.0 * np.pi * np.linalg.inv(self.lattice).T

    @property
    def nbas(self) -> int:
        return int(self.fn_alpha.shape[0])

    @property
    def nk(self) -> int:
        return int(np.prod(self.mesh))

    @property
    def ngrid(self) -> int:
        return int(np.prod(self.grid))


# Synthetic shell sets (exponents in bohr^-2).  Each function is one
# normalised primitive; "S" is the toy centre of the cubic cell.
SHELLS = {
    "S": [(0, 0.3), (0, 0.8), (0, 2.0), (0, 5.0)],
    "C": [(0, 3.5), (0, 0.45), (1, 1.6), (1, 0.35), (2, 0.6)],
    "H": [(0, 1.2), (0, 0.25), (1, 0.8)],
}
WELL_Z = {"S": 2.0, "C": 4.0, "H": 1.0}
WELL_BETA = 0.5
NFUNC_L = {0: 1, 1: 3, 2: 5}

CC_BOND = 2.64   # bohr
CH_BOND = 2.06   # bohr


def _expand_basis(cell: Cell) -> None:
    cen, ls, ms, al = [], [], [], []
    for a, kind in enumerate(cell.kinds):
        for (l, alpha) in SHELLS[kind]:
            for m in range(NFUNC_L[l]):
                cen.append(a)
                ls.append(l)
                ms.append(m)
                al.append(alpha)
    cell.fn_centre = np.array(cen, dtype=np.int64)
    cell.fn_l = np.array(ls, dtype=np.int64)
    cell.fn_m = np.array(ms, dtype=np.int64)
    cell.fn_alpha = np.array(al, dtype=np.float64)


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _benzene(rng, centre) -> tuple:
    """One ring: 6 C at radius CC_BOND, 6 H at CC_BOND + CH_BOND."""
    rot = _random_rotation(rng)
    pos, kinds = [], []
    for j in range(6):
        t = 2 * np.pi * j / 6
        u = np.array([np.cos(t), np.sin(t), 0.0])
        pos.append(centre + rot @ (CC_BOND * u))
        kinds.append("C")
    for j in range(6):
        t = 2 * np.pi * j / 6
        u = np.array([np.cos(t), np.sin(t), 0.0])
        pos.append(centre + rot @ ((CC_BOND + CH_BOND) * u))
        kinds.append("H")
    return pos, kinds


BENZENE_CELL = np.diag([13.9, 17.8, 12.9])
BENZENE_SITES = [(0, 0, 0), (0.5, 0.5, 0), (0, 0.5, 0.5), (0.5, 0, 0.5)]

CONFIGS = {
    # name: (kind, mesh, grid, nocc, nisdf, quad_stride)
    "C0": ("toy", (2, 2, 2), (16, 16, 16), 4, 48, 1),
    "C1": ("benzene", (3, 3, 3), (40, 40, 40), 60, 600, 2),
    "C2": ("benzene", (4, 4, 4), (40, 40, 40), 60, 1200, 2),
    "C3": ("benzene2", (6, 6, 6), (80, 40, 40), 120, 2400, 2),
}


def default_seed(name: str, index: int = 0) -> int:
    c = int(name[1:]) if name[1:].isdigit() else 9
    return 20230411 + 1000 * c + index


def make_cell(name: str = "C0", seed: int | None = None, mesh=None, grid=None,
              nocc=None, nisdf=None) -> Cell:
    """Build one seeded synthetic cell.  ``mesh``/``grid``/``nocc``/``nisdf``
    override the configuration (used for pin variants such as a 3x3x3 mesh)."""
    kind, mesh0, grid0, nocc0, nisdf0, stride = CONFIGS[name]
    seed = default_seed(name) if seed is None else seed
    rng = np.random.default_rng(seed)
    if kind == "toy":
        lattice = 6.0 * np.eye(3)
        cen = []
        while len(cen) < 4:
            p = rng.uniform(0, 1, size=3) @ lattice
            ok = True
            for c in cen:
                d = p - c
                f = d @ np.linalg.inv(lattice)
                f -= np.round(f)
                if np.linalg.norm(f @ lattice) < 1.5:
                    ok = False
            if ok:
                cen.append(p)
        kinds = ["S"] * 4
    else:
        ncell = 2 if kind == "benzene2" else 1
        lattice = BENZENE_CELL.copy()
        lattice[0] *= ncell
        cen, kinds = [], []
        for s in range(ncell):
            for site in BENZENE_SITES:
                c = (np.array(site) + np.array([s, 0, 0])) @ BENZENE_CELL
                pos, kk = _benzene(rng, c)
                cen += pos
                kinds += kk
        cen = np.array(cen) + rng.uniform(-0.1, 0.1, size=(len(cen), 3))
        # wrap into the cell
        f = np.array(cen) @ np.linalg.inv(lattice)
        cen = list((f - np.floor(f)) @ lattice)
    cell = Cell(name=name, lattice=lattice, centres=np.array(cen), kinds=kinds,
                grid=tuple(grid or grid0), mesh=tuple(mesh or mesh0),
                nocc=int(nocc or nocc0), nisdf=int(nisdf or nisdf0),
                quad_stride=stride, seed=seed)
    _expand_basis(cell)
    return cell


# ----------------------------------------------------------------------------
# k mesh and grids
# ----------------------------------------------------------------------------

def kmesh_frac(mesh) -> np.ndarray:
    """(N_k, 3) fractional k points, index (n1*N2 + n2)*N3 + n3."""
    n1, n2, n3 = mesh
    a, b, c = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    return np.stack([a.ravel() / n1, b.ravel() / n2, c.ravel() / n3], axis=1)


def kmesh_cart(cell: Cell) -> np.ndarray:
    return kmesh_frac(cell.mesh) @ cell.recip


def minus_k_index(mesh) -> np.ndarray:
    """Index of -k for every mesh k."""
    n1, n2, n3 = mesh
    a, b, c = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    return ((((-a) % n1) * n2 + ((-b) % n2)) * n3 + ((-c) % n3)).ravel()


def grid_points(cell: Cell, stride: int = 1) -> np.ndarray:
    """Cartesian grid points, C order over (g1, g2, g3), optionally strided."""
    g = cell.grid
    axes = [np.arange(0, g[i], stride) / g[i] for i in range(3)]
    f = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    return f @ cell.lattice


def grid_gvectors(shape, recip) -> np.ndarray:
    """G vectors in numpy FFT order for a grid of the given shape."""
    m = [np.fft.fftfreq(n, 1.0 / n) for n in shape]
    mi = np.stack(np.meshgrid(*m, indexing="ij"), axis=-1).reshape(-1, 3)
    return mi @ recip


# ----------------------------------------------------------------------------
# Bloch-summed Gaussian collocation
# ----------------------------------------------------------------------------

def _angular(l, m, alpha, d, xp=np):
    """Normalised real solid-harmonic prefactor of each primitive.

    d: (..., N, 3) displacement r - A.  Returns (..., N).  ``xp`` is numpy or
    torch (the accelerated collocation passes tensors)."""
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    n0 = (2.0 * alpha / np.pi) ** 0.75
    out = xp.ones_like(x)
    out = xp.where(l == 1, xp.where(m == 0, x, xp.where(m == 1, y, z)) * xp.sqrt(4 * alpha), out)
    d2 = xp.where(m == 0, x * y,
         xp.where(m == 1, y * z,
         xp.where(m == 2, (2 * z * z - x * x - y * y) / (2 * math.sqrt(3.0)),
         xp.where(m == 3, x * z, (x * x - y * y) / 2.0))))
    out = xp.where(l == 2, d2 * 4 * alpha, out)
    return out * n0


def _image_range(cell: Cell, rcut: float) -> list:
    vol = cell.volume
    a = cell.lattice
    h = [vol / np.linalg.norm(np.cross(a[(i + 1) % 3], a[(i + 2) % 3])) for i in range(3)]
    nmax = [int(math.floor(1 + rcut / h[i])) for i in range(3)]
    return [(i, j, k) for i in range(-nmax[0], nmax[0] + 1)
            for j in range(-nmax[1], nmax[1] + 1)
            for k in range(-nmax[2], nmax[2] + 1)]


def collocation_terms(cell: Cell, points: np.ndarray, chunk: int = 4096) -> list:
    """k-independent Gaussian values of every kept image term.

    Returns a list of (R, flat, val): lattice vector R (cartesian), flat index
    mu * Np + p, and phi_mu(r_p - R).  Images with |r - A - R| <= 20 bohr are
    kept unless their Gaussian factor is below exp(-36.8)."""
    npnt = points.shape[0]
    A = cell.centres[cell.fn_centre]                      # (N, 3)
    alpha = cell.fn_alpha
    rc2 = np.minimum(IMAGE_CUTOFF ** 2, GAUSS_DROP / alpha)  # (N,)
    images = _image_range(cell, float(np.sqrt(rc2.max())))
    terms = []
    for n in images:
        R = np.array(n, dtype=np.float64) @ cell.lattice
        flats, vals = [], []
        for p0 in range(0, npnt, chunk):
            pts = points[p0:p0 + chunk]
            d = pts[None, :, :] - (A + R)[:, None, :]      # (N, np, 3)
            r2 = (d * d).sum(-1)
            mask = r2 <= rc2[:, None]
            if not mask.any():
                continue
            mu, pp = np.nonzero(mask)
            val = _angular(cell.fn_l[mu], cell.fn_m[mu], alpha[mu], d[mu, pp]) \
                * np.exp(-alpha[mu] * r2[mu, pp])
            flats.append(mu * npnt + pp + p0)
            vals.append(val)
        if flats:
            terms.append((R, np.concatenate(flats), np.concatenate(vals)))
    return terms


def _bloch_collocation_accel(cell: Cell, points: np.ndarray, kfrac: np.ndarray, chunk: int = 1 << 16):
    """bloch_collocation on the accelerator, as a torch tensor (Nk, N, Np).

    The same image set, drop rule and image order as collocation_terms /
    bloch_collocation, evaluated densely over (function, point) per image
    with the dropped terms multiplied by zero, so each element sums the same
    terms in the same order (agreement to the rounding of exp)."""
    import torch
    dev = _ACCEL
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    A = t(cell.centres[cell.fn_centre])
    alpha = t(cell.fn_alpha)
    l, m = t(cell.fn_l), t(cell.fn_m)
    rc2 = np.minimum(IMAGE_CUTOFF ** 2, GAUSS_DROP / cell.fn_alpha)
    images = _image_range(cell, float(np.sqrt(rc2.max())))
    rc2 = t(rc2)
    kc = np.atleast_2d(kfrac) @ cell.recip
    pts = t(points)
    npnt = points.shape[0]
    X = torch.zeros((kc.shape[0], cell.nbas, npnt), dtype=torch.complex128, device=dev)
    for n in images:
        R = np.array(n, dtype=np.float64) @ cell.lattice
        ph = t(np.exp(1j * (kc @ R)))
        AR = A + t(R)
        for p0 in range(0, npnt, chunk):
            d = pts[None, p0:p0 + chunk, :] - AR[:, None, :]            # (N, np, 3)
            r2 = (d * d).sum(-1)
            mask = r2 <= rc2[:, None]
            if not bool(mask.any()):
                continue
            val = _angular(l[:, None], m[:, None], alpha[:, None], d, torch) \
                * torch.exp(-alpha[:, None] * r2) * mask
            X[:, :, p0:p0 + chunk] += ph[:, None, None] * val[None]
    return X


def bloch_collocation(cell: Cell, points: np.ndarray, kfrac: np.ndarray,
                      terms: list | None = None) -> np.ndarray:
    """X^k[mu, p] = sum_R exp(i k.R) phi_mu(r_p - R), shape (Nk, N, Np) c128."""
    if terms is None and _ACCEL is not None:
        return _bloch_collocation_accel(cell, points, kfrac).cpu().numpy()
    if terms is None:
        terms = collocation_terms(cell, points)
    kc = np.atleast_2d(kfrac) @ cell.recip
    nk, nb, npnt = kc.shape[0], cell.nbas, points.shape[0]
    X = np.zeros((nk, nb * npnt), dtype=np.complex128)
    for R, flat, val in terms:
        ph = np.exp(1j * (kc @ R))
        if nk == 1:
            X[0, flat] += ph[0] * val
        else:
            X[:, flat] += ph[:, None] * val[None, :]
    return X.reshape(nk, nb, npnt)


# ----------------------------------------------------------------------------
# model Hamiltonian and occupied coefficients
# ----------------------------------------------------------------------------

def well_potential(cell: Cell, points: np.ndarray) -> np.ndarray:
    """Sum over centres and images of -Z_A exp(-beta |r - A - R|^2)."""
    rc = math.sqrt(GAUSS_DROP / WELL_BETA)
    w = np.zeros(points.shape[0])
    for n in _image_range(cell, rc):
        R = np.array(n, dtype=np.float64) @ cell.lattice
        for A, kind in zip(cell.centres, cell.kinds):
            d = points - (A + R)
            w -= WELL_Z[kind] * np.exp(-WELL_BETA * np.einsum("pi,pi->p", d, d))
    return w


def occupied_coefficients(cell: Cell) -> np.ndarray:
    """C^k, shape (Nk, N, n_occ) c128, lowest eigenvectors of H^k C = S^k C e.

    Quadrature on the grid sub-sampled by ``quad_stride``.  For each +-k pair
    only one k is solved and ``C^{-k} = conj(C^k)``; at k = -k the problem is
    taken real."""
    return orbital_coefficients(cell, 0)[0]


def orbital_coefficients(cell: Cell, nvir: int) -> tuple:
    """(C_occ, C_vir): the n_occ lowest eigenvectors of H^k C = S^k C e, as
    occupied_coefficients gives them, and the next ``nvir`` (virtual
    orbitals, for orbital rotations), shapes (Nk, N, n_occ) and (Nk, N, nvir)."""
    import scipy.linalg as sla

    s = cell.quad_stride
    qshape = tuple(g // s for g in cell.grid)
    pts = grid_points(cell, s)
    ng = pts.shape[0]
    vol = cell.volume
    kf = kmesh_frac(cell.mesh)
    kc = kf @ cell.recip
    mk = minus_k_index(cell.mesh)
    G = grid_gvectors(qshape, cell.recip)
    wpot = well_potential(cell, pts)
    nk = kf.shape[0]
    nall = cell.nocc + int(nvir)
    if nall > cell.nbas:
        raise ValueError("more orbitals than basis functions")
    C = np.zeros((nk, cell.nbas, nall), dtype=np.complex128)
    done = np.zeros(nk, dtype=bool)
    terms = collocation_terms(cell, pts) if _ACCEL is None else None
    for k in range(nk):
        if done[k]:
            continue
        phi = bloch_collocation(cell, pts, kf[k:k + 1], terms)[0]  # (N, ng)
        S = (vol / ng) * _mm_h(phi, phi).conj()
        u = phi * np.exp(-1j * (pts @ kc[k]))[None, :]
        uh = np.fft.fftn(u.reshape((-1,) + qshape), axes=(1, 2, 3)).reshape(cell.nbas, -1) / ng
        kin = 0.5 * np.einsum("gi,gi->g", G + kc[k], G + kc[k])
        T = vol * _mm_h(uh * kin[None, :], uh).conj()
        Vw = (vol / ng) * _mm_h(phi * wpot[None, :], phi).conj()
        H = T + Vw
        H = 0.5 * (H + H.conj().T)
        S = 0.5 * (S + S.conj().T)
        if mk[k] == k:
            e, v = sla.eigh(H.real, S.real, subset_by_index=[0, nall - 1])
            C[k] = v
        else:
            e, v = sla.eigh(H, S, subset_by_index=[0, nall - 1])
            C[k] = v
            C[mk[k]] = v.conj()
            done[mk[k]] = True
        done[k] = True
    return np.ascontiguousarray(C[:, :, :cell.nocc]), np.ascontiguousarray(C[:, :, cell.nocc:])


def grid_orbitals(cell: Cell, C: np.ndarray, stride: int = 1, as_tensor: bool = False):
    """The input of the setup calls (interpolation-point selection and the
    ISDF kernel fit): the occupied orbitals' cell-periodic parts on the grid
    sub-sampled by ``stride``, U[f][r] = u^k_i(r) = exp(-i k.r) sum_mu
    X^k_mu(r) C^k_mu,i for f = (k, i), shape (N_k n_occ, N_g) c128.

    These are grid values for the setup stage; the build itself collocates
    the orbitals at the interpolation points (its step 1), which this module
    never does.  With an accelerator set and ``as_tensor``, U is returned as a
    torch tensor on that device."""
    pts = grid_points(cell, stride)
    kf = kmesh_frac(cell.mesh)
    kc = kf @ cell.recip
    if _ACCEL is not None:
        return _grid_orbitals_accel(cell, C, pts, kf, kc, as_tensor)
    terms = collocation_terms(cell, pts)
    nk, n = C.shape[0], C.shape[2]
    U = np.zeros((nk, n, pts.shape[0]), dtype=np.complex128)
    for k in range(nk):
        Xk = bloch_collocation(cell, pts, kf[k:k + 1], terms)[0]          # (N, ng)
        # C^T X: the conjugate of (conj(C)^T ...)^H products, as a @ b^H
        psi = _mm_h(np.ascontiguousarray(C[k].T), np.ascontiguousarray(Xk.T.conj()))
        U[k] = psi * np.exp(-1j * (pts @ kc[k]))[None, :]
    return U.reshape(nk * n, -1)


def _grid_orbitals_accel(cell, C, pts, kf, kc, as_tensor, kblock: int = 8):
    import torch
    nk, n = C.shape[0], C.shape[2]
    U = torch.empty((nk, n, pts.shape[0]), dtype=torch.complex128, device=_ACCEL)
    pt = torch.from_numpy(pts).to(_ACCEL)
    Ct = torch.from_numpy(np.ascontiguousarray(C)).to(_ACCEL)
    for k0 in range(0, nk, kblock):
        k1 = min(nk, k0 + kblock)
        Xk = _bloch_collocation_accel(cell, pts, kf[k0:k1])                  # (kb, N, ng)
        ph = torch.exp(-1j * (pt @ torch.from_numpy(kc[k0:k1]).to(_ACCEL).T)).T   # (kb, ng)
        U[k0:k1] = torch.matmul(Ct[k0:k1].transpose(1, 2), Xk) * ph[:, None, :]
        del Xk
    U = U.reshape(nk * n, -1)
    return U if as_tensor else U.cpu().numpy()


# ----------------------------------------------------------------------------
# interpolation points and the model kernel
# ----------------------------------------------------------------------------

def promolecular_density(cell: Cell, points: np.ndarray, beta: float = 1.0) -> np.ndarray:
    rc = math.sqrt(GAUSS_DROP / beta)
    rho = np.zeros(points.shape[0])
    for n in _image_range(cell, rc):
        R = np.array(n, dtype=np.float64) @ cell.lattice
        for A, kind in zip(cell.centres, cell.kinds):
            d = points - (A + R)
            rho += WELL_Z[kind] * np.exp(-beta * np.einsum("pi,pi->p", d, d))
    return rho


def _inclusion_probabilities(p: np.ndarray, n: int) -> np.ndarray:
    """pi_i = min(1, c p_i) with sum_i pi_i = n (c by bisection)."""
    lo, hi = 0.0, float(n) / p.min()
    for _ in range(200):
        c = 0.5 * (lo + hi)
        s = np.minimum(1.0, c * p).sum()
        if s < n:
            lo = c
        else:
            hi = c
    return np.minimum(1.0, hi * p)


def sample_points(cell: Cell, npoints: int | None = None, seed: int | None = None):
    """Interpolation points drawn from the quadrature grid with inclusion
    probabilities proportional to a promolecular density plus a floor.

    A stand-in for the paper's point selection (CVT k-means or QRCP) on cells
    too large for a CPU pivoted Cholesky.  Returns (full-grid indices sorted
    ascending, quadrature weight of each point).  The weight is the grid
    volume element divided by the point's inclusion probability (the
    Horvitz-Thompson weight), so the weights sum to about Omega."""
    npoints = cell.nisdf if npoints is None else npoints
    rng = np.random.default_rng((cell.seed if seed is None else seed) + 17)
    s = cell.quad_stride
    pts = grid_points(cell, s)
    ngq = pts.shape[0]
    rho = promolecular_density(cell, pts)
    p = rho + 0.05 * rho.mean()
    p /= p.sum()
    pi = _inclusion_probabilities(p, npoints)
    # systematic sampling in a random order gives exactly npoints with
    # inclusion probabilities pi
    order = rng.permutation(ngq)
    cum = np.cumsum(pi[order])
    u = rng.uniform(0.0, 1.0)
    hits = np.searchsorted(cum, u + np.arange(npoints), side="right")
    sel = order[np.clip(hits, 0, ngq - 1)]
    sel = np.unique(sel)
    if sel.size < npoints:                      # rounding at the ends
        rest = np.setdiff1d(np.argsort(-pi), sel, assume_unique=False)[: npoints - sel.size]
        sel = np.union1d(sel, rest)
    sel = sel[:npoints]
    q = tuple(g // s for g in cell.grid)
    i, j, k = np.unravel_index(sel, q)
    full = np.ravel_multi_index((i * s, j * s, k * s), cell.grid)
    order = np.argsort(full)
    weight = (cell.volume / ngq) / pi[sel]
    return full[order], weight[order]


def points_from_indices(cell: Cell, idx: np.ndarray) -> np.ndarray:
    return grid_points(cell, 1)[idx]


MODEL_SMEAR = 0.5        # Gaussian exponent a of the smeared interpolation vectors
MODEL_LOG_CUT = 13.8     # keep K with exp(-K^2/(2a)) >= exp(-13.8) ~ 1e-6


def _coset_vectors(cell: Cell, qfrac: np.ndarray, kmax: float) -> np.ndarray:
    """All K = q + G with |K| <= kmax (cartesian), G on the reciprocal lattice."""
    B = cell.recip
    hb = [2 * np.pi / np.linalg.norm(cell.lattice[i]) for i in range(3)]
    # plane spacing of the reciprocal lattice along b_i is 2 pi / |a_i|
    nmax = [int(math.ceil(kmax / hb[i])) + 1 for i in range(3)]
    r = [np.arange(-nmax[i], nmax[i] + 1) for i in range(3)]
    m = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3).astype(np.float64)
    K = (m + qfrac[None, :]) @ B
    K2 = np.einsum("gi,gi->g", K, K)
    keep = (K2 <= kmax * kmax) & (K2 > 1e-12)
    return K[keep]


def model_kernel(cell: Cell, points: np.ndarray, weights: np.ndarray | None = None,
                 smear: float = MODEL_SMEAR) -> np.ndarray:
    """V^q[P, Q] = w_P w_Q / (N_k Omega) sum_K 4 pi/|K|^2 exp(-|K|^2/(2a)) exp(-i K.(r_P - r_Q)).

    The interpolation vector of point P is w_P times a unit Gaussian of
    exponent a centred at r_P (w_P = Omega / N_P when no weights are given).
    K runs over the coset q + G inside a sphere, K = 0 excluded.  Shape
    (Nk, N_P, N_P) c128, q on the same mesh index as k."""
    kf = kmesh_frac(cell.mesh)
    mk = minus_k_index(cell.mesh)
    nk, npnt = kf.shape[0], points.shape[0]
    kmax = math.sqrt(2 * smear * MODEL_LOG_CUT)
    if weights is None:
        weights = np.full(npnt, cell.volume / npnt)
    pref = 1.0 / (nk * cell.volume)
    V = np.zeros((nk, npnt, npnt), dtype=np.complex128)
    done = np.zeros(nk, dtype=bool)
    for q in range(nk):
        if done[q]:
            continue
        K = _coset_vectors(cell, kf[q], kmax)
        K2 = np.einsum("gi,gi->g", K, K)
        w = pref * 4 * np.pi / K2 * np.exp(-K2 / (2 * smear))
        A = np.exp(-1j * (points @ K.T)) * np.sqrt(w)[None, :] * weights[:, None]
        Vq = _mm_h(A, A)
        Vq = 0.5 * (Vq + Vq.conj().T)
        if mk[q] == q:
            V[q] = Vq.real
        else:
            V[q] = Vq
            V[mk[q]] = Vq.conj()
            done[mk[q]] = True
        done[q] = True
    return V


# ----------------------------------------------------------------------------
# one-call problem factory
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    cell: Cell
    points: np.ndarray        # (N_P, 3) cartesian
    point_index: np.ndarray   # (N_P,) full-grid indices
    weights: np.ndarray       # (N_P,) quadrature weight of each point
    X: np.ndarray             # (Nk, N, N_P) c128
    C: np.ndarray             # (Nk, N, n) c128
    V: np.ndarray             # (Nk, N_P, N_P) c128

    @property
    def dims(self) -> dict:
        c = self.cell
        return dict(n1=c.mesh[0], n2=c.mesh[1], n3=c.mesh[2], nbas=c.nbas,
                    nocc=c.nocc, nisdf=self.points.shape[0])


_MEMO: dict = {}


def make_problem(name: str = "C0", seed: int | None = None, cache: bool = True, **over) -> Problem:
    """Cell, density-sampled points, X at the points, C^k and the model V^q."""
    key = (name, seed, tuple(sorted(over.items())))
    if cache and key in _MEMO:
        return _MEMO[key]
    cdir = os.environ.get("THC_CACHE_DIR")
    path = None
    if cdir:
        tag = "_".join([name, str(seed)] + [f"{k}{v}" for k, v in sorted(over.items())])
        tag = tag.replace(" ", "").replace("(", "").replace(")", "").replace(",", "x")
        path = os.path.join(cdir, f"problem_v2_{tag}.npz")
    cell = make_cell(name, seed, **over)
    if path and os.path.exists(path):
        z = np.load(path)
        prob = Problem(cell, z["points"], z["point_index"], z["weights"], z["X"], z["C"], z["V"])
    else:
        idx, wts = sample_points(cell)
        pts = points_from_indices(cell, idx)
        X = bloch_collocation(cell, pts, kmesh_frac(cell.mesh))
        C = occupied_coefficients(cell)
        V = model_kernel(cell, pts, wts)
        prob = Problem(cell, pts, idx, wts, X, C, V)
        if path:
            os.makedirs(cdir, exist_ok=True)
            np.savez(path, points=pts, point_index=idx, weights=wts, X=X, C=C, V=V)
    if cache:
        _MEMO[key] = prob
    return prob


def random_problem(nk_mesh=(2, 2, 2), nbas=8, nocc=3, nisdf=20, seed=1) -> dict:
    """Unstructured random inputs with the symmetries of the real ones.

    X, C random complex with X^{-k} = conj(X^k), C^{-k} = conj(C^k); V^q
    Hermitian PSD per q with V^{-q} = conj(V^q).  Used for edge-case shapes."""
    rng = np.random.default_rng(seed)
    nk = int(np.prod(nk_mesh))
    mk = minus_k_index(nk_mesh)

    def cplx(*shape):
        return rng.normal(size=shape) + 1j * rng.normal(size=shape)

    X = cplx(nk, nbas, nisdf) / np.sqrt(nbas)
    C = cplx(nk, nbas, nocc) / np.sqrt(nbas)
    V = np.zeros((nk, nisdf, nisdf), dtype=np.complex128)
    for q in range(nk):
        if mk[q] < q:
            continue
        A = cplx(nisdf, nisdf + 3) / (nisdf + 3)
        Vq = A @ A.conj().T
        Vq = 0.5 * (Vq + Vq.conj().T)
        if mk[q] == q:
            V[q] = Vq.real
        else:
            V[q] = Vq
            V[mk[q]] = Vq.conj()
    for k in range(nk):
        if mk[k] == k:
            X[k] = X[k].real
            C[k] = C[k].real
        elif mk[k] < k:
            X[k] = X[mk[k]].conj()
            C[k] = C[mk[k]].conj()
    return dict(mesh=tuple(nk_mesh), X=X, C=C, V=V)
