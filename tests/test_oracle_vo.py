"""Pins of the FP64 oracle of the THC-oo-K orbital gradient (the vo block).

No GPU.  The gradient is the derivative of the THC-oo-K exchange energy with
respect to an occupied-virtual rotation C^k -> C^k + Cv^k theta^k, with the
interpolation points fixed and the fit and the kernel redone (Sec. 2.3: the
interpolation vectors of Eq. orbprodoo depend on the occupied orbitals).  It
is pinned against finite differences of the numpy build, against the closed
form of its explicit term, against the brute-force grid exchange where the
kernel does not depend on the orbitals, and against the invariance of the
energy under rotations among the occupied orbitals."""
import numpy as np
import pytest

from oracle import setup_oracle as S
from oracle import vo_oracle as VO
from paper_2304_05505_gb300 import cells

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def prob():
    """C0 cell, 3x1x2 k-mesh (k = -k and +-k pairs), an 8^3 grid, 4 occupied
    and 4 virtual orbitals per k, 24 points by pivoted Cholesky (a partial fit,
    so the kernel depends on the orbitals)."""
    c = cells.make_cell("C0", mesh=(3, 1, 2), grid=(8, 8, 8))
    kf = cells.kmesh_frac(c.mesh)
    Xg = cells.bloch_collocation(c, cells.grid_points(c, 1), kf)
    C, Cv = cells.orbital_coefficients(c, 4)
    p = dict(lattice=c.lattice, grid=c.grid, mesh=c.mesh, kfrac=kf, Xg=Xg, points=None)
    P = S.pivoted_cholesky(VO.grid_orbitals(p, C), 24)["points"]
    p["points"] = P
    p["C"], p["Cv"] = C, Cv
    p["V"] = S.fit_kernel(c.lattice, c.grid, c.mesh, VO.grid_orbitals(p, C), P)
    return p


def _directional_fd(f, h=1e-4):
    """Five-point central difference of f at 0 (error O(h^4))."""
    return (8.0 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12.0 * h)


def test_torch_energy_is_the_build(prob):
    """The torch restatement gives the numpy build's E_x, refitted and fixed."""
    C = prob["C"]
    E = VO.energy(prob, C)
    Et = VO._energy_torch(prob, torch.from_numpy(C), None, torch).item()
    Ef = VO._energy_torch(prob, torch.from_numpy(C), prob["V"], torch).item()
    assert abs(Et - E) <= 1e-12 * abs(E)
    assert abs(Ef - E) <= 1e-12 * abs(E)


def test_fixed_kernel_gradient_is_the_closed_form(prob):
    """With the kernel held fixed, autograd of the restatement equals
    -(4/N_k) Cv^H (K C), K C the build's output."""
    C, Cv, V = prob["C"], prob["Cv"], prob["V"]
    g = VO.vo_gradient(prob, C, Cv, V_fixed=V)
    ge = VO.explicit_gradient(prob, C, Cv, V)
    assert np.abs(g - ge).max() <= 1e-12 * np.abs(ge).max()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_refit_gradient_matches_finite_differences(prob, seed):
    """Re sum conj(g) theta equals the derivative of E_x (kernel refitted at
    every step) along theta, from five-point differences of the numpy build."""
    C, Cv = prob["C"], prob["Cv"]
    g = VO.vo_gradient(prob, C, Cv)
    rng = np.random.default_rng(seed)
    th = rng.normal(size=g.shape) + 1j * rng.normal(size=g.shape)
    pred = float(np.real(np.sum(g.conj() * th)))
    fd = _directional_fd(lambda s: VO.energy(prob, C + s * (Cv @ th)))
    assert abs(fd - pred) <= 1e-8 * np.abs(g).sum() * np.abs(th).max()


def test_refit_term_is_not_small(prob):
    """The kernel's dependence on the orbitals changes the gradient by more
    than its size here, so the finite-difference pin fails if it is dropped."""
    C, Cv, V = prob["C"], prob["Cv"], prob["V"]
    g = VO.vo_gradient(prob, C, Cv)
    ge = VO.explicit_gradient(prob, C, Cv, V)
    assert np.abs(g - ge).max() >= 0.5 * np.abs(g).max()


def test_occupied_rotations_leave_the_energy_invariant(prob):
    """D^k and the pair Gram matrix depend on the occupied orbitals only
    through sum_i u^k_i conj(u^k_i), so E_x is unchanged by a unitary rotation
    among them: the gradient with Cv = C (theta anti-Hermitian directions) is
    Hermitian for every k."""
    C = prob["C"]
    g = VO.vo_gradient(prob, C, C)
    gh = np.conj(np.transpose(g, (0, 2, 1)))
    assert np.abs(g - gh).max() <= 1e-11 * np.abs(g).max()
    assert np.abs(g).max() > 1e-3


def test_full_grid_gradient_is_the_grid_exchange_gradient():
    """With every grid point an interpolation point and xi = delta the kernel
    is the closed-form full-grid kernel, independent of the orbitals; the
    closed form of the explicit term then equals the derivative of the
    brute-force grid exchange along theta."""
    c = cells.make_cell("C0", mesh=(3, 1, 1), grid=(6, 6, 6))  # a +-k pair: complex orbitals
    kf = cells.kmesh_frac(c.mesh)
    Xg = cells.bloch_collocation(c, cells.grid_points(c, 1), kf)
    C, Cv = cells.orbital_coefficients(c, 3)
    ng = int(np.prod(c.grid))
    p = dict(lattice=c.lattice, grid=c.grid, mesh=c.mesh, kfrac=kf, Xg=Xg, points=np.arange(ng))
    V = S.full_grid_kernel(c.lattice, c.grid, c.mesh)
    g = VO.explicit_gradient(p, C, Cv, V)
    rng = np.random.default_rng(7)
    th = rng.normal(size=g.shape) + 1j * rng.normal(size=g.shape)
    pred = float(np.real(np.sum(g.conj() * th)))
    fd = _directional_fd(
        lambda s: S.brute_force_exchange(c.lattice, c.grid, c.mesh, Xg, C + s * (Cv @ th))["Ex"])
    assert abs(fd - pred) <= 1e-8 * np.abs(g).sum() * np.abs(th).max()


def test_refit_gradient_on_a_zone_boundary_mesh():
    """The same finite-difference pin on a 2x2x1 mesh, whose q = (1/2, ., .)
    have two minimum-image representatives each (the kernel averages them),
    and a 7x6x5 grid (odd axes keep every frequency, the even one drops its
    Nyquist plane)."""
    c = cells.make_cell("C0", mesh=(2, 2, 1), grid=(7, 6, 5))
    kf = cells.kmesh_frac(c.mesh)
    Xg = cells.bloch_collocation(c, cells.grid_points(c, 1), kf)
    C, Cv = cells.orbital_coefficients(c, 3)
    p = dict(lattice=c.lattice, grid=c.grid, mesh=c.mesh, kfrac=kf, Xg=Xg, points=None)
    p["points"] = S.pivoted_cholesky(VO.grid_orbitals(p, C), 30)["points"]
    g = VO.vo_gradient(p, C, Cv)
    rng = np.random.default_rng(11)
    for _ in range(2):
        th = rng.normal(size=g.shape) + 1j * rng.normal(size=g.shape)
        pred = float(np.real(np.sum(g.conj() * th)))
        fd = _directional_fd(lambda s: VO.energy(p, C + s * (Cv @ th)))
        assert abs(fd - pred) <= 1e-8 * np.abs(g).sum() * np.abs(th).max()
