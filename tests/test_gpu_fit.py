"""GPU FP64 ISDF kernel fit vs the oracle, through the C ABI.

The kernel of the toy cubic cell (16^3 grid, 2x2x2 and 3x3x3 k, 4 occupied
orbitals) from pivoted-Cholesky points, element by element within 1e-10 of
its largest entry (FP64 with a different summation order), and the error
paths of the entry point."""
import numpy as np
import pytest

from oracle import setup_oracle as S
from paper_2304_05505_gb300 import cells

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def thc_mod(cuda_required):
    import os

    from paper_2304_05505_gb300 import build_lib, thc
    if not os.path.exists(thc.LIB_PATH):
        build_lib.build()
    thc.load()
    return thc


def toy_u(mesh, grid):
    c = cells.make_cell("C0", mesh=mesh, grid=grid)
    pts = cells.grid_points(c, 1)
    kf = cells.kmesh_frac(c.mesh)
    Xg = cells.bloch_collocation(c, pts, kf)
    C = cells.occupied_coefficients(c)
    psi = np.einsum("kmr,kmi->kir", Xg, C)
    phase = np.exp(-1j * (pts @ (kf @ c.recip).T)).T
    U = np.ascontiguousarray((psi * phase[:, None, :]).reshape(-1, pts.shape[0]))
    return c, U


@pytest.mark.parametrize("mesh,grid,npts", [((2, 2, 2), (16, 16, 16), 48), ((3, 3, 3), (8, 8, 8), 40),
                                            ((1, 1, 1), (9, 8, 7), 8)])
def test_fit_matches_oracle(thc_mod, mesh, grid, npts):
    import torch
    c, U = toy_u(mesh, grid)
    P = S.pivoted_cholesky(U, npts)["points"]
    ref = S.fit_kernel(c.lattice, c.grid, c.mesh, U, P)
    xi_ref = S.isdf_fit(U, P)
    V, xi = thc_mod.thc_fit_kernel(torch.from_numpy(U).cuda(), c.grid, c.lattice, c.mesh, P, want_xi=True)
    V = V.cpu().numpy()
    assert np.abs(V - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.abs(xi.cpu().numpy() - xi_ref).max() <= 1e-9 * np.abs(xi_ref).max()


def test_fit_feeds_the_build(thc_mod):
    """The fitted kernel goes straight into thc_set_kernel: the FP64 build
    with it equals the oracle build with the oracle's fitted kernel."""
    import torch
    from oracle import thc_oracle as O
    c, U = toy_u((2, 2, 2), (16, 16, 16))
    P = S.pivoted_cholesky(U, 48)["points"]
    V = thc_mod.thc_fit_kernel(torch.from_numpy(U).cuda(), c.grid, c.lattice, c.mesh, P)
    pts = cells.grid_points(c, 1)[P]
    X = cells.bloch_collocation(c, pts, cells.kmesh_frac(c.mesh))
    C = cells.occupied_coefficients(c)
    dims = dict(n1=2, n2=2, n3=2, nbas=X.shape[1], nocc=C.shape[2], nisdf=48)
    eb = thc_mod.ExchangeBuild(dims, "fp64")
    eb.set_collocation(X)
    eb.set_kernel(V)
    KC, ex = eb.build(torch.from_numpy(C).cuda())
    eb.sync()
    ref = O.build(X, C, S.fit_kernel(c.lattice, c.grid, c.mesh, U, P), c.mesh)
    assert np.abs(KC.cpu().numpy() - ref["KC"]).max() <= 1e-10 * np.abs(ref["KC"]).max()
    assert abs(float(ex[0]) - ref["Ex"]) <= 1e-10 * abs(ref["Ex"])
    eb.close()


def test_bad_points_rejected(thc_mod):
    import torch
    c, U = toy_u((1, 1, 1), (8, 8, 8))
    Ud = torch.from_numpy(U).cuda()
    with pytest.raises(thc_mod.ThcError):
        thc_mod.thc_fit_kernel(Ud, c.grid, c.lattice, c.mesh, [3, 3])         # repeated point
    with pytest.raises(thc_mod.ThcError):
        thc_mod.thc_fit_kernel(Ud, c.grid, c.lattice, c.mesh, [0, 512])       # out of range
    # more points than the Gram rank (10): the metric is singular
    P = S.pivoted_cholesky(U, 10)["points"]
    extra = [i for i in range(512) if i not in set(P.tolist())][:3]
    with pytest.raises(thc_mod.ThcError):
        thc_mod.thc_fit_kernel(Ud, c.grid, c.lattice, c.mesh, list(P) + extra)


@pytest.mark.parametrize("mesh,grid,npts", [((2, 2, 2), (16, 16, 16), 48), ((3, 3, 3), (8, 8, 8), 40)])
def test_rebuild_fp64_is_the_fit(thc_mod, mesh, grid, npts):
    """The FP64 rebuild is thc_fit_kernel, bit for bit, and reports its step times."""
    import torch
    c, U = toy_u(mesh, grid)
    P = S.pivoted_cholesky(U, npts)["points"]
    Ud = torch.from_numpy(U).cuda()
    V0 = thc_mod.thc_fit_kernel(Ud, c.grid, c.lattice, c.mesh, P)
    V1, ms = thc_mod.thc_rebuild_kernel(Ud, c.grid, c.lattice, c.mesh, P, "fp64")
    assert torch.equal(V0, V1)
    assert len(ms) == 5 and all(t >= 0 for t in ms) and sum(ms) > 0


@pytest.mark.parametrize("mesh,grid,npts", [((2, 2, 2), (16, 16, 16), 48), ((3, 3, 3), (8, 8, 8), 40),
                                            ((4, 4, 4), (12, 12, 12), 64)])
def test_rebuild_mixed_matches_oracle(thc_mod, mesh, grid, npts):
    """The kernel contraction on tensor cores against the oracle's FP64 fit:
    within 1e-6 of the largest entry (the vectors are rounded to FP32,
    6e-8 relative, before the exact-chunked slice products), and the FP64
    build with it within 1e-6 relative of the build with the oracle's kernel
    in E_x and KC."""
    import torch
    from oracle import thc_oracle as O
    c, U = toy_u(mesh, grid)
    P = S.pivoted_cholesky(U, npts)["points"]
    ref = S.fit_kernel(c.lattice, c.grid, c.mesh, U, P)
    V, ms = thc_mod.thc_rebuild_kernel(torch.from_numpy(U).cuda(), c.grid, c.lattice, c.mesh, P, "mixed")
    V = V.cpu().numpy()
    assert np.abs(V - ref).max() <= 1e-6 * np.abs(ref).max()
    X = cells.bloch_collocation(c, cells.points_from_indices(c, P), cells.kmesh_frac(c.mesh))
    C = cells.occupied_coefficients(c)
    a = O.build(X, C, ref, c.mesh)
    b = O.build(X, C, V, c.mesh)
    assert abs(a["Ex"] - b["Ex"]) <= 1e-6 * abs(a["Ex"])
    assert np.abs(a["KC"] - b["KC"]).max() <= 1e-6 * np.abs(a["KC"]).max()
