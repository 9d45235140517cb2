"""The target configuration on an ISDF-fitted kernel (4x4x4 k, N_P = 1200,
n = 60, N = 432, 40^3 grid).

The other full-size tests use the model kernel of the seeded generator.  Here
the kernel is the one the method feeds the build:
* the interpolation points are the FP64 full-grid pivoted Cholesky of the
  occupied pair products (thc_select_points on the orbitals on all 64,000
  grid points; Sec. 2.1, in the pivoted-Cholesky reading of the QRCP
  selection);
* V^q is the least-squares fit of those products and its Coulomb kernel
  (thc_rebuild_kernel, Sec. 2.2 and the first three steps of Algorithm 2),
  in FP64 and with the contraction on tensor cores.
Tolerances.  Both mixed forms meet the target in E_x, |dE_x| <= 1e-6 Ha per
cell (measured 1e-8 to 1.3e-7 for either form, depending on the GEMMs'
summation order), and are held to the general mixed-precision bound in KC,
max|dKC| <= 1e-6 max|KC| (max|KC| = 0.74 here).  The target's max|dKC| <=
1e-7 is not met on this kernel: THC_MIXED measures 3.6e-7 to 4.3e-7 and
THC_MIXED_EXT 1.5e-7 to 1.9e-7.  The fitted M^k makes Y = M Psi
cancel (sum |M| |Psi| is about 6 |Y|):
* in THC_MIXED the FP32 k-convolution dominates (the FP32 rounding of M alone
  gives 1e-7 in KC, the FP32 DFT arithmetic about 3.5e-7);
* the extended convolution carries M to about 1e-11, and what remains comes
  from the FP32 Psi, D and Y, each near 5e-8 in KC after the amplification.
The tensor-core kernel must agree with the FP64 one (1e-6 of its largest
entry; the oracle builds with the two within 1e-6 relative in E_x)."""
import time

import numpy as np
import pytest

from oracle import thc_oracle as O
from paper_2304_05505_gb300 import cells

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def fitted(cuda_required):
    import os

    import torch
    from paper_2304_05505_gb300 import build_lib, thc
    if not os.path.exists(thc.LIB_PATH):
        build_lib.build()
    t0 = time.perf_counter()
    cell = cells.make_cell("C2")
    cells.set_accelerator("cuda")
    try:
        C = cells.occupied_coefficients(cell)
        U = cells.grid_orbitals(cell, C)
    finally:
        cells.set_accelerator(None)
    t1 = time.perf_counter()
    Ud = torch.from_numpy(U).cuda()
    del U
    pts, _ = thc.thc_select_points(Ud, cell.nisdf)
    t2 = time.perf_counter()
    V64, ms64 = thc.thc_rebuild_kernel(Ud, cell.grid, cell.lattice, cell.mesh, pts, "fp64")
    Vtc, mstc = thc.thc_rebuild_kernel(Ud, cell.grid, cell.lattice, cell.mesh, pts, "mixed")
    del Ud
    X = cells.bloch_collocation(cell, cells.points_from_indices(cell, pts), cells.kmesh_frac(cell.mesh))
    print(f"fitted C2: inputs {t1 - t0:.0f} s, points {t2 - t1:.1f} s, rebuild FP64 {sum(ms64):.0f} ms "
          f"{[round(x, 1) for x in ms64]}, tensor cores {sum(mstc):.0f} ms {[round(x, 1) for x in mstc]}")
    return cell, X, C, V64.cpu().numpy(), Vtc.cpu().numpy()


@pytest.fixture(scope="module")
def fitted_ref(fitted):
    cell, X, C, V64, _ = fitted
    return O.build(X, C, V64, cell.mesh, route="fft")


def _fitted_build(fitted, precision):
    from paper_2304_05505_gb300 import thc
    cell, X, C, V64, _ = fitted
    dims = dict(n1=4, n2=4, n3=4, nbas=cell.nbas, nocc=cell.nocc, nisdf=cell.nisdf)
    eb = thc.ExchangeBuild(dims, precision)
    try:
        eb.set_collocation(X)
        eb.set_kernel(V64)
        KC, ex = eb.build(C)
        eb.sync()
        return KC.cpu().numpy(), float(ex[0]), thc.thc_hermitian_kernel(eb.ctx)
    finally:
        eb.close()


@pytest.mark.parametrize("precision", ["mixed_ext", "mixed"])
def test_fitted_kernel_mixed_build(fitted, fitted_ref, precision):
    kc, ex, herm = _fitted_build(fitted, precision)
    dkc = float(np.abs(kc - fitted_ref["KC"]).max())
    dex = abs(ex - fitted_ref["Ex"])
    print(f"fitted C2 {precision}: max|dKC| = {dkc:.3e}, |dE_x| = {dex:.3e}, E_x = {fitted_ref['Ex']:.9f}, "
          f"Hermitian form {herm}")
    assert herm                          # the fitted kernel is exactly Hermitian per q
    assert dkc <= 1e-6 * float(np.abs(fitted_ref["KC"]).max()), dkc
    assert dex <= 1e-6, dex


def test_tensor_core_rebuild_matches_fp64(fitted, fitted_ref):
    cell, X, C, V64, Vtc = fitted
    dv = float(np.abs(Vtc - V64).max()) / float(np.abs(V64).max())
    a = fitted_ref
    b = O.build(X, C, Vtc, cell.mesh, route="fft")
    print(f"fitted C2 rebuild: max|dV|/max|V| = {dv:.3e}, dE_x = {abs(a['Ex'] - b['Ex']):.3e}")
    assert dv <= 1e-6, dv
    assert abs(a["Ex"] - b["Ex"]) <= 1e-6 * abs(a["Ex"])
