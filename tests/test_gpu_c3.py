"""The precision form at scale (the largest synthetic cell): a 2x1x1 supercell
of the benzene-shaped cell, 96 centres, N = 864, n = 120, 80 x 40 x 40 grid,
6 x 6 x 6 k (N_k = 216), N_P = 2400; the model kernel V^q is 20 GB in
complex128.  The mixed build and the FP64 GPU build are compared element by
element with the FP64 oracle, which runs steps 2-4a a block of rows at a time
(D and M of this cell are 20 GB each in complex128).

Tolerances: the target bounds of the 4x4x4 cell, max|dKC| <= 1e-7 and
|dE_x| <= 1e-6 Ha per cell, for the mixed build; 1e-10 / 1e-9 for FP64.

The inputs take a few minutes to make on the host, with their large matrix
products run through torch on the GPU (cells.set_accelerator)."""
import time

import numpy as np
import pytest

from oracle import thc_oracle as O
from paper_2304_05505_gb300 import cells

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def c3(cuda_required):
    import os
    from paper_2304_05505_gb300 import build_lib, thc
    if not os.path.exists(thc.LIB_PATH):
        build_lib.build()
    t0 = time.perf_counter()
    cells.set_accelerator("cuda")
    try:
        p = cells.make_problem("C3")
    finally:
        cells.set_accelerator(None)
    t1 = time.perf_counter()
    ref = O.build_rowblocks(p.X, p.C, p.V, p.cell.mesh)
    print(f"C3 inputs {t1 - t0:.0f} s, oracle {time.perf_counter() - t1:.0f} s, E_x = {ref['Ex']:.9f}")
    return p, ref


def _gpu_build(p, precision):
    from paper_2304_05505_gb300 import thc
    eb = thc.ExchangeBuild(p.dims, precision)
    try:
        eb.set_collocation(p.X)
        eb.set_kernel(p.V)
        KC, ex = eb.build(p.C)
        eb.sync()
        return KC.cpu().numpy(), float(ex[0])
    finally:
        eb.close()


def test_c3_mixed_target(c3):
    p, ref = c3
    kc, ex = _gpu_build(p, "mixed")
    dkc = float(np.abs(kc - ref["KC"]).max())
    dex = abs(ex - ref["Ex"])
    print(f"C3 mixed: max|dKC| = {dkc:.3e}, |dE_x| = {dex:.3e}, max|KC| = {np.abs(ref['KC']).max():.3f}")
    assert dkc <= 1e-7, dkc
    assert dex <= 1e-6, dex


def test_c3_fp64(c3):
    p, ref = c3
    kc, ex = _gpu_build(p, "fp64")
    dkc = float(np.abs(kc - ref["KC"]).max())
    dex = abs(ex - ref["Ex"])
    print(f"C3 fp64: max|dKC| = {dkc:.3e}, |dE_x| = {dex:.3e}")
    assert dkc <= 1e-10, dkc
    assert dex <= 1e-9, dex
