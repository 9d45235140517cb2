"""Failure detection without a GPU fault (through the C ABI).

* A bounded device-side wait that runs out: a test hook shortens the limit of
  the context's waits to a few hundred clock cycles, so the first wait of the
  next build gives up before its TMA data arrives.  The kernels let their
  copies and MMAs in flight finish and stop; thc_sync reports THC_ERR_TIMEOUT.
  With the default limit restored, the same context builds correctly again
  (checked against the FP64 oracle).
* A device allocation that fails inside thc_create (a host-side fake of the
  allocator's out-of-memory answer, at several positions): THC_ERR_OOM, no
  context, and the device's free memory unchanged (nothing leaked).
"""
import numpy as np
import pytest

from oracle import thc_oracle as O
from paper_2304_05505_gb300 import cells

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(cuda_required):
    import os
    from paper_2304_05505_gb300 import build_lib, thc
    if not os.path.exists(thc.LIB_PATH):
        build_lib.build()
    return thc


def _check(got, ref):
    kc, ex = got
    scale = float(np.abs(ref["KC"]).max())
    assert float(np.abs(kc.cpu().numpy() - ref["KC"]).max()) <= 1e-6 * scale
    assert abs(float(ex[0]) - ref["Ex"]) <= 1e-6 * abs(ref["Ex"])


def test_wait_timeout_is_reported_and_context_recovers(lib):
    thc = lib
    mesh = (4, 4, 4)
    r = cells.random_problem(mesh, nbas=24, nocc=5, nisdf=64, seed=3)
    ref = O.build(r["X"], r["C"], r["V"], mesh)
    dims = dict(n1=4, n2=4, n3=4, nbas=24, nocc=5, nisdf=64)
    eb = thc.ExchangeBuild(dims, "mixed")
    try:
        eb.set_collocation(r["X"])
        eb.set_kernel(r["V"])
        assert thc.thc_hermitian_kernel(eb.ctx)      # the TMA-fed convolution and the tcgen05 GEMMs
        _check(eb.build(r["C"]), ref)
        eb.sync()
        thc.thc_debug_set_wait_limit(eb.ctx, 200)    # cycles: shorter than any DRAM round trip
        eb.build(r["C"])
        with pytest.raises(thc.ThcError) as e:
            eb.sync()
        assert e.value.code == 5                      # THC_ERR_TIMEOUT
        thc.thc_debug_set_wait_limit(eb.ctx, 0)      # the default limit again
        got = eb.build(r["C"])
        eb.sync()                                     # no timeout left over
        _check(got, ref)
    finally:
        thc.thc_debug_set_wait_limit(eb.ctx, 0)
        eb.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_create_oom_is_reported_without_leak(lib, precision):
    import torch
    thc = lib
    dims = dict(n1=3, n2=3, n3=3, nbas=40, nocc=6, nisdf=130)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for nth in (0, 2, 5):
        thc.thc_debug_fail_alloc(nth)
        with pytest.raises(thc.ThcError) as e:
            thc.thc_create(dims, thc.PRECISIONS[precision])
        assert e.value.code == 2                      # THC_ERR_OOM
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (nth, free0 - free1)
    thc.thc_debug_fail_alloc(-1)
    ctx = thc.thc_create(dims, thc.PRECISIONS[precision])   # the hook is spent: this one succeeds
    thc.thc_destroy(ctx)
