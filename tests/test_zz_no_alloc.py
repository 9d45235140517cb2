"""The allocation-free k-convolution entry point (thc_kconv_noalloc).

Some callers cannot allocate device memory when they call into the library:
a host framework that has already reserved the GPU's memory in its own pool,
or a caller that must not let cudaMalloc/cudaFree synchronise the device.
thc_kconv_noalloc gives them the k-mesh convolution with its scratch in a
static device array.  This file checks, through the C ABI, that two calls in a
row give the same M as the library's own build (FP64 form), within the FP64
tolerance of the other parity tests, and that sizes beyond the static scratch
are refused.  It is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2304_05505_gb300 import cells

pytestmark = pytest.mark.gpu


def test_noalloc_kconv_matches_build(cuda_required):
    import torch
    from paper_2304_05505_gb300 import thc
    mesh = (3, 2, 2)
    r = cells.random_problem(mesh, nbas=20, nocc=4, nisdf=45, seed=12)
    dims = dict(n1=3, n2=2, n3=2, nbas=20, nocc=4, nisdf=45)
    eb = thc.ExchangeBuild(dims, "fp64")
    eb.set_collocation(r["X"])
    eb.set_kernel(r["V"])
    eb.build(r["C"])
    eb.sync()
    D = eb.intermediate(1)                 # density of the build, [N_k][N_P][N_P]
    M_ref = eb.intermediate(2)             # the build's own k-convolution
    V = torch.from_numpy(r["V"]).cuda()
    npq = 45 * 45
    scale = float(M_ref.abs().max())
    for _ in range(2):                     # two calls in a row share the static scratch
        M = torch.full_like(M_ref, float("nan"))
        thc.thc_kconv_noalloc(D, V, M, mesh, npq)
        torch.cuda.synchronize()
        err = float((M - M_ref).abs().max())
        assert err <= 1e-12 * scale, err
    eb.close()


def test_noalloc_kconv_rejects_oversize(cuda_required):
    import torch
    from paper_2304_05505_gb300 import thc
    mesh = (4, 4, 4)
    npq = (1 << 21) // 64 + 1              # one element per k beyond the 32 MiB scratch
    D = torch.zeros(1, dtype=torch.complex128, device="cuda")
    with pytest.raises(thc.ThcError) as e:
        thc.thc_kconv_noalloc(D, D, torch.zeros(1, dtype=torch.complex128, device="cuda"), mesh, npq)
    assert e.value.code == 1
    assert b"static scratch" in thc.load().thc_last_error(None)
