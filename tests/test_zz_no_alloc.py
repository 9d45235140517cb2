"""The allocation-free k-convolution entry point (thc_kconv_noalloc).

Some callers cannot allocate device memory when they call into the library:
a host framework that has already reserved the GPU's memory in its own pool,
or a caller that must not let cudaMalloc/cudaFree synchronise the device.
thc_kconv_noalloc gives them the k-mesh convolution with its scratch in a
static device array.  These tests call it through the C ABI twice in a row,
with a different mesh, size and kernel the second time (so a stale prepared
kernel left in the shared scratch would show), and compare each result with
the FP64 oracle's direct k' sum; they also check that sizes beyond the static
scratch and outputs that overlap an input are refused.  The file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from oracle import thc_oracle as O

gpu = pytest.mark.gpu


def _case(mesh, npq, seed):
    rng = np.random.default_rng(seed)
    nk = int(np.prod(mesh))
    D = rng.normal(size=(nk, npq)) + 1j * rng.normal(size=(nk, npq))
    V = rng.normal(size=(nk, npq)) + 1j * rng.normal(size=(nk, npq))
    return D, V, O.kconv_direct(D, V, mesh)


@gpu
def test_noalloc_kconv_two_calls_match_oracle(cuda_required):
    import torch
    from paper_2304_05505_gb300 import thc
    for mesh, npq, seed in (((3, 2, 2), 45 * 45, 12), ((2, 2, 2), 37 * 37, 13)):
        D, V, M_ref = _case(mesh, npq, seed)
        Dd = torch.from_numpy(D).cuda()
        Vd = torch.from_numpy(V).cuda()
        M = torch.full_like(Dd, float("nan"))
        thc.thc_kconv_noalloc(Dd, Vd, M, mesh, npq)
        torch.cuda.synchronize()
        err = float(np.abs(M.cpu().numpy() - M_ref).max())
        assert err <= 1e-12 * float(np.abs(M_ref).max()), (mesh, err)


@gpu
def test_noalloc_kconv_rejects_oversize_and_overlap(cuda_required):
    import torch
    from paper_2304_05505_gb300 import thc
    lib = thc.load()
    buf = torch.zeros(2 * 64, dtype=torch.complex128, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = buf.data_ptr()
    # one element per k beyond the 32 MiB scratch: refused before any device access
    assert lib.thc_kconv_noalloc(p, p, p + 16 * 64, 4, 4, 4, (1 << 21) // 64 + 1, stream) == 1
    assert b"static scratch" in lib.thc_last_error(None)
    # M overlapping D
    assert lib.thc_kconv_noalloc(p, p + 16 * 64, p, 4, 4, 4, 1, stream) == 1
    assert b"overlaps" in lib.thc_last_error(None)


def test_noalloc_wrapper_checks_sizes_before_the_call():
    """The binding refuses tensors whose size does not match the mesh and npq
    before it reaches the C call (no device needed)."""
    import torch
    from paper_2304_05505_gb300 import thc
    a = torch.zeros(8 * 4, dtype=torch.complex128)
    short = torch.zeros(8 * 4 - 1, dtype=torch.complex128)
    with pytest.raises(ValueError):
        thc.thc_kconv_noalloc(a, a, short, (2, 2, 2), 4)
    with pytest.raises(ValueError):
        thc.thc_kconv_noalloc(short, a, a, (2, 2, 2), 4)
    with pytest.raises(TypeError):          # right sizes, but host tensors
        thc.thc_kconv_noalloc(a, a, a, (2, 2, 2), 4)
