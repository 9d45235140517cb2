"""The C-ABI library loads and exports what include/thc.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

from paper_2304_05505_gb300 import build_lib, thc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(thc.LIB_PATH):
        build_lib.build()
    return thc.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "thc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(thc_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_functions()
    for f in ["thc_create", "thc_set_collocation", "thc_set_kernel", "thc_build", "thc_destroy"]:
        assert f in names


def test_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_covers_header():
    assert set(declared_functions()) <= set(thc.EXPORTS)


def test_status_strings(lib):
    for code in range(8):
        s = lib.thc_status_string(code)
        assert s and s != b"unknown status"
    assert lib.thc_status_string(99) == b"unknown status"


def test_memory_bytes_arithmetic():
    """Device bytes a context holds, counted from the array shapes."""
    d = dict(n1=4, n2=4, n3=4, nbas=432, nocc=60, nisdf=1200)
    nk, N, n, P = 64, 432, 60, 1200
    common = 2 * 16 * nk * N * n + 16 + 2 * 1216 * 8 + 64 + 64
    simt = 8 * (nk * N * P + nk * P * P + 2 * nk * P * n + 2 * nk * P * P) + common
    assert thc.thc_memory_bytes(d, thc.THC_MIXED_SIMT) == simt
    fp64 = 16 * (nk * N * P + nk * P * P + 2 * nk * P * n + 2 * nk * P * P) + common
    assert thc.thc_memory_bytes(d, thc.THC_FP64) == fp64

    def pad8(x):
        return (x + 7) // 8 * 8
    # fp16 planes of Psi (A of S2), embedded C, Psi^H and Psi / Y (B operands);
    # X itself is kept once in FP32 with rows padded to an even length
    planes = nk * (P * pad8(2 * n) + 2 * n * pad8(2 * N) + 2 * P * pad8(2 * n) + 2 * n * pad8(2 * P))
    x32 = 8 * nk * N * (P + P % 2)
    exps = nk * (N + 3 * P + 2 * n)
    def chunks(rows, kr):
        # split-K chunks: the fewest of at most 32 K blocks of 32 reals, one
        # more when a split product has fewer than 6 x 152 tile-chunk units
        nkb = -(-kr // 32)
        c = -(-nkb // 32)
        if 1 < c < nkb and nk * -(-rows // 128) * -(-(2 * n) // 128) * c < 6 * 152:
            c += 1
        return -(-nkb // -(-nkb // c))

    assert (chunks(P, 2 * N), chunks(P, 2 * P), chunks(N, 2 * P)) == (1, 3, 4)   # S1, S4a, S4b
    part = max(c * nk * rows * 2 * n if c > 1 else 0
               for rows, c in ((P, chunks(P, 2 * N)), (P, chunks(P, 2 * P)), (N, chunks(N, 2 * P))))
    # row and column keys of the Hermitian convolution: tiles of 8 rows by
    # 32 / n1 columns, n1 slots of ceil(N2 N3 / 2) words per row
    hkey = (-(-P // 8) + -(-P // 8)) * P * 4 * 8 + -(-P // 8) + 1   # + the tile table
    tc = 8 * (nk * P * P + 2 * nk * P * n + 2 * nk * P * P) + x32 + 3 * 2 * planes \
        + 4 * exps + 64 + 8 * part + 4 * hkey + common
    assert thc.thc_memory_bytes(d, thc.THC_MIXED) == tc
    # odd N_P: M's slices are kept in HBM as well (FP32 rows not 16-byte strided)
    d1 = dict(d, nisdf=P + 1)
    extra = 3 * 2 * nk * (P + 1) * pad8(2 * (P + 1))
    # (and the Hermitian convolution, which needs 16-byte strided FP32 rows too, has no keys)
    assert thc.thc_memory_bytes(d1, thc.THC_MIXED) - extra > thc.thc_memory_bytes(d, thc.THC_MIXED) - 4 * hkey


@pytest.mark.parametrize("bad", [
    dict(n1=0, n2=1, n3=1, nbas=4, nocc=2, nisdf=4),
    dict(n1=9, n2=1, n3=1, nbas=4, nocc=2, nisdf=4),
    dict(n1=1, n2=1, n3=1, nbas=4, nocc=0, nisdf=4),
    dict(n1=1, n2=1, n3=1, nbas=4, nocc=5, nisdf=4),
    dict(n1=1, n2=1, n3=1, nbas=4, nocc=2, nisdf=0),
])
def test_bad_dims_rejected(bad):
    with pytest.raises(thc.ThcError) as e:
        thc.thc_memory_bytes(bad, thc.THC_FP64)
    assert e.value.code == 1


def test_bad_precision_rejected():
    with pytest.raises(thc.ThcError) as e:
        thc.thc_memory_bytes(dict(n1=1, n2=1, n3=1, nbas=4, nocc=2, nisdf=4), 7)
    assert e.value.code == 1


def test_null_context_calls(lib):
    assert lib.thc_build(None, None, None, None) == 1
    assert lib.thc_destroy(None) == 1
    assert lib.thc_set_kernel(None, None) == 1


def test_memory_bytes_extended_form():
    """THC_MIXED_EXT adds one 32-bit remainder pair per element of M on the
    meshes its extended k-convolution covers (2 x 2 x 2 and 4 x 4 x 4, N_P a
    multiple of 4); elsewhere it holds what THC_MIXED holds."""
    d = dict(n1=4, n2=4, n3=4, nbas=432, nocc=60, nisdf=1200)
    nk, P = 64, 1200
    assert thc.thc_memory_bytes(d, thc.THC_MIXED_EXT) - thc.thc_memory_bytes(d, thc.THC_MIXED) == 4 * nk * P * P
    for other in (dict(d, n1=3, n2=3, n3=3), dict(d, n1=4, n2=4, n3=2), dict(d, nisdf=1202)):
        assert thc.thc_memory_bytes(other, thc.THC_MIXED_EXT) == thc.thc_memory_bytes(other, thc.THC_MIXED)


def _vo_args(nk=2, nocc=3, nvir=2, grid=(4, 3, 2), npts=5, **over):
    import torch
    ng = grid[0] * grid[1] * grid[2]
    a = dict(U=torch.zeros((nk * nocc, ng), dtype=torch.complex128),
             Uv=torch.zeros((nk * nvir, ng), dtype=torch.complex128), nk=nk, grid=grid,
             lattice=[[5.0, 0, 0], [0, 5.0, 0], [0, 0, 5.0]], mesh=(nk, 1, 1), points=list(range(npts)),
             V=torch.zeros((nk, npts, npts), dtype=torch.complex128))
    a.update(over)
    return a


@pytest.mark.parametrize("change,exc", [
    (dict(nk=3), ValueError),                                    # mesh has 2 points
    (dict(grid=(4, 3, 3)), ValueError),                          # N_g of U is 24
    (dict(points=list(range(6))), ValueError),                   # V is [2][5][5]
    (dict(precision="fp32"), ValueError),
    ({}, TypeError),                                             # CPU tensors
])
def test_vo_gradient_wrapper_checks_before_launch(change, exc):
    """The binding of thc_vo_gradient rejects inconsistent sizes, an unknown
    precision and non-CUDA tensors on the host, before any allocation or
    launch (so no call reaches the library here)."""
    a = _vo_args()
    change = dict(change)
    prec = change.pop("precision", "fp64")
    a.update(change)
    with pytest.raises(exc):
        thc.thc_vo_gradient(a["U"], a["Uv"], a["nk"], a["grid"], a["lattice"], a["mesh"], a["points"], a["V"], prec)


def test_vo_gradient_wrapper_rejects_mismatched_rows():
    import torch
    a = _vo_args()
    bad = torch.zeros((5, 24), dtype=torch.complex128)   # 5 rows is not a multiple of N_k = 2
    with pytest.raises(ValueError):
        thc.thc_vo_gradient(bad, a["Uv"], 2, a["grid"], a["lattice"], a["mesh"], a["points"], a["V"])
    with pytest.raises(ValueError):
        thc.thc_vo_gradient(a["U"], torch.zeros((4, 23), dtype=torch.complex128), 2, a["grid"], a["lattice"],
                            a["mesh"], a["points"], a["V"])


def _vo_call(lib, U=256, nocc=2, Uv=512, nvir=2, grid=(4, 3, 2), mesh=(2, 1, 1), points=(0, 1, 2), V=768,
             precision=0, g=1024):
    gr = (ctypes.c_int * 3)(*grid)
    me = (ctypes.c_int * 3)(*mesh)
    lat = (ctypes.c_double * 9)(5.0, 0, 0, 0, 5.0, 0, 0, 0, 5.0)
    pts = (ctypes.c_int * len(points))(*points)
    return lib.thc_vo_gradient(ctypes.c_void_p(U), nocc, ctypes.c_void_p(Uv), nvir, gr, lat, me, pts, len(points),
                               ctypes.c_void_p(V), precision, ctypes.c_void_p(g), None, None, None, None)


@pytest.mark.parametrize("change", [
    dict(U=0), dict(Uv=0), dict(V=0), dict(g=0),            # null pointers
    dict(U=264),                                             # not 16-byte aligned
    dict(nocc=0), dict(nvir=0),
    dict(precision=2),                                       # only THC_FP64 and THC_MIXED
    dict(points=(0, 1, 1)),                                  # repeated point
    dict(points=(0, 24)),                                    # out of the 24-point grid
    dict(mesh=(9, 1, 1)),                                    # mesh axis above 8
])
def test_vo_gradient_c_entry_rejects_bad_arguments(lib, change):
    """thc_vo_gradient returns THC_ERR_ARG for each bad argument on the host,
    before any CUDA call (the device pointers here are never dereferenced)."""
    assert _vo_call(lib, **change) == 1
