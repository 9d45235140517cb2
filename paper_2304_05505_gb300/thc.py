"""Python binding of libthc (include/thc.h): argument marshalling only.

Every step of the build runs in the library's CUDA kernels.  The functions
here carry the C names; they take torch tensors (complex128, contiguous, on
the context's device) or numpy arrays (for the host-buffer build) and pass
their pointers.  There is no fallback: if the library or a GPU is missing,
the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libthc.so")

THC_FP64 = 0
THC_MIXED = 1
THC_MIXED_SIMT = 2
THC_MIXED_EXT = 3
PRECISIONS = {"fp64": THC_FP64, "mixed": THC_MIXED, "mixed_simt": THC_MIXED_SIMT, "mixed_ext": THC_MIXED_EXT}

STATUS = {0: "THC_OK", 1: "THC_ERR_ARG", 2: "THC_ERR_OOM", 3: "THC_ERR_CUDA",
          4: "THC_ERR_NONFINITE", 5: "THC_ERR_TIMEOUT", 6: "THC_ERR_STATE",
          7: "THC_ERR_UNSUPPORTED"}

EXPORTS = ["thc_create", "thc_memory_bytes", "thc_set_collocation", "thc_set_kernel",
           "thc_build", "thc_build_host", "thc_get_intermediate", "thc_stage_times",
           "thc_launches_per_build", "thc_hermitian_kernel", "thc_destroy", "thc_status_string", "thc_last_error",
           "thc_profile_begin", "thc_profile_end", "thc_sync", "thc_kconv_noalloc",
           "thc_select_points", "thc_fit_kernel", "thc_profile_kernels", "thc_mlp_features", "thc_mlp_score",
           "thc_mlp_workspace_bytes", "thc_mlp_train_step", "thc_mlp_candidates", "thc_select_points_among",
           "thc_debug_set_wait_limit", "thc_debug_fail_alloc", "thc_rebuild_kernel", "thc_build_K",
           "thc_measure_fp64_rate", "thc_vo_gradient"]

MLP_NPARAM = 8641


class ThcDims(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("n3", ctypes.c_int),
                ("nbas", ctypes.c_int), ("nocc", ctypes.c_int), ("nisdf", ctypes.c_int)]


class ThcError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}" + (f" ({detail})" if detail else ""))


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libthc.so (built by build_lib.build()).  Raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libthc.so not built at {p}; run paper_2304_05505_gb300.build_lib.build()")
    lib = ctypes.CDLL(p)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p
    lib.thc_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ThcDims), ip, vp]
    lib.thc_memory_bytes.argtypes = [ctypes.POINTER(ThcDims), ip, ctypes.POINTER(ctypes.c_size_t)]
    lib.thc_set_collocation.argtypes = [vp, dp]
    lib.thc_set_kernel.argtypes = [vp, dp]
    lib.thc_build.argtypes = [vp, dp, dp, dp]
    lib.thc_build_host.argtypes = [vp, dp, dp, dp]
    lib.thc_build_K.argtypes = [vp, dp, dp, dp]
    lib.thc_get_intermediate.argtypes = [vp, ip, dp]
    lib.thc_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    lib.thc_launches_per_build.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.thc_hermitian_kernel.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.thc_profile_begin.argtypes = [vp, ip]
    lib.thc_profile_end.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)]
    lib.thc_profile_kernels.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    lib.thc_destroy.argtypes = [vp]
    lib.thc_sync.argtypes = [vp]
    lib.thc_debug_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
    lib.thc_debug_fail_alloc.argtypes = [ip]
    lib.thc_measure_fp64_rate.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.thc_kconv_noalloc.argtypes = [dp, dp, dp, ip, ip, ip, ctypes.c_long, vp]
    lib.thc_select_points.argtypes = [dp, ip, ip, ip, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), dp, vp]
    lib.thc_rebuild_kernel.argtypes = [dp, ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ip, ip, dp,
                                       ctypes.POINTER(ctypes.c_float), vp]
    lib.thc_fit_kernel.argtypes = [dp, ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ip, dp, dp, vp]
    lib.thc_vo_gradient.argtypes = [dp, ip, dp, ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ip, dp, ip, dp, dp,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float), vp]
    fp = ctypes.POINTER(ctypes.c_float)
    lib.thc_mlp_features.argtypes = [dp, ip, ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ip, dp, vp]
    lib.thc_mlp_score.argtypes = [dp, fp, dp, ip, dp, vp]
    lib.thc_mlp_workspace_bytes.argtypes = [ip, ctypes.POINTER(ctypes.c_size_t)]
    lib.thc_mlp_train_step.argtypes = [dp, dp, dp, ip, ctypes.c_float, fp, dp, dp, ip, ctypes.c_float, dp,
                                       ctypes.c_size_t, dp, dp, vp]
    lib.thc_mlp_candidates.argtypes = [dp, ip, ip, ctypes.POINTER(ctypes.c_int), vp]
    lib.thc_select_points_among.argtypes = [dp, ip, ip, ctypes.POINTER(ctypes.c_int), ip, ip, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), vp]
    lib.thc_status_string.argtypes = [ip]
    lib.thc_status_string.restype = ctypes.c_char_p
    lib.thc_last_error.argtypes = [vp]
    lib.thc_last_error.restype = ctypes.c_char_p
    for f in EXPORTS:
        if f not in ("thc_status_string", "thc_last_error"):
            getattr(lib, f).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def _check(code: int, where: str, ctx=None):
    if code != 0:
        detail = ""
        try:
            detail = load().thc_last_error(ctx).decode()
        except Exception:
            pass
        raise ThcError(code, where, detail)


def _dims(d: dict) -> ThcDims:
    return ThcDims(int(d["n1"]), int(d["n2"]), int(d["n3"]), int(d["nbas"]), int(d["nocc"]),
                   int(d["nisdf"]))


def _dev_ptr(t, shape=None, name="tensor", dtype=None) -> int:
    import torch
    dtype = torch.complex128 if dtype is None else dtype
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)} != {tuple(shape)}")
    return t.data_ptr()


# ---------------------------------------------------------------------------
# C calls, same names
# ---------------------------------------------------------------------------

def thc_memory_bytes(dims: dict, precision: int) -> int:
    b = ctypes.c_size_t(0)
    _check(load().thc_memory_bytes(ctypes.byref(_dims(dims)), int(precision), ctypes.byref(b)),
           "thc_memory_bytes")
    return int(b.value)


def thc_create(dims: dict, precision: int, stream: int | None = None) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    h = ctypes.c_void_p(0)
    _check(load().thc_create(ctypes.byref(h), ctypes.byref(_dims(dims)), int(precision),
                             ctypes.c_void_p(stream)), "thc_create")
    return h


def thc_set_collocation(ctx, X) -> None:
    _check(load().thc_set_collocation(ctx, _dev_ptr(X, name="X")), "thc_set_collocation", ctx)


def thc_set_kernel(ctx, V) -> None:
    _check(load().thc_set_kernel(ctx, _dev_ptr(V, name="V")), "thc_set_kernel", ctx)


def thc_build(ctx, C, KC, ex) -> None:
    import torch
    if not (isinstance(ex, torch.Tensor) and ex.is_cuda and ex.dtype == torch.float64 and ex.numel() >= 2):
        raise TypeError("ex: expected a CUDA float64 tensor with 2 elements")
    _check(load().thc_build(ctx, _dev_ptr(C, name="C"), _dev_ptr(KC, name="KC"), ex.data_ptr()),
           "thc_build", ctx)


def _host_ptr(a, dtype, name) -> int:
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != dtype or not a.is_contiguous():
            raise TypeError(f"{name}: expected a contiguous host tensor of {dtype}")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name}: must be contiguous")
        return a.ctypes.data
    raise TypeError(f"{name}: expected a host tensor or numpy array")


def thc_build_K(ctx, C, K, ex) -> None:
    """THC-AO-K build (see include/thc.h): K [N_k][nbas][nbas] complex128."""
    import torch
    if not (isinstance(ex, torch.Tensor) and ex.is_cuda and ex.dtype == torch.float64 and ex.numel() >= 2):
        raise TypeError("ex: expected a CUDA float64 tensor with 2 elements")
    _check(load().thc_build_K(ctx, _dev_ptr(C, name="C"), _dev_ptr(K, name="K"), ex.data_ptr()),
           "thc_build_K", ctx)


def thc_build_host(ctx, C_host, KC_host, ex_host) -> None:
    import torch
    _check(load().thc_build_host(ctx, _host_ptr(C_host, torch.complex128, "C_host"),
                                 _host_ptr(KC_host, torch.complex128, "KC_host"),
                                 _host_ptr(ex_host, torch.float64, "ex_host")),
           "thc_build_host", ctx)


def thc_get_intermediate(ctx, which: int, out) -> None:
    import torch
    dt = torch.float64 if int(which) == 4 else torch.complex128
    _check(load().thc_get_intermediate(ctx, int(which), _dev_ptr(out, name="out", dtype=dt)),
           "thc_get_intermediate", ctx)


STAGES = ["S1_collocate", "S2_density", "S3_kconv", "S4a_apply_M", "S4b_backproject", "S5_energy"]


def thc_profile_begin(ctx, max_builds: int) -> None:
    _check(load().thc_profile_begin(ctx, int(max_builds)), "thc_profile_begin", ctx)


def thc_profile_end(ctx) -> tuple:
    arr = (ctypes.c_float * 6)()
    n = ctypes.c_int(0)
    _check(load().thc_profile_end(ctx, arr, ctypes.byref(n)), "thc_profile_end", ctx)
    return [float(x) for x in arr], int(n.value)


def thc_profile_kernels(ctx) -> list:
    """Mean ms of each stage's main kernel in the last completed profile."""
    arr = (ctypes.c_float * 6)()
    _check(load().thc_profile_kernels(ctx, arr), "thc_profile_kernels", ctx)
    return [float(x) for x in arr]


def thc_stage_times(ctx) -> list:
    arr = (ctypes.c_float * 6)()
    _check(load().thc_stage_times(ctx, arr), "thc_stage_times", ctx)
    return [float(x) for x in arr]


def thc_hermitian_kernel(ctx) -> bool:
    """Whether the builds take the Hermitian form (see include/thc.h)."""
    n = ctypes.c_int(0)
    _check(load().thc_hermitian_kernel(ctx, ctypes.byref(n)), "thc_hermitian_kernel", ctx)
    return bool(n.value)


def thc_measure_fp64_rate(stream=None) -> float:
    """The device's measured FP64 FMA rate in TFLOP/s (see include/thc.h)."""
    r = ctypes.c_double(0.0)
    _check(load().thc_measure_fp64_rate(ctypes.c_void_p(_stream(stream)), ctypes.byref(r)), "thc_measure_fp64_rate")
    return r.value


def thc_launches_per_build(ctx) -> int:
    n = ctypes.c_int(0)
    _check(load().thc_launches_per_build(ctx, ctypes.byref(n)), "thc_launches_per_build", ctx)
    return int(n.value)


def thc_sync(ctx) -> None:
    _check(load().thc_sync(ctx), "thc_sync", ctx)


def thc_debug_set_wait_limit(ctx, cycles: int) -> None:
    """Test hook: the limit of the context's bounded device waits (see include/thc.h)."""
    _check(load().thc_debug_set_wait_limit(ctx, int(cycles)), "thc_debug_set_wait_limit", ctx)


def thc_debug_fail_alloc(nth: int) -> None:
    """Test hook: make allocation nth of the next thc_create fail (see include/thc.h)."""
    _check(load().thc_debug_fail_alloc(int(nth)), "thc_debug_fail_alloc")


def thc_kconv_noalloc(D, V, M, mesh, npq: int, stream: int | None = None) -> None:
    """k-mesh convolution without device allocation (see include/thc.h).

    D, V and M are complex128 CUDA tensors of N_k * npq elements each, on one
    device; the call runs on that device (its current stream unless `stream`
    is given).  Sizes are checked here, before anything is queued."""
    import torch
    nk = int(mesh[0]) * int(mesh[1]) * int(mesh[2])
    want = nk * int(npq)
    for t, nm in ((D, "D"), (V, "V"), (M, "M")):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{nm}: expected a CUDA tensor")
        if t.numel() != want:
            raise ValueError(f"{nm}: {t.numel()} elements, the mesh and npq need {want}")
    for t, nm in ((D, "D"), (V, "V"), (M, "M")):
        if not t.is_cuda:
            raise TypeError(f"{nm}: expected a CUDA tensor")
    if not (D.device == V.device == M.device):
        raise ValueError("D, V and M must be on one device")
    with torch.cuda.device(D.device):
        if stream is None:
            stream = torch.cuda.current_stream(D.device).cuda_stream
        _check(load().thc_kconv_noalloc(_dev_ptr(D, name="D"), _dev_ptr(V, name="V"), _dev_ptr(M, name="M"),
                                        int(mesh[0]), int(mesh[1]), int(mesh[2]), int(npq),
                                        ctypes.c_void_p(stream)),
               "thc_kconv_noalloc")


def thc_select_points(U, npts: int, rel_tol: float = 1e-14, stream: int | None = None):
    """FP64 pivoted-Cholesky interpolation points (see include/thc.h).

    U: CUDA complex128 tensor [nfunc][ncand].  Returns (points, residual diagonal)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    nfunc, ncand = U.shape
    pts = (ctypes.c_int * int(npts))()
    cnt = ctypes.c_int(0)
    resid = torch.empty(ncand, dtype=torch.float64, device=U.device)
    _check(load().thc_select_points(_dev_ptr(U, name="U"), int(nfunc), int(ncand), int(npts), float(rel_tol),
                                    pts, ctypes.byref(cnt), resid.data_ptr(), ctypes.c_void_p(stream)),
           "thc_select_points")
    return np.array(pts[: cnt.value], dtype=np.int64), resid


def thc_fit_kernel(U, grid, lattice, mesh, points, want_xi: bool = False, stream: int | None = None):
    """FP64 ISDF kernel of the interpolation points (see include/thc.h).

    U: CUDA complex128 tensor [nfunc][N_g] on the whole grid; grid, mesh:
    3 ints; lattice: 3 x 3 (rows a1, a2, a3); points: grid indices.  Returns
    V [N_k][npts][npts] complex128 (CUDA tensor), and xi [npts][N_g] if asked."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    nfunc, ng = U.shape
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    m = (ctypes.c_int * 3)(*[int(x) for x in mesh])
    lat = (ctypes.c_double * 9)(*[float(x) for x in np.asarray(lattice, dtype=np.float64).ravel()])
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int32))
    npts = int(pts.size)
    nk = int(np.prod([int(x) for x in mesh]))
    V = torch.empty((nk, npts, npts), dtype=torch.complex128, device=U.device)
    xi = torch.empty((npts, ng), dtype=torch.float64, device=U.device) if want_xi else None
    _check(load().thc_fit_kernel(_dev_ptr(U, name="U"), int(nfunc), g, lat, m,
                                 pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), npts, V.data_ptr(),
                                 xi.data_ptr() if xi is not None else None, ctypes.c_void_p(stream)),
           "thc_fit_kernel")
    return (V, xi) if want_xi else V


def thc_rebuild_kernel(U, grid, lattice, mesh, points, precision="mixed", stream: int | None = None):
    """The per-iteration kernel rebuild (see include/thc.h): V [N_k][npts][npts]
    complex128 (CUDA tensor) and the device ms of its five steps (metric,
    Cholesky, solve, FFT, contraction)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    nfunc, ng = U.shape
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    m = (ctypes.c_int * 3)(*[int(x) for x in mesh])
    lat = (ctypes.c_double * 9)(*[float(x) for x in np.asarray(lattice, dtype=np.float64).ravel()])
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int32))
    npts = int(pts.size)
    nk = int(np.prod([int(x) for x in mesh]))
    V = torch.empty((nk, npts, npts), dtype=torch.complex128, device=U.device)
    ms = (ctypes.c_float * 5)()
    _check(load().thc_rebuild_kernel(_dev_ptr(U, name="U"), int(nfunc), g, lat, m,
                                     pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), npts,
                                     int(PRECISIONS.get(precision, precision)), V.data_ptr(), ms,
                                     ctypes.c_void_p(stream)),
           "thc_rebuild_kernel")
    return V, [float(x) for x in ms]


def thc_vo_gradient(U, Uv, nk: int, grid, lattice, mesh, points, V, precision="fp64", stream: int | None = None):
    """The THC-oo-K orbital gradient with the kernel's response (see
    include/thc.h): U [N_k n_occ][N_g] and Uv [N_k n_vir][N_g] complex128 CUDA
    tensors, V [N_k][npts][npts] the kernel fitted to U at `points`, all on one
    device; precision "fp64" or "mixed" (the grid-sized contractions on the
    tensor cores).  Sizes and devices are checked here, before anything is
    allocated or queued; the call runs on that device (its current stream
    unless `stream` is given).  Returns (g, g_explicit, E_x, step_ms): g and
    g_explicit [N_k][n_vir][n_occ] complex128 CUDA tensors (the full gradient
    and its fixed-kernel term), E_x from sum_q W^q o V^q, and the device ms of
    the five steps."""
    import torch
    nk = int(nk)
    for t, nm in ((U, "U"), (Uv, "Uv"), (V, "V")):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{nm}: expected a CUDA tensor")
    if U.dim() != 2 or Uv.dim() != 2 or Uv.shape[1] != U.shape[1]:
        raise ValueError("U and Uv must be [rows][N_g] with the same N_g")
    nfo, ng = U.shape
    nfv = Uv.shape[0]
    if int(np.prod([int(x) for x in mesh])) != nk:
        raise ValueError("nk must be the number of k-mesh points")
    if int(np.prod([int(x) for x in grid])) != ng:
        raise ValueError("the grid must have N_g points, the length of the rows of U")
    if nfo % nk or nfv % nk or nfo == 0 or nfv == 0:
        raise ValueError("U and Uv rows must be N_k times the orbitals per k")
    nocc, nvir = nfo // nk, nfv // nk
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int32))
    npts = int(pts.size)
    if tuple(V.shape) != (nk, npts, npts):
        raise ValueError(f"V: shape {tuple(V.shape)} != {(nk, npts, npts)}")
    if precision not in PRECISIONS and precision not in PRECISIONS.values():
        raise ValueError(f"precision: {precision!r}")
    for t, nm in ((U, "U"), (Uv, "Uv"), (V, "V")):
        if not t.is_cuda:
            raise TypeError(f"{nm}: expected a CUDA tensor")
    if not (U.device == Uv.device == V.device):
        raise ValueError("U, Uv and V must be on one device")
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    m = (ctypes.c_int * 3)(*[int(x) for x in mesh])
    lat = (ctypes.c_double * 9)(*[float(x) for x in np.asarray(lattice, dtype=np.float64).ravel()])
    with torch.cuda.device(U.device):
        if stream is None:
            stream = torch.cuda.current_stream(U.device).cuda_stream
        gout = torch.empty((nk, nvir, nocc), dtype=torch.complex128, device=U.device)
        gexp = torch.empty_like(gout)
        ex = ctypes.c_double(0.0)
        ms = (ctypes.c_float * 5)()
        _check(load().thc_vo_gradient(_dev_ptr(U, (nfo, ng), name="U"), nocc, _dev_ptr(Uv, (nfv, ng), name="Uv"),
                                      nvir, g, lat, m, pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), npts,
                                      _dev_ptr(V, (nk, npts, npts), name="V"),
                                      int(PRECISIONS.get(precision, precision)), gout.data_ptr(), gexp.data_ptr(),
                                      ctypes.byref(ex), ms, ctypes.c_void_p(stream)),
               "thc_vo_gradient")
    return gout, gexp, float(ex.value), [float(x) for x in ms]


def _f32_dev(t, n=None, name="tensor") -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name}: expected a contiguous CUDA float32 tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name}: {t.numel()} elements, expected {n}")
    return t.data_ptr()


def _stream(stream):
    import torch
    return torch.cuda.current_stream().cuda_stream if stream is None else stream


def thc_mlp_features(U, nk: int, grid, lattice, centres, stream=None):
    """[N_g][3] float32 CUDA tensor of point features (see include/thc.h)."""
    import torch
    nfunc, ng = U.shape
    feat = torch.empty((ng, 3), dtype=torch.float32, device=U.device)
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    lat = (ctypes.c_double * 9)(*[float(x) for x in np.asarray(lattice, dtype=np.float64).ravel()])
    cen = np.ascontiguousarray(np.asarray(centres, dtype=np.float64))
    _check(load().thc_mlp_features(_dev_ptr(U, name="U"), int(nfunc), int(nk), g, lat,
                                   cen.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(cen.shape[0]),
                                   feat.data_ptr(), ctypes.c_void_p(_stream(stream))), "thc_mlp_features")
    return feat


def _norm(norm):
    return (ctypes.c_float * 6)(*[float(x) for x in np.asarray(norm).ravel()])


def thc_mlp_score(params, norm, feat, stream=None):
    """Logits [n] (float32 CUDA tensor) of features feat [n][3]."""
    import torch
    n = feat.shape[0]
    score = torch.empty(n, dtype=torch.float32, device=feat.device)
    _check(load().thc_mlp_score(_f32_dev(params, MLP_NPARAM, "params"), _norm(norm), _f32_dev(feat, name="feat"),
                                int(n), score.data_ptr(), ctypes.c_void_p(_stream(stream))), "thc_mlp_score")
    return score


class MlpTrainer:
    """Parameters, Adam moments and workspace of thc_mlp_train_step."""

    def __init__(self, params, norm, n: int, device=None):
        import torch
        self.torch = torch
        self.params = params.to(device or "cuda", dtype=torch.float32).contiguous().clone()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.norm = np.asarray(norm, dtype=np.float32)
        self.n = int(n)
        b = ctypes.c_size_t(0)
        _check(load().thc_mlp_workspace_bytes(self.n, ctypes.byref(b)), "thc_mlp_workspace_bytes")
        self.ws = torch.empty(int(b.value), dtype=torch.uint8, device=self.params.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.params.device)
        self.grad = torch.zeros_like(self.params)
        self.t = 0

    def step(self, feat, labels, pos_weight: float, lr: float, stream=None):
        """One Adam step (lr > 0) or the gradient alone (lr = 0, step count kept)."""
        if feat.shape[0] != self.n or labels.numel() != self.n:
            raise ValueError("batch size differs from the workspace's")
        t = self.t + 1 if lr > 0 else max(self.t, 1)
        _check(load().thc_mlp_train_step(self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), int(t),
                                         float(lr), _norm(self.norm), _f32_dev(feat, name="feat"),
                                         _f32_dev(labels, name="labels"), self.n, float(pos_weight),
                                         self.ws.data_ptr(), int(self.ws.numel()), self.loss.data_ptr(),
                                         self.grad.data_ptr(), ctypes.c_void_p(_stream(stream))),
               "thc_mlp_train_step")
        if lr > 0:
            self.t = t
        return self.loss, self.grad


def thc_mlp_candidates(score, k: int, stream=None):
    """Indices (numpy, ascending) of the k highest scores."""
    out = (ctypes.c_int * int(k))()
    _check(load().thc_mlp_candidates(_f32_dev(score, name="score"), int(score.numel()), int(k), out,
                                     ctypes.c_void_p(_stream(stream))), "thc_mlp_candidates")
    return np.array(out[:], dtype=np.int64)


def thc_select_points_among(U, cand, npts: int, rel_tol: float = 1e-14, stream=None):
    """Pivoted-Cholesky points among the candidate grid indices `cand`."""
    nfunc, ng = U.shape
    c = np.ascontiguousarray(np.asarray(cand, dtype=np.int32))
    pts = (ctypes.c_int * int(npts))()
    cnt = ctypes.c_int(0)
    _check(load().thc_select_points_among(_dev_ptr(U, name="U"), int(nfunc), int(ng),
                                          c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(c.size), int(npts),
                                          float(rel_tol), pts, ctypes.byref(cnt), ctypes.c_void_p(_stream(stream))),
           "thc_select_points_among")
    return np.array(pts[: cnt.value], dtype=np.int64)


def thc_destroy(ctx) -> None:
    _check(load().thc_destroy(ctx), "thc_destroy")


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class ExchangeBuild:
    """One context: set X and V once, then call build(C) every SCF iteration."""

    def __init__(self, dims: dict, precision="mixed", device=None, stream=None):
        import torch
        self.torch = torch
        self.dims = dict(dims)
        self.precision = PRECISIONS.get(precision, precision)
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.stream = stream or torch.cuda.current_stream(self.device)
            self.ctx = thc_create(self.dims, self.precision, self.stream.cuda_stream)
        d = self.dims
        self.nk = d["n1"] * d["n2"] * d["n3"]
        self.kc_shape = (self.nk, d["nbas"], d["nocc"])

    def set_collocation(self, X):
        thc_set_collocation(self.ctx, self._to_dev(X))

    def set_kernel(self, V):
        thc_set_kernel(self.ctx, self._to_dev(V))

    def _to_dev(self, a):
        t = self.torch
        if isinstance(a, np.ndarray):
            a = t.from_numpy(np.ascontiguousarray(a, dtype=np.complex128))
        return a.to(self.device, non_blocking=False).contiguous()

    def build(self, C, KC=None, ex=None):
        t = self.torch
        C = self._to_dev(C)
        if KC is None:
            KC = t.empty(self.kc_shape, dtype=t.complex128, device=self.device)
        if ex is None:
            ex = t.empty(2, dtype=t.float64, device=self.device)
        thc_build(self.ctx, C, KC, ex)
        return KC, ex

    def build_K(self, C, K=None, ex=None):
        """THC-AO-K: the full AO exchange matrix K^k = conj(X^k) M^k X^{kT} and E_x."""
        t = self.torch
        C = self._to_dev(C)
        d = self.dims
        if K is None:
            K = t.empty((self.nk, d["nbas"], d["nbas"]), dtype=t.complex128, device=self.device)
        if ex is None:
            ex = t.empty(2, dtype=t.float64, device=self.device)
        thc_build_K(self.ctx, C, K, ex)
        return K, ex

    def sync(self):
        thc_sync(self.ctx)

    def intermediate(self, which: int):
        t = self.torch
        d = self.dims
        if which == 4:
            out = t.empty((self.nk, d["nisdf"]), dtype=t.float64, device=self.device)
            thc_get_intermediate(self.ctx, which, out)
            return out
        shape = (self.nk, d["nisdf"], d["nocc"]) if which in (0, 3) else (self.nk, d["nisdf"], d["nisdf"])
        out = t.empty(shape, dtype=t.complex128, device=self.device)
        thc_get_intermediate(self.ctx, which, out)
        return out

    def stage_times(self):
        return thc_stage_times(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            thc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
