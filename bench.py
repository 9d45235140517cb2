#!/usr/bin/env python3
"""THC-oo-K exchange-build benchmark (arXiv 2304.05505, Algorithm 2's K build).

One step is one exchange build (S1 collocation, S2 point-space density, S3
k-convolution, S4 back-projection, S5 energy) on the benzene-shaped cell:
4 x 4 x 4 k, N_P = 1200 interpolation points, n = 60 occupied orbitals,
N = 432 basis functions, with X and V already resident on the GPU.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is mixed-precision builds/s summed
over ranks (each rank runs its own independent build: weak scaling, no
collective on the data path).  The FP64 GPU build, per-stage times, the
error against the FP64 CPU oracle, the end-to-end host-buffer number and the
oracle's own CPU rate are reported beside it.  --impl reference times the
FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "THC-oo-K exchange builds/s, mixed vs FP64 on one GB300 at <=1e-6 Ha; % roofline"
WORKLOADS = {
    "C1": ("benzene-shaped orthorhombic cell 13.9x17.8x12.9 bohr, 48 centres, N=432, n_occ=60, "
           "3x3x3 k (N_k=27), N_ISDF=600, 40^3 grid (config C1)"),
    "C2": ("benzene-shaped orthorhombic cell 13.9x17.8x12.9 bohr, 48 centres, N=432, n_occ=60, "
           "4x4x4 k (N_k=64), N_ISDF=1200, 40^3 grid (config C2)"),
    "C3": ("2x1x1 supercell of the benzene-shaped cell, 27.8x17.8x12.9 bohr, 96 centres, N=864, n_occ=120, "
           "6x6x6 k (N_k=216), N_ISDF=2400, 80x40x40 grid (config C3)"),
}
SAMPLE_FRACTION = 8      # the CPU oracle sample is 1/8 of a build
# fp16 slice products per real product of each tensor-core GEMM (the
# library's plan: S1 and S2 rounded to FP32 take 6, the back-projections 8)
SLICE_PRODUCTS = {"S1_collocate": 6, "S2_density": 6, "S4a_apply_M": 8, "S4b_backproject": 8}


def kernel_names(hermitian: bool) -> dict:
    """The main kernel of each stage of the tensor-core build."""
    return {"S1_collocate": "tc_gemm_kernel<0, 6, 0, 2> (S1, X^T read from FP32 X and sliced in the GEMM)",
            "S2_density": ("tc_gemm_kernel<0, 6, 1, 0> (S2, A resident, Hermitian tiles)" if hermitian else
                           "tc_gemm_kernel<0, 6, 1, 0> (S2, A resident, Hermitian tiles mirrored)"),
            "S3_kconv": ("kconv_herm_kernel<4, 4, 4> (S3, Hermitian tiles)" if hermitian else
                         "kconv_tile_kernel (S3, TMA-fed shared-memory DFTs)"),
            "S4a_apply_M": "tc_gemm_kernel<2, 8, 0, 1> (S4a, split-K, M sliced in the GEMM)",
            "S4b_backproject": "tc_gemm_kernel<2, 8, 0, 1> (S4b, split-K, X sliced in the GEMM)",
            "S5_energy": "ex_final (S5; the partial sums of <Psi, Y> are formed in S4a's split-K combine)"}


def s4a_split(d: dict) -> bool:
    """Whether S4a (Y = M Psi, K = 2 N_P reals) is split along K with 16-byte
    result rows (n_occ even): then its combine kernel forms E_x's partial sums
    and S5 is the final sum alone.  The chunk rule of the library: the fewest
    chunks of at most 1024 real K."""
    return 2 * d["nisdf"] > 1024 and d["nocc"] % 2 == 0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-samples", type=int, default=4)
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle error and CPU baseline")
    ap.add_argument("--config", default="C2", choices=sorted(WORKLOADS),
                    help="C2 (default: the headline workload), C1 (3x3x3 k) or C3, the 6x6x6-k supercell "
                         "at scale, timed once for the record (its inputs take minutes to make)")
    ap.add_argument("--kernel", default="model", choices=["model", "fitted"],
                    help="model: the generator's model kernel at density-sampled points (default); fitted: "
                         "points from the FP64 full-grid pivoted Cholesky and V^q from the library's kernel "
                         "rebuild (tensor-core contraction), as the method feeds the build")
    ap.add_argument("--no-rebuild", action="store_true",
                    help="skip timing the per-iteration kernel rebuild (C2 only)")
    ap.add_argument("--rebuild-fp64", action="store_true",
                    help="also time the all-FP64 kernel rebuild (about a minute at C2)")
    ap.add_argument("--vo-gradient", action="store_true",
                    help="also time the FP64 THC-oo-K orbital gradient with the kernel's response (all virtual "
                         "orbitals) at --config; seconds at C1, minutes at C2")
    ap.add_argument("--mixed-only", action="store_true",
                    help="time the mixed build alone (no host-buffer, CUDA-core, FP64 or oracle arms): "
                         "the small process a profiler capture runs")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------

def dist_setup(gpus: int):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", str(self.dev)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------

def peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return dict(hbm_gbs=float(p["hbm_gbs"]), bf16_tflops=float(p["bf16_tflops"]),
                    bf16_tflops_sustained=float(p.get("bf16_tflops_sustained", p["bf16_tflops"])),
                    sm_max_mhz=float(p.get("sm_max_mhz", 2070.0)), source="measured")
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, sm_max_mhz=2070.0,
                source="fallback")


def stage_work(d: dict, hermitian: bool = False) -> dict:
    """Algorithmic work of each stage's main kernel in one build: complex
    multiply-adds at 8 flops, and the arrays the step must read and write once
    at complex64 (KC and the C input at complex128).  In the Hermitian form
    (every V^q Hermitian, so D^k and M^k are) S2 forms and writes the
    P (P + 1) / 2 elements of D on and above the diagonal, and S3 reads that
    half of D and of the prepared kernel and writes all of M."""
    nk = d["n1"] * d["n2"] * d["n3"]
    N, n, P = d["nbas"], d["nocc"], d["nisdf"]
    c64 = 8
    half = P * (P + 1) / 2 if hermitian else P * P
    # S2 multiplies only the tiles that reach the diagonal in both forms (the
    # other form writes the mirror image too)
    return {
        "S1_collocate": dict(flops=8.0 * nk * P * n * N, bytes=c64 * nk * (N * P + P * n) + 16 * nk * N * n),
        "S2_density": dict(flops=8.0 * nk * P * (P + 1) / 2 * n, bytes=c64 * nk * (P * n + half)),
        "S3_kconv": dict(flops=None, bytes=c64 * nk * (2.0 * half + P * P)),
        "S4a_apply_M": dict(flops=8.0 * nk * P * P * n, bytes=c64 * nk * (P * P + 2 * P * n)),
        "S4b_backproject": dict(flops=8.0 * nk * N * n * P, bytes=c64 * nk * (N * P + P * n) + 16 * nk * N * n),
        "S5_energy": dict(flops=None, bytes=2.0 * c64 * nk * P * n),
    }


def fp64_roofline(d: dict, stages_ms: dict, fp64_tflops: float, pk: dict) -> dict:
    """The FP64 build against its own peaks: its four GEMMs (full D in S2) run
    on the FP64 pipe of the CUDA cores, reported against the measured FP64
    FMA rate; its k-convolution (complex128 D, Vh and M) against the copy
    bandwidth."""
    nk = d["n1"] * d["n2"] * d["n3"]
    N, n, P = d["nbas"], d["nocc"], d["nisdf"]
    flops = {"S1_collocate": 8.0 * nk * P * n * N, "S2_density": 8.0 * nk * P * P * n,
             "S4a_apply_M": 8.0 * nk * P * P * n, "S4b_backproject": 8.0 * nk * N * n * P}
    out = {"fp64_peak_tflops": fp64_tflops, "peak_source": "measured FP64 FMA rate (thc_measure_fp64_rate)"}
    for st, f in flops.items():
        a = f / (stages_ms[st] * 1e-3) / 1e12
        out[st] = {"bound": "fp64", "achieved_tflops": a, "frac": a / fp64_tflops}
    b = 16.0 * nk * 3 * P * P
    a = b / (stages_ms["S3_kconv"] * 1e-3) / 1e9
    out["S3_kconv"] = {"bound": "hbm", "achieved_gbs": a, "frac": a / pk["hbm_gbs"]}
    return out


def kernel_roofline(stage: str, ms: float, work: dict, pk: dict, config: str = "C2") -> dict:
    """Roofline of one stage's main kernel (or the stage) at `ms` per build.

    The bound is whichever lower limit is larger: algorithmic bytes over the
    measured copy bandwidth, or algorithmic flops over the sustained bf16
    tensor peak (the kernels run inside a multi-millisecond build; fp16 runs
    at the bf16 rate).  The tensor-core GEMMs issue 6 or 8 fp16 slice
    products per real product (SLICE_PRODUCTS), so their issued tensor
    fraction is also given."""
    w = work[stage]
    sec = ms * 1e-3
    t_hbm = w["bytes"] / (pk["hbm_gbs"] * 1e9)
    t_ten = (w["flops"] / (pk["bf16_tflops_sustained"] * 1e12)) if w["flops"] else 0.0
    out = {"kernel": stage, "ms": ms, "algorithmic_bytes": w["bytes"], "traffic": measured_traffic(stage, config)}
    if t_ten > t_hbm:
        achieved = w["flops"] / sec / 1e12
        peak = pk["bf16_tflops_sustained"]
        out.update(bound="tensor", achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                   peak_source=f"{pk['source']} bf16 sustained (cuBLAS)")
    else:
        achieved = w["bytes"] / sec / 1e9
        peak = pk["hbm_gbs"]
        out.update(bound="hbm", achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak,
                   peak_source=f"{pk['source']} copy bandwidth")
    if w["flops"]:
        tf = w["flops"] / sec / 1e12
        issued = SLICE_PRODUCTS.get(stage, 10)
        out.update(algorithmic_flops=w["flops"], tensor_tflops=tf,
                   tensor_frac=tf / pk["bf16_tflops_sustained"], slice_products=issued,
                   issued_tensor_frac=issued * tf / pk["bf16_tflops_sustained"])
    return out


# the sources that define each stage's main kernel and its launch (the
# measured traffic of a capture stays valid while these are unchanged)
KERNEL_SOURCES = {
    "S1_collocate": ("tc_gemm.cu", "tc_gemm.cuh", "slices.cuh", "mbarrier.cuh", "thc_abi.cu"),
    "S2_density": ("tc_gemm.cu", "tc_gemm.cuh", "slices.cuh", "mbarrier.cuh", "thc_abi.cu"),
    "S3_kconv": ("kconv.cu", "mbarrier.cuh", "thc_internal.cuh", "thc_abi.cu"),
    "S4a_apply_M": ("tc_gemm.cu", "tc_gemm.cuh", "slices.cuh", "mbarrier.cuh", "thc_abi.cu"),
    "S4b_backproject": ("tc_gemm.cu", "tc_gemm.cuh", "slices.cuh", "mbarrier.cuh", "thc_abi.cu"),
}


def source_hash(stage: str) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2304_05505_gb300", "csrc")
    for f in KERNEL_SOURCES[stage]:
        h.update(f.encode())
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(stage: str, config: str = "C2"):
    """DRAM bytes per launch from the committed ncu capture, if it was taken
    on this workload and on the current sources of that kernel; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path) or stage not in KERNEL_SOURCES:
        return None
    try:
        t = json.load(open(path))
    except Exception:
        return None
    if t.get("config", "C2") != config or t.get("source_hashes", {}).get(stage) != source_hash(stage):
        return None
    v = t.get("per_launch_bytes", {}).get(stage)
    return float(v) if v is not None else None


# ---------------------------------------------------------------------------
# the CPU oracle (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

def oracle_sample_step(p, part: int):
    """1/SAMPLE_FRACTION of one oracle build: steps 1, 2, 4 on a slice of the
    k-points and step 3 (FFT route) on a slice of the P rows."""
    from oracle import thc_oracle as O
    nk = p.X.shape[0]
    f = SAMPLE_FRACTION
    ks = slice(part * nk // f, (part + 1) * nk // f)
    Psi = O.collocate(p.X[ks], p.C[ks])
    D = O.density(Psi)
    P = p.V.shape[1]
    rows = slice(part * P // f, (part + 1) * P // f)
    Dfull = np.zeros((nk, P // f if P % f == 0 else rows.stop - rows.start, P), dtype=np.complex128)
    Dfull[ks] = D[:, rows, :]
    M = O.kconv_fft(Dfull, p.V[:, rows, :], p.cell.mesh)
    Y = O.apply_M(np.ascontiguousarray(M[ks]), Psi)
    O.backproject(np.ascontiguousarray(p.X[ks][:, :, rows]), Y)
    return Y


def cpu_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(int(i.get("num_threads", 1)) for i in info)
    except Exception:
        pass
    return os.cpu_count() or 1


def time_oracle(p, steps: int, warmup: int) -> dict:
    for i in range(warmup):
        oracle_sample_step(p, i % SAMPLE_FRACTION)
    t = []
    for i in range(steps):
        t0 = time.perf_counter()
        oracle_sample_step(p, i % SAMPLE_FRACTION)
        t.append(time.perf_counter() - t0)
    step_s = sum(t) / len(t)
    return {"value": 1.0 / (step_s * SAMPLE_FRACTION), "unit": "builds/s", "cores": cpu_threads(),
            "kind": "oracle", "step_s": step_s,
            "sample": f"each step = 1/{SAMPLE_FRACTION} of one FP64 oracle build (steps 1, 2, 4 on "
                      f"{{N_k/{SAMPLE_FRACTION}}} k-points, FFT-route step 3 on N_P/{SAMPLE_FRACTION} rows); "
                      f"builds/s = 1 / ({SAMPLE_FRACTION} x mean step time); {steps} steps"}


import numpy as np  # noqa: E402  (after sys.path set-up)


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_2304_05505_gb300 import cells
    p = make_inputs(args.config)
    steps = args.steps
    warm = args.warmup
    cb = time_oracle(p, steps, warm)
    line = {"metric": METRIC, "value": cb["value"], "unit": "builds/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": cb["step_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config], "impl": "FP64 CPU oracle (oracle/thc_oracle.py)"},
            "impl": "reference",
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": "builds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_ext(args, thc, d, p, C, KC, ex, dev, stream, world, e0, e1) -> dict:
    """THC_MIXED_EXT on the same inputs: device-timed builds/s and its KC, E_x."""
    import torch
    ee = thc.ExchangeBuild(d, "mixed_ext", device=dev, stream=stream)
    ee.set_collocation(p.X)
    ee.set_kernel(p.V)
    for _ in range(3):
        ee.build(C, KC, ex)
    torch.cuda.synchronize()
    n = max(3, min(args.steps, 20))
    e0.record(stream)
    for _ in range(n):
        ee.build(C, KC, ex)
    e1.record(stream)
    torch.cuda.synchronize()
    ee.sync()
    ms = max_over_ranks(world, e0.elapsed_time(e1)) / n
    thc.thc_profile_begin(ee.ctx, n)        # stage times from a profiled pass
    for _ in range(n):
        ee.build(C, KC, ex)
    torch.cuda.synchronize()
    st, _ = thc.thc_profile_end(ee.ctx)
    out = {"value": world / (ms * 1e-3), "unit": "builds/s", "ms_per_step": ms,
           "stages_ms": dict(zip(thc.STAGES, st)), "hermitian_form": thc.thc_hermitian_kernel(ee.ctx),
           "KC": KC.cpu().numpy(), "Ex": float(ex[0])}
    ee.close()
    del ee
    torch.cuda.empty_cache()
    return out


def run_simt(args, thc, d, p, C, KC, ex, dev, stream, world, e0, e1):
    """The mixed precision on CUDA cores: ms per build, stage ms, KC, E_x."""
    import torch
    es = thc.ExchangeBuild(d, "mixed_simt", device=dev, stream=stream)
    es.set_collocation(p.X)
    es.set_kernel(p.V)
    for _ in range(2):
        es.build(C, KC, ex)
    torch.cuda.synchronize()
    nsimt = max(3, min(args.steps, 10))
    thc.thc_profile_begin(es.ctx, nsimt)
    e0.record(stream)
    for _ in range(nsimt):
        es.build(C, KC, ex)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_simt = max_over_ranks(world, e0.elapsed_time(e1)) / nsimt
    st_simt, _ = thc.thc_profile_end(es.ctx)
    KC_simt = KC.cpu().numpy()
    ex_simt = ex.cpu().numpy().copy()
    es.close()
    del es
    torch.cuda.empty_cache()

    return ms_simt, st_simt, KC_simt, ex_simt


def time_rebuild(p, thc, args) -> dict:
    """The per-iteration kernel rebuild of THC-oo-K at the bench's cell (the
    fit of the interpolation vectors to the current orbitals, their FFT and
    the contraction over G; Algorithm 2's first three steps): device ms per
    step, with the points of the FP64 full-grid pivoted Cholesky (chosen once
    before the SCF loop, as Algorithm 2 chooses its points)."""
    import torch
    from paper_2304_05505_gb300 import cells
    cell = p.cell
    cells.set_accelerator("cuda")
    try:
        Ud = cells.grid_orbitals(cell, p.C, as_tensor=True)
    finally:
        cells.set_accelerator(None)
    t0 = time.perf_counter()
    pts, _ = thc.thc_select_points(Ud, cell.nisdf)
    t_sel = time.perf_counter() - t0
    names = ["metric_B_R_S", "cholesky", "solve", "fft", "contraction"]
    thc.thc_rebuild_kernel(Ud, cell.grid, cell.lattice, cell.mesh, pts, "mixed")   # warm-up
    runs = [thc.thc_rebuild_kernel(Ud, cell.grid, cell.lattice, cell.mesh, pts, "mixed")[1] for _ in range(3)]
    mean = [sum(r[i] for r in runs) / len(runs) for i in range(5)]
    out = {"unit": "ms per rebuild (device time of its steps)", "grid": list(cell.grid), "n_grid": int(np.prod(cell.grid)),
           "points": f"{cell.nisdf} from the FP64 full-grid pivoted Cholesky ({t_sel:.2f} s, once)",
           "mixed": {"ms": sum(mean), "steps_ms": dict(zip(names, mean)),
                     "form": "metric, Cholesky, solve and FFT in FP64; contraction on tcgen05 (FP32 operands, "
                             "3 fp16 slices, 8 products, exact K chunks)"}}
    if args.rebuild_fp64:
        ms = thc.thc_rebuild_kernel(Ud, cell.grid, cell.lattice, cell.mesh, pts, "fp64")[1]
        out["fp64"] = {"ms": sum(ms), "steps_ms": dict(zip(names, ms))}
    del Ud
    torch.cuda.empty_cache()
    return out


def qrep_pairs(mesh) -> int:
    """Number of (q, representative) pairs of a mesh: a q on the zone
    boundary of an even axis has two minimum-image representatives there."""
    n = 1
    for m in mesh:
        n *= sum(2 if (2 * c == m) else 1 for c in range(m))
    return n


def time_vo_gradient(p, thc, fp64_rate: float) -> dict:
    """The THC-oo-K orbital gradient with the kernel's response (Sec. 2.3)
    over all virtual orbitals, FP64, at the bench's cell: device ms per step,
    beside the kernel rebuild it follows in an iteration, and the (q, G)
    contraction that dominates it against the measured FP64 rate."""
    import torch
    from paper_2304_05505_gb300 import cells
    cell = p.cell
    nvir = cell.nbas - cell.nocc
    cells.set_accelerator("cuda")
    try:
        C, Cv = cells.orbital_coefficients(cell, nvir)
        Ud = cells.grid_orbitals(cell, C, as_tensor=True)
        Uvd = cells.grid_orbitals(cell, Cv, as_tensor=True)
    finally:
        cells.set_accelerator(None)
    pts, _ = thc.thc_select_points(Ud, cell.nisdf)
    V, reb = thc.thc_rebuild_kernel(Ud, cell.grid, cell.lattice, cell.mesh, pts, "mixed")
    nk = int(np.prod(cell.mesh))
    names = ["fixed_kernel_D_W_M_Y", "fit_B_R_S_chol_solve_fft", "contraction_qG", "adjoint_dft_solve_Sbar",
             "orbital_T1_T2_G1_G2"]
    h = [(g - 1) // 2 for g in cell.grid]
    nG = (2 * h[0] + 1) * (2 * h[1] + 1) * (2 * h[2] + 1)
    flops = 8.0 * qrep_pairs(cell.mesh) * cell.nisdf ** 2 * nG
    out = {"unit": "ms per gradient (device time of its steps)", "n_vir": nvir, "n_occ": cell.nocc,
           "kernel": "V from the tensor-core kernel rebuild at the FP64 full-grid pivoted-Cholesky points",
           "rebuild_ms": sum(reb), "contraction_flops": flops}
    grads = {}
    for prec in ("fp64", "mixed"):
        thc.thc_vo_gradient(Ud, Uvd, nk, cell.grid, cell.lattice, cell.mesh, pts, V, prec)   # warm-up
        runs = []
        for _ in range(2):
            g, _, _, ms = thc.thc_vo_gradient(Ud, Uvd, nk, cell.grid, cell.lattice, cell.mesh, pts, V, prec)
            runs.append(ms)
        grads[prec] = g
        mean = [sum(r[i] for r in runs) / len(runs) for i in range(5)]
        achieved = flops / (mean[2] * 1e-3) / 1e12
        out[prec] = {"ms": sum(mean), "steps_ms": dict(zip(names, mean)), "ratio_to_rebuild": sum(mean) / sum(reb),
                     "contraction_achieved_tflops": achieved}
    out["fp64"]["contraction_roofline"] = {
        "bound": "fp64", "achieved": out["fp64"]["contraction_achieved_tflops"], "peak": fp64_rate,
        "unit": "TFLOP/s", "frac": out["fp64"]["contraction_achieved_tflops"] / fp64_rate if fp64_rate else None,
        "peak_source": "measured FP64 FMA rate (thc_measure_fp64_rate)"}
    out["mixed"]["form"] = ("(q, G) contraction on tcgen05 (FP32 operands sliced into 3 fp16 slices, 8 products, "
                            "exact K chunks); the other steps FP64")
    out["mixed"]["max_abs_dg_vs_fp64_rel"] = float((grads["mixed"] - grads["fp64"]).abs().max()
                                                   / grads["fp64"].abs().max())
    del Ud, Uvd, V, grads
    torch.cuda.empty_cache()
    return out


def time_aok(d, p, thc, dev, stream) -> dict:
    """The THC-AO-K form of the build (Algorithm 1's K step: the full AO
    exchange matrix K^k = conj(X^k) M^k X^{kT}) on the same inputs: mixed
    builds/s, and one FP64 build."""
    import torch
    out = {"unit": "builds/s", "output": "K^k [N_k][N][N] complex128 and E_x"}
    for prec, nb in (("mixed", 10), ("fp64", 1)):
        eb = thc.ExchangeBuild(d, prec, device=dev, stream=stream)
        eb.set_collocation(p.X)
        eb.set_kernel(p.V)
        C = torch.from_numpy(p.C).to(dev)
        K, ex = eb.build_K(C)
        torch.cuda.synchronize()
        thc.thc_profile_begin(eb.ctx, nb)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nb):
            eb.build_K(C, K, ex)
        e1.record(stream)
        torch.cuda.synchronize()
        eb.sync()
        st, _ = thc.thc_profile_end(eb.ctx)
        ms = e0.elapsed_time(e1) / nb
        out[prec] = {"value": 1e3 / ms, "ms_per_step": ms,
                     "stages_ms": dict(zip(["S1", "S2", "S3", "Z=M X^T", "K=conj(X) Z", "E_x"], st)),
                     "Ex": float(ex[0])}
        eb.close()
        del eb, K, C
        torch.cuda.empty_cache()
    return out


def make_inputs(config: str, kernel: str = "model"):
    """The seeded synthetic cell of `config`, its large products and
    collocations made through torch on the GPU (input generation only).
    kernel "fitted" replaces the model kernel and its sampled points by the
    ones the method feeds the build: the FP64 full-grid pivoted-Cholesky
    points and V^q from the library's kernel rebuild at those points."""
    import torch
    from paper_2304_05505_gb300 import cells
    cells.set_accelerator("cuda" if torch.cuda.is_available() else None)
    try:
        if kernel == "model":
            return cells.make_problem(config)
        from paper_2304_05505_gb300 import thc
        thc.load()
        cell = cells.make_cell(config)
        C = cells.occupied_coefficients(cell)
        U = cells.grid_orbitals(cell, C, as_tensor=True)
        idx, _ = thc.thc_select_points(U, cell.nisdf)
        V, _ = thc.thc_rebuild_kernel(U, cell.grid, cell.lattice, cell.mesh, idx, "mixed")
        del U
        pts = cells.points_from_indices(cell, idx)
        X = cells.bloch_collocation(cell, pts, cells.kmesh_frac(cell.mesh))
        p = cells.Problem(cell, pts, idx, np.zeros(len(idx)), X, C, V.cpu().numpy())
        del V
        torch.cuda.empty_cache()
        return p
    finally:
        cells.set_accelerator(None)


def run_ours(args, world, rank, local):
    import torch
    from paper_2304_05505_gb300 import cells, thc

    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    if not os.path.exists(thc.LIB_PATH):
        raise RuntimeError("libthc.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    thc.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    p = make_inputs(args.config, args.kernel)
    d = p.dims
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    # --- mixed build, device-resident inputs -----------------------------
    eb = thc.ExchangeBuild(d, "mixed", device=dev, stream=stream)
    eb.set_collocation(p.X)
    eb.set_kernel(p.V)
    hermitian = thc.thc_hermitian_kernel(eb.ctx)
    C = torch.from_numpy(p.C).to(dev)
    KC = torch.empty(eb.kc_shape, dtype=torch.complex128, device=dev)
    ex = torch.empty(2, dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        eb.build(C, KC, ex)
    torch.cuda.synchronize()
    barrier(world)
    clk = Clocks(dev.index)
    clk.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(world)
    # the timed builds run as the library runs them unprofiled (one CUDA graph
    # launch each); the per-stage and per-kernel times come from a second,
    # profiled pass of the same builds
    e0.record(stream)
    for _ in range(args.steps):
        eb.build(C, KC, ex)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    ms_total = max_over_ranks(world, e0.elapsed_time(e1))
    eb.sync()   # raises if a device-side wait gave up during the timed builds
    nprof_steps = max(3, min(args.steps, 20))
    thc.thc_profile_begin(eb.ctx, nprof_steps)
    for _ in range(nprof_steps):
        eb.build(C, KC, ex)
    torch.cuda.synchronize()
    stage_ms, nprof = thc.thc_profile_end(eb.ctx)
    kernel_ms = thc.thc_profile_kernels(eb.ctx)
    eb.sync()
    launches = thc.thc_launches_per_build(eb.ctx) * args.steps
    KC_mixed = KC.cpu().numpy()
    ex_mixed = ex.cpu().numpy().copy()
    ms_per = ms_total / args.steps
    value = world * args.steps / (ms_total * 1e-3)

    if args.mixed_only:
        eb.close()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "builds/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per,
                              "mode": "mixed build only", "stages_ms": dict(zip(thc.STAGES, stage_ms)),
                              "kernels_ms": dict(zip(thc.STAGES, kernel_ms)), "clocks": clocks}), flush=True)
        return

    # --- end to end through the host-buffer call ---------------------------
    Ch = torch.from_numpy(p.C).pin_memory()
    KCh = torch.empty(eb.kc_shape, dtype=torch.complex128).pin_memory()
    exh = torch.empty(2, dtype=torch.float64).pin_memory()
    for _ in range(2):
        thc.thc_build_host(eb.ctx, Ch, KCh, exh)
    ne2e = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(ne2e):
        thc.thc_build_host(eb.ctx, Ch, KCh, exh)
    t_e2e = max_over_ranks(world, time.perf_counter() - t0)
    e2e = {"value": world * ne2e / t_e2e, "unit": "builds/s",
           "h2d_bytes_per_step": int(Ch.numel() * 16), "d2h_bytes_per_step": int(KCh.numel() * 16 + 16),
           "steps": ne2e, "api": "thc_build_host (pinned host C in, KC and E_x out)"}
    eb.close()
    del eb
    torch.cuda.empty_cache()

    # --- the extended form (THC_MIXED_EXT): M carried to about 35 bits ---------
    ext = time_ext(args, thc, d, p, C, KC, ex, dev, stream, world, e0, e1) if args.config == "C2" else None

    # --- the same precision on CUDA cores (comparison; the headline cell only) --
    ms_simt, st_simt, KC_simt, ex_simt = None, [0.0] * 6, None, None
    if args.config == "C2":
        ms_simt, st_simt, KC_simt, ex_simt = run_simt(args, thc, d, p, C, KC, ex, dev, stream, world, e0, e1)

    # --- FP64 GPU build -----------------------------------------------------
    e64 = thc.ExchangeBuild(d, "fp64", device=dev, stream=stream)
    e64.set_collocation(p.X)
    e64.set_kernel(p.V)
    e64.build(C, KC, ex)
    torch.cuda.synchronize()
    thc.thc_profile_begin(e64.ctx, args.fp64_steps)
    e0.record(stream)
    for _ in range(args.fp64_steps):
        e64.build(C, KC, ex)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = max_over_ranks(world, e0.elapsed_time(e1)) / args.fp64_steps
    st64, _ = thc.thc_profile_end(e64.ctx)
    KC_64 = KC.cpu().numpy()
    ex_64 = ex.cpu().numpy().copy()
    e64.close()
    fp64_rate = thc.thc_measure_fp64_rate(stream.cuda_stream)

    rebuild = None
    if args.config == "C2" and not args.no_rebuild:
        rebuild = time_rebuild(p, thc, args)
    aok = time_aok(d, p, thc, dev, stream) if args.config == "C2" else None
    vo = time_vo_gradient(p, thc, fp64_rate) if args.vo_gradient else None

    if rank != 0:
        return
    pk = peaks()
    work = stage_work(d, hermitian)
    names = thc.STAGES
    stages = {nm: ms for nm, ms in zip(names, stage_ms)}
    kernels = {nm: ms for nm, ms in zip(names, kernel_ms)}
    dominant = max(kernels, key=kernels.get)
    roof = kernel_roofline(dominant, kernels[dominant], work, pk, args.config)
    roof["name"] = kernel_names(hermitian)[dominant]
    # (S5 fused into S4a's combine moves only its partial sums: no roofline of its own)
    per_kernel = {nm: kernel_roofline(nm, kernels[nm], work, pk, args.config) for nm in names
                  if not (nm == "S5_energy" and s4a_split(d))}


    line = {"metric": METRIC, "value": value, "unit": "builds/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp16-slices/f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config],
                       "precision": "mixed: S1/S2/S4a/S4b tcgen05 GEMMs on 3-slice fixed-point fp16 operands "
                                    "(8+11+11 bits; 6, 6, 8, 8 slice products; exact leading sums, FP32 "
                                    "remainders), X and M sliced inside the GEMMs, S3 FP32, E_x FP64 sum",
                       "kernel_source": ("model kernel V^q (Gaussian-smeared point deltas), density-sampled points"
                                         if args.kernel == "model" else
                                         "ISDF-fitted V^q (kernel rebuild, tcgen05 contraction) at the FP64 "
                                         "full-grid pivoted-Cholesky points"),
                       "hermitian_form": hermitian,
                       "l2": "inputs larger than L2 (prepared kernel complex64 > 700 MB, X FP32 > 260 MB)",
                       "parallelism": f"{world} independent builds (one per GPU)"},
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
            "stages_ms": stages, "kernels_ms": kernels,
            "kernel_roofline": {k: {"frac": v["frac"], "bound": v["bound"], "achieved": v["achieved"],
                                    "unit": v["unit"], **({"issued_tensor_frac": v["issued_tensor_frac"]}
                                                          if "issued_tensor_frac" in v else {})}
                                for k, v in per_kernel.items()},
            "fp64_gpu": {"value": world / (ms64 * 1e-3), "unit": "builds/s", "ms_per_step": ms64,
                         "stages_ms": {nm: ms for nm, ms in zip(names, st64)},
                         "roofline": fp64_roofline(d, dict(zip(names, st64)), fp64_rate, pk)},
            "Ex_mixed": float(ex_mixed[0]), "Ex_fp64_gpu": float(ex_64[0])}
    if rebuild is not None:
        line["kernel_rebuild"] = rebuild
    if aok is not None:
        line["thc_ao_k"] = aok
    if vo is not None:
        line["vo_gradient"] = vo
    if ext is not None:
        line["mixed_ext"] = {k: v for k, v in ext.items() if k not in ("KC", "Ex")}
    if ms_simt is not None:
        line["mixed_cuda_cores"] = {"value": world / (ms_simt * 1e-3), "unit": "builds/s", "ms_per_step": ms_simt,
                                    "stages_ms": {nm: ms for nm, ms in zip(names, st_simt)}}
    if not args.no_oracle:
        from oracle import thc_oracle as O
        t0 = time.perf_counter()
        if args.config == "C2":
            ref = O.build(p.X, p.C, p.V, p.cell.mesh, route="fft")
        else:   # D and M of the largest cell do not fit in host memory whole
            ref = O.build_rowblocks(p.X, p.C, p.V, p.cell.mesh)
        t_full = time.perf_counter() - t0
        line["accuracy_vs_oracle"] = {
            "mixed": {"max_abs_dKC": float(np.abs(KC_mixed - ref["KC"]).max()),
                      "abs_dEx": abs(float(ex_mixed[0]) - ref["Ex"])},
            "fp64_gpu": {"max_abs_dKC": float(np.abs(KC_64 - ref["KC"]).max()),
                         "abs_dEx": abs(float(ex_64[0]) - ref["Ex"])},
            "Ex_oracle": ref["Ex"], "oracle_full_build_s": t_full}
        if ext is not None:
            line["accuracy_vs_oracle"]["mixed_ext"] = {
                "max_abs_dKC": float(np.abs(ext["KC"] - ref["KC"]).max()), "abs_dEx": abs(ext["Ex"] - ref["Ex"])}
        if KC_simt is not None:
            line["accuracy_vs_oracle"]["mixed_cuda_cores"] = {
                "max_abs_dKC": float(np.abs(KC_simt - ref["KC"]).max()), "abs_dEx": abs(float(ex_simt[0]) - ref["Ex"])}
        cb = time_oracle(p, args.cpu_samples, 1)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    import torch
    world, rank, local = dist_setup(args.gpus)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
