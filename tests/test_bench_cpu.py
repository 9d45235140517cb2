"""Host logic of bench.py (no GPU): the algorithmic work of each stage, the
roofline arithmetic and the bookkeeping of the measured DRAM traffic."""
import json
import os

import pytest

import bench

C2 = dict(n1=4, n2=4, n3=4, nbas=432, nocc=60, nisdf=1200)


def test_stage_work_counts():
    nk, N, n, P = 64, 432, 60, 1200
    full = bench.stage_work(C2, hermitian=False)
    herm = bench.stage_work(C2, hermitian=True)
    # S3 moves D and Vh in and M out, complex64; the Hermitian form reads the
    # P (P + 1) / 2 elements on and above the diagonal of D and Vh
    assert full["S3_kconv"]["bytes"] == 3 * 8 * nk * P * P
    assert herm["S3_kconv"]["bytes"] == 8 * nk * (P * (P + 1) + P * P)
    # S2 forms all of D^k = Psi Psi^H, or its upper part
    # S2 multiplies only the tiles that reach the diagonal in both forms
    assert full["S2_density"]["flops"] == herm["S2_density"]["flops"] == 8 * nk * n * P * (P + 1) / 2
    # the stages the form does not touch are the same
    for st in ("S1_collocate", "S4a_apply_M", "S4b_backproject", "S5_energy"):
        assert full[st] == herm[st]
    assert full["S4a_apply_M"]["flops"] == 8 * nk * P * P * n
    assert full["S4b_backproject"]["bytes"] == 8 * nk * (N * P + P * n) + 16 * nk * N * n


def test_roofline_arithmetic():
    pk = dict(hbm_gbs=6000.0, bf16_tflops=2000.0, bf16_tflops_sustained=1500.0, sm_max_mhz=2070.0,
              source="test")
    work = bench.stage_work(C2, hermitian=True)
    r = bench.kernel_roofline("S3_kconv", 0.5, work, pk)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(work["S3_kconv"]["bytes"] / 0.5e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)
    g = bench.kernel_roofline("S4a_apply_M", 0.4, work, pk)
    # at n = 60 the bytes bind, not the flops; the issued tensor fraction
    # counts the 8 slice products per real product of S4a
    assert g["bound"] == "hbm"
    tf = work["S4a_apply_M"]["flops"] / 0.4e-3 / 1e12
    assert g["tensor_tflops"] == pytest.approx(tf)
    assert g["issued_tensor_frac"] == pytest.approx(8 * tf / 1500.0)
    s2 = bench.kernel_roofline("S2_density", 0.2, work, pk)
    assert s2["slice_products"] == 6


def test_measured_traffic_follows_the_sources(monkeypatch, tmp_path):
    # a capture counts for a stage only while that stage's sources hash as
    # they did when it was taken
    os.makedirs(tmp_path / "profiles")
    stages = list(bench.KERNEL_SOURCES)
    t = {"source_hashes": {st: "h-" + st for st in stages},
         "per_launch_bytes": {st: 1000 + i for i, st in enumerate(stages)}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(t))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda st: "h-" + st)
    for i, st in enumerate(stages):
        assert bench.measured_traffic(st) == 1000 + i
    monkeypatch.setattr(bench, "source_hash", lambda st: "changed" if st == "S3_kconv" else "h-" + st)
    assert bench.measured_traffic("S3_kconv") is None
    assert bench.measured_traffic("S4a_apply_M") == 1000 + stages.index("S4a_apply_M")
    assert bench.measured_traffic("S5_energy") is None          # no capture for S5
    # a capture counts only for the workload it was taken on
    assert bench.measured_traffic("S4a_apply_M", "C3") is None


def test_source_hash_covers_the_kernel_files():
    # every file a stage's hash names exists, and the hash changes with them
    csrc = os.path.join(bench.ROOT, "paper_2304_05505_gb300", "csrc")
    for st, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(csrc, f)), (st, f)
        assert len(bench.source_hash(st)) == 16
    assert bench.source_hash("S1_collocate") == bench.source_hash("S4a_apply_M")   # the same GEMM sources
    assert bench.source_hash("S1_collocate") != bench.source_hash("S3_kconv")


def test_fp64_roofline_arithmetic():
    # the FP64 build computes all of D; its GEMMs are reported against the
    # FP64 rate, its convolution (complex128) against the copy bandwidth
    pk = dict(hbm_gbs=6000.0)
    st = {"S1_collocate": 10.0, "S2_density": 40.0, "S3_kconv": 5.0, "S4a_apply_M": 40.0, "S4b_backproject": 10.0}
    r = bench.fp64_roofline(C2, st, 1.25, pk)
    nk, N, n, P = 64, 432, 60, 1200
    assert r["S2_density"]["achieved_tflops"] == pytest.approx(8 * nk * P * P * n / 40e-3 / 1e12)
    assert r["S1_collocate"]["frac"] == pytest.approx(8 * nk * P * n * N / 10e-3 / 1e12 / 1.25)
    assert r["S3_kconv"]["achieved_gbs"] == pytest.approx(16 * nk * 3 * P * P / 5e-3 / 1e9)


def test_s4a_split_rule():
    # S4a's K is 2 N_P reals: split (and, n_occ even, carrying S5's partial sums) above 1024
    assert bench.s4a_split(C2)
    assert not bench.s4a_split(dict(C2, nisdf=512))
    assert bench.s4a_split(dict(C2, nisdf=513))
    assert not bench.s4a_split(dict(C2, nocc=61))      # odd n_occ: the combine kernel, S5 whole


@pytest.mark.parametrize("mesh", [(4, 4, 4), (3, 3, 3), (2, 2, 1), (6, 1, 3)])
def test_qrep_pairs_counts_the_representatives(mesh):
    """The (q, representative) pairs the vo-gradient contraction runs over are
    the setup oracle's minimum-image representatives of every q."""
    from oracle import setup_oracle as S
    from oracle import thc_oracle as O
    n = sum(len(S.representatives(co, mesh)) for co in O.mesh_coords(mesh))
    assert bench.qrep_pairs(mesh) == n
