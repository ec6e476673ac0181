"""The benchmark's roofline arithmetic on the host: the useful work of one H_eff.theta
(the (L.theta).W1.W2.R order of Sec. 4.2), the derived FP64 peak, the fraction the line
reports, and the DRAM-traffic table, whose entries must still belong to the kernels'
current sources (an entry whose source file changed since its capture reads as null).
No GPU."""
import hashlib
import os

import pytest

import bench

pytestmark = pytest.mark.cpu


def test_matvec_work_counts_the_two_contraction_orders():
    # chi = 256, d = 4, D = 4: 8 (2 D d^2 chi^3 + 2 D^2 d^3 chi^2) real FLOPs
    chi, d, D = 256, 4, 4
    assert bench.FLOP_MATVEC == 8 * (2 * D * d * d * chi ** 3 + 2 * D * D * d ** 3 * chi ** 2)
    assert abs(bench.FLOP_MATVEC - 18.25e9) < 0.01e9


def test_fp64_peak_is_sms_times_clock_times_two_fmas():
    assert bench.fp64_peak_gflops({"sm_max_mhz": 2070.0}) == pytest.approx(152 * 2070e6 * 4 / 1e9)


def test_roofline_fraction_is_achieved_over_peak():
    peaks = {"hbm_gbs": 6791.7, "bf16_tflops": 1927.7, "sm_max_mhz": 2070.0}
    # two launches of 2.9 GFLOP in 27.7 ms (the FP64 class of the tridiagonal reduction)
    r = bench.roofline("heig_tridiag", 27.7, 2, 2 * 2.896e9, peaks, "measured")
    assert r["bound"] == "alu" and r["unit"] == "GFLOP/s"
    assert r["achieved"] == pytest.approx(2 * 2.896e9 / 27.7e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.fp64_peak_gflops(peaks))
    h = bench.roofline("multiaxpy32", 10.0, 176, 176 * 2.9e8, peaks, "measured")
    assert h["bound"] == "hbm" and h["frac"] == pytest.approx(h["achieved"] / 6791.7)


@pytest.mark.parametrize("cls", sorted(bench.TRAFFIC))
def test_traffic_entries_belong_to_current_sources(cls):
    nbytes, src, sha, _ = bench.TRAFFIC[cls]
    path = os.path.join(bench.ROOT, "paper_1610_02244_gb300", "csrc", src)
    with open(path, "rb") as f:
        cur = hashlib.sha256(f.read()).hexdigest()[:16]
    assert cur == sha, f"{cls}: {src} changed since its ncu capture; capture again"
    assert bench.traffic_for(cls) == nbytes > 0
