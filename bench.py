#!/usr/bin/env python
"""Benchmark of the two-site update at the H_eff.theta micro-benchmark shape.

Workload (synthetic, seeded): left/right environments 256 x 4 x 256 with the channel
structure of DMRG environments of the Bose-Hubbard MPO (identity channel, a gapped block
Hamiltonian in its eigenbasis, a Gaussian boundary operator and its adjoint), the
Bose-Hubbard MPO tensor (d = 4, D = 4, J = 1, U = 2, mu = 0), site tensors A, B of
256 x 4 x 256 with i.i.d. complex Gaussian entries.

One step = one two-site DMRG update on that data, every row of the hot path:
  theta = A.B (a1); Lanczos on H_eff to convergence (tolerance 1e-12, 32 Krylov vectors
  then restart, at most 300 matvecs), FP64 vectors, CGS2 (a3, a4), and with split-TF32
  matvecs one FP64 matvec for the Rayleigh quotient and the true residual (a9); truncated
  SVD of theta as a 1024 x 1024 matrix to chi = 256, S renormalised (a5, a6, a7);
  left-environment growth with the new site tensor (a8).
metric: useful H_eff.theta FLOP/s of the update = (matvecs x 18.25 GFLOP) / update time;
the same line carries the plain FP64 path's update time on the same data, the energy and
state of both against the FP64 CPU oracle's converged update on the same inputs, and the
DMRG s/sweep of the 8-site chain (mixed and FP64).
"""
from __future__ import annotations

import argparse
import faulthandler
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CHI, D_PHYS, D_MPO = 256, 4, 4
J, U, MU = 1.0, 2.0, 0.0
KRYLOV = 32
MAXIT = 300
LZ_TOL = 1e-12
CHI_MAX = 256
METRIC = "DMRG s/sweep & H_eff·θ TFLOP/s, mixed vs FP64 on GB300 at |ΔE|≤1e-10"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
TF32_PER_BF16 = 1.1 / 2.25     # nominal dense ratio (profiling recipe table)
FP64_FLOP_PER_CLK_SM = 4.0     # 2 DFMA per clock per SM on GB300 (a DFMA-only probe on the
                               # pool measured 1.256 TFLOP/s at 2070 MHz over 152 SMs)
N_SM = 152


def fp64_peak_gflops(peaks):
    """FP64 ALU peak derived from the SM count and the maximum SM clock."""
    return N_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6 * FP64_FLOP_PER_CLK_SM / 1e9


def matvec_cmacs(chl, d, D, chr_):
    """Complex multiply-adds of one H_eff.theta in the (L.theta).W1.W2.R order."""
    return D * d * d * chl * chr_ * (chl + chr_) + 2 * D * D * d ** 3 * chl * chr_


FLOP_MATVEC = 8 * matvec_cmacs(CHI, D_PHYS, D_MPO, CHI)   # 18.25e9
N_THETA = CHI * D_PHYS * D_PHYS * CHI


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return PEAKS_FALLBACK, "fallback"


def synth_inputs(seed=0):
    """Seeded draws for one update (generator only: no product code, no oracle)."""
    from paper_1610_02244_gb300 import synth
    g = synth.rng(seed)
    Le = synth.block_env(g, CHI, "left")
    Re = synth.block_env(g, CHI, "right")
    A = synth.complex_gaussian(g, (CHI, D_PHYS, CHI))
    B = synth.complex_gaussian(g, (CHI, D_PHYS, CHI))
    return {"L": Le, "R": Re, "A": A, "B": B}


def oracle_mpo_site():
    """A bulk Bose-Hubbard MPO tensor from the oracle's own construction (Eq. 2)."""
    from oracle import bose_hubbard as bh
    Ws, _, _ = bh.bh_mpo(3, D_PHYS - 1, J, U, MU)
    return Ws[1]


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def dist_max(x: float, ws: int) -> float:
    """Maximum of x over the ranks (the slowest replica sets the job time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- the oracle (CPU)
def oracle_update(inp, W, max_matvec=MAXIT):
    """The FP64 CPU oracle's two-site update on the same inputs, every phase timed:
    theta = A.B, its own Lanczos (CGS twice, the same stopping rule) for at most
    max_matvec matvecs, the truncated SVD of theta, the left-environment growth."""
    from oracle import contract as oc
    from oracle import lanczos as olz
    from oracle import svd as osvd
    Le, Re, A, B = inp["L"], inp["R"], inp["A"], inp["B"]
    t = {}
    t0 = time.perf_counter()
    th = oc.theta_form(A, B)
    t["theta"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    E, x, nmv, resid, conv = olz.lanczos_ground(lambda v: oc.heff_apply(Le, W, W, Re, v), th,
                                                tol=LZ_TOL, krylov_cap=KRYLOV,
                                                max_matvec=max_matvec)
    t["lanczos"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    Uo, S, Vh, bq, info = osvd.svd_truncate(x.reshape(CHI * D_PHYS, -1),
                                            np.zeros(CHI * D_PHYS, np.int64),
                                            np.zeros(CHI * D_PHYS, np.int64),
                                            osvd.TruncParams(chi_max=CHI_MAX))
    t["svd"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    oc.env_left(Le, W, Uo.reshape(CHI, D_PHYS, -1))
    t["env"] = time.perf_counter() - t0
    return {"t_update": sum(t.values()), "t": t, "E": E, "x": x, "n_matvec": nmv,
            "resid": resid, "converged": bool(conv)}


def threads_used():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max((i.get("num_threads", 1) for i in info), default=os.cpu_count())
    except Exception:
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args, ws, rank):
    """The oracle as it stands on the host cores: each step a measured, bounded sample of
    the update (theta, the first m matvecs of its Lanczos solve, SVD, environment growth),
    m chosen from the warm-up so that the whole run ends within a few minutes; the rate is
    the matvec FLOPs done over the time taken, nothing scaled."""
    if rank != 0:
        return 0
    inp = synth_inputs(0)
    W = oracle_mpo_site()
    cal = oracle_update(inp, W, max_matvec=4)
    # later Krylov steps orthogonalise against more vectors (up to 32): the mean cost of a
    # step over a restart cycle is about 1.6 times that of the first four
    t_mv = 1.6 * cal["t"]["lanczos"] / max(1, cal["n_matvec"])
    fixed = cal["t"]["theta"] + cal["t"]["svd"] + cal["t"]["env"]
    budget = min(30.0, max(3.0, 150.0 / max(1, args.steps + args.warmup)))
    m = int(min(MAXIT, max(1, (budget - fixed) / max(t_mv, 1e-6))))
    for _ in range(max(0, args.warmup - 1)):
        oracle_update(inp, W, max_matvec=m)
    vals, times, nmvs = [], [], []
    for _ in range(args.steps):
        s = oracle_update(inp, W, max_matvec=m)
        vals.append(s["n_matvec"] * FLOP_MATVEC / s["t_update"] / 1e12)
        times.append(s["t_update"])
        nmvs.append(s["n_matvec"])
    v = statistics.median(vals)
    sample = (f"theta + the first {m} matvecs of the oracle's Lanczos solve (a converged "
              f"solve takes ~150) + SVD + environment growth, timed as run")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, "f64"),
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": threads_used(),
                             "kind": "oracle", "sample": sample},
            "matvecs_per_step": statistics.median(nmvs),
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_dict(args, dtype):
    return {"workload": "two-site DMRG update, Bose-Hubbard MPO, chi=256 d=4 D=4 "
                        "(L,R 256x4x256 with DMRG channel structure, theta 256x4x4x256), "
                        "Lanczos to 1e-12 (32 Krylov vectors, restart, <=300 matvecs), "
                        "SVD to chi=256",
            "chi": CHI, "d": D_PHYS, "D": D_MPO, "krylov_cap": KRYLOV, "lanczos_tol": LZ_TOL,
            "lanczos_maxit": MAXIT, "chi_max": CHI_MAX,
            "precision": args.precision, "matvec_dtype": dtype,
            "fp64_gemm": getattr(args, "fp64_gemm", "fma"),
            "l2": "inputs larger than L2 (Krylov basis 32 x 16 MiB per step)"}


# ---------------------------------------------------------------- DMRG (8-site chain)
DMRG_L, DMRG_N, DMRG_NMAX, DMRG_U, DMRG_CHI, DMRG_SWEEPS = 8, 8, 3, 2.0, 32, 4


def dmrg_sweeps(ctx, tnt, A, q, mpo, prec, n):
    """n independent 4-sweep runs from the seeded start in one precision: ms per sweep
    (CUDA events on the library's stream) and the last run's final sweep statistics."""
    import torch
    ctx.set_params(chi_max=DMRG_CHI, precision=prec, lanczos_tol=LZ_TOL, lanczos_maxit=MAXIT,
                   krylov_cap=KRYLOV)
    ctx.set_fp64_gemm(tnt.TNT_FP64_GEMM_TC if prec == tnt.TNT_PREC_MIXED else tnt.TNT_FP64_GEMM_FMA)
    states = [ctx.mps_create(A, q, chi_cap=DMRG_CHI) for _ in range(n)]
    runs = [ctx.dmrg_create(m, mpo) for m in states]
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    last = None
    for r in runs:
        for _ in range(DMRG_SWEEPS):
            last = r.sweep()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / (n * DMRG_SWEEPS), last


def dmrg_oracle(A, q):
    """The oracle's 4-sweep run of the 8-site chain from the same start, timed, and the
    exact ground-state energy of the N = 8 sector by exact diagonalisation."""
    from oracle import bose_hubbard as bh
    from oracle import dmrg as od
    from oracle import ed
    Ws, l, r = bh.bh_mpo(DMRG_L, DMRG_NMAX, J, DMRG_U)
    t0 = time.perf_counter()
    _, _, hist = od.dmrg(A, q, Ws, l, r, DMRG_CHI, DMRG_SWEEPS)
    t_or = (time.perf_counter() - t0) / DMRG_SWEEPS
    Es, _ = ed.lowest(ed.hamiltonian(DMRG_L, DMRG_N, DMRG_NMAX, J, DMRG_U, MU), 1)
    return t_or, hist[-1]["E"], float(Es[0])


# ---------------------------------------------------------------- our arm
def run_ours(args, ws, rank, local):
    import torch

    from paper_1610_02244_gb300 import build as b
    from paper_1610_02244_gb300 import synth, tnt
    b.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = tnt.Context(local)
    prec = tnt.TNT_PREC_MIXED if args.precision == "mixed" else tnt.TNT_PREC_FP64

    def set_prec(pr):
        ctx.set_params(chi_max=CHI_MAX, krylov_cap=KRYLOV, lanczos_maxit=MAXIT, precision=pr,
                       lanczos_tol=LZ_TOL)
        ctx.set_fp64_gemm(tnt.TNT_FP64_GEMM_TC if pr == tnt.TNT_PREC_MIXED
                          else tnt.TNT_FP64_GEMM_FMA)

    set_prec(prec)
    inp = synth_inputs(rank)
    inp_dev = dict(inp, W=tnt.bh_mpo_site(D_PHYS - 1, J, U, MU, 0.0, 2.0, 0.0))
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in inp_dev.items()}
    theta = torch.empty((CHI, D_PHYS, D_PHYS, CHI), dtype=torch.complex128, device=dev)
    Lnew = torch.empty((CHI, D_MPO, CHI), dtype=torch.complex128, device=dev)
    stats = {}

    def step(tin):
        ctx.theta_form(tin["A"], tin["B"], out=theta)
        res = ctx.lanczos_ground(tin["L"], tin["W"], tin["W"], tin["R"], theta)
        Uo, X, S, bq, info = ctx.svd_trunc(theta.view(CHI * D_PHYS, D_PHYS * CHI),
                                           side=tnt.TNT_SVD_LEFT, renorm=True)
        k = info["chi"]
        ctx.env_left(tin["L"], tin["W"], Uo.reshape(CHI, D_PHYS, k),
                     out=Lnew if k == CHI else None)
        stats["res"], stats["info"] = res, info
        return Uo, X, res

    st = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        step(t)
    torch.cuda.synchronize()

    # phase breakdown (one untimed step, events on the library's stream); the converged
    # eigenvector of the mixed solve is kept for the comparison with the oracle
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    ev[0].record(st)
    ctx.theta_form(t["A"], t["B"], out=theta)
    ev[1].record(st)
    res = ctx.lanczos_ground(t["L"], t["W"], t["W"], t["R"], theta)
    ev[2].record(st)
    x_main = theta.cpu().numpy()
    Uo, X, S, bq, info = ctx.svd_trunc(theta.view(CHI * D_PHYS, D_PHYS * CHI),
                                       side=tnt.TNT_SVD_LEFT, renorm=True)
    ev[3].record(st)
    ctx.env_left(t["L"], t["W"], Uo.reshape(CHI, D_PHYS, info["chi"]))
    ev[4].record(st)
    torch.cuda.synchronize()
    res_main = res
    phases = {n: ev[i].elapsed_time(ev[i + 1])
              for i, n in enumerate(["theta_ms", "lanczos_ms", "svd_ms", "env_ms"])}

    # dominant kernel class by summed device time over one step
    per_class = {}
    for cls in CLASSES:
        ctx.profile_select(cls)
        step(t)
        per_class[cls] = ctx.profile_read()
    ctx.profile_select(None)
    dom = max(per_class, key=lambda k: per_class[k][0])

    # timed region: K steps, dominant class timed live with events on the same stream
    ctx.profile_select(dom)
    ctx.profile_read()
    launches0 = ctx.launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nmv = 0
    with ClockSampler(local) as clk:
        e0.record(st)
        for _ in range(args.steps):
            step(t)
            nmv += stats["res"]["n_matvec"]
        e1.record(st)
        torch.cuda.synchronize()
    barrier(ws)
    ms_total = e0.elapsed_time(e1)
    dom_ms, dom_n, dom_work = ctx.profile_read()
    ctx.profile_select(None)
    launches = ctx.launch_count() - launches0
    ms_step = dist_max(ms_total / args.steps, ws)
    flops_step = nmv / args.steps * FLOP_MATVEC
    value = ws * flops_step / (ms_step * 1e-3) / 1e12

    # end to end through the public API with host buffers (pinned), copies inside
    hin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in inp_dev.items()}
    hout_u = torch.empty((CHI * D_PHYS * CHI,), dtype=torch.complex128).pin_memory()
    hout_x = torch.empty((CHI * D_PHYS * CHI,), dtype=torch.complex128).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in hin.values())
    d2h = 2 * hout_u.numel() * hout_u.element_size() + 8
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    e2e_nmv = 0
    for _ in range(e2e_steps):
        tin = {k: v.to(dev, non_blocking=True) for k, v in hin.items()}
        Uo, X, r = step(tin)
        e2e_nmv += r["n_matvec"]
        hout_u[: Uo.numel()].copy_(Uo.reshape(-1), non_blocking=True)
        hout_x[: X.numel()].copy_(X.reshape(-1), non_blocking=True)
        torch.cuda.synchronize()
        _ = r["E_rq"]
    t_e2e = dist_max((time.perf_counter() - t0) / e2e_steps, ws)
    e2e = ws * (e2e_nmv / e2e_steps) * FLOP_MATVEC / t_e2e / 1e12

    # the other precision on the same data (the plain FP64 path: FP64 FMA everywhere)
    other = tnt.TNT_PREC_FP64 if prec == tnt.TNT_PREC_MIXED else tnt.TNT_PREC_MIXED
    set_prec(other)
    step(t)
    n_other = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    e0.record(st)
    nmv_o = 0
    for _ in range(n_other):
        step(t)
        nmv_o += stats["res"]["n_matvec"]
    e1.record(st)
    torch.cuda.synchronize()
    ms_other = dist_max(e0.elapsed_time(e1) / n_other, ws)
    ctx.theta_form(t["A"], t["B"], out=theta)
    res_other = ctx.lanczos_ground(t["L"], t["W"], t["W"], t["R"], theta)
    x_other = theta.cpu().numpy()
    set_prec(prec)
    name, oname = ("mixed", "fp64") if prec == tnt.TNT_PREC_MIXED else ("fp64", "mixed")
    upd = {name: {"s_per_update": ms_step / 1e3, "matvecs": nmv / args.steps,
                  "tflops_useful": value / ws, "E": res_main["E_rq"],
                  "resid_fp64": res_main["resid_fp64"], "converged": res_main["converged"]},
           oname: {"s_per_update": ms_other / 1e3, "matvecs": nmv_o / n_other,
                   "tflops_useful": nmv_o / n_other * FLOP_MATVEC / (ms_other * 1e-3) / 1e12,
                   "E": res_other["E_rq"], "resid_fp64": res_other["resid_fp64"],
                   "converged": res_other["converged"]}}
    xs = {name: x_main, oname: x_other}

    # DMRG of the 8-site chain (s/sweep, mixed and FP64)
    A8, q8 = synth.random_charged_mps(synth.rng(0), DMRG_L, DMRG_NMAX + 1, DMRG_N, DMRG_CHI)
    mpo8 = ctx.mpo_bose_hubbard(DMRG_L, DMRG_NMAX, J, DMRG_U)
    dmrg_sweeps(ctx, tnt, A8, q8, mpo8, tnt.TNT_PREC_MIXED, 1)
    ms_sw_mixed, sw_mixed = dmrg_sweeps(ctx, tnt, A8, q8, mpo8, tnt.TNT_PREC_MIXED, 3)
    ms_sw_fp64, sw_fp64 = dmrg_sweeps(ctx, tnt, A8, q8, mpo8, tnt.TNT_PREC_FP64, 2)
    set_prec(prec)
    dmrg = {"workload": "Bose-Hubbard L=8 N=8 n_max=3 J=1 U=2 chi_max=32, 4 two-site sweeps "
                        "from a seeded random MPS in the N=8 blocks",
            "s_per_sweep": {"mixed": dist_max(ms_sw_mixed, ws) * 1e-3,
                            "fp64": dist_max(ms_sw_fp64, ws) * 1e-3},
            "E": {"mixed": sw_mixed["E"], "fp64": sw_fp64["E"]}}

    line = None
    if rank == 0:
        peaks, src = load_peaks()
        roof = roofline(dom, dom_ms, dom_n, dom_work, peaks, src)
        kernel_roofs = {k: roofline(k, *v, peaks, src) for k, v in per_class.items() if v[1] > 0}
        cpu = None
        acc = None
        if ws == 1 and not args.no_cpu_baseline:
            o = oracle_update(inp, oracle_mpo_site())
            cpu = {"value": o["n_matvec"] * FLOP_MATVEC / o["t_update"] / 1e12,
                   "unit": "TFLOP/s", "cores": threads_used(), "kind": "oracle",
                   "sample": "one whole converged update on the same inputs (theta, "
                             f"{o['n_matvec']} Lanczos matvecs, SVD, environment growth)",
                   "s_per_update": o["t_update"], "phases_s": o["t"],
                   "converged": o["converged"]}
            acc = {"E_oracle": o["E"]}
            xo = o["x"].reshape(-1)
            for k in upd:
                xk = xs[k].reshape(-1)
                ov = abs(np.vdot(xo, xk)) / (np.linalg.norm(xo) * np.linalg.norm(xk))
                acc[k] = {"dE_rel": abs(upd[k]["E"] - o["E"]) / abs(o["E"]),
                          "one_minus_overlap": 1.0 - ov}
            t_or, E_or, E_ed = dmrg_oracle(A8, q8)
            dmrg["oracle_s_per_sweep"] = t_or
            dmrg["oracle_cores"] = threads_used()
            dmrg["E_oracle"] = E_or
            dmrg["E_exact"] = E_ed
            dmrg["dE_rel_vs_oracle"] = {k: abs(v - E_or) / abs(E_or) for k, v in dmrg["E"].items()}
            dmrg["dE_rel_vs_exact"] = {k: abs(v - E_ed) / abs(E_ed) for k, v in dmrg["E"].items()}
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if prec == tnt.TNT_PREC_FP64 else "tf32x3+f64",
                "data": "synthetic", "config": config_dict(args, "f64" if prec == 0 else "tf32x3"),
                "update": upd, "fp64_over_mixed_time": upd["fp64"]["s_per_update"] / upd["mixed"]["s_per_update"],
                "accuracy_vs_oracle": acc, "dmrg_chain8": dmrg,
                "s_per_update": ms_step / 1e3, "matvecs_per_step": nmv / args.steps,
                "phases_ms": phases, "kernel_ms_per_step": {k: v[0] for k, v in per_class.items()},
                "kernel_rooflines": kernel_roofs,
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "clocks": clk.summary(),
                "lanczos": {k: stats["res"][k] for k in ("E", "E_rq", "resid_fp64", "n_matvec",
                                                         "converged")},
                "svd": {k: stats["info"][k] for k in ("chi", "err", "disc")}}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


# kernel class -> (bound, what its work counts).  The library sums, per launch, the
# algorithmic work: useful complex-product FLOPs (8 M N K; the split-TF32 repeats are not
# counted) for the GEMM classes, FP64 FLOPs for the eigensolver and for the FP64 Lanczos dot
# products and updates (on GB300 their 4 FP64 FMAs per complex element outrun HBM), bytes
# read plus written for the memory-bound kernels (conversions, and the FP32-arithmetic
# Gram-Schmidt passes of the split-TF32 phase).
CLASSES = {
    "cgemm_tf32x3": ("tensor", "flop"), "zgemm_f64": ("alu", "flop"), "op_apply": ("alu", "flop"),
    "op_mixed": ("hbm", "byte"), "split_theta": ("hbm", "byte"), "multidot": ("alu", "flop"),
    "multiaxpy": ("alu", "flop"), "multidot_cond": ("alu", None), "multiaxpy_cond": ("alu", None),
    "multidot32": ("hbm", "byte"), "multiaxpy32": ("hbm", "byte"), "heig_tridiag": ("alu", "flop"),
    "heig_tridiag_eig": ("alu", None), "heig_backtransform": ("alu", "flop"),
    "cgemm_grouped": ("tensor", "flop"), "zgemm_grouped": ("alu", "flop"),
    "u1_wop": ("hbm", "byte"), "u1_pack_theta": ("hbm", "byte"), "u1_gather": ("hbm", "byte"),
    "oz_gemm": ("tensor_fp64", "flop"), "oz_slice": ("hbm", "byte"),
}
OZ_TENSOR_PER_USEFUL = 45.0  # slice pairs per complex product: 45 x 4 real MMAs / (8 / 2) FLOPs


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu
# capture per kernel class, valid while the class's source file is unchanged: class ->
# (bytes per launch, source file under csrc/, sha256 prefix of that file, capture).
TRAFFIC = {
    # both launches of one matvec (T1 = L theta: 22.78 + 1.90 MB; y = T3 R^T: 71.63 + 3.22 MB),
    # averaged: profiles/cgemm_tf32x3_heff_cfg2.md (the key follows the file; since the
    # capture only the gather kernel in it changed)
    "cgemm_tf32x3": (49.76e6, "tc_mixed.cu", "8430c4ff3cf17339", "ncu, bench.py update step"),
    # two launches per update: the 1024-row Gram block (16.93 MB, ncu; the matrix read once)
    # and the ~231-row tail block (its entries x the same 16.1 B per entry: 0.86 MB), averaged:
    # profiles/tridiag_rows_gram1024.md
    "heig_tridiag": (8.9e6, "heig.cu", "6808812dfa05a999", "ncu, svd_large_block_cfg2_shape"),
}


def traffic_for(cls):
    e = TRAFFIC.get(cls)
    if not e:
        return None
    nbytes, src, sha, _ = e
    path = os.path.join(ROOT, "paper_1610_02244_gb300", "csrc", src)
    with open(path, "rb") as f:
        cur = hashlib.sha256(f.read()).hexdigest()[:16]
    return nbytes if cur == sha else None


def roofline(cls, ms, n, work, peaks, src):
    """Roofline of one kernel class: algorithmic work per launch / mean launch duration."""
    if n == 0 or ms <= 0:
        return None
    bound, unit = CLASSES[cls]
    secs = ms * 1e-3
    bf16 = peaks.get("bf16_tflops", 1900.0)
    base = {"kernel": cls, "bound": bound, "launches": n, "mean_ms": ms / n,
            "traffic": traffic_for(cls), "work_per_launch": work / n if n else None}
    if unit is None or work <= 0:
        return dict(base, achieved=None, peak=None, unit=None, frac=None)
    if bound == "tensor_fp64":
        pk = bf16 * TF32_PER_BF16 / OZ_TENSOR_PER_USEFUL
        ach = work / secs / 1e12
        return dict(base, bound="tensor", achieved=ach, peak=pk, unit="TFLOP/s", frac=ach / pk,
                    peak_source=f"{src} bf16 burst x nominal tf32/bf16 ratio / 45 slice pairs "
                                "(FP64-accurate products on the TF32 pipe)")
    if bound == "tensor":
        pk = bf16 * TF32_PER_BF16
        ach = work / secs / 1e12
        return dict(base, achieved=ach, peak=pk, unit="TFLOP/s", frac=ach / pk,
                    peak_source=f"{src} bf16 burst x nominal tf32/bf16 ratio")
    if bound == "hbm":
        pk = peaks.get("hbm_gbs", 6800.0)
        ach = work / secs / 1e9
        return dict(base, achieved=ach, peak=pk, unit="GB/s", frac=ach / pk,
                    peak_source=f"{src} copy bandwidth")
    pk = fp64_peak_gflops(peaks)
    ach = work / secs / 1e9
    return dict(base, achieved=ach, peak=pk, unit="GFLOP/s", frac=ach / pk,
                peak_source=f"derived: {N_SM} SMs x {src} max SM clock x 2 DFMA/clk "
                            "(a DFMA-only probe measured 1.256 TFLOP/s)")


# ---------------------------------------------------------------- grouped U(1) workloads
def u1_problem_inputs(seed, chi_l, chi_r, q_l, q_r, n_sec_l, n_sec_r, d, U):
    """Synthetic U(1) H_eff problem: Gaussian sector profiles on both bonds, Hermitian
    masked environments, the Bose-Hubbard MPO at (J = 1, U), compact random theta."""
    from paper_1610_02244_gb300 import synth, tnt
    g = synth.rng(seed)
    qa = synth.gaussian_sector_labels(chi_l, n_sec_l, 2.0, q_l)
    qb = synth.gaussian_sector_labels(chi_r, n_sec_r, 2.0, q_r)
    Le = synth.hermitian_env(g, chi_l) * synth.env_mask(qa, qa)
    Re = synth.hermitian_env(g, chi_r) * synth.env_mask(qb, qb)
    W = tnt.bh_mpo_site(d - 1, J, U, MU, 0.0, 2.0, 0.0)
    return {"L": Le, "R": Re, "W": W, "qa": qa, "qb": qb, "g": g}


def run_grouped(args, ws, rank, local):
    """--workload u1: one U(1) two-site eigensolve at chi = 1024, d = 5 (sector sizes 1..~200,
    15 sectors); --workload chains: 32 independent chains (chi = 256, d = 5, U/J = 1..8) whose
    eigensolves run in lock step with one grouped matvec per Krylov step."""
    import torch

    from paper_1610_02244_gb300 import build as b
    from paper_1610_02244_gb300 import synth, tnt
    b.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = tnt.Context(local)
    prec = tnt.TNT_PREC_MIXED if args.precision == "mixed" else tnt.TNT_PREC_FP64
    ctx.set_params(krylov_cap=KRYLOV, lanczos_maxit=KRYLOV, precision=prec, lanczos_tol=1e-12)
    if args.workload == "u1":
        specs = [(1024, 1024, 31, 33, 15, 15, 5, 3.4)]
        desc = ("U(1) two-site eigensolve, Bose-Hubbard d=5 D=4 U=3.4, chi=1024 both bonds, "
                "15 charge sectors of 1..~200 (Gaussian profile), 32 Krylov steps")
    else:
        specs = [(256, 256, 15, 17, 9, 9, 5, float(u)) for u in np.linspace(1.0, 8.0, 32)]
        desc = ("32 independent U(1) chains, Bose-Hubbard d=5 D=4, U/J = 1..8, chi=256, "
                "9 charge sectors each, lock-step eigensolves, 32 Krylov steps")
    probs, keep, xs = [], [], []
    for i, sp in enumerate(specs):
        inp = u1_problem_inputs(2000 + 97 * rank + i, *sp)
        tl = {k: torch.from_numpy(np.ascontiguousarray(inp[k])).to(dev) for k in ("L", "R", "W")}
        p = tnt.U1Problem(tl["L"], tl["W"], tl["W"], tl["R"], inp["qa"], inp["qb"], synth.BH_WQ)
        probs.append(p)
        keep.append((tl, inp))
        n = ctx.u1_size(p)
        xs.append(torch.from_numpy(synth.complex_gaussian(inp["g"], (n,))).to(dev))
    x0 = torch.cat(xs)
    x = torch.empty_like(x0)
    solve = (lambda: ctx.lanczos_ground_u1(probs[0], x)) if len(probs) == 1 else \
        (lambda: ctx.lanczos_ground_u1_batched(probs, x))
    _, flops_mv = ctx.heff_apply_u1(probs, x0, precision=prec)
    st = torch.cuda.current_stream(dev)

    def timed(pr, n):
        ctx.set_params(precision=pr)
        x.copy_(x0)
        solve()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(n):
            x.copy_(x0)
            solve()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    # the same eigensolves in the other precision, for the mixed-vs-FP64 comparison
    other = tnt.TNT_PREC_FP64 if prec == tnt.TNT_PREC_MIXED else tnt.TNT_PREC_MIXED
    solve_ms = {("fp64" if other == tnt.TNT_PREC_FP64 else "mixed"): timed(other, max(1, min(args.steps, 2)))}
    ctx.set_params(precision=prec)
    for _ in range(args.warmup):
        x.copy_(x0)
        solve()
    torch.cuda.synchronize()
    # kernel classes (plain launches so each is timed with events)
    per_class = {}
    for cls in ("cgemm_grouped", "zgemm_grouped", "u1_wop", "u1_pack_theta", "u1_gather",
                "multidot", "multiaxpy", "multidot_cond", "multiaxpy_cond", "multidot32",
                "multiaxpy32"):
        ctx.profile_select(cls)
        x.copy_(x0)
        solve()
        per_class[cls] = ctx.profile_read()
    ctx.profile_select(None)
    dom = max(per_class, key=lambda k: per_class[k][0])
    ctx.profile_select(dom)
    ctx.profile_read()
    launches0 = ctx.launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nmv = 0
    with ClockSampler(local) as clk:
        e0.record(st)
        for _ in range(args.steps):
            x.copy_(x0)
            r = solve()
            rs = r if isinstance(r, list) else [r]
            nmv += max(q["n_matvec"] for q in rs)
        e1.record(st)
        torch.cuda.synchronize()
    barrier(ws)
    ms_step = dist_max(e0.elapsed_time(e1) / args.steps, ws)
    solve_ms[args.precision] = ms_step
    dom_ms, dom_n, dom_work = ctx.profile_read()
    ctx.profile_select(None)
    launches = ctx.launch_count() - launches0
    flops_step = nmv / args.steps * flops_mv
    value = ws * flops_step / (ms_step * 1e-3) / 1e12
    if rank == 0:
        peaks, src = load_peaks()
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if prec == tnt.TNT_PREC_FP64 else "tf32x3+f64", "data": "synthetic",
                "config": {"workload": desc, "problems": len(probs), "precision": args.precision,
                           "compact_entries": int(x0.numel()), "block_flops_per_matvec": flops_mv,
                           "l2": "inputs larger than L2 (Krylov basis per step)"},
                "solve_ms": solve_ms, "fp64_over_mixed_time": solve_ms["fp64"] / solve_ms["mixed"],
                "kernel_ms_per_step": {k: v[0] for k, v in per_class.items()},
                "kernel_rooflines": {k: roofline(k, *v, peaks, src) for k, v in per_class.items() if v[1] > 0},
                "roofline": roofline(dom, dom_ms, dom_n, dom_work, peaks, src),
                "gpu_launches": launches, "clocks": clk.summary(),
                "energies": [q["E_rq"] for q in rs][:4]}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


# ---------------------------------------------------------------- DMRG and TEBD drivers
def run_dmrg(args, ws, rank, local):
    """--workload dmrg: the 8-site Bose-Hubbard ground state (N = 8, n_max = 3, J = 1, U = 2,
    chi_max = 32) by 4 two-site sweeps from the seeded random MPS; one step = the 4-sweep
    run (each from a fresh copy of the start state), metric s/sweep, mixed and FP64."""
    import torch

    from paper_1610_02244_gb300 import build as b
    from paper_1610_02244_gb300 import synth, tnt
    b.build()
    torch.cuda.set_device(local)
    ctx = tnt.Context(local)
    A, q = synth.random_charged_mps(synth.rng(0), DMRG_L, DMRG_NMAX + 1, DMRG_N, DMRG_CHI)
    mpo = ctx.mpo_bose_hubbard(DMRG_L, DMRG_NMAX, J, DMRG_U)
    for _ in range(max(1, args.warmup)):
        dmrg_sweeps(ctx, tnt, A, q, mpo, tnt.TNT_PREC_MIXED, 1)
    launches0 = ctx.launch_count()
    with ClockSampler(local) as clk:
        ms_mixed, st_mixed = dmrg_sweeps(ctx, tnt, A, q, mpo, tnt.TNT_PREC_MIXED, args.steps)
    launches = ctx.launch_count() - launches0
    ms_fp64, st_fp64 = dmrg_sweeps(ctx, tnt, A, q, mpo, tnt.TNT_PREC_FP64, max(1, min(args.steps, 3)))
    ms_mixed = dist_max(ms_mixed, ws)
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            t_or, E_or, E_ed = dmrg_oracle(A, q)
            cpu = {"value": t_or, "unit": "s/sweep", "cores": threads_used(), "kind": "oracle",
                   "sample": f"the same {DMRG_SWEEPS}-sweep run", "E": E_or, "E_exact": E_ed,
                   "dE_mixed_rel": abs(st_mixed["E"] - E_or) / abs(E_or),
                   "dE_fp64_rel": abs(st_fp64["E"] - E_or) / abs(E_or)}
        line = {"metric": METRIC, "value": ms_mixed * 1e-3, "unit": "s/sweep", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_mixed * DMRG_SWEEPS,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "tf32x3+f64", "data": "synthetic",
                "config": {"workload": "two-site DMRG, Bose-Hubbard L=8 N=8 n_max=3 J=1 U=2 "
                                       "chi_max=32, 4 sweeps from a seeded random MPS in the N=8 blocks",
                           "sweeps_per_step": DMRG_SWEEPS},
                "s_per_sweep": {"mixed": ms_mixed * 1e-3, "fp64": ms_fp64 * 1e-3},
                "E": {"mixed": st_mixed["E"], "fp64": st_fp64["E"]},
                "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


U1S_L, U1S_N, U1S_NMAX, U1S_U, U1S_CHI = 64, 64, 4, 3.4, 1024


def run_u1_sweep(args, ws, rank, local):
    """--workload u1_sweep: U(1) DMRG of the Bose-Hubbard chain L = 64, N = 64, d = 5,
    J = 1, U = 3.4 from a seeded random start (Gaussian sector profile, chi = 64): warm-up
    sweeps ramp chi_max 64 -> 128 -> 256 -> 512 (W of them), then K timed sweeps at
    chi_max = 1024 in split TF32 with the sweep's FP64 finish (metric s/sweep).  The
    state after the ramp is saved, and the four central two-site updates are timed from it
    in both precisions (the FP64 sweep itself would take several minutes)."""
    import tempfile

    import torch

    from paper_1610_02244_gb300 import build as b
    from paper_1610_02244_gb300 import synth, tnt
    b.build()
    torch.cuda.set_device(local)
    ctx = tnt.Context(local)
    chi = args.chi or U1S_CHI
    A, q = synth.random_charged_mps(synth.rng(0), U1S_L, U1S_NMAX + 1, U1S_N, 64, "gauss", 2.0)
    ctx.set_params(chi_max=64, precision=tnt.TNT_PREC_MIXED, lanczos_tol=LZ_TOL,
                   lanczos_maxit=MAXIT, krylov_cap=KRYLOV)
    ctx.set_fp64_gemm(tnt.TNT_FP64_GEMM_TC)
    mps = ctx.mps_create(A, q, chi_cap=chi)
    mpo = ctx.mpo_bose_hubbard(U1S_L, U1S_NMAX, J, U1S_U)
    dm = ctx.dmrg_create(mps, mpo)
    ramp = [c_ for c_ in (64, 128, 256, 512) if c_ < chi][: max(1, args.warmup)]
    hist = []
    for c_ in ramp:
        ctx.set_params(chi_max=c_)
        hist.append(dm.sweep())
    ctx.set_params(chi_max=chi)
    path = os.path.join(tempfile.mkdtemp(), "u1_state.tnt")
    mps.save(path)
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(st)
        for _ in range(args.steps):
            hist.append(dm.sweep())
        e1.record(st)
        torch.cuda.synchronize()
    s_sweep = dist_max(e0.elapsed_time(e1) * 1e-3 / args.steps, ws)
    launches = ctx.launch_count() - launches0
    # central updates from the saved state, both precisions: move the centre to bond c
    # with single updates, then time the updates at bonds c .. c+3 (left to right)
    c = U1S_L // 2 - 2
    central = {}
    for name, prec in (("mixed", tnt.TNT_PREC_MIXED), ("fp64", tnt.TNT_PREC_FP64)):
        ctx.set_params(precision=tnt.TNT_PREC_MIXED)  # the centre is walked in split TF32
        ctx.set_fp64_gemm(tnt.TNT_FP64_GEMM_TC)
        m2 = ctx.mps_load(path, chi_cap=chi)
        d2 = ctx.dmrg_create(m2, mpo)
        for i in range(c):
            d2.update(i, +1)
        ctx.set_params(precision=prec)
        ctx.set_fp64_gemm(tnt.TNT_FP64_GEMM_TC if prec == tnt.TNT_PREC_MIXED else tnt.TNT_FP64_GEMM_FMA)
        torch.cuda.synchronize()
        e0.record(st)
        nmv = 0
        Es = []
        for i in range(c, c + 4):
            lz, _ = d2.update(i, +1)
            nmv += lz["n_matvec"]
            Es.append(lz["E_rq"])
        e1.record(st)
        torch.cuda.synchronize()
        central[name] = {"s_per_update": e0.elapsed_time(e1) * 1e-3 / 4, "matvecs": nmv / 4,
                         "E": Es}
        del d2, m2
    if rank == 0:
        line = {"metric": METRIC, "value": s_sweep, "unit": "s/sweep", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": s_sweep * 1e3,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "tf32x3+f64", "data": "synthetic",
                "config": {"workload": f"U(1) DMRG sweep, Bose-Hubbard L={U1S_L} N={U1S_N} d={U1S_NMAX + 1} "
                                       f"U/J={U1S_U}, chi_max={chi} after a chi ramp {ramp}",
                           "ramp": ramp},
                "E": hist[-1]["E"], "max_chi": hist[-1]["max_chi"],
                "sweeps": [{k: h[k] for k in ("E", "max_err", "max_chi", "total_matvecs",
                                              "unconverged", "seconds", "t_plan", "t_eig",
                                              "t_svd", "t_env")} for h in hist],
                "central_updates": central,
                "fp64_over_mixed_time_central": central["fp64"]["s_per_update"] / central["mixed"]["s_per_update"],
                "gpu_launches": launches, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


CH_P, CH_L, CH_N, CH_NMAX, CH_CHI = 32, 32, 32, 4, 256


def run_chains_sweep(args, ws, rank, local):
    """--workload chains_sweep: 32 independent Bose-Hubbard chains (L = 32, N = 32, d = 5,
    J = 1, U/J = linspace(1, 8, 32), chi_max = 256, U(1)) from their own seeded random
    starts, swept in lock step (tnt_dmrg_sweep_batched): every bond's 32 eigensolves in
    one grouped Lanczos.  W warm-up sweeps, then K timed sweeps in split TF32 (with the
    sweep's FP64 finish), and the same W warm-up sweeps and one timed sweep in FP64 from the
    same starts; metric s/sweep of all 32 chains.""" 
    import torch

    from paper_1610_02244_gb300 import build as b
    from paper_1610_02244_gb300 import synth, tnt
    b.build()
    torch.cuda.set_device(local)
    ctx = tnt.Context(local)
    Us = np.linspace(1.0, 8.0, CH_P)
    chi = args.chi or CH_CHI
    starts = [synth.random_charged_mps(synth.rng(100 + 1000 * rank + k), CH_L, CH_NMAX + 1, CH_N,
                                       chi, "gauss", 2.0) for k in range(CH_P)]
    st = torch.cuda.current_stream()

    def arm(prec):
        ctx.set_params(chi_max=chi, precision=prec, lanczos_tol=LZ_TOL, lanczos_maxit=MAXIT,
                       krylov_cap=KRYLOV)
        ctx.set_fp64_gemm(tnt.TNT_FP64_GEMM_TC if prec == tnt.TNT_PREC_MIXED else tnt.TNT_FP64_GEMM_FMA)
        states = [ctx.mps_create(A, q, chi_cap=chi) for A, q in starts]
        runs = [ctx.dmrg_create(m, ctx.mpo_bose_hubbard(CH_L, CH_NMAX, J, float(u)))
                for m, u in zip(states, Us)]
        for _ in range(args.warmup):
            ctx.dmrg_sweep_batched(runs)
        torch.cuda.synchronize()
        launches0 = ctx.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            e0.record(st)
            for _ in range(args.steps):
                last = ctx.dmrg_sweep_batched(runs)
            e1.record(st)
            torch.cuda.synchronize()
        s_sweep = dist_max(e0.elapsed_time(e1) * 1e-3 / args.steps, ws)
        return s_sweep, last, ctx.launch_count() - launches0, clk.summary(), states

    s_mixed, st_mixed, launches, clocks, states = arm(tnt.TNT_PREC_MIXED)
    steps_saved = args.steps
    args.steps = 1  # the FP64 arm: its first timed sweep (several times slower)
    s_fp64, st_fp64, _, _, _ = arm(tnt.TNT_PREC_FP64)
    args.steps = steps_saved
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            cpu = _oracle_chain_sample(states[0], float(Us[0]), chi)
        E_m = [x["E"] for x in st_mixed]
        E_f = [x["E"] for x in st_fp64]
        line = {"metric": METRIC, "value": s_mixed, "unit": "s/sweep", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": s_mixed * 1e3,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "tf32x3+f64", "data": "synthetic",
                "config": {"workload": f"{CH_P} independent U(1) Bose-Hubbard chains L={CH_L} N={CH_N} "
                                       f"d={CH_NMAX + 1} U/J=1..8, chi_max={chi}, lock-step batched sweeps "
                                       "(one grouped Lanczos per bond), sweeps after warm-up",
                           "chains": CH_P},
                "s_per_sweep": {"mixed": s_mixed, "fp64": s_fp64},
                "fp64_over_mixed_time": s_fp64 / s_mixed,
                "E_per_chain": {"mixed": E_m, "fp64": E_f},
                "max_dE_rel_mixed_vs_fp64": max(abs(a - b) / abs(b) for a, b in zip(E_m, E_f)),
                "matvecs_per_sweep": {"mixed": sum(x["total_matvecs"] for x in st_mixed),
                                      "fp64": sum(x["total_matvecs"] for x in st_fp64)},
                "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def _oracle_chain_sample(mps, U_, chi):
    """The oracle's two-site update timed at the two central bonds of chain 0's GPU state
    (centre moved there by the oracle's exact SVD moves), scaled to 2(L-1) updates of all
    32 chains."""
    from oracle import bose_hubbard as bh
    from oracle import contract as oc
    from oracle import dmrg as od
    from oracle import tebd as ot
    from oracle.svd import TruncParams
    L_ = mps.L
    A = mps.tensors()
    q = [np.asarray(mps.charges(k), dtype=np.int64) for k in range(L_ + 1)]
    Ws, l, r = bh.bh_mpo(L_, CH_NMAX, J, U_)
    hs = [bh.bond_hamiltonian(CH_NMAX, J, U_, *bh.bond_weights(L_, j + 1)) for j in range(L_ - 1)]
    mover = ot.Tebd.from_bond_hamiltonians(A, q, hs, 0.0, od.EXACT)
    c = L_ // 2 - 1
    while mover.centre < c:
        mover._move_right()
    A, q = mover.A, mover.q
    Lenv = [None] * (L_ + 1)
    Lenv[0] = oc.boundary_left(l)
    for j in range(c):
        Lenv[j + 1] = oc.env_left(Lenv[j], Ws[j], A[j])
    Renv = [None] * (L_ + 1)
    Renv[L_] = oc.boundary_right(r)
    for j in range(L_ - 1, c + 1, -1):
        Renv[j] = oc.env_right(Renv[j + 1], Ws[j], A[j])
    lz = {"tol": 1e-12, "krylov_cap": 32, "max_matvec": 300}
    tr = TruncParams(chi_max=chi)
    t0 = time.perf_counter()
    st1 = od.two_site_update(A, q, Ws, Lenv, Renv, c, +1, tr, lz)
    Lenv[c + 1] = oc.env_left(Lenv[c], Ws[c], A[c])
    st2 = od.two_site_update(A, q, Ws, Lenv, Renv, c + 1, +1, tr, lz)
    t = (time.perf_counter() - t0) / 2
    return {"value": t * 2 * (L_ - 1) * CH_P, "unit": "s/sweep", "cores": threads_used(),
            "kind": "oracle", "sample": f"2 two-site updates at bonds {c},{c + 1} of chain 0's GPU "
            f"state ({st1['matvecs']}+{st2['matvecs']} matvecs), x 2(L-1) updates x {CH_P} chains",
            "s_per_update": t}


TEBD_L, TEBD_NMAX, TEBD_U, TEBD_DT, TEBD_CHI, TEBD_ERR = 64, 4, 2.0, 0.01, 512, 1e-10


def run_tebd(args, ws, rank, local):
    """--workload tebd: quench from the Mott state |1...1> of the 64-site chain (d = 5,
    J = 1, U = 2), second-order Trotter steps of dt = 0.01 at chi_max = 512 and truncation
    error 1e-10; one step = one Trotter step (95 two-site gates), metric s/step."""
    import torch

    from paper_1610_02244_gb300 import build as b
    from paper_1610_02244_gb300 import tnt
    b.build()
    torch.cuda.set_device(local)
    ctx = tnt.Context(local)
    ctx.set_params(chi_max=TEBD_CHI, trunc_err=TEBD_ERR, trunc_abs=-1.0, trunc_rel=1e-16, trunc_type=0)
    mps = ctx.mps_product([1] * TEBD_L, TEBD_NMAX + 1, TEBD_CHI)
    mpo = ctx.mpo_bose_hubbard(TEBD_L, TEBD_NMAX, J, TEBD_U)
    E0 = mps.expect_mpo(mpo)
    tb = ctx.tebd_create(mps, TEBD_NMAX, J, TEBD_U, TEBD_DT)
    for _ in range(args.warmup):
        tb.step()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    t0 = time.perf_counter()
    stats = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            stats.append(tb.step())
        torch.cuda.synchronize()
    dt = dist_max((time.perf_counter() - t0) / args.steps, ws)
    launches = ctx.launch_count() - launches0
    n2 = mps.norm2()
    if rank == 0:
        line = {"metric": METRIC, "value": dt, "unit": "s/step", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "TEBD quench from |1...1>, Bose-Hubbard L=64 d=5 J=1 U=2, "
                                       "2nd-order Trotter dt=0.01, chi_max=512, eps=1e-10",
                           "time_reached": TEBD_DT * (args.warmup + args.steps)},
                "device_s_per_step": statistics.mean(s["seconds"] for s in stats),
                "max_chi": stats[-1]["max_chi"], "err_sum_last_step": stats[-1]["err_sum"],
                "norm_loss": 1 - n2, "energy_drift": mps.expect_mpo(mpo) / n2 - E0,
                "gpu_launches": launches, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


SPIN_L, SPIN_TWO_S = 101, 2
SPIN_DMRG_CHI, SPIN_TEBD_CHI, SPIN_TEBD_DT, SPIN_TEBD_ERR = 200, 1000, 0.05, 1e-10
# the paper's single-node times for these two workloads (Sec. 6, Tables 1 and 2, U(1)
# blocking, fastest library stack): context from other hardware, not a target
PAPER_SPIN1_DMRG_S_PER_SWEEP, PAPER_SPIN1_TEBD_S_PER_STEP = 135.0, 57.0


def _spin_bond_terms(L_):
    from oracle import bose_hubbard as bh  # noqa: F401  (weights only)
    from oracle import spin as osp
    return [osp.bond_hamiltonian(SPIN_TWO_S, 1.0, 1.0, 0.0, *bh.bond_weights(L_, j + 1))
            for j in range(L_ - 1)]


def run_spin1_dmrg(args, ws, rank, local):
    """--workload spin1_dmrg: two-site DMRG sweeps of the isotropic spin-1 Heisenberg chain,
    L = 101, chi = 200, U(1) in S^z (the workload of the paper's Table 1), from a seeded
    random MPS in the S^z = 0 sector with a Gaussian sector profile (width 2) on every
    bond; W warm-up sweeps, then K timed sweeps; metric s/sweep (2(L-1) updates)."""
    import torch

    from paper_1610_02244_gb300 import build as b
    from paper_1610_02244_gb300 import synth, tnt
    b.build()
    torch.cuda.set_device(local)
    ctx = tnt.Context(local)
    prec = tnt.TNT_PREC_MIXED if args.precision == "mixed" else tnt.TNT_PREC_FP64
    chi = args.chi or SPIN_DMRG_CHI
    ctx.set_params(chi_max=chi, precision=prec, lanczos_tol=1e-12, lanczos_maxit=300,
                   krylov_cap=32)
    ctx.set_fp64_gemm(tnt.TNT_FP64_GEMM_TC if args.fp64_gemm == "tc" else tnt.TNT_FP64_GEMM_FMA)
    g = synth.rng(0)
    N = SPIN_L * SPIN_TWO_S // 2
    A, q = synth.random_charged_mps(g, SPIN_L, SPIN_TWO_S + 1, N, chi, "gauss", 2.0)
    mps = ctx.mps_create(A, q, chi_cap=chi)
    mpo = ctx.mpo_spin_heisenberg(SPIN_L, SPIN_TWO_S, 1.0)
    dm = ctx.dmrg_create(mps, mpo)
    hist = [dm.sweep() for _ in range(max(1, args.warmup))]
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(st)
        for _ in range(args.steps):
            hist.append(dm.sweep())
        e1.record(st)
        torch.cuda.synchronize()
    s_sweep = dist_max(e0.elapsed_time(e1) * 1e-3 / args.steps, ws)
    launches = ctx.launch_count() - launches0
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            cpu = _oracle_spin_dmrg_sample(mps, chi)
        E = hist[-1]["E"]
        line = {"metric": METRIC, "value": s_sweep, "unit": "s/sweep", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": s_sweep * 1e3,
                "higher_is_better": False, "scaling": "weak",
                "vs_baseline": s_sweep / PAPER_SPIN1_DMRG_S_PER_SWEEP if chi == SPIN_DMRG_CHI else None,
                "dtype": "tf32x3+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": f"two-site DMRG sweep, spin-1 Heisenberg L=101 chi={chi}, "
                                       "U(1) in S^z, S^z_total=0, seeded random MPS with a "
                                       "Gaussian sector profile, sweeps after warm-up",
                           "precision": args.precision, "fp64_gemm": args.fp64_gemm},
                "E": E, "E_per_bond": E / (SPIN_L - 1),
                "sweeps": [{k: h[k] for k in ("E", "max_err", "total_matvecs", "unconverged",
                                              "seconds", "t_plan", "t_eig", "t_svd", "t_env")}
                           for h in hist],
                "paper_s_per_sweep": PAPER_SPIN1_DMRG_S_PER_SWEEP,
                "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_spin1_dmrg1(args, ws, rank, local):
    """--workload spin1_dmrg1: single-site sweeps with subspace expansion of the spin-1
    Heisenberg chain, L = 101, chi = 200, U(1) in S^z (the chain of the paper's Table 1);
    W warm-up sweeps with alpha = 1e-3 10^-s, then K timed sweeps at alpha = 1e-6;
    metric s/sweep (2(L-1) one-site updates, FP64 eigensolves)."""
    import torch

    from paper_1610_02244_gb300 import build as b
    from paper_1610_02244_gb300 import synth, tnt
    b.build()
    torch.cuda.set_device(local)
    ctx = tnt.Context(local)
    chi = args.chi or SPIN_DMRG_CHI
    ctx.set_params(chi_max=chi, precision=tnt.TNT_PREC_FP64, lanczos_tol=1e-12,
                   lanczos_maxit=300, krylov_cap=32)
    ctx.set_fp64_gemm(tnt.TNT_FP64_GEMM_TC if args.fp64_gemm == "tc" else tnt.TNT_FP64_GEMM_FMA)
    N = SPIN_L * SPIN_TWO_S // 2
    A, q = synth.random_charged_mps(synth.rng(0), SPIN_L, SPIN_TWO_S + 1, N, chi, "gauss", 2.0)
    mps = ctx.mps_create(A, q, chi_cap=chi)
    dm = ctx.dmrg_create(mps, ctx.mpo_spin_heisenberg(SPIN_L, SPIN_TWO_S, 1.0))
    hist = [dm.sweep1(1e-3 * 10.0 ** (-s)) for s in range(max(1, args.warmup))]
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(st)
        for _ in range(args.steps):
            hist.append(dm.sweep1(1e-6))
        e1.record(st)
        torch.cuda.synchronize()
    s_sweep = dist_max(e0.elapsed_time(e1) * 1e-3 / args.steps, ws)
    if rank == 0:
        line = {"metric": METRIC, "value": s_sweep, "unit": "s/sweep", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": s_sweep * 1e3,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"single-site DMRG sweep with subspace expansion, spin-1 "
                                       f"Heisenberg L=101 chi={chi}, U(1) in S^z, S^z_total=0",
                           "fp64_gemm": args.fp64_gemm},
                "sweeps": [{k: h[k] for k in ("E", "max_err", "total_matvecs", "unconverged",
                                              "seconds", "max_chi")} for h in hist],
                "cpu_baseline": None, "gpu_launches": ctx.launch_count() - launches0,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def _oracle_spin_dmrg_sample(mps, chi):
    """The oracle's two-site update timed at the two central bonds of the GPU's state (centre
    moved there by the oracle's exact SVD moves, environments grown by the oracle), scaled
    to the 2(L-1) updates of a sweep (every bond but the outer four is at chi)."""
    from oracle import contract as oc
    from oracle import dmrg as od
    from oracle import spin as osp
    from oracle import tebd as ot
    from oracle.svd import TruncParams
    L_ = mps.L
    A = mps.tensors()
    q = [np.asarray(mps.charges(k), dtype=np.int64) for k in range(L_ + 1)]
    Ws, l, r, _ = osp.heisenberg_mpo(L_, SPIN_TWO_S, 1.0, 1.0)
    mover = ot.Tebd.from_bond_hamiltonians(A, q, _spin_bond_terms(L_), 0.0, od.EXACT)
    c = L_ // 2 - 1
    while mover.centre < c:
        mover._move_right()
    A, q = mover.A, mover.q
    Lenv = [None] * (L_ + 1)
    Lenv[0] = oc.boundary_left(l)
    for j in range(c):
        Lenv[j + 1] = oc.env_left(Lenv[j], Ws[j], A[j])
    Renv = [None] * (L_ + 1)
    Renv[L_] = oc.boundary_right(r)
    for j in range(L_ - 1, c + 1, -1):  # Renv[j]: sites j..L-1, down to j = c + 2
        Renv[j] = oc.env_right(Renv[j + 1], Ws[j], A[j])
    lz = {"tol": 1e-12, "krylov_cap": 32, "max_matvec": 300}
    tr = TruncParams(chi_max=chi)
    t0 = time.perf_counter()
    st1 = od.two_site_update(A, q, Ws, Lenv, Renv, c, +1, tr, lz)
    Lenv[c + 1] = oc.env_left(Lenv[c], Ws[c], A[c])
    st2 = od.two_site_update(A, q, Ws, Lenv, Renv, c + 1, +1, tr, lz)
    t = (time.perf_counter() - t0) / 2
    return {"value": t * 2 * (L_ - 1), "unit": "s/sweep", "cores": threads_used(),
            "kind": "oracle", "sample": f"2 two-site updates at bonds {c},{c + 1} of the GPU "
            f"state ({st1['matvecs']}+{st2['matvecs']} matvecs), x 2(L-1)",
            "s_per_update": t}


def _tebd_moves_per_step(L_):
    """Centre moves of one steady-state Trotter step: layers on bonds 0,2,.. | 1,3,.. |
    0,2,.. alternating direction; a gate needs the centre on i or i+1 and leaves it on
    i+1 (ascending) or i (descending)."""
    c, up, moves = 0, True, 0
    for rep in range(2):
        moves = 0
        for first in (0, 1, 0):
            bonds = list(range(first, L_ - 1, 2))
            for i in (bonds if up else bonds[::-1]):
                if c < i:
                    moves, c = moves + i - c, i
                elif c > i + 1:
                    moves, c = moves + c - i - 1, i + 1
                c = i + 1 if up else i
            up = not up
    return moves


def run_spin1_tebd(args, ws, rank, local):
    """--workload spin1_tebd: second-order Trotter steps of the isotropic spin-1 Heisenberg
    chain, L = 101, chi_max = 1000, U(1) in S^z (the workload of the paper's Table 2),
    dt = 0.05, truncation error 1e-10, on a seeded random MPS at chi = 1000 in the
    S^z_total = +1 sector (one spin flip above S^z = 0) with a Gaussian sector profile:
    every gate works at the full bond dimension.  W warm-up steps, K timed; s/step."""
    import torch

    from paper_1610_02244_gb300 import build as b
    from paper_1610_02244_gb300 import synth, tnt
    b.build()
    torch.cuda.set_device(local)
    ctx = tnt.Context(local)
    chi = args.chi or SPIN_TEBD_CHI
    ctx.set_params(chi_max=chi, trunc_err=SPIN_TEBD_ERR, trunc_abs=-1.0, trunc_rel=1e-16,
                   trunc_type=0)
    ctx.set_fp64_gemm(tnt.TNT_FP64_GEMM_TC if args.fp64_gemm == "tc" else tnt.TNT_FP64_GEMM_FMA)
    g = synth.rng(0)
    N = SPIN_L * SPIN_TWO_S // 2 + 1
    A, q = synth.random_charged_mps(g, SPIN_L, SPIN_TWO_S + 1, N, chi, "gauss", 2.0)
    mps = ctx.mps_create(A, q, chi_cap=chi)
    del A
    tb = ctx.tebd_create_spin(mps, SPIN_TWO_S, 1.0, SPIN_TEBD_DT)
    for _ in range(args.warmup):
        tb.step()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    stats = []
    t0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            stats.append(tb.step())
        torch.cuda.synchronize()
    s_step = dist_max((time.perf_counter() - t0) / args.steps, ws)
    launches = ctx.launch_count() - launches0
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            cpu = _oracle_spin_tebd_sample(mps, chi)
        line = {"metric": METRIC, "value": s_step, "unit": "s/step", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": s_step * 1e3,
                "higher_is_better": False, "scaling": "weak",
                "vs_baseline": s_step / PAPER_SPIN1_TEBD_S_PER_STEP if chi == SPIN_TEBD_CHI else None,
                "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": f"TEBD step, spin-1 Heisenberg L=101 chi_max={chi}, U(1) in "
                                       "S^z, S^z_total=+1, dt=0.05, eps=1e-10, seeded random MPS "
                                       f"at chi={chi} with a Gaussian sector profile",
                           "fp64_gemm": args.fp64_gemm},
                "device_s_per_step": statistics.mean(s["seconds"] for s in stats),
                "max_chi": stats[-1]["max_chi"], "err_sum_last_step": stats[-1]["err_sum"],
                "paper_s_per_step": PAPER_SPIN1_TEBD_S_PER_STEP,
                "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def _oracle_spin_tebd_sample(mps, chi):
    """The oracle's gate (theta, G theta, truncated SVD) and one exact centre move timed at
    the central bond of the GPU's state, scaled to one step's gates and centre moves."""
    from oracle import tebd as ot
    from oracle.svd import TruncParams
    L_ = mps.L
    c = L_ // 2 - 1
    A = mps.tensors()
    q = [np.asarray(mps.charges(k), dtype=np.int64) for k in range(L_ + 1)]
    ev = ot.Tebd.from_bond_hamiltonians(A, q, _spin_bond_terms(L_), SPIN_TEBD_DT,
                                        TruncParams(chi_max=chi, err_tol=SPIN_TEBD_ERR))
    ev.centre = c  # timing only: the cost of a gate does not depend on the gauge
    t0 = time.perf_counter()
    ev.apply_gate(c, ev.gates[("full", c)], True)
    t_gate = time.perf_counter() - t0
    t0 = time.perf_counter()
    ev._move_right()
    t_move = time.perf_counter() - t0
    n_gates = 2 * len(range(0, L_ - 1, 2)) + len(range(1, L_ - 1, 2))
    n_moves = _tebd_moves_per_step(L_)
    return {"value": n_gates * t_gate + n_moves * t_move, "unit": "s/step",
            "cores": threads_used(), "kind": "oracle",
            "sample": f"1 gate and 1 centre move at bond {c} of the GPU state, x {n_gates} gates "
                      f"and {n_moves} moves per step", "s_per_gate": t_gate, "s_per_move": t_move}


def main():
    faulthandler.enable()
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["update", "u1", "u1_sweep", "chains", "chains_sweep", "dmrg", "tebd",
                                           "spin1_dmrg", "spin1_dmrg1", "spin1_tebd"],
                    default="update")
    ap.add_argument("--chi", type=int, default=None,
                    help="bond dimension of the spin1_dmrg / spin1_tebd workloads (default: "
                         "the paper's 200 / 1000)")
    ap.add_argument("--fp64-gemm", choices=["tc", "fma"], default=None,
                    help="engine of the FP64 products (default: tc with --precision mixed, "
                         "fma with --precision fp64, the plain FP64 path)")
    args = ap.parse_args()
    if args.fp64_gemm is None:
        args.fp64_gemm = "tc" if args.precision == "mixed" else "fma"
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload in ("u1", "chains"):
        return run_grouped(args, ws, rank, local)
    if args.workload == "dmrg":
        return run_dmrg(args, ws, rank, local)
    if args.workload == "chains_sweep":
        return run_chains_sweep(args, ws, rank, local)
    if args.workload == "u1_sweep":
        return run_u1_sweep(args, ws, rank, local)
    if args.workload == "tebd":
        return run_tebd(args, ws, rank, local)
    if args.workload == "spin1_dmrg":
        return run_spin1_dmrg(args, ws, rank, local)
    if args.workload == "spin1_dmrg1":
        return run_spin1_dmrg1(args, ws, rank, local)
    if args.workload == "spin1_tebd":
        return run_spin1_tebd(args, ws, rank, local)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
