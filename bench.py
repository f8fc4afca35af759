#!/usr/bin/env python3
"""Throughput of the matrix-free neo-Hookean tangent application on one GB300.

One step = one application v = A(u) du of the constrained tangent operator (Algorithm 1 /
its cached-point variant) on the Q2 64^3 unit-cube workload (6,440,067 DoFs), FP64.
`value` is whole-job GDoF/s (DoFs per step / device time per step, summed over replicas).

Also printed on the same JSON line: the other strategies and precisions and the Q4 32^3
companion workload (`variants`), the roofline of the apply kernel, an end-to-end number
through the C ABI with host buffers, the CPU oracle timed on a bounded sample, clocks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import nhmf_inputs as inp  # noqa: E402

METRIC = "tangent-apply GDoF/s (FP64, FP32) and Newton time to 1e-8 vs plain FP64 CG"
MAIN = "q2_64_clamp"
COMPANION = "q4_32_clamp"
LARGE = "q4_64_compress"   # the 51 M-DoF workload: FP64 and FP32 applies, both strategies
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# FP64: 2 DFMA per clock per SM (measured 1.20 TFLOP/s on this GPU with an FMA loop);
# FP32: 128 FFMA per clock per SM.  Peaks at the maximum SM clock.
FP64_PEAK_TFLOPS = SM_COUNT * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP32_PEAK_TFLOPS = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12


KERNEL_SOURCES = ["include/nhmf.h", "paper_2505_15535_gb300/csrc/operators.cu",
                  "paper_2505_15535_gb300/csrc/sumfact.cuh", "paper_2505_15535_gb300/csrc/df64.cuh",
                  "paper_2505_15535_gb300/csrc/internal.h"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_apply_fp64_cached_q2_64.traffic.json")


def kernel_source_hash() -> str:
    import hashlib
    hsh = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()


def measured_traffic():
    """DRAM bytes per apply of the FP64 cached Q2 64^3 kernel from the committed ncu capture,
    or None when the kernel sources changed since that capture."""
    try:
        d = json.load(open(TRAFFIC_FILE))
    except Exception:
        return None
    return d.get("dram_bytes_per_apply") if d.get("source_sha256") == kernel_source_hash() else None


def canonical_flops(w: inp.Workload, strategy: str) -> float:
    """Algorithmic FLOPs of one apply: 2 n^4 per 1D pass per scalar field per element
    (54 passes on the fly: 18 for u, 18 for du, 18 back; 36 cached) plus the point code
    (230 FLOP per point on the fly, 150 cached; FMA = 2)."""
    n = w.degree + 1
    passes, point = (54, 230) if strategy == "otf" else (36, 150)
    return w.n_elements * passes * 2 * n ** 4 + w.n_qp * point


def compulsory_bytes(w: inp.Workload, strategy: str, b: int) -> float:
    """Bytes one apply must move: u, du, v (on the fly) or du, v and the 10-value cache."""
    if strategy == "otf":
        return 3 * b * w.n_dofs
    return 2 * b * w.n_dofs + 10 * b * w.n_qp


def describe(w: inp.Workload) -> str:
    u = "u=(h/p)U(+-%g)" % w.u_amp if w.u_rule == "scaled" else "u=U(+-%g)" % w.u_amp
    du = "du~N(0,1)" if w.du_rule == "normal" else "du=U(+-%g)" % w.du_amp
    bc = {0: "no Dirichlet", 1: "clamp x=0", 2: "compression"}[w.bc]
    return (f"Q{w.degree} hex {w.n_el}^3 unit cube ({w.n_dofs:,} DoFs, {w.n_qp:,} Gauss points), "
            f"mu={w.mu:g}, lambda={w.lam:g}, {bc}, {u}, {du}")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[3], parts[4:]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3][1:]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle
CPU_ROUTE = ("the oracle's plain sum-factorised FP64 apply (oracle/sumfact.c, Algorithm 1 element by "
             "element, OpenMP over the elements of each colour class)")


def oracle_sumfact(w: inp.Workload, u, strategy: str):
    """The oracle's sum-factorised CPU operator for workload w (cache built for 'cached')."""
    from oracle.sumfact import SumFactOperator, threads
    op = SumFactOperator(w.n_el, w.degree, w.mu, w.lam, w.bc)
    if strategy == "cached":
        op.set_cache(u)
    return op, threads()


def oracle_sample(w: inp.Workload, u, du, strategy: str, budget_s: float):
    """Median time of whole-workload CPU applies, repeated until `budget_s` is spent (at least 3)."""
    op, nthreads = oracle_sumfact(w, u, strategy)
    v = np.empty(w.n_dofs)
    times = []
    while len(times) < 3 or sum(times) < budget_s:
        t0 = time.perf_counter()
        op.apply(u, du, cached=strategy == "cached", out=v)
        times.append(time.perf_counter() - t0)
    med = statistics.median(times)
    return w.n_dofs / med / 1e9, len(times), sum(times), nthreads


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = inp.WORKLOADS[args.apply_workload]
    u, du = inp.draw_u(w), inp.draw_du(w)
    op, nthreads = oracle_sumfact(w, u, args.strategy)
    cached = args.strategy == "cached"
    v = np.empty(w.n_dofs)
    for _ in range(args.warmup):
        op.apply(u, du, cached=cached, out=v)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        op.apply(u, du, cached=cached, out=v)
        times.append(time.perf_counter() - t0)
    step = sum(times) / len(times)
    value = w.n_dofs / step / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.apply_workload}: " + describe(w) + f"; FP64 tangent apply, {args.strategy} strategy",
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": nthreads, "kind": "oracle",
                         "sample": f"the whole workload every step ({w.n_dofs:,} DoFs): " + CPU_ROUTE +
                                   f", {args.strategy} strategy, {nthreads} threads"},
        "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU
def time_applies(torch, prob, nhmf, du, v, prec, strat, steps, flush):
    """Mean device time per apply (ms) with an L2 flush between steps, and kernel-only time."""
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    nhmf.nhmf_profile_read(prob.ctx, nhmf.NHMF_KIND_APPLY)
    nhmf.nhmf_profile_enable(prob.ctx, 1)
    for a, b in ev:
        flush.add_(1.0)
        a.record(st)
        prob.apply(du, v, prec, strat)
        b.record(st)
    torch.cuda.synchronize()
    nhmf.nhmf_profile_enable(prob.ctx, 0)
    kms, launches = nhmf.nhmf_profile_read(prob.ctx, nhmf.NHMF_KIND_APPLY)
    step_ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    return step_ms, kms / steps, launches


def max_over_ranks(values, dist, device=None):
    """Element-wise maximum of a list of floats over all ranks (the slowest rank's times)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(values)
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def run_gpu(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    import __graft_entry__ as g
    g.build()
    from paper_2505_15535_gb300 import nhmf

    dev = torch.device("cuda", local)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    strategy = args.strategy
    if strategy == "spatial":
        raise SystemExit("--strategy spatial is measured by --mode kernel (and reported as a variant)")
    strat = nhmf.NHMF_CACHED if strategy == "cached" else nhmf.NHMF_ON_THE_FLY

    main = args.apply_workload
    w = inp.WORKLOADS[main]
    u, du = inp.draw_u(w), inp.draw_du(w)
    prob = nhmf.Problem.from_workload(w)
    ut = torch.from_numpy(u).to(dev)
    t0 = time.perf_counter()
    # the variants reuse this problem's FP32, double-float and Algorithm 2 caches
    prob.set_linearization(ut, nhmf.NHMF_CACHE_FP64 if args.no_variants else
                           nhmf.NHMF_CACHE_FP64 | nhmf.NHMF_CACHE_FP32 | nhmf.NHMF_CACHE_DF64 |
                           nhmf.NHMF_CACHE_SPATIAL)
    torch.cuda.synchronize()
    cache_build_s = time.perf_counter() - t0
    dut = torch.from_numpy(du).to(dev)
    v = torch.empty_like(dut)
    for _ in range(args.warmup):
        prob.apply(dut, v, nhmf.NHMF_FP64, strat)

    # ---- timed region: exactly K steps
    barrier()
    with ClockSampler(local) as clk:
        step_ms, kernel_ms, launches = time_applies(torch, prob, nhmf, dut, v, nhmf.NHMF_FP64, strat,
                                                    args.steps, flush)
        barrier()
    clocks = clk.summary()
    step_ms, kernel_ms = max_over_ranks([step_ms, kernel_ms], dist, dev)
    value = world * w.n_dofs / (step_ms * 1e-3) / 1e9

    # ---- end to end through the C ABI with pinned host buffers: every step uploads its du from
    # pinned host memory, applies, and downloads v.  Steps are pipelined over three streams with
    # two buffer sets, so that the upload of step k+1 and the download of step k-1 overlap the
    # apply of step k (whole-job throughput of a stream of independent applications).
    du_h = torch.from_numpy(du).pin_memory()
    v_h = [torch.empty(du_h.shape, dtype=torch.float64).pin_memory() for _ in range(2)]
    d_in = [torch.empty_like(dut) for _ in range(2)]
    v_out = [torch.empty_like(dut) for _ in range(2)]
    s_comp = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    in_done = [torch.cuda.Event() for _ in range(2)]
    comp_done = [torch.cuda.Event() for _ in range(2)]
    out_done = [torch.cuda.Event() for _ in range(2)]

    def e2e_run(nsteps):
        for e in in_done + comp_done + out_done:
            e.record(s_comp)
        for k in range(nsteps):
            i = k & 1
            s_in.wait_event(comp_done[i])                  # d_in[i] is free once apply k-2 is done
            with torch.cuda.stream(s_in):
                d_in[i].copy_(du_h, non_blocking=True)
            in_done[i].record(s_in)
            s_comp.wait_event(in_done[i])
            s_comp.wait_event(out_done[i])                 # v_out[i] is free once download k-2 is done
            prob.apply(d_in[i], v_out[i], nhmf.NHMF_FP64, strat)
            comp_done[i].record(s_comp)
            s_out.wait_event(comp_done[i])
            with torch.cuda.stream(s_out):
                v_h[i].copy_(v_out[i], non_blocking=True)
            out_done[i].record(s_out)
        for e in out_done:
            s_comp.wait_event(e)

    e2e_steps = max(3, min(args.steps, 50))
    e2e_run(2)
    torch.cuda.synchronize()
    barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s_comp)
    e2e_run(e2e_steps)
    b.record(s_comp)
    barrier()
    e2e_ms = max_over_ranks([a.elapsed_time(b) / e2e_steps], dist, dev)[0]
    torch.cuda.synchronize()
    assert torch.equal(v_h[(e2e_steps - 1) & 1], v_out[(e2e_steps - 1) & 1].cpu()), "e2e download mismatch"
    e2e = {"value": world * w.n_dofs / (e2e_ms * 1e-3) / 1e9, "unit": "GDoF/s",
           "h2d_bytes_per_step": int(du_h.numel() * 8), "d2h_bytes_per_step": int(v_h[0].numel() * 8),
           "pipeline": "3 streams, 2 buffer sets: upload k+1 and download k-1 overlap apply k"}

    # ---- roofline of the apply kernel (FP64 pipe)
    flops = canonical_flops(w, strategy)
    achieved = flops / (kernel_ms * 1e-3) / 1e12
    fma_measured = {"fp64": nhmf.nhmf_measure_fma_peak(nhmf.NHMF_FP64),
                    "fp32": nhmf.nhmf_measure_fma_peak(nhmf.NHMF_FP32)}
    traffic = measured_traffic() if (main == MAIN and strategy == "cached") else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                "algorithmic_bytes": compulsory_bytes(w, strategy, 8),
                "kernel": f"k_apply<{w.degree},double,{strategy}> (8 colour launches per apply)",
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 FLOP x 2070 MHz",
                "fma_peak_measured_tflops": fma_measured,
                "frac_of_measured_fp64_fma": achieved / fma_measured["fp64"] if fma_measured["fp64"] else None,
                "flops_per_apply": flops}

    # ---- variants (not the headline): both strategies, both precisions, both C2 meshes
    variants = {}
    if not args.no_variants:
        vs = max(5, min(args.steps, 30))
        hbm_peak = MEASURED.get("hbm_gbs") or 6800.0
        names = (main, COMPANION, LARGE) if main == MAIN else (main,)
        for name in names:
            wv = inp.WORKLOADS[name]
            large = name == LARGE
            if name == main:
                pv, dv = prob, dut
            else:
                pv = nhmf.Problem.from_workload(wv)
                pv.set_linearization(torch.from_numpy(inp.draw_u(wv)).to(dev),
                                     nhmf.NHMF_CACHE_FP64 | nhmf.NHMF_CACHE_FP32 |
                                     (0 if large else nhmf.NHMF_CACHE_DF64 | nhmf.NHMF_CACHE_SPATIAL))
                dv = torch.from_numpy(inp.draw_du(wv)).to(dev)
            for prec_name, prec, dt in (("fp64", nhmf.NHMF_FP64, torch.float64), ("fp32", nhmf.NHMF_FP32, torch.float32)):
                x = dv.to(dt)
                y = torch.empty_like(x)
                for sname, sid in (("otf", nhmf.NHMF_ON_THE_FLY), ("cached", nhmf.NHMF_CACHED)):
                    for _ in range(3):
                        pv.apply(x, y, prec, sid)
                    sm, km, _ = time_applies(torch, pv, nhmf, x, y, prec, sid, vs, flush)
                    fl = canonical_flops(wv, sname)
                    peak = FP64_PEAK_TFLOPS if prec_name == "fp64" else FP32_PEAK_TFLOPS
                    bts = compulsory_bytes(wv, sname, 8 if prec_name == "fp64" else 4)
                    # roofline: the larger of the ALU time and the HBM time of the algorithmic work
                    t_alu, t_hbm = fl / (peak * 1e12), bts / (hbm_peak * 1e9)
                    variants[f"{name}/{prec_name}/{sname}"] = {
                        "gdofs": wv.n_dofs / (sm * 1e-3) / 1e9, "ms": sm, "kernel_ms": km,
                        "tflops": fl / (km * 1e-3) / 1e12, "alu_frac": fl / (km * 1e-3) / 1e12 / peak,
                        "hbm_gbs": bts / (km * 1e-3) / 1e9, "hbm_frac": bts / (km * 1e-3) / 1e9 / hbm_peak,
                        "bound": "alu" if t_alu >= t_hbm else "hbm",
                        "roofline_frac": max(t_alu, t_hbm) / (km * 1e-3)}
            if large:
                pv.close()
                continue
            # Algorithm 2 (partial assembly in the current configuration), FP64
            x = dv
            y = torch.empty_like(x)
            for _ in range(3):
                pv.apply(x, y, nhmf.NHMF_FP64, nhmf.NHMF_SPATIAL)
            sm, km, _ = time_applies(torch, pv, nhmf, x, y, nhmf.NHMF_FP64, nhmf.NHMF_SPATIAL, vs, flush)
            n = wv.degree + 1
            fl = wv.n_elements * 36 * 2 * n ** 4 + wv.n_qp * 260
            variants[f"{name}/fp64/spatial"] = {
                "gdofs": wv.n_dofs / (sm * 1e-3) / 1e9, "ms": sm, "kernel_ms": km,
                "tflops": fl / (km * 1e-3) / 1e12, "alu_frac": fl / (km * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                "hbm_gbs": (2 * 8 * wv.n_dofs + 36 * 8 * wv.n_qp) / (km * 1e-3) / 1e9}
            # FP64-accurate double-float arithmetic on the FP32 pipe (cached strategy)
            x = dv
            y = torch.empty_like(x)
            for _ in range(3):
                pv.apply(x, y, nhmf.NHMF_DF64, nhmf.NHMF_CACHED)
            sm, km, _ = time_applies(torch, pv, nhmf, x, y, nhmf.NHMF_DF64, nhmf.NHMF_CACHED, vs, flush)
            fl = canonical_flops(wv, "cached")
            variants[f"{name}/df64/cached"] = {
                "gdofs": wv.n_dofs / (sm * 1e-3) / 1e9, "ms": sm, "kernel_ms": km,
                "fp64_equivalent_tflops": fl / (km * 1e-3) / 1e12,
                "hbm_gbs": compulsory_bytes(wv, "cached", 8) / (km * 1e-3) / 1e9,
                "note": "FP64-accurate double-float arithmetic on the FP32 pipe: canonical FP64 FLOPs per "
                        "second, no pipe fraction claimed (one FP64 operation costs several FP32 ones)"}
            if pv is not prob:
                pv.close()
        # the split neo-Hookean model (Eq. hypcomplex): on the fly and Algorithm 2
        ws = inp.WORKLOADS[main]
        ps = nhmf.Problem(ws.n_el, ws.degree, ws.mu, 5.0, ws.bc, model=nhmf.NHMF_MODEL_SPLIT)
        ps.set_linearization(torch.from_numpy(u).to(dev), nhmf.NHMF_CACHE_SPATIAL)
        y = torch.empty_like(dut)
        for sname, sid in (("otf", nhmf.NHMF_ON_THE_FLY), ("spatial", nhmf.NHMF_SPATIAL)):
            for _ in range(3):
                ps.apply(dut, y, nhmf.NHMF_FP64, sid)
            sm, km, _ = time_applies(torch, ps, nhmf, dut, y, nhmf.NHMF_FP64, sid, vs, flush)
            variants[f"{main}_split_kappa5/fp64/{sname}"] = {"gdofs": ws.n_dofs / (sm * 1e-3) / 1e9, "ms": sm,
                                                           "kernel_ms": km}
        ps.close()

    # ---- Newton to 1e-8: plain FP64 Jacobi-CG vs mixed-precision multigrid, first two load
    # steps of the Q2 64^3 compression workload (the second half of the metric; bounded time)
    newton = None
    if not args.no_newton:
        wn = inp.WORKLOADS["q2_64_compress"]
        pn = nhmf.Problem.from_workload(wn)
        newton = {"workload": f"q2_64_compress: {describe(wn)}; load steps 1-2 of {wn.load_steps}"}
        for sname, sid, outer in (("plain_fp64_jacobi_cg", nhmf.NHMF_SOLVER_JACOBI_CG, nhmf.NHMF_FP64),
                                  ("mixed_fp32_gmg", nhmf.NHMF_SOLVER_MIXED_GMG, nhmf.NHMF_FP64),
                                  ("mixed_fp32_gmg_df64_outer", nhmf.NHMF_SOLVER_MIXED_GMG, nhmf.NHMF_DF64)):
            un = torch.zeros(wn.n_dofs, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = pn.solve(un, solver=sid, load_steps=wn.load_steps, compression=wn.compression, last_step=2,
                          linear_rtol=1e-8, outer_apply=outer)
            torch.cuda.synchronize()
            newton[sname] = {"seconds": time.perf_counter() - t0, "newton_iters": sum(st["newton_iters"]),
                             "outer_iters": st["total_linear_iters"], "rel_residual": max(st["rel_residual"])}
        newton["speedup"] = newton["plain_fp64_jacobi_cg"]["seconds"] / newton["mixed_fp32_gmg"]["seconds"]
        newton["speedup_df64_outer"] = (newton["plain_fp64_jacobi_cg"]["seconds"] /
                                        newton["mixed_fp32_gmg_df64_outer"]["seconds"])
        pn.close()

    # ---- CPU oracle (rank 0, N = 1): whole-workload applies on all host cores, ~cpu_seconds
    cpu = None
    if world == 1 and not args.no_cpu:
        gd, napp, spent, nthreads = oracle_sample(w, u, du, strategy, budget_s=args.cpu_seconds)
        cpu = {"value": gd, "unit": "GDoF/s", "cores": nthreads, "kind": "oracle",
               "sample": f"{napp} applies of the whole workload ({w.n_dofs:,} DoFs) in {spent:.1f} s, median: " +
                         CPU_ROUTE + f", {strategy} strategy, {nthreads} threads (nproc {os.cpu_count()})"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{main}: " + describe(w) + f"; FP64 tangent apply, {strategy} strategy",
                       "l2": "flushed between timed steps (256 MB write outside the timed events)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches + args.steps),   # 8 colour launches + 1 Dirichlet fix per step
            "clocks": clocks, "cache_build_s": cache_build_s, "variants": variants, "newton": newton,
        }
        print(json.dumps(line), flush=True)
    prob.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ Newton mode
UNET_LAYERS = [("conv", 3, 16), ("conv", 16, 16), ("down", 16, 16), ("conv", 16, 16), ("down", 16, 16),
               ("conv", 16, 16), ("up", 16, 16), ("conv", 16, 16), ("up", 16, 16), ("conv", 16, 16),
               ("conv", 16, 3)]


def he_init_flat(seed=5000):
    """Initial U-Net parameters in the library's flat layout: He-normal weights
    (std sqrt(2 / (27 c_in))) from seeded N(0, 1) draws, zero biases."""
    parts = []
    for k, (_, cin, cout) in enumerate(UNET_LAYERS):
        parts.append(inp.normal(seed + k, cin * cout * 27) * np.sqrt(2.0 / (27 * cin)))
        parts.append(np.zeros(cout))
    return np.concatenate(parts)

NEWTON_METRIC = "Newton time to 1e-8 (mixed FP32-inner / learned vs plain FP64 Jacobi-CG)"


def run_kernel(args):
    """One apply kernel alone (for profiling the variants): `--precision` x `--strategy` on
    `--apply-workload`, only the point cache it reads built, `--warmup` + `--steps` applies;
    prints the mean device time per apply."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2505_15535_gb300 import nhmf
    dev = torch.device("cuda", 0)
    w = inp.WORKLOADS[args.apply_workload]
    prec = {"fp64": nhmf.NHMF_FP64, "fp32": nhmf.NHMF_FP32, "df64": nhmf.NHMF_DF64}[args.precision]
    strat = {"cached": nhmf.NHMF_CACHED, "otf": nhmf.NHMF_ON_THE_FLY, "spatial": nhmf.NHMF_SPATIAL}[args.strategy]
    mask = {nhmf.NHMF_FP64: nhmf.NHMF_CACHE_FP64, nhmf.NHMF_FP32: nhmf.NHMF_CACHE_FP32,
            nhmf.NHMF_DF64: nhmf.NHMF_CACHE_DF64}[prec]
    if strat == nhmf.NHMF_SPATIAL:
        mask = nhmf.NHMF_CACHE_SPATIAL
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(torch.from_numpy(inp.draw_u(w)).to(dev), mask if strat != nhmf.NHMF_ON_THE_FLY else 0)
    dt = torch.float32 if prec == nhmf.NHMF_FP32 else torch.float64
    du = torch.from_numpy(inp.draw_du(w)).to(dev).to(dt)
    v = torch.empty_like(du)
    for _ in range(args.warmup):
        prob.apply(du, v, prec, strat)
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    step_ms, kernel_ms, launches = time_applies(torch, prob, nhmf, du, v, prec, strat, args.steps, flush)
    print(json.dumps({"mode": "kernel", "workload": w.name, "precision": args.precision, "strategy": args.strategy,
                      "steps": args.steps, "kernel_ms": kernel_ms, "step_ms": step_ms,
                      "gdofs": w.n_dofs / (step_ms * 1e-3) / 1e9}), flush=True)
    prob.close()
    return 0


def run_newton(args):
    """Load steps of the compression workload, one solve call per step, for each solver.

    plain: FP64 Jacobi-CG; mixed: FP64 flexible CG with an FP32 inner Jacobi-CG; learned and
    mixed_learned: the U-Net preconditioner trained on pairs recorded during the plain solve of
    the first `train_steps` load steps.  Per step: wall time, Newton/outer/inner iterations,
    the final relative FP64 residual, the relative difference to the plain solver's state, and
    (plain solver) the FP32 apply's error against the FP64 apply at that state.  The FP64 apply
    and residual are parity-tested against the oracle, at full size on sampled rows of a solved
    state too, so the benchmark runs no oracle code here."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2505_15535_gb300 import nhmf
    dev = torch.device("cuda", 0)
    w = inp.WORKLOADS[args.workload]
    S = w.load_steps
    last = min(S, args.last_step) if args.last_step else S
    prob = nhmf.Problem(w.n_el, w.degree, w.mu, w.lam, w.bc)
    solvers = [s.strip() for s in args.solvers.split(",") if s.strip()]
    LEARNED = ("learned", "mixed_learned", "mixed_gmg_learned")
    learned = any(s in LEARNED for s in solvers)
    # the learned correction of the multigrid solver trains on pairs recorded by mixed_gmg
    # solves; the other learned solvers on pairs recorded by the plain solver
    base_solver = "mixed_gmg" if "mixed_gmg_learned" in solvers else "plain"
    if learned and base_solver not in solvers:
        raise SystemExit(f"--solvers must include {base_solver} (it records the training pairs)")
    if learned:
        nhmf.nhmf_unet_create(prob.ctx, args.pairs)
        nhmf.nhmf_unet_set_params(prob.ctx, he_init_flat())
    base = dict(compression=w.compression, load_steps=S, linear_rtol=args.linear_rtol,
                newton_rtol=1e-8, inner_rtol=args.inner_rtol, inner_max_iter=args.inner_max_iter,
                smoother_degree=args.smoother_degree, smoother_range=args.smoother_range)
    outer = {"fp64": nhmf.NHMF_FP64, "df64": nhmf.NHMF_DF64}[args.outer]
    ids = {"plain": nhmf.NHMF_SOLVER_JACOBI_CG, "mixed": nhmf.NHMF_SOLVER_MIXED_FCG,
           "learned": nhmf.NHMF_SOLVER_LEARNED_FCG, "mixed_learned": nhmf.NHMF_SOLVER_MIXED_LEARNED,
           "gmg": nhmf.NHMF_SOLVER_GMG, "mixed_gmg": nhmf.NHMF_SOLVER_MIXED_GMG,
           "mixed_gmg_learned": nhmf.NHMF_SOLVER_MIXED_GMG_LEARNED}
    du_err = torch.from_numpy(inp.draw_vector(77, w.n_dofs)).to(dev)

    def fp32_error(uu):
        """FP32 apply (cached and on the fly) vs the FP64 cached apply at the linearisation point
        uu; the FP64 apply equals the oracle's to 1e-12 (parity tests, at full size too)."""
        prob.set_linearization(uu, nhmf.NHMF_CACHE_FP64 | nhmf.NHMF_CACHE_FP32)
        v64 = torch.empty_like(du_err)
        v32 = torch.empty(w.n_dofs, dtype=torch.float32, device=dev)
        prob.apply(du_err, v64, nhmf.NHMF_FP64, nhmf.NHMF_CACHED)
        out = {}
        for sname, sid in (("cached", nhmf.NHMF_CACHED), ("otf", nhmf.NHMF_ON_THE_FLY)):
            prob.apply(du_err.float(), v32, nhmf.NHMF_FP32, sid)
            out[sname] = float(torch.linalg.norm(v32.double() - v64) / torch.linalg.norm(v64))
        return out

    out = {"metric": NEWTON_METRIC, "mode": "newton", "workload": f"{w.name}: " + describe(w) +
           f"; {S} load steps of {w.compression / S:g}", "steps_run": last, "solvers": {},
           "outer_apply": args.outer + " (flexible solvers; plain Jacobi-CG always FP64)",
           "smoother": {"degree": args.smoother_degree or 3, "range": args.smoother_range or 15.0}}
    states = {}
    for name in solvers:
        u = torch.zeros(w.n_dofs, dtype=torch.float64, device=dev)
        per = []
        first = 1
        if name in LEARNED:
            # start from the recording solver's state after the training steps
            first = args.train_steps + 1
            u = states[base_solver][args.train_steps - 1].clone()
        for step in range(first, last + 1):
            kw = dict(base, first_step=step, last_step=step, solver=ids[name],
                      outer_apply=nhmf.NHMF_FP64 if name == "plain" else outer)
            if name == base_solver and learned and step <= args.train_steps:
                if base_solver == "plain":
                    kw.update(record_pairs=1, cg_pair_every=8, synthetic_pairs=args.synthetic)
                else:
                    kw.update(record_pairs=1, cg_pair_every=args.gmg_pair_iters)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = prob.solve(u, **kw)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            states.setdefault(name, []).append(u.clone())
            rec = {"step": step, "seconds": dt, "newton": st["newton_iters"][0], "outer": st["linear_iters"][0],
                   "inner": st["inner_iters"][0], "fallbacks": st["fallbacks"][0], "rel_residual": st["rel_residual"][0]}
            per.append(rec)
            if name == base_solver and learned and step == args.train_steps:
                t0 = time.perf_counter()
                l0, l1 = nhmf.nhmf_unet_train(prob.ctx, args.epochs, 1e-3)
                torch.cuda.synchronize()
                out["training"] = {"pairs": nhmf.nhmf_unet_num_pairs(prob.ctx), "epochs": args.epochs,
                                   "loss_first": l0, "loss_last": l1, "seconds": time.perf_counter() - t0}
        out["solvers"][name] = {"steps": per, "seconds": sum(r["seconds"] for r in per),
                                "outer": sum(r["outer"] for r in per), "inner": sum(r["inner"] for r in per),
                                "newton": sum(r["newton"] for r in per), "fallbacks": sum(r["fallbacks"] for r in per)}
    # per-step agreement with the reference solver's states (plain if it ran, else the first)
    ref_solver = "plain" if "plain" in states else (solvers[0] if solvers else None)
    if ref_solver in states:
        refs = states[ref_solver]
        for name, lst in states.items():
            off = args.train_steps if name in LEARNED else 0
            for k, uu in enumerate(lst):
                rec = out["solvers"][name]["steps"][k]
                ref = refs[k + off]
                rec[f"rel_diff_vs_{ref_solver}"] = float(torch.linalg.norm(uu - ref) / torch.linalg.norm(ref))
    # FP32 apply error vs the FP64 apply at each converged state of the first solver
    first_solver = solvers[0] if solvers else None
    if first_solver in states:
        for k, uu in enumerate(states[first_solver]):
            out["solvers"][first_solver]["steps"][k]["fp32_apply_rel_err_vs_fp64"] = fp32_error(uu)
    sp = out["solvers"]
    for ref_name in ("plain", "mixed_gmg"):
        if ref_name not in sp:
            continue
        for name in sp:
            if name == ref_name:
                continue
            off = args.train_steps if name in LEARNED else 0
            t_ref = sum(r["seconds"] for r in sp[ref_name]["steps"][off:])
            sp[name][f"speedup_vs_{ref_name}_same_steps"] = t_ref / sp[name]["seconds"] if sp[name]["seconds"] else None
    print(json.dumps(out), flush=True)
    prob.close()
    return 0


# ------------------------------------------------------------------ U-Net mode
def unet_flops(M):
    """Algorithmic FLOPs of one forward pass on an M^3 grid: 2 * 27 * c_in * c_out per output
    voxel of each stride-1 and stride-2 convolution, and per coarse input voxel of each
    transposed convolution (the channel counts the network defines; 3-channel ends counted
    at 3)."""
    M1 = (M - 1) // 2 + 1
    M2 = (M1 - 1) // 2 + 1
    v0, v1, v2 = M ** 3, M1 ** 3, M2 ** 3
    macs = 27 * (v0 * 3 * 16 + v0 * 256 + v1 * 256 + v1 * 256 + v2 * 256 + v2 * 256 + v2 * 256 +
                 v1 * 256 + v1 * 256 + v0 * 256 + v0 * 16 * 3)
    return 2.0 * macs


def run_unet(args):
    """Forward pass and one training step (forward, loss, backward, Adam) of the U-Net on the
    Q2 64^3 nodal grid (129^3), timed with CUDA events over `steps` repetitions."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2505_15535_gb300 import nhmf
    w = inp.WORKLOADS["q2_64_compress"]
    M = w.n_nodes_1d
    dev = torch.device("cuda", 0)
    prob = nhmf.Problem(w.n_el, w.degree, w.mu, w.lam, w.bc)
    nhmf.nhmf_unet_create(prob.ctx, 1)
    nhmf.nhmf_unet_set_params(prob.ctx, he_init_flat())
    x = torch.from_numpy(inp.normal(31, w.n_dofs)).to(dev)
    e = torch.from_numpy(inp.normal(32, w.n_dofs)).to(dev)
    nhmf.nhmf_unet_record_pair(prob.ctx, x, e)
    xf = x.float()
    y = torch.empty_like(xf)
    st = torch.cuda.current_stream()
    for _ in range(args.warmup):
        nhmf.nhmf_unet_forward(prob.ctx, xf, y)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    for _ in range(args.steps):
        nhmf.nhmf_unet_forward(prob.ctx, xf, y)
    b.record(st)
    torch.cuda.synchronize()
    fwd_ms = a.elapsed_time(b) / args.steps
    t0 = time.perf_counter()
    nhmf.nhmf_unet_train(prob.ctx, args.steps, 1e-4)
    torch.cuda.synchronize()
    train_ms = (time.perf_counter() - t0) / args.steps * 1e3
    fl = unet_flops(M)
    peak = MEASURED.get("bf16_tflops")
    out = {"mode": "unet", "grid": f"{M}^3 (Q2 64^3 nodes)", "forward_ms": fwd_ms,
           "forward_tflops": fl / (fwd_ms * 1e-3) / 1e12, "train_step_ms": train_ms,
           "train_tflops": 3 * fl / (train_ms * 1e-3) / 1e12, "flops_forward": fl,
           "bf16_peak_tflops_measured": peak,
           "forward_frac_of_bf16_peak": (fl / (fwd_ms * 1e-3) / 1e12 / peak) if peak else None}
    print(json.dumps(out), flush=True)
    prob.close()
    return 0


def _measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


MEASURED = _measured_peaks()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--strategy", choices=["cached", "otf", "spatial"], default="cached",
                    help="apply and kernel modes (spatial: kernel mode only)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-newton", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--mode", choices=["apply", "newton", "unet", "kernel"], default="apply")
    ap.add_argument("--precision", choices=["fp64", "fp32", "df64"], default="fp64",
                    help="kernel mode: arithmetic of the apply")
    ap.add_argument("--workload", default="q2_64_compress")
    ap.add_argument("--apply-workload", default=MAIN)
    ap.add_argument("--solvers", default="plain,mixed,learned,mixed_learned")
    ap.add_argument("--last-step", type=int, default=0)
    ap.add_argument("--train-steps", type=int, default=5)
    ap.add_argument("--synthetic", type=int, default=8)
    ap.add_argument("--pairs", type=int, default=150)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--outer", choices=["fp64", "df64"], default="fp64",
                    help="newton mode: arithmetic of the flexible solvers' outer applies")
    ap.add_argument("--gmg-pair-iters", type=int, default=4,
                    help="newton mode: pairs per linear solve recorded by mixed_gmg for mixed_gmg_learned")
    ap.add_argument("--smoother-degree", type=int, default=0,
                    help="multigrid solvers: Chebyshev steps per smoothing (0: the library's default, 3)")
    ap.add_argument("--smoother-range", type=float, default=0.0,
                    help="multigrid solvers: lmax / lmin of the Chebyshev interval (0: the library's default, 15)")
    ap.add_argument("--linear-rtol", type=float, default=1e-8)
    ap.add_argument("--inner-rtol", type=float, default=1e-3)
    ap.add_argument("--inner-max-iter", type=int, default=1000)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "kernel":
        return run_kernel(args)
    if args.mode == "newton":
        return run_newton(args)
    if args.mode == "unet":
        return run_unet(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
