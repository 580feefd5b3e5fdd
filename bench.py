#!/usr/bin/env python
"""Benchmark: time to a 1e-8 relative residual of MGR-preconditioned FGMRES.

Headline workload (the largest single-GPU configuration): the compositional
flow system with wells on a 128x128x32 grid, 4x4 blocks (pressure and three
component masses per cell) plus 16 vertical wells (well pressure, rate;
padded to 4x4), 2,097,216 unknowns; three-level MGR (component masses
block-Jacobi, wells exact 2x2, pressure AMG V(1,1)) inside FGMRES(30), x0 = 0.
A step is one complete solve to ||b - A x|| <= 1e-8 ||b|| with the inputs
resident in HBM; setup is timed separately.  `value` is the plain FP64 form;
the FP32-preconditioner form (V-cycle stored and run in FP32 inside FP64
FGMRES) is measured in the same run, and both solutions are compared with
the CPU oracle's.  L2 (129 MB) is flushed by a 256 MB write before every
timed step.  The other configurations (the 64^3 hybrid mimetic system among
them) are reported under `configs`.

`--impl reference` times the CPU oracle (plain C, OpenMP over the solve
loops on every core of the affinity set) on the same system, one full solve
per step.
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

METRIC = "time to 1e-8 rel. residual, FP64 vs FP32-MGR; V-cycle HBM GB/s vs 8 TB/s"
# GB300 nominal FP64 rate (2 flops per FMA), used only when the measurement
# of the device's FP64 FMA rate fails
FP64_NOMINAL_GFLOPS = 1250.0
HEADLINE = "compositional_128x128x32"
DESCR = {
    "two_phase_16x16x8": "two-phase TPFA 16x16x8, 2x2 blocks, MGR (saturation l1-Jacobi, pressure AMG)",
    "mimetic_64": "hybrid mimetic single-phase 64^3, MGR_P (cells Jacobi, faces AMG V(1,1))",
    "mimetic_64_tpfa_mgr_pi": "mimetic 64^3 TPFA, MGR_Pi (faces Jacobi, cells AMG V(1,1))",
    "compositional_128x128x32": ("compositional 128x128x32 + 16 wells, 4x4 blocks, 3-level MGR "
                                 "(component masses block-Jacobi, wells exact 2x2, pressure AMG V(1,1))"),
    "compositional_128x128x32_4level": ("compositional 128x128x32 + 16 wells, 4x4 blocks, the 4-level "
                                        "order of Sec. 4.2 (wells on the coarsest grid)"),
    "poromech_64": "poromechanics 64^3 + 48x48 fracture, 3x3 blocks, MGR_P (fracture p l1-Jacobi, "
                   "displacement AMG, 3 functions)",
    "poromech_64_mgr_u": "poromechanics 64^3 + 48x48 fracture, 3x3 blocks, MGR_U (displacement AMG "
                         "F-relaxation, fracture p AMG)",
}
OTHER_CONFIGS = ("mimetic_64", "two_phase_16x16x8", "mimetic_64_tpfa_mgr_pi",
                 "compositional_128x128x32_4level", "poromech_64", "poromech_64_mgr_u")
L2_NOTE = "256 MB write before every timed step"


def workload(name, n):
    return f"{DESCR.get(name, name)} ({n:,} unknowns), FGMRES(30)"


def config_dict(args, name, n, world):
    """The workload's description; both arms print this same dict."""
    return {"workload": workload(name, n), "config": name, "unknowns": int(n), "rtol": args.rtol,
            "l2": L2_NOTE,
            "parallelism": f"{world} independent replicas" if world > 1 else "single GPU"}


def newton_values(cs, k):
    """The values of a later Newton step of a fracture system: the blocks in
    pressure rows or columns scaled by seeded U[0.9, 1.1] (the displacement
    block and the identity padding unchanged)."""
    rng = np.random.default_rng(1000 + k)
    NN = (cs.meta["ne"] + 1) ** 3
    rows = np.repeat(np.arange(cs.nb), np.diff(cs.row_ptr))
    sel = (rows >= NN) | (cs.col_idx >= NN)
    val = cs.val.copy()
    val[sel] *= rng.uniform(0.9, 1.1, int(sel.sum()))[:, None, None]
    if cs.n_pad:
        last = np.flatnonzero((rows == cs.nb - 1) & (cs.col_idx == cs.nb - 1))[0]
        for q in range(cs.b - cs.n_pad, cs.b):
            val[last, q, q] = cs.val[last, q, q]
    return val

def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--config", default=HEADLINE, choices=sorted(DESCR))
    p.add_argument("--rtol", type=float, default=1e-8)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-profile", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-configs", action="store_true")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 50 ms) of SM clock and throttle reasons; only
    samples stamped inside the marked region count."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            # wait for the first sample so the region is covered from its start
            deadline = time.time() + 5.0
            while time.time() < deadline and os.path.getsize(self.f.name) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    @staticmethod
    def _stamp(text):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(text, fmt).timestamp()
            except ValueError:
                pass
        return None

    def summary(self):
        if not self.f:
            return None
        self.f.flush()
        rows = []
        try:
            for line in open(self.f.name):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        except Exception:
            return None
        finally:
            try:
                os.unlink(self.f.name)
            except Exception:
                pass
        if self.t0 is not None and self.t1 is not None:
            inside = [r for r in rows
                      if (lambda ts: ts is not None and self.t0 - 0.05 <= ts <= self.t1 + 0.05)(self._stamp(r[0]))]
        else:
            inside = rows
        if not inside:
            return None
        sm = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in inside if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(inside),
                "interval_ms": 50}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "gb300" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v, dev):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sources_sha1(names):
    """SHA-1 over the named kernel sources (csrc/), in the given order."""
    import hashlib
    h = hashlib.sha1()
    for name in names:
        h.update(open(os.path.join(ROOT, "paper_2101_11649_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def ncu_traffic(config, kernel_class):
    """DRAM bytes per launch of a kernel class of a configuration from the
    committed ncu capture (profiles/traffic.json), or None when there is
    none or the sources of that kernel (its entry's "sources") changed
    since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
        k = d.get("configs", {}).get(config, {}).get(kernel_class)
        if not k or "note" in k or k.get("sources_sha1") != sources_sha1(k["sources"]):
            return None
    except Exception:
        return None
    return k["dram_bytes"]


def make_system(name):
    from paper_2101_11649_gb300.synth import CONFIGS
    return CONFIGS[name]()


def oracle_solves(o, sysm, rtol, steps, warmup):
    """`warmup` + `steps` full oracle solves; per-step ms, iterations and the
    last solution."""
    for _ in range(warmup):
        o.solve(sysm.rhs, rtol=rtol, maxit=1000)
    ts, its, r = [], [], None
    for _ in range(steps):
        t0 = time.perf_counter()
        r = o.solve(sysm.rhs, rtol=rtol, maxit=1000)
        ts.append((time.perf_counter() - t0) * 1e3)
        its.append(r["iters"])
    return ts, its, r


def run_reference(args, world, rank):
    if rank != 0:
        return
    from oracle import oracle as O
    sysm = make_system(args.config)
    cores = O.set_threads(O.affinity_cores())
    o = O.Oracle(sysm)
    ts, its, _ = oracle_solves(o, sysm, args.rtol, args.steps, args.warmup)
    ms = statistics.mean(ts)
    sample = (f"{args.warmup} warm-up + {args.steps} timed full solves to {args.rtol:g} of the "
              f"whole workload (setup untimed), {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": round(ms, 3), "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, args.config, sysm.n, world),
            "iterations": its[-1] if its else None,
            "cpu_baseline": {"value": round(ms, 3), "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(ms, 3), "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    torch.cuda.set_device(local)
    # every launch and every timing event of this arm on one (non-legacy) stream:
    # the solvers take the current stream at construction
    with torch.cuda.stream(torch.cuda.Stream()):
        run_gb300(args, world, rank, local)


def error_vs(x, xo, sysm):
    """Error of a GPU solution against the oracle's: relative 2-norm, the
    largest entry difference over the largest oracle entry, and the same per
    MGR level's F set and the final coarse block (the worst of them)."""
    d = np.abs(x - xo)
    lv = np.asarray(sysm.dof_level)
    per_set = 0.0
    for l in range(int(sysm.num_levels) + 1):
        S = lv == l
        if S.any():
            per_set = max(per_set, float(d[S].max() / max(np.abs(xo[S]).max(), 1e-300)))
    return {"rel_l2": float(np.linalg.norm(x - xo) / np.linalg.norm(xo)),
            "max_rel": float(d.max() / np.abs(xo).max()), "max_rel_per_set": per_set}


def run_gb300(args, world, rank, local):
    import torch
    from paper_2101_11649_gb300 import mgr as M

    dev = torch.device("cuda", local)
    peak_gbs, peak_kind = peaks()
    try:
        fp64_gflops = round(2.0 * M.measure_fp64_fma(10) / 1e9, 1)
        fp64_kind = "measured: independent FMA chains on every SM, best of 10 launches"
    except Exception:
        fp64_gflops, fp64_kind = FP64_NOMINAL_GFLOPS, "nominal"
    name = args.config
    sysm = make_system(name)
    n = sysm.n
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def ev_ms(fn, reps):
        """median of reps event-timed calls (L2 flushed before each)"""
        ts, out = [], None
        for _ in range(reps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st); out = fn(); e1.record(st); e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), out

    def vcycle_of(sv, nn):
        """one V-cycle: algorithmic bytes from one profiled apply, time from
        event-timed applies"""
        v = torch.randn(nn, dtype=torch.float64, device=dev)
        z = torch.empty_like(v)
        sv.profile(True)
        sv.apply(v, z)
        tab = sv.profile_table()
        sv.profile(False)
        vbytes = sum(r["bytes_per_launch"] * r["launches"] for r in tab)
        vfma = sum(r["fp64_fma_per_launch"] * r["launches"] for r in tab)
        vms, _ = ev_ms(lambda: sv.apply(v, z), 20)
        return {"ms": round(vms, 4), "bytes": vbytes, "kernels": len(tab),
                "gbs": round(vbytes / (vms / 1e3) / 1e9, 1),
                "frac": round(vbytes / (vms / 1e3) / 1e9 / peak_gbs, 4),
                "fp64_gflops": round(2 * vfma / (vms / 1e3) / 1e9, 1),
                "fp64_frac": round(2 * vfma / (vms / 1e3) / 1e9 / fp64_gflops, 4)}

    def spmv_of(sv, cs):
        """the outer block product alone against its algorithmic bytes"""
        xq = torch.randn(cs.n, dtype=torch.float64, device=dev)
        yq = torch.empty_like(xq)
        for _ in range(3):
            sv.spmv(xq, yq)
        ms, _ = ev_ms(lambda: sv.spmv(xq, yq), 20)
        by = cs.col_idx.size * (cs.b * cs.b * 8 + 4) + 4 * (cs.nb + 1) + 16 * cs.n
        fma = cs.col_idx.size * cs.b * cs.b
        return {"us": round(ms * 1e3, 2), "gbs": round(by / (ms / 1e3) / 1e9, 1),
                "frac": round(by / (ms / 1e3) / 1e9 / peak_gbs, 4),
                "fp64_frac": round(2 * fma / (ms / 1e3) / 1e9 / fp64_gflops, 4)}

    def timed_setup(system, prec, reps=3):
        """median wall time of `reps` setups after an untimed one (the first
        launches of a process also load the kernels); returns the last solver"""
        M.MGRSolver.from_system(system, precision=prec).close()
        ts, sv = [], None
        for _ in range(reps):
            if sv is not None:
                sv.close()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sv = M.MGRSolver.from_system(system, precision=prec)
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        return sv, statistics.median(ts)

    s64, setup64_ms = timed_setup(sysm, "fp64")
    s32, setup32_ms = timed_setup(sysm, "fp32")

    b = torch.as_tensor(sysm.rhs, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)

    def solve(sv):
        x.zero_()
        _, info = sv.solve(b, x, rtol=args.rtol, maxit=1000)
        if info["status"] != 0:
            raise RuntimeError(f"solve failed: {info}")
        return info

    def timed(sv, k):
        """k solves, each bracketed by CUDA events on the current stream, L2
        flushed before each; returns per-step ms and the last info."""
        times, info = [], None
        for _ in range(k):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            info = solve(sv)
            e1.record(st)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return times, info

    for _ in range(args.warmup):
        solve(s64)
        solve(s32)

    # ---- timed region (FP64 headline, then FP32-MGR), clocks sampled during it
    barrier(world)
    torch.cuda.synchronize()
    l0 = M.launch_count()
    with ClockSampler(local) as cs_:
        cs_.start()
        t64, info64 = timed(s64, args.steps)
        torch.cuda.synchronize()
        x64 = x.cpu().numpy()
        barrier(world)
        t32, info32 = timed(s32, args.steps)
        torch.cuda.synchronize()
        cs_.stop()
    x32 = x.cpu().numpy()
    launches = M.launch_count() - l0
    clocks = cs_.summary()
    ms64 = max_over_ranks(world, statistics.mean(t64), dev)
    ms32 = max_over_ranks(world, statistics.mean(t32), dev)

    # ---- per-kernel-class event timing over a second timed pass
    roofline, kernels = None, []
    vcycle = {}
    if not args.no_profile:
        s64.profile(True)
        timed(s64, args.steps)
        kernels = s64.profile_table()
        s64.profile(False)
        kernels.sort(key=lambda r: -r["ms"])
        top = kernels[0]
        avg_s = top["ms"] / top["launches"] / 1e3
        gbs = top["bytes_per_launch"] / avg_s / 1e9
        gflops = 2.0 * top["fp64_fma_per_launch"] / avg_s / 1e9
        hbm_frac, alu_frac = gbs / peak_gbs, gflops / fp64_gflops
        alu = alu_frac > hbm_frac
        for pname, sv in (("fp64", s64), ("fp32", s32)):
            vcycle[pname] = vcycle_of(sv, n)
        roofline = {"bound": "alu" if alu else "hbm", "kernel": top["name"],
                    "achieved": round(gflops if alu else gbs, 1),
                    "peak": fp64_gflops if alu else peak_gbs,
                    "peak_kind": f"FP64 FMA rate, {fp64_kind}" if alu else f"HBM copy, {peak_kind}",
                    "unit": "GFLOP/s" if alu else "GB/s",
                    "frac": round(alu_frac if alu else hbm_frac, 4),
                    "traffic": ncu_traffic(name, top["name"]),
                    "hbm": {"achieved": round(gbs, 1), "peak": peak_gbs, "frac": round(hbm_frac, 4)},
                    "fp64": {"achieved": round(gflops, 1), "peak": fp64_gflops,
                             "frac": round(alu_frac, 4)},
                    "avg_launch_us": round(avg_s * 1e6, 2),
                    "bytes_per_launch": top["bytes_per_launch"],
                    "fp64_fma_per_launch": top["fp64_fma_per_launch"],
                    "share_of_solve": round(top["ms"] / sum(k["ms"] for k in kernels), 4),
                    # the MGR V-cycle as one unit (all its launches): algorithmic
                    # bytes of one cycle over its event time, both forms
                    "vcycle": {p: {"gbs": v["gbs"], "frac": v["frac"], "ms": v["ms"],
                                   "bytes": v["bytes"]} for p, v in vcycle.items()}}

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        bh = torch.as_tensor(sysm.rhs).pin_memory()
        xh = torch.empty(n, dtype=torch.float64).pin_memory()
        bd = torch.empty(n, dtype=torch.float64, device=dev)
        xd = torch.empty(n, dtype=torch.float64, device=dev)
        ts = []
        for k in range(args.warmup + args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bd.copy_(bh, non_blocking=True)
            xd.zero_()
            _, info = s64.solve(bd, xd, rtol=args.rtol, maxit=1000)
            xh.copy_(xd, non_blocking=True)
            torch.cuda.synchronize()
            if k >= args.warmup:
                ts.append((time.perf_counter() - t0) * 1e3)
        # host wall clock: the median over steps (one host stall must not decide
        # it); the mean is reported beside it
        e2e = {"value": round(max_over_ranks(world, statistics.median(ts), dev), 3), "unit": "ms",
               "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8,
               "mean_ms": round(statistics.mean(ts), 3), "max_ms": round(max(ts), 3)}
    headline_spmv = spmv_of(s64, sysm)
    s64.close()
    s32.close()

    # ---- batched form: 48 uneven two-phase systems, one launch per kernel class
    batched = None
    if not args.no_batched:
        from paper_2101_11649_gb300.synth import make_batch
        systems, _ = make_batch(48)
        nunk = sum(q.n for q in systems)
        rhs = [torch.as_tensor(q.rhs, device=dev) for q in systems]
        batched = {"workload": f"48 two-phase TPFA systems, grids 16^3..96x96x48, {nunk} unknowns",
                   "rtol": args.rtol}
        for prec in ("fp64", "fp32"):
            t0 = time.perf_counter()
            bt = M.MGRBatch(systems, precision=prec)
            torch.cuda.synchronize()
            setup_ms = (time.perf_counter() - t0) * 1e3
            for _ in range(max(1, args.warmup)):
                bt.solve(rhs, rtol=args.rtol)
            ms, (_, infos) = ev_ms(lambda: bt.solve(rhs, rtol=args.rtol), max(1, min(args.steps, 5)))
            its = [i["iterations"] for i in infos]
            batched[prec] = {"ms": round(ms, 3), "setup_ms": round(setup_ms, 1),
                             "iterations_max": max(its), "iterations_mean": round(sum(its) / len(its), 2),
                             "all_converged": all(i["status"] == 0 for i in infos),
                             "unknowns_per_s": round(nunk / (ms / 1e3), 1)}
            # the batched V-cycle against HBM: each member's cycle bytes (a
            # profiled apply through its own handle) times its iterations,
            # over the summed event time of the batched V-cycle launches of
            # one profiled batched solve (graphs off while profiling)
            vbytes = 0.0
            for i, q in enumerate(systems):
                sv = bt.system(i)
                v = torch.randn(q.n, dtype=torch.float64, device=dev)
                sv.profile(True)
                sv.apply(v, torch.empty_like(v))
                vb = sum(r["bytes_per_launch"] * r["launches"] for r in sv.profile_table())
                sv.profile(False)
                vbytes += vb * its[i]
            sv0 = bt.system(0)
            sv0.profile(True)
            bt.solve(rhs, rtol=args.rtol)
            tab = sv0.profile_table()
            sv0.profile(False)
            outside = ("batched_spmv_A", "batched_arnoldi", "batched_givens", "batched_vec_scale",
                       "batched_residual")
            vms = sum(r["ms"] for r in tab if not r["name"].startswith(outside))
            if vms > 0:
                batched[prec]["vcycle"] = {"bytes": vbytes, "ms": round(vms, 3),
                                           "gbs": round(vbytes / (vms / 1e3) / 1e9, 1),
                                           "frac": round(vbytes / (vms / 1e3) / 1e9 / peak_gbs, 4)}
            if prec == "fp64":
                # the same systems one after another through their single-system handles
                seq = 0.0
                for i in range(len(systems)):
                    sv = bt.system(i)
                    x1 = torch.zeros_like(rhs[i])
                    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    sv.solve(rhs[i], x1, rtol=args.rtol)
                    e1.record(st)
                    e1.synchronize()
                    seq += e0.elapsed_time(e1)
                batched["sequential_fp64_ms"] = round(seq, 3)
                batched["speedup_vs_sequential_fp64"] = round(seq / ms, 3)
            bt.close()

    # ---- the other configurations: setup, solve times, V-cycle and outer product
    configs = None
    if not args.no_configs:
        configs = {}
        for cname in OTHER_CONFIGS:
            if cname == name:
                continue
            cs = make_system(cname)
            bq = torch.as_tensor(cs.rhs, device=dev)
            ent = {"n": cs.n, "b": cs.b, "nnzb": int(cs.col_idx.size), "mgr_levels": cs.num_levels}
            for prec in ("fp64", "fp32"):
                sv, sms = timed_setup(cs, prec)
                ent[f"setup_{prec}_ms"] = round(sms, 1)
                for _ in range(2):
                    sv.solve(bq, rtol=args.rtol)
                ms, (_, inf) = ev_ms(lambda: sv.solve(bq, rtol=args.rtol), 5)
                ent[f"{prec}_ms"] = round(ms, 3)
                ent[f"{prec}_iterations"] = inf["iterations"]
                ent[f"{prec}_rel_residual"] = inf["rel_residual"]
                vc = vcycle_of(sv, cs.n)
                ent[f"vcycle_{prec}"] = {"ms": vc["ms"], "gbs": vc["gbs"], "frac": vc["frac"]}
                if prec == "fp64":
                    ent["spmv"] = spmv_of(sv, cs)
                    if cs.meta.get("strategy") == "mgr_u":
                        # setup reuse: a Newton step that changes the pressure
                        # rows and couplings, not the relaxed block
                        ts_ = []
                        for k in range(3):
                            # the Jacobian of a Newton step is assembled on the device
                            vk = torch.as_tensor(newton_values(cs, k), device=dev)
                            torch.cuda.synchronize()
                            t0 = time.perf_counter()
                            sv.refresh(vk)
                            torch.cuda.synchronize()
                            ts_.append((time.perf_counter() - t0) * 1e3)
                        ent["refresh_fp64_ms"] = round(statistics.median(ts_), 1)
                        _, rinf = sv.solve(bq, rtol=args.rtol)
                        ent["refresh_fp64_iterations"] = rinf["iterations"]
                sv.close()
            configs[cname] = ent

    # ---- CPU oracle baseline (rank 0, N = 1 only): all cores and one thread;
    # its solution also gives the error of each GPU result
    cpu, errors = None, None
    setup = {"gpu_fp64_ms": round(setup64_ms, 1), "gpu_fp32_ms": round(setup32_ms, 1)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        cores = O.set_threads(O.affinity_cores())
        t0 = time.perf_counter()
        o = O.Oracle(sysm)
        osetup = (time.perf_counter() - t0) * 1e3
        ts, its, ro = oracle_solves(o, sysm, args.rtol, 1, 0)
        O.set_threads(1)
        ts1, _, _ = oracle_solves(o, sysm, args.rtol, 1, 0)
        O.set_threads(cores)
        o.close()
        setup["oracle_ms"] = round(osetup, 1)
        setup["oracle_threads"] = 1
        setup["speedup_fp64"] = round(osetup / setup64_ms, 1)
        cpu = {"value": round(ts[0], 1), "unit": "ms", "cores": cores, "kind": "oracle",
               "sample": f"one full solve of the same system to {args.rtol:g} (setup untimed), "
                         f"{cores} threads, {its[0]} iterations",
               "single_thread_ms": round(ts1[0], 1)}
        xo = ro["x"]
        errors = {"vs": f"the oracle's FP64 solution of the same system at rtol {args.rtol:g}",
                  "fp64": error_vs(x64, xo, sysm), "fp32_mgr": error_vs(x32, xo, sysm)}

    if rank == 0:
        line = {"metric": METRIC, "value": round(ms64, 3), "unit": "ms", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms64, 3),
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": config_dict(args, name, n, world),
                "solves_per_s_job": round(world * 1e3 / ms64, 2),
                "iterations": info64["iterations"], "rel_residual": info64["rel_residual"],
                "fp32_mgr": {"ms": round(ms32, 3), "iterations": info32["iterations"],
                             "rel_residual": info32["rel_residual"],
                             "speedup_vs_fp64": round(ms64 / ms32, 3),
                             "error_vs_oracle": errors["fp32_mgr"] if errors else None},
                "error_vs_oracle": errors,
                "peaks": {"hbm_gbs": peak_gbs, "hbm_kind": peak_kind,
                          "fp64_gflops": fp64_gflops, "fp64_kind": fp64_kind},
                "setup_ms": {"fp64": round(setup64_ms, 1), "fp32": round(setup32_ms, 1)},
                "setup": setup, "spmv": headline_spmv,
                "levels": {"mgr": info64["mgr_levels"], "amg": info64["amg_levels"],
                           "rows": info64["level_rows"], "nnz": info64["level_nnz"],
                           "operator_complexity": round(info64["operator_complexity"], 3)},
                "vcycle": vcycle, "batched": batched, "configs": configs,
                "kernels": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()}
                            for r in kernels[:12]],
                "gpu_launches": int(launches), "clocks": clocks, "e2e": e2e,
                "cpu_baseline": cpu, "roofline": roofline}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
