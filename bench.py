"""Benchmark: time-to-1e-10-residual of the mixed-precision even-odd CG solver
on one GB300, against plain FP64 CG, with the hopping stencil's roofline.

One step = one complete solve D x = b (FP64 true residual <= 1e-10 on all
sites): link preparation is cached per gauge field, everything else (source
preparation, the CG iterations with their reliable updates, reconstruction of
the odd sites, the final FP64 residual) runs inside the step.  Inputs are
resident in HBM when the timed region starts.  value = solves per second over
all ranks.  Under torchrun every rank solves its own seeded system (weak
scaling, no collective on the data path; a barrier brackets the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--inner f16|bf16|f32|f64] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import ctypes
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

METRIC = "CG time-to-1e-10 residual & Dslash GB/s (% HBM peak), mixed vs FP64 CG on GB300"
DEFAULT_WORKLOAD = "wilson_32x32x32x64_exp0.6"
# iteration count of plain FP64 CG on the normal equations over the full
# lattice (the oracle's algorithm) for each seeded workload, used to scale the
# oracle's per-iteration time to a time-to-solution
# (measured by running the oracle's own CGNR to 1e-10 on the seeded systems)
ORACLE_CGNR_ITERS = {"wilson_32x32x32x64_exp0.6": 100, "wilson_16x16x16x32_exp0.4": 173}


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def aggregate_throughput(local_ms, steps, world, device):
    """Whole-job throughput: every rank solved `steps` systems in its own
    timed region; the job's time is the slowest rank's (MAX all-reduce, the
    only collective, outside the timed region).  Returns (solves/s, max ms)."""
    total_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    return world * steps / (total_ms / 1e3), total_ms


def rank_source_seed(workload, rank):
    """Seed of the source solved by `rank`: rank 0 solves the workload's own
    system, every other rank an independent seeded source on the same links."""
    from paper_2001_05218_gb300 import inputs as I
    base = I.workload_seed(I.WORKLOADS[workload]["index"])
    return base if rank == 0 else base + 1000 * rank


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        """Starts sampling every 50 ms and waits (up to 5 s) for the first
        sample, so that the region marked next is covered from its start."""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_end = time.monotonic() + 5.0
            while not self.lines and time.monotonic() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark(self):
        """Start of the timed region."""
        self.t0 = time.monotonic()

    def stop(self):
        """Samples taken between mark() and now (plus the one that follows)."""
        t1 = time.monotonic()
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t_end = t1 + 0.5
        while not any(t >= t1 for t, _ in self.lines) and time.monotonic() < t_end:
            time.sleep(0.01)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        t0 = getattr(self, "t0", 0.0)
        after = [t for t, _ in self.lines if t >= t1]
        t_last = min(after) if after else t1
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in self.lines:
            if t < t0 or t > t_last:
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_hash():
    """Hash of the code (comments and blank lines removed) of the files that
    define the stencil kernel (storage formats and the kernel template): a
    DRAM-traffic figure is only reported for the kernel it was measured on."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2001_05218_gb300", "csrc")
    for f in ("dw_common.cuh", "dw_kernels.cuh"):
        text = open(os.path.join(csrc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = [ln.rstrip() for ln in text.splitlines() if ln.strip()]
        h.update("\n".join(code).encode())
    return h.hexdigest()[:16]


def ncu_traffic(workload, kernel_name):
    """DRAM bytes per launch of the stencil from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        e = d.get(workload, {}).get(kernel_name)
        if e and e.get("source_hash") == source_hash():
            return e.get("dram_bytes_per_launch_full")
    except Exception:
        return None
    return None


# ---------------------------------------------------------------------- reference arm (the CPU oracle)
def oracle_iteration_seconds(dims, kappa, U, b, reps):
    from oracle import oracle as O
    t0 = time.perf_counter()
    for _ in range(reps):
        w = O.dirac(dims, kappa, U, b)
        O.dirac(dims, kappa, U, w, dag=True)
    return (time.perf_counter() - t0) / reps


def cpu_baseline(workload, dims, kappa, U, b, iters_needed, budget_s=20.0):
    """The oracle timed on all host cores (the reported value) and on one
    core, per CGNR iteration, scaled by the iterations its CGNR needs."""
    from oracle import oracle as O
    O.build()
    cores = O.num_threads()
    t1 = oracle_iteration_seconds(dims, kappa, U, b, 1)
    reps = max(1, min(20, int(budget_s / max(t1, 1e-3))))
    t = oracle_iteration_seconds(dims, kappa, U, b, reps)
    solve_s = t * iters_needed
    O.set_num_threads(1)
    try:
        t_one = oracle_iteration_seconds(dims, kappa, U, b, 1)
    finally:
        O.set_num_threads(cores)
    return {"value": 1.0 / solve_s, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": "%d+1 CGNR iterations (D then D^dag, FP64, full lattice %s) of the oracle, %.3f s each, "
                      "scaled by the %d iterations plain FP64 CGNR needs on this system" %
                      (reps, "x".join(map(str, dims)), t, iters_needed),
            "single_core": {"value": 1.0 / (t_one * iters_needed), "unit": "solves/s", "cores": 1,
                            "s_per_iteration": t_one,
                            "sample": "1 CGNR iteration on one host core, scaled the same way"}}


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    from paper_2001_05218_gb300 import inputs as I
    from oracle import oracle as O
    O.build()
    dims, kappa, U, b = I.make_workload(args.workload)
    iters = ORACLE_CGNR_ITERS.get(args.workload)
    if iters is None:
        print(json.dumps({"impl": "reference", "unavailable": "no recorded oracle iteration count for %s"
                          % args.workload}))
        return
    for _ in range(args.warmup):
        oracle_iteration_seconds(dims, kappa, U, b, 1)
    ts = []
    for _ in range(args.steps):
        ts.append(oracle_iteration_seconds(dims, kappa, U, b, 1))
    t = float(np.mean(ts))
    value = 1.0 / (t * iters)
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * iters * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)", "impl": "reference",
            "config": {"workload": args.workload, "lattice": list(dims), "kappa": kappa},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": "each step: one CGNR iteration (D then D^dag, FP64, full lattice) of the "
                                       "oracle (%.3f s mean), scaled by the %d iterations plain FP64 CGNR needs"
                                       % (t, iters)},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------- stencil-only mode
def run_dslash(args):
    """Repeated even-site Schur applications Dhat = 1 - k^2 H_eo H_oe (two
    stencil launches each) in one storage precision, with L2 written over
    between applications; prints per-launch time and algorithmic GB/s.  Not
    the benchmark line: this is the small, targeted command used for kernel
    captures."""
    import torch
    torch.cuda.set_device(0)
    from paper_2001_05218_gb300 import dw
    from paper_2001_05218_gb300 import inputs as I
    prec = dw.PREC[args.dslash]
    c12 = args.compress12 if args.compress12 is not None else (1 if args.dslash in ("f16", "bf16", "i16") else 0)
    dims, kappa, U, b = I.make_workload(args.workload)
    V = int(np.prod(dims))
    s = np.arange(V)
    par = (s % dims[0] + (s // dims[0]) % dims[1] + (s // (dims[0] * dims[1])) % dims[2] +
           s // (dims[0] * dims[1] * dims[2])) % 2
    Ug = dw.gauge(dims, kappa, U, prec=prec, compress12=c12)
    src = b[par == 0] if args.nrhs == 1 else np.stack([np.roll(b[par == 0], r, axis=0) for r in range(args.nrhs)])
    x = dw.spinor(dims, src, kind=dw.DW_SPINOR_EVEN, prec=prec, nrhs=args.nrhs)
    y = dw.spinor(dims, kind=dw.DW_SPINOR_EVEN, prec=prec, nrhs=args.nrhs)
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    scratch = torch.empty(2 * l2, dtype=torch.uint8, device="cuda")
    if args.norm:  # the reducing epilogue: out and |out|^2 (FP64 grid reduction) in the second launch
        op = lambda U_, x_, y_: dw.apply_norm(U_, x_, y_)  # noqa: E731
    else:
        op = dw.laplace_apply if args.op == "laplace" else dw.apply
    for _ in range(max(1, args.warmup)):
        op(Ug, x, y)
    torch.cuda.synchronize()
    dw.profile_start(time_stencils=True)
    for _ in range(args.steps):
        scratch.fill_(1)
        op(Ug, x, y)
    prof, launches = dw.profile_stop()
    peak, kind = peaks()
    out = {"mode": "dslash", "op": args.op + ("+norm" if args.norm else ""), "workload": args.workload,
           "prec": args.dslash, "compress12": c12,
           "nrhs": args.nrhs,
           "kernels": {}}
    for k, e in prof.items():
        pl = e["total_ms"] / e["launches"]
        gbs = e["bytes"] / e["launches"] / (pl / 1e3) / 1e9
        out["kernels"][k] = {"launches": e["launches"], "ms_per_launch": pl,
                             "bytes_per_launch": e["bytes"] / e["launches"], "gbs": gbs, "frac_hbm": gbs / peak,
                             "gflops": e["flops"] / e["launches"] / pl / 1e6}
    out["peak_gbs"] = peak
    print(json.dumps(out))


# ---------------------------------------------------------------------- host transfer mode
def run_copies(args):
    """Host<->device copy times of the end-to-end step's buffers (U and b up,
    x down) with plain PyTorch copies between page-locked host memory and
    device memory, each synchronised and timed on the host; no library call.
    Shows the platform's copy rate per step, including its occasional slow
    steps, the same copies split over several streams, and DMA against SM
    kernels that access the page-locked memory directly (alone and together).
    Not the benchmark line."""
    import torch
    torch.cuda.set_device(0)
    from paper_2001_05218_gb300 import inputs as I
    dims = I.WORKLOADS[args.workload]["dims"]
    V = int(np.prod(dims))
    nU, nb = V * 4 * 9 * 2, V * 12 * 2  # float64 counts of complex128 U and one spinor
    Uh = torch.empty(nU, dtype=torch.float64).pin_memory()
    bh = torch.empty(nb, dtype=torch.float64).pin_memory()
    xh = torch.empty(nb, dtype=torch.float64).pin_memory()
    Ud = torch.empty(nU, dtype=torch.float64, device="cuda")
    bd = torch.empty(nb, dtype=torch.float64, device="cuda")

    def t(fn):
        a = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - a) * 1e3

    rows = []
    for _ in range(args.warmup + args.steps):
        rows.append([t(lambda: Ud.copy_(Uh, non_blocking=True)), t(lambda: bd.copy_(bh, non_blocking=True)),
                     t(lambda: xh.copy_(bd, non_blocking=True))])
    rows = np.array(rows[args.warmup:])
    med = np.median(rows, axis=0)
    gb = np.array([nU * 8, nb * 8, nb * 8]) / 1e9
    out = {"mode": "copies", "workload": args.workload, "bytes": [int(v * 1e9) for v in gb],
           "median_ms": med.round(3).tolist(), "median_gbs": (gb / (med / 1e3)).round(1).tolist(),
           "max_ms": rows.max(axis=0).round(3).tolist(),
           "slow_steps": [i for i, r in enumerate(rows) if np.any(r > 2 * med)],
           "step_ms": rows.round(2).tolist()}
    # the same copies split into k chunks on k streams (separate copy engines)
    split = {}
    for k in (2, 4, 8):
        streams = [torch.cuda.Stream() for _ in range(k)]

        def chunked(dst, src):
            n = dst.numel()
            step = (n + k - 1) // k
            cur = torch.cuda.current_stream()
            ev = torch.cuda.Event()
            ev.record(cur)
            for i, st_ in enumerate(streams):
                st_.wait_event(ev)
                with torch.cuda.stream(st_):
                    dst[i * step:(i + 1) * step].copy_(src[i * step:(i + 1) * step], non_blocking=True)
            for st_ in streams:
                cur.wait_stream(st_)

        ts = []
        for _ in range(args.warmup + args.steps):
            ts.append([t(lambda: chunked(Ud, Uh)), t(lambda: chunked(xh, bd))])
        ts = np.array(ts[args.warmup:])
        m = np.median(ts, axis=0)
        split[str(k)] = {"median_ms": m.round(3).tolist(),
                         "median_gbs": (gb[[0, 2]] / (m / 1e3)).round(1).tolist()}
    out["split_streams"] = split

    # DMA against an SM kernel reading / writing the page-locked buffer through
    # its device address (a tensor aliasing it), alone and together on two
    # streams over disjoint parts (fraction f by DMA)
    class _HostView:
        def __init__(self, h):
            self.__cuda_array_interface__ = {"shape": (h.numel(),), "typestr": "<f8", "data": (h.data_ptr(), False),
                                             "version": 3}

    Uv = torch.as_tensor(_HostView(Uh), device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def med_gbs(fn):
        ts = [t(fn) for _ in range(args.warmup + max(3, args.steps // 4))][args.warmup:]
        return round(gb[0] / (float(np.median(ts)) / 1e3), 1)

    def both(f, up):
        k = int(nU * f)
        cur = torch.cuda.current_stream()
        for st_ in (s1, s2):
            st_.wait_stream(cur)
        with torch.cuda.stream(s1):
            (Ud[:k].copy_(Uh[:k], non_blocking=True) if up else Uh[:k].copy_(Ud[:k], non_blocking=True))
        with torch.cuda.stream(s2):
            (torch.add(Uv[k:], 0.0, out=Ud[k:]) if up else torch.add(Ud[k:], 0.0, out=Uv[k:]))
        cur.wait_stream(s1)
        cur.wait_stream(s2)

    dma_sm = {"bytes": int(gb[0] * 1e9),
              "h2d": {"dma": med_gbs(lambda: Ud.copy_(Uh, non_blocking=True)),
                      "sm": med_gbs(lambda: torch.add(Uv, 0.0, out=Ud))},
              "d2h": {"dma": med_gbs(lambda: Uh.copy_(Ud, non_blocking=True)),
                      "sm": med_gbs(lambda: torch.add(Ud, 0.0, out=Uv))}}
    for f in (0.5, 0.6, 0.7, 0.8, 0.9):
        dma_sm["h2d"]["both_f%.1f" % f] = med_gbs(lambda: both(f, True))
        dma_sm["d2h"]["both_f%.1f" % f] = med_gbs(lambda: both(f, False))
    torch.cuda.synchronize()
    out["dma_vs_sm_gbs"] = dma_sm
    print(json.dumps(out))


def measured_fp64_gflops(n=4096, reps=3):
    """FP64 rate measured here: cuBLAS DGEMM (2 n^3 flops) through torch."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b_ = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b_)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for _ in range(reps):
        e0.record()
        torch.matmul(a, b_)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return 2.0 * n ** 3 / (best / 1e3) / 1e9


def run_rates(args):
    """FP64 and FP32 arithmetic rates of this GPU (cuBLAS DGEMM and SGEMM with
    TF32 off, 2 n^3 flops, best of a few) beside the FP64 stencil's own rate:
    the ALU rooflines of the IEEE-FP64 and FP32 stencils.  Not the benchmark
    line."""
    import torch
    torch.cuda.set_device(0)
    torch.backends.cuda.matmul.allow_tf32 = False
    out = {"mode": "rates"}
    for name, dt, n in (("dgemm_gflops", torch.float64, 4096), ("sgemm_gflops", torch.float32, 8192)):
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b_ = torch.randn(n, n, dtype=dt, device="cuda")
        torch.matmul(a, b_)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = None
        for _ in range(3):
            e0.record()
            torch.matmul(a, b_)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out[name] = 2.0 * n ** 3 / (best / 1e3) / 1e9
    out["sm_count"] = torch.cuda.get_device_properties(0).multi_processor_count
    print(json.dumps(out))


# ---------------------------------------------------------------------- all workloads
def run_suite(args):
    """Time-to-solution of every workload configuration, mixed precision
    against FP64, each after one warm-up solve (CUDA events, stream time)."""
    import ctypes as C
    import torch
    torch.cuda.set_device(0)
    from paper_2001_05218_gb300 import dw
    from paper_2001_05218_gb300 import inputs as I
    st = torch.cuda.current_stream()

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            out = fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    out = {"mode": "suite"}
    F64 = dict(tol=1e-10, inner="f64", maxiter=100000)
    MIX16 = dict(tol=1e-10, inner="f16", compress12=1, outer="df64", maxiter=100000)
    MIX32 = dict(tol=1e-10, inner="f32", outer="df64", maxiter=100000)
    MIXI16 = dict(tol=1e-10, inner="i16", compress12=1, outer="df64", maxiter=100000)
    MIXB16 = dict(tol=1e-10, inner="bf16", compress12=1, outer="df64", maxiter=100000)
    if args.delta is not None:
        MIX16["delta"] = args.delta
    if args.delta32 is not None:
        MIX32["delta"] = args.delta32

    def zero(*fields):
        for f in fields:
            f.storage.zero_()

    def single(name, configs):
        dims, kappa, U, b = I.make_workload(name)
        Ug, bg, xg = dw.gauge(dims, kappa, U), dw.spinor(dims, b), dw.spinor(dims)
        res = {}
        for label, kw in configs:
            p = dw.params(**kw)
            ms, (s, stt) = timed(lambda: (zero(xg), dw.cg_solve(Ug, bg, xg, p))[1])
            res[label] = {"ms": ms, "iters": stt[0]["iters"], "reliable_updates": stt[0]["reliable_updates"],
                          "true_rel_resid": stt[0]["true_rel_resid"]}
        return res

    out["wilson_4x4x4x4_haar"] = single("wilson_4x4x4x4_haar", [("f64_full_lattice", dict(F64, eo=0)),
                                                                 ("f64_eo", F64)])
    out["wilson_16x16x16x32_exp0.4"] = single("wilson_16x16x16x32_exp0.4", [
        ("f64", F64), ("df64", dict(tol=1e-10, inner="df64")), ("f32_mixed", MIX32), ("f16_mixed", MIX16),
        ("f32_defect_correction", dict(MIX32, defect_correction=1)),
        # 12- against 18-real links in the FP32 inner solve, and the full-lattice
        # (not even-odd) CGNR, whose operator uses every link twice per launch
        ("f32_mixed_12real_links", dict(MIX32, compress12=1)), ("i16_mixed", MIXI16),
        ("f64_full_lattice", dict(F64, eo=0)), ("f16_mixed_full_lattice", dict(MIX16, eo=0))])
    # the second stencil (covariant Laplacian) on the same links and sources
    def single_laplace(name, configs):
        dims, kappa, U, b = I.make_workload(name)
        Ug, bg, xg = dw.gauge(dims, kappa, U), dw.spinor(dims, b), dw.spinor(dims)
        res = {}
        for label, kw in configs:
            p = dw.params(**kw)
            ms, (s, stt) = timed(lambda: (zero(xg), dw.cg_solve_laplace(Ug, bg, xg, p))[1])
            res[label] = {"ms": ms, "iters": stt[0]["iters"], "reliable_updates": stt[0]["reliable_updates"],
                          "true_rel_resid": stt[0]["true_rel_resid"]}
        return res

    LAP = [("f64", F64), ("f32_mixed", MIX32), ("f16_mixed", MIX16)]
    out["laplace_16x16x16x32_exp0.4"] = single_laplace("wilson_16x16x16x32_exp0.4", LAP)
    out["laplace_32x32x32x64_exp0.6"] = single_laplace("wilson_32x32x32x64_exp0.6", LAP[1:])
    out["wilson_32x32x32x64_exp0.6"] = single("wilson_32x32x32x64_exp0.6", [
        ("f16_mixed_eo", MIX16), ("f16_mixed_full_lattice", dict(MIX16, eo=0)),
        ("f32_mixed_eo", MIX32), ("f32_mixed_12real_links", dict(MIX32, compress12=1)), ("i16_mixed_eo", MIXI16),
        ("bf16_mixed_eo", MIXB16)])
    # 12 point sources on 24^3x48: one multi-RHS solve vs 12 single solves
    name = "wilson_24x24x24x48_exp0.4_12src"
    dims, kappa, U, _ = I.make_workload(name, with_source=False)
    srcs = np.stack([I.point_source(dims, s_, c_) for s_ in range(4) for c_ in range(3)])
    Ug = dw.gauge(dims, kappa, U)
    bg, xg = dw.spinor(dims, srcs, nrhs=12), dw.spinor(dims, nrhs=12)
    r = {}
    for label, kw in (("f16_mixed_12rhs", MIX16), ("f64_12rhs", F64)):
        p = dw.params(**kw)
        ms, (s, stt) = timed(lambda: (zero(xg), dw.cg_solve(Ug, bg, xg, p))[1], reps=1)
        r[label] = {"ms": ms, "iters_max": max(x["iters"] for x in stt),
                    "true_rel_resid_max": max(x["true_rel_resid"] for x in stt)}
    b1, x1 = dw.spinor(dims, srcs[0]), dw.spinor(dims)
    p = dw.params(**MIX16)
    ms, (s, stt) = timed(lambda: (zero(x1), dw.cg_solve(Ug, b1, x1, p))[1], reps=1)
    r["f16_mixed_one_rhs_x12"] = {"ms": 12 * ms, "iters": stt[0]["iters"]}
    out[name] = r
    # ragged batch of 8 lattices: one batched solve vs the 8 solved one by one
    systems = I.ragged_batch()
    Us = [dw.gauge(d, k, U_) for d, k, U_, b_ in systems]
    bs = [dw.spinor(d, b_) for d, k, U_, b_ in systems]
    xs = [dw.spinor(d) for d, k, U_, b_ in systems]
    r = {}
    for label, kw in (("f16_mixed_batched", MIX16), ("f64_batched", F64)):
        p = dw.params(**kw)
        ms, (s, stt) = timed(lambda: (zero(*xs), dw.cg_solve_batched(Us, bs, xs, p))[1], reps=1)
        r[label] = {"ms": ms, "iters": [x["iters"] for x in stt]}
    p = dw.params(**MIX16)
    ms, _ = timed(lambda: [(zero(xs[i]), dw.cg_solve(Us[i], bs[i], xs[i], p)) for i in range(len(Us))], reps=1)
    r["f16_mixed_one_by_one"] = {"ms": ms}
    out["ragged_batch_8"] = r
    # differentiation: x = (D^dag D)^{-1} b forward, then grad_b and grad_U
    dims, kappa, U, b = I.make_workload("wilson_16x16x16x32_exp0.4_grad")
    g = I.gaussian_spinor(dims, I.workload_seed(4), I.STREAM_SOURCE2)
    Ug, bg, gx = dw.gauge(dims, kappa, U), dw.spinor(dims, b), dw.spinor(dims, g)
    xg, gb, gU = dw.spinor(dims), dw.spinor(dims), dw.Field(Ug.lat, dw.DW_GAUGE)
    r = {}
    for label, kw in (("f32_mixed", MIX32), ("f64", F64)):
        p = dw.params(**kw)
        sts = (dw.dw_solver_stats * 2)()

        def fwd_bwd():
            zero(xg)
            dw.cg_solve_normal(Ug, bg, xg, p)
            dw.check(dw.dw_cg_backward(Ug.handle, bg.handle, gx.handle, xg.handle, gb.handle, gU.handle, 1,
                                       C.byref(p), sts, dw.current_stream()))
        p.recompute_fwd = 0
        ms, _ = timed(fwd_bwd, reps=1)
        r[label] = {"ms": ms, "adjoint_iters": sts[1].iters, "adjoint_resid": sts[1].true_rel_resid}
    out["wilson_16x16x16x32_exp0.4_grad"] = r
    print(json.dumps(out))


# ---------------------------------------------------------------------- our arm
def run_multi(args):
    """The 12-source workload: 12 spin-colour point sources on 24^3x48 in one
    multi-RHS solve, against one of them solved alone (x12).  Each solve runs
    once as a graph after a warm-up (CUDA events, median of --steps), then once
    host-stepped with CUDA events around every stencil launch (the per-kernel
    split).  Not the benchmark line."""
    import torch
    torch.cuda.set_device(0)
    from paper_2001_05218_gb300 import dw
    from paper_2001_05218_gb300 import inputs as I
    name = "wilson_24x24x24x48_exp0.4_12src"
    dims, kappa, U, _ = I.make_workload(name, with_source=False)
    srcs = np.stack([I.point_source(dims, s_, c_) for s_ in range(4) for c_ in range(3)])
    Ug = dw.gauge(dims, kappa, U)
    p = dw.params(tol=1e-10, inner=args.inner or "f16", compress12=1 if args.compress12 is None else args.compress12,
                  outer=args.outer, maxiter=100000)
    st = torch.cuda.current_stream()
    out = {"mode": "multi", "workload": name, "inner": args.inner or "f16", "outer": args.outer}
    for nr in (12, 1):
        bg = dw.spinor(dims, srcs if nr == 12 else srcs[0], nrhs=nr)
        xg = dw.spinor(dims, nrhs=nr)
        ts = []
        for k in range(max(1, args.warmup) + max(1, args.steps)):
            xg.storage.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _, stt = dw.cg_solve(Ug, bg, xg, p)
            e1.record(st)
            torch.cuda.synchronize()
            if k >= max(1, args.warmup):
                ts.append(e0.elapsed_time(e1))
        xg.storage.zero_()
        torch.cuda.synchronize()
        dw.profile_start(time_stencils=True)
        dw.cg_solve(Ug, bg, xg, p)
        prof, launches = dw.profile_stop()
        out["rhs%d" % nr] = {"ms_median": float(np.median(ts)), "ms": [round(t, 3) for t in ts],
                             "iters": [x["iters"] for x in stt],
                             "reliable_updates": [x["reliable_updates"] for x in stt],
                             "true_rel_resid_max": max(x["true_rel_resid"] for x in stt),
                             "host_stepped": {"launches": launches,
                                              "kernels": {k: {"launches": v["launches"], "ms": round(v["total_ms"], 3)}
                                                          for k, v in prof.items()}}}
    out["speedup_vs_12_single"] = 12 * out["rhs1"]["ms_median"] / out["rhs12"]["ms_median"]
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--inner", default=None)
    ap.add_argument("--compress12", type=int, default=None)
    ap.add_argument("--outer", default="df64", help="precision of the reliable updates: df64 or f64")
    ap.add_argument("--delta", type=float, default=None,
                    help="reliable-update threshold (default: automatic); in --suite mode, of the 16-bit solves")
    ap.add_argument("--delta32", type=float, default=None, help="--suite mode: threshold of the FP32-inner solves")
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--dslash", default=None, help="stencil-only mode: f64|f32|f16|bf16|i16|df64 (Schur operator applies)")
    ap.add_argument("--nrhs", type=int, default=1, help="stencil-only mode: right-hand sides per field")
    ap.add_argument("--norm", action="store_true",
                    help="stencil-only mode: second launch with the reducing epilogue (dw_apply_norm)")
    ap.add_argument("--op", default="wilson", choices=["wilson", "laplace"],
                    help="stencil-only mode: the Wilson operator or the covariant Laplacian")
    ap.add_argument("--suite", action="store_true", help="time every workload configuration (not the benchmark line)")
    ap.add_argument("--copies", action="store_true", help="host<->device copy times of the e2e buffers (not the benchmark line)")
    ap.add_argument("--rates", action="store_true", help="FP64 and FP32 GEMM rates of this GPU (not the benchmark line)")
    ap.add_argument("--multi", action="store_true",
                    help="12 point sources on 24^3x48: one multi-RHS solve against single solves (not the benchmark line)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.dslash:
        return run_dslash(args)
    if args.suite:
        return run_suite(args)
    if args.copies:
        return run_copies(args)
    if args.rates:
        return run_rates(args)
    if args.multi:
        return run_multi(args)

    import torch
    rank, world, local = rank_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2001_05218_gb300 import dw
    from paper_2001_05218_gb300 import inputs as I

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    wl = args.workload
    big = I.WORKLOADS[wl]["dims"][3] >= 64
    inner = args.inner or ("f16" if big else "f32")
    c12 = args.compress12 if args.compress12 is not None else (1 if inner in ("f16", "bf16") else 0)
    dims, kappa, U, b = I.make_workload(wl)
    if rank > 0:  # independent system per rank: a different seeded source
        b = I.gaussian_spinor(dims, rank_source_seed(wl, rank), I.STREAM_SOURCE)
    V = int(np.prod(dims))
    Ug = dw.gauge(dims, kappa, U)
    bg = dw.spinor(dims, b)
    xg = dw.spinor(dims)
    p_mix = dw.params(tol=1e-10, inner=inner, compress12=c12, maxiter=40000, outer=args.outer)
    if args.delta is not None:
        p_mix.delta = args.delta
    p_64 = dw.params(tol=1e-10, inner="f64", maxiter=40000)
    zero = torch.zeros(xg.nbytes, dtype=torch.uint8, device="cuda")
    l2_bytes = torch.cuda.get_device_properties(0).L2_cache_size
    working_set = Ug.nbytes + bg.nbytes + xg.nbytes
    flush = working_set < 4 * l2_bytes
    scratch = torch.empty(2 * l2_bytes, dtype=torch.uint8, device="cuda") if flush else None

    def reset_x():
        xg.storage[xg.offset:xg.offset + xg.nbytes].copy_(zero)

    def solve(p):
        reset_x()
        if flush:
            scratch.fill_(1)
        return dw.cg_solve(Ug, bg, xg, p)

    for _ in range(max(3, args.warmup)):
        solve(p_mix)
    barrier()
    clk = ClockSampler(local)
    clk.start()
    clk.mark()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    dw.profile_start(time_stencils=False)  # counts kernel executions; the solver loop stays a CUDA graph
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    stats = []
    for k in range(args.steps):
        reset_x()
        if flush:
            scratch.fill_(1)
        ev[k][0].record(stream)
        s, st = dw.cg_solve(Ug, bg, xg, p_mix)
        ev[k][1].record(stream)
        stats.append(st[0])
    t1.record(stream)
    barrier()
    _, launches = dw.profile_stop()
    clocks = clk.stop()
    step_ms = [a.elapsed_time(b_) for a, b_ in ev]
    value, total_ms = aggregate_throughput(t0.elapsed_time(t1), args.steps, world, "cuda")
    solve_ms = float(np.mean(step_ms))
    st0 = stats[-1]

    # the configuration as written for this workload: the same mixed solve with
    # IEEE-FP64 (not double-float) reliable updates, median of three solves
    outer64 = None
    if args.outer != "f64" and not args.no_fp64:
        p_m64 = dw.params(tol=1e-10, inner=inner, compress12=c12, maxiter=40000, outer="f64")
        solve(p_m64)
        ts, st64m = [], None
        for _ in range(3):
            reset_x()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st64m = dw.cg_solve(Ug, bg, xg, p_m64)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        outer64 = {"ms": float(np.median(ts)), "iters": st64m[0]["iters"],
                   "reliable_updates": st64m[0]["reliable_updates"], "true_rel_resid": st64m[0]["true_rel_resid"],
                   "outer": "f64 (IEEE accumulator and reliable-update residual)", "statistic": "median of 3"}

    # per-launch stencil times: one more solve of the same system, stepped from
    # the host with CUDA events around every stencil launch on its stream
    reset_x()
    if flush:
        scratch.fill_(1)
    dw.profile_start(time_stencils=True)
    dw.cg_solve(Ug, bg, xg, p_mix)
    prof, _ = dw.profile_stop()
    peak_hbm, peak_kind = peaks()
    peak_fp64 = measured_fp64_gflops()  # GFLOP/s, cuBLAS DGEMM measured on this GPU

    def roof(name, e):
        pl_ms = e["total_ms"] / e["launches"]
        bpl = e["bytes"] / e["launches"]
        gbs = bpl / (pl_ms / 1e3) / 1e9
        gfl = e["flops"] / e["launches"] / (pl_ms / 1e3) / 1e9
        if name.startswith("hop f64"):
            return {"bound": "alu", "kernel": name, "achieved": gfl, "peak": peak_fp64, "unit": "GFLOP/s",
                    "frac": gfl / peak_fp64, "peak_kind": "measured FP64 rate (cuBLAS DGEMM)", "traffic": None,
                    "bytes_per_launch": bpl, "ms_per_launch": pl_ms, "launches": e["launches"], "achieved_gbs": gbs,
                    "frac_hbm": gbs / peak_hbm}
        return {"bound": "hbm", "kernel": name, "achieved": gbs, "peak": peak_hbm, "unit": "GB/s",
                "frac": gbs / peak_hbm, "peak_kind": peak_kind, "traffic": ncu_traffic(wl, name),
                "bytes_per_launch": bpl, "ms_per_launch": pl_ms, "launches": e["launches"], "gflops": gfl}

    stencils = {k: v for k, v in prof.items() if k.startswith("hop ") or k.startswith("laplace ")}
    dom_name, dom = max(stencils.items(), key=lambda kv: kv[1]["total_ms"])
    inner_name = [k for k in stencils if not k.startswith("hop f64") and not k.startswith("hop df64")]
    hop_total_ms = sum(v["total_ms"] for v in prof.values())

    # FP64 CG on the same system, same GPU
    fp64 = None
    if not args.no_fp64:
        solve(p_64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reset_x()
        e0.record(stream)
        s64, st64 = dw.cg_solve(Ug, bg, xg, p_64)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64 = {"ms": e0.elapsed_time(e1), "iters": st64[0]["iters"], "true_rel_resid": st64[0]["true_rel_resid"],
                "arith": "IEEE FP64 throughout"}
        # the same CG with every FP64 stencil in double-float arithmetic (FP64 storage size)
        p_df = dw.params(tol=1e-10, inner="df64", maxiter=40000)
        solve(p_df)
        torch.cuda.synchronize()
        reset_x()
        e0.record(stream)
        sdf, stdf = dw.cg_solve(Ug, bg, xg, p_df)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64["df64_cg"] = {"ms": e0.elapsed_time(e1), "iters": stdf[0]["iters"],
                           "true_rel_resid": stdf[0]["true_rel_resid"]}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        Uh = torch.from_numpy(U.reshape(-1).view(np.float64)).pin_memory()
        bh = torch.from_numpy(b.reshape(-1).view(np.float64)).pin_memory()
        xh = torch.empty(bh.numel(), dtype=torch.float64).pin_memory()
        sp = dw.current_stream()

        def e2e_step():
            dw.check(dw.dw_field_upload(Ug.handle, ctypes.c_void_p(Uh.data_ptr()), sp))
            dw.check(dw.dw_field_upload(bg.handle, ctypes.c_void_p(bh.data_ptr()), sp))
            reset_x()
            dw.cg_solve(Ug, bg, xg, p_mix)
            dw.check(dw.dw_field_download(xg.handle, ctypes.c_void_p(xh.data_ptr()), sp))
            torch.cuda.current_stream().synchronize()

        e2e_step()
        barrier()
        # each step timed on the host clock (it ends with a stream synchronise);
        # the median over the steps is reported, the mean and every step beside it
        ne = max(5, args.steps)
        wall = []
        # CUDA events around each step's two uploads (asynchronous: device time of
        # the copies and layout kernels), beside the step's host clock
        up_ev = []
        for _ in range(ne):
            d = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            a0 = time.perf_counter()
            d[0].record(stream)
            dw.check(dw.dw_field_upload(Ug.handle, ctypes.c_void_p(Uh.data_ptr()), sp))
            d[1].record(stream)
            dw.check(dw.dw_field_upload(bg.handle, ctypes.c_void_p(bh.data_ptr()), sp))
            d[2].record(stream)
            reset_x()
            dw.cg_solve(Ug, bg, xg, p_mix)
            dw.check(dw.dw_field_download(xg.handle, ctypes.c_void_p(xh.data_ptr()), sp))
            torch.cuda.current_stream().synchronize()
            wall.append(time.perf_counter() - a0)
            up_ev.append(d)
        torch.cuda.synchronize()
        barrier()
        # whole job: the slowest rank's median step, as for the device-timed value
        e2e_value, e2e_ms = aggregate_throughput(float(np.median(wall)) * 1e3, 1, world, "cuda")
        e2e_s = e2e_ms / 1e3
        # three more steps with events between the phases (stream time); the
        # median of each phase is reported
        names = ["upload_U", "upload_b", "solve", "download_x"]
        samples = {k: [] for k in names}
        for _ in range(3):
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            evs[0].record(stream)
            dw.check(dw.dw_field_upload(Ug.handle, ctypes.c_void_p(Uh.data_ptr()), sp))
            evs[1].record(stream)
            dw.check(dw.dw_field_upload(bg.handle, ctypes.c_void_p(bh.data_ptr()), sp))
            evs[2].record(stream)
            reset_x()
            dw.cg_solve(Ug, bg, xg, p_mix)
            evs[3].record(stream)
            dw.check(dw.dw_field_download(xg.handle, ctypes.c_void_p(xh.data_ptr()), sp))
            evs[4].record(stream)
            torch.cuda.synchronize()
            for i, k in enumerate(names):
                samples[k].append(evs[i].elapsed_time(evs[i + 1]))
        phases = {k: float(np.median(v)) for k, v in samples.items()}
        e2e = {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(Uh.numel() * 8 + bh.numel() * 8),
               "d2h_bytes_per_step": int(xh.numel() * 8), "ms_per_step": e2e_s * 1e3, "statistic": "median",
               "steps": ne, "mean_ms_per_step": float(np.mean(wall)) * 1e3,
               "step_ms": [round(w * 1e3, 3) for w in wall],
               "step_upload_ms": [[round(d[0].elapsed_time(d[1]), 3), round(d[1].elapsed_time(d[2]), 3)]
                                  for d in up_ev], "phases_ms": phases}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        iters = ORACLE_CGNR_ITERS.get(wl)
        how = "recorded"
        if iters is None:
            # same recurrence as the oracle (CGNR, full lattice) measured here
            xf = dw.spinor(dims)
            _, stf = dw.cg_solve(Ug, bg, xf, dw.params(tol=1e-10, inner="f32", eo=0, maxiter=100000))
            iters = stf[0]["iters"]
            how = "measured with the full-lattice CGNR of this library (FP32 inner, FP64 reliable updates)"
        cpu = cpu_baseline(wl, dims, kappa, U, b, iters)
        cpu["iters_source"] = how

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": solve_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("%s-storage/fp32-arith inner, %s reliable updates, f64 certification" % (inner, args.outer))
        if inner not in ("f64", "df64") else inner,
        "data": "synthetic (seeded exp(i a H) links, Gaussian source)",
        "config": {"workload": wl, "lattice": list(dims), "kappa": kappa, "solver": "even-odd CGNR",
                   "inner": inner, "compress12": c12, "outer": args.outer,
                   "delta": p_mix.delta if p_mix.delta > 0 else ("auto: 0.01" if inner in ("f16", "bf16") else "auto: 1e-4"),
                   "certification": "IEEE FP64",
                   "tol": 1e-10, "global_batch": world, "parallelism": "replicas",
                   "l2": "flushed between steps" if flush else "inputs larger than L2 (%d MB working set)" %
                         (working_set >> 20)},
        "mixed_cg": {"ms": solve_ms, "iters": st0["iters"], "reliable_updates": st0["reliable_updates"],
                     "true_rel_resid": st0["true_rel_resid"], "ms_median": float(np.median(step_ms)),
                     "ms_max": float(np.max(step_ms)), "step_ms": [round(v, 3) for v in step_ms]},
        "mixed_cg_outer_f64": outer64,
        "fp64_cg": fp64,
        "speedup_vs_fp64": (fp64["ms"] / solve_ms) if fp64 else None,
        "roofline": roof(dom_name, dom),
        "fp64_peak_gflops": peak_fp64,
        "roofline_inner": roof(inner_name[0], prof[inner_name[0]]) if inner_name else None,
        "stencil_profile": {"note": "one host-stepped solve with CUDA events around every stencil launch",
                            "kernels": {k: {"launches": v["launches"], "ms": v["total_ms"]} for k, v in prof.items()},
                            "stencil_ms": hop_total_ms},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
