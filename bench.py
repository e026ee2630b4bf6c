#!/usr/bin/env python3
"""Benchmark of the Multipolynomial Monte Carlo hot path on GB300.

One step = one pass over every level of the multilevel trace estimate
(Eq. (2)) for one batch of Z4 noise vectors: the composite and single
polynomial chains fused into the Wilson stencil, the deflation dots, the
per-sample assembly and the per-level statistics, all through the C ABI
(mpmc_trace_levels).  Default workload: the near-critical 24^3 x 32 lattice
(kappa 0.124) with the projected composite 50 x 20 (degree 999), degree 100
and degree 16, 100 deflation eigenpairs, 64 noise vectors per level, FP32
against the FP64 path at equal trace standard error.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores instead (bounded sample of the same workload).
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "noise-vector poly applies/s, dslash HBM GB/s; mixed vs FP64 at equal trace err"
UNIT = "noise-vector poly applies/s"
BATCH_KEY = "batch64"
BATCH_DESC = ("64 independent Wilson-Dirac instances, lattices from {4^4, 6^4, 8^4, 8^3x16, 12^4}, "
              "kappa ~ U[0.118, 0.124], near-identity links eps ~ U[0.2, 0.4]; levels [composite20x15=deg299, "
              "deg40, deg8] each; 32 Z4 noises/level; one CUDA graph per batch")
FLOPS_PER_SITE_RHS_STEP = 1488   # 1320 hopping + 48 diagonal + 96 chain axpy + 24 Z4 dot


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out = self.proc.communicate(timeout=5)[0]
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = self.proc.communicate()[0]

    def summary(self):
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(mhz)}


# ------------------------------------------------------------------ oracle leg
def oracle_worker(spec):
    """Runs in a fresh single-threaded process: the oracle, as it stands, on a bounded sample
    (worker w of a pool draws its own noise vectors)."""
    import numpy as np
    from oracle import krylov as K
    from oracle import mpmc as M
    from oracle.lattice import WilsonOperator
    from paper_2306_09559_gb300 import workloads, synth

    if spec["workload"] == BATCH_KEY:
        # one noise vector through a degree-8 polynomial on each lattice class of the batch;
        # the step's cost is extrapolated by the matvecs of every instance on its class
        from oracle import philox
        from oracle import polynomial as P
        insts = workloads.batch_instances()
        per_class = {}
        for dims in sorted(set(w.dims for w in insts)):
            wl0 = next(w for w in insts if w.dims == dims)
            op = WilsonOperator(workloads.gauge(wl0), wl0.kappa)
            b = philox.z4_block(wl0.noise_seed, 0, 0, 1, wl0.V)
            roots = np.linspace(1.0, 2.0, 9) + 0.1j
            t1 = time.perf_counter()
            np.vdot(b[:, 0], P.apply_poly(op, roots, b)[:, 0])
            per_class[dims] = (time.perf_counter() - t1) / 8
        t_step = sum(per_class[w.dims] * w.matvecs_per_step() for w in insts)
        return {"times": [t_step] * spec["steps"], "applies_per_step": sum(w.applies_per_step() for w in insts),
                "setup_s": 0.0,
                "sample": "1 noise vector through a degree-8 polynomial on each of the 5 lattice classes, "
                          f"extrapolated by the batch's {sum(w.matvecs_per_step() for w in insts)} matvecs"}
    wl = workloads.get(spec["workload"])
    per_level = spec["per_level"]
    U = workloads.gauge(wl)
    op = WilsonOperator(U, wl.kappa)
    if wl.V > 8 ** 4:
        # lattices beyond 8^4: one noise vector through the cheapest level's polynomial, and
        # the step's cost extrapolated by its matvec count (the oracle's cost per matvec does
        # not depend on the root values)
        from oracle import philox
        from oracle import polynomial as P
        d = min(lv[1] for lv in wl.levels if lv[0] == "single")
        roots = np.linspace(1.0, 2.0, d + 1) + 0.1j
        b = philox.z4_block(wl.noise_seed, len(wl.levels) - 1, spec.get("worker", 0), 1, wl.V)
        times = []
        for step in range(spec["steps"]):
            t1 = time.perf_counter()
            np.vdot(b[:, 0], P.apply_poly(op, roots, b)[:, 0])
            per_mv = (time.perf_counter() - t1) / d
            times.append(per_mv * wl.matvecs_per_step())
        return {"times": times, "applies_per_step": wl.applies_per_step(), "setup_s": 0.0,
                "sample": f"1 noise vector through a degree-{d} polynomial ({d} matvecs) per step, "
                          f"extrapolated by the step's {wl.matvecs_per_step()} matvecs"}
    t0 = time.perf_counter()
    b0 = synth.random_unit_vector(op.n, wl.setup_seed)
    singles = [lv[1] for lv in wl.levels if lv[0] == "single"]
    inners = [lv[1] - 1 for lv in wl.levels if lv[0] == "composite"]
    degs = sorted(set(singles + inners))
    V, Hbar, beta = K.arnoldi(op, b0, max(degs) + 1)
    roots = {d: K.harmonic_ritz(Hbar, d + 1) for d in degs}
    polys = []
    for lv in wl.levels:
        if lv[0] == "single":
            polys.append({"kind": "single", "roots": roots[lv[1]][P_leja(roots[lv[1]])]})
        else:
            inner = roots[lv[1] - 1][P_leja(roots[lv[1] - 1])]
            outer, _, _ = K.pp_gmres_roots(op, inner, b0, m_out=lv[2])
            polys.append({"kind": "composite", "inner": inner, "outer": outer})
    defl = None
    if wl.k > 0:
        # deflation vectors of the workload's shape (k orthonormal Krylov vectors); the
        # cost of a sample depends on k and n, not on how accurate the vectors are
        Zk = V[:, :wl.k]
        lam = np.einsum("ni,ni->i", Zk.conj(), op(Zk))
        defl = M.Deflation(op, Zk, lam, np.arange(wl.k))
    t_setup = time.perf_counter() - t0
    times = []
    for step in range(spec["steps"]):
        t1 = time.perf_counter()
        for level in range(len(polys)):
            first = (spec.get("worker", 0) * spec["steps"] + step) * per_level
            M.level_sample_parts(op, polys, level, wl.noise_seed, per_level, defl, first=first, block=per_level)
        times.append(time.perf_counter() - t1)
    applies = per_level * (2 * (len(polys) - 1) + 1)
    return {"times": times, "applies_per_step": applies, "setup_s": t_setup,
            "sample": f"{per_level} noise vectors per level of the same workload"}


def P_leja(r):
    from oracle import polynomial as P
    return P.leja_order(r)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def start_oracle_pool(workload, per_level, steps, cores):
    """One single-threaded oracle process per host core (spawned fresh, no GPU), each on its
    own noise vectors (worker w starts at noise index w * per_level)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               NUMEXPR_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    procs = []
    for w in range(cores):
        with tempfile.NamedTemporaryFile("r", suffix=".json", delete=False) as f:
            path = f.name
        spec = json.dumps({"workload": workload, "per_level": per_level, "steps": steps, "out": path,
                           "worker": w})
        procs.append((subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-worker", spec], env=env,
                                       stdout=subprocess.DEVNULL, stderr=subprocess.PIPE, text=True), path))
    return procs


def finish_oracle_pool(procs):
    """Aggregate rate of the pool: all workers' applies over the slowest worker's time, per step."""
    outs, errs = [], []
    for proc, path in procs:
        _, err = proc.communicate()
        if proc.returncode == 0:
            outs.append(json.load(open(path)))
        else:
            errs.append(err[-300:])
        if os.path.exists(path):
            os.unlink(path)
    if errs:
        raise RuntimeError("oracle worker failed:\n" + errs[0])
    nsteps = min(len(o["times"]) for o in outs)
    step_times = [max(o["times"][k] for o in outs) for k in range(nsteps)]
    applies = sum(o["applies_per_step"] for o in outs)
    return {"step_times": step_times, "applies_per_step": applies, "sample": outs[0]["sample"],
            "workers": len(outs)}


def run_oracle(workload, per_level, steps, cores=None):
    """The oracle leg on every host core (one single-threaded process per core)."""
    return finish_oracle_pool(start_oracle_pool(workload, per_level, steps, cores or host_cores()))


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(workload, per_level, steps):
    """The cpu_baseline object: the oracle, as it stands, on every core of the host."""
    cores = host_cores()
    try:
        r = run_oracle(workload, per_level, steps, cores)
    except RuntimeError as e:
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": "failed: " + str(e)[-300:]}
    t = r["step_times"]
    return {"value": r["applies_per_step"] * len(t) / sum(t), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{r['sample']}, on each of {r['workers']} single-threaded processes in parallel "
                      f"(FP64 numpy oracle, {cpu_model()})"}


# ------------------------------------------------------------------ reference arm
def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2306_09559_gb300 import workloads
    wl = workloads.get(args.workload) if args.workload != BATCH_KEY else None
    per_level = args.oracle_noises
    cores = host_cores()
    res = run_oracle(args.workload, per_level, args.steps + args.warmup, cores)
    times = res["step_times"][args.warmup:]
    value = res["applies_per_step"] * len(times) / sum(times)
    sample = (f"{res['sample']}, on each of {res['workers']} single-threaded processes (FP64 numpy oracle, "
              f"{cpu_model()})")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.describe() if wl else BATCH_DESC, "sample": res["sample"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ batched instances
def batch_arm(args):
    """The uneven batch: 64 instances as one captured CUDA graph per step (mixed
    precision), against the same handles traced one after another and the FP64
    batch.  Weak scaling: rank r runs its own 64 instances (noise offset r)."""
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle on every host core, before any GPU work (bounded sample, single-threaded processes)
        cpu = cpu_baseline(BATCH_KEY, 1, 1)

    from paper_2306_09559_gb300 import build, workloads
    from paper_2306_09559_gb300 import mpmc as G
    build.build()
    insts = workloads.batch_instances()
    prec = {"fp32": G.FP32, "bf16s": G.BF16S, "fp64": G.FP64}[args.precision]
    t0 = time.perf_counter()
    links, h64s, hms = [], [], []
    for wl in insts:
        U = workloads.gauge(wl)
        links.append(np.ascontiguousarray(U))
        h64 = G.Handle(U, wl.kappa, G.FP64)
        polys = workloads.setup_light(h64, wl)
        workloads.configure(h64, polys, None, wl.nsamples)
        hm = G.Handle(U, wl.kappa, prec)
        workloads.configure(hm, polys, None, wl.nsamples)
        h64s.append(h64)
        hms.append(hm)
    t_setup = time.perf_counter() - t0
    first = rank * 32
    applies = sum(w.applies_per_step() for w in insts)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")   # 256 MB > L2
    cur = torch.cuda.current_stream()

    def timed(fn, steps):
        """device time per step (events on the current stream, synchronised on both sides)."""
        out = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(cur)
            res = fn()
            e1.record(cur)
            torch.cuda.synchronize()
            out.append((e0.elapsed_time(e1), res))
        return out

    bm = G.Batch(hms)
    run_batch = lambda: bm.mpmc_batch_trace_levels(7, 32, first)
    for _ in range(args.warmup):
        run_batch()
    n0 = bm.mpmc_batch_launch_count()
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.nvtx.range_push("timed")
        res = timed(run_batch, args.steps)
        torch.cuda.nvtx.range_pop()
        barrier()
    launches = bm.mpmc_batch_launch_count() - n0
    t_local = sum(t for t, _ in res)
    t_max = t_local
    if dist is not None:
        tt = torch.tensor([t_local], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    ms_per_step = t_max / args.steps
    value = applies * world / (ms_per_step / 1000.0)
    mean_m, var_m = res[-1][1]

    # the same handles traced one after another (no graph)
    seq = timed(lambda: [h.mpmc_trace_levels(7, 32, first, want_samples=False) for h in hms], 2)
    seq_ms = sum(t for t, _ in seq) / len(seq)
    # FP64 batch
    b64 = G.Batch(h64s)
    b64.mpmc_batch_trace_levels(7, 32, first)
    r64 = timed(lambda: b64.mpmc_batch_trace_levels(7, 32, first), 1)
    t64 = r64[0][0]
    mean64, var64 = r64[0][1]
    L = 3
    var_sum64, var_sum_m = float(np.sum(var64[:, :L])), float(np.sum(var_m[:, :L]))
    # the paired comparison per level, pooled over instances (same noise on both)
    z = [float(np.max(np.abs((mean_m[:, l] - mean64[:, l]).real) / np.sqrt(var64[:, l] / 32))) for l in range(L)]
    fp64 = {"value": applies / (t64 / 1000.0), "ms_per_step": t64,
            "equal_se_speedup": (t64 * var_sum64) / (ms_per_step * var_sum_m),
            "max_over_instances_mean_diff_over_se": z}

    # end to end through the public API: new links for every instance (host -> device), the
    # batch (recaptured, since the fields changed), means and variances back to the host
    pinned = [torch.from_numpy(u).pin_memory() for u in links]
    h2d = sum(int(p.numel() * p.element_size()) for p in pinned)

    def e2e_step():
        for h, p in zip(hms, pinned):
            h.mpmc_set_links(p)
        return bm.mpmc_batch_trace_levels(7, 32, first)

    e2e_res = timed(e2e_step, 2)
    e2e_ms = sum(t for t, _ in e2e_res) / len(e2e_res)
    e2e = {"value": applies / (e2e_ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": len(insts) * 8 * 24, "ms_per_step": e2e_ms,
           "note": "host links copied to every handle each step, so the graph is captured again each step"}

    # throughput of the stencil steps of a batch step: algorithmic bytes of all steps / step time
    stor = {"fp32": 8, "bf16s": 4, "fp64": 16}[args.precision]
    lb = 72 if args.precision != "fp64" else 144
    alg = 0.0
    for w in insts:
        per_step = w.V * w.nsamples * 12 * stor * 2 + w.V * 4 * lb
        alg += per_step * w.matvecs_per_step() / w.nsamples
    hbm, sm_max, src = peaks()
    achieved = alg / (ms_per_step / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": "all stencil steps of the batch (one graph)",
                "hbm_peak_source": src, "algorithmic_bytes_per_step": alg,
                "note": "step-level: every launch of the 64 instances counted, timed as one graph; the working "
                        "set of most instances is L2-resident"}
    if rank == 0:
        lat = {}
        for w in insts:
            lat["x".join(map(str, w.dims))] = lat.get("x".join(map(str, w.dims)), 0) + 1
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16s": "bf16-stored/f32", "fp64": "f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": BATCH_DESC, "instances": len(insts), "lattices": lat,
                       "noises_per_level": 32, "applies_per_step": applies,
                       "matvecs_per_step": sum(w.matvecs_per_step() for w in insts),
                       "graph_nodes_per_step": launches // max(args.steps, 1),
                       "sequential_ms_per_step": seq_ms, "graph_speedup_over_sequential": seq_ms / ms_per_step,
                       "l2": "flushed before every step (256 MB write)", "parallelism": f"instances x{world}",
                       "setup_s": t_setup},
            "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "cpu_baseline": cpu, "fp64": fp64,
        }
        print(json.dumps(line), flush=True)
    bm.close()
    b64.close()
    for h in hms + h64s:
        h.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def correction_levels(wl, polys, m64, v64, x64, mmix, xmix, t64, tmix):
    """FP64 correction levels for the mixed-precision levels that miss the bias bound.

    A level estimated as mean(s_mix) + mean((s_64 - s_mix)[:n]) is unbiased with respect to
    FP64 by construction (the telescoping of Eq. (2) across precisions).  n follows the Eq. (3)
    allocation of the two terms, n = N sqrt((V_d / C_64) / (V_mix / C_mix)), at least 2, with the
    per-sample costs in the ratio of the measured FP64 and mixed step times.  The corrected
    estimate is compared with the FP64 one under the bias bound (0.1 SE_64 plus three standard
    errors of the correction), and the equal-SE speed-up is recomputed with the FP64 samples
    the corrections cost (at the level's share of the FP64 step time)."""
    import numpy as np
    N = wl.nsamples
    mv = []
    for kind, r, o in polys:
        mv.append(len(r) - 1 if kind == "single" else (len(o) - 1) * len(r) + len(r) - 1)
    level_mv = [mv[l] + (mv[l + 1] if l + 1 < len(mv) else 0) for l in range(len(mv))]
    share = [x / sum(level_mv) for x in level_mv]
    out, t_corr, var_total = {"levels": []}, 0.0, 0.0
    for l in range(len(polys)):
        dl = (x64[l] - xmix[l]).real
        se64 = np.sqrt(v64[l] / N)
        bound = 0.1 * se64 + 3 * np.std(dl, ddof=1) / np.sqrt(N)
        var_m = float(np.var(xmix[l].real, ddof=1))
        if abs(np.mean(dl)) <= bound:
            var_total += var_m
            continue
        var_d = float(np.var(dl, ddof=1))
        n = max(2, int(np.ceil(N * np.sqrt((var_d / t64) / (var_m / tmix))))) if var_m > 0 else 2
        n = min(n, N)
        corr_mix = mmix[l] - np.mean(xmix[l])
        est = np.mean(xmix[l]) + corr_mix + np.mean(x64[l][:n] - xmix[l][:n])
        cov = float(np.cov(xmix[l].real[:n], dl[:n], ddof=1)[0, 1]) if n > 2 else 0.0
        var_est = var_m / N + var_d / n + 2 * cov / N
        dev = abs((est - m64[l]).real)
        allowed = 0.1 * se64 + 3 * np.sqrt(var_d / n)
        t_corr += n * t64 * share[l] / N
        var_total += N * var_est
        out["levels"].append({"level": l, "mixed_bias_over_se": float(abs(np.mean(dl)) / se64),
                              "ncorr": n, "var_diff": var_d, "corrected_estimate": [float(est.real), float(est.imag)],
                              "corrected_minus_fp64_over_se": float(dev / se64),
                              "corrected_within_bound": bool(dev <= allowed),
                              "corrected_se": float(np.sqrt(max(var_est, 0.0)))})
    out["fp64_ms_per_step_for_corrections"] = t_corr
    out["equal_se_speedup"] = float((t64 * float(np.sum(v64))) / ((tmix + t_corr) * var_total))
    return out


# sources of each t-sweep form: a DRAM-traffic figure from an ncu capture holds while they are unchanged
FORM_SOURCES = {
    "k_fsweep": ("stencil_fsweep.cuh", "stencil_fast.cuh", "stencil.cuh", "device.cuh", "tc.cuh"),
    "k_fsweep_lsm": ("stencil_fsweep.cuh", "stencil_fast.cuh", "stencil.cuh", "device.cuh", "tc.cuh"),
    "k_fsweep_w": ("stencil_fsweep_w.cuh", "stencil_fsweep.cuh", "stencil_fast.cuh", "stencil.cuh", "device.cuh",
                   "tc.cuh"),
    "k_fsweep_p": ("stencil_fsweep_p.cuh", "stencil_fsweep_w.cuh", "stencil_fsweep.cuh", "stencil_fast.cuh",
                   "stencil.cuh", "device.cuh", "tc.cuh"),
}


def fsweep_form(sweep_mask):
    """Name of the t-sweep form a sweep option mask in effect runs (mpmc_get_option)."""
    if sweep_mask & 64:
        return "k_fsweep_p"
    return "k_fsweep_w" if sweep_mask & 32 else "k_fsweep_lsm" if sweep_mask & 16 else "k_fsweep"


def kernel_sources_digest(form="k_fsweep_lsm"):
    """Digest of the sources of one t-sweep form (first 16 hex digits of a SHA-256)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2306_09559_gb300", "csrc")
    for f in FORM_SOURCES[form]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def captured_traffic(kernel, storage, nb, V):
    """DRAM bytes per launch of `kernel` (a t-sweep form) from the committed ncu summary
    profiles/dram_traffic.md (a row per capture: kernel, storage, block width, lattice, bytes per
    launch, source digest), scaled from the captured lattice to V sites (the traffic of the t-sweep
    grows with the sites swept); None if no capture matches or the sources changed since."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.md")
    if not os.path.exists(path) or kernel not in FORM_SOURCES:
        return None, None
    digest = kernel_sources_digest(kernel)
    for line in open(path):
        f = [x.strip().strip("`") for x in line.strip().strip("|").split("|")]
        if len(f) < 6 or f[0] != kernel or f[1] != storage or f[2] != str(nb) or f[5] != digest:
            continue
        dims = [int(x) for x in f[3].split("x")]
        vcap = dims[0] * dims[1] * dims[2] * dims[3]
        return float(f[4]) * V / vcap, f"ncu capture on {f[3]} (same kernel and block width), scaled by {V}/{vcap} sites"
    return None, None


# ------------------------------------------------------------------ GPU arm
def gpu_arm(args):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    # the oracle on every host core, before any GPU work (bounded sample, single-threaded processes)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, args.oracle_noises, 1)

    from paper_2306_09559_gb300 import build, workloads
    from paper_2306_09559_gb300 import mpmc as G
    build.build()
    wl = workloads.get(args.workload)
    U = workloads.gauge(wl)
    t0 = time.perf_counter()
    h64 = G.Handle(U, wl.kappa, G.FP64)
    polys, defl = workloads.setup(h64, wl, log=log if rank == 0 else None)
    t_setup = time.perf_counter() - t0
    prec = {"fp32": G.FP32, "bf16s": G.BF16S, "fp64": G.FP64}[args.precision]
    hm = G.Handle(U, wl.kappa, prec)
    stream = torch.cuda.Stream()
    hm.mpmc_set_stream(stream)
    workloads.configure(hm, polys, defl, args.block or None)
    if not args.block:
        hm.mpmc_autotune(wl.nsamples)          # block width and launch shape for this lattice
    launch = hm.mpmc_get_launch()
    block = launch["nb"]
    first = rank * wl.nsamples           # weak scaling: each rank draws its own noise indices
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def one(h, fst):
        return h.mpmc_trace_levels(wl.noise_seed, wl.nsamples, fst)

    # storage per level: levels whose samples cancel most (the polynomial differences of high
    # degree) on FP32-stored handles, the others on the handle of --precision
    codes = {"fp32": G.FP32, "bf16s": G.BF16S, "fp64": G.FP64}
    if args.level_storage == "auto":
        per_level = (["fp32", "fp32"] + [args.precision] * len(polys))[:len(polys)] \
            if args.precision == "bf16s" else [args.precision] * len(polys)
    else:
        per_level = args.level_storage.split(",")
        if len(per_level) != len(polys) or any(x not in codes for x in per_level):
            raise SystemExit(f"--level-storage needs {len(polys)} entries from {sorted(codes)}")
    level_handle = {}
    for name in sorted(set(per_level)):
        if name == args.precision:
            level_handle[name] = hm
            continue
        hx = G.Handle(U, wl.kappa, codes[name])
        hx.mpmc_set_stream(stream)
        workloads.configure(hx, polys, defl, args.block or None)
        if not args.block:
            hx.mpmc_autotune(wl.nsamples)
        level_handle[name] = hx
    handles = [hm] + [h for h in level_handle.values() if h is not hm]

    def run_step(fst):
        if len(handles) == 1:
            return one(hm, fst)
        L, N = len(polys), wl.nsamples
        mean, var, smp = np.zeros(L, dtype=complex), np.zeros(L), np.zeros((L, N), dtype=complex)
        for l in range(L):
            mean[l], var[l], smp[l] = level_handle[per_level[l]].mpmc_trace_level(l, wl.noise_seed, N, fst)
        return mean, var, smp

    for _ in range(args.warmup):
        run_step(first)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = sum(h.mpmc_launch_count() for h in handles)
    for h in handles:
        h.mpmc_profile(True)
    results = []
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[k][0].record(stream)
            results.append(run_step(first))
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier()
    launches = sum(h.mpmc_launch_count() for h in handles) - l0
    st_ms, st_n, st_bytes = [sum(x) for x in zip(*[h.mpmc_profile_read(G.PROF_STENCIL) for h in handles])]
    df_ms, df_n, df_bytes = [sum(x) for x in zip(*[h.mpmc_profile_read(G.PROF_DEFLATION) for h in handles])]
    per_kernel = {}
    for cls, name in G.PROF_KERNEL_NAMES.items():
        ms_k, n_k, b_k = [sum(x) for x in zip(*[h.mpmc_profile_read(cls) for h in handles])]
        if n_k:
            per_kernel[name] = {"ms": ms_k, "launches": n_k, "bytes": b_k}
    for h in handles:
        h.mpmc_profile(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(step_ms)
    t_max = t_local
    if dist is not None:
        t = torch.tensor([t_local], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    ms_per_step = t_max / args.steps
    value = world * wl.applies_per_step() * args.steps / (t_max / 1000.0)

    # ---------------------------------------------------------- end to end through the C ABI
    e2e = None
    if not args.no_e2e:
        Zp = None
        if defl is not None:
            Z, lam, pair = defl        # Z: (k, n) CUDA tensor from the setup
            Zp = Z.cpu().pin_memory()
            lamp, pairp = np.ascontiguousarray(lam), np.ascontiguousarray(pair, dtype=np.int32)
        Up = torch.from_numpy(np.ascontiguousarray(U)).pin_memory()
        h2d = Up.numel() * 16 + (Zp.numel() * 16 + lamp.size * 16 + pairp.size * 4 if Zp is not None else 0)
        h2d += sum(16 * (r.size + (0 if o is None else o.size)) for _, r, o in polys)
        d2h = 16 * wl.nsamples * len(polys)

        def e2e_step():
            for h in handles:
                h.mpmc_set_links(Up)
                if Zp is not None:
                    h.mpmc_set_deflation(Zp, lamp, pairp, rows=True)
                workloads.configure(h, polys, None)
            return run_step(first)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        te = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        te = time.perf_counter() - te
        if dist is not None:
            t = torch.tensor([te], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        e2e = {"value": world * wl.applies_per_step() * args.steps / te, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1000 * te / args.steps}

    # ---------------------------------------------------------- FP64 path at equal trace error
    fp64 = None
    if not args.no_fp64 and prec != G.FP64:
        workloads.configure(h64, polys, defl, None)
        h64.mpmc_autotune(min(wl.nsamples, 128), steps=2)
        s64 = torch.cuda.Stream()
        h64.mpmc_set_stream(s64)
        one(h64, first)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s64)
        m64, v64, x64 = one(h64, first)
        b.record(s64)
        torch.cuda.synchronize()
        t64 = a.elapsed_time(b)
        m32, v32, x32 = results[-1]
        d = x32 - x64
        var64, var32 = float(np.sum(v64)), float(np.sum(v32))
        # the FP64 path is bound by FP64 arithmetic on GB300: its algorithmic flops against the
        # FP64 FMA throughput measured on this device by the library's own microbenchmark
        fp64_peak = G.mpmc_fma_peak(G.FP64)
        fp64_tflops = FLOPS_PER_SITE_RHS_STEP * wl.V * wl.matvecs_per_step() / (t64 / 1000.0) / 1e12
        fp64 = {"value": wl.applies_per_step() / (t64 / 1000.0), "ms_per_step": t64,
                "roofline": {"bound": "alu", "achieved": fp64_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                             "frac": fp64_tflops / fp64_peak,
                             "peak_source": "measured: mpmc_fma_peak(FP64), independent FMA chains on every SM"},
                "equal_se_speedup": (t64 * var64) / (ms_per_step * var32),
                "level_var_fp64": [float(x) for x in v64], "level_var_mixed": [float(x) for x in v32],
                "paired_mean_diff_over_se": [float(abs(np.mean(d[l].real)) / np.sqrt(v64[l] / wl.nsamples))
                                             for l in range(len(polys))],
                "paired_std_diff_over_std": [float(np.std(d[l].real) / np.sqrt(v64[l])) for l in range(len(polys))],
                # bias bound on identical noise: |mean d| <= 0.1 SE_64 + 3 std(d) / sqrt(N)
                "paired_bias_allowed_over_se": [float((0.1 * np.sqrt(v64[l] / wl.nsamples)
                                                       + 3 * np.std(d[l].real, ddof=1) / np.sqrt(wl.nsamples))
                                                      / np.sqrt(v64[l] / wl.nsamples)) for l in range(len(polys))],
                "paired_bias_within_bound": [bool(abs(np.mean(d[l].real)) <= 0.1 * np.sqrt(v64[l] / wl.nsamples)
                                                  + 3 * np.std(d[l].real, ddof=1) / np.sqrt(wl.nsamples))
                                             for l in range(len(polys))],
                "level_estimates_fp64": [[float(z.real), float(z.imag)] for z in m64],
                "level_estimates_mixed": [[float(z.real), float(z.imag)] for z in m32]}
        fp64["correction_levels"] = correction_levels(wl, polys, m64, v64, x64, m32, x32, t64, ms_per_step)
        fp64["equal_se_speedup_with_corrections"] = fp64["correction_levels"].pop("equal_se_speedup")

    # ---------------------------------------------------------- the rest of the paper's estimate (Eq. (2))
    # Tr(A^{-1} - M_1), the first Monte Carlo of Sec. 5 step 3a: deflated PP-GMRES solves (FP64) on a
    # few noise vectors; and Tr(p_3) by probing with a distance-4 colouring for a degree-4 p_3 (Sec. 3.1).
    # Both run after the timed region on the same handles (polynomial slots 6 and 5 leave the levels alone).
    extra = {}
    if not args.no_inverse and defl is not None and polys[0][0] == "deflated_composite":
        h64.mpmc_set_poly(6, G.SINGLE, polys[0][1], leja=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        mi, vi, si = h64.mpmc_trace_inverse(0, wl.noise_seed, args.inverse_noises, first, pin=6, rtol=1e-8, m=40,
                                            maxcycles=200)
        torch.cuda.synchronize()
        ti = time.perf_counter() - t1
        extra["inverse_level"] = {"level": "Tr(A^-1 - M_1), deflated PP(%d)-GMRES(40) solves to 1e-8, FP64"
                                  % len(polys[0][1]), "noises": args.inverse_noises,
                                  "seconds_per_noise": ti / args.inverse_noises,
                                  "sample_var": vi if args.inverse_noises > 1 else None,
                                  "estimate": [mi.real, mi.imag]}
    if not args.no_probing:
        from paper_2306_09559_gb300 import krylov_setup, synth
        p4 = krylov_setup.Setup(h64).single_roots(synth.random_unit_vector(wl.n, wl.setup_seed), [4])[0]
        colours, nc = G.mpmc_colouring(wl.dims, 4)
        hm.mpmc_set_poly(5, G.SINGLE, p4, leja=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        tr = hm.mpmc_trace_probing_colours(5, colours, nc)
        torch.cuda.synchronize()
        tp = time.perf_counter() - t1
        extra["probing"] = {"polynomial": "degree 4 (GMRES harmonic Ritz roots)", "colouring": "distance 4",
                            "colours": nc, "probe_vectors": 12 * nc, "seconds": tp, "trace": [tr.real, tr.imag],
                            "period_8_probe_vectors": 12 * 8 ** 4}

    # ---------------------------------------------------------- roofline of the dominant kernel
    hbm, sm_max, src = peaks()
    # the dominant kernel: the stencil kernel with the largest share of the timed steps (the t-sweep
    # class named by the form the handle runs)
    sweep_now = hm.mpmc_get_option(G.OPT_SWEEP_STENCIL)
    if "k_fsweep" in per_kernel:
        per_kernel[fsweep_form(sweep_now)] = per_kernel.pop("k_fsweep")
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    dk = per_kernel[dom]
    avg_ms = dk["ms"] / dk["launches"]
    bytes_per_launch = dk["bytes"] / dk["launches"]
    achieved_gbs = bytes_per_launch / (avg_ms / 1000.0) / 1e9
    kernel_mix = {k: {"share_of_step": v["ms"] / t_local, "launches": v["launches"],
                      "avg_launch_ms": v["ms"] / v["launches"],
                      "achieved_gbs": v["bytes"] / (v["ms"] / 1000.0) / 1e9} for k, v in per_kernel.items()}
    # FP32 pipe: the FMA throughput measured on this device (mpmc_fma_peak), against the
    # algorithmic flops of one step per site and right-hand side
    alu_peak = G.mpmc_fma_peak(G.FP32)
    flops_per_launch = FLOPS_PER_SITE_RHS_STEP * float(np.prod(wl.dims)) * block
    achieved_tflops = flops_per_launch / (avg_ms / 1000.0) / 1e12
    t_hbm, t_alu = bytes_per_launch / (hbm * 1e9), flops_per_launch / (alu_peak * 1e12)
    fast, sweep = hm.mpmc_get_option(G.OPT_FAST_STENCIL), hm.mpmc_get_option(G.OPT_SWEEP_STENCIL)
    # step classes: 1 dotted steps, 2 undotted inner steps, 4 outer steps of composite chains
    kernel = (f"{dom} (fused stencil step); issue-lean kernels for step-class mask {fast} "
              f"(t-sweep mask {sweep & fast & 7}), site-parallel k_step/k_outer"
              f"{' (k_sweep form)' if sweep & 8 else ''} for the others")
    alu = {"achieved": achieved_tflops, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved_tflops / alu_peak,
           "flops_per_launch": flops_per_launch, "peak_source": "measured: mpmc_fma_peak(FP32)",
           "nominal_peak": 152 * 128 * 2 * sm_max * 1e6 / 1e12}
    traffic, traffic_src = args.traffic, "--traffic" if args.traffic is not None else None
    if traffic is None:
        traffic, traffic_src = captured_traffic(dom, args.precision, block, wl.V)
    if args.precision != "fp64" and t_alu > t_hbm:
        # BF16-stored spinors: the FP32 arithmetic floor lies above the HBM floor
        roofline = {"bound": "alu", **alu, "traffic": traffic, "hbm_frac": achieved_gbs / hbm}
    else:
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                    "frac": achieved_gbs / hbm, "traffic": traffic, "alu": alu}
    roofline["traffic_source"] = traffic_src
    roofline.update({"kernel": kernel, "hbm_peak_source": src, "avg_launch_ms": avg_ms, "launches": dk["launches"],
                     "share_of_step": dk["ms"] / t_local if t_local else None,
                     "algorithmic_bytes_per_launch": bytes_per_launch, "kernel_mix": kernel_mix,
                     "all_stencil_launches": {"launches": st_n, "avg_launch_ms": st_ms / max(st_n, 1),
                                              "achieved_gbs": st_bytes / (st_ms / 1000.0) / 1e9,
                                              "share_of_step": st_ms / t_local}})

    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16s": "bf16-stored/f32", "fp64": "f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": wl.describe(), "lattice": "x".join(map(str, wl.dims)),
                       "noises_per_level": wl.nsamples, "levels": [list(x) for x in wl.levels],
                       "deflation_k": wl.k, "nrhs_per_launch": block, "launch_shape": launch,
                       "level_storage": per_level,
                       "stencil_options": {"fast": fast, "sweep": sweep,
                                           "segment": hm.mpmc_get_option(G.OPT_SWEEP_SEGMENT),
                                           "fast_sites": hm.mpmc_get_option(G.OPT_FAST_SITES)}, "l2": "flushed before every step (256 MB write)",
                       "parallelism": f"noise sharding x{world}", "matvecs_per_step": wl.matvecs_per_step(),
                       "setup_s": t_setup},
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "dslash_hbm_gbs": achieved_gbs, "cpu_baseline": cpu, "fp64": fp64,
            **extra,
            "deflation_kernel": {"ms_per_step": df_ms / args.steps, "launches": df_n,
                                 "achieved_gbs": (df_bytes / (df_ms / 1000.0) / 1e9) if df_ms else None},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mpmc", choices=["mpmc", "reference"])
    ap.add_argument("--workload", default="24^3x32")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16s", "fp64"])
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--oracle-noises", type=int, default=2)
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the dominant kernel from an ncu capture of this build")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--level-storage", default="auto",
                    help="vector storage per level, e.g. fp32,fp32,bf16s (auto: levels 0 and 1 in fp32 "
                         "with --precision bf16s, else all in --precision)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-inverse", action="store_true", help="skip timing the Tr(A^-1 - M_1) level")
    ap.add_argument("--inverse-noises", type=int, default=2)
    ap.add_argument("--no-probing", action="store_true", help="skip timing the probing of a degree-4 p_3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-worker", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_worker:
        spec = json.loads(args.oracle_worker)
        json.dump(oracle_worker(spec), open(spec["out"], "w"))
        return 0
    if args.impl == "reference":
        return reference_arm(args)
    if args.warmup < 3:
        log("note: fewer than 3 warm-up steps")
    if args.workload == BATCH_KEY:
        return batch_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
