"""Throughput of batched Whittle–Matérn field sampling on GB300.

One step = one call of the sampler (the whole hot path): Philox white-noise
loads for 256 samples, the integer-part solve and the 71 shifted solves of
every sample (18,432 systems of 25,352 DOFs, batched PCG with the float32
multigrid V-cycle, float64 outer iteration), and the float64 sinc sum, on the
six-patch unit sphere with 64 x 64 bi-quadratic elements per patch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun rank r samples fields r*256 .. r*256+255 of one noise sequence
(no collective on the data path: weak scaling); rank 0 prints one JSON line.
"""
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

from wm_workloads import WORKLOADS  # noqa: E402

METRIC = "field samples/s & DOF-solves/s at ≤1e-6 rel err: batched mixed vs plain FP64"
WORKLOAD = "sphere_p2_j6_mixed_s256"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# CUDA-core peaks of GB300 from unit counts and the 2070 MHz maximum SM clock:
# FP32: 152 SMs x 128 lanes x 2 flop x 2.07 GHz; FP64: the recipe's nominal 1.25 TFLOP/s
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "wm_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for name, val in zip(names[1:], f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def init_group(world, rank, backend):
    """One process per GPU (torchrun environment); the N > 1 path has no
    data-path collective: only the barriers and the max-over-ranks timing."""
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        kw = {}
        if backend == "nccl":
            import torch
            kw["device_id"] = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend, rank=rank, world_size=world, **kw)


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    torch.cuda.set_device(local)
    init_group(world, rank, "nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cuda"):
    """The slowest rank's value (each rank times its own replica)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_samples(rank, samples_per_rank):
    """Sample range [first, first + n) of a rank: the job's samples 0 .. N n - 1
    under one noise seed, split into contiguous blocks (rank r draws the same
    loads and fields as rows r n .. (r + 1) n - 1 of a one-GPU run of N n)."""
    return rank * samples_per_rank, samples_per_rank


def job_rate(world, samples_per_rank, ms_per_step):
    """Whole-job samples/s: all ranks' samples over the slowest rank's step time."""
    return world * samples_per_rank / (ms_per_step / 1e3)


# ------------------------------------------------------------------ oracle timing
def oracle_estimate(c, n_shifts=4, n_sub=2):
    """Oracle cost of the workload from a bounded sample, extrapolated linearly.

    Times the oracle's assembly, its loads for n_sub samples, and the sparse LU
    factorisation plus n_sub solves for n_shifts of the shifted matrices; the
    full workload is n_nodes + n_int shifted matrices, each solved for every sample.
    """
    import numpy as np
    from oracle import geometry as geo
    from oracle.assembly import assemble
    from oracle.fractional import Shifted, sinc_rule, split_beta
    from oracle.noise import noise_loads
    from oracle.space import GluedSpace

    t0 = time.perf_counter()
    s = geo.Surface(c["kind"], c["p"], c["n_u"], c["n_v"], c.get("R", 1.0), c.get("r", 0.4))
    sp_ = GluedSpace(s)
    S, M = assemble(sp_)
    t_asm = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = noise_loads(sp_, c["seed"], n_sub)
    t_noise = (time.perf_counter() - t0) / n_sub
    n, bp, passes = split_beta(c["beta"], c["split"])
    y, _ = sinc_rule(bp, c["k"], c["l_lo"], c["l_hi"])
    sig = np.exp(y) + c["kappa"] ** 2
    n_mats = len(y) + (1 if n > 0 else 0)
    sh = Shifted(S, M)
    t_fact, t_solve = 0.0, 0.0
    for k in range(n_shifts):
        sg = float(sig[(k * 17) % len(sig)])
        t0 = time.perf_counter()
        sh.solve(sg, b[:1].T)
        t1 = time.perf_counter()
        sh.solve(sg, b.T)
        t2 = time.perf_counter()
        t_fact += (t1 - t0) - (t2 - t1) / n_sub
        t_solve += (t2 - t1) / n_sub
    t_fact /= n_shifts
    t_solve /= n_shifts
    ns = c["n_samples"]
    total = t_asm + ns * t_noise + n_mats * t_fact + n_mats * passes * ns * t_solve
    sample = ("assembly, loads of %d samples, LU factorisation of %d of the %d shifted matrices with %d solves "
              "each; extrapolated linearly to %d matrices x %d samples" % (n_sub, n_shifts, n_mats, n_sub, n_mats, ns))
    return ns / total, total, sample, sp_.N


def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c = WORKLOADS[args.workload]
    vals, times = [], []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        v, _, sample, N = oracle_estimate(c, n_shifts=1, n_sub=2)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            vals.append(v)
            times.append(dt)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "dofs": N},
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": 1, "host_cores": os.cpu_count(),
                             "kind": "oracle", "sample": "per step: " + sample},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def roofline(prof, pk, pk_kind):
    """Dominant kernel category by device time; achieved vs peak of its bound."""
    name, d = max(prof.items(), key=lambda kv: kv[1]["ms"])
    sec = d["ms"] / 1e3
    if sec <= 0 or d["timed"] == 0:
        return None, name
    gbs = d["bytes"] / sec / 1e9
    tfl = d["flops"] / sec / 1e12
    is64 = name in ("true_residual_f64",)
    alu_peak = FP64_PEAK_TFLOPS if is64 else FP32_PEAK_TFLOPS
    t_alu = d["flops"] / (alu_peak * 1e12)
    t_hbm = d["bytes"] / (pk["hbm_gbs"] * 1e9)
    per_launch = d["bytes"] / d["timed"]
    if t_hbm >= t_alu:
        r = {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
             "peak_kind": pk_kind + " (MEASURED_PEAKS.json hbm_gbs)" if pk_kind == "measured" else pk_kind}
    else:
        r = {"bound": "alu", "achieved": tfl, "peak": alu_peak, "unit": "TFLOP/s", "frac": tfl / alu_peak,
             "peak_kind": ("nominal FP64 1.25 TFLOP/s" if is64 else
                           "FP32 CUDA cores 152 SMs x 128 lanes x 2 x 2.07 GHz")}
    r.update({"kernel": name, "launches": d["timed"], "avg_launch_ms": d["ms"] / d["timed"],
              "alg_bytes_per_launch": per_launch, "alg_flops_per_launch": d["flops"] / d["timed"],
              "traffic": traffic_for(name, per_launch)})
    return r, name


def traffic_for(name, alg_bytes_per_launch):
    """DRAM bytes per launch of category `name`: the committed ncu capture's
    DRAM bytes per algorithmic byte (taken on a smaller case of the same
    kernel) times this run's algorithmic bytes per launch, if the capture was
    taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(name)
    if not e:
        return None
    src = os.path.join(ROOT, "paper_2605_24882_gb300", "csrc", e["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != e["source_sha"]:
        return None
    return e["dram_per_alg_byte"] * alg_bytes_per_launch


def surface_text(c):
    if c["kind"] == "sphere":
        return "unit sphere, 6 patches x %d x %d elements, p = %d" % (c["n_u"], c["n_v"], c["p"])
    return "torus R = %g, r = %g, one periodic patch of %d x %d elements, p = %d" % (
        c.get("R", 1.0), c.get("r", 0.4), c["n_u"], c["n_v"], c["p"])


def fp64_legs(hier, kw, u_mixed, N, systems_per_sample, args):
    """The same fields by the plain FP64 path, outside the timed region: (1) the
    batched solve in FP64 (same kernels, FP64 V-cycle); (2) one system at a
    time (max_systems = 1, FP64), timed on a bounded number of samples.  Also
    the relative M-norm distance of the mixed fields from the FP64 ones."""
    import torch

    out = {}
    ns = kw["n_samples"]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kwb = dict(kw, precision="fp64")
    u64 = torch.empty_like(u_mixed)
    hier.sample_fields(out=u64, **kwb)  # warm-up (FP64 workspace, shift tables)
    torch.cuda.synchronize()
    e0.record(stream)
    hier.sample_fields(out=u64, **kwb)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    out["batched_fp64"] = {"value": ns / t, "unit": "samples/s", "ms_per_step": 1e3 * t,
                           "dof_solves_per_s": N * systems_per_sample * ns / t}
    d = u_mixed - u64
    md = hier.apply_mass(d)
    mu = hier.apply_mass(u64)
    rel = torch.sqrt((d * md).sum(1) / (u64 * mu).sum(1))
    out["mixed_vs_fp64_rel_mnorm_max"] = float(rel.max())
    n1 = max(1, args.plain_samples)
    kwp = dict(kw, n_samples=n1, precision="fp64", max_systems=1)
    u1 = torch.empty((n1, N), dtype=torch.float64, device="cuda")
    hier.sample_fields(out=u1, **dict(kwp, n_samples=1))  # warm-up
    torch.cuda.synchronize()
    e0.record(stream)
    hier.sample_fields(out=u1, **kwp)
    e1.record(stream)
    torch.cuda.synchronize()
    t1 = e0.elapsed_time(e1) / 1e3
    out["plain_fp64_one_system_at_a_time"] = {
        "value": n1 / t1, "unit": "samples/s", "dof_solves_per_s": N * systems_per_sample * n1 / t1,
        "sample": "%d sample(s) = %d systems, each solved alone (one tile, FP64 V-cycle and CG, same rtol)"
                  % (n1, n1 * systems_per_sample)}
    return out


def tuned_setting(hier, c, args):
    """Smoother pair and kernel schedule of a workload: the autotuner's cache
    entry for this workload and GPU when there is one (applied to `hier`),
    else the workload's smoother pair and the library's default schedule;
    --smoother-degree / --cheb-ratio override the pair."""
    import torch
    from paper_2605_24882_gb300 import autotune
    key = autotune.cache_key(c, c["n_samples"], torch.cuda.get_device_name())
    entry = autotune.lookup(key)
    if entry:
        smoother, source = autotune.apply(hier, entry), "autotune cache " + key
    else:
        smoother = {"smoother_degree": c.get("smoother_degree", 4), "cheb_ratio": c.get("cheb_ratio", 12.0),
                    "smoother_degree_coarse": 0}
        source = "workload defaults (no cache entry for %s)" % key
    if args.smoother_degree:
        smoother["smoother_degree"] = args.smoother_degree
    if args.cheb_ratio:
        smoother["cheb_ratio"] = args.cheb_ratio
    return {"source": source, "smoother": smoother, "schedule": hier.schedule()}


def secondary_leg(wm, name, pk, pk_kind, args):
    """A second workload on the same GPU, same protocol at fewer steps: one
    warm-up step, `secondary_steps` timed steps with profiling off, then one
    profiled step for the per-kernel times and the dominant kernel's roofline."""
    import torch
    c = WORKLOADS[name]
    hier = wm.Hierarchy(wm.Geometry(c["kind"], c["p"], c["n_u"], c["n_v"], c.get("R", 1.0), c.get("r", 0.4)),
                        c["levels"])
    N = hier.num_dofs(0)
    ns = c["n_samples"]
    tuning = tuned_setting(hier, c, argparse.Namespace(smoother_degree=0, cheb_ratio=0.0))
    kw = dict(kappa=c["kappa"], beta=c["beta"], sinc_k=c["k"], l_lo=c["l_lo"], l_hi=c["l_hi"], n_samples=ns,
              seed=c["seed"], split=c["split"], precision=c["precision"], rtol=c["rtol"], **tuning["smoother"])
    u = torch.empty((ns, N), dtype=torch.float64, device="cuda")
    _, stats = hier.sample_fields(out=u, **kw)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.secondary_steps):
        _, stats = hier.sample_fields(out=u, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.secondary_steps
    wm.profile_enable(True)
    hier.sample_fields(out=u, **kw)
    torch.cuda.synchronize()
    prof = wm.profile_read()
    wm.profile_enable(False)
    rl, _ = roofline(prof, pk, pk_kind)
    n_int, _, passes = wm.beta_plan(c["beta"], c["split"])
    systems = ns * (n_int + passes * (c["l_hi"] - c["l_lo"] + 1))
    out = {"workload": name, "surface": surface_text(c), "dofs": N, "samples": ns, "systems_per_step": systems,
           "value": ns / (ms / 1e3), "unit": "samples/s", "ms_per_step": ms, "steps": args.secondary_steps,
           "warmup": 1, "dof_solves_per_s": N * systems / (ms / 1e3), "precision": c["precision"],
           "solver": {k: stats[k] for k in ("max_iterations", "n_not_converged", "max_rel_residual", "n_batches")},
           "roofline": rl, "kernel_ms_per_step": {k: v["ms"] for k, v in prof.items() if v["ms"] > 0},
           "tuning": tuning}
    del u, hier
    torch.cuda.empty_cache()
    return out


def uneven_arm(args):
    """The uneven batch: 96 sphere and torus instances (levels 3..9, seed 11) in
    one wm_sample_fields_batched call per step, one hierarchy per distinct
    surface.  A first call with per-launch profiling gives the per-category
    times and the roofline; the timed steps run with profiling off."""
    import torch

    import paper_2605_24882_gb300 as wm
    from wm_workloads import uneven_instances

    pk, pk_kind = peaks()
    insts = uneven_instances()
    hiers, H, D = {}, [], []
    t0 = time.perf_counter()
    for c in insts:
        key = (c["kind"], c["n_u"], c["n_v"])
        if key not in hiers:
            hiers[key] = wm.Hierarchy(wm.Geometry(c["kind"], c["p"], c["n_u"], c["n_v"], c.get("R", 1.0),
                                                  c.get("r", 0.4)), c["levels"])
        H.append(hiers[key])
        D.append(wm.Hierarchy.make_desc(c["kappa"], c["beta"], c["k"], c["l_lo"], c["l_hi"], c["n_samples"],
                                        c["seed"], c["split"], c["precision"], c["rtol"]))
    setup_s = time.perf_counter() - t0
    outs = [torch.empty((d.n_samples, h.num_dofs(0)), dtype=torch.float64, device="cuda") for h, d in zip(H, D)]
    wm.profile_enable(True)
    _, stats = wm.sample_fields_batched(H, D, outs=outs)
    torch.cuda.synchronize()
    prof = wm.profile_read()
    wm.profile_enable(False)
    rl, _ = roofline(prof, pk, pk_kind)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    e0.record(stream)
    for _ in range(args.steps):
        _, stats = wm.sample_fields_batched(H, D, outs=outs)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    samples = sum(d.n_samples for d in D)
    dof_solves = sum(h.num_dofs(0) * st["n_systems"] for h, st in zip(H, stats))
    line = {"metric": METRIC, "value": samples / (ms / 1e3), "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
            "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": "uneven96", "instances": len(D), "surfaces": len(hiers),
                       "dofs": [min(h.num_dofs(0) for h in H), max(h.num_dofs(0) for h in H)],
                       "samples": samples, "systems_per_step": sum(st["n_systems"] for st in stats),
                       "precision": "mixed", "rtol": insts[0]["rtol"], "split": "improved",
                       "hierarchy_setup_s": setup_s},
            "dof_solves_per_s": dof_solves / (ms / 1e3),
            "solver": {"n_not_converged": sum(st["n_not_converged"] for st in stats),
                       "max_rel_residual": max(st["max_rel_residual"] for st in stats),
                       "max_iterations": max(st["max_iterations"] for st in stats)},
            "gpu_launches": sum(v["launches"] for v in prof.values()),
            "roofline": rl, "kernel_ms_profiled_call": {k: v["ms"] for k, v in prof.items() if v["ms"] > 0},
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def our_arm(args):
    import torch

    import paper_2605_24882_gb300 as wm

    world, rank, local = dist_setup(args.gpus)
    c = WORKLOADS[args.workload]
    pk, pk_kind = peaks()
    hier = wm.Hierarchy(wm.Geometry(c["kind"], c["p"], c["n_u"], c["n_v"], c.get("R", 1.0), c.get("r", 0.4)),
                        c["levels"])
    N = hier.num_dofs(0)
    ns = args.samples or c["n_samples"]
    tuning = tuned_setting(hier, c, args)
    kw = dict(kappa=c["kappa"], beta=c["beta"], sinc_k=c["k"], l_lo=c["l_lo"], l_hi=c["l_hi"], n_samples=ns,
              seed=c["seed"], sample0=rank_samples(rank, ns)[0], split=c["split"], precision=c["precision"],
              rtol=c["rtol"], preconditioner=args.preconditioner, **tuning["smoother"])
    u = torch.empty((ns, N), dtype=torch.float64, device="cuda")
    stats = None
    for _ in range(args.warmup):
        _, stats = hier.sample_fields(out=u, **kw)
    torch.cuda.synchronize()
    # timed region: no per-launch events (profiling off); launches are counted
    wm.profile_enable(False)
    before = wm.profile_read()
    barrier(world)
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, stats = hier.sample_fields(out=u, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    after = wm.profile_read()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    launches = sum(after[k]["launches"] - before[k]["launches"] for k in after)
    # a separate profiled pass (CUDA events around every launch) gives the
    # per-category device times and the dominant kernel's roofline
    prof = {}
    if args.profile and args.profile_steps > 0:
        wm.profile_enable(True)
        for _ in range(args.profile_steps):
            hier.sample_fields(out=u, **kw)
        torch.cuda.synchronize()
        prof = wm.profile_read()
        wm.profile_enable(False)
    value = job_rate(world, ns, ms)
    n_int, bf, passes = wm.beta_plan(c["beta"], c["split"])
    n_nodes = c["l_hi"] - c["l_lo"] + 1
    dof_solves = world * N * (n_int + passes * n_nodes) * ns / (ms / 1e3)
    # end to end through the C ABI with a pinned host output buffer: the
    # device->host copy of every step's fields is inside the timed region
    host = torch.empty((ns, N), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        hier.sample_fields(out=host, **kw)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / max(1, args.e2e_steps), world)
    rl, dominant = roofline(prof, pk, pk_kind) if prof else (None, None)
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": args.workload, "surface": surface_text(c),
                       "dofs": N, "samples_per_gpu": ns, "integer_solves": n_int, "sinc_nodes": n_nodes,
                       "systems_per_step": ns * (n_int + passes * n_nodes), "rtol": c["rtol"],
                       "precision": c["precision"], "parallelism": "replicas" if world > 1 else "single GPU",
                       "preconditioner": args.preconditioner,
                       "smoother": {"chebyshev_degree": kw["smoother_degree"], "interval_ratio": kw["cheb_ratio"],
                                    "chebyshev_degree_coarse": kw["smoother_degree_coarse"] or kw["smoother_degree"]},
                       "tuning": tuning,
                       "l2": "inputs larger than L2: the batch working set is %.0f GB per step"
                             % (N * ns * (n_int + passes * n_nodes) * 40 / 1e9)},
            "dof_solves_per_s": dof_solves,
            "solver": {k: stats[k] for k in ("max_iterations", "total_iterations", "n_not_converged",
                                             "max_rel_residual", "n_systems", "n_batches", "n_replacements",
                                             "n_df_fallbacks")},
            "e2e": {"value": world * ns / (e2e_ms / 1e3) if args.e2e_steps else None, "unit": "samples/s",
                    "h2d_bytes_per_step": 120, "d2h_bytes_per_step": ns * N * 8},
            "gpu_launches": launches,
            "roofline": rl,
            "kernel_ms_per_step": {k: v["ms"] / args.profile_steps for k, v in prof.items() if v["ms"] > 0},
            "kernel_alg_gbs": {k: v["bytes"] / (v["ms"] * 1e6) for k, v in prof.items()
                               if v["ms"] > 0 and v["bytes"] > 0},
            "profiled_steps": args.profile_steps if prof else 0,
            "clocks": clocks}
    if not args.no_fp64_legs:
        legs = fp64_legs(hier, kw, u, N, n_int + passes * n_nodes, args)
        legs["speedup_batched_mixed_vs_plain_fp64"] = value / world / legs["plain_fp64_one_system_at_a_time"]["value"]
        legs["speedup_batched_mixed_vs_batched_fp64"] = value / world / legs["batched_fp64"]["value"]
        line["fp64_comparison"] = legs
    if world == 1 and args.secondary and args.secondary != args.workload:
        del u, hier
        torch.cuda.empty_cache()
        line["secondary"] = secondary_leg(wm, args.secondary, pk, pk_kind, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, total, sample, _ = oracle_estimate(c)
        line["cpu_baseline"] = {"value": v, "unit": "samples/s", "cores": 1, "host_cores": os.cpu_count(),
                                "kind": "oracle", "sample": sample, "extrapolated_seconds_per_step": total}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--samples", type=int, default=0, help="override the samples per GPU (profiling runs)")
    ap.add_argument("--no-fp64-legs", action="store_true", help="skip the plain FP64 comparison legs")
    ap.add_argument("--preconditioner", default="vcycle", choices=["vcycle", "bpx"])
    ap.add_argument("--plain-samples", type=int, default=1,
                    help="samples timed on the one-system-at-a-time FP64 path")
    ap.add_argument("--smoother-degree", type=int, default=0, help="0: the workload's tuned value")
    ap.add_argument("--cheb-ratio", type=float, default=0.0, help="0: the workload's tuned value")
    ap.add_argument("--no-profile", dest="profile", action="store_false")
    ap.add_argument("--profile-steps", type=int, default=2,
                    help="steps of the separate profiled pass (per-kernel times, roofline)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--secondary", default="torus_p3_512x256_s1024",
                    help="a second workload reported in the line's `secondary` object ('' for none)")
    ap.add_argument("--secondary-steps", type=int, default=2)
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "uneven96":
        uneven_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
