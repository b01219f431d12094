"""Autotuning of the batched sampler: smoother and kernel schedule, with a cache.

The Chebyshev smoother of the V-cycle has three knobs: its degree (steps per
pre- and post-smoothing sweep) on the finest level and on the coarser ones,
and the ratio r of its interval [lambda_max / r, 1.1 lambda_max].  A higher degree costs more per V-cycle but
saves outer iterations; the best pair depends on the spline degree, the mesh
and the shifts.  The kernel schedule of a hierarchy (wm_schedule: tiles per
run of the one-shift stencil kernels, their grid target in waves, rows per
block of the vector and coarse-level kernels, the fused coarse end of the
V-cycle) changes how the batched solves
map onto the SMs, not their results beyond rounding order.

`tune` times `sample_fields` on the caller's problem (CUDA events, after a
warm-up call) for each candidate smoother pair, then improves the schedule one
knob at a time at the best pair (coordinate descent, two sweeps at most), and
returns the fastest setting.  `save` / `lookup` keep results in a JSON cache
keyed by (surface kind, spline degree, elements, levels, samples, precision,
GPU name); bench.py reads it at start-up.

    python -m paper_2605_24882_gb300.autotune --workload sphere_p2_j6_mixed_s256 [--write]
"""
import argparse
import itertools
import json
import os

import torch

DEGREES = (2, 3, 4, 5, 6)
RATIOS = (8.0, 12.0, 16.0, 24.0, 32.0)
SCHEDULE_CHOICES = {
    "uni_run": (2, 4, 8),
    "uni_waves": (2, 4, 8, 16),
    "vec_rows": (64, 128, 256, 512),
    "vcycle_rows": (8, 16, 32),
    "tail_fused": (0, 1),
}
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def _time(hier, kw):
    """ms of one sample_fields call after a warm-up call, or None when a system missed rtol."""
    _, st = hier.sample_fields(check_convergence=False, **kw)
    if st["n_not_converged"]:
        return None, st
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, st = hier.sample_fields(check_convergence=False, **kw)
    e1.record()
    torch.cuda.synchronize()
    if st["n_not_converged"]:
        return None, st
    return e0.elapsed_time(e1), st


def tune_smoother(hier, degrees=DEGREES, ratios=RATIOS, n_samples=32, **kw):
    """Time sample_fields for every (degree, ratio) pair on `n_samples` samples,
    then, at the best pair, every other degree on the coarser levels.

    kw: the remaining sample_fields arguments (kappa, beta, sinc_k, ...).
    Returns {"best": {"smoother_degree", "cheb_ratio", "smoother_degree_coarse",
    "ms"}, "table": [...]} (smoother_degree_coarse 0: the same degree).
    Settings whose solves do not converge are skipped.
    """
    kw = dict(kw, n_samples=n_samples)
    table = []
    for deg, ratio in itertools.product(degrees, ratios):
        ms, st = _time(hier, dict(kw, smoother_degree=deg, cheb_ratio=ratio))
        if ms is None:
            continue
        table.append({"smoother_degree": deg, "cheb_ratio": ratio, "smoother_degree_coarse": 0, "ms": ms,
                      "max_iterations": st["max_iterations"]})
    if not table:
        raise RuntimeError("no smoother setting converged")
    best = min(table, key=lambda r: r["ms"])
    for dc in degrees:
        if dc == best["smoother_degree"]:
            continue
        args = dict(kw, smoother_degree=best["smoother_degree"], cheb_ratio=best["cheb_ratio"],
                    smoother_degree_coarse=dc)
        ms, st = _time(hier, args)
        if ms is None:
            continue
        row = {"smoother_degree": best["smoother_degree"], "cheb_ratio": best["cheb_ratio"],
               "smoother_degree_coarse": dc, "ms": ms, "max_iterations": st["max_iterations"]}
        table.append(row)
    best = min(table, key=lambda r: r["ms"])
    return {"best": best, "table": table}


def tune_schedule(hier, choices=SCHEDULE_CHOICES, sweeps=2, **kw):
    """Coordinate descent over the hierarchy's kernel schedule for sample_fields(**kw).

    Starts from the hierarchy's current schedule; each sweep tries every value
    of each knob with the others fixed and keeps the fastest.  Leaves the best
    schedule set on the hierarchy and returns {"best": schedule, "ms", "table"}.
    """
    best = hier.schedule()
    best_ms, _ = _time(hier, kw)
    table = [dict(best, ms=best_ms)]
    for _ in range(sweeps):
        changed = False
        for knob, values in choices.items():
            for v in values:
                if v == best[knob]:
                    continue
                trial = dict(best, **{knob: v})
                hier.set_schedule(**trial)
                ms, _ = _time(hier, kw)
                table.append(dict(trial, ms=ms))
                if ms is not None and (best_ms is None or ms < best_ms):
                    best, best_ms, changed = trial, ms, True
            hier.set_schedule(**best)
        if not changed:
            break
    hier.set_schedule(**best)
    return {"best": best, "ms": best_ms, "table": table}


def cache_key(c, n_samples, gpu_name):
    """Key of a workload description (wm_workloads entry) on a GPU."""
    return "%s/p%d/%dx%d/L%d/s%d/%s/%s" % (c["kind"], c["p"], c["n_u"], c["n_v"], c["levels"], n_samples,
                                         c["precision"], gpu_name)


def lookup(key, path=CACHE):
    """The cached setting of `key`, or None."""
    if not os.path.exists(path):
        return None
    return json.load(open(path)).get(key)


def save(key, entry, path=CACHE):
    d = json.load(open(path)) if os.path.exists(path) else {}
    d[key] = entry
    with open(path, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)


def apply(hier, entry):
    """Set a cached entry's schedule on `hier`; returns its smoother kwargs."""
    hier.set_schedule(**entry["schedule"])
    return {"smoother_degree": entry["smoother_degree"], "cheb_ratio": entry["cheb_ratio"],
            "smoother_degree_coarse": entry.get("smoother_degree_coarse", 0)}


def tune(hier, c, n_samples, smoother_samples=0):
    """Smoother (on `smoother_samples` samples, 0: `n_samples`), then the
    schedule (on `n_samples`) for the workload description `c`; returns the
    cache entry.  The smoother is swept on the batch it will run: a pair that
    wins on a few samples can lose on the full batch (on the 256-sample sphere
    workload the best pair on 32 samples cost 3% at 256)."""
    kw = dict(kappa=c["kappa"], beta=c["beta"], sinc_k=c["k"], l_lo=c["l_lo"], l_hi=c["l_hi"], seed=c["seed"],
              split=c["split"], precision=c["precision"], rtol=c["rtol"])
    sm = tune_smoother(hier, n_samples=smoother_samples or n_samples, **kw)["best"]
    kw.update(n_samples=n_samples, smoother_degree=sm["smoother_degree"], cheb_ratio=sm["cheb_ratio"],
              smoother_degree_coarse=sm["smoother_degree_coarse"])
    sc = tune_schedule(hier, **kw)
    return {"smoother_degree": sm["smoother_degree"], "cheb_ratio": sm["cheb_ratio"],
            "smoother_degree_coarse": sm["smoother_degree_coarse"], "schedule": sc["best"],
            "ms": sc["ms"], "n_samples": n_samples, "table": sc["table"]}


def main():
    import paper_2605_24882_gb300 as wm
    from wm_workloads import WORKLOADS

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="sphere_p2_j6_mixed_s256")
    ap.add_argument("--samples", type=int, default=0, help="samples of the schedule sweep (0: the workload's)")
    ap.add_argument("--smoother-samples", type=int, default=0, help="samples of the smoother sweep (0: as above)")
    ap.add_argument("--write", action="store_true", help="store the result in the cache")
    ap.add_argument("--cache", default=CACHE, help="cache file (default: the package's tuned.json)")
    args = ap.parse_args()
    c = WORKLOADS[args.workload]
    hier = wm.Hierarchy(wm.Geometry(c["kind"], c["p"], c["n_u"], c["n_v"], c.get("R", 1.0), c.get("r", 0.4)),
                        c["levels"])
    ns = args.samples or c["n_samples"]
    entry = tune(hier, c, ns, args.smoother_samples)
    key = cache_key(c, c["n_samples"], torch.cuda.get_device_name())
    if args.write:
        save(key, {k: v for k, v in entry.items() if k != "table"}, args.cache)
    print(json.dumps(dict(entry, key=key, workload=args.workload)))


if __name__ == "__main__":
    main()
