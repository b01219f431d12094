"""Smoother autotuning for the batched sampler.

The Chebyshev smoother of the V-cycle has two knobs: its degree (steps per
pre- and post-smoothing sweep) and the ratio r of its interval
[lambda_max / r, 1.1 lambda_max].  A higher degree costs more per V-cycle but
saves outer iterations; the best pair depends on the spline degree, the mesh
and the shifts.  `tune_smoother` times `sample_fields` on a small number of
samples of the caller's problem for each candidate pair (CUDA events, after a
warm-up call) and returns the fastest.

    python -m paper_2605_24882_gb300.autotune --workload torus_p3_512x256_s1024
"""
import argparse
import itertools
import json

import torch

DEGREES = (2, 3, 4, 5, 6)
RATIOS = (8.0, 12.0, 16.0, 24.0, 32.0)


def tune_smoother(hier, degrees=DEGREES, ratios=RATIOS, n_samples=32, **kw):
    """Time sample_fields for every (degree, ratio) pair on `n_samples` samples.

    kw: the remaining sample_fields arguments (kappa, beta, sinc_k, ...).
    Returns {"best": {"smoother_degree", "cheb_ratio", "ms"}, "table": [...]}.
    Pairs whose solves do not converge are skipped.
    """
    kw = dict(kw, n_samples=n_samples)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    table = []
    for deg, ratio in itertools.product(degrees, ratios):
        args = dict(kw, smoother_degree=deg, cheb_ratio=ratio)
        _, st = hier.sample_fields(check_convergence=False, **args)  # warm-up (shift tables, workspace)
        if st["n_not_converged"]:
            continue
        torch.cuda.synchronize()
        e0.record()
        _, st = hier.sample_fields(check_convergence=False, **args)
        e1.record()
        torch.cuda.synchronize()
        if st["n_not_converged"]:
            continue
        table.append({"smoother_degree": deg, "cheb_ratio": ratio, "ms": e0.elapsed_time(e1),
                      "max_iterations": st["max_iterations"]})
    if not table:
        raise RuntimeError("no smoother setting converged")
    best = min(table, key=lambda r: r["ms"])
    return {"best": best, "table": table}


def main():
    import paper_2605_24882_gb300 as wm
    from wm_workloads import WORKLOADS

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="sphere_p2_j6_mixed_s256")
    ap.add_argument("--samples", type=int, default=32)
    args = ap.parse_args()
    c = WORKLOADS[args.workload]
    hier = wm.Hierarchy(wm.Geometry(c["kind"], c["p"], c["n_u"], c["n_v"], c.get("R", 1.0), c.get("r", 0.4)),
                        c["levels"])
    res = tune_smoother(hier, n_samples=args.samples, kappa=c["kappa"], beta=c["beta"], sinc_k=c["k"],
                        l_lo=c["l_lo"], l_hi=c["l_hi"], seed=c["seed"], split=c["split"], precision=c["precision"],
                        rtol=c["rtol"])
    print(json.dumps(dict(res, workload=args.workload, samples=args.samples)))


if __name__ == "__main__":
    main()
