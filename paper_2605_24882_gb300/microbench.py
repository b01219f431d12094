"""Component micro-benchmarks of the sampler's kernels on synthetic inputs.

    python -m paper_2605_24882_gb300.microbench vcycle [--kind sphere] [--p 2]
        [--elems 64] [--levels 6] [--tiles 71] [--tiles-per-shift 1] [--degree 4]
        [--ratio 12] [--precision mixed] [--reps 3] [--schedule knob=value ...]

`vcycle` runs `reps` V-cycles (the preconditioner of the batched solves) on
`tiles` x 32 seeded random residuals, 32 x `tiles-per-shift` per shift, the
shifts spread geometrically over [25 + e^-10, 25 + e^10] (sample-major packing
of a sinc pass puts n_s / 32 consecutive tiles on one shift), and prints the
mean time per V-cycle (`--schedule` sets fields of the hierarchy's kernel
schedule first, e.g. tail_fused=0).  It is the driver for kernel profiles of the smoother, residual and
transfer kernels.

    python -m paper_2605_24882_gb300.microbench sqrt [--kind sphere] [--p 2]
        [--elems 64] [--samples 64] [--nodes 12] [--rtol 1e-10] [--reps 2]

    python -m paper_2605_24882_gb300.microbench adjoint [--precision fp64]

`adjoint` times the differentiation workload (sphere 6 x 128 x 128, p = 3,
101,402 DOFs, 64 samples, kappa = 4, beta = 0.8, loss against target fields of
seed 7): the forward call keeping its per-node solutions, the backward that
reuses them, and the backward that re-solves them, each after a warm-up.

`sqrt` draws `samples` loads f = sqrt(M) y with the `nodes`-point rule on the
library's mass spectrum bounds `reps` times and prints the mean time per call
and the CG iterations.
"""
import argparse
import json

import numpy as np
import torch

import paper_2605_24882_gb300 as wm


def vcycle(args):
    hier = wm.Hierarchy(wm.Geometry(args.kind, args.p, args.elems), args.levels)
    if args.schedule:
        hier.set_schedule(**{k: int(v) for k, v in (a.split("=") for a in args.schedule)})
    n = hier.num_dofs(0)
    nsh = (args.tiles + args.tiles_per_shift - 1) // args.tiles_per_shift
    sig = np.repeat(np.exp(np.linspace(-10.0, 10.0, nsh)) + 25.0, 32 * args.tiles_per_shift)[:args.tiles * 32]
    g = torch.Generator(device="cuda").manual_seed(0)
    r = torch.randn((args.tiles * 32, n), dtype=torch.float64, device="cuda", generator=g)
    z = hier.vcycle(r, sig, precision=args.precision, smoother_degree=args.degree, cheb_ratio=args.ratio)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        z = hier.vcycle(r, sig, precision=args.precision, smoother_degree=args.degree, cheb_ratio=args.ratio)
    e1.record()
    torch.cuda.synchronize()
    cats = {}
    if args.profile:  # per-category device time of one more V-cycle (CUDA events per launch)
        wm.profile_enable(True)
        hier.vcycle(r, sig, precision=args.precision, smoother_degree=args.degree, cheb_ratio=args.ratio)
        torch.cuda.synchronize()
        prof = wm.profile_read()
        wm.profile_enable(False)
        cats = {k: {"ms": round(v["ms"], 4), "launches": v["timed"],
                    "gbs": round(v["bytes"] / (v["ms"] * 1e6), 1) if v["ms"] > 0 else None}
                for k, v in prof.items() if v["timed"] > 0}
    print(json.dumps({"bench": "vcycle", "dofs": n, "systems": args.tiles * 32, "levels": args.levels,
                      "schedule": hier.schedule(),
                      "tiles_per_shift": args.tiles_per_shift, "categories": cats,
                      "degree": args.degree, "ms_per_vcycle": e0.elapsed_time(e1) / max(1, args.reps),
                      "max_abs_z": float(z.abs().max())}))


def sqrt_noise(args):
    g = wm.Geometry(args.kind, args.p, args.elems)
    hier = wm.Hierarchy(g, 1)
    lo, hi = g.mass_bounds(0)
    f, it = hier.noise_loads_sqrt(1, args.samples, lo, hi, args.nodes, rtol=args.rtol)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for r in range(args.reps):
        f, it = hier.noise_loads_sqrt(2 + r, args.samples, lo, hi, args.nodes, rtol=args.rtol)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"bench": "sqrt_noise", "dofs": hier.num_dofs(0), "samples": args.samples,
                      "nodes": args.nodes, "systems": args.samples * args.nodes, "iterations": it,
                      "ms_per_call": e0.elapsed_time(e1) / max(1, args.reps),
                      "finite": bool(torch.isfinite(f).all())}))


def adjoint(args):
    from wm_workloads import WORKLOADS
    c = WORKLOADS["sphere_p3_j7_adjoint_s64"]
    hier = wm.Hierarchy(wm.Geometry(c["kind"], c["p"], c["n_u"]), c["levels"])
    ns, N = c["n_samples"], hier.num_dofs(0)
    kw = dict(beta=c["beta"], sinc_k=c["k"], l_lo=c["l_lo"], l_hi=c["l_hi"], n_samples=ns, kappa=c["kappa"],
              precision=args.precision, rtol=c["rtol"] if args.precision == "fp64" else 1e-8, max_iter=400)
    b = hier.noise_loads(c["seed"], ns)
    g = torch.stack([wm.normals(c["target_seed"], s, 1, 0, N) for s in range(ns)])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"bench": "adjoint", "dofs": N, "samples": ns, "precision": args.precision}

    def timed(fn):
        fn()  # warm-up
        torch.cuda.synchronize()
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    ms_f, (u, st) = timed(lambda: hier.sample_fields(b=b, ckpt="keep", **kw))
    grad_u = 2.0 * hier.apply_mass(u - g)
    ms_b, (_, gk, sb) = timed(lambda: hier.sample_fields_backward(b, grad_u, ckpt="keep", return_stats=True, **kw))
    ms_r, (_, gk_r, sr) = timed(lambda: hier.sample_fields_backward(b, grad_u, return_stats=True, **kw))
    out.update({"forward_ms": ms_f, "forward_kept": st["ckpt_kept"], "backward_from_checkpoint_ms": ms_b,
                "backward_ckpt_used": sb["ckpt_used"], "backward_recompute_ms": ms_r,
                "samples_per_s_forward_plus_backward": ns / ((ms_f + ms_b) / 1e3),
                "dLdkappa": gk, "dLdkappa_recompute": gk_r,
                "systems_backward": sb["n_systems"], "systems_backward_recompute": sr["n_systems"]})
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["vcycle", "sqrt", "adjoint"])
    ap.add_argument("--kind", default="sphere", choices=["sphere", "torus"])
    ap.add_argument("--p", type=int, default=2)
    ap.add_argument("--elems", type=int, default=64)
    ap.add_argument("--levels", type=int, default=6)
    ap.add_argument("--tiles", type=int, default=71)
    ap.add_argument("--tiles-per-shift", type=int, default=1)
    ap.add_argument("--profile", action="store_true", help="per-category times of one extra V-cycle")
    ap.add_argument("--degree", type=int, default=4)
    ap.add_argument("--ratio", type=float, default=12.0)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--samples", type=int, default=64)
    ap.add_argument("--nodes", type=int, default=12)
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--schedule", nargs="*", default=[], help="vcycle: schedule fields as knob=value")
    args = ap.parse_args()
    if args.what == "vcycle":
        vcycle(args)
    elif args.what == "adjoint":
        adjoint(args)
    else:
        sqrt_noise(args)


if __name__ == "__main__":
    main()
