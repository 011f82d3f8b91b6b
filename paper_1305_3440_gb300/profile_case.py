"""A short, fixed run of the sweep kernels for profilers (ncu -k ... -c ...).

    python -m paper_1305_3440_gb300.profile_case [--dims 32 32 32 32] [--bulk fp32_12]
                                                 [--bulk-sweeps 8] [--polish-sweeps 4]
                                                 [--polish anchor] [--launch-config K]

Creates one context on cuda:0, runs `--bulk-sweeps` sweeps in the bulk
precision, promotes (G applied to the FP64 input, then the polish set-up) and runs
`--polish-sweeps` polish sweeps, then one exact measurement.  Profilers
serialise launches, which misleads the autotuner: pass `--launch-config` to
profile the configuration a normal run picks.  A 32^4 lattice
keeps the FP32 links (201 MB for 12 reals) larger than the 129 MB L2 while the
whole context stays under 2 GB of device memory, and every half-sweep launch
covers the same 524288 sites as a 32^4 gauge fixing.
"""
import argparse

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[32, 32, 32, 32])
    ap.add_argument("--eps", type=float, default=0.5)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--gauge", default="landau", choices=["landau", "coulomb"])
    ap.add_argument("--bulk", default="fp32_12", choices=["fp32_12", "fp32_18", "fp64"])
    ap.add_argument("--omega", type=float, default=1.7)
    ap.add_argument("--bulk-sweeps", type=int, default=8)
    ap.add_argument("--polish-sweeps", type=int, default=4)
    ap.add_argument("--polish", default="anchor", choices=["anchor", "pair", "fp64"])
    ap.add_argument("--launch-config", type=int, default=-1,
                    help="force launch configuration k of the sweep kernels (-1: autotuned)")
    args = ap.parse_args(argv)

    import torch
    from . import lgt, synth
    dims = tuple(args.dims)
    U = synth.field(dims, args.eps, args.seed)
    dev = torch.from_numpy(U).cuda()
    bulk = {"fp32_12": lgt.LGT_FP32_12, "fp32_18": lgt.LGT_FP32_18, "fp64": lgt.LGT_FP64}[args.bulk]
    gauge = lgt.LGT_LANDAU if args.gauge == "landau" else lgt.LGT_COULOMB
    polish = {"anchor": lgt.LGT_POLISH_ANCHOR, "pair": lgt.LGT_POLISH_PAIR, "fp64": lgt.LGT_POLISH_FP64}[args.polish]
    p = lgt.lgt_params_default(dims=dims, gauge=gauge, omega=args.omega, bulk=bulk, polish=polish,
                               launch_config=args.launch_config + 1)
    ctx = lgt.lgt_create(p, dev)
    try:
        lgt.lgt_sweep(ctx, args.bulk_sweeps)
        lgt.lgt_promote(ctx)
        lgt.lgt_sweep(ctx, args.polish_sweeps)
        F, theta, plaq = lgt.lgt_measure(ctx)
        st = lgt.lgt_get_stats(ctx)
        print(f"dims={dims} bulk={args.bulk} sweeps={args.bulk_sweeps}+{args.polish_sweeps} "
              f"F={F:.15f} theta={theta:.3e} plaquette={plaq:.15f} "
              f"launch_config={list(st.launch_config)}")
        if not np.isfinite(F):
            raise SystemExit("non-finite F")
    finally:
        lgt.lgt_destroy(ctx)


if __name__ == "__main__":
    main()
