"""A short, fixed run of the sweep kernels for profilers (ncu -k ... -c ...).

    python -m paper_1305_3440_gb300.profile_case [--dims 32 32 32 32] [--bulk fp32_12]
                                                 [--bulk-sweeps 8] [--polish-sweeps 4]

Creates one context on cuda:0, runs `--bulk-sweeps` sweeps in the bulk
precision, promotes (G applied to the FP64 input, pair storage) and runs
`--polish-sweeps` polish sweeps, then one exact measurement.  A 32^4 lattice
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
    args = ap.parse_args(argv)

    import torch
    from . import lgt, synth
    dims = tuple(args.dims)
    U = synth.field(dims, args.eps, args.seed)
    dev = torch.from_numpy(U).cuda()
    bulk = {"fp32_12": lgt.LGT_FP32_12, "fp32_18": lgt.LGT_FP32_18, "fp64": lgt.LGT_FP64}[args.bulk]
    gauge = lgt.LGT_LANDAU if args.gauge == "landau" else lgt.LGT_COULOMB
    p = lgt.lgt_params_default(dims=dims, gauge=gauge, omega=args.omega, bulk=bulk)
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
