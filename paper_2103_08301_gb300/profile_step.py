"""Run the fused step kernel on an airway channel of a chosen size (for ncu).

The channel is the benchmark geometry scaled to nx x ny: walls top and
bottom, wall films ny/32 thick, a liquid plug nx/16 long at x = nx/4,
pressure columns with a drop of 1e-3, CS EOS at 0.85 Tc, tau = 1, k = 1,
kappa = 0.5, seeded synthetic initial density.

  python -m paper_2103_08301_gb300.profile_step --nx 4096 --ny 2048 --steps 5 [--precision 32] [--mask]
      [--inplace]

Prints the mean step time and effective bandwidth (72 B/node in FP32; 116
B/node for an in-place context, whose step is a density pass and a collide pass).
"""
from __future__ import annotations

import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--staged", type=int, default=1, help="1: bulk-copy staged kernel, 0: register prefetch")
    ap.add_argument("--prefetch", type=int, default=-1, help="LBM_OPT_PREFETCH (row pairs ahead); -1: default")
    ap.add_argument("--mask", action="store_true",
                    help="constrictions on both walls every 2048 columns (the general-geometry kernels)")
    ap.add_argument("--inplace", action="store_true", help="an lbm_init_inplace context (in-place streaming)")
    args = ap.parse_args()

    import torch

    import paper_2103_08301_gb300 as lbm
    from paper_2103_08301_gb300 import build

    build.build()
    eos = lbm.lbm_eos(1.0, 4.0, 1.0, 0.85, 1.0, 0.5)
    _, g, l, _ = lbm.lbm_coexistence(eos)
    nx, ny = args.nx, args.ny
    rho0 = lbm.lbm_airway_rho0(nx, ny, ny / 32.0, nx / 4.0, nx / 16.0, l, g)
    stream = torch.cuda.Stream()
    mask = None
    if args.mask:
        import numpy as np
        mask = np.zeros((ny, nx), np.uint8)
        for x0 in range(1024, nx - 512, 2048):
            mask[1:ny // 4, x0:x0 + 64] = 1
            mask[ny - ny // 4:ny - 1, x0:x0 + 64] = 1
    with lbm.Lattice(nx, ny, rho0, walls=True, bc_x=True, precision=args.precision, T_over_Tc=0.85,
                     kappa=0.5, dp=1e-3, stream=stream, mask=mask, inplace=args.inplace) as lat:
        lat.set_option(lbm.LBM_OPT_STAGED, args.staged)
        if args.ctas_per_sm:
            lat.set_option(lbm.LBM_OPT_CTAS_PER_SM, args.ctas_per_sm)
        if args.prefetch >= 0:
            lat.set_option(lbm.LBM_OPT_PREFETCH, args.prefetch)
        lat.step(2)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lat.step(args.steps)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        info = lat.launch_info()
        nan = lat.diag()["nan_detected"]
    bpn = (116 if args.inplace else 72) if args.precision == 32 else (232 if args.inplace else 144)
    print(json.dumps({"nx": nx, "ny": ny, "precision": args.precision, "inplace": args.inplace, "ms_per_step": ms,
                      "GBps": bpn * nx * ny / ms / 1e6, "MLUPS": nx * ny / ms / 1e3,
                      "launch": info, "nan": nan}))


if __name__ == "__main__":
    main()
