"""Run the discrete adjoint (forward with checkpoints, backward) on an airway
channel (for ncu and timing).

The channel is the adjoint workload's geometry scaled to nx x ny: walls top
and bottom, film 6, plug 48 at x = nx/4 (plug_len nx * 3/32 when nx != 512),
pressure columns with a drop of 1e-3, CS EOS at 0.85 Tc, kappa = 0.5, seeded
synthetic initial density (noise 1e-3).

  python -m paper_2103_08301_gb300.profile_adjoint --nx 512 --ny 128 --steps 2000 [--precision 32]
      [--reverse-precision 32]

Prints the forward and backward wall times and the reverse throughput.
"""
from __future__ import annotations

import argparse
import json
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--ny", type=int, default=128)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--block-steps", type=int, default=100)
    ap.add_argument("--reverse-precision", type=int, default=64, choices=[32, 64])
    ap.add_argument("--repeat", type=int, default=1, help="backward passes timed (the first is reported too)")
    args = ap.parse_args()

    import torch

    import paper_2103_08301_gb300 as lbm
    from paper_2103_08301_gb300 import adjoint as adjm
    from paper_2103_08301_gb300 import build

    build.build()
    nx, ny = args.nx, args.ny
    _, g, l, _ = lbm.lbm_coexistence(lbm.lbm_eos(1.0, 4.0, 1.0, 0.85, 1.0, 0.5))
    plug = 48.0 if nx == 512 else nx * 3 / 32
    r0 = lbm.lbm_airway_rho0(nx, ny, 6.0, nx / 4, plug, l, g, 4.0, 1e-3, 1)
    out = {"nx": nx, "ny": ny, "steps": args.steps, "precision": args.precision,
           "reverse_precision": args.reverse_precision}
    with adjm.Adjoint(nx, ny, args.steps, walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5,
                      block_steps=args.block_steps, precision=args.precision,
                      reverse_precision=args.reverse_precision) as adj:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J = adj.forward(r0, dp=1e-3)
        t1 = time.perf_counter()
        bw = []
        for _ in range(args.repeat):
            t2 = time.perf_counter()
            gr, gd = adj.backward(1.0, 1.0)
            bw.append(time.perf_counter() - t2)
    out.update({"J": list(J), "forward_s": t1 - t0, "backward_s": bw, "grad_dp": gd["dp"],
                "grad_rho0_sum": float(gr.sum()),
                "reverse_mlups": nx * ny * args.steps / min(bw) / 1e6})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
