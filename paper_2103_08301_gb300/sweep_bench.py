"""Batched parameter sweep versus sequential single-channel runs.

The sweep of the paper's Sec. 3.3 as a synthetic workload: 64 airway channels
of uneven size (height 128-512, length 1024-4096) with seeded pressure drop in
[5e-4, 3e-3], plug length in [64, 256] at x = length/4 and film thickness in
[4, 24] (SplitMix64 seed 3), CS EOS at 0.85 Tc, FP32. Both forms step every
channel the same number of steps; throughput is total node updates per second.

  python -m paper_2103_08301_gb300.sweep_bench --steps 200
  python -m paper_2103_08301_gb300.sweep_bench --batched-only --tma 1 --channels 16 --steps 5

`--batched-only` steps only the batch, with its default plan (no autotune),
tensor loads on or off (`--tma`) and a band height of the work order
(`--band`, 0 = strip by strip), for profiling one batch launch.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sweep_channels(n, seed):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import synth
    return synth.sweep_channels(n=n, seed=seed)


def shard_channels(sizes, world):
    """Split channels of `sizes` (node counts) over `world` ranks: largest
    first onto the least-loaded rank (ties to the lower rank), so every rank
    computes the same assignment. Returns one sorted list of channel indices
    per rank. The channels are independent problems: no data crosses ranks."""
    loads = [0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(world), key=lambda q: (loads[q], q))
        out[r].append(i)
        loads[r] += sizes[i]
    return [sorted(o) for o in out]


def run_sharded(rank, world, dist=None, steps=200, n=64, seed=3, precision=32):
    """The sweep split over `world` ranks (one GPU each): rank `rank` steps its
    shard of the channels as one batch; the time is the maximum over ranks
    (a barrier on both sides) and the throughput is all channels' node
    updates over it."""
    import torch

    import paper_2103_08301_gb300 as lbm

    kw = dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5)
    eos = lbm.lbm_eos(1.0, 4.0, 1.0, kw["T_over_Tc"], 1.0, kw["kappa"])
    _, g, l, _ = lbm.lbm_coexistence(eos)
    specs = _sweep_channels(n, seed)
    shard = shard_channels([s["nx"] * s["ny"] for s in specs], world)[rank]
    chans = [{"nx": specs[i]["nx"], "ny": specs[i]["ny"], "dp": specs[i]["dp"],
              "rho0": lbm.lbm_airway_rho0(specs[i]["nx"], specs[i]["ny"], specs[i]["film"], specs[i]["plug_x"],
                                          specs[i]["plug_len"], l, g)} for i in shard]
    nodes = sum(s["nx"] * s["ny"] for s in specs)
    with lbm.Batch(chans, precision=precision, **kw) as b:
        b.step(64)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        b.step(steps)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t = time.perf_counter() - t0
    if dist:
        tt = torch.tensor([t], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return {"channels": len(specs), "ranks": world, "shard_channels": len(shard), "nodes": nodes,
            "steps": steps, "batched_mlups": nodes * steps / t / 1e6, "scaling": "strong",
            "workload": "64 airway channels split over the ranks by node count (largest first)"}


def run(steps=200, n=64, seed=3, precision=32):
    import torch

    import paper_2103_08301_gb300 as lbm
    from paper_2103_08301_gb300 import build

    build.build()
    kw = dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5)
    eos = lbm.lbm_eos(1.0, 4.0, 1.0, kw["T_over_Tc"], 1.0, kw["kappa"])
    _, g, l, _ = lbm.lbm_coexistence(eos)
    specs = _sweep_channels(n, seed)
    chans = [{"nx": s["nx"], "ny": s["ny"], "dp": s["dp"],
              "rho0": lbm.lbm_airway_rho0(s["nx"], s["ny"], s["film"], s["plug_x"], s["plug_len"], l, g)}
             for s in specs]
    nodes = sum(c["nx"] * c["ny"] for c in chans)

    # sequential: one context after the other, each stepped alone
    stream = torch.cuda.Stream()
    seq_t = 0.0
    for c in chans:
        with lbm.Lattice(c["nx"], c["ny"], c["rho0"], precision=precision, dp=c["dp"], stream=stream,
                         **kw) as lat:
            lat.step(3)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lat.step(steps)
            torch.cuda.synchronize()
            seq_t += time.perf_counter() - t0

    # batched: one launch per step over every channel, one CTA per strip
    # column, replayed from graphs (the default), and one persistent
    # cooperative launch; autotuned plan
    bat = {}
    for mode, persistent in (("per_step", 0), ("persistent", 1)):
        with lbm.Batch(chans, precision=precision, **kw) as b:
            b.set_option(lbm.LBM_OPT_PERSISTENT, persistent)
            tune = b.autotune(trial_steps=10)
            b.step(64)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.step(steps)
            torch.cuda.synchronize()
            bat[mode] = (time.perf_counter() - t0, tune, b.launch_info(),
                         any(b.diag(i)["nan_detected"] for i in range(len(chans))))
    bat_t, tune, info, nan = bat["per_step"]
    return {
        "channels": len(chans), "nodes": nodes, "steps": steps, "precision": precision,
        "batched_mlups": nodes * steps / bat_t / 1e6, "sequential_mlups": nodes * steps / seq_t / 1e6,
        "persistent_launch_mlups": nodes * steps / bat["persistent"][0] / 1e6,
        "speedup": seq_t / bat_t, "autotune": tune, "launch": info, "nan": bool(nan or bat["persistent"][3]),
        "mode": "batched_mlups: one launch per step, one CTA per strip column, CUDA graphs (the library "
                "default); persistent_launch_mlups: one persistent cooperative launch",
        "workload": "64 airway channels, H 128-512, L 1024-4096, dp 5e-4..3e-3, plug 64-256, film 4-24 "
                    "(SplitMix64 seed 3), FP32",
    }


def run_batched_only(steps=5, n=16, seed=3, precision=32, tma=1, band=-1):
    import torch

    import paper_2103_08301_gb300 as lbm
    from paper_2103_08301_gb300 import build

    build.build()
    kw = dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5)
    eos = lbm.lbm_eos(1.0, 4.0, 1.0, kw["T_over_Tc"], 1.0, kw["kappa"])
    _, g, l, _ = lbm.lbm_coexistence(eos)
    chans = [{"nx": s["nx"], "ny": s["ny"], "dp": s["dp"],
              "rho0": lbm.lbm_airway_rho0(s["nx"], s["ny"], s["film"], s["plug_x"], s["plug_len"], l, g)}
             for s in _sweep_channels(n, seed)]
    nodes = sum(c["nx"] * c["ny"] for c in chans)
    with lbm.Batch(chans, precision=precision, **kw) as b:
        b.set_option(lbm.LBM_OPT_TMA, tma)
        b.set_option(lbm.LBM_OPT_BAND, band)
        b.step(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.step(steps)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        info = b.launch_info()
    return {"channels": n, "nodes": nodes, "steps": steps, "tma": tma, "band": band,
            "batched_mlups": nodes * steps / t / 1e6,
            "launch": info}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--channels", type=int, default=64)
    ap.add_argument("--batched-only", action="store_true")
    ap.add_argument("--tma", type=int, default=1, choices=[0, 1])
    ap.add_argument("--band", type=int, default=-1, help="LBM_OPT_BAND of the batched-only run")
    args = ap.parse_args()
    if args.batched_only:
        print(json.dumps(run_batched_only(steps=args.steps, n=args.channels, tma=args.tma, band=args.band)))
    else:
        print(json.dumps(run(steps=args.steps, n=args.channels)))


if __name__ == "__main__":
    main()
