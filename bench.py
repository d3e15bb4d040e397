"""Benchmark of the fused EOS-multiphase LBM step on GB300.

Workload (one "step" = one lattice time step, i.e. one pass of the whole hot
path over the lattice): the airway channel scaled to 16384 x 2048 nodes
(walls top and bottom, wall films 64 nodes thick, a liquid plug over
x in [4096, 5120), pressure inlet/outlet with a drop of 1e-3, Carnahan-Starling
EOS at T = 0.85 Tc, tau = 1, k = 1, kappa = 0.5), FP32 populations, synthetic
seeded initial density. The channel sits at the method's own coexistence: the
inlet column at its saturation pressure p* (p_ref = p* - dp/2, so the upstream
vapour is saturated rather than supersaturated), films and plug at its liquid
density in its vapour (p*, rho_g*, rho_l* from a relaxed flat slab). The 2.4 GB
state (two population arrays) is far larger than L2, so no flush is needed
between steps.

Metric: MLUPS (million lattice-node updates per second, nx*ny*steps/t/1e6),
whole job over N GPUs, each GPU stepping its own replica of the channel (the
path shards by independent channels: weak scaling, no collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NX, NY = 16384, 2048
FILM, PLUG_X, PLUG_LEN = 64.0, 4096.0, 1024.0
PHYS = dict(T_over_Tc=0.85, k=1.0, kappa=0.5, tau=1.0, dp=1e-3)
BYTES_PER_NODE = {32: 72, 64: 144}  # 9 populations read + 9 written
METRIC = "MLUPS and % of HBM roofline (FP32 D2Q9 EOS step, 1xGB300) vs FP64 CPU oracle"
WORKLOAD = ("airway channel 16384x2048, FP32, CS EOS T=0.85Tc, dp=1e-3, inlet at the method's coexistence "
            "pressure (roofline stress)")
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e nominal
KERNEL_SRC = [os.path.join(ROOT, "paper_2103_08301_gb300", "csrc", f) for f in ("lbm_kernels.cuh", "lbm_rows2.cuh")]
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "step_kernel_rows2_fp32_16384x2048.md")


def _dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm_gb_s"):
                if k in d and d[k]:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def _kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SRC:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def _profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    vals = {}
    for line in open(PROFILE_SUMMARY):
        if ":" in line and line.strip().startswith("-"):
            k, v = line.strip("- \n").split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256_16") != _kernel_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


def _operating_point(stream=None):
    """(rho_g*, rho_l*, p*): the method's own coexistence at the workload's EOS,
    tau, k and kappa, from a relaxed flat slab on the GPU (FP64)."""
    import paper_2103_08301_gb300 as lbm
    eos = lbm.lbm_eos(1.0, 4.0, 1.0, PHYS["T_over_Tc"], PHYS["k"], PHYS["kappa"])
    c = lbm.lbm_relaxed_coexistence(eos, PHYS["tau"], None, 64, 192, 40000, stream=stream)
    return c["rho_g"], c["rho_l"], c["p_gas"]


def _oracle_operating_point():
    """The same operating point from the oracle's own relaxed slab (for the CPU legs)."""
    import oracle
    import synth
    s = oracle.Setup(nx=2, ny=192, T_over_Tc=PHYS["T_over_Tc"], k=PHYS["k"], kappa=PHYS["kappa"], tau=PHYS["tau"])
    g, l, _ = s.coexistence()
    f, _ = oracle.run(s, oracle.init(s, synth.slab_rho0(2, 192, 48, 144, l, g, width=4)), 40000)
    r = oracle.fields(s, f)["rho"][:, 0]
    return r[0], r[96], PHYS["k"] ** 2 * oracle.cs_p0(s.a, s.b, s.R, s.T, r[0])


def _rho0(op, nx=NX, ny=NY, plug_x=PLUG_X, plug_len=PLUG_LEN, film=FILM):
    import paper_2103_08301_gb300 as lbm
    g, l, _ = op
    return lbm.lbm_airway_rho0(nx, ny, film, plug_x, plug_len, l, g)


def _lattice_kw(precision, op):
    return dict(walls=True, bc_x=True, precision=precision, T_over_Tc=PHYS["T_over_Tc"], k=PHYS["k"],
                kappa=PHYS["kappa"], tau=PHYS["tau"], dp=PHYS["dp"], p_ref=op[2] - 0.5 * PHYS["dp"])


def _timed_steps(lat, stream, steps):
    """Milliseconds per step of lat over `steps` steps (CUDA events on its stream)."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat.step(5)
    torch.cuda.synchronize()
    a.record(stream)
    lat.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def _extras(stream, op):
    """Throughput of the other scope rows on the same GPU: the FP64 step and
    the Peng-Robinson + MRT step on the 16384 x 2048 channel, the adjoint
    (forward with checkpoints, backward) on the 512 x 128 airway over 2000 FP64
    steps, the general-geometry step, the other single-lattice workloads and
    the rupture trend sweep. Not part of the headline value."""
    import numpy as np

    import paper_2103_08301_gb300 as lbm
    out = {}
    nodes = NX * NY
    rho0 = _rho0(op)
    with lbm.Lattice(NX, NY, rho0, stream=stream, **_lattice_kw(64, op)) as lat:
        ms = _timed_steps(lat, stream, 100)
    out["fp64_step"] = {"ms_per_step": ms, "mlups": nodes / ms / 1e3,
                        "hbm_gbs": BYTES_PER_NODE[64] * nodes / ms / 1e6}
    # in-place streaming (one population array plus a density plane): 40 B per
    # node stored, 116 B per node and step moved (36 + 4 by the density pass,
    # 36 + 36 + 4 by the step)
    peak, _ = _hbm_peak()
    with lbm.Lattice(NX, NY, rho0, stream=stream, inplace=True, **_lattice_kw(32, op)) as lat:
        ms = _timed_steps(lat, stream, 200)
        nan = lat.diag()["nan_detected"]
    out["inplace_fp32_step"] = {"ms_per_step": ms, "mlups": nodes / ms / 1e3, "nan": bool(nan),
                                "storage_bytes_per_node": 40, "traffic_bytes_per_node": 116,
                                "hbm_gbs": 116 * nodes / ms / 1e6, "frac_of_measured": 116 * nodes / ms / 1e6 / peak,
                                "workload": "same channel, FP32, lbm_init_inplace (AA pattern)"}
    pr = dict(walls=True, bc_x=True, precision=32, eos="pr", a=2 / 49, b=2 / 21, T_over_Tc=0.8, k=1.0,
              kappa=0.01, tau=1.2, dp=1e-4, collision="mrt", s_e=1.64, s_eps=1.54, s_q=1 / 1.2, s_j=1 / 1.2)
    _, g, l, _ = lbm.lbm_coexistence(lbm.lbm_eos(2 / 49, 2 / 21, 1.0, 0.8, 1.0, 0.01, lbm.LBM_EOS_PR, 0.344))
    rho_pr = lbm.lbm_airway_rho0(NX, NY, 64, 4096, 1024, l, g)
    with lbm.Lattice(NX, NY, rho_pr, stream=stream, **pr) as lat:
        ms = _timed_steps(lat, stream, 100)
        nan = lat.diag()["nan_detected"]
    out["pr_mrt_fp32_step"] = {"ms_per_step": ms, "mlups": nodes / ms / 1e3, "nan": bool(nan),
                               "workload": "same channel, Peng-Robinson water 0.8 Tc, MRT, tau 1.2"}
    from paper_2103_08301_gb300 import adjoint as adjm
    nx, ny, steps = 512, 128, 2000
    _, g, l, _ = lbm.lbm_coexistence(lbm.lbm_eos(1.0, 4.0, 1.0, 0.85, 1.0, 0.5))
    r0 = lbm.lbm_airway_rho0(nx, ny, 6.0, 128, 48.0, l, g, 4.0, 1e-3, 1)
    for key, prec, rev in (("adjoint", 32, 64), ("adjoint_fp32_reverse", 32, 32), ("adjoint_fp64_forward", 64, 64)):
        with adjm.Adjoint(nx, ny, steps, walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5, block_steps=100,
                          precision=prec, reverse_precision=rev) as adj:
            t0 = time.perf_counter()
            adj.forward(r0, dp=1e-3)
            t1 = time.perf_counter()
            adj.backward(1.0, 1.0)
            t2 = time.perf_counter()
        out[key] = {"workload": f"512x128 airway, 2000 steps, FP{prec} forward with checkpoints every 100, "
                                f"FP{rev} reverse",
                    "forward_s": t1 - t0, "backward_s": t2 - t1,
                    "reverse_mlups": nx * ny * steps / (t2 - t1) / 1e6}
    # the same channel with a wall mask (a constriction on both walls every
    # 2048 columns): the general-geometry kernels
    mask = np.zeros((NY, NX), np.uint8)
    for x0 in range(1024, NX - 512, 2048):
        mask[1:NY // 4, x0:x0 + 64] = 1
        mask[NY - NY // 4:NY - 1, x0:x0 + 64] = 1
    with lbm.Lattice(NX, NY, rho0, stream=stream, mask=mask, **_lattice_kw(32, op)) as lat:
        ms = _timed_steps(lat, stream, 50)
        nan = lat.diag()["nan_detected"]
    out["masked_fp32_step"] = {"ms_per_step": ms, "mlups": nodes / ms / 1e3, "nan": bool(nan),
                               "hbm_gbs_at_72B": 72 * nodes / ms / 1e6,
                               "workload": "same channel, constrictions on both walls every 2048 columns "
                                           "(general-geometry kernels)"}
    # past 2^31 population slots: the step with 64-bit population offsets
    # (16384 x 14600 periodic two-phase slabs, 2 x 8.6 GB of FP32 populations)
    bx, by = 16384, 14600
    eos8 = lbm.lbm_eos(1.0, 4.0, 1.0, 0.8, 1.0, 0.5)
    _, g8, l8, _ = lbm.lbm_coexistence(eos8)
    xs = np.arange(bx)
    row = g8 + (l8 - g8) * 0.5 * (1 - np.tanh(2 * (np.abs((xs % 512) - 256.0) - 100.0) / 4.0))
    big_rho = np.broadcast_to(row, (by, bx))
    with lbm.Lattice(bx, by, big_rho, stream=stream, precision=32, T_over_Tc=0.8, kappa=0.5) as lat:
        del big_rho
        ms = _timed_steps(lat, stream, 20)
        nan = lat.diag()["nan_detected"]
    out["fp32_step_64bit_offsets"] = {"ms_per_step": ms, "mlups": bx * by / ms / 1e3, "nan": bool(nan),
                                      "hbm_gbs_at_72B": 72 * bx * by / ms / 1e6,
                                      "workload": "16384x14600 periodic, liquid slabs every 512 columns, "
                                                  "9 nx ny = 2.15e9 population slots (64-bit offsets)"}
    out["configs"] = _configs(stream, op)
    out["trends"] = _trends(stream, op)
    return out


def _trends(stream, op):
    """Plug rupture under the paper's body-force drive on its proportions
    (1500 x 202 lattice, R = 100, film 0.15 R, plug 1 R at x = 200), one
    parameter varied at a time (Sec. 3.3, Figs. 10-12)."""
    from paper_2103_08301_gb300 import trends
    base = dict(nx=1500, ny=202, film=15, plug_len=100, force=5e-7)
    rows = trends.sweep(base, {"force": [4e-7, 5e-7, 6e-7, 8e-7], "plug_len": [60, 80, 120], "film": [10, 20]},
                        coex=op, max_steps=60000, every=250, window=1500, settle=1000, plug_x=200, stream=stream)
    return {"base": base, "rows": [{"vary": n, "value": v, "rupture_step": r["rupture_step"],
                                    "dP_wall": r["dP_wall"], "dtau_wall": r["dtau_wall"],
                                    "droplet_mass": r["droplet_mass"], "nan": r["nan"]} for n, v, r in rows]}


def _oracle_mlups(s, f, budget_s):
    """Oracle MLUPS on as many steps of state f as fit in about budget_s seconds."""
    import oracle
    t0 = time.perf_counter()
    f, _ = oracle.run(s, f, 1)
    one = time.perf_counter() - t0
    steps = max(1, int(budget_s / max(one, 1e-6)))
    t0 = time.perf_counter()
    oracle.run(s, f, steps)
    dt = time.perf_counter() - t0
    return s.nx * s.ny * steps / dt / 1e6, steps


def _configs(stream, op, budget_s=2.0):
    """The two single-lattice workloads not timed above, on the GPU and with the
    oracle on all host cores and on one core (bounded samples of the same
    state): the 128 x 128 periodic droplet (FP64, 10000 steps) and the
    2048 x 256 airway channel (FP32, its full 100000 steps at the method's
    coexistence, with the plug's state at the end; its 38 MB state sits in L2,
    so its GB/s is algorithmic traffic, not DRAM), plus that channel under the
    paper's body-force drive (G = dp / nx, ends at p*) until its plug ruptures."""
    import numpy as np

    import oracle
    import synth
    import paper_2103_08301_gb300 as lbm
    from paper_2103_08301_gb300 import trends
    peak, _ = _hbm_peak()
    out = {}
    rg, rl, ps = op
    org, orl, ops = _oracle_operating_point()  # the oracle samples take the oracle's own
    dp = 1e-3
    cases = [
        ("droplet_128x128_fp64", 128, 128, 64, 10000,
         dict(walls=False, bc_x=False, T_over_Tc=0.8, k=1.0, kappa=0.5, tau=1.0)),
        ("airway_2048x256_fp32", 2048, 256, 32, 100000,
         dict(walls=True, bc_x=True, T_over_Tc=0.85, k=1.0, kappa=0.5, tau=1.0, dp=dp, p_ref=ps - 0.5 * dp)),
    ]
    for name, nx, ny, prec, steps, kw in cases:
        s = oracle.Setup(nx=nx, ny=ny, **kw)
        g, l, _ = s.coexistence()
        if name.startswith("droplet"):
            rho0 = o_rho0 = synth.disk_rho0(nx, ny, 30, l, g, noise=1e-3, seed=1)
        else:
            rho0 = synth.airway_rho0(nx, ny, 8.0, 512.0, 128.0, rl, rg)
            o_rho0 = synth.airway_rho0(nx, ny, 8.0, 512.0, 128.0, orl, org)
            s = oracle.Setup(nx=nx, ny=ny, **dict(kw, p_ref=ops - 0.5 * dp))
        plug = None
        with lbm.Lattice(nx, ny, rho0, precision=prec, stream=stream, **kw) as lat:
            ms = _timed_steps(lat, stream, steps)
            if name.startswith("airway"):
                st = lbm.lbm_plug_analysis(lat.fields()["rho"].astype(np.float64), 0.5 * (rg + rl))
                plug = {"after_steps": steps + 5, "x_rear": st["x_rear"], "x_front": st["x_front"],
                        "intact": st["intact"], "n_droplets": st["n_droplets"],
                        "nan": bool(lat.diag()["nan_detected"])}
        mlups = nx * ny / ms / 1e3
        gbs = BYTES_PER_NODE[prec] * nx * ny / ms / 1e6
        f0 = oracle.init(s, o_rho0)
        ncores = oracle.num_threads()
        o_all, n_all = _oracle_mlups(s, f0, budget_s)
        oracle.set_num_threads(1)
        try:
            o_one, n_one = _oracle_mlups(s, f0, budget_s)
        finally:
            oracle.set_num_threads(ncores)
        out[name] = {"gpu_mlups": mlups, "gpu_gbs": gbs, "roofline_frac_of_measured": gbs / peak,
                     "gpu_steps": steps, "oracle_mlups": o_all, "oracle_cores": ncores,
                     "oracle_mlups_1core": o_one,
                     "oracle_sample": f"{n_all} steps on {ncores} cores, {n_one} steps on 1 core"}
        if plug is not None:
            out[name]["plug_at_end"] = plug
    r = trends.rupture_run(2048, 256, 8.0, 128.0, dp / 2048, plug_x=512, coex=op, max_steps=100000, every=500,
                           window=1500, settle=1000, stream=stream)
    out["airway_2048x256_body_force_rupture"] = {
        "force": dp / 2048, "rupture_step": r["rupture_step"], "steps": r["steps"], "dP_wall": r["dP_wall"],
        "dtau_wall": r["dtau_wall"], "droplet_mass": r["droplet_mass"], "nan": r["nan"]}
    return out


def _cpu_baseline(budget_s=15.0):
    """The oracle, as it stands, on a bounded sample of the workload: a window of
    the same channel (full 2048-row height, 1024 columns with the plug inside),
    timed for as many steps as fit in about budget_s seconds."""
    import oracle
    import synth
    nx, ny = 1024, NY
    rg, rl, ps = _oracle_operating_point()
    s = oracle.Setup(nx=nx, ny=ny, walls=True, bc_x=True, T_over_Tc=PHYS["T_over_Tc"], k=PHYS["k"],
                     kappa=PHYS["kappa"], tau=PHYS["tau"], dp=PHYS["dp"], p_ref=ps - 0.5 * PHYS["dp"])
    f = oracle.init(s, synth.airway_rho0(nx, ny, FILM, 256.0, 256.0, rl, rg))
    t0 = time.perf_counter()
    f, _ = oracle.run(s, f, 1)
    one = time.perf_counter() - t0
    steps = max(1, min(200, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    f, _ = oracle.run(s, f, steps)
    dt = time.perf_counter() - t0
    return {"value": nx * ny * steps / dt / 1e6, "unit": "MLUPS", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{steps} FP64 oracle steps of a 1024x2048 window of the same channel "
                      f"(walls, pressure columns, film 64, plug 256 long), {dt:.1f} s"}


def allreduce_max(value: float, dist=None, device="cpu") -> float:
    """Max over ranks of a per-rank time (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world: int, nodes: int, steps: int, t_max: float) -> float:
    """Weak scaling: every rank steps its own channel of `nodes` nodes."""
    return world * nodes * steps / t_max / 1e6


def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle timed on the host cores, each step a
    bounded sample of the workload (a window of the channel) so the whole run
    finishes within a few minutes."""
    if rank != 0:
        return
    import oracle
    import synth
    oracle.build()
    budget = 150.0
    ny = 256
    g, l, ps = _oracle_operating_point()
    p_ref = ps - 0.5 * PHYS["dp"]
    s_probe = oracle.Setup(nx=512, ny=ny, walls=True, bc_x=True, T_over_Tc=PHYS["T_over_Tc"], k=PHYS["k"],
                           kappa=PHYS["kappa"], tau=PHYS["tau"], dp=PHYS["dp"], p_ref=p_ref)
    f = oracle.init(s_probe, synth.airway_rho0(512, ny, 8.0, 128.0, 128.0, l, g))
    t0 = time.perf_counter()
    oracle.run(s_probe, f, 3)
    rate = 512 * ny * 3 / (time.perf_counter() - t0)  # node updates / s
    per_step = budget / max(1, args.steps + args.warmup)
    nx = int(max(64, min(NX, rate * per_step / ny)))
    s = oracle.Setup(nx=nx, ny=ny, walls=True, bc_x=True, T_over_Tc=PHYS["T_over_Tc"], k=PHYS["k"],
                     kappa=PHYS["kappa"], tau=PHYS["tau"], dp=PHYS["dp"], p_ref=p_ref)
    f = oracle.init(s, synth.airway_rho0(nx, ny, 8.0, nx / 4, nx / 8, l, g))
    f, _ = oracle.run(s, f, args.warmup)
    t0 = time.perf_counter()
    f, _ = oracle.run(s, f, args.steps)
    dt = time.perf_counter() - t0
    val = nx * ny * args.steps / dt / 1e6
    sample = f"{args.steps} FP64 oracle steps of a {nx}x{ny} airway window (walls, pressure columns, film, plug)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_nx": nx, "sample_ny": ny},
        "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2103_08301_gb300 as lbm
    from paper_2103_08301_gb300 import build as lbm_build

    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(lbm.LIB_PATH):
        lbm_build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()

    precision = 32
    stream = torch.cuda.Stream()
    op = _operating_point(stream)
    rho0 = _rho0(op)
    lat = lbm.Lattice(NX, NY, rho0, stream=stream, **_lattice_kw(precision, op))
    info = lat.launch_info()
    lat.step(args.warmup)
    torch.cuda.synchronize()

    # timed region: K steps, one CUDA-event pair per kernel on the solver's stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            lat.step(1)
            ev[i][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    kern = [a.elapsed_time(b) / 1e3 for a, b in ev]
    t_max = allreduce_max(elapsed, dist, "cuda")
    d = lat.diag()
    lat.close()
    clocks = clk.summary()

    nodes = NX * NY
    value = whole_job_mlups(world, nodes, args.steps, t_max)
    kmean = sum(kern) / len(kern)
    bytes_per_launch = BYTES_PER_NODE[precision] * nodes
    achieved = bytes_per_launch / kmean / 1e9
    peak, peak_src = _hbm_peak()

    # end to end through the public API: host (pinned) rho0 -> lbm_init (H2D),
    # per step lbm_step + lbm_diag_async (D2H of the step's diagnostics into
    # pinned host memory), each step's result read on the host one step later
    # while the next step runs, final fields to host
    rho_pinned = torch.empty((NY, NX), dtype=torch.float64, pin_memory=True)
    rho_pinned.numpy()[:] = rho0
    out_rho = torch.empty((NY, NX), dtype=torch.float32, pin_memory=True)
    dbuf = [torch.empty(7, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    devs = [torch.cuda.Event() for _ in range(2)]
    mass_seen = 0.0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    lat2 = lbm.Lattice(NX, NY, rho_pinned.numpy(), stream=stream, **_lattice_kw(precision, op))
    for k in range(args.steps):
        lat2.step(1)
        lat2.diag_async(dbuf[k & 1])
        devs[k & 1].record(stream)
        if k:
            devs[(k - 1) & 1].synchronize()
            mass_seen = float(dbuf[(k - 1) & 1][0])  # the host read of step k-1's result
    devs[(args.steps - 1) & 1].synchronize()
    mass_seen = float(dbuf[(args.steps - 1) & 1][0])
    lat2.fields_into(rho=out_rho.numpy())
    lat2.close()
    e2e_t = time.perf_counter() - t0
    assert mass_seen > 0
    e2e_val = whole_job_mlups(world, nodes, args.steps, allreduce_max(e2e_t, dist, "cuda"))

    sweep = None
    if world == 1 and not args.no_sweep:
        from paper_2103_08301_gb300 import sweep_bench
        sweep = sweep_bench.run(steps=200)
    elif not args.no_sweep:
        # the sweep's channels are independent problems: shard them over the
        # ranks, no collective on the data path
        from paper_2103_08301_gb300 import sweep_bench
        sweep = sweep_bench.run_sharded(rank, world, dist, steps=200)
    extras = _extras(stream, op) if (rank == 0 and world == 1 and not args.no_sweep) else None

    if rank == 0:
        cpu = _cpu_baseline() if world == 1 else None
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "precision": precision,
                       "operating_point": {"rho_g": op[0], "rho_l": op[1], "p_star": op[2],
                                           "p_ref": op[2] - 0.5 * PHYS["dp"]},
                       "l2": "state 2.4 GB > 129 MB L2 (no flush needed)",
                       "launch": info, "parallelism": f"{world} independent channel replicas"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_src,
                         "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
                         "traffic": _profiled_traffic(),
                         "algorithmic_bytes_per_launch": bytes_per_launch,
                         "kernel_ms_mean": kmean * 1e3,
                         "kernel_ms_min": min(kern) * 1e3},
            "clocks": clocks,
            "e2e": {"value": e2e_val, "unit": "MLUPS",
                    "h2d_bytes_per_step": NX * NY * 8 / args.steps,
                    "d2h_bytes_per_step": 7 * 8 + NX * NY * 4 / args.steps},
            "gpu_launches": args.steps,
            "cpu_baseline": cpu,
            "diag": {"mass": d["mass"], "wall_shear_sum": d["wall_shear_sum"], "nan": d["nan_detected"]},
            "batched_sweep": sweep,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-sweep", action="store_true", help="skip the batched-sweep comparison")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = _dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
