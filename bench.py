"""Throughput of the MD hot path on GB300: atom-steps/s of the mixed-precision
path under the learned scheduler against the plain fp64 path under the
pair-count partition, on the porous Lennard-Jones system.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints ONE JSON line on rank 0.  A step is one velocity-Verlet step of the
whole path (gated rebuild: binning + list; forces; kicks and drift) through
md_step.  `value` is device-timed (CUDA events on the library's stream,
inputs resident in HBM); `e2e` times the same steps through the C ABI from
pinned host buffers (upload, md_set_state, md_step, md_get_state, download).
With N > 1 each rank advances its own replica (no exchange: weak scaling).
`--impl reference` times the CPU oracle instead, on a bounded sample.
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1611_00075_gb300 import inputs  # noqa: E402

FP32_LANES_PER_SM = 128  # fp32 FMA lanes per Blackwell SM
METRIC = "atom-steps/s at 1 GB300 (mixed+learned vs plain FP64) at stated force error"
POROUS_DESC = ("porous Lennard-Jones solid: 160^3 fcc cells = 16,384,000 sites at rho*=0.8442, "
               "spherical voids r~U(3,15) until >=40% removed (9,828,959 atoms), T*=0.3, "
               "rc=2.5, skin=0.3, dt=0.005, half-skin rebuilds")

# DRAM bytes (read + write) per atom of one force launch, from an ncu capture
# of a smaller porous case (profiles/); the figure is used only while the
# kernel sources still hash to the captured version.
FORCE_SOURCES = ("paper_1611_00075_gb300/csrc/k_lj.cu", "paper_1611_00075_gb300/csrc/k_common.cuh",
                 "paper_1611_00075_gb300/csrc/md_internal.cuh",
                 "paper_1611_00075_gb300/csrc/k_pair.cuh")
PROFILED_TRAFFIC = {
    # kernel: (sources sha1[:16], DRAM bytes per atom, capture)
    "lj_mixed_persist_paired": ("766f90ca9261abed", 365.8,
                                "ncu --set full, porous 80^3 cells (1,223,941 atoms) equilibrated "
                                "as the bench's input, two atoms per thread, one FM_FUSED_FULL "
                                "launch of the timed range"),
    "lj_mixed_persist": ("9e866177b4ed5d5f", 485.0,
                         "ncu --set full, porous 80^3 cells (1,223,941 atoms) equilibrated as the "
                         "bench's input, per-atom lists, one FM_FUSED_FULL launch of the timed "
                         "range"),
}


def sources_sha1() -> str:
    import hashlib
    h = hashlib.sha1()
    for f in FORCE_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    return parse_args(None)


def parse_args(argv):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="porous",
                    choices=["porous", "fcc", "sc", "eam", "alloy", "layer", "ensemble"])
    ap.add_argument("--compare-steps", type=int, default=100,
                    help="steps timed for each other scheduler (0 = skip the comparison)")
    ap.add_argument("--scheduler", default="mlp",
                    choices=["grid", "paircount", "mlp", "dynamic"])
    ap.add_argument("--fp64-steps", type=int, default=50,
                    help="steps timed for the plain fp64 comparison (slow path)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--nc", type=int, default=0,
                    help="fcc cells per side (0 = the workload's own size; smaller for profiling)")
    ap.add_argument("--force-variant", default="auto", choices=["auto", "paired", "full"],
                    help="force layout of the timed steps: two atoms per thread (union "
                         "lists), one atom per thread (per-atom lists), or auto: the "
                         "measured faster one for the workload's potential (two atoms per "
                         "thread for Lennard-Jones and Sutton-Chen, per-atom lists for the "
                         "embedded-atom potential)")
    ap.add_argument("--no-equilibrate", dest="equilibrate", action="store_false",
                    help="porous: time from the generated state instead of the equilibrated one")
    return ap.parse_args(argv)


def rank_barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def rank_max(x: float, world: int, device=None) -> float:
    """The largest value over all ranks (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(atoms_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Whole-job atom-steps/s: every rank advances its own replica (weak
    scaling), timed by the slowest rank."""
    return atoms_per_rank * steps * world / (ms_max * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_workload(name: str, nc: int = 0):
    if name == "ensemble":
        reps = inputs.lj_ensemble(count=nc or 64)
        n = sum(r.n for r in reps)
        desc = ("batched ensemble: %d Lennard-Jones fcc replicas, sizes log-uniform 1,000-200,000 "
                "(%d atoms in all), rho* U(0.7,0.9), T* U(0.5,1.5), rc=2.5, skin=0.3, dt=0.005, "
                "one launch per phase over all replicas, steps replayed from CUDA graphs"
                % (len(reps), n))
        return reps, desc
    if name == "porous" and nc:
        s = inputs.lj_porous(nc=nc)
        return s, "porous Lennard-Jones solid, %d^3 fcc cells (profiling size), %d atoms" % (nc, s.n)
    if name == "porous":
        s = inputs.lj_porous()
        desc = POROUS_DESC
    elif name == "fcc":
        k = nc or 64
        s = inputs.lj_fcc(nc=k, T=1.2)
        desc = ("Lennard-Jones liquid %d^3 fcc cells = %d atoms melted from fcc at rho*=0.8442 "
                "(2,000 untimed mixed-precision steps, velocities rescaled every 50 steps to "
                "T*=2.4 for 1,000 steps, then to T*=1.2), T*=1.2, rc=2.5, skin=0.3, dt=0.005, "
                "half-skin rebuilds" % (k, s.n))
    elif name in ("alloy", "layer"):
        if name == "alloy":
            k = nc or 105
            s = inputs.lj_alloy(nc=k)
            what = "random alloy, 25 % Au-like (the paper's Alloy size)"
        else:
            k = nc or 99
            s = inputs.lj_layer(nc=k)
            what = "slabs of 9 fcc cells, alternately Cu-like and Au-like (near the Layer size)"
        desc = ("Cu-Au-like binary Lennard-Jones fcc %d^3 cells = %d atoms, %s; eps 1 / 1.12, "
                "sigma 1 / 1.128 (Lorentz-Berthelot), mass 1 / 3.10, a0=1.625, rc=2.5, skin=0.3, "
                "T*=0.063, dt=0.002" % (k, s.n, what))
    elif name == "eam":
        k = nc or 126
        s = inputs.eam_bcc(nc=k)
        desc = ("piecewise embedded-atom bcc metal (Fe126 size) %d^3 cells = %d atoms, a0=1, "
                "Phi: 7 truncated-cubic knots, psi: 1, F = -0.5 sqrt(rho), rc=1.8, skin=0.15, "
                "T*=0.018, dt=0.002" % (k, s.n))
    else:
        k = nc or 128
        s = inputs.sc_fcc(nc=k)
        desc = ("Sutton-Chen fcc %d^3 cells = %d atoms, a0=a=1, c=39.432, n=9, m=6, "
                "rc=2a, skin=0.2, T*=2.088, dt=7.6e-4" % (k, s.n))
    return s, desc


def make_workload_desc(args):
    """The GPU arm's workload description, without generating its atoms."""
    if args.workload == "porous" and not args.nc:
        return None, POROUS_DESC
    return make_workload(args.workload, args.nc)


def md_kwargs(s):
    p = dict(s.params)
    kw = dict(eps=p.get("eps", 1.0), sigma=p.get("sigma", 1.0), rc=p["rc"], skin=p["skin"],
              dt=p["dt"], mass=p["mass"], potential=p["potential"])
    if p["potential"] == "sc":
        kw.update(c=p["c"], n_exp=p["n_exp"], m_exp=p["m_exp"])
    if p["potential"] == "eam":
        kw.update(eam={k: p[k] for k in ("phi_r", "phi_a", "psi_r", "psi_a", "F_sqrt",
                                         "F_quad")})
        del kw["eps"], kw["sigma"]
    if "types" in p:
        kw.update(species=(p["types"], p["t_eps"], p["t_sigma"], p["t_mass"]))
    return kw


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        return rows

    @staticmethod
    def summarize(rows):
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows
                                   if r[3].replace(".", "").isdigit()) if rows else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ GPU arm

def run_gpu(args, rank, world, local):
    import torch
    from paper_1611_00075_gb300 import md

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    md.lib()
    stream = torch.cuda.Stream(device=dev)
    s, desc = make_workload(args.workload, args.nc)
    ensemble = args.workload == "ensemble"
    if ensemble:
        reps = s
        s = inputs.System(name="ensemble", pos=np.concatenate([r.pos for r in reps]),
                          vel=np.concatenate([r.vel for r in reps]), box=reps[0].box,
                          params=reps[0].params)
        if args.scheduler not in ("grid", "dynamic"):
            args.scheduler = "grid"  # measured faster than the dynamic queue for batches
        args.fp64_steps = 0  # batches run the mixed path; per-replica fp64 is not the comparison
    kw = md_kwargs(s)
    if (kw["potential"] != "lj" or "species" in kw) and args.scheduler != "grid":
        args.scheduler = "grid"  # the persistent schedulers drive the Lennard-Jones kernel
    sched = {"grid": md.MD_SCHED_GRID, "paircount": md.MD_SCHED_PAIRCOUNT,
             "mlp": md.MD_SCHED_MLP, "dynamic": md.MD_SCHED_DYNAMIC}[args.scheduler]
    # the two-atom layout serves every one-species potential (batches under
    # the hardware block scheduler); on the embedded-atom workload it was
    # measured slower, so auto keeps per-atom lists there
    two_atom_ok = (kw["potential"] in ("lj", "sc", "eam") and
                   (not ensemble or args.scheduler == "grid"))
    paired = two_atom_ok and (args.force_variant == "paired" or
                              (args.force_variant == "auto" and kw["potential"] != "eam"))
    fv = md.MD_FORCE_PAIRED if paired else md.MD_FORCE_FULL
    kw["force_variant"] = fv

    def barrier():
        rank_barrier(world)

    def max_over_ranks(x: float) -> float:
        return rank_max(x, world, dev)

    def n_of(sysobj):
        return sysobj.n * world

    def timed(sysobj, nsteps, events=True, nvtx=None):
        # md_set_timing also zeroes the handle's launch counter
        md.md_set_timing(sysobj.h, events)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if nvtx:
            torch.cuda.nvtx.range_push(nvtx)  # lets a profiler select the timed launches
        e0.record(stream)
        md.md_step(sysobj.h, nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        if nvtx:
            torch.cuda.nvtx.range_pop()
        barrier()
        ms = e0.elapsed_time(e1)
        st = json.loads(md.md_stats(sysobj.h))
        md.md_set_timing(sysobj.h, False)
        return ms, st

    sampler = ClockSampler(local)
    with torch.cuda.stream(stream):
        if ensemble:
            mixed = md.Batch([(r.pos, r.vel, r.box) for r in reps], precision="mixed",
                             stream=stream, **kw)
        else:
            mixed = md.System(s.pos, s.vel, s.box, precision="mixed", stream=stream, **kw)
        sched_info = {}
        if args.workload == "fcc":
            # config 2 is a liquid melted from the crystal; the melted state is
            # the start of every leg below
            t0 = time.perf_counter()
            gpu_melt(md, mixed, kw["mass"], dev)
            p_m, v_m, _ = mixed.state()
            s = inputs.System(name=s.name + "_melted", pos=p_m.cpu().numpy(), vel=v_m.cpu().numpy(),
                              box=s.box, params=s.params)
            sched_info["melt"] = {"seconds": time.perf_counter() - t0, "steps": sum(
                k for _, k in inputs.MELT_SCHEDULE), "schedule": inputs.MELT_SCHEDULE}
        elif args.workload == "porous" and args.equilibrate:
            # the porous solid relaxes its surfaces and heats at first: every
            # leg below starts from it at its steady rebuild rate
            t0 = time.perf_counter()
            gpu_melt(md, mixed, kw["mass"], dev, inputs.POROUS_EQUIL_SCHEDULE)
            p_m, v_m, _ = mixed.state()
            s = inputs.System(name=s.name + "_equilibrated", pos=p_m.cpu().numpy(),
                              vel=v_m.cpu().numpy(), box=s.box, params=s.params)
            sched_info["equilibration"] = {
                "seconds": time.perf_counter() - t0,
                "steps": sum(k for _, k in inputs.POROUS_EQUIL_SCHEDULE),
                "schedule": inputs.POROUS_EQUIL_SCHEDULE,
                "rescale_every": inputs.MELT_RESCALE_EVERY}
        md.md_step(mixed.h, args.warmup)
        if ensemble:
            s0 = mixed.state()[:2]

            def batch_from_s0(code, variant):
                md.md_set_state(mixed.h, s0[0], s0[1])
                md.md_set_variant(mixed.h, variant, code)
                md.md_forces(mixed.h)
                torch.cuda.synchronize()

            if args.compare_steps > 0:
                sched_info["per_replica_launches"] = per_replica(md, reps, kw, stream,
                                                                 args.compare_steps, args.warmup)
                # the batch from the same state under each scheduler it supports,
                # plain device time (graphs on)
                legs = [("grid", md.MD_SCHED_GRID, md.MD_FORCE_FULL),
                        ("dynamic", md.MD_SCHED_DYNAMIC, md.MD_FORCE_FULL),
                        ("paired_grid", md.MD_SCHED_GRID, md.MD_FORCE_PAIRED)]
                for name, code, variant in legs:
                    batch_from_s0(code, variant)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    md.md_step(mixed.h, args.compare_steps)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    sched_info["batched_graphs_" + name] = {
                        "atom_steps_per_s": mixed.n * args.compare_steps / (e0.elapsed_time(e1) * 1e-3),
                        "steps": args.compare_steps,
                        "layout": "two atoms per thread" if variant == md.MD_FORCE_PAIRED
                        else "per-atom lists"}
            batch_from_s0(sched, fv)
        elif kw["potential"] == "lj" and "species" not in kw:
            # the learned part first: per-cell clock64 timings of this state,
            # then the network trained on the GPU
            if args.scheduler == "mlp" or args.compare_steps > 0:
                md.md_set_variant(mixed.h, fv, md.MD_SCHED_DYNAMIC)
                t0 = time.perf_counter()
                nsamp = md.md_cost_model(mixed.h, md.MD_COST_SAMPLE)
                loss = md.md_cost_model(mixed.h, md.MD_COST_TRAIN)
                t1 = time.perf_counter()
                sched_info["mlp_training"] = {"samples": int(nsamp), "final_mse": loss,
                                              "sample_and_train_s": t1 - t0}
            # every scheduler and force variant runs from the same saved state
            # (a porous system warms up as its surfaces relax, so runs taken one
            # after another would see different work)
            s0 = mixed.state()[:2]

            def from_s0(force_variant, code):
                md.md_set_state(mixed.h, s0[0], s0[1])
                md.md_set_variant(mixed.h, force_variant, code)
                md.md_forces(mixed.h)  # forces ready: timed regions hold whole steps only
                torch.cuda.synchronize()

            if args.compare_steps > 0:
                for name, code in (("grid", md.MD_SCHED_GRID), ("paircount", md.MD_SCHED_PAIRCOUNT),
                                   ("dynamic", md.MD_SCHED_DYNAMIC), ("mlp", md.MD_SCHED_MLP)):
                    from_s0(fv, code)
                    msx, stx = timed(mixed, args.compare_steps)
                    sched_info[name] = {
                        "atom_steps_per_s": n_of(mixed) * args.compare_steps / (msx * 1e-3),
                        "force_ms_per_launch": stx["ms"]["force"] / max(1, stx["count"]["force"])}
                    if code != md.MD_SCHED_GRID:
                        sched_info[name]["cta_imbalance"] = md.md_cost_model(mixed.h, md.MD_COST_PROFILE)
                # the same static partitions with no dynamically claimed tail:
                # the cost estimate alone balances the CTAs
                for name, code in (("paircount", md.MD_SCHED_PAIRCOUNT), ("mlp", md.MD_SCHED_MLP)):
                    from_s0(fv, code)
                    md.md_set_schedule(mixed.h, 0, 0)
                    msx, stx = timed(mixed, args.compare_steps)
                    sched_info[name + "_static"] = {
                        "atom_steps_per_s": n_of(mixed) * args.compare_steps / (msx * 1e-3),
                        "force_ms_per_launch": stx["ms"]["force"] / max(1, stx["count"]["force"]),
                        "cta_imbalance": md.md_cost_model(mixed.h, md.MD_COST_PROFILE),
                        "note": "static ranges only (md_set_schedule tail_percent = 0)"}
                    md.md_set_schedule(mixed.h, 0, -1)  # the layout's default tail
                # the Newton's-third-law variants (half lists) against the full list
                variants = {}
                for name, code in (("full", md.MD_FORCE_FULL),
                                   ("paired", md.MD_FORCE_PAIRED),
                                   ("half_color", md.MD_FORCE_HALF_COLOR),
                                   ("half_atomic", md.MD_FORCE_HALF_ATOMIC),
                                   ("cluster_pairs", md.MD_FORCE_CLUSTER)):
                    from_s0(code, md.MD_SCHED_GRID)
                    msx, stx = timed(mixed, args.compare_steps)
                    variants[name] = {
                        "atom_steps_per_s": n_of(mixed) * args.compare_steps / (msx * 1e-3),
                        "force_ms_per_launch": stx["ms"]["force"] / max(1, stx["count"]["force"]),
                        "rebuild_ms_per_step": stx["ms"]["rebuild"] / args.compare_steps}
                    if code == md.MD_FORCE_CLUSTER:
                        variants[name]["cluster_pairs"] = stx["cluster_pairs"]
                        variants[name]["pair_slots_per_atom"] = 32.0 * stx["cluster_pairs"] / n_of(mixed)
                    if code == md.MD_FORCE_PAIRED:
                        variants[name]["slot_entries_per_atom"] = stx["slot_entries"] / n_of(mixed)
                    if code == md.MD_FORCE_FULL:
                        variants[name]["list_entries_per_atom"] = stx["list_entries"] / n_of(mixed)
                variants["note"] = "every layout under the hardware block scheduler"
                sched_info["force_variants"] = variants
                # the inner/outer split of Sec. 2.1 (virtual domains, boundary
                # positions exchanged on a second stream) against the fused pass
                split = {"fused": variants["full"]}
                for dd in ((2, 2, 2), (4, 4, 4)):
                    from_s0(md.MD_FORCE_FULL, md.MD_SCHED_GRID)
                    md.md_set_decomposition(mixed.h, *dd)
                    msx, stx = timed(mixed, args.compare_steps)
                    split["%dx%dx%d" % dd] = {
                        "atom_steps_per_s": n_of(mixed) * args.compare_steps / (msx * 1e-3),
                        "force_ms_per_launch": stx["ms"]["force"] / max(1, stx["count"]["force"])}
                    md.md_set_decomposition(mixed.h, 1, 1, 1)
                sched_info["inner_outer_split"] = split
            from_s0(fv, sched)
        else:
            md.md_set_variant(mixed.h, fv, sched)
        builds0 = json.loads(md.md_stats(mixed.h))["builds"]
        sampler.start()
        # batches of small replicas are launch-bound: their timed region replays
        # graphs, which per-launch events would disable
        ms, st = timed(mixed, args.steps, events=not ensemble, nvtx="timed")
        builds_timed = st["builds"] - builds0
        clock_rows = sampler.stop()
        launches_timed = st["launches"]
        if ensemble:
            # kernel durations from a separate run with per-launch events
            kb_steps = min(args.steps, 200)
            _, st = timed(mixed, kb_steps)
            sched_info["kernel_breakdown_steps"] = kb_steps
            st["launches"] = launches_timed
        ms = max_over_ranks(ms)
        ke, pe = md.md_energy(mixed.h)
        st_e = json.loads(md.md_stats(mixed.h))
        pos, vel, force = mixed.state()
        n = mixed.n
        value = job_throughput(n, args.steps, world, ms)

        # plain fp64 path, same workload, under the pair-count partition (the
        # persistent schedulers serve Lennard-Jones; Sutton-Chen runs a grid)
        fp64 = None
        if args.fp64_steps > 0:
            sched64 = "paircount" if (kw["potential"] == "lj" and "species" not in kw) else "grid"
            kw64 = dict(kw, force_variant=md.MD_FORCE_FULL)  # the plain method: per-atom lists
            plain = md.System(s.pos, s.vel, s.box, precision="fp64", stream=stream,
                              scheduler=md.MD_SCHED_PAIRCOUNT if sched64 == "paircount"
                              else md.MD_SCHED_GRID, **kw64)
            md.md_step(plain.h, min(args.warmup, 3))
            ms64, st64 = timed(plain, args.fp64_steps)
            ms64 = max_over_ranks(ms64)
            fp64 = {"value": n * args.fp64_steps * world / (ms64 * 1e-3), "steps": args.fp64_steps,
                    "scheduler": sched64,
                    "ms_per_step": ms64 / args.fp64_steps,
                    "force_ms_per_launch": st64["ms"]["force"] / max(1, st64["count"]["force"])}
            plain.close()

        # end to end through the C ABI with pinned host buffers
        e2e = None
        if not args.no_e2e:
            hp = torch.from_numpy(np.ascontiguousarray(s.pos)).pin_memory()
            hv = torch.from_numpy(np.ascontiguousarray(s.vel)).pin_memory()
            op = torch.empty_like(hp).pin_memory()
            ov = torch.empty_like(hv).pin_memory()
            dp = torch.empty(hp.shape, dtype=torch.float64, device=dev)
            dv = torch.empty_like(dp)
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            dp.copy_(hp, non_blocking=True)
            dv.copy_(hv, non_blocking=True)
            md.md_set_state(mixed.h, dp, dv)
            md.md_step(mixed.h, args.steps)
            md.md_get_state(mixed.h, dp, dv, None)
            op.copy_(dp, non_blocking=True)
            ov.copy_(dv, non_blocking=True)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            barrier()
            te = max_over_ranks(t1 - t0)
            nbytes = hp.numel() * 8 + hv.numel() * 8
            e2e = {"value": n * args.steps * world / te, "unit": "atom-steps/s",
                   "h2d_bytes_per_step": nbytes / args.steps,
                   "d2h_bytes_per_step": nbytes / args.steps,
                   "note": "per run: upload pos+vel, md_set_state, md_step(K), md_get_state, "
                           "download pos+vel; bytes amortised over K steps"}
        # the force check of the CPU leg runs at generator positions (the start
        # perturbed by a seeded Gaussian) loaded into the running system: the
        # oracle never sees positions the GPU produced
        if ensemble:
            pos_chk = np.concatenate([np.mod(r.pos + 0.05 * inputs.gaussian(
                inputs.SEED_BASE + 98 + k, r.pos.size).reshape(-1, 3), r.box)
                for k, r in enumerate(reps)])
        else:
            pos_chk = np.mod(s.pos + 0.03 * inputs.gaussian(inputs.SEED_BASE + 98, s.pos.size)
                             .reshape(-1, 3), s.box)
        md.md_set_state(mixed.h, torch.as_tensor(pos_chk, device=dev), None)
        md.md_forces(mixed.h)
        force = mixed.state()[2]
        pos = pos_chk
        mixed.close()

    peaks, peak_src = measured_peaks()
    # roofline of the force kernel (dominant launch): algorithmic work per launch
    n_force = max(1, st["count"]["force"])
    t_force = st["ms"]["force"] / n_force * 1e-3
    entries = st_e["list_entries"]
    pairs = st_e["pairs_cut"]
    if kw["potential"] == "lj" and kw.get("force_variant") == md.MD_FORCE_PAIRED:
        # two atoms per thread: 12 flops per evaluated (atom, entry) and 14 per
        # pair inside r_c; 168 B of state per atom, 8 B per slot (its first
        # atom and list length) and 4 B per union-list entry
        entries = st_e["slot_entries"]
        flops = 12.0 * 2 * entries + 14.0 * pairs
        bytes_ = 168.0 * n + 8.0 * st_e["slots"] + 4.0 * entries
    elif kw["potential"] == "lj":
        flops = 12.0 * entries + 14.0 * pairs
        bytes_ = 168.0 * n + 4.0 * entries
    elif kw["potential"] == "eam":
        # both passes: the distance test per entry; per in-cutoff pair r (2)
        # and, per knot, max, square, cube and multiply-adds (5 for rho; 6
        # for value and derivative in the force pass) plus the force (7)
        nphi, npsi = len(s.params["phi_r"]), len(s.params["psi_r"])
        flops = 2 * (12.0 * entries) + pairs * (2 + 5 * npsi) + pairs * (2 + 6 * (nphi + npsi) + 7)
        bytes_ = 2 * 4.0 * entries + 250.0 * n
        if kw.get("force_variant") == md.MD_FORCE_PAIRED:
            # over two-atom slots: each union entry tested against both atoms
            # in both passes, the union list and 8 B per slot read by each
            entries = st_e["slot_entries"]
            flops = 2 * (12.0 * 2 * entries) + pairs * (2 + 5 * npsi) + \
                pairs * (2 + 6 * (nphi + npsi) + 7)
            bytes_ = 2 * (4.0 * entries + 8.0 * st_e["slots"]) + 250.0 * n
    elif kw.get("force_variant") == md.MD_FORCE_PAIRED:
        # Sutton-Chen over two-atom slots: both passes test each union entry
        # against both atoms (12 flops each) and read the union list, the
        # slot's first atom and its length
        entries = st_e["slot_entries"]
        flops = 2 * (12.0 * 2 * entries) + 10.0 * pairs + 26.0 * pairs
        bytes_ = 2 * (4.0 * entries + 8.0 * st_e["slots"]) + 250.0 * n
    else:
        flops = 2 * (12.0 * entries) + 10.0 * pairs + 26.0 * pairs
        bytes_ = 2 * 4.0 * entries + 250.0 * n
    traffic, traffic_note = None, "no capture of this kernel version"
    kname = (("lj_mixed_persist_paired" if paired else "lj_mixed_persist")
             if (kw["potential"] == "lj" and args.scheduler != "grid" and not ensemble) else None)
    if kname in PROFILED_TRAFFIC and PROFILED_TRAFFIC[kname][0] == sources_sha1():
        traffic = PROFILED_TRAFFIC[kname][1] * n
        traffic_note = PROFILED_TRAFFIC[kname][2] + ", scaled by atoms"
    clk = ClockSampler.summarize(clock_rows)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = torch.cuda.get_device_properties(dev).multi_processor_count * \
        FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    hbm_peak = float(peaks["hbm_gbs"])
    ach_flops = flops / t_force / 1e12
    ach_gbs = bytes_ / t_force / 1e9
    ai = flops / bytes_
    hbm_bound = ai * hbm_peak * 1e9 < fp32_peak * 1e12
    roof = {"bound": "hbm" if hbm_bound else "alu",
            "achieved": ach_gbs if hbm_bound else ach_flops,
            "peak": hbm_peak if hbm_bound else fp32_peak,
            "unit": "GB/s" if hbm_bound else "TFLOP/s",
            "frac": (ach_gbs / hbm_peak) if hbm_bound else (ach_flops / fp32_peak),
            "traffic": traffic,
            "traffic_note": traffic_note,
            "kernel": (("lj_typed_pair_kernel<FM_FUSED_FULL>" if paired else
                        "lj_typed_kernel<FM_FUSED_FULL>") if "species" in kw else
                       ("lj_mixed_persist<FM_FUSED_FULL, two-atom slots> (%s)" if paired else
                        "lj_mixed_persist<FM_FUSED_FULL> (%s)") % args.scheduler
                       if args.scheduler != "grid" else
                       ("lj_pair_kernel<FM_FUSED_FULL>" if paired else
                        "lj_mixed_kernel<FM_FUSED_FULL>")) if kw["potential"] == "lj" else
                      (("eam_density_pair + eam_force_pair" if paired else
                        "eam_density_mixed + eam_force_mixed") if kw["potential"] == "eam" else
                       ("sc_density_pair + sc_force_pair" if paired else
                        "sc_density_mixed + sc_force_mixed")),
            "multi_box": ensemble,
            "peak_source": peak_src,
            "algorithmic_bytes_per_launch": bytes_, "algorithmic_flops_per_launch": flops,
            "launch_ms": t_force * 1e3,
            "fp32": {"achieved_tflops": ach_flops, "peak_tflops": fp32_peak,
                     "frac": ach_flops / fp32_peak,
                     "peak_note": "SMs x 128 fp32 lanes x 2 x max SM clock"}}
    force, box, n_chk = force.cpu().numpy(), s.box, n
    if ensemble:
        # the force check runs on the largest replica (its own box)
        k = int(np.argmax([r.n for r in reps]))
        a0 = sum(r.n for r in reps[:k])
        pos, force, box, n_chk = pos[a0:a0 + reps[k].n], force[a0:a0 + reps[k].n], reps[k].box, reps[k].n
    return dict(n=n, value=value, ms=ms, st=st, st_e=st_e, fp64=fp64, e2e=e2e, roof=roof, paired=paired,
                clk=clk, desc=desc, pos=pos, force=force, n_check=n_chk,
                box=box, params=s.params, ke=ke, pe=pe, builds_timed=builds_timed,
                sched_info=sched_info)


def start_state(info):
    """How the timed state was prepared (untimed), for the JSON line."""
    for key, what in (("melt", "melted"), ("equilibration", "equilibrated")):
        if key in info:
            stages = ", ".join("%d steps at T*=%g" % (k, T) for T, k in info[key]["schedule"])
            return ("%s on the GPU before timing (untimed): %s, velocities rescaled every %d steps"
                    % (what, stages, inputs.MELT_RESCALE_EVERY))
    return "as generated"


def gpu_melt(md, sysobj, mass, device, schedule=None):
    """Melts (or equilibrates) the system in place on the GPU, untimed input
    preparation: the schedule (inputs.MELT_SCHEDULE by default) with the
    velocities rescaled to each stage's temperature every
    inputs.MELT_RESCALE_EVERY steps and once at the end."""
    import torch
    every = inputs.MELT_RESCALE_EVERY
    schedule = schedule or inputs.MELT_SCHEDULE

    def rescale(T):
        v = sysobj.state()[1].cpu().numpy()
        v = torch.from_numpy(inputs.rescale_velocities(v, T, mass)).to(device)
        md.md_set_state(sysobj.h, None, v)

    for T, nsteps in schedule:
        for _ in range(nsteps // every):
            rescale(T)
            md.md_step(sysobj.h, every)
    rescale(schedule[-1][0])
    torch.cuda.synchronize()


def per_replica(md, reps, kw, stream, steps, warmup):
    """The same replicas as separate systems, each advanced by its own
    md_step calls (its own launches and graphs), one after the other."""
    import torch
    systems = [md.System(r.pos, r.vel, r.box, precision="mixed", stream=stream, **kw)
               for r in reps]
    for a in systems:
        md.md_step(a.h, warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for a in systems:
        md.md_step(a.h, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    n = sum(a.n for a in systems)
    for a in systems:
        a.close()
    return {"atom_steps_per_s": n * steps / (e0.elapsed_time(e1) * 1e-3), "steps": steps,
            "note": "each replica its own system: md_step per replica in turn, graphs on"}


# ------------------------------------------------------------------ CPU legs

def oracle_sample_system(args, orc):
    """Bounded sample of the workload for the CPU oracle: the same generator
    at a smaller size (porous: 72^3 fcc cells, same density and void radii)."""
    if args.workload == "porous":
        return inputs.lj_porous(nc=72), "porous LJ 72^3 fcc cells (same rho*, voids U(3,15), >=40%)"
    if args.workload == "fcc":
        s = inputs.lj_fcc(nc=16, T=1.2)
        p = s.params
        prm = orc.make_params(potential=orc.POT_LJ, rc=p["rc"], skin=p["skin"], dt=p["dt"],
                              mass=p["mass"])
        pos, vel = orc.melt(prm, s.pos, s.vel, s.box, inputs.MELT_SCHEDULE,
                            inputs.MELT_RESCALE_EVERY,
                            lambda v, T: inputs.rescale_velocities(v, T, p["mass"]))
        m = inputs.System("lj_melt_16", pos, vel, s.box, dict(p))
        return inputs.tile(m, 2), ("LJ liquid: 16^3 fcc cells melted by the oracle (same "
                                   "schedule), tiled 2 x 2 x 2")
    if args.workload == "ensemble":
        reps = inputs.lj_ensemble(count=args.nc or 64)
        k = max((r for r in range(len(reps)) if reps[r].n <= 150000), key=lambda r: reps[r].n)
        return reps[k], "ensemble replica %d (the largest with <= 150,000 atoms)" % k
    if args.workload == "eam":
        return inputs.eam_bcc(nc=40), "piecewise-EAM bcc 40^3 cells"
    if args.workload == "alloy":
        return inputs.lj_alloy(nc=40), "Cu-Au-like random alloy 40^3 fcc cells"
    if args.workload == "layer":
        return inputs.lj_layer(nc=36), "Cu-Au-like slabs 36^3 fcc cells"
    return inputs.sc_fcc(nc=48), "Sutton-Chen fcc 48^3 cells"


def oracle_params(orc, p: dict):
    if p["potential"] == "eam":
        t = orc.make_eam(p["phi_r"], p["phi_a"], p["psi_r"], p["psi_a"], p["F_sqrt"], p["F_quad"])
        return orc.make_params(potential=orc.POT_EAM, rc=p["rc"], skin=p["skin"], dt=p["dt"],
                               mass=p["mass"], eam=t)
    if p["potential"] == "lj" and "types" in p:
        return orc.make_params(potential=orc.POT_LJ, rc=p["rc"], skin=p["skin"], dt=p["dt"],
                               types=p["types"], t_eps=p["t_eps"], t_sigma=p["t_sigma"],
                               t_mass=p["t_mass"])
    if p["potential"] == "lj":
        return orc.make_params(potential=orc.POT_LJ, eps=p["eps"], sigma=p["sigma"], rc=p["rc"],
                               skin=p["skin"], dt=p["dt"], mass=p["mass"])
    return orc.make_params(potential=orc.POT_SC, eps=p["eps"], sigma=p["sigma"], c=p["c"],
                           n_exp=p["n_exp"], m_exp=p["m_exp"], rc=p["rc"], skin=p["skin"],
                           dt=p["dt"], mass=p["mass"])


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                name = line.split(":", 1)[1].strip()
                if name and not name.isdigit():
                    return name
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_baseline_leg(args, gpu=None, steps=None, repeats=5):
    """Times the CPU oracle (as it stands) on a bounded sample on all host
    cores -- `repeats` runs of `steps` steps after a list build, reported as
    the mean with the standard deviation over the runs (the paper's timing
    protocol, Sec. 3.3) -- and measures the GPU snapshot's force error
    against it."""
    import oracle as orc
    orc.build()
    cores = os.cpu_count() or 1
    orc.set_threads(cores)
    s, what = oracle_sample_system(args, orc)
    prm = oracle_params(orc, s.params)
    k = steps
    if k is None:
        # about 2.5 s per run (a dozen seconds of CPU work in all): the step
        # count from one force evaluation with its list build
        t0 = time.perf_counter()
        orc.forces_once(prm, s.pos, s.box)
        est = time.perf_counter() - t0
        k = int(min(200, max(10, round(2.5 / max(est, 1e-6)))))
    rates = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        orc.forces_once(prm, s.pos, s.box)
        t1 = time.perf_counter()
        orc.md_run(prm, s.pos, s.vel, s.box, k, want_energies=False)
        t2 = time.perf_counter()
        per_step = max(1e-9, ((t2 - t1) - (t1 - t0)) / k)  # the first list build excluded
        rates.append(s.n / per_step)
    out = {"value": statistics.mean(rates), "std": statistics.stdev(rates) if repeats > 1 else 0.0,
           "repeats": repeats, "unit": "atom-steps/s", "cores": cores, "cpu": cpu_model(),
           "kind": "oracle",
           "sample": "%s, %d atoms, %d runs of %d velocity-Verlet steps after a list build "
                     "(fp64 C oracle, OpenMP over atoms); mean and standard deviation over "
                     "the runs" % (what, s.n, repeats, k)}
    if gpu is not None:
        rng_idx = (inputs.splitmix64(inputs.SEED_BASE + 99, 4096) % gpu["n_check"]).astype(np.int64)
        idx = np.unique(rng_idx)
        fref, _ = orc.forces_sample(oracle_params(orc, gpu["params"]), gpu["pos"], gpu["box"], idx)
        f = gpu["force"][idx]
        err = np.linalg.norm(f - fref, axis=1)
        fn = np.linalg.norm(fref, axis=1)
        rms = math.sqrt(float(np.mean(fn * fn)))
        out["force_error"] = {"atoms": int(idx.size), "max_abs": float(err.max()),
                              "rms_abs": float(math.sqrt(np.mean(err * err))),
                              "max_rel_to_max(|f|,rms)": float(np.max(err / np.maximum(fn, rms))),
                              "rms_force": rms}
    return out


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, for the GPU arm's metric and
    workload: each step is a step of a bounded sample of that workload."""
    if rank != 0:
        return
    import oracle as orc
    orc.build()
    cores = os.cpu_count() or 1
    orc.set_threads(cores)
    s, what = oracle_sample_system(args, orc)
    prm = oracle_params(orc, s.params)
    out = orc.md_run(prm, s.pos, s.vel, s.box, args.warmup, want_energies=False)
    t0 = time.perf_counter()
    orc.forces_once(prm, out["pos"], s.box)
    t1 = time.perf_counter()
    orc.md_run(prm, out["pos"], out["vel"], s.box, args.steps, want_energies=False)
    t2 = time.perf_counter()
    # md_run starts with a list build that the GPU arm's timed steps do not
    # contain (its list exists before them): one list build + force pass out
    sec = max(1e-9, (t2 - t1) - (t1 - t0))
    value = s.n * args.steps / sec
    _, desc = make_workload_desc(args)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "atom-steps/s",
            "cpu": cpu_model(),
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc},
            "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": cores,
                             "cpu": cpu_model(), "kind": "oracle",
                             "sample": "%s, %d atoms, %d velocity-Verlet steps after the first "
                                       "list build (fp64 C oracle, OpenMP over atoms)"
                                       % (what, s.n, args.steps)},
            "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    g = run_gpu(args, rank, world, local)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baseline_leg(args, gpu=g)
    st = g["st"]
    line = {
        "metric": METRIC,
        "value": g["value"], "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": g["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 pair terms / f64 state",
        "data": "synthetic",
        "config": {"workload": g["desc"], "atoms": g["n"], "precision": "mixed",
                   "force_variant": ("two atoms per thread, union lists"
                                     if g["paired"] else "one atom per thread, per-atom lists"),
                   "scheduler": args.scheduler,
                   "l2": "inputs larger than L2 (%.1f GB resident state + list)"
                         % ((g["n"] * 300 + 4 * (g["st_e"]["slot_entries"] if g["paired"]
                                                  else g["st_e"]["list_entries"])) / 1e9),
                   "list_builds_in_timed_steps": g["builds_timed"],
                   "start_state": start_state(g["sched_info"])},
        "fp64_baseline": g["fp64"],
        "speedup_vs_fp64": (g["value"] / g["fp64"]["value"]) if g["fp64"] else None,
        "roofline": g["roof"],
        "clocks": g["clk"],
        "e2e": g["e2e"],
        "gpu_launches": st["launches"],
        "schedulers": g["sched_info"],
        "kernel_ms": {"rebuild": st["ms"]["rebuild"], "force": st["ms"]["force"],
                      "integrate": st["ms"]["integrate"], "counts": st["count"]},
        "energy": {"ke": g["ke"], "pe": g["pe"]},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
