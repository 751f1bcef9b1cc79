"""Runs each kernel family of the library once, inside an NVTX range named
"k", so that a profiler can select exactly those launches:

    python -m paper_1611_00075_gb300.kernel_survey [part] [nc]

part is one of lj, half_atomic, half_color, cluster, paired, split, mlp,
persist, eam, typed, sc, chain (default: all).  The systems are about 1.2 M
atoms each, so their state and lists exceed the 129 MB L2:
- lj .. persist: porous Lennard-Jones, 80^3 fcc cells (1,223,941 atoms), one
  system that switches force variant and scheduler between parts;
- eam: bcc, 84^3 cells (1,185,408 atoms), the Fe-like piecewise table;
- typed: the Cu-Au-like random alloy, 66^3 fcc cells (1,149,984 atoms);
- sc: Sutton-Chen fcc, 66^3 cells (1,149,984 atoms);
- chain: the rebuild chain of the headline layout -- porous Lennard-Jones
  with two atoms per thread under the learned scheduler (cost model sampled
  and trained first), three host-driven rebuilds (md_build_neighbors: the
  binning with the pairing order, slot tables, union lists, scheduler
  inputs); nc fcc cells per side, 80 by default (160: the 9.8 M-atom
  benchmark system).
Each part runs a few steps first, so that the captured launches are warm.
"""
from __future__ import annotations

import sys

import torch

from . import inputs, md

PARTS = ("lj", "half_atomic", "half_color", "cluster", "paired", "split", "mlp", "persist",
         "eam", "typed", "sc", "chain")


def main(only: str = "all", nc: int = 80) -> None:
    if only != "all" and only not in PARTS:
        raise SystemExit("unknown part %r; one of %s" % (only, ", ".join(PARTS)))
    torch.cuda.set_device(0)
    md.lib()

    def run(name, fn):
        if only not in ("all", name):
            return
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("k")
        fn()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()

    def wanted(*names):
        return only == "all" or only in names

    if wanted("lj", "half_atomic", "half_color", "cluster", "paired", "split", "mlp", "persist"):
        s = inputs.lj_porous(nc=80)
        with md.System(s.pos, s.vel, s.box, precision="mixed") as m:
            md.md_step(m.h, 5)
            # three fused steps (one rebuild among them) and one list build
            run("lj", lambda: (md.md_step(m.h, 3), md.md_build_neighbors(m.h)))
            for name, code in (("half_atomic", md.MD_FORCE_HALF_ATOMIC),
                               ("half_color", md.MD_FORCE_HALF_COLOR),
                               ("cluster", md.MD_FORCE_CLUSTER),
                               ("paired", md.MD_FORCE_PAIRED)):
                md.md_set_variant(m.h, code, md.MD_SCHED_GRID)
                run(name, lambda: md.md_step(m.h, 2))
            md.md_set_variant(m.h, md.MD_FORCE_FULL, md.MD_SCHED_GRID)
            md.md_set_decomposition(m.h, 2, 2, 2)
            run("split", lambda: md.md_step(m.h, 2))
            md.md_set_decomposition(m.h, 1, 1, 1)
            md.md_set_variant(m.h, md.MD_FORCE_FULL, md.MD_SCHED_DYNAMIC)
            md.md_cost_model(m.h, md.MD_COST_SAMPLE)
            run("mlp", lambda: md.md_cost_model(m.h, md.MD_COST_TRAIN))
            md.md_set_variant(m.h, md.MD_FORCE_FULL, md.MD_SCHED_MLP)
            run("persist", lambda: md.md_step(m.h, 3))
    if wanted("eam"):
        e = inputs.eam_bcc(nc=84)
        p = e.params
        tab = {k: p[k] for k in ("phi_r", "phi_a", "psi_r", "psi_a", "F_sqrt", "F_quad")}
        with md.System(e.pos, e.vel, e.box, precision="mixed", eam=tab, rc=p["rc"],
                       skin=p["skin"], dt=p["dt"]) as m:
            md.md_step(m.h, 2)
            run("eam", lambda: md.md_step(m.h, 2))
    if wanted("typed"):
        a = inputs.lj_alloy(nc=66)
        p = a.params
        with md.System(a.pos, a.vel, a.box, precision="mixed",
                       species=(p["types"], p["t_eps"], p["t_sigma"], p["t_mass"]),
                       rc=p["rc"], skin=p["skin"], dt=p["dt"]) as m:
            md.md_step(m.h, 2)
            run("typed", lambda: md.md_step(m.h, 2))
    if wanted("sc"):
        c = inputs.sc_fcc(nc=66)
        p = c.params
        with md.System(c.pos, c.vel, c.box, potential="sc", precision="mixed", eps=p["eps"],
                       sigma=p["sigma"], c=p["c"], n_exp=p["n_exp"], m_exp=p["m_exp"],
                       rc=p["rc"], skin=p["skin"], dt=p["dt"]) as m:
            md.md_step(m.h, 2)
            run("sc", lambda: md.md_step(m.h, 2))
    if wanted("chain"):
        s = inputs.lj_porous(nc=nc)
        with md.System(s.pos, s.vel, s.box, precision="mixed", force_variant=md.MD_FORCE_PAIRED,
                       scheduler=md.MD_SCHED_MLP) as m:
            md.md_step(m.h, 20)
            md.md_cost_model(m.h, md.MD_COST_SAMPLE)
            md.md_cost_model(m.h, md.MD_COST_TRAIN)
            md.md_step(m.h, 5)
            run("chain", lambda: [md.md_build_neighbors(m.h) for _ in range(3)])
    print("kernel survey ok (%s)" % only)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "all",
         int(sys.argv[2]) if len(sys.argv) > 2 else 80)
