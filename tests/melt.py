"""Liquid inputs melted from fcc by the oracle (test helper).

The schedule is inputs.MELT_SCHEDULE: velocity-Verlet steps of the oracle
(Sec. 3.3) in chunks of inputs.MELT_RESCALE_EVERY, with the velocities
rescaled to each stage's temperature before every chunk and once at the end.
Only the oracle runs the steps, so the melted state is an input both sides
receive, never an output of the CUDA path."""
import numpy as np

from paper_1611_00075_gb300 import inputs

_cache = {}


def oracle_melt(orc, nc):
    """An nc^3-cell LJ fcc crystal (rho* = 0.8442) melted and held at T* = 1.2.
    Returns an inputs.System."""
    if nc in _cache:
        return _cache[nc]
    s = inputs.lj_fcc(nc=nc, T=1.2)
    p = s.params
    prm = orc.make_params(potential=orc.POT_LJ, eps=p["eps"], sigma=p["sigma"], rc=p["rc"],
                          skin=p["skin"], dt=p["dt"], mass=p["mass"])
    pos, vel = orc.melt(prm, s.pos, s.vel, s.box, inputs.MELT_SCHEDULE,
                        inputs.MELT_RESCALE_EVERY,
                        lambda v, T: inputs.rescale_velocities(v, T, p["mass"]))
    m = inputs.System("lj_melt_%d" % nc, np.ascontiguousarray(pos), vel, s.box.copy(), dict(p))
    _cache[nc] = m
    return m


def lattice_msd(s_melt, nc):
    """Mean squared minimum-image displacement from the fcc sites the atoms
    started on (a crystal keeps it near the thermal amplitude; a liquid that
    diffused for 10 time units is far beyond)."""
    s0 = inputs.lj_fcc(nc=nc, T=1.2)
    d = s_melt.pos - s0.pos
    d -= s0.box * np.round(d / s0.box)
    return float(np.mean(np.sum(d * d, axis=1)))
