"""The cluster-pair layout of the Lennard-Jones force pass (the clustering the
paper compares its SIMD scheme with, Sec. 4.1): forces and energies against
the oracle with the mixed-path bars, 100 steps of config 1 against the
oracle's trajectory, graph replay, the per-atom list it keeps for export, and
its argument checks."""
import math

import numpy as np
import pytest

from paper_1611_00075_gb300 import inputs

from cutoff_bounds import lj_straddle_bound

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def md():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_00075_gb300 import build
    build.build()
    from paper_1611_00075_gb300 import md as _md
    torch.cuda.set_device(0)
    _md.lib()
    return _md


def systems(name):
    if name == "fcc4000":
        s = inputs.lj_fcc(nc=10, T=0.72)
        amp, seed = 0.05, 991
    elif name == "porous":
        s = inputs.lj_porous(nc=14, fraction=0.4, rmin=2.0, rmax=5.0)
        amp, seed = 0.05, 992
    else:  # hot and disordered: cells of very different occupancy
        s = inputs.lj_fcc(nc=8, T=1.2)
        amp, seed = 0.12, 993
    g = inputs.gaussian(seed, s.pos.size).reshape(-1, 3)
    return s, np.mod(s.pos + amp * g, s.box)


def near_cutoff(pos, box, off, ids, rc, delta):
    rows = np.repeat(np.arange(len(pos)), np.diff(off))
    d = pos[ids] - pos[rows]
    d -= box * np.round(d / box)
    r = np.sqrt(np.sum(d * d, axis=1))
    bad = np.zeros(len(pos), bool)
    bad[rows[np.abs(r - rc) < delta]] = True
    return bad


@pytest.mark.parametrize("name", ["fcc4000", "porous", "disordered"])
def test_cluster_forces_and_energy_match_oracle(md, orc, name):
    s, pos = systems(name)
    off, ids = orc.neighbors_cells(pos, s.box, 2.8)
    U0, f0 = orc.lj_list(pos, s.box, off, ids)
    bad = near_cutoff(pos, s.box, off, ids, 2.5, 1e-5)
    with md.System(pos, s.vel, s.box, precision="mixed",
                   force_variant=md.MD_FORCE_CLUSTER) as sy:
        f = sy.state()[2].cpu().numpy()
        ke, pe = sy.energy()
        st = sy.stats()
        goff, gids = sy.neighbors()
    fn = np.linalg.norm(f0, axis=1)
    rms = math.sqrt(np.mean(fn * fn))
    err = np.linalg.norm(f - f0, axis=1)
    assert np.all((err <= 2e-4 * fn + 1e-5 * max(1.0, rms)) | bad)
    slack = lj_straddle_bound(orc, pos, s.box, off, ids, 2.5, 1e-5)
    assert abs(pe - U0) <= 2e-6 * abs(U0) + slack, (pe, U0)
    # the per-atom list is kept for export
    np.testing.assert_array_equal(goff.cpu().numpy(), off)
    np.testing.assert_array_equal(gids.cpu().numpy(), ids)
    assert st["cluster_pairs"] > 0
    print("%s: %d atoms, %d cluster pairs, %.1f pair slots per in-cutoff pair"
          % (name, s.n, st["cluster_pairs"], 32.0 * st["cluster_pairs"] / st["pairs_cut"]))


def test_cluster_steps_track_the_oracle(md, orc):
    """100 steps of config 1 on the cluster layout: total energy within 1e-6
    relative of the oracle's trajectory after every tenth step; on a side
    stream (graph replay) the run ends bit-equal to plain launches."""
    s = inputs.lj_fcc(nc=10, T=0.72)
    p = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    E0 = orc.md_run(p, s.pos, s.vel, s.box, 100)["energies"]
    states = []
    for stream in (None, torch.cuda.Stream()):
        ctx = torch.cuda.stream(stream if stream is not None else torch.cuda.default_stream())
        with ctx, md.System(s.pos, s.vel, s.box, precision="mixed", stream=stream,
                            force_variant=md.MD_FORCE_CLUSTER) as sy:
            es = [sy.energy()]
            for _ in range(10):
                sy.step(10)
                es.append(sy.energy())
            states.append(sy.state())
        es = np.array(es)
        rel = np.abs(es[:, 0] + es[:, 1] - E0[::10, 2]) / np.abs(E0[::10, 2])
        print("cluster pairs: max relative total-energy error %.3g" % rel.max())
        assert rel.max() < 1e-6, rel.max()
    for x, y in zip(states[0], states[1]):
        assert torch.equal(x, y)


def test_cluster_variant_switch_and_checks(md, orc):
    s, pos = systems("fcc4000")
    with md.System(pos, s.vel, s.box, precision="mixed") as sy:
        f_full = sy.state()[2].cpu().numpy()
        md.md_set_variant(sy.h, md.MD_FORCE_CLUSTER, md.MD_SCHED_GRID)
        md.md_forces(sy.h)
        f_cl = sy.state()[2].cpu().numpy()
        sy.step(20)
        with pytest.raises(md.MDError):
            md.md_set_variant(sy.h, md.MD_FORCE_CLUSTER, md.MD_SCHED_PAIRCOUNT)
        md.md_set_variant(sy.h, md.MD_FORCE_FULL, md.MD_SCHED_GRID)
        sy.step(5)
    assert np.max(np.abs(f_cl - f_full)) < 1e-4
    with pytest.raises(md.MDError):
        md.System(pos, s.vel, s.box, precision="fp64", force_variant=md.MD_FORCE_CLUSTER)
