"""Parity at the full workload sizes, in the configuration bench.py times,
on sampled outputs the oracle computes one by one: list rows bit-exact,
forces within the mixed-path bar, for atoms drawn by a seeded sampler."""
import math

import numpy as np
import pytest

from paper_1611_00075_gb300 import inputs

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


def sample_ids(n, k, seed):
    return np.unique((inputs.splitmix64(seed, k) % n).astype(np.int64))


def check_rows(orc, md_sys, pos, box, r_list, idx):
    """GPU list rows of the sampled atoms equal the oracle's definition."""
    off, ids = md_sys.neighbors()
    off, ids = off.cpu().numpy(), ids.cpu().numpy()
    ooff, oids = orc.neighbors_sample(pos, box, r_list, idx)
    for k, i in enumerate(idx):
        np.testing.assert_array_equal(ids[off[i]:off[i + 1]], oids[ooff[k]:ooff[k + 1]])
    return ooff, oids


def check_forces(orc, prm, f, pos, box, idx, ooff, oids, rc, bar_rel, bar_abs):
    """Sampled forces within |df| <= bar_rel |f| + bar_abs max(1, rms f); atoms
    with a pair within 1e-5 of r_c are left out (rounding may move that pair
    across the cutoff)."""
    f0, _ = orc.forces_sample(prm, pos, box, idx)
    bad = np.zeros(idx.size, bool)
    for k, i in enumerate(idx):
        d = pos[oids[ooff[k]:ooff[k + 1]]] - pos[i]
        d -= box * np.round(d / box)
        bad[k] = np.any(np.abs(np.sqrt(np.sum(d * d, axis=1)) - rc) < 1e-5)
    fn = np.linalg.norm(f0, axis=1)
    rms = math.sqrt(np.mean(fn * fn))
    err = np.linalg.norm(f[idx] - f0, axis=1)
    ok = (err <= bar_rel * fn + bar_abs * max(1.0, rms)) | bad
    assert ok.all(), (int((~ok).sum()), float(np.max(err / np.maximum(fn, rms))))
    return float(np.max(err[~bad] / np.maximum(fn[~bad], rms)))


def test_porous_9_8m_learned_scheduler(md, orc):
    """160^3-cell porous LJ (9,828,959 atoms), mixed path, learned scheduler
    trained on the run's own timings, as bench.py runs it."""
    s = inputs.lj_porous()
    p = s.params
    prm = orc.make_params(potential=orc.POT_LJ, rc=p["rc"], skin=p["skin"], dt=p["dt"])
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        with md.System(s.pos, s.vel, s.box, precision="mixed", stream=st, rc=p["rc"],
                       skin=p["skin"], dt=p["dt"]) as a:
            a.step(5)
            md.md_set_variant(a.h, md.MD_FORCE_FULL, md.MD_SCHED_DYNAMIC)
            assert md.md_cost_model(a.h, md.MD_COST_SAMPLE) > 100000
            assert np.isfinite(md.md_cost_model(a.h, md.MD_COST_TRAIN))
            md.md_set_variant(a.h, md.MD_FORCE_FULL, md.MD_SCHED_MLP)
            a.step(20)
            md.md_build_neighbors(a.h)
            pos, _, f = a.state()
            pos, f = pos.cpu().numpy(), f.cpu().numpy()
            idx = sample_ids(a.n, 600, inputs.SEED_BASE + 301)
            ooff, oids = check_rows(orc, a, pos, s.box, p["rc"] + p["skin"], idx)
            md.md_forces(a.h)
            f = a.state()[2].cpu().numpy()
    check_forces(orc, prm, f, pos, s.box, idx, ooff, oids, p["rc"], 2e-4, 1e-5)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_lj_liquid_1m(md, orc, precision):
    """64^3-cell LJ at T* = 1.2 (1,048,576 atoms), both precisions."""
    s = inputs.lj_fcc(nc=64, T=1.2)
    prm = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    with md.System(s.pos, s.vel, s.box, precision=precision) as a:
        a.step(30)
        md.md_build_neighbors(a.h)  # the rows below are for the current positions
        md.md_forces(a.h)
        pos, _, f = a.state()
        pos, f = pos.cpu().numpy(), f.cpu().numpy()
        idx = sample_ids(a.n, 600, inputs.SEED_BASE + 302)
        ooff, oids = check_rows(orc, a, pos, s.box, 2.8, idx)
    if precision == "fp64":
        check_forces(orc, prm, f, pos, s.box, idx, ooff, oids, 2.5, 1e-5, 1e-9)
    else:
        check_forces(orc, prm, f, pos, s.box, idx, ooff, oids, 2.5, 2e-4, 1e-5)


def test_sutton_chen_8m(md, orc):
    """128^3-cell Sutton-Chen fcc (8,388,608 atoms), mixed path, two passes."""
    s = inputs.sc_fcc(nc=128)
    p = s.params
    prm = orc.make_params(potential=orc.POT_SC, eps=p["eps"], sigma=p["sigma"], c=p["c"],
                          n_exp=p["n_exp"], m_exp=p["m_exp"], rc=p["rc"], skin=p["skin"],
                          dt=p["dt"])
    with md.System(s.pos, s.vel, s.box, potential="sc", precision="mixed", eps=p["eps"],
                   sigma=p["sigma"], c=p["c"], n_exp=p["n_exp"], m_exp=p["m_exp"], rc=p["rc"],
                   skin=p["skin"], dt=p["dt"]) as a:
        a.step(10)
        md.md_build_neighbors(a.h)
        md.md_forces(a.h)
        pos, _, f = a.state()
        pos, f = pos.cpu().numpy(), f.cpu().numpy()
        idx = sample_ids(a.n, 200, inputs.SEED_BASE + 304)
        ooff, oids = check_rows(orc, a, pos, s.box, p["rc"] + p["skin"], idx)
    check_forces(orc, prm, f, pos, s.box, idx, ooff, oids, p["rc"], 2e-4, 1e-5)


def test_ensemble_64_replicas(md, orc):
    """The 64-replica ensemble (2,428,400 atoms) as one batch: sampled atoms
    of each of eight replicas against the oracle on that replica's box."""
    reps = inputs.lj_ensemble()
    prm = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    with md.Batch([(r.pos, r.vel, r.box) for r in reps], precision="mixed",
                  scheduler=md.MD_SCHED_DYNAMIC) as b:
        b.step(30)
        md.md_build_neighbors(b.h)
        md.md_forces(b.h)
        pos, _, f = b.state()
        pos, f = pos.cpu().numpy(), f.cpu().numpy()
        off, ids = b.neighbors()
        off, ids = off.cpu().numpy(), ids.cpu().numpy()
    for r in range(0, 64, 8):
        a0, a1 = b.offsets[r], b.offsets[r + 1]
        box = np.asarray(reps[r].box)
        p_r = np.ascontiguousarray(pos[a0:a1])
        idx = sample_ids(a1 - a0, 80, inputs.SEED_BASE + 305 + r)
        ooff, oids = orc.neighbors_sample(p_r, box, 2.8, idx)
        for k, i in enumerate(idx):
            np.testing.assert_array_equal(ids[off[a0 + i]:off[a0 + i + 1]] - a0,
                                          oids[ooff[k]:ooff[k + 1]])
        check_forces(orc, prm, np.ascontiguousarray(f[a0:a1]), p_r, box, idx, ooff, oids, 2.5,
                     2e-4, 1e-5)
