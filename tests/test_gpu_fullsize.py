"""Parity at the full workload sizes, in the configuration bench.py times,
on sampled outputs the oracle computes one by one: list rows bit-exact,
forces within the mixed-path bar, for atoms drawn by a seeded sampler.

Each system first runs steps (rebuilds, graph replay, the scheduler it is
benchmarked with); then positions drawn from the input generator (the start
perturbed by a seeded Gaussian) are loaded into the running system, which
rebins and relists them, and its rows and forces at those positions are
compared with the oracle's.  The oracle only ever sees generator inputs."""
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


def perturbed(pos, box, amp, seed):
    g = inputs.gaussian(seed, pos.size).reshape(-1, 3)
    return np.mod(pos + amp * g, box)


def load(md, a, pos, vel):
    """Generator positions into the running system; list and forces for them."""
    md.md_set_state(a.h, torch.as_tensor(pos, device="cuda"), torch.as_tensor(vel, device="cuda"))
    md.md_build_neighbors(a.h)
    md.md_forces(a.h)
    return a.state()[2].cpu().numpy()


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
            pos = perturbed(s.pos, s.box, 0.05, inputs.SEED_BASE + 311)
            f = load(md, a, pos, s.vel)
            idx = sample_ids(a.n, 600, inputs.SEED_BASE + 301)
            ooff, oids = check_rows(orc, a, pos, s.box, p["rc"] + p["skin"], idx)
    check_forces(orc, prm, f, pos, s.box, idx, ooff, oids, p["rc"], 2e-4, 1e-5)


@pytest.fixture(scope="module")
def liquid_1m(orc):
    """The config-2 liquid at full size: a 16^3-cell fcc block melted by the
    oracle (2,000 steps, T* 2.4 then 1.2) and tiled 4 x 4 x 4 into 64^3
    cells, 1,048,576 atoms at rho* = 0.8442."""
    from melt import oracle_melt
    return inputs.tile(oracle_melt(orc, 16), 4)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_lj_liquid_1m(md, orc, liquid_1m, precision):
    """The melted 64^3-cell LJ liquid (1,048,576 atoms), both precisions:
    30 steps, then a second melted state (the same liquid, perturbed)."""
    s = liquid_1m
    prm = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    with md.System(s.pos, s.vel, s.box, precision=precision) as a:
        assert a.n == 1048576
        a.step(30)
        pos = perturbed(s.pos, s.box, 0.02, inputs.SEED_BASE + 312)
        f = load(md, a, pos, s.vel)
        idx = sample_ids(a.n, 600, inputs.SEED_BASE + 302)
        ooff, oids = check_rows(orc, a, pos, s.box, 2.8, idx)
    if precision == "fp64":
        check_forces(orc, prm, f, pos, s.box, idx, ooff, oids, 2.5, 1e-5, 1e-9)
    else:
        check_forces(orc, prm, f, pos, s.box, idx, ooff, oids, 2.5, 2e-4, 1e-5)


@pytest.mark.parametrize("variant", ["full", "paired"])
def test_sutton_chen_8m(md, orc, variant):
    """128^3-cell Sutton-Chen fcc (8,388,608 atoms), mixed path, two passes,
    with per-atom lists and with two atoms per thread."""
    s = inputs.sc_fcc(nc=128)
    p = s.params
    prm = orc.make_params(potential=orc.POT_SC, eps=p["eps"], sigma=p["sigma"], c=p["c"],
                          n_exp=p["n_exp"], m_exp=p["m_exp"], rc=p["rc"], skin=p["skin"],
                          dt=p["dt"])
    fv = md.MD_FORCE_PAIRED if variant == "paired" else md.MD_FORCE_FULL
    with md.System(s.pos, s.vel, s.box, potential="sc", precision="mixed", eps=p["eps"],
                   sigma=p["sigma"], c=p["c"], n_exp=p["n_exp"], m_exp=p["m_exp"], rc=p["rc"],
                   skin=p["skin"], dt=p["dt"], force_variant=fv) as a:
        a.step(10)
        pos = perturbed(s.pos, s.box, 0.03, inputs.SEED_BASE + 313)
        f = load(md, a, pos, s.vel)
        idx = sample_ids(a.n, 200, inputs.SEED_BASE + 304)
        ooff, oids = check_rows(orc, a, pos, s.box, p["rc"] + p["skin"], idx)
    check_forces(orc, prm, f, pos, s.box, idx, ooff, oids, p["rc"], 2e-4, 1e-5)


@pytest.mark.parametrize("variant", ["full", "paired"])
def test_eam_fe126_4m(md, orc, variant):
    """126^3-cell bcc under the piecewise embedded-atom potential (4,000,752
    atoms, the size of the paper's Fe126), mixed path, both passes, with
    per-atom lists and with two atoms per thread."""
    s = inputs.eam_bcc(nc=126)
    p = s.params
    keys = ("phi_r", "phi_a", "psi_r", "psi_a", "F_sqrt", "F_quad")
    t_orc = orc.make_eam(*[p[k] for k in keys])
    prm = orc.make_params(potential=orc.POT_EAM, rc=p["rc"], skin=p["skin"], dt=p["dt"],
                          eam=t_orc)
    fv = md.MD_FORCE_PAIRED if variant == "paired" else md.MD_FORCE_FULL
    with md.System(s.pos, s.vel, s.box, precision="mixed", eam=md.make_eam(*[p[k] for k in keys]),
                   rc=p["rc"], skin=p["skin"], dt=p["dt"], mass=p["mass"], force_variant=fv) as a:
        assert a.n == 4000752
        a.step(10)
        pos = perturbed(s.pos, s.box, 0.04, inputs.SEED_BASE + 314)
        f = load(md, a, pos, s.vel)
        idx = sample_ids(a.n, 300, inputs.SEED_BASE + 306)
        ooff, oids = check_rows(orc, a, pos, s.box, p["rc"] + p["skin"], idx)
    check_forces(orc, prm, f, pos, s.box, idx, ooff, oids, p["rc"], 2e-4, 1e-5)


@pytest.mark.parametrize("variant", ["full", "paired"])
def test_alloy_4_6m(md, orc, variant):
    """The Cu-Au-like random alloy on 105^3 fcc cells (4,630,500 atoms, the
    paper's Alloy size), mixed path with species parameters and masses, with
    per-atom lists and with two atoms per thread."""
    s = inputs.lj_alloy(nc=105)
    p = s.params
    sp = (p["types"], p["t_eps"], p["t_sigma"], p["t_mass"])
    prm = orc.make_params(potential=orc.POT_LJ, rc=p["rc"], skin=p["skin"], dt=p["dt"],
                          types=p["types"], t_eps=p["t_eps"], t_sigma=p["t_sigma"],
                          t_mass=p["t_mass"])
    fv = md.MD_FORCE_PAIRED if variant == "paired" else md.MD_FORCE_FULL
    with md.System(s.pos, s.vel, s.box, precision="mixed", species=sp, rc=p["rc"],
                   skin=p["skin"], dt=p["dt"], force_variant=fv) as a:
        assert a.n == 4630500
        a.step(10)
        pos = perturbed(s.pos, s.box, 0.04, inputs.SEED_BASE + 315)
        f = load(md, a, pos, s.vel)
        idx = sample_ids(a.n, 300, inputs.SEED_BASE + 307)
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
        pos = np.concatenate([perturbed(r.pos, r.box, 0.05, inputs.SEED_BASE + 320 + k)
                              for k, r in enumerate(reps)])
        f = load(md, b, pos, np.concatenate([r.vel for r in reps]))
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


@pytest.mark.parametrize("variant", ["paired", "cluster", "split", "half_atomic"])
def test_porous_9_8m_force_variants(md, orc, variant):
    """The other force layouts at the headline size (9,828,959 porous atoms,
    mixed path), as bench.py's comparison runs them: 10 steps (rebuilds and
    graph replay), then generator positions loaded, and the sampled forces
    against the oracle.  The list rows (kept per atom by every layout) are
    checked too."""
    s = inputs.lj_porous()
    p = s.params
    prm = orc.make_params(potential=orc.POT_LJ, rc=p["rc"], skin=p["skin"], dt=p["dt"])
    code = {"paired": md.MD_FORCE_PAIRED, "cluster": md.MD_FORCE_CLUSTER,
            "split": md.MD_FORCE_FULL, "half_atomic": md.MD_FORCE_HALF_ATOMIC}[variant]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        with md.System(s.pos, s.vel, s.box, precision="mixed", stream=st, rc=p["rc"],
                       skin=p["skin"], dt=p["dt"], force_variant=code) as a:
            if variant == "split":
                md.md_set_decomposition(a.h, 2, 2, 2)
            a.step(10)
            pos = perturbed(s.pos, s.box, 0.05, inputs.SEED_BASE + 313)
            f = load(md, a, pos, s.vel)
            idx = sample_ids(a.n, 400, inputs.SEED_BASE + 303)
            if variant == "half_atomic":
                # a half list exports the pairs it owns; the full rows come from the oracle
                ooff, oids = orc.neighbors_sample(pos, s.box, p["rc"] + p["skin"], idx)
            else:
                ooff, oids = check_rows(orc, a, pos, s.box, p["rc"] + p["skin"], idx)
    check_forces(orc, prm, f, pos, s.box, idx, ooff, oids, p["rc"], 2e-4, 1e-5)
