"""Batches of uneven replicas in one system (md_create_batch) and CUDA-graph
replay of the time step, against the oracle and against separate systems."""
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


def ensemble(count=5):
    """Uneven replicas (864 .. ~5300 atoms, rho 0.7-0.9, T 0.5-1.5), each
    perturbed off its lattice so that forces are non-zero."""
    reps = inputs.lj_ensemble(count=count, nmin=800, nmax=6000, seed=inputs.SEED_BASE + 55)
    out = []
    for r, s in enumerate(reps):
        g = inputs.gaussian(inputs.SEED_BASE + 560 + r, s.pos.size).reshape(-1, 3)
        out.append((np.mod(s.pos + 0.05 * g, s.box), s.vel, s.box))
    return out


def tiny_and_large():
    """Ten dilute replicas of 27-125 atoms (jittered simple-cubic sites 2.9
    apart, boxes of 3-5 spacings), so that one 256-atom block of the force
    kernel spans several boxes, then two dense ones from the ensemble."""
    out = []
    for r in range(10):
        m = 3 + r % 3
        a = 2.9
        g = np.arange(m) * a
        site = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 0.5 * a
        jit = inputs.gaussian(inputs.SEED_BASE + 580 + r, site.size).reshape(-1, 3)
        vel = 0.3 * inputs.gaussian(inputs.SEED_BASE + 600 + r, site.size).reshape(-1, 3)
        box = (m * a,) * 3
        out.append((np.mod(site + 0.25 * jit, box), vel, box))
    return out + ensemble(2)


def near_cutoff(pos, box, off, ids, rc, delta):
    rows = np.repeat(np.arange(len(pos)), np.diff(off))
    d = pos[ids] - pos[rows]
    d -= box * np.round(d / box)
    r = np.sqrt(np.sum(d * d, axis=1))
    bad = np.zeros(len(pos), bool)
    bad[rows[np.abs(r - rc) < delta]] = True
    return bad


def variant_code(md, variant):
    return md.MD_FORCE_PAIRED if variant == "paired" else md.MD_FORCE_FULL


@pytest.mark.parametrize("variant", ["full", "paired"])
@pytest.mark.parametrize("which", ["uneven", "tiny_and_large"])
def test_batch_cells_lists_forces_match_oracle(md, orc, which, variant):
    """Cells and lists bit-exact, forces and energies within the mixed bars,
    per replica, with per-atom lists and with two atoms per thread (each box's
    cells in the pairing order, slot lists built with the box's geometry).
    With tiny replicas a block of the force kernel spans more than two boxes
    and reads the global shift table; otherwise the shift tables of its (at
    most two) boxes sit in shared memory."""
    reps = ensemble() if which == "uneven" else tiny_and_large()
    with md.Batch(reps, precision="mixed", force_variant=variant_code(md, variant)) as b:
        nc, cell_of, start = b.cells()
        off, ids = b.neighbors()
        _, _, f = b.state()
        ke, pe = b.energies()
    cell_of, start, off, ids, f = (t.cpu().numpy() for t in (cell_of, start, off, ids, f))
    cell0 = 0
    for r, (pos, vel, box) in enumerate(reps):
        a0, a1 = b.offsets[r], b.offsets[r + 1]
        onc, ocell, ostart, _ = orc.bin_cells(pos, box, 2.8)
        nr = int(np.prod(onc))
        np.testing.assert_array_equal(cell_of[a0:a1], ocell + cell0)
        np.testing.assert_array_equal(start[cell0:cell0 + nr + 1], ostart + a0)
        cell0 += nr
        ooff, oids = orc.neighbors_cells(pos, box, 2.8)
        np.testing.assert_array_equal(off[a0:a1 + 1] - off[a0], ooff)
        np.testing.assert_array_equal(ids[off[a0]:off[a1]], oids + a0)
        U0, f0 = orc.lj_list(pos, box, ooff, oids)
        bad = near_cutoff(pos, np.asarray(box), ooff, oids, 2.5, 1e-5)
        fn = np.linalg.norm(f0, axis=1)
        rms = math.sqrt(np.mean(fn * fn))
        err = np.linalg.norm(f[a0:a1] - f0, axis=1)
        ok = (err <= 2e-4 * fn + 1e-5 * max(1.0, rms)) | bad
        assert ok.all(), (r, int((~ok).sum()))
        # pairs within 1e-5 of r_c may fall on either side: at most their own energy
        slack = lj_straddle_bound(orc, pos, np.asarray(box), ooff, oids, 2.5, 1e-5)
        assert abs(pe[r] - U0) <= 2e-6 * abs(U0) + slack, (r, pe[r], U0, slack)
        assert abs(ke[r] - 0.5 * np.sum(vel ** 2)) <= 1e-12 * ke[r]
    assert cell0 == nc[0] and nc[1] == nc[2] == 1
    assert len(start) == cell0 + 1


@pytest.mark.parametrize("variant", ["full", "paired"])
def test_batch_dynamics_equal_separate_systems(md, variant):
    """Before the first rebuild a replica in a batch runs exactly the
    arithmetic it runs alone (same cells, same list order, and with two atoms
    per thread the same slots): bit-equal.  Later
    the batch rebuilds every replica whenever one of them needs it; a rebuild
    moves atoms to new cells and changes the float32 rounding of their
    cell-relative coordinates, so the trajectories then separate at the rate
    of the dynamics' own chaos, far below any cross-talk between replicas."""
    reps = ensemble()
    fv = variant_code(md, variant)
    for nsteps, tol in ((3, 0.0), (60, 1e-4)):
        sep = []
        for pos, vel, box in reps:
            with md.System(pos, vel, box, precision="mixed", force_variant=fv) as a:
                b0 = a.stats()["builds"]
                a.step(nsteps)
                sep.append((a.state()[0].cpu().numpy(), sum(a.energy()),
                            a.stats()["builds"] - b0))
        with md.Batch(reps, precision="mixed", force_variant=fv) as b:
            b0 = b.stats()["builds"]
            b.step(nsteps)
            pos = b.state()[0].cpu().numpy()
            ke, pe = b.energies()
            builds = b.stats()["builds"] - b0
        if tol == 0.0 and (builds > 0 or any(x[2] > 0 for x in sep)):
            continue  # a rebuild happened already: only the loose check applies
        for r, (_, _, box) in enumerate(reps):
            d = pos[b.offsets[r]:b.offsets[r + 1]] - sep[r][0]
            d -= np.asarray(box) * np.round(d / np.asarray(box))
            assert np.max(np.abs(d)) <= tol, (nsteps, r, np.max(np.abs(d)))
            assert abs(ke[r] + pe[r] - sep[r][1]) <= max(tol, 1e-12) * abs(sep[r][1]), (nsteps, r)


@pytest.mark.parametrize("variant", ["full", "paired"])
def test_batch_energy_tracks_oracle(md, orc, variant):
    reps = ensemble(3)
    sched = md.MD_SCHED_DYNAMIC if variant == "full" else md.MD_SCHED_GRID
    with md.Batch(reps, precision="mixed", scheduler=sched,
                  force_variant=variant_code(md, variant)) as b:
        b.step(40)
        ke, pe = b.energies()
    p = orc.make_params(potential=orc.POT_LJ, dt=0.005)
    for r, (pos, vel, box) in enumerate(reps):
        E = orc.md_run(p, pos, vel, box, 40)["energies"][-1, 2]
        assert abs(ke[r] + pe[r] - E) < 1e-4 * abs(E), (r, ke[r] + pe[r], E)


def test_batch_rejects_unsupported_modes(md):
    reps = ensemble(2)
    with pytest.raises(md.MDError):
        md.Batch(reps, precision="fp64")
    with pytest.raises(md.MDError):
        md.Batch(reps, scheduler=md.MD_SCHED_MLP)
    with pytest.raises(md.MDError):  # two atoms per thread: the grid launch only
        md.Batch(reps, force_variant=md.MD_FORCE_PAIRED, scheduler=md.MD_SCHED_DYNAMIC)
    with md.Batch(reps) as b:
        with pytest.raises(md.MDError):
            md.md_set_variant(b.h, md.MD_FORCE_HALF_COLOR, md.MD_SCHED_GRID)
        with pytest.raises(md.MDError):
            md.md_set_variant(b.h, md.MD_FORCE_PAIRED, md.MD_SCHED_DYNAMIC)
        with pytest.raises(md.MDError):
            md.md_cost_model(b.h, md.MD_COST_SAMPLE)


@pytest.mark.parametrize("sched", ["grid", "paircount"])
def test_graph_replay_equals_plain_launches(md, sched):
    """md_step on a non-default stream replays a captured step, whose rebuild
    chain sits under a conditional graph node; with per-launch timing on, the
    force kernels launch one by one around that conditional chain; on the
    default stream every kernel launches on its own (the gated chain included).
    All three must agree bit for bit, and the first two must count the same
    kernel launches (the chain only when it ran).  Under the pair-count
    scheduler the chain also recomputes the persistent kernel's partition."""
    s = inputs.lj_fcc(nc=8, T=1.0)
    code = md.MD_SCHED_GRID if sched == "grid" else md.MD_SCHED_PAIRCOUNT
    out, launches = [], []
    for mode in ("graphs", "timing", "default_stream"):
        st = torch.cuda.default_stream() if mode == "default_stream" else torch.cuda.Stream()
        with torch.cuda.stream(st):
            a = md.System(s.pos, s.vel, s.box, precision="mixed", stream=st, scheduler=code)
            md.md_set_timing(a.h, mode == "timing")
            a.step(40)
            a.step(25)
            out.append(a.state())
            stats = a.stats()
            a.close()
        assert stats["builds"] >= 2
        launches.append(stats["launches"])
    for other in out[1:]:
        for x, y in zip(out[0], other):
            assert torch.equal(x, y)
    assert launches[0] == launches[1]
    assert launches[2] > launches[0]  # the gated chain's launches on steps without a rebuild


def test_batch_paired_graph_replay_and_variant_switch(md):
    """Two atoms per thread in a batch: graph replay, timed launches and plain
    launches on the default stream agree bit for bit over steps with
    rebuilds; switching a running batch between the layouts rebuilds its
    lists and keeps it on the same trajectory within the mixed bar."""
    reps = ensemble(4)
    out = []
    for mode in ("graphs", "timing", "default_stream"):
        st = torch.cuda.default_stream() if mode == "default_stream" else torch.cuda.Stream()
        with torch.cuda.stream(st):
            b = md.Batch(reps, precision="mixed", stream=st, force_variant=md.MD_FORCE_PAIRED)
            md.md_set_timing(b.h, mode == "timing")
            b.step(30)
            b.step(20)
            out.append(b.state())
            builds = b.stats()["builds"]
            b.close()
        assert builds >= 2
    for other in out[1:]:
        for x, y in zip(out[0], other):
            assert torch.equal(x, y)
    with md.Batch(reps, precision="mixed") as b:
        b.step(10)
        md.md_set_variant(b.h, md.MD_FORCE_PAIRED, md.MD_SCHED_GRID)
        b.step(10)
        md.md_set_variant(b.h, md.MD_FORCE_FULL, md.MD_SCHED_GRID)
        b.step(10)
        ke, pe = b.energies()
    with md.Batch(reps, precision="mixed") as c:
        c.step(30)
        ke2, pe2 = c.energies()
    for r in range(len(reps)):
        assert abs(ke[r] + pe[r] - ke2[r] - pe2[r]) < 1e-4 * abs(ke2[r] + pe2[r]), r
