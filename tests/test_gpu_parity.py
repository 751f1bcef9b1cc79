"""GPU path vs the CPU oracle, element by element, through the C ABI.

Bars (the tolerances every parity test below applies):
  * cells and neighbour sets: bit-exact.
  * forces, fp64 path: |df_i| <= 1e-5 |f_i| + 1e-9 rms(f) per atom.
  * forces, mixed path: |df_i| <= 2e-4 |f_i| + 1e-5 * max(1, rms(f)) per atom
    (absolute part scaled with the force scale, 1e-5 at unit forces).
  * energies: fp64 1e-10 relative per evaluation, 1e-6 relative per step over
    100 velocity-Verlet steps.
Atoms with a pair within delta of the cutoff are compared separately: there a
different rounding may put the pair on the other side of r_c, a legitimate
difference of one pair term (checked to be exactly that size bound).
"""
import math

import numpy as np
import pytest

from paper_1611_00075_gb300 import inputs

from cutoff_bounds import sc_straddle_bound

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


def perturbed(s, amp, seed):
    g = inputs.gaussian(seed, s.pos.size).reshape(-1, 3)
    return np.mod(s.pos + amp * g, s.box)


def pair_distances(pos, box, off, ids):
    rows = np.repeat(np.arange(len(pos)), np.diff(off))
    d = pos[ids] - pos[rows]
    d -= box * np.round(d / box)
    return rows, np.sqrt(np.sum(d * d, axis=1))


def near_cutoff(pos, box, off, ids, rc, delta):
    rows, r = pair_distances(pos, box, off, ids)
    bad = np.zeros(len(pos), bool)
    bad[rows[np.abs(r - rc) < delta]] = True
    return bad


def lj_system(name):
    if name == "melt4000":
        # the config-2 liquid at 4,000 atoms, melted by the oracle
        import oracle
        from melt import oracle_melt
        oracle.build()
        s = oracle_melt(oracle, 10)
        return s, s.pos
    if name == "fcc4000":
        s = inputs.lj_fcc(nc=10, T=0.72)
        return s, perturbed(s, 0.05, 101)
    if name == "liquid_like":
        # hot, disordered start; larger displacements put pairs near r = 0.7
        # where dt = 0.005 is unstable for any integrator
        s = inputs.lj_fcc(nc=8, T=1.2)
        return s, perturbed(s, 0.06, 102)
    if name == "porous":
        s = inputs.lj_porous(nc=12, fraction=0.4, rmin=2.0, rmax=5.0)
        return s, perturbed(s, 0.05, 103)
    raise KeyError(name)


def sc_system():
    s = inputs.sc_fcc(nc=10)
    return s, perturbed(s, 0.03, 104)


def sc_kw(s):
    p = s.params
    return dict(potential="sc", eps=p["eps"], sigma=p["sigma"], c=p["c"], n_exp=p["n_exp"],
                m_exp=p["m_exp"], rc=p["rc"], skin=p["skin"], dt=p["dt"])


def oracle_sc_params(orc, s):
    p = s.params
    return orc.make_params(potential=orc.POT_SC, eps=p["eps"], sigma=p["sigma"], c=p["c"],
                           n_exp=p["n_exp"], m_exp=p["m_exp"], rc=p["rc"], skin=p["skin"],
                           dt=p["dt"])


def check_forces(f, f0, bad, precision):
    fn = np.linalg.norm(f0, axis=1)
    rms = math.sqrt(np.mean(fn * fn))
    err = np.linalg.norm(f - f0, axis=1)
    if precision == "fp64":
        tol = 1e-5 * fn + 1e-9 * rms
    else:
        tol = 2e-4 * fn + 1e-5 * max(1.0, rms)
    ok = (err <= tol) | bad
    assert ok.all(), (precision, int((~ok).sum()), float(np.max((err / np.maximum(tol, 1e-300))[~bad])))
    return float(np.max(err[~bad] / np.maximum(fn[~bad], rms)))


# ------------------------------------------------------------------ cells

@pytest.mark.parametrize("name", ["fcc4000", "porous", "melt4000"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cells_bit_exact(md, orc, name, precision):
    """Cells and cell starts of a generator state against the oracle; after
    25 steps, the cells of the drifted state (absolute positions rebuilt from
    cell-relative ones) equal those of the same exported positions loaded
    back; and a second generator state loaded into the running system bins as
    the oracle bins it."""
    s, pos = lj_system(name)
    with md.System(pos, s.vel, s.box, precision=precision) as sy:
        nc, cell_of, start = sy.cells()
        onc, ocell, ostart, _ = orc.bin_cells(pos, s.box, 2.8)
        assert list(onc) == nc
        np.testing.assert_array_equal(cell_of.cpu().numpy(), ocell)
        np.testing.assert_array_equal(start.cpu().numpy(), ostart)
        sy.step(25)
        md.md_bin_cells(sy.h)
        _, cell1, start1 = sy.cells()
        p1, v1, _ = sy.state()
        md.md_set_state(sy.h, p1, v1)
        md.md_bin_cells(sy.h)
        _, cell2, start2 = sy.cells()
        assert torch.equal(cell1, cell2) and torch.equal(start1, start2)
        pos2 = np.mod(pos + 0.03 * inputs.gaussian(inputs.SEED_BASE + 131, pos.size).reshape(-1, 3),
                      s.box)
        md.md_set_state(sy.h, torch.as_tensor(pos2, device="cuda"), v1)
        md.md_bin_cells(sy.h)
        _, cell3, start3 = sy.cells()
    onc, ocell, ostart, _ = orc.bin_cells(pos2, s.box, 2.8)
    np.testing.assert_array_equal(cell3.cpu().numpy(), ocell)
    np.testing.assert_array_equal(start3.cpu().numpy(), ostart)


# ------------------------------------------------------------------ lists

@pytest.mark.parametrize("name", ["fcc4000", "liquid_like", "porous", "melt4000"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_neighbors_bit_exact(md, orc, name, precision):
    """Lists of a generator state against the oracle; after 40 steps and a
    rebuild, the list equals the one built for the same exported positions
    loaded back; a second generator state loaded into the running system
    lists as the oracle does (full list, and its half export j > i)."""
    s, pos = lj_system(name)
    with md.System(pos, s.vel, s.box, precision=precision) as sy:
        off, ids = sy.neighbors()
        ooff, oids = orc.neighbors_cells(pos, s.box, 2.8)
        np.testing.assert_array_equal(off.cpu().numpy(), ooff)
        np.testing.assert_array_equal(ids.cpu().numpy(), oids)
        sy.step(40)
        md.md_build_neighbors(sy.h)
        off1, ids1 = sy.neighbors()
        p1, v1, _ = sy.state()
        md.md_set_state(sy.h, p1, v1)
        md.md_build_neighbors(sy.h)
        off2, ids2 = sy.neighbors()
        assert torch.equal(off1, off2) and torch.equal(ids1, ids2)
        pos2 = np.mod(pos + 0.03 * inputs.gaussian(inputs.SEED_BASE + 132, pos.size).reshape(-1, 3),
                      s.box)
        md.md_set_state(sy.h, torch.as_tensor(pos2, device="cuda"), v1)
        md.md_build_neighbors(sy.h)
        off, ids = sy.neighbors()
        ooff, oids = orc.neighbors_cells(pos2, s.box, 2.8)
        np.testing.assert_array_equal(off.cpu().numpy(), ooff)
        np.testing.assert_array_equal(ids.cpu().numpy(), oids)
        off, ids = sy.neighbors(half=True)
        ooff, oids = orc.neighbors_cells(pos2, s.box, 2.8, half=True)
        np.testing.assert_array_equal(off.cpu().numpy(), ooff)
        np.testing.assert_array_equal(ids.cpu().numpy(), oids)


@pytest.mark.parametrize("jitter", [0.0, 3e-9])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_neighbors_shell_on_list_radius(md, orc, jitter, precision):
    """An fcc lattice whose 5th shell (24 neighbours at a0 sqrt(5/2)) lies on
    r_list = 2.8: every atom has two dozen candidates inside the float32
    band, where only the float64 definition decides (and whose rounding puts
    some just inside and some just outside).  Jitter of a few 1e-9 moves
    pairs across r_list both ways."""
    a0 = 2.8 / math.sqrt(2.5)
    nc = 6
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.stack(np.meshgrid(*[np.arange(nc)] * 3, indexing="ij"), -1).reshape(-1, 1, 3)
    pos = ((g + base[None]) * a0).reshape(-1, 3)
    box = np.full(3, nc * a0)
    if jitter:
        pos = np.mod(pos + jitter * inputs.gaussian(inputs.SEED_BASE + 77, pos.size).reshape(-1, 3),
                     box)
    with md.System(pos, np.zeros_like(pos), box, precision=precision) as sy:
        off, ids = sy.neighbors()
    ooff, oids = orc.neighbors_cells(pos, box, 2.8)
    np.testing.assert_array_equal(off.cpu().numpy(), ooff)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    counts = np.diff(ooff)
    assert counts.min() >= 54 and counts.max() <= 78  # shells 1-4 always, shell 5 in part


def test_neighbors_perfect_lattice_counts(md, orc):
    s = inputs.lj_fcc(nc=10, T=0.0)
    with md.System(s.pos, s.vel, s.box, precision="mixed") as sy:
        off, ids = sy.neighbors()
        assert np.all(np.diff(off.cpu().numpy()) == 78)


# ------------------------------------------------------------------ forces

@pytest.mark.parametrize("name", ["fcc4000", "liquid_like", "porous", "melt4000"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lj_forces_and_energy(md, orc, name, precision):
    s, pos = lj_system(name)
    off, ids = orc.neighbors_cells(pos, s.box, 2.8)
    U0, f0 = orc.lj_list(pos, s.box, off, ids)
    delta = 1e-12 if precision == "fp64" else 1e-5
    bad = near_cutoff(pos, s.box, off, ids, 2.5, delta)
    with md.System(pos, s.vel, s.box, precision=precision) as sy:
        _, _, f = sy.state()
        ke, pe = sy.energy()
    check_forces(f.cpu().numpy(), f0, bad, precision)
    ke0 = 0.5 * np.sum(s.vel * s.vel)
    assert abs(ke - ke0) <= 1e-12 * ke0
    tol = 1e-10 if precision == "fp64" else 2e-6
    assert abs(pe - U0) <= tol * abs(U0), (pe, U0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sc_density_forces_energy(md, orc, precision):
    s, pos = sc_system()
    off, ids = orc.neighbors_cells(pos, s.box, 2.2)
    U0, f0, rho0, dF0 = orc.sc_list(pos, s.box, off, ids, c=s.params["c"])
    delta = 1e-12 if precision == "fp64" else 1e-5
    bad = near_cutoff(pos, s.box, off, ids, 2.0, delta)
    with md.System(pos, s.vel, s.box, precision=precision, **sc_kw(s)) as sy:
        _, _, f = sy.state()
        rho = torch.empty(s.n, dtype=torch.float64, device="cuda")
        dF = torch.empty_like(rho)
        md.md_get_density(sy.h, rho, dF)
        ke, pe = sy.energy()
    rho, dF = rho.cpu().numpy(), dF.cpu().numpy()
    ok = ~bad
    rtol = 1e-12 if precision == "fp64" else 2e-6
    np.testing.assert_allclose(rho[ok], rho0[ok], rtol=rtol)
    np.testing.assert_allclose(dF[ok], dF0[ok], rtol=rtol if precision == "fp64" else 1e-6)
    check_forces(f.cpu().numpy(), f0, bad, precision)
    tol = 1e-10 if precision == "fp64" else 2e-6
    # pairs within delta of r_c may fall on either side: at most their own energy
    slack = sc_straddle_bound(orc, pos, s.box, off, ids, delta, c=s.params["c"])
    assert abs(pe - U0) <= tol * abs(U0) + slack, (pe, U0, slack)


# ------------------------------------------------------------------ dynamics

def test_nve_100_steps_fp64_config1(md, orc):
    """4000-atom fcc at T*=0.72, dt 0.005: total energy after every step
    within 1e-6 relative of the oracle's own trajectory."""
    s = inputs.lj_fcc(nc=10, T=0.72)
    p = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    ref = orc.md_run(p, s.pos, s.vel, s.box, 100)
    E0 = ref["energies"]
    with md.System(s.pos, s.vel, s.box, precision="fp64") as sy:
        ke, pe = sy.energy()
        es = [(ke, pe)]
        for k in range(100):
            sy.step(1)
            es.append(sy.energy())
    es = np.array(es)
    tot = es[:, 0] + es[:, 1]
    rel = np.abs(tot - E0[:, 2]) / np.abs(E0[:, 2])
    print("fp64 config 1: max relative total-energy error over 100 steps %.3g" % rel.max())
    assert np.max(rel) < 1e-6, np.max(rel)


def test_nve_100_steps_mixed_config1(md, orc):
    """The same bar on the mixed path (float32 pair terms, float64 state and
    sums): 4000-atom fcc at T*=0.72, dt 0.005, total energy after every one
    of 100 steps within 1e-6 relative of the oracle's float64 trajectory."""
    s = inputs.lj_fcc(nc=10, T=0.72)
    p = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    E0 = orc.md_run(p, s.pos, s.vel, s.box, 100)["energies"]
    with md.System(s.pos, s.vel, s.box, precision="mixed") as sy:
        es = [sy.energy()]
        for k in range(100):
            sy.step(1)
            es.append(sy.energy())
    es = np.array(es)
    rel = np.abs(es[:, 0] + es[:, 1] - E0[:, 2]) / np.abs(E0[:, 2])
    print("mixed config 1: max relative total-energy error over 100 steps %.3g" % rel.max())
    assert np.max(rel) < 1e-6, np.max(rel)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nve_100_steps_melted_liquid(md, orc, precision):
    """The config-2 liquid (4,000 atoms melted by the oracle, T* = 1.2):
    total energy after every one of 100 steps within 1e-6 relative of the
    oracle's float64 trajectory, on both paths."""
    s, pos = lj_system("melt4000")
    p = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    E0 = orc.md_run(p, pos, s.vel, s.box, 100)["energies"]
    with md.System(pos, s.vel, s.box, precision=precision) as sy:
        es = [sy.energy()]
        for k in range(100):
            sy.step(1)
            es.append(sy.energy())
    es = np.array(es)
    rel = np.abs(es[:, 0] + es[:, 1] - E0[:, 2]) / np.abs(E0[:, 2])
    print("%s melted liquid: max relative total-energy error over 100 steps %.3g"
          % (precision, rel.max()))
    assert np.max(rel) < 1e-6, np.max(rel)


def test_step_chunks_equal_single_steps(md):
    """md_step(n) equals n calls of md_step(1) bit for bit (fp64, deterministic)."""
    s, pos = lj_system("liquid_like")
    with md.System(pos, s.vel, s.box, precision="fp64") as a, \
            md.System(pos, s.vel, s.box, precision="fp64") as b:
        a.step(30)
        for _ in range(30):
            b.step(1)
        pa, va, fa = a.state()
        pb, vb, fb = b.state()
    # merged half kicks differ from separate ones only by rounding
    assert torch.max(torch.abs(pa - pb)).item() < 1e-12
    assert torch.max(torch.abs(va - vb)).item() < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_resume_bit_exact(md, precision):
    """A state saved after 20 steps and loaded back continues bit for bit like
    the uninterrupted run.  Loading a state rebinds the cells and rebuilds the
    list (Sec. 3.3: any move that may invalidate the list forces a rebuild),
    and a rebuild re-rounds the cell-relative coordinates, so the
    uninterrupted run rebuilds at the same step (md_build_neighbors)."""
    s, pos = lj_system("liquid_like")
    with md.System(pos, s.vel, s.box, precision=precision) as a:
        a.step(20)
        md.md_build_neighbors(a.h)
        a.step(20)
        p2, v2, f2 = a.state()
    with md.System(pos, s.vel, s.box, precision=precision) as b:
        b.step(20)
        p, v, _ = b.state()
        md.md_set_state(b.h, p, v)
        b.step(20)
        q2, w2, g2 = b.state()
    assert torch.equal(q2, p2)
    assert torch.equal(w2, v2)
    assert torch.equal(g2, f2)


def test_runs_are_deterministic(md):
    s, pos = lj_system("porous")
    out = []
    for _ in range(2):
        with md.System(pos, s.vel, s.box, precision="mixed") as a:
            a.step(50)
            out.append(a.state())
    for x, y in zip(out[0], out[1]):
        assert torch.equal(x, y)


def test_mixed_energy_tracks_fp64(md):
    s = inputs.lj_fcc(nc=10, T=0.72)
    E = []
    for prec in ("fp64", "mixed"):
        with md.System(s.pos, s.vel, s.box, precision=prec) as a:
            a.step(100)
            E.append(sum(a.energy()))
    assert abs(E[1] - E[0]) < 1e-4 * abs(E[0])



@pytest.mark.parametrize("stream", ["default", "own"])
@pytest.mark.parametrize("variant", ["full", "paired"])
def test_timing_skips_launches_a_list_overflow_voids(md, stream, variant):
    """A list that overflows in a rebuild inside md_step stops every later
    launch of the call until the host has grown it and enqueued the steps
    again.  Per-launch timing counts the work that ran: one force launch per
    step however many repairs there were, the repairs as rebuilds.  A dilute
    lattice (spacing 2) is compressed by an inward velocity field, so the
    neighbour counts outgrow the list's headroom within a few steps."""
    nc = 12
    side = 2.0
    g = np.stack(np.meshgrid(*[np.arange(nc)] * 3, indexing="ij"), -1).reshape(-1, 3)
    box = np.full(3, nc * side)
    pos = (g + 0.5) * side
    vel = -8.0 * (pos - box / 2)
    fv = md.MD_FORCE_PAIRED if variant == "paired" else md.MD_FORCE_FULL
    st = torch.cuda.default_stream() if stream == "default" else torch.cuda.Stream()
    with torch.cuda.stream(st), md.System(pos, vel, box, precision="mixed", stream=st,
                                          force_variant=fv) as a:
        md.md_forces(a.h)
        s0 = a.stats()
        nsteps = 8
        md.md_set_timing(a.h, True)
        a.step(nsteps)
        s1 = a.stats()
        md.md_set_timing(a.h, False)
    grew = (s1["slots"] and s1["slot_max"] > s0["slot_max"]) or s1["cap"] > s0["cap"]
    print("%s/%s: builds %d -> %d, counts %s, ms %s" % (variant, stream, s0["builds"],
          s1["builds"], s1["count"], {k: round(v, 3) for k, v in s1["ms"].items()}))
    assert grew
    assert s1["count"]["force"] == nsteps
    assert s1["count"]["integrate"] == 1
    # one rebuild mark per step, plus one per host repair (at least one)
    assert s1["count"]["rebuild"] > nsteps
    assert s1["count"]["rebuild"] - nsteps <= s1["builds"] - s0["builds"]


# ------------------------------------------------------------------ errors

def test_invalid_arguments(md):
    s = inputs.lj_fcc(nc=10)
    with pytest.raises(md.MDError) as e:
        md.System(s.pos, s.vel, s.box, rc=-1.0)
    assert e.value.status == md.MD_ERR_INVALID
    with pytest.raises(md.MDError) as e:
        md.System(s.pos, s.vel, [5.0, 5.0, 5.0])
    assert e.value.status == md.MD_ERR_INVALID
    with md.System(s.pos, s.vel, s.box) as a:
        with pytest.raises(md.MDError) as e:
            md.md_step(a.h, -1)
        assert e.value.status == md.MD_ERR_INVALID


@pytest.mark.parametrize("stream", ["default", "own"])
def test_capacity_limit_and_regrow(md, orc, stream):
    """A state that outgrows the list capacity: creation with a fixed
    max_neighbors fails with MD_ERR_LIST_OVERFLOW; without it md_step grows
    the list and repeats the step.  On its own stream the steps replay
    captured graphs, which the regrowth drops (they hold the old list)."""
    # dilute start: lattice spacing 2.0 -> few neighbours; the list is sized small
    nc = 12
    side = 2.0
    g = np.stack(np.meshgrid(*[np.arange(nc)] * 3, indexing="ij"), -1).reshape(-1, 3)
    box = np.full(3, nc * side)
    dilute = (g + 0.5) * side
    # dense: same atoms packed into a cube of spacing 1.1 (still a valid LJ state)
    dense = (g + 0.5) * 1.1
    vel = np.zeros_like(dilute)
    with pytest.raises(md.MDError) as e:
        md.System(dense, vel, box, max_neighbors=8)
    assert e.value.status == md.MD_ERR_LIST_OVERFLOW
    st = torch.cuda.default_stream() if stream == "default" else torch.cuda.Stream()
    with torch.cuda.stream(st), md.System(dilute, vel, box, precision="fp64", stream=st) as a:
        a.step(3)                       # on its own stream: graphs captured
        md.md_set_state(a.h, torch.as_tensor(dilute, device="cuda"), torch.as_tensor(vel, device="cuda"))
        cap0 = a.stats()["cap"]
        md.md_set_state(a.h, torch.as_tensor(dense, device="cuda"), None)
        a.step(5)                       # the rebuild overflows and is repaired
        assert a.stats()["cap"] > cap0
        p, v, f = a.state()
    pr = orc.make_params(potential=orc.POT_LJ, dt=0.005)
    ref = orc.md_run(pr, dense, vel, box, 5)
    np.testing.assert_allclose(p.cpu().numpy(), ref["pos"], atol=1e-10)
