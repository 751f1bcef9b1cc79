"""Edge cases of the path, through the C ABI: an empty system, one atom with
no neighbour, inputs outside the periodic box, atoms exactly on cell faces,
and a non-finite state reported through the device status word.

Bars as in test_gpu_parity.py: cells and lists bit-exact; forces within
1e-5 |f| + 1e-9 rms(f) (fp64) or 2e-4 |f| + 1e-5 max(1, rms(f)) (mixed)."""
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


def check_forces(f, f0, precision, bad=None):
    """Per-atom bars; atoms flagged in `bad` (a pair within rounding of the
    cutoff) are left out."""
    fn = np.linalg.norm(f0, axis=1)
    rms = math.sqrt(np.mean(fn * fn))
    err = np.linalg.norm(f - f0, axis=1)
    tol = 1e-5 * fn + 1e-9 * rms if precision == "fp64" else 2e-4 * fn + 1e-5 * max(1.0, rms)
    ok = err <= tol
    if bad is not None:
        ok |= bad
    assert np.all(ok), (precision, int(np.sum(~ok)))


def near_cutoff(pos, box, off, ids, rc, delta):
    rows = np.repeat(np.arange(len(pos)), np.diff(off))
    d = pos[ids] - pos[rows]
    d -= box * np.round(d / box)
    r = np.sqrt(np.sum(d * d, axis=1))
    bad = np.zeros(len(pos), bool)
    bad[rows[np.abs(r - rc) < delta]] = True
    return bad


def test_empty_system_is_rejected(md):
    with pytest.raises(md.MDError) as e:
        md.System(np.zeros((0, 3)), np.zeros((0, 3)), [10.0, 10.0, 10.0])
    assert e.value.status == md.MD_ERR_INVALID


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_single_atom_free_flight(md, precision):
    """No neighbour: zero force and energy, and 400 steps of straight flight
    that cross cells (with rebuilds) and the periodic boundary in x and y."""
    box = np.array([9.0, 9.5, 10.0])
    pos = np.array([[8.95, 0.02, 5.0]])
    vel = np.array([[1.3, -0.7, 0.2]])
    with md.System(pos, vel, box, precision=precision) as a:
        b0 = a.stats()["builds"]
        a.step(400)
        p, v, f = (t.cpu().numpy() for t in a.state())
        ke, pe = a.energy()
        builds = a.stats()["builds"] - b0
    assert builds >= 2
    d = p - np.mod(pos + 400 * 0.005 * vel, box)
    d -= box * np.round(d / box)
    assert np.max(np.abs(d)) < 1e-12
    assert np.all(f == 0.0) and pe == 0.0
    np.testing.assert_array_equal(v, vel)
    assert ke == pytest.approx(0.5 * np.sum(vel ** 2), rel=1e-15)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_wrap_at_the_box_faces_is_exact(md, orc, precision):
    """Lattice atoms on the x = 0, y = 0 and z = 0 faces handed in as -0.0,
    -1e-18 (x + L rounds to L itself) and L: each wraps to exactly the
    generator's 0.0, so the state equals the generator's positions bit for
    bit and the oracle, given those positions only, bins and lists them the
    same way."""
    s = inputs.lj_fcc(nc=6, T=0.72)
    L = np.asarray(s.box)
    pos0 = np.array(s.pos)
    moved = pos0.copy()
    for d in range(3):
        at0 = np.flatnonzero(pos0[:, d] == 0.0)
        assert len(at0) >= 9
        moved[at0[0::3], d] = -0.0
        moved[at0[1::3], d] = -1e-18
        moved[at0[2::3], d] = L[d]
    with md.System(moved, s.vel, s.box, precision=precision) as a:
        p = a.state()[0].cpu().numpy()
        nc, cell_of, start = a.cells()
        off, ids = a.neighbors()
    assert np.all((p >= 0.0) & (p < L))
    assert np.array_equal(p, pos0)
    onc, ocell, ostart, _ = orc.bin_cells(pos0, L, 2.8)
    np.testing.assert_array_equal(cell_of.cpu().numpy(), ocell)
    np.testing.assert_array_equal(start.cpu().numpy(), ostart)
    ooff, oids = orc.neighbors_cells(pos0, L, 2.8)
    np.testing.assert_array_equal(off.cpu().numpy(), ooff)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_positions_outside_the_box_are_wrapped(md, orc, precision):
    """Inputs shifted by -2..2 box lengths per component: the system holds the
    wrapped positions, and cells, lists and forces are those of the oracle on
    them."""
    s = inputs.lj_fcc(nc=6, T=0.72)
    L = np.asarray(s.box)
    g = inputs.gaussian(inputs.SEED_BASE + 701, s.pos.size).reshape(-1, 3)
    pos0 = np.mod(s.pos + 0.05 * g, L)
    k = (inputs.splitmix64(inputs.SEED_BASE + 702, s.pos.size) % 5).astype(np.int64) - 2
    shifted = pos0 + k.reshape(-1, 3) * L
    with md.System(shifted, s.vel, s.box, precision=precision) as a:
        p, _, f = (t.cpu().numpy() for t in a.state())
        nc, cell_of, start = a.cells()
        off, ids = a.neighbors()
    assert np.all((p >= 0.0) & (p < L))
    d = p - pos0
    d -= L * np.round(d / L)
    assert np.max(np.abs(d)) < 1e-12
    onc, ocell, ostart, _ = orc.bin_cells(p, L, 2.8)
    assert list(onc) == nc
    np.testing.assert_array_equal(cell_of.cpu().numpy(), ocell)
    np.testing.assert_array_equal(start.cpu().numpy(), ostart)
    ooff, oids = orc.neighbors_cells(p, L, 2.8)
    np.testing.assert_array_equal(off.cpu().numpy(), ooff)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    prm = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    _, f0 = orc.forces_once(prm, p, L)
    check_forces(f, f0, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_atoms_on_cell_faces(md, orc, precision):
    """Simple-cubic sites at whole multiples of the cell width (2.9 > r_list),
    the body centres, and sites 1.07 from the corners along x: every
    coordinate of the first set, and y and z of the third, lie on a cell face,
    where the floor of x * n / L decides the cell.  Cells, lists and forces
    match the oracle's definition."""
    n, w = 4, 2.9
    g = np.arange(n) * w
    corners = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pos = np.concatenate([corners, corners + 0.5 * w, corners + np.array([0.37 * w, 0.0, 0.0])])
    box = np.full(3, n * w)
    vel = np.zeros_like(pos)
    with md.System(pos, vel, box, precision=precision) as a:
        nc, cell_of, start = a.cells()
        off, ids = a.neighbors()
        _, _, f = (t.cpu().numpy() for t in a.state())
    onc, ocell, ostart, _ = orc.bin_cells(pos, box, 2.8)
    assert list(onc) == nc == [n, n, n]
    np.testing.assert_array_equal(cell_of.cpu().numpy(), ocell)
    np.testing.assert_array_equal(start.cpu().numpy(), ostart)
    ooff, oids = orc.neighbors_cells(pos, box, 2.8)
    np.testing.assert_array_equal(off.cpu().numpy(), ooff)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    prm = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    _, f0 = orc.forces_once(prm, pos, box)
    check_forces(f, f0, precision)


def test_non_finite_state_is_reported(md):
    """A NaN coordinate gets cell index 0 in that dimension (the float64
    floor-convert of NaN is clamped into the grid), the atom meets no
    neighbour (every comparison with NaN is false), and the first drift
    reports MD_ERR_NONFINITE through the status word; the handle stays usable
    for inspection."""
    s = inputs.lj_fcc(nc=6, T=0.72)
    pos = s.pos.copy()
    pos[17, 1] = np.nan
    with md.System(pos, s.vel, s.box, precision="mixed") as a:
        with pytest.raises(md.MDError) as e:
            a.step(3)
        assert e.value.status == md.MD_ERR_NONFINITE
        assert a.stats()["status"] == md.MD_ERR_NONFINITE


def orthorhombic():
    """A 6 x 8 x 11 fcc block at rho* = 0.8442, perturbed: 3 x 4 x 6 cells
    whose widths differ between x, y (3.36) and z (3.08)."""
    a0 = (4.0 / 0.8442) ** (1.0 / 3.0)
    nc = (6, 8, 11)
    box = a0 * np.array(nc, dtype=np.float64)
    g = inputs.gaussian(inputs.SEED_BASE + 710, 3 * 4 * int(np.prod(nc))).reshape(-1, 3)
    pos = np.mod(inputs.fcc_lattice(nc, a0) + 0.05 * g, box)
    vel = inputs.maxwell_boltzmann(len(pos), 0.72, 1.0, inputs.SEED_BASE + 711)
    return pos, vel, box


@pytest.mark.parametrize("variant", ["full", "color", "atomic"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_orthorhombic_box(md, orc, precision, variant):
    """Different cell counts and widths per dimension: cells and lists
    bit-exact, forces within the bars, and 60 steps with rebuilds against the
    oracle's total energy (1e-6 relative on the fp64 path, 1e-4 mixed).  The
    half-list variants colour a 3 x 4 x 6 grid."""
    pos, vel, box = orthorhombic()
    code = {"full": md.MD_FORCE_FULL, "color": md.MD_FORCE_HALF_COLOR,
            "atomic": md.MD_FORCE_HALF_ATOMIC}[variant]
    with md.System(pos, vel, box, precision=precision, force_variant=code) as a:
        nc, cell_of, start = a.cells()
        off, ids = a.neighbors(half=variant != "full")
        f = a.state()[2].cpu().numpy()
        b0 = a.stats()["builds"]
        a.step(60)
        builds = a.stats()["builds"] - b0
        ke, pe = a.energy()
    onc, ocell, ostart, _ = orc.bin_cells(pos, box, 2.8)
    assert list(onc) == nc == [3, 4, 6]
    np.testing.assert_array_equal(cell_of.cpu().numpy(), ocell)
    np.testing.assert_array_equal(start.cpu().numpy(), ostart)
    ooff, oids = orc.neighbors_cells(pos, box, 2.8, half=variant != "full")
    np.testing.assert_array_equal(off.cpu().numpy(), ooff)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    prm = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    _, f0 = orc.forces_once(prm, pos, box)
    check_forces(f, f0, precision)
    assert builds >= 1
    E = orc.md_run(prm, pos, vel, box, 60)["energies"][-1, 2]
    tol = 1e-6 if precision == "fp64" else 1e-4
    assert abs(ke + pe - E) <= tol * abs(E), (ke + pe, E)


@pytest.mark.parametrize("variant", ["paired", "cluster"])
def test_orthorhombic_box_clustered_layouts(md, orc, variant):
    """The two clustered layouts (mixed path only) on the 3 x 4 x 6-cell
    orthorhombic box: exported rows bit-exact, forces within the mixed bars,
    and 60 steps with rebuilds against the oracle's total energy."""
    pos, vel, box = orthorhombic()
    code = {"paired": md.MD_FORCE_PAIRED, "cluster": md.MD_FORCE_CLUSTER}[variant]
    with md.System(pos, vel, box, precision="mixed", force_variant=code) as a:
        off, ids = a.neighbors()
        f = a.state()[2].cpu().numpy()
        b0 = a.stats()["builds"]
        a.step(60)
        builds = a.stats()["builds"] - b0
        ke, pe = a.energy()
    ooff, oids = orc.neighbors_cells(pos, box, 2.8)
    np.testing.assert_array_equal(off.cpu().numpy(), ooff)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    prm = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    _, f0 = orc.forces_once(prm, pos, box)
    check_forces(f, f0, "mixed", near_cutoff(pos, box, ooff, oids, 2.5, 1e-5))
    assert builds >= 1
    E = orc.md_run(prm, pos, vel, box, 60)["energies"][-1, 2]
    assert abs(ke + pe - E) <= 1e-4 * abs(E), (ke + pe, E)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sutton_chen_orthorhombic_box(md, orc, precision):
    """Sutton-Chen on a 7 x 8 x 9 fcc block (3 x 3 x 4 cells): densities and
    forces of both passes against the oracle."""
    s = inputs.sc_fcc(nc=7)
    p = s.params
    nc = (7, 8, 9)
    box = np.array(nc, dtype=np.float64)
    g = inputs.gaussian(inputs.SEED_BASE + 720, 3 * 4 * int(np.prod(nc))).reshape(-1, 3)
    pos = np.mod(inputs.fcc_lattice(nc, 1.0) + 0.03 * g, box)
    vel = np.zeros_like(pos)
    kw = dict(potential="sc", eps=p["eps"], sigma=p["sigma"], c=p["c"], n_exp=p["n_exp"],
              m_exp=p["m_exp"], rc=p["rc"], skin=p["skin"], dt=p["dt"])
    with md.System(pos, vel, box, precision=precision, **kw) as a:
        nc_gpu = a.cells()[0]
        f = a.state()[2].cpu().numpy()
        ke, pe = a.energy()
    prm = orc.make_params(potential=orc.POT_SC, eps=p["eps"], sigma=p["sigma"], c=p["c"],
                          n_exp=p["n_exp"], m_exp=p["m_exp"], rc=p["rc"], skin=p["skin"],
                          dt=p["dt"])
    U0, f0 = orc.forces_once(prm, pos, box)
    ooff, oids = orc.neighbors_cells(pos, box, 2.2)
    # the 8th fcc shell lies at r_c = 2a: jittered pairs straddle the cutoff
    delta = 1e-12 if precision == "fp64" else 1e-5
    bad = near_cutoff(pos, box, ooff, oids, 2.0, delta)
    assert nc_gpu == [3, 3, 4]
    check_forces(f, f0, precision, bad)
    tol = 1e-10 if precision == "fp64" else 2e-6
    # pairs within delta of r_c may fall on either side: at most their own energy
    slack = sc_straddle_bound(orc, pos, box, ooff, oids, delta, a=p["sigma"], c=p["c"],
                              n_exp=p["n_exp"], m_exp=p["m_exp"], rc=p["rc"], eps=p["eps"])
    assert abs(pe - U0) <= tol * abs(U0) + slack, (pe, U0, slack)


def test_batch_of_orthorhombic_and_shifted_boxes(md, orc):
    """One batch holding the orthorhombic block and an fcc crystal given with
    positions shifted by whole box lengths: per replica, cells and lists
    bit-exact and forces within the mixed bars."""
    pos1, vel1, box1 = orthorhombic()
    s = inputs.lj_fcc(nc=7, T=0.72)
    box2 = np.asarray(s.box)
    g = inputs.gaussian(inputs.SEED_BASE + 730, s.pos.size).reshape(-1, 3)
    pos2 = np.mod(s.pos + 0.05 * g, box2)
    k = (inputs.splitmix64(inputs.SEED_BASE + 731, s.pos.size) % 3).astype(np.int64) - 1
    reps = [(pos1, vel1, box1), (pos2 + k.reshape(-1, 3) * box2, s.vel, box2)]
    with md.Batch(reps, precision="mixed") as b:
        nc, cell_of, start = b.cells()
        off, ids = b.neighbors()
        p, _, f = (t.cpu().numpy() for t in b.state())
    cell_of, start, off, ids = (t.cpu().numpy() for t in (cell_of, start, off, ids))
    cell0 = 0
    prm = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    for r, (pos_r, box_r) in enumerate(((pos1, box1), (pos2, box2))):
        a0, a1 = b.offsets[r], b.offsets[r + 1]
        pr = p[a0:a1]
        d = pr - pos_r
        d -= box_r * np.round(d / box_r)
        assert np.max(np.abs(d)) < 1e-12
        onc, ocell, ostart, _ = orc.bin_cells(pr, box_r, 2.8)
        nr = int(np.prod(onc))
        np.testing.assert_array_equal(cell_of[a0:a1], ocell + cell0)
        np.testing.assert_array_equal(start[cell0:cell0 + nr + 1], ostart + a0)
        cell0 += nr
        ooff, oids = orc.neighbors_cells(pr, box_r, 2.8)
        np.testing.assert_array_equal(off[a0:a1 + 1] - off[a0], ooff)
        np.testing.assert_array_equal(ids[off[a0]:off[a1]], oids + a0)
        _, f0 = orc.forces_once(prm, pr, box_r)
        check_forces(f[a0:a1], f0, "mixed")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_non_unit_parameters_and_fixed_rebuild_interval(md, orc, precision):
    """eps 1.7, sigma 0.9, mass 2.5 and a list rebuilt every 7 steps (the
    paper's fixed interval) instead of the half-skin rule: forces at the
    start and the total energy after 50 steps against the oracle."""
    eps, sig, mass = 1.7, 0.9, 2.5
    s = inputs.lj_fcc(nc=6, T=0.72)
    box = np.asarray(s.box) * sig
    g = inputs.gaussian(inputs.SEED_BASE + 740, s.pos.size).reshape(-1, 3)
    pos = np.mod(s.pos * sig + 0.04 * g, box)
    vel = inputs.maxwell_boltzmann(len(pos), 0.72 * eps, mass, inputs.SEED_BASE + 741)
    kw = dict(eps=eps, sigma=sig, rc=2.5 * sig, skin=0.3 * sig, dt=0.004, mass=mass,
              rebuild_every=7)
    with md.System(pos, vel, box, precision=precision, **kw) as a:
        f = a.state()[2].cpu().numpy()
        b0 = a.stats()["builds"]
        a.step(50)
        builds = a.stats()["builds"] - b0
        ke, pe = a.energy()
    prm = orc.make_params(potential=orc.POT_LJ, **kw)
    _, f0 = orc.forces_once(prm, pos, box)
    check_forces(f, f0, precision)
    assert builds == 50 // 7
    E = orc.md_run(prm, pos, vel, box, 50)["energies"][-1, 2]
    tol = 1e-6 if precision == "fp64" else 1e-4
    assert abs(ke + pe - E) <= tol * abs(E), (ke + pe, E)
