"""The multi-element Lennard-Jones path (the Cu-Au Alloy and Layer systems of
Sec. 3.1; per-pair parameters of Sec. 2.2's pair loop) against the oracle,
element by element, through the C ABI: cells and lists bit-exact, forces and
energies within the bars of test_gpu_parity.py, 100-step NVE trajectories
with species masses, one-species equality with the plain kernels, and the
argument checks of md_create_typed."""
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


def species(s):
    p = s.params
    return p["types"], p["t_eps"], p["t_sigma"], p["t_mass"]


def system(which, amp=0.04, seed=981):
    s = inputs.lj_alloy(nc=8) if which == "alloy" else inputs.lj_layer(nc=8, slab=2)
    g = inputs.gaussian(seed, s.pos.size).reshape(-1, 3)
    return s, np.mod(s.pos + amp * g, s.box)


def kw(s):
    p = s.params
    return dict(rc=p["rc"], skin=p["skin"], dt=p["dt"])


def near_cutoff(pos, box, off, ids, rc, delta):
    rows = np.repeat(np.arange(len(pos)), np.diff(off))
    d = pos[ids] - pos[rows]
    d -= box * np.round(d / box)
    r = np.sqrt(np.sum(d * d, axis=1))
    bad = np.zeros(len(pos), bool)
    bad[rows[np.abs(r - rc) < delta]] = True
    return bad


# (precision, layout): the float64 path with per-atom lists; the mixed path
# with per-atom lists and with two atoms per thread (a slot's two atoms may
# be of different species)
MODES = [("fp64", "full"), ("mixed", "full"), ("mixed", "paired")]


def variant(md, layout):
    return md.MD_FORCE_PAIRED if layout == "paired" else md.MD_FORCE_FULL


@pytest.mark.parametrize("which", ["alloy", "layer"])
@pytest.mark.parametrize("precision,layout", MODES)
def test_typed_cells_lists_forces_energy(md, orc, which, precision, layout):
    s, pos = system(which)
    types, te, ts, tm = species(s)
    with md.System(pos, s.vel, s.box, precision=precision, species=species(s),
                   force_variant=variant(md, layout), **kw(s)) as sy:
        nc, cell_of, start = sy.cells()
        off, ids = sy.neighbors()
        f = sy.state()[2].cpu().numpy()
        ke, pe = sy.energy()
    onc, ocell, ostart, _ = orc.bin_cells(pos, s.box, 2.8)
    np.testing.assert_array_equal(cell_of.cpu().numpy(), ocell)
    np.testing.assert_array_equal(start.cpu().numpy(), ostart)
    ooff, oids = orc.neighbors_cells(pos, s.box, 2.8)
    np.testing.assert_array_equal(off.cpu().numpy(), ooff)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    U0, f0, _ = orc.lj_typed_list(pos, s.box, ooff, oids, types, te, ts)
    delta = 1e-12 if precision == "fp64" else 1e-5
    bad = near_cutoff(pos, s.box, ooff, oids, 2.5, delta)
    fn = np.linalg.norm(f0, axis=1)
    rms = math.sqrt(np.mean(fn * fn))
    err = np.linalg.norm(f - f0, axis=1)
    tol = (1e-5 * fn + 1e-9 * rms) if precision == "fp64" else (2e-4 * fn + 1e-5 * max(1.0, rms))
    assert np.all((err <= tol) | bad), int(((err > tol) & ~bad).sum())
    # straddling pairs: at most their own (shifted, so tiny) energy; the largest
    # eps and sigma bound every species pair's slope at r_c
    slack = lj_straddle_bound(orc, pos, s.box, ooff, oids, 2.5, delta, eps=te.max(),
                              sigma=ts.max())
    etol = 1e-10 if precision == "fp64" else 2e-6
    assert abs(pe - U0) <= etol * abs(U0) + slack, (pe, U0)
    ke0 = 0.5 * np.sum(tm[types][:, None] * s.vel ** 2)
    assert abs(ke - ke0) <= 1e-12 * ke0


@pytest.mark.parametrize("precision,layout", MODES)
def test_typed_nve_100_steps(md, orc, precision, layout):
    """A 6^3-cell random alloy at T* 0.3 (dt 0.002): total energy after every
    one of 100 steps within 1e-6 relative of the oracle's trajectory, with
    the species' masses in both integrators."""
    s = inputs.lj_alloy(nc=6, T=0.3)
    types, te, ts, tm = species(s)
    prm = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=s.params["dt"], types=types,
                          t_eps=te, t_sigma=ts, t_mass=tm)
    E0 = orc.md_run(prm, s.pos, s.vel, s.box, 100)["energies"]
    with md.System(s.pos, s.vel, s.box, precision=precision, species=species(s),
                   force_variant=variant(md, layout), **kw(s)) as sy:
        es = [sy.energy()]
        for _ in range(100):
            sy.step(1)
            es.append(sy.energy())
    es = np.array(es)
    rel = np.abs(es[:, 0] + es[:, 1] - E0[:, 2]) / np.abs(E0[:, 2])
    print("alloy %s %s: max relative total-energy error over 100 steps %.3g"
          % (precision, layout, rel.max()))
    assert rel.max() < 1e-6, rel.max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_one_species_equals_plain_kernels(md, precision):
    """Every atom of species 0 with the plain parameters: the species path
    gives the plain path's forces bit for bit (same arithmetic per pair) and
    the same 40 steps."""
    s = inputs.lj_fcc(nc=6, T=0.72)
    pos = np.mod(s.pos + 0.04 * inputs.gaussian(982, s.pos.size).reshape(-1, 3), s.box)
    sp = (np.zeros(s.n, np.int32), [[1.0]], [[1.0]], [1.0])
    out = []
    for spec in (None, sp):
        with md.System(pos, s.vel, s.box, precision=precision, species=spec) as sy:
            f0 = sy.state()[2]
            sy.step(40)
            out.append((f0,) + sy.state())
    for x, y in zip(out[0], out[1]):
        assert torch.equal(x, y)


def test_typed_rejects_bad_input(md):
    s = inputs.lj_alloy(nc=6)
    types, te, ts, tm = species(s)
    pos = torch.as_tensor(s.pos, device="cuda")
    prm = md.make_params(rc=2.5, skin=0.3, dt=0.002)
    bad_types = torch.as_tensor(np.where(types > 0, 2, 0).astype(np.int32), device="cuda")
    with pytest.raises(md.MDError) as e:
        md.md_create_typed(prm, md.make_lj_types(te, ts, tm), bad_types, pos, None, s.box)
    assert e.value.status == md.MD_ERR_INVALID and "species" in str(e.value)
    asym = np.array(te)
    asym[0, 1] *= 1.01
    t_ok = torch.as_tensor(types, device="cuda")
    with pytest.raises(md.MDError) as e:
        md.md_create_typed(prm, md.make_lj_types(asym, ts, tm), t_ok, pos, None, s.box)
    assert "symmetric" in str(e.value)
    with pytest.raises(md.MDError):
        md.md_create_typed(md.make_params(rc=2.5, skin=0.3, dt=0.002,
                                          scheduler=md.MD_SCHED_PAIRCOUNT),
                           md.make_lj_types(te, ts, tm), t_ok, pos, None, s.box)
    with md.System(s.pos, s.vel, s.box, species=species(s), **kw(s)) as sy:
        with pytest.raises(md.MDError):
            md.md_set_variant(sy.h, md.MD_FORCE_HALF_COLOR, md.MD_SCHED_GRID)
        with pytest.raises(md.MDError):  # two atoms per thread: the grid launch only
            md.md_set_variant(sy.h, md.MD_FORCE_PAIRED, md.MD_SCHED_MLP)
        md.md_set_variant(sy.h, md.MD_FORCE_PAIRED, md.MD_SCHED_GRID)
        sy.step(3)
        md.md_set_variant(sy.h, md.MD_FORCE_FULL, md.MD_SCHED_GRID)
        with pytest.raises(md.MDError):
            md.md_cost_model(sy.h, md.MD_COST_SAMPLE)
        sy.step(3)
