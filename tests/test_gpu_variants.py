"""Newton's-third-law strategies (full list, half list + cell colouring, half
list + float64 atomics) against the oracle and against each other."""
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


def perturbed(s, amp, seed):
    g = inputs.gaussian(seed, s.pos.size).reshape(-1, 3)
    return np.mod(s.pos + amp * g, s.box)


def systems():
    a = inputs.lj_fcc(nc=10, T=0.72)
    b = inputs.lj_porous(nc=13, fraction=0.4, rmin=2.0, rmax=5.0)   # 4 cells + tail colours
    return {"fcc4000": (a, perturbed(a, 0.05, 701)), "porous13": (b, perturbed(b, 0.05, 702))}


def variant_code(md, name):
    return {"color": md.MD_FORCE_HALF_COLOR, "atomic": md.MD_FORCE_HALF_ATOMIC}[name]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("variant", ["color", "atomic"])
@pytest.mark.parametrize("sysname", ["fcc4000", "porous13"])
def test_half_variants_match_oracle(md, orc, variant, sysname, precision):
    s, pos = systems()[sysname]
    off, ids = orc.neighbors_cells(pos, s.box, 2.8)
    U0, f0 = orc.lj_list(pos, s.box, off, ids)
    rows = np.repeat(np.arange(len(pos)), np.diff(off))
    d = pos[ids] - pos[rows]
    d -= s.box * np.round(d / s.box)
    r = np.sqrt((d * d).sum(1))
    bad = np.zeros(len(pos), bool)
    bad[rows[np.abs(r - 2.5) < (1e-5 if precision == "mixed" else 1e-12)]] = True
    with md.System(pos, s.vel, s.box, precision=precision,
                   force_variant=variant_code(md, variant)) as sy:
        _, _, f = sy.state()
        ke, pe = sy.energy()
        hoff, hids = sy.neighbors(half=True)
        with pytest.raises(md.MDError):
            sy.neighbors(half=False)     # a half list cannot export the full set
    f = f.cpu().numpy()
    fn = np.linalg.norm(f0, axis=1)
    rms = math.sqrt(np.mean(fn * fn))
    err = np.linalg.norm(f - f0, axis=1)
    if precision == "mixed":
        assert np.all((err <= 2e-4 * fn + 1e-5 * max(1.0, rms)) | bad)
        assert abs(pe - U0) <= 2e-6 * abs(U0)
    else:
        assert np.all((err <= 1e-5 * fn + 1e-9 * rms) | bad)
        assert abs(pe - U0) <= 1e-10 * abs(U0)
    ho, hi = orc.neighbors_cells(pos, s.box, 2.8, half=True)
    np.testing.assert_array_equal(hoff.cpu().numpy(), ho)
    np.testing.assert_array_equal(hids.cpu().numpy(), hi)


def test_variants_agree_over_a_trajectory(md):
    s, pos = systems()["porous13"]
    out = {}
    for name, code in (("full", md.MD_FORCE_FULL), ("color", md.MD_FORCE_HALF_COLOR),
                       ("atomic", md.MD_FORCE_HALF_ATOMIC)):
        with md.System(pos, s.vel, s.box, precision="mixed", force_variant=code) as a:
            a.step(50)
            out[name] = [t.cpu().numpy() for t in a.state()]
            out[name].append(sum(a.energy()))
    for name in ("color", "atomic"):
        dp = out[name][0] - out["full"][0]
        dp -= s.box * np.round(dp / s.box)
        assert np.max(np.abs(dp)) < 1e-5, name
        assert abs(out[name][3] - out["full"][3]) < 1e-5 * abs(out["full"][3])


def test_switch_variant_rebuilds_list(md):
    s, pos = systems()["fcc4000"]
    with md.System(pos, s.vel, s.box, precision="mixed") as a:
        off_full, _ = a.neighbors()
        md.md_set_variant(a.h, md.MD_FORCE_HALF_COLOR, md.MD_SCHED_GRID)
        off_half, _ = a.neighbors(half=True)
        assert off_half[-1].item() * 2 == off_full[-1].item()
        md.md_set_variant(a.h, md.MD_FORCE_FULL, md.MD_SCHED_GRID)
        off2, _ = a.neighbors()
        assert torch.equal(off2, off_full)


@pytest.mark.parametrize("variant", ["color", "atomic"])
def test_switch_variant_under_graph_replay(md, orc, variant):
    """On a non-default stream the step replays captured graphs; switching to
    a half list must drop them, or a stale full-list force kernel would run on
    the half list.  After the switch and 30 more steps the energy stays
    within 1e-4 of the oracle's own trajectory; then a second generator state
    loaded into the running system gets the oracle's forces."""
    s, pos = systems()["fcc4000"]
    p = perturbed(s, 0.05, 703)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        with md.System(pos, s.vel, s.box, precision="mixed", stream=st) as a:
            a.step(30)                      # graphs captured and replayed
            md.md_set_variant(a.h, variant_code(md, variant), md.MD_SCHED_GRID)
            a.step(30)
            ke, pe = a.energy()
            md.md_set_state(a.h, torch.as_tensor(p, device="cuda"), None)
            md.md_forces(a.h)
            f = a.state()[2].cpu().numpy()
    prm = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    _, f0 = orc.forces_once(prm, p, s.box)
    fn = np.linalg.norm(f0, axis=1)
    rms = math.sqrt(np.mean(fn * fn))
    err = np.linalg.norm(f - f0, axis=1)
    off, ids = orc.neighbors_cells(p, s.box, 2.8)
    rows = np.repeat(np.arange(len(p)), np.diff(off))
    d = p[ids] - p[rows]
    d -= s.box * np.round(d / s.box)
    r = np.sqrt((d * d).sum(1))
    bad = np.zeros(len(p), bool)
    bad[rows[np.abs(r - 2.5) < 1e-5]] = True
    assert np.all((err <= 2e-4 * fn + 1e-5 * max(1.0, rms)) | bad)
    E = orc.md_run(prm, pos, s.vel, s.box, 60)["energies"][-1, 2]
    assert abs(ke + pe - E) < 1e-4 * abs(E), (ke + pe, E)


@pytest.mark.parametrize("variant", ["color", "atomic"])
def test_half_lists_fp64_nve_config1(md, orc, variant):
    """The float64 half-list passes on config 1 (4,000-atom fcc, T* 0.72):
    total energy after every tenth of 100 steps within 1e-6 relative of the
    oracle's trajectory, with the list rebuilt on the way."""
    s = inputs.lj_fcc(nc=10, T=0.72)
    p = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    E0 = orc.md_run(p, s.pos, s.vel, s.box, 100)["energies"]
    with md.System(s.pos, s.vel, s.box, precision="fp64",
                   force_variant=variant_code(md, variant)) as sy:
        es = [sy.energy()]
        for _ in range(10):
            sy.step(10)
            es.append(sy.energy())
        builds = sy.stats()["builds"]
    es = np.array(es)
    rel = np.abs(es[:, 0] + es[:, 1] - E0[::10, 2]) / np.abs(E0[::10, 2])
    print("fp64 half list (%s): max relative total-energy error %.3g, %d builds"
          % (variant, rel.max(), builds))
    assert rel.max() < 1e-6, rel.max()
    assert builds > 2
