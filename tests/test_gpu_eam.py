"""The piecewise embedded-atom path (the paper's Fe form, Sec. 3.1, Eq. 1-2)
against the oracle, element by element, through the C ABI: lists, rho_i,
F'(rho_i), forces and energies on bcc systems, 100-step NVE trajectories,
and the argument checks of md_create_eam.

Bars as in test_gpu_parity.py: fp64 forces 1e-5 |f| + 1e-9 rms, mixed
2e-4 |f| + 1e-5 max(1, rms); rho 1e-12 (fp64) and 2e-6 (mixed) relative;
energies 1e-10 (fp64) and 2e-6 (mixed) relative per evaluation, 1e-6 per
step over 100 steps.  Every piece vanishes at its knot and every knot lies
at or below r_c, so a pair that rounding moves across r_c changes nothing:
no atom is set aside."""
import math

import numpy as np
import pytest

from paper_1611_00075_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

P = inputs.EAM_FE_LIKE
# a second table: a density function of two pieces and a quadratic embedding term
P2 = dict(P, psi_r=(1.8, 1.2), psi_a=(1.0, 0.7), F_quad=0.01)


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


def tables(orc, md, p):
    keys = ("phi_r", "phi_a", "psi_r", "psi_a", "F_sqrt", "F_quad")
    return orc.make_eam(*[p[k] for k in keys]), md.make_eam(*[p[k] for k in keys])


def system(nc=8, amp=0.05, seed=961):
    s = inputs.eam_bcc(nc=nc)
    g = inputs.gaussian(seed, s.pos.size).reshape(-1, 3)
    return s, np.mod(s.pos + amp * g, s.box)


def kw(p):
    return dict(rc=p["rc"], skin=p["skin"], dt=p["dt"], mass=p["mass"])


def check_forces(f, f0, precision):
    fn = np.linalg.norm(f0, axis=1)
    rms = math.sqrt(np.mean(fn * fn))
    err = np.linalg.norm(f - f0, axis=1)
    if precision == "fp64":
        tol = 1e-5 * fn + 1e-9 * rms
    else:
        tol = 2e-4 * fn + 1e-5 * max(1.0, rms)
    assert np.all(err <= tol), (precision, int((err > tol).sum()), float(np.max(err / np.maximum(fn, rms))))


# (precision, layout): the float64 path with per-atom lists; the mixed path
# with per-atom lists and with two atoms per thread (union lists of slots)
MODES = [("fp64", "full"), ("mixed", "full"), ("mixed", "paired")]


def variant(md, layout):
    return md.MD_FORCE_PAIRED if layout == "paired" else md.MD_FORCE_FULL


@pytest.mark.parametrize("table", ["fe_like", "two_psi_pieces"])
@pytest.mark.parametrize("precision,layout", MODES)
def test_eam_lists_density_forces_energy(md, orc, precision, layout, table):
    p = P if table == "fe_like" else P2
    t_orc, t_md = tables(orc, md, p)
    s, pos = system()
    rl = p["rc"] + p["skin"]
    off, ids = orc.neighbors_cells(pos, s.box, rl)
    U0, f0, rho0, dF0, e0 = orc.eam_list(pos, s.box, off, ids, t_orc, p["rc"])
    with md.System(pos, s.vel, s.box, precision=precision, eam=t_md,
                   force_variant=variant(md, layout), **kw(p)) as sy:
        goff, gids = sy.neighbors()
        f = sy.state()[2].cpu().numpy()
        rho = torch.empty(s.n, dtype=torch.float64, device="cuda")
        dF = torch.empty_like(rho)
        md.md_get_density(sy.h, rho, dF)
        ke, pe = sy.energy()
        e = torch.empty(s.n, dtype=torch.float64, device="cuda")
        md.md_get_atom_energy(sy.h, e)
    np.testing.assert_array_equal(goff.cpu().numpy(), off)
    np.testing.assert_array_equal(gids.cpu().numpy(), ids)
    rtol = 1e-12 if precision == "fp64" else 2e-6
    np.testing.assert_allclose(rho.cpu().numpy(), rho0, rtol=rtol)
    # F'(rho) = -A / (2 sqrt(rho)) + 2 B rho: its two terms partly cancel, so the
    # bar is relative to the terms' sizes (rho's own error, carried through)
    scale = p["F_sqrt"] / (2 * np.sqrt(rho0)) + 2 * abs(p["F_quad"]) * rho0
    assert np.all(np.abs(dF.cpu().numpy() - dF0) <= rtol * scale)
    check_forces(f, f0, precision)
    tol = 1e-10 if precision == "fp64" else 2e-6
    assert abs(pe - U0) <= tol * abs(U0), (pe, U0)
    np.testing.assert_allclose(e.cpu().numpy(), e0, rtol=1e-9 if precision == "fp64" else 1e-5,
                               atol=1e-12 if precision == "fp64" else 1e-5)
    assert abs(ke - 0.5 * np.sum(s.vel ** 2)) <= 1e-12 * ke


@pytest.mark.parametrize("precision,layout", MODES)
def test_eam_nve_100_steps(md, orc, precision, layout):
    """Fe-like bcc, 8^3 cells at T* = 0.018 (dt 0.002): total energy after
    every one of 100 steps within 1e-6 relative of the oracle's float64
    trajectory."""
    t_orc, t_md = tables(orc, md, P)
    s = inputs.eam_bcc(nc=8)
    prm = orc.make_params(potential=orc.POT_EAM, rc=P["rc"], skin=P["skin"], dt=P["dt"],
                          eam=t_orc)
    E0 = orc.md_run(prm, s.pos, s.vel, s.box, 100)["energies"]
    with md.System(s.pos, s.vel, s.box, precision=precision, eam=t_md,
                   force_variant=variant(md, layout), **kw(P)) as sy:
        es = [sy.energy()]
        for _ in range(100):
            sy.step(1)
            es.append(sy.energy())
    es = np.array(es)
    rel = np.abs(es[:, 0] + es[:, 1] - E0[:, 2]) / np.abs(E0[:, 2])
    print("EAM %s %s: max relative total-energy error over 100 steps %.3g"
          % (precision, layout, rel.max()))
    assert rel.max() < 1e-6, rel.max()


@pytest.mark.parametrize("layout", ["full", "paired"])
def test_eam_steps_with_rebuilds_against_the_oracle(md, orc, layout):
    """A hotter bcc box (T* 0.2) rebuilds its list several times in 300
    mixed-precision steps; the energy stays on the oracle's trajectory and
    the graph-replayed run on a side stream equals the plain one bit for bit."""
    t_orc, t_md = tables(orc, md, P2)
    s = inputs.eam_bcc(nc=8, T=0.2)
    prm = orc.make_params(potential=orc.POT_EAM, rc=P2["rc"], skin=P2["skin"], dt=P2["dt"],
                          eam=t_orc)
    ref = orc.md_run(prm, s.pos, s.vel, s.box, 300)
    out = []
    for stream in (None, torch.cuda.Stream()):
        ctx = torch.cuda.stream(stream) if stream is not None else torch.cuda.stream(
            torch.cuda.default_stream())
        with ctx, md.System(s.pos, s.vel, s.box, precision="mixed", eam=t_md, stream=stream,
                            force_variant=variant(md, layout), **kw(P2)) as sy:
            b0 = sy.stats()["builds"]
            sy.step(300)
            builds = sy.stats()["builds"] - b0
            ke, pe = sy.energy()
            out.append(sy.state())
    assert builds >= 2 and ref["builds"] >= 3
    # after 300 steps of a hot system the two trajectories have separated; the
    # energy difference is bounded by the integrator's own fluctuation, taken
    # from the oracle's run (max - min of its total energy), plus the 1e-6 bar
    Es = ref["energies"][:, 2]
    E = Es[-1]
    assert abs(ke + pe - E) <= 2.0 * (Es.max() - Es.min()) + 1e-6 * abs(E), (ke + pe, E)
    for x, y in zip(out[0], out[1]):
        assert torch.equal(x, y)


def test_eam_rejects_bad_tables(md):
    s = inputs.eam_bcc(nc=6)
    good = md.make_eam(P["phi_r"], P["phi_a"], P["psi_r"], P["psi_a"], P["F_sqrt"], P["F_quad"])
    beyond = md.make_eam(P["phi_r"][:-1] + (1.9,), P["phi_a"], P["psi_r"], P["psi_a"],
                         P["F_sqrt"], P["F_quad"])
    pos = torch.as_tensor(s.pos, device="cuda")
    with pytest.raises(md.MDError) as e:
        md.md_create_eam(md.make_params(potential="eam", **kw(P)), beyond, pos, None, s.box)
    assert e.value.status == md.MD_ERR_INVALID and "knot" in str(e.value)
    with pytest.raises(md.MDError) as e:
        md.md_create(md.make_params(potential="eam", **kw(P)), pos, None, s.box)
    assert e.value.status == md.MD_ERR_INVALID
    with pytest.raises(md.MDError) as e:
        md.md_create_eam(md.make_params(potential="eam", scheduler=md.MD_SCHED_PAIRCOUNT,
                                        **kw(P)), good, pos, None, s.box)
    assert e.value.status == md.MD_ERR_INVALID
    with md.System(s.pos, None, s.box, eam=good, **kw(P)) as sy:
        with pytest.raises(md.MDError):
            md.md_set_variant(sy.h, md.MD_FORCE_HALF_ATOMIC, md.MD_SCHED_GRID)
        sy.step(2)  # still usable
