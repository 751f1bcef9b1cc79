"""The inner/outer split of the force pass (Sec. 2.1's seven-step algorithm
for domain decomposition, on one GPU): intra-domain forces while the boundary
atoms' positions are exchanged on a second stream, then inter-domain forces
from the received copy.  Forces and energies against the oracle with the
mixed-path bars, 100-step NVE against the oracle's trajectory, the same steps
under graph replay, and the split's own bookkeeping."""
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


def porous():
    s = inputs.lj_porous(nc=14, fraction=0.35, rmin=2.0, rmax=4.0)
    g = inputs.gaussian(inputs.SEED_BASE + 990, s.pos.size).reshape(-1, 3)
    return s, np.mod(s.pos + 0.05 * g, s.box)


@pytest.mark.parametrize("dd", [(2, 2, 2), (3, 1, 2), (8, 8, 8)])
def test_split_forces_match_oracle(md, orc, dd):
    s, pos = porous()  # 8 cells per side: (8, 8, 8) makes every cell a domain
    off, ids = orc.neighbors_cells(pos, s.box, 2.8)
    U0, f0 = orc.lj_list(pos, s.box, off, ids)
    with md.System(pos, s.vel, s.box, precision="mixed") as sy:
        ref = sy.state()[2].cpu().numpy()
        md.md_set_decomposition(sy.h, *dd)
        md.md_forces(sy.h)
        f = sy.state()[2].cpu().numpy()
        ke, pe = sy.energy()
        md.md_set_decomposition(sy.h, 1, 1, 1)
        ke1, pe1 = sy.energy()
    fn = np.linalg.norm(f0, axis=1)
    rms = math.sqrt(np.mean(fn * fn))
    for g in (f, ref):
        err = np.linalg.norm(g - f0, axis=1)
        assert np.all(err <= 2e-4 * fn + 1e-5 * max(1.0, rms))
    # the split only reorders float32 partial sums
    assert np.max(np.abs(f - ref)) <= 1e-5 * max(1.0, rms)
    assert abs(pe - U0) <= 2e-6 * abs(U0) and abs(pe - pe1) <= 2e-6 * abs(U0)


@pytest.mark.parametrize("stream", ["default", "side"])
def test_split_steps_track_the_oracle(md, orc, stream):
    """100 steps of config 1 (4,000-atom fcc, T* 0.72) with 2 x 2 x 2 domains:
    total energy after every step within 1e-6 relative of the oracle's
    trajectory; on a side stream the steps replay captured graphs that hold
    both streams, and end where the plain launches end."""
    s = inputs.lj_fcc(nc=10, T=0.72)
    p = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=0.005)
    E0 = orc.md_run(p, s.pos, s.vel, s.box, 100)["energies"]
    st = torch.cuda.default_stream() if stream == "default" else torch.cuda.Stream()
    with torch.cuda.stream(st), md.System(s.pos, s.vel, s.box, precision="mixed",
                                          stream=None if stream == "default" else st) as sy:
        md.md_set_decomposition(sy.h, 2, 2, 2)
        es = [sy.energy()]
        for _ in range(10):
            sy.step(10)
            es.append(sy.energy())
        state = sy.state()
    es = np.array(es)
    rel = np.abs(es[:, 0] + es[:, 1] - E0[::10, 2]) / np.abs(E0[::10, 2])
    print("inner/outer split: max relative total-energy error %.3g" % rel.max())
    assert rel.max() < 1e-6, rel.max()
    if stream == "side":
        with md.System(s.pos, s.vel, s.box, precision="mixed") as sy:
            md.md_set_decomposition(sy.h, 2, 2, 2)
            sy.energy()
            for _ in range(10):
                sy.step(10)
                sy.energy()
            plain = sy.state()
        for x, y in zip(state, plain):
            assert torch.equal(x, y)


def test_split_rejects_what_it_does_not_cover(md):
    s = inputs.lj_fcc(nc=6, T=0.72)
    with md.System(s.pos, s.vel, s.box, precision="fp64") as sy:
        with pytest.raises(md.MDError):
            md.md_set_decomposition(sy.h, 2, 1, 1)
    with md.System(s.pos, s.vel, s.box, precision="mixed") as sy:
        with pytest.raises(md.MDError):
            md.md_set_decomposition(sy.h, 4, 1, 1)  # 3 cells per side
        md.md_set_decomposition(sy.h, 3, 3, 3)
        with pytest.raises(md.MDError):
            md.md_set_variant(sy.h, md.MD_FORCE_HALF_ATOMIC, md.MD_SCHED_GRID)
        sy.step(5)
