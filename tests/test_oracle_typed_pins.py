"""Pins of the oracle's multi-element Lennard-Jones routines (the Cu-Au
alloy and layer systems of Sec. 3.1, per-pair parameters of Sec. 2.2's pair
loop): a dimer of unlike species at its force zero, equality with the
one-species routines when every atom has one species, brute force against the
list, finite differences, per-species masses in the integrator (momentum
sum m v conserved, energy conserved) and the sampled-atom routine.  CPU only."""
import math

import numpy as np
import pytest

from paper_1611_00075_gb300 import inputs


def tp(s):
    p = s.params
    return p["types"], p["t_eps"], p["t_sigma"], p["t_mass"]


def test_unlike_dimer_at_its_force_zero(orc):
    e, sg = inputs.mixing_rules((1.0, 1.12), (1.0, 1.128))
    assert e[0, 1] == pytest.approx(math.sqrt(1.12)) and sg[0, 1] == pytest.approx(1.064)
    r = sg[0, 1] * 2 ** (1 / 6)  # the minimum of 4 eps [(s/r)^12 - (s/r)^6]
    pos = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
    box = np.array([20.0, 20.0, 20.0])
    U, f = orc.lj_typed_brute(pos, box, [0, 1], e, sg, 2.5)
    sr6 = (sg[0, 1] / 2.5) ** 6
    assert U == pytest.approx(-e[0, 1] - 4 * e[0, 1] * (sr6 * sr6 - sr6), rel=1e-14)
    assert np.max(np.abs(f)) < 1e-13


def test_one_species_equals_plain_lj(orc):
    s = inputs.lj_fcc(nc=5)
    pos = np.mod(s.pos + 0.06 * inputs.gaussian(971, s.pos.size).reshape(-1, 3), s.box)
    off, ids = orc.neighbors_cells(pos, s.box, 2.8)
    U0, f0, e0 = orc.lj_list(pos, s.box, off, ids, per_atom=True)
    types = np.zeros(len(pos), np.int32)
    U1, f1, e1 = orc.lj_typed_list(pos, s.box, off, ids, types, [[1.0]], [[1.0]], 2.5)
    np.testing.assert_array_equal(f1, f0)
    np.testing.assert_array_equal(e1, e0)


@pytest.mark.parametrize("which", ["alloy", "layer"])
def test_list_equals_brute_force_and_gradient(orc, which):
    s = inputs.lj_alloy(nc=4) if which == "alloy" else inputs.lj_layer(nc=6, slab=2)
    types, te, ts, tm = tp(s)
    pos = np.mod(s.pos + 0.05 * inputs.gaussian(972, s.pos.size).reshape(-1, 3), s.box)
    off, ids = orc.neighbors_cells(pos, s.box, 2.8)
    U1, f1, _ = orc.lj_typed_list(pos, s.box, off, ids, types, te, ts)
    U2, f2 = orc.lj_typed_brute(pos, s.box, types, te, ts)
    np.testing.assert_allclose(f1, f2, rtol=1e-11, atol=1e-11)
    assert U1 == pytest.approx(U2, rel=1e-12)
    assert np.max(np.abs(f2.sum(axis=0))) < 1e-9
    h = 1e-6
    for i in (0, 33, 150):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            up = orc.lj_typed_brute(pp, s.box, types, te, ts)[0]
            um = orc.lj_typed_brute(pm, s.box, types, te, ts)[0]
            assert f2[i, d] == pytest.approx(-(up - um) / (2 * h), rel=1e-6, abs=1e-7)


def test_md_with_species_masses(orc):
    s = inputs.lj_alloy(nc=6, T=0.3)
    types, te, ts, tm = tp(s)
    prm = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, dt=s.params["dt"],
                          types=types, t_eps=te, t_sigma=ts, t_mass=tm)
    out = orc.md_run(prm, s.pos, s.vel, s.box, 400)
    m = tm[types][:, None]
    E = out["energies"]
    assert E[0, 0] == pytest.approx(0.5 * np.sum(m * s.vel ** 2), rel=1e-13)
    assert np.max(np.abs(E[:, 2] - E[0, 2])) < 1e-5 * abs(E[0, 2])
    assert np.max(np.abs((m * out["vel"]).sum(axis=0))) < 1e-10
    assert out["builds"] >= 2


def test_forces_sample_equals_all_atom(orc):
    s = inputs.lj_layer(nc=8, slab=2)
    types, te, ts, tm = tp(s)
    pos = np.mod(s.pos + 0.05 * inputs.gaussian(973, s.pos.size).reshape(-1, 3), s.box)
    prm = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3, types=types, t_eps=te,
                          t_sigma=ts, t_mass=tm)
    off, ids = orc.neighbors_cells(pos, s.box, 2.8)
    _, f, e = orc.lj_typed_list(pos, s.box, off, ids, types, te, ts)
    idx = np.arange(0, s.n, 23, dtype=np.int64)
    fs, es = orc.forces_sample(prm, pos, s.box, idx)
    np.testing.assert_array_equal(fs, f[idx])
    np.testing.assert_array_equal(es, e[idx])
