"""Pins of the oracle's piecewise embedded-atom routines (the Fe form of
Sec. 3.1: pair and density functions that are sums of truncated cubics,
F(rho) = -A sqrt(rho) + B rho^2, evaluated in the three steps of Eq. 1-2):
a hand-computed dimer, the closed-form bcc lattice sum over shells found by
integer search, brute force against the list, finite-difference forces (a
dropped (F'_i + F'_j) term or a wrong sign fails them), conservation laws,
and the sampled-atom routine against the all-atom one.  CPU only."""
import itertools
import math

import numpy as np
import pytest

from paper_1611_00075_gb300 import inputs

P = inputs.EAM_FE_LIKE


def table(orc, **over):
    p = dict(P)
    p.update(over)
    return orc.make_eam(p["phi_r"], p["phi_a"], p["psi_r"], p["psi_a"], p["F_sqrt"], p["F_quad"])


def test_dimer_by_hand(orc):
    # one knot each: Phi = 2 (1 - r)^3, psi = (1 - r)^3, F = -3 sqrt(rho) + 0.5 rho^2
    t = orc.make_eam([1.0], [2.0], [1.0], [1.0], 3.0, 0.5)
    box = np.array([10.0, 10.0, 10.0])
    pos = np.array([[1.0, 1.0, 1.0], [1.5, 1.0, 1.0]])  # r = 0.5
    U, f, rho = orc.eam_brute(pos, box, t, 1.0)
    # Phi = 2/8, rho = 1/8 each, F = -3 sqrt(1/8) + 0.5/64
    assert rho[0] == rho[1] == 0.125
    assert U == pytest.approx(0.25 + 2 * (-3 * math.sqrt(0.125) + 0.5 / 64), rel=1e-15)
    # dU/dr = Phi' + 2 F'(rho) psi' with Phi' = -6 (1/2)^2, psi' = -3 (1/2)^2,
    # F' = -3 / (2 sqrt(1/8)) + 1/8; the force on atom 0 points along -x by -dU/dr
    g = -1.5 + 2 * (-1.5 / math.sqrt(0.125) + 0.125) * -0.75
    np.testing.assert_allclose(f[0], [g, 0.0, 0.0], rtol=1e-14)
    np.testing.assert_allclose(f[1], [-g, 0.0, 0.0], rtol=1e-14)
    # at r exactly on the knot both functions vanish (strict r < knot)
    pos2 = np.array([[1.0, 1.0, 1.0], [2.0, 1.0, 1.0]])
    U2, f2, rho2 = orc.eam_brute(pos2, box, t, 1.5)
    assert U2 == 0.0 and np.all(f2 == 0.0) and np.all(rho2 == 0.0)


def bcc_shells(a0, rmax):
    """bcc neighbour shells by integer search: lattice vectors (a0/2)(i, j, k)
    with i, j, k all even or all odd."""
    out = {}
    R = range(-8, 9)
    for i, j, k in itertools.product(R, R, R):
        if (i or j or k) and (i % 2 == j % 2 == k % 2):
            r = a0 * math.sqrt(i * i + j * j + k * k) / 2
            if r < rmax:
                key = round(r, 12)  # groups a shell; its radius keeps full precision
                rr, z = out.get(key, (r, 0))
                out[key] = (rr, z + 1)
    return {rr: z for rr, z in out.values()}


def test_bcc_shells_are_crystallography():
    sh = bcc_shells(1.0, 2.05)
    assert [sh[k] for k in sorted(sh)] == [8, 6, 12, 24, 8, 6]


@pytest.mark.parametrize("a0", [1.0, 0.97])
def test_bcc_lattice_energy_closed_form(orc, a0):
    t = table(orc)
    s = inputs.eam_bcc(nc=6, a0=a0, T=0.0)
    off, ids = orc.neighbors_cells(s.pos, s.box, P["rc"] + P["skin"])
    U, f, rho, dF, e = orc.eam_list(s.pos, s.box, off, ids, t, P["rc"])

    def cubic_sum(knots, coef, r):
        return sum(c * (k - r) ** 3 for k, c in zip(knots, coef) if r < k)

    sh = bcc_shells(a0, P["rc"])
    rho0 = sum(z * cubic_sum(P["psi_r"], P["psi_a"], r) for r, z in sh.items())
    u0 = 0.5 * sum(z * cubic_sum(P["phi_r"], P["phi_a"], r) for r, z in sh.items()) \
        - P["F_sqrt"] * math.sqrt(rho0) + P["F_quad"] * rho0 ** 2
    np.testing.assert_allclose(rho, rho0, rtol=1e-13)
    assert U / s.n == pytest.approx(u0, rel=1e-12)
    assert np.max(np.abs(f)) < 1e-10
    if a0 == 1.0:
        assert u0 == pytest.approx(-3.00835, abs=1e-5)  # the fitted cohesive energy


def perturbed_bcc(nc, amp, seed):
    s = inputs.eam_bcc(nc=nc)
    g = inputs.gaussian(seed, s.pos.size).reshape(-1, 3)
    return s, np.mod(s.pos + amp * g, s.box)


def test_list_equals_brute_force(orc):
    t = table(orc, F_quad=0.01, psi_r=(1.8, 1.2), psi_a=(1.0, 0.7))
    s, pos = perturbed_bcc(4, 0.06, 951)
    off, ids = orc.neighbors_cells(pos, s.box, P["rc"] + P["skin"])
    U1, f1, rho1, _, _ = orc.eam_list(pos, s.box, off, ids, t, P["rc"])
    U2, f2, rho2 = orc.eam_brute(pos, s.box, t, P["rc"])
    np.testing.assert_allclose(rho1, rho2, rtol=1e-13)
    np.testing.assert_allclose(f1, f2, rtol=1e-11, atol=1e-11)
    assert U1 == pytest.approx(U2, rel=1e-12)
    assert np.max(np.abs(f1.sum(axis=0))) < 1e-10


def test_forces_are_minus_gradient(orc):
    t = table(orc, F_quad=0.01, psi_r=(1.8, 1.2), psi_a=(1.0, 0.7))
    s, pos = perturbed_bcc(4, 0.06, 952)
    _, f, _ = orc.eam_brute(pos, s.box, t, P["rc"])
    h = 1e-6
    for i in (0, 17, 101):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            up = orc.eam_brute(pp, s.box, t, P["rc"])[0]
            um = orc.eam_brute(pm, s.box, t, P["rc"])[0]
            assert f[i, d] == pytest.approx(-(up - um) / (2 * h), rel=2e-6, abs=1e-8)


def test_nve_conserves_energy_and_momentum(orc):
    s = inputs.eam_bcc(nc=8)
    t = table(orc)
    prm = orc.make_params(potential=orc.POT_EAM, rc=P["rc"], skin=P["skin"], dt=P["dt"], eam=t)
    out = orc.md_run(prm, s.pos, s.vel, s.box, 1000)
    E = out["energies"][:, 2]
    assert np.max(np.abs(E - E[0])) < 2e-6 * abs(E[0])
    assert np.max(np.abs(out["vel"].sum(axis=0))) < 1e-10
    assert out["builds"] >= 2


def test_forces_sample_equals_all_atom(orc):
    t = table(orc, F_quad=0.01)
    s, pos = perturbed_bcc(6, 0.05, 953)
    prm = orc.make_params(potential=orc.POT_EAM, rc=P["rc"], skin=P["skin"], eam=t)
    off, ids = orc.neighbors_cells(pos, s.box, P["rc"] + P["skin"])
    _, f, _, _, e = orc.eam_list(pos, s.box, off, ids, t, P["rc"])
    idx = np.unique(np.concatenate([np.argsort(pos[:, 0])[:5], np.argsort(-pos[:, 2])[:5],
                                    np.arange(0, s.n, 37)])).astype(np.int64)
    fs, es = orc.forces_sample(prm, pos, s.box, idx)
    np.testing.assert_array_equal(fs, f[idx])
    np.testing.assert_array_equal(es, e[idx])
