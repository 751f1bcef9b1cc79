"""Pins of the CPU oracle to facts that do not come from the oracle itself:
closed-form fcc lattice sums, brute force on tiny inputs, finite-difference
gradients, conservation laws, textbook dimer values and hand-computable
network cases.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from paper_1611_00075_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "textbook.json")))


def fcc_shells(kmax):
    """Shell multiplicities of fcc by integer search: lattice vectors are
    (a0/2)(i, j, k) with i + j + k even; shell index s = (i^2+j^2+k^2)/2."""
    lim = int(math.isqrt(2 * kmax)) + 1
    r = np.arange(-lim, lim + 1)
    I, J, K = np.meshgrid(r, r, r, indexing="ij")
    ok = ((I + J + K) % 2 == 0)
    s2 = (I * I + J * J + K * K)[ok]
    s2 = s2[(s2 > 0) & (s2 <= 2 * kmax)]
    ks, counts = np.unique(s2 // 2, return_counts=True)
    assert np.all(s2 % 2 == 0)
    return dict(zip(ks.tolist(), counts.tolist()))


def perturbed(system, amp, seed):
    g = inputs.gaussian(seed, system.pos.size).reshape(-1, 3)
    pos = system.pos + amp * g
    return np.mod(pos, system.box)


# --------------------------------------------------------------------- lists

def test_fcc_shell_search_matches_crystallography():
    sh = fcc_shells(10)
    gold = GOLD["fcc_shells"]
    assert [sh[k] for k in gold["k"]] == gold["z"]


@pytest.mark.parametrize("half", [False, True])
@pytest.mark.parametrize("case", ["lj_small", "lj_tight_box", "sc_small", "sparse"])
def test_cell_list_equals_brute_force(orc, case, half):
    if case == "lj_small":
        s = inputs.lj_fcc(nc=4)
        pos, r_list = perturbed(s, 0.08, 11), 2.8
    elif case == "lj_tight_box":
        # L just above 2 r_list: cells per side = 2, stencil cells coincide
        s = inputs.lj_fcc(nc=4, rho=1.0)            # L = 4 * 1.5874 = 6.35
        pos, r_list = perturbed(s, 0.05, 12), 3.17
        assert s.box[0] > 2 * r_list
    elif case == "sc_small":
        s = inputs.sc_fcc(nc=5)
        pos, r_list = perturbed(s, 0.03, 13), 2.2
    else:
        s = inputs.lj_fcc(nc=5)
        keep = inputs.uniform(14, s.n) < 0.1          # 10% of sites: many empty cells
        pos, r_list = perturbed(s, 0.2, 15)[keep], 2.8
    ob, ib = orc.neighbors_brute(pos, s.box, r_list, half)
    oc, ic = orc.neighbors_cells(pos, s.box, r_list, half)
    np.testing.assert_array_equal(ob, oc)
    np.testing.assert_array_equal(ib, ic)
    # symmetric (full) / each unordered pair once (half)
    n = pos.shape[0]
    pairs = set()
    for i in range(n):
        for j in ib[ob[i]:ob[i + 1]]:
            pairs.add((i, int(j)))
    if half:
        assert all(i < j for i, j in pairs)
    else:
        assert all((j, i) in pairs for i, j in pairs)


def test_perfect_fcc_neighbour_counts(orc):
    # LJ: a0 = (4/0.8442)^(1/3), r_list = 2.8 reaches shells a0 sqrt(k/2) < 2.8
    s = inputs.lj_fcc(nc=5, T=0.0)
    a0 = s.box[0] / 5
    sh = fcc_shells(12)
    want = sum(z for k, z in sh.items() if a0 * math.sqrt(k / 2) < 2.8)
    off, _ = orc.neighbors_cells(s.pos, s.box, 2.8)
    assert want == 78
    assert np.all(np.diff(off) == want)
    off, _ = orc.neighbors_cells(s.pos, s.box, 2.8, half=True)
    assert np.all(np.diff(off)[:1] >= 0) and off[-1] == want * s.n // 2
    # Sutton-Chen: a0 = 1, r_list = 2.2 -> shells 1..9 (k = 9 at 2.121, k = 10 at 2.236)
    s = inputs.sc_fcc(nc=6, T=0.0)
    want = sum(z for k, z in sh.items() if math.sqrt(k / 2) < 2.2)
    off, _ = orc.neighbors_cells(s.pos, s.box, 2.2)
    assert want == 176
    assert np.all(np.diff(off) == want)


def test_pair_r2_definition(orc):
    box = np.array([10.0, 11.0, 12.0])
    pos = np.array([[0.5, 10.5, 6.0], [9.5, 0.25, 0.5]])
    # x: 9.5 - 0.5 = 9 > 5 -> -1;  y: 0.25 - 10.5 = -10.25 < -5.5 -> 0.75;
    # z: 0.5 - 6.0 = -5.5, not < -6 -> -5.5
    want = (-1.0) ** 2 + 0.75 ** 2 + 5.5 ** 2
    assert orc.pair_r2(pos, box, 0, 1) == want


# ----------------------------------------------------------------- binning

def test_binning_definition(orc):
    s = inputs.lj_porous(nc=8, fraction=0.3, rmin=1.5, rmax=3.0)
    pos = perturbed(s, 0.1, 21)
    r_list = 2.8
    ncell, cell_of, start, order = orc.bin_cells(pos, s.box, r_list)
    assert np.all(ncell == np.floor(s.box / r_list))
    w = s.box / ncell
    c3 = np.stack([cell_of % ncell[0], (cell_of // ncell[0]) % ncell[1],
                   cell_of // (ncell[0] * ncell[1])], axis=1)
    # every atom's cell contains its position
    assert np.all(c3 * w <= pos + 1e-12) and np.all(pos < (c3 + 1) * w + 1e-12)
    # start is the exclusive prefix of the counts; order is stable by (cell, id)
    counts = np.bincount(cell_of, minlength=int(np.prod(ncell)))
    np.testing.assert_array_equal(start, np.concatenate([[0], np.cumsum(counts)]))
    np.testing.assert_array_equal(order, np.lexsort((np.arange(len(pos)), cell_of)))


# ------------------------------------------------------------------ energies

def test_lj_dimer_textbook(orc):
    for key in ("lj_dimer_minimum", "lj_dimer_sigma"):
        g = GOLD[key]
        box = np.array([20.0, 20.0, 20.0])
        pos = np.array([[5.0, 5.0, 5.0], [5.0 + g["r"], 5.0, 5.0]])
        rc = 9.0
        shift = 4 * (rc ** -12 - rc ** -6)
        U, f = orc.lj_brute(pos, box, rc=rc)
        assert abs(U - (g["phi"] - shift)) < 1e-12
        # Sec. 2.2 sign: repulsive force pushes atom 0 towards -x
        assert abs(f[0, 0] + g["force"]) < 1e-9 and abs(f[1, 0] - g["force"]) < 1e-9


def lj_phi(r, rc):
    return 4 * (r ** -12 - r ** -6) - 4 * (rc ** -12 - rc ** -6)


def test_lj_fcc_lattice_energy_closed_form(orc):
    s = inputs.lj_fcc(nc=5, T=0.0)
    a0 = s.box[0] / 5
    sh = fcc_shells(12)
    u = 0.5 * sum(z * lj_phi(a0 * math.sqrt(k / 2), 2.5) for k, z in sh.items()
                  if a0 * math.sqrt(k / 2) < 2.5)
    U, f = orc.lj_brute(s.pos, s.box)
    assert abs(U / s.n - u) <= 1e-12 * abs(u)
    assert np.max(np.abs(f)) < 1e-11
    off, ids = orc.neighbors_cells(s.pos, s.box, 2.8)
    U2, f2 = orc.lj_list(s.pos, s.box, off, ids)
    assert abs(U2 / s.n - u) <= 1e-12 * abs(u)
    assert np.max(np.abs(f2)) < 1e-11


def test_sc_fcc_lattice_energy_closed_form(orc):
    p = inputs.SC_DEFAULT
    s = inputs.sc_fcc(nc=5, T=0.0)
    sh = fcc_shells(12)
    rs = [(math.sqrt(k / 2), z) for k, z in sh.items() if math.sqrt(k / 2) < p["rc"]]
    # shell 8 sits at exactly r = 2a = r_c and is excluded by the strict cutoff
    assert len(rs) == 7
    rho = sum(z * r ** -6 for r, z in rs)
    u = 0.5 * sum(z * r ** -9 for r, z in rs) - p["c"] * math.sqrt(rho)
    off, ids = orc.neighbors_cells(s.pos, s.box, 2.2)
    U, f, rho_o, dF = orc.sc_list(s.pos, s.box, off, ids)
    assert abs(U / s.n - u) <= 1e-12 * abs(u)
    np.testing.assert_allclose(rho_o, rho, rtol=1e-13)
    np.testing.assert_allclose(dF, -p["c"] / (2 * math.sqrt(rho)), rtol=1e-13)
    assert np.max(np.abs(f)) < 1e-10
    Ub, fb, _ = orc.sc_brute(s.pos, s.box)
    assert abs(Ub - U) <= 1e-11 * abs(U)   # different summation order


def _fd_check(energy, pos, box, idx, h=1e-5):
    out = []
    for (i, d) in idx:
        p1 = pos.copy(); p1[i, d] += h
        p2 = pos.copy(); p2[i, d] -= h
        out.append(-(energy(p1) - energy(p2)) / (2 * h))
    return np.array(out)


def _min_gap_to_cutoff(orc, pos, box, rc):
    off, ids = orc.neighbors_brute(pos, box, rc + 0.5)
    r = np.array([math.sqrt(orc.pair_r2(pos, box, i, int(j)))
                  for i in range(len(pos)) for j in ids[off[i]:off[i + 1]]])
    return np.min(np.abs(r - rc))


def test_lj_forces_are_minus_gradient(orc):
    s = inputs.lj_fcc(nc=4)
    pos = perturbed(s, 0.06, 31)
    h = 2e-6
    assert _min_gap_to_cutoff(orc, pos, s.box, 2.5) > 10 * h   # no pair crosses r_c
    U, f = orc.lj_brute(pos, s.box)
    idx = [(int(i), int(d)) for i, d in zip(inputs.splitmix64(32, 12) % s.n,
                                            inputs.splitmix64(33, 12) % 3)]
    fd = _fd_check(lambda p: orc.lj_brute(p, s.box)[0], pos, s.box, idx, h=h)
    want = np.array([f[i, d] for i, d in idx])
    np.testing.assert_allclose(fd, want, rtol=1e-6, atol=1e-7 * np.sqrt(np.mean(f * f)))
    assert np.max(np.abs(f.sum(axis=0))) < 1e-11 * np.sum(np.abs(f))
    # list form equals the all-pairs form
    off, ids = orc.neighbors_cells(pos, s.box, 2.8)
    U2, f2 = orc.lj_list(pos, s.box, off, ids)
    assert abs(U2 - U) < 1e-11 * abs(U)
    np.testing.assert_allclose(f2, f, rtol=1e-10, atol=1e-11)


def test_sc_forces_are_minus_gradient(orc):
    s = inputs.sc_fcc(nc=5)
    pos = perturbed(s, 0.03, 41)
    h = 2e-6
    assert _min_gap_to_cutoff(orc, pos, s.box, 2.0) > 10 * h   # no pair crosses r_c
    off, ids = orc.neighbors_cells(pos, s.box, 2.2)
    U, f, rho, dF = orc.sc_list(pos, s.box, off, ids)
    idx = [(int(i), int(d)) for i, d in zip(inputs.splitmix64(42, 10) % s.n,
                                            inputs.splitmix64(43, 10) % 3)]
    fd = _fd_check(lambda p: orc.sc_brute(p, s.box)[0], pos, s.box, idx, h=h)
    want = np.array([f[i, d] for i, d in idx])
    # |U| ~ 1e5 makes the difference quotient's round-off ~1e-5 absolute
    np.testing.assert_allclose(fd, want, rtol=1e-6, atol=1e-6 * np.sqrt(np.mean(f * f)))
    assert np.max(np.abs(f.sum(axis=0))) < 1e-11 * np.sum(np.abs(f))
    Ub, fb, rhob = orc.sc_brute(pos, s.box)
    assert abs(Ub - U) < 1e-11 * abs(U)
    np.testing.assert_allclose(fb, f, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(rhob, rho, rtol=1e-12)


def test_sc_many_body_term_is_not_pairwise(orc):
    # Dropping the (F'_i + F'_j) psi' term, or using only F'_i, breaks F = -grad U
    # on an asymmetric cluster; this pins the three-step order of Sec. 3.1.
    box = np.array([30.0, 30.0, 30.0])
    pos = np.array([[10, 10, 10], [11.0, 10, 10], [10, 11.1, 10], [10.2, 10.1, 11.05]])
    U, f, rho = orc.sc_brute(pos, box, rc=5.0)
    assert len(set(np.round(rho, 12))) > 1
    idx = [(i, d) for i in range(4) for d in range(3)]
    fd = _fd_check(lambda p: orc.sc_brute(p, box, rc=5.0)[0], pos, box, idx, h=1e-6)
    np.testing.assert_allclose(fd, f.ravel(), rtol=1e-6, atol=1e-6)


# --------------------------------------------------------------- integrator

def _lj_params(orc, **kw):
    return orc.make_params(potential=orc.POT_LJ, **kw)


def test_momentum_conserved_and_nve(orc):
    s = inputs.lj_fcc(nc=6, T=0.72)
    out = orc.md_run(_lj_params(orc), s.pos, s.vel, s.box, 200)
    p0 = s.vel.sum(axis=0)
    p1 = out["vel"].sum(axis=0)
    assert np.max(np.abs(p1 - p0)) < 1e-10
    E = out["energies"][:, 2]
    assert np.max(np.abs(E - E[0])) / abs(E[0]) < 2e-4
    assert out["builds"] >= 1


@pytest.mark.slow
def test_nve_energy_drift_config1(orc):
    s = inputs.lj_fcc(nc=10, T=0.72)
    out = orc.md_run(_lj_params(orc), s.pos, s.vel, s.box, 1000)
    E = out["energies"][:, 2]
    # mean of the last 100 steps against the first 100: secular drift
    drift = abs(E[-100:].mean() - E[:100].mean()) / abs(E[0])
    assert drift < 5e-5


def test_time_reversibility(orc):
    s = inputs.lj_fcc(nc=5, T=0.72)
    p = _lj_params(orc, rebuild_every=1)
    a = orc.md_run(p, s.pos, s.vel, s.box, 50, want_energies=False)
    b = orc.md_run(p, a["pos"], -a["vel"], s.box, 50, want_energies=False)
    d = b["pos"] - s.pos
    d -= s.box * np.round(d / s.box)
    assert np.max(np.abs(d)) < 1e-9
    np.testing.assert_allclose(-b["vel"], s.vel, atol=1e-9)


def test_energy_error_scales_as_dt_squared(orc):
    s = inputs.lj_fcc(nc=5, T=0.72)
    errs = []
    for dt, n in ((0.004, 100), (0.002, 200)):
        out = orc.md_run(_lj_params(orc, dt=dt, rebuild_every=1), s.pos, s.vel, s.box, n)
        E = out["energies"][:, 2]
        errs.append(np.max(np.abs(E - E[0])))
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.5, ratio


def test_rebuild_rule_keeps_forces_exact(orc):
    # Half-skin rule: the list-based trajectory equals the one rebuilt every step.
    s = inputs.lj_fcc(nc=5, T=1.5)
    a = orc.md_run(_lj_params(orc, rebuild_every=0), s.pos, s.vel, s.box, 60)
    b = orc.md_run(_lj_params(orc, rebuild_every=1), s.pos, s.vel, s.box, 60)
    assert 1 < a["builds"] < b["builds"]
    np.testing.assert_allclose(a["pos"], b["pos"], atol=1e-11)
    np.testing.assert_allclose(a["energies"], b["energies"], rtol=1e-12, atol=1e-9)


def test_sc_md_runs_and_conserves(orc):
    s = inputs.sc_fcc(nc=5)
    p = orc.make_params(potential=orc.POT_SC, eps=1.0, sigma=1.0, c=39.432, n_exp=9.0,
                        m_exp=6.0, rc=2.0, skin=0.2, dt=7.6e-4, mass=1.0)
    out = orc.md_run(p, s.pos, s.vel, s.box, 50)
    E = out["energies"][:, 2]
    assert np.max(np.abs(out["vel"].sum(axis=0) - s.vel.sum(axis=0))) < 1e-9
    # At a0 = a the 8th fcc shell sits exactly at r_c = 2a; the unshifted
    # cutoff lets about half of those pairs enter on the first step, a jump
    # of ~3e-4 of |E|.  After that the total energy stays flat.
    assert np.max(np.abs(E - E[0])) / abs(E[0]) < 1e-3
    assert np.max(np.abs(E[5:] - E[5])) / abs(E[0]) < 5e-5


# ---------------------------------------------------------------- cost model

def _rand_params(orc, seed):
    return 0.3 * inputs.gaussian(seed, orc.mlp_nparams())


def test_mlp_hand_computable(orc):
    # Only hidden unit 0 of each layer is live: y = w3 relu(w2 relu(w1.x + b1) + b2) + b3
    H = orc.MLP_HIDDEN
    P = np.zeros(orc.mlp_nparams())
    W1 = P[:3 * H].reshape(H, 3); b1 = P[3 * H:4 * H]
    W2 = P[4 * H:4 * H + H * H].reshape(H, H); b2 = P[4 * H + H * H:5 * H + H * H]
    W3 = P[5 * H + H * H:6 * H + H * H]; b3 = P[6 * H + H * H:]
    W1[0] = [0.5, -1.0, 2.0]; b1[0] = 0.25
    W2[0, 0] = 1.5; b2[0] = -0.1
    W3[0] = 2.0; b3[0] = 0.3
    x = np.array([[1.0, 0.5, 0.75]])
    z1 = 0.5 - 0.5 + 1.5 + 0.25            # 1.75
    z2 = 1.5 * z1 - 0.1                     # 2.525
    y = 2.0 * z2 + 0.3                      # 5.35
    assert abs(orc.mlp_forward(x, P)[0] - y) < 1e-14
    target = np.array([5.0])
    loss, G = orc.mlp_loss_grad(x, target, P)
    e = y - 5.0
    assert abs(loss - e * e) < 1e-14
    gG = G
    dy = 2 * e
    assert abs(gG[6 * H + H * H] - dy) < 1e-13                     # db3
    assert abs(gG[5 * H + H * H] - dy * z2) < 1e-13                # dW3[0]
    assert abs(gG[4 * H + H * H] - dy * 2.0) < 1e-13               # db2[0]
    assert abs(gG[4 * H] - dy * 2.0 * z1) < 1e-13                  # dW2[0,0]
    assert abs(gG[3 * H] - dy * 2.0 * 1.5) < 1e-13                 # db1[0]
    np.testing.assert_allclose(gG[0:3], dy * 2.0 * 1.5 * x[0], atol=1e-13)
    # dead units get no gradient
    assert np.all(gG[3:3 * H] == 0)


def test_mlp_gradient_finite_difference(orc):
    P = _rand_params(orc, 51)
    X = inputs.gaussian(52, 3 * 40).reshape(40, 3)
    y = inputs.gaussian(53, 40)
    loss, G = orc.mlp_loss_grad(X, y, P)
    k = inputs.splitmix64(54, 25) % P.size
    h = 1e-6
    for j in k:
        a = P.copy(); a[j] += h
        b = P.copy(); b[j] -= h
        fd = (orc.mlp_loss_grad(X, y, a)[0] - orc.mlp_loss_grad(X, y, b)[0]) / (2 * h)
        assert abs(fd - G[j]) < 1e-6 * max(1.0, abs(G[j])), (j, fd, G[j])


def test_adam_first_step_closed_form(orc):
    P = _rand_params(orc, 61)
    G = inputs.gaussian(62, P.size)
    m = np.zeros_like(P); v = np.zeros_like(P)
    P1 = P.copy()
    orc.adam(P1, G, m, v, 1, lr=1e-2, eps=1e-8)
    # t = 1: bias-corrected m = g, v = g^2, step = lr g / (|g| + eps)
    np.testing.assert_allclose(P1, P - 1e-2 * G / (np.abs(G) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * G, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * G * G, rtol=1e-13)   # 1 - 0.999 is inexact


def test_adam_training_reduces_loss(orc):
    P = _rand_params(orc, 71)
    X = inputs.uniform(72, 3 * 256).reshape(256, 3)
    y = 2.0 * X[:, 0] + np.sqrt(X[:, 1]) + X[:, 2] ** 2
    m = np.zeros_like(P); v = np.zeros_like(P)
    l0 = orc.mlp_loss_grad(X, y, P)[0]
    for t in range(1, 301):
        loss, G = orc.mlp_loss_grad(X, y, P)
        orc.adam(P, G, m, v, t, lr=3e-3)
    assert loss < 0.05 * l0


def test_partition_brute_force(orc):
    rng_costs = [np.array([5, 0, 0, 3, 7, 1, 1, 0, 9, 2]),
                 np.ones(17, np.int64), np.zeros(5, np.int64),
                 (inputs.splitmix64(81, 300) % 50).astype(np.int64)]
    for cost in rng_costs:
        for B in (1, 2, 3, 7):
            b = orc.partition(cost, B)
            assert b[0] == 0 and b[-1] == len(cost) and np.all(np.diff(b) >= 0)
            T = int(cost.sum())
            pref = np.concatenate([[0], np.cumsum(cost)])
            for part in range(1, B):
                # brute force: smallest k such that the prefix through cell k exceeds part/B
                k = next((kk for kk in range(len(cost)) if pref[kk + 1] * B > part * T),
                         len(cost))
                assert b[part] == k
            if T > 0:
                loads = [pref[b[q + 1]] - pref[b[q]] for q in range(B)]
                assert max(loads) <= T / B + cost.max()


def test_oracle_melt_is_a_liquid(orc):
    """The config-2 input protocol (heat fcc at T* = 2.4, hold at 1.2, 2,000
    oracle steps) leaves no crystal: atoms have diffused far from their
    lattice sites and the temperature is the target's."""
    from melt import lattice_msd, oracle_melt
    m = oracle_melt(orc, 6)
    assert lattice_msd(m, 6) > 1.0
    ke = 0.5 * np.sum(m.vel ** 2)
    assert abs(ke / (0.5 * (3 * m.n - 3)) - 1.2) < 1e-12
