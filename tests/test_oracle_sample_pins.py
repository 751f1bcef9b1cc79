"""Pins of the oracle's sampled-atom routines (forces_sample,
neighbors_sample), which check the full-size GPU runs one atom at a time.

They are pinned to the all-atom routines, which are pinned on their own
(brute force, closed-form lattice sums, finite differences): for every
sampled atom the pair forces of Sec. 2.2, the three-step Sutton-Chen forces
of Eq. 1-2 and Sec. 3.1, the per-atom energies and the list rows of Sec. 2.1
must equal the all-atom results element by element.  Both sides add the same
terms in ascending neighbour order, so the comparison is exact.  The systems
are chosen so that a plausible slip would show: samples on every box face
(the neighbourhoods of i and of its neighbours j wrap), a Sutton-Chen shell
that straddles r_c, a box side under 3 r_c (stencil cells coincide), and
rows just below and just above the routines' 4096-entry capacity.  CPU only.
"""
import numpy as np
import pytest

from paper_1611_00075_gb300 import inputs

A0 = (4.0 / 0.8442) ** (1.0 / 3.0)


def _perturbed(pos, box, amp, seed):
    g = inputs.gaussian(seed, pos.size).reshape(-1, 3)
    return np.mod(pos + amp * g, box)


def _face_samples(pos, box, per_face=6):
    """The atoms nearest to each of the six box faces, plus a spread of
    interior atoms."""
    idx = []
    for d in range(3):
        idx += list(np.argsort(pos[:, d])[:per_face])
        idx += list(np.argsort(box[d] - pos[:, d])[:per_face])
    idx += list(range(0, len(pos), max(1, len(pos) // 40)))
    return np.unique(np.array(idx, dtype=np.int64))


def _system(case):
    """(pos, box, potential parameters, sampled atoms)."""
    if case == "porous_lj":
        s = inputs.lj_porous(nc=10, fraction=0.3, rmin=1.5, rmax=3.0)
        pos = _perturbed(s.pos, s.box, 0.06, 901)
        prm = dict(potential="lj", rc=2.5, skin=0.3)
        return pos, s.box, prm, _face_samples(pos, s.box)
    if case == "sc_shell8_straddles_rc":
        # a0 = a = 1: the 8th fcc shell lies at r = 2 = r_c; a small
        # perturbation puts about half its pairs inside the cutoff
        s = inputs.sc_fcc(nc=8)
        pos = _perturbed(s.pos, s.box, 0.01, 902)
        prm = dict(potential="sc", rc=2.0, skin=0.2, eps=1.0, sigma=1.0, c=39.432, n_exp=9.0,
                   m_exp=6.0)
        return pos, s.box, prm, _face_samples(pos, s.box)
    # orthorhombic LJ block 6 x 8 x 4 fcc cells: z = 6.72 lies between
    # 2 r_list and 3 r_c, so the r_c cell grid has 2 cells along z
    nc = (6, 8, 4)
    box = A0 * np.array(nc, dtype=np.float64)
    pos = _perturbed(inputs.fcc_lattice(nc, A0), box, 0.07, 903)
    prm = dict(potential="lj", rc=2.5, skin=0.3)
    return pos, box, prm, _face_samples(pos, box)


def _params(orc, prm):
    if prm["potential"] == "lj":
        return orc.make_params(potential=orc.POT_LJ, rc=prm["rc"], skin=prm["skin"])
    return orc.make_params(potential=orc.POT_SC, eps=prm["eps"], sigma=prm["sigma"],
                           c=prm["c"], n_exp=prm["n_exp"], m_exp=prm["m_exp"], rc=prm["rc"],
                           skin=prm["skin"])


CASES = ["porous_lj", "sc_shell8_straddles_rc", "orthorhombic_lj"]


@pytest.mark.parametrize("case", CASES)
def test_forces_sample_equals_all_atom_routines(orc, case):
    pos, box, prm, idx = _system(case)
    off, ids = orc.neighbors_cells(pos, box, prm["rc"] + prm["skin"])
    if prm["potential"] == "lj":
        _, f, e = orc.lj_list(pos, box, off, ids, rc=prm["rc"], per_atom=True)
    else:
        _, f, _, _, e = orc.sc_list(pos, box, off, ids, eps=prm["eps"], a=prm["sigma"],
                                    c=prm["c"], n_exp=prm["n_exp"], m_exp=prm["m_exp"],
                                    rc=prm["rc"], per_atom=True)
        # the sample touches pairs on both sides of r_c
        r = np.array([np.sqrt(orc.pair_r2(pos, box, int(i), int(j)))
                      for i in idx for j in ids[off[i]:off[i + 1]]])
        assert np.sum(np.abs(r - prm["rc"]) < 0.02) > 50
        assert np.any((r < prm["rc"]) & (r > prm["rc"] - 0.02))
        assert np.any((r >= prm["rc"]) & (r < prm["rc"] + 0.02))
    fs, es = orc.forces_sample(_params(orc, prm), pos, box, idx)
    # face samples must wrap: some of their neighbours sit across the box
    far = [np.max(np.abs(pos[ids[off[i]:off[i + 1]]] - pos[i])) for i in idx[:12]]
    assert max(far) > 0.5 * np.min(box)
    np.testing.assert_array_equal(fs, f[idx])
    np.testing.assert_array_equal(es, e[idx])


@pytest.mark.parametrize("case", CASES)
def test_neighbors_sample_equals_cell_list(orc, case):
    pos, box, prm, idx = _system(case)
    r_list = prm["rc"] + prm["skin"]
    off, ids = orc.neighbors_cells(pos, box, r_list)
    so, si = orc.neighbors_sample(pos, box, r_list, idx)
    assert so[-1] == sum(off[i + 1] - off[i] for i in idx)
    for k, i in enumerate(idx):
        np.testing.assert_array_equal(si[so[k]:so[k + 1]], ids[off[i]:off[i + 1]])


def _dense_ball(count, radius, centre, box, seed):
    """count atoms spread uniformly in a ball (for capacity cases)."""
    u = inputs.uniform(seed, 3 * count).reshape(count, 3)
    g = inputs.gaussian(seed + 1, 3 * count).reshape(count, 3)
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    r = radius * np.cbrt(u[:, 0])[:, None]
    return np.mod(centre + r * g, box)


@pytest.mark.parametrize("extra", [0, 1])
def test_sample_rows_at_and_over_capacity(orc, extra):
    """Row of the centre atom with exactly 4096 neighbours is returned in
    full; with 4097 both routines report ORC_ERR_CAPACITY."""
    box = np.array([30.0, 30.0, 30.0])
    c = np.array([15.0, 15.0, 15.0])
    pos = np.vstack([c, _dense_ball(4096 + extra, 2.0, c, box, 904)])
    idx = np.array([0], dtype=np.int64)
    prm = orc.make_params(potential=orc.POT_LJ, rc=2.5, skin=0.3)
    if extra == 0:
        so, si = orc.neighbors_sample(pos, box, 2.8, idx, cap=8192)
        assert so[-1] == 4096
        off, ids = orc.neighbors_cells(pos, box, 2.8)
        np.testing.assert_array_equal(si, ids[off[0]:off[1]])
        fs, es = orc.forces_sample(prm, pos, box, idx)
        _, f, e = orc.lj_list(pos, box, off, ids, per_atom=True)
        np.testing.assert_array_equal(fs[0], f[0])
        np.testing.assert_array_equal(es[0], e[0])
    else:
        with pytest.raises(RuntimeError, match=r"\(-4\)"):
            orc.neighbors_sample(pos, box, 2.8, idx, cap=8192)
        with pytest.raises(RuntimeError, match=r"\(-4\)"):
            orc.forces_sample(prm, pos, box, idx)


def test_sc_sample_over_capacity_through_a_neighbour(orc):
    """The sampled atom has a short row, but one of its neighbours j has
    4097 within r_c: rho_j cannot be formed, so forces_sample must fail."""
    box = np.array([30.0, 30.0, 30.0])
    c = np.array([15.0, 15.0, 15.0])
    ball = _dense_ball(4097, 1.0, c, box, 905)
    i_pos = c + np.array([1.95, 0.0, 0.0])
    pos = np.vstack([i_pos, c, ball])
    prm = orc.make_params(potential=orc.POT_SC, eps=1.0, sigma=1.0, c=39.432, n_exp=9.0,
                          m_exp=6.0, rc=2.0, skin=0.2)
    so, _ = orc.neighbors_sample(pos, box, 2.0, np.array([0], dtype=np.int64), cap=8192)
    assert 1 <= so[-1] < 4096
    with pytest.raises(RuntimeError, match=r"\(-4\)"):
        orc.forces_sample(prm, pos, box, np.array([0], dtype=np.int64))
