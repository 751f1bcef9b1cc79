"""Energy bounds for pairs that straddle the cutoff (test helper).

A pair whose distance lies within delta of r_c may legitimately be counted on
one side by the oracle's float64 test and on the other by a float32 path.
Such pairs may move the potential energy by at most their own contribution,
which these helpers take from the oracle instead of a blanket constant.
"""
import numpy as np


def straddling_pairs(orc, pos, box, off, ids, rc, delta):
    """Number of unordered pairs of a full list with |r_ij - r_c| < delta.
    Candidates come from a vectorised minimum-image distance with a wide
    margin; the oracle's own r^2 decides each candidate."""
    rows = np.repeat(np.arange(len(pos)), np.diff(off))
    d = pos[ids] - pos[rows]
    d -= box * np.round(d / box)
    r = np.sqrt(np.sum(d * d, axis=1))
    cand = np.nonzero((np.abs(r - rc) < delta + 1e-9) & (ids > rows))[0]
    return sum(1 for k in cand
               if abs(np.sqrt(orc.pair_r2(pos, box, int(rows[k]), int(ids[k]))) - rc) < delta)


def lj_straddle_bound(orc, pos, box, off, ids, rc, delta, eps=1.0, sigma=1.0):
    """Largest energy change if any subset of the straddling pairs switched
    sides.  The energy is shifted to zero at r_c, so such a pair contributes
    |phi(r) - phi(r_c)| <= 2 delta |dphi/dr| near r_c; |dphi/dr| is the
    oracle's dimer force at r_c - delta (it varies by far less than the 2x
    margin across the band)."""
    n = straddling_pairs(orc, pos, box, off, ids, rc, delta)
    if n == 0:
        return 0.0
    dimer = np.array([[0.0, 0.0, 0.0], [rc - delta, 0.0, 0.0]])
    _, f = orc.lj_brute(dimer, np.array([10.0, 10.0, 10.0]) * rc, eps, sigma, rc)
    return n * 2.0 * delta * float(np.abs(f[0, 0])) * 2.0


def sc_straddle_bound(orc, pos, box, off, ids, delta, a=1.0, c=39.432, n_exp=9.0, m_exp=6.0,
                      rc=2.0, eps=1.0):
    """The many-body energy is not shifted: the oracle's energy with every
    straddling pair inside (cutoff r_c + delta) and with every one outside
    (r_c - delta) brackets the change; nothing else depends on the cutoff."""
    u_in = orc.sc_list(pos, box, off, ids, eps=eps, a=a, c=c, n_exp=n_exp, m_exp=m_exp,
                       rc=rc + delta)[0]
    u_out = orc.sc_list(pos, box, off, ids, eps=eps, a=a, c=c, n_exp=n_exp, m_exp=m_exp,
                        rc=rc - delta)[0]
    return abs(u_in - u_out)
