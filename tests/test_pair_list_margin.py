"""The accept test of the two-atom union lists, on the CPU.

A slot's union list holds every candidate j within r_list of either of its
atoms x0, x1.  The build tests each candidate once against the midpoint
m = (x0 + x1) / 2 and half separation u = (x1 - x0) / 2: with e = x_j - m,
min(|x_j - x0|^2, |x_j - x1|^2) = |e|^2 + |u|^2 - 2 |e.u|, so j is accepted
when |e|^2 - 2 |e.u| < r_list^2 (1 + 2^-14) - |u|^2, evaluated in float32.
These tests check the identity in float64, and that the float32 evaluation
(positions relative to the cell centre, the midpoint moved by the stencil
shift, every operation rounded) stays far inside the 2^-14 margin, so no
pair within r_list is ever missed.  The geometry is the porous benchmark's:
cells of width 2.83 sigma, r_list = 2.8 sigma, two atoms of one cell."""
import numpy as np

from paper_1611_00075_gb300 import inputs

R_LIST = 2.8
W = 2.8286


def geometry(n, seed):
    """Slot atoms anywhere in the home cell, candidates anywhere in one of
    the 27 stencil cells (cell-relative coordinates in [-W/2, W/2))."""
    u = inputs.uniform(seed, 12 * n).reshape(n, 12)
    q0 = (u[:, 0:3] - 0.5) * W
    q1 = (u[:, 3:6] - 0.5) * W
    qj = (u[:, 6:9] - 0.5) * W
    d = np.floor(u[:, 9:12] * 3.0) - 1.0  # stencil shift of j's cell, -1..1 per axis
    return q0, q1, qj, d


def test_midpoint_identity_float64():
    q0, q1, qj, d = geometry(200000, inputs.SEED_BASE + 901)
    xj = qj + d * W
    m, u = 0.5 * (q0 + q1), 0.5 * (q1 - q0)
    e = xj - m
    lhs = np.minimum(np.sum((xj - q0) ** 2, 1), np.sum((xj - q1) ** 2, 1))
    rhs = np.sum(e * e, 1) + np.sum(u * u, 1) - 2.0 * np.abs(np.sum(e * u, 1))
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12)


def test_float32_midpoint_test_stays_inside_the_margin():
    f = np.float32
    q0, q1, qj, d = geometry(1000000, inputs.SEED_BASE + 902)
    q0f, q1f, qjf = q0.astype(f), q1.astype(f), qj.astype(f)
    uf = f(0.5) * (q1f - q0f)
    mf = q0f + uf
    sf = mf - d.astype(f) * f(W)          # the midpoint moved against the shift
    ef = qjf - sf
    r2 = (ef[:, 0] * ef[:, 0] + ef[:, 1] * ef[:, 1]) + ef[:, 2] * ef[:, 2]
    p = (ef[:, 0] * uf[:, 0] + ef[:, 1] * uf[:, 1]) + ef[:, 2] * uf[:, 2]
    uu = (uf[:, 0] * uf[:, 0] + uf[:, 1] * uf[:, 1]) + uf[:, 2] * uf[:, 2]
    lhs32 = (r2 - f(2.0) * np.abs(p)).astype(np.float64) + uu.astype(np.float64)
    # the exact nearer-atom distance of the float32 inputs
    xj = qjf.astype(np.float64) + d * np.float64(f(W))
    exact = np.minimum(np.sum((xj - q0f.astype(np.float64)) ** 2, 1),
                       np.sum((xj - q1f.astype(np.float64)) ** 2, 1))
    err = np.abs(lhs32 - exact)
    margin = R_LIST * R_LIST * 2.0 ** -14
    print("float32 midpoint test: max error %.3g sigma^2 against a margin of %.3g sigma^2"
          % (err.max(), margin))
    assert err.max() < 0.05 * margin
    # hence: every candidate inside r_list passes the accept bound
    hi = f(R_LIST * R_LIST * (1.0 + 2.0 ** -14))
    inside = exact < R_LIST * R_LIST
    accepted = (r2 - f(2.0) * np.abs(p)) < (hi - uu)
    assert np.all(accepted[inside])
    assert inside.sum() > 50000  # the sample does reach the boundary region
