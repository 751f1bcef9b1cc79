"""Plain double-precision CPU oracle for the MD hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it.  The arithmetic lives in ``md_oracle.c`` (plain C,
fp64, ``-ffp-contract=off``); this module only compiles it with gcc and
marshals numpy arrays through ctypes.

Functions and the passages of Mangiardi & Meyer they follow:

* ``cell_grid``, ``bin_cells``   -- cell decomposition (Sec. 2.1)
* ``neighbors_brute``, ``neighbors_cells`` -- Verlet lists with r_list =
  r_c + skin (Sec. 2.1, Sec. 3.3)
* ``lj_brute``, ``lj_list``      -- pair forces F = -(1/d) dPhi/dr R (Sec. 2.2);
  ``lj_typed_*`` with per-species parameters (the Cu-Au systems of Sec. 3.1)
* ``sc_brute``, ``sc_list``      -- many-body energy Eq. 1-2 evaluated in three
  steps (Sec. 3.1)
* ``eam_brute``, ``eam_list``    -- the same with piecewise cubic pair and
  density functions, the form of the paper's Fe potential (Sec. 3.1, Table 2)
* ``md_run``, ``forces_once``    -- velocity-Verlet with the half-skin rebuild
  rule (Sec. 3.3); ``melt`` runs md_run in chunks for an input protocol
* ``mlp_forward``, ``mlp_loss_grad``, ``adam``, ``partition`` -- the per-cell
  cost model and equal-cost partition (not in the paper; they address its
  load-balance problem of inhomogeneous systems, Sec. 1 and Sec. 2.1)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "md_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

POT_LJ = 0
POT_SC = 1
POT_EAM = 2
EAM_MAX_KNOTS = 16


def build(force: bool = False) -> str:
    """Compile md_oracle.c with gcc (OpenMP, no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class EamTable(C.Structure):
    """Piecewise embedded-atom functions: Phi(r) = sum_k a_k (r_k - r)^3 and
    psi(r) = sum_k b_k (s_k - r)^3 over the knots beyond r, and
    F(rho) = -F_sqrt sqrt(rho) + F_quad rho^2."""
    _fields_ = [("n_phi", C.c_int32), ("n_psi", C.c_int32),
                ("phi_r", C.c_double * EAM_MAX_KNOTS), ("phi_a", C.c_double * EAM_MAX_KNOTS),
                ("psi_r", C.c_double * EAM_MAX_KNOTS), ("psi_a", C.c_double * EAM_MAX_KNOTS),
                ("F_sqrt", C.c_double), ("F_quad", C.c_double)]


def make_eam(phi_r, phi_a, psi_r, psi_a, F_sqrt, F_quad) -> EamTable:
    t = EamTable()
    t.n_phi, t.n_psi = len(phi_r), len(psi_r)
    for k, (r, a) in enumerate(zip(phi_r, phi_a)):
        t.phi_r[k], t.phi_a[k] = r, a
    for k, (r, a) in enumerate(zip(psi_r, psi_a)):
        t.psi_r[k], t.psi_a[k] = r, a
    t.F_sqrt, t.F_quad = F_sqrt, F_quad
    return t


class Params(C.Structure):
    _fields_ = [("potential", C.c_int32), ("rebuild_every", C.c_int32),
                ("eps", C.c_double), ("sigma", C.c_double), ("c", C.c_double),
                ("n_exp", C.c_double), ("m_exp", C.c_double), ("rc", C.c_double),
                ("skin", C.c_double), ("dt", C.c_double), ("mass", C.c_double),
                ("eam", C.POINTER(EamTable)),
                ("ntypes", C.c_int32), ("types", C.POINTER(C.c_int32)),
                ("t_eps", C.POINTER(C.c_double)), ("t_sigma", C.POINTER(C.c_double)),
                ("t_mass", C.POINTER(C.c_double))]


def make_params(potential=POT_LJ, eps=1.0, sigma=1.0, c=0.0, n_exp=12.0, m_exp=6.0,
                rc=2.5, skin=0.3, dt=0.005, mass=1.0, rebuild_every=0, eam=None,
                types=None, t_eps=None, t_sigma=None, t_mass=None) -> Params:
    """eam: an EamTable (potential POT_EAM).  types (n int32 species),
    t_eps / t_sigma (nt x nt) and t_mass (nt): a multi-element Lennard-Jones
    system.  The arrays are kept alive by the returned Params."""
    p = Params(potential, rebuild_every, eps, sigma, c, n_exp, m_exp, rc, skin, dt, mass,
               C.pointer(eam) if eam is not None else None)
    p._eam_ref = eam
    if types is not None:
        tt = np.ascontiguousarray(types, np.int32)
        te = np.ascontiguousarray(t_eps, np.float64).ravel()
        ts = np.ascontiguousarray(t_sigma, np.float64).ravel()
        tm = np.ascontiguousarray(t_mass, np.float64).ravel()
        assert te.size == ts.size == tm.size ** 2
        p.ntypes = tm.size
        p.types, p.t_eps = _P(tt, C.c_int32), _P(te, C.c_double)
        p.t_sigma, p.t_mass = _P(ts, C.c_double), _P(tm, C.c_double)
        p._typed_ref = (tt, te, ts, tm)
    return p


def _P(a, dtype):
    return a.ctypes.data_as(C.POINTER(dtype))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            d, i64, i32 = C.c_double, C.c_int64, C.c_int32
            pd, pi64, pi32 = C.POINTER(d), C.POINTER(i64), C.POINTER(i32)
            L.orc_pair_r2.restype = d
            L.orc_pair_r2.argtypes = [pd, pd, i64, i64]
            L.orc_cell_grid.restype = C.c_int
            L.orc_cell_grid.argtypes = [pd, d, pi32, pd]
            L.orc_bin.restype = C.c_int
            L.orc_bin.argtypes = [i64, pd, pi32, pd, pi32, pi64, pi64]
            for fn in (L.orc_neighbors_brute, L.orc_neighbors_cells):
                fn.restype = i64
                fn.argtypes = [i64, pd, pd, d, C.c_int, pi64, pi32, i64]
            L.orc_lj_brute.restype = d
            L.orc_lj_brute.argtypes = [i64, pd, pd, d, d, d, pd]
            L.orc_lj_list.restype = d
            L.orc_lj_list.argtypes = [i64, pd, pd, d, d, d, pi64, pi32, pd, pd]
            L.orc_sc_list.restype = d
            L.orc_sc_list.argtypes = [i64, pd, pd, d, d, d, d, d, d, pi64, pi32, pd, pd, pd, pd]
            L.orc_sc_brute.restype = d
            L.orc_sc_brute.argtypes = [i64, pd, pd, d, d, d, d, d, d, pd, pd]
            L.orc_lj_typed_brute.restype = d
            L.orc_lj_typed_brute.argtypes = [i64, pd, pd, i32, pi32, pd, pd, d, pd]
            L.orc_lj_typed_list.restype = d
            L.orc_lj_typed_list.argtypes = [i64, pd, pd, i32, pi32, pd, pd, d, pi64, pi32, pd, pd]
            L.orc_eam_list.restype = d
            L.orc_eam_list.argtypes = [i64, pd, pd, C.POINTER(EamTable), d, pi64, pi32, pd, pd,
                                       pd, pd]
            L.orc_eam_brute.restype = d
            L.orc_eam_brute.argtypes = [i64, pd, pd, C.POINTER(EamTable), d, pd, pd]
            L.orc_md_run.restype = i64
            L.orc_md_run.argtypes = [C.POINTER(Params), i64, pd, pd, pd, i64, pd, pd]
            L.orc_forces_once.restype = d
            L.orc_forces_once.argtypes = [C.POINTER(Params), i64, pd, pd, pd]
            L.orc_mlp_nparams.restype = C.c_int
            L.orc_mlp_forward.restype = None
            L.orc_mlp_forward.argtypes = [i64, pd, pd, pd]
            L.orc_mlp_loss_grad.restype = d
            L.orc_mlp_loss_grad.argtypes = [i64, pd, pd, pd, pd]
            L.orc_adam.restype = None
            L.orc_adam.argtypes = [i64, pd, pd, pd, pd, i64, d, d, d, d]
            L.orc_partition.restype = None
            L.orc_partition.argtypes = [i64, pi64, i32, pi64]
        return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle's per-atom loops may use."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))
    try:
        libgomp = C.CDLL("libgomp.so.1")
        libgomp.omp_set_num_threads(C.c_int(int(n)))
    except OSError:
        pass


def pair_r2(pos, box, i, j) -> float:
    pos, box = _f64(pos, (-1, 3)), _f64(box, (3,))
    return lib().orc_pair_r2(_P(pos, C.c_double), _P(box, C.c_double), i, j)


def cell_grid(box, r_list):
    box = _f64(box, (3,))
    ncell = np.zeros(3, np.int32)
    inv_w = np.zeros(3, np.float64)
    st = lib().orc_cell_grid(_P(box, C.c_double), float(r_list), _P(ncell, C.c_int32),
                             _P(inv_w, C.c_double))
    if st != 0:
        raise ValueError("invalid box / r_list")
    return ncell, inv_w


def bin_cells(pos, box, r_list):
    """Returns (ncell[3], cell_of_atom[n], cell_start[ncells+1], order[n])."""
    pos = _f64(pos, (-1, 3))
    n = pos.shape[0]
    ncell, inv_w = cell_grid(box, r_list)
    ncells = int(np.prod(ncell.astype(np.int64)))
    cell_of = np.zeros(n, np.int32)
    start = np.zeros(ncells + 1, np.int64)
    order = np.zeros(n, np.int64)
    lib().orc_bin(n, _P(pos, C.c_double), _P(ncell, C.c_int32), _P(inv_w, C.c_double),
                  _P(cell_of, C.c_int32), _P(start, C.c_int64), _P(order, C.c_int64))
    return ncell, cell_of, start, order


def _neighbors(fn, pos, box, r_list, half):
    pos, box = _f64(pos, (-1, 3)), _f64(box, (3,))
    n = pos.shape[0]
    offsets = np.zeros(n + 1, np.int64)
    cap = max(1024, 96 * n)
    while True:
        ids = np.zeros(cap, np.int32)
        t = fn(n, _P(pos, C.c_double), _P(box, C.c_double), float(r_list), int(bool(half)),
               _P(offsets, C.c_int64), _P(ids, C.c_int32), cap)
        if t >= 0:
            return offsets, ids[:t].copy()
        if t != -4:
            raise ValueError("neighbour list failed (%d)" % t)
        cap = int(offsets[-1]) + 1024 if offsets[-1] > cap else 2 * cap


def neighbors_brute(pos, box, r_list, half=False):
    """CSR (offsets[n+1], ids) of {j != i : r_ij^2 < r_list^2}, ascending j."""
    return _neighbors(lib().orc_neighbors_brute, pos, box, r_list, half)


def neighbors_cells(pos, box, r_list, half=False):
    """Same set as neighbors_brute, found with the 27-cell stencil."""
    return _neighbors(lib().orc_neighbors_cells, pos, box, r_list, half)


def lj_brute(pos, box, eps=1.0, sigma=1.0, rc=2.5):
    pos, box = _f64(pos, (-1, 3)), _f64(box, (3,))
    f = np.zeros_like(pos)
    U = lib().orc_lj_brute(pos.shape[0], _P(pos, C.c_double), _P(box, C.c_double), eps, sigma,
                           rc, _P(f, C.c_double))
    return U, f


def lj_list(pos, box, offsets, ids, eps=1.0, sigma=1.0, rc=2.5, per_atom=False):
    pos, box = _f64(pos, (-1, 3)), _f64(box, (3,))
    offsets = np.ascontiguousarray(offsets, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    f = np.zeros_like(pos)
    e = np.zeros(pos.shape[0]) if per_atom else None
    U = lib().orc_lj_list(pos.shape[0], _P(pos, C.c_double), _P(box, C.c_double), eps, sigma,
                          rc, _P(offsets, C.c_int64), _P(ids, C.c_int32), _P(f, C.c_double),
                          _P(e, C.c_double) if per_atom else None)
    return (U, f, e) if per_atom else (U, f)


def sc_list(pos, box, offsets, ids, eps=1.0, a=1.0, c=39.432, n_exp=9.0, m_exp=6.0, rc=2.0,
            per_atom=False):
    """Returns (U, f, rho, dF) from a full list, and the per-atom energies
    as a fifth value when per_atom is set."""
    pos, box = _f64(pos, (-1, 3)), _f64(box, (3,))
    offsets = np.ascontiguousarray(offsets, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    n = pos.shape[0]
    f = np.zeros_like(pos)
    rho = np.zeros(n)
    dF = np.zeros(n)
    e = np.zeros(n) if per_atom else None
    U = lib().orc_sc_list(n, _P(pos, C.c_double), _P(box, C.c_double), eps, a, c, n_exp, m_exp,
                          rc, _P(offsets, C.c_int64), _P(ids, C.c_int32), _P(f, C.c_double),
                          _P(rho, C.c_double), _P(dF, C.c_double),
                          _P(e, C.c_double) if per_atom else None)
    return (U, f, rho, dF, e) if per_atom else (U, f, rho, dF)


def sc_brute(pos, box, eps=1.0, a=1.0, c=39.432, n_exp=9.0, m_exp=6.0, rc=2.0):
    pos, box = _f64(pos, (-1, 3)), _f64(box, (3,))
    f = np.zeros_like(pos)
    rho = np.zeros(pos.shape[0])
    U = lib().orc_sc_brute(pos.shape[0], _P(pos, C.c_double), _P(box, C.c_double), eps, a, c,
                           n_exp, m_exp, rc, _P(f, C.c_double), _P(rho, C.c_double))
    return U, f, rho


def lj_typed_brute(pos, box, types, t_eps, t_sigma, rc=2.5):
    """Multi-element LJ over all pairs: (U, f)."""
    pos, box = _f64(pos, (-1, 3)), _f64(box, (3,))
    tt = np.ascontiguousarray(types, np.int32)
    te, ts = _f64(t_eps).ravel(), _f64(t_sigma).ravel()
    nt = int(round(te.size ** 0.5))
    f = np.zeros_like(pos)
    U = lib().orc_lj_typed_brute(pos.shape[0], _P(pos, C.c_double), _P(box, C.c_double), nt,
                                 _P(tt, C.c_int32), _P(te, C.c_double), _P(ts, C.c_double), rc,
                                 _P(f, C.c_double))
    return U, f


def lj_typed_list(pos, box, offsets, ids, types, t_eps, t_sigma, rc=2.5):
    """Multi-element LJ from a full list: (U, f, e_atom)."""
    pos, box = _f64(pos, (-1, 3)), _f64(box, (3,))
    offsets = np.ascontiguousarray(offsets, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    tt = np.ascontiguousarray(types, np.int32)
    te, ts = _f64(t_eps).ravel(), _f64(t_sigma).ravel()
    nt = int(round(te.size ** 0.5))
    f = np.zeros_like(pos)
    e = np.zeros(pos.shape[0])
    U = lib().orc_lj_typed_list(pos.shape[0], _P(pos, C.c_double), _P(box, C.c_double), nt,
                                _P(tt, C.c_int32), _P(te, C.c_double), _P(ts, C.c_double), rc,
                                _P(offsets, C.c_int64), _P(ids, C.c_int32), _P(f, C.c_double),
                                _P(e, C.c_double))
    return U, f, e


def eam_list(pos, box, offsets, ids, table: EamTable, rc):
    """Returns (U, f, rho, dF, e_atom) from a full list."""
    pos, box = _f64(pos, (-1, 3)), _f64(box, (3,))
    offsets = np.ascontiguousarray(offsets, np.int64)
    ids = np.ascontiguousarray(ids, np.int32)
    n = pos.shape[0]
    f = np.zeros_like(pos)
    rho, dF, e = np.zeros(n), np.zeros(n), np.zeros(n)
    U = lib().orc_eam_list(n, _P(pos, C.c_double), _P(box, C.c_double), C.byref(table), rc,
                           _P(offsets, C.c_int64), _P(ids, C.c_int32), _P(f, C.c_double),
                           _P(rho, C.c_double), _P(dF, C.c_double), _P(e, C.c_double))
    return U, f, rho, dF, e


def eam_brute(pos, box, table: EamTable, rc):
    """Returns (U, f, rho) over all pairs."""
    pos, box = _f64(pos, (-1, 3)), _f64(box, (3,))
    f = np.zeros_like(pos)
    rho = np.zeros(pos.shape[0])
    U = lib().orc_eam_brute(pos.shape[0], _P(pos, C.c_double), _P(box, C.c_double),
                            C.byref(table), rc, _P(f, C.c_double), _P(rho, C.c_double))
    return U, f, rho


def md_run(params: Params, pos, vel, box, nsteps, want_energies=True):
    """nsteps velocity-Verlet steps on copies of pos/vel.

    Returns dict(pos, vel, force, energies[(nsteps+1) x 3] = KE, PE, KE+PE,
    builds)."""
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    box = _f64(box, (3,))
    n = pos.shape[0]
    E = np.zeros((nsteps + 1, 3)) if want_energies else None
    f = np.zeros_like(pos)
    b = lib().orc_md_run(C.byref(params), n, _P(pos, C.c_double), _P(vel, C.c_double),
                         _P(box, C.c_double), int(nsteps),
                         _P(E, C.c_double) if want_energies else None, _P(f, C.c_double))
    if b < 0:
        raise RuntimeError("oracle md_run failed (%d)" % b)
    return {"pos": pos, "vel": vel, "force": f, "energies": E, "builds": int(b)}


def melt(params: Params, pos, vel, box, schedule, every, rescale):
    """Runs md_run in chunks of `every` steps over the (T, steps) stages of
    `schedule`, with rescale(vel, T) applied before every chunk and once at
    the end (the velocity rescaling of an input protocol, supplied by the
    caller).  Returns (pos, vel)."""
    for T, nsteps in schedule:
        for _ in range(nsteps // every):
            vel = rescale(vel, T)
            out = md_run(params, pos, vel, box, every, want_energies=False)
            pos, vel = out["pos"], out["vel"]
    return pos, rescale(vel, schedule[-1][0])


def forces_once(params: Params, pos, box):
    pos, box = _f64(pos, (-1, 3)), _f64(box, (3,))
    f = np.zeros_like(pos)
    U = lib().orc_forces_once(C.byref(params), pos.shape[0], _P(pos, C.c_double),
                              _P(box, C.c_double), _P(f, C.c_double))
    return U, f


# ---- cost model -----------------------------------------------------------

MLP_HIDDEN = 32


def mlp_nparams() -> int:
    return int(lib().orc_mlp_nparams())


def mlp_forward(X, P):
    X = _f64(X, (-1, 3))
    P = _f64(P)
    y = np.zeros(X.shape[0])
    lib().orc_mlp_forward(X.shape[0], _P(X, C.c_double), _P(P, C.c_double), _P(y, C.c_double))
    return y


def mlp_loss_grad(X, y, P):
    X = _f64(X, (-1, 3))
    y = _f64(y)
    P = _f64(P)
    G = np.zeros_like(P)
    loss = lib().orc_mlp_loss_grad(X.shape[0], _P(X, C.c_double), _P(y, C.c_double),
                                   _P(P, C.c_double), _P(G, C.c_double))
    return loss, G


def adam(P, G, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays P, m, v."""
    for a in (P, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    G = _f64(G)
    lib().orc_adam(P.size, _P(P, C.c_double), _P(G, C.c_double), _P(m, C.c_double),
                   _P(v, C.c_double), int(t), lr, beta1, beta2, eps)


def partition(cost, nparts):
    cost = np.ascontiguousarray(cost, np.int64)
    bounds = np.zeros(nparts + 1, np.int64)
    lib().orc_partition(cost.size, _P(cost, C.c_int64), int(nparts), _P(bounds, C.c_int64))
    return bounds


def _sample_sigs():
    L = lib()
    if getattr(L, "_sample_ready", False):
        return L
    d, i64 = C.c_double, C.c_int64
    pd, pi64, pi32 = C.POINTER(d), C.POINTER(i64), C.POINTER(C.c_int32)
    L.orc_forces_sample.restype = C.c_int
    L.orc_forces_sample.argtypes = [C.POINTER(Params), i64, pd, pd, i64, pi64, pd, pd]
    L.orc_neighbors_sample.restype = i64
    L.orc_neighbors_sample.argtypes = [i64, pd, pd, d, i64, pi64, pi64, pi32, i64]
    L._sample_ready = True
    return L


def forces_sample(params: Params, pos, box, idx):
    """Forces and per-atom energies of the atoms idx (original ids) only."""
    L = _sample_sigs()
    pos, box = _f64(pos, (-1, 3)), _f64(box, (3,))
    idx = np.ascontiguousarray(idx, np.int64)
    f = np.zeros((idx.size, 3))
    e = np.zeros(idx.size)
    st = L.orc_forces_sample(C.byref(params), pos.shape[0], _P(pos, C.c_double),
                             _P(box, C.c_double), idx.size, _P(idx, C.c_int64),
                             _P(f, C.c_double), _P(e, C.c_double))
    if st != 0:
        raise RuntimeError("oracle forces_sample failed (%d)" % st)
    return f, e


def neighbors_sample(pos, box, r_list, idx, cap=None):
    """List rows (ascending original id) of the sampled atoms idx; cap is the
    room for entries in all (default 512 per sampled atom)."""
    L = _sample_sigs()
    pos, box = _f64(pos, (-1, 3)), _f64(box, (3,))
    idx = np.ascontiguousarray(idx, np.int64)
    off = np.zeros(idx.size + 1, np.int64)
    cap = int(cap) if cap is not None else 512 * max(1, idx.size)
    ids = np.zeros(cap, np.int32)
    t = L.orc_neighbors_sample(pos.shape[0], _P(pos, C.c_double), _P(box, C.c_double),
                               float(r_list), idx.size, _P(idx, C.c_int64), _P(off, C.c_int64),
                               _P(ids, C.c_int32), cap)
    if t < 0:
        raise RuntimeError("oracle neighbors_sample failed (%d)" % t)
    return off, ids[:t].copy()
