"""Python binding of the C ABI in include/md_gb300.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: torch tensors supply device memory and the CUDA
stream, and their data pointers are handed to the library.  Importing this
module loads lib/libmd_gb300.so and fails loudly if it is missing; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmd_gb300.so")

MD_OK = 0
MD_ERR_INVALID = -1
MD_ERR_OOM = -2
MD_ERR_CUDA = -3
MD_ERR_LIST_OVERFLOW = -4
MD_ERR_NONFINITE = -5
MD_ERR_TIMEOUT = -6
MD_ERR_STATE = -7
STATUS_NAMES = {0: "MD_OK", -1: "MD_ERR_INVALID", -2: "MD_ERR_OOM", -3: "MD_ERR_CUDA",
                -4: "MD_ERR_LIST_OVERFLOW", -5: "MD_ERR_NONFINITE", -6: "MD_ERR_TIMEOUT",
                -7: "MD_ERR_STATE"}

MD_POT_LJ, MD_POT_SC, MD_POT_EAM = 0, 1, 2
MD_EAM_MAX_KNOTS = 16
MD_FP64, MD_MIXED = 0, 1
MD_FORCE_FULL, MD_FORCE_HALF_COLOR, MD_FORCE_HALF_ATOMIC, MD_FORCE_CLUSTER, MD_FORCE_PAIRED = 0, 1, 2, 3, 4
MD_SCHED_GRID, MD_SCHED_PAIRCOUNT, MD_SCHED_MLP, MD_SCHED_DYNAMIC = 0, 1, 2, 3
MD_COST_TRAIN, MD_COST_PREDICT, MD_COST_RESET, MD_COST_SAMPLE, MD_COST_PROFILE = 0, 1, 2, 3, 4
MLP_NPARAMS = 1217


class MDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class md_params(C.Structure):
    _fields_ = [("potential", C.c_int32), ("precision", C.c_int32),
                ("force_variant", C.c_int32), ("rebuild_every", C.c_int32),
                ("scheduler", C.c_int32), ("max_neighbors", C.c_int32),
                ("reserved0", C.c_int32), ("reserved1", C.c_int32),
                ("eps", C.c_double), ("sigma", C.c_double), ("c", C.c_double),
                ("n_exp", C.c_double), ("m_exp", C.c_double), ("rc", C.c_double),
                ("skin", C.c_double), ("dt", C.c_double), ("mass", C.c_double)]


class md_eam(C.Structure):
    _fields_ = [("n_phi", C.c_int32), ("n_psi", C.c_int32),
                ("phi_r", C.c_double * MD_EAM_MAX_KNOTS), ("phi_a", C.c_double * MD_EAM_MAX_KNOTS),
                ("psi_r", C.c_double * MD_EAM_MAX_KNOTS), ("psi_a", C.c_double * MD_EAM_MAX_KNOTS),
                ("F_sqrt", C.c_double), ("F_quad", C.c_double)]


MD_MAX_TYPES = 4


class md_lj_types(C.Structure):
    _fields_ = [("ntypes", C.c_int32), ("reserved", C.c_int32),
                ("eps", C.c_double * (MD_MAX_TYPES * MD_MAX_TYPES)),
                ("sigma", C.c_double * (MD_MAX_TYPES * MD_MAX_TYPES)),
                ("mass", C.c_double * MD_MAX_TYPES)]


def make_lj_types(t_eps, t_sigma, t_mass) -> md_lj_types:
    """Species table from nt x nt eps and sigma and nt masses (nested lists or arrays)."""
    t = md_lj_types()
    nt = len(t_mass)
    t.ntypes = nt
    for a in range(nt):
        t.mass[a] = float(t_mass[a])
        for b in range(nt):
            t.eps[a * nt + b] = float(t_eps[a][b])
            t.sigma[a * nt + b] = float(t_sigma[a][b])
    return t


def make_eam(phi_r, phi_a, psi_r, psi_a, F_sqrt, F_quad) -> md_eam:
    t = md_eam()
    t.n_phi, t.n_psi = len(phi_r), len(psi_r)
    for k, (r, a) in enumerate(zip(phi_r, phi_a)):
        t.phi_r[k], t.phi_a[k] = r, a
    for k, (r, a) in enumerate(zip(psi_r, psi_a)):
        t.psi_r[k], t.psi_a[k] = r, a
    t.F_sqrt, t.F_quad = F_sqrt, F_quad
    return t


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("CUDA library %s is missing: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "md_create": [C.POINTER(vp), C.POINTER(md_params), i64, vp, vp, vp, vp],
        "md_create_eam": [C.POINTER(vp), C.POINTER(md_params), C.POINTER(md_eam), i64, vp, vp,
                          vp, vp],
        "md_create_typed": [C.POINTER(vp), C.POINTER(md_params), C.POINTER(md_lj_types), vp,
                            i64, vp, vp, vp, vp],
        "md_bin_cells": [vp], "md_build_neighbors": [vp], "md_forces": [vp],
        "md_step": [vp, i64], "md_energy": [vp, vp, vp],
        "md_get_state": [vp, vp, vp, vp], "md_set_state": [vp, vp, vp],
        "md_get_neighbors": [vp, i32, vp, vp, i64, vp],
        "md_get_cells": [vp, vp, vp, vp], "md_get_density": [vp, vp, vp],
        "md_get_atom_energy": [vp, vp], "md_set_variant": [vp, i32, i32],
        "md_cost_model": [vp, i32, vp], "md_stats": [vp, C.c_char_p, C.c_size_t],
        "md_set_timing": [vp, i32], "md_color_cells": [vp, vp, vp],
        "md_set_schedule": [vp, i32, i32],
        "md_set_decomposition": [vp, i32, i32, i32],
        "md_get_cell_costs": [vp, vp, vp, vp],
        "md_create_batch": [C.POINTER(vp), C.POINTER(md_params), i32, vp, vp, vp, vp, vp],
        "md_energy_batch": [vp, vp, vp],
        "md_mlp_forward": [vp, i64, vp, vp, vp],
        "md_mlp_loss_grad": [vp, vp, i64, vp, vp, vp, vp],
        "md_mlp_adam": [vp, vp, vp, vp, i64, i64, C.c_float, C.c_float, C.c_float,
                        C.c_float, vp],
        "md_partition": [vp, i64, i32, vp, vp],
        "md_partition_noalloc": [vp, i64, i32, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.md_last_error.argtypes = [vp]
    L.md_last_error.restype = C.c_char_p
    L.md_destroy.argtypes = [vp]
    L.md_destroy.restype = None
    _lib = L
    return L


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream) -> int | None:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check(st: int, h=None, what: str = ""):
    if st != MD_OK:
        msg = lib().md_last_error(h)
        raise MDError(st, (what + ": " if what else "") + (msg.decode() if msg else ""))


def make_params(potential="lj", precision="mixed", force_variant=MD_FORCE_FULL,
                rebuild_every=0, scheduler=MD_SCHED_GRID, max_neighbors=0, eps=1.0, sigma=1.0,
                c=0.0, n_exp=12.0, m_exp=6.0, rc=2.5, skin=0.3, dt=0.005, mass=1.0,
                **_ignored) -> md_params:
    pot = {"lj": MD_POT_LJ, "sc": MD_POT_SC, "eam": MD_POT_EAM}.get(potential, potential)
    prec = {"fp64": MD_FP64, "mixed": MD_MIXED}.get(precision, precision)
    return md_params(pot, prec, force_variant, rebuild_every, scheduler, max_neighbors, 0, 0,
                     eps, sigma, c, n_exp, m_exp, rc, skin, dt, mass)


# ---- the C entry points ------------------------------------------------------

def md_create(params: md_params, pos: torch.Tensor, vel: torch.Tensor | None, box,
              stream=None) -> int:
    n = pos.shape[0]
    assert pos.dtype == torch.float64 and pos.shape == (n, 3)
    box_arr = (C.c_double * 3)(*[float(b) for b in box])
    h = C.c_void_p()
    st = lib().md_create(C.byref(h), C.byref(params), n, C.cast(box_arr, C.c_void_p),
                         _ptr(pos), _ptr(vel), _stream(stream))
    _check(st, None, "md_create")
    return h.value


def md_create_eam(params: md_params, eam: md_eam, pos: torch.Tensor, vel: torch.Tensor | None,
                  box, stream=None) -> int:
    n = pos.shape[0]
    assert pos.dtype == torch.float64 and pos.shape == (n, 3)
    box_arr = (C.c_double * 3)(*[float(b) for b in box])
    h = C.c_void_p()
    st = lib().md_create_eam(C.byref(h), C.byref(params), C.byref(eam), n,
                             C.cast(box_arr, C.c_void_p), _ptr(pos), _ptr(vel), _stream(stream))
    _check(st, None, "md_create_eam")
    return h.value


def md_create_typed(params: md_params, types: md_lj_types, type_dev: torch.Tensor,
                    pos: torch.Tensor, vel: torch.Tensor | None, box, stream=None) -> int:
    n = pos.shape[0]
    assert pos.dtype == torch.float64 and pos.shape == (n, 3)
    assert type_dev.dtype == torch.int32 and type_dev.numel() == n
    box_arr = (C.c_double * 3)(*[float(b) for b in box])
    h = C.c_void_p()
    st = lib().md_create_typed(C.byref(h), C.byref(params), C.byref(types), _ptr(type_dev), n,
                               C.cast(box_arr, C.c_void_p), _ptr(pos), _ptr(vel),
                               _stream(stream))
    _check(st, None, "md_create_typed")
    return h.value


def md_create_batch(params: md_params, n_each, pos: torch.Tensor, vel, boxes,
                    stream=None) -> int:
    R = len(n_each)
    ne = (C.c_int64 * R)(*[int(x) for x in n_each])
    bx = (C.c_double * (3 * R))(*[float(b) for box in boxes for b in box])
    h = C.c_void_p()
    st = lib().md_create_batch(C.byref(h), C.byref(params), R, C.cast(ne, C.c_void_p),
                               C.cast(bx, C.c_void_p), _ptr(pos), _ptr(vel), _stream(stream))
    _check(st, None, "md_create_batch")
    return h.value


def md_energy_batch(h, R: int):
    ke = (C.c_double * R)()
    pe = (C.c_double * R)()
    _check(lib().md_energy_batch(h, C.cast(ke, C.c_void_p), C.cast(pe, C.c_void_p)), h,
           "md_energy_batch")
    return list(ke), list(pe)


def md_bin_cells(h):
    _check(lib().md_bin_cells(h), h, "md_bin_cells")


def md_build_neighbors(h):
    _check(lib().md_build_neighbors(h), h, "md_build_neighbors")


def md_forces(h):
    _check(lib().md_forces(h), h, "md_forces")


def md_step(h, nsteps: int):
    _check(lib().md_step(h, int(nsteps)), h, "md_step")


def md_energy(h):
    ke, pe = C.c_double(), C.c_double()
    _check(lib().md_energy(h, C.byref(ke), C.byref(pe)), h, "md_energy")
    return ke.value, pe.value


def md_get_state(h, pos=None, vel=None, force=None):
    _check(lib().md_get_state(h, _ptr(pos), _ptr(vel), _ptr(force)), h, "md_get_state")


def md_set_state(h, pos=None, vel=None):
    _check(lib().md_set_state(h, _ptr(pos), _ptr(vel)), h, "md_set_state")


def md_get_neighbors(h, half: int, offsets: torch.Tensor, ids: torch.Tensor | None, cap: int):
    total = C.c_int64()
    st = lib().md_get_neighbors(h, int(half), _ptr(offsets), _ptr(ids), int(cap),
                                C.byref(total))
    return st, total.value


def md_get_cells(h, cell_of_atom: torch.Tensor, cell_start: torch.Tensor | None):
    nc = (C.c_int32 * 3)()
    _check(lib().md_get_cells(h, _ptr(cell_of_atom), _ptr(cell_start), C.cast(nc, C.c_void_p)),
           h, "md_get_cells")
    return [nc[0], nc[1], nc[2]]


def md_get_density(h, rho=None, dF=None):
    _check(lib().md_get_density(h, _ptr(rho), _ptr(dF)), h, "md_get_density")


def md_get_atom_energy(h, e):
    _check(lib().md_get_atom_energy(h, _ptr(e)), h, "md_get_atom_energy")


def md_set_variant(h, force_variant: int, scheduler: int):
    _check(lib().md_set_variant(h, int(force_variant), int(scheduler)), h, "md_set_variant")


def md_set_schedule(h, rounds: int, tail_percent: int):
    _check(lib().md_set_schedule(h, int(rounds), int(tail_percent)), h, "md_set_schedule")


def md_set_decomposition(h, px: int, py: int, pz: int):
    _check(lib().md_set_decomposition(h, int(px), int(py), int(pz)), h, "md_set_decomposition")


def md_cost_model(h, op: int) -> float:
    loss = C.c_float(float("nan"))
    _check(lib().md_cost_model(h, int(op), C.byref(loss)), h, "md_cost_model")
    return loss.value


def md_get_cell_costs(h, cycles=None, predicted=None, paircount=None):
    _check(lib().md_get_cell_costs(h, _ptr(cycles), _ptr(predicted), _ptr(paircount)), h,
           "md_get_cell_costs")


def md_set_timing(h, on: bool):
    _check(lib().md_set_timing(h, int(bool(on))), h, "md_set_timing")


def md_color_cells(ncell):
    """Cell colours of the half-list colouring (host call, no GPU); returns a
    list of int colours in linear cell order and the colour count."""
    nc = (C.c_int32 * 3)(*[int(x) for x in ncell])
    total = int(ncell[0]) * int(ncell[1]) * int(ncell[2])
    col = (C.c_int32 * total)()
    k = C.c_int32()
    _check(lib().md_color_cells(C.cast(nc, C.c_void_p), C.cast(col, C.c_void_p), C.byref(k)),
           None, "md_color_cells")
    return list(col), k.value


def md_stats(h) -> str:
    buf = C.create_string_buffer(4096)
    _check(lib().md_stats(h, buf, 4096), h, "md_stats")
    return buf.value.decode()


def md_destroy(h):
    if h:
        lib().md_destroy(h)


def md_mlp_forward(X: torch.Tensor, P: torch.Tensor, y: torch.Tensor, stream=None):
    _check(lib().md_mlp_forward(_ptr(X), X.shape[0], _ptr(P), _ptr(y), _stream(stream)),
           None, "md_mlp_forward")


def md_mlp_loss_grad(X, y, P, G, loss, stream=None):
    _check(lib().md_mlp_loss_grad(_ptr(X), _ptr(y), X.shape[0], _ptr(P), _ptr(G), _ptr(loss),
                                  _stream(stream)), None, "md_mlp_loss_grad")


def md_mlp_adam(P, G, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().md_mlp_adam(_ptr(P), _ptr(G), _ptr(m), _ptr(v), P.numel(), int(t), lr, beta1,
                             beta2, eps, _stream(stream)), None, "md_mlp_adam")


def _partition_args(cost, nparts, bounds, what):
    """The C calls read cost as ncells int64 words and write nparts + 1 int64
    bounds on the device: anything else is refused before the call."""
    for name, t, need in (("cost", cost, 1), ("bounds", bounds, int(nparts) + 1)):
        if (not isinstance(t, torch.Tensor) or t.dtype != torch.int64 or not t.is_cuda
                or not t.is_contiguous() or t.numel() < need):
            raise MDError(MD_ERR_INVALID, "%s: %s must be a contiguous int64 CUDA tensor of at "
                                          "least %d elements" % (what, name, need))


def md_partition(cost: torch.Tensor, nparts: int, bounds: torch.Tensor, stream=None):
    _partition_args(cost, nparts, bounds, "md_partition")
    _check(lib().md_partition(_ptr(cost), cost.numel(), int(nparts), _ptr(bounds),
                              _stream(stream)), None, "md_partition")


def md_partition_noalloc(cost: torch.Tensor, nparts: int, bounds: torch.Tensor, stream=None):
    """md_partition without any device allocation (fixed scratch inside the
    library; ncells <= 1,048,576; overlapping calls race on the scratch)."""
    _partition_args(cost, nparts, bounds, "md_partition_noalloc")
    _check(lib().md_partition_noalloc(_ptr(cost), cost.numel(), int(nparts), _ptr(bounds),
                                      _stream(stream)), None, "md_partition_noalloc")


# ---- convenience wrapper -----------------------------------------------------

class System:
    """Owns one md_system handle.  pos/vel: (n, 3) float64 tensors (any device;
    copied to the GPU), box: 3 floats, params: md_params or keyword dict."""

    def __init__(self, pos, vel, box, params=None, stream=None, eam=None, species=None, **kw):
        """eam: an md_eam table (or a dict of make_eam's arguments) for the
        embedded-atom potential (md_create_eam).  species: (types, t_eps,
        t_sigma, t_mass) of a multi-element Lennard-Jones system
        (md_create_typed)."""
        self.h = None
        if eam is not None:
            kw.setdefault("potential", "eam")
            if isinstance(eam, dict):
                eam = make_eam(*[eam[k] for k in ("phi_r", "phi_a", "psi_r", "psi_a",
                                                  "F_sqrt", "F_quad")])
        if params is None:
            params = make_params(**kw)
        elif isinstance(params, dict):
            params = make_params(**params)
        self.params = params
        self.stream = stream
        dev = torch.device("cuda", torch.cuda.current_device())
        p = torch.as_tensor(pos, dtype=torch.float64).to(dev).contiguous()
        v = None if vel is None else torch.as_tensor(vel, dtype=torch.float64).to(dev).contiguous()
        self.n = p.shape[0]
        self.box = [float(b) for b in box]
        if eam is not None:
            self.h = md_create_eam(params, eam, p, v, self.box, stream)
        elif species is not None:
            types, t_eps, t_sigma, t_mass = species
            td = torch.as_tensor(types, dtype=torch.int32).to(dev).contiguous()
            self.h = md_create_typed(params, make_lj_types(t_eps, t_sigma, t_mass), td, p, v,
                                     self.box, stream)
        else:
            self.h = md_create(params, p, v, self.box, stream)

    def close(self):
        if getattr(self, "h", None):
            md_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, n):
        md_step(self.h, n)

    def forces(self):
        md_forces(self.h)

    def energy(self):
        return md_energy(self.h)

    def state(self):
        dev = torch.device("cuda", torch.cuda.current_device())
        pos = torch.empty((self.n, 3), dtype=torch.float64, device=dev)
        vel = torch.empty_like(pos)
        f = torch.empty_like(pos)
        md_get_state(self.h, pos, vel, f)
        torch.cuda.synchronize()
        return pos, vel, f

    def neighbors(self, half=False):
        dev = torch.device("cuda", torch.cuda.current_device())
        off = torch.empty(self.n + 1, dtype=torch.int64, device=dev)
        st, total = md_get_neighbors(self.h, int(half), off, None, 0)
        if st not in (MD_OK, MD_ERR_LIST_OVERFLOW):
            _check(st, self.h, "md_get_neighbors")
        ids = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
        st, total = md_get_neighbors(self.h, int(half), off, ids, ids.numel())
        _check(st, self.h, "md_get_neighbors")
        return off, ids[:total]

    def cells(self):
        dev = torch.device("cuda", torch.cuda.current_device())
        cell_of = torch.empty(self.n, dtype=torch.int32, device=dev)
        nc = md_get_cells(self.h, cell_of, None)
        ncells = nc[0] * nc[1] * nc[2]
        start = torch.empty(ncells + 1, dtype=torch.int64, device=dev)
        md_get_cells(self.h, cell_of, start)
        return nc, cell_of, start

    def stats(self):
        import json
        return json.loads(md_stats(self.h))


class Batch(System):
    """Several independent replicas advanced as one system (md_create_batch).
    replicas: list of (pos, vel, box); atoms are concatenated in that order."""

    def __init__(self, replicas, params=None, stream=None, **kw):
        self.h = None
        if params is None:
            params = make_params(**kw)
        elif isinstance(params, dict):
            params = make_params(**params)
        self.params = params
        self.stream = stream
        dev = torch.device("cuda", torch.cuda.current_device())
        self.sizes = [int(len(r[0])) for r in replicas]
        self.offsets = [0]
        for n in self.sizes:
            self.offsets.append(self.offsets[-1] + n)
        p = torch.cat([torch.as_tensor(r[0], dtype=torch.float64) for r in replicas]).to(dev)
        v = torch.cat([torch.as_tensor(r[1], dtype=torch.float64) for r in replicas]).to(dev)
        self.n = p.shape[0]
        self.boxes = [[float(b) for b in r[2]] for r in replicas]
        self.box = self.boxes[0]
        self.h = md_create_batch(params, self.sizes, p.contiguous(), v.contiguous(), self.boxes,
                                 stream)

    def energies(self):
        return md_energy_batch(self.h, len(self.sizes))
