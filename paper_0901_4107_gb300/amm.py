"""Thin ctypes binding of libamm (include/amm.h).

Argument marshalling only: every step of the update runs in the library's
CUDA kernels.  The functions carry the C names; arrays are numpy (host) or,
for the *_device calls, integer device addresses (e.g. torch.Tensor.data_ptr()).
Errors raise AmmError with the library's status code and message.  If the
shared library has not been built this module raises on first use -- there
is no fallback.
"""
import ctypes
import os

import numpy as np

from . import _build

AMM_OK = 0
AMM_ERR_INVALID_ARG = -1
AMM_ERR_OPEN_CELL = -2
AMM_ERR_NONPOSITIVE_STATE = -3
AMM_ERR_CUDA = -4
AMM_ERR_NUMERIC = -5
AMM_ERR_NOT_READY = -6
AMM_ERR_TIMEOUT = -7

AMM_FP64, AMM_FP32, AMM_FP32_LEARNED = 0, 1, 2
AMM_EULERIAN, AMM_LAGRANGIAN, AMM_EXPLICIT_W = 0, 1, 2

PRECISIONS = {"fp64": AMM_FP64, "fp32": AMM_FP32, "fp32_learned": AMM_FP32_LEARNED}
MOTIONS = {"eulerian": AMM_EULERIAN, "lagrangian": AMM_LAGRANGIAN, "explicit": AMM_EXPLICIT_W}


class AmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libamm status %d: %s" % (code, msg))
        self.code = code


class amm_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("mesh_motion", ctypes.c_int), ("limiter", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("riemann_tol", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("n_boxes", ctypes.c_int64), ("box_cells", ctypes.POINTER(ctypes.c_int64)),
                ("box_faces", ctypes.POINTER(ctypes.c_int64)), ("fp64_accumulate", ctypes.c_int),
                ("entropy", ctypes.c_int), ("mach_thresh", ctypes.c_double), ("alpha_s", ctypes.c_double),
                ("regularize", ctypes.c_int), ("eta", ctypes.c_double), ("chi", ctypes.c_double)]


class amm_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("faces", ctypes.c_int64), ("newton_iters", ctypes.c_int64),
                ("newton_fail", ctypes.c_int64), ("fallback_faces", ctypes.c_int64),
                ("vacuum_faces", ctypes.c_int64), ("guard_faces", ctypes.c_int64),
                ("nonpositive_cells", ctypes.c_int64), ("newton_max", ctypes.c_int32), ("status", ctypes.c_uint32),
                ("newton_hist", ctypes.c_int64 * 16), ("entropy_kept", ctypes.c_int64)]


class amm_cycle_stats(ctypes.Structure):
    _fields_ = [("substeps", ctypes.c_int64), ("face_fluxes", ctypes.c_int64), ("activations", ctypes.c_int64),
                ("deepest_bin", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double

_SIGS = {
    "amm_default_options": (None, [_P]),
    "amm_last_error": (ctypes.c_char_p, [_P]),
    "amm_create": (_I, [ctypes.POINTER(_P), _I, _I64, _P, _I64, _P, _P, _P, _P, _P, _P, _D, _P]),
    "amm_create_device": (_I, [ctypes.POINTER(_P), _I, _I64, _P, _I64, _P, _P, _P, _P, _P, _P, _D, _P]),
    "amm_destroy": (_I, [_P]),
    "amm_set_state": (_I, [_P, _P]),
    "amm_set_state_device": (_I, [_P, _P]),
    "amm_set_mesh_velocity": (_I, [_P, _P]),
    "amm_gradients": (_I, [_P]),
    "amm_timestep": (_I, [_P, _D, _P]),
    "amm_step": (_I, [_P, _D]),
    "amm_step_boxes": (_I, [_P, _P]),
    "amm_advance": (_I, [_P, _D, _I64, _I]),
    "amm_tess_build": (_I, [ctypes.POINTER(_P), _I, _I64, _P, _P, _P]),
    "amm_tess_last_error": (ctypes.c_char_p, []),
    "amm_tess_num_faces": (_I64, [_P]),
    "amm_tess_faces": (_I, [_P, _P, _P, _P, _P]),
    "amm_tess_cells": (_I, [_P, _P, _P, _P]),
    "amm_tess_check": (_I, [_P, _P, _P]),
    "amm_tess_destroy": (_I, [_P]),
    "amm_retessellate": (_I, [_P]),
    "amm_get_num_faces": (_I64, [_P]),
    "amm_get_faces": (_I, [_P, _P, _P]),
    "amm_advance_individual": (_I, [_P, _D, _D, _I, _I, _P]),
    "amm_get_bins": (_I, [_P, _P]),
    "amm_individual_host_loop": (_I, [_P, _I]),
    "amm_drift": (_I, [_P, _D]),
    "amm_sync": (_I, [_P]),
    "amm_get_state": (_I, [_P, _P]),
    "amm_get_state_device": (_I, [_P, _P]),
    "amm_get_primitives": (_I, [_P, _P]),
    "amm_get_gradients": (_I, [_P, _P]),
    "amm_get_face_flux": (_I, [_P, _P]),
    "amm_get_geometry": (_I, [_P, _P, _P]),
    "amm_get_totals": (_I, [_P, _P]),
    "amm_get_dt": (_I, [_P, _P]),
    "amm_get_generators": (_I, [_P, _P]),
    "amm_get_stats": (_I, [_P, _P]),
    "amm_get_entropy": (_I, [_P, _P, _P]),
    "amm_set_entropy": (_I, [_P, _P]),
    "amm_reset_stats": (_I, [_P]),
    "amm_get_box_status": (_I, [_P, _P]),
    "amm_profile": (_I, [_P, _I]),
    "amm_set_tuning": (_I, [_P, _P]),
    "amm_get_tuning": (_I, [_P, _P]),
    "amm_autotune": (_I, [_P, _D, _I, _P]),
    "amm_timestep_noalloc": (_I, [_I, _I64, _P, _P, _P, _D, _D, _P, _P]),
    "amm_alu_peak": (_I, [_I, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_float), _P]),
    "amm_mlp_create": (_I, [ctypes.POINTER(_P), _D, _P]),
    "amm_mlp_destroy": (None, [_P]),
    "amm_mlp_last_error": (ctypes.c_char_p, [_P]),
    "amm_mlp_num_params": (_I, []),
    "amm_mlp_set_params": (_I, [_P, _P]),
    "amm_mlp_get_params": (_I, [_P, _P]),
    "amm_mlp_forward": (_I, [_P, _P, _I64, _P]),
    "amm_mlp_grads": (_I, [_P, _P, _P, _P, _I64, _P, _P]),
    "amm_mlp_train_step": (_I, [_P, _P, _P, _P, _I64, ctypes.c_float, _P]),
    "amm_mlp_sync": (_I, [_P]),
    "amm_mlp_attach": (_I, [_P, _P]),
    "amm_harvest": (_I, [_P, _D, _P]),
    "amm_mlp_features": (_I, [_D, _I64, _P, _P, _P, _P, _P, _P]),
    "amm_riemann_pstar": (_I, [_D, _I64, _P, _D, _P, _P]),
    "amm_mlp_targets": (_I, [_D, _I64, _P, _D, _P, _P]),
    "amm_get_kernel_times": (_I, [_P, _P]),
}


def library_path():
    return _build.LIB


def lib():
    """Loads libamm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libamm.so is not built (%s); run __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class Context:
    """Owns an amm_ctx*; remembers dim, sizes and boxes for the getters."""

    def __init__(self, handle, dim, n, nf, nboxes):
        self.handle = handle
        self.dim, self.n, self.nf, self.nboxes = dim, n, nf, nboxes

    def __del__(self):
        try:
            if self.handle:
                lib().amm_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def _check(ctx, rc):
    if rc != AMM_OK:
        h = ctx.handle if isinstance(ctx, Context) else ctx
        msg = lib().amm_last_error(h).decode() if h else ""
        raise AmmError(rc, msg)


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def amm_default_options(precision="fp64", mesh_motion="lagrangian", limiter=True, max_iter=64, riemann_tol=0.0,
                        stream=None, fp64_accumulate=False, entropy=False, mach_thresh=1.1, alpha_s=0.01,
                        regularize=False, eta=0.25, chi=1.0):
    o = amm_options()
    lib().amm_default_options(ctypes.byref(o))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.mesh_motion = MOTIONS[mesh_motion] if isinstance(mesh_motion, str) else int(mesh_motion)
    o.limiter = int(bool(limiter))
    o.max_iter = int(max_iter)
    o.riemann_tol = float(riemann_tol)
    o.stream = stream
    o.fp64_accumulate = int(bool(fp64_accumulate))
    o.entropy = int(bool(entropy))
    o.mach_thresh = float(mach_thresh)
    o.alpha_s = float(alpha_s)
    o.regularize = int(bool(regularize))
    o.eta = float(eta)
    o.chi = float(chi)
    return o


def amm_create(dim, generators, face_cells, face_shift, face_area, face_centroid, box, cell_Q, gamma, opt=None,
               box_cells=None, box_faces=None):
    """Creates a context; `box` is [dim] or [n_boxes, dim]; with several boxes
    pass the cell and face offsets ([n_boxes+1] each)."""
    gen = _arr(generators, np.float64)
    cells = _arr(face_cells, np.int32)
    shift = _arr(face_shift, np.int8)
    area = _arr(face_area, np.float64)
    cen = _arr(face_centroid, np.float64)
    boxa = _arr(box, np.float64).reshape(-1, dim)
    Q = _arr(cell_Q, np.float64)
    n, nf = gen.shape[0], area.shape[0]
    if opt is None:
        opt = amm_default_options()
    keep = []
    if boxa.shape[0] > 1:
        bc = _arr(box_cells, np.int64)
        bf = _arr(box_faces, np.int64)
        keep += [bc, bf]
        opt.n_boxes = boxa.shape[0]
        opt.box_cells = bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        opt.box_faces = bf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    else:
        opt.n_boxes = 1
    h = ctypes.c_void_p()
    rc = lib().amm_create(ctypes.byref(h), dim, n, gen.ctypes.data, nf, cells.ctypes.data, shift.ctypes.data,
                          area.ctypes.data, cen.ctypes.data, boxa.ctypes.data, Q.ctypes.data, float(gamma),
                          ctypes.byref(opt))
    if rc != AMM_OK:
        raise AmmError(rc, "amm_create failed (details on stderr)")
    return Context(h, dim, n, nf, boxa.shape[0])


def amm_create_device(dim, n, nf, gen_ptr, cells_ptr, shift_ptr, area_ptr, cen_ptr, box, Q_ptr, gamma, opt=None):
    """amm_create from device arrays (pointers); `box` is a host array
    ([dim] or [n_boxes, dim]; several boxes need the options' offsets)."""
    boxa = _arr(box, np.float64).reshape(-1, dim)
    if opt is None:
        opt = amm_default_options()
    if boxa.shape[0] == 1:
        opt.n_boxes = 1
    h = ctypes.c_void_p()
    rc = lib().amm_create_device(ctypes.byref(h), dim, int(n), _ptr(gen_ptr), int(nf), _ptr(cells_ptr), _ptr(shift_ptr),
                                 _ptr(area_ptr), _ptr(cen_ptr), boxa.ctypes.data, _ptr(Q_ptr), float(gamma),
                                 ctypes.byref(opt))
    if rc != AMM_OK:
        raise AmmError(rc, "amm_create_device failed (details on stderr)")
    return Context(h, dim, int(n), int(nf), boxa.shape[0])


def amm_destroy(ctx):
    if ctx.handle:
        lib().amm_destroy(ctx.handle)
        ctx.handle = None


def amm_set_state(ctx, Q):
    Q = _arr(Q, np.float64)
    assert Q.shape == (ctx.n, ctx.dim + 2)
    _check(ctx, lib().amm_set_state(ctx.handle, Q.ctypes.data))


def amm_set_state_device(ctx, q_ptr):
    _check(ctx, lib().amm_set_state_device(ctx.handle, ctypes.c_void_p(int(q_ptr))))


def amm_set_mesh_velocity(ctx, w):
    w = _arr(w, np.float64)
    assert w.shape == (ctx.n, ctx.dim)
    _check(ctx, lib().amm_set_mesh_velocity(ctx.handle, w.ctypes.data))


def amm_gradients(ctx):
    _check(ctx, lib().amm_gradients(ctx.handle))


def amm_timestep(ctx, cfl):
    out = np.empty(ctx.nboxes)
    _check(ctx, lib().amm_timestep(ctx.handle, float(cfl), out.ctypes.data))
    return out


def amm_step(ctx, dt):
    _check(ctx, lib().amm_step(ctx.handle, float(dt)))


def amm_step_boxes(ctx, dt):
    dt = _arr(dt, np.float64)
    assert dt.shape == (ctx.nboxes,)
    _check(ctx, lib().amm_step_boxes(ctx.handle, dt.ctypes.data))


def amm_advance(ctx, cfl, nsteps=1, use_graph=True):
    _check(ctx, lib().amm_advance(ctx.handle, float(cfl), int(nsteps), int(bool(use_graph))))


class Tess:
    """A GPU tessellation (amm_tess*): device face and cell arrays owned by
    the library, freed with the object."""

    def __init__(self, handle, dim, n):
        self.handle, self.dim, self.n = handle, dim, n

    def __del__(self):
        try:
            if self.handle:
                lib().amm_tess_destroy(self.handle)
                self.handle = None
        except Exception:
            pass

    @property
    def n_faces(self):
        return int(lib().amm_tess_num_faces(self.handle))

    def device_faces(self):
        """Device pointers (cells, shift, area, centroid)."""
        p = [_P() for _ in range(4)]
        rc = lib().amm_tess_faces(self.handle, *[ctypes.byref(x) for x in p])
        if rc != 0:
            raise AmmError(rc, "amm_tess_faces")
        return tuple(x.value for x in p)

    def device_cells(self):
        """Device pointers (volume, centre of mass, half-faces per cell)."""
        p = [_P() for _ in range(3)]
        rc = lib().amm_tess_cells(self.handle, *[ctypes.byref(x) for x in p])
        if rc != 0:
            raise AmmError(rc, "amm_tess_cells")
        return tuple(x.value for x in p)

    def to_host(self):
        """Copies of the face and cell arrays (numpy): cells [F, 2], shift
        [F, dim], area [F], centroid [F, dim], volume [n], com [n, dim]."""
        import torch
        F, d, n = self.n_faces, self.dim, self.n
        c, s, a, cen = self.device_faces()
        v, m, _ = self.device_cells()

        def host(ptr, shape, typestr):
            class _View:
                __cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (int(ptr), False),
                                            "version": 2}
            return torch.as_tensor(_View(), device="cuda").cpu().numpy().copy()

        return (host(c, (F, 2), "<i4"), host(s, (F, d), "|i1"), host(a, (F,), "<f8"), host(cen, (F, d), "<f8"),
                host(v, (n,), "<f8"), host(m, (n, d), "<f8"))

    def check(self):
        a = ctypes.c_int64(0)
        r = ctypes.c_double(0.0)
        lib().amm_tess_check(self.handle, ctypes.byref(a), ctypes.byref(r))
        return a.value, r.value


def amm_tess_build(dim, n, gen_ptr, box, stream=None):
    """Voronoi tessellation of device generators gen_ptr [n][dim] in the
    periodic box (host sequence of dim lengths)."""
    h = _P()
    b = _arr(box, np.float64)
    rc = lib().amm_tess_build(ctypes.byref(h), int(dim), int(n), ctypes.c_void_p(int(gen_ptr)), b.ctypes.data,
                              stream)
    if rc != 0:
        raise AmmError(rc, "amm_tess_build: " + lib().amm_tess_last_error().decode())
    return Tess(h.value, dim, n)


def amm_retessellate(ctx):
    """A new GPU tessellation of the context's current generators; cells keep
    their conserved quantities."""
    _check(ctx, lib().amm_retessellate(ctx.handle))
    ctx.nf = int(lib().amm_get_num_faces(ctx.handle))


def amm_get_faces(ctx):
    """(cells [F, 2], area [F]) of the current mesh, caller numbering."""
    F = int(lib().amm_get_num_faces(ctx.handle))
    cells = np.empty((F, 2), np.int32)
    area = np.empty(F)
    _check(ctx, lib().amm_get_faces(ctx.handle, cells.ctypes.data, area.ctypes.data))
    return cells, area


def amm_advance_individual(ctx, cfl, dt_max, max_depth=30, signal_speed=True):
    """One cycle of individual time steps (Sec. 7.2); returns the cycle's
    counters as a dict."""
    st = amm_cycle_stats()
    _check(ctx, lib().amm_advance_individual(ctx.handle, float(cfl), float(dt_max), int(max_depth),
                                             int(bool(signal_speed)), ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in st._fields_ if f != "reserved"}


def amm_individual_host_loop(ctx, enable=True):
    _check(ctx, lib().amm_individual_host_loop(ctx.handle, int(bool(enable))))


def amm_get_bins(ctx):
    b = np.empty(ctx.n, np.int32)
    _check(ctx, lib().amm_get_bins(ctx.handle, b.ctypes.data))
    return b


def amm_drift(ctx, dt):
    _check(ctx, lib().amm_drift(ctx.handle, float(dt)))


def amm_sync(ctx):
    _check(ctx, lib().amm_sync(ctx.handle))


def amm_get_state(ctx, out=None):
    Q = np.empty((ctx.n, ctx.dim + 2)) if out is None else out
    _check(ctx, lib().amm_get_state(ctx.handle, Q.ctypes.data))
    return Q


def amm_get_state_device(ctx, q_ptr):
    _check(ctx, lib().amm_get_state_device(ctx.handle, ctypes.c_void_p(int(q_ptr))))


def amm_get_primitives(ctx):
    W = np.empty((ctx.n, ctx.dim + 2))
    _check(ctx, lib().amm_get_primitives(ctx.handle, W.ctypes.data))
    return W


def amm_get_gradients(ctx):
    g = np.empty((ctx.n, ctx.dim + 2, ctx.dim))
    _check(ctx, lib().amm_get_gradients(ctx.handle, g.ctypes.data))
    return g


def amm_get_face_flux(ctx):
    F = np.empty((ctx.nf, ctx.dim + 2))
    _check(ctx, lib().amm_get_face_flux(ctx.handle, F.ctypes.data))
    return F


def amm_get_geometry(ctx):
    V = np.empty(ctx.n)
    s = np.empty((ctx.n, ctx.dim))
    _check(ctx, lib().amm_get_geometry(ctx.handle, V.ctypes.data, s.ctypes.data))
    return V, s


def amm_get_totals(ctx):
    t = np.empty((ctx.nboxes, ctx.dim + 2))
    _check(ctx, lib().amm_get_totals(ctx.handle, t.ctypes.data))
    return t


def amm_get_dt(ctx):
    d = np.empty(ctx.nboxes)
    _check(ctx, lib().amm_get_dt(ctx.handle, d.ctypes.data))
    return d


def amm_get_generators(ctx):
    g = np.empty((ctx.n, ctx.dim))
    _check(ctx, lib().amm_get_generators(ctx.handle, g.ctypes.data))
    return g


def amm_get_stats(ctx):
    s = amm_stats()
    _check(ctx, lib().amm_get_stats(ctx.handle, ctypes.byref(s)))
    d = {f: getattr(s, f) for f, _ in amm_stats._fields_ if f != "newton_hist"}
    d["newton_hist"] = list(s.newton_hist)
    return d


def amm_get_entropy(ctx):
    """(S [n], kept [n] 0/1) of a context with the entropy switch."""
    S = np.empty(ctx.n)
    kept = np.empty(ctx.n, np.uint8)
    _check(ctx, lib().amm_get_entropy(ctx.handle, S.ctypes.data, kept.ctypes.data))
    return S, kept


def amm_set_entropy(ctx, S):
    S = _arr(S, np.float64)
    _check(ctx, lib().amm_set_entropy(ctx.handle, S.ctypes.data))


def amm_get_box_status(ctx):
    s = np.empty(ctx.nboxes, np.uint32)
    _check(ctx, lib().amm_get_box_status(ctx.handle, s.ctypes.data))
    return s


def amm_reset_stats(ctx):
    _check(ctx, lib().amm_reset_stats(ctx.handle))


def amm_profile(ctx, enable=True):
    _check(ctx, lib().amm_profile(ctx.handle, int(bool(enable))))


KERNEL_GROUPS = ("gradients", "flux", "update", "finish")


def amm_get_kernel_times(ctx):
    ms = (ctypes.c_float * 4)()
    _check(ctx, lib().amm_get_kernel_times(ctx.handle, ms))
    return dict(zip(KERNEL_GROUPS, list(ms)))


class amm_tuning(ctypes.Structure):
    _fields_ = [("grad_lanes", ctypes.c_int), ("update_lanes", ctypes.c_int), ("flux_block", ctypes.c_int),
                ("persistent", ctypes.c_int), ("step_ms", ctypes.c_float)]


def _tuning_dict(t):
    return {f: getattr(t, f) for f, _ in amm_tuning._fields_}


def amm_set_tuning(ctx, grad_lanes=4, update_lanes=4, flux_block=256, persistent=0):
    t = amm_tuning(int(grad_lanes), int(update_lanes), int(flux_block), int(persistent), 0.0)
    _check(ctx, lib().amm_set_tuning(ctx.handle, ctypes.byref(t)))


def amm_get_tuning(ctx):
    t = amm_tuning()
    _check(ctx, lib().amm_get_tuning(ctx.handle, ctypes.byref(t)))
    return _tuning_dict(t)


def amm_autotune(ctx, cfl=0.3, reps=5):
    t = amm_tuning()
    _check(ctx, lib().amm_autotune(ctx.handle, float(cfl), int(reps), ctypes.byref(t)))
    return _tuning_dict(t)


def amm_timestep_noalloc(dim, n_cells, W_ptr, V_ptr, wmesh_ptr, gamma, cfl, dt_ptr, stream=None):
    """Allocation-free Courant step on caller-owned device buffers (integer
    device addresses); asynchronous on `stream`.  Raises AmmError on failure."""
    rc = lib().amm_timestep_noalloc(int(dim), int(n_cells), ctypes.c_void_p(int(W_ptr)), ctypes.c_void_p(int(V_ptr)),
                                    ctypes.c_void_p(int(wmesh_ptr)) if wmesh_ptr else None, float(gamma), float(cfl),
                                    ctypes.c_void_p(int(dt_ptr)), ctypes.c_void_p(int(stream)) if stream else None)
    if rc != AMM_OK:
        raise AmmError(rc, "amm_timestep_noalloc failed")


def amm_alu_peak(fp64, iters, stream=None):
    """FMA-chain throughput probe of the current device: returns (FLOPs, ms)."""
    flop = _D(0.0)
    ms = ctypes.c_float(0.0)
    rc = lib().amm_alu_peak(int(bool(fp64)), int(iters), ctypes.byref(flop), ctypes.byref(ms),
                            ctypes.c_void_p(int(stream)) if stream else None)
    if rc != AMM_OK:
        raise AmmError(rc, "amm_alu_peak failed")
    return flop.value, ms.value


class Mlp:
    """Owns an amm_mlp* (the learned p* proposal network)."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        try:
            if self.handle:
                lib().amm_mlp_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def _mcheck(net, rc):
    if rc != AMM_OK:
        raise AmmError(rc, lib().amm_mlp_last_error(net.handle).decode())


def _ptr(p):
    return ctypes.c_void_p(int(p)) if p else None


def amm_mlp_create(gamma, stream=None):
    h = ctypes.c_void_p()
    rc = lib().amm_mlp_create(ctypes.byref(h), float(gamma), _ptr(stream))
    if rc != AMM_OK:
        raise AmmError(rc, "amm_mlp_create failed")
    return Mlp(h)


def amm_mlp_num_params():
    return int(lib().amm_mlp_num_params())


def amm_mlp_set_params(net, params):
    p = _arr(params, np.float32)
    assert p.shape == (amm_mlp_num_params(),)
    _mcheck(net, lib().amm_mlp_set_params(net.handle, p.ctypes.data))


def amm_mlp_get_params(net):
    p = np.empty(amm_mlp_num_params(), np.float32)
    _mcheck(net, lib().amm_mlp_get_params(net.handle, p.ctypes.data))
    return p


def amm_mlp_forward(net, x_ptr, n, y_ptr):
    _mcheck(net, lib().amm_mlp_forward(net.handle, _ptr(x_ptr), int(n), _ptr(y_ptr)))


def amm_mlp_grads(net, x_ptr, t_ptr, idx_ptr, n):
    g = np.empty(amm_mlp_num_params(), np.float32)
    loss = ctypes.c_float(0.0)
    _mcheck(net, lib().amm_mlp_grads(net.handle, _ptr(x_ptr), _ptr(t_ptr), _ptr(idx_ptr), int(n), g.ctypes.data,
                                     ctypes.byref(loss)))
    return g, float(loss.value)


def amm_mlp_train_step(net, x_ptr, t_ptr, idx_ptr, n, lr, loss_ptr=0):
    _mcheck(net, lib().amm_mlp_train_step(net.handle, _ptr(x_ptr), _ptr(t_ptr), _ptr(idx_ptr), int(n), float(lr),
                                          _ptr(loss_ptr)))


def amm_mlp_sync(net):
    _mcheck(net, lib().amm_mlp_sync(net.handle))


def amm_mlp_attach(ctx, net):
    _check(ctx, lib().amm_mlp_attach(ctx.handle, net.handle))


def amm_harvest(ctx, cfl, states_ptr):
    _check(ctx, lib().amm_harvest(ctx.handle, float(cfl), _ptr(states_ptr)))


def amm_mlp_features(gamma, n, states_ptr, x_ptr, pbar_ptr=0, pts_ptr=0, ratio_ptr=0, stream=None):
    rc = lib().amm_mlp_features(float(gamma), int(n), _ptr(states_ptr), _ptr(x_ptr), _ptr(pbar_ptr), _ptr(pts_ptr),
                                _ptr(ratio_ptr), _ptr(stream))
    if rc != AMM_OK:
        raise AmmError(rc, "amm_mlp_features failed")


def amm_riemann_pstar(gamma, n, states_ptr, tol, pstar_ptr, stream=None):
    rc = lib().amm_riemann_pstar(float(gamma), int(n), _ptr(states_ptr), float(tol), _ptr(pstar_ptr), _ptr(stream))
    if rc != AMM_OK:
        raise AmmError(rc, "amm_riemann_pstar failed")


def amm_mlp_targets(gamma, n, states_ptr, tol, target_ptr, stream=None):
    rc = lib().amm_mlp_targets(float(gamma), int(n), _ptr(states_ptr), float(tol), _ptr(target_ptr), _ptr(stream))
    if rc != AMM_OK:
        raise AmmError(rc, "amm_mlp_targets failed")


def pack_params(p):
    """oracle-style dict (W1,b1,W2,b2,W3,b3) -> flat parameter vector"""
    return np.concatenate([np.asarray(p[k], np.float64).reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def unpack_params(v):
    v = np.asarray(v, np.float64)
    out, o = {}, 0
    for k, shp in (("W1", (64, 6)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (1, 64)), ("b3", (1,))):
        size = int(np.prod(shp))
        out[k] = v[o:o + size].reshape(shp)
        o += size
    return out


def create_from_mesh(mesh, Q, gamma, precision="fp64", mesh_motion="lagrangian", **kw):
    """Convenience: a context from any object with dim, points, cells, shift,
    area, centroid and box attributes (e.g. a host tessellation)."""
    opt = amm_default_options(precision, mesh_motion, **kw)
    return amm_create(mesh.dim, mesh.points, mesh.cells, mesh.shift, mesh.area, mesh.centroid, mesh.box, Q, gamma,
                      opt)
