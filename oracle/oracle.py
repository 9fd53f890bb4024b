"""numpy-facing binding of the FP64 oracle (oracle/amm_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, the smoke check and bench.py's CPU-baseline
leg use it; the CUDA path never does.

Layouts: Q and W are [n, dim+2] (m, p, E) and (rho, v, P); gradients are
[n, dim+2, dim]; fluxes are [F, dim+2] per unit face area.
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None
_P = ctypes.c_void_p
_L = ctypes.c_long
_D = ctypes.c_double
_I = ctypes.c_int


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build())
        L.ora_geometry.restype = _I
        L.ora_geometry.argtypes = [_I, _L, _P, _L, _P, _P, _P, _P, _P, _P, _P]
        L.ora_primitives.restype = None
        L.ora_primitives.argtypes = [_I, _L, _P, _P, _D, _P]
        L.ora_gradients.restype = None
        L.ora_gradients.argtypes = [_I, _L, _P, _P, _P, _P, _L, _P, _P, _P, _P, _P, _I, _P]
        L.ora_timestep.restype = _D
        L.ora_timestep.argtypes = [_I, _L, _P, _P, _P, _D, _D, _P]
        L.ora_riemann_batch.restype = _L
        L.ora_riemann_batch.argtypes = [_D, _L, _P, _P, _D, _I, _P, _P]
        L.ora_face_velocities.restype = None
        L.ora_face_velocities.argtypes = [_I, _L, _P, _P, _P, _P, _P, _P, _P]
        L.ora_fluxes.restype = _I
        L.ora_fluxes.argtypes = [_I, _L, _P, _P, _P, _P, _P, _L, _P, _P, _P, _P, _P, _D, _D, _D, _I, _P, _P]
        L.ora_update.restype = None
        L.ora_update.argtypes = [_I, _L, _P, _L, _P, _P, _P, _D, _P]
        L.ora_totals.restype = None
        L.ora_totals.argtypes = [_I, _L, _P, _P]
        L.ora_drift.restype = None
        L.ora_drift.argtypes = [_I, _L, _P, _P, _P, _D]
        L.ora_step.restype = _I
        L.ora_step.argtypes = [_I, _L, _P, _L, _P, _P, _P, _P, _P, _P, _P, _P, _D, _I, _P, _D, _D, _I, _D, _I,
                               _P, _P, _P]
        L.ora_fluxes_entropy.restype = _I
        L.ora_fluxes_entropy.argtypes = [_I, _L, _P, _P, _P, _P, _P, _L, _P, _P, _P, _P, _P, _D, _D, _D, _I, _P,
                                         _P, _P, _P, _P, _P]
        L.ora_entropy_init.restype = None
        L.ora_entropy_init.argtypes = [_I, _L, _P, _P, _D, _P]
        L.ora_step_entropy.restype = _I
        L.ora_step_entropy.argtypes = [_I, _L, _P, _L, _P, _P, _P, _P, _P, _P, _P, _P, _P, _D, _I, _P, _D, _D,
                                       _I, _D, _I, _D, _D, _P, _P, _P, _P, _P]
        L.ora_shape_correction.restype = None
        L.ora_shape_correction.argtypes = [_I, _L, _P, _P, _P, _P, _P, _D, _D, _D, _P]
        L.ora_signal_timestep.restype = None
        L.ora_signal_timestep.argtypes = [_I, _L, _P, _P, _P, _P, _D, _D, _I, _P]
        L.ora_advance_individual.restype = _I
        L.ora_advance_individual.argtypes = [_I, _L, _P, _L, _P, _P, _P, _P, _P, _P, _P, _P, _D, _D, _D, _I, _I,
                                             _I, _D, _I, _P, _P, _P]
        L.ora_set_threads.restype = None
        L.ora_set_threads.argtypes = [_I]
        L.ora_get_threads.restype = _I
        L.ora_get_threads.argtypes = []
        _lib = L
    return _lib


def set_threads(t):
    """Host threads for the per-cell and per-face loops (default 1); the
    results do not depend on it."""
    lib().ora_set_threads(int(t))


def get_threads():
    return lib().ora_get_threads()


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Mesh:
    """Face list + generators in the dtypes the oracle expects."""

    def __init__(self, tess):
        self.dim = int(tess.dim)
        self.n = int(tess.n_cells)
        self.nf = int(tess.n_faces)
        self.gen = _c(tess.points, np.float64)
        self.cells = _c(tess.cells, np.int32)
        self.shift = _c(tess.shift, np.int8)
        self.area = _c(tess.area, np.float64)
        self.cen = _c(tess.centroid, np.float64)
        self.box = _c(tess.box, np.float64)

    def args(self):
        return (self.cells.ctypes.data, self.shift.ctypes.data, self.area.ctypes.data, self.cen.ctypes.data,
                self.box.ctypes.data)


MODES = {"eulerian": 0, "lagrangian": 1, "explicit": 2}


def geometry(mesh):
    """A0: volumes and centres of mass from the pyramid sums."""
    V = np.empty(mesh.n)
    s = np.empty((mesh.n, mesh.dim))
    rc = lib().ora_geometry(mesh.dim, mesh.n, mesh.gen.ctypes.data, mesh.nf, *mesh.args(), V.ctypes.data,
                            s.ctypes.data)
    if rc != 0:
        raise ValueError("non-positive cell volume")
    return V, s


def primitives(mesh, Q, V, gamma):
    Q = _c(Q, np.float64)
    W = np.empty_like(Q)
    lib().ora_primitives(mesh.dim, mesh.n, Q.ctypes.data, _c(V, np.float64).ctypes.data, gamma, W.ctypes.data)
    return W


def gradients(mesh, W, V, s, limit=True):
    W = _c(W, np.float64)
    V = _c(V, np.float64)
    s = _c(s, np.float64)
    g = np.empty((mesh.n, mesh.dim + 2, mesh.dim))
    lib().ora_gradients(mesh.dim, mesh.n, W.ctypes.data, mesh.gen.ctypes.data, V.ctypes.data, s.ctypes.data,
                        mesh.nf, *mesh.args(), int(bool(limit)), g.ctypes.data)
    return g


def timestep(mesh, W, V, wmesh, gamma, cfl):
    W = _c(W, np.float64)
    V = _c(V, np.float64)
    wm = None if wmesh is None else _c(wmesh, np.float64)
    dtc = np.empty(mesh.n)
    dt = lib().ora_timestep(mesh.dim, mesh.n, W.ctypes.data, V.ctypes.data, None if wm is None else wm.ctypes.data,
                            gamma, cfl, dtc.ctypes.data)
    return dt, dtc


def riemann(gamma, WL, WR, tol=1e-12, maxit=64):
    """Batch exact Riemann problems: WL, WR [m,3] (rho,u,p) -> out [m,6]
    (rho,u,p sampled at x/t=0, p*, u*, side) and Newton iterations [m]."""
    WL = _c(np.atleast_2d(WL), np.float64)
    WR = _c(np.atleast_2d(WR), np.float64)
    m = WL.shape[0]
    out = np.empty((m, 6))
    it = np.empty(m, np.int32)
    bad = lib().ora_riemann_batch(gamma, m, WL.ctypes.data, WR.ctypes.data, tol, maxit, out.ctypes.data,
                                  it.ctypes.data)
    return out, it, int(bad)


def face_velocities(mesh, wmesh):
    wm = _c(wmesh, np.float64)
    wf = np.empty((mesh.nf, mesh.dim))
    lib().ora_face_velocities(mesh.dim, mesh.nf, mesh.cells.ctypes.data, mesh.shift.ctypes.data,
                              mesh.gen.ctypes.data, mesh.cen.ctypes.data, mesh.box.ctypes.data, wm.ctypes.data,
                              wf.ctypes.data)
    return wf


def fluxes(mesh, W, grad, s, wmesh, gamma, dt, tol=1e-12, maxit=64):
    W = _c(W, np.float64)
    grad = _c(grad, np.float64)
    s = _c(s, np.float64)
    wm = None if wmesh is None else _c(wmesh, np.float64)
    F = np.empty((mesh.nf, mesh.dim + 2))
    cnt = np.zeros(4, np.int64)
    rc = lib().ora_fluxes(mesh.dim, mesh.n, W.ctypes.data, grad.ctypes.data, mesh.gen.ctypes.data, s.ctypes.data,
                          None if wm is None else wm.ctypes.data, mesh.nf, *mesh.args(), gamma, dt, tol, maxit,
                          F.ctypes.data, cnt.ctypes.data)
    return F, cnt, rc


def fluxes_entropy(mesh, W, grad, s, wmesh, gamma, dt, A, gA, tol=1e-12, maxit=64):
    """fluxes() plus, per face, the entropy flux per unit area and the largest
    shock Mach number of its Riemann problem (Sec. 3.5); A is the entropic
    function per cell and gA its limited gradient [n, dim]."""
    A = _c(A, np.float64)
    gA = _c(gA, np.float64)
    W = _c(W, np.float64)
    grad = _c(grad, np.float64)
    s = _c(s, np.float64)
    wm = None if wmesh is None else _c(wmesh, np.float64)
    F = np.empty((mesh.nf, mesh.dim + 2))
    FS = np.empty(mesh.nf)
    MF = np.empty(mesh.nf)
    cnt = np.zeros(4, np.int64)
    rc = lib().ora_fluxes_entropy(mesh.dim, mesh.n, W.ctypes.data, grad.ctypes.data, mesh.gen.ctypes.data,
                                  s.ctypes.data, None if wm is None else wm.ctypes.data, mesh.nf, *mesh.args(), gamma,
                                  dt, tol, maxit, A.ctypes.data, gA.ctypes.data, F.ctypes.data, FS.ctypes.data,
                                  MF.ctypes.data, cnt.ctypes.data)
    return F, FS, MF, cnt, rc


def update(mesh, Q, F, dt):
    Q = _c(Q, np.float64)
    F = _c(F, np.float64)
    Qn = np.empty_like(Q)
    lib().ora_update(mesh.dim, mesh.n, Q.ctypes.data, mesh.nf, mesh.cells.ctypes.data, mesh.area.ctypes.data,
                     F.ctypes.data, dt, Qn.ctypes.data)
    return Qn


def totals(mesh, Q):
    Q = _c(Q, np.float64)
    t = np.empty(mesh.dim + 2)
    lib().ora_totals(mesh.dim, mesh.n, Q.ctypes.data, t.ctypes.data)
    return t


def drift(mesh, wmesh, dt):
    gen = mesh.gen.copy()
    lib().ora_drift(mesh.dim, mesh.n, gen.ctypes.data, _c(wmesh, np.float64).ctypes.data, mesh.box.ctypes.data, dt)
    return gen


def step(mesh, Q, gamma, mode="lagrangian", wmesh=None, dt=0.0, cfl=0.3, limit=True, tol=1e-12, maxit=64,
         geom=None):
    """One whole update (Sec. 3 steps 2-7).  Returns (Qnew, dt_used, counters, rc)."""
    V, s = geometry(mesh) if geom is None else geom
    Q = _c(Q, np.float64)
    Qn = np.empty_like(Q)
    dtu = ctypes.c_double(0.0)
    cnt = np.zeros(4, np.int64)
    wm = None if wmesh is None else _c(wmesh, np.float64)
    rc = lib().ora_step(mesh.dim, mesh.n, mesh.gen.ctypes.data, mesh.nf, *mesh.args(), V.ctypes.data,
                        s.ctypes.data, Q.ctypes.data, gamma, MODES[mode], None if wm is None else wm.ctypes.data,
                        dt, cfl, int(bool(limit)), tol, maxit, Qn.ctypes.data, ctypes.byref(dtu), cnt.ctypes.data)
    return Qn, dtu.value, cnt, rc


def entropy_init(mesh, Q, V, gamma):
    """S = M P / rho^gamma per cell (Sec. 3.5)."""
    Q = _c(Q, np.float64)
    S = np.empty(mesh.n)
    lib().ora_entropy_init(mesh.dim, mesh.n, Q.ctypes.data, _c(V, np.float64).ctypes.data, gamma, S.ctypes.data)
    return S


def step_entropy(mesh, Q, S, gamma, mode="lagrangian", wmesh=None, dt=0.0, cfl=0.3, limit=True, tol=1e-12,
                 maxit=64, mach_thresh=1.1, alpha_s=0.0, geom=None):
    """One update with the entropy switch of Sec. 3.5.  Returns (Qnew, Snew,
    kept [n] 0/1, dt_used, counters[5], rc); counters[4] = cells that kept
    their advected entropy."""
    V, s = geometry(mesh) if geom is None else geom
    Q = _c(Q, np.float64)
    S = _c(S, np.float64)
    Qn = np.empty_like(Q)
    Sn = np.empty_like(S)
    kept = np.empty(mesh.n, np.int32)
    dtu = ctypes.c_double(0.0)
    cnt = np.zeros(5, np.int64)
    wm = None if wmesh is None else _c(wmesh, np.float64)
    rc = lib().ora_step_entropy(mesh.dim, mesh.n, mesh.gen.ctypes.data, mesh.nf, *mesh.args(), V.ctypes.data,
                                s.ctypes.data, Q.ctypes.data, S.ctypes.data, gamma, MODES[mode],
                                None if wm is None else wm.ctypes.data, dt, cfl, int(bool(limit)), tol, maxit,
                                mach_thresh, alpha_s, Qn.ctypes.data, Sn.ctypes.data, kept.ctypes.data, ctypes.byref(dtu),
                                cnt.ctypes.data)
    return Qn, Sn, kept, dtu.value, cnt, rc


def shape_correction(mesh, W, V, s, w, gamma, eta=0.25, chi=1.0):
    """Mesh velocity with the regularity correction of Sec. 4.1,
    eq. (EqnShapeCorrVel); w is the uncorrected mesh velocity [n, dim]."""
    W, V, s, w = (_c(a, np.float64) for a in (W, V, s, w))
    out = np.empty_like(w)
    lib().ora_shape_correction(mesh.dim, mesh.n, mesh.gen.ctypes.data, s.ctypes.data, V.ctypes.data, W.ctypes.data,
                               w.ctypes.data, gamma, eta, chi, out.ctypes.data)
    return out


def signal_timestep(mesh, W, V, gamma, cfl, signal=True):
    """Per-cell time-step criterion of eq. (EqnTiStepIndividual) on a static
    mesh (signal=False: eq. EqnTiStep alone).  [n]"""
    W = _c(W, np.float64)
    dt = np.empty(mesh.n)
    lib().ora_signal_timestep(mesh.dim, mesh.n, mesh.gen.ctypes.data, mesh.box.ctypes.data, W.ctypes.data,
                              _c(V, np.float64).ctypes.data, gamma, cfl, int(bool(signal)), dt.ctypes.data)
    return dt


def advance_individual(mesh, Q, gamma, cfl, dt_max, max_depth=30, signal=True, limit=True, tol=1e-12, maxit=64,
                       geom=None):
    """One cycle of individual power-of-two time steps of length dt_max on the
    static mesh (Sec. 7.2).  Returns (Qnew, bins, counters[7], rc); counters:
    fallback faces, vacuum faces, Newton iterations, Newton failures,
    sub-steps, face flux evaluations, cell activations."""
    V, s = geometry(mesh) if geom is None else geom
    Q = _c(Q, np.float64)
    Qn = np.empty_like(Q)
    bins = np.zeros(mesh.n, np.int32)
    cnt = np.zeros(7, np.int64)
    rc = lib().ora_advance_individual(mesh.dim, mesh.n, mesh.gen.ctypes.data, mesh.nf, *mesh.args(), V.ctypes.data,
                                      s.ctypes.data, Q.ctypes.data, gamma, cfl, dt_max, int(max_depth),
                                      int(bool(signal)), int(bool(limit)), tol, maxit, Qn.ctypes.data,
                                      bins.ctypes.data, cnt.ctypes.data)
    return Qn, bins, cnt, rc
