"""A moving-mesh run: the method's whole cycle (Sec. 3, steps 1-8) with the
tessellation rebuilt on the host every step.

Each step takes the Courant step and the mesh velocities w of the current
state, moves the generators by w dt, updates the conserved quantities on the
current tessellation (its faces move with the velocities derived from the
same w), and then tessellates the moved generators, which keep their cells'
conserved quantities.  Two backends take the same steps: the library, in any
of its forms, and the FP64 oracle (test infrastructure only); run_on_device
keeps the whole cycle on the GPU (amm_retessellate)."""
import numpy as np

from .ics import gresho_profile
from .tess import tessellate


class LibraryBackend:
    """One context per tessellation through the C ABI: amm_timestep (which
    also forms the mesh velocities), amm_drift with them, amm_step."""

    def __init__(self, amm, precision="fp64", mesh_motion="lagrangian", **options):
        self.amm = amm
        self.precision = precision
        self.mesh_motion = mesh_motion
        self.options = options

    def step(self, tess, Q, gamma, cfl, t_left):
        amm = self.amm
        ctx = amm.create_from_mesh(tess, Q, gamma, precision=self.precision, mesh_motion=self.mesh_motion,
                                   **self.options)
        try:
            dt = min(float(amm.amm_timestep(ctx, cfl)[0]), t_left)
            amm.amm_drift(ctx, dt)
            amm.amm_step(ctx, dt)
            Qn = amm.amm_get_state(ctx)
            gen = amm.amm_get_generators(ctx)
        finally:
            amm.amm_destroy(ctx)
        return Qn, gen, dt


class OracleBackend:
    """The same step from the FP64 oracle: mesh velocity zero (eulerian), the
    cell velocity (lagrangian), optionally with the regularity correction of
    Sec. 4.1."""

    def __init__(self, oracle, mesh_motion="lagrangian", regularize=False, eta=0.25, chi=1.0):
        self.O = oracle
        self.mesh_motion = mesh_motion
        self.regularize = regularize
        self.eta, self.chi = eta, chi

    def step(self, tess, Q, gamma, cfl, t_left):
        O = self.O
        M = O.Mesh(tess)
        V, s = O.geometry(M)
        W = O.primitives(M, Q, V, gamma)
        if self.mesh_motion == "eulerian":
            w = np.zeros((M.n, M.dim))
        else:
            w = W[:, 1:1 + M.dim].copy()
            if self.regularize:
                w = O.shape_correction(M, W, V, s, w, gamma, self.eta, self.chi)
        dt, _ = O.timestep(M, W, V, w, gamma, cfl)
        dt = min(dt, t_left)
        gen = O.drift(M, w, dt)
        Qn, _, _, rc = O.step(M, Q, gamma, "explicit", wmesh=w, dt=dt, geom=(V, s))
        if rc != 0:
            raise RuntimeError("oracle step failed")
        return Qn, gen, dt


def run_on_device(amm, problem, precision="fp64", mesh_motion="lagrangian", t_end=None, steps=None, cfl=0.3,
                  **options):
    """The same cycle with everything on the device: one context, whose mesh
    amm_retessellate rebuilds on the GPU after every drift.  Returns
    (generators, Q, t, steps) in the problem's cell numbering."""
    ctx = amm.create_from_mesh(problem.tess, problem.conserved(), problem.gamma, precision=precision,
                               mesh_motion=mesh_motion, **options)
    try:
        t, k = 0.0, 0
        while (steps is None or k < steps) and (t_end is None or t < t_end * (1 - 1e-14)):
            dt = float(amm.amm_timestep(ctx, cfl)[0])
            if t_end is not None:
                dt = min(dt, t_end - t)
            amm.amm_drift(ctx, dt)
            amm.amm_step(ctx, dt)
            amm.amm_retessellate(ctx)
            t += dt
            k += 1
        return amm.amm_get_generators(ctx), amm.amm_get_state(ctx), t, k
    finally:
        amm.amm_destroy(ctx)


def run(problem, backend, t_end=None, steps=None, cfl=0.3, nthreads=0, tess=None, Q=None, t0=0.0):
    """Advances `problem` (or the given tessellation and state) to t_end, or
    for `steps` steps, with a new tessellation after every step; returns
    (tessellation, Q, t, steps)."""
    tess = problem.tess if tess is None else tess
    Q = problem.conserved() if Q is None else Q
    t, k = t0, 0
    while (steps is None or k < steps) and (t_end is None or t < t_end * (1 - 1e-14)):
        t_left = np.inf if t_end is None else t_end - t
        Q, gen, dt = backend.step(tess, Q, problem.gamma, cfl, t_left)
        tess = tessellate(gen, tess.box, nthreads)
        t += dt
        k += 1
    return tess, Q, t, k


def gresho_l1(tess, Q, t, v_vortex=0.0):
    """L1 norm of the azimuthal velocity error at time t: the mean over cells
    of |v_phi - v_phi,exact| at the generators, about the vortex centre carried
    along x with v_vortex (minimum periodic image), in the vortex frame."""
    m = Q[:, 0]
    v = Q[:, 1:3] / m[:, None]
    c = np.array([np.mod(0.5 + v_vortex * t, 1.0), 0.5])
    d = tess.points - c
    d -= np.round(d / tess.box) * tess.box
    r = np.hypot(d[:, 0], d[:, 1])
    rs = np.where(r > 0, r, 1.0)
    vphi = (-(v[:, 0] - v_vortex) * d[:, 1] + v[:, 1] * d[:, 0]) / rs
    return float(np.mean(np.abs(vphi - gresho_profile(r)[0])))
