"""Pins of the oracle's entropy switch (Sec. 3.5): the total entropy S = M A,
A = P / rho^gamma, advected with the face fluxes rho_F u_F A_upwind, kept
where the surrounding Riemann problems hold no shock above a threshold Mach
number (or, optionally, where the flow is cold), re-initialised from the
energy elsewhere."""
import json
import os

import numpy as np

from harness import ics
from harness.ics import Problem, lattice_nodes
from harness.tess import tessellate
from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _prims(P):
    M = O.Mesh(P.tess)
    geom = O.geometry(M)
    Q = P.conserved()
    return M, geom, Q


def test_never_keeping_reduces_to_the_plain_step():
    """With the switch off (threshold 0, no cold criterion) the conserved
    update is the plain one, bit for bit, and S is the re-initialised
    M P / rho^gamma of the new state."""
    P = ics.turbulent_3d(10, seed=2)
    M, geom, Q = _prims(P)
    S = O.entropy_init(M, Q, geom[0], P.gamma)
    ref, dt, cnt, rc = O.step(M, Q, P.gamma, "lagrangian", cfl=0.3, geom=geom)
    Qn, Sn, kept, dte, cnte, rce = O.step_entropy(M, Q, S, P.gamma, "lagrangian", cfl=0.3, mach_thresh=0.0,
                                                  geom=geom)
    assert rc == 0 and rce == 0 and dte == dt
    assert np.array_equal(Qn, ref)
    assert kept.sum() == 0 and cnte[4] == 0
    Wn = O.primitives(M, Qn, geom[0], P.gamma)
    np.testing.assert_allclose(Sn, Qn[:, 0] * Wn[:, 4] / Wn[:, 0] ** P.gamma, rtol=1e-13)


def test_isentropic_field_stays_isentropic():
    """P = K rho^gamma everywhere (log-normal density, turbulent velocities):
    with every cell keeping its advected entropy, the entropy flux is K times
    the mass flux, so A = S/M stays K to roundoff in every cell, and the total
    entropy changes only by roundoff."""
    P = ics.lognormal_3d(10, seed=5, sigma=0.8, mach=1.0)
    K = 1.7
    P.pres = K * P.rho ** P.gamma
    M, geom, Q = _prims(P)
    S = O.entropy_init(M, Q, geom[0], P.gamma)
    np.testing.assert_allclose(S / Q[:, 0], K, rtol=1e-14)
    Qn, Sn, kept, dt, cnt, rc = O.step_entropy(M, Q, S, P.gamma, "lagrangian", cfl=0.3, mach_thresh=np.inf,
                                               geom=geom)
    assert rc == 0 and kept.all()
    np.testing.assert_allclose(Sn / Qn[:, 0], K, rtol=1e-12)
    assert abs(Sn.sum() - S.sum()) < 1e-13 * np.abs(S).sum()
    # the kept thermal energy is the isentropic one: P_new = K rho_new^gamma
    Wn = O.primitives(M, Qn, geom[0], P.gamma)
    np.testing.assert_allclose(Wn[:, 4], K * Wn[:, 0] ** P.gamma, rtol=1e-11)


def _entropic(M, W, geom, gamma, dim):
    """A = P / rho^gamma per cell and its limited gradient (the limiter acts
    per variable, so A may take the pressure's slot)."""
    A = W[:, dim + 1] / W[:, 0] ** gamma
    WA = W.copy()
    WA[:, dim + 1] = A
    gA = O.gradients(M, WA, geom[0], geom[1])[:, dim + 1, :]
    return A, gA


def _shock_tube(nx, ny, left, right, gamma):
    """Exact 2D lattice on [0,2]x[0,1]: `left` (rho, u, p) for 0.5<x<1.5, `right` elsewhere."""
    box = np.array([2.0, 1.0])
    pts, _ = lattice_nodes((nx, ny), box)
    T = tessellate(pts, box, 0)
    inside = (pts[:, 0] > 0.5) & (pts[:, 0] < 1.5)
    rho = np.where(inside, left[0], right[0])
    pres = np.where(inside, left[2], right[2])
    vel = np.zeros((len(pts), 2))
    return Problem("tube", 2, gamma, T, rho, vel, pres, {})


def test_face_shock_mach_is_the_papers():
    """Sec. 8.2's shock tube (Mach 1.48 printed): on a stationary lattice the
    limiter flattens both cells at the jump, so the faces there solve the
    printed Riemann problem and report its shock Mach number; faces in
    uniform gas report 1 (no shock)."""
    g = json.load(open(os.path.join(GOLD, "sod_paper_variant.json")))
    P = _shock_tube(16, 4, g["left"], g["right"], g["gamma"])
    M, geom, Q = _prims(P)
    W = O.primitives(M, Q, geom[0], P.gamma)
    grad = O.gradients(M, W, geom[0], geom[1])
    A, gA = _entropic(M, W, geom, P.gamma, 2)
    F, FS, MF, cnt, rc = O.fluxes_entropy(M, W, grad, geom[1], None, P.gamma, 1e-3, A, gA)
    assert rc == 0
    xL = P.tess.points[P.tess.cells[:, 0], 0]
    xR = P.tess.points[P.tess.cells[:, 1], 0]
    jump = ((xL < 0.5) != (xR < 0.5)) | ((xL < 1.5) != (xR < 1.5))
    jump &= np.abs(xL - xR) < 0.5          # not the periodic wrap at x = 0
    assert jump.sum() == 2 * 4
    assert np.all(np.round(MF[jump], g["shock_mach_digits"]) == g["shock_mach"])
    far = (np.minimum(np.abs(xL - 0.5), np.abs(xL - 1.5)) > 0.3) & (np.minimum(np.abs(xR - 0.5), np.abs(xR - 1.5)) > 0.3)
    assert far.any() and np.all(MF[far] == 1.0) and np.all(FS[far] == 0.0)


def test_entropy_flux_is_upwind():
    """A contact (density jump, uniform P and v) advected to +x on a stationary
    lattice: the Riemann solution is the contact itself, so every face's
    entropy flux is its mass flux times A of the upwind (left, -x) state."""
    box = np.array([2.0, 1.0])
    pts, _ = lattice_nodes((16, 4), box)
    T = tessellate(pts, box, 0)
    gam = 5.0 / 3.0
    x = pts[:, 0]
    rho = np.where((x > 0.5) & (x < 1.5), 2.0, 1.0)
    vel = np.zeros((len(pts), 2))
    vel[:, 0] = 0.7
    pres = np.full(len(pts), 0.6)
    P = Problem("contact", 2, gam, T, rho, vel, pres, {})
    M, geom, Q = _prims(P)
    W = O.primitives(M, Q, geom[0], gam)
    grad = O.gradients(M, W, geom[0], geom[1])
    A, gA = _entropic(M, W, geom, gam, 2)
    F, FS, MF, cnt, rc = O.fluxes_entropy(M, W, grad, geom[1], None, gam, 1e-3, A, gA)
    # faces normal to x (the flow direction); the left cell of each is upwind
    # when the face normal points to +x
    nx = (T.points[T.cells[:, 1], 0] + T.shift[:, 0] * box[0]) - T.points[T.cells[:, 0], 0]
    along = np.abs(nx) > 1e-9
    up = np.where(nx[along] > 0, T.cells[along, 0], T.cells[along, 1])
    Aup = pres[up] / rho[up] ** gam
    np.testing.assert_allclose(FS[along], F[along, 0] * Aup, rtol=1e-13)
    assert np.all(MF <= 1.0 + 1e-12)


def test_cold_flow_switch_keeps_an_underresolved_box_positive():
    """An under-resolved Mach-1.8 turbulent box (17^3, stationary mesh): the
    plain energy update reaches a non-positive pressure within 50 steps;
    with the shock switch (Mach 1.1) and the cold-flow criterion
    (alpha_S = 0.01) every pressure stays positive and the total entropy of
    the kept cells never decreases below its advected value."""
    P = ics.turbulent_3d(17, seed=1311, mach=1.8)
    M, geom, Q0 = _prims(P)
    Q, failed_at = Q0.copy(), None
    for k in range(50):
        Q, dt, cnt, rc = O.step(M, Q, P.gamma, "eulerian", cfl=0.3, geom=geom)
        W = O.primitives(M, Q, geom[0], P.gamma)
        if (W[:, 4] <= 0).any():
            failed_at = k
            break
    assert failed_at is not None
    Q = Q0.copy()
    S = O.entropy_init(M, Q, geom[0], P.gamma)
    for k in range(50):
        Q, S, kept, dt, cnt, rc = O.step_entropy(M, Q, S, P.gamma, "eulerian", cfl=0.3, mach_thresh=1.1,
                                                 alpha_s=0.01, geom=geom)
        W = O.primitives(M, Q, geom[0], P.gamma)
        assert rc == 0 and (W[:, 4] > 0).all() and (S > 0).all(), k
