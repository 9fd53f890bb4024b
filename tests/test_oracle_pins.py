"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the property it checks and the passage it comes from.  A
plausible slip in the oracle (a dropped c_ij term, a wrong sign on the
normal, a limiter using max for min, a predictor in the wrong frame, a flux
applied with the wrong sign) fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

from harness import ics
from harness.tess import tessellate
from oracle import oracle as O

from . import _structured

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rel_err(a, b, floor):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), floor))


def q_floor(Q, dim, gamma, W=None):
    """Per-component floor of the parity norm: RMS|Q_k| for mass and energy,
    RMS(m c) for the momentum components."""
    fl = np.sqrt(np.mean(Q * Q, axis=0))
    if W is not None:
        c = np.sqrt(gamma * W[:, dim + 1] / W[:, 0])
        fl[1:1 + dim] = np.sqrt(np.mean((Q[:, 0] * c) ** 2))
    return fl


# ------------------------------------------------------------------ geometry
def test_pyramid_volumes_match_direct_integration(turb16):
    """Sec. 2.3: V_i from the pyramid sums equals the polytope volume; s_i
    from pyramid centroids equals the polytope centre of mass."""
    M = O.Mesh(turb16.tess)
    V, s = O.geometry(M)
    assert np.max(np.abs(V - turb16.tess.volume) / V) < 1e-12
    h = 1.0 / 16
    assert np.max(np.abs(s - turb16.tess.com)) < 1e-12 * h
    assert abs(V.sum() - 1.0) < 1e-13


def test_pyramid_volumes_2d(sod_small):
    M = O.Mesh(sod_small.tess)
    V, s = O.geometry(M)
    assert np.max(np.abs(V - sod_small.tess.volume) / V) < 1e-12
    assert np.max(np.abs(s - sod_small.tess.com)) < 1e-12 / 16


# ------------------------------------------------------------------ gradient
def _interior(T):
    """cells none of whose faces crosses the periodic boundary"""
    cross = np.any(T.shift != 0, axis=1)
    bad = np.zeros(T.n_cells, bool)
    bad[T.cells[cross, 0]] = True
    bad[T.cells[cross, 1]] = True
    return ~bad


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_exact_for_linear_fields(dim):
    """Eq. (eqngrad2) is exact to linear order for any Voronoi mesh."""
    rng = np.random.default_rng(21)
    box = np.ones(dim)
    dims = (12,) * dim if dim == 3 else (24, 24)
    pts = ics.jittered_lattice(dims, box, 0.3, rng)
    T = tessellate(pts, box)
    M = O.Mesh(T)
    V, s = O.geometry(M)
    B = rng.normal(size=(dim + 2, dim))
    a0 = np.array([2.0] + [0.3] * dim + [3.0])
    W = a0[None, :] + pts @ B.T
    g = O.gradients(M, W, V, s, limit=False)
    inner = _interior(T)
    assert inner.sum() > 0.3 * T.n_cells
    err = np.abs(g[inner] - B[None]) / np.abs(B).max()
    assert err.max() < 1e-11
    # without the c_ij term (the plain Green-Gauss estimate) it is not exact:
    # the pin is sensitive to that term
    gg = np.zeros_like(g)
    rL = T.points[T.cells[:, 0]]
    rR = T.points[T.cells[:, 1]] + T.shift * T.box
    nrm = (rR - rL) / np.linalg.norm(rR - rL, axis=1)[:, None]
    phiL, phiR = W[T.cells[:, 0]], W[T.cells[:, 1]]
    contrib = T.area[:, None, None] * 0.5 * (phiL + phiR)[:, :, None] * nrm[:, None, :]
    np.add.at(gg, T.cells[:, 0], contrib)
    np.add.at(gg, T.cells[:, 1], -contrib)
    gg /= V[:, None, None]
    assert np.max(np.abs(gg[inner] - B[None])) > 1e-3


def test_volume_weighted_sum_exact_for_linear_field(turb16):
    """Sec. 3.1: sum_i phi(r_i) V_i integrates a linear phi exactly; with the
    periodic box this is checked on a field linear in one direction away
    from the wrap via the identity sum_i V_i (r_i - s_i) = 0."""
    M = O.Mesh(turb16.tess)
    V, s = O.geometry(M)
    d = turb16.tess.points - s
    assert np.max(np.abs((V[:, None] * d).sum(0))) < 1e-14


def test_limiter_bounds_and_scaling(turb16):
    """Sec. 3.1: the limited reconstruction at every face centroid stays within
    [phi_min, phi_max] over the neighbours and the cell itself, and the limited
    gradient is alpha times the unlimited one with 0 <= alpha <= 1."""
    rng = np.random.default_rng(4)
    T = turb16.tess
    M = O.Mesh(T)
    V, s = O.geometry(M)
    n = T.n_cells
    W = np.column_stack([rng.uniform(0.5, 2, n), rng.normal(size=(n, 3)), rng.uniform(0.5, 2, n)])
    g0 = O.gradients(M, W, V, s, limit=False)
    g1 = O.gradients(M, W, V, s, limit=True)
    # alpha per (cell, variable)
    num = np.sum(g1 * g0, axis=2)
    den = np.sum(g0 * g0, axis=2)
    alpha = num / den
    assert alpha.min() >= -1e-14 and alpha.max() <= 1 + 1e-14
    assert np.max(np.abs(g1 - alpha[:, :, None] * g0)) < 1e-12 * np.abs(g0).max()
    assert (alpha < 0.999).mean() > 0.2          # the limiter is active on noise
    # bounds at face centroids from both sides
    L, R = T.cells[:, 0], T.cells[:, 1]
    fL = T.centroid
    fR = T.centroid - T.shift * T.box
    wmax = W.copy()
    wmin = W.copy()
    np.maximum.at(wmax, L, W[R])
    np.maximum.at(wmax, R, W[L])
    np.minimum.at(wmin, L, W[R])
    np.minimum.at(wmin, R, W[L])
    for cell, f in ((L, fL), (R, fR)):
        rec = W[cell] + np.einsum("fvd,fd->fv", g1[cell], f - s[cell])
        tol = 1e-12 * np.abs(W).max()
        assert np.all(rec <= wmax[cell] + tol)
        assert np.all(rec >= wmin[cell] - tol)


# ------------------------------------------------------------- face velocity
@pytest.mark.parametrize("dim", [2, 3])
def test_face_velocity_gives_volume_rate(dim):
    """Eq. (eqnvolchange) / Fig. FigSketchVelFace: sum over a cell's faces of
    A (w_face . n_out) is dV_i/dt, checked against a central finite
    difference of the tessellated volumes under r -> r +- eps w."""
    rng = np.random.default_rng(8)
    box = np.ones(dim)
    dims = (8,) * dim if dim == 3 else (16, 16)
    pts = ics.jittered_lattice(dims, box, 0.3, rng)
    T = tessellate(pts, box)
    M = O.Mesh(T)
    w = rng.normal(size=pts.shape)
    wf = O.face_velocities(M, w)
    rL = T.points[T.cells[:, 0]]
    rR = T.points[T.cells[:, 1]] + T.shift * T.box
    nrm = (rR - rL) / np.linalg.norm(rR - rL, axis=1)[:, None]
    flux = T.area * np.sum(wf * nrm, axis=1)
    dV = np.zeros(T.n_cells)
    np.add.at(dV, T.cells[:, 0], flux)
    np.add.at(dV, T.cells[:, 1], -flux)
    eps = 1e-6 / dims[0]
    Vp = tessellate(np.mod(pts + eps * w, box), box).volume
    Vm = tessellate(np.mod(pts - eps * w, box), box).volume
    fd = (Vp - Vm) / (2 * eps)
    scale = np.abs(fd).max()
    assert np.max(np.abs(dV - fd)) < 1e-6 * scale
    # the eq. (eqnvolchange) form written per cell agrees as well
    c = T.centroid - 0.5 * (rL + rR)
    rij = np.linalg.norm(rR - rL, axis=1)
    wl, wr = w[T.cells[:, 0]], w[T.cells[:, 1]]
    # for i = L: r_ij = rL - rR = -rij*n; for i = R: +rij*n
    tL = -T.area * (np.sum(c * (wr - wl), 1) / rij + np.sum(-nrm * (wr + wl), 1) / 2)
    tR = -T.area * (np.sum(c * (wl - wr), 1) / rij + np.sum(nrm * (wl + wr), 1) / 2)
    dV2 = np.zeros(T.n_cells)
    np.add.at(dV2, T.cells[:, 0], tL)
    np.add.at(dV2, T.cells[:, 1], tR)
    assert np.max(np.abs(dV2 - fd)) < 1e-6 * scale


# ------------------------------------------------------------------ Riemann
def test_riemann_sod_textbook():
    g = json.load(open(os.path.join(GOLD, "sod_textbook.json")))
    out, it, bad = O.riemann(g["gamma"], g["left"], g["right"])
    assert bad == 0
    assert abs(out[0, 3] - g["p_star"]) <= g["rel_tol"] * g["p_star"]
    assert abs(out[0, 4] - g["u_star"]) <= g["rel_tol"] * g["u_star"]


def test_riemann_paper_sod_shock_mach():
    """Sec. 8.2 prints shock Mach number 1.48 for its shock-tube states."""
    g = json.load(open(os.path.join(GOLD, "sod_paper_variant.json")))
    gam = g["gamma"]
    out, it, bad = O.riemann(gam, g["left"], g["right"])
    rhoR, uR, pR = g["right"]
    ps = out[0, 3]
    # Rankine-Hugoniot: post-shock density and mass flux fix the shock speed
    rs = rhoR * (ps / pR + (gam - 1) / (gam + 1)) / ((gam - 1) / (gam + 1) * ps / pR + 1)
    us = out[0, 4]
    S = (rs * us - rhoR * uR) / (rs - rhoR)
    mach = (S - uR) / np.sqrt(gam * pR / rhoR)
    assert round(mach, g["shock_mach_digits"]) == g["shock_mach"]


def _random_problems(rng, m, vacuum_free=True, gam=1.4):
    rL = np.exp(rng.uniform(-3, 3, m))
    rR = np.exp(rng.uniform(-3, 3, m))
    pL = np.exp(rng.uniform(-4, 4, m))
    pR = np.exp(rng.uniform(-4, 4, m))
    cL, cR = np.sqrt(gam * pL / rL), np.sqrt(gam * pR / rR)
    uL = rng.normal(size=m) * 2 * cL
    uR = rng.normal(size=m) * 2 * cR
    if vacuum_free:
        ok = 2 * (cL + cR) / (gam - 1) > (uR - uL) * 1.05
        rL, uL, pL, rR, uR, pR = (a[ok] for a in (rL, uL, pL, rR, uR, pR))
    return np.column_stack([rL, uL, pL]), np.column_stack([rR, uR, pR])


def test_riemann_star_satisfies_jump_conditions():
    """The star state must satisfy, across each wave, the Rankine-Hugoniot
    conditions (shock: conservation of mass, momentum and energy in the shock
    frame) or the isentropic relation and the Riemann invariant
    (rarefaction), with p and u continuous across the contact -- conservation
    laws, not the pressure function the oracle iterates on."""
    gam = 1.4
    rng = np.random.default_rng(12)
    WL, WR = _random_problems(rng, 4000, gam=gam)
    out, it, bad = O.riemann(gam, WL, WR, tol=1e-12)
    assert bad == 0
    ps, us = out[:, 3], out[:, 4]
    worst = 0.0
    for W, sgn in ((WL, -1.0), (WR, 1.0)):
        rho, u, p = W.T
        c = np.sqrt(gam * p / rho)
        shock = ps > p
        # shock branch: post-shock density from the Hugoniot, speed from mass
        # conservation, then momentum and energy conservation must hold
        g6 = (gam - 1) / (gam + 1)
        rs = rho * (ps / p + g6) / (g6 * ps / p + 1)
        S = (rs * us - rho * u) / (rs - rho)
        j = rho * (u - S)
        mom = (rho * (u - S) ** 2 + p) - (rs * (us - S) ** 2 + ps)
        e0 = p / ((gam - 1) * rho) + 0.5 * (u - S) ** 2 + p / rho
        e1 = ps / ((gam - 1) * rs) + 0.5 * (us - S) ** 2 + ps / rs
        sc = np.maximum(p, ps)
        err_s = np.maximum(np.abs(mom) / sc, np.abs(e0 - e1) * rho / sc)
        # the shock moves away from the contact on its side
        assert np.all(sgn * (S - us)[shock] > 0)
        # rarefaction branch: isentrope and Riemann invariant
        cs = c * (ps / p) ** ((gam - 1) / (2 * gam))
        err_r = np.abs((u - sgn * 2 * c / (gam - 1)) - (us - sgn * 2 * cs / (gam - 1))) / c
        err = np.where(shock, err_s, err_r)
        worst = max(worst, err.max())
        del j
    assert worst < 1e-9


def test_riemann_newton_matches_bisection():
    """p* from Newton equals the bracketed root found by bisection on the
    velocity mismatch of the two wave curves (independent of the guess)."""
    gam = 5.0 / 3.0
    rng = np.random.default_rng(13)
    WL, WR = _random_problems(rng, 2000, gam=gam)
    out, it, bad = O.riemann(gam, WL, WR, tol=1e-12)

    def u_after(W, p, sgn):
        rho, u, pk = W.T
        c = np.sqrt(gam * pk / rho)
        A = 2 / ((gam + 1) * rho)
        B = (gam - 1) / (gam + 1) * pk
        fs = (p - pk) * np.sqrt(A / (p + B))
        fr = 2 * c / (gam - 1) * ((p / pk) ** ((gam - 1) / (2 * gam)) - 1)
        return u - sgn * np.where(p > pk, fs, fr)

    lo = np.full(len(WL), 1e-300)
    hi = np.full(len(WL), 1e6)
    for _ in range(1200):
        mid = np.sqrt(lo * hi) if _ < 1000 else 0.5 * (lo + hi)
        d = u_after(WL, mid, 1) - u_after(WR, mid, -1)   # decreasing in p
        lo = np.where(d > 0, mid, lo)
        hi = np.where(d > 0, hi, mid)
    pb = 0.5 * (lo + hi)
    assert np.max(np.abs(out[:, 3] - pb) / pb) < 1e-11
    assert it.max() <= 12


def test_riemann_converges_next_to_vacuum():
    """Strong rarefactions just short of vacuum generation, with widely
    different states on the two sides: f(p) near p* is a small difference of
    large terms, so the relative change of a Newton step stays above 1e-12;
    the iteration still ends (its residual reaches rounding) and p* is the
    root found by bisection in log p, to the accuracy its conditioning
    allows."""
    gam = 5.0 / 3.0
    rng = np.random.default_rng(17)
    m = 4000
    rL, rR = np.exp(rng.uniform(-25, 5, m)), np.exp(rng.uniform(-25, 5, m))
    pL, pR = np.exp(rng.uniform(-30, 5, m)), np.exp(rng.uniform(-30, 5, m))
    cL, cR = np.sqrt(gam * pL / rL), np.sqrt(gam * pR / rR)
    du = rng.uniform(0.99, 0.99995, m) * 2 * (cL + cR) / (gam - 1)
    WL = np.stack([rL, -0.5 * du, pL], 1)
    WR = np.stack([rR, 0.5 * du, pR], 1)
    out, it, bad = O.riemann(gam, WL, WR, tol=1e-12, maxit=64)
    assert bad == 0 and np.asarray(it).max() < 64

    def mismatch(p):
        f = np.zeros(m)
        for W in (WL, WR):
            rho, u, pk = W.T
            c = np.sqrt(gam * pk / rho)
            f += np.where(p > pk, (p - pk) * np.sqrt(2 / ((gam + 1) * rho) / (p + (gam - 1) / (gam + 1) * pk)),
                          2 * c / (gam - 1) * ((p / pk) ** ((gam - 1) / (2 * gam)) - 1))
        return f + du

    lo, hi = np.full(m, 1e-300), np.full(m, 1e6)
    for _ in range(1100):
        mid = np.sqrt(lo * hi)
        neg = mismatch(mid) < 0                 # f increases with p
        lo = np.where(neg, mid, lo)
        hi = np.where(neg, hi, mid)
    pb = np.sqrt(lo * hi)
    assert np.median(np.abs(out[:, 3] / pb - 1)) < 1e-9
    assert np.max(np.abs(out[:, 3] / pb - 1)) < 1e-4


def test_riemann_vacuum_cases():
    """Vacuum: left vacuum, right vacuum, and vacuum generated between two
    rarefactions; x/t=0 in vacuum gives rho = P = 0 and zero flux."""
    gam = 1.4
    c = np.sqrt(1.4)
    # generated vacuum symmetric about x/t=0
    out, it, bad = O.riemann(gam, [1, -10 * c, 1], [1, 10 * c, 1])
    assert out[0, 0] == 0 and out[0, 2] == 0
    # right-vacuum: left state expanding into vacuum; x/t=0 inside the fan
    out, _, _ = O.riemann(gam, [1, 0, 1], [0, 0, 0])
    cf = 2 / (gam + 1) * c       # fan sound speed at x/t=0 for u_L=0
    assert abs(out[0, 1] - cf) < 1e-14 and abs(out[0, 0] - (cf / c) ** (2 / (gam - 1))) < 1e-14
    # left vacuum mirrored
    out2, _, _ = O.riemann(gam, [0, 0, 0], [1, 0, 1])
    assert abs(out2[0, 1] + cf) < 1e-14 and abs(out2[0, 0] - out[0, 0]) < 1e-14


def test_riemann_galilean_sampling():
    """Sampling the boosted problem at x/t = 0 equals sampling the original at
    x/t = -V in the solution's own frame: the star state is frame-invariant."""
    gam = 1.4
    rng = np.random.default_rng(2)
    WL, WR = _random_problems(rng, 500, gam=gam)
    v0 = 0.37
    a, _, _ = O.riemann(gam, WL, WR)
    b, _, _ = O.riemann(gam, WL + [0, v0, 0], WR + [0, v0, 0])
    assert np.max(np.abs(a[:, 3] - b[:, 3]) / a[:, 3]) < 1e-12
    assert np.max(np.abs(a[:, 4] + v0 - b[:, 4])) < 1e-10


# ------------------------------------------------------------- whole step
def test_conservation_to_roundoff(turb16):
    """Eq. (eqnupdate) is manifestly conservative: sum_i Q_i is unchanged."""
    M = O.Mesh(turb16.tess)
    Q = turb16.conserved()
    Qn, dt, cnt, rc = O.step(M, Q, turb16.gamma, "lagrangian", cfl=0.3)
    assert rc == 0
    dQ = np.abs(Qn - Q).sum(0)
    d = np.abs(O.totals(M, Qn) - O.totals(M, Q))
    assert np.all(d <= 1e-13 * np.maximum(dQ, 1e-300) + 1e-15 * np.abs(Q).sum(0))


def test_uniform_flow_is_steady():
    """A uniform state with bulk velocity is an exact solution; with a static
    mesh the update leaves it unchanged to roundoff."""
    rng = np.random.default_rng(1)
    pts = ics.jittered_lattice((10, 10, 10), np.ones(3), 0.3, rng)
    T = tessellate(pts, np.ones(3))
    M = O.Mesh(T)
    n = T.n_cells
    Q = ics.conserved_from_primitives(np.full(n, 1.3), np.tile([0.7, -0.2, 0.4], (n, 1)), np.full(n, 2.0),
                                      T.volume, 5.0 / 3.0)
    for mode in ("eulerian", "lagrangian"):
        Qn, dt, cnt, rc = O.step(M, Q, 5.0 / 3.0, mode, cfl=0.4)
        assert rel_err(Qn, Q, q_floor(Q, 3, 5 / 3)) < 1e-13


def test_moving_contact_is_exact():
    """Sec. 8.1: a contact advected with the mesh (w = v, uniform v and P) has
    zero error to machine precision on the moving mesh."""
    P = ics.contact_3d(12)
    M = O.Mesh(P.tess)
    Q = P.conserved()
    Qn, dt, cnt, rc = O.step(M, Q, P.gamma, "lagrangian", cfl=0.4)
    assert rel_err(Qn, Q, q_floor(Q, 3, P.gamma)) < 1e-13
    # while the static mesh smears it (the pin is sensitive to the mesh motion)
    Qe, _, _, _ = O.step(M, Q, P.gamma, "eulerian", dt=dt)
    assert rel_err(Qe, Q, q_floor(Q, 3, P.gamma)) > 1e-3


def G(Q, v0, dim):
    """Eq. (eqngal1): conserved state seen from a frame moving with -v0."""
    m, p, E = Q[:, 0], Q[:, 1:1 + dim], Q[:, dim + 1]
    return np.column_stack([m, p + m[:, None] * v0, E + p @ v0 + 0.5 * m * (v0 @ v0)])


def test_galilean_invariance(turb16):
    """Sec. 3.4: with the mesh moving with the fluid, the update of a boosted
    system equals the boosted update, G(Q_new, v0) = Q_new(boosted)."""
    v0 = 10 * np.sqrt(turb16.gamma) * np.array([1.0, 2.0, 3.0]) / np.sqrt(14)
    M = O.Mesh(turb16.tess)
    Q = turb16.conserved()
    Qa, dt, _, _ = O.step(M, Q, turb16.gamma, "lagrangian", cfl=0.3)
    Qb, _, _, _ = O.step(M, G(Q, v0, 3), turb16.gamma, "lagrangian", dt=dt)
    back = G(Qb, -v0, 3)
    W = O.primitives(M, Q, turb16.tess.volume, turb16.gamma)
    fl = q_floor(Q, 3, turb16.gamma, W)
    assert rel_err(back, Qa, fl) < 1e-12
    # an Eulerian mesh is not invariant: the same check fails clearly
    Qe, _, _, _ = O.step(M, Q, turb16.gamma, "eulerian", dt=dt)
    Qeb, _, _, _ = O.step(M, G(Q, v0, 3), turb16.gamma, "eulerian", dt=dt)
    assert rel_err(G(Qeb, -v0, 3), Qe, fl) > 1e-4


@pytest.mark.parametrize("dims", [(12, 10, 8), (32, 16)])
def test_cartesian_reduction(dims):
    """Sec. 3.2 / Sec. 10: on a stationary Cartesian lattice the scheme is
    the standard unsplit MUSCL-Hancock method (c_ij = 0, gradients become
    central differences)."""
    dim = len(dims)
    h = 1.0 / 16
    box = np.array(dims, np.float64) * h
    nodes, _ = ics.lattice_nodes(dims, box)
    T = tessellate(nodes, box)
    M = O.Mesh(T)
    gam = 1.4
    x = nodes
    rho = 1 + 0.3 * np.sin(2 * np.pi * x[:, 0] / box[0]) + 0.6 * (x[:, 1] > 0.5 * box[1])
    P = 1 + 0.2 * np.cos(2 * np.pi * x[:, 1] / box[1]) + 0.5 * (x[:, 0] < 0.3 * box[0])
    vel = np.column_stack([0.5 * np.sin(2 * np.pi * x[:, d] / box[d] + d) for d in range(dim)])
    Q = ics.conserved_from_primitives(rho, vel, P, T.volume, gam)
    dt = 0.2 * h
    Qn, _, cnt, rc = O.step(M, Q, gam, "eulerian", dt=dt)
    W = np.column_stack([rho, vel, P]).T.reshape((dim + 2,) + dims)

    def riem(a, b):
        return O.riemann(gam, a, b)[0]

    Qs = _structured.step(W, h, dt, gam, riem).reshape(dim + 2, -1).T
    fl = q_floor(Q, dim, gam, np.column_stack([rho, vel, P]))
    assert rel_err(Qn, Qs, fl) < 1e-13
    # the limiter is exercised
    assert rel_err(Qn, _structured.step(W, h, dt, gam, riem, limit=False).reshape(dim + 2, -1).T, fl) > 1e-6


def _sod_exact(x, t, gam=1.4):
    """Exact density of the periodic double shock tube at time t (two mirrored
    Riemann problems at x = 0.5 and 1.5, no wave interaction before t ~ 0.2),
    sampled through the oracle's Riemann solver in the shifted frame."""
    hi = [1.0, 0.0, 1.0]
    lo = [0.125, 0.0, 0.1]
    xr = np.where(x < 1.0, x - 0.5, 1.5 - x)   # mirror the left problem
    S = xr / t
    WL = np.tile(lo, (len(x), 1))
    WR = np.tile(hi, (len(x), 1))
    # solution at x/t = S equals the solution at 0 of the problem seen moving with S
    WL[:, 1] -= S
    WR[:, 1] -= S
    out, _, _ = O.riemann(gam, WL, WR)
    return out[:, 0]


def test_sod_converges_to_exact_solution():
    """Shock tube (Sec. 8.2 family): the L1 density error against the exact
    self-similar solution falls as the resolution doubles (static mesh,
    CFL 0.3, t = 0.2).  No L1 value is printed in the paper for this setup,
    so only the trend is pinned."""
    errs = []
    for nx in (32, 64):
        P = ics.sod_2d(nx, nx // 2, seed=1)
        M = O.Mesh(P.tess)
        V, s = O.geometry(M)
        Q = P.conserved()
        t = 0.0
        while t < 0.2 - 1e-12:
            W = O.primitives(M, Q, V, P.gamma)
            dt, _ = O.timestep(M, W, V, None, P.gamma, 0.3)
            dt = min(dt, 0.2 - t)
            Q, _, cnt, rc = O.step(M, Q, P.gamma, "eulerian", dt=dt, geom=(V, s))
            assert rc == 0
            t += dt
        rho = Q[:, 0] / V
        xs = s[:, 0]
        ex = _sod_exact(xs, 0.2)
        errs.append(np.sum(np.abs(rho - ex) * V) / V.sum())
    assert errs[1] < 0.75 * errs[0]
    assert errs[1] < 0.02


def test_thread_count_does_not_change_the_step():
    """The oracle's per-cell and per-face loops may run on several host
    threads; every output (state, time step, counters) is bit-identical to
    the single-thread run."""
    P = ics.turbulent_3d(12, seed=2)
    M = O.Mesh(P.tess)
    Q = P.conserved()
    O.set_threads(1)
    ref = O.step(M, Q, P.gamma, "lagrangian", cfl=0.3)
    try:
        for t in (3, 8):
            O.set_threads(t)
            out = O.step(M, Q, P.gamma, "lagrangian", cfl=0.3)
            assert np.array_equal(out[0], ref[0]) and out[1] == ref[1]
            assert np.array_equal(np.asarray(out[2]), np.asarray(ref[2])) and out[3] == ref[3]
    finally:
        O.set_threads(1)
