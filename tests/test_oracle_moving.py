"""The oracle's whole moving-mesh cycle with a new tessellation every step
(Sec. 3, steps 1-8), pinned on Gresho's triangle vortex (Sec. 8.5):

- the initial pressure balances the centrifugal force (the profile's
  defining property), checked by finite differences;
- Galilean invariance: on the moving mesh the vortex's azimuthal-velocity
  error does not depend on the bulk velocity v_vortex (Sec. 8.5 reports the
  same to machine precision), while on the fixed mesh it grows with it;
- mass, momentum and energy are conserved across the re-tessellations.
A dropped or mis-signed face-velocity term breaks the invariance; a face
missed in the update breaks conservation."""
import numpy as np
import pytest

from harness import ics, moving
from oracle import oracle as O


def test_gresho_profile_is_in_equilibrium():
    r = np.linspace(0.01, 0.6, 3000)
    r = r[np.min(np.abs(r[:, None] - np.array([0.2, 0.4])[None, :]), axis=1) > 2e-3]
    h = 1e-6
    _, pp = ics.gresho_profile(r + h)
    _, pm = ics.gresho_profile(r - h)
    v, _ = ics.gresho_profile(r)
    np.testing.assert_allclose((pp - pm) / (2 * h), v * v / r, rtol=1e-6, atol=1e-7)
    # continuous at the two kinks
    for rk in (0.2, 0.4):
        vl, pl = ics.gresho_profile(rk - 1e-12)
        vr, pr = ics.gresho_profile(rk + 1e-12)
        assert abs(vl - vr) < 1e-10 and abs(pl - pr) < 1e-10
    assert abs(ics.gresho_profile(0.0)[1] - 5.0) < 1e-15


def _run(v_vortex, mode, n=16, t_end=0.1, regularize=False):
    O.set_threads(4)
    P = ics.gresho_2d(n, jitter=0.1, seed=3, v_vortex=v_vortex)
    tess, Q, t, k = moving.run(P, moving.OracleBackend(O, mode, regularize=regularize), t_end=t_end)
    return P, tess, Q, t, k


@pytest.mark.parametrize("regularize", [False, True])
def test_moving_mesh_is_galilean_invariant(regularize):
    runs = {v: _run(v, "lagrangian", regularize=regularize) for v in (0.0, 3.0)}
    (P0, T0, Q0, t0, k0), (P3, T3, Q3, t3, k3) = runs[0.0], runs[3.0]
    assert k0 == k3 and abs(t0 - t3) < 1e-15
    l0, l3 = moving.gresho_l1(T0, Q0, t0, 0.0), moving.gresho_l1(T3, Q3, t3, 3.0)
    assert l0 > 1e-3                                  # the vortex did evolve
    assert abs(l0 - l3) < 1e-9 * l0, (l0, l3)
    # cell by cell: the same masses and energies in the vortex frame
    np.testing.assert_allclose(Q3[:, 0], Q0[:, 0], rtol=1e-10)
    v0 = Q0[:, 1:3] / Q0[:, :1]
    v3 = Q3[:, 1:3] / Q3[:, :1] - np.array([3.0, 0.0])
    np.testing.assert_allclose(v3, v0, atol=1e-9)
    d = T3.points - T0.points - np.array([3.0 * t3, 0.0])
    d -= np.round(d)
    assert np.abs(d).max() < 1e-10


def test_fixed_mesh_error_grows_with_bulk_velocity():
    l1 = {}
    for v in (0.0, 3.0):
        P, T, Q, t, k = _run(v, "eulerian")
        l1[v] = moving.gresho_l1(T, Q, t, v)
    assert l1[3.0] > 1.2 * l1[0.0], l1


def test_moving_mesh_conserves_across_retessellation():
    P, T, Q, t, k = _run(1.0, "lagrangian", n=20, t_end=0.1)
    assert k > 10 and T.n_cells == P.tess.n_cells
    tot0, tot = P.conserved().sum(0), Q.sum(0)
    np.testing.assert_allclose(tot, tot0, rtol=1e-12, atol=1e-13)
    # the neighbourhoods changed: faces came and went
    pairs = lambda tess: {(min(a, b), max(a, b)) for a, b in tess.cells.tolist()}
    assert len(pairs(T) ^ pairs(P.tess)) > 10


def test_gresho_l1_converges_on_the_fixed_mesh():
    """Sec. 8.5: the azimuthal-velocity error converges below second order
    (the paper fits N^-1.4 at t = 3; the vorticity jumps at r = 0.2 and 0.4
    limit it); here at t = 1 from 16^2 to 64^2 the overall slope lies in
    [1, 2], and the error at 32^2 is a few per cent of the peak speed."""
    O.set_threads(8)
    l1 = {}
    for n in (16, 32, 64):
        P = ics.gresho_2d(n)
        M = O.Mesh(P.tess)
        V, s = O.geometry(M)
        Q, t = P.conserved(), 0.0
        while t < 1.0 * (1 - 1e-14):
            W = O.primitives(M, Q, V, P.gamma)
            dt = min(O.timestep(M, W, V, None, P.gamma, 0.3)[0], 1.0 - t)
            Q, _, _, rc = O.step(M, Q, P.gamma, "eulerian", dt=dt, geom=(V, s))
            assert rc == 0
            t += dt
        l1[n] = moving.gresho_l1(P.tess, Q, t)
    slope = np.log(l1[16] / l1[64]) / np.log(4.0)
    assert 1.0 < slope < 2.0, l1
    assert l1[32] < 0.05, l1
