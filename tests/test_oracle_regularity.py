"""Pins of the oracle's mesh-regularity correction (Sec. 4.1, eq.
EqnShapeCorrVel): an extra generator velocity chi c_i towards the cell's
centre of mass, ramped in over 0.9-1.1 eta R_i of generator-to-centroid
distance."""
from types import SimpleNamespace

import numpy as np

from harness import ics
from harness.ics import Problem, lattice_nodes
from harness.tess import tessellate
from oracle import oracle as O


def test_centroidal_lattice_needs_no_correction():
    """On an exact lattice every generator is its cell's centre of mass, so
    the corrected mesh velocity is the uncorrected one, exactly."""
    box = np.array([1.0, 1.0, 1.0])
    pts, _ = lattice_nodes((6, 6, 6), box)
    T = tessellate(pts, box, 0)
    M = O.Mesh(T)
    V, s = O.geometry(M)
    W = np.column_stack([np.ones(len(pts)), np.zeros((len(pts), 3)), np.ones(len(pts))])
    w = np.random.default_rng(1).normal(size=(len(pts), 3))
    assert np.array_equal(O.shape_correction(M, W, V, s, w, 5.0 / 3.0), w)


def test_ramp_of_the_correction():
    """A single cell of volume V (R = (3V/4pi)^(1/3)) with its centre of mass
    at distance d along a fixed direction: no correction below 0.9 eta R, the
    full chi c_i from 1.1 eta R, linear in between, always towards s."""
    gam, eta, chi = 5.0 / 3.0, 0.25, 0.8
    V = np.array([1.0])
    R = (3 * V[0] / (4 * np.pi)) ** (1 / 3)
    W = np.array([[2.0, 0.0, 0.0, 0.0, 3.0]])
    c = np.sqrt(gam * 3.0 / 2.0)
    u = np.array([2.0, -1.0, 2.0]) / 3.0
    for q, ramp in ((0.5, 0.0), (0.89, 0.0), (0.95, 0.25), (1.0, 0.5), (1.05, 0.75), (1.1, 1.0), (2.0, 1.0)):
        gen = np.array([[0.3, 0.2, 0.1]])
        s = gen + q * eta * R * u
        mesh = SimpleNamespace(dim=3, n=1, gen=gen)
        w = np.array([[0.1, 0.2, 0.3]])
        dw = O.shape_correction(mesh, W, V, s, w, gam, eta, chi) - w
        np.testing.assert_allclose(dw[0], chi * c * ramp * u, rtol=1e-12, atol=1e-15)


def test_correction_makes_cells_rounder():
    """One step of generator motion by the correction alone (Delta t = eta R
    / (2 c)), then a new tessellation: the generators end closer to their
    cells' centres of mass (the Lloyd-like relaxation the correction is
    for)."""
    P = ics.turbulent_3d(10, jitter=0.45, seed=8)
    M = O.Mesh(P.tess)
    V, s = O.geometry(M)
    W = O.primitives(M, P.conserved(), V, P.gamma)
    w0 = np.zeros((P.n_cells, 3))
    dw = O.shape_correction(M, W, V, s, w0, P.gamma)
    moved = np.linalg.norm(dw, axis=1) > 0
    assert moved.mean() > 0.1
    R = np.cbrt(3 * V / (4 * np.pi))
    d0 = np.linalg.norm(s - M.gen, axis=1) / R
    dt = 0.25 * R.mean() / (2 * np.sqrt(P.gamma))
    pts = np.mod(P.tess.points + dw * dt, 1.0)
    T1 = tessellate(pts, np.ones(3), 0)
    M1 = O.Mesh(T1)
    V1, s1 = O.geometry(M1)
    d1 = np.linalg.norm(s1 - M1.gen, axis=1) / np.cbrt(3 * V1 / (4 * np.pi))
    assert d1[moved].mean() < 0.9 * d0[moved].mean()
    assert d1.max() < d0.max()
