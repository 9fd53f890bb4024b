"""The oracle's global Courant step, eq. (EqnTiStep) of Sec. 7.1, pinned by
cases whose answer is known without the oracle's formula:

- on an exact Cartesian lattice every cell is a cube (square) of side h, so
  the cell's effective radius is that of the sphere (disc) of the same
  volume: (4/3) pi R^3 = h^3 in 3D, pi R^2 = h^2 in 2D.  The states are
  chosen so that the signal speed is a round number (c = 1 for rho = 1,
  P = 3/5, gamma = 5/3; |v| = 5 from v = (3, 4, 0)), so the step inverts to
  R = dt (c + |v - w|) / C, and that R must satisfy the volume identity;
- the velocity that enters is the one relative to the mesh: w = 0 (static
  mesh) sees c + |v|, w = v (cells moving with the flow) sees c alone, and
  an explicit w sees c + |v - w| -- a |v| in place of |v - w| fails the last
  two;
- one hot cell (P raised 100-fold, so c = 10) sets the global minimum, at
  that cell, with the value known by hand; the other cells keep theirs;
- on a jittered mesh the cells differ in volume and the per-cell step
  follows each cell's own volume (the tessellator's direct polytope
  integral), so the radius must be taken per cell, in the right dimension.
"""
import math

import numpy as np
import pytest

from harness import ics
from harness.tess import tessellate
from oracle import oracle as O

GAMMA = 5.0 / 3.0
CFL = 0.3


def _lattice(dim, n):
    box = np.ones(dim)
    pts, _ = ics.lattice_nodes((n,) * dim, box)
    T = tessellate(pts, box)
    M = O.Mesh(T)
    V, _ = O.geometry(M)
    return T, M, V


def _state(n_cells, dim, v):
    W = np.zeros((n_cells, dim + 2))
    W[:, 0] = 1.0
    W[:, dim + 1] = 0.6                       # c = sqrt(gamma P / rho) = 1
    W[:, 1:dim + 1] = v[:dim]
    return W


def _radius_from_volume_identity(dim, h):
    """The radius of the sphere (disc) whose volume (area) is h^dim."""
    return (3.0 * h ** 3 / (4.0 * math.pi)) ** (1.0 / 3.0) if dim == 3 else h / math.sqrt(math.pi)


@pytest.mark.parametrize("dim,n", [(3, 8), (2, 16)])
def test_courant_step_on_exact_lattice(dim, n):
    T, M, V = _lattice(dim, n)
    h = 1.0 / n
    np.testing.assert_allclose(V, h ** dim, rtol=1e-13)
    v = np.array([3.0, 4.0, 0.0])             # |v| = 5
    W = _state(T.n_cells, dim, v)
    R = _radius_from_volume_identity(dim, h)
    # static mesh: c + |v| = 6
    dt, dtc = O.timestep(M, W, V, None, GAMMA, CFL)
    np.testing.assert_allclose(dtc, CFL * R / 6.0, rtol=1e-14)
    assert dt == dtc.min()
    # the inverted radius satisfies the volume identity
    Rg = dt * 6.0 / CFL
    vol = (4.0 / 3.0) * math.pi * Rg ** 3 if dim == 3 else math.pi * Rg ** 2
    assert abs(vol - h ** dim) <= 1e-13 * h ** dim
    # cells moving with the flow: only c = 1 remains
    dtl, _ = O.timestep(M, W, V, W[:, 1:dim + 1].copy(), GAMMA, CFL)
    assert abs(dtl - CFL * R) <= 1e-14 * CFL * R
    # an explicit mesh velocity: |v - w| = |(3, 4) - (0, 4)| = 3, so c + 3 = 4
    w = np.zeros((T.n_cells, dim))
    w[:, 1] = 4.0
    dte, dtce = O.timestep(M, W, V, w, GAMMA, CFL)
    np.testing.assert_allclose(dtce, CFL * R / 4.0, rtol=1e-14)
    # and the CFL number enters linearly
    dt2, _ = O.timestep(M, W, V, w, GAMMA, 2 * CFL)
    assert abs(dt2 - 2 * dte) <= 1e-15 * dte


@pytest.mark.parametrize("dim,n", [(3, 8), (2, 16)])
def test_hot_cell_sets_the_global_minimum(dim, n):
    T, M, V = _lattice(dim, n)
    h = 1.0 / n
    R = _radius_from_volume_identity(dim, h)
    W = _state(T.n_cells, dim, np.zeros(3))
    hot = T.n_cells // 3
    W[hot, dim + 1] = 60.0                    # c = 10 there
    dt, dtc = O.timestep(M, W, V, None, GAMMA, CFL)
    assert int(np.argmin(dtc)) == hot
    assert abs(dt - CFL * R / 10.0) <= 1e-14 * dt
    cold = np.delete(dtc, hot)
    np.testing.assert_allclose(cold, CFL * R, rtol=1e-14)
    # a heavier hot cell at the same pressure has a lower sound speed:
    # rho = 100 brings c back to 1 and the minimum back to C R
    W[hot, 0] = 100.0
    dt, _ = O.timestep(M, W, V, None, GAMMA, CFL)
    assert abs(dt - CFL * R) <= 1e-14 * dt


@pytest.mark.parametrize("dim,n,jit", [(3, 7, 0.3), (2, 13, 0.3)])
def test_step_follows_each_cells_own_volume(dim, n, jit):
    rng = np.random.default_rng(11)
    box = np.ones(dim)
    pts = ics.jittered_lattice((n,) * dim, box, jit, rng)
    T = tessellate(pts, box)
    M = O.Mesh(T)
    V, _ = O.geometry(M)
    # the volumes the tessellator integrated directly from each polytope
    np.testing.assert_allclose(V, T.volume, rtol=1e-12)
    assert V.std() > 0.05 * V.mean()
    W = _state(T.n_cells, dim, np.zeros(3))
    _, dtc = O.timestep(M, W, V, None, GAMMA, CFL)
    Rg = dtc / CFL                           # c = 1, v = 0
    vol = (4.0 / 3.0) * np.pi * Rg ** 3 if dim == 3 else np.pi * Rg ** 2
    np.testing.assert_allclose(vol, T.volume, rtol=1e-12)
    # the largest cell has the longest step, the smallest the shortest
    assert int(np.argmax(dtc)) == int(np.argmax(T.volume))
    assert int(np.argmin(dtc)) == int(np.argmin(T.volume))
