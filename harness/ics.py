"""Seeded synthetic initial conditions shaped like the paper's test problems.

Every generator draws from `numpy.random.default_rng(seed)` in a fixed order,
so a (config, seed) pair always yields the same points and states.  The
recipes (lattice sizes, jitter, spectra, amplitudes) are the workloads the
hydro update is exercised on:

* `sod_2d`: the two-dimensional shock tube (Sec. 8.2 test family) as a
  periodic box [0,2]x[0,1] holding two mirrored Riemann problems.
* `turbulent_3d`: a jittered 3D lattice with a random-phase Gaussian velocity
  field, P(k) ~ k^-4 on 2 <= |k| <= 8 (units of 2 pi / L), at a given rms Mach
  number.
* `lognormal_3d`: log-normal density (sigma_lnrho given), p = rho^gamma, and
  the same Gaussian velocity spectrum.
* `ensemble`: many independent periodic boxes of log-uniform size.
* `contact_3d` / `lattice_*`: the special cases the tests use.

Conserved states are built from primitives with the cell volumes the
tessellator integrated directly: m = rho V, p = m v, E = V (P/(gamma-1) +
rho v^2 / 2).
"""
from dataclasses import dataclass, field

import numpy as np

from .tess import Tessellation, tessellate


@dataclass
class Problem:
    name: str
    dim: int
    gamma: float
    tess: Tessellation
    rho: np.ndarray          # [n]
    vel: np.ndarray          # [n, dim]
    pres: np.ndarray         # [n]
    meta: dict = field(default_factory=dict)

    @property
    def n_cells(self):
        return self.tess.n_cells

    @property
    def n_faces(self):
        return self.tess.n_faces

    def conserved(self):
        return conserved_from_primitives(self.rho, self.vel, self.pres, self.tess.volume, self.gamma)


def conserved_from_primitives(rho, vel, pres, vol, gamma):
    """Q = (m, p, E) per cell from (rho, v, P) and the cell volume."""
    m = rho * vol
    mom = m[:, None] * vel
    ene = vol * (pres / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=1))
    return np.concatenate([m[:, None], mom, ene[:, None]], axis=1)


def lattice_nodes(dims, box):
    """Cell-centred lattice nodes, row-major with the last axis fastest."""
    dims = tuple(int(d) for d in dims)
    h = np.asarray(box, np.float64) / np.asarray(dims, np.float64)
    idx = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), -1).reshape(-1, len(dims))
    return (idx + 0.5) * h, h


def jittered_lattice(dims, box, jitter, rng):
    """Lattice nodes displaced by U(-jitter*h, +jitter*h) per coordinate."""
    nodes, h = lattice_nodes(dims, box)
    pts = nodes + rng.uniform(-1.0, 1.0, nodes.shape) * (jitter * h)
    box = np.asarray(box, np.float64)
    pts = np.mod(pts, box)
    return np.where(pts >= box, pts - box, pts)


def gaussian_field(shape, kmin, kmax, slope, rng):
    """Zero-mean, unit-variance Gaussian random field on a periodic grid.

    White noise filtered in Fourier space by sqrt(P(k)) with P(k) ~ k^slope on
    kmin <= |k| <= kmax (k in units of the fundamental mode), zero elsewhere.
    """
    white = rng.standard_normal(shape)
    fk = np.fft.rfftn(white)
    ks = [np.fft.fftfreq(n) * n for n in shape[:-1]] + [np.fft.rfftfreq(shape[-1]) * shape[-1]]
    grids = np.meshgrid(*ks, indexing="ij", sparse=True)
    kk = np.sqrt(sum(g * g for g in grids))
    ksafe = np.where(kk > 0, kk, 1.0)
    amp = np.where((kk >= kmin) & (kk <= kmax), ksafe ** (0.5 * slope), 0.0)
    f = np.fft.irfftn(fk * amp, s=shape, axes=tuple(range(len(shape))))
    f -= f.mean()
    f /= f.std()
    return f


def velocity_field(dims, rng, rms, kmin=2, kmax=8, slope=-4.0):
    """Per-component independent Gaussian fields rescaled to rms |v| = rms."""
    comps = [gaussian_field(tuple(dims), kmin, kmax, slope, rng).reshape(-1) for _ in range(len(dims))]
    v = np.stack(comps, axis=1)
    v -= v.mean(axis=0)
    v *= rms / np.sqrt(np.mean(np.sum(v * v, axis=1)))
    return v


def sod_2d(nx=128, ny=64, jitter=0.1, seed=1, gamma=1.4, nthreads=0):
    """Periodic [0,2]x[0,1]: rho=1,P=1 for 0.5<x<1.5, rho=0.125,P=0.1 elsewhere, v=0."""
    rng = np.random.default_rng(seed)
    box = np.array([2.0, 1.0])
    pts = jittered_lattice((nx, ny), box, jitter, rng)
    T = tessellate(pts, box, nthreads)
    inside = (pts[:, 0] > 0.5) & (pts[:, 0] < 1.5)
    rho = np.where(inside, 1.0, 0.125)
    pres = np.where(inside, 1.0, 0.1)
    vel = np.zeros((len(pts), 2))
    return Problem("sod_2d", 2, gamma, T, rho, vel, pres,
                   dict(dims=(nx, ny), jitter=jitter, seed=seed, cfl=0.3, t_end=0.2))


def turbulent_3d(n=64, jitter=0.2, seed=2, mach=2.0, gamma=5.0 / 3.0, nthreads=0, box=1.0):
    """rho=1, P=1, Gaussian velocity field (k^-4, 2<=k<=8) at rms Mach `mach`."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    boxv = np.array([box] * 3, np.float64)
    pts = jittered_lattice(dims, boxv, jitter, rng)
    T = tessellate(pts, boxv, nthreads)
    cs = np.sqrt(gamma * 1.0 / 1.0)
    vel = velocity_field(dims, rng, mach * cs)
    rho = np.ones(len(pts))
    pres = np.ones(len(pts))
    return Problem("turbulent_3d", 3, gamma, T, rho, vel, pres,
                   dict(dims=dims, jitter=jitter, seed=seed, mach=mach))


def lognormal_3d(n=192, jitter=0.2, seed=3, sigma=1.0, mach=3.0, gamma=5.0 / 3.0, nthreads=0):
    """ln rho Gaussian (k^-4, 2<=k<=8) with sigma_lnrho, mean rho 1; P = rho^gamma; rms v = mach c_s(rho=1)."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    boxv = np.ones(3)
    pts = jittered_lattice(dims, boxv, jitter, rng)
    T = tessellate(pts, boxv, nthreads)
    g = gaussian_field(dims, 2, 8, -4.0, rng).reshape(-1)
    rho = np.exp(sigma * g - 0.5 * sigma * sigma)
    rho /= rho.mean()
    pres = rho ** gamma
    cs = np.sqrt(gamma)
    vel = velocity_field(dims, rng, mach * cs)
    return Problem("lognormal_3d", 3, gamma, T, rho, vel, pres,
                   dict(dims=dims, jitter=jitter, seed=seed, sigma=sigma, mach=mach))


def gresho_profile(r):
    """Azimuthal velocity and pressure of the triangle vortex (Sec. 8.5) at
    radius r: v_phi = 5r, 2 - 5r, 0 on r < 0.2, 0.2 <= r < 0.4, r >= 0.4, and
    P = 5 + 25/2 r^2, 9 + 25/2 r^2 - 20r + 4 ln(r/0.2), 3 + 4 ln 2 there, so
    that dP/dr = rho v_phi^2 / r with rho = 1."""
    r = np.asarray(r, np.float64)
    vphi = np.where(r < 0.2, 5 * r, np.where(r < 0.4, 2 - 5 * r, 0.0))
    mid = 9 + 12.5 * r * r - 20 * r + 4 * np.log(np.clip(r, 0.2, 0.4) / 0.2)
    pres = np.where(r < 0.2, 5 + 12.5 * r * r, np.where(r < 0.4, mid, 3 + 4 * np.log(2.0)))
    return vphi, pres


def gresho_2d(n=40, jitter=0.0, seed=11, v_vortex=0.0, gamma=5.0 / 3.0, nthreads=0):
    """Gresho's triangle vortex (Sec. 8.5): unit periodic box, rho = 1, the
    profile of gresho_profile about (0.5, 0.5) sampled at the generators, plus
    a uniform v_vortex along x; n x n generators (a Cartesian lattice unless
    jittered)."""
    rng = np.random.default_rng(seed)
    box = np.array([1.0, 1.0])
    pts = jittered_lattice((n, n), box, jitter, rng)
    T = tessellate(pts, box, nthreads)
    dx, dy = pts[:, 0] - 0.5, pts[:, 1] - 0.5
    r = np.hypot(dx, dy)
    vphi, pres = gresho_profile(r)
    rs = np.where(r > 0, r, 1.0)
    vel = np.column_stack([-vphi * dy / rs + v_vortex, vphi * dx / rs])
    rho = np.ones(len(pts))
    return Problem("gresho_2d", 2, gamma, T, rho, vel, pres, dict(n=n, jitter=jitter, seed=seed, v_vortex=v_vortex))


def sedov(dim=3, n=64, jitter=0.0, seed=13, E=1.0, rho0=1.0, p0=1e-4, gamma=5.0 / 3.0, nthreads=0):
    """Point explosion (Sec. 8.4): a cold uniform gas (rho0, p0) in the
    periodic unit box, n^dim generators, with the energy E put into the one
    cell whose generator lies nearest to the box centre; that generator is
    the explosion centre (meta['centre'])."""
    rng = np.random.default_rng(seed)
    box = np.ones(dim)
    pts = jittered_lattice((n,) * dim, box, jitter, rng)
    T = tessellate(pts, box, nthreads)
    c = int(np.argmin(np.sum((pts - 0.5) ** 2, axis=1)))
    rho = np.full(len(pts), rho0)
    vel = np.zeros((len(pts), dim))
    pres = np.full(len(pts), p0)
    pres[c] += (gamma - 1.0) * E / T.volume[c]
    return Problem("sedov_%dd" % dim, dim, gamma, T, rho, vel, pres,
                   dict(n=n, jitter=jitter, seed=seed, E=E, rho0=rho0, p0=p0, centre=pts[c].copy(), cell=c))


def sedov_radius(t, E=1.0, rho0=1.0, beta=1.15):
    """Shock radius of the self-similar blast wave, beta (E t^2 / rho0)^(1/5)
    (3D; beta = 1.15 for gamma = 5/3, Sec. 8.4)."""
    return beta * (E * t * t / rho0) ** 0.2


def contact_3d(n=12, jitter=0.2, seed=7, v=(1.0, 0.5, -0.25), gamma=5.0 / 3.0):
    """Uniform velocity and pressure P=3/5, density 1 | 2 across x=0.5 (moving contact)."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    boxv = np.ones(3)
    pts = jittered_lattice(dims, boxv, jitter, rng)
    T = tessellate(pts, boxv)
    rho = np.where(pts[:, 0] < 0.5, 1.0, 2.0)
    pres = np.full(len(pts), 0.6)
    vel = np.tile(np.asarray(v, np.float64), (len(pts), 1))
    return Problem("contact_3d", 3, gamma, T, rho, vel, pres, dict(dims=dims, seed=seed))


def ensemble_sizes(nboxes=64, seed=5, nmin=16, nmax=96):
    """Per-box lattice size n_b = round(exp(U(ln nmin, ln nmax))) and rms Mach U[0.5, 4]."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), nboxes))).astype(int)
    machs = rng.uniform(0.5, 4.0, nboxes)
    seeds = rng.integers(0, 2**31 - 1, nboxes)
    return sizes, machs, seeds


def ensemble(nboxes=64, seed=5, nmin=16, nmax=96, jitter=0.2, gamma=5.0 / 3.0, nthreads=0):
    """Independent unit periodic boxes, each a `turbulent_3d` field of its own size and Mach."""
    sizes, machs, seeds = ensemble_sizes(nboxes, seed, nmin, nmax)
    return [turbulent_3d(int(n), jitter, int(s), float(m), gamma, nthreads) for n, m, s in zip(sizes, machs, seeds)]


def boosted(problem, v0):
    """The same problem seen from a frame moving with -v0: every fluid velocity gets +v0."""
    v0 = np.asarray(v0, np.float64)
    return Problem(problem.name + "_boosted", problem.dim, problem.gamma, problem.tess, problem.rho.copy(),
                   problem.vel + v0[None, :], problem.pres.copy(), dict(problem.meta, boost=v0.tolist()))


@dataclass
class Ensemble:
    """Independent periodic boxes concatenated into one face list: global cell
    indices, per-box box lengths and the cell/face offsets of each box."""
    dim: int
    points: np.ndarray
    cells: np.ndarray
    shift: np.ndarray
    area: np.ndarray
    centroid: np.ndarray
    box: np.ndarray            # [n_boxes, dim]
    Q: np.ndarray
    box_cells: np.ndarray      # [n_boxes+1]
    box_faces: np.ndarray      # [n_boxes+1]
    gamma: float
    problems: list

    @property
    def n_cells(self):
        return len(self.points)

    @property
    def n_faces(self):
        return len(self.area)


def concat(problems):
    """Concatenates problems (same dim and gamma) into an Ensemble."""
    dim = problems[0].dim
    gamma = problems[0].gamma
    pts, cells, sh, ar, cen, boxes, Qs = [], [], [], [], [], [], []
    bc, bf = [0], [0]
    for P in problems:
        assert P.dim == dim and P.gamma == gamma
        T = P.tess
        off = bc[-1]
        pts.append(T.points)
        cells.append(T.cells + off)
        sh.append(T.shift)
        ar.append(T.area)
        cen.append(T.centroid)
        boxes.append(T.box)
        Qs.append(P.conserved())
        bc.append(off + T.n_cells)
        bf.append(bf[-1] + T.n_faces)
    return Ensemble(dim, np.concatenate(pts), np.concatenate(cells).astype(np.int32), np.concatenate(sh),
                    np.concatenate(ar), np.concatenate(cen), np.stack(boxes), np.concatenate(Qs),
                    np.asarray(bc, np.int64), np.asarray(bf, np.int64), gamma, list(problems))
