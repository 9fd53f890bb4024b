"""Independent structured-grid MUSCL-Hancock step (periodic Cartesian grid,
static mesh), the textbook scheme the moving-mesh method reduces to when the
generators form a stationary Cartesian lattice (Sec. 3.2 and Sec. 10).

Written on array axes with central-difference slopes, the same limiter
definition, the same half-step predictor and the same exact Riemann solver
(called through the oracle, which is pinned separately), so the unstructured
machinery (face geometry, Voronoi gradient, limiter over face centroids,
predictor, flux assembly, signed update) is checked against a formulation
that shares none of it.  Test helper only.
"""
import numpy as np


def step(W, h, dt, gamma, riemann, limit=True):
    """W: [nv, *grid] primitives (rho, v_1..v_D, P).  Returns Q_new [nv, *grid]
    (cell totals m, p, E) after one step."""
    dim = W.ndim - 1
    nv = dim + 2
    grid = W.shape[1:]
    vol = h ** dim
    area = h ** (dim - 1)
    # central-difference gradients g[var, axis]
    g = np.empty((nv, dim) + grid)
    for a in range(dim):
        g[:, a] = (np.roll(W, -1, axis=1 + a) - np.roll(W, 1, axis=1 + a)) / (2.0 * h)
    if limit:
        nbrs = [np.roll(W, s, axis=1 + a) for a in range(dim) for s in (1, -1)]
        wmax = np.max(np.stack([W] + nbrs), axis=0)
        wmin = np.min(np.stack([W] + nbrs), axis=0)
        alpha = np.ones_like(W)
        for a in range(dim):
            for sgn in (1.0, -1.0):
                dphi = g[:, a] * (sgn * 0.5 * h)
                with np.errstate(divide="ignore", invalid="ignore"):
                    psi = np.where(dphi > 0, (wmax - W) / dphi, np.where(dphi < 0, (wmin - W) / dphi, 1.0))
                alpha = np.minimum(alpha, psi)
        g = g * alpha[:, None]
    rho, v, P = W[0], W[1:1 + dim], W[dim + 1]
    divv = sum(g[1 + a, a] for a in range(dim))
    dW = np.empty_like(W)
    dW[0] = -(sum(v[a] * g[0, a] for a in range(dim)) + rho * divv)
    for b in range(dim):
        dW[1 + b] = -sum(v[a] * g[1 + b, a] for a in range(dim)) - g[dim + 1, b] / rho
    dW[dim + 1] = -(gamma * P * divv + sum(v[a] * g[dim + 1, a] for a in range(dim)))
    m = rho * vol
    Q = np.concatenate([m[None], m[None] * v, (vol * (P / (gamma - 1) + 0.5 * rho * np.sum(v * v, 0)))[None]])
    for a in range(dim):
        # face between cell c and its +a neighbour
        WL = W + 0.5 * h * g[:, a] + 0.5 * dt * dW
        Wn, gn, dWn = (np.roll(x, -1, axis=1 + a) for x in (W, g[:, a], dW))
        WR = Wn - 0.5 * h * gn + 0.5 * dt * dWn
        bad = (WL[0] <= 0) | (WL[dim + 1] <= 0) | (WR[0] <= 0) | (WR[dim + 1] <= 0)
        WL = np.where(bad[None], W, WL)
        WR = np.where(bad[None], Wn, WR)
        prob_l = np.stack([WL[0], WL[1 + a], WL[dim + 1]], -1).reshape(-1, 3)
        prob_r = np.stack([WR[0], WR[1 + a], WR[dim + 1]], -1).reshape(-1, 3)
        out = riemann(prob_l, prob_r).reshape(grid + (6,))
        rF, uF, PF, side = out[..., 0], out[..., 1], out[..., 2], out[..., 5]
        vt = np.where(side[None] > 0.5, WR[1:1 + dim], WL[1:1 + dim])
        vlab = vt.copy()
        vlab[a] = uF
        F = np.empty_like(W)
        F[0] = rF * uF
        for b in range(dim):
            F[1 + b] = rF * vlab[b] * uF + (PF if b == a else 0.0)
        F[dim + 1] = (0.5 * rF * np.sum(vlab * vlab, 0) + PF / (gamma - 1)) * uF + PF * uF
        Q = Q - dt * area * (F - np.roll(F, 1, axis=1 + a))
    return Q
