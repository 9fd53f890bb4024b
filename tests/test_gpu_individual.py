"""Individual power-of-two time steps on the GPU (amm_advance_individual,
Sec. 7.2) against the oracle's cycle (oracle.advance_individual): the same
bins, the same counters (sub-steps, face fluxes, activations) and the same
state (FP64 1e-12, FP32 2e-5 per element against max(|Q|, the column's
scale)), on the point explosion (Sec. 8.4) in 2D and 3D, a translating
linear profile, and a turbulent box; a one-bin cycle is one global step; at
64^3 the explosion reaches the self-similar radius with several times fewer
face fluxes than global steps."""
import math

import numpy as np
import pytest

from harness import ics
from harness.tess import tessellate
from oracle import oracle as O

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module")
def amm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_4107_gb300 import amm as A
    O.set_threads(8)
    return A


def rel_err(out, ref, Q0, M, V, gamma):
    d = M.dim
    W = O.primitives(M, Q0, V, gamma)
    fl = np.sqrt(np.mean(Q0 * Q0, axis=0))
    c = np.sqrt(gamma * W[:, d + 1] / W[:, 0])
    fl[1:d + 1] = np.sqrt(np.mean((Q0[:, 0] * c) ** 2))
    return np.max(np.abs(out - ref) / np.maximum(np.abs(ref), fl))


def run_both(amm, tess, Q, gamma, prec, dt_max, cycles=1, signal=True, cfl=0.3, depth=30):
    M = O.Mesh(tess)
    V, s = O.geometry(M)
    ctx = amm.create_from_mesh(tess, Q, gamma, precision=prec, mesh_motion="eulerian")
    Qo, Qg = Q.copy(), None
    out = []
    for _ in range(cycles):
        Qo, bo, co, rc = O.advance_individual(M, Qo, gamma, cfl, dt_max, max_depth=depth, signal=signal, geom=(V, s))
        assert rc == 0
        st = amm.amm_advance_individual(ctx, cfl, dt_max, depth, signal)
        Qg = amm.amm_get_state(ctx)
        bg = amm.amm_get_bins(ctx)
        out.append((Qo.copy(), bo, co, Qg, bg, st))
    amm.amm_destroy(ctx)
    return M, V, out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sedov_2d_cycles_match_oracle(amm, prec):
    P = ics.sedov(2, 45)
    Q0 = P.conserved()
    M, V, out = run_both(amm, P.tess, Q0, P.gamma, prec, 0.01, cycles=3 if prec == "fp64" else 1)
    for c, (Qo, bo, co, Qg, bg, st) in enumerate(out):
        assert np.array_equal(bo, bg), (c, np.sum(bo != bg))
        assert (st["substeps"], st["face_fluxes"], st["activations"]) == (co[4], co[5], co[6]), (c, st, co)
        assert st["deepest_bin"] >= bo.max() and len(np.unique(bo)) >= 3
        e = rel_err(Qg, Qo, Q0, M, V, P.gamma)
        assert e < TOL[prec] * (1 + 4 * c), (c, prec, e)


@pytest.mark.parametrize("signal", [True, False])
def test_sedov_3d_cycle_matches_oracle(amm, signal):
    P = ics.sedov(3, 16)
    Q0 = P.conserved()
    M, V, out = run_both(amm, P.tess, Q0, P.gamma, "fp64", 0.02, signal=signal)
    Qo, bo, co, Qg, bg, st = out[0]
    assert np.array_equal(bo, bg)
    assert (st["substeps"], st["face_fluxes"], st["activations"]) == (co[4], co[5], co[6])
    assert rel_err(Qg, Qo, Q0, M, V, P.gamma) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_linear_profile_and_turbulent_box_match_oracle(amm, prec):
    rng = np.random.default_rng(4)
    box = np.array([2.0, 0.5])
    T = tessellate(ics.jittered_lattice((64, 16), box, 0.0, rng), box)
    M = O.Mesh(T)
    V, s = O.geometry(M)
    g, u = 5.0 / 3.0, -0.5
    m = V * (0.3 + 1.35 * s[:, 0])
    Q = np.column_stack([m, m * u, 0.0 * m, V / (g - 1) + 0.5 * m * u * u])
    M, V, out = run_both(amm, T, Q, g, prec, 0.008)
    Qo, bo, co, Qg, bg, st = out[0]
    assert np.array_equal(bo, bg) and len(np.unique(bo)) >= 3
    assert rel_err(Qg, Qo, Q, M, V, g) < TOL[prec]
    P = ics.turbulent_3d(12, seed=3)
    Q = P.conserved()
    M, V, out = run_both(amm, P.tess, Q, P.gamma, prec, 0.01)
    Qo, bo, co, Qg, bg, st = out[0]
    assert np.array_equal(bo, bg)
    assert rel_err(Qg, Qo, Q, M, V, P.gamma) < TOL[prec]


def test_one_bin_cycle_is_a_global_step(amm):
    P = ics.turbulent_3d(12, seed=5)
    Q = P.conserved()
    ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision="fp64", mesh_motion="eulerian")
    dt = 0.5 * float(amm.amm_timestep(ctx, 0.3)[0]) * 0.5     # below every cell's signal-speed criterion
    st = amm.amm_advance_individual(ctx, 0.3, dt, 20, True)
    Qi = amm.amm_get_state(ctx)
    assert st["substeps"] == 1 and st["face_fluxes"] == P.tess.n_faces and np.all(amm.amm_get_bins(ctx) == 0)
    amm.amm_set_state(ctx, Q)
    amm.amm_step(ctx, dt)
    Qs = amm.amm_get_state(ctx)
    amm.amm_destroy(ctx)
    assert np.max(np.abs(Qi - Qs) / np.abs(Q).max(axis=0)) < 1e-14


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sedov_64_radius_and_savings(amm, prec):
    n, t_end, cycles = 64, 0.06, 6
    P = ics.sedov(3, n)
    Q0 = P.conserved()
    ctx = amm.create_from_mesh(P.tess, Q0, P.gamma, precision=prec, mesh_motion="eulerian")
    evals = 0
    for _ in range(cycles):
        st = amm.amm_advance_individual(ctx, 0.3, t_end / cycles, 30, True)
        evals += st["face_fluxes"]
    Q = amm.amm_get_state(ctx)
    # global steps over the same time, for the face-flux count
    amm.amm_set_state(ctx, Q0)
    t, k = 0.0, 0
    while t < t_end * (1 - 1e-14):
        dt = min(float(amm.amm_timestep(ctx, 0.3)[0]), t_end - t)
        amm.amm_step(ctx, dt)
        t += dt
        k += 1
    amm.amm_destroy(ctx)
    assert k * P.tess.n_faces > 3 * evals, (k, evals)
    rho = Q[:, 0] / P.tess.volume
    d = P.tess.points - P.meta["centre"]
    d -= np.round(d)
    r = np.linalg.norm(d, axis=1)
    edges = np.arange(0.0, 0.8, 0.5 / n)
    idx = np.digitize(r, edges)
    prof = np.array([rho[idx == i].mean() if np.any(idx == i) else 0.0 for i in range(1, len(edges))])
    i = int(np.argmax(prof))
    assert abs(0.5 * (edges[i] + edges[i + 1]) / ics.sedov_radius(t_end) - 1) < 0.03
    tot0 = np.array([math.fsum(c) for c in Q0.T])
    tot = np.array([math.fsum(c) for c in Q.T])
    np.testing.assert_allclose(tot[[0, 4]], tot0[[0, 4]], rtol=1e-12)


def test_host_loop_gives_the_same_cycle(amm):
    P = ics.sedov(3, 16)
    Q0 = P.conserved()
    out = {}
    for host in (False, True):
        ctx = amm.create_from_mesh(P.tess, Q0, P.gamma, precision="fp32", mesh_motion="eulerian")
        amm.amm_individual_host_loop(ctx, host)
        st = [amm.amm_advance_individual(ctx, 0.3, 0.01, 30, True) for _ in range(2)]
        out[host] = (amm.amm_get_state(ctx), amm.amm_get_bins(ctx), st)
        amm.amm_destroy(ctx)
    assert np.array_equal(out[False][0], out[True][0])
    assert np.array_equal(out[False][1], out[True][1])
    assert out[False][2] == out[True][2]
