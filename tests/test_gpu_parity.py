"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle,
element by element on the same seeded inputs.

Tolerances (per cell and component, relative with the floor of the parity
norm: RMS|Q_k| for mass and energy, RMS(m c) for momentum): 1e-12 for the
FP64 form, 2e-5 for the FP32 form.
"""
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
    return A


def floor_of(Q, dim, gamma, W):
    fl = np.sqrt(np.mean(Q * Q, axis=0))
    c = np.sqrt(gamma * W[:, dim + 1] / W[:, 0])
    fl[1:1 + dim] = np.sqrt(np.mean((Q[:, 0] * c) ** 2))
    return fl


def errs(out, ref, floor):
    e = np.abs(out - ref) / np.maximum(np.abs(ref), floor)
    return float(e.max()), float(np.quantile(e, 0.999))


CASES = {
    "sod2d_eulerian": lambda: (ics.sod_2d(32, 16, seed=1), "eulerian"),
    "sod2d_ragged": lambda: (ics.sod_2d(21, 13, seed=3), "lagrangian"),
    "turb16_lagrangian": lambda: (ics.turbulent_3d(16, seed=2), "lagrangian"),
    "turb16_eulerian": lambda: (ics.turbulent_3d(16, seed=4, mach=1.0), "eulerian"),
    "lognormal16_lagrangian": lambda: (ics.lognormal_3d(16, seed=3), "lagrangian"),
    "tiny5_lagrangian": lambda: (ics.turbulent_3d(5, seed=9), "lagrangian"),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    P, mode = CASES[request.param]()
    M = O.Mesh(P.tess)
    Q = P.conserved()
    geom = O.geometry(M)
    W = O.primitives(M, Q, geom[0], P.gamma)
    Qn, dt, cnt, rc = O.step(M, Q, P.gamma, mode, cfl=0.3, geom=geom)
    assert rc == 0
    return dict(name=request.param, P=P, mode=mode, M=M, Q=Q, geom=geom, W=W, ref=Qn, dt=dt, cnt=cnt)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_parity(amm, case, prec):
    P = case["P"]
    ctx = amm.create_from_mesh(P.tess, case["Q"], P.gamma, precision=prec, mesh_motion=case["mode"])
    amm.amm_step(ctx, case["dt"])
    out = amm.amm_get_state(ctx)
    fl = floor_of(case["Q"], P.dim, P.gamma, case["W"])
    emax, e999 = errs(out, case["ref"], fl)
    assert emax < TOL[prec], (case["name"], prec, emax, e999)
    st = amm.amm_get_stats(ctx)
    assert st["steps"] == 1 and st["faces"] == P.n_faces
    assert st["newton_fail"] == 0 and st["nonpositive_cells"] == 0
    assert st["fallback_faces"] == case["cnt"][0]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_timestep_parity(amm, case, prec):
    P = case["P"]
    ctx = amm.create_from_mesh(P.tess, case["Q"], P.gamma, precision=prec, mesh_motion=case["mode"])
    dt = amm.amm_timestep(ctx, 0.3)[0]
    rel = abs(dt - case["dt"]) / case["dt"]
    assert rel < (1e-14 if prec == "fp64" else 1e-6), rel


def test_geometry_matches_oracle(amm, case):
    P = case["P"]
    ctx = amm.create_from_mesh(P.tess, case["Q"], P.gamma, precision="fp64")
    V, s = amm.amm_get_geometry(ctx)
    Vo, so = case["geom"]
    assert np.max(np.abs(V - Vo) / Vo) < 1e-13
    h = np.mean(Vo) ** (1.0 / P.dim)
    assert np.max(np.abs(s - so)) < 1e-13 * h


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gradients_and_flux_parity(amm, case, prec):
    P = case["P"]
    M = case["M"]
    V, s = case["geom"]
    W = case["W"]
    ctx = amm.create_from_mesh(P.tess, case["Q"], P.gamma, precision=prec, mesh_motion=case["mode"])
    g = amm.amm_get_gradients(ctx)
    go = O.gradients(M, W, V, s, limit=True)
    gscale = np.abs(go).reshape(len(go), -1).max(axis=1)[:, None, None] + 1e-300
    var_scale = np.abs(W).max(axis=0)[None, :, None] / np.mean(V) ** (1.0 / P.dim)
    eg = np.abs(g - go) / np.maximum(gscale, var_scale)
    assert eg.max() < (1e-11 if prec == "fp64" else 5e-4), eg.max()
    amm.amm_step(ctx, case["dt"])
    AF = amm.amm_get_face_flux(ctx)
    wm = None if case["mode"] == "eulerian" else W[:, 1:1 + P.dim]
    F, cnt, rc = O.fluxes(M, W, go, s, wm, P.gamma, case["dt"])
    AFo = F * P.tess.area[:, None]
    fscale = np.abs(AFo).max(axis=0)
    ef = np.abs(AF - AFo) / fscale
    assert ef.max() < (1e-11 if prec == "fp64" else 2e-4), ef.max()


def test_conservation_and_totals(amm, case):
    P = case["P"]
    for prec in ("fp64", "fp32"):
        ctx = amm.create_from_mesh(P.tess, case["Q"], P.gamma, precision=prec, mesh_motion=case["mode"])
        t0 = amm.amm_get_totals(ctx)[0]
        assert np.allclose(t0, case["Q"].sum(0), rtol=1e-13, atol=1e-15 * np.abs(case["Q"]).sum(0).max())
        amm.amm_step(ctx, case["dt"])
        t1 = amm.amm_get_totals(ctx)[0]
        out = amm.amm_get_state(ctx)
        dQ = np.abs(out - case["Q"]).sum(0)
        scale = np.abs(case["Q"]).sum(0)
        # each face flux is applied with both signs: only FP64 summation roundoff
        assert np.all(np.abs(t1 - t0) <= 1e-13 * dQ + 1e-15 * scale), (prec, t1 - t0)
        assert np.allclose(t1, out.sum(0), rtol=1e-13, atol=1e-15 * scale.max())


def test_newton_iterations_match_oracle_fp64(amm, case):
    P = case["P"]
    ctx = amm.create_from_mesh(P.tess, case["Q"], P.gamma, precision="fp64", mesh_motion=case["mode"])
    amm.amm_step(ctx, case["dt"])
    st = amm.amm_get_stats(ctx)
    # the same algorithm in the same precision: iteration totals agree up to
    # roundoff flips of the convergence tests (the relative change against
    # 1e-12, and the residual against 64 ulps of its terms, which the two
    # sides evaluate with different rounding): a few per thousand faces
    assert abs(st["newton_iters"] - case["cnt"][2]) <= max(8, 2e-3 * case["cnt"][2])


def test_explicit_mesh_velocity(amm):
    P = ics.turbulent_3d(12, seed=5)
    M = O.Mesh(P.tess)
    Q = P.conserved()
    rng = np.random.default_rng(0)
    w = 0.5 * P.vel + rng.normal(scale=0.3, size=P.vel.shape)
    ref, dt, _, rc = O.step(M, Q, P.gamma, "explicit", wmesh=w, cfl=0.3)
    W = O.primitives(M, Q, P.tess.volume, P.gamma)
    fl = floor_of(Q, 3, P.gamma, W)
    for prec in ("fp64", "fp32"):
        ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision=prec, mesh_motion="explicit")
        amm.amm_set_mesh_velocity(ctx, w)
        assert abs(amm.amm_timestep(ctx, 0.3)[0] - dt) / dt < 1e-6
        amm.amm_step(ctx, dt)
        emax, _ = errs(amm.amm_get_state(ctx), ref, fl)
        assert emax < TOL[prec], (prec, emax)


def test_galilean_invariance_on_gpu(amm):
    """Sec. 3.4 on the device: a boosted run equals the boosted unboosted run."""
    P = ics.turbulent_3d(12, seed=6)
    v0 = 10 * np.sqrt(P.gamma) * np.array([1.0, 2.0, 3.0]) / np.sqrt(14)
    Q = P.conserved()
    Pb = ics.boosted(P, v0)
    Qb = Pb.conserved()
    W = O.primitives(O.Mesh(P.tess), Q, P.tess.volume, P.gamma)
    fl = floor_of(Q, 3, P.gamma, W)
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-3)):
        a = amm.create_from_mesh(P.tess, Q, P.gamma, precision=prec)
        b = amm.create_from_mesh(P.tess, Qb, P.gamma, precision=prec)
        dt = amm.amm_timestep(a, 0.3)[0]
        amm.amm_step(a, dt)
        amm.amm_step(b, dt)
        qa = amm.amm_get_state(a)
        qb = amm.amm_get_state(b)
        m, p, E = qb[:, 0], qb[:, 1:4], qb[:, 4]
        back = np.column_stack([m, p - m[:, None] * v0, E - p @ v0 + 0.5 * m * (v0 @ v0)])
        emax, _ = errs(back, qa, fl)
        assert emax < tol, (prec, emax)


def test_bitwise_reproducible_and_resume(amm):
    """No atomics on the data path: two runs agree bit for bit, and a run
    resumed from a checkpoint equals the uninterrupted run."""
    P = ics.turbulent_3d(16, seed=7)
    Q = P.conserved()
    for prec in ("fp64", "fp32"):
        a = amm.create_from_mesh(P.tess, Q, P.gamma, precision=prec, mesh_motion="eulerian")
        b = amm.create_from_mesh(P.tess, Q, P.gamma, precision=prec, mesh_motion="eulerian")
        for _ in range(4):
            amm.amm_advance(a, 0.3, 1, use_graph=False)
        amm.amm_advance(b, 0.3, 2, use_graph=True)
        mid = amm.amm_get_state(b)
        c = amm.create_from_mesh(P.tess, Q, P.gamma, precision=prec, mesh_motion="eulerian")
        amm.amm_set_state(c, mid)
        amm.amm_advance(c, 0.3, 2, use_graph=True)
        amm.amm_advance(b, 0.3, 2, use_graph=False)
        qa, qb, qc = amm.amm_get_state(a), amm.amm_get_state(b), amm.amm_get_state(c)
        assert np.array_equal(qa, qb), prec
        assert np.array_equal(qa, qc), prec


def test_advance_matches_host_driven_steps(amm):
    """amm_advance (device-side time step) equals amm_timestep + amm_step."""
    P = ics.sod_2d(32, 16, seed=1)
    Q = P.conserved()
    a = amm.create_from_mesh(P.tess, Q, P.gamma, precision="fp64", mesh_motion="eulerian")
    b = amm.create_from_mesh(P.tess, Q, P.gamma, precision="fp64", mesh_motion="eulerian")
    for _ in range(3):
        dt = amm.amm_timestep(a, 0.3)[0]
        amm.amm_step(a, dt)
    amm.amm_advance(b, 0.3, 3, use_graph=True)
    assert np.array_equal(amm.amm_get_state(a), amm.amm_get_state(b))
    assert amm.amm_get_dt(b)[0] == dt


def test_multistep_eulerian_against_oracle(amm):
    """Twenty Eulerian steps on a fixed tessellation (CFL 0.3), FP64 and FP32."""
    P = ics.lognormal_3d(16, seed=3, sigma=0.5, mach=1.5)
    M = O.Mesh(P.tess)
    geom = O.geometry(M)
    Q = P.conserved()
    Qo = Q.copy()
    dts = []
    for _ in range(20):
        Qo, dt, cnt, rc = O.step(M, Qo, P.gamma, "eulerian", cfl=0.3, geom=geom)
        assert rc == 0 and cnt[3] == 0
        dts.append(dt)
    W = O.primitives(M, Q, geom[0], P.gamma)
    fl = floor_of(Q, 3, P.gamma, W)
    for prec, tol in (("fp64", 1e-10), ("fp32", 5e-4)):
        ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision=prec, mesh_motion="eulerian")
        for dt in dts:
            amm.amm_step(ctx, dt)
        emax, e999 = errs(amm.amm_get_state(ctx), Qo, fl)
        assert emax < tol, (prec, emax, e999)


def test_nonpositive_pressure_is_reported(amm):
    """An under-resolved log-normal Mach-3 field drives some cells to P <= 0
    within a few Eulerian steps (the oracle shows the same); the library
    reports AMM_ERR_NUMERIC with the count instead of flooring or crashing."""
    P = ics.lognormal_3d(12, seed=3, sigma=1.0, mach=3.0)
    M = O.Mesh(P.tess)
    geom = O.geometry(M)
    Qo = P.conserved()
    for _ in range(4):
        Qo, dt, cnt, rc = O.step(M, Qo, P.gamma, "eulerian", cfl=0.3, geom=geom)
    Wo = O.primitives(M, Qo, geom[0], P.gamma)
    assert (Wo[:, 4] <= 0).sum() > 0
    ctx = amm.create_from_mesh(P.tess, P.conserved(), P.gamma, precision="fp64", mesh_motion="eulerian")
    amm.amm_advance(ctx, 0.3, 4, use_graph=False)
    with pytest.raises(amm.AmmError) as e:
        amm.amm_sync(ctx)
    assert e.value.code == amm.AMM_ERR_NUMERIC
    assert amm.amm_get_stats(ctx)["nonpositive_cells"] > 0


def test_drift_moves_generators(amm):
    P = ics.turbulent_3d(8, seed=2)
    Q = P.conserved()
    ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision="fp64", mesh_motion="lagrangian")
    dt = 1e-3
    amm.amm_drift(ctx, dt)
    g = amm.amm_get_generators(ctx)
    ref = O.drift(O.Mesh(P.tess), Q[:, 1:4] / Q[:, :1], dt)
    d = np.abs(g - ref)
    d = np.minimum(d, 1.0 - d)
    assert d.max() < 1e-15


def test_set_state_rejects_nonpositive_pressure(amm):
    P = ics.turbulent_3d(6, seed=1)
    Q = P.conserved()
    ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision="fp64")
    Qb = Q.copy()
    Qb[3, 4] = 0.0          # E = 0 -> P < 0
    with pytest.raises(amm.AmmError) as e:
        amm.amm_set_state(ctx, Qb)
    assert e.value.code == amm.AMM_ERR_NONPOSITIVE_STATE


def test_open_cell_rejected(amm):
    """A face removed from a valid tessellation leaves two cells open."""
    P = ics.turbulent_3d(6, seed=1)
    T = P.tess
    keep = np.ones(T.n_faces, bool)
    keep[10] = False
    with pytest.raises(amm.AmmError) as e:
        amm.amm_create(3, T.points, T.cells[keep], T.shift[keep], T.area[keep], T.centroid[keep], T.box,
                       P.conserved(), P.gamma)
    assert e.value.code == amm.AMM_ERR_OPEN_CELL


def test_full_size_config2(amm):
    """64^3 Lagrangian, the benchmark workload, whole state against the oracle."""
    P = ics.turbulent_3d(64, seed=2)
    M = O.Mesh(P.tess)
    Q = P.conserved()
    geom = O.geometry(M)
    W = O.primitives(M, Q, geom[0], P.gamma)
    ref, dt, cnt, rc = O.step(M, Q, P.gamma, "lagrangian", cfl=0.3, geom=geom)
    fl = floor_of(Q, 3, P.gamma, W)
    for prec in ("fp64", "fp32"):
        ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision=prec)
        dtg = amm.amm_timestep(ctx, 0.3)[0]
        assert abs(dtg - dt) / dt < 1e-6
        amm.amm_advance(ctx, 0.3, 1, use_graph=True)
        out = amm.amm_get_state(ctx)
        emax, e999 = errs(out, ref, fl)
        assert emax < TOL[prec], (prec, emax, e999)


def test_fixed_point_accumulation_matches_fp64_accumulation(amm):
    """The FP32 form's exact int64 flux sums and the FP64 floating-point sums
    of the same FP32 fluxes differ only by FP64 rounding of the sums."""
    P = ics.lognormal_3d(16, seed=11)
    Q = P.conserved()
    W = O.primitives(O.Mesh(P.tess), Q, P.tess.volume, P.gamma)
    fl = floor_of(Q, 3, P.gamma, W)
    out = []
    for acc64 in (False, True):
        ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision="fp32", fp64_accumulate=acc64)
        amm.amm_step(ctx, 2e-3)
        out.append(amm.amm_get_state(ctx))
    emax, _ = errs(out[0], out[1], fl)
    assert emax < 1e-13, emax


@pytest.mark.parametrize("tuning", [(1, 1, 128), (2, 8, 256), (8, 2, 128), (4, 4, 256)])
def test_launch_shapes_keep_parity(amm, tuning):
    """Every launch shape the autotuner may pick gives oracle parity."""
    P = ics.turbulent_3d(16, seed=2)
    M = O.Mesh(P.tess)
    Q = P.conserved()
    ref, dt, _, _ = O.step(M, Q, P.gamma, "lagrangian", cfl=0.3)
    W = O.primitives(M, Q, P.tess.volume, P.gamma)
    fl = floor_of(Q, 3, P.gamma, W)
    for prec in ("fp64", "fp32"):
        ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision=prec)
        amm.amm_set_tuning(ctx, *tuning)
        amm.amm_step(ctx, dt)
        emax, _ = errs(amm.amm_get_state(ctx), ref, fl)
        assert emax < TOL[prec], (prec, tuning, emax)


def test_autotune_restores_state_and_keeps_parity(amm):
    P = ics.turbulent_3d(16, seed=3)
    M = O.Mesh(P.tess)
    Q = P.conserved()
    ref, dt, _, _ = O.step(M, Q, P.gamma, "lagrangian", cfl=0.3)
    W = O.primitives(M, Q, P.tess.volume, P.gamma)
    fl = floor_of(Q, 3, P.gamma, W)
    ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision="fp32")
    t = amm.amm_autotune(ctx, 0.3, reps=2)
    assert t["grad_lanes"] in (1, 2, 4, 8) and t["flux_block"] in (128, 256) and t["step_ms"] > 0
    assert np.array_equal(amm.amm_get_state(ctx), Q)
    assert amm.amm_get_stats(ctx)["steps"] == 0
    amm.amm_step(ctx, dt)
    emax, _ = errs(amm.amm_get_state(ctx), ref, fl)
    assert emax < TOL["fp32"]


def test_create_from_device_arrays(amm):
    """amm_create_device copies the same inputs from device memory: the
    context steps bit-identically to one made from host arrays."""
    import torch
    P = ics.turbulent_3d(12, seed=6)
    T = P.tess
    Q = P.conserved()
    outs = []
    for dev in (False, True):
        opt = amm.amm_default_options("fp64", "lagrangian")
        if dev:
            t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
                 (T.points, T.cells.astype(np.int32), T.shift.astype(np.int8), T.area, T.centroid, Q)]
            ctx = amm.amm_create_device(3, T.n_cells, T.n_faces, *[x.data_ptr() for x in t[:5]], T.box,
                                        t[5].data_ptr(), P.gamma, opt)
        else:
            ctx = amm.create_from_mesh(T, Q, P.gamma, precision="fp64")
        amm.amm_advance(ctx, 0.3, 2, use_graph=False)
        outs.append(amm.amm_get_state(ctx))
    assert np.array_equal(outs[0], outs[1])
