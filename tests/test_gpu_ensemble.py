"""Batched ensemble: independent boxes of uneven size in one context, each
with its own Courant step, advanced by one persistent launch per step."""
import numpy as np
import pytest

from harness import ics
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


@pytest.fixture(scope="module")
def ens():
    sizes = (5, 9, 6, 11, 7, 8)
    machs = (0.5, 2.0, 1.0, 2.0, 1.2, 1.5)
    return ics.concat([ics.turbulent_3d(n, seed=20 + k, mach=m) for k, (n, m) in enumerate(zip(sizes, machs))])


def create(amm, E, prec, **kw):
    opt = amm.amm_default_options(prec, "lagrangian", **kw)
    return amm.amm_create(3, E.points, E.cells, E.shift, E.area, E.centroid, E.box, E.Q, E.gamma, opt,
                          box_cells=E.box_cells, box_faces=E.box_faces)


def oracle_boxes(E, cfl=0.3):
    out, dts = [], []
    for P in E.problems:
        M = O.Mesh(P.tess)
        Qn, dt, _, rc = O.step(M, P.conserved(), P.gamma, "lagrangian", cfl=cfl)
        assert rc == 0
        out.append(Qn)
        dts.append(dt)
    return np.concatenate(out), np.array(dts)


def floor_box(P):
    Q = P.conserved()
    W = O.primitives(O.Mesh(P.tess), Q, P.tess.volume, P.gamma)
    fl = np.sqrt(np.mean(Q * Q, axis=0))
    c = np.sqrt(P.gamma * W[:, 4] / W[:, 0])
    fl[1:4] = np.sqrt(np.mean((Q[:, 0] * c) ** 2))
    return fl


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_per_box_timestep_and_step(amm, ens, prec):
    ref, dts = oracle_boxes(ens)
    ctx = create(amm, ens, prec)
    dt = amm.amm_timestep(ctx, 0.3)
    assert np.max(np.abs(dt - dts) / dts) < (1e-14 if prec == "fp64" else 1e-6)
    assert len(set(np.round(dts, 12))) == len(dts)          # the boxes really differ
    amm.amm_step_boxes(ctx, dts)
    out = amm.amm_get_state(ctx)
    for b, P in enumerate(ens.problems):
        s = slice(ens.box_cells[b], ens.box_cells[b + 1])
        e = np.max(np.abs(out[s] - ref[s]) / np.maximum(np.abs(ref[s]), floor_box(P)))
        assert e < TOL[prec], (prec, b, e)
    tot = amm.amm_get_totals(ctx)
    for b in range(len(ens.problems)):
        s = slice(ens.box_cells[b], ens.box_cells[b + 1])
        assert np.allclose(tot[b], out[s].sum(0), rtol=1e-12, atol=1e-15 * np.abs(out[s]).sum())
    assert np.allclose(amm.amm_get_dt(ctx), dts, rtol=0, atol=0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_persistent_launch_matches_kernel_sequence(amm, ens, prec):
    """One cooperative launch per step (grid barriers between phases) gives
    bit-identical results to the per-phase launches of the same shapes, with
    and without graph capture, and the device-side per-box Courant step."""
    ref, dts = oracle_boxes(ens)
    outs = []
    for persistent, graph in ((0, False), (1, False), (1, True)):
        ctx = create(amm, ens, prec)
        amm.amm_set_tuning(ctx, 4, 1, 256, persistent)
        amm.amm_advance(ctx, 0.3, 3, use_graph=graph)
        amm.amm_sync(ctx)
        outs.append(amm.amm_get_state(ctx))
        d = amm.amm_get_dt(ctx)
        assert np.all(d > 0) and len(set(d.tolist())) == len(d)
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])
    # first step agrees with the oracle per box (device dt = oracle dt to rounding)
    ctx = create(amm, ens, prec)
    amm.amm_set_tuning(ctx, 4, 1, 256, 1)
    amm.amm_advance(ctx, 0.3, 1, use_graph=True)
    out = amm.amm_get_state(ctx)
    for b, P in enumerate(ens.problems):
        s = slice(ens.box_cells[b], ens.box_cells[b + 1])
        e = np.max(np.abs(out[s] - ref[s]) / np.maximum(np.abs(ref[s]), floor_box(P)))
        assert e < TOL[prec], (prec, b, e)


def test_autotune_picks_a_step_mode(amm, ens):
    ctx = create(amm, ens, "fp32")
    t = amm.amm_autotune(ctx, 0.3, reps=2)
    assert t["persistent"] in (0, 1)
    amm.amm_advance(ctx, 0.3, 2, use_graph=True)
    amm.amm_sync(ctx)


def test_failed_box_is_flagged_and_others_complete(amm):
    """A coarse Mach-4 box develops a non-positive pressure within a step (the
    oracle agrees); it is flagged in its own status word while the other
    boxes of the ensemble still match the oracle."""
    probs = [ics.turbulent_3d(6, seed=30, mach=1.0), ics.turbulent_3d(7, seed=24, mach=4.0),
             ics.turbulent_3d(8, seed=32, mach=1.5)]
    E = ics.concat(probs)
    ref, dts = oracle_boxes(E)
    W1 = O.primitives(O.Mesh(probs[1].tess), ref[E.box_cells[1]:E.box_cells[2]], probs[1].tess.volume, E.gamma)
    assert (W1[:, 4] <= 0).sum() > 0
    ctx = create(amm, E, "fp64")
    amm.amm_step_boxes(ctx, dts)
    with pytest.raises(amm.AmmError):
        amm.amm_sync(ctx)
    st = amm.amm_get_box_status(ctx)
    assert st[1] != 0 and st[0] == 0 and st[2] == 0
    out = amm.amm_get_state_device if False else None
    Q = np.empty_like(ref)
    lib = amm.lib()
    assert lib.amm_get_state(ctx.handle, Q.ctypes.data) == amm.AMM_ERR_NUMERIC   # data still returned
    for b in (0, 2):
        s = slice(E.box_cells[b], E.box_cells[b + 1])
        e = np.max(np.abs(Q[s] - ref[s]) / np.maximum(np.abs(ref[s]), floor_box(probs[b])))
        assert e < 1e-12, (b, e)
