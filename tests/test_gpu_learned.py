"""The FP32 learned form: the proposal network fused into the flux kernel.

Newton still converges to the same tolerance, so the learned form must keep
the FP32 parity bar against the oracle whatever the weights; a network
trained on harvested face states must lower the Newton iteration count on a
held-out run (what the proposal gains over the standard guess)."""
import numpy as np
import pytest

from harness import ics
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_4107_gb300 import amm, learned
    return torch, amm, learned


@pytest.fixture(scope="module")
def trained(env):
    torch, amm, learned = env
    net, stats = learned.train_proposal(ics, torch, small=True, epochs=3)
    return net, stats


def floor_of(Q, W, gamma):
    fl = np.sqrt(np.mean(Q * Q, axis=0))
    c = np.sqrt(gamma * W[:, 4] / W[:, 0])
    fl[1:4] = np.sqrt(np.mean((Q[:, 0] * c) ** 2))
    return fl


def test_harvest_records_every_face(env):
    torch, amm, learned = env
    P = ics.turbulent_3d(10, seed=3)
    st = learned.harvest(P.tess, P.conserved(), P.gamma, "lagrangian", 2, torch=torch)
    assert st.shape == (2 * P.n_faces, 6)
    s = st.cpu().numpy()
    assert np.all(np.isfinite(s)) and np.all(s[:, [0, 2, 3, 5]] > 0)


def test_learned_form_keeps_parity(env, trained):
    torch, amm, learned = env
    net, _ = trained
    for P, mode in ((ics.turbulent_3d(16, seed=2), "lagrangian"), (ics.sod_2d(32, 16, seed=1), "eulerian"),
                    (ics.lognormal_3d(16, seed=3), "lagrangian")):
        M = O.Mesh(P.tess)
        Q = P.conserved()
        ref, dt, _, rc = O.step(M, Q, P.gamma, mode, cfl=0.3)
        W = O.primitives(M, Q, P.tess.volume, P.gamma)
        if P.dim == 2:
            W = np.column_stack([W[:, :3], np.zeros(len(W)), W[:, 3]])
        ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision="fp32_learned", mesh_motion=mode)
        with pytest.raises(amm.AmmError):
            amm.amm_step(ctx, dt)           # no weights yet
        amm.amm_mlp_attach(ctx, net)
        amm.amm_step(ctx, dt)
        out = amm.amm_get_state(ctx)
        fl = floor_of(np.column_stack([Q[:, :P.dim + 1], np.zeros((len(Q), 3 - P.dim)), Q[:, -1:]]) if P.dim == 2
                      else Q, W, P.gamma)
        if P.dim == 2:
            fl = np.concatenate([fl[:3], fl[4:]])
        e = np.max(np.abs(out - ref) / np.maximum(np.abs(ref), fl))
        assert e < 2e-5, (P.name, e)
        st = amm.amm_get_stats(ctx)
        assert st["newton_fail"] == 0 and st["faces"] == P.n_faces


def test_trained_proposal_saves_newton_iterations(env, trained):
    """Held-out run (a seed the network never saw): mean Newton iterations
    per face, standard guess vs learned proposal, same tolerance.  The
    proposal stands in for the two-shock estimate (the approximate branch of
    the standard guess)."""
    torch, amm, learned = env
    net, stats = trained
    assert stats["val_mse"] < 0.5 * stats.get("train_mse", 1.0) + 1e-2
    P = ics.turbulent_3d(24, seed=9)
    Q = P.conserved()
    iters = {}
    for prec in ("fp32", "fp32_learned"):
        ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision=prec)
        if prec == "fp32_learned":
            amm.amm_mlp_attach(ctx, net)
        amm.amm_advance(ctx, 0.3, 1, use_graph=False)
        s = amm.amm_get_stats(ctx)
        iters[prec] = s["newton_iters"] / s["faces"]
    assert iters["fp32_learned"] < iters["fp32"], iters


def test_persistent_learned_ensemble_matches_kernel_sequence(env, trained):
    """The learned form of the batched ensemble: one cooperative launch per
    step (two tensor-core MMA groups per CTA) runs the same per-face
    arithmetic as the per-phase launches; the two kernels are compiled under
    different register budgets, so the compiler may contract a multiply-add
    differently and the states agree to FP32 rounding (bit for bit between
    graph replay and direct launches of the same mode); each box's first
    step keeps the FP32 parity bar against the oracle."""
    torch, amm, learned = env
    net, _ = trained
    sizes, machs = (5, 9, 6, 11, 7, 8), (0.5, 2.0, 1.0, 2.0, 1.2, 1.5)
    E = ics.concat([ics.turbulent_3d(n, seed=20 + k, mach=m) for k, (n, m) in enumerate(zip(sizes, machs))])

    def create():
        opt = amm.amm_default_options("fp32_learned", "lagrangian")
        ctx = amm.amm_create(3, E.points, E.cells, E.shift, E.area, E.centroid, E.box, E.Q, E.gamma, opt,
                             box_cells=E.box_cells, box_faces=E.box_faces)
        amm.amm_mlp_attach(ctx, net)
        return ctx

    outs, stats = [], []
    for persistent, graph in ((0, False), (1, False), (1, True)):
        ctx = create()
        amm.amm_set_tuning(ctx, 4, 1, 256, persistent)
        amm.amm_advance(ctx, 0.3, 3, use_graph=graph)
        amm.amm_sync(ctx)
        outs.append(amm.amm_get_state(ctx))
        stats.append(amm.amm_get_stats(ctx))
    assert np.array_equal(outs[1], outs[2])
    scale = np.abs(outs[0]).max(axis=0)
    assert np.max(np.abs(outs[0] - outs[1]) / scale) < 1e-6
    assert abs(stats[0]["newton_iters"] - stats[1]["newton_iters"]) <= 1e-3 * stats[0]["newton_iters"]
    assert stats[1]["faces"] == 3 * E.n_faces
    ctx = create()
    amm.amm_set_tuning(ctx, 4, 1, 256, 1)
    amm.amm_advance(ctx, 0.3, 1, use_graph=True)
    out = amm.amm_get_state(ctx)
    for b, P in enumerate(E.problems):
        M = O.Mesh(P.tess)
        Q = P.conserved()
        ref, _, _, rc = O.step(M, Q, P.gamma, "lagrangian", cfl=0.3)
        assert rc == 0
        W = O.primitives(M, Q, P.tess.volume, P.gamma)
        s = slice(E.box_cells[b], E.box_cells[b + 1])
        e = np.max(np.abs(out[s] - ref) / np.maximum(np.abs(ref), floor_of(Q, W, P.gamma)))
        assert e < 2e-5, (b, e)
