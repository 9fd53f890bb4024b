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
