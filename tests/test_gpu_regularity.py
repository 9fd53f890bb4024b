"""The mesh-regularity correction of Sec. 4.1 on the GPU (amm_options.
regularize) against the oracle: the same step as the oracle's with the
corrected generator velocities given explicitly."""
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


def floor_of(Q, W, gamma):
    fl = np.sqrt(np.mean(Q * Q, axis=0))
    c = np.sqrt(gamma * W[:, 4] / W[:, 0])
    fl[1:4] = np.sqrt(np.mean((Q[:, 0] * c) ** 2))
    return fl


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("mode", ["lagrangian", "explicit"])
def test_step_and_drift_match_oracle(amm, prec, mode):
    P = ics.turbulent_3d(12, jitter=0.45, seed=8)
    M = O.Mesh(P.tess)
    V, s = O.geometry(M)
    Q = P.conserved()
    W = O.primitives(M, Q, V, P.gamma)
    base = W[:, 1:4] if mode == "lagrangian" else 0.5 * W[:, 1:4] + 0.2
    wc = O.shape_correction(M, W, V, s, base, P.gamma, eta=0.25, chi=1.0)
    assert (np.linalg.norm(wc - base, axis=1) > 0).mean() > 0.05      # the correction is active
    ref, dt, cnt, rc = O.step(M, Q, P.gamma, "explicit", wmesh=wc, cfl=0.3)
    assert rc == 0
    ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision=prec, mesh_motion=mode, regularize=True)
    if mode == "explicit":
        amm.amm_set_mesh_velocity(ctx, base)
    dtg = amm.amm_timestep(ctx, 0.3)[0]
    assert abs(dtg - dt) / dt < (1e-13 if prec == "fp64" else 1e-6)
    amm.amm_step(ctx, dt)
    out = amm.amm_get_state(ctx)
    e = np.max(np.abs(out - ref) / np.maximum(np.abs(ref), floor_of(Q, W, P.gamma)))
    assert e < TOL[prec], (prec, mode, e)
    # the generators move with the corrected velocities
    gen0 = amm.amm_get_generators(ctx)
    amm.amm_drift(ctx, dt)
    moved = amm.amm_get_generators(ctx) - gen0
    moved -= np.round(moved)                                          # periodic wrap of the unit box
    np.testing.assert_allclose(moved, wc * dt, atol=1e-12 if prec == "fp64" else 1e-5 * np.abs(wc).max() * dt)


def test_eulerian_mesh_rejects_the_correction(amm):
    P = ics.turbulent_3d(6, seed=2)
    with pytest.raises(amm.AmmError):
        amm.create_from_mesh(P.tess, P.conserved(), P.gamma, precision="fp64", mesh_motion="eulerian",
                             regularize=True)
