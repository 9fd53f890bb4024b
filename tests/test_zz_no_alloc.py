"""The allocation-free Courant step against the context-based one.

amm_timestep_noalloc serves callers that cannot allocate device memory (their
device memory belongs to another allocator, or they must not risk the device
synchronisation cudaMalloc/cudaFree can cause).  It must agree with
amm_timestep on the same state.  This file sorts last so that a run stopping
at the first failure has already run every other test; it also passes alone
in a fresh process.
"""
import numpy as np
import pytest

from harness import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_4107_gb300 import amm
    return torch, amm


def _device_inputs(torch, amm, ctx):
    W = amm.amm_get_primitives(ctx)
    V, _ = amm.amm_get_geometry(ctx)
    return torch.from_numpy(W).cuda(), torch.from_numpy(V).cuda()


@pytest.mark.parametrize("motion", ["eulerian", "explicit"])
def test_noalloc_timestep_matches_context_timestep_twice(env, motion):
    torch, amm = env
    results = []
    for seed, cfl in ((2, 0.3), (5, 0.45)):          # two calls in a row, different inputs
        P = ics.turbulent_3d(12, seed=seed, mach=1.5)
        ctx = amm.create_from_mesh(P.tess, P.conserved(), P.gamma, precision="fp64", mesh_motion=motion)
        w = None
        if motion == "explicit":
            w = 0.5 * P.vel
            amm.amm_set_mesh_velocity(ctx, w)
        ref = amm.amm_timestep(ctx, cfl)[0]
        Wd, Vd = _device_inputs(torch, amm, ctx)
        wd = torch.from_numpy(np.ascontiguousarray(w)).cuda() if w is not None else None
        dt = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        s = torch.cuda.current_stream()
        amm.amm_timestep_noalloc(3, P.n_cells, Wd.data_ptr(), Vd.data_ptr(), wd.data_ptr() if wd is not None else 0,
                                 P.gamma, cfl, dt.data_ptr(), s.cuda_stream)
        got = float(dt.cpu().item())
        assert abs(got - ref) <= 1e-13 * ref, (got, ref)
        results.append(got)
    assert results[0] != results[1]


@pytest.mark.parametrize("motion", ["eulerian", "explicit"])
def test_noalloc_timestep_2d_matches_context_timestep_twice(env, motion):
    """The 2D branch (radius sqrt(V / pi)) on the config-1 mesh: 128 x 64
    jittered generators in [0,2] x [0,1], the Sod states with a velocity
    field added so that |v - w| matters; two calls in a row."""
    torch, amm = env
    P = ics.sod_2d(128, 64, seed=1)
    x, y = P.tess.points[:, 0], P.tess.points[:, 1]
    results = []
    for k, cfl in ((1, 0.3), (2, 0.45)):
        P.vel = np.stack([0.7 * k * np.sin(2 * np.pi * y), -0.4 * k * np.cos(np.pi * x)], axis=1)
        ctx = amm.create_from_mesh(P.tess, P.conserved(), P.gamma, precision="fp64", mesh_motion=motion)
        w = None
        if motion == "explicit":
            w = np.ascontiguousarray(0.5 * P.vel[:, ::-1])
            amm.amm_set_mesh_velocity(ctx, w)
        ref = amm.amm_timestep(ctx, cfl)[0]
        Wd, Vd = _device_inputs(torch, amm, ctx)
        wd = torch.from_numpy(w).cuda() if w is not None else None
        dt = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        s = torch.cuda.current_stream()
        amm.amm_timestep_noalloc(2, P.n_cells, Wd.data_ptr(), Vd.data_ptr(), wd.data_ptr() if wd is not None else 0,
                                 P.gamma, cfl, dt.data_ptr(), s.cuda_stream)
        got = float(dt.cpu().item())
        assert abs(got - ref) <= 1e-13 * ref, (got, ref)
        results.append(got)
        amm.amm_destroy(ctx)
    assert results[0] != results[1]


def test_noalloc_rejects_oversize_and_bad_arguments(env):
    torch, amm = env
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    W = torch.ones((8, 5), dtype=torch.float64, device="cuda")
    V = torch.ones(8, dtype=torch.float64, device="cuda")
    with pytest.raises(amm.AmmError) as e:
        amm.amm_timestep_noalloc(3, 16384 * 4096 + 1, W.data_ptr(), V.data_ptr(), 0, 5 / 3, 0.3, dt.data_ptr())
    assert e.value.code == amm.AMM_ERR_INVALID_ARG
    with pytest.raises(amm.AmmError):
        amm.amm_timestep_noalloc(4, 8, W.data_ptr(), V.data_ptr(), 0, 5 / 3, 0.3, dt.data_ptr())
