"""The moving-mesh cycle on the device (amm_retessellate: a GPU Voronoi mesh
of the drifted generators, cells keeping their conserved quantities) against
the host cycle and the oracle: the rebuilt mesh has the host tessellator's
faces and areas; re-tessellating does not change the state; steps on the
rebuilt mesh match the host-driven cycle (FP64 1e-10) and the oracle's."""
import numpy as np
import pytest

from harness import ics, moving
from harness.tess import tessellate
from oracle import oracle as O

pytestmark = pytest.mark.gpu


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


def pairs_areas(cells, area, shift=None):
    m = {}
    for k in range(len(area)):
        a, b = int(cells[k, 0]), int(cells[k, 1])
        key = (min(a, b), max(a, b))
        m.setdefault(key, []).append(area[k])
    return {k: sorted(v) for k, v in m.items()}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rebuilt_mesh_matches_host_tessellation(amm, prec):
    P = ics.turbulent_3d(14, jitter=0.3, seed=6)
    ctx = amm.create_from_mesh(P.tess, P.conserved(), P.gamma, precision=prec, mesh_motion="lagrangian")
    dt = float(amm.amm_timestep(ctx, 0.3)[0])
    amm.amm_drift(ctx, dt)
    amm.amm_step(ctx, dt)
    Q_before = amm.amm_get_state(ctx)
    amm.amm_retessellate(ctx)
    assert np.array_equal(amm.amm_get_state(ctx), Q_before)
    H = tessellate(amm.amm_get_generators(ctx), P.tess.box)
    cells, area = amm.amm_get_faces(ctx)
    mh, mg = pairs_areas(H.cells, H.area), pairs_areas(cells, area)
    assert set(mh) == set(mg)
    tol = 1e-9 if prec == "fp64" else 1e-6
    for k in mh:
        np.testing.assert_allclose(mg[k], mh[k], rtol=tol, atol=tol * np.mean(H.area))
    V, s = amm.amm_get_geometry(ctx)
    np.testing.assert_allclose(V, H.volume, rtol=1e-9)
    amm.amm_destroy(ctx)


def test_device_cycle_matches_host_cycle_and_oracle(amm):
    P = ics.gresho_2d(24, jitter=0.1, seed=3, v_vortex=1.0)
    gd, Qd, td, kd = moving.run_on_device(amm, P, "fp64", "lagrangian", t_end=0.08)
    Th, Qh, th, kh = moving.run(P, moving.LibraryBackend(amm, "fp64", "lagrangian"), t_end=0.08)
    To, Qo, to, ko = moving.run(P, moving.OracleBackend(O, "lagrangian"), t_end=0.08)
    assert kd == kh == ko and abs(td - th) < 1e-14
    scale = np.abs(P.conserved()).max(axis=0)
    assert np.max(np.abs(Qd - Qh) / scale) < 1e-10
    assert np.max(np.abs(Qd - Qo) / scale) < 1e-9
    d = gd - Th.points
    d -= np.round(d)
    assert np.abs(d).max() < 1e-12
    np.testing.assert_allclose(Qd.sum(0), P.conserved().sum(0), rtol=1e-12, atol=1e-13)


def test_device_cycle_3d_regularised(amm):
    P = ics.turbulent_3d(12, jitter=0.3, seed=7)
    gd, Qd, td, kd = moving.run_on_device(amm, P, "fp64", "lagrangian", steps=5, regularize=True)
    Th, Qh, th, kh = moving.run(P, moving.LibraryBackend(amm, "fp64", "lagrangian", regularize=True), steps=5)
    scale = np.abs(P.conserved()).max(axis=0)
    assert np.max(np.abs(Qd - Qh) / scale) < 1e-10


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_many_device_steps_keep_the_host_mesh(amm, prec):
    """Twelve Lagrangian steps of a Mach-2 box with a new GPU mesh after each
    (the face count changes every step, the face buffers are reused within
    their capacity): the final mesh equals the host tessellation of the final
    generators, and mass, momentum and energy are conserved."""
    P = ics.turbulent_3d(16, jitter=0.2, seed=11)
    Q0 = P.conserved()
    ctx = amm.create_from_mesh(P.tess, Q0, P.gamma, precision=prec, mesh_motion="lagrangian")
    counts = []
    for _ in range(12):
        dt = float(amm.amm_timestep(ctx, 0.3)[0])
        amm.amm_drift(ctx, dt)
        amm.amm_step(ctx, dt)
        amm.amm_retessellate(ctx)
        counts.append(int(amm.amm_get_faces(ctx)[0].shape[0]))
    assert len(set(counts)) > 1
    H = tessellate(amm.amm_get_generators(ctx), P.tess.box)
    cells, area = amm.amm_get_faces(ctx)
    mh, mg = pairs_areas(H.cells, H.area), pairs_areas(cells, area)
    assert set(mh) == set(mg)
    Q = amm.amm_get_state(ctx)
    tot0, tot = Q0.sum(0), Q.sum(0)
    np.testing.assert_allclose(tot[[0, 4]], tot0[[0, 4]], rtol=1e-12)
    assert np.abs(tot[1:4] - tot0[1:4]).max() < 1e-12 * np.abs(Q0[:, 1:4]).sum()
    amm.amm_destroy(ctx)
