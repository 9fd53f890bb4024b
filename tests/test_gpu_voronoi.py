"""The GPU Voronoi builder (amm_tess_build, Sec. 2) against the host
tessellator, which is pinned against qhull (tests/test_harness.py): the same
faces (cell pairs and periodic images), areas and centroids to 1e-9 of the
mean face scale, volumes and centres of mass; every face found from both
sides; volumes summing to the box; and a hydro step on the GPU-built mesh
equal to the step on the host-built one."""
import numpy as np
import pytest

from harness import ics
from harness.tess import tessellate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_4107_gb300 import amm as A
    return A


def gpu_tess(amm, pts, box):
    import torch
    g = torch.from_numpy(np.ascontiguousarray(pts, np.float64)).to("cuda")
    t = amm.amm_tess_build(pts.shape[1], len(pts), g.data_ptr(), box)
    out = t.to_host()
    return t, out


def face_key_map(cells, shift, area, cen):
    """(i, j, shift) -> (area, centroid), keyed from the smaller index."""
    m = {}
    for k in range(len(area)):
        m[(int(cells[k, 0]), int(cells[k, 1])) + tuple(int(x) for x in shift[k])] = (area[k], cen[k])
    return m


CASES = [(3, 12, 0.25, 1), (3, 16, 0.45, 2), (2, 40, 0.3, 3), (2, 24, 0.0, 4), (3, 10, 0.0, 5)]


@pytest.mark.parametrize("dim,n,jitter,seed", CASES)
def test_matches_host_tessellator(amm, dim, n, jitter, seed):
    rng = np.random.default_rng(seed)
    box = np.array([1.0, 0.8, 1.2][:dim])
    pts = ics.jittered_lattice((n,) * dim, box, jitter, rng)
    H = tessellate(pts, box)
    t, (cells, shift, area, cen, vol, com) = gpu_tess(amm, pts, box)
    asym, maxrel = t.check()
    assert asym == 0 and maxrel < 1e-9
    mh = face_key_map(H.cells, H.shift, H.area, H.centroid)
    mg = face_key_map(cells, shift, area, cen)
    assert set(mh) == set(mg), (len(set(mh) ^ set(mg)), len(mh))
    scale = np.mean(H.area)
    for k, (a, c) in mh.items():
        ag, cg = mg[k]
        assert abs(ag - a) < 1e-9 * scale, (k, a, ag)
        assert np.abs(cg - c).max() < 1e-9 * scale ** (1.0 / (dim - 1)), (k, c, cg)
    np.testing.assert_allclose(vol, H.volume, rtol=1e-9)
    np.testing.assert_allclose(com, H.com, atol=1e-9 * np.prod(box) ** (1 / dim))
    assert abs(vol.sum() - np.prod(box)) < 1e-10 * np.prod(box)


def test_random_points_and_step_on_gpu_mesh(amm):
    """Uniform random generators (no lattice): the GPU mesh equals the host
    mesh, and one FP64 step on either gives the same state."""
    rng = np.random.default_rng(9)
    box = np.ones(3)
    pts = rng.uniform(0.0, 1.0, (3000, 3))
    H = tessellate(pts, box)
    t, (cells, shift, area, cen, vol, com) = gpu_tess(amm, pts, box)
    assert set(face_key_map(H.cells, H.shift, H.area, H.centroid)) == set(face_key_map(cells, shift, area, cen))
    gam = 5.0 / 3.0
    rho = 1.0 + 0.3 * rng.standard_normal(len(pts)) ** 2
    vel = 0.5 * rng.standard_normal((len(pts), 3))
    P = 1.0 + 0.2 * rng.uniform(size=len(pts))
    Q = ics.conserved_from_primitives(rho, vel, P, H.volume, gam)
    ctx_h = amm.create_from_mesh(H, Q, gam, precision="fp64", mesh_motion="lagrangian")
    dt = float(amm.amm_timestep(ctx_h, 0.3)[0])
    amm.amm_step(ctx_h, dt)
    Qh = amm.amm_get_state(ctx_h)
    opt = amm.amm_default_options("fp64", "lagrangian")
    ctx_g = amm.amm_create(3, pts, cells, shift, area, cen, box, Q, gam, opt)
    amm.amm_step(ctx_g, dt)
    Qg = amm.amm_get_state(ctx_g)
    scale = np.abs(Q).max(axis=0)
    assert np.max(np.abs(Qg - Qh) / scale) < 1e-10


def test_full_size_turbulent_box(amm):
    """The 64^3 jittered lattice of the turbulent workload: the GPU builder's
    face count, total area and volumes against the host tessellator."""
    P = ics.turbulent_3d(64, seed=2)
    t, (cells, shift, area, cen, vol, com) = gpu_tess(amm, P.tess.points, P.tess.box)
    assert t.n_faces == P.tess.n_faces
    assert t.check()[0] == 0
    np.testing.assert_allclose(np.sort(area), np.sort(P.tess.area), rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(vol, P.tess.volume, rtol=1e-9)


@pytest.mark.parametrize("dim,n,jitter,seed", [(3, 5, 0.3, 21), (2, 10, 0.35, 22)])
def test_matches_definitional_oracle(amm, dim, n, jitter, seed):
    """Against oracle/voronoi.py (every periodic image, half-space
    intersection by a library primitive): the same listed faces, areas and
    centroids to 1e-10 of the spacing, volumes to 1e-10."""
    from oracle import voronoi as OV
    rng = np.random.default_rng(seed)
    box = np.array([1.0, 1.2, 0.9][:dim])
    pts = ics.jittered_lattice((n,) * dim, box, jitter, rng)
    faces, vol_o = OV.tessellate(pts, box)
    ref = OV.face_list(faces, dim)
    t, (cells, shift, area, cen, vol, com) = gpu_tess(amm, pts, box)
    got = {(int(cells[k, 0]), int(cells[k, 1])) + tuple(int(v) for v in shift[k]): (area[k], cen[k])
           for k in range(len(area))}
    assert set(got) == set(ref)
    h = (np.prod(box) / len(pts)) ** (1.0 / dim)
    for k, (a, c) in ref.items():
        assert abs(got[k][0] - a) < 1e-10 * h ** (dim - 1)
        assert np.abs(got[k][1] - c).max() < 1e-10 * h
    np.testing.assert_allclose(vol, vol_o, rtol=1e-10)
