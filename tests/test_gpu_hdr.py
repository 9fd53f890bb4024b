"""The FP32 forms on a field of high dynamic range: the point explosion of
Sec. 8.4 (energy 1 in one cell of a 32^3 box of cold gas, P0 = 1e-4) after
30 steps, where the blast's cells hold ~1e8 times the energy of the ambient
ones.  The parity norm of the other tests floors each error at an RMS over
the box, which the blast dominates; here every cell's error is measured
against that cell's own magnitude (mass and energy), or its own m c
(momentum, zero in the gas at rest).

The exact fixed-point flux sums quantise every face flux to a multiple of
2^(e + headroom - 188), with e the biased exponent of the box's largest
|A F| of the component and 2^headroom above every cell's face count; a
flux is truncated toward zero, so one cell's sum is off by less than
n_faces(i) quanta, i.e. by less than n_faces(i) 2^(headroom - 61)
max|A F| per unit time.  The test asserts that bound against the FP64
accumulation of the same FP32 fluxes, cell by cell, and each form against
the FP64 oracle on the cell's own scale."""
import numpy as np
import pytest

from harness import ics
from oracle import oracle as O

pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def amm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_4107_gb300 import amm as A
    return A


def own_scale(Q, gamma):
    """|Q| per cell and component, with m c for the momentum components"""
    m = Q[:, 0]
    P = (gamma - 1.0) * (Q[:, 4] - 0.5 * (Q[:, 1:4] ** 2).sum(1) / m)   # P V
    c = np.sqrt(gamma * P / m)                                          # sqrt(gamma P / rho)
    s = np.abs(Q).copy()
    s[:, 1:4] = np.maximum(s[:, 1:4], (m * c)[:, None])
    return s


@pytest.fixture(scope="module")
def blast(amm):
    P = ics.sedov(3, 32)
    ctx = amm.create_from_mesh(P.tess, P.conserved(), P.gamma, precision="fp32", mesh_motion="eulerian")
    amm.amm_advance(ctx, 0.3, 30, use_graph=False)
    Q = amm.amm_get_state(ctx)
    amm.amm_destroy(ctx)
    return P, Q


def test_blast_has_high_dynamic_range(blast):
    P, Q = blast
    assert Q[:, 4].max() / Q[:, 4].min() > 1e6
    assert np.all(Q[:, 0] > 0)


def test_each_cell_matches_the_oracle_on_its_own_scale(amm, blast):
    P, Q = blast
    ref, dt, _, rc = O.step(O.Mesh(P.tess), Q, P.gamma, "eulerian", cfl=0.3)
    assert rc == 0
    scale = own_scale(ref, P.gamma)
    for prec, acc64, tol in (("fp64", False, 1e-12), ("fp32", False, 2e-5), ("fp32", True, 2e-5)):
        ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision=prec, mesh_motion="eulerian", fp64_accumulate=acc64)
        amm.amm_step(ctx, dt)
        out = amm.amm_get_state(ctx)
        e = np.abs(out - ref) / scale
        # the ambient gas far from the blast holds ~1e-8 of its energy
        far = ref[:, 4] < 1e-6 * ref[:, 4].max()
        assert far.sum() > 1000
        assert e.max() < tol, (prec, acc64, e.max(), e[far].max())


def test_fixed_point_truncation_within_its_bound(amm, blast):
    P, Q = blast
    dt = O.step(O.Mesh(P.tess), Q, P.gamma, "eulerian", cfl=0.3)[1]
    out, AF = {}, None
    for acc64 in (False, True):
        ctx = amm.create_from_mesh(P.tess, Q, P.gamma, precision="fp32", mesh_motion="eulerian", fp64_accumulate=acc64)
        amm.amm_step(ctx, dt)
        out[acc64] = amm.amm_get_state(ctx)
        if not acc64:
            AF = amm.amm_get_face_flux(ctx)
    cells = P.tess.cells
    n = P.n_cells
    nfaces = np.bincount(cells[:, 0], minlength=n) + np.bincount(cells[:, 1], minlength=n)
    headroom = 1
    while (1 << headroom) < nfaces.max() + 1:
        headroom += 1
    headroom += 1
    absAF = np.abs(AF)
    # per cell: the sum of |A F| over its faces (scale of the FP64 sums' rounding)
    sabs = np.zeros((n, 5))
    np.add.at(sabs, cells[:, 0], absAF)
    np.add.at(sabs, cells[:, 1], absAF)
    quantum = 2.0 ** (headroom - 61) * absAF.max(axis=0)
    bound = dt * (nfaces[:, None] * quantum[None, :] + (nfaces[:, None] + 2) * EPS64 * sabs) + \
        4 * EPS64 * (np.abs(Q) + dt * sabs)
    diff = np.abs(out[False] - out[True])
    assert np.all(diff <= 2 * bound), float((diff / (2 * bound)).max())
    # on the ambient cells' own scale the truncation is far below FP32
    # rounding of their fluxes
    scale = own_scale(out[True], P.gamma)
    far = out[True][:, 4] < 1e-6 * out[True][:, 4].max()
    assert (diff[far] / scale[far]).max() < 1e-9
