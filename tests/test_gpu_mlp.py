"""GPU checks of the learned-proposal network and its data path against the
FP64 numpy oracle (oracle/mlp.py) and the FP64 Riemann oracle."""
import numpy as np
import pytest

from oracle import mlp as M
from oracle import oracle as O

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


def bf16(a):
    """round to bfloat16 (nearest even) and back, in float64"""
    a = np.asarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(p, x):
    """the oracle forward with the kernel's rounding points: BF16 weights,
    BF16 inputs to each tensor-core layer, FP32-or-better elsewhere"""
    z1 = bf16(x) @ bf16(p["W1"]).T + p["b1"]
    h1 = M.silu(z1)
    z2 = bf16(h1) @ bf16(p["W2"]).T + p["b2"]
    return (M.silu(z2) @ bf16(p["W3"]).T)[:, 0] + p["b3"][0]


@pytest.mark.parametrize("n", [1000, 128, 77])
def test_forward_matches_oracle(env, n):
    torch, amm = env
    rng = np.random.default_rng(n)
    p = M.init_params(rng)
    for k in p:
        p[k] = p[k] + 0.1 * rng.normal(size=p[k].shape)
    p = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    x = rng.normal(size=(n, 6)).astype(np.float32).astype(np.float64)
    net = amm.amm_mlp_create(1.4)
    amm.amm_mlp_set_params(net, amm.pack_params(p))
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    yd = torch.empty(n, dtype=torch.float32, device="cuda")
    amm.amm_mlp_forward(net, xd.data_ptr(), n, yd.data_ptr())
    y = yd.cpu().numpy().astype(np.float64)
    yb = forward_bf16(p, x)
    scale = np.abs(yb).max()
    assert np.max(np.abs(y - yb)) < 2e-3 * scale, np.max(np.abs(y - yb)) / scale
    y64, _ = M.forward(p, x)
    assert np.max(np.abs(y - y64)) < 5e-2 * np.abs(y64).max()


def test_features_and_exact_pstar(env):
    torch, amm = env
    rng = np.random.default_rng(7)
    m = 3000
    gam = 5.0 / 3.0
    rL, rR = np.exp(rng.uniform(-2, 2, m)), np.exp(rng.uniform(-2, 2, m))
    pL, pR = np.exp(rng.uniform(-3, 3, m)), np.exp(rng.uniform(-3, 3, m))
    uL, uR = rng.normal(size=m), rng.normal(size=m)
    st = np.column_stack([rL, uL, pL, rR, uR, pR]).astype(np.float32)
    sd = torch.from_numpy(st).cuda()
    xd = torch.empty((m, 6), dtype=torch.float32, device="cuda")
    pb = torch.empty(m, dtype=torch.float32, device="cuda")
    amm.amm_mlp_features(gam, m, sd.data_ptr(), xd.data_ptr(), pb.data_ptr())
    ps = torch.empty(m, dtype=torch.float32, device="cuda")
    amm.amm_riemann_pstar(gam, m, sd.data_ptr(), 1e-12, ps.data_ptr())
    torch.cuda.synchronize()
    s64 = st.astype(np.float64)
    x_ref, pb_ref = M.features(s64[:, 0], s64[:, 2], s64[:, 1], s64[:, 3], s64[:, 5], s64[:, 4], gam)
    assert np.max(np.abs(xd.cpu().numpy() - x_ref)) < 1e-5
    assert np.max(np.abs(pb.cpu().numpy() - pb_ref) / pb_ref) < 1e-6
    out, it, bad = O.riemann(gam, s64[:, :3], s64[:, 3:], tol=1e-12)
    vac = 2 * (np.sqrt(gam * s64[:, 2] / s64[:, 0]) + np.sqrt(gam * s64[:, 5] / s64[:, 3])) / (gam - 1) <= \
        s64[:, 4] - s64[:, 1]
    p_gpu = ps.cpu().numpy()
    assert np.all(np.isnan(p_gpu[vac]))
    ok = ~vac
    assert np.max(np.abs(p_gpu[ok] - out[ok, 3]) / out[ok, 3]) < 2e-7


def _blocks(g):
    from paper_0901_4107_gb300 import amm
    return amm.unpack_params(g)


@pytest.mark.parametrize("n", [1000, 300])
def test_gradients_match_oracle(env, n):
    """Tensor-core backward (BF16 operands, FP32 accumulation) against the
    FP64 oracle's analytic backward, block by block."""
    torch, amm = env
    rng = np.random.default_rng(100 + n)
    p = M.init_params(rng)
    for k in p:
        p[k] = (p[k] + 0.1 * rng.normal(size=p[k].shape)).astype(np.float32).astype(np.float64)
    x = rng.normal(size=(n, 6)).astype(np.float32).astype(np.float64)
    t = rng.normal(size=n).astype(np.float32).astype(np.float64)
    net = amm.amm_mlp_create(1.4)
    amm.amm_mlp_set_params(net, amm.pack_params(p))
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    g, loss = amm.amm_mlp_grads(net, xd.data_ptr(), td.data_ptr(), 0, n)
    loss_ref, gref = M.loss_and_grads(p, x, t)
    assert abs(loss - loss_ref) < 2e-2 * loss_ref
    gb = _blocks(g)
    for k in gref:
        err = np.linalg.norm(gb[k] - gref[k]) / max(np.linalg.norm(gref[k]), 1e-12)
        assert err < 5e-2, (k, err)
    # a permuted index list gives the same gradient (sums are per sample)
    perm = rng.permutation(n).astype(np.int32)
    idx = torch.from_numpy(perm).cuda()
    g2, loss2 = amm.amm_mlp_grads(net, xd.data_ptr(), td.data_ptr(), idx.data_ptr(), n)
    assert np.allclose(g2, g, rtol=1e-3, atol=1e-6 * np.abs(g).max())


def test_training_reduces_loss(env):
    """Adam on a smooth target (a fixed teacher network) lowers the loss."""
    torch, amm = env
    rng = np.random.default_rng(3)
    n = 8192
    teacher = M.init_params(rng)
    x = rng.normal(size=(n, 6))
    y, _ = M.forward(teacher, x)
    net = amm.amm_mlp_create(1.4)
    amm.amm_mlp_set_params(net, amm.pack_params(M.init_params(np.random.default_rng(4))))
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    td = torch.from_numpy(y.astype(np.float32)).cuda()
    _, l0 = amm.amm_mlp_grads(net, xd.data_ptr(), td.data_ptr(), 0, n)
    for step in range(300):
        idx = torch.randint(0, n, (1024,), dtype=torch.int32, device="cuda", generator=None)
        amm.amm_mlp_train_step(net, xd.data_ptr(), td.data_ptr(), idx.data_ptr(), 1024, 3e-3)
    amm.amm_mlp_sync(net)
    _, l1 = amm.amm_mlp_grads(net, xd.data_ptr(), td.data_ptr(), 0, n)
    assert l1 < 0.1 * l0, (l0, l1)
