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
    # the training target log(p*/p_TS) against the oracle's p* and the
    # kernel's own FP32 two-shock estimate p_TS
    pts = torch.empty(m, dtype=torch.float32, device="cuda")
    tg = torch.empty(m, dtype=torch.float32, device="cuda")
    amm.amm_mlp_features(gam, m, sd.data_ptr(), xd.data_ptr(), 0, pts.data_ptr(), 0)
    amm.amm_mlp_targets(gam, m, sd.data_ptr(), 1e-12, tg.data_ptr())
    torch.cuda.synchronize()
    t_gpu, pts_h = tg.cpu().numpy().astype(np.float64), pts.cpu().numpy().astype(np.float64)
    assert np.all(np.isnan(t_gpu[vac]))
    good = ok & (pts_h > 0)
    assert np.max(np.abs(t_gpu[good] - np.log(out[good, 3] / pts_h[good]))) < 1e-6


def _blocks(g):
    from paper_0901_4107_gb300 import amm
    return amm.unpack_params(g)


def backward_bf16(p, x, t):
    """FP64 evaluation of the backward with the kernel's rounding points: BF16
    copies of the weights and of every tensor-core operand (x, h1, dZ2, dZ1),
    everything else unrounded.  Returns the gradients and, per entry, the
    sum of the magnitudes of the terms it adds up (the scale of its rounding
    error)."""
    xb, W1b, W2b, W3b = bf16(x), bf16(p["W1"]), bf16(p["W2"]), bf16(p["W3"])
    B = x.shape[0]
    z1 = xb @ W1b.T + p["b1"]
    h1b = bf16(M.silu(z1))
    z2 = h1b @ W2b.T + p["b2"]
    h2 = M.silu(z2)
    y = (h2 @ W3b.T)[:, 0] + p["b3"][0]
    dy = (2.0 / B) * (y - t)
    dz2 = dy[:, None] * W3b * M.dsilu(z2)
    dz2b = bf16(dz2)
    dz1 = (dz2b @ W2b) * M.dsilu(z1)
    dz1b = bf16(dz1)
    g = {"W3": dy[None, :] @ h2, "b3": np.array([dy.sum()]), "W2": dz2b.T @ h1b, "b2": dz2.sum(0),
         "W1": dz1b.T @ xb, "b1": dz1.sum(0)}
    S = {"W3": np.abs(dy)[None, :] @ np.abs(h2), "b3": np.array([np.abs(dy).sum()]),
         "W2": np.abs(dz2).T @ np.abs(h1b), "b2": np.abs(dz2).sum(0), "W1": np.abs(dz1).T @ np.abs(xb),
         "b1": np.abs(dz1).sum(0)}
    return g, S


def _entrywise(a, ref, scale):
    """per-entry error relative to max(|ref|, the entry's error scale)"""
    return float(np.max(np.abs(a - ref) / np.maximum(np.abs(ref), scale)))


def propagated_scales(p, x, t):
    """First-order running error scale of each gradient entry: the backward
    evaluated on magnitudes, with each BF16 rounding upstream (h1 before the
    second layer, and through it y, dy and dZ2) contributing one BF16 ulp of
    the magnitude it rounds.  Needed where an entry is a small difference of
    terms that the rounding of an earlier layer shifts."""
    U = 2.0 ** -8
    B = x.shape[0]
    aW2, aW3 = np.abs(p["W2"]), np.abs(p["W3"])
    z1 = x @ p["W1"].T + p["b1"]
    h1 = M.silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = M.silu(z2)
    y = (h2 @ p["W3"].T)[:, 0] + p["b3"][0]
    A2 = np.abs(h1) @ aW2.T + np.abs(p["b2"])
    H2 = np.abs(h2) + U * A2
    Y = (H2 @ aW3.T)[:, 0] + abs(p["b3"][0])
    Dy = (2.0 / B) * (np.abs(y - t) + U * Y)
    D2 = Dy[:, None] * aW3 * (np.abs(M.dsilu(z2)) + U * A2)
    D1 = (D2 @ aW2) * np.abs(M.dsilu(z1))
    return {"W3": Dy[None, :] @ H2, "b3": np.array([Dy.sum()]), "W2": D2.T @ np.abs(h1), "b2": D2.sum(0),
            "W1": D1.T @ np.abs(x), "b1": D1.sum(0)}


@pytest.mark.parametrize("n", [1000, 300, 77])
def test_gradients_match_oracle(env, n):
    """Tensor-core backward (BF16 operands, FP32 accumulation), entry by entry:
    within 1e-2 of the FP64 oracle's analytic backward for every parameter
    block (relative to the entry, or to the sum of the magnitudes of its
    terms where the sum cancels), and within 5e-4 of the FP64 evaluation at
    the kernel's BF16 rounding points, which leaves only the FP32
    accumulation and rare one-ulp differences of a BF16 rounding (one ulp,
    2^-8, of one term of a sum of hundreds is a few 1e-5 of its scale)."""
    torch, amm = env
    rng = np.random.default_rng(100 + n)
    p = M.init_params(rng)
    for k in p:
        p[k] = (p[k] + 0.1 * rng.normal(size=p[k].shape)).astype(np.float32).astype(np.float64)
    # weights and inputs on the BF16 grid: the network the kernel evaluates
    # is then exactly the oracle's (the FP32 master copies only feed Adam)
    for k in ("W1", "W2", "W3"):
        p[k] = bf16(p[k])
    x = bf16(rng.normal(size=(n, 6)))
    t = rng.normal(size=n).astype(np.float32).astype(np.float64)
    net = amm.amm_mlp_create(1.4)
    amm.amm_mlp_set_params(net, amm.pack_params(p))
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    g, loss = amm.amm_mlp_grads(net, xd.data_ptr(), td.data_ptr(), 0, n)
    loss_ref, gref = M.loss_and_grads(p, x, t)
    assert abs(loss - loss_ref) < 2e-2 * loss_ref
    gb = _blocks(g)
    gemu, S = backward_bf16(p, x, t)
    Sp = propagated_scales(p, x, t)
    for k in gref:
        assert gb[k].shape == gref[k].shape, k
        e_oracle = _entrywise(gb[k], gref[k], np.maximum(S[k], Sp[k]))
        assert e_oracle < 1e-2, (k, e_oracle)
        e_emu = _entrywise(gb[k], gemu[k], S[k])
        assert e_emu < 5e-4, (k, e_emu)
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
