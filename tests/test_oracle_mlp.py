"""Pins of the FP64 MLP oracle: a hand-evaluated tiny network, central finite
differences of the loss, torch autograd in float64, and the Adam formula on a
quadratic whose minimiser is known."""
import numpy as np
import pytest

from oracle import mlp


def test_forward_hand_evaluated():
    """Only unit 0 of each layer is live: y = w3 * silu(w2 * silu(w1 . x + b1) + b2) + b3."""
    p = {k: np.zeros_like(v) for k, v in mlp.init_params(np.random.default_rng(0)).items()}
    p["W1"][0] = [0.5, -1.0, 0.25, 0.0, 2.0, 0.0]
    p["b1"][0] = 0.1
    p["W2"][0, 0] = 1.5
    p["b2"][0] = -0.2
    p["W3"][0, 0] = 2.0
    p["b3"][0] = 0.3
    x = np.array([[1.0, 2.0, -4.0, 9.0, 0.5, 7.0]])
    z1 = 0.5 - 2.0 - 1.0 + 1.0 + 0.1            # -1.4
    h1 = z1 / (1 + np.exp(-z1))
    z2 = 1.5 * h1 - 0.2
    h2 = z2 / (1 + np.exp(-z2))
    y_hand = 2.0 * h2 + 0.3
    # the other 63 hidden units have zero pre-activation: silu(0) = 0, no effect
    y, _ = mlp.forward(p, x)
    assert abs(y[0] - y_hand) < 1e-15


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = mlp.init_params(rng)
    for k in p:
        p[k] = p[k] + 0.05 * rng.normal(size=p[k].shape)
    x = rng.normal(size=(32, 6))
    t = rng.normal(size=32)
    _, g = mlp.loss_and_grads(p, x, t)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp, _ = mlp.loss_and_grads(p, x, t)
            flat[i] = old - h
            lm, _ = mlp.loss_and_grads(p, x, t)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[k].reshape(-1)[i] - fd) <= 1e-7 * max(1.0, abs(fd)), (k, i)


def test_backward_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    p = mlp.init_params(rng)
    x = rng.normal(size=(64, 6))
    t = rng.normal(size=64)
    loss, g = mlp.loss_and_grads(p, x, t)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    tx = torch.tensor(x, dtype=torch.float64)
    h1 = torch.nn.functional.silu(tx @ tp["W1"].T + tp["b1"])
    h2 = torch.nn.functional.silu(h1 @ tp["W2"].T + tp["b2"])
    y = (h2 @ tp["W3"].T + tp["b3"])[:, 0]
    tl = torch.mean((y - torch.tensor(t)) ** 2)
    tl.backward()
    assert abs(tl.item() - loss) < 1e-14
    for k in p:
        assert np.allclose(tp[k].grad.numpy(), g[k], rtol=1e-12, atol=1e-14), k


def test_features_are_scale_and_frame_free():
    """The normalisation makes the features invariant to rescaling rho and p
    (and velocities with c); the target log(p*/pbar) is invariant too."""
    rng = np.random.default_rng(3)
    a = [rng.uniform(0.5, 2, 5) for _ in range(6)]
    x1, pb1 = mlp.features(*a, 1.4)
    s_rho, s_p = 3.0, 7.0
    cfac = np.sqrt(s_p / s_rho)
    b = [a[0] * s_rho, a[1] * s_p, a[2] * cfac, a[3] * s_rho, a[4] * s_p, a[5] * cfac]
    x2, pb2 = mlp.features(*b, 1.4)
    assert np.allclose(x1, x2, rtol=1e-14, atol=1e-14)
    assert np.allclose(pb2, pb1 * s_p)


def test_adam_reaches_known_minimum():
    """Adam on L = sum (w - c)^2 converges to c."""
    c = np.array([1.0, -2.0, 0.5])
    p = {"w": np.zeros(3)}
    st = {}
    for _ in range(3000):
        p = mlp.adam_step(p, {"w": 2 * (p["w"] - c)}, st, lr=0.01)
    assert np.allclose(p["w"], c, atol=1e-6)


def test_bf16_rounding_model_is_within_the_gpu_tolerance():
    """The GPU backward is held to 1e-2 (per entry, against max(|g|, its error
    scale)) of this oracle.  The FP64 evaluation at the kernel's BF16
    rounding points stays inside that bound on many random networks, so the
    bound leaves room only for the FP32 accumulation; and the mistakes a
    kernel could make (a transposed or mis-indexed block, a sign, a scale)
    are far outside it."""
    from oracle import mlp as M
    from tests.test_gpu_mlp import _entrywise, backward_bf16, bf16, propagated_scales
    worst = 0.0
    planted = []
    for n in (1000, 300, 77, 33):
        for seed in range(4):
            rng = np.random.default_rng(100 + n + 1000 * seed)
            p = M.init_params(rng)
            for k in p:
                p[k] = (p[k] + 0.1 * rng.normal(size=p[k].shape)).astype(np.float32).astype(np.float64)
            for k in ("W1", "W2", "W3"):
                p[k] = bf16(p[k])
            x = bf16(rng.normal(size=(n, 6)))
            t = rng.normal(size=n).astype(np.float32).astype(np.float64)
            _, gref = M.loss_and_grads(p, x, t)
            gemu, S = backward_bf16(p, x, t)
            Sp = propagated_scales(p, x, t)
            F = {k: np.maximum(S[k], Sp[k]) for k in S}
            worst = max(worst, max(_entrywise(gemu[k], gref[k], F[k]) for k in gref))
            planted.append(min(_entrywise(gemu["W2"].T, gref["W2"], F["W2"]),
                               _entrywise(gemu["W1"][::-1], gref["W1"], F["W1"]),
                               _entrywise(-gemu["b1"], gref["b1"], F["b1"]),
                               _entrywise(np.roll(gemu["b2"], 1), gref["b2"], F["b2"]),
                               _entrywise(2 * gemu["W3"], gref["W3"], F["W3"])))
    assert worst < 1e-2, worst
    assert min(planted) > 0.1, min(planted)
