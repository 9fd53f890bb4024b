"""FP64 numpy oracle of the learned Riemann-pressure proposal.

TEST INFRASTRUCTURE ONLY (tests/, smoke check, CPU-baseline leg).

The proposal is a 6 -> 64 -> 64 -> 1 multilayer perceptron with SiLU
activations that maps a normalised face state to y = log(p* / pbar), where
pbar = (p_L + p_R)/2; the Newton iteration of the exact Riemann solver then
starts from pbar * exp(y).  The paper has no such component; the layer sizes,
activation and target are the specification of the learned form.

Features (normalisation): with rhobar = (rho_L + rho_R)/2, pbar as above and
cbar = sqrt(gamma pbar / rhobar):
  x = (log(rho_L/rhobar), log(p_L/pbar), u_L/cbar,
       log(rho_R/rhobar), log(p_R/pbar), u_R/cbar).

Parameters are a dict with W1 [64,6], b1 [64], W2 [64,64], b2 [64],
W3 [1,64], b3 [1] (row = output unit, as in y = W x + b).
"""
import numpy as np

N_IN, N_HID = 6, 64


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def features(rhoL, pL, uL, rhoR, pR, uR, gamma):
    rhoL, pL, uL, rhoR, pR, uR = (np.asarray(a, np.float64) for a in (rhoL, pL, uL, rhoR, pR, uR))
    rhob = 0.5 * (rhoL + rhoR)
    pb = 0.5 * (pL + pR)
    cb = np.sqrt(gamma * pb / rhob)
    x = np.stack([np.log(rhoL / rhob), np.log(pL / pb), uL / cb, np.log(rhoR / rhob), np.log(pR / pb), uR / cb], 1)
    return x, pb


def init_params(rng, scale=1.0):
    """He-style random initialisation (used for tests and as the training start)."""
    p = {
        "W1": rng.standard_normal((N_HID, N_IN)) * scale * np.sqrt(2.0 / N_IN),
        "b1": np.zeros(N_HID),
        "W2": rng.standard_normal((N_HID, N_HID)) * scale * np.sqrt(2.0 / N_HID),
        "b2": np.zeros(N_HID),
        "W3": rng.standard_normal((1, N_HID)) * scale * np.sqrt(1.0 / N_HID),
        "b3": np.zeros(1),
    }
    return p


def forward(params, x):
    """Returns y [B] and the cache of pre-activations."""
    z1 = x @ params["W1"].T + params["b1"]
    h1 = silu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = silu(z2)
    y = (h2 @ params["W3"].T + params["b3"])[:, 0]
    return y, (x, z1, h1, z2, h2)


def loss_and_grads(params, x, t):
    """Mean squared error L = mean((y - t)^2) and dL/dparams (analytic backward)."""
    y, (x, z1, h1, z2, h2) = forward(params, x)
    B = x.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = (2.0 / B) * r                       # [B]
    gW3 = dy[None, :] @ h2                   # [1,64]
    gb3 = np.array([dy.sum()])
    dh2 = dy[:, None] * params["W3"]         # [B,64]
    dz2 = dh2 * dsilu(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dh1 = dz2 @ params["W2"]
    dz1 = dh1 * dsilu(z1)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(0)
    return loss, {"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3}


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) on FP64 copies; `state` holds m, v, t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    new = {}
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        g = grads[k]
        m[...] = beta1 * m + (1 - beta1) * g
        v[...] = beta2 * v + (1 - beta2) * g * g
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        new[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return new
