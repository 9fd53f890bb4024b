"""Training driver of the learned Riemann-pressure proposal.

Argument marshalling and data plumbing only: face states are harvested by
the library's own flux kernel (amm_harvest), exact p* targets come from its
FP64 Riemann kernel (amm_riemann_pstar), features from amm_mlp_features, and
every forward/backward/Adam step runs in its tensor-core kernels
(amm_mlp_train_step).  PyTorch only holds device buffers and draws the
minibatch permutations.

Recipe: states harvested from the method's own runs (the 2D shock tube run
to its end time and single steps of 3D turbulent boxes of several seeds,
sizes and Mach numbers), kept where the proposal is used (strong
compression: the linearised star pressure above TRAIN_GATE times the larger
side pressure), target the correction log(p*/p_TS) of the two-shock estimate,
an 80/20 split by a seeded permutation, Adam with a step-decayed learning
rate, MSE loss.
"""
import numpy as np

from . import amm

# training keeps faces a little below the inference gate, so the network also
# covers the states just around it
TRAIN_GATE = 1.1


def harvest(tess, Q, gamma, mesh_motion, steps, cfl=0.3, torch=None):
    """Runs `steps` FP32 steps of one problem, recording every face's Riemann
    inputs; returns a [steps * n_faces, 6] float32 device tensor."""
    ctx = amm.create_from_mesh(tess, Q, gamma, precision="fp32", mesh_motion=mesh_motion)
    nf = tess.n_faces
    out = torch.empty((steps, nf, 6), dtype=torch.float32, device="cuda")
    for s in range(steps):
        amm.amm_harvest(ctx, cfl, out[s].data_ptr())
    try:
        amm.amm_sync(ctx)
    except amm.AmmError as e:
        # a cell driven non-positive by the last update does not spoil the
        # recorded inputs of that update's Riemann problems
        if e.code != amm.AMM_ERR_NUMERIC:
            raise
    amm.amm_destroy(ctx)
    return out.reshape(-1, 6)


def dataset(states, gamma, torch, gate=TRAIN_GATE):
    """(features, targets) on the device for the faces whose compression
    ratio ppv / max(p_L, p_R) exceeds `gate`; target log(p*/p_TS).  Faces
    without a star region (vacuum generated) are dropped."""
    m = states.shape[0]
    x = torch.empty((m, 6), dtype=torch.float32, device="cuda")
    ratio = torch.empty(m, dtype=torch.float32, device="cuda")
    t = torch.empty(m, dtype=torch.float32, device="cuda")
    amm.amm_mlp_features(gamma, m, states.data_ptr(), x.data_ptr(), 0, 0, ratio.data_ptr())
    amm.amm_mlp_targets(gamma, m, states.data_ptr(), 1e-12, t.data_ptr())
    torch.cuda.synchronize()
    # selection only (the kernels computed features and targets)
    ok = torch.isfinite(t) & torch.isfinite(x).all(dim=1) & (ratio > gate)
    return x[ok].contiguous(), t[ok].contiguous()


def init_params(seed):
    """He-style initialisation of the parameter vector (W1,b1,W2,b2,W3,b3)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((64, 6)) * np.sqrt(2.0 / 6)
    W2 = rng.standard_normal((64, 64)) * np.sqrt(2.0 / 64)
    W3 = rng.standard_normal((1, 64)) * np.sqrt(1.0 / 64)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3.ravel(), np.zeros(1)])


def train(x, t, torch, epochs=4, batch=4096, lr=2e-3, seed=4, gamma=5.0 / 3.0, log=None, decay=0.5):
    """Trains a fresh network on (x, t) with an 80/20 split; returns
    (net, stats) with train/validation MSE."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    m = x.shape[0]
    perm = torch.randperm(m, generator=g, device="cuda").to(torch.int32)
    ntr = int(0.8 * m)
    tr, va = perm[:ntr].contiguous(), perm[ntr:].contiguous()
    net = amm.amm_mlp_create(gamma)
    amm.amm_mlp_set_params(net, init_params(seed))
    steps_per_epoch = max(1, ntr // batch)
    for ep in range(epochs):
        order = tr[torch.randperm(ntr, generator=g, device="cuda")].contiguous()
        rate = lr * (decay ** ep)
        for s in range(steps_per_epoch):
            idx = order[s * batch:(s + 1) * batch]
            amm.amm_mlp_train_step(net, x.data_ptr(), t.data_ptr(), idx.data_ptr(), idx.shape[0], rate)
        amm.amm_mlp_sync(net)
        if log:
            _, lv = amm.amm_mlp_grads(net, x.data_ptr(), t.data_ptr(), va.data_ptr(), va.shape[0])
            log("epoch %d lr %.2e val_mse %.3e" % (ep, rate, lv))
    _, ltr = amm.amm_mlp_grads(net, x.data_ptr(), t.data_ptr(), tr.data_ptr(), min(ntr, 1 << 20))
    _, lva = amm.amm_mlp_grads(net, x.data_ptr(), t.data_ptr(), va.data_ptr(), va.shape[0])
    # the two-shock estimate itself predicts a zero correction
    base = float((t[va.long()] ** 2).mean().item())
    return net, {"train_mse": ltr, "val_mse": lva, "two_shock_val_mse": base, "samples": m, "epochs": epochs,
                 "batch": batch}


def default_sources(ics, small=False):
    """The harvest sources: the 2D shock tube (gamma 1.4) stepped to t=0.2,
    one step of 64^3 turbulent boxes (gamma 5/3) of several seeds, and one
    step of coarser turbulent boxes at rms Mach 2 to 4, where strong
    compression is common.  Seeds 9 and 20-99 are left for held-out tests."""
    if small:
        return [(ics.sod_2d(64, 32, seed=1), "eulerian", 40)] + \
               [(ics.turbulent_3d(20, seed=100 + k, mach=m), "lagrangian", 1)
                for k, m in enumerate((2.0, 3.0, 4.0, 2.5, 3.5, 2.0))]
    return [(ics.sod_2d(128, 64, seed=1), "eulerian", 160)] + \
           [(ics.turbulent_3d(64, seed=s), "lagrangian", 1) for s in range(2, 9)] + \
           [(ics.turbulent_3d(n, seed=100 + k, mach=m), mode, 1)
            for k, (n, m, mode) in enumerate([(24, 2.0, "lagrangian"), (24, 3.0, "lagrangian"), (24, 4.0, "eulerian"),
                                               (32, 2.5, "lagrangian"), (32, 3.5, "eulerian"), (32, 4.0, "lagrangian"),
                                               (40, 3.0, "lagrangian"), (40, 4.0, "eulerian"), (24, 2.5, "eulerian"),
                                               (32, 2.0, "eulerian")])]


def train_proposal(ics, torch, small=False, epochs=12, log=None):
    """Harvest -> dataset -> train; returns (net, stats).  gamma of each
    source is kept for its own targets; the network sees normalised states."""
    xs, ts = [], []
    for P, motion, steps in default_sources(ics, small):
        st = harvest(P.tess, P.conserved(), P.gamma, motion, steps, torch=torch)
        x, t = dataset(st, P.gamma, torch)
        xs.append(x)
        ts.append(t)
        del st
    x = torch.cat(xs).contiguous()
    t = torch.cat(ts).contiguous()
    return train(x, t, torch, epochs=epochs, log=log, batch=2048, decay=0.75)
