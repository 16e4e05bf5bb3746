"""Train the learned shock sensor on labels of the plain sensor (Eq. 42-43).

    python -m paper_2209_15333_gb300.train_sensor [--out PATH] [--quick]

Data (all generated here, seeded): the 42 features (cfd_sensor_features) and
the plain sensor's node classes (cfd_get_flags) of
  * isotropic-turbulence blocks of the ensemble recipe (dims from
    {32,48,64,96,128}, Mt in [0.3, 0.7]), snapshots while they evolve;
  * the Mach 2.9, 24 degree compression ramp at reduced resolution
    (512 x 128 x 16), snapshots while the corner shock forms.
Training set: turbulence blocks 0..7 and ramp snapshots at even indices;
validation: blocks 8..11 and ramp snapshots at odd indices.
The model (42 -> 32 -> 32 -> 3, ReLU) is trained with PyTorch on the host
(seed 7, class-weighted cross entropy, an extra penalty on choosing a less
dissipative scheme than the label), its inputs standardised with the
training statistics folded into the first layer, then evaluated with the
kernel's roundings (bf16 weights, features and activations).

UD7 nodes are subsampled when collected; each sample carries the weight of
the nodes it stands for, so rates on the validation set are rates over all
nodes.  The training set is balanced, which shifts the model's prior
towards the WENO classes; a logit offset for UD7 (folded into b3) and the
confidence threshold are then chosen on the validation set: the smallest
fallback rate whose unsafe rate (a less dissipative class than the plain
sensor's, taken with confidence) stays below 2e-5 of all nodes.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "sensor_mlp.npz")


def collect(quick=False):
    import torch
    from . import build, cases
    from .solver import Solver
    build.build()
    torch.cuda.init()
    X, Y, G, Wt = [], [], [], []  # features, labels, group id (train 0 / validation 1), sample weights

    def snap(s, group, keep_ud7=0.08, rng=None):
        s.rhs()                   # plain sensor classes of the current state
        c = s.flags().ravel()
        f = s.sensor_features().reshape(42, -1).T
        idx_w = np.nonzero(c > 0)[0]
        idx_u = np.nonzero(c == 0)[0]
        take = rng.choice(idx_u, size=min(len(idx_u), max(2000, int(keep_ud7 * len(idx_u)))), replace=False)
        sel = np.concatenate([idx_w, take])
        X.append(f[sel])
        Y.append(c[sel])
        G.append(np.full(len(sel), group, np.int8))
        Wt.append(np.concatenate([np.ones(len(idx_w)), np.full(len(take), len(idx_u) / max(1, len(take)))]))

    rng = np.random.default_rng(7)
    blocks = cases.ensemble_blocks(6 if quick else 12, seed=1234)
    for b, blk in enumerate(blocks):
        group = 0 if b < (4 if quick else 8) else 1
        with Solver(blk["shape"], blk["metrics"], scheme=3, Re=blk["Re"], Ma=blk["Mt"], visc_law=1,
                    visc_omega=0.76) as s:
            s.set_state(blk["U"])
            dt = s.cfl_dt(0.5)
            for t in range(3 if quick else 5):
                s.step(dt, 40)
                snap(s, group, rng=rng)
    nx, ny, nz = (256, 64, 8) if quick else (512, 128, 16)
    rc = cases.ramp_case(nx, ny, nz, 24.0, 2.9, Tw=2.8)
    with Solver((nx, ny, nz), rc["metrics2d"], bc_lo=(2, 1, 0), bc_hi=(3, 3, 0), scheme=3, Re=20000.0, Ma=2.9,
                T_wall=2.8, visc_law=0, T_ref=108.1) as s:
        s.set_inflow(rc["inflow"])
        s.set_state(rc["U"])
        dt = s.cfl_dt(0.4)
        for t in range(6 if quick else 12):
            s.step(dt, 100)
            snap(s, t % 2, keep_ud7=0.02, rng=rng)
    return (np.concatenate(X).astype(np.float32), np.concatenate(Y).astype(np.int64), np.concatenate(G),
            np.concatenate(Wt))


def bf16(a):
    from .solver import from_bf16_bits, to_bf16_bits
    return from_bf16_bits(to_bf16_bits(np.asarray(a, np.float32)))


def forward_kernel_rounding(F, W):
    x = bf16(F)
    h = np.maximum(x @ bf16(W["w1"]).T + W["b1"], 0.0)
    h = np.maximum(bf16(h) @ bf16(W["w2"]).T + W["b2"], 0.0)
    return bf16(h) @ bf16(W["w3"]).T + W["b3"]


def scores(logits, y, conf_min=0.0, w=None):
    """Rates over the nodes the samples stand for (weights w).  With a
    confidence threshold, a node below it takes the plain sensor's class:
    it counts as a fallback and is then classified correctly."""
    w = np.ones(len(y)) if w is None else w
    p = np.exp(logits - logits.max(axis=1, keepdims=True))
    p /= p.sum(axis=1, keepdims=True)
    pred = p.argmax(axis=1)
    fb = p.max(axis=1) < conf_min if conf_min > 0 else np.zeros(len(y), bool)
    used = np.where(fb, y, pred)
    W = w.sum()
    out = {"n": int(len(y)), "nodes": float(W), "misclassification": float((w * (used != y)).sum() / W),
           "unsafe_rate": float((w * (used < y)).sum() / W)}
    for c in range(3):
        m = y == c
        out["recall_%d" % c] = float((w[m] * (used[m] == c)).sum() / w[m].sum()) if m.any() else None
    if conf_min > 0:
        out["fallback_rate"] = float((w * fb).sum() / W)
    return out


def calibrate(logits, y, w, unsafe_max=2e-5):
    """UD7 logit offset and confidence threshold: the smallest fallback
    rate with the unsafe rate at most unsafe_max (validation set)."""
    best = None
    for off in np.linspace(0.0, 6.0, 25):
        lg = logits.copy()
        lg[:, 0] += off
        for conf in (0.5, 0.6, 0.7, 0.8, 0.9, 0.95, 0.98, 0.99):
            sc = scores(lg, y, conf, w)
            if sc["unsafe_rate"] <= unsafe_max and (best is None or sc["fallback_rate"] < best[2]["fallback_rate"]):
                best = (float(off), conf, sc)
    return best


def train(X, Y, G, epochs=30, seed=7):
    import torch
    torch.manual_seed(seed)
    tr, va = G == 0, G == 1
    mu = X[tr].mean(axis=0)
    sd = X[tr].std(axis=0) + 1e-6
    xt = torch.tensor((X[tr] - mu) / sd)
    yt = torch.tensor(Y[tr])
    counts = np.bincount(Y[tr], minlength=3).astype(np.float64)
    wcls = torch.tensor((counts.sum() / (3.0 * np.maximum(counts, 1.0))).astype(np.float32))
    net = torch.nn.Sequential(torch.nn.Linear(42, 32), torch.nn.ReLU(), torch.nn.Linear(32, 32), torch.nn.ReLU(),
                              torch.nn.Linear(32, 3))
    opt = torch.optim.Adam(net.parameters(), lr=3e-3)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, epochs)
    n = len(xt)
    gen = torch.Generator().manual_seed(seed)
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen)
        for i in range(0, n, 4096):
            b = perm[i:i + 4096]
            logits = net(xt[b])
            loss = torch.nn.functional.cross_entropy(logits, yt[b], weight=wcls)
            # penalise probability mass on schemes less dissipative than the label
            prob = torch.softmax(logits, dim=1)
            cls = torch.arange(3).unsqueeze(0)
            loss = loss + 2.0 * (prob * (cls < yt[b].unsqueeze(1)).float()).sum(dim=1).mean()
            opt.zero_grad()
            loss.backward()
            opt.step()
        sched.step()
    layers = [m for m in net if isinstance(m, torch.nn.Linear)]
    w1 = layers[0].weight.detach().numpy().astype(np.float64)
    b1 = layers[0].bias.detach().numpy().astype(np.float64)
    # fold the standardisation into the first layer: W (x - mu)/sd + b
    W = {"w1": (w1 / sd).astype(np.float32), "b1": (b1 - (w1 / sd) @ mu).astype(np.float32),
         "w2": layers[1].weight.detach().numpy(), "b2": layers[1].bias.detach().numpy(),
         "w3": layers[2].weight.detach().numpy(), "b3": layers[2].bias.detach().numpy()}
    return W, tr, va


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--unsafe-max", type=float, default=2e-5)
    a = ap.parse_args()
    t0 = time.time()
    X, Y, G, Wt = collect(a.quick)
    W, tr, va = train(X, Y, G, epochs=10 if a.quick else 30)
    lv = forward_kernel_rounding(X[va], W)
    uncal = scores(lv, Y[va], 0.9, Wt[va])
    cal = calibrate(lv, Y[va], Wt[va], a.unsafe_max)
    off, conf = (cal[0], cal[1]) if cal else (0.0, 0.9)
    W["b3"] = W["b3"].copy()
    W["b3"][0] += off
    a.conf_min = conf
    report = {"train": scores(forward_kernel_rounding(X[tr], W), Y[tr], 0.0, Wt[tr]),
              "validation": scores(forward_kernel_rounding(X[va], W), Y[va], conf, Wt[va]),
              "validation_uncalibrated_conf_0.9": uncal, "ud7_logit_offset": off,
              "class_counts": np.bincount(Y, minlength=3).tolist(), "conf_min": conf,
              "seconds": time.time() - t0}
    from .solver import to_bf16_bits
    np.savez(a.out, w1=to_bf16_bits(W["w1"]), w2=to_bf16_bits(W["w2"]), w3=to_bf16_bits(W["w3"]),
             b1=W["b1"], b2=W["b2"], b3=W["b3"], conf_min=np.float32(a.conf_min), report=json.dumps(report))
    print(json.dumps(report))


def load(path=DEFAULT_OUT):
    """Weights as float arrays (from their bf16 bits) and the stored report."""
    from .solver import from_bf16_bits
    z = np.load(path)
    W = {k: from_bf16_bits(z[k]) for k in ("w1", "w2", "w3")}
    W.update({k: z[k] for k in ("b1", "b2", "b3")})
    return W, float(z["conf_min"]), json.loads(str(z["report"]))


if __name__ == "__main__":
    sys.exit(main())
