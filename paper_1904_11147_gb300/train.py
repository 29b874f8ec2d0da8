"""Training of the learned troubled-cell indicator with the library's own kernels.

Data: tuples (features, TVB flag, label) harvested by ``dg_harvest`` from the plain
method's own runs (TVB indicator + CSWENO limiter) on seeded random four-quadrant Riemann
problems.  The learned indicator filters the TVB flags (a cell is limited when the TVB
indicator flags it and the network's logit exceeds tau), so it is trained on the
TVB-flagged cells; the label is "the limiter changes the cell by more than tol s_v".
Training: weighted binary cross-entropy and Adam, by ``dg_mlp_train_step``.  The threshold
tau is the largest value that keeps a target recall of the labels on held-out data.
PyTorch only holds device memory here; every computation runs in the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import BC_OUTFLOW, EULER, IND_TVB, MLP, Mesh, n_features
from . import workloads as W


def harvest_quadrants(seeds, n=96, N=2, steps=120, every=3, keep_unflagged=0.0, stream=None, positivity=False):
    """Runs the plain method on four-quadrant problems (one per seed) and returns device
    tensors X [S, F] (float32), TVB flags [S] (uint8) and the limiter's relative change [S]
    (float32; zero for unflagged cells).  positivity: apply the positivity-preserving
    scaling after every stage's limiter and take every step's time step from the wave
    speeds at the scaling's check points (CFL 0.1), as the batched P3 workload does (P3
    runs lose positivity without both).  A run whose state stops being finite ends there;
    samples with non-finite features are dropped."""
    st = stream or torch.cuda.current_stream()
    F = n_features(2, EULER, N)
    xs, fs, ls = [], [], []
    gen = torch.Generator(device="cuda").manual_seed(1234)
    for seed in seeds:
        w = W.euler_2d_quadrant(n, N, seed=seed)
        m = Mesh(2, EULER, N, [n], [n], w.box, bc=BC_OUTFLOW, stream=st.cuda_stream)
        m.project_ic(w.ic, w.params[0])
        ws = m.max_wavespeed()[0]
        dt = 0.1 / (ws[0] * n + ws[1] * n)
        X = torch.empty(n * n, F, dtype=torch.float32, device="cuda")
        fl = torch.empty(n * n, dtype=torch.uint8, device="cuda")
        lab = torch.empty(n * n, dtype=torch.float32, device="cuda")
        k = 0
        with torch.cuda.stream(st):
            for step in range(steps):
                if positivity:
                    sp = m.max_wavespeed(points=True)[0]
                    dt = 0.1 / max(sp[0] * n + sp[1] * n, 1e-300)
                    if not math.isfinite(dt):
                        break
                for s in (1, 2, 3):
                    m.rk_stage(s, dt)
                    if k % every == 0:
                        m.harvest(X, fl, lab)
                        keep = (fl > 0) | (torch.rand(n * n, device="cuda", generator=gen) < keep_unflagged)
                        keep &= torch.isfinite(X).all(dim=1) & torch.isfinite(lab)
                        xs.append(X[keep].clone())
                        fs.append(fl[keep].clone())
                        ls.append(lab[keep].clone())
                    else:
                        m.flag_cells(IND_TVB, w.tvb_M)
                        m.cswenolimit()
                    if positivity:
                        m.positivity_limit()
                    k += 1
        st.synchronize()
        m.close()
    return torch.cat(xs), torch.cat(fs), torch.cat(ls)


def train(net, X, y, epochs=6, batch=8192, lr=2e-3, pos_weight=4.0, seed=0):
    """Mini-batch Adam over shuffled batches; returns the per-epoch mean losses."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    S = X.shape[0]
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(S, device="cuda", generator=g)
        tot, nb = 0.0, 0
        for i in range(0, S - batch + 1, batch):
            idx = perm[i:i + batch]
            xb, yb = X[idx].contiguous(), y[idx].contiguous()
            want = (i // batch) % 16 == 0
            l = net.train_step(xb, yb, pos_weight=pos_weight, lr=lr, want_loss=want)
            if want:
                tot += l
                nb += 1
        hist.append(tot / max(nb, 1))
    return hist


def choose_tau(net, X, y, recall=0.995):
    """Largest threshold whose recall of the positive labels on (X, y) is at least `recall`."""
    z = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    net.predict(X, z)
    torch.cuda.synchronize()
    pos = z[y > 0].double().cpu().numpy()
    if pos.size == 0:
        return 0.0
    pos.sort()
    k = int(math.floor((1.0 - recall) * pos.size))
    return float(pos[k] - 1e-3)


def train_indicator(seeds_train=(11, 12, 13, 14, 15, 16), seeds_val=(21, 22), n=96, steps=120, recall=0.995,
                    epochs=6, seed=0, tol=0.05, stream=None, N=2, positivity=False):
    """Harvest, train and calibrate a 2D Euler P^N indicator; returns (net, tau, info).
    Label: TVB-flagged and changed by the limiter by more than tol (relative to s_v)."""
    Xt, ft, ct = harvest_quadrants(seeds_train, n=n, N=N, steps=steps, stream=stream, positivity=positivity)
    Xv, fv, cv = harvest_quadrants(seeds_val, n=n, N=N, steps=steps, stream=stream, positivity=positivity)
    yt = (ct > tol).to(torch.uint8)
    yv = (cv > tol).to(torch.uint8)
    net = MLP(Xt.shape[1], seed=seed, stream=(stream or torch.cuda.current_stream()).cuda_stream)
    hist = train(net, Xt, yt, epochs=epochs, seed=seed)
    tau = choose_tau(net, Xv, yv, recall)
    z = torch.empty(Xv.shape[0], dtype=torch.float32, device="cuda")
    net.predict(Xv, z)
    pred = z > tau
    tp = int((pred & (yv > 0)).sum())
    info = {"train_samples": int(Xt.shape[0]), "val_samples": int(Xv.shape[0]),
            "val_positive": int((yv > 0).sum()), "val_tvb_flagged": int((fv > 0).sum()),
            "val_predicted": int(pred.sum()), "val_recall": tp / max(int((yv > 0).sum()), 1),
            "loss": hist, "tau": tau, "tol": tol}
    return net, tau, info
