"""GPU checks of the learned troubled-cell indicator against the FP64 reference in
oracle/mlp.py: harvested features, flags and labels; gradients, loss and the Adam step of
the training kernels; tensor-core inference; and what the trained network gains."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
import paper_1904_11147_gb300 as dgl
from paper_1904_11147_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _bf16(a):
    """Round-to-nearest-even to bfloat16 (kept in float64)."""
    a = np.asarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _unpack(p, F):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + 32 * F].reshape(32, F); o += 32 * F
    b1 = p[o:o + 32]; o += 32
    W2 = p[o:o + 1024].reshape(32, 32); o += 1024
    b2 = p[o:o + 32]; o += 32
    w3 = p[o:o + 32]; o += 32
    b3 = p[o:o + 1]
    return {"W1": W1, "b1": b1, "W2": W2, "b2": b2, "w3": w3, "b3": b3}


def _pack(d):
    return np.concatenate([d["W1"].ravel(), d["b1"], d["W2"].ravel(), d["b2"], d["w3"], d["b3"]]).astype(np.float32)


@pytest.mark.parametrize("dim,pde,N,nx,ny,bc", [(2, 1, 2, 40, 33, 1), (2, 0, 2, 37, 21, 0), (1, 1, 3, 300, 1, 1),
                                                (2, 1, 3, 24, 20, 1)])
def test_harvest_features_flags_labels(dim, pde, N, nx, ny, bc):
    import torch
    o = oracle.Mesh(dim, pde, N, nx, ny, bc=bc)
    g = dgl.Mesh(dim, pde, N, [nx], [ny], None, bc=bc)
    rng = np.random.default_rng(31 + N)
    u = W.random_modes(dim, pde, N, nx * ny, rng, smooth=0.15 if pde == 0 else 0.02)
    g.set_modes(u)
    F = dgl.n_features(dim, pde, N)
    assert F == omlp.n_features(dim, pde, N)
    X = torch.empty(nx * ny, F, dtype=torch.float32, device="cuda")
    fl = torch.empty(nx * ny, dtype=torch.uint8, device="cuda")
    ch = torch.empty(nx * ny, dtype=torch.float32, device="cuda")
    g.harvest(X, fl, ch)
    torch.cuda.synchronize()
    Xo = omlp.features(o, u)
    np.testing.assert_allclose(X.cpu().numpy(), Xo, rtol=1e-6, atol=1e-6 * np.abs(Xo).max())
    fo, lo, co = omlp.labels(o, u)
    assert np.array_equal(fl.cpu().numpy(), fo)
    np.testing.assert_allclose(ch.cpu().numpy(), co, rtol=1e-6, atol=1e-12)
    assert (co > 0).sum() > 0
    # the harvest also limited the state exactly as the plain method does
    ref = o.limit(u, fo)
    got = g.get_modes()
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_training_kernels_match_reference():
    import torch
    F, B = 116, 3000
    rng = np.random.default_rng(5)
    ref = omlp.init_params(F, rng)
    for k in ref:
        ref[k] = ref[k] + 0.02 * rng.normal(size=np.shape(ref[k]))
    X = rng.normal(size=(B, F)).astype(np.float32)
    y = (rng.uniform(size=B) < 0.25).astype(np.uint8)
    net = dgl.MLP(F, seed=1)
    p32 = _pack(ref)
    net.set_params(p32)
    ref = _unpack(p32, F)  # the reference uses exactly the FP32 parameters
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    g, loss = net.grad(Xd, yd, pos_weight=3.0)
    X64 = X.astype(np.float64)
    assert abs(loss - omlp.loss(ref, X64, y.astype(np.float64), 3.0)) < 1e-5
    gr = omlp.grads(ref, X64, y.astype(np.float64), 3.0)
    gref = _pack(gr).astype(np.float64)
    assert np.abs(g - gref).max() <= 1e-4 * np.abs(gref).max()
    # one Adam step: from zero moments the bias-corrected step is lr g / (|g| + eps); check
    # it against the reference optimiser fed with the GPU's own FP32 gradient (where |g|
    # is near eps the step is sensitive to the gradient's last bits, so only bound it)
    net.set_params(p32)
    net.train_step(Xd, yd, pos_weight=3.0, lr=1e-3)
    after = net.get_params().astype(np.float64)
    refp = omlp.adam_step(_unpack(p32, F), _unpack(g, F), {}, lr=1e-3)
    big = np.abs(g) > 1e-6
    np.testing.assert_allclose(after[big], _pack(refp).astype(np.float64)[big], rtol=0, atol=2e-6)
    assert np.abs(after - p32).max() <= 1e-3 * (1 + 1e-5)
    # forward pass
    z = torch.empty(B, dtype=torch.float32, device="cuda")
    net.set_params(p32)
    net.predict(Xd, z)
    zr, _ = omlp.forward(ref, X64)
    np.testing.assert_allclose(z.cpu().numpy(), zr, rtol=1e-4, atol=1e-4)
    # the gradient is reduced in a fixed order: repeated calls agree bit for bit, and so
    # do two networks trained from the same parameters on the same batches
    g2, _ = net.grad(Xd, yd, pos_weight=3.0)
    assert np.array_equal(g, g2)
    nets = [dgl.MLP(F, seed=1) for _ in range(2)]
    for nt in nets:
        nt.set_params(p32)
        for _ in range(3):
            nt.train_step(Xd, yd, pos_weight=3.0, lr=1e-3)
    assert np.array_equal(nets[0].get_params(), nets[1].get_params())


def test_training_pipeline_is_reproducible():
    """Harvest, training and the threshold choice twice from the same seeds: the same
    parameters bit for bit and the same tau (the harvest follows the deterministic plain
    method; the gradient is reduced in a fixed order)."""
    from paper_1904_11147_gb300 import train as T
    runs = [T.train_indicator(seeds_train=(11, 12), seeds_val=(21,), n=32, steps=30, epochs=2) for _ in range(2)]
    (n1, t1, i1), (n2, t2, i2) = runs
    assert np.array_equal(n1.get_params(), n2.get_params())
    assert t1 == t2 and i1["train_samples"] == i2["train_samples"] > 0


def test_tensor_core_inference_matches_reference():
    """Fused flagging pass (BF16 features and weights on the tensor cores, FP32
    accumulation) against the FP64 network applied to the same BF16-rounded inputs; the
    hidden activations are rounded to BF16 on the GPU as well, hence the tolerance."""
    import torch
    n = 64
    w = W.euler_2d_quadrant(n, 2, seed=77)
    g = dgl.Mesh(2, 1, 2, [n], [n], w.box, bc=1)
    o = oracle.Mesh(2, 1, 2, n, n, box=w.box[0], bc=1)
    g.project_ic(w.ic, w.params[0])
    ws = g.max_wavespeed()[0]
    dt = 0.1 / (ws[0] * n + ws[1] * n)
    for _ in range(20):
        g.step(dt)
    g.rk_stage(1, dt)
    u = g.get_modes()
    F = dgl.n_features(2, 1, 2)
    rng = np.random.default_rng(8)
    ref = omlp.init_params(F, rng)
    for k in ref:
        ref[k] = ref[k] + 0.05 * rng.normal(size=np.shape(ref[k]))
    net = dgl.MLP(F)
    net.set_params(_pack(ref))
    tau = 0.1
    g.set_indicator(net, tau)
    z = torch.empty(n * n, dtype=torch.float32, device="cuda")
    g.logits(z)
    tvb, _, _ = g.flag_cells(dgl.IND_TVB, 0.01, want=True)
    fl, nf, _ = g.flag_cells(dgl.IND_MLP, 0.01, want=True)
    torch.cuda.synchronize()
    z = z.cpu().numpy()
    Xo = omlp.features(o, u)
    refb = {k: (_bf16(v) if k in ("W1", "W2") else np.asarray(v, dtype=np.float32).astype(np.float64))
            for k, v in ref.items()}
    zr, _ = omlp.forward(refb, _bf16(Xo))
    err = np.abs(z - zr)
    assert np.median(err) < 5e-3 and err.max() < 0.1 * (1 + np.abs(zr).max()), (np.median(err), err.max())
    # the learned flags are the TVB flags the network keeps (same tensor-core pass)
    keep = (tvb == 1) & (z > tau)
    assert np.array_equal(fl[tvb == 1], keep[tvb == 1].astype(np.uint8))
    assert nf == int(keep.sum()) and 0 < nf < int(tvb.sum())
    clear = (np.abs(zr - tau) > 0.2) & (tvb == 1)
    assert np.array_equal(fl[clear], (zr[clear] > tau).astype(np.uint8))


@pytest.mark.parametrize("tol,recall", [(0.05, 0.995), (0.2, 0.95)])
def test_trained_indicator_gains(tol, recall):
    """The network trained on harvested data from other seeds keeps the recall of the
    limiter-relevant cells while limiting fewer cells than the TVB indicator; the learned
    run (CUDA graph with the positivity fallback) stays finite and positive, and its
    density error against a run on a mesh twice as fine stays within 5 % (L1) of the
    plain run's.  Two label definitions: a limiter change above 5 % at 99.5 % recall, and
    above 20 % at 95 % recall (the benchmark's)."""
    import torch
    from paper_1904_11147_gb300 import train as T
    net, tau, info = T.train_indicator(seeds_train=(11, 12, 13, 14), seeds_val=(21,), n=64, steps=80, epochs=4,
                                       tol=tol, recall=recall)
    print(info)
    assert info["val_recall"] >= recall - 0.005
    assert info["val_predicted"] < info["val_tvb_flagged"]
    n = 64
    w = W.euler_2d_quadrant(n, 2, seed=31)
    st = torch.cuda.Stream()

    def run(mesh_n, ind, steps):
        m = dgl.Mesh(2, 1, 2, [mesh_n], [mesh_n], w.box, bc=1, stream=st.cuda_stream)
        m.project_ic(w.ic, w.params[0])
        if ind == dgl.IND_MLP:
            m.set_indicator(net, tau)
        ws = m.max_wavespeed()[0]
        dt = 0.1 / (ws[0] * mesh_n + ws[1] * mesh_n)
        with torch.cuda.stream(st):
            for _ in range(steps):
                m.step(dt, ind, 0.01)
        st.synchronize()
        tvbf, limited, passes = m.flag_statistics()
        assert passes == 3 * steps
        fb = m.positivity_report() if ind == dgl.IND_MLP else (0, 0)
        return m.get_modes(), tvbf, limited, fb, dt

    plain, f_tvb, f_plain, _, dt = run(n, dgl.IND_TVB, 150)
    learned, _, f_learned, (fallbacks, failures), _ = run(n, dgl.IND_MLP, 150)
    assert f_tvb == f_plain
    assert np.isfinite(learned).all() and failures == 0
    assert f_learned < f_plain
    fine, _, _, _, dtf = run(2 * n, dgl.IND_TVB, 300)
    rho_f = fine[:, 0, 0].reshape(2 * n, 2 * n)
    rho_ref = 0.25 * (rho_f[0::2, 0::2] + rho_f[1::2, 0::2] + rho_f[0::2, 1::2] + rho_f[1::2, 1::2])
    e_plain = np.abs(plain[:, 0, 0].reshape(n, n) - rho_ref).mean()
    e_learned = np.abs(learned[:, 0, 0].reshape(n, n) - rho_ref).mean()
    print("limited cells plain %d learned %d (fallbacks %d); L1 plain %.3e learned %.3e"
          % (f_plain, f_learned, fallbacks, e_plain, e_learned))
    assert abs(dtf - dt / 2) < 1e-12 * dt
    assert e_learned <= 1.05 * e_plain


def test_positivity_fallback_restores_plain_limiting():
    """A network that never flags (tau far above every logit) leaves the shock cells of a
    strong four-quadrant problem unlimited; the positivity screen must then fall back to the
    TVB flags for that instance, and the result stays positive."""
    import torch
    F = dgl.n_features(2, 1, 2)
    net = dgl.MLP(F, seed=3)
    n = 48
    w = W.euler_2d_quadrant(n, 2, seed=1904)
    st = torch.cuda.Stream()
    m = dgl.Mesh(2, 1, 2, [n], [n], w.box, bc=1, stream=st.cuda_stream)
    m.project_ic(w.ic, w.params[0])
    m.set_indicator(net, 1e30)
    ws = m.max_wavespeed()[0]
    dt = 0.1 / (ws[0] * n + ws[1] * n)
    with torch.cuda.stream(st):
        for _ in range(60):
            m.step(dt, dgl.IND_MLP, 0.01)
    st.synchronize()
    fallbacks, failures = m.positivity_report()
    tvbf, limited, _ = m.flag_statistics()
    u = m.get_modes()
    print("fallbacks %d failures %d tvb %d limited %d" % (fallbacks, failures, tvbf, limited))
    assert fallbacks > 0 and failures == 0 and limited > 0
    assert np.isfinite(u).all()
