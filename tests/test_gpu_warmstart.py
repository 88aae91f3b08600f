"""Learned warm start (GPU): the network's kernels against the FP64 reference,
the coefficient round trip, and what a trained network gains over starting
the EM loop at W = 0."""
import numpy as np
import pytest

from oracle import warmstart as ref
from paper_2006_06281_gb300 import cpd, datagen, warmstart

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_06281_gb300 import build
    build.build()
    cpd.load()


def test_forward_and_gradients_match_the_fp64_reference():
    n_out, N, B = 7, 16, 3
    net = warmstart.Net(n_out, N, max_batch=4, seed=5)
    p = net.params().astype(np.float64)
    rng = np.random.default_rng(6)
    Y = rng.uniform(-1, 1, (B, N, 3)).astype(np.float32)
    tgt = rng.normal(0, 1, (B, n_out)).astype(np.float32)
    Yd = torch.tensor(Y, device="cuda")
    pred = net.forward(Yd)
    pred_ref, _ = ref.forward(p, Y.astype(np.float64), n_out)
    np.testing.assert_allclose(pred, pred_ref, rtol=1e-4, atol=1e-5 * np.abs(pred_ref).max())
    g, loss = net.gradients(Yd, tgt)
    g_ref = ref.gradients(p, Y.astype(np.float64), tgt.astype(np.float64), n_out)
    assert loss == pytest.approx(ref.loss(pred_ref, tgt), rel=1e-4)
    # per layer, relative to the layer's largest gradient (FP32 sums)
    o = 0
    for fi, fo in ref.shapes(n_out):
        for size in (fi * fo, fo):
            a, b = g[o:o + size], g_ref[o:o + size]
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-4 * max(np.abs(b).max(), 1e-12))
            o += size
    net.close()


# --- BF16 precision: the per-point products on the tensor cores -------------

def _bf16(x):
    """Nearest BF16 (ties to even; torch's conversion) as float64."""
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _random_params(n_out, seed):
    """He-scaled weights and small nonzero biases (the epilogue adds them)."""
    rng = np.random.default_rng(seed)
    out = []
    for fi, fo in ref.shapes(n_out):
        out.append(rng.normal(0, np.sqrt(2.0 / fi), fi * fo))
        out.append(rng.normal(0, 0.05, fo))
    return np.concatenate(out).astype(np.float32)


def _bf16_operand_reference(p, Y, tgt, n_out):
    """The FP64 network with the operands of the tensor-core products rounded
    to BF16 exactly where the BF16 precision rounds them: h1, h2, W2, W3
    forward; h1, h2, dh3, dh2, W2, W3 in the backward products.  Everything
    else (first layer, max-pool, head, bias gradients) is the FP64 reference.
    Returns the prediction, the flat gradients, and h3 (B, N, 256)."""
    (W0, b0), (W1, b1), (W2, b2), (W3, b3), (W4, b4) = ref.unpack(np.asarray(p, np.float64), n_out)
    B, N, _ = Y.shape
    x = np.asarray(Y, np.float64).reshape(B * N, 3)
    h1 = np.maximum(x @ W0 + b0, 0)
    h2 = np.maximum(_bf16(h1) @ _bf16(W1) + b1, 0)
    h3 = np.maximum(_bf16(h2) @ _bf16(W2) + b2, 0)
    H3 = h3.reshape(B, N, 256)
    g, arg = H3.max(1), H3.argmax(1)
    z = np.maximum(g @ W3 + b3, 0)
    pred = z @ W4 + b4
    dpred = 2.0 * (pred - np.asarray(tgt, np.float64)) / pred.size
    grads = [None] * 5
    grads[4] = (z.T @ dpred, dpred.sum(0))
    dz = (dpred @ W4.T) * (z > 0)
    grads[3] = (g.T @ dz, dz.sum(0))
    dg = dz @ W3.T
    dh3 = np.zeros((B, N, 256))
    bi, fi = np.meshgrid(np.arange(B), np.arange(256), indexing="ij")
    dh3[bi, arg, fi] = dg
    dh3 = dh3.reshape(B * N, 256) * (h3 > 0)
    grads[2] = (_bf16(h2).T @ _bf16(dh3), dh3.sum(0))
    dh2 = (_bf16(dh3) @ _bf16(W2).T) * (h2 > 0)
    grads[1] = (_bf16(h1).T @ _bf16(dh2), dh2.sum(0))
    dh1 = (_bf16(dh2) @ _bf16(W1).T) * (h1 > 0)
    grads[0] = (x.T @ dh1, dh1.sum(0))
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return pred, flat, H3


def _max_gap(H3):
    """Smallest relative gap between the largest and second-largest value of
    a live (positive) max-pool feature; routing is unambiguous above it."""
    s = np.sort(H3, axis=1)
    top = s[:, -1, :]
    sec = s[:, -2, :] if H3.shape[1] > 1 else np.zeros_like(top)
    live = top > 0
    return float(((top - sec) / np.where(live, top, 1.0))[live].min()) if live.any() else 1.0


def _per_layer(a, b, n_out, frac):
    o = 0
    for fi, fo in ref.shapes(n_out):
        for size in (fi * fo, fo):
            x, y = a[o:o + size], b[o:o + size]
            np.testing.assert_allclose(x, y, rtol=0, atol=frac * max(np.abs(y).max(), 1e-12))
            o += size


# BF16 bound against the FP64 network: each product rounds both operands
# (relative 2^-9 each) and errors pass through at most five rounded products
# on the way to a gradient, 5 * 2 * 2^-9 < 2^-5, taken relative to the
# layer's largest entry.  Against the BF16-operand reference only FP32
# accumulation and rare BF16 rounding-boundary flips remain: 1e-3.
BF16_VS_FP64 = 2.0 ** -5
BF16_VS_EMULATED = 1e-3


@pytest.mark.parametrize("B,N,seed", [(1, 5, 19), (3, 100, 15)])
def test_bf16_forward_and_gradients_match_the_bf16_operand_reference(B, N, seed):
    # R = B N points: one ragged row tile, and three tiles with a ragged tail
    # (also in the contraction of the weight gradients: 300 = 4 x 64 + 44)
    n_out = 7
    rng = np.random.default_rng(seed)
    Y = rng.uniform(-1, 1, (B, N, 3)).astype(np.float32)
    tgt = rng.normal(0, 1, (B, n_out)).astype(np.float32)
    p = _random_params(n_out, 100 + seed)
    pred_e, g_e, H3 = _bf16_operand_reference(p, Y, tgt, n_out)
    # the seeds are chosen so that no max-pool feature is near a tie
    assert _max_gap(H3) > 5e-4
    net = warmstart.Net(n_out, N, max_batch=B, seed=0, precision=warmstart.NET_BF16)
    assert net.precision == warmstart.NET_BF16
    net.set_params(p)
    Yd = torch.tensor(Y, device="cuda")
    pred = net.forward(Yd)
    scale = np.abs(pred_e).max()
    np.testing.assert_allclose(pred, pred_e, rtol=0, atol=BF16_VS_EMULATED * scale)
    pred_ref, _ = ref.forward(p.astype(np.float64), Y.astype(np.float64), n_out)
    np.testing.assert_allclose(pred, pred_ref, rtol=0, atol=BF16_VS_FP64 * np.abs(pred_ref).max())
    g, loss = net.gradients(Yd, tgt)
    assert loss == pytest.approx(ref.loss(pred_e, tgt), rel=1e-3)
    _per_layer(g, g_e, n_out, BF16_VS_EMULATED)
    net.close()


def test_bf16_gradients_within_the_bf16_bound_of_the_fp64_network():
    # one point per scene: the max-pool routes nothing, so the FP64 network's
    # gradients are the target; 300 scenes = three row tiles, ragged
    n_out, B, N = 5, 300, 1
    rng = np.random.default_rng(21)
    Y = rng.uniform(-1, 1, (B, N, 3)).astype(np.float32)
    tgt = rng.normal(0, 1, (B, n_out)).astype(np.float32)
    p = _random_params(n_out, 22)
    net = warmstart.Net(n_out, N, max_batch=B, seed=0, precision=warmstart.NET_BF16)
    net.set_params(p)
    g, _ = net.gradients(torch.tensor(Y, device="cuda"), tgt)
    g_ref = ref.gradients(p.astype(np.float64), Y.astype(np.float64), tgt.astype(np.float64), n_out)
    _per_layer(g, g_ref, n_out, BF16_VS_FP64)
    _, g_e, _ = _bf16_operand_reference(p, Y, tgt, n_out)
    _per_layer(g, g_e, n_out, BF16_VS_EMULATED)
    net.close()


def test_bf16_long_contraction_and_many_tiles():
    # 4 scenes x 4096 points: 128 row tiles, and weight-gradient contractions
    # of 16384 points split into 128 chunks of two 64-point steps.  Forward:
    # random points.  Gradients: every scene repeats one point, so which
    # point the max-pool routes to cannot change a gradient.
    n_out, B, N = 9, 4, 4096
    rng = np.random.default_rng(31)
    p = _random_params(n_out, 32)
    net = warmstart.Net(n_out, N, max_batch=B, seed=0, precision=warmstart.NET_BF16)
    net.set_params(p)
    Y = rng.uniform(-1, 1, (B, N, 3)).astype(np.float32)
    tgt = rng.normal(0, 1, (B, n_out)).astype(np.float32)
    pred = net.forward(torch.tensor(Y, device="cuda"))
    pred_e, _, _ = _bf16_operand_reference(p, Y, tgt, n_out)
    np.testing.assert_allclose(pred, pred_e, rtol=0, atol=BF16_VS_EMULATED * np.abs(pred_e).max())
    Yr = np.repeat(rng.uniform(-1, 1, (B, 1, 3)), N, axis=1).astype(np.float32)
    g, _ = net.gradients(torch.tensor(Yr, device="cuda"), tgt)
    _, g_e, _ = _bf16_operand_reference(p, Yr, tgt, n_out)
    _per_layer(g, g_e, n_out, BF16_VS_EMULATED)
    net.close()


def test_bf16_gemm_wait_timeout_is_reported_and_recoverable(monkeypatch):
    """Host fault injection: every full barrier of the BF16 tensor-core GEMM
    expects 16 bytes more than its copies carry, so its bounded waits run
    out (50 ms); the call reports CPD_ETIMEOUT, the GPU stays usable and the
    next call equals one before the fault."""
    n_out, B, N = 5, 3, 100
    rng = np.random.default_rng(41)
    Yd = torch.tensor(rng.uniform(-1, 1, (B, N, 3)).astype(np.float32), device="cuda")
    net = warmstart.Net(n_out, N, max_batch=B, seed=2, precision=warmstart.NET_BF16)
    before = net.forward(Yd)
    monkeypatch.setenv("CPD_FAULT", "gemm_wait")
    with pytest.raises(cpd.CpdError) as ei:
        net.forward(Yd)
    assert ei.value.status == cpd.ETIMEOUT
    monkeypatch.delenv("CPD_FAULT")
    np.testing.assert_array_equal(net.forward(Yd), before)
    net.close()


@pytest.mark.parametrize("precision", [warmstart.NET_FP32, warmstart.NET_BF16])
def test_training_reduces_the_loss(precision):
    # a target that depends on the point set: its centroid and extent
    N, B = 64, 16
    rng = np.random.default_rng(7)
    Y = rng.uniform(-1, 1, (256, N, 3)).astype(np.float32) * rng.uniform(0.3, 1.0, (256, 1, 3)).astype(np.float32)
    tgt = np.concatenate([Y.mean(1), Y.max(1) - Y.min(1)], axis=1).astype(np.float32)
    net = warmstart.Net(6, N, max_batch=B, seed=1, precision=precision)
    Yd = torch.tensor(Y, device="cuda")
    first = last = None
    for s in range(400):
        idx = rng.choice(256, B, replace=False)
        loss = net.train_step(Yd[idx].contiguous(), tgt[idx], 1e-3)
        first = loss if first is None else first
        last = loss
    assert last < 0.1 * first, (first, last)
    net.close()


def test_coefficients_and_warm_start_round_trip():
    ps = datagen.gen(500, seed=3)
    X = torch.tensor(ps.X, dtype=torch.float32, device="cuda")
    Y = torch.tensor(ps.Y, dtype=torch.float32, device="cuda")
    with cpd.Context(X, precision=cpd.FP32, K=40) as c:
        T, s2, _ = c.iterate(Y, 20)
        coef = c.coefficients(40)
        # in the top-K basis T - X lies in span(U): T = X + U c
        c.warm_start(coef, s2)
        T2, s2b, it = c.iterate(Y, 0)
        assert it == 0 and s2b == pytest.approx(s2)
        np.testing.assert_allclose(T2.cpu().numpy(), T.cpu().numpy(), rtol=0, atol=2e-6)
        # n_coef = 0: T = X
        c.warm_start(np.zeros((0, 3), np.float32), 1.0)
        T0, _, _ = c.iterate(Y, 0)
        np.testing.assert_array_equal(T0.cpu().numpy(), ps.X.astype(np.float32))


@pytest.fixture(scope="module")
def _ws_data():
    """Scenes and method-generated targets of the small warm-start workload."""
    cfg = datagen.WARMSTART_WORKLOADS["fp32_warmstart_m512_k32"]
    X = datagen.gen(cfg["M"], seed=cfg["seed_x"]).X.astype(np.float32)
    n = cfg["n_train"] + cfg["n_val"] + cfg["n_test"]
    sets = [datagen.gen_from_template(X, cfg["seed0"] + i, amp=cfg["amp"], noise=cfg["noise"]) for i in range(n)]
    Ys = np.stack([s.Y.astype(np.float32) for s in sets])
    with cpd.Context(torch.tensor(X, device="cuda"), precision=cpd.FP32, w=cfg["omega"], beta=cfg["beta"],
                     lam=cfg["lam"], K=cfg["K"]) as ctx:
        targets = warmstart.registration_targets(ctx, Ys[:cfg["n_train"] + cfg["n_val"]], cfg["K"], cfg["iters"])
    return cfg, X, Ys, targets


@pytest.mark.parametrize("precision", [warmstart.NET_FP32, warmstart.NET_BF16])
def test_learned_warm_start_needs_fewer_iterations(_ws_data, precision):
    cfg, X, Ys, targets = _ws_data
    with cpd.Context(torch.tensor(X, device="cuda"), precision=cpd.FP32, w=cfg["omega"], beta=cfg["beta"],
                     lam=cfg["lam"], K=cfg["K"]) as ctx:
        tr, va = cfg["n_train"], cfg["n_train"] + cfg["n_val"]
        ws = warmstart.WarmStart(cfg["K"], cfg["M"], max_batch=cfg["batch"], seed=3, precision=precision)
        losses = ws.fit(Ys[:tr], targets[:tr], cfg["steps"], cfg["batch"], cfg["lr"])
        assert np.mean(losses[-50:]) < 0.5 * np.mean(losses[:20])
        ws.calibrate(Ys[tr:va], targets[tr:va], cfg["M"])
        # held-out end points: the predicted displacement |U c| within 30 % of the true one
        c, _ = ws.predict(Ys[tr:va])
        ct = targets[tr:va, :-1].reshape(c.shape)
        err = np.linalg.norm(c - ct) / np.linalg.norm(ct)
        print(f"held-out relative coefficient error {err:.3f}")
        assert err < 0.3
        cold, warm = [], []
        for Y in Ys[va:]:
            Yd = torch.tensor(Y, device="cuda")
            # the registration's end point, then iterations until RMSE(T, end) <= 1e-3
            ctx.reset()
            Tend, _, _ = ctx.iterate(Yd, 150)
            ctx.set_ground_truth(Tend, 1e-3)
            ctx.reset()
            _, _, it_cold = ctx.iterate(Yd, 150, want_T=False)
            ws.start(ctx, Y)
            _, _, it_warm = ctx.iterate(Yd, 150, want_T=False)
            ctx.set_ground_truth(None)
            cold.append(it_cold)
            warm.append(it_warm)
        print(f"iterations to RMSE(T, T_end) <= 1e-3: cold {np.mean(cold):.1f}, warm {np.mean(warm):.1f}")
        assert np.mean(warm) < 0.8 * np.mean(cold)


def test_coefficients_of_a_given_T_and_the_mixed_context():
    """cpd_coefficients_of(T) equals cpd_coefficients for the context's own
    T, and shared-model registrations give the targets the one-at-a-time
    registrations give; a CPD_MIXED context (FP16 basis of the same
    eigenvectors) takes the same coefficients: its warm-start T = X + U c
    matches the FP32 context's to the FP16 rounding of U."""
    M, K = 600, 24
    X = datagen.gen(M, seed=71).X.astype(np.float32)
    Ys = [datagen.gen_from_template(X, 7100 + i, amp=0.15, noise=0.01).Y.astype(np.float32) for i in range(5)]
    Xd = torch.tensor(X, device="cuda")
    with cpd.Context(Xd, precision=cpd.FP32, K=K) as ctx:
        T, _, _ = ctx.iterate(torch.tensor(Ys[0], device="cuda"), 20)
        np.testing.assert_allclose(ctx.coefficients_of(T, K), ctx.coefficients(K), rtol=0, atol=1e-6)
        seq = warmstart.registration_targets(ctx, Ys, K, 30, group=1)
        grp = warmstart.registration_targets(ctx, Ys, K, 30, group=4)
        assert np.abs(seq - grp).max() <= 1e-4 * max(np.abs(seq).max(), 1.0)
        c = seq[0, :-1].reshape(K, 3)
        ctx.warm_start(c, 1e-3)
        T32 = ctx.iterate(torch.tensor(Ys[0], device="cuda"), 0)[0].double().cpu().numpy()
    with cpd.Context(Xd, precision=cpd.MIXED, K=K) as cm:
        cm.warm_start(c, 1e-3)
        Tm = cm.iterate(torch.tensor(Ys[0], device="cuda"), 0)[0].double().cpu().numpy()
        cm_c = cm.coefficients(K)
    D = T32 - X.astype(np.float64)
    assert np.linalg.norm(Tm - T32) <= 2.0 ** -10 * np.linalg.norm(D)
    np.testing.assert_allclose(cm_c, c, rtol=0, atol=2.0 ** -9 * np.abs(c).max())
