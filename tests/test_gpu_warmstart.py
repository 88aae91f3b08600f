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


def test_training_reduces_the_loss():
    # a target that depends on the point set: its centroid and extent
    N, B = 64, 16
    rng = np.random.default_rng(7)
    Y = rng.uniform(-1, 1, (256, N, 3)).astype(np.float32) * rng.uniform(0.3, 1.0, (256, 1, 3)).astype(np.float32)
    tgt = np.concatenate([Y.mean(1), Y.max(1) - Y.min(1)], axis=1).astype(np.float32)
    net = warmstart.Net(6, N, max_batch=B, seed=1)
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


def test_learned_warm_start_needs_fewer_iterations():
    cfg = datagen.WARMSTART_WORKLOADS["fp32_warmstart_m512_k32"]
    X = datagen.gen(cfg["M"], seed=cfg["seed_x"]).X.astype(np.float32)
    n = cfg["n_train"] + cfg["n_val"] + cfg["n_test"]
    sets = [datagen.gen_from_template(X, cfg["seed0"] + i, amp=cfg["amp"], noise=cfg["noise"]) for i in range(n)]
    Ys = np.stack([s.Y.astype(np.float32) for s in sets])
    with cpd.Context(torch.tensor(X, device="cuda"), precision=cpd.FP32, w=cfg["omega"], beta=cfg["beta"],
                     lam=cfg["lam"], K=cfg["K"]) as ctx:
        tr, va = cfg["n_train"], cfg["n_train"] + cfg["n_val"]
        targets = warmstart.registration_targets(ctx, Ys[:va], cfg["K"], cfg["iters"])
        ws = warmstart.WarmStart(cfg["K"], cfg["M"], max_batch=cfg["batch"], seed=3)
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
