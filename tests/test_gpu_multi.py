"""Several registrations against one model (cpd_iterate_shared, GPU).

Each scene is registered from W = 0 exactly as cpd_iterate would; only the
M-step products of a group of scenes share one pass over the eigenbasis:
up to 8 scenes per SIMT streaming kernel in an FP32 context, up to 32 per
tensor-core (tcgen05) pass over the FP16 basis of a CPD_MIXED context.
Every scene's T and sigma2 must equal an independent single-scene
registration's up to the summation order (and, on the tensor cores, the
2^-22 residue of splitting each right-hand side into two FP16 parts), and
the FP64 oracle's at the FP32 tolerance (mixed: at the mixed-precision
bound of test_gpu_parity).
"""
import numpy as np
import pytest

import oracle
from paper_2006_06281_gb300 import cpd, datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_06281_gb300 import build
    build.build()
    cpd.load()


def f32dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def scenes_for(X, n, seed0):
    # deformations of one template with uneven scene sizes (outliers, missing points)
    out = []
    for i in range(n):
        s = datagen.gen_from_template(X, seed0 + i, amp=0.15, noise=0.01)
        Y = s.Y.astype(np.float32)
        if i % 3 == 1:
            Y = np.vstack([Y, np.random.default_rng(seed0 + i).uniform(-1, 1, (57, 3)).astype(np.float32)])
        elif i % 3 == 2:
            Y = Y[: len(Y) - 101]
        out.append(Y)
    return out


@pytest.mark.parametrize("M,n_scenes,iters", [(1500, 5, 40), (300, 11, 25)])
def test_each_scene_equals_its_own_registration(M, n_scenes, iters):
    X = datagen.gen(M, seed=51).X.astype(np.float32)
    Ys = scenes_for(X, n_scenes, 700 + M)
    with cpd.Context(f32dev(X), precision=cpd.FP32) as ctx:
        res = ctx.iterate_shared([f32dev(Y) for Y in Ys], iters)
        # the context's own registration is untouched and still works
        T0, s20, it0 = ctx.iterate(f32dev(Ys[0]), iters)
    assert it0 == iters
    for i, (Y, (T, s2)) in enumerate(zip(Ys, res)):
        with cpd.Context(f32dev(X), precision=cpd.FP32) as single:
            Ts, s2s, _ = single.iterate(f32dev(Y), iters)
        T = T.cpu().numpy().astype(np.float64)
        Ts = Ts.cpu().numpy().astype(np.float64)
        assert rel(T, Ts) <= 5e-6, i
        assert abs(s2 - s2s) <= 1e-5 * s2s, i
    np.testing.assert_allclose(res[0][0].cpu().numpy(), T0.cpu().numpy(), rtol=0, atol=1e-5)


def test_a_shared_registration_against_the_oracle():
    X = datagen.gen(800, seed=52).X.astype(np.float32)
    Ys = scenes_for(X, 3, 900)
    with cpd.Context(f32dev(X), precision=cpd.FP32) as ctx:
        res = ctx.iterate_shared([Y for Y in Ys], 30)          # host arrays in and out
    for Y, (T, s2) in zip(Ys, res):
        ref = oracle.register(X.astype(np.float64), Y.astype(np.float64), w=0.1, beta=2.0, lam_reg=2.0, n_iter=30)
        assert ref["status"] == oracle.OK
        assert isinstance(T, np.ndarray)
        assert rel(T.astype(np.float64), ref["T"]) <= 1e-4
        assert abs(s2 - ref["sigma2"]) <= 1e-4 * ref["sigma2"]


def test_shared_registrations_need_a_context_without_flags():
    X = datagen.gen(200, seed=53).X.astype(np.float32)
    Y = f32dev(datagen.gen(200, seed=54).Y)
    for kw in (dict(precision=cpd.FP32, flags=cpd.FLAG_PRUNE),
               dict(precision=cpd.FP32, flags=cpd.FLAG_SPECTRAL_TRIM)):
        with cpd.Context(f32dev(X), **kw) as ctx:
            if kw.get("flags") == cpd.FLAG_SPECTRAL_TRIM and ctx.trim_info()[0] == 0:
                continue                                   # nothing trimmed: a plain context
            with pytest.raises(cpd.CpdError) as ei:
                ctx.iterate_shared([Y], 3)
            assert ei.value.status == cpd.EINVAL


# ------------------------------------------------ tensor-core products (MIXED)
@pytest.mark.parametrize("M,K,n_scenes,iters", [(1500, 0, 5, 40), (2000, 200, 16, 30), (300, 0, 33, 20)])
def test_mixed_tensor_core_products_equal_single_registrations(M, K, n_scenes, iters):
    """S scenes in one tcgen05 pass (npad = 2 x 3S rounded to 16: 32, 96,
    192 + 32 for the 33rd scene in a second group) against each scene's own
    CPD_MIXED registration (single-scene FP16-basis M-step)."""
    X = datagen.gen(M, seed=61).X.astype(np.float32)
    Ys = scenes_for(X, n_scenes, 800 + M)
    with cpd.Context(f32dev(X), precision=cpd.MIXED, K=K) as ctx:
        res = ctx.iterate_shared([f32dev(Y) for Y in Ys], iters)
    worst = 0.0
    for i, (Y, (T, s2)) in enumerate(zip(Ys, res)):
        with cpd.Context(f32dev(X), precision=cpd.MIXED, K=K) as single:
            Ts, s2s, _ = single.iterate(f32dev(Y), iters)
        Ts = Ts.cpu().numpy().astype(np.float64)
        d = rel(T.cpu().numpy().astype(np.float64), Ts)
        worst = max(worst, d)
        assert d <= 2e-5, (i, d)
        # sigma2 follows T's difference amplified by 2 |T|_rms / sqrt(3 sigma2)
        # (a mean of |y - t|^2 / 3 at distances ~ sqrt(3 sigma2)); the mixed
        # E-step's exponent rounding (~1e-3 at its floor) lets two mixed
        # registrations whose products round differently drift apart at the
        # 1e-5 level in T
        t_rms = float(np.sqrt((Ts ** 2).sum(1).mean()))
        s2tol = 2e-5 * max(1.0, 2.0 * t_rms / np.sqrt(3.0 * s2s))
        assert abs(s2 - s2s) <= s2tol * s2s, (i, abs(s2 - s2s) / s2s, s2tol)
    print(f"[shared mixed] M={M} K={K} S={n_scenes}: largest T difference vs single registrations {worst:.2e}")


def test_mixed_tensor_core_shared_registration_against_the_oracle():
    X = datagen.gen(900, seed=62).X.astype(np.float32)
    Ys = scenes_for(X, 3, 950)
    with cpd.Context(f32dev(X), precision=cpd.MIXED) as ctx:
        res = ctx.iterate_shared([Y for Y in Ys], 30)
    for Y, (T, s2) in zip(Ys, res):
        ref = oracle.register(X.astype(np.float64), Y.astype(np.float64), w=0.1, beta=2.0, lam_reg=2.0, n_iter=30)
        err = rel(T.astype(np.float64), ref["T"])
        print(f"[shared mixed] T vs oracle {err:.2e}, sigma2 {abs(s2 - ref['sigma2']) / ref['sigma2']:.2e}")
        assert err <= 3e-4
        assert abs(s2 - ref["sigma2"]) <= 1e-2 * ref["sigma2"]


def test_mixed_tensor_core_wait_timeout_is_reported_and_recoverable(monkeypatch):
    """Host fault injection: every full barrier of the tcgen05 kernel expects
    16 bytes more than its copies carry, so each bounded wait runs out
    (50 ms); the call reports CPD_ETIMEOUT, the GPU stays usable and the
    next call equals a fresh one."""
    X = datagen.gen(400, seed=63).X.astype(np.float32)
    Ys = [f32dev(Y) for Y in scenes_for(X, 2, 990)]
    with cpd.Context(f32dev(X), precision=cpd.MIXED) as ctx:
        ref = ctx.iterate_shared(Ys, 5)
        monkeypatch.setenv("CPD_FAULT", "umma_wait")
        with pytest.raises(cpd.CpdError) as ei:
            ctx.iterate_shared(Ys, 2)
        assert ei.value.status == cpd.ETIMEOUT
        monkeypatch.delenv("CPD_FAULT")
        again = ctx.iterate_shared(Ys, 5)
    for (a, _), (b, _) in zip(ref, again):
        assert torch.equal(a, b)
