"""Several registrations against one model (cpd_iterate_shared, GPU).

Each scene is registered from W = 0 exactly as cpd_iterate would; only the
M-step products of up to 8 scenes share one pass over the eigenbasis (one
streaming kernel with 3 S right-hand sides).  Every scene's T and sigma2 must
equal an independent single-scene registration's up to the summation order
of those products, and the FP64 oracle's at the FP32 tolerance.
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


def test_shared_registrations_need_a_plain_fp32_context():
    X = datagen.gen(200, seed=53).X.astype(np.float32)
    Y = f32dev(datagen.gen(200, seed=54).Y)
    for kw in (dict(precision=cpd.MIXED), dict(precision=cpd.FP32, flags=cpd.FLAG_PRUNE),
               dict(precision=cpd.FP32, flags=cpd.FLAG_SPECTRAL_TRIM)):
        with cpd.Context(f32dev(X), **kw) as ctx:
            if kw.get("flags") == cpd.FLAG_SPECTRAL_TRIM and ctx.trim_info()[0] == 0:
                continue                                   # nothing trimmed: a plain context
            with pytest.raises(cpd.CpdError) as ei:
                ctx.iterate_shared([Y], 3)
            assert ei.value.status == cpd.EINVAL
