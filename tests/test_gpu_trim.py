"""Spectral trim of the M-step (CPD_FLAG_SPECTRAL_TRIM, GPU).

In the full eigenbasis (Eq. 17), direction k enters T through
s_k (U^T R)_k with s_k = l_k / (l_k + lambda sigma2).  The trimmed M-step
keeps the leading k_cap directions and runs only while every dropped one has
s_k < 2^-24; the dropped part of T then has norm <= 2^-24 |R|, so T and
sigma2 must agree with the full M-step to FP32 rounding, and with the FP64
oracle to the FP32 tolerance.
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


def run(X, Y, iters, flags=0, precision=cpd.FP32, K=0, want_W=False):
    with cpd.Context(f32dev(X), precision=precision, K=K, flags=flags) as c:
        T, s2, it = c.iterate(f32dev(Y), iters)
        info = c.trim_info()
        hist = c.history(it)
        W = c.W().cpu().numpy().astype(np.float64) if want_W else None
    return T.cpu().numpy().astype(np.float64), s2, it, info, hist, W


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def scene():
    return datagen.gen(2000, n_out=200, amp=0.15, noise=0.01, seed=31)


def test_trimmed_registration_equals_the_full_one(scene):
    iters = 60
    T, s2, it, (k_cap, n_trim), h, _ = run(scene.X, scene.Y, iters, cpd.FLAG_SPECTRAL_TRIM)
    Tf, s2f, _, (k_full, n_full), hf, _ = run(scene.X, scene.Y, iters)
    assert k_full == 0 and n_full == 0
    print(f"k_cap {k_cap} of {scene.X.shape[0]}; trimmed iterations {n_trim} of {it}")
    assert 0 < k_cap < scene.X.shape[0] // 4
    assert n_trim == iters          # sigma2 stays above the floor throughout
    assert rel(T, Tf) <= 5e-6
    assert abs(s2 - s2f) <= 1e-5 * s2f
    np.testing.assert_allclose(h["sigma2"], hf["sigma2"], rtol=1e-5)


def test_trimmed_registration_against_the_oracle():
    ps = datagen.gen(1200, n_out=0, amp=0.15, noise=0.01, seed=32)
    X, Y = ps.X.astype(np.float32), ps.Y.astype(np.float32)
    ref = oracle.register(X.astype(np.float64), Y.astype(np.float64), w=0.1, beta=2.0, lam_reg=2.0, n_iter=40)
    assert ref["status"] == oracle.OK
    T, s2, it, (k_cap, n_trim), _, _ = run(X, Y, 40, cpd.FLAG_SPECTRAL_TRIM)
    assert k_cap > 0 and n_trim == 40
    assert rel(T, ref["T"]) <= 1e-4
    assert abs(s2 - ref["sigma2"]) <= 1e-4 * ref["sigma2"]


def test_below_the_variance_floor_the_full_mstep_runs():
    # a scene with little noise: sigma2 falls below the trim floor (1e-4 x the
    # model's variance per axis); from the iteration whose sigma2 makes the
    # largest dropped eigenvalue's s_k reach 2^-24 on, the full M-step runs --
    # the switch happens on the device inside one captured graph
    ps = datagen.gen(1500, n_out=0, amp=0.05, noise=1e-3, seed=33)
    iters, lam_reg, eps = 80, 2.0, 2.0 ** -24
    with cpd.Context(f32dev(ps.X), precision=cpd.FP32, flags=cpd.FLAG_SPECTRAL_TRIM) as c:
        _, lam = c.basis()
        T, s2, it = c.iterate(f32dev(ps.Y), iters)
        k_cap, n_trim = c.trim_info()
        h = c.history(it)
    T = T.cpu().numpy().astype(np.float64)
    Tf, s2f, _, _, hf, _ = run(ps.X, ps.Y, iters)
    # the sigma2 each iteration's M-step used: sigma2_0, then the history
    s2_in = np.concatenate([[oracle.sigma2_init(ps.X.astype(np.float32).astype(np.float64),
                                                ps.Y.astype(np.float32).astype(np.float64))], h["sigma2"][:-1]])
    l_drop = float(lam[k_cap])
    pred = int((l_drop < eps * (l_drop + lam_reg * s2_in)).sum())
    print(f"k_cap {k_cap}; trimmed {n_trim} of {iters}; predicted {pred}")
    assert k_cap > 0 and 0 < n_trim < iters
    assert abs(n_trim - pred) <= 1
    assert rel(T, Tf) <= 5e-6
    np.testing.assert_allclose(h["sigma2"], hf["sigma2"], rtol=1e-4)


def test_trim_in_mixed_precision_and_top_k(scene):
    T, s2, _, (k_cap, n_trim), _, _ = run(scene.X, scene.Y, 40, cpd.FLAG_SPECTRAL_TRIM, precision=cpd.MIXED)
    Tf, s2f, _, _, _, _ = run(scene.X, scene.Y, 40, precision=cpd.MIXED)
    assert k_cap > 0 and n_trim == 40
    assert rel(T, Tf) <= 5e-6
    # top-K basis larger than k_cap: trimmed to k_cap; smaller: unchanged
    Tk, _, _, (kk, nk), _, _ = run(scene.X, scene.Y, 40, cpd.FLAG_SPECTRAL_TRIM, K=1000)
    Tkf, _, _, _, _, _ = run(scene.X, scene.Y, 40, K=1000)
    assert kk == k_cap and nk == 40 and rel(Tk, Tkf) <= 5e-6
    _, _, _, (k64, n64), _, _ = run(scene.X, scene.Y, 5, cpd.FLAG_SPECTRAL_TRIM, K=64)
    assert k64 == 0 and n64 == 0


def test_trimmed_W_keeps_phi_W():
    ps = datagen.gen(600, seed=5)
    X = ps.X.astype(np.float64)
    T, _, _, (k_cap, n_trim), _, W = run(ps.X, ps.Y, 30, cpd.FLAG_SPECTRAL_TRIM, want_W=True)
    Tf, _, _, _, _, Wf = run(ps.X, ps.Y, 30, want_W=True)
    assert k_cap > 0 and n_trim == 30
    d2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    Phi = np.exp(-d2 / 8.0)
    # Phi W = T - X (Eq. 17) for both; W itself differs in the dropped
    # directions, where it is ill-posed (the full W is dominated by them)
    ref = Phi @ Wf
    tol = 1e-3 * np.abs(ref).max()
    np.testing.assert_allclose(Phi @ W, ref, rtol=0, atol=tol)
    np.testing.assert_allclose(Phi @ W, T - X, rtol=0, atol=tol)
    assert np.linalg.norm(W) < np.linalg.norm(Wf)


@pytest.mark.parametrize("M,N", [(129, 1025), (1025, 129), (2049, 2047)])
def test_trim_on_ragged_sizes(M, N):
    ps = datagen.gen(M, n_out=max(N - M, 0), n_in=min(M, N), amp=0.15, noise=0.01, seed=13 * M + N)
    T, s2, it, (k_cap, n_trim), _, _ = run(ps.X, ps.Y, 25, cpd.FLAG_SPECTRAL_TRIM)
    Tf, s2f, _, _, _, _ = run(ps.X, ps.Y, 25)
    assert it == 25
    assert (k_cap == 0 and n_trim == 0) or (0 < k_cap < M and n_trim > 0)
    assert rel(T, Tf) <= 5e-6
    assert abs(s2 - s2f) <= 1e-5 * s2f
