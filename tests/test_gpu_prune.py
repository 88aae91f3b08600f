"""Exact pruning of the FP32 E-step over spatially ordered points (GPU).

With CPD_FLAG_PRUNE an FP32 context keeps its points in Morton order; once
sigma2 is small, the E-step skips tile pairs whose Gaussians are all exactly
0 in FP32.  Skipping
must change nothing: the sums are the same bit for bit as evaluating every
tile pair of the same layout.
"""
import math

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


def run(ps, iters, flags=0, K=0, gt=False):
    with cpd.Context(f32dev(ps.X), precision=cpd.FP32, K=K, flags=flags) as c:
        if gt:
            c.set_ground_truth(f32dev(ps.Yhat), 0.0)
        T, s2, it = c.iterate(f32dev(ps.Y), iters)
        hist = c.history(it)
        work = c.work(it)
        order = c.spatial_order
    return T.cpu().numpy(), s2, hist, work, order


@pytest.fixture(scope="module")
def scene():
    # outliers and missing points make rows/columns of uneven mass
    return datagen.gen(4000, n_out=600, amp=0.15, noise=0.01, seed=21, n_in=3800)


def test_skipping_is_bit_identical_to_evaluating_every_tile(scene):
    T_skip, s2_skip, h_skip, w_skip, order = run(scene, 80, cpd.FLAG_PRUNE_ALWAYS)
    T_all, s2_all, h_all, w_all, _ = run(scene, 80, cpd.FLAG_PRUNE_ALWAYS | cpd.FLAG_PRUNE_NOSKIP)
    assert order
    np.testing.assert_array_equal(T_skip, T_all)
    assert s2_skip == s2_all
    np.testing.assert_array_equal(h_skip["sigma2"], h_all["sigma2"])
    np.testing.assert_array_equal(h_skip["loglik"], h_all["loglik"])
    # the no-skip run evaluates every pair; the skipping run prunes most of
    # them once sigma2 has shrunk
    np.testing.assert_allclose(w_all, 1.0)
    print(f"evaluated fraction: first {w_skip[0]:.3f}, last {w_skip[-1]:.3f}")
    assert w_skip[-1] < 0.6 and w_skip[0] > 0.9


def test_automatic_pruning_against_the_oracle_and_dense_order(scene):
    iters = 80
    X, Y = scene.X.astype(np.float32), scene.Y.astype(np.float32)
    ref = oracle.register(X.astype(np.float64), Y.astype(np.float64), w=0.1, beta=2.0, lam_reg=2.0, n_iter=iters)
    T, s2, hist, work, order = run(scene, iters, cpd.FLAG_PRUNE, gt=True)
    Td, s2d, histd, workd, orderd = run(scene, iters, 0, gt=True)
    assert order and not orderd
    rel = np.linalg.norm(T - ref["T"]) / np.linalg.norm(ref["T"])
    reld = np.linalg.norm(Td - ref["T"]) / np.linalg.norm(ref["T"])
    assert rel <= 1e-4 and reld <= 1e-4
    # the same registration in either order (summation order differs)
    assert np.linalg.norm(T - Td) / np.linalg.norm(Td) <= 2e-5
    np.testing.assert_allclose(hist["rmse"], histd["rmse"], rtol=1e-4)
    np.testing.assert_allclose(workd, 1.0)
    # dense while sigma2 is large, pruned (fraction < 1) once it is small
    assert work[0] == 1.0
    assert work[-1] < 0.6


def test_spatial_order_is_invisible_in_every_output():
    ps = datagen.gen(600, seed=5)
    X = f32dev(ps.X)
    with cpd.Context(X, precision=cpd.FP32, K=50, flags=cpd.FLAG_PRUNE) as c, \
            cpd.Context(X, precision=cpd.FP32, K=50) as cd:
        assert c.spatial_order and not cd.spatial_order
        U, lam = c.basis()
        Ud, lamd = cd.basis()
        # U Lambda U^T against Phi of the caller's points (rows in the caller's order)
        d2 = ((ps.X[:, None, :] - ps.X[None, :, :]) ** 2).sum(-1)
        Phi = np.exp(-d2 / 8.0)
        lo = (U.astype(np.float64) * lam) @ U.astype(np.float64).T
        assert np.abs(lo - Phi).max() <= 2e-3 * np.abs(Phi).max()
        np.testing.assert_allclose(lam, lamd, rtol=1e-9, atol=1e-9 * lamd[0])
        Y = f32dev(ps.Y)
        c.iterate(Y, 5)
        cd.iterate(Y, 5)
        W, Wd = c.W().cpu().numpy(), cd.W().cpu().numpy()
        Yt = f32dev(ps.Yhat)             # any M x 3 array serves as Ytil
        Tm = c.mstep(Yt, 1e-3).cpu().numpy()
        Tmd = cd.mstep(Yt, 1e-3).cpu().numpy()
    # W is dominated by small-eigenvalue directions: compare Phi W (= T - X)
    np.testing.assert_allclose(Phi @ W, Phi @ Wd, rtol=0, atol=1e-3 * np.abs(Phi @ Wd).max())
    np.testing.assert_allclose(Tm, Tmd, rtol=0, atol=2e-5)


# (M = N = 1 collapses sigma2 to 0 within a few iterations; see test_gpu_parity)
@pytest.mark.parametrize("M,N", [(1, 2), (2, 3), (3, 5), (129, 1025), (1025, 129), (2049, 2047)])
def test_pruned_layout_on_ragged_sizes_against_the_oracle(M, N):
    ps = datagen.gen(M, n_out=max(N - M, 0), n_in=min(M, N), amp=0.15, noise=0.01, seed=11 * M + N)
    X, Y = ps.X.astype(np.float32), ps.Y.astype(np.float32)
    if M < 4:
        Y = datagen.gen(max(N, 4), seed=7 * N + 1).Y[:N].astype(np.float32)
    ref = oracle.register(X.astype(np.float64), Y.astype(np.float64), w=0.1, beta=2.0, lam_reg=2.0, n_iter=12)
    assert ref["status"] == oracle.OK
    with cpd.Context(f32dev(X), precision=cpd.FP32, flags=cpd.FLAG_PRUNE_ALWAYS) as c:
        T, s2, it = c.iterate(f32dev(Y), 12)
    T = T.cpu().numpy().astype(np.float64)
    assert it == 12
    assert np.linalg.norm(T - ref["T"]) <= 1e-4 * np.linalg.norm(ref["T"])
