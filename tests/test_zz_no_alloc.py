"""cpd_estep_noalloc against cpd_estep (GPU).

cpd_estep_noalloc is for callers that cannot allocate device memory when they
need an E-step (loops that must not stall on cudaMalloc/cudaFree, programs
that reserve all device memory up front under a fixed budget): it takes its
scratch from a static device array instead of cudaMalloc.  It must give what
cpd_estep gives, call after call, even though every call reuses the same
array.  This file is collected
last so a failure here does not stop the rest of the suite.
"""
import math

import numpy as np
import pytest

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


def _den_rtol(sigma2):
    # the FP32 E-step tolerance used by the parity tests (see test_gpu_parity)
    q = math.sqrt(1.4426950408889634 / (2 * sigma2))
    return 3e-6 * q + 2e-6


def _case(M, N, seed):
    ps = datagen.gen(M, n_out=max(N - M, 0), n_in=min(M, N), amp=0.15, noise=0.01, seed=seed)
    T = torch.tensor(ps.Yhat, dtype=torch.float32, device="cuda")
    Y = torch.tensor(ps.Y, dtype=torch.float32, device="cuda")
    return T, Y


def _compare(a, b, sigma2):
    np.testing.assert_allclose(b["den"].cpu().numpy(), a["den"].cpu().numpy(), rtol=_den_rtol(sigma2))
    np.testing.assert_allclose(b["P1"].cpu().numpy(), a["P1"].cpu().numpy(), rtol=1e-5,
                               atol=1e-7 * float(a["P1"].max()))
    ya, yb = a["Ytil"].double().cpu().numpy(), b["Ytil"].double().cpu().numpy()
    assert np.linalg.norm(yb - ya) <= 1e-5 * np.linalg.norm(ya)
    assert b["vsum"] == pytest.approx(a["vsum"], rel=1e-5)
    assert b["loglik"] == pytest.approx(a["loglik"], rel=1e-5, abs=1e-3)


def test_two_calls_in_a_row_match_cpd_estep():
    cases = [(3000, 3500, 1e-3, 0.1, 31), (1200, 900, 1e-4, 0.2, 32)]
    for M, N, sigma2, w, seed in cases:      # the second call reuses the array the first one filled
        T, Y = _case(M, N, seed)
        ref = cpd.estep(T, Y, sigma2, w, cpd.FP32)
        got = cpd.estep_noalloc(T, Y, sigma2, w)
        torch.cuda.synchronize()
        _compare(ref, got, sigma2)


def test_rejects_what_it_cannot_hold():
    T, Y = _case(64, 64, 33)
    big = torch.zeros((32769, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(cpd.CpdError) as ei:
        cpd.estep_noalloc(big, Y, 1e-3, 0.1)
    assert ei.value.status == cpd.EINVAL and "32768" in str(ei.value)
    with pytest.raises(TypeError):
        cpd.estep_noalloc(T.cpu(), Y, 1e-3, 0.1)
    # a host array through the C ABI is refused, not staged
    Th = np.ascontiguousarray(T.cpu().numpy())
    out = torch.empty((64, 3), dtype=torch.float32, device="cuda")
    st = cpd.load().cpd_estep_noalloc(Th.ctypes.data, 64, Y.data_ptr(), 64, 1e-3, 0.1, out.data_ptr(), None, None,
                                      None, None)
    assert st == cpd.EINVAL


@pytest.mark.parametrize("M,N", [(32768, 32768), (2048, 32768)])
def test_largest_sizes_fit_and_match_cpd_estep(M, N):
    """The declared limit M, N <= 32768 holds: the widest partial-sum layouts
    fit the static array and give what cpd_estep gives."""
    T, Y = _case(M, N, 34)
    sigma2 = 2e-3
    ref = cpd.estep(T, Y, sigma2, 0.1, cpd.FP32)
    got = cpd.estep_noalloc(T, Y, sigma2, 0.1)
    torch.cuda.synchronize()
    _compare(ref, got, sigma2)


def test_two_streams_one_after_the_other():
    """Each call synchronises its own stream before it returns, so calls on two
    streams made one after the other (not overlapping) both stay correct even
    though they share the array."""
    cases = [(1500, 1700, 1e-3, 0.1, 35), (900, 1300, 3e-4, 0.3, 36)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    refs, outs = [], []
    for (M, N, sigma2, w, seed), st in zip(cases, streams):
        T, Y = _case(M, N, seed)
        refs.append(cpd.estep(T, Y, sigma2, w, cpd.FP32))
        with torch.cuda.stream(st):
            outs.append(cpd.estep_noalloc(T, Y, sigma2, w, stream=st))
    torch.cuda.synchronize()
    for ref, got, (M, N, sigma2, w, seed) in zip(refs, outs, cases):
        _compare(ref, got, sigma2)
