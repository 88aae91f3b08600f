"""Pass B in row pieces beside the projection (FCPD_SPLIT_B pieces), against
the FP64 oracle.

Each piece of model rows runs pass B, its row reduction and its log-domain
fix-up; the projection U^T R of the rows a piece finished starts on a side
stream while the next piece's pass B runs, and the diagonal update sums all
pieces' partials.  The arithmetic per row is that of the whole pass B; only
the split of the scene points into partial sums differs (each piece fills
the GPU on its own), so T is held to the FP32 figure against the oracle,
and it differs from the unsplit path's T in the low bits only -- which also
shows that the split path ran.  Model sizes span several pass B row tiles
(2048 rows each) so that 2 and 3 pieces are possible."""
import numpy as np
import pytest

import oracle
from paper_2006_06281_gb300 import cpd, datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_06281_gb300 import build
    build.build()
    cpd.load()


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def rel(a, b):
    a = a.double().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def sig_err(got, ref):
    got, ref = np.atleast_1d(np.asarray(got, np.float64)), np.atleast_1d(np.asarray(ref, np.float64))
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


def run(monkeypatch, pieces, X, Y, n_iter, **kw):
    monkeypatch.setenv("FCPD_SPLIT_B", str(pieces))
    with cpd.Context(dev(X), precision=cpd.FP32, **kw) as ctx:     # the split is planned here
        assert ctx.pass_b_pieces() == pieces
        T, s2, it = ctx.iterate(dev(Y), n_iter)
        hist = ctx.history(it)
    return T, s2, it, hist


@pytest.mark.parametrize("pieces", [2, 3])
def test_register_in_pieces_against_the_oracle(monkeypatch, pieces):
    cfg = datagen.WORKLOADS["fp32_m5000"]
    ps = datagen.gen(cfg["M"], amp=cfg["amp"], noise=0.01, seed=cfg["seed"])
    X, Y = ps.X.astype(np.float32), ps.Y.astype(np.float32)
    ref = oracle.register(X, Y, w=cfg["omega"], beta=cfg["beta"], lam_reg=cfg["lam"], n_iter=cfg["iters"])
    kw = dict(w=cfg["omega"], beta=cfg["beta"], lam=cfg["lam"])
    T, s2, it, hist = run(monkeypatch, pieces, X, Y, cfg["iters"], **kw)
    T1, _, _, _ = run(monkeypatch, 1, X, Y, cfg["iters"], **kw)
    assert it == cfg["iters"]
    e, e1, d = rel(T, ref["T"]), rel(T1, ref["T"]), rel(T, T1.double().cpu().numpy())
    es = sig_err(hist["sigma2"], ref["sigma2_hist"])
    print(f"[pieces {pieces}] T relative error {e:.2e} (unsplit {e1:.2e}; split vs unsplit {d:.2e}); "
          f"sigma2 history {es:.2e}")
    assert e <= FP32_TOL and es <= FP32_TOL
    assert sig_err(s2, ref["sigma2"]) <= FP32_TOL
    assert 0.0 < d <= FP32_TOL           # the split ran (other partial sums) and agrees


@pytest.mark.parametrize("pieces", [2, 3])
def test_log_domain_fixups_in_several_pieces(monkeypatch, pieces):
    """Model rows whose FP32 mass flushes to zero in the first iteration (no
    outlier term, a small initial variance, model points beyond the scene's
    -x face) at the start and at the end of the row order, so that the first
    and the last piece each fix up their own rows -- and only theirs."""
    ps = datagen.gen(4480, amp=0.15, noise=0.01, seed=78)
    rng = np.random.default_rng(6)
    yo = np.column_stack([np.full(25, 1.3), rng.uniform(-0.8, 0.8, 25), rng.uniform(-0.8, 0.8, 25)])
    xo = np.column_stack([np.full(16, -1.3), rng.uniform(-0.8, 0.8, 16), rng.uniform(-0.8, 0.8, 16)])
    X = np.vstack([xo[:8], ps.X, xo[8:]]).astype(np.float32).astype(np.float64)
    Y = np.vstack([ps.Y, yo]).astype(np.float32).astype(np.float64)
    assert X.shape[0] > 2 * 2048
    ref = oracle.register(X, Y, w=0.0, beta=2.0, lam_reg=2.0, n_iter=10, sigma2_0=2e-4)
    assert ref["status"] == oracle.OK
    T, s2, it, _ = run(monkeypatch, pieces, X, Y, 10, w=0.0, beta=2.0, lam=2.0, sigma2_init=2e-4)
    assert it == 10
    e = rel(T, ref["T"])
    print(f"[pieces {pieces}, fix-ups] T relative error {e:.2e}, sigma2 {sig_err(s2, ref['sigma2']):.2e}")
    assert e <= FP32_TOL
    assert sig_err(s2, ref["sigma2"]) <= FP32_TOL


def test_default_piece_count(monkeypatch):
    """Without FCPD_SPLIT_B: 3 pieces for a wide FP32 basis from 8192 model
    points, one below that, for narrow bases and in the other modes."""
    monkeypatch.delenv("FCPD_SPLIT_B", raising=False)
    cases = [(9000, 0, cpd.FP32, 3), (5000, 0, cpd.FP32, 1), (9000, 200, cpd.FP32, 1), (9000, 0, cpd.MIXED, 1)]
    for M, K, prec, want in cases:
        X = datagen.gen(M, seed=3).X.astype(np.float32)
        with cpd.Context(dev(X), precision=prec, K=K) as ctx:
            assert ctx.pass_b_pieces() == want, (M, K, prec)


def test_device_loop_in_pieces_stops_where_the_fixed_count_path_would(monkeypatch):
    """The device-side loop (tolerance set) with pass B in pieces: the same
    stop and bit for bit the T of the fixed-count path in pieces."""
    monkeypatch.setenv("FCPD_SPLIT_B", "2")
    ps = datagen.gen(4500, amp=0.15, noise=0.01, seed=19)
    X, Y = dev(ps.X), dev(ps.Y)
    with cpd.Context(X, precision=cpd.FP32) as ctx:
        ctx.set_ground_truth(dev(ps.Yhat), 8e-3)
        T_tol, _, it = ctx.iterate(Y, 300)
        h = ctx.history(it)
    assert 3 < it < 300 and h["rmse"][-1] <= 8e-3 and np.all(h["rmse"][:-1] > 8e-3)
    with cpd.Context(X, precision=cpd.FP32) as ref:
        T_fixed, _, itf = ref.iterate(Y, it)
    assert itf == it
    assert torch.equal(T_tol, T_fixed)
