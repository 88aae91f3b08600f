"""Thin ctypes binding of the fast-CPD C ABI (include/fcpd.h).

Argument marshalling only: every step of the EM loop runs in libfcpd.so's
sm_103a kernels.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays;
outputs follow the inputs (CUDA tensors in, CUDA tensors out; host arrays in,
numpy arrays out).  There is no CPU fallback: if the library has not been
built, the first call raises.

Names follow the paper (Fast Coherent Point Drift, arXiv 2006.06281):
X model points (they move), Y scene points, T = X + Phi W, w outlier
weight, beta kernel width, lam the regularisation weight lambda.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfcpd.so")

FP64, FP32, MIXED = 0, 1, 2    # MIXED: FP32 points and E-step, FP16 eigenbasis
STATUS = {0: "CPD_OK", 1: "CPD_EINVAL", 2: "CPD_ENOMEM", 3: "CPD_ECUDA", 4: "CPD_ESOLVER",
          5: "CPD_ENUMERIC", 6: "CPD_ETIMEOUT", 7: "CPD_ESTATE"}
OK, EINVAL, ENOMEM, ECUDA, ESOLVER, ENUMERIC, ETIMEOUT, ESTATE = range(8)
FLAG_PRUNE, FLAG_PRUNE_ALWAYS, FLAG_PRUNE_NOSKIP, FLAG_SPECTRAL_TRIM, FLAG_FULL_EIG = 1, 2, 4, 8, 16

# Every symbol include/fcpd.h declares (checked by the tests).
EXPORTS = ["cpd_abi_version", "cpd_status_string", "cpd_last_error", "cpd_params_default",
           "cpd_setup", "cpd_iterate", "cpd_iterate_profiled", "cpd_reset", "cpd_set_ground_truth", "cpd_get_state",
           "cpd_get_history", "cpd_get_W", "cpd_get_basis", "cpd_basis_rank", "cpd_eig_info", "cpd_mstep",
           "cpd_estep", "cpd_estep_noalloc", "cpd_register", "cpd_get_work", "cpd_spatial_order", "cpd_get_trim", "cpd_pass_b_pieces", "cpd_iterate_shared", "cpd_destroy",
           "cpd_coefficients", "cpd_coefficients_of", "cpd_warm_start", "cpd_net_create", "cpd_net_create_ex",
           "cpd_net_precision", "cpd_net_num_params", "cpd_net_get_params", "cpd_net_set_params", "cpd_net_forward", "cpd_net_gradients", "cpd_net_train_step", "cpd_net_destroy",
           "cpd_batch_create", "cpd_batch_iterate", "cpd_batch_state", "cpd_batch_get_T", "cpd_batch_info",
           "cpd_batch_launch_shape", "cpd_batch_phase_ms", "cpd_batch_reset", "cpd_batch_autotune",
           "cpd_batch_destroy"]


class CpdParams(C.Structure):
    _fields_ = [("D", C.c_int32), ("precision", C.c_int32), ("w", C.c_double), ("beta", C.c_double),
                ("lam", C.c_double), ("sigma2_init", C.c_double), ("K", C.c_int64),
                ("max_iter", C.c_int32), ("flags", C.c_int32), ("tol", C.c_double)]


class CpdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def load():
    """Load libfcpd.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = C.CDLL(LIB_PATH)
            vp, i64, i32, d, dp = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int32)
            pp = C.POINTER(CpdParams)
            sig = {
                "cpd_abi_version": ([], i32),
                "cpd_status_string": ([C.c_int], C.c_char_p),
                "cpd_last_error": ([], C.c_char_p),
                "cpd_params_default": ([pp], None),
                "cpd_setup": ([vp, i64, pp, vp, C.POINTER(vp)], C.c_int),
                "cpd_iterate": ([vp, vp, i64, i32, vp, dp, ip], C.c_int),
                "cpd_iterate_profiled": ([vp, vp, i64, i32, C.POINTER(C.c_float)], C.c_int),
                "cpd_reset": ([vp], C.c_int),
                "cpd_set_ground_truth": ([vp, vp, d], C.c_int),
                "cpd_get_state": ([vp, dp, ip, ip], C.c_int),
                "cpd_get_history": ([vp, i32, vp, vp, vp], C.c_int),
                "cpd_get_W": ([vp, vp], C.c_int),
                "cpd_get_basis": ([vp, vp, vp], C.c_int),
                "cpd_basis_rank": ([vp], i64),
                "cpd_eig_info": ([vp, ip, ip], C.c_int),
                "cpd_mstep": ([vp, vp, d, vp, vp], C.c_int),
                "cpd_estep": ([vp, i64, vp, i64, i32, d, d, vp, vp, vp, dp, vp], C.c_int),
                "cpd_estep_noalloc": ([vp, i64, vp, i64, d, d, vp, vp, vp, dp, vp], C.c_int),
                "cpd_register": ([vp, i64, vp, i64, pp, vp, vp, vp, dp, ip], C.c_int),
                "cpd_destroy": ([vp], None),
                "cpd_get_work": ([vp, i32, vp], C.c_int),
                "cpd_get_trim": ([vp, C.POINTER(i64), C.POINTER(i32)], C.c_int),
                "cpd_pass_b_pieces": ([vp, C.POINTER(i32)], C.c_int),
                "cpd_iterate_shared": ([vp, i32, C.POINTER(vp), C.POINTER(i64), i32, C.POINTER(vp), dp], C.c_int),
                "cpd_coefficients": ([vp, i32, vp], C.c_int),
                "cpd_coefficients_of": ([vp, i32, vp, vp], C.c_int),
                "cpd_warm_start": ([vp, i32, vp, d], C.c_int),
                "cpd_net_create": ([i32, i32, i32, C.c_uint64, vp, C.POINTER(vp)], C.c_int),
                "cpd_net_create_ex": ([i32, i32, i32, C.c_uint64, i32, vp, C.POINTER(vp)], C.c_int),
                "cpd_net_precision": ([vp], i32),
                "cpd_net_num_params": ([vp], i64),
                "cpd_net_get_params": ([vp, vp], C.c_int),
                "cpd_net_set_params": ([vp, vp], C.c_int),
                "cpd_net_forward": ([vp, vp, i32, vp], C.c_int),
                "cpd_net_gradients": ([vp, vp, vp, i32, vp, vp], C.c_int),
                "cpd_net_train_step": ([vp, vp, vp, i32, C.c_float, vp], C.c_int),
                "cpd_net_destroy": ([vp], None),
                "cpd_spatial_order": ([vp], i32),
                "cpd_batch_create": ([i32, C.POINTER(vp), C.POINTER(i64), C.POINTER(vp), C.POINTER(i64), pp, d, vp,
                                      C.POINTER(vp)], C.c_int),
                "cpd_batch_iterate": ([vp, i32], C.c_int),
                "cpd_batch_state": ([vp, dp, ip, ip], C.c_int),
                "cpd_batch_get_T": ([vp, i32, vp], C.c_int),
                "cpd_batch_info": ([vp, i32, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)], C.c_int),
                "cpd_batch_launch_shape": ([vp, ip, ip, ip], C.c_int),
                "cpd_batch_phase_ms": ([vp, C.POINTER(C.c_float)], C.c_int),
                "cpd_batch_reset": ([vp], C.c_int),
                "cpd_batch_autotune": ([vp, i32, ip, ip, C.POINTER(C.c_float)], C.c_int),
                "cpd_batch_destroy": ([vp], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _check(status: int):
    if status != OK:
        msg = load().cpd_last_error().decode()
        raise CpdError(status, msg)


# ----------------------------------------------------------------- marshalling
def _is_torch(a):
    try:
        import torch
        return isinstance(a, torch.Tensor)
    except ImportError:
        return False


def _dtype_of(precision):
    return np.float64 if precision == FP64 else np.float32


def _prep(a, precision, name):
    """Returns (object kept alive, pointer, is_cuda)."""
    want = _dtype_of(precision)
    if _is_torch(a):
        import torch
        td = torch.float64 if precision == FP64 else torch.float32
        if a.dtype != td:
            raise TypeError(f"{name}: expected {td}, got {a.dtype}")
        a = a.contiguous()
        return a, a.data_ptr(), a.is_cuda
    arr = np.ascontiguousarray(a, dtype=want)
    return arr, arr.ctypes.data, False


def _out_like(n, cols, precision, cuda, device=None):
    if cuda:
        import torch
        td = torch.float64 if precision == FP64 else torch.float32
        t = torch.empty((n, cols), dtype=td, device=device)
        return t, t.data_ptr()
    arr = np.empty((n, cols), dtype=_dtype_of(precision))
    return arr, arr.ctypes.data


def _stream_handle(stream, cuda):
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    if cuda:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    return 0


def make_params(precision=FP32, w=0.1, beta=2.0, lam=2.0, K=0, max_iter=50, tol=0.0,
                sigma2_init=0.0, flags=0) -> CpdParams:
    p = CpdParams()
    load().cpd_params_default(C.byref(p))
    p.precision, p.w, p.beta, p.lam, p.K = int(precision), float(w), float(beta), float(lam), int(K)
    p.max_iter, p.tol, p.sigma2_init, p.flags = int(max_iter), float(tol), float(sigma2_init), int(flags)
    return p


class Context:
    """A registration context: setup (Gram matrix + eigendecomposition) once,
    then EM iterations against one or more scenes."""

    def __init__(self, X, precision=FP32, w=0.1, beta=2.0, lam=2.0, K=0, tol=0.0, sigma2_init=0.0,
                 stream=None, flags=0):
        lib = load()
        self.precision = precision
        self._X, px, self.cuda = _prep(X, precision, "X")
        self.device = self._X.device if self.cuda else None
        self.M = int(self._X.shape[0])
        self.stream = _stream_handle(stream, self.cuda)
        self.params = make_params(precision, w, beta, lam, K, 0, tol, sigma2_init, flags)
        h = C.c_void_p()
        _check(lib.cpd_setup(px, self.M, C.byref(self.params), self.stream, C.byref(h)))
        self._h = h
        self.K = int(lib.cpd_basis_rank(h))
        self.spatial_order = bool(lib.cpd_spatial_order(h))

    def iterate(self, Y, n_iter, want_T=True):
        """Runs n_iter EM iterations; returns (T or None, sigma2, iterations so far)."""
        Yk, py, ycuda = _prep(Y, self.precision, "Y")
        T, pt = _out_like(self.M, 3, self.precision, ycuda, self.device) if want_T else (None, None)
        s2, it = C.c_double(0), C.c_int32(0)
        _check(load().cpd_iterate(self._h, py, int(Yk.shape[0]), int(n_iter), pt, C.byref(s2), C.byref(it)))
        return T, s2.value, it.value

    def iterate_shared(self, Ys, n_iter):
        """Registers each scene of Ys against this context's model (fresh,
        n_iter iterations each; the M-step products of up to 8 scenes share
        one pass over the basis).  Returns [(T, sigma2)] in the order of Ys."""
        n = len(Ys)
        keep = [_prep(Y, self.precision, f"Ys[{i}]") for i, Y in enumerate(Ys)]
        outs = [_out_like(self.M, 3, self.precision, k[2], self.device) for k in keep]
        ys = (C.c_void_p * n)(*[k[1] for k in keep])
        ns = (C.c_int64 * n)(*[int(k[0].shape[0]) for k in keep])
        ts = (C.c_void_p * n)(*[o[1] for o in outs])
        s2 = (C.c_double * n)()
        _check(load().cpd_iterate_shared(self._h, n, ys, ns, int(n_iter), ts, s2))
        return [(outs[i][0], s2[i]) for i in range(n)]

    def iterate_into(self, Y, n_iter, T_out):
        """Runs n_iter iterations writing T into the caller's buffer T_out
        (host or device); returns (sigma2, iterations so far)."""
        Yk, py, _ = _prep(Y, self.precision, "Y")
        _, pt, _ = _prep(T_out, self.precision, "T_out")
        s2, it = C.c_double(0), C.c_int32(0)
        _check(load().cpd_iterate(self._h, py, int(Yk.shape[0]), int(n_iter), pt, C.byref(s2), C.byref(it)))
        return s2.value, it.value

    def iterate_profiled(self, Y, n_iter):
        """n_iter iterations from a graph with timing events after every
        kernel; returns the 9 phase times (ms) described in fcpd.h."""
        Yk, py, _ = _prep(Y, self.precision, "Y")
        out = (C.c_float * 9)()
        _check(load().cpd_iterate_profiled(self._h, py, int(Yk.shape[0]), int(n_iter), out))
        return list(out)

    def iterate_async(self, Y, n_iter, T_out=None):
        """Enqueues n_iter iterations without synchronising (device arrays only)."""
        Yk, py, _ = _prep(Y, self.precision, "Y")
        pt = None
        if T_out is not None:
            _, pt, _ = _prep(T_out, self.precision, "T_out")
        _check(load().cpd_iterate(self._h, py, int(Yk.shape[0]), int(n_iter), pt, None, None))

    def reset(self):
        _check(load().cpd_reset(self._h))

    def set_ground_truth(self, Yhat, rmse_tol=0.0):
        if Yhat is None:
            _check(load().cpd_set_ground_truth(self._h, None, float(rmse_tol)))
            return
        self._gt, p, _ = _prep(Yhat, self.precision, "Yhat")
        _check(load().cpd_set_ground_truth(self._h, p, float(rmse_tol)))

    def state(self):
        s2, it, ds = C.c_double(0), C.c_int32(0), C.c_int32(0)
        _check(load().cpd_get_state(self._h, C.byref(s2), C.byref(it), C.byref(ds)))
        return s2.value, it.value, ds.value

    def history(self, n):
        a, b, c = np.empty(n), np.empty(n), np.empty(n)
        _check(load().cpd_get_history(self._h, int(n), a.ctypes.data, b.ctypes.data, c.ctypes.data))
        return dict(sigma2=a, loglik=b, rmse=c)

    def W(self):
        W, pw = _out_like(self.M, 3, self.precision, self.cuda, self.device)
        _check(load().cpd_get_W(self._h, pw))
        return W

    def eig_info(self):
        """(method, steps): 0 = dense eigensolver, 1 = top-K subspace
        iteration, and the subspace iteration's Rayleigh-Ritz steps."""
        m, n = C.c_int32(), C.c_int32()
        _check(load().cpd_eig_info(self._h, C.byref(m), C.byref(n)))
        return m.value, n.value

    def trim_info(self):
        """(k_cap, trimmed_iters): directions kept by the spectral trim (0: none)
        and iterations of this registration that ran the trimmed M-step."""
        k = C.c_int64()
        n = C.c_int32()
        _check(load().cpd_get_trim(self._h, C.byref(k), C.byref(n)))
        return k.value, n.value

    def pass_b_pieces(self):
        """Row pieces pass B runs in (1: one launch; > 1: each piece's
        projection overlaps the next piece's pass B)."""
        n = C.c_int32()
        _check(load().cpd_pass_b_pieces(self._h, C.byref(n)))
        return n.value

    def work(self, n):
        """Fraction of the 2 M N Gaussian pairs evaluated by each of the first n iterations."""
        out = np.empty(n)
        _check(load().cpd_get_work(self._h, int(n), out.ctypes.data))
        return out

    def coefficients(self, n_coef):
        """U[:, :n_coef]^T (T - X) of the current T (n_coef x 3, numpy)."""
        out = np.empty((int(n_coef), 3), dtype=np.float32)
        _check(load().cpd_coefficients(self._h, int(n_coef), out.ctypes.data))
        return out

    def coefficients_of(self, T, n_coef):
        """U[:, :n_coef]^T (T - X) of a given T (n_coef x 3, numpy)."""
        _, pt, _ = _prep(T, self.precision, "T")
        out = np.empty((int(n_coef), 3), dtype=np.float32)
        _check(load().cpd_coefficients_of(self._h, int(n_coef), pt, out.ctypes.data))
        return out

    def warm_start(self, coef, sigma2_0):
        """Next registration starts at T = X + U[:, :n] coef with variance sigma2_0."""
        c = np.ascontiguousarray(coef, dtype=np.float32).reshape(-1, 3)
        _check(load().cpd_warm_start(self._h, int(c.shape[0]), c.ctypes.data, float(sigma2_0)))

    def basis(self):
        U = np.empty((self.M, self.K), dtype=_dtype_of(self.precision))
        lam = np.empty(self.K)
        _check(load().cpd_get_basis(self._h, U.ctypes.data, lam.ctypes.data))
        return U, lam

    def mstep(self, Ytil, sigma2, want_W=False):
        Yk, py, ycuda = _prep(Ytil, self.precision, "Ytil")
        T, pt = _out_like(self.M, 3, self.precision, ycuda, self.device)
        W, pw = _out_like(self.M, 3, self.precision, ycuda, self.device) if want_W else (None, None)
        _check(load().cpd_mstep(self._h, py, float(sigma2), pt, pw))
        return (T, W) if want_W else T

    def close(self):
        if getattr(self, "_h", None):
            load().cpd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many independent registrations (X_i, Y_i) advanced together by one
    persistent kernel launch per `iterate` call (cpd_batch_*).  Points are
    FP32; precision MIXED stores the eigenbasis in FP16."""

    def __init__(self, Xs, Ys, w=0.1, beta=2.0, lam=2.0, K=0, tol=0.0, sigma2_init=0.0,
                 barrier_timeout_s=0.0, stream=None, precision=FP32):
        lib = load()
        if len(Xs) != len(Ys) or not Xs:
            raise ValueError("Xs and Ys must be non-empty lists of equal length")
        n = len(Xs)
        self._keep = []
        px, py = (C.c_void_p * n)(), (C.c_void_p * n)()
        M, N = (C.c_int64 * n)(), (C.c_int64 * n)()
        cuda = False
        for i, (X, Y) in enumerate(zip(Xs, Ys)):
            xk, xp, xc = _prep(X, FP32, f"X[{i}]")
            yk, yp, _ = _prep(Y, FP32, f"Y[{i}]")
            self._keep += [xk, yk]
            px[i], py[i], M[i], N[i] = xp, yp, int(xk.shape[0]), int(yk.shape[0])
            cuda = cuda or xc
        self.n = n
        self.M, self.N = list(M), list(N)
        self.stream = _stream_handle(stream, True)
        self.params = make_params(precision, w, beta, lam, K, 0, tol, sigma2_init)
        h = C.c_void_p()
        _check(lib.cpd_batch_create(n, px, M, py, N, C.byref(self.params), float(barrier_timeout_s), self.stream,
                                    C.byref(h)))
        self._h = h
        self._keep = []                  # the library holds its own copies
        self.K = []
        for i in range(n):
            k = C.c_int64()
            _check(lib.cpd_batch_info(h, i, None, None, C.byref(k)))
            self.K.append(k.value)

    def iterate(self, n_iter):
        _check(load().cpd_batch_iterate(self._h, int(n_iter)))

    def state(self):
        """(sigma2 array, iterations array, device status array) of all pairs."""
        s2 = np.empty(self.n)
        it = np.empty(self.n, dtype=np.int32)
        stt = np.empty(self.n, dtype=np.int32)
        _check(load().cpd_batch_state(self._h, s2.ctypes.data_as(C.POINTER(C.c_double)),
                                      it.ctypes.data_as(C.POINTER(C.c_int32)),
                                      stt.ctypes.data_as(C.POINTER(C.c_int32))))
        return s2, it, stt

    def T(self, i, device=None):
        """T of pair i (numpy, or a CUDA tensor on `device`)."""
        if device is not None:
            import torch
            out = torch.empty((self.M[i], 3), dtype=torch.float32, device=device)
            _check(load().cpd_batch_get_T(self._h, int(i), out.data_ptr()))
            torch.cuda.synchronize(device)
            return out
        out = np.empty((self.M[i], 3), dtype=np.float32)
        _check(load().cpd_batch_get_T(self._h, int(i), out.ctypes.data))
        return out

    def launch_shape(self):
        """(pairs, grid blocks, work items per iteration)."""
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().cpd_batch_launch_shape(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def phase_ms(self):
        """Milliseconds of GPU time per iteration inside the 4 phases' work
        items in the last call: pass A (+ column reduction), pass B (+ row
        reduction), projection (+ diagonal update), expansion (+ T and Eq.
        18).  Phases of different pairs overlap."""
        return self.phase_profile()[0]

    def phase_profile(self):
        """(GPU ms per iteration inside the 4 phases' items, fraction of the
        blocks' time on each phase's items spent working rather than waiting
        for the pair's previous phase) for the last call."""
        out = (C.c_float * 8)()
        _check(load().cpd_batch_phase_ms(self._h, out))
        return list(out[:4]), list(out[4:])

    def reset(self):
        _check(load().cpd_batch_reset(self._h))

    def autotune(self, n_iter=3):
        """Times eight work-item plans, keeps the fastest (registrations restart).
        Returns (e_items, proj_kb, ms per candidate)."""
        e, p = C.c_int32(), C.c_int32()
        ms = (C.c_float * 8)()
        _check(load().cpd_batch_autotune(self._h, int(n_iter), C.byref(e), C.byref(p), ms))
        return e.value, p.value, list(ms)

    def close(self):
        if getattr(self, "_h", None):
            load().cpd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def estep(T, Y, sigma2, w, precision=FP32, stream=None):
    """One E-step (Eq. 4 + Eq. 5).  Returns dict(Ytil, P1, den, vsum, loglik)."""
    Tk, pt, tcuda = _prep(T, precision, "T")
    Yk, py, _ = _prep(Y, precision, "Y")
    M, N = int(Tk.shape[0]), int(Yk.shape[0])
    dev = Tk.device if tcuda else None
    Ytil, pyt = _out_like(M, 3, precision, tcuda, dev)
    if tcuda:
        import torch
        P1 = torch.empty(M, dtype=torch.float64, device=dev)
        den = torch.empty(N, dtype=torch.float64, device=dev)
        pp1, pden = P1.data_ptr(), den.data_ptr()
    else:
        P1, den = np.empty(M), np.empty(N)
        pp1, pden = P1.ctypes.data, den.ctypes.data
    sums = (C.c_double * 2)()
    _check(load().cpd_estep(pt, M, py, N, int(precision), float(sigma2), float(w), pyt, pp1, pden, sums,
                            _stream_handle(stream, tcuda)))
    return dict(Ytil=Ytil, P1=P1, den=den, vsum=sums[0], loglik=sums[1])


def estep_noalloc(T, Y, sigma2, w, stream=None):
    """cpd_estep_noalloc: the FP32 E-step with no device allocation (CUDA
    tensors of one device only).  The call is made with that device current,
    on its current stream unless `stream` is given.  Returns dict(Ytil, P1,
    den, vsum, loglik) like estep()."""
    import torch
    Tk, pt, tcuda = _prep(T, FP32, "T")
    Yk, py, ycuda = _prep(Y, FP32, "Y")
    if not (tcuda and ycuda):
        raise TypeError("estep_noalloc takes CUDA tensors")
    if Tk.device != Yk.device:
        raise ValueError(f"estep_noalloc: T is on {Tk.device} and Y on {Yk.device}; they must share a device")
    M, N = int(Tk.shape[0]), int(Yk.shape[0])
    with torch.cuda.device(Tk.device):
        Ytil = torch.empty((M, 3), dtype=torch.float32, device=Tk.device)
        P1 = torch.empty(M, dtype=torch.float64, device=Tk.device)
        den = torch.empty(N, dtype=torch.float64, device=Tk.device)
        sums = (C.c_double * 2)()
        _check(load().cpd_estep_noalloc(pt, M, py, N, float(sigma2), float(w), Ytil.data_ptr(), P1.data_ptr(),
                                        den.data_ptr(), sums, _stream_handle(stream, True)))
    return dict(Ytil=Ytil, P1=P1, den=den, vsum=sums[0], loglik=sums[1])


def register(X, Y, precision=FP32, w=0.1, beta=2.0, lam=2.0, K=0, max_iter=50, tol=0.0,
             sigma2_init=0.0, want_W=False, stream=None, flags=0):
    """Whole registration through cpd_register.  Returns (T, W or None, sigma2, iters)."""
    Xk, px, xcuda = _prep(X, precision, "X")
    Yk, py, _ = _prep(Y, precision, "Y")
    M = int(Xk.shape[0])
    dev = Xk.device if xcuda else None
    T, pt = _out_like(M, 3, precision, xcuda, dev)
    W, pw = _out_like(M, 3, precision, xcuda, dev) if want_W else (None, None)
    p = make_params(precision, w, beta, lam, K, max_iter, tol, sigma2_init, flags)
    s2, it = C.c_double(0), C.c_int32(0)
    _check(load().cpd_register(px, M, py, int(Yk.shape[0]), C.byref(p), _stream_handle(stream, xcuda),
                               pt, pw, C.byref(s2), C.byref(it)))
    return T, W, s2.value, it.value
