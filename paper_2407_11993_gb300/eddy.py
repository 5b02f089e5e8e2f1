"""Python binding of the C ABI in include/eddy_theta.h (ctypes; marshalling only).

Every step of the theta-method runs in the CUDA library; this module only turns
numpy arrays (host memory) or CUDA torch tensors (device memory) into pointers
and sizes.  Importing it does not load the library; the first call does, and
raises if the compiled library is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int64, c_longlong, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libeddy_theta.so")

EC_FORM_PLAIN, EC_FORM_MODAL = 0, 1
EC_MEM_HOST, EC_MEM_DEVICE = 0, 1
EC_SOLVE_INVERSE, EC_SOLVE_SUBSTITUTION = 0, 1
EC_PREC_FP64, EC_PREC_BF16, EC_PREC_BF16X3 = 0, 1, 2
EC_PREC_FP32 = 3
EC_PREC_FP32X2 = 4
_GEMM = {"tensor": 0, "fp64": 1, "tensor_pairsymv": 2}
_PREC = {"fp64": EC_PREC_FP64, "bf16": EC_PREC_BF16, "bf16x3": EC_PREC_BF16X3, "fp32": EC_PREC_FP32,
         "fp32x2": EC_PREC_FP32X2}

STATUS = {
    0: "EC_OK", 1: "EC_ERR_ARG", 2: "EC_ERR_SHAPE", 3: "EC_ERR_NOT_SPD", 4: "EC_ERR_RANK",
    5: "EC_ERR_OOM", 6: "EC_ERR_CUDA", 7: "EC_ERR_TIMEOUT", 8: "EC_ERR_STATE",
    9: "EC_ERR_NOT_CONVERGED", 10: "EC_ERR_UNSUPPORTED",
}

EXPORTS = ("ec_create", "ec_setup", "ec_set_step", "ec_run", "ec_set_current", "ec_state_size",
           "ec_get_state", "ec_set_state", "ec_get_modes", "ec_timings", "ec_sync",
           "ec_last_info", "ec_error_string", "ec_destroy", "ec_selftest_wait_timeout",
           "ec_launch_count", "ec_solve_z", "ec_get_inverse_factor", "ec_solve_inverse_noalloc",
           "ec_grad", "ec_gemm_bf16", "ec_set_mode_count", "ec_phasors", "ec_batch_run",
           "ec_selftest_fail_alloc", "ec_gemm_f64_emulated", "ec_set_precision")
NOALLOC_MAX_N = 8192


class ec_config(ctypes.Structure):
    _fields_ = [("form", c_int), ("theta", c_double), ("dt", c_double), ("stream", c_void_p),
                ("device", c_int), ("spin_limit", c_longlong), ("profile", c_int),
                ("plain_solver", c_int), ("precision", c_int), ("integrator", c_int),
                ("rhs_mode", c_int), ("refine_steps", c_int), ("tile_variant", c_int),
                ("setup_gemm", c_int), ("release_inputs", c_int)]


class ec_timing(ctypes.Structure):
    _fields_ = [("elim_ms", c_double), ("factor_ms", c_double), ("reduce_ms", c_double),
                ("tridiag_ms", c_double), ("eig_ms", c_double), ("backtransform_ms", c_double),
                ("project_ms", c_double), ("setup_ms", c_double), ("run_ms", c_double),
                ("run_steps", c_int64), ("fwd_ms", c_double), ("bwd_ms", c_double),
                ("scan_ms", c_double), ("fwd_launches", c_int64), ("bwd_launches", c_int64),
                ("scan_launches", c_int64), ("tile_variant", c_int64),
                ("tile_tune_ms", c_double * 4)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["tile_tune_ms"] = list(d["tile_tune_ms"])
        return d


class EcError(RuntimeError):
    def __init__(self, code: int, where: str, info: int = -1):
        self.code = code
        self.info = info
        super().__init__(f"{where}: {STATUS.get(code, code)} ({_text(code)}) info={info}")


_lib = None


def lib() -> ctypes.CDLL:
    """Load the compiled library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} missing "
                               "(run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        P = c_void_p
        sig = {
            "ec_create": (c_int, [POINTER(c_void_p), POINTER(ec_config)]),
            "ec_setup": (c_int, [P, c_int64, P, P, c_int64, P, c_int64, P, P, c_int64, P, c_int]),
            "ec_set_step": (c_int, [P, c_double, c_double]),
            "ec_set_precision": (c_int, [P, c_int]),
            "ec_run": (c_int, [P, c_int64, P, P, P, c_int64, P, c_int]),
            "ec_set_current": (c_int, [P, P, c_int]),
            "ec_state_size": (c_int64, [P]),
            "ec_get_state": (c_int, [P, P, c_int]),
            "ec_set_state": (c_int, [P, P, c_int]),
            "ec_get_modes": (c_int, [P, P, P, c_int]),
            "ec_timings": (c_int, [P, POINTER(ec_timing)]),
            "ec_sync": (c_int, [P]),
            "ec_last_info": (c_int64, [P]),
            "ec_error_string": (ctypes.c_char_p, [c_int]),
            "ec_destroy": (None, [P]),
            "ec_selftest_wait_timeout": (c_int, [c_longlong, POINTER(c_int)]),
            "ec_launch_count": (c_int64, []),
            "ec_solve_z": (c_int, [P, P, P, c_int]),
            "ec_get_inverse_factor": (c_int, [P, P, c_int]),
            "ec_solve_inverse_noalloc": (c_int, [c_int64, P, c_int64, P, P, P]),
            "ec_grad": (c_int, [P, c_int64, P, P, c_int64, P, P, P, c_int]),
            "ec_gemm_bf16": (c_int, [c_int64, c_int64, c_int64, P, P, P, P]),
            "ec_set_mode_count": (c_int, [P, c_int64]),
            "ec_phasors": (c_int, [c_int64, c_int64, P, c_double, c_double, c_int64, P, P, c_int]),
            "ec_batch_run": (c_int, [P, c_int, c_int64, P, P, P, c_int64, P, c_int]),
            "ec_selftest_fail_alloc": (c_int, [c_int64]),
            "ec_gemm_f64_emulated": (c_int, [c_int, c_int, c_int64, c_int64, c_int64, c_double, P,
                                             c_int64, P, c_int64, c_double, P, c_int64, c_int, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _text(code: int) -> str:
    try:
        return lib().ec_error_string(code).decode()
    except Exception:  # noqa: BLE001 - best-effort message only
        return ""


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, mem: int):
    """(pointer, keepalive) for an array in the requested memory space."""
    if x is None:
        return None, None
    if mem == EC_MEM_DEVICE:
        if not _is_torch(x) or not x.is_cuda:
            raise TypeError("device memory requires a CUDA torch tensor")
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x, dtype=np.float64)
    return c_void_p(a.ctypes.data), a


def check(code: int, where: str, ctx=None) -> None:
    if code != 0:
        info = lib().ec_last_info(ctx) if ctx else -1
        raise EcError(code, where, info)


def gemm_bf16(A, B, C=None, stream=None):
    """C = bf16(A) bf16(B), FP32 accumulation on the tensor cores (CUDA float64 tensors)."""
    import torch
    M, K = A.shape
    K2, N = B.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    # column-major views: pass A^T / B^T row-major buffers
    At = A.t().contiguous()
    Bt = B.t().contiguous()
    Ct = torch.empty((N, M), dtype=torch.float64, device=A.device) if C is None else C
    check(lib().ec_gemm_bf16(M, N, K, c_void_p(At.data_ptr()), c_void_p(Bt.data_ptr()),
                             c_void_p(Ct.data_ptr()), c_void_p(stream or 0)), "ec_gemm_bf16")
    return Ct.t()


def gemm_f64_emulated(A, B, C=None, alpha: float = 1.0, beta: float = 0.0, ta: bool = False,
                      tb: bool = False, lower: bool = False, stream=None,
                      kept_slices: bool = False):
    """C = alpha op(A) op(B) + beta C to FP64 accuracy on the tensor cores (CUDA float64
    tensors, any memory order is copied to column-major; returns C as a tensor).
    kept_slices: the path of the modal snapshot products (op(A) cut once into its own
    slice buffer; alpha = 1, no lower-triangle mode)."""
    import torch
    opA = A.t() if ta else A
    opB = B.t() if tb else B
    M, K = opA.shape
    K2, N = opB.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    # column-major buffers: the memory of X^T in row-major order
    Acm = A.t().contiguous()          # column-major A (rows x cols of A)
    Bcm = B.t().contiguous()
    lda = max(1, A.shape[0])
    ldb = max(1, B.shape[0])
    Ct = torch.zeros((N, M), dtype=torch.float64, device=A.device) if C is None else \
        C.t().contiguous()
    check(lib().ec_gemm_f64_emulated(int(ta), int(tb), M, N, K, float(alpha),
                                     c_void_p(Acm.data_ptr()), lda, c_void_p(Bcm.data_ptr()), ldb,
                                     float(beta), c_void_p(Ct.data_ptr()), max(1, M),
                                     int(lower) | (2 if kept_slices else 0),
                                     c_void_p(stream or 0)), "ec_gemm_f64_emulated")
    return Ct.t()


def phasors(probes, t0: float, dt: float, freqs):
    """probes (P, T) host array -> (F, P) complex phasors computed on the GPU."""
    y = np.ascontiguousarray(np.asarray(probes, np.float64).T)       # T x P
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    out = np.empty((f.size, y.shape[1], 2))
    check(lib().ec_phasors(y.shape[0], y.shape[1], c_void_p(y.ctypes.data), float(t0), float(dt),
                           f.size, c_void_p(f.ctypes.data), c_void_p(out.ctypes.data),
                           EC_MEM_HOST), "ec_phasors")
    return out[..., 0] + 1j * out[..., 1]


def launch_count() -> int:
    """Kernels the library has launched in this process so far."""
    return int(lib().ec_launch_count())


def selftest_wait_timeout(spin_limit: int) -> int:
    out = c_int(-1)
    check(lib().ec_selftest_wait_timeout(spin_limit, ctypes.byref(out)), "ec_selftest_wait_timeout")
    return out.value


def selftest_fail_alloc(after: int) -> None:
    """Arm (after >= 0) or disarm (after < 0) the library's out-of-memory test hook."""
    check(lib().ec_selftest_fail_alloc(int(after)), "ec_selftest_fail_alloc")


def solve_inverse_noalloc(Winv, b, x, stream=None, n: int | None = None,
                          ldw: int | None = None) -> None:
    """x = Winv^T (Winv b) on device tensors without any device allocation.

    ``Winv`` is the column-major inverse Cholesky factor as returned by
    ``ThetaMethod.inverse_factor(mem=EC_MEM_DEVICE)`` (its memory is C^{-1} in
    column-major order with leading dimension ``ldw``, default n).  ``stream`` is a
    raw cudaStream_t.  Sizes and devices are checked here, before anything runs:
    Winv must hold at least ldw (n - 1) + n elements and b, x at least n, and all
    three must be contiguous float64 tensors on one CUDA device, on which the call
    then runs.
    """
    n = int(b.shape[0]) if n is None else int(n)
    ldw = n if ldw is None else int(ldw)
    if n < 1 or ldw < n:
        raise ValueError("need 1 <= n <= ldw")
    for name, t, need in (("Winv", Winv, ldw * (n - 1) + n), ("b", b, n), ("x", x, n)):
        if not _is_torch(t):
            raise TypeError(f"{name} must be a torch tensor")
        if t.numel() < need:
            raise ValueError(f"{name} holds {t.numel()} elements, needs at least {need}")
    if not (Winv.device == b.device == x.device):
        raise ValueError("Winv, b and x must be on one device")
    pw, k1 = _ptr(Winv, EC_MEM_DEVICE)
    pb, k2 = _ptr(b, EC_MEM_DEVICE)
    px, k3 = _ptr(x, EC_MEM_DEVICE)
    import torch
    with torch.cuda.device(b.device):
        check(lib().ec_solve_inverse_noalloc(n, pw, ldw, pb, px, c_void_p(stream or 0)),
              "ec_solve_inverse_noalloc")


class ThetaMethod:
    """One context of the C library: setup once, then run / continue.

    Array conventions (row-major numpy shapes): L, R (N, N); E (m, N); M (N, S) coil
    mutual columns; MD (N, m); C (P, N); src (S, T+1); iD (m, T+1).  Results:
    probes (P, T) and snaps (N, T // stride).  ``mem`` selects host numpy
    arrays or CUDA torch tensors for inputs and outputs alike.
    """

    def __init__(self, form: str = "plain", theta: float = 0.5, dt: float = 1e-6,
                 device: int = 0, stream: int | None = None, spin_limit: int = 0,
                 profile: bool = False, solver: str = "inverse", precision: str = "fp64",
                 integrator: str = "theta", rhs: str = "sum", tile_variant: int = 0,
                 refine_steps: int = 0, log_path: str | None = None, setup_gemm: str = "tensor",
                 release_inputs: bool = False):
        if solver not in ("inverse", "substitution"):
            raise ValueError("solver must be 'inverse' or 'substitution'")
        if precision not in _PREC:
            raise ValueError("precision must be 'fp64', 'bf16', 'bf16x3', 'fp32' or 'fp32x2'")
        if integrator not in ("theta", "exact"):
            raise ValueError("integrator must be 'theta' or 'exact'")
        if rhs not in ("sum", "independent", "paired"):
            raise ValueError("rhs must be 'sum', 'independent' or 'paired'")
        if not 0 <= int(tile_variant) <= 3:
            raise ValueError("tile_variant must be 0 (autotune) or 1 .. 3")
        if setup_gemm not in _GEMM:
            raise ValueError("setup_gemm must be 'tensor', 'fp64' or 'tensor_pairsymv'")
        cfg = ec_config(EC_FORM_MODAL if form == "modal" else EC_FORM_PLAIN, float(theta),
                        float(dt), c_void_p(stream or 0), int(device), int(spin_limit),
                        int(bool(profile)),
                        EC_SOLVE_SUBSTITUTION if solver == "substitution" else EC_SOLVE_INVERSE,
                        _PREC[precision], 1 if integrator == "exact" else 0,
                        {"sum": 0, "independent": 1, "paired": 2}[rhs], int(refine_steps),
                        int(tile_variant), _GEMM[setup_gemm],
                        int(bool(release_inputs)))
        self.rhs = rhs
        self.log_path = log_path
        self._desc = {"form": form, "theta": float(theta), "dt": float(dt), "solver": solver,
                      "precision": precision, "integrator": integrator, "rhs": rhs,
                      "refine_steps": int(refine_steps), "device": int(device),
                      "setup_gemm": setup_gemm}
        h = c_void_p()
        check(lib().ec_create(ctypes.byref(h), ctypes.byref(cfg)), "ec_create")
        self._h = h
        self.form = form
        self.n = self.m = self.S = self.P = 0

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().ec_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def setup(self, L, R, E=None, M=None, MD=None, C=None, mem: int = EC_MEM_HOST) -> None:
        n = int(L.shape[0])
        m = 0 if E is None else int(E.shape[0])
        S = 0 if M is None else int(M.shape[1])
        P = 0 if C is None else int(C.shape[0])
        tr = (lambda a: a.t().contiguous()) if mem == EC_MEM_DEVICE else (lambda a: np.ascontiguousarray(a.T))
        keep = []
        pL, k = _ptr(L, mem); keep.append(k)
        pR, k = _ptr(R, mem); keep.append(k)
        pE, k = _ptr(E if m else None, mem); keep.append(k)
        pM, k = _ptr(tr(M) if S else None, mem); keep.append(k)
        pMD, k = _ptr(tr(MD) if (m and MD is not None) else None, mem); keep.append(k)
        pC, k = _ptr(C if P else None, mem); keep.append(k)
        check(lib().ec_setup(self._h, n, pL, pR, m, pE, S, pM, pMD, P, pC, mem), "ec_setup", self._h)
        self.n, self.m, self.S, self.P = n, m, S, P

    def set_step(self, theta: float, dt: float) -> None:
        check(lib().ec_set_step(self._h, float(theta), float(dt)), "ec_set_step", self._h)

    def set_precision(self, precision: str) -> None:
        """Modal form: switch the arithmetic of the products with U ('fp64', 'bf16',
        'bf16x3', 'fp32', 'fp32x2') without repeating the eigensolve."""
        if precision not in _PREC:
            raise ValueError("precision must be 'fp64', 'bf16', 'bf16x3', 'fp32' or 'fp32x2'")
        check(lib().ec_set_precision(self._h, _PREC[precision]), "ec_set_precision", self._h)
        self._desc["precision"] = precision

    def run(self, T: int, src=None, iD=None, snap_stride: int = 0, mem: int = EC_MEM_HOST,
            probes_out=None, snaps_out=None):
        """Advance T steps; returns (probes (P, T), snaps (N, nsnap))."""
        nsnap = T // snap_stride if snap_stride else 0
        nt = 1 if self.rhs == "sum" else self.S
        pout = 1 if self.rhs == "paired" else self.P
        pshape = (T, pout) if nt == 1 else (T, nt, pout)
        sshape = (nsnap, self.n) if nt == 1 else (nsnap, nt, self.n)
        if mem == EC_MEM_DEVICE:
            import torch
            dev = torch.device("cuda")
            probes = probes_out if probes_out is not None else torch.empty(pshape, dtype=torch.float64, device=dev)
            snaps = snaps_out if snaps_out is not None else torch.empty(sshape, dtype=torch.float64, device=dev)
        else:
            probes = np.empty(pshape) if probes_out is None else probes_out
            snaps = np.empty(sshape) if snaps_out is None else snaps_out
        ps, k1 = _ptr(src if self.S else None, mem)
        pi, k2 = _ptr(iD if self.m else None, mem)
        pp = c_void_p(probes.data_ptr() if mem == EC_MEM_DEVICE else probes.ctypes.data) if self.P else None
        pn = c_void_p(snaps.data_ptr() if mem == EC_MEM_DEVICE else snaps.ctypes.data) if nsnap else None
        check(lib().ec_run(self._h, int(T), ps, pi, pp, int(snap_stride) if nsnap else 0, pn, mem),
              "ec_run", self._h)
        if self.log_path:
            append_run_record(self.log_path, dict(self._desc, n=self.n, m=self.m, S=self.S,
                                                  P=self.P, T=int(T), snap_stride=int(snap_stride)),
                              self.timings())
        if nt > 1:
            # (T, nt, pout) -> (nt, pout, T); (nsnap, nt, n) -> (nt, n, nsnap)
            return probes.transpose(1, 2, 0) if mem != EC_MEM_DEVICE else probes.permute(1, 2, 0), \
                snaps.transpose(1, 2, 0) if mem != EC_MEM_DEVICE else snaps.permute(1, 2, 0)
        return probes.T, snaps.T

    def state_size(self) -> int:
        return int(lib().ec_state_size(self._h))

    def get_state(self) -> np.ndarray:
        out = np.empty(self.state_size())
        check(lib().ec_get_state(self._h, c_void_p(out.ctypes.data), EC_MEM_HOST), "ec_get_state", self._h)
        return out

    def set_state(self, state) -> None:
        p, k = _ptr(state, EC_MEM_HOST)
        check(lib().ec_set_state(self._h, p, EC_MEM_HOST), "ec_set_state", self._h)

    def set_current(self, I) -> None:
        p, k = _ptr(I, EC_MEM_HOST)
        check(lib().ec_set_current(self._h, p, EC_MEM_HOST), "ec_set_current", self._h)

    def set_mode_count(self, n_keep: int) -> None:
        """Integrate only the n_keep slowest modes (modal form)."""
        check(lib().ec_set_mode_count(self._h, int(n_keep)), "ec_set_mode_count", self._h)

    def modes(self):
        n0 = self.state_size()
        tau = np.empty(n0)
        U = np.empty((n0, n0))
        check(lib().ec_get_modes(self._h, c_void_p(tau.ctypes.data), c_void_p(U.ctypes.data),
                                 EC_MEM_HOST), "ec_get_modes", self._h)
        return tau, U.T   # column-major in the ABI

    def solve_z(self, b, mem: int = EC_MEM_HOST):
        """x = Z^{-1} b in the internal basis (plain form)."""
        if mem == EC_MEM_DEVICE:
            import torch
            x = torch.empty_like(b)
            pb, k = _ptr(b, mem)
            px = c_void_p(x.data_ptr())
        else:
            x = np.empty(self.state_size())
            pb, k = _ptr(b, mem)
            px = c_void_p(x.ctypes.data)
        check(lib().ec_solve_z(self._h, pb, px, mem), "ec_solve_z", self._h)
        return x

    def inverse_factor(self, out=None, mem: int = EC_MEM_HOST):
        """C^{-1} (N0 x N0, lower) of the plain form's Cholesky factor."""
        n0 = self.state_size()
        if mem == EC_MEM_DEVICE:
            import torch
            W = out if out is not None else torch.empty((n0, n0), dtype=torch.float64, device="cuda")
            pw = c_void_p(W.data_ptr())
        else:
            W = np.empty((n0, n0)) if out is None else out
            pw = c_void_p(W.ctypes.data)
        check(lib().ec_get_inverse_factor(self._h, pw, mem), "ec_get_inverse_factor", self._h)
        return W   # column-major buffer: as a row-major array this is (C^{-1})^T

    def grad(self, T: int, src, v, ckpt_every: int = 250):
        """(J, dJ/dR_diag (N,), dJ/dsrc (S, T+1)) of J = sum_k ||C I^k - v^k||^2 (host arrays).

        ``v`` is (P, T) like the probe outputs of ``run``.
        """
        J = np.zeros(1)
        gR = np.empty(self.n)
        gs = np.empty((self.S, T + 1))
        ps, k1 = _ptr(src if self.S else None, EC_MEM_HOST)
        pv, k2 = _ptr(np.ascontiguousarray(np.asarray(v).T), EC_MEM_HOST)
        check(lib().ec_grad(self._h, int(T), ps, pv, int(ckpt_every), c_void_p(J.ctypes.data),
                            c_void_p(gR.ctypes.data), c_void_p(gs.ctypes.data) if self.S else None,
                            EC_MEM_HOST), "ec_grad", self._h)
        return float(J[0]), gR, gs

    def timings(self) -> dict:
        t = ec_timing()
        check(lib().ec_timings(self._h, ctypes.byref(t)), "ec_timings", self._h)
        return t.as_dict()

    def sync(self) -> None:
        check(lib().ec_sync(self._h), "ec_sync", self._h)


EC_BATCH_MAX = 64


def append_run_record(path: str, config: dict, timings: dict) -> dict:
    """Append one JSON line describing a run (configuration, sizes, the library's phase
    timings and the derived steps/s) to ``path``; returns the record."""
    import json
    import time

    rec = {"time": time.time(), "config": config, "timings": timings}
    run_ms = float(timings.get("run_ms") or 0.0)
    steps = int(timings.get("run_steps") or 0)
    rec["steps_per_s"] = steps / (run_ms / 1e3) if run_ms > 0 else None
    with open(path, "a") as f:
        f.write(json.dumps(rec) + "\n")
    return rec


def batch_run(models, T: int, srcs=None, iDs=None, snap_stride: int = 0):
    """ec_batch_run on host arrays: advance every plain-form ThetaMethod in ``models``
    by T steps in one batched, graph-captured pass.

    ``srcs[i]`` / ``iDs[i]`` are model i's src / iD as for ``run`` (None where the model
    has no coils / electrodes).  Returns a list of (probes (P, T), snaps (N, nsnap)).
    """
    count = len(models)
    if not 1 <= count <= EC_BATCH_MAX:
        raise ValueError(f"batch of 1 .. {EC_BATCH_MAX} models")
    keep = []
    nsnap = T // snap_stride if snap_stride else 0
    Handles = c_void_p * count
    Ptrs = c_void_p * count
    hs = Handles(*[m._h for m in models])
    ps, pi, pp, pn = Ptrs(), Ptrs(), Ptrs(), Ptrs()
    outs = []
    for i, m in enumerate(models):
        s = srcs[i] if (srcs is not None and m.S) else None
        d = iDs[i] if (iDs is not None and m.m) else None
        a, k = _ptr(s, EC_MEM_HOST); keep.append(k); ps[i] = a
        a, k = _ptr(d, EC_MEM_HOST); keep.append(k); pi[i] = a
        probes = np.empty((T, m.P))
        snaps = np.empty((nsnap, m.n))
        pp[i] = c_void_p(probes.ctypes.data) if m.P else None
        pn[i] = c_void_p(snaps.ctypes.data) if nsnap else None
        outs.append((probes, snaps))
    check(lib().ec_batch_run(hs, count, int(T), ps, pi, pp, int(snap_stride) if nsnap else 0, pn,
                             EC_MEM_HOST), "ec_batch_run", models[0]._h)
    return [(p.T, s.T) for p, s in outs]
