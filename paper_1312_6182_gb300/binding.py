"""ctypes binding of libgpspca (C ABI in include/gpspca.h).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  PyTorch supplies device memory (tensors) and nothing else.  If the
library has not been built, ``load()`` raises; there is no fallback.

Layout: A is passed as a tensor ``At`` of shape (n, ld) whose row i holds
column a_i of the p x n matrix A (its first p entries), i.e. A column-major.
Results come back as X (m, p) and Z (m, n): row j is column j of the paper's
X (p x m) and Z (n x m).
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libgpspca.so")

FORMS = {"SL1": 0, "SL0": 1, "BL1": 2, "BL0": 3}
F32, BF16, FP8_E4M3, F64 = 0, 1, 2, 3
DEVICE, HOST = 0, 1

OK, PENDING = 0, 1
EINVAL, ENOMEM, ENONFINITE, ETIMEDOUT, EDEGENERATE, ECUDA, ENOTFOUND = -1, -2, -3, -4, -5, -6, -7
CONVERGED, MAXIT, ZERO, DEGENERATE = 0, 1, 2, 3
GAMMA_RELATIVE = 1
EAGER = 2  # kernels launched one by one, host-driven loop (for profilers)
NO_TENSOR_CORES = 4  # CUDA-core fused sweep even where the tensor-core sweep applies
INJECT_TIMEOUT = 8  # test hook: the solve returns ETIMEDOUT after running
TIME_T_PASS = 16  # time_sweep: the tensor-core sweep's T pass alone
MAX_M = 64

ERROR_NAMES = {
    EINVAL: "EINVAL", ENOMEM: "ENOMEM", ENONFINITE: "ENONFINITE", ETIMEDOUT: "ETIMEDOUT",
    EDEGENERATE: "EDEGENERATE", ECUDA: "ECUDA", ENOTFOUND: "ENOTFOUND",
}

EXPORTED = ("gpspca_create", "gpspca_solve", "gpspca_submit", "gpspca_poll", "gpspca_destroy",
            "gpspca_last_error", "gpspca_time_sweep", "gpspca_sweep_static", "gpspca_synth_spikes",
            "gpspca_solve_batch", "gpspca_solve_deflated", "gpspca_project", "gpspca_tune", "gpspca_tune_save",
            "gpspca_tune_load", "gpspca_plan_launches", "gpspca_upload")


class Matrix(ctypes.Structure):
    _fields_ = [
        ("data", ctypes.c_void_p),
        ("dtype", ctypes.c_int),
        ("location", ctypes.c_int),
        ("p", ctypes.c_int64),
        ("n", ctypes.c_int64),
        ("ld", ctypes.c_int64),
        ("col_scale", ctypes.c_void_p),
    ]


class Out(ctypes.Structure):
    _fields_ = [
        ("location", ctypes.c_int),
        ("X", ctypes.c_void_p),
        ("Z", ctypes.c_void_p),
        ("support", ctypes.c_void_p),
        ("objective", ctypes.c_void_p),
        ("iters", ctypes.c_void_p),
        ("status", ctypes.c_void_p),
        ("gamma_abs", ctypes.c_void_p),
    ]


class Request(ctypes.Structure):
    _fields_ = [
        ("A", Matrix),
        ("form", ctypes.c_int),
        ("gamma", ctypes.POINTER(ctypes.c_double)),
        ("m", ctypes.c_int32),
        ("mu", ctypes.POINTER(ctypes.c_double)),
        ("tol", ctypes.c_double),
        ("maxit", ctypes.c_int32),
        ("x0", ctypes.c_void_p),
        ("flags", ctypes.c_uint32),
        ("out", Out),
    ]


_lib = None


def load(path: str = LIB_PATH):
    """Load libgpspca.so (raises if it is missing: build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run __graft_entry__.build() or python -m paper_1312_6182_gb300.build")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    lib.gpspca_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_size_t, P]
    lib.gpspca_create.restype = ctypes.c_int
    lib.gpspca_solve.argtypes = [P, ctypes.POINTER(Matrix), ctypes.c_int, D, ctypes.c_int32, D, ctypes.c_double,
                                 ctypes.c_int32, P, ctypes.c_uint32, ctypes.POINTER(Out)]
    lib.gpspca_solve.restype = ctypes.c_int
    lib.gpspca_solve_deflated.argtypes = [P, ctypes.POINTER(Matrix), ctypes.c_int, D, ctypes.c_int32,
                                          ctypes.c_double, ctypes.c_int32, ctypes.c_uint32, ctypes.POINTER(Out)]
    lib.gpspca_solve_deflated.restype = ctypes.c_int
    lib.gpspca_project.argtypes = [P, ctypes.POINTER(Matrix), P, ctypes.c_int32, P]
    lib.gpspca_project.restype = ctypes.c_int
    lib.gpspca_submit.argtypes = [P, ctypes.POINTER(Matrix), ctypes.c_int, D, ctypes.c_int32, D, ctypes.c_double,
                                  ctypes.c_int32, ctypes.c_uint32, ctypes.POINTER(Out),
                                  ctypes.POINTER(ctypes.c_uint64)]
    lib.gpspca_submit.restype = ctypes.c_int
    lib.gpspca_poll.argtypes = [P, ctypes.c_uint64, ctypes.c_int32]
    lib.gpspca_poll.restype = ctypes.c_int
    lib.gpspca_destroy.argtypes = [P]
    lib.gpspca_destroy.restype = ctypes.c_int
    lib.gpspca_last_error.argtypes = []
    lib.gpspca_last_error.restype = ctypes.c_char_p
    lib.gpspca_time_sweep.argtypes = [P, ctypes.POINTER(Matrix), ctypes.c_int, D, ctypes.c_int32, D,
                                      ctypes.c_uint32, ctypes.c_int32, D]
    lib.gpspca_time_sweep.restype = ctypes.c_int
    lib.gpspca_sweep_static.argtypes = [ctypes.POINTER(Matrix), ctypes.c_int, ctypes.c_double, P, P, P, P, P]
    lib.gpspca_sweep_static.restype = ctypes.c_int
    lib.gpspca_synth_spikes.argtypes = [P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                        D, ctypes.c_double, ctypes.c_uint64, P]
    lib.gpspca_synth_spikes.restype = ctypes.c_int
    lib.gpspca_solve_batch.argtypes = [P, ctypes.c_int32, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_int32)]
    lib.gpspca_solve_batch.restype = ctypes.c_int
    lib.gpspca_tune.argtypes = [P, ctypes.POINTER(Matrix), ctypes.c_int, D, ctypes.c_int32, D, ctypes.c_uint32,
                                ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), D, D]
    lib.gpspca_tune.restype = ctypes.c_int
    lib.gpspca_tune_save.argtypes = [P, ctypes.c_char_p]
    lib.gpspca_tune_save.restype = ctypes.c_int
    lib.gpspca_tune_load.argtypes = [P, ctypes.c_char_p]
    lib.gpspca_tune_load.restype = ctypes.c_int
    lib.gpspca_plan_launches.argtypes = [P, ctypes.POINTER(Matrix), ctypes.c_int, D, ctypes.c_int32, D,
                                         ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32)]
    lib.gpspca_plan_launches.restype = ctypes.c_int
    lib.gpspca_upload.argtypes = [P, ctypes.POINTER(Matrix), ctypes.POINTER(Matrix)]
    lib.gpspca_upload.restype = ctypes.c_int
    _lib = lib
    return lib


def last_error() -> str:
    return load().gpspca_last_error().decode()


class GpspcaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(rc: int, allow=(OK,)):
    if rc not in allow:
        raise GpspcaError(rc, last_error())
    return rc


def _dtype_code(t):
    import torch

    table = {torch.float32: F32, torch.float64: F64, torch.bfloat16: BF16}
    if hasattr(torch, "float8_e4m3fn"):
        table[torch.float8_e4m3fn] = FP8_E4M3
    if t.dtype not in table:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return table[t.dtype]


def _darr(vals: Optional[Sequence[float]], m: int):
    if vals is None:
        return None
    arr = (ctypes.c_double * m)(*[float(v) for v in vals])
    return arr


def matrix(At, p: Optional[int] = None, col_scale=None) -> Matrix:
    """Descriptor for At (n, ld) holding A column-major (first p entries of each row)."""
    if At.dim() != 2 or At.stride(1) != 1:
        raise ValueError("At must be 2-D with unit stride along its rows")
    n, ld = At.shape
    if p is None:
        p = ld
    M = Matrix()
    M.data = At.data_ptr() if At.numel() else None
    M.dtype = _dtype_code(At)
    M.location = DEVICE if At.is_cuda else HOST
    M.p = int(p)
    M.n = int(n)
    M.ld = int(At.stride(0)) if n > 1 else int(max(ld, p))
    M.col_scale = col_scale.data_ptr() if col_scale is not None else None
    return M


@dataclass
class Result:
    X: "object"          # (m, p): row j = column j of X
    Z: "object"          # (m, n)
    support: "object"    # (m, ceil(n/32)) int32 bit words
    objective: "object"  # (m,) float64
    iters: "object"      # (m,) int32
    status: "object"     # (m,) int32
    gamma_abs: "object"  # (m,) float64
    rc: int = OK


def alloc_result(m: int, p: int, n: int, device, tc, pin: bool = False) -> Result:
    import torch

    kw = dict(device=device)
    pm = dict(pin_memory=True) if (pin and str(device) == "cpu") else {}
    nw = (n + 31) // 32
    return Result(
        X=torch.empty((m, p), dtype=tc, **kw, **pm),
        Z=torch.empty((m, n), dtype=tc, **kw, **pm),
        support=torch.empty((m, nw), dtype=torch.int32, **kw, **pm),
        objective=torch.empty((m,), dtype=torch.float64, **kw, **pm),
        iters=torch.empty((m,), dtype=torch.int32, **kw, **pm),
        status=torch.empty((m,), dtype=torch.int32, **kw, **pm),
        gamma_abs=torch.empty((m,), dtype=torch.float64, **kw, **pm),
    )


def out_struct(res: Result) -> Out:
    o = Out()
    o.location = DEVICE if res.X.is_cuda else HOST
    o.X = res.X.data_ptr() if res.X.numel() else None
    o.Z = res.Z.data_ptr() if res.Z.numel() else None
    o.support = res.support.data_ptr() if res.support.numel() else None
    o.objective = res.objective.data_ptr()
    o.iters = res.iters.data_ptr()
    o.status = res.status.data_ptr()
    o.gamma_abs = res.gamma_abs.data_ptr()
    if o.X is None:
        o.X = o.objective  # zero-length outputs: any non-NULL pointer
    if o.Z is None:
        o.Z = o.objective
    return o


class Context:
    """A libgpspca context on one CUDA device (its own stream)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, stream=None):
        """stream: a torch.cuda.Stream (or raw cudaStream_t int) to run on;
        None lets the library create its own."""
        self.lib = load()
        self.ptr = ctypes.c_void_p()
        handle = None
        if stream is not None:
            handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check(self.lib.gpspca_create(ctypes.byref(self.ptr), int(device), int(budget_bytes), handle))
        self.device = device
        self.stream = stream

    def close(self):
        if self.ptr:
            self.lib.gpspca_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _sync_torch(*tensors):
        import torch

        if any(t is not None and getattr(t, "is_cuda", False) for t in tensors):
            torch.cuda.current_stream().synchronize()

    def solve(self, At, form: str, gamma, mu=None, tol: float = 1e-6, maxit: int = 1000, x0=None,
              gamma_relative: bool = False, p: Optional[int] = None, col_scale=None,
              out: Optional[Result] = None, allow_degenerate: bool = True, eager: bool = False,
              tensor_cores: bool = True, extra_flags: int = 0) -> Result:
        """One synchronous solve.  gamma: m values; mu: block weights.  eager: launch
        the kernels one by one with a host-driven loop instead of the CUDA graph.
        tensor_cores=False keeps the CUDA-core sweep where the tcgen05 one applies.
        extra_flags: further GPSPCA_* flag bits (e.g. INJECT_TIMEOUT)."""
        import torch

        gamma = [float(g) for g in (gamma if hasattr(gamma, "__len__") else [gamma])]
        m = len(gamma)
        M = matrix(At, p, col_scale)
        tc = torch.float64 if At.dtype == torch.float64 else torch.float32
        if out is None:
            out = alloc_result(m, int(M.p), int(M.n), At.device, tc)
        o = out_struct(out)
        self._sync_torch(At, x0, out.X)
        rc = self.lib.gpspca_solve(self.ptr, ctypes.byref(M), FORMS[form], _darr(gamma, m), m, _darr(mu, m),
                                   float(tol), int(maxit), x0.data_ptr() if x0 is not None else None,
                                   (GAMMA_RELATIVE if gamma_relative else 0) | (EAGER if eager else 0)
                                   | (0 if tensor_cores else NO_TENSOR_CORES) | int(extra_flags), ctypes.byref(o))
        allow = (OK, EDEGENERATE) if allow_degenerate else (OK,)
        _check(rc, allow)
        out.rc = rc
        return out

    def solve_deflated(self, At, form: str, gamma, tol: float = 1e-6, maxit: int = 1000,
                       gamma_relative: bool = False, p: Optional[int] = None, col_scale=None,
                       out: Optional[Result] = None, eager: bool = False) -> Result:
        """Several single-unit components (form SL1 or SL0) by projection
        deflation (gpspca_solve_deflated): component j solves with gamma[j] on
        A_{j-1} = A_{j-2} (I - z_{j-1} z_{j-1}^T).  A is not modified."""
        import torch

        gamma = [float(g) for g in (gamma if hasattr(gamma, "__len__") else [gamma])]
        m = len(gamma)
        M = matrix(At, p, col_scale)
        tc = torch.float64 if At.dtype == torch.float64 else torch.float32
        if out is None:
            out = alloc_result(m, int(M.p), int(M.n), At.device, tc)
        o = out_struct(out)
        self._sync_torch(At, None, out.X)
        rc = self.lib.gpspca_solve_deflated(self.ptr, ctypes.byref(M), FORMS[form], _darr(gamma, m), m, float(tol),
                                            int(maxit), (GAMMA_RELATIVE if gamma_relative else 0)
                                            | (EAGER if eager else 0), ctypes.byref(o))
        _check(rc, (OK, EDEGENERATE))
        out.rc = rc
        return out

    def project(self, Bt, Z, col_scale=None, p: Optional[int] = None, out=None):
        """Scores S = B Z (gpspca_project).  Bt: (q, ld) tensor holding B
        column-major like At; Z: (m, n) tensor, row j = loading j (a solve's
        Result.Z); returns (m, q), row j = column j of S, in Z's device."""
        import torch

        M = matrix(Bt, p, col_scale)
        m = int(Z.shape[0])
        tc = torch.float64 if Bt.dtype == torch.float64 else torch.float32
        if Z.dtype != tc or not Z.is_contiguous() or Z.shape[1] != M.n:
            raise ValueError(f"Z must be a contiguous ({m}, {int(M.n)}) {tc} tensor")
        if (Z.device.type == "cuda") != (M.location == DEVICE):
            raise ValueError("Z must be in the same location as B")
        if out is None:
            out = torch.empty((m, int(M.p)), dtype=tc, device=Z.device)
        self._sync_torch(Bt, Z, out)
        _check(self.lib.gpspca_project(self.ptr, ctypes.byref(M), Z.data_ptr(), m, out.data_ptr()), (OK,))
        return out

    def solve_batch(self, items, allow_degenerate: bool = True):
        """Independent solves run concurrently (gpspca_solve_batch), stream-ordered
        with the context's stream.  items: dicts with the keyword arguments of
        solve (At, form, gamma; optional mu, tol, maxit, x0, gamma_relative, p,
        col_scale, out, eager, tensor_cores).  Returns the list of Results."""
        import torch

        n = len(items)
        reqs = (Request * n)()
        keep, outs = [], []
        for k, it in enumerate(items):
            At = it["At"]
            gamma = [float(g) for g in (it["gamma"] if hasattr(it["gamma"], "__len__") else [it["gamma"]])]
            m = len(gamma)
            M = matrix(At, it.get("p"), it.get("col_scale"))
            tc = torch.float64 if At.dtype == torch.float64 else torch.float32
            out = it.get("out") or alloc_result(m, int(M.p), int(M.n), At.device, tc)
            g_arr, mu_arr = _darr(gamma, m), _darr(it.get("mu"), m)
            keep += [g_arr, mu_arr]
            x0 = it.get("x0")
            reqs[k].A = M
            reqs[k].form = FORMS[it["form"]]
            reqs[k].gamma = ctypes.cast(g_arr, ctypes.POINTER(ctypes.c_double))
            reqs[k].m = m
            reqs[k].mu = ctypes.cast(mu_arr, ctypes.POINTER(ctypes.c_double)) if mu_arr is not None else None
            reqs[k].tol = float(it.get("tol", 1e-6))
            reqs[k].maxit = int(it.get("maxit", 1000))
            reqs[k].x0 = x0.data_ptr() if x0 is not None else None
            reqs[k].flags = ((GAMMA_RELATIVE if it.get("gamma_relative") else 0) | (EAGER if it.get("eager") else 0)
                             | (0 if it.get("tensor_cores", True) else NO_TENSOR_CORES))
            reqs[k].out = out_struct(out)
            outs.append(out)
            self._sync_torch(At, x0, out.X)
        rcs = (ctypes.c_int32 * n)()
        self.lib.gpspca_solve_batch(self.ptr, n, reqs, rcs)
        allow = (OK, EDEGENERATE) if allow_degenerate else (OK,)
        for k in range(n):
            _check(rcs[k], allow)
            outs[k].rc = rcs[k]
        return outs

    def upload(self, hA, dA, p: Optional[int] = None, host_scale=None, dev_scale=None):
        """Asynchronous copy of the host tensor hA (page-locked for overlap)
        into the device tensor dA of the same dtype and shape (gpspca_upload);
        returns at once.  Later solves of this context on dA wait for the
        copy on the device.  FP8: host_scale / dev_scale, the n column
        scales on either side."""
        H = matrix(hA, p, host_scale)
        D = matrix(dA, p, dev_scale)
        if H.location != HOST or D.location != DEVICE:
            raise ValueError("upload copies a host tensor into a device tensor")
        self._sync_torch(dA, dev_scale)
        _check(self.lib.gpspca_upload(self.ptr, ctypes.byref(H), ctypes.byref(D)))
        return dA

    def submit(self, At, form: str, gamma, mu=None, tol: float = 1e-6, maxit: int = 1000,
               gamma_relative: bool = False, p: Optional[int] = None, col_scale=None,
               out: Optional[Result] = None):
        """Queue a solve (device buffers only); returns (ticket, out)."""
        import torch

        gamma = [float(g) for g in (gamma if hasattr(gamma, "__len__") else [gamma])]
        m = len(gamma)
        M = matrix(At, p, col_scale)
        tc = torch.float64 if At.dtype == torch.float64 else torch.float32
        if out is None:
            out = alloc_result(m, int(M.p), int(M.n), At.device, tc)
        o = out_struct(out)
        self._sync_torch(At, out.X)
        t = ctypes.c_uint64()
        _check(self.lib.gpspca_submit(self.ptr, ctypes.byref(M), FORMS[form], _darr(gamma, m), m, _darr(mu, m),
                                      float(tol), int(maxit), GAMMA_RELATIVE if gamma_relative else 0,
                                      ctypes.byref(o), ctypes.byref(t)))
        return t.value, out

    def poll(self, ticket: int, wait_us: int = 0) -> int:
        """PENDING, or the ticket's result code (once)."""
        return self.lib.gpspca_poll(self.ptr, ctypes.c_uint64(ticket), int(wait_us))

    def time_sweep(self, At, form: str, gamma, mu=None, reps: int = 20, gamma_relative: bool = False,
                   p: Optional[int] = None, col_scale=None, tensor_cores: bool = True, t_pass: bool = False) -> float:
        """Mean milliseconds of one fused sweep (all component passes), CUDA events;
        t_pass: the tensor-core sweep's T pass alone."""
        gamma = [float(g) for g in (gamma if hasattr(gamma, "__len__") else [gamma])]
        m = len(gamma)
        M = matrix(At, p, col_scale)
        self._sync_torch(At)
        ms = ctypes.c_double()
        _check(self.lib.gpspca_time_sweep(self.ptr, ctypes.byref(M), FORMS[form], _darr(gamma, m), m,
                                          _darr(mu, m), (GAMMA_RELATIVE if gamma_relative else 0)
                                          | (0 if tensor_cores else NO_TENSOR_CORES)
                                          | (TIME_T_PASS if t_pass else 0), int(reps), ctypes.byref(ms)))
        return ms.value


    def plan_launches(self, At, form: str, gamma, mu=None, gamma_relative: bool = False, p: Optional[int] = None,
                      col_scale=None, tensor_cores: bool = True):
        """Kernel launches of one solve of this problem (gpspca_plan_launches):
        (before the iterations, per iteration, after them)."""
        gamma = [float(g) for g in (gamma if hasattr(gamma, "__len__") else [gamma])]
        m = len(gamma)
        M = matrix(At, p, col_scale)
        self._sync_torch(At)
        c = (ctypes.c_int32 * 3)()
        _check(self.lib.gpspca_plan_launches(self.ptr, ctypes.byref(M), FORMS[form], _darr(gamma, m), m,
                                             _darr(mu, m), (GAMMA_RELATIVE if gamma_relative else 0)
                                             | (0 if tensor_cores else NO_TENSOR_CORES), c))
        return int(c[0]), int(c[1]), int(c[2])

    def tune(self, At, form: str, gamma, mu=None, reps: int = 10, gamma_relative: bool = False,
             p: Optional[int] = None, col_scale=None, tensor_cores: bool = True):
        """Time every candidate sweep layout for this shape and keep the fastest
        (gpspca_tune).  Returns (layouts timed, best ms per sweep, default ms)."""
        gamma = [float(g) for g in (gamma if hasattr(gamma, "__len__") else [gamma])]
        m = len(gamma)
        M = matrix(At, p, col_scale)
        self._sync_torch(At)
        nc, best, dflt = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
        _check(self.lib.gpspca_tune(self.ptr, ctypes.byref(M), FORMS[form], _darr(gamma, m), m, _darr(mu, m),
                                    (GAMMA_RELATIVE if gamma_relative else 0)
                                    | (0 if tensor_cores else NO_TENSOR_CORES), int(reps), ctypes.byref(nc),
                                    ctypes.byref(best), ctypes.byref(dflt)))
        return nc.value, best.value, dflt.value

    def tune_save(self, path: str):
        """Write the tuned layouts to a file (gpspca_tune_save)."""
        _check(self.lib.gpspca_tune_save(self.ptr, str(path).encode()))

    def tune_load(self, path: str):
        """Merge the tuned layouts of a file into this context (gpspca_tune_load)."""
        _check(self.lib.gpspca_tune_load(self.ptr, str(path).encode()))


def sweep_static(At, form: str, gamma: float, x, x_next, t, objective, p: Optional[int] = None, stream=None) -> int:
    """One allocation-free single-unit sweep (gpspca_sweep_static).

    At: float32 CUDA tensor (n, ld); x, x_next: float32 CUDA tensors of p
    entries; t: float32 CUDA tensor of n entries; objective: float64 CUDA
    tensor of one entry.  Every buffer is the caller's; the library allocates
    nothing.  Returns OK or raises GpspcaError.
    """
    import torch

    lib = load()
    n, ld = At.shape
    pp = ld if p is None else int(p)
    if not (At.is_cuda and At.dtype == torch.float32):
        raise GpspcaError(EINVAL, "sweep_static: At must be a float32 CUDA tensor")
    for name, ten, dt, count in (("x", x, torch.float32, pp), ("x_next", x_next, torch.float32, pp),
                                 ("t", t, torch.float32, n), ("objective", objective, torch.float64, 1)):
        if not (ten.is_cuda and ten.device == At.device and ten.dtype == dt and ten.is_contiguous()
                and ten.numel() == count):
            raise GpspcaError(EINVAL, f"sweep_static: {name} must be a contiguous {dt} tensor of {count} entries "
                                      f"on {At.device}")
    M = matrix(At, p)
    torch.cuda.current_stream().synchronize()
    handle = None
    if stream is not None:
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    with torch.cuda.device(At.device):  # the library works on the current device
        rc = lib.gpspca_sweep_static(ctypes.byref(M), FORMS[form], float(gamma), x.data_ptr(), x_next.data_ptr(),
                                     t.data_ptr(), objective.data_ptr(), handle)
    return _check(rc)


def synth_spikes(At, k: int, theta, support_frac: float, seed: int, p: Optional[int] = None, stream=None) -> int:
    """Fill the float32 / bfloat16 CUDA tensor At (n, ld) with the seeded
    planted-spike matrix of gpspca_synth_spikes (rows = columns of A).
    Asynchronous on `stream` (a torch.cuda.Stream; default: the current one)."""
    import torch

    lib = load()
    n, ld = At.shape
    p = ld if p is None else int(p)
    if stream is None:
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    rc = lib.gpspca_synth_spikes(At.data_ptr(), _dtype_code(At), int(p), int(n), int(At.stride(0)), int(k),
                                 _darr(theta, k) if k > 0 else None, float(support_frac), int(seed) & (2**64 - 1),
                                 handle)
    return _check(rc)
