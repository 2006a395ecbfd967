"""GB300-native rigid multiblob mobility solver (wall-corrected RPY).

Thin Python binding over the C ABI of libmb.so (include/mb.h).  It only
marshals arguments: every step runs in the library's CUDA kernels.  Arrays are
torch tensors (float64, contiguous; int64 for blob offsets) on the context's
CUDA device, or CPU tensors where a call accepts host memory.  If libmb.so has
not been built, every call raises — there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "MBError",
    "Context",
    "FP64",
    "FP32_KAHAN",
    "MIXED_REFINE",
    "DF64",
    "library_path",
    "load_library",
    "EXPORTED_SYMBOLS",
    "mobility_matvec_noalloc",
    "NOALLOC_MAX_BLOBS",
    "Server",
]

FP64, FP32_KAHAN, MIXED_REFINE, DF64 = 0, 1, 2, 3
_PREC = {"fp64": FP64, "fp32": FP32_KAHAN, "fp32_kahan": FP32_KAHAN, "mixed": MIXED_REFINE,
         "df64": DF64}

STATUS = {
    0: "MB_OK",
    1: "MB_EINVAL",
    2: "MB_ENOMEM",
    3: "MB_ECUDA",
    4: "MB_ENOTCONVERGED",
    5: "MB_ETIMEOUT",
    6: "MB_ESINGULAR",
}

EXPORTED_SYMBOLS = [
    "mb_status_string",
    "mb_last_error",
    "mb_context_create",
    "mb_context_destroy",
    "mb_context_workspace_bytes",
    "mb_context_set_pair_variant",
    "mb_context_set_wait_limit",
    "mb_context_pair_variant",
    "mb_profile_enable",
    "mb_profile_read",
    "mb_measure_fma_rate",
    "mb_mobility_matvec",
    "mb_mobility_matvec_noalloc",
    "mb_blob_positions",
    "mb_K_apply",
    "mb_KT_apply",
    "mb_mobility_eval",
    "mb_render_flow",
    "mb_lambda_moments",
    "mb_precond_setup",
    "mb_precond_setup_shared",
    "mb_precond_apply",
    "mb_solve_mobility",
    "mb_solve_resistance",
    "mb_solve_mobility_permeable",
    "mb_solve_batch",
    "mb_server_create",
    "mb_server_destroy",
    "mb_server_submit",
    "mb_server_step",
    "mb_server_poll",
    "mb_server_finished",
]

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libmb.so")


class MBError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{self.name}: {message}")


class Params(ctypes.Structure):
    _fields_ = [
        ("a", ctypes.c_double),
        ("eta", ctypes.c_double),
        ("wall", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("maxit", ctypes.c_int),
        ("restart", ctypes.c_int),
        ("prec", ctypes.c_int),
        ("precond", ctypes.c_int),
    ]


PRECOND_WALL, PRECOND_FREE_SHARED = 0, 1
_PRECOND = {"wall": PRECOND_WALL, "free_shared": PRECOND_FREE_SHARED}


def _precond(kind):
    if isinstance(kind, str):
        return _PRECOND[kind]
    return int(kind)


class Problem(ctypes.Structure):
    _fields_ = [
        ("n_bodies", ctypes.c_int64),
        ("n_blobs", ctypes.c_int64),
        ("q", ctypes.c_void_p),
        ("theta", ctypes.c_void_p),
        ("blob_start", ctypes.c_void_p),
        ("rho", ctypes.c_void_p),
        ("F", ctypes.c_void_p),
        ("T", ctypes.c_void_p),
        ("slip", ctypes.c_void_p),
        ("U", ctypes.c_void_p),
        ("Omega", ctypes.c_void_p),
        ("lam", ctypes.c_void_p),
    ]


class ServerLimits(ctypes.Structure):
    _fields_ = [
        ("max_blobs", ctypes.c_int64),
        ("max_bodies", ctypes.c_int64),
        ("max_precond_bytes", ctypes.c_int64),
        ("max_requests", ctypes.c_int),
        ("tick_pairs", ctypes.c_double),
        ("max_bypass", ctypes.c_int),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("rel_residual", ctypes.c_double),
        ("setup_ms", ctypes.c_double),
        ("solve_ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library():
    """Load libmb.so (built by paper_1602_02170_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library not built ({path} missing); run "
            "`python -c 'import __graft_entry__ as g; g.build()'` first"
        )
    L = ctypes.CDLL(path)
    vp, i64, dbl, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    L.mb_status_string.restype = ctypes.c_char_p
    L.mb_status_string.argtypes = [ci]
    L.mb_last_error.restype = ctypes.c_char_p
    L.mb_last_error.argtypes = [vp]
    L.mb_context_create.argtypes = [ctypes.POINTER(vp), ci, ctypes.c_size_t]
    L.mb_context_destroy.argtypes = [vp]
    L.mb_context_workspace_bytes.restype = ctypes.c_size_t
    L.mb_context_workspace_bytes.argtypes = [vp]
    L.mb_context_set_pair_variant.argtypes = [vp, ci]
    L.mb_context_set_wait_limit.argtypes = [vp, dbl]
    L.mb_context_pair_variant.argtypes = [vp, i64, ci, ctypes.POINTER(ci)]
    L.mb_profile_enable.argtypes = [vp, ci]
    L.mb_profile_read.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i64),
                                  ctypes.POINTER(i64), ci]
    L.mb_measure_fma_rate.argtypes = [vp, ci, ctypes.POINTER(dbl), vp]
    L.mb_mobility_matvec.argtypes = [vp, vp, vp, i64, dbl, dbl, ci, ci, vp, vp]
    L.mb_mobility_matvec_noalloc.argtypes = [vp, vp, i64, dbl, dbl, ci, vp, vp]
    L.mb_blob_positions.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp]
    L.mb_K_apply.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp]
    L.mb_KT_apply.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp]
    L.mb_precond_setup.argtypes = [vp, i64, i64, vp, vp, vp, dbl, dbl, ci, vp]
    L.mb_lambda_moments.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp]
    L.mb_mobility_eval.argtypes = [vp, vp, i64, vp, vp, i64, dbl, dbl, ci, ci, vp, vp]
    L.mb_render_flow.argtypes = [vp, vp, i64, vp, vp, i64, vp, ci, dbl, dbl, ci, ci, vp, vp]
    L.mb_precond_setup_shared.argtypes = [vp, i64, i64, vp, vp, vp, dbl, dbl, vp]
    L.mb_precond_apply.argtypes = [vp, vp, vp, vp, vp, vp]
    L.mb_solve_mobility.argtypes = [
        vp, i64, i64, vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(Params), vp, vp, vp,
        ctypes.POINTER(Info), vp,
    ]
    L.mb_solve_mobility_permeable.argtypes = [
        vp, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(Params), vp, vp, vp,
        ctypes.POINTER(Info), vp,
    ]
    L.mb_solve_resistance.argtypes = [
        vp, i64, i64, vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(Params), vp, vp, vp,
        ctypes.POINTER(Info), vp,
    ]
    L.mb_solve_batch.argtypes = [vp, ci, ctypes.POINTER(Problem), ctypes.POINTER(Params),
                                 ctypes.POINTER(Info), vp]
    L.mb_server_create.argtypes = [vp, ctypes.POINTER(Params), ctypes.POINTER(ServerLimits),
                                   ctypes.POINTER(vp)]
    L.mb_server_destroy.argtypes = [vp]
    L.mb_server_submit.argtypes = [vp, ctypes.POINTER(Problem), ctypes.POINTER(i64)]
    L.mb_server_step.argtypes = [vp, vp, ctypes.POINTER(ci), ctypes.POINTER(ci)]
    L.mb_server_poll.argtypes = [vp, i64, ctypes.POINTER(ci), ctypes.POINTER(Info),
                                 ctypes.POINTER(ci)]
    L.mb_server_finished.argtypes = [vp, ctypes.POINTER(i64), ci, ctypes.POINTER(ci)]
    for name in EXPORTED_SYMBOLS:
        if name not in ("mb_status_string", "mb_last_error", "mb_context_workspace_bytes"):
            getattr(L, name).restype = ci  # mb_status
    _lib = L
    return L


def _prec(p) -> int:
    if isinstance(p, str):
        return _PREC[p.lower()]
    return int(p)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


NOALLOC_MAX_BLOBS = 65536


def mobility_matvec_noalloc(r, f, a, eta=1.0, wall=True, out=None, stream=None):
    """u = M(r) f through mb_mobility_matvec_noalloc: FP32 pair kernel, no
    context and no device allocation inside the library (its scratch is a
    fixed device array for up to NOALLOC_MAX_BLOBS blobs; concurrent calls
    on the GPU race on it).  r, f, out: contiguous float64 (N, 3) CUDA
    tensors on the current device.  `out` is allocated here by torch if not
    given; pass it to keep the call allocation-free end to end."""
    import torch

    L = load_library()
    n = int(r.shape[0])
    if not r.is_cuda:
        raise ValueError("r must be a CUDA tensor")
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float64, device=r.device)
    for t in (r, f, out):
        if t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != (n, 3):
            raise ValueError("r, f, out must be contiguous float64 (N, 3)")
        if t.device != r.device:
            raise ValueError("r, f and out must be on the same CUDA device")
    with torch.cuda.device(r.device):
        if stream is None:
            stream = torch.cuda.current_stream(r.device)
        st = L.mb_mobility_matvec_noalloc(_ptr(r), _ptr(f), n, float(a), float(eta),
                                          int(bool(wall)), _ptr(out),
                                          ctypes.c_void_p(stream.cuda_stream))
    if st != 0:
        raise MBError(st, L.mb_last_error(None).decode())
    return out


class Context:
    """A library context on one CUDA device (owns all workspace)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        import torch

        self._torch = torch
        self.L = load_library()
        self.device = torch.device("cuda", device)
        h = ctypes.c_void_p()
        st = self.L.mb_context_create(ctypes.byref(h), device, hbm_budget_bytes)
        if st != 0:
            raise MBError(st, self.L.mb_last_error(None).decode())
        self.handle = h

    # ------------------------------------------------------------ plumbing
    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.L.mb_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st):
        if st != 0:
            raise MBError(st, self.L.mb_last_error(self.handle).decode())

    def _stream(self, stream):
        if stream is None:
            stream = self._torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(stream.cuda_stream)

    def workspace_bytes(self) -> int:
        return int(self.L.mb_context_workspace_bytes(self.handle))

    def set_wait_limit(self, seconds: float):
        """Bound the host waits of solves, preconditioner setup and host-pointer
        matvecs (MB_ETIMEOUT past it); <= 0 waits without limit."""
        self._check(self.L.mb_context_set_wait_limit(self.handle, float(seconds)))

    def set_pair_variant(self, variant: int):
        """-1 autotune (default), 0 scalar, 1 packed x2, 2 packed x4, 3 symmetric,
        4 packed in 32-thread CTAs (small problems)."""
        self._check(self.L.mb_context_set_pair_variant(self.handle, int(variant)))

    def pair_variant(self, n: int, wall: bool = True) -> int:
        """Variant used for N blobs (-1 if the autotuner has not run yet)."""
        v = ctypes.c_int()
        self._check(self.L.mb_context_pair_variant(self.handle, int(n), int(bool(wall)),
                                                    ctypes.byref(v)))
        return v.value

    def profile_enable(self, on: bool = True):
        self._check(self.L.mb_profile_enable(self.handle, int(bool(on))))

    def profile_read(self, reset: bool = True):
        """(summed pair-kernel ms, pair-kernel launches, running kernel-launch count)."""
        ms = ctypes.c_double()
        pl = ctypes.c_int64()
        kl = ctypes.c_int64()
        self._check(self.L.mb_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(pl),
                                           ctypes.byref(kl), int(bool(reset))))
        return ms.value, pl.value, kl.value

    def measure_fma_rate(self, prec="fp32", stream=None) -> float:
        """Measured FMA rate of the device in flop/s (2 x FMAs per second):
        prec "fp32" for the FP32 pipe, "fp64" for the FP64 pipe."""
        v = ctypes.c_double()
        self._check(self.L.mb_measure_fma_rate(self.handle, _prec(prec), ctypes.byref(v),
                                               self._stream(stream)))
        return v.value

    def _dev(self, t, shape=None, dtype=None):
        torch = self._torch
        dtype = dtype or torch.float64
        if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
            raise ValueError(f"expected a contiguous {dtype} CUDA tensor")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
        return t

    # ------------------------------------------------------------ calls
    def mobility_matvec(self, r, f, a, eta=1.0, wall=True, prec="fp32", out=None, stream=None):
        """u = M(r) f.  r, f: (N, 3) float64, all on the GPU or all on the
        host (then the library stages them and returns after u is written)."""
        torch = self._torch
        n = int(r.shape[0])
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float64, device=r.device)
        for t in (r, f, out):
            if t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != (n, 3):
                raise ValueError("r, f, out must be contiguous float64 (N, 3)")
        st = self.L.mb_mobility_matvec(
            self.handle, _ptr(r), _ptr(f), n, float(a), float(eta), int(bool(wall)), _prec(prec),
            _ptr(out), self._stream(stream),
        )
        self._check(st)
        return out

    def blob_positions(self, q, theta, blob_start, rho, out=None, stream=None):
        torch = self._torch
        nb, n = int(q.shape[0]), int(rho.shape[0])
        self._dev(q, (nb, 3)); self._dev(theta, (nb, 4)); self._dev(rho, (n, 3))
        self._dev(blob_start, (nb + 1,), torch.int64)
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float64, device=q.device)
        self._check(self.L.mb_blob_positions(
            self.handle, nb, n, _ptr(q), _ptr(theta), _ptr(blob_start), _ptr(rho), _ptr(out),
            self._stream(stream)))
        return out

    def K_apply(self, r, q, blob_start, UO, out=None, stream=None):
        torch = self._torch
        nb, n = int(q.shape[0]), int(r.shape[0])
        self._dev(r, (n, 3)); self._dev(q, (nb, 3)); self._dev(UO, (nb, 6))
        self._dev(blob_start, (nb + 1,), torch.int64)
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float64, device=r.device)
        self._check(self.L.mb_K_apply(self.handle, nb, n, _ptr(r), _ptr(q), _ptr(blob_start),
                                      _ptr(UO), _ptr(out), self._stream(stream)))
        return out

    def KT_apply(self, r, q, blob_start, lam, out=None, stream=None):
        torch = self._torch
        nb, n = int(q.shape[0]), int(r.shape[0])
        self._dev(r, (n, 3)); self._dev(q, (nb, 3)); self._dev(lam, (n, 3))
        self._dev(blob_start, (nb + 1,), torch.int64)
        if out is None:
            out = torch.empty((nb, 6), dtype=torch.float64, device=r.device)
        self._check(self.L.mb_KT_apply(self.handle, nb, n, _ptr(r), _ptr(q), _ptr(blob_start),
                                       _ptr(lam), _ptr(out), self._stream(stream)))
        return out

    def mobility_eval(self, x, r, f, a, eta=1.0, wall=True, prec="fp32", out=None, stream=None):
        """Velocity at points x (n_points x 3) driven by blob forces f at r."""
        torch = self._torch
        nt, n = int(x.shape[0]), int(r.shape[0])
        self._dev(x, (nt, 3)); self._dev(r, (n, 3)); self._dev(f, (n, 3))
        if out is None:
            out = torch.empty((nt, 3), dtype=torch.float64, device=x.device)
        self._check(self.L.mb_mobility_eval(self.handle, _ptr(x), nt, _ptr(r), _ptr(f), n,
                                            float(a), float(eta), int(bool(wall)), _prec(prec),
                                            _ptr(out), self._stream(stream)))
        return out

    def render_flow(self, x, r, lam, sub_offsets, a_sub, eta=1.0, wall=True, prec="fp32",
                    out=None, stream=None):
        """Appendix B: flow at points x with every blob split into the
        sub_offsets (n_sub x 3) blobs of radius a_sub sharing its force."""
        torch = self._torch
        nt, n, ns = int(x.shape[0]), int(r.shape[0]), int(sub_offsets.shape[0])
        self._dev(x, (nt, 3)); self._dev(r, (n, 3)); self._dev(lam, (n, 3))
        self._dev(sub_offsets, (ns, 3))
        if out is None:
            out = torch.empty((nt, 3), dtype=torch.float64, device=x.device)
        self._check(self.L.mb_render_flow(self.handle, _ptr(x), nt, _ptr(r), _ptr(lam), n,
                                          _ptr(sub_offsets), ns, float(a_sub), float(eta),
                                          int(bool(wall)), _prec(prec), _ptr(out),
                                          self._stream(stream)))
        return out

    def lambda_moments(self, r, q, blob_start, lam, out=None, stream=None):
        """S_p = sum_i lambda_i (x) (r_i - q_p), one 3 x 3 matrix per body."""
        torch = self._torch
        nb, n = int(q.shape[0]), int(r.shape[0])
        self._dev(r, (n, 3)); self._dev(q, (nb, 3)); self._dev(lam, (n, 3))
        self._dev(blob_start, (nb + 1,), torch.int64)
        if out is None:
            out = torch.empty((nb, 3, 3), dtype=torch.float64, device=r.device)
        self._check(self.L.mb_lambda_moments(self.handle, nb, n, _ptr(r), _ptr(q), _ptr(blob_start),
                                             _ptr(lam), _ptr(out), self._stream(stream)))
        return out

    def precond_setup(self, r, q, blob_start, a, eta=1.0, wall=True, stream=None):
        torch = self._torch
        nb, n = int(q.shape[0]), int(r.shape[0])
        self._dev(r, (n, 3)); self._dev(q, (nb, 3))
        self._dev(blob_start, (nb + 1,), torch.int64)
        self._check(self.L.mb_precond_setup(self.handle, nb, n, _ptr(r), _ptr(q),
                                            _ptr(blob_start), float(a), float(eta),
                                            int(bool(wall)), self._stream(stream)))

    def precond_setup_shared(self, theta, blob_start, rho, a, eta=1.0, stream=None):
        """Unbounded-domain block preconditioner shared by bodies of the same
        shape (MB_PRECOND_FREE_SHARED), applied through each body's rotation."""
        torch = self._torch
        nb, n = int(theta.shape[0]), int(rho.shape[0])
        self._dev(theta, (nb, 4)); self._dev(rho, (n, 3))
        self._dev(blob_start, (nb + 1,), torch.int64)
        self._check(self.L.mb_precond_setup_shared(self.handle, nb, n, _ptr(theta),
                                                   _ptr(blob_start), _ptr(rho), float(a),
                                                   float(eta), self._stream(stream)))

    def precond_apply(self, w, g, stream=None):
        torch = self._torch
        lam = torch.empty_like(w)
        UO = torch.empty_like(g)
        self._dev(w); self._dev(g)
        self._check(self.L.mb_precond_apply(self.handle, _ptr(w), _ptr(g), _ptr(lam), _ptr(UO),
                                            self._stream(stream)))
        return lam, UO

    def solve_mobility(self, q, theta, blob_start, rho, F, T, a, eta=1.0, wall=True, slip=None,
                       tol=1e-10, maxit=200, restart=100, prec="fp64", stream=None,
                       raise_on_nonconvergence=True, precond="wall", shift=None):
        """Solve Eq. saddle_M; returns (U, Omega, lambda, info dict).
        precond: "wall" (per-body blocks with the wall) or "free_shared"
        (unbounded-domain blocks, one per body shape).  shift: per-blob
        kappa_p / (eta dV_i) of permeable bodies (Appendix C), or None."""
        torch = self._torch
        nb, n = int(q.shape[0]), int(rho.shape[0])
        self._dev(q, (nb, 3)); self._dev(theta, (nb, 4)); self._dev(rho, (n, 3))
        self._dev(F, (nb, 3)); self._dev(T, (nb, 3))
        self._dev(blob_start, (nb + 1,), torch.int64)
        if slip is not None:
            self._dev(slip, (n, 3))
        U = torch.empty((nb, 3), dtype=torch.float64, device=q.device)
        Om = torch.empty((nb, 3), dtype=torch.float64, device=q.device)
        lam = torch.empty((n, 3), dtype=torch.float64, device=q.device)
        p = Params(float(a), float(eta), int(bool(wall)), float(tol), int(maxit), int(restart),
                   _prec(prec), _precond(precond))
        info = Info()
        if shift is not None:
            self._dev(shift, (n,))
            st = self.L.mb_solve_mobility_permeable(
                self.handle, nb, n, _ptr(q), _ptr(theta), _ptr(blob_start), _ptr(rho), _ptr(F),
                _ptr(T), _ptr(slip), _ptr(shift), ctypes.byref(p), _ptr(U), _ptr(Om), _ptr(lam),
                ctypes.byref(info), self._stream(stream))
            if st == 4 and not raise_on_nonconvergence:
                return U, Om, lam, info.as_dict()
            self._check(st)
            return U, Om, lam, info.as_dict()
        st = self.L.mb_solve_mobility(
            self.handle, nb, n, _ptr(q), _ptr(theta), _ptr(blob_start), _ptr(rho), _ptr(F),
            _ptr(T), _ptr(slip), ctypes.byref(p), _ptr(U), _ptr(Om), _ptr(lam),
            ctypes.byref(info), self._stream(stream))
        if st == 4 and not raise_on_nonconvergence:
            return U, Om, lam, info.as_dict()
        self._check(st)
        return U, Om, lam, info.as_dict()

    def solve_resistance(self, q, theta, blob_start, rho, U, Omega, a, eta=1.0, wall=True,
                         slip=None, tol=1e-10, maxit=500, restart=100, prec="fp64", stream=None,
                         raise_on_nonconvergence=True, precond="wall"):
        """Solve Eq. resistance_problem; returns (F, T, lambda, info dict)."""
        torch = self._torch
        nb, n = int(q.shape[0]), int(rho.shape[0])
        self._dev(q, (nb, 3)); self._dev(theta, (nb, 4)); self._dev(rho, (n, 3))
        self._dev(U, (nb, 3)); self._dev(Omega, (nb, 3))
        self._dev(blob_start, (nb + 1,), torch.int64)
        if slip is not None:
            self._dev(slip, (n, 3))
        F = torch.empty((nb, 3), dtype=torch.float64, device=q.device)
        T = torch.empty((nb, 3), dtype=torch.float64, device=q.device)
        lam = torch.empty((n, 3), dtype=torch.float64, device=q.device)
        p = Params(float(a), float(eta), int(bool(wall)), float(tol), int(maxit), int(restart),
                   _prec(prec), _precond(precond))
        info = Info()
        st = self.L.mb_solve_resistance(
            self.handle, nb, n, _ptr(q), _ptr(theta), _ptr(blob_start), _ptr(rho), _ptr(U),
            _ptr(Omega), _ptr(slip), ctypes.byref(p), _ptr(F), _ptr(T), _ptr(lam),
            ctypes.byref(info), self._stream(stream))
        if st == 4 and not raise_on_nonconvergence:
            return F, T, lam, info.as_dict()
        self._check(st)
        return F, T, lam, info.as_dict()

    def solve_batch(self, problems, a, eta=1.0, wall=True, tol=1e-10, maxit=200, restart=100,
                    prec="mixed", stream=None, raise_on_nonconvergence=True):
        """Solve independent problems together (mb_solve_batch).

        problems: list of dicts with CUDA tensors q (n_b,3), theta (n_b,4),
        blob_start (n_b+1, int64), rho (N,3), F, T (n_b,3) and optional slip
        (N,3).  Returns a list of (U, Omega, lambda, info dict)."""
        torch = self._torch
        n = len(problems)
        arr = (Problem * max(1, n))()
        outs = []
        keep = []
        for k, P in enumerate(problems):
            nb, nbl = int(P["q"].shape[0]), int(P["rho"].shape[0])
            self._dev(P["q"], (nb, 3)); self._dev(P["theta"], (nb, 4)); self._dev(P["rho"], (nbl, 3))
            self._dev(P["F"], (nb, 3)); self._dev(P["T"], (nb, 3))
            self._dev(P["blob_start"], (nb + 1,), torch.int64)
            slip = P.get("slip")
            if slip is not None:
                self._dev(slip, (nbl, 3))
            dev = P["q"].device
            U = torch.empty((nb, 3), dtype=torch.float64, device=dev)
            Om = torch.empty((nb, 3), dtype=torch.float64, device=dev)
            lam = torch.empty((nbl, 3), dtype=torch.float64, device=dev)
            outs.append((U, Om, lam))
            keep.append(P)
            arr[k] = Problem(nb, nbl, P["q"].data_ptr(), P["theta"].data_ptr(),
                             P["blob_start"].data_ptr(), P["rho"].data_ptr(), P["F"].data_ptr(),
                             P["T"].data_ptr(), 0 if slip is None else slip.data_ptr(),
                             U.data_ptr(), Om.data_ptr(), lam.data_ptr())
        infos = (Info * max(1, n))()
        p = Params(float(a), float(eta), int(bool(wall)), float(tol), int(maxit), int(restart),
                   _prec(prec))
        st = self.L.mb_solve_batch(self.handle, n, arr, ctypes.byref(p), infos,
                                   self._stream(stream))
        if not (st == 4 and not raise_on_nonconvergence):
            self._check(st)
        return [(U, Om, lam, infos[k].as_dict()) for k, (U, Om, lam) in enumerate(outs)]


class Server:
    """Continuous-batching solver service on a context (mb_server_*).

    submit() queues a problem (dict of CUDA tensors as for
    Context.solve_batch) and returns a ticket; step() runs one scheduling
    tick; poll() reports (state, info, status) with state 0 queued,
    1 running, 2 done, 3 failed.  Results land in the tensors returned by
    submit(); keep the inputs alive until the ticket is done.  tick_pairs
    caps the pair evaluations one request's FP32 Arnoldi matvec takes per
    tick (0: 1e9, < 0: no cap); larger matvecs are spread over ticks.
    Admission takes every queued request that fits, in arrival order; one
    overtaken max_bypass times (0: 64, < 0: strict first come, first served)
    stops later ones until it is admitted.  finished() lists the tickets
    done since its last call."""

    QUEUED, RUNNING, DONE, FAILED = 0, 1, 2, 3

    def __init__(self, ctx, a, eta=1.0, wall=True, tol=1e-10, maxit=200, restart=60,
                 prec="mixed", max_blobs=1 << 20, max_bodies=1 << 16,
                 max_precond_bytes=4 << 30, max_requests=256, tick_pairs=0.0, max_bypass=0):
        self.ctx = ctx
        self.L = ctx.L
        self._torch = ctx._torch
        p = Params(float(a), float(eta), int(bool(wall)), float(tol), int(maxit), int(restart),
                   _prec(prec))
        lim = ServerLimits(int(max_blobs), int(max_bodies), int(max_precond_bytes),
                           int(max_requests), float(tick_pairs), int(max_bypass))
        h = ctypes.c_void_p()
        self._check(self.L.mb_server_create(ctx.handle, ctypes.byref(p), ctypes.byref(lim),
                                            ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def _check(self, st):
        if st != 0:
            raise MBError(st, self.L.mb_last_error(self.ctx.handle).decode())

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.L.mb_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, P):
        """Queue a problem; returns (ticket, (U, Omega, lambda) output tensors)."""
        torch = self._torch
        nb, nbl = int(P["q"].shape[0]), int(P["rho"].shape[0])
        dev = P["q"].device
        U = torch.empty((nb, 3), dtype=torch.float64, device=dev)
        Om = torch.empty((nb, 3), dtype=torch.float64, device=dev)
        lam = torch.empty((nbl, 3), dtype=torch.float64, device=dev)
        slip = P.get("slip")
        pr = Problem(nb, nbl, P["q"].data_ptr(), P["theta"].data_ptr(), P["blob_start"].data_ptr(),
                     P["rho"].data_ptr(), P["F"].data_ptr(), P["T"].data_ptr(),
                     0 if slip is None else slip.data_ptr(), U.data_ptr(), Om.data_ptr(),
                     lam.data_ptr())
        t = ctypes.c_int64()
        self._check(self.L.mb_server_submit(self.handle, ctypes.byref(pr), ctypes.byref(t)))
        self._keep[t.value] = (P, U, Om, lam)
        return t.value, (U, Om, lam)

    def step(self, stream=None):
        """One scheduling tick; returns (n_running, n_queued)."""
        nr, nq = ctypes.c_int(), ctypes.c_int()
        self._check(self.L.mb_server_step(self.handle, self.ctx._stream(stream), ctypes.byref(nr),
                                          ctypes.byref(nq)))
        return nr.value, nq.value

    def poll(self, ticket):
        st, res = ctypes.c_int(), ctypes.c_int()
        info = Info()
        self._check(self.L.mb_server_poll(self.handle, int(ticket), ctypes.byref(st),
                                          ctypes.byref(info), ctypes.byref(res)))
        if st.value in (self.DONE, self.FAILED):
            self._keep.pop(int(ticket), None)
        return st.value, info.as_dict(), STATUS.get(res.value, str(res.value))

    def finished(self, max_tickets=4096):
        """Tickets of the requests finished since the last call (oldest first)."""
        buf = (ctypes.c_int64 * max_tickets)()
        n = ctypes.c_int()
        out = []
        while True:
            self._check(self.L.mb_server_finished(self.handle, buf, max_tickets, ctypes.byref(n)))
            out.extend(buf[k] for k in range(n.value))
            if n.value < max_tickets:
                return out

    def run_until_idle(self, stream=None, max_ticks=1_000_000):
        for _ in range(max_ticks):
            nr, nq = self.step(stream)
            if nr == 0 and nq == 0:
                return
        raise RuntimeError("server did not drain")

