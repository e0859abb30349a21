"""GB300-native Kubo-formula anomalous Hall conductivity (Yahagi & Kato, arXiv 2309.06675).

Thin Python binding over the C ABI of ``libkubo.so`` (declared in include/kubo.h).  Every
step of the computation runs in the library's CUDA kernels; this module only marshals
arguments (device pointers of PyTorch tensors, host arrays, the current CUDA stream) and
maps status codes to exceptions.  There is no CPU fallback: if the library is missing
the import of a compute function raises.

Entry points (same names as the C ABI, without the ``kubo_`` prefix):
  ahc(H_R, R, kmesh, E_F, eta=..., etas=None, kT=0, ...)       -> S [n_eta, n_EF]
  ahc_host(H_R_np, R, kmesh, E_F_np, ...)                       -> numpy S (host in/out)
  ahc_k(H_R, R, kmesh, kidx, eta=..., etas=None)                -> (E [n_k, W], Omega [n_eta, n_k, W])
  bloch(H_R, R, kmesh, kidx)                                    -> packed H, dHx, dHy
  eigh_batched(A_packed, W)                                     -> (E, U)
  berry_batched(E, U, dHx_packed, dHy_packed, eta | etas)       -> Omega
  ahc_grad(H_R, R, kmesh, E_F, dL_dout, ...)                    -> G = dL/dH(R) (and S)
  AHC.apply(H_R, R, kmesh, E_F, eta, etas, kT)                  -> S, differentiable in H_R
  ahc_batched([(H_R, R, kmesh, E_F[, eta]), ...], ...)          -> [S per model], schedule
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "KuboError", "lib", "ahc", "ahc_host", "ahc_k", "bloch", "eigh_batched", "berry_batched",
    "workspace_size", "max_orbitals", "pack_hermitian", "unpack_hermitian", "FP64", "MIXED",
    "LIB_PATH", "Profile", "Options", "STAGES", "ahc_grad", "grad_workspace_size", "AHC",
    "ahc_batched", "Problem", "BatchSchedule", "MIXED_DF", "debug_fail_allocations",
]

FP64 = 0
MIXED = 1             # tensor-core Fourier sum, FP64 eigensolver, FP32 rotations
MIXED_FOURIER = 2     # error-budget mode: only the Fourier sum on the tensor cores
MIXED_ROTATION = 3    # error-budget mode: only the rotations in FP32
MIXED_DF = 4          # MIXED with the eigensolver in double-float (FP32 pairs) instead of FP64
_PREC = {"fp64": FP64, "mixed": MIXED, "mixed_fourier": MIXED_FOURIER,
         "mixed_rotation": MIXED_ROTATION, "mixed_df": MIXED_DF}
_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libkubo.so")

_STATUS = {
    0: "KUBO_OK", 1: "KUBO_ERR_INVALID_ARG", 2: "KUBO_ERR_NOT_HERMITIAN",
    3: "KUBO_ERR_R_NOT_CLOSED", 4: "KUBO_ERR_UNSUPPORTED", 5: "KUBO_ERR_OOM",
    6: "KUBO_ERR_CUDA", 7: "KUBO_ERR_NO_CONVERGENCE", 8: "KUBO_ERR_WORKSPACE",
    9: "KUBO_ERR_TIMEOUT",
}


class KuboError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = _STATUS.get(code, str(code))


STAGES = ("prep", "fourier", "tridiag", "ql", "backtransform", "berry", "ksum", "fixup", "adjoint")


class Profile(ctypes.Structure):
    """Per-stage launch counts and device milliseconds (kubo_profile of include/kubo.h)."""
    _fields_ = [("launches", ctypes.c_int64 * len(STAGES)), ("ms", ctypes.c_double * len(STAGES)),
                ("fixup_k", ctypes.c_int64)]

    def as_dict(self):
        return {s: {"launches": int(self.launches[i]), "ms": float(self.ms[i])}
                for i, s in enumerate(STAGES)}


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("n_eta", ctypes.c_int),
        ("etas", ctypes.POINTER(ctypes.c_double)),
        ("kT", ctypes.c_double),
        ("k_begin", ctypes.c_int64),
        ("k_end", ctypes.c_int64),
        ("stream", ctypes.c_void_p),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("chunk_k", ctypes.c_int),
        ("profile", ctypes.POINTER(Profile)),
        ("mixed_fixup_rel", ctypes.c_double),
        ("grad_eps", ctypes.c_double),
        ("layout_unpadded", ctypes.c_int),
        ("fourier_separable", ctypes.c_int),
        ("rotation_tc", ctypes.c_int),
        ("ql_max_sweeps", ctypes.c_int),
        ("ql_fp64", ctypes.c_int),
    ]


class Problem(ctypes.Structure):
    """kubo_problem of include/kubo.h (one model of a batched call)."""
    _fields_ = [
        ("H_R", ctypes.c_void_p), ("R_vecs", ctypes.c_void_p), ("W", ctypes.c_int),
        ("N_R", ctypes.c_int), ("kmesh", ctypes.c_int32 * 3), ("E_F", ctypes.c_void_p),
        ("n_EF", ctypes.c_int), ("eta", ctypes.c_double), ("out", ctypes.c_void_p),
        ("status", ctypes.c_int),
    ]


class BatchSchedule(ctypes.Structure):
    """kubo_batch_schedule of include/kubo.h."""
    _fields_ = [
        ("tune", ctypes.c_int), ("streams", ctypes.c_int), ("chunk_k", ctypes.c_int),
        ("graph", ctypes.c_int), ("probe_ms", ctypes.c_double), ("tuned_candidates", ctypes.c_int),
        ("fourier_group_m", ctypes.c_int), ("symv_parts", ctypes.c_int), ("rotation", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """The loaded libkubo (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libkubo.so not found at {LIB_PATH}; build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, D, V = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                           ctypes.c_void_p)
        OPT = ctypes.POINTER(Options)
        sig = {
            "kubo_options_init": (None, [OPT]),
            "kubo_status_string": (ctypes.c_char_p, [I]),
            "kubo_max_orbitals": (I, [I]),
            "kubo_workspace_size": (ctypes.c_size_t, [I, I, P, I, OPT]),
            "kubo_grad_workspace_size": (ctypes.c_size_t, [I, I, P, I, OPT]),
            "kubo_ahc_grad": (I, [P, P, I, I, P, P, I, D, P, P, P, OPT]),
            "kubo_ahc_batched": (I, [ctypes.POINTER(Problem), I, OPT, ctypes.POINTER(BatchSchedule)]),
            "kubo_check_bounded_wait": (I, [ctypes.c_uint32, P]),
            "kubo_debug_fail_allocations": (None, [I]),
            "kubo_ahc": (I, [P, P, I, I, P, P, I, D, P, OPT]),
            "kubo_ahc_host": (I, [P, P, I, I, P, P, I, D, P, OPT]),
            "kubo_ahc_k": (I, [P, P, I, I, P, P, I64, D, P, P, OPT]),
            "kubo_bloch": (I, [P, P, I, I, P, P, I64, P, P, P, OPT]),
            "kubo_eigh_batched": (I, [P, I, I64, P, P, OPT]),
            "kubo_berry_batched": (I, [P, P, P, P, I, I64, D, P, OPT]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int, what: str):
    if code != 0:
        msg = lib().kubo_status_string(code).decode()
        raise KuboError(code, f"{what}: {msg}")


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _host_int32(a, shape_last=None):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    if shape_last is not None and arr.shape[-1] != shape_last:
        raise ValueError(f"expected trailing dimension {shape_last}, got {arr.shape}")
    return arr


def _dev(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _options(precision=FP64, etas=None, kT=0.0, k_range=None, stream=None, chunk_k=0,
             workspace=None, keep=None, profile=None, ql_max_sweeps=0, ql_fp64=False):
    o = Options()
    lib().kubo_options_init(ctypes.byref(o))
    o.precision = _PREC.get(precision, precision)
    if etas is not None:
        e = np.ascontiguousarray(np.asarray(etas, dtype=np.float64).ravel())
        if keep is not None:
            keep.append(e)
        o.n_eta = int(e.size)
        o.etas = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    o.kT = float(kT)
    if k_range is not None:
        o.k_begin, o.k_end = int(k_range[0]), int(k_range[1])
    o.stream = _stream_ptr(stream)
    o.chunk_k = int(chunk_k)
    if workspace is not None:
        o.workspace = ctypes.c_void_p(workspace.data_ptr())
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    if profile is not None:
        o.profile = ctypes.pointer(profile)
    o.ql_max_sweeps = int(ql_max_sweeps)
    o.ql_fp64 = 1 if ql_fp64 else 0
    return o


_ROTATION = {"auto": 0, "exact": 1, "simt": 2, "tf32": 3}


def _rotation(rotation, rotation_tc=False) -> int:
    if rotation is None:
        return 1 if rotation_tc else 0
    return _ROTATION[rotation]


def debug_fail_allocations(n: int) -> None:
    """Make the library's next n device allocations fail as out-of-memory (test hook)."""
    lib().kubo_debug_fail_allocations(int(n))


def max_orbitals(precision=FP64) -> int:
    return int(lib().kubo_max_orbitals(_PREC.get(precision, precision)))


def workspace_size(W, N_R, kmesh, n_EF, precision=FP64, n_eta=1, kT=0.0, k_range=None,
                   chunk_k=0) -> int:
    km = _host_int32(kmesh)
    keep = []
    o = Options()
    lib().kubo_options_init(ctypes.byref(o))
    o.precision = _PREC.get(precision, precision)
    if n_eta > 1:
        e = np.full(n_eta, 1e-3)
        keep.append(e)
        o.n_eta = n_eta
        o.etas = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    o.kT = kT
    if k_range is not None:
        o.k_begin, o.k_end = k_range
    o.chunk_k = chunk_k
    return int(lib().kubo_workspace_size(int(W), int(N_R), km.ctypes.data_as(ctypes.c_void_p),
                                         int(n_EF), ctypes.byref(o)))


def ahc(H_R, R, kmesh, E_F, eta=1e-3, etas=None, kT=0.0, precision=FP64, k_range=None,
        stream=None, chunk_k=0, workspace=None, out=None, profile=None, fixup_rel=0.0,
        unpadded=False, separable=False, rotation_tc=False, ql_max_sweeps=0, rotation=None,
        ql_fp64=False):
    """S(E_F) for every broadening: returns a float64 CUDA tensor [n_eta, n_EF].

    ql_fp64 (MIXED): the QL iteration in FP64 too, its eigenvalues reported (default: QL shifts
    in double-float, eigenvalues the FP64 Rayleigh quotients of the FP64 eigenvectors).

    rotation: the FP32-grade step (3) kernel of the reduced modes, "auto" (the default:
    "tf32" above W = 40, else "simt"), "tf32" (tensor cores, 3xTF32), "exact" (tensor cores,
    exact BF16 slices; rotation_tc=True) or "simt" (FP32 FMA pipe).

    H_R: complex128 CUDA tensor [N_R, W, W]; R: host int [N_R, 3]; E_F: float64 CUDA [n_EF].
    """
    torch = _torch()
    Rh = _host_int32(R, 3)
    km = _host_int32(kmesh)
    N_R, W = int(H_R.shape[0]), int(H_R.shape[1])
    n_EF = int(E_F.numel())
    n_eta = 1 if etas is None else int(np.asarray(etas).size)
    if out is None:
        out = torch.empty((n_eta, n_EF), dtype=torch.float64, device=H_R.device)
    keep = []
    o = _options(precision, etas, kT, k_range, stream, chunk_k, workspace, keep, profile,
                 ql_max_sweeps, ql_fp64)
    o.mixed_fixup_rel = float(fixup_rel)
    o.layout_unpadded = 1 if unpadded else 0
    o.fourier_separable = 1 if separable else 0
    o.rotation_tc = _rotation(rotation, rotation_tc)
    code = lib().kubo_ahc(_dev(H_R, torch.complex128, "H_R"), Rh.ctypes.data_as(ctypes.c_void_p),
                          W, N_R, km.ctypes.data_as(ctypes.c_void_p),
                          _dev(E_F, torch.float64, "E_F"), n_EF, float(eta),
                          _dev(out, torch.float64, "out"), ctypes.byref(o))
    _check(code, "kubo_ahc")
    return out


def ahc_grad(H_R, R, kmesh, E_F, dL_dout, eta=1e-3, etas=None, kT=0.0, k_range=None,
             stream=None, chunk_k=0, workspace=None, profile=None, grad_eps=0.0,
             with_value=False):
    """Gradient G(R) = dL/dRe H(R) + i dL/dIm H(R) of L = sum dL_dout[e, j] S_e(E_F_j).

    dL_dout: float64 CUDA [n_eta, n_EF].  Returns a complex128 CUDA tensor [N_R, W, W]
    (and S [n_eta, n_EF] of the same call when with_value).  FP64.
    """
    torch = _torch()
    Rh = _host_int32(R, 3)
    km = _host_int32(kmesh)
    N_R, W = int(H_R.shape[0]), int(H_R.shape[1])
    n_EF = int(E_F.numel())
    n_eta = 1 if etas is None else int(np.asarray(etas).size)
    g = dL_dout.to(torch.float64).contiguous().reshape(n_eta, n_EF)
    G = torch.empty((N_R, W, W), dtype=torch.complex128, device=H_R.device)
    S = torch.empty((n_eta, n_EF), dtype=torch.float64, device=H_R.device) if with_value else None
    keep = []
    o = _options(FP64, etas, kT, k_range, stream, chunk_k, workspace, keep, profile)
    o.grad_eps = float(grad_eps)
    code = lib().kubo_ahc_grad(_dev(H_R, torch.complex128, "H_R"), Rh.ctypes.data_as(ctypes.c_void_p),
                               W, N_R, km.ctypes.data_as(ctypes.c_void_p),
                               _dev(E_F, torch.float64, "E_F"), n_EF, float(eta),
                               _dev(g, torch.float64, "dL_dout"), _dev(G, torch.complex128, "G"),
                               _dev(S, torch.float64, "out") if with_value else None,
                               ctypes.byref(o))
    _check(code, "kubo_ahc_grad")
    return (G, S) if with_value else G


def ahc_batched(problems, etas=None, kT=0.0, precision=FP64, stream=None, tune=False, streams=0,
                chunk_k=0, graph=True, fourier_group_m=0, symv_parts=0, rotation=0):
    """S(E_F) of many models in one call (kubo_ahc_batched).

    problems: sequence of (H_R complex128 CUDA [N_R, W, W], R host [N_R, 3], kmesh,
    E_F float64 CUDA [n_EF][, eta]).  Returns (list of float64 CUDA [n_eta, n_EF], schedule
    dict, list of per-model status names).  Raises KuboError if any model failed.
    """
    torch = _torch()
    n = len(problems)
    arr = (Problem * n)()
    keep, outs = [], []
    n_eta = 1 if etas is None else int(np.asarray(etas).size)
    for i, pr in enumerate(problems):
        H_R, R, kmesh, E_F = pr[:4]
        eta = float(pr[4]) if len(pr) > 4 else 1e-3
        Rh = _host_int32(R, 3)
        keep.append(Rh)
        out = torch.empty((n_eta, int(E_F.numel())), dtype=torch.float64, device=H_R.device)
        outs.append(out)
        a = arr[i]
        a.H_R = _dev(H_R, torch.complex128, "H_R")
        a.R_vecs = Rh.ctypes.data_as(ctypes.c_void_p)
        a.W, a.N_R = int(H_R.shape[1]), int(H_R.shape[0])
        for q in range(3):
            a.kmesh[q] = int(kmesh[q])
        a.E_F = _dev(E_F, torch.float64, "E_F")
        a.n_EF = int(E_F.numel())
        a.eta = eta
        a.out = _dev(out, torch.float64, "out")
        a.status = -1
    o = _options(precision, etas, kT, None, stream, 0, None, keep)
    sc = BatchSchedule()
    sc.tune = 1 if tune else 0
    sc.streams = int(streams)
    sc.chunk_k = int(chunk_k)
    sc.graph = 0 if graph else -1
    sc.fourier_group_m = int(fourier_group_m)
    sc.symv_parts = int(symv_parts)
    sc.rotation = _ROTATION[rotation] if isinstance(rotation, str) else int(rotation)
    code = lib().kubo_ahc_batched(arr, n, ctypes.byref(o), ctypes.byref(sc))
    status = [_STATUS.get(arr[i].status, str(arr[i].status)) for i in range(n)]
    _check(code, f"kubo_ahc_batched (per-model status: {status})")
    return outs, sc.as_dict(), status


def grad_workspace_size(W, N_R, kmesh, n_EF, n_eta=1, kT=0.0, k_range=None, chunk_k=0) -> int:
    km = _host_int32(kmesh)
    keep = []
    o = Options()
    lib().kubo_options_init(ctypes.byref(o))
    if n_eta > 1:
        e = np.full(n_eta, 1e-3)
        keep.append(e)
        o.n_eta = n_eta
        o.etas = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    o.kT = kT
    if k_range is not None:
        o.k_begin, o.k_end = k_range
    o.chunk_k = chunk_k
    return int(lib().kubo_grad_workspace_size(int(W), int(N_R), km.ctypes.data_as(ctypes.c_void_p),
                                              int(n_EF), ctypes.byref(o)))


def _make_autograd_function():
    torch = _torch()

    class _AHC(torch.autograd.Function):
        """S(E_F) = kubo_ahc(H_R, ...) with backward = kubo_ahc_grad (FP64).

        H_R must be Hermitian-paired (H(-R) = H(R)^dagger); its gradient is
        dL/dRe H(R) + i dL/dIm H(R), PyTorch's convention for complex inputs.
        """

        @staticmethod
        def forward(ctx, H_R, R, kmesh, E_F, eta=1e-3, etas=None, kT=0.0, k_range=None):
            ctx.save_for_backward(H_R, E_F)
            ctx.args = (R, kmesh, eta, etas, kT, k_range)
            return ahc(H_R.detach(), R, kmesh, E_F, eta=eta, etas=etas, kT=kT, k_range=k_range)

        @staticmethod
        def backward(ctx, grad_out):
            H_R, E_F = ctx.saved_tensors
            R, kmesh, eta, etas, kT, k_range = ctx.args
            G = ahc_grad(H_R.detach(), R, kmesh, E_F, grad_out.contiguous(), eta=eta, etas=etas,
                         kT=kT, k_range=k_range)
            return G, None, None, None, None, None, None, None

    return _AHC


class _LazyAHC:
    """Deferred torch.autograd.Function (torch is imported on first use)."""
    _fn = None

    def apply(self, *args):
        if _LazyAHC._fn is None:
            _LazyAHC._fn = _make_autograd_function()
        return _LazyAHC._fn.apply(*args)


AHC = _LazyAHC()


def ahc_host(H_R, R, kmesh, E_F, eta=1e-3, etas=None, kT=0.0, precision=FP64, k_range=None,
             stream=None, chunk_k=0, workspace=None, profile=None, separable=False):
    """Host-buffer variant: H_R complex128 numpy [N_R, W, W], E_F float64 numpy -> numpy S."""
    H = np.ascontiguousarray(H_R, dtype=np.complex128)
    EF = np.ascontiguousarray(E_F, dtype=np.float64).ravel()
    Rh = _host_int32(R, 3)
    km = _host_int32(kmesh)
    N_R, W = H.shape[0], H.shape[1]
    n_eta = 1 if etas is None else int(np.asarray(etas).size)
    out = np.empty((n_eta, EF.size), dtype=np.float64)
    keep = []
    o = _options(precision, etas, kT, k_range, stream, chunk_k, workspace, keep, profile)
    o.fourier_separable = 1 if separable else 0
    code = lib().kubo_ahc_host(H.ctypes.data_as(ctypes.c_void_p), Rh.ctypes.data_as(ctypes.c_void_p),
                               W, N_R, km.ctypes.data_as(ctypes.c_void_p),
                               EF.ctypes.data_as(ctypes.c_void_p), int(EF.size), float(eta),
                               out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o))
    _check(code, "kubo_ahc_host")
    return out


def ahc_k(H_R, R, kmesh, kidx, eta=1e-3, etas=None, precision=FP64, stream=None, chunk_k=0,
          rotation_tc=False, ql_max_sweeps=0, rotation=None, ql_fp64=False):
    """Per-k eigenvalues and band curvatures for the listed mesh points."""
    torch = _torch()
    Rh = _host_int32(R, 3)
    km = _host_int32(kmesh)
    N_R, W = int(H_R.shape[0]), int(H_R.shape[1])
    n_k = int(kidx.numel())
    n_eta = 1 if etas is None else int(np.asarray(etas).size)
    E = torch.empty((n_k, W), dtype=torch.float64, device=H_R.device)
    Om = torch.empty((n_eta, n_k, W), dtype=torch.float64, device=H_R.device)
    keep = []
    o = _options(precision, etas, 0.0, None, stream, chunk_k, None, keep,
                 ql_max_sweeps=ql_max_sweeps, ql_fp64=ql_fp64)
    o.rotation_tc = _rotation(rotation, rotation_tc)
    code = lib().kubo_ahc_k(_dev(H_R, torch.complex128, "H_R"), Rh.ctypes.data_as(ctypes.c_void_p),
                            W, N_R, km.ctypes.data_as(ctypes.c_void_p),
                            _dev(kidx, torch.int64, "kidx"), n_k, float(eta),
                            _dev(E, torch.float64, "E"), _dev(Om, torch.float64, "Omega"),
                            ctypes.byref(o))
    _check(code, "kubo_ahc_k")
    return E, Om


def bloch(H_R, R, kmesh, kidx, precision=FP64, stream=None):
    """Packed Hermitian H(k), d_x H(k), d_y H(k) [n_k, W*W] each (float64 CUDA).

    precision="mixed" evaluates the sum on the tensor cores (split-BF16, FP32 accumulation)."""
    torch = _torch()
    Rh = _host_int32(R, 3)
    km = _host_int32(kmesh)
    N_R, W = int(H_R.shape[0]), int(H_R.shape[1])
    n_k = int(kidx.numel())
    outs = [torch.empty((n_k, W * W), dtype=torch.float64, device=H_R.device) for _ in range(3)]
    o = _options(precision=precision, stream=stream)
    code = lib().kubo_bloch(_dev(H_R, torch.complex128, "H_R"), Rh.ctypes.data_as(ctypes.c_void_p),
                            W, N_R, km.ctypes.data_as(ctypes.c_void_p),
                            _dev(kidx, torch.int64, "kidx"), n_k,
                            *[_dev(x, torch.float64, "out") for x in outs], ctypes.byref(o))
    _check(code, "kubo_bloch")
    return tuple(outs)


def eigh_batched(A, W, vectors=True, stream=None, chunk_k=0, ql_max_sweeps=0):
    """Batched FP64 Hermitian eigh of packed matrices A [n, W*W] -> (E [n, W], U [n, W, W] or None)."""
    torch = _torch()
    n = int(A.shape[0])
    E = torch.empty((n, W), dtype=torch.float64, device=A.device)
    U = torch.empty((n, W, W), dtype=torch.complex128, device=A.device) if vectors else None
    o = _options(stream=stream, chunk_k=chunk_k, ql_max_sweeps=ql_max_sweeps)
    code = lib().kubo_eigh_batched(_dev(A, torch.float64, "A"), int(W), n, _dev(E, torch.float64, "E"),
                                   _dev(U, torch.complex128, "U") if vectors else None,
                                   ctypes.byref(o))
    _check(code, "kubo_eigh_batched")
    return E, U


def berry_batched(E, U, dHx, dHy, eta=1e-3, etas=None, stream=None):
    """Band Berry curvatures [n_eta, n, W] from eigenpairs and packed velocity matrices."""
    torch = _torch()
    n, W = int(E.shape[0]), int(E.shape[1])
    n_eta = 1 if etas is None else int(np.asarray(etas).size)
    Om = torch.empty((n_eta, n, W), dtype=torch.float64, device=E.device)
    keep = []
    o = _options(etas=etas, stream=stream, keep=keep)
    code = lib().kubo_berry_batched(_dev(E, torch.float64, "E"), _dev(U, torch.complex128, "U"),
                                    _dev(dHx, torch.float64, "dHx"), _dev(dHy, torch.float64, "dHy"),
                                    W, n, float(eta), _dev(Om, torch.float64, "Omega"),
                                    ctypes.byref(o))
    _check(code, "kubo_berry_batched")
    return Om


def pack_hermitian(A):
    """Packed Hermitian layout of include/kubo.h: P[i][j] = Re A_ij (i <= j), Im A_ji (i > j)."""
    torch = _torch()
    W = A.shape[-1]
    iu = torch.triu(torch.ones(W, W, dtype=torch.bool, device=A.device))
    re = A.real
    im_t = A.imag.transpose(-1, -2)
    return torch.where(iu, re, im_t).reshape(*A.shape[:-2], W * W).contiguous()


def unpack_hermitian(P, W):
    """Inverse of pack_hermitian: complex128 [..., W, W]."""
    torch = _torch()
    P = P.reshape(*P.shape[:-1], W, W)
    iu = torch.triu(torch.ones(W, W, dtype=torch.bool, device=P.device), diagonal=1)
    diag = torch.eye(W, dtype=torch.bool, device=P.device)
    Pt = P.transpose(-1, -2)
    re = torch.where(iu, P, torch.where(diag, P, Pt))
    im = torch.where(iu, Pt, torch.where(diag, torch.zeros_like(P), -P))
    return torch.complex(re, im)
