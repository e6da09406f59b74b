"""Python binding of libffgpu (ctypes).  Argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
turns torch tensors into pointers, leading dimensions and the current CUDA
stream, and turns status codes into exceptions.  PyTorch is used for device
memory and streams only.  There is no CPU fallback: if the library is missing
or a call fails, an exception is raised.

Tensors are row-major 2-D CUDA tensors of dtype torch.uint32 or torch.int32
(the bits are read as uint32 words) with unit stride along rows.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libffgpu.so")

STATUS = {
    0: "FFGPU_OK",
    -1: "FFGPU_ERR_INVALID",
    -2: "FFGPU_ERR_UNSUPPORTED_P",
    -3: "FFGPU_ERR_NOMEM",
    -4: "FFGPU_ERR_CUDA",
    -5: "FFGPU_ERR_TIMEOUT",
    -6: "FFGPU_ERR_BUDGET",
    -7: "FFGPU_ERR_SINGULAR",
}


class FFGPUError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__("%s%s" % (STATUS.get(status, "status %d" % status), (": " + what) if what else ""))


class PlanInfo(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("moduli", ctypes.c_uint32 * 16), ("k_chunk", ctypes.c_int32),
                ("k_slices", ctypes.c_int32), ("tile_m", ctypes.c_int32),
                ("tile_n", ctypes.c_int32), ("tile_k", ctypes.c_int32),
                ("mma_flops", ctypes.c_double)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("winograd_levels", ctypes.c_int32), ("unreduced", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


PATHS = {"rns": 0, "fp64": 1, "fp32": 2, "simt": 3}


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("side", ctypes.c_int32), ("uplo", ctypes.c_int32),
                ("diag", ctypes.c_int32), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("k", ctypes.c_int64), ("p", ctypes.c_uint32), ("alpha", ctypes.c_uint32),
                ("beta", ctypes.c_uint32), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("C_in", ctypes.c_void_p),
                ("ldc_in", ctypes.c_int64), ("out", ctypes.c_void_p), ("ldo", ctypes.c_int64),
                ("tag", ctypes.c_uint64)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("t_submit_us", ctypes.c_double),
                ("t_admit_us", ctypes.c_double), ("t_done_us", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "admitted", "completed", "failed", "pending",
                                               "inflight", "peak_inflight", "peak_bytes", "budget_bytes",
                                               "used_bytes")]


class Tuned(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("winograd_levels", ctypes.c_int32),
                ("chunk_steps", ctypes.c_int32), ("route", ctypes.c_int32), ("raster_rows", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3), ("ms", ctypes.c_double)]


class FgemmDesc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("p", ctypes.c_uint32), ("alpha", ctypes.c_uint32), ("beta", ctypes.c_uint32),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("B", ctypes.c_void_p),
                ("ldb", ctypes.c_int64), ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64)]


class MultimodDesc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("B", ctypes.c_void_p),
                ("ldb", ctypes.c_int64), ("C", ctypes.POINTER(ctypes.c_void_p)), ("ldc", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None

_I64, _U32, _VP, _I32 = ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int
# name -> argument types (restype is int status unless listed in _RESTYPES)
SIGNATURES = {
    "ffgpu_status_string": [_I32],
    "ffgpu_version": [],
    "ffgpu_fgemm": [_I64, _I64, _I64, _U32, _U32, _VP, _I64, _VP, _I64, _U32, _VP, _I64, _VP],
    "ffgpu_fgemm_workspace_size": [_I64, _I64, _I64, _U32, ctypes.POINTER(ctypes.c_size_t)],
    "ffgpu_fgemm_ws": [_I64, _I64, _I64, _U32, _U32, _VP, _I64, _VP, _I64, _U32, _VP, _I64,
                       _VP, ctypes.c_size_t, _VP],
    "ffgpu_fgemm_plan": [_I64, _I64, _I64, _U32, ctypes.POINTER(PlanInfo)],
    "ffgpu_last_device_error": [_VP],
    "ffgpu_release_workspaces": [],
    "ffgpu_fgemm_noalloc": [_I64, _I64, _I64, _U32, _U32, _VP, _I64, _VP, _I64, _U32, _VP, _I64, _VP],
    "ffgpu_fgemm_ex": [_I64, _I64, _I64, _U32, _U32, _VP, _I64, _VP, _I64, _U32, _VP, _I64,
                       ctypes.POINTER(Options), _VP],
    "ffgpu_server_create": [_I32, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)],
    "ffgpu_server_submit": [_VP, ctypes.POINTER(Request)],
    "ffgpu_server_poll": [_VP, ctypes.POINTER(Completion), _I32, ctypes.POINTER(ctypes.c_int), _I32],
    "ffgpu_server_get_stats": [_VP, ctypes.POINTER(ServerStats)],
    "ffgpu_server_destroy": [_VP],
    "ffgpu_fgemm_batched": [_I64, ctypes.POINTER(FgemmDesc), _VP],
    "ffgpu_fgemm_multimod_batched": [_I64, ctypes.POINTER(MultimodDesc), _I32, _I32, ctypes.POINTER(_U32), _VP],
    "ffgpu_fgemm_multimod": [_I64, _I64, _I64, _I32, _VP, _I64, _VP, _I64, _I32, ctypes.POINTER(_U32),
                             ctypes.POINTER(_VP), _I64, _VP],
    "ffgpu_fgemm_batched_plan_create": [_I64, ctypes.POINTER(FgemmDesc), ctypes.POINTER(_VP)],
    "ffgpu_fgemm_batched_plan_run": [_VP, _VP],
    "ffgpu_fgemm_batched_plan_error": [_VP],
    "ffgpu_fgemm_batched_plan_info": [_VP, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                      ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)],
    "ffgpu_fgemm_batched_plan_destroy": [_VP],
    "ffgpu_ftrsm": [_I32, _I32, _I32, _I64, _I64, _U32, _U32, _VP, _I64, _VP, _I64, _VP],
    "ffgpu_ftrsm_ex": [_I32, _I32, _I32, _I64, _I64, _U32, _U32, _VP, _I64, _VP, _I64, _I32, _VP],
    "ffgpu_ftrsm_cascade_params": [_U32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64)],
    "ffgpu_selftest_wait_timeout": [_I64, _VP],
    "ffgpu_autotune": [_I64, _I64, _I64, _U32, _I32, _VP, ctypes.POINTER(Tuned)],
    "ffgpu_autotune_lookup": [_I64, _I64, _I64, _U32, _I32, ctypes.POINTER(Tuned)],
    "ffgpu_autotune_save": [ctypes.c_char_p],
    "ffgpu_autotune_load": [ctypes.c_char_p],
    "ffgpu_autotune_clear": [],
    "ffgpu_autotune_batched": [_I64, ctypes.POINTER(FgemmDesc), _VP, ctypes.POINTER(ctypes.c_int64)],
    "ffgpu_fgemm_auto": [_I64, _I64, _I64, _U32, _U32, _VP, _I64, _VP, _I64, _U32, _VP, _I64, _I32, _VP],
    "ffgpu_profile_enable": [_I32],
    "ffgpu_profile_read": [ctypes.POINTER(KernelTime), _I32, ctypes.POINTER(ctypes.c_int)],
    "ffgpu_set_small_threshold": [_I64],
    "ffgpu_peak_probe": [_I32, _I64, ctypes.POINTER(ctypes.c_double), _VP],
    "ffgpu_winograd_unreduced_kmax": [_U32, _I32, ctypes.POINTER(ctypes.c_int64)],
    "ffgpu_get_small_threshold": [],
    "ffgpu_lqup": [_I64, _I64, _U32, _VP, _I64, ctypes.POINTER(ctypes.c_int64), _VP, _VP, _VP],
    "ffgpu_rank": [_I64, _I64, _U32, _VP, _I64, ctypes.POINTER(ctypes.c_int64), _VP],
    "ffgpu_det": [_I64, _U32, _VP, _I64, ctypes.POINTER(_U32), _VP],
    "ffgpu_inverse": [_I64, _U32, _VP, _I64, _VP, _I64, _VP],
}
_RESTYPES = {"ffgpu_status_string": ctypes.c_char_p, "ffgpu_get_small_threshold": ctypes.c_int64}


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libffgpu.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            for name, args in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = _RESTYPES.get(name, ctypes.c_int)
            _lib = L
    return _lib


def check(status: int, what: str = "") -> None:
    if status != 0:
        raise FFGPUError(status, what)


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _mat(t, name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype not in (torch.uint32, torch.int32):
        raise TypeError("%s must be uint32 or int32, got %s" % (name, t.dtype))
    if t.dim() != 2:
        raise ValueError("%s must be 2-D" % name)
    if t.numel() > 0 and t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError("%s must have unit stride along rows" % name)
    ld = t.stride(0) if t.shape[0] > 1 else max(t.shape[1], 1)
    return t.data_ptr(), max(ld, t.shape[1], 1)


def fgemm(A, B, p: int, alpha: int = 1, beta: int = 0, C=None, stream=None):
    """C <- (alpha*A@B + beta*C) mod p on the GPU; allocates C (zeros) if None. Returns C."""
    import torch
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ: %d vs %d" % (k, k2))
    if C is None:
        C = torch.zeros((m, n), dtype=torch.uint32, device=A.device)
        beta = 0
    if tuple(C.shape) != (m, n):
        raise ValueError("C has shape %s, expected %s" % (tuple(C.shape), (m, n)))
    a, lda = _mat(A, "A")
    b, ldb = _mat(B, "B")
    c, ldc = _mat(C, "C")
    check(lib().ffgpu_fgemm(m, n, k, p, alpha % 2**32, a, lda, b, ldb, beta % 2**32, c, ldc,
                            _stream_ptr(stream)), "ffgpu_fgemm")
    return C


def fgemm_ptr(m, n, k, p, alpha, A_ptr, lda, B_ptr, ldb, beta, C_ptr, ldc, stream_ptr=0) -> int:
    """The raw C-ABI call on device pointers; returns the status code."""
    return lib().ffgpu_fgemm(m, n, k, p, alpha, A_ptr, lda, B_ptr, ldb, beta, C_ptr, ldc, stream_ptr)


def fgemm_ex(A, B, p: int, alpha: int = 1, beta: int = 0, C=None, path: str = "rns",
             winograd_levels: int = 0, stream=None, unreduced: bool = False):
    """fgemm through a chosen arithmetic path ("rns", "fp64", "fp32", "simt") with
    `winograd_levels` levels of Winograd's variant; unreduced=True runs the
    levels over Z with one reduction at the end (Theorem 3.1's admission).
    Returns C."""
    import torch
    m, k = A.shape
    n = B.shape[1]
    if C is None:
        C = torch.zeros((m, n), dtype=torch.uint32, device=A.device)
        beta = 0
    a, lda = _mat(A, "A")
    b, ldb = _mat(B, "B")
    c, ldc = _mat(C, "C")
    opt = Options(PATHS[path], winograd_levels, 1 if unreduced else 0)
    check(lib().ffgpu_fgemm_ex(m, n, k, p, alpha % 2**32, a, lda, b, ldb, beta % 2**32, c, ldc,
                               ctypes.byref(opt), _stream_ptr(stream)), "ffgpu_fgemm_ex")
    return C


def fgemm_multimod(A, B, primes, bits: int, C=None, stream=None):
    """C_i = (A @ B) mod p_i for every p in primes, from ONE exact integer
    product (ffgpu_fgemm_multimod).  A (m x k) and B (k x n) are int32 CUDA
    tensors with |entries| <= 2^bits; returns the list of C_i (int32 tensors
    holding the residues in [0, p_i))."""
    import torch
    if A.dtype != torch.int32 or B.dtype != torch.int32:
        raise ValueError("A and B must be int32")
    m, k = A.shape
    if B.shape[0] != k:
        raise ValueError("inner dimensions differ")
    n = B.shape[1]
    primes = [int(p) for p in primes]
    if C is None:
        C = [torch.empty((m, n), dtype=torch.int32, device=A.device) for _ in primes]
    a, lda = _mat(A, "A")
    b, ldb = _mat(B, "B")
    ldc = None
    ptrs = []
    for Ci in C:
        if tuple(Ci.shape) != (m, n):
            raise ValueError("every C must be m x n")
        c, ldc_i = _mat(Ci, "C")
        if ldc is None:
            ldc = ldc_i
        elif ldc_i != ldc:
            raise ValueError("every C must have the same leading dimension")
        ptrs.append(c)
    if ldc is None:
        ldc = max(n, 1)
    parr = (_U32 * max(1, len(primes)))(*primes)
    carr = (_VP * max(1, len(ptrs)))(*ptrs)
    check(lib().ffgpu_fgemm_multimod(m, n, k, bits, a, lda, b, ldb, len(primes), parr, carr, ldc,
                                     _stream_ptr(stream)), "ffgpu_fgemm_multimod")
    return C


def multimod_descs(problems):
    """Host descriptors (ffgpu_multimod_desc[]) for problems (A, B, [C_1..C_P])
    of int32 A, B and int32 C_i CUDA tensors; returns (array, count, keep),
    `keep` holding the per-problem pointer arrays alive."""
    probs = list(problems)
    arr = (MultimodDesc * max(1, len(probs)))()
    keep = []
    for i, (A, B, Cs) in enumerate(probs):
        m, k = A.shape
        n = B.shape[1]
        a, lda = _mat(A, "A")
        b, ldb = _mat(B, "B")
        ptrs, ldc = [], None
        for Ci in Cs:
            c, l = _mat(Ci, "C")
            if ldc is None:
                ldc = l
            elif l != ldc:
                raise ValueError("problem %d: every C must have the same leading dimension" % i)
            ptrs.append(c)
        parr = (_VP * max(1, len(ptrs)))(*ptrs)
        keep.append(parr)
        arr[i] = MultimodDesc(m, n, k, a, lda, b, ldb, parr, ldc if ldc is not None else max(n, 1))
    return arr, len(probs), keep


def fgemm_multimod_batched_descs(descs, count: int, primes, bits: int, stream=None):
    """ffgpu_fgemm_multimod_batched on a prebuilt descriptor array (see multimod_descs)."""
    parr = (_U32 * max(1, len(primes)))(*[int(p) for p in primes])
    check(lib().ffgpu_fgemm_multimod_batched(count, descs, bits, len(primes), parr, _stream_ptr(stream)),
          "ffgpu_fgemm_multimod_batched")


def fgemm_multimod_batched(problems, primes, bits: int, stream=None):
    """For every (A, B, [C_1..C_P]): C_i = (A @ B) mod primes[i], one exact
    integer product per problem, all problems in grouped launches."""
    arr, n, keep = multimod_descs(problems)
    fgemm_multimod_batched_descs(arr, n, primes, bits, stream)
    del keep


def batched_descs(problems):
    """The host descriptor array (ffgpu_fgemm_desc[]) of a list of problems
    (A, B, C, p, alpha, beta) on CUDA tensors; it stays valid while the tensors
    live and can be passed to fgemm_batched_descs any number of times."""
    probs = list(problems)
    arr = (FgemmDesc * max(1, len(probs)))()
    for i, (A, B, C, p, alpha, beta) in enumerate(probs):
        m, k = A.shape
        n = B.shape[1]
        if B.shape[0] != k or tuple(C.shape) != (m, n):
            raise ValueError("problem %d: shapes %s %s %s do not match" % (i, tuple(A.shape), tuple(B.shape), tuple(C.shape)))
        a, lda = _mat(A, "A")
        b, ldb = _mat(B, "B")
        c, ldc = _mat(C, "C")
        arr[i] = FgemmDesc(m, n, k, p, alpha % 2**32, beta % 2**32, a, lda, b, ldb, c, ldc)
    return arr, len(probs)


def fgemm_batched_descs(descs, count: int, stream=None):
    """ffgpu_fgemm_batched on a prebuilt descriptor array (see batched_descs)."""
    check(lib().ffgpu_fgemm_batched(count, descs, _stream_ptr(stream)), "ffgpu_fgemm_batched")


def fgemm_batched(problems, stream=None):
    """problems: iterable of (A, B, C, p, alpha, beta) with CUDA tensors; every
    C <- (alpha*A@B + beta*C) mod p, all in one batched call. Returns the Cs."""
    probs = list(problems)
    arr, count = batched_descs(probs)
    fgemm_batched_descs(arr, count, stream)
    return [pr[2] for pr in probs]


TRSM_ALGORITHMS = {"default": -1, "recursive": 0, "delayed": 1, "cascade": 2}


def ftrsm_cascade_params(p: int) -> dict:
    """t_del, t_update and t_split of the double cascade (Algorithms 2-3) for p."""
    a, b, c = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    check(lib().ffgpu_ftrsm_cascade_params(p, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
          "ffgpu_ftrsm_cascade_params")
    return {"t_del": a.value, "t_update": b.value, "t_split": c.value}


def ftrsm(T, B, p: int, alpha: int = 1, side: str = "L", uplo: str = "L", diag: str = "U", stream=None,
          algorithm: str = "default"):
    """In place: B <- alpha*T^{-1}*B (side "L") or alpha*B*T^{-1} (side "R") mod p. Returns B.
    algorithm: "recursive" (Algorithm 1), "delayed" (left-looking, one reduction
    per block), "cascade" (Algorithms 2-3: updates and leaves over Z) or
    "default"."""
    m, n = B.shape
    nt = m if side == "L" else n
    if tuple(T.shape) != (nt, nt):
        raise ValueError("T must be %d x %d" % (nt, nt))
    t, ldt = _mat(T, "T")
    b, ldb = _mat(B, "B")
    check(lib().ffgpu_ftrsm_ex(0 if side == "L" else 1, 0 if uplo == "L" else 1, 1 if diag == "U" else 0,
                               m, n, p, alpha % 2**32, t, ldt, b, ldb, TRSM_ALGORITHMS[algorithm],
                               _stream_ptr(stream)), "ffgpu_ftrsm_ex")
    return B


def set_small_threshold(max_macs: int) -> None:
    """Products with m*n*k <= max_macs run on the CUDA cores (0: none)."""
    check(lib().ffgpu_set_small_threshold(max_macs), "ffgpu_set_small_threshold")


PEAK_KINDS = {"int8": 0, "bf16": 1, "fp64": 2}


def peak_probe(kind: str = "int8", iters: int = 100000, stream=None) -> float:
    """Measured peak of a warp-level MMA unit (mma.sync), in operations/s."""
    out = ctypes.c_double(0.0)
    check(lib().ffgpu_peak_probe(PEAK_KINDS[kind], iters, ctypes.byref(out), _stream_ptr(stream)),
          "ffgpu_peak_probe")
    return float(out.value)


def winograd_unreduced_kmax(p: int, levels: int) -> int:
    """Largest k that `levels` unreduced Winograd levels admit for p (0: none)."""
    out = ctypes.c_int64(0)
    check(lib().ffgpu_winograd_unreduced_kmax(p, levels, ctypes.byref(out)), "ffgpu_winograd_unreduced_kmax")
    return int(out.value)


def get_small_threshold() -> int:
    return int(lib().ffgpu_get_small_threshold())


def lqup(A, p: int, stream=None):
    """In-place packed LQUP of A mod p (p prime): afterwards
    A[rowperm][:, colperm] = L U, L strictly below the diagonal of A's first r
    columns (unit diagonal implied), U on and above the diagonal of its first
    r rows.  Returns (r, rowperm, colperm), the permutations as int32 CUDA
    tensors.  Host-synchronous."""
    import torch
    m, n = A.shape
    a, lda = _mat(A, "A")
    rowperm = torch.empty(m, dtype=torch.int32, device=A.device)
    colperm = torch.empty(n, dtype=torch.int32, device=A.device)
    r = ctypes.c_int64(0)
    check(lib().ffgpu_lqup(m, n, p, a, lda, ctypes.byref(r), rowperm.data_ptr(), colperm.data_ptr(),
                           _stream_ptr(stream)), "ffgpu_lqup")
    return int(r.value), rowperm, colperm


def rank(A, p: int, stream=None) -> int:
    """Rank of A mod p (p prime); A is not modified."""
    m, n = A.shape
    a, lda = _mat(A, "A")
    r = ctypes.c_int64(0)
    check(lib().ffgpu_rank(m, n, p, a, lda, ctypes.byref(r), _stream_ptr(stream)), "ffgpu_rank")
    return int(r.value)


def det(A, p: int, stream=None) -> int:
    """Determinant of the square matrix A mod p (p prime), in [0, p)."""
    n, n2 = A.shape
    if n != n2:
        raise ValueError("det needs a square matrix")
    a, lda = _mat(A, "A")
    d = ctypes.c_uint32(0)
    check(lib().ffgpu_det(n, p, a, lda, ctypes.byref(d), _stream_ptr(stream)), "ffgpu_det")
    return int(d.value)


def inverse(A, p: int, X=None, stream=None):
    """A^{-1} mod p (p prime) into X (allocated if None); raises FFGPUError
    with FFGPU_ERR_SINGULAR (-7) if A is singular mod p.  Returns X."""
    import torch
    n, n2 = A.shape
    if n != n2:
        raise ValueError("inverse needs a square matrix")
    if X is None:
        X = torch.zeros((n, n), dtype=torch.uint32, device=A.device)
    a, lda = _mat(A, "A")
    x, ldx = _mat(X, "X")
    check(lib().ffgpu_inverse(n, p, a, lda, x, ldx, _stream_ptr(stream)), "ffgpu_inverse")
    return X


def fgemm_noalloc_ptr(m, n, k, p, alpha, A_ptr, lda, B_ptr, ldb, beta, C_ptr, ldc, stream_ptr=0) -> int:
    """ffgpu_fgemm_noalloc on device pointers (scratch from the library's static
    device array, no allocation); returns the status code."""
    return lib().ffgpu_fgemm_noalloc(m, n, k, p, alpha, A_ptr, lda, B_ptr, ldb, beta, C_ptr, ldc,
                                     stream_ptr)


def fgemm_workspace_size(m, n, k, p) -> int:
    out = ctypes.c_size_t(0)
    check(lib().ffgpu_fgemm_workspace_size(m, n, k, p, ctypes.byref(out)), "workspace_size")
    return out.value


def fgemm_ws(A, B, p, alpha, beta, C, workspace, stream=None):
    """ffgpu_fgemm_ws with a caller-owned workspace tensor (any dtype, contiguous, CUDA)."""
    m, k = A.shape
    n = B.shape[1]
    a, lda = _mat(A, "A")
    b, ldb = _mat(B, "B")
    c, ldc = _mat(C, "C")
    nbytes = workspace.numel() * workspace.element_size()
    check(lib().ffgpu_fgemm_ws(m, n, k, p, alpha % 2**32, a, lda, b, ldb, beta % 2**32, c, ldc,
                               workspace.data_ptr(), nbytes, _stream_ptr(stream)), "ffgpu_fgemm_ws")
    return C


def fgemm_plan(m: int, n: int, k: int, p: int) -> dict:
    info = PlanInfo()
    check(lib().ffgpu_fgemm_plan(m, n, k, p, ctypes.byref(info)), "plan")
    return dict(mode=info.mode, channels=info.channels, moduli=list(info.moduli[: info.channels]),
                k_chunk=info.k_chunk, k_slices=info.k_slices,
                tile=(info.tile_m, info.tile_n, info.tile_k), mma_flops=info.mma_flops)


def last_device_error(stream=None) -> int:
    return lib().ffgpu_last_device_error(_stream_ptr(stream))


def selftest_wait_timeout(limit_cycles: int = 2_000_000, stream=None) -> None:
    """Launch the bounded-wait self-test kernel (see include/ffgpu.h)."""
    check(lib().ffgpu_selftest_wait_timeout(limit_cycles, _stream_ptr(stream)), "selftest_wait_timeout")


def release_workspaces() -> None:
    check(lib().ffgpu_release_workspaces(), "release_workspaces")


def status_string(code: int) -> str:
    return lib().ffgpu_status_string(code).decode()


def version() -> int:
    return lib().ffgpu_version()


def profile_enable(on: bool = True) -> None:
    """Record CUDA events around every library kernel launch (on its stream)."""
    check(lib().ffgpu_profile_enable(1 if on else 0), "profile_enable")


def profile_read() -> dict:
    """{kernel name: (launches, total ms)} since the last read; synchronizes the events."""
    cap = 64
    arr = (KernelTime * cap)()
    cnt = ctypes.c_int(0)
    check(lib().ffgpu_profile_read(arr, cap, ctypes.byref(cnt)), "profile_read")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(cnt.value, cap))}


class BatchedPlan:
    """A fixed batch of fgemms captured once in a CUDA graph
    (ffgpu_fgemm_batched_plan_*): run() recomputes every C from the current
    contents of its A, B and C.  The tensors are kept alive by the plan."""

    def __init__(self, problems):
        self._problems = list(problems)
        self._descs, n = batched_descs(self._problems)
        self._h = _VP()
        check(lib().ffgpu_fgemm_batched_plan_create(n, self._descs, ctypes.byref(self._h)),
              "ffgpu_fgemm_batched_plan_create")

    def run(self, stream=None):
        check(lib().ffgpu_fgemm_batched_plan_run(self._h, _stream_ptr(stream)), "ffgpu_fgemm_batched_plan_run")

    def error(self) -> int:
        """Synchronizes; the plan's device error word (0 = none), cleared."""
        return int(lib().ffgpu_fgemm_batched_plan_error(self._h))

    def info(self) -> dict:
        w, sg = _I32(0), _I32(0)
        nodes, nbytes = ctypes.c_size_t(0), ctypes.c_size_t(0)
        check(lib().ffgpu_fgemm_batched_plan_info(self._h, ctypes.byref(w), ctypes.byref(sg), ctypes.byref(nodes),
                                                  ctypes.byref(nbytes)), "ffgpu_fgemm_batched_plan_info")
        return {"waves": w.value, "singles": sg.value, "graph_nodes": nodes.value, "device_bytes": nbytes.value}

    def close(self):
        if self._h:
            lib().ffgpu_fgemm_batched_plan_destroy(self._h)
            self._h = _VP()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (ffgpu_server_*).  Operands are host
    numpy arrays (uint32, C-contiguous rows; pinned memory overlaps better);
    the caller keeps them alive until the request's completion is polled."""

    def __init__(self, streams: int = 4, budget_bytes: int = 40 << 30):
        h = ctypes.c_void_p()
        check(lib().ffgpu_server_create(streams, budget_bytes, ctypes.byref(h)), "server_create")
        self.h = h

    def submit_fgemm(self, A, B, out, p, alpha=1, beta=0, C=None, tag=0):
        r = Request(kind=0, m=A.shape[0], n=B.shape[1], k=A.shape[1], p=p, alpha=alpha % 2**32,
                    beta=beta % 2**32, A=A.ctypes.data, lda=A.strides[0] // 4, B=B.ctypes.data,
                    ldb=B.strides[0] // 4, C_in=C.ctypes.data if C is not None else None,
                    ldc_in=(C.strides[0] // 4) if C is not None else 0, out=out.ctypes.data,
                    ldo=out.strides[0] // 4, tag=tag)
        check(lib().ffgpu_server_submit(self.h, ctypes.byref(r)), "server_submit")

    def submit_ftrsm(self, T, B, out, p, alpha=1, side="L", uplo="L", diag="U", tag=0):
        r = Request(kind=1, side=0 if side == "L" else 1, uplo=0 if uplo == "L" else 1,
                    diag=1 if diag == "U" else 0, m=B.shape[0], n=B.shape[1], k=0, p=p,
                    alpha=alpha % 2**32, beta=0, A=T.ctypes.data, lda=T.strides[0] // 4,
                    B=B.ctypes.data, ldb=B.strides[0] // 4, out=out.ctypes.data,
                    ldo=out.strides[0] // 4, tag=tag)
        check(lib().ffgpu_server_submit(self.h, ctypes.byref(r)), "server_submit")

    def poll(self, wait_ms: int = 0, cap: int = 256):
        arr = (Completion * cap)()
        cnt = ctypes.c_int(0)
        check(lib().ffgpu_server_poll(self.h, arr, cap, ctypes.byref(cnt), wait_ms), "server_poll")
        return [(int(arr[i].tag), int(arr[i].status), arr[i].t_submit_us, arr[i].t_admit_us, arr[i].t_done_us)
                for i in range(cnt.value)]

    def stats(self) -> dict:
        st = ServerStats()
        check(lib().ffgpu_server_get_stats(self.h, ctypes.byref(st)), "server_stats")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            check(lib().ffgpu_server_destroy(self.h), "server_destroy")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


_KERNELS = {-1: "default", 0: "single", 1: "pair"}
_ROUTES = {-1: "default", 0: "tensor", 1: "cuda_cores"}


def _tuned(t: "Tuned") -> dict:
    return dict(kernel=_KERNELS.get(t.kernel, t.kernel), winograd_levels=t.winograd_levels,
                chunk_steps=t.chunk_steps, route=_ROUTES.get(t.route, t.route), raster_rows=t.raster_rows,
                ms=t.ms)


def autotune_batched(descs, count: int, stream=None) -> int:
    """Time the batch (a prebuilt descriptor array, see batched_descs) for the
    batched launch's CUDA-core threshold; keep and return the fastest.  Every
    C receives alpha*A@B (beta taken as 0)."""
    out = ctypes.c_int64(0)
    check(lib().ffgpu_autotune_batched(count, descs, _stream_ptr(stream), ctypes.byref(out)), "autotune_batched")
    return out.value


def autotune(m: int, n: int, k: int, p: int, path: str = "rns", stream=None) -> dict:
    """Time the candidate plans for this problem class on the device; cache and return the best."""
    t = Tuned()
    check(lib().ffgpu_autotune(m, n, k, p, PATHS[path], _stream_ptr(stream), ctypes.byref(t)), "autotune")
    return _tuned(t)


def autotune_lookup(m: int, n: int, k: int, p: int, path: str = "rns"):
    """The cached plan for this problem class, or None."""
    t = Tuned()
    if lib().ffgpu_autotune_lookup(m, n, k, p, PATHS[path], ctypes.byref(t)) != 0:
        return None
    return _tuned(t)


def autotune_save(path: str) -> None:
    check(lib().ffgpu_autotune_save(path.encode()), "autotune_save")


def autotune_load(path: str) -> None:
    check(lib().ffgpu_autotune_load(path.encode()), "autotune_load")


def autotune_clear() -> None:
    check(lib().ffgpu_autotune_clear(), "autotune_clear")


def fgemm_auto(A, B, p: int, alpha: int = 1, beta: int = 0, C=None, path: str = "rns", stream=None):
    """fgemm with the autotuned plan for its problem class (tuning on a cache miss)."""
    import torch
    m, k = A.shape
    n = B.shape[1]
    if C is None:
        C = torch.zeros((m, n), dtype=torch.uint32, device=A.device)
        beta = 0
    a, lda = _mat(A, "A")
    b, ldb = _mat(B, "B")
    c, ldc = _mat(C, "C")
    check(lib().ffgpu_fgemm_auto(m, n, k, p, alpha % 2**32, a, lda, b, ldb, beta % 2**32, c, ldc,
                                 PATHS[path], _stream_ptr(stream)), "ffgpu_fgemm_auto")
    return C
