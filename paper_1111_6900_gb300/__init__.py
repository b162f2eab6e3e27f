"""Python binding of the GB300 GF(2^e) bitsliced matmul library (libm4rie_gpu.so).

Thin argument marshalling over the C ABI declared in include/m4rie_gpu.h: the
functions keep the C names, take torch CUDA tensors (for device memory and
streams) and pass raw pointers.  Every step of the computation runs in the
library's CUDA kernels; there is no CPU fallback.  Importing this package
without the built library raises ImportError.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libm4rie_gpu.so")

(OK, ERR_ARG, ERR_POLY, ERR_ALIAS, ERR_RANGE, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_SCRATCH,
 ERR_SINGULAR) = range(11)
FORM_AUTO, FORM_POPC, FORM_TC_F8, FORM_MMA_S8, FORM_TC_F4, FORM_MMA_B1, FORM_NEWTON_JOHN = range(7)
SCHED_AUTO, SCHED_ALPHA_B, SCHED_KARATSUBA = range(3)
FORMS = {"auto": FORM_AUTO, "popc": FORM_POPC, "tc_f8": FORM_TC_F8, "mma_s8": FORM_MMA_S8, "tc_f4": FORM_TC_F4,
         "mma_b1": FORM_MMA_B1, "newton_john": FORM_NEWTON_JOHN}
SCHEDULES = {"auto": SCHED_AUTO, "alpha_b": SCHED_ALPHA_B, "karatsuba": SCHED_KARATSUBA}


class M4rieError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {status_string(status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class _Problem(ctypes.Structure):
    _fields_ = [("e", ctypes.c_int32), ("f", ctypes.c_uint32), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("k", ctypes.c_int64), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("accumulate", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
                          "(needs nvcc for sm_103a)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, u32, i64, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "m4rie_create": (i32, [ctypes.POINTER(vp), vp]),
        "m4rie_destroy": (None, [vp]),
        "m4rie_set_form": (i32, [vp, i32]),
        "m4rie_set_schedule": (i32, [vp, i32]),
        "m4rie_mul": (i32, [vp, i32, u32, i64, i64, i64, vp, vp, vp]),
        "m4rie_addmul": (i32, [vp, i32, u32, i64, i64, i64, vp, vp, vp]),
        "m4rie_gemm": (i32, [vp, i32, u32, i64, i64, i64, vp, i64, vp, i64, vp, i64, i32]),
        "m4rie_trsm_upper_left": (i32, [vp, i32, u32, i64, i64, vp, i64, vp, i64]),
        "m4rie_trsm_lower_left": (i32, [vp, i32, u32, i64, i64, vp, i64, vp, i64]),
        "m4rie_echelonize": (i32, [vp, i32, u32, i64, i64, vp, i64, ctypes.POINTER(i64), vp]),
        "m4rie_ple": (i32, [vp, i32, u32, i64, i64, vp, i64, ctypes.POINTER(i64), vp, vp]),
        "m4rie_mul_host": (i32, [vp, i32, u32, i64, i64, i64, vp, vp, vp, i32]),
        "m4rie_pack": (i32, [vp, i32, i64, i64, vp, vp, i64]),
        "m4rie_unpack": (i32, [vp, i32, i64, i64, vp, i64, vp]),
        "m4rie_mul_batched": (i32, [vp, i32, vp]),
        "m4rie_packed_width": (i32, [i32]),
        "m4rie_to_packed": (i32, [vp, i32, i64, i64, vp, i64, vp, i64]),
        "m4rie_from_packed": (i32, [vp, i32, i64, i64, vp, i64, vp, i64]),
        "m4rie_mul_packed": (i32, [vp, i32, u32, i64, i64, i64, vp, i64, vp, i64, vp, i64, i32]),
        "m4rie_get_device_status": (i32, [vp]),
        "m4rie_schedule_products": (i32, [i32, u32, i32]),
        "m4rie_schedule_masks": (i32, [i32, u32, i32, i32, vp, vp, vp]),
        "m4rie_validate": (i32, [i32, u32, i64, i64, i64, vp, vp, vp]),
        "m4rie_resolve_form": (i32, [vp, i32, i64, i64, i64]),
        "m4rie_status_string": (ctypes.c_char_p, [i32]),
        "m4rie_last_error": (ctypes.c_char_p, [vp]),
        "m4rie_kernel_launches": (i64, [vp]),
        "m4rie_set_wait_limit_ns": (i32, [vp, u64]),
        "m4rie_enable_timing": (i32, [vp, i32]),
        "m4rie_mul_noalloc": (i32, [i32, u32, i64, i64, i64, vp, vp, vp, i32, vp, vp]),
        "m4rie_tune": (i32, [vp, i32, u32, i64, i64, i64]),
        "m4rie_tune_batched": (i32, [vp, i32, vp]),
        "m4rie_set_test_hook": (i32, [vp, i32]),
        "m4rie_tuned_choice": (i32, [vp, i32, i64, i64, i64, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                     ctypes.POINTER(ctypes.c_double)]),
        "m4rie_tune_save": (i32, [vp, ctypes.c_char_p]),
        "m4rie_tune_load": (i32, [vp, ctypes.c_char_p]),
        "m4rie_phase_times": (i32, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64), i32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


lib = _load()


def status_string(status: int) -> str:
    return lib.m4rie_status_string(int(status)).decode()


def elem_dtype_torch(e: int):
    import torch
    return torch.uint8 if e <= 8 else torch.uint16


def _ptr(t):
    return None if t is None or t.numel() == 0 else ctypes.c_void_p(t.data_ptr())


def _host_matrix(x, e, name, shape, writable=False):
    """Address of a host matrix for the host-buffer entry point: a torch CPU
    tensor or a numpy array, 2-D of the given shape, C-contiguous, one integer
    element of the field's width per entry (1 byte for e <= 8, 2 for e > 8).
    None for a matrix without entries."""
    import numpy as np
    width = 1 if e <= 8 else 2
    if hasattr(x, "data_ptr"):
        import torch
        if x.device.type != "cpu":
            raise TypeError(f"{name} must be a host tensor (device tensors go through mul / addmul)")
        integer = not (x.dtype.is_floating_point or x.dtype.is_complex or x.dtype == torch.bool)
        size, contiguous, ok_write, addr = x.element_size(), x.is_contiguous(), True, x.data_ptr()
    elif isinstance(x, np.ndarray):
        integer = x.dtype.kind in "ui"
        size, contiguous, ok_write, addr = x.itemsize, x.flags.c_contiguous, x.flags.writeable, x.ctypes.data
    else:
        raise TypeError(f"{name} must be a torch CPU tensor or a numpy array")
    if tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name} must be {shape[0]} x {shape[1]}, not {tuple(x.shape)}")
    if not integer or size != width:
        raise TypeError(f"{name} must hold {8 * width}-bit integers for e = {e}")
    if not contiguous:
        raise ValueError(f"{name} must be C-contiguous (row-major)")
    if writable and not ok_write:
        raise ValueError(f"{name} must be writable")
    return ctypes.c_void_p(addr) if shape[0] * shape[1] else None


def _fields_per_word(e: int) -> int:
    """Fields of the packed representation per 64-bit word."""
    w = packed_width(e)
    if w <= 0:
        raise ValueError(f"e = {e} is outside 2..10")
    return 64 // w


def _check_words(t, name, dims):
    """A contiguous CUDA tensor of 64-bit words with `dims` dimensions."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.element_size() != 8 or t.is_floating_point():
        raise TypeError(f"{name} must be a CUDA tensor of 64-bit words")
    if t.dim() != dims or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dims}-D tensor")


def _check_word_window(t, name):
    """A 2-D CUDA tensor of 64-bit words with unit column stride (any row stride)."""
    if not t.is_cuda or t.dtype.itemsize != 8 or t.dim() != 2 or (t.shape[1] > 1 and t.stride(1) != 1):
        raise TypeError(f"{name} must be a 2-D CUDA tensor of 64-bit words with unit column stride")


def _check_dev(t, e, name, strided=False):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != elem_dtype_torch(e):
        raise TypeError(f"{name} must be {elem_dtype_torch(e)} for e = {e}")
    if strided:
        if t.dim() != 2 or (t.numel() and t.shape[1] > 1 and t.stride(1) != 1):
            raise ValueError(f"{name} must be a 2-D window with unit column stride")
    elif not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous (row-major)")


def _ld(t):
    """Row stride of a 2-D window (elements); any value >= its width is valid for one row."""
    return max(int(t.stride(0)), int(t.shape[1])) if t.shape[0] > 1 else int(t.shape[1])


def problem_array(problems):
    """The m4rie_problem array of a list of (e, f, A, B, C, accumulate) with
    CUDA tensors; mul_batched and tune_batched also take such an array, so
    that a batch replayed many times is marshalled once."""
    arr = (_Problem * len(problems))()
    for i, (e, f, A, B, C, acc) in enumerate(problems):
        for t, nm in ((A, "A"), (B, "B"), (C, "C")):
            _check_dev(t, e, f"{nm} of problem {i}")
        m, k = A.shape
        k2, n = B.shape
        if k2 != k or tuple(C.shape) != (m, n):
            raise ValueError(f"problem {i}: shapes do not match (A m x k, B k x n, C m x n)")
        arr[i] = _Problem(e, f, m, n, k, A.data_ptr(), B.data_ptr(), C.data_ptr(), 1 if acc else 0, 0)
    return arr


class Context:
    """An m4rie_ctx bound to the current device and a torch CUDA stream."""

    def __init__(self, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = ctypes.c_void_p()
        st = lib.m4rie_create(ctypes.byref(handle), ctypes.c_void_p(stream.cuda_stream))
        if st != OK:
            raise M4rieError(st, "m4rie_create")
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None):
            lib.m4rie_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, st, where):
        if st != OK:
            raise M4rieError(st, where, lib.m4rie_last_error(self.handle).decode())

    def set_form(self, form):
        self._raise(lib.m4rie_set_form(self.handle, FORMS.get(form, form)), "m4rie_set_form")

    def set_schedule(self, schedule):
        self._raise(lib.m4rie_set_schedule(self.handle, SCHEDULES.get(schedule, schedule)), "m4rie_set_schedule")

    def set_test_hook(self, flags: int):
        self._raise(lib.m4rie_set_test_hook(self.handle, int(flags)), "m4rie_set_test_hook")

    def set_wait_limit_ns(self, ns: int):
        self._raise(lib.m4rie_set_wait_limit_ns(self.handle, int(ns)), "m4rie_set_wait_limit_ns")

    def mul(self, e: int, f: int, A, B, C=None):
        """C = A B over GF(2^e); allocates C when not given.  Asynchronous."""
        import torch
        _check_dev(A, e, "A")
        _check_dev(B, e, "B")
        m, k = A.shape
        k2, n = B.shape
        if k2 != k:
            raise ValueError("inner dimensions differ")
        if C is None:
            C = torch.empty((m, n), dtype=A.dtype, device=A.device)
        _check_dev(C, e, "C")
        if tuple(C.shape) != (m, n):
            raise ValueError(f"C must be {m} x {n}, not {tuple(C.shape)}")
        self._raise(lib.m4rie_mul(self.handle, e, f, m, n, k, _ptr(A), _ptr(B), _ptr(C)), "m4rie_mul")
        return C

    def addmul(self, e: int, f: int, A, B, C):
        """C += A B over GF(2^e), in place.  Asynchronous."""
        for t, nm in ((A, "A"), (B, "B"), (C, "C")):
            _check_dev(t, e, nm)
        m, k = A.shape
        k2, n = B.shape
        if k2 != k or tuple(C.shape) != (m, n):
            raise ValueError("shapes do not match: A m x k, B k x n, C m x n")
        self._raise(lib.m4rie_addmul(self.handle, e, f, m, n, k, _ptr(A), _ptr(B), _ptr(C)), "m4rie_addmul")
        return C

    def gemm(self, e: int, f: int, A, B, C, accumulate: bool = False):
        """C = A B (or C += A B) on 2-D windows of larger tensors (row strides
        from the tensors, unit column stride).  Asynchronous."""
        for t, nm in ((A, "A"), (B, "B"), (C, "C")):
            _check_dev(t, e, nm, strided=True)
        m, k = A.shape
        k2, n = B.shape
        if k2 != k or tuple(C.shape) != (m, n):
            raise ValueError("shapes do not match")
        self._raise(lib.m4rie_gemm(self.handle, e, f, m, n, k, _ptr(A), _ld(A), _ptr(B), _ld(B), _ptr(C), _ld(C),
                                   1 if accumulate else 0), "m4rie_gemm")
        return C

    def trsm(self, e: int, f: int, T, B, upper: bool = True):
        """B <- T^{-1} B in place (Algorithm 5), T square triangular (the
        other triangle is not read); windows with unit column stride.
        Asynchronous; a zero diagonal shows as ERR_SINGULAR in device_status()."""
        _check_dev(T, e, "T", strided=True)
        _check_dev(B, e, "B", strided=True)
        m = T.shape[0]
        if T.shape[1] != m or B.shape[0] != m:
            raise ValueError("T must be m x m and B m x n")
        n = B.shape[1]
        fn = lib.m4rie_trsm_upper_left if upper else lib.m4rie_trsm_lower_left
        self._raise(fn(self.handle, e, f, m, n, _ptr(T), _ld(T), _ptr(B), _ld(B)),
                    "m4rie_trsm_upper_left" if upper else "m4rie_trsm_lower_left")
        return B

    def echelonize(self, e: int, f: int, A):
        """Reduced row echelon form of A in place (Algorithm 4); returns
        (rank, list of pivot columns).  Synchronous."""
        import numpy as np
        _check_dev(A, e, "A", strided=True)
        m, n = A.shape
        rank = ctypes.c_int64()
        piv = np.zeros(max(1, min(m, n)), dtype=np.int64)
        self._raise(lib.m4rie_echelonize(self.handle, e, f, m, n, _ptr(A), _ld(A) if m else n, ctypes.byref(rank),
                                         ctypes.c_void_p(piv.ctypes.data)), "m4rie_echelonize")
        return int(rank.value), [int(v) for v in piv[:rank.value]]

    def ple(self, e: int, f: int, A):
        """PLE decomposition of A in place (Section 4.2); returns (rank, P,
        Q) with P (m swap partners) and Q (n entries, pivot columns first) as
        int64 numpy arrays.  Layout of A afterwards: see m4rie_ple in the C
        header.  Synchronous."""
        import numpy as np
        _check_dev(A, e, "A", strided=True)
        m, n = A.shape
        rank = ctypes.c_int64()
        P = np.zeros(max(1, m), dtype=np.int64)
        Q = np.zeros(max(1, n), dtype=np.int64)
        self._raise(lib.m4rie_ple(self.handle, e, f, m, n, _ptr(A), _ld(A) if m else n, ctypes.byref(rank),
                                  ctypes.c_void_p(P.ctypes.data), ctypes.c_void_p(Q.ctypes.data)), "m4rie_ple")
        return int(rank.value), P[:m].copy(), Q[:n].copy()

    def mul_host(self, e: int, f: int, A, B, C, accumulate: bool = False):
        """Host-buffer product (torch CPU tensors or numpy arrays, row-major,
        one element of 1 byte for e <= 8 and 2 bytes for e > 8); synchronous.
        C is written in place."""
        if len(getattr(A, "shape", ())) != 2 or len(getattr(B, "shape", ())) != 2:
            raise ValueError("A and B must be 2-D")
        m, k = A.shape
        n = B.shape[1]
        pa = _host_matrix(A, e, "A", (m, k))
        pb = _host_matrix(B, e, "B", (k, n))
        pc = _host_matrix(C, e, "C", (m, n), writable=True)
        self._raise(lib.m4rie_mul_host(self.handle, e, f, m, n, k, pa, pb, pc, 1 if accumulate else 0),
                    "m4rie_mul_host")
        return C

    def pack(self, e: int, elems, ld_words: int | None = None):
        """Slicing (Section 3.2): returns int64 tensor (e, rows, ld_words) of 64-bit words."""
        import torch
        _check_dev(elems, e, "elems")
        rows, cols = elems.shape
        if ld_words is None:
            ld_words = (cols + 63) // 64
        S = torch.empty((e, rows, ld_words), dtype=torch.int64, device=elems.device)
        self._raise(lib.m4rie_pack(self.handle, e, rows, cols, _ptr(elems), _ptr(S), ld_words), "m4rie_pack")
        return S

    def unpack(self, e: int, slices, cols: int):
        """Clinging: (e, rows, ld_words) words -> rows x cols elements."""
        import torch
        _check_words(slices, "slices", 3)
        if slices.shape[0] != e:
            raise ValueError(f"slices must hold e = {e} slices, not {slices.shape[0]}")
        _, rows, ld_words = slices.shape
        X = torch.empty((rows, cols), dtype=elem_dtype_torch(e), device=slices.device)
        self._raise(lib.m4rie_unpack(self.handle, e, rows, cols, _ptr(slices), ld_words, _ptr(X)), "m4rie_unpack")
        return X

    def to_packed(self, e: int, elems, ld_words: int | None = None):
        """Packed representation (Section 3.1) of a 2-D window of elements:
        int64 tensor (rows, ld_words) holding the 64-bit words."""
        import torch
        _check_dev(elems, e, "elems", strided=True)
        rows, cols = elems.shape
        per = _fields_per_word(e)
        if ld_words is None:
            ld_words = (cols + per - 1) // per
        W = torch.empty((rows, ld_words), dtype=torch.int64, device=elems.device)
        self._raise(lib.m4rie_to_packed(self.handle, e, rows, cols, _ptr(elems), _ld(elems) if rows else cols,
                                        _ptr(W), ld_words), "m4rie_to_packed")
        return W

    def from_packed(self, e: int, words, cols: int, out=None):
        """Elements of a packed matrix (int64 words, rows x ld_words)."""
        import torch
        _check_words(words, "words", 2)
        rows, ld_words = words.shape
        X = out if out is not None else torch.empty((rows, cols), dtype=elem_dtype_torch(e), device=words.device)
        _check_dev(X, e, "out", strided=True)
        if tuple(X.shape) != (rows, cols):
            raise ValueError(f"out must be {rows} x {cols}, not {tuple(X.shape)}")
        self._raise(lib.m4rie_from_packed(self.handle, e, rows, cols, _ptr(words), ld_words, _ptr(X),
                                          _ld(X) if rows else cols), "m4rie_from_packed")
        return X

    def mul_packed(self, e: int, f: int, A, B, C, n: int, k: int, accumulate: bool = False):
        """Newton-John product of packed matrices (int64 word tensors, row
        strides from the tensors): C = A B or C += A B, A m x k, B k x n."""
        for t, nm in ((A, "A"), (B, "B"), (C, "C")):
            _check_word_window(t, nm)
        m = A.shape[0]
        per = _fields_per_word(e)
        kw, nw = -(-k // per), -(-n // per)
        if B.shape[0] != k or C.shape[0] != m:
            raise ValueError("shapes do not match")
        if A.shape[1] < kw or B.shape[1] < nw or C.shape[1] < nw:
            raise ValueError(f"rows of A need {kw} words, rows of B and C {nw}")
        self._raise(lib.m4rie_mul_packed(self.handle, e, f, m, n, k, _ptr(A), _ld(A), _ptr(B), _ld(B), _ptr(C),
                                         _ld(C), 1 if accumulate else 0), "m4rie_mul_packed")
        return C

    def mul_batched(self, problems):
        """problems: list of (e, f, A, B, C, accumulate) with CUDA tensors, or
        the array problem_array() made of one."""
        arr = problems if isinstance(problems, ctypes.Array) else problem_array(problems)
        self._raise(lib.m4rie_mul_batched(self.handle, len(problems), arr), "m4rie_mul_batched")

    def tune_batched(self, problems):
        """m4rie_tune_batched: measure the schedule per (e, shape class) of this
        batch for later mul_batched calls; the batch's tensors are not touched."""
        arr = problems if isinstance(problems, ctypes.Array) else problem_array(problems)
        self._raise(lib.m4rie_tune_batched(self.handle, len(problems), arr), "m4rie_tune_batched")

    def enable_timing(self, on: bool = True):
        self._raise(lib.m4rie_enable_timing(self.handle, 1 if on else 0), "m4rie_enable_timing")

    def phase_times(self, reset: bool = True):
        """(pack_ms, gemm_ms, recombine_ms, products) accumulated since the last reset."""
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int64()
        self._raise(lib.m4rie_phase_times(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                          ctypes.byref(n), 1 if reset else 0), "m4rie_phase_times")
        return a.value, b.value, c.value, n.value

    def tune(self, e: int, f: int, m: int, n: int, k: int):
        """Autotune the shape class of (e, m, n, k); returns (form, schedule, ms)."""
        self._raise(lib.m4rie_tune(self.handle, e, f, m, n, k), "m4rie_tune")
        return self.tuned_choice(e, m, n, k)

    def tuned_choice(self, e: int, m: int, n: int, k: int):
        fo, sc, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._raise(lib.m4rie_tuned_choice(self.handle, e, m, n, k, ctypes.byref(fo), ctypes.byref(sc),
                                           ctypes.byref(ms)), "m4rie_tuned_choice")
        if fo.value == 0:
            return None, None, 0.0          # shape class not tuned
        inv_f = {v: k for k, v in FORMS.items()}
        inv_s = {v: k for k, v in SCHEDULES.items()}
        return inv_f.get(fo.value, fo.value), inv_s.get(sc.value, sc.value), ms.value

    def tune_save(self, path: str):
        self._raise(lib.m4rie_tune_save(self.handle, path.encode()), "m4rie_tune_save")

    def tune_load(self, path: str):
        self._raise(lib.m4rie_tune_load(self.handle, path.encode()), "m4rie_tune_load")

    def device_status(self) -> int:
        return lib.m4rie_get_device_status(self.handle)

    def kernel_launches(self) -> int:
        return int(lib.m4rie_kernel_launches(self.handle))

    def resolve_form(self, e, m, n, k) -> int:
        return int(lib.m4rie_resolve_form(self.handle, e, m, n, k))


def mul_noalloc(e: int, f: int, A, B, C, accumulate: bool = False, device_status=None, stream=None) -> int:
    """m4rie_mul_noalloc on CUDA tensors; returns the m4rie_status code.

    A (m x k), B (k x n) and C (m x n) are contiguous CUDA tensors of the
    field's element type (uint8 for e <= 8, uint16 for e = 9, 10), checked here
    because the entry point takes bare pointers and row strides equal to the
    widths.  device_status: None or a CUDA int32 tensor of at least one element
    (its first element receives the device-detected status bits)."""
    import torch
    for t, nm in ((A, "A"), (B, "B"), (C, "C")):
        _check_dev(t, e, nm)
    if A.dim() != 2 or B.dim() != 2 or C.dim() != 2:
        raise ValueError("A, B and C must be 2-D")
    m, k = A.shape
    k2, n = B.shape
    if k2 != k or tuple(C.shape) != (m, n):
        raise ValueError("shapes do not match: A m x k, B k x n, C m x n")
    if device_status is not None:
        if (not isinstance(device_status, torch.Tensor) or not device_status.is_cuda
                or device_status.dtype != torch.int32):
            raise TypeError("device_status must be a CUDA int32 tensor")
        if device_status.numel() < 1:
            raise ValueError("device_status must have at least one element")
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(lib.m4rie_mul_noalloc(e, f, m, n, k, _ptr(A), _ptr(B), _ptr(C), 1 if accumulate else 0,
                                     _ptr(device_status), ctypes.c_void_p(stream.cuda_stream)))


def packed_width(e: int) -> int:
    """Bits per element in the packed representation (Section 3.1)."""
    return int(lib.m4rie_packed_width(e))


def schedule_products(e: int, f: int, schedule) -> int:
    return int(lib.m4rie_schedule_products(e, f, SCHEDULES.get(schedule, schedule)))


def schedule_masks(e: int, f: int, schedule):
    """(amask list, bmask list, out_mask list of 10) of a schedule."""
    cap = 128
    am = (ctypes.c_uint16 * cap)()
    bm = (ctypes.c_uint16 * cap)()
    om = (ctypes.c_uint64 * 10)()
    r = lib.m4rie_schedule_masks(e, f, SCHEDULES.get(schedule, schedule), cap, am, bm, om)
    if r < 0:
        raise M4rieError(-r, "m4rie_schedule_masks")
    return list(am[:r]), list(bm[:r]), list(om)


def validate(e, f, m, n, k, A=None, B=None, C=None) -> int:
    """Host-side argument check; A, B, C are integer addresses (or None)."""
    v = lambda x: None if x is None else ctypes.c_void_p(x)
    return int(lib.m4rie_validate(e, f, m, n, k, v(A), v(B), v(C)))
