"""Python binding of librlu.so, the GB300 sparse randomized LU library.

Argument marshalling only: every step of the factorization runs in the
library's CUDA kernels.  torch supplies device memory and streams.  The
functions mirror the C ABI in include/rlu.h (same names, same order of
arguments); `RandLU` is a small convenience wrapper over them.

If librlu.so has not been built (see `build`), importing works but every
call raises RuntimeError: there is no CPU fallback.
"""
import ctypes
import os
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librlu.so")

RLU_OK, RLU_EINVAL, RLU_ENOMEM, RLU_ECUDA, RLU_ETIMEOUT, RLU_ENONFINITE, RLU_EBADCSR = 0, 1, 2, 3, 4, 5, 6
RLU_ETOOLARGE = 7
RLU_NOALLOC_MAX_N, RLU_NOALLOC_MAX_L1, RLU_NOALLOC_MAX_L = 65536, 4096, 1024
RLU_WRANK = 100
RLU_F64, RLU_F32, RLU_BF16 = 0, 1, 2
RLU_PREC_F64, RLU_PREC_F32, RLU_PREC_BF16, RLU_PREC_BF16_REFINE = 0, 1, 2, 3
PREC = {"f64": RLU_PREC_F64, "f32": RLU_PREC_F32, "bf16": RLU_PREC_BF16, "bf16_refine": RLU_PREC_BF16_REFINE}
RLU_XFORM_HARTLEY, RLU_XFORM_SRHT, RLU_XFORM_SRFT = 0, 1, 2
TRANSFORM = {"hartley": RLU_XFORM_HARTLEY, "srht": RLU_XFORM_SRHT, "srft": RLU_XFORM_SRFT}

#: every entry point declared in include/rlu.h
C_SYMBOLS = ("rlu_create", "rlu_create_in", "rlu_set_precision", "rlu_workspace_bytes", "rlu_factor_dense",
             "rlu_factor_dense_async", "rlu_factor_csr", "rlu_factor_dense_host", "rlu_destroy",
             "rlu_strerror", "rlu_debug_sketch_params", "rlu_debug_Y", "rlu_debug_B", "rlu_debug_enable",
             "rlu_debug_timing", "rlu_debug_stage_ms", "rlu_debug_launch_count", "rlu_sketch_dense_noalloc",
             "rlu_csr_workspace_bytes", "rlu_set_csr_workspace", "rlu_graph_capture_dense", "rlu_graph_launch",
             "rlu_graph_destroy", "rlu_copy_block_async", "rlu_set_max_ctas",
             "rlu_debug_recip", "rlu_set_second_sketch", "rlu_debug_status_of_flags", "rlu_debug_wait_timeout",
             "rlu_debug_alu_peak", "rlu_set_transform", "rlu_set_column_pivoting", "rlu_debug_set_lu_block",
             "rlu_debug_lu_block", "rlu_debug_lu_Y", "rlu_debug_lu_panels", "rlu_debug_set_tma_a")

#: stage names reported by rlu_debug_stage_ms, in order
STAGES = ("params", "sketch", "panel_lu", "gram", "chol", "wform", "bgemm", "lu_b", "assemble")

_lib = None


def build(force=False):
    """Compile librlu.so for sm_103a (in-tree) and load it."""
    from . import _build
    _build.build(force=force)
    return load(reload=True)


def load(reload=False):
    global _lib
    if _lib is not None and not reload:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("librlu.so is not built; run paper_1601_04280_gb300.build() (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    c = ctypes
    vp, i64, i32, u64 = c.c_void_p, c.c_int64, c.c_int32, c.c_uint64
    sig = {
        "rlu_create": ([i64, i64, i32, i32, i32, u64, c.POINTER(vp)], c.c_int),
        "rlu_create_in": ([i64, i64, i32, i32, i32, u64, vp, c.c_size_t, vp, c.POINTER(vp)], c.c_int),
        "rlu_set_precision": ([vp, c.c_int], c.c_int),
        "rlu_workspace_bytes": ([i64, i64, i32, i32, i32, c.c_int, c.POINTER(c.c_size_t)], c.c_int),
        "rlu_factor_dense": ([vp, vp, i64, c.c_int, vp, vp, vp, vp, vp], c.c_int),
        "rlu_factor_dense_async": ([vp, vp, i64, c.c_int, vp, vp, vp, vp, vp, vp], c.c_int),
        "rlu_factor_csr": ([vp, vp, vp, vp, i64, c.c_int, vp, vp, vp, vp, vp], c.c_int),
        "rlu_factor_dense_host": ([vp, vp, c.c_int, vp, vp, vp, vp, vp], c.c_int),
        "rlu_destroy": ([vp], c.c_int),
        "rlu_strerror": ([c.c_int], c.c_char_p),
        "rlu_debug_sketch_params": ([vp, vp, vp, vp, vp], c.c_int),
        "rlu_debug_Y": ([vp, vp], c.c_int),
        "rlu_debug_B": ([vp, vp], c.c_int),
        "rlu_debug_enable": ([vp, c.c_int], c.c_int),
        "rlu_debug_timing": ([vp, c.c_int], c.c_int),
        "rlu_debug_stage_ms": ([vp, vp, c.c_int, c.POINTER(c.c_int)], c.c_int),
        "rlu_debug_launch_count": ([c.POINTER(i64)], c.c_int),
        "rlu_sketch_dense_noalloc": ([vp, i64, c.c_int, i64, i64, i32, i32, u64, vp, vp, vp], c.c_int),
        "rlu_csr_workspace_bytes": ([i64, i64, i32, i64, c.POINTER(c.c_size_t)], c.c_int),
        "rlu_set_csr_workspace": ([vp, i64, vp, c.c_size_t], c.c_int),
        "rlu_graph_capture_dense": ([vp, vp, i64, c.c_int, vp, vp, vp, vp, vp, vp, c.POINTER(vp)], c.c_int),
        "rlu_graph_launch": ([vp, vp], c.c_int),
        "rlu_graph_destroy": ([vp], c.c_int),
        "rlu_copy_block_async": ([vp, i64, vp, i64, i64, i64, vp], c.c_int),
        "rlu_set_max_ctas": ([vp, i32], c.c_int),
        "rlu_debug_recip": ([vp, vp, i64], c.c_int),
        "rlu_set_second_sketch": ([vp, i32, i32, u64], c.c_int),
        "rlu_debug_status_of_flags": ([c.c_uint32, c.POINTER(c.c_int)], c.c_int),
        "rlu_debug_wait_timeout": ([c.c_int, c.POINTER(c.c_int)], c.c_int),
        "rlu_debug_alu_peak": ([c.c_int, c.POINTER(c.c_double)], c.c_int),
        "rlu_set_transform": ([vp, c.c_int], c.c_int),
        "rlu_set_column_pivoting": ([vp, c.c_int], c.c_int),
        "rlu_debug_set_lu_block": ([vp, c.c_int32], c.c_int),
        "rlu_debug_lu_block": ([vp, c.POINTER(c.c_int32)], c.c_int),
        "rlu_debug_lu_Y": ([vp, vp, vp], c.c_int),
        "rlu_debug_set_tma_a": ([vp, c.c_int], c.c_int),
        "rlu_debug_lu_panels": ([vp, c.c_int, c.POINTER(c.c_int32), c.POINTER(c.c_int32), c.POINTER(c.c_double)],
                                c.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


class RluError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (status %d)" % (where, strerror(code), code))


def strerror(code):
    return load().rlu_strerror(int(code)).decode()


def _check(code, where, allow_warn=True):
    if code == RLU_OK or (allow_warn and code == RLU_WRANK):
        return code
    raise RluError(code, where)


# ---- C-ABI mirrors -----------------------------------------------------------
def rlu_create(m, n, k, l, l1, seed):
    h = ctypes.c_void_p()
    _check(load().rlu_create(m, n, k, l, l1, ctypes.c_uint64(seed & (2**64 - 1)), ctypes.byref(h)), "rlu_create")
    return h


def rlu_create_in(m, n, k, l, l1, seed, workspace_ptr, workspace_bytes, stream_ptr):
    h = ctypes.c_void_p()
    _check(load().rlu_create_in(m, n, k, l, l1, ctypes.c_uint64(seed & (2**64 - 1)), workspace_ptr,
                                workspace_bytes, stream_ptr, ctypes.byref(h)), "rlu_create_in")
    return h


def rlu_set_precision(h, prec):
    return _check(load().rlu_set_precision(h, PREC.get(prec, prec)), "rlu_set_precision")


def rlu_set_transform(h, transform):
    return _check(load().rlu_set_transform(h, TRANSFORM.get(transform, transform)), "rlu_set_transform")


def rlu_set_column_pivoting(h, on):
    return _check(load().rlu_set_column_pivoting(h, 1 if on else 0), "rlu_set_column_pivoting")


def rlu_debug_set_lu_block(h, block):
    return _check(load().rlu_debug_set_lu_block(h, int(block)), "rlu_debug_set_lu_block")


def rlu_debug_set_tma_a(h, on):
    return _check(load().rlu_debug_set_tma_a(h, int(on)), "rlu_debug_set_tma_a")


def rlu_debug_lu_block(h):
    """(block setting, widest panel the handle holds)."""
    bmax = ctypes.c_int32(0)
    rc = load().rlu_debug_lu_block(h, ctypes.byref(bmax))
    if rc not in (-1, 0, 16, 32, 64):
        _check(rc, "rlu_debug_lu_block")
    return rc, int(bmax.value)


def rlu_set_second_sketch(h, k2, l2, seed2):
    return _check(load().rlu_set_second_sketch(h, int(k2), int(l2), ctypes.c_uint64(seed2 & (2**64 - 1))),
                  "rlu_set_second_sketch")


def rlu_set_max_ctas(h, max_ctas):
    return _check(load().rlu_set_max_ctas(h, int(max_ctas)), "rlu_set_max_ctas")


def rlu_workspace_bytes(m, n, k, l, l1, prec):
    out = ctypes.c_size_t()
    _check(load().rlu_workspace_bytes(m, n, k, l, l1, PREC.get(prec, prec), ctypes.byref(out)), "rlu_workspace_bytes")
    return out.value


def rlu_csr_workspace_bytes(m, n, k, max_nnz):
    out = ctypes.c_size_t()
    _check(load().rlu_csr_workspace_bytes(m, n, k, max_nnz, ctypes.byref(out)), "rlu_csr_workspace_bytes")
    return out.value


def rlu_set_csr_workspace(h, max_nnz, workspace_ptr, workspace_bytes):
    return _check(load().rlu_set_csr_workspace(h, max_nnz, workspace_ptr, workspace_bytes), "rlu_set_csr_workspace")


def rlu_factor_dense(h, A_ptr, lda, dtype, L_ptr, U_ptr, p_ptr, q_ptr, stream_ptr):
    return load().rlu_factor_dense(h, A_ptr, lda, dtype, L_ptr, U_ptr, p_ptr, q_ptr, stream_ptr)


def rlu_factor_dense_async(h, A_ptr, lda, dtype, L_ptr, U_ptr, p_ptr, q_ptr, status_ptr, stream_ptr):
    return load().rlu_factor_dense_async(h, A_ptr, lda, dtype, L_ptr, U_ptr, p_ptr, q_ptr, status_ptr, stream_ptr)


def rlu_graph_capture_dense(h, A_ptr, lda, dtype, L_ptr, U_ptr, p_ptr, q_ptr, status_ptr, stream_ptr):
    g = ctypes.c_void_p()
    _check(load().rlu_graph_capture_dense(h, A_ptr, lda, dtype, L_ptr, U_ptr, p_ptr, q_ptr, status_ptr, stream_ptr,
                                          ctypes.byref(g)), "rlu_graph_capture_dense", allow_warn=False)
    return g


def rlu_copy_block_async(dst_ptr, dst_pitch, src_ptr, src_pitch, width_bytes, rows, stream_ptr):
    return _check(load().rlu_copy_block_async(dst_ptr, dst_pitch, src_ptr, src_pitch, width_bytes, rows, stream_ptr),
                  "rlu_copy_block_async", allow_warn=False)


def rlu_graph_launch(g, stream_ptr):
    return _check(load().rlu_graph_launch(g, stream_ptr), "rlu_graph_launch", allow_warn=False)


def rlu_graph_destroy(g):
    return load().rlu_graph_destroy(g)


def rlu_factor_csr(h, rowptr_ptr, colind_ptr, val_ptr, nnz, dtype, L_ptr, U_ptr, p_ptr, q_ptr, stream_ptr):
    return load().rlu_factor_csr(h, rowptr_ptr, colind_ptr, val_ptr, nnz, dtype, L_ptr, U_ptr, p_ptr, q_ptr,
                                 stream_ptr)


def rlu_factor_dense_host(h, A_ptr, dtype, L_ptr, U_ptr, p_ptr, q_ptr, stream_ptr):
    return load().rlu_factor_dense_host(h, A_ptr, dtype, L_ptr, U_ptr, p_ptr, q_ptr, stream_ptr)


def rlu_destroy(h):
    return load().rlu_destroy(h)


def rlu_sketch_dense_noalloc(A_ptr, lda, dtype, m, n, l, l1, seed, Y_ptr, status_ptr, stream_ptr):
    """Sketch Y = A S D H R / sqrt(l1) without any allocation (see include/rlu.h)."""
    return load().rlu_sketch_dense_noalloc(A_ptr, lda, dtype, m, n, l, l1, ctypes.c_uint64(seed & (2**64 - 1)),
                                           Y_ptr, status_ptr, stream_ptr)


def rlu_debug_recip(x):
    """The device FP64 reciprocal of the Cholesky step on host values (test hook)."""
    import numpy as np
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    _check(load().rlu_debug_recip(x.ctypes.data, out.ctypes.data, x.size), "rlu_debug_recip")
    return out


def rlu_debug_status_of_flags(flags):
    """Status code the library reports for device flag bits (no GPU needed)."""
    out = ctypes.c_int()
    _check(load().rlu_debug_status_of_flags(int(flags), ctypes.byref(out)), "rlu_debug_status_of_flags")
    return out.value


def rlu_debug_wait_timeout(which):
    """Run a bounded device wait that can never complete; returns its status."""
    out = ctypes.c_int()
    _check(load().rlu_debug_wait_timeout(int(which), ctypes.byref(out)), "rlu_debug_wait_timeout")
    return out.value


def rlu_debug_alu_peak(which):
    """FP64 (which=0) or FP32 (which=1) FMA throughput of the current GPU, TFLOP/s."""
    out = ctypes.c_double()
    _check(load().rlu_debug_alu_peak(int(which), ctypes.byref(out)), "rlu_debug_alu_peak")
    return out.value


def rlu_debug_launch_count():
    out = ctypes.c_int64()
    _check(load().rlu_debug_launch_count(ctypes.byref(out)), "rlu_debug_launch_count")
    return out.value


# ---- convenience wrapper (torch tensors) ---------------------------------------
@dataclass
class Factors:
    L: object
    U: object
    p: object
    q: object
    status: int


def _dtype_code(t):
    import torch
    return {torch.float64: RLU_F64, torch.float32: RLU_F32, torch.bfloat16: RLU_BF16}[t.dtype]


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class RandLU:
    """One handle: fixed sizes, seed and precision; reusable across calls."""

    def __init__(self, m, n, k, l, l1, seed, prec="f32", workspace=None, stream=None):
        """workspace: optional device tensor (uint8, >= rlu_workspace_bytes) the handle
        uses instead of allocating; the caller keeps it alive until close()."""
        self.m, self.n, self.k, self.l, self.l1, self.seed = m, n, k, l, l1, seed
        if workspace is None:
            self.h = rlu_create(m, n, k, l, l1, seed)
        else:
            self.h = rlu_create_in(m, n, k, l, l1, seed, ctypes.c_void_p(workspace.data_ptr()),
                                   workspace.numel() * workspace.element_size(), _stream_ptr(stream))
        self.prec = prec
        rlu_set_precision(self.h, prec)

    def set_second_sketch(self, k2, l2, seed2):
        """B by the paper's second projection (k2 x m, l2 buckets); k2 = 0: exact pseudo-inverse."""
        rlu_set_second_sketch(self.h, k2, l2, seed2)

    def set_transform(self, transform):
        """The projection of step 2: "hartley" (default), "srht" or "srft"."""
        rlu_set_transform(self.h, transform)

    def set_column_pivoting(self, on=True):
        """Order the sketch's columns by QR with column pivoting before the panel LU."""
        rlu_set_column_pivoting(self.h, on)

    def set_lu_block(self, block):
        """Panel width of the LU of the sketch: 0 automatic, -1 unblocked, 16/32/64."""
        rlu_debug_set_lu_block(self.h, block)

    def set_tma_a(self, on):
        """BF16 A of B = W A fed by TMA where aligned (True, the default) or by the converter warps."""
        rlu_debug_set_tma_a(self.h, 1 if on else 0)

    def set_max_ctas(self, max_ctas):
        """Bound the CTAs of the grid-synchronised kernels (0: one per SM)."""
        rlu_set_max_ctas(self.h, max_ctas)

    def set_csr_workspace(self, workspace, max_nnz):
        """Caller-owned CSR scratch (device uint8 tensor, >= rlu_csr_workspace_bytes)."""
        rlu_set_csr_workspace(self.h, max_nnz, ctypes.c_void_p(workspace.data_ptr()),
                              workspace.numel() * workspace.element_size())

    @property
    def out_dtype(self):
        import torch
        return torch.float64 if self.prec == "f64" else torch.float32

    def alloc_outputs(self, device="cuda"):
        import torch
        L = torch.empty((self.m, self.k), dtype=self.out_dtype, device=device)
        U = torch.empty((self.k, self.n), dtype=self.out_dtype, device=device)
        p = torch.empty(self.m, dtype=torch.int64, device=device)
        q = torch.empty(self.n, dtype=torch.int64, device=device)
        return L, U, p, q

    def factor(self, A, out=None, stream=None, check=True):
        assert A.is_cuda and A.dim() == 2 and A.shape == (self.m, self.n) and A.stride(1) == 1
        L, U, p, q = out if out is not None else self.alloc_outputs(A.device)
        code = rlu_factor_dense(self.h, ctypes.c_void_p(A.data_ptr()), A.stride(0), _dtype_code(A),
                                ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(U.data_ptr()),
                                ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(q.data_ptr()), _stream_ptr(stream))
        if check:
            _check(code, "rlu_factor_dense")
        return Factors(L, U, p, q, code)

    def factor_async(self, A, out, status, stream=None):
        L, U, p, q = out
        code = rlu_factor_dense_async(self.h, ctypes.c_void_p(A.data_ptr()), A.stride(0), _dtype_code(A),
                                      ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(U.data_ptr()),
                                      ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                      ctypes.c_void_p(status.data_ptr()), _stream_ptr(stream))
        return _check(code, "rlu_factor_dense_async", allow_warn=False)

    def factor_csr(self, rowptr, colind, val, out=None, stream=None, check=True):
        L, U, p, q = out if out is not None else self.alloc_outputs(val.device)
        code = rlu_factor_csr(self.h, ctypes.c_void_p(rowptr.data_ptr()), ctypes.c_void_p(colind.data_ptr()),
                              ctypes.c_void_p(val.data_ptr()), val.numel(), _dtype_code(val),
                              ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(U.data_ptr()),
                              ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(q.data_ptr()), _stream_ptr(stream))
        if check:
            _check(code, "rlu_factor_csr")
        return Factors(L, U, p, q, code)

    def factor_host(self, A_host, out_host, stream=None, check=True):
        """A_host, outputs: CPU tensors (pinned for full copy speed)."""
        L, U, p, q = out_host
        code = rlu_factor_dense_host(self.h, ctypes.c_void_p(A_host.data_ptr()), _dtype_code(A_host),
                                     ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(U.data_ptr()),
                                     ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                     _stream_ptr(stream))
        if check:
            _check(code, "rlu_factor_dense_host")
        return Factors(L, U, p, q, code)

    def debug_enable(self, on=True):
        _check(load().rlu_debug_enable(self.h, 1 if on else 0), "rlu_debug_enable")

    def debug_timing(self, on=True):
        _check(load().rlu_debug_timing(self.h, 1 if on else 0), "rlu_debug_timing")

    def debug_stage_ms(self):
        import numpy as np
        ms = np.zeros(len(STAGES), np.float32)
        cnt = ctypes.c_int()
        _check(load().rlu_debug_stage_ms(self.h, ms.ctypes.data, len(STAGES), ctypes.byref(cnt)),
               "rlu_debug_stage_ms")
        return dict(zip(STAGES, ms[: cnt.value].tolist()))

    def debug_sketch_params(self):
        import numpy as np
        h = np.empty(self.n, np.int32)
        s = np.empty(self.n, np.int8)
        d = np.empty(self.l1, np.int8)
        R = np.empty(self.l, np.int32)
        _check(load().rlu_debug_sketch_params(self.h, h.ctypes.data, s.ctypes.data, d.ctypes.data, R.ctypes.data),
               "rlu_debug_sketch_params")
        return h, s, d, R

    def debug_Y(self):
        import numpy as np
        Y = np.empty((self.m, self.l), np.float64)
        _check(load().rlu_debug_Y(self.h, Y.ctypes.data), "rlu_debug_Y")
        return Y

    def debug_lu_Y(self):
        """Y after step 3 (rows in original order) and the row permutation."""
        import numpy as np
        Y = np.empty((self.m, self.l), np.float64)
        perm = np.empty(self.m, np.int64)
        _check(load().rlu_debug_lu_Y(self.h, Y.ctypes.data, perm.ctypes.data), "rlu_debug_lu_Y")
        return Y, perm

    def debug_lu_panels(self, which=0):
        """(panel width or 0, launches, summed ms) of the pivoted-LU kernel in the
        last timed factorization: which = 0 the LU of Y, 1 the LU of B^T."""
        w, n, ms = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0.0)
        _check(load().rlu_debug_lu_panels(self.h, int(which), ctypes.byref(w), ctypes.byref(n), ctypes.byref(ms)),
               "rlu_debug_lu_panels")
        return int(w.value), int(n.value), float(ms.value)

    def debug_B(self):
        import numpy as np
        B = np.empty((self.k, self.n), np.float64)
        _check(load().rlu_debug_B(self.h, B.ctypes.data), "rlu_debug_B")
        return B

    def close(self):
        if getattr(self, "h", None):
            rlu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
