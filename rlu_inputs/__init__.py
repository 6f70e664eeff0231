"""Seeded synthetic inputs for the sparse randomized LU path.

This module only makes test and benchmark matrices; it holds none of the
method's arithmetic and is shared by the oracle side and the CUDA side.  The
shapes and spectra follow the workloads of the paper's experiments (Sec. 4:
square dense matrices with prescribed singular values, built from orthonormal
factors) scaled to the sizes used here, plus a sparse CSR family.

Every generator is a pure function of its arguments (numpy PCG64 streams).
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse


@dataclass(frozen=True)
class Workload:
    name: str
    m: int
    n: int
    k: int
    l: int
    l1: int
    dtype: str       # storage dtype of A: "f64", "f32", "bf16"
    sparse: bool
    data_seed: int
    sketch_seed: int


#: the four single-factorization workloads (dense FP64, dense FP32, CSR FP32,
#: dense BF16 precision form)
DENSE_F64_1K = Workload("dense_f64_1024x1024_k20", 1024, 1024, 20, 30, 240, "f64", False, 1000, 2000)
DENSE_F32_8K = Workload("dense_f32_8192x8192_k200", 8192, 8192, 200, 220, 1600, "f32", False, 1001, 2001)
CSR_F32_200K = Workload("csr_f32_200000x50000_k100", 200000, 50000, 100, 120, 960, "f32", True, 1002, 2002)
DENSE_BF16_32K = Workload("dense_bf16_32768x16384_k500", 32768, 16384, 500, 520, 4000, "bf16", False, 1003, 2003)

WORKLOADS = {w.name: w for w in (DENSE_F64_1K, DENSE_F32_8K, CSR_F32_200K, DENSE_BF16_32K)}


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def orthonormal(rows, cols, rng):
    """Orthonormal columns from the QR of a Gaussian matrix, R with a positive
    diagonal (so the factor is uniquely defined by the Gaussian draw)."""
    G = rng.standard_normal((rows, cols))
    Q, R = np.linalg.qr(G, mode="reduced")
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    return Q * sgn[None, :]


def geometric_spectrum(count, decade_per=10.0):
    """sigma_i = 10^(-(i-1)/decade_per), i = 1..count."""
    return 10.0 ** (-np.arange(count, dtype=np.float64) / decade_per)


def inverse_square_spectrum(count):
    """sigma_i = 1 / i^2, i = 1..count."""
    i = np.arange(1, count + 1, dtype=np.float64)
    return 1.0 / (i * i)


def dense_spectrum(m, n, sigma, seed):
    """A = X diag(sigma) Y^T, X (m x r) and Y (n x r) orthonormal, r = len(sigma)."""
    rng = _rng(seed)
    r = len(sigma)
    X = orthonormal(m, r, rng)
    Y = orthonormal(n, r, rng)
    return (X * sigma[None, :]) @ Y.T


def dense_low_rank_plus_noise(m, n, rank, noise, seed, dtype=np.float32):
    """A = G1 G2 + noise * N(0,1), G1 (m x rank) and G2 (rank x n) Gaussian."""
    rng = _rng(seed)
    G1 = rng.standard_normal((m, rank))
    G2 = rng.standard_normal((rank, n))
    A = G1 @ G2
    if noise:
        A += noise * rng.standard_normal((m, n))
    return A.astype(dtype)


def exact_rank(m, n, rank, seed, dtype=np.float64):
    """An exactly rank-`rank` product of Gaussians (no noise)."""
    return dense_low_rank_plus_noise(m, n, rank, 0.0, seed, dtype=np.float64).astype(dtype)


def csr_sparse_plus_low_rank(m, n, nnz_per_row, lr_rows, lr_rank, seed, dtype=np.float32):
    """CSR matrix: `nnz_per_row` distinct uniform columns per row with N(0,1)
    values, plus a dense rank-`lr_rank` Gaussian product U V^T added to
    `lr_rows` randomly chosen rows (those rows become dense).

    Returns (rowptr int64, colind int32, val dtype, m, n).
    """
    rng = _rng(seed)
    npr = min(nnz_per_row, n)
    # distinct sorted columns per row: a random subset of size npr
    cols = np.empty((m, npr), dtype=np.int64)
    for r0 in range(0, m, 8192):
        r1 = min(m, r0 + 8192)
        keys = rng.random((r1 - r0, n)) if n <= 4096 else None
        if keys is not None:
            cols[r0:r1] = np.sort(np.argpartition(keys, npr - 1, axis=1)[:, :npr], axis=1)
        else:
            for r in range(r0, r1):
                cols[r] = np.sort(rng.choice(n, size=npr, replace=False))
    vals = rng.standard_normal((m, npr))
    dense_rows = np.sort(rng.choice(m, size=min(lr_rows, m), replace=False)) if lr_rows else np.zeros(0, np.int64)
    U = rng.standard_normal((len(dense_rows), lr_rank)) if lr_rows else None
    V = rng.standard_normal((n, lr_rank)) if lr_rows else None
    is_dense = np.zeros(m, dtype=bool)
    is_dense[dense_rows] = True
    counts = np.where(is_dense, n, npr).astype(np.int64)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    colind = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=dtype)
    sparse_rows = np.nonzero(~is_dense)[0]
    # sparse rows
    starts = rowptr[sparse_rows]
    idx = (starts[:, None] + np.arange(npr)[None, :]).ravel()
    colind[idx] = cols[sparse_rows].ravel()
    val[idx] = vals[sparse_rows].ravel().astype(dtype)
    # dense rows: sparse entries plus the low-rank part on every column
    full = np.arange(n, dtype=np.int32)
    for t, r in enumerate(dense_rows):
        row = U[t] @ V.T
        row[cols[r]] += vals[r]
        s0 = rowptr[r]
        colind[s0:s0 + n] = full
        val[s0:s0 + n] = row.astype(dtype)
    return rowptr, colind, val, m, n


def csr_to_scipy(rowptr, colind, val, m, n):
    return scipy.sparse.csr_matrix((np.asarray(val, dtype=np.float64), colind, rowptr), shape=(m, n))


def round_to_bf16(x):
    """Round-to-nearest-even to bfloat16, returned as float32 values and as the
    raw uint16 bit patterns."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)
    bits = r.astype(np.uint16)
    back = (bits.astype(np.uint32) << np.uint32(16)).view(np.float32)
    return back, bits


def make_dense(w: Workload, m=None, n=None):
    """The dense matrix of workload `w`, optionally at a reduced size with the
    same construction.  Returns a numpy array in the storage dtype (bf16 is
    returned as float32 values already rounded to bf16)."""
    m = w.m if m is None else m
    n = w.n if n is None else n
    if w is DENSE_F64_1K or w.name == DENSE_F64_1K.name:
        r = min(m, n)
        return dense_spectrum(m, n, geometric_spectrum(r), w.data_seed)
    if w.name == DENSE_F32_8K.name:
        return dense_low_rank_plus_noise(m, n, w.k, 1e-6, w.data_seed)
    if w.name == DENSE_BF16_32K.name:
        r = min(m, n, 2048)
        A = dense_spectrum(m, n, inverse_square_spectrum(r), w.data_seed)
        return round_to_bf16(A)[0]
    raise ValueError(w.name)
