"""Plain FP64 CPU oracle for the sparse randomized LU hot path.

TEST INFRASTRUCTURE ONLY.  This module is the correctness oracle for the CUDA
path.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
may import or execute it; the product path never does, and the two share no
code (not even the random-number generator: each side implements Philox
from its published definition).

It follows Aizenbud, Shabat and Averbuch, "Randomized LU decomposition using
sparse projections" (arXiv 1601.04280), step by step and in FP64:

  step 1 of Algorithm 1   draw the sparse embedding matrix S (Sec. 2.2) and
                          the random signs and column subsample of the
                          FFT-based projection (Sec. 2.1);
  step 2                  Y = A S D H R / sqrt(l1): CountSketch (Sec. 2.2),
                          signs, real Hartley transform, subsample;
  step 3                  P Y = L_Y U_Y, partial (row) pivoting; L_y is the
                          first k columns of L_Y;
  steps 5-6 (replaced)    B = L_y^+ P A with the exact pseudo-inverse, the
                          object bounded by Corollary 3.3 (col:A_LLA), or
                          (factor_two_sketch) the paper's own steps 4-5:
                          B = (Omega_2 L_1)^+ Omega_2 P A;
  step 6                  B Q = L_b U_b, LU with right (column) pivoting;
  step 7                  L = L_y L_b, U = U_b.

Points the paper leaves open are read as follows, and each function restates
the reading it uses: the FFT-based projection is real (random +-1 signs and
the real Hartley transform cas = cos + sin, i.e. Re - Im of the DFT, scaled by
1/sqrt(l1)), because the LU that follows must be real; the l-column sketch is
factored for l steps and then truncated to rank k <= l; in the LU with right
pivoting U is the unit-diagonal factor; pivots follow LAPACK getf2 (first
maximal magnitude wins; an exactly zero pivot skips the division).
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg
import scipy.sparse

from .philox import stream_blocks

#: second key word of every Philox stream of the method ("RANDLU" in ASCII)
KEY_TAG = 0x52414E444C5500

STATUS_OK = 0
STATUS_WRANK = 100  # an exact zero pivot was met; the factors are still valid


# ---------------------------------------------------------------------------
# Step 1: the random structures
# ---------------------------------------------------------------------------
#: the FFT-based projections of step 2 (transform of the l1 bucket sums)
TRANSFORMS = ("hartley", "srht", "srft")


@dataclass
class SketchParams:
    h: np.ndarray  # (n,) int64, bucket of column j, in [0, l1)
    s: np.ndarray  # (n,) float64, sign of column j, +-1
    d: np.ndarray  # (l1,) float64, random sign of Hartley input b, +-1
    R: np.ndarray  # (l,) int64, kept frequencies, in key order
    R_keys: np.ndarray = field(repr=False, default=None)  # (l1,) uint64
    theta: np.ndarray = field(repr=False, default=None)  # (l1,) phases of the complex D (srft)


def bucket_of_word(w, l1):
    """Bucket in [0, l1) of a uniform 64-bit word: floor(w * l1 / 2^64),
    exact in Python integers (the multiply-high form of a uniform draw)."""
    return (int(w) * int(l1)) >> 64


def sign_of_word(w):
    """Random sign of a uniform 64-bit word: -1 when its top bit is set."""
    return -1.0 if int(w) >= 2 ** 63 else 1.0


def sketch_params(n, l1, l, seed):
    """Draw h, s, d and R for one factorization (step 1 of Algorithm 1).

    Sec. 2.2: the sparse embedding matrix has, for every column index j, one
    nonzero entry at bucket h(j) with a uniform random sign s(j); h is uniform
    over the l1 buckets (reading of the "probability 1/t" passage).
    Sec. 2.1: D is a diagonal of random unit-modulus entries (here +-1, the
    real reading) and S a selection of l of the l1 transform outputs.

    Philox4x64-10 with key (seed, KEY_TAG); the block at counter
    (index, stream, 0, 0) gives words w0..w3:
      stream 0, j < n : h(j) = floor(w0 * l1 / 2^64), s(j) = -1 if w1 >= 2^63
      stream 1, b < l1: d(b) = -1 if w0 >= 2^63
      stream 2, b < l1: selection key w0; R = the l indices b with the
                        smallest (w0, b), in increasing key order.
    """
    if not (1 <= l <= l1):
        raise ValueError("need 1 <= l <= l1")
    key = (np.uint64(seed & 0xFFFFFFFFFFFFFFFF), np.uint64(KEY_TAG))
    b0 = stream_blocks(key, 0, n)
    h = np.array([bucket_of_word(w, l1) for w in b0[:, 0]], dtype=np.int64)
    s = np.array([sign_of_word(w) for w in b0[:, 1]], dtype=np.float64)
    b1 = stream_blocks(key, 1, l1)
    d = np.array([sign_of_word(w) for w in b1[:, 0]], dtype=np.float64)
    b2 = stream_blocks(key, 2, l1)
    keys = b2[:, 0]
    order = sorted(range(l1), key=lambda b: (int(keys[b]), b))
    R = np.array(order[:l], dtype=np.int64)
    # stream 3, b < l1: the phase of the complex unit-modulus D of the SRFT
    b3 = stream_blocks(key, 3, l1)
    theta = np.array([phase_of_word(w) for w in b3[:, 0]], dtype=np.float64)
    return SketchParams(h=h, s=s, d=d, R=R, R_keys=keys, theta=theta)


def phase_of_word(w):
    """A uniform phase in [0, 2 pi) from a 64-bit word: 2 pi u with u the top
    53 bits of w over 2^53 (exact in FP64, so u < 1)."""
    return 2.0 * np.pi * ((int(w) >> 11) * 2.0 ** -53)


def sem_matrix(params, l1):
    """The n x l1 sparse embedding matrix S: S[j, h(j)] = s(j) (Sec. 2.2).

    The paper writes the SEM as l1 x n with one nonzero per column; this is
    its transpose, applied on the right of A.
    """
    n = params.h.shape[0]
    return scipy.sparse.csr_matrix(
        (params.s, (np.arange(n), params.h)), shape=(n, l1), dtype=np.float64)


# ---------------------------------------------------------------------------
# Step 2: the sketch Y = A * Omega_1^T
# ---------------------------------------------------------------------------
def countsketch(A, params, l1):
    """Y1 = A S, i.e. Y1[i, h(j)] += s(j) A[i, j] (Sec. 2.2, Lemma 2.6 cost).

    Computed as the product with the sparse S (one term per entry of A), so
    the cost is that of reading A once, as the paper states for the SEM.
    """
    S = sem_matrix(params, l1)
    if scipy.sparse.issparse(A):
        return np.asarray((A.tocsr().astype(np.float64) @ S).todense())
    A = np.asarray(A, dtype=np.float64)
    return np.asarray((S.T.tocsr() @ A.T).T)


def hartley_columns(l1, freqs):
    """cas(2 pi b f / l1) for b < l1 and f in freqs: an l1 x len(freqs) array.

    The real Hartley kernel cas = cos + sin is Re - Im of the DFT kernel of
    Sec. 2.1 (reading for real data).  The product b*f is reduced modulo l1
    in integers before the angle is formed, so the angle is exact to FP64.
    """
    b = np.arange(l1, dtype=np.int64)[:, None]
    t = (b * np.asarray(freqs, dtype=np.int64)[None, :]) % l1
    ang = 2.0 * np.pi * t.astype(np.float64) / l1
    return np.cos(ang) + np.sin(ang)


def hadamard_columns(l1, cols):
    """Columns `cols` of the l1 x l1 Walsh-Hadamard matrix in Sylvester order,
    H[b, c] = (-1)^popcount(b & c), l1 a power of two (the SRHT of Sec. 4)."""
    if l1 & (l1 - 1):
        raise ValueError("the Walsh-Hadamard transform needs l1 a power of two")
    b = np.arange(l1, dtype=np.int64)[:, None]
    x = b & np.asarray(cols, dtype=np.int64)[None, :]
    par = np.zeros_like(x)
    while np.any(x):
        par ^= x & 1
        x >>= 1
    return 1.0 - 2.0 * par


def srft_columns(l1, theta, freqs):
    """The real form of the complex SRFT of Sec. 2.1 (Pi = D F S with D
    diagonal of unit-modulus entries exp(i theta_b) and F the DFT): for each
    kept frequency f, the real and imaginary parts of exp(i theta_b) exp(-2 pi
    i b f / l1), interleaved: columns (cos phi, sin phi), phi_b = theta_b -
    2 pi (b f mod l1) / l1.  An l1 x 2 len(freqs) array."""
    b = np.arange(l1, dtype=np.int64)[:, None]
    t = (b * np.asarray(freqs, dtype=np.int64)[None, :]) % l1
    phi = theta[:, None] - 2.0 * np.pi * t.astype(np.float64) / l1
    out = np.empty((l1, 2 * len(freqs)))
    out[:, 0::2] = np.cos(phi)
    out[:, 1::2] = np.sin(phi)
    return out


def transform_matrix(params, l1, l, transform="hartley"):
    """The l1 x l matrix M of step 2's FFT-based projection, Y = Y1 M.

      hartley: D H R / sqrt(l1) with D = diag(d) (+-1), H the real Hartley
               kernel cas(2 pi b f / l1) (the default reading for real data);
      srht:    D W R / sqrt(l1) with W the Walsh-Hadamard matrix (l1 a power
               of two);
      srft:    the complex D F R with D = diag(exp(i theta)), realified: the
               first l/2 kept frequencies give the real and imaginary parts as
               two columns each, scaled by sqrt(2 / l1) (l even).
    Every variant keeps the l columns of R in key order.
    """
    if transform == "hartley":
        return params.d[:, None] * hartley_columns(l1, params.R) / np.sqrt(l1)
    if transform == "srht":
        return params.d[:, None] * hadamard_columns(l1, params.R) / np.sqrt(l1)
    if transform == "srft":
        if l % 2:
            raise ValueError("the realified SRFT needs an even l")
        return srft_columns(l1, params.theta, params.R[: l // 2]) * np.sqrt(2.0 / l1)
    raise ValueError("unknown transform %r" % (transform,))


def fjl(Y1, params, l1, transform="hartley"):
    """Y = Y1 M with M = transform_matrix(...): signs (or phases), the
    transform, the subsample.

    Direct O(l1 * l) sum per row (Lemma 2.1 states the fast-transform cost; the
    oracle deliberately uses the plain definition instead).
    """
    return Y1 @ transform_matrix(params, l1, len(params.R), transform)


# ---------------------------------------------------------------------------
# Steps 3 and 6: LU with partial pivoting
# ---------------------------------------------------------------------------
@dataclass
class LUResult:
    lu: np.ndarray    # packed factors of the row-permuted input, m x n
    perm: np.ndarray  # (m,) int64: row i of the permuted input is input row perm[i]
    zero_pivot: bool  # an exactly zero pivot column was met
    gaps: np.ndarray  # (steps,) relative gap between the two largest candidates
    top: np.ndarray = None  # (steps, 2) the two largest candidate magnitudes


def lu_partial_pivot(X, steps=None):
    """Right-looking LU with partial pivoting, `steps` elimination steps.

    LAPACK getf2 semantics: at step j the pivot is the first row (in the
    current, already swapped order) among j..m-1 attaining max |X[:, j]|;
    rows j and pivot are swapped; if the pivot is nonzero the column below it
    is divided by it, and the trailing block receives the rank-1 update.  An
    exactly zero pivot skips the division (the column is zero anyway) and is
    reported.  The `gaps` record, per step, (top1 - top2) / top1 of the
    candidate magnitudes and `top` the two magnitudes themselves, so that
    callers can tell well-separated pivots.
    """
    X = np.array(X, dtype=np.float64, copy=True)
    m, n = X.shape
    if steps is None:
        steps = min(m, n)
    perm = np.arange(m, dtype=np.int64)
    gaps = np.zeros(steps)
    top = np.zeros((steps, 2))
    zero_pivot = False
    for j in range(steps):
        col = np.abs(X[j:, j])
        pj = j + int(np.argmax(col))
        if col.size > 1:
            top2 = np.partition(col, col.size - 2)[-2:]
            t1, t2 = top2[1], top2[0]
            gaps[j] = (t1 - t2) / t1 if t1 > 0 else 0.0
            top[j] = (t1, t2)
        else:
            gaps[j] = 1.0
            top[j] = (col[0], 0.0)
        if pj != j:
            X[[j, pj], :] = X[[pj, j], :]
            perm[[j, pj]] = perm[[pj, j]]
        piv = X[j, j]
        if piv != 0.0:
            X[j + 1:, j] /= piv
            X[j + 1:, j + 1:] -= np.outer(X[j + 1:, j], X[j, j + 1:])
        else:
            zero_pivot = True
    return LUResult(lu=X, perm=perm, zero_pivot=zero_pivot, gaps=gaps, top=top)


def unit_lower(lu, k):
    """First k columns of the unit lower trapezoidal factor in packed `lu`."""
    L = np.tril(lu[:, :k], -1)
    L[np.arange(k), np.arange(k)] = 1.0
    return L


# ---------------------------------------------------------------------------
# Steps 5-6: B = L_y^+ (P A)
# ---------------------------------------------------------------------------
def pinv_householder(Ly):
    """L_y^+ = R^{-1} Q^T from the Householder QR L_y = Q R (full column rank).

    Corollary 3.3 (col:A_LLA) uses L L^+ P A; for a full-column-rank L the
    Moore-Penrose pseudo-inverse is R^{-1} Q^T.
    """
    Q, Rq = np.linalg.qr(Ly, mode="reduced")
    return scipy.linalg.solve_triangular(Rq, Q.T, lower=False)


def row_gather(A, p):
    if scipy.sparse.issparse(A):
        return A.tocsr()[p]
    return np.asarray(A, dtype=np.float64)[p]


# ---------------------------------------------------------------------------
# The whole path
# ---------------------------------------------------------------------------
@dataclass
class OracleResult:
    L: np.ndarray       # m x k, lower trapezoidal (rows in P order)
    U: np.ndarray       # k x n, unit upper trapezoidal (columns in Q order)
    p: np.ndarray       # (m,) int64: (P A)[i, :] = A[p[i], :]
    q: np.ndarray       # (n,) int64: (A Q)[:, j] = A[:, q[j]]
    status: int
    params: SketchParams
    Y: np.ndarray       # m x l sketch
    Ly: np.ndarray      # m x k unit lower trapezoidal
    W: np.ndarray       # k x m, L_y^+
    B: np.ndarray       # k x n
    Lb: np.ndarray      # k x k lower
    Ub: np.ndarray      # k x n unit upper
    gaps_y: np.ndarray  # pivot separation of the panel LU
    gaps_b: np.ndarray  # pivot separation of the LU of B
    top_y: np.ndarray = None  # (l, 2) two largest candidate magnitudes per step
    top_b: np.ndarray = None  # (k, 2)
    Y2: np.ndarray = None     # k2 x n, Omega_2 P A (second projection only)
    Z: np.ndarray = None      # k2 x k, Omega_2 L_y (second projection only)
    ycols: np.ndarray = None  # (l,) column order of the sketch (column pivoting; identity otherwise)


def check_sizes(m, n, k, l, l1):
    if not (1 <= k <= l <= l1):
        raise ValueError("need 1 <= k <= l <= l1")
    if l > m or k > min(m, n):
        raise ValueError("need l <= m and k <= min(m, n)")


def column_order_greedy(Y):
    """Column order of Y by QR with column pivoting (Businger and Golub): at
    each step the column with the largest norm after removing the span of the
    columns already chosen; ties to the smallest index (LAPACK geqp3).
    Written as the greedy pivoted Cholesky of Y^T Y, which makes the same
    choices in exact arithmetic: the diagonal of the Schur complement holds
    the squared residual norms."""
    G = np.array(Y.T @ Y, dtype=np.float64)
    l = G.shape[0]
    order = np.arange(l)
    for j in range(l):
        d = np.diag(G)[j:]
        c = j + int(np.argmax(d))
        if c != j:
            G[[j, c], :] = G[[c, j], :]
            G[:, [j, c]] = G[:, [c, j]]
            order[[j, c]] = order[[c, j]]
        piv = G[j, j]
        if piv <= 0.0:
            break  # the remaining columns lie in the span of the chosen ones
        r = G[j, j + 1:] / np.sqrt(piv)
        G[j + 1:, j + 1:] -= np.outer(r, r)
        G[j + 1:, j] = G[j, j + 1:] = 0.0
    return order


def factor(A, k, l, l1, seed, transform="hartley", column_pivoting=False):
    """Sparse randomized LU of A (dense ndarray or scipy.sparse), all FP64.
    `transform` selects step 2's FFT-based projection (transform_matrix).
    `column_pivoting` orders the sketch's columns by QR with column pivoting
    before the panel LU (a rank-revealing choice of the k columns that span
    L_y, beyond Algorithm 1): Y := Y[:, column_order_greedy(Y)]."""
    m, n = A.shape
    check_sizes(m, n, k, l, l1)
    status = STATUS_OK
    # step 1
    params = sketch_params(n, l1, l, seed)
    # step 2
    Y = fjl(countsketch(A, params, l1), params, l1, transform)
    ycols = np.arange(l)
    if column_pivoting:
        ycols = column_order_greedy(Y)
        Y = Y[:, ycols]
    # step 3: l elimination steps on the m x l sketch, then truncate to k
    ly = lu_partial_pivot(Y, steps=l)
    if ly.zero_pivot:
        status = STATUS_WRANK
    p = ly.perm
    Ly = unit_lower(ly.lu, k)
    # steps 5-6 with the exact pseudo-inverse
    W = pinv_householder(Ly)
    PA = row_gather(A, p)
    if scipy.sparse.issparse(PA):
        B = np.asarray((PA.T @ W.T).T)
    else:
        B = W @ PA
    # step 6: right (column) pivoting = partial pivoting of B^T, k steps.
    # B^T[q] = L_x U_x  =>  B Q = U_x^T L_x^T: L_b = U_x^T (lower, non-unit),
    # U_b = L_x^T (unit upper, |U_b| <= 1).
    lb = lu_partial_pivot(B.T, steps=k)
    if lb.zero_pivot:
        status = STATUS_WRANK
    q = lb.perm
    Lb = np.triu(lb.lu[:k, :k]).T
    Ub = unit_lower(lb.lu, k).T
    # step 7
    L = Ly @ Lb
    return OracleResult(L=L, U=Ub, p=p, q=q, status=status, params=params,
                        Y=Y, Ly=Ly, W=W, B=B, Lb=Lb, Ub=Ub,
                        gaps_y=ly.gaps, gaps_b=lb.gaps, top_y=ly.top, top_b=lb.top, ycols=ycols)


def second_projection(M, params2, l2):
    """Omega_2 M for an m x c matrix M: the second sparse projection of
    Algorithm 1 (steps 4-5), Omega_2 = Pi_2 S_2 of size k2 x m, acting on the
    rows of M.  It is the first projection applied to M^T: CountSketch of the
    m rows into l2 buckets (S_2, Sec. 2.2), signs, real Hartley transform,
    subsample of k2 outputs (Pi_2, Sec. 2.1), transposed back."""
    if scipy.sparse.issparse(M):
        Mt = M.T.tocsr()
    else:
        Mt = np.asarray(M, dtype=np.float64).T
    return fjl(countsketch(Mt, params2, l2), params2, l2).T


def factor_two_sketch(A, k, l, l1, k2, l2, seed, seed2):
    """Algorithm 1 with its own second projection (steps 4-6).

    Steps 1-3 as in factor().  Step 4 draws Omega_2 = Pi_2 S_2 (k2 x m) from
    seed2; step 5 forms Z = Omega_2 L_1 and its pseudo-inverse; step 6 factors
    B = Z^+ Omega_2 P A with right pivoting.  Reading: S_2 hashes the ORIGINAL
    row index i of A (bucket h_2(i), sign s_2(i)), i.e. the sketch of P A is
    Omega_2' P^T with Omega_2' acting on A's rows; P does not depend on
    Omega_2, so this is an SEM of the same law, and it lets both Omega_2 P A =
    Omega_2' A and Omega_2 L_1 = Omega_2' Lk (Lk = L_1 with its rows put back in
    the original order) be formed without gathering rows.
    """
    m, n = A.shape
    check_sizes(m, n, k, l, l1)
    if not (k <= k2 <= l2):
        raise ValueError("need k <= k2 <= l2")
    status = STATUS_OK
    params = sketch_params(n, l1, l, seed)
    Y = fjl(countsketch(A, params, l1), params, l1)
    ly = lu_partial_pivot(Y, steps=l)
    if ly.zero_pivot:
        status = STATUS_WRANK
    p = ly.perm
    Ly = unit_lower(ly.lu, k)
    # steps 4-5: Omega_2 over the original rows
    params2 = sketch_params(m, l2, k2, seed2)
    Lk = np.empty_like(Ly)
    Lk[p] = Ly
    Z = second_projection(Lk, params2, l2)    # k2 x k
    Y2 = second_projection(A, params2, l2)    # k2 x n
    W = pinv_householder(Z)                   # k x k2
    B = W @ Y2
    lb = lu_partial_pivot(B.T, steps=k)
    if lb.zero_pivot:
        status = STATUS_WRANK
    q = lb.perm
    Lb = np.triu(lb.lu[:k, :k]).T
    Ub = unit_lower(lb.lu, k).T
    L = Ly @ Lb
    return OracleResult(L=L, U=Ub, p=p, q=q, status=status, params=params,
                        Y=Y, Ly=Ly, W=W, B=B, Lb=Lb, Ub=Ub,
                        gaps_y=ly.gaps, gaps_b=lb.gaps, top_y=ly.top, top_b=lb.top, Y2=Y2, Z=Z)


def relative_residual(A, L, U, p, q):
    """||L U - P A Q||_F / ||A||_F in FP64 (the error of Sec. 1, Eq. (1)).

    Dense A: the difference is formed explicitly.  Sparse A: the expansion
    ||LU||^2 - 2 <LU, PAQ> + ||A||^2 avoids densifying A; ||LU||_F^2 is
    trace((L^T L)(U U^T)) and the inner product runs over the nonzeros.
    """
    L = np.asarray(L, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    p = np.asarray(p, dtype=np.int64)
    q = np.asarray(q, dtype=np.int64)
    if not scipy.sparse.issparse(A):
        A = np.asarray(A, dtype=np.float64)
        D = L @ U - A[p][:, q]
        return float(np.linalg.norm(D) / np.linalg.norm(A))
    A = A.tocoo()
    m, n = A.shape
    pinv = np.empty(m, dtype=np.int64)
    pinv[p] = np.arange(m)
    qinv = np.empty(n, dtype=np.int64)
    qinv[q] = np.arange(n)
    lu2 = float(np.sum((L.T @ L) * (U @ U.T)))
    a2 = float(np.sum(A.data.astype(np.float64) ** 2))
    inner = 0.0
    chunk = 1 << 20
    for s0 in range(0, A.nnz, chunk):
        r = pinv[A.row[s0:s0 + chunk]]
        c = qinv[A.col[s0:s0 + chunk]]
        v = A.data[s0:s0 + chunk].astype(np.float64)
        inner += float(np.sum(v * np.einsum("ij,ji->i", L[r], U[:, c])))
    return float(np.sqrt(max(lu2 - 2.0 * inner + a2, 0.0) / a2))
