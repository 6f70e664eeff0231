"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each pin compares an oracle step with an independent route: numpy's own
Philox, numpy's FFT, scipy's LAPACK LU, SVD-based projectors, closed forms
from the paper (Lemma 2.2, Lemma 2.4 and its remark, Theorem 2.3,
Corollary 3.3) and brute force on tiny inputs.  The planted-mistake tests at
the end show that plausible slips in the oracle fail at least one pin.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse

import oracle
import rlu_inputs as ri


# ---------------------------------------------------------------------------
# Philox4x64-10 (the generator of step 1 of Algorithm 1)
# ---------------------------------------------------------------------------
def test_mulhilo64_exact():
    rng = np.random.default_rng(1)
    a = rng.integers(0, 2**64, size=200, dtype=np.uint64)
    b = rng.integers(0, 2**64, size=200, dtype=np.uint64)
    a[0], b[0] = np.uint64(2**64 - 1), np.uint64(2**64 - 1)
    hi, lo = oracle.mulhilo64(a, b)
    for x, y, h, l in zip(a, b, hi, lo):
        p = int(x) * int(y)
        assert int(h) == p >> 64 and int(l) == p & (2**64 - 1)


def numpy_philox_block(key, counter_before):
    """One block from numpy's Philox, its state set word by word as uint64
    (numpy's constructor would pass large counters through float64)."""
    bg = np.random.Philox(key=[0, 0])
    st = bg.state
    st["state"]["counter"] = np.array(counter_before, dtype=np.uint64)
    st["state"]["key"] = np.array(key, dtype=np.uint64)
    st["buffer_pos"] = 4
    bg.state = st
    return bg.random_raw(4)


@pytest.mark.parametrize("key", [(0, 0), (1, 2), (2**64 - 1, oracle.KEY_TAG), (12345, 2**63 + 7)])
def test_philox_matches_numpy(key):
    # numpy's Philox is an independent implementation of the same published
    # generator; it increments its 256-bit counter before each block, so the
    # block for counter c comes from a generator started at c - 1.
    rng = np.random.default_rng(7)
    for _ in range(20):
        c = [int(x) for x in rng.integers(0, 2**64, size=4, dtype=np.uint64)]
        c[0] = max(c[0], 1)  # keep c - 1 free of a borrow across words
        ref = numpy_philox_block(key, [c[0] - 1] + c[1:])
        mine = oracle.philox4x64_10([c], key)[0]
        assert list(map(int, ref)) == list(map(int, mine))
    # a borrow across words: index 0 of stream 5
    ref = numpy_philox_block(key, [2**64 - 1, 4, 0, 0])
    mine = oracle.stream_blocks(key, 5, 1)[0]
    assert list(map(int, ref)) == list(map(int, mine))


# ---------------------------------------------------------------------------
# Step 1's mapping from Philox words to h, s, d and R, restated from its
# specification with numpy's own Philox stepping through each stream
# ---------------------------------------------------------------------------
def numpy_stream(key, stream, count):
    """Blocks (i, stream, 0, 0), i < count, from numpy's Philox: started one
    below counter (0, stream, 0, 0) (a 256-bit little-endian integer, so the
    decrement borrows across words), it increments before each block."""
    before = ((stream << 64) - 1) % (1 << 256)
    words = [(before >> (64 * i)) & (2**64 - 1) for i in range(4)]
    bg = np.random.Philox(key=[0, 0])
    st = bg.state
    st["state"]["counter"] = np.array(words, dtype=np.uint64)
    st["state"]["key"] = np.array(key, dtype=np.uint64)
    st["buffer_pos"] = 4
    bg.state = st
    return bg.random_raw(4 * count).reshape(count, 4)


@pytest.mark.parametrize("n,l1,l,seed", [(1000, 240, 30, 1), (3000, 1600, 220, 2001), (500, 4000, 520, 2**63 + 5),
                                         (64, 7, 7, 0)])
def test_sketch_params_from_numpy_philox(n, l1, l, seed):
    """h(j) = floor(w0 l1 / 2^64), s(j) = -1 iff w1 >= 2^63 on stream 0;
    d(b) = -1 iff w0 >= 2^63 on stream 1; R = the l indices b of smallest
    (w0, b) on stream 2, in that order.  Words from numpy's generator, the
    mapping written out here with Python integers."""
    key = [seed % 2**64, oracle.KEY_TAG]
    p = oracle.sketch_params(n, l1, l, seed)
    b0 = numpy_stream(key, 0, n)
    assert [int(x) for x in p.h] == [(int(w) * l1) >> 64 for w in b0[:, 0]]
    assert [int(x) for x in p.s] == [-1 if int(w) >> 63 else 1 for w in b0[:, 1]]
    b1 = numpy_stream(key, 1, l1)
    assert [int(x) for x in p.d] == [-1 if int(w) >> 63 else 1 for w in b1[:, 0]]
    b2 = numpy_stream(key, 2, l1)
    ranked = sorted(range(l1), key=lambda b: (int(b2[b, 0]), b))
    assert [int(x) for x in p.R] == ranked[:l]


def test_word_mapping_boundaries():
    """The edges of the word-to-bucket and word-to-sign maps."""
    for l1 in (7, 240, 1600, 4000, 16384):
        assert oracle.bucket_of_word(0, l1) == 0
        assert oracle.bucket_of_word(2**64 - 1, l1) == l1 - 1
        for b in (1, l1 // 2, l1 - 1):
            first = -(-(b << 64) // l1)  # smallest word of bucket b: ceil(b 2^64 / l1)
            assert oracle.bucket_of_word(first, l1) == b
            assert oracle.bucket_of_word(first - 1, l1) == b - 1
    assert oracle.sign_of_word(2**63) == -1.0
    assert oracle.sign_of_word(2**63 - 1) == 1.0
    assert oracle.sign_of_word(0) == 1.0 and oracle.sign_of_word(2**64 - 1) == -1.0


# ---------------------------------------------------------------------------
# Sparse embedding matrix (Sec. 2.2)
# ---------------------------------------------------------------------------
def test_sketch_params_ranges_and_selection():
    n, l1, l = 5000, 240, 30
    p = oracle.sketch_params(n, l1, l, seed=99)
    assert p.h.min() >= 0 and p.h.max() < l1
    assert set(np.unique(p.s)) <= {-1.0, 1.0} and set(np.unique(p.d)) <= {-1.0, 1.0}
    assert len(set(p.R.tolist())) == l
    keys = [(int(p.R_keys[b]), b) for b in p.R]
    assert keys == sorted(keys)
    # the selected keys are the l smallest of all l1 keys
    allkeys = sorted((int(p.R_keys[b]), b) for b in range(l1))
    assert keys == allkeys[:l]
    # uniformity of h: chi-square over the l1 buckets, loose 6-sigma bound
    counts = np.bincount(p.h, minlength=l1)
    chi2 = float(np.sum((counts - n / l1) ** 2 / (n / l1)))
    assert abs(chi2 - (l1 - 1)) < 6 * math.sqrt(2 * (l1 - 1))
    # signs are balanced within 6 sigma
    assert abs(p.s.sum()) < 6 * math.sqrt(n)


def test_sketch_params_prefix_stable():
    # h, s of the first columns do not depend on n; d does not depend on l
    a = oracle.sketch_params(100, 64, 8, seed=5)
    b = oracle.sketch_params(300, 64, 16, seed=5)
    assert np.array_equal(a.h, b.h[:100]) and np.array_equal(a.s, b.s[:100])
    assert np.array_equal(a.d, b.d)
    assert np.array_equal(a.R, b.R[:8])


@pytest.mark.parametrize("n,l1", [(1024, 240), (8192, 1600), (3000, 4000)])
def test_sem_identities(n, l1):
    p = oracle.sketch_params(n, l1, min(l1, 8), seed=2024)
    S = oracle.sem_matrix(p, l1).toarray()  # n x l1, the transpose of the paper's SEM
    kappa = np.bincount(p.h, minlength=l1)
    # Lemma (Sec. 2.2): ||S||_F = sqrt(n)
    assert np.isclose(np.linalg.norm(S), math.sqrt(n), rtol=0, atol=1e-9)
    # Lemma 2.4 and its remark: S^T S = diag(kappa) (one nonzero per column
    # of the paper's l1 x n SEM), so the singular values are sqrt(kappa)
    assert np.array_equal(S.T @ S, np.diag(kappa.astype(float)))
    assert kappa.sum() == n
    sv = np.linalg.svd(S, compute_uv=False)
    assert np.allclose(np.sort(sv)[::-1][: np.count_nonzero(kappa)],
                       np.sort(np.sqrt(kappa[kappa > 0]))[::-1], atol=1e-9)
    assert np.isclose(sv.max(), math.sqrt(kappa.max()), atol=1e-9)
    # Theorem 2.3 (whp, "n large enough"): max bucket <= n/l1 + sqrt(2 (n/l1) log l1)
    if n > l1:
        bound = n / l1 + math.sqrt(2 * (n / l1) * math.log(l1))
        assert kappa.max() <= bound + 3 * math.sqrt(n / l1)


def test_countsketch_brute_force():
    rng = np.random.default_rng(3)
    m, n, l1 = 7, 40, 9
    A = rng.standard_normal((m, n))
    p = oracle.sketch_params(n, l1, 4, seed=11)
    Y1 = oracle.countsketch(A, p, l1)
    ref = np.zeros((m, l1))
    for i in range(m):
        for j in range(n):
            ref[i, int(p.h[j])] += p.s[j] * A[i, j]
    assert np.allclose(Y1, ref, rtol=0, atol=1e-13)
    # sparse input gives the same sketch
    As = scipy.sparse.csr_matrix(np.where(np.abs(A) > 0.8, A, 0.0))
    assert np.allclose(oracle.countsketch(As, p, l1), oracle.countsketch(As.toarray(), p, l1), atol=1e-13)


# ---------------------------------------------------------------------------
# Real Hartley transform and the FFT-based projection (Sec. 2.1)
# ---------------------------------------------------------------------------
def fft_route_Y(Y1, p, l1):
    """Y computed through numpy's FFT: DHT = Re X - Im X of X = fft(x)."""
    X = np.fft.fft(Y1 * p.d[None, :], axis=1)
    H = X.real - X.imag
    return H[:, p.R] / math.sqrt(l1)


@pytest.mark.parametrize("l1", [240, 1600, 960, 7, 251, 12])
def test_hartley_vs_numpy_fft(l1):
    rng = np.random.default_rng(l1)
    x = rng.standard_normal((3, l1))
    Hm = oracle.hartley_columns(l1, np.arange(l1))
    X = np.fft.fft(x, axis=1)
    assert np.allclose(x @ Hm, X.real - X.imag, atol=1e-9 * math.sqrt(l1))
    # self-inverse up to l1, symmetric, Parseval
    assert np.allclose(Hm @ Hm, l1 * np.eye(l1), atol=1e-8 * l1)
    assert np.allclose(Hm, Hm.T, atol=0)
    y = x @ Hm / math.sqrt(l1)
    assert np.allclose(np.sum(y * y, axis=1), np.sum(x * x, axis=1), rtol=1e-12)


def test_fjl_vs_fft_route():
    rng = np.random.default_rng(4)
    m, n, l1, l = 50, 300, 240, 30
    A = rng.standard_normal((m, n))
    p = oracle.sketch_params(n, l1, l, seed=8)
    Y1 = oracle.countsketch(A, p, l1)
    assert np.allclose(oracle.fjl(Y1, p, l1), fft_route_Y(Y1, p, l1), atol=1e-11)


# ---------------------------------------------------------------------------
# LU with partial pivoting (steps 3 and 6)
# ---------------------------------------------------------------------------
def ipiv_to_perm(ipiv, m):
    perm = np.arange(m)
    for j, pj in enumerate(ipiv):
        perm[[j, pj]] = perm[[pj, j]]
    return perm


@pytest.mark.parametrize("shape", [(9, 9), (40, 7), (200, 30), (64, 64)])
def test_lu_matches_lapack(shape):
    rng = np.random.default_rng(sum(shape))
    X = rng.standard_normal(shape)
    res = oracle.lu_partial_pivot(X)
    lu, piv = scipy.linalg.lu_factor(X)
    steps = min(shape)
    assert np.array_equal(res.perm, ipiv_to_perm(piv[:steps], shape[0]))
    assert np.allclose(res.lu, lu, atol=1e-12)
    L = oracle.unit_lower(res.lu, steps)
    Uf = np.triu(res.lu[:steps])
    assert np.allclose(L @ Uf, X[res.perm], atol=1e-12)
    assert np.all(np.abs(L) <= 1.0 + 1e-15)


def test_lu_partial_steps_truncation():
    # l steps followed by truncation to k: the first k columns of L_Y equal
    # those of a k-step factorization of the first k columns of Y
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((100, 12))
    full = oracle.lu_partial_pivot(Y, steps=12)
    part = oracle.lu_partial_pivot(Y[:, :5], steps=5)
    assert np.array_equal(full.perm[:5], part.perm[:5])
    assert np.allclose(oracle.unit_lower(full.lu, 5)[np.argsort(full.perm)],
                       oracle.unit_lower(part.lu, 5)[np.argsort(part.perm)], atol=1e-12)


def test_lu_ties_and_zero_pivots():
    # all zero: identity permutation, zero pivots reported, factors zero
    res = oracle.lu_partial_pivot(np.zeros((6, 3)))
    assert np.array_equal(res.perm, np.arange(6)) and res.zero_pivot
    # equal magnitudes: the first row in the current order wins
    X = np.array([[1.0, 2.0], [-3.0, 1.0], [3.0, 5.0], [2.0, 0.0]])
    res = oracle.lu_partial_pivot(X)
    lu, piv = scipy.linalg.lu_factor(X)
    assert res.perm[0] == 1
    assert np.array_equal(res.perm, ipiv_to_perm(piv, 4))
    # a zero column in the middle: no division, the factorization still holds
    X = np.array([[2.0, 0.0, 1.0], [1.0, 0.0, 4.0], [4.0, 0.0, 3.0]])
    X[:, 1] = 0.5 * X[:, 0]
    res = oracle.lu_partial_pivot(X)
    assert res.zero_pivot
    L = oracle.unit_lower(res.lu, 3)
    assert np.allclose(L @ np.triu(res.lu), X[res.perm], atol=1e-14)


# ---------------------------------------------------------------------------
# The pseudo-inverse (Corollary 3.3) and the whole path
# ---------------------------------------------------------------------------
def test_pinv_matches_svd_pinv():
    rng = np.random.default_rng(6)
    Ly = oracle.unit_lower(oracle.lu_partial_pivot(rng.standard_normal((80, 10))).lu, 10)
    W = oracle.pinv_householder(Ly)
    assert np.allclose(W @ Ly, np.eye(10), atol=1e-12)
    assert np.allclose(W, np.linalg.pinv(Ly), atol=1e-12)


def projector_error(A, Yk):
    """||(I - Pi_{range(Yk)}) A||_F / ||A||_F with the projector from an SVD."""
    Uy, sv, _ = np.linalg.svd(Yk, full_matrices=False)
    Uy = Uy[:, sv > sv[0] * 1e-13]
    Ad = A.toarray() if scipy.sparse.issparse(A) else A
    return np.linalg.norm(Ad - Uy @ (Uy.T @ Ad)) / np.linalg.norm(Ad)


def check_structure(r, m, n, k):
    assert r.L.shape == (m, k) and r.U.shape == (k, n)
    assert np.array_equal(np.sort(r.p), np.arange(m))
    assert np.array_equal(np.sort(r.q), np.arange(n))
    assert np.allclose(np.triu(r.L[:k], 1), 0.0)
    assert np.allclose(np.tril(r.U, -1)[:, :k], 0.0)
    assert np.allclose(np.diag(r.U), 1.0)
    assert np.all(np.abs(r.U) <= 1.0 + 1e-12)
    assert np.all(np.abs(r.Ly) <= 1.0 + 1e-12)
    assert np.allclose(np.diag(r.Ly), 1.0) and np.allclose(np.triu(r.Ly[:k], 1), 0.0)


@pytest.mark.parametrize("m,n,k,l,l1,seed", [(300, 200, 10, 15, 60, 1), (257, 301, 20, 30, 240, 2),
                                              (128, 512, 16, 16, 100, 3)])
def test_closed_form_error(m, n, k, l, l1, seed):
    # ||LU - PAQ||_F = ||(I - Pi_{Y[:, :k]}) A||_F: the pivots, L_b and U_b drop
    # out because range(L_y) = range(P Y[:, :k]) (Corollary 3.3 with LU = L_y B Q)
    A = ri.dense_spectrum(m, n, ri.geometric_spectrum(min(m, n), 15.0), seed)
    r = oracle.factor(A, k, l, l1, seed=seed + 10)
    e = oracle.relative_residual(A, r.L, r.U, r.p, r.q)
    assert np.isclose(e, projector_error(A, r.Y[:, :k]), rtol=1e-9)
    check_structure(r, m, n, k)
    # B Q = L_b U_b and the lower bound Delta_k (Eckart-Young)
    assert np.allclose(r.B[:, r.q], r.Lb @ r.Ub, atol=1e-10 * np.abs(r.B).max())
    sv = np.linalg.svd(A, compute_uv=False)
    assert e >= np.sqrt(np.sum(sv[k:] ** 2)) / np.linalg.norm(sv) * (1 - 1e-12)


def test_exact_rank_recovery():
    m, n, k = 300, 200, 10
    A = ri.exact_rank(m, n, k, seed=31)
    for l in (10, 14):
        r = oracle.factor(A, k, l, 60, seed=41)
        e = oracle.relative_residual(A, r.L, r.U, r.p, r.q)
        assert e < 1e-12, e


def test_k_equals_l_special_case():
    # k = l: no truncation; the path is Algorithm 1 with the exact L_y^+
    A = ri.dense_spectrum(200, 150, ri.geometric_spectrum(150, 8.0), 12)
    r = oracle.factor(A, 12, 12, 96, seed=13)
    e = oracle.relative_residual(A, r.L, r.U, r.p, r.q)
    assert np.isclose(e, projector_error(A, r.Y), rtol=1e-9)


def test_sparse_input_and_residual():
    rowptr, colind, val, m, n = ri.csr_sparse_plus_low_rank(400, 300, 6, 8, 5, seed=21, dtype=np.float64)
    As = ri.csr_to_scipy(rowptr, colind, val, m, n)
    r = oracle.factor(As, 12, 16, 96, seed=22)
    rd = oracle.factor(As.toarray(), 12, 16, 96, seed=22)
    assert np.array_equal(r.p, rd.p) and np.array_equal(r.q, rd.q)
    assert np.allclose(r.L, rd.L, atol=1e-10) and np.allclose(r.U, rd.U, atol=1e-10)
    e_s = oracle.relative_residual(As, r.L, r.U, r.p, r.q)
    e_d = oracle.relative_residual(As.toarray(), r.L, r.U, r.p, r.q)
    assert np.isclose(e_s, e_d, rtol=1e-8)
    assert np.isclose(e_d, projector_error(As, r.Y[:, :12]), rtol=1e-8)


def test_dense_f64_spectrum_closed_form():
    # sigma_i = 10^(-(i-1)/10): Delta_20 / ||A||_F = 10^-2 (1 - q^1004)^(1/2) /
    # (1 - q^1024)^(1/2), q = 10^-0.2, i.e. 0.0100 to 4 digits
    w = ri.DENSE_F64_1K
    A = ri.make_dense(w)
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(sv, ri.geometric_spectrum(1024), rtol=1e-9, atol=1e-14)
    d20 = np.sqrt(np.sum(sv[20:] ** 2)) / np.linalg.norm(sv)
    q = 10 ** -0.2
    assert np.isclose(d20, 1e-2 * math.sqrt((1 - q ** 1004) / (1 - q ** 1024)), rtol=1e-9)


# ---------------------------------------------------------------------------
# Planted mistakes: each must fail a pin
# ---------------------------------------------------------------------------
def _small_case():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((40, 90))
    p = oracle.sketch_params(90, 48, 12, seed=3)
    return A, p


def test_planted_mistakes_fail_the_pins(monkeypatch):
    A, p = _small_case()
    Y1 = oracle.countsketch(A, p, 48)
    ref = fft_route_Y(Y1, p, 48)
    # a dropped sign vector D
    bad = Y1 @ (oracle.hartley_columns(48, p.R) / math.sqrt(48))
    assert not np.allclose(bad, ref, atol=1e-6)
    # sin - cos instead of cos + sin (a transposed Hartley convention)
    b = np.arange(48)[:, None]
    ang = 2 * np.pi * ((b * p.R[None, :]) % 48) / 48
    bad = Y1 @ (p.d[:, None] * (np.cos(ang) - np.sin(ang)) / math.sqrt(48))
    assert not np.allclose(bad, ref, atol=1e-6)
    # a missing 1/sqrt(l1)
    assert not np.allclose(oracle.fjl(Y1, p, 48) * math.sqrt(48), ref, atol=1e-6)
    # the last (not first) maximal row as pivot
    X = np.array([[1.0, 2.0], [-3.0, 1.0], [3.0, 5.0], [2.0, 0.0]])
    _, piv = scipy.linalg.lu_factor(X)
    real_argmax = np.argmax

    def argmax_last(v):
        return len(v) - 1 - int(real_argmax(np.asarray(v)[::-1]))
    monkeypatch.setattr(oracle.rlu.np, "argmax", argmax_last)
    res = oracle.lu_partial_pivot(X)
    monkeypatch.undo()
    assert not np.array_equal(res.perm, ipiv_to_perm(piv, 4))
    # L_y^T in place of L_y^+
    Ly = oracle.unit_lower(oracle.lu_partial_pivot(A[:, :8]).lu, 8)
    assert not np.allclose(Ly.T @ Ly, np.eye(8), atol=1e-6)
    # an off-by-one bucket (h + 1 mod l1)
    p_bad = oracle.SketchParams(h=(p.h + 1) % 48, s=p.s, d=p.d, R=p.R)
    S = np.zeros((90, 48))
    S[np.arange(90), p.h] = p.s
    assert not np.allclose(oracle.countsketch(A, p_bad, 48), A @ S, atol=1e-6)
    # truncation to the last k columns instead of the first
    r = oracle.factor(A, 5, 8, 48, seed=4)
    e = oracle.relative_residual(A, r.L, r.U, r.p, r.q)
    assert not np.isclose(e, projector_error(A, r.Y[:, 3:8]), rtol=1e-6)


def test_planted_word_mapping_mistakes_fail_the_pin(monkeypatch):
    """h from w1 instead of w0, the sign from the wrong word, and a sign test
    shifted by one word value each break test_sketch_params_from_numpy_philox
    or test_word_mapping_boundaries."""
    n, l1, l, seed = 300, 240, 30, 9
    key = [seed, oracle.KEY_TAG]
    b0 = numpy_stream(key, 0, n)
    good_h = [(int(w) * l1) >> 64 for w in b0[:, 0]]
    good_s = [-1 if int(w) >> 63 else 1 for w in b0[:, 1]]
    real = oracle.rlu.stream_blocks

    def swapped(key_, stream, count):  # words 0 and 1 exchanged
        b = real(key_, stream, count).copy()
        b[:, [0, 1]] = b[:, [1, 0]]
        return b
    monkeypatch.setattr(oracle.rlu, "stream_blocks", swapped)
    p = oracle.sketch_params(n, l1, l, seed)
    monkeypatch.undo()
    assert [int(x) for x in p.h] != good_h and [int(x) for x in p.s] != good_s
    # a strict '>' in the sign test moves the word 2^63 to the wrong side
    monkeypatch.setattr(oracle.rlu, "sign_of_word", lambda w: -1.0 if int(w) > 2 ** 63 else 1.0)
    assert oracle.rlu.sign_of_word(2**63) != -1.0
    monkeypatch.undo()
