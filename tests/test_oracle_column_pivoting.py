"""Pins of the oracle's rank-revealing column order of the sketch: QR with
column pivoting (Businger and Golub) written as a greedy pivoted Cholesky of
Y^T Y.  Checked against LAPACK's geqp3 (scipy), a brute-force greedy that
projects explicitly, the closed form of Corollary 3.3 with the reordered
sketch, and its effect on the error (the oversampling now counts)."""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
import rlu_inputs as ri


def brute_force_order(Y):
    """At each step the column of largest norm after an explicit orthogonal
    projection away from the columns already chosen (first index on ties)."""
    l = Y.shape[1]
    chosen, Q = [], np.zeros((Y.shape[0], 0))
    for _ in range(l):
        R = Y - Q @ (Q.T @ Y)
        norms = np.linalg.norm(R, axis=0)
        norms[chosen] = -1.0
        c = int(np.argmax(norms))
        chosen.append(c)
        q = R[:, c] / np.linalg.norm(R[:, c])
        Q = np.column_stack([Q, q])
    return np.array(chosen)


@pytest.mark.parametrize("m,l,seed", [(200, 12, 1), (500, 40, 2), (64, 30, 3)])
def test_order_matches_lapack_geqp3(m, l, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((m, l)) * np.exp(rng.uniform(-3, 3, l))[None, :]
    _, _, piv = scipy.linalg.qr(Y, mode="economic", pivoting=True)
    assert np.array_equal(oracle.column_order_greedy(Y), piv)


def test_order_matches_brute_force():
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((50, 9)) @ np.diag([1, 5, 0.1, 3, 2, 7, 0.5, 4, 1.5])
    assert np.array_equal(oracle.column_order_greedy(Y), brute_force_order(Y))


def test_rank_deficient_sketch_gives_a_permutation():
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((40, 3)) @ rng.standard_normal((3, 8))
    order = oracle.column_order_greedy(Y)
    assert np.array_equal(np.sort(order), np.arange(8))
    # the first three columns already span the sketch
    Q, _ = np.linalg.qr(Y[:, order[:3]])
    assert np.linalg.norm(Y - Q @ (Q.T @ Y)) <= 1e-12 * np.linalg.norm(Y)


def projector_error(A, Yk):
    Q, _ = np.linalg.qr(Yk)
    return float(np.linalg.norm(A - Q @ (Q.T @ A)) / np.linalg.norm(A))


def test_column_pivoted_factor_closed_form_and_recovery():
    m, n, k, l, l1 = 400, 350, 15, 24, 192
    A = ri.dense_spectrum(m, n, ri.geometric_spectrum(min(m, n)), 8)
    r = oracle.factor(A, k, l, l1, seed=3, column_pivoting=True)
    assert np.array_equal(np.sort(r.ycols), np.arange(l))
    e = oracle.relative_residual(A, r.L, r.U, r.p, r.q)
    assert np.isclose(e, projector_error(A, r.Y[:, :k]), rtol=1e-9)
    sv = np.linalg.svd(A, compute_uv=False)
    assert e >= math.sqrt(np.sum(sv[k:] ** 2)) / np.linalg.norm(A) * (1 - 1e-12)
    Ax = ri.exact_rank(m, n, k, seed=9)
    rx = oracle.factor(Ax, k, l, l1, seed=3, column_pivoting=True)
    assert oracle.relative_residual(Ax, rx.L, rx.U, rx.p, rx.q) < 1e-12


def test_column_pivoting_lets_the_oversampling_count():
    """A step spectrum (200 singular values 1, then e^-10 decaying to e^-200)
    at k = 200, l = 220: the first k sketch columns leave e/Delta_k far above
    the column-pivoted choice (51.9 against 6.9 at 1500 x 1500; here 1000 x
    1000)."""
    m = n = 1000
    sig = np.concatenate([np.ones(200), np.exp(-10 - np.arange(m - 200) * 190.0 / m)])
    A = ri.dense_spectrum(m, n, sig, 5)
    k, l, l1 = 200, 220, 1600
    sv = np.linalg.svd(A, compute_uv=False)
    dk = math.sqrt(np.sum(sv[k:] ** 2)) / np.linalg.norm(A)
    e = {}
    for cp in (False, True):
        r = oracle.factor(A, k, l, l1, seed=2200, column_pivoting=cp)
        e[cp] = oracle.relative_residual(A, r.L, r.U, r.p, r.q)
    print("e / Delta_k: first k columns %.2f, column-pivoted %.2f" % (e[False] / dk, e[True] / dk))
    assert e[True] < 0.5 * e[False]


def test_planted_order_mistakes_fail():
    """Ordering by the initial column norms only (no downdating) and taking the
    last maximum both disagree with geqp3 on a designed sketch."""
    Y = np.array([[3.0, 2.9, 0.0], [0.0, 0.1, 2.0], [0.0, 0.0, 0.5]])
    _, _, piv = scipy.linalg.qr(Y, pivoting=True)
    assert np.array_equal(oracle.column_order_greedy(Y), piv)
    by_norm = np.argsort(-np.linalg.norm(Y, axis=0), kind="stable")
    assert not np.array_equal(by_norm, piv)
    Yt = np.array([[1.0, 1.0], [0.0, 0.0]])
    assert oracle.column_order_greedy(Yt)[0] == 0  # tie: the first index
