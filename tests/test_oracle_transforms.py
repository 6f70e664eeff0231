"""Pins of the oracle's three FFT-based projections of step 2 (Algorithm 1):
the real Hartley transform (the default reading for real data), the
subsampled randomized Hadamard transform the experiments of Sec. 4 used for
real data (SRHT), and the complex SRFT of Sec. 2.1 (Pi = D F S with D of
unit-modulus entries) in real form (real and imaginary parts of l/2 kept
frequencies).  Each is checked against an independent route: scipy's
Sylvester Hadamard matrix, a fast Walsh-Hadamard transform written here,
numpy's complex FFT, and the end-to-end closed form of Corollary 3.3.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
import rlu_inputs as ri


def fwht_rows(X):
    """Walsh-Hadamard transform of every row (length a power of two) by
    butterflies (x, y) -> (x + y, x - y), natural (Sylvester) order."""
    X = np.array(X, dtype=np.float64, copy=True)
    n = X.shape[1]
    h = 1
    while h < n:
        X = X.reshape(X.shape[0], -1, 2, h)
        a = X[:, :, 0, :].copy()
        b = X[:, :, 1, :].copy()
        X[:, :, 0, :] = a + b
        X[:, :, 1, :] = a - b
        X = X.reshape(X.shape[0], n)
        h *= 2
    return X


@pytest.mark.parametrize("l1", [1, 2, 8, 64, 1024])
def test_hadamard_is_sylvester(l1):
    H = oracle.hadamard_columns(l1, np.arange(l1))
    assert np.array_equal(H, scipy.linalg.hadamard(l1).astype(np.float64))
    # symmetric and self-inverse up to l1
    assert np.array_equal(H @ H, l1 * np.eye(l1))


def test_hadamard_needs_power_of_two():
    with pytest.raises(ValueError):
        oracle.hadamard_columns(240, [0, 1])


@pytest.mark.parametrize("m,n,l1,l", [(20, 300, 64, 16), (7, 5000, 1024, 100)])
def test_srht_matches_fast_walsh_hadamard(m, n, l1, l):
    rng = np.random.default_rng(l1)
    A = rng.standard_normal((m, n))
    p = oracle.sketch_params(n, l1, l, seed=31)
    Y1 = oracle.countsketch(A, p, l1)
    Y = oracle.fjl(Y1, p, l1, "srht")
    ref = fwht_rows(Y1 * p.d[None, :])[:, p.R] / math.sqrt(l1)
    assert np.allclose(Y, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # distinct Hadamard columns with +-1 signs: orthonormal columns
    M = oracle.transform_matrix(p, l1, l, "srht")
    assert np.allclose(M.T @ M, np.eye(l), atol=1e-12)


@pytest.mark.parametrize("m,n,l1,l", [(9, 400, 240, 30), (5, 3000, 1600, 220), (4, 100, 7, 6)])
def test_srft_matches_numpy_fft(m, n, l1, l):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((m, n))
    p = oracle.sketch_params(n, l1, l, seed=32)
    Y1 = oracle.countsketch(A, p, l1)
    Y = oracle.fjl(Y1, p, l1, "srft")
    Z = np.fft.fft(Y1 * np.exp(1j * p.theta)[None, :], axis=1)
    f = p.R[: l // 2]
    scale = math.sqrt(2.0 / l1)
    tol = 1e-11 * np.abs(Z).max() * scale
    assert np.allclose(Y[:, 0::2], scale * Z[:, f].real, rtol=0, atol=tol)
    assert np.allclose(Y[:, 1::2], scale * Z[:, f].imag, rtol=0, atol=tol)


def test_srft_with_unit_phases_is_the_dft():
    l1 = 12
    M = oracle.srft_columns(l1, np.zeros(l1), np.arange(l1))
    F = np.fft.fft(np.eye(l1), axis=0)  # F[b, f] = exp(-2 pi i b f / l1)
    assert np.allclose(M[:, 0::2], F.real, atol=1e-14) and np.allclose(M[:, 1::2], F.imag, atol=1e-14)


def test_srft_needs_even_l():
    p = oracle.sketch_params(50, 64, 7, seed=1)
    with pytest.raises(ValueError):
        oracle.transform_matrix(p, 64, 7, "srft")


def test_phases_uniform_and_mapped_exactly():
    assert oracle.phase_of_word(0) == 0.0
    assert oracle.phase_of_word(2**63) == math.pi
    assert 0.0 <= oracle.phase_of_word(2**64 - 1) < 2 * math.pi
    p = oracle.sketch_params(10, 4096, 8, seed=77)
    assert p.theta.min() >= 0.0 and p.theta.max() < 2 * math.pi
    # uniform: the mean of cos and sin of the phases vanish within 6 sigma
    assert abs(np.cos(p.theta).mean()) < 6 / math.sqrt(2 * 4096)
    assert abs(np.sin(p.theta).mean()) < 6 / math.sqrt(2 * 4096)


def projector_error(A, Yk):
    Q, _ = np.linalg.qr(Yk)
    return float(np.linalg.norm(A - Q @ (Q.T @ A)) / np.linalg.norm(A))


@pytest.mark.parametrize("transform,l1", [("hartley", 240), ("srht", 256), ("srft", 240)])
def test_every_transform_end_to_end(transform, l1):
    """Corollary 3.3's closed form ||LU - PAQ|| = ||(I - Pi_{Y[:, :k]}) A||,
    exact recovery of an exactly rank-k input, and e >= Delta_k, for each
    projection."""
    m, n, k, l = 300, 260, 12, 20
    A = ri.dense_spectrum(m, n, ri.geometric_spectrum(min(m, n)), 7)
    r = oracle.factor(A, k, l, l1, seed=9, transform=transform)
    e = oracle.relative_residual(A, r.L, r.U, r.p, r.q)
    assert np.isclose(e, projector_error(A, r.Y[:, :k]), rtol=1e-9)
    sv = np.linalg.svd(A, compute_uv=False)
    assert e >= math.sqrt(np.sum(sv[k:] ** 2)) / np.linalg.norm(A) * (1 - 1e-12)
    Ax = ri.exact_rank(m, n, k, seed=4)
    rx = oracle.factor(Ax, k, l, l1, seed=9, transform=transform)
    assert oracle.relative_residual(Ax, rx.L, rx.U, rx.p, rx.q) < 1e-12


def test_planted_transform_mistakes_fail_the_pins():
    """A conjugated DFT, a lost sqrt(2) and +-1 signs applied on top of the
    complex phases each break the numpy FFT pin; sequency (Walsh) order breaks
    the Sylvester pin."""
    l1, l, n = 240, 30, 400
    p = oracle.sketch_params(n, l1, l, seed=32)
    A = np.random.default_rng(3).standard_normal((6, n))
    Y1 = oracle.countsketch(A, p, l1)
    Z = np.fft.fft(Y1 * np.exp(1j * p.theta)[None, :], axis=1)[:, p.R[: l // 2]] * math.sqrt(2.0 / l1)
    good = np.empty((6, l))
    good[:, 0::2], good[:, 1::2] = Z.real, Z.imag
    assert np.allclose(oracle.fjl(Y1, p, l1, "srft"), good, atol=1e-10)
    conj = good.copy()
    conj[:, 1::2] *= -1
    assert not np.allclose(oracle.fjl(Y1, p, l1, "srft"), conj, atol=1e-6)
    assert not np.allclose(good / math.sqrt(2.0), oracle.fjl(Y1, p, l1, "srft"), atol=1e-6)
    signed = Y1 * p.d[None, :]
    assert not np.allclose(oracle.fjl(signed, p, l1, "srft"), good, atol=1e-6)
    # Walsh (sequency) order: rows sorted by their number of sign changes
    H = oracle.hadamard_columns(16, np.arange(16))
    walsh = H[np.argsort([np.count_nonzero(np.diff(r)) for r in H])]
    assert not np.array_equal(walsh, scipy.linalg.hadamard(16))


def test_transform_errors_side_by_side():
    """The three projections on the dense FP64 workload (1024 x 1024,
    sigma_i = 10^(-(i-1)/10), k = 20, l = 30; l1 = 240, or 256 for the
    Walsh-Hadamard transform), five sketch seeds each: e / (Delta_k/||A||)
    for each.  All three are O(Delta_k) (Corollary 3.3) and within a small
    factor of one another; printed for the record."""
    w = ri.DENSE_F64_1K
    A = ri.make_dense(w)
    sv = np.linalg.svd(A, compute_uv=False)
    dk = math.sqrt(np.sum(sv[w.k:] ** 2)) / np.linalg.norm(A)
    ratios = {}
    for transform, l1 in (("hartley", 240), ("srht", 256), ("srft", 240)):
        es = []
        for seed in range(2000, 2005):
            r = oracle.factor(A, w.k, w.l, l1, seed, transform=transform)
            es.append(oracle.relative_residual(A, r.L, r.U, r.p, r.q))
        ratios[transform] = float(np.mean(es) / dk)
        assert min(es) >= dk * (1 - 1e-12)
    print("e / Delta_k, mean of 5 seeds:", {t: round(v, 2) for t, v in ratios.items()})
    assert max(ratios.values()) < 10 and max(ratios.values()) / min(ratios.values()) < 2
