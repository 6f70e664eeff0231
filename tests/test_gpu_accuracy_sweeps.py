"""Accuracy sweeps in the shape of the paper's experiments (Sec. 4): 5000 x 5000
matrices with prescribed singular values, factored at increasing rank k.

  rank growth:   sigma_i = 1 for i <= r, then exponentially decaying from
                 e^-10 to e^-200 (Sec. 4.1), factored at k = r;
  fixed matrix:  sigma_i decaying exponentially from 1 to e^-100 (Sec. 4.2),
                 factored at increasing k.

No values are printed in the paper (its figures are absent), so the checks are
the mathematics: the error is never below the best rank-k error Delta_k
(Eckart-Young), and the first point of each sweep equals the FP64 oracle's.
The correctness theorem bounds the error by O(Delta_k) with unstated constants;
the measured ratios e / Delta_k (printed with pytest -s, recorded in the design
notes) grow about like sqrt(k): with L_y the first k columns of an l-step LU,
the oversampling l - k does not enter the projection.
"""
import numpy as np
import pytest

import oracle
import rlu_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 5000


def tail_ratio(sigma, k):
    return float(np.sqrt(np.sum(sigma[k:] ** 2) / np.sum(sigma ** 2)))


def step_spectrum(r):
    s = np.exp(-np.linspace(10.0, 200.0, N - r))
    return np.concatenate([np.ones(r), s])


def exp_spectrum():
    return np.exp(-100.0 * np.arange(N) / (N - 1))


@pytest.fixture(scope="module")
def rg():
    import paper_1601_04280_gb300 as rg
    rg.build()
    rg.load(reload=True)
    return rg


@pytest.fixture(scope="module")
def factors():
    rng = np.random.Generator(np.random.PCG64(5000))
    X = ri.orthonormal(N, N, rng)
    Yf = ri.orthonormal(N, N, rng)
    return X, Yf


def widths(k):
    # l1 = 8 k, at most 6000 (the FP64 sketch keeps two l1-point transforms in shared memory)
    return k + 20, min(8 * k, 6000)


def run(rg, A, k, seed):
    l, l1 = widths(k)
    h = rg.RandLU(N, N, k, l, l1, seed, prec="f64")
    f = h.factor(torch.from_numpy(A).cuda(), check=False)
    torch.cuda.synchronize()
    out = (f.L.cpu().numpy(), f.U.cpu().numpy(), f.p.cpu().numpy(), f.q.cpu().numpy(), f.status)
    h.close()
    return out


def test_rank_growth_step_spectrum(rg, factors):
    X, Yf = factors
    print()
    for r in (50, 100, 200, 400, 900):
        sigma = step_spectrum(r)
        A = (X * sigma) @ Yf.T
        L, U, p, q, st = run(rg, A, r, 3000 + r)
        assert st in (0, 100)
        e = oracle.relative_residual(A, L, U, p, q)
        d = tail_ratio(sigma, r)
        print("rank growth r=%4d  e=%.3e  Delta_r/||A||=%.3e  ratio=%.2f" % (r, e, d, e / d))
        assert e >= d * (1 - 1e-6)
        if r == 50:
            o = oracle.factor(A, r, *widths(r), 3000 + r)
            e_o = oracle.relative_residual(A, o.L, o.U, o.p, o.q)
            assert abs(e - e_o) <= 1e-12 + 1e-9 * e_o, (e, e_o)


def test_fixed_matrix_increasing_rank(rg, factors):
    X, Yf = factors
    sigma = exp_spectrum()
    A = (X * sigma) @ Yf.T
    print()
    for k in (50, 100, 200, 400, 800):
        L, U, p, q, st = run(rg, A, k, 4000 + k)
        assert st in (0, 100)
        e = oracle.relative_residual(A, L, U, p, q)
        d = tail_ratio(sigma, k)
        print("fixed matrix   k=%4d  e=%.3e  Delta_k/||A||=%.3e  ratio=%.2f" % (k, e, d, e / d))
        assert e >= d * (1 - 1e-6)
        if k == 50:
            o = oracle.factor(A, k, *widths(k), 4000 + k)
            e_o = oracle.relative_residual(A, o.L, o.U, o.p, o.q)
            assert abs(e - e_o) <= 1e-12 + 1e-9 * e_o, (e, e_o)
