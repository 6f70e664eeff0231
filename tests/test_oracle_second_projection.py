"""Pins of the oracle's second projection (Algorithm 1, steps 4-6).

Checked against what the paper and the mathematics fix, not against a retyped
copy: an explicit dense Omega_2 built entry by entry from the drawn hash,
signs and frequencies (and applied to P A and L_1 in P order, the literal
statement of step 5); exact recovery of exactly rank-k inputs; and the
deterministic bound in the proof of the correctness theorem,
||L_1 Z^+ Omega_2 P A - P A|| <= (||L_1 (Omega_2 L_1)^+ Omega_2||_2 + 1)
||P A - L_1 L_1^+ P A||, together with the optimality of the exact projection.
"""
import numpy as np
import pytest

import oracle
import rlu_inputs as ri


def dense_omega(m, params2, l2, k2):
    """Omega_2 (k2 x m) as a dense matrix, entry by entry: row f of the
    subsampled, signed Hartley transform of the CountSketch of unit vectors."""
    Om = np.zeros((k2, m))
    for i in range(m):
        b = params2.h[i]
        for r, f in enumerate(params2.R):
            ang = 2.0 * np.pi * ((b * f) % l2) / l2
            Om[r, i] = params2.s[i] * params2.d[b] * (np.cos(ang) + np.sin(ang)) / np.sqrt(l2)
    return Om


def test_second_projection_matches_dense_operator_in_p_order():
    m, n, k, l, l1, k2, l2 = 120, 90, 6, 9, 40, 24, 64
    A = ri.dense_low_rank_plus_noise(m, n, 8, 1e-3, seed=3, dtype=np.float64)
    o = oracle.factor_two_sketch(A, k, l, l1, k2, l2, seed=11, seed2=12)
    params2 = oracle.sketch_params(m, l2, k2, 12)
    Om_orig = dense_omega(m, params2, l2, k2)      # acts on A's original rows
    P = np.eye(m)[o.p]                              # (P A)[t] = A[p[t]]
    Om = Om_orig @ P.T                              # the same SEM law, acting on P A
    Z = Om @ o.Ly                                   # step 5, literally
    Y2 = Om @ (P @ A)
    B = np.linalg.pinv(Z) @ Y2                      # SVD pseudo-inverse
    assert np.allclose(o.Z, Z, rtol=0, atol=1e-12 * np.abs(Z).max())
    assert np.allclose(o.Y2, Y2, rtol=0, atol=1e-12 * np.abs(Y2).max())
    assert np.allclose(o.B, B, rtol=0, atol=1e-10 * np.abs(B).max())


def test_exact_rank_recovery_with_second_projection():
    m, n, k = 300, 200, 10
    A = ri.exact_rank(m, n, k, seed=21)
    o = oracle.factor_two_sketch(A, k, 14, 80, 40, 160, seed=5, seed2=6)
    e = oracle.relative_residual(A, o.L, o.U, o.p, o.q)
    assert e < 1e-12


@pytest.mark.parametrize("seed2", [1, 2, 3])
def test_error_between_exact_projection_and_proof_bound(seed2):
    m, n, k, l, l1, k2, l2 = 400, 300, 12, 18, 120, 36, 144
    A = ri.dense_spectrum(m, n, ri.geometric_spectrum(min(m, n)), 31)
    ex = oracle.factor(A, k, l, l1, seed=8)
    tw = oracle.factor_two_sketch(A, k, l, l1, k2, l2, seed=8, seed2=seed2)
    assert np.array_equal(ex.p, tw.p)              # steps 1-3 are shared
    e_ex = oracle.relative_residual(A, ex.L, ex.U, ex.p, ex.q)
    e_tw = oracle.relative_residual(A, tw.L, tw.U, tw.p, tw.q)
    params2 = oracle.sketch_params(m, l2, k2, seed2)
    Om = dense_omega(m, params2, l2, k2) @ np.eye(m)[tw.p].T
    c = np.linalg.norm(tw.Ly @ np.linalg.pinv(Om @ tw.Ly) @ Om, 2)
    assert e_ex <= e_tw * (1 + 1e-12)              # the exact projection is optimal in range(L_1)
    assert e_tw <= (c + 1) * e_ex * (1 + 1e-9)     # proof of the correctness theorem


def test_planted_row_order_mistake_is_caught():
    # sketching L_1 in P order against A in original order breaks step 5
    m, n, k, l, l1, k2, l2 = 120, 90, 6, 9, 40, 24, 64
    A = ri.dense_low_rank_plus_noise(m, n, 8, 1e-3, seed=3, dtype=np.float64)
    o = oracle.factor_two_sketch(A, k, l, l1, k2, l2, seed=11, seed2=12)
    params2 = oracle.sketch_params(m, l2, k2, 12)
    wrong = oracle.second_projection(o.Ly, params2, l2)   # rows in P order: the mistake
    assert not np.allclose(wrong, o.Z, rtol=0, atol=1e-6 * np.abs(o.Z).max())
