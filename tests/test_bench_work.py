"""The algorithmic work behind bench.py's roofline `achieved` figures (CPU).

The panel LU count is checked against the operations a plain l-step partial
pivoted LU (Algorithm 1, step 3) actually performs on a small matrix, counted
one by one; the dense and CSR B = W A counts against their definitions, and the
sketch's bytes against one read of A.
"""
import numpy as np
import pytest

import bench
import rlu_inputs as ri


def counted_panel_lu_flops(m, l, seed=0):
    """Run an l-step partial-pivoted LU of a random m x l matrix and count its
    floating-point operations: one division per entry below the pivot, and a
    multiply and a subtract per entry of the trailing block."""
    X = np.random.default_rng(seed).standard_normal((m, l))
    flops = 0
    for j in range(l):
        p = j + int(np.argmax(np.abs(X[j:, j])))
        X[[j, p]] = X[[p, j]]
        for i in range(j + 1, m):
            X[i, j] /= X[j, j]
            flops += 1
            for c in range(j + 1, l):
                X[i, c] -= X[i, j] * X[j, c]
                flops += 2
    return flops


@pytest.mark.parametrize("m,l", [(7, 4), (12, 12), (30, 9), (5, 1)])
def test_panel_lu_count_matches_the_algorithm(m, l):
    assert bench.algorithmic_flops_panel_lu(m, l) == counted_panel_lu_flops(m, l)


def test_dense_fp32_workload_figures():
    w = ri.DENSE_F32_8K
    a_bytes = 4 * w.m * w.n
    works = bench.stage_work("dense", w, a_bytes, w.m * w.n, "f32")
    assert works["sketch"] == (a_bytes, "bytes", "hbm")
    # the panel LU of Y: about 3.9e8 FP64 flop at m = 8192, l = 220
    assert works["panel_lu"][0] == pytest.approx(3.929e8, rel=1e-3)
    assert works["panel_lu"][1:] == ("fp64_flops", "alu")
    assert works["bgemm"] == (2.0 * w.k * w.m * w.n, "flops", "tensor")


def test_fp64_and_csr_products():
    w = ri.DENSE_F64_1K
    works = bench.stage_work("dense", w, 8 * w.m * w.n, w.m * w.n, "f64")
    assert works["bgemm"] == (2.0 * w.k * w.m * w.n, "fp64_flops", "alu")
    c = ri.CSR_F32_200K
    nnz = 12345
    works = bench.stage_work("csr", c, 8 * nnz, nnz, "f32")
    assert works["bgemm"][0] == 2.0 * c.k * nnz
