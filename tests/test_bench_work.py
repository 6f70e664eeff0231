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


def counted_blocked_panel_flops(m, l, b, seed=0):
    """The operations inside the panels of a blocked partial-pivoted LU (panel
    width b), counted one by one: each panel's steps on the rows not yet
    pivoted and the panel's own columns (the trailing updates are counted
    apart)."""
    X = np.random.default_rng(seed).standard_normal((m, l))
    flops = 0
    for j0 in range(0, l, b):
        wid = min(b, l - j0)
        for j in range(j0, j0 + wid):
            p = j + int(np.argmax(np.abs(X[j:, j])))
            X[[j, p]] = X[[p, j]]
            for i in range(j + 1, m):
                X[i, j] /= X[j, j]
                flops += 1
                for c in range(j + 1, j0 + wid):
                    X[i, c] -= X[i, j] * X[j, c]
                    flops += 2
        # trailing update of the columns right of the panel (not counted)
        if j0 + wid < l:
            L11 = np.tril(X[j0:j0 + wid, j0:j0 + wid], -1) + np.eye(wid)
            X[j0:j0 + wid, j0 + wid:] = np.linalg.solve(L11, X[j0:j0 + wid, j0 + wid:])
            X[j0 + wid:, j0 + wid:] -= X[j0 + wid:, j0:j0 + wid] @ X[j0:j0 + wid, j0 + wid:]
    return flops


@pytest.mark.parametrize("m,l,b", [(40, 10, 4), (33, 16, 16), (25, 9, 0), (50, 20, 8)])
def test_panel_launch_count_matches_the_algorithm(m, l, b):
    expect = counted_panel_lu_flops(m, l) if b == 0 else counted_blocked_panel_flops(m, l, b)
    assert bench.algorithmic_flops_lu_panels(m, l, b) == expect
    assert bench.lu_panels(l, b)[-1][0] + bench.lu_panels(l, b)[-1][1] == l


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


def test_reference_arm_json_line():
    """The reference arm (the oracle on the host cores) prints one JSON line
    with the contract's keys, on the small dense FP64 workload."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                          "dense_f64_1024x1024_k20", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"] == "dense_f64_1024x1024_k20"
