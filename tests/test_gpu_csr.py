"""CSR input: parity of the CUDA path with the FP64 oracle (scipy.sparse A).

Tolerances as in test_gpu_parity: FP32 |e_gpu - e_oracle| <= 1e-5, FP64 <= 1e-12;
pivots equal on the separated prefix; L, U and B entry by entry wherever the
GPU chose the oracle's pivots (parity_tools).  Rows with >= n/4 entries take
the dense (heavy) route, the others the sparse route; both are exercised.
"""
import numpy as np
import pytest
import scipy.sparse

import oracle
import parity_tools as pt
import rlu_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import check_pivots, check_structure, separated_prefix  # noqa: E402


@pytest.fixture(scope="module")
def rg():
    import paper_1601_04280_gb300 as rg
    rg.build()
    rg.load(reload=True)
    return rg


def run_csr(rg, As, k, l, l1, seed, prec, debug=False):
    As = As.tocsr()
    m, n = As.shape
    vdt = torch.float64 if prec == "f64" else torch.float32
    h = rg.RandLU(m, n, k, l, l1, seed, prec=prec)
    if debug:
        h.debug_enable(True)
    rowptr = torch.from_numpy(As.indptr.astype(np.int64)).cuda()
    colind = torch.from_numpy(As.indices.astype(np.int32)).cuda()
    val = torch.from_numpy(As.data).to(vdt).cuda()
    f = h.factor_csr(rowptr, colind, val, check=False)
    torch.cuda.synchronize()
    out = dict(L=f.L.double().cpu().numpy(), U=f.U.double().cpu().numpy(), p=f.p.cpu().numpy(),
               q=f.q.cpu().numpy(), status=f.status, handle=h)
    if debug:
        out["Y"] = h.debug_Y()
        out["B"] = h.debug_B()
    return out


def sparse_case(m, n, npr, heavy, rank, seed, dtype):
    rowptr, colind, val, m, n = ri.csr_sparse_plus_low_rank(m, n, npr, heavy, rank, seed, dtype=dtype)
    return ri.csr_to_scipy(rowptr, colind, val, m, n)


@pytest.mark.parametrize("m,n,npr,heavy,k,l,l1", [(3000, 2000, 12, 40, 30, 40, 320),   # light + heavy rows
                                                   (1500, 900, 9, 0, 20, 28, 240),     # light rows only
                                                   (300, 700, 5, 300, 16, 24, 128)])   # heavy rows only
def test_csr_f32_parity(rg, m, n, npr, heavy, k, l, l1):
    As = sparse_case(m, n, npr, heavy, 6, seed=m + heavy, dtype=np.float32)
    o = oracle.factor(As, k, l, l1, seed=5)
    g = run_csr(rg, As, k, l, l1, 5, "f32", debug=True)
    assert g["status"] == 0, rg.strerror(g["status"])
    check_structure(g, m, n, k)
    check_pivots(g, o, k)
    rown = np.sqrt(np.asarray(As.multiply(As).sum(axis=1)).ravel().max())
    assert np.abs(g["Y"] - o.Y).max() <= 5e-6 * rown
    e_o = oracle.relative_residual(As, o.L, o.U, o.p, o.q)
    e_g = oracle.relative_residual(As, g["L"], g["U"], g["p"], g["q"])
    assert abs(e_g - e_o) <= 1e-5, (e_g, e_o)
    if e_o >= 1e-4:
        assert abs(e_g / e_o - 1) <= 1e-2
    tau = pt.tolerances(As, o, k, l, "f32")
    done = pt.check_elementwise(g, o, k, tau, g["B"])
    print("csr %dx%d k=%d: tau %s, max rel. differences %s" % (m, n, k, tau, done))
    if separated_prefix(o.top_y, np.abs(o.Y).max(), 1e-4) >= k:
        assert "B" in done


def test_csr_f32_c2_shape(rg):
    """The sparse workload's code paths at a reduced height: 40 uniform
    columns per row, a dense rank-50 block on 2 % of the rows (160 rows of
    50000 entries: heavy rows, densified and sketched by the column-chunk
    kernel through the row map, their B on the tensor cores), k = 100,
    l = 120, l1 = 960."""
    m, n, k, l, l1 = 8000, 50000, 100, 120, 960
    As = sparse_case(m, n, 40, m // 50, 50, seed=77, dtype=np.float32)
    o = oracle.factor(As, k, l, l1, seed=97)
    g = run_csr(rg, As, k, l, l1, 97, "f32", debug=True)
    assert g["status"] == 0, rg.strerror(g["status"])
    check_structure(g, m, n, k)
    check_pivots(g, o, k)
    rown = np.sqrt(np.asarray(As.multiply(As).sum(axis=1)).ravel().max())
    assert np.abs(g["Y"] - o.Y).max() <= 5e-6 * rown
    e_o = oracle.relative_residual(As, o.L, o.U, o.p, o.q)
    e_g = oracle.relative_residual(As, g["L"], g["U"], g["p"], g["q"])
    assert abs(e_g - e_o) <= 1e-5, (e_g, e_o)
    if e_o >= 1e-4:
        assert abs(e_g / e_o - 1) <= 1e-2
    tau = pt.tolerances(As, o, k, l, "f32", draws=1)
    done = pt.check_elementwise(g, o, k, tau, g["B"])
    print("csr c2 shape: e_gpu %.4e e_oracle %.4e; tau %s; max rel. differences %s" % (e_g, e_o, tau, done))


def test_csr_f32_row_classes(rg):
    """Every route of the CSR sketch in one matrix: rows of 8 entries (direct
    evaluation against the projection's table), rows of 600 entries (more
    than the direct bound 4 l1 (log2 l1 + 1) / l = 288 for l1 = 320, l = 40,
    below n/4: the bucket sums and FFT), rows of 1200 entries (>= n/4:
    densified).  Same bars as test_csr_f32_parity."""
    rng = np.random.default_rng(21)
    m, n, k, l, l1 = 2000, 4000, 30, 40, 320
    counts = np.where(np.arange(m) % 10 == 3, 600, np.where(np.arange(m) % 50 == 7, 1200, 8))
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    cols = np.concatenate([np.sort(rng.choice(n, size=c, replace=False)) for c in counts]).astype(np.int32)
    U = rng.standard_normal((m, 8))
    V = rng.standard_normal((8, n))
    rows = np.repeat(np.arange(m), counts)
    vals = (np.einsum("ij,ji->i", U[rows], V[:, cols]) + 0.01 * rng.standard_normal(len(cols))).astype(np.float32)
    As = scipy.sparse.csr_matrix((vals, cols, indptr), shape=(m, n))
    o = oracle.factor(As, k, l, l1, seed=8)
    g = run_csr(rg, As, k, l, l1, 8, "f32", debug=True)
    assert g["status"] == 0, rg.strerror(g["status"])
    check_structure(g, m, n, k)
    check_pivots(g, o, k)
    rown = np.sqrt(np.asarray(As.multiply(As).sum(axis=1)).ravel())
    # row by row against the row's own norm: each route is checked on its rows
    assert np.all(np.abs(g["Y"] - o.Y).max(axis=1) <= 5e-6 * rown + 1e-30)
    e_o = oracle.relative_residual(As, o.L, o.U, o.p, o.q)
    e_g = oracle.relative_residual(As, g["L"], g["U"], g["p"], g["q"])
    assert abs(e_g - e_o) <= 1e-5, (e_g, e_o)
    if e_o >= 1e-4:
        assert abs(e_g / e_o - 1) <= 1e-2


def test_csr_f64_parity(rg):
    As = sparse_case(2000, 1500, 10, 30, 5, seed=9, dtype=np.float64)
    o = oracle.factor(As, 25, 32, 256, seed=6)
    g = run_csr(rg, As, 25, 32, 256, 6, "f64", debug=True)
    assert g["status"] == 0
    check_pivots(g, o, 25)
    assert np.abs(g["Y"] - o.Y).max() <= 1e-12 * np.abs(o.Y).max()
    assert np.abs(g["B"] - o.B).max() <= 1e-9 * np.abs(o.B).max()
    e_o = oracle.relative_residual(As, o.L, o.U, o.p, o.q)
    e_g = oracle.relative_residual(As, g["L"], g["U"], g["p"], g["q"])
    assert abs(e_g - e_o) <= 1e-12, (e_g, e_o)


def test_csr_unsorted_and_duplicate_entries(rg):
    # columns in random order within each row and repeated coordinates (summed), in light and heavy rows
    rng = np.random.default_rng(11)
    m, n = 800, 600
    rows, cols, vals = [], [], []
    for i in range(m):
        cnt = 400 if i % 97 == 0 else 8
        c = rng.integers(0, n, size=cnt)
        if i % 5 == 0:
            c[1] = c[0]  # a duplicate
        rows += [i] * cnt
        cols += list(c)
        vals += list(rng.standard_normal(cnt))
    coo = scipy.sparse.coo_matrix((np.array(vals), (np.array(rows), np.array(cols))), shape=(m, n))
    csr = coo.tocsr()
    csr.has_sorted_indices = False
    # rebuild with the original (unsorted, duplicated) entry order per row
    order = np.lexsort((np.arange(len(rows)), np.array(rows)))
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(np.array(rows), minlength=m), out=indptr[1:])
    As = scipy.sparse.csr_matrix((np.array(vals)[order], np.array(cols)[order], indptr), shape=(m, n))
    o = oracle.factor(As, 20, 26, 200, seed=3)
    g = run_csr(rg, As, 20, 26, 200, 3, "f64")
    assert g["status"] == 0
    e_o = oracle.relative_residual(As, o.L, o.U, o.p, o.q)
    e_g = oracle.relative_residual(As, g["L"], g["U"], g["p"], g["q"])
    assert abs(e_g - e_o) <= 1e-12, (e_g, e_o)


def test_csr_equals_dense_factorization(rg):
    As = sparse_case(1200, 800, 10, 20, 4, seed=2, dtype=np.float64)
    g = run_csr(rg, As, 16, 22, 176, 8, "f64")
    h = rg.RandLU(1200, 800, 16, 22, 176, 8, prec="f64")
    f = h.factor(torch.from_numpy(As.toarray()).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(g["p"], f.p.cpu().numpy()) and np.array_equal(g["q"], f.q.cpu().numpy())
    assert np.allclose(g["L"], f.L.cpu().numpy(), rtol=0, atol=1e-9 * np.abs(g["L"]).max())
    assert np.allclose(g["U"], f.U.cpu().numpy(), rtol=0, atol=1e-9)


def test_csr_invalid_structure_reported(rg):
    As = sparse_case(200, 150, 6, 0, 3, seed=4, dtype=np.float32).tocsr()
    h = rg.RandLU(200, 150, 8, 12, 64, 1, prec="f32")
    rowptr = As.indptr.astype(np.int64).copy()
    rowptr[50], rowptr[51] = rowptr[51], rowptr[50] - 1  # non-monotone
    f = h.factor_csr(torch.from_numpy(rowptr).cuda(), torch.from_numpy(As.indices.astype(np.int32)).cuda(),
                     torch.from_numpy(As.data.astype(np.float32)).cuda(), check=False)
    assert f.status == rg.RLU_EBADCSR
    colind = As.indices.astype(np.int32).copy()
    colind[17] = 150  # out of range
    f = h.factor_csr(torch.from_numpy(As.indptr.astype(np.int64)).cuda(), torch.from_numpy(colind).cuda(),
                     torch.from_numpy(As.data.astype(np.float32)).cuda(), check=False)
    assert f.status == rg.RLU_EBADCSR


def test_csr_deterministic_bitwise(rg):
    As = sparse_case(2500, 1800, 10, 25, 5, seed=13, dtype=np.float32)
    a = run_csr(rg, As, 24, 32, 256, 9, "f32")
    b = run_csr(rg, As, 24, 32, 256, 9, "f32")
    for key in ("L", "U", "p", "q"):
        assert np.array_equal(a[key], b[key]), key
