"""The blocked LU of the sketch (step 3 of Algorithm 1: panels on the FP64
pipe, trailing updates as exact digit products on the tensor cores) against
the oracle's getf2 on the GPU's own sketch Y, entry by entry, and against the
unblocked kernel on the same input.

Bars: both sides compute in FP64 (the trailing products carry 56-bit digits,
so each update is within a few units of 2^-53 of the operands' scales); over
l steps the entries of L_Y and U_Y then differ by at most about
l * 2^-53 * growth ~ 1e-13 of their largest magnitude, and the bar is 1e-11
of it.  A dropped or misplaced update, a wrong digit or scale, or a wrong
row shows up as an O(1) difference.  Pivots: equal on every step whose two
best candidates differ by more than 1e-9 of the largest entry of Y."""
import numpy as np
import pytest

import oracle
import rlu_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import check_pivots, check_structure, run, separated_prefix  # noqa: E402


@pytest.fixture(scope="module")
def rg():
    import paper_1601_04280_gb300 as rg
    rg.build()
    rg.load(reload=True)
    return rg


def factor_lu(rg, A, k, l, l1, seed, block, prec="f64"):
    m, n = A.shape
    h = rg.RandLU(m, n, k, l, l1, seed, prec=prec)
    h.set_lu_block(block)
    h.debug_enable(True)
    dt = torch.float64 if prec == "f64" else torch.float32
    f = h.factor(torch.from_numpy(np.ascontiguousarray(A)).to("cuda", dt), check=False)
    torch.cuda.synchronize()
    Y0 = h.debug_Y()
    Ylu, perm = h.debug_lu_Y()
    out = dict(status=f.status, Y=Y0, lu=Ylu, perm=perm, L=f.L.double().cpu().numpy(),
               U=f.U.double().cpu().numpy(), p=f.p.cpu().numpy(), q=f.q.cpu().numpy())
    h.close()
    return out


def compare_with_getf2(g, l):
    o = oracle.lu_partial_pivot(g["Y"], steps=l)
    scale = np.abs(g["Y"]).max()
    sp = separated_prefix(o.top, scale, 1e-9)
    assert np.array_equal(g["perm"][:sp], o.perm[:sp]), "pivots differ before step %d" % sp
    assert sp == l, "inputs chosen with well-separated pivots: %d of %d" % (sp, l)
    lu_pos = g["lu"][g["perm"]]  # rows in pivot order, as the oracle keeps them
    d = np.abs(lu_pos - o.lu).max()
    assert d <= 1e-11 * np.abs(o.lu).max(), d
    return d


@pytest.mark.parametrize("m,n,l,block", [
    (20000, 300, 120, 16),   # 8 panels, the last one 8 wide
    (6000, 500, 200, 32),    # 7 panels, ragged last panel
    (3000, 600, 260, 64),    # 5 panels
    (20000, 400, 130, 0),    # automatic width (64: panels 64, 64, 2); a ragged last row tile
    (200000, 200, 48, 16),   # 1316 rows per CTA in 16-wide panels, as in the 200000-row sparse workload
])
def test_blocked_lu_matches_getf2(rg, m, n, l, block):
    A = ri.dense_low_rank_plus_noise(m, n, min(n, 2 * l), 1e-2, seed=m + l, dtype=np.float64)
    g = factor_lu(rg, A, l - 10, l, 8 * l, 71, block)
    assert g["status"] == 0
    d = compare_with_getf2(g, l)
    print("m=%d l=%d block=%d: max |LU_gpu - LU_getf2| = %.2e" % (m, l, block, d))


def test_blocked_equals_unblocked(rg):
    m, n, l = 12000, 400, 160
    A = ri.dense_low_rank_plus_noise(m, n, 320, 1e-3, seed=5, dtype=np.float64)
    u = factor_lu(rg, A, 150, l, 1280, 9, -1)
    b = factor_lu(rg, A, 150, l, 1280, 9, 32)
    assert np.array_equal(u["Y"], b["Y"])  # same sketch
    assert np.array_equal(u["perm"], b["perm"])
    assert np.abs(u["lu"] - b["lu"]).max() <= 1e-11 * np.abs(u["lu"]).max()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_blocked_factor_parity(rg, prec):
    """The whole factorization with the blocked LU against the oracle (the
    bars of test_gpu_parity: FP64 |de| <= 1e-12, FP32 |de| <= 1e-5)."""
    m, n, k, l, l1 = 20000, 2000, 100, 120, 960
    A = ri.dense_low_rank_plus_noise(m, n, 110, 1e-5, seed=77, dtype=np.float64)
    Ain = A if prec == "f64" else A.astype(np.float32)
    o = oracle.factor(Ain.astype(np.float64), k, l, l1, seed=13)
    g = run(rg, Ain, k, l, l1, 13, prec, torch.float64 if prec == "f64" else torch.float32)
    assert g["status"] == 0
    check_structure(g, m, n, k)
    check_pivots(g, o, k)
    e_o = oracle.relative_residual(Ain.astype(np.float64), o.L, o.U, o.p, o.q)
    e_g = oracle.relative_residual(Ain.astype(np.float64), g["L"], g["U"], g["p"], g["q"])
    assert abs(e_g - e_o) <= (1e-12 if prec == "f64" else 1e-5), (e_g, e_o)


def test_lu_block_validation(rg):
    h = rg.RandLU(5000, 800, 100, 120, 960, 1, prec="f64")
    block, bmax = rg.rlu_debug_lu_block(h.h)
    assert block == 0 and bmax in (16, 32, 64)
    for bad in (8, 48, 128, 120):
        with pytest.raises(rg.RluError):
            h.set_lu_block(bad)
    h.set_lu_block(-1)
    assert rg.rlu_debug_lu_block(h.h)[0] == -1
    h.close()


def test_blocked_lu_does_not_depend_on_the_grid(rg):
    """rlu_set_max_ctas bounds the panel kernel's grid; the blocked form, its
    panel width and every result stay bit-for-bit those of the full grid."""
    m, n, k, l, l1 = 20000, 600, 110, 120, 960
    A = torch.from_numpy(ri.dense_low_rank_plus_noise(m, n, 200, 1e-3, seed=8)).cuda()
    outs = []
    for ctas in (0, 7, 40):
        h = rg.RandLU(m, n, k, l, l1, 3, prec="f32")
        h.set_max_ctas(ctas)
        f = h.factor(A, check=False)
        torch.cuda.synchronize()
        outs.append([t.cpu() for t in (f.L, f.U, f.p, f.q)])
        h.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert torch.equal(a, b)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_blocked_lu_of_B(rg, prec):
    """Step 6, B Q = L_b U_b by partial pivoting of B^T: with 45000 columns B^T
    does not fit the unblocked kernel's shared memory, so the default runs it
    blocked (float-float trailing updates in the FP32 form, FP64 in the FP64
    form).  Against the unblocked kernel on the same input: the same row
    pivots (the LU of Y is unblocked in both), the same column pivots on every
    step the oracle separates, L and U entry by entry where all column pivots
    agree; both within the oracle's bars."""
    m, n, k, l, l1 = 1200, 45000, 100, 120, 960
    A = ri.dense_low_rank_plus_noise(m, n, 110, 1e-5, seed=21, dtype=np.float64)
    Ain = A if prec == "f64" else A.astype(np.float32)
    dt = torch.float64 if prec == "f64" else torch.float32
    Ad = torch.from_numpy(np.ascontiguousarray(Ain)).to("cuda", dt)
    res = {}
    for block in (-1, 0):
        h = rg.RandLU(m, n, k, l, l1, 17, prec=prec)
        h.set_lu_block(block)
        f = h.factor(Ad, check=False)
        torch.cuda.synchronize()
        res[block] = dict(L=f.L.double().cpu().numpy(), U=f.U.double().cpu().numpy(), p=f.p.cpu().numpy(),
                          q=f.q.cpu().numpy(), status=f.status)
        h.close()
    u, b = res[-1], res[0]
    assert u["status"] == 0 and b["status"] == 0
    assert np.array_equal(u["p"], b["p"])
    o = oracle.factor(Ain.astype(np.float64), k, l, l1, seed=17)
    sb = separated_prefix(o.top_b, np.abs(o.B).max(), 1e-9 if prec == "f64" else 1e-4)
    assert sb >= 1
    assert np.array_equal(u["q"][:sb], b["q"][:sb]) and np.array_equal(b["q"][:sb], o.q[:sb])
    if np.array_equal(u["q"], b["q"]):
        tol = 1e-11 if prec == "f64" else 1e-6
        assert np.abs(u["U"] - b["U"]).max() <= tol * np.abs(u["U"]).max()
        assert np.abs(u["L"] - b["L"]).max() <= tol * np.abs(u["L"]).max()
    e_o = oracle.relative_residual(Ain.astype(np.float64), o.L, o.U, o.p, o.q)
    for g in (u, b):
        e_g = oracle.relative_residual(Ain.astype(np.float64), g["L"], g["U"], g["p"], g["q"])
        assert abs(e_g - e_o) <= (1e-12 if prec == "f64" else 1e-5), (e_g, e_o)
