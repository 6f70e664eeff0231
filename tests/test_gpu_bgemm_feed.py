"""The tensor-core product B = W A (step 6 of Algorithm 1) on BF16 input read
two ways: by TMA as A lies in memory (the MMA's A operand MN-major, the
default wherever A's rows are 16-byte aligned) and by the converter warps
(K-major tiles written from global loads).  Both issue the same BF16 products
in the same order into FP32 accumulators, so B agrees to FP32 rounding at
most (in practice bit for bit); a wrong descriptor, swizzle or box offset
moves whole entries of B.  The shapes cover W in one and in two blocks of
rows, a last column tile of 80 columns (second 64-column box partly outside
A) and one of 40 (second box wholly outside), and one, two or three W planes.
With one or two planes the TMA form runs persistent (one CTA per SM over all
tiles, two accumulators in tensor memory)."""
import numpy as np
import pytest

import oracle
import rlu_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rg():
    import paper_1601_04280_gb300 as rg
    rg.build()
    rg.load(reload=True)
    return rg


def factor_B(rg, A, k, l, l1, seed, prec, tma):
    m, n = A.shape
    h = rg.RandLU(m, n, k, l, l1, seed, prec=prec)
    h.set_tma_a(tma)
    h.debug_enable(True)
    f = h.factor(torch.from_numpy(np.ascontiguousarray(A)).to("cuda", torch.bfloat16), check=False)
    torch.cuda.synchronize()
    out = dict(status=f.status, B=h.debug_B(), L=f.L.double().cpu().numpy(), U=f.U.double().cpu().numpy(),
               p=f.p.cpu().numpy(), q=f.q.cpu().numpy())
    h.close()
    return out


@pytest.mark.parametrize("m,n,k,l,l1,prec", [
    (3000, 2000, 60, 80, 640, "bf16_refine"),   # one W block; last tile 80 columns
    (3000, 2000, 60, 80, 640, "bf16"),          # one W plane
    (3000, 2000, 60, 80, 640, "f32"),           # three W planes (the non-persistent kernel)
    (5000, 1960, 300, 320, 1600, "bf16_refine"),  # two W blocks of 160 rows; last tile 40 columns
])
def test_tma_feed_equals_converters(rg, m, n, k, l, l1, prec):
    A = ri.round_to_bf16(ri.dense_low_rank_plus_noise(m, n, min(n, l + 40), 1e-3, seed=m + n + k))[0]
    t = factor_B(rg, A, k, l, l1, 31, prec, True)
    c = factor_B(rg, A, k, l, l1, 31, prec, False)
    assert t["status"] == 0 and c["status"] == 0
    scale = np.abs(c["B"]).max()
    d = np.abs(t["B"] - c["B"]).max()
    print("%dx%d k=%d %s: max |B_tma - B_conv| = %.3e of max |B| %.3e (bitwise %s)"
          % (m, n, k, prec, d, scale, np.array_equal(t["B"], c["B"])))
    assert d <= 2.0 ** -20 * scale, d
    # the factorization of the same matrix by the oracle bounds both
    o = oracle.factor(A.astype(np.float64), k, l, l1, seed=31)
    e_o = oracle.relative_residual(A.astype(np.float64), o.L, o.U, o.p, o.q)
    for g in (t, c):
        e_g = oracle.relative_residual(A.astype(np.float64), g["L"], g["U"], g["p"], g["q"])
        assert e_g <= (2.0 if prec == "bf16" else 1.05) * e_o, (e_g, e_o)


def test_tma_switch_validation(rg):
    h = rg.RandLU(1000, 800, 20, 30, 240, 1, prec="bf16")
    with pytest.raises(rg.RluError):
        rg.rlu_debug_set_tma_a(h.h, 2)
    h.set_tma_a(False)
    h.set_tma_a(True)
    h.close()
