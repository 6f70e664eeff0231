"""The SRHT and the real form of the complex SRFT on the GPU (rlu_set_transform)
against the oracle's transform_matrix: the sketch Y entry by entry, whole
factorizations by their error and pivots.  Same bars as test_gpu_parity:
FP64 Y within 1e-12 of its largest entry, |e_gpu - e_oracle| <= 1e-12, B
within 1e-9; FP32 Y within 5e-6 of the largest row norm, |delta e| <= 1e-5."""
import numpy as np
import pytest

import oracle
import rlu_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import check_pivots, check_structure  # noqa: E402


@pytest.fixture(scope="module")
def rg():
    import paper_1601_04280_gb300 as rg
    rg.build()
    rg.load(reload=True)
    return rg


def run(rg, A_np, k, l, l1, seed, prec, transform, dtype):
    m, n = A_np.shape
    h = rg.RandLU(m, n, k, l, l1, seed, prec=prec)
    h.set_transform(transform)
    h.debug_enable(True)
    f = h.factor(torch.from_numpy(np.ascontiguousarray(A_np)).to("cuda", dtype), check=False)
    torch.cuda.synchronize()
    out = dict(L=f.L.double().cpu().numpy(), U=f.U.double().cpu().numpy(), p=f.p.cpu().numpy(),
               q=f.q.cpu().numpy(), status=f.status, Y=h.debug_Y(), B=h.debug_B())
    h.close()
    return out


@pytest.mark.parametrize("transform,l1", [("srht", 256), ("srft", 240), ("srft", 251)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_sketch_Y_transform(rg, transform, l1, prec):
    m, n, l = 130, 3000, 30
    rng = np.random.default_rng(l1 + len(prec))
    A = rng.standard_normal((m, n))
    dt = torch.float64 if prec == "f64" else torch.float32
    if prec == "f32":
        A = A.astype(np.float32)
    g = run(rg, A, 8, l, l1, 55, prec, transform, dt)
    p = oracle.sketch_params(n, l1, l, 55)
    Yo = oracle.fjl(oracle.countsketch(A.astype(np.float64), p, l1), p, l1, transform)
    if prec == "f64":
        assert np.abs(g["Y"] - Yo).max() <= 1e-12 * np.abs(Yo).max()
    else:
        rown = np.linalg.norm(A.astype(np.float64), axis=1).max()
        assert np.abs(g["Y"] - Yo).max() <= 5e-6 * rown


@pytest.mark.parametrize("transform,l1", [("srht", 256), ("srft", 240)])
def test_transform_factor_parity_f64(rg, transform, l1):
    w = ri.DENSE_F64_1K
    A = ri.make_dense(w)
    o = oracle.factor(A, w.k, w.l, l1, w.sketch_seed, transform=transform)
    g = run(rg, A, w.k, w.l, l1, w.sketch_seed, "f64", transform, torch.float64)
    assert g["status"] == 0
    check_structure(g, w.m, w.n, w.k)
    check_pivots(g, o, w.k)
    e_o = oracle.relative_residual(A, o.L, o.U, o.p, o.q)
    e_g = oracle.relative_residual(A, g["L"], g["U"], g["p"], g["q"])
    assert abs(e_g - e_o) <= 1e-12, (e_g, e_o)
    assert np.abs(g["B"] - o.B).max() <= 1e-9 * np.abs(o.B).max()
    print("%s: e_gpu %.6e e_oracle %.6e" % (transform, e_g, e_o))


@pytest.mark.parametrize("transform,l1", [("srht", 512), ("srft", 400)])
def test_transform_factor_parity_f32(rg, transform, l1):
    m, n, k, l = 1500, 1100, 30, 40
    A = ri.dense_low_rank_plus_noise(m, n, 30, 1e-5, seed=44)
    o = oracle.factor(A.astype(np.float64), k, l, l1, 66, transform=transform)
    g = run(rg, A, k, l, l1, 66, "f32", transform, torch.float32)
    assert g["status"] == 0
    check_structure(g, m, n, k)
    check_pivots(g, o, k)
    e_o = oracle.relative_residual(A, o.L, o.U, o.p, o.q)
    e_g = oracle.relative_residual(A, g["L"], g["U"], g["p"], g["q"])
    assert abs(e_g - e_o) <= 1e-5, (e_g, e_o)


def test_transform_validation(rg):
    h = rg.RandLU(300, 200, 10, 15, 240, 1, prec="f64")
    with pytest.raises(rg.RluError):
        h.set_transform("srht")  # 240 is not a power of two
    with pytest.raises(rg.RluError):
        h.set_transform("srft")  # l = 15 is odd
    with pytest.raises(rg.RluError):
        h.set_transform(7)
    h.close()
    h = rg.RandLU(300, 200, 10, 16, 256, 1, prec="f32")
    h.set_transform("srht")
    import scipy.sparse
    As = scipy.sparse.random(300, 200, density=0.05, random_state=2, format="csr", dtype=np.float32)
    f = h.factor_csr(torch.from_numpy(As.indptr.astype(np.int64)).cuda(), torch.from_numpy(As.indices).cuda(),
                     torch.from_numpy(As.data).cuda(), check=False)
    assert f.status == rg.RLU_EINVAL
    h.set_transform("hartley")
    f = h.factor_csr(torch.from_numpy(As.indptr.astype(np.int64)).cuda(), torch.from_numpy(As.indices).cuda(),
                     torch.from_numpy(As.data).cuda(), check=False)
    assert f.status in (rg.RLU_OK, rg.RLU_WRANK)
    h.close()
