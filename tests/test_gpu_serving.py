"""Serving loop on the GPU: results in the mix equal results alone, parity of a
sample of served requests with the FP64 oracle, captured-graph replay, and
caller-owned workspaces (rlu_create_in, rlu_set_csr_workspace).

"Alone" is the ordinary entry point on a fresh handle (rlu_create +
rlu_factor_*), one request at a time; "in the mix" is the server with six
slots and every request admitted at once, so kernels of different requests
share the GPU.  The bar is bitwise equality of L, U, p and q.
"""
import numpy as np
import pytest

import oracle
from rlu_inputs import serving as rs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import check_pivots, separated_prefix  # noqa: E402


@pytest.fixture(scope="module")
def rg():
    import paper_1601_04280_gb300 as rg
    rg.build()
    rg.load(reload=True)
    return rg


@pytest.fixture(scope="module")
def mix(rg):
    from paper_1601_04280_gb300 import serving
    specs = rs.make_trace(24, seed=77, size_max=3000)
    pool = rs.dense_base_pool(2, 3000, "cuda", seed=4100)
    reqs = []
    for s in specs:
        r = serving.Request(s.rid, s.m, s.n, s.k, s.l, s.l1, rs.SKETCH_SEED)
        if s.kind == "dense":
            r.A = rs.dense_request(pool, s)
        else:
            r.csr = rs.csr_request(s, "cuda")
        reqs.append(r)
    torch.cuda.synchronize()
    return reqs


def alone(rg, r):
    h = rg.RandLU(r.m, r.n, r.k, r.l, r.l1, r.seed, prec=r.prec)
    if r.csr is not None:
        f = h.factor_csr(*r.csr, check=False)
    else:
        f = h.factor(r.A, check=False)
    torch.cuda.synchronize()
    out = (f.L.cpu(), f.U.cpu(), f.p.cpu(), f.q.cpu(), f.status)
    h.close()
    return out


def test_mix_equals_alone(rg, mix):
    from paper_1601_04280_gb300 import serving
    assert {r.kind for r in mix} == {"dense", "csr"}
    pool_bytes = sum(serving.footprint(r) for r in mix)
    with serving.Server(pool_bytes, slots=6, keep_outputs=True) as srv:
        res, span = srv.run(mix, open_loop=False)
    assert len({r.slot for r in res}) > 1
    for r, q in zip(res, mix):
        assert r.status in (rg.RLU_OK, rg.RLU_WRANK), (q.rid, r.status, r.outputs)
        L, U, p, qq, st = alone(rg, q)
        assert st == r.status
        for a, b, name in zip(r.outputs, (L, U, p, qq), "LUpq"):
            assert torch.equal(a, b), (q.rid, q.kind, name)


def test_mix_under_a_small_pool(rg, mix):
    # admission by footprint: the pool holds about two requests at a time
    from paper_1601_04280_gb300 import serving
    fps = sorted(serving.footprint(r) for r in mix)
    with serving.Server(fps[-1] + fps[-2], slots=6, keep_outputs=True) as srv:
        res, _ = srv.run(mix[:10], open_loop=False)
        assert srv.pool.in_use == 0
    for r, q in zip(res, mix[:10]):
        L, U, p, qq, st = alone(rg, q)
        assert r.status == st and torch.equal(r.outputs[0], L) and torch.equal(r.outputs[1], U)


def test_served_sample_matches_oracle(rg, mix):
    from paper_1601_04280_gb300 import serving
    sample = [r for r in mix if r.kind == "dense"][:3] + [r for r in mix if r.kind == "csr"][:3]
    with serving.Server(sum(serving.footprint(r) for r in sample), slots=4, keep_outputs=True) as srv:
        res, _ = srv.run(sample, open_loop=False)
    for r, q in zip(res, sample):
        if q.csr is not None:
            import scipy.sparse
            rowptr, colind, val = (t.cpu().numpy() for t in q.csr)
            A = scipy.sparse.csr_matrix((val.astype(np.float64), colind, rowptr), shape=(q.m, q.n))
        else:
            A = q.A.cpu().double().numpy()
        o = oracle.factor(A, q.k, q.l, q.l1, seed=q.seed)
        L, U, p, qq = (t.numpy() for t in r.outputs)
        g = dict(L=L.astype(np.float64), U=U.astype(np.float64), p=p, q=qq)
        check_pivots(g, o, q.k)
        e_o = oracle.relative_residual(A, o.L, o.U, o.p, o.q)
        e_g = oracle.relative_residual(A, g["L"], g["U"], g["p"], g["q"])
        if q.csr is None:
            assert abs(e_g - e_o) <= 1e-5, (q.rid, e_g, e_o)
        else:
            # N(0,1) sparse noise has no spectral gap: pivots past the separated
            # prefix may legitimately differ, so the error agrees relatively
            assert abs(e_g / e_o - 1) <= 1e-2, (q.rid, e_g, e_o)


def test_graph_replay_equals_eager(rg):
    from paper_1601_04280_gb300 import serving
    m, n, k, l, l1 = 1024, 1024, 20, 30, 240
    pool = rs.dense_base_pool(1, 1024, "cuda", seed=4200)
    A1 = pool[0]
    A2 = (pool[0] * 0.5 + 0.25 * torch.roll(pool[0], 7, dims=1)).contiguous()
    bucket = serving.GraphBucket(m, n, k, l, l1, 11, prec="f32")
    try:
        before = rg.rlu_debug_launch_count()
        assert bucket.serve(A1) == 0          # eager run + capture
        eager_launches = rg.rlu_debug_launch_count() - before
        outs = []
        for A in (A2, A1, A2):
            before = rg.rlu_debug_launch_count()
            assert bucket.serve(A) == 0       # replay
            # the graph holds the eager path's kernels plus the status-code kernel
            assert rg.rlu_debug_launch_count() - before == eager_launches + 1
            outs.append(tuple(t.clone() for t in bucket.out))
        for A, o in zip((A2, A1, A2), outs):
            L, U, p, q, st = alone(rg, serving.Request(0, m, n, k, l, l1, 11, A=A))
            for a, b in zip(o, (L, U, p, q)):
                assert torch.equal(a.cpu(), b)
    finally:
        bucket.close()


@pytest.mark.parametrize("kind", ["dense", "csr"])
def test_max_ctas_does_not_change_results(rg, mix, kind):
    # the grid of the pivoted LUs and the Cholesky kernel is bounded; the
    # factors are bit-for-bit those of the default grid
    q = [r for r in mix if r.kind == kind][0]
    ref = alone(rg, q)
    for ctas in (1, 7, 40):
        h = rg.RandLU(q.m, q.n, q.k, q.l, q.l1, q.seed, prec=q.prec)
        h.set_max_ctas(ctas)
        f = h.factor_csr(*q.csr, check=False) if q.csr is not None else h.factor(q.A, check=False)
        torch.cuda.synchronize()
        for a, b in zip((f.L.cpu(), f.U.cpu(), f.p.cpu(), f.q.cpu()), ref[:4]):
            assert torch.equal(a, b), (kind, ctas)
        h.close()


def test_create_in_rejects_small_or_misaligned_workspace(rg):
    need = rg.rlu_workspace_bytes(500, 400, 10, 16, 64, "f32")
    buf = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    base = buf.data_ptr() + (-buf.data_ptr()) % 256
    import ctypes
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    with pytest.raises(rg.RluError):
        rg.rlu_create_in(500, 400, 10, 16, 64, 1, ctypes.c_void_p(base), need - 256, s)
    with pytest.raises(rg.RluError):
        rg.rlu_create_in(500, 400, 10, 16, 64, 1, ctypes.c_void_p(base + 16), need, s)
    h = rg.rlu_create_in(500, 400, 10, 16, 64, 1, ctypes.c_void_p(base), need, s)
    rg.rlu_destroy(h)


def test_csr_workspace_limit_enforced(rg):
    spec = rs.RequestSpec(0, "csr", 900, 700, 12, 32, 96, 51, 1.0)
    rowptr, colind, val = rs.csr_request(spec, "cuda")
    h = rg.RandLU(900, 700, 12, 32, 96, 3, prec="f32")
    nnz = int(val.numel())
    need = rg.rlu_csr_workspace_bytes(900, 700, 12, nnz - 1)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    h.set_csr_workspace(ws, nnz - 1)
    f = h.factor_csr(rowptr, colind, val, check=False)
    assert f.status == rg.RLU_EINVAL     # more entries than the scratch was sized for
    h.close()


def test_bucketed_graphs_match_plain(rg):
    """Graph replay per size bucket: requests whose m, n round up to the same
    bucket (1024 x 1024 here) share one captured graph; each is copied into
    the bucket's zero-padded input.  Restricted to the request, the padded
    factorization has the plain call's sketch and row pivots exactly (zero
    columns add exact zeros, zero rows never win a pivot, padded positions are
    never swapped).  B = W A is FP32-accurate and its split over the rows
    follows the padded m, so B differs by FP32 rounding: the column pivots
    agree on the steps the oracle separates (its two best candidates more
    than 1e-4 apart), L and U entry by entry (1e-4 of their largest entry)
    wherever all column pivots agree, |de| <= 1e-6, and every request within
    the FP32 bar of the oracle."""
    from paper_1601_04280_gb300 import serving
    base = rs.dense_base_pool(2, 1100, "cuda", seed=4300)
    sizes = [(900, 850), (1000, 990), (1024, 1024), (800, 780), (950, 1010), (1024, 900), (870, 1024), (999, 999)]
    reqs = [serving.Request(i, m, n, 20, 30, 240, 17, A=base[i % 2][:m, :n]) for i, (m, n) in enumerate(sizes)]
    assert len({serving.bucket_key(r) for r in reqs}) == 1
    pool_bytes = 2 * sum(serving.footprint(r) for r in reqs)
    # one slot: the bucket serves the requests one after another (with more
    # slots a request that finds its bucket busy runs on the ordinary path)
    with serving.Server(pool_bytes, slots=1, keep_outputs=True, graphs=True, graph_min_uses=1) as srv:
        res, _ = srv.run(reqs, open_loop=False)
        stats = dict(srv.graph_stats)
    assert stats["captures"] == 1 and stats["replays"] == len(reqs) - 1, stats
    full_q = 0
    for r, q in zip(res, reqs):
        assert r.status in (rg.RLU_OK, rg.RLU_WRANK), (q.rid, r.status, r.outputs)
        L, U, p, qq, st = alone(rg, q)
        assert torch.equal(r.outputs[2], p), q.rid
        A = q.A.cpu().double().numpy()
        o = oracle.factor(A, q.k, q.l, q.l1, seed=q.seed)
        sb = separated_prefix(o.top_b, np.abs(o.B).max(), 1e-4)
        assert torch.equal(r.outputs[3][:sb], qq[:sb]), q.rid
        if torch.equal(r.outputs[3], qq):
            full_q += 1
            assert (r.outputs[0] - L).abs().max() <= 1e-4 * L.abs().max()
            assert (r.outputs[1] - U).abs().max() <= 1e-4
        g = [t.double().numpy() if t.is_floating_point() else t.numpy() for t in r.outputs]
        e_b = oracle.relative_residual(A, *g)
        e_p = oracle.relative_residual(A, L.double().numpy(), U.double().numpy(), p.numpy(), qq.numpy())
        e_o = oracle.relative_residual(A, o.L, o.U, o.p, o.q)
        assert abs(e_b - e_p) <= 1e-6, (q.rid, e_b, e_p)
        assert abs(e_b - e_o) <= 1e-5, (q.rid, e_b, e_o)
    print("bucketed: %d of %d requests with every column pivot of the plain call" % (full_q, len(reqs)))
    assert full_q >= 1


def test_bucket_ladder():
    from paper_1601_04280_gb300 import serving
    assert serving.bucket_dim(1) == 512 and serving.bucket_dim(512) == 512
    assert serving.bucket_dim(513) == 768 and serving.bucket_dim(1024) == 1024
    assert serving.bucket_dim(16384) == 16384
    prev = 0
    for x in range(1, 16385, 37):
        b = serving.bucket_dim(x)
        assert b >= x and b % 64 == 0 and (b <= 1.5 * x or b == 512)
        assert b >= prev
        prev = b
