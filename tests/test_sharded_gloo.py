"""Row-sharded form of the path on world_size-2 gloo ranks (CPU).

A splits by rows over the ranks.  The sketch is row-local (S, D, R come from
the shared seed), so rank g computes Y_g with no communication; one
allgather assembles Y, every rank runs the same panel LU (same pivots as a
single process), forms its column slice W_g of W = L_y^+ P and the partial
B_g = W_g A_g; one allreduce sums B.  The LU of B and L = L_y L_b are again
identical on every rank.  These tests run that algebra with the FP64 oracle's
steps on two CPU processes and compare with the single-process factorization.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, A, k, l, l1, seed, out_q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m, n = A.shape
        rows = np.array_split(np.arange(m), world)[rank]
        A_g = A[rows]
        # 1. local sketch rows (no communication: the projection comes from the seed)
        params = oracle.sketch_params(n, l1, l, seed)
        Y_g = oracle.fjl(oracle.countsketch(A_g, params, l1), params, l1)
        # 2. allgather Y (ranks hold contiguous row blocks, in rank order; blocks padded to equal size)
        blocks = np.array_split(np.arange(m), world)
        mx = max(len(b) for b in blocks)
        mine = torch.zeros((mx, l), dtype=torch.float64)
        mine[: len(rows)] = torch.from_numpy(Y_g)
        parts = [torch.zeros((mx, l), dtype=torch.float64) for _ in blocks]
        dist.all_gather(parts, mine)
        Y = torch.cat([pt[: len(b)] for pt, b in zip(parts, blocks)]).numpy()
        # 3. the same panel LU everywhere
        ly = oracle.lu_partial_pivot(Y, steps=l)
        Ly = oracle.unit_lower(ly.lu, k)
        W = oracle.pinv_householder(Ly)            # k x m, columns in P order
        # W acts on P A; column t of W multiplies row p[t] of A.  Slice of this rank:
        pos = np.empty(m, dtype=np.int64)
        pos[ly.perm] = np.arange(m)
        W_g = W[:, pos[rows]]                      # columns for this rank's rows, in row order
        B_g = W_g @ A_g
        # 4. allreduce B
        B = torch.from_numpy(np.ascontiguousarray(B_g))
        dist.all_reduce(B)
        B = B.numpy()
        lb = oracle.lu_partial_pivot(B.T, steps=k)
        Lb = np.triu(lb.lu[:k, :k]).T
        Ub = oracle.unit_lower(lb.lu, k).T
        L = Ly @ Lb
        out_q.put((rank, ly.perm, lb.perm, L, Ub, B))
    finally:
        dist.destroy_process_group()


def _run_sharded(A, k, l, l1, seed, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, A, k, l, l1, seed, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res, key=lambda x: x[0])


@pytest.mark.parametrize("m,n,k,l,l1", [(301, 250, 12, 18, 96), (200, 400, 20, 30, 240)])
def test_row_sharded_factorization_matches_single_process(m, n, k, l, l1):
    import oracle
    import rlu_inputs as ri
    A = ri.dense_spectrum(m, n, ri.geometric_spectrum(min(m, n), 12.0), seed=m)
    single = oracle.factor(A, k, l, l1, seed=7)
    res = _run_sharded(A, k, l, l1, 7)
    for rank, p, q, L, U, B in res:
        assert np.array_equal(p, single.p)          # identical panel LU on every rank
        assert np.array_equal(q, single.q)
        assert np.allclose(B, single.B, rtol=0, atol=1e-12 * np.abs(single.B).max())
        assert np.allclose(L, single.L, rtol=0, atol=1e-10 * np.abs(single.L).max())
        assert np.allclose(U, single.U, rtol=0, atol=1e-10)
    e1 = oracle.relative_residual(A, single.L, single.U, single.p, single.q)
    e2 = oracle.relative_residual(A, res[0][3], res[0][4], res[0][1], res[0][2])
    assert abs(e1 - e2) <= 1e-12
    # every rank ends with the same factors
    assert np.array_equal(res[0][3], res[1][3]) and np.array_equal(res[0][4], res[1][4])


def test_sharded_sketch_rows_are_the_single_process_rows():
    # the sketch is row-local: rows computed on a shard equal the same rows of the full sketch
    import oracle
    rng = np.random.default_rng(3)
    A = rng.standard_normal((90, 200))
    params = oracle.sketch_params(200, 64, 16, 5)
    full = oracle.fjl(oracle.countsketch(A, params, 64), params, 64)
    for rows in np.array_split(np.arange(90), 3):
        part = oracle.fjl(oracle.countsketch(A[rows], params, 64), params, 64)
        assert np.array_equal(part, full[rows])
