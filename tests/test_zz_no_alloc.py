"""rlu_sketch_dense_noalloc: the sketch step for callers that cannot allocate.

A serving loop cannot afford cudaMalloc on its call path (it synchronizes the
device), and a process whose device memory belongs to another framework's
pool may have nothing left to allocate; such callers use the entry point that
keeps its scratch in a fixed device array of the library.  Its result must
equal the sketch that the ordinary handle-based path computes for the same
A, l, l1 and seed, on two calls in a row (the second call must not be
disturbed by what the first left in the shared scratch).  This file is
collected last so that a failure here never hides the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sketch_via_handle(rg, A, l, l1, seed, prec):
    m, n = A.shape
    h = rg.RandLU(m, n, min(l, 8), l, l1, seed, prec=prec)
    h.debug_enable(True)
    h.factor(A)
    torch.cuda.synchronize()
    Y = h.debug_Y()
    h.close()
    return Y


def _sketch_noalloc(rg, A, l, l1, seed):
    m, n = A.shape
    Y = torch.empty((m, l), dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    code = {torch.float64: rg.RLU_F64, torch.float32: rg.RLU_F32, torch.bfloat16: rg.RLU_BF16}[A.dtype]
    rc = rg.rlu_sketch_dense_noalloc(ctypes.c_void_p(A.data_ptr()), A.stride(0), code, m, n, l, l1, seed,
                                     ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(st.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, Y, st


def test_noalloc_sketch_matches_handle_path_on_two_calls():
    import paper_1601_04280_gb300 as rg
    rg.build()
    rg.load(reload=True)
    g = torch.Generator().manual_seed(5)
    cases = [
        # (m, n, l, l1, seed, dtype, prec of the handle path, row stride)
        # whole rows in shared memory:
        (300, 5000, 30, 240, 11, torch.float32, "f32", None),
        (257, 3000, 64, 1600, 12, torch.float64, "f64", None),
        # column chunks through the fixed scratch's per-chunk counters and lists:
        # n = the maximum, more than 32 entries per bucket (64 chunks x 1600 buckets)
        (40, 65536, 32, 1600, 13, torch.float32, "f32", None),
        # rows too long for shared memory at the maximum l1 (30 chunks x 4096 buckets)
        (24, 60000, 16, 4096, 14, torch.bfloat16, "f32", None),
        # a row stride that is not a multiple of 16 bytes: the register-staged kernel
        (50, 3000, 20, 240, 15, torch.float32, "f32", 3001),
    ]
    inputs, refs = [], []
    for m, n, l, l1, seed, dt, prec, lda in cases:
        full = torch.randn((m, lda or n), generator=g, dtype=torch.float64).to(dt).cuda()
        A = full[:, :n]
        inputs.append(A)
        refs.append(_sketch_via_handle(rg, A, l, l1, seed, prec))
    # two calls in a row, then compare both with the handle path
    outs = []
    for (m, n, l, l1, seed, dt, prec, lda), A in zip(cases, inputs):
        rc, Y, st = _sketch_noalloc(rg, A, l, l1, seed)
        assert rc == rg.RLU_OK, rg.strerror(rc)
        outs.append((Y, st))
    torch.cuda.synchronize()
    for (Y, st), ref in zip(outs, refs):
        assert int(st.item()) == rg.RLU_OK
        Yh = Y.cpu().numpy()
        # same tolerance as the FP64 sketch parity tests: 1e-12 of the largest entry
        assert np.abs(Yh - ref).max() <= 1e-12 * np.abs(ref).max()


def test_noalloc_sketch_rejects_sizes_beyond_its_scratch():
    import paper_1601_04280_gb300 as rg
    rg.load()
    A = torch.zeros((64, 8), dtype=torch.float32, device="cuda")
    Y = torch.empty((64, 32), dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    big_n = rg.RLU_NOALLOC_MAX_N + 1
    rc = rg.rlu_sketch_dense_noalloc(ctypes.c_void_p(A.data_ptr()), big_n, rg.RLU_F32, 64, big_n, 32, 64, 1,
                                     ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(st.data_ptr()), s)
    assert rc == rg.RLU_ETOOLARGE
    rc = rg.rlu_sketch_dense_noalloc(ctypes.c_void_p(A.data_ptr()), 8, rg.RLU_F32, 64, 8, 32,
                                     rg.RLU_NOALLOC_MAX_L1 + 1, 1, ctypes.c_void_p(Y.data_ptr()),
                                     ctypes.c_void_p(st.data_ptr()), s)
    assert rc == rg.RLU_ETOOLARGE
    assert "scratch" in rg.strerror(rg.RLU_ETOOLARGE)
