"""Seeded request traces and device-resident inputs for the serving form.

The serving workload is a stream of independent factorization requests of
uneven sizes: Poisson arrivals; m and n log-uniform in [512, 16384]; 70 %
dense FP32 matrices with the geometric spectrum sigma_i = 10^(-(i-1)/10) of
the dense workloads (Sec. 4 style: orthonormal factors times a prescribed
spectrum), 30 % CSR matrices at 0.5 % density with N(0,1) values; k uniform in
[16, 256], l = k + 20 and l1 = 8 k.

Like the rest of this package, nothing here is the method's arithmetic.  The
trace itself is numpy (a pure function of its seed).  The matrices are made
on the device with torch's seeded generators, because thousands of requests
of up to 16384 x 16384 cannot be staged from the host in reasonable time:
dense requests are the leading m x n blocks (row stride 16384) of a few
distinct rank-96 base matrices, cycled by the request's data seed; CSR
requests are generated one by one at their exact sizes.  A test that needs a
request on the host copies it back.
"""
from dataclasses import dataclass

import numpy as np

#: sizes of the serving trace
SIZE_MIN, SIZE_MAX = 512, 16384
K_MIN, K_MAX = 16, 256
DENSE_SHARE = 0.7
CSR_DENSITY = 0.005
BASE_RANK = 96          # sigma_97 = 10^-9.6: below FP32 resolution
SKETCH_SEED = 2004


@dataclass(frozen=True)
class RequestSpec:
    rid: int
    kind: str        # "dense" or "csr"
    m: int
    n: int
    k: int
    l: int
    l1: int
    data_seed: int
    gap: float       # inter-arrival gap before this request, in units of the mean gap


def make_trace(count=4096, seed=2004, size_max=SIZE_MAX):
    """The request trace: sizes, kinds and unit-mean exponential arrival gaps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = np.log(SIZE_MIN), np.log(size_max)
    out = []
    for rid in range(count):
        kind = "dense" if rng.random() < DENSE_SHARE else "csr"
        m = int(round(np.exp(rng.uniform(lo, hi))))
        n = int(round(np.exp(rng.uniform(lo, hi))))
        k = int(rng.integers(K_MIN, K_MAX + 1))
        gap = float(rng.exponential(1.0))
        out.append(RequestSpec(rid, kind, m, n, k, k + 20, 8 * k, 3000 + rid, gap))
    return out


def dense_base_pool(count, size, device, seed=3000, rank=BASE_RANK):
    """`count` distinct size x size FP32 matrices X diag(sigma) Y^T (X, Y with
    orthonormal columns from the QR of seeded Gaussians, sign-fixed by R's
    diagonal; sigma_i = 10^(-(i-1)/10), i <= rank), made on `device`."""
    import torch
    sig = torch.tensor(10.0 ** (-np.arange(rank) / 10.0), dtype=torch.float64, device=device)
    pool = []
    for b in range(count):
        g = torch.Generator(device=device)
        g.manual_seed(seed + b)
        fac = []
        for _ in range(2):
            G = torch.randn(size, rank, generator=g, device=device, dtype=torch.float64)
            Q, R = torch.linalg.qr(G)
            sgn = torch.sign(torch.diagonal(R))
            sgn[sgn == 0] = 1
            fac.append(Q * sgn)
        A = ((fac[0] * sig) @ fac[1].T).to(torch.float32)
        pool.append(A)
    return pool


def dense_request(pool, spec):
    """Leading m x n block of base matrix data_seed mod len(pool) (row stride = base width)."""
    base = pool[spec.data_seed % len(pool)]
    return base[: spec.m, : spec.n]


def csr_request(spec, device, density=CSR_DENSITY):
    """CSR at the request's exact size: round(density * n) (at least one) uniform
    columns per row, sorted, repeats allowed (they sum); N(0,1) FP32 values.
    Returns (rowptr int64, colind int32, val float32) on `device`."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(spec.data_seed)
    npr = max(1, int(round(density * spec.n)))
    cols = torch.randint(0, spec.n, (spec.m, npr), generator=g, device=device, dtype=torch.int64)
    cols = torch.sort(cols, dim=1).values.to(torch.int32).reshape(-1)
    val = torch.randn(spec.m * npr, generator=g, device=device, dtype=torch.float32)
    rowptr = torch.arange(spec.m + 1, device=device, dtype=torch.int64) * npr
    return rowptr, cols, val
