"""Failure detection on the GPU without a fault: the library's bounded device
waits give up on a condition that never comes true, report RLU_ETIMEOUT, and
leave the context usable for the next factorization."""
import time

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


@pytest.mark.parametrize("which", [0, 1], ids=["grid_barrier", "mbarrier"])
def test_bounded_wait_gives_up_and_context_survives(rg, which):
    t0 = time.perf_counter()
    status = rg.rlu_debug_wait_timeout(which)
    dt = time.perf_counter() - t0
    assert status == rg.RLU_ETIMEOUT
    # the limit is about a second of SM clock; allow for clock and launch slack
    assert 0.2 < dt < 20.0, dt
    # the same process and GPU then factor a matrix correctly
    A = ri.dense_spectrum(400, 300, ri.geometric_spectrum(300), 11)
    h = rg.RandLU(400, 300, 12, 16, 128, 5, prec="f64")
    f = h.factor(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    assert f.status == rg.RLU_OK
    o = oracle.factor(A, 12, 16, 128, 5)
    e_g = oracle.relative_residual(A, f.L.cpu().numpy(), f.U.cpu().numpy(), f.p.cpu().numpy(), f.q.cpu().numpy())
    e_o = oracle.relative_residual(A, o.L, o.U, o.p, o.q)
    assert abs(e_g - e_o) <= 1e-12
    assert np.array_equal(f.p.cpu().numpy()[:12], o.p[:12])
    h.close()


def test_alu_peak_probe_is_plausible(rg):
    """The FMA probe that the benchmark's ALU rooflines use: FP64 and FP32 rates
    of a GB300-class part (FP64 vector 1/64 of FP32)."""
    f64 = rg.rlu_debug_alu_peak(0)
    f32 = rg.rlu_debug_alu_peak(1)
    assert 0.3 < f64 < 10.0, f64
    assert 20.0 < f32 < 200.0, f32
    assert f32 > 8 * f64
