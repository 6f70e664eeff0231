"""Benchmark of the sparse randomized LU path on GB300.

One step = one whole factorization (sketch parameters, CountSketch + Hartley
sketch, FP64 panel LU, L_y^+ and B = L_y^+ P A, LU of B, assembly of L, U, p, q).
Default workload: CSR FP32 200000 x 50000, 40 uniform columns per row with
N(0,1) values plus a dense rank-50 block on 4000 rows (2.08e8 nonzeros, 1.67 GB
of values and column indices, larger than the 129 MB L2), k = 100, l = 120,
l1 = 960: the largest workload on one GPU.  Other workloads (--workload):
dense FP32 8192 x 8192 (k = 200), dense FP64 1024 x 1024 (k = 20), dense BF16
32768 x 16384 (k = 500; --prec bf16_refine | bf16 | f32), and the serving trace.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Prints one JSON line on rank 0.  Under torchrun (N > 1) each rank factors its
own matrix (independent problems: weak scaling, no data-path collective); the
timed region is bracketed by barriers and the max over ranks is reported.
The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores on the same workload (rank 0 only).
"""
import argparse
import json

import numpy as np
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rand-LU factorizations/s"
UNIT = "factorizations/s"
#: workload name -> (rlu_inputs workload, default precision, input kind)
WORKLOADS = {
    "dense_f32_8192x8192_k200": ("DENSE_F32_8K", "f32", "dense"),
    "dense_f64_1024x1024_k20": ("DENSE_F64_1K", "f64", "dense"),
    "csr_f32_200000x50000_k100": ("CSR_F32_200K", "f32", "csr"),
    "dense_bf16_32768x16384_k500": ("DENSE_BF16_32K", "bf16_refine", "dense"),
}
DEFAULT_WORKLOAD = "csr_f32_200000x50000_k100"
#: the serving form: a trace of independent requests of uneven sizes
SERVING_WORKLOAD = "serving_4096req_mixed_dense_f32_csr"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu capture
# of the current kernels (profiles/top_kernels_dense_f32_8192.md: k_pivoted_lu of Y);
# a workload without a capture of its current dominant kernel reports null.
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the dominant
# kernel from an ncu capture (profiles/panel_lu_f64_200000x16.md: a 16-wide
# panel over 200000 rows, the same launch shape as the sparse workload's
# panels); null for workloads without a capture of the current kernel
MEASURED_TRAFFIC = {("csr_f32_200000x50000_k100", "panel_lu"): 25674496 + 77568}

# FP64 vector peak from unit counts, used only when the measurement below is
# unavailable: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz = 1.259 TFLOP/s.
FP64_PEAK_UNIT_COUNT_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def fp64_peak(rg):
    """(TFLOP/s, how): the FP64 FMA rate measured on this GPU by the library's
    FMA-chain kernel, else the unit-count figure."""
    try:
        v = rg.rlu_debug_alu_peak(0)
        if v > 0:
            return v, "measured on this GPU in this run (rlu_debug_alu_peak: FP64 FMA chains, every SM)"
    except Exception:
        pass
    return FP64_PEAK_UNIT_COUNT_TFLOPS, "FP64 unit counts: 152 SM x 2 FMA/clk x 2 x 2.07 GHz"


def device_rel_error(kind, dev_in, m, n, L, U, p, q):
    """||L U - P A Q||_F / ||A||_F in FP64 on the device (one routine for the
    GPU's and the oracle's factors).  Dense: the difference formed explicitly.
    CSR: ||LU||^2 - 2 <LU, PAQ> + ||A||^2, with ||LU||_F^2 = trace((L^T L)(U U^T))
    and the inner product over the nonzeros in chunks."""
    import torch
    L = L.double()
    U = U.double()
    if kind != "csr":
        Ad = dev_in[0].double()
        r = float(torch.linalg.norm(L @ U - Ad[p][:, q]) / torch.linalg.norm(Ad))
        del Ad
        return r
    rowptr, colind, val = dev_in
    dev = L.device
    pinv = torch.empty(m, dtype=torch.int64, device=dev)
    pinv[p] = torch.arange(m, device=dev)
    qinv = torch.empty(n, dtype=torch.int64, device=dev)
    qinv[q] = torch.arange(n, device=dev)
    rows = torch.repeat_interleave(torch.arange(m, device=dev), rowptr[1:] - rowptr[:-1])
    lu2 = float(torch.sum((L.T @ L) * (U @ U.T)))
    v64 = val.double()
    a2 = float(torch.sum(v64 * v64))
    Ut = U.T.contiguous()
    inner = 0.0
    step = 1 << 21
    for s0 in range(0, val.numel(), step):
        r = pinv[rows[s0:s0 + step]]
        c = qinv[colind[s0:s0 + step].long()]
        inner += float(torch.sum(v64[s0:s0 + step] * torch.sum(L[r] * Ut[c], dim=1)))
    return float(np.sqrt(max(lu2 - 2.0 * inner + a2, 0.0) / a2))


ORACLE_CHILD_BUDGET_S = 150.0


def oracle_child(workload, second_json):
    """Runs in a child process with one BLAS/OpenMP thread: one oracle
    factorization of the workload, its seconds printed as JSON."""
    w, A = make_input(workload)
    second = json.loads(second_json) if second_json else None
    print(json.dumps({"seconds": oracle_factor_seconds(w, A, second)}), flush=True)
    return 0


def cpu_baseline(args, w, A, second, budget_s=40.0):
    """The FP64 oracle on the host cores: best of up to three full
    factorizations with all threads (while their total stays within budget_s),
    then one factorization with one thread in a child process (bounded by
    ORACLE_CHILD_BUDGET_S).  Returns (line object, the oracle's factors of the
    first run)."""
    import oracle
    Ao = oracle_input(w, A)
    runs, res = [], None
    while len(runs) < 3 and sum(runs) < budget_s:
        t0 = time.perf_counter()
        if second:
            r = oracle.factor_two_sketch(Ao, w.k, w.l, w.l1, second["k2"], second["l2"], w.sketch_seed,
                                         second["seed2"])
        else:
            r = oracle.factor(Ao, w.k, w.l, w.l1, w.sketch_seed)
        runs.append(time.perf_counter() - t0)
        res = res or r
    one = {"value": None, "unit": UNIT, "cores": 1, "runs_s": []}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", args.workload,
                              "--oracle-child-second", json.dumps(second) if second else ""],
                             capture_output=True, text=True, timeout=ORACLE_CHILD_BUDGET_S, env=env)
        secs = json.loads(out.stdout.strip().splitlines()[-1])["seconds"]
        one.update(value=1.0 / secs, runs_s=[secs])
    except Exception as exc:  # noqa: BLE001 - reported, not raised
        one["note"] = "not measured: %s" % type(exc).__name__
    cpu = {"value": 1.0 / min(runs), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": "best of %d full factorizations of the workload by the FP64 oracle (numpy/scipy, all host "
                     "threads), then one factorization with one thread" % len(runs),
           "runs_s": runs, "one_thread": one}
    return cpu, res


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "", 1).isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def make_input(name):
    """(workload, A): A dense ndarray (bf16 values held in float32) or a CSR tuple."""
    import rlu_inputs as ri
    w = getattr(ri, WORKLOADS[name][0])
    if WORKLOADS[name][2] == "csr":
        return w, ri.csr_sparse_plus_low_rank(w.m, w.n, 40, w.m // 50, 50, w.data_seed, dtype=np.float32)
    return w, ri.make_dense(w)


def oracle_input(w, A):
    import rlu_inputs as ri
    if isinstance(A, tuple):
        return ri.csr_to_scipy(*A)
    return A.astype(np.float64)


def oracle_factor_seconds(w, A, second=None):
    import oracle
    Ao = oracle_input(w, A)
    t0 = time.perf_counter()
    if second:
        oracle.factor_two_sketch(Ao, w.k, w.l, w.l1, second["k2"], second["l2"], w.sketch_seed, second["seed2"])
    else:
        oracle.factor(Ao, w.k, w.l, w.l1, w.sketch_seed)
    return time.perf_counter() - t0


def algorithmic_flops_panel_lu(m, l):
    # sum_j 2 (m - j - 1)(l - j - 1) + (m - j - 1) divisions, FP64
    return sum(2.0 * (m - j - 1) * (l - j - 1) + (m - j - 1) for j in range(l))


def lu_panels(l, b):
    """(first column, width) of the pivoted-LU kernel's launches: one over all
    l columns when unblocked (b = 0), else panels of b columns."""
    return [(0, l)] if b == 0 else [(j0, min(b, l - j0)) for j0 in range(0, l, b)]


def algorithmic_flops_lu_panels(m, l, b):
    """FP64 work of the pivoted-LU kernel's launches for the m x l LU with panel
    width b: each panel's own elimination (the unblocked count on the rows not
    yet pivoted and the panel's columns); the trailing updates between panels
    run in other kernels, on the tensor cores."""
    return sum(2.0 * (m - j0 - j - 1) * (wid - j - 1) + (m - j0 - j - 1)
               for j0, wid in lu_panels(l, b) for j in range(wid))


def run_reference(args, rank):
    if rank != 0:
        return 0
    w, A = make_input(args.workload)
    cores = os.cpu_count()
    # one step = one full oracle factorization (FP64, numpy/scipy on the host cores)
    for _ in range(args.warmup):
        oracle_factor_seconds(w, A)
    times = [oracle_factor_seconds(w, A) for _ in range(args.steps)]
    tot = sum(times)
    value = args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "m": w.m, "n": w.n, "k": w.k, "l": w.l, "l1": w.l1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d full factorizations of the workload by the FP64 oracle" % args.steps},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def stage_work(kind, w, a_bytes, nnz, prec="f32"):
    """Algorithmic work of each stage for one factorization: (amount, unit, bound).
    B = W A runs on the tensor cores except in FP64 (FP64 SIMT) and for the
    light CSR entries (sparse)."""
    m, n, k, l = w.m, w.n, w.k, w.l
    bflops = (2.0 * k * nnz) if kind == "csr" else (2.0 * k * m * n)
    return {
        "sketch": (a_bytes, "bytes", "hbm"),
        "panel_lu": (algorithmic_flops_panel_lu(m, l), "fp64_flops", "alu"),
        "bgemm": (bflops, "fp64_flops", "alu") if prec == "f64" else (bflops, "flops", "tensor"),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + [SERVING_WORKLOAD])
    ap.add_argument("--requests", type=int, default=4096, help="serving: requests in the trace")
    ap.add_argument("--slots", type=int, default=8, help="serving: concurrent slots")
    ap.add_argument("--pool-gb", type=float, default=48.0, help="serving: device pool for admission (GiB)")
    ap.add_argument("--e2e-requests", type=int, default=256, help="serving: requests of the host-arrival run")
    ap.add_argument("--coop-ctas", type=int, default=-1,
                    help="serving: CTAs of each request's grid-synchronised kernels (0 = one per SM, -1 = the "
                         "server's default, a quarter of the SMs)")
    ap.add_argument("--prec", default=None, help="override the workload's precision (f64, f32, bf16, bf16_refine)")
    ap.add_argument("--second-projection", action="store_true",
                    help="B by the paper's second projection (k2 = min(2 l, 1024), l2 = min(8 k2, 4096)) instead of the exact L_y^+")
    ap.add_argument("--oracle-child", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-child-second", default="", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_child:
        return oracle_child(args.oracle_child, args.oracle_child_second)
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.workload == SERVING_WORKLOAD:
            return run_serving_reference(args, rank)
        return run_reference(args, rank)
    if args.workload == SERVING_WORKLOAD:
        return run_serving(args, rank, world, local)

    import torch
    import torch.distributed as dist

    import paper_1601_04280_gb300 as rg

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    rg.load()

    _, prec_default, kind = WORKLOADS[args.workload]
    prec = args.prec or prec_default
    w, A_np = make_input(args.workload)
    m, n, k, l, l1 = w.m, w.n, w.k, w.l, w.l1
    dev = torch.device("cuda", local)
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[w.dtype]
    if kind == "csr":
        rowptr_np, colind_np, val_np = A_np[0], A_np[1], A_np[2]
        nnz = int(rowptr_np[-1])
        dev_in = (torch.from_numpy(rowptr_np).to(dev), torch.from_numpy(colind_np).to(dev),
                  torch.from_numpy(val_np).to(dev))
        a_bytes = nnz * (4 + val_np.itemsize) + 8 * (m + 1)
    else:
        nnz = m * n
        dev_in = (torch.from_numpy(A_np).to(dev, tdt),)
        a_bytes = dev_in[0].element_size() * m * n
    h = rg.RandLU(m, n, k, l, l1, w.sketch_seed + rank, prec=prec)
    second = None
    if args.second_projection:
        if kind == "csr":
            raise SystemExit("--second-projection is built for dense inputs")
        k2 = min(2 * l, 1024)
        second = {"k2": k2, "l2": min(8 * k2, 4096), "seed2": w.sketch_seed + 7}
        h.set_second_sketch(second["k2"], second["l2"], second["seed2"])
    outs = h.alloc_outputs(dev)
    stream = torch.cuda.current_stream(dev)

    def factor():
        if kind == "csr":
            return h.factor_csr(*dev_in, out=outs)
        return h.factor(dev_in[0], out=outs)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        factor()
    torch.cuda.synchronize()

    # device-timed region: K factorizations, per-step events for p50/p99
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    launches0 = rg.rlu_debug_launch_count()
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for i in range(args.steps):
            factor()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
    barrier()
    launches = rg.rlu_debug_launch_count() - launches0
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps / (total_ms / 1e3)

    # the same steps replayed from one captured launch graph (dense inputs)
    graph = None
    if kind == "dense":
        import ctypes
        st_dev = torch.zeros(1, dtype=torch.int32, device=dev)
        gstream = torch.cuda.Stream(dev)
        gstream.wait_stream(stream)
        sp = ctypes.c_void_p(gstream.cuda_stream)
        ptrs = [ctypes.c_void_p(x.data_ptr()) for x in (dev_in[0],) + tuple(outs)]
        g = rg.rlu_graph_capture_dense(h.h, ptrs[0], dev_in[0].stride(0), rg._dtype_code(dev_in[0]), *ptrs[1:],
                                       ctypes.c_void_p(st_dev.data_ptr()), sp)
        for _ in range(args.warmup):
            rg.rlu_graph_launch(g, sp)
        gev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        gstream.synchronize()
        gev[0].record(gstream)
        for i in range(args.steps):
            rg.rlu_graph_launch(g, sp)
            gev[i + 1].record(gstream)
        gstream.synchronize()
        gms = [gev[i].elapsed_time(gev[i + 1]) for i in range(args.steps)]
        gtot = gev[0].elapsed_time(gev[-1])
        graph = {"value": args.steps / (gtot / 1e3), "unit": UNIT, "ms_per_step": gtot / args.steps,
                 "latency_ms": {"p50": statistics.median(gms), "p99": float(np.percentile(gms, 99))},
                 "status": int(st_dev.item())}
        rg.rlu_graph_destroy(g)
        stream.wait_stream(gstream)

    # per-stage device times (events on the same stream between the stages)
    h.debug_timing(True)
    stage_acc = {}
    panel_ms = 0.0
    reps = min(args.steps, 10)
    for _ in range(reps):
        factor()
        for kname, v in h.debug_stage_ms().items():
            stage_acc[kname] = stage_acc.get(kname, 0.0) + v / reps
        panel_width, panel_launches, pms = h.debug_lu_panels(0)
        panel_ms += pms / reps
    h.debug_timing(False)

    # end to end through the public API with pinned host buffers: H2D of the
    # input, the factorization, D2H of L, U, p, q, every step
    od = torch.float64 if prec == "f64" else torch.float32
    oh = (torch.empty((m, k), dtype=od).pin_memory(), torch.empty((k, n), dtype=od).pin_memory(),
          torch.empty(m, dtype=torch.int64).pin_memory(), torch.empty(n, dtype=torch.int64).pin_memory())
    if kind == "csr":
        host_in = tuple(torch.from_numpy(x).pin_memory() for x in (rowptr_np, colind_np, val_np))
        dev_stage = tuple(torch.empty_like(x, device=dev) for x in host_in)

        def e2e_step():
            for dst, src in zip(dev_stage, host_in):
                dst.copy_(src, non_blocking=True)
            f = h.factor_csr(*dev_stage, out=outs)
            for dst, src in zip(oh, (f.L, f.U, f.p, f.q)):
                dst.copy_(src, non_blocking=True)
            torch.cuda.current_stream(dev).synchronize()
    else:
        A_host = torch.from_numpy(A_np).to(tdt).pin_memory()

        def e2e_step():
            h.factor_host(A_host, oh)
    for _ in range(2):
        e2e_step()
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_serial = world * e2e_steps / e2e_s

    # the same end-to-end steps with two requests in flight: a second handle on
    # its own stream, each driven by one host thread, so one request's copies
    # overlap the other's factorization (every step still copies its input in
    # and its factors out inside the timed region)
    h2 = rg.RandLU(m, n, k, l, l1, w.sketch_seed + rank, prec=prec)
    if second:
        h2.set_second_sketch(second["k2"], second["l2"], second["seed2"])
    slots = []
    for hh in (h, h2):
        s_ = torch.cuda.Stream(dev)
        oh_ = tuple(torch.empty_like(x).pin_memory() for x in oh)
        if kind == "csr":
            stage_ = tuple(torch.empty_like(x, device=dev) for x in host_in)
            out_ = hh.alloc_outputs(dev)
        else:
            stage_, out_ = None, None
        slots.append((hh, s_, oh_, stage_, out_))

    def slot_step(slot):
        hh, s_, oh_, stage_, out_ = slot
        if kind == "csr":
            with torch.cuda.stream(s_):
                for dst, src in zip(stage_, host_in):
                    dst.copy_(src, non_blocking=True)
                f = hh.factor_csr(*stage_, out=out_, stream=s_)
                for dst, src in zip(oh_, (f.L, f.U, f.p, f.q)):
                    dst.copy_(src, non_blocking=True)
            s_.synchronize()
        else:
            hh.factor_host(A_host, oh_, stream=s_)

    def run_slot(slot, count):
        torch.cuda.set_device(dev)
        for _ in range(count):
            slot_step(slot)

    from concurrent.futures import ThreadPoolExecutor
    pipe_steps = 4 * e2e_steps  # a longer window: two host threads make this figure noisier
    with ThreadPoolExecutor(2) as ex:
        list(ex.map(lambda sl: run_slot(sl, 1), slots))  # warm the second handle
        barrier()
        t0 = time.perf_counter()
        list(ex.map(lambda sl: run_slot(sl, pipe_steps // 2), slots))
        torch.cuda.synchronize()
        pipe_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([pipe_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        pipe_s = float(t.item())
    e2e_value = world * pipe_steps / pipe_s
    h2.close()
    h2d = a_bytes
    d2h = (8 if prec == "f64" else 4) * (m * k + k * n) + 8 * (m + n)

    # the GPU factors' relative error, and the oracle's (same device routine)
    resid = device_rel_error(kind, dev_in, m, n, *outs)
    f64_peak, f64_peak_kind = fp64_peak(rg)

    if rank == 0:
        peaks, peak_kind = measured_peaks()
        works = stage_work(kind, w, a_bytes, nnz, prec)
        dom = max(stage_acc, key=stage_acc.get)
        roof = {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": MEASURED_TRAFFIC.get((args.workload, dom)) if prec == prec_default else None}
        if dom == "panel_lu":
            # the dominant kernel: the pivoted-LU kernel's launches in the LU of
            # Y, per launch (their own FP64 work over their own event times)
            works["panel_lu"] = (algorithmic_flops_lu_panels(m, l, panel_width) / panel_launches,
                                 "fp64_flops", "alu")
            roof.update(kernel="k_pivoted_lu<double> (LU of Y: %d launch%s, panel width %s)"
                        % (panel_launches, "es" if panel_launches > 1 else "", panel_width or "l, unblocked"),
                        launches=panel_launches, stage_ms=stage_acc[dom],
                        note="achieved = the launch's algorithmic FP64 flop / its mean CUDA-event time; the "
                             "blocked form's trailing updates run on the tensor cores in other kernels")
        if dom in works:
            amount, unit, bound = works[dom]
            secs = stage_acc[dom] / 1e3
            if dom == "panel_lu":
                secs = panel_ms / panel_launches / 1e3
            if bound == "hbm":
                ach = amount / secs / 1e9
                roof.update(bound="hbm", achieved=ach, peak=peaks["hbm_gbs"], unit="GB/s",
                            frac=ach / peaks["hbm_gbs"], peak_kind=peak_kind)
            elif unit == "fp64_flops":
                ach = amount / secs / 1e12
                roof.update(bound="alu", achieved=ach, peak=f64_peak, unit="TFLOP/s", frac=ach / f64_peak,
                            peak_kind=f64_peak_kind)
            else:
                ach = amount / secs / 1e12
                roof.update(bound="tensor", achieved=ach, peak=peaks["bf16_tflops"], unit="TFLOP/s",
                            frac=ach / peaks["bf16_tflops"], peak_kind=peak_kind)
        cpu, e_oracle = None, None
        if not args.no_cpu_baseline and world == 1:
            cpu, ores = cpu_baseline(args, w, A_np, second)
            of = (torch.from_numpy(ores.L).to(dev), torch.from_numpy(ores.U).to(dev),
                  torch.from_numpy(ores.p).to(dev), torch.from_numpy(ores.q).to(dev))
            e_oracle = device_rel_error(kind, dev_in, m, n, *of)
            del of
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"f64": "f64", "f32": "f32+f64", "bf16": "bf16+f32+f64", "bf16_refine": "bf16+f32+f64"}[prec],
            "data": "synthetic",
            "config": {"workload": args.workload, "m": m, "n": n, "k": k, "l": l, "l1": l1, "A_dtype": w.dtype,
                       "precision": prec, "nnz": nnz,
                       "B": ("second projection (Algorithm 1 steps 4-6), k2=%d l2=%d" % (second["k2"], second["l2"])
                             if second else "exact pseudo-inverse L_y^+ (Corollary 3.3)"),
                       "l2": "inputs larger than L2 (A %.0f MB > 129 MB L2)" % (a_bytes / 1e6)
                       if a_bytes > 135e6 else "inputs smaller than L2 (latency-bound workload)",
                       "parallelism": "independent problems per GPU" if world > 1 else "single GPU"},
            "latency_ms": {"p50": statistics.median(step_ms), "p99": float(np.percentile(step_ms, 99))},
            "graph_replay": graph,
            "a_read_gbs": 2.0 * a_bytes / (total_ms / args.steps / 1e3) / 1e9,
            "a_read_frac_of_hbm": 2.0 * a_bytes / (total_ms / args.steps / 1e3) / 1e9 / peaks["hbm_gbs"],
            "stage_ms": stage_acc,
            "roofline": roof,
            "rel_error": resid,
            "e_oracle": e_oracle,
            "rel_error_over_oracle": (resid / e_oracle) if e_oracle else None,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "mode": "pinned host input copied in and factors copied out every step; two requests in "
                            "flight (two handles, streams and host threads)",
                    "one_at_a_time": e2e_serial},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def serving_requests(specs, device, base_count=8, base_size=16384):
    """Requests of the trace with inputs made on `device` (see rlu_inputs.serving)."""
    from paper_1601_04280_gb300 import serving
    from rlu_inputs import serving as rs
    used = sorted({s.data_seed % base_count for s in specs if s.kind == "dense"})
    base = [None] * base_count
    for b in used:
        base[b] = rs.dense_base_pool(1, base_size, device, seed=3000 + b)[0]
    out = []
    for s in specs:
        r = serving.Request(s.rid, s.m, s.n, s.k, s.l, s.l1, rs.SKETCH_SEED)
        if s.kind == "dense":
            r.A = base[s.data_seed % base_count][: s.m, : s.n]
        else:
            r.csr = rs.csr_request(s, device)
        out.append(r)
    return out


def request_input_bytes(r):
    if r.csr is not None:
        return 8 * (r.m + 1) + sum(t.element_size() * t.numel() for t in r.csr[1:])
    return r.A.element_size() * r.m * r.n


def oracle_request_seconds(r):
    import scipy.sparse

    import oracle
    if r.csr is not None:
        rowptr, colind, val = (t.cpu().numpy() for t in r.csr)
        A = scipy.sparse.csr_matrix((val.astype(np.float64), colind, rowptr), shape=(r.m, r.n))
    else:
        A = r.A.cpu().double().numpy()
    t0 = time.perf_counter()
    oracle.factor(A, r.k, r.l, r.l1, r.seed)
    return time.perf_counter() - t0


def oracle_sample(reqs, budget_s):
    """Oracle factorizations of the trace's requests in order until budget_s of CPU time."""
    done, tot = 0, 0.0
    for r in reqs:
        tot += oracle_request_seconds(r)
        done += 1
        if tot >= budget_s:
            break
    return done, tot


def run_serving(args, rank, world, local):
    """Serving form: slots x streams over one device pool, a 4096-request trace.

    value = requests / makespan with every request waiting at time 0 (the
    saturation throughput); then the same trace with Poisson arrivals at 0.5x
    and 0.9x of that rate (p50/p99 latency from arrival to factors ready), and
    one request at a time (a single slot) as the baseline.  Times are host
    wall-clock around the run: a request is done when its status is back.
    """
    import torch
    import torch.distributed as dist

    import paper_1601_04280_gb300 as rg
    from paper_1601_04280_gb300 import serving
    from rlu_inputs import serving as rs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    rg.load()
    specs = rs.make_trace(args.requests, seed=rs.SKETCH_SEED + rank)
    reqs = serving_requests(specs, dev)
    torch.cuda.synchronize()
    pool_bytes = int(args.pool_gb * 2 ** 30)
    nwarm = max(3, args.warmup) * args.slots
    warm = [serving.Request(10 ** 6 + i, r.m, r.n, r.k, r.l, r.l1, r.seed, A=r.A, csr=r.csr)
            for i, r in enumerate(reqs[:nwarm])]
    a_read = sum(2.0 * request_input_bytes(r) for r in reqs)

    def barrier():
        if world > 1:
            dist.barrier()

    def set_arrivals(rate):
        t = 0.0
        for r, s in zip(reqs, specs):
            t += s.gap / rate
            r.t_arrive = t

    coop = None if args.coop_ctas < 0 else args.coop_ctas
    with serving.Server(pool_bytes, slots=args.slots, coop_ctas=coop) as srv:
        srv.run(warm, open_loop=False)
        torch.cuda.synchronize()
        l0 = rg.rlu_debug_launch_count()
        barrier()
        with ClockSampler(local) as clk:
            res_sat, span_sat = srv.run(reqs, open_loop=False)
        barrier()
        launches = rg.rlu_debug_launch_count() - l0
        span_max = span_sat
        if world > 1:
            t = torch.tensor([span_sat], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            span_max = float(t.item())
        sat = len(reqs) / span_sat
        runs = {"saturation": serving.summarize(res_sat, span_sat)}
    # the same trace with dense requests served from captured graphs per size
    # bucket (m, n rounded up to the bucket ladder, zero-padded; a bucket's
    # graph is captured the second time its key comes)
    with serving.Server(pool_bytes, slots=args.slots, coop_ctas=coop, graphs=True, graph_min_uses=2) as gsrv:
        gsrv.run(warm, open_loop=False)
        res_g, span_g = gsrv.run(reqs, open_loop=False)
        runs["saturation_graph_buckets"] = dict(serving.summarize(res_g, span_g), **gsrv.graph_stats,
                                                buckets_cached=len(gsrv.buckets))
    with serving.Server(pool_bytes, slots=args.slots, coop_ctas=coop) as srv:
        srv.run(warm, open_loop=False)
        for frac in (0.5, 0.9):
            set_arrivals(frac * sat)
            res, span = srv.run(reqs, open_loop=True)
            runs["open_loop_%.1fx" % frac] = dict(serving.summarize(res, span), arrival_rate=frac * sat)
    with serving.Server(pool_bytes, slots=1, coop_ctas=0) as one:
        one.run(warm[:3], open_loop=False)
        res_one, span_one = one.run(reqs, open_loop=False)
        s1 = serving.summarize(res_one, span_one)
        svc = np.array([r.t_done - r.t_admit for r in res_one]) * 1e3
        s1.update(service_p50_ms=float(np.percentile(svc, 50)), service_p99_ms=float(np.percentile(svc, 99)))
        runs["one_at_a_time"] = s1
    failed = [r.rid for r in res_sat if r.status not in (rg.RLU_OK, rg.RLU_WRANK)]

    # end to end: the first requests arrive from page-locked host memory and
    # their L, U, p, q and status go back to page-locked host memory
    sub = reqs[: args.e2e_requests]
    host_base = {}
    hreqs = []
    for r in sub:
        q = serving.Request(r.rid, r.m, r.n, r.k, r.l, r.l1, r.seed)
        if r.csr is not None:
            q.csr = tuple(t.cpu().pin_memory() for t in r.csr)
        else:
            b = r.A.data_ptr()
            if b not in host_base:
                host_base[b] = r.A.as_strided((16384, 16384), (16384, 1)).cpu().pin_memory()
            q.A = host_base[b][: r.m, : r.n]
        hreqs.append(q)
    with serving.Server(pool_bytes, slots=args.slots, return_host=(16384, 16384, 256, "f32"),
                        coop_ctas=coop) as srv:
        srv.run(hreqs[: args.slots], open_loop=False)
        barrier()
        res_e2e, span_e2e = srv.run(hreqs, open_loop=False)
        barrier()
    h2d = sum(request_input_bytes(r) for r in sub) / len(sub)
    d2h = sum(4 * (r.m * r.k + r.k * r.n) + 8 * (r.m + r.n) + 4 for r in sub) / len(sub)
    e2e_value = len(hreqs) / span_e2e
    if world > 1:
        t = torch.tensor([span_e2e], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_value = world * len(hreqs) / float(t.item())

    if rank == 0:
        peaks, peak_kind = measured_peaks()
        ach = a_read / span_sat / 1e9
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            done, secs = oracle_sample(reqs, 20.0)
            cpu = {"value": done / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "the first %d requests of the trace, one after another, by the FP64 oracle" % done}
        line = {
            "metric": METRIC, "value": world * len(reqs) / span_max, "unit": UNIT, "n_gpus": world,
            "steps": len(reqs), "warmup": len(warm), "ms_per_step": 1e3 * span_sat / len(reqs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": SERVING_WORKLOAD, "requests": len(reqs), "slots": args.slots,
                       "coop_ctas": srv.coop_ctas,
                       "pool_gib": args.pool_gb, "m_n": "log-uniform [512, 16384]", "k": "uniform [16, 256]",
                       "l": "k + 20", "l1": "8 k", "dense_share": rs.DENSE_SHARE, "csr_density": rs.CSR_DENSITY,
                       "dense_inputs": "leading blocks of 8 rank-96 16384^2 FP32 matrices, geometric spectrum",
                       "l2": "inputs larger than L2 for most requests (mean dense A %.0f MB)" % (
                           np.mean([request_input_bytes(r) for r in reqs if r.csr is None]) / 1e6),
                       "parallelism": "replicas (independent traces per GPU)" if world > 1 else "single GPU"},
            "timing": "host wall clock around each run; a request is done when its status is on the host",
            "serving": runs,
            "speedup_vs_one_at_a_time": sat / runs["one_at_a_time"]["factorizations_per_s"],
            "latency_ms": {"p50": runs["open_loop_0.9x"]["p50_ms"], "p99": runs["open_loop_0.9x"]["p99_ms"],
                           "at": "Poisson arrivals at 0.9x the saturation throughput"},
            "failed_requests": failed,
            "a_read_gbs": ach,
            "roofline": {"kernel": "whole serving run (all kernels)", "bound": "hbm", "achieved": ach,
                         "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": None,
                         "peak_kind": peak_kind,
                         "note": "achieved = two algorithmic reads of every request's A / makespan"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "requests": len(hreqs),
                    "mode": "host arrival: A (or CSR arrays) from page-locked host memory, factors back to it"},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_serving_reference(args, rank):
    """The oracle on the serving trace's requests, one after another (host cores)."""
    if rank != 0:
        return 0
    from rlu_inputs import serving as rs
    specs = rs.make_trace(args.requests, seed=rs.SKETCH_SEED)
    budget = 30.0
    # inputs made on the host with torch's CPU generator (same recipe as the GPU arm)
    sample = []
    tot, done = 0.0, 0
    for i in range(0, len(specs), 8):
        reqs = serving_requests(specs[i:i + 8], "cpu", base_count=8)
        for r in reqs:
            if done >= args.warmup + args.steps or tot >= budget:
                break
            secs = oracle_request_seconds(r)
            if done >= args.warmup:
                sample.append(secs)
                tot += secs
            done += 1
        if done >= args.warmup + args.steps or tot >= budget:
            break
    value = len(sample) / sum(sample)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(sample), "warmup": args.warmup, "ms_per_step": 1e3 * sum(sample) / len(sample),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": SERVING_WORKLOAD, "requests": args.requests},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "%d requests of the trace in order, after %d warm-up, by the FP64 oracle"
                                   % (len(sample), args.warmup)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
