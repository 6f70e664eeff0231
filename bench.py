"""Benchmark of the sparse randomized LU path on GB300.

One step = one whole factorization (sketch parameters, CountSketch + Hartley
sketch, FP64 panel LU, L_y^+ and B = L_y^+ P A, LU of B, assembly of L, U, p, q).
Default workload: dense FP32 8192 x 8192, A = G1 G2 + 1e-6 N(0,1), G1 8192 x 200,
G2 200 x 8192 Gaussian, k = 200, l = 220, l1 = 1600.  A is 268 MB, larger than
the 129 MB L2, so consecutive steps do not hit in L2 for A.  Other workloads
(--workload): dense FP64 1024 x 1024 (k = 20), CSR FP32 200000 x 50000 (k = 100),
dense BF16 32768 x 16384 (k = 500; --prec bf16_refine | bf16 | f32).

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
DEFAULT_WORKLOAD = "dense_f32_8192x8192_k200"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 vector peak: 152 SMs x 2 FP64 FMA/clk/SM (1/64 of the 128 FP32 FMA/clk/SM)
# x 2 flop x 2.07 GHz max clock = 1.259 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


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


def oracle_factor_seconds(w, A):
    import oracle
    Ao = oracle_input(w, A)
    t0 = time.perf_counter()
    oracle.factor(Ao, w.k, w.l, w.l1, w.sketch_seed)
    return time.perf_counter() - t0


def algorithmic_flops_panel_lu(m, l):
    # sum_j 2 (m - j - 1)(l - j - 1) + (m - j - 1) divisions, FP64
    return sum(2.0 * (m - j - 1) * (l - j - 1) + (m - j - 1) for j in range(l))


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


def stage_work(kind, w, a_bytes, nnz):
    """Algorithmic work of each stage for one factorization: (amount, unit, bound)."""
    m, n, k, l = w.m, w.n, w.k, w.l
    return {
        "sketch": (a_bytes, "bytes", "hbm"),
        "panel_lu": (algorithmic_flops_panel_lu(m, l), "fp64_flops", "alu"),
        "bgemm": ((2.0 * k * nnz) if kind == "csr" else (2.0 * k * m * n), "flops", "tensor"),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default=None, help="override the workload's precision (f64, f32, bf16, bf16_refine)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

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

    # per-stage device times (events on the same stream between the stages)
    h.debug_timing(True)
    stage_acc = {}
    reps = min(args.steps, 10)
    for _ in range(reps):
        factor()
        for kname, v in h.debug_stage_ms().items():
            stage_acc[kname] = stage_acc.get(kname, 0.0) + v / reps
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
    e2e_value = world * e2e_steps / e2e_s
    h2d = a_bytes
    d2h = (8 if prec == "f64" else 4) * (m * k + k * n) + 8 * (m + n)

    # the GPU factors' own relative error (the parity tests compare it with the oracle's)
    L, U, p, q = (x.double() if x.is_floating_point() else x for x in outs)
    if kind == "csr":
        resid = None
    else:
        Ad = dev_in[0].double()
        resid = float(torch.linalg.norm(L @ U - Ad[p][:, q]) / torch.linalg.norm(Ad))
        del Ad

    if rank == 0:
        peaks, peak_kind = measured_peaks()
        works = stage_work(kind, w, a_bytes, nnz)
        dom = max(stage_acc, key=stage_acc.get)
        roof = {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None}
        if dom in works:
            amount, unit, bound = works[dom]
            secs = stage_acc[dom] / 1e3
            if bound == "hbm":
                ach = amount / secs / 1e9
                roof.update(bound="hbm", achieved=ach, peak=peaks["hbm_gbs"], unit="GB/s",
                            frac=ach / peaks["hbm_gbs"], peak_kind=peak_kind)
            elif unit == "fp64_flops":
                ach = amount / secs / 1e12
                roof.update(bound="alu", achieved=ach, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                            frac=ach / FP64_PEAK_TFLOPS,
                            peak_kind="FP64 vector peak from unit counts: 152 SM x 2 FMA/clk x 2 x 2.07 GHz")
            else:
                ach = amount / secs / 1e12
                roof.update(bound="tensor", achieved=ach, peak=peaks["bf16_tflops"], unit="TFLOP/s",
                            frac=ach / peaks["bf16_tflops"], peak_kind=peak_kind)
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            secs = oracle_factor_seconds(w, A_np)
            cpu = {"value": 1.0 / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "one full factorization of the workload by the FP64 oracle (numpy/scipy)"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"f64": "f64", "f32": "f32+f64", "bf16": "bf16+f32+f64", "bf16_refine": "bf16+f32+f64"}[prec],
            "data": "synthetic",
            "config": {"workload": args.workload, "m": m, "n": n, "k": k, "l": l, "l1": l1, "A_dtype": w.dtype,
                       "precision": prec, "nnz": nnz,
                       "l2": "inputs larger than L2 (A %.0f MB > 129 MB L2)" % (a_bytes / 1e6)
                       if a_bytes > 135e6 else "inputs smaller than L2 (latency-bound workload)",
                       "parallelism": "independent problems per GPU" if world > 1 else "single GPU"},
            "latency_ms": {"p50": statistics.median(step_ms), "p99": float(np.percentile(step_ms, 99))},
            "a_read_gbs": 2.0 * a_bytes / (total_ms / args.steps / 1e3) / 1e9,
            "a_read_frac_of_hbm": 2.0 * a_bytes / (total_ms / args.steps / 1e3) / 1e9 / peaks["hbm_gbs"],
            "stage_ms": stage_acc,
            "roofline": roof,
            "rel_error": resid,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
