"""Benchmark of the sparse randomized LU path on GB300.

One step = one whole factorization (sketch parameters, CountSketch + Hartley
sketch, FP64 panel LU, L_y^+ and B = L_y^+ P A, LU of B, assembly of L, U, p, q)
of the dense FP32 8192 x 8192 workload: A = G1 G2 + 1e-6 N(0,1), G1 8192 x 200,
G2 200 x 8192 Gaussian, k = 200, l = 220, l1 = 1600.  A is 268 MB, larger than
the 129 MB L2, so consecutive steps do not hit in L2 for A.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun (N > 1) each rank factors its
own matrix (independent problems: weak scaling, no data-path collective); the
timed region is bracketed by barriers and the max over ranks is reported.
The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores on the same workload (rank 0 only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "dense_f32_8192x8192_k200"
METRIC = "rand-LU factorizations/s"
UNIT = "factorizations/s"


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


def make_input():
    import rlu_inputs as ri
    return ri.DENSE_F32_8K, ri.make_dense(ri.DENSE_F32_8K)


def oracle_factor_seconds(w, A):
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    oracle.factor(A.astype(np.float64), w.k, w.l, w.l1, w.sketch_seed)
    return time.perf_counter() - t0


def algorithmic_flops_panel_lu(m, l):
    # sum_j 2 (m - j - 1)(l - j - 1) + (m - j - 1) divisions, FP64
    return sum(2.0 * (m - j - 1) * (l - j - 1) + (m - j - 1) for j in range(l))


def run_reference(args, rank):
    import numpy as np
    if rank != 0:
        return 0
    w, A = make_input()
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
        "config": {"workload": WORKLOAD, "m": w.m, "n": w.n, "k": w.k, "l": w.l, "l1": w.l1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d full factorizations of the workload by the FP64 oracle" % args.steps},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1601_04280_gb300 as rg

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    rg.load()

    w, A_np = make_input()
    m, n, k, l, l1 = w.m, w.n, w.k, w.l, w.l1
    dev = torch.device("cuda", local)
    A = torch.from_numpy(A_np).to(dev)
    h = rg.RandLU(m, n, k, l, l1, w.sketch_seed + rank, prec="f32")
    outs = h.alloc_outputs(dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up
    for _ in range(args.warmup):
        h.factor(A, out=outs)
    torch.cuda.synchronize()

    # device-timed region: K factorizations, per-step events for p50/p99
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    launches0 = rg.rlu_debug_launch_count()
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for i in range(args.steps):
            h.factor(A, out=outs)
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

    # per-stage device times (stage events on the same stream), dominant kernel
    h.debug_timing(True)
    stage_acc = {}
    reps = min(args.steps, 10)
    for _ in range(reps):
        h.factor(A, out=outs)
        for kname, v in h.debug_stage_ms().items():
            stage_acc[kname] = stage_acc.get(kname, 0.0) + v / reps
    h.debug_timing(False)

    # end to end through the host-buffer entry point (pinned host memory)
    A_host = torch.from_numpy(A_np).pin_memory()
    oh = (torch.empty((m, k)).pin_memory(), torch.empty((k, n)).pin_memory(),
          torch.empty(m, dtype=torch.int64).pin_memory(), torch.empty(n, dtype=torch.int64).pin_memory())
    for _ in range(2):
        h.factor_host(A_host, oh)
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        h.factor_host(A_host, oh)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * e2e_steps / e2e_s

    # accuracy of the timed configuration against the oracle's error: computed
    # by the parity tests; here only the GPU's own residual is reported
    L, U, p, q = (x.double() if x.is_floating_point() else x for x in outs)
    Ad = A.double()
    resid = float(torch.linalg.norm(L @ U - Ad[p][:, q]) / torch.linalg.norm(Ad))

    if rank == 0:
        peaks, peak_kind = measured_peaks()
        dom = max(stage_acc, key=stage_acc.get)
        stage_flops = {"panel_lu": algorithmic_flops_panel_lu(m, l),
                       "gram": float(m) * k * (k + 1),
                       "wform": 2.0 * k * k * k + 2.0 * k * k * m,
                       "bgemm": 2.0 * k * m * n}
        a_bytes = A.element_size() * m * n
        roof = None
        if dom in ("panel_lu", "gram", "wform"):
            ach = stage_flops[dom] / (stage_acc[dom] / 1e3) / 1e12
            roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                    "peak_kind": "FP64 vector peak derived from unit counts and the 2.07 GHz max clock"}
        elif dom == "sketch":
            ach = a_bytes / (stage_acc[dom] / 1e3) / 1e9
            roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_kind": peak_kind}
        else:
            ach = stage_flops.get(dom, 0.0) / (stage_acc[dom] / 1e3) / 1e12
            roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": 74.4, "unit": "TFLOP/s",
                    "frac": ach / 74.4, "traffic": None, "peak_kind": "FP32 FFMA measured by probe"}
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            secs = oracle_factor_seconds(w, A_np)
            cpu = {"value": 1.0 / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "one full factorization of the workload by the FP64 oracle (numpy/scipy)"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "m": m, "n": n, "k": k, "l": l, "l1": l1, "A_dtype": "f32",
                       "l2": "inputs larger than L2 (A = 268 MB > 129 MB L2)",
                       "parallelism": "independent problems per GPU" if world > 1 else "single GPU"},
            "latency_ms": {"p50": statistics.median(step_ms), "p99": float(np.percentile(step_ms, 99))},
            "a_read_gbs": 2.0 * a_bytes / (total_ms / args.steps / 1e3) / 1e9,
            "a_read_frac_of_hbm": 2.0 * a_bytes / (total_ms / args.steps / 1e3) / 1e9 / peaks["hbm_gbs"],
            "stage_ms": stage_acc,
            "roofline": roof,
            "rel_error": resid,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": a_bytes,
                    "d2h_bytes_per_step": 4 * (m * k + k * n) + 8 * (m + n)},
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
