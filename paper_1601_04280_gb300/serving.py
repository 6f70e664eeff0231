"""Continuous-batching serving loop for randomized LU factorizations (one GPU).

Requests (dense or CSR A resident on the device, each with its own m, n, k,
l, l1) arrive on a trace.  The scheduler admits a waiting request as soon as
a slot is free and the request's HBM footprint fits in the free part of one
device pool.  The footprint is exact: the handle's workspace
(rlu_workspace_bytes), the caller-owned CSR scratch for its nnz
(rlu_csr_workspace_bytes), and the outputs L, U, p, q.  Each slot owns a CUDA
stream and a worker thread.  The worker builds the handle inside its carve of
the pool (rlu_create_in: no allocation, no device-wide synchronisation), runs
the factorization through the C-ABI (ctypes drops the GIL for the call, so
the workers' host work overlaps too), and hands the carve back when the
status word is in.  The kernels of all admitted requests therefore share the
GPU, and a request that arrives while others run starts as soon as a slot and
memory free up.

Every kernel's tiling, grid and reduction order depend only on the request's
own sizes and the SM count, never on what else is running, so a request's
factors are bit-for-bit the same alone and in the mix.

Dense requests can also be served from captured launch graphs per size
bucket (Server(graphs=True)): m and n are rounded up to a ladder of sizes
(bucket_dim), the request is copied into the bucket's zero-padded input
buffer, and one graph per (bucket sizes, k, l, l1, seed, precision) replays
the whole factorization.  Zero columns add exact zeros to every sum of the
sketch and to B, zero rows never win a pivot (ties go to the smaller
position), and padded positions are never swapped, so the first m rows of L,
the first n columns of U, p[:m] and q[:n] are the request's factors (up to
the rounding of sums whose splits depend on the padded sizes).  A bucket's
memory stays in the pool while it is cached and is evicted, least recently
used first, when admission needs the room.  GraphBucket serves one exact
size outside the server.

This module is host-side orchestration only: every step of every
factorization runs in the library's kernels.
"""
import collections
import ctypes
import math
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import (PREC, RLU_BF16, RLU_F32, RLU_F64, RLU_OK, RLU_WRANK, load, rlu_copy_block_async, rlu_create_in,
               rlu_csr_workspace_bytes, rlu_destroy, rlu_graph_capture_dense, rlu_graph_destroy, rlu_graph_launch,
               rlu_set_csr_workspace, rlu_set_max_ctas, rlu_set_precision, rlu_workspace_bytes)

_ALIGN = 256


def _up(x, a=_ALIGN):
    return (x + a - 1) // a * a


@dataclass
class Request:
    """One factorization request.  `A` is a device tensor (dense, unit column
    stride) or None; `csr` is (rowptr int64, colind int32, val) on the device."""
    rid: int
    m: int
    n: int
    k: int
    l: int
    l1: int
    seed: int
    t_arrive: float = 0.0
    A: object = None
    csr: tuple = None
    prec: str = "f32"

    @property
    def kind(self):
        return "csr" if self.csr is not None else "dense"


@dataclass
class Result:
    rid: int
    status: int
    t_arrive: float
    t_admit: float
    t_done: float
    slot: int
    footprint: int
    outputs: tuple = None          # (L, U, p, q) on the host when kept

    @property
    def latency(self):
        return self.t_done - self.t_arrive


class DevicePool:
    """First-fit allocator over one device buffer, in 256-byte granules, with
    coalescing of neighbouring free ranges.  Host bookkeeping only."""

    def __init__(self, nbytes, device="cuda"):
        import torch
        self.nbytes = _up(int(nbytes))
        raw = torch.empty(self.nbytes + _ALIGN, dtype=torch.uint8, device=device)
        shift = (-raw.data_ptr()) % _ALIGN
        self.buf = raw[shift: shift + self.nbytes]
        self.base = self.buf.data_ptr()
        assert self.base % _ALIGN == 0
        self.free_ranges = [(0, self.nbytes)]   # sorted (offset, size)
        self.in_use = 0

    def alloc(self, nbytes):
        nbytes = _up(nbytes)
        for i, (off, size) in enumerate(self.free_ranges):
            if size >= nbytes:
                if size == nbytes:
                    del self.free_ranges[i]
                else:
                    self.free_ranges[i] = (off + nbytes, size - nbytes)
                self.in_use += nbytes
                return off
        return None

    def free(self, off, nbytes):
        nbytes = _up(nbytes)
        fr = self.free_ranges
        i = 0
        while i < len(fr) and fr[i][0] < off:
            i += 1
        fr.insert(i, (off, nbytes))
        # merge with the right, then the left neighbour
        if i + 1 < len(fr) and fr[i][0] + fr[i][1] == fr[i + 1][0]:
            fr[i] = (fr[i][0], fr[i][1] + fr[i + 1][1])
            del fr[i + 1]
        if i > 0 and fr[i - 1][0] + fr[i - 1][1] == fr[i][0]:
            fr[i - 1] = (fr[i - 1][0], fr[i - 1][1] + fr[i][1])
            del fr[i]
        self.in_use -= nbytes

    def tensor(self, off, shape, dtype):
        import torch
        count = int(np.prod(shape))
        esz = torch.empty((), dtype=dtype).element_size()
        return self.buf[off: off + count * esz].view(dtype).view(*shape)


def _out_dtype(prec):
    import torch
    return torch.float64 if prec == "f64" else torch.float32


def _dtype_code(t):
    import torch
    return {torch.float64: RLU_F64, torch.float32: RLU_F32, torch.bfloat16: RLU_BF16}[t.dtype]


@dataclass
class Carve:
    """Offsets of one request's pieces inside the pool."""
    off: int
    total: int
    parts: dict = field(default_factory=dict)   # name -> (offset, bytes)


def _on_host(t):
    return t is not None and not t.is_cuda


def plan_carve(req):
    """The request's pieces and their sizes (bytes), in pool order.  A request
    whose input sits in host memory also holds a device copy of it."""
    esz = 8 if req.prec == "f64" else 4
    parts = [("ws", rlu_workspace_bytes(req.m, req.n, req.k, req.l, req.l1, req.prec))]
    if req.csr is not None:
        rowptr, colind, val = req.csr
        parts.append(("csr_ws", rlu_csr_workspace_bytes(req.m, req.n, req.k, int(val.numel()))))
        if _on_host(val):
            parts += [("rowptr", 8 * (req.m + 1)), ("colind", 4 * int(colind.numel())),
                      ("val", val.element_size() * int(val.numel()))]
    elif _on_host(req.A):
        parts.append(("A", req.A.element_size() * req.m * req.n))
    parts += [("L", esz * req.m * req.k), ("U", esz * req.k * req.n), ("p", 8 * req.m), ("q", 8 * req.n),
              ("status", 4)]
    return parts


def footprint(req):
    """HBM bytes one request holds while admitted."""
    return sum(_up(b) for _, b in plan_carve(req))


def bucket_dim(x, lo=512):
    """Smallest value >= x of the ladder lo, lo sqrt 2, 2 lo, ... (each rounded
    up to a multiple of 64): zero padding to it costs at most 50 % per side."""
    i = 0
    while True:
        base = lo << (i // 2)  # powers of two exactly; the half steps rounded up
        b = base if i % 2 == 0 else int(math.ceil(base * math.sqrt(2.0) / 64.0)) * 64
        if b >= x:
            return b
        i += 1


def bucket_key(req):
    """Graph bucket of a dense request whose A is on the device, or None."""
    if req.csr is not None or req.A is None or _on_host(req.A):
        return None
    return (bucket_dim(req.m), bucket_dim(req.n), req.k, req.l, req.l1, req.seed, req.prec, str(req.A.dtype))


def plan_outputs(req):
    """The pieces of a request served from a graph bucket: its outputs only."""
    esz = 8 if req.prec == "f64" else 4
    return [("L", esz * req.m * req.k), ("U", esz * req.k * req.n), ("p", 8 * req.m), ("q", 8 * req.n),
            ("status", 4)]


def plan_bucket(key):
    """Pool pieces of one graph bucket: handle workspace, padded input, outputs."""
    mb, nb, k, l, l1, seed, prec, dt = key
    esz_in = {"torch.float64": 8, "torch.float32": 4, "torch.bfloat16": 2}[dt]
    esz = 8 if prec == "f64" else 4
    return [("ws", rlu_workspace_bytes(mb, nb, k, l, l1, prec)), ("A", esz_in * mb * nb), ("L", esz * mb * k),
            ("U", esz * k * nb), ("p", 8 * mb), ("q", 8 * nb), ("status", 4)]


@dataclass
class _Bucket:
    key: tuple
    carve: object
    h: object = None
    graph: object = None
    busy: bool = False
    last_used: float = 0.0
    replays: int = 0


class Server:
    """Slots x (stream, worker thread) over one device pool."""

    def __init__(self, pool_bytes, slots=8, device="cuda", keep_outputs=False, max_bypass=None, return_host=None,
                 coop_ctas=None, graphs=False, graph_min_uses=2):
        """return_host: None, or (max_m, max_n, max_k, prec): every request's L, U,
        p, q and status are copied back into page-locked host buffers of the
        slot (sized for those maxima) before the request counts as done.
        coop_ctas: bound on the CTAs of each request's grid-synchronised kernels
        (rlu_set_max_ctas; 0 = one per SM; None = a quarter of the SMs, so that
        several requests' eliminations run side by side).
        graphs: serve dense device requests from captured launch graphs per
        size bucket; a bucket is built (and its graph captured) when its key
        has come graph_min_uses times, and replayed from then on."""
        import torch
        load()
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.pool = DevicePool(pool_bytes, device)
        self.nslots = slots
        if coop_ctas is None:
            sms = torch.cuda.get_device_properties(self.device).multi_processor_count \
                if self.device.type == "cuda" else 0
            coop_ctas = max(1, sms // 4) if sms else 0
        self.coop_ctas = int(coop_ctas)
        self.keep_outputs = keep_outputs
        self.max_bypass = max_bypass if max_bypass is not None else 4 * slots
        cuda = self.device.type == "cuda"
        self.streams = [torch.cuda.Stream(device=self.device) if cuda else None for _ in range(slots)]
        self.jobs = [queue.Queue() for _ in range(slots)]
        self.done = queue.Queue()
        self.host_out = None
        if return_host is not None:
            mm, mn, mk, prec = return_host
            odt = _out_dtype(prec)
            self.host_out = [(torch.empty(mm * mk, dtype=odt, pin_memory=True),
                              torch.empty(mk * mn, dtype=odt, pin_memory=True),
                              torch.empty(mm, dtype=torch.int64, pin_memory=True),
                              torch.empty(mn, dtype=torch.int64, pin_memory=True),
                              torch.zeros(1, dtype=torch.int32, pin_memory=True)) for _ in range(slots)]
        self.graphs = bool(graphs) and self.device.type == "cuda"
        self.graph_min_uses = max(1, int(graph_min_uses))
        self.buckets = {}
        self.key_seen = collections.Counter()
        self.graph_stats = {"replays": 0, "captures": 0, "evictions": 0, "eager": 0}
        self.status_host = [torch.zeros(1, dtype=torch.int32, pin_memory=True) for _ in range(slots)] \
            if cuda else [None] * slots
        self.worker_error = None
        self.threads = [threading.Thread(target=self._worker, args=(s,), daemon=True) for s in range(slots)]
        for t in self.threads:
            t.start()

    # ---- worker side ----------------------------------------------------------
    def _worker(self, s):
        import torch
        stream = self.streams[s]
        sptr = None
        try:
            if stream is not None:
                torch.cuda.set_device(self.device.index)
                sptr = ctypes.c_void_p(stream.cuda_stream)
        except Exception as e:  # the scheduler sees a dead worker and raises
            self.worker_error = repr(e)
            return
        while True:
            job = self.jobs[s].get()
            if job is None:
                return
            req, carve, t0, bucket, ready = job
            try:
                if ready is not None:
                    # device inputs made on the caller's stream are complete
                    # before this slot's stream reads them
                    stream.wait_event(ready)
                if bucket is not None:
                    status, outputs = self._execute_bucket(req, carve, bucket, stream, sptr, s)
                else:
                    status, outputs = self._execute(req, carve, stream, sptr, s)
            except Exception as e:  # reported as a failed request, the loop goes on
                status, outputs = -1, repr(e)
            self.done.put((s, req, carve, status, time.perf_counter() - t0, outputs, bucket))

    def _execute(self, req, carve, stream, sptr, slot=0):
        import torch
        lib = load()
        P = carve.parts
        pool = self.pool
        ptr = lambda name: ctypes.c_void_p(pool.base + P[name][0])  # noqa: E731
        vptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731

        def upload(name, t):   # host tensor (rows with unit column stride) -> its carve
            rows, width = (t.shape[0], t.shape[1]) if t.dim() == 2 else (1, t.numel())
            pitch = t.stride(0) if t.dim() == 2 else width
            esz = t.element_size()
            rlu_copy_block_async(ptr(name), width * esz, vptr(t), pitch * esz, width * esz, rows, sptr)

        hout = self.host_out[slot] if self.host_out is not None else None
        h = rlu_create_in(req.m, req.n, req.k, req.l, req.l1, req.seed, ptr("ws"), P["ws"][1], sptr)
        try:
            rlu_set_precision(h, PREC[req.prec])
            if self.coop_ctas:
                rlu_set_max_ctas(h, self.coop_ctas)
            if req.csr is not None:
                rowptr, colind, val = req.csr
                nnz = int(val.numel())
                rlu_set_csr_workspace(h, nnz, ptr("csr_ws"), P["csr_ws"][1])
                if _on_host(val):
                    for name, t in (("rowptr", rowptr), ("colind", colind), ("val", val)):
                        upload(name, t)
                    rp, ci, va = ptr("rowptr"), ptr("colind"), ptr("val")
                else:
                    rp, ci, va = vptr(rowptr), vptr(colind), vptr(val)
                status = lib.rlu_factor_csr(h, rp, ci, va, nnz, _dtype_code(val), ptr("L"), ptr("U"), ptr("p"),
                                            ptr("q"), sptr)
                if hout is not None:
                    hout[4][0] = status
            else:
                A = req.A
                if _on_host(A):
                    upload("A", A)
                    a_ptr, lda = ptr("A"), req.n
                else:
                    a_ptr, lda = vptr(A), A.stride(0)
                if hout is None:
                    status = lib.rlu_factor_dense(h, a_ptr, lda, _dtype_code(A), ptr("L"), ptr("U"), ptr("p"),
                                                  ptr("q"), sptr)
                else:
                    status = lib.rlu_factor_dense_async(h, a_ptr, lda, _dtype_code(A), ptr("L"), ptr("U"), ptr("p"),
                                                        ptr("q"), ptr("status"), sptr)
                    if status == RLU_OK:
                        rlu_copy_block_async(vptr(hout[4]), 4, ptr("status"), 4, 4, 1, sptr)
            if hout is not None and status in (RLU_OK, RLU_WRANK):
                esz = 8 if req.prec == "f64" else 4
                for i, (name, nbytes) in enumerate((("L", esz * req.m * req.k), ("U", esz * req.k * req.n),
                                                    ("p", 8 * req.m), ("q", 8 * req.n))):
                    rlu_copy_block_async(vptr(hout[i]), nbytes, ptr(name), nbytes, nbytes, 1, sptr)
                stream.synchronize()
                status = int(hout[4][0])
        finally:
            rlu_destroy(h)
        outputs = None
        if self.keep_outputs:
            # page-locked copies (a copy into pageable memory would need this
            # thread inside the driver while other workers launch)
            odt = _out_dtype(req.prec)
            outputs = (torch.empty((req.m, req.k), dtype=odt, pin_memory=True),
                       torch.empty((req.k, req.n), dtype=odt, pin_memory=True),
                       torch.empty(req.m, dtype=torch.int64, pin_memory=True),
                       torch.empty(req.n, dtype=torch.int64, pin_memory=True))
            for t, name in zip(outputs, "LUpq"):
                nbytes = t.numel() * t.element_size()
                rlu_copy_block_async(vptr(t), nbytes, ptr(name), nbytes, nbytes, 1, sptr)
            stream.synchronize()
        return status, outputs

    def _execute_bucket(self, req, carve, bucket, stream, sptr, slot):
        """A dense request through its size bucket: copy A into the zero-padded
        bucket input, replay the bucket's graph (the first use runs eagerly and
        captures it), copy the request's part of the outputs to its carve."""
        import torch
        lib = load()
        mb, nb, k, l, l1, seed, prec, _ = bucket.key
        BP = bucket.carve.parts
        pool = self.pool
        bptr = lambda name: ctypes.c_void_p(pool.base + BP[name][0])  # noqa: E731
        ptr = lambda name: ctypes.c_void_p(pool.base + carve.parts[name][0])  # noqa: E731
        A = req.A
        esz_in = A.element_size()
        with torch.cuda.stream(stream):
            pool.tensor(BP["A"][0], (mb, nb), A.dtype).zero_()
        rlu_copy_block_async(bptr("A"), nb * esz_in, ctypes.c_void_p(A.data_ptr()), A.stride(0) * esz_in,
                             req.n * esz_in, req.m, sptr)
        code = _dtype_code(A)
        if bucket.h is None:
            bucket.h = rlu_create_in(mb, nb, k, l, l1, seed, bptr("ws"), BP["ws"][1], sptr)
            rlu_set_precision(bucket.h, PREC[prec])
            if self.coop_ctas:
                rlu_set_max_ctas(bucket.h, self.coop_ctas)
        if bucket.graph is None:
            status = lib.rlu_factor_dense(bucket.h, bptr("A"), nb, code, bptr("L"), bptr("U"), bptr("p"), bptr("q"),
                                          sptr)
            if status in (RLU_OK, RLU_WRANK):
                bucket.graph = rlu_graph_capture_dense(bucket.h, bptr("A"), nb, code, bptr("L"), bptr("U"),
                                                       bptr("p"), bptr("q"), bptr("status"), sptr)
                self.graph_stats["captures"] += 1
        else:
            rlu_graph_launch(bucket.graph, sptr)
            sh = self.status_host[slot]
            rlu_copy_block_async(ctypes.c_void_p(sh.data_ptr()), 4, bptr("status"), 4, 4, 1, sptr)
            stream.synchronize()
            status = int(sh[0])
            bucket.replays += 1
            self.graph_stats["replays"] += 1
        if status in (RLU_OK, RLU_WRANK):
            esz = 8 if prec == "f64" else 4
            # rows 0..m-1 of L and columns 0..n-1 of U, p[:m], q[:n]
            rlu_copy_block_async(ptr("L"), esz * req.m * k, bptr("L"), esz * req.m * k, esz * req.m * k, 1, sptr)
            rlu_copy_block_async(ptr("U"), esz * req.n, bptr("U"), esz * nb, esz * req.n, k, sptr)
            rlu_copy_block_async(ptr("p"), 8 * req.m, bptr("p"), 8 * req.m, 8 * req.m, 1, sptr)
            rlu_copy_block_async(ptr("q"), 8 * req.n, bptr("q"), 8 * req.n, 8 * req.n, 1, sptr)
        outputs = None
        if self.keep_outputs:
            odt = _out_dtype(req.prec)
            outputs = (torch.empty((req.m, req.k), dtype=odt, pin_memory=True),
                       torch.empty((req.k, req.n), dtype=odt, pin_memory=True),
                       torch.empty(req.m, dtype=torch.int64, pin_memory=True),
                       torch.empty(req.n, dtype=torch.int64, pin_memory=True))
            for t, name in zip(outputs, "LUpq"):
                nbytes = t.numel() * t.element_size()
                rlu_copy_block_async(ctypes.c_void_p(t.data_ptr()), nbytes, ptr(name), nbytes, nbytes, 1, sptr)
        stream.synchronize()
        return status, outputs

    # ---- scheduler side -------------------------------------------------------
    def _carve_parts(self, parts):
        total = sum(_up(b) for _, b in parts)
        off = self.pool.alloc(total)
        if off is None:
            return None
        c = Carve(off, total)
        o = off
        for name, b in parts:
            c.parts[name] = (o, b)
            o += _up(b)
        return c

    def _try_carve(self, req):
        return self._carve_parts(plan_carve(req))

    def _evict_one(self):
        """Drop the least recently used idle graph bucket; False if none."""
        idle = [b for b in self.buckets.values() if not b.busy]
        if not idle:
            return False
        b = min(idle, key=lambda x: x.last_used)
        if b.graph is not None:
            rlu_graph_destroy(b.graph)
        if b.h is not None:
            rlu_destroy(b.h)
        self.pool.free(b.carve.off, b.carve.total)
        del self.buckets[b.key]
        self.graph_stats["evictions"] += 1
        return True

    def _admit(self, req):
        """(carve, bucket) for the request, or None when the pool has no room."""
        key = bucket_key(req) if self.graphs else None
        if key is not None:
            self.key_seen[key] += 1
            b = self.buckets.get(key)
            if b is None and self.key_seen[key] >= self.graph_min_uses:
                bc = self._carve_parts(plan_bucket(key))
                if bc is not None:
                    b = _Bucket(key, bc)
                    self.buckets[key] = b
            if b is not None and not b.busy:
                carve = self._carve_parts(plan_outputs(req))
                if carve is not None:
                    b.busy = True
                    b.last_used = time.perf_counter()
                    return carve, b
            self.key_seen[key] -= 1  # counted again when it is admitted
        while True:
            carve = self._try_carve(req)
            if carve is not None:
                if key is not None:
                    self.key_seen[key] += 1
                    self.graph_stats["eager"] += 1
                return carve, None
            if not self._evict_one():
                return None

    def run(self, requests, open_loop=True):
        """Serve `requests` (t_arrive in seconds from the start; ignored when
        open_loop is False: all are waiting at time 0).  Returns the results in
        request order and the makespan in seconds."""
        too_big = [r.rid for r in requests if footprint(r) > self.pool.nbytes]
        if too_big:
            raise ValueError("requests larger than the whole pool: %s" % too_big[:8])
        pending = collections.deque(sorted(requests, key=lambda r: (r.t_arrive if open_loop else 0.0, r.rid)))
        waiting = collections.deque()
        free_slots = list(range(self.nslots))
        results = {}
        admitted_at = {}
        bypassed = 0
        import torch
        # the requests' device tensors may still be in flight on the caller's
        # stream: every slot stream waits for this point of it
        ready = torch.cuda.current_stream(self.device).record_event() if self.device.type == "cuda" else None
        t0 = time.perf_counter()
        n_total = len(requests)
        while len(results) < n_total:
            now = time.perf_counter() - t0
            while pending and (not open_loop or pending[0].t_arrive <= now):
                waiting.append(pending.popleft())
            # admission: arrival order; a later request may pass a head that does
            # not fit, at most max_bypass times in a row
            i = 0
            while free_slots and i < len(waiting):
                req = waiting[i]
                if i > 0 and bypassed >= self.max_bypass:
                    break
                got = self._admit(req)
                if got is None:
                    i += 1
                    continue
                carve, bucket = got
                del waiting[i]
                if i > 0:
                    bypassed += 1
                else:
                    bypassed = 0
                s = free_slots.pop()
                admitted_at[req.rid] = time.perf_counter() - t0
                self.jobs[s].put((req, carve, t0, bucket, ready))
            # wait for a completion or the next arrival (and look at the workers
            # at least once a second)
            timeout = 1.0
            if pending and open_loop:
                timeout = min(timeout, max(0.0, pending[0].t_arrive - (time.perf_counter() - t0)))
            try:
                item = self.done.get(timeout=timeout)
            except queue.Empty:
                if not all(t.is_alive() for t in self.threads):
                    raise RuntimeError("a serving worker stopped: %s" % self.worker_error)
                continue
            while True:
                s, req, carve, status, t_done, outputs, bucket = item
                self.pool.free(carve.off, carve.total)
                if bucket is not None:
                    bucket.busy = False
                free_slots.append(s)
                results[req.rid] = Result(req.rid, status, req.t_arrive if open_loop else 0.0, admitted_at[req.rid],
                                          t_done, s, carve.total, outputs)
                try:
                    item = self.done.get_nowait()
                except queue.Empty:
                    break
        makespan = max(r.t_done for r in results.values()) if results else 0.0
        return [results[r.rid] for r in requests], makespan

    def close(self):
        for q in self.jobs:
            q.put(None)
        for t in self.threads:
            t.join()
        for b in list(self.buckets.values()):
            if b.graph is not None:
                rlu_graph_destroy(b.graph)
            if b.h is not None:
                rlu_destroy(b.h)
        self.buckets.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class GraphBucket:
    """One exact size served by a captured launch graph: a handle, its input
    buffer, outputs and status word, all fixed, and the graph of the whole
    factorization over them.  serve(A) copies A into the input buffer and
    replays the graph; the first call runs eagerly and captures."""

    def __init__(self, m, n, k, l, l1, seed, prec="f32", dtype=None, device="cuda"):
        import torch
        from . import RandLU
        self.shape = (m, n)
        self.stream = torch.cuda.Stream(device=device)
        self.sptr = ctypes.c_void_p(self.stream.cuda_stream)
        self.handle = RandLU(m, n, k, l, l1, seed, prec=prec)
        dtype = dtype or (torch.float64 if prec == "f64" else torch.float32)
        self.A = torch.zeros((m, n), dtype=dtype, device=device)
        self.out = self.handle.alloc_outputs(device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.graph = None

    def _ptrs(self):
        L, U, p, q = self.out
        return [ctypes.c_void_p(t.data_ptr()) for t in (self.A, L, U, p, q)]

    def serve(self, A=None):
        """Factor A (device tensor of the bucket's shape; None = the buffer as
        it is).  Returns the status code."""
        import torch
        # A may still be in flight on the caller's stream
        self.stream.wait_stream(torch.cuda.current_stream(self.stream.device))
        with torch.cuda.stream(self.stream):
            if A is not None:
                self.A.copy_(A)
        a, L, U, p, q = self._ptrs()
        if self.graph is None:
            code = load().rlu_factor_dense(self.handle.h, a, self.A.stride(0), _dtype_code(self.A), L, U, p, q,
                                           self.sptr)
            if code not in (RLU_OK, RLU_WRANK):
                return code
            self.graph = rlu_graph_capture_dense(self.handle.h, a, self.A.stride(0), _dtype_code(self.A), L, U, p,
                                                 q, ctypes.c_void_p(self.status.data_ptr()), self.sptr)
            self.stream.synchronize()
            return code
        rlu_graph_launch(self.graph, self.sptr)
        self.stream.synchronize()
        return int(self.status.item())

    def close(self):
        if self.graph is not None:
            rlu_graph_destroy(self.graph)
            self.graph = None
        self.handle.close()


def summarize(results, makespan):
    """p50/p99 latency (ms), mean service share and throughput of one run."""
    lat = np.array([r.latency for r in results]) * 1e3
    ok = sum(1 for r in results if r.status in (RLU_OK, RLU_WRANK))
    return {"requests": len(results), "ok": ok, "makespan_s": makespan,
            "factorizations_per_s": len(results) / makespan if makespan > 0 else None,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean())}
