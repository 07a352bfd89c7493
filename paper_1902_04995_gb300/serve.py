"""Continuous-batching serving loop for batched 2-D LP requests.

The method is used iteratively in the paper's application (a crowd simulation solves
a fresh batch every time step, Sec. 1 and Sec. 5), and transfer costs amortise only
when work stays on the device (Sec. 6).  This engine keeps a fixed device arena (the
admission cap), admits each arriving request as soon as its buffers fit, and runs
it on one of several CUDA streams: one host-to-device copy of the packed request,
the solve through the C ABI, one device-to-host copy of the results.  Requests that
arrive while others are in flight are admitted as memory frees up, and their copies
and solves overlap on the GPU.  Each request is an independent batch with its own
seed, so its results do not depend on what else is in flight.

Layout of a request in the arena (and in its pinned host payload), each array
aligned to 256 bytes: ax, ay, b (float32 [n_c]), offsets (int64 [n_lp + 1]), obj
(float32 [2 n_lp]); then the results xy (float32 [2 n_lp]) and status (int32 [n_lp]),
and the 256-byte solver workspace.

Requests on resident data (ResidentPool, try_submit_resident): the LPs are placed in
device memory once and a request names a range of them with its own seed, so only
the results (12 bytes per LP) cross the host link; the arena then holds only each
request's results and workspace, and the results land in a pinned host ring.
"""
from __future__ import annotations

import bisect
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import lp2d

ALIGN = 256


def _up(n: int, a: int = ALIGN) -> int:
    return (n + a - 1) // a * a


class ArenaAllocator:
    """First-fit allocator of aligned byte ranges inside [0, capacity)."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        self.free = [(0, self.capacity)]  # sorted, non-adjacent (start, size)
        self.used = 0
        self.peak = 0

    def alloc(self, size: int):
        size = _up(max(int(size), 1))
        for i, (start, n) in enumerate(self.free):
            if n >= size:
                if n == size:
                    self.free.pop(i)
                else:
                    self.free[i] = (start + size, n - size)
                self.used += size
                self.peak = max(self.peak, self.used)
                return start, size
        return None

    def release(self, start: int, size: int):
        i = bisect.bisect_left(self.free, (start, 0))
        self.free.insert(i, (start, size))
        self.used -= size
        # merge with neighbours
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            self.free[i] = (self.free[i][0], self.free[i][1] + self.free[i + 1][1])
            self.free.pop(i + 1)
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            self.free.pop(i)


def request_layout(n_lp: int, n_c: int):
    """Byte offsets of the arrays of one request and the sizes of its input part
    (copied in), output part (copied out) and whole footprint."""
    off = {}
    pos = 0
    for name, nbytes in (("ax", 4 * n_c), ("ay", 4 * n_c), ("b", 4 * n_c), ("offsets", 8 * (n_lp + 1)),
                         ("obj", 8 * n_lp)):
        off[name] = pos
        pos += _up(nbytes)
    in_bytes = pos
    for name, nbytes in (("xy", 8 * n_lp), ("status", 4 * n_lp)):
        off[name] = pos
        pos += _up(nbytes)
    out_bytes = pos - in_bytes
    off["ws"] = pos
    pos += _up(lp2d.workspace_bytes(n_lp))
    return off, in_bytes, out_bytes, pos


class Payload:
    """A request packed into pinned host memory in the arena layout."""

    def __init__(self, batch, seed: int = 0):
        self.n_lp = int(len(batch["offsets"]) - 1)
        self.n_c = int(batch["offsets"][-1] - batch["offsets"][0])
        self.box = tuple(batch["box"])
        self.seed = seed
        self.off, self.in_bytes, self.out_bytes, self.total = request_layout(self.n_lp, self.n_c)
        buf = torch.zeros(self.in_bytes, dtype=torch.uint8).pin_memory()
        host = buf.numpy()
        o0 = int(batch["offsets"][0])
        for name, arr in (("ax", batch["ax"][o0:o0 + self.n_c]), ("ay", batch["ay"][o0:o0 + self.n_c]),
                          ("b", batch["b"][o0:o0 + self.n_c]), ("offsets", batch["offsets"] - o0),
                          ("obj", np.ascontiguousarray(batch["obj"]).reshape(-1))):
            raw = np.ascontiguousarray(arr).view(np.uint8)
            host[self.off[name]:self.off[name] + raw.size] = raw
        self.host_in = buf
        self.host_out = torch.empty(self.out_bytes, dtype=torch.uint8).pin_memory()

    def results(self):
        """(xy float32 [n_lp, 2], status int32 [n_lp]) from the last completed run."""
        base = self.off["xy"]
        h = self.host_out.numpy()
        xy = h[self.off["xy"] - base:self.off["xy"] - base + 8 * self.n_lp].view(np.float32).reshape(-1, 2)
        st = h[self.off["status"] - base:self.off["status"] - base + 4 * self.n_lp].view(np.int32)
        return xy.copy(), st.copy()


@dataclass
class _InFlight:
    rid: int
    payload: Payload
    arrival: float
    admitted: float
    start: int
    size: int
    done: torch.cuda.Event
    stream_idx: int


@dataclass
class ServeStats:
    latencies_ms: list = field(default_factory=list)
    lps: int = 0
    requests: int = 0
    wall_s: float = 0.0
    peak_bytes: int = 0

    def summary(self):
        lat = np.asarray(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"requests": self.requests, "lps_per_s": self.lps / self.wall_s if self.wall_s > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "peak_resident_bytes": int(self.peak_bytes),
                "wall_s": self.wall_s}


class ServeEngine:
    """Admission by device memory, overlapped execution on several streams."""

    def __init__(self, capacity_bytes: int = 20 << 30, n_streams: int = 4, device="cuda",
                 options: lp2d.Options | None = None):
        self.options = options if options is not None else lp2d.default_options()
        if self.options.precision == lp2d.PREC_FP64:
            # the request layout holds float32 vertices; FP64 callers use solve_batch_ex
            raise ValueError("ServeEngine serves the FP32 precisions only")
        self.device = torch.device(device)
        self.arena = torch.empty(int(capacity_bytes), dtype=torch.uint8, device=self.device)
        self.alloc = ArenaAllocator(capacity_bytes)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_streams)]
        self.load = [0] * n_streams
        self.inflight: list[_InFlight] = []
        self.host_out = None  # pinned result ring of the resident requests (make_host_ring)
        self.host_alloc = None
        self._next_id = 0

    def _view(self, start, off, name, dtype, count):
        lo = start + off[name]
        nbytes = count * torch.empty(0, dtype=dtype).element_size()
        return self.arena[lo:lo + nbytes].view(dtype)

    def try_submit(self, payload: Payload, arrival: float) -> bool:
        """Admit and enqueue a request if its footprint fits the arena now."""
        got = self.alloc.alloc(payload.total)
        if got is None:
            return False
        start, size = got
        si = min(range(len(self.streams)), key=lambda i: self.load[i])
        s = self.streams[si]
        off, n_lp, n_c = payload.off, payload.n_lp, payload.n_c
        with torch.cuda.stream(s):
            self.arena[start:start + payload.in_bytes].copy_(payload.host_in, non_blocking=True)
            ws = self._view(start, off, "ws", torch.uint8, lp2d.workspace_bytes(n_lp))
            lp2d.workspace_init(ws, stream=s)
            opts = lp2d.Options.from_buffer_copy(self.options)
            opts.seed = payload.seed
            lp2d.solve_batch_ex(self._view(start, off, "ax", torch.float32, n_c),
                                self._view(start, off, "ay", torch.float32, n_c),
                                self._view(start, off, "b", torch.float32, n_c),
                                self._view(start, off, "offsets", torch.int64, n_lp + 1),
                                self._view(start, off, "obj", torch.float32, 2 * n_lp), payload.box,
                                self._view(start, off, "xy", torch.float32, 2 * n_lp),
                                self._view(start, off, "status", torch.int32, n_lp), opts, ws, stream=s)
            lo = start + off["xy"]
            payload.host_out.copy_(self.arena[lo:lo + payload.out_bytes], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        self.load[si] += payload.total
        self.inflight.append(_InFlight(self._next_id, payload, arrival, time.perf_counter(), start, size, ev, si))
        self._next_id += 1
        return True

    # ---- requests on device-resident data
    def make_host_ring(self, nbytes: int):
        """Pinned host memory that the results of resident requests are copied into
        (first-fit, freed when a request retires)."""
        self.host_out = torch.empty(int(nbytes), dtype=torch.uint8).pin_memory()
        self.host_alloc = ArenaAllocator(int(nbytes))

    def try_submit_resident(self, pool: "ResidentPool", req: "ResidentRequest", arrival: float) -> bool:
        """Admit a request on LPs already resident in device memory: only its results
        and workspace take arena memory, and only its results cross the host link."""
        n_lp = req.hi - req.lo
        xy_b, st_b, ws_b = _up(8 * n_lp), _up(4 * n_lp), _up(lp2d.workspace_bytes(n_lp))
        got = self.alloc.alloc(xy_b + st_b + ws_b)
        if got is None:
            return False
        hgot = self.host_alloc.alloc(xy_b + st_b)
        if hgot is None:
            self.alloc.release(*got)
            return False
        start, size = got
        si = min(range(len(self.streams)), key=lambda i: self.load[i])
        s = self.streams[si]
        t = pool.t
        with torch.cuda.stream(s):
            ws = self.arena[start + xy_b + st_b:start + xy_b + st_b + ws_b]
            lp2d.workspace_init(ws, stream=s)
            opts = lp2d.Options.from_buffer_copy(self.options)
            opts.seed = req.seed
            xy = self.arena[start:start + 8 * n_lp].view(torch.float32)
            st = self.arena[start + xy_b:start + xy_b + 4 * n_lp].view(torch.int32)
            lp2d.solve_batch_ex(t["ax"], t["ay"], t["b"], t["offsets"][req.lo:req.hi + 1],
                                t["obj"][2 * req.lo:2 * req.hi], pool.box, xy, st, opts, ws, stream=s)
            self.host_out[hgot[0]:hgot[0] + xy_b + st_b].copy_(self.arena[start:start + xy_b + st_b],
                                                                 non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        self.load[si] += size
        r = _InFlight(self._next_id, req, arrival, time.perf_counter(), start, size, ev, si)
        r.host = hgot
        self.inflight.append(r)
        self._next_id += 1
        return True

    def resident_results(self, r):
        """(xy float32 [n_lp, 2], status int32 [n_lp]) of a retired resident request,
        from the host ring (valid until the ring range is reused)."""
        n_lp = r.payload.hi - r.payload.lo
        h = self.host_out.numpy()[r.host[0]:r.host[0] + r.host[1]]
        xy = h[:8 * n_lp].view(np.float32).reshape(-1, 2)
        st = h[_up(8 * n_lp):_up(8 * n_lp) + 4 * n_lp].view(np.int32)
        return xy.copy(), st.copy()

    def run_resident_stream(self, pool, requests, arrivals, max_wall_s: float = 120.0,
                            keep_results: bool = False) -> ServeStats:
        """Serve resident requests[i] arriving at arrivals[i] seconds, in order of
        arrival; latency = results in host memory minus arrival."""
        stats = ServeStats()
        t0 = time.perf_counter()
        pending = 0
        n = len(requests)
        self.results = {}
        while (pending < n or self.inflight) and time.perf_counter() - t0 < max_wall_s:
            now = time.perf_counter() - t0
            while pending < n and arrivals[pending] <= now:
                if not self.try_submit_resident(pool, requests[pending], t0 + arrivals[pending]):
                    break
                pending += 1
            for r, t_done in self._poll_records():
                stats.latencies_ms.append(1e3 * (t_done - r.arrival))
                stats.lps += r.payload.hi - r.payload.lo
                stats.requests += 1
                if keep_results:
                    self.results[r.rid] = self.resident_results(r)
                self.host_alloc.release(*r.host)
        stats.wall_s = time.perf_counter() - t0
        stats.peak_bytes = self.alloc.peak + pool.bytes
        return stats

    def _poll_records(self):
        done, keep = [], []
        for r in self.inflight:
            if r.done.query():
                t = time.perf_counter()
                self.alloc.release(r.start, r.size)
                self.load[r.stream_idx] -= r.size
                done.append((r, t))
            else:
                keep.append(r)
        self.inflight = keep
        return done

    def poll(self):
        """Retire finished requests: free their memory; return [(rid, payload, arrival, t_done)]."""
        done, keep = [], []
        for r in self.inflight:
            if r.done.query():
                t = time.perf_counter()
                self.alloc.release(r.start, r.size)
                self.load[r.stream_idx] -= r.payload.total
                done.append((r.rid, r.payload, r.arrival, t))
            else:
                keep.append(r)
        self.inflight = keep
        return done

    def drain(self):
        out = []
        while self.inflight:
            out += self.poll()
        return out

    def run_stream(self, payloads, arrivals, max_wall_s: float = 120.0) -> ServeStats:
        """Serve requests payloads[i] arriving at arrivals[i] seconds (non-decreasing),
        in order of arrival; latency = result in host memory minus arrival."""
        stats = ServeStats()
        t0 = time.perf_counter()
        pending = 0
        n = len(payloads)
        while (pending < n or self.inflight) and time.perf_counter() - t0 < max_wall_s:
            now = time.perf_counter() - t0
            while pending < n and arrivals[pending] <= now:
                if not self.try_submit(payloads[pending], t0 + arrivals[pending]):
                    break  # wait for memory to free up (admission in arrival order)
                pending += 1
            for _, p, arr, t_done in self.poll():
                stats.latencies_ms.append(1e3 * (t_done - arr))
                stats.lps += p.n_lp
                stats.requests += 1
        stats.wall_s = time.perf_counter() - t0
        stats.peak_bytes = self.alloc.peak
        return stats


class ResidentPool:
    """LPs placed in device memory once; requests name ranges of them (the serving
    case where a request picks a payload that is already resident)."""

    def __init__(self, batch, device="cuda"):
        dev = torch.device(device)
        self.t = {k: torch.from_numpy(np.ascontiguousarray(batch[k])).to(dev).reshape(-1)
                  for k in ("ax", "ay", "b", "offsets", "obj")}
        self.offsets = np.asarray(batch["offsets"])
        self.n_lp = int(len(self.offsets) - 1)
        self.box = tuple(batch["box"])
        self.bytes = int(sum(v.numel() * v.element_size() for v in self.t.values()))


@dataclass
class ResidentRequest:
    lo: int    # first LP of the pool
    hi: int    # one past the last
    seed: int


def resident_requests(pool: ResidentPool, n_distinct: int, seed: int, lo_lp=1024, hi_lp=65536):
    """n_distinct requests: a log-uniform number of LPs in [lo_lp, hi_lp] starting at a
    uniform LP of the pool, each with its own seed."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_distinct):
        n = int(min(np.floor(np.exp(rng.uniform(np.log(lo_lp), np.log(hi_lp + 1)))), pool.n_lp))
        lo = int(rng.integers(0, pool.n_lp - n + 1))
        out.append(ResidentRequest(lo, lo + n, seed + 1000 * i))
    return out


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int):
    """Arrival times of a Poisson process of the given rate on [0, duration)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            return np.asarray(out)
        out.append(t)
