"""Continuous-batching request loop for CPM charge updates on one GPU.

Requests (an electrolyte configuration, electrode potentials and a geometry key)
arrive over time.  Each geometry owns a CPM context (its S, tables and per-step
scratch stay resident in HBM) and a CUDA stream.  Whenever a geometry's stream
is idle and it has queued requests, up to ``max_batch`` of them are packed into
one batch (shorter electrolytes padded with zero charges) and launched
asynchronously; batches of different geometries overlap on the device.
Geometries are admitted by an HBM budget: a new geometry's context is created
only when its device memory fits next to the resident ones; idle geometries are
evicted least-recently-used first, and requests of a geometry that cannot be
admitted yet wait.  Latency is measured from a request's arrival to the moment
its result is on the host.

The scheduling policy is plain Python over two small backends: ``GpuBackend``
drives the CUDA library through the C ABI; tests drive ``Scheduler`` with a
fake backend on the CPU.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    key: str                    # geometry
    xyz: np.ndarray             # (N_e, 3) electrolyte positions
    Q: np.ndarray               # (N_e,) charges
    psi: np.ndarray             # (N_g,) electrode potentials
    arrival: float = 0.0
    done: float = -1.0
    q: np.ndarray | None = None
    qtot: float | None = None


def context_bytes(n: int, n_e: int, max_batch: int, nk_grid: int = 0) -> int:
    """Device bytes a geometry needs: A, factor, S (FP64), S (FP32), tables and per-step scratch."""
    dense = n * n * (3 * 8 + 4)
    per_step = max_batch * (n_e * 120 + n * 64 + nk_grid * 16) + 64 * n * 8
    return int(dense + per_step + (64 << 20))


class Scheduler:
    """Admission by budget, per-geometry queues, one in-flight batch per geometry."""

    def __init__(self, backend, hbm_budget: int, max_batch: int = 16):
        self.backend = backend
        self.budget = int(hbm_budget)
        self.max_batch = int(max_batch)
        self.queues: dict[str, collections.deque] = collections.defaultdict(collections.deque)
        self.resident: collections.OrderedDict[str, int] = collections.OrderedDict()   # key -> bytes (LRU order)
        self.inflight: dict[str, list] = {}
        self.finished: list[Request] = []
        self.geometries: dict[str, object] = {}
        self.evictions = 0

    # -- geometry management
    def add_geometry(self, key: str, geometry, est_bytes: int):
        self.geometries[key] = (geometry, int(est_bytes))

    def _used(self) -> int:
        return sum(self.resident.values())

    def _admit(self, key: str) -> bool:
        if key in self.resident:
            self.resident.move_to_end(key)
            return True
        geom, need = self.geometries[key]
        if need > self.budget:
            raise ValueError(f"geometry {key} needs {need} bytes, more than the whole budget {self.budget}")
        # evict idle geometries, least recently used first, until the new one fits
        for k in list(self.resident):
            if self._used() + need <= self.budget:
                break
            if k not in self.inflight and not self.queues[k]:
                self.backend.release(k)
                del self.resident[k]
                self.evictions += 1
        if self._used() + need > self.budget:
            return False
        self.backend.create(key, geom)
        self.resident[key] = need
        return True

    # -- request flow
    def submit(self, req: Request):
        self.queues[req.key].append(req)

    def pump(self):
        """Collect finished batches, then launch every geometry that is idle and has work."""
        for key in list(self.inflight):
            if self.backend.ready(key):
                batch = self.inflight.pop(key)
                q, qt = self.backend.collect(key)
                now = self.backend.now()
                for r, req in enumerate(batch):
                    req.q, req.qtot, req.done = q[r], float(qt[r]), now
                    self.finished.append(req)
        for key, dq in self.queues.items():
            if not dq or key in self.inflight:
                continue
            if not self._admit(key):
                continue
            batch = [dq.popleft() for _ in range(min(self.max_batch, len(dq)))]
            self.backend.launch(key, batch)
            self.inflight[key] = batch

    def idle(self) -> bool:
        return not self.inflight and not any(self.queues.values())


class GpuBackend:
    """One CPM context and CUDA stream per resident geometry."""

    def __init__(self, s_prec: str = "fp32", k_prec: str = "fp32", max_batch: int = 16):
        import torch
        self.torch = torch
        self.s_prec, self.k_prec = s_prec, k_prec
        self.max_batch = max_batch
        self.ctx: dict[str, object] = {}
        self.stream: dict[str, object] = {}
        self.event: dict[str, object] = {}
        self.out: dict[str, tuple] = {}
        self.bufs: dict[str, dict] = {}

    def now(self) -> float:
        return time.perf_counter()

    def create(self, key, el):
        from .cpm import CPM
        torch = self.torch
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx = CPM.for_electrodes(el, s_prec=self.s_prec, k_prec=self.k_prec, stream=st).setup(el)
        self.ctx[key], self.stream[key] = ctx, st
        self.bufs[key] = {}

    def release(self, key):
        self.ctx.pop(key).close()
        self.stream.pop(key, None)
        self.bufs.pop(key, None)

    def _buf(self, key, name, shape, dtype, pinned=False):
        torch = self.torch
        b = self.bufs[key].get(name)
        if b is None or b.shape != shape:
            b = torch.empty(shape, dtype=dtype, pin_memory=True) if pinned else \
                torch.empty(shape, dtype=dtype, device="cuda")
            self.bufs[key][name] = b
        return b

    def launch(self, key, batch):
        torch = self.torch
        ctx, st = self.ctx[key], self.stream[key]
        m = len(batch)
        ne = max(r.Q.shape[0] for r in batch)
        hx = self._buf(key, "hx", (m * ne, 3), torch.float64, pinned=True)
        hQ = self._buf(key, "hQ", (m * ne,), torch.float64, pinned=True)
        hp = self._buf(key, "hp", (m, ctx.n_groups), torch.float64, pinned=True)
        hx.zero_(); hQ.zero_()
        for r, req in enumerate(batch):
            k = req.Q.shape[0]
            hx[r * ne:r * ne + k] = torch.from_numpy(req.xyz)
            if k < ne:
                hx[r * ne + k:(r + 1) * ne] = torch.from_numpy(req.xyz[:1]) if k else 0.0
            hQ[r * ne:r * ne + k] = torch.from_numpy(req.Q)
            hp[r] = torch.from_numpy(req.psi)
        dx = self._buf(key, f"dx{m}", (m * ne, 3), torch.float64)
        dQ = self._buf(key, f"dQ{m}", (m * ne,), torch.float64)
        dp = self._buf(key, f"dp{m}", (m, ctx.n_groups), torch.float64)
        b = self._buf(key, f"b{m}", (m, ctx.n), torch.float64)
        q = self._buf(key, f"q{m}", (m, ctx.n), torch.float64)
        qt = self._buf(key, f"qt{m}", (m,), torch.float64)
        hq = self._buf(key, f"hq{m}", (m, ctx.n), torch.float64, pinned=True)
        hqt = self._buf(key, f"hqt{m}", (m,), torch.float64, pinned=True)
        with torch.cuda.stream(st):
            dx.copy_(hx, non_blocking=True)
            dQ.copy_(hQ, non_blocking=True)
            dp.copy_(hp, non_blocking=True)
            ctx.cpm_bvec(m, ne, dx, dQ, b)
            ctx.cpm_update(m, dp, b, q, qt)
            hq.copy_(q, non_blocking=True)
            hqt.copy_(qt, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        self.event[key] = ev
        self.out[key] = (hq, hqt)

    def ready(self, key) -> bool:
        return self.event[key].query()

    def collect(self, key):
        hq, hqt = self.out.pop(key)
        return hq.numpy().copy(), hqt.numpy().copy()


def run_stream(requests, scheduler, arrivals=None, clock=time.perf_counter, spin_sleep=0.0):
    """Feed requests at their arrival times (seconds from start) and pump until all finish."""
    t0 = clock()
    order = sorted(range(len(requests)), key=lambda i: arrivals[i] if arrivals is not None else 0.0)
    k = 0
    while k < len(order) or not scheduler.idle():
        now = clock() - t0
        while k < len(order) and (arrivals is None or arrivals[order[k]] <= now):
            req = requests[order[k]]
            req.arrival = t0 + (arrivals[order[k]] if arrivals is not None else 0.0)
            scheduler.submit(req)
            k += 1
        scheduler.pump()
        if spin_sleep:
            time.sleep(spin_sleep)
    return time.perf_counter() - t0


def latency_stats(reqs):
    lat = np.array([r.done - r.arrival for r in reqs])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "n": len(reqs)}
