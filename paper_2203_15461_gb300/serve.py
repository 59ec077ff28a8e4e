"""Continuous-batching request loop for CPM charge updates on one GPU.

Requests (an electrolyte configuration, electrode potentials and a geometry key)
arrive over time.  Each geometry owns a CPM context (its S, tables and per-step
scratch stay resident in HBM) and a CUDA stream.  Whenever a geometry's stream
is idle and it has queued requests, up to ``max_batch`` of them are packed into
one batch (shorter electrolytes padded with zero charges) and launched
asynchronously; batches of different geometries overlap on the device.
Geometries are admitted by an HBM budget: a new geometry's context is created
only when its device memory fits next to the resident ones (measured by the
library once a geometry has been admitted); idle geometries are evicted
least-recently-used first and come back from a host-memory checkpoint of S, and
requests of a geometry that cannot be admitted yet wait.  Each batch is one
replay of a captured step graph.  Latency is measured from a request's arrival
to the moment its result is on the host.

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
    """Admission by budget, per-geometry queues, one in-flight batch per geometry.

    A geometry's device bytes are known once it has been admitted (the backend's ``create``
    returns the context's measured ``cpm_device_bytes``); before that the estimate given to
    ``add_geometry`` is used.  Admission evicts idle geometries (nothing in flight, nothing
    queued), least recently used first, until the new one fits; when the measured size turns
    out larger than the estimate, more idle geometries are evicted, and if it still does not
    fit the new context is released again and its requests wait."""

    def __init__(self, backend, hbm_budget: int, max_batch: int = 16):
        self.backend = backend
        self.budget = int(hbm_budget)
        self.max_batch = int(max_batch)
        self.queues: dict[str, collections.deque] = collections.defaultdict(collections.deque)
        self.resident: collections.OrderedDict[str, int] = collections.OrderedDict()   # key -> bytes (LRU order)
        self.inflight: dict[str, list] = {}
        self.finished: list[Request] = []
        self.geometries: dict[str, object] = {}
        self.measured: dict[str, int] = {}
        self.evictions = 0
        self.admissions = 0
        self.peak_bytes = 0

    # -- geometry management
    def add_geometry(self, key: str, geometry, est_bytes: int):
        self.geometries[key] = (geometry, int(est_bytes))

    def _used(self) -> int:
        return sum(self.resident.values())

    def _need(self, key: str) -> int:
        return self.measured.get(key, self.geometries[key][1])

    def _evict_idle(self, need: int, keep: str | None = None):
        for k in list(self.resident):
            if self._used() + need <= self.budget:
                break
            if k != keep and k not in self.inflight and not self.queues[k]:
                self.backend.release(k)
                del self.resident[k]
                self.evictions += 1

    def _admit(self, key: str) -> bool:
        if key in self.resident:
            self.resident.move_to_end(key)
            return True
        geom, _ = self.geometries[key]
        need = self._need(key)
        if need > self.budget:
            raise ValueError(f"geometry {key} needs {need} bytes, more than the whole budget {self.budget}")
        self._evict_idle(need)
        if self._used() + need > self.budget:
            return False
        got = self.backend.create(key, geom)
        self.admissions += 1
        actual = int(got) if got else need
        self.measured[key] = actual
        self.resident[key] = actual
        if self._used() > self.budget:
            self._evict_idle(0, keep=key)
            if self._used() > self.budget:
                self.backend.release(key)
                del self.resident[key]
                return False
        self.peak_bytes = max(self.peak_bytes, self._used())
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


def _pow2_at_least(m: int) -> int:
    p = 1
    while p < m:
        p *= 2
    return p


class GpuBackend:
    """One CPM context and CUDA stream per resident geometry.

    The first admission of a geometry assembles and inverts it, keeps a checkpoint of S, SG and u in
    page-locked host memory (``cpm_export``) and frees A and the factor workspace; a later admission
    after an eviction restores the context from that checkpoint (``cpm_prepare`` + ``cpm_import``)
    without assembling again.  Batches are padded to a power-of-two replica count (zero-charge
    replicas) and every replica to the batch's charge bucket (quarters of ``ne_max[key]``; zero
    charges enter no cell list and cost only reciprocal-space work), so a geometry replays at most
    (log2(max_batch) + 1) x 4 captured step graphs (``cpm_step_graph``); the largest is captured at
    admission (it sizes the scratch), the others at their first use."""

    def __init__(self, s_prec: str = "fp32", k_prec: str = "fp32", max_batch: int = 16, ne_max=None,
                 graphs: bool = True):
        import torch
        self.torch = torch
        self.s_prec, self.k_prec = s_prec, k_prec
        self.max_batch = max_batch
        self.ne_max = dict(ne_max or {})
        self.graphs = graphs
        self.ctx: dict[str, object] = {}
        self.stream: dict[str, object] = {}
        self.event: dict[str, object] = {}
        self.out: dict[str, tuple] = {}
        self.bufs: dict[str, dict] = {}
        self.host: dict[str, object] = {}          # key -> pinned checkpoint
        self.restores = 0
        self.create_seconds: dict[str, list] = collections.defaultdict(list)

    def now(self) -> float:
        return time.perf_counter()

    def _sizes(self):
        out, p = [], 1
        while p < self.max_batch:
            out.append(p)
            p *= 2
        return sorted(set(out + [self.max_batch]), reverse=True)

    def create(self, key, el):
        from .cpm import CPM
        torch = self.torch
        t0 = time.perf_counter()
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx = CPM.for_electrodes(el, s_prec=self.s_prec, k_prec=self.k_prec, stream=st)
            if key in self.host:
                dev = "cuda"
                ctx.cpm_prepare(torch.as_tensor(np.ascontiguousarray(el.xyz), device=dev),
                                torch.as_tensor(np.ascontiguousarray(el.eta), device=dev),
                                torch.as_tensor(np.ascontiguousarray(el.group, dtype=np.int32), device=dev),
                                el.n_groups)
                ctx.cpm_import(self.host[key])
                self.restores += 1
            else:
                ctx.setup(el)
                self.host[key] = ctx.cpm_export()
                ctx.cpm_release_assembly()
        self.ctx[key], self.stream[key] = ctx, st
        self.bufs[key] = {}
        if key not in self.ne_max:
            self.ne_max[key] = 2 * el.n
        if self.graphs:
            # the largest batch and charge bucket first: it sizes the scratch for every later graph
            self._launch(key, [], self.max_batch, self._bucket(key, self.ne_max[key]))
            st.synchronize()
        self.create_seconds[key].append(time.perf_counter() - t0)
        return ctx.cpm_device_bytes()

    def release(self, key):
        self.torch.cuda.synchronize()
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

    def _bucket(self, key, ne_batch):
        """Charges per replica of a batch: the geometry's maximum in four steps (multiples of 64)."""
        ne_max = self.ne_max[key]
        step = max(64, ((ne_max + 3) // 4 + 63) // 64 * 64)
        return min(max(step, -(-ne_batch // step) * step), -(-ne_max // 64) * 64)

    def _launch(self, key, batch, mp, ne=None):
        torch = self.torch
        ctx, st = self.ctx[key], self.stream[key]
        if ne is None:
            ne = self._bucket(key, max((r.Q.shape[0] for r in batch), default=0))
        ng = ctx.n_groups
        tag = f"{mp}_{ne}"
        hx = self._buf(key, f"hx{tag}", (mp * ne, 3), torch.float64, pinned=True)
        hQ = self._buf(key, f"hQ{tag}", (mp * ne,), torch.float64, pinned=True)
        hp = self._buf(key, f"hp{tag}", (mp, ng), torch.float64, pinned=True)
        xv, Qv, pv = hx.numpy().reshape(mp, ne, 3), hQ.numpy().reshape(mp, ne), hp.numpy()
        for r, req in enumerate(batch):
            k = req.Q.shape[0]
            if k > ne:
                raise ValueError(f"request {req.rid} has {k} charges, more than the {ne} of geometry {key}")
            xv[r, :k] = req.xyz
            xv[r, k:] = req.xyz[0] if k else 0.0
            Qv[r, :k] = req.Q
            Qv[r, k:] = 0.0
            pv[r] = req.psi
        xv[len(batch):] = 0.0
        Qv[len(batch):] = 0.0
        pv[len(batch):] = 0.0
        dx = self._buf(key, f"dx{tag}", (mp * ne, 3), torch.float64)
        dQ = self._buf(key, f"dQ{tag}", (mp * ne,), torch.float64)
        dp = self._buf(key, f"dp{tag}", (mp, ng), torch.float64)
        b = self._buf(key, f"b{tag}", (mp, ctx.n), torch.float64)
        q = self._buf(key, f"q{tag}", (mp, ctx.n), torch.float64)
        qt = self._buf(key, f"qt{tag}", (mp,), torch.float64)
        hq = self._buf(key, f"hq{tag}", (mp, ctx.n), torch.float64, pinned=True)
        hqt = self._buf(key, f"hqt{tag}", (mp,), torch.float64, pinned=True)
        with torch.cuda.stream(st):
            dx.copy_(hx, non_blocking=True)
            dQ.copy_(hQ, non_blocking=True)
            dp.copy_(hp, non_blocking=True)
            if self.graphs:
                ctx.cpm_step_graph(mp, ne, dx, dQ, dp, b, q, qt)
            else:
                ctx.cpm_bvec(mp, ne, dx, dQ, b)
                ctx.cpm_update(mp, dp, b, q, qt)
            hq.copy_(q, non_blocking=True)
            hqt.copy_(qt, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return ev, hq, hqt

    def launch(self, key, batch):
        mp = min(_pow2_at_least(len(batch)), self.max_batch) if self.graphs else len(batch)
        mp = max(mp, len(batch))
        ev, hq, hqt = self._launch(key, batch, mp)
        self.event[key] = ev
        self.out[key] = (hq, hqt, len(batch))

    def ready(self, key) -> bool:
        return self.event[key].query()

    def collect(self, key):
        hq, hqt, m = self.out.pop(key)
        return hq.numpy()[:m].copy(), hqt.numpy()[:m].copy()


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
