"""Benchmark of the CPM charge update (b-vector + S (v - b)) on one GB300 per rank.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--replicas M] [--k-prec P]

Workload: the 4,320-site graphene-like EDL capacitor (3 layers per electrode, 60 A gap,
1,800 rigid 3-site waters + 150 Na+ + 150 Cl-, slab correction).  One step updates
M independent replicas of that system (each its own seeded electrolyte, positions
random-walked by N(0, 0.05 A) per step): b for every replica, then q = S (v - b) and
the FP64 neutrality fix.  ``value`` is updates per second (replica-updates) of the
mixed path (FP32 b and S, FP64 neutrality and totals; by default the two reciprocal-space
contractions of b run on the tensor cores as two-term fp16 products, ``--k-prec fp32``
keeps them on the CUDA cores); the plain FP64 path is timed beside it.  Inputs are
resident in HBM; L2 is flushed (a 256 MB write, then a 256 MB read of a second buffer)
before every timed step and only the step itself is inside the CUDA events.  Extra fields:
256 replicas of the 216-site capacitor per step, a Poisson serving stream, and the
single-precision S product alone at 16,384 sites (S32 = 1.07 GB) against the HBM peak.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CPM charge updates/s (b-vector + S·b) batched-mixed vs plain FP64, 1 GB300"
WORKLOAD = "edl_capacitor_4320"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _fp32_peak_tflops(sm_mhz: float) -> float:
    # 152 SMs x 128 FP32 lanes x 2 flop per FMA x clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def rank_seed(rank: int) -> int:
    """Electrolyte seeds of a rank's replicas: ranks work on disjoint, independent replicas."""
    return 1000 * (rank + 1)


def aggregate(ms_local: float, m: int, K: int, world: int, dist=None):
    """Whole-job throughput: world x m x K updates over the slowest rank's time (max over ranks)."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device="cuda" if dist and dist.get_backend() == "nccl" else "cpu")
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return world * m * K / (ms_max / 1e3), ms_max


def make_trajectories(el, base_elyt_fn, m, steps, seed):
    """m replicas x steps configurations (random walk), replica-major per step: (steps, m*ne, 3), (m*ne,)."""
    from paper_2203_15461_gb300 import systems as s
    reps = [base_elyt_fn(seed + r) for r in range(m)]
    ne = max(e.n for e in reps)
    rng = np.random.default_rng(seed + 10007)
    xyz = np.zeros((steps, m, ne, 3))
    Q = np.zeros((m, ne))
    for r, e in enumerate(reps):
        Q[r, :e.n] = e.Q
        cur = e.xyz.copy()
        for t in range(steps):
            cur = cur + rng.normal(scale=0.05, size=cur.shape)
            xyz[t, r, :e.n] = cur
    return xyz.reshape(steps, m * ne, 3), Q.reshape(-1), ne


class L2Flush:
    """Before every timed step: write a 256 MB buffer (more than the 126 MB L2), then read another
    256 MB buffer, so that the flush's own dirty lines are written back before the timed region
    starts and the step begins with a cold, clean L2."""

    def __init__(self, torch):
        self.w = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        self.r = torch.zeros(256 << 20, dtype=torch.uint8, device="cuda")

    def __call__(self):
        self.w.zero_()
        self.r.max()


def time_path(torch, ctx, xyz_dev, Q_dev, psi_dev, m, ne, warmup, steps, flush, profile=False):
    """Per-step CUDA-event timing on the context stream; L2 flushed before every step."""
    n = ctx.n
    b = torch.empty((m, n), dtype=torch.float64, device="cuda")
    q = torch.empty((m, n), dtype=torch.float64, device="cuda")
    qt = torch.empty((m,), dtype=torch.float64, device="cuda")
    T = xyz_dev.shape[0]
    for t in range(warmup):
        ctx.cpm_bvec(m, ne, xyz_dev[t % T], Q_dev, b)
        ctx.cpm_update(m, psi_dev, b, q, qt)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = ctx.cpm_launch_count()
    if profile:
        ctx.cpm_profile_read(reset=True)
        ctx.cpm_profile(True)
    for t in range(steps):
        flush()
        evs[t][0].record()
        ctx.cpm_bvec(m, ne, xyz_dev[(warmup + t) % T], Q_dev, b)
        ctx.cpm_update(m, psi_dev, b, q, qt)
        evs[t][1].record()
    torch.cuda.synchronize()
    if profile:
        ctx.cpm_profile(False)
    launches = ctx.cpm_launch_count() - launches0
    ms = [a.elapsed_time(bb) for a, bb in evs]
    prof = ctx.cpm_profile_read(reset=True) if profile else None
    return sum(ms), launches, prof, q, qt


def time_graph(torch, ctx, st, xyz_dev, Q_dev, psi_dev, m, ne, warmup, steps, flush):
    """The step as one CUDA graph (cpm_step_graph): per step the new positions are copied into the
    captured input buffer and the graph is replayed; CUDA events on the context's stream around both,
    L2 flushed before every step."""
    n = ctx.n
    with torch.cuda.stream(st):
        dx = torch.empty_like(xyz_dev[0])
        b = torch.empty((m, n), dtype=torch.float64, device="cuda")
        q = torch.empty((m, n), dtype=torch.float64, device="cuda")
        qt = torch.empty((m,), dtype=torch.float64, device="cuda")
    T = xyz_dev.shape[0]
    for t in range(warmup):
        with torch.cuda.stream(st):
            dx.copy_(xyz_dev[t % T])
            ctx.cpm_step_graph(m, ne, dx, Q_dev, psi_dev, b, q, qt)
    st.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = ctx.cpm_launch_count()
    for t in range(steps):
        with torch.cuda.stream(st):
            flush()
            evs[t][0].record(st)
            dx.copy_(xyz_dev[(warmup + t) % T])
            ctx.cpm_step_graph(m, ne, dx, Q_dev, psi_dev, b, q, qt)
            evs[t][1].record(st)
    st.synchronize()
    launches = ctx.cpm_launch_count() - launches0
    return sum(a.elapsed_time(bb) for a, bb in evs), launches, q, qt


def real_pairs(el, xyz_steps, Q, ne, m, step):
    """(site, charge) pairs within rcut over the periodic images of the Ewald cell, summed over replicas."""
    from scipy.spatial import cKDTree
    box = np.asarray(el.box, dtype=np.float64)
    sites = np.mod(el.xyz, box)
    tree = cKDTree(sites, boxsize=box)
    tot = 0
    for r in range(m):
        x = xyz_steps[step, r * ne:(r + 1) * ne]
        q = Q[r * ne:(r + 1) * ne]
        x = np.mod(x[q != 0.0], box)
        tot += int(tree.count_neighbors(cKDTree(x, boxsize=box), el.rcut))
    return tot


# Algorithmic work per unit (a cost model of the method itself, not of the kernels' own
# shortcuts): a real-space pair inside r_c costs two erfc, a square root and a division (60 flop,
# also for the tabulated single-precision kernel); a reciprocal term costs 16 flop per (charge, k)
# for the structure factor and 14 per (site, k) for the site sum on the CUDA cores.  On the tensor
# cores the contraction itself is counted (one complex multiply-add, 8 flop, per (charge, k) and
# per (site, k)) against the tensor rate of the emulated FP32 product.
FLOP_PAIR, FLOP_SF, FLOP_SITE, FLOP_CMAC = 60.0, 16.0, 14.0, 8.0


def kernel_work(el, nk, ne, m, pairs=None, tensor=False, s_bytes=4):
    """Algorithmic work per launch of the per-step kernels: (kind, amount) with kind flop | tflop | byte."""
    n = el.n
    if tensor:
        w = {"sf": ("tflop", FLOP_CMAC * ne * nk * m), "site": ("tflop", FLOP_CMAC * n * nk * m)}
    else:
        w = {"sf": ("flop", FLOP_SF * ne * nk * m), "site": ("flop", FLOP_SITE * n * nk * m)}
    # S streamed once per pass of eight replicas (single precision) or once per replica (FP64)
    w["gemv"] = ("byte", float(s_bytes) * n * n * (((m + 7) // 8) if s_bytes == 4 else m))
    if pairs is not None:
        w["real"] = ("flop", FLOP_PAIR * pairs)
    return w


def roofline(prof, work, peaks, src, names, alu_peak, alu_src, ms_step):
    """Roofline entry of the kernel with the largest share of the kernel-by-kernel step."""
    top = max((kk for kk in prof if prof[kk][1] > 0), key=lambda kk: prof[kk][0])
    avg_ms = prof[top][0] / prof[top][1]
    kind, amount = work.get(top, ("flop", float("nan")))
    if kind == "tflop":
        # fp16 tensor rate = the measured bf16 rate (same nominal peak); three fp16 products per FP32 product
        peak = float(peaks.get("bf16_tflops", 1900.0)) / 3.0
        roof = {"bound": "tensor", "unit": "TFLOP/s", "achieved": amount / (avg_ms / 1e3) / 1e12, "peak": peak,
                "peak_source": f"bf16_tflops ({src}) / 3: two-term fp16 operands, three products per FP32 product"}
    elif kind == "flop":
        roof = {"bound": "alu", "unit": "TFLOP/s", "achieved": amount / (avg_ms / 1e3) / 1e12, "peak": alu_peak,
                "peak_source": alu_src}
    else:
        peak = float(peaks["hbm_gbs"])
        roof = {"bound": "hbm", "unit": "GB/s", "achieved": amount / (avg_ms / 1e3) / 1e9, "peak": peak,
                "peak_source": f"hbm_gbs ({src})"}
    roof["kernel"] = names.get(top, top)
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["ms_per_launch"] = avg_ms
    roof["share_of_step"] = prof[top][0] / ms_step
    roof["all_kernels"] = {kk: {"ms_per_launch": prof[kk][0] / max(1, prof[kk][1]),
                                "achieved": (work[kk][1] / (prof[kk][0] / max(1, prof[kk][1]) / 1e3)
                                             / (1e9 if work[kk][0] == "byte" else 1e12)),
                                "unit": "GB/s" if work[kk][0] == "byte" else "TFLOP/s"}
                           for kk in work if kk in prof and prof[kk][1] > 0}
    return top, roof


# ----------------------------------------------------------------------------- CPU baseline leg
# The FP64 oracle as it stands, on the host cores of the GPU machine.  Only this leg runs the oracle:
# its own timing, and the oracle charges that the GPU results are compared with.

_THREAD_VARS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


class _OneThreadEnv:
    """Processes started inside this block run their BLAS on one thread."""

    def __enter__(self):
        self.saved = {k: os.environ.get(k) for k in _THREAD_VARS}
        os.environ.update({k: "1" for k in _THREAD_VARS})

    def __exit__(self, *a):
        for k, v in self.saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _oracle_sites(args):
    """Worker: the oracle's b at a chunk of sites (single thread), with its time."""
    el, ely, sites = args
    from oracle import cpm_oracle as o
    t0 = time.perf_counter()
    b = o.bvec(el, ely, sites=sites)
    return b, time.perf_counter() - t0


def _oracle_rows(args):
    el, rows = args
    from oracle import cpm_oracle as o
    return o.assemble_A(el, rows=rows)


def _serial_update(el, ely, psi, req, res):
    """Worker: one complete oracle update on one thread: b for every site, then q = S (v - b) with
    the S the parent sends once it has it; reports both times and the results."""
    from oracle import cpm_oracle as o
    t0 = time.perf_counter()
    b = o.bvec(el, ely)
    tb = time.perf_counter() - t0
    S = req.get()
    t0 = time.perf_counter()
    q = o.charges(S, el, psi, b)
    res.put((tb, time.perf_counter() - t0, b, q))


class OraclePool:
    """The oracle over all host cores (spawned processes, one BLAS thread each): site chunks of b,
    row chunks of A.  Each chunk of b evaluates its configuration's structure factor once."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        self.procs = procs or (os.cpu_count() or 1)
        with _OneThreadEnv():
            self.pool = mp.get_context("spawn").Pool(self.procs)

    def close(self):
        self.pool.terminate()
        self.pool.join()

    def assemble_A(self, el):
        chunks = [c for c in np.array_split(np.arange(el.n), min(el.n, self.procs)) if len(c)]
        return np.vstack(self.pool.map(_oracle_rows, [(el, c) for c in chunks]))

    def capacitance(self, el):
        from oracle import cpm_oracle as o
        return o.capacitance_matrix(self.assemble_A(el))

    def update(self, el, ely, psi, S):
        """One full oracle update on all cores: (q, b, wall seconds, summed worker seconds)."""
        from oracle import cpm_oracle as o
        chunks = [c for c in np.array_split(np.arange(el.n), min(el.n, self.procs)) if len(c)]
        t0 = time.perf_counter()
        parts = self.pool.map(_oracle_sites, [(el, ely, c) for c in chunks])
        b = np.concatenate([p[0] for p in parts])
        q = o.charges(S, el, psi, b)
        return q, b, time.perf_counter() - t0, sum(p[1] for p in parts)


class SerialOracle:
    """One oracle update of one configuration in a single-threaded spawned process, started before
    the first GPU call and run beside the GPU legs (it keeps one of the host's cores busy)."""

    def __init__(self, el, ely, psi):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.req, self.res = ctx.Queue(), ctx.Queue()
        with _OneThreadEnv():
            self.proc = ctx.Process(target=_serial_update, args=(el, ely, psi, self.req, self.res), daemon=True)
            self.proc.start()

    def finish(self, S, timeout=1800.0):
        self.req.put(S)
        tb, tq, b, q = self.res.get(timeout=timeout)
        self.proc.join(timeout=60)
        return tb, tq, b, q


def oracle_bvec(el, ely):
    """The oracle's b of one configuration (the P3M leg's accuracy check)."""
    from oracle import cpm_oracle as o
    return o.bvec(el, ely)


def cpu_baseline_edl(pool, serial, el, ely, psi):
    """The oracle on the headline system (one configuration, every site, every k-vector): S by the
    oracle over all cores (not timed: a one-time cost), then one full update single-threaded (the
    serial worker) and one on all cores; the oracle's q of that configuration is returned too."""
    t0 = time.perf_counter()
    S = pool.capacitance(el)
    t_S = time.perf_counter() - t0
    tb, tq, b1, q1 = serial.finish(S)
    q, b, wall, cpu_s = pool.update(el, ely, psi, S)
    out = {"value": 1.0 / wall, "unit": "updates/s", "cores": pool.procs, "kind": "oracle",
           "sample": ("one complete, unsampled FP64 oracle update of the EDL capacitor (4,320 sites, 5,700 charges, "
                      f"every k-vector): b at all sites in {pool.procs} processes over site chunks (each evaluates "
                      "the structure factor of all charges), then q = S (v - b); S from the oracle beforehand"),
           "single_thread": {"value": 1.0 / (tb + tq), "seconds": tb + tq, "cores": 1,
                             "sample": "the same update in one single-threaded process"},
           "all_cores_seconds": wall, "worker_cpu_seconds": cpu_s, "oracle_S_seconds": t_S,
           "agree_single_vs_all_cores": float(np.abs(q - q1).max() / np.abs(q1).max())}
    return out, S, q1


def cpu_baseline_small(pool, el_tiny, tiny_elyts, psi_tiny, el_coax10):
    """Oracle values of the small configurations: q of sampled cfg3 replicas and of the cfg1 step,
    and the co-axial C0/L of the 10-cell tube (the per-length value the 100-cell tube must repeat)."""
    from oracle import cpm_oracle as o
    S = o.capacitance_matrix(o.assemble_A(el_tiny))
    q = {r: o.charges(S, el_tiny, psi_tiny[r], o.bvec(el_tiny, e)) for r, e in tiny_elyts.items()}
    Sc = pool.capacitance(el_coax10)
    c0 = float(o.electrode_capacitance(Sc, el_coax10)[1, 1] / el_coax10.box[2])
    return q, c0


def bench_tiny_flow(torch, CPM, s, n_updates=10):
    """Configuration 1: the 216-site Au(111) capacitor in FP64, the whole flow: assemble, invert and
    ten sequential charge updates (positions random-walked by N(0, 0.05 A) per update)."""
    el, ely, psi = s.workload_tiny_slab(seed=1)
    rng = np.random.default_rng(2024)
    confs = []
    cur = ely
    for _ in range(n_updates):
        cur = s.jitter(cur, 0.05, rng)
        confs.append(cur)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = CPM.for_electrodes(el, s_prec="fp64", k_prec="fp64")
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    ctx.cpm_assemble(dev(el.xyz), dev(el.eta), dev(el.group.astype(np.int32)), el.n_groups)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    ctx.cpm_invert()
    t2 = time.perf_counter()
    xs = [dev(c.xyz) for c in confs]
    Qd = dev(ely.Q)
    pd = dev(psi[None])
    b = torch.empty((1, el.n), dtype=torch.float64, device="cuda")
    q = torch.empty_like(b)
    qt = torch.empty(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t3 = time.perf_counter()
    e0.record()
    for x in xs:
        ctx.cpm_bvec(1, ely.n, x, Qd, b)
        ctx.cpm_update(1, pd, b, q, qt)
    e1.record()
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    ms_upd = e0.elapsed_time(e1) / n_updates
    out = {"workload": "au111_tiny_216, FP64: assemble + invert + 10 sequential updates", "n_sites": el.n,
           "n_charges": ely.n, "assemble_ms": 1e3 * (t1 - t0), "invert_ms": 1e3 * (t2 - t1),
           "update_ms": ms_upd, "updates_per_s": 1e3 / ms_upd, "flow_ms": 1e3 * (t2 - t0 + t4 - t3),
           "max_abs_qtot": float(qt.abs().max())}
    qlast = q.cpu().numpy()[0]
    ctx.close()
    return out, (el, confs[-1], psi, qlast)


def bench_batched_tiny(torch, CPM, s, flush, K, W, m=256, k_prec="fp32", sample=(0, 85, 170, 255)):
    """Configuration 3: 256 replicas of the 216-site Au(111) capacitor per step (one shared S,
    each its own seeded electrolyte), graph-captured, with S in FP64, FP32 and split bf16 (three
    terms, tensor cores).  Returns the q of sampled replicas of the last step for the oracle leg."""
    el, _, psi = s.workload_tiny_slab(seed=1)
    xyz, Q, ne = make_trajectories(el, lambda sd: s.ions_in_gap(el, 100, seed=sd), m, K + W, 5000)
    psis = np.column_stack([np.zeros(m), np.linspace(0.0, 2.0, m)])
    out = {"workload": "au111_tiny_216 x 256 replicas", "replicas_per_step": m, "k_prec": k_prec}
    qs = {}
    for s_prec in ("fp64", "fp32", "bf16x3"):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx = CPM.for_electrodes(el, s_prec=s_prec, k_prec=k_prec, stream=st).setup(el)
            dx = torch.as_tensor(xyz[0], device="cuda").clone()
            dQ = torch.as_tensor(Q, device="cuda")
            dp = torch.as_tensor(psis, device="cuda")
            b = torch.empty((m, el.n), dtype=torch.float64, device="cuda")
            q = torch.empty_like(b)
            qt = torch.empty(m, dtype=torch.float64, device="cuda")
            xs = torch.as_tensor(xyz, device="cuda")
        st.synchronize()
        tot = 0.0
        for t in range(W + K):
            with torch.cuda.stream(st):
                flush()
                dx.copy_(xs[t])
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                ctx.cpm_step_graph(m, ne, dx, dQ, dp, b, q, qt)
                e1.record(st)
            st.synchronize()
            if t >= W:
                tot += e0.elapsed_time(e1)
        out[f"value_{s_prec}_S"] = m * K / (tot / 1e3)
        out[f"ms_per_step_{s_prec}_S"] = tot / K
        out[f"max_abs_qtot_{s_prec}_S"] = float(qt.abs().max())
        qn = q.cpu().numpy()
        qs[s_prec] = {r: qn[r] for r in sample}
        ctx.close()
    out["unit"] = "updates/s"
    last = {r: s.Electrolyte(xyz=xyz[W + K - 1, r * ne:(r + 1) * ne], Q=Q[r * ne:(r + 1) * ne]) for r in sample}
    return out, (el, last, {r: psis[r] for r in sample}, qs)


def bench_coax(torch, CPM, s, cells=100, alpha=0.15, rcut=24.0):
    """Configuration 5: the co-axial (10,10)/(20,20) nanotube capacitor, 100 cells (12,000 sites),
    1D boundary term, vacuum.  FP64 assembly of A, then the capacitance C0 two ways: FP64 Cholesky,
    inverse and projection (S, then G^T S G), and FP32 Cholesky with FP64 iterative refinement
    (no inverse).  Times of each stage and C0/L of each against 2 pi eps0 / ln(R2/R1)."""
    el = s.coaxial_tubes(cells, alpha=alpha, rcut=rcut, ktol=1e-8)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    ctx = CPM.for_electrodes(el, s_prec="fp64", k_prec="fp64")
    x, e, g = dev(el.xyz), dev(el.eta), dev(el.group.astype(np.int32))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.cpm_assemble(x, e, g, el.n_groups)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    C_ir, iters, resid = ctx.cpm_capacitance_ir()
    t2 = time.perf_counter()
    ctx.cpm_invert()
    C64 = ctx.cpm_capacitance()
    t3 = time.perf_counter()
    nk = int(len(ctx.cpm_kvectors()))
    ctx.close()
    # the same capacitor with the reciprocal part of A from P3M (FP64 mesh, 64 x 64 x 128, order 7)
    elp = s.Electrodes(**{**el.__dict__, "p3m_mesh": (64, 64, 128), "p3m_order": 7, "p3m_matrix": True})
    ctxp = CPM.for_electrodes(elp, s_prec="fp64", k_prec="fp64")
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    ctxp.cpm_assemble(x, e, g, el.n_groups)
    torch.cuda.synchronize()
    t5 = time.perf_counter()
    ctxp.cpm_invert()
    Cp = ctxp.cpm_capacitance()
    ctxp.close()
    L = float(el.box[2])
    eps0 = 1.0 / (4.0 * math.pi * 14.399645)
    ana = 2.0 * math.pi * eps0 / math.log(s.tube_radius(20) / s.tube_radius(10))
    n = el.n
    return {"workload": f"coaxial (10,10)/(20,20) tubes, {cells} cells, {n} sites, 1D correction",
            "assemble_p3m_matrix_s": t5 - t4, "p3m_matrix": {"mesh": [64, 64, 128], "order": 7},
            "C0_per_L_p3m_matrix": float(Cp[1, 1]) / L,
            "rel_diff_p3m_matrix_vs_ewald": abs(float(Cp[1, 1]) / float(C64[1, 1]) - 1.0),
            "n_sites": n, "n_kvectors": nk, "alpha": alpha, "rcut": rcut,
            "assemble_s": t1 - t0, "assemble_recip_tflops_fp64": 2.0 * n * n * nk / (t1 - t0) / 1e12,
            "fp64_cholesky_inverse_s": t3 - t2, "fp32_cholesky_ir_s": t2 - t1, "ir_sweeps": iters,
            "ir_residual": resid, "C0_per_L_fp64": float(C64[1, 1]) / L, "C0_per_L_fp32_ir": float(C_ir[1, 1]) / L,
            "rel_diff_fp32_ir_vs_fp64": abs(float(C_ir[1, 1]) / float(C64[1, 1]) - 1.0),
            "C0_per_L_analytic": ana, "ratio_to_analytic": float(C64[1, 1]) / L / ana}


def bench_s_products(torch, CPM, s, flush, peaks, src, sizes=((8192, (32, 16)), (16384, (32, 32))),
                     ms=(8, 64, 128, 256), K=5, W=2):
    """The S product alone where S is far larger than L2: two graphene electrodes of two sheets,
    8,192 and 16,384 sites, assembled once with a small Ewald alpha (0.1, r_c = 35 A: few k-vectors,
    the assembly stays short; the S product does not depend on the split).  For m replicas of a
    random b: the single-precision S stream (k_gemv_tma, S read once per eight replicas) and the
    persistent tensor-core product (k_tc_sb with its tuned tile plan, S as three bf16 planes read
    once per launch), each through cpm_update with L2 flushed before every call; the kernels alone
    from the library's per-kernel events."""
    out = {}
    bf16_peak, hbm = float(peaks.get("bf16_tflops", 1900.0)), float(peaks["hbm_gbs"])
    for n_target, (cx, cy) in sizes:
        el = s.graphene_plates(cx, cy, 2, 40.0, alpha=0.1, rcut=35.0)
        n = el.n
        t0 = time.perf_counter()
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx = CPM.for_electrodes(el, s_prec="fp32", k_prec="fp32", stream=st).setup(el)
        st.synchronize()
        res = {"n_sites": n, "setup_seconds": time.perf_counter() - t0, "s_fp32_bytes": 4.0 * n * n,
               "s_bf16x3_bytes": 6.0 * n * n}
        rng = np.random.default_rng(7)
        for m in ms:
            with torch.cuda.stream(st):
                b = torch.as_tensor(rng.normal(0.0, 1.0, (m, n)), device="cuda")
                psi = torch.as_tensor(np.tile([0.0, 1.0], (m, 1)), device="cuda")
                q = torch.empty((m, n), dtype=torch.float64, device="cuda")
                qt = torch.empty(m, dtype=torch.float64, device="cuda")
            row = {}
            q_prev = None
            for prec in ("fp32", "bf16x3"):
                ctx.cpm_set_s_prec(prec)
                plan = ctx.cpm_gemm_plan(m) if prec == "bf16x3" else None
                for _ in range(W):
                    with torch.cuda.stream(st):
                        ctx.cpm_update(m, psi, b, q, qt)
                st.synchronize()
                ctx.cpm_profile_read(reset=True)
                ctx.cpm_profile(True)
                evs = []
                for _ in range(K):
                    with torch.cuda.stream(st):
                        flush()
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(st)
                        ctx.cpm_update(m, psi, b, q, qt)
                        e1.record(st)
                        evs.append((e0, e1))
                st.synchronize()
                ctx.cpm_profile(False)
                prof = ctx.cpm_profile_read(reset=True)
                t_upd = sum(a.elapsed_time(bb) for a, bb in evs) / K
                r = {"update_ms": t_upd, "updates_per_s": m / (t_upd / 1e3),
                     "max_abs_qtot": float(qt.abs().max())}
                if prec == "fp32":
                    kms = prof["gemv"][0] / max(1, prof["gemv"][1])
                    nbytes = 4.0 * n * n * ((m + 7) // 8)
                    r.update({"kernel": "k_gemv_tma", "kernel_ms": kms, "achieved_gbs": nbytes / (kms / 1e3) / 1e9,
                              "hbm_frac": nbytes / (kms / 1e3) / 1e9 / hbm})
                else:
                    kms = prof["tcgemm"][0] / max(1, prof["tcgemm"][1])
                    flop = 2.0 * n * n * m * 6
                    nbytes = 6.0 * n * n
                    r.update({"kernel": "k_tc_sb", "kernel_ms": kms, "plan": plan,
                              "tflops_bf16": flop / (kms / 1e3) / 1e12,
                              "tensor_frac": flop / (kms / 1e3) / 1e12 / bf16_peak,
                              "s_gbs": nbytes / (kms / 1e3) / 1e9, "hbm_frac": nbytes / (kms / 1e3) / 1e9 / hbm,
                              "bound": "tensor" if flop / (bf16_peak * 1e12) > nbytes / (hbm * 1e9) else "hbm"})
                qn = q.cpu().numpy()
                if q_prev is not None:
                    r["rel_diff_vs_fp32"] = float(np.linalg.norm(qn - q_prev) / np.linalg.norm(q_prev))
                q_prev = qn
                row[prec] = r
            row["bf16x3_speedup_vs_fp32"] = row["fp32"]["update_ms"] / row["bf16x3"]["update_ms"]
            res[f"m{m}"] = row
        ctx.close()
        out[str(n)] = res
    out["peaks"] = {"bf16_tflops": bf16_peak, "hbm_gbs": hbm, "source": src}
    out["l2"] = "flushed before every update"
    return out


def bench_serving(torch, s, k_prec="f16x2", n_req=20000, rates=(2000.0, 8000.0, 32000.0, None), phases=8,
                  max_batch=16, p3m_large=False):
    """Configuration 4: a Poisson stream of charge-update requests over four slab geometries (two
    graphene electrodes of two sheets, 512, 2,048, 8,192 and 16,384 sites), each request with its
    own electrolyte (0.5, 1, 1.5 or 2 charges per site: +-1 ions and 3-site water, drawn from four
    seeded configurations per geometry and density) and electrode potential difference ~ U[0, 2] V.
    20,000 requests per offered rate; the rate is swept up to saturation (None: all requests at
    t = 0).  The stream runs in phases: the two small geometries are always asked for, the 8,192-
    and 16,384-site ones alternate by phase, and the HBM budget holds the small ones with one large
    one but not both, so admission and eviction act at every phase change (an evicted geometry
    returns from its host-memory checkpoint).  Latency: arrival to result on the host.  With p3m_large
    the 8,192- and 16,384-site geometries take the reciprocal parts of b and of A from P3M (order 7,
    mesh by systems.with_p3m) instead of the Ewald sum."""
    from paper_2203_15461_gb300.serve import GpuBackend, Request, Scheduler, context_bytes, latency_stats, run_stream
    sizes = (512, 2048, 8192, 16384)
    keys = [f"graphene_{n}" for n in sizes]
    geoms = {k: s.serving_electrodes(n) for k, n in zip(keys, sizes)}
    if p3m_large:   # the same mesh operator for b and for the elastance (the package's pppm/electrode)
        for k in keys[2:]:
            geoms[k] = s.with_p3m(geoms[k], matrix=True)
    dens = (0.5, 1.0, 1.5, 2.0)
    t0 = time.perf_counter()
    pools = {k: [s.workload_serving_geometry(n, seed=40 + j, charges_per_site=c)[1] for j, c in enumerate(dens)]
             for k, n in zip(keys, sizes)}
    t_inputs = time.perf_counter() - t0
    ne_max = {k: max(e.n for e in pools[k]) for k in keys}
    be = GpuBackend(s_prec="fp32", k_prec=k_prec, max_batch=max_batch, ne_max=ne_max)
    # first admissions (assembly, inversion, host checkpoint) outside the measured streams
    t0 = time.perf_counter()
    meas = {}
    for k in keys:
        meas[k] = be.create(k, geoms[k])
        be.release(k)
    t_setup = time.perf_counter() - t0
    budget = meas[keys[0]] + meas[keys[1]] + max(meas[keys[2]], meas[keys[3]]) + (64 << 20)
    rng = np.random.default_rng(11)
    per_phase = n_req // phases
    out = {"workload": "cfg4: Poisson requests over 4 graphene slab geometries", "geometries": dict(zip(keys, sizes)),
           "requests_per_rate": n_req, "phases": phases, "max_batch": max_batch, "path": "mixed (FP32 S)",
           "k_prec": k_prec, "device_bytes": meas, "hbm_budget": budget, "input_seconds": t_inputs,
           "reciprocal_A_and_b": {k: (f"P3M {tuple(geoms[k].p3m_mesh)} order {geoms[k].p3m_order}"
                                      if geoms[k].p3m_order else "Ewald") for k in keys},
           "first_admission_seconds": t_setup, "runs": []}
    for rate in rates:
        reqs = []
        for i in range(n_req):
            ph = min(i // per_phase, phases - 1)
            big = keys[2] if ph % 2 == 0 else keys[3]
            k = (keys[0], keys[1], big)[int(rng.choice(3, p=(0.3, 0.3, 0.4)))]
            e = pools[k][int(rng.integers(len(dens)))]
            reqs.append(Request(rid=i, key=k, xyz=e.xyz, Q=e.Q, psi=np.array([0.0, rng.uniform(0.0, 2.0)])))
        sch = Scheduler(be, hbm_budget=budget, max_batch=max_batch)
        for k in keys:
            sch.add_geometry(k, geoms[k], meas[k])
        restores0 = be.restores
        arrivals = np.zeros(n_req) if rate is None else np.cumsum(rng.exponential(1.0 / rate, n_req))
        wall = run_stream(reqs, sch, arrivals=arrivals)
        for k in list(sch.resident):
            be.release(k)
        st = latency_stats(sch.finished)
        by = {}
        for k in keys:
            fk = [r for r in sch.finished if r.key == k]
            if fk:
                by[k] = {**latency_stats(fk), "requests": len(fk)}
        st.update({"offered_rate_per_s": rate if rate is not None else "all at t=0", "updates_per_s": n_req / wall,
                   "wall_s": wall, "admissions": sch.admissions, "evictions": sch.evictions,
                   "restores_from_host": be.restores - restores0, "peak_resident_bytes": sch.peak_bytes,
                   "max_abs_qtot": float(max(abs(r.qtot) for r in sch.finished)), "by_geometry": by})
        out["runs"].append(st)
    return out


P3M_MESH, P3M_ORDER = (32, 32, 128), 7


def bvec_once(torch, ctx, st, xyz_dev, Q_dev, m, ne):
    """b of m replicas (one cpm_bvec on the context's stream) as a host array."""
    with torch.cuda.stream(st):
        b = torch.empty((m, ctx.n), dtype=torch.float64, device="cuda")
        ctx.cpm_bvec(m, ne, xyz_dev, Q_dev, b)
    st.synchronize()
    return b.cpu().numpy()


def bench_p3m(torch, CPM, el, xyz_dev, Q_dev, psi_dev, m, ne, W, K, flush):
    """The headline step with the reciprocal part of b from P3M (mesh 32 x 32 x 128, order 7) instead of
    the Ewald sum: graph-captured step, kernel split, and b of replica 0 at the first timed step against
    the Ewald b (both FP64 on the GPU) and against the mixed P3M path."""
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        ctx = CPM.for_electrodes(el, s_prec="fp32", k_prec="fp32", stream=st, p3m=(P3M_MESH, P3M_ORDER)).setup(el)
    ms, launches, _, _ = time_graph(torch, ctx, st, xyz_dev, Q_dev, psi_dev, m, ne, W, K, flush)
    with torch.cuda.stream(st):
        msp, _, prof, _, _ = time_path(torch, ctx, xyz_dev, Q_dev, psi_dev, m, ne, W, K, flush, profile=True)
    x1, Q1 = xyz_dev[W][:ne], Q_dev[:ne]
    b_mix = bvec_once(torch, ctx, st, x1, Q1, 1, ne)[0]
    ctx.close()
    st64 = torch.cuda.Stream()
    with torch.cuda.stream(st64):
        p64 = CPM.for_electrodes(el, s_prec="fp64", k_prec="fp64", stream=st64, p3m=(P3M_MESH, P3M_ORDER)).setup(el)
        e64 = CPM.for_electrodes(el, s_prec="fp64", k_prec="fp64", stream=st64).setup(el)
    b_p3m = bvec_once(torch, p64, st64, x1, Q1, 1, ne)[0]
    b_ew = bvec_once(torch, e64, st64, x1, Q1, 1, ne)[0]
    p64.close()
    e64.close()
    return {"workload": f"edl_capacitor_4320, {m} replicas per graph step, P3M mesh {P3M_MESH} order {P3M_ORDER}",
            "value": m * K / (ms / 1e3), "unit": "updates/s", "ms_per_step": ms / K, "gpu_launches": int(launches),
            "kernel_ms_per_step": {kk: v[0] / K for kk, v in prof.items() if v[1]},
            "ms_per_step_kernel_by_kernel": msp / K,
            "b_rel_diff_p3m_vs_ewald_fp64": rel_l2(b_p3m, b_ew),
            "b_rel_diff_mixed_vs_fp64_p3m": rel_l2(b_mix, b_p3m),
            "path": "mixed: FP32 real space, FP32 P3M (fixed-point charge assignment, FP32 transforms), FP32 S"}, b_p3m


def edl_first_config(s, xyz, Q, ne, step):
    """Replica 0 of the headline trajectories at one step, as an electrolyte of its own."""
    return s.Electrolyte(xyz=np.ascontiguousarray(xyz[step, :ne]), Q=np.ascontiguousarray(Q[:ne]))


def run_reference(args):
    """--impl reference: the FP64 CPU oracle on the host cores, as it stands: every step is one
    complete, unsampled update of one headline configuration (b at every site over all host cores
    in site chunks, then q = S (v - b)); S from the oracle once beforehand (not timed)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2203_15461_gb300 import systems as s
    el, _, psi = s.workload_edl_capacitor(seed=1)
    W, K = args.warmup, args.steps
    xyz, Q, ne = make_trajectories(el, lambda sd: s.workload_edl_capacitor(seed=sd)[1], 1, W + K, rank_seed(0))
    pool = OraclePool()
    try:
        t0 = time.perf_counter()
        S = pool.capacitance(el)
        t_S = time.perf_counter() - t0
        walls = []
        for t in range(W + K):
            _, _, wall, _ = pool.update(el, edl_first_config(s, xyz, Q, ne, t), psi, S)
            if t >= W:
                walls.append(wall)
    finally:
        pool.close()
    tot = sum(walls)
    val = K / tot
    line = {"metric": METRIC, "value": val, "unit": "updates/s", "n_gpus": args.gpus, "steps": K,
            "warmup": W, "ms_per_step": 1e3 * tot / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_sites": el.n, "n_charges": ne, "replicas_per_step": 1},
            "impl": "reference",
            "cpu_baseline": {"value": val, "unit": "updates/s", "cores": pool.procs, "kind": "oracle",
                             "sample": (f"per step one complete, unsampled FP64 oracle update of the EDL capacitor "
                                        f"(4,320 sites, {ne} charges, every k-vector) on {pool.procs} processes "
                                        f"over site chunks; S from the oracle once before the steps "
                                        f"({t_S:.1f} s, not timed)")},
            "e2e": {"value": val, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--replicas", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="headline, kernel split and end-to-end legs only")
    ap.add_argument("--k-prec", default="f16x2", choices=["fp32", "f16x2"],
                    help="b-vector arithmetic of the mixed path (f16x2: reciprocal sums on the tensor cores)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    args.steps = max(1, args.steps)
    if args.impl == "reference":
        return run_reference(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_2203_15461_gb300 import systems as s

    el, ely0, psi = s.workload_edl_capacitor(seed=1)
    m, K, W = args.replicas, args.steps, args.warmup
    seed = rank_seed(rank)
    T = K + W
    xyz, Q, ne = make_trajectories(el, lambda sd: s.workload_edl_capacitor(seed=sd)[1], m, T, seed)
    # the oracle's single-threaded full update of replica 0 at the first timed step runs beside the GPU
    # legs in a spawned process started before the first GPU call
    cpu_leg = rank == 0 and not args.no_cpu_baseline
    ely_ref = edl_first_config(s, xyz, Q, ne, W)
    serial = SerialOracle(el, ely_ref, psi) if cpu_leg else None

    import torch
    import torch.distributed as dist
    from paper_2203_15461_gb300.cpm import CPM
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    xyz_dev = torch.as_tensor(xyz, device="cuda")
    Q_dev = torch.as_tensor(Q, device="cuda")
    psi_dev = torch.as_tensor(np.tile(psi, (m, 1)), device="cuda")
    flush = L2Flush(torch)

    t_setup = time.perf_counter()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        mixed = CPM.for_electrodes(el, s_prec="fp32", k_prec=args.k_prec, stream=st).setup(el)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    plain = CPM.for_electrodes(el, s_prec="fp64", k_prec="fp64").setup(el)
    nk = int(len(mixed.cpm_kvectors()))

    # mixed, batched: the headline
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ms, launches, q_mix, _ = time_graph(torch, mixed, st, xyz_dev, Q_dev, psi_dev, m, ne, W, K, flush)
    value, ms_max = aggregate(ms, m, K, world, dist if world > 1 else None)

    # end to end through the public host-buffer call: per step the caller's positions, charges and
    # potentials go host -> device from pinned buffers, the captured step replays (cpm_step_host on a
    # context with its own stream) and q and the totals come back to pinned host buffers
    hx = torch.empty((m * ne, 3), dtype=torch.float64).pin_memory()
    hQ = torch.as_tensor(Q).pin_memory()
    hpsi = torch.as_tensor(np.tile(psi, (m, 1))).pin_memory()
    hq = torch.empty((m, el.n), dtype=torch.float64).pin_memory()
    hqt = torch.empty((m,), dtype=torch.float64).pin_memory()
    xyz_host = torch.as_tensor(xyz)
    for t in range(W):
        hx.copy_(xyz_host[t % T])
        mixed.cpm_step_host(m, ne, hx, hQ, hpsi, hq, hqt)
    e2e_times = []
    for t in range(K):
        hx.copy_(xyz_host[(W + t) % T])   # the caller's new positions, already in its pinned buffer
        t0 = time.perf_counter()
        mixed.cpm_step_host(m, ne, hx, hQ, hpsi, hq, hqt)
        e2e_times.append(time.perf_counter() - t0)
    e2e_value, _ = aggregate(1e3 * sum(e2e_times), m, K, world, dist if world > 1 else None)   # max over ranks
    if rank != 0:
        # only rank 0 reports: the other ranks leave after the timed headline and end-to-end legs
        dist.barrier()
        dist.destroy_process_group()
        return 0
    e2e = {"value": e2e_value, "unit": "updates/s",
           "h2d_bytes_per_step": int(8 * (m * ne * 4 + m * el.n_groups)),
           "d2h_bytes_per_step": int(8 * (m * el.n + m)),
           "path": "cpm_step_host (C ABI, host buffers) on pinned torch buffers: H2D copies, the captured step "
                   "replayed, D2H of q and the totals, synchronised; wall clock per call"}

    # the same steps launched kernel by kernel with CUDA events around each kernel: the per-kernel split
    with torch.cuda.stream(st):
        ms_prof, _, prof, _, _ = time_path(torch, mixed, xyz_dev, Q_dev, psi_dev, m, ne, W, K, flush, profile=True)
    # the headline with the reciprocal sums on the CUDA cores (--k-prec fp32) beside it
    other_k = "fp32" if args.k_prec == "f16x2" else "f16x2"
    st2 = torch.cuda.Stream()
    with torch.cuda.stream(st2):
        mixed2 = CPM.for_electrodes(el, s_prec="fp32", k_prec=other_k, stream=st2).setup(el)
    ms2, _, _, _ = time_graph(torch, mixed2, st2, xyz_dev, Q_dev, psi_dev, m, ne, W, K, flush)
    mixed2.close()

    # plain FP64, one replica per step (the 1x of the metric), with its kernel split
    K64 = max(3, min(K, 10))
    x1, Q1, ne1 = xyz_dev[:, :ne], Q_dev[:ne], ne
    ms64, _, prof64, q64, _ = time_path(torch, plain, x1, Q1, psi_dev[:1], 1, ne1, 3, K64, flush, profile=True)
    fp64_value = K64 / (ms64 / 1e3)
    # mixed, one replica per step (configuration 2's sequential MD updates)
    with torch.cuda.stream(st):
        ms1, _, _, q1, _ = time_path(torch, mixed, x1, Q1, psi_dev[:1], 1, ne1, 3, K, flush)
    seq_value = K / (ms1 / 1e3)
    # the same sequential updates as the captured step (cpm_step_graph: what an MD code calls per step)
    ms1g, _, _, _ = time_graph(torch, mixed, st, x1, Q1, psi_dev[:1], 1, ne1, 3, K, flush)
    seq_graph_value = K / (ms1g / 1e3)
    # mixed and FP64 on replica 0 at the first timed step (the configuration the oracle leg updates)
    _, _, _, qa, qta = time_path(torch, plain, x1[W:W + 1], Q1, psi_dev[:1], 1, ne1, 0, 1, flush)
    with torch.cuda.stream(st):
        _, _, _, qb, qtb = time_path(torch, mixed, x1[W:W + 1], Q1, psi_dev[:1], 1, ne1, 0, 1, flush)
    st.synchronize()
    q64_ref, qmix_ref = qa[0].cpu().numpy(), qb[0].cpu().numpy()
    err_mixed = rel_l2(qmix_ref, q64_ref)
    qtot_max = float(max(abs(qta).max(), abs(qtb).max()))

    peaks, src = _peaks()
    alu_peak = _fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
    alu_src = f"FP32 FMA issue rate 152 SM x 128 lanes x 2 x {peaks.get('sm_max_mhz', 2070.0)} MHz"
    pairs = real_pairs(el, xyz, Q, ne, m, W)
    work = kernel_work(el, nk, ne, m, pairs, tensor=args.k_prec == "f16x2")
    kname = {"real": "k_real_blk", "sf": "k_tc_sf" if args.k_prec == "f16x2" else "k_sf32",
             "site": "k_tc_site" if args.k_prec == "f16x2" else "k_site32", "gemv": "k_gemv_tma"}
    top, roof = roofline(prof, work, peaks, src, kname, alu_peak, alu_src, ms_prof)
    roof["pairs_in_rcut_per_launch"] = pairs
    roof["flop_per_unit"] = {"real_pair": FLOP_PAIR, "sf_charge_k": FLOP_SF, "site_k": FLOP_SITE,
                             "tensor_complex_mac": FLOP_CMAC}
    # DRAM bytes (read + write) per launch from the committed ncu capture of these kernels on this
    # workload (cold caches); a stored figure, not measured by this run
    traffic_ncu = {"sf": 58.60e6, "site": 15.56e6, "gemv": 75.07e6, "real": 1.42e6}
    roof["traffic"] = traffic_ncu.get(top)
    roof["traffic_source"] = ("stored: ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch, "
                              "profiles/launches_edl_capacitor_4320.md")
    pairs1 = real_pairs(el, xyz, Q, ne, 1, W)
    work64 = kernel_work(el, nk, ne, 1, pairs1, tensor=False, s_bytes=8)
    k64 = {"real": "k_real_b<double>", "sf": "k_sf<double>", "site": "k_site<double>", "gemv": "k_gemv_t<double>"}
    fp64_peak = 1.25   # nominal GB300 FP64 rate (TFLOP/s); no measured FP64 peak on this machine
    _, roof64 = roofline(prof64, work64, peaks, src, k64, fp64_peak, "nominal GB300 FP64 rate, 1.25 TFLOP/s", ms64)

    line = {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_sites": el.n, "n_charges": ne, "n_kvectors": nk,
                       "replicas_per_step": m, "k_prec": args.k_prec,
                       "path": ("mixed: FP32 b (reciprocal sums as fp16x2 tensor-core products) and S, FP64 "
                                "neutrality and totals" if args.k_prec == "f16x2" else
                                "mixed: FP32 b and S, FP64 neutrality and totals"),
                       "boundary": "slab EW3DC", "alpha": el.alpha, "rcut": el.rcut,
                       "l2": "flushed before every timed step (256 MB write, then a 256 MB read of a second "
                             "buffer so the flush's dirty lines are written back outside the timed region)",
                       "parallelism": f"replicas x{world}",
                       "launch": "one CUDA graph per step (cpm_step_graph), positions copied in place"},
            "e2e": e2e, "gpu_launches": int(launches), "roofline": roof,
            f"value_k_prec_{other_k}": m * K / (ms2 / 1e3),
            "fp64_value": fp64_value, "speedup_vs_fp64": value / fp64_value,
            "fp64_kernel_ms_per_step": {kk: v[0] / K64 for kk, v in prof64.items()}, "fp64_roofline": roof64,
            "cfg2_sequential": {"workload": "edl_capacitor_4320, one replica, sequential updates (MD semantics)",
                                "mixed_value": seq_value, "mixed_graph_value": seq_graph_value,
                                "fp64_value": fp64_value, "unit": "updates/s",
                                "paths": "mixed_value: cpm_bvec + cpm_update launched kernel by kernel; "
                                         "mixed_graph_value: the captured step (cpm_step_graph)"},
            "rel_err_mixed_vs_fp64": err_mixed, "max_abs_qtot": qtot_max, "setup_seconds": t_setup,
            "kernel_ms_per_step": {kk: v[0] / K for kk, v in prof.items()},
            "ms_per_step_kernel_by_kernel": ms_prof / K}
    plain.close()
    mixed.close()
    clocks = clk.summary()
    line["clocks"] = clocks

    if not args.no_extra:
        cfg1, cfg1_q = bench_tiny_flow(torch, CPM, s)
        cfg3, cfg3_q = bench_batched_tiny(torch, CPM, s, flush, K, W, k_prec=args.k_prec)
        line["cfg1_tiny_fp64"] = cfg1
        line["cfg3_batched_tiny_256"] = cfg3
        line["cfg4_serving"] = bench_serving(torch, s, k_prec=args.k_prec)
        line["cfg4_serving_p3m_large"] = bench_serving(torch, s, k_prec=args.k_prec, rates=(8000.0, 32000.0, None),
                                                       p3m_large=True)
        line["cfg5_coax_12000"] = bench_coax(torch, CPM, s)
        sp = bench_s_products(torch, CPM, s, flush, peaks, src)
        line["s_products"] = sp
        f16 = sp.get("16384", {}).get("m8", {}).get("fp32", {})
        line["s_stream_16384"] = {"kernel": "k_gemv_tma", "replicas": 8, "ms_per_launch": f16.get("kernel_ms"),
                                  "achieved_gbs": f16.get("achieved_gbs"), "frac": f16.get("hbm_frac"),
                                  "hbm_peak_gbs": float(peaks["hbm_gbs"]), "l2": "flushed before every update"}
        line["p3m_edl_4320"], b_p3m0 = bench_p3m(torch, CPM, el, xyz_dev, Q_dev, psi_dev, m, ne, W, K, flush)

    if cpu_leg:
        pool = OraclePool()
        try:
            cb, _, q_or = cpu_baseline_edl(pool, serial, el, ely_ref, psi)
            cb["rel_err_vs_oracle"] = {"mixed_headline_path": rel_l2(qmix_ref, q_or), "fp64_path": rel_l2(q64_ref, q_or)}
            if not args.no_extra:   # the GPU's FP64 P3M b against the oracle's P3M b (same mesh and order)
                el_p = s.Electrodes(**{**el.__dict__, "p3m_mesh": P3M_MESH, "p3m_order": P3M_ORDER})
                line["p3m_edl_4320"]["b_rel_err_fp64_vs_oracle"] = rel_l2(b_p3m0, oracle_bvec(el_p, ely_ref))
            if not args.no_extra:
                el_t, last, psis, qs = cfg3_q
                el1, conf1, psi1, q1last = cfg1_q
                tiny = dict(last)
                tiny[-1] = conf1
                psis = dict(psis)
                psis[-1] = psi1
                q_small, c0_10 = cpu_baseline_small(pool, el_t, tiny, psis,
                                                    s.coaxial_tubes(10, alpha=0.15, rcut=24.0, ktol=1e-8))
                line["cfg1_tiny_fp64"]["rel_err_vs_oracle"] = rel_l2(q1last, q_small[-1])
                line["cfg3_batched_tiny_256"]["rel_err_vs_oracle"] = {
                    sp: max(rel_l2(qs[sp][r], q_small[r]) for r in last) for sp in qs}
                line["cfg3_batched_tiny_256"]["rel_err_replicas_checked"] = sorted(last)
                c5 = line["cfg5_coax_12000"]
                c5["C0_per_L_oracle_10_cells"] = c0_10
                c5["rel_err_vs_oracle_fp64"] = abs(c5["C0_per_L_fp64"] / c0_10 - 1.0)
                c5["rel_err_vs_oracle_fp32_ir"] = abs(c5["C0_per_L_fp32_ir"] / c0_10 - 1.0)
        finally:
            pool.close()
        line["cpu_baseline"] = cb
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
