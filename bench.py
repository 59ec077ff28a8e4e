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


def kernel_work(ctx, el, nk, ne, m, pairs=None, tensor=False):
    """Algorithmic work per launch of the per-step kernels (flops or bytes).

    With ``tensor`` the two reciprocal contractions run on the tensor cores ("tflop": the same
    algorithmic flops, measured against the tensor-core peak of the emulated FP32 product)."""
    n = el.n
    fk = "tflop" if tensor else "flop"
    w = {
        "sf": (fk, 8.0 * ne * nk * m),                # one complex multiply-add per (charge, k)
        "site": (fk, 8.0 * n * nk * m),               # one complex multiply-add per (site, k)
        "gemv": ("byte", 4.0 * n * n * ((m + 7) // 8)),   # S streamed once (FP32) per 8 replicas
    }
    if pairs is not None:
        w["real"] = ("flop", 16.0 * pairs)            # tabulated pair function per pair inside rcut
    return w


def cpu_baseline(el, ely, psi, frac=8):
    """The oracle's update, timed on a bounded sample and scaled to one full update."""
    from oracle import cpm_oracle as o
    sites = np.arange(0, el.n, frac)
    box = np.asarray(el.box)
    V = float(np.prod(box))
    _, k, k2 = o.kvectors(box, el.kcut)
    ksub = np.arange(0, len(k), frac)
    t0 = time.perf_counter()
    bre = o.bvec(type(el)(**{**el.__dict__, "kcut": 1e-9}), ely, sites=sites)      # real space (+ tiny terms)
    t1 = time.perf_counter()
    rho = o.structure_factor(k[ksub], ely)
    t2 = time.perf_counter()
    w = o.kweights(k2[ksub], el.alpha, V)
    ph = el.xyz[sites] @ k[ksub].T
    _ = (np.cos(ph) * rho.real + np.sin(ph) * rho.imag) @ w
    t3 = time.perf_counter()
    Sfake = np.eye(el.n)
    v = o.site_potentials(el, psi)
    t4 = time.perf_counter()
    _ = Sfake @ (v - np.zeros(el.n))
    t5 = time.perf_counter()
    per_update = (t1 - t0) * frac + (t2 - t1) * frac + (t3 - t2) * frac * frac + (t5 - t4)
    return {"value": 1.0 / per_update, "unit": "updates/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"numpy FP64 oracle on the same system: real-space b at 1/{frac} of the sites, structure "
                       f"factor over 1/{frac} of the k-vectors, site k-sum over both subsets, one n x n matvec; "
                       f"each part scaled by its sampled fraction to one full update (elementwise numpy on one "
                       f"thread, BLAS on {os.cpu_count()})"),
            "sample_seconds": t5 - t0}


def bench_batched_tiny(torch, CPM, s, flush, K, W, m=256, k_prec="fp32"):
    """256 replicas of the 216-site Au(111) capacitor per step (one shared S), graph-captured."""
    el, _, psi = s.workload_tiny_slab(seed=1)
    xyz, Q, ne = make_trajectories(el, lambda sd: s.ions_in_gap(el, 100, seed=sd), m, K + W, 5000)
    out = {"workload": "au111_tiny_216 x 256 replicas", "replicas_per_step": m, "k_prec": k_prec}
    for s_prec in ("fp32", "bf16x3"):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx = CPM.for_electrodes(el, s_prec=s_prec, k_prec=k_prec, stream=st).setup(el)
            dx = torch.as_tensor(xyz[0], device="cuda").clone()
            dQ = torch.as_tensor(Q, device="cuda")
            dp = torch.as_tensor(np.tile(psi, (m, 1)), device="cuda")
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
        ctx.close()
    out["unit"] = "updates/s"
    return out


def bench_s_stream(torch, CPM, s, flush, peaks, K=10, W=3, m=8):
    """The single-precision S product alone at the size where S is far larger than L2: two graphene
    electrodes of two sheets, 16,384 sites (S32 = 1.07 GB), assembled with a small Ewald alpha (0.1,
    r_c = 35 A: few k-vectors, the assembly stays short; the S product does not depend on the split).
    b is random; per update the library's profiler times the S stream (k_gemv_tma) on the context
    stream, with L2 flushed before every update."""
    import time as _t
    el = s.graphene_plates(32, 32, 2, 40.0, alpha=0.1, rcut=35.0)
    n = el.n
    t0 = _t.perf_counter()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        ctx = CPM.for_electrodes(el, s_prec="fp32", k_prec="fp32", stream=st).setup(el)
    st.synchronize()
    setup_s = _t.perf_counter() - t0
    rng = np.random.default_rng(7)
    with torch.cuda.stream(st):
        b = torch.as_tensor(rng.normal(0.0, 1.0, (m, n)), device="cuda")
        psi = torch.as_tensor(np.tile([0.0, 1.0], (m, 1)), device="cuda")
        q = torch.empty((m, n), dtype=torch.float64, device="cuda")
        qt = torch.empty(m, dtype=torch.float64, device="cuda")
    for _ in range(W):
        with torch.cuda.stream(st):
            ctx.cpm_update(m, psi, b, q, qt)
    st.synchronize()
    ctx.cpm_profile_read(reset=True)
    ctx.cpm_profile(True)
    for _ in range(K):
        with torch.cuda.stream(st):
            flush()
            ctx.cpm_update(m, psi, b, q, qt)
    st.synchronize()
    ctx.cpm_profile(False)
    prof = ctx.cpm_profile_read(reset=True)
    ms = prof["gemv"][0] / max(1, prof["gemv"][1])
    nbytes = 4.0 * n * n
    gbs = nbytes / (ms / 1e3) / 1e9
    hbm = float(peaks["hbm_gbs"])
    ctx.close()
    return {"workload": f"graphene 32x32, 2 sheets per electrode: {n} sites, {m} replicas per pass",
            "kernel": "k_gemv_tma", "s_bytes": nbytes, "ms_per_launch": ms, "achieved_gbs": gbs,
            "hbm_peak_gbs": hbm, "frac": gbs / hbm, "max_abs_qtot": float(qt.abs().max()),
            "setup_seconds": setup_s, "l2": "flushed before every update"}


def bench_serving(torch, s, n_req=600, rate=4000.0, k_prec="fp32"):
    """Poisson stream of charge-update requests over three slab geometries (216, 512 and 2,048 sites)."""
    from paper_2203_15461_gb300.serve import GpuBackend, Request, Scheduler, context_bytes, latency_stats, run_stream
    geoms = {"au111_216": s.workload_tiny_slab(seed=1)[0], "graphene_512": s.workload_serving_geometry(512)[0],
             "graphene_2048": s.workload_serving_geometry(2048)[0]}
    be = GpuBackend(s_prec="fp32", k_prec=k_prec, max_batch=16)
    sch = Scheduler(be, hbm_budget=4 << 30, max_batch=16)
    for k, el in geoms.items():
        sch.add_geometry(k, el, context_bytes(el.n, 2 * el.n, 16))
    rng = np.random.default_rng(11)
    pools = {k: [s.workload_serving_geometry(el.n, seed=40 + j)[1] if k != "au111_216" else
                 s.ions_in_gap(el, 100, seed=40 + j) for j in range(8)] for k, el in geoms.items()}
    keys = list(geoms)
    reqs = []
    for i in range(n_req):
        k = keys[int(rng.integers(len(keys)))]
        e = pools[k][int(rng.integers(8))]
        reqs.append(Request(rid=i, key=k, xyz=e.xyz + rng.normal(scale=0.05, size=e.xyz.shape), Q=e.Q,
                            psi=np.array([0.0, rng.uniform(0.0, 2.0)])))
    # warm the three contexts outside the measured stream
    warm = [Request(rid=-1 - j, key=k, xyz=pools[k][0].xyz, Q=pools[k][0].Q, psi=np.zeros(2)) for j, k in enumerate(keys)]
    run_stream(warm, sch, arrivals=np.zeros(len(warm)))
    sch.finished.clear()
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    wall = run_stream(reqs, sch, arrivals=arrivals)
    st = latency_stats(sch.finished)
    st.update({"requests": n_req, "offered_rate_per_s": rate, "updates_per_s": n_req / wall,
               "geometries": {k: el.n for k, el in geoms.items()}, "max_batch": 16, "path": "mixed",
               "k_prec": k_prec})
    return st


def run_reference(args):
    """--impl reference: the FP64 CPU oracle on the host cores, same workload, sampled per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2203_15461_gb300 import systems as s
    el, ely, psi = s.workload_edl_capacitor(seed=1)
    samples = []
    for t in range(args.warmup + args.steps):
        r = cpu_baseline(el, s.jitter(ely, 0.05, np.random.default_rng(t)), psi)
        if t >= args.warmup:
            samples.append(1.0 / r["value"])
    tot = sum(samples)
    val = args.steps / tot
    line = {"metric": METRIC, "value": val, "unit": "updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_sites": el.n, "n_charges": ely.n, "replicas_per_step": 1},
            "impl": "reference",
            "cpu_baseline": {"value": val, "unit": "updates/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": val, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--replicas", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--k-prec", default="f16x2", choices=["fp32", "f16x2"],
                    help="b-vector arithmetic of the mixed path (f16x2: reciprocal sums on the tensor cores)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    args.steps = max(1, args.steps)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_2203_15461_gb300 import systems as s
    from paper_2203_15461_gb300.cpm import CPM

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    el, ely0, psi = s.workload_edl_capacitor(seed=1)
    m, K, W = args.replicas, args.steps, args.warmup
    seed = rank_seed(rank)
    T = K + W
    xyz, Q, ne = make_trajectories(el, lambda sd: s.workload_edl_capacitor(seed=sd)[1], m, T, seed)
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
    # the same steps launched kernel by kernel with CUDA events around each kernel: the per-kernel split
    with torch.cuda.stream(st):
        ms_prof, _, prof, _, _ = time_path(torch, mixed, xyz_dev, Q_dev, psi_dev, m, ne, W, K, flush, profile=True)

    # plain FP64, one replica per step (the 1x of the metric)
    K64 = max(3, min(K, 10))
    x1, Q1, ne1 = xyz_dev[:, :ne], Q_dev[:ne], ne
    ms64, _, _, q64, _ = time_path(torch, plain, x1, Q1, psi_dev[:1], 1, ne1, 3, K64, flush)
    fp64_value = K64 / (ms64 / 1e3)
    # mixed, one replica per step
    with torch.cuda.stream(st):
        ms1, _, _, q1, _ = time_path(torch, mixed, x1, Q1, psi_dev[:1], 1, ne1, 3, K, flush)
    seq_value = K / (ms1 / 1e3)
    # mixed vs FP64 on the same configuration
    _, _, _, qa, qta = time_path(torch, plain, x1[:1], Q1, psi_dev[:1], 1, ne1, 0, 1, flush)
    with torch.cuda.stream(st):
        _, _, _, qb, qtb = time_path(torch, mixed, x1[:1], Q1, psi_dev[:1], 1, ne1, 0, 1, flush)
    st.synchronize()
    err_mixed = float(torch.linalg.norm(qb[0] - qa[0]) / torch.linalg.norm(qa[0]))
    qtot_max = float(max(abs(qta).max(), abs(qtb).max()))

    # end to end through the public API: per step the inputs go host -> device from pinned buffers,
    # the graph-captured step runs (cpm_step_graph), and q and the totals come back to the host
    hx = torch.empty((m * ne, 3), dtype=torch.float64).pin_memory()
    hQ = torch.as_tensor(Q).pin_memory()
    hpsi = torch.as_tensor(np.tile(psi, (m, 1))).pin_memory()
    hq = torch.empty((m, el.n), dtype=torch.float64).pin_memory()
    hqt = torch.empty((m,), dtype=torch.float64).pin_memory()
    with torch.cuda.stream(st):
        ex = torch.empty((m * ne, 3), dtype=torch.float64, device="cuda")
        eQ = torch.empty((m * ne,), dtype=torch.float64, device="cuda")
        ep = torch.empty((m, el.n_groups), dtype=torch.float64, device="cuda")
        eb = torch.empty((m, el.n), dtype=torch.float64, device="cuda")
        eq = torch.empty((m, el.n), dtype=torch.float64, device="cuda")
        eqt = torch.empty((m,), dtype=torch.float64, device="cuda")
    xyz_host = torch.as_tensor(xyz)

    def e2e_step():
        with torch.cuda.stream(st):
            ex.copy_(hx, non_blocking=True)
            eQ.copy_(hQ, non_blocking=True)
            ep.copy_(hpsi, non_blocking=True)
            mixed.cpm_step_graph(m, ne, ex, eQ, ep, eb, eq, eqt)
            hq.copy_(eq, non_blocking=True)
            hqt.copy_(eqt, non_blocking=True)
        st.synchronize()

    for t in range(W):
        hx.copy_(xyz_host[t % T])
        e2e_step()
    e2e_times = []
    for t in range(K):
        hx.copy_(xyz_host[(W + t) % T])   # the caller's new positions, already in its pinned buffer
        t0 = time.perf_counter()
        e2e_step()
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
           "path": "pinned host buffers -> cpm_step_graph -> pinned host buffers, wall clock per step"}

    # batched replicas of the tiny capacitor: 256 electrolytes sharing one S, one CUDA graph per step
    batched = bench_batched_tiny(torch, CPM, s, flush, K, W, k_prec=args.k_prec)
    # serving stream: Poisson arrivals over three geometries, continuous batching
    serving = bench_serving(torch, s, k_prec=args.k_prec)
    s_stream = bench_s_stream(torch, CPM, s, flush, _peaks()[0])

    # roofline of the dominant kernel
    peaks, src = _peaks()
    # DRAM bytes (read + write) per launch from one ncu capture of the current kernels on the full
    # workload (cold caches: ncu flushes them before each launch); None for a kernel not captured
    traffic_ncu = {"real": 0.75e6, "sf": 58.59e6, "site": 15.57e6, "gemv": 75.06e6}
    kname = {"real": "k_real_cells", "sf": "k_tc_sf" if args.k_prec == "f16x2" else "k_sf32",
             "site": "k_tc_site" if args.k_prec == "f16x2" else "k_site32", "gemv": "k_gemv_tma"}
    pairs = real_pairs(el, xyz, Q, ne, m, W)
    work = kernel_work(mixed, el, nk, ne, m, pairs, tensor=args.k_prec == "f16x2")
    top = max((kk for kk in prof if prof[kk][1] > 0), key=lambda kk: prof[kk][0])
    avg_ms = prof[top][0] / prof[top][1]
    kind, amount = work.get(top, ("flop", float("nan")))
    if kind == "tflop":
        # fp16 tensor rate = the measured bf16 rate (same nominal peak); three fp16 products per FP32 product
        peak = float(peaks.get("bf16_tflops", 1900.0)) / 3.0
        achieved = amount / (avg_ms / 1e3) / 1e12
        roof = {"kernel": kname.get(top, top), "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_ncu.get(top),
                "peak_source": f"bf16_tflops ({src}) / 3: two-term fp16 operands, three products per FP32 product"}
    elif kind == "flop":
        peak = _fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
        achieved = amount / (avg_ms / 1e3) / 1e12
        roof = {"kernel": kname.get(top, top), "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_ncu.get(top),
                "peak_source": f"FP32 FMA issue rate 152 SM x 128 lanes x 2 x {peaks.get('sm_max_mhz', 2070.0)} MHz"}
    else:
        peak = float(peaks["hbm_gbs"])
        achieved = amount / (avg_ms / 1e3) / 1e9
        roof = {"kernel": kname.get(top, top), "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic_ncu.get(top), "peak_source": f"hbm_gbs ({src})"}
    roof["share_of_step"] = prof[top][0] / ms_prof
    roof["all_kernels"] = {kk: {"ms_per_launch": prof[kk][0] / max(1, prof[kk][1]),
                                "achieved": (work[kk][1] / (prof[kk][0] / max(1, prof[kk][1]) / 1e3)
                                             / (1e9 if work[kk][0] == "byte" else 1e12)),
                                "unit": "GB/s" if work[kk][0] == "byte" else "TFLOP/s"}
                           for kk in work if kk in prof and prof[kk][1] > 0}
    roof["pairs_in_rcut_per_launch"] = pairs

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
            "fp64_value": fp64_value, "speedup_vs_fp64": value / fp64_value, "sequential_mixed_value": seq_value,
            "rel_err_mixed_vs_fp64": err_mixed, "max_abs_qtot": qtot_max, "setup_seconds": t_setup,
            "kernel_ms_per_step": {kk: v[0] / K for kk, v in prof.items()},
            "ms_per_step_kernel_by_kernel": ms_prof / K,
            "batched_tiny_256": batched, "serving": serving, "s_stream_16384": s_stream}
    clocks = clk.summary()
    line["clocks"] = clocks
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(el, ely0, psi)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
