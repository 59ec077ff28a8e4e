"""Continuous batching on the GPU: requests for two geometries arrive over time, are batched per geometry and
overlap on the device; every result equals the same request computed alone (within the path's tolerance)."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_l2, run_bvec, run_update, make_ctx
from paper_2203_15461_gb300 import systems as s
from paper_2203_15461_gb300.serve import GpuBackend, Request, Scheduler, context_bytes, latency_stats, run_stream

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_mixed_stream_equals_alone(prec, tol):
    need_gpu()
    geoms = {"tiny": s.workload_tiny_slab(seed=1)[0], "g512": s.workload_serving_geometry(512)[0]}
    be = GpuBackend(s_prec=prec, k_prec=prec, max_batch=8)
    sch = Scheduler(be, hbm_budget=2 << 30, max_batch=8)
    for k, el in geoms.items():
        sch.add_geometry(k, el, context_bytes(el.n, 600, 8))
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(40):
        key = "tiny" if i % 2 else "g512"
        el = geoms[key]
        ely = s.ions_in_gap(el, 100, seed=2000 + i) if key == "tiny" else s.workload_serving_geometry(512, seed=3000 + i)[1]
        reqs.append(Request(rid=i, key=key, xyz=ely.xyz, Q=ely.Q, psi=np.array([0.0, rng.uniform(0, 2)])))
    arrivals = np.sort(rng.uniform(0, 0.05, len(reqs)))
    run_stream(reqs, sch, arrivals=arrivals)
    assert len(sch.finished) == len(reqs)
    # each request alone, in its own fresh context, one replica per call
    alone = {k: make_ctx(el, s_prec=prec, k_prec=prec).setup(el) for k, el in geoms.items()}
    worst = 0.0
    for r in sch.finished:
        ctx = alone[r.key]
        b = run_bvec(ctx, [s.Electrolyte(xyz=r.xyz, Q=r.Q)])
        q, qt = run_update(ctx, r.psi, b)
        worst = max(worst, rel_l2(r.q, q[0]))
        assert abs(r.qtot) <= 1e-12
    assert worst <= tol, worst
    st = latency_stats(sch.finished)
    assert st["p99_ms"] >= st["p50_ms"] > 0
