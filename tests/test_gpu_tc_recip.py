"""Reciprocal-space b on the tensor cores (k_prec "f16x2"): the structure factor and the site potentials as
two-term fp16 products on tcgen05, everything else as in the single-precision path.

Checked against the oracle (b within 2e-6 relative L2 on ragged replicas, including a non-neutral one and
an empty electrolyte), against the CUDA-core single-precision path for replica counts that exercise every
layout of the site stage (one replica, non-power-of-two column groups, two replica blocks), and against the
FP64 path on the full-size EDL capacitor (b within 2e-6, q within 1e-5, neutral to 1e-12 e).
"""
import numpy as np
import pytest

from gpu_util import dev, make_ctx, need_gpu, rel_l2, run_bvec, run_update, torch
from oracle import cpm_oracle as o
from paper_2203_15461_gb300 import systems as s

pytestmark = pytest.mark.gpu


def test_tc_bvec_ragged_replicas_match_oracle():
    need_gpu()
    el, ely, _ = s.workload_tiny_slab(seed=3)
    e2 = s.ions_in_gap(el, 60, seed=11)
    e3 = s.Electrolyte(xyz=ely.xyz[:37], Q=ely.Q[:37])      # non-neutral: background term
    ctx = make_ctx(el, k_prec="f16x2").setup(el)
    b = run_bvec(ctx, [ely, e2, e3])
    for r, e in enumerate([ely, e2, e3]):
        assert rel_l2(b[r], o.bvec(el, e)) <= 2e-6
    empty = run_bvec(ctx, [s.Electrolyte(xyz=np.zeros((0, 3)), Q=np.zeros(0))])
    assert np.abs(empty).max() == 0.0


@pytest.mark.parametrize("m", [1, 3, 20, 130])
def test_tc_bvec_layouts_match_cuda_core_path(m):
    need_gpu()
    el, _, psi = s.workload_tiny_slab(seed=3)
    elyts = [s.ions_in_gap(el, 40 + 7 * (r % 9), seed=700 + r) for r in range(m)]
    c32 = make_ctx(el, k_prec="fp32").setup(el)
    ctc = make_ctx(el, k_prec="f16x2").setup(el)
    b32 = run_bvec(c32, elyts)
    btc = run_bvec(ctc, elyts)
    for r in range(m):
        assert rel_l2(btc[r], b32[r]) <= 2e-6, r
    for r in sorted({0, m // 2, m - 1}):
        assert rel_l2(btc[r], o.bvec(el, elyts[r])) <= 2e-6, r


def test_tc_bvec_wire_coax_matches_oracle():
    """Wire geometry (z-periodic coaxial tubes): another column layout and the EW3DC wire term."""
    need_gpu()
    el = s.coaxial_tubes(2)
    rng = np.random.default_rng(2)
    ely = s.Electrolyte(xyz=np.column_stack([rng.uniform(35, 45, 20), rng.uniform(35, 45, 20),
                                             rng.uniform(0, el.box[2], 20)]), Q=np.tile([1.0, -1.0], 10))
    ctx = make_ctx(el, k_prec="f16x2").setup(el)
    b = run_bvec(ctx, [ely])
    assert rel_l2(b[0], o.bvec(el, ely)) <= 2e-6


def test_tc_edl_capacitor_against_fp64():
    need_gpu()
    el, ely, psi = s.workload_edl_capacitor(seed=1)
    elyts = [s.jitter(ely, 0.05, np.random.default_rng(r)) for r in range(8)]
    c64 = make_ctx(el).setup(el)
    ctc = make_ctx(el, s_prec="fp32", k_prec="f16x2").setup(el)
    b64 = run_bvec(c64, elyts)
    btc = run_bvec(ctc, elyts)
    q64, _ = run_update(c64, psi, b64)
    qtc, qt = run_update(ctc, psi, btc)
    for r in range(len(elyts)):
        assert rel_l2(btc[r], b64[r]) <= 2e-6, r
        assert rel_l2(qtc[r], q64[r]) <= 1e-5, r
    assert np.abs(qt).max() <= 1e-12
    sites = np.random.default_rng(2).choice(el.n, 8, replace=False)
    assert rel_l2(btc[0][sites], o.bvec(el, elyts[0], sites=sites)) <= 2e-6


def test_tc_step_graph_equals_separate_calls():
    need_gpu()
    el, _, psi = s.workload_tiny_slab(seed=3)
    elyts = [s.ions_in_gap(el, 100, seed=900 + r) for r in range(16)]
    st = torch.cuda.Stream()
    ctx = make_ctx(el, s_prec="fp32", k_prec="f16x2", stream=st).setup(el)
    from gpu_util import stack_replicas
    xyz, Q, n_e = stack_replicas(elyts)
    m = len(elyts)
    b = torch.empty((m, ctx.n), dtype=torch.float64, device="cuda")
    q = torch.empty((m, ctx.n), dtype=torch.float64, device="cuda")
    qt = torch.empty((m,), dtype=torch.float64, device="cuda")
    dx, dQ, dp = dev(xyz), dev(Q), dev(np.tile(psi, (m, 1)))
    with torch.cuda.stream(st):
        for _ in range(2):
            ctx.cpm_step_graph(m, n_e, dx, dQ, dp, b, q, qt)
    st.synchronize()
    b_ref = run_bvec(ctx, elyts)
    q_ref, _ = run_update(ctx, psi, b_ref)
    assert np.array_equal(b.cpu().numpy(), b_ref)
    assert np.array_equal(q.cpu().numpy(), q_ref)


@pytest.mark.parametrize("k_prec", ["fp32", "f16x2"])
def test_three_stream_b_equals_one_stream_order(k_prec):
    """The electrolyte vector runs as three chains on side streams; with the library's per-kernel
    profiling on, the same kernels run on the context stream alone.  Both orders give bit-identical
    b and q (the chains touch disjoint scratch and every reduction has a fixed order)."""
    need_gpu()
    el, _, psi = s.workload_tiny_slab(seed=3)
    elyts = [s.ions_in_gap(el, 90, seed=1300 + r) for r in range(5)]
    ctx = make_ctx(el, s_prec="fp32", k_prec=k_prec).setup(el)
    b_fork = run_bvec(ctx, elyts)
    q_fork, qt_fork = run_update(ctx, psi, b_fork)
    ctx.cpm_profile(True)
    b_one = run_bvec(ctx, elyts)
    q_one, qt_one = run_update(ctx, psi, b_one)
    ctx.cpm_profile(False)
    assert np.array_equal(b_fork, b_one)
    assert np.array_equal(q_fork, q_one)
    assert np.array_equal(qt_fork, qt_one)
