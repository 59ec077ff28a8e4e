"""Charges of the fast paths against the FP64 oracle, element by element, at the sizes where the
production kernels run.

* The mixed path that the benchmark times (single-precision S streamed by the TMA kernel, which
  runs for n >= 256 with n a multiple of 4; reciprocal sums as two-term fp16 tensor-core products)
  on the 512- and 2,048-site serving geometries for 1, 3, 8 and 11 replicas (one and two replica
  chunks of the S stream), and on the full 4,320-site EDL capacitor with eight replicas through the
  graph-captured step (the benchmark's launch configuration) and one replica through the separate
  calls.
* The tensor-core S product (S and b as three bf16 terms each, tcgen05) with the oracle's own b as
  input, so the product alone is measured: the 216-site capacitor for 1, 20, 64 and 130 replicas,
  and the 2,048-site geometry for 64 and 128 replicas.
* The FP64 path at 2,048 sites.
* The 16,384-site serving geometry, where the oracle cannot form S: sampled rows of A and b give
  the stationarity residual of the FP64 path; the mixed path against the FP64 path.

Tolerances: relative L2 error of q at most 1e-5 (mixed) and 1e-10 (FP64) for every replica, total
electrode charge within 1e-12 e (Eq. S, Sec. II.A; Eq. electrode-wise, Sec. II.B).  The oracle
values come from ``oracle.cpm_oracle`` evaluated over the host's cores (``oracle_pool``).
"""
import numpy as np
import pytest

from gpu_util import dev, make_ctx, need_gpu, rel_l2, stack_replicas, torch
from oracle import cpm_oracle as o
from oracle_pool import OraclePool, oracle_S
from paper_2203_15461_gb300 import systems as s

pytestmark = pytest.mark.gpu

MIXED_TOL, FP64_TOL, QTOT_TOL = 1e-5, 1e-10, 1e-12


@pytest.fixture(scope="module")
def pool():
    need_gpu()
    with OraclePool() as p:
        yield p


def _psi(m):
    """Distinct electrode potentials per replica: (0, 0.4 + 0.13 r) V."""
    return np.column_stack([np.zeros(m), 0.4 + 0.13 * np.arange(m)])


def _q_ref(S, el, psi, b):
    return np.stack([o.charges(S, el, psi[r], b[r]) for r in range(len(b))])


def _bvec_update(ctx, elyts, psi):
    xyz, Q, n_e = stack_replicas(elyts)
    m = len(elyts)
    b = torch.empty((m, ctx.n), dtype=torch.float64, device="cuda")
    q = torch.empty_like(b)
    qt = torch.empty((m,), dtype=torch.float64, device="cuda")
    ctx.cpm_bvec(m, n_e, dev(xyz), dev(Q), b)
    ctx.cpm_update(m, dev(psi), b, q, qt)
    ctx.cpm_sync()
    return q.cpu().numpy(), qt.cpu().numpy()


def _update(ctx, b, psi):
    m = b.shape[0]
    q = torch.empty((m, ctx.n), dtype=torch.float64, device="cuda")
    qt = torch.empty((m,), dtype=torch.float64, device="cuda")
    ctx.cpm_update(m, dev(psi), dev(b), q, qt)
    ctx.cpm_sync()
    return q.cpu().numpy(), qt.cpu().numpy()


def _graph_step(el, elyts, psi, s_prec="fp32", k_prec="f16x2"):
    st = torch.cuda.Stream()
    ctx = make_ctx(el, s_prec=s_prec, k_prec=k_prec, stream=st).setup(el)
    xyz, Q, n_e = stack_replicas(elyts)
    m = len(elyts)
    with torch.cuda.stream(st):
        dx, dQ, dp = dev(xyz), dev(Q), dev(psi)
        b = torch.empty((m, el.n), dtype=torch.float64, device="cuda")
        q = torch.empty_like(b)
        qt = torch.empty((m,), dtype=torch.float64, device="cuda")
        for _ in range(2):   # capture, then replay
            ctx.cpm_step_graph(m, n_e, dx, dQ, dp, b, q, qt)
    ctx.cpm_sync()
    return q.cpu().numpy(), qt.cpu().numpy()


def _check(q, qt, q_ref, tol):
    errs = [rel_l2(q[r], q_ref[r]) for r in range(len(q_ref))]
    assert max(errs) <= tol, errs
    assert np.abs(qt).max() <= QTOT_TOL
    assert np.abs(q.sum(axis=1)).max() <= QTOT_TOL


# ----------------------------------------------------------------------------- serving geometries

@pytest.fixture(scope="module", params=[512, 2048], ids=["n512", "n2048"])
def serving(request, pool):
    n = request.param
    el, _, _ = s.workload_serving_geometry(n, seed=1)
    elyts = [s.workload_serving_geometry(n, seed=100 + r)[1] for r in range(11)]
    _, S = oracle_S(el, pool)
    b = np.stack(pool.bvec(el, elyts))
    return el, S, elyts, b


@pytest.mark.parametrize("m", [1, 3, 8, 11])
def test_headline_path_matches_oracle(serving, m):
    el, S, elyts, b = serving
    assert el.n % 4 == 0 and el.n >= 256          # the TMA S stream runs
    psi = _psi(m)
    ctx = make_ctx(el, s_prec="fp32", k_prec="f16x2").setup(el)
    q, qt = _bvec_update(ctx, elyts[:m], psi)
    _check(q, qt, _q_ref(S, el, psi, b[:m]), MIXED_TOL)


def test_headline_graph_step_matches_oracle(serving):
    el, S, elyts, b = serving
    psi = _psi(8)
    q, qt = _graph_step(el, elyts[:8], psi)
    _check(q, qt, _q_ref(S, el, psi, b[:8]), MIXED_TOL)


def test_single_precision_s_stream_alone_matches_oracle(serving):
    """The oracle's b as input: the S product of the TMA stream alone (two replica chunks)."""
    el, S, _, b = serving
    psi = _psi(11)
    ctx = make_ctx(el, s_prec="fp32", k_prec="fp32").setup(el)
    q, qt = _update(ctx, b, psi)
    _check(q, qt, _q_ref(S, el, psi, b), MIXED_TOL)


def test_fp64_path_matches_oracle(serving):
    el, S, elyts, b = serving
    psi = _psi(3)
    ctx = make_ctx(el).setup(el)
    q, qt = _bvec_update(ctx, elyts[:3], psi)
    _check(q, qt, _q_ref(S, el, psi, b[:3]), FP64_TOL)


@pytest.mark.parametrize("m", [64, 128])
def test_tensor_core_s_product_matches_oracle_2048(serving, m):
    el, S, _, b = serving
    if el.n != 2048:
        pytest.skip("the tensor-core product is checked at 2,048 sites")
    # m distinct b vectors from the oracle's eleven: scaled copies (q is linear in b)
    bm = np.stack([b[r % len(b)] * (1.0 + 0.01 * r) for r in range(m)])
    psi = _psi(m)
    ctx = make_ctx(el, s_prec="bf16x3").setup(el)
    q, qt = _update(ctx, bm, psi)
    _check(q, qt, _q_ref(S, el, psi, bm), MIXED_TOL)


# ----------------------------------------------------------------------------- 216-site capacitor

@pytest.fixture(scope="module")
def tiny(pool):
    el, _, _ = s.workload_tiny_slab(seed=1)
    elyts = [s.ions_in_gap(el, 100, seed=4000 + r) for r in range(130)]
    _, S = oracle_S(el)
    b = np.stack(pool.bvec(el, elyts))
    return el, S, b


@pytest.mark.parametrize("m", [1, 20, 64, 130])
def test_tensor_core_s_product_matches_oracle_tiny(tiny, m):
    el, S, b = tiny
    psi = _psi(m)
    ctx = make_ctx(el, s_prec="bf16x3").setup(el)
    q, qt = _update(ctx, b[:m], psi)
    _check(q, qt, _q_ref(S, el, psi, b[:m]), MIXED_TOL)


# ----------------------------------------------------------------------------- 4,320-site EDL capacitor

@pytest.fixture(scope="module")
def edl(pool):
    el, _, _ = s.workload_edl_capacitor(seed=1)
    rng = np.random.default_rng(77)
    elyts = [s.jitter(s.workload_edl_capacitor(seed=1000 + r)[1], 0.05, rng) for r in range(8)]
    _, S = oracle_S(el, pool)
    b = np.stack(pool.bvec(el, elyts))
    return el, S, elyts, b


def test_edl_capacitor_graph_step_matches_oracle(edl):
    """The benchmark's workload and launch: eight replicas per graph-captured step."""
    el, S, elyts, b = edl
    psi = _psi(8)
    q, qt = _graph_step(el, elyts, psi)
    _check(q, qt, _q_ref(S, el, psi, b), MIXED_TOL)


def test_edl_capacitor_one_replica_matches_oracle(edl):
    el, S, elyts, b = edl
    psi = _psi(1)
    for k_prec in ("f16x2", "fp32"):
        ctx = make_ctx(el, s_prec="fp32", k_prec=k_prec).setup(el)
        q, qt = _bvec_update(ctx, elyts[:1], psi)
        _check(q, qt, _q_ref(S, el, psi, b[:1]), MIXED_TOL)


# ----------------------------------------------------------------------------- tile plans of the tensor-core product

@pytest.mark.parametrize("bn,stages", [(32, 2), (32, 3), (64, 2), (64, 3), (128, 2)])
def test_every_tile_plan_matches_oracle(serving, bn, stages):
    """Every built (BN, stages) pair of the persistent tensor-core product, each with one item per CTA,
    several items per CTA and many items per CTA (both TMEM accumulators reused), against the oracle."""
    el, S, _, b = serving
    m = 37 if bn < 128 else 150          # ragged replica tiles
    bm = np.stack([b[r % len(b)] * (1.0 - 0.003 * r) for r in range(m)])
    psi = _psi(m)
    ctx = make_ctx(el, s_prec="bf16x3").setup(el)
    for splits, ctas in ((1, 152), (3, 7), (5, 2)):
        ctx.cpm_gemm_set_plan(m, bn, stages, splits, ctas)
        plan = ctx.cpm_gemm_plan(m)
        assert (plan["BN"], plan["stages"]) == (bn, stages) and plan["splits"] >= 1
        q, qt = _update(ctx, bm, psi)
        _check(q, qt, _q_ref(S, el, psi, bm), MIXED_TOL)


def test_autotuned_plan_is_timed_and_kept(serving):
    el, S, _, b = serving
    m = 64
    ctx = make_ctx(el, s_prec="bf16x3").setup(el)
    plan = ctx.cpm_gemm_plan(m)
    assert plan["candidates"] > 1 and plan["ms"] > 0
    assert ctx.cpm_gemm_plan(m) == plan            # kept per (n, m), not tuned again
    other = make_ctx(el, s_prec="bf16x3").setup(el)
    assert other.cpm_gemm_plan(m) == plan          # another context of the same n reuses it


# ----------------------------------------------------------------------------- the largest serving geometry

def test_serving_16384_sampled_rows_against_oracle():
    """16,384 sites (the largest serving geometry), where the oracle cannot form S: sampled rows of the
    oracle's A and b give the stationarity residual A q + b - v, which for the charges of Eq. (S) is the
    same constant (the neutrality multiplier) on every site (Sec. II.A).  Checked for the GPU's FP64
    path at six sampled sites of both electrodes, with the FP64 b of those sites against the oracle
    element by element; the mixed path (FP32 S stream, tensor-core reciprocal sums) against the FP64
    path for every site."""
    need_gpu()
    el, ely, psi = s.workload_serving_geometry(16384, seed=5)
    rng = np.random.default_rng(3)
    rows = np.sort(np.concatenate([rng.choice(np.where(el.group == g)[0], 3, replace=False) for g in (0, 1)]))
    A_rows = o.assemble_A(el, rows=rows)
    b_rows = o.bvec(el, ely, sites=rows)
    v = o.site_potentials(el, psi)
    ctx = make_ctx(el).setup(el)
    ctx.cpm_release_assembly()
    (q64, b64), qt64 = _bvec_update_b(ctx, [ely], psi[None])
    assert np.abs(b64[0][rows] - b_rows).max() <= 1e-10 * np.abs(b_rows).max()
    res = A_rows @ q64[0] + b_rows - v[rows]
    assert np.abs(res - res.mean()).max() <= 1e-8 * np.abs(v[rows] - b_rows).max(), res
    assert abs(qt64[0]) <= QTOT_TOL
    del ctx
    mixed = make_ctx(el, s_prec="fp32", k_prec="f16x2").setup(el)
    mixed.cpm_release_assembly()
    (qm, _), qtm = _bvec_update_b(mixed, [ely], psi[None])
    assert rel_l2(qm[0], q64[0]) <= MIXED_TOL
    assert abs(qtm[0]) <= QTOT_TOL


def _bvec_update_b(ctx, elyts, psi):
    """(q, b) and the totals of one bvec + update."""
    xyz, Q, n_e = stack_replicas(elyts)
    m = len(elyts)
    b = torch.empty((m, ctx.n), dtype=torch.float64, device="cuda")
    q = torch.empty_like(b)
    qt = torch.empty((m,), dtype=torch.float64, device="cuda")
    ctx.cpm_bvec(m, n_e, dev(xyz), dev(Q), b)
    ctx.cpm_update(m, dev(psi), b, q, qt)
    ctx.cpm_sync()
    return (q.cpu().numpy(), b.cpu().numpy()), qt.cpu().numpy()
