"""Tensor-core (tcgen05) batched update: S and b split into three bf16 terms on the 5th-gen tensor cores.

Checked against the FP64 path on the same b: q within 1e-5 relative L2 per replica, neutral to 1e-12 e.
"""
import numpy as np
import pytest

from gpu_util import dev, make_ctx, need_gpu, rel_l2, run_bvec, run_update, torch
from paper_2203_15461_gb300 import systems as s

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m", [1, 20, 64, 130])
def test_tc_update_matches_fp64_tiny(m):
    need_gpu()
    el, _, psi = s.workload_tiny_slab(seed=3)
    elyts = [s.ions_in_gap(el, 100, seed=500 + r) for r in range(m)]
    c64 = make_ctx(el).setup(el)
    ctc = make_ctx(el, s_prec="bf16x3").setup(el)
    b = run_bvec(c64, elyts)
    q64, _ = run_update(c64, psi, b)
    qtc, qt = run_update(ctc, psi, b)
    for r in range(m):
        assert rel_l2(qtc[r], q64[r]) <= 1e-5
    assert np.abs(qt).max() <= 1e-12


def test_tc_update_matches_fp64_edl():
    need_gpu()
    el, ely, psi = s.workload_edl_capacitor(seed=1)
    elyts = [s.jitter(ely, 0.05, np.random.default_rng(r)) for r in range(48)]
    c64 = make_ctx(el).setup(el)
    ctc = make_ctx(el, s_prec="bf16x3").setup(el)
    b = run_bvec(c64, elyts)
    q64, _ = run_update(c64, psi, b)
    qtc, qt = run_update(ctc, psi, b)
    errs = [rel_l2(qtc[r], q64[r]) for r in range(len(elyts))]
    assert max(errs) <= 1e-5, max(errs)
    assert np.abs(qt).max() <= 1e-12


def test_bounded_wait_reports_timeout_and_context_survives():
    """Failure detection without a fault: a wait that nothing completes runs out after 50 ms, the kernel
    records a timeout, the host reads CPM_E_TIMEOUT, and the same context then computes correctly."""
    need_gpu()
    el, ely, psi = s.workload_tiny_slab(seed=3)
    ctc = make_ctx(el, s_prec="bf16x3").setup(el)
    assert ctc.cpm_selftest_timeout(50.0) == "CPM_E_TIMEOUT"
    ctc.cpm_sync()
    c64 = make_ctx(el).setup(el)
    b = run_bvec(c64, [ely])
    q64, _ = run_update(c64, psi, b)
    qtc, _ = run_update(ctc, psi, b)
    assert rel_l2(qtc[0], q64[0]) <= 1e-5
