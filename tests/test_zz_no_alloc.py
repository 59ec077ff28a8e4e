"""cpm_bvec_noalloc: the allocation-free b entry point agrees with cpm_bvec.

Some callers cannot allocate device memory (another framework owns the memory pool,
or allocation is forbidden after start-up); they use cpm_bvec_noalloc, whose only
scratch is a fixed array built into the library.  This file is collected last so a
run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from gpu_util import dev, make_ctx, need_gpu, rel_l2, run_bvec, torch
from paper_2203_15461_gb300 import systems as s
from paper_2203_15461_gb300.cpm import CPMError, cpm_bvec_noalloc

pytestmark = pytest.mark.gpu


def test_noalloc_matches_cpm_bvec_on_two_calls_in_a_row():
    need_gpu()
    el, ely, _ = s.workload_tiny_slab(seed=5)
    ctx = make_ctx(el)
    ctx.cpm_assemble(dev(el.xyz), dev(el.eta), dev(el.group, torch.int32), el.n_groups)
    sx, se = dev(el.xyz), dev(el.eta)
    configs = [ely, s.ions_in_gap(el, 64, seed=8)]
    for e in configs:                       # two calls in a row share the fixed scratch
        ref = run_bvec(ctx, [e])[0]
        b = torch.full((el.n,), float("nan"), dtype=torch.float64, device="cuda")
        cpm_bvec_noalloc(ctx.params, sx, se, dev(e.xyz), dev(e.Q), b)
        torch.cuda.synchronize()
        assert rel_l2(b.cpu().numpy(), ref) <= 1e-11


def test_noalloc_rejects_a_grid_beyond_its_scratch():
    need_gpu()
    el, ely, _ = s.workload_tiny_slab(seed=5)
    big = make_ctx(s.Electrodes(**{**el.__dict__, "box": np.array([200.0, 200.0, 200.0])}))
    b = torch.zeros(el.n, dtype=torch.float64, device="cuda")
    with pytest.raises(CPMError, match="CPM_E_BUDGET"):
        cpm_bvec_noalloc(big.params, dev(el.xyz), dev(el.eta), dev(ely.xyz), dev(ely.Q), b)
