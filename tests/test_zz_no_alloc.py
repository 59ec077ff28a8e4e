"""cpm_bvec_noalloc: the allocation-free b entry point agrees with cpm_bvec and with the oracle.

Some callers cannot allocate device memory (another framework owns the memory pool,
or allocation is forbidden after start-up); they use cpm_bvec_noalloc, whose only
scratch is a fixed array built into the library.  The cases cover the three boundary
types (slab and wire dipole terms, tin-foil 3D) and a non-neutral electrolyte (the
background term).  This file is collected last so a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from gpu_util import dev, make_ctx, need_gpu, rel_l2, run_bvec, torch
from oracle import cpm_oracle as o
from paper_2203_15461_gb300 import systems as s
from paper_2203_15461_gb300.cpm import CPMError, cpm_bvec_noalloc

pytestmark = pytest.mark.gpu


def _case(bc):
    """Electrodes and two configurations (neutral, then non-neutral) per boundary type."""
    rng = np.random.default_rng(21)
    if bc == "slab":
        el, ely, _ = s.workload_tiny_slab(seed=5)
        return el, [ely, s.ions_in_gap(el, 64, seed=8), s.Electrolyte(xyz=ely.xyz[:37], Q=ely.Q[:37])]
    if bc == "wire":
        el = s.coaxial_tubes(2)
        x = np.column_stack([rng.uniform(35, 45, 20), rng.uniform(35, 45, 20), rng.uniform(0, el.box[2], 20)])
        return el, [s.Electrolyte(xyz=x, Q=np.tile([1.0, -1.0], 10)),
                    s.Electrolyte(xyz=x[:13], Q=np.tile([1.0, -1.0], 10)[:13])]
    n, box = 40, np.array([14.0, 15.0, 16.0])
    el = s.Electrodes(xyz=rng.uniform(0, 1, (n, 3)) * box, eta=rng.uniform(1.5, 2.0, n),
                      group=(np.arange(n) % 2).astype(np.int32), n_groups=2, box=box, boundary="3d", alpha=0.35,
                      rcut=10.0, kcut=s.kcut_from_tol(0.35, 1e-10))
    x = rng.uniform(0, 1, (30, 3)) * box
    return el, [s.Electrolyte(xyz=x, Q=np.tile([1.0, -1.0], 15)), s.Electrolyte(xyz=x[:17], Q=np.tile([1.0, -1.0], 15)[:17])]


@pytest.mark.parametrize("bc", ["slab", "wire", "3d"])
def test_noalloc_matches_cpm_bvec_on_two_calls_in_a_row(bc):
    need_gpu()
    el, configs = _case(bc)
    ctx = make_ctx(el)
    ctx.cpm_assemble(dev(el.xyz), dev(el.eta), dev(el.group, torch.int32), el.n_groups)
    sx, se = dev(el.xyz), dev(el.eta)
    for e in configs:                       # calls in a row share the fixed scratch
        ref = run_bvec(ctx, [e])[0]
        b = torch.full((el.n,), float("nan"), dtype=torch.float64, device="cuda")
        cpm_bvec_noalloc(ctx.params, sx, se, dev(e.xyz), dev(e.Q), b)
        torch.cuda.synchronize()
        got = b.cpu().numpy()
        assert rel_l2(got, ref) <= 1e-11
        assert rel_l2(got, o.bvec(el, e)) <= 1e-10


def test_noalloc_rejects_a_grid_beyond_its_scratch():
    need_gpu()
    el, ely, _ = s.workload_tiny_slab(seed=5)
    b = torch.zeros(el.n, dtype=torch.float64, device="cuda")
    for box in ([200.0, 200.0, 200.0], [1e12, 10.0, 10.0]):   # too many harmonics; an overflowing count
        big = make_ctx(s.Electrodes(**{**el.__dict__, "box": np.array(box)}))
        with pytest.raises(CPMError, match="CPM_E_BUDGET"):
            cpm_bvec_noalloc(big.params, dev(el.xyz), dev(el.eta), dev(ely.xyz), dev(ely.Q), b)
