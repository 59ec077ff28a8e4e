"""The exact 2D-periodic slab sum (EW2D, Sec. II.E) through the C ABI against the FP64 oracle.

A within 1e-12 and S within 1e-10 (relative), b within 1e-11 (FP64) and 2e-6 (single precision) for
neutral, charged and empty electrolytes, q within 1e-10 (FP64) and 1e-5 (mixed), total charge within 1e-12 e.
"""
import numpy as np
import pytest

from gpu_util import dev, make_ctx, need_gpu, rel_l2, run_bvec, run_update, torch
from oracle import cpm_oracle as o
from paper_2203_15461_gb300 import systems as s

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slab2d():
    need_gpu()
    base, ely, psi = s.workload_tiny_slab(seed=7)
    el = s.Electrodes(**{**base.__dict__, "boundary": "ew2d"})
    A = o.assemble_A(el)
    S = o.capacitance_matrix(A)
    elyts = [ely, s.ions_in_gap(el, 60, seed=70), s.Electrolyte(xyz=ely.xyz[:33], Q=ely.Q[:33])]
    return el, psi, A, S, elyts


def test_ew2d_elastance_and_capacitance(slab2d):
    el, _, A, S, _ = slab2d
    ctx = make_ctx(el).setup(el)
    Ag = ctx.cpm_get_matrix("A").cpu().numpy()
    assert np.abs(Ag - A).max() <= 1e-12 * np.abs(A).max()
    assert np.array_equal(Ag, Ag.T)
    assert rel_l2(ctx.cpm_get_matrix("S").cpu().numpy(), S) <= 1e-10


@pytest.mark.parametrize("s_prec,k_prec,btol,qtol", [("fp64", "fp64", 1e-11, 1e-10), ("fp32", "fp32", 2e-6, 1e-5)])
def test_ew2d_bvec_and_charges(slab2d, s_prec, k_prec, btol, qtol):
    el, psi, _, S, elyts = slab2d
    ctx = make_ctx(el, s_prec=s_prec, k_prec=k_prec).setup(el)
    b = run_bvec(ctx, elyts)
    q, qt = run_update(ctx, psi, b)
    for r, e in enumerate(elyts):
        b_ref = o.bvec(el, e)
        assert rel_l2(b[r], b_ref) <= btol, (r, rel_l2(b[r], b_ref))
        q_ref = o.charges(S, el, psi, b_ref)
        assert rel_l2(q[r], q_ref) <= qtol
        assert abs(qt[r]) <= 1e-12
    empty = run_bvec(ctx, [s.Electrolyte(xyz=np.zeros((0, 3)), Q=np.zeros(0))])
    assert np.abs(empty).max() == 0.0


def test_ew2d_refuses_a_short_cell_and_tensor_core_sums(slab2d):
    from paper_2203_15461_gb300.cpm import CPMError
    el, _, _, _, _ = slab2d
    with pytest.raises(CPMError, match="CPM_E_ARG"):
        make_ctx(el, k_prec="f16x2")
    short = s.Electrodes(**{**el.__dict__, "box": np.array([el.box[0], el.box[1], 35.0])})
    ctx = make_ctx(short)
    with pytest.raises(CPMError, match="CPM_E_ARG"):
        ctx.cpm_assemble(dev(short.xyz), dev(short.eta), dev(short.group, torch.int32), short.n_groups)
