"""Constant charge method (Sec. II.C, Eq. ewise-conq), thermo-potentiostat (Sec. II.D, Eq. deissenbeck) and
finite field (Sec. II.F, Eq. cpm-ffield) through the C ABI against the FP64 oracle, element by element.

Tolerances as for the CPM update: relative L2 error of q at most 1e-10 with FP64 S and 1e-5 with the
single-precision and tensor-core S products; electrode potentials and capacitor charges likewise.
"""
import numpy as np
import pytest

from gpu_util import dev, make_ctx, need_gpu, rel_l2, run_bvec, torch
from oracle import cpm_oracle as o
from paper_2203_15461_gb300 import systems as s

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5, "bf16x3": 1e-5}


@pytest.fixture(scope="module")
def tiny():
    need_gpu()
    el, _, _ = s.workload_tiny_slab(seed=3)
    elyts = [s.ions_in_gap(el, 100, seed=900 + r) for r in range(3)]
    elyts.append(s.Electrolyte(xyz=elyts[0].xyz[:41], Q=elyts[0].Q[:41]))      # non-neutral electrolyte
    A = o.assemble_A(el)
    S = o.capacitance_matrix(A)
    return el, elyts, A, S


def _three_electrodes(el):
    """The tiny capacitor with its top electrode split in two by x: three electrodes (Sec. II.B)."""
    g = el.group.copy()
    g[(el.group == 1) & (el.xyz[:, 0] > el.box[0] / 2)] = 2
    return s.Electrodes(**{**el.__dict__, "group": g.astype(np.int32), "n_groups": 3})


@pytest.mark.parametrize("s_prec", ["fp64", "fp32", "bf16x3"])
@pytest.mark.parametrize("three", [False, True], ids=["2el", "3el"])
def test_ccm_matches_oracle(tiny, s_prec, three):
    el, elyts, A, _ = tiny
    if three:
        el = _three_electrodes(el)
    m = len(elyts)
    rng = np.random.default_rng(8)
    qt = rng.normal(0.0, 0.8, (m, el.n_groups))
    qt[:2] -= qt[:2].mean(axis=1, keepdims=True)        # two neutral replicas, two charged ones
    ctx = make_ctx(el, s_prec=s_prec, k_prec="fp64").setup(el)
    b = run_bvec(ctx, elyts)
    q = torch.empty((m, el.n), dtype=torch.float64, device="cuda")
    qtot = torch.empty(m, dtype=torch.float64, device="cuda")
    v = torch.empty((m, el.n_groups), dtype=torch.float64, device="cuda")
    ctx.cpm_update_ccm(m, dev(qt), dev(b), q, qtot, v)
    ctx.cpm_sync()
    q, qtot, v = q.cpu().numpy(), qtot.cpu().numpy(), v.cpu().numpy()
    G = o.indicator(el)
    for r in range(m):
        q_ref, v_ref = o.ccm_charges(A, el, qt[r], o.bvec(el, elyts[r]))
        assert rel_l2(q[r], q_ref) <= TOL[s_prec], (r, rel_l2(q[r], q_ref))
        assert np.abs(G.T @ q[r] - qt[r]).max() <= (1e-11 if s_prec == "fp64" else TOL[s_prec] * np.abs(q[r]).sum())
        assert abs(qtot[r] - qt[r].sum()) <= 1e-12
        if s_prec == "fp64":
            assert np.abs(v[r] - v_ref).max() <= 1e-9 * np.abs(v_ref).max()


@pytest.mark.parametrize("s_prec", ["fp64", "fp32"])
def test_thermo_potentiostat_step_matches_oracle(tiny, s_prec):
    el, elyts, A, S = tiny
    m = 3
    rng = np.random.default_rng(12)
    qcap = np.array([0.0, 0.6, -0.3])
    X = rng.normal(size=m)
    dt, tau, T, dv0 = 1.0, 3.0, 300.0, 1.2
    ctx = make_ctx(el, s_prec=s_prec, k_prec="fp64").setup(el)
    b = run_bvec(ctx, elyts[:m])
    q = torch.empty((m, el.n), dtype=torch.float64, device="cuda")
    qn = torch.empty(m, dtype=torch.float64, device="cuda")
    dv = torch.empty(m, dtype=torch.float64, device="cuda")
    ctx.cpm_update_tp(m, dt, tau, T, dv0, dev(qcap), dev(X), dev(b), q, qn, dv)
    ctx.cpm_sync()
    q, qn, dv = q.cpu().numpy(), qn.cpu().numpy(), dv.cpu().numpy()
    for r in range(m):
        qn_ref, dv_ref, qs_ref = o.tp_step(A, S, el, qcap[r], dv0, o.bvec(el, elyts[r]), dt, tau, T, X[r])
        assert abs(qn[r] - qn_ref) <= TOL[s_prec] * max(1.0, abs(qn_ref))
        assert abs(dv[r] - dv_ref) <= TOL[s_prec] * max(1.0, abs(dv_ref))
        assert rel_l2(q[r], qs_ref) <= TOL[s_prec]
        assert abs(q[r].sum()) <= 1e-12


@pytest.mark.parametrize("s_prec", ["fp64", "fp32"])
def test_finite_field_matches_oracle(s_prec):
    """Two Au(111) sheets in a fully periodic cell (no vacuum padding) with ions between them."""
    need_gpu()
    base = s.au111_slab(seed_layers=1, gap=20.0, slab_factor=12.0)
    el = s.Electrodes(**{**base.__dict__, "box": np.array([base.box[0], base.box[1], 60.0]), "boundary": "3d"})
    rng = np.random.default_rng(3)
    ions = [s.Electrolyte(xyz=np.column_stack([rng.uniform(0, el.box[0], 30), rng.uniform(0, el.box[1], 30),
                                               rng.uniform(4.0, 17.0, 30)]), Q=np.tile([1.0, -1.0], 15))
            for _ in range(2)]
    A = o.assemble_A(el)
    S = o.capacitance_matrix(A)
    dv0 = np.array([1.0, -0.7])
    ctx = make_ctx(el, s_prec=s_prec, k_prec="fp64").setup(el)
    b = run_bvec(ctx, ions)
    q = torch.empty((2, el.n), dtype=torch.float64, device="cuda")
    qt = torch.empty(2, dtype=torch.float64, device="cuda")
    ctx.cpm_update_ffield(2, dev(dv0), dev(b), q, qt)
    ctx.cpm_sync()
    q = q.cpu().numpy()
    for r in range(2):
        ref = o.ffield_charges(S, el, dv0[r], o.bvec(el, ions[r]))
        assert rel_l2(q[r], ref) <= TOL[s_prec]
        assert abs(q[r].sum()) <= 1e-12


def test_finite_field_needs_a_periodic_cell(tiny):
    from paper_2203_15461_gb300.cpm import CPMError
    el, elyts, _, _ = tiny
    ctx = make_ctx(el).setup(el)
    b = torch.zeros((1, el.n), dtype=torch.float64, device="cuda")
    with pytest.raises(CPMError, match="CPM_E_ARG"):
        ctx.cpm_update_ffield(1, dev(np.ones(1)), b, torch.empty_like(b))
