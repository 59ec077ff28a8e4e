"""P3M reciprocal part of b (Introduction; SI Sec. 1.A-B; Hockney and Eastwood) through the C ABI
against the FP64 oracle's P3M, element by element, and against the Ewald sum it approximates.

Tolerances: b within 1e-12 (FP64 path) and
2e-6 (single-precision transforms) relative L2 of the oracle's P3M b; q within 1e-10 (FP64) and 1e-5
(mixed) of the oracle's q for that b; total charge within 1e-12 e.  The mesh solution itself is
deterministic: the same inputs give the same bits, eagerly and in a captured step.
"""
import numpy as np
import pytest

from gpu_util import dev, make_ctx, need_gpu, rel_l2, run_bvec, run_update, stack_replicas, torch
from oracle import cpm_oracle as o
from paper_2203_15461_gb300 import systems as s

pytestmark = pytest.mark.gpu


def with_p3m(el, mesh, order):
    return s.Electrodes(**{**el.__dict__, "p3m_mesh": tuple(mesh), "p3m_order": int(order)})


@pytest.fixture(scope="module")
def tiny():
    need_gpu()
    el, ely, psi = s.workload_tiny_slab(seed=5)
    S = o.capacitance_matrix(o.assemble_A(el))
    elyts = [ely, s.ions_in_gap(el, 80, seed=51), s.Electrolyte(xyz=ely.xyz[:37], Q=ely.Q[:37])]   # ragged, charged
    return el, psi, S, elyts


@pytest.mark.parametrize("mesh,order", [((16, 16, 64), 5), ((32, 32, 128), 7), ((8, 16, 32), 2), ((16, 8, 64), 3),
                                        ((16, 16, 32), 4), ((32, 16, 64), 6)])
def test_p3m_b_and_q_match_oracle_fp64(tiny, mesh, order):
    el0, psi, S, elyts = tiny
    el = with_p3m(el0, mesh, order)
    ctx = make_ctx(el).setup(el)
    b = run_bvec(ctx, elyts)
    q, qt = run_update(ctx, psi, b)
    for r, e in enumerate(elyts):
        b_ref = o.bvec(el, e)
        assert rel_l2(b[r], b_ref) <= 1e-12, (r, rel_l2(b[r], b_ref))
        assert rel_l2(q[r], o.charges(S, el, psi, b_ref)) <= 1e-10
        assert abs(qt[r]) <= 1e-12


@pytest.mark.parametrize("k_prec", ["fp32", "f16x2"])
def test_p3m_mixed_matches_oracle(tiny, k_prec):
    el0, psi, S, elyts = tiny
    el = with_p3m(el0, (32, 32, 128), 7)
    ctx = make_ctx(el, s_prec="fp32", k_prec=k_prec).setup(el)
    b = run_bvec(ctx, elyts)
    q, qt = run_update(ctx, psi, b)
    for r, e in enumerate(elyts):
        b_ref = o.bvec(el, e)
        assert rel_l2(b[r], b_ref) <= 2e-6, (r, rel_l2(b[r], b_ref))
        assert rel_l2(q[r], o.charges(S, el, psi, b_ref)) <= 1e-5
        assert abs(qt[r]) <= 1e-12


def test_p3m_other_boundaries_match_oracle():
    """3D periodic (the slab cell without vacuum) and 1D periodic (co-axial tubes, wire correction)."""
    need_gpu()
    base, ely, _ = s.workload_tiny_slab(seed=9)
    el3 = s.Electrodes(**{**base.__dict__, "box": np.array([base.box[0], base.box[1], 40.0]), "boundary": "3d"})
    tube = s.coaxial_tubes(4)
    rng = np.random.default_rng(4)
    R = np.sqrt(rng.uniform(8.0 ** 2, 12.0 ** 2, 40))
    th = rng.uniform(0, 2 * np.pi, 40)
    wire_ions = s.Electrolyte(xyz=np.column_stack([tube.box[0] / 2 + R * np.cos(th), tube.box[1] / 2 + R * np.sin(th),
                                                   rng.uniform(0, tube.box[2], 40)]), Q=np.tile([1.0, -1.0], 20))
    for el, e, mesh in ((el3, ely, (16, 16, 32)), (tube, wire_ions, (32, 32, 16))):
        elp = with_p3m(el, mesh, 5)
        for k_prec, tol in (("fp64", 1e-12), ("fp32", 2e-6)):
            ctx = make_ctx(elp, k_prec=k_prec).setup(elp)
            b = run_bvec(ctx, [e])
            assert rel_l2(b[0], o.bvec(elp, e)) <= tol, (el.boundary, k_prec)


def test_p3m_approaches_ewald(tiny):
    """The GPU mesh solution is as close to the Ewald b as the oracle's own P3M (convergence pinned there)."""
    el0, _, _, elyts = tiny
    ew = [o.bvec(el0, e) for e in elyts]
    for mesh, order, bound in (((16, 16, 64), 5, 1e-4), ((32, 32, 128), 7, 1e-8)):
        el = with_p3m(el0, mesh, order)
        b = run_bvec(make_ctx(el).setup(el), elyts)
        for r in range(len(elyts)):
            err, err_oracle = rel_l2(b[r], ew[r]), rel_l2(o.bvec(el, elyts[r]), ew[r])
            assert err <= bound and abs(err - err_oracle) <= 1e-3 * err_oracle, (mesh, order, err, err_oracle)


def test_p3m_is_deterministic_and_graph_equals_eager(tiny):
    el0, psi, _, elyts = tiny
    el = with_p3m(el0, (32, 32, 128), 7)
    ctx = make_ctx(el, s_prec="fp32", k_prec="fp32", stream=torch.cuda.Stream()).setup(el)
    xyz, Q, ne = stack_replicas(elyts)
    m = len(elyts)
    xyz_d, Q_d = dev(xyz), dev(Q)
    torch.cuda.synchronize()   # the inputs were written on the default stream
    outs = []
    for _ in range(2):
        b = torch.empty((m, ctx.n), dtype=torch.float64, device="cuda")
        ctx.cpm_bvec(m, ne, xyz_d, Q_d, b)
        ctx.cpm_sync()
        outs.append(b.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    psi_d = dev(np.tile(psi, (m, 1)))
    torch.cuda.synchronize()
    for _ in range(2):
        b = torch.empty((m, ctx.n), dtype=torch.float64, device="cuda")
        q = torch.empty((m, ctx.n), dtype=torch.float64, device="cuda")
        ctx.cpm_step_graph(m, ne, xyz_d, Q_d, psi_d, b, q)
        ctx.cpm_sync()
        assert np.array_equal(b.cpu().numpy(), outs[0])


def test_p3m_edge_cases(tiny):
    """No charges, replicas of zero charges, an odd replica count (the last mesh pair half empty)."""
    el0, _, _, elyts = tiny
    el = with_p3m(el0, (16, 16, 64), 5)
    ctx = make_ctx(el).setup(el)
    empty = run_bvec(ctx, [s.Electrolyte(xyz=np.zeros((0, 3)), Q=np.zeros(0))] * 3)
    assert np.abs(empty).max() == 0.0
    zero = s.Electrolyte(xyz=elyts[0].xyz, Q=np.zeros(elyts[0].n))
    b = run_bvec(ctx, [zero, elyts[1], zero, elyts[0], elyts[2]])
    # a replica shares its complex mesh with its neighbour: the transforms leave rounding of the
    # partner's potential in it, nothing more
    for r in (0, 2):
        assert np.abs(b[r]).max() <= 1e-13 * np.abs(b[r + 1]).max(), r
    for r, e in ((1, elyts[1]), (3, elyts[0]), (4, elyts[2])):
        assert rel_l2(b[r], o.bvec(el, e)) <= 1e-12


def test_p3m_full_edl_capacitor_matches_oracle():
    """The 4,320-site EDL capacitor, 5,700 charges per replica, mesh 32 x 32 x 128, order 7, three replicas in
    one launch on the mixed path: b against the oracle's P3M and against the Ewald sum."""
    need_gpu()
    el0, ely, psi = s.workload_edl_capacitor(seed=1)
    el = with_p3m(el0, (32, 32, 128), 7)
    rng = np.random.default_rng(2)
    elyts = [ely] + [s.jitter(ely, 0.05, rng) for _ in range(2)]
    ctx = make_ctx(el, s_prec="fp32", k_prec="f16x2").setup(el)
    b = run_bvec(ctx, elyts)
    for r in (0, 2):
        b_ref = o.bvec(el, elyts[r])
        assert rel_l2(b[r], b_ref) <= 2e-6, (r, rel_l2(b[r], b_ref))
    assert rel_l2(b[0], o.bvec(el0, ely)) <= 3e-6


def test_p3m_refuses_bad_parameters(tiny):
    from paper_2203_15461_gb300.cpm import CPMError
    el0, _, _, _ = tiny
    for mesh, order in (((16, 16, 64), 8), ((16, 16, 64), 1), ((12, 16, 64), 5), ((16, 16, 1024), 5),
                        ((256, 128, 64), 5)):
        with pytest.raises(CPMError, match="cpm_create"):
            make_ctx(with_p3m(el0, mesh, order), k_prec="fp32")
    with pytest.raises(CPMError, match="cpm_create"):
        make_ctx(with_p3m(s.Electrodes(**{**el0.__dict__, "boundary": "ew2d"}), (16, 16, 64), 5))


@pytest.mark.parametrize("m", [1, 20])
def test_p3m_replica_counts(tiny, m):
    """One replica (a half-empty mesh pair) and twenty (ten pairs, charge splits over many bricks)."""
    el0, _, _, _ = tiny
    el = with_p3m(el0, (16, 16, 64), 6)
    elyts = [s.ions_in_gap(el0, 40 + 3 * r, seed=700 + r) for r in range(m)]
    b = run_bvec(make_ctx(el, k_prec="fp32").setup(el), elyts)
    for r in sorted({0, m // 2, m - 1}):
        assert rel_l2(b[r], o.bvec(el, elyts[r])) <= 2e-6, r


def test_p3m_fp64_largest_plane_and_host_step(tiny):
    """FP64 with a 64 x 64 xy plane (64 KiB of complex doubles in shared memory), through the host-buffer
    step (cpm_step_host: copies, captured step, q back)."""
    el0, psi, S, elyts = tiny
    el = with_p3m(el0, (64, 64, 32), 4)
    ctx = make_ctx(el, stream=torch.cuda.Stream()).setup(el)
    xyz, Q, ne = stack_replicas(elyts)
    m = len(elyts)
    q = np.zeros((m, el.n))
    qt = np.zeros(m)
    ctx.cpm_step_host(m, ne, xyz, Q, np.tile(psi, (m, 1)), q, qt)
    for r, e in enumerate(elyts):
        assert rel_l2(q[r], o.charges(S, el, psi, o.bvec(el, e))) <= 1e-10
        assert abs(qt[r]) <= 1e-12


def test_p3m_with_constant_charge(tiny):
    """The constant charge method (Sec. II.C) on a P3M b."""
    el0, _, _, elyts = tiny
    el = with_p3m(el0, (32, 32, 128), 7)
    A = o.assemble_A(el0)
    ctx = make_ctx(el).setup(el)
    b = run_bvec(ctx, elyts[:2])
    qt = np.array([[0.3, -0.3], [0.0, 0.5]])
    q = torch.empty((2, el.n), dtype=torch.float64, device="cuda")
    ctx.cpm_update_ccm(2, dev(qt), dev(b), q, None, None)
    ctx.cpm_sync()
    q = q.cpu().numpy()
    for r in range(2):
        q_ref, _ = o.ccm_charges(A, el, qt[r], o.bvec(el, elyts[r]))
        assert rel_l2(q[r], q_ref) <= 1e-10


# ----------------------------------------------------------------------------- the P3M elastance

def with_p3m_matrix(el, mesh, order):
    return s.Electrodes(**{**el.__dict__, "p3m_mesh": tuple(mesh), "p3m_order": int(order), "p3m_matrix": True})


@pytest.mark.parametrize("mesh,order", [((16, 16, 64), 5), ((32, 32, 128), 7)])
def test_p3m_elastance_matches_oracle(tiny, mesh, order):
    """A with the P3M reciprocal part (FP64 mesh arithmetic) within 1e-12 of the oracle's, S within 1e-10, the
    charges of the FP64 path within 1e-10 and of the mixed path within 1e-5 of the oracle's (P3M A and b)."""
    el0, psi, _, elyts = tiny
    el = with_p3m_matrix(el0, mesh, order)
    A = o.assemble_A(el)
    S = o.capacitance_matrix(A)
    ctx = make_ctx(el).setup(el)
    Ag = ctx.cpm_get_matrix("A").cpu().numpy()
    assert np.abs(Ag - A).max() <= 1e-12 * np.abs(A).max()
    assert np.array_equal(Ag, Ag.T)
    assert rel_l2(ctx.cpm_get_matrix("S").cpu().numpy(), S) <= 1e-10
    for s_prec, k_prec, tol in (("fp64", "fp64", 1e-10), ("fp32", "fp32", 1e-5), ("fp32", "f16x2", 1e-5)):
        c = ctx if s_prec == "fp64" else make_ctx(el, s_prec=s_prec, k_prec=k_prec).setup(el)
        b = run_bvec(c, elyts)
        q, qt = run_update(c, psi, b)
        for r, e in enumerate(elyts):
            assert rel_l2(q[r], o.charges(S, el, psi, o.bvec(el, e))) <= tol, (s_prec, k_prec, r)
            assert abs(qt[r]) <= 1e-12


def test_p3m_elastance_other_boundaries():
    """3D periodic and the wire correction (co-axial tubes): A against the oracle."""
    need_gpu()
    base, _, _ = s.workload_tiny_slab(seed=9)
    el3 = s.Electrodes(**{**base.__dict__, "box": np.array([base.box[0], base.box[1], 40.0]), "boundary": "3d"})
    for el, mesh in ((el3, (16, 16, 32)), (s.coaxial_tubes(4), (32, 32, 16))):
        elp = with_p3m_matrix(el, mesh, 5)
        A = o.assemble_A(elp)
        Ag = make_ctx(elp, k_prec="fp32").setup(elp).cpm_get_matrix("A").cpu().numpy()
        assert np.abs(Ag - A).max() <= 1e-12 * np.abs(A).max(), el.boundary


def test_p3m_elastance_edl_capacitor_sampled_rows():
    """The 4,320-site EDL capacitor: sampled rows of the P3M elastance against the oracle's rows."""
    need_gpu()
    el0, _, _ = s.workload_edl_capacitor(seed=1)
    el = with_p3m_matrix(el0, (32, 32, 128), 7)
    rows = np.array([0, 777, 2159, 2160, 3001, 4319])
    A_ref = o.assemble_A(el, rows=rows)
    Ag = make_ctx(el, s_prec="fp32", k_prec="f16x2").setup(el).cpm_get_matrix("A").cpu().numpy()
    assert np.abs(Ag[rows] - A_ref).max() <= 1e-12 * np.abs(A_ref).max()
