"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs.

Tolerances: FP64 path q within 1e-10 relative L2 of the oracle, mixed path within
1e-5, total electrode charge within 1e-12 e for both; A within 1e-12 and S within
1e-10 (relative, FP64); the k-vector set bit-exact.
"""
import numpy as np
import pytest

from gpu_util import dev, make_ctx, need_gpu, rel_l2, run_bvec, run_update, torch
from oracle import cpm_oracle as o
from paper_2203_15461_gb300 import systems as s

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    need_gpu()
    el, ely, psi = s.workload_tiny_slab(seed=3)
    A = o.assemble_A(el)
    S = o.capacitance_matrix(A)
    return el, ely, psi, A, S


def _kset(nidx):
    return set(map(tuple, np.asarray(nidx, dtype=np.int64).tolist()))


@pytest.mark.parametrize("which", ["tiny", "edl", "coax"])
def test_kvector_set_bit_exact(which):
    need_gpu()
    el = {"tiny": lambda: s.au111_slab(), "edl": lambda: s.graphene_plates(18, 10, 3, 60.0),
          "coax": lambda: s.coaxial_tubes(2)}[which]()
    ctx = make_ctx(el)
    xyz = dev(el.xyz)
    ctx.cpm_assemble(xyz, dev(el.eta), dev(el.group, torch.int32), el.n_groups)
    got = ctx.cpm_kvectors()
    nidx, _, _ = o.kvectors(el.box, el.kcut)
    assert len(got) == len(nidx)
    assert _kset(got) == _kset(nidx)
    if which == "tiny":
        assert len(got) == 3293


def test_elastance_and_capacitance_parity(tiny):
    el, _, _, A, S = tiny
    ctx = make_ctx(el).setup(el)
    Ag = ctx.cpm_get_matrix("A").cpu().numpy()
    assert np.abs(Ag - A).max() <= 1e-12 * np.abs(A).max()
    assert np.array_equal(Ag, Ag.T)
    Sg = ctx.cpm_get_matrix("S").cpu().numpy()
    assert rel_l2(Sg, S) <= 1e-10
    C = ctx.cpm_capacitance()
    assert np.abs(C - o.electrode_capacitance(S, el)).max() <= 1e-10 * abs(C[0, 0])


@pytest.mark.parametrize("k_prec,tol", [("fp64", 1e-11), ("fp32", 2e-6)])
def test_bvec_parity_replicas_ragged(tiny, k_prec, tol):
    """Three replicas of different sizes (zero-charge padding) and one empty electrolyte."""
    el, ely, _, _, _ = tiny
    e2 = s.ions_in_gap(el, 60, seed=11)
    e3 = s.Electrolyte(xyz=ely.xyz[:37], Q=ely.Q[:37])      # non-neutral: background term
    ctx = make_ctx(el, k_prec=k_prec)
    ctx.cpm_assemble(dev(el.xyz), dev(el.eta), dev(el.group, torch.int32), el.n_groups)
    b = run_bvec(ctx, [ely, e2, e3])
    for r, e in enumerate([ely, e2, e3]):
        ref = o.bvec(el, e)
        assert rel_l2(b[r], ref) <= tol
    empty = run_bvec(ctx, [s.Electrolyte(xyz=np.zeros((0, 3)), Q=np.zeros(0))])
    assert np.abs(empty).max() == 0.0


@pytest.mark.parametrize("s_prec,k_prec,tol", [("fp64", "fp64", 1e-10), ("fp32", "fp32", 1e-5)])
def test_charge_update_parity(tiny, s_prec, k_prec, tol):
    el, ely, psi, A, S = tiny
    ctx = make_ctx(el, s_prec=s_prec, k_prec=k_prec).setup(el)
    elyts = [s.jitter(ely, 0.05, np.random.default_rng(k)) for k in range(4)]
    b = run_bvec(ctx, elyts)
    q, qt = run_update(ctx, psi, b)
    for r, e in enumerate(elyts):
        q_ref = o.charges(S, el, psi, o.bvec(el, e))
        assert rel_l2(q[r], q_ref) <= tol
        assert abs(q[r].sum()) <= 1e-12
        assert abs(qt[r]) <= 1e-12


def test_vacuum_capacitor_charges_match_SG(tiny):
    """No electrolyte: b = 0 and q = S G psi exactly as the oracle."""
    el, _, psi, _, S = tiny
    ctx = make_ctx(el).setup(el)
    b = run_bvec(ctx, [s.Electrolyte(xyz=np.zeros((0, 3)), Q=np.zeros(0))])
    q, _ = run_update(ctx, psi, b)
    assert rel_l2(q[0], S @ o.site_potentials(el, psi)) <= 1e-12


def test_symm_off_gives_inverse(tiny):
    el, ely, psi, A, _ = tiny
    ctx = make_ctx(el, symm=False).setup(el)
    Ainv = o.capacitance_matrix(A, symm=False)
    assert rel_l2(ctx.cpm_get_matrix("S").cpu().numpy(), Ainv) <= 1e-10
    b = run_bvec(ctx, [ely])
    q, qt = run_update(ctx, psi, b)
    ref = Ainv @ (o.site_potentials(el, psi) - o.bvec(el, ely))
    assert rel_l2(q[0], ref) <= 1e-10
    assert abs(qt[0] - ref.sum()) <= 1e-10


@pytest.mark.parametrize("s_prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("big", [False, True], ids=["216", "512"])
def test_symm_off_single_precision_products(tiny, s_prec, big):
    """S = A^-1 (no projection) with the single-precision and tensor-core products: the rows of A^-1 do
    not sum to zero, so the centred products must add b_i sum_j S_ij back (216 sites: the two-column
    kernel; 512 sites: the TMA stream)."""
    if big:
        el, ely = s.workload_serving_geometry(512, seed=4)[:2]
        A = o.assemble_A(el)
    else:
        el, ely, _, A, _ = tiny
    psi = np.array([0.0, 1.0])
    Ainv = o.capacitance_matrix(A, symm=False)
    ctx = make_ctx(el, symm=False, s_prec=s_prec, k_prec="fp64").setup(el)
    b = run_bvec(ctx, [ely, ely])
    q, qt = run_update(ctx, psi, b)
    ref = Ainv @ (o.site_potentials(el, psi) - o.bvec(el, ely))
    for r in range(2):
        assert rel_l2(q[r], ref) <= 1e-5, (r, rel_l2(q[r], ref))
        assert abs(qt[r] - q[r].sum()) <= 1e-10 * np.abs(q[r]).sum()


def test_step_host_equals_device_path(tiny):
    el, ely, psi, _, _ = tiny
    ctx = make_ctx(el).setup(el)
    b = run_bvec(ctx, [ely])
    q_dev, qt_dev = run_update(ctx, psi, b)
    q = np.zeros((1, el.n))
    qt = np.zeros(1)
    ctx.cpm_step_host(1, ely.n, np.ascontiguousarray(ely.xyz), np.ascontiguousarray(ely.Q), psi.copy(), q, qt)
    assert np.array_equal(q, q_dev) and np.array_equal(qt, qt_dev)


@pytest.mark.parametrize("s_prec,k_prec", [("fp64", "fp64"), ("fp32", "f16x2")])
def test_step_host_pinned_buffers(tiny, s_prec, k_prec):
    """Page-locked host buffers on a context with its own stream: the copies become nodes of the captured
    step.  Each call must read the caller's current positions and write fresh charges, equal to the
    device path's; pageable buffers (the other path) give the same bits."""
    el, ely, psi, _, _ = tiny
    ctx = make_ctx(el, s_prec=s_prec, k_prec=k_prec, stream=torch.cuda.Stream()).setup(el)
    m, ne = 2, ely.n
    rng = np.random.default_rng(17)
    hx = torch.empty((m * ne, 3), dtype=torch.float64).pin_memory()
    hQ = torch.as_tensor(np.tile(ely.Q, m)).pin_memory()
    hpsi = torch.as_tensor(np.tile(psi, (m, 1))).pin_memory()
    hq = torch.empty((m, el.n), dtype=torch.float64).pin_memory()
    hqt = torch.empty((m,), dtype=torch.float64).pin_memory()
    for step in range(3):
        x = np.concatenate([ely.xyz + rng.normal(0, 0.05, ely.xyz.shape) for _ in range(m)])
        hx.copy_(torch.as_tensor(x))
        ctx.cpm_step_host(m, ne, hx, hQ, hpsi, hq, hqt)
        q_ref = np.zeros((m, el.n))
        qt_ref = np.zeros(m)
        ctx.cpm_step_host(m, ne, np.ascontiguousarray(x), np.tile(ely.Q, m), np.tile(psi, (m, 1)), q_ref, qt_ref)
        assert np.array_equal(hq.numpy(), q_ref) and np.array_equal(hqt.numpy(), qt_ref), step


def test_save_load_roundtrip(tiny, tmp_path):
    el, ely, psi, _, _ = tiny
    a = make_ctx(el).setup(el)
    path = str(tmp_path / "S.bin")
    a.cpm_save(path)
    b = make_ctx(el)
    b.cpm_assemble(dev(el.xyz), dev(el.eta), dev(el.group, torch.int32), el.n_groups)
    b.cpm_load(path)
    assert torch.equal(a.cpm_get_matrix("S"), b.cpm_get_matrix("S"))
    other = s.au111_slab(gap=22.0)
    c = make_ctx(other)
    c.cpm_assemble(dev(other.xyz), dev(other.eta), dev(other.group, torch.int32), other.n_groups)
    with pytest.raises(Exception, match="CPM_E_ARG"):
        c.cpm_load(path)


def test_errors_are_status_codes(tiny):
    from paper_2203_15461_gb300.cpm import CPMError
    el, ely, psi, _, _ = tiny
    ctx = make_ctx(el)
    b = torch.zeros((1, el.n), dtype=torch.float64, device="cuda")
    with pytest.raises(CPMError, match="CPM_E_STATE"):
        ctx.cpm_update(1, dev(psi[None]), b, torch.empty_like(b))
    bad = el.eta.copy()
    bad[5] = -1.0
    with pytest.raises(CPMError, match="CPM_E_NONFINITE"):
        ctx.cpm_assemble(dev(el.xyz), dev(bad), dev(el.group, torch.int32), el.n_groups)
    g = el.group.copy()
    g[0] = 7
    with pytest.raises(CPMError, match="CPM_E_NONFINITE"):
        ctx.cpm_assemble(dev(el.xyz), dev(el.eta), dev(g, torch.int32), el.n_groups)
    small = make_ctx(el, hbm_budget=1 << 20)
    with pytest.raises(CPMError, match="CPM_E_BUDGET"):
        small.cpm_assemble(dev(el.xyz), dev(el.eta), dev(el.group, torch.int32), el.n_groups)


def test_wire_coaxial_parity():
    need_gpu()
    el = s.coaxial_tubes(2)
    A = o.assemble_A(el)
    S = o.capacitance_matrix(A)
    ctx = make_ctx(el).setup(el)
    assert np.abs(ctx.cpm_get_matrix("A").cpu().numpy() - A).max() <= 1e-12 * np.abs(A).max()
    C = ctx.cpm_capacitance()
    assert abs(C[1, 1] / o.electrode_capacitance(S, el)[1, 1] - 1) <= 1e-10
    rng = np.random.default_rng(2)
    ely = s.Electrolyte(xyz=np.column_stack([rng.uniform(35, 45, 20), rng.uniform(35, 45, 20),
                                             rng.uniform(0, el.box[2], 20)]), Q=np.tile([1.0, -1.0], 10))
    b = run_bvec(ctx, [ely])
    assert rel_l2(b[0], o.bvec(el, ely)) <= 1e-11


def test_tinfoil_3d_parity():
    need_gpu()
    rng = np.random.default_rng(9)
    n = 40
    box = np.array([14.0, 15.0, 16.0])
    el = s.Electrodes(xyz=rng.uniform(0, 1, (n, 3)) * box, eta=rng.uniform(1.5, 2.0, n),
                      group=(np.arange(n) % 2).astype(np.int32), n_groups=2, box=box, boundary="3d", alpha=0.35,
                      rcut=10.0, kcut=s.kcut_from_tol(0.35, 1e-10))
    A = o.assemble_A(el)
    ctx = make_ctx(el).setup(el)
    assert np.abs(ctx.cpm_get_matrix("A").cpu().numpy() - A).max() <= 1e-12 * np.abs(A).max()
    ely = s.Electrolyte(xyz=rng.uniform(0, 1, (30, 3)) * box, Q=np.tile([1.0, -1.0], 15))
    b = run_bvec(ctx, [ely])
    assert rel_l2(b[0], o.bvec(el, ely)) <= 1e-11


# ----------------------------------------------------------------------------- full-size workloads

@pytest.fixture(scope="module")
def edl():
    """4,320-site EDL capacitor (1,800 waters + 300 ions): GPU FP64 and mixed contexts."""
    need_gpu()
    el, ely, psi = s.workload_edl_capacitor(seed=1)
    c64 = make_ctx(el).setup(el)
    c32 = make_ctx(el, s_prec="fp32", k_prec="fp32").setup(el)
    return el, ely, psi, c64, c32


def test_edl_capacitor_sampled_elastance_rows(edl):
    el, _, _, c64, _ = edl
    rows = np.random.default_rng(0).choice(el.n, 12, replace=False)
    A_rows = o.assemble_A(el, rows=rows)
    Ag = c64.cpm_get_matrix("A").cpu().numpy()[rows]
    assert np.abs(Ag - A_rows).max() <= 1e-12 * np.abs(A_rows).max()


def test_edl_capacitor_b_sampled_and_q_optimal(edl):
    """b at sampled sites against the oracle; q satisfies the stationarity condition A q + b - v = lambda e
    on sampled rows of the oracle's A; the mixed path agrees with FP64 within 1e-5 and both are neutral."""
    el, ely, psi, c64, c32 = edl
    sites = np.random.default_rng(1).choice(el.n, 12, replace=False)
    b64 = run_bvec(c64, [ely])
    assert rel_l2(b64[0][sites], o.bvec(el, ely, sites=sites)) <= 1e-11
    q64, qt64 = run_update(c64, psi, b64)
    A_rows = o.assemble_A(el, rows=sites)
    v = o.site_potentials(el, psi)
    r = A_rows @ q64[0] + b64[0][sites] - v[sites]
    assert np.abs(r - r.mean()).max() <= 1e-9 * np.abs(v - b64[0]).max()
    b32 = run_bvec(c32, [ely])
    q32, qt32 = run_update(c32, psi, b32)
    assert rel_l2(q32[0], q64[0]) <= 1e-5
    assert abs(qt64[0]) <= 1e-12 and abs(qt32[0]) <= 1e-12
    assert abs(q64[0].sum()) <= 1e-12 and abs(q32[0].sum()) <= 1e-12


def test_batched_replicas_of_the_tiny_capacitor(tiny):
    """256 replicas sharing one S (each its own seeded electrolyte) in one launch sequence; replicas checked
    against the oracle one by one."""
    el, _, psi, _, S = tiny
    elyts = [s.ions_in_gap(el, 100, seed=1000 + r) for r in range(256)]
    for s_prec, k_prec, tol in (("fp64", "fp64", 1e-10), ("fp32", "fp32", 1e-5)):
        ctx = make_ctx(el, s_prec=s_prec, k_prec=k_prec).setup(el)
        b = run_bvec(ctx, elyts)
        q, qt = run_update(ctx, psi, b)
        for r in (0, 77, 255):
            q_ref = o.charges(S, el, psi, o.bvec(el, elyts[r]))
            assert rel_l2(q[r], q_ref) <= tol
        assert np.abs(qt).max() <= 1e-12


def test_step_graph_replays_the_same_launches(tiny):
    """cpm_step_graph: one captured bvec + update graph, replayed for new inputs in the same buffers."""
    el, ely, psi, _, S = tiny
    st = torch.cuda.Stream()
    ctx = make_ctx(el, s_prec="fp32", k_prec="fp32", stream=st).setup(el)
    m = 4
    elyts = [s.ions_in_gap(el, 100, seed=700 + r) for r in range(2 * m)]
    from gpu_util import stack_replicas
    x1, Q1, ne = stack_replicas(elyts[:m])
    x2, Q2, _ = stack_replicas(elyts[m:], n_e=ne)
    dx, dQ = dev(x1), dev(Q1)
    dpsi = dev(np.tile(psi, (m, 1)))
    b = torch.empty((m, el.n), dtype=torch.float64, device="cuda")
    q = torch.empty_like(b)
    qt = torch.empty(m, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(st):
        ctx.cpm_step_graph(m, ne, dx, dQ, dpsi, b, q, qt)
    st.synchronize()
    first = q.cpu().numpy().copy()
    with torch.cuda.stream(st):
        dx.copy_(dev(x2)); dQ.copy_(dev(Q2))
        ctx.cpm_step_graph(m, ne, dx, dQ, dpsi, b, q, qt)
    st.synchronize()
    second = q.cpu().numpy().copy()
    ref = make_ctx(el, s_prec="fp32", k_prec="fp32").setup(el)
    for got, batch in ((first, elyts[:m]), (second, elyts[m:])):
        qr, _ = run_update(ref, psi, run_bvec(ref, batch))
        assert np.array_equal(got, qr)


@pytest.mark.parametrize("which", ["tiny", "coax"])
def test_capacitance_by_fp32_factor_and_fp64_refinement(which):
    """C~ from the FP32 Cholesky factor with FP64 iterative refinement equals C~ from the FP64 inverse."""
    need_gpu()
    el = s.au111_slab() if which == "tiny" else s.coaxial_tubes(2)
    ctx = make_ctx(el).setup(el)
    C64 = ctx.cpm_capacitance()
    C, it, res = ctx.cpm_capacitance_ir()
    assert it >= 1 and res < 1e-12
    assert np.abs(C - C64).max() <= 1e-10 * np.abs(C64).max()


def test_step_host_on_a_stream_replays_the_graph(tiny):
    """cpm_step_host on a context with its own stream runs the captured step: the same q as
    cpm_step_graph on device buffers, bit for bit, and the same on a second call with new inputs."""
    el, _, psi, _, _ = tiny
    st = torch.cuda.Stream()
    ctx = make_ctx(el, s_prec="fp32", k_prec="f16x2", stream=st).setup(el)
    ref = make_ctx(el, s_prec="fp32", k_prec="f16x2", stream=torch.cuda.Stream()).setup(el)
    from gpu_util import stack_replicas
    m = 3
    for seed in (40, 41):
        elyts = [s.ions_in_gap(el, 100, seed=10 * seed + r) for r in range(m)]
        xyz, Q, ne = stack_replicas(elyts)
        psis = np.tile(psi, (m, 1))
        q = np.zeros((m, el.n))
        qt = np.zeros(m)
        ctx.cpm_step_host(m, ne, np.ascontiguousarray(xyz), np.ascontiguousarray(Q), psis.copy(), q, qt)
        with torch.cuda.stream(ref.stream):
            b = torch.empty((m, el.n), dtype=torch.float64, device="cuda")
            qd = torch.empty_like(b)
            qtd = torch.empty(m, dtype=torch.float64, device="cuda")
            ref.cpm_step_graph(m, ne, dev(xyz), dev(Q), dev(psis), b, qd, qtd)
        ref.stream.synchronize()
        assert np.array_equal(q, qd.cpu().numpy()) and np.array_equal(qt, qtd.cpu().numpy())


def test_checkpoint_in_host_memory_restores_without_assembly(tiny):
    """cpm_export / cpm_import through host memory, into a context prepared without A (cpm_prepare):
    the same S and the same charges as the assembled, inverted context; cpm_release_assembly frees A
    and W and the context still updates."""
    from paper_2203_15461_gb300.cpm import CPMError
    el, ely, psi, _, _ = tiny
    a = make_ctx(el).setup(el)
    buf = a.cpm_export()
    b = make_ctx(el)
    b.cpm_prepare(dev(el.xyz), dev(el.eta), dev(el.group, torch.int32), el.n_groups)
    with pytest.raises(CPMError, match="CPM_E_STATE"):
        b.cpm_invert()
    b.cpm_import(buf)
    assert torch.equal(a.cpm_get_matrix("S"), b.cpm_get_matrix("S"))
    q_a, _ = run_update(a, psi, run_bvec(a, [ely]))
    q_b, _ = run_update(b, psi, run_bvec(b, [ely]))
    assert np.array_equal(q_a, q_b)
    held = a.cpm_device_bytes()
    a.cpm_release_assembly()
    assert held - a.cpm_device_bytes() >= 2 * 8 * el.n * el.n
    with pytest.raises(CPMError, match="CPM_E_STATE"):
        a.cpm_get_matrix("A")
    q_c, _ = run_update(a, psi, run_bvec(a, [ely]))
    assert np.array_equal(q_a, q_c)
    other = s.au111_slab(gap=22.0)
    c = make_ctx(other)
    c.cpm_prepare(dev(other.xyz), dev(other.eta), dev(other.group, torch.int32), other.n_groups)
    with pytest.raises(CPMError, match="CPM_E_ARG"):
        c.cpm_import(buf)


def test_several_captured_graphs_are_kept(tiny):
    """Graphs for different batch sizes are kept side by side and replay the same charges as the
    separate calls."""
    el, _, psi, _, _ = tiny
    st = torch.cuda.Stream()
    ctx = make_ctx(el, s_prec="fp32", k_prec="fp32", stream=st).setup(el)
    from gpu_util import stack_replicas
    bufs = {}
    for m in (1, 2, 4, 1, 4, 2):
        elyts = [s.ions_in_gap(el, 100, seed=60 * m + r) for r in range(m)]
        xyz, Q, ne = stack_replicas(elyts, n_e=100)
        if m not in bufs:
            with torch.cuda.stream(st):
                bufs[m] = [torch.empty((m * ne, 3), dtype=torch.float64, device="cuda"),
                           torch.empty(m * ne, dtype=torch.float64, device="cuda"),
                           dev(np.tile(psi, (m, 1))), torch.empty((m, el.n), dtype=torch.float64, device="cuda"),
                           torch.empty((m, el.n), dtype=torch.float64, device="cuda"),
                           torch.empty(m, dtype=torch.float64, device="cuda")]
        dx, dQ, dp, b, q, qt = bufs[m]
        with torch.cuda.stream(st):
            dx.copy_(dev(xyz)); dQ.copy_(dev(Q))
            ctx.cpm_step_graph(m, ne, dx, dQ, dp, b, q, qt)
        st.synchronize()
        got = q.cpu().numpy().copy()
        ref = make_ctx(el, s_prec="fp32", k_prec="fp32").setup(el)
        qr, _ = run_update(ref, psi, run_bvec(ref, elyts))
        assert np.array_equal(got, qr)


@pytest.mark.parametrize("which", ["tiny", "coax"])
def test_fp32_factor_with_fp64_refinement_forms_S(which):
    """cpm_params.chol = FP32_IR: A X = I solved with the FP32 Cholesky factor and refined in FP64 against the
    FP64 A; S (Eq. S) and the charges match the oracle to the FP64 tolerances."""
    need_gpu()
    el = s.au111_slab() if which == "tiny" else s.coaxial_tubes(2)
    A = o.assemble_A(el)
    S = o.capacitance_matrix(A)
    ctx = make_ctx(el, chol="fp32_ir").setup(el)
    sweeps, resid = ctx.cpm_inversion_info()
    assert sweeps >= 1 and resid < 1e-10
    assert rel_l2(ctx.cpm_get_matrix("S").cpu().numpy(), S) <= 1e-10
    ely = s.ions_in_gap(el, 60, seed=2) if which == "tiny" else s.Electrolyte(
        xyz=np.column_stack([np.full(6, 40.0), np.full(6, 41.0), np.linspace(0.5, 4.0, 6)]), Q=np.tile([1.0, -1.0], 3))
    b = run_bvec(ctx, [ely])
    q, qt = run_update(ctx, np.array([0.0, 1.0]), b)
    q_ref = o.charges(S, el, np.array([0.0, 1.0]), o.bvec(el, ely))
    assert rel_l2(q[0], q_ref) <= 1e-10 and abs(qt[0]) <= 1e-12


def test_zero_charge_padding_is_left_out(tiny):
    """Replicas padded with Q = 0 charges stacked on one position (as a server pads a batch) give the same b as
    without padding: zero charges enter no cell of the real-space list."""
    el, ely, _, _, _ = tiny
    ctx = make_ctx(el).setup(el)
    ref = run_bvec(ctx, [ely])[0]
    m, ne = 3, 10 * ely.n
    xyz = np.zeros((m, ne, 3))
    Q = np.zeros((m, ne))
    xyz[:] = ely.xyz[0]
    xyz[1, :ely.n] = ely.xyz
    Q[1, :ely.n] = ely.Q
    b = torch.empty((m, el.n), dtype=torch.float64, device="cuda")
    ctx.cpm_bvec(m, ne, dev(xyz.reshape(-1, 3)), dev(Q.reshape(-1)), b)
    torch.cuda.synchronize()
    b = b.cpu().numpy()
    assert rel_l2(b[1], ref) <= 1e-13
    assert np.abs(b[0]).max() == 0.0 and np.abs(b[2]).max() == 0.0
