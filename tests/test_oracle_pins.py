"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the part of the method it pins and why a plausible mistake
there (a dropped term, a wrong sign, factor or index) would fail it.
"""
import math

import numpy as np
import pytest

import bruteforce as bf
from oracle import cpm_oracle as o
from paper_2203_15461_gb300 import systems as s

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _sites(xyz, eta, box, boundary, alpha, rcut, ktol, group=None, n_groups=1):
    n = len(xyz)
    return s.Electrodes(xyz=np.asarray(xyz, float), eta=np.asarray(eta, float),
                        group=np.zeros(n, np.int32) if group is None else np.asarray(group, np.int32),
                        n_groups=n_groups, box=np.asarray(box, float), boundary=boundary, alpha=alpha,
                        rcut=rcut, kcut=s.kcut_from_tol(alpha, ktol))


# ----------------------------------------------------------------------------- units

def test_coulomb_constant_from_codata():
    """K_E = e / (4 pi eps0 * 1 Angstrom) in volts, from the SI-exact e and CODATA 2018 eps0."""
    e = 1.602176634e-19
    eps0 = 8.8541878128e-12
    assert abs(e / (4 * math.pi * eps0 * 1e-10) / o.K_E - 1) < 1e-7


# ----------------------------------------------------------------------------- pair law (Sec. III.B)

@pytest.mark.parametrize("ei,ej,r", [(1.979, 1.979, 0.0), (1.805, 1.805, 0.0), (1.979, 1.979, 0.8),
                                     (1.805, 1.2, 2.1), (1.805, 1.2, 0.25)])
def test_gaussian_pair_law_by_quadrature(ei, ej, r):
    """Two unit Gaussian clouds of Sec. III.B interact as erf(eta_ij r)/r, 1/eta_ij^2 = 1/eta_i^2 + 1/eta_j^2;
    r = 0 with eta_i = eta_j is one cloud's self energy sqrt(2) eta/sqrt(pi).  This pins the combination
    rule and the self term that brute-force sums below (and the oracle's A) rely on."""
    E = bf.gaussian_pair_energy(ei, ej, r)
    ref = bf._self_phi(ei) if (r == 0 and ei == ej) else (
        2 * ei * ej / math.sqrt(ei * ei + ej * ej) / math.sqrt(math.pi) if r == 0 else bf._pair_phi(ei, ej, r))
    assert abs(E / ref - 1) < 1e-10


# ----------------------------------------------------------------------------- brute-force lattice sums

def _small_system(seed, n, extent):
    rng = np.random.default_rng(seed)
    xyz = np.column_stack([rng.uniform(0, extent[0], n), rng.uniform(0, extent[1], n),
                           rng.uniform(0, extent[2], n)])
    eta = rng.uniform(1.2, 2.0, n)
    q = rng.normal(size=n)
    return xyz, eta, q - q.mean()


def test_wire_elastance_matches_direct_line_sum():
    """Ewald A + the 1D correction of Eq. (ew3dc_wire) converges, as the x/y vacuum grows, to the direct sum
    over images along z.  Without the correction (or with the wrong sign or factor) the error at 60 A of
    padding is ~1e-4."""
    Lz = 6.0
    xyz, eta, q = _small_system(5, 5, (6, 6, Lz))
    Rs = [400, 800, 1600, 3200, 6400]
    E_direct = bf.extrapolate(Rs, [bf.lattice_energy("wire", (0, 0, Lz), xyz, eta, q, R) for R in Rs], [2, 4])
    Es, Ps = [], [60.0, 90.0, 120.0]
    for P in Ps:
        el = _sites(xyz + [P / 2, P / 2, 0], eta, (P, P, Lz), "wire", 0.35, 16.0, 1e-16)
        Es.append(0.5 * q @ o.assemble_A(el) @ q / o.K_E)
    E_ewald = bf.extrapolate(Ps, Es, [4, 6])
    assert abs(E_ewald / E_direct - 1) < 2e-8
    el3 = _sites(xyz + [30, 30, 0], eta, (60, 60, Lz), "3d", 0.35, 16.0, 1e-16)
    assert abs(0.5 * q @ o.assemble_A(el3) @ q / o.K_E / E_direct - 1) > 1e-4


def test_slab_elastance_matches_direct_plane_sum():
    """Ewald A + the slab correction of Eq. (ew3dc_slab) (electrode-electrode part z_i z_j) equals the direct
    sum over the 2D lattice of images (square truncation, extrapolated); tin-foil 3D does not."""
    Lx, Ly = 7.0, 6.0
    xyz, eta, q = _small_system(7, 5, (Lx, Ly, 4.0))
    Rs = [30, 40, 60, 80, 120, 160]
    E_direct = bf.extrapolate(Rs, [bf.lattice_energy("slab", (Lx, Ly, 0), xyz, eta, q, R) for R in Rs],
                              [1, 2, 3, 4])
    el = _sites(xyz, eta, (Lx, Ly, 40.0), "slab", 0.4, 14.0, 1e-16)
    E = 0.5 * q @ o.assemble_A(el) @ q / o.K_E
    assert abs(E / E_direct - 1) < 1e-7
    el3 = _sites(xyz, eta, (Lx, Ly, 40.0), "3d", 0.4, 14.0, 1e-16)
    assert abs(0.5 * q @ o.assemble_A(el3) @ q / o.K_E / E_direct - 1) > 1e-3


def test_tinfoil_3d_elastance_matches_cube_sum_minus_surface_term():
    """Tin-foil Ewald = direct sum over a growing cube of cells minus the surface term 2 pi |M|^2 / 3V
    (de Leeuw, Perram and Smith); pins the reciprocal weights, self and background terms in 3D."""
    L = (6.5, 6.5, 6.5)   # a cube of cubic cells has the sphere's depolarisation factors 1/3
    xyz, eta, q = _small_system(11, 4, L)
    Rs = [8, 10, 12, 16, 20, 24]
    E_cube = bf.extrapolate(Rs, [bf.lattice_energy("3d", L, xyz, eta, q, R) for R in Rs], [1, 2, 3])
    M = q @ xyz
    V = L[0] * L[1] * L[2]
    el = _sites(xyz, eta, L, "3d", 0.5, 12.0, 1e-16)
    E = 0.5 * q @ o.assemble_A(el) @ q / o.K_E
    assert abs(E - (E_cube - 2 * math.pi * (M @ M) / (3 * V))) < 1e-6 * abs(E)


@pytest.mark.parametrize("kind", ["wire", "slab"])
def test_electrolyte_vector_matches_direct_cross_sum(kind):
    """q^T b equals the direct image sum of Gaussian-site / point-charge energies erf(eta_i r)/r, including the
    electrolyte part of the boundary term (z_i M_z for the slab, x_i M_x + y_i M_y for the wire)."""
    rng = np.random.default_rng(3)
    if kind == "wire":
        Lz = 5.0
        xyz, eta, q = _small_system(13, 4, (5, 5, Lz))
        rj = np.column_stack([rng.uniform(0, 5, 4), rng.uniform(0, 5, 4), rng.uniform(0, Lz, 4)])
        Q = np.array([1.0, -1.0, 0.5, -0.5])
        Rs = [400, 800, 1600, 3200, 6400]
        ref = bf.extrapolate(Rs, [bf.lattice_cross("wire", (0, 0, Lz), xyz, eta, q, rj, Q, R) for R in Rs], [2, 4])
        Es, Ps = [], [60.0, 90.0, 120.0]
        for P in Ps:
            sh = np.array([P / 2, P / 2, 0])
            el = _sites(xyz + sh, eta, (P, P, Lz), "wire", 0.35, 16.0, 1e-16)
            Es.append(q @ o.bvec(el, s.Electrolyte(xyz=rj + sh, Q=Q)) / o.K_E)
        got = bf.extrapolate(Ps, Es, [4, 6])
        assert abs(got / ref - 1) < 2e-8
    else:
        Lx, Ly = 6.0, 7.0
        xyz, eta, q = _small_system(17, 4, (Lx, Ly, 3.0))
        rj = np.column_stack([rng.uniform(0, Lx, 4), rng.uniform(0, Ly, 4), rng.uniform(3, 8, 4)])
        Q = np.array([1.0, -1.0, 0.5, -0.5])
        Rs = [30, 40, 60, 80, 120, 160]
        ref = bf.extrapolate(Rs, [bf.lattice_cross("slab", (Lx, Ly, 0), xyz, eta, q, rj, Q, R) for R in Rs],
                             [1, 2, 3, 4])
        el = _sites(xyz, eta, (Lx, Ly, 60.0), "slab", 0.4, 14.0, 1e-16)
        got = q @ o.bvec(el, s.Electrolyte(xyz=rj, Q=Q)) / o.K_E
        assert abs(got / ref - 1) < 1e-7


# ----------------------------------------------------------------------------- Ewald splitting

def test_alpha_independence_of_A_b_S_q():
    """A (with its background constant), b for a NON-neutral electrolyte, S and q do not depend on the Ewald
    splitting alpha once both sums are converged.  A wrong reciprocal weight, self term, background term or
    cut-off rule breaks this at the 1e-3 level."""
    el0, ely, psi = s.workload_tiny_slab(seed=4)
    pick = np.r_[0:21, 50:70]   # 21 cations, 20 anions: net charge +1 e
    ely = s.Electrolyte(xyz=ely.xyz[pick], Q=ely.Q[pick])
    assert abs(ely.Q.sum() - 1.0) < 1e-12
    res = []
    for a in (0.28, 0.34, 0.42):
        rc = 6.0 / a   # erfc(6) ~ 2e-17
        el = s.Electrodes(**{**el0.__dict__, "alpha": a, "rcut": rc, "kcut": s.kcut_from_tol(a, 1e-17)})
        A = o.assemble_A(el)
        b = o.bvec(el, ely)
        S = o.capacitance_matrix(A)
        res.append((A, b, S, o.charges(S, el, psi, b)))
    for A, b, S, q in res[1:]:
        A0, b0, S0, q0 = res[0]
        assert np.linalg.norm(A - A0) / np.linalg.norm(A0) < 1e-11
        assert np.linalg.norm(b - b0) / np.linalg.norm(b0) < 1e-11
        assert np.linalg.norm(S - S0) / np.linalg.norm(S0) < 1e-10
        assert np.linalg.norm(q - q0) / np.linalg.norm(q0) < 1e-10


# ----------------------------------------------------------------------------- Eq. (S) and the charge solution

@pytest.fixture(scope="module")
def tiny():
    el, ely, psi = s.workload_tiny_slab(seed=2)
    A = o.assemble_A(el)
    S = o.capacitance_matrix(A)
    b = o.bvec(el, ely)
    return el, ely, psi, A, S, b


def test_A_symmetric_positive_definite(tiny):
    el, _, _, A, _, _ = tiny
    assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


def test_S_projection_properties(tiny):
    """Eq. (S): S symmetric, S e = 0, and S is unchanged when c e e^T is added to A (so the background
    constant and any uniform shift of A drop out)."""
    el, _, _, A, S, _ = tiny
    e = np.ones(el.n)
    assert np.abs(S - S.T).max() <= 1e-12 * np.abs(S).max()
    assert np.linalg.norm(S @ e) <= 1e-13 * np.linalg.norm(S) * math.sqrt(el.n)
    S2 = o.capacitance_matrix(A + 3.7 * np.outer(e, e))
    assert np.linalg.norm(S2 - S) <= 1e-11 * np.linalg.norm(S)
    Sinv = o.capacitance_matrix(A, symm=False)
    assert np.linalg.norm(Sinv @ A - np.eye(el.n)) < 1e-10


def test_charges_neutral_optimal_and_kkt(tiny):
    """q* = S(v - b) is neutral, satisfies A q* + b - v = lambda e (stationarity with the neutrality
    multiplier) and no neutral perturbation lowers the Eq. (coulomb) energy."""
    el, _, psi, A, S, b = tiny
    q = o.charges(S, el, psi, b)
    v = o.site_potentials(el, psi)
    assert abs(q.sum()) < 1e-12
    r = A @ q + b - v
    assert np.abs(r - r.mean()).max() < 1e-10 * np.abs(v - b).max()
    U0 = o.energy(A, b, v, q)
    rng = np.random.default_rng(0)
    for _ in range(5):
        d = rng.normal(size=el.n) * 1e-3
        d -= d.mean()
        assert o.energy(A, b, v, q + d) > U0


def test_charges_linear_in_potential(tiny):
    """Eq. (electrode-wise): at fixed b the charges are affine in psi; in vacuum they scale with psi."""
    el, _, _, _, S, b = tiny
    q = lambda p: o.charges(S, el, np.asarray(p, float), b)
    lhs = q([0.3, 1.1]) + q([-0.2, 0.6]) - q([0.0, 0.0])
    assert np.linalg.norm(lhs - q([0.1, 1.7])) < 1e-12 * np.linalg.norm(lhs)
    z = np.zeros(el.n)
    assert np.linalg.norm(o.charges(S, el, [0, 2.0], z) - 2 * o.charges(S, el, [0, 1.0], z)) < 1e-13


def test_slab_translation_invariance():
    """Shifting every electrode site and ion by the same z leaves q unchanged for a neutral electrolyte:
    the origin of the dipole terms of Sec. II.E drops out after the neutral projection."""
    el, ely, psi = s.workload_tiny_slab(seed=6)
    q0 = o.charges(o.capacitance_matrix(o.assemble_A(el)), el, psi, o.bvec(el, ely))
    sh = np.array([0.0, 0.0, 3.3])
    el2 = s.Electrodes(**{**el.__dict__, "xyz": el.xyz + sh})
    ely2 = s.Electrolyte(xyz=ely.xyz + sh, Q=ely.Q)
    q1 = o.charges(o.capacitance_matrix(o.assemble_A(el2)), el2, psi, o.bvec(el2, ely2))
    assert np.linalg.norm(q1 - q0) / np.linalg.norm(q0) < 1e-11


# ----------------------------------------------------------------------------- physics closed forms

def test_gauss_law_field_between_plates():
    """Between two charged plates the potential is linear in z with slope sigma/eps0 (Gauss's law), sigma the
    charge per area of the positive electrode.  Ties the normalisation of b (probe potential) to A."""
    el = s.au111_slab()
    S = o.capacitance_matrix(o.assemble_A(el))
    q = S @ o.site_potentials(el, [0.0, 1.0])
    Q2 = q[el.group == 1].sum()
    zs = np.linspace(el.z_inner[0] + 7, el.z_inner[1] - 7, 7)
    probes = np.column_stack([np.full(7, 3.1), np.full(7, 5.2), zs])
    pel = s.Electrodes(xyz=probes, eta=np.full(7, 1.979), group=np.zeros(7, np.int32), n_groups=1, box=el.box,
                       boundary="slab", alpha=el.alpha, rcut=el.rcut, kcut=el.kcut)
    phi = o.bvec(pel, s.Electrolyte(xyz=el.xyz, Q=q))
    slope, icpt = np.polyfit(zs, phi, 1)
    assert abs(slope / (Q2 / (o.EPS0 * el.area)) - 1) < 1e-6
    assert np.abs(np.polyval([slope, icpt], zs) - phi).max() < 1e-7


def test_parallel_plate_capacitance_slope():
    """Vacuum capacitor: 1/C0 is linear in the gap d with slope 1/(eps0 Area) (C0 = eps0 A / d_eff).
    C0 = g_2^T S g_2 (Sec. II.C, III.B)."""
    inv = []
    ds = (20.0, 30.0, 40.0)
    for d in ds:
        el = s.au111_slab(gap=d)
        C = o.electrode_capacitance(o.capacitance_matrix(o.assemble_A(el)), el)
        assert abs(C[0, 0] - C[1, 1]) < 1e-12 and abs(C[0, 1] + C[1, 1]) < 1e-12
        inv.append(1.0 / C[1, 1])
    area = s.au111_slab().area
    for sl in np.diff(inv) / np.diff(ds):
        assert abs(sl * o.EPS0 * area - 1) < 1e-6


def test_coaxial_capacitor_sec_IIIB():
    """Sec. III.B: co-axial tubes with the 1D correction.  C0/L is the same for 1, 2 and 3 periodic cells (it
    is a property per length), approaches 2 pi eps0 / ln(R2/R1) as the radii grow at a fixed ratio, and is
    larger for wider Gaussians (smaller eta)."""
    CL = []
    for nc in (1, 2, 3):
        el = s.coaxial_tubes(nc)
        CL.append(o.electrode_capacitance(o.capacitance_matrix(o.assemble_A(el)), el)[1, 1] / el.box[2])
    assert max(CL) - min(CL) < 1e-9 * CL[0]
    ana = 2 * math.pi * o.EPS0 / math.log(2.0)
    dev_small = CL[0] / ana - 1
    el = s.coaxial_tubes(1, n_inner=20, n_outer=40, pad=2.0)
    dev_large = o.electrode_capacitance(o.capacitance_matrix(o.assemble_A(el)), el)[1, 1] / el.box[2] / ana - 1
    assert 0 < dev_large < dev_small < 0.1
    C_eta = []
    for eta in (1.5, 1.805, 2.2):
        el = s.coaxial_tubes(1, eta=eta)
        C_eta.append(o.electrode_capacitance(o.capacitance_matrix(o.assemble_A(el)), el)[1, 1])
    assert C_eta[0] > C_eta[1] > C_eta[2]


# ----------------------------------------------------------------------------- constant charge method (Sec. II.C)

def test_ccm_totals_and_stationarity(tiny):
    """Eq. (ewise-conq): the charges carry exactly the prescribed electrode totals (also non-neutral ones) and
    are stationary for the Eq. (coulomb) energy under those constraints: A q + b - G v~ = 0, the electrode
    potentials v~ being the multipliers of the electrode totals."""
    el, _, _, A, _, b = tiny
    G = o.indicator(el)
    for qt in ([-0.7, 0.7], [0.25, 1.1]):
        q, v = o.ccm_charges(A, el, qt, b)
        assert np.abs(G.T @ q - np.asarray(qt)).max() < 1e-12
        r = A @ q + b - G @ v
        assert np.abs(r).max() < 1e-10 * np.abs(b).max()


def test_ccm_reproduces_cpm_at_its_totals(tiny):
    """Prescribing the electrode totals that the CPM (Eq. electrode-wise) produces at potentials psi gives back the
    same charges, and potentials that differ from psi by one constant (S fixes v only up to a uniform shift)."""
    el, _, psi, A, S, b = tiny
    q_cpm = o.charges(S, el, psi, b)
    q, v = o.ccm_charges(A, el, o.indicator(el).T @ q_cpm, b)
    assert np.linalg.norm(q - q_cpm) < 1e-10 * np.linalg.norm(q_cpm)
    d = v - np.asarray(psi)
    assert abs(d[1] - d[0]) < 1e-10


def test_ccm_vacuum_capacitor_voltage_slope():
    """Vacuum plate capacitor at charges (-Q, Q): the potential difference is Q / C0 and grows with the gap at
    1 / (eps0 Area) per Angstrom per unit charge (parallel-plate law), independent of the CPM path."""
    Q = 0.8
    dv = []
    ds = (20.0, 30.0, 40.0)
    for d in ds:
        el = s.au111_slab(gap=d)
        _, v = o.ccm_charges(o.assemble_A(el), el, [-Q, Q], np.zeros(el.n))
        dv.append(v[1] - v[0])
    area = s.au111_slab().area
    for sl in np.diff(dv) / np.diff(ds):
        assert abs(sl * o.EPS0 * area / Q - 1) < 1e-6


# ----------------------------------------------------------------------------- finite field (Sec. II.F)

def _sheets(gap, Lz=None):
    el = s.au111_slab(seed_layers=1, gap=gap, slab_factor=12.0)
    if Lz is None:
        return el
    return s.Electrodes(**{**el.__dict__, "box": np.array([el.box[0], el.box[1], Lz]), "boundary": "3d"})


def test_ffield_periodic_cell_approaches_the_vacuum_capacitor():
    """Eq. (cpm-ffield): a plate capacitor in a fully periodic cell driven by the field term, without vacuum
    padding, carries the charge of the same plates under the CPM with slab correction and a large vacuum,
    at Delta psi = Delta v0: the difference shrinks as the periodic length grows (about 1/L) and is below
    1e-2 at L = 600 A.  A wrong sign, or the zeta offset on the wrong electrode, fails by far."""
    dv0 = 1.0
    el_v = _sheets(20.0)
    q_cpm = o.charges(o.capacitance_matrix(o.assemble_A(el_v)), el_v, [0.0, dv0], np.zeros(el_v.n))
    Q_ref = q_cpm[el_v.group == 1].sum()
    devs = []
    for Lz in (150.0, 300.0, 600.0):
        el = _sheets(20.0, Lz)
        q = o.ffield_charges(o.capacitance_matrix(o.assemble_A(el)), el, dv0, np.zeros(el.n))
        assert abs(q.sum()) < 1e-12
        devs.append(abs(q[el.group == 1].sum() / Q_ref - 1))
    assert devs[0] > devs[1] > devs[2] and devs[2] < 1e-2, devs
    assert 1.6 < devs[0] / devs[1] < 2.4 and 1.6 < devs[1] / devs[2] < 2.4


def test_ffield_charges_linear_in_field(tiny):
    el = _sheets(20.0, 150.0)
    S = o.capacitance_matrix(o.assemble_A(el))
    z = np.zeros(el.n)
    assert np.linalg.norm(o.ffield_charges(S, el, 2.0, z) - 2 * o.ffield_charges(S, el, 1.0, z)) < 1e-13


# ----------------------------------------------------------------------------- thermo-potentiostat (Sec. II.D)

@pytest.fixture(scope="module")
def tp_system():
    el, ely, _ = s.workload_tiny_slab(seed=4)
    A = o.assemble_A(el)
    S = o.capacitance_matrix(A)
    return el, A, S, o.bvec(el, ely)


def test_tp_deterministic_limit_is_the_cpm_charge(tp_system):
    """Eq. (deissenbeck) with T = 0 and tau << dt: one step sets the capacitor charge to the CPM charge of
    electrode 1 at Delta v0 with the same electrolyte (Eq. electrode-wise), and the site charges to the CPM
    charges."""
    el, A, S, b = tp_system
    dv0 = 1.3
    q_new, _, qs = o.tp_step(A, S, el, 0.37, dv0, b, dt=1.0, tau=1.0 / 60.0, T=0.0, X=0.0)
    q_cpm = o.charges(S, el, [0.0, dv0], b)
    assert abs(q_new - q_cpm[el.group == 1].sum()) < 1e-10 * abs(q_new)
    assert np.linalg.norm(qs - q_cpm) < 1e-10 * np.linalg.norm(q_cpm)


def test_tp_relaxes_geometrically(tp_system):
    """T = 0: q_n - q_eq = a^n (q_0 - q_eq) with a = exp(-dt/tau) exactly (linear response of the circuit)."""
    el, A, S, b = tp_system
    dv0, dt, tau = 0.8, 1.0, 3.0
    q_eq = o.charges(S, el, [0.0, dv0], b)[el.group == 1].sum()
    q0 = q = -0.4
    for n in range(1, 6):
        q, _, _ = o.tp_step(A, S, el, q, dv0, b, dt, tau, 0.0, 0.0)
        assert abs((q - q_eq) - math.exp(-n * dt / tau) * (q0 - q_eq)) < 1e-11


def test_tp_fluctuation_dissipation():
    """At temperature T the capacitor charge fluctuates about the CPM charge with variance k_B T C0 (the
    fluctuation-dissipation relation the thermo-potentiostat is built on); 20,000 seeded steps of an 8-site
    capacitor, variance within 6 % (3.5 standard errors) and mean within 4 standard errors."""
    rng = np.random.default_rng(5)
    xyz = np.array([[0, 0, 0], [4, 0, 0], [0, 4, 0], [4, 4, 0], [0, 0, 10], [4, 0, 10], [0, 4, 10], [4, 4, 10.0]])
    el = _sites(xyz + 1.0, np.full(8, 1.805), [8.0, 8.0, 40.0], "slab", 0.35, 7.0, 1e-10,
                group=[0, 0, 0, 0, 1, 1, 1, 1], n_groups=2)
    A = o.assemble_A(el)
    S = o.capacitance_matrix(A)
    C0 = o.electrode_capacitance(S, el)[1, 1]
    T, dv0, dt, tau = 300.0, 0.5, 1.0, 1.0 / math.log(2.0)     # a = 1/2
    b = np.zeros(el.n)
    q, qs = C0 * dv0, []
    for k in range(20500):
        q, _, _ = o.tp_step(A, S, el, q, dv0, b, dt, tau, T, rng.normal())
        if k >= 500:
            qs.append(q)
    qs = np.asarray(qs)
    var = o.K_B * T * C0
    assert abs(qs.var() / var - 1) < 0.06
    n_eff = len(qs) * (1 - 0.5) / (1 + 0.5)
    assert abs(qs.mean() - C0 * dv0) < 4 * math.sqrt(var / n_eff)


# ----------------------------------------------------------------------------- EW2D (Sec. II.E)

def test_ew2d_elastance_matches_direct_plane_sum():
    """The exact 2D Ewald sum (EW2D) equals the direct sum over the 2D lattice of images with no vacuum and no
    dipole correction: tighter than EW3DC at 40 A of vacuum (1e-7), because nothing is approximated."""
    Lx, Ly = 7.0, 6.0
    xyz, eta, q = _small_system(7, 5, (Lx, Ly, 4.0))
    Rs = [30, 40, 60, 80, 120, 160]
    E_direct = bf.extrapolate(Rs, [bf.lattice_energy("slab", (Lx, Ly, 0), xyz, eta, q, R) for R in Rs],
                              [1, 2, 3, 4])
    for alpha in (0.4, 0.6):
        el = _sites(xyz, eta, (Lx, Ly, 1.0), "ew2d", alpha, 14.0, 1e-16)
        E = 0.5 * q @ o.assemble_A(el) @ q / o.K_E
        assert abs(E / E_direct - 1) < 2e-9, (alpha, E / E_direct - 1)


def test_ew2d_electrolyte_vector_matches_direct_cross_sum():
    """q^T b under EW2D equals the direct 2D image sum of Gaussian-site / point-charge energies, for a charged
    electrolyte too (the h = 0 term carries the slab's mean field)."""
    Lx, Ly = 7.0, 6.5
    xyz, eta, q = _small_system(3, 4, (Lx, Ly, 3.0))
    rng = np.random.default_rng(4)
    rj = np.column_stack([rng.uniform(0, Lx, 3), rng.uniform(0, Ly, 3), rng.uniform(5, 9, 3)])
    Q = np.array([1.0, -0.4, 0.7])
    Rs = [30, 40, 60, 80, 120, 160]
    E_direct = bf.extrapolate(Rs, [bf.lattice_cross("slab", (Lx, Ly, 0), xyz, eta, q, rj, Q, R) for R in Rs],
                              [1, 2, 3, 4])
    el = _sites(xyz, eta, (Lx, Ly, 1.0), "ew2d", 0.45, 14.0, 1e-16)
    E = q @ o.bvec(el, s.Electrolyte(xyz=rj, Q=Q)) / o.K_E
    assert abs(E / E_direct - 1) < 1e-8, E / E_direct - 1


def test_ew3dc_converges_to_ew2d_with_vacuum():
    """Sec. II.E: the dipole-corrected 3D sum approaches the exact 2D sum as the vacuum grows."""
    el, ely, psi = s.workload_tiny_slab(seed=2)
    q2 = o.charges(o.capacitance_matrix(o.assemble_A(s.Electrodes(**{**el.__dict__, "boundary": "ew2d"}))),
                   el, psi, o.bvec(s.Electrodes(**{**el.__dict__, "boundary": "ew2d"}), ely))
    errs = []
    for f in (3.0, 6.0):
        e3 = s.au111_slab(slab_factor=f)
        q3 = o.charges(o.capacitance_matrix(o.assemble_A(e3)), e3, psi, o.bvec(e3, ely))
        errs.append(np.linalg.norm(q3 - q2) / np.linalg.norm(q2))
    assert errs[1] < errs[0] < 5e-2, errs


def test_ew2d_constant_leaves_S_unchanged(tiny):
    """The undetermined constant of the EW2D elastance (c e e^T) drops out of S (Eq. S)."""
    el = s.Electrodes(**{**tiny[0].__dict__, "boundary": "ew2d"})
    S1 = o.capacitance_matrix(o.assemble_A(el))
    el2 = s.Electrodes(**{**el.__dict__, "box": el.box * np.array([1.0, 1.0, 1.7])})
    S2 = o.capacitance_matrix(o.assemble_A(el2))
    assert np.linalg.norm(S2 - S1) < 1e-11 * np.linalg.norm(S1)


# ----------------------------------------------------------------------------- P3M (Introduction; SI Sec. 1.A-B; Hockney and Eastwood)

def _p3m(el, K, p):
    return s.Electrodes(**{**el.__dict__, "p3m_mesh": K, "p3m_order": p})


def test_p3m_converges_to_the_ewald_sum(tiny):
    """The mesh solution approaches the (pinned) Ewald reciprocal sum as the mesh is refined, at least as
    fast as h^p: order 7 reaches 1e-8 of the reciprocal part on a 32 x 32 x 128 mesh and 1e-10 on 64 x 64 x 256."""
    el, ely, _, _, _, _ = tiny
    elk = s.Electrodes(**{**el.__dict__, "kcut": s.kcut_from_tol(el.alpha, 1e-14)})
    box = np.asarray(el.box)
    _, k, k2 = o.kvectors(box, elk.kcut)
    rho = o.structure_factor(k, ely)
    ph = el.xyz @ k.T
    ref = (np.cos(ph) * rho.real + np.sin(ph) * rho.imag) @ o.kweights(k2, el.alpha, float(np.prod(box)))
    errs = {}
    for p in (5, 7):
        for K in ((16, 16, 64), (32, 32, 128), (64, 64, 256)):
            b = o.p3m_recip(_p3m(elk, K, p), ely)
            errs[p, K] = np.linalg.norm(b - ref) / np.linalg.norm(ref)
    for p in (5, 7):
        e = [errs[p, K] for K in ((16, 16, 64), (32, 32, 128), (64, 64, 256))]
        assert e[0] / e[1] > 2 ** (p - 1) and e[1] / e[2] > 2 ** (p - 1), (p, e)
    assert errs[7, (32, 32, 128)] < 1e-8 and errs[7, (64, 64, 256)] < 1e-10


def test_p3m_shift_by_one_mesh_spacing(tiny):
    """Moving every site and charge by one mesh spacing along each axis leaves the mesh solution unchanged
    (to rounding): the assignment, the periodic wrap and the transforms use one and the same mesh."""
    el, ely, _, _, _, _ = tiny
    K = (16, 16, 64)
    elp = _p3m(el, K, 5)
    b0 = o.p3m_recip(elp, ely)
    for d in range(3):
        sh = np.zeros(3)
        sh[d] = el.box[d] / K[d]
        b1 = o.p3m_recip(s.Electrodes(**{**elp.__dict__, "xyz": el.xyz + sh}), s.Electrolyte(xyz=ely.xyz + sh, Q=ely.Q))
        assert np.abs(b1 - b0).max() < 1e-12 * np.abs(b0).max()


def test_p3m_weights_partition_unity():
    """The order-p assignment weights of any point sum to one over the mesh and vanish beyond p points."""
    x = np.random.default_rng(3).uniform(0, 10.0, 50)
    for p in (2, 5, 7):
        W = o.p3m_weights(x, 10.0, 32, p)
        assert np.abs(W.sum(axis=1) - 1).max() < 1e-13
        assert ((W > 0).sum(axis=1) <= p).all()


def _p3m_matrix(el, K, p):
    return s.Electrodes(**{**el.__dict__, "p3m_mesh": K, "p3m_order": p, "p3m_matrix": True})


def test_p3m_matrix_converges_to_the_ewald_elastance(tiny):
    """A with its reciprocal part from P3M approaches the (pinned) Ewald A at least as h^(p-1) per mesh
    doubling (order 7: within 1e-8 at 32 x 32 x 128); the charges follow."""
    el, ely, psi, _, _, _ = tiny
    elk = s.Electrodes(**{**el.__dict__, "kcut": s.kcut_from_tol(el.alpha, 1e-14)})
    Ae = o.assemble_A(elk)
    for p in (5, 7):
        e = [np.linalg.norm(o.assemble_A(_p3m_matrix(el, K, p)) - Ae) / np.linalg.norm(Ae)
             for K in ((16, 16, 64), (32, 32, 128))]
        assert e[0] / e[1] > 2 ** (p - 1), (p, e)
    elp = _p3m_matrix(el, (32, 32, 128), 7)
    Ap = o.assemble_A(elp)
    assert np.linalg.norm(Ap - Ae) / np.linalg.norm(Ae) < 1e-8
    q_ew = o.charges(o.capacitance_matrix(Ae), el, psi, o.bvec(elk, ely))
    q_p3m = o.charges(o.capacitance_matrix(Ap), el, psi, o.bvec(elp, ely))
    assert np.linalg.norm(q_p3m - q_ew) / np.linalg.norm(q_ew) < 1e-7


def test_p3m_matrix_is_the_b_operator(tiny):
    """The matrix applied to charges q at the sites equals the mesh potential that the b path computes
    for point charges q placed at the same positions (one operator, two evaluations: site by site, and
    all charges in one mesh), and it is symmetric."""
    el, _, _, _, _, _ = tiny
    elp = _p3m_matrix(el, (16, 16, 64), 6)
    R = o.p3m_matrix_recip(elp)
    q = np.random.default_rng(5).normal(size=el.n)
    b = o.p3m_recip(elp, s.Electrolyte(xyz=el.xyz, Q=q))
    assert np.linalg.norm(R @ q - b) <= 1e-13 * np.linalg.norm(b)
    assert np.linalg.norm(R - R.T) <= 1e-14 * np.linalg.norm(R)
