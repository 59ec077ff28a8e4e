"""The single-precision real-space part of b (gathered candidate lists, fitted pair function with
the tabulated function inside the Gaussian cores) against the oracle, through the C ABI.

Cases: charges 0.05 to 2 A from sites of two Gaussian widths (the tabulated branch and two
tables), dense electrolytes whose candidate lists overflow the kernel's shared-memory list (the
list is evaluated in pieces), charges on the periodic faces of the cell, and splittings whose
fit needs the higher polynomial degree or none (the tabulated kernel).  b within 2e-6 relative L2
of the oracle (single-precision real and reciprocal sums), and bit-identical on a second call.
"""
import numpy as np
import pytest

from gpu_util import dev, make_ctx, need_gpu, rel_l2, run_bvec, torch
from oracle import cpm_oracle as o
from paper_2203_15461_gb300 import systems as s

pytestmark = pytest.mark.gpu


def _ctx(el, k_prec="fp32"):
    ctx = make_ctx(el, k_prec=k_prec)
    ctx.cpm_assemble(dev(el.xyz), dev(el.eta), dev(el.group, torch.int32), el.n_groups)
    return ctx


def _two_widths(el):
    eta = el.eta.copy()
    eta[1::2] = 2.6
    return s.Electrodes(**{**el.__dict__, "eta": eta})


def _close_charges(el, rng, dists=(0.05, 0.3, 1.0, 1.6, 2.0)):
    """Charges at the given distances from randomly chosen sites, in random directions."""
    pick = rng.choice(el.n, size=len(dists) * 3, replace=False)
    xyz, Q = [], []
    for k, i in enumerate(pick):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        xyz.append(el.xyz[i] + dists[k % len(dists)] * d)
        Q.append(1.0 if k % 2 else -1.0)
    return np.array(xyz), np.array(Q)


def test_charges_inside_the_gaussian_cores_two_widths():
    need_gpu()
    el = _two_widths(s.au111_slab())
    rng = np.random.default_rng(5)
    ions = s.ions_in_gap(el, 80, seed=6)
    cx, cq = _close_charges(el, rng)
    ely = s.Electrolyte(xyz=np.vstack([ions.xyz, cx]), Q=np.concatenate([ions.Q, cq]))
    ctx = _ctx(el)
    b = run_bvec(ctx, [ely, ions])
    assert rel_l2(b[0], o.bvec(el, ely)) <= 2e-6
    assert rel_l2(b[1], o.bvec(el, ions)) <= 2e-6
    assert np.array_equal(run_bvec(ctx, [ely, ions]), b)


def test_dense_electrolyte_overflows_the_candidate_list():
    """About 2,800 candidates per site chunk: the kernel evaluates its list in pieces."""
    need_gpu()
    el = s.au111_slab()
    rng = np.random.default_rng(9)
    n = 4000
    zlo, zhi = el.z_inner[0] + 1.0, el.z_inner[1] - 1.0
    xyz = np.column_stack([rng.uniform(0, el.box[0], n), rng.uniform(0, el.box[1], n), rng.uniform(zlo, zhi, n)])
    Q = rng.choice([-1.0, 1.0], size=n) * rng.uniform(0.2, 1.0, n)
    ely = s.Electrolyte(xyz=xyz, Q=Q)
    ctx = _ctx(el)
    b = run_bvec(ctx, [ely, s.jitter(ely, 0.3, rng)])
    assert rel_l2(b[0], o.bvec(el, ely)) <= 2e-6
    assert np.array_equal(run_bvec(ctx, [ely, s.jitter(ely, 0.3, np.random.default_rng(9))])[0], b[0])


def test_charges_on_the_periodic_faces():
    """Charges exactly on x = 0, x = L_x, y = 0 and outside the cell (wrapped by the cell list)."""
    need_gpu()
    el = s.au111_slab()
    ions = s.ions_in_gap(el, 60, seed=12)
    xyz = ions.xyz.copy()
    xyz[0, 0] = 0.0
    xyz[1, 0] = el.box[0]
    xyz[2, 1] = 0.0
    xyz[3, 1] = el.box[1] * 2.0 - 1e-9
    xyz[4, :2] -= el.box[:2] * 3.0
    ely = s.Electrolyte(xyz=xyz, Q=ions.Q)
    b = run_bvec(_ctx(el), [ely])
    assert rel_l2(b[0], o.bvec(el, ely)) <= 2e-6


@pytest.mark.parametrize("rcut", [12.0, 15.0, 20.0, 24.0], ids=["deg12", "deg12_wide", "deg14", "table"])
def test_splittings(rcut):
    """alpha r_c = 3.6, 4.5, 6 and 7.2: the degree-12 fit of erfcx (twice), the degree-14 fit, and the
    tabulated kernel (the fit is not used past alpha r_c = 7)."""
    need_gpu()
    el = s.au111_slab(rcut=rcut)
    elyts = [s.ions_in_gap(el, 100, seed=20 + k) for k in range(3)]
    b = run_bvec(_ctx(el), elyts)
    for r, e in enumerate(elyts):
        assert rel_l2(b[r], o.bvec(el, e)) <= 2e-6, r


def test_wire_and_tinfoil():
    need_gpu()
    for el in (s.coaxial_tubes(2), s.Electrodes(**{**s.au111_slab().__dict__, "boundary": "3d"})):
        ely = s.ions_in_gap(s.au111_slab(), 60, seed=3) if el.boundary == "3d" else None
        if ely is None:
            rng = np.random.default_rng(4)
            n = 120
            c = el.box / 2.0
            ang = rng.uniform(0, 2 * np.pi, n)
            rad = rng.uniform(s.tube_radius(10) + 2.0, s.tube_radius(20) - 2.0, n)
            ely = s.Electrolyte(xyz=np.column_stack([c[0] + rad * np.cos(ang), c[1] + rad * np.sin(ang),
                                                     rng.uniform(0, el.box[2], n)]),
                                Q=np.where(np.arange(n) % 2 == 0, 1.0, -1.0))
        b = run_bvec(_ctx(el), [ely])
        assert rel_l2(b[0], o.bvec(el, ely)) <= 2e-6, el.boundary
