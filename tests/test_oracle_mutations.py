"""Planted mistakes in the oracle (on the CPU) must be caught by the pins: each test patches one part of the
oracle with a plausible error and checks that the corresponding pin's criterion fails."""
import math

import numpy as np
import pytest

import bruteforce as bf
from oracle import cpm_oracle as o
from paper_2203_15461_gb300 import systems as s


def _alpha_spread(el0, ely):
    out = []
    for a in (0.28, 0.4):
        el = s.Electrodes(**{**el0.__dict__, "alpha": a, "rcut": 6.0 / a, "kcut": s.kcut_from_tol(a, 1e-17)})
        out.append((o.assemble_A(el), o.bvec(el, ely)))
    (A0, b0), (A1, b1) = out
    return np.linalg.norm(A1 - A0) / np.linalg.norm(A0), np.linalg.norm(b1 - b0) / np.linalg.norm(b0)


@pytest.fixture(scope="module")
def small():
    el, ely, _ = s.workload_tiny_slab(seed=4)
    return el, s.Electrolyte(xyz=ely.xyz[:30], Q=ely.Q[:30])


def test_pin_sees_correct_oracle(small):
    dA, db = _alpha_spread(*small)
    assert dA < 1e-11 and db < 1e-11


@pytest.mark.parametrize("mutation", ["half_weights", "no_background", "wrong_self", "erfc_scale"])
def test_alpha_independence_catches(small, monkeypatch, mutation):
    if mutation == "half_weights":
        orig = o.kweights
        monkeypatch.setattr(o, "kweights", lambda k2, a, V: 0.5 * orig(k2, a, V))
    elif mutation == "no_background":
        orig = o.assemble_A
        monkeypatch.setattr(o, "assemble_A",
                            lambda el, rows=None, kchunk=2048: orig(el, rows, kchunk) + o.K_E * math.pi / (
                                float(np.prod(el.box)) * el.alpha ** 2))
    elif mutation == "wrong_self":
        orig = o.assemble_A
        monkeypatch.setattr(o, "assemble_A", lambda el, rows=None, kchunk=2048: orig(el, rows, kchunk) + np.diag(
            np.full(el.n, o.K_E * el.alpha / math.sqrt(math.pi))))
    else:
        orig = o.erfc
        monkeypatch.setattr(o, "erfc", lambda x: orig(x * (1 + 1e-4)))
    dA, db = _alpha_spread(*small)
    assert max(dA, db) > 1e-6


def test_slab_lattice_sum_catches_missing_dipole_term(monkeypatch):
    rng = np.random.default_rng(7)
    Lx, Ly = 7.0, 6.0
    xyz = np.column_stack([rng.uniform(0, Lx, 5), rng.uniform(0, Ly, 5), rng.uniform(0, 4, 5)])
    eta = rng.uniform(1.2, 2.0, 5)
    q = rng.normal(size=5)
    q -= q.mean()
    Rs = [30, 40, 60, 80, 120, 160]
    E_direct = bf.extrapolate(Rs, [bf.lattice_energy("slab", (Lx, Ly, 0), xyz, eta, q, R) for R in Rs], [1, 2, 3, 4])
    el = s.Electrodes(xyz=xyz, eta=eta, group=np.zeros(5, np.int32), n_groups=1, box=np.array([Lx, Ly, 40.0]),
                      boundary="slab", alpha=0.4, rcut=14.0, kcut=s.kcut_from_tol(0.4, 1e-16))
    good = 0.5 * q @ o.assemble_A(el) @ q / o.K_E
    orig = o.assemble_A
    # the slab term with the wrong factor (2 pi instead of 4 pi on the electrode-electrode part)
    monkeypatch.setattr(o, "assemble_A", lambda e, rows=None, kchunk=2048: orig(e, rows, kchunk) - o.K_E * (
        2.0 * math.pi / float(np.prod(e.box))) * np.outer(e.xyz[:, 2], e.xyz[:, 2]))
    bad = 0.5 * q @ o.assemble_A(el) @ q / o.K_E
    assert abs(good / E_direct - 1) < 1e-7 and abs(bad / E_direct - 1) > 1e-4


def test_cross_sum_catches_sign_of_b(monkeypatch):
    rng = np.random.default_rng(3)
    Lx, Ly = 6.0, 7.0
    r2 = np.random.default_rng(17)
    xyz = np.column_stack([r2.uniform(0, Lx, 4), r2.uniform(0, Ly, 4), r2.uniform(0, 3.0, 4)])
    eta = r2.uniform(1.2, 2.0, 4)
    q = r2.normal(size=4)
    q -= q.mean()
    rj = np.column_stack([rng.uniform(0, Lx, 4), rng.uniform(0, Ly, 4), rng.uniform(3, 8, 4)])
    Q = np.array([1.0, -1.0, 0.5, -0.5])
    Rs = [30, 40, 60, 80, 120, 160]
    ref = bf.extrapolate(Rs, [bf.lattice_cross("slab", (Lx, Ly, 0), xyz, eta, q, rj, Q, R) for R in Rs], [1, 2, 3, 4])
    el = s.Electrodes(xyz=xyz, eta=eta, group=np.zeros(4, np.int32), n_groups=1, box=np.array([Lx, Ly, 60.0]),
                      boundary="slab", alpha=0.4, rcut=14.0, kcut=s.kcut_from_tol(0.4, 1e-16))
    orig = o.bvec
    monkeypatch.setattr(o, "bvec", lambda e, ely, sites=None, kchunk=4096: -orig(e, ely, sites, kchunk))
    got = q @ o.bvec(el, s.Electrolyte(xyz=rj, Q=Q)) / o.K_E
    assert abs(got / ref - 1) > 1.0


def test_capacitance_projection_catches_missing_term(monkeypatch):
    el, _, _ = s.workload_tiny_slab(seed=2)
    A = o.assemble_A(el)
    orig = o.capacitance_matrix
    monkeypatch.setattr(o, "capacitance_matrix", lambda A_, symm=True: orig(A_, symm=False))
    S = o.capacitance_matrix(A)
    e = np.ones(el.n)
    assert np.linalg.norm(S @ e) > 1e-6 * np.linalg.norm(S) * math.sqrt(el.n)
