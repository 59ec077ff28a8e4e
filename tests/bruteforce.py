"""Independent references used to pin the oracle (no Ewald sums, no oracle code).

* ``gaussian_pair_energy`` integrates the Coulomb energy of two normalised
  Gaussian charge clouds (the electrode charge model of Sec. III.B) by plain
  quadrature: the potential of one cloud from Gauss's law, averaged over the
  other cloud's density.
* ``lattice_energy`` / ``lattice_cross`` sum pair energies directly over the
  periodic images of a small cell (a line of images for a wire, a disc for a
  slab, a sphere for 3D) and extrapolate in the truncation radius.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial.legendre import leggauss
from scipy.special import erf


def _gl(a, b, n):
    x, w = leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def _density(eta, t):
    return (eta * eta / math.pi) ** 1.5 * np.exp(-eta * eta * t * t)


def gaussian_potential(eta, s, n=160):
    """Potential at distance s of a unit Gaussian cloud, by Gauss's law and quadrature."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    x, w = leggauss(n)
    # charge inside radius s over s, plus the potential of the shells outside s
    t_in = 0.5 * s[:, None] * (x[None, :] + 1.0)
    inner = np.sum(0.5 * s[:, None] * w * 4.0 * math.pi * t_in * t_in * _density(eta, t_in), axis=1)
    inner = np.divide(inner, s, out=np.zeros_like(s), where=s > 0)
    tail = 12.0 / eta
    t_out = s[:, None] + 0.5 * tail * (x[None, :] + 1.0)
    outer = np.sum(0.5 * tail * w * 4.0 * math.pi * t_out * _density(eta, t_out), axis=1)
    return inner + outer


def gaussian_pair_energy(eta_i, eta_j, r, nu=120, nc=96):
    """Interaction energy of unit Gaussians (eta_i at 0, eta_j at distance r), e^2/Angstrom."""
    u, wu = _gl(0.0, 9.0 / eta_j, nu)
    c, wc = _gl(-1.0, 1.0, nc)
    U, C = np.meshgrid(u, c, indexing="ij")
    s = np.sqrt(np.maximum(r * r + U * U + 2.0 * r * U * C, 0.0)).ravel()
    # the potential is smooth in s; tabulate on a dense grid and interpolate with a high-order rule
    grid = np.linspace(0.0, s.max() + 1e-9, 4001)
    phi_grid = gaussian_potential(eta_i, grid)
    from scipy.interpolate import CubicSpline
    phi = CubicSpline(grid, phi_grid)(s).reshape(U.shape)
    avg = 0.5 * (phi @ wc)
    return float(np.sum(wu * 4.0 * math.pi * u * u * _density(eta_j, u) * avg))


def _pair_phi(eta_i, eta_j, r):
    """erf(eta_ij r)/r for Gaussians (eta = inf for a point charge), the quadrature-pinned pair law."""
    if np.isinf(eta_i) and np.isinf(eta_j):
        return 1.0 / r
    e = eta_j if np.isinf(eta_i) else eta_i if np.isinf(eta_j) else eta_i * eta_j / math.sqrt(eta_i ** 2 + eta_j ** 2)
    return erf(e * r) / r


def _self_phi(eta):
    """r -> 0 limit of erf(eta r / sqrt 2)/r: the self energy factor of one Gaussian."""
    return math.sqrt(2.0) * eta / math.sqrt(math.pi)


def _lattice_points(kind, box, R):
    if kind == "wire":
        m = int(R // box[2])
        return [np.array([0.0, 0.0, j * box[2]]) for j in range(-m, m + 1)]
    # slab and 3D: R is the number of cells on each side of the central one (a square or cube of
    # whole cells), so the truncated sum is a smooth function of R with no lattice-count noise
    m = int(R)
    ar = np.arange(-m, m + 1)
    if kind == "slab":
        a, b = np.meshgrid(ar, ar, indexing="ij")
        return np.column_stack([a.ravel() * box[0], b.ravel() * box[1], np.zeros(a.size)])
    a, b, c = np.meshgrid(ar, ar, ar, indexing="ij")
    return np.column_stack([a.ravel() * box[0], b.ravel() * box[1], c.ravel() * box[2]])


def lattice_energy(kind, box, xyz, eta, q, R):
    """1/2 sum_ij sum_{|n| <= R} q_i q_j erf(eta_ij |R_ij + n|)/|..| including the Gaussian self energies."""
    pts = np.asarray(_lattice_points(kind, box, R))
    n = len(q)
    E = 0.0
    for i in range(n):
        for j in range(n):
            d = xyz[i] - xyz[j] + pts
            r = np.sqrt(np.einsum("ij,ij->i", d, d))
            e = eta[i] * eta[j] / math.sqrt(eta[i] ** 2 + eta[j] ** 2)
            if i == j:
                r = r[r > 0]
                E += 0.5 * q[i] * q[j] * _self_phi(eta[i])
            E += 0.5 * q[i] * q[j] * np.sum(erf(e * r) / r)
    return E


def lattice_cross(kind, box, xyz, eta, q, rj, Q, R):
    """sum_i sum_j sum_{|n| <= R} q_i Q_j erf(eta_i |R_i - r_j + n|)/|..| (Gaussian sites, point charges)."""
    pts = np.asarray(_lattice_points(kind, box, R))
    E = 0.0
    for i in range(len(q)):
        for j in range(len(Q)):
            d = xyz[i] - rj[j] + pts
            r = np.sqrt(np.einsum("ij,ij->i", d, d))
            E += q[i] * Q[j] * np.sum(erf(eta[i] * r) / r)
    return E


def extrapolate(Rs, Es, powers):
    """Least-squares fit E(R) = E_inf + sum_p c_p / R^p; returns E_inf."""
    Rs = np.asarray(Rs, dtype=np.float64)
    M = np.column_stack([np.ones_like(Rs)] + [Rs ** (-p) for p in powers])
    coef, *_ = np.linalg.lstsq(M, np.asarray(Es), rcond=None)
    return float(coef[0])
