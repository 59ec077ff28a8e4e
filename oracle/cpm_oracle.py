"""Plain FP64 CPU oracle of the constant potential method (CPM) charge update.

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. It shares no code with
the CUDA library and imports nothing from it; the two meet only at the seeded
input arrays.

What it computes (ELECTRODE paper, arXiv 2203.15461):

* The electrode energy is the quadratic form of Eq. (coulomb), Sec. II.A,
  U(q) = 1/2 q^T A q - b^T q - v^T q, with the elastance A fixed by the
  electrode sites and b the electrolyte term.  This module follows the sign
  convention of the library API: ``b`` is the electrostatic potential of the
  electrolyte at each site (the negative of the paper's b), so the minimiser
  is q = S (v - b).
* The electrode charges are Gaussians (Sec. III.B),
  rho_i(r) = q_i (eta^2/pi)^{3/2} exp(-eta^2 |r - R_i|^2).  Two such Gaussians
  interact as erf(eta_ij r)/r with 1/eta_ij^2 = 1/eta_i^2 + 1/eta_j^2; a
  Gaussian and a point charge as erf(eta_i r)/r.  These pair energies are
  summed over the periodic images by the Ewald split used by the paper's
  ``ewald/electrode`` solver (SI Sec. 1.A): a real-space erfc part, a
  reciprocal part over |k| <= kcut, the Ewald self term, the Gaussian self
  energy and the neutralising-background constant.
* Boundary corrections of Sec. II.E: the slab dipole term of Eq. (ew3dc_slab),
  J = 2 pi M_z^2 / V, split into electrode and electrolyte parts as in the last
  equation of Sec. II.E; the wire term of Eq. (ew3dc_wire),
  J = pi (M_x^2 + M_y^2) / V; none for tin-foil 3D.  The exact slab sum (EW2D,
  Sec. II.E) replaces the 3D reciprocal sum, background and dipole term by the
  2D Ewald sum over the in-plane lattice (``ew2d_recip``).
* Inversion and the charge-neutral capacitance matrix of Eq. (S), Sec. II.A:
  S = A^-1 - A^-1 e e^T A^-1 / (e^T A^-1 e).
* The electrode-wise potentials of Sec. II.B: v = G psi, q* = S (v - b)
  (Eq. electrode-wise in API sign), and the electrode-wise capacitance
  C~ = G^T S G (Sec. II.C with S in place of A^-1; Sec. III.B uses it for C0).
* Electrodes at prescribed total charge (Sec. II.C, Eq. ewise-conq), the
  thermo-potentiostat step (Sec. II.D, Eq. deissenbeck) and the finite-field
  site potentials (Sec. II.F, Eq. cpm-ffield).
* The reciprocal part of b by P3M, the mesh solver of the paper's package
  (Introduction; SI Sec. 1.A-B), when the electrodes carry a mesh and an order (``p3m_recip``);
  with ``p3m_matrix`` the reciprocal part of A by the same mesh operator (``p3m_matrix_recip``),
  otherwise A keeps the Ewald sum.

Readings of what the paper leaves open (units, cut-offs, the slab vacuum) are
fixed by the arguments: positions in Angstrom, charges in e, potentials in V,
A in V/e and S in e/V with the Coulomb constant K_E below.  Real-space pairs
count when |r| < rcut over all images of the Ewald cell; reciprocal vectors
count when |k|^2 <= kcut^2, computed as ((kx*kx + ky*ky) + kz*kz) with
k = (2 pi / L) * n per axis.

Parity status: every function here is pinned by tests/test_oracle_pins.py
(brute-force lattice sums, Gaussian-overlap quadrature, alpha independence,
Gauss's law between plates, the co-axial capacitor of Sec. III.B).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import linalg as sla
from scipy.special import erf, erfc, erfcx

#: Coulomb constant e / (4 pi eps0 Angstrom) expressed in volts.
K_E = 14.399645
#: vacuum permittivity in e / (V Angstrom)
EPS0 = 1.0 / (4.0 * math.pi * K_E)

_BC = {"3d": 0, "slab": 1, "wire": 2, "ew2d": 3}


# --------------------------------------------------------------------------- reciprocal lattice

def kvectors(box, kcut):
    """Half-space reciprocal vectors 0 < |k| <= kcut of the Ewald cell ``box``.

    Returns (nidx int64 (Nk,3), k (Nk,3), k2 (Nk,)).  Half space: nx > 0, or
    nx == 0 and ny > 0, or nx == ny == 0 and nz > 0; the other half is its mirror
    image and enters through the factor 2 in the weights.
    """
    box = np.asarray(box, dtype=np.float64)
    tp = 2.0 * np.pi / box
    nmax = [int(math.floor(kcut / tp[d])) + 1 for d in range(3)]
    gx, gy, gz = np.meshgrid(np.arange(0, nmax[0] + 1), np.arange(-nmax[1], nmax[1] + 1),
                             np.arange(-nmax[2], nmax[2] + 1), indexing="ij")
    nidx = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1).astype(np.int64)
    half = (nidx[:, 0] > 0) | ((nidx[:, 0] == 0) & (nidx[:, 1] > 0)) | \
           ((nidx[:, 0] == 0) & (nidx[:, 1] == 0) & (nidx[:, 2] > 0))
    nidx = nidx[half]
    k = nidx * tp
    k2 = k[:, 0] * k[:, 0] + k[:, 1] * k[:, 1] + k[:, 2] * k[:, 2]
    keep = k2 <= kcut * kcut
    return nidx[keep], k[keep], k2[keep]


def kweights(k2, alpha, volume):
    """Half-space Ewald weights 2 * (4 pi / V) exp(-k^2 / 4 alpha^2) / k^2."""
    return (8.0 * np.pi / volume) * np.exp(-k2 / (4.0 * alpha * alpha)) / k2


def kvectors2d(box, kcut):
    """Half-plane 2D reciprocal vectors 0 < |h| <= kcut of the periodic cell (Lx, Ly) of a slab:
    h = 2 pi (nx / Lx, ny / Ly) with nx > 0, or nx == 0 and ny > 0.  Returns (h (Nh, 2), |h| (Nh,))."""
    box = np.asarray(box, dtype=np.float64)
    tp = 2.0 * np.pi / box[:2]
    nmax = [int(math.floor(kcut / tp[d])) + 1 for d in range(2)]
    gx, gy = np.meshgrid(np.arange(0, nmax[0] + 1), np.arange(-nmax[1], nmax[1] + 1), indexing="ij")
    nidx = np.stack([gx.ravel(), gy.ravel()], axis=1)
    half = (nidx[:, 0] > 0) | ((nidx[:, 0] == 0) & (nidx[:, 1] > 0))
    h = nidx[half] * tp
    h2 = h[:, 0] * h[:, 0] + h[:, 1] * h[:, 1]
    keep = h2 <= kcut * kcut
    return h[keep], np.sqrt(h2[keep])


def _ew2d_zfactor(hn, z, alpha):
    """e^{h z} erfc(h / 2a + a z) + e^{-h z} erfc(h / 2a - a z), written with the scaled complementary
    error function where its argument is positive so that no factor overflows."""
    out = np.zeros(np.broadcast(hn, z).shape)
    for sgn in (1.0, -1.0):
        x = hn / (2.0 * alpha) + sgn * alpha * z
        pos = x >= 0
        direct = np.exp(np.where(pos, 0.0, sgn * hn * z)) * erfc(np.where(pos, 0.0, x))
        scaled = erfcx(np.where(pos, x, 0.0)) * np.exp(np.where(pos, -(hn / (2.0 * alpha)) ** 2 - (alpha * z) ** 2, 0.0))
        out += np.where(pos, scaled, direct)
    return out


def ew2d_recip(Ri, Rj, box, alpha, kcut):
    """Long-range part of the slab interaction summed over the 2D lattice exactly (the EW2D method named in
    Sec. II.E; Parry's and Heyes' 2D Ewald sum): for every pair, with rho the in-plane and z the normal
    displacement,
      (pi / A) sum_{h != 0} cos(h . rho) / |h| [e^{|h| z} erfc(|h|/2a + a z) + e^{-|h| z} erfc(|h|/2a - a z)]
      - (2 pi / A) [z erf(a z) + exp(-a^2 z^2) / (a sqrt(pi))],
    A = Lx Ly; the sum over h != 0 runs over the full plane (twice the half plane)."""
    Ri = np.asarray(Ri, dtype=np.float64)
    Rj = np.asarray(Rj, dtype=np.float64)
    area = float(box[0] * box[1])
    h, hn = kvectors2d(box, kcut)
    d = Ri[:, None, :] - Rj[None, :, :]
    z = d[..., 2]
    out = -(2.0 * np.pi / area) * (z * erf(alpha * z) + np.exp(-(alpha * z) ** 2) / (alpha * math.sqrt(math.pi)))
    for k in range(len(hn)):
        ph = h[k, 0] * d[..., 0] + h[k, 1] * d[..., 1]
        out += (2.0 * np.pi / area) * np.cos(ph) / hn[k] * _ew2d_zfactor(hn[k], z, alpha)
    return out


# --------------------------------------------------------------------------- real space

def _image_range(dmin, dmax, L, rcut):
    lo = int(math.floor((-rcut - dmax) / L))
    hi = int(math.ceil((rcut - dmin) / L))
    return range(lo, hi + 1)


def _realspace(Ri, Rj, eta_pair, box, alpha, rcut, same=None, zperiodic=True):
    """sum over images n with |Ri - Rj + n| < rcut of [erfc(alpha r) - erfc(eta r)] / r.

    ``same`` (bool array like eta_pair) marks pairs that are one and the same
    site: for those the n = 0 image is left out (it is the self energy).
    ``zperiodic`` False: images along x and y only (a slab summed in 2D).
    """
    d = Ri[:, None, :] - Rj[None, :, :]
    out = np.zeros(d.shape[:2])
    ranges = [_image_range(d[..., a].min(), d[..., a].max(), box[a], rcut) for a in range(3)]
    if not zperiodic:
        ranges[2] = range(0, 1)
    for ix in ranges[0]:
        for iy in ranges[1]:
            for iz in ranges[2]:
                s = np.array([ix * box[0], iy * box[1], iz * box[2]])
                dd = d + s
                r2 = dd[..., 0] * dd[..., 0] + dd[..., 1] * dd[..., 1] + dd[..., 2] * dd[..., 2]
                m = r2 < rcut * rcut
                if same is not None and ix == 0 and iy == 0 and iz == 0:
                    m &= ~same
                if not m.any():
                    continue
                r = np.sqrt(r2[m])
                e = eta_pair[m] if np.ndim(eta_pair) else eta_pair
                out[m] += (erfc(alpha * r) - erfc(e * r)) / r
    return out


# --------------------------------------------------------------------------- elastance A

def assemble_A(el, rows=None, kchunk=2048):
    """Elastance matrix A (Eq. coulomb) of electrode sites ``el`` in V/e.

    ``rows`` selects a subset of rows (for sampled checks of large systems);
    default all n rows, giving the full symmetric n x n matrix.
    """
    xyz = np.asarray(el.xyz, dtype=np.float64)
    eta = np.asarray(el.eta, dtype=np.float64)
    n = len(xyz)
    rows = np.arange(n) if rows is None else np.asarray(rows)
    box = np.asarray(el.box, dtype=np.float64)
    V = float(box[0] * box[1] * box[2])
    a = el.alpha
    A = np.zeros((len(rows), n))
    # real space: Gaussian-Gaussian pairs, erf(eta_ij r)/r minus the erf(alpha r)/r Ewald part
    for c0 in range(0, len(rows), 256):
        rr = rows[c0:c0 + 256]
        ei, ej = eta[rr][:, None], eta[None, :]
        eta_ij = ei * ej / np.sqrt(ei * ei + ej * ej)
        same = rr[:, None] == np.arange(n)[None, :]
        A[c0:c0 + 256] += _realspace(xyz[rr], xyz, eta_ij, box, a, el.rcut, same, zperiodic=el.boundary != "ew2d")
    if el.boundary == "ew2d":
        # exact 2D-periodic long-range part (no vacuum padding, no dipole correction); the energy of a net
        # charge per cell is undefined in 2D, so A is fixed only up to c e e^T (S and every neutral result
        # do not depend on c): c = (2 pi / A) L_z with L_z = box[2], at least the slab's thickness
        for c0 in range(0, len(rows), 256):
            A[c0:c0 + 256] += ew2d_recip(xyz[rows[c0:c0 + 256]], xyz, box, a, el.kcut)
        A += 2.0 * math.pi * box[2] / (box[0] * box[1])
    elif getattr(el, "p3m_matrix", False) and getattr(el, "p3m_order", 0):
        # reciprocal space by P3M: row i is the mesh potential of a unit charge at site i, interpolated at
        # every site (the operator of p3m_recip applied to one site at a time)
        A += p3m_matrix_recip(el, rows)
        A += -math.pi / (V * a * a)
    else:
        # reciprocal space: sum_k w_k cos(k.(R_i - R_j)) = sum_k w_k [c_i c_j + s_i s_j]
        _, k, k2 = kvectors(box, el.kcut)
        w = kweights(k2, a, V)
        for c0 in range(0, len(k), kchunk):
            kk, ww = k[c0:c0 + kchunk], w[c0:c0 + kchunk]
            ph_all = xyz @ kk.T
            ph_r = ph_all[rows]
            A += (np.cos(ph_r) * ww) @ np.cos(ph_all).T + (np.sin(ph_r) * ww) @ np.sin(ph_all).T
        # neutralising background
        A += -math.pi / (V * a * a)
    # Ewald self term and Gaussian self energy, lim_{r->0} erf(eta r / sqrt2) / r
    A[np.arange(len(rows)), rows] += (math.sqrt(2.0) * eta[rows] - 2.0 * a) / math.sqrt(math.pi)
    # boundary correction, electrode-electrode part (Sec. II.E)
    if el.boundary == "slab":
        A += (4.0 * math.pi / V) * np.outer(xyz[rows, 2], xyz[:, 2])
    elif el.boundary == "wire":
        A += (2.0 * math.pi / V) * (np.outer(xyz[rows, 0], xyz[:, 0]) + np.outer(xyz[rows, 1], xyz[:, 1]))
    return K_E * A


# --------------------------------------------------------------------------- electrolyte vector b

def structure_factor(k, elyt):
    """rho(k) = sum_j Q_j exp(i k . r_j) for the rows of ``k``."""
    ph = np.asarray(elyt.xyz) @ k.T
    Q = np.asarray(elyt.Q)
    return Q @ np.cos(ph) + 1j * (Q @ np.sin(ph))


def bvec(el, elyt, sites=None, kchunk=4096):
    """Electrolyte potential b_i (V) at electrode sites ``sites`` (default all).

    b_i = sum_j Q_j sum_n erf(eta_i |R_i - r_j + n|) / |...| by the same Ewald split as A,
    plus the background and the electrolyte part of the boundary term.
    """
    xyz = np.asarray(el.xyz, dtype=np.float64)
    sites = np.arange(len(xyz)) if sites is None else np.asarray(sites)
    R = xyz[sites]
    eta = np.asarray(el.eta)[sites]
    r = np.asarray(elyt.xyz, dtype=np.float64)
    Q = np.asarray(elyt.Q, dtype=np.float64)
    box = np.asarray(el.box, dtype=np.float64)
    V = float(box[0] * box[1] * box[2])
    a = el.alpha
    b = np.zeros(len(sites))
    if len(Q) and el.boundary == "ew2d":
        for c0 in range(0, len(sites), 256):
            pair = _realspace(R[c0:c0 + 256], r, eta[c0:c0 + 256][:, None] * np.ones((1, len(r))), box, a,
                              el.rcut, zperiodic=False)
            b[c0:c0 + 256] += pair @ Q + ew2d_recip(R[c0:c0 + 256], r, box, a, el.kcut) @ Q
        b += 2.0 * math.pi * box[2] / (box[0] * box[1]) * float(Q.sum())    # the constant c of A, per unit charge
        return K_E * b
    if len(Q) and getattr(el, "p3m_order", 0):
        for c0 in range(0, len(sites), 256):
            pair = _realspace(R[c0:c0 + 256], r, eta[c0:c0 + 256][:, None] * np.ones((1, len(r))), box, a,
                              el.rcut)
            b[c0:c0 + 256] += pair @ Q
        b += p3m_recip(el, elyt, sites)
    elif len(Q):
        for c0 in range(0, len(sites), 256):
            pair = _realspace(R[c0:c0 + 256], r, eta[c0:c0 + 256][:, None] * np.ones((1, len(r))), box, a,
                              el.rcut)
            b[c0:c0 + 256] += pair @ Q
        _, k, k2 = kvectors(box, el.kcut)
        w = kweights(k2, a, V)
        for c0 in range(0, len(k), kchunk):
            kk = k[c0:c0 + kchunk]
            rho = structure_factor(kk, elyt)
            ph = R @ kk.T
            b += (np.cos(ph) * rho.real + np.sin(ph) * rho.imag) @ w[c0:c0 + kchunk]
    Qtot = float(Q.sum())
    b += -math.pi * Qtot / (V * a * a)
    if el.boundary == "slab":
        b += (4.0 * math.pi / V) * R[:, 2] * float(Q @ r[:, 2]) if len(Q) else 0.0
    elif el.boundary == "wire" and len(Q):
        b += (2.0 * math.pi / V) * (R[:, 0] * float(Q @ r[:, 0]) + R[:, 1] * float(Q @ r[:, 1]))
    return K_E * b


# --------------------------------------------------------------------------- P3M reciprocal part

def bspline(p, x):
    """Cardinal B-spline M_p(x) of order p (support [0, p)) by its recursion:
    M_1 = 1 on [0, 1), M_n(x) = (x M_{n-1}(x) + (n - x) M_{n-1}(x - 1)) / (n - 1)."""
    x = np.asarray(x, dtype=np.float64)
    if p == 1:
        return ((x >= 0) & (x < 1)).astype(np.float64)
    return (x * bspline(p - 1, x) + (p - x) * bspline(p - 1, x - 1)) / (p - 1)


def p3m_weights(x, L, K, p):
    """Charge-assignment weights of points x (N,) on the K mesh points m h (h = L / K) of one periodic
    axis: W((x - m h) / h) with W(s) = M_p(s + p / 2), the order-p assignment function centred on the
    point, taken at the nearest periodic image; dense (N, K)."""
    h = L / K
    u = np.mod(np.asarray(x, dtype=np.float64), L) / h
    d = u[:, None] - np.arange(K)[None, :]
    d -= K * np.round(d / K)
    return bspline(p, d + p / 2.0)


def p3m_influence(box, K, p, alpha, nalias=2):
    """Optimal influence function for potentials (Hockney and Eastwood) on the mesh wave vectors
    k = 2 pi n / L (FFT order): G(k) = sum_m U^2(k_m) R(k_m) / (sum_m U^2(k_m))^2 over the aliases
    k_m = k + 2 pi m / h, m in [-nalias, nalias]^3, with U(k) = prod_d sinc(k_d h_d / 2)^p the
    transform of the assignment function and R(k) = 4 pi exp(-k^2 / 4 alpha^2) / k^2; G(0) = 0."""
    box = np.asarray(box, dtype=np.float64)
    h = [box[d] / K[d] for d in range(3)]
    ks = [2.0 * np.pi * np.fft.fftfreq(K[d], d=h[d]) for d in range(3)]
    ms = range(-nalias, nalias + 1)
    u2 = [[np.sinc((ks[d] + 2.0 * np.pi * m / h[d]) * h[d] / (2.0 * np.pi)) ** (2 * p) for m in ms] for d in range(3)]
    num = np.zeros(tuple(K))
    for ix, mx in enumerate(ms):
        kx = ks[0] + 2.0 * np.pi * mx / h[0]
        for iy, my in enumerate(ms):
            ky = ks[1] + 2.0 * np.pi * my / h[1]
            for iz, mz in enumerate(ms):
                kz = ks[2] + 2.0 * np.pi * mz / h[2]
                k2 = kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2
                with np.errstate(divide="ignore", invalid="ignore"):
                    R = np.where(k2 > 0, 4.0 * np.pi * np.exp(-k2 / (4.0 * alpha * alpha)) / k2, 0.0)
                num += u2[0][ix][:, None, None] * u2[1][iy][None, :, None] * u2[2][iz][None, None, :] * R
    den = sum(u2[0])[:, None, None] * sum(u2[1])[None, :, None] * sum(u2[2])[None, None, :]
    G = num / (den * den)
    G[0, 0, 0] = 0.0
    return G


def p3m_matrix_recip(el, rows=None, batch=16):
    """Reciprocal part of A (before K_E) by P3M: entry (i, j) is the potential at site j of the mesh
    solution for a unit charge at site i (rows i, default all), with the assignment function,
    influence function and interpolation of ``p3m_recip``."""
    box = np.asarray(el.box, dtype=np.float64)
    K, p = tuple(int(v) for v in el.p3m_mesh), int(el.p3m_order)
    V = float(box[0] * box[1] * box[2])
    xyz = np.asarray(el.xyz, dtype=np.float64)
    rows = np.arange(len(xyz)) if rows is None else np.asarray(rows)
    W = [p3m_weights(xyz[:, d], box[d], K[d], p) for d in range(3)]
    G = p3m_influence(box, K, p, el.alpha)
    out = np.zeros((len(rows), len(xyz)))
    for c0 in range(0, len(rows), batch):
        rr = rows[c0:c0 + batch]
        rho = np.einsum("bx,by,bz->bxyz", W[0][rr], W[1][rr], W[2][rr])
        phi = (K[0] * K[1] * K[2] / V) * np.real(np.fft.ifftn(G[None] * np.fft.fftn(rho, axes=(1, 2, 3)),
                                                               axes=(1, 2, 3)))
        out[c0:c0 + batch] = np.einsum("ix,iy,iz,bxyz->bi", W[0], W[1], W[2], phi, optimize=True)
    return out


def p3m_recip(el, elyt, sites=None):
    """Reciprocal part of b (before K_E) by P3M (particle-particle particle-mesh, the k-space solver
    of the paper's package): the charges assigned to the mesh, the mesh transformed, multiplied by
    the influence function and transformed back, the mesh potential interpolated at the sites with
    the same assignment function:  phi_m = (1/V) sum_{n != 0} G(k_n) rho^(n) e^{i k_n x_m}.  The mesh
    (el.p3m_mesh) and the order (el.p3m_order) come with the electrodes."""
    box = np.asarray(el.box, dtype=np.float64)
    K, p = tuple(int(v) for v in el.p3m_mesh), int(el.p3m_order)
    V = float(box[0] * box[1] * box[2])
    xyz = np.asarray(el.xyz, dtype=np.float64)
    R = xyz if sites is None else xyz[np.asarray(sites)]
    r = np.asarray(elyt.xyz, dtype=np.float64)
    Q = np.asarray(elyt.Q, dtype=np.float64)
    Wq = [p3m_weights(r[:, d], box[d], K[d], p) for d in range(3)]
    rho = np.einsum("j,jx,jy,jz->xyz", Q, Wq[0], Wq[1], Wq[2], optimize=True)
    G = p3m_influence(box, K, p, el.alpha)
    phi = (K[0] * K[1] * K[2] / V) * np.real(np.fft.ifftn(G * np.fft.fftn(rho)))
    Ws = [p3m_weights(R[:, d], box[d], K[d], p) for d in range(3)]
    return np.einsum("ix,iy,iz,xyz->i", Ws[0], Ws[1], Ws[2], phi, optimize=True)


# --------------------------------------------------------------------------- inversion and charges

def capacitance_matrix(A, symm=True):
    """A^-1 by Cholesky, then the neutral projection of Eq. (S) when ``symm``.

    Raises numpy.linalg.LinAlgError when A is not positive definite.
    """
    n = A.shape[0]
    L = np.linalg.cholesky(A)
    Ainv = sla.cho_solve((L, True), np.eye(n))
    if not symm:
        return Ainv
    e = np.ones(n)
    d = Ainv @ e
    return Ainv - np.outer(d, d) / (e @ d)


def site_potentials(el, psi):
    """v = G psi: the applied potential of each site's electrode (Sec. II.B)."""
    return np.asarray(psi, dtype=np.float64)[np.asarray(el.group)]


def charges(S, el, psi, b):
    """q* = S (v - b) for one electrolyte vector b (n,) or several (n, m)."""
    v = site_potentials(el, psi)
    if np.ndim(b) == 2:
        return S @ (v[:, None] - b)
    return S @ (v - b)


def electrode_capacitance(S, el):
    """C~ = G^T S G, the electrode-wise capacitance matrix (N_g x N_g)."""
    G = np.zeros((el.n, el.n_groups))
    G[np.arange(el.n), np.asarray(el.group)] = 1.0
    return G.T @ S @ G


def energy(A, b, v, q):
    """Electrode energy of Eq. (coulomb) in API sign: 1/2 q^T A q + b^T q - v^T q."""
    return 0.5 * q @ A @ q + b @ q - v @ q


def update(S, el, elyt, psi):
    """One charge update: b for this electrolyte, q = S (v - b), and the total charge."""
    b = bvec(el, elyt)
    q = charges(S, el, psi, b)
    return b, q, float(q.sum())


# --------------------------------------------------------------------------- constant charge method

def indicator(el):
    """Indicator matrix G of Sec. II.B: G[i, g] = 1 when site i belongs to electrode g."""
    G = np.zeros((el.n, el.n_groups))
    G[np.arange(el.n), np.asarray(el.group)] = 1.0
    return G


def ccm_charges(A, el, qtilde, b):
    """Charges at prescribed electrode-wise totals (Sec. II.C, Eq. ewise-conq).

    With the capacitance matrix A^-1 (not S): the totals are q~ = G^T A^-1 (G v~ - b) in the API
    sign of b, i.e. q~ = q~_b + C~ v~ with q~_b = -G^T A^-1 b and C~ = G^T A^-1 G.  Solved for the
    electrode potentials v~, which the CPM then applies: q = A^-1 (G v~ - b).  Returns (q, v~).
    """
    G = indicator(el)
    L = np.linalg.cholesky(A)
    AiG = sla.cho_solve((L, True), G)
    Aib = sla.cho_solve((L, True), np.asarray(b, dtype=np.float64))
    C = G.T @ AiG
    qb = -(G.T @ Aib)
    v = np.linalg.solve(C, np.asarray(qtilde, dtype=np.float64) - qb)
    return AiG @ v - Aib, v


# --------------------------------------------------------------------------- finite-field method

def ffield_zeta(el):
    """zeta of Sec. II.F: z_i / L_z, plus one for the sites of the bottom electrode (the one of lower
    mean z), so that the two electrodes face each other across the periodic z boundary
    (conductor-centred cell).  Two electrodes only."""
    if el.n_groups != 2:
        raise ValueError("the finite-field method takes two electrodes")
    z = np.asarray(el.xyz, dtype=np.float64)[:, 2]
    g = np.asarray(el.group)
    bottom = 0 if z[g == 0].mean() < z[g == 1].mean() else 1
    return z / float(el.box[2]) + (g == bottom).astype(np.float64)


def ffield_charges(S, el, dv0, b):
    """q* = S (v - b) with the site potentials v = -dv0 zeta of Eq. (cpm-ffield) (API sign of b)."""
    return S @ (-float(dv0) * ffield_zeta(el) - np.asarray(b, dtype=np.float64))


# --------------------------------------------------------------------------- thermo-potentiostat

#: Boltzmann constant in eV / K
K_B = 8.617333262e-5


def tp_step(A, S, el, q_cap, dv0, b, dt, tau, T, X):
    """One thermo-potentiostat step (Sec. II.D, Eq. deissenbeck) for two electrodes.

    q_cap is the charge of electrode 1 (electrode 0 carries -q_cap).  The effective potential
    difference dv = v~_1 - v~_0 of the present charges follows from the constant-charge relation
    (Eq. ewise-conq); the vacuum capacitance is C0 = g_1^T S g_1 (Sec. III.B); X is the standard
    normal number of this step.  The new capacitor charge is applied by the constant charge method.
    Returns (q_new, dv, site charges at (-q_new, q_new)).
    """
    if el.n_groups != 2:
        raise ValueError("the thermo-potentiostat takes two electrodes")
    C0 = float(electrode_capacitance(S, el)[1, 1])
    _, v = ccm_charges(A, el, np.array([-q_cap, q_cap]), b)
    dv = float(v[1] - v[0])
    a = math.exp(-dt / tau)
    q_new = q_cap - C0 * (dv - dv0) * (1.0 - a) + X * math.sqrt(K_B * T * C0 * (1.0 - a * a))
    q_sites, _ = ccm_charges(A, el, np.array([-q_new, q_new]), b)
    return q_new, dv, q_sites
