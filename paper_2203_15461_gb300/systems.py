"""Seeded synthetic inputs for the constant potential method (CPM) workloads.

This module only builds inputs: electrode site positions, Gaussian widths and
electrode group ids, electrolyte point charges, the Ewald box and the cut-offs.
It evaluates nothing of the method itself (no Ewald sums, no matrices, no
charges), so the CUDA library and the FP64 CPU oracle can both take their
inputs from here without sharing any of the method's arithmetic.

The paper's own systems (the Au/NaCl(aq) capacitor of Sec. III.A, the co-axial
nanotubes of Sec. III.B) need equilibrated structures that are not available;
these generators stand in for them with the same shapes: layered FCC(111) gold
and hexagonal graphene-like electrodes, armchair nanotubes, and randomly placed
ions and rigid 3-site waters with a minimum separation.

Units throughout: Angstrom, elementary charge, volt.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

BOUNDARIES = ("3d", "slab", "wire", "ew2d")


@dataclass
class Electrodes:
    """Fixed electrode sites of one geometry (Sec. II.A: A depends only on them)."""

    xyz: np.ndarray          # (n, 3) float64 site positions, row-major
    eta: np.ndarray          # (n,) float64 inverse Gaussian widths (Sec. III.B)
    group: np.ndarray        # (n,) int32 electrode index of each site (Sec. II.B)
    n_groups: int
    box: np.ndarray          # (3,) Ewald cell (Lx, Ly, Lz); vacuum padding included
    boundary: str            # "3d" tin-foil, "slab" (EW3DC, Eq. ew3dc_slab), "wire" (Eq. ew3dc_wire),
                             # "ew2d" (exact 2D-periodic slab sum; box[2] is then not a period)
    alpha: float             # Ewald splitting parameter, 1/Angstrom
    rcut: float              # real-space cut-off, Angstrom
    kcut: float              # reciprocal-space cut-off |k| <= kcut, 1/Angstrom
    area: float = 0.0        # electrode area in the periodic plane (slab only)
    z_inner: tuple = ()      # z of the inner surface layer of the bottom / top electrode
    name: str = ""
    p3m_mesh: tuple = ()     # P3M mesh points per axis (powers of two) for the reciprocal part of b
    p3m_order: int = 0       # P3M assignment order (0: Ewald sum)
    p3m_matrix: bool = False # the reciprocal part of A by P3M as well (else the Ewald sum)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


@dataclass
class Electrolyte:
    """Point charges of one electrolyte configuration."""

    xyz: np.ndarray          # (N_e, 3) float64
    Q: np.ndarray            # (N_e,) float64 charges in e
    kinds: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int8))

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


def kcut_from_tol(alpha: float, tol: float) -> float:
    """Reciprocal cut-off at which the Gaussian screening factor exp(-k^2/4a^2) equals tol."""
    return 2.0 * alpha * math.sqrt(-math.log(tol))


# --------------------------------------------------------------------------- electrodes

def _fcc111_layer(nx: int, ny: int, a_nn: float, shift: tuple) -> np.ndarray:
    """Hexagonal close-packed layer in a rectangular nx x ny cell (ny even)."""
    row = a_nn * math.sqrt(3.0) / 2.0
    pts = []
    for r in range(ny):
        for i in range(nx):
            pts.append(((i + 0.5 * (r % 2)) * a_nn + shift[0], r * row + shift[1]))
    return np.asarray(pts, dtype=np.float64)


def au111_slab(seed_layers: int = 3, nx: int = 6, ny: int = 6, a: float = 4.08, gap: float = 20.0,
               eta: float = 1.979, slab_factor: float = 3.0, alpha: float = 0.3, rcut: float = 12.0,
               ktol: float = 1e-8) -> Electrodes:
    """Two Au(111)-like FCC electrodes, `seed_layers` layers of nx x ny atoms each, ABC stacked."""
    a_nn = a / math.sqrt(2.0)
    dz = a / math.sqrt(3.0)
    Lx, Ly = nx * a_nn, ny * a_nn * math.sqrt(3.0) / 2.0
    # ABC stacking: successive layers shift by one third of the rectangular cell diagonal
    shifts = [(0.0, 0.0), (a_nn / 2.0, a_nn / (2.0 * math.sqrt(3.0))), (0.0, a_nn / math.sqrt(3.0))]
    xyz, grp = [], []
    for e in range(2):
        for l in range(seed_layers):
            z = l * dz if e == 0 else (seed_layers - 1) * dz + gap + l * dz
            st = shifts[l % 3] if e == 0 else shifts[(seed_layers - 1 - l) % 3]
            xy = _fcc111_layer(nx, ny, a_nn, st)
            xyz.append(np.column_stack([np.mod(xy[:, 0], Lx), np.mod(xy[:, 1], Ly), np.full(len(xy), z)]))
            grp.append(np.full(len(xy), e, np.int32))
    xyz = np.concatenate(xyz)
    h = xyz[:, 2].max() - xyz[:, 2].min()
    z_in = ((seed_layers - 1) * dz, (seed_layers - 1) * dz + gap)
    return Electrodes(xyz=xyz, eta=np.full(len(xyz), eta), group=np.concatenate(grp), n_groups=2,
                      box=np.array([Lx, Ly, slab_factor * h]), boundary="slab", alpha=alpha, rcut=rcut,
                      kcut=kcut_from_tol(alpha, ktol), area=Lx * Ly, z_inner=z_in, name="au111")


def _graphene_layer(cx: int, cy: int, shift: tuple, acc: float = 1.42) -> np.ndarray:
    """Graphene sheet built from rectangular 4-atom cells (sqrt(3)acc x 3acc)."""
    a, b = math.sqrt(3.0) * acc, 3.0 * acc
    basis = np.array([[0.0, 0.0], [a / 2, acc / 2], [a / 2, 1.5 * acc], [0.0, 2.0 * acc]])
    pts = [basis + np.array([i * a, j * b]) for j in range(cy) for i in range(cx)]
    xy = np.concatenate(pts) + np.asarray(shift)
    return np.column_stack([np.mod(xy[:, 0], cx * a), np.mod(xy[:, 1], cy * b)])


def graphene_plates(cx: int, cy: int, layers: int, gap: float, eta: float = 1.805, interlayer: float = 3.35,
                    slab_factor: float = 3.0, alpha: float = 0.3, rcut: float = 12.0, ktol: float = 1e-8,
                    acc: float = 1.42) -> Electrodes:
    """Two graphite-like electrodes of `layers` AB-stacked sheets, inner sheets `gap` apart."""
    a, b = math.sqrt(3.0) * acc, 3.0 * acc
    Lx, Ly = cx * a, cy * b
    xyz, grp = [], []
    top0 = (layers - 1) * interlayer + gap
    for e in range(2):
        for l in range(layers):
            z = l * interlayer if e == 0 else top0 + l * interlayer
            st = (0.0, 0.0) if l % 2 == 0 else (0.0, acc)
            xy = _graphene_layer(cx, cy, st, acc)
            xyz.append(np.column_stack([xy, np.full(len(xy), z)]))
            grp.append(np.full(len(xy), e, np.int32))
    xyz = np.concatenate(xyz)
    h = xyz[:, 2].max() - xyz[:, 2].min()
    return Electrodes(xyz=xyz, eta=np.full(len(xyz), eta), group=np.concatenate(grp), n_groups=2,
                      box=np.array([Lx, Ly, slab_factor * h]), boundary="slab", alpha=alpha, rcut=rcut,
                      kcut=kcut_from_tol(alpha, ktol), area=Lx * Ly,
                      z_inner=((layers - 1) * interlayer, top0), name=f"graphene{cx}x{cy}x{layers}")


def armchair_tube(nch: int, n_cells: int, center: tuple, acc: float = 1.42) -> np.ndarray:
    """Atoms of an (nch, nch) armchair nanotube, axis along z, n_cells unit cells of length sqrt(3)acc."""
    a = math.sqrt(3.0) * acc
    circ = 3.0 * acc * nch
    r = circ / (2.0 * math.pi)
    pts = []
    for c in range(n_cells):
        for k in range(nch):
            s0 = 3.0 * acc * k
            for s, z in ((s0, 0.0), (s0 + acc, 0.0), (s0 + 1.5 * acc, a / 2), (s0 + 2.5 * acc, a / 2)):
                th = s / r
                pts.append((center[0] + r * math.cos(th), center[1] + r * math.sin(th), c * a + z))
    return np.asarray(pts, dtype=np.float64)


def coaxial_tubes(n_cells: int, n_inner: int = 10, n_outer: int = 20, eta: float = 1.805, pad: float = 3.0,
                  alpha: float = 0.3, rcut: float = 12.0, ktol: float = 1e-8, acc: float = 1.42) -> Electrodes:
    """Co-axial armchair tubes, periodic along z only (Sec. III.B); x, y padded with vacuum."""
    a = math.sqrt(3.0) * acc
    r_out = 3.0 * acc * n_outer / (2.0 * math.pi)
    Lxy = pad * 2.0 * r_out
    c = (Lxy / 2.0, Lxy / 2.0)
    inner = armchair_tube(n_inner, n_cells, c, acc)
    outer = armchair_tube(n_outer, n_cells, c, acc)
    xyz = np.concatenate([inner, outer])
    grp = np.concatenate([np.zeros(len(inner), np.int32), np.ones(len(outer), np.int32)])
    return Electrodes(xyz=xyz, eta=np.full(len(xyz), eta), group=grp, n_groups=2,
                      box=np.array([Lxy, Lxy, n_cells * a]), boundary="wire", alpha=alpha, rcut=rcut,
                      kcut=kcut_from_tol(alpha, ktol), name=f"coax{n_inner}-{n_outer}x{n_cells}")


def tube_radius(nch: int, acc: float = 1.42) -> float:
    return 3.0 * acc * nch / (2.0 * math.pi)


# --------------------------------------------------------------------------- electrolytes

def _min_image_ok(p: np.ndarray, acc: np.ndarray, box_xy: tuple, dmin: float) -> bool:
    if len(acc) == 0:
        return True
    d = acc - p
    d[:, 0] -= box_xy[0] * np.round(d[:, 0] / box_xy[0])
    d[:, 1] -= box_xy[1] * np.round(d[:, 1] / box_xy[1])
    return bool(np.min(np.einsum("ij,ij->i", d, d)) >= dmin * dmin)


def _place_centers(rng: np.random.Generator, count: int, box_xy: tuple, zlo: float, zhi: float,
                   dmin: float, max_tries: int = 200000) -> np.ndarray:
    """Random sequential placement with a periodic (x, y) minimum separation."""
    acc = np.zeros((0, 3))
    out = np.zeros((count, 3))
    k = tries = 0
    while k < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place electrolyte centres at the requested density")
        p = np.array([rng.uniform(0, box_xy[0]), rng.uniform(0, box_xy[1]), rng.uniform(zlo, zhi)])
        if _min_image_ok(p, acc[:k] if k else acc, box_xy, dmin):
            out[k] = p
            acc = out
            k += 1
    return out


def ions_in_gap(el: Electrodes, n_ions: int, seed: int, margin: float = 2.5, dmin: float = 2.5) -> Electrolyte:
    """n_ions point charges +-1 e (half each) uniform in the slab gap, dmin apart."""
    rng = np.random.default_rng(seed)
    zlo, zhi = el.z_inner[0] + margin, el.z_inner[1] - margin
    xyz = _place_centers(rng, n_ions, (el.box[0], el.box[1]), zlo, zhi, dmin)
    Q = np.where(np.arange(n_ions) < n_ions // 2, 1.0, -1.0)
    return Electrolyte(xyz=xyz, Q=Q, kinds=np.where(Q > 0, 1, 2).astype(np.int8))


WATER_Q = (-0.8476, 0.4238, 0.4238)


def _water_hydrogens(rng: np.random.Generator, O: np.ndarray, r_oh: float = 1.0,
                     angle_deg: float = 109.47) -> tuple:
    n = len(O)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    t = rng.normal(size=(n, 3))
    t -= np.einsum("ij,ij->i", t, u)[:, None] * u
    t /= np.linalg.norm(t, axis=1)[:, None]
    th = math.radians(angle_deg)
    u2 = math.cos(th) * u + math.sin(th) * t
    return O + r_oh * u, O + r_oh * u2


def water_and_ions(el: Electrodes, n_water: int, n_cat: int, n_an: int, seed: int, margin: float = 2.5,
                   dmin: float = 2.5) -> Electrolyte:
    """Rigid 3-site waters (O -0.8476, H +0.4238, 1.0 A, 109.47 deg) plus +1/-1 ions in the gap."""
    rng = np.random.default_rng(seed)
    zlo, zhi = el.z_inner[0] + margin, el.z_inner[1] - margin
    centers = _place_centers_grid(rng, n_water + n_cat + n_an, (el.box[0], el.box[1]), zlo, zhi, dmin)
    O = centers[:n_water]
    H1, H2 = _water_hydrogens(rng, O)
    ions = centers[n_water:]
    xyz = np.concatenate([O, H1, H2, ions])
    Q = np.concatenate([np.full(n_water, WATER_Q[0]), np.full(2 * n_water, WATER_Q[1]),
                        np.ones(n_cat), -np.ones(n_an)])
    kinds = np.concatenate([np.full(n_water, 3), np.full(2 * n_water, 4), np.full(n_cat, 1),
                            np.full(n_an, 2)]).astype(np.int8)
    return Electrolyte(xyz=xyz, Q=Q, kinds=kinds)


def _place_centers_grid(rng: np.random.Generator, count: int, box_xy: tuple, zlo: float, zhi: float,
                        dmin: float, max_tries_factor: int = 200) -> np.ndarray:
    """Random sequential placement using a cell grid (for thousands of centres)."""
    nxc = max(1, int(box_xy[0] // dmin))
    nyc = max(1, int(box_xy[1] // dmin))
    nzc = max(1, int((zhi - zlo) // dmin))
    cells: dict = {}
    out = np.zeros((count, 3))
    k = tries = 0
    while k < count:
        tries += 1
        if tries > max_tries_factor * count:
            raise RuntimeError("could not place electrolyte centres at the requested density")
        p = np.array([rng.uniform(0, box_xy[0]), rng.uniform(0, box_xy[1]), rng.uniform(zlo, zhi)])
        ci = (int(p[0] / box_xy[0] * nxc) % nxc, int(p[1] / box_xy[1] * nyc) % nyc,
              min(nzc - 1, int((p[2] - zlo) / (zhi - zlo) * nzc)))
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    key = ((ci[0] + dx) % nxc, (ci[1] + dy) % nyc, ci[2] + dz)
                    for j in cells.get(key, ()):
                        d = out[j] - p
                        d[0] -= box_xy[0] * round(d[0] / box_xy[0])
                        d[1] -= box_xy[1] * round(d[1] / box_xy[1])
                        if d @ d < dmin * dmin:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            out[k] = p
            cells.setdefault(ci, []).append(k)
            k += 1
    return out


def jitter(elyt: Electrolyte, sigma: float, rng: np.random.Generator) -> Electrolyte:
    """One random-walk step of all electrolyte positions, N(0, sigma) per coordinate."""
    return replace(elyt, xyz=elyt.xyz + rng.normal(scale=sigma, size=elyt.xyz.shape))


# --------------------------------------------------------------------------- named workloads

def workload_tiny_slab(seed: int = 1):
    """Au(111) 3 layers x 6 x 6 per electrode (216 sites), 100 ions in a 20 A gap; psi = (0, 1) V."""
    el = au111_slab()
    return el, ions_in_gap(el, 100, seed), np.array([0.0, 1.0])


#: Ewald splitting of the EDL capacitor, balanced between the real-space and reciprocal sums for
#: 5,700 charges and 4,320 sites at fixed accuracy (erfc(alpha rcut) = erfc(3.6), k tolerance 1e-8):
#: on a GB300 the per-update time is flat for alpha in [0.18, 0.22] and 26% higher at 0.3.
EDL_ALPHA = 0.2


def workload_edl_capacitor(seed: int = 1, cells=(18, 10), layers: int = 3, gap: float = 60.0,
                           n_water: int = 1800, n_ion: int = 150, alpha: float = EDL_ALPHA):
    """Graphene-like 3-layer electrodes (4,320 sites), 1,800 waters + 150 Na+ + 150 Cl- in a 60 A gap."""
    el = graphene_plates(cells[0], cells[1], layers, gap, alpha=alpha, rcut=3.6 / alpha)
    return el, water_and_ions(el, n_water, n_ion, n_ion, seed), np.array([0.0, 1.0])


#: Ewald splitting of the serving geometries at the same accuracy (erfc(alpha r_c) = erfc(3.6), k tolerance
#: 1e-8).  The reciprocal set grows as V alpha^3 and the one-time FP64 assembly as n^2 N_k, so the two
#: large boxes take a smaller alpha (longer real-space cut-off): about 34k and 29k k-vectors instead of
#: 116k and 225k at alpha = 0.3.
SERVING_ALPHA = {512: 0.3, 2048: 0.3, 8192: 0.2, 16384: 0.15}


def serving_electrodes(n_sites: int, gap: float = 40.0) -> Electrodes:
    """Two electrodes of two graphene sheets each with n_sites sites in total (512 ... 16,384)."""
    per_layer = n_sites // 4
    cells = per_layer // 4
    table = {32: (8, 4), 128: (16, 8), 512: (32, 16), 1024: (32, 32)}
    cx, cy = table[cells]
    alpha = SERVING_ALPHA.get(n_sites, 0.3)
    return graphene_plates(cx, cy, 2, gap, alpha=alpha, rcut=3.6 / alpha)


def with_p3m(el: Electrodes, order: int = 7, h_alpha: float = 0.35, matrix: bool = False) -> Electrodes:
    """The electrodes with the reciprocal part of b (and with ``matrix`` of A) from P3M: per axis the
    smallest power-of-two mesh (at least 8 points) whose spacing h keeps h alpha <= h_alpha (0.35 with
    order 7 puts b within about 1e-7 of the Ewald sum for the geometries here)."""
    K = tuple(int(max(8, 2 ** math.ceil(math.log2(math.ceil(L * el.alpha / h_alpha))))) for L in el.box)
    return Electrodes(**{**el.__dict__, "p3m_mesh": K, "p3m_order": order, "p3m_matrix": matrix})


def workload_serving_geometry(n_sites: int, seed: int = 1, charges_per_site: float = 1.0, gap: float = 40.0):
    """Serving geometry (``serving_electrodes``) with an electrolyte of charges_per_site x n_sites charges."""
    el = serving_electrodes(n_sites, gap)
    rng = np.random.default_rng(seed)
    n_q = int(round(charges_per_site * n_sites))
    n_ion = max(1, n_q // 6)
    n_water = max(0, (n_q - 2 * n_ion) // 3)
    # above one charge per site the 40 A gap is too crowded for random sequential placement at a
    # 2.5 A minimum separation of the water oxygens and ions; 2.2 A still keeps every pair apart
    dmin = 2.5 if charges_per_site <= 1.0 else 2.2
    return el, water_and_ions(el, n_water, n_ion, n_ion, int(rng.integers(1 << 30)), dmin=dmin), np.array([0.0, 1.0])
