"""Seeded synthetic inputs: atomic structures, surface meshes, parameter sets, frequency grids.

This module holds no arithmetic of the omega-FQ method or of the BEM operator --
only positions (bohr), surface geometry (normals, element areas, curvatures),
parameter values (atomic units) and frequency lists.  It is the one module that
both the CUDA path and the CPU oracle take their inputs from.

Structures follow the systems of the paper's Section 4: chiral and armchair
carbon nanotubes (Table "CNT data"), graphene disks cut from the honeycomb
lattice (Table "GD data"), hexagonal graphene flakes, and fcc metal
nanoparticles (the sodium nanorod system of Section 4.4 is 3D fcc metal).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903
HARTREE_EV = 27.211386245988
C_AU = 137.035999084          # speed of light, atomic units

CC_BOND_ANG = 1.42            # graphene C-C distance (Section 4, CNT/GD structures)
GRAPHENE_A_ANG = CC_BOND_ANG * math.sqrt(3.0)   # lattice constant, 2.4595 A


def ev(x):
    """Energy in eV -> hartree (frequencies are given to the library in hartree)."""
    return np.asarray(x, dtype=np.float64) / HARTREE_EV


# --------------------------------------------------------------------------- params
# Parameter values are not printed in the paper (they are taken there from earlier
# works); these are this project's documented, unpinned choices.  Only the
# combination 2 n0 * area enters the solution, and the GPU path and the oracle
# always receive the same values.

def carbon_params(eps_fermi_ev: float = 1.51, tau: float = 170.0) -> dict:
    """Graphene / nanotube parameter set (atomic units).

    r0: C-C equilibrium distance; widths from eta via the Eq. 4 width rule; the
    Drude density scales linearly with the Fermi energy (higher eps_F -> more
    carriers, blue shift, as described in Section 4.1)."""
    return {
        "eta": 0.60,
        "d_fermi": 12.0,
        "s_fermi": 1.1,
        "r0": CC_BOND_ANG * BOHR_PER_ANGSTROM,
        "area": 1.0,
        "n0": 0.010 * (eps_fermi_ev / 1.51),
        "tau": float(tau),
        "cutoff_eps": 1e-16,
    }


def sodium_params(tau: float = 170.0) -> dict:
    """fcc sodium-like metal parameter set (atomic units); r0 = a/sqrt(2) for a = 4.23 A."""
    return {
        "eta": 0.35,
        "d_fermi": 12.0,
        "s_fermi": 1.1,
        "r0": 4.23 / math.sqrt(2.0) * BOHR_PER_ANGSTROM,
        "area": 1.0,
        "n0": 0.0080,
        "tau": float(tau),
        "cutoff_eps": 1e-16,
    }


# --------------------------------------------------------------------------- graphene

def _graphene_vectors():
    a = GRAPHENE_A_ANG
    a1 = np.array([a, 0.0])
    a2 = np.array([0.5 * a, 0.5 * math.sqrt(3.0) * a])
    return a1, a2


def honeycomb_flake(n_rings: int) -> np.ndarray:
    """Hexagonal graphene flake with zigzag edges, n_rings hexagons per edge:
    6 n^2 atoms (benzene n=1, coronene n=2, ...).  Planar (z = 0), centred, bohr."""
    if n_rings < 1:
        raise ValueError("n_rings >= 1")
    a1, a2 = _graphene_vectors()
    delta = (a1 + a2) / 3.0
    pts = {}
    for i in range(-(n_rings - 1), n_rings):
        for j in range(-(n_rings - 1), n_rings):
            if max(abs(i), abs(j), abs(i + j)) > n_rings - 1:
                continue
            c = i * a1 + j * a2 + 2.0 * delta
            for k in range(6):
                th = math.radians(90.0 + 60.0 * k)
                p = c + CC_BOND_ANG * np.array([math.cos(th), math.sin(th)])
                key = (round(p[0] * 1e5), round(p[1] * 1e5))
                pts[key] = p
    xy = np.array([pts[k] for k in sorted(pts)])
    xy -= xy.mean(axis=0)
    xyz = np.zeros((len(xy), 3))
    xyz[:, :2] = xy
    return xyz * BOHR_PER_ANGSTROM


def graphene_disk(diameter_nm: float, vacancy_frac: float = 0.0, seed: int | None = None):
    """Graphene disk cut from the honeycomb lattice around a hexagon centre,
    all atoms with |r| < d/2 kept (dangling atoms on the edge are retained, as
    in Section 4.2).  Optionally a fraction of atoms is removed as vacancies by
    a seeded uniform draw.  Planar (z = 0), bohr."""
    a1, a2 = _graphene_vectors()
    delta = (a1 + a2) / 3.0
    centre = 2.0 * delta
    R = 0.5 * diameter_nm * 10.0
    m = int(math.ceil(R / GRAPHENE_A_ANG * 1.2)) + 3
    i, j = np.meshgrid(np.arange(-m, m + 1), np.arange(-m, m + 1), indexing="ij")
    i = i.ravel().astype(np.float64)
    j = j.ravel().astype(np.float64)
    A = np.outer(i, a1) + np.outer(j, a2)
    B = A + delta
    P = np.concatenate([A, B]) - centre
    keep = np.einsum("ij,ij->i", P, P) < R * R
    P = P[keep]
    order = np.lexsort((P[:, 0], P[:, 1]))
    P = P[order]
    if vacancy_frac > 0.0:
        rng = np.random.default_rng(seed)
        nrem = int(round(vacancy_frac * len(P)))
        drop = rng.choice(len(P), size=nrem, replace=False)
        mask = np.ones(len(P), dtype=bool)
        mask[drop] = False
        P = P[mask]
    xyz = np.zeros((len(P), 3))
    xyz[:, :2] = P
    return xyz * BOHR_PER_ANGSTROM


def nanotube_cell(n: int, m: int):
    """Translational unit cell of the (n, m) nanotube: returns
    (atoms_per_cell, period_angstrom, diameter_angstrom)."""
    dR = math.gcd(2 * m + n, 2 * n + m)
    nhex = 2 * (n * n + m * m + n * m) // dR
    ch = GRAPHENE_A_ANG * math.sqrt(n * n + m * m + n * m)
    period = math.sqrt(3.0) * ch / dR
    return 2 * nhex, period, ch / math.pi


def nanotube(n: int, m: int, ncells: int) -> np.ndarray:
    """(n, m) single-walled carbon nanotube of `ncells` translational unit cells,
    rolled from the honeycomb lattice; axis along z, centred, bohr.  The atom
    count is exactly ncells * atoms_per_cell (e.g. (8,12) x 27 cells = 8208)."""
    if n < 0 or m < 0 or n + m == 0:
        raise ValueError("bad chirality")
    dR = math.gcd(2 * m + n, 2 * n + m)
    t1 = (2 * m + n) // dR
    t2 = -(2 * n + m) // dR
    den = n * t2 - m * t1              # lattice-units cross product C_h x T
    # lattice points (u, v) -> alpha along C_h, beta along T, both exact rationals
    corners_u = [0, n, ncells * t1, n + ncells * t1]
    corners_v = [0, m, ncells * t2, m + ncells * t2]
    ui = np.arange(min(corners_u) - 2, max(corners_u) + 3)
    vi = np.arange(min(corners_v) - 2, max(corners_v) + 3)
    U, V = np.meshgrid(ui, vi, indexing="ij")
    U = U.ravel().astype(np.int64)
    V = V.ravel().astype(np.int64)
    out = []
    for off in (0, 1):                 # sublattice A at (u, v), B at (u + 1/3, v + 1/3)
        U3 = 3 * U + off
        V3 = 3 * V + off
        an = U3 * t2 - V3 * t1         # alpha = an / (3 den)
        bn = n * V3 - m * U3           # beta  = bn / (3 den)
        d3 = 3 * den
        if d3 < 0:
            an, bn, d3 = -an, -bn, -d3
        ok = (an >= 0) & (an < d3) & (bn >= 0) & (bn < ncells * d3)
        out.append(np.stack([an[ok] / d3, bn[ok] / d3], axis=1))
    ab = np.concatenate(out)
    cnt, period, diam = nanotube_cell(n, m)
    assert len(ab) == cnt * ncells, (len(ab), cnt * ncells)
    radius = 0.5 * diam
    phi = 2.0 * math.pi * ab[:, 0]
    zc = ab[:, 1] * period
    xyz = np.stack([radius * np.cos(phi), radius * np.sin(phi), zc], axis=1)
    xyz[:, 2] -= 0.5 * ncells * period
    order = np.lexsort((phi, xyz[:, 2]))
    return xyz[order] * BOHR_PER_ANGSTROM


def fcc_sphere(a_ang: float, radius_ang: float, jitter_ang: float = 0.0,
               seed: int | None = None) -> np.ndarray:
    """Atom-centred fcc nanosphere (lattice constant a, all sites with |r| <= R).
    Surface atoms -- fewer than 12 neighbours within 1.1 * a / sqrt(2) -- are
    displaced by a seeded U(-jitter, +jitter) per coordinate.  Bohr."""
    m = int(math.ceil(radius_ang / a_ang)) + 1
    g = np.arange(-m, m + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    base = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1).astype(np.float64)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    P = (base[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a_ang
    P = P[np.einsum("ij,ij->i", P, P) <= radius_ang ** 2 * (1 + 1e-12)]
    P = P[np.lexsort((P[:, 0], P[:, 1], P[:, 2]))]
    if jitter_ang > 0.0:
        from scipy.spatial import cKDTree
        tree = cKDTree(P)
        nn = tree.query_ball_point(P, r=1.1 * a_ang / math.sqrt(2.0), return_length=True) - 1
        surf = nn < 12
        rng = np.random.default_rng(seed)
        shift = rng.uniform(-jitter_ang, jitter_ang, size=(len(P), 3))
        P = P + shift * surf[:, None]
    return P * BOHR_PER_ANGSTROM


def fcc_sphere_radius_for(n_atoms: int, a_ang: float) -> float:
    """Sphere radius (A) whose volume holds about n_atoms fcc sites (4 per a^3)."""
    return (3.0 * n_atoms * a_ang ** 3 / (4.0 * 4.0 * math.pi)) ** (1.0 / 3.0)


def random_cluster(n: int, seed: int, spacing_bohr: float = 2.7, jitter: float = 0.2,
                   planar: bool = False) -> np.ndarray:
    """n atoms drawn without replacement from a jittered cubic (or square) grid:
    no two atoms closer than (1 - 2 jitter) * spacing.  For tests."""
    rng = np.random.default_rng(seed)
    dim = 2 if planar else 3
    side = int(math.ceil((2.0 * n) ** (1.0 / dim)))
    grid = np.stack(np.meshgrid(*[np.arange(side)] * dim, indexing="ij"), axis=-1).reshape(-1, dim)
    pick = rng.choice(len(grid), size=n, replace=False)
    pts = grid[pick].astype(np.float64) + rng.uniform(-jitter, jitter, size=(n, dim))
    pts *= spacing_bohr
    xyz = np.zeros((n, 3))
    xyz[:, :dim] = pts
    xyz -= xyz.mean(axis=0)
    return xyz


# --------------------------------------------------------------------------- surfaces
# Collocation meshes for the continuum (BEM) operator of Section 2.3: one point per surface
# element, with its outward unit normal, its area and the surface's mean curvature there.

def spheroid_surface(n: int, a_bohr: float, b_bohr: float) -> dict:
    """Spheroid x^2/b^2 + y^2/b^2 + z^2/a^2 = 1 (a = b: sphere) with n collocation points.

    The points are a Fibonacci lattice on the unit sphere (polar cosine 1 - (2k+1)/n,
    azimuth k times the golden angle; n cells of equal solid angle 4 pi / n) mapped to the
    spheroid by (b sin t cos p, b sin t sin p, a cos t).  Each element's area is its solid
    angle times the map's area factor b sqrt(a^2 sin^2 t + b^2 cos^2 t); the mean curvature
    is the average of the meridian (a b / q^3) and parallel (a / (b q)) curvatures,
    q = sqrt(a^2 sin^2 t + b^2 cos^2 t).  Seed-free.  Returns xyz, normal (n x 3), area,
    curvature (n), bohr units."""
    k = np.arange(n, dtype=np.float64)
    ct = 1.0 - (2.0 * k + 1.0) / n
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    ph = math.pi * (3.0 - math.sqrt(5.0)) * k
    a, b = float(a_bohr), float(b_bohr)
    q = np.sqrt(a * a * st * st + b * b * ct * ct)
    xyz = np.stack([b * st * np.cos(ph), b * st * np.sin(ph), a * ct], axis=1)
    normal = np.stack([a * st * np.cos(ph), a * st * np.sin(ph), b * ct], axis=1) / q[:, None]
    area = (4.0 * math.pi / n) * b * q
    curvature = 0.5 * (a * b / q ** 3 + a / (b * q))
    return {"xyz": np.ascontiguousarray(xyz), "normal": np.ascontiguousarray(normal),
            "area": area, "curvature": curvature}


def drude_metal_params(omega_p_ev: float = 5.9, gamma_ev: float = 0.1, eps_inf: float = 1.0,
                       eps_out: float = 1.0) -> dict:
    """Free-electron (Drude) metal in a uniform host: eps_in(w) = eps_inf - wp^2 / (w (w + i g)),
    eps_out real.  Defaults: a sodium-like free-electron metal in vacuum (plasma energy 5.9 eV,
    damping 0.1 eV; the sphere's dipole resonance eps_in = -2 eps_out lies at 3.41 eV).
    Atomic units (hartree)."""
    return {"eps_out": float(eps_out), "eps_inf": float(eps_inf),
            "omega_p": omega_p_ev / HARTREE_EV, "gamma": gamma_ev / HARTREE_EV}


def random_complex(shape, seed: int) -> np.ndarray:
    """Seeded standard complex normal array (apply-only inputs)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


# --------------------------------------------------------------------------- workloads

def workload(name: str) -> dict:
    """Named synthetic workloads (positions in bohr, frequencies in hartree).

    flake1k   hexagonal zigzag graphene flake, 13 rings, N = 1014; one frequency at
              the flake's dipolar resonance (0.52 eV with carbon_params(1.51)); x
    cnt20k    armchair (10,10) nanotube, 500 cells, N = 20000; 64 frequencies evenly
              over 0.05-2.0 eV; directions x, y, z
    sphere150k fcc sphere a = 4.23 A, ~150k atoms, surface jitter +-0.05 A; 32
              frequencies over 0.9-1.8 eV; x, y, z
    disk1m    graphene disk with ~1.01M sites, 1% vacancies; 16 frequencies over
              0.05-0.20 eV; direction x
    bem_spheroid30k  continuum (BEM) prolate spheroid, semi-axes 20 nm (z) and 10 nm,
              30000 collocation points, Drude metal in vacuum (drude_metal_params());
              64 frequencies evenly over 2.0-4.5 eV; x, y, z
    """
    dirs3 = np.eye(3)
    if name == "flake1k":
        return {"xyz": honeycomb_flake(13), "params": carbon_params(1.51),
                "omega": ev([0.52]), "dirs": dirs3[:1]}
    if name == "cnt20k":
        return {"xyz": nanotube(10, 10, 500), "params": carbon_params(1.04),
                "omega": ev(np.linspace(0.05, 2.0, 64)), "dirs": dirs3}
    if name == "sphere150k":
        a = 4.23
        R = fcc_sphere_radius_for(150_000, a)
        return {"xyz": fcc_sphere(a, R, 0.05, seed=20210301), "params": sodium_params(),
                "omega": ev(np.linspace(0.9, 1.8, 32)), "dirs": dirs3}
    if name == "disk1m":
        return {"xyz": graphene_disk(183.58, vacancy_frac=0.01, seed=20210304),
                "params": carbon_params(1.84),
                "omega": ev(np.linspace(0.05, 0.20, 16)), "dirs": dirs3[:1]}
    if name == "bem_spheroid30k":
        nm = 10.0 * BOHR_PER_ANGSTROM
        surf = spheroid_surface(30000, 20.0 * nm, 10.0 * nm)
        return {"xyz": surf["xyz"], "surface": surf, "bem": drude_metal_params(),
                "omega": ev(np.linspace(2.0, 4.5, 64)), "dirs": dirs3}
    raise KeyError(name)


def serving_mix(n_requests: int = 2000, seed: int = 20210305, pool_size: str = "small") -> dict:
    """Seeded serving stream over a resident pool of structures from the paper's three
    families (honeycomb flakes, armchair (n, n) nanotubes, fcc sodium-like spheres).

    pool      list of dicts: name, xyz (bohr), params, band (eV) -- 1k to 20k atoms; with
              pool_size="full" also the largest members of each family's range (a 50k-atom
              flake, an 80k-atom (15,15) tube, a 100k-atom sphere)
    requests  list of (structure index, omega (hartree, sorted), dirs (ndir x 3)); each
              request draws its structure uniformly from the pool, 1-64 frequencies
              uniform in the family's band and 1-3 field directions (x, then y, then z)
    gaps      Poisson-process inter-arrival times in units of the mean gap (Exp(1))
    """
    a_na = 4.23
    pool = [
        {"name": "flake1k", "xyz": honeycomb_flake(13), "params": carbon_params(1.51), "band": (0.05, 2.0)},
        {"name": "flake5k", "xyz": honeycomb_flake(29), "params": carbon_params(1.51), "band": (0.05, 2.0)},
        {"name": "flake15k", "xyz": honeycomb_flake(50), "params": carbon_params(1.51), "band": (0.05, 2.0)},
        {"name": "cnt5_5k", "xyz": nanotube(5, 5, 250), "params": carbon_params(1.04), "band": (0.05, 2.0)},
        {"name": "cnt10_10k", "xyz": nanotube(10, 10, 250), "params": carbon_params(1.04), "band": (0.05, 2.0)},
        {"name": "cnt15_20k", "xyz": nanotube(15, 15, 334), "params": carbon_params(1.04), "band": (0.05, 2.0)},
        {"name": "sphere2k", "xyz": fcc_sphere(a_na, fcc_sphere_radius_for(2000, a_na), 0.05, seed=seed),
         "params": sodium_params(), "band": (0.9, 1.8)},
        {"name": "sphere10k", "xyz": fcc_sphere(a_na, fcc_sphere_radius_for(10000, a_na), 0.05, seed=seed + 1),
         "params": sodium_params(), "band": (0.9, 1.8)},
    ]
    if pool_size == "full":
        pool += [
            {"name": "flake50k", "xyz": honeycomb_flake(91), "params": carbon_params(1.51), "band": (0.05, 2.0)},
            {"name": "cnt15_80k", "xyz": nanotube(15, 15, 1334), "params": carbon_params(1.04), "band": (0.05, 2.0)},
            {"name": "sphere100k", "xyz": fcc_sphere(a_na, fcc_sphere_radius_for(100000, a_na), 0.05, seed=seed + 2),
             "params": sodium_params(), "band": (0.9, 1.8)},
        ]
    elif pool_size != "small":
        raise ValueError(pool_size)
    rng = np.random.default_rng(seed)
    dirs3 = np.eye(3)
    reqs = []
    for _ in range(n_requests):
        si = int(rng.integers(0, len(pool)))
        nf = int(rng.integers(1, 65))
        nd = int(rng.integers(1, 4))
        lo, hi = pool[si]["band"]
        reqs.append((si, ev(np.sort(rng.uniform(lo, hi, size=nf))), dirs3[:nd]))
    gaps = rng.exponential(1.0, size=n_requests)
    return {"pool": pool, "requests": reqs, "gaps": gaps}
