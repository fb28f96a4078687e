"""Seeded synthetic workloads shaped like the paper's indentation cells.

Each builder returns a dict with positions x (n,3), velocities v, box, fixed mask,
mass, species, region (ACE weight), indenter, and the potential parameter dicts.
The paper's own cells (Tabs. setup_parameters_copper / setup_parameters_tungsten)
and its trained potentials are not available; these stand in for them.
"""
import numpy as np

from .lattice import bcc, fcc, maxwell_velocities, orthorhombic_box, random_displacements
from .potentials import ace_potential, eam_potential

MS_TO_AFS = 1e-5           # 1 m/s = 1e-5 Angstrom/fs


def _bundle(species, x, v, box, fixed, region, indenter, ind_vel):
    eam = eam_potential(species)
    return {"species": species, "x": x, "v": v, "box": box, "fixed": fixed,
            "mass": float(eam["mass_amu"]), "region": region, "indenter": indenter,
            "ind_vel": None if ind_vel is None else np.asarray(ind_vel, dtype=np.float64),
            "eam": eam, "ace": ace_potential(species)}


def cu_bulk(ncell=8, a=3.615, sigma=0.05, seed=1001, r_in=10.0, r_sw=3.0):
    """Cu FCC bulk, fully periodic, Gaussian displacements; ACE sphere at the box centre."""
    x = fcc(a, ncell, ncell, ncell)
    x = x + random_displacements(len(x), sigma, seed)
    L = ncell * a
    box = orthorhombic_box(L, L, L, (1, 1, 1))
    region = {"kind": "sphere", "center": (L / 2, L / 2, L / 2), "r_in": r_in, "r_sw": r_sw}
    return _bundle("Cu", x, np.zeros_like(x), box, np.zeros(len(x), dtype=np.uint8), region, None, None)


def w_bulk(ncell=6, a=3.165, sigma=0.05, seed=1011, r_in=5.0, r_sw=3.0):
    """W BCC bulk, fully periodic, Gaussian displacements; ACE sphere at the box centre."""
    x = bcc(a, ncell, ncell, ncell)
    x = x + random_displacements(len(x), sigma, seed)
    L = ncell * a
    box = orthorhombic_box(L, L, L, (1, 1, 1))
    region = {"kind": "sphere", "center": (L / 2, L / 2, L / 2), "r_in": r_in, "r_sw": r_sw}
    return _bundle("W", x, np.zeros_like(x), box, np.zeros(len(x), dtype=np.uint8), region, None, None)


def w_slab(ncell=40, nz=None, a=3.165, temperature=300.0, seed=1002, r_in=50.0, r_sw=4.0,
           R=40.0, K=10.0, v_ms=10.0, penetration=1.0, n_fixed_layers=3, vacuum=10.0):
    """W BCC (001) indentation slab: periodic x/y, free top surface, bottom layers fixed.

    The ACE region is a sphere centred on the surface point under the tip, so inside the
    slab it is the hemisphere of the paper's fixed-zone scheme (Sec. 2.2.3).  The tip
    centre starts at z_surf + R - penetration and moves down at v_ms.
    """
    nz = ncell if nz is None else nz
    x = bcc(a, ncell, ncell, nz)
    n = len(x)
    zs = np.unique(np.round(x[:, 2], 6))
    fixed = (x[:, 2] < zs[n_fixed_layers] - 1e-6).astype(np.uint8)
    mass = float(eam_potential("W")["mass_amu"])
    v = maxwell_velocities(n, temperature, mass, seed, fixed)
    L = ncell * a
    z_top = x[:, 2].max()
    box = orthorhombic_box(L, L, z_top + 2 * vacuum, (1, 1, 0), origin=(0.0, 0.0, -vacuum))
    center = (L / 2, L / 2, z_top)
    region = {"kind": "sphere", "center": center, "r_in": r_in, "r_sw": r_sw}
    ind = {"center": (L / 2, L / 2, z_top + R - penetration), "R": R, "K": K, "dir": (0.0, 0.0, -1.0)}
    return _bundle("W", x, v, box, fixed, region, ind, (0.0, 0.0, v_ms * MS_TO_AFS))


def cu_slab(nx=100, nz=50, a=3.615, temperature=300.0, seed=1003, r_hemi=82.6, r_sw=4.0,
            R=60.0, K=10.0, v_ms=25.0, penetration=1.0, n_fixed_layers=3, vacuum=10.0, sigma=0.0):
    """Cu FCC (001) indentation slab (the precision-sweep cell), same layout as w_slab; the
    ACE hemisphere's outer radius r_hemi (w > 0 inside it) holds 5 % of the atoms.  sigma > 0
    displaces the free atoms by N(0, sigma^2) per component (a thermal snapshot: 0.066 A is
    the 300 K amplitude of the synthetic Cu EAM's Einstein oscillator)."""
    x = fcc(a, nx, nx, nz)
    n = len(x)
    zs = np.unique(np.round(x[:, 2], 6))
    fixed = (x[:, 2] < zs[n_fixed_layers] - 1e-6).astype(np.uint8)
    if sigma > 0.0:
        x = x + random_displacements(n, sigma, seed + 100) * (1 - fixed)[:, None]
    mass = float(eam_potential("Cu")["mass_amu"])
    v = maxwell_velocities(n, temperature, mass, seed, fixed)
    L = nx * a
    z_top = x[:, 2].max()
    box = orthorhombic_box(L, L, z_top + 2 * vacuum, (1, 1, 0), origin=(0.0, 0.0, -vacuum))
    region = {"kind": "sphere", "center": (L / 2, L / 2, z_top), "r_in": r_hemi - r_sw, "r_sw": r_sw}
    ind = {"center": (L / 2, L / 2, z_top + R - penetration), "R": R, "K": K, "dir": (0.0, 0.0, -1.0)}
    return _bundle("Cu", x, v, box, fixed, region, ind, (0.0, 0.0, v_ms * MS_TO_AFS))


def strained_w_cell(ncell, seed, strain=0.02, vacancy=0.01, sigma=0.1, a=3.165):
    """Triclinic W cell: symmetric strain U(-strain, strain), vacancies, Gaussian noise."""
    rng = np.random.default_rng(seed)
    x = bcc(a, ncell, ncell, ncell)
    keep = rng.random(len(x)) >= vacancy
    if keep.sum() < 2:
        keep[:2] = True
    x = x[keep]
    e = rng.uniform(-strain, strain, size=(3, 3))
    e = 0.5 * (e + e.T)
    F = np.eye(3) + e
    x = x @ F.T + rng.normal(0.0, sigma, size=x.shape)
    h = (np.diag([ncell * a] * 3) @ F.T).ravel()
    box = {"h": h, "origin": np.zeros(3), "periodic": (1, 1, 1)}
    return _bundle("W", x, np.zeros_like(x), box, np.zeros(len(x), dtype=np.uint8), None, None, None)


# ---------------------------------------------------------------------------------------
# serving workload: independent structures of uneven size arriving as a Poisson stream
# ---------------------------------------------------------------------------------------
_SPEC = {"Cu": ("fcc", 3.615), "W": ("bcc", 3.165)}


def _cells_for(n_target, atoms_per_cell, aspect=(1, 1, 1)):
    k = max(1.0, (n_target / atoms_per_cell / (aspect[0] * aspect[1] * aspect[2])) ** (1.0 / 3.0))
    return [max(2, int(round(k * a))) for a in aspect]


def _oriented_110(species, nx, ny, nz):
    """Orthorhombic cell with x || [1-10], y || [001], z || [110] (periodic lengths exact)."""
    kind, a = _SPEC[species]
    lat = fcc if kind == "fcc" else bcc
    px = a / np.sqrt(2) if kind == "fcc" else a * np.sqrt(2)
    pz = a / np.sqrt(2) if kind == "fcc" else a * np.sqrt(2) / 2
    Lx, Ly, Lz = nx * px, ny * a, nz * pz
    m = int(np.ceil(max(Lx, Ly, Lz) / a)) + 2
    x = lat(a, 2 * m, 2 * m, 2 * m) - m * a
    ex = np.array([1.0, -1.0, 0.0]) / np.sqrt(2)
    ey = np.array([0.0, 0.0, 1.0])
    ez = np.array([1.0, 1.0, 0.0]) / np.sqrt(2)
    y = np.stack([x @ ex, x @ ey, x @ ez], axis=1)
    eps = 1e-6
    keep = (y[:, 0] >= -eps) & (y[:, 0] < Lx - eps) & (y[:, 1] >= -eps) & (y[:, 1] < Ly - eps) & \
           (y[:, 2] >= -eps) & (y[:, 2] < Lz - eps)
    return y[keep], (Lx, Ly, Lz)


GEOMETRIES = ("bulk", "vacancy", "surface001", "surface110", "indented")


def serving_request(rid, rng, species=None, geometry=None, n_target=None):
    """One request: structure, weight region, steps.  Sizes log-uniform 64..50,000 atoms,
    species Cu/W 50/50, geometry uniform over GEOMETRIES (any of the three may be fixed)."""
    sp = "Cu" if rng.random() < 0.5 else "W"
    species = sp if species is None else species
    kind, a = _SPEC[species]
    per_cell = 4 if kind == "fcc" else 2
    lat = fcc if kind == "fcc" else bcc
    nt = int(np.exp(rng.uniform(np.log(64), np.log(50000))))
    n_target = nt if n_target is None else n_target
    g = GEOMETRIES[rng.integers(5)]
    geom = g if geometry is None else geometry
    vac = 10.0
    if geom in ("bulk", "vacancy"):
        c = _cells_for(n_target, per_cell)
        x = lat(a, *c)
        L = np.array(c, dtype=float) * a
        box = orthorhombic_box(*L, (1, 1, 1))
        if geom == "vacancy":
            x = np.delete(x, rng.integers(len(x)), axis=0)
    elif geom == "surface110":
        px = a / np.sqrt(2) if kind == "fcc" else a * np.sqrt(2)
        pz = a / np.sqrt(2) if kind == "fcc" else a * np.sqrt(2) / 2
        k = max(2, int(round((n_target / (per_cell * (px / a) * (pz / a) * 2)) ** (1 / 3))))
        x, (Lx, Ly, Lz) = _oriented_110(species, k, k, 2 * k)
        box = orthorhombic_box(Lx, Ly, Lz + 2 * vac, (1, 1, 0), origin=(0.0, 0.0, -vac))
    else:
        c = _cells_for(n_target, per_cell, (1, 1, 1))
        x = lat(a, *c)
        L = np.array(c, dtype=float) * a
        box = orthorhombic_box(L[0], L[1], L[2] + 2 * vac, (1, 1, 0), origin=(0.0, 0.0, -vac))
        if geom == "indented":
            z_top = x[:, 2].max()
            tip = np.array([L[0] / 2, L[1] / 2, z_top + 0.6 * L[0]])
            x = x[np.linalg.norm(x - tip, axis=1) > 0.6 * L[0] + 0.5 * a]
    T = rng.uniform(0.0, 1000.0)
    mass = float(eam_potential(species)["mass_amu"])
    x = x + rng.normal(0.0, 0.1 * np.sqrt(T / 1000.0), size=x.shape)
    v = maxwell_velocities(len(x), T, mass, int(rng.integers(1 << 30)))
    h = np.asarray(box["h"]).reshape(3, 3)
    center = box["origin"] + 0.5 * np.diag(h)
    if box["periodic"][2] == 0:
        center[2] = x[:, 2].max()
    frac = rng.uniform(0.0, 1.0)
    r_in = frac ** (1.0 / 3.0) * 0.5 * float(np.linalg.norm(np.diag(h)[:2] if box["periodic"][2] == 0 else np.diag(h)))
    region = {"kind": "sphere", "center": tuple(center), "r_in": r_in, "r_sw": 2.0}
    req = _bundle(species, x, v, box, np.zeros(len(x), dtype=np.uint8), region, None, None)
    req.update({"id": rid, "geometry": geom, "temperature": T, "ace_fraction_target": frac,
                "n_steps": int(rng.integers(1, 101))})
    return req


def serving_requests(n, seed=1005, rate_per_s=50.0):
    """n requests with Poisson arrival times (seconds from 0) at rate_per_s."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    out = []
    for k in range(n):
        r = serving_request(k, rng)
        r["arrival_s"] = float(t[k])
        out.append(r)
    return out
