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
            R=60.0, K=10.0, v_ms=25.0, penetration=1.0, n_fixed_layers=3, vacuum=10.0):
    """Cu FCC (001) indentation slab (the precision-sweep cell), same layout as w_slab."""
    x = fcc(a, nx, nx, nz)
    n = len(x)
    zs = np.unique(np.round(x[:, 2], 6))
    fixed = (x[:, 2] < zs[n_fixed_layers] - 1e-6).astype(np.uint8)
    mass = float(eam_potential("Cu")["mass_amu"])
    v = maxwell_velocities(n, temperature, mass, seed, fixed)
    L = nx * a
    z_top = x[:, 2].max()
    box = orthorhombic_box(L, L, z_top + 2 * vacuum, (1, 1, 0), origin=(0.0, 0.0, -vacuum))
    region = {"kind": "sphere", "center": (L / 2, L / 2, z_top), "r_in": r_hemi, "r_sw": r_sw}
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
