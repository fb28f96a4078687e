"""Lattices, boxes, displacements and velocities (seeded)."""
import numpy as np

KB_EV = 8.617333262e-5          # Boltzmann constant, eV/K
FTM = 0.0096485332              # 1 eV/(Angstrom amu) in Angstrom/fs^2

_FCC = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
_BCC = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])


def _lattice(basis, a, nx, ny, nz):
    # z slowest so that atomic layers are contiguous in index order
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    return pos


def fcc(a, nx, ny, nz):
    return _lattice(_FCC, a, nx, ny, nz)


def bcc(a, nx, ny, nz):
    return _lattice(_BCC, a, nx, ny, nz)


def orthorhombic_box(lx, ly, lz, periodic=(1, 1, 1), origin=(0.0, 0.0, 0.0)):
    return {"h": np.diag([lx, ly, lz]).astype(np.float64).ravel(),
            "origin": np.asarray(origin, dtype=np.float64),
            "periodic": tuple(int(p) for p in periodic)}


def random_displacements(n, sigma, seed):
    return np.random.default_rng(seed).normal(0.0, sigma, size=(n, 3))


def maxwell_velocities(n, temperature, mass, seed, fixed=None):
    """Velocities in Angstrom/fs with the centre-of-mass momentum of free atoms removed."""
    rng = np.random.default_rng(seed)
    s = np.sqrt(KB_EV * temperature * FTM / mass)
    v = rng.normal(0.0, s, size=(n, 3))
    free = np.ones(n, dtype=bool) if fixed is None else ~np.asarray(fixed, dtype=bool)
    if free.any():
        v[free] -= v[free].mean(axis=0)
    v[~free] = 0.0
    return v
