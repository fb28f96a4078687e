"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds no arithmetic of the method: it builds lattices, random
displacements, velocities, box and region descriptions, and it loads or draws the
potential parameters (the paper's printed W EAM table, the stated synthetic Cu EAM,
and the synthetic ACE basis list with seeded N(0, 0.1^2) coefficients).  Both the
oracle and the GPU library receive these as plain arrays.
"""
from .potentials import ace_basis, ace_potential, eam_potential  # noqa: F401
from .lattice import (  # noqa: F401
    bcc, fcc, maxwell_velocities, orthorhombic_box, random_displacements,
)
from . import configs  # noqa: F401,E402
