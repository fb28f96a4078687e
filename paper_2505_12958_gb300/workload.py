"""Work accounting for roofline figures (host-side bookkeeping, no physics).

ACE, per atom of the compacted list (Sec. 2.2.2, Eq. energy_ace), for the factored
evaluation the kernel uses.  FLOPs count an FMA as 2.  Only (n, n') pairs that carry a
structurally nonzero coefficient are counted: for an l-triple with l1 = l2 the first two
factors are ordered (n1 <= n2), for l2 = l3 the last two (n2 <= n3).

  per l-triple t and active (n1, n2) pair, forward:   P = sum G A A      3 nnz_t
                                                      R = P . A_n3       16 W3
                                                      phi1, phi2         32
  adjoint, (n1, n2) mapping:                          c1 + s c2          16
                                                      Q = c . A_n3       16 W3
                                                      dA1, dA2           5 nnz_t
  adjoint, (n1, n3) mapping:                          c1 + s c2          16
                                                      T = c . A_n2       16 W2
                                                      dA3                3 nnz_t
  two-factor terms: 64 pairs x 25 x 2 (forward) + 64 x 25 x 4 (adjoint) + 64 x 5 x 8
  per neighbour inside the cutoff: A = g Y (400), basis values (~100), pair force
  (25 x (32 + 10) + radial 40, ~1090).
"""
from .csrc_constants import NNZ, TRIPLES

PER_NEIGHBOR_FLOPS = 400 + 100 + 25 * 42 + 40


def _active_pairs(l1, l2, l3):
    x = 36 if l1 == l2 else 64
    if l1 == l2 and l2 == l3:
        y = 36
    else:
        y = 64
    return x, y


def ace_contract_flops_per_atom():
    """FLOPs of the contraction kernel per atom (products, densities, dE/dA; no neighbour terms)."""
    return ace_flops_per_atom(0)


def ace_flops_per_atom(n_neighbors):
    tot = 0
    for (l1, l2, l3), nnz in zip(TRIPLES, NNZ):
        w2, w3 = 2 * l2 + 1, 2 * l3 + 1
        px, py = _active_pairs(l1, l2, l3)
        tot += px * (3 * nnz + 16 * w3 + 32)
        tot += px * (16 + 16 * w3 + 5 * nnz)
        tot += py * (16 + 16 * w2 + 3 * nnz)
    tot += 64 * 25 * 2 + 64 * 25 * 4 + 64 * 5 * 8
    return tot + PER_NEIGHBOR_FLOPS * n_neighbors


def eam_bytes_per_atom(n_list):
    """Minimum HBM bytes of the two EAM passes per atom with a materialised list:
    list entries read twice (4 B each), own position/weight 16 B twice, forces 12 B,
    energies 16 B, u xi' 4 B written and read, virial 24 B."""
    return 2 * 4 * n_list + 2 * 16 + 12 + 16 + 8 + 24
