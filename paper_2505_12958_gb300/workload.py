"""Work accounting for roofline figures (host-side bookkeeping, no physics).

ACE, per atom of the compacted list (Sec. 2.2.2, Eq. energy_ace): the arithmetic that the
factored evaluation cannot avoid.  FLOPs count an FMA as 2.  Only index combinations with a
structurally nonzero coefficient are counted: an l-triple with l1 = l2 has ordered first
factors (n1 <= n2), one with l2 = l3 ordered last factors (n2 <= n3), so each triple has
512, 288 or 120 (n1, n2, n3) combinations.  The real-Gaunt pattern of each triple has nnz
entries in g12 groups sharing (m1, m2), and the product of the two factors of a group is
formed once.

  per active (n1, n2) pair, forward:    P = sum G A A          g12 + 2 nnz
  per (n1, n2, n3) combination:         r = P . A_n3, phi1, phi2   2 W3 + 4
  adjoint, per combination:             c1 + s c2, Q = c . A_n3     2 + 2 W3
          per active (n1, n2) pair:     dA1, dA2               2 nnz + 3 g12
  adjoint, per combination:             c1 + s c2, T = c . A_n2     2 + 2 W2
          per active (n1, n3) pair:     dA3                    g12 + 2 nnz
  two-factor terms over the 36 pairs n1 <= n2 and each l: W_l FMA and two densities
  forward, W_l FMA plus one coefficient FMA and W_l multiplies adjoint; one-factor terms.
  per neighbour inside the cutoff: A = g Y (400), basis values (~100), pair force
  (25 x (32 + 10) + radial 40, ~1090).
"""
from .csrc_constants import KERNEL_TRIPLES, NNZ, TRIPLES

PER_NEIGHBOR_FLOPS = 400 + 100 + 25 * 42 + 40


def _pattern(l1, l2, l3):
    """(m1, m2, m3) entries of a triple's real-Gaunt pattern (an even number of negative m,
    the largest |m| the sum of the other two)."""
    out = []
    for m1 in range(-l1, l1 + 1):
        for m2 in range(-l2, l2 + 1):
            for m3 in range(-l3, l3 + 1):
                a = sorted((abs(m1), abs(m2), abs(m3)))
                if ((m1 < 0) + (m2 < 0) + (m3 < 0)) % 2 == 0 and a[2] == a[0] + a[1]:
                    out.append((m1, m2, m3))
    return out


def ace_contract_flops_per_atom():
    """FLOPs of the contraction per atom (products, densities, dE/dA; no neighbour terms)."""
    return ace_flops_per_atom(0)


def ace_flops_per_atom(n_neighbors):
    tot = 0
    for (l1, l2, l3), nnz in zip(TRIPLES, NNZ):
        pat = _pattern(l1, l2, l3)
        assert len(pat) == nnz
        g12 = len({(a, b) for a, b, _ in pat})
        w2, w3 = 2 * l2 + 1, 2 * l3 + 1
        combos = [(n1, n2, n3) for n1 in range(8) for n2 in range(8) for n3 in range(8)
                  if (l1 != l2 or n1 <= n2) and (l2 != l3 or n2 <= n3)]
        px = len({(a, b) for a, b, _ in combos})
        py = len({(a, c) for a, _, c in combos})
        t3 = len(combos)
        tot += px * (g12 + 2 * nnz) + t3 * (2 * w3 + 4)
        tot += t3 * (2 + 2 * w3) + px * (2 * nnz + 3 * g12)
        tot += t3 * (2 + 2 * w2) + py * (g12 + 2 * nnz)
    tot += 36 * sum(2 * (2 * l + 1) + 4 for l in range(5)) + 36 * sum(2 + 3 * (2 * l + 1) for l in range(5))
    tot += 8 * 4 + 8 * 2
    return tot + PER_NEIGHBOR_FLOPS * n_neighbors


def ace_tc_contract_work():
    """Work per compacted atom of the tensor-core contraction kernel (FMA = 2 FLOPs), counted
    over structurally nonzero index combinations as above:

      fp32:   the arithmetic left on the FP32 lanes, with each triple's factors in the
              kernel's order ((2, 3, 3) and (2, 4, 4) taken as (3, 3, 2) and (4, 4, 2)): the
              Gaunt products P of the nine triples
              with l1 > 0 (per active (n1, n2) pair g12 + 2 nnz; 36 pairs when l1 = l2, else
              64) and their factor gradients (per ordered pair: 2 nnz + 3 g12 for d1 and d2;
              for l1 = l2 only d1, 2 nnz + g12, taken twice; none for l1 = l2 = l3, whose
              gradient is three times the third-factor one from R); for the two-factor terms with
              the five (0, l, l) triples folded in, per l and nonzero pair (36): the folded
              coefficient, phi and the A[n1, 00] gradient of both densities (68), and the
              adjoint coefficient (2); the A[n1, 00] gradient's combination and warp sum; the
              epilogue per l3 (phi and the third-factor gradient); the one-factor terms.
      tensor: the coefficient contractions R = C^T P and Q = C [A; sA] over the active pairs
              (2 x 16 x pairs x W3 FLOPs each; no Q for l1 = l2 = l3), and the two-factor Gram products
              mm_l = A_l A_l^T (36 pairs x W_l) and their adjoint (CT + CT^T) A_l (64 x W_l).
      tensor_executed: what the mma.sync m16n8k8 tiles execute (2048 FLOPs each; 3xTF32 =
              three per product): R over 8 K steps (5 for the packed l1 = l2 triples) and Q
              over 4 row tiles (3 packed; none for l1 = l2 = l3), two column tiles where
              W3 = 9; per l one Gram and
              one adjoint tile (two K steps or two column tiles at l = 4)."""
    mma = 2 * 16 * 8 * 8
    fp32 = tensor = executed = 0
    for (l1, l2, l3), nnz in zip(KERNEL_TRIPLES, NNZ):
        if l1 == 0:
            continue
        g12 = len({(a, b) for a, b, _ in _pattern(l1, l2, l3)})
        w3 = 2 * l3 + 1
        sym = l1 == l2
        sym3 = sym and l2 == l3                                  # the gradient is 3 x the third-factor one
        pairs = 36 if sym else 64
        nt = (w3 + 7) // 8
        fp32 += pairs * (g12 + 2 * nnz)
        if not sym3:
            fp32 += 64 * (2 * nnz + g12) if sym else 64 * (2 * nnz + 3 * g12)
        tensor += (1 if sym3 else 2) * (2 * 16 * pairs * w3)
        executed += 3 * mma * nt * (5 if sym else 8)            # R: K steps x column tiles
        if not sym3:
            executed += 3 * mma * nt * 2 * (3 if sym else 4)    # Q: row tiles x 2 densities
    for l in range(5):
        w = 2 * l + 1
        fp32 += 36 * (68 + 2)
        tensor += 2 * 36 * w + 2 * 64 * w
        executed += 2 * 3 * mma * (2 if l == 4 else 1)
    fp32 += 32 * 2 * 8 + 2 * 8 * 31
    fp32 += 2 * 2 * 8 * sum(2 * l + 1 for l in (2, 3, 4)) + 2 * 8 * sum(2 * l + 1 for l in (2, 3, 4))
    fp32 += 8 * 4 + 8 * 2
    return {"fp32": fp32, "tensor": tensor, "tensor_executed": executed}


def eam_bytes_per_atom(n_list):
    """Minimum HBM bytes of the two EAM passes per atom with a materialised list:
    list entries read twice (4 B each), own position/weight 16 B twice, forces 12 B,
    energies 16 B, u xi' 4 B written and read, virial 24 B."""
    return 2 * 4 * n_list + 2 * 16 + 12 + 16 + 8 + 24
