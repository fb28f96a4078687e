"""The work count behind the contraction's roofline figure: its index combinations must be
exactly the three-factor basis functions of the synthetic ACE, and its pattern sizes the
real-Gaunt entries of each l-triple."""
import numpy as np

import synth
from paper_2505_12958_gb300 import workload
from paper_2505_12958_gb300.csrc_constants import KERNEL_TRIPLES, NNZ, TRIPLES


def test_counted_combinations_are_the_three_factor_functions():
    idx = synth.ace_basis()
    nu3 = idx[idx[:, 0] == 3]
    # (l, n) sorted triples of the basis, grouped by l-triple
    per_triple = {}
    for row in nu3:
        key = tuple(sorted([(row[2], row[1]), (row[4], row[3]), (row[6], row[5])]))
        per_triple.setdefault(tuple(k[0] for k in key), set()).add(key)
    for (l1, l2, l3) in TRIPLES:
        combos = [(n1, n2, n3) for n1 in range(8) for n2 in range(8) for n3 in range(8)
                  if (l1 != l2 or n1 <= n2) and (l2 != l3 or n2 <= n3)]
        assert len(combos) == len(per_triple[(l1, l2, l3)])
    assert sum(len(v) for v in per_triple.values()) == len(nu3) == 3976


def test_pattern_sizes_and_total():
    for (l1, l2, l3), nnz in zip(TRIPLES, NNZ):
        assert len(workload._pattern(l1, l2, l3)) == nnz
    assert sum(NNZ) == 418
    f = workload.ace_contract_flops_per_atom()
    assert f == 403704
    assert workload.ace_flops_per_atom(10) == f + 10 * workload.PER_NEIGHBOR_FLOPS


def test_tensor_core_kernel_work_split():
    """The tensor-core kernel's work: the coefficient contractions over the active (n1, n2)
    pairs of the nine triples with l1 > 0 (36 pairs when l1 = l2, in the kernel's factor
    order), the two-factor Gram products and their adjoint, and the 3xTF32 m16n8k8 tiles that
    run them (the packed l1 = l2 triples: 5 K steps of R and 3 row tiles of Q)."""
    # the kernel's order permutes the factors of four triples only
    for t, k in zip(TRIPLES, KERNEL_TRIPLES):
        assert sorted(t) == sorted(k)
    assert [k for t, k in zip(TRIPLES, KERNEL_TRIPLES) if t != k] == [(2, 3, 1), (3, 4, 1), (3, 3, 2), (4, 4, 2)]
    w = workload.ace_tc_contract_work()
    tc = [(t, 36 if t[0] == t[1] else 64) for t in KERNEL_TRIPLES if min(t) > 0]
    assert len(tc) == 9 and sum(1 for t, p in tc if p == 36) == 7
    gram = sum(2 * 36 * (2 * l + 1) + 2 * 64 * (2 * l + 1) for l in range(5))
    # (2, 2, 2) and (4, 4, 4): R only (their gradient is three times the third-factor one)
    sym3 = [t for t, _ in tc if t[0] == t[1] == t[2]]
    assert sym3 == [(2, 2, 2), (4, 4, 4)]
    assert w["tensor"] == sum((1 if t in sym3 else 2) * 2 * 16 * p * (2 * t[2] + 1) for t, p in tc) + gram
    tile = 2 * 16 * 8 * 8
    r_tiles = sum((5 if t[0] == t[1] else 8) * (2 if t[2] == 4 else 1) for t, _ in tc)
    q_tiles = sum(2 * (3 if t[0] == t[1] else 4) * (2 if t[2] == 4 else 1) for t, _ in tc if t not in sym3)
    assert w["tensor_executed"] == 3 * tile * (r_tiles + q_tiles + 2 * 6)
    assert w == {"fp32": 115572, "tensor": 121736, "tensor_executed": 835584}
