"""Structure of the compiled ACE basis (mirrors csrc/ace_pattern.h): the 14 sorted
l-triples, the number of (m1, m2, m3) entries of each triple's real-Gaunt pattern
(an even number of negative m and the largest |m| equal to the sum of the other two), and
the order in which the contraction kernel takes each triple's factors."""


def _pattern_count(l1, l2, l3):
    c = 0
    for m1 in range(-l1, l1 + 1):
        for m2 in range(-l2, l2 + 1):
            for m3 in range(-l3, l3 + 1):
                neg = (m1 < 0) + (m2 < 0) + (m3 < 0)
                a = sorted((abs(m1), abs(m2), abs(m3)))
                if neg % 2 == 0 and a[2] == a[0] + a[1]:
                    c += 1
    return c


TRIPLES = [(0, 0, 0), (0, 1, 1), (0, 2, 2), (0, 3, 3), (0, 4, 4), (1, 1, 2), (1, 2, 3), (1, 3, 4),
           (2, 2, 2), (2, 2, 4), (2, 3, 3), (2, 4, 4), (3, 3, 4), (4, 4, 4)]
NNZ = [_pattern_count(*t) for t in TRIPLES]

# the contraction kernel's factor order: (1, 2, 3), (1, 3, 4), (2, 3, 3) and (2, 4, 4) as
# (2, 3, 1), (3, 4, 1), (3, 3, 2) and (4, 4, 2)
KERNEL_TRIPLES = [(t[1], t[2], t[0]) if k in (6, 7, 10, 11) else t for k, t in enumerate(TRIPLES)]
