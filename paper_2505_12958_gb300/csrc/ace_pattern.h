// ace_pattern.h -- compile-time structure of the synthetic ACE product basis.
//
// The product basis of Sec. 2.2.2 (Eq. energy_ace) is specialised here to n_max = 8
// radial functions and l_max = 4.  Three-factor functions couple (l1, l2, l3) with the
// real Gaunt coefficients G = integral(Y_l1m1 Y_l2m2 Y_l3m3).  For real harmonics
// (cos(m phi) for m > 0, sin(|m| phi) for m < 0) the phi integral vanishes unless an
// even number of the m are negative and the largest |m| equals the sum of the other
// two; that rule, evaluated at compile time, fixes which (m1, m2, m3) entries each
// l-triple carries, so the kernels can keep every operand in registers.  The values
// come from the host generator (Racah formula) in the same entry order.
#pragma once

namespace ap {

constexpr int kNmax = 8;                  // radial functions n = 0..7
constexpr int kLmax = 4;                  // l = 0..4
constexpr int kNLM = 25;                  // (l, m) pairs
constexpr int kApad = 36;                 // padded (l, m) stride per n: l-blocks of 4, 4, 8, 8, 12
constexpr int kNT = 14;                   // sorted l-triples with even sum and the triangle rule

__host__ __device__ constexpr int lblk(int l) { return l == 0 ? 0 : l == 1 ? 4 : l == 2 ? 8 : l == 3 ? 16 : 24; }

__host__ __device__ constexpr int tri_l(int t, int k) {
    // (0,0,0) (0,1,1) (0,2,2) (0,3,3) (0,4,4) (1,1,2) (1,2,3) (1,3,4)
    // (2,2,2) (2,2,4) (2,3,3) (2,4,4) (3,3,4) (4,4,4)
    constexpr int L[kNT][3] = {{0, 0, 0}, {0, 1, 1}, {0, 2, 2}, {0, 3, 3}, {0, 4, 4}, {1, 1, 2}, {1, 2, 3},
                               {1, 3, 4}, {2, 2, 2}, {2, 2, 4}, {2, 3, 3}, {2, 4, 4}, {3, 3, 4}, {4, 4, 4}};
    return L[t][k];
}

// The order in which the contraction kernel takes the factors of triple t: the real Gaunt
// coefficient is symmetric in its three (l, m) pairs, so a triple's function does not depend
// on the order of its factors.  The two triples with l1 < l2 = l3, (2, 3, 3) and (2, 4, 4), are
// taken as (3, 3, 2) and (4, 4, 2): their equal pair comes first, where the kernel packs the
// symmetric (n1, n2) pairs, and their third factor has 5 columns instead of 7 or 9.  The two
// with l1 = 1 < l2 < l3, (1, 2, 3) and (1, 3, 4), are taken as (2, 3, 1) and (3, 4, 1): their
// third factor has 3 columns instead of 7 or 9.
__host__ __device__ constexpr int kern_perm(int t, int k) {
    return (t == 6 || t == 7 || t == 10 || t == 11) ? (k + 1) % 3 : k;
}
__host__ __device__ constexpr int ktri_l(int t, int k) { return tri_l(t, kern_perm(t, k)); }

__host__ __device__ constexpr int iabs_c(int a) { return a < 0 ? -a : a; }

__host__ __device__ constexpr bool gaunt_allowed(int m1, int m2, int m3) {
    int neg = (m1 < 0) + (m2 < 0) + (m3 < 0);
    if (neg & 1) return false;
    int a = iabs_c(m1), b = iabs_c(m2), c = iabs_c(m3);
    int mx = a > b ? (a > c ? a : c) : (b > c ? b : c);
    return 2 * mx == a + b + c;
}

__host__ __device__ constexpr int pat_count(int l1, int l2, int l3) {
    int c = 0;
    for (int m1 = -l1; m1 <= l1; ++m1)
        for (int m2 = -l2; m2 <= l2; ++m2)
            for (int m3 = -l3; m3 <= l3; ++m3)
                if (gaunt_allowed(m1, m2, m3)) ++c;
    return c;
}

// which = 0, 1, 2: m1, m2, m3 of the e-th allowed entry (order m1, m2, m3 ascending)
__host__ __device__ constexpr int pat_entry(int l1, int l2, int l3, int e, int which) {
    int c = 0;
    for (int m1 = -l1; m1 <= l1; ++m1)
        for (int m2 = -l2; m2 <= l2; ++m2)
            for (int m3 = -l3; m3 <= l3; ++m3)
                if (gaunt_allowed(m1, m2, m3)) {
                    if (c == e) return which == 0 ? m1 : which == 1 ? m2 : m3;
                    ++c;
                }
    return 0;
}

// (the count does not depend on the order of the factors)
__host__ __device__ constexpr int tri_count(int t) { return pat_count(tri_l(t, 0), tri_l(t, 1), tri_l(t, 2)); }

__host__ __device__ constexpr int tri_offset(int t) {
    int o = 0;
    for (int k = 0; k < t; ++k) o += tri_count(k);
    return o;
}

constexpr int kNG = tri_offset(kNT);      // 418 entries (two of them are accidental zeros)

__host__ __device__ constexpr int tri_index(int l1, int l2, int l3) {
    for (int t = 0; t < kNT; ++t)
        if (tri_l(t, 0) == l1 && tri_l(t, 1) == l2 && tri_l(t, 2) == l3) return t;
    return -1;
}

}  // namespace ap
