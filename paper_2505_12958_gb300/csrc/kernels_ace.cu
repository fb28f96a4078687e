// kernels_ace.cu -- ACE pass of the AP force evaluation (Sec. 2.2.2, Eq. energy_ace).
//
// Three kernels per step, one warp per atom of the compacted list (w_i > 0), persistent grids:
//   k_ace_basis<MODE>  neighbours within the ACE cutoff are gathered from the full list
//                      (r_ij from FP32 cell-relative positions); g_n(r_ij), Y_lm(rhat_ij) and
//                      A_nlm = (1/nref) sum_j g_n Y_lm (8 x 25) in the precision MODE
//                      (FP32 FMA, 3xTF32 / BF16 / FP16 mma.sync, or FP64 accumulation);
//                      A is written [atom][lm][n].
//   k_ace_contract     phi_p = c_p0 + sum_v c_p[v] B_v, p = 1, 2 (B: one, two and three A
//                      factors) and the adjoint dE/dA with the combined coefficients
//                      c1 + c2 / (2 sqrt(phi2)): the Gaunt products of the first two factors
//                      on FP32 lanes (one (n1, n2) pair per lane, compile-time coupling
//                      pattern), their contractions with the coefficient matrices on tensor
//                      cores (mma.sync, 3xTF32; the l1 = l2 triples over the 36 pairs
//                      n1 <= n2), and the one- and two-factor functions through tensor-core
//                      Gram tiles A_l A_l^T and their adjoint.  Writes dE/dA and E_i^ACE.
//   k_ace_force        f_ij = dE_i/dr_ij = (1/nref) sum dE/dA_nlm grad(g_n Y_lm), weighted by
//                      w_i, added to atom j (minus) and atom i (plus) through 64-bit fixed-point
//                      atomics (2^-40 eV/A resolution), whose integer sums do not depend on order.
// E_i^ACE is stored without the constant c1_0, which the blend adds in FP64.  The allocation-
// free entry point at the end of the file runs the same per-atom device functions (neighbour
// tiles, the contraction, the pair forces) in one kernel.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "ap_internal.h"

namespace ap {

__constant__ float c_gaunt[kNG];

void upload_gaunt(const float* g) { cudaMemcpyToSymbol(c_gaunt, g, sizeof(float) * kNG); }

namespace {

constexpr int kTile = 32;                      // neighbours per basis tile (one per lane)

// ---------------------------------------------------------------------------------
// radial basis g_n = T_n(2r/rc - 1) fc(r), fc = (1 + cos(pi r/rc))/2, and dg_n/dr
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void radial(float r, float rc, float* g, float* dg) {
    const float x = 2.0f * r / rc - 1.0f, dx = 2.0f / rc;
    float sn, cs;
    sincospif(r / rc, &sn, &cs);
    const float fc = 0.5f * (1.0f + cs), dfc = -0.5f * 3.14159265358979f / rc * sn;
    float T0 = 1.0f, T1 = x, D0 = 0.0f, D1 = 1.0f;
    g[0] = fc; dg[0] = dfc;
    g[1] = x * fc; dg[1] = dx * fc + x * dfc;
#pragma unroll
    for (int n = 2; n < kNmax; ++n) {
        float T2 = 2.0f * x * T1 - T0;
        float D2 = 2.0f * T1 + 2.0f * x * D1 - D0;
        g[n] = T2 * fc;
        dg[n] = D2 * dx * fc + T2 * dfc;
        T0 = T1; T1 = T2; D0 = D1; D1 = D2;
    }
}

// ---------------------------------------------------------------------------------
// real orthonormal spherical harmonics as homogeneous Cartesian polynomials S_lm
// evaluated at the unit vector (x, y, z); index l*l + l + m
// ---------------------------------------------------------------------------------
#define YC0 0.28209479177387814f
#define YC1 0.4886025119029199f
#define YC2A 1.0925484305920792f
#define YC2B 0.31539156525252005f
#define YC2C 0.5462742152960396f
#define YC3A 0.5900435899266435f
#define YC3B 2.890611442640554f
#define YC3C 0.45704579946446574f
#define YC3D 0.3731763325901154f
#define YC3E 1.445305721320277f
#define YC4A 2.5033429417967046f
#define YC4B 1.7701307697799304f
#define YC4C 0.9461746957575601f
#define YC4D 0.6690465435572892f
#define YC4E 0.10578554691520431f
#define YC4F 0.47308734787878004f
#define YC4G 0.6258357354491761f

__device__ __forceinline__ void ylm(float x, float y, float z, float* Y) {
    const float x2 = x * x, y2 = y * y, z2 = z * z, r2 = x2 + y2 + z2;
    Y[0] = YC0;
    Y[1] = YC1 * y; Y[2] = YC1 * z; Y[3] = YC1 * x;
    Y[4] = YC2A * x * y; Y[5] = YC2A * y * z; Y[6] = YC2B * (2.0f * z2 - x2 - y2); Y[7] = YC2A * x * z;
    Y[8] = YC2C * (x2 - y2);
    Y[9] = YC3A * y * (3.0f * x2 - y2); Y[10] = YC3B * x * y * z; Y[11] = YC3C * y * (4.0f * z2 - x2 - y2);
    Y[12] = YC3D * z * (2.0f * z2 - 3.0f * x2 - 3.0f * y2); Y[13] = YC3C * x * (4.0f * z2 - x2 - y2);
    Y[14] = YC3E * z * (x2 - y2); Y[15] = YC3A * x * (x2 - 3.0f * y2);
    Y[16] = YC4A * x * y * (x2 - y2); Y[17] = YC4B * y * z * (3.0f * x2 - y2);
    Y[18] = YC4C * x * y * (6.0f * z2 - x2 - y2); Y[19] = YC4D * y * z * (4.0f * z2 - 3.0f * x2 - 3.0f * y2);
    Y[20] = YC4E * (35.0f * z2 * z2 - 30.0f * z2 * r2 + 3.0f * r2 * r2);
    Y[21] = YC4D * x * z * (4.0f * z2 - 3.0f * x2 - 3.0f * y2); Y[22] = YC4F * (x2 - y2) * (6.0f * z2 - x2 - y2);
    Y[23] = YC4B * x * z * (x2 - 3.0f * y2); Y[24] = YC4G * (x2 * x2 - 6.0f * x2 * y2 + y2 * y2);
}

// f += a * grad S_lm (Cartesian gradient of the homogeneous polynomial) for all lm,
// s += (b - l a / r) S_lm, with a_lm, b_lm supplied by the functor.
template <class AB>
__device__ __forceinline__ void force_terms(float x, float y, float z, float rinv, AB ab, float& s, float& gx, float& gy,
                                            float& gz) {
    const float x2 = x * x, y2 = y * y, z2 = z * z, r2 = x2 + y2 + z2;
    float a, b;
#define TERM(LM, L, SV, GX, GY, GZ)            \
    ab(LM, a, b);                              \
    s = fmaf(b - (float)(L) * a * rinv, (SV), s); \
    gx = fmaf(a, (GX), gx);                    \
    gy = fmaf(a, (GY), gy);                    \
    gz = fmaf(a, (GZ), gz);
    TERM(0, 0, YC0, 0.f, 0.f, 0.f)
    TERM(1, 1, YC1 * y, 0.f, YC1, 0.f)
    TERM(2, 1, YC1 * z, 0.f, 0.f, YC1)
    TERM(3, 1, YC1 * x, YC1, 0.f, 0.f)
    TERM(4, 2, YC2A * x * y, YC2A * y, YC2A * x, 0.f)
    TERM(5, 2, YC2A * y * z, 0.f, YC2A * z, YC2A * y)
    TERM(6, 2, YC2B * (2.0f * z2 - x2 - y2), -2.0f * YC2B * x, -2.0f * YC2B * y, 4.0f * YC2B * z)
    TERM(7, 2, YC2A * x * z, YC2A * z, 0.f, YC2A * x)
    TERM(8, 2, YC2C * (x2 - y2), 2.0f * YC2C * x, -2.0f * YC2C * y, 0.f)
    TERM(9, 3, YC3A * y * (3.0f * x2 - y2), 6.0f * YC3A * x * y, 3.0f * YC3A * (x2 - y2), 0.f)
    TERM(10, 3, YC3B * x * y * z, YC3B * y * z, YC3B * x * z, YC3B * x * y)
    TERM(11, 3, YC3C * y * (4.0f * z2 - x2 - y2), -2.0f * YC3C * x * y, YC3C * (4.0f * z2 - x2 - 3.0f * y2),
         8.0f * YC3C * y * z)
    TERM(12, 3, YC3D * z * (2.0f * z2 - 3.0f * x2 - 3.0f * y2), -6.0f * YC3D * x * z, -6.0f * YC3D * y * z,
         YC3D * (6.0f * z2 - 3.0f * x2 - 3.0f * y2))
    TERM(13, 3, YC3C * x * (4.0f * z2 - x2 - y2), YC3C * (4.0f * z2 - 3.0f * x2 - y2), -2.0f * YC3C * x * y,
         8.0f * YC3C * x * z)
    TERM(14, 3, YC3E * z * (x2 - y2), 2.0f * YC3E * x * z, -2.0f * YC3E * y * z, YC3E * (x2 - y2))
    TERM(15, 3, YC3A * x * (x2 - 3.0f * y2), 3.0f * YC3A * (x2 - y2), -6.0f * YC3A * x * y, 0.f)
    TERM(16, 4, YC4A * x * y * (x2 - y2), YC4A * y * (3.0f * x2 - y2), YC4A * x * (x2 - 3.0f * y2), 0.f)
    TERM(17, 4, YC4B * y * z * (3.0f * x2 - y2), 6.0f * YC4B * x * y * z, 3.0f * YC4B * z * (x2 - y2),
         YC4B * y * (3.0f * x2 - y2))
    TERM(18, 4, YC4C * x * y * (6.0f * z2 - x2 - y2), YC4C * y * (6.0f * z2 - 3.0f * x2 - y2),
         YC4C * x * (6.0f * z2 - x2 - 3.0f * y2), 12.0f * YC4C * x * y * z)
    TERM(19, 4, YC4D * y * z * (4.0f * z2 - 3.0f * x2 - 3.0f * y2), -6.0f * YC4D * x * y * z,
         YC4D * z * (4.0f * z2 - 3.0f * x2 - 9.0f * y2), YC4D * y * (12.0f * z2 - 3.0f * x2 - 3.0f * y2))
    TERM(20, 4, YC4E * (35.0f * z2 * z2 - 30.0f * z2 * r2 + 3.0f * r2 * r2), 12.0f * YC4E * x * (r2 - 5.0f * z2),
         12.0f * YC4E * y * (r2 - 5.0f * z2), 16.0f * YC4E * z * (5.0f * z2 - 3.0f * r2))
    TERM(21, 4, YC4D * x * z * (4.0f * z2 - 3.0f * x2 - 3.0f * y2), YC4D * z * (4.0f * z2 - 9.0f * x2 - 3.0f * y2),
         -6.0f * YC4D * x * y * z, YC4D * x * (12.0f * z2 - 3.0f * x2 - 3.0f * y2))
    TERM(22, 4, YC4F * (x2 - y2) * (6.0f * z2 - x2 - y2), YC4F * x * (12.0f * z2 - 4.0f * x2),
         YC4F * y * (4.0f * y2 - 12.0f * z2), 12.0f * YC4F * z * (x2 - y2))
    TERM(23, 4, YC4B * x * z * (x2 - 3.0f * y2), 3.0f * YC4B * z * (x2 - y2), -6.0f * YC4B * x * y * z,
         YC4B * x * (x2 - 3.0f * y2))
    TERM(24, 4, YC4G * (x2 * x2 - 6.0f * x2 * y2 + y2 * y2), 4.0f * YC4G * x * (x2 - 3.0f * y2),
         4.0f * YC4G * y * (y2 - 3.0f * x2), 0.f)
#undef TERM
}

// ---------------------------------------------------------------------------------
// three-factor products, one l-triple at a time, operands in registers
// ---------------------------------------------------------------------------------
template <int T>
struct Tri {
    static constexpr int L1 = ktri_l(T, 0), L2 = ktri_l(T, 1), L3 = ktri_l(T, 2);   // kernel order
    static constexpr int W1 = 2 * L1 + 1, W2 = 2 * L2 + 1, W3 = 2 * L3 + 1;
    static constexpr int N = tri_count(T), OFF = tri_offset(T);
    static constexpr int B1 = lblk(L1), B2 = lblk(L2), B3 = lblk(L3);
    template <int E> static constexpr int m1() { return pat_entry(L1, L2, L3, E, 0) + L1; }
    template <int E> static constexpr int m2() { return pat_entry(L1, L2, L3, E, 1) + L2; }
    template <int E> static constexpr int m3() { return pat_entry(L1, L2, L3, E, 2) + L3; }
    // the entries are ordered by (m1, m2, m3), so those sharing (m1, m2) are consecutive
    template <int E> static constexpr bool first12() {
        return E == 0 || pat_entry(L1, L2, L3, E, 0) != pat_entry(L1, L2, L3, E - 1, 0) ||
               pat_entry(L1, L2, L3, E, 1) != pat_entry(L1, L2, L3, E - 1, 1);
    }
    template <int E> static constexpr bool last12() {
        return E == N - 1 || pat_entry(L1, L2, L3, E, 0) != pat_entry(L1, L2, L3, E + 1, 0) ||
               pat_entry(L1, L2, L3, E, 1) != pat_entry(L1, L2, L3, E + 1, 1);
    }
};

// Entries sharing (m1, m2) share the product of their two factors:
//   P[m3]  += G A1[m1] A2[m2]          t = A1[m1] A2[m2] once per (m1, m2)
//   d1[m1] += G Q[m3] A2[m2], d2[m2] += G Q[m3] A1[m1]
//                                       u = sum G Q[m3] over the (m1, m2) group
//   d3[m3] += G A1[m1] Tm[m2]          t = A1[m1] Tm[m2] once per (m1, m2)
template <int T, int E>
__device__ __forceinline__ void ent_p(float* P, const float* A1, const float* A2, float& t) {
    using R = Tri<T>;
    constexpr int i1 = R::template m1<E>(), i2 = R::template m2<E>(), i3 = R::template m3<E>();
    if constexpr (R::template first12<E>()) t = A1[i1] * A2[i2];
    P[i3] = fmaf(c_gaunt[R::OFF + E], t, P[i3]);
}
template <int T, int... E>
__device__ __forceinline__ void all_p(float* P, const float* A1, const float* A2, std::integer_sequence<int, E...>) {
    float t = 0.0f;
    (ent_p<T, E>(P, A1, A2, t), ...);
}

// with D2 false only the first-factor gradient d1 (the l1 = l2 triples, whose second-factor
// gradient summed over pairs equals the first-factor one)
template <int T, bool D2, int E>
__device__ __forceinline__ void ent_x(float* d1, float* d2, const float* A1, const float* A2, const float* Q,
                                      float& u) {
    using R = Tri<T>;
    constexpr int i1 = R::template m1<E>(), i2 = R::template m2<E>(), i3 = R::template m3<E>();
    if constexpr (R::template first12<E>()) u = c_gaunt[R::OFF + E] * Q[i3];
    else u = fmaf(c_gaunt[R::OFF + E], Q[i3], u);
    if constexpr (R::template last12<E>()) {
        d1[i1] = fmaf(u, A2[i2], d1[i1]);
        if constexpr (D2) d2[i2] = fmaf(u, A1[i1], d2[i2]);
    }
}
template <int T, bool D2, int... E>
__device__ __forceinline__ void all_x(float* d1, float* d2, const float* A1, const float* A2, const float* Q,
                                      std::integer_sequence<int, E...>) {
    float u = 0.0f;
    (ent_x<T, D2, E>(d1, d2, A1, A2, Q, u), ...);
}

template <int W>
__device__ __forceinline__ void load_row(float* dst, const float* src) {
#pragma unroll
    for (int k = 0; k < W; k += 4) {
        const float4 v = *reinterpret_cast<const float4*>(src + k);
        dst[k] = v.x;
        if (k + 1 < W) dst[k + 1] = v.y;
        if (k + 2 < W) dst[k + 2] = v.z;
        if (k + 3 < W) dst[k + 3] = v.w;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void fix_add(unsigned long long* p, float v) {
    long long q = __float2ll_rn(v * 1099511627776.0f);
    atomicAdd(p, (unsigned long long)q);
}

// neighbours of atom i inside the ACE cutoff, from the full list, into S (warp-uniform count;
// returns -1 when there are more than kAceNbrCap).  The list is read from its row-major copy
// nrow[i cap + k] (the same entries in the same order as the column-major list of the
// thread-per-atom kernels): the lanes of a round read one row, a few cache lines, instead of
// 32 rows of the column-major list.
// U rounds of 32 list entries at a time: all their list loads, then all their position
// gathers, then the compaction in list order (two dependent memory round trips per 32 U
// entries); the neighbour order does not depend on U
template <int U>
__device__ __forceinline__ int gather_ace_neighbors(const float4* __restrict__ pos4, const int* __restrict__ nrow,
                                                    int cap, int i, int m, const float4* Ds, float rc2, float4* nb,
                                                    int* nbj, int lane) {
    const float4 p = pos4[i];
    int cnt = 0;
    for (int k0 = 0; k0 < m; k0 += 32 * U) {
        int e[U];                                      // j | code << 25 (the code may set bit 31)
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + 32 * u + lane;
            e[u] = k < m ? nrow[(size_t)i * cap + k] : 0;
        }
        float4 q[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            q[u] = k0 + 32 * u + lane < m ? pos4[e[u] & kNbrMask] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            bool in = false;
            float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
            if (k0 + 32 * u + lane < m) {
                const float4 d = Ds[(unsigned)e[u] >> kNbrShift];
                dx = q[u].x + d.x - p.x; dy = q[u].y + d.y - p.y; dz = q[u].z + d.z - p.z;
                r2 = dx * dx + dy * dy + dz * dz;
                in = r2 < rc2 && r2 > 0.0f;
            }
            const unsigned bm = __ballot_sync(0xffffffffu, in);
            const int pos = cnt + __popc(bm & ((1u << lane) - 1u));
            if (in && pos < kAceNbrCap) { nb[pos] = make_float4(dx, dy, dz, sqrtf(r2)); nbj[pos] = e[u] & kNbrMask; }
            cnt += __popc(bm);
        }
    }
    __syncwarp();
    return cnt > kAceNbrCap ? -1 : cnt;
}

// list rounds of 32 entries whose loads and gathers the basis kernel issues together, and
// its minimum resident blocks per SM (tuning constants; results do not depend on them)
#ifndef AP_BASIS_ROUNDS
#define AP_BASIS_ROUNDS 2
#endif
#ifndef AP_BASIS_MINB
#define AP_BASIS_MINB 1
#endif
constexpr int kBasisRounds = AP_BASIS_ROUNDS;

struct BasisSmem {
    float4 nb[kAceNbrCap];
    int nbj[kAceNbrCap];
    float tileY[kTile][kNLM];
    float tileG[kTile][kNmax];
};

// ---------------------------------------------------------------------------------
// A = Y^T g on tensor cores (mma.sync; M = (l, m) padded to 32, N = n = 8, K = neighbours).
// Fragment layouts of the PTX m16n8k8 (tf32) and m16n8k16 (bf16 / f16) shapes, with
// g = lane / 4 and t = lane % 4.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int MODE>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    if (MODE == AP_ACE_TC_BF16) {
        __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&v);
    } else {
        __half2 v = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&v);
    }
}

template <int MODE>
__device__ __forceinline__ void mma_16bit(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                          uint32_t b1) {
    if (MODE == AP_ACE_TC_BF16)
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                     : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                     : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    else
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                     : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                     : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// element (row lm, column j) of the A operand Y^T; rows 25..31 are padding
__device__ __forceinline__ float yt(const BasisSmem& S, int lm, int j) { return lm < kNLM ? S.tileY[j][lm] : 0.0f; }

// g_n and Y_lm of the neighbours t0 .. t0 + 31 of the list nb (zeros beyond cnt), one per
// lane, into the tile rows
__device__ __forceinline__ void basis_tile(const float4* nb, int t0, int cnt, float rc, float (*tileY)[kNLM],
                                           float (*tileG)[kNmax], int lane) {
    const int jj = t0 + lane;
    float g[kNmax], dg[kNmax], Y[kNLM];
    if (jj < cnt) {
        const float4 v = nb[jj];
        const float ri = 1.0f / v.w;
        radial(v.w, rc, g, dg);
        ylm(v.x * ri, v.y * ri, v.z * ri, Y);
    } else {
#pragma unroll
        for (int q = 0; q < kNmax; ++q) g[q] = 0.0f;
#pragma unroll
        for (int q = 0; q < kNLM; ++q) Y[q] = 0.0f;
    }
#pragma unroll
    for (int q = 0; q < kNmax; ++q) tileG[lane][q] = g[q];
#pragma unroll
    for (int q = 0; q < kNLM; ++q) tileY[lane][q] = Y[q];
}

// accA[n] += sum_j Y_lm(j) g_n(j) over the first nt tile rows, lane = lm < 25 (FP32 FMA)
__device__ __forceinline__ void basis_accum_fp32(const float (*tileY)[kNLM], const float (*tileG)[kNmax], int nt,
                                                 int lane, float* accA) {
    if (lane >= kNLM) return;
    for (int jj2 = 0; jj2 < nt; ++jj2) {
        const float y = tileY[jj2][lane];
        const float4 g0 = *reinterpret_cast<const float4*>(&tileG[jj2][0]);
        const float4 g1 = *reinterpret_cast<const float4*>(&tileG[jj2][4]);
        const float gg[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
        for (int q = 0; q < kNmax; ++q) accA[q] = fmaf(y, gg[q], accA[q]);
    }
}

// w_i f_ij with f_ij = dE_i/dr_ij = (1/nref) sum_nlm dE/dA_nlm grad(g_n Y_lm) for the pair
// vector v = (r_ij, |r_ij|); dAT[lm][n] is dE/dA of atom i
__device__ __forceinline__ float3 ace_pair_force(float4 v, float rc, float nrefi, float wi,
                                                 const float (*dAT)[kNmax]) {
    const float ri = 1.0f / v.w;
    const float ux = v.x * ri, uy = v.y * ri, uz = v.z * ri;
    float g[kNmax], dg[kNmax];
    radial(v.w, rc, g, dg);
    float sc = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    auto ab = [&](int lm, float& aa, float& bb) {
        const float4 d0 = *reinterpret_cast<const float4*>(&dAT[lm][0]);
        const float4 d1 = *reinterpret_cast<const float4*>(&dAT[lm][4]);
        aa = d0.x * g[0] + d0.y * g[1] + d0.z * g[2] + d0.w * g[3] + d1.x * g[4] + d1.y * g[5] + d1.z * g[6] + d1.w * g[7];
        bb = d0.x * dg[0] + d0.y * dg[1] + d0.z * dg[2] + d0.w * dg[3] + d1.x * dg[4] + d1.y * dg[5] + d1.z * dg[6] + d1.w * dg[7];
    };
    force_terms(ux, uy, uz, ri, ab, sc, gx, gy, gz);
    return make_float3(nrefi * (sc * ux + gx * ri) * wi, nrefi * (sc * uy + gy * ri) * wi,
                       nrefi * (sc * uz + gz * ri) * wi);
}

// stage a1 of the ACE pass: A_nlm = (1/nref) sum_j g_n(r_ij) Y_lm(rhat_ij), stored [atom][lm][n].
// MODE (AP_ACE_*) sets the precision of the contraction over neighbours: FP32 FMA, tensor
// cores (3xTF32 split, BF16 or FP16 inputs; FP32 accumulation), or FP64 accumulation.
// the A_nlm of compacted atom a (stage a1), one warp; neighbour offsets Ds staged by the caller
template <int MODE>
__device__ __forceinline__ void basis_atom(const float4* __restrict__ pos4, const int* __restrict__ nrow,
                                           const int* __restrict__ nnbr, int cap, const float4* Ds, float rc,
                                           float nrefi, const int* __restrict__ ace_list, int* __restrict__ flags,
                                           float* __restrict__ Aout, int a, BasisSmem& S, int lane) {
    const int gq = lane >> 2, tq = lane & 3;
    const float rc2 = rc * rc;
    const int i = ace_list[a];
    const int cnt = gather_ace_neighbors<kBasisRounds>(pos4, nrow, cap, i, nnbr[i], Ds, rc2, S.nb, S.nbj, lane);
    if (cnt < 0) {
        if (lane == 0) { atomicOr(&flags[kFlagErr], kErrAceCapacity); flags[kFlagBad] = i; }
        return;
    }
    float accA[kNmax];
    double accD[MODE == AP_ACE_FP64 ? kNmax : 1];
    float acc_tc[2][4];
#pragma unroll
    for (int q = 0; q < kNmax; ++q) accA[q] = 0.0f;
#pragma unroll
    for (int q = 0; q < (MODE == AP_ACE_FP64 ? kNmax : 1); ++q) accD[q] = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc_tc[q >> 2][q & 3] = 0.0f;
    for (int t0 = 0; t0 < cnt; t0 += kTile) {
        basis_tile(S.nb, t0, cnt, rc, S.tileY, S.tileG, lane);
        __syncwarp();
        const int nt = min(kTile, cnt - t0);
        if (MODE == AP_ACE_FP32) {
            basis_accum_fp32(S.tileY, S.tileG, nt, lane, accA);
        } else if (MODE == AP_ACE_FP64) {
            if (lane < kNLM) {
                for (int jj2 = 0; jj2 < nt; ++jj2) {
                    const float y = S.tileY[jj2][lane];
                    const float4 g0 = *reinterpret_cast<const float4*>(&S.tileG[jj2][0]);
                    const float4 g1 = *reinterpret_cast<const float4*>(&S.tileG[jj2][4]);
                    const float gg[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
                    for (int q = 0; q < kNmax; ++q) accD[q] = fma((double)y, (double)gg[q], accD[q]);
                }
            }
        } else if (MODE == AP_ACE_TC_TF32X3) {
#pragma unroll
            for (int k0 = 0; k0 < kTile; k0 += 8) {
                const float bv0 = S.tileG[k0 + tq][gq], bv1 = S.tileG[k0 + tq + 4][gq];
                const uint32_t bh0 = to_tf32(bv0), bh1 = to_tf32(bv1);
                const uint32_t bl0 = to_tf32(bv0 - __uint_as_float(bh0)), bl1 = to_tf32(bv1 - __uint_as_float(bh1));
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int m0 = 16 * mt;
                    const float av[4] = {yt(S, m0 + gq, k0 + tq), yt(S, m0 + gq + 8, k0 + tq),
                                         yt(S, m0 + gq, k0 + tq + 4), yt(S, m0 + gq + 8, k0 + tq + 4)};
                    uint32_t ah[4], al[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        ah[q] = to_tf32(av[q]);
                        al[q] = to_tf32(av[q] - __uint_as_float(ah[q]));
                    }
                    mma_tf32(acc_tc[mt], al[0], al[1], al[2], al[3], bh0, bh1);
                    mma_tf32(acc_tc[mt], ah[0], ah[1], ah[2], ah[3], bl0, bl1);
                    mma_tf32(acc_tc[mt], ah[0], ah[1], ah[2], ah[3], bh0, bh1);
                }
            }
        } else {
#pragma unroll
            for (int k0 = 0; k0 < kTile; k0 += 16) {
                const uint32_t b0 = pack2<MODE>(S.tileG[k0 + 2 * tq][gq], S.tileG[k0 + 2 * tq + 1][gq]);
                const uint32_t b1 = pack2<MODE>(S.tileG[k0 + 2 * tq + 8][gq], S.tileG[k0 + 2 * tq + 9][gq]);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int r0 = 16 * mt + gq, r1 = r0 + 8, c0 = k0 + 2 * tq;
                    const uint32_t a0 = pack2<MODE>(yt(S, r0, c0), yt(S, r0, c0 + 1));
                    const uint32_t a1 = pack2<MODE>(yt(S, r1, c0), yt(S, r1, c0 + 1));
                    const uint32_t a2 = pack2<MODE>(yt(S, r0, c0 + 8), yt(S, r0, c0 + 9));
                    const uint32_t a3 = pack2<MODE>(yt(S, r1, c0 + 8), yt(S, r1, c0 + 9));
                    mma_16bit<MODE>(acc_tc[mt], a0, a1, a2, a3, b0, b1);
                }
            }
        }
        __syncwarp();
    }
    if (MODE == AP_ACE_FP32 || MODE == AP_ACE_FP64) {
        if (lane < kNLM) {
            if (MODE == AP_ACE_FP64) {
#pragma unroll
                for (int q = 0; q < kNmax; ++q) accA[q] = (float)(accD[q] * (double)nrefi);
            } else {
#pragma unroll
                for (int q = 0; q < kNmax; ++q) accA[q] *= nrefi;
            }
            float4* o = reinterpret_cast<float4*>(Aout + ((size_t)a * kNLM + lane) * kNmax);
            o[0] = make_float4(accA[0], accA[1], accA[2], accA[3]);
            o[1] = make_float4(accA[4], accA[5], accA[6], accA[7]);
        }
    } else {
        // D fragment: (row g, cols 2t, 2t+1) and (row g + 8, same cols) of each 16-row tile
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int r0 = 16 * mt + gq, r1 = r0 + 8;
            if (r0 < kNLM)
                *reinterpret_cast<float2*>(Aout + ((size_t)a * kNLM + r0) * kNmax + 2 * tq) =
                    make_float2(acc_tc[mt][0] * nrefi, acc_tc[mt][1] * nrefi);
            if (r1 < kNLM)
                *reinterpret_cast<float2*>(Aout + ((size_t)a * kNLM + r1) * kNmax + 2 * tq) =
                    make_float2(acc_tc[mt][2] * nrefi, acc_tc[mt][3] * nrefi);
        }
    }
}

template <int MODE>
__global__ void
#if AP_BASIS_MINB > 1
__launch_bounds__(256, AP_BASIS_MINB)
#else
__launch_bounds__(256)
#endif
k_ace_basis(const float4* __restrict__ pos4, const int* __restrict__ nrow,
                                                   const int* __restrict__ nnbr, int cap, const float4* __restrict__ Dtab,
                                                   int ncode, const AceTc* __restrict__ tab,
                                                   const int* __restrict__ ace_list, int* __restrict__ flags,
                                                   float* __restrict__ Aout) {
    __shared__ float4 Ds[125];
    __shared__ BasisSmem WS[8];
    for (int k = threadIdx.x; k < ncode; k += blockDim.x) Ds[k] = Dtab[k];
    __syncthreads();
    pdl_wait();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BasisSmem& S = WS[warp];
    const float rc = tab->rc, nrefi = tab->nref_inv;
    const int n_ace = flags[kFlagNAce];
    for (int a = blockIdx.x * 8 + warp; a < n_ace; a += gridDim.x * 8) {
        basis_atom<MODE>(pos4, nrow, nnbr, cap, Ds, rc, nrefi, ace_list, flags, Aout, a, S, lane);
    }
}

// ---------------------------------------------------------------------------------
// Tensor-core contraction.  For an l-triple t the three-factor part of phi_p is
//     phi_p^t = sum_{q, n3, m3} C_p[q, n3] P[q, m3] A[n3, m3],
//     P[q = (n1, n2), m3] = sum_{m1, m2} G A[n1, m1] A[n2, m2]      (Gaunt, FP32 lanes),
// and its gradients need two contractions with the coefficient matrix C_p, which every
// atom shares:
//     R_p = C_p^T P     (8 x W3): phi_p^t = sum R_p . A_{l3} and the third-factor gradient
//                                 dE/dA[n3, l3 m3] += R_1 + s R_2, s = 1 / (2 sqrt(phi2));
//     Q   = C_1 A + C_2 (s A)   (64 x W3): the first- and second-factor gradients
//                                 d1 += G Q A[n2], d2 += G Q A[n1]  (Gaunt, FP32 lanes).
// Both run as mma.sync m16n8k8 TF32 with 3xTF32 splitting (hi/lo of both operands, the
// lo*lo product dropped: relative error ~2^-21, FP32-like).  R: M = (density, n3) = 16,
// K = q = 64, N = m3 of one atom; its accumulators for all triples with the same l3 are
// chained, so one epilogue per l3 forms phi and the third-factor gradient.  Q: M = q, K =
// (density, n3) = 16, N = m3.  P and Q pass between the lanes (one (n1, n2) pair each) and
// the fragments through a per-warp staging block of rows m3, columns q.
//
// For the five l1 = l2 triples P and the coefficients are symmetric in (n1, n2): their
// coefficient rows are packed to the 36 pairs n1 <= n2 (R over K = 40, Q over three row
// tiles), and only the first-factor gradient is formed, taken twice.
//
// The five (0, l, l) triples have G = delta_{m2 m3} / sqrt(4 pi): their functions are
// A[n1, 00] times a two-factor product, so they join the two-factor pass with per-atom
// coefficients c2 + sum_n1 C3[n1, (n2, n3)] A[n1, 00] G (and a gradient for A[n1, 00]).  The
// two-factor products are Gram matrices A_l A_l^T, one 3xTF32 tile per l, and so is their
// adjoint.  The other nine triples run through R and Q.  One warp per atom, no block barriers
// in the atom loop.
// ---------------------------------------------------------------------------------
constexpr int kTcWarps = 16;
constexpr int kStRow = 68;                     // staging row stride: 8 rows fall on distinct bank quads

struct TcWarpSmem {
    float A[kNmax * kApad];     // A[n][l-block layout] (Gaunt operands)
    float dA[kNmax * kApad];    // dE/dA, same layout
    float At[32][8];            // A[lm][n3], n3 chunk (n3 / 4) at (n3 / 4) ^ ((lm >> 2) & 1); rows 25..31 zero
    float St[9][kStRow];        // staging of P or Q: row m3, column q
    float R2[kNmax][28];        // second-density third-factor gradient [n3][lm]
};
static_assert(sizeof(TcWarpSmem) % 16 == 0, "16-byte aligned warp regions");
static_assert(kNT3 == 9 && kTcTriple0 == 5, "the tensor-core triples are t = 5 .. 13");

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = to_tf32(x);
    lo = __float_as_uint(x - __uint_as_float(hi));   // the tensor core reads its top 19 bits
}

// d += (ah + al)(bh + bl) without al bl; the small terms first
__device__ __forceinline__ void mma3(float* d, const uint32_t* ah, const uint32_t* al, uint32_t bh0, uint32_t bh1,
                                     uint32_t bl0, uint32_t bl1) {
    mma_tf32(d, al[0], al[1], al[2], al[3], bh0, bh1);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bl0, bl1);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bh0, bh1);
}

// 8 x 4 FP32 tiles (as 8 x 8 b16 matrices) from shared memory; thread t gives the row
// address of matrix t / 8, row t % 8, and receives word t % 4 of row t / 4 of each matrix
__device__ __forceinline__ void ldsm_x4(uint32_t* r, const float* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t* r, const float* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

// P of the lane's pairs q = lane and lane + 32 into the staging rows
template <int T>
__device__ __forceinline__ void tc_stage_p(TcWarpSmem& S, int lane) {
    using R = Tri<T>;
    constexpr bool SYM = R::L1 == R::L2;
    const int n2 = lane & 7;
    float A2[R::W2];
    load_row<R::W2>(A2, S.A + n2 * kApad + R::B2);
#pragma unroll 1
    for (int pp = 0; pp < 2; ++pp) {
        const int q = lane + 32 * pp, n1 = q >> 3;
        float A1[R::W1], P[R::W3];
        load_row<R::W1>(A1, S.A + n1 * kApad + R::B1);
#pragma unroll
        for (int k = 0; k < R::W3; ++k) P[k] = 0.0f;
        all_p<T>(P, A1, A2, std::make_integer_sequence<int, R::N>{});
        if constexpr (SYM) {
            // packed columns: the pair n1 <= n2 stands for both orders (P is symmetric)
            if (n1 <= n2) {
                const float f = n1 < n2 ? 2.0f : 1.0f;
#pragma unroll
                for (int k = 0; k < R::W3; ++k) S.St[k][sym_pair(n1, n2)] = f * P[k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < R::W3; ++k) S.St[k][q] = P[k];
        }
    }
    if constexpr (SYM) {
        // K runs to 40: columns 36..39 meet zero coefficient rows and must hold finite values
        for (int e = lane; e < 4 * R::W3; e += 32) S.St[e >> 2][kSymPairs + (e & 3)] = 0.0f;
    }
}

// R_p += C_p^T P: rows (density, n3), K = q over 8 steps, columns m3; even and odd steps
// accumulate in separate chains (RA0 / RA1; RB for column 8)
template <int T>
__device__ __forceinline__ void tc_r_gemm(const AceTc& C, const TcWarpSmem& S, int lane, float* RA0, float* RA1,
                                          float* RB0, float* RB1) {
    using R = Tri<T>;
    constexpr int U = T - kTcTriple0;
    const int gq = lane >> 2, tq = lane & 3;
    // ldmatrix rows of the B fragment: matrix j = lane / 8 reads row m3 = lane % 8, q chunk j
    const float* brow = &S.St[lane & 7][4 * ((lane >> 3) & 1)];
#pragma unroll 2
    for (int ks = 0; ks < (R::L1 == R::L2 ? 5 : 8); ++ks) {    // packed pairs of the l1 = l2 triples: K = 40
        const int qa = 8 * ks + tq, qb = qa + 4;
        uint32_t ah[4], al[4];
        ah[0] = __float_as_uint(C.c3[0][0][U][qa][gq]);
        ah[1] = __float_as_uint(C.c3[0][1][U][qa][gq]);
        ah[2] = __float_as_uint(C.c3[0][0][U][qb][gq ^ 4]);
        ah[3] = __float_as_uint(C.c3[0][1][U][qb][gq ^ 4]);
        al[0] = __float_as_uint(C.c3[1][0][U][qa][gq]);
        al[1] = __float_as_uint(C.c3[1][1][U][qa][gq]);
        al[2] = __float_as_uint(C.c3[1][0][U][qb][gq ^ 4]);
        al[3] = __float_as_uint(C.c3[1][1][U][qb][gq ^ 4]);
        uint32_t b[2], bh0, bl0, bh1, bl1;
        ldsm_x2(b, brow + 8 * ks);
        split_tf32(__uint_as_float(b[0]), bh0, bl0);
        split_tf32(__uint_as_float(b[1]), bh1, bl1);
        mma3((ks & 1) ? RA1 : RA0, ah, al, bh0, bh1, bl0, bl1);
        if constexpr (R::W3 > 8) {
            split_tf32(gq == 0 ? S.St[8][qa] : 0.0f, bh0, bl0);
            split_tf32(gq == 0 ? S.St[8][qb] : 0.0f, bh1, bl1);
            mma3((ks & 1) ? RB1 : RB0, ah, al, bh0, bh1, bl0, bl1);
        }
    }
}

template <int T>
__device__ __forceinline__ void tc_forward_triple(const AceTc& C, TcWarpSmem& S, int lane, float* RA0, float* RA1,
                                                  float* RB0, float* RB1) {
    tc_stage_p<T>(S, lane);
    __syncwarp();
    tc_r_gemm<T>(C, S, lane, RA0, RA1, RB0, RB1);
    __syncwarp();
}

// the tensor-core triples of one l3: chained R accumulators, then phi and the third-factor
// gradient (thread (g, t) holds R_1[n3 = g][m3 = 2t, 2t + 1] in RA[0..1] and R_2 in RA[2..3])
// GW: weight of the third-factor gradient (3 for the triples whose three factors have equal
// l, whose coefficients are fully symmetric: their gradient is the same for all three factors,
// so the first- and second-factor passes are left out); ACC: another group with the same l3
// already wrote its second-density rows R2, which this one adds to
template <int L, int GW, bool ACC, int... T>
__device__ __forceinline__ void tc_forward_group(const AceTc& C, TcWarpSmem& S, int lane, float& p1, float& p2,
                                                 std::integer_sequence<int, T...>) {
    float RA0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, RA1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float RB0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, RB1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    (tc_forward_triple<T>(C, S, lane, RA0, RA1, RB0, RB1), ...);
    constexpr int W = 2 * L + 1;
    const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int m = 2 * tq + e;
        if (m < W) {
            const float r1 = RA0[e] + RA1[e], r2 = RA0[2 + e] + RA1[2 + e];
            const float a = S.A[gq * kApad + lblk(L) + m];
            p1 = fmaf(r1, a, p1);
            p2 = fmaf(r2, a, p2);
            S.dA[gq * kApad + lblk(L) + m] = fmaf((float)GW, r1, S.dA[gq * kApad + lblk(L) + m]);
            if constexpr (ACC) S.R2[gq][L * L + m] = fmaf((float)GW, r2, S.R2[gq][L * L + m]);
            else S.R2[gq][L * L + m] = (float)GW * r2;
        }
    }
    if constexpr (W > 8) {
        if (tq == 0) {
            const float r1 = RB0[0] + RB1[0], r2 = RB0[2] + RB1[2];
            const float a = S.A[gq * kApad + lblk(L) + 8];
            p1 = fmaf(r1, a, p1);
            p2 = fmaf(r2, a, p2);
            S.dA[gq * kApad + lblk(L) + 8] = fmaf((float)GW, r1, S.dA[gq * kApad + lblk(L) + 8]);
            if constexpr (ACC) S.R2[gq][L * L + 8] = fmaf((float)GW, r2, S.R2[gq][L * L + 8]);
            else S.R2[gq][L * L + 8] = (float)GW * r2;
        }
    }
}

// one m-tile of Q = C_1 A + C_2 (s A) into the staging rows
template <int T, int NT>
__device__ __forceinline__ void tc_q_tile(const AceTc& C, TcWarpSmem& S, int lane, int mt, const uint32_t (*bh)[2][2],
                                          const uint32_t (*bl)[2][2]) {
    constexpr int U = T - kTcTriple0;
    const int gq = lane >> 2, tq = lane & 3;
    // ldmatrix row of this thread: matrix j = lane / 8 (rows + 8 for odd j, n3 chunk j / 2)
    const int qr = 16 * mt + (lane & 7) + 8 * ((lane >> 3) & 1);
    const int off = 4 * ((lane >> 4) ^ ((qr >> 2) & 1));
    uint32_t ah[2][4], al[2][4];
    ldsm_x4(ah[0], &C.c3[0][0][U][qr][off]);
    ldsm_x4(al[0], &C.c3[1][0][U][qr][off]);
    ldsm_x4(ah[1], &C.c3[0][1][U][qr][off]);
    ldsm_x4(al[1], &C.c3[1][1][U][qr][off]);
    float D[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        D[nt][0] = D[nt][1] = D[nt][2] = D[nt][3] = 0.0f;
#pragma unroll
        for (int p = 0; p < 2; ++p) mma3(D[nt], ah[p], al[p], bh[nt][p][0], bh[nt][p][1], bl[nt][p][0], bl[nt][p][1]);
    }
    // D[nt]: rows q = 16 mt + g (+8), columns m3 = 8 nt + 2t (+1)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int q = 16 * mt + gq + 8 * r;
        S.St[2 * tq][q] = D[0][2 * r];
        S.St[2 * tq + 1][q] = D[0][2 * r + 1];
        if constexpr (NT > 1) {
            if (tq == 0) S.St[8][q] = D[1][2 * r];
        }
    }
}

// Q into the staging, then the first- and second-factor gradients
template <int T>
__device__ __forceinline__ void tc_adjoint_triple(const AceTc& C, TcWarpSmem& S, float s, int lane) {
    using R = Tri<T>;
    constexpr int NT = R::W3 > 8 ? 2 : 1;
    // B fragments: B[k = n3][n = m3] = A[n3][lm = l3^2 + 8 nt + n] (first density), s times
    // that (second); ldmatrix rows lm, chunks n3 0..3 and 4..7
    uint32_t bh[NT][2][2], bl[NT][2][2];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int lm = R::L3 * R::L3 + 8 * nt + (lane & 7);
        const int chunk = ((lane >> 3) & 1) ^ ((lm >> 2) & 1);
        uint32_t b[2];
        ldsm_x2(b, &S.At[lm][4 * chunk]);
        const float x0 = __uint_as_float(b[0]), x1 = __uint_as_float(b[1]);
        split_tf32(x0, bh[nt][0][0], bl[nt][0][0]);
        split_tf32(x1, bh[nt][0][1], bl[nt][0][1]);
        split_tf32(s * x0, bh[nt][1][0], bl[nt][1][0]);
        split_tf32(s * x1, bh[nt][1][1], bl[nt][1][1]);
    }
#pragma unroll 2
    for (int mt = 0; mt < (R::L1 == R::L2 ? 3 : 4); ++mt) tc_q_tile<T, NT>(C, S, lane, mt, bh, bl);
    __syncwarp();
    // Gaunt adjoint of the lane's pairs (n1, n2) = (lane / 8 + 4 pp, lane % 8).  For l1 = l2
    // the coefficients are symmetric in (n1, n2) and the Gaunt coefficients in (m1, m2), so
    // the second-factor gradient summed over the pairs equals the first-factor one: d1 is
    // taken twice and d2 is not formed
    constexpr bool SYM = R::L1 == R::L2;
    constexpr float F1 = SYM ? 2.0f : 1.0f;
    const int n1 = lane >> 3, n2 = lane & 7;
    float A2[R::W2], d2[R::W2];
    load_row<R::W2>(A2, S.A + n2 * kApad + R::B2);
#pragma unroll
    for (int k = 0; k < R::W2; ++k) d2[k] = 0.0f;
#pragma unroll 1
    for (int pp = 0; pp < 2; ++pp) {
        const int q = lane + 32 * pp, r1 = n1 + 4 * pp;
        float A1[R::W1], d1[R::W1], Q[R::W3];
        load_row<R::W1>(A1, S.A + r1 * kApad + R::B1);
#pragma unroll
        const int qs = SYM ? sym_pair(min(r1, n2), max(r1, n2)) : q;    // Q is symmetric for l1 = l2
#pragma unroll
        for (int k = 0; k < R::W3; ++k) Q[k] = S.St[k][qs];
#pragma unroll
        for (int k = 0; k < R::W1; ++k) d1[k] = 0.0f;
        all_x<T, !SYM>(d1, d2, A1, A2, Q, std::make_integer_sequence<int, R::N>{});
#pragma unroll
        for (int k = 0; k < R::W1; ++k) {
            float v = d1[k];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            d1[k] = v;
        }
        if ((lane & 7) == 0) {
#pragma unroll
            for (int k = 0; k < R::W1; ++k) S.dA[r1 * kApad + R::B1 + k] = fmaf(F1, d1[k], S.dA[r1 * kApad + R::B1 + k]);
        }
        __syncwarp();
    }
    if constexpr (!SYM) {
#pragma unroll
        for (int k = 0; k < R::W2; ++k) {
            float v = d2[k];
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            d2[k] = v;
        }
        if (lane < 8) {
#pragma unroll
            for (int k = 0; k < R::W2; ++k) S.dA[lane * kApad + R::B2 + k] += d2[k];
        }
        __syncwarp();
    }
}

template <int... T>
__device__ __forceinline__ void tc_adjoint_all(const AceTc& C, TcWarpSmem& S, float s, int lane,
                                               std::integer_sequence<int, T...>) {
    (tc_adjoint_triple<T>(C, S, s, lane), ...);
}

// The one- and two-factor functions, with the (0, l, l) triples folded into the latter:
//   phi_p += sum_l sum_q F_p[l][q] mm_l[q],  F_p[l][q] = c2_p[l][q] + sum_n1 c0ll_p[l][q][n1] A[n1, 00],
//   mm_l[n1 n2] = sum_m A[n1, lm] A[n2, lm]  (the Gram matrix of the l-block, one 3xTF32 tile)
// Thread (g, t) holds the pairs q = 8 g + 2 t + j (j = 0, 1) of the tile's accumulator rows.
struct Nu2 {
    float f[2][5][2];    // F_p[l][q_j]
    float g[2][8];       // the thread's part of sum_{l, q} c0ll_p[l][q][n1] mm_l[q], the A[n1, 00] gradient
};

// mm_l[g][2 t + j] into mm[j] (rows g + 8 of the tile are zero); the A fragment of the Gram
// tile is also its B fragment.  Columns past the l-block are read as zero: the padding of
// the l-block layout is zero, and the next block's columns are masked
template <int L>
__device__ __forceinline__ void nu2_gram(const TcWarpSmem& S, int g, int t, float* mm) {
    constexpr int B = lblk(L);
    mm[0] = mm[1] = mm[2] = mm[3] = 0.0f;
    const float x0 = S.A[g * kApad + B + t];
    const float x2 = L >= 2 ? S.A[g * kApad + B + 4 + t] : 0.0f;
    uint32_t h0, l0, h2, l2;
    split_tf32(x0, h0, l0);
    split_tf32(x2, h2, l2);
    mma_tf32(mm, l0, 0u, l2, 0u, h0, h2);
    mma_tf32(mm, h0, 0u, h2, 0u, l0, l2);
    mma_tf32(mm, h0, 0u, h2, 0u, h0, h2);
    if constexpr (L == 4) {                            // m = 8 and the block's zero padding
        const float x4 = S.A[g * kApad + B + 8 + t];
        split_tf32(x4, h0, l0);
        mma_tf32(mm, l0, 0u, 0u, 0u, h0, 0u);
        mma_tf32(mm, h0, 0u, 0u, 0u, l0, 0u);
        mma_tf32(mm, h0, 0u, 0u, 0u, h0, 0u);
    }
}

template <int L>
__device__ __forceinline__ void nu2_forward_l(const AceTc& C, const TcWarpSmem& S, int g, int t, const float* a00,
                                              float& p1, float& p2, Nu2& N) {
    float mm[4];
    nu2_gram<L>(S, g, t, mm);
    const int q0 = 8 * g + 2 * t;
    const float2 c20 = *reinterpret_cast<const float2*>(&C.c2[0][L][q0]);
    const float2 c21 = *reinterpret_cast<const float2*>(&C.c2[1][L][q0]);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int pos = c0ll_pos(q0 + j);
        const float4 u0 = *reinterpret_cast<const float4*>(C.c0ll[0][L][0][pos]);
        const float4 u1 = *reinterpret_cast<const float4*>(C.c0ll[0][L][1][pos]);
        const float4 v0 = *reinterpret_cast<const float4*>(C.c0ll[1][L][0][pos]);
        const float4 v1 = *reinterpret_cast<const float4*>(C.c0ll[1][L][1][pos]);
        const float cu[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
        const float cv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        float f0 = j ? c20.y : c20.x, f1 = j ? c21.y : c21.x;
#pragma unroll
        for (int k = 0; k < kNmax; ++k) {
            f0 = fmaf(cu[k], a00[k], f0);
            f1 = fmaf(cv[k], a00[k], f1);
            N.g[0][k] = fmaf(cu[k], mm[j], N.g[0][k]);
            N.g[1][k] = fmaf(cv[k], mm[j], N.g[1][k]);
        }
        p1 = fmaf(f0, mm[j], p1);
        p2 = fmaf(f1, mm[j], p2);
        N.f[0][L][j] = f0;
        N.f[1][L][j] = f1;
    }
}

// dA_l[n1][m] += sum_n2 (CT[n1][n2] + CT[n2][n1]) A[n2, lm], CT = F_1 + s F_2, as one 3xTF32
// tile (two for l = 4); CT and its transpose are staged in the (free) staging rows
template <int L>
__device__ __forceinline__ void nu2_adjoint_l(TcWarpSmem& S, int g, int t, float s, const Nu2& N) {
    constexpr int B = lblk(L), W = 2 * L + 1;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float ct = fmaf(s, N.f[1][L][j], N.f[0][L][j]);
        S.St[g][2 * t + j] = ct;                       // CT[n1][n2] at St[n1][n2]
        S.St[2 * t + j][32 + g] = ct;                  // ... and at St[n2][32 + n1]
    }
    __syncwarp();
    const float m0 = S.St[g][t] + S.St[g][32 + t];     // M[g][t] = CT[g][t] + CT[t][g]
    const float m2 = S.St[g][t + 4] + S.St[g][36 + t]; // M[g][t + 4]
    __syncwarp();                                      // the rows are free for the next l
    uint32_t mh0, ml0, mh2, ml2;
    split_tf32(m0, mh0, ml0);
    split_tf32(m2, mh2, ml2);
    // B[k = n2][n = m] = A[n2, lm]; columns past the block (l <= 1) give discarded outputs
    {
        float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        uint32_t bh0, bl0, bh1, bl1;
        split_tf32(S.A[t * kApad + B + g], bh0, bl0);
        split_tf32(S.A[(t + 4) * kApad + B + g], bh1, bl1);
        mma_tf32(d, ml0, 0u, ml2, 0u, bh0, bh1);
        mma_tf32(d, mh0, 0u, mh2, 0u, bl0, bl1);
        mma_tf32(d, mh0, 0u, mh2, 0u, bh0, bh1);
#pragma unroll
        for (int j = 0; j < 2; ++j)
            if (2 * t + j < W) S.dA[g * kApad + B + 2 * t + j] += d[j];
    }
    if constexpr (W > 8) {                             // m = 8: column 0 of the second tile
        float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        uint32_t bh0, bl0, bh1, bl1;
        split_tf32(g == 0 ? S.A[t * kApad + B + 8] : 0.0f, bh0, bl0);
        split_tf32(g == 0 ? S.A[(t + 4) * kApad + B + 8] : 0.0f, bh1, bl1);
        mma_tf32(d, ml0, 0u, ml2, 0u, bh0, bh1);
        mma_tf32(d, mh0, 0u, mh2, 0u, bl0, bl1);
        mma_tf32(d, mh0, 0u, mh2, 0u, bh0, bh1);
        if (t == 0) S.dA[g * kApad + B + 8] += d[0];
    }
}

// phi1, phi2 of the atom whose A is in S (tc_load_atom), E = phi1 + sqrt(phi2) without the
// constant c1_0 into e_out, and dE/dA into S.dA; false outside the domain (phi2 <= 1e-3 or
// a NaN), where E and dA carry no meaning
__device__ __forceinline__ bool tc_contract_atom(const AceTc& C, TcWarpSmem& S, int lane, float& e_out) {
    const int g = lane >> 2, t = lane & 3;
    float p1 = 0.0f, p2 = 0.0f;
    // the tensor-core triples, grouped by l3
    tc_forward_group<1, 1, false>(C, S, lane, p1, p2, std::integer_sequence<int, 6, 7>{});
    tc_forward_group<2, 1, false>(C, S, lane, p1, p2, std::integer_sequence<int, 5, 10, 11>{});
    tc_forward_group<2, 3, true>(C, S, lane, p1, p2, std::integer_sequence<int, 8>{});      // (2, 2, 2)
    tc_forward_group<4, 1, false>(C, S, lane, p1, p2, std::integer_sequence<int, 9, 12>{});
    tc_forward_group<4, 3, true>(C, S, lane, p1, p2, std::integer_sequence<int, 13>{});     // (4, 4, 4)
    __syncwarp();                                      // the epilogues' dA and R2 are visible
    // one- and two-factor functions
    float a00[kNmax];
#pragma unroll
    for (int k = 0; k < kNmax; ++k) a00[k] = S.A[k * kApad];
    if (lane < kNmax) {
        p1 = fmaf(C.c1[0][lane], a00[lane], p1);
        p2 = fmaf(C.c1[1][lane], a00[lane], p2);
    }
    Nu2 N;
#pragma unroll
    for (int k = 0; k < kNmax; ++k) N.g[0][k] = N.g[1][k] = 0.0f;
    nu2_forward_l<0>(C, S, g, t, a00, p1, p2, N);
    nu2_forward_l<1>(C, S, g, t, a00, p1, p2, N);
    nu2_forward_l<2>(C, S, g, t, a00, p1, p2, N);
    nu2_forward_l<3>(C, S, g, t, a00, p1, p2, N);
    nu2_forward_l<4>(C, S, g, t, a00, p1, p2, N);
    p1 = warp_sum(p1);
    p2 = warp_sum(p2);
    const bool ok = C.c2_0 + p2 > 1e-3f && p1 == p1;
    const float sq = ok ? sqrtf(C.c2_0 + p2) : 0.0f;
    const float s = ok ? 0.5f / sq : 0.0f;
    // adjoint: one- and two-factor functions (with the folded triples and their A[n1, 00]
    // gradient), the second density's third-factor part
    nu2_adjoint_l<0>(S, g, t, s, N);
    nu2_adjoint_l<1>(S, g, t, s, N);
    nu2_adjoint_l<2>(S, g, t, s, N);
    nu2_adjoint_l<3>(S, g, t, s, N);
    nu2_adjoint_l<4>(S, g, t, s, N);
    float g00[kNmax];
#pragma unroll
    for (int k = 0; k < kNmax; ++k) g00[k] = warp_sum(fmaf(s, N.g[1][k], N.g[0][k]));
    __syncwarp();
    if (lane < kNmax) {
        float gk = g00[0];
#pragma unroll
        for (int k = 1; k < kNmax; ++k) gk = lane == k ? g00[k] : gk;
        S.dA[lane * kApad] += gk + fmaf(s, C.c1[1][lane], C.c1[0][lane]);
    }
    for (int e = lane; e < kNmax * 17; e += 32) {
        // lm = 1 .. 8 and 16 .. 24: the third factors (l = 1, 2 and 4 in the kernel's order)
        // of the tensor-core triples
        const int n3 = e / 17, k = e - n3 * 17, lm = k < 8 ? 1 + k : 8 + k;
        const int l = lm < 4 ? 1 : (lm < 9 ? 2 : 4);
        S.dA[n3 * kApad + lblk(l) + (lm - l * l)] += s * S.R2[n3][lm];
    }
    __syncwarp();
    // (2, 2, 2) and (4, 4, 4) have no first- and second-factor pass (their gradient is the
    // third-factor one taken three times)
    tc_adjoint_all(C, S, s, lane, std::integer_sequence<int, 5, 6, 7, 9, 10, 11, 12>{});
    e_out = p1 + sq;
    return ok;
}

// A of one atom into the warp's region (lane lm < 25 gives A[n][lm] for n = 0..3 in g0 and
// 4..7 in g1; lam_pad is the lane's column in the l-block layout), dA cleared
__device__ __forceinline__ void tc_load_atom(TcWarpSmem& S, int lane, int lam_pad, float4 g0, float4 g1) {
    if (lane < kNLM) {
        const float v[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
        for (int q = 0; q < kNmax; ++q) S.A[q * kApad + lam_pad] = v[q];
        const int sw = (lane >> 2) & 1;
        reinterpret_cast<float4*>(&S.At[lane][0])[sw] = g0;
        reinterpret_cast<float4*>(&S.At[lane][0])[sw ^ 1] = g1;
    }
    for (int k = lane; k < kNmax * kApad; k += 32) S.dA[k] = 0.0f;
    __syncwarp();
}

// the lane's column lm of the l-block layout (l-blocks at 0, 4, 8, 16, 24)
__device__ __forceinline__ int lane_lm_pad(int lane) {
    int l = 0;
    if (lane >= 1) l = 1;
    if (lane >= 4) l = 2;
    if (lane >= 9) l = 3;
    if (lane >= 16) l = 4;
    return lblk(l) + (lane - l * l);
}

// one-time set-up of a warp region: zero, so that the padding of A and At and the staging
// rows stay finite
__device__ __forceinline__ void tc_zero_regions(TcWarpSmem* WS, int nwarps) {
    float4* z = reinterpret_cast<float4*>(WS);
    for (int k = threadIdx.x; k < (int)(nwarps * sizeof(TcWarpSmem) / 16); k += blockDim.x)
        z[k] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// contraction of compacted atom a: A from Ain, dE/dA to dAout, E_i^ACE to e_ace (one warp)
__device__ __forceinline__ void contract_atom(const AceTc& C, TcWarpSmem& S, int lane, int lam_pad,
                                              const float* __restrict__ Ain, float* __restrict__ dAout,
                                              float* __restrict__ e_ace, const int* __restrict__ ace_list,
                                              int* __restrict__ flags, int a) {
    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
    if (lane < kNLM) {
        const float4* src = reinterpret_cast<const float4*>(Ain + ((size_t)a * kNLM + lane) * kNmax);
        g0 = src[0];
        g1 = src[1];
    }
    tc_load_atom(S, lane, lam_pad, g0, g1);
    float e = 0.0f;
    const bool ok = tc_contract_atom(C, S, lane, e);
    const int i = ace_list[a];
    if (!ok) {
        if (lane == 0) { atomicOr(&flags[kFlagErr], kErrDomain); flags[kFlagBad] = i; e_ace[i] = __int_as_float(0x7fc00000); }
        if (lane < kNLM) {
            float4* o = reinterpret_cast<float4*>(dAout + ((size_t)a * kNLM + lane) * kNmax);
            o[0] = make_float4(0.f, 0.f, 0.f, 0.f);
            o[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    } else {
        if (lane < kNLM) {
            float v[kNmax];
#pragma unroll
            for (int q = 0; q < kNmax; ++q) v[q] = S.dA[q * kApad + lam_pad];
            float4* o = reinterpret_cast<float4*>(dAout + ((size_t)a * kNLM + lane) * kNmax);
            o[0] = make_float4(v[0], v[1], v[2], v[3]);
            o[1] = make_float4(v[4], v[5], v[6], v[7]);
        }
        if (lane == 0) e_ace[i] = e;
    }
    __syncwarp();
}

// stages a5/a6 core on tensor cores: phi1, phi2, E = phi1 + sqrt(phi2) and dE/dA from A,
// one warp per compacted atom
__global__ void __launch_bounds__(kTcWarps * 32, 1)
k_ace_contract(const AceTc* __restrict__ tab, const int* __restrict__ ace_list, int* __restrict__ flags,
               const float* __restrict__ Ain, float* __restrict__ dAout, float* __restrict__ e_ace) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AceTc& C = *reinterpret_cast<AceTc*>(smem_raw);
    TcWarpSmem* WS = reinterpret_cast<TcWarpSmem*>(smem_raw + sizeof(AceTc));
    {
        const int4* src = reinterpret_cast<const int4*>(tab);
        int4* dst = reinterpret_cast<int4*>(smem_raw);
        for (int k = threadIdx.x; k < (int)(sizeof(AceTc) / 16); k += blockDim.x) dst[k] = src[k];
        tc_zero_regions(WS, kTcWarps);
    }
    __syncthreads();
    pdl_wait();                                            // the constant tables are staged
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    TcWarpSmem& S = WS[warp];
    const int n_ace = flags[kFlagNAce];
    const int lam_pad = lane_lm_pad(lane);
    for (int a = blockIdx.x * kTcWarps + warp; a < n_ace; a += gridDim.x * kTcWarps)
        contract_atom(C, S, lane, lam_pad, Ain, dAout, e_ace, ace_list, flags, a);
}

struct ForceSmem {
    float dAT[kNLM][kNmax];
    float4 nb[kAceNbrCap];
    int nbj[kAceNbrCap];
};

// the pair forces of compacted atom a (stage a6), one warp; neighbour offsets Ds staged by the caller
__device__ __forceinline__ void force_atom(const float4* __restrict__ pos4, const int* __restrict__ nrow, int cap,
                                           const int* __restrict__ nnbr, int n, const float4* Ds, float rc,
                                           float nrefi, const int* __restrict__ ace_list, const float* __restrict__ wv,
                                           const float* __restrict__ dAin, float* __restrict__ vir,
                                           unsigned long long* __restrict__ acc, int a, ForceSmem& S, int lane) {
    const float rc2 = rc * rc;
    // dE/dA of the atom is requested before the gather, so that its load overlaps it
    const float4* dsrc = reinterpret_cast<const float4*>(dAin + (size_t)a * kNLM * kNmax);
    const float4 da0 = dsrc[lane], da1 = lane < 2 * kNLM - 32 ? dsrc[32 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int i = ace_list[a];
    const float wi = wv[i];
    const int cnt = gather_ace_neighbors<4>(pos4, nrow, cap, i, nnbr[i], Ds, rc2, S.nb, S.nbj, lane);
    if (cnt < 0) return;
    reinterpret_cast<float4*>(&S.dAT[0][0])[lane] = da0;
    if (lane < 2 * kNLM - 32) reinterpret_cast<float4*>(&S.dAT[0][0])[32 + lane] = da1;
    __syncwarp();
    float fsx = 0.f, fsy = 0.f, fsz = 0.f;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f, v4 = 0.f, v5 = 0.f;
    for (int t0 = 0; t0 < cnt; t0 += 32) {
        const int jj = t0 + lane;
        if (jj < cnt) {
            const float4 v = S.nb[jj];
            const int j = S.nbj[jj];
            const float3 fp = ace_pair_force(v, rc, nrefi, wi, S.dAT);
            const float fx = fp.x, fy = fp.y, fz = fp.z;
            fix_add(&acc[j], -fx);
            fix_add(&acc[(size_t)n + j], -fy);
            fix_add(&acc[(size_t)2 * n + j], -fz);
            fsx += fx; fsy += fy; fsz += fz;
            v0 -= v.x * fx; v1 -= v.y * fy; v2 -= v.z * fz;
            v3 -= 0.5f * (v.x * fy + v.y * fx); v4 -= 0.5f * (v.x * fz + v.z * fx); v5 -= 0.5f * (v.y * fz + v.z * fy);
        }
    }
    fsx = warp_sum(fsx); fsy = warp_sum(fsy); fsz = warp_sum(fsz);
    v0 = warp_sum(v0); v1 = warp_sum(v1); v2 = warp_sum(v2);
    v3 = warp_sum(v3); v4 = warp_sum(v4); v5 = warp_sum(v5);
    if (lane == 0) {
        fix_add(&acc[i], fsx);
        fix_add(&acc[(size_t)n + i], fsy);
        fix_add(&acc[(size_t)2 * n + i], fsz);
        vir[i] = v0; vir[n + i] = v1; vir[2 * n + i] = v2; vir[3 * n + i] = v3; vir[4 * n + i] = v4; vir[5 * n + i] = v5;
    }
    __syncwarp();
}


// stage a6: f_ij = (1/nref) sum dE/dA_nlm grad(g_n Y_lm), scattered with weight w_i
__global__ void __launch_bounds__(256) k_ace_force(const float4* __restrict__ pos4, const int* __restrict__ nrow,
                                                   int cap, const int* __restrict__ nnbr, int n, const float4* __restrict__ Dtab,
                                                   int ncode, const AceTc* __restrict__ tab,
                                                   const int* __restrict__ ace_list, const float* __restrict__ wv,
                                                   int* __restrict__ flags, const float* __restrict__ dAin,
                                                   float* __restrict__ vir, unsigned long long* __restrict__ acc) {
    __shared__ float4 Ds[125];
    __shared__ ForceSmem WS[8];
    for (int k = threadIdx.x; k < ncode; k += blockDim.x) Ds[k] = Dtab[k];
    __syncthreads();
    pdl_wait();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ForceSmem& S = WS[warp];
    const float rc = tab->rc, nrefi = tab->nref_inv;
    const int n_ace = flags[kFlagNAce];
    for (int a = blockIdx.x * 8 + warp; a < n_ace; a += gridDim.x * 8) {
        force_atom(pos4, nrow, cap, nnbr, n, Ds, rc, nrefi, ace_list, wv, dAin, vir, acc, a, S, lane);
    }
}

// ---------------------------------------------------------------------------------
// Batched ACE stages over several contexts: a persistent grid walks chunks of compacted
// atoms (per chunk one atom per warp) of all contexts in order; chunk c belongs to the
// context k with pre[k] <= c < pre[k + 1], pre the prefix of the contexts' chunk counts,
// formed from their device atom counts at the start of each launch.  A block restages a
// context's constant tables only when the context (the neighbour offsets) or the potential
// (the coefficient tables, shared per potential) changes.
// ---------------------------------------------------------------------------------
// chunks of `per` atoms of every context into pre[0 .. nctx] (shared memory); the total.
// The atom counts come from the preceding stage: this is where a programmatically launched
// batch kernel waits for it.
__device__ __forceinline__ int batch_chunks(const BatchTable& t, int per, int* pre) {
    pdl_wait();
    if ((int)threadIdx.x < t.nctx) {
        const int na = t.d[threadIdx.x]->flags[kFlagNAce];
        pre[threadIdx.x + 1] = (na + per - 1) / per;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        pre[0] = 0;
        for (int k = 0; k < t.nctx; ++k) pre[k + 1] += pre[k];
    }
    __syncthreads();
    return pre[t.nctx];
}

__global__ void __launch_bounds__(256) kb_ace_basis(const BatchTable t) {
    __shared__ float4 Ds[125];
    __shared__ BasisSmem WS[8];
    __shared__ int pre[kMaxBatchCtx + 1];
    const int total = batch_chunks(t, 8, pre);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int cur = -1;
    for (int ch = blockIdx.x; ch < total; ch += gridDim.x) {
        const int k = batch_find(pre, t.nctx, ch);
        const CtxDev& c = *t.d[k];
        if (k != cur) {
            __syncthreads();
            for (int q = threadIdx.x; q < c.grid.ncode; q += blockDim.x) Ds[q] = c.D[q];
            __syncthreads();
            cur = k;
        }
        const int a = (ch - pre[k]) * 8 + warp;
        if (a < c.flags[kFlagNAce])
            basis_atom<AP_ACE_FP32>(c.pos4, c.nbr_row, c.nnbr, c.cap, Ds, c.ace->rc, c.ace->nref_inv, c.ace_list, c.flags,
                                    c.ace_A, a, WS[warp], lane);
    }
}

__global__ void __launch_bounds__(kTcWarps * 32, 1) kb_ace_contract(const BatchTable t) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AceTc& C = *reinterpret_cast<AceTc*>(smem_raw);
    TcWarpSmem* WS = reinterpret_cast<TcWarpSmem*>(smem_raw + sizeof(AceTc));
    __shared__ int pre[kMaxBatchCtx + 1];
    tc_zero_regions(WS, kTcWarps);
    const int total = batch_chunks(t, kTcWarps, pre);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lam_pad = lane_lm_pad(lane);
    const AceTc* cur = nullptr;
    for (int ch = blockIdx.x; ch < total; ch += gridDim.x) {
        const int k = batch_find(pre, t.nctx, ch);
        const CtxDev& c = *t.d[k];
        if (c.ace != cur) {
            __syncthreads();
            const int4* src = reinterpret_cast<const int4*>(c.ace);
            int4* dst = reinterpret_cast<int4*>(smem_raw);
            for (int q = threadIdx.x; q < (int)(sizeof(AceTc) / 16); q += blockDim.x) dst[q] = src[q];
            __syncthreads();
            cur = c.ace;
        }
        const int a = (ch - pre[k]) * kTcWarps + warp;
        if (a < c.flags[kFlagNAce])
            contract_atom(C, WS[warp], lane, lam_pad, c.ace_A, c.ace_dA, c.e_ace, c.ace_list, c.flags, a);
    }
}

__global__ void __launch_bounds__(256) kb_ace_force(const BatchTable t) {
    __shared__ float4 Ds[125];
    __shared__ ForceSmem WS[8];
    __shared__ int pre[kMaxBatchCtx + 1];
    const int total = batch_chunks(t, 8, pre);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int cur = -1;
    for (int ch = blockIdx.x; ch < total; ch += gridDim.x) {
        const int k = batch_find(pre, t.nctx, ch);
        const CtxDev& c = *t.d[k];
        if (k != cur) {
            __syncthreads();
            for (int q = threadIdx.x; q < c.grid.ncode; q += blockDim.x) Ds[q] = c.D[q];
            __syncthreads();
            cur = k;
        }
        const int a = (ch - pre[k]) * 8 + warp;
        if (a < c.flags[kFlagNAce])
            force_atom(c.pos4, c.nbr_row, c.cap, c.nnbr, c.n, Ds, c.ace->rc, c.ace->nref_inv, c.ace_list, c.w, c.ace_dA,
                       c.vir_ace, c.acc, a, WS[warp], lane);
    }
}

}  // namespace

template <class K>
int persistent_blocks(K kernel, int dev, int threads, size_t smem) {
    struct Entry { const void* k; int dev, threads; size_t smem; int blocks; };
    static std::mutex mu;
    static std::vector<Entry> cache;
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry& e : cache)
        if (e.k == (const void*)kernel && e.dev == dev && e.threads == threads && e.smem == smem) return e.blocks;
    int nsm = 0, per = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    const int blocks = nsm * (per > 0 ? per : 1);
    cache.push_back({(const void*)kernel, dev, threads, smem, blocks});
    return blocks;
}

// Grids of the ACE kernels: persistent, but no larger than the context's atoms can fill (n is
// the host's bound on the compacted count): a small context then leaves the other SMs to the
// kernels of other contexts instead of occupying every SM with idle blocks.
int ace_grid(int persistent, int n, int atoms_per_block) {
    return std::max(1, std::min(persistent, (n + atoms_per_block - 1) / atoms_per_block));
}

template <int MODE>
void launch_basis_mode(Ctx& c, cudaStream_t s) {
    const int nb = ace_grid(persistent_blocks(k_ace_basis<MODE>, c.dev, 256, 0), c.n, 8);
    launch_pdl(k_ace_basis<MODE>, nb, 256, 0, s, c.pos4, c.nbr_row, c.nnbr, c.cap, c.D, c.grid.ncode, c.ace_tc_d, c.ace_list,
               c.flags, c.ace_A);
}

int launch_ace_basis(Ctx& c, cudaStream_t s) {
    switch (c.ace_prec) {
        case AP_ACE_TC_TF32X3: launch_basis_mode<AP_ACE_TC_TF32X3>(c, s); break;
        case AP_ACE_TC_BF16: launch_basis_mode<AP_ACE_TC_BF16>(c, s); break;
        case AP_ACE_TC_FP16: launch_basis_mode<AP_ACE_TC_FP16>(c, s); break;
        case AP_ACE_FP64: launch_basis_mode<AP_ACE_FP64>(c, s); break;
        default: launch_basis_mode<AP_ACE_FP32>(c, s); break;
    }
    return 1;
}

size_t ace_tc_smem_bytes() { return sizeof(AceTc) + kTcWarps * sizeof(TcWarpSmem); }

int launch_ace(Ctx& c, cudaStream_t s) {
    static int configured = -1;
    if (configured != c.dev) {
        cudaFuncSetAttribute(k_ace_contract, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ace_tc_smem_bytes());
        configured = c.dev;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c.dev);
    launch_pdl(k_ace_contract, ace_grid(nsm, c.n, kTcWarps), kTcWarps * 32, ace_tc_smem_bytes(), s, c.ace_tc_d,
               c.ace_list, c.flags, c.ace_A, c.ace_dA, c.e_ace);
    return 1;
}

int launch_batch_ace(const BatchTable& t, int dev, cudaStream_t s) {
    if (t.nctx < 1 || t.nctx > kMaxBatchCtx) return 0;
    static int configured = -1;
    if (configured != dev) {
        cudaFuncSetAttribute(kb_ace_contract, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ace_tc_smem_bytes());
        configured = dev;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    launch_pdl(kb_ace_basis, ace_grid(persistent_blocks(kb_ace_basis, dev, 256, 0), t.atoms, 8), 256, 0, s, t);
    launch_pdl(kb_ace_contract, ace_grid(nsm, t.atoms, kTcWarps), kTcWarps * 32, ace_tc_smem_bytes(), s, t);
    launch_pdl(kb_ace_force, ace_grid(persistent_blocks(kb_ace_force, dev, 256, 0), t.atoms, 8), 256, 0, s, t);
    return 3;
}

int launch_ace_force(Ctx& c, cudaStream_t s) {
    const int nb = ace_grid(persistent_blocks(k_ace_force, c.dev, 256, 0), c.n, 8);
    launch_pdl(k_ace_force, nb, 256, 0, s, c.pos4, c.nbr_row, c.cap, c.nnbr, c.n, c.D, c.grid.ncode, c.ace_tc_d, c.ace_list, c.w,
               c.flags, c.ace_dA, c.vir_ace, c.acc);
    return 1;
}


}  // namespace ap

// =====================================================================================
// Allocation-free variant: ACE forces for environments the caller supplies.
//
// Some callers of this library cannot create device allocations of their own: a host
// program or plugin whose GPU memory is owned entirely by another allocator (a
// framework's caching pool that must see every byte), or a time-critical step loop that
// forbids the latency and the failure modes of cudaMalloc after start-up.  For them
// ap_ace_forces_noalloc evaluates the ACE pass (the same per-atom device functions as the
// context path) on neighbour lists they pass in, and keeps its scratch - the coefficient
// tables and the 64-bit fixed-point force accumulators - in the file-scope array below,
// which every GPU that loads this library holds until the process exits.
// =====================================================================================
namespace ap {

namespace {

constexpr int kNoAllocMaxAtoms = 65536;
constexpr size_t kNoAllocTableBytes = (sizeof(AceTc) + 255) / 256 * 256;
constexpr size_t kNoAllocBytes = kNoAllocTableBytes + 3 * (size_t)kNoAllocMaxAtoms * sizeof(unsigned long long);

}  // namespace

}  // namespace ap

// ~1.7 MB: the coefficient tables, then accumulators for up to 65,536 atoms.  In host
// code this name is only a stand-in; kernels receive its device address, obtained once
// per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_ace_noalloc_scratch[ap::kNoAllocBytes];

namespace ap {

namespace {

constexpr int kNaWarps = 8;

struct NoallocWarpSmem {
    TcWarpSmem tc;
    float4 nb[kAceNbrCap];
    int nbj[kAceNbrCap];
    float tileY[kTile][kNLM];
    float tileG[kTile][kNmax];
    float dAT[kNLM][kNmax];
};
static_assert(sizeof(NoallocWarpSmem) % 16 == 0, "16-byte aligned warp regions");

size_t noalloc_smem_bytes() { return sizeof(AceTc) + kNaWarps * sizeof(NoallocWarpSmem); }

__global__ void __launch_bounds__(kNaWarps * 32, 1)
k_ace_noalloc(const int* __restrict__ nbr_idx, const float* __restrict__ rvec, int n, int max_nb,
              const float* __restrict__ wv, unsigned char* __restrict__ scratch, double* __restrict__ e_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AceTc& C = *reinterpret_cast<AceTc*>(smem_raw);
    NoallocWarpSmem* WS = reinterpret_cast<NoallocWarpSmem*>(smem_raw + sizeof(AceTc));
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(scratch + kNoAllocTableBytes);
    {
        const int4* src = reinterpret_cast<const int4*>(scratch);
        int4* dst = reinterpret_cast<int4*>(smem_raw);
        for (int k = threadIdx.x; k < (int)(sizeof(AceTc) / 16); k += blockDim.x) dst[k] = src[k];
        float4* z = reinterpret_cast<float4*>(WS);
        for (int k = threadIdx.x; k < (int)(kNaWarps * sizeof(NoallocWarpSmem) / 16); k += blockDim.x)
            z[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    NoallocWarpSmem& S = WS[warp];
    const float rc = C.rc, rc2 = rc * rc, nrefi = C.nref_inv;
    const int lam_pad = lane_lm_pad(lane);
    for (int i = blockIdx.x * kNaWarps + warp; i < n; i += gridDim.x * kNaWarps) {
        const float wi = wv ? wv[i] : 1.0f;
        if (!(wi > 0.0f)) {
            if (lane == 0) e_out[i] = 0.0;
            continue;
        }
        // neighbours inside the cutoff; S.nbj keeps the atom index (max_nb <= kAceNbrCap)
        int cnt = 0;
        for (int k0 = 0; k0 < max_nb; k0 += 32) {
            const int k = k0 + lane;
            bool in = false;
            float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
            int j = -1;
            if (k < max_nb) {
                j = nbr_idx[(size_t)i * max_nb + k];
                if (j >= 0 && j < n) {
                    const float* v = rvec + 3 * ((size_t)i * max_nb + k);
                    dx = v[0]; dy = v[1]; dz = v[2];
                    r2 = dx * dx + dy * dy + dz * dz;
                    in = r2 < rc2 && r2 > 0.0f;
                }
            }
            const unsigned bm = __ballot_sync(0xffffffffu, in);
            const int pos = cnt + __popc(bm & ((1u << lane) - 1u));
            if (in) { S.nb[pos] = make_float4(dx, dy, dz, sqrtf(r2)); S.nbj[pos] = j; }
            cnt += __popc(bm);
        }
        __syncwarp();
        float accA[kNmax];
#pragma unroll
        for (int q = 0; q < kNmax; ++q) accA[q] = 0.0f;
        for (int t0 = 0; t0 < cnt; t0 += kTile) {
            basis_tile(S.nb, t0, cnt, rc, S.tileY, S.tileG, lane);
            __syncwarp();
            basis_accum_fp32(S.tileY, S.tileG, min(kTile, cnt - t0), lane, accA);
            __syncwarp();
        }
        tc_load_atom(S.tc, lane, lam_pad, make_float4(accA[0] * nrefi, accA[1] * nrefi, accA[2] * nrefi, accA[3] * nrefi),
                     make_float4(accA[4] * nrefi, accA[5] * nrefi, accA[6] * nrefi, accA[7] * nrefi));
        float e = 0.0f;
        if (!tc_contract_atom(C, S.tc, lane, e)) {
            if (lane == 0) e_out[i] = __longlong_as_double(0x7ff8000000000000ll);
            continue;
        }
        if (lane < kNLM) {
#pragma unroll
            for (int q = 0; q < kNmax; ++q) S.dAT[lane][q] = S.tc.dA[q * kApad + lam_pad];
        }
        __syncwarp();
        float fsx = 0.f, fsy = 0.f, fsz = 0.f;
        for (int t0 = 0; t0 < cnt; t0 += 32) {
            const int jj = t0 + lane;
            if (jj < cnt) {
                const int j = S.nbj[jj];
                const float3 fp = ace_pair_force(S.nb[jj], rc, nrefi, wi, S.dAT);
                fix_add(&acc[j], -fp.x);
                fix_add(&acc[(size_t)n + j], -fp.y);
                fix_add(&acc[(size_t)2 * n + j], -fp.z);
                fsx += fp.x; fsy += fp.y; fsz += fp.z;
            }
        }
        fsx = warp_sum(fsx); fsy = warp_sum(fsy); fsz = warp_sum(fsz);
        if (lane == 0) {
            fix_add(&acc[i], fsx);
            fix_add(&acc[(size_t)n + i], fsy);
            fix_add(&acc[(size_t)2 * n + i], fsz);
            e_out[i] = (double)C.c1_0 + (double)e;
        }
        __syncwarp();
    }
}

__global__ void k_ace_noalloc_forces(const unsigned char* __restrict__ scratch, int n, float* __restrict__ f_out) {
    const unsigned long long* acc = reinterpret_cast<const unsigned long long*>(scratch + kNoAllocTableBytes);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < 3; ++k)
        f_out[3 * (size_t)i + k] = (float)((double)(long long)acc[(size_t)k * n + i] * (1.0 / kFixScale));
}

std::mutex g_noalloc_mu;
struct NoallocDevice {
    void* scratch = nullptr;             // device address of the scratch array on this device
    unsigned long long key = 0;          // content hash of the potential whose tables it holds
    bool tables = false;
};
NoallocDevice g_noalloc_dev[64];
AceDev g_noalloc_dev_tables;             // host staging of the tables (guarded by the mutex)
AceTc g_noalloc_tables;

// FNV-1a over the bytes that define the ACE tables of a potential
unsigned long long potential_key(const ap_potential& p) {
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](const void* d, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(d);
        for (size_t k = 0; k < n; ++k) { h ^= b[k]; h *= 1099511628211ull; }
    };
    mix(&p.ace_rc, sizeof(double));
    mix(&p.ace_nref, sizeof(double));
    mix(&p.ace_nmax, sizeof(int));
    mix(&p.ace_lmax, sizeof(int));
    mix(&p.ace_nfunc, sizeof(int));
    mix(&p.ace_c1_0, sizeof(double));
    mix(&p.ace_c2_0, sizeof(double));
    if (p.ace_nfunc > 0 && p.ace_idx && p.ace_c1 && p.ace_c2) {
        mix(p.ace_idx, sizeof(int) * 7 * (size_t)p.ace_nfunc);
        mix(p.ace_c1, sizeof(double) * (size_t)p.ace_nfunc);
        mix(p.ace_c2, sizeof(double) * (size_t)p.ace_nfunc);
    }
    return h;
}

ap_status noalloc_fail(ap_status st, const std::string& m) {
    set_global_error(m);
    return st;
}

}  // namespace

}  // namespace ap

extern "C" ap_status ap_ace_forces_noalloc(const ap_potential* pot, int n_atoms, int max_nb, const int* d_nbr_idx,
                                           const float* d_rvec, const float* d_w, float* d_force, double* d_energy,
                                           void* stream) {
    using namespace ap;
    if (!pot || !d_nbr_idx || !d_rvec || !d_force || !d_energy || n_atoms < 1 || max_nb < 0)
        return noalloc_fail(AP_ERR_ARG, "ap_ace_forces_noalloc: missing argument, n_atoms < 1 or max_nb < 0");
    if (n_atoms > kNoAllocMaxAtoms || max_nb > kAceNbrCap)
        return noalloc_fail(AP_ERR_ARG, "ap_ace_forces_noalloc: at most 65536 atoms and 128 neighbour slots per atom");
    if (pot->ace_precision != AP_ACE_FP32)
        return noalloc_fail(AP_ERR_ARG, "ap_ace_forces_noalloc: only ace_precision = AP_ACE_FP32 is built");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return noalloc_fail(AP_ERR_CUDA, "ap_ace_forces_noalloc: no current CUDA device");
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    NoallocDevice& D = g_noalloc_dev[dev];
    const unsigned long long key = potential_key(*pot);
    if (!D.scratch || !D.tables || D.key != key) {
        // the set-up and the table upload are synchronous or read pageable host memory, which
        // a stream capture would record or reject: refuse them while `stream` is capturing
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
            (void)cudaGetLastError();
            cs = cudaStreamCaptureStatusActive;
        }
        if (cs != cudaStreamCaptureStatusNone)
            return noalloc_fail(AP_ERR_STATE, "ap_ace_forces_noalloc: the first call on a device and the first call "
                                              "with a new potential upload tables and cannot run under stream capture");
    }
    if (!D.scratch) {
        // once per device, with that device current (the first call on a device does this)
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_ace_noalloc_scratch) != cudaSuccess || !p)
            return noalloc_fail(AP_ERR_CUDA, "ap_ace_forces_noalloc: cudaGetSymbolAddress failed for the scratch array");
        static float gv[kNG];
        std::string err;
        if (gaunt_values(gv, err)) return noalloc_fail(AP_ERR_ARG, err);
        upload_gaunt(gv);
        if (cudaFuncSetAttribute(k_ace_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)noalloc_smem_bytes()) !=
            cudaSuccess)
            return noalloc_fail(AP_ERR_CUDA, "ap_ace_forces_noalloc: cudaFuncSetAttribute failed");
        D.scratch = p;
    }
    unsigned char* scratch = static_cast<unsigned char*>(D.scratch);
    cudaError_t e = cudaSuccess;
    // the coefficient tables are built and uploaded when the potential differs from the one
    // whose tables the array holds (the first call on a device, or a new potential)
    if (!D.tables || D.key != key) {
        std::string err;
        if (build_ace_tables(*pot, g_noalloc_dev_tables, err)) return noalloc_fail(AP_ERR_ARG, err);
        build_ace_tc(g_noalloc_dev_tables, g_noalloc_tables);
        D.tables = false;
        // pageable source: the call returns once the host buffer has been read, and the copy
        // is ordered on `stream` after the previous call's kernels there
        e = cudaMemcpyAsync(scratch, &g_noalloc_tables, sizeof(AceTc), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return noalloc_fail(AP_ERR_CUDA, std::string("ap_ace_forces_noalloc: ") + cudaGetErrorString(e));
        D.tables = true;
        D.key = key;
    }
    // the accumulators must start at zero; the array keeps whatever the last call left
    e = cudaMemsetAsync(scratch + kNoAllocTableBytes, 0, 3 * (size_t)n_atoms * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return noalloc_fail(AP_ERR_CUDA, std::string("ap_ace_forces_noalloc: ") + cudaGetErrorString(e));
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    k_ace_noalloc<<<nsm, kNaWarps * 32, noalloc_smem_bytes(), s>>>(d_nbr_idx, d_rvec, n_atoms, max_nb, d_w, scratch, d_energy);
    k_ace_noalloc_forces<<<(n_atoms + 255) / 256, 256, 0, s>>>(scratch, n_atoms, d_force);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(AP_ERR_CUDA, std::string("ap_ace_forces_noalloc: ") + cudaGetErrorString(e));
    return AP_OK;
}
