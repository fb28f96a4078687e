// kernels_eam.cu -- EAM pass of the AP force evaluation (Sec. 2.2.1, Eq. energy_eam).
//
// With u_i = 1 - w_i the EAM share of the energy is sum_i u_i [xi(rho_i) + Delta xi +
// 1/2 sum_j Phi(r_ij)], rho_i = sum_j zeta(r_ij).  Its negative gradient on atom i is
//   F_i = sum_j [ (u_i xi'(rho_i) + u_j xi'(rho_j)) zeta'(r_ij) + (u_i + u_j)/2 Phi'(r_ij) ] rhat_ij,
// evaluated from i's side over the full list, so no atomics are needed and the sum
// order is fixed.  Per step two passes: density (rho, xi, u xi' per atom), then forces.
// On request a third pass gives accurate per-atom energies and the per-atom virial
// -1/2 sum_j c_ij r_ij (x) rhat_ij.  The embedding function is evaluated in FP64 (one
// square root per atom); pair terms are FP32 piecewise polynomials from the host tables.
#include "ap_internal.h"
#include "eam_table.h"
#include "geom.cuh"

namespace ap {

namespace {

// list entries whose gathers are issued together per thread, and the block size of the
// thread-per-atom EAM kernels (tuning constants; results do not depend on them)
#ifndef AP_EAM_BATCH
#define AP_EAM_BATCH 4
#endif
#ifndef AP_EAM_BLOCK
#define AP_EAM_BLOCK 128
#endif
constexpr int kEamBatch = AP_EAM_BATCH;
constexpr int kEamBlock = AP_EAM_BLOCK;

__device__ __forceinline__ void stage_tables(EamDev* sm, const EamDev* __restrict__ gm, float4* Ds,
                                             const float4* __restrict__ D, int ncode) {
    const int4* src = reinterpret_cast<const int4*>(gm);
    int4* dst = reinterpret_cast<int4*>(sm);
    for (int k = threadIdx.x; k < (int)(sizeof(EamDev) / 16); k += blockDim.x) dst[k] = src[k];
    for (int k = threadIdx.x; k < ncode; k += blockDim.x) Ds[k] = D[k];
    __syncthreads();
}

// The image offset D[code] of a pair.  In an orthorhombic box it is (o0 cx, o1 cy, o2 cz) with
// cell offsets o in -2..2 and c the FP32 cell edges: those products are exact, and equal the
// host table's FP32 entries, so a 4-byte offset record replaces the 16-byte table read.
struct PairOffsets {
    char4 o[125];
    float cx, cy, cz;
    int ortho;
};

__device__ __forceinline__ void stage_offsets(PairOffsets& P, const GridDev& g) {
    const int w1 = 2 * g.S[1] + 1, w2 = 2 * g.S[2] + 1;
    for (int k = threadIdx.x; k < g.ncode; k += blockDim.x)
        P.o[k] = make_char4((char)(k / (w1 * w2) - g.S[0]), (char)((k / w2) % w1 - g.S[1]), (char)(k % w2 - g.S[2]), 0);
    if (threadIdx.x == 0) {
        P.cx = (float)g.cellvec[0];
        P.cy = (float)g.cellvec[4];
        P.cz = (float)g.cellvec[8];
        P.ortho = g.ortho;
    }
}

__device__ __forceinline__ float4 pair_offset(const PairOffsets& P, const float4* Ds, int code) {
    if (P.ortho) {
        const char4 o = P.o[code];
        return make_float4((float)o.x * P.cx, (float)o.y * P.cy, (float)o.z * P.cz, 0.0f);
    }
    return Ds[code];
}

// ---------------------------------------------------------------------------------
// On-demand EAM energies with compensated FP32 arithmetic.  Plain FP32 pair distances
// and polynomials are accurate to a few ulp, but in a perfect lattice every equivalent
// atom repeats the same rounding and the per-atom energies are off coherently by
// ~1e-6 eV.  Here every pair vector is an error-free double-float sum (TwoSum) of the
// cell-relative positions, their FP32 residuals and the offset table with its residuals;
// r = sqrt(r2) carries a first-order correction, and each polynomial is evaluated as
// p(t_hi) + p'(t_hi) t_lo with t_hi = r_f - mid exact in FP32.  Sums are compensated too.
// Only FP32 instructions run per pair (GB300's FP64 rate is 1/64 of its FP32 rate).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void acc_add(float& hi, float& lo, float v) {
    float s, e;
    two_sum(hi, v, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
}

// zeta and Phi at rf + tl (FP32 rf, first-order correction tl), each added into its
// double-float sum: the constant terms enter as c0 (hi + lo) through TwoSum, the rest in FP32
__device__ __forceinline__ void pair_acc_df(const EamDev& T, float rf, float tl, bool with_z, float& zh, float& zl,
                                            float& ph, float& pl) {
    int sp;
    const int k = eam_seg(T, rf, sp);
    const EamSeg& g = T.seg[k];
    const float4 q0 = g.q0, q1 = g.q1, q2 = g.q2;
    const float x = __fsub_rn(rf, q0.x);            // exact: mid is an FP32 number near rf
    if (with_z) {
        const float u = fmaf(fmaf(q0.w, x, q0.z), x, q0.y);
        const float d = fmaf(fmaf(3.0f * q0.w, x, 2.0f * q0.z), x, q0.y);
        const float xu = __fmul_rn(x, u), xue = fmaf(x, u, -xu);
        acc_add(zh, zl, q2.x);
        acc_add(zh, zl, xu);
        zl = __fadd_rn(zl, __fadd_rn(__fadd_rn(q2.y, xue), d * tl));
    }
    float c4 = 0.0f, c5 = 0.0f;
    if (sp) {
        const int kind = (int)q2.w;
        if (kind == kSegZbl) {
            const float r = rf + tl, xr = r * T.zbl_ainv;
            acc_add(ph, pl, T.zbl_k * (0.1818f * expf(-3.2f * xr) + 0.5099f * expf(-0.9423f * xr) +
                                       0.2802f * expf(-0.4029f * xr) + 0.02817f * expf(-0.2016f * xr)) / r);
            return;
        }
        if (kind == kSegQuintic) { c4 = g.q3.x; c5 = g.q3.y; }
    }
    const float u = fmaf(fmaf(fmaf(fmaf(c5, x, c4), x, q1.z), x, q1.y), x, q1.x);
    const float d = fmaf(fmaf(fmaf(fmaf(5.0f * c5, x, 4.0f * c4), x, 3.0f * q1.z), x, 2.0f * q1.y), x, q1.x);
    const float xu = __fmul_rn(x, u), xue = fmaf(x, u, -xu);
    acc_add(ph, pl, q1.w);
    acc_add(ph, pl, xu);
    pl = __fadd_rn(pl, __fadd_rn(__fadd_rn(q2.z, xue), d * tl));
}


// the pair vector d + dlo of the energy pass as an error-free sum of the cell-relative
// positions, their FP32 residuals and the image offset (dh, dl); r2 = |d + dlo|^2 as a
// double-float (r2h, r2l)
__device__ __forceinline__ void pair_vec_df(const float4& p, const float4& pl, const float4& q, const float4& ql,
                                            const float4& dh, const float4& dl, float* d, float& r2h, float& r2l) {
    float dlo[3];
    const float qa[3] = {q.x, q.y, q.z}, pa[3] = {p.x, p.y, p.z};
    const float qla[3] = {ql.x, ql.y, ql.z}, pla[3] = {pl.x, pl.y, pl.z};
    const float dha[3] = {dh.x, dh.y, dh.z}, dla[3] = {dl.x, dl.y, dl.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float s1, e1, s2, e2;
        two_sum(qa[c], -pa[c], s1, e1);
        two_sum(s1, dha[c], s2, e2);
        d[c] = s2;
        dlo[c] = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fsub_rn(qla[c], pla[c]), dla[c]));
    }
    r2h = 0.f;
    r2l = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float sq = __fmul_rn(d[c], d[c]);
        const float sqe = fmaf(d[c], d[c], -sq);
        acc_add(r2h, r2l, sq);
        r2l = __fadd_rn(r2l, fmaf(2.0f * d[c], dlo[c], sqe));
    }
}

// one pair's zeta (inside its cutoff rcr) and Phi into the compensated sums, at rf = sqrt(r2h)
// with the first-order correction of r2l
__device__ __forceinline__ void pair_energy_df(const EamDev& T, float r2h, float r2l, float rf, float rcr, float& rh,
                                               float& rl, float& ph, float& pl) {
    const float pp = __fmul_rn(rf, rf), pe = fmaf(rf, rf, -pp);
    const float tl = __fdiv_rn(__fadd_rn(__fsub_rn(__fsub_rn(r2h, pp), pe), r2l), 2.0f * rf);
    pair_acc_df(T, rf, tl, rf < rcr, rh, rl, ph, pl);
}

// E_i^EAM = xi(rho_i) + Delta xi + 1/2 sum_j Phi(r_ij) from the compensated sums (FP64)
__device__ __forceinline__ double site_energy_df(const EamDev& T, float rh, float rl, float ph, float pl) {
    const double rho = (double)rh + (double)rl;
    double F = T.F_dxi;
    if (rho > 0.0) F += T.F_a1 * sqrt(rho) + T.F_a2 * rho * rho;
    return F + 0.5 * ((double)ph + (double)pl);
}

// ENERGY: the same pass also forms the compensated energy sums of the on-request energy
// pass (k_eam_energy without the virial) in its own gather loop, from the FP32 residuals
// pos_lo and Dlo, and writes E_i^EAM to e_acc: the arithmetic of that pass, pair by pair in
// list order, so the two give the same bits
template <bool ENERGY>
__device__ __forceinline__ void eam_density_body(const float4* __restrict__ pos4, const int* __restrict__ nbr,
                                                 const int* __restrict__ nnbr, int n, const EamDev* __restrict__ eam,
                                                 const float4* __restrict__ D, const GridDev& g,
                                                 float* __restrict__ uxi, double* __restrict__ e_emb,
                                                 int* __restrict__ flags, const float4* __restrict__ pos_lo,
                                                 const float4* __restrict__ Dlo, double* __restrict__ e_acc, int bid) {
    __shared__ EamDev T;
    __shared__ float4 Ds[125];
    __shared__ PairOffsets PO;
    __shared__ float4 Dl[ENERGY ? 125 : 1];
    stage_offsets(PO, g);
    if (ENERGY)
        for (int k = threadIdx.x; k < g.ncode; k += blockDim.x) Dl[k] = Dlo[k];
    stage_tables(&T, eam, Ds, D, g.ncode);        // constant tables: before the wait
    pdl_wait();
    int i = bid * blockDim.x + threadIdx.x;
    if (i == 0) flags[kFlagRebuild] = 0;        // the list built this step is in use now
    if (i >= n) return;
    float4 p = pos4[i];
    float u = p.w;
    if (u <= 0.0f) {
        uxi[i] = 0.0f;
        e_emb[i] = 0.0;
        if (ENERGY) e_acc[i] = 0.0;
        return;
    }
    const float rc2 = T.rc_rho * T.rc_rho;
    float rho = 0.0f;
    const float4 pl = ENERGY ? pos_lo[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float rcE2 = T.rc * T.rc, rcr = T.rc_rho;
    float rh = 0.f, rl = 0.f, ph = 0.f, pl_ = 0.f;
    const int m = nnbr[i];
    auto pair = [&](int e, const float4& q, const float4& ql) {
        const int code = (int)((unsigned)e >> kNbrShift);
        const float4 d = pair_offset(PO, Ds, code);
        const float dx = q.x + d.x - p.x, dy = q.y + d.y - p.y, dz = q.z + d.z - p.z;
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < rc2) rho += eam_zeta(T, sqrtf(r2));
        if (ENERGY) {
            float de[3], r2h, r2l;
            pair_vec_df(p, pl, q, ql, Ds[code], Dl[code], de, r2h, r2l);
            if (r2h >= rcE2) return;
            const float us = p.w + q.w;
            if (us <= 0.0f) return;
            pair_energy_df(T, r2h, r2l, sqrtf(r2h), rcr, rh, rl, ph, pl_);
        }
    };
    // four list entries at a time: their gathers are independent and overlap in flight
    int k = 0;
    for (; k + kEamBatch <= m; k += kEamBatch) {
        int e[kEamBatch];
        float4 q[kEamBatch], ql[kEamBatch];
#pragma unroll
        for (int b = 0; b < kEamBatch; ++b) e[b] = nbr[(size_t)(k + b) * n + i];
#pragma unroll
        for (int b = 0; b < kEamBatch; ++b) {
            q[b] = pos4[e[b] & kNbrMask];
            if (ENERGY) ql[b] = pos_lo[e[b] & kNbrMask];
        }
#pragma unroll
        for (int b = 0; b < kEamBatch; ++b) pair(e[b], q[b], ENERGY ? ql[b] : q[b]);
    }
    for (; k < m; ++k) {
        const int e = nbr[(size_t)k * n + i];
        const int j = e & kNbrMask;
        pair(e, pos4[j], ENERGY ? pos_lo[j] : pos4[j]);
    }
    double R = rho, F, dF;
    if (R > 0.0) {
        double sq = sqrt(R);
        F = T.F_a1 * sq + T.F_a2 * R * R + T.F_dxi;
        dF = 0.5 * T.F_a1 / sq + 2.0 * T.F_a2 * R;
    } else {
        F = T.F_dxi;
        dF = 0.0;
        if (R < 0.0 || !(R == R)) { atomicOr(&flags[kFlagErr], kErrDomain); flags[kFlagBad] = i; }
    }
    uxi[i] = (float)(u * dF);
    e_emb[i] = F;
    if (ENERGY) e_acc[i] = site_energy_df(T, rh, rl, ph, pl_);
}

template <bool ENERGY>
__global__ void __launch_bounds__(kEamBlock) k_eam_density(const float4* __restrict__ pos4, const int* __restrict__ nbr,
                                                     const int* __restrict__ nnbr, int n, const EamDev* __restrict__ eam,
                                                     const float4* __restrict__ D, const GridDev g, float* __restrict__ uxi,
                                                     double* __restrict__ e_emb, int* __restrict__ flags,
                                                     const float4* __restrict__ pos_lo, const float4* __restrict__ Dlo,
                                                     double* __restrict__ e_acc) {
    eam_density_body<ENERGY>(pos4, nbr, nnbr, n, eam, D, g, uxi, e_emb, flags, pos_lo, Dlo, e_acc, blockIdx.x);
}

// per step: EAM forces.  The pair value Phi is needed only for the FP32 estimate of E_i^EAM
// that the weight-gradient force of transition atoms (0 < w < 1) uses; exact energies and
// the virial come from the on-request energy pass.
__device__ __forceinline__ void eam_force_body(const float4* __restrict__ pos4, const int* __restrict__ nbr,
                                                   const int* __restrict__ nnbr, int n, const EamDev* __restrict__ eam,
                                                   const float4* __restrict__ D, const GridDev& g,
                                                   const float* __restrict__ uxi, const double* __restrict__ e_emb,
                                                   const float* __restrict__ wv, float* __restrict__ f,
                                                   double* __restrict__ e_eam, int bid) {
    __shared__ EamDev T;
    __shared__ float4 Ds[125];
    __shared__ PairOffsets PO;
    stage_offsets(PO, g);
    stage_tables(&T, eam, Ds, D, g.ncode);        // constant tables: before the wait
    pdl_wait();
    int i = bid * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = pos4[i];
    const float ui = p.w, xi = uxi[i];
    const float wi = wv[i];
    const bool want_e = wi > 0.0f && wi < 1.0f;   // the same test as the blend's weight-gradient term
    const float rc2 = T.rc * T.rc;
    float fx = 0.f, fy = 0.f, fz = 0.f, eph = 0.f;
    const int m = nnbr[i];
    auto pair = [&](int e, const float4& q, float xj) {
        const float4 d = pair_offset(PO, Ds, (int)((unsigned)e >> kNbrShift));
        const float dx = q.x + d.x - p.x, dy = q.y + d.y - p.y, dz = q.z + d.z - p.z;
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float us = ui + q.w;
        if (r2 >= rc2 || us <= 0.0f) return;   // beyond the cutoff, or both atoms fully ACE
        const float r = sqrtf(r2), ri = 1.0f / r;
        float dz_, dp, pf = 0.f;
        if (want_e) eam_pair_der<true>(T, r, dz_, dp, pf);
        else eam_pair_der<false>(T, r, dz_, dp, pf);
        const float cr = ((xi + xj) * dz_ + 0.5f * us * dp) * ri;
        fx += cr * dx; fy += cr * dy; fz += cr * dz;
        eph += pf;
    };
    int k = 0;
    for (; k + kEamBatch <= m; k += kEamBatch) {
        int e[kEamBatch];
        float4 q[kEamBatch];
        float xj[kEamBatch];
#pragma unroll
        for (int u = 0; u < kEamBatch; ++u) e[u] = nbr[(size_t)(k + u) * n + i];
#pragma unroll
        for (int u = 0; u < kEamBatch; ++u) {
            const int j = e[u] & kNbrMask;
            q[u] = pos4[j];
            xj[u] = uxi[j];
        }
#pragma unroll
        for (int u = 0; u < kEamBatch; ++u) pair(e[u], q[u], xj[u]);
    }
    for (; k < m; ++k) {
        const int e = nbr[(size_t)k * n + i];
        const int j = e & kNbrMask;
        pair(e, pos4[j], uxi[j]);
    }
    f[i] = fx; f[n + i] = fy; f[2 * n + i] = fz;
    if (want_e) e_eam[i] = e_emb[i] + 0.5 * (double)eph;
}

__global__ void __launch_bounds__(kEamBlock) k_eam_force(const float4* __restrict__ pos4, const int* __restrict__ nbr,
                                                   const int* __restrict__ nnbr, int n, const EamDev* __restrict__ eam,
                                                   const float4* __restrict__ D, const GridDev g, const float* __restrict__ uxi,
                                                   const double* __restrict__ e_emb, const float* __restrict__ wv,
                                                   float* __restrict__ f, double* __restrict__ e_eam) {
    eam_force_body(pos4, nbr, nnbr, n, eam, D, g, uxi, e_emb, wv, f, e_eam, blockIdx.x);
}

// the FP32 residual of x_rel for the energy pass: the FP64 difference x - cell origin that
// k_prepare rounded to FP32, minus that FP32 value
__global__ void k_pos_lo(const double* __restrict__ x, int n, const GridDev g, const int* __restrict__ cell,
                         const float4* __restrict__ pos4, float4* __restrict__ pos_lo) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cc[3];
    cell_coords(g, cell[i], cc);
    double o[3];
    cell_origin(g, cc, o);
    const float4 p = pos4[i];
    pos_lo[i] = make_float4((float)((x[i] - o[0]) - (double)p.x), (float)((x[n + i] - o[1]) - (double)p.y),
                            (float)((x[2 * (size_t)n + i] - o[2]) - (double)p.z), 0.0f);
}

template <bool VIR>
__global__ void __launch_bounds__(256) k_eam_energy(const float4* __restrict__ pos4, const float4* __restrict__ pos_lo,
                                                    const int* __restrict__ nbr, const int* __restrict__ nnbr, int n,
                                                    const EamDev* __restrict__ eam, const float4* __restrict__ D,
                                                    const float4* __restrict__ Dlo, int ncode,
                                                    const float* __restrict__ uxi, double* __restrict__ e_eam,
                                                    float* __restrict__ vir) {
    __shared__ EamDev T;
    __shared__ float4 Ds[125];
    __shared__ float4 Dl[125];
    stage_tables(&T, eam, Ds, D, ncode);
    for (int k = threadIdx.x; k < ncode; k += blockDim.x) Dl[k] = Dlo[k];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = pos4[i], pl = pos_lo[i];
    const float ui = p.w, xi = uxi[i];
    const bool own = ui > 0.0f;               // the atom has an EAM energy share
    const float rc2 = T.rc * T.rc, rcr = T.rc_rho;
    float rh = 0.f, rl = 0.f, ph = 0.f, pl_ = 0.f;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f, v4 = 0.f, v5 = 0.f;
    const int m = nnbr[i];
    auto pair = [&](int e, const float4& q, const float4& ql, float xj) {
        const unsigned code = (unsigned)e >> kNbrShift;
        float d[3], r2h, r2l;
        pair_vec_df(p, pl, q, ql, Ds[code], Dl[code], d, r2h, r2l);
        if (r2h >= rc2) return;
        const float us = ui + q.w;
        if (us <= 0.0f) return;
        const float rf = sqrtf(r2h);
        if (VIR) {
            // virial -1/2 c_ij r_ij (x) rhat_ij with the bond coefficient of the force pass
            float dz_, dp, pf;
            eam_pair_der<false>(T, rf, dz_, dp, pf);
            const float sc = -0.5f * ((xi + xj) * dz_ + 0.5f * us * dp) / rf;
            v0 += sc * d[0] * d[0]; v1 += sc * d[1] * d[1]; v2 += sc * d[2] * d[2];
            v3 += sc * d[0] * d[1]; v4 += sc * d[0] * d[2]; v5 += sc * d[1] * d[2];
        }
        if (!own) return;
        pair_energy_df(T, r2h, r2l, rf, rcr, rh, rl, ph, pl_);
    };
    // kEamBatch list entries at a time: their gathers are independent and overlap in flight
    // (the pairs are still added in list order)
    int k = 0;
    for (; k + kEamBatch <= m; k += kEamBatch) {
        int e[kEamBatch];
        float4 q[kEamBatch], ql[kEamBatch];
        float xj[kEamBatch];
#pragma unroll
        for (int b = 0; b < kEamBatch; ++b) e[b] = nbr[(size_t)(k + b) * n + i];
#pragma unroll
        for (int b = 0; b < kEamBatch; ++b) {
            const int j = e[b] & kNbrMask;
            q[b] = pos4[j];
            ql[b] = pos_lo[j];
            xj[b] = uxi[j];
        }
#pragma unroll
        for (int b = 0; b < kEamBatch; ++b) pair(e[b], q[b], ql[b], xj[b]);
    }
    for (; k < m; ++k) {
        const int e = nbr[(size_t)k * n + i];
        const int j = e & kNbrMask;
        pair(e, pos4[j], pos_lo[j], uxi[j]);
    }
    if (VIR) {
        vir[i] = v0; vir[n + i] = v1; vir[2 * n + i] = v2; vir[3 * n + i] = v3; vir[4 * n + i] = v4; vir[5 * n + i] = v5;
    }
    if (!own) { e_eam[i] = 0.0; return; }
    e_eam[i] = site_energy_df(T, rh, rl, ph, pl_);
}

__global__ void __launch_bounds__(kEamBlock) kb_eam_density(const BatchTable t) {
    const int k = batch_find(t.b128, t.nctx, blockIdx.x);
    const CtxDev& c = *t.d[k];
    eam_density_body<false>(c.pos4, c.nbr, c.nnbr, c.n, c.eam, c.D, c.grid, c.uxi, c.e_emb, c.flags, nullptr, nullptr,
                            nullptr, blockIdx.x - t.b128[k]);
}

__global__ void __launch_bounds__(kEamBlock) kb_eam_force(const BatchTable t) {
    const int k = batch_find(t.b128, t.nctx, blockIdx.x);
    const CtxDev& c = *t.d[k];
    eam_force_body(c.pos4, c.nbr, c.nnbr, c.n, c.eam, c.D, c.grid, c.uxi, c.e_emb, c.w, c.f, c.e_eam,
                   blockIdx.x - t.b128[k]);
}

}  // namespace

int launch_eam_energy(Ctx& c, cudaStream_t s, bool virial) {
    k_pos_lo<<<(c.n + 255) / 256, 256, 0, s>>>(c.x, c.n, c.grid, c.cell, c.pos4, c.pos_lo);
    if (virial)
        k_eam_energy<true><<<(c.n + 255) / 256, 256, 0, s>>>(c.pos4, c.pos_lo, c.nbr, c.nnbr, c.n, c.eam_d, c.D,
                                                             c.Dlo, c.grid.ncode, c.uxi, c.e_eam_acc, c.vir_eam);
    else
        k_eam_energy<false><<<(c.n + 255) / 256, 256, 0, s>>>(c.pos4, c.pos_lo, c.nbr, c.nnbr, c.n, c.eam_d, c.D,
                                                              c.Dlo, c.grid.ncode, c.uxi, c.e_eam_acc, c.vir_eam);
    return 2;
}

int launch_eam_density(Ctx& c, cudaStream_t s) {
    launch_pdl(k_eam_density<false>, (c.n + kEamBlock - 1) / kEamBlock, kEamBlock, 0, s, c.pos4, c.nbr, c.nnbr, c.n,
               c.eam_d, c.D, c.grid, c.uxi, c.e_emb, c.flags, (const float4*)nullptr, (const float4*)nullptr,
               (double*)nullptr);
    return 1;
}

int launch_eam_density_energy(Ctx& c, cudaStream_t s) {
    k_pos_lo<<<(c.n + 255) / 256, 256, 0, s>>>(c.x, c.n, c.grid, c.cell, c.pos4, c.pos_lo);
    launch_pdl(k_eam_density<true>, (c.n + kEamBlock - 1) / kEamBlock, kEamBlock, 0, s, c.pos4, c.nbr, c.nnbr, c.n,
               c.eam_d, c.D, c.grid, c.uxi, c.e_emb, c.flags, (const float4*)c.pos_lo, (const float4*)c.Dlo,
               c.e_eam_acc);
    return 2;
}

int launch_eam_force(Ctx& c, cudaStream_t s) {
    launch_pdl(k_eam_force, (c.n + kEamBlock - 1) / kEamBlock, kEamBlock, 0, s, c.pos4, c.nbr, c.nnbr, c.n, c.eam_d,
               c.D, c.grid, c.uxi, c.e_emb, c.w, c.f, c.e_eam);
    return 1;
}


int launch_batch_eam(const BatchTable& t, cudaStream_t s) {
    static_assert(kEamBlock == 128, "the batch table counts EAM blocks of 128 threads");
    launch_pdl(kb_eam_density, t.b128[t.nctx], kEamBlock, 0, s, t);
    launch_pdl(kb_eam_force, t.b128[t.nctx], kEamBlock, 0, s, t);
    return 2;
}

}  // namespace ap
