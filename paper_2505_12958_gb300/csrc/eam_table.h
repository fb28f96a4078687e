// eam_table.h -- lookup and evaluation of the merged EAM pair table (EamDev), shared by
// the EAM kernels and by the host check that replays them (ap_eam_table_eval, which 2/3).
#pragma once

#include <cmath>

#include "ap_internal.h"

namespace ap {

// segment of r: one 16-byte bin record and two compares
__host__ __device__ __forceinline__ int eam_seg(const EamDev& T, float r, int& special) {
    int b = (int)(r * T.bin_inv);
    b = b < kNBin - 1 ? b : kNBin - 1;
    const EamBin e = T.bin[b];
    special = e.special;
    return e.k + (r >= e.s1 ? 1 : 0) + (r >= e.s2 ? 1 : 0);
}

// screened Coulomb Z^2/(4 pi eps0 r) phi(r/a), phi a sum of four exponentials, and its derivative
__host__ __device__ __forceinline__ void eam_zbl(float r, float zk, float zainv, float& f, float& df) {
    const float x = r * zainv;
    const float e0 = 0.1818f * expf(-3.2f * x), e1 = 0.5099f * expf(-0.9423f * x);
    const float e2 = 0.2802f * expf(-0.4029f * x), e3 = 0.02817f * expf(-0.2016f * x);
    const float ph = e0 + e1 + e2 + e3;
    const float dph = -(3.2f * e0 + 0.9423f * e1 + 0.4029f * e2 + 0.2016f * e3);
    const float ri = 1.0f / r;
    f = zk * ph * ri;
    df = zk * (dph * zainv * ri - ph * ri * ri);
}

// zeta(r)
__host__ __device__ __forceinline__ float eam_zeta(const EamDev& T, float r) {
    int sp;
    const int k = eam_seg(T, r, sp);
    const float4 q0 = T.seg[k].q0;
    const float x = r - q0.x;
    return fmaf(fmaf(fmaf(q0.w, x, q0.z), x, q0.y), x, T.seg[k].q2.x);
}

// zeta'(r), Phi'(r) and, with PHI_VAL, Phi(r)
template <bool PHI_VAL>
__host__ __device__ __forceinline__ void eam_pair_der(const EamDev& T, float r, float& dz, float& dp, float& pf) {
    int sp;
    const int k = eam_seg(T, r, sp);
    const float4 q0 = T.seg[k].q0, q1 = T.seg[k].q1;
    const float x = r - q0.x;
    dz = fmaf(fmaf(3.0f * q0.w, x, 2.0f * q0.z), x, q0.y);
    dp = fmaf(fmaf(3.0f * q1.z, x, 2.0f * q1.y), x, q1.x);
    if (PHI_VAL) pf = fmaf(fmaf(fmaf(q1.z, x, q1.y), x, q1.x), x, q1.w);
    if (sp) {
        const int kind = (int)T.seg[k].q2.w;
        if (kind == kSegZbl) {
            float f;
            eam_zbl(r, T.zbl_k, T.zbl_ainv, f, dp);
            if (PHI_VAL) pf = f;
        } else if (kind == kSegQuintic) {
            const float4 q3 = T.seg[k].q3;
            dp = fmaf(fmaf(fmaf(fmaf(5.0f * q3.y, x, 4.0f * q3.x), x, 3.0f * q1.z), x, 2.0f * q1.y), x, q1.x);
            if (PHI_VAL) pf = fmaf(fmaf(fmaf(fmaf(fmaf(q3.y, x, q3.x), x, q1.z), x, q1.y), x, q1.x), x, q1.w);
        }
    }
}

}  // namespace ap
