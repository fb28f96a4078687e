// geom.cuh -- cell coordinates and origins, distances to the fixed-zone centre and to the indenter, and the weight switch.
//
// FP64 is kept to the few operations whose rounding would show (the difference of absolute
// coordinates, its square, and the distances to the two shell radii); the switch itself is
// evaluated in FP32 from arguments formed as (d^2 - r^2) / (d + r), so w and 1 - w both carry
// FP32 relative precision.
#pragma once

#include "ap_internal.h"

namespace ap {

// nearest periodic image of the vector d (orthorhombic boxes: one rint per periodic edge)
__device__ __forceinline__ void min_image_vec(const GridDev& g, double* d) {
    if (g.ortho) {
        for (int k = 0; k < 3; ++k)
            if (g.periodic[k]) d[k] -= g.L[k] * rint(d[k] * g.Linv[k]);
        return;
    }
    double s[3];
    for (int k = 0; k < 3; ++k) s[k] = d[0] * g.hinv[k] + d[1] * g.hinv[3 + k] + d[2] * g.hinv[6 + k];
    for (int k = 0; k < 3; ++k)
        if (g.periodic[k]) {
            const double m = rint(s[k]);
            for (int q = 0; q < 3; ++q) d[q] -= m * g.h[3 * k + q];
        }
}

// integer coordinates of cell c (c = (c0 nc1 + c1) nc2 + c2)
__device__ __forceinline__ void cell_coords(const GridDev& g, int c, int* cc) {
    cc[2] = c % g.nc[2];
    int r = c / g.nc[2];
    cc[1] = r % g.nc[1];
    cc[0] = r / g.nc[1];
}

// origin of cell cc (FP64); x_rel = x - origin is what the force kernels see
__device__ __forceinline__ void cell_origin(const GridDev& g, const int* cc, double* o) {
    if (g.ortho) {
        for (int q = 0; q < 3; ++q) o[q] = g.origin[q] + cc[q] * g.cellvec[4 * q];
    } else {
        for (int q = 0; q < 3; ++q)
            o[q] = g.origin[q] + cc[0] * g.cellvec[q] + cc[1] * g.cellvec[3 + q] + cc[2] * g.cellvec[6 + q];
    }
}

// FP32 |d|^2 after the nearest-image shift of an FP32 vector (orthorhombic boxes; pre-tests)
__device__ __forceinline__ float min_image_d2_f32v(const GridDev& g, const float* d) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float x = d[k];
        if (g.periodic[k]) x = fmaf(-g.Lf[k], rintf(x * g.Linvf[k]), x);
        s = fmaf(x, x, s);
    }
    return s;
}

// FP32 estimate of |d|^2 after the nearest-image shift, orthorhombic boxes only (relative
// error below 1e-6 for the box sizes here); a pre-test that decides far-away atoms without
// FP64 arithmetic, which runs at 1/64 of the FP32 rate on this GPU
__device__ __forceinline__ float min_image_d2_f32(const GridDev& g, const double* d) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float x = (float)d[k];
        if (g.periodic[k]) x = fmaf(-g.Lf[k], rintf(x * g.Linvf[k]), x);
        s = fmaf(x, x, s);
    }
    return s;
}

// cosine switch S(d) = 1 (d < r_in), (1 + cos(pi a))/2 with a = (d - r_in)/r_sw, 0 (d >= r_in +
// r_sw), from d2 = d^2.  S is evaluated as cos^2(pi a/2) = sin^2(pi b/2), b = (r_in + r_sw - d)/r_sw,
// and 1 - S as sin^2(pi a/2): both keep FP32 relative precision at their small ends, so S > 0
// for every d < r_in + r_sw, the compaction rule.  a and b are formed as (d^2 - r^2) / ((d + r)
// r_sw): only the differences of squares, where cancellation would show, are taken in FP64
// (FP64 runs at 1/64 of the FP32 rate on this GPU); the square root and the quotients in
// FP32 keep FP32 relative precision.  *u receives 1 - S, *dS receives dS/dd.
__device__ __forceinline__ float switch_weight(double d2, double r_in, double r_sw, float* u, float* dS) {
    *dS = 0.0f;
    const double ri2 = r_in * r_in;
    if (d2 < ri2) { *u = 0.0f; return 1.0f; }
    const double ro = r_in + r_sw, ro2 = ro * ro;
    if (d2 >= ro2) { *u = 1.0f; return 0.0f; }
    const float dist = sqrtf((float)d2), rsw = (float)r_sw;
    const float a = (float)(d2 - ri2) / ((dist + (float)r_in) * rsw);   // (d - r_in)/r_sw
    const float b = (float)(ro2 - d2) / ((dist + (float)ro) * rsw);     // (r_in + r_sw - d)/r_sw
    const float sa = sinpif(0.5f * a), sb = sinpif(0.5f * b);
    *u = sa * sa;
    *dS = -3.14159265358979f / rsw * sa * sb;                          // -(pi/2r_sw) sin(pi a)
    return sb * sb;
}

}  // namespace ap
