// geom.cuh -- distances to the fixed-zone centre and to the indenter, and the weight switch.
//
// FP64 is kept to the few operations whose rounding would show (the difference of absolute
// coordinates, its square, and d^2 - r_in^2); the switch itself is evaluated in FP32 from an
// argument formed as (d^2 - r_in^2) / (d + r_in), so w carries FP32 relative precision.
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

// cosine switch S(d) = 1 (d < r_in), (1 + cos(pi (d - r_in)/r_sw))/2, 0 (d >= r_in + r_sw),
// from d2 = d^2; *dS receives dS/dd (0 outside the shell)
__device__ __forceinline__ float switch_weight(double d2, double r_in, double r_sw, float* dS) {
    *dS = 0.0f;
    if (d2 < r_in * r_in) return 1.0f;
    const double ro = r_in + r_sw;
    if (d2 >= ro * ro) return 0.0f;
    const float dist = sqrtf((float)d2);
    const float x = (float)((d2 - r_in * r_in) / ((double)dist + r_in) / r_sw);   // (d - r_in)/r_sw
    float sn, cs;
    sincospif(x, &sn, &cs);
    *dS = -0.5f * 3.14159265358979f / (float)r_sw * sn;
    return 0.5f * (1.0f + cs);
}

}  // namespace ap
