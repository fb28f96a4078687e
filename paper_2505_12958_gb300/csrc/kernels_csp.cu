// kernels_csp.cu -- the centro-symmetry parameter (CSP) and the switching weights it drives
// (Sec. 2.2.3; the switching function of Appendix B and its parameters).
//
// CSP_i: of the n_nb nearest neighbours of atom i within rc (n_nb = 12 for FCC, 14 for BCC,
// the first two BCC shells), every pair (j, k) gives |R_j + R_k|^2, and CSP_i is the sum of
// the n_nb/2 smallest.  Fewer than n_nb neighbours within rc marks a surface atom (-1).
// One thread per atom reads the full neighbour list; the n_nb nearest and the n_nb/2
// smallest pair sums are kept in registers by fully unrolled insertion.
//
// Weights (readings, the map itself is in the cited AP work): block averages of CSP give
// w0 = clamp((CSP - CSP_lo)/(CSP_hi - CSP_lo), 0, 1); atoms of the precise zone (the
// hemisphere under the tip) have w0 = 1; surface atoms outside it w0 = 0.  Every atom with
// w0 > 0 seeds w_i = max_j w0_j T(|r_ij|), T = 1 up to r_lo and cos^2 down to 0 at r_hi,
// and a new w_i replaces the old one only when it differs by at least dlam_min.
#include <cfloat>

#include "ap_internal.h"
#include "geom.cuh"

namespace ap {

namespace {

constexpr int kCspBlock = 128;

template <int NNB>
__global__ void __launch_bounds__(kCspBlock) k_csp(const float4* __restrict__ pos4, const int* __restrict__ nbr,
                                                   const int* __restrict__ nnbr, int n, const float4* __restrict__ Dtab,
                                                   int ncode, float rc2, float* __restrict__ csp,
                                                   double* __restrict__ sum, int* __restrict__ under) {
    __shared__ float4 Ds[125];
    for (int k = threadIdx.x; k < ncode; k += blockDim.x) Ds[k] = Dtab[k];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = pos4[i];
    float r2s[NNB], vx[NNB], vy[NNB], vz[NNB];
#pragma unroll
    for (int k = 0; k < NNB; ++k) { r2s[k] = FLT_MAX; vx[k] = vy[k] = vz[k] = 0.0f; }
    int cnt = 0;
    const int m = nnbr[i];
    for (int k = 0; k < m; ++k) {
        const int e = nbr[(size_t)k * n + i];
        const float4 d = Ds[(unsigned)e >> kNbrShift];
        const float4 q = pos4[e & kNbrMask];
        float x = q.x + d.x - p.x, y = q.y + d.y - p.y, z = q.z + d.z - p.z;
        float r2 = x * x + y * y + z * z;
        if (!(r2 < rc2)) continue;
        ++cnt;
        // insert into the sorted n_nb nearest (the largest falls off the end)
#pragma unroll
        for (int s = 0; s < NNB; ++s) {
            const bool sw = r2 < r2s[s];
            const float t2 = r2s[s], tx = vx[s], ty = vy[s], tz = vz[s];
            r2s[s] = sw ? r2 : t2; vx[s] = sw ? x : tx; vy[s] = sw ? y : ty; vz[s] = sw ? z : tz;
            r2 = sw ? t2 : r2; x = sw ? tx : x; y = sw ? ty : y; z = sw ? tz : z;
        }
    }
    float c = -1.0f;
    if (cnt >= NNB) {
        constexpr int H = NNB / 2;
        float best[H];
#pragma unroll
        for (int s = 0; s < H; ++s) best[s] = FLT_MAX;
#pragma unroll
        for (int a = 0; a < NNB; ++a)
#pragma unroll
            for (int b = a + 1; b < NNB; ++b) {
                const float sx = vx[a] + vx[b], sy = vy[a] + vy[b], sz = vz[a] + vz[b];
                float v = fmaf(sx, sx, fmaf(sy, sy, sz * sz));
#pragma unroll
                for (int s = 0; s < H; ++s) {
                    const float t = best[s];
                    best[s] = fminf(t, v);
                    v = fmaxf(t, v);
                }
            }
        c = 0.0f;
#pragma unroll
        for (int s = 0; s < H; ++s) c += best[s];
    }
    if (csp) csp[i] = c;
    if (c < 0.0f) under[i] += 1;
    else sum[i] += (double)c;
}

// w0 from the block averages, the precise zone and the surface rule; seeds (w0 > 0) are
// compacted; the accumulators are cleared for the next block
__global__ void k_csp_w0(const double* __restrict__ x, int n, const GridDev g, const ap_csp_params P, int nacc,
                         double* __restrict__ sum, int* __restrict__ under, float* __restrict__ w0,
                         float* __restrict__ wnew, int* __restrict__ seeds, int* __restrict__ nseed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float v = 0.0f;
    if (i < n) {
        const int u = under[i];
        double d[3] = {x[i] - P.zone_center[0], x[n + i] - P.zone_center[1], x[2 * n + i] - P.zone_center[2]};
        min_image_vec(g, d);
        const bool zone = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < P.zone_r * P.zone_r;
        if (zone) {
            v = 1.0f;
        } else if (2 * u > nacc || u == nacc) {
            v = 0.0f;                                      // surface atom outside the zone
        } else {
            const double avg = sum[i] / (double)(nacc - u);
            const double t = (avg - P.csp_lo) / (P.csp_hi - P.csp_lo);
            v = (float)(t <= 0.0 ? 0.0 : (t >= 1.0 ? 1.0 : t));
        }
        w0[i] = v;
        wnew[i] = v;
        sum[i] = 0.0;
        under[i] = 0;
    }
    const bool seed = (i < n) && v > 0.0f;
    const unsigned mask = __ballot_sync(0xffffffffu, seed);
    if (mask) {
        const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(nseed, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (seed) seeds[base + __popc(mask & ((1u << lane) - 1u))] = i;
    }
}

// w_i = max over seeds j of w0_j T(|r_ij|): one thread per seed visits the cells within
// r_hi (offsets -S..S per edge, every periodic image) and raises w_i with an atomic max
// on the bits of a non-negative float
__global__ void k_csp_spread(const float4* __restrict__ pos4, const int* __restrict__ cell,
                             const int* __restrict__ cell_start, const int* __restrict__ cell_atoms, const GridDev g,
                             int S0, int S1, int S2, float rlo, float rhi, const float* __restrict__ w0,
                             const int* __restrict__ seeds, const int* __restrict__ nseed, float* __restrict__ wnew) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= *nseed) return;
    const int j = seeds[s];
    const float wj = w0[j];
    const float4 pj = pos4[j];
    const int cj = cell[j];
    int cc[3];
    cc[2] = cj % g.nc[2];
    cc[1] = (cj / g.nc[2]) % g.nc[1];
    cc[0] = cj / (g.nc[2] * g.nc[1]);
    const float rhi2 = rhi * rhi, inv = 1.0f / (rhi - rlo);
    const int S[3] = {S0, S1, S2};
    for (int o0 = -S[0]; o0 <= S[0]; ++o0)
        for (int o1 = -S[1]; o1 <= S[1]; ++o1)
            for (int o2 = -S[2]; o2 <= S[2]; ++o2) {
                const int o[3] = {o0, o1, o2};
                int nc[3];
                bool ok = true;
                for (int k = 0; k < 3; ++k) {
                    int v = cc[k] + o[k];
                    if (g.periodic[k]) {
                        v %= g.nc[k];
                        if (v < 0) v += g.nc[k];
                    } else if (v < 0 || v >= g.nc[k]) {
                        ok = false;
                    }
                    nc[k] = v;
                }
                if (!ok) continue;
                // the neighbour cell's origin relative to j's cell origin, in FP32
                float ox = 0.f, oy = 0.f, oz = 0.f;
                for (int k = 0; k < 3; ++k) {
                    ox += (float)(o[k] * g.cellvec[3 * k + 0]);
                    oy += (float)(o[k] * g.cellvec[3 * k + 1]);
                    oz += (float)(o[k] * g.cellvec[3 * k + 2]);
                }
                const int cn = (nc[0] * g.nc[1] + nc[1]) * g.nc[2] + nc[2];
                for (int q = cell_start[cn], e = cell_start[cn + 1]; q < e; ++q) {
                    const int i = cell_atoms[q];
                    const float4 pi = pos4[i];
                    const float dx = pi.x + ox - pj.x, dy = pi.y + oy - pj.y, dz = pi.z + oz - pj.z;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    if (!(r2 < rhi2)) continue;
                    float t = 1.0f;
                    const float r = sqrtf(r2);
                    if (r > rlo) {
                        const float c = cospif(0.5f * (r - rlo) * inv);   // cos^2 form of the cosine switch
                        t = c * c;
                    }
                    const float v = wj * t;
                    if (v > 0.0f) atomicMax(reinterpret_cast<int*>(&wnew[i]), __float_as_int(v));
                }
            }
}

// replace w_i by the new weight when it moved by at least dlam_min
__global__ void k_csp_final(int n, const float* __restrict__ wnew, double dlam_min, double* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = (double)wnew[i];
    if (fabs(v - w[i]) >= dlam_min) w[i] = v;
}

}  // namespace

int launch_csp(Ctx& c, cudaStream_t s, const ap_csp_params& P, float* d_csp) {
    const int nb = (c.n + kCspBlock - 1) / kCspBlock;
    const float rc2 = (float)(P.rc * P.rc);
    if (P.n_nb == 12)
        k_csp<12><<<nb, kCspBlock, 0, s>>>(c.pos4, c.nbr, c.nnbr, c.n, c.D, c.grid.ncode, rc2, d_csp, c.csp_sum, c.csp_under);
    else
        k_csp<14><<<nb, kCspBlock, 0, s>>>(c.pos4, c.nbr, c.nnbr, c.n, c.D, c.grid.ncode, rc2, d_csp, c.csp_sum, c.csp_under);
    return 1;
}

int launch_csp_weights(Ctx& c, cudaStream_t s, const ap_csp_params& P, int nacc, const int S[3]) {
    const int nb = (c.n + 255) / 256;
    cudaMemsetAsync(c.csp_nseed, 0, sizeof(int), s);
    k_csp_w0<<<nb, 256, 0, s>>>(c.x, c.n, c.grid, P, nacc, c.csp_sum, c.csp_under, c.csp_w0, c.csp_wnew, c.csp_seeds,
                                c.csp_nseed);
    k_csp_spread<<<nb, 256, 0, s>>>(c.pos4, c.cell, c.cell_start, c.cell_atoms, c.grid, S[0], S[1], S[2], (float)P.r_lo,
                                    (float)P.r_hi, c.csp_w0, c.csp_seeds, c.csp_nseed, c.csp_wnew);
    k_csp_final<<<nb, 256, 0, s>>>(c.n, c.csp_wnew, P.dlam_min, c.w_fixed);
    return 3;
}

}  // namespace ap
