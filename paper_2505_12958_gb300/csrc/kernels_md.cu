// kernels_md.cu -- blend, indenter, reductions and velocity-Verlet integration.
//
// Blend (Sec. 2.2.3, Eq. energy_hyb with w = 1 - lambda): E_i = w_i E_i^ACE + (1 - w_i)
// E_i^EAM.  The EAM and ACE force shares already carry their weights; a position-
// dependent weight adds -grad w_i (E_i^ACE - E_i^EAM).  Indenter (Sec. 2.1, Eq.
// V_indenter): V = K/3 (R - d)^3 for d < R, F = K (R - d)^2 (r - c)/d; load (Sec. 3.1,
// Eq. P_ind) = sum F . dir.  Totals are summed per block in FP64 and then by one block
// in a fixed order, so they are reproducible run to run.
#include <cmath>
#include <cstdint>

#include "ap_internal.h"
#include "geom.cuh"

namespace ap {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kNP = 10;                     // e_pot, e_ind, vir[6], load, spare

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    return s;                               // valid on thread 0
}

// NV sums over a block of kRedBlock threads in a fixed order (each value added once: FP64
// adds run at 1/64 of the FP32 rate on this GPU, so no butterfly that repeats them on every
// lane); red holds NV * (kRedBlock + 1) doubles.  Thread k < NV returns sum k.
template <int NV>
__device__ __forceinline__ double block_sums(const double* v, double* red) {
    constexpr int kChunks = kRedBlock / 32;
    const int t = threadIdx.x;
    for (int k = 0; k < NV; ++k) red[k * (kRedBlock + 1) + t] = v[k];
    __syncthreads();
    double part = 0.0;
    if (t < NV * kChunks) {
        const double* r = red + (t / kChunks) * (kRedBlock + 1) + 32 * (t % kChunks);
        part = r[0];
        for (int q = 1; q < 32; ++q) part += r[q];
    }
    __syncthreads();
    if (t < NV * kChunks) red[t] = part;
    __syncthreads();
    double s = 0.0;
    if (t < NV) {
        s = red[t * kChunks];
        for (int c = 1; c < kChunks; ++c) s += red[t * kChunks + c];
    }
    return s;
}

__global__ void k_pos_in(const double* __restrict__ pos, int n, double* __restrict__ x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] = pos[3 * i];
    x[n + i] = pos[3 * i + 1];
    x[2 * n + i] = pos[3 * i + 2];
}

// per step: F_i = F_i^EAM (carries u) + ACE sum (carries w) - grad w_i (E^ACE - E^EAM) + F_ind
__device__ __forceinline__ void blend_body(
    const double* __restrict__ x, int n, const GridDev g, const DynDev dy, const double* __restrict__ tptr,
    const float4* __restrict__ pos4, const int* __restrict__ cell,
    const float* __restrict__ wv, float* __restrict__ f, unsigned long long* __restrict__ acc,
    const float* __restrict__ e_ace, const double* __restrict__ e_eam, double c1_0, float* __restrict__ out_aos,
    int* __restrict__ flags, double hdta, const unsigned char* __restrict__ fixed, double* __restrict__ v,
    const long long* __restrict__ step, long long* __restrict__ load_ring, int load_cap, int bid) {
    pdl_wait();
    // FP64 runs at 1/64 of the FP32 rate on this GPU.  Positions are taken in FP32 from the
    // cell origin and x_rel (absolute error ~1e-5 A) for the indenter pre-test, inside its
    // margin, and for the weight-gradient force of the switching shell, whose relative error
    // of ~1e-6 stays far below the force bar; only atoms near the tip read FP64 positions.
    __shared__ float sh[12];         // box origin, cell edges, tip centre and zone centre at time t
    const int i = bid * blockDim.x + threadIdx.x;
    // Every load of the atom's own data is issued here, before the block barrier and before
    // any store: a store to acc or v between loads of the same array would order them into a
    // chain of dependent memory round trips (the compiler cannot rule out that the k-th and
    // (k+1)-th components alias).
    const bool kick = hdta != 0.0;
    float wi = 0.0f, F0[3] = {0.0f, 0.0f, 0.0f};
    long long qa[3] = {0, 0, 0};
    float4 p = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int ci = 0;
    bool fixed_i = true;
    double vv[3] = {0.0, 0.0, 0.0};
    if (i < n) {
        wi = wv[i];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            qa[k] = (long long)acc[(size_t)k * n + i];
            F0[k] = f[(size_t)k * n + i];
        }
        p = pos4[i];
        ci = cell[i];
        if (kick) {
            fixed_i = fixed[i] != 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) vv[k] = v[(size_t)k * n + i];
        }
    }
    if (threadIdx.x == 0 && g.ortho) {
        const double t = *tptr;
        for (int q = 0; q < 3; ++q) {
            sh[q] = (float)g.origin[q];
            sh[3 + q] = (float)g.cellvec[4 * q];
            sh[6 + q] = (float)(dy.ind_c0[q] - dy.ind_vel[q] * t);
            sh[9 + q] = (float)(dy.reg_c0[q] - (dy.follow ? dy.ind_vel[q] * t : 0.0));
        }
    }
    __syncthreads();
    if (i >= n) return;
    float F[3];
    for (int k = 0; k < 3; ++k) {
        const long long q = qa[k];
        acc[(size_t)k * n + i] = 0ull;
        // q 2^-40 without FP64 instructions: q = hi 2^32 + lo, lo in [0, 2^32); hi 2^-8 is
        // exact in FP32 for forces below 2^16 eV/A and the sum is rounded once
        const int hi = (int)(q >> 32);
        const unsigned lo = (unsigned)(q & 0xffffffffll);
        F[k] = F0[k] + fmaf((float)hi, 0x1p-8f, (float)lo * 0x1p-40f);
    }
    const bool trans = dy.reg_kind == AP_REGION_SPHERE && wi > 0.0f && wi < 1.0f;
    bool near_tip = dy.ind_on;
    if (g.ortho && (trans || near_tip)) {
        int cc[3];
        cell_coords(g, ci, cc);
        float xf[3];
        xf[0] = fmaf((float)cc[0], sh[3], sh[0]) + p.x;
        xf[1] = fmaf((float)cc[1], sh[4], sh[1]) + p.y;
        xf[2] = fmaf((float)cc[2], sh[5], sh[2]) + p.z;
        if (near_tip) {
            const float d[3] = {xf[0] - sh[6], xf[1] - sh[7], xf[2] - sh[8]};
            near_tip = min_image_d2_f32v(g, d) < dy.ind_R2_hi;
        }
        if (trans) {
            float d[3] = {xf[0] - sh[9], xf[1] - sh[10], xf[2] - sh[11]};
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (g.periodic[k]) d[k] = fmaf(-g.Lf[k], rintf(d[k] * g.Linvf[k]), d[k]);
            const float d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], dist = sqrtf(d2);
            const float rin = (float)dy.r_in, rsw = (float)dy.r_sw;
            const float a = fminf(fmaxf((dist - rin) / rsw, 0.0f), 1.0f);
            const float dS = -3.14159265358979f / rsw * sinpif(0.5f * a) * cospif(0.5f * a);
            const float de = (float)((c1_0 + (double)e_ace[i]) - e_eam[i]);
            const float gi = dS * de / dist;
            for (int k = 0; k < 3; ++k) F[k] -= gi * d[k];
        }
    }
    if ((trans && !g.ortho) || near_tip) {
        const double t = *tptr;
        const double r[3] = {x[i], x[n + i], x[2 * n + i]};
        if (trans && !g.ortho) {
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = r[k] - (dy.reg_c0[k] - (dy.follow ? dy.ind_vel[k] * t : 0.0));
            min_image_vec(g, d);
            const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            float uS, dS;
            switch_weight(d2, dy.r_in, dy.r_sw, &uS, &dS);
            const float de = (float)((c1_0 + (double)e_ace[i]) - e_eam[i]);
            const float gi = dS * de * rsqrtf((float)d2);
            for (int k = 0; k < 3; ++k) F[k] -= gi * (float)d[k];
        }
        if (near_tip) {
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = r[k] - (dy.ind_c0[k] - dy.ind_vel[k] * t);
            min_image_vec(g, d);
            const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (d2 < dy.R * dy.R && d2 > 0.0) {
                const double dist = sqrt(d2), h = dy.R - dist, c = dy.K * h * h / dist;
                for (int k = 0; k < 3; ++k) F[k] += (float)(c * d[k]);
                if (load_ring) {
                    // this atom's share of Eq. P_ind in fixed point: integer sums do not
                    // depend on the order of the atomics
                    const double l = c * (d[0] * dy.ind_dir[0] + d[1] * dy.ind_dir[1] + d[2] * dy.ind_dir[2]);
                    atomicAdd(reinterpret_cast<unsigned long long*>(&load_ring[*step % load_cap]),
                              (unsigned long long)__double2ll_rn(l * kLoadScale));
                }
            }
        }
    }
    for (int k = 0; k < 3; ++k) f[(size_t)k * n + i] = F[k];
    if (out_aos)
        for (int k = 0; k < 3; ++k) out_aos[3 * (size_t)i + k] = F[k];
    // the second half kick of a velocity-Verlet step, when nothing else adds to F before it
    // (the same arithmetic as k_kick)
    if (kick && !fixed_i)
        for (int k = 0; k < 3; ++k) v[(size_t)k * n + i] = vv[k] + hdta * (double)F[k];
    if (!(F[0] == F[0]) || !(F[1] == F[1]) || !(F[2] == F[2])) {
        atomicOr(&flags[kFlagErr], kErrDomain);
        flags[kFlagBad] = i;
    }
}

__global__ void __launch_bounds__(kRedBlock) k_blend(
    const double* __restrict__ x, int n, const GridDev g, const DynDev dy, const double* __restrict__ tptr,
    const float4* __restrict__ pos4, const int* __restrict__ cell,
    const float* __restrict__ wv, float* __restrict__ f, unsigned long long* __restrict__ acc,
    const float* __restrict__ e_ace, const double* __restrict__ e_eam, double c1_0, float* __restrict__ out_aos,
    int* __restrict__ flags, double hdta, const unsigned char* __restrict__ fixed, double* __restrict__ v,
    const long long* __restrict__ step, long long* __restrict__ load_ring, int load_cap) {
    blend_body(x, n, g, dy, tptr, pos4, cell, wv, f, acc, e_ace, e_eam, c1_0, out_aos, flags, hdta, fixed, v, step, load_ring, load_cap, blockIdx.x);
}

// on request: per-atom E_i + V_ind, and block sums of the energies, the virial and the load
__global__ void __launch_bounds__(kRedBlock) k_energy_blend(
    const double* __restrict__ x, int n, const GridDev g, const DynDev dy, const double* __restrict__ tptr,
    const float* __restrict__ wv, const float4* __restrict__ pos4, const int* __restrict__ cell,
    const float* __restrict__ e_ace, const double* __restrict__ e_eam, double c1_0,
    const float* __restrict__ vir_eam, const float* __restrict__ vir_ace, double* __restrict__ e_atom,
    double* __restrict__ partials, int* __restrict__ flags, int with_virial) {
    __shared__ double red[9 * (kRedBlock + 1)];
    __shared__ float sh[9];          // box origin, cell edges (orthorhombic), tip centre at time t
    if (threadIdx.x == 0 && dy.ind_on && g.ortho) {
        const double t = *tptr;
        for (int q = 0; q < 3; ++q) {
            sh[q] = (float)g.origin[q];
            sh[3 + q] = (float)g.cellvec[4 * q];
            sh[6 + q] = (float)(dy.ind_c0[q] - dy.ind_vel[q] * t);
        }
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};     // E, V_ind, virial (6), load
    if (i < n) {
        const float4 p = pos4[i];
        const double wi = wv[i], ui = p.w;              // both weights at FP32 relative precision
        const double Ei = (wi > 0.0 ? wi * (c1_0 + (double)e_ace[i]) : 0.0) + (ui > 0.0 ? ui * e_eam[i] : 0.0);
        double V = 0.0;
        bool near_tip = dy.ind_on;
        if (near_tip && g.ortho) {
            // FP32 pre-test (positions to ~1e-5 A, inside the margin of ind_R2_hi)
            int cc[3];
            cell_coords(g, cell[i], cc);
            const float h[3] = {p.x, p.y, p.z};
            float d[3];
            for (int q = 0; q < 3; ++q) d[q] = (fmaf((float)cc[q], sh[3 + q], sh[q]) - sh[6 + q]) + h[q];
            near_tip = min_image_d2_f32v(g, d) < dy.ind_R2_hi;
        }
        if (near_tip) {
            const double t = *tptr;
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = x[(size_t)k * n + i] - (dy.ind_c0[k] - dy.ind_vel[k] * t);
            min_image_vec(g, d);
            const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (d2 < dy.R * dy.R && d2 > 0.0) {
                const double dist = sqrt(d2), h = dy.R - dist;
                V = dy.K * h * h * h / 3.0;
                const double c = dy.K * h * h / dist;
                acc[8] = c * (d[0] * dy.ind_dir[0] + d[1] * dy.ind_dir[1] + d[2] * dy.ind_dir[2]);
            }
        }
        e_atom[i] = Ei + V;
        acc[0] = Ei;
        acc[1] = V;
        // per-atom virial: the FP32 sum of the two parts (relative error ~6e-8 per atom)
        if (with_virial)
            for (int k = 0; k < 6; ++k)
                acc[2 + k] = (double)(vir_eam[(size_t)k * n + i] + (wi > 0.0 ? vir_ace[(size_t)k * n + i] : 0.0f));
        if (!(Ei == Ei)) {
            atomicOr(&flags[kFlagErr], kErrDomain);
            flags[kFlagBad] = i;
        }
    }
    const double s = block_sums<9>(acc, red);
    if (threadIdx.x < 9) partials[(size_t)blockIdx.x * kNP + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kRedBlock) k_kinetic(const double* __restrict__ v, const unsigned char* __restrict__ fixed,
                                                       int n, double mass, double* __restrict__ partials) {
    __shared__ double sh[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (i < n) {
        const double a = v[i], b = v[n + i], c = v[2 * n + i];
        ke = 0.5 * mass * (a * a + b * b + c * c) / kFtm;
    }
    double s = block_sum(ke, sh);
    if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kNP + 9] = s;
}

__global__ void __launch_bounds__(kRedBlock) k_reduce(const double* __restrict__ partials, int nblk,
                                                        double* __restrict__ totals, int with_ke) {
    __shared__ double red[kNP * (kRedBlock + 1)];
    double v[kNP] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += kRedBlock)
        for (int k = 0; k < kNP; ++k) v[k] += partials[(size_t)b * kNP + k];
    const double s = block_sums<kNP>(v, red);
    if (threadIdx.x < kNP && (threadIdx.x != 9 || with_ke)) totals[threadIdx.x] = s;
}

// first half kick and drift; the neighbour-list displacement test of the step is taken here,
// where x is in registers (an atom that moved more than skin/2 since the last build sets the
// rebuild flag), and the compaction counter of the coming force pass is reset
__device__ __forceinline__ void kick_drift_body(double* __restrict__ x, double* __restrict__ v, const float* __restrict__ f,
                             const unsigned char* __restrict__ fixed, int n, double hdta, double dt,
                             double* __restrict__ tptr, long long* __restrict__ step,
                             const double* __restrict__ xb, double lim2, int* __restrict__ flags,
                             long long* __restrict__ load_ring, double* __restrict__ load_ring_t, int load_cap, int bid) {
    pdl_wait();
    const int i = bid * blockDim.x + threadIdx.x;
    if (i == 0) {
        *tptr += dt;
        *step += 1;
        flags[kFlagNAce] = 0;
        if (load_ring) {
            // the slot of this step starts at zero; the blend of its force pass adds the load
            const long long slot = *step % load_cap;
            load_ring[slot] = 0;
            load_ring_t[slot] = *tptr;
        }
    }
    if (i >= n) return;
    // all loads first (see blend_body): the stores to v and x would otherwise order the
    // component loads into dependent round trips
    double v0[3], x0[3], b0[3];
    float f0[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v0[k] = v[(size_t)k * n + i];
        f0[k] = f[(size_t)k * n + i];
        x0[k] = x[(size_t)k * n + i];
        b0[k] = xb[(size_t)k * n + i];
    }
    if (fixed[i]) return;
    double d2 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double vk = v0[k] + hdta * (double)f0[k];
        v[(size_t)k * n + i] = vk;
        const double xk = x0[k] + dt * vk;
        x[(size_t)k * n + i] = xk;
        const double d = xk - b0[k];
        d2 += d * d;
    }
    if (d2 > lim2) flags[kFlagRebuild] = 1;
}

__global__ void k_kick_drift(double* __restrict__ x, double* __restrict__ v, const float* __restrict__ f,
                             const unsigned char* __restrict__ fixed, int n, double hdta, double dt,
                             double* __restrict__ tptr, long long* __restrict__ step,
                             const double* __restrict__ xb, double lim2, int* __restrict__ flags,
                             long long* __restrict__ load_ring, double* __restrict__ load_ring_t, int load_cap) {
    kick_drift_body(x, v, f, fixed, n, hdta, dt, tptr, step, xb, lim2, flags, load_ring, load_ring_t, load_cap, blockIdx.x);
}

__global__ void k_kick(double* __restrict__ v, const float* __restrict__ f, const unsigned char* __restrict__ fixed,
                       int n, double hdta) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || fixed[i]) return;
    for (int k = 0; k < 3; ++k) v[(size_t)k * n + i] += hdta * (double)f[(size_t)k * n + i];
}

// Nose-Hoover half step on the group: block sums of the group's kinetic energy, one block
// that advances xi and eta and computes the velocity scale, then the scaling
__global__ void __launch_bounds__(kRedBlock) k_group_ke(const double* __restrict__ v,
                                                        const unsigned char* __restrict__ group, int n, double mass,
                                                        double* __restrict__ partials) {
    __shared__ double sh[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (i < n && group[i]) {
        const double a = v[i], b = v[n + i], c = v[2 * n + i];
        ke = 0.5 * mass * (a * a + b * b + c * c) / kFtm;
    }
    const double s = block_sum(ke, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_nh_update(const double* __restrict__ partials, int nblk, double* __restrict__ st, double dt,
                            double nfkt, double Q) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += partials[b];
    double ke = block_sum(v, sh);
    if (threadIdx.x == 0) {
        double xi = st[0], eta = st[1];
        xi += 0.25 * dt * (2.0 * ke - nfkt) / Q;
        const double sc = exp(-0.5 * dt * xi);
        ke *= sc * sc;
        eta += 0.5 * dt * xi;
        xi += 0.25 * dt * (2.0 * ke - nfkt) / Q;
        st[0] = xi;
        st[1] = eta;
        st[2] = sc;
    }
}

__global__ void k_scale_group(double* __restrict__ v, const unsigned char* __restrict__ group, int n,
                              const double* __restrict__ st) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !group[i]) return;
    const double sc = st[2];
    for (int k = 0; k < 3; ++k) v[(size_t)k * n + i] *= sc;
}

// Philox4x32-10 (Salmon et al., SC'11): ten multiply-xor rounds with Weyl key increments
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

// Langevin drag and random force on the group, added to the forces of this step
__global__ void k_langevin(const double* __restrict__ v, float* __restrict__ f, const unsigned char* __restrict__ group,
                           int n, const long long* __restrict__ step, long long base, unsigned long long seed,
                           double drag, double sig) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !group[i]) return;
    uint32_t w[4] = {(uint32_t)i, (uint32_t)(*step - base), 0u, 0u};
    philox4x32_10(w, (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
    const double two32 = 4294967296.0, tpi = 6.283185307179586476925;
    const double r1 = sqrt(-2.0 * log(((double)w[0] + 1.0) / two32)), a1 = tpi * (((double)w[1] + 0.5) / two32);
    const double r2 = sqrt(-2.0 * log(((double)w[2] + 1.0) / two32)), a2 = tpi * (((double)w[3] + 0.5) / two32);
    const double g[3] = {r1 * cos(a1), r1 * sin(a1), r2 * cos(a2)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const size_t q = (size_t)k * n + i;
        f[q] = (float)((double)f[q] - drag * v[q] + sig * g[k]);
    }
}

// momentum zeroing every `every` steps: block sums of the free atoms' velocities, their mean,
// the subtraction
__global__ void __launch_bounds__(kRedBlock) k_com_partial(const double* __restrict__ v,
                                                           const unsigned char* __restrict__ fixed, int n,
                                                           const long long* __restrict__ step, long long base, int every,
                                                           double* __restrict__ part) {
    if ((*step - base) % every != 0) return;
    __shared__ double sh[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = i < n && !fixed[i];
    double q[4] = {on ? v[i] : 0.0, on ? v[n + i] : 0.0, on ? v[2 * n + i] : 0.0, on ? 1.0 : 0.0};
    for (int k = 0; k < 4; ++k) {
        const double s = block_sum(q[k], sh);
        if (threadIdx.x == 0) part[4 * blockIdx.x + k] = s;
    }
}

__global__ void k_com_final(const double* __restrict__ part, int nblk, const long long* __restrict__ step,
                            long long base, int every, double* __restrict__ com) {
    __shared__ double sh[32];
    const bool go = (*step - base) % every == 0;
    double tot[4];
    for (int k = 0; k < 4; ++k) {
        double v = 0.0;
        if (go)
            for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += part[4 * b + k];
        tot[k] = block_sum(v, sh);
    }
    if (threadIdx.x == 0) {
        const bool any = go && tot[3] > 0.0;
        for (int k = 0; k < 3; ++k) com[k] = any ? tot[k] / tot[3] : 0.0;
        com[3] = any ? 1.0 : 0.0;
    }
}

__global__ void k_sub_com(double* __restrict__ v, const unsigned char* __restrict__ fixed, int n,
                          const double* __restrict__ com) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || fixed[i] || com[3] == 0.0) return;
    for (int k = 0; k < 3; ++k) v[(size_t)k * n + i] -= com[k];
}

__global__ void __launch_bounds__(kRedBlock) kb_blend(const BatchTable t, double kick_dt, int record) {
    const int k = batch_find(t.b256, t.nctx, blockIdx.x);
    const CtxDev& c = *t.d[k];
    long long* ring = record && c.dyn.ind_on ? c.load_ring : nullptr;
    blend_body(c.x, c.n, c.grid, c.dyn, c.d_time, c.pos4, c.cell, c.w, c.f, c.acc, c.e_ace, c.e_eam, c.ace_c1_0,
               nullptr, c.flags, kick_dt > 0.0 ? 0.5 * kick_dt * kFtm / c.mass : 0.0, c.fixed, c.v, c.d_step, ring,
               c.load_cap, blockIdx.x - t.b256[k]);
}

__global__ void kb_kick_drift(const BatchTable t, double dt) {
    const int k = batch_find(t.b256, t.nctx, blockIdx.x);
    const CtxDev& c = *t.d[k];
    kick_drift_body(c.x, c.v, c.f, c.fixed, c.n, 0.5 * dt * kFtm / c.mass, dt, c.d_time, c.d_step, c.xb, c.lim2,
                    c.flags, c.load_ring, c.load_ring_t, c.load_cap, blockIdx.x - t.b256[k]);
}

}  // namespace

int launch_langevin(Ctx& c, cudaStream_t s, double dt) {
    k_langevin<<<(c.n + 255) / 256, 256, 0, s>>>(c.v, c.f, c.thermo_group, c.n, c.d_step, c.lv_base, c.lv_seed,
                                                 c.lv_drag, std::sqrt(c.lv_sig / dt));
    return 1;
}

int launch_zero_momentum(Ctx& c, cudaStream_t s) {
    k_com_partial<<<c.nred, kRedBlock, 0, s>>>(c.v, c.fixed, c.n, c.d_step, c.lv_base, c.lv_zero_every, c.com);
    k_com_final<<<1, 1024, 0, s>>>(c.com, c.nred, c.d_step, c.lv_base, c.lv_zero_every, c.com + 4 * (size_t)c.nred);
    k_sub_com<<<(c.n + 255) / 256, 256, 0, s>>>(c.v, c.fixed, c.n, c.com + 4 * (size_t)c.nred);
    return 3;
}

int launch_nh_half(Ctx& c, cudaStream_t s, double dt) {
    k_group_ke<<<c.nred, kRedBlock, 0, s>>>(c.v, c.thermo_group, c.n, c.mass, c.nh_partials);
    k_nh_update<<<1, 1024, 0, s>>>(c.nh_partials, c.nred, c.nh_state, dt, c.nh_nfkt, c.nh_Q);
    k_scale_group<<<(c.n + 255) / 256, 256, 0, s>>>(c.v, c.thermo_group, c.n, c.nh_state);
    return 3;
}

int launch_pos_in(Ctx& c, cudaStream_t s, const double* pos) {
    k_pos_in<<<(c.n + 255) / 256, 256, 0, s>>>(pos, c.n, c.x);
    return 1;
}

int launch_blend(Ctx& c, cudaStream_t s, float* out_aos, double kick_dt, bool in_step) {
    const double hdta = kick_dt > 0.0 ? 0.5 * kick_dt * kFtm / c.mass : 0.0;
    long long* ring = in_step && c.dyn.ind_on ? c.load_ring : nullptr;
    launch_pdl(k_blend, c.nred, kRedBlock, 0, s, c.x, c.n, c.grid, c.dyn, c.d_time, c.pos4, c.cell, c.w, c.f, c.acc,
               c.e_ace, c.e_eam, c.ace_c1_0, out_aos, c.flags, hdta, c.fixed, c.v, (const long long*)c.d_step, ring,
               c.load_cap);
    return 1;
}

int launch_energy_blend(Ctx& c, cudaStream_t s, bool virial) {
    k_energy_blend<<<c.nred, kRedBlock, 0, s>>>(c.x, c.n, c.grid, c.dyn, c.d_time, c.w, c.pos4, c.cell, c.e_ace,
                                                c.e_eam_acc, c.ace_c1_0, c.vir_eam, c.vir_ace, c.e_atom, c.partials,
                                                c.flags, virial ? 1 : 0);
    return 1;
}

int launch_energy(Ctx& c, cudaStream_t s, bool virial) {
    return launch_eam_energy(c, s, virial) + launch_energy_blend(c, s, virial);
}

int launch_reduce(Ctx& c, cudaStream_t s, int with_kinetic) {
    int k = 0;
    if (with_kinetic) {
        k_kinetic<<<c.nred, kRedBlock, 0, s>>>(c.v, c.fixed, c.n, c.mass, c.partials);
        ++k;
    }
    k_reduce<<<1, kRedBlock, 0, s>>>(c.partials, c.nred, c.totals, with_kinetic);
    return k + 1;
}

int launch_kick_drift(Ctx& c, cudaStream_t s, double dt, int) {
    const double lim = 0.5 * c.skin;
    launch_pdl(k_kick_drift, (c.n + 255) / 256, 256, 0, s, c.x, c.v, c.f, c.fixed, c.n, 0.5 * dt * kFtm / c.mass, dt,
               c.d_time, c.d_step, c.xb, lim * lim, c.flags, c.load_ring, c.load_ring_t, c.load_cap);
    return 1;
}

int launch_kick(Ctx& c, cudaStream_t s, double dt) {
    launch_pdl(k_kick, (c.n + 255) / 256, 256, 0, s, c.v, c.f, c.fixed, c.n, 0.5 * dt * kFtm / c.mass);
    return 1;
}


int launch_batch_blend(const BatchTable& t, double kick_dt, int record, cudaStream_t s) {
    static_assert(kRedBlock == 256, "the batch table counts blend blocks of 256 threads");
    launch_pdl(kb_blend, t.b256[t.nctx], kRedBlock, 0, s, t, kick_dt, record);
    return 1;
}

int launch_batch_step_pre(const BatchTable& t, double dt, cudaStream_t s) {
    launch_pdl(kb_kick_drift, t.b256[t.nctx], 256, 0, s, t, dt);
    return 1;
}

}  // namespace ap
