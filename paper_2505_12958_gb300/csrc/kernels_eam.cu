// kernels_eam.cu -- EAM pass of the AP force evaluation (Sec. 2.2.1, Eq. energy_eam).
//
// With u_i = 1 - w_i the EAM share of the energy is sum_i u_i [xi(rho_i) + Delta xi +
// 1/2 sum_j Phi(r_ij)], rho_i = sum_j zeta(r_ij).  Its negative gradient on atom i is
//   F_i = sum_j [ (u_i xi'(rho_i) + u_j xi'(rho_j)) zeta'(r_ij) + (u_i + u_j)/2 Phi'(r_ij) ] rhat_ij,
// evaluated from i's side over the full list, so no atomics are needed and the sum
// order is fixed.  Two passes: density (rho, xi, u xi' per atom), then forces, per-atom
// energies and the per-atom virial -1/2 sum_j c_ij r_ij (x) rhat_ij.  The embedding
// function is evaluated in FP64 (one square root per atom); pair terms are FP32
// piecewise polynomials from the host tables.
#include "ap_internal.h"

namespace ap {

namespace {

__device__ __forceinline__ void poly_eval(const PolyTab& t, float r, float& f, float& df, float zk, float zainv) {
    int b = (int)(r * t.bin_inv);
    b = b < kNBin ? b : kNBin - 1;
    int k = t.bin[b];
    while (k + 1 < t.nint && r >= t.start[k + 1]) ++k;
    if (t.zbl && k == 0) {
        // screened Coulomb: Z^2/(4 pi eps0 r) phi(r/a), phi = sum of four exponentials
        float x = r * zainv;
        float e0 = 0.1818f * expf(-3.2f * x), e1 = 0.5099f * expf(-0.9423f * x);
        float e2 = 0.2802f * expf(-0.4029f * x), e3 = 0.02817f * expf(-0.2016f * x);
        float ph = e0 + e1 + e2 + e3;
        float dph = -(3.2f * e0 + 0.9423f * e1 + 0.4029f * e2 + 0.2016f * e3);
        float ri = 1.0f / r;
        f = zk * ph * ri;
        df = zk * (dph * zainv * ri - ph * ri * ri);
        return;
    }
    float x = r - t.mid[k];
    const float* c = t.c[k];
    f = ((((c[5] * x + c[4]) * x + c[3]) * x + c[2]) * x + c[1]) * x + c[0];
    df = (((5.0f * c[5] * x + 4.0f * c[4]) * x + 3.0f * c[3]) * x + 2.0f * c[2]) * x + c[1];
}

__device__ __forceinline__ void stage_tables(EamDev* sm, const EamDev* __restrict__ gm, float4* Ds,
                                             const float4* __restrict__ D, int ncode) {
    const int4* src = reinterpret_cast<const int4*>(gm);
    int4* dst = reinterpret_cast<int4*>(sm);
    for (int k = threadIdx.x; k < (int)(sizeof(EamDev) / 16); k += blockDim.x) dst[k] = src[k];
    for (int k = threadIdx.x; k < ncode; k += blockDim.x) Ds[k] = D[k];
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_eam_density(const float4* __restrict__ pos4, const int* __restrict__ nbr,
                                                     const int* __restrict__ nnbr, int n, const EamDev* __restrict__ eam,
                                                     const float4* __restrict__ D, int ncode, float* __restrict__ uxi,
                                                     double* __restrict__ e_emb, int* __restrict__ flags) {
    __shared__ EamDev T;
    __shared__ float4 Ds[125];
    stage_tables(&T, eam, Ds, D, ncode);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) flags[kFlagRebuild] = 0;        // the list built this step is in use now
    if (i >= n) return;
    float4 p = pos4[i];
    float u = p.w;
    if (u <= 0.0f) { uxi[i] = 0.0f; e_emb[i] = 0.0; return; }
    const float rc2 = T.rho.rcut * T.rho.rcut;
    float rho = 0.0f;
    int m = nnbr[i];
    for (int k = 0; k < m; ++k) {
        int e = nbr[(size_t)k * n + i];
        int j = e & kNbrMask;
        float4 d = Ds[(unsigned)e >> kNbrShift];
        float4 q = pos4[j];
        float dx = q.x + d.x - p.x, dy = q.y + d.y - p.y, dz = q.z + d.z - p.z;
        float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < rc2) {
            float f, df;
            poly_eval(T.rho, sqrtf(r2), f, df, 0.0f, 0.0f);
            rho += f;
        }
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
}

__global__ void __launch_bounds__(256) k_eam_force(const float4* __restrict__ pos4, const int* __restrict__ nbr,
                                                   const int* __restrict__ nnbr, int n, const EamDev* __restrict__ eam,
                                                   const float4* __restrict__ D, int ncode, const float* __restrict__ uxi,
                                                   const double* __restrict__ e_emb, float* __restrict__ f,
                                                   double* __restrict__ e_eam, float* __restrict__ vir) {
    __shared__ EamDev T;
    __shared__ float4 Ds[125];
    stage_tables(&T, eam, Ds, D, ncode);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 p = pos4[i];
    const float ui = p.w, xi = uxi[i];
    const float rc2 = T.rc * T.rc, rcr = T.rho.rcut, rcp = T.phi.rcut;
    float fx = 0.f, fy = 0.f, fz = 0.f, eph = 0.f;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f, v4 = 0.f, v5 = 0.f;
    int m = nnbr[i];
    for (int k = 0; k < m; ++k) {
        int e = nbr[(size_t)k * n + i];
        int j = e & kNbrMask;
        float4 d = Ds[(unsigned)e >> kNbrShift];
        float4 q = pos4[j];
        float dx = q.x + d.x - p.x, dy = q.y + d.y - p.y, dz = q.z + d.z - p.z;
        float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= rc2) continue;
        float us = ui + q.w;
        if (us <= 0.0f) continue;              // both atoms fully ACE
        float r = sqrtf(r2), ri = 1.0f / r;
        float zf = 0.f, dz_ = 0.f, pf = 0.f, dp = 0.f;
        if (r < rcr) poly_eval(T.rho, r, zf, dz_, 0.f, 0.f);
        if (r < rcp) poly_eval(T.phi, r, pf, dp, T.zbl_k, T.zbl_ainv);
        float c = (xi + uxi[j]) * dz_ + 0.5f * us * dp;
        float cr = c * ri;
        fx += cr * dx; fy += cr * dy; fz += cr * dz;
        eph += pf;
        float s = -0.5f * cr;
        v0 += s * dx * dx; v1 += s * dy * dy; v2 += s * dz * dz;
        v3 += s * dx * dy; v4 += s * dx * dz; v5 += s * dy * dz;
    }
    f[i] = fx; f[n + i] = fy; f[2 * n + i] = fz;
    e_eam[i] = ui > 0.0f ? e_emb[i] + 0.5 * (double)eph : 0.0;
    vir[i] = v0; vir[n + i] = v1; vir[2 * n + i] = v2; vir[3 * n + i] = v3; vir[4 * n + i] = v4; vir[5 * n + i] = v5;
}

// ---------------------------------------------------------------------------------
// On-demand FP64 EAM energies.  FP32 pair distances and polynomials are accurate to a few
// ulp, but in a perfect lattice every equivalent atom repeats the same rounding, which
// adds up coherently to ~1e-6 eV/atom; energies are therefore recomputed from the FP64
// positions (exact periodic image shifts) when a caller asks for them.
// ---------------------------------------------------------------------------------
__device__ double poly64(const PolyTab64& t, double r, double zk, double za) {
    if (r >= t.rcut) return 0.0;
    int k = 0;
    while (k + 1 < t.nint && r >= t.start[k + 1]) ++k;
    if (t.zbl && k == 0) {
        double xx = r / za;
        double ph = 0.1818 * exp(-3.2 * xx) + 0.5099 * exp(-0.9423 * xx) + 0.2802 * exp(-0.4029 * xx) +
                    0.02817 * exp(-0.2016 * xx);
        return zk * ph / r;
    }
    double x = r - t.mid[k];
    const double* c = t.c[k];
    return ((((c[5] * x + c[4]) * x + c[3]) * x + c[2]) * x + c[1]) * x + c[0];
}

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

__global__ void __launch_bounds__(128) k_eam_energy64(const double* __restrict__ x, int n, const GridDev g,
                                                      const int* __restrict__ cell, const int* __restrict__ nbr,
                                                      const int* __restrict__ nnbr, const float4* __restrict__ pos4,
                                                      const EamDev64* __restrict__ T, double* __restrict__ e_eam) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (pos4[i].w <= 0.0f) { e_eam[i] = 0.0; return; }
    int ci = cell[i];
    int cc[3] = {ci / (g.nc[1] * g.nc[2]), (ci / g.nc[2]) % g.nc[1], ci % g.nc[2]};
    const double xi = x[i], yi = x[n + i], zi = x[2 * n + i];
    const int w1 = 2 * g.S[1] + 1, w2 = 2 * g.S[2] + 1;
    double rho = 0.0, ph = 0.0;
    const int m = nnbr[i];
    for (int k = 0; k < m; ++k) {
        const int e = nbr[(size_t)k * n + i];
        const int j = e & kNbrMask;
        const int code = (int)((unsigned)e >> kNbrShift);
        int o[3] = {code / (w1 * w2) - g.S[0], (code / w2) % w1 - g.S[1], code % w2 - g.S[2]};
        double sh[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < 3; ++d) {
            if (!g.periodic[d]) continue;
            const int im = floor_div(cc[d] + o[d], g.nc[d]);
            if (im != 0)
                for (int q = 0; q < 3; ++q) sh[q] += im * g.h[3 * d + q];
        }
        const double dx = x[j] + sh[0] - xi, dy = x[n + j] + sh[1] - yi, dz = x[2 * n + j] + sh[2] - zi;
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (r < T->rho.rcut) rho += poly64(T->rho, r, 0.0, 1.0);
        if (r < T->phi.rcut) ph += poly64(T->phi, r, T->zbl_k, T->zbl_a);
    }
    double F = T->F_dxi;
    if (rho > 0.0) F += T->F_a1 * sqrt(rho) + T->F_a2 * rho * rho;
    e_eam[i] = F + 0.5 * ph;
}

}  // namespace

int launch_eam_energy64(Ctx& c, cudaStream_t s) {
    k_eam_energy64<<<(c.n + 127) / 128, 128, 0, s>>>(c.x, c.n, c.grid, c.cell, c.nbr, c.nnbr, c.pos4, c.eam64_d,
                                                     c.e_eam);
    return 1;
}

int launch_eam_density(Ctx& c, cudaStream_t s) {
    k_eam_density<<<(c.n + 255) / 256, 256, 0, s>>>(c.pos4, c.nbr, c.nnbr, c.n, c.eam_d, c.D, c.grid.ncode, c.uxi,
                                                   c.e_emb, c.flags);
    return 1;
}

int launch_eam_force(Ctx& c, cudaStream_t s) {
    k_eam_force<<<(c.n + 255) / 256, 256, 0, s>>>(c.pos4, c.nbr, c.nnbr, c.n, c.eam_d, c.D, c.grid.ncode, c.uxi,
                                                 c.e_emb, c.f, c.e_eam, c.vir_eam);
    return 1;
}

}  // namespace ap
