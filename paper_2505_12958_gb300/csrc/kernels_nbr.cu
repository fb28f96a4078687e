// kernels_nbr.cu -- cell binning, neighbour list, per-step preparation.
//
// The neighbour list is a full list (each pair appears from both sides) within
// r_list = max(EAM cutoff, ACE cutoff) + skin, stored column-major nbr[k * n + i]
// so that thread-per-atom kernels read it coalesced; the build also writes the same entries
// row by row, nrow[i * cap + k], for the warp-per-atom ACE kernels, whose lanes then read
// one atom's row (a few cache lines) instead of 32 rows.  An entry packs the neighbour
// index j with the code of the cell offset o (per edge -S..S) it was found in; the
// pair vector is then x_rel_j + D[code] - x_rel_i in FP32, where x_rel is the position
// relative to the atom's own cell origin.  This keeps every FP32 operand below the
// cell size (a few Angstrom), so forming r_ij costs no FP64 work per pair.
// The list is rebuilt only when some atom moved more than skin/2 since the last build;
// each rebuild kernel reads that device flag and returns at once when it is clear, so
// no host synchronisation is needed per step.  Cells keep their atoms in index order
// (insertion sort after the atomic scatter), which makes the list, and therefore every
// FP32 summation order, deterministic.
#include "ap_internal.h"
#include "geom.cuh"

namespace ap {

namespace {

__device__ __forceinline__ void check_body(const double* __restrict__ x, const double* __restrict__ xb, int n, double lim2,
                        int* flags, int bid) {
    pdl_wait();
    int i = bid * blockDim.x + threadIdx.x;
    if (i == 0) flags[kFlagNAce] = 0;
    if (i >= n) return;
    double dx = x[i] - xb[i], dy = x[n + i] - xb[n + i], dz = x[2 * n + i] - xb[2 * n + i];
    if (dx * dx + dy * dy + dz * dz > lim2) flags[kFlagRebuild] = 1;
}

__global__ void k_check(const double* __restrict__ x, const double* __restrict__ xb, int n, double lim2,
                        int* flags) {
    check_body(x, xb, n, lim2, flags, blockIdx.x);
}

__device__ __forceinline__ void wrap_bin_body(double* __restrict__ x, double* __restrict__ xb, int n, const GridDev g,
                           int* __restrict__ cell, int* __restrict__ cell_count, int* __restrict__ flags, int bid) {
    pdl_wait();
    if (flags[kFlagRebuild] == 0) return;
    int i = bid * blockDim.x + threadIdx.x;
    if (i == 0) flags[kFlagRebuilds] += 1;
    if (i >= n) return;
    double r[3] = {x[i], x[n + i], x[2 * n + i]};
    double d[3] = {r[0] - g.origin[0], r[1] - g.origin[1], r[2] - g.origin[2]};
    double s[3];
    for (int k = 0; k < 3; ++k) s[k] = d[0] * g.hinv[k] + d[1] * g.hinv[3 + k] + d[2] * g.hinv[6 + k];
    int c[3];
    for (int k = 0; k < 3; ++k) {
        if (g.periodic[k]) {
            double m = floor(s[k]);
            if (m != 0.0) {
                for (int q = 0; q < 3; ++q) r[q] -= m * g.h[3 * k + q];
                s[k] -= m;
            }
        }
        int ck = (int)floor(s[k] * g.nc[k]);
        c[k] = ck < 0 ? 0 : (ck >= g.nc[k] ? g.nc[k] - 1 : ck);
    }
    for (int q = 0; q < 3; ++q) { x[q * n + i] = r[q]; xb[q * n + i] = r[q]; }
    int ci = (c[0] * g.nc[1] + c[1]) * g.nc[2] + c[2];
    cell[i] = ci;
    atomicAdd(&cell_count[ci], 1);
}

__global__ void k_wrap_bin(double* __restrict__ x, double* __restrict__ xb, int n, const GridDev g,
                           int* __restrict__ cell, int* __restrict__ cell_count, int* __restrict__ flags) {
    wrap_bin_body(x, xb, n, g, cell, cell_count, flags, blockIdx.x);
}

// exclusive scan of cell_count into cell_start (one block); the counters are cleared so
// that the scatter can reuse them as fill pointers
__device__ __forceinline__ void scan_body(int* __restrict__ cell_count, int* __restrict__ cell_start, int ncell,
                       const int* __restrict__ flags, int bid) {
    pdl_wait();
    if (flags[kFlagRebuild] == 0) return;
    __shared__ int part[1024];
    int tid = threadIdx.x, nt = blockDim.x;
    int per = (ncell + nt - 1) / nt;
    int b = tid * per, e = min(b + per, ncell);
    int s = 0;
    for (int c = b; c < e; ++c) s += cell_count[c];
    part[tid] = s;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        int v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int run = part[tid] - s;
    for (int c = b; c < e; ++c) {
        cell_start[c] = run;
        run += cell_count[c];
        cell_count[c] = 0;
    }
    if (tid == nt - 1) cell_start[ncell] = part[nt - 1];
}

__global__ void k_scan(int* __restrict__ cell_count, int* __restrict__ cell_start, int ncell,
                       const int* __restrict__ flags) {
    scan_body(cell_count, cell_start, ncell, flags, blockIdx.x);
}

__device__ __forceinline__ void scatter_body(const int* __restrict__ cell, int n, const int* __restrict__ cell_start,
                          int* __restrict__ fill, int* __restrict__ cell_atoms, const int* __restrict__ flags, int bid) {
    pdl_wait();
    if (flags[kFlagRebuild] == 0) return;
    int i = bid * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cell[i];
    int slot = atomicAdd(&fill[c], 1);
    cell_atoms[cell_start[c] + slot] = i;
}

__global__ void k_scatter(const int* __restrict__ cell, int n, const int* __restrict__ cell_start,
                          int* __restrict__ fill, int* __restrict__ cell_atoms, const int* __restrict__ flags) {
    scatter_body(cell, n, cell_start, fill, cell_atoms, flags, blockIdx.x);
}

// order each cell's atoms by index and clear the per-cell counters for the next build: one
// warp per cell; each atom's slot is the number of smaller indices in its cell (indices are
// distinct), so cells of up to 128 atoms take one pass of loads and one of stores
constexpr int kSortBlock = 256;
constexpr int kSortPerLane = 4;

__device__ __forceinline__ void sort_cells_body(int* __restrict__ cell_atoms, const int* __restrict__ cell_start, int* __restrict__ fill,
                             int ncell, const int* __restrict__ flags, int bid) {
    pdl_wait();
    if (flags[kFlagRebuild] == 0) return;
    const int lane = threadIdx.x & 31;
    const int c = bid * (kSortBlock / 32) + (threadIdx.x >> 5);
    if (c >= ncell) return;
    const int b = cell_start[c], m = cell_start[c + 1] - b;
    if (m <= 32 * kSortPerLane) {
        int v[kSortPerLane], rank[kSortPerLane];
#pragma unroll
        for (int u = 0; u < kSortPerLane; ++u) {
            v[u] = 32 * u + lane < m ? cell_atoms[b + 32 * u + lane] : 0x7fffffff;
            rank[u] = 0;
        }
        for (int u2 = 0; u2 < kSortPerLane && 32 * u2 < m; ++u2) {
            for (int k = 0; k < 32 && 32 * u2 + k < m; ++k) {
                int w = 0;
#pragma unroll
                for (int t = 0; t < kSortPerLane; ++t) if (t == u2) w = __shfl_sync(0xffffffffu, v[t], k);
#pragma unroll
                for (int u = 0; u < kSortPerLane; ++u) rank[u] += w < v[u] ? 1 : 0;
            }
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < kSortPerLane; ++u)
            if (32 * u + lane < m) cell_atoms[b + rank[u]] = v[u];
    } else if (lane == 0) {
        const int e = b + m;
        for (int p = b + 1; p < e; ++p) {
            int v = cell_atoms[p];
            int q = p - 1;
            while (q >= b && cell_atoms[q] > v) { cell_atoms[q + 1] = cell_atoms[q]; --q; }
            cell_atoms[q + 1] = v;
        }
    }
    if (lane == 0) fill[c] = 0;
}

__global__ void __launch_bounds__(kSortBlock) k_sort_cells(int* __restrict__ cell_atoms, const int* __restrict__ cell_start, int* __restrict__ fill,
                             int ncell, const int* __restrict__ flags) {
    sort_cells_body(cell_atoms, cell_start, fill, ncell, flags, blockIdx.x);
}

// Per step: x_rel = x - cell origin as FP32 (the force kernels' coordinates), the weight
// w_i of the fixed zone, and the compaction of the atoms with w > 0.  FP64 runs at 1/64 of
// the FP32 rate on this GPU, so the region test is first taken in FP32 from the cell origin
// and x_rel (absolute error ~1e-5 A, far inside the pre-test margins); only atoms the FP32
// test cannot place (the switching shell and its edges) take the FP64 path.  The FP32
// residual of x_rel is formed on demand, for the energy pass (k_pos_lo).
__device__ __forceinline__ void prepare_body(const double* __restrict__ x, int n, const GridDev g, const DynDev dy,
                          const double* __restrict__ tptr, const int* __restrict__ cell,
                          const double* __restrict__ w_fixed, float4* __restrict__ pos4,
                          float* __restrict__ wout, int* __restrict__ ace_list, int* __restrict__ flags, int bid) {
    pdl_wait();
    __shared__ float sh[9];          // box origin, cell edges (orthorhombic), zone centre at time t
    if (threadIdx.x == 0 && dy.reg_kind == AP_REGION_SPHERE && g.ortho) {
        const double t = *tptr;
        for (int q = 0; q < 3; ++q) {
            sh[q] = (float)g.origin[q];
            sh[3 + q] = (float)g.cellvec[4 * q];
            sh[6 + q] = (float)(dy.reg_c0[q] - (dy.follow ? dy.ind_vel[q] * t : 0.0));
        }
    }
    __syncthreads();
    int i = bid * blockDim.x + threadIdx.x;
    float wf = 0.0f;
    bool need = false;                 // w > 0, decided in the precision w is given in
    if (i < n) {
        double r[3] = {x[i], x[n + i], x[2 * n + i]};
        int cc[3];
        cell_coords(g, cell[i], cc);
        double o[3];
        cell_origin(g, cc, o);
        const float hx = (float)(r[0] - o[0]), hy = (float)(r[1] - o[1]), hz = (float)(r[2] - o[2]);
        float u = 1.0f;
        if (dy.reg_kind == AP_REGION_CONST) {
            wf = (float)dy.w_const;
            u = (float)(1.0 - dy.w_const);
            need = dy.w_const > 0.0;
        } else if (dy.reg_kind == AP_REGION_EXPLICIT) {
            const double w = w_fixed[i];
            wf = (float)w;
            u = (float)(1.0 - w);
            need = w > 0.0;
        } else if (dy.reg_kind == AP_REGION_SPHERE) {
            float d2f = -1.0f;
            if (g.ortho) {
                const float h[3] = {hx, hy, hz};
                float d[3];
                for (int q = 0; q < 3; ++q) d[q] = (fmaf((float)cc[q], sh[3 + q], sh[q]) - sh[6 + q]) + h[q];
                d2f = min_image_d2_f32v(g, d);
            }
            if (d2f >= 0.0f && d2f < dy.reg_in2_lo) {
                wf = 1.0f;
                u = 0.0f;
            } else if (!(d2f > dy.reg_out2_hi)) {
                const double t = *tptr;
                double d[3];
                for (int q = 0; q < 3; ++q) d[q] = r[q] - (dy.reg_c0[q] - (dy.follow ? dy.ind_vel[q] * t : 0.0));
                min_image_vec(g, d);
                float dS;
                wf = switch_weight(d[0] * d[0] + d[1] * d[1] + d[2] * d[2], dy.r_in, dy.r_sw, &u, &dS);
            }
            need = wf > 0.0f;
        }
        pos4[i] = make_float4(hx, hy, hz, u);
        wout[i] = wf;
    }
    // warp-aggregated compaction of the atoms that need ACE
    unsigned mask = __ballot_sync(0xffffffffu, need);
    if (mask) {
        int lane = threadIdx.x & 31;
        int leader = __ffs(mask) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&flags[kFlagNAce], __popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (need) ace_list[base + __popc(mask & ((1u << lane) - 1u))] = i;
    }
}

__global__ void k_prepare(const double* __restrict__ x, int n, const GridDev g, const DynDev dy,
                          const double* __restrict__ tptr, const int* __restrict__ cell,
                          const double* __restrict__ w_fixed, float4* __restrict__ pos4,
                          float* __restrict__ wout, int* __restrict__ ace_list, int* __restrict__ flags) {
    prepare_body(x, n, g, dy, tptr, cell, w_fixed, pos4, wout, ace_list, flags, blockIdx.x);
}

// Full neighbour list, r < r_list.  Each atom's entries are written in order of distance
// band (kBands bands of r_list / kBands; within a band, in cell-scan order): the pair kernels
// visit the k-th entries of neighbouring atoms together, and with band-ordered lists those
// sit at similar distances, so the lanes of a warp mostly read the same pair-table segment.
// Two passes over the candidate cells: counts per band, then placement.  The cell-scan order
// is: offset codes in order, and within a cell its atoms in index order; both build kernels
// below visit candidates in that order, so they write identical lists.
constexpr int kBands = 16;
constexpr int kBuildBlock = 128;

// squared length of the pair vector x_rel_j + D[code] - x_rel_i, with every rounding fixed
// (no contraction left to the compiler), so that both build kernels include the same pairs
__device__ __forceinline__ float pair_r2(const float4& pj, const float4& d, const float4& p) {
    const float dx = __fsub_rn(__fadd_rn(pj.x, d.x), p.x);
    const float dy = __fsub_rn(__fadd_rn(pj.y, d.y), p.y);
    const float dz = __fsub_rn(__fadd_rn(pj.z, d.z), p.z);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// distance band of a list entry, r = r2 rsqrt(r2) with the hardware reciprocal square root:
// both build kernels evaluate it with the same instructions, so they order entries alike
__device__ __forceinline__ int list_band(float r2, float bscale) {
    return min(kBands - 1, (int)(r2 * rsqrtf(r2) * bscale));
}

__device__ __forceinline__ void load_codes(const GridDev& g, const float4* __restrict__ Dtab, float4* D, char4* O) {
    const int w1 = 2 * g.S[1] + 1, w2 = 2 * g.S[2] + 1;
    for (int k = threadIdx.x; k < g.ncode; k += blockDim.x) {
        D[k] = Dtab[k];
        O[k] = make_char4((char)(k / (w1 * w2) - g.S[0]), (char)((k / w2) % w1 - g.S[1]), (char)(k % w2 - g.S[2]), 0);
    }
}

// count the band entries of atom i (pass 1), then place them (pass 2) from the band counters
// band[b * bstride] of this thread; scan(visit) runs the cell scan.  Returns the entry count.
template <class BT, class Scan>
__device__ __forceinline__ int place_banded(int i, int n, int* __restrict__ nbr, int* __restrict__ nrow,
                                            int* __restrict__ nnbr, int cap,
                                            int* __restrict__ flags, int count_only, BT* band, int bstride, Scan&& scan) {
    for (int b = 0; b < kBands; ++b) band[b * bstride] = 0;
    int cnt = 0;
    scan([&](int, int b) { ++cnt; band[b * bstride] += 1; });
    if (!count_only) {
        int run = 0;
        for (int b = 0; b < kBands; ++b) {
            const int c = band[b * bstride];
            band[b * bstride] = (BT)run;
            run += c;
        }
        scan([&](int e, int b) {
            const int at = band[b * bstride];
            band[b * bstride] = (BT)(at + 1);
            if (at < cap) {
                nbr[(size_t)at * n + i] = e;
                nrow[(size_t)i * cap + at] = e;
            }
        });
        nnbr[i] = cnt < cap ? cnt : cap;
        if (cnt > cap) atomicOr(&flags[kFlagErr], kErrCapacity);
    }
    return cnt;
}

// the largest entry count of a warp into flags[kFlagMaxNbr] (one atomic per warp)
__device__ __forceinline__ void max_nbr_warp(int cnt, int* flags) {
    const int m = __reduce_max_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0) atomicMax(&flags[kFlagMaxNbr], m);
}

// atom i from global memory: the ranges of four cells, and then the indices and positions of
// up to four atoms of a cell, are loaded together (the scan is a chain of dependent loads)
template <class BT>
__device__ __forceinline__ int build_atom_global(int i, const float4* __restrict__ pos4, const int* __restrict__ cell,
                                                 int n, const GridDev& g, const float4* D, const char4* O,
                                                 const int* __restrict__ cell_start, const int* __restrict__ cell_atoms,
                                                 int* __restrict__ nbr, int* __restrict__ nrow, int* __restrict__ nnbr, int cap,
                                                 int* __restrict__ flags, int count_only, BT* band, int bstride) {
    const float4 p = pos4[i];
    int cc[3];
    cell_coords(g, cell[i], cc);
    const float bscale = (float)kBands * rsqrtf(g.rlist2);
    auto scan = [&](auto&& visit) {
        for (int c0 = 0; c0 < g.ncode; c0 += 4) {
            int beg[4], end[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                beg[u] = end[u] = 0;
                const int code = c0 + u;
                if (code >= g.ncode) continue;
                const char4 oc = O[code];
                const int o[3] = {oc.x, oc.y, oc.z};
                int nc[3];
                bool ok = true;
                for (int k = 0; k < 3; ++k) {
                    int v = cc[k] + o[k];             // |o| <= S <= 2: at most two wraps
                    if (g.periodic[k]) {
                        while (v < 0) v += g.nc[k];
                        while (v >= g.nc[k]) v -= g.nc[k];
                    } else if (v < 0 || v >= g.nc[k]) {
                        ok = false;
                    }
                    nc[k] = v;
                }
                if (!ok) continue;
                const int cn = (nc[0] * g.nc[1] + nc[1]) * g.nc[2] + nc[2];
                beg[u] = cell_start[cn];
                end[u] = cell_start[cn + 1];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int code = c0 + u;
                if (beg[u] >= end[u]) continue;
                const bool self_cell = O[code].x == 0 && O[code].y == 0 && O[code].z == 0;
                const float4 d = D[code];
                for (int q0 = beg[u]; q0 < end[u]; q0 += 4) {
                    int jj[4];
                    float4 pj[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) jj[t] = q0 + t < end[u] ? cell_atoms[q0 + t] : -1;
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (jj[t] >= 0) pj[t] = pos4[jj[t]];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int j = jj[t];
                        if (j < 0 || (self_cell && j == i)) continue;
                        const float r2 = pair_r2(pj[t], d, p);
                        if (r2 < g.rlist2) visit(j | (code << kNbrShift), list_band(r2, bscale));
                    }
                }
            }
        }
    };
    return place_banded(i, n, nbr, nrow, nnbr, cap, flags, count_only, band, bstride, scan);
}

// thread per atom, atoms in index order (the batched launches)
__device__ __forceinline__ void build_body(const float4* __restrict__ pos4, const int* __restrict__ cell,
                                                       int n, const GridDev g, const float4* __restrict__ Dtab,
                                                       const int* __restrict__ cell_start,
                                                       const int* __restrict__ cell_atoms, int* __restrict__ nbr,
                                                       int* __restrict__ nrow, int* __restrict__ nnbr, int cap,
                                                       int* __restrict__ flags, int count_only, int bid) {
    pdl_wait();
    if (!count_only && flags[kFlagRebuild] == 0) return;
    __shared__ float4 D[125];
    __shared__ char4 O[125];                          // cell offset of each code (no divisions in the scan)
    __shared__ int band_at[kBands][kBuildBlock];      // counts, then running write positions
    load_codes(g, Dtab, D, O);
    __syncthreads();
    const int i = bid * blockDim.x + threadIdx.x;
    int cnt = 0;
    if (i < n)
        cnt = build_atom_global(i, pos4, cell, n, g, D, O, cell_start, cell_atoms, nbr, nrow, nnbr, cap, flags, count_only,
                                &band_at[0][threadIdx.x], kBuildBlock);
    max_nbr_warp(cnt, flags);
}

__global__ void __launch_bounds__(kBuildBlock) k_build(const float4* __restrict__ pos4, const int* __restrict__ cell,
                                                       int n, const GridDev g, const float4* __restrict__ Dtab,
                                                       const int* __restrict__ cell_start,
                                                       const int* __restrict__ cell_atoms, int* __restrict__ nbr,
                                                       int* __restrict__ nrow, int* __restrict__ nnbr, int cap,
                                                       int* __restrict__ flags, int count_only) {
    build_body(pos4, cell, n, g, Dtab, cell_start, cell_atoms, nbr, nrow, nnbr, cap, flags, count_only, blockIdx.x);
}

// Staged build: one block per box of sb cells.  The block first copies the positions of every
// atom of the cells within S of its box (the region) into shared memory, then each thread
// scans the 27 (up to 125) cells of one of the box's atoms there, once: each hit goes to the
// atom's row of the scratch list (its staged slot, code and band packed in one int, stored
// 16 bytes at a time) while the band counts accumulate, and the row is then placed by band.
// The per-thread kernel above scans twice instead (counts, then placement).  A block whose
// region holds more than kStCap atoms scans from global memory like the per-thread kernel.
constexpr int kStBlock = 256;
constexpr int kStCap = 3072;          // staged atoms per block (48 KB of dynamic shared memory; < 4096)
constexpr int kStRegCap = 216;        // region cells per block
constexpr int kStOwnCap = 27;         // cells per box

__global__ void __launch_bounds__(kStBlock) k_build_staged(const float4* __restrict__ pos4, const int* __restrict__ cell,
                                                          int n, const GridDev g, const float4* __restrict__ Dtab,
                                                          const int* __restrict__ cell_start,
                                                          const int* __restrict__ cell_atoms, int* __restrict__ nbr,
                                                          int* __restrict__ nrow, int* __restrict__ tmp,
                                                          int* __restrict__ nnbr, int cap,
                                                          int* __restrict__ flags, int count_only, int3 sb, int3 nsb) {
    pdl_wait();
    if (!count_only && flags[kFlagRebuild] == 0) return;
    extern __shared__ float4 st[];                   // staged x_rel, with the atom index in .w
    __shared__ int rbeg[kStRegCap + 1];
    __shared__ int rgc[kStRegCap];                   // global cell of a region cell, -1 beyond a free face
    __shared__ int own_pre[kStOwnCap + 1];
    __shared__ int own_reg[kStOwnCap];
    __shared__ unsigned short band[kBands][kStBlock];
    __shared__ float4 D[125];
    __shared__ char4 O[125];
    __shared__ int wsum[kStBlock / 32];
    load_codes(g, Dtab, D, O);
    const int bx = blockIdx.x / (nsb.y * nsb.z), by = (blockIdx.x / nsb.z) % nsb.y, bz = blockIdx.x % nsb.z;
    const int base[3] = {bx * sb.x, by * sb.y, bz * sb.z};
    const int ext[3] = {min(sb.x, g.nc[0] - base[0]), min(sb.y, g.nc[1] - base[1]), min(sb.z, g.nc[2] - base[2])};
    const int R1 = ext[1] + 2 * g.S[1], R2 = ext[2] + 2 * g.S[2];
    const int nreg = (ext[0] + 2 * g.S[0]) * R1 * R2;     // <= kStRegCap (host)
    // region cells, their atom counts and the exclusive prefix of the counts
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int cntr = 0;
    if (tid < nreg) {
        const int l[3] = {tid / (R1 * R2), (tid / R2) % R1, tid % R2};
        int v[3];
        bool ok = true;
        for (int k = 0; k < 3; ++k) {
            int x = base[k] - g.S[k] + l[k];
            if (g.periodic[k]) {
                while (x < 0) x += g.nc[k];
                while (x >= g.nc[k]) x -= g.nc[k];
            } else if (x < 0 || x >= g.nc[k]) {
                ok = false;
            }
            v[k] = x;
        }
        const int gc = ok ? (v[0] * g.nc[1] + v[1]) * g.nc[2] + v[2] : -1;
        rgc[tid] = gc;
        if (ok) cntr = cell_start[gc + 1] - cell_start[gc];
    }
    int incl = cntr;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    int wpre = 0;
    for (int w = 0; w < wid; ++w) wpre += wsum[w];
    if (tid < nreg) rbeg[tid + 1] = wpre + incl;
    if (tid == 0) {
        rbeg[0] = 0;
        int k = 0;
        for (int a0 = 0; a0 < ext[0]; ++a0)
            for (int a1 = 0; a1 < ext[1]; ++a1)
                for (int a2 = 0; a2 < ext[2]; ++a2, ++k) own_reg[k] = ((a0 + g.S[0]) * R1 + (a1 + g.S[1])) * R2 + (a2 + g.S[2]);
    }
    __syncthreads();
    const int nown = ext[0] * ext[1] * ext[2];
    if (tid == 0) {
        int run = 0;
        for (int k = 0; k < nown; ++k) {
            own_pre[k] = run;
            run += rbeg[own_reg[k] + 1] - rbeg[own_reg[k]];
        }
        own_pre[nown] = run;
    }
    const int total = rbeg[nreg];
    const bool staged = total <= kStCap;
    if (staged) {
        for (int q = tid; q < total; q += kStBlock) {
            int lo = 0, hi = nreg - 1;                   // region cell r with rbeg[r] <= q < rbeg[r + 1]
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (rbeg[mid] <= q) lo = mid; else hi = mid - 1;
            }
            const int j = cell_atoms[cell_start[rgc[lo]] + (q - rbeg[lo])];
            const float4 pj = pos4[j];
            st[q] = make_float4(pj.x, pj.y, pj.z, __int_as_float(j));
        }
    }
    __syncthreads();
    const int n_atoms_box = own_pre[nown];
    const float bscale = (float)kBands * rsqrtf(g.rlist2);
    for (int t0 = 0; t0 < n_atoms_box; t0 += kStBlock) {
        const int t = t0 + tid;
        int cnt = 0;
        if (t < n_atoms_box) {
            int oc = 0;
            while (own_pre[oc + 1] <= t) ++oc;
            const int r0 = own_reg[oc];
            if (staged) {
                const int q = rbeg[r0] + (t - own_pre[oc]);
                const float4 p = st[q];
                const int i = __float_as_int(p.w);
                const int l0 = r0 / (R1 * R2), l1 = (r0 / R2) % R1, l2 = r0 % R2;
                // visit(q, code, band) for every candidate inside r_list, in cell-scan order
                auto scan = [&](auto&& visit) {
                    for (int code = 0; code < g.ncode; ++code) {
                        const char4 oc4 = O[code];
                        const int rr = ((l0 + oc4.x) * R1 + (l1 + oc4.y)) * R2 + (l2 + oc4.z);
                        const int qb = rbeg[rr], qe = rbeg[rr + 1];
                        if (qb >= qe) continue;
                        const bool self_cell = oc4.x == 0 && oc4.y == 0 && oc4.z == 0;
                        const float4 d = D[code];
                        // two candidates per iteration (independent chains), visited in order
                        int qq = qb;
                        for (; qq + 2 <= qe; qq += 2) {
                            const float4 pa = st[qq], pb = st[qq + 1];
                            const float ra = pair_r2(pa, d, p), rb = pair_r2(pb, d, p);
                            const bool ha = ra < g.rlist2 && !(self_cell && __float_as_int(pa.w) == i);
                            const bool hb = rb < g.rlist2 && !(self_cell && __float_as_int(pb.w) == i);
                            if (ha) visit(qq, code, list_band(ra, bscale));
                            if (hb) visit(qq + 1, code, list_band(rb, bscale));
                        }
                        if (qq < qe) {
                            const float4 pa = st[qq];
                            const float ra = pair_r2(pa, d, p);
                            if (ra < g.rlist2 && !(self_cell && __float_as_int(pa.w) == i))
                                visit(qq, code, list_band(ra, bscale));
                        }
                    }
                };
                if (count_only) {
                    scan([&](int, int, int) { ++cnt; });
                } else {
                    for (int bb = 0; bb < kBands; ++bb) band[bb][tid] = 0;
                    int4* trow = reinterpret_cast<int4*>(tmp + (size_t)i * cap);     // cap % 4 == 0
                    int4 w4 = make_int4(0, 0, 0, 0);
                    scan([&](int q, int code, int bb) {
                        band[bb][tid] += 1;
                        if (cnt < cap) {                  // selects, not branches: lanes stay converged
                            const int v = q | (code << 12) | (bb << 19), sl = cnt & 3;
                            w4.x = sl == 0 ? v : w4.x;
                            w4.y = sl == 1 ? v : w4.y;
                            w4.z = sl == 2 ? v : w4.z;
                            w4.w = sl == 3 ? v : w4.w;
                            if (sl == 3) trow[cnt >> 2] = w4;
                        }
                        ++cnt;
                    });
                    const int m = cnt < cap ? cnt : cap;
                    if (m & 3) trow[m >> 2] = w4;                 // the partial last vector
                    int run = 0;
                    for (int bb = 0; bb < kBands; ++bb) {
                        const int c = band[bb][tid];
                        band[bb][tid] = (unsigned short)run;
                        run += c;
                    }
                    if (cnt > cap) {
                        // overflow: the row holds only the first cap hits in scan order, whose
                        // band positions would leave some slots below cap unwritten; place the
                        // cap lowest positions by a second scan instead (the list is then the
                        // per-thread kernel's, and every slot below nnbr holds a valid entry)
                        scan([&](int q, int code, int bb) {
                            const int at = band[bb][tid];
                            band[bb][tid] = (unsigned short)(at + 1);
                            if (at < cap) {
                                const int e = __float_as_int(st[q].w) | (code << kNbrShift);
                                nbr[(size_t)at * n + i] = e;
                                nrow[(size_t)i * cap + at] = e;
                            }
                        });
                    }
                    for (int k4 = 0; k4 < m && cnt <= cap; k4 += 4) {
                        const int4 v4 = trow[k4 >> 2];
                        const int vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if (k4 + u >= m) break;
                            const int v = vv[u], bb = v >> 19, code = (v >> 12) & 0x7f;
                            const int j = __float_as_int(st[v & 0xfff].w);
                            const int at = band[bb][tid];
                            band[bb][tid] = (unsigned short)(at + 1);
                            if (at < cap) {
                                nbr[(size_t)at * n + i] = j | (code << kNbrShift);
                                nrow[(size_t)i * cap + at] = j | (code << kNbrShift);
                            }
                        }
                    }
                    nnbr[i] = m;
                    if (cnt > cap) atomicOr(&flags[kFlagErr], kErrCapacity);
                }
            } else {
                const int i = cell_atoms[cell_start[rgc[r0]] + (t - own_pre[oc])];
                cnt = build_atom_global(i, pos4, cell, n, g, D, O, cell_start, cell_atoms, nbr, nrow, nnbr, cap, flags,
                                        count_only, &band[0][tid], kStBlock);
            }
        }
        max_nbr_warp(cnt, flags);
    }
}

// the box of cells of one staged block: up to 3 cells per axis, as many as keep the region
// within kStRegCap cells and, at 0.1 atoms / A^3 (metallic density bound), within kStCap atoms
// and the box near 256 atoms at the typical two thirds of that bound
void staged_boxes(const GridDev& g, int3& sb, int3& nsb) {
    double vol = 1.0;
    for (int k = 0; k < 3; ++k) vol *= g.cw[k];
    const double a = 0.1 * vol;
    int best[3] = {1, 1, 1}, best_own = 0;
    for (int s0 = 1; s0 <= std::min(3, g.nc[0]); ++s0)
        for (int s1 = 1; s1 <= std::min(3, g.nc[1]); ++s1)
            for (int s2 = 1; s2 <= std::min(3, g.nc[2]); ++s2) {
                const int own = s0 * s1 * s2;
                const int reg = (s0 + 2 * g.S[0]) * (s1 + 2 * g.S[1]) * (s2 + 2 * g.S[2]);
                if (reg > kStRegCap || reg * a > kStCap || own * a * (2.0 / 3.0) > kStBlock) continue;
                if (own > best_own) { best_own = own; best[0] = s0; best[1] = s1; best[2] = s2; }
            }
    sb = make_int3(best[0], best[1], best[2]);
    nsb = make_int3((g.nc[0] + sb.x - 1) / sb.x, (g.nc[1] + sb.y - 1) / sb.y, (g.nc[2] + sb.z - 1) / sb.z);
}

// batched launches: block b of a launch over several contexts acts as block b - start[k] of
// context k (start: the per-context prefix of blocks)
__device__ __forceinline__ const CtxDev& batch_ctx(const BatchTable& t, const int* start, int& bid) {
    const int k = batch_find(start, t.nctx, blockIdx.x);
    bid = blockIdx.x - start[k];
    return *t.d[k];
}

__global__ void kb_check(const BatchTable t) {
    int bid;
    const CtxDev& c = batch_ctx(t, t.b256, bid);
    check_body(c.x, c.xb, c.n, c.lim2, c.flags, bid);
}

__global__ void kb_wrap_bin(const BatchTable t) {
    int bid;
    const CtxDev& c = batch_ctx(t, t.b256, bid);
    wrap_bin_body(c.x, c.xb, c.n, c.grid, c.cell, c.cell_count, c.flags, bid);
}

__global__ void kb_scan(const BatchTable t) {          // one block per context
    const CtxDev& c = *t.d[blockIdx.x];
    scan_body(c.cell_count, c.cell_start, c.grid.ncell, c.flags, 0);
}

__global__ void kb_scatter(const BatchTable t) {
    int bid;
    const CtxDev& c = batch_ctx(t, t.b256, bid);
    scatter_body(c.cell, c.n, c.cell_start, c.cell_count, c.cell_atoms, c.flags, bid);
}

__global__ void kb_sort_cells(const BatchTable t) {
    int bid;
    const CtxDev& c = batch_ctx(t, t.bcell, bid);
    sort_cells_body(c.cell_atoms, c.cell_start, c.cell_count, c.grid.ncell, c.flags, bid);
}

__global__ void kb_prepare(const BatchTable t) {
    int bid;
    const CtxDev& c = batch_ctx(t, t.b256, bid);
    prepare_body(c.x, c.n, c.grid, c.dyn, c.d_time, c.cell, c.w_fixed, c.pos4, c.w, c.ace_list, c.flags, bid);
}

__global__ void __launch_bounds__(kBuildBlock) kb_build(const BatchTable t) {
    int bid;
    const CtxDev& c = batch_ctx(t, t.b128, bid);
    build_body(c.pos4, c.cell, c.n, c.grid, c.D, c.cell_start, c.cell_atoms, c.nbr, c.nbr_row, c.nnbr, c.cap, c.flags, 0,
               bid);
}

}  // namespace

int launch_batch_check(const BatchTable& t, cudaStream_t s) {
    launch_pdl(kb_check, t.b256[t.nctx], 256, 0, s, t);
    return 1;
}

int launch_batch_rebuild(const BatchTable& t, cudaStream_t s) {
    launch_pdl(kb_wrap_bin, t.b256[t.nctx], 256, 0, s, t);
    launch_pdl(kb_scan, t.nctx, 1024, 0, s, t);
    launch_pdl(kb_scatter, t.b256[t.nctx], 256, 0, s, t);
    launch_pdl(kb_sort_cells, t.bcell[t.nctx], kSortBlock, 0, s, t);
    return 4;
}

int launch_batch_prepare(const BatchTable& t, cudaStream_t s) {
    launch_pdl(kb_prepare, t.b256[t.nctx], 256, 0, s, t);
    launch_pdl(kb_build, t.b128[t.nctx], kBuildBlock, 0, s, t);
    return 2;
}

int launch_check(Ctx& c, cudaStream_t s) {
    double lim = 0.5 * c.skin;
    launch_pdl(k_check, (c.n + 255) / 256, 256, 0, s, c.x, c.xb, c.n, lim * lim, c.flags);
    return 1;
}

int launch_rebuild(Ctx& c, cudaStream_t s) {
    int nb = (c.n + 255) / 256;
    launch_pdl(k_wrap_bin, nb, 256, 0, s, c.x, c.xb, c.n, c.grid, c.cell, c.cell_count, c.flags);
    launch_pdl(k_scan, 1, 1024, 0, s, c.cell_count, c.cell_start, c.grid.ncell, c.flags);
    launch_pdl(k_scatter, nb, 256, 0, s, c.cell, c.n, c.cell_start, c.cell_count, c.cell_atoms, c.flags);
    launch_pdl(k_sort_cells, (c.grid.ncell + kSortBlock / 32 - 1) / (kSortBlock / 32), kSortBlock, 0, s, c.cell_atoms,
               c.cell_start, c.cell_count, c.grid.ncell, c.flags);
    return 4;
}

int launch_prepare(Ctx& c, cudaStream_t s) {
    launch_pdl(k_prepare, (c.n + 255) / 256, 256, 0, s, c.x, c.n, c.grid, c.dyn, c.d_time, c.cell, c.w_fixed, c.pos4,
               c.w, c.ace_list, c.flags);
    return 1;
}

int launch_build(Ctx& c, cudaStream_t s, int count_only) {
    const int reg_min = (1 + 2 * c.grid.S[0]) * (1 + 2 * c.grid.S[1]) * (1 + 2 * c.grid.S[2]);
    if (reg_min > kStRegCap) {                       // (S = 2 on every axis) per-thread scan
        launch_pdl(k_build, (c.n + kBuildBlock - 1) / kBuildBlock, kBuildBlock, 0, s, c.pos4, c.cell, c.n, c.grid, c.D,
                   c.cell_start, c.cell_atoms, c.nbr, c.nbr_row, c.nnbr, c.cap, c.flags, count_only);
        return 1;
    }
    static int attr_dev = -1;
    if (attr_dev != c.dev) {
        cudaFuncSetAttribute(k_build_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kStCap * sizeof(float4)));
        attr_dev = c.dev;
    }
    int3 sb, nsb;
    staged_boxes(c.grid, sb, nsb);
    launch_pdl(k_build_staged, nsb.x * nsb.y * nsb.z, kStBlock, kStCap * sizeof(float4), s, c.pos4, c.cell, c.n, c.grid,
               c.D, c.cell_start, c.cell_atoms, c.nbr, c.nbr_row, c.nbr_tmp, c.nnbr, c.cap, c.flags, count_only, sb, nsb);
    return 1;
}

}  // namespace ap
