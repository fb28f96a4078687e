// ap_internal.h -- device data layout, context and kernel launchers of the AP library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>

#include "ap.h"
#include "ace_pattern.h"

namespace ap {

// ---------------------------------------------------------------------------------
// EAM functions as piecewise polynomials (degree <= 5) in t = r - mid on each interval.
// Built on the host in FP64 from the Appendix B forms, evaluated on the device in FP32.
// ---------------------------------------------------------------------------------
constexpr int kNBin = 256;

// EAM pair functions zeta(r) and Phi(r) on one merged partition of [0, rc): the union of
// both functions' knots (and of r_lo, r_hi, r_cut^rho), split into pieces of at most
// 0.25 A.  On each segment zeta is a cubic and Phi a cubic, the quintic bridge or the ZBL
// form, expanded in FP64 on the host about the segment midpoint (an FP32 number) and
// stored in FP32 with the constant terms' residuals for the compensated energy pass.
constexpr int kMaxSeg = 48;
constexpr int kSegCubic = 0, kSegQuintic = 1, kSegZbl = 2;   // kinds of the Phi piece

struct EamSeg {
    float4 q0;                // (mid, zeta c1, zeta c2, zeta c3)
    float4 q1;                // (Phi c1, Phi c2, Phi c3, Phi c0)
    float4 q2;                // (zeta c0, zeta c0 residual, Phi c0 residual, kind)
    float4 q3;                // (Phi c4, Phi c5, 0, 0): the quintic bridge only
};

// r in bin b = (int)(r * bin_inv) lies in segment k + (r >= s1) + (r >= s2); special is set
// when one of those segments has a non-cubic Phi piece
struct EamBin {
    int k;
    float s1, s2;
    int special;
};

struct alignas(16) EamDev {
    EamSeg seg[kMaxSeg];
    EamBin bin[kNBin];
    int nseg, pad0;
    float rc_rho, rc_phi;     // zeta and Phi vanish at and beyond these
    float rc;                 // max of the two
    float bin_inv;            // kNBin / rc
    float zbl_k;              // Z^2 / (4 pi eps0), eV Angstrom
    float zbl_ainv;           // 1 / a_ZBL
    double F_a1, F_a2, F_dxi;
};

// ACE coefficient tensors on the host, zero-padded to full n-ranges (a basis function sits at
// its sorted (n, l) position; the other orderings carry zero); the device tables (AceTc)
// are built from them.
struct AceDev {
    float c3[2][kNT][8][64];  // [density][l-triple][n3][n1 * 8 + n2]
    float c2[2][5][64];       // [density][l][n1 * 8 + n2]
    float c1[2][8];           // [density][n]
    float c1_0, c2_0, nref_inv, rc;
};

// Coefficient tables of the tensor-core contraction.  The five (0, l, l) triples, whose
// Gaunt coefficients are delta_{m2 m3} G_l (G_l = 1/sqrt(4 pi)), are stored for the
// two-factor pass as c0ll[p][l][n1 / 4][c0ll_pos(n2 * 8 + n3)][n1 % 4] = G_l C3[n1, n2, n3]:
// rows of four n1 (16 bytes) at a permuted pair position, so that the pass's 16-byte reads
// (the pairs 8 g + 2 t + j of an mma accumulator tile) fall on distinct bank groups.  For the other nine triples
// (t = 5 .. 13) and density p the coefficients form a 64 x 8 matrix C[q = n1 * 8 + n2][n3].
// For the l1 = l2 triples the product of the first two factors is symmetric in (n1, n2): their
// rows are packed, row sym_pair(n1, n2) (n1 <= n2, 36 rows, the rest zero) holding the mean of
// the coefficients of (n1, n2) and (n2, n1).  Each entry is split into two
// TF32 numbers hi + lo (13 low mantissa bits zero) for 3xTF32 products, and n3 is stored at
// position n3 ^ (4 ((q >> 2) & 1)) so that the kernel's two fragment reads of the matrix
// (as C and as its transpose) are free of shared-memory bank conflicts.
// position of pair q = 8 g + 2 t + j (g = q / 8, t = (q / 2) % 4, j = q % 2) in the c0ll rows:
// (g / 2, j, g % 2, t), so that the eight threads of a quarter warp (g in {2i, 2i + 1}, all t)
// read eight distinct 16-byte units modulo 128 bytes
__host__ __device__ constexpr int c0ll_pos(int q) {
    return (q & 0x30) | ((q & 1) << 3) | (((q >> 3) & 1) << 2) | ((q >> 1) & 3);
}
// packed index of the unordered pair n1 <= n2 (row-major upper triangle of 8 x 8)
constexpr int kSymPairs = 36;
__host__ __device__ constexpr int sym_pair(int n1, int n2) { return n1 * (15 - n1) / 2 + n2; }
constexpr int kNT3 = 9;             // l-triples on tensor cores
constexpr int kTcTriple0 = 5;       // ... t = 5 .. 13
struct alignas(16) AceTc {
    float c3[2][2][kNT3][64][8];    // [hi/lo][density][t - 5][q][n3 (swizzled)]
    float c0ll[2][5][2][64][4];     // [density][l][n1 / 4][c0ll_pos(n2 * 8 + n3)][n1 % 4]
    float c2[2][5][64];             // as AceDev
    float c1[2][8];
    float c1_0, c2_0, nref_inv, rc;
};

// Cell grid: cells are the parallelepipeds of the box divided n_d times along each edge;
// an atom's FP32 position is stored relative to its cell's origin, and a neighbour in
// the cell offset o (per edge, -S..S) is at x_rel_j + D[code(o)] - x_rel_i.
struct GridDev {
    double origin[3];
    double h[9];              // edge vectors as rows
    double hinv[9];           // s = (r - origin) . hinv gives fractional coordinates
    double cellvec[9];        // h rows / n_d
    double cw[3];             // perpendicular width of a cell along each edge
    int periodic[3];
    int nc[3];
    int S[3];
    int ncode;                // (2 S0 + 1)(2 S1 + 1)(2 S2 + 1) <= 125
    int ncell;
    float rlist2;
    int ortho;                // edge vectors along x, y, z
    double L[3], Linv[3];     // edge lengths (orthorhombic boxes)
    float Lf[3], Linvf[3];    // the same in FP32 (pre-tests only)
};

struct DynDev {               // time-dependent geometry; time is read from device memory
    double reg_c0[3];
    double r_in, r_sw, w_const;
    int reg_kind;
    int follow;
    int ind_on;
    int pad;
    double ind_c0[3], ind_vel[3], ind_dir[3];
    double R, K;
    // FP32 pre-tests (orthorhombic boxes): below reg_in2_lo an atom is surely inside the
    // inner radius, above reg_out2_hi surely outside the shell, above ind_R2_hi surely
    // outside the indenter; squared radii with a 1e-5 relative margin
    float reg_in2_lo, reg_out2_hi, ind_R2_hi, pad2;
};

enum : int { kFlagRebuild = 0, kFlagNAce = 1, kFlagErr = 2, kFlagBad = 3, kFlagMaxNbr = 4, kFlagRebuilds = 5, kFlagCount = 8 };
enum : int { kErrDomain = 1, kErrCapacity = 2, kErrAceCapacity = 4 };

constexpr int kNbrShift = 25;               // neighbour entry = j | code << 25
constexpr int kNbrMask = (1 << kNbrShift) - 1;
constexpr int kMaxAtoms = (1 << kNbrShift) - 1;
constexpr double kFixScale = 1099511627776.0;   // 2^40: fixed-point scale of ACE force sums
constexpr double kLoadScale = 4294967296.0;      // 2^32: fixed-point scale of the load history
constexpr double kFtm = 0.0096485332;           // 1 eV/(Angstrom amu) in Angstrom/fs^2
constexpr int kAceNbrCap = 128;                 // neighbours within the ACE cutoff per atom
constexpr int kRedBlock = 256;

struct Ctx {
    int n = 0, dev = 0;
    cudaStream_t stream = nullptr;
    double mass = 1.0, skin = 1.0, rc_eam = 0.0, rc_ace = 0.0, rc_list = 0.0;
    int ace_prec = AP_ACE_FP32;
    int region_kind = AP_REGION_NONE;

    EamDev eam_h{};
    EamDev* eam_d = nullptr;
    bool energy_fresh = false;                           // energy pass done for the last forces
    AceDev* ace_h = nullptr;                             // host coefficient tensors
    const AceTc* ace_tc_d = nullptr;                     // device ACE tables (shared per potential)
    struct CtxDev* desc_d = nullptr;                     // device descriptor for batched launches
    unsigned char desc_h[1024];                          // its last uploaded contents
    bool desc_valid = false;
    GridDev grid{};
    float4* D = nullptr;                                 // cell-offset vectors, FP32
    float4* Dlo = nullptr;                               // their FP32 residuals (o . cellvec - D)
    DynDev dyn{};

    double *x = nullptr, *v = nullptr, *xb = nullptr;   // SoA [3][n]
    float* f = nullptr;                                  // SoA [3][n]
    float4* pos4 = nullptr;                              // x_rel (3) and u = 1 - w
    float4* pos_lo = nullptr;                            // FP32 residual of x_rel (energy pass)
    float* uxi = nullptr;                                // u_i xi'(rho_i)
    float* w = nullptr;
    double* e_emb = nullptr;                             // xi(rho_i) + Delta xi
    double* e_eam = nullptr;                             // E_i^EAM (FP64) of the force pass (the blend's -grad w term)
    double* e_eam_acc = nullptr;                         // E_i^EAM of the compensated energy pass
    float* e_ace = nullptr;                              // E_i^ACE - c1_0
    float* ace_A = nullptr;                              // [n_ace][25][8] atomic base of the compacted atoms
    float* ace_dA = nullptr;                             // [n_ace][25][8] dE/dA
    double ace_c1_0 = 0.0;
    float* vir_eam = nullptr;                            // [6][n]
    float* vir_ace = nullptr;                            // [6][n]
    unsigned long long* acc = nullptr;                   // [3][n] fixed-point ACE forces
    unsigned char* fixed = nullptr;
    double* w_fixed = nullptr;
    int *cell = nullptr, *cell_count = nullptr, *cell_start = nullptr, *cell_atoms = nullptr;
    int* nbr = nullptr;                                  // [cap][n]
    int* nbr_tmp = nullptr;                              // [n][cap]: hits of the staged list build
    int* nbr_row = nullptr;                              // [n][cap]: nbr row by row (the warp-per-atom ACE kernels)
    int* nnbr = nullptr;
    int cap = 0;
    int* ace_list = nullptr;
    int* flags = nullptr;                                // kFlag*
    double* d_time = nullptr;
    double* partials = nullptr;
    double* totals = nullptr;                            // 16 doubles
    double* e_atom = nullptr;
    double* csp_sum = nullptr;                           // CSP block sums (valid evaluations)
    int* csp_under = nullptr;                            // evaluations that found a surface atom
    float *csp_w0 = nullptr, *csp_wnew = nullptr;
    int *csp_seeds = nullptr, *csp_nseed = nullptr;
    int csp_nacc = 0;                                    // evaluations in the current block
    int thermo_kind = 0;                                 // AP_THERMO_*
    double nh_nfkt = 0.0, nh_Q = 0.0;                    // N_f k_B T (eV) and Q (eV fs^2)
    unsigned char* thermo_group = nullptr;
    double* nh_state = nullptr;                          // xi (1/fs), eta, velocity scale of the last half step
    double* nh_partials = nullptr;                       // [nred] group kinetic energies
    double lv_drag = 0.0, lv_sig = 0.0;                  // Langevin drag (eV fs/A^2) and noise amplitude (eV/A)
    unsigned long long lv_seed = 0;
    long long lv_base = 0;                               // step count at ap_set_thermostat
    int lv_zero_every = 0;
    long long* d_step = nullptr;                         // device step counter (advanced by k_kick_drift)
    long long* load_ring = nullptr;                      // [load_cap] load of step k in slot k % load_cap (2^-32 eV/A)
    double* load_ring_t = nullptr;                       // [load_cap] time of that step (fs)
    int load_cap = 0;                                    // 0: no load history is recorded
    long long load_step0 = 0;                            // step count when recording started
    double* com = nullptr;                               // [4 nred + 4] momentum-zeroing partials and result
    double* pos_stage = nullptr;                         // n x 3 host-transfer staging
    float* f_stage = nullptr;                            // n x 3 host-transfer staging
    int nred = 0;
    int ncell_cap = 0;                                   // allocated length of the cell arrays
    long long layout_gen = 0;                            // bumped when kernel arguments change

    int* h_flags = nullptr;                              // pinned
    double* h_totals = nullptr;                          // pinned
    long long launches = 0, rebuilds = 0, step = 0;
    size_t dev_bytes = 0;                                // device bytes this context holds
    double t = 0.0;
    bool forces_valid = false;
    std::string err;

    int prof = 0;                                        // 0 off, 1 every stage, 2 the ACE contraction only
    cudaEvent_t ev[2] = {nullptr, nullptr};
    double stage_ms[AP_NSTAGE] = {0};
    long long stage_n[AP_NSTAGE] = {0};
};

// Programmatic dependent launch.  The kernels of a force pass and a step are launched with
// launch_pdl, so that each may be scheduled while the previous kernel on the stream drains.
// Each calls pdl_wait() before its first access to device data that an earlier kernel
// writes or reads; before it, only constant tables (potential, cell offsets) are read.  A
// kernel that ends only after its wait keeps the order transitive.  Launched plainly, the
// wait returns at once.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

static_assert(sizeof(EamDev) % 16 == 0, "EamDev is staged in 16-byte words");
static_assert(sizeof(AceDev) % 16 == 0, "AceDev is staged in 16-byte words");
static_assert(sizeof(AceTc) % 16 == 0, "AceTc is staged in 16-byte words");

// kernel launchers (one per stage); each returns the number of kernels launched
int launch_rebuild(Ctx& c, cudaStream_t s);          // wrap, bin, scan, scatter, sort (skip when no rebuild)
int launch_prepare(Ctx& c, cudaStream_t s);          // x_rel, weights, compaction
int launch_build(Ctx& c, cudaStream_t s, int count_only);
int launch_eam_density(Ctx& c, cudaStream_t s);
int launch_eam_density_energy(Ctx& c, cudaStream_t s);  // + the compensated EAM energies (no virial)
int launch_eam_force(Ctx& c, cudaStream_t s);
int launch_ace_basis(Ctx& c, cudaStream_t s);        // A_nlm of the compacted atoms
int launch_ace(Ctx& c, cudaStream_t s);              // products, densities, dE/dA
int launch_ace_force(Ctx& c, cudaStream_t s);        // pair forces and scatter
// kick_dt > 0: fused second half kick; in_step: the evaluation of an MD step (adds its load to
// the load history when one is recorded)
int launch_blend(Ctx& c, cudaStream_t s, float* out_aos, double kick_dt = 0.0, bool in_step = false);
int launch_energy(Ctx& c, cudaStream_t s, bool virial = true);   // compensated EAM energies + energy blend (+ virial)
int launch_eam_energy(Ctx& c, cudaStream_t s, bool virial);       // the compensated EAM energies alone
int launch_energy_blend(Ctx& c, cudaStream_t s, bool virial);     // the energy blend alone (after the two above)
int launch_reduce(Ctx& c, cudaStream_t s, int with_kinetic);
int launch_kick_drift(Ctx& c, cudaStream_t s, double dt, int first_half);
int launch_kick(Ctx& c, cudaStream_t s, double dt);
int launch_nh_half(Ctx& c, cudaStream_t s, double dt);
int launch_langevin(Ctx& c, cudaStream_t s, double dt);
int launch_zero_momentum(Ctx& c, cudaStream_t s);
int launch_pos_in(Ctx& c, cudaStream_t s, const double* pos_aos);
int launch_csp(Ctx& c, cudaStream_t s, const ap_csp_params& P, float* d_csp);
int launch_csp_weights(Ctx& c, cudaStream_t s, const ap_csp_params& P, int nacc, const int S[3]);
int launch_check(Ctx& c, cudaStream_t s);

// ---------------------------------------------------------------------------------
// Batched launches (serving): one launch per stage runs the stage for several contexts.
// The contexts' device pointers and parameters travel as an array of descriptors; a
// per-atom stage gives context k the blocks start[k] .. start[k + 1] - 1 of its grid (block
// b acts as block b - start[k] of that context), and the ACE stages share a persistent grid
// over chunks of compacted atoms of all contexts (prefix sums of the device atom counts).
// ---------------------------------------------------------------------------------
struct CtxDev {
    int n, ncode, cap, load_cap;
    double mass;                      // amu (the half kick is 0.5 dt kFtm / mass, as on the host)
    double lim2;                      // (skin / 2)^2: the list displacement bound
    double ace_c1_0;
    GridDev grid;
    DynDev dyn;
    double *x, *v, *xb;
    float* f;
    float4* pos4;
    float *uxi, *w, *e_ace, *ace_A, *ace_dA, *vir_ace;
    double *e_emb, *e_eam, *w_fixed, *d_time;
    unsigned long long* acc;
    unsigned char* fixed;
    int *cell, *cell_count, *cell_start, *cell_atoms, *nbr, *nbr_row, *nnbr, *ace_list, *flags;
    long long* d_step;
    long long* load_ring;
    double* load_ring_t;
    const EamDev* eam;
    const AceTc* ace;
    const float4* D;
};

// The batch travels as a kernel parameter (about 5 KB): each context's resident descriptor and
// the block prefixes of the per-atom stages.
constexpr int kMaxBatchCtx = 256;
struct BatchTable {
    int nctx;
    int atoms;                        // sum of the contexts' atom counts
    const CtxDev* d[kMaxBatchCtx];
    int b256[kMaxBatchCtx + 1];       // blocks of 256 threads per context (atoms)
    int b128[kMaxBatchCtx + 1];       // blocks of 128 threads per context (atoms)
    int bcell[kMaxBatchCtx + 1];      // blocks of 256 threads per context (cells, a warp per cell)
};

static_assert(sizeof(CtxDev) <= sizeof(Ctx::desc_h), "descriptor copy fits its host record");

void fill_ctx_dev(const Ctx& c, CtxDev& d);
int launch_batch_step_pre(const BatchTable& t, double dt, cudaStream_t s);
int launch_batch_check(const BatchTable& t, cudaStream_t s);
int launch_batch_rebuild(const BatchTable& t, cudaStream_t s);
int launch_batch_prepare(const BatchTable& t, cudaStream_t s);
int launch_batch_eam(const BatchTable& t, cudaStream_t s);
int launch_batch_ace(const BatchTable& t, int dev, cudaStream_t s);
int launch_batch_blend(const BatchTable& t, double kick_dt, int record, cudaStream_t s);

// ACE device tables shared by every context of the same potential on a device (built once,
// kept until the process exits): a batched contraction stages them once per block
const AceTc* shared_ace_tables(const AceTc& host, int dev, std::string& err);

__host__ __device__ __forceinline__ int batch_find(const int* start, int nctx, int b) {
    int lo = 0, hi = nctx - 1;                    // the k with start[k] <= b < start[k + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// host-side tables (tables.cpp)
int build_eam_tables(const ap_potential& p, EamDev& out, std::string& err);
int build_ace_tables(const ap_potential& p, AceDev& out, std::string& err);
void build_ace_tc(const AceDev& in, AceTc& out);     // split, symmetrised, swizzled copy of in
double gaunt_real_racah(int l1, int m1, int l2, int m2, int l3, int m3);
int gaunt_values(float* out, std::string& err);      // kNG entries in pattern order
// which = 0: Phi, 1: zeta from the FP64 segments; 2: Phi, 3: zeta from the FP32 device
// table through the kernels' own segment lookup (eam_table.h)
int eam_table_eval(const ap_potential& p, int which, double r, double* f, double* df);
void upload_gaunt(const float* g);                   // kernels_ace.cu
void set_global_error(const std::string& m);         // capi.cu: the text of ap_last_error(NULL)

}  // namespace ap
