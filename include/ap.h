/*
 * ap.h -- C ABI of the GB300 (sm_103a) adaptive-precision EAM+ACE force library.
 *
 * The library evaluates, on one GPU, the adaptive-precision (AP) energy of arXiv
 * 2505.12958 (Sec. 2.2.3, Eq. energy_hyb)
 *     E = sum_i [ w_i E_i^ACE + (1 - w_i) E_i^EAM ] + sum_i V_ind(r_i)
 * and its exact negative gradient, and integrates Newton's equations with velocity
 * Verlet.  w_i is the ACE weight; the paper's switching parameter is lambda_i = 1 - w_i
 * (lambda = 1 is the fast EAM description).  One MD step is: cell binning and
 * neighbour list (rebuilt when an atom has moved more than skin/2), ACE weights and
 * stream compaction of the atoms with w_i > 0, the EAM density / embedding / pair pass
 * (Sec. 2.2.1, Eq. energy_eam; Appendix B forms), the ACE pass on the compacted atoms
 * (Sec. 2.2.2, Eq. energy_ace), the blend with the spherical indenter (Sec. 2.1,
 * Eq. V_indenter) and the indentation load (Sec. 3.1, Eq. P_ind), and the FP64
 * velocity-Verlet update.
 *
 * Conventions.  Units eV, Angstrom, fs, amu.  Positions and velocities are FP64,
 * forces FP32, energies, virial and load FP64.  Arrays of vectors are row-major n x 3
 * (AoS), like numpy / torch (n, 3) tensors.  "device" pointers are CUDA device memory
 * on the current device, "host" pointers are host memory (pinned memory makes the
 * copies asynchronous).  A cuda stream argument of NULL means the stream given to
 * ap_init.  Every call returns an ap_status; nothing aborts, prints, or traps on the
 * device.  Device-side errors (domain, capacity) are sticky and reported by the next
 * synchronising call (ap_energy, ap_check).  Only ap_init (with counted list sizing),
 * ap_energy, ap_check, ap_get_state, ap_get_forces, ap_compute_forces_host and ap_destroy
 * synchronise.  A context is not thread-safe; distinct contexts share no device state.
 * The library is exercised from one host thread: calls on distinct contexts from several
 * threads at once are not supported.
 */
#ifndef AP_H
#define AP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AP_API_VERSION 1

typedef struct ap_ctx ap_ctx;

typedef enum {
    AP_OK = 0,
    AP_ERR_ARG = -1,       /* invalid argument or unsupported parameter              */
    AP_ERR_OOM = -2,       /* device or host allocation failed                       */
    AP_ERR_CUDA = -3,      /* a CUDA runtime call failed (text in ap_last_error)     */
    AP_ERR_DOMAIN = -4,    /* phi2 <= 1e-3, rho < 0 or a non-finite value; atom index in ap_last_error */
    AP_ERR_CAPACITY = -5,  /* neighbour-list capacity exceeded: the call that reports it grows the
                              list (AP_ERR_OOM instead when that allocation fails) and the next
                              evaluation rebuilds it; the evaluation that overflowed is discarded */
    AP_ERR_TIMEOUT = -6,   /* reserved for bounded waits                             */
    AP_ERR_STATE = -7,     /* call not valid in the current state                   */
    AP_ERR_LIMIT = -8      /* a fixed limit of this build was exceeded: more than 128 neighbours
                              within the ACE cutoff of one atom (index in ap_last_error).  Sticky
                              and not retried: the structure is outside what the build evaluates */
} ap_status;

/* Precision of the atomic-base contraction A_nlm = sum_j g_n(r_ij) Y_lm(rhat_ij). */
enum {
    AP_ACE_FP32 = 0,       /* FP32 FMA (default)                                     */
    AP_ACE_TC_TF32X3 = 1,  /* tensor cores, mma.sync TF32 with hi/lo split, 3 products */
    AP_ACE_TC_BF16 = 2,    /* tensor cores, BF16 inputs, FP32 accumulate             */
    AP_ACE_TC_FP16 = 3,    /* tensor cores, FP16 inputs, FP32 accumulate             */
    AP_ACE_FP64 = 4        /* FP64 FMA                                               */
};

/* Potential parameters (copied by ap_init).
 * EAM, Appendix B: xi(x) = a1 sqrt(x) + a2 x^2 + Delta xi (Eqs. eam_F_Marinica,
 * tungsten_F_up); Phi(r) = sum_i a_i (d_i - r)^3 Theta(d_i - r) (Eq. eam_Phi_Marinica),
 * replaced by the ZBL form below r_lo and by sum_m b_m r^m on [r_lo, r_hi] when
 * eam_zbl = 1 (Eq. tungsten_Phi_up); zeta_0(r) = same cubic-knot form (Eq.
 * eam_rho_Marinica), held at zeta_0(r_clamp) for r <= r_clamp when r_clamp > 0
 * (Eq. tungsten_rho_up).
 * ACE, Sec. 2.2.2: E_i = phi1 + sqrt(phi2), phi_p = c_p0 + sum_v c_p[v] B_v (Eq.
 * energy_ace), B_v products of A_nlm = (1/nref) sum_j g_n(r_ij) Y_lm(rhat_ij) with
 * g_n = T_n(2r/rc - 1) (1 + cos(pi r/rc))/2 and real orthonormal Y_lm.  The basis is a
 * host table ace_idx (ace_nfunc x 7 ints): (nu, n1, l1, n2, l2, n3, l3), unused -1;
 * nu = 1: A_n00; nu = 2: sum_m A_n1lm A_n2lm; nu = 3: sum_m1m2m3 G A A A with the real
 * Gaunt coefficients G.  Supported: ace_nmax = 8, ace_lmax = 4, nu <= 3. */
typedef struct {
    int eam_n_phi;
    double eam_phi_a[32], eam_phi_d[32];
    int eam_n_rho;
    double eam_rho_a[16], eam_rho_d[16];
    double eam_rho_rclamp;
    double eam_F_a1, eam_F_a2, eam_F_dxi;
    int eam_zbl;
    double eam_zbl_Z, eam_zbl_eps0, eam_zbl_a, eam_r_lo, eam_r_hi, eam_b[6];

    double ace_rc, ace_nref;
    int ace_nmax, ace_lmax, ace_nfunc;
    const int* ace_idx;          /* host, ace_nfunc x 7, copied                     */
    const double* ace_c1;        /* host, ace_nfunc, copied                         */
    const double* ace_c2;        /* host, ace_nfunc, copied                         */
    double ace_c1_0, ace_c2_0;
    int ace_precision;           /* AP_ACE_*                                        */

    double mass_amu;             /* one species per context                         */
    double skin;                 /* neighbour-list skin (Angstrom), e.g. 1.0         */
    int list_sizing;             /* neighbour slots per atom: AP_LIST_COUNTED (0) from a
                                    counting pass over the first binning, which makes
                                    ap_init synchronise once; AP_LIST_BOUND (1) from the
                                    bound 0.1 atoms / A^3 inside the list sphere (no
                                    synchronisation; a denser structure reports
                                    AP_ERR_CAPACITY at its first check, which grows the
                                    list, and the next evaluation is complete)      */
} ap_potential;

enum { AP_LIST_COUNTED = 0, AP_LIST_BOUND = 1 };

/* Box: edge vectors as rows of h (triclinic allowed), lower corner at origin.  In a
 * non-periodic direction the box only sizes the cell grid; atoms may leave it. */
typedef struct {
    double h[9];
    double origin[3];
    int periodic[3];
} ap_box;

/* ACE weight w_i.  AP_REGION_NONE: w = 0 (pure EAM).  AP_REGION_CONST: w = w_const.
 * AP_REGION_EXPLICIT: w from a host array (frozen between ap_set_weights calls).
 * AP_REGION_SPHERE: w = S(d), d = |r_i - c| (minimum image in periodic directions),
 * S = 1 for d < r_in, (1 + cos(pi (d - r_in)/r_switch))/2 up to r_in + r_switch, 0
 * beyond; the force then carries -grad w_i (E_i^ACE - E_i^EAM).  A sphere centred on
 * the surface point under the tip is the hemisphere of the paper's fixed zones
 * (Sec. 2.2.3).  follow_indenter moves c with the indenter.  ACE runs on w_i > 0. */
enum { AP_REGION_NONE = 0, AP_REGION_SPHERE = 1, AP_REGION_EXPLICIT = 2, AP_REGION_CONST = 3 };
typedef struct {
    int kind;
    double center[3];
    double r_in, r_switch;
    int follow_indenter;
    const double* w_explicit;    /* host, n, for AP_REGION_EXPLICIT, copied          */
    double w_const;
} ap_region;

/* Spherical indenter, Eq. V_indenter: V = (K/3) Theta(R - d) (R - d)^3, d = |r - c(t)|,
 * c(t) = center0 - vel t.  load = sum_i F_ind,i . dir (Eq. P_ind; dir is the unit
 * indentation direction, e.g. (0,0,-1)). */
typedef struct {
    int enabled;
    double center0[3];
    double vel[3];               /* Angstrom/fs */
    double R, K;
    double dir[3];
} ap_indenter;

/* Results of the last force evaluation (ap_energy). */
typedef struct {
    double e_total;              /* e_pot + e_ind                                    */
    double e_pot;                /* sum_i w_i E_i^ACE + (1 - w_i) E_i^EAM             */
    double e_ind;                /* sum_i V_ind(r_i)                                 */
    double e_kin;                /* sum_i m v_i^2 / 2 of the current velocities       */
    double virial[6];            /* xx yy zz xy xz yz of -sum_i sum_j r_ij (x) dE_i/dr_ij */
    double load;                 /* Eq. P_ind                                        */
    double time_fs;
    long long step;
    int n_ace;                   /* atoms with w > 0                                 */
    int n_atoms;
    double e_thermostat;         /* Q xi^2 / 2 + N_f k_B T eta of the Nose-Hoover thermostat:
                                    e_total + e_kin + e_thermostat is conserved (0 without) */
} ap_report;

/* Create a context on the current CUDA device: copies parameters and the host arrays
 * pos (n x 3), vel (n x 3 or NULL = 0) and fixed (n bytes, nonzero = frozen, or NULL),
 * builds the tables, allocates device memory, and evaluates nothing yet.  n >= 1.
 * Errors: AP_ERR_ARG (bad parameter, box thinner than half the list cutoff),
 * AP_ERR_OOM, AP_ERR_CUDA.  Synchronises once with pot->list_sizing = AP_LIST_COUNTED;
 * with AP_LIST_BOUND it issues its uploads on `stream` and returns without waiting. */
ap_status ap_init(const ap_potential* pot, const ap_box* box, const ap_region* region,
                  const ap_indenter* indenter, int n_atoms, const double* pos,
                  const double* vel, const unsigned char* fixed, void* stream, ap_ctx** out);

/* One AP force evaluation of the internal positions, or of d_pos (device, n x 3 FP64;
 * copied into the context state first) when not NULL.  Forces (n x 3 FP32) go to
 * d_force (device) when not NULL and to the context.  Asynchronous. */
ap_status ap_compute_forces(ap_ctx* ctx, const double* d_pos, float* d_force, void* stream);

/* The same with host buffers: h_pos (n x 3 FP64) is copied in, h_force (n x 3 FP32)
 * and *h_energy (total energy) are copied out.  *h_energy is the e_pot + e_ind that a
 * following ap_energy reports, bit for bit: the EAM density pass of this evaluation forms
 * the same compensated per-atom energies as ap_energy's own pass (without the per-atom
 * virial, which ap_energy then computes).  On a stream other than the legacy default
 * stream (profiling off) the kernels between the copies replay as one CUDA graph, captured
 * once per stream, buffer layout and choice of h_pos / h_energy.  Synchronises. */
ap_status ap_compute_forces_host(ap_ctx* ctx, const double* h_pos, float* h_force,
                                 double* h_energy, void* stream);

/* n_steps velocity-Verlet steps of dt_fs on the library-owned positions and velocities.
 * Fixed atoms keep x and v.  The indenter (and a following region) advance with time.
 * On a stream other than the legacy default stream one step (and a block of 8 steps) is
 * captured as a CUDA graph on first need and replayed.  With only the ACE contraction profiled
 * (ap_profile 2 or 3) one step at a time is replayed, the timed steps from a graph whose
 * event-record nodes around the contraction are set to a fresh event pair each time; with every stage profiled (ap_profile 1),
 * or on the legacy stream, steps are plain launches.  The results are the same bits on
 * every path.  Asynchronous. */
ap_status ap_step(ap_ctx* ctx, int n_steps, double dt_fs, void* stream);

/* Serving form: n_steps[k] velocity-Verlet steps (dt_fs) for each of n_ctx independent
 * contexts, batched: every stage of a step (kick-drift, neighbour rebuild, weights and
 * compaction, list build, EAM density and forces, ACE basis, contraction and pair forces,
 * blend with the second half kick) is ONE kernel launch on `stream` for all contexts that
 * still have steps to go.  The per-atom stages give each context its own blocks of the
 * launch; the ACE stages share one persistent grid over the compacted atoms of all contexts,
 * and contexts with the same potential share one coefficient table, staged once per block.
 * The batch waits for each context's earlier work on its own stream, and each context's
 * stream waits for the batch, so calls on the contexts before and after stay ordered.  A
 * context with a thermostat, stage timing or a precision mode other than AP_ACE_FP32 (and
 * any beyond the first 256) is stepped on its own stream instead.  Every context's results
 * are the same bits as when it is stepped alone (the same per-atom arithmetic, and the
 * integer force sums do not depend on order).  Asynchronous; returns the first error. */
ap_status ap_step_batch(ap_ctx* const* ctxs, const int* n_steps, int n_ctx, double dt_fs, void* stream);

/* Serving form of ap_compute_forces: one AP force evaluation of the library-owned positions
 * of each of n_ctx contexts, batched as ap_step_batch (one launch per stage on `stream`).
 * Arguments are checked before anything is launched (AP_ERR_ARG for a NULL entry).
 * Asynchronous; returns the first error. */
ap_status ap_compute_forces_batch(ap_ctx* const* ctxs, int n_ctx, void* stream);

/* Thermostat of a group of atoms (Appendix A: during the indentation the central part of
 * the slab is an NVT ensemble, Nose-Hoover with damping time gamma_T^NH = 0.1 ps at 300 K
 * for W, 292 K for Cu).  One thermostat variable xi (chain length 1); before and after each
 * velocity-Verlet step of ap_step a half step
 *   xi += dt/4 G;  v_G *= exp(-xi dt/2);  eta += xi dt/2;  xi += dt/4 G,
 *   G = (2 KE_G - N_f k_B T) / Q,  N_f = 3 |G|,  Q = N_f k_B T tau^2,
 * all on the device (the step graph includes it).
 * AP_THERMO_LANGEVIN (equilibration, Appendix A): after each force evaluation the group's
 * forces get a drag -(m/tau) v (v of the half step) and a random force sqrt(2 m k_B T /
 * (tau dt)) g per component; g is standard normal, by Box-Muller from Philox4x32-10 at
 * counter (atom index, step since ap_set_thermostat, 0, 0) and key (seed low, seed high):
 * u1 = (w0 + 1)/2^32, u2 = (w1 + 0.5)/2^32, g_x, g_y = sqrt(-2 ln u1) (cos, sin)(2 pi u2),
 * g_z the cosine branch of (w2, w3).  With zero_every > 0 the centre-of-mass velocity of the
 * free atoms is removed every zero_every steps after the final kick.
 * group: host mask of n bytes (nonzero = thermostatted; fixed atoms are excluded), NULL =
 * every free atom.  kind AP_THERMO_NONE removes the thermostat.  Resets the thermostat
 * state.  AP_ERR_ARG for t_target <= 0 or tau_fs <= 0.  Synchronises. */
enum { AP_THERMO_NONE = 0, AP_THERMO_NOSE_HOOVER = 1, AP_THERMO_LANGEVIN = 2 };
typedef struct {
    int kind;
    double t_target;           /* K */
    double tau_fs;             /* damping time, fs (the paper: 100 for Nose-Hoover; Langevin 100 - 10000) */
    unsigned long long seed;   /* Langevin: key of the random numbers */
    int zero_every;            /* Langevin: zero the centre-of-mass velocity of the free atoms
                                  every zero_every steps (0: never; the paper: every 1 ps) */
} ap_thermostat;
ap_status ap_set_thermostat(ap_ctx* ctx, const ap_thermostat* t, const unsigned char* group);

/* CSP-driven switching weights (Sec. 2.2.3, the switching function of Appendix B with
 * the parameters of Tab. model_parameters_tungsten).  The centro-symmetry parameter of atom
 * i is the sum of the n_nb/2 smallest |R_j + R_k|^2 over pairs of its n_nb nearest
 * neighbours within rc (fewer than n_nb there: a surface atom).  ap_csp_accumulate adds the
 * CSP of the current positions to per-atom block sums (d_csp: optional device copy, n FP32,
 * -1 for surface atoms); ap_csp_update_weights turns the block averages into weights and
 * starts a new block (the paper averages over 110 steps):
 *   w0 = clamp((CSP - csp_lo) / (csp_hi - csp_lo), 0, 1);  w0 = 1 inside the precise zone
 *   (|r - zone_center| < zone_r, nearest image); w0 = 0 for surface atoms outside it;
 *   w_i = max_j w0_j T(|r_ij|), T = 1 for r <= r_lo, cos^2(pi (r - r_lo) / (2 (r_hi - r_lo)))
 *   below r_hi, 0 beyond; the stored weight changes only where |w_new - w| >= dlam_min.
 * The w0 map, the spatial form and the hysteresis are this library's readings (the paper
 * names the parameters; the map is in its cited AP work).  The context must use
 * AP_REGION_EXPLICIT; the weights act from the next force evaluation.  rc must not exceed
 * the neighbour-list cutoff.  *n_seeds (nullable) receives the number of atoms with w0 > 0.
 * AP_ERR_ARG on bad parameters, AP_ERR_STATE for a non-explicit context or an empty block.
 * ap_csp_update_weights synchronises. */
typedef struct {
    int n_nb;                  /* 12 (FCC) or 14 (BCC: the first two shells) */
    double rc;                 /* CSP neighbour cutoff, between shells n_nb and n_nb + 1 (A) */
    double csp_lo, csp_hi;     /* A^2 (the paper: 1.5, 1.6) */
    double r_lo, r_hi;         /* spatial transition (A; the paper: 4, 12) */
    double dlam_min;           /* smallest applied change of a weight (the paper: 0.01) */
    double zone_center[3];     /* precise zone, w0 = 1 inside */
    double zone_r;
} ap_csp_params;
ap_status ap_csp_accumulate(ap_ctx* ctx, const ap_csp_params* p, float* d_csp);
ap_status ap_csp_update_weights(ap_ctx* ctx, const ap_csp_params* p, int* n_seeds);

/* Indentation load history kept on the device (Sec. 3.1, Eq. P_ind).  With capacity > 0,
 * every later MD step of ap_step adds the load of its force evaluation, sum_i F_ind,i . dir,
 * to a device ring of `capacity` (time, load) entries, without any synchronisation; the
 * per-atom terms are summed as 64-bit fixed point (2^-32 eV/A), so the history is the same
 * bits in every run.  capacity = 0 stops recording and frees the ring.  Synchronises.
 * AP_ERR_STATE for a context without an indenter, AP_ERR_OOM when the ring cannot be
 * allocated. */
ap_status ap_record_load(ap_ctx* ctx, int capacity);
/* Host copy of the recorded load history: the most recent min(max, steps recorded,
 * capacity) entries, oldest first, t_fs[k] the time after the step (fs) and load[k] its
 * load (eV/A); *count receives how many were written.  Synchronises (one read-back of the
 * ring).  AP_ERR_STATE when no history is recorded. */
ap_status ap_load_history(ap_ctx* ctx, double* t_fs, double* load, int max, int* count);

/* Totals of the last force evaluation; d_e_atom (device, n FP64, nullable) receives
 * the per-atom energies E_i + V_ind(r_i).  Synchronises; returns sticky device errors. */
ap_status ap_energy(ap_ctx* ctx, ap_report* out, double* d_e_atom);

/* Synchronise and return the sticky device error status (AP_OK if none). */
ap_status ap_check(ap_ctx* ctx);

/* Host copies of positions, velocities (n x 3, either may be NULL) and time. */
ap_status ap_get_state(ap_ctx* ctx, double* x, double* v, double* t_fs);
/* Replace positions / velocities (host, n x 3, either may be NULL) and time; forces a
 * neighbour rebuild and a fresh force evaluation before the next step. */
ap_status ap_set_state(ap_ctx* ctx, const double* x, const double* v, double t_fs);
/* Replace the box (e.g. a strained cell); positions are not changed.  The cell grid and
 * the neighbour list are rebuilt by the next evaluation.  AP_ERR_ARG if the new box is
 * thinner than half the list cutoff.  Synchronises. */
ap_status ap_set_box(ap_ctx* ctx, const ap_box* box);
/* Host copy of the last forces (n x 3 FP32). */
ap_status ap_get_forces(ap_ctx* ctx, float* f);
/* Host copy of the weights w_i (n FP64) of the last force evaluation; weights set by
 * ap_set_weights or ap_csp_update_weights appear after the next evaluation. */
ap_status ap_get_weights(ap_ctx* ctx, double* w);
/* Replace explicit weights (AP_REGION_EXPLICIT contexts only; host, n). */
ap_status ap_set_weights(ap_ctx* ctx, const double* w);

/* Per-stage CUDA-event timing of later calls and its readout: enable = 1 brackets every
 * stage with a pair of events (about 2.5 us per stage on the stream), enable = 2 only the
 * ACE contraction stage (the dominant kernel, for its roofline), enable = 3 the ACE
 * contraction of one step in eight of ap_step's graph replays (the others replay the
 * untimed step graph: two event-record nodes cost about 10 us per replayed step),
 * enable = 0 stops.  Stepping with every stage profiled uses plain launches, not the
 * captured graphs.  ms[k] is the accumulated time of stage k over launches[k] launches, stages
 * AP_STAGE_*; reading drains the pending events (synchronises).  AP_ERR_ARG for other
 * values of enable. */
enum { AP_STAGE_NEIGHBOR = 0, AP_STAGE_PREPARE = 1, AP_STAGE_EAM_DENSITY = 2,
       AP_STAGE_EAM_FORCE = 3, AP_STAGE_ACE = 4, AP_STAGE_BLEND = 5, AP_STAGE_INTEGRATE = 6,
       AP_STAGE_ACE_BASIS = 7, AP_STAGE_ACE_FORCE = 8, AP_NSTAGE = 9 };
/* (AP_STAGE_ACE is the contraction kernel: products, densities and dE/dA.) */
ap_status ap_profile(ap_ctx* ctx, int enable);
ap_status ap_profile_read(ap_ctx* ctx, double* ms, long long* launches);

/* Number of kernels this context has launched since creation. */
long long ap_launch_count(const ap_ctx* ctx);
/* Neighbour-list capacity per atom and the number of list rebuilds so far. */
ap_status ap_neighbor_info(ap_ctx* ctx, int* capacity, long long* rebuilds);
/* Device bytes a context of n atoms needs: an upper estimate for structures of metallic
 * density (at most 0.1 atoms / A^3 inside the list sphere) whose binning grid has at most
 * one cell per atom.  ace_fraction is accepted for callers that know it; the ACE arrays
 * are sized for every atom because the region may move.  No device access. */
size_t ap_footprint_bytes(const ap_potential* pot, int n_atoms, double ace_fraction);
/* Device bytes ctx holds right now (its stream-ordered allocations, including any
 * capacity growth); 0 for NULL. */
size_t ap_memory_bytes(const ap_ctx* ctx);
/* Test hook for the failure paths: the next `count` device allocations of this library
 * (context arenas, capacity growth) fail as if the device were out of memory, so the calls
 * that make them return AP_ERR_OOM.  count <= 0 clears pending failures.  Host-side only: no
 * device state is touched and nothing is launched. */
void ap_inject_alloc_failures(int count);

/* Text of the last error of ctx, or with ctx NULL of the last failed ap_init or
 * ap_ace_forces_noalloc call of this thread. */
const char* ap_last_error(const ap_ctx* ctx);
void ap_destroy(ap_ctx* ctx);
int ap_version(void);

/* Measurement helper: FP32 FMA throughput of the current device (TFLOP/s), from one
 * timed launch of a kernel of independent FMA chains on 8 blocks of 256 threads per SM
 * (after a short warm-up launch).  iters in [1, 2^20] sets its length (2e5: ~25 ms).
 * The roofline denominator of the ACE contraction, which is plain FP32 arithmetic.
 * *ms_out (nullable) receives the launch time.  Synchronises the device. */
ap_status ap_probe_fp32_peak(int iters, double* tflops, double* ms_out);

/* Allocation-free ACE forces for neighbour environments the caller supplies.  The paper
 * has no counterpart: this entry point exists for callers that cannot create device
 * allocations of their own - a program or plugin whose GPU memory is owned entirely by
 * another allocator (a framework's caching pool that must account for every byte), or a
 * time-critical loop that rules out the latency and the failure modes of cudaMalloc once
 * it is running.  It evaluates E = sum_i w_i E_i^ACE (Eq. energy_ace, with the frozen
 * weights w_i) and F_k = -dE/dr_k for up to 65,536 atoms, and calls no cudaMalloc, cudaFree
 * or other allocating routine.
 *   d_nbr_idx  device, n_atoms x max_nb ints: neighbour atom index j of atom i, -1 = unused
 *   d_rvec     device, n_atoms x max_nb x 3 FP32: r_j (image) - r_i for those slots
 *   d_w        device, n_atoms FP32 weights w_i, or NULL for w = 1 (atoms with w = 0 are skipped)
 *   d_force    device, n_atoms x 3 FP32 output: the weighted forces F_k above
 *   d_energy   device, n_atoms FP64 output: the unweighted E_i^ACE (0 where w = 0, NaN
 *              where phi2 <= 1e-3)
 * Limits: n_atoms <= 65536, max_nb <= 128, ace_precision AP_ACE_FP32, else AP_ERR_ARG; the
 * reason is in ap_last_error(NULL).  Scratch (the coefficient tables and 64-bit force
 * accumulators, ~1.6 MB) is one file-scope device array that every GPU loading the library
 * holds until the process exits.  The first call on a device looks up its address and
 * uploads constant tables, and a call whose potential differs from the previous call's on
 * that device uploads its coefficient tables; make those calls before any stream capture
 * (while `stream` is capturing they return AP_ERR_STATE and issue nothing).
 * Every call shares the array and clears the accumulators it uses before its kernels run;
 * calls that overlap on the GPU (other streams, other threads) race on it.  Asynchronous on
 * `stream`; errors of the launch are returned, a domain error shows as a NaN energy. */
ap_status ap_ace_forces_noalloc(const ap_potential* pot, int n_atoms, int max_nb, const int* d_nbr_idx,
                                const float* d_rvec, const float* d_w, float* d_force, double* d_energy,
                                void* stream);

/* Host-side table generators, exposed so that they can be checked without a GPU.
 * ap_gaunt_real: real Gaunt coefficient integral(Y_l1m1 Y_l2m2 Y_l3m3) from the Racah
 * formula for Wigner 3j symbols and the complex-to-real transform (l <= 4).
 * ap_eam_table_eval: the pair functions of Appendix B as the kernels hold them: the merged
 * piecewise-polynomial partition re-expanded in FP64 about each segment midpoint and
 * evaluated in FP64 (which = 0: Phi, 1: zeta), or the FP32 device table read through the
 * kernels' own segment lookup and evaluated in FP32 on the host (which = 2: Phi, 3: zeta).
 * Zero at and beyond each function's cutoff. */
ap_status ap_gaunt_real(int l1, int m1, int l2, int m2, int l3, int m3, double* out);
ap_status ap_eam_table_eval(const ap_potential* pot, int which, double r, double* f, double* df);

#ifdef __cplusplus
}
#endif
#endif
