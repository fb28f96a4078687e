/*
 * oracle.h -- plain FP64 CPU oracle for the adaptive-precision (AP) EAM+ACE force
 * evaluation of arXiv 2505.12958 ("Nanoindentation simulations for copper and tungsten
 * with adaptive-precision potentials").
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path.  Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may load it.
 * It shares no code, header, table or constant generator with the CUDA library.
 *
 * Units: eV, Angstrom, fs, amu.  All arithmetic is IEEE double precision.
 *
 * Weight convention: w_i is the ACE weight.  The paper (Sec. 2.2.3, Eq. energy_hyb)
 * writes E_i = lambda_i E_i^EAM + (1 - lambda_i) E_i^ACE, so w_i = 1 - lambda_i.
 */
#ifndef AP_ORACLE_H
#define AP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* EAM in the form of Sec. 2.2.1 (Eq. energy_eam) with the tungsten forms of Appendix B
 * (Eqs. eam_F_Marinica, eam_Phi_Marinica, eam_rho_Marinica, tungsten_rho_up,
 * tungsten_F_up, tungsten_Phi_up).  A potential without ZBL sets zbl = 0. */
typedef struct {
    int n_phi;            /* number of cubic knots of the pair potential Phi   */
    double phi_a[32];     /* a_i^Phi                                            */
    double phi_d[32];     /* delta_i^Phi                                        */
    int n_rho;            /* number of cubic knots of the density zeta_0        */
    double rho_a[16];     /* a_i^rho                                            */
    double rho_d[16];     /* delta_i^rho                                        */
    double rho_rclamp;    /* r_cut^rho: zeta(r) = zeta_0(r_cut^rho) below it; <=0 off */
    double F_a1, F_a2;    /* xi(x) = a1 sqrt(x) + a2 x^2                        */
    double F_dxi;         /* Delta xi, added to every atom's embedding energy   */
    int zbl;              /* 1: ZBL below r_lo and quintic bridge on [r_lo, r_hi] */
    double zbl_Z, zbl_eps0, zbl_a, r_lo, r_hi;
    double b[6];          /* Phi^int(r) = sum_m b_m r^m                          */
} or_eam;

/* Synthetic ACE (Sec. 2.2.2, Eq. energy_ace): E_i = phi1 + sqrt(phi2),
 * phi_p = c_p0 + sum_v c_p[v] B_v.  Basis functions are listed explicitly:
 * idx[7*v .. 7*v+6] = (nu, n1, l1, n2, l2, n3, l3), unused slots -1. */
typedef struct {
    double rc;            /* cutoff of the radial basis                         */
    double nref;          /* A_nlm = (1/nref) sum_j g_n(r_ij) Y_lm(rhat_ij)     */
    int nmax, lmax;       /* n = 0..nmax-1, l = 0..lmax                        */
    int nfunc;
    const int* idx;
    const double* c1;
    const double* c2;
    double c1_0, c2_0;    /* coefficients of the constant basis function B_0=1  */
} or_ace;

/* Box: edge vectors as rows of h, lower corner at origin. */
typedef struct {
    int n;
    const double* x;      /* n x 3 row-major positions                          */
    double h[9];
    double origin[3];
    int periodic[3];
} or_system;

/* ACE weight.  kind 0: w from w_explicit (constant per atom, no gradient term).
 * kind 1: sphere, w = S(|r - c|) with the cosine switch, and the gradient term
 * -grad w_i (E_i^ACE - E_i^EAM) in the force.  kind 2: constant w_const. */
typedef struct {
    int kind;
    double center[3];
    double r_in, r_sw;
    const double* w_explicit;
    double w_const;
} or_region;

/* Spherical indenter, Eq. V_indenter: V = (K/3) Theta(R-d) (R-d)^3, d = |r - c|.
 * The load (Eq. P_ind) is the sum of indenter forces projected on dir (unit). */
typedef struct {
    int enabled;
    double center[3];
    double R, K;
    double dir[3];
} or_indenter;

typedef struct {
    double e_total;       /* sum over evaluated atoms of E_i + V_ind(r_i)       */
    double virial[6];     /* xx yy zz xy xz yz of -sum r_ij (x) dE_i/dr_ij      */
    double load;
    double e_indenter;
    int n_ace;            /* atoms with w > 0 among the evaluated ones          */
    int status;           /* 0 ok; -4 domain error (phi2 <= 1e-3 or rho < 0)    */
    int bad_atom;
} or_result;

/* Full evaluation.  centers: NULL = all atoms; else a 0/1 mask of atoms whose energy
 * terms are evaluated.  forces (n x 3) receive every contribution of the evaluated
 * centers, so F_k is complete when k and all its neighbours are centers.
 * e_atom, e_eam, e_ace, w_out may be NULL.  nthreads <= 0: all available. */
int or_evaluate(const or_system* sys, const or_eam* eam, const or_ace* ace,
                const or_region* reg, const or_indenter* ind,
                const unsigned char* centers, int nthreads,
                double* forces, double* e_atom, double* e_eam, double* e_ace,
                double* w_out, or_result* res);

/* Neighbour search within rc (all periodic images).  mode 0: cell list, mode 1:
 * brute force over all pairs and images.  Returns the pair count, or -1 if
 * cap is too small.  Pairs are (i, j, rx, ry, rz) with r = r_j(image) - r_i. */
long or_neighbors(const or_system* sys, double rc, int mode, long cap,
                  int* pi, int* pj, double* rvec);

/* Elementary functions, exposed for the pins. */
void or_eam_phi(const or_eam* p, double r, double* f, double* df);
void or_eam_rho(const or_eam* p, double r, double* f, double* df);
void or_eam_embed(const or_eam* p, double rho, double* f, double* df);
double or_eam_cutoff(const or_eam* p);

/* Real orthonormal Y_lm(r/|r|) for l <= 4 at index l*l + l + m, and the gradient
 * with respect to the vector r (3 entries per function). grad may be NULL. */
void or_ylm(double x, double y, double z, double* Y, double* grad);
/* Radial basis g_n(r) = T_n(2r/rc - 1) fc(r), n < nmax, and dg/dr. */
void or_radial(double r, double rc, int nmax, double* g, double* dg);
/* Real Gaunt coefficient integral(Y_l1m1 Y_l2m2 Y_l3m3) by exact quadrature. */
double or_gaunt(int l1, int m1, int l2, int m2, int l3, int m3);

/* One ACE atom from its neighbour vectors (r_j - r_i, nn x 3).  Writes E_i,
 * phi1, phi2, the basis values B (nfunc) if B != NULL, and f (nn x 3) with
 * f_j = dE_i / d r_ij if f != NULL.  Returns 0 or -4 (phi2 <= 1e-3). */
int or_ace_atom(const or_ace* ace, int nn, const double* rvec,
                double* E, double* phi1, double* phi2, double* B, double* f);

/* Velocity Verlet (masses in amu, dt in fs).  fixed atoms keep x and v.  The
 * indenter centre moves by -ind_vel * dt per step and, if region_follows, the
 * region centre moves with it.  Per step k (0..nsteps) writes epot[k], ekin[k]
 * (k = 0 is the initial state).  x and v (n x 3) are updated in place. */
int or_md(const or_system* sys, const or_eam* eam, const or_ace* ace,
          const or_region* reg, const or_indenter* ind, const double* ind_vel,
          int region_follows, const unsigned char* fixed, double mass, double dt,
          int nsteps, int nthreads, double* x, double* v, double* epot, double* ekin);

/* Centro-symmetry parameter, as the switching function of Appendix B uses it (Sec. 2.2.3):
 * for atom i the n_nb nearest neighbours within rc (n_nb = 12 for FCC, 14 for BCC: the
 * first two BCC shells), every pair (j, k) of them gives |R_j + R_k|^2, and the CSP is
 * the sum of the n_nb/2 smallest.  An atom with fewer than n_nb neighbours within rc
 * (a surface atom) gets -1.  coord (nullable) receives the neighbour count within rc.
 * n_nb even, 2 <= n_nb <= 16.  Returns 0, or -1 on bad arguments. */
int or_csp(const or_system* sys, int n_nb, double rc, double* csp, int* coord);

/* Velocity Verlet with a Nose-Hoover thermostat on a group of atoms (Appendix A: the
 * central part of the slab is simulated as NVT during the indentation, Nose-Hoover with
 * damping time tau = gamma_T^NH).  One thermostat variable xi (chain length 1), integrated
 * by the time-reversible split: before and after each velocity-Verlet step a half step
 *   xi += dt/4 G;  v_G *= exp(-xi dt/2);  eta += xi dt/2;  xi += dt/4 G,
 * G = (2 KE_G - N_f k_B T) / Q,  N_f = 3 |G|,  Q = N_f k_B T tau^2  (tau in fs).
 * group: 0/1 mask (fixed atoms are never in it).  Writes per step k (0..nsteps) epot,
 * ekin (all atoms) and ethermo = Q xi^2 / 2 + N_f k_B T eta, so that epot + ekin +
 * ethermo is conserved.  Other arguments as or_md. */
int or_md_nh(const or_system* sys, const or_eam* eam, const or_ace* ace,
             const or_region* reg, const or_indenter* ind, const double* ind_vel,
             int region_follows, const unsigned char* fixed, const unsigned char* group,
             double t_target, double tau, double mass, double dt, int nsteps, int nthreads,
             double* x, double* v, double* epot, double* ekin, double* ethermo);

/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
 * the 4-word multiply-xor round with the published multipliers and Weyl key increments.
 * out[4] = philox4x32_10(ctr[4], key[2]). */
void or_philox4x32_10(const unsigned int* ctr, const unsigned int* key, unsigned int* out);

/* Velocity Verlet with a Langevin thermostat on a group (Appendix A: equilibration steps 1
 * and 3, damping time gamma^L): after each force evaluation the group's forces get a drag
 * -(m / tau) v (v of the half step) and a random force sqrt(2 m k_B T / (tau dt)) g per
 * component, g a standard normal number.  The normal numbers of atom i at step s (1-based)
 * come from philox4x32_10(ctr = (i, s, 0, 0), key = (seed_lo, seed_hi)) by Box-Muller:
 * u1 = (w0 + 1) / 2^32, u2 = (w1 + 0.5) / 2^32, g_x = sqrt(-2 ln u1) cos(2 pi u2),
 * g_y = sqrt(-2 ln u1) sin(2 pi u2); g_z from (w2, w3) the same way (its cosine branch).
 * zero_every > 0: every zero_every steps the centre-of-mass velocity of the free atoms is
 * subtracted from them (the momentum zeroing of Appendix A).  Other arguments as or_md. */
int or_md_langevin(const or_system* sys, const or_eam* eam, const or_ace* ace,
                   const or_region* reg, const or_indenter* ind, const double* ind_vel,
                   int region_follows, const unsigned char* fixed, const unsigned char* group,
                   double t_target, double tau, unsigned long long seed, int zero_every,
                   double mass, double dt, int nsteps, int nthreads,
                   double* x, double* v, double* epot, double* ekin);

int or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
