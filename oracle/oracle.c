/*
 * oracle.c -- plain FP64 CPU oracle for the adaptive-precision (AP) EAM+ACE force
 * evaluation of arXiv 2505.12958.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Everything here is the definition written out:
 *   - energy blend, Sec. 2.2.3 Eq. energy_hyb (with w = 1 - lambda, see oracle.h);
 *   - EAM, Sec. 2.2.1 Eq. energy_eam, forms of Appendix B (Eqs. eam_F_Marinica,
 *     eam_Phi_Marinica, eam_rho_Marinica, tungsten_rho_up, tungsten_F_up,
 *     tungsten_Phi_up, the ZBL screening function and a_ZBL);
 *   - ACE, Sec. 2.2.2 Eq. energy_ace, E = phi1 + sqrt(phi2), phi_p = sum_v c_v B_v,
 *     with the synthetic basis stated in oracle.h;
 *   - the spherical indenter, Eq. V_indenter, and the load, Eq. P_ind.
 * Forces are the exact negative gradient: every per-atom energy E_i is a function
 * of its neighbour vectors r_ij = r_j - r_i, and dE_i/dr_ij is pushed to atoms j
 * (-) and i (+).  Gradients of the angular functions use forward-mode dual numbers.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define LMAXO 4
#define NLMO ((LMAXO + 1) * (LMAXO + 1))

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* dual numbers: a value and its gradient with respect to a 3-vector           */
/* ------------------------------------------------------------------------- */
typedef struct { double v, g[3]; } dual;

static dual d_const(double c) { dual r; r.v = c; r.g[0] = r.g[1] = r.g[2] = 0.0; return r; }
static dual d_var(double x, int k) { dual r = d_const(x); r.g[k] = 1.0; return r; }
static dual d_add(dual a, dual b) { dual r; r.v = a.v + b.v; for (int k = 0; k < 3; ++k) r.g[k] = a.g[k] + b.g[k]; return r; }
static dual d_sub(dual a, dual b) { dual r; r.v = a.v - b.v; for (int k = 0; k < 3; ++k) r.g[k] = a.g[k] - b.g[k]; return r; }
static dual d_mul(dual a, dual b) { dual r; r.v = a.v * b.v; for (int k = 0; k < 3; ++k) r.g[k] = a.g[k] * b.v + a.v * b.g[k]; return r; }
static dual d_scale(dual a, double s) { dual r; r.v = a.v * s; for (int k = 0; k < 3; ++k) r.g[k] = a.g[k] * s; return r; }
static dual d_div(dual a, dual b) {
    dual r; r.v = a.v / b.v;
    for (int k = 0; k < 3; ++k) r.g[k] = (a.g[k] * b.v - a.v * b.g[k]) / (b.v * b.v);
    return r;
}
static dual d_sqrt(dual a) {
    dual r; r.v = sqrt(a.v);
    for (int k = 0; k < 3; ++k) r.g[k] = a.g[k] / (2.0 * r.v);
    return r;
}

/* ------------------------------------------------------------------------- */
/* real spherical harmonics by the associated Legendre recurrence              */
/* ------------------------------------------------------------------------- */
static double factorial(int n) { double f = 1.0; for (int k = 2; k <= n; ++k) f *= k; return f; }

/* Y_lm(rhat), orthonormal on the sphere, real form without the Condon-Shortley
 * phase:  m > 0: sqrt2 N_lm P_l^m(cos t) cos(m phi); m < 0: sqrt2 N_l|m| P_l^|m| sin(|m| phi);
 * m = 0: N_l0 P_l(cos t).  P_l^m(t)/(1-t^2)^(m/2) follows the three-term recurrence in l,
 * and (1-t^2)^(m/2) e^{i m phi} = ((x + i y)/r)^m. */
static void ylm_dual(dual x, dual y, dual z, dual* Y) {
    dual r = d_sqrt(d_add(d_add(d_mul(x, x), d_mul(y, y)), d_mul(z, z)));
    dual t = d_div(z, r), u = d_div(x, r), v = d_div(y, r);
    dual Q[LMAXO + 1][LMAXO + 1];
    for (int m = 0; m <= LMAXO; ++m) {
        double dfact = 1.0;                       /* (2m-1)!! */
        for (int k = 2 * m - 1; k > 1; k -= 2) dfact *= k;
        Q[m][m] = d_const(dfact);
        if (m + 1 <= LMAXO) Q[m + 1][m] = d_scale(d_mul(t, Q[m][m]), 2.0 * m + 1.0);
        for (int l = m + 2; l <= LMAXO; ++l) {
            dual a = d_scale(d_mul(t, Q[l - 1][m]), 2.0 * l - 1.0);
            dual b = d_scale(Q[l - 2][m], (double)(l + m - 1));
            Q[l][m] = d_scale(d_sub(a, b), 1.0 / (double)(l - m));
        }
    }
    dual cr[LMAXO + 1], ci[LMAXO + 1];
    cr[0] = d_const(1.0); ci[0] = d_const(0.0);
    for (int m = 1; m <= LMAXO; ++m) {
        cr[m] = d_sub(d_mul(cr[m - 1], u), d_mul(ci[m - 1], v));
        ci[m] = d_add(d_mul(cr[m - 1], v), d_mul(ci[m - 1], u));
    }
    for (int l = 0; l <= LMAXO; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double N = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
            dual val;
            if (m == 0) val = d_scale(Q[l][0], N);
            else if (m > 0) val = d_scale(d_mul(Q[l][am], cr[am]), sqrt(2.0) * N);
            else val = d_scale(d_mul(Q[l][am], ci[am]), sqrt(2.0) * N);
            Y[l * l + l + m] = val;
        }
    }
}

void or_ylm(double x, double y, double z, double* Y, double* grad) {
    dual Yd[NLMO];
    ylm_dual(d_var(x, 0), d_var(y, 1), d_var(z, 2), Yd);
    for (int k = 0; k < NLMO; ++k) {
        Y[k] = Yd[k].v;
        if (grad) { grad[3 * k] = Yd[k].g[0]; grad[3 * k + 1] = Yd[k].g[1]; grad[3 * k + 2] = Yd[k].g[2]; }
    }
}

/* ------------------------------------------------------------------------- */
/* Gaunt coefficients by quadrature: Gauss-Legendre (16) in cos(theta) times   */
/* the 32-point trapezoid rule in phi; exact for the degree-12 integrands here */
/* ------------------------------------------------------------------------- */
#define GL_N 16
#define PH_N 32
static double g_gaunt[LMAXO + 1][LMAXO + 1][LMAXO + 1][2 * LMAXO + 1][2 * LMAXO + 1][2 * LMAXO + 1];
static int g_gaunt_ready = 0;

static void gauss_legendre(int n, double* xs, double* ws) {
    for (int i = 0; i < n; ++i) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
            double dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
        double dp = n * (x * p1 - p0) / (x * x - 1.0);
        xs[i] = x;
        ws[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

static void gaunt_build(void) {
    if (g_gaunt_ready) return;
    double xs[GL_N], ws[GL_N];
    gauss_legendre(GL_N, xs, ws);
    static double Yq[GL_N * PH_N][NLMO];
    static double Wq[GL_N * PH_N];
    for (int a = 0; a < GL_N; ++a)
        for (int b = 0; b < PH_N; ++b) {
            double ct = xs[a], st = sqrt(1.0 - ct * ct), ph = 2.0 * M_PI * b / PH_N;
            or_ylm(st * cos(ph), st * sin(ph), ct, Yq[a * PH_N + b], NULL);
            Wq[a * PH_N + b] = ws[a] * 2.0 * M_PI / PH_N;
        }
    for (int l1 = 0; l1 <= LMAXO; ++l1)
        for (int l2 = 0; l2 <= LMAXO; ++l2)
            for (int l3 = 0; l3 <= LMAXO; ++l3)
                for (int m1 = -l1; m1 <= l1; ++m1)
                    for (int m2 = -l2; m2 <= l2; ++m2)
                        for (int m3 = -l3; m3 <= l3; ++m3) {
                            double s = 0.0;
                            for (int q = 0; q < GL_N * PH_N; ++q)
                                s += Wq[q] * Yq[q][l1 * l1 + l1 + m1] * Yq[q][l2 * l2 + l2 + m2] * Yq[q][l3 * l3 + l3 + m3];
                            if (fabs(s) < 1e-13) s = 0.0;
                            g_gaunt[l1][l2][l3][m1 + LMAXO][m2 + LMAXO][m3 + LMAXO] = s;
                        }
    g_gaunt_ready = 1;
}

double or_gaunt(int l1, int m1, int l2, int m2, int l3, int m3) {
    gaunt_build();
    if (l1 < 0 || l2 < 0 || l3 < 0 || l1 > LMAXO || l2 > LMAXO || l3 > LMAXO) return 0.0;
    if (m1 < -l1 || m1 > l1 || m2 < -l2 || m2 > l2 || m3 < -l3 || m3 > l3) return 0.0;
    return g_gaunt[l1][l2][l3][m1 + LMAXO][m2 + LMAXO][m3 + LMAXO];
}

/* ------------------------------------------------------------------------- */
/* radial basis: g_n(r) = T_n(2r/rc - 1) * fc(r), fc = (1 + cos(pi r / rc))/2   */
/* ------------------------------------------------------------------------- */
void or_radial(double r, double rc, int nmax, double* g, double* dg) {
    if (r >= rc) { for (int n = 0; n < nmax; ++n) { g[n] = 0.0; dg[n] = 0.0; } return; }
    double x = 2.0 * r / rc - 1.0, dxdr = 2.0 / rc;
    double fc = 0.5 * (1.0 + cos(M_PI * r / rc));
    double dfc = -0.5 * M_PI / rc * sin(M_PI * r / rc);
    double T[64], dT[64];
    T[0] = 1.0; dT[0] = 0.0;
    if (nmax > 1) { T[1] = x; dT[1] = 1.0; }
    for (int n = 2; n < nmax; ++n) {
        T[n] = 2.0 * x * T[n - 1] - T[n - 2];
        dT[n] = 2.0 * T[n - 1] + 2.0 * x * dT[n - 1] - dT[n - 2];
    }
    for (int n = 0; n < nmax; ++n) {
        g[n] = T[n] * fc;
        dg[n] = dT[n] * dxdr * fc + T[n] * dfc;
    }
}

/* ------------------------------------------------------------------------- */
/* EAM functions (Appendix B)                                                  */
/* ------------------------------------------------------------------------- */
static double max_knot(const double* d, int n) { double m = 0.0; for (int i = 0; i < n; ++i) if (d[i] > m) m = d[i]; return m; }

double or_eam_cutoff(const or_eam* p) {
    double a = max_knot(p->phi_d, p->n_phi), b = max_knot(p->rho_d, p->n_rho);
    return a > b ? a : b;
}

static void cubic_knots(const double* a, const double* d, int n, double r, double* f, double* df) {
    double s = 0.0, ds = 0.0;
    for (int i = 0; i < n; ++i) {
        double t = d[i] - r;
        if (t >= 0.0) { s += a[i] * t * t * t; ds -= 3.0 * a[i] * t * t; }   /* Theta(0) = 1 */
    }
    *f = s; *df = ds;
}

void or_eam_phi(const or_eam* p, double r, double* f, double* df) {
    if (p->zbl && r < p->r_lo) {
        /* Phi^ZBL = Z^2 / (4 pi eps0 r) * phi(r / a_ZBL) */
        const double c[4] = {0.1818, 0.5099, 0.2802, 0.02817};
        const double e[4] = {3.2, 0.9423, 0.4029, 0.2016};
        double k = p->zbl_Z * p->zbl_Z / (4.0 * M_PI * p->zbl_eps0);
        double x = r / p->zbl_a, ph = 0.0, dph = 0.0;
        for (int i = 0; i < 4; ++i) { double t = c[i] * exp(-e[i] * x); ph += t; dph -= e[i] * t; }
        *f = k * ph / r;
        *df = k * (dph / p->zbl_a / r - ph / (r * r));
        return;
    }
    if (p->zbl && r <= p->r_hi) {
        double s = 0.0, ds = 0.0, rp = 1.0;
        for (int m = 0; m < 6; ++m) { s += p->b[m] * rp; if (m < 5) ds += (m + 1) * p->b[m + 1] * rp; rp *= r; }
        *f = s; *df = ds;
        return;
    }
    cubic_knots(p->phi_a, p->phi_d, p->n_phi, r, f, df);
}

void or_eam_rho(const or_eam* p, double r, double* f, double* df) {
    if (p->rho_rclamp > 0.0 && r <= p->rho_rclamp) {
        double g;
        cubic_knots(p->rho_a, p->rho_d, p->n_rho, p->rho_rclamp, f, &g);
        *df = 0.0;
        return;
    }
    cubic_knots(p->rho_a, p->rho_d, p->n_rho, r, f, df);
}

void or_eam_embed(const or_eam* p, double rho, double* f, double* df) {
    /* reading: xi(rho <= 0) = 0, xi' = 0 (sqrt undefined; isolated atom has rho = 0) */
    if (rho <= 0.0) { *f = p->F_dxi; *df = 0.0; return; }
    double sq = sqrt(rho);
    *f = p->F_a1 * sq + p->F_a2 * rho * rho + p->F_dxi;
    *df = 0.5 * p->F_a1 / sq + 2.0 * p->F_a2 * rho;
}

/* ------------------------------------------------------------------------- */
/* ACE for one atom                                                            */
/* ------------------------------------------------------------------------- */
static int lmi(int l, int m) { return l * l + l + m; }

int or_ace_atom(const or_ace* ace, int nn, const double* rvec,
                double* E, double* phi1_out, double* phi2_out, double* B, double* f) {
    gaunt_build();
    const int NM = ace->nmax, LM = ace->lmax, NLM = (LM + 1) * (LM + 1);
    double* bval = (double*)calloc((size_t)(nn > 0 ? nn : 1) * NM * NLM, sizeof(double));
    double* bgrd = (double*)calloc((size_t)(nn > 0 ? nn : 1) * NM * NLM * 3, sizeof(double));
    double* A = (double*)calloc((size_t)NM * NLM, sizeof(double));
    double* dA = (double*)calloc((size_t)NM * NLM, sizeof(double));
    double g[64], dg[64], Y[NLMO], gY[3 * NLMO];

    /* atomic base A_nlm = (1/nref) sum_j g_n(r_ij) Y_lm(rhat_ij) */
    for (int j = 0; j < nn; ++j) {
        const double* rv = rvec + 3 * j;
        double r = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
        if (r >= ace->rc || r <= 0.0) continue;
        or_radial(r, ace->rc, NM, g, dg);
        or_ylm(rv[0], rv[1], rv[2], Y, gY);
        for (int n = 0; n < NM; ++n)
            for (int k = 0; k < NLM; ++k) {
                size_t o = ((size_t)j * NM + n) * NLM + k;
                bval[o] = g[n] * Y[k];
                for (int c = 0; c < 3; ++c) bgrd[3 * o + c] = dg[n] * (rv[c] / r) * Y[k] + g[n] * gY[3 * k + c];
                A[n * NLM + k] += bval[o] / ace->nref;
            }
    }

    /* product basis and the two densities */
    double phi1 = ace->c1_0, phi2 = ace->c2_0;
    for (int v = 0; v < ace->nfunc; ++v) {
        const int* q = ace->idx + 7 * v;
        double bv = 0.0;
        if (q[0] == 1) {
            bv = A[q[1] * NLM + lmi(0, 0)];
        } else if (q[0] == 2) {
            int l = q[2];
            for (int m = -l; m <= l; ++m) bv += A[q[1] * NLM + lmi(l, m)] * A[q[3] * NLM + lmi(l, m)];
        } else if (q[0] == 3) {
            int n1 = q[1], l1 = q[2], n2 = q[3], l2 = q[4], n3 = q[5], l3 = q[6];
            for (int m1 = -l1; m1 <= l1; ++m1)
                for (int m2 = -l2; m2 <= l2; ++m2)
                    for (int m3 = -l3; m3 <= l3; ++m3) {
                        double G = g_gaunt[l1][l2][l3][m1 + LMAXO][m2 + LMAXO][m3 + LMAXO];
                        if (G == 0.0) continue;
                        bv += G * A[n1 * NLM + lmi(l1, m1)] * A[n2 * NLM + lmi(l2, m2)] * A[n3 * NLM + lmi(l3, m3)];
                    }
        }
        if (B) B[v] = bv;
        phi1 += ace->c1[v] * bv;
        phi2 += ace->c2[v] * bv;
    }
    if (phi1_out) *phi1_out = phi1;
    if (phi2_out) *phi2_out = phi2;
    int status = 0;
    if (!(phi2 > 1e-3)) {
        status = -4;
        *E = NAN;
        if (f) for (int j = 0; j < 3 * nn; ++j) f[j] = 0.0;
        goto done;
    }
    *E = phi1 + sqrt(phi2);
    if (f) {
        /* dE/dA = sum_v (c1_v + c2_v / (2 sqrt(phi2))) dB_v/dA */
        double s = 0.5 / sqrt(phi2);
        for (int v = 0; v < ace->nfunc; ++v) {
            const int* q = ace->idx + 7 * v;
            double cf = ace->c1[v] + s * ace->c2[v];
            if (q[0] == 1) {
                dA[q[1] * NLM + lmi(0, 0)] += cf;
            } else if (q[0] == 2) {
                int l = q[2];
                for (int m = -l; m <= l; ++m) {
                    dA[q[1] * NLM + lmi(l, m)] += cf * A[q[3] * NLM + lmi(l, m)];
                    dA[q[3] * NLM + lmi(l, m)] += cf * A[q[1] * NLM + lmi(l, m)];
                }
            } else if (q[0] == 3) {
                int n1 = q[1], l1 = q[2], n2 = q[3], l2 = q[4], n3 = q[5], l3 = q[6];
                for (int m1 = -l1; m1 <= l1; ++m1)
                    for (int m2 = -l2; m2 <= l2; ++m2)
                        for (int m3 = -l3; m3 <= l3; ++m3) {
                            double G = g_gaunt[l1][l2][l3][m1 + LMAXO][m2 + LMAXO][m3 + LMAXO];
                            if (G == 0.0) continue;
                            double a1 = A[n1 * NLM + lmi(l1, m1)], a2 = A[n2 * NLM + lmi(l2, m2)], a3 = A[n3 * NLM + lmi(l3, m3)];
                            dA[n1 * NLM + lmi(l1, m1)] += cf * G * a2 * a3;
                            dA[n2 * NLM + lmi(l2, m2)] += cf * G * a1 * a3;
                            dA[n3 * NLM + lmi(l3, m3)] += cf * G * a1 * a2;
                        }
            }
        }
        /* f_j = dE/dr_ij = (1/nref) sum_{n,lm} dE/dA_nlm grad_j (g_n Y_lm) */
        for (int j = 0; j < nn; ++j)
            for (int c = 0; c < 3; ++c) {
                double s3 = 0.0;
                for (int n = 0; n < NM; ++n)
                    for (int k = 0; k < NLM; ++k)
                        s3 += dA[n * NLM + k] * bgrd[3 * (((size_t)j * NM + n) * NLM + k) + c];
                f[3 * j + c] = s3 / ace->nref;
            }
    }
done:
    free(bval); free(bgrd); free(A); free(dA);
    return status;
}

/* ------------------------------------------------------------------------- */
/* neighbour search                                                            */
/* ------------------------------------------------------------------------- */
static void inv3(const double* M, double* R) {
    double a = M[0], b = M[1], c = M[2], d = M[3], e = M[4], f = M[5], g = M[6], h = M[7], i = M[8];
    double det = a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
    R[0] = (e * i - f * h) / det; R[1] = (c * h - b * i) / det; R[2] = (b * f - c * e) / det;
    R[3] = (f * g - d * i) / det; R[4] = (a * i - c * g) / det; R[5] = (c * d - a * f) / det;
    R[6] = (d * h - e * g) / det; R[7] = (b * g - a * h) / det; R[8] = (a * e - b * d) / det;
}

static void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1]; c[1] = a[2] * b[0] - a[0] * b[2]; c[2] = a[0] * b[1] - a[1] * b[0];
}

typedef struct {
    const or_system* sys;
    double Minv[9];
    int nc[3], S[3];
    double* xw;        /* wrapped positions */
    int* cell;         /* cell of each atom */
    int* cstart;       /* CSR over cells   */
    int* catoms;
} grid_t;

static void perp_widths(const double* h, double* w) {
    double c[3], V;
    cross3(h + 3, h + 6, c);
    V = fabs(h[0] * c[0] + h[1] * c[1] + h[2] * c[2]);
    w[0] = V / sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    cross3(h + 6, h + 0, c); w[1] = V / sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    cross3(h + 0, h + 3, c); w[2] = V / sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
}

static void grid_build(grid_t* G, const or_system* sys, double rc) {
    G->sys = sys;
    inv3(sys->h, G->Minv);
    double pw[3];
    perp_widths(sys->h, pw);
    for (int d = 0; d < 3; ++d) {
        int n = (int)floor(pw[d] / rc);
        if (n < 1) n = 1;
        if (n > 400) n = 400;
        G->nc[d] = n;
        G->S[d] = (int)ceil(rc * n / pw[d] - 1e-12);
        if (G->S[d] < 1) G->S[d] = 1;
    }
    int N = sys->n;
    size_t ncell = (size_t)G->nc[0] * G->nc[1] * G->nc[2];
    G->xw = (double*)malloc(sizeof(double) * 3 * (N > 0 ? N : 1));
    G->cell = (int*)malloc(sizeof(int) * (N > 0 ? N : 1));
    G->cstart = (int*)calloc(ncell + 1, sizeof(int));
    G->catoms = (int*)malloc(sizeof(int) * (N > 0 ? N : 1));
    for (int i = 0; i < N; ++i) {
        double d[3], s[3];
        for (int k = 0; k < 3; ++k) d[k] = sys->x[3 * i + k] - sys->origin[k];
        for (int k = 0; k < 3; ++k) s[k] = d[0] * G->Minv[0 + k] + d[1] * G->Minv[3 + k] + d[2] * G->Minv[6 + k];
        int c[3];
        for (int k = 0; k < 3; ++k) {
            if (sys->periodic[k]) s[k] -= floor(s[k]);
            c[k] = (int)floor(s[k] * G->nc[k]);
            if (c[k] < 0) c[k] = 0;
            if (c[k] >= G->nc[k]) c[k] = G->nc[k] - 1;
        }
        for (int k = 0; k < 3; ++k)
            G->xw[3 * i + k] = sys->origin[k] + s[0] * sys->h[0 + k] + s[1] * sys->h[3 + k] + s[2] * sys->h[6 + k];
        G->cell[i] = (c[0] * G->nc[1] + c[1]) * G->nc[2] + c[2];
        G->cstart[G->cell[i] + 1]++;
    }
    for (size_t c = 0; c < ncell; ++c) G->cstart[c + 1] += G->cstart[c];
    int* fill = (int*)calloc(ncell, sizeof(int));
    for (int i = 0; i < N; ++i) { int c = G->cell[i]; G->catoms[G->cstart[c] + fill[c]++] = i; }
    free(fill);
}

static void grid_free(grid_t* G) { free(G->xw); free(G->cell); free(G->cstart); free(G->catoms); }

/* Visit every (j, image) within rc of atom i.  cb == NULL counts only. */
typedef void (*pair_cb)(void* ctx, int i, int j, const double* r);
static long grid_visit(const grid_t* G, int i, double rc, pair_cb cb, void* ctx) {
    const or_system* sys = G->sys;
    int ci = G->cell[i];
    int c0 = ci / (G->nc[1] * G->nc[2]), c1 = (ci / G->nc[2]) % G->nc[1], c2 = ci % G->nc[2];
    long cnt = 0;
    double rc2 = rc * rc;
    for (int o0 = -G->S[0]; o0 <= G->S[0]; ++o0)
        for (int o1 = -G->S[1]; o1 <= G->S[1]; ++o1)
            for (int o2 = -G->S[2]; o2 <= G->S[2]; ++o2) {
                int n[3] = {c0 + o0, c1 + o1, c2 + o2}, img[3] = {0, 0, 0}, ok = 1;
                for (int k = 0; k < 3; ++k) {
                    if (sys->periodic[k]) {
                        img[k] = (int)floor((double)n[k] / G->nc[k]);
                        n[k] -= img[k] * G->nc[k];
                    } else if (n[k] < 0 || n[k] >= G->nc[k]) ok = 0;
                }
                if (!ok) continue;
                int cn = (n[0] * G->nc[1] + n[1]) * G->nc[2] + n[2];
                double shift[3];
                for (int k = 0; k < 3; ++k) shift[k] = img[0] * sys->h[0 + k] + img[1] * sys->h[3 + k] + img[2] * sys->h[6 + k];
                for (int q = G->cstart[cn]; q < G->cstart[cn + 1]; ++q) {
                    int j = G->catoms[q];
                    if (j == i && img[0] == 0 && img[1] == 0 && img[2] == 0) continue;
                    double r[3];
                    for (int k = 0; k < 3; ++k) r[k] = G->xw[3 * j + k] + shift[k] - G->xw[3 * i + k];
                    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                    if (r2 < rc2) { if (cb) cb(ctx, i, j, r); ++cnt; }
                }
            }
    return cnt;
}

typedef struct { long* cnt; long cap; int* pi; int* pj; double* rv; int over; } collect_t;
static void collect_pair(void* ctx, int i, int j, const double* r) {
    collect_t* a = (collect_t*)ctx;
    if (*a->cnt >= a->cap) { a->over = 1; return; }
    long c = *a->cnt;
    a->pi[c] = i; a->pj[c] = j;
    for (int k = 0; k < 3; ++k) a->rv[3 * c + k] = r[k];
    *a->cnt = c + 1;
}

long or_neighbors(const or_system* sys, double rc, int mode, long cap, int* pi, int* pj, double* rvec) {
    long cnt = 0;
    if (mode == 1) {
        double pw[3];
        int S[3];
        perp_widths(sys->h, pw);
        for (int k = 0; k < 3; ++k) S[k] = sys->periodic[k] ? (int)ceil(rc / pw[k]) + 1 : 0;
        for (int i = 0; i < sys->n; ++i)
            for (int j = 0; j < sys->n; ++j)
                for (int a = -S[0]; a <= S[0]; ++a)
                    for (int b = -S[1]; b <= S[1]; ++b)
                        for (int c = -S[2]; c <= S[2]; ++c) {
                            if (i == j && a == 0 && b == 0 && c == 0) continue;
                            double r[3];
                            for (int k = 0; k < 3; ++k)
                                r[k] = sys->x[3 * j + k] + a * sys->h[k] + b * sys->h[3 + k] + c * sys->h[6 + k] - sys->x[3 * i + k];
                            if (r[0] * r[0] + r[1] * r[1] + r[2] * r[2] < rc * rc) {
                                if (cnt >= cap) return -1;
                                pi[cnt] = i; pj[cnt] = j;
                                for (int k = 0; k < 3; ++k) rvec[3 * cnt + k] = r[k];
                                ++cnt;
                            }
                        }
        return cnt;
    }
    grid_t G;
    grid_build(&G, sys, rc);
    collect_t acc = {&cnt, cap, pi, pj, rvec, 0};
    for (int i = 0; i < sys->n && !acc.over; ++i) grid_visit(&G, i, rc, collect_pair, &acc);
    grid_free(&G);
    return acc.over ? -1 : cnt;
}

/* per-center neighbour lists (CSR) */
typedef struct { int* j; double* r; long n; long cap; } nlist_t;
static void nl_push(void* ctx, int i, int j, const double* r) {
    (void)i;
    nlist_t* L = (nlist_t*)ctx;
    L->j[L->n] = j;
    for (int k = 0; k < 3; ++k) L->r[3 * L->n + k] = r[k];
    L->n++;
}

/* ------------------------------------------------------------------------- */
/* weights and indenter                                                        */
/* ------------------------------------------------------------------------- */
/* Cosine switch of the distance to the region centre.  In periodic directions the
 * distance is taken to the nearest image of the centre (fractional coordinates rounded). */
static void region_weight(const or_region* reg, int i, const or_system* sys, const double* Minv,
                          double* w, double* gw) {
    gw[0] = gw[1] = gw[2] = 0.0;
    if (reg == NULL) { *w = 0.0; return; }
    if (reg->kind == 0) { *w = reg->w_explicit ? reg->w_explicit[i] : 0.0; return; }
    if (reg->kind == 2) { *w = reg->w_const; return; }
    const double* x = sys->x + 3 * i;
    double d[3] = {x[0] - reg->center[0], x[1] - reg->center[1], x[2] - reg->center[2]};
    double s[3];
    for (int k = 0; k < 3; ++k) s[k] = d[0] * Minv[0 + k] + d[1] * Minv[3 + k] + d[2] * Minv[6 + k];
    for (int k = 0; k < 3; ++k)
        if (sys->periodic[k]) {
            double m = floor(s[k] + 0.5);
            for (int c = 0; c < 3; ++c) d[c] -= m * sys->h[3 * k + c];
        }
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (r < reg->r_in) { *w = 1.0; return; }
    if (r >= reg->r_in + reg->r_sw) { *w = 0.0; return; }
    /* S = (1 + cos a)/2, written as cos^2(a/2): the same function, but positive for every
     * r < r_in + r_sw in floating point, so that the compaction rule w > 0 selects exactly
     * the atoms inside the outer radius */
    double a = M_PI * (r - reg->r_in) / reg->r_sw;
    double ch = cos(0.5 * a);
    *w = ch * ch;
    double ds = -0.5 * M_PI / reg->r_sw * sin(a);
    for (int k = 0; k < 3; ++k) gw[k] = ds * d[k] / r;
}

/* ------------------------------------------------------------------------- */
/* the full AP evaluation                                                      */
/* ------------------------------------------------------------------------- */
int or_evaluate(const or_system* sys, const or_eam* eam, const or_ace* ace,
                const or_region* reg, const or_indenter* ind,
                const unsigned char* centers, int nthreads,
                double* forces, double* e_atom, double* e_eam_out, double* e_ace_out,
                double* w_out, or_result* res) {
    gaunt_build();
    const int N = sys->n;
    double rc = 0.0;
    if (eam) rc = or_eam_cutoff(eam);
    if (ace && ace->rc > rc) rc = ace->rc;
    memset(res, 0, sizeof(*res));
    res->bad_atom = -1;
    memset(forces, 0, sizeof(double) * 3 * (size_t)N);

    int nc = 0;
    int* clist = (int*)malloc(sizeof(int) * (N > 0 ? N : 1));
    for (int i = 0; i < N; ++i) if (!centers || centers[i]) clist[nc++] = i;

    grid_t G;
    grid_build(&G, sys, rc > 0.0 ? rc : 1.0);
    long* start = (long*)calloc((size_t)nc + 1, sizeof(long));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel for schedule(dynamic, 64)
    for (int q = 0; q < nc; ++q) start[q + 1] = grid_visit(&G, clist[q], rc, NULL, NULL);
    for (int q = 0; q < nc; ++q) start[q + 1] += start[q];
    long npair = start[nc];
    int* pj = (int*)malloc(sizeof(int) * (npair > 0 ? npair : 1));
    double* pr = (double*)malloc(sizeof(double) * 3 * (npair > 0 ? npair : 1));
    double* pd = (double*)calloc(3 * (size_t)(npair > 0 ? npair : 1), sizeof(double));  /* weighted dE_i/dr_ij */
    #pragma omp parallel for schedule(dynamic, 64)
    for (int q = 0; q < nc; ++q) {
        nlist_t L = {pj + start[q], pr + 3 * start[q], 0, 0};
        grid_visit(&G, clist[q], rc, nl_push, &L);
    }

    double* wv = (double*)calloc((size_t)nc + 1, sizeof(double));
    double* gw = (double*)calloc(3 * (size_t)nc + 1, sizeof(double));
    double* eE = (double*)calloc((size_t)nc + 1, sizeof(double));
    double* eA = (double*)calloc((size_t)nc + 1, sizeof(double));
    int* st = (int*)calloc((size_t)nc + 1, sizeof(int));

    #pragma omp parallel for schedule(dynamic, 8)
    for (int q = 0; q < nc; ++q) {
        int i = clist[q];
        long s0 = start[q], s1 = start[q + 1];
        int nn = (int)(s1 - s0);
        double w;
        region_weight(reg, i, sys, G.Minv, &w, gw + 3 * q);
        wv[q] = w;
        double u = 1.0 - w;
        if (u > 0.0 && eam) {
            /* E_i^EAM = xi(rho_i) + Delta xi + 1/2 sum_j Phi(r_ij), rho_i = sum_j zeta(r_ij) */
            double rho = 0.0, ephi = 0.0;
            for (long p = s0; p < s1; ++p) {
                const double* r = pr + 3 * p;
                double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                double f, df;
                or_eam_rho(eam, d, &f, &df);
                rho += f;
                or_eam_phi(eam, d, &f, &df);
                ephi += 0.5 * f;
            }
            if (rho < 0.0) st[q] = -4;
            double F, dF;
            or_eam_embed(eam, rho, &F, &dF);
            eE[q] = F + ephi;
            for (long p = s0; p < s1; ++p) {
                const double* r = pr + 3 * p;
                double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                double fr, dfr, fp, dfp;
                or_eam_rho(eam, d, &fr, &dfr);
                or_eam_phi(eam, d, &fp, &dfp);
                double c = dF * dfr + 0.5 * dfp;          /* dE_i/d|r_ij| */
                for (int k = 0; k < 3; ++k) pd[3 * p + k] += u * c * r[k] / d;
            }
        }
        if (w > 0.0 && ace) {
            double E, p1, p2;
            double* f = (double*)malloc(sizeof(double) * 3 * (nn > 0 ? nn : 1));
            int s = or_ace_atom(ace, nn, pr + 3 * s0, &E, &p1, &p2, NULL, f);
            if (s != 0) st[q] = s;
            eA[q] = E;
            for (int p = 0; p < nn; ++p)
                for (int k = 0; k < 3; ++k) pd[3 * (s0 + p) + k] += w * f[3 * p + k];
            free(f);
        }
    }

    /* accumulate: F_j -= dE_i/dr_ij, F_i += dE_i/dr_ij; virial -= r_ij (x) dE_i/dr_ij */
    double vir[3][3] = {{0}};
    for (int q = 0; q < nc; ++q) {
        int i = clist[q];
        for (long p = start[q]; p < start[q + 1]; ++p) {
            int j = pj[p];
            for (int k = 0; k < 3; ++k) {
                forces[3 * j + k] -= pd[3 * p + k];
                forces[3 * i + k] += pd[3 * p + k];
            }
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) vir[a][b] -= pr[3 * p + a] * pd[3 * p + b];
        }
    }
    res->virial[0] = vir[0][0]; res->virial[1] = vir[1][1]; res->virial[2] = vir[2][2];
    res->virial[3] = 0.5 * (vir[0][1] + vir[1][0]);
    res->virial[4] = 0.5 * (vir[0][2] + vir[2][0]);
    res->virial[5] = 0.5 * (vir[1][2] + vir[2][1]);

    double etot = 0.0, eind = 0.0, load = 0.0;
    for (int q = 0; q < nc; ++q) {
        int i = clist[q];
        double w = wv[q], u = 1.0 - w;
        double ei = 0.0;
        if (w > 0.0) { ei += w * eA[q]; res->n_ace++; }
        if (u > 0.0) ei += u * eE[q];
        /* position-dependent weight: -grad w_i (E_i^ACE - E_i^EAM) */
        if (reg && reg->kind == 1 && w > 0.0 && u > 0.0)
            for (int k = 0; k < 3; ++k) forces[3 * i + k] -= gw[3 * q + k] * (eA[q] - eE[q]);
        if (ind && ind->enabled) {
            /* the tip interacts with the nearest periodic image of each atom */
            double d[3] = {sys->x[3 * i] - ind->center[0], sys->x[3 * i + 1] - ind->center[1], sys->x[3 * i + 2] - ind->center[2]};
            double s[3];
            for (int k = 0; k < 3; ++k) s[k] = d[0] * G.Minv[0 + k] + d[1] * G.Minv[3 + k] + d[2] * G.Minv[6 + k];
            for (int k = 0; k < 3; ++k)
                if (sys->periodic[k]) {
                    double m = floor(s[k] + 0.5);
                    for (int c = 0; c < 3; ++c) d[c] -= m * sys->h[3 * k + c];
                }
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r < ind->R && r > 0.0) {
                double h = ind->R - r;
                double V = ind->K * h * h * h / 3.0;
                eind += V;
                ei += V;
                double fi[3];
                for (int k = 0; k < 3; ++k) { fi[k] = ind->K * h * h * d[k] / r; forces[3 * i + k] += fi[k]; }
                load += fi[0] * ind->dir[0] + fi[1] * ind->dir[1] + fi[2] * ind->dir[2];
            }
        }
        if (e_atom) e_atom[i] = ei;
        if (e_eam_out) e_eam_out[i] = eE[q];
        if (e_ace_out) e_ace_out[i] = eA[q];
        if (w_out) w_out[i] = w;
        etot += ei;
        if (st[q] != 0 && res->status == 0) { res->status = st[q]; res->bad_atom = i; }
    }
    res->e_total = etot;
    res->e_indenter = eind;
    res->load = load;

    free(clist); free(start); free(pj); free(pr); free(pd); free(wv); free(gw); free(eE); free(eA); free(st);
    grid_free(&G);
    return res->status;
}

/* ------------------------------------------------------------------------- */
/* velocity Verlet                                                             */
/* ------------------------------------------------------------------------- */
#define OR_FTM 0.0096485332   /* 1 eV/(Angstrom amu) in Angstrom/fs^2 */

int or_md(const or_system* sys0, const or_eam* eam, const or_ace* ace,
          const or_region* reg0, const or_indenter* ind0, const double* ind_vel,
          int region_follows, const unsigned char* fixed, double mass, double dt,
          int nsteps, int nthreads, double* x, double* v, double* epot, double* ekin) {
    const int N = sys0->n;
    or_system sys = *sys0;
    sys.x = x;
    or_region reg;
    or_indenter ind;
    if (reg0) reg = *reg0;
    if (ind0) ind = *ind0;
    double* F = (double*)malloc(sizeof(double) * 3 * (N > 0 ? N : 1));
    or_result res;
    int status = or_evaluate(&sys, eam, ace, reg0 ? &reg : NULL, ind0 ? &ind : NULL, NULL, nthreads, F, NULL, NULL, NULL, NULL, &res);
    double a = dt * OR_FTM / mass;
    for (int k = 0; k <= nsteps; ++k) {
        if (k > 0) {
            for (int i = 0; i < N; ++i) {
                if (fixed && fixed[i]) continue;
                for (int c = 0; c < 3; ++c) { v[3 * i + c] += 0.5 * a * F[3 * i + c]; x[3 * i + c] += dt * v[3 * i + c]; }
            }
            if (ind0 && ind_vel) for (int c = 0; c < 3; ++c) ind.center[c] -= ind_vel[c] * dt;
            if (reg0 && region_follows && ind_vel) for (int c = 0; c < 3; ++c) reg.center[c] -= ind_vel[c] * dt;
            int s = or_evaluate(&sys, eam, ace, reg0 ? &reg : NULL, ind0 ? &ind : NULL, NULL, nthreads, F, NULL, NULL, NULL, NULL, &res);
            if (s != 0 && status == 0) status = s;
            for (int i = 0; i < N; ++i) {
                if (fixed && fixed[i]) continue;
                for (int c = 0; c < 3; ++c) v[3 * i + c] += 0.5 * a * F[3 * i + c];
            }
        }
        double ke = 0.0;
        for (int i = 0; i < N; ++i)
            for (int c = 0; c < 3; ++c) ke += 0.5 * mass * v[3 * i + c] * v[3 * i + c] / OR_FTM;
        if (epot) epot[k] = res.e_total;
        if (ekin) ekin[k] = ke;
    }
    free(F);
    return status;
}

/* ------------------------------------------------------------------------- */
/* centro-symmetry parameter                                                   */
/* ------------------------------------------------------------------------- */
static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

typedef struct { double r2; double r[3]; } nbv_t;
static int cmp_nbv(const void* a, const void* b) {
    double x = ((const nbv_t*)a)->r2, y = ((const nbv_t*)b)->r2;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int or_csp(const or_system* sys, int n_nb, double rc, double* csp, int* coord) {
    if (n_nb < 2 || n_nb > 16 || (n_nb & 1) || !(rc > 0.0)) return -1;
    grid_t G;
    grid_build(&G, sys, rc);
    const int N = sys->n;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < N; ++i) {
        long m = grid_visit(&G, i, rc, NULL, NULL);
        int* jj = (int*)malloc(sizeof(int) * (m > 0 ? m : 1));
        double* rr = (double*)malloc(sizeof(double) * 3 * (m > 0 ? m : 1));
        nlist_t L = {jj, rr, 0, m};
        grid_visit(&G, i, rc, nl_push, &L);
        if (coord) coord[i] = (int)m;
        if (m < n_nb) {
            csp[i] = -1.0;
        } else {
            /* the n_nb nearest */
            nbv_t* v = (nbv_t*)malloc(sizeof(nbv_t) * m);
            for (long q = 0; q < m; ++q) {
                for (int k = 0; k < 3; ++k) v[q].r[k] = rr[3 * q + k];
                v[q].r2 = rr[3 * q] * rr[3 * q] + rr[3 * q + 1] * rr[3 * q + 1] + rr[3 * q + 2] * rr[3 * q + 2];
            }
            qsort(v, (size_t)m, sizeof(nbv_t), cmp_nbv);
            /* all pairs, the n_nb/2 smallest |R_j + R_k|^2 */
            const int np = n_nb * (n_nb - 1) / 2;
            double* ps = (double*)malloc(sizeof(double) * np);
            int c = 0;
            for (int a = 0; a < n_nb; ++a)
                for (int b = a + 1; b < n_nb; ++b) {
                    double s0 = v[a].r[0] + v[b].r[0], s1 = v[a].r[1] + v[b].r[1], s2 = v[a].r[2] + v[b].r[2];
                    ps[c++] = s0 * s0 + s1 * s1 + s2 * s2;
                }
            qsort(ps, (size_t)np, sizeof(double), cmp_double);
            double sum = 0.0;
            for (int q = 0; q < n_nb / 2; ++q) sum += ps[q];
            csp[i] = sum;
            free(ps);
            free(v);
        }
        free(jj);
        free(rr);
    }
    grid_free(&G);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Nose-Hoover thermostat on a group                                           */
/* ------------------------------------------------------------------------- */
#define OR_KB 8.617333262e-5    /* Boltzmann constant, eV/K */

static double group_ke(const double* v, const unsigned char* group, int N, double mass) {
    double ke = 0.0;
    for (int i = 0; i < N; ++i)
        if (group[i])
            for (int c = 0; c < 3; ++c) ke += 0.5 * mass * v[3 * i + c] * v[3 * i + c] / OR_FTM;
    return ke;
}

/* one half step dt/2 of the thermostat: updates xi, eta and the group velocities */
static void nh_half(double* v, const unsigned char* group, int N, double mass, double dt, double nfkt, double Q,
                    double* xi, double* eta) {
    double ke = group_ke(v, group, N, mass);
    *xi += 0.25 * dt * (2.0 * ke - nfkt) / Q;
    double s = exp(-0.5 * dt * (*xi));
    for (int i = 0; i < N; ++i)
        if (group[i])
            for (int c = 0; c < 3; ++c) v[3 * i + c] *= s;
    ke *= s * s;
    *eta += 0.5 * dt * (*xi);
    *xi += 0.25 * dt * (2.0 * ke - nfkt) / Q;
}

int or_md_nh(const or_system* sys0, const or_eam* eam, const or_ace* ace,
             const or_region* reg0, const or_indenter* ind0, const double* ind_vel,
             int region_follows, const unsigned char* fixed, const unsigned char* group,
             double t_target, double tau, double mass, double dt, int nsteps, int nthreads,
             double* x, double* v, double* epot, double* ekin, double* ethermo) {
    const int N = sys0->n;
    or_system sys = *sys0;
    sys.x = x;
    or_region reg;
    or_indenter ind;
    if (reg0) reg = *reg0;
    if (ind0) ind = *ind0;
    int ng = 0;
    for (int i = 0; i < N; ++i) if (group[i] && !(fixed && fixed[i])) ++ng;
    const double nfkt = 3.0 * ng * OR_KB * t_target, Q = nfkt * tau * tau;
    unsigned char* g = (unsigned char*)malloc(N > 0 ? N : 1);
    for (int i = 0; i < N; ++i) g[i] = group[i] && !(fixed && fixed[i]);
    double xi = 0.0, eta = 0.0;
    double* F = (double*)malloc(sizeof(double) * 3 * (N > 0 ? N : 1));
    or_result res;
    int status = or_evaluate(&sys, eam, ace, reg0 ? &reg : NULL, ind0 ? &ind : NULL, NULL, nthreads, F, NULL, NULL, NULL, NULL, &res);
    double a = dt * OR_FTM / mass;
    for (int k = 0; k <= nsteps; ++k) {
        if (k > 0) {
            if (ng > 0) nh_half(v, g, N, mass, dt, nfkt, Q, &xi, &eta);
            for (int i = 0; i < N; ++i) {
                if (fixed && fixed[i]) continue;
                for (int c = 0; c < 3; ++c) { v[3 * i + c] += 0.5 * a * F[3 * i + c]; x[3 * i + c] += dt * v[3 * i + c]; }
            }
            if (ind0 && ind_vel) for (int c = 0; c < 3; ++c) ind.center[c] -= ind_vel[c] * dt;
            if (reg0 && region_follows && ind_vel) for (int c = 0; c < 3; ++c) reg.center[c] -= ind_vel[c] * dt;
            int s = or_evaluate(&sys, eam, ace, reg0 ? &reg : NULL, ind0 ? &ind : NULL, NULL, nthreads, F, NULL, NULL, NULL, NULL, &res);
            if (s != 0 && status == 0) status = s;
            for (int i = 0; i < N; ++i) {
                if (fixed && fixed[i]) continue;
                for (int c = 0; c < 3; ++c) v[3 * i + c] += 0.5 * a * F[3 * i + c];
            }
            if (ng > 0) nh_half(v, g, N, mass, dt, nfkt, Q, &xi, &eta);
        }
        double ke = 0.0;
        for (int i = 0; i < N; ++i)
            for (int c = 0; c < 3; ++c) ke += 0.5 * mass * v[3 * i + c] * v[3 * i + c] / OR_FTM;
        if (epot) epot[k] = res.e_total;
        if (ekin) ekin[k] = ke;
        if (ethermo) ethermo[k] = 0.5 * Q * xi * xi + nfkt * eta;
    }
    free(F);
    free(g);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 and the Langevin thermostat                                   */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const unsigned int* ctr, const unsigned int* key, unsigned int* out) {
    unsigned int c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    unsigned int k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
        unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        unsigned int hi0 = (unsigned int)(p0 >> 32), lo0 = (unsigned int)p0;
        unsigned int hi1 = (unsigned int)(p1 >> 32), lo1 = (unsigned int)p1;
        unsigned int n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void gauss3(int i, int step, unsigned long long seed, double* g) {
    unsigned int ctr[4] = {(unsigned int)i, (unsigned int)step, 0u, 0u};
    unsigned int key[2] = {(unsigned int)(seed & 0xffffffffu), (unsigned int)(seed >> 32)};
    unsigned int w[4];
    or_philox4x32_10(ctr, key, w);
    const double two32 = 4294967296.0;
    double u1 = ((double)w[0] + 1.0) / two32, u2 = ((double)w[1] + 0.5) / two32;
    double r = sqrt(-2.0 * log(u1));
    g[0] = r * cos(2.0 * M_PI * u2);
    g[1] = r * sin(2.0 * M_PI * u2);
    double u3 = ((double)w[2] + 1.0) / two32, u4 = ((double)w[3] + 0.5) / two32;
    g[2] = sqrt(-2.0 * log(u3)) * cos(2.0 * M_PI * u4);
}

int or_md_langevin(const or_system* sys0, const or_eam* eam, const or_ace* ace,
                   const or_region* reg0, const or_indenter* ind0, const double* ind_vel,
                   int region_follows, const unsigned char* fixed, const unsigned char* group,
                   double t_target, double tau, unsigned long long seed, int zero_every,
                   double mass, double dt, int nsteps, int nthreads,
                   double* x, double* v, double* epot, double* ekin) {
    const int N = sys0->n;
    or_system sys = *sys0;
    sys.x = x;
    or_region reg;
    or_indenter ind;
    if (reg0) reg = *reg0;
    if (ind0) ind = *ind0;
    double* F = (double*)malloc(sizeof(double) * 3 * (N > 0 ? N : 1));
    or_result res;
    int status = or_evaluate(&sys, eam, ace, reg0 ? &reg : NULL, ind0 ? &ind : NULL, NULL, nthreads, F, NULL, NULL, NULL, NULL, &res);
    const double a = dt * OR_FTM / mass;
    /* drag and random force in eV/A: m v / tau with m in amu, v in A/fs -> / OR_FTM */
    const double drag = mass / (tau * OR_FTM);
    const double sig = sqrt(2.0 * mass * OR_KB * t_target / (tau * dt * OR_FTM));
    for (int k = 0; k <= nsteps; ++k) {
        if (k > 0) {
            for (int i = 0; i < N; ++i) {
                if (fixed && fixed[i]) continue;
                for (int c = 0; c < 3; ++c) { v[3 * i + c] += 0.5 * a * F[3 * i + c]; x[3 * i + c] += dt * v[3 * i + c]; }
            }
            if (ind0 && ind_vel) for (int c = 0; c < 3; ++c) ind.center[c] -= ind_vel[c] * dt;
            if (reg0 && region_follows && ind_vel) for (int c = 0; c < 3; ++c) reg.center[c] -= ind_vel[c] * dt;
            int s = or_evaluate(&sys, eam, ace, reg0 ? &reg : NULL, ind0 ? &ind : NULL, NULL, nthreads, F, NULL, NULL, NULL, NULL, &res);
            if (s != 0 && status == 0) status = s;
            for (int i = 0; i < N; ++i) {
                if (!group[i] || (fixed && fixed[i])) continue;
                double g[3];
                gauss3(i, k, seed, g);
                for (int c = 0; c < 3; ++c) F[3 * i + c] += -drag * v[3 * i + c] + sig * g[c];
            }
            for (int i = 0; i < N; ++i) {
                if (fixed && fixed[i]) continue;
                for (int c = 0; c < 3; ++c) v[3 * i + c] += 0.5 * a * F[3 * i + c];
            }
            if (zero_every > 0 && k % zero_every == 0) {
                double vc[3] = {0, 0, 0};
                int nf = 0;
                for (int i = 0; i < N; ++i) {
                    if (fixed && fixed[i]) continue;
                    for (int c = 0; c < 3; ++c) vc[c] += v[3 * i + c];
                    ++nf;
                }
                if (nf > 0)
                    for (int i = 0; i < N; ++i) {
                        if (fixed && fixed[i]) continue;
                        for (int c = 0; c < 3; ++c) v[3 * i + c] -= vc[c] / nf;
                    }
            }
        }
        double ke = 0.0;
        for (int i = 0; i < N; ++i)
            for (int c = 0; c < 3; ++c) ke += 0.5 * mass * v[3 * i + c] * v[3 * i + c] / OR_FTM;
        if (epot) epot[k] = res.e_total;
        if (ekin) ekin[k] = ke;
    }
    free(F);
    return status;
}
