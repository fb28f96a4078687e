// tables.cpp -- host-side table generators of the AP library.
//
//  * EAM (Appendix B, Eqs. eam_Phi_Marinica, eam_rho_Marinica, tungsten_rho_up,
//    tungsten_Phi_up): each function is split at its knots (and at r_lo, r_hi, r_cut^rho)
//    into intervals on which it is a single polynomial of degree <= 5.  The polynomial is
//    re-expanded in FP64 about the interval midpoint, so the FP32 device evaluation never
//    forms the large cancelling terms of the printed forms (a_1 = 3663.54 against
//    a_2 = -3663.85 at nearly the same knot; the quintic bridge coefficients of 1e4-1e5).
//  * Real Gaunt coefficients for the ACE product basis (Sec. 2.2.2): Racah's closed form
//    of the Wigner 3j symbol, the complex Gaunt integral
//      int Y_l1^m1 Y_l2^m2 Y_l3^m3 = sqrt((2l1+1)(2l2+1)(2l3+1)/4pi) (l1 l2 l3; 0 0 0)(l1 l2 l3; m1 m2 m3),
//    and the unitary change to real harmonics.
//  * ACE coefficient tensors: the basis table's coefficients placed at the sorted
//    (n, l) position of each product.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "ap_internal.h"
#include "eam_table.h"

namespace ap {

namespace {

// sum_i a_i (d_i - r)^3 over the knots with d_i >= b, expanded in t = r - mid
void cubic_expand(const double* amp, const double* d, int n, double b, double mid, double* c) {
    for (int k = 0; k < 6; ++k) c[k] = 0.0;
    for (int i = 0; i < n; ++i) {
        if (d[i] < b) continue;
        double e = d[i] - mid;
        c[0] += amp[i] * e * e * e;
        c[1] += -3.0 * amp[i] * e * e;
        c[2] += 3.0 * amp[i] * e;
        c[3] += -amp[i];
    }
}

double cubic_value(const double* amp, const double* d, int n, double r) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        double t = d[i] - r;
        if (t >= 0.0) s += amp[i] * t * t * t;
    }
    return s;
}

// The device forms t = r - mid in FP32.  With mid exactly representable in FP32 that
// difference is exact, so no pair in an interval sees a shifted expansion point (a shift
// shared by every pair of the interval would bias all densities and energies alike).
double fp32_exact(double v) { return (double)(float)v; }

// Intervals longer than kMaxPiece are split into equal pieces, each re-expanded about its
// own midpoint: over a long interval the FP32 Horner terms c_k t^k grow far beyond the value
// they sum to (a cubic over [0, 2.8] A evaluated at 2.5 A), and their rounding, not the
// function, sets the error of every pair energy and density.
constexpr double kMaxPiece = 0.25;

int pieces(double a, double b) { return std::max(1, (int)std::ceil((b - a) / kMaxPiece - 1e-9)); }

double piece_edge(double a, double b, int m, int j) { return j == m ? b : a + (b - a) * j / m; }

double binom(int m, int k) {
    double b = 1.0;
    for (int i = 1; i <= k; ++i) b = b * (m - k + i) / i;
    return b;
}

// One segment of the merged partition, in FP64: zeta cubic, Phi cubic / quintic / ZBL.
struct Seg {
    double a, b, mid;
    double z[4];
    double f[6];
    int kind;
};

int check_knots(const double* amp, const double* d, int n, int nmax, double& rcut, std::string& err) {
    (void)amp;
    if (n < 1 || n > nmax) { err = "EAM: bad number of knots"; return AP_ERR_ARG; }
    rcut = 0.0;
    for (int i = 0; i < n; ++i) rcut = std::max(rcut, d[i]);
    if (!(rcut > 0.0) || rcut > 20.0) { err = "EAM: knot radii must lie in (0, 20] Angstrom"; return AP_ERR_ARG; }
    return AP_OK;
}

// The merged partition of [0, rc): breakpoints of both functions, pieces of <= kMaxPiece.
int build_segments(const ap_potential& p, std::vector<Seg>& out, double& rc_rho, double& rc_phi, std::string& err) {
    out.clear();
    int s;
    if ((s = check_knots(p.eam_phi_a, p.eam_phi_d, p.eam_n_phi, 32, rc_phi, err))) return s;
    if ((s = check_knots(p.eam_rho_a, p.eam_rho_d, p.eam_n_rho, 16, rc_rho, err))) return s;
    const double rc = std::max(rc_phi, rc_rho);
    std::vector<double> br = {0.0, rc_rho, rc_phi};
    for (int i = 0; i < p.eam_n_phi; ++i) br.push_back(p.eam_phi_d[i]);
    for (int i = 0; i < p.eam_n_rho; ++i) br.push_back(p.eam_rho_d[i]);
    if (p.eam_zbl) {
        if (!(p.eam_r_lo > 0.0 && p.eam_r_hi > p.eam_r_lo && p.eam_r_hi < rc_phi)) { err = "EAM: bad r_lo/r_hi"; return AP_ERR_ARG; }
        br.push_back(p.eam_r_lo);
        br.push_back(p.eam_r_hi);
    }
    const double clamp = p.eam_rho_rclamp;
    if (clamp > 0.0) {
        if (clamp >= rc_rho) { err = "EAM: r_cut^rho beyond the density cutoff"; return AP_ERR_ARG; }
        br.push_back(clamp);
    }
    std::sort(br.begin(), br.end());
    br.erase(std::unique(br.begin(), br.end()), br.end());
    const double zclamp = clamp > 0.0 ? cubic_value(p.eam_rho_a, p.eam_rho_d, p.eam_n_rho, clamp) : 0.0;
    for (size_t k = 0; k + 1 < br.size() && br[k] < rc; ++k) {
        const int m = pieces(br[k], br[k + 1]);
        for (int j = 0; j < m; ++j) {
            Seg g{};
            g.a = piece_edge(br[k], br[k + 1], m, j);
            g.b = piece_edge(br[k], br[k + 1], m, j + 1);
            g.mid = fp32_exact(0.5 * (g.a + g.b));
            if (clamp > 0.0 && g.b <= clamp) g.z[0] = zclamp;
            else if (g.a < rc_rho) {
                double c[6];
                cubic_expand(p.eam_rho_a, p.eam_rho_d, p.eam_n_rho, g.b, g.mid, c);
                for (int q = 0; q < 4; ++q) g.z[q] = c[q];
            }
            if (p.eam_zbl && g.b <= p.eam_r_lo) {
                g.kind = kSegZbl;
            } else if (p.eam_zbl && g.b <= p.eam_r_hi) {
                g.kind = kSegQuintic;
                for (int q = 0; q <= 5; ++q)
                    for (int e = q; e <= 5; ++e) g.f[q] += p.eam_b[e] * binom(e, q) * std::pow(g.mid, e - q);
            } else if (g.a < rc_phi) {
                cubic_expand(p.eam_phi_a, p.eam_phi_d, p.eam_n_phi, g.b, g.mid, g.f);
            }
            out.push_back(g);
        }
    }
    if ((int)out.size() > kMaxSeg) { err = "EAM: too many table segments"; return AP_ERR_ARG; }
    return AP_OK;
}

double fact(int n) {
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
}

double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
    if (m1 + m2 + m3 != 0) return 0.0;
    if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
    if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
    double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
    double pre = std::sqrt(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) *
                           fact(j3 + m3) * fact(j3 - m3));
    int kmin = std::max(0, std::max(j2 - j3 - m1, j1 - j3 + m2));
    int kmax = std::min(j1 + j2 - j3, std::min(j1 - m1, j2 + m2));
    double s = 0.0;
    for (int k = kmin; k <= kmax; ++k) {
        double den = fact(k) * fact(j3 - j2 + k + m1) * fact(j3 - j1 + k - m2) * fact(j1 + j2 - j3 - k) *
                     fact(j1 - k - m1) * fact(j2 - k + m2);
        s += ((k & 1) ? -1.0 : 1.0) / den;
    }
    int ph = j1 - j2 - m3;
    return ((ph % 2 != 0) ? -1.0 : 1.0) * pre * s;
}

double gaunt_complex(int l1, int m1, int l2, int m2, int l3, int m3) {
    const double pi = 3.14159265358979323846;
    return std::sqrt((2.0 * l1 + 1) * (2.0 * l2 + 1) * (2.0 * l3 + 1) / (4.0 * pi)) *
           wigner3j(l1, l2, l3, 0, 0, 0) * wigner3j(l1, l2, l3, m1, m2, m3);
}

// U[m][m'] with Y_real(l, m) = sum_m' U[m][m'] Y_complex(l, m') (Condon-Shortley complex Y)
std::complex<double> ucr(int m, int mp) {
    const double s = 1.0 / std::sqrt(2.0);
    const double sg = (std::abs(m) % 2) ? -1.0 : 1.0;
    if (m == 0) return mp == 0 ? 1.0 : 0.0;
    if (m > 0) {
        if (mp == -m) return s;
        if (mp == m) return sg * s;
        return 0.0;
    }
    if (mp == m) return std::complex<double>(0.0, s);
    if (mp == -m) return std::complex<double>(0.0, -sg * s);
    return 0.0;
}

}  // namespace

double gaunt_real_racah(int l1, int m1, int l2, int m2, int l3, int m3) {
    std::complex<double> g = 0.0;
    for (int a = -l1; a <= l1; ++a) {
        std::complex<double> u1 = ucr(m1, a);
        if (u1 == 0.0) continue;
        for (int b = -l2; b <= l2; ++b) {
            std::complex<double> u2 = ucr(m2, b);
            if (u2 == 0.0) continue;
            int c = -a - b;
            if (c < -l3 || c > l3) continue;
            std::complex<double> u3 = ucr(m3, c);
            if (u3 == 0.0) continue;
            g += u1 * u2 * u3 * gaunt_complex(l1, a, l2, b, l3, c);
        }
    }
    return g.real();
}

int gaunt_values(float* out, std::string& err) {
    int e = 0;
    for (int t = 0; t < kNT; ++t) {
        // in the kernel's order of the factors (the pattern the kernel compiles)
        int l1 = ktri_l(t, 0), l2 = ktri_l(t, 1), l3 = ktri_l(t, 2);
        for (int m1 = -l1; m1 <= l1; ++m1)
            for (int m2 = -l2; m2 <= l2; ++m2)
                for (int m3 = -l3; m3 <= l3; ++m3) {
                    double g = gaunt_real_racah(l1, m1, l2, m2, l3, m3);
                    if (gaunt_allowed(m1, m2, m3)) {
                        out[e++] = (float)g;
                    } else if (std::fabs(g) > 1e-12) {
                        err = "Gaunt coefficient outside the compile-time pattern";
                        return AP_ERR_ARG;
                    }
                }
    }
    if (e != kNG) { err = "Gaunt pattern size mismatch"; return AP_ERR_ARG; }
    return AP_OK;
}

int build_eam_tables(const ap_potential& p, EamDev& out, std::string& err) {
    std::memset(&out, 0, sizeof(out));
    std::vector<Seg> sg;
    double rc_rho = 0.0, rc_phi = 0.0;
    int s = build_segments(p, sg, rc_rho, rc_phi, err);
    if (s) return s;
    if (p.eam_zbl) {
        if (!(p.eam_zbl_eps0 > 0.0 && p.eam_zbl_a > 0.0)) { err = "EAM: bad ZBL parameters"; return AP_ERR_ARG; }
        out.zbl_k = (float)(p.eam_zbl_Z * p.eam_zbl_Z / (4.0 * 3.14159265358979323846 * p.eam_zbl_eps0));
        out.zbl_ainv = (float)(1.0 / p.eam_zbl_a);
    }
    const double rc = std::max(rc_rho, rc_phi);
    out.nseg = (int)sg.size();
    out.rc_rho = (float)rc_rho;
    out.rc_phi = (float)rc_phi;
    out.rc = (float)rc;
    out.bin_inv = (float)(kNBin / rc);
    for (int k = 0; k < out.nseg; ++k) {
        const Seg& g = sg[k];
        EamSeg& e = out.seg[k];
        const float z0 = (float)g.z[0], f0 = (float)g.f[0];
        e.q0 = make_float4((float)g.mid, (float)g.z[1], (float)g.z[2], (float)g.z[3]);
        e.q1 = make_float4((float)g.f[1], (float)g.f[2], (float)g.f[3], f0);
        e.q2 = make_float4(z0, (float)(g.z[0] - (double)z0), (float)(g.f[0] - (double)f0), (float)g.kind);
        e.q3 = make_float4((float)g.f[4], (float)g.f[5], 0.0f, 0.0f);
    }
    // bin b holds every FP32 r with (int)(r * bin_inv) == b; its range is widened by 1 % on
    // both sides so that rounding of that product cannot land r outside the record
    const double binw = rc / kNBin;
    for (int b = 0; b < kNBin; ++b) {
        const double lo = std::max(0.0, (b - 0.01) * binw), hi = (b + 1.01) * binw;
        int k = 0;
        while (k + 1 < out.nseg && sg[k + 1].a <= lo) ++k;
        EamBin& e = out.bin[b];
        e.k = k;
        e.s1 = e.s2 = INFINITY;
        e.special = sg[k].kind != kSegCubic;
        if (k + 1 < out.nseg && sg[k + 1].a < hi) {
            e.s1 = (float)sg[k + 1].a;
            e.special |= sg[k + 1].kind != kSegCubic;
            if (k + 2 < out.nseg && sg[k + 2].a < hi) {
                e.s2 = (float)sg[k + 2].a;
                e.special |= sg[k + 2].kind != kSegCubic;
                if (k + 3 < out.nseg && sg[k + 3].a < hi) { err = "EAM: more than two knots in one table bin"; return AP_ERR_ARG; }
            }
        }
    }
    // The device compares r >= (float)start.  Where a start is not an FP32 number the boundary
    // moves by less than one ulp; the adjacent pieces join with continuous value and first
    // derivative (knots of the cubic sums, the bridge joins, the piece splits), so either
    // piece is correct there to rounding.
    out.F_a1 = p.eam_F_a1;
    out.F_a2 = p.eam_F_a2;
    out.F_dxi = p.eam_F_dxi;
    return AP_OK;
}

int eam_table_eval(const ap_potential& p, int which, double r, double* f, double* df) {
    *f = 0.0;
    *df = 0.0;
    std::string err;
    if (which >= 2) {
        EamDev T;
        int s = build_eam_tables(p, T, err);
        if (s) return s;
        const float rf = (float)r;
        if (!(rf < (which == 2 ? T.rc_phi : T.rc_rho)) || rf < 0.0f) return AP_OK;
        float dz, dp, pf;
        eam_pair_der<true>(T, rf, dz, dp, pf);
        if (which == 2) { *f = pf; *df = dp; }
        else { *f = eam_zeta(T, rf); *df = dz; }
        return AP_OK;
    }
    std::vector<Seg> sg;
    double rc_rho = 0.0, rc_phi = 0.0;
    int s = build_segments(p, sg, rc_rho, rc_phi, err);
    if (s) return s;
    if (r < 0.0 || r >= (which == 0 ? rc_phi : rc_rho)) return AP_OK;
    size_t k = 0;
    while (k + 1 < sg.size() && r >= sg[k + 1].a) ++k;
    const Seg& g = sg[k];
    if (which == 0 && g.kind == kSegZbl) {
        const double c[4] = {0.1818, 0.5099, 0.2802, 0.02817};
        const double e[4] = {3.2, 0.9423, 0.4029, 0.2016};
        double kz = p.eam_zbl_Z * p.eam_zbl_Z / (4.0 * 3.14159265358979323846 * p.eam_zbl_eps0);
        double x = r / p.eam_zbl_a, ph = 0.0, dph = 0.0;
        for (int i = 0; i < 4; ++i) { double t = c[i] * std::exp(-e[i] * x); ph += t; dph -= e[i] * t; }
        *f = kz * ph / r;
        *df = kz * (dph / p.eam_zbl_a / r - ph / (r * r));
        return AP_OK;
    }
    const double* c = which == 0 ? g.f : g.z;
    const int deg = which == 0 ? 5 : 3;
    double t = r - g.mid, v = 0.0, dv = 0.0;
    for (int q = deg; q >= 0; --q) v = v * t + c[q];
    for (int q = deg; q >= 1; --q) dv = dv * t + q * c[q];
    *f = v;
    *df = dv;
    return AP_OK;
}

int build_ace_tables(const ap_potential& p, AceDev& out, std::string& err) {
    // l-triple index of sorted (l1, l2, l3), -1 where none (a lookup: a context build visits
    // every three-factor function twice)
    static const auto tri_lut = [] {
        std::array<std::array<std::array<int, kLmax + 1>, kLmax + 1>, kLmax + 1> lut{};
        for (int a = 0; a <= kLmax; ++a)
            for (int b = 0; b <= kLmax; ++b)
                for (int c = 0; c <= kLmax; ++c) lut[a][b][c] = tri_index(a, b, c);
        return lut;
    }();
    std::memset(&out, 0, sizeof(out));
    if (p.ace_nmax != kNmax || p.ace_lmax != kLmax) { err = "ACE: only n_max = 8, l_max = 4 are built"; return AP_ERR_ARG; }
    if (!(p.ace_rc > 0.0) || !(p.ace_nref > 0.0)) { err = "ACE: rc and nref must be positive"; return AP_ERR_ARG; }
    if (p.ace_nfunc < 0 || (p.ace_nfunc > 0 && (!p.ace_idx || !p.ace_c1 || !p.ace_c2))) { err = "ACE: missing basis arrays"; return AP_ERR_ARG; }
    for (int v = 0; v < p.ace_nfunc; ++v) {
        const int* q = p.ace_idx + 7 * v;
        int nu = q[0];
        int nn[3] = {q[1], q[3], q[5]}, ll[3] = {q[2], q[4], q[6]};
        for (int k = 0; k < nu && k < 3; ++k)
            if (nn[k] < 0 || nn[k] >= kNmax || ll[k] < 0 || ll[k] > kLmax) { err = "ACE: basis index out of range"; return AP_ERR_ARG; }
        for (int d = 0; d < 2; ++d) {
            double c = d == 0 ? p.ace_c1[v] : p.ace_c2[v];
            if (nu == 1) {
                if (ll[0] != 0) { err = "ACE: one-factor functions need l = 0"; return AP_ERR_ARG; }
                out.c1[d][nn[0]] += (float)c;
            } else if (nu == 2) {
                if (ll[0] != ll[1]) { err = "ACE: two-factor functions need l1 = l2"; return AP_ERR_ARG; }
                int a = std::min(nn[0], nn[1]), b = std::max(nn[0], nn[1]);
                out.c2[d][ll[0]][a * 8 + b] += (float)c;
            } else if (nu == 3) {
                int key[3][2];
                for (int k = 0; k < 3; ++k) { key[k][0] = ll[k]; key[k][1] = nn[k]; }
                // sort the three factors by (l, n)
                for (int i = 0; i < 3; ++i)
                    for (int j = i + 1; j < 3; ++j)
                        if (key[j][0] < key[i][0] || (key[j][0] == key[i][0] && key[j][1] < key[i][1]))
                            for (int z = 0; z < 2; ++z) std::swap(key[i][z], key[j][z]);
                int t = tri_lut[key[0][0]][key[1][0]][key[2][0]];
                if (t < 0) {
                    int l1 = key[0][0], l2 = key[1][0], l3 = key[2][0];
                    bool zero = ((l1 + l2 + l3) & 1) || l3 > l1 + l2 || l3 < std::abs(l1 - l2);
                    if (zero) continue;      // the function vanishes identically
                    err = "ACE: unsupported l-triple";
                    return AP_ERR_ARG;
                }
                out.c3[d][t][key[2][1]][key[0][1] * 8 + key[1][1]] += (float)c;
            } else {
                err = "ACE: only nu = 1, 2, 3 (body order <= 4) are built";
                return AP_ERR_ARG;
            }
        }
    }
    out.c1_0 = (float)p.ace_c1_0;
    out.c2_0 = (float)p.ace_c2_0;
    out.nref_inv = (float)(1.0 / p.ace_nref);
    out.rc = (float)p.ace_rc;
    return AP_OK;
}

// FP32 -> TF32 rounding to nearest, ties away from zero (the rule of cvt.rna.tf32.f32): the
// result keeps 10 explicit mantissa bits, the 13 low bits are zero
static float tf32_rna(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

void build_ace_tc(const AceDev& in, AceTc& out) {
    std::memset(&out, 0, sizeof(out));
    for (int d = 0; d < 2; ++d) {
        for (int l = 0; l <= kLmax; ++l) {
            // triple t = l is (0, l, l): G = delta_{m2 m3} G_l
            const float g = (float)gaunt_real_racah(0, 0, l, 0, l, 0);
            for (int n1 = 0; n1 < kNmax; ++n1)
                for (int n2 = 0; n2 < kNmax; ++n2)
                    for (int n3 = 0; n3 < kNmax; ++n3)
                        out.c0ll[d][l][n1 / 4][c0ll_pos(n2 * 8 + n3)][n1 % 4] = g * in.c3[d][l][n3][n1 * 8 + n2];
        }
        for (int u = 0; u < kNT3; ++u) {
            const int t = kTcTriple0 + u;
            const bool sym = ktri_l(t, 0) == ktri_l(t, 1);
            const bool sym3 = sym && ktri_l(t, 1) == ktri_l(t, 2);
            // coefficient of the kernel's factors (n1, n2, n3); the factor order of the basis
            // is (tri_l(t, 0), tri_l(t, 1), tri_l(t, 2)) and kernel factor k is basis factor
            // kern_perm(t, k)
            auto coef = [&](int n1, int n2, int n3) {
                int nb[3];
                nb[kern_perm(t, 0)] = n1;
                nb[kern_perm(t, 1)] = n2;
                nb[kern_perm(t, 2)] = n3;
                return in.c3[d][t][nb[2]][nb[0] * 8 + nb[1]];
            };
            for (int n3 = 0; n3 < kNmax; ++n3)
                for (int n1 = 0; n1 < kNmax; ++n1)
                    for (int n2 = 0; n2 < kNmax; ++n2) {
                        if (sym && n1 > n2) continue;
                        // the product of the first two factors is symmetric in (n1, n2) when
                        // l1 = l2: the packed row of the pair n1 <= n2 holds the mean of both
                        // orders' coefficients (the kernel doubles the product of n1 < n2)
                        const int q = sym ? sym_pair(n1, n2) : n1 * 8 + n2;
                        float v = coef(n1, n2, n3);
                        if (sym3) {
                            // all three factors have equal l: the coefficient of the sorted
                            // (n1, n2, n3) spread evenly over its distinct orderings, so that the
                            // coefficients are symmetric in all three indices
                            int a = n1, b = n2, c = n3;
                            if (a > b) std::swap(a, b);
                            if (b > c) std::swap(b, c);
                            if (a > b) std::swap(a, b);
                            const int mult = (a == b && b == c) ? 1 : (a == b || b == c) ? 3 : 6;
                            v = coef(a, b, c) / (float)mult;
                        } else if (sym && n1 != n2) {
                            v = 0.5f * (coef(n1, n2, n3) + coef(n2, n1, n3));
                        }
                        const float hi = tf32_rna(v), lo = tf32_rna(v - hi);
                        const int pos = n3 ^ (4 * ((q >> 2) & 1));
                        out.c3[0][d][u][q][pos] = hi;
                        out.c3[1][d][u][q][pos] = lo;
                    }
        }
    }
    std::memcpy(out.c2, in.c2, sizeof(out.c2));
    std::memcpy(out.c1, in.c1, sizeof(out.c1));
    out.c1_0 = in.c1_0;
    out.c2_0 = in.c2_0;
    out.nref_inv = in.nref_inv;
    out.rc = in.rc;
}

}  // namespace ap
