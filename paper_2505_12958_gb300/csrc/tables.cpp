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
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "ap_internal.h"

namespace ap {

namespace {

struct Interval {
    double a, b, mid;
    double c[6];
    int zbl;
};

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

int build_intervals(const ap_potential& p, int which, std::vector<Interval>& out, double& rcut, std::string& err) {
    out.clear();
    const double* amp = which == 0 ? p.eam_phi_a : p.eam_rho_a;
    const double* d = which == 0 ? p.eam_phi_d : p.eam_rho_d;
    int n = which == 0 ? p.eam_n_phi : p.eam_n_rho;
    if (n < 1 || n > (which == 0 ? 32 : 16)) { err = "EAM: bad number of knots"; return AP_ERR_ARG; }
    rcut = 0.0;
    for (int i = 0; i < n; ++i) rcut = std::max(rcut, d[i]);
    if (!(rcut > 0.0) || rcut > 20.0) { err = "EAM: knot radii must lie in (0, 20] Angstrom"; return AP_ERR_ARG; }
    double r0 = 0.0;
    if (which == 0 && p.eam_zbl) {
        if (!(p.eam_r_lo > 0.0 && p.eam_r_hi > p.eam_r_lo && p.eam_r_hi < rcut)) { err = "EAM: bad r_lo/r_hi"; return AP_ERR_ARG; }
        Interval z{};
        z.a = 0.0; z.b = p.eam_r_lo; z.mid = 0.5 * z.b; z.zbl = 1;
        out.push_back(z);
        const int m_pieces = pieces(p.eam_r_lo, p.eam_r_hi);
        for (int j = 0; j < m_pieces; ++j) {
            Interval q{};
            q.a = piece_edge(p.eam_r_lo, p.eam_r_hi, m_pieces, j);
            q.b = piece_edge(p.eam_r_lo, p.eam_r_hi, m_pieces, j + 1);
            q.mid = fp32_exact(0.5 * (q.a + q.b));
            for (int k = 0; k <= 5; ++k)
                for (int m = k; m <= 5; ++m) q.c[k] += p.eam_b[m] * binom(m, k) * std::pow(q.mid, m - k);
            out.push_back(q);
        }
        r0 = p.eam_r_hi;
    }
    if (which == 1 && p.eam_rho_rclamp > 0.0) {
        if (p.eam_rho_rclamp >= rcut) { err = "EAM: r_cut^rho beyond the density cutoff"; return AP_ERR_ARG; }
        Interval q{};
        q.a = 0.0; q.b = p.eam_rho_rclamp; q.mid = 0.5 * q.b;
        q.c[0] = cubic_value(amp, d, n, p.eam_rho_rclamp);
        out.push_back(q);
        r0 = p.eam_rho_rclamp;
    }
    std::vector<double> br;
    br.push_back(r0);
    std::vector<double> ks(d, d + n);
    std::sort(ks.begin(), ks.end());
    for (double k : ks)
        if (k > r0 && k > br.back()) br.push_back(k);
    for (size_t k = 0; k + 1 < br.size(); ++k) {
        const int m_pieces = pieces(br[k], br[k + 1]);
        for (int j = 0; j < m_pieces; ++j) {
            Interval q{};
            q.a = piece_edge(br[k], br[k + 1], m_pieces, j);
            q.b = piece_edge(br[k], br[k + 1], m_pieces, j + 1);
            q.mid = fp32_exact(0.5 * (q.a + q.b));
            cubic_expand(amp, d, n, br[k + 1], q.mid, q.c);
            out.push_back(q);
        }
    }
    if ((int)out.size() > kMaxInt) { err = "EAM: too many intervals"; return AP_ERR_ARG; }
    return AP_OK;
}

void fill_tab(const std::vector<Interval>& iv, double rcut, PolyTab& t) {
    std::memset(&t, 0, sizeof(t));
    t.nint = (int)iv.size();
    t.zbl = iv.size() && iv[0].zbl ? 1 : 0;
    t.rcut = (float)rcut;
    t.bin_inv = (float)(kNBin / rcut);
    for (int k = 0; k < t.nint; ++k) {
        t.start[k] = (float)iv[k].a;
        t.mid[k] = (float)iv[k].mid;
        for (int c = 0; c < 6; ++c) t.c[k][c] = (float)iv[k].c[c];
        t.c0lo[k] = (float)(iv[k].c[0] - (double)t.c[k][0]);
    }
    t.start[t.nint] = (float)rcut;
    for (int b = 0; b < kNBin; ++b) {
        float r = (float)b / t.bin_inv;
        int k = 0;
        while (k + 1 < t.nint && r >= t.start[k + 1]) ++k;
        t.bin[b] = (unsigned char)k;
    }
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
        int l1 = tri_l(t, 0), l2 = tri_l(t, 1), l3 = tri_l(t, 2);
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
    std::vector<Interval> iv;
    double rc_phi = 0.0, rc_rho = 0.0;
    int s = build_intervals(p, 0, iv, rc_phi, err);
    if (s) return s;
    fill_tab(iv, rc_phi, out.phi);
    s = build_intervals(p, 1, iv, rc_rho, err);
    if (s) return s;
    fill_tab(iv, rc_rho, out.rho);
    if (p.eam_zbl) {
        if (!(p.eam_zbl_eps0 > 0.0 && p.eam_zbl_a > 0.0)) { err = "EAM: bad ZBL parameters"; return AP_ERR_ARG; }
        out.zbl_k = (float)(p.eam_zbl_Z * p.eam_zbl_Z / (4.0 * 3.14159265358979323846 * p.eam_zbl_eps0));
        out.zbl_ainv = (float)(1.0 / p.eam_zbl_a);
    }
    out.rc = (float)std::max(rc_phi, rc_rho);
    out.F_a1 = p.eam_F_a1;
    out.F_a2 = p.eam_F_a2;
    out.F_dxi = p.eam_F_dxi;
    return AP_OK;
}

int eam_table_eval_fp64(const ap_potential& p, int which, double r, double* f, double* df) {
    std::vector<Interval> iv;
    double rcut = 0.0;
    std::string err;
    int s = build_intervals(p, which, iv, rcut, err);
    if (s) return s;
    *f = 0.0; *df = 0.0;
    if (r >= rcut) return AP_OK;
    size_t k = 0;
    while (k + 1 < iv.size() && r >= iv[k + 1].a) ++k;
    if (iv[k].zbl) {
        const double c[4] = {0.1818, 0.5099, 0.2802, 0.02817};
        const double e[4] = {3.2, 0.9423, 0.4029, 0.2016};
        double kz = p.eam_zbl_Z * p.eam_zbl_Z / (4.0 * 3.14159265358979323846 * p.eam_zbl_eps0);
        double x = r / p.eam_zbl_a, ph = 0.0, dph = 0.0;
        for (int i = 0; i < 4; ++i) { double t = c[i] * std::exp(-e[i] * x); ph += t; dph -= e[i] * t; }
        *f = kz * ph / r;
        *df = kz * (dph / p.eam_zbl_a / r - ph / (r * r));
        return AP_OK;
    }
    double t = r - iv[k].mid, v = 0.0, dv = 0.0;
    for (int c = 5; c >= 0; --c) v = v * t + iv[k].c[c];
    for (int c = 5; c >= 1; --c) dv = dv * t + c * iv[k].c[c];
    *f = v; *df = dv;
    return AP_OK;
}

int build_ace_tables(const ap_potential& p, AceDev& out, std::string& err) {
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
                int t = tri_index(key[0][0], key[1][0], key[2][0]);
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

}  // namespace ap
