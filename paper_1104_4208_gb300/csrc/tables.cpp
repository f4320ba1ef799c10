// Reference-element tables of the Dubiner basis (host, FP64).
//
// The 3D Dubiner function of Sec. 4.2.2 is a product of univariate factors in
// the collapsed coordinates (xi, eta, zeta) of the reference tetrahedron,
//   x = xi, y = (1-xi) eta, z = (1-xi)(1-eta) zeta,
//   phi_ijk = (1-xi)^(i+j) (1-eta)^i L_i(2 zeta - 1) J_j^(2i+1,0)(2 eta - 1)
//             J_k^(2i+2j+2,0)(2 xi - 1),
// which is the tensor-product structure the method exploits (Sec. 3, item 1
// and 4 of the list of ingredients).  Derivatives of the univariate Jacobi
// factors use the identity d/dt P_n^(a,b) = (n+a+b+1)/2 P_{n-1}^(a+1,b+1); the
// Cartesian derivatives follow from the chain rule of the collapsed map.
// Integrals use tensor Gauss-Legendre rules in the collapsed coordinates with
// the Jacobian (1-xi)^2 (1-eta), exact for the polynomial integrands.
//
// Outputs are in the orthonormalised basis phi'_a = phi_a / ||phi_a|| (and
// psi'_g on faces), so that the lift operators are exact transposes of the
// trace operators and C_h, C_h^T share one rounded table.
//
// Host arithmetic is compiled with -ffp-contract=off so that the tables are
// bit-identical on x86-64 and aarch64.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dgm_internal.h"

namespace dgm {

void index3(int p, std::vector<int>& ijk) {
    ijk.clear();
    for (int i = 0; i <= p; ++i)
        for (int j = 0; j <= p - i; ++j)
            for (int k = 0; k <= p - i - j; ++k) {
                ijk.push_back(i);
                ijk.push_back(j);
                ijk.push_back(k);
            }
}

void index2(int p, std::vector<int>& ij) {
    ij.clear();
    for (int i = 0; i <= p; ++i)
        for (int j = 0; j <= p - i; ++j) {
            ij.push_back(i);
            ij.push_back(j);
        }
}

double dubiner3_norm2(int i, int j, int k) {
    return 1.0 / (2.0 * (2 * i + 1) * (i + j + 1) * (2 * i + 2 * j + 2 * k + 3));
}

double dubiner2_norm2(int i, int j) { return 1.0 / (2.0 * (2 * i + 1) * (i + j + 1)); }

namespace {

// Gauss-Legendre nodes/weights on [0,1] (Newton on P_n).
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double t = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = t; p0 = 1.0; }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = t; p0 = 1.0; }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
        }
        x[i] = 0.5 * (1.0 + t);
        w[i] = 1.0 / ((1.0 - t * t) * dp * dp);    // (2/((1-t^2) P'^2)) / 2
    }
}

// P_n^(a,b)(t) for n = 0..N.
void jacobi_all(int N, double a, double b, double t, double* out) {
    out[0] = 1.0;
    if (N == 0) return;
    out[1] = 0.5 * ((a + b + 2.0) * t + (a - b));
    for (int n = 1; n < N; ++n) {
        double c = 2.0 * n + a + b;
        double a1 = 2.0 * (n + 1) * (n + a + b + 1) * c;
        double a2 = (c + 1.0) * (a * a - b * b);
        double a3 = c * (c + 1.0) * (c + 2.0);
        double a4 = 2.0 * (n + a) * (n + b) * (c + 2.0);
        out[n + 1] = ((a2 + a3 * t) * out[n] - a4 * out[n - 1]) / a1;
    }
}

// P_n^(a,0)(t) and its derivative, n = 0..N.
void jacobi_d(int N, double a, double t, double* val, double* der) {
    jacobi_all(N, a, 0.0, t, val);
    std::vector<double> tmp(N + 1);
    der[0] = 0.0;
    if (N >= 1) {
        jacobi_all(N - 1, a + 1.0, 1.0, t, tmp.data());
        for (int n = 1; n <= N; ++n) der[n] = 0.5 * (n + a + 1.0) * tmp[n - 1];
    }
}

double ipow(double x, int n) {
    double r = 1.0;
    for (int i = 0; i < n; ++i) r *= x;
    return r;
}

// Values and Cartesian derivatives of all phi_ijk (|ijk| <= p) at the
// collapsed point (xi, eta, zeta) (interior: xi, eta < 1).
void phi3_at(int p, const std::vector<int>& idx, double xi, double eta, double zeta,
             double* val, double* dx, double* dy, double* dz) {
    const int N = (int)idx.size() / 3;
    std::vector<double> L(p + 1), Ld(p + 1), J(p + 1), Jd(p + 1), K(p + 1), Kd(p + 1);
    jacobi_d(p, 0.0, 2.0 * zeta - 1.0, L.data(), Ld.data());
    const double om_xi = 1.0 - xi, om_eta = 1.0 - eta;
    int lasti = -1, lastij = -1;
    for (int r = 0; r < N; ++r) {
        const int i = idx[3 * r], j = idx[3 * r + 1], k = idx[3 * r + 2];
        if (i != lasti) {
            jacobi_d(p - i, 2.0 * i + 1.0, 2.0 * eta - 1.0, J.data(), Jd.data());
            lasti = i;
            lastij = -1;
        }
        if (i + j != lastij) {
            jacobi_d(p - i - j, 2.0 * i + 2.0 * j + 2.0, 2.0 * xi - 1.0, K.data(), Kd.data());
            lastij = i + j;
        }
        const double A = L[i], Ad = 2.0 * Ld[i];
        const double B = ipow(om_eta, i) * J[j];
        const double Bd = (i > 0 ? -i * ipow(om_eta, i - 1) * J[j] : 0.0) + ipow(om_eta, i) * 2.0 * Jd[j];
        const double C = ipow(om_xi, i + j) * K[k];
        const double Cd = (i + j > 0 ? -(i + j) * ipow(om_xi, i + j - 1) * K[k] : 0.0)
                          + ipow(om_xi, i + j) * 2.0 * Kd[k];
        const double f = A * B * C;
        const double fxi = A * B * Cd, feta = A * Bd * C, fzeta = Ad * B * C;
        val[r] = f;
        if (dx) {
            dx[r] = fxi + eta / om_xi * feta + zeta / (om_xi * om_eta) * fzeta;
            dy[r] = feta / om_xi + zeta / (om_xi * om_eta) * fzeta;
            dz[r] = fzeta / (om_xi * om_eta);
        }
    }
}

// Values of phi_ijk at a Cartesian reference point (interior of a face or cell).
void phi3_cart(int p, const std::vector<int>& idx, const double* xh, double* val) {
    const double xi = xh[0];
    const double eta = xh[1] / (1.0 - xh[0]);
    const double zeta = xh[2] / (1.0 - xh[0] - xh[1]);
    phi3_at(p, idx, xi, eta, zeta, val, nullptr, nullptr, nullptr);
}

// psi_ij (Eq. (4)) at the collapsed face point (a, b): s = a, u = (1-a) b.
void psi2_at(int p, const std::vector<int>& idx, double a, double b, double* val) {
    const int N = (int)idx.size() / 2;
    std::vector<double> L(p + 1), Ld(p + 1), J(p + 1), Jd(p + 1);
    jacobi_d(p, 0.0, 2.0 * b - 1.0, L.data(), Ld.data());
    int lasti = -1;
    for (int r = 0; r < N; ++r) {
        const int i = idx[2 * r], j = idx[2 * r + 1];
        if (i != lasti) {
            jacobi_d(p - i, 2.0 * i + 1.0, 2.0 * a - 1.0, J.data(), Jd.data());
            lasti = i;
        }
        val[r] = L[i] * ipow(1.0 - a, i) * J[j];
    }
}

const double kVert[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

// Face traces T[g][a] = int psi'_g(s,u) phi'_a(face point) ds du of the
// orthonormal bases, built sum-factorised (Sec. 3.2.3, Sec. 4.2.2).
// On each reference face the restriction of phi_ijk factors in the face's
// collapsed coordinates (s, b = u / (1 - s)):
//   face 1 (x = 0):  (-1)^k psi_ij                                   (diagonal)
//   face 2 (y = 0):  (-1)^j P_i(2b-1) (1-s)^i [(1-s)^j P_k^(2i+2j+2,0)(2s-1)]
//   face 3 (z = 0):  (-1)^i [(1-b)^i P_j^(2i+1,0)(2b-1)] (1-s)^(i+j) P_k^(2i+2j+2,0)(2s-1)
//   face 0 (x+y+z = 1): the face-3 form without the sign, in the face's rotated
//     parametrisation (s~, u~) = (1 - s - u, s); a dense rotation block, the same
//     for every element and block diagonal in the face degree, maps it back.
// The brackets are expanded by 1D connection coefficients: in b against the
// Legendre P_m(2b-1) (weight 1), in s against P_n^(2m+1,0)(2s-1) (weight
// (1-s)^(2m+1)), each an exact Gauss-Legendre sum of a polynomial.

// int_0^1 w(s) p(s) q(s) ds for polynomials, by nq-point Gauss-Legendre
struct Line {
    std::vector<double> x, w;
    explicit Line(int nq) { gauss_legendre01(nq, x, w); }
};

// c_n = <g, P_n^(a,0)(2s-1)>_(1-s)^a / <P_n, P_n>_(1-s)^a, n = 0..nmax, for g given
// at the line's nodes
void jacobi_coeffs(const Line& L, double a, const std::vector<double>& g, int nmax, double* c) {
    std::vector<double> P(nmax + 1);
    std::vector<double> num(nmax + 1, 0.0), den(nmax + 1, 0.0);
    for (size_t q = 0; q < L.x.size(); ++q) {
        jacobi_all(nmax, a, 0.0, 2.0 * L.x[q] - 1.0, P.data());
        const double wq = L.w[q] * std::pow(1.0 - L.x[q], a);
        for (int n = 0; n <= nmax; ++n) {
            num[n] += wq * g[q] * P[n];
            den[n] += wq * P[n] * P[n];
        }
    }
    for (int n = 0; n <= nmax; ++n) c[n] = num[n] / den[n];
}

// unnormalised face-3 form (without sign) of phi_ijk: coefficients q[(m,n)] on psi_mn
void face3_form(int p, int i, int j, int k, const Line& L, const std::vector<int>& pos2, std::vector<double>& q) {
    const int N2 = (p + 1) * (p + 2) / 2;
    q.assign(N2, 0.0);
    const int nq = (int)L.x.size();
    std::vector<double> g(nq), P(p + 1), d(i + j + 1), e(p + 1);
    // (1-b)^i P_j^(2i+1,0)(2b-1) in Legendre P_m(2b-1)
    for (int r = 0; r < nq; ++r) {
        jacobi_all(j, 2.0 * i + 1.0, 0.0, 2.0 * L.x[r] - 1.0, P.data());
        g[r] = ipow(1.0 - L.x[r], i) * P[j];
    }
    jacobi_coeffs(L, 0.0, g, i + j, d.data());
    for (int m = 0; m <= i + j; ++m) {
        if (d[m] == 0.0) continue;
        // (1-s)^(i+j-m) P_k^(2i+2j+2,0)(2s-1) in P_n^(2m+1,0)(2s-1)
        for (int r = 0; r < nq; ++r) {
            jacobi_all(k, 2.0 * i + 2.0 * j + 2.0, 0.0, 2.0 * L.x[r] - 1.0, P.data());
            g[r] = ipow(1.0 - L.x[r], i + j - m) * P[k];
        }
        const int nmax = i + j - m + k;
        jacobi_coeffs(L, 2.0 * m + 1.0, g, nmax, e.data());
        for (int n = 0; n <= nmax; ++n) q[pos2[m * (p + 1) + n]] += d[m] * e[n];
    }
}

void face_trace_sf(int p, int f, std::vector<double>& T) {
    std::vector<int> i3, i2;
    index3(p, i3);
    index2(p, i2);
    const int N3 = (int)i3.size() / 3, N2 = (int)i2.size() / 2;
    std::vector<int> pos2((p + 1) * (p + 1), -1);
    for (int g = 0; g < N2; ++g) pos2[i2[2 * g] * (p + 1) + i2[2 * g + 1]] = g;
    std::vector<double> n2(N2);
    for (int g = 0; g < N2; ++g) n2[g] = dubiner2_norm2(i2[2 * g], i2[2 * g + 1]);
    const Line L(2 * p + 4);
    // face 0: R[g][h] = int psi_g(s,u) psi_h(1-s-u, s) ds du / ||psi_g||^2
    std::vector<double> R;
    if (f == 0) {
        R.assign((size_t)N2 * N2, 0.0);
        const int nq = p + 2;
        std::vector<double> xa, wa;
        gauss_legendre01(nq, xa, wa);
        std::vector<double> pg(N2), ph(N2);
        for (int qa = 0; qa < nq; ++qa)
            for (int qb = 0; qb < nq; ++qb) {
                const double s = xa[qa], u = (1.0 - xa[qa]) * xa[qb];
                const double w = wa[qa] * wa[qb] * (1.0 - xa[qa]);
                psi2_at(p, i2, xa[qa], xa[qb], pg.data());
                const double st = 1.0 - s - u;
                psi2_at(p, i2, st, s / (1.0 - st), ph.data());
                for (int g = 0; g < N2; ++g)
                    for (int h = 0; h < N2; ++h) R[(size_t)g * N2 + h] += w * pg[g] * ph[h];
            }
        for (int g = 0; g < N2; ++g)
            for (int h = 0; h < N2; ++h) R[(size_t)g * N2 + h] /= n2[g];
    }
    T.assign((size_t)N2 * N3, 0.0);
    std::vector<double> q, e(p + 1);
    for (int a = 0; a < N3; ++a) {
        const int i = i3[3 * a], j = i3[3 * a + 1], k = i3[3 * a + 2];
        // c[g]: coefficient of psi_g in the restriction of phi_ijk
        std::vector<double> c(N2, 0.0);
        if (f == 1) {
            c[pos2[i * (p + 1) + j]] = (k % 2) ? -1.0 : 1.0;
        } else if (f == 2) {
            const int nq = (int)L.x.size();
            std::vector<double> g(nq), P(p + 1);
            for (int r = 0; r < nq; ++r) {
                jacobi_all(k, 2.0 * i + 2.0 * j + 2.0, 0.0, 2.0 * L.x[r] - 1.0, P.data());
                g[r] = ipow(1.0 - L.x[r], j) * P[k];
            }
            jacobi_coeffs(L, 2.0 * i + 1.0, g, j + k, e.data());
            const double sg = (j % 2) ? -1.0 : 1.0;
            for (int n = 0; n <= j + k; ++n) c[pos2[i * (p + 1) + n]] = sg * e[n];
        } else {
            face3_form(p, i, j, k, L, pos2, q);
            if (f == 3) {
                const double sg = (i % 2) ? -1.0 : 1.0;
                for (int g = 0; g < N2; ++g) c[g] = sg * q[g];
            } else {
                for (int g = 0; g < N2; ++g) {
                    double acc = 0.0;
                    for (int h = 0; h < N2; ++h) acc += R[(size_t)g * N2 + h] * q[h];
                    c[g] = acc;
                }
            }
        }
        const double na = std::sqrt(dubiner3_norm2(i, j, k));
        // orthonormal table: (int psi_g phi_a) / (||psi_g|| ||phi_a||) = c_g ||psi_g|| / ||phi_a||
        for (int g = 0; g < N2; ++g) T[(size_t)g * N3 + a] = c[g] * std::sqrt(n2[g]) / na;
    }
}

}  // namespace

void collapsed_rule(int q1d, std::vector<double>& xh, std::vector<double>& w, std::vector<double>& col) {
    std::vector<double> g, gw;
    gauss_legendre01(q1d, g, gw);
    const int nq = q1d * q1d * q1d;
    xh.resize(3 * nq);
    w.resize(nq);
    col.resize(3 * nq);
    int q = 0;
    for (int a = 0; a < q1d; ++a)
        for (int b = 0; b < q1d; ++b)
            for (int c = 0; c < q1d; ++c, ++q) {
                const double xi = g[a], eta = g[b], zeta = g[c];
                xh[3 * q] = xi;
                xh[3 * q + 1] = (1.0 - xi) * eta;
                xh[3 * q + 2] = (1.0 - xi) * (1.0 - eta) * zeta;
                w[q] = gw[a] * gw[b] * gw[c] * (1.0 - xi) * (1.0 - xi) * (1.0 - eta);
                col[3 * q] = xi;
                col[3 * q + 1] = eta;
                col[3 * q + 2] = zeta;
            }
}

void phi_table(int p, int q1d, std::vector<double>& phi) {
    std::vector<double> xh, w, col;
    collapsed_rule(q1d, xh, w, col);
    std::vector<int> idx;
    index3(p, idx);
    const int N = (int)idx.size() / 3, nq = (int)w.size();
    phi.resize((size_t)nq * N);
    for (int q = 0; q < nq; ++q) {
        phi3_at(p, idx, col[3 * q], col[3 * q + 1], col[3 * q + 2], &phi[(size_t)q * N], nullptr, nullptr, nullptr);
        for (int a = 0; a < N; ++a)
            phi[(size_t)q * N + a] /= std::sqrt(dubiner3_norm2(idx[3 * a], idx[3 * a + 1], idx[3 * a + 2]));
    }
}

void phi_at_points(int p, const double* xh, int n, std::vector<double>& out) {
    std::vector<int> idx;
    index3(p, idx);
    const int N = (int)idx.size() / 3;
    out.assign((size_t)n * N, 0.0);
    for (int q = 0; q < n; ++q) {
        // keep the collapsed map away from its singular edges for points on faces/edges
        const double x = std::min(std::max(xh[3 * q], 0.0), 1.0 - 1e-13);
        const double y = std::min(std::max(xh[3 * q + 1], 0.0), 1.0 - x - 1e-13);
        const double z = std::min(std::max(xh[3 * q + 2], 0.0), 1.0 - x - y);
        const double eta = y / (1.0 - x), zeta = z / (1.0 - x - y);
        phi3_at(p, idx, x, eta, zeta, &out[(size_t)q * N], nullptr, nullptr, nullptr);
        for (int a = 0; a < N; ++a)
            out[(size_t)q * N + a] /= std::sqrt(dubiner3_norm2(idx[3 * a], idx[3 * a + 1], idx[3 * a + 2]));
    }
}

int build_ref_tables(int p, RefTables& t, bool equal_order) {
    if (p < 1 || p > DGM_PMAX) {
        set_error("p must be in [1, DGM_PMAX]");
        return DGM_ERR_INVALID_ARG;
    }
    // degree of H: p - 1 (V^{k+1} x V^k, Sec. 2) or p (the equal-order pair)
    const int ph = equal_order ? p : p - 1;
    std::vector<int> iE, iH, i2E, i2H;
    index3(p, iE);
    index3(ph, iH);
    index2(p, i2E);
    index2(ph, i2H);
    t.p = p;
    t.ph = ph;
    t.NE = (int)iE.size() / 3;
    t.NH = (int)iH.size() / 3;
    t.N2E = (int)i2E.size() / 2;
    t.N2H = (int)i2H.size() / 2;
    t.norm2E.resize(t.NE);
    for (int a = 0; a < t.NE; ++a) t.norm2E[a] = dubiner3_norm2(iE[3 * a], iE[3 * a + 1], iE[3 * a + 2]);

    // derivative tables: (d_d phi'_a, phi'_b), b over the basis of H's degree
    const int nq = p + 2;
    std::vector<double> gx, gw;
    gauss_legendre01(nq, gx, gw);
    for (int d = 0; d < 3; ++d) t.D[d].assign((size_t)t.NH * t.NE, 0.0);
    std::vector<double> v(t.NE), dx(t.NE), dy(t.NE), dz(t.NE), vh(t.NH);
    for (int a = 0; a < nq; ++a)
        for (int b = 0; b < nq; ++b)
            for (int c = 0; c < nq; ++c) {
                const double xi = gx[a], eta = gx[b], zeta = gx[c];
                const double w = gw[a] * gw[b] * gw[c] * (1.0 - xi) * (1.0 - xi) * (1.0 - eta);
                phi3_at(p, iE, xi, eta, zeta, v.data(), dx.data(), dy.data(), dz.data());
                phi3_at(ph, iH, xi, eta, zeta, vh.data(), nullptr, nullptr, nullptr);
                for (int bb = 0; bb < t.NH; ++bb) {
                    const double wb = w * vh[bb];
                    double* Dx = &t.D[0][(size_t)bb * t.NE];
                    double* Dy = &t.D[1][(size_t)bb * t.NE];
                    double* Dz = &t.D[2][(size_t)bb * t.NE];
                    for (int aa = 0; aa < t.NE; ++aa) {
                        Dx[aa] += wb * dx[aa];
                        Dy[aa] += wb * dy[aa];
                        Dz[aa] += wb * dz[aa];
                    }
                }
            }
    for (int bb = 0; bb < t.NH; ++bb) {
        const double nb = std::sqrt(dubiner3_norm2(iH[3 * bb], iH[3 * bb + 1], iH[3 * bb + 2]));
        for (int aa = 0; aa < t.NE; ++aa) {
            const double na = std::sqrt(t.norm2E[aa]);
            for (int d = 0; d < 3; ++d) t.D[d][(size_t)bb * t.NE + aa] /= (na * nb);
        }
    }
    // Exact zeros: d/dx_d phi_a has no component on phi_b for most pairs (the
    // sparsity the recurrences of Sec. 4.2.2 express); quadrature leaves such
    // entries at round-off level (below 1e-13 of the largest entry, against 5e-6 for
    // the smallest genuine entry at p = 8).  They are set to exactly zero, so that
    // sparse and dense applications of the tables are the same operator.
    {
        double mx = 0.0;
        for (int d = 0; d < 3; ++d)
            for (double x : t.D[d]) mx = std::max(mx, std::fabs(x));
        for (int d = 0; d < 3; ++d)
            for (double& x : t.D[d])
                if (std::fabs(x) < 1e-12 * mx) x = 0.0;
    }
    for (int f = 0; f < 4; ++f) {
        face_trace_sf(p, f, t.TrE[f]);
        face_trace_sf(ph, f, t.TrH[f]);
    }
    // face frames and reference orientation signs
    const double nhat[4][3] = {{1, 1, 1}, {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}};
    for (int f = 0; f < 4; ++f) {
        int v[3], c = 0;
        for (int q = 0; q < 4; ++q)
            if (q != f) v[c++] = q;
        for (int m = 0; m < 3; ++m) {
            t.that[f][0][m] = kVert[v[1]][m] - kVert[v[0]][m];
            t.that[f][1][m] = kVert[v[2]][m] - kVert[v[0]][m];
        }
        const double* a = t.that[f][0];
        const double* b = t.that[f][1];
        const double cr[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
        const double dot = cr[0] * nhat[f][0] + cr[1] * nhat[f][1] + cr[2] * nhat[f][2];
        t.sigma_hat[f] = dot > 0 ? 1.0 : -1.0;
    }
    t.pos2H.resize(t.N2H);
    for (int g = 0; g < t.N2H; ++g) {
        const int i = i2H[2 * g], j = i2H[2 * g + 1];
        int pos = -1;
        for (int q = 0; q < t.N2E; ++q)
            if (i2E[2 * q] == i && i2E[2 * q + 1] == j) pos = q;
        t.pos2H[g] = pos;
    }
    return DGM_OK;
}

void phi3_grad(int p, const std::vector<int>& idx, double xi, double eta, double zeta, double* val, double* grad) {
    const size_t n = idx.size() / 3;
    std::vector<double> dx(n), dy(n), dz(n);
    phi3_at(p, idx, xi, eta, zeta, val, dx.data(), dy.data(), dz.data());
    for (size_t r = 0; r < n; ++r) {
        grad[3 * r] = dx[r];
        grad[3 * r + 1] = dy[r];
        grad[3 * r + 2] = dz[r];
    }
}

namespace {

// psi_ij (Eq. (4)) and its Cartesian derivatives at the collapsed point (a, b):
// s = a, u = (1-a) b, psi = P_i(2b-1) (1-a)^i P_j^(2i+1,0)(2a-1);
// d/ds = d/da + b/(1-a) d/db, d/du = 1/(1-a) d/db.
void psi2_grad_at(int p, const std::vector<int>& idx, double a, double b, double* val, double* ds, double* du) {
    const int N = (int)idx.size() / 2;
    std::vector<double> L(p + 1), Ld(p + 1), J(p + 1), Jd(p + 1);
    jacobi_d(p, 0.0, 2.0 * b - 1.0, L.data(), Ld.data());
    const double om = 1.0 - a;
    int lasti = -1;
    for (int r = 0; r < N; ++r) {
        const int i = idx[2 * r], j = idx[2 * r + 1];
        if (i != lasti) {
            jacobi_d(p - i, 2.0 * i + 1.0, 2.0 * a - 1.0, J.data(), Jd.data());
            lasti = i;
        }
        const double A = L[i], Ab = 2.0 * Ld[i];
        const double B = ipow(om, i) * J[j];
        const double Ba = (i > 0 ? -i * ipow(om, i - 1) * J[j] : 0.0) + ipow(om, i) * 2.0 * Jd[j];
        val[r] = A * B;
        if (ds) {
            ds[r] = A * Ba + b / om * Ab * B;
            du[r] = Ab * B / om;
        }
    }
}

const double kVert2[3][2] = {{0, 0}, {1, 0}, {0, 1}};

// T[g][a] = int_0^1 psi'_a(edge f at s) L'_g(s) ds, g <= p
void edge_trace(int p, int f, std::vector<double>& T) {
    std::vector<int> i2;
    index2(p, i2);
    const int N = (int)i2.size() / 2, NG = p + 1;
    int v[2], c = 0;
    for (int q = 0; q < 3; ++q)
        if (q != f) v[c++] = q;
    std::vector<double> xs, ws;
    gauss_legendre01(p + 2, xs, ws);
    std::vector<double> psi(N), leg(NG);
    T.assign((size_t)NG * N, 0.0);
    for (size_t q = 0; q < xs.size(); ++q) {
        const double s = xs[q];
        const double x = kVert2[v[0]][0] + s * (kVert2[v[1]][0] - kVert2[v[0]][0]);
        const double y = kVert2[v[0]][1] + s * (kVert2[v[1]][1] - kVert2[v[0]][1]);
        // collapsed coordinates of (x, y); the vertex (1, 0) itself is never a Gauss point
        const double a = x, b = x < 1.0 ? y / (1.0 - x) : 0.0;
        psi2_at(p, i2, a, b, psi.data());
        jacobi_all(p, 0.0, 0.0, 2.0 * s - 1.0, leg.data());
        for (int g = 0; g < NG; ++g)
            for (int r = 0; r < N; ++r)
                T[(size_t)g * N + r] += ws[q] * std::sqrt(2.0 * g + 1.0) * leg[g] * psi[r];
    }
    for (int r = 0; r < N; ++r) {
        const double nr = std::sqrt(dubiner2_norm2(i2[2 * r], i2[2 * r + 1]));
        for (int g = 0; g < NG; ++g) T[(size_t)g * N + r] /= nr;
    }
}

}  // namespace

int build_ref_tables_2d(int p, RefTables2D& t) {
    if (p < 1 || p > DGM_PMAX) {
        set_error("p must be in [1, DGM_PMAX]");
        return DGM_ERR_INVALID_ARG;
    }
    std::vector<int> iE, iH;
    index2(p, iE);
    index2(p - 1, iH);
    t.p = p;
    t.NE = (int)iE.size() / 2;
    t.NH = (int)iH.size() / 2;
    t.norm2E.resize(t.NE);
    for (int a = 0; a < t.NE; ++a) t.norm2E[a] = dubiner2_norm2(iE[2 * a], iE[2 * a + 1]);
    // (d_d psi'_a, psi'_b) by collapsed Gauss quadrature (exact: degree <= 2p - 1)
    const int nq = p + 2;
    std::vector<double> ga, wa;
    gauss_legendre01(nq, ga, wa);
    for (int d = 0; d < 2; ++d) t.D[d].assign((size_t)t.NH * t.NE, 0.0);
    std::vector<double> v(t.NE), ds(t.NE), du(t.NE), vh(t.NH);
    for (int qa = 0; qa < nq; ++qa)
        for (int qb = 0; qb < nq; ++qb) {
            const double a = ga[qa], b = ga[qb];
            const double w = wa[qa] * wa[qb] * (1.0 - a);
            psi2_grad_at(p, iE, a, b, v.data(), ds.data(), du.data());
            psi2_at(p - 1, iH, a, b, vh.data());
            for (int r = 0; r < t.NH; ++r)
                for (int c = 0; c < t.NE; ++c) {
                    t.D[0][(size_t)r * t.NE + c] += w * vh[r] * ds[c];
                    t.D[1][(size_t)r * t.NE + c] += w * vh[r] * du[c];
                }
        }
    for (int r = 0; r < t.NH; ++r) {
        const double nb = std::sqrt(dubiner2_norm2(iH[2 * r], iH[2 * r + 1]));
        for (int c = 0; c < t.NE; ++c) {
            const double na = std::sqrt(t.norm2E[c]);
            for (int d = 0; d < 2; ++d) t.D[d][(size_t)r * t.NE + c] /= (na * nb);
        }
    }
    // exact zeros left at quadrature round-off, as for the 3D tables
    double mx = 0.0;
    for (int d = 0; d < 2; ++d)
        for (double x : t.D[d]) mx = std::max(mx, std::fabs(x));
    for (int d = 0; d < 2; ++d)
        for (double& x : t.D[d])
            if (std::fabs(x) < 1e-12 * mx) x = 0.0;
    for (int f = 0; f < 3; ++f) {
        edge_trace(p, f, t.TrE[f]);
        edge_trace(p - 1, f, t.TrH[f]);
    }
    return DGM_OK;
}

}  // namespace dgm
