// The d/dx relation of the 3D shape functions (Sec. 3.2.2, Sec. 4.2.2) and the
// backward sweep it gives (host side).
//
// Sec. 4.2.2 prints the support of a relation between shifts of d/dx phi_ijk
// and of phi_ijk: 16 monomials, with coefficients rational in (i, j, k) that the
// paper does not print.
//   sum_{s in SD} c_s d/dx phi_{(i,j,k)+s} + sum_{s in S0} c_s phi_{(i,j,k)+s} = 0
// At a concrete (i, j, k) the coefficients span the nullspace of this ansatz,
// read as an identity in x, y, z.  They are found here numerically:
// - the 16 functions are sampled at fixed interior points;
// - the lead coefficient (term S_j S_k^3 D_x) is set to 1;
// - the other 15 follow by least squares (Householder QR on scaled columns).
// Where those 15 columns are rank deficient, the index carries more than one
// relation (low indices); it is left to the dense operator.
//
// Sweep, the 3D analogue of the Legendre example of Sec. 3.2.2.  For
// u = sum a_ijk phi_ijk the indices are visited from the highest down, in the
// order (degree, k, j, i).  Where an index is the lead of a relation, its
// derivative is replaced by the relation's other terms: derivatives of
// indices lower in that order, and values of degree one less.  Everywhere
// else its dense column is added.

#include <algorithm>
#include <cmath>
#include <tuple>
#include <vector>

#include "dgm_internal.h"

namespace dgm {

namespace {

// printed support of the d/dx relation: shifts of the terms with D_x, then of those without
constexpr int kSD[12][3] = {{1, 1, 2}, {1, 0, 3}, {0, 2, 2}, {0, 1, 3}, {1, 1, 1}, {1, 0, 2},
                            {0, 2, 1}, {0, 1, 2}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}};
constexpr int kS0[4][3] = {{1, 1, 1}, {1, 0, 2}, {0, 2, 1}, {0, 1, 2}};
constexpr int kLead = 3;   // S_j S_k^3 D_x
constexpr int kPoints = 64;

struct Index3 {
    int p;
    std::vector<int> ijk;   // lexicographic, |ijk| <= p
    std::vector<int> pos;   // [(p+1)^3] position in ijk, -1 outside
    explicit Index3(int p_) : p(p_) {
        index3(p, ijk);
        pos.assign((size_t)(p + 1) * (p + 1) * (p + 1), -1);
        for (int r = 0; r < (int)ijk.size() / 3; ++r) pos[at(ijk[3 * r], ijk[3 * r + 1], ijk[3 * r + 2])] = r;
    }
    size_t at(int i, int j, int k) const { return ((size_t)i * (p + 1) + j) * (p + 1) + k; }
    int find(int i, int j, int k) const {
        if (i < 0 || j < 0 || k < 0 || i + j + k > p) return -1;
        return pos[at(i, j, k)];
    }
    int size() const { return (int)ijk.size() / 3; }
};

// least squares min |A c - y| for A [m][n] (column-major, n <= m) by Householder QR;
// returns false when the columns are rank deficient (relative to the largest pivot)
bool least_squares(int m, int n, std::vector<double> A, std::vector<double> y, std::vector<double>& c) {
    std::vector<double> diag(n);
    for (int k = 0; k < n; ++k) {
        double* a = &A[(size_t)k * m];
        double nrm = 0.0;
        for (int i = k; i < m; ++i) nrm += a[i] * a[i];
        nrm = std::sqrt(nrm);
        const double alpha = a[k] > 0 ? -nrm : nrm;
        diag[k] = alpha;
        if (nrm == 0.0) continue;
        a[k] -= alpha;
        double vv = 0.0;
        for (int i = k; i < m; ++i) vv += a[i] * a[i];
        if (vv == 0.0) continue;
        for (int j = k + 1; j < n; ++j) {
            double* b = &A[(size_t)j * m];
            double s = 0.0;
            for (int i = k; i < m; ++i) s += a[i] * b[i];
            s = 2.0 * s / vv;
            for (int i = k; i < m; ++i) b[i] -= s * a[i];
        }
        double s = 0.0;
        for (int i = k; i < m; ++i) s += a[i] * y[i];
        s = 2.0 * s / vv;
        for (int i = k; i < m; ++i) y[i] -= s * a[i];
    }
    double dmax = 0.0;
    for (double d : diag) dmax = std::max(dmax, std::fabs(d));
    for (double d : diag)
        if (!(std::fabs(d) > 1e-9 * dmax)) return false;
    c.assign(n, 0.0);
    for (int k = n - 1; k >= 0; --k) {
        double s = y[k];
        for (int j = k + 1; j < n; ++j) s -= A[(size_t)j * m + k] * c[j];
        c[k] = s / diag[k];
    }
    return true;
}

}  // namespace

int dx_relations(int p, std::vector<int>& ijk_out, std::vector<double>& coef_out) {
    ijk_out.clear();
    coef_out.clear();
    if (p < 4) return 0;
    const Index3 I(p);
    const int N = I.size();
    // samples of every phi and d/dx phi up to degree p at fixed interior collapsed points
    std::vector<double> val((size_t)kPoints * N), dx((size_t)kPoints * N);
    for (int q = 0; q < kPoints; ++q) {
        const double xi = 0.05 + 0.9 * std::fmod(0.6180339887498949 * (q + 1), 1.0);
        const double eta = 0.05 + 0.9 * std::fmod(0.7548776662466927 * (q + 1), 1.0);
        const double zeta = 0.05 + 0.9 * std::fmod(0.5698402909980532 * (q + 1), 1.0);
        phi3_values(p, I.ijk, xi, eta, zeta, &val[(size_t)q * N], &dx[(size_t)q * N]);
    }
    for (int r = 0; r < N; ++r) {
        const int i = I.ijk[3 * r], j = I.ijk[3 * r + 1], k = I.ijk[3 * r + 2];
        if (i + j + k + 4 > p) continue;
        // the 16 columns; column c of the lead is the right-hand side
        int cols[16];
        for (int s = 0; s < 12; ++s) cols[s] = I.find(i + kSD[s][0], j + kSD[s][1], k + kSD[s][2]);
        for (int s = 0; s < 4; ++s) cols[12 + s] = I.find(i + kS0[s][0], j + kS0[s][1], k + kS0[s][2]);
        std::vector<double> A((size_t)kPoints * 15), y(kPoints), scale(15);
        int c = 0;
        for (int s = 0; s < 16; ++s) {
            if (s == kLead) continue;
            const std::vector<double>& src = s < 12 ? dx : val;
            double nrm = 0.0;
            for (int q = 0; q < kPoints; ++q) nrm += src[(size_t)q * N + cols[s]] * src[(size_t)q * N + cols[s]];
            nrm = std::sqrt(nrm);
            scale[c] = nrm > 0.0 ? 1.0 / nrm : 1.0;
            for (int q = 0; q < kPoints; ++q) A[(size_t)c * kPoints + q] = src[(size_t)q * N + cols[s]] * scale[c];
            ++c;
        }
        double ynrm = 0.0;
        for (int q = 0; q < kPoints; ++q) {
            y[q] = -dx[(size_t)q * N + cols[kLead]];
            ynrm += y[q] * y[q];
        }
        std::vector<double> sol;
        if (!least_squares(kPoints, 15, A, y, sol)) continue;
        // the relation must hold at every sample, not only in the least-squares sense
        double res = 0.0;
        for (int q = 0; q < kPoints; ++q) {
            double s = -y[q];
            for (int t = 0; t < 15; ++t) s += A[(size_t)t * kPoints + q] * sol[t];
            res += s * s;
        }
        if (!(res <= 1e-18 * ynrm)) continue;
        ijk_out.insert(ijk_out.end(), {i, j, k});
        c = 0;
        for (int s = 0; s < 16; ++s) {
            if (s == kLead) {
                coef_out.push_back(1.0);
            } else {
                coef_out.push_back(sol[c] * scale[c]);
                ++c;
            }
        }
    }
    return (int)ijk_out.size() / 3;
}

int dx_sweep(int p, const double* a, double* b) {
    const Index3 IE(p);
    const Index3 IH(std::max(p - 1, 0));
    const int NE = IE.size(), NH = p >= 1 ? IH.size() : 0;
    for (int r = 0; r < NH; ++r) b[r] = 0.0;
    if (p < 1) return 0;
    // dense d/dx in the unnormalised basis by exact quadrature:
    // Dx[beta][alpha] = (d/dx phi_alpha, phi_beta) / ||phi_beta||^2
    std::vector<double> xh, w, col;
    collapsed_rule(p + 2, xh, w, col);
    const int nq = (int)w.size();
    std::vector<double> Dx((size_t)NH * NE, 0.0), v(NE), d(NE);
    for (int q = 0; q < nq; ++q) {
        phi3_values(p, IE.ijk, col[3 * q], col[3 * q + 1], col[3 * q + 2], v.data(), d.data());
        for (int bh = 0; bh < NH; ++bh) {
            const int be = IE.find(IH.ijk[3 * bh], IH.ijk[3 * bh + 1], IH.ijk[3 * bh + 2]);
            const double wb = w[q] * v[be];
            for (int al = 0; al < NE; ++al) Dx[(size_t)bh * NE + al] += wb * d[al];
        }
    }
    for (int bh = 0; bh < NH; ++bh) {
        const double n2 = dubiner3_norm2(IH.ijk[3 * bh], IH.ijk[3 * bh + 1], IH.ijk[3 * bh + 2]);
        for (int al = 0; al < NE; ++al) Dx[(size_t)bh * NE + al] /= n2;
    }
    // relations, indexed by their lead
    std::vector<int> rel_ijk;
    std::vector<double> rel_c;
    const int nrel = dx_relations(p, rel_ijk, rel_c);
    std::vector<int> lead_of(NE, -1);
    for (int r = 0; r < nrel; ++r) {
        const int i = rel_ijk[3 * r], j = rel_ijk[3 * r + 1], k = rel_ijk[3 * r + 2];
        lead_of[IE.find(i + kSD[kLead][0], j + kSD[kLead][1], k + kSD[kLead][2])] = r;
    }
    // visiting order: degree, then k, then j, then i, all descending
    std::vector<int> order(NE);
    for (int r = 0; r < NE; ++r) order[r] = r;
    auto key = [&](int r) {
        const int i = IE.ijk[3 * r], j = IE.ijk[3 * r + 1], k = IE.ijk[3 * r + 2];
        return std::make_tuple(i + j + k, k, j, i);
    };
    std::sort(order.begin(), order.end(), [&](int x, int y) { return key(x) > key(y); });
    std::vector<double> at(a, a + NE);
    int swept = 0;
    for (int r : order) {
        const double coef = at[r];
        if (coef == 0.0) continue;
        const int rel = lead_of[r];
        if (rel >= 0) {
            ++swept;
            const int i = rel_ijk[3 * rel], j = rel_ijk[3 * rel + 1], k = rel_ijk[3 * rel + 2];
            const double* c = &rel_c[(size_t)16 * rel];
            for (int s = 0; s < 12; ++s)
                if (s != kLead) at[IE.find(i + kSD[s][0], j + kSD[s][1], k + kSD[s][2])] -= coef * c[s];
            for (int s = 0; s < 4; ++s) b[IH.find(i + kS0[s][0], j + kS0[s][1], k + kS0[s][2])] -= coef * c[12 + s];
        } else {
            for (int bh = 0; bh < NH; ++bh) b[bh] += coef * Dx[(size_t)bh * NE + r];
        }
    }
    return swept;
}

}  // namespace dgm
