// Recurrences for the derivatives of the 3D shape functions (Sec. 3.2.2,
// Sec. 4.2.2) and the backward sweep they give (host side).
//
// A relation in direction d (x, y or z) ties shifts of d/dd phi_ijk to shifts
// of phi_ijk:
//   sum_{s in SD} c_s d/dd phi_{(i,j,k)+s} + sum_{s in S0} c_s phi_{(i,j,k)+s} = 0
// with coefficients rational in (i, j, k).
// - For d/dx, Sec. 4.2.2 prints the support: 12 derivative terms and 4 value
//   terms.  It prints no coefficients.
// - For d/dy and d/dz the paper states that such relations exist but prints
//   neither supports nor coefficients.  The supports below were found by a
//   numerical search: greedy elimination of monomials from a window of shifts,
//   keeping a one-dimensional nullspace, at a generic index.  The same search
//   gives back the printed d/dx support exactly.
//   - d/dy: 18 derivative terms and 2 value terms, shifts up to (1, 3, 4);
//   - d/dz: 18 derivative terms and 1 value term, shifts up to (2, 4, 4).
//
// At a concrete (i, j, k) the coefficients span the nullspace of the ansatz,
// read as an identity in x, y, z.  They are found numerically:
// - the functions are sampled at fixed interior points;
// - the lead coefficient is set to 1, the lead being the derivative term that is
//   highest in the order (degree, k, j, i);
// - the rest follow by least squares (Householder QR on scaled columns).
// Where the other columns are rank deficient, the index carries more than one
// relation (it happens exactly at i = 0); the one with the smallest
// coefficients is taken (minimum-norm least squares), as long as it reproduces
// the lead.  For d/dz at i = 0 the
// lead derivative itself vanishes (phi_0jk does not depend on z), and the
// index needs no relation.
//
// Sweep, the 3D analogue of the Legendre example of Sec. 3.2.2.  For
// u = sum a_ijk phi_ijk the indices are visited from the highest down, in that
// order.  Where an index is the lead of a relation, its derivative is replaced
// by the relation's other terms: derivatives of indices lower in the order, and
// values of degree one less.  Everywhere else its dense column is added.

#include <algorithm>
#include <cmath>
#include <tuple>
#include <vector>

#include "dgm_internal.h"

namespace dgm {

namespace {

// supports: shift (di, dj, dk) and whether the term carries the derivative
struct Support {
    int n;
    int lead;
    int sh[20][4];
};
// d/dx: printed in Sec. 4.2.2 (derivative terms, then value terms)
constexpr Support kSupX = {16, 3, {{1, 1, 2, 1}, {1, 0, 3, 1}, {0, 2, 2, 1}, {0, 1, 3, 1}, {1, 1, 1, 1}, {1, 0, 2, 1},
                                   {0, 2, 1, 1}, {0, 1, 2, 1}, {1, 1, 0, 1}, {1, 0, 1, 1}, {0, 2, 0, 1}, {0, 1, 1, 1},
                                   {1, 1, 1, 0}, {1, 0, 2, 0}, {0, 2, 1, 0}, {0, 1, 2, 0}}};
// d/dy and d/dz: found by the search described above (derivative terms by
// descending (degree, k, j, i), then value terms)
constexpr Support kSupY = {20, 0, {{0, 1, 4, 1}, {1, 0, 4, 1}, {0, 2, 3, 1}, {1, 1, 3, 1}, {0, 3, 2, 1}, {1, 2, 2, 1},
                                   {0, 1, 3, 1}, {1, 0, 3, 1}, {0, 2, 2, 1}, {1, 1, 2, 1}, {0, 3, 1, 1}, {1, 2, 1, 1},
                                   {0, 1, 2, 1}, {1, 0, 2, 1}, {0, 2, 1, 1}, {1, 1, 1, 1}, {0, 3, 0, 1}, {1, 2, 0, 1},
                                   {0, 2, 2, 0}, {1, 1, 2, 0}}};
constexpr Support kSupZ = {19, 0, {{0, 2, 4, 1}, {2, 0, 4, 1}, {0, 3, 3, 1}, {2, 1, 3, 1}, {0, 4, 2, 1}, {2, 2, 2, 1},
                                   {0, 2, 3, 1}, {2, 0, 3, 1}, {0, 3, 2, 1}, {2, 1, 2, 1}, {0, 4, 1, 1}, {2, 2, 1, 1},
                                   {0, 2, 2, 1}, {2, 0, 2, 1}, {0, 3, 1, 1}, {2, 1, 1, 1}, {0, 4, 0, 1}, {2, 2, 0, 1},
                                   {1, 2, 2, 0}}};
const Support& support(int dir) { return dir == 0 ? kSupX : (dir == 1 ? kSupY : kSupZ); }
int support_degree(const Support& S) {
    const int* l = S.sh[S.lead];
    return l[0] + l[1] + l[2];
}
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

// least squares min |A c - y| for A [m][n] (column-major, n <= m) by Householder
// QR that skips numerically dependent columns, then the minimum-norm solution
// of the triangular system.  For full rank that is back substitution.  Where the
// columns are dependent, with R = the first r rows of Q^T A (r the rank, all n
// columns) and b = the first r entries of Q^T y, it is c = R^T w with
// (R R^T) w = b, the smallest c.  The caller checks the residual.
void least_squares(int m, int n, std::vector<double> A, std::vector<double> y, std::vector<double>& c) {
    std::vector<double> colnorm(n);
    std::vector<char> kept(n, 0);
    for (int k = 0; k < n; ++k) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += A[(size_t)k * m + i] * A[(size_t)k * m + i];
        colnorm[k] = std::sqrt(s);
    }
    int rank = 0;
    for (int k = 0; k < n && rank < m; ++k) {
        double* a = &A[(size_t)k * m];
        double nrm = 0.0;
        for (int i = rank; i < m; ++i) nrm += a[i] * a[i];
        nrm = std::sqrt(nrm);
        if (!(nrm > 1e-9 * colnorm[k])) continue;   // in the span of the kept columns
        const double alpha = a[rank] > 0 ? -nrm : nrm;
        std::vector<double> v(a + rank, a + m);
        v[0] -= alpha;
        double vv = 0.0;
        for (double x : v) vv += x * x;
        // apply the reflector to every other column (also those skipped before) and to y
        for (int j = 0; j < n; ++j) {
            if (j == k || kept[j]) continue;
            double* b = &A[(size_t)j * m];
            double s = 0.0;
            for (int i = rank; i < m; ++i) s += v[i - rank] * b[i];
            s = 2.0 * s / vv;
            for (int i = rank; i < m; ++i) b[i] -= s * v[i - rank];
        }
        double s = 0.0;
        for (int i = rank; i < m; ++i) s += v[i - rank] * y[i];
        s = 2.0 * s / vv;
        for (int i = rank; i < m; ++i) y[i] -= s * v[i - rank];
        a[rank] = alpha;
        for (int i = rank + 1; i < m; ++i) a[i] = 0.0;
        kept[k] = 1;
        ++rank;
    }
    c.assign(n, 0.0);
    if (rank == n) {
        // full rank: back substitution on the triangle (no squared condition number)
        for (int r1 = n - 1; r1 >= 0; --r1) {
            double s = y[r1];
            for (int t = r1 + 1; t < n; ++t) s -= A[(size_t)t * m + r1] * c[t];
            c[r1] = s / A[(size_t)r1 * m + r1];
        }
        return;
    }
    // R [rank][n]: rows 0..rank-1 of the transformed columns; G = R R^T (SPD)
    std::vector<double> G((size_t)rank * rank, 0.0), w(y.begin(), y.begin() + rank);
    for (int r1 = 0; r1 < rank; ++r1)
        for (int r2 = 0; r2 <= r1; ++r2) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += A[(size_t)j * m + r1] * A[(size_t)j * m + r2];
            G[(size_t)r1 * rank + r2] = G[(size_t)r2 * rank + r1] = s;
        }
    // Cholesky G = L L^T, then w = G^{-1} b
    for (int r1 = 0; r1 < rank; ++r1) {
        for (int r2 = 0; r2 <= r1; ++r2) {
            double s = G[(size_t)r1 * rank + r2];
            for (int t = 0; t < r2; ++t) s -= G[(size_t)r1 * rank + t] * G[(size_t)r2 * rank + t];
            if (r1 == r2)
                G[(size_t)r1 * rank + r1] = std::sqrt(std::max(s, 1e-300));
            else
                G[(size_t)r1 * rank + r2] = s / G[(size_t)r2 * rank + r2];
        }
    }
    for (int r1 = 0; r1 < rank; ++r1) {
        double s = w[r1];
        for (int t = 0; t < r1; ++t) s -= G[(size_t)r1 * rank + t] * w[t];
        w[r1] = s / G[(size_t)r1 * rank + r1];
    }
    for (int r1 = rank - 1; r1 >= 0; --r1) {
        double s = w[r1];
        for (int t = r1 + 1; t < rank; ++t) s -= G[(size_t)t * rank + r1] * w[t];
        w[r1] = s / G[(size_t)r1 * rank + r1];
    }
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int r1 = 0; r1 < rank; ++r1) s += A[(size_t)j * m + r1] * w[r1];
        c[j] = s;
    }
}

}  // namespace

int grad_support(int dir, int* nterms, int* shifts, int* lead) {
    const Support& S = support(dir);
    if (nterms) *nterms = S.n;
    if (lead) *lead = S.lead;
    if (shifts)
        for (int t = 0; t < S.n; ++t)
            for (int c = 0; c < 4; ++c) shifts[4 * t + c] = S.sh[t][c];
    return S.n;
}

int grad_relations(int p, int dir, std::vector<int>& ijk_out, std::vector<double>& coef_out) {
    ijk_out.clear();
    coef_out.clear();
    const Support& S = support(dir);
    const int top = support_degree(S);
    if (p < top) return 0;
    const Index3 I(p);
    const int N = I.size();
    // samples of every phi and its derivative in direction dir at fixed interior collapsed points
    std::vector<double> val((size_t)kPoints * N), der((size_t)kPoints * N), g3(3 * (size_t)N);
    for (int q = 0; q < kPoints; ++q) {
        const double xi = 0.05 + 0.9 * std::fmod(0.6180339887498949 * (q + 1), 1.0);
        const double eta = 0.05 + 0.9 * std::fmod(0.7548776662466927 * (q + 1), 1.0);
        const double zeta = 0.05 + 0.9 * std::fmod(0.5698402909980532 * (q + 1), 1.0);
        phi3_grad(p, I.ijk, xi, eta, zeta, &val[(size_t)q * N], g3.data());
        for (int r = 0; r < N; ++r) der[(size_t)q * N + r] = g3[3 * (size_t)r + dir];
    }
    const int m = S.n - 1;   // unknowns besides the lead
    for (int r = 0; r < N; ++r) {
        const int i = I.ijk[3 * r], j = I.ijk[3 * r + 1], k = I.ijk[3 * r + 2];
        if (i + j + k + top > p) continue;
        int cols[20];
        for (int t = 0; t < S.n; ++t) cols[t] = I.find(i + S.sh[t][0], j + S.sh[t][1], k + S.sh[t][2]);
        std::vector<double> A((size_t)kPoints * m), y(kPoints), scale(m);
        int c = 0;
        for (int t = 0; t < S.n; ++t) {
            if (t == S.lead) continue;
            const std::vector<double>& src = S.sh[t][3] ? der : val;
            double nrm = 0.0;
            for (int q = 0; q < kPoints; ++q) nrm += src[(size_t)q * N + cols[t]] * src[(size_t)q * N + cols[t]];
            nrm = std::sqrt(nrm);
            scale[c] = nrm > 0.0 ? 1.0 / nrm : 1.0;
            for (int q = 0; q < kPoints; ++q) A[(size_t)c * kPoints + q] = src[(size_t)q * N + cols[t]] * scale[c];
            ++c;
        }
        double ynrm = 0.0;
        for (int q = 0; q < kPoints; ++q) {
            y[q] = -der[(size_t)q * N + cols[S.lead]];
            ynrm += y[q] * y[q];
        }
        if (!(ynrm > 0.0)) continue;   // the lead derivative vanishes (d/dz of phi_0jk)
        std::vector<double> sol;
        least_squares(kPoints, m, A, y, sol);
        // the relation must hold at every sample, not only in the least-squares sense
        double res = 0.0;
        for (int q = 0; q < kPoints; ++q) {
            double v = -y[q];
            for (int t = 0; t < m; ++t) v += A[(size_t)t * kPoints + q] * sol[t];
            res += v * v;
        }
        if (!(res <= 1e-18 * ynrm)) continue;
        ijk_out.insert(ijk_out.end(), {i, j, k});
        c = 0;
        for (int t = 0; t < S.n; ++t) {
            if (t == S.lead) {
                coef_out.push_back(1.0);
            } else {
                coef_out.push_back(sol[c] * scale[c]);
                ++c;
            }
        }
    }
    return (int)ijk_out.size() / 3;
}

int grad_sweep(int p, int dir, const double* a, double* b) {
    const Support& S = support(dir);
    const Index3 IE(p);
    const Index3 IH(std::max(p - 1, 0));
    const int NE = IE.size(), NH = p >= 1 ? IH.size() : 0;
    for (int r = 0; r < NH; ++r) b[r] = 0.0;
    if (p < 1) return 0;
    // dense derivative in the unnormalised basis by exact quadrature:
    // D[beta][alpha] = (d/dd phi_alpha, phi_beta) / ||phi_beta||^2
    std::vector<double> xh, w, col;
    collapsed_rule(p + 2, xh, w, col);
    const int nq = (int)w.size();
    std::vector<double> D((size_t)NH * NE, 0.0), v(NE), g3(3 * (size_t)NE);
    for (int q = 0; q < nq; ++q) {
        phi3_grad(p, IE.ijk, col[3 * q], col[3 * q + 1], col[3 * q + 2], v.data(), g3.data());
        for (int bh = 0; bh < NH; ++bh) {
            const int be = IE.find(IH.ijk[3 * bh], IH.ijk[3 * bh + 1], IH.ijk[3 * bh + 2]);
            const double wb = w[q] * v[be];
            for (int al = 0; al < NE; ++al) D[(size_t)bh * NE + al] += wb * g3[3 * (size_t)al + dir];
        }
    }
    for (int bh = 0; bh < NH; ++bh) {
        const double n2 = dubiner3_norm2(IH.ijk[3 * bh], IH.ijk[3 * bh + 1], IH.ijk[3 * bh + 2]);
        for (int al = 0; al < NE; ++al) D[(size_t)bh * NE + al] /= n2;
    }
    // relations, indexed by their lead
    std::vector<int> rel_ijk;
    std::vector<double> rel_c;
    const int nrel = grad_relations(p, dir, rel_ijk, rel_c);
    std::vector<int> lead_of(NE, -1);
    for (int r = 0; r < nrel; ++r) {
        const int i = rel_ijk[3 * r], j = rel_ijk[3 * r + 1], k = rel_ijk[3 * r + 2];
        const int* l = S.sh[S.lead];
        lead_of[IE.find(i + l[0], j + l[1], k + l[2])] = r;
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
            const double* c = &rel_c[(size_t)S.n * rel];
            for (int t = 0; t < S.n; ++t) {
                if (t == S.lead) continue;
                const int si = i + S.sh[t][0], sj = j + S.sh[t][1], sk = k + S.sh[t][2];
                if (S.sh[t][3])
                    at[IE.find(si, sj, sk)] -= coef * c[t];
                else
                    b[IH.find(si, sj, sk)] -= coef * c[t];
            }
        } else {
            for (int bh = 0; bh < NH; ++bh) b[bh] += coef * D[(size_t)bh * NE + r];
        }
    }
    return swept;
}

}  // namespace dgm
