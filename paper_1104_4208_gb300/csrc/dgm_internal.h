// Internal declarations shared by the host C++ and the CUDA translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dgm.h"

namespace dgm {

inline int n3(int q) { return q < 0 ? 0 : (q + 1) * (q + 2) * (q + 3) / 6; }
inline int n2(int q) { return q < 0 ? 0 : (q + 1) * (q + 2) / 2; }

void set_error(const std::string& msg);

// ---------------------------------------------------------------- tables
// Reference operators of the orthonormalised Dubiner basis phi_a / ||phi_a||
// (Sec. 3.2.2 gradients, Sec. 3.2.3 traces), FP64.
struct RefTables {
    int p = 0, ph = 0, NE = 0, NH = 0, N2E = 0, N2H = 0;   // ph: degree of H (p - 1, or p)
    std::vector<double> norm2E;          // [NE] ||phi_a||^2 (unnormalised basis)
    std::vector<double> D[3];            // [NH][NE]  (d_d phi'_a, phi'_b), b over H's basis
    std::vector<double> TrE[4];          // [N2E][NE] (phi'_a|_f, psi'_g) over degree-p face modes
    std::vector<double> TrH[4];          // [N2H][NH] (phi'_b|_f, psi'_g) for H's basis (degree ph)
    // Face-frame tangents of local face f in reference coordinates:
    // that[f][i][m], i = 0,1 (t_1 = v_b - v_a, t_2 = v_c - v_a).
    double that[4][2][3];
    // sign of nu_hat . (t_1 x t_2) for the outward reference normal of face f
    double sigma_hat[4];
    // position of each degree-ph face index (i,j) inside the degree-p list
    std::vector<int> pos2H;              // [N2H]
};

// equal_order: H of degree p like E (else p - 1)
int build_ref_tables(int p, RefTables& t, bool equal_order = false);

// Reference operators of the 2D triangle solver (TE fields: E in the plane of
// degree p, H along z of degree p - 1), orthonormalised Dubiner basis psi_a of
// Eq. (4) on the reference triangle (0,0), (1,0), (0,1):
//   D[d]  [N2(p-1)][N2(p)]   (d_d psi'_a, psi'_b), d = x, y
//   TrE[f] [p+1][N2(p)]      int_0^1 psi'_a(edge f at s) L'_g(s) ds, g <= p
//   TrH[f] [p][N2(p-1)]      the same for the degree p - 1 basis, g <= p - 1
// Edge f is opposite reference vertex f, parametrised from its lower-numbered
// vertex to its higher one; L'_g = sqrt(2g+1) P_g(2s-1), orthonormal on [0,1].
struct RefTables2D {
    int p = 0, NE = 0, NH = 0;
    std::vector<double> norm2E;          // [NE] ||psi_a||^2 (unnormalised basis)
    std::vector<double> D[2];
    std::vector<double> TrE[3];
    std::vector<double> TrH[3];
};
int build_ref_tables_2d(int p, RefTables2D& t);
// Squared norm of the unnormalised 3D Dubiner function (closed form).
double dubiner3_norm2(int i, int j, int k);
double dubiner2_norm2(int i, int j);
void index3(int p, std::vector<int>& ijk);   // 3 ints per entry, lexicographic
// Collapsed-coordinate Gauss-Legendre rule on the reference tetrahedron:
// xh [nq][3] Cartesian points, w [nq] weights (sum 1/6), col [nq][3] collapsed coords.
void collapsed_rule(int q1d, std::vector<double>& xh, std::vector<double>& w, std::vector<double>& col);
// Orthonormalised phi'_a at the collapsed rule's points, [nq][N3(p)].
void phi_table(int p, int q1d, std::vector<double>& phi);
// Unnormalised phi_ijk (Sec. 4.2.2) of the index list idx (lexicographic, |ijk| <= p)
// and their Cartesian gradients grad [n][3] at the collapsed point (xi, eta, zeta).
void phi3_grad(int p, const std::vector<int>& idx, double xi, double eta, double zeta, double* val, double* grad);
// Support of the derivative relation in direction dir (0 x, 1 y, 2 z): shifts
// [n][4] = (di, dj, dk, carries the derivative), the lead term's position; returns n.
int grad_support(int dir, int* nterms, int* shifts, int* lead);
// The relations at every (i, j, k) with the shifted indices <= p where the
// support carries a relation with a nonzero lead (the minimum-norm one where
// there are several; 3 ints and n coefficients each, lead coefficient 1, unnormalised basis).
int grad_relations(int p, int dir, std::vector<int>& ijk_out, std::vector<double>& coef_out);
// b [N3(p-1)] = modal derivative in direction dir of u = sum a_ijk phi_ijk
// (unnormalised basis, lexicographic order) by the backward sweep over those
// relations, dense columns elsewhere; returns how many coefficients a relation handled.
int grad_sweep(int p, int dir, const double* a, double* b);
// Orthonormalised phi'_a at n Cartesian reference points xh [n][3], [n][N3(p)].
void phi_at_points(int p, const double* xh, int n, std::vector<double>& out);
void index2(int p, std::vector<int>& ij);

// ---------------------------------------------------------------- mesh
struct MeshData {
    int64_t nv = 0, nt = 0, nfaces = 0, nboundary = 0;
    std::vector<double> xyz;             // [nv][3]
    std::vector<int32_t> tets;           // [nt][4], vertices by ascending key
    std::vector<int32_t> keys;           // [nt][4]
    std::vector<int32_t> nbr;            // [nt][4] neighbour element or -1 (PEC)
    std::vector<int8_t> nbr_face;        // [nt][4] neighbour's local face or -1
    std::vector<int64_t> face_id;        // [nt][4] global face index
    std::vector<int32_t> face_elem;      // [nfaces][2] (t*4+f) of the sides, second -1 on PEC
    std::vector<double> F;               // [nt][9] row-major, columns = edges
    std::vector<double> detF;            // [nt]
};

int build_mesh(int64_t nv, const double* xyz, int64_t nt, const int32_t* tets,
               const int32_t* vertex_key, MeshData& m);

}  // namespace dgm
