// Mesh preprocessing (host): key-ordered element maps and facet adjacency.
//
// Ordering the four vertices of every tetrahedron by ascending key makes the
// three vertices of each face appear in the same order from both sides.  With
// the face parametrisation x = X_a + s t_1 + u t_2 (a < b < c by key) both
// elements then share the face frame, and because the covariant transform
// preserves tangential components (Sec. 3.2.1: u . t = u_hat . t_hat for
// t = F t_hat), the tangential trace coefficients of a face agree between the
// two sides without any re-orientation.  Per element the mesh keeps nothing
// but its affine map and its neighbours (Sec. 3.4).

#include <algorithm>
#include <array>
#include <cmath>
#include <string>

#include "dgm_internal.h"

namespace dgm {

int build_mesh(int64_t nv, const double* xyz, int64_t nt, const int32_t* tets,
               const int32_t* vertex_key, MeshData& m) {
    if (nv <= 0 || nt <= 0 || !xyz || !tets) {
        set_error("mesh: empty or null input");
        return DGM_ERR_INVALID_ARG;
    }
    if (nt > (int64_t)1 << 29) {
        set_error("mesh: too many elements (limit 2^29)");
        return DGM_ERR_INVALID_ARG;
    }
    m.nv = nv;
    m.nt = nt;
    m.xyz.assign(xyz, xyz + 3 * nv);
    m.tets.resize(4 * nt);
    m.keys.resize(4 * nt);
    m.F.resize(9 * nt);
    m.detF.resize(nt);
    for (int64_t t = 0; t < nt; ++t) {
        std::array<std::pair<int64_t, int32_t>, 4> v;
        for (int q = 0; q < 4; ++q) {
            const int32_t id = tets[4 * t + q];
            if (id < 0 || id >= nv) {
                set_error("mesh: vertex id out of range in tet " + std::to_string(t));
                return DGM_ERR_INVALID_ARG;
            }
            v[q] = {vertex_key ? (int64_t)vertex_key[id] : (int64_t)id, id};
        }
        std::sort(v.begin(), v.end());
        for (int q = 0; q < 3; ++q)
            if (v[q].first == v[q + 1].first) {
                set_error("mesh: repeated vertex key in tet " + std::to_string(t));
                return DGM_ERR_INVALID_ARG;
            }
        for (int q = 0; q < 4; ++q) {
            m.tets[4 * t + q] = v[q].second;
            m.keys[4 * t + q] = (int32_t)v[q].first;
        }
        const double* X0 = xyz + 3 * (int64_t)v[0].second;
        double* F = &m.F[9 * t];
        double scale = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double* Xc = xyz + 3 * (int64_t)v[c + 1].second;
            for (int r = 0; r < 3; ++r) {
                F[3 * r + c] = Xc[r] - X0[r];
                scale = std::max(scale, std::fabs(F[3 * r + c]));
            }
        }
        const double det = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6])
                           + F[2] * (F[3] * F[7] - F[4] * F[6]);
        if (!(std::fabs(det) > 1e-12 * scale * scale * scale)) {
            set_error("mesh: degenerate tetrahedron " + std::to_string(t));
            return DGM_ERR_INVALID_ARG;
        }
        m.detF[t] = det;
    }

    // facet matching: sort (key triple, element-face) records
    struct Rec {
        int32_t k[3];
        int64_t tf;
    };
    std::vector<Rec> recs(4 * nt);
    for (int64_t t = 0; t < nt; ++t)
        for (int f = 0; f < 4; ++f) {
            Rec r;
            int c = 0;
            for (int q = 0; q < 4; ++q)
                if (q != f) r.k[c++] = m.keys[4 * t + q];
            r.tf = 4 * t + f;
            recs[4 * t + f] = r;
        }
    std::sort(recs.begin(), recs.end(), [](const Rec& a, const Rec& b) {
        if (a.k[0] != b.k[0]) return a.k[0] < b.k[0];
        if (a.k[1] != b.k[1]) return a.k[1] < b.k[1];
        if (a.k[2] != b.k[2]) return a.k[2] < b.k[2];
        return a.tf < b.tf;
    });
    m.nbr.assign(4 * nt, -1);
    m.nbr_face.assign(4 * nt, -1);
    size_t i = 0;
    while (i < recs.size()) {
        size_t j = i + 1;
        while (j < recs.size() && recs[j].k[0] == recs[i].k[0] && recs[j].k[1] == recs[i].k[1] &&
               recs[j].k[2] == recs[i].k[2])
            ++j;
        if (j - i > 2) {
            set_error("mesh: face shared by more than two tetrahedra");
            return DGM_ERR_INVALID_ARG;
        }
        if (j - i == 2) {
            const int64_t a = recs[i].tf, b = recs[i + 1].tf;
            if (a / 4 == b / 4) {
                set_error("mesh: tetrahedron glued to itself");
                return DGM_ERR_INVALID_ARG;
            }
            m.nbr[a] = (int32_t)(b / 4);
            m.nbr_face[a] = (int8_t)(b % 4);
            m.nbr[b] = (int32_t)(a / 4);
            m.nbr_face[b] = (int8_t)(a % 4);
        }
        i = j;
    }
    // faces numbered by first occurrence in (element, local face) order
    m.face_id.assign(4 * nt, -1);
    m.face_elem.clear();
    int64_t nf = 0, nb = 0;
    for (int64_t t = 0; t < nt; ++t)
        for (int f = 0; f < 4; ++f) {
            if (m.face_id[4 * t + f] >= 0) continue;
            m.face_id[4 * t + f] = nf;
            m.face_elem.push_back((int32_t)(4 * t + f));
            if (m.nbr[4 * t + f] >= 0) {
                const int64_t o = 4 * (int64_t)m.nbr[4 * t + f] + m.nbr_face[4 * t + f];
                m.face_id[o] = nf;
                m.face_elem.push_back((int32_t)o);
            } else {
                m.face_elem.push_back(-1);
                ++nb;
            }
            ++nf;
        }
    m.nfaces = nf;
    m.nboundary = nb;
    return DGM_OK;
}

}  // namespace dgm
