// Host mesh loader: tet validation, face matching and geometry.
//
// Geometry convention (shared with every consumer of the planes, so that the
// particle tracking is reproducible bit for bit):
//  * local face k of a tet is the face opposite its node k;
//  * faces are matched on sorted node triples; the owner is the tet with the
//    smaller index, faces are numbered by (owner, owner's local face);
//  * the face normal is cross(p_b - p_a, p_c - p_a) for the node ids a < b < c,
//    turned away from the owner's opposite node, divided componentwise by its
//    length sqrt((Nx Nx + Ny Ny) + Nz Nz); area = length / 2;
//  * plane offset d = n . ((p_a + p_b) + p_c) / 3 with dot products summed
//    left to right;
//  * boundary tangent basis t1 = (e_a x n)/|e_a x n| for the axis a of smallest
//    |n_a| (lowest index on ties), t2 = n x t1.
// This file is compiled with floating-point contraction disabled.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "ugkwp_internal.hpp"

namespace ugkwp {

namespace {
struct FaceKey {
    int32_t a, b, c;
    int32_t tet, k;
};
inline bool key_less(const FaceKey& x, const FaceKey& y) {
    if (x.a != y.a) return x.a < y.a;
    if (x.b != y.b) return x.b < y.b;
    if (x.c != y.c) return x.c < y.c;
    return x.tet < y.tet;
}
inline bool key_eq(const FaceKey& x, const FaceKey& y) { return x.a == y.a && x.b == y.b && x.c == y.c; }
inline void sort3(int32_t* v) {
    if (v[0] > v[1]) std::swap(v[0], v[1]);
    if (v[1] > v[2]) std::swap(v[1], v[2]);
    if (v[0] > v[1]) std::swap(v[0], v[1]);
}
inline double dot(const double* a, const double* b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }
inline void cross(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
}  // namespace

bool build_mesh(const ugkwp_mesh_desc& d, MeshHost& M, std::string& err) {
    const int32_t nn = d.n_nodes, nc = d.n_tets, nb = d.n_bfaces;
    M.nn = nn;
    M.nc = nc;
    M.xyz.assign(d.xyz, d.xyz + 3 * (size_t)nn);
    M.tet.assign(d.tets, d.tets + 4 * (size_t)nc);
    const double* X = M.xyz.data();
    M.vol.resize(nc);
    for (int32_t i = 0; i < nc; ++i) {
        const int32_t* t = &M.tet[4 * (size_t)i];
        for (int k = 0; k < 4; ++k)
            if (t[k] < 0 || t[k] >= nn) { err = "tet " + std::to_string(i) + ": node index out of range"; return false; }
        const double *p0 = X + 3 * (size_t)t[0], *p1 = X + 3 * (size_t)t[1], *p2 = X + 3 * (size_t)t[2],
                     *p3 = X + 3 * (size_t)t[3];
        double e1[3], e2[3], e3[3], c23[3];
        for (int c = 0; c < 3; ++c) { e1[c] = p1[c] - p0[c]; e2[c] = p2[c] - p0[c]; e3[c] = p3[c] - p0[c]; }
        cross(e2, e3, c23);
        const double V = dot(e1, c23) / 6.0;
        if (!(V > 0.0)) { err = "tet " + std::to_string(i) + " has non-positive volume"; return false; }
        M.vol[i] = V;
    }
    // --- face matching by sorting all 4 nc face keys
    std::vector<FaceKey> keys(4 * (size_t)nc);
    for (int32_t i = 0; i < nc; ++i)
        for (int k = 0; k < 4; ++k) {
            int32_t v[3], j = 0;
            for (int l = 0; l < 4; ++l) if (l != k) v[j++] = M.tet[4 * (size_t)i + l];
            sort3(v);
            keys[4 * (size_t)i + k] = FaceKey{v[0], v[1], v[2], i, k};
        }
    std::sort(keys.begin(), keys.end(), key_less);
    struct Face { int32_t own, own_k, nbr, nbr_k; };
    std::vector<Face> faces;
    faces.reserve(2 * (size_t)nc + 16);
    for (size_t q = 0; q < keys.size();) {
        size_t r = q + 1;
        while (r < keys.size() && key_eq(keys[r], keys[q])) ++r;
        if (r - q > 2) { err = "a face is shared by more than two tets"; return false; }
        Face f{keys[q].tet, keys[q].k, -1, -1};
        if (r - q == 2) { f.nbr = keys[q + 1].tet; f.nbr_k = keys[q + 1].k; }
        faces.push_back(f);
        q = r;
    }
    std::sort(faces.begin(), faces.end(), [](const Face& x, const Face& y) {
        return x.own != y.own ? x.own < y.own : x.own_k < y.own_k;
    });
    const int32_t nf = (int32_t)faces.size();
    M.nf = nf;
    M.f_own.resize(nf); M.f_own_k.resize(nf); M.f_nbr.resize(nf); M.f_nbr_k.resize(nf);
    M.cf.assign(4 * (size_t)nc, -1);
    M.cf_sign.assign(4 * (size_t)nc, 0);
    for (int32_t f = 0; f < nf; ++f) {
        M.f_own[f] = faces[f].own; M.f_own_k[f] = faces[f].own_k;
        M.f_nbr[f] = faces[f].nbr; M.f_nbr_k[f] = faces[f].nbr_k;
        M.cf[4 * (size_t)faces[f].own + faces[f].own_k] = f;
        M.cf_sign[4 * (size_t)faces[f].own + faces[f].own_k] = 1;
        if (faces[f].nbr >= 0) {
            M.cf[4 * (size_t)faces[f].nbr + faces[f].nbr_k] = f;
            M.cf_sign[4 * (size_t)faces[f].nbr + faces[f].nbr_k] = -1;
        }
    }
    // --- boundary tags: match the listed boundary faces by sorted triple
    std::vector<FaceKey> bkeys(nb);
    for (int32_t b = 0; b < nb; ++b) {
        int32_t v[3] = {d.bfaces[3 * (size_t)b], d.bfaces[3 * (size_t)b + 1], d.bfaces[3 * (size_t)b + 2]};
        sort3(v);
        bkeys[b] = FaceKey{v[0], v[1], v[2], d.bface_tags[b], b};
    }
    std::sort(bkeys.begin(), bkeys.end(), key_less);
    for (int32_t b = 1; b < nb; ++b)
        if (key_eq(bkeys[b], bkeys[b - 1])) { err = "a boundary face is listed twice"; return false; }
    M.f_tag.assign(nf, -1);
    M.bf_of_face.assign(nf, -1);
    M.face_of_bf.clear();
    int32_t matched = 0;
    for (int32_t f = 0; f < nf; ++f) {
        if (M.f_nbr[f] >= 0) continue;
        int32_t v[3], j = 0;
        for (int l = 0; l < 4; ++l) if (l != M.f_own_k[f]) v[j++] = M.tet[4 * (size_t)M.f_own[f] + l];
        sort3(v);
        FaceKey probe{v[0], v[1], v[2], -2147483647 - 1, 0};
        auto it = std::lower_bound(bkeys.begin(), bkeys.end(), probe, key_less);
        if (it == bkeys.end() || !(it->a == v[0] && it->b == v[1] && it->c == v[2])) {
            err = "face " + std::to_string(f) + " has one tet and no boundary tag";
            return false;
        }
        M.f_tag[f] = it->tet;  // tag stored in the tet slot of the key
        M.bf_of_face[f] = (int32_t)M.face_of_bf.size();
        M.face_of_bf.push_back(f);
        ++matched;
    }
    if (matched != nb) { err = "a listed boundary face is not a boundary face of the mesh"; return false; }
    M.nbf = matched;
    // --- face geometry
    M.f_n.resize(3 * (size_t)nf); M.f_area.resize(nf); M.f_d.resize(nf);
    M.f_t1.assign(3 * (size_t)nf, 0.0); M.f_t2.assign(3 * (size_t)nf, 0.0);
    M.f_c.resize(3 * (size_t)nf);
    for (int32_t f = 0; f < nf; ++f) {
        const int32_t o = M.f_own[f], k = M.f_own_k[f];
        int32_t v[3], j = 0;
        for (int l = 0; l < 4; ++l) if (l != k) v[j++] = M.tet[4 * (size_t)o + l];
        sort3(v);
        const double *pa = X + 3 * (size_t)v[0], *pb = X + 3 * (size_t)v[1], *pc = X + 3 * (size_t)v[2];
        const double* po = X + 3 * (size_t)M.tet[4 * (size_t)o + k];
        double eb[3], ec[3], eo[3], N[3];
        for (int c = 0; c < 3; ++c) { eb[c] = pb[c] - pa[c]; ec[c] = pc[c] - pa[c]; eo[c] = po[c] - pa[c]; }
        cross(eb, ec, N);
        const double side = dot(N, eo);
        if (side == 0.0) { err = "degenerate face " + std::to_string(f); return false; }
        if (side > 0.0) for (int c = 0; c < 3; ++c) N[c] = -N[c];
        const double len = std::sqrt(dot(N, N));
        double* n = &M.f_n[3 * (size_t)f];
        for (int c = 0; c < 3; ++c) n[c] = N[c] / len;
        M.f_area[f] = 0.5 * len;
        double cen[3];
        for (int c = 0; c < 3; ++c) cen[c] = ((pa[c] + pb[c]) + pc[c]) / 3.0;
        for (int c = 0; c < 3; ++c) M.f_c[3 * (size_t)f + c] = cen[c];
        M.f_d[f] = dot(n, cen);
        int ax = 0;
        if (std::fabs(n[1]) < std::fabs(n[ax])) ax = 1;
        if (std::fabs(n[2]) < std::fabs(n[ax])) ax = 2;
        double e[3] = {0.0, 0.0, 0.0}, t1[3], t2[3];
        e[ax] = 1.0;
        cross(e, n, t1);
        const double l1 = std::sqrt(dot(t1, t1));
        for (int c = 0; c < 3; ++c) t1[c] = t1[c] / l1;
        cross(n, t1, t2);
        for (int c = 0; c < 3; ++c) { M.f_t1[3 * (size_t)f + c] = t1[c]; M.f_t2[3 * (size_t)f + c] = t2[c]; }
    }
    // --- projected areas Delta S^d = 1/2 sum_k |n_d| |S| (Sec. 2.4 (a))
    M.dS.resize(3 * (size_t)nc);
    for (int32_t i = 0; i < nc; ++i)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k) {
                const int32_t f = M.cf[4 * (size_t)i + k];
                acc = acc + std::fabs(M.f_n[3 * (size_t)f + c] * M.f_area[f]);
            }
            M.dS[3 * (size_t)i + c] = 0.5 * acc;
        }
    return true;
}

}  // namespace ugkwp
