// Host-side mesh construction: validation, canonical edges, 1->4 midpoint
// subdivision and the circumcentric Hodge stars.
//
// Sec. 2.1 defines the embedded 2-simplicial complex (face maps E->V, T->E,
// no duplicate simplices, every vertex and edge in a triangle); Sec. 2.2.1
// describes binary (1->4) subdivision; Sec. 3.1.1 defines *0 (dual-cell
// areas) and *1 (dual/primal length ratio).  Edges are (lo, hi) with lo < hi
// in lexicographic order, found by a counting sort on lo.
#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>

#include "host.h"

namespace decimpl {

namespace {

struct HalfEdge {
    int32_t hi;
    int32_t h;  // 3 * triangle + k
};

}  // namespace

Status build_mesh(std::vector<double> verts, int dim, std::vector<int32_t> tris, HostMesh &out) {
    if (dim != 2 && dim != 3) return Status::fail(DEC_ERR_ARG, "dim must be 2 or 3");
    if (verts.size() % dim != 0 || tris.size() % 3 != 0) return Status::fail(DEC_ERR_ARG, "array sizes");
    const int64_t nv = (int64_t)verts.size() / dim;
    const int64_t nt = (int64_t)tris.size() / 3;
    if (nv < 1 || nt < 1) return Status::fail(DEC_ERR_ARG, "empty mesh");
    if (nv >= (int64_t)1 << 31 || 3 * nt >= (int64_t)1 << 31) return Status::fail(DEC_ERR_ARG, "mesh too large");
    for (int64_t i = 0; i < 3 * nt; ++i)
        if (tris[i] < 0 || tris[i] >= nv) return Status::fail(DEC_ERR_MESH, "triangle vertex index out of range");
    for (int64_t t = 0; t < nt; ++t) {
        int32_t a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
        if (a == b || b == c || a == c) return Status::fail(DEC_ERR_MESH, "a triangle repeats a vertex");
    }
    {  // every vertex in some triangle
        std::vector<uint8_t> used(nv, 0);
        for (int64_t i = 0; i < 3 * nt; ++i) used[tris[i]] = 1;
        for (int64_t v = 0; v < nv; ++v)
            if (!used[v]) return Status::fail(DEC_ERR_MESH, "a vertex lies in no triangle");
    }
    {  // no two triangles on the same vertex set: bucket sorted triples by their smallest vertex
        std::vector<int64_t> cnt(nv + 1, 0);
        std::vector<std::array<int32_t, 3>> key(nt);
        for (int64_t t = 0; t < nt; ++t) {
            std::array<int32_t, 3> k = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
            std::sort(k.begin(), k.end());
            key[t] = k;
            cnt[k[0] + 1]++;
        }
        std::partial_sum(cnt.begin(), cnt.end(), cnt.begin());
        std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
        std::vector<std::pair<int32_t, int32_t>> bucket(nt);
        for (int64_t t = 0; t < nt; ++t) bucket[pos[key[t][0]]++] = {key[t][1], key[t][2]};
        for (int64_t v = 0; v < nv; ++v) {
            auto b = bucket.begin() + cnt[v], e = bucket.begin() + cnt[v + 1];
            std::sort(b, e);
            if (std::adjacent_find(b, e) != e) return Status::fail(DEC_ERR_MESH, "two triangles share the same vertex set");
        }
    }
    // half-edges bucketed by their low vertex, then sorted by (hi, h) inside each bucket
    const int64_t nh = 3 * nt;
    std::vector<int64_t> off(nv + 1, 0);
    for (int64_t h = 0; h < nh; ++h) {
        int32_t s = tris[h], d = tris[(h / 3) * 3 + (h % 3 + 1) % 3];
        off[std::min(s, d) + 1]++;
    }
    std::partial_sum(off.begin(), off.end(), off.begin());
    std::vector<int64_t> fill(off.begin(), off.end() - 1);
    std::vector<HalfEdge> he(nh);
    for (int64_t h = 0; h < nh; ++h) {
        int32_t s = tris[h], d = tris[(h / 3) * 3 + (h % 3 + 1) % 3];
        he[fill[std::min(s, d)]++] = HalfEdge{std::max(s, d), (int32_t)h};
    }
    out.tri_edges.assign(nh, -1);
    out.edges.clear();
    out.edges.reserve(nh);  // upper bound 2 * ne <= 2 * nh
    int32_t ne = 0;
    for (int64_t v = 0; v < nv; ++v) {
        auto b = he.begin() + off[v], e = he.begin() + off[v + 1];
        std::sort(b, e, [](const HalfEdge &x, const HalfEdge &y) { return x.hi != y.hi ? x.hi < y.hi : x.h < y.h; });
        for (auto it = b; it != e;) {
            auto jt = it;
            while (jt != e && jt->hi == it->hi) ++jt;
            if (jt - it > 2) return Status::fail(DEC_ERR_MESH, "an edge lies in more than two triangles");
            for (auto k = it; k != jt; ++k) out.tri_edges[k->h] = ne;
            out.edges.push_back((int32_t)v);
            out.edges.push_back(it->hi);
            ++ne;
            it = jt;
        }
    }
    out.dim = dim;
    out.nv = nv;
    out.nt = nt;
    out.ne = ne;
    out.verts = std::move(verts);
    out.tris = std::move(tris);
    return Status::ok();
}

// Z-order keys of points [n x dim]: per axis q = floor((x - lo) * ((2^B - 1)/(hi - lo)))
// on the points' bounding box, clamped to [0, 2^B - 1], bits interleaved (axis 0 lowest).
void morton_keys(const double *pts, int64_t n, int dim, std::vector<uint64_t> &keys) {
    const int B = dim == 3 ? 21 : 31;
    const double top = (double)(((uint64_t)1 << B) - 1);
    keys.assign(n, 0);
    for (int d = 0; d < dim; ++d) {
        double lo = pts[d], hi = pts[d];
        for (int64_t i = 1; i < n; ++i) {
            lo = std::min(lo, pts[i * dim + d]);
            hi = std::max(hi, pts[i * dim + d]);
        }
        const double scale = hi > lo ? top / (hi - lo) : 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double q = std::floor((pts[i * dim + d] - lo) * scale);
            q = std::min(std::max(q, 0.0), top);
            const uint64_t qi = (uint64_t)q;
            uint64_t k = 0;
            for (int b = 0; b < B; ++b) k |= ((qi >> b) & 1u) << (dim * b + d);
            keys[i] |= k;
        }
    }
}

Status subdivide(const HostMesh &c, bool sphere, bool morton, HostMesh &f, std::vector<int32_t> *parents) {
    if (sphere && c.dim != 3) return Status::fail(DEC_ERR_ARG, "sphere projection needs 3-D vertices");
    const int dim = c.dim;
    const int64_t nc = c.nv, E = c.ne, T = c.nt;
    if (nc + E >= (int64_t)1 << 31 || 12 * T >= (int64_t)1 << 31) return Status::fail(DEC_ERR_ARG, "refined mesh too large");
    std::vector<double> fv((nc + E) * dim);
    std::copy(c.verts.begin(), c.verts.end(), fv.begin());
    for (int64_t e = 0; e < E; ++e) {
        const double *pa = &c.verts[(int64_t)c.edges[2 * e] * dim];
        const double *pb = &c.verts[(int64_t)c.edges[2 * e + 1] * dim];
        double m[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) m[d] = (pa[d] + pb[d]) * 0.5;
        if (sphere) {
            double s = m[0] * m[0] + m[1] * m[1];
            s = s + m[2] * m[2];
            double nrm = std::sqrt(s);
            for (int d = 0; d < 3; ++d) m[d] = m[d] / nrm;
        }
        for (int d = 0; d < dim; ++d) fv[(nc + e) * dim + d] = m[d];
    }
    // numbering of the new vertices: rank[e] = k for the midpoint of coarse edge e
    std::vector<int64_t> perm(E), rank(E);
    for (int64_t e = 0; e < E; ++e) perm[e] = e;
    if (morton && E > 0) {
        std::vector<uint64_t> keys;
        morton_keys(&fv[nc * dim], E, dim, keys);
        std::stable_sort(perm.begin(), perm.end(), [&](int64_t x, int64_t y) { return keys[x] < keys[y]; });
        std::vector<double> mids(fv.begin() + nc * dim, fv.end());
        for (int64_t k = 0; k < E; ++k)
            for (int d = 0; d < dim; ++d) fv[(nc + k) * dim + d] = mids[perm[k] * dim + d];
    }
    for (int64_t k = 0; k < E; ++k) rank[perm[k]] = k;
    if (parents) {
        parents->resize(2 * E);
        for (int64_t k = 0; k < E; ++k) {
            (*parents)[2 * k] = c.edges[2 * perm[k]];
            (*parents)[2 * k + 1] = c.edges[2 * perm[k] + 1];
        }
    }
    std::vector<int32_t> ft(12 * T);
    for (int64_t t = 0; t < T; ++t) {
        int32_t a = c.tris[3 * t], b = c.tris[3 * t + 1], cc = c.tris[3 * t + 2];
        int32_t mab = (int32_t)(nc + rank[c.tri_edges[3 * t]]);
        int32_t mbc = (int32_t)(nc + rank[c.tri_edges[3 * t + 1]]);
        int32_t mca = (int32_t)(nc + rank[c.tri_edges[3 * t + 2]]);
        int32_t *o = &ft[12 * t];
        o[0] = a;   o[1] = mab;  o[2] = mca;
        o[3] = mab; o[4] = b;    o[5] = mbc;
        o[6] = mca; o[7] = mbc;  o[8] = cc;
        o[9] = mab; o[10] = mbc; o[11] = mca;
    }
    return build_mesh(std::move(fv), dim, std::move(ft), f);
}

Status subdivide_cubic(const HostMesh &c, bool sphere, HostMesh &f, std::vector<int32_t> &map_idx,
                       std::vector<double> &map_w) {
    if (sphere && c.dim != 3) return Status::fail(DEC_ERR_ARG, "sphere projection needs 3-D vertices");
    const int dim = c.dim;
    const int64_t nc = c.nv, E = c.ne, T = c.nt;
    const int64_t nf = nc + 2 * E + T;
    if (nf >= (int64_t)1 << 31 || 27 * T >= (int64_t)1 << 31) return Status::fail(DEC_ERR_ARG, "refined mesh too large");
    std::vector<double> fv(nf * dim);
    std::copy(c.verts.begin(), c.verts.end(), fv.begin());
    auto put = [&](int64_t v, double *m) {
        if (sphere) {
            double s = m[0] * m[0] + m[1] * m[1];
            s = s + m[2] * m[2];
            const double nrm = std::sqrt(s);
            for (int d = 0; d < 3; ++d) m[d] = m[d] / nrm;
        }
        for (int d = 0; d < dim; ++d) fv[v * dim + d] = m[d];
    };
    for (int64_t e = 0; e < E; ++e) {
        const double *pl = &c.verts[(int64_t)c.edges[2 * e] * dim];
        const double *ph = &c.verts[(int64_t)c.edges[2 * e + 1] * dim];
        double m1[3] = {0, 0, 0}, m2[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) {
            m1[d] = (2.0 * pl[d] + ph[d]) / 3.0;
            m2[d] = (pl[d] + 2.0 * ph[d]) / 3.0;
        }
        put(nc + 2 * e, m1);
        put(nc + 2 * e + 1, m2);
    }
    for (int64_t t = 0; t < T; ++t) {
        const double *pa = &c.verts[(int64_t)c.tris[3 * t] * dim];
        const double *pb = &c.verts[(int64_t)c.tris[3 * t + 1] * dim];
        const double *pc = &c.verts[(int64_t)c.tris[3 * t + 2] * dim];
        double m[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) m[d] = ((pa[d] + pb[d]) + pc[d]) / 3.0;
        put(nc + 2 * E + t, m);
    }
    // the point of triangle t's edge k next to its corner `corner`
    auto near = [&](int64_t t, int k, int32_t corner) {
        const int64_t e = c.tri_edges[3 * t + k];
        return (int32_t)(nc + 2 * e + (corner != c.edges[2 * e] ? 1 : 0));
    };
    std::vector<int32_t> ft(27 * T);
    for (int64_t t = 0; t < T; ++t) {
        const int32_t a = c.tris[3 * t], b = c.tris[3 * t + 1], cc = c.tris[3 * t + 2];
        const int32_t ab1 = near(t, 0, a), ab2 = near(t, 0, b), bc1 = near(t, 1, b), bc2 = near(t, 1, cc);
        const int32_t ca1 = near(t, 2, cc), ca2 = near(t, 2, a), m = (int32_t)(nc + 2 * E + t);
        const int32_t sub[9][3] = {{a, ab1, ca2},  {ab1, ab2, m},  {ab2, b, bc1},  {ca2, m, ca1},  {m, bc1, bc2},
                                   {ca1, bc2, cc}, {ab1, m, ca2},  {ab2, bc1, m},  {m, bc2, ca1}};
        for (int q = 0; q < 9; ++q)
            for (int k = 0; k < 3; ++k) ft[27 * t + 3 * q + k] = sub[q][k];
    }
    map_idx.assign(3 * nf, 0);
    map_w.assign(3 * nf, 0.0);
    const double third = 1.0 / 3.0, two_thirds = 2.0 / 3.0;
    for (int64_t v = 0; v < nc; ++v) {
        map_idx[3 * v] = map_idx[3 * v + 1] = map_idx[3 * v + 2] = (int32_t)v;
        map_w[3 * v] = 1.0;
    }
    for (int64_t e = 0; e < E; ++e) {
        const int32_t lo = c.edges[2 * e], hi = c.edges[2 * e + 1];
        for (int s2 = 0; s2 < 2; ++s2) {
            const int64_t v = nc + 2 * e + s2;
            map_idx[3 * v] = lo;
            map_idx[3 * v + 1] = hi;
            map_idx[3 * v + 2] = lo;
            map_w[3 * v] = s2 == 0 ? two_thirds : third;
            map_w[3 * v + 1] = s2 == 0 ? third : two_thirds;
        }
    }
    for (int64_t t = 0; t < T; ++t) {
        const int64_t v = nc + 2 * E + t;
        for (int k = 0; k < 3; ++k) {
            map_idx[3 * v + k] = c.tris[3 * t + k];
            map_w[3 * v + k] = third;
        }
    }
    return build_mesh(std::move(fv), dim, std::move(ft), f);
}

void hodge_stars(const HostMesh &m, std::vector<double> &star0, std::vector<double> &star1) {
    star0.assign(m.nv, 0.0);
    star1.assign(m.ne, 0.0);
    const int dim = m.dim;
    for (int64_t t = 0; t < m.nt; ++t) {
        double P[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int k = 0; k < 3; ++k)
            for (int d = 0; d < dim; ++d) P[k][d] = m.verts[(int64_t)m.tris[3 * t + k] * dim + d];
        for (int k = 0; k < 3; ++k) {
            // edge k joins corners k and k+1; the opposite corner is k+2
            const double *A = P[k], *B = P[(k + 1) % 3], *O = P[(k + 2) % 3];
            double u[3], w[3];
            for (int d = 0; d < 3; ++d) {
                u[d] = A[d] - O[d];
                w[d] = B[d] - O[d];
            }
            double dot = u[0] * w[0] + u[1] * w[1] + u[2] * w[2];
            double cr;
            if (dim == 2) {
                cr = std::fabs(u[0] * w[1] - u[1] * w[0]);
            } else {
                double c0 = u[1] * w[2] - u[2] * w[1];
                double c1 = u[2] * w[0] - u[0] * w[2];
                double c2 = u[0] * w[1] - u[1] * w[0];
                cr = std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
            }
            double cot = dot / cr;
            double l2 = 0.0;
            for (int d = 0; d < 3; ++d) l2 += (B[d] - A[d]) * (B[d] - A[d]);
            star1[m.tri_edges[3 * t + k]] += 0.5 * cot;
            double c = l2 * cot / 8.0;
            star0[m.tris[3 * t + k]] += c;
            star0[m.tris[3 * t + (k + 1) % 3]] += c;
        }
    }
}

std::vector<uint8_t> boundary_vertices(const HostMesh &m) {
    std::vector<uint8_t> cnt(m.ne, 0), bv(m.nv, 0);
    for (int64_t i = 0; i < 3 * m.nt; ++i) cnt[m.tri_edges[i]]++;
    for (int64_t e = 0; e < m.ne; ++e)
        if (cnt[e] == 1) {
            bv[m.edges[2 * e]] = 1;
            bv[m.edges[2 * e + 1]] = 1;
        }
    return bv;
}

}  // namespace decimpl
