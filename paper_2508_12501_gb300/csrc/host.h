// Internal host-side data structures of libdec (mesh, hierarchy levels).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "dec.h"

namespace decimpl {

// Thread-local error message set by every failing entry point.
void set_error(const std::string &msg);

struct Status {
    int code = DEC_OK;
    std::string msg;
    static Status ok() { return Status(); }
    static Status fail(int c, const std::string &m) {
        Status s;
        s.code = c;
        s.msg = m;
        return s;
    }
    bool good() const { return code == DEC_OK; }
};

// Embedded 2-simplicial complex: points, triangles, canonical edges.
struct HostMesh {
    int dim = 2;
    int64_t nv = 0, ne = 0, nt = 0;
    std::vector<double> verts;      // [nv * dim]
    std::vector<int32_t> tris;      // [nt * 3]
    std::vector<int32_t> edges;     // [ne * 2] (lo, hi), lexicographic
    std::vector<int32_t> tri_edges; // [nt * 3] edge of (v0v1, v1v2, v2v0)
};

// Validates (Sec. 2.1 definition, plus at most two triangles per edge) and
// enumerates the canonical edges.
Status build_mesh(std::vector<double> verts, int dim, std::vector<int32_t> tris, HostMesh &out);

// One 1->4 midpoint subdivision; `parents` of fine vertex nc + e is coarse edge e.
// One 1->9 (cubic) subdivision: coarse edge e gets n_c + 2e at (2 x_lo + x_hi)/3
// and n_c + 2e + 1 at (x_lo + 2 x_hi)/3, triangle t its centroid n_c + 2E + t.
// map_idx / map_w (3 per fine vertex, row-major) receive the geometric map:
// the coarse vertices and barycentric weights of each fine vertex (padding:
// weight 0 on the first entry's vertex).
Status subdivide_cubic(const HostMesh &coarse, bool sphere, HostMesh &fine, std::vector<int32_t> &map_idx,
                       std::vector<double> &map_w);

// One 1->4 subdivision; with morton the new vertices are numbered in Z-order
// of their coordinates, else in coarse edge order.  parents (optional)
// receives the coarse edge endpoints of each new vertex, in new-vertex order.
Status subdivide(const HostMesh &coarse, bool sphere, bool morton, HostMesh &fine,
                 std::vector<int32_t> *parents = nullptr);

// Circumcentric diagonal Hodge stars (cotangent formulas).
void hodge_stars(const HostMesh &m, std::vector<double> &star0, std::vector<double> &star1);

// Vertices on edges that lie in exactly one triangle.
std::vector<uint8_t> boundary_vertices(const HostMesh &m);

// One level of the hierarchy, host copy.
struct HostLevel {
    HostMesh mesh;
    std::vector<double> star0, star1;
    std::vector<uint8_t> free_;      // 1 = unknown
    int K = 0;                       // ELL width (max valence)
    std::vector<int32_t> col;        // [K * nv] slot-major; padding: col = row
    std::vector<int32_t> slot_edge;  // [K * nv] edge id of each slot, -1 = padding
    std::vector<double> w;           // [K * nv] *1_e / *0_v, 0 on Dirichlet rows
    double lmax = 0.0;
    std::vector<int32_t> colors;
    int ncolors = 0;
};

}  // namespace decimpl

namespace decimpl {

// The whole hierarchy on the host.  levels[0] is the coarsest level used.
struct HostHierarchy {
    int bc = DEC_BC_DIRICHLET;
    bool sphere = false;
    dec_mg_opts opts{};
    std::vector<HostLevel> levels;
    std::vector<std::vector<int32_t>> parents;  // parents[l]: level-l edges = parents of level l+1 midpoints
    bool mapped = false;                        // transfers by the general maps below instead of parents:
                                                // cubic 1->9 subdivision or caller-supplied geometric maps
    std::vector<std::vector<int32_t>> map_idx;  // map_idx[l], map_w[l]: the map from level l to l+1,
    std::vector<std::vector<double>> map_w;     // 3 (coarse vertex, weight) pairs per level-(l+1) vertex
    std::vector<double> G;                      // [n0 * n0] coarse solution operator, row-major
};

Status build_hierarchy(const HostMesh &base, int nsub, int nlevels, int bc, bool sphere, bool morton, bool cubic,
                       const double *star1_scale, const dec_mg_opts &opts, HostHierarchy &H);

// A hierarchy on caller-given meshes (levels[0] coarsest) with caller-given
// geometric maps between consecutive levels: maps_idx[l], maps_w[l] hold three
// (level-l vertex, weight) slots per level-(l+1) vertex (Sec. 2.2, M(f)).
Status build_hierarchy_maps(const std::vector<const HostMesh *> &meshes,
                            const std::vector<const int32_t *> &maps_idx, const std::vector<const double *> &maps_w,
                            int bc, const double *star1_scale, const dec_mg_opts &opts, HostHierarchy &H);

// Rebuild ELL weights of one level from its (possibly new) star1.
Status level_weights(HostLevel &L, int bc);

// lambda_max(D^-1 L) by power iteration on the free vertices.
double power_lmax(const HostLevel &L, int iters);

// Z-order keys of points [n x dim] on their bounding box (host_mesh.cpp).
void morton_keys(const double *pts, int64_t n, int dim, std::vector<uint64_t> &keys);

// Halo tiles of one level of binary subdivision for the tiled cycle kernels
// (DEC_FUSE_PATCH).  Per tile, kPatchHdr ints:
//   [0] offset of its local vertices in gid, [1] offset of its local ELL in
//   lcol / lw, [2] owned vertices (locals 0 .. nown-1, written back),
//   [3] coarse rows (down tiles: locals 0 .. ncoarse-1 are the fine copies of
//   the tile's coarse vertices), [4 + k] |ring 0 .. ring k| for k = 0..3
//   (cumulative; entries past the depth repeat the last).
// Locals are numbered ring by ring.  The local ELL covers the rows of rings
// 0 .. depth-1 (m = entry [4 + depth - 1]): slot k of local row i at
// [row offset + k m + i], its column a local index, its weight the level's.
constexpr int kPatchHdr = 8;
constexpr int kPatchMaxDepth = 3;
struct HostPatch {
    int ntiles = 0, depth = 0;
    int cap = 0;                 // most locals of one tile
    std::vector<int32_t> hdr;    // [ntiles * kPatchHdr]
    std::vector<int32_t> gid;    // local -> level vertex, all tiles
    std::vector<int32_t> lcol;   // local ELL columns, all tiles
    std::vector<double> lw;      // local ELL weights (the level's w), all tiles
};

// Down tiles: chunks of `chunk` coarse vertices in Z-order; ring 0 is the
// fine closed neighbourhood of those vertices (what the restriction reads),
// rings 1..depth_down what the pre-smoothing steps and the residual read.
// Up tiles: ring 0 is the fine vertices the matching down tile owns (its
// coarse vertices' fine copies and the midpoints whose first parent is one of
// them: a partition of the fine level), rings 1..depth_up what the
// post-smoothing steps read.  parents: coarse edge endpoints of each midpoint.
Status build_patches(const HostLevel &F, const HostMesh &coarse, const std::vector<int32_t> &parents, int chunk,
                     int depth_down, int depth_up, HostPatch &down, HostPatch &up);

}  // namespace decimpl
