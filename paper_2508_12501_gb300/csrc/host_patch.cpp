// Halo tiles for the tiled cycle kernels (DEC_FUSE_PATCH), built on the host.
//
// Between two visits of the coarse grid, a level's share of a V-cycle
// (Sec. 2.2.1: smoothing, residual and restriction on the way down;
// interpolation, correction and smoothing on the way up) reads only
// neighbours.  A thread block that holds every vertex within `depth` edges of
// the vertices it is responsible for ("rings") can therefore run all of those
// steps out of shared memory, recomputing the ring vertices' values itself.
// With the same operations in the same order the results are bitwise those of
// one kernel per step, and the level costs one launch per direction.
#include <algorithm>
#include <climits>
#include <numeric>

#include "host.h"

namespace decimpl {

namespace {

// Completes one tile whose ring 0 is g (loc[v] = position of v in g for every
// v in g, -1 elsewhere): adds rings 1..depth, the local ELL of rings
// 0..depth-1 and the header, appends everything to P and clears loc again.
Status finish_tile(const HostLevel &F, std::vector<int32_t> &loc, std::vector<int32_t> &g, int nown, int ncoarse,
                   int depth, HostPatch &P) {
    const int64_t nf = F.mesh.nv;
    const int K = F.K;
    int32_t n[kPatchMaxDepth + 1];
    n[0] = (int32_t)g.size();
    size_t lo = 0;
    for (int k = 1; k <= depth; ++k) {
        // ring k: the new neighbours of ring k-1 (rings below k-1 have theirs already)
        const size_t hi = g.size();
        for (size_t i = lo; i < hi; ++i)
            for (int s = 0; s < K; ++s) {
                const int32_t c = F.col[(size_t)s * nf + g[i]];
                if (loc[c] < 0) {
                    loc[c] = (int32_t)g.size();
                    g.push_back(c);
                }
            }
        lo = hi;
        n[k] = (int32_t)g.size();
    }
    for (int k = depth + 1; k <= kPatchMaxDepth; ++k) n[k] = n[depth];
    const int32_t m = n[depth - 1];
    if (P.gid.size() + g.size() > (size_t)INT_MAX || P.lcol.size() + (size_t)K * m > (size_t)INT_MAX)
        return Status::fail(DEC_ERR_ARG, "tiled cycle tables exceed 2^31 entries");
    const int32_t hdr[kPatchHdr] = {(int32_t)P.gid.size(), (int32_t)P.lcol.size(), nown, ncoarse,
                                    n[0], n[1], n[2], n[3]};
    P.hdr.insert(P.hdr.end(), hdr, hdr + kPatchHdr);
    for (int s = 0; s < K; ++s)
        for (int32_t i = 0; i < m; ++i) {
            const size_t o = (size_t)s * nf + g[i];
            const int32_t c = loc[F.col[o]];
            if (c < 0) return Status::fail(DEC_ERR_ARG, "tiled cycle: a ring vertex lost a neighbour");
            P.lcol.push_back(c);
            P.lw.push_back(F.w[o]);
        }
    P.gid.insert(P.gid.end(), g.begin(), g.end());
    P.cap = std::max(P.cap, (int)g.size());
    P.ntiles += 1;
    for (int32_t v : g) loc[v] = -1;
    return Status::ok();
}

}  // namespace

Status build_patches(const HostLevel &F, const HostMesh &coarse, const std::vector<int32_t> &parents, int chunk,
                     int depth_down, int depth_up, HostPatch &down, HostPatch &up) {
    const int64_t nc = coarse.nv, nf = F.mesh.nv;
    if (nc <= 0 || nf != nc + (int64_t)parents.size() / 2)
        return Status::fail(DEC_ERR_ARG, "tiled cycle: the level is not a binary subdivision of the coarser one");
    if (depth_down < 1 || depth_down > kPatchMaxDepth || depth_up < 1 || depth_up > kPatchMaxDepth)
        return Status::fail(DEC_ERR_ARG, "tiled cycle: 1 to 3 smoothing steps per direction");
    chunk = std::max(1, chunk);
    down = HostPatch();
    up = HostPatch();
    down.depth = depth_down;
    up.depth = depth_up;

    // coarse vertices in Z-order, cut into chunks
    std::vector<uint64_t> keys;
    morton_keys(coarse.verts.data(), nc, coarse.dim, keys);
    std::vector<int32_t> order(nc);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return keys[a] < keys[b]; });
    const int64_t ntiles = (nc + chunk - 1) / chunk;
    std::vector<int32_t> tile_of(nc);
    for (int64_t i = 0; i < nc; ++i) tile_of[order[i]] = (int32_t)(i / chunk);

    // midpoints owned by the tile of their first parent, in increasing id (counting sort)
    std::vector<int64_t> moff(ntiles + 1, 0);
    for (int64_t m = nc; m < nf; ++m) moff[tile_of[parents[2 * (m - nc)]] + 1] += 1;
    for (int64_t t = 0; t < ntiles; ++t) moff[t + 1] += moff[t];
    std::vector<int32_t> mids(nf - nc);
    {
        std::vector<int64_t> fill(moff.begin(), moff.end() - 1);
        for (int64_t m = nc; m < nf; ++m) mids[fill[tile_of[parents[2 * (m - nc)]]]++] = (int32_t)m;
    }

    std::vector<int32_t> loc(nf, -1), g;
    for (int64_t t = 0; t < ntiles; ++t) {
        const int64_t c0 = t * chunk, c1 = std::min<int64_t>(nc, c0 + chunk);
        auto push = [&](int32_t v) {
            if (loc[v] < 0) {
                loc[v] = (int32_t)g.size();
                g.push_back(v);
            }
        };
        // owned: the fine copies of the tile's coarse vertices (fine id = coarse id), then its midpoints
        g.clear();
        for (int64_t i = c0; i < c1; ++i) push(order[i]);
        for (int64_t i = moff[t]; i < moff[t + 1]; ++i) push(mids[i]);
        const int nown = (int)g.size(), ncoarse = (int)(c1 - c0);
        const std::vector<int32_t> owned(g.begin(), g.end());
        // down ring 0: the rest of the coarse vertices' fine closed neighbourhoods
        for (int64_t i = c0; i < c1; ++i)
            for (int s = 0; s < F.K; ++s) push(F.col[(size_t)s * nf + order[i]]);
        Status st = finish_tile(F, loc, g, nown, ncoarse, depth_down, down);
        if (!st.good()) return st;
        // up ring 0: the owned vertices
        g.clear();
        for (int32_t v : owned) push(v);
        st = finish_tile(F, loc, g, nown, 0, depth_up, up);
        if (!st.good()) return st;
    }
    return Status::ok();
}

}  // namespace decimpl
