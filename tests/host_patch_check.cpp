// Host-side check of the halo tiles (host_patch.cpp), compiled and run by
// tests/test_host_patch.py with no GPU: builds a hierarchy on the mesh given
// on standard input, tiles every level above the coarsest and checks what the
// tiled kernels rely on:
//   - the owned vertices of the tiles partition the level, the down tiles'
//     coarse vertices partition the coarser level, and each down tile's first
//     ncoarse locals are its coarse vertices' fine copies;
//   - ring 0 is the owned set (up) or the coarse vertices' fine closed
//     neighbourhoods (down), and ring k+1 is exactly the neighbours of rings
//     0..k not in them (so every neighbour a phase reads is local);
//   - every local ELL slot names the local copy of the level's column.
// Input: nv dim nt sphere nsub nlevels bc chunk depth_down depth_up, then the
// vertex coordinates and the triangles.  Prints "ok <tiles per level>" or the
// first violation, exit status 1.
#include <cstdio>
#include <set>
#include <string>
#include <vector>

#include "host.h"

using namespace decimpl;

static int bad(const std::string &what) {
    std::printf("violation: %s\n", what.c_str());
    return 1;
}

static int check(const HostLevel &F, int64_t nc, const HostPatch &P, bool down, std::vector<int> &owner) {
    const int64_t nf = F.mesh.nv;
    const int K = F.K;
    std::vector<int> cowner(nc, -1);
    for (int t = 0; t < P.ntiles; ++t) {
        const int32_t *h = &P.hdr[(size_t)t * kPatchHdr];
        const int32_t loc_off = h[0], row_off = h[1], nown = h[2], ncoarse = h[3];
        const int32_t *n = h + 4;
        const int depth = P.depth;
        const int32_t cnt = n[depth], m = n[depth - 1];
        if (cnt > P.cap || nown > n[0] || ncoarse > nown) return bad("tile counts");
        const int32_t *g = &P.gid[loc_off];
        std::vector<int32_t> loc(nf, -1);
        for (int32_t i = 0; i < cnt; ++i) {
            if (g[i] < 0 || g[i] >= nf || loc[g[i]] >= 0) return bad("local ids");
            loc[g[i]] = i;
        }
        // ownership
        for (int32_t i = 0; i < nown; ++i) {
            if (down) {
                if (owner[g[i]] >= 0) return bad("a fine vertex owned twice");
                owner[g[i]] = t;
            } else if (owner[g[i]] != t) {
                return bad("up tile owns other vertices than its down tile");
            }
        }
        if (down) {
            for (int32_t j = 0; j < ncoarse; ++j) {
                if (g[j] >= nc || cowner[g[j]] >= 0) return bad("coarse vertices");
                cowner[g[j]] = t;
            }
            // ring 0: the coarse vertices' fine closed neighbourhoods
            std::set<int32_t> r0;
            for (int32_t j = 0; j < ncoarse; ++j) {
                r0.insert(g[j]);
                for (int s = 0; s < K; ++s) r0.insert(F.col[(size_t)s * nf + g[j]]);
            }
            if ((int32_t)r0.size() != n[0]) return bad("down ring 0 size");
            for (int32_t i = 0; i < n[0]; ++i)
                if (!r0.count(g[i])) return bad("down ring 0 members");
        } else if (n[0] != nown) {
            return bad("up ring 0 is not the owned set");
        }
        // ring k+1: the neighbours of rings 0..k outside them
        for (int k = 0; k < depth; ++k) {
            std::set<int32_t> nxt;
            for (int32_t i = 0; i < n[k]; ++i)
                for (int s = 0; s < K; ++s) {
                    const int32_t c = F.col[(size_t)s * nf + g[i]];
                    if (loc[c] < 0) return bad("a neighbour of an inner ring is not local");
                    if (loc[c] >= n[k]) nxt.insert(c);
                }
            if ((int32_t)nxt.size() != n[k + 1] - n[k]) return bad("ring size");
            for (int32_t i = n[k]; i < n[k + 1]; ++i)
                if (!nxt.count(g[i])) return bad("ring members");
        }
        // local ELL
        for (int s = 0; s < K; ++s)
            for (int32_t i = 0; i < m; ++i) {
                const int32_t lc = P.lcol[(size_t)row_off + (size_t)s * m + i];
                if (lc < 0 || lc >= cnt || g[lc] != F.col[(size_t)s * nf + g[i]]) return bad("local column");
            }
    }
    if (down) {
        for (int64_t v = 0; v < nf; ++v)
            if (owner[v] < 0) return bad("a fine vertex without owner");
        for (int64_t c = 0; c < nc; ++c)
            if (cowner[c] < 0) return bad("a coarse vertex in no tile");
    }
    return 0;
}

int main() {
    int64_t nv, nt;
    int dim, sphere, nsub, nlevels, bc, chunk, dd, du;
    if (std::scanf("%lld %d %lld %d %d %d %d %d %d %d", (long long *)&nv, &dim, (long long *)&nt, &sphere, &nsub,
                   &nlevels, &bc, &chunk, &dd, &du) != 10)
        return bad("input header");
    std::vector<double> verts((size_t)nv * dim);
    std::vector<int32_t> tris((size_t)nt * 3);
    for (auto &x : verts)
        if (std::scanf("%lf", &x) != 1) return bad("input vertices");
    for (auto &t : tris)
        if (std::scanf("%d", &t) != 1) return bad("input triangles");
    HostMesh base;
    Status st = build_mesh(verts, dim, tris, base);
    if (!st.good()) return bad(st.msg);
    dec_mg_opts o;
    dec_mg_default_opts(&o);
    HostHierarchy H;
    st = build_hierarchy(base, nsub, nlevels, bc, sphere != 0, false, false, nullptr, o, H);
    if (!st.good()) return bad(st.msg);
    std::string tiles;
    for (size_t l = 1; l < H.levels.size(); ++l) {
        HostPatch down, up;
        st = build_patches(H.levels[l], H.levels[l - 1].mesh, H.parents[l - 1], chunk, dd, du, down, up);
        if (!st.good()) return bad(st.msg);
        std::vector<int> owner(H.levels[l].mesh.nv, -1);
        if (check(H.levels[l], H.levels[l - 1].mesh.nv, down, true, owner)) return 1;
        if (check(H.levels[l], H.levels[l - 1].mesh.nv, up, false, owner)) return 1;
        tiles += " " + std::to_string(down.ntiles);
    }
    std::printf("ok%s\n", tiles.c_str());
    return 0;
}
