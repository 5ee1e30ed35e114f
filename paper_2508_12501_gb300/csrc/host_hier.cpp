// Host-side construction of the multigrid hierarchy: per-level operator in
// ELL form, lambda_max estimates, greedy colouring and the coarsest-level
// dense solution operator.
//
// The operator is rediscretized on each level (Sec. 3.1.1, last paragraph):
// L = *0^-1 d0^T *1 d0 with (L x)_v = sum over edges (v,w) of
// (*1_e / *0_v) (x_v - x_w).  Each row stores its neighbours in increasing
// vertex order in K = max-valence slots; unused slots point at the row
// itself with weight 0.  Dirichlet rows keep their columns but get weight 0.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>

#include "host.h"

namespace decimpl {

static Status build_ell(HostLevel &L) {
    const HostMesh &m = L.mesh;
    const int64_t n = m.nv;
    std::vector<int32_t> deg(n, 0);
    for (int64_t e = 0; e < m.ne; ++e) {
        deg[m.edges[2 * e]]++;
        deg[m.edges[2 * e + 1]]++;
    }
    int K = *std::max_element(deg.begin(), deg.end());
    if (K > 32) return Status::fail(DEC_ERR_MESH, "vertex valence above 32");
    L.K = K;
    L.col.assign((size_t)K * n, 0);
    L.slot_edge.assign((size_t)K * n, -1);
    for (int64_t v = 0; v < n; ++v)
        for (int k = 0; k < K; ++k) L.col[(size_t)k * n + v] = (int32_t)v;
    // edges are lexicographic in (lo, hi): appending in edge order lists each
    // vertex's lower neighbours (ascending) before its higher ones (ascending)
    std::vector<int32_t> fill(n, 0);
    for (int64_t e = 0; e < m.ne; ++e) {
        int32_t a = m.edges[2 * e], b = m.edges[2 * e + 1];
        size_t sa = (size_t)fill[a]++ * n + a;
        size_t sb = (size_t)fill[b]++ * n + b;
        L.col[sa] = b;
        L.slot_edge[sa] = (int32_t)e;
        L.col[sb] = a;
        L.slot_edge[sb] = (int32_t)e;
    }
    return Status::ok();
}

Status level_weights(HostLevel &L, int bc) {
    const int64_t n = L.mesh.nv;
    const int K = L.K;
    L.w.assign((size_t)K * n, 0.0);
    for (int64_t v = 0; v < n; ++v) {
        if (!L.free_[v]) continue;
        double diag = 0.0;
        for (int k = 0; k < K; ++k) {
            int32_t e = L.slot_edge[(size_t)k * n + v];
            if (e < 0) continue;
            double w = L.star1[e] / L.star0[v];
            L.w[(size_t)k * n + v] = w;
            diag += w;
        }
        if (!(diag > 0.0) || !std::isfinite(diag))
            return Status::fail(DEC_ERR_MESH, "a free vertex has a non-positive or non-finite Laplacian diagonal");
    }
    (void)bc;
    return Status::ok();
}

double power_lmax(const HostLevel &L, int iters) {
    const int64_t n = L.mesh.nv;
    const int K = L.K;
    std::vector<double> inv(n, 0.0), v(n), w(n);
    for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int k = 0; k < K; ++k) d += L.w[(size_t)k * n + i];
        inv[i] = L.free_[i] ? 1.0 / d : 0.0;
        uint64_t h = ((uint64_t)i * 2654435761ull) % 4294967296ull;
        v[i] = L.free_[i] ? (double)h / 4294967296.0 - 0.5 : 0.0;
    }
    double lam = 0.0;
    for (int it = 0; it < iters; ++it) {
        double nv2 = 0.0, nw2 = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) {
                size_t sl = (size_t)k * n + i;
                s += L.w[sl] * (v[i] - v[L.col[sl]]);
            }
            w[i] = inv[i] * s;
            nv2 += v[i] * v[i];
            nw2 += w[i] * w[i];
        }
        double nw = std::sqrt(nw2);
        lam = nw / std::sqrt(nv2);
        for (int64_t i = 0; i < n; ++i) v[i] = w[i] / nw;
    }
    return lam;
}

static void greedy_colour(HostLevel &L) {
    const int64_t n = L.mesh.nv;
    L.colors.assign(n, -1);
    int ncol = 0;
    std::vector<int64_t> seen(64, -1);
    for (int64_t v = 0; v < n; ++v) {
        for (int k = 0; k < L.K; ++k) {
            int32_t u = L.col[(size_t)k * n + v];
            if (u < v) seen[L.colors[u]] = v;
        }
        int c = 0;
        while (seen[c] == v) ++c;
        L.colors[v] = c;
        ncol = std::max(ncol, c + 1);
    }
    L.ncolors = ncol;
}

// LU with partial pivoting of a dense row-major n x n matrix, solving for
// `nrhs` right-hand sides stored row-major in B ([n * nrhs]).
static bool dense_solve(std::vector<double> A, int n, std::vector<double> &B, int nrhs) {
    std::vector<int> piv(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = std::fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(A[(size_t)i * n + k]) > best) {
                best = std::fabs(A[(size_t)i * n + k]);
                p = i;
            }
        if (!(best > 0.0)) return false;
        if (p != k) {
            for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
            for (int j = 0; j < nrhs; ++j) std::swap(B[(size_t)k * nrhs + j], B[(size_t)p * nrhs + j]);
        }
        double inv = 1.0 / A[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            double f = A[(size_t)i * n + k] * inv;
            if (f == 0.0) continue;
            A[(size_t)i * n + k] = f;
            for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
            for (int j = 0; j < nrhs; ++j) B[(size_t)i * nrhs + j] -= f * B[(size_t)k * nrhs + j];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double inv = 1.0 / A[(size_t)k * n + k];
        for (int j = 0; j < nrhs; ++j) {
            double s = B[(size_t)k * nrhs + j];
            for (int i = k + 1; i < n; ++i) s -= A[(size_t)k * n + i] * B[(size_t)i * nrhs + j];
            B[(size_t)k * nrhs + j] = s * inv;
        }
    }
    return true;
}

// Coarsest-level solution operator G with x = G b solving L x = b:
// Dirichlet -- interior block A_II^-1 diag(*0_I), zero elsewhere;
// gauge     -- (I - 1 m^T / sum m) (A + m m^T / sum m)^-1 diag(*0), m = *0.
static Status coarse_operator(const HostLevel &L, int bc, std::vector<double> &G) {
    const HostMesh &m = L.mesh;
    const int n = (int)m.nv;
    if (n > 4096) return Status::fail(DEC_ERR_MESH, "coarsest level has more than 4096 vertices");
    std::vector<double> A((size_t)n * n, 0.0);
    for (int64_t e = 0; e < m.ne; ++e) {
        int a = m.edges[2 * e], b = m.edges[2 * e + 1];
        double s = L.star1[e];
        A[(size_t)a * n + a] += s;
        A[(size_t)b * n + b] += s;
        A[(size_t)a * n + b] -= s;
        A[(size_t)b * n + a] -= s;
    }
    G.assign((size_t)n * n, 0.0);
    if (bc == DEC_BC_DIRICHLET) {
        std::vector<int> idx;
        for (int v = 0; v < n; ++v)
            if (L.free_[v]) idx.push_back(v);
        const int ni = (int)idx.size();
        if (ni == 0) return Status::ok();
        std::vector<double> Aii((size_t)ni * ni), B((size_t)ni * ni, 0.0);
        for (int i = 0; i < ni; ++i) {
            for (int j = 0; j < ni; ++j) Aii[(size_t)i * ni + j] = A[(size_t)idx[i] * n + idx[j]];
            B[(size_t)i * ni + i] = L.star0[idx[i]];
        }
        if (!dense_solve(Aii, ni, B, ni)) return Status::fail(DEC_ERR_MESH, "singular coarsest operator");
        for (int i = 0; i < ni; ++i)
            for (int j = 0; j < ni; ++j) G[(size_t)idx[i] * n + idx[j]] = B[(size_t)i * ni + j];
        return Status::ok();
    }
    double s = 0.0;
    for (int v = 0; v < n; ++v) s += L.star0[v];
    std::vector<double> K(A), B((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) K[(size_t)i * n + j] += L.star0[i] * L.star0[j] / s;
        B[(size_t)i * n + i] = L.star0[i];
    }
    if (!dense_solve(K, n, B, n)) return Status::fail(DEC_ERR_MESH, "singular coarsest operator");
    std::vector<double> mean(n, 0.0);  // m^T X / s per column
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) mean[j] += L.star0[i] * B[(size_t)i * n + j];
    for (int j = 0; j < n; ++j) mean[j] /= s;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) G[(size_t)i * n + j] = B[(size_t)i * n + j] - mean[j];
    return Status::ok();
}

// One level: Hodge stars (scaled *1 when star1_scale is given), the free
// mask, the ELL operator, lambda_max and the greedy colouring.
static Status make_level(const HostMesh &mesh, int bc, const double *star1_scale, const dec_mg_opts &opts,
                         HostLevel &L) {
    L.mesh = mesh;
    hodge_stars(L.mesh, L.star0, L.star1);
    if (star1_scale)
        for (int64_t e = 0; e < L.mesh.ne; ++e) L.star1[e] *= star1_scale[e];
    if (bc == DEC_BC_DIRICHLET) {
        L.free_ = boundary_vertices(L.mesh);
        for (auto &f : L.free_) f = !f;
    } else {
        L.free_.assign(L.mesh.nv, 1);
    }
    Status st = build_ell(L);
    if (!st.good()) return st;
    st = level_weights(L, bc);
    if (!st.good()) return st;
    L.lmax = power_lmax(L, opts.power_iters);
    greedy_colour(L);
    return Status::ok();
}

Status build_hierarchy(const HostMesh &base, int nsub, int nlevels, int bc, bool sphere, bool morton, bool cubic,
                       const double *star1_scale, const dec_mg_opts &opts, HostHierarchy &H) {
    if (nsub < 0 || nlevels < 1 || nlevels > nsub + 1 || nlevels > 16)
        return Status::fail(DEC_ERR_ARG, "nlevels must be in 1..min(nsub+1, 16)");
    if (bc != DEC_BC_DIRICHLET && bc != DEC_BC_GAUGE) return Status::fail(DEC_ERR_ARG, "bad boundary condition");
    H.bc = bc;
    H.sphere = sphere;
    H.opts = opts;
    H.levels.clear();
    H.parents.clear();
    H.mapped = cubic;  // cubic subdivision transfers by its geometric map
    H.map_idx.clear();
    H.map_w.clear();
    const int first = nsub + 1 - nlevels;
    HostMesh cur = base;
    for (int i = 0; i <= nsub; ++i) {
        if (i > 0) {
            HostMesh fine;
            if (cubic) {
                std::vector<int32_t> mi;
                std::vector<double> mw;
                Status st = subdivide_cubic(cur, sphere, fine, mi, mw);
                if (!st.good()) return st;
                if (i > first) {
                    H.map_idx.push_back(std::move(mi));
                    H.map_w.push_back(std::move(mw));
                }
            } else {
                std::vector<int32_t> par;
                Status st = subdivide(cur, sphere, morton, fine, &par);
                if (!st.good()) return st;
                if (i > first) H.parents.push_back(std::move(par));
            }
            cur = std::move(fine);
        }
        if (i < first) continue;
        HostLevel L;
        Status st = make_level(cur, bc, i == nsub ? star1_scale : nullptr, opts, L);
        if (!st.good()) return st;
        H.levels.push_back(std::move(L));
    }
    return coarse_operator(H.levels[0], bc, H.G);
}

Status build_hierarchy_maps(const std::vector<const HostMesh *> &meshes,
                            const std::vector<const int32_t *> &maps_idx, const std::vector<const double *> &maps_w,
                            int bc, const double *star1_scale, const dec_mg_opts &opts, HostHierarchy &H) {
    const int nl = (int)meshes.size();
    if (nl < 1 || nl > 16) return Status::fail(DEC_ERR_ARG, "nlevels must be in 1..16");
    if ((int)maps_idx.size() != nl - 1 || (int)maps_w.size() != nl - 1)
        return Status::fail(DEC_ERR_ARG, "one map per pair of consecutive levels");
    if (bc != DEC_BC_DIRICHLET && bc != DEC_BC_GAUGE) return Status::fail(DEC_ERR_ARG, "bad boundary condition");
    H.bc = bc;
    H.sphere = false;
    H.opts = opts;
    H.levels.clear();
    H.parents.clear();
    H.mapped = true;
    H.map_idx.clear();
    H.map_w.clear();
    for (int l = 0; l + 1 < nl; ++l) {
        // M(f) of Sec. 2.2: each fine vertex's image has barycentric coordinates in one
        // coarse triangle, so its weights are finite, sum to 1, and name coarse vertices
        const int64_t nf = meshes[l + 1]->nv, nc = meshes[l]->nv;
        if (!maps_idx[l] || !maps_w[l]) return Status::fail(DEC_ERR_ARG, "null map");
        std::vector<int32_t> mi(maps_idx[l], maps_idx[l] + 3 * nf);
        std::vector<double> mw(maps_w[l], maps_w[l] + 3 * nf);
        std::vector<uint8_t> hit(nc, 0);
        for (int64_t v = 0; v < nf; ++v) {
            double sum = 0.0;
            for (int q = 0; q < 3; ++q) {
                const int32_t c = mi[3 * v + q];
                const double w = mw[3 * v + q];
                if (c < 0 || c >= nc || !std::isfinite(w))
                    return Status::fail(DEC_ERR_ARG, "map " + std::to_string(l) + ": vertex " + std::to_string(v) +
                                                         " has a coarse index out of range or a non-finite weight");
                sum += w;
                if (w != 0.0) hit[c] = 1;
            }
            if (!(std::fabs(sum - 1.0) <= 1e-9))
                return Status::fail(DEC_ERR_ARG, "map " + std::to_string(l) + ": the weights of vertex " +
                                                     std::to_string(v) + " do not sum to 1");
        }
        for (int64_t c = 0; c < nc; ++c)
            if (!hit[c])
                return Status::fail(DEC_ERR_ARG, "map " + std::to_string(l) + ": coarse vertex " + std::to_string(c) +
                                                     " carries no weight (its restriction row would be empty)");
        H.map_idx.push_back(std::move(mi));
        H.map_w.push_back(std::move(mw));
    }
    for (int l = 0; l < nl; ++l) {
        HostLevel L;
        Status st = make_level(*meshes[l], bc, l == nl - 1 ? star1_scale : nullptr, opts, L);
        if (!st.good()) return st;
        H.levels.push_back(std::move(L));
    }
    return coarse_operator(H.levels[0], bc, H.G);
}

}  // namespace decimpl
