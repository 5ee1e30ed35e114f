// Batched solves: many right-hand sides on many hierarchies of uneven size,
// advanced together.  The right-hand sides of every hierarchy (entries that
// share a hierarchy are merged) are split into groups of k (a power of two)
// whose vectors are interleaved, value j of vertex v at [v * k + j], so one
// gather of a neighbour reads k contiguous values and one read of the
// operator serves the whole group.  Every operation of the cycle is one
// launch over all groups of all meshes: a tile list maps each block to
// (group level, item range), items being (vertex, right-hand side) pairs.
// Operations are aligned by depth below each hierarchy's finest level, so the
// number of launches per cycle follows the deepest hierarchy, not the number
// of meshes.
//
// Solvers (Sec. 3.1.2, with the mixed-precision pattern): FP32 cycles
// (Sec. 2.2.1 transfers, Jacobi or Chebyshev smoothing, dense coarsest solve)
// inside an FP64 outer iteration per right-hand side -- flexible MG-PCG in the
// *0 inner product (FP64 residual, dot products, updates and gauge
// projection), or iterative refinement x += C(b - L x) -- until every
// right-hand side satisfies ||b - L x||_2 / ||b||_2 <= tol.  The loop runs on
// the device as a CUDA graph with a while node; a group whose right-hand sides
// have all converged drops out of the loop's kernels (its blocks return at
// once) while the others go on.  The adjoint solve L mu = *0^-1 dJ/du shares
// the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "mg_device.h"

using decimpl::Status;
using namespace decimpl;
using decdev::pdl_prologue;
using decdev::Scal;
using decdev::skipped;

namespace {

constexpr int kBMaxNu = 8;

// One level of one right-hand-side group.
struct BLevel {
    int n, K, k, kshift;
    const int32_t *col;
    const float *w;
    const float *s0;
    const int2 *par;
    float *x[2], *d[2], *r, *b;
    int res_idx;  // buffer holding this level's cycle result
    float cpre[kBMaxNu], epre[kBMaxNu], cpost[kBMaxNu], epost[kBMaxNu];
    const float *G;  // level 0: dense solution operator
    // finest level: the FP64 outer iteration (refinement or MG-PCG)
    const double *w64;
    const uint8_t *freev;
    const double *star0;
    double *ox, *orr, *ob;
    double *op, *oq, *ozo;  // MG-PCG: search direction, L p, previous shifted preconditioned vector
    int rhs_base;     // index of this group's first right-hand side in the batch
    int gauge;
    double s0sum;     // sum of *0 over free vertices
    int group;        // index of the group
    const int *live;  // the group's flag: 0 once every right-hand side of the group has converged
    int *gpend;       // the group's count of right-hand sides still iterating (k_b_finalize)
};

// A group that has converged skips the loop's kernels: its blocks return at
// once.  (The flag changes only in k_b_finalize's last block, between passes.)
__device__ __forceinline__ bool group_done(const BLevel &L) { return *L.live == 0; }

struct BTile {
    int lev;          // index into the level descriptor array
    int begin, end;   // item range [begin, end), aligned to whole vertices
};

// ---------------------------------------------------------------------------
// kernels: block b works on tiles[b]; item i of a level is the interleaved
// vector index, i.e. vertex i >> kshift, right-hand side i & (k-1).
// ---------------------------------------------------------------------------

// Per-block path choice: groups whose width k is a multiple of 4 use 16-byte
// loads of 4 adjacent right-hand sides (one ELL row read per 4 values);
// other groups use one value per thread.  A tile belongs to one level, so the
// branch is uniform across the block.
template <int VW> struct VecT;
template <> struct VecT<1> {
    float v[1];
};
template <> struct VecT<4> {
    float v[4];
};

template <int VW>
__device__ __forceinline__ VecT<VW> vld(const float *p, int i) {
    VecT<VW> r;
    if constexpr (VW == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p + i);
        r.v[0] = q.x;
        r.v[1] = q.y;
        r.v[2] = q.z;
        r.v[3] = q.w;
    } else {
        r.v[0] = p[i];
    }
    return r;
}

template <int VW>
__device__ __forceinline__ void vst(float *p, int i, const VecT<VW> &a) {
    if constexpr (VW == 4)
        *reinterpret_cast<float4 *>(p + i) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
    else
        p[i] = a.v[0];
}

// s = sum_q w_q (x_i - x_col(q)), d = sum_q w_q for VW adjacent right-hand sides.
// Rows of 6 slots (interior valence 6) issue all their table loads, then all
// six neighbour gathers, before the first FMA: the gathers are in flight
// together.  The slot order of the sums is the same either way.
template <int VW>
__device__ __forceinline__ void brow(const BLevel &L, int v, int j, const float *x, VecT<VW> &s, float &d) {
    const VecT<VW> xi = vld<VW>(x, (v << L.kshift) + j);
#pragma unroll
    for (int c = 0; c < VW; ++c) s.v[c] = 0.f;
    d = 0.f;
    if (L.K == 6) {
        const int n = L.n, ks = L.kshift;
        int cq[6];
        float wq[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            cq[q] = __ldg(L.col + (size_t)q * n + v);
            wq[q] = __ldg(L.w + (size_t)q * n + v);
        }
        VecT<VW> xn[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) xn[q] = vld<VW>(x, (cq[q] << ks) + j);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
#pragma unroll
            for (int c = 0; c < VW; ++c) s.v[c] = fmaf(wq[q], xi.v[c] - xn[q].v[c], s.v[c]);
            d += wq[q];
        }
        return;
    }
    for (int q = 0; q < L.K; ++q) {
        const size_t o = (size_t)q * L.n + v;
        const float wk = __ldg(L.w + o);
        const VecT<VW> xn = vld<VW>(x, (__ldg(L.col + o) << L.kshift) + j);
#pragma unroll
        for (int c = 0; c < VW; ++c) s.v[c] = fmaf(wk, xi.v[c] - xn.v[c], s.v[c]);
        d += wk;
    }
}

template <int VW>
__device__ __forceinline__ void smooth0_body(const BLevel &L, const BTile &t, float e, int dout) {
    for (int i = t.begin + VW * threadIdx.x; i < t.end; i += VW * blockDim.x) {
        const int v = i >> L.kshift;
        float d = 0.f;
        for (int q = 0; q < L.K; ++q) d += __ldg(L.w + (size_t)q * L.n + v);
        const VecT<VW> bb = vld<VW>(L.b, i);
        VecT<VW> val;
#pragma unroll
        for (int c = 0; c < VW; ++c) val.v[c] = d != 0.f ? e * (bb.v[c] / d) : 0.f;
        vst<VW>(L.x[0], i, val);
        if (dout) vst<VW>(L.d[0], i, val);
    }
}

__global__ void k_b_smooth0(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, int cheb, float omega,
                            int dout, const int *skip, int ntiles) {
    pdl_prologue();
    if (skipped(skip)) return;
    for (int tb = blockIdx.x; tb < ntiles; tb += gridDim.x) {
        const BTile t = tiles[tb];
        const BLevel &L = lv[t.lev];
        if (group_done(L)) continue;
        const float e = cheb ? L.epre[0] : omega;
        if ((L.k & 3) == 0)
            smooth0_body<4>(L, t, e, dout);
        else
            smooth0_body<1>(L, t, e, dout);
    }
}

template <int VW>
__device__ __forceinline__ void smooth_body(const BLevel &L, const BTile &t, float e, float c, int src, int din,
                                            int dout) {
    const int dst = 1 - src;
    const float *xs = L.x[src];
    for (int i = t.begin + VW * threadIdx.x; i < t.end; i += VW * blockDim.x) {
        const int v = i >> L.kshift, j = i & (L.k - 1);
        VecT<VW> s;
        float d;
        brow<VW>(L, v, j, xs, s, d);
        const VecT<VW> bb = vld<VW>(L.b, i), xo = vld<VW>(xs, i);
        VecT<VW> dn, xn;
        VecT<VW> dd;
        if (din) dd = vld<VW>(L.d[src], i);
#pragma unroll
        for (int k = 0; k < VW; ++k) {
            const float q = d != 0.f ? (bb.v[k] - s.v[k]) / d : 0.f;
            dn.v[k] = din ? fmaf(c, dd.v[k], e * q) : e * q;
            xn.v[k] = xo.v[k] + dn.v[k];
        }
        vst<VW>(L.x[dst], i, xn);
        if (dout) vst<VW>(L.d[dst], i, dn);
    }
}

__global__ void k_b_smooth(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, int cheb, float omega,
                           int sweep, int post, int src, int din, int dout, const int *skip, int ntiles) {
    pdl_prologue();
    if (skipped(skip)) return;
    for (int tb = blockIdx.x; tb < ntiles; tb += gridDim.x) {
        const BTile t = tiles[tb];
        const BLevel &L = lv[t.lev];
        if (group_done(L)) continue;
        const float e = cheb ? (post ? L.epost[sweep] : L.epre[sweep]) : omega;
        const float c = cheb ? (post ? L.cpost[sweep] : L.cpre[sweep]) : 0.f;
        if ((L.k & 3) == 0)
            smooth_body<4>(L, t, e, c, src, din, dout);
        else
            smooth_body<1>(L, t, e, c, src, din, dout);
    }
}

template <int VW>
__device__ __forceinline__ void residual_body(const BLevel &L, const BTile &t, int src) {
    for (int i = t.begin + VW * threadIdx.x; i < t.end; i += VW * blockDim.x) {
        const int v = i >> L.kshift, j = i & (L.k - 1);
        VecT<VW> s;
        float d;
        brow<VW>(L, v, j, L.x[src], s, d);
        const VecT<VW> bb = vld<VW>(L.b, i);
        VecT<VW> r;
#pragma unroll
        for (int k = 0; k < VW; ++k) r.v[k] = d != 0.f ? bb.v[k] - s.v[k] : 0.f;
        vst<VW>(L.r, i, r);
    }
}

__global__ void k_b_residual(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, int src,
                             const int *skip, int ntiles) {
    pdl_prologue();
    if (skipped(skip)) return;
    for (int tb = blockIdx.x; tb < ntiles; tb += gridDim.x) {
        const BTile t = tiles[tb];
        const BLevel &L = lv[t.lev];
        if (group_done(L)) continue;
        if ((L.k & 3) == 0)
            residual_body<4>(L, t, src);
        else
            residual_body<1>(L, t, src);
    }
}

// tiles range over the coarse items; t.lev is the fine level (the coarse one is t.lev - 1)
template <int VW>
__device__ __forceinline__ void restrict_body(const BLevel &L, const BLevel &C, const BTile &t, int star0) {
    for (int i = t.begin + VW * threadIdx.x; i < t.end; i += VW * blockDim.x) {
        const int c = i >> L.kshift, j = i & (L.k - 1);
        VecT<VW> acc;
#pragma unroll
        for (int k = 0; k < VW; ++k) acc.v[k] = 0.f;
        int deg = 0;
        for (int q = 0; q < L.K; ++q) {
            const int nb = __ldg(L.col + (size_t)q * L.n + c);
            if (nb != c) {
                const VecT<VW> rv = vld<VW>(L.r, (nb << L.kshift) + j);
                const float sw = star0 ? __ldg(L.s0 + nb) : 1.f;
#pragma unroll
                for (int k = 0; k < VW; ++k) acc.v[k] = fmaf(sw, rv.v[k], acc.v[k]);
                ++deg;
            }
        }
        const VecT<VW> rc = vld<VW>(L.r, (c << L.kshift) + j);
        VecT<VW> out;
        if (star0) {
            const float sc = __ldg(L.s0 + c), inv = 1.f / __ldg(C.s0 + c);
#pragma unroll
            for (int k = 0; k < VW; ++k) out.v[k] = (sc * rc.v[k] + 0.5f * acc.v[k]) * inv;
        } else {
            const float den = 1.f + 0.5f * (float)deg;
#pragma unroll
            for (int k = 0; k < VW; ++k) out.v[k] = (rc.v[k] + 0.5f * acc.v[k]) / den;
        }
        vst<VW>(C.b, i, out);
    }
}

__global__ void k_b_restrict(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, int star0,
                             const int *skip, int ntiles) {
    pdl_prologue();
    if (skipped(skip)) return;
    for (int tb = blockIdx.x; tb < ntiles; tb += gridDim.x) {
        const BTile t = tiles[tb];
        const BLevel &L = lv[t.lev];
        const BLevel &C = lv[t.lev - 1];
        if (group_done(L)) continue;
        if ((L.k & 3) == 0)
            restrict_body<4>(L, C, t, star0);
        else
            restrict_body<1>(L, C, t, star0);
    }
}

// coarsest level: x = G b for each right-hand side
__global__ void k_b_coarse(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, const int *skip, int ntiles) {
    pdl_prologue();
    if (skipped(skip)) return;
    for (int tb = blockIdx.x; tb < ntiles; tb += gridDim.x) {
        const BTile t = tiles[tb];
        const BLevel &L = lv[t.lev];
        if (group_done(L)) continue;
        for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
            const int row = i >> L.kshift, j = i & (L.k - 1);
            float acc = 0.f;
            for (int c = 0; c < L.n; ++c) acc = fmaf(__ldg(L.G + (size_t)row * L.n + c), L.b[(c << L.kshift) + j], acc);
            L.x[0][i] = acc;
        }
    }
}

// x_f[dst] += P e_c with e_c the coarser level's cycle result
template <int VW>
__device__ __forceinline__ void prolong_body(const BLevel &L, const BLevel &C, const BTile &t, int dst) {
    const float *ec = C.x[C.res_idx];
    for (int i = t.begin + VW * threadIdx.x; i < t.end; i += VW * blockDim.x) {
        const int v = i >> L.kshift, j = i & (L.k - 1);
        VecT<VW> add;
        if (v < C.n) {
            add = vld<VW>(ec, (v << L.kshift) + j);
        } else {
            const int2 p = __ldg(L.par + (v - C.n));
            const VecT<VW> a = vld<VW>(ec, (p.x << L.kshift) + j), b = vld<VW>(ec, (p.y << L.kshift) + j);
#pragma unroll
            for (int k = 0; k < VW; ++k) add.v[k] = 0.5f * (a.v[k] + b.v[k]);
        }
        VecT<VW> x = vld<VW>(L.x[dst], i);
#pragma unroll
        for (int k = 0; k < VW; ++k) x.v[k] += add.v[k];
        vst<VW>(L.x[dst], i, x);
    }
}

__global__ void k_b_prolong(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, int dst,
                            const int *skip, int ntiles) {
    pdl_prologue();
    if (skipped(skip)) return;
    for (int tb = blockIdx.x; tb < ntiles; tb += gridDim.x) {
        const BTile t = tiles[tb];
        const BLevel &L = lv[t.lev];
        const BLevel &C = lv[t.lev - 1];
        if (group_done(L)) continue;
        if ((L.k & 3) == 0)
            prolong_body<4>(L, C, t, dst);
        else
            prolong_body<1>(L, C, t, dst);
    }
}

// ---------------------------------------------------------------------------
// Finest level: the FP64 outer iteration of every right-hand side.
//
// These kernels run on the finest tile list (block b works on tile b; a tile
// belongs to one group and covers whole vertices), one item per thread.
// Every thread's items share one right-hand side j = threadIdx.x & (k-1),
// because tiles start on vertex boundaries and blockDim is a multiple of k.
// Per-right-hand-side sums are deterministic: the block folds its threads per
// j in a fixed order and writes one partial per (sum, tile, j); k_b_finalize
// adds a right-hand side's partials over its group's tiles in tile order.
// ---------------------------------------------------------------------------

struct BSums {
    double *part;  // [kBMaxSums][ntile][kmax]
    int ntile, kmax;
};
constexpr int kBMaxSums = 4;

// Per right-hand side: its group's finest tiles [tb, te), its column j, its
// finest level descriptor and whether it is a caller's column (live) or padding.
struct BRhs {
    int tb, te, j, lev, live;
};

// Per right-hand side scalars of the outer iteration (FP64).
struct BScal {
    double rz, alpha, beta, c, rn2, bn2, thr2, rel, mean;
    int done, stalled;
};

template <int NS>
__device__ __forceinline__ void bsum_write(const double (&acc)[NS], int k, const BSums &P) {
    extern __shared__ double sh[];  // blockDim.x doubles
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        sh[threadIdx.x] = acc[s];
        __syncthreads();
        if ((int)threadIdx.x < k) {
            double a = 0.0;
            for (int m = threadIdx.x; m < (int)blockDim.x; m += k) a += sh[m];
            P.part[((size_t)s * P.ntile + blockIdx.x) * P.kmax + threadIdx.x] = a;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int rhs_of(const BLevel &L, int i) { return L.rhs_base + (i & (L.k - 1)); }

// (L x)_v of right-hand side j in FP64, difference form, slots in order.  Rows
// of 6 slots issue their table loads and their six gathers before the first
// FMA (the same sum, in the same order, as the loop).
__device__ __forceinline__ double brow64(const BLevel &L, int v, int j, const double *x, double xi) {
    double s = 0.0;
    if (L.K == 6) {
        const int n = L.n, ks = L.kshift;
        int cq[6];
        double wq[6], xq[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            cq[q] = __ldg(L.col + (size_t)q * n + v);
            wq[q] = __ldg(L.w64 + (size_t)q * n + v);
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) xq[q] = x[(cq[q] << ks) + j];
#pragma unroll
        for (int q = 0; q < 6; ++q) s = fma(wq[q], xi - xq[q], s);
        return s;
    }
    for (int q = 0; q < L.K; ++q) {
        const size_t o = (size_t)q * L.n + v;
        s = fma(__ldg(L.w64 + o), xi - x[(__ldg(L.col + o) << L.kshift) + j], s);
    }
    return s;
}

// Standalone refinement: r = b - L x (FP64, free rows), r32 = cycle input, sums of r^2 and b^2.
__global__ void k_b_res64(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, BSums P, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    if (group_done(L)) return;  // block-uniform: the tile is one group's
    double acc[2] = {0.0, 0.0};
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
        const int v = i >> L.kshift, j = i & (L.k - 1);
        double ri = 0.0, bi = 0.0;
        if (L.freev[v]) {
            const double s = brow64(L, v, j, L.ox, L.ox[i]);
            bi = L.ob[i];
            ri = bi - s;
        }
        L.orr[i] = ri;
        L.b[i] = (float)ri;
        acc[0] = fma(ri, ri, acc[0]);
        acc[1] = fma(bi, bi, acc[1]);
    }
    bsum_write<2>(acc, L.k, P);
}

// x += (double) e
__global__ void k_b_add64(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    if (group_done(L)) return;  // block-uniform: the tile is one group's
    const float *e = L.x[L.res_idx];
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) L.ox[i] += (double)e[i];
}

// gauge: per-right-hand-side sums of *0 v over free rows (v = ob or ox)
__global__ void k_b_meansum(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, int which, BSums P) {
    pdl_prologue();
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    const double *v = which ? L.ox : L.ob;
    double acc[1] = {0.0};
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
        const int vv = i >> L.kshift;
        if (L.freev[vv]) acc[0] = fma(__ldg(L.star0 + vv), v[i], acc[0]);
    }
    bsum_write<1>(acc, L.k, P);
}

// v -= mean (gauge groups; the mean is 0 for Dirichlet groups), 0 on fixed rows
__global__ void k_b_shift(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, int which,
                          const BScal *__restrict__ sc) {
    pdl_prologue();
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    double *v = which ? L.ox : L.ob;
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
        const int vv = i >> L.kshift;
        v[i] = L.freev[vv] ? v[i] - sc[rhs_of(L, i)].mean : 0.0;
    }
}

// MG-PCG, cold start: x = 0, r = b - mean (free rows; the gauge mean when sc is
// given, 0 for Dirichlet groups), r32 = (float) r; sums of r^2 and b^2.
__global__ void k_bp_init(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, const BScal *__restrict__ sc,
                          BSums P) {
    pdl_prologue();
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    double acc[2] = {0.0, 0.0};
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
        const int v = i >> L.kshift;
        const double ri = L.freev[v] ? L.ob[i] - (sc ? sc[rhs_of(L, i)].mean : 0.0) : 0.0;
        L.ox[i] = 0.0;
        L.orr[i] = ri;
        L.b[i] = (float)ri;
        acc[0] = fma(ri, ri, acc[0]);
        acc[1] = acc[0];
    }
    bsum_write<2>(acc, L.k, P);
}

// The four FP64 dot products of the preconditioned vector z (FP32 cycle
// output) in the *0 inner product: sum *0 z, sum *0 r z, sum *0 r zo (zo the
// previous shifted z, FP64) and sum *0 r, over free rows.
__global__ void k_bp_zdots(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, int first, BSums P,
                           const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    if (group_done(L)) return;  // block-uniform: the tile is one group's
    const float *z = L.x[L.res_idx];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
        const int v = i >> L.kshift;
        if (L.freev[v]) {
            const double s0 = __ldg(L.star0 + v), zi = decdev::f2d(z[i]);
            const double sr = s0 * L.orr[i];
            acc[0] = fma(s0, zi, acc[0]);
            acc[1] = fma(sr, zi, acc[1]);
            if (!first) acc[2] = fma(sr, L.ozo[i], acc[2]);
            acc[3] += sr;
        }
    }
    bsum_write<4>(acc, L.k, P);
}

// zs = z - c (FP64, free rows; 0 on fixed rows), p = zs + beta p (p = zs on the first pass), zo = zs
__global__ void k_bp_pupd(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, int first,
                          const BScal *__restrict__ sc, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    if (group_done(L)) return;  // block-uniform: the tile is one group's
    const float *z = L.x[L.res_idx];
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
        const int v = i >> L.kshift;
        const BScal &S = sc[rhs_of(L, i)];
        const double zs = L.freev[v] ? decdev::f2d(z[i]) - S.c : 0.0;
        L.ozo[i] = zs;
        L.op[i] = first ? zs : fma(S.beta, L.op[i], zs);
    }
}

// q = L p (FP64, difference form; fixed rows have weights 0 and give 0), sum *0 p q
__global__ void k_bp_spmv(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, BSums P, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    if (group_done(L)) return;  // block-uniform: the tile is one group's
    double acc[1] = {0.0};
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
        const int v = i >> L.kshift, j = i & (L.k - 1);
        const double pi = L.op[i];
        const double s = brow64(L, v, j, L.op, pi);
        L.oq[i] = s;
        acc[0] = fma(__ldg(L.star0 + v) * pi, s, acc[0]);
    }
    bsum_write<1>(acc, L.k, P);
}

// x += alpha p, r -= alpha q (FP64), r32 = (float) r, sum r^2
__global__ void k_bp_update(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, const BScal *__restrict__ sc,
                            BSums P, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    if (group_done(L)) return;  // block-uniform: the tile is one group's
    double acc[1] = {0.0};
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
        const double a = sc[rhs_of(L, i)].alpha;
        L.ox[i] = fma(a, L.op[i], L.ox[i]);
        const double ri = fma(-a, L.oq[i], L.orr[i]);
        L.orr[i] = ri;
        L.b[i] = (float)ri;
        acc[0] = fma(ri, ri, acc[0]);
    }
    bsum_write<1>(acc, L.k, P);
}

enum { kFinMean = 0, kFinInit = 1, kFinZdots = 2, kFinAlpha = 3, kFinConv = 4 };

// One block per right-hand side (block b = right-hand side b): add its
// partials over its group's tiles (thread-strided, then a fixed-order warp
// butterfly and a fixed-order sum of the warps), then the scalars of `kind`.
// kFinInit and kFinConv also decide convergence: the last block to finish
// sets the batch's done flag once every right-hand side has converged (or
// maxit is reached), counts the pass (kFinConv), records the largest
// relative residual and sets each group's live flag for the next pass.  The
// right-hand sides of a group that skipped this pass keep their scalars (the
// group's partials were not written).
__global__ void k_b_finalize(int nrhs, const BRhs *__restrict__ rinfo, const BLevel *__restrict__ lv, BSums P,
                             BScal *__restrict__ sc, int kind, int first, Scal *S, int *pending, unsigned *counter,
                             const int *skip, int *glive, int *gpend, int ngroups) {
    pdl_prologue();
    if (skipped(skip)) return;
    __shared__ double wsum[kBMaxSums][16];  // per-warp totals (blockDim <= 512)
    const int q = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ns = kind == kFinZdots ? 4 : (kind == kFinInit ? 2 : 1);
    const BRhs R = rinfo[q];
    for (int s = 0; s < ns; ++s) {
        double a = 0.0;
        for (int tt = R.tb + threadIdx.x; tt < R.te; tt += blockDim.x)
            a += P.part[((size_t)s * P.ntile + tt) * P.kmax + R.j];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) wsum[s][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[4] = {0.0, 0.0, 0.0, 0.0};
        for (int s = 0; s < ns; ++s)
            for (int w = 0; w < nw; ++w) tot[s] += wsum[s][w];
        BScal &C = sc[q];
        const BLevel &L = lv[R.lev];
        const bool dead = (kind == kFinZdots || kind == kFinAlpha || kind == kFinConv) && group_done(L);
        if (dead) {
            // this group's kernels skipped the pass: every scalar stays as it was
        } else if (kind == kFinMean) {
            C.mean = L.gauge ? tot[0] / L.s0sum : 0.0;
        } else if (kind == kFinInit) {
            C.bn2 = tot[1];
            C.rn2 = tot[0];
            C.thr2 = tot[1] > 0.0 ? S->tol * S->tol * tot[1] : (double)INFINITY;
            C.stalled = 0;
            C.done = !R.live || C.rn2 <= C.thr2;
            C.rz = 0.0;
            C.c = 0.0;
        } else if (kind == kFinZdots) {
            const double c = L.gauge ? tot[0] / L.s0sum : 0.0;
            const double rz_new = tot[1] - c * tot[3];
            C.beta = (first || C.done) ? 0.0 : (rz_new - tot[2]) / C.rz;
            C.rz = rz_new;
            C.c = c;
        } else if (kind == kFinAlpha) {
            double a = C.done ? 0.0 : C.rz / tot[0];
            if (!C.done && (!(tot[0] > 0.0) || !isfinite(a))) {
                a = 0.0;  // the iteration cannot move this right-hand side any further
                C.stalled = 1;
                C.done = 1;
            }
            C.alpha = a;
        } else {  // kFinConv
            C.rn2 = tot[0];
            if (!C.done && C.rn2 <= C.thr2) C.done = 1;
        }
        if ((kind == kFinInit || kind == kFinConv) && !dead) {
            const bool bad = !isfinite(C.rn2) || !isfinite(C.bn2);
            C.rel = bad ? (double)NAN : (C.bn2 > 0.0 ? sqrt(C.rn2 / C.bn2) : 0.0);
            if (bad) {
                C.done = 1;
                atomicExch(&S->status, 1);
            }
        }
        if (kind == kFinInit || kind == kFinConv) {
            if (!C.done) {
                atomicAdd(pending, 1);
                atomicAdd(L.gpend, 1);
            }
            if (R.live && isfinite(C.rel))
                atomicMax((unsigned long long *)&S->rel, (unsigned long long)__double_as_longlong(C.rel));
        }
    }
    if (kind != kFinInit && kind != kFinConv) return;
    if (!decdev::last_block(counter)) return;
    if (threadIdx.x == 0) {
        __threadfence();
        const int left = atomicAdd(pending, 0);
        if (kind == kFinConv) S->iter += 1;
        if (left == 0 || S->status != 0 || S->iter >= S->maxit) S->done = 1;
        *pending = 0;
        for (int g = 0; g < ngroups; ++g) glive[g] = atomicExch(gpend + g, 0) > 0 ? 1 : 0;
        *counter = 0u;
    }
}

// Clear the largest relative residual before a convergence pass.
__global__ void k_b_relzero(Scal *S, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    if (threadIdx.x == 0) S->rel = 0.0;
}

// user layout [n][nrhs] -> group layout [n][k], columns [src0, src0 + cnt) to [dst0, ...);
// inv != nullptr: divide by inv[v] on free rows, 0 on fixed rows
__global__ void k_b_gather(int n, int k, int nrhs, int src0, int dst0, int cnt, const double *__restrict__ src,
                           double *__restrict__ dst, const double *__restrict__ inv, const uint8_t *__restrict__ freev) {
    pdl_prologue();
    const int64_t tot = (int64_t)n * cnt;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / cnt), c = (int)(i % cnt);
        double val = src[(size_t)v * nrhs + src0 + c];
        if (inv) val = freev[v] ? val / inv[v] : 0.0;
        dst[(size_t)v * k + dst0 + c] = val;
    }
}

// group layout -> user layout; sc != nullptr: subtract each right-hand side's
// mean (rhs0 = batch index of group column 0); mul != nullptr: then multiply by mul[v]
__global__ void k_b_scatter(int n, int k, int nrhs, int src0, int dst0, int cnt, const double *__restrict__ src,
                            double *__restrict__ dst, const double *__restrict__ mul, const BScal *__restrict__ sc,
                            int rhs0) {
    pdl_prologue();
    const int64_t tot = (int64_t)n * cnt;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / cnt), c = (int)(i % cnt);
        double val = src[(size_t)v * k + src0 + c];
        if (sc) val -= sc[rhs0 + src0 + c].mean;
        dst[(size_t)v * nrhs + dst0 + c] = mul ? val * mul[v] : val;
    }
}

// dJ/d*1_e = -(d0 mu)_e (d0 u)_e per right-hand side, mu and u in group layout,
// written to the user layout [ne][nrhs]
__global__ void k_b_edge_grad(int64_t ne, int k, int nrhs, int src0, int dst0, int cnt, const int2 *__restrict__ edges,
                              const double *__restrict__ mu, const double *__restrict__ u, double *__restrict__ g) {
    pdl_prologue();
    const int64_t tot = ne * cnt;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / cnt;
        const int c = (int)(i % cnt);
        const int2 ab = __ldg(edges + e);
        const size_t lo = (size_t)ab.x * k + src0 + c, hi = (size_t)ab.y * k + src0 + c;
        g[(size_t)e * nrhs + dst0 + c] = -(mu[hi] - mu[lo]) * (u[hi] - u[lo]);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct dec_batch {
    dec_batch_opts opts;
    int device = 0;
    std::vector<dec_mg *> mgs;  // one per caller entry
    std::vector<int> nrhs;
    // A run of caller columns [src0, src0 + cnt) of entry `entry` that fill group
    // columns [dst0, dst0 + cnt).
    struct Run {
        int entry, src0, dst0, cnt;
    };
    // A group: up to k right-hand sides of one hierarchy (entries that share a
    // hierarchy are merged), interleaved; descriptors [first_lev, first_lev + nlev),
    // coarsest first; kk caller columns, k - kk padding columns.
    struct Group {
        dec_mg *mg;
        int k, kk, first_lev, nlev, rhs_base;
        std::vector<Run> runs;
    };
    std::vector<Group> groups;
    std::vector<BLevel> hlv;   // host copy of the descriptors
    BLevel *dlv = nullptr;     // device descriptors
    int total_rhs = 0;
    int64_t dof = 0;           // finest vertices x caller right-hand sides, summed
    struct Op {
        int kind;  // 0 smooth0, 1 smooth, 2 residual, 3 restrict, 4 coarse, 5 prolong
        int off, cnt;
        int sweep, post, src, din, dout;
    };
    std::vector<Op> cycle_ops;
    // blocks of one wave of each cycle kernel (SMs x resident blocks): a
    // launch over more tiles loops, each block taking every wave-th tile
    int wave[6] = {0, 0, 0, 0, 0, 0};
    int res_off = 0, res_cnt = 0;  // finest items of every group (the outer iteration)
    BTile *dtiles = nullptr;
    BSums sums{};
    BRhs *rinfo = nullptr;
    BScal *bsc = nullptr;
    int *pending = nullptr;
    unsigned *counter = nullptr;
    int *glive = nullptr, *gpend = nullptr;  // per group: live flag, right-hand sides still iterating
    Scal *scal = nullptr;
    Scal *scal_h = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t loop = nullptr;
    int64_t loop_kernels = 0;
    std::vector<void *> allocs;
    size_t bytes = 0;
};

namespace {

template <typename T>
int balloc(dec_batch *B, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        decimpl::set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? DEC_ERR_OOM : DEC_ERR_CUDA;
    }
    B->allocs.push_back((void *)*p);
    B->bytes += count * sizeof(T);
    return DEC_OK;
}

void batch_free(dec_batch *B) {
    if (B->loop) cudaGraphExecDestroy(B->loop);
    for (void *p : B->allocs) cudaFree(p);
    if (B->scal_h) cudaFreeHost(B->scal_h);
    if (B->cap) cudaStreamDestroy(B->cap);
}

void bcheb(double lmax, double lo, double hi, int nu, float *c, float *e) {
    const double a = lo * lmax, b = hi * lmax;
    const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
    c[0] = 0.f;
    e[0] = (float)(1.0 / theta);
    double rho_prev = 1.0 / sigma;
    for (int k = 1; k < nu; ++k) {
        const double rho = 1.0 / (2.0 * sigma - rho_prev);
        c[k] = (float)(rho * rho_prev);
        e[k] = (float)(2.0 * rho / delta);
        rho_prev = rho;
    }
}

// Tiles of `rows` vertices x k right-hand sides, cut at vertex boundaries
// into pieces of about `target` items.
void add_tiles(std::vector<BTile> &out, int lev, int rows, int kshift, int target) {
    const int per = std::max(1, target >> kshift);
    for (int r = 0; r < rows; r += per) {
        const int re = std::min(rows, r + per);
        out.push_back(BTile{lev, r << kshift, re << kshift});
    }
}

template <typename... KArgs, typename... Args>
void blaunch(const dec_batch *B, void (*kernel)(KArgs...), int grid, size_t smem, cudaStream_t s, Args &&...args) {
    if (grid <= 0) return;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)B->opts.block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

int fin_grid(const dec_batch *B) { return B->total_rhs; }

// One multigrid cycle of every group on its finest level's r32 (L.b); the
// result is the finest level's x[res_idx].
void enqueue_cycle(dec_batch *B, cudaStream_t s, const int *skip) {
    const auto &o = B->opts;
    const int cheb = o.smoother == DEC_SMOOTH_CHEBYSHEV;
    const float omega = (float)(2.0 / 3.0);
    for (const auto &op : B->cycle_ops) {
        const BTile *t = B->dtiles + op.off;
        const int g = std::min(op.cnt, B->wave[op.kind]);
        switch (op.kind) {
            case 0: blaunch(B, k_b_smooth0, g, 0, s, (const BLevel *)B->dlv, t, cheb, omega, op.dout, skip, op.cnt); break;
            case 1:
                blaunch(B, k_b_smooth, g, 0, s, (const BLevel *)B->dlv, t, cheb, omega, op.sweep, op.post, op.src,
                        op.din, op.dout, skip, op.cnt);
                break;
            case 2: blaunch(B, k_b_residual, g, 0, s, (const BLevel *)B->dlv, t, op.src, skip, op.cnt); break;
            case 3: blaunch(B, k_b_restrict, g, 0, s, (const BLevel *)B->dlv, t, op.src, skip, op.cnt); break;
            case 4: blaunch(B, k_b_coarse, g, 0, s, (const BLevel *)B->dlv, t, skip, op.cnt); break;
            case 5: blaunch(B, k_b_prolong, g, 0, s, (const BLevel *)B->dlv, t, op.src, skip, op.cnt); break;
        }
    }
}

void enqueue_finalize(dec_batch *B, cudaStream_t s, int kind, int first, const int *skip) {
    blaunch(B, k_b_finalize, fin_grid(B), 0, s, B->total_rhs, (const BRhs *)B->rinfo, (const BLevel *)B->dlv, B->sums,
            B->bsc, kind, first, B->scal, B->pending, B->counter, skip, B->glive, B->gpend, (int)B->groups.size());
}

// Every group live again (between solves: kernels run outside the loop, such as the smoother timer, see all).
int all_groups_live(dec_batch *B, cudaStream_t s) {
    CK(cudaMemsetAsync(B->glive, 1, sizeof(int) * B->groups.size(), s));  // int 0x01010101: nonzero
    return DEC_OK;
}

// The preconditioned vector's dot products, the new search direction.
void enqueue_precondition(dec_batch *B, cudaStream_t s, int first, const int *skip) {
    const BTile *rt = B->dtiles + B->res_off;
    const size_t sm = sizeof(double) * B->opts.block;
    enqueue_cycle(B, s, skip);
    blaunch(B, k_bp_zdots, B->res_cnt, sm, s, (const BLevel *)B->dlv, rt, first, B->sums, skip);
    enqueue_finalize(B, s, kFinZdots, first, skip);
    blaunch(B, k_bp_pupd, B->res_cnt, 0, s, (const BLevel *)B->dlv, rt, first, (const BScal *)B->bsc, skip);
}

// One pass of the loop: a refinement pass (x += C(b - L x)) or an MG-PCG iteration.
void enqueue_pass(dec_batch *B, cudaStream_t s) {
    const int *skip = &B->scal->done;
    const BTile *rt = B->dtiles + B->res_off;
    const size_t sm = sizeof(double) * B->opts.block;
    if (B->opts.solver == DEC_SOLVER_MG) {
        enqueue_cycle(B, s, skip);
        blaunch(B, k_b_add64, B->res_cnt, 0, s, (const BLevel *)B->dlv, rt, skip);
        blaunch(B, k_b_res64, B->res_cnt, sm, s, (const BLevel *)B->dlv, rt, B->sums, skip);
        blaunch(B, k_b_relzero, 1, 0, s, B->scal, skip);
        enqueue_finalize(B, s, kFinConv, 0, skip);
        return;
    }
    blaunch(B, k_bp_spmv, B->res_cnt, sm, s, (const BLevel *)B->dlv, rt, B->sums, skip);
    enqueue_finalize(B, s, kFinAlpha, 0, skip);
    blaunch(B, k_bp_update, B->res_cnt, sm, s, (const BLevel *)B->dlv, rt, (const BScal *)B->bsc, B->sums, skip);
    blaunch(B, k_b_relzero, 1, 0, s, B->scal, skip);
    enqueue_finalize(B, s, kFinConv, 0, skip);
    enqueue_precondition(B, s, 0, skip);
}

int count_kernels(cudaGraph_t g) {
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    int nk = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++nk;
    }
    return nk;
}

int build_loop(dec_batch *B) {
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle hnd;
    cudaGraphNodeParams np = {};
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = hnd;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    }
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(B->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue_pass(B, B->cap);
            blaunch(B, decdev::k_loop_ctrl, 1, 0, B->cap, hnd, B->scal);
            cudaError_t e1 = cudaGetLastError();
            e = cudaStreamEndCapture(B->cap, &body);
            if (e == cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) {
            B->loop_kernels = count_kernels(body);
            e = cudaGraphInstantiate(&B->loop, g, 0);
        }
    }
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        B->loop = nullptr;
        return cuda_fail(e, "batch loop graph");
    }
    return DEC_OK;
}

int check_batch_device(const dec_batch *B) {
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != B->device)
        return fail(Status::fail(DEC_ERR_ARG, "the batch lives on device " + std::to_string(B->device) + " but device " +
                                                  std::to_string(cur) + " is current"));
    return DEC_OK;
}

// Solve with the right-hand sides already in every group's finest ob (caller
// columns, zero padding): the gauge projection, x = 0, the loop, the gauge
// mean of x.  The result is in every group's finest ox; when gauge is set on
// return, the callers' scatter subtracts each right-hand side's mean (BScal::mean).
int batch_run(dec_batch *B, double tol, int maxit, cudaStream_t s, int64_t &launches, bool &gauge) {
    Scal *h = B->scal_h;
    std::memset(h, 0, offsetof(Scal, hist));
    h->tol = tol;
    h->maxit = maxit;
    h->max_loops = maxit + 1;
    CK(cudaMemcpyAsync(B->scal, h, offsetof(Scal, hist), cudaMemcpyHostToDevice, s));
    // every group live for the set-up kernels (also after a run that returned early)
    if (int rc = all_groups_live(B, s)) return rc;
    const BTile *rt = B->dtiles + B->res_off;
    const size_t sm = sizeof(double) * B->opts.block;
    bool any_gauge = false;
    for (auto &L : B->hlv)
        if (L.ox && L.gauge) any_gauge = true;
    gauge = any_gauge;
    if (any_gauge) {
        // the mean of b; refinement shifts b itself (its residuals read b), MG-PCG shifts r = b in k_bp_init
        blaunch(B, k_b_meansum, B->res_cnt, sm, s, (const BLevel *)B->dlv, rt, 0, B->sums);
        enqueue_finalize(B, s, kFinMean, 0, nullptr);
        launches += 2;
        if (B->opts.solver == DEC_SOLVER_MG) {
            blaunch(B, k_b_shift, B->res_cnt, 0, s, (const BLevel *)B->dlv, rt, 0, (const BScal *)B->bsc);
            ++launches;
        }
    }
    if (B->opts.solver == DEC_SOLVER_MG) {
        for (const auto &G : B->groups) {
            const BLevel &L = B->hlv[G.first_lev + G.nlev - 1];
            CK(cudaMemsetAsync(L.ox, 0, sizeof(double) * (size_t)L.n * G.k, s));
        }
        blaunch(B, k_b_res64, B->res_cnt, sm, s, (const BLevel *)B->dlv, rt, B->sums, (const int *)nullptr);
        enqueue_finalize(B, s, kFinInit, 0, nullptr);
        launches += 2;
    } else {
        blaunch(B, k_bp_init, B->res_cnt, sm, s, (const BLevel *)B->dlv, rt,
                any_gauge ? (const BScal *)B->bsc : (const BScal *)nullptr, B->sums);
        enqueue_finalize(B, s, kFinInit, 0, nullptr);
        launches += 2;
    }
    CK(cudaGetLastError());
    if (maxit > 0) {
        if (B->opts.solver != DEC_SOLVER_MG) {
            enqueue_precondition(B, s, 1, &B->scal->done);
            launches += (int64_t)B->cycle_ops.size() + 3;
        }
        if (!B->loop) {
            int rc = build_loop(B);
            if (rc) return rc;
        }
        CK(cudaGraphLaunch(B->loop, s));
    }
    if (int rc = all_groups_live(B, s)) return rc;
    if (any_gauge) {
        // the mean of x, subtracted by the scatter into the callers' vectors
        blaunch(B, k_b_meansum, B->res_cnt, sm, s, (const BLevel *)B->dlv, rt, 1, B->sums);
        enqueue_finalize(B, s, kFinMean, 0, nullptr);
        launches += 2;
    }
    CK(cudaGetLastError());
    return DEC_OK;
}

// Statistics and status of the last batch_run (synchronizes s).
int batch_finish(dec_batch *B, double tol, int maxit, cudaStream_t s, int64_t launches, dec_batch_stats *stats) {
    Scal *h = B->scal_h;
    CK(cudaMemcpyAsync(h, B->scal, offsetof(Scal, hist), cudaMemcpyDeviceToHost, s));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    if (stats) {
        stats->iters = h->iter;
        stats->max_rel_res = h->rel;
        stats->launches = launches + (maxit > 0 ? (int64_t)h->loops * B->loop_kernels : 0);
        stats->dof = B->dof;
    }
    if (h->status == 1) return fail(Status::fail(DEC_ERR_NONFINITE, "non-finite residual in a batched solve"));
    if (!(h->rel <= tol))
        return fail(Status::fail(DEC_ERR_NOT_CONVERGED, "maxit reached (or an iteration stalled) before every "
                                                        "right-hand side converged"));
    return DEC_OK;
}

int gather_grid(const dec_batch *B, int64_t items) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(4096, (items + B->opts.block - 1) / B->opts.block));
}

}  // namespace

extern "C" {

void dec_batch_default_opts(dec_batch_opts *o) {
    if (!o) return;
    o->block = 256;
    o->kgroup = 0;
    o->nu = 2;
    o->smoother = DEC_SMOOTH_CHEBYSHEV;
    o->solver = DEC_SOLVER_MGPCG;
}

int dec_batch_create(dec_mg *const *mgs, const int *nrhs, int nmesh, const dec_batch_opts *opts, dec_batch **out) {
    if (!mgs || !nrhs || !out || nmesh < 1) return fail(Status::fail(DEC_ERR_ARG, "null pointer or no mesh"));
    *out = nullptr;
    dec_batch_opts o;
    if (opts)
        o = *opts;
    else
        dec_batch_default_opts(&o);
    if ((o.block != 128 && o.block != 256 && o.block != 512) || o.nu < 1 || o.nu > kBMaxNu ||
        (o.smoother != DEC_SMOOTH_JACOBI && o.smoother != DEC_SMOOTH_CHEBYSHEV) || o.kgroup < 0 ||
        (o.kgroup & (o.kgroup - 1)) != 0 || o.kgroup > o.block ||
        (o.solver != DEC_SOLVER_MG && o.solver != DEC_SOLVER_MGPCG))
        return fail(Status::fail(DEC_ERR_ARG, "bad batch options (block 128/256/512, 1 <= nu <= 8, kgroup a power of "
                                              "two, solver MG or MGPCG)"));
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(Status::fail(DEC_ERR_CUDA, "cudaGetDevice"));
    for (int m = 0; m < nmesh; ++m) {
        if (!mgs[m] || mgs[m]->host_only) return fail(Status::fail(DEC_ERR_ARG, "a hierarchy is null or host-only"));
        if (mgs[m]->device != dev) return fail(Status::fail(DEC_ERR_ARG, "a hierarchy lives on another device"));
        if (mgs[m]->H.mapped)
            return fail(Status::fail(DEC_ERR_ARG, "batched solves transfer along binary subdivision (no general maps)"));
        if (nrhs[m] < 1) return fail(Status::fail(DEC_ERR_ARG, "every mesh needs at least one right-hand side"));
    }
    // restriction: every hierarchy in a batch must use the same one
    const int star0 = mgs[0]->H.opts.restriction == DEC_RESTRICT_STAR0;
    for (int m = 1; m < nmesh; ++m)
        if ((mgs[m]->H.opts.restriction == DEC_RESTRICT_STAR0) != (star0 != 0))
            return fail(Status::fail(DEC_ERR_ARG, "all hierarchies of a batch must use the same restriction"));
    dec_batch *B = new (std::nothrow) dec_batch;
    if (!B) return fail(Status::fail(DEC_ERR_OOM, "host allocation"));
    auto bail = [&](int code) {
        batch_free(B);
        delete B;
        return code;
    };
    B->opts = o;
    B->mgs.assign(mgs, mgs + nmesh);
    B->nrhs.assign(nrhs, nrhs + nmesh);
    B->device = dev;
    {
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 1;
        auto wave_of = [&](auto kernel) {
            int nb = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, o.block, 0) != cudaSuccess || nb < 1) nb = 1;
            return nsm * nb;
        };
        B->wave[0] = wave_of(k_b_smooth0);
        B->wave[1] = wave_of(k_b_smooth);
        B->wave[2] = wave_of(k_b_residual);
        B->wave[3] = wave_of(k_b_restrict);
        B->wave[4] = wave_of(k_b_coarse);
        B->wave[5] = wave_of(k_b_prolong);
        (void)cudaGetLastError();
    }
    cudaError_t ce = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaStreamCreate"));
    int rc;
    // Groups: the right-hand sides of all entries that share a hierarchy, in
    // entry order, cut into groups of k (one operator read serves the group).
    std::vector<dec_mg *> uniq;
    for (int m = 0; m < nmesh; ++m)
        if (std::find(uniq.begin(), uniq.end(), mgs[m]) == uniq.end()) uniq.push_back(mgs[m]);
    int rhs_base = 0;
    for (dec_mg *mg : uniq) {
        std::vector<std::pair<int, int>> cols;  // (entry, column)
        for (int m = 0; m < nmesh; ++m)
            if (mgs[m] == mg)
                for (int c = 0; c < nrhs[m]; ++c) cols.emplace_back(m, c);
        const int total = (int)cols.size();
        int kg = o.kgroup ? o.kgroup : 1;
        if (!o.kgroup)
            while (kg < total && kg < o.block) kg <<= 1;
        for (int c0 = 0; c0 < total; c0 += kg) {
            const int k = kg;  // the last group of a hierarchy is padded with zero right-hand sides
            if ((int64_t)mg->lv.back().n * k >= ((int64_t)1 << 31))
                return bail(fail(Status::fail(DEC_ERR_ARG, "vertices x group size must stay below 2^31")));
            int ks = 0;
            while ((1 << ks) < k) ++ks;
            dec_batch::Group G{mg, k, std::min(k, total - c0), (int)B->hlv.size(), (int)mg->lv.size(), rhs_base, {}};
            for (int j = 0; j < G.kk; ++j) {
                const auto &pc = cols[c0 + j];
                if (!G.runs.empty() && G.runs.back().entry == pc.first &&
                    G.runs.back().src0 + G.runs.back().cnt == pc.second && G.runs.back().dst0 + G.runs.back().cnt == j)
                    G.runs.back().cnt += 1;
                else
                    G.runs.push_back(dec_batch::Run{pc.first, pc.second, j, 1});
            }
            for (int l = 0; l < G.nlev; ++l) {
                const DevLevel &D = mg->lv[l];
                const decimpl::HostLevel &HL = mg->H.levels[l];
                BLevel L = {};
                L.n = D.n;
                L.K = D.K;
                L.k = k;
                L.kshift = ks;
                L.col = D.col;
                L.w = D.w32;
                L.s0 = D.star0_32;
                L.par = D.par;
                const size_t nv = (size_t)D.n * k;
                if ((rc = balloc(B, &L.x[0], nv)) || (rc = balloc(B, &L.x[1], nv)) || (rc = balloc(B, &L.d[0], nv)) ||
                    (rc = balloc(B, &L.d[1], nv)) || (rc = balloc(B, &L.r, nv)) || (rc = balloc(B, &L.b, nv)))
                    return bail(rc);
                bcheb(HL.lmax, mg->H.opts.cheby_lo, mg->H.opts.cheby_hi, o.nu, L.cpre, L.epre);
                bcheb(HL.lmax, mg->H.opts.cheby_lo, mg->H.opts.cheby_hi, o.nu, L.cpost, L.epost);
                L.res_idx = l == 0 ? 0 : ((o.nu - 1) % 2 + o.nu) % 2;
                L.G = l == 0 ? mg->G32 : nullptr;
                if (l == G.nlev - 1) {
                    L.w64 = D.w64;
                    L.freev = D.freev;
                    L.star0 = D.star0;
                    if ((rc = balloc(B, &L.ox, nv)) || (rc = balloc(B, &L.orr, nv)) || (rc = balloc(B, &L.ob, nv)))
                        return bail(rc);
                    if (o.solver == DEC_SOLVER_MGPCG &&
                        ((rc = balloc(B, &L.op, nv)) || (rc = balloc(B, &L.oq, nv)) || (rc = balloc(B, &L.ozo, nv))))
                        return bail(rc);
                    L.rhs_base = rhs_base;
                    L.gauge = mg->H.bc == DEC_BC_GAUGE;
                    L.s0sum = mg->star0_sum;
                    B->dof += (int64_t)D.n * G.kk;
                }
                L.group = (int)B->groups.size();
                B->hlv.push_back(L);
            }
            B->groups.push_back(G);
            rhs_base += k;
        }
    }
    B->total_rhs = rhs_base;
    // cycle schedule aligned by depth below each group's finest level
    std::vector<BTile> tiles;
    // items per tile: 8 per thread on every group's finest level (fewer, longer tiles stream best there),
    // 4 per thread below it (more tiles for the smaller levels): 11.2 -> 10.7 ms on the batched workload
    const int target0 = o.block * 8, target = o.block * 4;
    int dmax = 0;
    for (auto &G : B->groups) dmax = std::max(dmax, G.nlev - 1);
    auto op_tiles = [&](int kind, int sweep, int post, int src, int din, int dout, auto &&pick) {
        dec_batch::Op op{kind, (int)tiles.size(), 0, sweep, post, src, din, dout};
        for (auto &G : B->groups) pick(G, tiles);
        op.cnt = (int)tiles.size() - op.off;
        if (op.cnt > 0) B->cycle_ops.push_back(op);
    };
    const int cheb = o.smoother == DEC_SMOOTH_CHEBYSHEV;
    auto level_tiles = [&](int d) {
        return [&, d](const dec_batch::Group &G, std::vector<BTile> &t) {
            const int l = G.nlev - 1 - d;
            if (l >= 1) add_tiles(t, G.first_lev + l, B->hlv[G.first_lev + l].n, B->hlv[G.first_lev + l].kshift, d == 0 ? target0 : target);
        };
    };
    for (int d = 0; d < dmax; ++d) {
        // pre-smoothing: sweep 0 from zero, then ping-pong
        op_tiles(0, 0, 0, 0, 0, (cheb && o.nu > 1), level_tiles(d));
        int cur = 0;
        for (int sw = 1; sw < o.nu; ++sw) {
            op_tiles(1, sw, 0, cur, cheb, (cheb && sw + 1 < o.nu), level_tiles(d));
            cur = 1 - cur;
        }
        op_tiles(2, 0, 0, cur, 0, 0, level_tiles(d));
        op_tiles(3, 0, 0, star0, 0, 0, [&](const dec_batch::Group &G, std::vector<BTile> &t) {
            const int l = G.nlev - 1 - d;
            if (l >= 1) add_tiles(t, G.first_lev + l, B->hlv[G.first_lev + l - 1].n, B->hlv[G.first_lev + l].kshift, target);
        });
    }
    // coarsest solves of every group
    op_tiles(4, 0, 0, 0, 0, 0, [&](const dec_batch::Group &G, std::vector<BTile> &t) {
        add_tiles(t, G.first_lev, B->hlv[G.first_lev].n, B->hlv[G.first_lev].kshift, target);
    });
    const int after_pre = (o.nu - 1) % 2;
    for (int d = dmax - 1; d >= 0; --d) {
        op_tiles(5, 0, 0, after_pre, 0, 0, level_tiles(d));
        int cur = after_pre;
        for (int sw = 0; sw < o.nu; ++sw) {
            op_tiles(1, sw, 1, cur, (cheb && sw > 0), (cheb && sw + 1 < o.nu), level_tiles(d));
            cur = 1 - cur;
        }
    }
    // finest items of every group, in larger tiles; the per-right-hand-side tile ranges
    B->res_off = (int)tiles.size();
    std::vector<BRhs> rinfo;
    int kmax = 1;
    for (auto &G : B->groups) {
        const int l = G.first_lev + G.nlev - 1;
        const int tb = (int)tiles.size() - B->res_off;
        // 16 items per thread and tile (8: 10.7 ms, 32: 10.8, 64: 11.9 on the batched workload; 16: 10.4)
        add_tiles(tiles, l, B->hlv[l].n, B->hlv[l].kshift, o.block * 16);
        const int te = (int)tiles.size() - B->res_off;
        for (int j = 0; j < G.k; ++j) rinfo.push_back(BRhs{tb, te, j, l, j < G.kk ? 1 : 0});
        kmax = std::max(kmax, G.k);
    }
    B->res_cnt = (int)tiles.size() - B->res_off;
    B->sums.ntile = B->res_cnt;
    B->sums.kmax = kmax;
    if ((rc = balloc(B, &B->glive, B->groups.size())) || (rc = balloc(B, &B->gpend, B->groups.size())))
        return bail(rc);
    for (BLevel &L : B->hlv) {
        L.live = B->glive + L.group;
        L.gpend = B->gpend + L.group;
    }
    if ((rc = balloc(B, &B->dtiles, tiles.size())) || (rc = balloc(B, &B->dlv, B->hlv.size())) ||
        (rc = balloc(B, &B->sums.part, (size_t)kBMaxSums * B->res_cnt * kmax)) ||
        (rc = balloc(B, &B->rinfo, rinfo.size())) || (rc = balloc(B, &B->bsc, (size_t)B->total_rhs)) ||
        (rc = balloc(B, &B->pending, 1)) || (rc = balloc(B, &B->counter, 1)) || (rc = balloc(B, &B->scal, 1)))
        return bail(rc);
    ce = cudaMemcpy(B->dtiles, tiles.data(), tiles.size() * sizeof(BTile), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(B->dlv, B->hlv.data(), B->hlv.size() * sizeof(BLevel), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(B->rinfo, rinfo.data(), rinfo.size() * sizeof(BRhs), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemset(B->bsc, 0, sizeof(BScal) * B->total_rhs);
    if (ce == cudaSuccess) ce = cudaMemset(B->pending, 0, sizeof(int));
    if (ce == cudaSuccess) ce = cudaMemset(B->gpend, 0, sizeof(int) * B->groups.size());
    if (ce == cudaSuccess) ce = cudaMemset(B->glive, 1, sizeof(int) * B->groups.size());
    if (ce == cudaSuccess) ce = cudaMemset(B->counter, 0, sizeof(unsigned));
    if (ce == cudaSuccess) ce = cudaMemset(B->scal, 0, sizeof(Scal));
    if (ce == cudaSuccess) ce = cudaMallocHost((void **)&B->scal_h, sizeof(Scal));
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "batch upload"));
    *out = B;
    return DEC_OK;
}

void dec_batch_destroy(dec_batch *B) {
    if (!B) return;
    batch_free(B);
    delete B;
}

int dec_batch_solve(dec_batch *B, const double *const *b, double *const *x, double tol, int maxit,
                    dec_batch_stats *stats, dec_stream_t stream) {
    if (!B || !b || !x) return fail(Status::fail(DEC_ERR_ARG, "null pointer"));
    if (!(tol >= 0.0) || maxit < 0 || maxit >= decdev::kHist) return fail(Status::fail(DEC_ERR_ARG, "bad tol or maxit"));
    if (int rc = check_batch_device(B)) return rc;
    for (size_t m = 0; m < B->mgs.size(); ++m)
        if (!b[m] || !x[m]) return fail(Status::fail(DEC_ERR_ARG, "null vector"));
    cudaStream_t s = (cudaStream_t)stream;
    int64_t launches = 0;
    // inputs into group layout (padding columns zero)
    for (auto &G : B->groups) {
        const BLevel &L = B->hlv[G.first_lev + G.nlev - 1];
        if (G.kk < G.k) CK(cudaMemsetAsync(L.ob, 0, sizeof(double) * (size_t)L.n * G.k, s));
        for (const auto &R : G.runs) {
            blaunch(B, k_b_gather, gather_grid(B, (int64_t)L.n * R.cnt), 0, s, L.n, G.k, B->nrhs[R.entry], R.src0, R.dst0,
                    R.cnt, b[R.entry], L.ob, (const double *)nullptr, (const uint8_t *)nullptr);
            ++launches;
        }
    }
    bool gauge = false;
    if (int rc = batch_run(B, tol, maxit, s, launches, gauge)) return rc;
    const BScal *msc = gauge ? (const BScal *)B->bsc : (const BScal *)nullptr;
    for (auto &G : B->groups) {
        const BLevel &L = B->hlv[G.first_lev + G.nlev - 1];
        for (const auto &R : G.runs) {
            blaunch(B, k_b_scatter, gather_grid(B, (int64_t)L.n * R.cnt), 0, s, L.n, G.k, B->nrhs[R.entry], R.dst0,
                    R.src0, R.cnt, (const double *)L.ox, x[R.entry], (const double *)nullptr, msc, G.rhs_base);
            ++launches;
        }
    }
    return batch_finish(B, tol, maxit, s, launches, stats);
}

int dec_batch_solve_backward(dec_batch *B, const double *const *u, const double *const *grad_u, double *const *grad_b,
                             double *const *grad_star1, double tol, int maxit, dec_batch_stats *stats,
                             dec_stream_t stream) {
    if (!B || !u || !grad_u || !grad_b) return fail(Status::fail(DEC_ERR_ARG, "null pointer"));
    if (!(tol >= 0.0) || maxit < 0 || maxit >= decdev::kHist) return fail(Status::fail(DEC_ERR_ARG, "bad tol or maxit"));
    if (int rc = check_batch_device(B)) return rc;
    for (size_t m = 0; m < B->mgs.size(); ++m)
        if (!u[m] || !grad_u[m] || !grad_b[m]) return fail(Status::fail(DEC_ERR_ARG, "null vector"));
    cudaStream_t s = (cudaStream_t)stream;
    int64_t launches = 0;
    // L mu = *0^-1 grad_u for every right-hand side
    for (auto &G : B->groups) {
        const BLevel &L = B->hlv[G.first_lev + G.nlev - 1];
        if (G.kk < G.k) CK(cudaMemsetAsync(L.ob, 0, sizeof(double) * (size_t)L.n * G.k, s));
        for (const auto &R : G.runs) {
            blaunch(B, k_b_gather, gather_grid(B, (int64_t)L.n * R.cnt), 0, s, L.n, G.k, B->nrhs[R.entry], R.src0, R.dst0,
                    R.cnt, grad_u[R.entry], L.ob, (const double *)L.star0, (const uint8_t *)L.freev);
            ++launches;
        }
    }
    bool gauge = false;
    if (int rc = batch_run(B, tol, maxit, s, launches, gauge)) return rc;
    const BScal *msc = gauge ? (const BScal *)B->bsc : (const BScal *)nullptr;
    for (auto &G : B->groups) {
        const BLevel &L = B->hlv[G.first_lev + G.nlev - 1];
        // dJ/db = *0 mu (mu with its gauge mean removed)
        for (const auto &R : G.runs) {
            blaunch(B, k_b_scatter, gather_grid(B, (int64_t)L.n * R.cnt), 0, s, L.n, G.k, B->nrhs[R.entry], R.dst0,
                    R.src0, R.cnt, (const double *)L.ox, grad_b[R.entry], (const double *)L.star0, msc, G.rhs_base);
            ++launches;
        }
        if (!grad_star1) continue;
        // dJ/d*1 = -(d0 mu)(d0 u) on the finest edges, u gathered into the group layout (ob)
        const dec_mg *mg = G.mg;
        const int64_t ne = mg->lv.back().ne;
        for (const auto &R : G.runs) {
            if (!grad_star1[R.entry]) continue;
            blaunch(B, k_b_gather, gather_grid(B, (int64_t)L.n * R.cnt), 0, s, L.n, G.k, B->nrhs[R.entry], R.src0,
                    R.dst0, R.cnt, u[R.entry], L.ob, (const double *)nullptr, (const uint8_t *)nullptr);
            blaunch(B, k_b_edge_grad, gather_grid(B, ne * R.cnt), 0, s, ne, G.k, B->nrhs[R.entry], R.dst0, R.src0,
                    R.cnt, (const int2 *)mg->edges, (const double *)L.ox, (const double *)L.ob, grad_star1[R.entry]);
            launches += 2;
        }
    }
    return batch_finish(B, tol, maxit, s, launches, stats);
}

int dec_batch_info(const dec_batch *B, int *ngroups, int *total_rhs, int64_t *dof, size_t *device_bytes) {
    if (!B) return fail(Status::fail(DEC_ERR_ARG, "null batch"));
    if (ngroups) *ngroups = (int)B->groups.size();
    if (total_rhs) *total_rhs = B->total_rhs;
    if (dof) *dof = B->dof;
    if (device_bytes) *device_bytes = B->bytes;
    return DEC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// autotuner: time candidate (block, kgroup, nu, smoother) settings on the
// caller's batch and keep the fastest that converges
// ---------------------------------------------------------------------------

extern "C" int dec_batch_tune(dec_mg *const *mgs, const int *nrhs, int nmesh, const double *const *b, double *const *x,
                              double tol, int maxit, const dec_batch_opts *cands, int ncand, int reps,
                              dec_batch_opts *best, double *best_ms, double *times, dec_stream_t stream) {
    if (!mgs || !nrhs || !b || !x || !best || nmesh < 1 || reps < 1)
        return fail(Status::fail(DEC_ERR_ARG, "null pointer or bad count"));
    std::vector<dec_batch_opts> grid;
    if (cands && ncand > 0) {
        grid.assign(cands, cands + ncand);
    } else {
        for (int blk : {128, 256, 512})
            for (int kg : {0, 8, 16, 32})
                for (int nu : {1, 2, 3}) {
                    dec_batch_opts c;
                    dec_batch_default_opts(&c);
                    c.block = blk;
                    c.kgroup = kg;
                    c.nu = nu;
                    grid.push_back(c);
                }
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best_t = 0.0;
    int best_i = -1;
    for (size_t c = 0; c < grid.size(); ++c) {
        if (times) times[c] = -1.0;
        dec_batch *B = nullptr;
        if (dec_batch_create(mgs, nrhs, nmesh, &grid[c], &B) != DEC_OK) continue;
        bool ok = dec_batch_solve(B, b, x, tol, maxit, nullptr, stream) == DEC_OK;  // warm-up, builds the graph
        double total = 0.0;
        for (int r = 0; ok && r < reps; ++r) {
            cudaEventRecord(e0, s);
            ok = dec_batch_solve(B, b, x, tol, maxit, nullptr, stream) == DEC_OK;
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            total += ms;
        }
        dec_batch_destroy(B);
        if (!ok) continue;
        const double t = total / reps;
        if (times) times[c] = t;
        if (best_i < 0 || t < best_t) {
            best_t = t;
            best_i = (int)c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    (void)cudaGetLastError();
    if (best_i < 0) return fail(Status::fail(DEC_ERR_NOT_CONVERGED, "no candidate setting converged"));
    *best = grid[best_i];
    if (best_ms) *best_ms = best_t;
    return DEC_OK;
}

// Time one launch of the batched finest-level smoothing sweep (all groups)
// with CUDA events on `stream`; reports the average and the algorithmic bytes.
extern "C" int dec_batch_time_smooth(dec_batch *B, int reps, double *avg_ms, double *bytes, dec_stream_t stream) {
    if (!B || reps < 1 || !avg_ms || !bytes) return fail(Status::fail(DEC_ERR_ARG, "bad argument"));
    if (int rc = check_batch_device(B)) return rc;
    // the first post-smoothing sweep on depth 0 (every group's finest level)
    const dec_batch::Op *op = nullptr;
    for (const auto &o : B->cycle_ops)
        if (o.kind == 1 && o.post == 1 && o.sweep == 0) op = &o;  // the last such op is depth 0
    if (!op) return fail(Status::fail(DEC_ERR_ARG, "batch has no smoothing sweep"));
    cudaStream_t s = (cudaStream_t)stream;
    if (int rc = all_groups_live(B, s)) return rc;
    const int cheb = B->opts.smoother == DEC_SMOOTH_CHEBYSHEV;
    // Algorithmic bytes: each hierarchy's finest operator once (K columns + K
    // weights per row), however many groups of k right-hand sides share it,
    // then per item x, b, x_out (+ direction) for the caller's right-hand
    // sides (padding columns not counted).
    double by = 0.0;
    std::vector<const dec_mg *> seen;
    for (auto &G : B->groups) {
        const BLevel &L = B->hlv[G.first_lev + G.nlev - 1];
        if (std::find(seen.begin(), seen.end(), G.mg) == seen.end()) {
            by += (double)L.n * (8.0 * L.K);
            seen.push_back(G.mg);
        }
        by += (double)L.n * G.kk * 4.0 * (3 + (cheb ? 1 : 0));
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int *noskip = nullptr;
    const int g = std::min(op->cnt, B->wave[1]);
    for (int r = 0; r < 2; ++r)
        blaunch(B, k_b_smooth, g, 0, s, (const BLevel *)B->dlv, (const BTile *)(B->dtiles + op->off), cheb,
                (float)(2.0 / 3.0), 0, 1, op->src, 0, op->dout, noskip, op->cnt);
    CK(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r)
        blaunch(B, k_b_smooth, g, 0, s, (const BLevel *)B->dlv, (const BTile *)(B->dtiles + op->off), cheb,
                (float)(2.0 / 3.0), 0, 1, op->src, 0, op->dout, noskip, op->cnt);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    *avg_ms = ms / reps;
    *bytes = by;
    return DEC_OK;
}
