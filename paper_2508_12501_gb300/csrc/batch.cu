// Batched solves: many right-hand sides on many hierarchies of uneven size,
// advanced together.  Each hierarchy's right-hand sides are split into
// groups of k (a power of two) whose vectors are interleaved, value j of
// vertex v at [v * k + j], so one gather of a neighbour reads k contiguous
// values.  Every operation of the cycle is one launch over all groups of all
// meshes: a tile list maps each block to (group level, item range), items
// being (vertex, right-hand side) pairs.  Operations are aligned by depth
// below each hierarchy's finest level, so the number of launches per cycle
// follows the deepest hierarchy, not the number of meshes.
//
// Solver: FP32 cycles (Sec. 2.2.1 transfers, Jacobi or Chebyshev smoothing,
// dense coarsest solve) inside FP64 iterative refinement,
// x += C(b - L x), until every right-hand side satisfies
// ||b - L x||_2 / ||b||_2 <= tol (Sec. 3.1.2).  The refinement loop runs on
// the device as a CUDA graph with a while node.
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
    // finest level: FP64 outer refinement
    const double *w64;
    const uint8_t *freev;
    const double *star0;
    double *ox, *orr, *ob;
    int rhs_base;     // index of this group's first right-hand side in the batch
    int gauge;
    double s0sum;     // sum of *0 over free vertices
};

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

// s = sum_q w_q (x_i - x_col(q)), d = sum_q w_q for VW adjacent right-hand sides
template <int VW>
__device__ __forceinline__ void brow(const BLevel &L, int v, int j, const float *x, VecT<VW> &s, float &d) {
    const VecT<VW> xi = vld<VW>(x, (v << L.kshift) + j);
#pragma unroll
    for (int c = 0; c < VW; ++c) s.v[c] = 0.f;
    d = 0.f;
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
                            int dout, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    const float e = cheb ? L.epre[0] : omega;
    if ((L.k & 3) == 0)
        smooth0_body<4>(L, t, e, dout);
    else
        smooth0_body<1>(L, t, e, dout);
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
                           int sweep, int post, int src, int din, int dout, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    const float e = cheb ? (post ? L.epost[sweep] : L.epre[sweep]) : omega;
    const float c = cheb ? (post ? L.cpost[sweep] : L.cpre[sweep]) : 0.f;
    if ((L.k & 3) == 0)
        smooth_body<4>(L, t, e, c, src, din, dout);
    else
        smooth_body<1>(L, t, e, c, src, din, dout);
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
                             const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    if ((L.k & 3) == 0)
        residual_body<4>(L, t, src);
    else
        residual_body<1>(L, t, src);
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
                             const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    const BLevel &C = lv[t.lev - 1];
    if ((L.k & 3) == 0)
        restrict_body<4>(L, C, t, star0);
    else
        restrict_body<1>(L, C, t, star0);
}

// coarsest level: x = G b for each right-hand side
__global__ void k_b_coarse(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
        const int row = i >> L.kshift, j = i & (L.k - 1);
        float acc = 0.f;
        for (int c = 0; c < L.n; ++c) acc = fmaf(__ldg(L.G + (size_t)row * L.n + c), L.b[(c << L.kshift) + j], acc);
        L.x[0][i] = acc;
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
                            const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    const BLevel &C = lv[t.lev - 1];
    if ((L.k & 3) == 0)
        prolong_body<4>(L, C, t, dst);
    else
        prolong_body<1>(L, C, t, dst);
}

// Per-right-hand-side sums: a thread's items all share j = threadIdx.x & (k-1)
// (tiles start on vertex boundaries and blockDim is a multiple of k); the
// block folds its threads per j in shared memory, then adds once per j.
__device__ __forceinline__ void b_sum_per_rhs(double v, int k, int base, double *out) {
    extern __shared__ double sh[];
    sh[threadIdx.x] = v;
    __syncthreads();
    if ((int)threadIdx.x < k) {
        double a = 0.0;
        for (int m = threadIdx.x; m < (int)blockDim.x; m += k) a += sh[m];
        atomicAdd(out + base + threadIdx.x, a);
    }
}

// FP64 residual of the refinement: r = b - L x (free rows), r32 = cycle input, sums of r^2 (and b^2)
__global__ void k_b_res64(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, double *rn2, double *bn2,
                          const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    double acc = 0.0, accb = 0.0;
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
        const int v = i >> L.kshift, j = i & (L.k - 1);
        double ri = 0.0, bi = 0.0;
        if (L.freev[v]) {
            const double xi = L.ox[i];
            double s = 0.0;
            for (int q = 0; q < L.K; ++q) {
                const size_t o = (size_t)q * L.n + v;
                s = fma(__ldg(L.w64 + o), xi - L.ox[(__ldg(L.col + o) << L.kshift) + j], s);
            }
            bi = L.ob[i];
            ri = bi - s;
        }
        L.orr[i] = ri;
        L.b[i] = (float)ri;
        acc = fma(ri, ri, acc);
        if (bn2) accb = fma(bi, bi, accb);
    }
    b_sum_per_rhs(acc, L.k, L.rhs_base, rn2);
    if (bn2) {
        __syncthreads();
        b_sum_per_rhs(accb, L.k, L.rhs_base, bn2);
    }
}

// x += (double) e
__global__ void k_b_add64(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    const float *e = L.x[L.res_idx];
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) L.ox[i] += (double)e[i];
}

// gauge: per-right-hand-side *0-weighted sums of v (ob or ox), then v -= sum / sum(*0)
__global__ void k_b_mean(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, int which, double *msum) {
    pdl_prologue();
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    if (!L.gauge) return;  // uniform over the block
    const double *v = which ? L.ox : L.ob;
    double acc = 0.0;
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
        const int vv = i >> L.kshift;
        if (L.freev[vv]) acc = fma(__ldg(L.star0 + vv), v[i], acc);
    }
    b_sum_per_rhs(acc, L.k, L.rhs_base, msum);
}

__global__ void k_b_shift(const BLevel *__restrict__ lv, const BTile *__restrict__ tiles, int which,
                          const double *msum) {
    pdl_prologue();
    const BTile t = tiles[blockIdx.x];
    const BLevel &L = lv[t.lev];
    if (!L.gauge) return;
    double *v = which ? L.ox : L.ob;
    for (int i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
        const int vv = i >> L.kshift, j = i & (L.k - 1);
        v[i] = L.freev[vv] ? v[i] - msum[L.rhs_base + j] / L.s0sum : 0.0;
    }
}

// convergence of every right-hand side; resets the residual sums for the next pass
__global__ void k_b_conv(int nrhs, double *rn2, const double *bn2, double *rel, Scal *S, int count_iter) {
    pdl_prologue();
    __shared__ int all_ok;
    __shared__ int bad;
    __shared__ double worst;
    if (threadIdx.x == 0) {
        all_ok = 1;
        bad = 0;
        worst = 0.0;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nrhs; j += blockDim.x) {
        const double b2 = bn2[j], r2 = rn2[j];
        double rr;
        if (!isfinite(b2) || !isfinite(r2)) {
            rr = (double)NAN;
            atomicExch(&bad, 1);
        } else {
            rr = b2 > 0.0 ? sqrt(r2 / b2) : 0.0;
        }
        rel[j] = rr;
        if (!(rr <= S->tol)) atomicExch(&all_ok, 0);
        rn2[j] = 0.0;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nrhs; j += blockDim.x) {
        // max of the relative residuals (non-negative doubles compare like their bit patterns)
        if (isfinite(rel[j])) atomicMax((unsigned long long *)&worst, (unsigned long long)__double_as_longlong(rel[j]));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (count_iter) S->iter += 1;
        S->rel = worst;
        if (bad) {
            S->status = 1;
            S->done = 1;
        } else if (all_ok || S->iter >= S->maxit) {
            S->done = 1;
        }
    }
}

// user layout [n][nrhs] <-> group layout [n][k] for columns [col0, col0 + kk),
// kk <= k; the padding columns of a partial last group hold zeros
__global__ void k_b_gather(int n, int k, int kk, int nrhs, int col0, const double *__restrict__ src,
                           double *__restrict__ dst) {
    pdl_prologue();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * k; i += gridDim.x * blockDim.x) {
        const int j = i % k;
        dst[i] = j < kk ? src[(size_t)(i / k) * nrhs + col0 + j] : 0.0;
    }
}

__global__ void k_b_scatter(int n, int k, int kk, int nrhs, int col0, const double *__restrict__ src,
                            double *__restrict__ dst) {
    pdl_prologue();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * k; i += gridDim.x * blockDim.x) {
        const int j = i % k;
        if (j < kk) dst[(size_t)(i / k) * nrhs + col0 + j] = src[i];
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct dec_batch {
    dec_batch_opts opts;
    int device = 0;
    std::vector<dec_mg *> mgs;
    std::vector<int> nrhs;
    struct Group {
        int mesh, col0, k, first_lev, nlev;  // descriptors [first_lev, first_lev + nlev), coarsest first
    };
    std::vector<Group> groups;
    std::vector<BLevel> hlv;   // host copy of the descriptors
    BLevel *dlv = nullptr;     // device descriptors
    int total_rhs = 0;
    int64_t dof = 0;           // finest vertices x right-hand sides, summed
    // tile lists per operation
    struct Op {
        int kind;   // 0 smooth0, 1 smooth, 2 residual, 3 restrict, 4 coarse, 5 prolong, 6 add64, 7 res64
        int off, cnt;
        int sweep, post, src, din, dout;
    };
    std::vector<Op> cycle_ops;
    int res_off = 0, res_cnt = 0;      // finest items of every group (FP64 residual, add, gauge)
    BTile *dtiles = nullptr;
    double *rn2 = nullptr, *bn2 = nullptr, *rel = nullptr, *msum = nullptr;
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

// One refinement pass: cycle on the current residual, x += e, new residual, convergence.
void enqueue_pass(dec_batch *B, cudaStream_t s) {
    const int *skip = &B->scal->done;
    const auto &o = B->opts;
    const int cheb = o.smoother == DEC_SMOOTH_CHEBYSHEV;
    const float omega = (float)(2.0 / 3.0);
    for (const auto &op : B->cycle_ops) {
        const BTile *t = B->dtiles + op.off;
        switch (op.kind) {
            case 0: blaunch(B, k_b_smooth0, op.cnt, 0, s, (const BLevel *)B->dlv, t, cheb, omega, op.dout, skip); break;
            case 1:
                blaunch(B, k_b_smooth, op.cnt, 0, s, (const BLevel *)B->dlv, t, cheb, omega, op.sweep, op.post, op.src,
                        op.din, op.dout, skip);
                break;
            case 2: blaunch(B, k_b_residual, op.cnt, 0, s, (const BLevel *)B->dlv, t, op.src, skip); break;
            case 3: blaunch(B, k_b_restrict, op.cnt, 0, s, (const BLevel *)B->dlv, t, op.src, skip); break;
            case 4: blaunch(B, k_b_coarse, op.cnt, 0, s, (const BLevel *)B->dlv, t, skip); break;
            case 5: blaunch(B, k_b_prolong, op.cnt, 0, s, (const BLevel *)B->dlv, t, op.src, skip); break;
        }
    }
    const BTile *rt = B->dtiles + B->res_off;
    blaunch(B, k_b_add64, B->res_cnt, 0, s, (const BLevel *)B->dlv, rt, skip);
    blaunch(B, k_b_res64, B->res_cnt, sizeof(double) * o.block, s, (const BLevel *)B->dlv, rt, B->rn2, (double *)nullptr,
            skip);
    blaunch(B, k_b_conv, 1, 0, s, B->total_rhs, B->rn2, (const double *)B->bn2, B->rel, B->scal, 1);
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

}  // namespace

extern "C" {

void dec_batch_default_opts(dec_batch_opts *o) {
    if (!o) return;
    o->block = 256;
    o->kgroup = 0;
    o->nu = 2;
    o->smoother = DEC_SMOOTH_CHEBYSHEV;
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
        (o.kgroup & (o.kgroup - 1)) != 0 || o.kgroup > o.block)
        return fail(Status::fail(DEC_ERR_ARG, "bad batch options (block 128/256/512, 1 <= nu <= 8, kgroup a power of two)"));
    for (int m = 0; m < nmesh; ++m) {
        if (!mgs[m] || mgs[m]->host_only) return fail(Status::fail(DEC_ERR_ARG, "a hierarchy is null or host-only"));
        if (mgs[m]->H.mapped) return fail(Status::fail(DEC_ERR_ARG, "batched solves transfer along binary subdivision (no general maps)"));
        if (nrhs[m] < 1) return fail(Status::fail(DEC_ERR_ARG, "every mesh needs at least one right-hand side"));
    }
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
    cudaGetDevice(&B->device);
    cudaError_t ce = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaStreamCreate"));
    int rc;
    // groups and their level descriptors
    int rhs_base = 0;
    for (int m = 0; m < nmesh; ++m) {
        dec_mg *mg = mgs[m];
        int kg = o.kgroup ? o.kgroup : 1;
        if (!o.kgroup)
            while (kg < nrhs[m] && kg < o.block) kg <<= 1;
        for (int c0 = 0; c0 < nrhs[m]; c0 += kg) {
            const int k = kg;  // the last group of a mesh is padded with zero right-hand sides
            if ((int64_t)mg->lv.back().n * k >= ((int64_t)1 << 31))
                return bail(fail(Status::fail(DEC_ERR_ARG, "vertices x group size must stay below 2^31")));
            int ks = 0;
            while ((1 << ks) < k) ++ks;
            dec_batch::Group G{m, c0, k, (int)B->hlv.size(), (int)mg->lv.size()};
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
                    L.rhs_base = rhs_base;
                    L.gauge = mg->H.bc == DEC_BC_GAUGE;
                    L.s0sum = mg->star0_sum;
                    B->dof += (int64_t)D.n * std::min(k, nrhs[m] - c0);
                }
                B->hlv.push_back(L);
            }
            B->groups.push_back(G);
            rhs_base += k;
        }
    }
    B->total_rhs = rhs_base;
    // cycle schedule aligned by depth below each group's finest level
    std::vector<BTile> tiles;
    const int target = o.block * 8;
    int dmax = 0;
    for (auto &G : B->groups) dmax = std::max(dmax, G.nlev - 1);
    auto op_tiles = [&](int kind, int sweep, int post, int src, int din, int dout, auto &&pick) {
        dec_batch::Op op{kind, (int)tiles.size(), 0, sweep, post, src, din, dout};
        for (auto &G : B->groups) pick(G, tiles);
        op.cnt = (int)tiles.size() - op.off;
        if (op.cnt > 0) B->cycle_ops.push_back(op);
    };
    const int cheb = o.smoother == DEC_SMOOTH_CHEBYSHEV;
    for (int d = 0; d < dmax; ++d) {
        auto at_depth = [&](const dec_batch::Group &G) { return G.nlev - 1 - d; };  // level index, -1 if none
        // pre-smoothing: sweep 0 from zero, then ping-pong
        op_tiles(0, 0, 0, 0, 0, (cheb && o.nu > 1), [&](const dec_batch::Group &G, std::vector<BTile> &t) {
            int l = at_depth(G);
            if (l >= 1) add_tiles(t, G.first_lev + l, B->hlv[G.first_lev + l].n, B->hlv[G.first_lev + l].kshift, target);
        });
        int cur = 0;
        for (int sw = 1; sw < o.nu; ++sw) {
            op_tiles(1, sw, 0, cur, cheb, (cheb && sw + 1 < o.nu), [&](const dec_batch::Group &G, std::vector<BTile> &t) {
                int l = at_depth(G);
                if (l >= 1) add_tiles(t, G.first_lev + l, B->hlv[G.first_lev + l].n, B->hlv[G.first_lev + l].kshift, target);
            });
            cur = 1 - cur;
        }
        op_tiles(2, 0, 0, cur, 0, 0, [&](const dec_batch::Group &G, std::vector<BTile> &t) {
            int l = at_depth(G);
            if (l >= 1) add_tiles(t, G.first_lev + l, B->hlv[G.first_lev + l].n, B->hlv[G.first_lev + l].kshift, target);
        });
        op_tiles(3, 0, 0, 0, 0, 0, [&](const dec_batch::Group &G, std::vector<BTile> &t) {
            int l = at_depth(G);
            if (l >= 1) add_tiles(t, G.first_lev + l, B->hlv[G.first_lev + l - 1].n, B->hlv[G.first_lev + l].kshift, target);
        });
    }
    // restriction flag per op: every hierarchy in a batch must use the same restriction
    const int star0 = mgs[0]->H.opts.restriction == DEC_RESTRICT_STAR0;
    for (int m = 1; m < nmesh; ++m)
        if ((mgs[m]->H.opts.restriction == DEC_RESTRICT_STAR0) != (star0 != 0))
            return bail(fail(Status::fail(DEC_ERR_ARG, "all hierarchies of a batch must use the same restriction")));
    for (auto &op : B->cycle_ops)
        if (op.kind == 3) op.src = star0;
    // coarsest solves of every group
    op_tiles(4, 0, 0, 0, 0, 0, [&](const dec_batch::Group &G, std::vector<BTile> &t) {
        add_tiles(t, G.first_lev, B->hlv[G.first_lev].n, B->hlv[G.first_lev].kshift, target);
    });
    const int after_pre = (o.nu - 1) % 2;
    for (int d = dmax - 1; d >= 0; --d) {
        auto at_depth = [&](const dec_batch::Group &G) { return G.nlev - 1 - d; };
        op_tiles(5, 0, 0, after_pre, 0, 0, [&](const dec_batch::Group &G, std::vector<BTile> &t) {
            int l = at_depth(G);
            if (l >= 1) add_tiles(t, G.first_lev + l, B->hlv[G.first_lev + l].n, B->hlv[G.first_lev + l].kshift, target);
        });
        int cur = after_pre;
        for (int sw = 0; sw < o.nu; ++sw) {
            op_tiles(1, sw, 1, cur, (cheb && sw > 0), (cheb && sw + 1 < o.nu),
                     [&](const dec_batch::Group &G, std::vector<BTile> &t) {
                         int l = at_depth(G);
                         if (l >= 1)
                             add_tiles(t, G.first_lev + l, B->hlv[G.first_lev + l].n, B->hlv[G.first_lev + l].kshift, target);
                     });
            cur = 1 - cur;
        }
    }
    // finest items of every group, in larger tiles (fewer per-RHS atomics)
    B->res_off = (int)tiles.size();
    for (auto &G : B->groups) {
        const int l = G.first_lev + G.nlev - 1;
        add_tiles(tiles, l, B->hlv[l].n, B->hlv[l].kshift, o.block * 32);
    }
    B->res_cnt = (int)tiles.size() - B->res_off;
    if ((rc = balloc(B, &B->dtiles, tiles.size())) || (rc = balloc(B, &B->dlv, B->hlv.size())) ||
        (rc = balloc(B, &B->rn2, B->total_rhs)) || (rc = balloc(B, &B->bn2, B->total_rhs)) ||
        (rc = balloc(B, &B->rel, B->total_rhs)) || (rc = balloc(B, &B->msum, B->total_rhs)) ||
        (rc = balloc(B, &B->scal, 1)))
        return bail(rc);
    ce = cudaMemcpy(B->dtiles, tiles.data(), tiles.size() * sizeof(BTile), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(B->dlv, B->hlv.data(), B->hlv.size() * sizeof(BLevel), cudaMemcpyHostToDevice);
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
    {
        int cur = -1;
        CK(cudaGetDevice(&cur));
        if (cur != B->device)
            return fail(Status::fail(DEC_ERR_ARG, "the batch lives on device " + std::to_string(B->device) +
                                                      " but device " + std::to_string(cur) + " is current"));
    }
    for (size_t m = 0; m < B->mgs.size(); ++m)
        if (!b[m] || !x[m]) return fail(Status::fail(DEC_ERR_ARG, "null vector"));
    cudaStream_t s = (cudaStream_t)stream;
    int64_t launches = 0;
    // inputs into group layout, x = 0
    for (auto &G : B->groups) {
        const BLevel &L = B->hlv[G.first_lev + G.nlev - 1];
        const int nr = B->nrhs[G.mesh];
        const int kk = std::min(G.k, nr - G.col0);
        CK(cudaMemsetAsync(L.ox, 0, sizeof(double) * (size_t)L.n * G.k, s));
        blaunch(B, k_b_gather, (int)std::min<int64_t>(4096, ((int64_t)L.n * G.k + B->opts.block - 1) / B->opts.block), 0,
                s, L.n, G.k, kk, nr, G.col0, b[G.mesh], L.ob);
        ++launches;
    }
    Scal *h = B->scal_h;
    std::memset(h, 0, offsetof(Scal, hist));
    h->tol = tol;
    h->maxit = maxit;
    h->max_loops = maxit + 1;
    CK(cudaMemcpyAsync(B->scal, h, offsetof(Scal, hist), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(B->rn2, 0, sizeof(double) * B->total_rhs, s));
    CK(cudaMemsetAsync(B->bn2, 0, sizeof(double) * B->total_rhs, s));
    const BTile *rt = B->dtiles + B->res_off;
    bool any_gauge = false;
    for (auto &L : B->hlv)
        if (L.ox && L.gauge) any_gauge = true;
    if (any_gauge) {
        // (every group's mean is formed; Dirichlet groups are not shifted)
        CK(cudaMemsetAsync(B->msum, 0, sizeof(double) * B->total_rhs, s));
        blaunch(B, k_b_mean, B->res_cnt, sizeof(double) * B->opts.block, s, (const BLevel *)B->dlv, rt, 0, B->msum);
        blaunch(B, k_b_shift, B->res_cnt, 0, s, (const BLevel *)B->dlv, rt, 0, (const double *)B->msum);
        launches += 2;
    }
    blaunch(B, k_b_res64, B->res_cnt, sizeof(double) * B->opts.block, s, (const BLevel *)B->dlv, rt, B->rn2, B->bn2,
            (const int *)nullptr);
    blaunch(B, k_b_conv, 1, 0, s, B->total_rhs, B->rn2, (const double *)B->bn2, B->rel, B->scal, 0);
    launches += 2;
    CK(cudaGetLastError());
    if (maxit > 0) {
        if (!B->loop) {
            int rc = build_loop(B);
            if (rc) return rc;
        }
        CK(cudaGraphLaunch(B->loop, s));
    }
    if (any_gauge) {
        CK(cudaMemsetAsync(B->msum, 0, sizeof(double) * B->total_rhs, s));
        blaunch(B, k_b_mean, B->res_cnt, sizeof(double) * B->opts.block, s, (const BLevel *)B->dlv, rt, 1, B->msum);
        blaunch(B, k_b_shift, B->res_cnt, 0, s, (const BLevel *)B->dlv, rt, 1, (const double *)B->msum);
        launches += 2;
    }
    for (auto &G : B->groups) {
        const BLevel &L = B->hlv[G.first_lev + G.nlev - 1];
        const int nr = B->nrhs[G.mesh];
        const int kk = std::min(G.k, nr - G.col0);
        blaunch(B, k_b_scatter, (int)std::min<int64_t>(4096, ((int64_t)L.n * G.k + B->opts.block - 1) / B->opts.block), 0,
                s, L.n, G.k, kk, nr, G.col0, (const double *)L.ox, x[G.mesh]);
        ++launches;
    }
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
    if (!(h->rel <= tol)) return fail(Status::fail(DEC_ERR_NOT_CONVERGED, "maxit reached before every right-hand side converged"));
    return DEC_OK;
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
                for (int nu : {1, 2, 3}) grid.push_back(dec_batch_opts{blk, kg, nu, DEC_SMOOTH_CHEBYSHEV});
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
    // the first post-smoothing sweep on depth 0 (every group's finest level)
    const dec_batch::Op *op = nullptr;
    for (const auto &o : B->cycle_ops)
        if (o.kind == 1 && o.post == 1 && o.sweep == 0) op = &o;  // the last such op is depth 0
    if (!op) return fail(Status::fail(DEC_ERR_ARG, "batch has no smoothing sweep"));
    cudaStream_t s = (cudaStream_t)stream;
    const int cheb = B->opts.smoother == DEC_SMOOTH_CHEBYSHEV;
    // Algorithmic bytes: the finest operator of each mesh once (K columns + K
    // weights per row, whatever the number of its groups: the groups of a mesh
    // share one table), then per item x, b, x_out (+ direction) for the
    // right-hand sides the mesh actually has (padding columns excluded).
    double by = 0.0;
    std::vector<const int32_t *> seen;
    for (auto &G : B->groups) {
        const BLevel &L = B->hlv[G.first_lev + G.nlev - 1];
        if (std::find(seen.begin(), seen.end(), L.col) == seen.end()) {
            seen.push_back(L.col);
            by += (double)L.n * (8.0 * L.K);
        }
        const int kk = std::min(G.k, B->nrhs[G.mesh] - G.col0);
        by += (double)L.n * kk * 4.0 * (3 + (cheb ? 1 : 0));
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int *noskip = nullptr;
    for (int r = 0; r < 2; ++r)
        blaunch(B, k_b_smooth, op->cnt, 0, s, (const BLevel *)B->dlv, (const BTile *)(B->dtiles + op->off), cheb,
                (float)(2.0 / 3.0), 0, 1, op->src, 0, op->dout, noskip);
    CK(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r)
        blaunch(B, k_b_smooth, op->cnt, 0, s, (const BLevel *)B->dlv, (const BTile *)(B->dtiles + op->off), cheb,
                (float)(2.0 / 3.0), 0, 1, op->src, 0, op->dout, noskip);
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
