// The coarsest levels of an FP32 V-cycle in one thread block, out of shared
// memory.
//
// Below a few thousand vertices every kernel of the cycle is pure launch and
// L2 latency: about 2 us per dependent launch on GB300, against a fraction
// of a microsecond of work. When the operators of levels 0..top fit in one
// SM's shared memory, one 1024-thread block runs the whole sub-cycle:
//   - pre-smoothing, residual and restriction on each level going down;
//   - the dense coarsest solve;
//   - interpolation and post-smoothing going up.
// __syncthreads separates the phases. Every row is computed with the same
// operations, in the same order, as the one-kernel-per-step cycle
// (k_smooth0, k_smooth, k_residual, k_restrict, k_coarse, k_prolong), so the
// result is bitwise the same (V-cycles, gamma = 1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace decdev {

constexpr int kCoarseThreads = 1024;
constexpr int kCoarseRows = 4;                               // rows per thread and level
constexpr int kCoarseMaxN = kCoarseThreads * kCoarseRows;    // rows per fused level
constexpr int kCoarseMaxLevels = 5;
constexpr int kCoarseMaxNu = 8;
constexpr int kCoarseMaxK = 8;

struct CoarseLevel {
    int n, K;
    // byte offsets of this level's arrays in shared memory (-1: absent)
    int o_col, o_w, o_dg, o_x, o_dir, o_b, o_r, o_s0, o_par;
    // global sources, loaded once per launch
    const int16_t *col;  // [K][n] slot-major, local ids
    const float *w, *dg, *s0;
    const int16_t *par;  // [n - n_coarse][2]
    float e_pre[kCoarseMaxNu], c_pre[kCoarseMaxNu], e_post[kCoarseMaxNu], c_post[kCoarseMaxNu];
};

struct CoarseArgs {
    int top;  // finest level handled here
    int nu1, nu2, cheb, star0;
    const float *G;  // coarsest dense solution operator [n0][n0]
    const float *b;  // right-hand side of level `top` (global)
    float *x;        // result on level `top` (global)
    Scal *S;         // solver scalars: status 3 if the load wait gave up
    int top_mutable; // level `top` is the finest level (its w and dg change with dec_mg_set_star1)
    int wait_rounds; // try_wait rounds the load wait allows before it gives up (status 3)
    CoarseLevel lv[kCoarseMaxLevels];
};

// Shared-memory bytes the kernel keeps before the level arrays (its mbarrier).
constexpr int kCoarseHeader = 16;
// Default try_wait rounds before the load wait gives up (each round suspends
// the thread for at most a hardware time slice, so this bounds the wait to
// well under a second).  The first wait takes CoarseArgs::wait_rounds (this
// value unless the caller set another); the drain wait after a give-up always
// takes this one.
constexpr int kCoarseWaitRounds = 1 << 20;

__device__ __forceinline__ unsigned sm_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase 0 of the load barrier: at most `rounds` try_wait rounds.
__device__ __forceinline__ bool mbar_wait0(unsigned bar, int rounds) {
    for (int it = 0; it < rounds; ++it)
        if (mbar_try_wait(bar, 0)) return true;
    return false;
}

// Thread 0: queue one global -> shared bulk copy of `bytes` (a multiple of 16;
// both addresses 16-byte aligned) completing on the barrier.
__device__ __forceinline__ void bulk_load(unsigned dst, const void *src, unsigned bytes, unsigned bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :
                 : "r"(dst), "l"((unsigned long long)__cvta_generic_to_global(src)), "r"(bytes), "r"(bar)
                 : "memory");
}

// Bytes of an array that go by bulk copy: a 16-byte aligned source up to its
// last 16-byte boundary, nothing from any other source.
__device__ __forceinline__ int bulk_bytes(const void *src, int bytes) {
    return ((uintptr_t)src & 15) == 0 ? bytes & ~15 : 0;
}

// One array of the load phase (`bytes` a multiple of 4): thread 0 queues
// the bulk part (issue == true), the threads copy the rest by plain 4-byte
// loads (issue == false).
__device__ __forceinline__ void stage(unsigned char *sm, int off, const void *src, int bytes, unsigned bar,
                                      bool issue) {
    const int bulk = bulk_bytes(src, bytes);
    if (issue && threadIdx.x == 0 && bulk > 0) bulk_load(sm_addr(sm + off), src, (unsigned)bulk, bar);
    if (issue) return;
    const uint32_t *s4 = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d4 = reinterpret_cast<uint32_t *>(sm + off);
    for (int i = bulk / 4 + threadIdx.x; i < bytes / 4; i += kCoarseThreads) d4[i] = __ldg(s4 + i);
}

template <typename T>
__device__ __forceinline__ T *sm_at(unsigned char *sm, int off) {
    return reinterpret_cast<T *>(sm + off);
}

// s = sum_k w_k (x_i - x_col(k)) for one row, in slot order (row_apply);
// KT > 0 fixes the slot count at compile time, 0 reads K.  The row's
// d = sum_k w_k is the stored diagonal: k_diag adds the same weights in the
// same order, so it is the same float.
template <int KT>
__device__ __forceinline__ float sm_row(int i, int n, int K, const int16_t *col, const float *w, const float *x) {
    const int Kk = KT > 0 ? KT : K;
    const float xi = x[i];
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < (KT > 0 ? KT : kCoarseMaxK); ++k) {
        if (KT == 0 && k >= Kk) break;
        const int o = k * n + i;
        s = fmaf(w[o], xi - x[col[o]], s);
    }
    return s;
}

// One smoothing call of nu steps on level L.
template <int KT>
static __device__ void sm_smooth(unsigned char *sm, const CoarseLevel &L, int nu, bool post, bool cheb) {
    const int n = L.n, K = L.K;
    const int16_t *col = sm_at<int16_t>(sm, L.o_col);
    const float *w = sm_at<float>(sm, L.o_w), *dg = sm_at<float>(sm, L.o_dg), *b = sm_at<float>(sm, L.o_b);
    float *x = sm_at<float>(sm, L.o_x);
    float *dir = cheb ? sm_at<float>(sm, L.o_dir) : nullptr;
    int k0 = 0;
    if (!post) {
        // step 0 from x = 0 (k_smooth0): row-local
        const float e0 = L.e_pre[0];
        const bool dout = cheb && 1 < nu;
        for (int i = threadIdx.x; i < n; i += kCoarseThreads) {
            const float d = dg[i];
            const float v = d != 0.f ? e0 * (b[i] / d) : 0.f;
            x[i] = v;
            if (dout) dir[i] = v;
        }
        __syncthreads();
        k0 = 1;
    }
    for (int k = k0; k < nu; ++k) {
        const float e = post ? L.e_post[k] : L.e_pre[k];
        const float c = post ? L.c_post[k] : L.c_pre[k];
        const bool din = cheb && k > 0, dout = cheb && k + 1 < nu;
        float nx[kCoarseRows], nd[kCoarseRows];
#pragma unroll
        for (int r = 0; r < kCoarseRows; ++r) {
            const int i = threadIdx.x + r * kCoarseThreads;
            if (i < n) {
                const float s = sm_row<KT>(i, n, K, col, w, x), d = dg[i];
                const float q = d != 0.f ? (b[i] - s) / d : 0.f;
                nd[r] = smooth_delta<float>(din, c, din ? dir[i] : 0.f, e, q);
                nx[r] = add_rn(x[i], nd[r]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kCoarseRows; ++r) {
            const int i = threadIdx.x + r * kCoarseThreads;
            if (i < n) {
                x[i] = nx[r];
                if (dout) dir[i] = nd[r];
            }
        }
        __syncthreads();
    }
}

template <int KT>
__global__ void __launch_bounds__(kCoarseThreads, 1) k_coarse_cycle(const __grid_constant__ CoarseArgs A,
                                                                    const int *skip) {
    // Programmatic dependent launch, split: the operators of the coarse
    // levels and G never change after set-up, so their loads are queued
    // before waiting for the previous kernel and overlap its tail.  Only the
    // right-hand side (and the finest level's w and dg, which
    // dec_mg_set_star1 rewrites in stream order) wait.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(16) unsigned char sm[];
    const int top = A.top;
    const bool cheb = A.cheb != 0, star0 = A.star0 != 0;
    // Thread 0 queues one bulk copy per array (all in flight together) on an
    // mbarrier in the shared-memory header, armed with their byte count; the
    // threads copy the unaligned remainders meanwhile, then wait on the
    // barrier.  f(offset, source, bytes, before_wait).
    const unsigned bar = sm_addr(sm);
    auto each_array = [&](auto &&f) {
        for (int l = 0; l <= top; ++l) {
            const CoarseLevel &L = A.lv[l];
            const bool fixed = !(A.top_mutable && l == top);
            if (l > 0) {
                f(L.o_col, L.col, ((L.K * L.n * 2) + 3) & ~3, true);
                f(L.o_w, L.w, L.K * L.n * 4, fixed);
                f(L.o_dg, L.dg, L.n * 4, fixed);
                f(L.o_par, L.par, (L.n - A.lv[l - 1].n) * 4, true);
            }
            if (star0) f(L.o_s0, L.s0, L.n * 4, true);
        }
        f(A.lv[top].o_b, A.b, A.lv[top].n * 4, false);
    };
    if (threadIdx.x == 0) {
        unsigned tx = 0;
        each_array([&](int, const void *src, int bytes, bool pre) {
            if (pre) tx += (unsigned)bulk_bytes(src, bytes);
        });
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
        each_array([&](int off, const void *src, int bytes, bool pre) {
            if (pre) stage(sm, off, src, bytes, bar, true);
        });
        // G is read on the way back up: start it towards L2 now
        const int gbytes = (A.lv[0].n * A.lv[0].n * 4) & ~15;
        if (gbytes > 0 && ((uintptr_t)A.G & 15) == 0)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                             (unsigned long long)__cvta_generic_to_global(A.G)),
                         "r"(gbytes)
                         : "memory");
    }
    each_array([&](int off, const void *src, int bytes, bool pre) {
        if (pre) stage(sm, off, src, bytes, bar, false);
    });
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const bool skip_now = skipped(skip);
    if (threadIdx.x == 0) {
        unsigned tx = 0;
        if (!skip_now)
            each_array([&](int, const void *src, int bytes, bool pre) {
                if (!pre) tx += (unsigned)bulk_bytes(src, bytes);
            });
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
        if (!skip_now)
            each_array([&](int off, const void *src, int bytes, bool pre) {
                if (!pre) stage(sm, off, src, bytes, bar, true);
            });
    }
    if (!skip_now)
        each_array([&](int off, const void *src, int bytes, bool pre) {
            if (!pre) stage(sm, off, src, bytes, bar, false);
        });
    __syncthreads();  // the barrier is initialized before anyone waits on it
    const bool loaded = mbar_wait0(bar, A.wait_rounds);
    if (!__syncthreads_and(loaded)) {
        // copies still in flight after the bound: report, wait once more with the full
        // (bounded) limit so that no copy lands in shared memory after the block has left,
        // and leave x untouched
        if (threadIdx.x == 0) {
            A.S->status = 3;
            A.S->done = 1;
        }
        mbar_wait0(bar, kCoarseWaitRounds);
        return;
    }
    if (skip_now) return;  // the queued copies have landed

    // down: smooth from zero, residual, restriction
    for (int l = top; l >= 1; --l) {
        const CoarseLevel &L = A.lv[l], &C = A.lv[l - 1];
        if (A.nu1 > 0) {
            sm_smooth<KT>(sm, L, A.nu1, false, cheb);
        } else {
            float *x = sm_at<float>(sm, L.o_x);
            for (int i = threadIdx.x; i < L.n; i += kCoarseThreads) x[i] = 0.f;
            __syncthreads();
        }
        const int16_t *col = sm_at<int16_t>(sm, L.o_col);
        const float *w = sm_at<float>(sm, L.o_w), *b = sm_at<float>(sm, L.o_b), *x = sm_at<float>(sm, L.o_x);
        float *r = sm_at<float>(sm, L.o_r);
        const float *dg = sm_at<float>(sm, L.o_dg);
        for (int i = threadIdx.x; i < L.n; i += kCoarseThreads) {
            const float s = sm_row<KT>(i, L.n, L.K, col, w, x);
            r[i] = dg[i] != 0.f ? b[i] - s : 0.f;
        }
        __syncthreads();
        float *bc = sm_at<float>(sm, C.o_b);
        const float *s0f = star0 ? sm_at<float>(sm, L.o_s0) : nullptr;
        const float *s0c = star0 ? sm_at<float>(sm, C.o_s0) : nullptr;
        for (int c = threadIdx.x; c < C.n; c += kCoarseThreads) {
            float acc = 0.f;
            int deg = 0;
            const int Kk = KT > 0 ? KT : L.K;
#pragma unroll
            for (int k = 0; k < (KT > 0 ? KT : kCoarseMaxK); ++k) {
                if (KT == 0 && k >= Kk) break;
                const int j = col[k * L.n + c];
                if (j != c) {
                    acc = star0 ? fmaf(s0f[j], r[j], acc) : acc + r[j];
                    ++deg;
                }
            }
            bc[c] = star0 ? fmaf(s0f[c], r[c], 0.5f * acc) / s0c[c]
                          : fmaf(0.5f, acc, r[c]) / add_rn(1.f, mul_rn(0.5f, (float)deg));
        }
        __syncthreads();
    }

    // coarsest: x0 = G b0.  Each row is summed as in k_coarse (lane l adds
    // columns l, l+32, ... with fma, then a butterfly); a warp takes rows
    // warp, warp+32, ... and keeps up to 6 of them in flight.  G is read from
    // L2 in batches of 32 kCj columns: every load of a batch is issued before
    // its first fma, so a batch costs one round trip (n0 <= 192: one batch).
    {
        const CoarseLevel &L0 = A.lv[0];
        const int n0 = L0.n;
        const float *b0 = sm_at<float>(sm, L0.o_b);
        float *x0 = sm_at<float>(sm, L0.o_x);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        constexpr int kW = kCoarseThreads / 32;
        constexpr int kCj = 6;
        for (int row0 = warp; row0 < n0; row0 += 6 * kW) {
            float acc[6];
#pragma unroll
            for (int m = 0; m < 6; ++m) acc[m] = 0.f;
            for (int j0 = 0; j0 < n0; j0 += 32 * kCj) {
                float g[kCj][6];
#pragma unroll
                for (int c = 0; c < kCj; ++c) {
                    const int j = j0 + c * 32 + lane;
#pragma unroll
                    for (int m = 0; m < 6; ++m) {
                        const int row = row0 + m * kW;
                        g[c][m] = (row < n0 && j < n0) ? __ldg(A.G + (size_t)row * n0 + j) : 0.f;
                    }
                }
#pragma unroll
                for (int c = 0; c < kCj; ++c) {
                    const int j = j0 + c * 32 + lane;
                    if (j < n0) {
                        const float bj = b0[j];
#pragma unroll
                        for (int m = 0; m < 6; ++m)
                            if (row0 + m * kW < n0) acc[m] = fmaf(g[c][m], bj, acc[m]);
                    }
                }
            }
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                float a = acc[m];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                const int row = row0 + m * kW;
                if (lane == 0 && row < n0) x0[row] = a;
            }
        }
        __syncthreads();
    }

    // up: interpolation and correction, post-smoothing
    for (int l = 1; l <= top; ++l) {
        const CoarseLevel &L = A.lv[l], &C = A.lv[l - 1];
        const float *ec = sm_at<float>(sm, C.o_x);
        const int16_t *par = sm_at<int16_t>(sm, L.o_par);
        float *x = sm_at<float>(sm, L.o_x);
        for (int v = threadIdx.x; v < L.n; v += kCoarseThreads) {
            const float add = v < C.n ? ec[v] : mul_rn(0.5f, add_rn(ec[par[2 * (v - C.n)]], ec[par[2 * (v - C.n) + 1]]));
            x[v] = add_rn(x[v], add);
        }
        __syncthreads();
        if (A.nu2 > 0) sm_smooth<KT>(sm, L, A.nu2, true, cheb);
    }

    const float *xt = sm_at<float>(sm, A.lv[top].o_x);
    for (int i = threadIdx.x; i < A.lv[top].n; i += kCoarseThreads) A.x[i] = xt[i];
}

}  // namespace decdev
