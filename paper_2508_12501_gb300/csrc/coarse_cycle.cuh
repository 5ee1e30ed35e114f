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
    CoarseLevel lv[kCoarseMaxLevels];
};

template <typename T>
__device__ __forceinline__ T *sm_at(unsigned char *sm, int off) {
    return reinterpret_cast<T *>(sm + off);
}

// Copy `bytes` (a multiple of 4) from global to shared memory: 16-byte loads,
// two per thread in flight, then the 4-byte tail.  src and the shared
// offset are 16-byte aligned (cudaMalloc'ed arrays, 16-byte aligned layout).
__device__ __forceinline__ void sm_load(unsigned char *sm, int off, const void *src, int bytes) {
    const int n16 = bytes / 16;
    const uint4 *s16 = reinterpret_cast<const uint4 *>(src);
    uint4 *d16 = reinterpret_cast<uint4 *>(sm + off);
    for (int i0 = threadIdx.x; i0 < n16; i0 += 2 * kCoarseThreads) {
        uint4 v[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = i0 + u * kCoarseThreads;
            if (i < n16) v[u] = __ldg(s16 + i);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = i0 + u * kCoarseThreads;
            if (i < n16) d16[i] = v[u];
        }
    }
    const uint32_t *s4 = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d4 = reinterpret_cast<uint32_t *>(sm + off);
    for (int i = 4 * n16 + threadIdx.x; i < bytes / 4; i += kCoarseThreads) d4[i] = __ldg(s4 + i);
}

// s = sum_k w_k (x_i - x_col(k)) and d = sum_k w_k for one row, in slot order
// (row_apply); KT > 0 fixes the slot count at compile time, 0 reads K.
template <int KT>
__device__ __forceinline__ void sm_row(int i, int n, int K, const int16_t *col, const float *w, const float *x,
                                       float &s, float &d) {
    const int Kk = KT > 0 ? KT : K;
    const float xi = x[i];
    s = 0.f;
    d = 0.f;
#pragma unroll
    for (int k = 0; k < (KT > 0 ? KT : kCoarseMaxK); ++k) {
        if (KT == 0 && k >= Kk) break;
        const int o = k * n + i;
        const float wk = w[o];
        s = fmaf(wk, xi - x[col[o]], s);
        d += wk;
    }
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
                float s, d;
                sm_row<KT>(i, n, K, col, w, x, s, d);
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
    pdl_prologue();
    if (skipped(skip)) return;
    extern __shared__ __align__(16) unsigned char sm[];
    const int top = A.top;
    const bool cheb = A.cheb != 0, star0 = A.star0 != 0;
    // operators of every level, then the right-hand side of the top level
    for (int l = 0; l <= top; ++l) {
        const CoarseLevel &L = A.lv[l];
        if (l > 0) {
            sm_load(sm, L.o_col, L.col, ((L.K * L.n * 2) + 3) & ~3);
            sm_load(sm, L.o_w, L.w, L.K * L.n * 4);
            sm_load(sm, L.o_dg, L.dg, L.n * 4);
            sm_load(sm, L.o_par, L.par, (L.n - A.lv[l - 1].n) * 4);
        }
        if (star0) sm_load(sm, L.o_s0, L.s0, L.n * 4);
    }
    sm_load(sm, A.lv[top].o_b, A.b, A.lv[top].n * 4);
    __syncthreads();

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
        for (int i = threadIdx.x; i < L.n; i += kCoarseThreads) {
            float s, d;
            sm_row<KT>(i, L.n, L.K, col, w, x, s, d);
            r[i] = d != 0.f ? b[i] - s : 0.f;
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
    // warp, warp+32, ... and keeps up to 6 of them in flight.
    {
        const CoarseLevel &L0 = A.lv[0];
        const int n0 = L0.n;
        const float *b0 = sm_at<float>(sm, L0.o_b);
        float *x0 = sm_at<float>(sm, L0.o_x);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        constexpr int kW = kCoarseThreads / 32;
        for (int row0 = warp; row0 < n0; row0 += 6 * kW) {
            float acc[6];
#pragma unroll
            for (int m = 0; m < 6; ++m) acc[m] = 0.f;
            for (int j = lane; j < n0; j += 32) {
                const float bj = b0[j];
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    const int row = row0 + m * kW;
                    if (row < n0) acc[m] = fmaf(__ldg(A.G + (size_t)row * n0 + j), bj, acc[m]);
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
