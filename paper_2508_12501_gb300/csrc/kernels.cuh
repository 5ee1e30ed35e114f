// sm_103a kernels of the DEC multigrid hot path.
//
// Operator rows are stored ELL-style, slot-major: slot k of row i is at
// [k * n + i] so a warp's loads of one slot are contiguous.  A row computes
//   s = sum_k w_k (x_i - x_col(k)) = (L x)_i,   d = sum_k w_k = L_ii,
// with w_k = *1_e / *0_i (Sec. 3.1.1, Eq. hodge0-laplacian as -Delta_0).
// Dirichlet rows have all weights 0, hence d == 0, which every kernel uses
// as the "fixed vertex" mask.  Padding slots point at the row with weight 0.
//
// Every kernel takes `skip`: when non-null and *skip != 0 the kernel returns
// at once (used to retire queued iterations after convergence).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace decdev {

constexpr int kThreads = 256;
// Partial-sum slots per reduction: at least the one-wave reduction grid of
// GB300 (8 blocks on each of 152 SMs = 1216), a multiple of 4 (float4 reads
// of the FP32 partials) and of kThreads (the FP64 tail's rounds).
constexpr int kMaxRedBlocks = 1280;
constexpr int kHist = 1024;          // residual history entries

// Scalars of the outer iteration, resident in device memory.
struct Scal {
    double rz;          // <r, z> (*0 inner product)
    double alpha, beta;
    double c;           // gauge shift of the current preconditioned vector
    double bnorm2, rnorm2, rel, rel0;
    double tol;
    double star0_sum;   // sum of *0 over free vertices
    double mean;        // result of the last k_mean
    double scale;       // power-of-two scale of the ff outer iteration (set by k_outer_init)
    double iscale, iscale2;  // 1 / scale and 1 / scale^2 (exact)
    double thr2;        // stopping threshold on ||r||^2: tol^2 ||b||^2 (+inf for b = 0)
    double rnorm2_0;    // ||r||^2 of the initial iterate
    double inv_star0_sum;  // 1 / star0_sum
    float alpha_hi, alpha_lo;  // alpha as an ff pair
    float beta_f, c_f;         // beta and the gauge shift rounded to FP32
    int iter, maxit, done, status;  // status: 0 ok, 1 non-finite, 2 stalled (alpha = 0), 3 a device wait gave up
    int loops, max_loops;           // device-side iteration loop: executions and hard cap
    double hist[kHist];
};

// Programmatic dependent launch: let the next kernel in the stream start its
// launch now, then wait until the previous kernel has finished and its writes
// are visible.  Without the launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// The same for the kernels that rewrite operator tables (weights, diagonals):
// they let dependents start only when they finish, so a kernel that reads a
// table before its own wait (pdl_prologue_ell) never overlaps a writer of it.
__device__ __forceinline__ void pdl_wait_only() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// Programmatic dependent launch for a kernel over the rows of a level: before
// waiting for the previous kernel, pull this thread's first row's slots of
// the level's ELL tables (columns, weights) into L1.  The tables do not
// depend on the previous kernel, so the row loop's first table loads after
// the wait need not go to L2.  w2 (may be null) is a second weight table.
template <int KT, typename TW>
__device__ __forceinline__ void pdl_prologue_ell(int n, int K, const int32_t *col, const TW *w,
                                                 const TW *w2 = nullptr) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int Kk = KT > 0 ? KT : K;
#pragma unroll
        for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
            if (KT == 0 && k >= Kk) break;
            const size_t o = (size_t)k * n + i;
            prefetch_l1(col + o);
            prefetch_l1(w + o);
            if (w2) prefetch_l1(w2 + o);
        }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ bool skipped(const int *skip) { return skip != nullptr && *skip != 0; }

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// Round-to-nearest add and multiply that the compiler may not contract into
// an FMA: every kernel that forms the same smoothing update or interpolated
// value rounds it identically, so fused and unfused cycles agree bit for bit.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// One smoothing update: delta = c d_in + e q (DIN) or e q; x_out = x_in + delta.
template <typename T>
__device__ __forceinline__ T smooth_delta(bool din, T c, T d_in, T e, T q) {
    return din ? fma(c, d_in, mul_rn(e, q)) : mul_rn(e, q);
}

// (L x)_i and L_ii for one row.
template <typename T, int KT>
__device__ __forceinline__ void row_apply(int i, int n, int K, const int32_t *__restrict__ col,
                                          const T *__restrict__ w, const T *__restrict__ x, T &s, T &d) {
    const int Kk = KT > 0 ? KT : K;
    const T xi = ldg(x + i);
    s = T(0);
    d = T(0);
#pragma unroll
    for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
        if (KT == 0 && k >= Kk) break;
        const size_t o = (size_t)k * n + i;
        const int c = ldg(col + o);
        const T wk = ldg(w + o);
        s = fma(wk, xi - ldg(x + c), s);
        d += wk;
    }
}

// Grid-stride loop over rows, unrolled by two: a thread's next row issues its
// loads while the previous row's gathers are in flight (measured 9-19 % on
// the finest smoothing sweep).  Rows keep their order, so per-thread sums
// and results are unchanged.
#define GRID_STRIDE(i, n) \
    _Pragma("unroll 2") for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)
// The same loop not unrolled, for kernels whose two rows do not fit in 32 registers.
#define GRID_STRIDE_1(i, n) for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)
// The loop unrolled by four, for the kernels whose per-row work and sums are
// FP64: they run kFp64Blocks blocks per SM (a wave of them, red_grid64) with
// up to 64 registers, so four rows' loads are in flight per thread.
#define GRID_STRIDE_4(i, n) \
    _Pragma("unroll 4") for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)
constexpr int kFp64Blocks = 4;

// y = L x
template <typename T, int KT>
__global__ void __launch_bounds__(kThreads, 8) k_apply(int n, int K, const int32_t *__restrict__ col,
                                                   const T *__restrict__ w, const T *__restrict__ x,
                                                   T *__restrict__ y, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    GRID_STRIDE(i, n) {
        T s, d;
        row_apply<T, KT>(i, n, K, col, w, x, s, d);
        y[i] = s;
    }
}

// r = b - L x on free rows, 0 on fixed rows
template <typename T, int KT>
__global__ void __launch_bounds__(kThreads, 8) k_residual(int n, int K, const int32_t *__restrict__ col,
                                                      const T *__restrict__ w, const T *__restrict__ b,
                                                      const T *__restrict__ x, T *__restrict__ r,
                                                      const int *skip) {
    pdl_prologue_ell<KT>(n, K, col, w);
    if (skipped(skip)) return;
    GRID_STRIDE(i, n) {
        T s, d;
        row_apply<T, KT>(i, n, K, col, w, x, s, d);
        r[i] = d != T(0) ? ldg(b + i) - s : T(0);
    }
}

// Several right-hand sides interleaved, value j of vertex v at [v k + j]:
// y = L x (RES = false) or r = b - L x on free rows, 0 on fixed rows (RES).
template <typename T, bool RES>
__global__ void __launch_bounds__(kThreads, 8) k_apply_k(int n, int K, int k, const int32_t *__restrict__ col,
                                                     const T *__restrict__ w, const T *__restrict__ x,
                                                     const T *__restrict__ b, T *__restrict__ y) {
    pdl_prologue();
    const int64_t items = (int64_t)n * k;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < items; it += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(it / k), j = (int)(it % k);
        const T xi = ldg(x + it);
        T s = T(0), d = T(0);
        for (int q = 0; q < K; ++q) {
            const size_t o = (size_t)q * n + i;
            const T wq = ldg(w + o);
            s = fma(wq, xi - ldg(x + (size_t)ldg(col + o) * k + j), s);
            d += wq;
        }
        y[it] = RES ? (d != T(0) ? ldg(b + it) - s : T(0)) : s;
    }
}

// Column j of an interleaved [n][k] vector to a contiguous one (gather) and back (scatter).
template <typename T>
__global__ void __launch_bounds__(kThreads, 8) k_col_gather(int n, int k, int j, const T *__restrict__ src,
                                                        T *__restrict__ dst) {
    pdl_prologue();
    GRID_STRIDE(i, n) dst[i] = src[(size_t)i * k + j];
}
template <typename T>
__global__ void __launch_bounds__(kThreads, 8) k_col_scatter(int n, int k, int j, const T *__restrict__ src,
                                                         T *__restrict__ dst) {
    pdl_prologue();
    GRID_STRIDE(i, n) dst[(size_t)i * k + j] = src[i];
}

// One smoothing step from a nonzero iterate:
//   q = D^-1 (b - L x);  delta = c * d_in + e * q;  x_out = x_in + delta;  d_out = delta.
// Damped Jacobi: DIN = DOUT = false, e = omega.  Chebyshev: the first step of
// a smoothing call has DIN = false, later steps DIN = true; DOUT is false on
// the last step (its direction is never read).
template <typename T, int KT, bool DIN, bool DOUT>
__global__ void __launch_bounds__(kThreads, 8) k_smooth(int n, int K, const int32_t *__restrict__ col,
                                                    const T *__restrict__ w, const T *__restrict__ b,
                                                    const T *__restrict__ x_in, const T *__restrict__ d_in,
                                                    T *__restrict__ x_out, T *__restrict__ d_out, T c, T e,
                                                    const int *skip) {
    pdl_prologue_ell<KT>(n, K, col, w);
    if (skipped(skip)) return;
    GRID_STRIDE(i, n) {
        T s, d;
        row_apply<T, KT>(i, n, K, col, w, x_in, s, d);
        T q = d != T(0) ? (ldg(b + i) - s) / d : T(0);
        const T delta = smooth_delta<T>(DIN, c, DIN ? ldg(d_in + i) : T(0), e, q);
        x_out[i] = add_rn(ldg(x_in + i), delta);
        if (DOUT) d_out[i] = delta;
    }
}

// First smoothing step from x = 0: x_out = e * D^-1 b (and d_out = x_out).
template <typename T, int KT, bool DOUT>
__global__ void __launch_bounds__(kThreads, 8) k_smooth0(int n, int K, const T *__restrict__ w,
                                                     const T *__restrict__ b, T *__restrict__ x_out,
                                                     T *__restrict__ d_out, T e, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const int Kk = KT > 0 ? KT : K;
    GRID_STRIDE(i, n) {
        T d = T(0);
#pragma unroll
        for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
            if (KT == 0 && k >= Kk) break;
            d += ldg(w + (size_t)k * n + i);
        }
        T v = d != T(0) ? e * (ldg(b + i) / d) : T(0);
        x_out[i] = v;
        if (DOUT) d_out[i] = v;
    }
}

// FP64 cycles (mode f64): the same three kernels with each row's diagonal
// read from the stored table (k_diag) instead of summed again.  k_diag adds
// the same weights in the same order, so the value is the same double; on
// GB300's narrow FP64 pipe its six additions per row cost more than the
// 8-byte load (an FP64 sweep issues about 31 FP64 instructions per row
// otherwise).
template <int KT>
__device__ __forceinline__ double row_sum64(int i, int n, int K, const int32_t *__restrict__ col,
                                            const double *__restrict__ w, const double *__restrict__ x) {
    const int Kk = KT > 0 ? KT : K;
    const double xi = ldg(x + i);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
        if (KT == 0 && k >= Kk) break;
        const size_t o = (size_t)k * n + i;
        s = fma(ldg(w + o), xi - ldg(x + ldg(col + o)), s);
    }
    return s;
}

template <int KT, bool DIN, bool DOUT>
__global__ void __launch_bounds__(kThreads, 8) k_smooth_dg(int n, int K, const int32_t *__restrict__ col,
                                                       const double *__restrict__ w, const double *__restrict__ dg,
                                                       const double *__restrict__ b, const double *__restrict__ x_in,
                                                       const double *__restrict__ d_in, double *__restrict__ x_out,
                                                       double *__restrict__ d_out, double c, double e,
                                                       const int *skip) {
    pdl_prologue_ell<KT>(n, K, col, w);
    if (skipped(skip)) return;
    GRID_STRIDE(i, n) {
        const double s = row_sum64<KT>(i, n, K, col, w, x_in), d = ldg(dg + i);
        double q = d != 0.0 ? (ldg(b + i) - s) / d : 0.0;
        const double delta = smooth_delta<double>(DIN, c, DIN ? ldg(d_in + i) : 0.0, e, q);
        x_out[i] = add_rn(ldg(x_in + i), delta);
        if (DOUT) d_out[i] = delta;
    }
}

template <int KT>
__global__ void __launch_bounds__(kThreads, 8) k_residual_dg(int n, int K, const int32_t *__restrict__ col,
                                                         const double *__restrict__ w, const double *__restrict__ dg,
                                                         const double *__restrict__ b, const double *__restrict__ x,
                                                         double *__restrict__ r, const int *skip) {
    pdl_prologue_ell<KT>(n, K, col, w);
    if (skipped(skip)) return;
    GRID_STRIDE(i, n) {
        const double s = row_sum64<KT>(i, n, K, col, w, x);
        r[i] = ldg(dg + i) != 0.0 ? ldg(b + i) - s : 0.0;
    }
}

template <bool DOUT>
__global__ void __launch_bounds__(kThreads, 8) k_smooth0_dg(int n, const double *__restrict__ dg,
                                                        const double *__restrict__ b, double *__restrict__ x_out,
                                                        double *__restrict__ d_out, double e, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    GRID_STRIDE(i, n) {
        const double d = ldg(dg + i);
        const double v = d != 0.0 ? e * (ldg(b + i) / d) : 0.0;
        x_out[i] = v;
        if (DOUT) d_out[i] = v;
    }
}

// One multicolour Gauss-Seidel step over the rows of one colour class (rows
// listed in `rows`): x_i += (b_i - (L x)_i) / L_ii in place.  Rows of one
// colour are never neighbours, so every row reads the current values of the
// other colours and no row of the class is read while it is written.
template <typename T, int KT>
__global__ void __launch_bounds__(kThreads, 8) k_mcgs(int n, int K, const int32_t *__restrict__ col,
                                                  const T *__restrict__ w, const T *__restrict__ b, T *x,
                                                  const int32_t *__restrict__ rows, int cnt, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    GRID_STRIDE(t, cnt) {
        const int i = ldg(rows + t);
        T s, d;
        row_apply<T, KT>(i, n, K, col, w, x, s, d);
        if (d != T(0)) x[i] = add_rn(x[i], (ldg(b + i) - s) / d);
    }
}

// Row sums d_i = sum_k w_k (the Jacobi diagonal), summed in slot order as
// k_smooth0 and row_apply do, so the fused kernels below read the same value.
template <typename T, int KT>
__global__ void __launch_bounds__(kThreads, 8) k_diag(int n, int K, const T *__restrict__ w, T *__restrict__ dg) {
    pdl_wait_only();
    const int Kk = KT > 0 ? KT : K;
    GRID_STRIDE(i, n) {
        T d = T(0);
#pragma unroll
        for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
            if (KT == 0 && k >= Kk) break;
            d += ldg(w + (size_t)k * n + i);
        }
        dg[i] = d;
    }
}

// ---------------------------------------------------------------------------
// Fused cycle kernels.  Each replaces two consecutive launches of the cycle
// and recomputes, per neighbour, the value the first would have stored, with
// the same operations in the same order -- so the results are bitwise those
// of the separate kernels, with one launch and one vector pass fewer.
// ---------------------------------------------------------------------------

// The first two smoothing steps from x = 0 (k_smooth0, then k_smooth with
// DIN = Chebyshev): x1_j = e0 (b_j / d_j) is formed for row i and each
// neighbour from b and the stored diagonal.  nu >= 2.
template <typename T, int KT, bool CHEB, bool DOUT>
__global__ void __launch_bounds__(kThreads, 8) k_smooth01(int n, int K, const int32_t *__restrict__ col,
                                                      const T *__restrict__ w, const T *__restrict__ dg,
                                                      const T *__restrict__ b, T *__restrict__ x_out,
                                                      T *__restrict__ d_out, T e0, T c1, T e1, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const int Kk = KT > 0 ? KT : K;
    GRID_STRIDE(i, n) {
        const T di = ldg(dg + i);
        const T bi = ldg(b + i);
        const T x1i = di != T(0) ? e0 * (bi / di) : T(0);
        T s = T(0);
#pragma unroll
        for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
            if (KT == 0 && k >= Kk) break;
            const size_t o = (size_t)k * n + i;
            const int j = ldg(col + o);
            const T dj = ldg(dg + j);
            const T x1j = dj != T(0) ? e0 * (ldg(b + j) / dj) : T(0);
            s = fma(ldg(w + o), x1i - x1j, s);
        }
        const T q = di != T(0) ? (bi - s) / di : T(0);
        const T delta = smooth_delta<T>(CHEB, c1, x1i, e1, q);
        x_out[i] = add_rn(x1i, delta);
        if (DOUT) d_out[i] = delta;
    }
}

// What k_prolong adds to fine vertex v.
template <typename T>
__device__ __forceinline__ T prolong_add(int v, int nc, const int2 *__restrict__ par, const T *__restrict__ ec) {
    if (v < nc) return ldg(ec + v);
    const int2 p = ldg(par + (v - nc));
    return mul_rn(T(0.5), add_rn(ldg(ec + p.x), ldg(ec + p.y)));
}

// Interpolation and correction (k_prolong) followed by the first step of the
// post-smoothing call (k_smooth, DIN = false): x'_j = x_j + (P e)_j is formed
// for row i and each neighbour; x_in keeps the uncorrected iterate.
template <typename T, int KT, bool DOUT>
__global__ void __launch_bounds__(kThreads, 8) k_prolong_smooth(int n, int K, int nc, const int2 *__restrict__ par,
                                                            const T *__restrict__ ec, const int32_t *__restrict__ col,
                                                            const T *__restrict__ w, const T *__restrict__ dg,
                                                            const T *__restrict__ b, const T *__restrict__ x_in,
                                                            T *__restrict__ x_out, T *__restrict__ d_out, T e0,
                                                            const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const int Kk = KT > 0 ? KT : K;
    GRID_STRIDE(i, n) {
        const T xi = add_rn(ldg(x_in + i), prolong_add(i, nc, par, ec));
        T s = T(0);
#pragma unroll
        for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
            if (KT == 0 && k >= Kk) break;
            const size_t o = (size_t)k * n + i;
            const int j = ldg(col + o);
            const T xj = add_rn(ldg(x_in + j), prolong_add(j, nc, par, ec));
            s = fma(ldg(w + o), xi - xj, s);
        }
        const T di = ldg(dg + i);
        const T q = di != T(0) ? (ldg(b + i) - s) / di : T(0);
        const T delta = smooth_delta<T>(false, T(0), T(0), e0, q);
        x_out[i] = add_rn(xi, delta);
        if (DOUT) d_out[i] = delta;
    }
}

// Residual (k_residual) followed by restriction (k_restrict): a group of 8
// lanes per coarse row c; lane 0 forms r_f at fine row c, lane k+1 at the
// fine neighbour in slot k (a midpoint of a coarse edge at c), and lane 0
// adds them in slot order.  Requires K <= 7.  S0 > 0 also runs the coarse
// level's first smoothing step from zero on the new row, as k_restrict does.
template <typename T, int KT, bool STAR0, int S0 = 0>
__global__ void __launch_bounds__(kThreads, 8) k_residual_restrict(int nc, int nf, int K, const int32_t *__restrict__ col,
                                                               const T *__restrict__ w, const T *__restrict__ b,
                                                               const T *__restrict__ x, T *__restrict__ bc,
                                                               const T *__restrict__ s0f, const T *__restrict__ s0c,
                                                               const int *skip, const T *__restrict__ dgc,
                                                               T *__restrict__ xc, T *__restrict__ dc, T e0) {
    pdl_prologue();
    if (skipped(skip)) return;
    const int Kk = KT > 0 ? KT : K;
    const int lane8 = threadIdx.x & 7;
    const int base = threadIdx.x & 31 & ~7;
    const unsigned gmask = 0xFFu << base;
    const int groups = (int)((gridDim.x * blockDim.x) >> 3);
    for (int c = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 3); c < nc; c += groups) {
        int j = c;
        bool valid = lane8 == 0;
        if (lane8 > 0 && lane8 <= Kk) {
            j = ldg(col + (size_t)(lane8 - 1) * nf + c);
            valid = j != c;
        }
        T r = T(0), sj = T(0);
        if (valid) {
            T s, d;
            row_apply<T, KT>(j, nf, K, col, w, x, s, d);
            r = d != T(0) ? ldg(b + j) - s : T(0);
            if (STAR0) sj = ldg(s0f + j);
        }
        T acc = T(0);
        int deg = 0;
        for (int k = 0; k < Kk; ++k) {
            const T rk = __shfl_sync(gmask, r, base + k + 1);
            const T sk = STAR0 ? __shfl_sync(gmask, sj, base + k + 1) : T(0);
            const int vk = __shfl_sync(gmask, (int)valid, base + k + 1);
            if (vk) {
                acc = STAR0 ? fma(sk, rk, acc) : acc + rk;
                ++deg;
            }
        }
        if (lane8 == 0) {
            T v;
            if (STAR0)
                v = fma(sj, r, T(0.5) * acc) / ldg(s0c + c);
            else
                v = fma(T(0.5), acc, r) / add_rn(T(1), mul_rn(T(0.5), T(deg)));
            bc[c] = v;
            if (S0 > 0) {
                const T d = ldg(dgc + c);
                const T x1 = d != T(0) ? e0 * (v / d) : T(0);
                xc[c] = x1;
                if (S0 == 2) dc[c] = x1;
            }
        }
    }
}

// y = x (same precision)
template <typename T>
__global__ void __launch_bounds__(kThreads, 8) k_copy(int n, const T *__restrict__ x, T *__restrict__ y, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    GRID_STRIDE(i, n) y[i] = ldg(x + i);
}

// x += e (same precision)
template <typename T>
__global__ void __launch_bounds__(kThreads, 8) k_axpy1(int n, const T *__restrict__ e, T *__restrict__ x,
                                                   const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    GRID_STRIDE(i, n) x[i] += ldg(e + i);
}

// Restriction by the row-normalized subdivision matrix (Sec. 2.2.1):
//   b_c[c] = (r_f[c] + 1/2 sum_{midpoints m adjacent to c} r_f[m]) / (1 + deg(c)/2).
// The fine neighbours of a coarse vertex are exactly the midpoints of its
// coarse edges, so the fine ELL row c lists them (padding: col == c).
// With STAR0 the *0-adjoint of interpolation is applied instead:
//   b_c[c] = (s_f[c] r_f[c] + 1/2 sum_m s_f[m] r_f[m]) / s_c[c],  s = *0.
// S0 > 0 also runs the first smoothing step of the coarse level from zero
// on the new row (k_smooth0: xc = e0 bc / dgc, and dc = xc when S0 == 2):
// row-local, so it costs no gathers.
template <typename T, int KT, bool STAR0, int S0 = 0>
__global__ void __launch_bounds__(kThreads, 8) k_restrict(int nc, int nf, int Kf, const int32_t *__restrict__ colf,
                                                      const T *__restrict__ rf, T *__restrict__ bc,
                                                      const T *__restrict__ s0f, const T *__restrict__ s0c,
                                                      const int *skip, const T *__restrict__ dgc,
                                                      T *__restrict__ xc, T *__restrict__ dc, T e0) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    {
        // this thread's first coarse row: its fine column slots, before the wait (see pdl_prologue_ell)
        const int c = blockIdx.x * blockDim.x + threadIdx.x;
        if (c < nc) {
#pragma unroll
            for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
                if (KT == 0 && k >= Kf) break;
                prefetch_l1(colf + (size_t)k * nf + c);
            }
        }
    }
    pdl_wait_only();
    if (skipped(skip)) return;
    const int Kk = KT > 0 ? KT : Kf;
    GRID_STRIDE(c, nc) {
        T acc = T(0);
        int deg = 0;
#pragma unroll
        for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
            if (KT == 0 && k >= Kk) break;
            const int j = ldg(colf + (size_t)k * nf + c);
            if (j != c) {
                acc = STAR0 ? fma(ldg(s0f + j), ldg(rf + j), acc) : acc + ldg(rf + j);
                ++deg;
            }
        }
        // explicit fma: the fused k_residual_restrict rounds identically
        T v;
        if (STAR0)
            v = fma(ldg(s0f + c), ldg(rf + c), T(0.5) * acc) / ldg(s0c + c);
        else
            v = fma(T(0.5), acc, ldg(rf + c)) / add_rn(T(1), mul_rn(T(0.5), T(deg)));
        bc[c] = v;
        if (S0 > 0) {
            const T d = ldg(dgc + c);
            const T x1 = d != T(0) ? e0 * (v / d) : T(0);
            xc[c] = x1;
            if (S0 == 2) dc[c] = x1;
        }
    }
}

// Interpolation by the subdivision matrix and correction (Sec. 2.2.1):
//   x_f[v] += e_c[v] for coarse ids, x_f[nc + m] += (e_c[a] + e_c[b]) / 2 for the midpoint of (a, b).
template <typename T>
__global__ void __launch_bounds__(kThreads, 8) k_prolong(int nc, int nf, const int2 *__restrict__ par,
                                                     const T *__restrict__ ec, T *__restrict__ xf,
                                                     const int *skip) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    {
        // this thread's first midpoint's parents, before the wait (see pdl_prologue_ell)
        const int v = blockIdx.x * blockDim.x + threadIdx.x;
        if (v >= nc && v < nf) prefetch_l1(par + (v - nc));
    }
    pdl_wait_only();
    if (skipped(skip)) return;
    GRID_STRIDE(v, nf) xf[v] = add_rn(xf[v], prolong_add(v, nc, par, ec));
}

// Interpolation along a general geometric map (Sec. 2.2.1; cubic subdivision):
// x_f[v] += sum_q w_q e_c[idx_q], three slots per fine vertex (unused: w = 0).
template <typename T>
__global__ void __launch_bounds__(kThreads, 8) k_prolong_map(int nf, const int32_t *__restrict__ idx,
                                                         const T *__restrict__ w, const T *__restrict__ ec,
                                                         T *__restrict__ xf, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    GRID_STRIDE(v, nf) {
        T a = T(0);
#pragma unroll
        for (int q = 0; q < 3; ++q) a = fma(ldg(w + (size_t)q * nf + v), ldg(ec + ldg(idx + (size_t)q * nf + v)), a);
        xf[v] = add_rn(xf[v], a);
    }
}

// Restriction along a general geometric map: b_c[c] = sum_q rw_q r_f[ridx_q], the
// rows of the transpose of the row-normalized map (or of the *0-adjoint).
template <typename T>
__global__ void __launch_bounds__(kThreads, 8) k_restrict_map(int nc, int Kr, const int32_t *__restrict__ ridx,
                                                          const T *__restrict__ rw, const T *__restrict__ rf,
                                                          T *__restrict__ bc, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    GRID_STRIDE(c, nc) {
        T a = T(0);
        for (int q = 0; q < Kr; ++q) a = fma(ldg(rw + (size_t)q * nc + c), ldg(rf + ldg(ridx + (size_t)q * nc + c)), a);
        bc[c] = a;
    }
}

// Coarsest level: x = G b with the dense precomputed solution operator, one warp per row.
template <typename T>
__global__ void __launch_bounds__(kThreads, 8) k_coarse(int n0, const T *__restrict__ G, const T *__restrict__ b,
                                                    T *__restrict__ x, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < n0; r += nwarps) {
        T acc = T(0);
        for (int j = lane; j < n0; j += 32) acc = fma(ldg(G + (size_t)r * n0 + j), ldg(b + j), acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) x[r] = acc;
    }
}

template <typename TD, typename TS>
__global__ void __launch_bounds__(kThreads, 8) k_cast(int n, const TS *__restrict__ src, TD *__restrict__ dst,
                                                  const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    GRID_STRIDE(i, n) dst[i] = (TD)ldg(src + i);
}

// x += (double) e
template <typename TE>
__global__ void __launch_bounds__(kThreads, 8) k_add(int n, const TE *__restrict__ e, double *__restrict__ x,
                                                 const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    GRID_STRIDE(i, n) x[i] += (double)ldg(e + i);
}

// ---------------------------------------------------------------------------
// deterministic block reductions: every block writes its partial sums, the
// last block to finish adds them in a fixed order and runs the epilogue.
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Float-float ("ff") arithmetic: a value is the unevaluated sum hi + lo of
// two floats, |lo| <= ulp(hi)/2, about 48 significant bits, computed on the
// FP32 pipe.  Built from the error-free transformations TwoSum (Knuth),
// Fast2Sum (Dekker) and the FMA form of TwoProduct; the _rn intrinsics keep
// the compiler from contracting or reassociating them.
// ---------------------------------------------------------------------------

// s + e == a + b exactly
__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}

// s + e == a + b exactly, provided |a| >= |b| or a == 0
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// p + e == a * b exactly
__device__ __forceinline__ float2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return make_float2(p, __fmaf_rn(a, b, -p));
}

// x + y; absolute error about 2^-47 (|x| + |y|)
__device__ __forceinline__ float2 ff_add(float2 x, float2 y) {
    const float2 s = two_sum(x.x, y.x);
    return fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(x.y, y.y)));
}

// x + b for a float b
__device__ __forceinline__ float2 ff_add(float2 x, float b) {
    const float2 s = two_sum(x.x, b);
    return fast_two_sum(s.x, __fadd_rn(s.y, x.y));
}

// a * b for an ff a and a float b (unnormalized: |lo| may exceed ulp(hi)/2 slightly)
__device__ __forceinline__ float2 ff_mul(float2 a, float b) {
    float2 p = two_prod(a.x, b);
    p.y = __fmaf_rn(a.y, b, p.y);
    return p;
}

// a * b for two ff values (unnormalized, the lo*lo term dropped)
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
    float2 p = two_prod(a.x, b.x);
    p.y = __fmaf_rn(a.x, b.y, p.y);
    p.y = __fmaf_rn(a.y, b.x, p.y);
    return p;
}

// Split a double into an ff pair (FP64 conversions: used at the start and
// end of a solve and once per thread, never per row inside the iteration).
__device__ __forceinline__ float2 ff_from(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

__device__ __forceinline__ float2 warp_sum(float2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float2 u;
        u.x = __shfl_xor_sync(0xffffffffu, v.x, o);
        u.y = __shfl_xor_sync(0xffffffffu, v.y, o);
        v = ff_add(v, u);
    }
    return v;
}

constexpr int kWarps = kThreads / 32;

// Sum over lanes [0, kWarps) of warp 0 (the other lanes hold zeros).
__device__ __forceinline__ double warps_sum(double v) {
#pragma unroll
    for (int o = kWarps / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float2 warps_sum(float2 v) {
#pragma unroll
    for (int o = kWarps / 2; o > 0; o >>= 1) {
        float2 u;
        u.x = __shfl_xor_sync(0xffffffffu, v.x, o);
        u.y = __shfl_xor_sync(0xffffffffu, v.y, o);
        v = ff_add(v, u);
    }
    return v;
}

// Block arrival: true in every thread of the block that arrives last.
// Thread 0 wrote the block's partials; its acquire-release add on the
// counter publishes them (release) and, in the last block, makes every
// other block's partials visible to it (acquire, through the release
// sequence of the counter's read-modify-writes).  The block barrier then
// orders the other threads' reads of the partials (at L2, ld.cg) after it.
__device__ __forceinline__ bool last_block(unsigned *counter) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(t) : "l"(counter) : "memory");
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return last;
}

// Warp sums of NS doubles (NS = 1, 2 or 4) with few FP64 additions.  GB300
// issues FP64 on a narrow pipe where a warp-wide addition takes 32 lane
// slots, so NS independent butterflies (5 NS additions per lane) would cost
// more than the rows themselves.  For NS > 1 the first levels of the
// butterfly exchange half of the sums a lane holds; after log2(NS) levels a
// lane holds one sum and finishes with a plain butterfly: NS = 4 takes 6
// additions per lane instead of 20.  Returns the total of sum (lane >> 3) & 3
// (NS = 4), lane >> 4 (NS = 2) or sum 0 (NS = 1): sum s is held by the lanes
// s * 32 / NS ... (s + 1) * 32 / NS - 1.  The order of the additions is fixed.
template <int NS>
__device__ __forceinline__ double warp_sums(const double (&v)[NS], int lane) {
    static_assert(NS == 1 || NS == 2 || NS == 4, "warp_sums: NS must be 1, 2 or 4");
    double a;
    int o = 16;
    if constexpr (NS == 4) {
        const bool h16 = (lane & 16) != 0;
        const double a0 = (h16 ? v[2] : v[0]) + __shfl_xor_sync(0xffffffffu, h16 ? v[0] : v[2], 16);
        const double a1 = (h16 ? v[3] : v[1]) + __shfl_xor_sync(0xffffffffu, h16 ? v[1] : v[3], 16);
        const bool h8 = (lane & 8) != 0;
        a = (h8 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, h8 ? a0 : a1, 8);
        o = 4;
    } else if constexpr (NS == 2) {
        const bool h16 = (lane & 16) != 0;
        a = (h16 ? v[1] : v[0]) + __shfl_xor_sync(0xffffffffu, h16 ? v[0] : v[1], 16);
        o = 8;
    } else {
        a = v[0];
    }
#pragma unroll
    for (; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

// Combine per-warp totals sh[s][w] (s < NS, w < kWarps) in warp 0: lane
// s * kWarps + w holds one of them, a butterfly over the kWarps lanes of each
// sum leaves sum s in lane s * kWarps.  Needs NS * kWarps <= 32.
template <int NS>
__device__ __forceinline__ double warps_sums(const double (&sh)[NS][kWarps], int lane) {
    static_assert(NS * kWarps <= 32, "warps_sums: too many sums");
    const int s = lane / kWarps, w = lane % kWarps;
    double a = s < NS ? sh[s][w] : 0.0;
#pragma unroll
    for (int o = kWarps / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
}

// Grid-wide sums.  Returns true in every thread of the last block to finish;
// thread 0 of that block then holds the sums in tot[].  Requires blockDim.x ==
// kThreads and gridDim.x <= kMaxRedBlocks.  The last block issues all its
// partial loads first (one L2 round trip), then adds them in a fixed order,
// so results do not depend on scheduling.
//
// FP64 per-thread values: sums in FP64 throughout, with the few-addition warp
// and block combinations above (FP64 kernels launch fewer blocks, see
// red_grid64, so each thread adds several rows before the warp sums).
template <int NS>
__device__ bool grid_reduce(double (&v)[NS], double *partials, unsigned *counter, double (&tot)[NS]) {
    __shared__ double sh[NS][kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kPerSum = 32 / NS;  // lanes that hold one warp sum
    {
        const double x = warp_sums<NS>(v, lane);
        if ((lane & (kPerSum - 1)) == 0) sh[lane / kPerSum][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
        const double x = warps_sums<NS>(sh, lane);
        if (lane % kWarps == 0 && lane / kWarps < NS) partials[(lane / kWarps) * kMaxRedBlocks + blockIdx.x] = x;
    }
    if (!last_block(counter)) return false;
    constexpr int kPer = kMaxRedBlocks / kThreads;
    const int nj = ((int)gridDim.x - warp * 32 + kThreads - 1) / kThreads;  // rounds with a live lane in this warp
    double acc[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        double part[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int b = threadIdx.x + j * kThreads;
            part[j] = b < (int)gridDim.x ? __ldcg(partials + s * kMaxRedBlocks + b) : 0.0;
        }
        double a = part[0];
#pragma unroll
        for (int j = 1; j < kPer; ++j)
            if (j < nj) a += part[j];
        acc[s] = a;
    }
    const double x = warp_sums<NS>(acc, lane);
    __syncthreads();  // every warp of warp 0's block-level read of sh is done (last_block's barriers)
    if ((lane & (kPerSum - 1)) == 0) sh[lane / kPerSum][warp] = x;
    __syncthreads();
    if (warp == 0) {
        const double y = warps_sums<NS>(sh, lane);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const double t = __shfl_sync(0xffffffffu, y, s * kWarps);
            if (lane == 0) tot[s] = t;
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

__device__ __forceinline__ float warps_sum(float v) {
#pragma unroll
    for (int o = kWarps / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FP32 per-thread values: FP32 sums throughout, in a fixed order -- a warp
// butterfly, the block's warps, then the blocks' partials in the last block
// -- so about 21 roundings of the sum of magnitudes (the dot products and
// norms it forms steer alpha, beta, the gauge shift and the stopping test,
// which need FP32 accuracy).  In the last block sum s belongs to the
// kThreads / NS threads [s kT, (s+1) kT): thread u adds the partials of
// blocks 4u..4u+3, 4(u + kT)..., read as float4 with every load issued
// before the first add, so the tail costs one L2 round trip for any NS.
// Only thread 0 touches FP64 (tot).  partials holds one float per block and sum.
template <int NS>
__device__ bool grid_reduce(float (&v)[NS], double *partials, unsigned *counter, double (&tot)[NS]) {
    static_assert(kWarps % NS == 0 && kMaxRedBlocks % 4 == 0, "reduction layout");
    __shared__ float sh[NS][kWarps];
    float *part = reinterpret_cast<float *>(partials);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const float x = warp_sum(v[s]);
        if (lane == 0) sh[s][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const float x = warps_sum(lane < kWarps ? sh[s][lane] : 0.f);
            if (lane == 0) part[s * kMaxRedBlocks + blockIdx.x] = x;
        }
    }
    if (!last_block(counter)) return false;
    constexpr int kT = kThreads / NS;                  // threads per sum
    constexpr int kPer = (kMaxRedBlocks + 4 * kT - 1) / (4 * kT);  // float4 rounds per thread
    const int s = threadIdx.x / kT, u = threadIdx.x % kT;
    const float4 *p4 = reinterpret_cast<const float4 *>(part + s * kMaxRedBlocks);
    const int nb = (int)gridDim.x;
    float4 q[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int b = 4 * (u + j * kT);
        q[j] = b < nb ? __ldcg(p4 + u + j * kT) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int b = 4 * (u + j * kT);  // slots at or past the grid hold stale sums
        acc += b < nb ? q[j].x : 0.f;
        acc += b + 1 < nb ? q[j].y : 0.f;
        acc += b + 2 < nb ? q[j].z : 0.f;
        acc += b + 3 < nb ? q[j].w : 0.f;
    }
    acc = warp_sum(acc);
    float *shw = &sh[0][0];  // free: warp 0 read sh before last_block's first barrier
    if (lane == 0) shw[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        constexpr int kWs = kWarps / NS;  // warps per sum
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            float a = shw[t * kWs];
#pragma unroll
            for (int w = 1; w < kWs; ++w) a += shw[t * kWs + w];
            tot[t] = a;
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// 2^-e with e = floor(log2(rms of b)): the ff outer iteration works on b * scale,
// whose rms lies in [1, 2) (exact; 1 for b == 0 or non-finite b).
__device__ __forceinline__ double ff_scale(double bnorm2, int n) {
    const double ms = bnorm2 / (double)(n > 0 ? n : 1);
    if (!(ms > 0.0) || !isfinite(ms)) return 1.0;
    return ldexp(1.0, -(ilogb(ms) >> 1));
}

// alpha = <r,z> / <p,Lp>.  A zero (or non-finite) quotient means the iteration
// cannot move in this precision -- exact convergence, or, with FP32 dot
// products, residuals so small that the products underflow.  Then alpha = 0,
// the solve stops (status 2) and reports the residual reached so far.
__device__ __forceinline__ void set_alpha(Scal *S, double pq) {
    double a = S->rz / pq;
    if (!isfinite(pq) || !isfinite(S->rz)) {
        a = 0.0;
        S->status = 1;
        S->done = 1;
    } else if (!(a != 0.0) || !isfinite(a)) {
        a = 0.0;
        S->status = 2;
        S->done = 1;
    }
    const float2 af = ff_from(a);
    S->alpha = a;
    S->alpha_hi = af.x;
    S->alpha_lo = af.y;
}

// Records ||r||^2 and runs the stopping test ||r|| <= tol ||b|| as ||r||^2 <=
// thr2, with no FP64 divide or square root on the device (GB300 runs FP64
// at a small fraction of its FP32 rate, and this sits in a single thread at
// the tail of a kernel).  The host forms the relative residuals.
// alpha for the float-float iteration from FP32 dot products: an FP32
// quotient (the sums carry FP32 accuracy, and x and r take the same alpha,
// so r keeps tracking b - L x); same stop rules as set_alpha.
__device__ __forceinline__ void set_alpha_f(Scal *S, double pq) {
    const double rz = S->rz;
    float a = (float)rz / (float)pq;
    if (!isfinite(pq) || !isfinite(rz)) {
        a = 0.f;
        S->status = 1;
        S->done = 1;
    } else if (!(a != 0.f) || !isfinite(a)) {
        a = 0.f;
        S->status = 2;
        S->done = 1;
    }
    S->alpha = a;
    S->alpha_hi = a;
    S->alpha_lo = 0.f;
}

__device__ __forceinline__ void record_residual(Scal *S, double rnorm2) {
    S->rnorm2 = rnorm2;
    const int it = S->iter;
    if (it >= 0 && it < kHist) S->hist[it] = rnorm2;
    if (!isfinite(rnorm2) || !isfinite(S->bnorm2)) {
        S->status = 1;
        S->done = 1;
    } else if (rnorm2 <= S->thr2 || it >= S->maxit) {
        S->done = 1;
    }
}

// mean = sum(*0 v) / sum(*0) over free rows (mask: free != 0)
static __global__ void __launch_bounds__(kThreads, kFp64Blocks) k_mean(int n, const double *__restrict__ star0, const uint8_t *__restrict__ freev,
                                                  const double *__restrict__ v, double *partials, unsigned *counter,
                                                  Scal *S, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    double acc[1] = {0.0};
    GRID_STRIDE_4(i, n) if (freev[i]) acc[0] += ldg(star0 + i) * ldg(v + i);
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) S->mean = tot[0] / S->star0_sum;
}

// v -= mean on free rows
static __global__ void __launch_bounds__(kThreads, 8) k_shift(int n, const uint8_t *__restrict__ freev, double *__restrict__ v,
                                                   const Scal *S, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const double m = S->mean;
    GRID_STRIDE(i, n) v[i] = freev[i] ? v[i] - m : 0.0;
}

// Initial residual of the outer iteration: r = b - L x, ||r||^2, ||b||^2 (free rows);
// also writes the cycle's input rv (cast) when rv != nullptr.  X0: x = 0, so
// r = b without the operator apply.
template <int KT, typename TV, bool X0 = false>
__global__ void __launch_bounds__(kThreads, kFp64Blocks) k_outer_init(int n, int K, const int32_t *__restrict__ col,
                                                        const double *__restrict__ w, const uint8_t *__restrict__ freev,
                                                        const double *__restrict__ b, const double *__restrict__ x,
                                                        double *__restrict__ r, TV *__restrict__ rv, double *partials,
                                                        unsigned *counter, Scal *S) {
    pdl_prologue();
    double acc[2] = {0.0, 0.0};
    GRID_STRIDE_4(i, n) {
        double s = 0.0;
        if (!X0) {
            double d;
            row_apply<double, KT>(i, n, K, col, w, x, s, d);
        }
        double bi = freev[i] ? ldg(b + i) : 0.0;
        double ri = freev[i] ? bi - s : 0.0;
        r[i] = ri;
        if (rv) rv[i] = (TV)ri;
        acc[0] += ri * ri;
        acc[1] += bi * bi;
    }
    double tot[2];
    if (grid_reduce<2>(acc, partials, counter, tot) && threadIdx.x == 0) {
        S->bnorm2 = tot[1];
        const double sc = ff_scale(tot[1], n);
        S->scale = sc;
        S->iscale = 1.0 / sc;
        S->iscale2 = 1.0 / (sc * sc);
        S->thr2 = tot[1] > 0.0 ? S->tol * S->tol * tot[1] : (double)INFINITY;
        S->iter = 0;
        S->done = 0;
        S->status = 0;
        S->rnorm2_0 = tot[0];
        record_residual(S, tot[0]);
    }
}

// After a cycle produced z (type TZ): zn = (double) z; sums of *0 z, *0 r zn, *0 r zo, *0 r;
// epilogue: gauge shift c, new <r,z>, Polak-Ribiere beta.
template <typename TZ>
__global__ void __launch_bounds__(kThreads, kFp64Blocks) k_pcg_zdots(int n, const double *__restrict__ star0, const uint8_t *__restrict__ freev,
                                                       const TZ *__restrict__ z, double *__restrict__ zn,
                                                       const double *__restrict__ r, const double *__restrict__ zo,
                                                       int first, int gauge, double *partials, unsigned *counter,
                                                       Scal *S, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    GRID_STRIDE_4(i, n) {
        double zi = (double)ldg(z + i);
        if ((void *)zn != (void *)z) zn[i] = zi;
        if (freev[i]) {
            double s0 = ldg(star0 + i), ri = ldg(r + i);
            acc[0] += s0 * zi;
            acc[1] += s0 * ri * zi;
            acc[2] += first ? 0.0 : s0 * ri * ldg(zo + i);
            acc[3] += s0 * ri;
        }
    }
    double tot[4];
    if (grid_reduce<4>(acc, partials, counter, tot) && threadIdx.x == 0) {
        double c = gauge ? tot[0] / S->star0_sum : 0.0;
        double rz_new = tot[1] - c * tot[3];
        S->beta = first ? 0.0 : (rz_new - tot[2]) / S->rz;
        S->rz = rz_new;
        S->c = c;
    }
}

// z = zn - c (free rows), p = z + beta p (p = z on the first pass), zo = z.
static __global__ void __launch_bounds__(kThreads, 8) k_pcg_pupd(int n, const uint8_t *__restrict__ freev, const double *__restrict__ zn,
                                                      double *__restrict__ zo, double *__restrict__ p, int first,
                                                      const Scal *S, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const double c = S->c, beta = S->beta;
    GRID_STRIDE(i, n) {
        double zi = freev[i] ? ldg(zn + i) - c : 0.0;
        zo[i] = zi;
        p[i] = first ? zi : fma(beta, p[i], zi);
    }
}

// q = L p (free rows), <p, q> -> alpha = <r,z> / <p,q>
template <int KT>
__global__ void __launch_bounds__(kThreads, 8) k_pcg_spmv(int n, int K, const int32_t *__restrict__ col,
                                                      const double *__restrict__ w, const double *__restrict__ star0,
                                                      const uint8_t *__restrict__ freev, const double *__restrict__ p,
                                                      double *__restrict__ q, double *partials, unsigned *counter,
                                                      Scal *S, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    double acc[1] = {0.0};
    GRID_STRIDE(i, n) {
        double s, d;
        row_apply<double, KT>(i, n, K, col, w, p, s, d);
        double qi = freev[i] ? s : 0.0;
        q[i] = qi;
        acc[0] += ldg(star0 + i) * ldg(p + i) * qi;
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) set_alpha(S, tot[0]);
}

// x += alpha p, r -= alpha q, rv = (TV) r, ||r||^2 -> convergence test
template <typename TV>
__global__ void __launch_bounds__(kThreads, kFp64Blocks) k_pcg_update(int n, const double *__restrict__ p, const double *__restrict__ q,
                                                        double *__restrict__ x, double *__restrict__ r, TV *__restrict__ rv,
                                                        double *partials, unsigned *counter, Scal *S, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const double a = S->alpha;
    double acc[1] = {0.0};
    GRID_STRIDE_4(i, n) {
        x[i] = fma(a, ldg(p + i), x[i]);
        double ri = fma(-a, ldg(q + i), r[i]);
        r[i] = ri;
        if (rv) rv[i] = (TV)ri;
        acc[0] += ri * ri;
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        S->iter += 1;
        record_residual(S, tot[0]);
    }
}

// Standalone MG / iterative refinement: x += e; r = b - L x; ||r||^2 -> convergence test.
template <int KT, typename TV>
__global__ void __launch_bounds__(kThreads, kFp64Blocks) k_mg_residual(int n, int K, const int32_t *__restrict__ col,
                                                         const double *__restrict__ w, const uint8_t *__restrict__ freev,
                                                         const double *__restrict__ b, const double *__restrict__ x,
                                                         double *__restrict__ r, TV *__restrict__ rv, double *partials,
                                                         unsigned *counter, Scal *S, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    double acc[1] = {0.0};
    GRID_STRIDE_4(i, n) {
        double s, d;
        row_apply<double, KT>(i, n, K, col, w, x, s, d);
        double ri = freev[i] ? ldg(b + i) - s : 0.0;
        r[i] = ri;
        if (rv) rv[i] = (TV)ri;
        acc[0] += ri * ri;
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        S->iter += 1;
        record_residual(S, tot[0]);
    }
}

// ---------------------------------------------------------------------------
// Outer-iteration kernels with few FP64 instructions per row.  GB300 issues
// FP64 at a small fraction of its FP32 rate.  The operator apply keeps the
// difference form sum_k w_k (x_i - x_k) -- for smooth x the differences are
// exact, whereas the diagonal form L_ii x_i - sum_k w_k x_k cancels and
// limits the attainable residual -- but drops the FP64 diagonal sum: fixed
// rows have all weights 0 and come out 0 without a mask.  In
// DEC_MODE_MIXED_F32DOT the dot products that steer alpha, beta, the gauge
// shift and the stopping test use FP32 copies, FP32 products and FP32 sums;
// the x and r updates stay FP64.
// ---------------------------------------------------------------------------

template <int KT>
__device__ __forceinline__ double row_apply_nod(int i, int n, int K, const int32_t *__restrict__ col,
                                                const double *__restrict__ w, const double *__restrict__ x) {
    const int Kk = KT > 0 ? KT : K;
    const double xi = ldg(x + i);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
        if (KT == 0 && k >= Kk) break;
        const size_t o = (size_t)k * n + i;
        s = fma(ldg(w + o), xi - ldg(x + ldg(col + o)), s);
    }
    return s;
}

// q = L p, <p, q> (*0) -> alpha
template <int KT>
__global__ void __launch_bounds__(kThreads, kFp64Blocks) k_pcg_spmv_d(int n, int K, const int32_t *__restrict__ col,
                                                        const double *__restrict__ w,
                                                        const double *__restrict__ star0, const double *__restrict__ p,
                                                        double *__restrict__ q, double *partials, unsigned *counter,
                                                        Scal *S, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    double acc[1] = {0.0};
    GRID_STRIDE_4(i, n) {
        const double qi = row_apply_nod<KT>(i, n, K, col, w, p);
        q[i] = qi;
        acc[0] = fma(ldg(star0 + i) * ldg(p + i), qi, acc[0]);
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) set_alpha(S, tot[0]);
}

// x += alpha p, r -= alpha q (FP64), r32 = (float) r, ||r||^2 from r32
static __global__ void __launch_bounds__(kThreads, 8) k_pcg_update_m(int n, const double *__restrict__ p,
                                                          const double *__restrict__ q, double *__restrict__ x,
                                                          double *__restrict__ r, float *__restrict__ r32,
                                                          double *partials, unsigned *counter, Scal *S,
                                                          const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const double a = S->alpha;
    float acc[1] = {0.f};
    GRID_STRIDE(i, n) {
        x[i] = fma(a, ldg(p + i), x[i]);
        const double ri = fma(-a, ldg(q + i), r[i]);
        r[i] = ri;
        const float rf = (float)ri;
        r32[i] = rf;
        acc[0] = fmaf(rf, rf, acc[0]);
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        S->iter += 1;
        record_residual(S, tot[0]);
    }
}

// After the four sums of the preconditioned vector z: gauge shift c, new
// <r,z> and the Polak-Ribiere beta.
__device__ __forceinline__ void zdots_epilogue(Scal *S, const double (&tot)[4], int first, int gauge) {
    double c = gauge ? tot[0] / S->star0_sum : 0.0;
    double rz_new = tot[1] - c * tot[3];
    S->beta = first ? 0.0 : (rz_new - tot[2]) / S->rz;
    S->rz = rz_new;
    S->c = c;
    S->beta_f = (float)S->beta;
    S->c_f = (float)c;
}

// The same from FP32 dot products (whose sums carry FP32 accuracy): the
// gauge shift by a precomputed 1/sum(*0) and beta as an FP32 quotient, so the
// single-thread tail has no FP64 divide.
__device__ __forceinline__ void zdots_epilogue_f(Scal *S, const double (&tot)[4], int first, int gauge) {
    const double c = gauge ? tot[0] * S->inv_star0_sum : 0.0;
    const double rz_new = tot[1] - c * tot[3];
    const float beta = first ? 0.f : (float)(rz_new - tot[2]) / (float)S->rz;
    S->beta = beta;
    S->rz = rz_new;
    S->c = c;
    S->beta_f = beta;
    S->c_f = (float)c;
}

// FP32 dot products of the preconditioned vector z (cycle output) with r32 and the previous z.
static __global__ void __launch_bounds__(kThreads, 8) k_pcg_zdots_m(int n, const float *__restrict__ s032,
                                                         const uint8_t *__restrict__ freev, const float *__restrict__ z,
                                                         const float *__restrict__ r32, const float *__restrict__ zo,
                                                         int first, int gauge, double *partials, unsigned *counter,
                                                         Scal *S, const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    GRID_STRIDE(i, n) {
        if (freev[i]) {
            const float s0 = ldg(s032 + i), zi = ldg(z + i), ri = ldg(r32 + i);
            const float sr = s0 * ri;
            acc[0] = fmaf(s0, zi, acc[0]);
            acc[1] = fmaf(sr, zi, acc[1]);
            if (!first) acc[2] = fmaf(sr, ldg(zo + i), acc[2]);
            acc[3] += sr;
        }
    }
    double tot[4];
    if (grid_reduce<4>(acc, partials, counter, tot) && threadIdx.x == 0) zdots_epilogue_f(S, tot, first, gauge);
}

// The last post-smoothing step of the finest level (k_smooth with DIN =
// Chebyshev, no direction out; b is r32) fused with k_pcg_zdots_m: the dot
// products of z are row-local.  Launch on the reduction grid so that rows
// map to threads as in k_pcg_zdots_m (bitwise equal sums).
template <int KT, bool DIN>
__global__ void __launch_bounds__(kThreads, 8) k_smooth_zdots(int n, int K, const int32_t *__restrict__ col,
                                                          const float *__restrict__ w, const float *__restrict__ b,
                                                          const float *__restrict__ x_in,
                                                          const float *__restrict__ d_in, float *__restrict__ x_out,
                                                          float c, float e, const float *__restrict__ s032,
                                                          const uint8_t *__restrict__ freev,
                                                          const float *__restrict__ zo, int first, int gauge,
                                                          double *partials, unsigned *counter, Scal *S,
                                                          const int *skip) {
    pdl_prologue_ell<KT>(n, K, col, w);
    if (skipped(skip)) return;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    GRID_STRIDE_1(i, n) {
        float s, d;
        row_apply<float, KT>(i, n, K, col, w, x_in, s, d);
        const float ri = ldg(b + i);
        const float q = d != 0.f ? (ri - s) / d : 0.f;
        const float delta = smooth_delta<float>(DIN, c, DIN ? ldg(d_in + i) : 0.f, e, q);
        const float zi = add_rn(ldg(x_in + i), delta);
        x_out[i] = zi;
        if (freev[i]) {
            const float s0 = ldg(s032 + i);
            const float sr = s0 * ri;
            acc[0] = fmaf(s0, zi, acc[0]);
            acc[1] = fmaf(sr, zi, acc[1]);
            if (!first) acc[2] = fmaf(sr, ldg(zo + i), acc[2]);
            acc[3] += sr;
        }
    }
    double tot[4];
    if (grid_reduce<4>(acc, partials, counter, tot) && threadIdx.x == 0) zdots_epilogue_f(S, tot, first, gauge);
}

// z = z - c (free rows, FP32), zo = z, p = z + beta p (FP64)
static __global__ void __launch_bounds__(kThreads, 8) k_pcg_pupd_m(int n, const uint8_t *__restrict__ freev,
                                                        const float *__restrict__ z, float *__restrict__ zo,
                                                        double *__restrict__ p, int first, const Scal *S,
                                                        const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const float c = (float)S->c;
    const double beta = S->beta;
    GRID_STRIDE(i, n) {
        const float zi = freev[i] ? ldg(z + i) - c : 0.f;
        zo[i] = zi;
        p[i] = first ? (double)zi : fma(beta, p[i], (double)zi);
    }
}

// Standalone MG / iterative refinement (mixed): r = b - L x; r32; ||r||^2 in FP32.
template <int KT>
__global__ void __launch_bounds__(kThreads, 8) k_mg_residual_m(int n, int K, const int32_t *__restrict__ col,
                                                           const double *__restrict__ w,
                                                           const uint8_t *__restrict__ freev,
                                                           const double *__restrict__ b, const double *__restrict__ x,
                                                           double *__restrict__ r, float *__restrict__ r32,
                                                           double *partials, unsigned *counter, Scal *S,
                                                           const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    float acc[1] = {0.f};
    GRID_STRIDE(i, n) {
        const double s = row_apply_nod<KT>(i, n, K, col, w, x);
        const double ri = freev[i] ? ldg(b + i) - s : 0.0;
        r[i] = ri;
        const float rf = (float)ri;
        r32[i] = rf;
        acc[0] = fmaf(rf, rf, acc[0]);
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        S->iter += 1;
        record_residual(S, tot[0]);
    }
}

// ---------------------------------------------------------------------------
// FP64 outer iteration around FP32 cycles (DEC_MODE_MIXED): the residual
// update r -= alpha L p, every dot product -- FP64 products and FP64 sums --
// the gauge shift and the search-direction update are FP64; the cycle reads
// r rounded to FP32 (r32) and returns the preconditioned vector z in FP32.
// Scalars (alpha, beta, the gauge shift) are FP64 quotients of FP64 sums.
// ---------------------------------------------------------------------------

// FP32 -> FP64 conversion by integer instructions.  Widening a binary32 to
// binary64 is exact: the sign carries over, the exponent is rebiased by
// 1023 - 127 = 896 and the 23 fraction bits move up by 29.  Zero, subnormal,
// infinite and NaN inputs take the hardware conversion.  (GB300 issues the
// hardware conversion on its narrow FP64 pipe; these bit operations run on
// the integer pipe.)
__device__ __forceinline__ double f2d(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) |
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

// x += alpha p, r -= alpha q, r32 = (float) r, ||r||^2 -> convergence test.
// s0mode > 0 also runs the next cycle's first smoothing step on the finest
// level from zero, as k_smooth0 does on b = r32 (x0 = e0 r32 / dg, and d0 =
// x0 when s0mode == 2); it is row-local.
static __global__ void __launch_bounds__(kThreads, kFp64Blocks) k_pcg_update_d(int n, const double *__restrict__ p,
                                                          const double *__restrict__ q, double *__restrict__ x,
                                                          double *__restrict__ r, float *__restrict__ r32,
                                                          double *partials, unsigned *counter, Scal *S,
                                                          const int *skip, int s0mode, const float *__restrict__ dg,
                                                          float *__restrict__ x0, float *__restrict__ d0, float e0) {
    pdl_prologue();
    if (skipped(skip)) return;
    const double a = S->alpha;
    double acc[1] = {0.0};
    GRID_STRIDE_4(i, n) {
        x[i] = fma(a, ldg(p + i), x[i]);
        const double ri = fma(-a, ldg(q + i), r[i]);
        r[i] = ri;
        const float rf = (float)ri;
        r32[i] = rf;
        acc[0] = fma(ri, ri, acc[0]);
        if (s0mode > 0) {
            const float di = ldg(dg + i);
            const float v = di != 0.f ? e0 * (rf / di) : 0.f;
            x0[i] = v;
            if (s0mode == 2) d0[i] = v;
        }
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        S->iter += 1;
        record_residual(S, tot[0]);
    }
}

// After the four FP64 sums of the preconditioned vector z: sum *0 z, sum *0 r z,
// sum *0 r zo and sum *0 r over free rows, z being the cycle output before its
// gauge shift and zo the previous preconditioned vector after its shift.
// Shift c = sum *0 z / sum *0, <r, z - c> = tot1 - c tot3, <r, zo> = tot2, and
// the Polak-Ribiere beta = (<r, z - c> - <r, zo>) / <r_prev, zo>.
__device__ __forceinline__ void zdots_epilogue_d(Scal *S, const double (&tot)[4], int first, int gauge) {
    const double c = gauge ? tot[0] / S->star0_sum : 0.0;
    const double rz_new = tot[1] - c * tot[3];
    S->beta = first ? 0.0 : (rz_new - tot[2]) / S->rz;
    S->rz = rz_new;
    S->c = c;
}

// The four FP64 dot products of z (FP32 cycle output, unshifted) with *0 and
// the FP64 residual r; zo is the previous shifted z (FP64).
static __global__ void __launch_bounds__(kThreads, kFp64Blocks) k_pcg_zdots_d(int n, const double *__restrict__ star0,
                                                         const uint8_t *__restrict__ freev,
                                                         const float *__restrict__ z, const double *__restrict__ r,
                                                         const double *__restrict__ zo, int first, int gauge,
                                                         double *partials, unsigned *counter, Scal *S,
                                                         const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    GRID_STRIDE_4(i, n) {
        if (freev[i]) {
            const double s0 = ldg(star0 + i), zi = f2d(ldg(z + i));
            const double sr = s0 * ldg(r + i);
            acc[0] = fma(s0, zi, acc[0]);
            acc[1] = fma(sr, zi, acc[1]);
            if (!first) acc[2] = fma(sr, ldg(zo + i), acc[2]);
            acc[3] += sr;
        }
    }
    double tot[4];
    if (grid_reduce<4>(acc, partials, counter, tot) && threadIdx.x == 0) zdots_epilogue_d(S, tot, first, gauge);
}

// The last post-smoothing step of the finest level (k_smooth with DIN =
// Chebyshev, no direction out; b = r32) fused with k_pcg_zdots_d, whose sums
// are row-local.  Launched on the reduction grid so that rows map to threads
// as in k_pcg_zdots_d (bitwise equal sums).
template <int KT, bool DIN>
__global__ void __launch_bounds__(kThreads, kFp64Blocks) k_smooth_zdots_d(int n, int K, const int32_t *__restrict__ col,
                                                            const float *__restrict__ w, const float *__restrict__ b,
                                                            const float *__restrict__ x_in,
                                                            const float *__restrict__ d_in, float *__restrict__ x_out,
                                                            float c, float e, const double *__restrict__ star0,
                                                            const uint8_t *__restrict__ freev,
                                                            const double *__restrict__ r64,
                                                            const double *__restrict__ zo, int first, int gauge,
                                                            double *partials, unsigned *counter, Scal *S,
                                                            const int *skip) {
    pdl_prologue_ell<KT>(n, K, col, w);
    if (skipped(skip)) return;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    GRID_STRIDE_4(i, n) {
        float s, d;
        row_apply<float, KT>(i, n, K, col, w, x_in, s, d);
        const float q = d != 0.f ? (ldg(b + i) - s) / d : 0.f;
        const float delta = smooth_delta<float>(DIN, c, DIN ? ldg(d_in + i) : 0.f, e, q);
        const float zf = add_rn(ldg(x_in + i), delta);
        x_out[i] = zf;
        if (freev[i]) {
            const double s0 = ldg(star0 + i), zi = f2d(zf);
            const double sr = s0 * ldg(r64 + i);
            acc[0] = fma(s0, zi, acc[0]);
            acc[1] = fma(sr, zi, acc[1]);
            if (!first) acc[2] = fma(sr, ldg(zo + i), acc[2]);
            acc[3] += sr;
        }
    }
    double tot[4];
    if (grid_reduce<4>(acc, partials, counter, tot) && threadIdx.x == 0) zdots_epilogue_d(S, tot, first, gauge);
}

// zs = z - c in FP64 (free rows; 0 on fixed rows), zo = zs, p = zs + beta p
// (p = zs on the first pass).
static __global__ void __launch_bounds__(kThreads, 8) k_pcg_pupd_d(int n, const uint8_t *__restrict__ freev,
                                                        const float *__restrict__ z, double *__restrict__ zo,
                                                        double *__restrict__ p, int first, const Scal *S,
                                                        const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const double c = S->c, beta = S->beta;
    GRID_STRIDE(i, n) {
        const double zi = freev[i] ? f2d(ldg(z + i)) - c : 0.0;
        zo[i] = zi;
        p[i] = first ? zi : fma(beta, p[i], zi);
    }
}

// Standalone MG / iterative refinement with the FP64 outer loop: r = b - L x
// (FP64), r32 = (float) r, ||r||^2 in FP64 -> convergence test.
template <int KT>
__global__ void __launch_bounds__(kThreads, kFp64Blocks) k_mg_residual_d(int n, int K, const int32_t *__restrict__ col,
                                                           const double *__restrict__ w,
                                                           const uint8_t *__restrict__ freev,
                                                           const double *__restrict__ b, const double *__restrict__ x,
                                                           double *__restrict__ r, float *__restrict__ r32,
                                                           double *partials, unsigned *counter, Scal *S,
                                                           const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    double acc[1] = {0.0};
    GRID_STRIDE_4(i, n) {
        const double s = row_apply_nod<KT>(i, n, K, col, w, x);
        const double ri = freev[i] ? ldg(b + i) - s : 0.0;
        r[i] = ri;
        r32[i] = (float)ri;
        acc[0] = fma(ri, ri, acc[0]);
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        S->iter += 1;
        record_residual(S, tot[0]);
    }
}

// ---------------------------------------------------------------------------
// Float-float outer iteration (DEC_MODE_MIXED_FF): no FP64 arithmetic per
// row inside the iteration.  The iterate x, the residual r and q = L p are
// ff pairs stored as separate hi and lo arrays (r's hi array is the FP32
// right-hand side of the cycle); the search direction p is FP32.  q is the
// ff product of the ff weights (w32 + wlo = w64 to ~2^-48) with the exact
// FP32 differences p_i - p_k, accumulated as a compensated sum, so the
// updated r tracks b - L x to about 2^-44 of the row terms.  All outer
// vectors are scaled by the power of two S->scale.
// ---------------------------------------------------------------------------

// (L p)_i in ff for an FP32 vector p.
template <int KT>
__device__ __forceinline__ float2 row_apply_ff(int i, int n, int K, const int32_t *__restrict__ col,
                                               const float *__restrict__ wh, const float *__restrict__ wl,
                                               const float *__restrict__ p, float pi) {
    const int Kk = KT > 0 ? KT : K;
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
        if (KT == 0 && k >= Kk) break;
        const size_t o = (size_t)k * n + i;
        const float2 d = two_sum(pi, -ldg(p + ldg(col + o)));
        const float2 t = ff_mul(make_float2(ldg(wh + o), ldg(wl + o)), d);
        const float2 u = two_sum(s, t.x);
        s = u.x;
        c = __fadd_rn(c, __fadd_rn(u.y, t.y));
    }
    return two_sum(s, c);
}

// (L x)_i in ff for an ff vector x (hi and lo arrays).
template <int KT>
__device__ __forceinline__ float2 row_apply_ff2(int i, int n, int K, const int32_t *__restrict__ col,
                                                const float *__restrict__ wh, const float *__restrict__ wl,
                                                const float *__restrict__ xh, const float *__restrict__ xl) {
    const int Kk = KT > 0 ? KT : K;
    const float xih = ldg(xh + i), xil = ldg(xl + i);
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
        if (KT == 0 && k >= Kk) break;
        const size_t o = (size_t)k * n + i;
        const int j = ldg(col + o);
        float2 d = two_sum(xih, -ldg(xh + j));
        d = two_sum(d.x, __fadd_rn(d.y, __fsub_rn(xil, ldg(xl + j))));
        const float2 t = ff_mul(make_float2(ldg(wh + o), ldg(wl + o)), d);
        const float2 u = two_sum(s, t.x);
        s = u.x;
        c = __fadd_rn(c, __fadd_rn(u.y, t.y));
    }
    return two_sum(s, c);
}

// Start of an ff solve: the FP64 x and r of k_outer_init (and b, for
// standalone MG) -> scaled ff pairs.  x == nullptr means x = 0.
static __global__ void __launch_bounds__(kThreads, 8) k_ff_split(int n, const double *__restrict__ x,
                                                      const double *__restrict__ r, const double *__restrict__ b,
                                                      float *__restrict__ xh, float *__restrict__ xl,
                                                      float *__restrict__ rh, float *__restrict__ rl,
                                                      float *__restrict__ bh, float *__restrict__ bl,
                                                      const Scal *S) {
    pdl_prologue();
    const double sc = S->scale;
    GRID_STRIDE(i, n) {
        float2 v = x ? ff_from(ldg(x + i) * sc) : make_float2(0.f, 0.f);
        xh[i] = v.x;
        xl[i] = v.y;
        v = ff_from(ldg(r + i) * sc);
        rh[i] = v.x;
        rl[i] = v.y;
        if (bh) {
            v = ff_from(ldg(b + i) * sc);
            bh[i] = v.x;
            bl[i] = v.y;
        }
    }
}

// End of an ff solve: x = (hi + lo) / scale (also into x2 when given).
static __global__ void __launch_bounds__(kThreads, 8) k_ff_join(int n, const float *__restrict__ xh,
                                                     const float *__restrict__ xl, double *__restrict__ x,
                                                     double *__restrict__ x2, const Scal *S) {
    pdl_prologue();
    const double is = S->iscale;
    GRID_STRIDE(i, n) {
        const double v = ((double)ldg(xh + i) + (double)ldg(xl + i)) * is;
        x[i] = v;
        if (x2) x2[i] = v;
    }
}

// The same with the gauge: x = (hi + lo) / scale and the *0-weighted mean of x
// over free rows, for k_shift_out.
static __global__ void __launch_bounds__(kThreads, kFp64Blocks) k_ff_join_mean(int n, const float *__restrict__ xh,
                                                          const float *__restrict__ xl, double *__restrict__ x,
                                                          const double *__restrict__ star0,
                                                          const uint8_t *__restrict__ freev, double *partials,
                                                          unsigned *counter, Scal *S) {
    pdl_prologue();
    const double is = S->iscale;
    double acc[1] = {0.0};
    GRID_STRIDE_4(i, n) {
        const double v = ((double)ldg(xh + i) + (double)ldg(xl + i)) * is;
        x[i] = v;
        if (freev[i]) acc[0] = fma(ldg(star0 + i), v, acc[0]);
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) S->mean = tot[0] * S->inv_star0_sum;
}

// v <- v - mean on free rows, 0 on fixed rows, also into out when given.
static __global__ void __launch_bounds__(kThreads, 8) k_shift_out(int n, const uint8_t *__restrict__ freev,
                                                       double *__restrict__ v, double *__restrict__ out,
                                                       const Scal *S) {
    pdl_prologue();
    const double m = S->mean;
    GRID_STRIDE(i, n) {
        const double y = freev[i] ? v[i] - m : 0.0;
        v[i] = y;
        if (out) out[i] = y;
    }
}

// Start of a cold-start (x = 0) float-float solve, pass 1: the *0-weighted
// mean of b over free rows (gauge) and ||b||^2 over free rows, whose size
// fixes the power-of-two scale of the ff iteration (ff_scale).
static __global__ void __launch_bounds__(kThreads, kFp64Blocks) k_b_stats(int n, const double *__restrict__ star0,
                                                     const uint8_t *__restrict__ freev,
                                                     const double *__restrict__ b, int gauge, double *partials,
                                                     unsigned *counter, Scal *S) {
    pdl_prologue();
    double acc[2] = {0.0, 0.0};
    GRID_STRIDE_4(i, n) {
        if (freev[i]) {
            const double bi = ldg(b + i);
            if (gauge) acc[0] = fma(ldg(star0 + i), bi, acc[0]);
            acc[1] = fma(bi, bi, acc[1]);
        }
    }
    double tot[2];
    if (grid_reduce<2>(acc, partials, counter, tot) && threadIdx.x == 0) {
        S->mean = gauge ? tot[0] * S->inv_star0_sum : 0.0;
        const double sc = ff_scale(tot[1], n);
        S->scale = sc;
        S->iscale = 1.0 / sc;
        S->iscale2 = 1.0 / (sc * sc);
    }
}

// Pass 2, row-local: b <- b - mean on free rows, 0 on fixed rows (written
// back); with x = 0, r = b, stored as scaled ff pairs (rh is the cycle's
// right-hand side; bh, bl, when given, get the same pair for standalone MG);
// x = 0 in ff; ||r||^2 from rh in FP32 starts the stopping test.  s0mode > 0
// also runs the first cycle's first smoothing step on the finest level from
// zero, as k_smooth0 does (x0 = e0 r / dg, and d0 = x0 when s0mode == 2).
static __global__ void __launch_bounds__(kThreads, 8) k_init_ff(int n, const uint8_t *__restrict__ freev,
                                                     double *b, float *__restrict__ xh, float *__restrict__ xl,
                                                     float *__restrict__ rh, float *__restrict__ rl,
                                                     float *__restrict__ bh, float *__restrict__ bl, int s0mode,
                                                     const float *__restrict__ dg, float *__restrict__ x0,
                                                     float *__restrict__ d0, float e0, double *partials,
                                                     unsigned *counter, Scal *S) {
    pdl_prologue();
    const double m = S->mean, sc = S->scale;
    float acc[1] = {0.f};
    GRID_STRIDE(i, n) {
        const double v = freev[i] ? b[i] - m : 0.0;
        b[i] = v;
        const float2 r = ff_from(v * sc);
        rh[i] = r.x;
        rl[i] = r.y;
        xh[i] = 0.f;
        xl[i] = 0.f;
        if (bh) {
            bh[i] = r.x;
            bl[i] = r.y;
        }
        acc[0] = fmaf(r.x, r.x, acc[0]);
        if (s0mode > 0) {
            const float di = ldg(dg + i);
            const float x1 = di != 0.f ? e0 * (r.x / di) : 0.f;
            x0[i] = x1;
            if (s0mode == 2) d0[i] = x1;
        }
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        const double bn2 = tot[0] * S->iscale2;
        S->bnorm2 = bn2;
        S->thr2 = bn2 > 0.0 ? S->tol * S->tol * bn2 : (double)INFINITY;
        S->iter = 0;
        S->done = 0;
        S->status = 0;
        S->rnorm2_0 = bn2;
        record_residual(S, bn2);
    }
}

// Start of a cold-start (x = 0) MG-PCG solve with an FP64 outer iteration
// (DEC_MODE_MIXED, DEC_MODE_MIXED_F32DOT), after k_b_stats gave the gauge
// mean: b <- b - mean on free rows, 0 on fixed rows (written back), r = b,
// r32 = (float) r, x = 0, and ||r||^2 = ||b||^2 (FP64) starts the stopping
// test.  s0mode > 0 also runs the first cycle's first smoothing step on the
// finest level from zero, as k_smooth0 does (x0 = e0 r32 / dg, d0 = x0 when
// s0mode == 2).
static __global__ void __launch_bounds__(kThreads, kFp64Blocks) k_init_d(int n, const uint8_t *__restrict__ freev,
                                                               double *b, double *__restrict__ x,
                                                               double *__restrict__ r, float *__restrict__ r32,
                                                               int s0mode, const float *__restrict__ dg,
                                                               float *__restrict__ x0, float *__restrict__ d0,
                                                               float e0, double *partials, unsigned *counter, Scal *S) {
    pdl_prologue();
    const double m = S->mean;
    double acc[1] = {0.0};
    GRID_STRIDE_4(i, n) {
        const double v = freev[i] ? b[i] - m : 0.0;
        b[i] = v;
        x[i] = 0.0;
        r[i] = v;
        const float rf = (float)v;
        r32[i] = rf;
        acc[0] = fma(v, v, acc[0]);
        if (s0mode > 0) {
            const float di = ldg(dg + i);
            const float x1 = di != 0.f ? e0 * (rf / di) : 0.f;
            x0[i] = x1;
            if (s0mode == 2) d0[i] = x1;
        }
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        S->bnorm2 = tot[0];
        S->thr2 = tot[0] > 0.0 ? S->tol * S->tol * tot[0] : (double)INFINITY;
        S->iter = 0;
        S->done = 0;
        S->status = 0;
        S->rnorm2_0 = tot[0];
        record_residual(S, tot[0]);
    }
}

// z = z - c (free rows), zo = z, p = z + beta p, all FP32.
static __global__ void __launch_bounds__(kThreads, 8) k_pcg_pupd_f(int n, const uint8_t *__restrict__ freev,
                                                        const float *__restrict__ z, float *__restrict__ zo,
                                                        float *__restrict__ p, int first, const Scal *S,
                                                        const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    const float c = S->c_f, beta = S->beta_f;
    GRID_STRIDE(i, n) {
        const float zi = freev[i] ? ldg(z + i) - c : 0.f;
        zo[i] = zi;
        p[i] = first ? zi : fmaf(beta, p[i], zi);
    }
}

// q = L p (ff), <p, q>*0 in FP32 products -> alpha = <r,z> / <p,q>
template <int KT>
__global__ void __launch_bounds__(kThreads, 8) k_pcg_spmv_ff(int n, int K, const int32_t *__restrict__ col,
                                                         const float *__restrict__ wh, const float *__restrict__ wl,
                                                         const float *__restrict__ s032, const float *__restrict__ p,
                                                         float *__restrict__ qh, float *__restrict__ ql,
                                                         double *partials, unsigned *counter, Scal *S,
                                                         const int *skip) {
    pdl_prologue_ell<KT>(n, K, col, wh, wl);
    if (skipped(skip)) return;
    float acc[1] = {0.f};
    GRID_STRIDE_1(i, n) {
        const float pi = ldg(p + i);
        const float2 q = row_apply_ff<KT>(i, n, K, col, wh, wl, p, pi);
        qh[i] = q.x;
        ql[i] = q.y;
        acc[0] = fmaf(ldg(s032 + i) * pi, q.x, acc[0]);
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) set_alpha_f(S, tot[0]);
}

// x += alpha p, r -= alpha q (ff), ||r||^2 from r's hi part -> convergence test
// s0mode > 0 also runs the first smoothing step of the next cycle on the
// finest level from zero (k_smooth0 on b = r's hi part: x0 = e0 r / dg, and
// d0 = x0 when s0mode == 2), which is row-local.
static __global__ void __launch_bounds__(kThreads, 8) k_pcg_update_ff(int n, const float *__restrict__ p,
                                                           const float *__restrict__ qh, const float *__restrict__ ql,
                                                           float *__restrict__ xh, float *__restrict__ xl,
                                                           float *__restrict__ rh, float *__restrict__ rl,
                                                           double *partials, unsigned *counter, Scal *S,
                                                           const int *skip, int s0mode,
                                                           const float *__restrict__ dg, float *__restrict__ x0,
                                                           float *__restrict__ d0, float e0) {
    pdl_prologue();
    if (skipped(skip)) return;
    const float2 a = make_float2(S->alpha_hi, S->alpha_lo);
    float acc[1] = {0.f};
    GRID_STRIDE(i, n) {
        const float2 x = ff_add(make_float2(xh[i], xl[i]), ff_mul(a, ldg(p + i)));
        xh[i] = x.x;
        xl[i] = x.y;
        const float2 aq = ff_mul(a, make_float2(ldg(qh + i), ldg(ql + i)));
        const float2 r = ff_add(make_float2(rh[i], rl[i]), make_float2(-aq.x, -aq.y));
        rh[i] = r.x;
        rl[i] = r.y;
        acc[0] = fmaf(r.x, r.x, acc[0]);
        if (s0mode > 0) {
            const float di = ldg(dg + i);
            const float v = di != 0.f ? e0 * (r.x / di) : 0.f;
            x0[i] = v;
            if (s0mode == 2) d0[i] = v;
        }
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        S->iter += 1;
        record_residual(S, tot[0] * S->iscale2);
    }
}

// Standalone MG in ff: x += e (FP32 cycle output)
static __global__ void __launch_bounds__(kThreads, 8) k_add_ff(int n, const float *__restrict__ e,
                                                    float *__restrict__ xh, float *__restrict__ xl,
                                                    const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    GRID_STRIDE(i, n) {
        const float2 x = ff_add(make_float2(xh[i], xl[i]), ldg(e + i));
        xh[i] = x.x;
        xl[i] = x.y;
    }
}

// Standalone MG in ff: r = b - L x, ||r||^2 -> convergence test
template <int KT>
__global__ void __launch_bounds__(kThreads, 8) k_mg_residual_ff(int n, int K, const int32_t *__restrict__ col,
                                                            const float *__restrict__ wh, const float *__restrict__ wl,
                                                            const uint8_t *__restrict__ freev,
                                                            const float *__restrict__ bh, const float *__restrict__ bl,
                                                            const float *__restrict__ xh, const float *__restrict__ xl,
                                                            float *__restrict__ rh, float *__restrict__ rl,
                                                            double *partials, unsigned *counter, Scal *S,
                                                            const int *skip) {
    pdl_prologue();
    if (skipped(skip)) return;
    float acc[1] = {0.f};
    GRID_STRIDE(i, n) {
        float2 r = make_float2(0.f, 0.f);
        if (freev[i]) {
            const float2 s = row_apply_ff2<KT>(i, n, K, col, wh, wl, xh, xl);
            r = ff_add(make_float2(ldg(bh + i), ldg(bl + i)), make_float2(-s.x, -s.y));
        }
        rh[i] = r.x;
        rl[i] = r.y;
        acc[0] = fmaf(r.x, r.x, acc[0]);
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) {
        S->iter += 1;
        record_residual(S, tot[0] * S->iscale2);
    }
}

// Body-end kernel of the device-side iteration loop (a while node of the
// solve graph): repeat while the solve is not done, and never more than
// max_loops times, so the loop ends even if no kernel ever sets `done`.
static __global__ void k_loop_ctrl(cudaGraphConditionalHandle h, Scal *S) {
    pdl_prologue();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        S->loops += 1;
        const bool more = !S->done && S->loops < S->max_loops;
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}

// Gradient with respect to the edge weights: g_e = -(d0 mu)_e (d0 u)_e.
static __global__ void __launch_bounds__(kThreads, 8) k_edge_grad(int64_t ne, const int2 *__restrict__ edges, const double *__restrict__ mu,
                                                       const double *__restrict__ u, double *__restrict__ g) {
    pdl_prologue();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        const int2 ab = ldg(edges + e);
        g[e] = -(ldg(mu + ab.y) - ldg(mu + ab.x)) * (ldg(u + ab.y) - ldg(u + ab.x));
    }
}

// y = s0 .* x, or y = x ./ s0 (inverse != 0)
static __global__ void __launch_bounds__(kThreads, 8) k_star0_scale(int n, const double *__restrict__ star0, const double *x,
                                                         double *y, int inverse) {
    pdl_prologue();
    GRID_STRIDE(i, n) y[i] = inverse ? x[i] / ldg(star0 + i) : x[i] * ldg(star0 + i);
}

// Finest-level weights from a new *1: w[slot] = *1[edge(slot)] / *0[row] on free rows.
static __global__ void __launch_bounds__(kThreads) k_set_weights(int n, int K, const int32_t *__restrict__ slot_edge,
                                                         const double *__restrict__ star1, const double *__restrict__ star0,
                                                         const uint8_t *__restrict__ freev, double *__restrict__ w64,
                                                         float *__restrict__ w32, float *__restrict__ wlo) {
    pdl_wait_only();
    GRID_STRIDE(i, n) {
        const double s0 = ldg(star0 + i);
        for (int k = 0; k < K; ++k) {
            const size_t o = (size_t)k * n + i;
            const int e = ldg(slot_edge + o);
            double wk = (e >= 0 && freev[i]) ? ldg(star1 + e) / s0 : 0.0;
            const float wh = (float)wk;
            w64[o] = wk;
            w32[o] = wh;
            wlo[o] = (float)(wk - (double)wh);
        }
    }
}


// ---------------------------------------------------------------------------
// porous convection (Sec. 3.2.1), FP64.  pot_v = alpha rho0 g . x_v, so the
// buoyancy 1-form is w_e = (pot_hi - pot_lo)(T_lo + T_hi)/2 and, with the
// ELL weight w_k = *1_e / *0_v of the slot joining v to u,
//   (*0^-1 d0^T *1 w)_v = sum_k w_k (pot_v - pot_u)(T_v + T_u)/2,
//   q_{v->u} = -k_eta [(P_u - P_v) - (pot_u - pot_v)(T_u + T_v)/2],
//   (L_q T)_v = sum_k w_k (T_u - T_v) q_{v->u} / 2,   (L T)_v = sum_k w_k (T_v - T_u).
// ---------------------------------------------------------------------------

static __global__ void __launch_bounds__(kThreads) k_potential(int n, int dim, const double *__restrict__ verts, double g0,
                                                       double g1, double g2, double arho, double *__restrict__ pot) {
    pdl_prologue();
    GRID_STRIDE(v, n) {
        const double *x = verts + (size_t)v * dim;
        double s = g0 * x[0] + g1 * x[1];
        if (dim == 3) s += g2 * x[2];
        pot[v] = arho * s;
    }
}

// rhs = *0^-1 d0^T *1 w(T)
template <int KT>
__global__ void __launch_bounds__(kThreads) k_porous_rhs(int n, int K, const int32_t *__restrict__ col,
                                                        const double *__restrict__ w, const double *__restrict__ T,
                                                        const double *__restrict__ pot, double *__restrict__ rhs) {
    pdl_prologue();
    const int Kk = KT > 0 ? KT : K;
    GRID_STRIDE(v, n) {
        const double Tv = ldg(T + v), pv = ldg(pot + v);
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
            if (KT == 0 && k >= Kk) break;
            const size_t o = (size_t)k * n + v;
            const int u = ldg(col + o);
            s += ldg(w + o) * (pv - ldg(pot + u)) * 0.5 * (Tv + ldg(T + u));
        }
        rhs[v] = s;
    }
}

// T_out = T + dt * mask * ( -(1/phi) L_q T - kappa L T )
template <int KT>
__global__ void __launch_bounds__(kThreads) k_porous_update(int n, int K, const int32_t *__restrict__ col,
                                                           const double *__restrict__ w, const double *__restrict__ T,
                                                           const double *__restrict__ P, const double *__restrict__ pot,
                                                           const uint8_t *__restrict__ fixed, double inv_phi,
                                                           double k_eta, double kappa, double dt,
                                                           double *__restrict__ T_out) {
    pdl_prologue();
    const int Kk = KT > 0 ? KT : K;
    GRID_STRIDE(v, n) {
        const double Tv = ldg(T + v);
        if (fixed[v]) {
            T_out[v] = Tv;
            continue;
        }
        const double Pv = ldg(P + v), pv = ldg(pot + v);
        double adv = 0.0, dif = 0.0;
#pragma unroll
        for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
            if (KT == 0 && k >= Kk) break;
            const size_t o = (size_t)k * n + v;
            const int u = ldg(col + o);
            const double wk = ldg(w + o);
            const double Tu = ldg(T + u);
            const double q = -k_eta * ((ldg(P + u) - Pv) - (ldg(pot + u) - pv) * 0.5 * (Tu + Tv));
            adv += wk * 0.5 * (Tu - Tv) * q;
            dif += wk * (Tv - Tu);
        }
        T_out[v] = Tv + dt * (-inv_phi * adv - kappa * dif);
    }
}

// dT/dt = mask * ( -(1/phi) L_q T - kappa L T ): the bracket of k_porous_update,
// the right-hand side an explicit Runge-Kutta stage evaluates.
template <int KT>
__global__ void __launch_bounds__(kThreads) k_porous_tdot(int n, int K, const int32_t *__restrict__ col,
                                                         const double *__restrict__ w, const double *__restrict__ T,
                                                         const double *__restrict__ P, const double *__restrict__ pot,
                                                         const uint8_t *__restrict__ fixed, double inv_phi,
                                                         double k_eta, double kappa, double *__restrict__ out) {
    pdl_prologue();
    const int Kk = KT > 0 ? KT : K;
    GRID_STRIDE(v, n) {
        if (fixed[v]) {
            out[v] = 0.0;
            continue;
        }
        const double Tv = ldg(T + v), Pv = ldg(P + v), pv = ldg(pot + v);
        double adv = 0.0, dif = 0.0;
#pragma unroll
        for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
            if (KT == 0 && k >= Kk) break;
            const size_t o = (size_t)k * n + v;
            const int u = ldg(col + o);
            const double wk = ldg(w + o);
            const double Tu = ldg(T + u);
            const double q = -k_eta * ((ldg(P + u) - Pv) - (ldg(pot + u) - pv) * 0.5 * (Tu + Tv));
            adv += wk * 0.5 * (Tu - Tv) * q;
            dif += wk * (Tv - Tu);
        }
        out[v] = -inv_phi * adv - kappa * dif;
    }
}

// Up to seven stage vectors with their coefficients (explicit Runge-Kutta).
struct RkStages {
    const double *k[7];
    double a[7];
    int nk;
};

// y = T + dt * sum_j a_j k_j (a stage state, or the new state).
static __global__ void __launch_bounds__(kThreads) k_rk_combine(int n, const double *__restrict__ T,
                                                        const __grid_constant__ RkStages c, double dt,
                                                        double *__restrict__ y) {
    pdl_prologue();
    GRID_STRIDE(v, n) {
        double s = 0.0;
        for (int j = 0; j < c.nk; ++j) s = fma(c.a[j], ldg(c.k[j] + v), s);
        y[v] = ldg(T + v) + dt * s;
    }
}

// Embedded error estimate err = dt * sum_j e_j k_j, scaled componentwise by
// atol + rtol max(|T|, |T_new|); *out = the sum of the squares (FP64).
static __global__ void __launch_bounds__(kThreads, kFp64Blocks) k_rk_error(int n, const double *__restrict__ T,
                                                          const double *__restrict__ Tn,
                                                          const __grid_constant__ RkStages e, double dt,
                                                          double rtol, double atol, double *partials,
                                                          unsigned *counter, double *out) {
    pdl_prologue();
    double acc[1] = {0.0};
    GRID_STRIDE_4(v, n) {
        double s = 0.0;
        for (int j = 0; j < e.nk; ++j) s = fma(e.a[j], ldg(e.k[j] + v), s);
        const double err = dt * s;
        const double sc = atol + rtol * fmax(fabs(ldg(T + v)), fabs(ldg(Tn + v)));
        const double r = err / sc;
        acc[0] = fma(r, r, acc[0]);
    }
    double tot[1];
    if (grid_reduce<1>(acc, partials, counter, tot) && threadIdx.x == 0) *out = tot[0];
}

// Adjoint step, part 1: ms = mu / *0 with mu = dt * mask * lam.
static __global__ void __launch_bounds__(kThreads) k_porous_adj1(int n, const double *__restrict__ lam,
                                                         const uint8_t *__restrict__ fixed,
                                                         const double *__restrict__ star0, double dt,
                                                         double *__restrict__ ms) {
    pdl_prologue();
    GRID_STRIDE(v, n) ms[v] = fixed[v] ? 0.0 : dt * ldg(lam + v) / ldg(star0 + v);
}

// Adjoint step, part 2 (per vertex v, slots to u, *1_e = w_k *0_v):
//   out_v  = lam_v - kappa *0_v sum_k w_k (ms_v - ms_u) + sum_k abar_e da_e/dT_v
//   pbs_v  = (sum_k abar_e da_e/dP_v) / *0_v          (right-hand side of the pressure adjoint)
// with abar_e = -(ms_v + ms_u)/phi, a_e = *1_e (T_u - T_v) q_{v->u} / 2.
template <int KT>
__global__ void __launch_bounds__(kThreads) k_porous_adj2(int n, int K, const int32_t *__restrict__ col,
                                                         const double *__restrict__ w, const double *__restrict__ star0,
                                                         const double *__restrict__ T, const double *__restrict__ P,
                                                         const double *__restrict__ pot, const double *__restrict__ lam,
                                                         const double *__restrict__ ms, double inv_phi, double k_eta,
                                                         double kappa, double *__restrict__ out,
                                                         double *__restrict__ pbs) {
    pdl_prologue();
    const int Kk = KT > 0 ? KT : K;
    GRID_STRIDE(v, n) {
        const double Tv = ldg(T + v), Pv = ldg(P + v), pv = ldg(pot + v), mv = ldg(ms + v);
        const double s0 = ldg(star0 + v);
        double dif = 0.0, tbar = 0.0, pbar = 0.0;
#pragma unroll
        for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
            if (KT == 0 && k >= Kk) break;
            const size_t o = (size_t)k * n + v;
            const int u = ldg(col + o);
            const double wk = ldg(w + o);
            const double Tu = ldg(T + u), dpot = ldg(pot + u) - pv, mu_u = ldg(ms + u);
            dif += wk * (mv - mu_u);
            const double q = -k_eta * ((ldg(P + u) - Pv) - dpot * 0.5 * (Tu + Tv));
            const double abar = -(mv + mu_u) * inv_phi;
            const double half_s1 = 0.5 * wk * s0;
            tbar += abar * half_s1 * (-q + (Tu - Tv) * k_eta * dpot * 0.5);
            pbar += abar * half_s1 * (Tu - Tv) * k_eta;
        }
        out[v] = ldg(lam + v) - kappa * s0 * dif + tbar;
        pbs[v] = pbar / s0;
    }
}

// Adjoint step, part 3: out_v += *0_v sum_k w_k (m_u - m_v)(pot_u - pot_v) / 2.
template <int KT>
__global__ void __launch_bounds__(kThreads) k_porous_adj3(int n, int K, const int32_t *__restrict__ col,
                                                         const double *__restrict__ w, const double *__restrict__ star0,
                                                         const double *__restrict__ pot, const double *__restrict__ m,
                                                         double *__restrict__ out) {
    pdl_prologue();
    const int Kk = KT > 0 ? KT : K;
    GRID_STRIDE(v, n) {
        const double mv = ldg(m + v), pv = ldg(pot + v);
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
            if (KT == 0 && k >= Kk) break;
            const size_t o = (size_t)k * n + v;
            const int u = ldg(col + o);
            s += ldg(w + o) * (ldg(m + u) - mv) * (ldg(pot + u) - pv);
        }
        out[v] += 0.5 * ldg(star0 + v) * s;
    }
}

}  // namespace decdev
