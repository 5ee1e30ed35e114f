// Tiled cycle kernels (DEC_FUSE_PATCH): one thread block per halo tile runs a
// level's whole share of a V-cycle in one direction out of shared memory.
//
//   k_patch_down: nu1 smoothing steps from zero, the residual and the
//     restriction (Sec. 2.2.1) -- writes the iterate on the tile's owned
//     vertices and the coarse right-hand side of the tile's coarse vertices;
//   k_patch_up: interpolation and correction, then nu2 smoothing steps --
//     writes the corrected, smoothed iterate on the owned vertices.
//
// Every tile recomputes its ring vertices (the vertices within nu edges of its
// own, see host_patch.cpp).  Each phase computes exactly the rings the next
// phase reads: down, the first step (from zero, row-local) covers every ring,
// step k of nu covers rings 0 .. nu-k, and the residual ring 0; up, the
// interpolation covers every ring and step k rings 0 .. nu-1-k.  Each row takes the same
// operations in the same order as k_smooth0 / k_smooth / k_residual /
// k_restrict / k_prolong, so the results are bitwise those of the per-step
// kernels, with two launches per level and cycle instead of 2 nu + 2 or more.
// No block waits for another: the tiles only read what earlier kernels wrote.
#pragma once

#include "kernels.cuh"

namespace decdev {

constexpr int kPatchThreads = 256;
constexpr int kPatchHdrInts = 8;  // the host's kPatchHdr
constexpr int kPatchDepth = 3;    // the host's kPatchMaxDepth

template <typename T>
struct PatchArgs {
    const int32_t *hdr;   // kPatchHdrInts per tile (host_patch.cpp)
    const int32_t *gid;   // local -> level vertex
    const int32_t *lcol;  // local ELL columns (local indices), per tile slot-major
    const T *lw;          // local ELL weights
    int K;                // slots per row
    int depth;            // smoothing steps = rings
    int cheb;             // Chebyshev (directions carried) or damped Jacobi
    T c[kPatchDepth], e[kPatchDepth];  // the smoothing call's coefficients, steps 0 .. depth-1
    const T *b;           // the level's right-hand side
    T *x_out;             // the iterate after the tile's steps (owned vertices)
    // down
    const T *dg;          // stored Jacobi diagonal (the first step from zero)
    T *bc;                // coarse right-hand side
    int star0;            // restriction: *0-adjoint of interpolation instead of row-normalized
    const T *s0f, *s0c;   // *0 of this level and of the coarser one (star0)
    // up
    const T *x_in;        // the pre-smoothed iterate
    const T *ec;          // coarse correction
    const int2 *par;      // midpoint parents
    int nc;               // coarse vertex count
};

// |rings 0 .. k| from the header counts, without indexing the array by a runtime value
// (which would place it in local memory).
__device__ __forceinline__ int ring_count(const int n[kPatchDepth + 1], int k) {
    return k <= 0 ? n[0] : k == 1 ? n[1] : k == 2 ? n[2] : n[3];
}

// Dynamic shared memory of one block over a tile of `cap` locals: four vectors
// (b, two iterates, the direction) and three int arrays (vertex ids, parents).
template <typename T>
constexpr int patch_smem_bytes(int cap) { return cap * (4 * (int)sizeof(T) + 3 * (int)sizeof(int)); }

// Tile header of this block; returns the local ELL row count m.
__device__ __forceinline__ int patch_hdr(const int32_t *hdr, int depth, int &loc_off, int &row_off, int &nown,
                                         int &ncoarse, int n[kPatchDepth + 1]) {
    const int32_t *h = hdr + (size_t)blockIdx.x * kPatchHdrInts;
    loc_off = ldg(h);
    row_off = ldg(h + 1);
    nown = ldg(h + 2);
    ncoarse = ldg(h + 3);
#pragma unroll
    for (int k = 0; k <= kPatchDepth; ++k) n[k] = ldg(h + 4 + k);
    return ring_count(n, depth - 1);
}

// Before waiting for the previous kernel: pull the tile's local ELL into L1
// (it does not depend on earlier kernels; see pdl_prologue_ell).
template <typename T>
__device__ __forceinline__ void patch_prefetch(const int32_t *lcol, const T *lw, int count) {
    constexpr int kc = 128 / sizeof(int32_t), kw = 128 / sizeof(T);  // entries per 128-byte line
    for (int o = threadIdx.x * kc; o < count; o += blockDim.x * kc) prefetch_l1(lcol + o);
    for (int o = threadIdx.x * kw; o < count; o += blockDim.x * kw) prefetch_l1(lw + o);
}

// (L x)_i and L_ii from the local ELL and the shared-memory iterate, in
// row_apply's order.
template <typename T, int KT>
__device__ __forceinline__ void patch_row(int i, int m, int K, const int32_t *__restrict__ lc,
                                          const T *__restrict__ lw, const T *xs, T &s, T &d) {
    const int Kk = KT > 0 ? KT : K;
    const T xi = xs[i];
    s = T(0);
    d = T(0);
#pragma unroll
    for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
        if (KT == 0 && k >= Kk) break;
        const int o = k * m + i;
        const int j = ldg(lc + o);
        const T wk = ldg(lw + o);
        s = fma(wk, xi - xs[j], s);
        d += wk;
    }
}

// One smoothing step from a nonzero iterate on locals [0, rows) (k_smooth):
// xo = xi + delta, dd <- delta when dout (in place: a row reads only its own direction).
template <typename T, int KT>
__device__ __forceinline__ void patch_step(int rows, int m, int K, const int32_t *__restrict__ lc,
                                           const T *__restrict__ lw, const T *bs, const T *xi, T *xo, T *dd,
                                           bool din, bool dout, T c, T e) {
    for (int i = threadIdx.x; i < rows; i += blockDim.x) {
        T s, d;
        patch_row<T, KT>(i, m, K, lc, lw, xi, s, d);
        const T q = d != T(0) ? (bs[i] - s) / d : T(0);
        const T delta = smooth_delta<T>(din, c, din ? dd[i] : T(0), e, q);
        xo[i] = add_rn(xi[i], delta);
        if (dout) dd[i] = delta;
    }
}

template <typename T, int KT>
__global__ void __launch_bounds__(kPatchThreads) k_patch_down(PatchArgs<T> A, const int *skip) {
    extern __shared__ __align__(16) unsigned char patch_smem[];
    int loc_off, row_off, nown, ncoarse, n[kPatchDepth + 1];
    const int m = patch_hdr(A.hdr, A.depth, loc_off, row_off, nown, ncoarse, n);
    const int cap = ring_count(n, A.depth);
    T *bs = reinterpret_cast<T *>(patch_smem);
    T *xa = bs + cap, *xb = xa + cap, *dd = xb + cap;
    int *vid = reinterpret_cast<int *>(dd + cap);
    const int32_t *g = A.gid + loc_off;
    const int32_t *lc = A.lcol + row_off;
    const T *lw = A.lw + row_off;
    const int Kk = A.K;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    patch_prefetch(lc, lw, Kk * m);
    // before the wait: the tile's vertex ids and diagonals (no earlier kernel writes them);
    // each thread keeps the locals it reads again below
    for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        const int v = ldg(g + i);
        vid[i] = v;
        dd[i] = ldg(A.dg + v);
    }
    pdl_wait_only();
    if (skipped(skip)) return;
    const int nu = A.depth;
    // step 0 from zero on every ring (k_smooth0): x = e0 b / d
    const bool dout0 = A.cheb && nu > 1;
    for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        const T bi = ldg(A.b + vid[i]), di = dd[i];
        const T x1 = di != T(0) ? A.e[0] * (bi / di) : T(0);
        bs[i] = bi;
        xa[i] = x1;
        if (dout0) dd[i] = x1;
    }
    __syncthreads();
    T *xc = xa, *xn = xb;
    for (int k = 1; k < nu; ++k) {
        patch_step<T, KT>(ring_count(n, nu - k), m, Kk, lc, lw, bs, xc, xn, dd, A.cheb != 0, A.cheb && k + 1 < nu, A.c[k],
                          A.e[k]);
        __syncthreads();
        T *t = xc;
        xc = xn;
        xn = t;
    }
    // residual on ring 0 (k_residual), into the free buffer
    T *rs = xn;
    for (int i = threadIdx.x; i < n[0]; i += blockDim.x) {
        T s, d;
        patch_row<T, KT>(i, m, Kk, lc, lw, xc, s, d);
        rs[i] = d != T(0) ? bs[i] - s : T(0);
    }
    __syncthreads();
    // restriction onto the tile's coarse vertices (k_restrict): local row j is the
    // fine copy of coarse vertex g[j]; its slots list the adjacent midpoints
    for (int j = threadIdx.x; j < ncoarse; j += blockDim.x) {
        const int c = vid[j];
        T acc = T(0);
        int deg = 0;
#pragma unroll
        for (int k = 0; k < (KT > 0 ? KT : 32); ++k) {
            if (KT == 0 && k >= Kk) break;
            const int jj = ldg(lc + k * m + j);
            if (jj != j) {
                acc = A.star0 ? fma(ldg(A.s0f + vid[jj]), rs[jj], acc) : acc + rs[jj];
                ++deg;
            }
        }
        T v;
        if (A.star0)
            v = fma(ldg(A.s0f + c), rs[j], T(0.5) * acc) / ldg(A.s0c + c);
        else
            v = fma(T(0.5), acc, rs[j]) / add_rn(T(1), mul_rn(T(0.5), T(deg)));
        A.bc[c] = v;
    }
    for (int i = threadIdx.x; i < nown; i += blockDim.x) A.x_out[vid[i]] = xc[i];
}

template <typename T, int KT>
__global__ void __launch_bounds__(kPatchThreads) k_patch_up(PatchArgs<T> A, const int *skip) {
    extern __shared__ __align__(16) unsigned char patch_smem[];
    int loc_off, row_off, nown, ncoarse, n[kPatchDepth + 1];
    const int m = patch_hdr(A.hdr, A.depth, loc_off, row_off, nown, ncoarse, n);
    const int cap = ring_count(n, A.depth);
    T *bs = reinterpret_cast<T *>(patch_smem);
    T *xa = bs + cap, *xb = xa + cap, *dd = xb + cap;
    int *vid = reinterpret_cast<int *>(dd + cap), *pa = vid + cap, *pb = pa + cap;
    const int32_t *g = A.gid + loc_off;
    const int32_t *lc = A.lcol + row_off;
    const T *lw = A.lw + row_off;
    const int Kk = A.K;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    patch_prefetch(lc, lw, Kk * m);
    // before the wait: vertex ids and midpoint parents (no earlier kernel writes them)
    for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        const int v = ldg(g + i);
        vid[i] = v;
        if (v >= A.nc) {
            const int2 p = ldg(A.par + (v - A.nc));
            pa[i] = p.x;
            pb[i] = p.y;
        }
    }
    pdl_wait_only();
    if (skipped(skip)) return;
    const int nu = A.depth;
    // interpolation and correction on every ring (k_prolong, prolong_add's rounding)
    for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        const int v = vid[i];
        const T e = v < A.nc ? ldg(A.ec + v) : mul_rn(T(0.5), add_rn(ldg(A.ec + pa[i]), ldg(A.ec + pb[i])));
        xa[i] = add_rn(ldg(A.x_in + v), e);
        if (i < m) bs[i] = ldg(A.b + v);
    }
    __syncthreads();
    T *xc = xa, *xn = xb;
    for (int k = 0; k < nu; ++k) {
        patch_step<T, KT>(ring_count(n, nu - 1 - k), m, Kk, lc, lw, bs, xc, xn, dd, A.cheb && k > 0, A.cheb && k + 1 < nu,
                          A.c[k], A.e[k]);
        __syncthreads();
        T *t = xc;
        xc = xn;
        xn = t;
    }
    for (int i = threadIdx.x; i < nown; i += blockDim.x) A.x_out[vid[i]] = xc[i];
}

}  // namespace decdev
