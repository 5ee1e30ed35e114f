// Device-side state of a libdec hierarchy (struct dec_mg) and the launch
// helpers shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <type_traits>
#include <vector>

#include "coarse_cycle.cuh"
#include "host.h"
#include "kernels.cuh"
#include "patch.cuh"

namespace decimpl {

struct DevLevel {
    int n = 0, K = 0, nc = 0;  // nc: vertex count of the next coarser level
    int64_t ne = 0;
    int32_t *col = nullptr;
    double *w64 = nullptr;
    float *w32 = nullptr;
    float *wlo = nullptr;  // finest level: w64 - w32 rounded to FP32 (ff weights w32 + wlo)
    float *dg32 = nullptr;     // row sums of w32 / w64 (the Jacobi diagonal), read by fused kernels
    // general geometric map to the next coarser level (cubic subdivision): 3 (coarse vertex,
    // weight) slots per row, slot-major; restriction rows of the coarser level, Kr slots
    int32_t *gidx = nullptr;
    float *gw32 = nullptr;
    double *gw64 = nullptr;
    int gKr = 0;
    int32_t *ridx = nullptr;
    float *rw32 = nullptr;
    double *rw64 = nullptr;
    int32_t *crow = nullptr;   // rows sorted by greedy colour (multicolour Gauss-Seidel)
    std::vector<int> coff;     // colour c owns crow[coff[c] .. coff[c+1])
    int16_t *col16 = nullptr;  // levels of the shared-memory coarse cycle: col and parents as int16
    int16_t *par16 = nullptr;
    double *dg64 = nullptr;
    double *star0 = nullptr;
    float *star0_32 = nullptr;
    uint8_t *freev = nullptr;
    int2 *par = nullptr;
    float *x32[2] = {nullptr, nullptr}, *d32[2] = {nullptr, nullptr}, *r32 = nullptr, *b32 = nullptr;
    double *x64[2] = {nullptr, nullptr}, *d64[2] = {nullptr, nullptr}, *r64 = nullptr, *b64 = nullptr;
    // W-cycles (gamma > 1): accumulated coarse correction and the right-hand side of a repeat
    float *y32 = nullptr, *c32 = nullptr;
    double *y64 = nullptr, *c64 = nullptr;
    // Chebyshev coefficients (c_k, e_k) of one smoothing call of nu1 and nu2 steps
    std::vector<double> c_pre, e_pre, c_post, e_post;
    // halo tiles of this level (DEC_FUSE_PATCH, host_patch.cpp): ntiles == 0 if none
    struct Tiles {
        int ntiles = 0, depth = 0, threads = 0, smem32 = 0, smem64 = 0;  // smem: bytes per block, FP32 / FP64
        int32_t *hdr = nullptr, *gid = nullptr, *lcol = nullptr;
        float *lw32 = nullptr;
        double *lw64 = nullptr;
    };
    Tiles tdown, tup;
};

template <typename T> struct P;
template <> struct P<float> {
    static float *x(DevLevel &L, int i) { return L.x32[i]; }
    static float *d(DevLevel &L, int i) { return L.d32[i]; }
    static float *r(DevLevel &L) { return L.r32; }
    static float *b(DevLevel &L) { return L.b32; }
    static const float *w(const DevLevel &L) { return L.w32; }
    static const float *s0(const DevLevel &L) { return L.star0_32; }
    static const float *dg(const DevLevel &L) { return L.dg32; }
    static const float *gw(const DevLevel &L) { return L.gw32; }
    static const float *rw(const DevLevel &L) { return L.rw32; }
    static float *y(DevLevel &L) { return L.y32; }
    static float *c(DevLevel &L) { return L.c32; }
    static const float *lw(const DevLevel::Tiles &t) { return t.lw32; }
    static int smem(const DevLevel::Tiles &t) { return t.smem32; }
};
template <> struct P<double> {
    static double *x(DevLevel &L, int i) { return L.x64[i]; }
    static double *d(DevLevel &L, int i) { return L.d64[i]; }
    static double *r(DevLevel &L) { return L.r64; }
    static double *b(DevLevel &L) { return L.b64; }
    static const double *w(const DevLevel &L) { return L.w64; }
    static const double *s0(const DevLevel &L) { return L.star0; }
    static const double *dg(const DevLevel &L) { return L.dg64; }
    static const double *gw(const DevLevel &L) { return L.gw64; }
    static const double *rw(const DevLevel &L) { return L.rw64; }
    static double *y(DevLevel &L) { return L.y64; }
    static double *c(DevLevel &L) { return L.c64; }
    static const double *lw(const DevLevel::Tiles &t) { return t.lw64; }
    static int smem(const DevLevel::Tiles &t) { return t.smem64; }
};

template <typename F>
void dispatch_k(int K, F &&f) {
    if (K == 6)
        f(std::integral_constant<int, 6>{});
    else
        f(std::integral_constant<int, 0>{});
}

}  // namespace decimpl

struct dec_mg {
    decimpl::HostHierarchy H;
    int device = 0;
    int nsm = 152;
    std::vector<decimpl::DevLevel> lv;
    int n0 = 0;
    double *G64 = nullptr;
    float *G32 = nullptr;
    // shared-memory coarse cycle (DEC_FUSE_COARSE): levels 0..coarse_top, -1 if none fits
    int coarse_top = -1;
    int coarse_smem = 0;
    bool coarse_k6 = false;  // every fused level above the coarsest has 6 stencil slots
    decdev::CoarseArgs coarse_args{};
    // finest-level extras
    int32_t *slot_edge = nullptr;
    int2 *edges = nullptr;
    double *verts = nullptr;  // [n * dim] finest coordinates
    int dim = 2;
    double *pot = nullptr, *ptmp = nullptr, *prhs = nullptr;  // porous-step work vectors
    // outer-iteration workspace (finest level, FP64)
    double *ox = nullptr, *orr = nullptr, *op = nullptr, *oq = nullptr, *ozn = nullptr, *ozo = nullptr, *ob = nullptr;
    float *zo32 = nullptr;     // previous preconditioned vector (mixed precision)
    // float-float outer iteration: hi/lo arrays of x, r (hi = the finest b32), q, b; FP32 p
    float *fxh = nullptr, *fxl = nullptr, *frl = nullptr, *fqh = nullptr, *fql = nullptr, *fp = nullptr;
    float *fbh = nullptr, *fbl = nullptr;
    double *tmp = nullptr;
    // contiguous columns for calls with several interleaved right-hand sides (allocated on first use)
    double *kx64 = nullptr;
    float *kb32 = nullptr, *kx32 = nullptr;
    double *partials = nullptr;
    unsigned *counter = nullptr;
    decdev::Scal *scal = nullptr;
    decdev::Scal *scal_h = nullptr;  // pinned host mirror
    double star0_sum = 0.0;
    cudaStream_t cap = nullptr;
    // [solver][mode]
    cudaGraphExec_t graphs[3][4] = {};
    // whole iteration loop on the device: a while node around one iteration
    cudaGraphExec_t loops[3][4] = {};
    bool no_device_loop = false;  // set if the driver refuses conditional nodes
    int64_t loop_kernels[3][4] = {};  // kernel nodes in one pass of a loop body
    std::vector<void *> allocs;
    size_t bytes = 0;
    bool host_only = false;
    bool pdl = true;  // programmatic dependent launch between consecutive kernels
    // live kernel timing (dec_mg_profile)
    int64_t launches = 0;       // kernels enqueued outside graph capture
    int64_t graph_kernels[3][4] = {};  // kernel nodes per captured iteration graph
    int prof = 0;               // 0 off, 1 finest level, 2 all levels
    bool prof_capture = false;  // true while a profiled iteration graph is being captured
    bool capturing = false;     // true while any iteration graph is being captured
    struct Slot {
        cudaEvent_t a, b;
        int kind, level;
    };
    std::vector<Slot> slots;
    double prof_ms[DEC_PK_COUNT][16] = {};
    int64_t prof_n[DEC_PK_COUNT][16] = {};
};

namespace decimpl {

using decdev::kMaxRedBlocks;
using decdev::kThreads;

inline int fail(const Status &s) {
    decimpl::set_error(s.msg);
    return s.code;
}

inline int cuda_fail(cudaError_t e, const char *where) {
    decimpl::set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return DEC_ERR_CUDA;
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);       \
    } while (0)

template <typename T>
inline int dalloc(dec_mg *mg, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        decimpl::set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? DEC_ERR_OOM : DEC_ERR_CUDA;
    }
    mg->allocs.push_back((void *)*p);
    mg->bytes += count * sizeof(T);
    return DEC_OK;
}

template <typename T>
inline int upload(dec_mg *mg, T **p, const T *src, size_t count) {
    int rc = dalloc(mg, p, count);
    if (rc) return rc;
    CK(cudaMemcpy(*p, src, count * sizeof(T), cudaMemcpyHostToDevice));
    return DEC_OK;
}

// Every kernel goes through here: a plain launch, or one with programmatic
// stream serialization (PDL) so that consecutive kernels overlap their launch
// latency; inside stream capture this becomes a programmatic graph edge.
template <typename... KArgs, typename... Args>
inline void launch(const dec_mg *mg, void (*kernel)(KArgs...), int grid, cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = mg->pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// A launch with an explicit block size and dynamic shared memory (PDL as above).
template <typename... KArgs, typename... Args>
inline void launch_block(const dec_mg *mg, void (*kernel)(KArgs...), int grid, int block, int smem, cudaStream_t s,
                         Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = mg->pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

inline int grid_for(const dec_mg *mg, int64_t n) {
    int64_t g = (n + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)mg->nsm * 8;
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

inline int red_grid(const dec_mg *mg, int64_t n) {
    int64_t g = (n + kThreads - 1) / kThreads;
    int64_t cap = std::min<int64_t>(kMaxRedBlocks, (int64_t)mg->nsm * 8);
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

// Grid of a kernel whose per-row work and sums are FP64: one wave of
// decdev::kFp64Blocks blocks per SM (half the blocks of the FP32 kernels), so
// every thread adds about twice the rows before its FP64 warp and block sums
// -- on GB300's narrow FP64 pipe those sums cost more than the rows at one or
// two rows per thread -- and, with 64 registers, keeps four rows' loads in flight.
inline int red_grid64(const dec_mg *mg, int64_t n) {
    int64_t g = (n + kThreads - 1) / kThreads;
    int64_t cap = std::min<int64_t>(kMaxRedBlocks, (int64_t)mg->nsm * decdev::kFp64Blocks);
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

}  // namespace decimpl
