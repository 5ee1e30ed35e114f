// Device orchestration of libdec: hierarchy upload, the multigrid cycle,
// the outer FP64 iterations (standalone MG / iterative refinement, flexible
// MG-preconditioned CG, plain CG), the adjoint solve, and their C ABI.
//
// The cycle follows Sec. 2.2.1 and Sec. 3.1.1: smoothing, residual,
// restriction by the row-normalized transpose of the subdivision matrix,
// recursion, interpolation by the subdivision matrix, smoothing; the
// coarsest level applies a dense precomputed solution operator.  The outer
// CG uses the *0 inner product in which L is self-adjoint and the
// Polak-Ribiere beta because the V-cycle is only approximately symmetric.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "host.h"
#include "kernels.cuh"
#include "mg_device.h"

using decimpl::Status;
using namespace decdev;
using namespace decimpl;

const decimpl::HostMesh *dec_mesh_host(const dec_mesh *m);


namespace {

void clear_slots(dec_mg *mg);
void drop_graphs(dec_mg *mg);

void free_all(dec_mg *mg) {
    drop_graphs(mg);
    for (void *p : mg->allocs) cudaFree(p);
    mg->allocs.clear();
    if (mg->scal_h) cudaFreeHost(mg->scal_h);
    if (mg->cap) cudaStreamDestroy(mg->cap);
}

// Brackets one kernel launch with an event pair while the profiled iteration
// graph is being captured.
struct ProfScope {
    dec_mg *mg;
    cudaStream_t s;
    int idx = -1;
    ProfScope(dec_mg *m, int kind, int level, cudaStream_t st) : mg(m), s(st) {
        if (!mg->capturing) mg->launches += 1;
        if (!mg->prof_capture) return;
        if (mg->prof == 1 && level != (int)mg->lv.size() - 1) return;
        dec_mg::Slot sl{nullptr, nullptr, kind, level};
        if (cudaEventCreate(&sl.a) != cudaSuccess || cudaEventCreate(&sl.b) != cudaSuccess) return;
        idx = (int)mg->slots.size();
        mg->slots.push_back(sl);
        // inside stream capture only an "external" record becomes an event-record node
        cudaEventRecordWithFlags(sl.a, s, cudaEventRecordExternal);
    }
    ~ProfScope() {
        if (idx >= 0) cudaEventRecordWithFlags(mg->slots[idx].b, s, cudaEventRecordExternal);
    }
};

void clear_slots(dec_mg *mg) {
    for (auto &sl : mg->slots) {
        cudaEventDestroy(sl.a);
        cudaEventDestroy(sl.b);
    }
    mg->slots.clear();
}

void drop_graphs(dec_mg *mg) {
    for (auto &row : mg->graphs)
        for (auto &g : row)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    for (auto &row : mg->loops)
        for (auto &g : row)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    clear_slots(mg);
}

void accumulate_slots(dec_mg *mg) {
    for (auto &sl : mg->slots) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, sl.a, sl.b) == cudaSuccess) {
            mg->prof_ms[sl.kind][sl.level] += ms;
            mg->prof_n[sl.kind][sl.level] += 1;
        } else {
            (void)cudaGetLastError();  // a failed read must not surface as a later launch error
        }
    }
}

void cheb_coeffs(double lmax, double lo, double hi, int nu, std::vector<double> &c, std::vector<double> &e) {
    c.clear();
    e.clear();
    const double a = lo * lmax, b = hi * lmax;
    const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
    c.push_back(0.0);
    e.push_back(1.0 / theta);
    double rho_prev = 1.0 / sigma;
    for (int k = 1; k < nu; ++k) {
        double rho = 1.0 / (2.0 * sigma - rho_prev);
        c.push_back(rho * rho_prev);
        e.push_back(2.0 * rho / delta);
        rho_prev = rho;
    }
}

// ---------------------------------------------------------------------------
// the cycle
// ---------------------------------------------------------------------------

// nu smoothing steps on level l; if from_zero the iterate starts at 0.
// `cur` is the x buffer index holding the iterate on entry/exit.
// The outer dot products of the preconditioned vector, to be fused into the
// last post-smoothing step of the finest level (DEC_FUSE_OUTER).
struct DotsArgs {
    int first = 0, gauge = 0;
    bool d64 = false;   // FP64 dot products with the FP64 residual (DEC_MODE_MIXED)
    bool done = false;  // set once the fused kernel has been enqueued
};

// Steps k_start .. nu-1 of one smoothing call on level l.  From zero with
// fused kernels, steps 0 and 1 run as one k_smooth01 launch.
// A DEC_FUSE_* bit on a level of n rows: the row-local fusions apply on
// every level, the gathering ones (SMOOTH01, RESTRICT, PROLONG) on levels of
// at most fuse_max_rows rows (0: every level).
inline bool fuse_here(const dec_mg_opts &o, int bit, int64_t n) {
    if (!(o.fuse & bit)) return false;
    const bool gathering = (bit & (DEC_FUSE_SMOOTH01 | DEC_FUSE_RESTRICT | DEC_FUSE_PROLONG)) != 0;
    return !gathering || o.fuse_max_rows <= 0 || n <= o.fuse_max_rows;
}

template <typename T>
void smooth(dec_mg *mg, int l, const T *b, int nu, bool from_zero, bool post, int &cur, cudaStream_t s,
            const int *skip, int k_start = 0, DotsArgs *da = nullptr) {
    DevLevel &L = mg->lv[l];
    const dec_mg_opts &o = mg->H.opts;
    if (o.smoother == DEC_SMOOTH_MCGS) {
        // multicolour Gauss-Seidel: nu sweeps over the colour classes in increasing
        // colour order, in place on the current iterate (zero when from_zero)
        if (from_zero) {
            cur = 0;
            cudaMemsetAsync(P<T>::x(L, 0), 0, sizeof(T) * L.n, s);
        }
        T *x = P<T>::x(L, cur);
        dispatch_k(L.K, [&](auto kt) {
            constexpr int KT = decltype(kt)::value;
            for (int k = k_start; k < nu; ++k)
                for (size_t c = 0; c + 1 < L.coff.size(); ++c) {
                    const int cnt = L.coff[c + 1] - L.coff[c];
                    ProfScope ps(mg, DEC_PK_SMOOTH, l, s);
                    launch(mg, k_mcgs<T, KT>, grid_for(mg, cnt), s, L.n, L.K, (const int32_t *)L.col, P<T>::w(L), b, x,
                           (const int32_t *)(L.crow + L.coff[c]), cnt, skip);
                }
        });
        return;
    }
    const bool cheb = o.smoother == DEC_SMOOTH_CHEBYSHEV;
    const std::vector<double> &cc = post ? L.c_post : L.c_pre;
    const std::vector<double> &ee = post ? L.e_post : L.e_pre;
    const int g = grid_for(mg, L.n);
    const T *w = P<T>::w(L);
    dispatch_k(L.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        if (from_zero && k_start == 0 && nu >= 2 && fuse_here(o, DEC_FUSE_SMOOTH01, L.n)) {
            const T e0 = (T)(cheb ? ee[0] : o.omega), e1 = (T)(cheb ? ee[1] : o.omega);
            const T c1 = (T)(cheb ? cc[1] : 0.0);
            const bool dout = cheb && 2 < nu;
            ProfScope ps(mg, DEC_PK_SMOOTH01, l, s);
            const T *dg = P<T>::dg(L);
            T *xo = P<T>::x(L, 1), *dn = dout ? P<T>::d(L, 1) : nullptr;
            if (cheb && dout)
                launch(mg, k_smooth01<T, KT, true, true>, g, s, L.n, L.K, L.col, w, dg, b, xo, dn, e0, c1, e1, skip);
            else if (cheb)
                launch(mg, k_smooth01<T, KT, true, false>, g, s, L.n, L.K, L.col, w, dg, b, xo, dn, e0, c1, e1, skip);
            else
                launch(mg, k_smooth01<T, KT, false, false>, g, s, L.n, L.K, L.col, w, dg, b, xo, dn, e0, c1, e1, skip);
            cur = 1;
            k_start = 2;
        }
        for (int k = k_start; k < nu; ++k) {
            const T e = (T)(cheb ? ee[k] : o.omega);
            const T c = (T)(cheb ? cc[k] : 0.0);
            const bool dout = cheb && k + 1 < nu;
            if (k == 0 && from_zero) {
                cur = 0;
                ProfScope ps(mg, DEC_PK_SMOOTH0, l, s);
                if constexpr (std::is_same<T, double>::value) {
                    // FP64: the stored diagonal (the same double) instead of six FP64 additions per row
                    if (dout)
                        launch(mg, k_smooth0_dg<true>, g, s, L.n, (const double *)L.dg64, b, P<T>::x(L, 0),
                               P<T>::d(L, 0), e, skip);
                    else
                        launch(mg, k_smooth0_dg<false>, g, s, L.n, (const double *)L.dg64, b, P<T>::x(L, 0),
                               (double *)nullptr, e, skip);
                } else if (dout)
                    launch(mg, k_smooth0<T, KT, true>, g, s, L.n, L.K, w, b, P<T>::x(L, 0), P<T>::d(L, 0), e, skip);
                else
                    launch(mg, k_smooth0<T, KT, false>, g, s, L.n, L.K, w, b, P<T>::x(L, 0), nullptr, e, skip);
                continue;
            }
            const int nxt = 1 - cur;
            const bool din = cheb && k > 0;
            T *xi = P<T>::x(L, cur), *xo = P<T>::x(L, nxt);
            T *di = P<T>::d(L, cur), *dn = P<T>::d(L, nxt);
            if constexpr (std::is_same<T, float>::value) {
                if (da && post && k == nu - 1) {
                    DevLevel &F = mg->lv.back();
                    ProfScope ps(mg, DEC_PK_SMOOTHDOTS, l, s);
                    const int rg = da->d64 ? red_grid64(mg, L.n) : red_grid(mg, L.n);
                    if (da->d64) {
                        if (din)
                            launch(mg, k_smooth_zdots_d<KT, true>, rg, s, L.n, L.K, (const int32_t *)L.col, w, b,
                                   (const float *)xi, (const float *)di, xo, c, e, (const double *)F.star0,
                                   (const uint8_t *)F.freev, (const double *)mg->orr, (const double *)mg->ozo,
                                   da->first, da->gauge, mg->partials, mg->counter, mg->scal, skip);
                        else
                            launch(mg, k_smooth_zdots_d<KT, false>, rg, s, L.n, L.K, (const int32_t *)L.col, w, b,
                                   (const float *)xi, (const float *)nullptr, xo, c, e, (const double *)F.star0,
                                   (const uint8_t *)F.freev, (const double *)mg->orr, (const double *)mg->ozo,
                                   da->first, da->gauge, mg->partials, mg->counter, mg->scal, skip);
                    } else if (din)
                        launch(mg, k_smooth_zdots<KT, true>, rg, s, L.n, L.K, (const int32_t *)L.col, w, b,
                               (const float *)xi, (const float *)di, xo, c, e, (const float *)F.star0_32,
                               (const uint8_t *)F.freev, (const float *)mg->zo32, da->first, da->gauge,
                               mg->partials, mg->counter, mg->scal, skip);
                    else
                        launch(mg, k_smooth_zdots<KT, false>, rg, s, L.n, L.K, (const int32_t *)L.col, w, b,
                               (const float *)xi, (const float *)nullptr, xo, c, e, (const float *)F.star0_32,
                               (const uint8_t *)F.freev, (const float *)mg->zo32, da->first, da->gauge,
                               mg->partials, mg->counter, mg->scal, skip);
                    da->done = true;
                    cur = nxt;
                    continue;
                }
            }
            ProfScope ps(mg, DEC_PK_SMOOTH, l, s);
            if constexpr (std::is_same<T, double>::value) {
                const double *dg = L.dg64;
                if (din && dout)
                    launch(mg, k_smooth_dg<KT, true, true>, g, s, L.n, L.K, L.col, w, dg, b, xi, di, xo, dn, c, e, skip);
                else if (din)
                    launch(mg, k_smooth_dg<KT, true, false>, g, s, L.n, L.K, L.col, w, dg, b, xi, di, xo,
                           (double *)nullptr, c, e, skip);
                else if (dout)
                    launch(mg, k_smooth_dg<KT, false, true>, g, s, L.n, L.K, L.col, w, dg, b, xi, (const double *)nullptr,
                           xo, dn, c, e, skip);
                else
                    launch(mg, k_smooth_dg<KT, false, false>, g, s, L.n, L.K, L.col, w, dg, b, xi,
                           (const double *)nullptr, xo, (double *)nullptr, c, e, skip);
            } else if (din && dout)
                launch(mg, k_smooth<T, KT, true, true>, g, s, L.n, L.K, L.col, w, b, xi, di, xo, dn, c, e, skip);
            else if (din)
                launch(mg, k_smooth<T, KT, true, false>, g, s, L.n, L.K, L.col, w, b, xi, di, xo, nullptr, c, e, skip);
            else if (dout)
                launch(mg, k_smooth<T, KT, false, true>, g, s, L.n, L.K, L.col, w, b, xi, nullptr, xo, dn, c, e, skip);
            else
                launch(mg, k_smooth<T, KT, false, false>, g, s, L.n, L.K, L.col, w, b, xi, nullptr, xo, nullptr, c, e, skip);
            cur = nxt;
        }
    });
}

// Enqueue one cycle C_l(b) with zero initial guess; returns the level-l
// buffer that holds the result.
// pre0_done: the first pre-smoothing step (from zero) of this level already
// ran, fused into the kernel that produced b; x[0] (and d[0]) hold it.
// da: fuse the last post-smoothing step of this (finest) level with the
// outer dot products.
// kind: the cycle below this level -- gamma repetitions of the same kind (V
// for gamma = 1, W), a single V, or F (an F-cycle, then a V-cycle); -1 takes
// the hierarchy's option.
enum { kCycGamma = 0, kCycV = 1, kCycF = 2 };
// Level l runs as halo tiles (DEC_FUSE_PATCH; tiles exist only where setup_patches built them).
inline bool patch_at(const dec_mg *mg, int l) {
    return (mg->H.opts.fuse & DEC_FUSE_PATCH) && l >= 1 && l < (int)mg->lv.size() && mg->lv[l].tdown.ntiles > 0;
}
template <typename T>
T *cycle(dec_mg *mg, int l, const T *b, cudaStream_t s, const int *skip, bool pre0_done = false,
         DotsArgs *da = nullptr, int kind = -1) {
    if (kind < 0) kind = mg->H.opts.fcycle ? kCycF : kCycGamma;
    DevLevel &L = mg->lv[l];
    if (l == 0) {
        const T *G;
        if constexpr (std::is_same<T, float>::value) G = mg->G32; else G = mg->G64;
        int g = (int)std::min<int64_t>(mg->nsm * 4, (L.n * 32 + kThreads - 1) / kThreads);
        ProfScope ps(mg, DEC_PK_COARSE, 0, s);
        launch(mg, k_coarse<T>, g, s, L.n, G, b, P<T>::x(L, 0), skip);
        return P<T>::x(L, 0);
    }
    const dec_mg_opts &o = mg->H.opts;
    if constexpr (std::is_same<T, float>::value) {
        if ((o.fuse & DEC_FUSE_COARSE) && l == mg->coarse_top) {
            decdev::CoarseArgs A = mg->coarse_args;
            A.b = b;
            A.x = L.x32[0];
            ProfScope ps(mg, DEC_PK_COARSECYCLE, l, s);
            if (mg->coarse_k6)
                launch_block(mg, decdev::k_coarse_cycle<6>, 1, decdev::kCoarseThreads, mg->coarse_smem, s, A, skip);
            else
                launch_block(mg, decdev::k_coarse_cycle<0>, 1, decdev::kCoarseThreads, mg->coarse_smem, s, A, skip);
            return L.x32[0];
        }
    }
    if (patch_at(mg, l)) {
        // halo tiles: pre-smoothing, residual and restriction in one launch; interpolation,
        // correction and post-smoothing in another (patch.cuh), bitwise the per-step kernels
        DevLevel &C = mg->lv[l - 1];
        const bool cheb = o.smoother == DEC_SMOOTH_CHEBYSHEV;
        decdev::PatchArgs<T> A{};
        A.K = L.K;
        A.cheb = cheb ? 1 : 0;
        A.b = b;
        auto tiles = [&](const DevLevel::Tiles &t, const std::vector<double> &cc, const std::vector<double> &ee) {
            A.hdr = t.hdr;
            A.gid = t.gid;
            A.lcol = t.lcol;
            A.lw = P<T>::lw(t);
            A.depth = t.depth;
            for (int k = 0; k < t.depth; ++k) {
                A.c[k] = (T)(cheb ? cc[k] : 0.0);
                A.e[k] = (T)(cheb ? ee[k] : o.omega);
            }
        };
        tiles(L.tdown, L.c_pre, L.e_pre);
        A.x_out = P<T>::x(L, 0);
        A.dg = P<T>::dg(L);
        A.bc = P<T>::b(C);
        A.star0 = o.restriction == DEC_RESTRICT_STAR0 ? 1 : 0;
        A.s0f = P<T>::s0(L);
        A.s0c = P<T>::s0(C);
        dispatch_k(L.K, [&](auto kt) {
            constexpr int KT = decltype(kt)::value;
            ProfScope ps(mg, DEC_PK_PATCHDOWN, l, s);
            launch_block(mg, decdev::k_patch_down<T, KT>, L.tdown.ntiles, L.tdown.threads, P<T>::smem(L.tdown),
                         s, A, skip);
        });
        T *ec = cycle<T>(mg, l - 1, P<T>::b(C), s, skip, false, nullptr, kind);
        tiles(L.tup, L.c_post, L.e_post);
        A.x_in = P<T>::x(L, 0);
        A.ec = ec;
        A.par = L.par;
        A.nc = C.n;
        A.x_out = P<T>::x(L, 1);
        dispatch_k(L.K, [&](auto kt) {
            constexpr int KT = decltype(kt)::value;
            ProfScope ps(mg, DEC_PK_PATCHUP, l, s);
            launch_block(mg, decdev::k_patch_up<T, KT>, L.tup.ntiles, L.tup.threads, P<T>::smem(L.tup), s, A,
                         skip);
        });
        return P<T>::x(L, 1);
    }
    DevLevel &C = mg->lv[l - 1];
    int cur = 0;
    if (o.nu1 > 0)
        smooth<T>(mg, l, b, o.nu1, true, false, cur, s, skip, pre0_done ? 1 : 0);
    else
        cudaMemsetAsync(P<T>::x(L, 0), 0, sizeof(T) * L.n, s);
    // the coarse level's first smoothing step rides on the restriction
    // (not into the shared-memory coarse cycle, which starts from b itself)
    const bool coarse_next = std::is_same<T, float>::value && (o.fuse & DEC_FUSE_COARSE) && l - 1 == mg->coarse_top;
    const bool mapped = mg->H.mapped;  // general map transfers (k_restrict_map, k_prolong_map), unfused
    // (nor into halo tiles, which recompute it on their rings)
    const bool restrict0 = (o.fuse & DEC_FUSE_RESTRICT0) && l - 1 > 0 && o.nu1 > 0 && !coarse_next &&
                           o.smoother != DEC_SMOOTH_MCGS && !mapped && !patch_at(mg, l - 1);
    bool coarse_pre0 = false;
    const int g = grid_for(mg, L.n);
    const T *w = P<T>::w(L);
    dispatch_k(L.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        if (fuse_here(o, DEC_FUSE_RESTRICT, L.n) && L.K <= 7 && !mapped) {
            ProfScope ps(mg, DEC_PK_RESRESTRICT, l, s);
            const int gr = grid_for(mg, (int64_t)C.n * 8);
            const T *s0l = P<T>::s0(L), *s0c = P<T>::s0(C);
            const bool st0 = o.restriction == DEC_RESTRICT_STAR0;
            // with DEC_FUSE_RESTRICT0 the coarse level's first smoothing step rides along (S0)
            const int s0 = restrict0 ? (o.smoother == DEC_SMOOTH_CHEBYSHEV && 1 < o.nu1 ? 2 : 1) : 0;
            const T e0 = restrict0 ? (T)(o.smoother == DEC_SMOOTH_CHEBYSHEV ? C.e_pre[0] : o.omega) : T(0);
            const T *dgc = P<T>::dg(C);
            T *xc = P<T>::x(C, 0), *dc = P<T>::d(C, 0), *bcv = P<T>::b(C);
            const T *xl = P<T>::x(L, cur);
            auto go = [&](auto st0c, auto s0c_) {
                constexpr bool ST0 = decltype(st0c)::value;
                constexpr int S0 = decltype(s0c_)::value;
                launch(mg, k_residual_restrict<T, KT, ST0, S0>, gr, s, C.n, L.n, L.K, L.col, w, b, xl, bcv,
                       ST0 ? s0l : (const T *)nullptr, ST0 ? s0c : (const T *)nullptr, skip, dgc, xc, dc, e0);
            };
            using F = std::false_type;
            using Tr = std::true_type;
            using I0 = std::integral_constant<int, 0>;
            using I1 = std::integral_constant<int, 1>;
            using I2 = std::integral_constant<int, 2>;
            if (st0) {
                if (s0 == 2) go(Tr{}, I2{}); else if (s0 == 1) go(Tr{}, I1{}); else go(Tr{}, I0{});
            } else {
                if (s0 == 2) go(F{}, I2{}); else if (s0 == 1) go(F{}, I1{}); else go(F{}, I0{});
            }
            coarse_pre0 = s0 > 0;
            return;
        }
        {
            ProfScope ps(mg, DEC_PK_RESIDUAL, l, s);
            if constexpr (std::is_same<T, double>::value)
                launch(mg, k_residual_dg<KT>, g, s, L.n, L.K, L.col, w, (const double *)L.dg64, b,
                       (const double *)P<T>::x(L, cur), P<T>::r(L), skip);
            else
                launch(mg, k_residual<T, KT>, g, s, L.n, L.K, L.col, w, b, P<T>::x(L, cur), P<T>::r(L), skip);
        }
        {
            ProfScope ps(mg, DEC_PK_RESTRICT, l, s);
            const int gc = grid_for(mg, C.n);
            if (mapped) {
                launch(mg, k_restrict_map<T>, gc, s, C.n, L.gKr, (const int32_t *)L.ridx, P<T>::rw(L),
                       (const T *)P<T>::r(L), P<T>::b(C), skip);
            } else if (restrict0) {
                const bool cheb = o.smoother == DEC_SMOOTH_CHEBYSHEV;
                const T e0 = (T)(cheb ? C.e_pre[0] : o.omega);
                const bool dout = cheb && 1 < o.nu1;
                const T *dgc = P<T>::dg(C);
                T *xc = P<T>::x(C, 0), *dc = P<T>::d(C, 0);
                const T *s0l = P<T>::s0(L), *s0c = P<T>::s0(C);
                if (o.restriction == DEC_RESTRICT_STAR0) {
                    if (dout)
                        launch(mg, k_restrict<T, KT, true, 2>, gc, s, C.n, L.n, L.K, L.col, P<T>::r(L), P<T>::b(C),
                               s0l, s0c, skip, dgc, xc, dc, e0);
                    else
                        launch(mg, k_restrict<T, KT, true, 1>, gc, s, C.n, L.n, L.K, L.col, P<T>::r(L), P<T>::b(C),
                               s0l, s0c, skip, dgc, xc, dc, e0);
                } else {
                    if (dout)
                        launch(mg, k_restrict<T, KT, false, 2>, gc, s, C.n, L.n, L.K, L.col, P<T>::r(L), P<T>::b(C),
                               (const T *)nullptr, (const T *)nullptr, skip, dgc, xc, dc, e0);
                    else
                        launch(mg, k_restrict<T, KT, false, 1>, gc, s, C.n, L.n, L.K, L.col, P<T>::r(L), P<T>::b(C),
                               (const T *)nullptr, (const T *)nullptr, skip, dgc, xc, dc, e0);
                }
                coarse_pre0 = true;
            } else if (o.restriction == DEC_RESTRICT_STAR0)
                launch(mg, k_restrict<T, KT, true>, gc, s, C.n, L.n, L.K, L.col, P<T>::r(L), P<T>::b(C),
                       P<T>::s0(L), P<T>::s0(C), skip, (const T *)nullptr, (T *)nullptr, (T *)nullptr, T(0));
            else
                launch(mg, k_restrict<T, KT, false>, gc, s, C.n, L.n, L.K, L.col, P<T>::r(L), P<T>::b(C),
                       (const T *)nullptr, (const T *)nullptr, skip, (const T *)nullptr, (T *)nullptr, (T *)nullptr,
                       T(0));
        }
    });
    T *ec = cycle<T>(mg, l - 1, P<T>::b(C), s, skip, coarse_pre0, nullptr, kind);
    const int reps = kind == kCycF ? 2 : (kind == kCycGamma ? o.gamma : 1);
    if (reps > 1 && l - 1 > 0) {
        // W- or F-cycle: repeat the coarse correction, ec <- ec + C(b_c - L_c ec), gamma
        // times with the same cycle (W) or once with a V-cycle (F); not on the
        // coarsest level, whose dense solve is exact
        const int gc = grid_for(mg, C.n);
        const T *wc = P<T>::w(C);
        for (int rep = 1; rep < reps; ++rep) {
            launch(mg, k_copy<T>, gc, s, C.n, (const T *)ec, P<T>::y(C), skip);
            dispatch_k(C.K, [&](auto kt) {
                constexpr int KT = decltype(kt)::value;
                ProfScope ps(mg, DEC_PK_RESIDUAL, l - 1, s);
                launch(mg, k_residual<T, KT>, gc, s, C.n, C.K, (const int32_t *)C.col, wc, (const T *)P<T>::b(C),
                       (const T *)P<T>::y(C), P<T>::c(C), skip);
            });
            T *e2 = cycle<T>(mg, l - 1, P<T>::c(C), s, skip, false, nullptr, kind == kCycF ? kCycV : kind);
            launch(mg, k_axpy1<T>, gc, s, C.n, (const T *)e2, P<T>::y(C), skip);
            ec = P<T>::y(C);
        }
    }
    if (fuse_here(o, DEC_FUSE_PROLONG, L.n) && o.nu2 > 0 && o.smoother != DEC_SMOOTH_MCGS && !mapped) {
        const bool cheb = o.smoother == DEC_SMOOTH_CHEBYSHEV;
        const T e0 = (T)(cheb ? L.e_post[0] : o.omega);
        const bool dout = cheb && 1 < o.nu2;
        const int nxt = 1 - cur;
        T *xo = P<T>::x(L, nxt), *dn = dout ? P<T>::d(L, nxt) : nullptr;
        const T *xi = P<T>::x(L, cur), *dg = P<T>::dg(L);
        dispatch_k(L.K, [&](auto kt) {
            constexpr int KT = decltype(kt)::value;
            ProfScope ps(mg, DEC_PK_PROLSMOOTH, l, s);
            if (dout)
                launch(mg, k_prolong_smooth<T, KT, true>, g, s, L.n, L.K, C.n, (const int2 *)L.par, (const T *)ec,
                       (const int32_t *)L.col, w, dg, b, xi, xo, dn, e0, skip);
            else
                launch(mg, k_prolong_smooth<T, KT, false>, g, s, L.n, L.K, C.n, (const int2 *)L.par, (const T *)ec,
                       (const int32_t *)L.col, w, dg, b, xi, xo, dn, e0, skip);
        });
        cur = nxt;
        smooth<T>(mg, l, b, o.nu2, false, true, cur, s, skip, 1, da);
        return P<T>::x(L, cur);
    }
    {
        ProfScope ps(mg, DEC_PK_PROLONG, l, s);
        if (mapped)
            launch(mg, k_prolong_map<T>, g, s, L.n, (const int32_t *)L.gidx, P<T>::gw(L), (const T *)ec,
                   P<T>::x(L, cur), skip);
        else
            launch(mg, k_prolong<T>, g, s, C.n, L.n, L.par, ec, P<T>::x(L, cur), skip);
    }
    if (o.nu2 > 0) smooth<T>(mg, l, b, o.nu2, false, true, cur, s, skip, 0, da);
    return P<T>::x(L, cur);
}

// ---------------------------------------------------------------------------
// outer iterations
// ---------------------------------------------------------------------------

// x0: the iterate is zero (a cold start), so r = b without the operator apply.
template <typename TV>
void enqueue_outer_init(dec_mg *mg, TV *rv, cudaStream_t s, bool x0) {
    DevLevel &F = mg->lv.back();
    ProfScope ps(mg, DEC_PK_AUX, (int)mg->lv.size() - 1, s);
    dispatch_k(F.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        if (x0)
            launch(mg, k_outer_init<KT, TV, true>, red_grid64(mg, F.n), s, F.n, F.K, F.col, F.w64, F.freev, mg->ob,
                   mg->ox, mg->orr, rv, mg->partials, mg->counter, mg->scal);
        else
            launch(mg, k_outer_init<KT, TV, false>, red_grid64(mg, F.n), s, F.n, F.K, F.col, F.w64, F.freev, mg->ob,
                   mg->ox, mg->orr, rv, mg->partials, mg->counter, mg->scal);
    });
}

void enqueue_mean_shift(dec_mg *mg, double *v, cudaStream_t s, const int *skip) {
    DevLevel &F = mg->lv.back();
    const int top = (int)mg->lv.size() - 1;
    ProfScope p1(mg, DEC_PK_AUX, top, s), p2(mg, DEC_PK_AUX, top, s);
    launch(mg, k_mean, red_grid64(mg, F.n), s, F.n, F.star0, F.freev, v, mg->partials, mg->counter, mg->scal, skip);
    launch(mg, k_shift, grid_for(mg, F.n), s, F.n, F.freev, v, mg->scal, skip);
}

// z <- M r, then the dot products and the new search direction.
// first_pre0: the first iteration's finest first smoothing step already ran
// (k_init_ff), as the fused ff update provides it on later iterations.
void enqueue_precondition(dec_mg *mg, int solver, int mode, bool first, cudaStream_t s, const int *skip,
                          bool first_pre0 = false) {
    DevLevel &F = mg->lv.back();
    const int gauge = mg->H.bc == DEC_BC_GAUGE;
    const int rg = red_grid(mg, F.n), rg64 = red_grid64(mg, F.n);
    const int top = (int)mg->lv.size() - 1;
    if (solver == DEC_SOLVER_CG) {
        ProfScope ps(mg, DEC_PK_ZDOTS, top, s);
        launch(mg, k_pcg_zdots<double>, rg64, s, F.n, F.star0, F.freev, mg->orr, mg->ozn, mg->orr, mg->ozo, first,
                                                    gauge, mg->partials, mg->counter, mg->scal, skip);
    } else if (mode != DEC_MODE_F64) {
        // z is the FP32 cycle output.  DEC_MODE_MIXED: FP64 dot products with
        // the FP64 residual and FP64 search directions; DEC_MODE_MIXED_F32DOT:
        // FP32 dot products with r32, FP64 directions; DEC_MODE_MIXED_FF: FP32
        // dot products and FP32 directions (float-float outer iteration)
        const dec_mg_opts &o = mg->H.opts;
        const bool outer = (o.fuse & DEC_FUSE_OUTER) != 0;
        const bool d64 = mode == DEC_MODE_MIXED;
        DotsArgs da;
        da.first = first ? 1 : 0;
        da.gauge = gauge;
        da.d64 = d64;
        // after an outer update with the fused first smoothing step, the cycle starts at step 1
        const bool pre0 = (outer && !first && (mode == DEC_MODE_MIXED_FF || mode == DEC_MODE_MIXED) && o.nu1 > 0 &&
                           o.smoother != DEC_SMOOTH_MCGS) ||
                          (first && first_pre0);
        float *z = cycle<float>(mg, top, F.b32, s, skip, pre0, outer ? &da : nullptr);
        if (!da.done) {
            ProfScope ps(mg, DEC_PK_ZDOTS, top, s);
            if (d64)
                launch(mg, k_pcg_zdots_d, rg64, s, F.n, (const double *)F.star0, (const uint8_t *)F.freev,
                       (const float *)z, (const double *)mg->orr, (const double *)mg->ozo, first ? 1 : 0, gauge,
                       mg->partials, mg->counter, mg->scal, skip);
            else
                launch(mg, k_pcg_zdots_m, rg, s, F.n, (const float *)F.star0_32, (const uint8_t *)F.freev,
                       (const float *)z, (const float *)F.b32, (const float *)mg->zo32, first ? 1 : 0, gauge,
                       mg->partials, mg->counter, mg->scal, skip);
        }
        ProfScope ps(mg, DEC_PK_PUPD, top, s);
        if (mode == DEC_MODE_MIXED_FF)
            launch(mg, k_pcg_pupd_f, grid_for(mg, F.n), s, F.n, (const uint8_t *)F.freev, (const float *)z, mg->zo32,
                   mg->fp, first ? 1 : 0, (const Scal *)mg->scal, skip);
        else if (d64)
            launch(mg, k_pcg_pupd_d, grid_for(mg, F.n), s, F.n, (const uint8_t *)F.freev, (const float *)z, mg->ozo,
                   mg->op, first ? 1 : 0, (const Scal *)mg->scal, skip);
        else
            launch(mg, k_pcg_pupd_m, grid_for(mg, F.n), s, F.n, (const uint8_t *)F.freev, (const float *)z, mg->zo32,
                   mg->op, first ? 1 : 0, (const Scal *)mg->scal, skip);
        return;
    } else {
        double *z = cycle<double>(mg, top, mg->orr, s, skip);
        ProfScope ps(mg, DEC_PK_ZDOTS, top, s);
        launch(mg, k_pcg_zdots<double>, rg64, s, F.n, F.star0, F.freev, z, mg->ozn, mg->orr, mg->ozo, first, gauge,
                                                    mg->partials, mg->counter, mg->scal, skip);
    }
    ProfScope ps(mg, DEC_PK_PUPD, top, s);
    launch(mg, k_pcg_pupd, grid_for(mg, F.n), s, F.n, F.freev, mg->ozn, mg->ozo, mg->op, first ? 1 : 0, mg->scal,
                                                      skip);
}

void enqueue_pcg_iteration(dec_mg *mg, int solver, int mode, cudaStream_t s) {
    DevLevel &F = mg->lv.back();
    const int *skip = &mg->scal->done;
    const int rg = red_grid(mg, F.n), rg64 = red_grid64(mg, F.n);
    const int top = (int)mg->lv.size() - 1;
    if (mode == DEC_MODE_MIXED_FF && solver != DEC_SOLVER_CG) {
        dispatch_k(F.K, [&](auto kt) {
            constexpr int KT = decltype(kt)::value;
            ProfScope ps(mg, DEC_PK_SPMV64, top, s);
            launch(mg, k_pcg_spmv_ff<KT>, rg, s, F.n, F.K, (const int32_t *)F.col, (const float *)F.w32,
                   (const float *)F.wlo, (const float *)F.star0_32, (const float *)mg->fp, mg->fqh, mg->fql,
                   mg->partials, mg->counter, mg->scal, skip);
        });
        {
            ProfScope ps(mg, DEC_PK_UPDATE, top, s);
            const dec_mg_opts &o = mg->H.opts;
            int s0mode = 0;
            float e0 = 0.f;
            if ((o.fuse & DEC_FUSE_OUTER) && o.nu1 > 0 && o.smoother != DEC_SMOOTH_MCGS) {
                const bool cheb = o.smoother == DEC_SMOOTH_CHEBYSHEV;
                s0mode = cheb && 1 < o.nu1 ? 2 : 1;
                e0 = (float)(cheb ? F.e_pre[0] : o.omega);
            }
            launch(mg, k_pcg_update_ff, rg, s, F.n, (const float *)mg->fp, (const float *)mg->fqh,
                   (const float *)mg->fql, mg->fxh, mg->fxl, F.b32, mg->frl, mg->partials, mg->counter, mg->scal,
                   skip, s0mode, (const float *)F.dg32, F.x32[0], F.d32[0], e0);
        }
        enqueue_precondition(mg, solver, mode, false, s, skip);
        return;
    }
    dispatch_k(F.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        ProfScope ps(mg, DEC_PK_SPMV64, top, s);
        launch(mg, k_pcg_spmv_d<KT>, rg64, s, F.n, F.K, (const int32_t *)F.col, (const double *)F.w64,
               (const double *)F.star0, (const double *)mg->op, mg->oq, mg->partials, mg->counter, mg->scal, skip);
    });
    {
    ProfScope ps(mg, DEC_PK_UPDATE, top, s);
    if (mode == DEC_MODE_MIXED && solver != DEC_SOLVER_CG) {
        const dec_mg_opts &o = mg->H.opts;
        int s0mode = 0;
        float e0 = 0.f;
        if ((o.fuse & DEC_FUSE_OUTER) && o.nu1 > 0 && o.smoother != DEC_SMOOTH_MCGS) {
            const bool cheb = o.smoother == DEC_SMOOTH_CHEBYSHEV;
            s0mode = cheb && 1 < o.nu1 ? 2 : 1;
            e0 = (float)(cheb ? F.e_pre[0] : o.omega);
        }
        launch(mg, k_pcg_update_d, rg64, s, F.n, (const double *)mg->op, (const double *)mg->oq, mg->ox, mg->orr, F.b32,
               mg->partials, mg->counter, mg->scal, skip, s0mode, (const float *)F.dg32, F.x32[0], F.d32[0], e0);
    } else if (mode == DEC_MODE_MIXED_F32DOT && solver != DEC_SOLVER_CG)
        launch(mg, k_pcg_update_m, rg, s, F.n, (const double *)mg->op, (const double *)mg->oq, mg->ox, mg->orr, F.b32,
               mg->partials, mg->counter, mg->scal, skip);
    else
        launch(mg, k_pcg_update<double>, rg64, s, F.n, mg->op, mg->oq, mg->ox, mg->orr, nullptr, mg->partials,
                                                     mg->counter, mg->scal, skip);
    }
    enqueue_precondition(mg, solver, mode, false, s, skip);
}

void enqueue_mg_iteration(dec_mg *mg, int mode, cudaStream_t s) {
    DevLevel &F = mg->lv.back();
    const int *skip = &mg->scal->done;
    const int top = (int)mg->lv.size() - 1;
    const int rg = red_grid(mg, F.n), rg64 = red_grid64(mg, F.n);
    if (mode == DEC_MODE_MIXED_FF) {
        float *e = cycle<float>(mg, top, F.b32, s, skip);
        {
            ProfScope ps(mg, DEC_PK_ADD, top, s);
            launch(mg, k_add_ff, grid_for(mg, F.n), s, F.n, (const float *)e, mg->fxh, mg->fxl, skip);
        }
        dispatch_k(F.K, [&](auto kt) {
            constexpr int KT = decltype(kt)::value;
            ProfScope ps(mg, DEC_PK_MGRES, top, s);
            launch(mg, k_mg_residual_ff<KT>, rg, s, F.n, F.K, (const int32_t *)F.col, (const float *)F.w32,
                   (const float *)F.wlo, (const uint8_t *)F.freev, (const float *)mg->fbh, (const float *)mg->fbl,
                   (const float *)mg->fxh, (const float *)mg->fxl, F.b32, mg->frl, mg->partials, mg->counter,
                   mg->scal, skip);
        });
    } else if (mode == DEC_MODE_MIXED || mode == DEC_MODE_MIXED_F32DOT) {
        float *e = cycle<float>(mg, top, F.b32, s, skip);
        {
            ProfScope ps(mg, DEC_PK_ADD, top, s);
            launch(mg, k_add<float>, grid_for(mg, F.n), s, F.n, e, mg->ox, skip);
        }
        dispatch_k(F.K, [&](auto kt) {
            constexpr int KT = decltype(kt)::value;
            ProfScope ps(mg, DEC_PK_MGRES, top, s);
            if (mode == DEC_MODE_MIXED)
                launch(mg, k_mg_residual_d<KT>, rg64, s, F.n, F.K, (const int32_t *)F.col, (const double *)F.w64,
                       (const uint8_t *)F.freev, (const double *)mg->ob, (const double *)mg->ox, mg->orr, F.b32,
                       mg->partials, mg->counter, mg->scal, skip);
            else
                launch(mg, k_mg_residual_m<KT>, rg, s, F.n, F.K, (const int32_t *)F.col, (const double *)F.w64,
                       (const uint8_t *)F.freev, (const double *)mg->ob,
                       (const double *)mg->ox, mg->orr, F.b32, mg->partials, mg->counter, mg->scal, skip);
        });
    } else {
        double *e = cycle<double>(mg, top, mg->orr, s, skip);
        {
            ProfScope ps(mg, DEC_PK_ADD, top, s);
            launch(mg, k_add<double>, grid_for(mg, F.n), s, F.n, e, mg->ox, skip);
        }
        dispatch_k(F.K, [&](auto kt) {
            constexpr int KT = decltype(kt)::value;
            ProfScope ps(mg, DEC_PK_MGRES, top, s);
            launch(mg, k_mg_residual<KT, double>, rg64, s, F.n, F.K, F.col, F.w64, F.freev, mg->ob, mg->ox, mg->orr,
                                                              (double *)nullptr, mg->partials, mg->counter, mg->scal,
                                                              skip);
        });
    }
}

// One iteration of the chosen solver, as a CUDA graph captured on first use.
int iteration_graph(dec_mg *mg, int solver, int mode, cudaGraphExec_t *out) {
    cudaGraphExec_t &slot = mg->graphs[solver][mode];
    if (!slot && mg->prof) {
        // profiled graphs own the event slots: keep one profiled graph at a time
        drop_graphs(mg);
    }
    if (!slot) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(mg->cap, cudaStreamCaptureModeThreadLocal));
        mg->prof_capture = mg->prof != 0;
        mg->capturing = true;
        if (solver == DEC_SOLVER_MG)
            enqueue_mg_iteration(mg, mode, mg->cap);
        else
            enqueue_pcg_iteration(mg, solver, mode, mg->cap);
        mg->prof_capture = false;
        mg->capturing = false;
        cudaError_t e1 = cudaGetLastError();
        cudaError_t e2 = cudaStreamEndCapture(mg->cap, &g);
        if (e1 != cudaSuccess) return cuda_fail(e1, "capture");
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(g, nodes.data(), &nn);
        int64_t nk = 0;
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++nk;
        }
        mg->graph_kernels[solver][mode] = nk;
        cudaError_t e3 = cudaGraphInstantiate(&slot, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) {
            slot = nullptr;
            return cuda_fail(e3, "cudaGraphInstantiate");
        }
    }
    *out = slot;
    return DEC_OK;
}

// The whole iteration loop as one graph: while (!done && loops < max_loops) { iteration }.
int loop_graph(dec_mg *mg, int solver, int mode, cudaGraphExec_t *out) {
    cudaGraphExec_t &slot = mg->loops[solver][mode];
    if (slot) {
        *out = slot;
        return DEC_OK;
    }
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle hnd;
    cudaError_t e = cudaGraphConditionalHandleCreate(&hnd, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNode_t node;
    cudaGraphNodeParams np = {};
    if (e == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = hnd;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    }
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        (void)cudaGetLastError();
        mg->no_device_loop = true;
        return DEC_ERR_CUDA;
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(mg->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        mg->capturing = true;
        if (solver == DEC_SOLVER_MG)
            enqueue_mg_iteration(mg, mode, mg->cap);
        else
            enqueue_pcg_iteration(mg, solver, mode, mg->cap);
        launch(mg, k_loop_ctrl, 1, mg->cap, hnd, mg->scal);
        mg->capturing = false;
        cudaError_t e1 = cudaGetLastError();
        e = cudaStreamEndCapture(mg->cap, &body);
        if (e == cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) {
        size_t nn = 0;
        cudaGraphGetNodes(body, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(body, nodes.data(), &nn);
        int64_t nk = 0;
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++nk;
        }
        mg->loop_kernels[solver][mode] = nk;
        e = cudaGraphInstantiate(&slot, g, 0);
    }
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        slot = nullptr;
        (void)cudaGetLastError();
        mg->no_device_loop = true;
        return DEC_ERR_CUDA;
    }
    *out = slot;
    return DEC_OK;
}

// b_host / x_host: b and x are host arrays (pinned or pageable): b is copied
// straight into the solver's right-hand side and the result out of its
// iterate, so no device copy of either is made.
int solve_impl(dec_mg *mg, const double *b, double *x, const dec_solve_opts *po, dec_stats *stats,
               cudaStream_t s, bool b_host = false, bool x_host = false) {
    dec_solve_opts o;
    if (po)
        o = *po;
    else
        dec_solve_default_opts(&o);
    if (o.solver < 0 || o.solver > 2 || o.mode < DEC_MODE_F64 || o.mode > DEC_MODE_MIXED_F32DOT || o.maxit < 0 ||
        o.maxit >= kHist || !(o.tol >= 0.0))
        return fail(Status::fail(DEC_ERR_ARG, "bad solve options"));
    if (o.check_every < 1) o.check_every = 1;
    DevLevel &F = mg->lv.back();
    const size_t vb = sizeof(double) * F.n;
    const bool gauge = mg->H.bc == DEC_BC_GAUGE;
    // plain CG runs in FP64 whatever the mode
    if (o.solver == DEC_SOLVER_CG) o.mode = DEC_MODE_F64;
    const bool mixed = o.mode != DEC_MODE_F64;
    const bool ff = o.mode == DEC_MODE_MIXED_FF;
    const int64_t launches0 = mg->launches;
    int64_t graph_launches = 0;
    // A cold float-float solve (x = 0, so r = b) starts in two kernels: the
    // gauge mean and the ff scale from one pass over b, then the shifted b as
    // ff pairs with x = 0 and the first cycle's first smoothing step.
    const bool cold_ff = ff && !o.warm_start;
    // A cold MG-PCG solve with an FP64 outer iteration starts the same way: the
    // gauge mean from one pass over b, then r = b - mean, x = 0, ||r||^2 and the
    // first cycle's first smoothing step in one pass.
    const bool cold_d = (o.mode == DEC_MODE_MIXED || o.mode == DEC_MODE_MIXED_F32DOT) && !o.warm_start &&
                        o.solver == DEC_SOLVER_MGPCG;
    const dec_mg_opts &mo = mg->H.opts;
    int s0mode = 0;
    float e0 = 0.f;
    if ((cold_ff || cold_d) && o.solver == DEC_SOLVER_MGPCG && (mo.fuse & DEC_FUSE_OUTER) && mo.nu1 > 0 &&
        mo.smoother != DEC_SMOOTH_MCGS) {
        const bool cheb = mo.smoother == DEC_SMOOTH_CHEBYSHEV;
        s0mode = cheb && 1 < mo.nu1 ? 2 : 1;
        e0 = (float)(cheb ? F.e_pre[0] : mo.omega);
    }
    CK(cudaMemcpyAsync(mg->ob, b, vb, b_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    if (o.warm_start)
        CK(cudaMemcpyAsync(mg->ox, x, vb, x_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    else if (!cold_ff && !cold_d)
        CK(cudaMemsetAsync(mg->ox, 0, vb, s));
    // scalar header (everything before the history)
    Scal *h = mg->scal_h;
    std::memset(h, 0, offsetof(Scal, hist));
    h->tol = o.tol;
    h->maxit = o.maxit;
    h->max_loops = o.maxit + 1;
    h->star0_sum = mg->star0_sum;
    h->inv_star0_sum = mg->star0_sum > 0.0 ? 1.0 / mg->star0_sum : 0.0;
    CK(cudaMemcpyAsync(mg->scal, h, offsetof(Scal, hist), cudaMemcpyHostToDevice, s));
    if (cold_ff) {
        ProfScope p1(mg, DEC_PK_AUX, (int)mg->lv.size() - 1, s), p2(mg, DEC_PK_AUX, (int)mg->lv.size() - 1, s);
        const bool mg_solver = o.solver == DEC_SOLVER_MG;
        const int rg = red_grid(mg, F.n);
        launch(mg, k_b_stats, red_grid64(mg, F.n), s, F.n, (const double *)F.star0, (const uint8_t *)F.freev, (const double *)mg->ob,
               gauge ? 1 : 0, mg->partials, mg->counter, mg->scal);
        launch(mg, k_init_ff, rg, s, F.n, (const uint8_t *)F.freev, mg->ob, mg->fxh, mg->fxl, F.b32, mg->frl,
               mg_solver ? mg->fbh : nullptr, mg_solver ? mg->fbl : nullptr, s0mode, (const float *)F.dg32,
               F.x32[0], F.d32[0], e0, mg->partials, mg->counter, mg->scal);
    } else if (cold_d) {
        ProfScope p1(mg, DEC_PK_AUX, (int)mg->lv.size() - 1, s), p2(mg, DEC_PK_AUX, (int)mg->lv.size() - 1, s);
        const int rg64 = red_grid64(mg, F.n);
        launch(mg, k_b_stats, rg64, s, F.n, (const double *)F.star0, (const uint8_t *)F.freev, (const double *)mg->ob,
               gauge ? 1 : 0, mg->partials, mg->counter, mg->scal);
        launch(mg, k_init_d, rg64, s, F.n, (const uint8_t *)F.freev, mg->ob, mg->ox, mg->orr, F.b32, s0mode,
               (const float *)F.dg32, F.x32[0], F.d32[0], e0, mg->partials, mg->counter, mg->scal);
    } else {
    if (gauge) {
        enqueue_mean_shift(mg, mg->ob, s, nullptr);
        if (o.warm_start) enqueue_mean_shift(mg, mg->ox, s, nullptr);
    }
    if (mixed)
        enqueue_outer_init<float>(mg, F.b32, s, !o.warm_start);
    else
        enqueue_outer_init<double>(mg, (double *)nullptr, s, !o.warm_start);
    }
    if (ff && !cold_ff) {
        ProfScope ps(mg, DEC_PK_AUX, (int)mg->lv.size() - 1, s);
        const bool mg_solver = o.solver == DEC_SOLVER_MG;
        launch(mg, k_ff_split, grid_for(mg, F.n), s, F.n, o.warm_start ? (const double *)mg->ox : nullptr,
               (const double *)mg->orr, (const double *)mg->ob, mg->fxh, mg->fxl, F.b32, mg->frl,
               mg_solver ? mg->fbh : nullptr, mg_solver ? mg->fbl : nullptr, (const Scal *)mg->scal);
    }
    CK(cudaGetLastError());
    int rc = DEC_OK;
    // Default: the iteration loop runs on the device (one graph with a while
    // node) and the host waits once at the end.  With live profiling, or if
    // conditional nodes are unavailable, the host relaunches one iteration at
    // a time and reads the residual in between.
    cudaGraphExec_t lg = nullptr;
    if (!mg->prof && !mg->no_device_loop && !o.host_loop && o.maxit > 0) {
        if (loop_graph(mg, o.solver, o.mode, &lg) != DEC_OK) lg = nullptr;
    }
    int64_t loop_runs = 0;
    if (lg) {
        if (o.solver != DEC_SOLVER_MG)
            enqueue_precondition(mg, o.solver, o.mode, true, s, &mg->scal->done, s0mode > 0);
        CK(cudaGraphLaunch(lg, s));
        loop_runs = 1;
    } else {
    CK(cudaMemcpyAsync(h, mg->scal, offsetof(Scal, hist), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!h->done && o.maxit > 0) {
        if (o.solver != DEC_SOLVER_MG) enqueue_precondition(mg, o.solver, o.mode, true, s, nullptr, s0mode > 0);
        cudaGraphExec_t ge;
        rc = iteration_graph(mg, o.solver, o.mode, &ge);
        if (rc) return rc;
        int launched = 0;
        const int every = mg->prof ? 1 : o.check_every;
        while (launched < o.maxit) {
            int chunk = std::min(every, o.maxit - launched);
            for (int k = 0; k < chunk; ++k) CK(cudaGraphLaunch(ge, s));
            graph_launches += chunk;
            launched += chunk;
            CK(cudaMemcpyAsync(h, mg->scal, offsetof(Scal, hist), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (h->done) break;
            if (mg->prof) accumulate_slots(mg);
        }
    }
    }
    if (ff) {
        // x = (hi + lo) / scale straight into the caller's x (and ox); with the
        // gauge, the mean of x comes out of the same pass
        const int top = (int)mg->lv.size() - 1;
        if (gauge) {
            ProfScope p1(mg, DEC_PK_AUX, top, s), p2(mg, DEC_PK_AUX, top, s);
            launch(mg, k_ff_join_mean, red_grid64(mg, F.n), s, F.n, (const float *)mg->fxh, (const float *)mg->fxl,
                   mg->ox, (const double *)F.star0, (const uint8_t *)F.freev, mg->partials, mg->counter, mg->scal);
            launch(mg, k_shift_out, grid_for(mg, F.n), s, F.n, (const uint8_t *)F.freev, mg->ox,
                   x_host ? nullptr : x, (const Scal *)mg->scal);
        } else {
            ProfScope p1(mg, DEC_PK_AUX, top, s);
            launch(mg, k_ff_join, grid_for(mg, F.n), s, F.n, (const float *)mg->fxh, (const float *)mg->fxl, mg->ox,
                   x_host ? nullptr : x, (const Scal *)mg->scal);
        }
    } else if (gauge) {
        // the mean shift writes the caller's x as it goes
        const int top = (int)mg->lv.size() - 1;
        ProfScope p1(mg, DEC_PK_AUX, top, s), p2(mg, DEC_PK_AUX, top, s);
        launch(mg, k_mean, red_grid64(mg, F.n), s, F.n, F.star0, F.freev, (const double *)mg->ox, mg->partials,
               mg->counter, mg->scal, (const int *)nullptr);
        launch(mg, k_shift_out, grid_for(mg, F.n), s, F.n, (const uint8_t *)F.freev, mg->ox,
               x_host ? nullptr : x, (const Scal *)mg->scal);
    } else if (!x_host) {
        CK(cudaMemcpyAsync(x, mg->ox, vb, cudaMemcpyDeviceToDevice, s));
    }
    if (x_host) CK(cudaMemcpyAsync(x, mg->ox, vb, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h, mg->scal, offsetof(Scal, hist), cudaMemcpyDeviceToHost, s));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    // relative residuals from the squared norms the device recorded; converged
    // means the device's own test ||r||^2 <= tol^2 ||b||^2 held
    auto rel_of = [&](double rn2) {
        if (!std::isfinite(rn2) || !std::isfinite(h->bnorm2)) return (double)NAN;
        return h->bnorm2 > 0.0 ? std::sqrt(rn2 / h->bnorm2) : 0.0;
    };
    const bool converged = std::isfinite(h->bnorm2) && h->rnorm2 <= h->thr2;
    if (stats) {
        stats->iters = h->iter;
        stats->rel_res = rel_of(h->rnorm2);
        stats->rel_res0 = rel_of(h->rnorm2_0);
        stats->launches = (mg->launches - launches0) + graph_launches * mg->graph_kernels[o.solver][o.mode] +
                          (loop_runs ? (int64_t)h->loops * mg->loop_kernels[o.solver][o.mode] : 0);
    }
    if (h->status == 3)
        return fail(Status::fail(DEC_ERR_CUDA, "a device-side wait gave up (shared-memory coarse cycle load)"));
    if (h->status == 1) {
        char buf[160];
        snprintf(buf, sizeof(buf), "non-finite residual at iteration %d (||b||^2 = %.3e, last rel = %.3e, rz = %.3e)",
                 h->iter, h->bnorm2, rel_of(h->rnorm2), h->rz);
        return fail(Status::fail(DEC_ERR_NONFINITE, buf));
    }
    if (!converged)
        return fail(Status::fail(DEC_ERR_NOT_CONVERGED, h->status == 2 ? "iteration stalled (<r,z> or <p,Lp> is zero "
                                                                         "in working precision) before tol"
                                                                       : "maxit reached before tol"));
    return rc;
}

int check_mg(const dec_mg *mg) {
    if (!mg) return fail(Status::fail(DEC_ERR_ARG, "null handle"));
    return DEC_OK;
}

// A compute call needs a device handle whose device is the current one: its
// tables, its work vectors and the caller's vectors all live there.
int check_dev(const dec_mg *mg) {
    if (!mg) return fail(Status::fail(DEC_ERR_ARG, "null handle"));
    if (mg->host_only) return fail(Status::fail(DEC_ERR_ARG, "handle was built with DEC_HOST_ONLY"));
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != mg->device)
        return fail(Status::fail(DEC_ERR_ARG, "the hierarchy lives on device " + std::to_string(mg->device) +
                                                  " but device " + std::to_string(cur) + " is current"));
    return DEC_OK;
}

// Row sums of the level weights (FP32 and FP64), on `s` (0: legacy stream).
void update_diagonals(dec_mg *mg, DevLevel &D, cudaStream_t s) {
    const int g = grid_for(mg, D.n);
    dispatch_k(D.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        launch(mg, k_diag<float, KT>, g, s, D.n, D.K, (const float *)D.w32, D.dg32);
        launch(mg, k_diag<double, KT>, g, s, D.n, D.K, (const double *)D.w64, D.dg64);
    });
}

// Device tables of the general map from level l-1 to level l: the 3 slots per
// fine vertex (slot-major) and the restriction rows of level l-1 -- the
// transpose of the row-normalized map, or its *0-adjoint -- in FP64 and FP32.
int upload_map(dec_mg *mg, int l, DevLevel &D) {
    const decimpl::HostHierarchy &H = mg->H;
    const std::vector<int32_t> &mi = H.map_idx[l - 1];
    const std::vector<double> &mw = H.map_w[l - 1];
    const int nf = D.n, nc = (int)H.levels[l - 1].mesh.nv;
    std::vector<int32_t> gi(3 * (size_t)nf);
    std::vector<double> gw(3 * (size_t)nf);
    // interpolation x_f += free_f * M(f)^T e_c: a fixed (Dirichlet) fine vertex gets no
    // correction, whatever coarse vertices its image lies between
    const std::vector<uint8_t> &ff = H.levels[l].free_;
    for (int v = 0; v < nf; ++v)
        for (int q = 0; q < 3; ++q) {
            gi[(size_t)q * nf + v] = mi[3 * (size_t)v + q];
            gw[(size_t)q * nf + v] = ff[v] ? mw[3 * (size_t)v + q] : 0.0;
        }
    // restriction rows: every (fine v, weight) whose map slot points at coarse c, in increasing v
    std::vector<int> cnt(nc + 1, 0);
    for (int v = 0; v < nf; ++v)
        for (int q = 0; q < 3; ++q)
            if (mw[3 * (size_t)v + q] != 0.0) cnt[mi[3 * (size_t)v + q] + 1] += 1;
    int Kr = 1;
    for (int c = 0; c < nc; ++c) Kr = std::max(Kr, cnt[c + 1]);
    for (int c = 0; c < nc; ++c) cnt[c + 1] += cnt[c];
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    std::vector<int32_t> ent_v(cnt[nc]);
    std::vector<double> ent_w(cnt[nc]);
    for (int v = 0; v < nf; ++v)
        for (int q = 0; q < 3; ++q) {
            const double w = mw[3 * (size_t)v + q];
            if (w == 0.0) continue;
            const int c = mi[3 * (size_t)v + q];
            ent_v[fill[c]] = v;
            ent_w[fill[c]++] = w;
        }
    const bool star0 = H.opts.restriction == DEC_RESTRICT_STAR0;
    const std::vector<double> &s0f = H.levels[l].star0, &s0c = H.levels[l - 1].star0;
    std::vector<int32_t> ri((size_t)Kr * nc, 0);
    std::vector<double> rw((size_t)Kr * nc, 0.0);
    for (int c = 0; c < nc; ++c) {
        double rs = 0.0;
        for (int k = cnt[c]; k < cnt[c + 1]; ++k) rs += ent_w[k];
        for (int k = cnt[c], q = 0; k < cnt[c + 1]; ++k, ++q) {
            ri[(size_t)q * nc + c] = ent_v[k];
            rw[(size_t)q * nc + c] = star0 ? s0f[ent_v[k]] * ent_w[k] / s0c[c] : ent_w[k] / rs;
        }
        for (int q = cnt[c + 1] - cnt[c]; q < Kr; ++q) ri[(size_t)q * nc + c] = cnt[c + 1] > cnt[c] ? ent_v[cnt[c]] : 0;
    }
    std::vector<float> gw32(gw.begin(), gw.end()), rw32(rw.begin(), rw.end());
    int rc;
    if ((rc = upload(mg, &D.gidx, gi.data(), gi.size())) || (rc = upload(mg, &D.gw64, gw.data(), gw.size())) ||
        (rc = upload(mg, &D.gw32, gw32.data(), gw32.size())) || (rc = upload(mg, &D.ridx, ri.data(), ri.size())) ||
        (rc = upload(mg, &D.rw64, rw.data(), rw.size())) || (rc = upload(mg, &D.rw32, rw32.data(), rw32.size())))
        return rc;
    D.gKr = Kr;
    return DEC_OK;
}

// Choose the levels 0..top of the shared-memory coarse cycle (the most that
// fit in one block's shared memory, at least levels 0 and 1), lay out their
// arrays and upload int16 copies of their column and parent tables.
int setup_coarse_cycle(dec_mg *mg) {
    using namespace decdev;
    mg->coarse_top = -1;
    const dec_mg_opts &o = mg->H.opts;
    const int nl = (int)mg->lv.size();
    if (nl < 2 || o.gamma != 1 || o.fcycle || o.nu1 > kCoarseMaxNu || o.nu2 > kCoarseMaxNu ||
        o.smoother == DEC_SMOOTH_MCGS || mg->H.mapped)
        return DEC_OK;
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, mg->device);
    const bool cheb = o.smoother == DEC_SMOOTH_CHEBYSHEV, star0 = o.restriction == DEC_RESTRICT_STAR0;
    auto al = [](int64_t b) { return (b + 15) & ~(int64_t)15; };
    CoarseArgs A{};
    int64_t off = kCoarseHeader;
    int top = -1;
    int64_t top_bytes = 0;
    for (int l = 0; l < std::min(nl, kCoarseMaxLevels); ++l) {
        const DevLevel &D = mg->lv[l];
        const int max_rows = o.coarse_max_rows > 0 ? std::min(o.coarse_max_rows, kCoarseMaxN) : kCoarseMaxN;
        if (D.n > max_rows || D.K > kCoarseMaxK) break;
        CoarseLevel &L = A.lv[l];
        L = CoarseLevel{};
        L.n = D.n;
        L.K = D.K;
        L.o_col = L.o_w = L.o_dg = L.o_dir = L.o_r = L.o_s0 = L.o_par = -1;
        int64_t b = off;
        auto take = [&](int &o_, int64_t bytes) {
            o_ = (int)b;
            b += al(bytes);
        };
        take(L.o_x, 4 * (int64_t)D.n);
        take(L.o_b, 4 * (int64_t)D.n);
        if (star0) take(L.o_s0, 4 * (int64_t)D.n);
        if (l > 0) {
            take(L.o_col, 2 * (int64_t)D.K * D.n);
            take(L.o_w, 4 * (int64_t)D.K * D.n);
            take(L.o_dg, 4 * (int64_t)D.n);
            take(L.o_r, 4 * (int64_t)D.n);
            take(L.o_par, 4 * (int64_t)(D.n - mg->lv[l - 1].n));
            if (cheb) take(L.o_dir, 4 * (int64_t)D.n);
        }
        if (b > smem_max) break;
        off = b;
        if (l > 0) {
            top = l;
            top_bytes = off;
        }
    }
    if (top < 1) return DEC_OK;
    for (int l = 0; l <= top; ++l) {
        DevLevel &D = mg->lv[l];
        CoarseLevel &L = A.lv[l];
        L.s0 = D.star0_32;
        if (l > 0) {
            const decimpl::HostLevel &HL = mg->H.levels[l];
            std::vector<int16_t> c16(((size_t)D.K * D.n + 1) & ~(size_t)1, 0);  // even count: 4-byte loads
            for (size_t i = 0; i < (size_t)D.K * D.n; ++i) c16[i] = (int16_t)HL.col[i];
            const std::vector<int32_t> &par = mg->H.parents[l - 1];
            std::vector<int16_t> p16(par.begin(), par.end());
            int rc;
            if ((rc = upload(mg, &D.col16, c16.data(), c16.size())) || (rc = upload(mg, &D.par16, p16.data(), p16.size())))
                return rc;
            L.col = D.col16;
            L.par = D.par16;
            L.w = D.w32;
            L.dg = D.dg32;
        }
        for (int k = 0; k < kCoarseMaxNu; ++k) {
            L.e_pre[k] = (float)(cheb ? (k < (int)D.e_pre.size() ? D.e_pre[k] : 0.0) : o.omega);
            L.c_pre[k] = (float)(cheb ? (k < (int)D.c_pre.size() ? D.c_pre[k] : 0.0) : 0.0);
            L.e_post[k] = (float)(cheb ? (k < (int)D.e_post.size() ? D.e_post[k] : 0.0) : o.omega);
            L.c_post[k] = (float)(cheb ? (k < (int)D.c_post.size() ? D.c_post[k] : 0.0) : 0.0);
        }
    }
    A.top = top;
    A.nu1 = o.nu1;
    A.nu2 = o.nu2;
    A.cheb = cheb ? 1 : 0;
    A.star0 = star0 ? 1 : 0;
    A.G = mg->G32;
    A.S = mg->scal;
    A.top_mutable = top == nl - 1 ? 1 : 0;
    A.wait_rounds = kCoarseWaitRounds;
    // The dynamic shared-memory limit is a property of the kernel, shared by
    // every hierarchy on the device: raise it once to the device maximum
    // (each layout is at most that), never to one hierarchy's size.
    if (cudaFuncSetAttribute(k_coarse_cycle<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) != cudaSuccess ||
        cudaFuncSetAttribute(k_coarse_cycle<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) != cudaSuccess) {
        (void)cudaGetLastError();
        return DEC_OK;  // leave the shared-memory cycle off for this hierarchy
    }
    bool k6 = true;
    for (int l = 1; l <= top; ++l) k6 = k6 && mg->lv[l].K == 6;
    mg->coarse_k6 = k6;
    mg->coarse_args = A;
    mg->coarse_smem = (int)top_bytes;
    mg->coarse_top = top;
    return DEC_OK;
}

}  // namespace

namespace {

// Contiguous column buffers for calls with k > 1 interleaved right-hand
// sides, allocated on the first such call.
static_assert(decdev::kPatchDepth == decimpl::kPatchMaxDepth && decdev::kPatchHdrInts == decimpl::kPatchHdr,
              "tile header layout");

constexpr int kPatchChunk = 24;

int upload_tiles(dec_mg *mg, const decimpl::HostPatch &H, int threads, DevLevel::Tiles &T) {
    int rc;
    std::vector<float> w32(H.lw.size());
    for (size_t i = 0; i < w32.size(); ++i) w32[i] = (float)H.lw[i];
    if ((rc = upload(mg, &T.hdr, H.hdr.data(), H.hdr.size())) || (rc = upload(mg, &T.gid, H.gid.data(), H.gid.size())) ||
        (rc = upload(mg, &T.lcol, H.lcol.data(), H.lcol.size())) ||
        (rc = upload(mg, &T.lw64, H.lw.data(), H.lw.size())) || (rc = upload(mg, &T.lw32, w32.data(), w32.size())))
        return rc;
    T.ntiles = H.ntiles;
    T.depth = H.depth;
    T.threads = threads;
    T.smem32 = decdev::patch_smem_bytes<float>(H.cap);
    T.smem64 = decdev::patch_smem_bytes<double>(H.cap);
    return DEC_OK;
}

// Halo tiles (DEC_FUSE_PATCH) for the levels strictly between the coarsest and
// the finest, up to patch_max_rows rows: binary subdivision, V-cycles, Jacobi
// or Chebyshev with 1 to 3 steps per smoothing call.  A level whose largest
// FP64 tile would not fit in a block's shared memory keeps the per-step kernels.
int setup_patches(dec_mg *mg) {
    const dec_mg_opts &o = mg->H.opts;
    const int nl = (int)mg->lv.size();
    if (!(o.fuse & DEC_FUSE_PATCH) || mg->H.mapped || o.gamma != 1 || o.fcycle ||
        (o.smoother != DEC_SMOOTH_JACOBI && o.smoother != DEC_SMOOTH_CHEBYSHEV) || o.nu1 < 1 || o.nu2 < 1 ||
        o.nu1 > decimpl::kPatchMaxDepth || o.nu2 > decimpl::kPatchMaxDepth)
        return DEC_OK;
    int smem_optin = 0;
    CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, mg->device));
    int need32 = 0, need64 = 0;
    for (int l = 1; l + 1 < nl; ++l) {
        DevLevel &D = mg->lv[l];
        if (o.patch_max_rows > 0 && D.n > o.patch_max_rows) continue;
        const decimpl::HostMesh &HC = mg->H.levels[l - 1].mesh;
        // 24 coarse vertices per tile (about 180 locals with two rings): the fastest of 12 to 48
        // in whole solves on the icosphere benchmark (FP32 and FP64 cycles)
        const int chunk = o.patch_chunk > 0 ? o.patch_chunk : kPatchChunk;
        decimpl::HostPatch pd, pu;
        Status st = decimpl::build_patches(mg->H.levels[l], HC, mg->H.parents[l - 1], chunk, o.nu1, o.nu2, pd, pu);
        if (!st.good()) return fail(st);
        if ((int64_t)decdev::patch_smem_bytes<double>(1) * std::max(pd.cap, pu.cap) > smem_optin) continue;
        int rc;
        const int threads = o.patch_threads > 0 ? o.patch_threads : decdev::kPatchThreads;
        if ((rc = upload_tiles(mg, pd, threads, D.tdown)) || (rc = upload_tiles(mg, pu, threads, D.tup))) return rc;
        need32 = std::max({need32, D.tdown.smem32, D.tup.smem32});
        need64 = std::max({need64, D.tdown.smem64, D.tup.smem64});
    }
    // blocks above the default 48 KB of dynamic shared memory need the opt-in
    bool ok = true;
    if (need32 > 48 * 1024)
        ok = ok && cudaFuncSetAttribute(decdev::k_patch_down<float, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, need32) == cudaSuccess &&
             cudaFuncSetAttribute(decdev::k_patch_down<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, need32) == cudaSuccess &&
             cudaFuncSetAttribute(decdev::k_patch_up<float, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, need32) == cudaSuccess &&
             cudaFuncSetAttribute(decdev::k_patch_up<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, need32) == cudaSuccess;
    if (need64 > 48 * 1024)
        ok = ok && cudaFuncSetAttribute(decdev::k_patch_down<double, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, need64) == cudaSuccess &&
             cudaFuncSetAttribute(decdev::k_patch_down<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, need64) == cudaSuccess &&
             cudaFuncSetAttribute(decdev::k_patch_up<double, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, need64) == cudaSuccess &&
             cudaFuncSetAttribute(decdev::k_patch_up<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, need64) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        for (DevLevel &D : mg->lv) D.tdown.ntiles = D.tup.ntiles = 0;  // keep the per-step kernels
    }
    return DEC_OK;
}

int column_buffers(dec_mg *mg) {
    const int n = mg->lv.back().n;
    int rc;
    if (!mg->kx64 && (rc = dalloc(mg, &mg->kx64, n))) return rc;
    if (!mg->kb32 && (rc = dalloc(mg, &mg->kb32, n))) return rc;
    if (!mg->kx32 && (rc = dalloc(mg, &mg->kx32, n))) return rc;
    return DEC_OK;
}

// Options of a build: the defaults when opts is null, validated.
int build_opts(const dec_mg_opts *opts, dec_mg_opts &o) {
    if (opts)
        o = *opts;
    else
        dec_mg_default_opts(&o);
    if (o.smoother != DEC_SMOOTH_JACOBI && o.smoother != DEC_SMOOTH_CHEBYSHEV && o.smoother != DEC_SMOOTH_MCGS)
        return fail(Status::fail(DEC_ERR_ARG, "unknown smoother"));
    if (o.restriction != DEC_RESTRICT_ROWNORM && o.restriction != DEC_RESTRICT_STAR0)
        return fail(Status::fail(DEC_ERR_ARG, "unknown restriction"));
    if (o.fuse < 0 || o.fuse > DEC_FUSE_ALL) return fail(Status::fail(DEC_ERR_ARG, "fuse must be a DEC_FUSE_* mask"));
    if (o.fuse_max_rows < 0) return fail(Status::fail(DEC_ERR_ARG, "fuse_max_rows must be >= 0"));
    if (o.coarse_max_rows < 0) return fail(Status::fail(DEC_ERR_ARG, "coarse_max_rows must be >= 0"));
    if (o.patch_max_rows < 0 || o.patch_chunk < 0)
        return fail(Status::fail(DEC_ERR_ARG, "patch_max_rows and patch_chunk must be >= 0"));
    if (o.patch_threads < 0 || o.patch_threads % 32 != 0 || o.patch_threads > decdev::kPatchThreads)
        return fail(Status::fail(DEC_ERR_ARG, "patch_threads must be a multiple of 32 up to 256"));
    if (o.fcycle != 0 && o.fcycle != 1) return fail(Status::fail(DEC_ERR_ARG, "fcycle must be 0 or 1"));
    if (o.nu1 < 0 || o.nu2 < 0 || o.nu1 > 16 || o.nu2 > 16 || o.gamma < 1 || o.gamma > 4 || o.power_iters < 1 ||
        !(o.cheby_hi > o.cheby_lo) || !(o.cheby_lo > 0.0))
        return fail(Status::fail(DEC_ERR_ARG, "bad multigrid options"));
    return DEC_OK;
}

// Device part of a build: uploads every level's tables, allocates the work
// vectors and the outer-iteration workspace, sets up the shared-memory coarse
// cycle.  On failure the caller frees the handle.
int device_build(dec_mg *mg) {
    const dec_mg_opts &o = mg->H.opts;
    int rc = DEC_OK;
    cudaError_t ce = cudaGetDevice(&mg->device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    cudaDeviceGetAttribute(&mg->nsm, cudaDevAttrMultiProcessorCount, mg->device);
    ce = cudaStreamCreateWithFlags(&mg->cap, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamCreate");
    const int nl = (int)mg->H.levels.size();
    mg->lv.resize(nl);
    for (int l = 0; l < nl; ++l) {
        decimpl::HostLevel &HL = mg->H.levels[l];
        DevLevel &D = mg->lv[l];
        D.n = (int)HL.mesh.nv;
        D.K = HL.K;
        D.ne = HL.mesh.ne;
        D.nc = l > 0 ? (int)mg->H.levels[l - 1].mesh.nv : 0;
        const size_t slots = (size_t)HL.K * D.n;
        std::vector<float> w32(slots);
        for (size_t i = 0; i < slots; ++i) w32[i] = (float)HL.w[i];
        if ((rc = upload(mg, &D.col, HL.col.data(), slots))) return rc;
        if ((rc = upload(mg, &D.w64, HL.w.data(), slots))) return rc;
        if ((rc = upload(mg, &D.w32, w32.data(), slots))) return rc;
        if ((rc = upload(mg, &D.star0, HL.star0.data(), D.n))) return rc;
        {
            std::vector<float> s32(HL.star0.begin(), HL.star0.end());
            if ((rc = upload(mg, &D.star0_32, s32.data(), D.n))) return rc;
        }
        if ((rc = upload(mg, &D.freev, HL.free_.data(), D.n))) return rc;
        if (l > 0 && !mg->H.mapped) {
            const std::vector<int32_t> &par = mg->H.parents[l - 1];
            if ((rc = upload(mg, &D.par, reinterpret_cast<const int2 *>(par.data()), par.size() / 2))) return rc;
        }
        if (l > 0 && mg->H.mapped) {
            if ((rc = upload_map(mg, l, D))) return rc;
        }
        for (int i = 0; i < 2; ++i) {
            if ((rc = dalloc(mg, &D.x32[i], D.n)) || (rc = dalloc(mg, &D.d32[i], D.n)) ||
                (rc = dalloc(mg, &D.x64[i], D.n)) || (rc = dalloc(mg, &D.d64[i], D.n)))
                return rc;
        }
        if ((rc = dalloc(mg, &D.r32, D.n)) || (rc = dalloc(mg, &D.b32, D.n)) || (rc = dalloc(mg, &D.r64, D.n)) ||
            (rc = dalloc(mg, &D.b64, D.n)))
            return rc;
        if ((o.gamma > 1 || o.fcycle) && (((rc = dalloc(mg, &D.y32, D.n))) || (rc = dalloc(mg, &D.c32, D.n)) ||
                            (rc = dalloc(mg, &D.y64, D.n)) || (rc = dalloc(mg, &D.c64, D.n))))
            return rc;
        cheb_coeffs(HL.lmax, o.cheby_lo, o.cheby_hi, std::max(o.nu1, 1), D.c_pre, D.e_pre);
        cheb_coeffs(HL.lmax, o.cheby_lo, o.cheby_hi, std::max(o.nu2, 1), D.c_post, D.e_post);
        if ((rc = dalloc(mg, &D.dg32, D.n)) || (rc = dalloc(mg, &D.dg64, D.n))) return rc;
        update_diagonals(mg, D, nullptr);
        if (o.smoother == DEC_SMOOTH_MCGS) {
            // rows by colour, ascending row id within a colour (counting sort)
            D.coff.assign(HL.ncolors + 1, 0);
            for (int v = 0; v < D.n; ++v) D.coff[HL.colors[v] + 1] += 1;
            for (int c = 0; c < HL.ncolors; ++c) D.coff[c + 1] += D.coff[c];
            std::vector<int32_t> rows(D.n);
            std::vector<int> fill(D.coff.begin(), D.coff.end() - 1);
            for (int v = 0; v < D.n; ++v) rows[fill[HL.colors[v]]++] = v;
            if ((rc = upload(mg, &D.crow, rows.data(), rows.size()))) return rc;
        }
    }
    // coarsest dense operator
    {
        mg->n0 = mg->lv[0].n;
        const std::vector<double> &G = mg->H.G;
        std::vector<float> G32(G.size());
        for (size_t i = 0; i < G.size(); ++i) G32[i] = (float)G[i];
        if ((rc = upload(mg, &mg->G64, G.data(), G.size())) || (rc = upload(mg, &mg->G32, G32.data(), G32.size())))
            return rc;
    }
    // finest extras and outer workspace
    {
        decimpl::HostLevel &HF = mg->H.levels.back();
        const int n = (int)HF.mesh.nv;
        if ((rc = upload(mg, &mg->slot_edge, HF.slot_edge.data(), HF.slot_edge.size()))) return rc;
        if ((rc = upload(mg, &mg->edges, reinterpret_cast<const int2 *>(HF.mesh.edges.data()), (size_t)HF.mesh.ne)))
            return rc;
        mg->dim = HF.mesh.dim;
        if ((rc = upload(mg, &mg->verts, HF.mesh.verts.data(), HF.mesh.verts.size()))) return rc;
        if ((rc = dalloc(mg, &mg->pot, n)) || (rc = dalloc(mg, &mg->ptmp, n)) || (rc = dalloc(mg, &mg->prhs, n)))
            return rc;
        double **vecs[] = {&mg->ox, &mg->orr, &mg->op, &mg->oq, &mg->ozn, &mg->ozo, &mg->ob, &mg->tmp};
        for (double **v : vecs)
            if ((rc = dalloc(mg, v, n))) return rc;
        if ((rc = dalloc(mg, &mg->zo32, n))) return rc;
        float **fvecs[] = {&mg->fxh, &mg->fxl, &mg->frl, &mg->fqh, &mg->fql, &mg->fp, &mg->fbh, &mg->fbl};
        for (float **v : fvecs)
            if ((rc = dalloc(mg, v, n))) return rc;
        {
            DevLevel &DF = mg->lv.back();
            const size_t slots = (size_t)HF.K * n;
            std::vector<float> wlo(slots);
            for (size_t i = 0; i < slots; ++i) wlo[i] = (float)(HF.w[i] - (double)(float)HF.w[i]);
            if ((rc = upload(mg, &DF.wlo, wlo.data(), slots))) return rc;
        }

        if ((rc = dalloc(mg, &mg->partials, 8 * kMaxRedBlocks))) return rc;
        if ((rc = dalloc(mg, &mg->counter, 1))) return rc;
        if ((rc = dalloc(mg, &mg->scal, 1))) return rc;
        ce = cudaMemset(mg->scal, 0, sizeof(Scal));
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaMemset");
        ce = cudaMemset(mg->counter, 0, sizeof(unsigned));
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaMemset");
        ce = cudaMallocHost((void **)&mg->scal_h, sizeof(Scal));
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaMallocHost");
        double s = 0.0;
        for (int v = 0; v < n; ++v)
            if (HF.free_[v]) s += HF.star0[v];
        mg->star0_sum = s;
    }
    if ((rc = setup_coarse_cycle(mg))) return rc;
    if ((rc = setup_patches(mg))) return rc;
    ce = cudaDeviceSynchronize();
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaDeviceSynchronize");
    return DEC_OK;
}

}  // namespace

extern "C" {

int dec_mg_build(const dec_mesh *base, int nsub, int nlevels, int bc, uint32_t flags, const double *star1_scale,
                 const dec_mg_opts *opts, dec_mg **out) {
    if (!base || !out) return fail(Status::fail(DEC_ERR_ARG, "null pointer"));
    *out = nullptr;
    if (nsub < 0 || nsub > 14) return fail(Status::fail(DEC_ERR_ARG, "nsub out of range"));
    dec_mg_opts o;
    if (int rc = build_opts(opts, o)) return rc;
    dec_mg *mg = new (std::nothrow) dec_mg;
    if (!mg) return fail(Status::fail(DEC_ERR_OOM, "host allocation"));
    int rc = DEC_OK;
    auto bail = [&](int code) {
        free_all(mg);
        delete mg;
        return code;
    };
    try {
        if ((flags & DEC_SUBDIV_CUBIC) && (flags & DEC_ORDER_MORTON))
            return bail(fail(Status::fail(DEC_ERR_ARG, "cubic subdivision keeps the edge order")));
        Status st = decimpl::build_hierarchy(*dec_mesh_host(base), nsub, nlevels, bc, (flags & DEC_SPHERE_PROJECT) != 0,
                                             (flags & DEC_ORDER_MORTON) != 0, (flags & DEC_SUBDIV_CUBIC) != 0,
                                             star1_scale, o, mg->H);
        if (!st.good()) return bail(fail(st));
    } catch (const std::bad_alloc &) {
        return bail(fail(Status::fail(DEC_ERR_OOM, "host allocation")));
    }
    if (flags & DEC_HOST_ONLY) {
        mg->host_only = true;
        *out = mg;
        return DEC_OK;
    }
    if ((rc = device_build(mg))) return bail(rc);
    *out = mg;
    return DEC_OK;
}

int dec_mg_build_maps(const dec_mesh *const *meshes, int nlevels, const int32_t *const *map_idx,
                      const double *const *map_w, int bc, uint32_t flags, const double *star1_scale,
                      const dec_mg_opts *opts, dec_mg **out) {
    if (!meshes || !out || (nlevels > 1 && (!map_idx || !map_w))) return fail(Status::fail(DEC_ERR_ARG, "null pointer"));
    *out = nullptr;
    if (nlevels < 1 || nlevels > 16) return fail(Status::fail(DEC_ERR_ARG, "nlevels must be in 1..16"));
    if (flags & ~(uint32_t)DEC_HOST_ONLY) return fail(Status::fail(DEC_ERR_ARG, "the only flag is DEC_HOST_ONLY"));
    dec_mg_opts o;
    if (int rc = build_opts(opts, o)) return rc;
    dec_mg *mg = new (std::nothrow) dec_mg;
    if (!mg) return fail(Status::fail(DEC_ERR_OOM, "host allocation"));
    auto bail = [&](int code) {
        free_all(mg);
        delete mg;
        return code;
    };
    try {
        std::vector<const decimpl::HostMesh *> ms;
        for (int l = 0; l < nlevels; ++l) {
            if (!meshes[l]) return bail(fail(Status::fail(DEC_ERR_ARG, "null mesh")));
            ms.push_back(dec_mesh_host(meshes[l]));
        }
        std::vector<const int32_t *> mi(map_idx ? map_idx : nullptr, map_idx ? map_idx + (nlevels - 1) : nullptr);
        std::vector<const double *> mw(map_w ? map_w : nullptr, map_w ? map_w + (nlevels - 1) : nullptr);
        Status st = decimpl::build_hierarchy_maps(ms, mi, mw, bc, star1_scale, o, mg->H);
        if (!st.good()) return bail(fail(st));
    } catch (const std::bad_alloc &) {
        return bail(fail(Status::fail(DEC_ERR_OOM, "host allocation")));
    }
    if (flags & DEC_HOST_ONLY) {
        mg->host_only = true;
        *out = mg;
        return DEC_OK;
    }
    if (int rc = device_build(mg)) return bail(rc);
    *out = mg;
    return DEC_OK;
}

void dec_mg_destroy(dec_mg *mg) {
    if (!mg) return;
    free_all(mg);
    delete mg;
}

int dec_mg_info(const dec_mg *mg, dec_mg_info_t *info) {
    if (int rc = check_mg(mg)) return rc;
    if (!info) return fail(Status::fail(DEC_ERR_ARG, "null info"));
    std::memset(info, 0, sizeof(*info));
    info->nlevels = (int)mg->H.levels.size();
    for (int l = 0; l < info->nlevels; ++l) {
        const decimpl::HostLevel &L = mg->H.levels[l];
        info->nv[l] = L.mesh.nv;
        info->ne[l] = L.mesh.ne;
        info->nt[l] = L.mesh.nt;
        info->ell_width[l] = L.K;
        info->lmax[l] = L.lmax;
        info->ncolors[l] = L.ncolors;
    }
    info->bc = mg->H.bc;
    info->dim = mg->H.levels.back().mesh.dim;
    info->device_bytes = mg->bytes;
    for (int l = 0; l < (int)mg->lv.size() && l < 16; ++l) info->tiles[l] = mg->lv[l].tdown.ntiles;
    return DEC_OK;
}

int dec_mg_copy_table(const dec_mg *mg, int level, int what, void *out) {
    if (int rc = check_mg(mg)) return rc;
    if (!out || level < 0 || level >= (int)mg->H.levels.size()) return fail(Status::fail(DEC_ERR_ARG, "bad level"));
    const decimpl::HostLevel &L = mg->H.levels[level];
    switch (what) {
        case DEC_TABLE_VERTS: std::memcpy(out, L.mesh.verts.data(), L.mesh.verts.size() * 8); break;
        case DEC_TABLE_TRIS: std::memcpy(out, L.mesh.tris.data(), L.mesh.tris.size() * 4); break;
        case DEC_TABLE_EDGES: std::memcpy(out, L.mesh.edges.data(), L.mesh.edges.size() * 4); break;
        case DEC_TABLE_MAP_IDX:
        case DEC_TABLE_MAP_W: {
            // the map from level to level + 1: three (coarse vertex, weight) slots per fine vertex
            if (level + 1 >= (int)mg->H.levels.size())
                return fail(Status::fail(DEC_ERR_ARG, "the finest level has no map to a finer level"));
            const int nf = (int)mg->H.levels[level + 1].mesh.nv, nc = (int)L.mesh.nv;
            std::vector<int32_t> mi;
            std::vector<double> mw;
            if (mg->H.mapped) {
                mi = mg->H.map_idx[level];
                mw = mg->H.map_w[level];
            } else {
                const std::vector<int32_t> &par = mg->H.parents[level];
                mi.assign(3 * (size_t)nf, 0);
                mw.assign(3 * (size_t)nf, 0.0);
                for (int v = 0; v < nf; ++v) {
                    const bool kept = v < nc;
                    const int32_t a = kept ? v : par[2 * (size_t)(v - nc)], b = kept ? v : par[2 * (size_t)(v - nc) + 1];
                    mi[3 * (size_t)v] = a;
                    mi[3 * (size_t)v + 1] = b;
                    mi[3 * (size_t)v + 2] = a;
                    mw[3 * (size_t)v] = kept ? 1.0 : 0.5;
                    mw[3 * (size_t)v + 1] = kept ? 0.0 : 0.5;
                }
            }
            if (what == DEC_TABLE_MAP_IDX)
                std::memcpy(out, mi.data(), mi.size() * 4);
            else
                std::memcpy(out, mw.data(), mw.size() * 8);
            break;
        }
        case DEC_TABLE_PARENTS: {
            // the coarse edge of each new vertex of level + 1, in that level's vertex order
            if (level + 1 >= (int)mg->H.levels.size())
                return fail(Status::fail(DEC_ERR_ARG, "the finest level has no parents table"));
            if (mg->H.mapped) return fail(Status::fail(DEC_ERR_ARG, "hierarchies with general-map transfers store DEC_TABLE_MAP_*"));
            const std::vector<int32_t> &par = mg->H.parents[level];
            std::memcpy(out, par.data(), par.size() * 4);
            break;
        }
        case DEC_TABLE_STAR0: std::memcpy(out, L.star0.data(), L.star0.size() * 8); break;
        case DEC_TABLE_STAR1: std::memcpy(out, L.star1.data(), L.star1.size() * 8); break;
        case DEC_TABLE_FREE: {
            int32_t *o = (int32_t *)out;
            for (size_t i = 0; i < L.free_.size(); ++i) o[i] = L.free_[i];
            break;
        }
        case DEC_TABLE_COLORS: std::memcpy(out, L.colors.data(), L.colors.size() * 4); break;
        default: return fail(Status::fail(DEC_ERR_ARG, "unknown table"));
    }
    return DEC_OK;
}

int dec_mg_set_star1(dec_mg *mg, const double *star1, dec_stream_t stream) {
    if (int rc = check_dev(mg)) return rc;
    if (!star1) return fail(Status::fail(DEC_ERR_ARG, "null star1"));
    cudaStream_t s = (cudaStream_t)stream;
    DevLevel &F = mg->lv.back();
    launch(mg, k_set_weights, grid_for(mg, F.n), s, F.n, F.K, mg->slot_edge, star1, F.star0, F.freev, F.w64, F.w32, F.wlo);
    update_diagonals(mg, F, s);
    CK(cudaGetLastError());
    return DEC_OK;
}

int dec_laplace0_apply(const dec_mg *mgc, int level, const void *x, void *y, int k, int prec, dec_stream_t stream) {
    if (int rc = check_dev(mgc)) return rc;
    dec_mg *mg = const_cast<dec_mg *>(mgc);
    if (!x || !y || level < 0 || level >= (int)mg->lv.size() || k < 1 || (prec != DEC_F64 && prec != DEC_F32))
        return fail(Status::fail(DEC_ERR_ARG, "bad argument"));
    cudaStream_t s = (cudaStream_t)stream;
    DevLevel &L = mg->lv[level];
    if (k > 1) {
        const int g = grid_for(mg, (int64_t)L.n * k);
        if (prec == DEC_F64)
            launch(mg, k_apply_k<double, false>, g, s, L.n, L.K, k, (const int32_t *)L.col, (const double *)L.w64,
                   (const double *)x, (const double *)nullptr, (double *)y);
        else
            launch(mg, k_apply_k<float, false>, g, s, L.n, L.K, k, (const int32_t *)L.col, (const float *)L.w32,
                   (const float *)x, (const float *)nullptr, (float *)y);
        CK(cudaGetLastError());
        return DEC_OK;
    }
    dispatch_k(L.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        if (prec == DEC_F64)
            launch(mg, k_apply<double, KT>, grid_for(mg, L.n), s, L.n, L.K, L.col, L.w64, (const double *)x,
                                                                      (double *)y, nullptr);
        else
            launch(mg, k_apply<float, KT>, grid_for(mg, L.n), s, L.n, L.K, L.col, L.w32, (const float *)x,
                                                                     (float *)y, nullptr);
    });
    CK(cudaGetLastError());
    return DEC_OK;
}

int dec_residual(const dec_mg *mgc, int level, const void *b, const void *x, void *r, int k, int prec,
                 dec_stream_t stream) {
    if (int rc = check_dev(mgc)) return rc;
    dec_mg *mg = const_cast<dec_mg *>(mgc);
    if (!b || !x || !r || level < 0 || level >= (int)mg->lv.size() || k < 1 || (prec != DEC_F64 && prec != DEC_F32))
        return fail(Status::fail(DEC_ERR_ARG, "bad argument"));
    cudaStream_t s = (cudaStream_t)stream;
    DevLevel &L = mg->lv[level];
    if (k > 1) {
        const int g = grid_for(mg, (int64_t)L.n * k);
        if (prec == DEC_F64)
            launch(mg, k_apply_k<double, true>, g, s, L.n, L.K, k, (const int32_t *)L.col, (const double *)L.w64,
                   (const double *)x, (const double *)b, (double *)r);
        else
            launch(mg, k_apply_k<float, true>, g, s, L.n, L.K, k, (const int32_t *)L.col, (const float *)L.w32,
                   (const float *)x, (const float *)b, (float *)r);
        CK(cudaGetLastError());
        return DEC_OK;
    }
    dispatch_k(L.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        if (prec == DEC_F64)
            launch(mg, k_residual_dg<KT>, grid_for(mg, L.n), s, L.n, L.K, L.col, (const double *)L.w64,
                   (const double *)L.dg64, (const double *)b, (const double *)x, (double *)r, (const int *)nullptr);
        else
            launch(mg, k_residual<float, KT>, grid_for(mg, L.n), s, L.n, L.K, L.col, L.w32, (const float *)b,
                                                                        (const float *)x, (float *)r, nullptr);
    });
    CK(cudaGetLastError());
    return DEC_OK;
}

int dec_mg_vcycle(dec_mg *mg, const void *b, void *x, int k, int prec, dec_stream_t stream) {
    if (int rc = check_dev(mg)) return rc;
    if (!b || !x || k < 1 || (prec != DEC_F64 && prec != DEC_F32)) return fail(Status::fail(DEC_ERR_ARG, "bad argument"));
    cudaStream_t s = (cudaStream_t)stream;
    const int top = (int)mg->lv.size() - 1;
    DevLevel &F = mg->lv[top];
    const int g = grid_for(mg, F.n);
    if (k > 1) {
        // one column at a time through contiguous copies
        if (int rc = column_buffers(mg)) return rc;
        for (int j = 0; j < k; ++j) {
            if (prec == DEC_F64) {
                launch(mg, k_col_gather<double>, g, s, F.n, k, j, (const double *)b, mg->tmp);
                launch(mg, k_col_gather<double>, g, s, F.n, k, j, (const double *)x, mg->kx64);
            } else {
                launch(mg, k_col_gather<float>, g, s, F.n, k, j, (const float *)b, mg->kb32);
                launch(mg, k_col_gather<float>, g, s, F.n, k, j, (const float *)x, mg->kx32);
            }
            const int rc = dec_mg_vcycle(mg, prec == DEC_F64 ? (const void *)mg->tmp : (const void *)mg->kb32,
                                         prec == DEC_F64 ? (void *)mg->kx64 : (void *)mg->kx32, 1, prec, stream);
            if (rc) return rc;
            if (prec == DEC_F64)
                launch(mg, k_col_scatter<double>, g, s, F.n, k, j, (const double *)mg->kx64, (double *)x);
            else
                launch(mg, k_col_scatter<float>, g, s, F.n, k, j, (const float *)mg->kx32, (float *)x);
        }
        CK(cudaGetLastError());
        return DEC_OK;
    }
    dispatch_k(F.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        if (prec == DEC_F64) {
            launch(mg, k_residual_dg<KT>, g, s, F.n, F.K, F.col, (const double *)F.w64, (const double *)F.dg64,
                   (const double *)b, (const double *)x, F.b64, (const int *)nullptr);
            double *e = cycle<double>(mg, top, F.b64, s, nullptr);
            launch(mg, k_axpy1<double>, g, s, F.n, e, (double *)x, nullptr);
        } else {
            launch(mg, k_residual<float, KT>, g, s, F.n, F.K, F.col, F.w32, (const float *)b, (const float *)x,
                                                         F.b32, nullptr);
            float *e = cycle<float>(mg, top, F.b32, s, nullptr);
            launch(mg, k_axpy1<float>, g, s, F.n, e, (float *)x, nullptr);
        }
    });
    CK(cudaGetLastError());
    return DEC_OK;
}

int dec_mg_set_wait_limit(dec_mg *mg, int rounds) {
    if (int rc = check_dev(mg)) return rc;
    if (mg->coarse_top < 0) return DEC_OK;  // no device-side wait in this hierarchy's cycles
    const int r = rounds < 0 ? decdev::kCoarseWaitRounds : std::min(rounds, decdev::kCoarseWaitRounds);
    if (r != mg->coarse_args.wait_rounds) {
        mg->coarse_args.wait_rounds = r;
        drop_graphs(mg);  // captured graphs hold the old argument block
    }
    return DEC_OK;
}

int dec_mg_profile(dec_mg *mg, int enable) {
    if (int rc = check_dev(mg)) return rc;
    if (enable < 0 || enable > 2) return fail(Status::fail(DEC_ERR_ARG, "enable must be 0, 1 or 2"));
    drop_graphs(mg);
    mg->prof = enable;
    std::memset(mg->prof_ms, 0, sizeof(mg->prof_ms));
    std::memset(mg->prof_n, 0, sizeof(mg->prof_n));
    return DEC_OK;
}

int dec_mg_profile_read(const dec_mg *mg, dec_prof_entry *out, int max, int *count) {
    if (int rc = check_dev(mg)) return rc;
    if (!count || (max > 0 && !out)) return fail(Status::fail(DEC_ERR_ARG, "null pointer"));
    int c = 0;
    for (int k = 0; k < DEC_PK_COUNT; ++k)
        for (int l = 0; l < (int)mg->lv.size(); ++l) {
            if (mg->prof_n[k][l] == 0) continue;
            if (c < max) out[c] = dec_prof_entry{k, l, mg->prof_n[k][l], mg->prof_ms[k][l], (int64_t)mg->lv[l].n};
            ++c;
        }
    *count = std::min(c, max);
    return DEC_OK;
}

int dec_mg_time_smooth(dec_mg *mg, int level, int reps, double *avg_ms, double *bytes, dec_stream_t stream) {
    if (int rc = check_dev(mg)) return rc;
    const int nl = (int)mg->lv.size();
    if (level < 0) level += nl;
    if (reps < 1 || !avg_ms || !bytes || level < 1 || level >= nl)
        return fail(Status::fail(DEC_ERR_ARG, "bad argument (level must lie above the coarsest)"));
    if (mg->H.opts.smoother == DEC_SMOOTH_MCGS)
        return fail(Status::fail(DEC_ERR_ARG, "dec_mg_time_smooth times the Jacobi / Chebyshev sweep"));
    DevLevel &L = mg->lv[level];
    const bool cheb = mg->H.opts.smoother == DEC_SMOOTH_CHEBYSHEV;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = sizeof(float) * L.n;
    CK(cudaMemsetAsync(L.x32[0], 0, vb, s));
    CK(cudaMemsetAsync(L.x32[1], 0, vb, s));
    CK(cudaMemsetAsync(L.d32[0], 0, vb, s));
    CK(cudaMemsetAsync(L.b32, 0, vb, s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int g = grid_for(mg, L.n);
    const int *noskip = nullptr;
    // the last step of a smoothing call: reads x, b and (Chebyshev) a direction, writes x
    auto sweep = [&](int it) {
        float *xi = L.x32[it & 1], *xo = L.x32[1 - (it & 1)];
        dispatch_k(L.K, [&](auto kt) {
            constexpr int KT = decltype(kt)::value;
            if (cheb)
                launch(mg, k_smooth<float, KT, true, false>, g, s, L.n, L.K, (const int32_t *)L.col,
                       (const float *)L.w32, (const float *)L.b32, (const float *)xi, (const float *)L.d32[0], xo,
                       (float *)nullptr, 0.5f, 0.5f, noskip);
            else
                launch(mg, k_smooth<float, KT, false, false>, g, s, L.n, L.K, (const int32_t *)L.col,
                       (const float *)L.w32, (const float *)L.b32, (const float *)xi, (const float *)nullptr, xo,
                       (float *)nullptr, 0.f, (float)mg->H.opts.omega, noskip);
        });
    };
    for (int r = 0; r < 3; ++r) sweep(r);
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) sweep(r);
    cudaEventRecord(e1, s);
    cudaError_t ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ce != cudaSuccess) return cuda_fail(ce, "dec_mg_time_smooth");
    CK(cudaGetLastError());
    *avg_ms = ms / reps;
    // per row: K column indices and K weights, x_i, b_i, the new x_i (+ the direction)
    *bytes = (double)L.n * (8.0 * L.K + 4.0 * (3 + (cheb ? 1 : 0)));
    return DEC_OK;
}

int dec_mg_time_kernel(dec_mg *mg, int kind, int level, int reps, double *avg_ms, double *bytes, dec_stream_t stream) {
    if (kind == DEC_PK_SMOOTH) return dec_mg_time_smooth(mg, level, reps, avg_ms, bytes, stream);
    if (int rc = check_dev(mg)) return rc;
    const int nl = (int)mg->lv.size();
    if (level < 0) level += nl;
    const dec_mg_opts &o = mg->H.opts;
    if (reps < 1 || !avg_ms || !bytes || level != nl - 1 || o.smoother == DEC_SMOOTH_MCGS ||
        (kind != DEC_PK_SMOOTHDOTS && kind != DEC_PK_SPMV64 && kind != DEC_PK_UPDATE))
        return fail(Status::fail(DEC_ERR_ARG, "bad argument (finest level; DEC_PK_SMOOTH, SMOOTHDOTS, SPMV64 or UPDATE)"));
    DevLevel &F = mg->lv.back();
    const bool cheb = o.smoother == DEC_SMOOTH_CHEBYSHEV;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = sizeof(float) * F.n;
    // zeroed FP32 work vectors: the same kernels and launch shapes as in the mixed_ff loop
    float *zero[] = {F.x32[0], F.x32[1], F.d32[0], F.b32, mg->zo32, mg->fp, mg->fqh, mg->fql, mg->fxh, mg->fxl, mg->frl};
    for (float *z : zero) CK(cudaMemsetAsync(z, 0, vb, s));
    // the reduction epilogues update the solver's scalars (iteration count, history slot): start them at zero
    CK(cudaMemsetAsync(mg->scal, 0, sizeof(Scal), s));
    const int rg = red_grid(mg, F.n);
    const int *noskip = nullptr;
    const int gauge = mg->H.bc == DEC_BC_GAUGE;
    int s0mode = 0;  // the outer update carries the first smoothing step as in the solve
    float e0s = 0.f;
    if ((o.fuse & DEC_FUSE_OUTER) && o.nu1 > 0) {
        s0mode = cheb && 1 < o.nu1 ? 2 : 1;
        e0s = (float)(cheb ? F.e_pre[0] : o.omega);
    }
    auto one = [&]() {
        dispatch_k(F.K, [&](auto kt) {
            constexpr int KT = decltype(kt)::value;
            if (kind == DEC_PK_SMOOTHDOTS) {
                const float e = (float)(cheb ? F.e_post.back() : o.omega), c = (float)(cheb ? F.c_post.back() : 0.0);
                if (cheb)
                    launch(mg, k_smooth_zdots<KT, true>, rg, s, F.n, F.K, (const int32_t *)F.col, (const float *)F.w32,
                           (const float *)F.b32, (const float *)F.x32[0], (const float *)F.d32[0], F.x32[1], c, e,
                           (const float *)F.star0_32, (const uint8_t *)F.freev, (const float *)mg->zo32, 0, gauge,
                           mg->partials, mg->counter, mg->scal, noskip);
                else
                    launch(mg, k_smooth_zdots<KT, false>, rg, s, F.n, F.K, (const int32_t *)F.col,
                           (const float *)F.w32, (const float *)F.b32, (const float *)F.x32[0], (const float *)nullptr,
                           F.x32[1], c, e, (const float *)F.star0_32, (const uint8_t *)F.freev,
                           (const float *)mg->zo32, 0, gauge, mg->partials, mg->counter, mg->scal, noskip);
            } else if (kind == DEC_PK_SPMV64) {
                launch(mg, k_pcg_spmv_ff<KT>, rg, s, F.n, F.K, (const int32_t *)F.col, (const float *)F.w32,
                       (const float *)F.wlo, (const float *)F.star0_32, (const float *)mg->fp, mg->fqh, mg->fql,
                       mg->partials, mg->counter, mg->scal, noskip);
            } else {
                launch(mg, k_pcg_update_ff, rg, s, F.n, (const float *)mg->fp, (const float *)mg->fqh,
                       (const float *)mg->fql, mg->fxh, mg->fxl, F.b32, mg->frl, mg->partials, mg->counter, mg->scal,
                       noskip, s0mode, (const float *)F.dg32, F.x32[0], F.d32[0], e0s);
            }
        });
    };
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int r = 0; r < 3; ++r) one();
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) one();
    cudaEventRecord(e1, s);
    cudaError_t ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ce != cudaSuccess) return cuda_fail(ce, "dec_mg_time_kernel");
    CK(cudaGetLastError());
    *avg_ms = ms / reps;
    const double K = F.K, n = F.n;
    if (kind == DEC_PK_SMOOTHDOTS)  // operator, b = r32, x, direction, new x; *0, free mask, previous z
        *bytes = n * (8.0 * K + 4.0 * (3 + (cheb ? 1 : 0)) + 4.0 + 1.0 + 4.0);
    else if (kind == DEC_PK_SPMV64)  // col, w32 + wlo, p_i, q hi+lo, *0
        *bytes = n * (12.0 * K + 4.0 + 8.0 + 4.0);
    else  // p, q hi+lo, x and r hi+lo read and written; fused: the diagonal, the first step's x (and direction)
        *bytes = n * (4.0 + 8.0 + 16.0 + 16.0 + (s0mode ? 8.0 : 0.0) + (s0mode == 2 ? 4.0 : 0.0));
    return DEC_OK;
}

int dec_solve(dec_mg *mg, const double *b, double *x, int k, const dec_solve_opts *opts, dec_stats *stats,
              dec_stream_t stream) {
    if (int rc = check_dev(mg)) return rc;
    if (!b || !x || k < 1) return fail(Status::fail(DEC_ERR_ARG, "bad argument"));
    if (k == 1) return solve_impl(mg, b, x, opts, stats, (cudaStream_t)stream);
    // several interleaved right-hand sides: one solve per column through contiguous copies
    cudaStream_t s = (cudaStream_t)stream;
    if (int rc = column_buffers(mg)) return rc;
    const DevLevel &F = mg->lv.back();
    const int g = grid_for(mg, F.n);
    const bool warm = opts && opts->warm_start;
    dec_stats tot{}, one{};
    int worst = DEC_OK;
    for (int j = 0; j < k; ++j) {
        launch(mg, k_col_gather<double>, g, s, F.n, k, j, b, mg->tmp);
        if (warm) launch(mg, k_col_gather<double>, g, s, F.n, k, j, (const double *)x, mg->kx64);
        const int rc = solve_impl(mg, mg->tmp, mg->kx64, opts, &one, s);
        if (rc != DEC_OK && rc != DEC_ERR_NOT_CONVERGED) return rc;
        if (rc != DEC_OK) worst = rc;
        launch(mg, k_col_scatter<double>, g, s, F.n, k, j, (const double *)mg->kx64, x);
        tot.iters = std::max(tot.iters, one.iters);
        tot.rel_res = std::max(tot.rel_res, one.rel_res);
        tot.rel_res0 = std::max(tot.rel_res0, one.rel_res0);
        tot.launches += one.launches + (warm ? 3 : 2);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    if (stats) *stats = tot;
    if (worst != DEC_OK) return fail(Status::fail(worst, "a right-hand side did not reach tol within maxit"));
    return DEC_OK;
}

int dec_solve_host(dec_mg *mg, const double *b, double *x, int k, const dec_solve_opts *opts, dec_stats *stats,
                   dec_stream_t stream) {
    if (int rc = check_dev(mg)) return rc;
    if (!b || !x || k != 1)
        return fail(Status::fail(DEC_ERR_ARG, "host-buffer solves take one right-hand side (k = 1)"));
    return solve_impl(mg, b, x, opts, stats, (cudaStream_t)stream, true, true);
}

int dec_solve_backward(dec_mg *mg, const double *u, const double *grad_u, double *grad_b, double *grad_star1,
                       const dec_solve_opts *opts, dec_stats *stats, dec_stream_t stream) {
    if (int rc = check_dev(mg)) return rc;
    if (!u || !grad_u || !grad_b) return fail(Status::fail(DEC_ERR_ARG, "null pointer"));
    cudaStream_t s = (cudaStream_t)stream;
    DevLevel &F = mg->lv.back();
    // L mu = *0^-1 grad_u, solved into grad_b, then grad_b = *0 mu
    launch(mg, k_star0_scale, grid_for(mg, F.n), s, F.n, F.star0, grad_u, mg->tmp, 1);
    CK(cudaGetLastError());
    int rc = solve_impl(mg, mg->tmp, grad_b, opts, stats, s);
    if (rc != DEC_OK && rc != DEC_ERR_NOT_CONVERGED) return rc;
    if (grad_star1) {
        launch(mg, k_edge_grad, grid_for(mg, F.ne), s, F.ne, mg->edges, grad_b, u, grad_star1);
    }
    launch(mg, k_star0_scale, grid_for(mg, F.n), s, F.n, F.star0, grad_b, grad_b, 0);
    CK(cudaGetLastError());
    if (stats) stats->launches += grad_star1 ? 3 : 2;
    return rc;
}

}  // extern "C"

// ===========================================================================
// dec_mg_vcycle_noalloc: the FP32 cycle of dec_mg_vcycle with its level work
// vectors taken from one file-scope device array instead of memory that the
// handle allocated.  For callers that may not allocate device memory at the
// point where they run the cycle (see include/dec.h).
// ===========================================================================

// Scratch shared by every call on a device: per level six float vectors
// (two iterates, two Chebyshev directions, residual, right-hand side), each
// starting on a 256-byte boundary.
static __device__ __align__(256) float g_noalloc_scratch[DEC_NOALLOC_SCRATCH_BYTES / sizeof(float)];

namespace {

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
float *g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the host-side symbol is only a stand-in, never a device address).
int noalloc_scratch(float **out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(Status::fail(DEC_ERR_ARG, "device index out of range"));
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[dev] = (float *)p;
    }
    *out = g_noalloc_ptr[dev];
    return DEC_OK;
}

struct NoallocLevel {
    float *x[2], *d[2], *r, *b;
};

inline size_t noalloc_stride(int n) { return ((size_t)n + 63) / 64 * 64; }  // floats, 256-byte multiple

size_t noalloc_floats(const dec_mg *mg) {
    size_t f = 0;
    for (const DevLevel &L : mg->lv) f += 6 * noalloc_stride(L.n);
    return f;
}

void noalloc_smooth(dec_mg *mg, int l, NoallocLevel &B, const float *b, int nu, bool from_zero, bool post, int &cur,
                    cudaStream_t s) {
    DevLevel &L = mg->lv[l];
    const dec_mg_opts &o = mg->H.opts;
    const bool cheb = o.smoother == DEC_SMOOTH_CHEBYSHEV;
    const std::vector<double> &cc = post ? L.c_post : L.c_pre;
    const std::vector<double> &ee = post ? L.e_post : L.e_pre;
    const int g = grid_for(mg, L.n);
    dispatch_k(L.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        for (int k = 0; k < nu; ++k) {
            const float e = (float)(cheb ? ee[k] : o.omega);
            const float c = (float)(cheb ? cc[k] : 0.0);
            const bool dout = cheb && k + 1 < nu;
            if (k == 0 && from_zero) {
                cur = 0;
                if (dout)
                    launch(mg, k_smooth0<float, KT, true>, g, s, L.n, L.K, L.w32, b, B.x[0], B.d[0], e, nullptr);
                else
                    launch(mg, k_smooth0<float, KT, false>, g, s, L.n, L.K, L.w32, b, B.x[0], nullptr, e, nullptr);
                continue;
            }
            const int nxt = 1 - cur;
            const bool din = cheb && k > 0;
            if (din && dout)
                launch(mg, k_smooth<float, KT, true, true>, g, s, L.n, L.K, L.col, L.w32, b, B.x[cur], B.d[cur],
                                                                       B.x[nxt], B.d[nxt], c, e, nullptr);
            else if (din)
                launch(mg, k_smooth<float, KT, true, false>, g, s, L.n, L.K, L.col, L.w32, b, B.x[cur], B.d[cur],
                                                                        B.x[nxt], nullptr, c, e, nullptr);
            else if (dout)
                launch(mg, k_smooth<float, KT, false, true>, g, s, L.n, L.K, L.col, L.w32, b, B.x[cur], nullptr,
                                                                        B.x[nxt], B.d[nxt], c, e, nullptr);
            else
                launch(mg, k_smooth<float, KT, false, false>, g, s, L.n, L.K, L.col, L.w32, b, B.x[cur], nullptr,
                                                                         B.x[nxt], nullptr, c, e, nullptr);
            cur = nxt;
        }
    });
}

// err keeps the first failed enqueue that is not a kernel launch (launch
// errors surface through cudaGetLastError).
float *noalloc_cycle(dec_mg *mg, std::vector<NoallocLevel> &B, int l, const float *b, cudaStream_t s,
                     cudaError_t &err) {
    DevLevel &L = mg->lv[l];
    if (l == 0) {
        int g = (int)std::min<int64_t>(mg->nsm * 4, (L.n * 32 + kThreads - 1) / kThreads);
        launch(mg, k_coarse<float>, g, s, L.n, mg->G32, b, B[0].x[0], nullptr);
        return B[0].x[0];
    }
    const dec_mg_opts &o = mg->H.opts;
    DevLevel &C = mg->lv[l - 1];
    int cur = 0;
    if (o.nu1 > 0) {
        noalloc_smooth(mg, l, B[l], b, o.nu1, true, false, cur, s);
    } else {
        const cudaError_t e = cudaMemsetAsync(B[l].x[0], 0, sizeof(float) * L.n, s);  // the iterate starts at zero
        if (e != cudaSuccess && err == cudaSuccess) err = e;
    }
    const int g = grid_for(mg, L.n);
    dispatch_k(L.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        launch(mg, k_residual<float, KT>, g, s, L.n, L.K, L.col, L.w32, b, B[l].x[cur], B[l].r, nullptr);
        if (o.restriction == DEC_RESTRICT_STAR0)
            launch(mg, k_restrict<float, KT, true>, grid_for(mg, C.n), s, C.n, L.n, L.K, L.col, B[l].r, B[l - 1].b,
                   L.star0_32, C.star0_32, nullptr, (const float *)nullptr, (float *)nullptr, (float *)nullptr, 0.f);
        else
            launch(mg, k_restrict<float, KT, false>, grid_for(mg, C.n), s, C.n, L.n, L.K, L.col, B[l].r, B[l - 1].b,
                   (const float *)nullptr, (const float *)nullptr, nullptr, (const float *)nullptr, (float *)nullptr,
                   (float *)nullptr, 0.f);
    });
    float *ec = noalloc_cycle(mg, B, l - 1, B[l - 1].b, s, err);
    launch(mg, k_prolong<float>, g, s, C.n, L.n, L.par, ec, B[l].x[cur], nullptr);
    if (o.nu2 > 0) noalloc_smooth(mg, l, B[l], b, o.nu2, false, true, cur, s);
    return B[l].x[cur];
}

}  // namespace

extern "C" int dec_mg_vcycle_noalloc(dec_mg *mg, const float *b, float *x, dec_stream_t stream) {
    if (int rc = check_dev(mg)) return rc;
    if (!b || !x) return fail(Status::fail(DEC_ERR_ARG, "null pointer"));
    if (mg->H.opts.gamma != 1 || mg->H.opts.fcycle)
        return fail(Status::fail(DEC_ERR_ARG, "the allocation-free cycle is a V-cycle (gamma = 1)"));
    if (mg->H.opts.smoother == DEC_SMOOTH_MCGS)
        return fail(Status::fail(DEC_ERR_ARG, "the allocation-free cycle smooths with Jacobi or Chebyshev"));
    if (mg->H.mapped) return fail(Status::fail(DEC_ERR_ARG, "the allocation-free cycle transfers along binary subdivision (no general maps)"));
    const size_t need = noalloc_floats(mg) * sizeof(float);
    if (need > DEC_NOALLOC_SCRATCH_BYTES)
        return fail(Status::fail(DEC_ERR_ARG, "hierarchy needs " + std::to_string(need) +
                                                  " bytes of cycle scratch, above the DEC_NOALLOC_SCRATCH_BYTES limit of " +
                                                  std::to_string((size_t)DEC_NOALLOC_SCRATCH_BYTES)));
    float *base = nullptr;
    if (int rc = noalloc_scratch(&base)) return rc;
    std::vector<NoallocLevel> B(mg->lv.size());
    float *p = base;
    for (size_t l = 0; l < mg->lv.size(); ++l) {
        const size_t st = noalloc_stride(mg->lv[l].n);
        float **slots[6] = {&B[l].x[0], &B[l].x[1], &B[l].d[0], &B[l].d[1], &B[l].r, &B[l].b};
        for (float **q : slots) {
            *q = p;
            p += st;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int top = (int)mg->lv.size() - 1;
    DevLevel &F = mg->lv[top];
    const int g = grid_for(mg, F.n);
    dispatch_k(F.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        launch(mg, k_residual<float, KT>, g, s, F.n, F.K, F.col, F.w32, b, x, B[top].b, nullptr);
    });
    cudaError_t err = cudaSuccess;
    float *e = noalloc_cycle(mg, B, top, B[top].b, s, err);
    launch(mg, k_axpy1<float>, g, s, F.n, e, x, nullptr);
    if (err != cudaSuccess) {
        (void)cudaGetLastError();
        return cuda_fail(err, "cudaMemsetAsync (allocation-free cycle)");
    }
    CK(cudaGetLastError());
    return DEC_OK;
}

// ===========================================================================
// porous convection: forward steps and the checkpointed adjoint (Sec. 3.2)
// ===========================================================================

namespace {

struct PorousRun {
    dec_mg *mg;
    cudaStream_t s;
    dec_porous_params prm;
    const uint8_t *fixed;
    dec_solve_opts so;
    int64_t iters = 0;
    double worst = 0.0;
    int64_t launches = 0;
};

int porous_check(dec_mg *mg, const dec_porous_params *prm, dec_porous_params &out) {
    if (int rc = check_dev(mg)) return rc;
    if (mg->H.bc != DEC_BC_GAUGE) return fail(Status::fail(DEC_ERR_ARG, "porous steps need a DEC_BC_GAUGE hierarchy"));
    if (prm)
        out = *prm;
    else
        dec_porous_default_params(&out);
    if (!(out.dt > 0.0) || !(out.phi > 0.0) || !(out.tol >= 0.0) || out.maxit < 1 || out.maxit >= kHist)
        return fail(Status::fail(DEC_ERR_ARG, "bad porous parameters (dt, phi, tol, maxit)"));
    if (out.alpha_rho0 <= 0.0) {
        double gn = std::sqrt(out.g[0] * out.g[0] + out.g[1] * out.g[1] + out.g[2] * out.g[2]);
        if (!(gn > 0.0)) return fail(Status::fail(DEC_ERR_ARG, "zero gravity with alpha_rho0 <= 0"));
        out.alpha_rho0 = 1.0 / gn;
    }
    return DEC_OK;
}

void porous_potential(PorousRun &R) {
    dec_mg *mg = R.mg;
    DevLevel &F = mg->lv.back();
    launch(mg, k_potential, grid_for(mg, F.n), R.s, F.n, mg->dim, mg->verts, R.prm.g[0], R.prm.g[1], R.prm.g[2],
                                                        R.prm.alpha_rho0, mg->pot);
    R.launches += 1;
}

// rhs(T); P <- solve (warm); T_out = update(T_in, P)
int porous_one_step(PorousRun &R, const double *T_in, double *P, double *T_out) {
    dec_mg *mg = R.mg;
    DevLevel &F = mg->lv.back();
    const int g = grid_for(mg, F.n);
    dispatch_k(F.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        launch(mg, k_porous_rhs<KT>, g, R.s, F.n, F.K, F.col, F.w64, T_in, mg->pot, mg->prhs);
    });
    dec_stats st{};
    int rc = solve_impl(mg, mg->prhs, P, &R.so, &st, R.s);
    if (rc != DEC_OK) decimpl::set_error("pressure solve: " + std::string(dec_last_error()));
    R.iters += st.iters;
    R.worst = std::max(R.worst, st.rel_res);
    R.launches += st.launches + 2;
    if (rc != DEC_OK) return rc;
    dispatch_k(F.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        launch(mg, k_porous_update<KT>, g, R.s, F.n, F.K, F.col, F.w64, T_in, P, mg->pot, R.fixed,
                                                    1.0 / R.prm.phi, R.prm.k_eta, R.prm.kappa, R.prm.dt, T_out);
    });
    CK(cudaGetLastError());
    return DEC_OK;
}

// lam <- (dT_{n+1}/dT_n)^T lam at the state (T, P) of step n; uses `out`, `ms`, `pbs`, `m` as work vectors.
int porous_adjoint_step(PorousRun &R, const double *T, const double *P, double *&lam, double *&out, double *ms,
                        double *pbs, double *m) {
    dec_mg *mg = R.mg;
    DevLevel &F = mg->lv.back();
    const int g = grid_for(mg, F.n);
    launch(mg, k_porous_adj1, g, R.s, F.n, lam, R.fixed, F.star0, R.prm.dt, ms);
    dispatch_k(F.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        launch(mg, k_porous_adj2<KT>, g, R.s, F.n, F.K, F.col, F.w64, F.star0, T, P, mg->pot, lam, ms,
                                                  1.0 / R.prm.phi, R.prm.k_eta, R.prm.kappa, out, pbs);
    });
    dec_solve_opts so = R.so;  // adjoint pressure solve, warm-started from the previous m
    dec_stats st{};
    int rc = solve_impl(mg, pbs, m, &so, &st, R.s);
    if (rc != DEC_OK) decimpl::set_error("adjoint pressure solve: " + std::string(dec_last_error()));
    R.iters += st.iters;
    R.worst = std::max(R.worst, st.rel_res);
    R.launches += st.launches + 3;
    if (rc != DEC_OK) return rc;
    dispatch_k(F.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        launch(mg, k_porous_adj3<KT>, g, R.s, F.n, F.K, F.col, F.w64, F.star0, mg->pot, m, out);
    });
    CK(cudaGetLastError());
    std::swap(lam, out);
    return DEC_OK;
}

void porous_stats(const PorousRun &R, dec_stats *stats) {
    if (!stats) return;
    stats->iters = (int)std::min<int64_t>(R.iters, INT32_MAX);
    stats->rel_res = R.worst;
    stats->rel_res0 = 0.0;
    stats->launches = R.launches;
}

}  // namespace

extern "C" {

void dec_porous_default_params(dec_porous_params *p) {
    if (!p) return;
    p->g[0] = 0.0;
    p->g[1] = -9.81;
    p->g[2] = 0.0;
    p->alpha_rho0 = 0.0;
    p->phi = 0.1;
    p->k_eta = 1.0;
    p->kappa = 2.0;
    p->dt = 0.0;
    p->tol = 1e-8;
    p->mode = DEC_MODE_MIXED;
    p->maxit = 100;
}

int dec_porous_step(dec_mg *mg, double *T, double *P, const uint8_t *fixed, const dec_porous_params *prm, int nsteps,
                    double *checkpoints, int ckpt_every, dec_stats *stats, dec_stream_t stream) {
    PorousRun R{mg, (cudaStream_t)stream, {}, fixed, {}};
    if (int rc = porous_check(mg, prm, R.prm)) return rc;
    if (!T || !P || !fixed || nsteps < 0 || (checkpoints && ckpt_every < 1))
        return fail(Status::fail(DEC_ERR_ARG, "bad argument"));
    dec_solve_default_opts(&R.so);
    R.so.mode = R.prm.mode;
    R.so.tol = R.prm.tol;
    R.so.maxit = R.prm.maxit;
    R.so.warm_start = 1;
    const int n = mg->lv.back().n;
    const size_t vb = sizeof(double) * n;
    porous_potential(R);
    double *cur = T, *other = mg->ptmp;
    int ck = 0;
    for (int step = 0; step < nsteps; ++step) {
        if (checkpoints && step % ckpt_every == 0)
            CK(cudaMemcpyAsync(checkpoints + (size_t)ck++ * n, cur, vb, cudaMemcpyDeviceToDevice, R.s));
        if (int rc = porous_one_step(R, cur, P, other)) {
            porous_stats(R, stats);
            return rc;
        }
        std::swap(cur, other);
    }
    if (checkpoints && nsteps % ckpt_every == 0)
        CK(cudaMemcpyAsync(checkpoints + (size_t)ck * n, cur, vb, cudaMemcpyDeviceToDevice, R.s));
    if (cur != T) CK(cudaMemcpyAsync(T, cur, vb, cudaMemcpyDeviceToDevice, R.s));
    CK(cudaStreamSynchronize(R.s));
    porous_stats(R, stats);
    return DEC_OK;
}

// Tsitouras' 5(4) pair (Ch. Tsitouras, Comput. Math. Appl. 62 (2011) 770-775),
// the "Tsit5" integrator of Sec. 3.2.2: the strictly lower coupling
// coefficients (row 6 doubles as the 5th-order weights: first same as last;
// the model is autonomous, so the nodes are not needed) and the error
// weights of the embedded 4th-order solution.
constexpr double kTsA[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {0.161, 0, 0, 0, 0, 0},
    {-0.008480655492356989, 0.335480655492357, 0, 0, 0, 0},
    {2.897153057105493, -6.359448489975075, 4.3622954328695815, 0, 0, 0},
    {5.325864828439257, -11.748883564062828, 7.4955393428898365, -0.09249506636175525, 0, 0},
    {5.86145544294642, -12.92096931784711, 8.159367898576159, -0.071584973281401, -0.028269050394068383, 0},
    {0.09646076681806523, 0.01, 0.4798896504144996, 1.379008574103742, -3.290069515436081, 2.324710524099774}};
constexpr double kTsE[7] = {-0.00178001105222577714, -0.0008164344596567469, 0.007880878010261995,
                            -0.1447110071732629,     0.5823571654525552,     -0.45808210592918697,
                            1.0 / 66.0};

// k = f(Y): the pressure of Y (MG-PCG, warm-started from P), then dT/dt.
int porous_rate(PorousRun &R, const double *Y, double *P, double *k) {
    dec_mg *mg = R.mg;
    DevLevel &F = mg->lv.back();
    const int g = grid_for(mg, F.n);
    dispatch_k(F.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        launch(mg, k_porous_rhs<KT>, g, R.s, F.n, F.K, F.col, F.w64, Y, mg->pot, mg->prhs);
    });
    dec_stats st{};
    int rc = solve_impl(mg, mg->prhs, P, &R.so, &st, R.s);
    if (rc != DEC_OK) decimpl::set_error("pressure solve: " + std::string(dec_last_error()));
    R.iters += st.iters;
    R.worst = std::max(R.worst, st.rel_res);
    R.launches += st.launches + 2;
    if (rc != DEC_OK) return rc;
    dispatch_k(F.K, [&](auto kt) {
        constexpr int KT = decltype(kt)::value;
        launch(mg, k_porous_tdot<KT>, g, R.s, F.n, F.K, F.col, F.w64, Y, (const double *)P, mg->pot, R.fixed,
               1.0 / R.prm.phi, R.prm.k_eta, R.prm.kappa, k);
    });
    CK(cudaGetLastError());
    return DEC_OK;
}

int dec_porous_rk(dec_mg *mg, double *T, double *P, const uint8_t *fixed, const dec_porous_params *prm,
                  double t_end, double dt0, double rtol, double atol, int64_t max_steps, int fixed_step,
                  dec_rk_stats *stats, dec_stream_t stream) {
    if (int rc = check_dev(mg)) return rc;
    dec_porous_params p;
    if (prm)
        p = *prm;
    else
        dec_porous_default_params(&p);
    p.dt = dt0;
    PorousRun R{mg, (cudaStream_t)stream, {}, fixed, {}};
    if (int rc = porous_check(mg, &p, R.prm)) return rc;
    if (!T || !P || !fixed || !(t_end >= 0.0) || !std::isfinite(t_end) || !(rtol >= 0.0) || !(atol >= 0.0) ||
        (!fixed_step && !(rtol > 0.0 || atol > 0.0)) || max_steps < 1)
        return fail(Status::fail(DEC_ERR_ARG, "bad argument (T, P, fixed, t_end, dt0, rtol, atol, max_steps)"));
    dec_solve_default_opts(&R.so);
    R.so.mode = R.prm.mode;
    R.so.tol = R.prm.tol;
    R.so.maxit = R.prm.maxit;
    R.so.warm_start = 1;
    DevLevel &F = mg->lv.back();
    const int n = F.n;
    const size_t vb = sizeof(double) * n;
    // device work: the seven stage rates, the current and the next state, the
    // pressure of the current state and one scalar.  T and P are written only
    // by finish(), so on every return T is the state at out.t and P its pressure.
    double *work = nullptr;
    cudaError_t ce = cudaMalloc(&work, 10 * vb + sizeof(double));
    if (ce != cudaSuccess)
        return ce == cudaErrorMemoryAllocation ? fail(Status::fail(DEC_ERR_OOM, "cudaMalloc")) : cuda_fail(ce, "cudaMalloc");
    double *k[7];
    for (int j = 0; j < 7; ++j) k[j] = work + (size_t)j * n;
    double *cur = work + (size_t)7 * n, *nxt = work + (size_t)8 * n, *pacc = work + (size_t)9 * n;
    double *esum = work + (size_t)10 * n;
    dec_rk_stats out{};
    double t = 0.0, dt = dt0;  // time reached and next step (reported on every return)
    const int g = grid_for(mg, n), rg = red_grid64(mg, n);
    auto finish = [&](int code) {
        out.t = t;
        out.dt = dt;
        cudaError_t e = cudaMemcpyAsync(T, cur, vb, cudaMemcpyDeviceToDevice, R.s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(P, pacc, vb, cudaMemcpyDeviceToDevice, R.s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(R.s);
        if (e != cudaSuccess && code == DEC_OK) code = cuda_fail(e, "dec_porous_rk");
        cudaFree(work);
        out.pressure_iters = R.iters;
        out.pressure_rel_res = R.worst;
        if (stats) *stats = out;
        return code;
    };
    ce = cudaMemcpyAsync(cur, T, vb, cudaMemcpyDeviceToDevice, R.s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(pacc, P, vb, cudaMemcpyDeviceToDevice, R.s);
    if (ce != cudaSuccess) {
        cudaFree(work);
        return cuda_fail(ce, "dec_porous_rk");
    }
    porous_potential(R);
    if (int rc = porous_rate(R, cur, P, k[0])) return finish(rc);
    if ((ce = cudaMemcpyAsync(pacc, P, vb, cudaMemcpyDeviceToDevice, R.s)) != cudaSuccess)
        return finish(cuda_fail(ce, "dec_porous_rk"));
    out.nfev = 1;
    const double slack = 1e-12 * t_end;
    bool rejected_last = false;
    while (t < t_end && out.naccept + out.nreject < max_steps) {
        const bool last = dt >= t_end - t - slack;
        const double h = last ? t_end - t : dt;
        // stages 2..7; stage 7's state is the new state (first same as last)
        for (int i = 1; i < 7; ++i) {
            RkStages c{};
            for (int j = 0; j < i; ++j) {
                c.k[j] = k[j];
                c.a[j] = kTsA[i][j];
            }
            c.nk = i;
            double *y = i < 6 ? mg->ptmp : nxt;
            launch(mg, k_rk_combine, g, R.s, n, (const double *)cur, c, h, y);
            if (int rc = porous_rate(R, y, P, k[i])) return finish(rc);
        }
        out.nfev += 6;
        RkStages e{};
        for (int j = 0; j < 7; ++j) {
            e.k[j] = k[j];
            e.a[j] = kTsE[j];
        }
        e.nk = 7;
        launch(mg, k_rk_error, rg, R.s, n, (const double *)cur, (const double *)nxt, e, h, rtol, atol,
               mg->partials, mg->counter, esum);
        double ssum = 0.0;
        ce = cudaMemcpyAsync(&ssum, esum, sizeof(double), cudaMemcpyDeviceToHost, R.s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(R.s);
        if (ce != cudaSuccess) return finish(cuda_fail(ce, "dec_porous_rk step error"));
        const double en = std::sqrt(ssum / (double)n);
        if (!std::isfinite(en) && !fixed_step) return finish(fail(Status::fail(DEC_ERR_NONFINITE, "non-finite step error")));
        if (fixed_step || en <= 1.0) {
            t = last ? t_end : t + h;
            std::swap(cur, nxt);
            std::swap(k[0], k[6]);
            // P holds the pressure of the accepted stage-7 state
            if ((ce = cudaMemcpyAsync(pacc, P, vb, cudaMemcpyDeviceToDevice, R.s)) != cudaSuccess)
                return finish(cuda_fail(ce, "dec_porous_rk"));
            out.naccept += 1;
            if (!fixed_step) {
                const double grow = rejected_last ? 1.0 : 10.0;
                dt = h * (en == 0.0 ? grow : std::min(grow, std::max(0.2, 0.9 * std::pow(en, -0.2))));
            }
            rejected_last = false;
        } else {
            out.nreject += 1;
            dt = h * std::max(0.2, 0.9 * std::pow(en, -0.2));
            rejected_last = true;
        }
    }
    if (t < t_end) return finish(fail(Status::fail(DEC_ERR_NOT_CONVERGED, "max_steps reached before t_end")));
    return finish(DEC_OK);
}

int dec_porous_backward(dec_mg *mg, const double *T0, const double *P0, const uint8_t *fixed,
                        const dec_porous_params *prm, int nsteps, int ckpt_every, const double *grad_TN,
                        double *grad_T0, dec_stats *stats, dec_stream_t stream) {
    PorousRun R{mg, (cudaStream_t)stream, {}, fixed, {}};
    if (int rc = porous_check(mg, prm, R.prm)) return rc;
    if (!T0 || !P0 || !fixed || !grad_TN || !grad_T0 || nsteps < 0 || ckpt_every < 1)
        return fail(Status::fail(DEC_ERR_ARG, "bad argument"));
    dec_solve_default_opts(&R.so);
    R.so.mode = R.prm.mode;
    R.so.tol = R.prm.tol;
    R.so.maxit = R.prm.maxit;
    R.so.warm_start = 1;
    const int n = mg->lv.back().n;
    const size_t vb = sizeof(double) * n;
    const int nseg = (nsteps + ckpt_every - 1) / ckpt_every;
    // device work memory for this call: segment-start states, one segment of states, 8 vectors
    const size_t nvec = (size_t)2 * std::max(nseg, 1) + (size_t)2 * ckpt_every + 8;
    double *work = nullptr;
    cudaError_t ce = cudaMalloc(&work, nvec * vb);
    if (ce != cudaSuccess) return ce == cudaErrorMemoryAllocation ? fail(Status::fail(DEC_ERR_OOM, "cudaMalloc")) : cuda_fail(ce, "cudaMalloc");
    auto V = [&](size_t i) { return work + i * n; };
    double *ckT = V(0), *ckP = V(nseg);
    double *segT = V(2 * (size_t)nseg), *segP = V(2 * (size_t)nseg + ckpt_every);
    size_t b0 = 2 * (size_t)nseg + 2 * ckpt_every;
    double *A = V(b0), *B = V(b0 + 1), *Pw = V(b0 + 2), *lam = V(b0 + 3), *out = V(b0 + 4), *ms = V(b0 + 5),
           *pbs = V(b0 + 6), *m = V(b0 + 7);
    int rc = DEC_OK;
    auto done = [&](int code) {
        cudaStreamSynchronize(R.s);
        cudaFree(work);
        porous_stats(R, stats);
        return code;
    };
    // every failure below releases `work` through done()
#define CKW(call)                                                         \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return done(cuda_fail(_e, #call));         \
    } while (0)
    porous_potential(R);
    // forward pass, keeping the state (T, warm-start P) at each segment start
    CKW(cudaMemcpyAsync(A, T0, vb, cudaMemcpyDeviceToDevice, R.s));
    CKW(cudaMemcpyAsync(Pw, P0, vb, cudaMemcpyDeviceToDevice, R.s));
    for (int step = 0; step < nsteps; ++step) {
        if (step % ckpt_every == 0) {
            const int sgi = step / ckpt_every;
            CKW(cudaMemcpyAsync(ckT + (size_t)sgi * n, A, vb, cudaMemcpyDeviceToDevice, R.s));
            CKW(cudaMemcpyAsync(ckP + (size_t)sgi * n, Pw, vb, cudaMemcpyDeviceToDevice, R.s));
        }
        if ((rc = porous_one_step(R, A, Pw, B))) return done(rc);
        std::swap(A, B);
    }
    CKW(cudaMemcpyAsync(lam, grad_TN, vb, cudaMemcpyDeviceToDevice, R.s));
    CKW(cudaMemsetAsync(m, 0, vb, R.s));
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
        const int first = sgi * ckpt_every;
        const int len = std::min(ckpt_every, nsteps - first);
        CKW(cudaMemcpyAsync(A, ckT + (size_t)sgi * n, vb, cudaMemcpyDeviceToDevice, R.s));
        CKW(cudaMemcpyAsync(Pw, ckP + (size_t)sgi * n, vb, cudaMemcpyDeviceToDevice, R.s));
        for (int j = 0; j < len; ++j) {  // recompute the segment: T_n and the pressure P_n of step n
            CKW(cudaMemcpyAsync(segT + (size_t)j * n, A, vb, cudaMemcpyDeviceToDevice, R.s));
            if ((rc = porous_one_step(R, A, Pw, B))) return done(rc);
            CKW(cudaMemcpyAsync(segP + (size_t)j * n, Pw, vb, cudaMemcpyDeviceToDevice, R.s));
            std::swap(A, B);
        }
        for (int j = len - 1; j >= 0; --j)
            if ((rc = porous_adjoint_step(R, segT + (size_t)j * n, segP + (size_t)j * n, lam, out, ms, pbs, m))) {
                decimpl::set_error("adjoint step " + std::to_string(first + j) + ": " + std::string(dec_last_error()));
                return done(rc);
            }
    }
    CKW(cudaMemcpyAsync(grad_T0, lam, vb, cudaMemcpyDeviceToDevice, R.s));
    return done(DEC_OK);
#undef CKW
}

}  // extern "C"
