/*
 * dec.h -- C ABI of libdec: geometric multigrid for the DEC 0-form Laplacian
 * on triangle meshes nested by 1->4 midpoint subdivision, on one GB300 GPU.
 *
 * The operator is L = *0^-1 d0^T *1 d0 (Sec. 3.1.1, Eq. hodge0-laplacian,
 * with the sign chosen so that L is positive semidefinite: L = -Delta_0).
 * Interpolation is the matrix of the subdivision map and restriction its
 * row-normalized transpose (Sec. 2.2.1).  Solvers: standalone multigrid and
 * multigrid-preconditioned CG (Sec. 3.1.2), in plain FP64 or with FP32
 * V-cycles inside an FP64 outer iteration.
 *
 * Conventions shared by every call:
 *   - Every function returns an int status (DEC_OK = 0 on success).  On
 *     failure dec_last_error() returns a message for the calling thread.
 *   - Host arrays (double*, int32_t*) passed to *_create / *_build are
 *     copied; the caller keeps ownership.
 *   - Vector arguments of the compute calls are DEVICE pointers on the
 *     device that was current when the hierarchy was built; the caller owns
 *     them.  They are enqueued on `stream` (a cudaStream_t, 0 = legacy
 *     default stream); the call returns after enqueueing unless stated.
 *   - Vertex vectors are in the library's vertex order, which is the order
 *     produced by the subdivision itself: the coarse vertices keep their ids
 *     and the midpoint of coarse edge e gets id n_coarse + e.  With k > 1
 *     right-hand sides a vector is interleaved: value j of vertex v at
 *     [v * k + j].
 *   - A handle may be used by one thread / one stream at a time, with its
 *     device current: a compute call made while another device is current
 *     returns DEC_ERR_ARG.
 */
#ifndef DEC_H
#define DEC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dec_mesh dec_mesh;
typedef struct dec_mg dec_mg;
typedef struct CUstream_st *dec_stream_t; /* same type as cudaStream_t */

/* ---- status codes ------------------------------------------------------ */
enum {
    DEC_OK = 0,
    DEC_ERR_ARG = 1,           /* bad argument (null pointer, size, enum)          */
    DEC_ERR_MESH = 2,          /* mesh violates the simplicial-complex definition  */
    DEC_ERR_CUDA = 3,          /* a CUDA runtime call failed                        */
    DEC_ERR_OOM = 4,           /* host or device allocation failed                  */
    DEC_ERR_NOT_CONVERGED = 5, /* maxit reached; the output holds the last iterate  */
    DEC_ERR_NONFINITE = 6      /* NaN or Inf met in the input or in the iteration   */
};

/* ---- enums ------------------------------------------------------------- */
/* dec_mg_build / dec_mesh_refine flags: DEC_SPHERE_PROJECT pushes new
 * midpoints to the unit sphere; DEC_HOST_ONLY (dec_mg_build) builds the host
 * tables only (no device memory, no CUDA call) so they can be inspected with
 * dec_mg_info / dec_mg_copy_table; compute calls on such a handle return
 * DEC_ERR_ARG.  DEC_ORDER_MORTON numbers each level's new vertices along a
 * space-filling curve instead of the default coarse edge order (see
 * dec_mesh_refine). */
enum { DEC_SPHERE_PROJECT = 1u, DEC_HOST_ONLY = 2u, DEC_ORDER_MORTON = 4u, DEC_SUBDIV_CUBIC = 8u };
enum { DEC_BC_DIRICHLET = 0, DEC_BC_GAUGE = 1 };
enum { DEC_F64 = 0, DEC_F32 = 1 };           /* precision of a single operator call */
/* Smoothers: damped Jacobi (omega); Chebyshev on [cheby_lo, cheby_hi] * lambda_max(D^-1 L);
 * multicolour Gauss-Seidel -- the paper's Gauss-Seidel (Sec. 3.1.2) over the colour classes
 * of a greedy vertex colouring (smallest colour not taken by a lower-numbered neighbour),
 * in increasing colour order, one kernel per class. */
enum { DEC_SMOOTH_JACOBI = 0, DEC_SMOOTH_CHEBYSHEV = 1, DEC_SMOOTH_MCGS = 2 };
/* Restriction: DEC_RESTRICT_ROWNORM is the paper's transpose of the
 * row-normalized subdivision matrix (Sec. 2.2.1); DEC_RESTRICT_STAR0 is the
 * *0-adjoint of interpolation, r_c = *0c^-1 M(f) *0f r_f, which makes the
 * cycle self-adjoint in the *0 inner product (an option, not the paper's). */
enum { DEC_RESTRICT_ROWNORM = 0, DEC_RESTRICT_STAR0 = 1 };
enum { DEC_SOLVER_MG = 0, DEC_SOLVER_MGPCG = 1, DEC_SOLVER_CG = 2 };
/* Precision of a solve (Sec. 3.1.2 with the mixed-precision pattern):
 *   DEC_MODE_F64       cycles and outer iteration in FP64;
 *   DEC_MODE_MIXED     FP32 cycles (smoothing, transfers, coarse solve)
 *                      inside an FP64 outer iteration: the residual b - L x
 *                      and its updates, every dot product (FP64 products and
 *                      FP64 sums), the search directions, the iterate and the
 *                      gauge projection are FP64; the cycle reads the residual
 *                      rounded to FP32 and returns its correction in FP32;
 *   DEC_MODE_MIXED_FF  FP32 cycles inside a float-float outer iteration
 *                      (not in the paper): x, r and L p as unevaluated sums
 *                      of two floats (~48 bits), search directions in FP32,
 *                      all on the FP32 pipe.  The updated residual tracks
 *                      b - L x to about 1e-12 of ||b|| on 10^6-vertex meshes,
 *                      so tolerances down to ~1e-10 are met by the true
 *                      residual; use DEC_MODE_MIXED or DEC_MODE_F64 below that;
 *   DEC_MODE_MIXED_F32DOT  as DEC_MODE_MIXED (FP64 residual, iterate and
 *                      updates), but the dot products that steer alpha, beta,
 *                      the gauge shift and the stopping test are formed from
 *                      FP32 copies with FP32 products and sums (not in the
 *                      paper; fewer FP64 instructions per row).
 * Plain CG (DEC_SOLVER_CG) always runs in FP64. */
enum { DEC_MODE_F64 = 0, DEC_MODE_MIXED = 1, DEC_MODE_MIXED_FF = 2, DEC_MODE_MIXED_F32DOT = 3 };

/* Multigrid options.  dec_mg_default_opts() fills the defaults:
 * Jacobi, nu1 = nu2 = 2, omega = 2/3, Chebyshev interval
 * [0.3, 1.1] * lambda_max(D^-1 L) with lambda_max from 10 power iterations,
 * gamma = 1 (V-cycle; 2 gives a W-cycle, up to 4), no F-cycle, the paper's restriction,
 * the row-local kernel fusions.
 * With gamma > 1 each coarse correction is repeated gamma times,
 * e <- e + C(b - L e), except on the coarsest level whose solve is exact. */
typedef struct dec_mg_opts {
    int smoother;
    int nu1, nu2;
    double omega;
    double cheby_lo, cheby_hi;
    int power_iters;
    int gamma;
    int restriction;  /* DEC_RESTRICT_* */
    int fcycle;       /* 1: F-cycles -- the coarse correction is an F-cycle followed by a
                         V-cycle (gamma ignored); 0: gamma-cycles */
    int coarse_max_rows; /* DEC_FUSE_COARSE: largest level (rows) run in the shared-memory
                            block; 0 (default): the library's choice */
    int fuse;         /* DEC_FUSE_* mask of fused cycle kernels, each bitwise equal to
                         the separate kernels it replaces; default DEC_FUSE_RESTRICT0 |
                         DEC_FUSE_OUTER | DEC_FUSE_COARSE | DEC_FUSE_PATCH (the fusions that
                         gather a second vector measured slower on GB300) */
    int fuse_max_rows; /* the gathering fusions (DEC_FUSE_SMOOTH01, _RESTRICT, _PROLONG) run
                          on levels of at most this many rows, the separate kernels on larger
                          ones; 0 (default): every level */
    int patch_max_rows; /* DEC_FUSE_PATCH: largest level (rows) run as halo tiles; 0 (default):
                           every level between the coarsest and the finest */
    int patch_chunk;    /* DEC_FUSE_PATCH: coarse vertices per tile (consecutive in Z-order);
                           0 (default): 24 */
    int patch_threads;  /* DEC_FUSE_PATCH: threads per tile block, a multiple of 32 up to 256;
                           0 (default): 256 */
} dec_mg_opts;
/* Fused cycle kernels.  Gathering a second vector per neighbour:
 *   DEC_FUSE_SMOOTH01  the first two pre-smoothing steps from zero;
 *   DEC_FUSE_RESTRICT  residual with restriction (stencils of at most 7 slots);
 *   DEC_FUSE_PROLONG   interpolation and correction with the first post-smoothing step.
 * Row-local, no extra gathers:
 *   DEC_FUSE_RESTRICT0 restriction with the first smoothing step of the coarse level;
 *   DEC_FUSE_OUTER     in MG-PCG with FP32 cycles (mixed modes): the outer update with the
 *                      first smoothing step of the finest level, and the last post-smoothing
 *                      step with the dot products of the preconditioned vector. */
/*   DEC_FUSE_COARSE    the coarsest levels whose operators fit in one SM's shared memory
 *                      (FP32 V-cycles) run as one 1024-thread block, __syncthreads between
 *                      phases instead of kernel boundaries.
 *   DEC_FUSE_PATCH     halo tiles: on the levels between the coarsest and the finest (binary
 *                      subdivision, V-cycles, Jacobi or Chebyshev, 1 to 3 steps per smoothing
 *                      call) one block per tile runs the pre-smoothing, residual and restriction
 *                      (one launch) and the interpolation, correction and post-smoothing (one
 *                      launch) out of shared memory, recomputing the values of the vertices
 *                      within nu edges of its own.  Takes precedence over the three gathering
 *                      fusions on those levels. */
enum {
    DEC_FUSE_SMOOTH01 = 1, DEC_FUSE_RESTRICT = 2, DEC_FUSE_PROLONG = 4, DEC_FUSE_RESTRICT0 = 8,
    DEC_FUSE_OUTER = 16, DEC_FUSE_COARSE = 32, DEC_FUSE_PATCH = 64, DEC_FUSE_ALL = 127
};

/* Solver options.  dec_solve_default_opts(): MG-PCG, mixed precision,
 * tol = 1e-8, maxit = 100, no warm start, device-side iteration loop. */
typedef struct dec_solve_opts {
    int solver;       /* DEC_SOLVER_*                                           */
    int mode;         /* DEC_MODE_*                                               */
    double tol;       /* stop when ||b - L x||_2 / ||b||_2 <= tol (free vertices) */
    int maxit;        /* outer iterations                                         */
    int warm_start;   /* nonzero: x holds the initial guess on entry              */
    int check_every;  /* with host_loop: host reads the residual every this many iterations */
    int host_loop;    /* 0: the iteration loop runs on the device (one graph with a while
                         node, one host wait per solve); 1: the host relaunches a
                         one-iteration graph and reads the residual in between (same
                         kernels; for tools that cannot see conditional graphs)   */
} dec_solve_opts;

typedef struct dec_stats {
    int iters;        /* outer iterations taken                                  */
    double rel_res;   /* final relative residual (recurrence value for PCG)      */
    double rel_res0;  /* relative residual of the initial guess                  */
    int64_t launches; /* libdec kernels launched by this call (graph nodes included) */
} dec_stats;

typedef struct dec_mg_info_t {
    int nlevels;          /* levels in the hierarchy, 0 = coarsest                */
    int64_t nv[16];       /* vertices per level                                   */
    int64_t ne[16];       /* edges per level                                      */
    int64_t nt[16];       /* triangles per level                                  */
    int ell_width[16];    /* stored stencil slots per vertex per level            */
    double lmax[16];      /* power-iteration lambda_max(D^-1 L) per level         */
    int ncolors[16];      /* greedy colour count per level (multicolour GS)       */
    int bc;               /* DEC_BC_*                                             */
    int dim;              /* coordinate dimension of the vertices (2 or 3)        */
    size_t device_bytes;  /* device memory held by the handle                     */
    int tiles[16];        /* halo tiles per level (DEC_FUSE_PATCH); 0: per-step kernels */
} dec_mg_info_t;

/* What dec_mg_copy_table copies (host output, element type in brackets). */
enum {
    DEC_TABLE_VERTS = 0,   /* [nv * dim] double, vertex coordinates               */
    DEC_TABLE_TRIS = 1,    /* [nt * 3] int32, triangles                           */
    DEC_TABLE_EDGES = 2,   /* [ne * 2] int32, (lo, hi), lexicographic             */
    DEC_TABLE_STAR0 = 3,   /* [nv] double, circumcentric dual areas               */
    DEC_TABLE_STAR1 = 4,   /* [ne] double, dual/primal length ratios (scaled)     */
    DEC_TABLE_FREE = 5,    /* [nv] int32, 1 = unknown, 0 = Dirichlet vertex       */
    DEC_TABLE_PARENTS = 6, /* [ne(level) * 2] int32, coarse edge (a, b) of each new vertex
                              n(level) + k of level+1, k = 0 .. ne(level)-1 (not the finest) */
    DEC_TABLE_COLORS = 7,  /* [nv] int32, greedy colour of each vertex            */
    DEC_TABLE_MAP_IDX = 8, /* [nv(level+1) * 3] int32: the geometric map from level to level+1,
                              three coarse vertices per fine vertex (not the finest)        */
    DEC_TABLE_MAP_W = 9    /* [nv(level+1) * 3] double: their barycentric weights (0 = unused) */
};

/* ---- errors, defaults --------------------------------------------------- */
const char *dec_last_error(void);
void dec_mg_default_opts(dec_mg_opts *opts);
void dec_solve_default_opts(dec_solve_opts *opts);

/* ---- meshes (host only; no GPU needed) ----------------------------------
 * dec_mesh_create: an embedded 2-simplicial complex (Sec. 2.1, Def. of an
 * embedded simplicial complex): nv points of dimension dim (2 or 3, row
 * major [nv * dim]) and nt triangles ([nt * 3] vertex ids).  Edges are
 * enumerated once as (lo, hi), lo < hi, in lexicographic order.
 * Errors: DEC_ERR_ARG for null pointers or sizes out of range (nv, nt >= 1,
 * nv < 2^31); DEC_ERR_MESH for an index out of range, a triangle repeating a
 * vertex, two triangles on the same vertex set, a vertex in no triangle or
 * an edge in more than two triangles.  *out is owned by the caller and
 * released with dec_mesh_destroy. */
int dec_mesh_create(const double *verts, int64_t nv, int dim,
                    const int32_t *tris, int64_t nt, dec_mesh **out);
void dec_mesh_destroy(dec_mesh *mesh);
/* Sizes and coordinate dimension of a mesh.  Any output pointer may be null. */
int dec_mesh_sizes(const dec_mesh *mesh, int64_t *nv, int64_t *ne, int64_t *nt, int *dim);
/* dec_mesh_refine: nsub successive 1->4 midpoint subdivisions (Sec. 2.2.1,
 * binary subdivision) on the host.  Coarse ids are kept, so every level's
 * vertices are a prefix of the finer levels'.  Triangle t = (a,b,c) becomes
 * 4t+0 = (a,m_ab,m_ca), 4t+1 = (m_ab,b,m_bc), 4t+2 = (m_ca,m_bc,c),
 * 4t+3 = (m_ab,m_bc,m_ca).  The new vertices n_coarse .. n_coarse+E-1 are the
 * midpoints of the coarse edges: by default the midpoint of coarse edge e is
 * n_coarse + e, so the midpoints around each coarse vertex are consecutive.
 * With DEC_ORDER_MORTON they are numbered in Z-order of their coordinates
 * instead -- each coordinate quantized on the midpoints' bounding box to B
 * bits (B = 21 in 3-D, 31 in 2-D) as floor((x - lo) * ((2^B - 1)/(hi - lo))),
 * bits interleaved, ties kept in coarse edge order.  (On GB300 the edge order
 * gathered faster; the Z-order is kept as an option.)  flags & DEC_SPHERE_PROJECT pushes each new
 * midpoint to the unit sphere.  With DEC_SUBDIV_CUBIC each step is the
 * cubic 1->9 subdivision instead (Sec. 2.2.1): coarse edge e = (lo, hi) gets
 * n_coarse + 2e at (2 x_lo + x_hi)/3 and n_coarse + 2e + 1 at (x_lo + 2 x_hi)/3,
 * triangle t = (a,b,c) its centroid n_coarse + 2E + t at ((x_a + x_b) + x_c)/3
 * and becomes the nine lattice triangles (a,ab1,ca2), (ab1,ab2,m), (ab2,b,bc1),
 * (ca2,m,ca1), (m,bc1,bc2), (ca1,bc2,c), (ab1,m,ca2), (ab2,bc1,m), (m,bc2,ca1)
 * (xy1 next to x, xy2 next to y, m the centroid), numbered 9t .. 9t+8; not
 * with DEC_ORDER_MORTON.  *out is a new mesh owned by the caller. */
int dec_mesh_refine(const dec_mesh *mesh, int nsub, uint32_t flags, dec_mesh **out);
/* Copy DEC_TABLE_VERTS / TRIS / EDGES / STAR0 / STAR1 of a mesh to host memory.
 * STAR0 and STAR1 are the circumcentric Hodge stars (Sec. 3.1.1). */
int dec_mesh_copy_table(const dec_mesh *mesh, int what, void *host_out);

/* ---- hierarchy ------------------------------------------------------------
 * dec_mg_build: subdivide `base` nsub times and keep the finest nlevels
 * meshes as the multigrid hierarchy (nlevels in 1..min(nsub+1, 16)).  The
 * operator L = *0^-1 d0^T *1 d0 is rediscretized on every level (Sec. 3.1.1,
 * last paragraph).  bc = DEC_BC_DIRICHLET fixes boundary vertices to 0;
 * DEC_BC_GAUGE treats the constants as the nullspace and works with
 * *0-weighted mean-zero vectors.  star1_scale (host, nullable, one value per
 * finest edge) multiplies *1 on the finest level.  opts may be null
 * (defaults).  Builds on the host, then uploads every table to the current
 * CUDA device.  Errors: DEC_ERR_ARG, DEC_ERR_MESH (also: a free vertex whose
 * diagonal is not positive, or a coarsest level above 8192 unknowns),
 * DEC_ERR_CUDA, DEC_ERR_OOM.  Release with dec_mg_destroy. */
int dec_mg_build(const dec_mesh *base, int nsub, int nlevels, int bc, uint32_t flags,
                 const double *star1_scale, const dec_mg_opts *opts, dec_mg **out);
void dec_mg_destroy(dec_mg *mg);
/* dec_mg_build_maps: a hierarchy on caller-given meshes related by
 * caller-given geometric maps, for transfers beyond nested subdivision
 * (Sec. 2.2: a PL map f from the fine mesh to the coarse one and its matrix
 * M(f), whose column j holds the global barycentric coordinates of the image
 * of fine vertex j; Sec. 2.2.1: interpolation is M(f)^T, restriction the
 * transpose of the row-normalized M(f), or the *0-adjoint of interpolation
 * with DEC_RESTRICT_STAR0).  meshes: host array of nlevels mesh handles,
 * coarsest first (level 0), copied.  map_idx[l], map_w[l] (l = 0 ..
 * nlevels-2; host arrays, copied): for each vertex v of level l+1, three
 * vertices of level l at [3v .. 3v+2] and their weights -- the nonzeros of
 * column v of M(f), padded with weight 0 -- the layout of DEC_TABLE_MAP_IDX /
 * DEC_TABLE_MAP_W.  The operator is discretized on every mesh (Sec. 3.1.1,
 * last paragraph); bc and star1_scale (finest edges) as for dec_mg_build;
 * flags: DEC_HOST_ONLY or 0.  Interpolation leaves fixed (Dirichlet) fine
 * vertices at 0.  Errors: DEC_ERR_ARG for a null pointer, an index outside
 * level l, a non-finite weight, a vertex whose weights do not sum to 1
 * (within 1e-9), or a coarse vertex that carries no weight (its restriction
 * row would be empty); the errors of dec_mg_build otherwise.  The cycle runs
 * on the general transfer kernels (as for DEC_SUBDIV_CUBIC). */
int dec_mg_build_maps(const dec_mesh *const *meshes, int nlevels, const int32_t *const *map_idx,
                      const double *const *map_w, int bc, uint32_t flags, const double *star1_scale,
                      const dec_mg_opts *opts, dec_mg **out);
int dec_mg_info(const dec_mg *mg, dec_mg_info_t *info);
/* Copy a host-side table of one level (DEC_TABLE_*) into host_out. */
int dec_mg_copy_table(const dec_mg *mg, int level, int what, void *host_out);

/* dec_mg_set_star1: replace the finest-level *1 (device pointer, [ne] double,
 * unscaled final values) and rebuild the finest operator's weights on the
 * device.  Coarser levels keep their geometric operators. */
int dec_mg_set_star1(dec_mg *mg, const double *star1, dec_stream_t stream);

/* ---- operator --------------------------------------------------------------
 * dec_laplace0_apply: y = L_level x (Sec. 3.1.1, Eq. hodge0-laplacian, as
 * -Delta_0), i.e. y_v = (1 / star0_v) sum_{e=(v,w)} *1_e (x_v - x_w); rows of
 * Dirichlet vertices are 0.  prec = DEC_F64 (double x, y) or DEC_F32 (float
 * x, y, weights rounded to float).  k >= 1: right-hand sides, interleaved
 * ([v * k + j]).  x and y must not overlap. */
int dec_laplace0_apply(const dec_mg *mg, int level, const void *x, void *y, int k,
                       int prec, dec_stream_t stream);
/* dec_residual: r = b - L_level x on free vertices, 0 on Dirichlet vertices;
 * k >= 1 interleaved right-hand sides as for dec_laplace0_apply. */
int dec_residual(const dec_mg *mg, int level, const void *b, const void *x, void *r, int k,
                 int prec, dec_stream_t stream);

/* ---- cycles and solves -------------------------------------------------------
 * dec_mg_vcycle: x <- x + C(b - L x) on the finest level, where C is one
 * multigrid cycle with zero initial guess: pre-smoothing, residual,
 * restriction by the row-normalized transpose of the subdivision matrix,
 * recursion (gamma times), interpolation by the subdivision matrix,
 * post-smoothing (Sec. 2.2.1; Sec. 3.1.1 last paragraph), and a dense
 * direct solve on the coarsest level.  prec as for dec_laplace0_apply.  With
 * k > 1 interleaved right-hand sides every column gets its own cycle, one
 * after the other through contiguous copies (three finest-level vectors
 * allocated on the first such call); the batch (dec_batch_*) advances many
 * right-hand sides together. */
int dec_mg_vcycle(dec_mg *mg, const void *b, void *x, int k, int prec, dec_stream_t stream);

/* dec_mg_vcycle_noalloc: the same FP32 cycle as dec_mg_vcycle(prec =
 * DEC_F32, k = 1), x <- x + C(b - L x), for callers that may not allocate
 * device memory when they run it.  (The paper has no counterpart: this is a
 * deployment variant.)  Such callers include runtimes that reserve all device
 * memory at start-up and forbid later allocation to keep latency and memory
 * footprint predictable, plug-ins whose host application owns every device
 * allocation, and code that runs where cudaMalloc is not allowed or would
 * synchronize the device.  The call allocates nothing: its work vectors live
 * in one file-scope device array of DEC_NOALLOC_SCRATCH_BYTES (32 MiB) that
 * every GPU which loads libdec holds until the process exits.  The handle's
 * tables (built earlier by dec_mg_build) and the caller's b and x (float
 * device vectors of nv(finest) entries, x updated in place) are the inputs
 * and outputs.
 *   - The first call on a device looks up the device address of the array
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls on a device share the array, which keeps the last call's
 *     contents; every vector is written before it is read within a call, so
 *     nothing needs clearing.  Calls whose executions overlap on the GPU (two
 *     streams, two host threads, two handles) race on the array: serialize
 *     them.
 *   - Only V-cycles (gamma = 1); other hierarchies get DEC_ERR_ARG.
 *   - Hierarchies whose six FP32 vectors per level (each rounded up to 256
 *     bytes) need more than DEC_NOALLOC_SCRATCH_BYTES are rejected with
 *     DEC_ERR_ARG; 32 MiB covers a finest level of about one million vertices.
 */
#define DEC_NOALLOC_SCRATCH_BYTES (32u << 20)
int dec_mg_vcycle_noalloc(dec_mg *mg, const float *b, float *x, dec_stream_t stream);

/* dec_solve: solve L x = b on the finest level to ||b - L x||_2/||b||_2 <= tol
 * (Sec. 3.1.2).  Standalone multigrid, or flexible CG in the *0 inner
 * product preconditioned by one cycle (Sec. 3.1.2 cross-comparison), or
 * plain CG.  DEC_MODE_MIXED runs the cycles in FP32 inside the FP64 outer
 * iteration (residuals and updates in FP64); DEC_MODE_MIXED_FF inside a
 * float-float one (see the DEC_MODE_* enum).  b and x are
 * double device vectors of nv(finest) * k entries, interleaved for k > 1; each
 * column is then solved on its own, one after the other (stats: the largest
 * iteration count and residuals; launches summed); the batch
 * (dec_batch_*) solves many right-hand sides together.  Under DEC_BC_GAUGE,
 * b is projected to *0-weighted mean zero and so is x.  Synchronizes
 * `stream` while iterating.  Returns DEC_ERR_NOT_CONVERGED (x holds the last
 * iterate) or DEC_ERR_NONFINITE; stats may be null. */
int dec_solve(dec_mg *mg, const double *b, double *x, int k, const dec_solve_opts *opts,
              dec_stats *stats, dec_stream_t stream);
/* dec_solve_host: dec_solve with b and x in HOST memory (k = 1; nv(finest)
 * doubles each, pinned or pageable; pinned memory lets the copies run as DMA).  b is
 * copied straight into the solver's own right-hand side and the result out
 * of its own iterate (x is read first when opts->warm_start), so the call
 * makes no device copy of either; it returns once x holds the result.  Same
 * options, status codes and gauge handling as dec_solve. */
int dec_solve_host(dec_mg *mg, const double *b, double *x, int k, const dec_solve_opts *opts, dec_stats *stats,
                   dec_stream_t stream);

/* dec_solve_backward: adjoint of x = L^-1 b.  Given u = L^-1 b and
 * grad_u = dJ/du (device, [nv]), solve L mu = *0^-1 grad_u with the same
 * hierarchy (L^T = d0^T *1 d0 *0^-1 = *0 L *0^-1), then
 * grad_b = dJ/db = *0 mu and, if grad_star1 is not null,
 * grad_star1[e] = dJ/d*1_e = -(d0 mu)_e (d0 u)_e on the finest edges. */
int dec_solve_backward(dec_mg *mg, const double *u, const double *grad_u, double *grad_b,
                       double *grad_star1, const dec_solve_opts *opts, dec_stats *stats,
                       dec_stream_t stream);

/* ---- batched solves ------------------------------------------------------------
 * (Not in the paper: solves many right-hand sides on many hierarchies together.)
 * The right-hand sides of every hierarchy -- of all entries that pass the
 * same handle, in entry order -- are split into groups of k (a power of two,
 * kgroup, or the smallest power of two >= their count, at most `block`, when
 * kgroup = 0) whose vectors are interleaved, value j of vertex v at
 * [v*k + j], so a neighbour gather reads k contiguous values and one read of
 * the operator serves the group; every operation of the cycle is one launch
 * over all groups of all meshes.  Solvers (Sec. 3.1.2 with the
 * mixed-precision pattern): FP32 cycles inside an FP64 outer iteration per
 * right-hand side -- flexible MG-PCG in the *0 inner product (FP64 residual,
 * dot products, updates, gauge projection; DEC_SOLVER_MGPCG, the default) or
 * iterative refinement x += C(b - L x) (DEC_SOLVER_MG) -- until every
 * right-hand side has ||b - L x||_2 / ||b||_2 <= tol.  A right-hand side that
 * converged stops moving (step 0) while the others continue.  The loop runs
 * on the device.  Per-right-hand-side sums are formed in a fixed order, so
 * results are bitwise reproducible.  All hierarchies must use the same
 * restriction and live on the current device; the batch uses its own
 * smoother and sweep count (nu1 = nu2 = nu) with each hierarchy's Chebyshev
 * interval and lambda_max.  The hierarchies must outlive the batch and must
 * not be solved concurrently with it. */
typedef struct dec_batch dec_batch;
typedef struct dec_batch_opts {
    int block;    /* threads per block of the batched kernels: 128, 256 or 512 */
    int kgroup;   /* right-hand sides per interleaved group (power of two <= block), 0: per hierarchy */
    int nu;       /* smoothing sweeps before and after the coarse correction, 1..8 */
    int smoother; /* DEC_SMOOTH_JACOBI or DEC_SMOOTH_CHEBYSHEV */
    int solver;   /* DEC_SOLVER_MGPCG (default) or DEC_SOLVER_MG (refinement) */
} dec_batch_opts;
typedef struct dec_batch_stats {
    int iters;          /* outer iterations (MG-PCG) or refinement passes      */
    double max_rel_res; /* largest final relative residual                     */
    int64_t launches;   /* libdec kernels launched by the call                 */
    int64_t dof;        /* finest vertices x right-hand sides over all meshes   */
} dec_batch_stats;
void dec_batch_default_opts(dec_batch_opts *opts);
/* mgs: host array of nmesh hierarchies (an entry may repeat a handle: its
 * right-hand sides join that hierarchy's groups); nrhs: host array of
 * right-hand-side counts.  Allocates the batch's device vectors.  Errors:
 * DEC_ERR_ARG, DEC_ERR_OOM, DEC_ERR_CUDA. */
int dec_batch_create(dec_mg *const *mgs, const int *nrhs, int nmesh, const dec_batch_opts *opts, dec_batch **out);
void dec_batch_destroy(dec_batch *batch);
/* b, x: host arrays of nmesh DEVICE pointers, entry m's vectors being double
 * [nv_finest(m) * nrhs(m)] in [v * nrhs + j] order.  Under DEC_BC_GAUGE each
 * right-hand side is projected to *0-weighted mean zero and so is its
 * solution.  A group whose right-hand sides have all converged stops
 * iterating while the others go on: every group's result is the one it gets
 * solved alone.  Synchronizes `stream`.  Errors as for dec_solve. */
int dec_batch_solve(dec_batch *batch, const double *const *b, double *const *x, double tol, int maxit,
                    dec_batch_stats *stats, dec_stream_t stream);
/* dec_batch_solve_backward: the adjoint of every solve of the batch (as
 * dec_solve_backward, per right-hand side).  Given u = L^-1 b and grad_u =
 * dJ/du (host arrays of nmesh device pointers, layout as for dec_batch_solve),
 * solves L mu = *0^-1 grad_u on the same batch, then writes grad_b = *0 mu
 * and, where grad_star1 (nullable array; nullable entries) gives a device
 * vector of [ne_finest(m) * nrhs(m)] doubles, grad_star1[e * nrhs + j] =
 * -(d0 mu_j)_e (d0 u_j)_e.  Same options, tolerance and errors as
 * dec_batch_solve. */
int dec_batch_solve_backward(dec_batch *batch, const double *const *u, const double *const *grad_u,
                             double *const *grad_b, double *const *grad_star1, double tol, int maxit,
                             dec_batch_stats *stats, dec_stream_t stream);
int dec_batch_info(const dec_batch *batch, int *ngroups, int *total_rhs, int64_t *dof, size_t *device_bytes);
/* dec_batch_tune: the batch autotuner.  For each candidate setting (cands,
 * or when null a grid of block {128,256,512} x kgroup {0,8,16,32} x nu
 * {1,2,3}, Chebyshev, MG-PCG) it builds a batch, solves once to warm up, times
 * `reps` solves of b with CUDA events on `stream`, and keeps the fastest
 * that converges.  times (nullable, one per candidate) receives the mean
 * milliseconds, -1 for a failed candidate.  x receives the last solution. */
int dec_batch_tune(dec_mg *const *mgs, const int *nrhs, int nmesh, const double *const *b, double *const *x,
                   double tol, int maxit, const dec_batch_opts *cands, int ncand, int reps, dec_batch_opts *best,
                   double *best_ms, double *times, dec_stream_t stream);
/* dec_batch_time_smooth: mean duration of one launch of the batched
 * finest-level smoothing sweep (every group), over `reps` back-to-back
 * launches timed with CUDA events on `stream`, and its algorithmic bytes
 * (each hierarchy's finest operator once, however many groups share it --
 * K column indices and K weights per row -- and per right-hand side x, b,
 * the new x and, for Chebyshev, a direction vector; padding columns not
 * counted). */
int dec_batch_time_smooth(dec_batch *batch, int reps, double *avg_ms, double *bytes, dec_stream_t stream);

/* ---- porous convection (Sec. 3.2) -------------------------------------------
 * One explicit step of the DEC porous-convection model of Sec. 3.2.1 with the
 * constants of Sec. 3.2.2, on the finest level of a DEC_BC_GAUGE hierarchy
 * (the pressure problem is pure Neumann):
 *   w   = alpha rho0 (g^flat wedge T),  (g^flat wedge T)_e = g.(x_hi - x_lo) (T_lo + T_hi)/2
 *   L P = *0^-1 d0^T *1 w              (Delta P = delta w; MG-PCG, warm-started from P)
 *   q   = -(k/eta) (d0 P - w)
 *   T  += dt * mask * ( -(1/phi) L_q T - kappa L T ),
 *         (L_q T)_v = (1 / star0_v) sum_{e ni v} (1/2) *1_e (d0 T)_e q_e,
 * mask = 0 where fixed[v] != 0 (the bc operation of Sec. 3.2.1: top and
 * bottom rows).  dec_porous_default_params: g = (0, -9.81, 0),
 * alpha_rho0 = 1/|g|, phi = 0.1, k_eta = 1, kappa = 2 (= Ra^-1 g alpha rho0
 * k_eta dT y_max / phi with Ra = 1000, dT = 200, y_max = 1), tol = 1e-8,
 * mixed precision, maxit = 100; dt must be set by the caller (> 0). */
typedef struct dec_porous_params {
    double g[3];       /* gravity; the first dim components are used                */
    double alpha_rho0; /* alpha * rho0; <= 0 selects 1/|g|                          */
    double phi;        /* porosity                                                   */
    double k_eta;      /* permeability / viscosity                                   */
    double kappa;      /* thermal diffusivity lambda / (rho0 c_p)                    */
    double dt;         /* forward-Euler time step                                    */
    double tol;        /* relative-residual tolerance of every pressure solve        */
    int mode;          /* DEC_MODE_* of the pressure solves                           */
    int maxit;         /* MG-PCG iterations per pressure solve                       */
} dec_porous_params;
void dec_porous_default_params(dec_porous_params *prm);

/* dec_porous_step: nsteps steps in place.  T, P: double device vectors
 * [nv(finest)] (P is the warm start on entry and the last pressure on exit);
 * fixed: uint8 device mask [nv].  checkpoints (nullable, device): receives T
 * before steps 0, ckpt_every, 2 ckpt_every, ... and after the last step when
 * nsteps is a multiple of ckpt_every: [(nsteps / ckpt_every + 1) * nv].
 * stats (nullable): iters = pressure iterations summed over the steps,
 * rel_res = the largest final pressure residual.  Errors: DEC_ERR_ARG (not a
 * gauge hierarchy, dt <= 0, null pointers), and the errors of dec_solve.
 * Synchronizes `stream`. */
int dec_porous_step(dec_mg *mg, double *T, double *P, const uint8_t *fixed, const dec_porous_params *prm,
                    int nsteps, double *checkpoints, int ckpt_every, dec_stats *stats, dec_stream_t stream);

/* dec_porous_rk: adaptive explicit integration of the same model from t = 0
 * to t_end, in place: Tsitouras' 5(4) Runge-Kutta pair, the "Tsit5" method
 * of Sec. 3.2.2.  Seven stages, the last evaluated at the new state and
 * reused as the next step's first, so a step costs six right-hand sides,
 * each an MG-PCG pressure solve warm-started from P.  Error norm: the root
 * mean square over all vertices of err_v / (atol + rtol max(|T_v|, |T_new_v|));
 * a step is accepted when it is <= 1; the next step is dt * min(10, max(0.2,
 * 0.9 norm^(-1/5))), at most dt right after a rejection; the last step ends
 * exactly at t_end.  dt0: first step (fixed_step != 0: every step, no error
 * control).  P: warm start on entry.  On every return, also an error
 * return, T is the last accepted state (the state at stats->t) and P its
 * pressure (P is unchanged when the first pressure solve fails); a
 * rejected or failed step leaves neither.  prm as for dec_porous_step,
 * prm->dt ignored.  stats (nullable): accepted and rejected steps,
 * right-hand-side evaluations, the time reached, the next step, pressure
 * iterations summed and the worst final pressure residual.  Errors:
 * DEC_ERR_ARG; DEC_ERR_NOT_CONVERGED when max_steps attempts end before
 * t_end; DEC_ERR_NONFINITE; the errors of dec_solve.  Allocates 10 work
 * vectors for the call.  Synchronizes `stream` once per step. */
typedef struct dec_rk_stats {
    int64_t naccept, nreject, nfev;
    double t, dt;
    int64_t pressure_iters;
    double pressure_rel_res;
} dec_rk_stats;
int dec_porous_rk(dec_mg *mg, double *T, double *P, const uint8_t *fixed, const dec_porous_params *prm,
                  double t_end, double dt0, double rtol, double atol, int64_t max_steps, int fixed_step,
                  dec_rk_stats *stats, dec_stream_t stream);

/* dec_porous_backward: reverse-mode derivative of T_N = step^N(T_0):
 * given grad_TN = dF/dT_N, writes grad_T0 = dF/dT_0.  Checkpoints every
 * ckpt_every steps are kept on the device and each segment is recomputed
 * forward before it is differentiated (memory: (nsteps/ckpt_every + 2 *
 * ckpt_every + 8) vectors, allocated inside this call).  Each adjoint step
 * costs one adjoint pressure solve on the same hierarchy.  Arguments as for
 * dec_porous_step; T0 and P0 are not modified. */
int dec_porous_backward(dec_mg *mg, const double *T0, const double *P0, const uint8_t *fixed,
                        const dec_porous_params *prm, int nsteps, int ckpt_every, const double *grad_TN,
                        double *grad_T0, dec_stats *stats, dec_stream_t stream);

/* dec_mg_set_wait_limit: the bound on the one device-side wait of the
 * cycle -- the shared-memory coarse cycle (DEC_FUSE_COARSE) waits on an
 * mbarrier for the bulk copies of its tables.  After `rounds` try_wait rounds
 * without completion the block records the failure, waits for the copies
 * in flight with the default bound so that none lands after it exits, and
 * returns without touching its output; every later kernel of the solve is
 * skipped and dec_solve returns DEC_ERR_CUDA ("a device-side wait gave
 * up"), x holding the iterate from before the failed cycle.  rounds < 0
 * restores the default (2^20 rounds, well under a second); larger values are
 * clamped to it; 0 makes the wait give up at once, which exercises the
 * failure path without a fault.  Applies to later calls (captured solve
 * graphs are rebuilt).  Not in the paper. */
int dec_mg_set_wait_limit(dec_mg *mg, int rounds);

/* ---- live kernel timing ------------------------------------------------------
 * dec_mg_profile: enable = 1 records a CUDA event pair around every launch of
 * the finest level inside the repeated part of dec_solve (the captured
 * iteration), enable = 2 around the launches of every level, 0 turns it off.
 * Events are recorded on the solve's stream, so each pair brackets exactly one
 * kernel.  Enabling clears the counters.  While enabled, dec_solve reads the
 * events after every iteration (check_every is treated as 1); the iteration
 * in which the solve converges is not counted.
 * dec_mg_profile_read copies up to `max` non-empty (kind, level) totals. */
enum {
    DEC_PK_SMOOTH0 = 0, /* first smoothing step from zero                     */
    DEC_PK_SMOOTH,      /* smoothing step                                      */
    DEC_PK_RESIDUAL,    /* residual inside the cycle                           */
    DEC_PK_RESTRICT,    /* restriction (launched on the fine level)            */
    DEC_PK_PROLONG,     /* interpolation and correction                        */
    DEC_PK_COARSE,      /* coarsest-level dense solve                          */
    DEC_PK_SPMV64,      /* outer FP64 operator apply with <p, Lp>              */
    DEC_PK_UPDATE,      /* outer x, r update with ||r||                        */
    DEC_PK_ZDOTS,       /* outer preconditioned-vector dot products            */
    DEC_PK_PUPD,        /* outer search-direction update                       */
    DEC_PK_MGRES,       /* standalone-MG residual with ||r||                   */
    DEC_PK_ADD,         /* standalone-MG correction                            */
    DEC_PK_AUX,         /* set-up kernels of a solve (gauge mean, initial residual) */
    DEC_PK_SMOOTH01,    /* fused first two smoothing steps from zero           */
    DEC_PK_RESRESTRICT, /* fused residual and restriction (launched on the fine level) */
    DEC_PK_PROLSMOOTH,  /* fused interpolation, correction and first post-smoothing step */
    DEC_PK_SMOOTHDOTS,  /* fused last post-smoothing step and preconditioned-vector dot products */
    DEC_PK_COARSECYCLE, /* the coarsest levels' whole sub-cycle in one block (launched on its top level) */
    DEC_PK_PATCHDOWN,   /* halo tiles: pre-smoothing, residual and restriction of one level */
    DEC_PK_PATCHUP,     /* halo tiles: interpolation, correction and post-smoothing of one level */
    DEC_PK_COUNT
};
typedef struct dec_prof_entry {
    int kind;          /* DEC_PK_*                                   */
    int level;         /* hierarchy level of the launch              */
    int64_t launches;  /* launches timed                             */
    double total_ms;   /* summed event-to-event time                 */
    int64_t rows;      /* vertices of that level (units per launch)  */
} dec_prof_entry;
int dec_mg_profile(dec_mg *mg, int enable);
int dec_mg_profile_read(const dec_mg *mg, dec_prof_entry *out, int max, int *count);
/* dec_mg_time_smooth: mean duration of one FP32 smoothing sweep on `level`
 * (1 .. nlevels-1, or negative from the finest), the same kernel and launch
 * configuration as the last step of a smoothing call inside the cycle, over
 * `reps` back-to-back launches timed with CUDA events on `stream` (no events
 * between launches), and its algorithmic bytes per launch (per row K column
 * indices and K weights, x_i, b_i, the new x_i and, for Chebyshev, the
 * direction).  Overwrites that level's FP32 cycle work vectors with zeros
 * first (a timing call, not a computation). */
int dec_mg_time_smooth(dec_mg *mg, int level, int reps, double *avg_ms, double *bytes, dec_stream_t stream);
/* dec_mg_time_kernel: the same for other finest-level kernels of the mixed_ff
 * MG-PCG loop -- kind DEC_PK_SMOOTH (as dec_mg_time_smooth, any level),
 * DEC_PK_SMOOTHDOTS (last smoothing step fused with the dot products),
 * DEC_PK_SPMV64 (float-float q = L p) or DEC_PK_UPDATE (float-float x, r
 * update) -- on zeroed FP32 work vectors, with their algorithmic bytes per
 * launch; overwrites the finest level's work vectors and the solver's
 * scalar block (a timing call, not a computation). */
int dec_mg_time_kernel(dec_mg *mg, int kind, int level, int reps, double *avg_ms, double *bytes, dec_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* DEC_H */
