// extern "C" entry points that need no GPU: errors, defaults, meshes.
#include <cstring>
#include <new>

#include "host.h"

struct dec_mesh {
    decimpl::HostMesh m;
};

namespace decimpl {
static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
}  // namespace decimpl

using decimpl::Status;

static int fail(const Status &s) {
    decimpl::set_error(s.msg);
    return s.code;
}

extern "C" {

const char *dec_last_error(void) { return decimpl::g_err.c_str(); }

void dec_mg_default_opts(dec_mg_opts *o) {
    if (!o) return;
    o->smoother = DEC_SMOOTH_JACOBI;
    o->nu1 = 2;
    o->nu2 = 2;
    o->omega = 2.0 / 3.0;
    o->cheby_lo = 0.3;
    o->cheby_hi = 1.1;
    o->power_iters = 10;
    o->gamma = 1;
    o->restriction = DEC_RESTRICT_ROWNORM;
    o->fcycle = 0;
    o->fuse = DEC_FUSE_RESTRICT0 | DEC_FUSE_OUTER | DEC_FUSE_COARSE | DEC_FUSE_PATCH;
    o->coarse_max_rows = 0;
    o->fuse_max_rows = 0;
    o->patch_max_rows = 0;
    o->patch_chunk = 0;
    o->patch_threads = 0;
}

void dec_solve_default_opts(dec_solve_opts *o) {
    if (!o) return;
    o->solver = DEC_SOLVER_MGPCG;
    o->mode = DEC_MODE_MIXED;
    o->tol = 1e-8;
    o->maxit = 100;
    o->warm_start = 0;
    o->check_every = 1;
    o->host_loop = 0;
}

int dec_mesh_create(const double *verts, int64_t nv, int dim, const int32_t *tris, int64_t nt, dec_mesh **out) {
    if (!verts || !tris || !out) return fail(Status::fail(DEC_ERR_ARG, "null pointer"));
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(Status::fail(DEC_ERR_ARG, "dim must be 2 or 3"));
    if (nv < 1 || nt < 1 || nv >= ((int64_t)1 << 31) || nt >= ((int64_t)1 << 29))
        return fail(Status::fail(DEC_ERR_ARG, "nv or nt out of range"));
    dec_mesh *m = new (std::nothrow) dec_mesh;
    if (!m) return fail(Status::fail(DEC_ERR_OOM, "host allocation"));
    try {
        std::vector<double> v(verts, verts + nv * dim);
        std::vector<int32_t> t(tris, tris + nt * 3);
        Status s = decimpl::build_mesh(std::move(v), dim, std::move(t), m->m);
        if (!s.good()) {
            delete m;
            return fail(s);
        }
    } catch (const std::bad_alloc &) {
        delete m;
        return fail(Status::fail(DEC_ERR_OOM, "host allocation"));
    }
    *out = m;
    return DEC_OK;
}

void dec_mesh_destroy(dec_mesh *mesh) { delete mesh; }

int dec_mesh_sizes(const dec_mesh *mesh, int64_t *nv, int64_t *ne, int64_t *nt, int *dim) {
    if (!mesh) return fail(Status::fail(DEC_ERR_ARG, "null mesh"));
    if (dim) *dim = mesh->m.dim;
    if (nv) *nv = mesh->m.nv;
    if (ne) *ne = mesh->m.ne;
    if (nt) *nt = mesh->m.nt;
    return DEC_OK;
}

int dec_mesh_refine(const dec_mesh *mesh, int nsub, uint32_t flags, dec_mesh **out) {
    if (!mesh || !out) return fail(Status::fail(DEC_ERR_ARG, "null pointer"));
    *out = nullptr;
    if (nsub < 0 || nsub > 14) return fail(Status::fail(DEC_ERR_ARG, "nsub out of range"));
    dec_mesh *m = new (std::nothrow) dec_mesh;
    if (!m) return fail(Status::fail(DEC_ERR_OOM, "host allocation"));
    try {
        m->m = mesh->m;
        for (int i = 0; i < nsub; ++i) {
            decimpl::HostMesh f;
            Status s;
            if (flags & DEC_SUBDIV_CUBIC) {
                if (flags & DEC_ORDER_MORTON) return fail(Status::fail(DEC_ERR_ARG, "cubic subdivision keeps the edge order"));
                std::vector<int32_t> mi;
                std::vector<double> mw;
                s = decimpl::subdivide_cubic(m->m, (flags & DEC_SPHERE_PROJECT) != 0, f, mi, mw);
            } else {
                s = decimpl::subdivide(m->m, (flags & DEC_SPHERE_PROJECT) != 0, (flags & DEC_ORDER_MORTON) != 0, f);
            }
            if (!s.good()) {
                delete m;
                return fail(s);
            }
            m->m = std::move(f);
        }
    } catch (const std::bad_alloc &) {
        delete m;
        return fail(Status::fail(DEC_ERR_OOM, "host allocation"));
    }
    *out = m;
    return DEC_OK;
}

int dec_mesh_copy_table(const dec_mesh *mesh, int what, void *host_out) {
    if (!mesh || !host_out) return fail(Status::fail(DEC_ERR_ARG, "null pointer"));
    const decimpl::HostMesh &m = mesh->m;
    switch (what) {
        case DEC_TABLE_VERTS:
            std::memcpy(host_out, m.verts.data(), m.verts.size() * sizeof(double));
            return DEC_OK;
        case DEC_TABLE_TRIS:
            std::memcpy(host_out, m.tris.data(), m.tris.size() * sizeof(int32_t));
            return DEC_OK;
        case DEC_TABLE_EDGES:
            std::memcpy(host_out, m.edges.data(), m.edges.size() * sizeof(int32_t));
            return DEC_OK;
        case DEC_TABLE_STAR0:
        case DEC_TABLE_STAR1: {
            std::vector<double> s0, s1;
            decimpl::hodge_stars(m, s0, s1);
            const std::vector<double> &s = what == DEC_TABLE_STAR0 ? s0 : s1;
            std::memcpy(host_out, s.data(), s.size() * sizeof(double));
            return DEC_OK;
        }
        default:
            return fail(Status::fail(DEC_ERR_ARG, "table not available for a mesh"));
    }
}

}  // extern "C"

// accessor for the device-side translation unit
const decimpl::HostMesh *dec_mesh_host(const dec_mesh *m) { return m ? &m->m : nullptr; }
