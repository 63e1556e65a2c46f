// C ABI of libdvm (declared in include/dvm.h): context, state checks, device
// memory, host<->device transfers and the step loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/dvm.h"
#include "hs.hpp"
#include "kernels.hpp"
#include "lbm.hpp"
#include "learned.hpp"
#include "mesh.hpp"
#include "partition.hpp"
#include "mlp.hpp"

struct dvm_ctx {
    dvm_config cfg{};
    std::string err;
    cudaStream_t stream = nullptr;
    void *(*alloc_fn)(size_t, void *) = nullptr;
    void (*free_fn)(void *, void *) = nullptr;
    void *alloc_user = nullptr;
    int state = 0;  // 0 created, 1 mesh, 2 velocity grid, 3 f set
    dvm::Mesh mesh;
    // velocity grid
    int n[3] = {0, 0, 0}, half[3] = {0, 0, 0};
    int nv = 0, P = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, hv[3] = {0, 0, 0}, dV = 0;
    std::vector<double> xi;
    double amag[96] = {0};
    float amag_f[96] = {0};
    double fs_rho = 1.0, fs_u[3] = {0, 0, 0}, fs_T = 1.0;
    // device
    void *d_f[2] = {nullptr, nullptr};
    int cur = 0;
    size_t f_elems = 0;
    int32_t *d_src = nullptr;
    void *d_w = nullptr;
    uint8_t *d_cnt = nullptr;
    void *d_invh = nullptr;
    double *d_amag = nullptr;
    float *d_amag_f = nullptr;
    double *d_xi = nullptr;
    double *d_mom = nullptr;     // step moments [ncells][5]
    double *d_mom2 = nullptr;    // moments of stored f
    // conservation residual of the last step's collision term, [ncells][5]:
    // FP64 sums in psi = (1, xi, |xi|^2) of q (hard sphere, learned), or
    // double-float pairs of the centred-basis moments of M~ - f* (BGK)
    double *d_res = nullptr;
    bool have_res = false;
    bool res_pairs = false;
    // phase timing of dvm_step (dvm_set_timing): events and running totals
    bool timing = false;
    cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};
    double tms[3] = {0.0, 0.0, 0.0};
    int64_t tsteps = 0;
    int *d_status = nullptr;
    unsigned long long *d_counter = nullptr;
    bool have_step_moments = false;
    bool mesh_on_device = false;
    dvm::HsTables hs;
    dvm::Mlp mlp;
    bool mlp_set = false;
    // learned collision: Knudsen threshold, sensor stencil and per-cell buffers
    double kn_thr = 0.0;
    bool learned_cfg = false;
    int64_t l_cells = 0;            // cells the buffers below hold (0: not allocated)
    int32_t *d_kn_start = nullptr, *d_kn_nb = nullptr;
    double *d_kn_coef = nullptr;
    double *d_knl = nullptr;        // local Kn per cell
    float *d_la = nullptr;          // network input a [ncells][64]
    float *d_lo = nullptr;          // network output o [ncells][64]
    int32_t *d_used = nullptr;      // 1 where the learned term was applied
    int32_t *d_list = nullptr;      // cells left to the hard-sphere operator
    int *d_lcount = nullptr;        // their number
    // lattice Boltzmann (dvm_lbm_*): velocity set, f as [q][ld] in two
    // buffers (column ncells the inflow ghost), upwind codes
    dvm::LbmLattice lat;
    int lbm_state = 0;              // 0 no lattice, 1 lattice set, 2 f set
    int64_t lbm_ld = 0, lbm_novf = 0;
    void *d_lf[2] = {nullptr, nullptr};
    int lcur = 0;
    uint32_t *d_lcodes = nullptr, *d_lovf = nullptr;
    uint8_t *d_llev = nullptr;
    double *d_lmom = nullptr;
    int *d_lstatus = nullptr;
    double l_rho = 1.0, l_u[3] = {0, 0, 0};
    // local-Kn sensor outside the learned collision (dvm_kn_local)
    int64_t ks_cells = 0;
    int32_t *d_ks_start = nullptr, *d_ks_nb = nullptr;
    double *d_ks_coef = nullptr, *d_ks_knl = nullptr;
};

namespace {

int fail(dvm_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

size_t elem_size(int prec) { return prec == DVM_F64 ? 8 : prec == DVM_F32 ? 4 : 2; }
size_t tc_size(int prec) { return prec == DVM_F64 ? 8 : 4; }

void *dev_alloc(dvm_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (c->alloc_fn) return c->alloc_fn(bytes, c->alloc_user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(dvm_ctx *c, void *&p)
{
    if (!p) return;
    if (c->free_fn) c->free_fn(p, c->alloc_user);
    else cudaFree(p);
    p = nullptr;
}

template <typename T> T *dev_alloc_t(dvm_ctx *c, size_t count)
{
    return static_cast<T *>(dev_alloc(c, count * sizeof(T)));
}

int cuda_check(dvm_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return DVM_OK;
    return fail(c, DVM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void free_learned_buffers(dvm_ctx *c)
{
    dev_free(c, reinterpret_cast<void *&>(c->d_kn_start));
    dev_free(c, reinterpret_cast<void *&>(c->d_kn_nb));
    dev_free(c, reinterpret_cast<void *&>(c->d_kn_coef));
    dev_free(c, reinterpret_cast<void *&>(c->d_knl));
    dev_free(c, reinterpret_cast<void *&>(c->d_la));
    dev_free(c, reinterpret_cast<void *&>(c->d_lo));
    dev_free(c, reinterpret_cast<void *&>(c->d_used));
    dev_free(c, reinterpret_cast<void *&>(c->d_list));
    dev_free(c, reinterpret_cast<void *&>(c->d_lcount));
    c->l_cells = 0;
}

void free_mesh_buffers(dvm_ctx *c)
{
    free_learned_buffers(c);
    dev_free(c, reinterpret_cast<void *&>(c->d_ks_start));
    dev_free(c, reinterpret_cast<void *&>(c->d_ks_nb));
    dev_free(c, reinterpret_cast<void *&>(c->d_ks_coef));
    dev_free(c, reinterpret_cast<void *&>(c->d_ks_knl));
    c->ks_cells = 0;
    dev_free(c, reinterpret_cast<void *&>(c->d_src));
    dev_free(c, c->d_w);
    dev_free(c, reinterpret_cast<void *&>(c->d_cnt));
    dev_free(c, c->d_invh);
}

void free_grid_buffers(dvm_ctx *c)
{
    dev_free(c, c->d_f[0]);
    dev_free(c, c->d_f[1]);
    dev_free(c, reinterpret_cast<void *&>(c->d_amag));
    dev_free(c, reinterpret_cast<void *&>(c->d_amag_f));
    dev_free(c, reinterpret_cast<void *&>(c->d_xi));
    dev_free(c, reinterpret_cast<void *&>(c->d_mom));
    dev_free(c, reinterpret_cast<void *&>(c->d_mom2));
    dev_free(c, reinterpret_cast<void *&>(c->d_res));
    c->f_elems = 0;
    c->have_step_moments = false;
    c->have_res = false;
}

int64_t ncells_of(const dvm_ctx *c) { return (int64_t)c->mesh.leaf_of_cell.size(); }

void free_lbm_buffers(dvm_ctx *c)
{
    dev_free(c, c->d_lf[0]);
    dev_free(c, c->d_lf[1]);
    dev_free(c, reinterpret_cast<void *&>(c->d_lcodes));
    dev_free(c, reinterpret_cast<void *&>(c->d_lovf));
    dev_free(c, reinterpret_cast<void *&>(c->d_llev));
    dev_free(c, reinterpret_cast<void *&>(c->d_lmom));
    dev_free(c, reinterpret_cast<void *&>(c->d_lstatus));
    c->lbm_state = 0;
    c->lbm_ld = c->lbm_novf = 0;
}

// The mesh is host work; the device is first touched by set_velocity_grid.
int ensure_device(dvm_ctx *c)
{
    if (c->d_status) return DVM_OK;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(c, DVM_ECUDA, "no CUDA device available");
    }
    if (cudaMalloc(&c->d_status, 16) != cudaSuccess || cudaMemset(c->d_status, 0, 16) != cudaSuccess) {
        cudaGetLastError();
        c->d_status = nullptr;
        return fail(c, DVM_ECUDA, "device status word allocation failed");
    }
    // the step kernel's cell dispenser shares the allocation
    c->d_counter = reinterpret_cast<unsigned long long *>(c->d_status + 2);
    return DVM_OK;
}

int upload_mesh(dvm_ctx *c)
{
    free_mesh_buffers(c);
    const dvm::Mesh &m = c->mesh;
    const int64_t nc = ncells_of(c);
    const size_t tcs = tc_size(c->cfg.precision);
    c->d_src = dev_alloc_t<int32_t>(c, nc * 24);
    c->d_w = dev_alloc(c, nc * 24 * tcs);
    c->d_cnt = dev_alloc_t<uint8_t>(c, nc * 8);
    c->d_invh = dev_alloc(c, nc * tcs);
    if (!c->d_src || !c->d_w || !c->d_cnt || !c->d_invh) return fail(c, DVM_ENOMEM, "device allocation (stencils)");
    std::vector<double> invh(nc);
    for (int64_t q = 0; q < nc; q++) invh[q] = std::ldexp(1.0, m.leaves[m.leaf_of_cell[q]].lev);
    // Device encoding of a stencil source: the cell to read (bits 0-27) and
    // the sign-group flip applied to the group index (bits 28-30).
    std::vector<int32_t> enc;
    dvm::encode_stencils(m.st_src, nc, enc);
    if (nc >= (1 << 28)) return fail(c, DVM_ENOTIMPL, "more than 2^28 cells");
    int rc = cuda_check(c, cudaMemcpy(c->d_src, enc.data(), nc * 24 * sizeof(int32_t), cudaMemcpyHostToDevice), "copy stencils");
    if (rc) return rc;
    rc = cuda_check(c, cudaMemcpy(c->d_cnt, m.st_cnt.data(), nc * 8, cudaMemcpyHostToDevice), "copy stencil counts");
    if (rc) return rc;
    if (c->cfg.precision == DVM_F64) {
        rc = cuda_check(c, cudaMemcpy(c->d_w, m.st_w.data(), nc * 24 * 8, cudaMemcpyHostToDevice), "copy weights");
        if (rc) return rc;
        rc = cuda_check(c, cudaMemcpy(c->d_invh, invh.data(), nc * 8, cudaMemcpyHostToDevice), "copy 1/h");
    } else {
        std::vector<float> w(m.st_w.begin(), m.st_w.end()), ih(invh.begin(), invh.end());
        rc = cuda_check(c, cudaMemcpy(c->d_w, w.data(), nc * 24 * 4, cudaMemcpyHostToDevice), "copy weights");
        if (rc) return rc;
        rc = cuda_check(c, cudaMemcpy(c->d_invh, ih.data(), nc * 4, cudaMemcpyHostToDevice), "copy 1/h");
    }
    return rc;
}

double maxwellian(double rho, const double u[3], double T, const double *x)
{
    double d2 = 0.0;
    for (int d = 0; d < 3; d++) d2 += (x[d] - u[d]) * (x[d] - u[d]);
    const double tp = 2.0 * M_PI * T;
    return rho / (tp * std::sqrt(tp)) * std::exp(-d2 / (2.0 * T));
}

// The inflow ghost: one extra cell after the last one in both f buffers,
// holding the freestream Maxwellian sampled at the nodes (FP64, rounded to
// the storage precision).  Steps read it and never write it.
int upload_freestream(dvm_ctx *c)
{
    if (!c->d_f[0]) return DVM_OK;
    std::vector<double> m(c->nv);
    for (int v = 0; v < c->nv; v++) m[v] = maxwellian(c->fs_rho, c->fs_u, c->fs_T, &c->xi[3 * v]);
    double *stage = nullptr;
    if (cudaMalloc(&stage, c->nv * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, DVM_ENOMEM, "device allocation (freestream)");
    }
    int rc = cuda_check(c, cudaMemcpy(stage, m.data(), c->nv * 8, cudaMemcpyHostToDevice), "copy freestream");
    const size_t es = elem_size(c->cfg.precision);
    for (int b = 0; b < 2 && !rc; b++)
        rc = dvm::launch_from_f64(c->cfg.precision, stage, static_cast<char *>(c->d_f[b]) + c->f_elems * es,
                                  c->nv, c->stream);
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "freestream");
    cudaFree(stage);
    return rc;
}

// Buffers of the learned collision for the current mesh, the sensor
// stencil, and network work space for one row per cell.
int learned_prepare(dvm_ctx *c)
{
    const int64_t nc = ncells_of(c);
    if (!dvm::learned_grid_supported(c->n))
        return fail(c, DVM_ENOTIMPL, "velocity grid not supported by the learned kernels (n <= 32 even, n_z/2 % 4 == 0)");
    if (c->cfg.precision != DVM_F32) return fail(c, DVM_ENOTIMPL, "the learned collision needs FP32 storage");
    if (c->l_cells != nc) {
        free_learned_buffers(c);
        dvm::KnStencil ks;
        dvm::build_kn_stencil(c->mesh, ks);
        const size_t ne = ks.nb.size();
        c->d_kn_start = dev_alloc_t<int32_t>(c, (size_t)nc + 1);
        c->d_kn_nb = dev_alloc_t<int32_t>(c, ne);
        c->d_kn_coef = dev_alloc_t<double>(c, 3 * ne);
        c->d_knl = dev_alloc_t<double>(c, (size_t)nc);
        c->d_la = dev_alloc_t<float>(c, (size_t)nc * 128);  // a, then a of the cells' Maxwellians
        c->d_lo = dev_alloc_t<float>(c, (size_t)nc * 128);  // the network at both
        c->d_used = dev_alloc_t<int32_t>(c, (size_t)nc);
        c->d_list = dev_alloc_t<int32_t>(c, (size_t)nc);
        c->d_lcount = dev_alloc_t<int>(c, 4);
        if (!c->d_kn_start || !c->d_kn_nb || !c->d_kn_coef || !c->d_knl || !c->d_la || !c->d_lo || !c->d_used ||
            !c->d_list || !c->d_lcount) {
            free_learned_buffers(c);
            return fail(c, DVM_ENOMEM, "device allocation (learned collision)");
        }
        int rc = cuda_check(c, cudaMemcpy(c->d_kn_start, ks.start.data(), ks.start.size() * 4, cudaMemcpyHostToDevice), "copy sensor stencil");
        if (!rc && ne) rc = cuda_check(c, cudaMemcpy(c->d_kn_nb, ks.nb.data(), ne * 4, cudaMemcpyHostToDevice), "copy sensor stencil");
        if (!rc && ne) rc = cuda_check(c, cudaMemcpy(c->d_kn_coef, ks.coef.data(), ne * 24, cudaMemcpyHostToDevice), "copy sensor stencil");
        if (rc) {
            free_learned_buffers(c);
            return rc;
        }
        c->l_cells = nc;
    }
    int rc = DVM_OK;
    if (c->mlp_set) {
        rc = dvm::mlp_reserve(c->mlp, 2 * nc, [c](size_t b) { return dev_alloc(c, b); }, [c](void *p) { void *q = p; dev_free(c, q); });
        if (rc) return fail(c, rc, "device allocation (network work buffers)");
    }
    rc = dvm::hs_prepare(c->hs, nc, [c](size_t b) { return dev_alloc(c, b); }, [c](void *q) { void *r = q; dev_free(c, r); });
    return rc ? fail(c, rc, "hard-sphere scratch allocation failed") : DVM_OK;
}

dvm::StepParams collision_params(dvm_ctx *c, double *mom)
{
    dvm::StepParams p{};
    p.dim = c->mesh.spec.dim;
    p.prec = c->cfg.precision;
    p.ncells = ncells_of(c);
    p.nv = c->nv;
    p.P = c->P;
    p.mom_out = mom;
    p.dV = c->dV;
    p.status = c->d_status;
    p.stream = c->stream;
    return p;
}

// Learned collision update of f (FP32, [ncells][nv]) whose moments are mom:
// sensor, projection, network (or the given device o), application with the
// checks, then the hard-sphere operator on the cells left over.
int learned_collide_device(dvm_ctx *c, float *f, double *mom, double dt, const float *o_in, float *q_out,
                           cudaEvent_t mid = nullptr)
{
    const int64_t nc = ncells_of(c);
    int rc = dvm::launch_kn_local(mom, c->d_kn_start, c->d_kn_nb, c->d_kn_coef, nc, c->cfg.kn, c->d_knl, c->stream);
    if (!rc) rc = cuda_check(c, cudaMemsetAsync(c->d_lcount, 0, sizeof(int), c->stream), "reset fallback count");
    if (rc) return rc;
    const float *o = o_in, *o_eq = nullptr;
    if (!o) {
        // the network on a and on the projection of each cell's Maxwellian
        rc = dvm::launch_hermite_project(f, mom, c->d_amag, nc, c->n, c->dV, 0, nullptr, nullptr, c->d_la,
                                         c->d_la + (size_t)nc * 64, c->d_status, c->stream);
        if (!rc) rc = dvm::mlp_forward(c->mlp, c->d_la, 2 * nc, c->d_lo, c->d_status, c->stream);
        if (rc) return fail(c, rc, "projection or network launch failed");
        o = c->d_lo;
        o_eq = c->d_lo + (size_t)nc * 64;
    }
    rc = dvm::launch_learned_apply(f, mom, o, o_eq, c->d_knl, c->kn_thr, c->d_amag, nc, c->n, dt / c->cfg.kn, c->d_used,
                                   c->d_list, c->d_lcount, q_out, c->dV, c->d_res, c->d_status, c->stream);
    if (rc) return fail(c, rc, "learned collision launch failed");
    if (mid) cudaEventRecord(mid, c->stream);
    dvm::StepParams p = collision_params(c, mom);
    p.res_out = c->d_res;  // the cells left to the hard-sphere operator
    rc = dvm::launch_hs_general(c->hs, p, f, c->d_list, c->d_lcount, nullptr, c->cfg.kn, dt);
    return rc ? fail(c, rc, "hard-sphere fallback launch failed") : DVM_OK;
}

int read_status(dvm_ctx *c, const char *what)
{
    int st = 0;
    int rc = cuda_check(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read status");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), what);
    if (rc) return rc;
    if (!st) return DVM_OK;
    cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
    if (st & dvm::ST_TIMEOUT) return fail(c, DVM_ETIMEOUT, "a bounded wait for an asynchronous tile copy gave up");
    std::string why;
    if (st & dvm::ST_NONPOS) why += " non-positive density or temperature;";
    if (st & dvm::ST_SINGULAR) why += " singular correction system;";
    if (st & dvm::ST_NUDT) why += " relaxation factor above 1 (dt too large for Kn);";
    return fail(c, DVM_EUNSTABLE, std::string("unstable ") + what + ":" + why);
}

}  // namespace

extern "C" {

int dvm_create(dvm_ctx **out, const dvm_config *cfg)
{
    if (!out || !cfg) return DVM_EINVAL;
    *out = nullptr;
    if (cfg->precision < DVM_F64 || cfg->precision > DVM_BF16) return DVM_EINVAL;
    if (cfg->collision < DVM_COLL_NONE || cfg->collision > DVM_COLL_BGK_ENTROPIC) return DVM_EINVAL;
    if (cfg->collision != DVM_COLL_NONE && !(cfg->kn > 0.0)) return DVM_EINVAL;
    dvm_ctx *c = new (std::nothrow) dvm_ctx();
    if (!c) return DVM_ENOMEM;
    c->cfg = *cfg;
    *out = c;
    return DVM_OK;
}

void dvm_destroy(dvm_ctx *c)
{
    if (!c) return;
    free_grid_buffers(c);
    free_mesh_buffers(c);
    free_lbm_buffers(c);
    dvm::hs_free(c->hs, [c](void *p) { void *q = p; dev_free(c, q); });
    dvm::mlp_free(c->mlp, [c](void *p) { void *q = p; dev_free(c, q); });
    if (c->d_status) cudaFree(c->d_status);
    for (int k = 0; k < 4; k++)
        if (c->tev[k]) cudaEventDestroy(c->tev[k]);
    delete c;
}

const char *dvm_last_error(const dvm_ctx *c) { return c ? c->err.c_str() : "null context"; }

int dvm_set_stream(dvm_ctx *c, void *stream)
{
    if (!c) return DVM_EINVAL;
    c->stream = static_cast<cudaStream_t>(stream);
    return DVM_OK;
}

int dvm_set_allocator(dvm_ctx *c, void *(*alloc_fn)(size_t, void *), void (*free_fn)(void *, void *), void *user)
{
    if (!c) return DVM_EINVAL;
    if (c->state != 0) return fail(c, DVM_ESTATE, "set the allocator before building the tree");
    if ((alloc_fn == nullptr) != (free_fn == nullptr)) return fail(c, DVM_EINVAL, "give both allocator functions or neither");
    c->alloc_fn = alloc_fn;
    c->free_fn = free_fn;
    c->alloc_user = user;
    return DVM_OK;
}

static int after_mesh(dvm_ctx *c)
{
    free_grid_buffers(c);
    free_mesh_buffers(c);
    const int lattice = c->lat.kind;
    free_lbm_buffers(c);
    c->mesh_on_device = false;
    c->state = 1;
    if (lattice) {
        const int rc = dvm_lbm_set_lattice(c, lattice);
        if (rc) return rc;
    }
    if (c->nv > 0) {
        int n[3] = {c->n[0], c->n[1], c->n[2]};
        double lo[3] = {c->lo[0], c->lo[1], c->lo[2]}, hi[3] = {c->hi[0], c->hi[1], c->hi[2]};
        return dvm_set_velocity_grid(c, n, lo, hi);
    }
    return DVM_OK;
}

int dvm_build_tree(dvm_ctx *c, const dvm_tree_spec *spec)
{
    if (!c || !spec) return DVM_EINVAL;
    std::string err;
    int rc = dvm::build_mesh(*spec, c->mesh, err);
    if (rc) return fail(c, rc, err);
    return after_mesh(c);
}

int dvm_refine(dvm_ctx *c, const uint8_t *flag, int64_t n)
{
    if (!c || !flag) return DVM_EINVAL;
    if (c->state < 1) return fail(c, DVM_ESTATE, "build the tree first");
    std::string err;
    int rc = dvm::refine_mesh(c->mesh, flag, n, err);
    if (rc) return fail(c, rc, err);
    return after_mesh(c);
}

int dvm_refine_project(dvm_ctx *c, const uint8_t *flag, int64_t n)
{
    if (!c || !flag) return DVM_EINVAL;
    if (c->state < 3) return fail(c, DVM_ESTATE, "f is not set (dvm_refine changes the mesh alone)");
    // the old mesh's leaves and the device row of each old cell
    const dvm::Mesh old = c->mesh;
    const int64_t onc = ncells_of(c);
    std::string err;
    int rc = dvm::refine_mesh(c->mesh, flag, n, err);
    if (rc) return fail(c, rc, err);
    // keep the old f buffer (cells and inflow ghost) past the rebuild
    void *oldf = c->d_f[c->cur];
    c->d_f[c->cur] = nullptr;
    const int64_t row = (int64_t)c->nv * (int64_t)elem_size(c->cfg.precision);
    rc = after_mesh(c);
    // new cell i takes the old cell whose leaf contains it (refinement only
    // splits, so one does); a new fluid cell inside an old solid leaf takes
    // the freestream (the old inflow ghost row)
    std::vector<int64_t> rows;
    const dvm::Mesh &m = c->mesh;
    if (!rc) {
        const int64_t nnc = ncells_of(c);
        rows.reserve(4 * (size_t)nnc);
        size_t o = 0;
        for (int64_t q = 0; q < nnc; q++) {
            const dvm::Leaf &x = m.leaves[m.leaf_of_cell[q]];
            // old leaves are in Morton order and tile the domain: the containing
            // one is the last with key <= the new leaf's key
            while (o + 1 < old.leaves.size() && old.leaves[o + 1].key <= x.key) o++;
            const dvm::Leaf &y = old.leaves[o];
            bool inside = y.lev <= x.lev;
            for (int d = 0; d < m.spec.dim && inside; d++) inside = (x.i[d] >> (x.lev - y.lev)) == y.i[d];
            const int64_t oc = inside ? old.cell_of_leaf[o] : -1;
            rows.insert(rows.end(), {0, q, 1, oc >= 0 ? oc : onc});
        }
    }
    void **d_bufs = nullptr;
    int64_t *d_rows = nullptr;
    if (!rc) {
        d_bufs = static_cast<void **>(dev_alloc(c, 2 * sizeof(void *)));
        d_rows = static_cast<int64_t *>(dev_alloc(c, std::max<size_t>(rows.size(), 4) * sizeof(int64_t)));
        if (!d_bufs || !d_rows) rc = fail(c, DVM_ENOMEM, "device allocation (projection)");
    }
    if (!rc) {
        void *hb[2] = {c->d_f[c->cur], oldf};
        rc = cuda_check(c, cudaMemcpy(d_bufs, hb, sizeof hb, cudaMemcpyHostToDevice), "projection buffers");
        if (!rc) rc = cuda_check(c, cudaMemcpy(d_rows, rows.data(), rows.size() * sizeof(int64_t), cudaMemcpyHostToDevice),
                                 "projection rows");
        if (!rc) rc = dvm::launch_copy_rows(d_bufs, d_rows, (int64_t)rows.size() / 4, row, c->stream);
        if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "projection");
    }
    void *p1 = d_bufs, *p2 = d_rows;
    dev_free(c, p1);
    dev_free(c, p2);
    dev_free(c, oldf);
    if (rc) return rc;
    c->state = 3;
    c->have_step_moments = false;
    return DVM_OK;
}

int dvm_coarsen(dvm_ctx *c, const uint8_t *flag, int64_t n)
{
    if (!c || !flag) return DVM_EINVAL;
    if (c->state < 1) return fail(c, DVM_ESTATE, "build the tree first");
    std::string err;
    int rc = dvm::coarsen_mesh(c->mesh, flag, n, err);
    if (rc) return fail(c, rc, err);
    return after_mesh(c);
}

int dvm_coarsen_project(dvm_ctx *c, const uint8_t *flag, int64_t n)
{
    if (!c || !flag) return DVM_EINVAL;
    if (c->state < 3) return fail(c, DVM_ESTATE, "f is not set (dvm_coarsen changes the mesh alone)");
    const dvm::Mesh old = c->mesh;
    const int64_t onc = ncells_of(c);
    std::string err;
    int rc = dvm::coarsen_mesh(c->mesh, flag, n, err);
    if (rc) return fail(c, rc, err);
    void *oldf = c->d_f[c->cur];
    c->d_f[c->cur] = nullptr;
    rc = after_mesh(c);
    // each new cell: its own old cell if its leaf is unchanged, else the mean
    // of the old fluid cells among its 2^dim children (the freestream ghost
    // row when all of them were solid)
    std::vector<int64_t> start, idx;
    if (!rc) {
        const dvm::Mesh &m = c->mesh;
        const int dim = m.spec.dim, L = m.spec.max_level;
        std::unordered_map<uint64_t, int64_t> at;  // (level, Morton key) of an old leaf -> old cell
        at.reserve(old.leaves.size() * 2);
        for (size_t q = 0; q < old.leaves.size(); q++)
            at[old.leaves[q].key * 64 + (uint64_t)old.leaves[q].lev] = old.cell_of_leaf[q];
        const int64_t nnc = ncells_of(c);
        start.reserve(nnc + 1);
        start.push_back(0);
        for (int64_t q = 0; q < nnc; q++) {
            const dvm::Leaf &x = m.leaves[m.leaf_of_cell[q]];
            const auto it = at.find(x.key * 64 + (uint64_t)x.lev);
            if (it != at.end() && it->second >= 0) {
                idx.push_back(it->second);
            } else {
                // children of a merged parent share its key prefix; child k
                // sets the dim bits below the parent's level
                const int sh = dim * (L - x.lev - 1);
                size_t before = idx.size();
                for (int k = 0; k < (1 << dim); k++) {
                    const auto jt = at.find((x.key | ((uint64_t)k << sh)) * 64 + (uint64_t)(x.lev + 1));
                    if (jt != at.end() && jt->second >= 0) idx.push_back(jt->second);
                }
                if (idx.size() == before) idx.push_back(onc);
            }
            start.push_back((int64_t)idx.size());
        }
    }
    int64_t *d_start = nullptr, *d_idx = nullptr;
    if (!rc) {
        d_start = dev_alloc_t<int64_t>(c, start.size());
        d_idx = dev_alloc_t<int64_t>(c, std::max<size_t>(idx.size(), 1));
        if (!d_start || !d_idx) rc = fail(c, DVM_ENOMEM, "device allocation (projection)");
    }
    if (!rc) rc = cuda_check(c, cudaMemcpy(d_start, start.data(), start.size() * 8, cudaMemcpyHostToDevice), "projection");
    if (!rc) rc = cuda_check(c, cudaMemcpy(d_idx, idx.data(), idx.size() * 8, cudaMemcpyHostToDevice), "projection");
    if (!rc) rc = dvm::launch_mean_rows(c->cfg.precision, c->d_f[c->cur], oldf, d_start, d_idx,
                                        (int64_t)start.size() - 1, c->nv, c->stream);
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "projection");
    void *p1 = d_start, *p2 = d_idx;
    dev_free(c, p1);
    dev_free(c, p2);
    dev_free(c, oldf);
    if (rc) return rc;
    c->state = 3;
    c->have_step_moments = false;
    return DVM_OK;
}

int dvm_get_counts(const dvm_ctx *c, int64_t *nleaves, int64_t *ncells, int64_t *nfaces, int64_t *nbfaces, int64_t *nv)
{
    if (!c) return DVM_EINVAL;
    if (nleaves) *nleaves = (int64_t)c->mesh.leaves.size();
    if (ncells) *ncells = ncells_of(c);
    if (nfaces) *nfaces = (int64_t)c->mesh.fm.size();
    if (nbfaces) *nbfaces = (int64_t)c->mesh.bl.size();
    if (nv) *nv = c->nv;
    return DVM_OK;
}

int dvm_get_leaves(const dvm_ctx *c, uint64_t *keys, uint8_t *levels, uint8_t *solid)
{
    if (!c) return DVM_EINVAL;
    if (c->state < 1) return DVM_ESTATE;
    for (size_t q = 0; q < c->mesh.leaves.size(); q++) {
        if (keys) keys[q] = c->mesh.leaves[q].key;
        if (levels) levels[q] = (uint8_t)c->mesh.leaves[q].lev;
        if (solid) solid[q] = c->mesh.leaves[q].solid;
    }
    return DVM_OK;
}

int dvm_get_faces(const dvm_ctx *c, int64_t *minus, int64_t *plus, uint8_t *axis, double *area)
{
    if (!c) return DVM_EINVAL;
    if (c->state < 1) return DVM_ESTATE;
    const dvm::Mesh &m = c->mesh;
    for (size_t q = 0; q < m.fm.size(); q++) {
        if (minus) minus[q] = m.fm[q];
        if (plus) plus[q] = m.fp[q];
        if (axis) axis[q] = m.fax[q];
        if (area) area[q] = m.farea[q];
    }
    return DVM_OK;
}

int dvm_get_bfaces(const dvm_ctx *c, int64_t *leaf, uint8_t *axis, uint8_t *side, uint8_t *kind, int64_t *other, double *area)
{
    if (!c) return DVM_EINVAL;
    if (c->state < 1) return DVM_ESTATE;
    const dvm::Mesh &m = c->mesh;
    for (size_t q = 0; q < m.bl.size(); q++) {
        if (leaf) leaf[q] = m.bl[q];
        if (axis) axis[q] = m.bax[q];
        if (side) side[q] = m.bside[q];
        if (kind) kind[q] = m.bkind[q];
        if (other) other[q] = m.bother[q];
        if (area) area[q] = m.barea[q];
    }
    return DVM_OK;
}

int dvm_cell_centres(const dvm_ctx *c, double *xyz, double *h)
{
    if (!c || !xyz) return DVM_EINVAL;
    if (c->state < 1) return DVM_ESTATE;
    const dvm::Mesh &m = c->mesh;
    for (size_t q = 0; q < m.leaf_of_cell.size(); q++) {
        const dvm::Leaf &x = m.leaves[m.leaf_of_cell[q]];
        const double hh = std::ldexp(1.0, -x.lev);
        for (int d = 0; d < 3; d++) xyz[3 * q + d] = d < m.spec.dim ? (x.i[d] + 0.5) * hh : 0.5;
        if (h) h[q] = hh;
    }
    return DVM_OK;
}

int dvm_set_velocity_grid(dvm_ctx *c, const int n[3], const double lo[3], const double hi[3])
{
    if (!c || !n || !lo || !hi) return DVM_EINVAL;
    if (c->state < 1) return fail(c, DVM_ESTATE, "build the tree first");
    const int vec = c->cfg.precision == DVM_F64 ? 2 : 4;
    for (int d = 0; d < 3; d++) {
        if (n[d] < 2 || n[d] % 2 || n[d] > 64) return fail(c, DVM_EINVAL, "each n must be even and at most 64");
        if (!(hi[d] > 0.0) || lo[d] != -hi[d]) return fail(c, DVM_EINVAL, "the velocity grid must be symmetric (lo = -hi)");
    }
    if ((n[2] / 2) % vec) return fail(c, DVM_EINVAL, "nz/2 must be a multiple of the vector width");
    int drc = ensure_device(c);
    if (drc) return drc;
    if (!c->mesh_on_device) {
        drc = upload_mesh(c);
        if (drc) return drc;
        c->mesh_on_device = true;
    }
    free_grid_buffers(c);
    for (int d = 0; d < 3; d++) {
        c->n[d] = n[d];
        c->half[d] = n[d] / 2;
        c->lo[d] = lo[d];
        c->hi[d] = hi[d];
        c->hv[d] = (hi[d] - lo[d]) / n[d];
    }
    c->dV = c->hv[0] * c->hv[1] * c->hv[2];
    c->nv = n[0] * n[1] * n[2];
    c->P = c->nv / 8;
    // node values lo + (k + 1/2) h in sign-group order
    c->xi.assign(3 * (size_t)c->nv, 0.0);
    int v = 0;
    for (int o = 0; o < 8; o++)
        for (int mx = 0; mx < c->half[0]; mx++)
            for (int my = 0; my < c->half[1]; my++)
                for (int mz = 0; mz < c->half[2]; mz++, v++) {
                    const int m3[3] = {mx, my, mz};
                    for (int d = 0; d < 3; d++) {
                        const bool pos = (o >> (2 - d)) & 1;
                        const int k = pos ? c->half[d] + m3[d] : c->half[d] - 1 - m3[d];
                        c->xi[3 * (size_t)v + d] = c->lo[d] + ((double)k + 0.5) * c->hv[d];
                    }
                }
    for (int d = 0; d < 3; d++)
        for (int m = 0; m < 32; m++) {
            const double val = m < c->half[d] ? c->lo[d] + ((double)(c->half[d] + m) + 0.5) * c->hv[d] : 0.0;
            c->amag[32 * d + m] = val;
            c->amag_f[32 * d + m] = (float)val;
        }
    const int64_t nc = ncells_of(c);
    c->f_elems = (size_t)nc * c->nv;
    const size_t fb = c->f_elems * elem_size(c->cfg.precision);
    // one extra cell: the inflow ghost
    const size_t fbg = fb + (size_t)c->nv * elem_size(c->cfg.precision);
    c->d_f[0] = dev_alloc(c, fbg);
    c->d_f[1] = dev_alloc(c, fbg);
    c->d_amag = dev_alloc_t<double>(c, 96);
    c->d_amag_f = dev_alloc_t<float>(c, 96);
    c->d_xi = dev_alloc_t<double>(c, 3 * (size_t)c->nv);
    c->d_mom = dev_alloc_t<double>(c, 5 * (size_t)nc);
    c->d_mom2 = dev_alloc_t<double>(c, 5 * (size_t)nc);
    c->d_res = dev_alloc_t<double>(c, 5 * (size_t)nc);
    if (!c->d_f[0] || !c->d_f[1] || !c->d_amag || !c->d_amag_f || !c->d_xi || !c->d_mom || !c->d_mom2 || !c->d_res) {
        free_grid_buffers(c);
        return fail(c, DVM_ENOMEM, "device allocation (f buffers)");
    }
    int rc = cuda_check(c, cudaMemcpy(c->d_amag, c->amag, sizeof c->amag, cudaMemcpyHostToDevice), "copy |xi|");
    if (!rc) rc = cuda_check(c, cudaMemcpy(c->d_amag_f, c->amag_f, sizeof c->amag_f, cudaMemcpyHostToDevice), "copy |xi|");
    if (!rc) rc = cuda_check(c, cudaMemcpy(c->d_xi, c->xi.data(), c->xi.size() * 8, cudaMemcpyHostToDevice), "copy xi");
    if (!rc) rc = upload_freestream(c);
    if (rc) return rc;
    c->cur = 0;
    c->state = 2;
    return DVM_OK;
}

int dvm_get_velocities(const dvm_ctx *c, double *xi)
{
    if (!c || !xi) return DVM_EINVAL;
    if (c->state < 2) return DVM_ESTATE;
    std::memcpy(xi, c->xi.data(), c->xi.size() * sizeof(double));
    return DVM_OK;
}

int dvm_set_freestream(dvm_ctx *c, double rho, const double u[3], double T)
{
    if (!c || !u || !(rho > 0.0) || !(T > 0.0)) return DVM_EINVAL;
    c->fs_rho = rho;
    c->fs_T = T;
    for (int d = 0; d < 3; d++) c->fs_u[d] = u[d];
    return upload_freestream(c);
}

int dvm_init_maxwellian(dvm_ctx *c, int nmix, const double *w, const double *rho, const double *u, const double *T)
{
    if (!c || nmix < 1 || !w || !rho || !u || !T) return DVM_EINVAL;
    if (c->state < 2) return fail(c, DVM_ESTATE, "set the velocity grid first");
    const int64_t nc = ncells_of(c);
    const size_t k = (size_t)nc * nmix;
    for (size_t q = 0; q < k; q++)
        if (!(rho[q] >= 0.0) || !(T[q] > 0.0)) return fail(c, DVM_EINVAL, "need rho >= 0 and T > 0");
    double *dw = dev_alloc_t<double>(c, k), *dr = dev_alloc_t<double>(c, k);
    double *du = dev_alloc_t<double>(c, 3 * k), *dT = dev_alloc_t<double>(c, k);
    int rc = DVM_OK;
    if (!dw || !dr || !du || !dT) rc = fail(c, DVM_ENOMEM, "device allocation (init)");
    if (!rc) rc = cuda_check(c, cudaMemcpy(dw, w, k * 8, cudaMemcpyHostToDevice), "copy w");
    if (!rc) rc = cuda_check(c, cudaMemcpy(dr, rho, k * 8, cudaMemcpyHostToDevice), "copy rho");
    if (!rc) rc = cuda_check(c, cudaMemcpy(du, u, 3 * k * 8, cudaMemcpyHostToDevice), "copy u");
    if (!rc) rc = cuda_check(c, cudaMemcpy(dT, T, k * 8, cudaMemcpyHostToDevice), "copy T");
    if (!rc) rc = dvm::launch_init_maxwellian(c->cfg.precision, c->d_f[c->cur], nc, c->nv, nmix, dw, dr, du, dT, c->d_xi, c->stream);
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "init_maxwellian");
    void *p;
    p = dw; dev_free(c, p);
    p = dr; dev_free(c, p);
    p = du; dev_free(c, p);
    p = dT; dev_free(c, p);
    if (!rc) {
        c->state = 3;
        c->have_step_moments = false;
    }
    return rc;
}

static int convert_chunks(dvm_ctx *c, double *host_out, const double *host_in, int64_t count)
{
    const int64_t total = (int64_t)c->f_elems;
    if (count != total) return fail(c, DVM_EINVAL, "count must be ncells*nv");
    const int64_t chunk = std::min<int64_t>(total, 1 << 24);
    double *stage = dev_alloc_t<double>(c, chunk);
    if (!stage) return fail(c, DVM_ENOMEM, "device allocation (staging)");
    const size_t es = elem_size(c->cfg.precision);
    int rc = DVM_OK;
    for (int64_t s = 0; s < total && !rc; s += chunk) {
        const int64_t n = std::min(chunk, total - s);
        char *fdev = static_cast<char *>(c->d_f[c->cur]) + s * es;
        if (host_out) {
            rc = dvm::launch_to_f64(c->cfg.precision, fdev, stage, n, c->stream);
            if (!rc) rc = cuda_check(c, cudaMemcpyAsync(host_out + s, stage, n * 8, cudaMemcpyDeviceToHost, c->stream), "copy f");
        } else {
            rc = cuda_check(c, cudaMemcpyAsync(stage, host_in + s, n * 8, cudaMemcpyHostToDevice, c->stream), "copy f");
            if (!rc) rc = dvm::launch_from_f64(c->cfg.precision, stage, fdev, n, c->stream);
        }
        if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "convert f");
    }
    void *p = stage;
    dev_free(c, p);
    return rc;
}

int dvm_get_f(dvm_ctx *c, double *f, int64_t count)
{
    if (!c || !f) return DVM_EINVAL;
    if (c->state < 3) return fail(c, DVM_ESTATE, "f is not set");
    return convert_chunks(c, f, nullptr, count);
}

int dvm_get_f_rows(dvm_ctx *c, int64_t n, const int64_t *cells, double *out)
{
    if (!c || n < 0 || (n > 0 && (!cells || !out))) return DVM_EINVAL;
    if (c->state < 3) return fail(c, DVM_ESTATE, "f is not set");
    const int64_t nc = ncells_of(c);
    for (int64_t i = 0; i < n; i++)
        if (cells[i] < 0 || cells[i] >= nc) return fail(c, DVM_EINVAL, "cell index out of range");
    if (n == 0) return DVM_OK;
    const size_t es = elem_size(c->cfg.precision);
    const int64_t nv = c->nv;
    const int64_t rows = std::max<int64_t>(1, std::min<int64_t>(n, (1 << 24) / nv));
    int64_t *didx = dev_alloc_t<int64_t>(c, rows);
    char *gath = dev_alloc_t<char>(c, (size_t)(rows * nv) * es);
    double *stage = dev_alloc_t<double>(c, rows * nv);
    int rc = DVM_OK;
    if (!didx || !gath || !stage) rc = fail(c, DVM_ENOMEM, "device allocation (row gather)");
    for (int64_t s0 = 0; s0 < n && !rc; s0 += rows) {
        const int64_t k = std::min(rows, n - s0);
        rc = cuda_check(c, cudaMemcpyAsync(didx, cells + s0, k * 8, cudaMemcpyHostToDevice, c->stream), "copy cells");
        if (!rc) rc = dvm::launch_rows_indexed(true, gath, c->d_f[c->cur], didx, k, nv * (int64_t)es, c->stream);
        if (!rc) rc = dvm::launch_to_f64(c->cfg.precision, gath, stage, k * nv, c->stream);
        if (!rc) rc = cuda_check(c, cudaMemcpyAsync(out + s0 * nv, stage, k * nv * 8, cudaMemcpyDeviceToHost, c->stream), "copy rows");
        if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "row gather");
    }
    void *p = didx;
    dev_free(c, p);
    p = gath;
    dev_free(c, p);
    p = stage;
    dev_free(c, p);
    return rc;
}

int dvm_set_f(dvm_ctx *c, const double *f, int64_t count)
{
    if (!c || !f) return DVM_EINVAL;
    if (c->state < 2) return fail(c, DVM_ESTATE, "set the velocity grid first");
    int rc = convert_chunks(c, nullptr, f, count);
    if (!rc) {
        c->state = 3;
        c->have_step_moments = false;
    }
    return rc;
}

int dvm_upload_f(dvm_ctx *c, const void *host, int64_t bytes)
{
    if (!c || !host) return DVM_EINVAL;
    if (c->state < 2) return fail(c, DVM_ESTATE, "set the velocity grid first");
    if ((size_t)bytes != c->f_elems * elem_size(c->cfg.precision)) return fail(c, DVM_EINVAL, "byte count differs from the f buffer");
    int rc = cuda_check(c, cudaMemcpyAsync(c->d_f[c->cur], host, bytes, cudaMemcpyHostToDevice, c->stream), "upload f");
    if (!rc) {
        c->state = 3;
        c->have_step_moments = false;
    }
    return rc;
}

int dvm_download_f(dvm_ctx *c, void *host, int64_t bytes)
{
    if (!c || !host) return DVM_EINVAL;
    if (c->state < 3) return fail(c, DVM_ESTATE, "f is not set");
    if ((size_t)bytes != c->f_elems * elem_size(c->cfg.precision)) return fail(c, DVM_EINVAL, "byte count differs from the f buffer");
    int rc = cuda_check(c, cudaMemcpyAsync(host, c->d_f[c->cur], bytes, cudaMemcpyDeviceToHost, c->stream), "download f");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "download f");
    return rc;
}

int dvm_f_device(const dvm_ctx *c, void **ptr, int64_t *bytes)
{
    if (!c || !ptr) return DVM_EINVAL;
    if (c->state < 2) return DVM_ESTATE;
    *ptr = c->d_f[c->cur];
    if (bytes) *bytes = (int64_t)(c->f_elems * elem_size(c->cfg.precision));
    return DVM_OK;
}

int dvm_dt_cfl(const dvm_ctx *c, double cfl, double *dt)
{
    if (!c || !dt || !(cfl > 0.0)) return DVM_EINVAL;
    if (c->state < 2) return DVM_ESTATE;
    double smax = 0.0;
    for (int v = 0; v < c->nv; v++) {
        double s = 0.0;
        for (int d = 0; d < c->mesh.spec.dim; d++) s += std::fabs(c->xi[3 * (size_t)v + d]);
        smax = std::max(smax, s);
    }
    *dt = cfl * std::ldexp(1.0, -c->mesh.max_cell_level) / smax;
    return DVM_OK;
}

static int set_tables(dvm_ctx *c, int trials, uint64_t seed, bool lattice)
{
    if (!c || trials < 1) return DVM_EINVAL;
    if (c->state < 2) return fail(c, DVM_ESTATE, "set the velocity grid first");
    if (c->cfg.precision != DVM_F32) return fail(c, DVM_ENOTIMPL, "the hard-sphere operator runs on FP32 storage");
    std::string err;
    int rc = dvm::hs_build(c->hs, c->n, c->lo, c->hv, c->xi, trials, seed, lattice, err,
                           [c](size_t b) { return dev_alloc(c, b); },
                           [c](void *p) { void *q = p; dev_free(c, q); });
    if (rc) return fail(c, rc, err);
    return DVM_OK;
}

int dvm_set_collision_tables(dvm_ctx *c, int trials, uint64_t seed) { return set_tables(c, trials, seed, false); }

int dvm_set_collision_tables_lattice(dvm_ctx *c, int trials, uint64_t seed)
{
    return set_tables(c, trials, seed, true);
}

int dvm_get_collision_tables(const dvm_ctx *c, int32_t *gam, int32_t *l, int32_t *m, float *b, int64_t *discarded)
{
    if (!c) return DVM_EINVAL;
    if (!c->hs.ready) return DVM_ESTATE;
    const size_t n = c->hs.host_b.size();
    for (size_t q = 0; q < n; q++) {
        const uint32_t w0 = c->hs.host_idx[2 * q], w1 = c->hs.host_idx[2 * q + 1];
        if (gam) gam[q] = (int32_t)(w0 & 0xffffu);
        if (l) l[q] = (int32_t)(w0 >> 16);
        if (m) m[q] = (int32_t)w1;
        if (b) b[q] = c->hs.host_b[q];
    }
    if (discarded) *discarded = c->hs.discarded;
    return DVM_OK;
}

int dvm_step(dvm_ctx *c, int nsteps, double dt)
{
    if (!c || nsteps < 0) return DVM_EINVAL;
    if (c->state < 3) return fail(c, DVM_ESTATE, "f is not set");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, DVM_EINVAL, "dt must be positive");
    if ((c->cfg.collision == DVM_COLL_HS || c->cfg.collision == DVM_COLL_LEARNED) && !c->hs.ready)
        return fail(c, DVM_ESTATE, "set the collision tables first");
    if (c->cfg.collision == DVM_COLL_LEARNED && (!c->mlp_set || !c->learned_cfg))
        return fail(c, DVM_ESTATE, "set the network weights and the Knudsen threshold first");
    dvm::StepParams p{};
    p.dim = c->mesh.spec.dim;
    p.prec = c->cfg.precision;
    p.coll = (c->cfg.collision == DVM_COLL_BGK || c->cfg.collision == DVM_COLL_BGK_ENTROPIC) ? c->cfg.collision
                                                                                                : DVM_COLL_NONE;
    p.ncells = ncells_of(c);
    p.nv = c->nv;
    p.P = c->P;
    for (int d = 0; d < 3; d++) { p.half[d] = c->half[d]; p.n[d] = c->n[d]; p.hv[d] = c->hv[d]; }
    p.st_src = c->d_src;
    p.st_w = c->d_w;
    p.st_cnt = c->d_cnt;
    p.inv_h = c->d_invh;
    p.amag = c->d_amag;
    p.amag_f = c->d_amag_f;
    p.dt = dt;
    p.kn = c->cfg.kn;
    p.dV = c->dV;
    p.mom_out = c->d_mom;
    p.status = c->d_status;
    p.counter = c->d_counter;
    p.stream = c->stream;
    // the BGK step kernel writes the residual of its collision term; the
    // hard-sphere and learned updates write theirs after the transport launch
    const bool bgk = c->cfg.collision == DVM_COLL_BGK || c->cfg.collision == DVM_COLL_BGK_ENTROPIC;
    if (c->cfg.collision == DVM_COLL_HS) {
        int rc = dvm::hs_prepare(c->hs, p.ncells, [c](size_t b) { return dev_alloc(c, b); },
                                 [c](void *q) { void *r = q; dev_free(c, r); });
        if (rc) return fail(c, rc, "hard-sphere scratch allocation failed");
    }
    if (c->cfg.collision == DVM_COLL_LEARNED) {
        int rc = learned_prepare(c);
        if (rc) return rc;
    }
    for (int s = 0; s < nsteps; s++) {
        p.f_in = c->d_f[c->cur];
        p.f_out = c->d_f[1 - c->cur];
        p.res_out = nullptr;
        p.res_phi = bgk ? reinterpret_cast<float2 *>(c->d_res) : nullptr;
        if (c->timing) cudaEventRecord(c->tev[0], c->stream);
        if (cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, DVM_ECUDA, "counter reset failed");
        }
        int rc = dvm::launch_step(p);
        if (rc) return fail(c, rc, rc == DVM_ENOTIMPL ? "velocity grid too large for the step kernel" : "step launch failed");
        if (c->timing) cudaEventRecord(c->tev[1], c->stream);
        p.res_out = c->d_res;
        p.res_phi = nullptr;
        if (c->cfg.collision == DVM_COLL_HS) {
            rc = dvm::launch_hs_collide(c->hs, p, c->d_f[1 - c->cur], c->cfg.kn, dt);
            if (rc) return fail(c, rc, "hard-sphere collision launch failed");
            if (c->timing) cudaEventRecord(c->tev[2], c->stream);
        }
        if (c->cfg.collision == DVM_COLL_LEARNED) {
            rc = learned_collide_device(c, static_cast<float *>(c->d_f[1 - c->cur]), c->d_mom, dt, nullptr, nullptr,
                                        c->timing ? c->tev[2] : nullptr);
            if (rc) return rc;
        }
        if (c->timing) {
            if (bgk || c->cfg.collision == DVM_COLL_NONE) cudaEventRecord(c->tev[2], c->stream);
            cudaEventRecord(c->tev[3], c->stream);
            rc = cuda_check(c, cudaEventSynchronize(c->tev[3]), "phase timing");
            if (rc) return rc;
            float t[3] = {0, 0, 0};
            for (int k = 0; k < 3; k++) cudaEventElapsedTime(&t[k], c->tev[k], c->tev[k + 1]);
            for (int k = 0; k < 3; k++) c->tms[k] += t[k];
            c->tsteps++;
        }
        c->cur = 1 - c->cur;
    }
    c->have_step_moments = nsteps > 0 || c->have_step_moments;
    if (nsteps > 0) {
        c->have_res = c->cfg.collision != DVM_COLL_NONE;
        c->res_pairs = c->cfg.collision == DVM_COLL_BGK || c->cfg.collision == DVM_COLL_BGK_ENTROPIC;
    }
    int st = 0;
    int rc = cuda_check(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read status");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "step");
    if (rc) return rc;
    if (st & dvm::ST_TIMEOUT) {
        cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
        return fail(c, DVM_ETIMEOUT, "a bounded wait for an asynchronous tile copy gave up");
    }
    if (st) {
        cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
        std::string why;
        if (st & dvm::ST_NONPOS) why += " non-positive density or temperature;";
        if (st & dvm::ST_SINGULAR) why += " singular correction system;";
        if (st & dvm::ST_NUDT) why += " relaxation factor above 1 (dt too large for Kn);";
        return fail(c, DVM_EUNSTABLE, "unstable step:" + why);
    }
    return DVM_OK;
}

int dvm_partition_info(const dvm_ctx *c, int nparts, int part, int64_t *c0, int64_t *c1, int64_t *nghost,
                       int64_t *ghosts, int64_t cap)
{
    if (!c || nparts < 1 || part < 0 || part >= nparts) return DVM_EINVAL;
    dvm_ctx *cc = const_cast<dvm_ctx *>(c);
    if (c->state < 1) return fail(cc, DVM_ESTATE, "build the tree first");
    const int64_t nc = ncells_of(c);
    if (nparts > nc) return fail(cc, DVM_EINVAL, "more parts than cells");
    std::vector<int32_t> enc;
    dvm::encode_stencils(c->mesh.st_src, nc, enc);
    std::vector<dvm::Part> parts;
    dvm::partition_cells(nc, nparts, enc, c->mesh.st_cnt, parts);
    const dvm::Part &pt = parts[part];
    if (c0) *c0 = pt.c0;
    if (c1) *c1 = pt.c1;
    if (nghost) *nghost = (int64_t)pt.ghosts.size();
    if (ghosts) {
        if (cap < (int64_t)pt.ghosts.size()) return fail(cc, DVM_EINVAL, "ghost buffer too small");
        std::copy(pt.ghosts.begin(), pt.ghosts.end(), ghosts);
    }
    return DVM_OK;
}

int dvm_partition_weighted(const dvm_ctx *c, int nparts, const double *weights, int part, int64_t *c0, int64_t *c1,
                           int64_t *nghost, int64_t *ghosts, int64_t cap)
{
    if (!c || !weights || nparts < 1 || part < 0 || part >= nparts) return DVM_EINVAL;
    dvm_ctx *cc = const_cast<dvm_ctx *>(c);
    if (c->state < 1) return fail(cc, DVM_ESTATE, "build the tree first");
    const int64_t nc = ncells_of(c);
    if (nparts > nc) return fail(cc, DVM_EINVAL, "more parts than cells");
    for (int64_t q = 0; q < nc; q++)
        if (!(weights[q] >= 0.0) || !std::isfinite(weights[q])) return fail(cc, DVM_EINVAL, "weights must be finite and >= 0");
    std::vector<int32_t> enc;
    dvm::encode_stencils(c->mesh.st_src, nc, enc);
    std::vector<dvm::Part> parts;
    dvm::partition_cells(nc, nparts, enc, c->mesh.st_cnt, parts, weights);
    const dvm::Part &pt = parts[part];
    if (c0) *c0 = pt.c0;
    if (c1) *c1 = pt.c1;
    if (nghost) *nghost = (int64_t)pt.ghosts.size();
    if (ghosts) {
        if (cap < (int64_t)pt.ghosts.size()) return fail(cc, DVM_EINVAL, "ghost buffer too small");
        std::copy(pt.ghosts.begin(), pt.ghosts.end(), ghosts);
    }
    return DVM_OK;
}

int dvm_step_partitioned(dvm_ctx *c, int nparts, int nsteps, double dt)
{
    if (!c || nsteps < 0 || nparts < 1) return DVM_EINVAL;
    if (c->state < 3) return fail(c, DVM_ESTATE, "f is not set");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, DVM_EINVAL, "dt must be positive");
    if (c->cfg.collision != DVM_COLL_BGK && c->cfg.collision != DVM_COLL_BGK_ENTROPIC &&
        c->cfg.collision != DVM_COLL_NONE)
        return fail(c, DVM_ENOTIMPL, "the partitioned step runs transport and BGK only");
    const int64_t nc = ncells_of(c);
    if (nparts > nc) return fail(c, DVM_EINVAL, "more parts than cells");
    const size_t es = elem_size(c->cfg.precision), tcs = tc_size(c->cfg.precision);
    const int64_t row = (int64_t)c->nv * (int64_t)es;

    std::vector<int32_t> enc;
    dvm::encode_stencils(c->mesh.st_src, nc, enc);
    std::vector<dvm::Part> parts;
    dvm::partition_cells(nc, nparts, enc, c->mesh.st_cnt, parts);

    // per part: two f buffers of (owned + ghosts + inflow ghost) rows and the
    // stencils in local numbering; the weights, counts and 1/h are slices of
    // the global arrays
    struct Dev {
        void *f[2] = {nullptr, nullptr};
        int32_t *src = nullptr;
        double *mom = nullptr;
    };
    std::vector<Dev> dev(nparts);
    std::vector<void *> tmp;  // everything to free
    auto alloc = [&](size_t bytes) {
        void *q = dev_alloc(c, bytes);
        if (q) tmp.push_back(q);
        return q;
    };
    int rc = DVM_OK;
    std::vector<int64_t> halo;  // {dst part, dst row, src part, src row}
    for (int p = 0; p < nparts && !rc; p++) {
        const dvm::Part &pt = parts[p];
        const int64_t nloc = pt.c1 - pt.c0, ng = (int64_t)pt.ghosts.size(), rows = nloc + ng + 1;
        Dev &d = dev[p];
        d.f[0] = alloc((size_t)rows * row);
        d.f[1] = alloc((size_t)rows * row);
        d.src = static_cast<int32_t *>(alloc((size_t)nloc * 24 * sizeof(int32_t)));
        d.mom = static_cast<double *>(alloc((size_t)nloc * 5 * sizeof(double)));
        if (!d.f[0] || !d.f[1] || !d.src || !d.mom) {
            rc = fail(c, DVM_ENOMEM, "device allocation (partitions)");
            break;
        }
        std::vector<int32_t> local;
        dvm::local_stencils(pt, nc, enc, local);
        rc = cuda_check(c, cudaMemcpy(d.src, local.data(), local.size() * sizeof(int32_t), cudaMemcpyHostToDevice),
                        "copy local stencils");
        // owned rows and the inflow ghost row into the first buffer, the inflow
        // ghost also into the second
        const char *g = static_cast<const char *>(c->d_f[c->cur]);
        if (!rc)
            rc = cuda_check(c, cudaMemcpyAsync(d.f[0], g + pt.c0 * row, (size_t)nloc * row, cudaMemcpyDeviceToDevice,
                                               c->stream), "scatter f");
        for (int b = 0; b < 2 && !rc; b++)
            rc = cuda_check(c, cudaMemcpyAsync(static_cast<char *>(d.f[b]) + (nloc + ng) * row, g + nc * row, row,
                                               cudaMemcpyDeviceToDevice, c->stream), "inflow ghost");
        for (int64_t k = 0; k < ng; k++) {
            const int64_t s = pt.ghosts[k];
            int q = 0;
            while (parts[q].c1 <= s) q++;
            halo.insert(halo.end(), {(int64_t)p, nloc + k, (int64_t)q, s - parts[q].c0});
        }
    }
    // the two sets of current buffers (step parity) and the halo list
    void **d_bufs = nullptr;
    int64_t *d_halo = nullptr;
    if (!rc) {
        d_bufs = static_cast<void **>(alloc(2 * nparts * sizeof(void *)));
        d_halo = static_cast<int64_t *>(alloc(std::max<size_t>(halo.size(), 4) * sizeof(int64_t)));
        if (!d_bufs || !d_halo) rc = fail(c, DVM_ENOMEM, "device allocation (halo)");
    }
    if (!rc) {
        std::vector<void *> hb(2 * nparts);
        for (int p = 0; p < nparts; p++) {
            hb[p] = dev[p].f[0];
            hb[nparts + p] = dev[p].f[1];
        }
        rc = cuda_check(c, cudaMemcpy(d_bufs, hb.data(), hb.size() * sizeof(void *), cudaMemcpyHostToDevice), "buffers");
        if (!rc && !halo.empty())
            rc = cuda_check(c, cudaMemcpy(d_halo, halo.data(), halo.size() * sizeof(int64_t), cudaMemcpyHostToDevice),
                            "halo list");
    }

    dvm::StepParams base{};
    base.dim = c->mesh.spec.dim;
    base.prec = c->cfg.precision;
    base.coll = (c->cfg.collision == DVM_COLL_BGK || c->cfg.collision == DVM_COLL_BGK_ENTROPIC) ? c->cfg.collision
                                                                                                   : DVM_COLL_NONE;
    base.nv = c->nv;
    base.P = c->P;
    for (int d = 0; d < 3; d++) { base.half[d] = c->half[d]; base.n[d] = c->n[d]; base.hv[d] = c->hv[d]; }
    base.amag = c->d_amag;
    base.amag_f = c->d_amag_f;
    base.dt = dt;
    base.kn = c->cfg.kn;
    base.dV = c->dV;
    base.status = c->d_status;
    base.counter = c->d_counter;
    base.stream = c->stream;
    for (int s = 0; s < nsteps && !rc; s++) {
        const int b = s & 1;
        // the halo exchange: every ghost row from its owner's current buffer
        rc = dvm::launch_copy_rows(d_bufs + b * nparts, d_halo, (int64_t)halo.size() / 4, row, c->stream);
        if (rc) rc = fail(c, rc, "halo exchange launch failed");
        for (int p = 0; p < nparts && !rc; p++) {
            const dvm::Part &pt = parts[p];
            dvm::StepParams q = base;
            q.ncells = pt.c1 - pt.c0;
            q.f_in = dev[p].f[b];
            q.f_out = dev[p].f[1 - b];
            q.st_src = dev[p].src;
            q.st_w = static_cast<const char *>(c->d_w) + pt.c0 * 24 * tcs;
            q.st_cnt = c->d_cnt + pt.c0 * 8;
            q.inv_h = static_cast<const char *>(c->d_invh) + pt.c0 * tcs;
            q.mom_out = dev[p].mom;
            rc = cuda_check(c, cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream), "counter reset");
            if (!rc) rc = dvm::launch_step(q);
            if (rc && rc != DVM_ECUDA) rc = fail(c, rc, "step launch failed");
        }
    }
    // owned rows and step moments back into the global state
    const int fb = nsteps & 1;
    char *g = static_cast<char *>(c->d_f[c->cur]);
    for (int p = 0; p < nparts && !rc && nsteps > 0; p++) {
        const dvm::Part &pt = parts[p];
        const int64_t nloc = pt.c1 - pt.c0;
        rc = cuda_check(c, cudaMemcpyAsync(g + pt.c0 * row, dev[p].f[fb], (size_t)nloc * row, cudaMemcpyDeviceToDevice,
                                           c->stream), "gather f");
        if (!rc)
            rc = cuda_check(c, cudaMemcpyAsync(c->d_mom + pt.c0 * 5, dev[p].mom, (size_t)nloc * 5 * sizeof(double),
                                               cudaMemcpyDeviceToDevice, c->stream), "gather moments");
    }
    int st = 0;
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read status");
    const int rs = cuda_check(c, cudaStreamSynchronize(c->stream), "partitioned step");
    if (!rc) rc = rs;
    for (void *q : tmp) dev_free(c, q);
    if (rc) return rc;
    c->have_step_moments = nsteps > 0 || c->have_step_moments;
    if (nsteps > 0) c->have_res = false;
    if (st) {
        cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
        return fail(c, DVM_EUNSTABLE, "unstable step (non-positive moments, singular system or nu dt > 1)");
    }
    return DVM_OK;
}

static int copy_moments(dvm_ctx *c, const double *dsrc, double *rho, double *u, double *T)
{
    const int64_t nc = ncells_of(c);
    std::vector<double> h(5 * (size_t)nc);
    int rc = cuda_check(c, cudaMemcpyAsync(h.data(), dsrc, h.size() * 8, cudaMemcpyDeviceToHost, c->stream), "copy moments");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "moments");
    if (rc) return rc;
    for (int64_t q = 0; q < nc; q++) {
        if (rho) rho[q] = h[5 * q];
        if (u) for (int d = 0; d < 3; d++) u[3 * q + d] = h[5 * q + 1 + d];
        if (T) T[q] = h[5 * q + 4];
    }
    return DVM_OK;
}

int dvm_moments(dvm_ctx *c, double *rho, double *u, double *T)
{
    if (!c) return DVM_EINVAL;
    if (c->state < 3) return fail(c, DVM_ESTATE, "f is not set");
    int rc = dvm::launch_moments(c->cfg.precision, c->d_f[c->cur], ncells_of(c), c->nv, c->d_xi, c->dV, c->d_mom2, c->stream);
    if (rc) return fail(c, rc, "moments launch failed");
    return copy_moments(c, c->d_mom2, rho, u, T);
}

// Local Knudsen number of every cell from the moments of the stored f (the
// continuum-breakdown sensor of Sec. 2.3 / Sec. 3.4); its sensor stencil is
// built on first use for the current mesh.
static int kn_local_device(dvm_ctx *c)
{
    const int64_t nc = ncells_of(c);
    if (c->ks_cells != nc) {
        dev_free(c, reinterpret_cast<void *&>(c->d_ks_start));
        dev_free(c, reinterpret_cast<void *&>(c->d_ks_nb));
        dev_free(c, reinterpret_cast<void *&>(c->d_ks_coef));
        dev_free(c, reinterpret_cast<void *&>(c->d_ks_knl));
        c->ks_cells = 0;
        dvm::KnStencil ks;
        dvm::build_kn_stencil(c->mesh, ks);
        const size_t ne = ks.nb.size();
        c->d_ks_start = dev_alloc_t<int32_t>(c, (size_t)nc + 1);
        c->d_ks_nb = dev_alloc_t<int32_t>(c, std::max<size_t>(ne, 1));
        c->d_ks_coef = dev_alloc_t<double>(c, 3 * std::max<size_t>(ne, 1));
        c->d_ks_knl = dev_alloc_t<double>(c, (size_t)nc);
        if (!c->d_ks_start || !c->d_ks_nb || !c->d_ks_coef || !c->d_ks_knl)
            return fail(c, DVM_ENOMEM, "device allocation (Knudsen sensor)");
        int rc = cuda_check(c, cudaMemcpy(c->d_ks_start, ks.start.data(), ks.start.size() * 4, cudaMemcpyHostToDevice), "copy sensor stencil");
        if (!rc && ne) rc = cuda_check(c, cudaMemcpy(c->d_ks_nb, ks.nb.data(), ne * 4, cudaMemcpyHostToDevice), "copy sensor stencil");
        if (!rc && ne) rc = cuda_check(c, cudaMemcpy(c->d_ks_coef, ks.coef.data(), ne * 24, cudaMemcpyHostToDevice), "copy sensor stencil");
        if (rc) return rc;
        c->ks_cells = nc;
    }
    int rc = dvm::launch_moments(c->cfg.precision, c->d_f[c->cur], nc, c->nv, c->d_xi, c->dV, c->d_mom2, c->stream);
    if (!rc) rc = dvm::launch_kn_local(c->d_mom2, c->d_ks_start, c->d_ks_nb, c->d_ks_coef, nc, c->cfg.kn, c->d_ks_knl, c->stream);
    return rc ? fail(c, rc, "Knudsen sensor launch") : DVM_OK;
}

int dvm_kn_local(dvm_ctx *c, double *knl)
{
    if (!c || !knl) return DVM_EINVAL;
    if (c->state < 3) return fail(c, DVM_ESTATE, "f is not set");
    if (!(c->cfg.kn > 0.0)) return fail(c, DVM_EINVAL, "the context's Kn must be positive");
    int rc = kn_local_device(c);
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(knl, c->d_ks_knl, (size_t)ncells_of(c) * 8, cudaMemcpyDeviceToHost, c->stream), "copy Kn");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "Knudsen sensor");
    return rc;
}

int dvm_flag_kinetic(dvm_ctx *c, double threshold, uint8_t *kinetic, int64_t *nkinetic)
{
    if (!c || !kinetic || !(threshold >= 0.0)) return DVM_EINVAL;
    const int64_t nc = ncells_of(c);
    std::vector<double> knl((size_t)nc);
    int rc = dvm_kn_local(c, knl.data());
    if (rc) return rc;
    int64_t k = 0;
    for (int64_t q = 0; q < nc; q++) {
        kinetic[q] = knl[q] > threshold ? 1 : 0;
        k += kinetic[q];
    }
    if (nkinetic) *nkinetic = k;
    return DVM_OK;
}

int dvm_step_moments(dvm_ctx *c, double *rho, double *u, double *T)
{
    if (!c) return DVM_EINVAL;
    if (!c->have_step_moments) return fail(c, DVM_ESTATE, "no step has run since f was set");
    return copy_moments(c, c->d_mom, rho, u, T);
}

int dvm_set_timing(dvm_ctx *c, int enable)
{
    if (!c) return DVM_EINVAL;
    if (enable && !c->tev[0])
        for (int k = 0; k < 4; k++)
            if (cudaEventCreate(&c->tev[k]) != cudaSuccess) {
                cudaGetLastError();
                return fail(c, DVM_ECUDA, "event creation failed");
            }
    c->timing = enable != 0;
    c->tms[0] = c->tms[1] = c->tms[2] = 0.0;
    c->tsteps = 0;
    return DVM_OK;
}

int dvm_step_timing(dvm_ctx *c, double *ms, int64_t *steps)
{
    if (!c || !ms) return DVM_EINVAL;
    for (int k = 0; k < 3; k++) ms[k] = c->tms[k];
    if (steps) *steps = c->tsteps;
    c->tms[0] = c->tms[1] = c->tms[2] = 0.0;
    c->tsteps = 0;
    return DVM_OK;
}

int dvm_step_residual(dvm_ctx *c, double *res)
{
    if (!c || !res) return DVM_EINVAL;
    if (!c->have_res) return fail(c, DVM_ESTATE, "no collision step has run since the grid was set");
    const int64_t nc = ncells_of(c);
    int rc = cuda_check(c, cudaMemcpyAsync(res, c->d_res, (size_t)nc * 5 * sizeof(double), cudaMemcpyDeviceToHost,
                                           c->stream), "copy residual");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "residual");
    if (rc || !c->res_pairs) return rc;
    // BGK: the kernel left sum_i phi_r (M~ - f*)_i dV, phi = (1, c, |c|^2 - 3),
    // c = (xi - u)/sqrt(T), as double-float pairs; with the step moments the
    // host takes it to psi = (1, xi, |xi|^2) (xi = sqrt(T) c + u) and to the
    // collision term q = nu (M~ - f*), nu = sqrt(8/pi) rho sqrt(T) / Kn
    std::vector<double> mom(5 * (size_t)nc);
    rc = cuda_check(c, cudaMemcpyAsync(mom.data(), c->d_mom, mom.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                       c->stream), "copy moments");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "residual");
    if (rc) return rc;
    std::vector<float> pr(10 * (size_t)nc);
    std::memcpy(pr.data(), res, pr.size() * sizeof(float));
    for (int64_t q = 0; q < nc; q++) {
        double r[5];
        for (int k = 0; k < 5; k++) r[k] = (double)pr[10 * q + 2 * k] + (double)pr[10 * q + 2 * k + 1];
        const double rho = mom[5 * q], T = mom[5 * q + 4], sT = std::sqrt(T);
        const double u[3] = {mom[5 * q + 1], mom[5 * q + 2], mom[5 * q + 3]};
        const double nu = 1.5957691216057308 * rho * sT / c->cfg.kn;
        double *o = res + 5 * q;
        o[0] = nu * r[0];
        double dot = 0.0, uu = 0.0;
        for (int d = 0; d < 3; d++) {
            o[1 + d] = nu * (sT * r[1 + d] + u[d] * r[0]);
            dot += u[d] * r[1 + d];
            uu += u[d] * u[d];
        }
        o[4] = nu * (T * (r[4] + 3.0 * r[0]) + 2.0 * sT * dot + uu * r[0]);
    }
    return DVM_OK;
}

int dvm_hs_collide_noalloc(dvm_ctx *c, float *f, int64_t ncells, double dt)
{
    if (!c || !f || ncells < 1) return DVM_EINVAL;
    if (reinterpret_cast<uintptr_t>(f) % 16)
        return fail(c, DVM_EINVAL, "f must be 16-byte aligned (each cell's row is read by one bulk copy)");
    if (c->state < 2 || !c->hs.ready) return fail(c, DVM_ESTATE, "set the velocity grid and the collision tables first");
    if (c->cfg.precision != DVM_F32) return fail(c, DVM_ENOTIMPL, "the hard-sphere operator runs on FP32 storage");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, DVM_EINVAL, "dt must be positive");
    const double need = (double)ncells * (8.0 * c->nv + 40.0);
    if (need > (double)DVM_HS_NOALLOC_SCRATCH_BYTES)
        return fail(c, DVM_EINVAL, "ncells * (8 nv + 40) bytes exceed the fixed scratch of "
                                   "DVM_HS_NOALLOC_SCRATCH_BYTES");
    dvm::StepParams p{};
    p.dim = c->mesh.spec.dim;
    p.prec = c->cfg.precision;
    p.ncells = ncells;
    p.nv = c->nv;
    p.P = c->P;
    p.status = c->d_status;
    p.stream = c->stream;
    int rc = dvm::launch_hs_collide_noalloc(c->hs, p, f, c->d_xi, c->dV, c->cfg.kn, dt);
    if (rc) return fail(c, rc, rc == DVM_EINVAL ? "scratch too small" : "hard-sphere launch failed");
    int st = 0;
    rc = cuda_check(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read status");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "hard-sphere collision");
    if (rc) return rc;
    if (st) {
        cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
        if (st & dvm::ST_TIMEOUT) return fail(c, DVM_ETIMEOUT, "a bounded wait for an asynchronous tile copy gave up");
        return fail(c, DVM_EUNSTABLE, "unstable collision update (singular correction or dt/Kn max(P B) > 1)");
    }
    return DVM_OK;
}

// ---------------------------------------------------------------- network
static int mlp_ready(dvm_ctx *c)
{
    int rc = ensure_device(c);
    if (rc) return rc;
    rc = dvm::mlp_init(c->mlp, [c](size_t b) { return dev_alloc(c, b); });
    return rc ? fail(c, rc, "device allocation (network)") : DVM_OK;
}

static int status_check(dvm_ctx *c)
{
    int st = 0;
    int rc = cuda_check(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read status");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "network");
    if (rc) return rc;
    if (st) {
        cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
        return fail(c, st & dvm::ST_TIMEOUT ? DVM_ETIMEOUT : DVM_EUNSTABLE, "network kernel reported an error");
    }
    return DVM_OK;
}

int dvm_learned_set_weights(dvm_ctx *c, const float *params)
{
    if (!c || !params) return DVM_EINVAL;
    int rc = mlp_ready(c);
    if (rc) return rc;
    rc = cuda_check(c, cudaMemcpy(c->mlp.w, params, DVM_MLP_NPARAM * 4, cudaMemcpyHostToDevice), "copy weights");
    if (!rc) rc = cuda_check(c, cudaMemset(c->mlp.m, 0, DVM_MLP_NPARAM * 4), "reset optimiser");
    if (!rc) rc = cuda_check(c, cudaMemset(c->mlp.v, 0, DVM_MLP_NPARAM * 4), "reset optimiser");
    c->mlp.steps = 0;
    if (!rc) rc = dvm::mlp_cast(c->mlp, c->stream);
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "cast weights");
    c->mlp_set = !rc;
    return rc;
}

int dvm_learned_get_weights(dvm_ctx *c, float *params)
{
    if (!c || !params) return DVM_EINVAL;
    if (!c->mlp_set) return fail(c, DVM_ESTATE, "no weights set");
    return cuda_check(c, cudaMemcpy(params, c->mlp.w, DVM_MLP_NPARAM * 4, cudaMemcpyDeviceToHost), "copy weights");
}

namespace {
struct DevArr {
    dvm_ctx *c;
    void *p = nullptr;
    DevArr(dvm_ctx *cc, size_t bytes) : c(cc) { p = dev_alloc(cc, bytes); }
    ~DevArr() { dev_free(c, p); }
    float *f() { return static_cast<float *>(p); }
};
}  // namespace

int dvm_mlp_forward(dvm_ctx *c, const float *x, int64_t n, float *y)
{
    if (!c || !x || !y || n < 1) return DVM_EINVAL;
    if (!c->mlp_set) return fail(c, DVM_ESTATE, "no weights set");
    int rc = dvm::mlp_reserve(c->mlp, n, [c](size_t b) { return dev_alloc(c, b); }, [c](void *p) { void *q = p; dev_free(c, q); });
    if (rc) return fail(c, rc, "device allocation (network work buffers)");
    DevArr dx(c, (size_t)n * 64 * 4), dy(c, (size_t)n * 64 * 4);
    if (!dx.p || !dy.p) return fail(c, DVM_ENOMEM, "device allocation (network rows)");
    rc = cuda_check(c, cudaMemcpyAsync(dx.p, x, (size_t)n * 256, cudaMemcpyHostToDevice, c->stream), "copy x");
    if (!rc) rc = dvm::mlp_forward(c->mlp, dx.f(), n, dy.f(), c->d_status, c->stream);
    if (rc) return fail(c, rc, "network forward failed");
    rc = cuda_check(c, cudaMemcpyAsync(y, dy.p, (size_t)n * 256, cudaMemcpyDeviceToHost, c->stream), "copy y");
    return rc ? rc : status_check(c);
}

int dvm_mlp_loss_grad(dvm_ctx *c, const float *x, const float *t, int64_t n, float *grad, double *loss)
{
    if (!c || !x || !t || n < 1) return DVM_EINVAL;
    if (!c->mlp_set) return fail(c, DVM_ESTATE, "no weights set");
    int rc = dvm::mlp_reserve(c->mlp, n, [c](size_t b) { return dev_alloc(c, b); }, [c](void *p) { void *q = p; dev_free(c, q); });
    if (rc) return fail(c, rc, "device allocation (network work buffers)");
    DevArr dx(c, (size_t)n * 256), dt(c, (size_t)n * 256);
    if (!dx.p || !dt.p) return fail(c, DVM_ENOMEM, "device allocation (network rows)");
    rc = cuda_check(c, cudaMemcpyAsync(dx.p, x, (size_t)n * 256, cudaMemcpyHostToDevice, c->stream), "copy x");
    if (!rc) rc = cuda_check(c, cudaMemcpyAsync(dt.p, t, (size_t)n * 256, cudaMemcpyHostToDevice, c->stream), "copy t");
    if (!rc) rc = dvm::mlp_grad(c->mlp, dx.f(), dt.f(), n, c->d_status, c->stream);
    if (rc) return fail(c, rc, "network gradient failed");
    double L = 0.0;
    rc = cuda_check(c, cudaMemcpyAsync(&L, c->mlp.loss, 8, cudaMemcpyDeviceToHost, c->stream), "copy loss");
    if (!rc && grad) rc = cuda_check(c, cudaMemcpyAsync(grad, c->mlp.g, DVM_MLP_NPARAM * 4, cudaMemcpyDeviceToHost, c->stream), "copy grad");
    if (!rc) rc = status_check(c);
    if (!rc && loss) *loss = L / ((double)n * 64.0);
    return rc;
}

int dvm_learned_train(dvm_ctx *c, const float *x, const float *t, int64_t n, int epochs, int batch, double lr,
                      uint64_t seed, double *loss)
{
    if (!c || !x || !t || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.0)) return DVM_EINVAL;
    if (!c->mlp_set) return fail(c, DVM_ESTATE, "no weights set");
    const int64_t nb = std::min<int64_t>(batch, n);
    int rc = dvm::mlp_reserve(c->mlp, nb, [c](size_t b) { return dev_alloc(c, b); }, [c](void *p) { void *q = p; dev_free(c, q); });
    if (rc) return fail(c, rc, "device allocation (network work buffers)");
    DevArr dx(c, (size_t)n * 256), dt(c, (size_t)n * 256);
    if (!dx.p || !dt.p) return fail(c, DVM_ENOMEM, "device allocation (training rows)");
    std::vector<int64_t> perm(n);
    std::vector<float> xs((size_t)n * 64), ts((size_t)n * 64);
    double last = 0.0;
    for (int e = 0; e < epochs && !rc; e++) {
        // seeded Fisher-Yates permutation of the rows
        for (int64_t q = 0; q < n; q++) perm[q] = q;
        for (int64_t q = n - 1; q > 0; q--) {
            const uint64_t r = dvm::splitmix64_at(seed + (uint64_t)e, (uint64_t)q) % (uint64_t)(q + 1);
            std::swap(perm[q], perm[(int64_t)r]);
        }
        for (int64_t q = 0; q < n; q++) {
            std::memcpy(&xs[(size_t)q * 64], x + perm[q] * 64, 256);
            std::memcpy(&ts[(size_t)q * 64], t + perm[q] * 64, 256);
        }
        rc = cuda_check(c, cudaMemcpyAsync(dx.p, xs.data(), (size_t)n * 256, cudaMemcpyHostToDevice, c->stream), "copy x");
        if (!rc) rc = cuda_check(c, cudaMemcpyAsync(dt.p, ts.data(), (size_t)n * 256, cudaMemcpyHostToDevice, c->stream), "copy t");
        double sum = 0.0;
        int64_t rows = 0;
        for (int64_t s0 = 0; s0 < n && !rc; s0 += nb) {
            const int64_t m = std::min(nb, n - s0);
            rc = dvm::mlp_grad(c->mlp, dx.f() + s0 * 64, dt.f() + s0 * 64, m, c->d_status, c->stream);
            if (!rc) rc = dvm::mlp_adam(c->mlp, lr, c->stream);
            double L = 0.0;
            if (!rc) rc = cuda_check(c, cudaMemcpyAsync(&L, c->mlp.loss, 8, cudaMemcpyDeviceToHost, c->stream), "copy loss");
            if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "train");
            sum += L;
            rows += m;
        }
        last = sum / ((double)rows * 64.0);
    }
    if (!rc) rc = status_check(c);
    if (!rc && loss) *loss = last;
    return rc;
}

int dvm_learned_configure(dvm_ctx *c, double kn_threshold)
{
    if (!c || !(kn_threshold >= 0.0)) return DVM_EINVAL;
    c->kn_thr = kn_threshold;
    c->learned_cfg = true;
    return DVM_OK;
}

int dvm_learned_collide(dvm_ctx *c, double dt, const float *o_in, double *knl, float *a, float *o, int32_t *used,
                        float *q)
{
    if (!c || !(dt > 0.0)) return DVM_EINVAL;
    if (c->state < 3) return fail(c, DVM_ESTATE, "f is not set");
    if (!c->hs.ready) return fail(c, DVM_ESTATE, "set the collision tables first");
    if (!c->learned_cfg || (!o_in && !c->mlp_set)) return fail(c, DVM_ESTATE, "set the network weights and the Knudsen threshold first");
    int rc = learned_prepare(c);
    if (rc) return rc;
    const int64_t nc = ncells_of(c);
    float *f = static_cast<float *>(c->d_f[c->cur]);
    rc = dvm::launch_moments(DVM_F32, f, nc, c->nv, c->d_xi, c->dV, c->d_mom2, c->stream);
    if (rc) return fail(c, rc, "moments launch failed");
    if (o_in) rc = cuda_check(c, cudaMemcpyAsync(c->d_lo, o_in, (size_t)nc * 256, cudaMemcpyHostToDevice, c->stream), "copy o");
    if (!rc && o_in && a)
        rc = dvm::launch_hermite_project(f, c->d_mom2, c->d_amag, nc, c->n, c->dV, 0, nullptr, nullptr, c->d_la,
                                         nullptr, c->d_status, c->stream);
    if (rc) return fail(c, rc, "projection launch failed");
    DevArr dq(c, q ? (size_t)nc * c->nv * 4 : 16);
    if (!dq.p) return fail(c, DVM_ENOMEM, "device allocation (collision term)");
    if (q) rc = cuda_check(c, cudaMemsetAsync(dq.p, 0, (size_t)nc * c->nv * 4, c->stream), "clear q");
    if (!rc) rc = learned_collide_device(c, f, c->d_mom2, dt, o_in ? c->d_lo : nullptr, q ? dq.f() : nullptr);
    if (rc) return rc;
    rc = read_status(c, "learned collision");
    if (rc) return rc;
    if (knl) rc = cuda_check(c, cudaMemcpy(knl, c->d_knl, (size_t)nc * 8, cudaMemcpyDeviceToHost), "copy Kn");
    if (!rc && a) rc = cuda_check(c, cudaMemcpy(a, c->d_la, (size_t)nc * 256, cudaMemcpyDeviceToHost), "copy a");
    if (!rc && o) rc = cuda_check(c, cudaMemcpy(o, c->d_lo, (size_t)nc * 256, cudaMemcpyDeviceToHost), "copy o");
    if (!rc && used) rc = cuda_check(c, cudaMemcpy(used, c->d_used, (size_t)nc * 4, cudaMemcpyDeviceToHost), "copy used");
    if (!rc && q) rc = cuda_check(c, cudaMemcpy(q, dq.p, (size_t)nc * c->nv * 4, cudaMemcpyDeviceToHost), "copy q");
    c->have_step_moments = false;
    c->have_res = true;
    c->res_pairs = false;
    return rc;
}

int dvm_learned_pairs(dvm_ctx *c, float *a, float *o)
{
    if (!c || !a || !o) return DVM_EINVAL;
    if (c->state < 3) return fail(c, DVM_ESTATE, "f is not set");
    if (!c->hs.ready) return fail(c, DVM_ESTATE, "set the collision tables first");
    if (c->cfg.precision != DVM_F32) return fail(c, DVM_ENOTIMPL, "training pairs need FP32 storage");
    if (!dvm::learned_grid_supported(c->n)) return fail(c, DVM_ENOTIMPL, "velocity grid not supported by the learned kernels");
    const int64_t nc = ncells_of(c);
    int rc = dvm::hs_prepare(c->hs, nc, [c](size_t b) { return dev_alloc(c, b); }, [c](void *q) { void *r = q; dev_free(c, r); });
    if (rc) return fail(c, rc, "hard-sphere scratch allocation failed");
    DevArr dq(c, (size_t)nc * c->nv * 4), da(c, (size_t)nc * 256), dout(c, (size_t)nc * 256);
    if (!dq.p || !da.p || !dout.p) return fail(c, DVM_ENOMEM, "device allocation (training pairs)");
    float *f = static_cast<float *>(c->d_f[c->cur]);
    rc = dvm::launch_moments(DVM_F32, f, nc, c->nv, c->d_xi, c->dV, c->d_mom2, c->stream);
    if (!rc) rc = dvm::launch_hermite_project(f, c->d_mom2, c->d_amag, nc, c->n, c->dV, 0, nullptr, nullptr, da.f(),
                                              nullptr, c->d_status, c->stream);
    dvm::StepParams p = collision_params(c, c->d_mom2);
    if (!rc) rc = dvm::launch_hs_general(c->hs, p, f, nullptr, nullptr, dq.f(), c->cfg.kn, 0.0);
    if (!rc) rc = dvm::launch_hermite_project(dq.f(), c->d_mom2, c->d_amag, nc, c->n, c->dV, 1, nullptr, nullptr,
                                              dout.f(), nullptr, c->d_status, c->stream);
    if (rc) return fail(c, rc, "training-pair launch failed");
    rc = read_status(c, "training pairs");
    if (!rc) rc = cuda_check(c, cudaMemcpy(a, da.p, (size_t)nc * 256, cudaMemcpyDeviceToHost), "copy a");
    if (!rc) rc = cuda_check(c, cudaMemcpy(o, dout.p, (size_t)nc * 256, cudaMemcpyDeviceToHost), "copy o");
    return rc;
}

int dvm_learned_fallback_count(dvm_ctx *c, int64_t *n)
{
    if (!c || !n) return DVM_EINVAL;
    if (!c->d_lcount) return fail(c, DVM_ESTATE, "no learned collision has run");
    int v = 0;
    int rc = cuda_check(c, cudaMemcpyAsync(&v, c->d_lcount, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "copy count");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "count");
    *n = v;
    return rc;
}

// ---------------------------------------------------------------- lattice Boltzmann

static void lbm_feq(const dvm::LbmLattice &L, double rho, const double u[3], double *out)
{
    // second-order equilibrium with c_s^2 = 1/3 (Sec. 4)
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < L.q; i++) {
        const double cu = L.c[i][0] * u[0] + L.c[i][1] * u[1] + L.c[i][2] * u[2];
        out[i] = L.w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

static void store_elem(int prec, void *base, size_t k, double v)
{
    if (prec == DVM_F64) static_cast<double *>(base)[k] = v;
    else static_cast<float *>(base)[k] = (float)v;
}

static double load_elem(int prec, const void *base, size_t k)
{
    return prec == DVM_F64 ? static_cast<const double *>(base)[k] : (double)static_cast<const float *>(base)[k];
}

// the inflow ghost column of both buffers
static int lbm_upload_ghost(dvm_ctx *c)
{
    double g[27];
    lbm_feq(c->lat, c->l_rho, c->l_u, g);
    const int prec = c->cfg.precision;
    const size_t es = elem_size(prec);
    std::vector<unsigned char> col((size_t)c->lat.q * es);
    for (int i = 0; i < c->lat.q; i++) store_elem(prec, col.data(), i, g[i]);
    const int64_t nc = ncells_of(c);
    for (int b = 0; b < 2; b++) {
        int rc = cuda_check(c, cudaMemcpy2D(static_cast<char *>(c->d_lf[b]) + nc * es, c->lbm_ld * es, col.data(), es,
                                            es, c->lat.q, cudaMemcpyHostToDevice), "upload the inflow ghost");
        if (rc) return rc;
    }
    return DVM_OK;
}

int dvm_lbm_set_lattice(dvm_ctx *c, int lattice)
{
    if (!c) return DVM_EINVAL;
    if (c->state < 1) return fail(c, DVM_ESTATE, "build the tree first");
    dvm::LbmLattice lat;
    if (!dvm::lbm_lattice(lattice, lat)) return fail(c, DVM_EINVAL, "unknown lattice");
    if ((lattice == DVM_LBM_D2Q9) != (c->mesh.spec.dim == 2))
        return fail(c, DVM_EINVAL, "D2Q9 needs a 2D tree, D3Q19 and D3Q27 a 3D tree");
    if (c->cfg.precision != DVM_F64 && c->cfg.precision != DVM_F32)
        return fail(c, DVM_ENOTIMPL, "the lattice Boltzmann step stores f in FP64 or FP32");
    int rc = ensure_device(c);
    if (rc) return rc;
    free_lbm_buffers(c);
    std::vector<uint32_t> codes, ovf;
    std::vector<uint8_t> lev;
    std::string err;
    rc = dvm::lbm_build_codes(c->mesh, codes, ovf, lev, err);
    if (rc) return fail(c, rc, err);
    const int64_t nc = ncells_of(c);
    const int64_t ld = (nc + 1 + 31) / 32 * 32;
    const size_t fb = (size_t)lat.q * ld * elem_size(c->cfg.precision);
    c->d_lf[0] = dev_alloc(c, fb);
    c->d_lf[1] = dev_alloc(c, fb);
    c->d_lcodes = dev_alloc_t<uint32_t>(c, codes.size());
    c->d_lovf = dev_alloc_t<uint32_t>(c, std::max<size_t>(ovf.size(), 1));
    c->d_llev = dev_alloc_t<uint8_t>(c, std::max<int64_t>(nc, 1));
    c->d_lmom = dev_alloc_t<double>(c, 4 * std::max<int64_t>(nc, 1));
    c->d_lstatus = dev_alloc_t<int>(c, 1);
    if (!c->d_lf[0] || !c->d_lf[1] || !c->d_lcodes || !c->d_lovf || !c->d_llev || !c->d_lmom || !c->d_lstatus) {
        free_lbm_buffers(c);
        return fail(c, DVM_ENOMEM, "device allocation (lattice Boltzmann buffers)");
    }
    rc = cuda_check(c, cudaMemcpy(c->d_lcodes, codes.data(), codes.size() * 4, cudaMemcpyHostToDevice), "copy codes");
    if (!rc && !ovf.empty())
        rc = cuda_check(c, cudaMemcpy(c->d_lovf, ovf.data(), ovf.size() * 4, cudaMemcpyHostToDevice), "copy codes");
    if (!rc) rc = cuda_check(c, cudaMemcpy(c->d_llev, lev.data(), lev.size(), cudaMemcpyHostToDevice), "copy levels");
    if (!rc) rc = cuda_check(c, cudaMemset(c->d_lf[0], 0, fb), "clear f");
    if (!rc) rc = cuda_check(c, cudaMemset(c->d_lf[1], 0, fb), "clear f");
    if (rc) {
        free_lbm_buffers(c);
        return rc;
    }
    c->lat = lat;
    c->lbm_ld = ld;
    c->lbm_novf = (int64_t)ovf.size();
    c->lcur = 0;
    c->lbm_state = 1;
    return lbm_upload_ghost(c);
}

int dvm_lbm_get_codes(const dvm_ctx *c, uint32_t *codes, uint32_t *ovf, int64_t *novf)
{
    if (!c || !novf) return DVM_EINVAL;
    if (c->state < 1) return fail(const_cast<dvm_ctx *>(c), DVM_ESTATE, "build the tree first");
    std::vector<uint32_t> cd, ov;
    std::vector<uint8_t> lev;
    std::string err;
    const int rc = dvm::lbm_build_codes(c->mesh, cd, ov, lev, err);
    if (rc) return fail(const_cast<dvm_ctx *>(c), rc, err);
    if (codes) std::memcpy(codes, cd.data(), cd.size() * 4);
    if (ovf && !ov.empty()) std::memcpy(ovf, ov.data(), ov.size() * 4);
    *novf = (int64_t)ov.size();
    return DVM_OK;
}

int dvm_lbm_lattice(int lattice, int *q, int32_t *cv, double *w)
{
    dvm::LbmLattice lat;
    if (!dvm::lbm_lattice(lattice, lat)) return DVM_EINVAL;
    if (q) *q = lat.q;
    for (int i = 0; i < lat.q; i++) {
        if (cv)
            for (int d = 0; d < 3; d++) cv[3 * i + d] = lat.c[i][d];
        if (w) w[i] = lat.w[i];
    }
    return DVM_OK;
}

int dvm_lbm_get_velocities(const dvm_ctx *c, int32_t *cv, double *w)
{
    if (!c || !cv || !w) return DVM_EINVAL;
    if (c->lbm_state < 1) return DVM_ESTATE;
    for (int i = 0; i < c->lat.q; i++) {
        for (int d = 0; d < 3; d++) cv[3 * i + d] = c->lat.c[i][d];
        w[i] = c->lat.w[i];
    }
    return DVM_OK;
}

int dvm_lbm_info(const dvm_ctx *c, int *q, int64_t *ld, int64_t *noverflow)
{
    if (!c) return DVM_EINVAL;
    if (c->lbm_state < 1) return DVM_ESTATE;
    if (q) *q = c->lat.q;
    if (ld) *ld = c->lbm_ld;
    if (noverflow) *noverflow = c->lbm_novf;
    return DVM_OK;
}

int dvm_lbm_set_inflow(dvm_ctx *c, double rho, const double u[3])
{
    if (!c || !u || !(rho > 0.0)) return DVM_EINVAL;
    if (c->lbm_state < 1) return fail(c, DVM_ESTATE, "set the lattice first");
    c->l_rho = rho;
    for (int d = 0; d < 3; d++) c->l_u[d] = u[d];
    return lbm_upload_ghost(c);
}

// host [q][ld] image in storage precision -> the current buffer
static int lbm_upload(dvm_ctx *c, const std::vector<unsigned char> &img)
{
    int rc = cuda_check(c, cudaMemcpy(c->d_lf[c->lcur], img.data(), img.size(), cudaMemcpyHostToDevice), "upload f");
    if (!rc) rc = lbm_upload_ghost(c);
    if (!rc) c->lbm_state = 2;
    return rc;
}

int dvm_lbm_init_equilibrium(dvm_ctx *c, const double *rho, const double *u)
{
    if (!c || !rho || !u) return DVM_EINVAL;
    if (c->lbm_state < 1) return fail(c, DVM_ESTATE, "set the lattice first");
    const int64_t nc = ncells_of(c), ld = c->lbm_ld;
    const int prec = c->cfg.precision;
    std::vector<unsigned char> img((size_t)c->lat.q * ld * elem_size(prec), 0);
    double g[27];
    for (int64_t q = 0; q < nc; q++) {
        lbm_feq(c->lat, rho[q], &u[3 * q], g);
        for (int i = 0; i < c->lat.q; i++) store_elem(prec, img.data(), (size_t)i * ld + q, g[i]);
    }
    return lbm_upload(c, img);
}

int dvm_lbm_set_f(dvm_ctx *c, const double *f, int64_t count)
{
    if (!c || !f) return DVM_EINVAL;
    if (c->lbm_state < 1) return fail(c, DVM_ESTATE, "set the lattice first");
    const int64_t nc = ncells_of(c), ld = c->lbm_ld;
    if (count != nc * c->lat.q) return fail(c, DVM_EINVAL, "count differs from ncells * q");
    const int prec = c->cfg.precision;
    std::vector<unsigned char> img((size_t)c->lat.q * ld * elem_size(prec), 0);
    for (int64_t q = 0; q < nc; q++)
        for (int i = 0; i < c->lat.q; i++) store_elem(prec, img.data(), (size_t)i * ld + q, f[q * c->lat.q + i]);
    return lbm_upload(c, img);
}

int dvm_lbm_get_f(dvm_ctx *c, double *f, int64_t count)
{
    if (!c || !f) return DVM_EINVAL;
    if (c->lbm_state < 2) return fail(c, DVM_ESTATE, "f is not set");
    const int64_t nc = ncells_of(c), ld = c->lbm_ld;
    if (count != nc * c->lat.q) return fail(c, DVM_EINVAL, "count differs from ncells * q");
    const int prec = c->cfg.precision;
    std::vector<unsigned char> img((size_t)c->lat.q * ld * elem_size(prec));
    int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "download f");
    if (!rc) rc = cuda_check(c, cudaMemcpy(img.data(), c->d_lf[c->lcur], img.size(), cudaMemcpyDeviceToHost), "download f");
    if (rc) return rc;
    for (int64_t q = 0; q < nc; q++)
        for (int i = 0; i < c->lat.q; i++) f[q * c->lat.q + i] = load_elem(prec, img.data(), (size_t)i * ld + q);
    return DVM_OK;
}

int dvm_lbm_dt_cfl(const dvm_ctx *c, double cfl, double *dt)
{
    if (!c || !dt || !(cfl > 0.0)) return DVM_EINVAL;
    if (c->lbm_state < 1) return DVM_ESTATE;
    int smax = 0;
    for (int i = 0; i < c->lat.q; i++) {
        int s = 0;
        for (int d = 0; d < c->mesh.spec.dim; d++) s += std::abs(c->lat.c[i][d]);
        smax = std::max(smax, s);
    }
    *dt = cfl * std::ldexp(1.0, -c->mesh.max_cell_level) / smax;
    return DVM_OK;
}

int dvm_lbm_step(dvm_ctx *c, int nsteps, double dt, double tau)
{
    if (!c || nsteps < 0 || !(dt > 0.0) || !(tau > 0.0)) return DVM_EINVAL;
    if (c->lbm_state < 2) return fail(c, DVM_ESTATE, "f is not set");
    if (dt / tau > 1.0) return fail(c, DVM_EUNSTABLE, "dt / tau above 1");
    if (nsteps == 0) return DVM_OK;
    int rc = cuda_check(c, cudaMemsetAsync(c->d_lstatus, 0, sizeof(int), c->stream), "clear status");
    if (rc) return rc;
    dvm::LbmParams p{};
    p.prec = c->cfg.precision;
    p.dim = c->mesh.spec.dim;
    p.q = c->lat.q;
    p.ncells = ncells_of(c);
    p.ld = c->lbm_ld;
    p.codes = c->d_lcodes;
    p.ovf = c->d_lovf;
    p.lev = c->d_llev;
    p.dt = dt;
    p.omega = dt / tau;
    p.status = c->d_lstatus;
    p.stream = c->stream;
    for (int s = 0; s < nsteps; s++) {
        p.f_in = c->d_lf[c->lcur];
        p.f_out = c->d_lf[c->lcur ^ 1];
        rc = dvm::launch_lbm(p);
        if (rc) return fail(c, rc, std::string("lattice Boltzmann launch: ") + cudaGetErrorString(cudaGetLastError()));
        c->lcur ^= 1;
    }
    int st = 0;
    rc = cuda_check(c, cudaMemcpyAsync(&st, c->d_lstatus, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "status");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "lattice Boltzmann step");
    if (rc) return rc;
    if (st) return fail(c, DVM_EUNSTABLE, "a cell reached rho <= 0 or non-finite moments");
    return DVM_OK;
}

int dvm_lbm_moments(dvm_ctx *c, double *rho, double *u)
{
    if (!c || !rho || !u) return DVM_EINVAL;
    if (c->lbm_state < 2) return fail(c, DVM_ESTATE, "f is not set");
    const int64_t nc = ncells_of(c);
    int rc = dvm::launch_lbm_moments(c->cfg.precision, c->lat.q, c->d_lf[c->lcur], nc, c->lbm_ld, c->d_lmom, c->stream);
    if (rc) return fail(c, rc, "lattice Boltzmann moments launch");
    std::vector<double> m((size_t)nc * 4);
    rc = cuda_check(c, cudaMemcpyAsync(m.data(), c->d_lmom, m.size() * 8, cudaMemcpyDeviceToHost, c->stream), "moments");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "moments");
    if (rc) return rc;
    for (int64_t q = 0; q < nc; q++) {
        rho[q] = m[4 * q];
        for (int d = 0; d < 3; d++) u[3 * q + d] = m[4 * q + 1 + d];
    }
    return DVM_OK;
}

int dvm_launch_count(int64_t *count)
{
    if (!count) return DVM_EINVAL;
    *count = dvm::launches_issued();
    return DVM_OK;
}

}  // extern "C"
