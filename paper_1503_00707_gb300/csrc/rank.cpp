// One rank of the Morton-range partition (paper Sec. 3.3): the multi-GPU
// form of the step.  Each rank owns a contiguous range of the Morton-ordered
// cells and holds on its device only its own cells, then its halo (the cells
// of other ranks that its upwind stencils read), then the inflow ghost, in
// that order (the paper stores inner cells first, then ghost cells).  Before
// every step the halo rows are replaced by their owners' current rows: the
// library packs the rows a peer needs into a caller buffer and unpacks the
// rows received; moving the buffers between processes (NCCL or any other
// transport) and the two global reductions (minimum dt, conserved totals)
// are the caller's.  The tree is built on every rank from the same spec; the
// ranges are those of dvm_partition_info.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dvm.h"
#include "grid.hpp"
#include "kernels.hpp"
#include "mesh.hpp"
#include "partition.hpp"

struct dvm_rank {
    dvm_config cfg{};
    std::string err;
    cudaStream_t stream = nullptr;
    dvm::Mesh mesh;
    int nparts = 1, part = 0;
    std::vector<dvm::Part> parts;
    int64_t nown = 0, nhalo = 0;
    std::vector<int32_t> local;               // owned stencils in local numbering
    std::vector<std::vector<int64_t>> send;   // per peer: owned cells (global) in its halo, ascending
    std::vector<std::vector<int64_t>> recv;   // per peer: halo cells (global) it owns, ascending
    // device
    bool dev = false;
    dvm::Vgrid g;
    double fs_rho = 1.0, fs_u[3] = {0, 0, 0}, fs_T = 1.0;
    void *d_f[2] = {nullptr, nullptr};
    int cur = 0;
    bool f_set = false;
    int32_t *d_src = nullptr;
    void *d_w = nullptr, *d_invh = nullptr;
    uint8_t *d_cnt = nullptr;
    double *d_amag = nullptr, *d_xi = nullptr, *d_mom = nullptr, *d_mom2 = nullptr;
    float *d_amag_f = nullptr;
    int *d_status = nullptr;
    unsigned long long *d_counter = nullptr;
    std::vector<int64_t *> d_send, d_recv;    // per peer: local rows
    std::vector<int64_t> send_off, recv_off;
    int64_t *d_rows = nullptr;                // all peers' local rows
};

namespace {

int rfail(dvm_rank *r, int code, const std::string &msg)
{
    if (r) r->err = msg;
    return code;
}

size_t esize(int prec) { return prec == DVM_F64 ? 8 : prec == DVM_F32 ? 4 : 2; }
size_t tsize(int prec) { return prec == DVM_F64 ? 8 : 4; }

template <typename T> T *dalloc(size_t count)
{
    void *p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count * sizeof(T), 16)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<T *>(p);
}

void dfree(void *p)
{
    if (p) cudaFree(p);
}

void free_device(dvm_rank *r)
{
    for (void *p : {r->d_f[0], r->d_f[1], (void *)r->d_src, r->d_w, r->d_invh, (void *)r->d_cnt, (void *)r->d_amag,
                    (void *)r->d_xi, (void *)r->d_mom, (void *)r->d_mom2, (void *)r->d_amag_f, (void *)r->d_status,
                    (void *)r->d_rows})
        dfree(p);
    r->d_f[0] = r->d_f[1] = nullptr;
    r->d_src = nullptr;
    r->d_w = r->d_invh = nullptr;
    r->d_cnt = nullptr;
    r->d_amag = r->d_xi = r->d_mom = r->d_mom2 = nullptr;
    r->d_amag_f = nullptr;
    r->d_status = nullptr;
    r->d_counter = nullptr;
    r->d_rows = nullptr;
    r->d_send.clear();
    r->d_recv.clear();
    r->dev = false;
    r->f_set = false;
}

int check(dvm_rank *r, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return DVM_OK;
    cudaGetLastError();
    return rfail(r, DVM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

double maxwellian(double rho, const double u[3], double T, const double *x)
{
    double d2 = 0.0;
    for (int d = 0; d < 3; d++) d2 += (x[d] - u[d]) * (x[d] - u[d]);
    const double tp = 2.0 * M_PI * T;
    return rho / (tp * std::sqrt(tp)) * std::exp(-d2 / (2.0 * T));
}

// the freestream Maxwellian into the inflow ghost row of both buffers
int upload_ghost(dvm_rank *r)
{
    const int64_t row = r->nown + r->nhalo;
    std::vector<double> m(r->g.nv);
    for (int v = 0; v < r->g.nv; v++) m[v] = maxwellian(r->fs_rho, r->fs_u, r->fs_T, &r->g.xi[3 * (size_t)v]);
    double *stage = dalloc<double>(r->g.nv);
    if (!stage) return rfail(r, DVM_ENOMEM, "device allocation (freestream)");
    int rc = check(r, cudaMemcpy(stage, m.data(), r->g.nv * 8, cudaMemcpyHostToDevice), "copy freestream");
    const size_t es = esize(r->cfg.precision);
    for (int b = 0; b < 2 && !rc; b++)
        rc = dvm::launch_from_f64(r->cfg.precision, stage, static_cast<char *>(r->d_f[b]) + row * r->g.nv * es, r->g.nv,
                                  r->stream);
    if (!rc) rc = check(r, cudaStreamSynchronize(r->stream), "freestream");
    cudaFree(stage);
    return rc;
}

int read_status(dvm_rank *r)
{
    int st = 0;
    int rc = check(r, cudaMemcpyAsync(&st, r->d_status, sizeof(int), cudaMemcpyDeviceToHost, r->stream), "read status");
    if (!rc) rc = check(r, cudaStreamSynchronize(r->stream), "step");
    if (rc) return rc;
    if (!st) return DVM_OK;
    cudaMemsetAsync(r->d_status, 0, sizeof(int), r->stream);
    return rfail(r, DVM_EUNSTABLE, "unstable step (non-positive moments, singular system or nu dt > 1)");
}

}  // namespace

extern "C" {

int dvm_rank_create(dvm_rank **out, const dvm_config *cfg, const dvm_tree_spec *spec, int nparts, int part)
{
    if (!out || !cfg || !spec || nparts < 1 || part < 0 || part >= nparts) return DVM_EINVAL;
    *out = nullptr;
    if (cfg->precision < DVM_F64 || cfg->precision > DVM_BF16) return DVM_EINVAL;
    if (cfg->collision != DVM_COLL_NONE && cfg->collision != DVM_COLL_BGK && cfg->collision != DVM_COLL_BGK_ENTROPIC)
        return DVM_ENOTIMPL;
    dvm_rank *r = new (std::nothrow) dvm_rank;
    if (!r) return DVM_ENOMEM;
    r->cfg = *cfg;
    int rc = dvm::build_mesh(*spec, r->mesh, r->err);
    if (rc) {
        delete r;
        return rc;
    }
    const int64_t nc = (int64_t)r->mesh.leaf_of_cell.size();
    if (nparts > nc) {
        delete r;
        return DVM_EINVAL;
    }
    std::vector<int32_t> enc;
    dvm::encode_stencils(r->mesh.st_src, nc, enc);
    dvm::partition_cells(nc, nparts, enc, r->mesh.st_cnt, r->parts);
    r->nparts = nparts;
    r->part = part;
    const dvm::Part &pt = r->parts[part];
    r->nown = pt.c1 - pt.c0;
    r->nhalo = (int64_t)pt.ghosts.size();
    dvm::local_stencils(pt, nc, enc, r->local);
    // the plan: what this rank sends to and receives from every peer
    r->send.assign(nparts, {});
    r->recv.assign(nparts, {});
    for (int64_t s : pt.ghosts) {
        int q = 0;
        while (r->parts[q].c1 <= s) q++;
        r->recv[q].push_back(s);
    }
    for (int q = 0; q < nparts; q++) {
        if (q == part) continue;
        for (int64_t s : r->parts[q].ghosts)
            if (s >= pt.c0 && s < pt.c1) r->send[q].push_back(s);
    }
    *out = r;
    return DVM_OK;
}

void dvm_rank_destroy(dvm_rank *r)
{
    if (!r) return;
    free_device(r);
    delete r;
}

const char *dvm_rank_last_error(const dvm_rank *r) { return r ? r->err.c_str() : "null rank"; }

int dvm_rank_info(const dvm_rank *r, int64_t *ncells_global, int64_t *c0, int64_t *c1, int64_t *nhalo)
{
    if (!r) return DVM_EINVAL;
    if (ncells_global) *ncells_global = (int64_t)r->mesh.leaf_of_cell.size();
    if (c0) *c0 = r->parts[r->part].c0;
    if (c1) *c1 = r->parts[r->part].c1;
    if (nhalo) *nhalo = r->nhalo;
    return DVM_OK;
}

int dvm_rank_plan(const dvm_rank *r, int peer, int64_t *nsend, int64_t *send_cells, int64_t *nrecv, int64_t *recv_cells)
{
    if (!r || peer < 0 || peer >= r->nparts) return DVM_EINVAL;
    if (nsend) *nsend = (int64_t)r->send[peer].size();
    if (nrecv) *nrecv = (int64_t)r->recv[peer].size();
    if (send_cells) std::copy(r->send[peer].begin(), r->send[peer].end(), send_cells);
    if (recv_cells) std::copy(r->recv[peer].begin(), r->recv[peer].end(), recv_cells);
    return DVM_OK;
}

int dvm_rank_set_stream(dvm_rank *r, void *stream)
{
    if (!r) return DVM_EINVAL;
    r->stream = static_cast<cudaStream_t>(stream);
    return DVM_OK;
}

int dvm_rank_set_velocity_grid(dvm_rank *r, const int n[3], const double lo[3], const double hi[3])
{
    if (!r || !n || !lo || !hi) return DVM_EINVAL;
    int rc = dvm::make_vgrid(n, lo, hi, r->cfg.precision == DVM_F64 ? 2 : 4, r->g, r->err);
    if (rc) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return rfail(r, DVM_ECUDA, "no CUDA device available");
    }
    free_device(r);
    const int prec = r->cfg.precision;
    const size_t es = esize(prec), tcs = tsize(prec);
    const int64_t rows = r->nown + r->nhalo + 1, nv = r->g.nv;
    const int64_t c0 = r->parts[r->part].c0;
    r->d_f[0] = dalloc<char>((size_t)rows * nv * es);
    r->d_f[1] = dalloc<char>((size_t)rows * nv * es);
    r->d_src = dalloc<int32_t>((size_t)r->nown * 24);
    r->d_w = dalloc<char>((size_t)r->nown * 24 * tcs);
    r->d_invh = dalloc<char>((size_t)r->nown * tcs);
    r->d_cnt = dalloc<uint8_t>((size_t)r->nown * 8);
    r->d_amag = dalloc<double>(96);
    r->d_amag_f = dalloc<float>(96);
    r->d_xi = dalloc<double>(3 * (size_t)nv);
    r->d_mom = dalloc<double>(5 * (size_t)r->nown);
    r->d_mom2 = dalloc<double>(5 * (size_t)r->nown);
    r->d_status = dalloc<int>(4);
    int64_t nrows = 0;
    for (int q = 0; q < r->nparts; q++) nrows += (int64_t)(r->send[q].size() + r->recv[q].size());
    r->d_rows = dalloc<int64_t>((size_t)std::max<int64_t>(nrows, 1));
    r->dev = true;
    if (!r->d_f[0] || !r->d_f[1] || !r->d_src || !r->d_w || !r->d_invh || !r->d_cnt || !r->d_amag || !r->d_amag_f ||
        !r->d_xi || !r->d_mom || !r->d_mom2 || !r->d_status || !r->d_rows) {
        free_device(r);
        return rfail(r, DVM_ENOMEM, "device allocation (rank)");
    }
    r->d_counter = reinterpret_cast<unsigned long long *>(r->d_status + 2);
    rc = check(r, cudaMemset(r->d_status, 0, 16), "status");
    // owned stencils: local sources, weights, counts and 1/h of cells c0 ..
    std::vector<double> invh(r->nown), w64((size_t)r->nown * 24);
    for (int64_t q = 0; q < r->nown; q++)
        invh[q] = std::ldexp(1.0, r->mesh.leaves[r->mesh.leaf_of_cell[c0 + q]].lev);
    std::copy(r->mesh.st_w.begin() + c0 * 24, r->mesh.st_w.begin() + (c0 + r->nown) * 24, w64.begin());
    if (!rc) rc = check(r, cudaMemcpy(r->d_src, r->local.data(), r->local.size() * 4, cudaMemcpyHostToDevice), "stencils");
    if (!rc)
        rc = check(r, cudaMemcpy(r->d_cnt, r->mesh.st_cnt.data() + c0 * 8, (size_t)r->nown * 8, cudaMemcpyHostToDevice),
                   "counts");
    if (!rc && prec == DVM_F64) {
        rc = check(r, cudaMemcpy(r->d_w, w64.data(), w64.size() * 8, cudaMemcpyHostToDevice), "weights");
        if (!rc) rc = check(r, cudaMemcpy(r->d_invh, invh.data(), invh.size() * 8, cudaMemcpyHostToDevice), "1/h");
    } else if (!rc) {
        std::vector<float> wf(w64.begin(), w64.end()), hf(invh.begin(), invh.end());
        rc = check(r, cudaMemcpy(r->d_w, wf.data(), wf.size() * 4, cudaMemcpyHostToDevice), "weights");
        if (!rc) rc = check(r, cudaMemcpy(r->d_invh, hf.data(), hf.size() * 4, cudaMemcpyHostToDevice), "1/h");
    }
    if (!rc) rc = check(r, cudaMemcpy(r->d_amag, r->g.amag, sizeof r->g.amag, cudaMemcpyHostToDevice), "|xi|");
    if (!rc) rc = check(r, cudaMemcpy(r->d_amag_f, r->g.amag_f, sizeof r->g.amag_f, cudaMemcpyHostToDevice), "|xi|");
    if (!rc) rc = check(r, cudaMemcpy(r->d_xi, r->g.xi.data(), r->g.xi.size() * 8, cudaMemcpyHostToDevice), "xi");
    // the plan's local rows: owned cell s -> s - c0, halo cell -> nown + its place in the halo
    if (!rc) {
        const std::vector<int64_t> &gh = r->parts[r->part].ghosts;
        std::vector<int64_t> rowsv;
        r->send_off.assign(r->nparts, 0);
        r->recv_off.assign(r->nparts, 0);
        for (int q = 0; q < r->nparts; q++) {
            r->send_off[q] = (int64_t)rowsv.size();
            for (int64_t s : r->send[q]) rowsv.push_back(s - c0);
            r->recv_off[q] = (int64_t)rowsv.size();
            for (int64_t s : r->recv[q])
                rowsv.push_back(r->nown + (std::lower_bound(gh.begin(), gh.end(), s) - gh.begin()));
        }
        if (!rowsv.empty())
            rc = check(r, cudaMemcpy(r->d_rows, rowsv.data(), rowsv.size() * 8, cudaMemcpyHostToDevice), "plan rows");
    }
    if (!rc) rc = upload_ghost(r);
    if (rc) {
        free_device(r);
        return rc;
    }
    r->cur = 0;
    return DVM_OK;
}

int dvm_rank_set_freestream(dvm_rank *r, double rho, const double u[3], double T)
{
    if (!r || !u || !(rho > 0.0) || !(T > 0.0)) return DVM_EINVAL;
    r->fs_rho = rho;
    for (int d = 0; d < 3; d++) r->fs_u[d] = u[d];
    r->fs_T = T;
    return r->dev ? upload_ghost(r) : DVM_OK;
}

int dvm_rank_cell_centres(const dvm_rank *r, double *xyz, double *h)
{
    if (!r) return DVM_EINVAL;
    const int64_t c0 = r->parts[r->part].c0;
    for (int64_t q = 0; q < r->nown; q++) {
        const dvm::Leaf &L = r->mesh.leaves[r->mesh.leaf_of_cell[c0 + q]];
        const double e = std::ldexp(1.0, -L.lev);
        for (int d = 0; d < 3; d++)
            if (xyz) xyz[3 * q + d] = d < r->mesh.spec.dim ? (L.i[d] + 0.5) * e : 0.5;
        if (h) h[q] = e;
    }
    return DVM_OK;
}

int dvm_rank_init_maxwellian(dvm_rank *r, int nmix, const double *w, const double *rho, const double *u, const double *T)
{
    if (!r || nmix < 1 || !w || !rho || !u || !T) return DVM_EINVAL;
    if (!r->dev) return rfail(r, DVM_ESTATE, "set the velocity grid first");
    const int64_t n = r->nown * nmix;
    double *dw = dalloc<double>(n), *dr = dalloc<double>(n), *du = dalloc<double>(3 * n), *dT = dalloc<double>(n);
    int rc = (dw && dr && du && dT) ? DVM_OK : rfail(r, DVM_ENOMEM, "device allocation (initial state)");
    if (!rc) rc = check(r, cudaMemcpy(dw, w, n * 8, cudaMemcpyHostToDevice), "copy");
    if (!rc) rc = check(r, cudaMemcpy(dr, rho, n * 8, cudaMemcpyHostToDevice), "copy");
    if (!rc) rc = check(r, cudaMemcpy(du, u, 3 * n * 8, cudaMemcpyHostToDevice), "copy");
    if (!rc) rc = check(r, cudaMemcpy(dT, T, n * 8, cudaMemcpyHostToDevice), "copy");
    if (!rc)
        rc = dvm::launch_init_maxwellian(r->cfg.precision, r->d_f[r->cur], r->nown, r->g.nv, nmix, dw, dr, du, dT,
                                         r->d_xi, r->stream);
    if (!rc) rc = check(r, cudaStreamSynchronize(r->stream), "initial state");
    for (void *p : {(void *)dw, (void *)dr, (void *)du, (void *)dT}) dfree(p);
    r->f_set = rc == DVM_OK;
    return rc;
}

int dvm_rank_row_bytes(const dvm_rank *r, int64_t *bytes)
{
    if (!r || !bytes) return DVM_EINVAL;
    if (!r->dev) return DVM_ESTATE;
    *bytes = (int64_t)r->g.nv * (int64_t)esize(r->cfg.precision);
    return DVM_OK;
}

int dvm_rank_pack(dvm_rank *r, int peer, void *dev_buf)
{
    if (!r || peer < 0 || peer >= r->nparts) return DVM_EINVAL;
    if (!r->f_set) return rfail(r, DVM_ESTATE, "f is not set");
    const int64_t n = (int64_t)r->send[peer].size();
    if (n == 0) return DVM_OK;
    if (!dev_buf) return DVM_EINVAL;
    const int rc = dvm::launch_rows_indexed(true, dev_buf, r->d_f[r->cur], r->d_rows + r->send_off[peer], n,
                                            (int64_t)r->g.nv * (int64_t)esize(r->cfg.precision), r->stream);
    return rc ? rfail(r, rc, "pack launch failed") : DVM_OK;
}

int dvm_rank_unpack(dvm_rank *r, int peer, const void *dev_buf)
{
    if (!r || peer < 0 || peer >= r->nparts) return DVM_EINVAL;
    if (!r->f_set) return rfail(r, DVM_ESTATE, "f is not set");
    const int64_t n = (int64_t)r->recv[peer].size();
    if (n == 0) return DVM_OK;
    if (!dev_buf) return DVM_EINVAL;
    const int rc = dvm::launch_rows_indexed(false, r->d_f[r->cur], dev_buf, r->d_rows + r->recv_off[peer], n,
                                            (int64_t)r->g.nv * (int64_t)esize(r->cfg.precision), r->stream);
    return rc ? rfail(r, rc, "unpack launch failed") : DVM_OK;
}

int dvm_rank_dt_cfl(const dvm_rank *r, double cfl, double *dt)
{
    if (!r || !dt || !(cfl > 0.0)) return DVM_EINVAL;
    if (!r->dev) return DVM_ESTATE;
    const int dim = r->mesh.spec.dim;
    double smax = 0.0;
    for (int v = 0; v < r->g.nv; v++) {
        double s = 0.0;
        for (int d = 0; d < dim; d++) s += std::fabs(r->g.xi[3 * (size_t)v + d]);
        smax = std::max(smax, s);
    }
    int lmax = 0;
    const int64_t c0 = r->parts[r->part].c0;
    for (int64_t q = 0; q < r->nown; q++) lmax = std::max(lmax, r->mesh.leaves[r->mesh.leaf_of_cell[c0 + q]].lev);
    *dt = cfl * std::ldexp(1.0, -lmax) / smax;
    return DVM_OK;
}

int dvm_rank_step(dvm_rank *r, double dt)
{
    if (!r) return DVM_EINVAL;
    if (!r->f_set) return rfail(r, DVM_ESTATE, "f is not set");
    if (!(dt > 0.0) || !std::isfinite(dt)) return rfail(r, DVM_EINVAL, "dt must be positive");
    dvm::StepParams p{};
    p.dim = r->mesh.spec.dim;
    p.prec = r->cfg.precision;
    p.coll = r->cfg.collision;
    p.ncells = r->nown;
    p.nv = r->g.nv;
    p.P = r->g.P;
    for (int d = 0; d < 3; d++) { p.half[d] = r->g.half[d]; p.n[d] = r->g.n[d]; p.hv[d] = r->g.hv[d]; }
    p.f_in = r->d_f[r->cur];
    p.f_out = r->d_f[1 - r->cur];
    p.st_src = r->d_src;
    p.st_w = r->d_w;
    p.st_cnt = r->d_cnt;
    p.inv_h = r->d_invh;
    p.amag = r->d_amag;
    p.amag_f = r->d_amag_f;
    p.dt = dt;
    p.kn = r->cfg.kn;
    p.dV = r->g.dV;
    p.mom_out = r->d_mom;
    p.status = r->d_status;
    p.counter = r->d_counter;
    p.stream = r->stream;
    int rc = check(r, cudaMemsetAsync(r->d_counter, 0, sizeof(unsigned long long), r->stream), "counter reset");
    if (!rc) rc = dvm::launch_step(p);
    if (rc) return rc == DVM_ECUDA ? rc : rfail(r, rc, "step launch failed");
    r->cur = 1 - r->cur;
    return read_status(r);
}

int dvm_rank_moments(dvm_rank *r, double *rho, double *u, double *T)
{
    if (!r) return DVM_EINVAL;
    if (!r->f_set) return rfail(r, DVM_ESTATE, "f is not set");
    int rc = dvm::launch_moments(r->cfg.precision, r->d_f[r->cur], r->nown, r->g.nv, r->d_xi, r->g.dV, r->d_mom2,
                                 r->stream);
    if (rc) return rfail(r, rc, "moments launch failed");
    std::vector<double> h(5 * (size_t)r->nown);
    rc = check(r, cudaMemcpyAsync(h.data(), r->d_mom2, h.size() * 8, cudaMemcpyDeviceToHost, r->stream), "copy moments");
    if (!rc) rc = check(r, cudaStreamSynchronize(r->stream), "moments");
    if (rc) return rc;
    for (int64_t q = 0; q < r->nown; q++) {
        if (rho) rho[q] = h[5 * q];
        if (u)
            for (int d = 0; d < 3; d++) u[3 * q + d] = h[5 * q + 1 + d];
        if (T) T[q] = h[5 * q + 4];
    }
    return DVM_OK;
}

int dvm_rank_get_f(dvm_rank *r, double *f, int64_t count)
{
    if (!r || !f) return DVM_EINVAL;
    if (!r->f_set) return rfail(r, DVM_ESTATE, "f is not set");
    if (count != r->nown * r->g.nv) return rfail(r, DVM_EINVAL, "count must be owned cells x nv");
    double *d = dalloc<double>((size_t)count);
    if (!d) return rfail(r, DVM_ENOMEM, "device allocation (f copy)");
    int rc = dvm::launch_to_f64(r->cfg.precision, r->d_f[r->cur], d, count, r->stream);
    if (!rc) rc = check(r, cudaMemcpyAsync(f, d, (size_t)count * 8, cudaMemcpyDeviceToHost, r->stream), "copy f");
    if (!rc) rc = check(r, cudaStreamSynchronize(r->stream), "copy f");
    cudaFree(d);
    return rc;
}

int dvm_rank_totals(dvm_rank *r, double *out)
{
    if (!r || !out) return DVM_EINVAL;
    std::vector<double> rho(r->nown), u(3 * (size_t)r->nown), T(r->nown), h(r->nown);
    int rc = dvm_rank_moments(r, rho.data(), u.data(), T.data());
    if (rc) return rc;
    dvm_rank_cell_centres(r, nullptr, h.data());
    const int dim = r->mesh.spec.dim;
    for (int k = 0; k < 5; k++) out[k] = 0.0;
    for (int64_t q = 0; q < r->nown; q++) {
        const double V = std::pow(h[q], dim), m = V * rho[q];
        double uu = 0.0;
        for (int d = 0; d < 3; d++) {
            out[1 + d] += m * u[3 * q + d];
            uu += u[3 * q + d] * u[3 * q + d];
        }
        out[0] += m;
        out[4] += m * (uu + 3.0 * T[q]);
    }
    return DVM_OK;
}

}  // extern "C"
