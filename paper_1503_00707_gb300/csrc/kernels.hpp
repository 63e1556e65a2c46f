// Launch interface between the C ABI layer and the CUDA kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dvm {

// Status bits raised by the step kernels (OR-ed into one device word).
enum : int {
    ST_NONPOS = 1,      // non-positive or non-finite density/temperature
    ST_SINGULAR = 2,    // singular or non-finite 5x5 correction system
    ST_NUDT = 4,        // relaxation factor nu*dt (or dt/Kn * max P B) above 1
    ST_TIMEOUT = 8,     // a bounded wait on an asynchronous copy gave up
};

struct StepParams {
    int dim;              // 2 or 3 physical dimensions
    int prec;             // DVM_F64 / DVM_F32 / DVM_BF16
    int coll;             // DVM_COLL_NONE / DVM_COLL_BGK
    int64_t ncells;
    int nv;               // velocity nodes per cell
    int P;                // nodes per sign group = nv / 8
    int half[3];          // n[d] / 2
    int n[3];
    const void *f_in;     // [ncells + 1][nv] storage precision (last: inflow ghost)
    void *f_out;
    const int32_t *st_src;   // [ncells][6][4]: source cell | group flip << 28
    const void *st_w;        // [ncells][6][4]  compute precision
    const uint8_t *st_cnt;   // [ncells][8]
    const void *inv_h;       // [ncells]        compute precision
    const double *amag;      // [3][32] |xi| of the positive-side nodes m = 0..half-1
    const float *amag_f;     // same, rounded to FP32
    double dt, kn, dV;
    double hv[3];            // velocity spacing per axis
    double *mom_out;         // [ncells][5]: rho, u[3], T of f*
    double *res_out;         // [ncells][5] or null: sum_i psi_r q_i dV of the hard-sphere or
                             // learned collision term, psi = (1, xi, |xi|^2)
    float2 *res_phi;         // [ncells][5] or null: sum_i phi_r (M~ - f*)_i dV of the BGK
                             // step, phi = (1, c, |c|^2 - 3), as double-float pairs
    int *status;
    unsigned long long *counter;  // cell dispenser of the step kernel, zeroed before each launch
    cudaStream_t stream;
};

int launch_step(const StepParams &p);

// f[c][v] = sum_m w[c][m] M(rho[c][m], u[c][m], T[c][m]; xi_v), FP64 math
int launch_init_maxwellian(int prec, void *f, int64_t ncells, int nv, int nmix,
                           const double *w, const double *rho, const double *u,
                           const double *T, const double *xi, cudaStream_t s);

// Moments of the stored f in FP64: out [ncells][5] = rho, u[3], T
int launch_moments(int prec, const void *f, int64_t ncells, int nv, const double *xi,
                   double dV, double *out, cudaStream_t s);

// Convert count elements between storage precision and FP64.
int launch_to_f64(int prec, const void *src, double *dst, int64_t count, cudaStream_t s);
int launch_from_f64(int prec, const double *src, void *dst, int64_t count, cudaStream_t s);

// Copies of whole rows (one cell's f) between buffers: rows [n][4] =
// {destination buffer, row, source buffer, row} indexing bufs (device arrays).
int launch_copy_rows(void *const *bufs, const int64_t *rows, int64_t n, int64_t row_bytes, cudaStream_t s);

// gather: dst row r = src row idx[r]; scatter: dst row idx[r] = src row r
// (n rows of row_bytes, a multiple of 16).
int launch_rows_indexed(bool gather, void *dst, const void *src, const int64_t *idx, int64_t n, int64_t row_bytes,
                        cudaStream_t s);

// dst row r = mean of src rows idx[start[r] .. start[r+1]) (nv values per row).
int launch_mean_rows(int prec, void *dst, const void *src, const int64_t *start, const int64_t *idx, int64_t nrows,
                     int nv, cudaStream_t s);

int64_t launches_issued();

}  // namespace dvm
