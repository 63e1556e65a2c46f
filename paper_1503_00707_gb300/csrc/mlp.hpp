// Device state of the learned collision operator's network.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <functional>

namespace dvm {

// 64 -> 256 -> 256 -> 256 -> 64; flat parameter order W1[256][64] b1[256]
// W2[256][256] b2 W3[256][256] b3 W4[64][256] b4[64] (W[out][in]).
constexpr int64_t MLP_NPARAM = 164672;

enum { W_X = 0, W_XT, W_Z, W_H, W_HT, W_O, W_T, W_DO, W_DOT, W_DOF, W_DH, W_DZ, W_DZT, W_DZF, MLP_NWORK };

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    void reset(const std::function<void(void *)> &dfree)
    {
        if (p) dfree(p);
        p = nullptr;
        bytes = 0;
    }
};

struct Mlp {
    bool ready = false;
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;  // FP32 master, Adam moments, gradient
    double *loss = nullptr;
    __nv_bfloat16 *W[4] = {nullptr, nullptr, nullptr, nullptr};    // [out][in]
    __nv_bfloat16 *WT[4] = {nullptr, nullptr, nullptr, nullptr};   // [in][out]
    int64_t steps = 0;
    int64_t cap = 0;  // rows the work buffers hold (multiple of 64)
    DevBuf work[MLP_NWORK];
};

using DevAllocF = std::function<void *(size_t)>;
using DevFreeF = std::function<void(void *)>;

int mlp_init(Mlp &m, const DevAllocF &alloc);
void mlp_free(Mlp &m, const DevFreeF &dfree);
int mlp_cast(Mlp &m, cudaStream_t s);                    // master -> BF16 copies
int mlp_reserve(Mlp &m, int64_t n, const DevAllocF &alloc, const DevFreeF &dfree);
int mlp_forward(Mlp &m, const float *x_dev, int64_t n, float *y_dev, int *status, cudaStream_t s);
int mlp_grad(Mlp &m, const float *x_dev, const float *t_dev, int64_t n, int *status, cudaStream_t s);
int mlp_adam(Mlp &m, double lr, cudaStream_t s);

}  // namespace dvm
