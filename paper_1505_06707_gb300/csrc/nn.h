// State of the learned preconditioner correction (nn.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace soft {

constexpr int NN_PARAMS = 32 * 2 * 9 + 32 + 32 * 32 * 9 + 32 + 2 * 32 * 9 + 2;   // 10434

// fields per convolution launch (the grid's z dimension)
constexpr int NN_MAX_FIELDS = 65535;

struct NNState {
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;     // FP32 master, grad, Adam
    __nv_bfloat16 *w1 = nullptr, *w2 = nullptr, *w3 = nullptr, *b3 = nullptr, *b2 = nullptr;
    __nv_bfloat16 *h1 = nullptr, *h2 = nullptr, *g1 = nullptr, *g2 = nullptr;
    float *out = nullptr, *gout = nullptr;
    void *xin = nullptr, *tgt = nullptr;
    float* part = nullptr;
    double *lpart = nullptr, *lval = nullptr;
    int* idx = nullptr;
    float *sin_ = nullptr, *sout = nullptr;
    unsigned* err = nullptr;           // tensor-core convolution wait ran out (bit 0)
    int64_t act_cap = 0, part_cap = 0, batch_cap = 0;
    int scale_cap = 0;
    int adam_t = 0;

    int init(uint64_t seed);
    int set(const float* host);
    int pack(cudaStream_t st);
    int ensure_act(int64_t npix, int fields);
    int forward_c64(const void* x, int F, int H, int W, cudaStream_t st);
    int grad(const void* x, const void* t, int F, int H, int W, cudaStream_t st);
    int train_step(const void* x, const void* t, int F, int H, int W, float lr, cudaStream_t st);
    int correct_c128(void* z, int F, int H, int W, const int* active, cudaStream_t st);
    int take_err(cudaStream_t st);     // SOFT_ERR_TIMEOUT if a convolution wait ran out (clears it)
    ~NNState();
};

}  // namespace soft
