// The learned correction to the FFT preconditioner: a 2 -> 32 -> 32 -> 2
// 3x3 convolution network (ReLU between layers, periodic padding) whose
// output is added to z = P^-1 r inside a flexible CG.  Forward and
// backward-data passes run on the tensor cores (tcgen05 for the layers with
// 32 input channels, conv_tc.cuh; mma.sync for those with 2, conv.cuh); weight gradients,
// the loss and Adam are plain reductions here.  Parameters are FP32 masters
// with BF16 copies packed for the convolution kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>

#include "conv.cuh"
#include "conv_tc.cuh"
#include "nn.h"
#include "plan_internal.h"

namespace soft {

// parameter offsets in the FP32 master vector
constexpr int P_W1 = 0, P_B1 = P_W1 + 32 * 2 * 9, P_W2 = P_B1 + 32, P_B2 = P_W2 + 32 * 32 * 9,
              P_W3 = P_B2 + 32, P_B3 = P_W3 + 2 * 32 * 9, P_TOTAL = P_B3 + 2;
static_assert(P_TOTAL == NN_PARAMS, "parameter layout");

// bf16 packed weights: rows o (padded), row pitch K + 8, k = tap-major
constexpr int PK1 = 32 * ConvK<2>::KPITCH;     // layer 1 forward (CIN 2, COUT 32)
constexpr int PK2 = 32 * ConvK<32>::KPITCH;    // layer 2 forward
constexpr int PK3 = 8 * ConvK<32>::KPITCH;     // layer 3 forward (COUT 2 padded to 8)
constexpr int PB3 = 32 * ConvK<2>::KPITCH;     // layer 3 backward-data (CIN 2, COUT 32)
constexpr int PB2 = 32 * ConvK<32>::KPITCH;    // layer 2 backward-data

__global__ void pack_kernel(const float* __restrict__ P, __nv_bfloat16* __restrict__ w1,
                            __nv_bfloat16* __restrict__ w2, __nv_bfloat16* __restrict__ w3,
                            __nv_bfloat16* __restrict__ b3, __nv_bfloat16* __restrict__ b2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int K1 = ConvK<2>::KPITCH, K2 = ConvK<32>::KPITCH;
    // forward layer 1: W1[o][c][tap] at k = 2 tap + c
    if (i < PK1) {
        const int o = i / K1, k = i % K1;
        float v = 0.f;
        if (k < 18) v = P[P_W1 + (o * 2 + (k % 2)) * 9 + k / 2];
        w1[i] = __float2bfloat16(v);
    }
    // forward layer 2: W2[o][c][tap] at k = 32 tap + c
    if (i < PK2) {
        const int o = i / K2, k = i % K2;
        float v = 0.f;
        if (k < 288) v = P[P_W2 + (o * 32 + (k % 32)) * 9 + k / 32];
        w2[i] = __float2bfloat16(v);
        // backward-data layer 2: W'[i][o][t] = W2[o][i][8 - t], k = 32 t + o
        float vb = 0.f;
        if (k < 288) vb = P[P_W2 + ((k % 32) * 32 + o) * 9 + (8 - k / 32)];
        b2[i] = __float2bfloat16(vb);
    }
    // forward layer 3 (rows 2..7 zero)
    if (i < PK3) {
        const int o = i / K2, k = i % K2;
        float v = 0.f;
        if (o < 2 && k < 288) v = P[P_W3 + (o * 32 + (k % 32)) * 9 + k / 32];
        w3[i] = __float2bfloat16(v);
    }
    // backward-data layer 3: output channel i (of 32), input o (of 2): W'[i][o][t] = W3[o][i][8 - t], k = 2 t + o
    if (i < PB3) {
        const int ii = i / K1, k = i % K1;
        float v = 0.f;
        if (k < 18) v = P[P_W3 + ((k % 2) * 32 + ii) * 9 + (8 - k / 2)];
        b3[i] = __float2bfloat16(v);
    }
}

// Weight and bias gradients of one layer as per-CTA partials:
// dW[o][c][tap] += sum_p g[p][o] in[p + tap][c], db[o] += sum_p g[p][o].
// CTA = (field, band of ROWS rows); each thread owns a set of (o, c, tap).
template <int CIN, int COUT, int INK, int GK /*0 bf16 NHWC, 1 float2 [H][W][2]*/>
__global__ void __launch_bounds__(256)
wgrad_kernel(const void* __restrict__ in, const void* __restrict__ gout, int H, int W, int rows,
             float* __restrict__ part /* [gridDim.x * gridDim.y][COUT*CIN*9 + COUT] */)
{
    constexpr int NW = COUT * CIN * 9, NP = NW + COUT;
    constexpr int PER = (NP + 255) / 256;
    const int f = blockIdx.y, r0 = blockIdx.x * rows;
    extern __shared__ float sm[];
    float* tin = sm;                        // [3][W+2][CIN]
    float* tg = sm + 3 * (W + 2) * CIN;     // [W][COUT]
    float acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q] = 0.f;
    for (int y = r0; y < r0 + rows && y < H; ++y) {
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * (W + 2) * CIN; i += blockDim.x) {
            const int c = i % CIN, px = (i / CIN) % (W + 2), r = i / (CIN * (W + 2));
            const int yy = (y + r - 1 + H) % H, xx = (px - 1 + W) % W;
            const int64_t pix = (int64_t)f * H * W + (int64_t)yy * W + xx;
            float v;
            if (INK == IN_BF16) v = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(in)[pix * CIN + c]);
            else v = reinterpret_cast<const float*>(in)[pix * 2 + c];
            tin[i] = v;
        }
        for (int i = threadIdx.x; i < W * COUT; i += blockDim.x) {
            const int64_t pix = (int64_t)f * H * W + (int64_t)y * W + i / COUT;
            float v;
            if (GK == 0) v = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(gout)[pix * COUT + i % COUT]);
            else v = reinterpret_cast<const float*>(gout)[pix * 2 + i % COUT];
            tg[i] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int id = threadIdx.x + q * 256;
            if (id >= NP) continue;
            float s = 0.f;
            if (id < NW) {
                const int tap = id % 9, c = (id / 9) % CIN, o = id / (9 * CIN);
                const int dy = tap / 3 - 1, dx = tap % 3 - 1;
                const float* src = tin + ((dy + 1) * (W + 2) + dx + 1) * CIN + c;
                for (int x = 0; x < W; ++x) s += tg[x * COUT + o] * src[x * CIN];
            } else {
                const int o = id - NW;
                for (int x = 0; x < W; ++x) s += tg[x * COUT + o];
            }
            acc[q] += s;
        }
    }
    const int64_t cta = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int id = threadIdx.x + q * 256;
        if (id < NP) part[cta * NP + id] = acc[q];
    }
}

// sum the CTA partials of one layer into the gradient vector (fixed order)
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int ncta, int np, int nw,
                                    float* __restrict__ gW, float* __restrict__ gb) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= np) return;
    double s = 0;
    for (int c = 0; c < ncta; ++c) s += part[(int64_t)c * np + id];
    if (id < nw) gW[id] = (float)s;
    else gb[id - nw] = (float)s;
}

// loss = mean |out - target|^2 over all elements; gout = 2 (out - target)/n
__global__ void loss_kernel(const float* __restrict__ out, const float* __restrict__ tgt, int64_t n,
                            float* __restrict__ gout, double* __restrict__ loss_part) {
    __shared__ double red[8];
    double acc = 0;
    const float inv = 2.0f / (float)n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = out[i] - tgt[i];
        gout[i] = inv * d;
        acc += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        loss_part[blockIdx.x] = s;
    }
}

__global__ void loss_reduce_kernel(const double* __restrict__ part, int np, int64_t n, double* __restrict__ out) {
    double s = 0;
    for (int i = 0; i < np; ++i) s += part[i];
    *out = s / (double)n;
}

__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                            float* __restrict__ V, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// gather minibatch crops: dst[b] = src[idx[b]] (complex64 fields)
__global__ void gather_kernel(const float2* __restrict__ src, const int* __restrict__ idx, int64_t fsz,
                              float2* __restrict__ dst, int B) {
    const int b = blockIdx.y;
    const int64_t o = (int64_t)idx[b] * fsz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < fsz; i += (int64_t)gridDim.x * blockDim.x)
        dst[(int64_t)b * fsz + i] = src[o + i];
}

// per-field RMS of a complex128 field: scale_in = 1/rms, scale_out = rms
__global__ void rms_kernel(const double2* __restrict__ z, int64_t N, const int* __restrict__ active,
                           float* __restrict__ sin_, float* __restrict__ sout) {
    const int f = blockIdx.x;
    if (active && !active[f]) return;
    __shared__ double red[32];
    double acc = 0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double2 v = z[(int64_t)f * N + i];
        acc += v.x * v.x + v.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        const double rms = sqrt(s / (2.0 * (double)N));
        sin_[f] = rms > 0 ? (float)(1.0 / rms) : 0.f;
        sout[f] = (float)rms;
    }
}

// ------------------------------------------------------------------ state
NNState::~NNState() {
    void* v[] = {P, G, M, V, w1, w2, w3, b3, b2, h1, h2, g1, g2, out, gout, xin, tgt, part,
                 lpart, lval, idx, sin_, sout, err};
    for (void* b : v) cudaFree(b);
}

static int nn_alloc(void** p, size_t bytes) { return cuda_status(cudaMalloc(p, bytes)); }

int NNState::init(uint64_t seed) {
    int rc;
    if ((rc = nn_alloc((void**)&P, sizeof(float) * NN_PARAMS))) return rc;
    if ((rc = nn_alloc((void**)&G, sizeof(float) * NN_PARAMS))) return rc;
    if ((rc = nn_alloc((void**)&M, sizeof(float) * NN_PARAMS))) return rc;
    if ((rc = nn_alloc((void**)&V, sizeof(float) * NN_PARAMS))) return rc;
    if ((rc = nn_alloc((void**)&w1, sizeof(__nv_bfloat16) * PK1))) return rc;
    if ((rc = nn_alloc((void**)&w2, sizeof(__nv_bfloat16) * PK2))) return rc;
    if ((rc = nn_alloc((void**)&w3, sizeof(__nv_bfloat16) * PK3))) return rc;
    if ((rc = nn_alloc((void**)&b3, sizeof(__nv_bfloat16) * PB3))) return rc;
    if ((rc = nn_alloc((void**)&b2, sizeof(__nv_bfloat16) * PB2))) return rc;
    if ((rc = nn_alloc((void**)&lval, sizeof(double)))) return rc;
    if ((rc = nn_alloc((void**)&err, sizeof(unsigned)))) return rc;
    if ((rc = cuda_status(cudaMemset(err, 0, sizeof(unsigned))))) return rc;
    // He-style initial weights, small last layer (the correction starts near 0)
    std::vector<float> h(NN_PARAMS, 0.f);
    std::mt19937_64 gen(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    for (int i = 0; i < 32 * 2 * 9; ++i) h[P_W1 + i] = nd(gen) * std::sqrt(2.f / 18.f);
    for (int i = 0; i < 32 * 32 * 9; ++i) h[P_W2 + i] = nd(gen) * std::sqrt(2.f / 288.f);
    for (int i = 0; i < 2 * 32 * 9; ++i) h[P_W3 + i] = 0.1f * nd(gen) * std::sqrt(2.f / 288.f);
    return set(h.data());
}

int NNState::set(const float* host) {
    int rc;
    if ((rc = cuda_status(cudaMemcpy(P, host, sizeof(float) * NN_PARAMS, cudaMemcpyHostToDevice)))) return rc;
    cudaMemset(M, 0, sizeof(float) * NN_PARAMS);
    cudaMemset(V, 0, sizeof(float) * NN_PARAMS);
    adam_t = 0;
    return pack(0);
}

int NNState::pack(cudaStream_t st) {
    const int n = std::max(std::max(PK1, PK2), std::max(PK3, PB3));
    pack_kernel<<<(n + 255) / 256, 256, 0, st>>>(P, w1, w2, w3, b3, b2);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

int NNState::ensure_act(int64_t npix, int fields) {
    if (npix <= act_cap) return SOFT_OK;
    void* v[] = {h1, h2, g1, g2, out, gout};
    for (void* b : v) cudaFree(b);
    h1 = h2 = g1 = g2 = nullptr; out = gout = nullptr;
    int rc;
    if ((rc = nn_alloc((void**)&h1, sizeof(__nv_bfloat16) * 32 * npix))) return rc;
    if ((rc = nn_alloc((void**)&h2, sizeof(__nv_bfloat16) * 32 * npix))) return rc;
    if ((rc = nn_alloc((void**)&g1, sizeof(__nv_bfloat16) * 32 * npix))) return rc;
    if ((rc = nn_alloc((void**)&g2, sizeof(__nv_bfloat16) * 32 * npix))) return rc;
    if ((rc = nn_alloc((void**)&out, sizeof(float) * 2 * npix))) return rc;
    if ((rc = nn_alloc((void**)&gout, sizeof(float) * 2 * npix))) return rc;
    act_cap = npix;
    (void)fields;
    return SOFT_OK;
}

static ConvArgs cargs(const void* in, const __nv_bfloat16* w, const float* bias, void* out, int H, int W,
                      unsigned* err = nullptr) {
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.in = in; a.w = w; a.bias = bias; a.out = out; a.H = H; a.W = W; a.err = err;
    a.field_stride_in = a.field_stride_out = (int64_t)H * W;
    return a;
}

int NNState::take_err(cudaStream_t st) {
    unsigned h = 0;
    int rc;
    if ((rc = cuda_status(cudaMemcpyAsync(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st)))) return rc;
    if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
    if (!h) return SOFT_OK;
    if ((rc = cuda_status(cudaMemsetAsync(err, 0, sizeof(unsigned), st)))) return rc;
    return SOFT_ERR_TIMEOUT;
}

// forward of a batch of complex64 fields [F][H][W] -> out float2 [F][H][W]
int NNState::forward_c64(const void* x, int F, int H, int W, cudaStream_t st) {
    int rc;
    ConvArgs a = cargs(x, w1, P + P_B1, h1, H, W);
    if ((rc = launch_conv<2, 32, IN_C64, OUT_BF16_RELU>(a, F, st))) return SOFT_ERR_CUDA;
    a = cargs(h1, w2, P + P_B2, h2, H, W, err);
    if ((rc = launch_conv32_tc<32, OUT_BF16_RELU>(a, F, st))) return SOFT_ERR_CUDA;
    a = cargs(h2, w3, P + P_B3, out, H, W, err);
    if ((rc = launch_conv32_tc<2, OUT_F32>(a, F, st))) return SOFT_ERR_CUDA;
    return SOFT_OK;
}

template <int CIN, int COUT, int INK, int GK>
static int wgrad(NNState& S, const void* in, const void* g, int F, int H, int W, float* gW, float* gb,
                 cudaStream_t st) {
    constexpr int NP = COUT * CIN * 9 + COUT;
    const int rows = 16;
    dim3 grid((H + rows - 1) / rows, F);
    const int64_t ncta = (int64_t)grid.x * grid.y;
    if (ncta * NP > S.part_cap) {
        cudaFree(S.part);
        S.part = nullptr;
        int rc = nn_alloc((void**)&S.part, sizeof(float) * ncta * NP);
        if (rc) return rc;
        S.part_cap = ncta * NP;
    }
    const size_t smem = sizeof(float) * (3 * (W + 2) * CIN + W * COUT);
    auto k = wgrad_kernel<CIN, COUT, INK, GK>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SOFT_ERR_CUDA;
    k<<<grid, 256, smem, st>>>(in, g, H, W, rows, S.part);
    wgrad_reduce_kernel<<<(NP + 255) / 256, 256, 0, st>>>(S.part, (int)ncta, NP, NP - COUT, gW, gb);
    return cudaGetLastError() == cudaSuccess ? SOFT_OK : SOFT_ERR_CUDA;
}

// loss and parameter gradient G of the batch x (complex64 [F][H][W]) with targets t
int NNState::grad(const void* x, const void* t, int F, int H, int W, cudaStream_t st) {
    int rc;
    if ((rc = forward_c64(x, F, H, W, st))) return rc;
    const int64_t n = (int64_t)F * H * W * 2;
    if (!lpart && (rc = nn_alloc((void**)&lpart, sizeof(double) * 256))) return rc;
    loss_kernel<<<256, 256, 0, st>>>(out, (const float*)t, n, gout, lpart);
    loss_reduce_kernel<<<1, 1, 0, st>>>(lpart, 256, n, lval);
    // layer 3: weight gradient, then the data gradient through ReLU of h2
    if ((rc = wgrad<32, 2, IN_BF16, 1>(*this, h2, gout, F, H, W, G + P_W3, G + P_B3, st))) return rc;
    ConvArgs a = cargs(gout, b3, nullptr, g2, H, W);
    a.mask = h2;
    if ((rc = launch_conv<2, 32, IN_C64, OUT_BF16_MASK>(a, F, st))) return SOFT_ERR_CUDA;
    // layer 2
    if ((rc = wgrad<32, 32, IN_BF16, 0>(*this, h1, g2, F, H, W, G + P_W2, G + P_B2, st))) return rc;
    a = cargs(g2, b2, nullptr, g1, H, W, err);
    a.mask = h1;
    if ((rc = launch_conv32_tc<32, OUT_BF16_MASK>(a, F, st))) return SOFT_ERR_CUDA;
    // layer 1
    return wgrad<2, 32, IN_C64, 0>(*this, x, g1, F, H, W, G + P_W1, G + P_B1, st);
}

// one Adam step on the batch
int NNState::train_step(const void* x, const void* t, int F, int H, int W, float lr, cudaStream_t st) {
    int rc;
    if ((rc = grad(x, t, F, H, W, st))) return rc;
    ++adam_t;
    const float b1 = 0.9f, b2_ = 0.999f;
    adam_kernel<<<(NN_PARAMS + 255) / 256, 256, 0, st>>>(P, G, M, V, NN_PARAMS, lr, b1, b2_, 1e-8f,
                                                         1.f - std::pow(b1, (float)adam_t),
                                                         1.f - std::pow(b2_, (float)adam_t));
    if (cudaGetLastError() != cudaSuccess) return SOFT_ERR_CUDA;
    return pack(st);
}

// z += rms(z) NN(z / rms(z)) for the active complex128 fields [F][H][W]
int NNState::correct_c128(void* z, int F, int H, int W, const int* active, cudaStream_t st) {
    int rc;
    if (F > NN_MAX_FIELDS) return SOFT_ERR_TOO_LARGE;
    if ((rc = ensure_act((int64_t)F * H * W, F))) return rc;
    if (F > scale_cap) {
        cudaFree(sin_); cudaFree(sout);
        sin_ = sout = nullptr;
        if ((rc = nn_alloc((void**)&sin_, sizeof(float) * F))) return rc;
        if ((rc = nn_alloc((void**)&sout, sizeof(float) * F))) return rc;
        scale_cap = F;
    }
    rms_kernel<<<F, 512, 0, st>>>((const double2*)z, (int64_t)H * W, active, sin_, sout);
    ConvArgs a = cargs(z, w1, P + P_B1, h1, H, W);
    a.in_scale = sin_; a.active = active;
    if ((rc = launch_conv<2, 32, IN_C128, OUT_BF16_RELU>(a, F, st))) return SOFT_ERR_CUDA;
    a = cargs(h1, w2, P + P_B2, h2, H, W, err);
    a.active = active;
    if ((rc = launch_conv32_tc<32, OUT_BF16_RELU>(a, F, st))) return SOFT_ERR_CUDA;
    a = cargs(h2, w3, P + P_B3, z, H, W, err);
    a.active = active; a.out_scale = sout;
    if ((rc = launch_conv32_tc<2, OUT_ADD_C128>(a, F, st))) return SOFT_ERR_CUDA;
    return SOFT_OK;
}

}  // namespace soft

// ------------------------------------------------------------------- ABI
using namespace soft;

static NNState* nn_of(soft_plan* P, int* rc) {
    *rc = SOFT_OK;
    if (!P || P->kind != 2) { *rc = SOFT_ERR_INVALID_ARG; return nullptr; }
    if (!P->nn) {
        P->nn = new NNState();
        if ((*rc = P->nn->init(1505))) return nullptr;
    }
    return P->nn;
}

extern "C" {

static int sse_nn_set_weights_impl(soft_plan* P, const float* w) {
    int rc;
    NNState* S = nn_of(P, &rc);
    if (!S) return rc;
    if (!w) return SOFT_ERR_INVALID_ARG;
    return S->set(w);
}
int sse_nn_set_weights(soft_plan* P, const float* w) {
    return abi_guard([&] { return sse_nn_set_weights_impl(P, w); });
}

static int sse_nn_get_weights_impl(soft_plan* P, float* w) {
    int rc;
    NNState* S = nn_of(P, &rc);
    if (!S) return rc;
    if (!w) return SOFT_ERR_INVALID_ARG;
    return cuda_status(cudaMemcpy(w, S->P, sizeof(float) * NN_PARAMS, cudaMemcpyDeviceToHost));
}
int sse_nn_get_weights(soft_plan* P, float* w) {
    return abi_guard([&] { return sse_nn_get_weights_impl(P, w); });
}

static int sse_nn_forward_impl(soft_plan* P, const void* x, int nfields, int H, int W, void* out, void* stream) {
    int rc;
    NNState* S = nn_of(P, &rc);
    if (!S) return rc;
    if (!x || !out || nfields <= 0 || H < 3 || W < 128 || W % 128) return SOFT_ERR_INVALID_ARG;
    if (nfields > NN_MAX_FIELDS) return SOFT_ERR_TOO_LARGE;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = S->ensure_act((int64_t)nfields * H * W, nfields))) return rc;
    if ((rc = S->forward_c64(x, nfields, H, W, st))) return rc;
    return cuda_status(cudaMemcpyAsync(out, S->out, sizeof(float) * 2 * (size_t)nfields * H * W,
                                       cudaMemcpyDeviceToDevice, st));
}
int sse_nn_forward(soft_plan* P, const void* x, int nfields, int H, int W, void* out, void* stream) {
    return abi_guard([&] { return sse_nn_forward_impl(P, x, nfields, H, W, out, stream); });
}

static int sse_nn_grad_impl(soft_plan* P, const void* inputs, const void* targets, int n, int H, int W,
                            float* grad_out, double* loss_out, void* stream) {
    int rc;
    NNState* S = nn_of(P, &rc);
    if (!S) return rc;
    if (!inputs || !targets || !grad_out || n <= 0 || H < 3 || W < 128 || W % 128) return SOFT_ERR_INVALID_ARG;
    if (n > NN_MAX_FIELDS) return SOFT_ERR_TOO_LARGE;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = S->ensure_act((int64_t)n * H * W, n))) return rc;
    if ((rc = S->grad(inputs, targets, n, H, W, st))) return rc;
    if ((rc = cuda_status(cudaMemcpyAsync(grad_out, S->G, sizeof(float) * NN_PARAMS, cudaMemcpyDeviceToHost, st)))) return rc;
    double l = 0;
    if ((rc = cuda_status(cudaMemcpyAsync(&l, S->lval, sizeof(double), cudaMemcpyDeviceToHost, st)))) return rc;
    if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
    if ((rc = S->take_err(st))) return rc;
    if (loss_out) *loss_out = l;
    return SOFT_OK;
}
int sse_nn_grad(soft_plan* P, const void* inputs, const void* targets, int n, int H, int W,
                float* grad_out, double* loss_out, void* stream) {
    return abi_guard([&] { return sse_nn_grad_impl(P, inputs, targets, n, H, W, grad_out, loss_out, stream); });
}

static int sse_nn_train_impl(soft_plan* P, const void* inputs, const void* targets, int ncrops, int H, int W,
                             int steps, int batch, double lr, uint64_t seed, double* loss_out, void* stream) {
    int rc;
    NNState* S = nn_of(P, &rc);
    if (!S) return rc;
    if (!inputs || !targets || ncrops <= 0 || steps <= 0 || batch <= 0 || !(lr > 0) || H < 3 ||
        W < 128 || W % 128)
        return SOFT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int B = std::min(batch, ncrops);
    if (B > NN_MAX_FIELDS) return SOFT_ERR_TOO_LARGE;
    const int64_t fsz = (int64_t)H * W;
    if ((rc = S->ensure_act((int64_t)B * fsz, B))) return rc;
    if (B * fsz > S->batch_cap) {
        cudaFree(S->xin); cudaFree(S->tgt);
        S->xin = S->tgt = nullptr;
        if ((rc = nn_alloc((void**)&S->xin, sizeof(float2) * B * fsz))) return rc;
        if ((rc = nn_alloc((void**)&S->tgt, sizeof(float2) * B * fsz))) return rc;
        S->batch_cap = B * fsz;
    }
    // minibatch indices for every step, drawn on the host from the seed
    std::vector<int> idx((size_t)steps * B);
    std::mt19937_64 gen(seed);
    for (int s = 0; s < steps; ++s) {
        std::vector<int> perm(ncrops);
        for (int i = 0; i < ncrops; ++i) perm[i] = i;
        for (int i = 0; i < B; ++i) {
            std::uniform_int_distribution<int> u(i, ncrops - 1);
            std::swap(perm[i], perm[u(gen)]);
            idx[(size_t)s * B + i] = perm[i];
        }
    }
    cudaFree(S->idx);
    S->idx = nullptr;
    if ((rc = upload((void**)&S->idx, idx.data(), idx.size() * sizeof(int)))) return rc;
    std::vector<double> losses(steps);
    for (int s = 0; s < steps; ++s) {
        gather_kernel<<<dim3(64, B), 256, 0, st>>>((const float2*)inputs, S->idx + (size_t)s * B, fsz,
                                                   (float2*)S->xin, B);
        gather_kernel<<<dim3(64, B), 256, 0, st>>>((const float2*)targets, S->idx + (size_t)s * B, fsz,
                                                   (float2*)S->tgt, B);
        if ((rc = S->train_step(S->xin, S->tgt, B, H, W, (float)lr, st))) return rc;
        if (loss_out)
            if ((rc = cuda_status(cudaMemcpyAsync(&losses[s], S->lval, sizeof(double), cudaMemcpyDeviceToHost, st))))
                return rc;
    }
    if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
    if ((rc = S->take_err(st))) return rc;
    if (loss_out) std::memcpy(loss_out, losses.data(), sizeof(double) * steps);
    return SOFT_OK;
}
int sse_nn_train(soft_plan* P, const void* inputs, const void* targets, int ncrops, int H, int W,
                 int steps, int batch, double lr, uint64_t seed, double* loss_out, void* stream) {
    return abi_guard([&] { return sse_nn_train_impl(P, inputs, targets, ncrops, H, W, steps, batch, lr, seed, loss_out, stream); });
}

}  // extern "C"
