// 3x3 convolution with periodic padding as an implicit GEMM on the tensor
// cores (BF16 inputs, FP32 accumulation, warp-level mma.sync m16n8k16).
// The network uses it for the layers with 2 input channels; the layers with
// 32 input channels run on tcgen05 (conv_tc.cuh).
//
//   out[p][o] = b[o] + sum_k A[p][k] W[o][k],  k = (tap, c):
//     CIN = 32: k = 32 tap + c   (K = 288)
//     CIN = 2:  k = 2 tap + c    (K = 18, zero-padded to 32)
//   A[p][k] = in[(y + dy)][(x + dx)][c] with (dy, dx) = tap, indices mod H, W.
//
// One CTA computes ROWS consecutive row segments of 128 pixels of one field
// (8 warps x 16 pixels per row) for all output channels; the input rows
// y0-1 .. y0+ROWS (with a one pixel halo) and the weights are staged in
// shared memory with padded pitches so that the fragment loads are
// bank-conflict free.  Several rows per CTA read each input row (ROWS+2)/ROWS
// times instead of three times.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace soft {

enum ConvIn { IN_BF16 = 0, IN_C128 = 1, IN_C64 = 2 };
enum ConvOut { OUT_BF16_RELU = 0, OUT_F32 = 1, OUT_ADD_C128 = 2, OUT_BF16_MASK = 3 };

struct ConvArgs {
    const void* in;            // IN_BF16: bf16 [F][H][W][CIN]; IN_C128/C64: complex field [F][H][W]
    const float* in_scale;     // per-field multiplier of complex inputs (NULL = 1)
    const __nv_bfloat16* w;    // [COUTP][KPITCH] (padded rows)
    const float* bias;         // [COUT] (NULL: none)
    void* out;                 // per ConvOut
    const float* out_scale;    // per-field multiplier of OUT_ADD_C128 (NULL = 1)
    const __nv_bfloat16* mask; // OUT_BF16_MASK: the forward activation [F][H][W][COUT]
    const int* active;         // per-field flags (NULL: all)
    unsigned* err;             // bit 0 set by a tensor-core CTA whose completion wait ran out (NULL: none)
    int H, W;
    int64_t field_stride_in, field_stride_out;   // elements (pixels) per field
};

template <int CIN> struct ConvK {
    static constexpr int K = CIN == 2 ? 32 : 9 * CIN;       // padded GEMM depth
    static constexpr int KPITCH = K + 8;                    // weight row pitch (bf16)
    static constexpr int PPITCH = CIN == 2 ? 2 : CIN + 8;   // pixel pitch in the tile (bf16)
    static constexpr int KSTEPS = K / 16;
};

__device__ __forceinline__ void mma_bf16(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

template <int CIN, int COUT, int INK, int OUTK, int ROWS>
__global__ void __launch_bounds__(256)
conv3x3_kernel(ConvArgs a)
{
    using KC = ConvK<CIN>;
    constexpr int COUTP = COUT < 8 ? 8 : COUT;
    constexpr int NT = COUTP / 8;
    constexpr int TP = 130;                       // 128 pixels + halo
    const int f = blockIdx.z;
    if (a.active && !a.active[f]) return;
    const int y0 = blockIdx.y * ROWS;
    const int x0 = blockIdx.x * 128;
    const int H = a.H, W = a.W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* tile = reinterpret_cast<__nv_bfloat16*>(smem_raw);          // [ROWS+2][TP][PPITCH]
    __nv_bfloat16* wsm = tile + (ROWS + 2) * TP * KC::PPITCH;                     // [COUTP][KPITCH]

    // weights
    for (int i = threadIdx.x; i < COUTP * KC::KPITCH / 2; i += blockDim.x)
        reinterpret_cast<uint32_t*>(wsm)[i] = reinterpret_cast<const uint32_t*>(a.w)[i];
    // input rows y0-1..y0+ROWS, pixels x0-1..x0+128 (periodic)
    const float sc = a.in_scale ? a.in_scale[f] : 1.0f;
    for (int i = threadIdx.x; i < (ROWS + 2) * TP * (CIN / 2); i += blockDim.x) {
        const int cp = i % (CIN / 2), px = (i / (CIN / 2)) % TP, r = i / ((CIN / 2) * TP);
        const int yy = (y0 + r - 1 + H) % H, xx = (x0 + px - 1 + W) % W;
        const int64_t pix = (int64_t)f * a.field_stride_in + (int64_t)yy * W + xx;
        uint32_t v;
        if (INK == IN_BF16) {
            v = reinterpret_cast<const uint32_t*>(a.in)[pix * (CIN / 2) + cp];
        } else if (INK == IN_C128) {
            const double2 z = reinterpret_cast<const double2*>(a.in)[pix];
            v = pack_bf16((float)z.x * sc, (float)z.y * sc);
        } else {
            const float2 z = reinterpret_cast<const float2*>(a.in)[pix];
            v = pack_bf16(z.x * sc, z.y * sc);
        }
        *reinterpret_cast<uint32_t*>(&tile[(r * TP + px) * KC::PPITCH + 2 * cp]) = v;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
    for (int ry = 0; ry < ROWS; ++ry) {
        const int y = y0 + ry;
        float acc[NT][4];
    #pragma unroll
        for (int j = 0; j < NT; ++j)
    #pragma unroll
            for (int q = 0; q < 4; ++q) acc[j][q] = 0.0f;
        const int p0 = warp * 16 + g;                // this lane's first pixel (tile column p0 + 1)
        auto ld = [&](int tap, int px, int c) -> uint32_t {
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
            return *reinterpret_cast<const uint32_t*>(&tile[((ry + dy + 1) * TP + px + dx + 1) * KC::PPITCH + c]);
        };
    #pragma unroll
        for (int s = 0; s < KC::KSTEPS; ++s) {
            uint32_t a0, a1, a2, a3;
            if (CIN == 2) {
                const int ta = 8 * s + t, tb = 8 * s + t + 4;
                a0 = ta < 9 ? ld(ta, p0, 0) : 0u;
                a1 = ta < 9 ? ld(ta, p0 + 8, 0) : 0u;
                a2 = tb < 9 ? ld(tb, p0, 0) : 0u;
                a3 = tb < 9 ? ld(tb, p0 + 8, 0) : 0u;
            } else {
                const int tap = s / (CIN / 16), c = (s % (CIN / 16)) * 16 + 2 * t;
                a0 = ld(tap, p0, c);
                a1 = ld(tap, p0 + 8, c);
                a2 = ld(tap, p0, c + 8);
                a3 = ld(tap, p0 + 8, c + 8);
            }
    #pragma unroll
            for (int j = 0; j < NT; ++j) {
                const __nv_bfloat16* wr = wsm + (8 * j + g) * KC::KPITCH + 16 * s + 2 * t;
                const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wr);
                const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wr + 8);
                mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
            }
        }

        // epilogue: acc[j][0..1] -> (pixel p0, channels 8j+2t, +1); acc[j][2..3] -> pixel p0 + 8
    #pragma unroll
        for (int hlf = 0; hlf < 2; ++hlf) {
            const int xx = x0 + p0 + 8 * hlf;
            const int64_t pix = (int64_t)f * a.field_stride_out + (int64_t)y * W + xx;
    #pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int ch = 8 * j + 2 * t;
                if (ch >= COUT) continue;
                float v0 = acc[j][2 * hlf], v1 = acc[j][2 * hlf + 1];
                if (a.bias) { v0 += a.bias[ch]; v1 += a.bias[ch + 1]; }
                if (OUTK == OUT_BF16_RELU) {
                    reinterpret_cast<uint32_t*>(a.out)[(pix * COUT + ch) / 2] =
                        pack_bf16(fmaxf(v0, 0.0f), fmaxf(v1, 0.0f));
                } else if (OUTK == OUT_BF16_MASK) {
                    const __nv_bfloat162 m = reinterpret_cast<const __nv_bfloat162*>(a.mask)[(pix * COUT + ch) / 2];
                    reinterpret_cast<uint32_t*>(a.out)[(pix * COUT + ch) / 2] =
                        pack_bf16(__bfloat162float(m.x) > 0.0f ? v0 : 0.0f, __bfloat162float(m.y) > 0.0f ? v1 : 0.0f);
                } else if (OUTK == OUT_F32) {
                    reinterpret_cast<float2*>(a.out)[pix] = make_float2(v0, v1);
                } else {
                    const double s2 = a.out_scale ? (double)a.out_scale[f] : 1.0;
                    double2* o = reinterpret_cast<double2*>(a.out) + pix;
                    double2 z = *o;
                    z.x += s2 * (double)v0;
                    z.y += s2 * (double)v1;
                    *o = z;
                }
            }
        }
    }   // rows
}

template <int CIN, int COUT, int INK, int OUTK, int ROWS>
int launch_conv_rows(const ConvArgs& a, int nfields, cudaStream_t st) {
    using KC = ConvK<CIN>;
    constexpr int COUTP = COUT < 8 ? 8 : COUT;
    const size_t smem = sizeof(__nv_bfloat16) * ((ROWS + 2) * 130 * KC::PPITCH + COUTP * KC::KPITCH);
    auto k = conv3x3_kernel<CIN, COUT, INK, OUTK, ROWS>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -4;
    if (nfields <= 0) return 0;
    dim3 grid(a.W / 128, a.H / ROWS, nfields);
    k<<<grid, 256, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

// four output rows per CTA where the height allows, else one
template <int CIN, int COUT, int INK, int OUTK>
int launch_conv(const ConvArgs& a, int nfields, cudaStream_t st) {
    if (a.H % 4 == 0) return launch_conv_rows<CIN, COUT, INK, OUTK, 4>(a, nfields, st);
    return launch_conv_rows<CIN, COUT, INK, OUTK, 1>(a, nfields, st);
}

}  // namespace soft
