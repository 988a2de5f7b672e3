// 3x3 convolution with 32 input channels (periodic padding) as an implicit
// GEMM on the 5th-generation tensor cores: tcgen05.mma kind::f16, BF16
// operands in shared memory, FP32 accumulators in tensor memory (TMEM).
//
//   out[p][o] = b[o] + sum_{tap, c} in[y + dy][x + dx][c] W[o][32 tap + c]
//
// One CTA of 256 threads computes ROWS consecutive rows of a 128-pixel
// segment of one field for all output channels.  The MMA shape is
// M = 128 pixels (one row), N = NP output channels (COUT padded to 16),
// K = 16 input channels; a row takes 9 taps x 2 channel halves = 18 MMAs
// accumulating into NP TMEM columns, and the ROWS rows use disjoint column
// ranges, so one thread issues every MMA of the CTA back to back and one
// commit signals their completion.
//
// Operand layouts (K-major, no swizzle; a core matrix is 8 rows of 16 bytes
// stored contiguously):
//   input tile  [ROWS + 2 rows][4 channel groups][130 pixels][8 channels]:
//     the core matrix of pixels p .. p+7 and channel group g of a row is the
//     128 contiguous bytes at pixel p, so the operand of tap (dy, dx) is the
//     same tile with its start address moved by dx pixels (16 bytes) and dy
//     rows; consecutive 8-pixel groups are 128 bytes apart (the descriptor's
//     stride byte offset) and the two channel groups of a K-step one slab,
//     130 x 16 bytes, apart (the leading byte offset);
//   weights [9 taps][4 channel groups][NP outputs][8 channels].
// Epilogue: warp w reads TMEM lanes 32 (w mod 4) + lane (pixel = lane) with
// tcgen05.ld for the rows ry = w / 4, w / 4 + 2, ..., adds the bias,
// applies ReLU or the backward mask, and writes 64 contiguous bytes per
// pixel.  All 8 warps stage the tile (the CTA's input rows are in flight
// together); one thread issues the MMAs.
//
// The completion wait is bounded: if it runs out, the CTA sets bit 0 of
// *err (when given), writes NaN to its outputs, waits once more (bounded)
// for its MMAs, frees its TMEM and returns.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "conv.cuh"
#include "device_common.cuh"

namespace soft {
namespace tc5 {

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t start, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((start & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
template <int M, int N>
__host__ __device__ constexpr uint32_t idesc_bf16() {
    static_assert(M == 128 && N % 16 == 0 && N >= 16 && N <= 256, "M = 128 needs N = 16 .. 256, step 16");
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ void bar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// wait for phase `ph` of the barrier, at most `limit` polls
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t ph, int limit) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(saddr(bar)), "r"(ph) : "memory");
    return done != 0;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// TMEM allocation of NCOL columns (one full warp); the base address lands in *slot
template <int NCOL>
__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
    static_assert(NCOL >= 32 && NCOL <= 512 && (NCOL & (NCOL - 1)) == 0, "power of 2 columns, 32 .. 512");
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
template <int NCOL>
__device__ __forceinline__ void tmem_free(uint32_t base) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(NCOL));
}

// 32 lanes x NC consecutive 32-bit columns (lane = thread of the warp)
template <int NC> __device__ __forceinline__ void tmem_ld(uint32_t ta, uint32_t* r);
template <> __device__ __forceinline__ void tmem_ld<16>(uint32_t ta, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                   "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
template <> __device__ __forceinline__ void tmem_ld<32>(uint32_t ta, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                   "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
                   "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
                   "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
                   "=r"(r[31])
                 : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

constexpr int SM_SMEM = 233472;      // shared memory of one SM (228 KB)
constexpr int CTA_RESERVED = 1024;   // per-CTA shared memory the system reserves
constexpr int WAIT_POLLS = 1 << 20;  // bounded completion wait

}  // namespace tc5

template <int COUT, int ROWS>
struct ConvTC {
    static constexpr int NP = COUT < 16 ? 16 : COUT;            // MMA N
    static constexpr int WROWS = COUT < 8 ? 8 : COUT;           // rows of the packed weights
    static constexpr int TP = 130;                              // 128 pixels + halo
    static constexpr int SLAB = TP * 16;                        // one row, one channel group
    static constexpr int TILEB = (ROWS + 2) * 4 * SLAB;
    static constexpr int WB = 9 * 4 * NP * 16;
    static constexpr int SMEM = TILEB + WB;
    static constexpr int NCOL = ROWS * NP <= 32 ? 32 : ROWS * NP <= 64 ? 64 : ROWS * NP <= 128 ? 128 : 256;
    // every CTA the shared memory lets reside on an SM gets its TMEM at once
    static_assert(tc5::SM_SMEM / (SMEM + tc5::CTA_RESERVED) * NCOL <= 512, "TMEM oversubscribed");
    static_assert(COUT == 32 || COUT == 2, "layers with 32 or 2 outputs");
};

template <int COUT, int OUTK, int ROWS>
__global__ void __launch_bounds__(256)
conv3x3_tc_kernel(ConvArgs a)
{
    using Q = ConvTC<COUT, ROWS>;
    constexpr int NP = Q::NP, SLAB = Q::SLAB, TP = Q::TP, NT = 256;
    constexpr int KP = ConvK<32>::KPITCH;
    const int f = blockIdx.z;
    if (a.active && !a.active[f]) return;
    const int y0 = blockIdx.y * ROWS, x0 = blockIdx.x * 128;
    const int H = a.H, W = a.W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* tile = smem_raw;
    unsigned char* wsm = smem_raw + Q::TILEB;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) tc5::tmem_alloc<Q::NCOL>(&tslot);
    if (tid == 0) tc5::bar_init(&bar);
    // weights: the 16 bytes (tap, channel group g, output n) = packed row n at k = 32 tap + 8 g
    for (int i = tid; i < 9 * 4 * NP; i += NT) {
        const int n = i % NP, g = (i / NP) & 3, tap = i / (4 * NP);
        uint4* dst = reinterpret_cast<uint4*>(wsm) + i;
        if (n < Q::WROWS) cp_async<16>(dst, a.w + (size_t)n * KP + 32 * tap + 8 * g);
        else *dst = make_uint4(0u, 0u, 0u, 0u);
    }
    // input rows y0-1 .. y0+ROWS, pixels x0-1 .. x0+128 (periodic: each
    // index is at most one period outside), 4 x 16 bytes per pixel
    const unsigned char* in = reinterpret_cast<const unsigned char*>(a.in) + (int64_t)f * a.field_stride_in * 64;
#pragma unroll 1
    for (int r = 0; r < ROWS + 2; ++r) {
        int yy = y0 + r - 1;
        yy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
        const unsigned char* row = in + (int64_t)yy * W * 64;
        unsigned char* trow = tile + r * 4 * SLAB;
        for (int j = tid; j < TP * 4; j += NT) {
            const int px = j >> 2, g = j & 3;
            int xx = x0 + px - 1;
            xx = xx < 0 ? xx + W : (xx >= W ? xx - W : xx);
            cp_async<16>(trow + (g * TP + px) * 16, row + (int64_t)xx * 64 + g * 16);
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    tc5::fence_async_smem();          // the generic-proxy writes, visible to the tensor cores
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const uint32_t tbase = tslot;

    if (tid == 0) {
        constexpr uint32_t ID = tc5::idesc_bf16<128, NP>();
        const uint32_t ts = tc5::saddr(tile), ws = tc5::saddr(wsm);
        for (int ry = 0; ry < ROWS; ++ry)
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3, dx = tap % 3;       // tile row ry + dy, tile pixel p + dx
                for (int h = 0; h < 2; ++h) {
                    const uint64_t ad = tc5::sdesc(ts + (uint32_t)(((ry + dy) * 4 + 2 * h) * SLAB + dx * 16),
                                                   SLAB, 128);
                    const uint64_t bd = tc5::sdesc(ws + (uint32_t)((tap * 4 + 2 * h) * NP * 16), NP * 16, 128);
                    tc5::mma(tbase + (uint32_t)(ry * NP), ad, bd, ID, (tap | h) != 0);
                }
            }
        tc5::commit(&bar);
    }
    bool ok = tc5::bar_wait(&bar, 0, tc5::WAIT_POLLS);
    ok = __any_sync(0xffffffffu, ok);          // the phase completes for every thread at once
    tc5::fence_after();
    if (!ok && lane == 0 && a.err) atomicOr(a.err, 1u);

    float bias[COUT];
#pragma unroll
    for (int j = 0; j < COUT; ++j) bias[j] = a.bias ? a.bias[j] : 0.0f;
    const int p = 32 * (warp & 3) + lane;      // pixel of the segment = TMEM lane
    const uint32_t tl = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll 1
    for (int ry = warp >> 2; ry < ROWS; ry += NT / 128) {
        uint32_t r[NP];
        if (ok) {
            tc5::tmem_ld<NP>(tl + (uint32_t)(ry * NP), r);
        } else {
#pragma unroll
            for (int j = 0; j < NP; ++j) r[j] = 0x7fc00000u;
        }
        const int64_t pix = (int64_t)f * a.field_stride_out + (int64_t)(y0 + ry) * W + x0 + p;
        if constexpr (OUTK == OUT_BF16_RELU || OUTK == OUT_BF16_MASK) {
            static_assert(COUT == 32, "bf16 activations have 32 channels");
            uint32_t pk[16];
            if constexpr (OUTK == OUT_BF16_MASK) {
                const uint4* mk = reinterpret_cast<const uint4*>(a.mask) + pix * 4;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 m4 = mk[q];
                    const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(&mw[e]);
                        const int j = 4 * q + e;
                        const float v0 = __uint_as_float(r[2 * j]), v1 = __uint_as_float(r[2 * j + 1]);
                        pk[j] = pack_bf16(__bfloat162float(m.x) > 0.0f ? v0 : 0.0f,
                                          __bfloat162float(m.y) > 0.0f ? v1 : 0.0f);
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float v0 = __uint_as_float(r[2 * j]) + bias[2 * j];
                    const float v1 = __uint_as_float(r[2 * j + 1]) + bias[2 * j + 1];
                    pk[j] = pack_bf16(fmaxf(v0, 0.0f), fmaxf(v1, 0.0f));
                }
            }
            uint4* o = reinterpret_cast<uint4*>(a.out) + pix * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
        } else {
            static_assert(COUT == 2, "two output channels");
            const float v0 = __uint_as_float(r[0]) + bias[0], v1 = __uint_as_float(r[1]) + bias[1];
            if constexpr (OUTK == OUT_F32) {
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
    // after a wait that ran out, wait once more (bounded) for the MMAs before
    // the accumulator columns are released
    if (!ok) tc5::bar_wait(&bar, 0, tc5::WAIT_POLLS);
    tc5::fence_before();
    __syncthreads();
    if (warp == 0) tc5::tmem_free<Q::NCOL>(tbase);
}

template <int COUT, int OUTK, int ROWS>
int launch_conv_tc_rows(const ConvArgs& a, int nfields, cudaStream_t st) {
    using Q = ConvTC<COUT, ROWS>;
    auto k = conv3x3_tc_kernel<COUT, OUTK, ROWS>;
    if (Q::SMEM > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Q::SMEM) != cudaSuccess)
        return -4;
    if (nfields <= 0) return 0;
    if (a.W % 128 != 0 || a.H % ROWS != 0) return -2;
    dim3 grid(a.W / 128, a.H / ROWS, nfields);
    k<<<grid, 256, Q::SMEM, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

// 32 input channels: four output rows per CTA where the height allows, else one
template <int COUT, int OUTK>
int launch_conv32_tc(const ConvArgs& a, int nfields, cudaStream_t st) {
    if (a.H % 4 == 0) return launch_conv_tc_rows<COUT, OUTK, 4>(a, nfields, st);
    return launch_conv_tc_rows<COUT, OUTK, 1>(a, nfields, st);
}

}  // namespace soft
