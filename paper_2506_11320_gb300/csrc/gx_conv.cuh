// gx_conv.cuh -- mma.sync m16n8k16 helpers (BF16 operands, FP32 accumulation)
// and the halo-tile loader of the weight-gradient kernel of the learned
// preconditioner: dW is a contraction over pixels (M = output channels, K =
// pixels), whose operands come transposed out of the pixel-major activation
// tiles through ldmatrix.trans.  The convolutions themselves (forward and data
// gradient) run on the tcgen05 tensor cores (gx_convtc.cuh).
//
// Tile: 8 rows x 16 columns of pixels with a one-pixel halo, staged in shared
// memory with row strides padded by 8 elements so that ldmatrix is
// conflict-free.  Activations are channel-blocked BF16 images with a
// one-pixel halo ring ([B][C/8][H+2][W+2][8]), the channel count padded to the
// MMA shapes.
#pragma once

#include <cuda_bf16.h>

#include "gx_internal.cuh"

namespace gxc {

typedef __nv_bfloat16 bf16;

constexpr int kTH = 8, kTW = 16;                // CTA tile: 8 rows x 16 columns
constexpr int kHalo = (kTH + 2) * (kTW + 2);    // 180 input pixels per tile

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t &r0, uint32_t &r1, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t &r0, uint32_t &r1, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma16816(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int wrapn(int i, int n) {
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
}

// load the (TH+2) x (TW+2) pixel tile of CIN channels of image b (rows
// y0-1 .. y0+TH, columns x0-1 .. x0+TW) into shared memory (row stride CIN +
// 8) from a channel-blocked image with a one-pixel halo ring,
// [B][CIN/8][H+2][W+2][8] (the ring holds the periodic copies or zeros); zero
// beyond the ring
template <int CIN>
__device__ __forceinline__ void load_tile_halo(bf16 *sIn, const bf16 *in, int b, int H, int W, int y0, int x0) {
    constexpr int S = CIN + 8;
    constexpr int V = CIN / 8;   // 16-byte chunks per pixel
    for (int t = threadIdx.x; t < kHalo * V; t += blockDim.x) {
        const int v = t / kHalo, pix = t % kHalo;     // consecutive threads: consecutive pixels of one chunk
        const int yy = y0 - 1 + pix / (kTW + 2), xx = x0 - 1 + pix % (kTW + 2);
        uint4 val = make_uint4(0, 0, 0, 0);
        if (yy <= H && xx <= W)
            val = *reinterpret_cast<const uint4 *>(
                in + ((((int64_t)b * V + v) * (H + 2) + yy + 1) * (W + 2) + xx + 1) * 8);
        *reinterpret_cast<uint4 *>(sIn + pix * S + v * 8) = val;
    }
}

}  // namespace gxc
