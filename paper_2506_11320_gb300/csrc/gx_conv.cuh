// gx_conv.cuh -- the 3x3 convolution of the learned preconditioner on the
// tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation), shared
// by the network kernels and the solver kernel that applies the network.
//
// Implicit GEMM: M = 16 pixels of a row, N = output channels, K = 9 taps x
// input channels.  A CTA of 8 warps computes 8 rows x 16 columns; the input
// tile with its one-pixel halo and the weights are staged in shared memory
// with row strides padded by 8 elements so that ldmatrix is conflict-free.
// Activations are NHWC BF16 with the channel count padded to the MMA shapes.
#pragma once

#include <cuda_bf16.h>

#include "gx_internal.cuh"

namespace gxc {

typedef __nv_bfloat16 bf16;

constexpr int kTH = 8, kTW = 16;                // CTA tile: 8 rows x 16 columns
constexpr int kHalo = (kTH + 2) * (kTW + 2);    // 180 input pixels per tile

enum { EPI_RELU = 0, EPI_F32 = 1, EPI_MASK = 2 };

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

// load the (TH+2) x (TW+2) pixel halo tile of CIN channels of image b into
// shared memory (row stride CIN + 8), zero or periodic outside the image
// (CG: read through L2 only, for activations other CTAs of the same launch wrote)
// 16-byte asynchronous copy global -> shared through L2 only (cp.async.cg);
// with valid == false nothing is read and the 16 bytes are zero-filled
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// load the (TH+2) x (TW+2) pixel halo tile of CIN channels of image b into
// shared memory (row stride CIN + 8), zero or periodic outside the image
template <int CIN>
__device__ __forceinline__ void load_tile(bf16 *sIn, const bf16 *in, int b, int H, int W, int y0, int x0,
                                          int periodic) {
    constexpr int S = CIN + 8;
    constexpr int V = CIN / 8;   // 16-byte vectors per pixel
    for (int t = threadIdx.x; t < kHalo * V; t += blockDim.x) {
        const int pix = t / V, v = t % V;
        int yy = y0 - 1 + pix / (kTW + 2), xx = x0 - 1 + pix % (kTW + 2);
        uint4 val = make_uint4(0, 0, 0, 0);
        bool ok = true;
        if (periodic) {
            yy = wrapn(yy, H);
            xx = wrapn(xx, W);
        } else {
            ok = yy >= 0 && yy < H && xx >= 0 && xx < W;
        }
        if (ok) val = *reinterpret_cast<const uint4 *>(in + (((int64_t)b * H + yy) * W + xx) * CIN + v * 8);
        *reinterpret_cast<uint4 *>(sIn + pix * S + v * 8) = val;
    }
}

// start loading the (TH+2) x (TW+2) pixel halo tile of CIN channels of image b
// into shared memory (row stride CIN + 8), zero or periodic outside the image
template <int CIN>
__device__ __forceinline__ void load_tile_async(bf16 *sIn, const bf16 *in, int b, int H, int W, int y0, int x0,
                                                int periodic) {
    constexpr int S = CIN + 8;
    constexpr int V = CIN / 8;   // 16-byte vectors per pixel
    for (int t = threadIdx.x; t < kHalo * V; t += blockDim.x) {
        const int pix = t / V, v = t % V;
        int yy = y0 - 1 + pix / (kTW + 2), xx = x0 - 1 + pix % (kTW + 2);
        bool ok = true;
        if (periodic) {
            yy = wrapn(yy, H);
            xx = wrapn(xx, W);
        } else {
            ok = yy >= 0 && yy < H && xx >= 0 && xx < W;
        }
        const bf16 *src = ok ? in + (((int64_t)b * H + yy) * W + xx) * CIN + v * 8 : in;
        cp_async16(sIn + pix * S + v * 8, src, ok);
    }
}

struct ConvArgs {
    const bf16 *in;      // [B][H][W][CIN]
    const bf16 *w;       // [COUT][9][CIN]
    const float *bias;   // [COUT] or null
    void *out;           // [B][H][W][COUT] bf16 (or float for EPI_F32)
    const bf16 *mask;    // [B][H][W][COUT] (EPI_MASK): multiply by (mask > 0)
    const int *skip;     // nothing to do when *skip != 0 (the solver has finished); may be null
    int B, H, W, periodic;
};

// shared memory of conv_tiles<CIN, COUT>: two input tiles + weights (bf16 elements)
template <int CIN, int COUT>
__host__ __device__ constexpr int conv_smem_elems() { return 2 * kHalo * (CIN + 8) + COUT * (9 * CIN + 8); }

// out = epilogue(conv3x3(in, w) + bias) over the tiles cta, cta + ncta, ...;
// every CTA loads the weights once, and the next tile's input is loaded
// asynchronously while the current one is computed.  The input goes through
// L2 only, so activations written by other CTAs of the same launch (after a
// grid barrier) are seen.  sm: conv_smem_elems<CIN, COUT>() bf16.
template <int CIN, int COUT, int EPI>
__device__ __forceinline__ void conv_tiles(const ConvArgs &a, bf16 *sm, int cta, int ncta) {
    constexpr int SI = CIN + 8, SWr = 9 * CIN + 8;
    constexpr int NT = COUT / 8;
    bf16 *sW = sm + 2 * kHalo * SI;
    // weights
    constexpr int WV = 9 * CIN / 8;
    for (int t = threadIdx.x; t < COUT * WV; t += blockDim.x) {
        const int co = t / WV, v = t % WV;
        *reinterpret_cast<uint4 *>(sW + co * SWr + v * 8) = *reinterpret_cast<const uint4 *>(a.w + (size_t)co * 9 * CIN + v * 8);
    }
    const int tx = (a.W + kTW - 1) / kTW, ty = (a.H + kTH - 1) / kTH;
    const int64_t ntiles = (int64_t)tx * ty * a.B;
    auto issue = [&](int64_t t, bf16 *dst) {
        const int bb = (int)(t / ((int64_t)tx * ty)), rr = (int)(t % ((int64_t)tx * ty));
        load_tile_async<CIN>(dst, a.in, bb, a.H, a.W, (rr / tx) * kTH, (rr % tx) * kTW, a.periodic);
    };
    if (cta < ntiles) issue(cta, sm);
    cp_async_commit();
    int it = 0;
    for (int64_t tile = cta; tile < ntiles; tile += ncta, ++it) {
    const int b = (int)(tile / ((int64_t)tx * ty)), rem = (int)(tile % ((int64_t)tx * ty));
    const int x0 = (rem % tx) * kTW, y0 = (rem / tx) * kTH;
    bf16 *sIn = sm + (it & 1) * kHalo * SI;
    if (tile + ncta < ntiles) issue(tile + ncta, sm + ((it + 1) & 1) * kHalo * SI);
    cp_async_commit();
    cp_async_wait1();        // this tile's copies (all groups but the newest) are done
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mi = lane >> 3, r = lane & 7;
    float acc[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap % 3;
#pragma unroll
        for (int kc = 0; kc < CIN / 16; ++kc) {
            uint32_t a0, a1, a2, a3;
            {
                const int p = r + 8 * (mi & 1), koff = 8 * (mi >> 1);
                ldsm_x4(a0, a1, a2, a3, sIn + ((warp + ky) * (kTW + 2) + p + kx) * SI + kc * 16 + koff);
            }
            if (NT >= 2) {
#pragma unroll
                for (int np = 0; np < NT / 2; ++np) {
                    uint32_t b0, b1, b2, b3;
                    const int co = np * 16 + 8 * (mi >> 1) + r, k = tap * CIN + kc * 16 + 8 * (mi & 1);
                    ldsm_x4(b0, b1, b2, b3, sW + co * SWr + k);
                    mma16816(acc[2 * np], a0, a1, a2, a3, b0, b1);
                    mma16816(acc[2 * np + 1], a0, a1, a2, a3, b2, b3);
                }
            } else {
                uint32_t b0, b1;
                const int co = r, k = tap * CIN + kc * 16 + 8 * (mi & 1);
                ldsm_x2(b0, b1, sW + co * SWr + k);
                mma16816(acc[0], a0, a1, a2, a3, b0, b1);
            }
        }
    }
    // epilogue: thread holds pixels g and g+8 of the row, channels 2t, 2t+1 of each n-tile
    const int gq = lane >> 2, tq = lane & 3;
    const int yy = y0 + warp;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int xx = x0 + gq + 8 * h;
        if (yy >= a.H || xx >= a.W) continue;
        const int64_t pix = ((int64_t)b * a.H + yy) * a.W + xx;
#pragma unroll
        for (int n = 0; n < NT; ++n) {
            const int co = n * 8 + 2 * tq;
            float v0 = acc[n][2 * h], v1 = acc[n][2 * h + 1];
            if (a.bias) { v0 += a.bias[co]; v1 += a.bias[co + 1]; }
            if (EPI == EPI_F32) {
                *reinterpret_cast<float2 *>(reinterpret_cast<float *>(a.out) + pix * COUT + co) = make_float2(v0, v1);
            } else {
                if (EPI == EPI_RELU) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                } else {   // EPI_MASK
                    const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162 *>(a.mask + pix * COUT + co);
                    if (!(__bfloat162float(m.x) > 0.f)) v0 = 0.f;
                    if (!(__bfloat162float(m.y) > 0.f)) v1 = 0.f;
                }
                *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<bf16 *>(a.out) + pix * COUT + co) =
                    __floats2bfloat162_rn(v0, v1);
            }
        }
    }
    __syncthreads();   // this staging buffer is refilled two tiles later
    }   // tiles
}


}  // namespace gxc
