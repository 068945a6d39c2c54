// gx_net.cu -- learned GMRES preconditioner (an addition of this project; the
// paper has no learned preconditioner).
//
// Network N: four 3x3 convolutions, channels 3 -> 32 -> 32 -> 32 -> 3, ReLU
// between them, on the 2D node grid (H = ny rows, W = nx columns), BF16 weights
// and activations with FP32 accumulation.  Inside FGMRES it corrects the 3x3
// block-Jacobi preconditioner D^-1 of the field operator A:
//     z = D^-1 r + s N(r / s),   s = ||r||_2 / sqrt(3 N),  periodic padding.
// D^-1 carries what varies from node to node (the plasma's mass-matrix block,
// which the network, seeing only r, could not know); the network learns the
// translation-invariant remainder A^-1 r - D^-1 r, a few per cent of z at the
// usual time steps, so its BF16 rounding error is relative to that remainder.
//
// Kernels:
//   * k_convtc: the implicit-GEMM convolution of gx_convtc.cuh on the tcgen05
//     tensor cores (fed by TMA bulk copies, BF16 operands, FP32 accumulators
//     in tensor memory).  The forward pass and the data gradient (the same convolution
//     with the kernel flipped and the channel roles swapped, masked by the
//     ReLU of the layer input) both use it; inside the solver the forward pass
//     runs in the solver's own kernel.
//   * k_wgrad: weight gradient dW[co][tap][ci] = sum_p dY[p][co] X[p+tap][ci],
//     a contraction over pixels (mma.sync m16n8k16 with ldmatrix.trans
//     operands), accumulated by a persistent grid in registers and added to
//     FP32 global sums once per CTA.
//   * Adam on an FP32 master copy; BF16 copies refreshed after each update.
// Channel counts are padded for the MMA shapes: 3 input channels -> 16,
// 3 output channels -> 8 (stored forward output; 32 in the MMA) or 16
// (gradient).  BF16 activations are channel-blocked images with a one-pixel
// halo ring, [B][C/8][H+2][W+2][8].
#include <cuda_bf16.h>

#include <cstring>
#include <random>

#include "gx_conv.cuh"
#include "gx_convtc.cuh"
#include "gx_netpipe.cuh"

#include <cooperative_groups.h>

using namespace gxc;

namespace {

constexpr int kNL = 4;
constexpr int kCin[kNL] = {3, 32, 32, 32};
constexpr int kCout[kNL] = {32, 32, 32, 3};
constexpr int kCinP[kNL] = {16, 32, 32, 32};    // padded input channels (storage of the layer input)
constexpr int kCoutP[kNL] = {32, 32, 32, 8};    // padded output channels (forward storage)
constexpr int kNmma[kNL] = {32, 32, 32, 32};    // output channels of the forward MMA (one row block)
constexpr int kGCoutP[kNL] = {32, 32, 32, 16};  // padded output channels of the gradient (dY) storage

constexpr int64_t layer_w_count(int l) { return (int64_t)kCout[l] * kCin[l] * 9; }
inline int64_t param_offset(int l) {
    int64_t o = 0;
    for (int k = 0; k < l; ++k) o += layer_w_count(k) + kCout[k];
    return o;
}
inline int64_t param_count() { return param_offset(kNL); }

// the forward/data-gradient convolution as a kernel (a persistent grid of
// tensor-core CTAs, gx_convtc.cuh); R image rows per unit of work
constexpr int kConvRows = 4;

// the solver's application of the network to one vector, as one cooperative
// kernel running the same pipeline as the solver: pack v / s into the layer-0
// image, clear the completion flags, grid barrier, four layers
__global__ void __launch_bounds__(2 * gxv::kThreads, 1) k_net_apply(gxn::PipeArgs p, gxv::bf16 *x0, float inv_s) {
    extern __shared__ __align__(128) unsigned char dsm[];
    unsigned char *sm = dsm + ((128 - (gxt::smem_addr(dsm) & 127)) & 127);
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    const int64_t HW = (int64_t)p.H * p.W;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < HW; q += (int64_t)gridDim.x * blockDim.x) {
        const __nv_bfloat162 p01 = __floats2bfloat162_rn((float)p.v[q] * inv_s, (float)p.v[HW + q] * inv_s);
        const __nv_bfloat162 p2 = __floats2bfloat162_rn((float)p.v[2 * HW + q] * inv_s, 0.f);
        const uint4 val[2] = {make_uint4(*reinterpret_cast<const uint32_t *>(&p01),
                                         *reinterpret_cast<const uint32_t *>(&p2), 0, 0),
                              make_uint4(0, 0, 0, 0)};
        gxv::store_with_halo<16>(x0, 0, (int)(q / p.W), (int)(q % p.W), p.H, p.W, 1, val);
    }
    gxn::pipe_clear_flags(p.flags, p.H, p.W, blockIdx.x, gridDim.x);
    grid.sync();
    gxn::net_pipeline(p, sm, blockIdx.x, gridDim.x);
}

template <int CIN, int N, int COUTG, int EPI>
__global__ void __launch_bounds__(2 * gxv::kThreads) k_convtc(const gxv::bf16 *in, gxv::Args a, const int *skip) {
    extern __shared__ __align__(128) unsigned char dsm[];
    if (skip && *skip) return;
    unsigned char *sm = dsm + ((128 - (gxt::smem_addr(dsm) & 127)) & 127);
    gxv::conv_tc<CIN, N, COUTG, kConvRows, EPI>(a, in, sm, blockIdx.x, gridDim.x);
}

struct WgArgs {
    const bf16 *dy;      // [B][COUTP/8][H+2][W+2][8] gradient wrt the layer output (halo ring)
    const bf16 *x;       // [B][CIN/8][H+2][W+2][8] layer input (halo ring: periodic copies or zeros)
    float *gw;           // [COUTP][9][CIN] FP32 sums
    float *gb;           // [COUTP]
    int B, H, W, periodic;
};

// dW[co][tap][ci] += sum_p dY[p][co] X[p + off(tap)][ci],  dB[co] += sum_p dY[p][co]
template <int CIN, int COUTP>
__global__ void __launch_bounds__(256) k_wgrad(WgArgs a) {
    constexpr int SI = CIN + 8, SD = COUTP + 8;
    constexpr int MT = COUTP / 16, NTN = 9 * CIN / 8, NTILE = MT * NTN;
    constexpr int PER = (NTILE + 7) / 8;          // output tiles per warp
    __shared__ __align__(16) bf16 sX[kHalo * SI];
    __shared__ __align__(16) bf16 sD[kTH * kTW * SD];
    __shared__ float sB[COUTP];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mi = lane >> 3, r = lane & 7;
    float acc[PER][4];
#pragma unroll
    for (int i = 0; i < PER; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    for (int i = threadIdx.x; i < COUTP; i += blockDim.x) sB[i] = 0.f;
    const int tx = (a.W + kTW - 1) / kTW, ty = (a.H + kTH - 1) / kTH;
    const int64_t ntiles = (int64_t)tx * ty * a.B;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int b = (int)(t / (tx * ty)), rem = (int)(t % (tx * ty));
        const int y0 = (rem / tx) * kTH, x0 = (rem % tx) * kTW;
        __syncthreads();
        load_tile_halo<CIN>(sX, a.x, b, a.H, a.W, y0, x0);
        constexpr int DV = COUTP / 8;
        for (int q = threadIdx.x; q < kTH * kTW * DV; q += blockDim.x) {
            const int v = q / (kTH * kTW), pix = q % (kTH * kTW);   // consecutive threads: consecutive pixels
            const int yy = y0 + pix / kTW, xx = x0 + pix % kTW;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (yy < a.H && xx < a.W)
                val = *reinterpret_cast<const uint4 *>(a.dy + gxv::blk_off(b, v, yy, xx, a.H, a.W, DV));
            *reinterpret_cast<uint4 *>(sD + pix * SD + v * 8) = val;
        }
        __syncthreads();
        // bias gradient
        for (int co = threadIdx.x; co < COUTP; co += blockDim.x) {
            float s = 0.f;
            for (int pix = 0; pix < kTH * kTW; ++pix) s += __bfloat162float(sD[pix * SD + co]);
            sB[co] += s;
        }
        // K loop: one tile row of 16 pixels per step
#pragma unroll 1
        for (int row = 0; row < kTH; ++row) {
            uint32_t af[MT][4];
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                const int p = r + 8 * (mi >> 1), coff = 8 * (mi & 1);
                ldsm_x4_t(af[m][0], af[m][1], af[m][2], af[m][3], sD + (row * kTW + p) * SD + m * 16 + coff);
            }
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int tile = warp + 8 * i;
                if (tile >= NTILE) break;
                const int m = tile / NTN, nt = tile % NTN;
                const int kk = nt * 8, tap = kk / CIN, ci0 = kk % CIN;
                const int ky = tap / 3, kx = tap % 3;
                uint32_t b0, b1;
                const int p = r + 8 * (mi & 1);
                ldsm_x2_t(b0, b1, sX + ((row + ky) * (kTW + 2) + p + kx) * SI + ci0);
                mma16816(acc[i], af[m][0], af[m][1], af[m][2], af[m][3], b0, b1);
            }
        }
    }
    __syncthreads();
    const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int tile = warp + 8 * i;
        if (tile >= NTILE) break;
        const int m = tile / NTN, nt = tile % NTN;
        const int co0 = m * 16 + gq, k0 = nt * 8 + 2 * tq;
        atomicAdd(a.gw + (size_t)co0 * 9 * CIN + k0, acc[i][0]);
        atomicAdd(a.gw + (size_t)co0 * 9 * CIN + k0 + 1, acc[i][1]);
        atomicAdd(a.gw + (size_t)(co0 + 8) * 9 * CIN + k0, acc[i][2]);
        atomicAdd(a.gw + (size_t)(co0 + 8) * 9 * CIN + k0 + 1, acc[i][3]);
    }
    for (int co = threadIdx.x; co < COUTP; co += blockDim.x) atomicAdd(a.gb + co, sB[co]);
}

// FP32 master parameters (layout W[co][ci][ky][kx], b[co] per layer) -> BF16
// forward weights [coutP][9][cinP], FP32 bias [coutP], BF16 data-gradient
// weights [cin][9][gcoutP] (flipped taps, channel roles swapped)
// FP32 master weights -> BF16 operands of the tensor-core convolution, packed
// as its weight slabs: for kernel column kx and 8-input-channel group kg, the
// 3 NP rows (kernel rows ky = 2, 1, 0, NP output channels each) of 8 channels,
// element (kx, kg, (2 - ky) NP + n, j) at ((kx CINP/8 + kg) 3 NP + (2 - ky) NP
// + n) 8 + j, zero for padded n or channels.
//   wf: the forward kernel, n = output channel (NP = nP);
//   wd: the data-gradient kernel (flipped taps, channel roles swapped),
//       n = input channel of the layer (NP = cin), channels = output channels
//       of the layer padded to gcoutP.
__global__ void k_pack_weights(const float *params, bf16 *wf, float *bias, bf16 *wd, int cin, int cout, int cinP,
                               int nP, int coutP, int gcoutP, int64_t off) {
    const float *W = params + off, *bsrc = params + off + (int64_t)cout * cin * 9;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 9 * cinP * nP; t += gridDim.x * blockDim.x) {
        const int j = t % 8, n3 = (t / 8) % (3 * nP), kgx = t / (8 * 3 * nP);
        const int kx = kgx / (cinP / 8), ci = (kgx % (cinP / 8)) * 8 + j;
        const int ky = 2 - n3 / nP, n = n3 % nP;
        const float v = (n < cout && ci < cin) ? W[((n * cin + ci) * 9) + ky * 3 + kx] : 0.f;
        wf[t] = __float2bfloat16_rn(v);
    }
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < coutP; t += gridDim.x * blockDim.x)
        bias[t] = t < cout ? bsrc[t] : 0.f;
    if (wd) {
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 9 * gcoutP * cin; t += gridDim.x * blockDim.x) {
            const int j = t % 8, n3 = (t / 8) % (3 * cin), kgx = t / (8 * 3 * cin);
            const int kx = kgx / (gcoutP / 8), co = (kgx % (gcoutP / 8)) * 8 + j;
            const int ky = 2 - n3 / cin, n = n3 % cin;
            const float v = co < cout ? W[((co * cin + n) * 9) + (8 - (ky * 3 + kx))] : 0.f;
            wd[t] = __float2bfloat16_rn(v);
        }
    }
}

// padded FP32 gradient sums -> gradient in the master layout (scaled)
__global__ void k_unpack_grad(const float *gw, const float *gb, float *grad, int cin, int cout, int cinP,
                              int64_t off, float scale) {
    const int64_t nw = (int64_t)cout * cin * 9;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nw + cout; t += (int64_t)gridDim.x * blockDim.x) {
        if (t < nw) {
            const int co = (int)(t / (cin * 9)), rem = (int)(t % (cin * 9)), ci = rem / 9, tap = rem % 9;
            grad[off + t] = scale * gw[((int64_t)co * 9 + tap) * cinP + ci];
        } else {
            grad[off + t] = scale * gb[t - nw];
        }
    }
}

__global__ void k_adam(float *p, const float *g, float *m1, float *m2, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi, b = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = b;
        p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
}

// [3][H][W] FP32 or FP64 field times `scale` -> BF16 NHWC image with 16
// channels (3 used) and a halo ring (periodic copies or zeros)
template <typename T>
__global__ void k_pack_input(const T *src, int H, int W, double scale, int periodic, bf16 *dst) {
    const int64_t HW = (int64_t)H * W;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < HW; p += (int64_t)gridDim.x * blockDim.x) {
        const __nv_bfloat162 p01 = __floats2bfloat162_rn((float)(src[p] * scale), (float)(src[HW + p] * scale));
        const __nv_bfloat162 p2 = __floats2bfloat162_rn((float)(src[2 * HW + p] * scale), 0.f);
        const uint4 val[2] = {make_uint4(*reinterpret_cast<const uint32_t *>(&p01),
                                         *reinterpret_cast<const uint32_t *>(&p2), 0, 0),
                              make_uint4(0, 0, 0, 0)};
        gxv::store_with_halo<16>(dst, 0, (int)(p / W), (int)(p % W), H, W, periodic, val);
    }
}

// training crops: for crop b, input = r / s_b on a (C+8)^2 window (4-pixel halo,
// periodic in the source field) and target = t / s_b on the central C^2, where
// the pair stores t = e - D^-1 r (the remainder the network learns), with
// s_b = ||r||_2 / sqrt(3 N) over the whole field, the scale the solver uses
struct CropSpec {
    int pair, y0, x0, pad;
};
__global__ void k_crop_scale(const float *pairs, int64_t N, const CropSpec *spec, float *scale) {
    const CropSpec sp = spec[blockIdx.x];
    const float *r = pairs + (size_t)sp.pair * 6 * N;
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < 3 * N; t += blockDim.x) {
        const double v = r[t];
        s += v * v;
    }
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        const double rms = sqrt(t / (3.0 * N));
        scale[blockIdx.x] = rms > 0 ? (float)rms : 1.f;
    }
}
__global__ void k_crop_gather(const float *pairs, int64_t N, int nx, int ny, const CropSpec *spec, int C,
                              const float *scale, bf16 *x0, float *target) {
    const int b = blockIdx.y;
    const CropSpec sp = spec[b];
    const float *r = pairs + (size_t)sp.pair * 6 * N, *e = r + 3 * N;
    const int S = C + 8;
    const float inv = 1.f / scale[b];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < S * S; t += gridDim.x * blockDim.x) {
        const int yy = t / S, xx = t % S;
        const int gy = wrapn(sp.y0 + yy - 4, ny), gx = wrapn(sp.x0 + xx - 4, nx);
        const int64_t q = gy * (int64_t)nx + gx;
        const __nv_bfloat162 p01 = __floats2bfloat162_rn(r[q] * inv, r[N + q] * inv);
        const __nv_bfloat162 p2 = __floats2bfloat162_rn(r[2 * N + q] * inv, 0.f);
        const uint4 val[2] = {make_uint4(*reinterpret_cast<const uint32_t *>(&p01),
                                         *reinterpret_cast<const uint32_t *>(&p2), 0, 0),
                              make_uint4(0, 0, 0, 0)};
        gxv::store_with_halo<16>(x0, b, yy, xx, S, S, 0, val);
        const bool inner = yy >= 4 && yy < 4 + C && xx >= 4 && xx < 4 + C;
#pragma unroll
        for (int c = 0; c < 3; ++c) target[((int64_t)b * S * S + t) * 3 + c] = inner ? e[c * N + q] * inv : 0.f;
    }
}

// loss = sum over the loss region of (y - t)^2 / (2 Nout) and dY = (y - t) / Nout
// there (zero elsewhere), dY stored BF16 with 16 channels and a zero halo ring
__global__ void k_loss(const float *y, const float *target, int B, int H, int W, int ry0, int rx0, int RH, int RW,
                       float inv_nout, bf16 *dy, double *loss) {
    double s = 0.0;
    const int64_t npix = (int64_t)B * H * W;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const int rem = (int)(p % (H * W)), yy = rem / W, xx = rem % W;
        const bool in = yy >= ry0 && yy < ry0 + RH && xx >= rx0 && xx < rx0 + RW;
        __align__(16) bf16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
        if (in) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float d = y[p * 8 + c] - target[p * 3 + c];
                s += (double)d * d;
                v[c] = __float2bfloat16_rn(d * inv_nout);
            }
        }
        const uint4 val[2] = {reinterpret_cast<uint4 *>(v)[0], reinterpret_cast<uint4 *>(v)[1]};
        gxv::store_with_halo<16>(dy, (int)(p / (H * W)), yy, xx, H, W, 0, val);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, 0.5 * s * inv_nout);
}

__global__ void k_f32_to_chw3(const float *y, int64_t HW, float *out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < HW; p += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) out[c * HW + p] = y[p * 8 + c];
}
__global__ void k_chw3_to_target(const float *t, int64_t HW, float *out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < HW; p += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) out[p * 3 + c] = t[c * HW + p];
}

// pair slot [2][3][N] = (r, t) with t = e - D^-1 r, jd = [N][9] inverse blocks.
// k_store_r: r (FP64) -> slot; k_store_t: t from e = eth - en and the slot's
// FP32 r; k_store_rt: both from FP64 r and e.
__global__ void k_store_r(const double *r, int64_t n3, float *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)r[i];
}
__global__ void k_store_t(const double *jd, const double *eth, const double *en, int64_t N, float *dst) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        const double *o = jd + (size_t)q * 9;
        const double r0 = dst[q], r1 = dst[N + q], r2 = dst[2 * N + q];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double e = eth[c * N + q] - en[c * N + q];
            dst[3 * N + c * N + q] = (float)(e - (o[3 * c] * r0 + o[3 * c + 1] * r1 + o[3 * c + 2] * r2));
        }
    }
}
__global__ void k_store_rt(const double *jd, const double *r, const double *e, int64_t N, float *dst) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        const double *o = jd + (size_t)q * 9;
        const double r0 = r[q], r1 = r[N + q], r2 = r[2 * N + q];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dst[c * N + q] = (float)r[c * N + q];
            dst[3 * N + c * N + q] = (float)(e[c * N + q] - (o[3 * c] * r0 + o[3 * c + 1] * r1 + o[3 * c + 2] * r2));
        }
    }
}

// crop store: sum of squares of a pair slot's r (for its scale), and the cut of
// `count` windows of S^2 nodes (periodic) at positions drawn from a counter-based
// hash of (seed, counter), stored scaled as [2][3][S][S] (r / s, t / s)
__global__ void k_sumsq_r(const float *r, int64_t n3, double *acc) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)r[i] * r[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
struct CutArgs {
    const float *pair;        // [2][3][N] (r, t)
    int64_t N;
    int nx, ny, S;
    uint64_t seed, counter;   // crop b of this cut: position from splitmix64(seed ^ splitmix64(counter + b))
    const double *sumsq;      // sum of r^2 over the field
    float *crops, *scales;    // the store [cap][6][S][S], [cap]
    int cap, next;
};
__global__ void k_cut_crops(CutArgs a) {
    const int b = blockIdx.y;
    const uint64_t h = splitmix64(a.seed ^ splitmix64(a.counter + (uint64_t)b));
    const int x0 = (int)((h & 0xffffffffull) % (uint64_t)a.nx), y0 = (int)((h >> 32) % (uint64_t)a.ny);
    const double rms = sqrt(*a.sumsq / (3.0 * a.N));
    const float s = rms > 0 ? (float)rms : 1.f, inv = 1.f / s;
    const int slot = (a.next + b) % a.cap;
    float *dst = a.crops + (size_t)slot * 6 * a.S * a.S;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.scales[slot] = s;
    const int SS = a.S * a.S;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < SS; t += gridDim.x * blockDim.x) {
        const int yy = t / a.S, xx = t % a.S;
        const int gy = wrapn(y0 + yy, a.ny), gx = wrapn(x0 + xx, a.nx);
        const int64_t q = gy * (int64_t)a.nx + gx;
#pragma unroll
        for (int c = 0; c < 6; ++c) dst[(size_t)c * SS + t] = a.pair[(size_t)c * a.N + q] * inv;
    }
}
// a training batch from the crop store: input r / s (BF16, halo ring), target t / s
// on the central C^2
__global__ void k_crop_gather_store(const float *crops, const CropSpec *spec, int C, bf16 *x0, float *target) {
    const int b = blockIdx.y;
    const int S = C + 8, SS = S * S;
    const float *src = crops + (size_t)spec[b].pair * 6 * SS;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < SS; t += gridDim.x * blockDim.x) {
        const int yy = t / S, xx = t % S;
        const __nv_bfloat162 p01 = __floats2bfloat162_rn(src[t], src[SS + t]);
        const __nv_bfloat162 p2 = __floats2bfloat162_rn(src[2 * SS + t], 0.f);
        const uint4 val[2] = {make_uint4(*reinterpret_cast<const uint32_t *>(&p01),
                                         *reinterpret_cast<const uint32_t *>(&p2), 0, 0),
                              make_uint4(0, 0, 0, 0)};
        gxv::store_with_halo<16>(x0, b, yy, xx, S, S, 0, val);
        const bool inner = yy >= 4 && yy < 4 + C && xx >= 4 && xx < 4 + C;
#pragma unroll
        for (int c = 0; c < 3; ++c) target[((int64_t)b * SS + t) * 3 + c] = inner ? src[(3 + c) * SS + t] : 0.f;
    }
}

inline int nblk(int64_t n, int b = 256) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + b - 1) / b, 152 * 16)); }

}  // namespace

struct Net {
    float *params = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    bf16 *wf[kNL] = {}, *wd[kNL] = {};
    float *bias[kNL] = {};
    float *gw[kNL] = {}, *gb[kNL] = {};
    int have_weights = 0;
    // activations: channel-blocked BF16 images with a halo ring [B][C/8][H+2][W+2][8]; y, target [B][H][W][*]
    int64_t cap_pix = 0, cap_halo = 0;
    bf16 *x0 = nullptr, *h1 = nullptr, *h2 = nullptr, *h3 = nullptr;
    bf16 *d4 = nullptr, *d3 = nullptr, *d2 = nullptr, *d1 = nullptr;
    float *y = nullptr, *target = nullptr;
    double *dsum = nullptr;    // [0] sum of squares, [1] loss
    unsigned *flags = nullptr; // completion flags of the network pipeline [3][units]
    int cap_flags = 0;
    // collected pairs: [cap][2][3][N] FP32 (r0, e)
    float *pairs = nullptr;
    int cap_pairs = 0, npairs = 0, next_pair = 0, collect = 0;
    int pending_pair = 0;
    // crop store (gx_precond_collect_crops): [cap][2][3][S][S] scaled windows and their
    // scales; the pair slots above then hold one field pair, the cut's source
    float *crops = nullptr, *cscales = nullptr;
    double *csum = nullptr;
    int crop_mode = 0, cap_crops = 0, ncrops = 0, next_crop = 0, crop_C = 0, per_pair = 0;
    uint64_t crop_seed = 0, crop_counter = 0;
    int adam_t = 0;
};

static int net_alloc(gx_ctx *c) {
    if (c->net) return GX_OK;
    Net *n = new Net();
    c->net = n;
    const int64_t P = param_count();
    GX_CHECK(c, cudaMalloc(&n->params, P * sizeof(float)));
    GX_CHECK(c, cudaMalloc(&n->grad, P * sizeof(float)));
    GX_CHECK(c, cudaMalloc(&n->m1, P * sizeof(float)));
    GX_CHECK(c, cudaMalloc(&n->m2, P * sizeof(float)));
    GX_CHECK(c, cudaMemset(n->m1, 0, P * sizeof(float)));
    GX_CHECK(c, cudaMemset(n->m2, 0, P * sizeof(float)));
    for (int l = 0; l < kNL; ++l) {
        GX_CHECK(c, cudaMalloc(&n->wf[l], (size_t)kNmma[l] * 9 * kCinP[l] * sizeof(bf16)));
        GX_CHECK(c, cudaMalloc(&n->bias[l], kCoutP[l] * sizeof(float)));
        if (l > 0) GX_CHECK(c, cudaMalloc(&n->wd[l], (size_t)kCin[l] * 9 * kGCoutP[l] * sizeof(bf16)));
        GX_CHECK(c, cudaMalloc(&n->gw[l], (size_t)kGCoutP[l] * 9 * kCinP[l] * sizeof(float)));
        GX_CHECK(c, cudaMalloc(&n->gb[l], kGCoutP[l] * sizeof(float)));
    }
    GX_CHECK(c, cudaMalloc(&n->dsum, 4 * sizeof(double)));
    // default initialisation: small random weights (He scale), zero biases
    std::vector<float> h(P, 0.f);
    std::mt19937_64 rng(12345);
    std::normal_distribution<float> nd(0.f, 1.f);
    for (int l = 0; l < kNL; ++l) {
        const float sc = std::sqrt(2.f / (9.f * kCin[l])) * (l == kNL - 1 ? 0.1f : 1.f);
        const int64_t off = param_offset(l);
        for (int64_t i = 0; i < layer_w_count(l); ++i) h[off + i] = sc * nd(rng);
    }
    GX_CHECK(c, cudaMemcpy(n->params, h.data(), P * sizeof(float), cudaMemcpyHostToDevice));
    return GX_OK;
}

static int net_refresh(gx_ctx *c, cudaStream_t st) {
    Net *n = c->net;
    for (int l = 0; l < kNL; ++l) {
        k_pack_weights<<<64, 256, 0, st>>>(n->params, n->wf[l], n->bias[l], l > 0 ? n->wd[l] : nullptr, kCin[l],
                                            kCout[l], kCinP[l], kNmma[l], kCoutP[l], kGCoutP[l], param_offset(l));
        GX_LAUNCHED(c);
    }
    n->have_weights = 1;
    return GX_OK;
}

// activation buffers for B images of H x W
static int net_reserve(gx_ctx *c, int B, int H, int W) {
    Net *n = c->net;
    const int64_t pix = (int64_t)B * H * W, halo = (int64_t)B * (H + 2) * (W + 2);
    if (pix <= n->cap_pix && halo <= n->cap_halo) return GX_OK;
    bf16 **b16[] = {&n->x0, &n->h1, &n->h2, &n->h3, &n->d4, &n->d3, &n->d2, &n->d1};
    const int ch[] = {16, 32, 32, 32, 16, 32, 32, 32};
    for (int i = 0; i < 8; ++i) {
        if (*b16[i]) cudaFree(*b16[i]);
        *b16[i] = nullptr;
        GX_CHECK(c, cudaMalloc(b16[i], (size_t)halo * ch[i] * sizeof(bf16)));
    }
    if (n->y) cudaFree(n->y);
    if (n->target) cudaFree(n->target);
    GX_CHECK(c, cudaMalloc(&n->y, (size_t)pix * 8 * sizeof(float)));
    GX_CHECK(c, cudaMalloc(&n->target, (size_t)pix * 3 * sizeof(float)));
    n->cap_pix = pix;
    n->cap_halo = halo;
    return GX_OK;
}

// one persistent wave of k_convtc over the units of a, input `in` with CIN channels
template <int CIN, int N, int COUTG, int EPI>
static int launch_conv(gx_ctx *c, const bf16 *in, gxv::Args a, cudaStream_t st, const int *skip = nullptr) {
    constexpr int smem = gxv::smem_bytes<CIN, N, kConvRows>() + 128;   // + alignment slack
    const void *kfn = (const void *)k_convtc<CIN, N, COUTG, EPI>;
    static int cap = 0;     // resident CTAs on the device
    if (!cap) {
        int dev = 0, nsm = 0, per = 0;
        GX_CHECK(c, cudaGetDevice(&dev));
        GX_CHECK(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        GX_CHECK(c, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        GX_CHECK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kfn, 2 * gxv::kThreads, smem));
        // tensor memory: 512 columns per SM, kTmemCols per resident CTA
        per = std::min(per, 512 / gxv::Shape<CIN, N, kConvRows>::kTmemCols);
        cap = std::max(1, per * nsm);
    }
    a.err = &c->dflags->timeout;
    const int64_t units = (int64_t)a.B * ((a.H + kConvRows - 1) / kConvRows) * ((a.W + gxv::kTW - 1) / gxv::kTW);
    k_convtc<CIN, N, COUTG, EPI><<<(unsigned)std::min<int64_t>(units, cap), 2 * gxv::kThreads, smem, st>>>(in, a, skip);
    GX_LAUNCHED(c);
    return GX_OK;
}

template <int CIN, int N, int COUTG, int EPI>
static int conv(gx_ctx *c, const bf16 *in, const bf16 *w, const float *bias, void *out, const bf16 *mask, int B, int H,
                int W, int periodic, cudaStream_t st, const int *skip = nullptr) {
    gxv::Args a{};
    a.wtc = w;
    a.bias = bias;
    a.out = out;
    a.mask = mask;
    a.B = B;
    a.H = H;
    a.W = W;
    a.periodic = periodic;
    return launch_conv<CIN, N, COUTG, EPI>(c, in, a, st, skip);
}

template <int CIN, int COUTP>
static int wgrad(gx_ctx *c, const bf16 *dy, const bf16 *x, float *gw, float *gb, int B, int H, int W, int periodic,
                 cudaStream_t st) {
    WgArgs a{dy, x, gw, gb, B, H, W, periodic};
    const int64_t tiles = (int64_t)((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH) * B;
    k_wgrad<CIN, COUTP><<<(unsigned)std::min<int64_t>(tiles, 152 * 2), 256, 0, st>>>(a);
    GX_LAUNCHED(c);
    return GX_OK;
}

// forward through the four layers (input in n->x0), output FP32 [pix][8] in n->y
static int net_forward(gx_ctx *c, int B, int H, int W, int periodic, cudaStream_t st, const int *skip = nullptr) {
    using gxv::EPI_RELU;
    Net *n = c->net;
    int rc;
    if ((rc = conv<16, 32, 32, EPI_RELU>(c, n->x0, n->wf[0], n->bias[0], n->h1, nullptr, B, H, W, periodic, st, skip)))
        return rc;
    if ((rc = conv<32, 32, 32, EPI_RELU>(c, n->h1, n->wf[1], n->bias[1], n->h2, nullptr, B, H, W, periodic, st, skip)))
        return rc;
    if ((rc = conv<32, 32, 32, EPI_RELU>(c, n->h2, n->wf[2], n->bias[2], n->h3, nullptr, B, H, W, periodic, st, skip)))
        return rc;
    return conv<32, 32, 8, gxv::EPI_F32>(c, n->h3, n->wf[3], n->bias[3], n->y, nullptr, B, H, W, periodic, st, skip);
}

// backward from dY4 (in n->d4): weight gradients (FP32 sums, zeroed here) and
// data gradients down to layer 1; then the gradient in the master layout
static int net_backward(gx_ctx *c, int B, int H, int W, int periodic, float grad_scale, cudaStream_t st) {
    Net *n = c->net;
    int rc;
    for (int l = 0; l < kNL; ++l) {
        GX_CHECK(c, cudaMemsetAsync(n->gw[l], 0, (size_t)kGCoutP[l] * 9 * kCinP[l] * sizeof(float), st));
        GX_CHECK(c, cudaMemsetAsync(n->gb[l], 0, kGCoutP[l] * sizeof(float), st));
    }
    if ((rc = wgrad<32, 16>(c, n->d4, n->h3, n->gw[3], n->gb[3], B, H, W, periodic, st))) return rc;
    if ((rc = conv<16, 32, 32, gxv::EPI_MASK>(c, n->d4, n->wd[3], nullptr, n->d3, n->h3, B, H, W, periodic, st)))
        return rc;
    if ((rc = wgrad<32, 32>(c, n->d3, n->h2, n->gw[2], n->gb[2], B, H, W, periodic, st))) return rc;
    if ((rc = conv<32, 32, 32, gxv::EPI_MASK>(c, n->d3, n->wd[2], nullptr, n->d2, n->h2, B, H, W, periodic, st)))
        return rc;
    if ((rc = wgrad<32, 32>(c, n->d2, n->h1, n->gw[1], n->gb[1], B, H, W, periodic, st))) return rc;
    if ((rc = conv<32, 32, 32, gxv::EPI_MASK>(c, n->d2, n->wd[1], nullptr, n->d1, n->h1, B, H, W, periodic, st)))
        return rc;
    if ((rc = wgrad<16, 32>(c, n->d1, n->x0, n->gw[0], n->gb[0], B, H, W, periodic, st))) return rc;
    for (int l = 0; l < kNL; ++l) {
        k_unpack_grad<<<64, 256, 0, st>>>(n->gw[l], n->gb[l], n->grad, kCin[l], kCout[l], kCinP[l], param_offset(l),
                                          grad_scale);
        GX_LAUNCHED(c);
    }
    return GX_OK;
}

// ------------------------------------------------------------ solver hooks
// pointers for the solver kernel, which applies the network to its Krylov
// columns itself (weights refreshed, activations sized for the grid)
int gx_net_solver_args(gx_ctx *c, NetSolverArgs *out, cudaStream_t st) {
    if (c->dim != 2) { c->err = "the learned preconditioner is 2D"; return GX_ENOTIMPL; }
    int rc = net_alloc(c);
    if (rc) return rc;
    Net *n = c->net;
    if (!n->have_weights && (rc = net_refresh(c, st))) return rc;
    const int H = c->n[1], W = c->n[0];
    if ((rc = net_reserve(c, 1, H, W))) return rc;
    for (int l = 0; l < kNL; ++l) { out->w[l] = n->wf[l]; out->b[l] = n->bias[l]; }
    out->x0 = n->x0; out->h1 = n->h1; out->h2 = n->h2; out->h3 = n->h3;
    const int nflags = 3 * gxn::pipe_units(H, W);
    if (nflags > n->cap_flags) {
        if (n->flags) cudaFree(n->flags);
        n->flags = nullptr;
        GX_CHECK(c, cudaMalloc(&n->flags, (size_t)nflags * sizeof(unsigned)));
        n->cap_flags = nflags;
    }
    out->flags = n->flags;
    return GX_OK;
}

// collection of (residual, error) pairs around one solve with initial guess
// E^n: the first residual r0 = b - A E^n is kept when the solve starts and the
// error e = E^{n+theta} - E^n is added once it has converged.  The inputs the
// preconditioner sees inside FGMRES are Krylov vectors, which carry far more
// small-scale content than r0, so the first kKrylovPairs basis vectors V_j of
// the solve are added too, as exact pairs (A V_j, V_j) at one matrix-vector
// product each.
constexpr int kKrylovPairs = 6;

int gx_net_collecting(const gx_ctx *c) { return c->net && c->net->collect && c->net->cap_pairs > 0; }

int gx_net_pair_begin(gx_ctx *c, const double *r0, cudaStream_t st) {
    Net *n = c->net;
    if (!n || !n->collect || n->cap_pairs < 1) return GX_OK;
    // the targets need D^-1 of this solve's operator
    if (c->cfg.precond == GX_PRECOND_NONE) {
        int rc = gx_build_jacobi(c, st);
        if (rc) return rc;
    }
    float *dst = n->pairs + (size_t)n->next_pair * 6 * c->N;
    k_store_r<<<nblk(3 * c->N), 256, 0, st>>>(r0, 3 * c->N, dst);
    GX_LAUNCHED(c);
    n->pending_pair = 1;
    return GX_OK;
}

// the pair slot next_pair is complete: keep it (ring of field pairs), or, with the
// crop store, cut its windows and reuse the slot
static int advance_slot(gx_ctx *c, cudaStream_t st) {
    Net *n = c->net;
    if (!n->crop_mode) {
        n->next_pair = (n->next_pair + 1) % n->cap_pairs;
        n->npairs = std::min(n->npairs + 1, n->cap_pairs);
        return GX_OK;
    }
    const float *pair = n->pairs + (size_t)n->next_pair * 6 * c->N;
    GX_CHECK(c, cudaMemsetAsync(n->csum, 0, sizeof(double), st));
    k_sumsq_r<<<nblk(3 * c->N), 256, 0, st>>>(pair, 3 * c->N, n->csum);
    GX_LAUNCHED(c);
    CutArgs a{};
    a.pair = pair; a.N = c->N; a.nx = c->n[0]; a.ny = c->n[1]; a.S = n->crop_C + 8;
    a.seed = n->crop_seed; a.counter = n->crop_counter; a.sumsq = n->csum;
    a.crops = n->crops; a.scales = n->cscales; a.cap = n->cap_crops; a.next = n->next_crop;
    const int cnt = std::min(n->per_pair, n->cap_crops);
    k_cut_crops<<<dim3(std::max(1, (a.S * a.S + 255) / 256), cnt), 256, 0, st>>>(a);
    GX_LAUNCHED(c);
    n->crop_counter += (uint64_t)cnt;
    n->next_crop = (n->next_crop + cnt) % n->cap_crops;
    n->ncrops = std::min(n->ncrops + cnt, n->cap_crops);
    return GX_OK;
}

int gx_net_pair_end(gx_ctx *c, int converged, int nbasis, cudaStream_t st) {
    Net *n = c->net;
    if (!n || !n->pending_pair) return GX_OK;
    n->pending_pair = 0;
    if (!converged) return GX_OK;
    const int64_t n3 = 3 * c->N;
    float *dst = n->pairs + (size_t)n->next_pair * 6 * c->N;
    k_store_t<<<nblk(c->N), 256, 0, st>>>(c->jdiag, c->Eth, c->E, c->N, dst);
    GX_LAUNCHED(c);
    int rc = advance_slot(c, st);
    if (rc) return rc;
    // the mixed-precision solve keeps its Krylov basis in FP32: only (r0, e) then
    const int nv = c->cfg.gmres_mixed ? 0 : std::min(nbasis, kKrylovPairs);
    for (int j = 0; j < nv; ++j) {
        const double *v = c->V + (size_t)j * n3;
        rc = gx_apply_A(c, v, c->w, st);
        if (rc) return rc;
        dst = n->pairs + (size_t)n->next_pair * 6 * c->N;
        k_store_rt<<<nblk(c->N), 256, 0, st>>>(c->jdiag, c->w, v, c->N, dst);
        GX_LAUNCHED(c);
        if ((rc = advance_slot(c, st))) return rc;
    }
    return GX_OK;
}

void gx_net_free(gx_ctx *c) {
    Net *n = c->net;
    if (!n) return;
    void *ps[] = {n->params, n->grad, n->m1, n->m2, n->x0, n->h1, n->h2, n->h3, n->d4, n->d3, n->d2, n->d1, n->y,
                  n->target, n->dsum, n->pairs, n->flags, n->crops, n->cscales, n->csum};
    for (void *p : ps)
        if (p) cudaFree(p);
    for (int l = 0; l < kNL; ++l) {
        void *qs[] = {n->wf[l], n->wd[l], n->bias[l], n->gw[l], n->gb[l]};
        for (void *q : qs)
            if (q) cudaFree(q);
    }
    delete n;
    c->net = nullptr;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

int64_t gx_precond_param_count(void) { return param_count(); }

int gx_precond_set_weights(gx_ctx *c, const float *params, int64_t n, int ptr_is_device) {
    if (!c || !params || n != param_count()) {
        if (c) c->err = "gx_precond_set_weights: need gx_precond_param_count() values";
        return GX_EINVAL;
    }
    int rc = net_alloc(c);
    if (rc) return rc;
    GX_CHECK(c, cudaMemcpy(c->net->params, params, n * sizeof(float),
                           ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    GX_CHECK(c, cudaMemset(c->net->m1, 0, n * sizeof(float)));
    GX_CHECK(c, cudaMemset(c->net->m2, 0, n * sizeof(float)));
    c->net->adam_t = 0;
    rc = net_refresh(c, 0);
    if (rc) return rc;
    GX_CHECK(c, cudaStreamSynchronize(0));
    return GX_OK;
}

int gx_precond_get_weights(gx_ctx *c, float *params, int64_t n, int ptr_is_device) {
    if (!c || !params || n != param_count()) return GX_EINVAL;
    int rc = net_alloc(c);
    if (rc) return rc;
    GX_CHECK(c, cudaMemcpy(params, c->net->params, n * sizeof(float),
                           ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    return GX_OK;
}

int gx_precond_collect(gx_ctx *c, int capacity) {
    if (!c || capacity < 0) return GX_EINVAL;
    if (c->dim != 2) { c->err = "the learned preconditioner is 2D"; return GX_ENOTIMPL; }
    int rc = net_alloc(c);
    if (rc) return rc;
    Net *n = c->net;
    if (capacity == 0) { n->collect = 0; return GX_OK; }
    n->crop_mode = 0;
    if (capacity != n->cap_pairs) {
        if (n->pairs) cudaFree(n->pairs);
        n->pairs = nullptr;
        GX_CHECK(c, cudaMalloc(&n->pairs, (size_t)capacity * 6 * c->N * sizeof(float)));
        n->cap_pairs = capacity;
        n->npairs = 0;
        n->next_pair = 0;
    }
    n->collect = 1;
    return GX_OK;
}

int gx_precond_collect_crops(gx_ctx *c, int capacity, int crop, int per_pair, uint64_t seed) {
    if (!c || capacity < 0 || (capacity > 0 && (crop < 8 || per_pair < 1))) return GX_EINVAL;
    if (c->dim != 2) { c->err = "the learned preconditioner is 2D"; return GX_ENOTIMPL; }
    int rc = net_alloc(c);
    if (rc) return rc;
    Net *n = c->net;
    if (capacity == 0) { n->collect = 0; return GX_OK; }
    const int S = crop + 8;
    if (S > c->n[0] || S > c->n[1]) { c->err = "crop + 8 exceeds the grid"; return GX_EINVAL; }
    // one field pair slot as the cut's source
    if (n->cap_pairs != 1) {
        if (n->pairs) cudaFree(n->pairs);
        n->pairs = nullptr;
        GX_CHECK(c, cudaMalloc(&n->pairs, (size_t)6 * c->N * sizeof(float)));
        n->cap_pairs = 1;
    }
    n->npairs = 0;
    n->next_pair = 0;
    if (capacity != n->cap_crops || crop != n->crop_C) {
        if (n->crops) cudaFree(n->crops);
        if (n->cscales) cudaFree(n->cscales);
        n->crops = nullptr;
        n->cscales = nullptr;
        GX_CHECK(c, cudaMalloc(&n->crops, (size_t)capacity * 6 * S * S * sizeof(float)));
        GX_CHECK(c, cudaMalloc(&n->cscales, (size_t)capacity * sizeof(float)));
        n->cap_crops = capacity;
        n->crop_C = crop;
        n->ncrops = 0;
        n->next_crop = 0;
    }
    if (!n->csum) GX_CHECK(c, cudaMalloc(&n->csum, sizeof(double)));
    n->per_pair = per_pair;
    n->crop_seed = seed;
    n->crop_mode = 1;
    n->collect = 1;
    return GX_OK;
}

int gx_precond_crop(gx_ctx *c, int k, float *out, float *scale) {
    if (!c || !out || !scale) return GX_EINVAL;
    Net *n = c->net;
    if (!n || !n->crop_mode || k < 0 || k >= n->ncrops) { if (c) c->err = "no such crop"; return GX_EINVAL; }
    const int S = n->crop_C + 8;
    GX_CHECK(c, cudaMemcpy(out, n->crops + (size_t)k * 6 * S * S, (size_t)6 * S * S * sizeof(float),
                           cudaMemcpyDeviceToHost));
    GX_CHECK(c, cudaMemcpy(scale, n->cscales + k, sizeof(float), cudaMemcpyDeviceToHost));
    return GX_OK;
}

int gx_precond_pairs(gx_ctx *c) {
    if (!c) return -1;
    if (!c->net) return 0;
    return c->net->crop_mode ? c->net->ncrops : c->net->npairs;
}

int gx_precond_train(gx_ctx *c, int npairs, int crop, int batch, int epochs, float lr, uint64_t seed,
                     float *loss_out, void *stream) {
    if (!c || npairs < 1 || crop < 8 || batch < 1 || epochs < 1 || !(lr > 0)) return GX_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Net *n = c->net;
    const bool from_crops = n && n->crop_mode;
    if (!n || (from_crops ? n->ncrops : n->npairs) < 1) {
        c->err = "no collected pairs: call gx_precond_collect and run some solves";
        return GX_ESTATE;
    }
    if (from_crops && crop != n->crop_C) { c->err = "crop differs from the collected crops' size"; return GX_EINVAL; }
    if (!n->have_weights) { int rc = net_refresh(c, st); if (rc) return rc; }
    const int S = crop + 8;
    int rc = net_reserve(c, batch, S, S);
    if (rc) return rc;
    CropSpec *dspec = nullptr;
    float *dscale = nullptr;
    GX_CHECK(c, cudaMalloc(&dspec, batch * sizeof(CropSpec)));
    GX_CHECK(c, cudaMalloc(&dscale, batch * sizeof(float)));
    std::mt19937_64 rng(seed);
    std::vector<CropSpec> spec(batch);
    const int64_t P = param_count();
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const int total_steps = epochs * ((npairs + batch - 1) / batch);
    int step_i = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        GX_CHECK(c, cudaMemsetAsync(n->dsum + 1, 0, sizeof(double), st));
        int nb = 0;
        for (int done = 0; done < npairs; done += batch, ++nb) {
            const int B = std::min(batch, npairs - done);
            for (int b = 0; b < B; ++b) {
                spec[b].pair = (int)(rng() % (uint64_t)(from_crops ? n->ncrops : n->npairs));
                spec[b].y0 = (int)(rng() % (uint64_t)c->n[1]);
                spec[b].x0 = (int)(rng() % (uint64_t)c->n[0]);
                spec[b].pad = 0;
            }
            GX_CHECK(c, cudaMemcpyAsync(dspec, spec.data(), B * sizeof(CropSpec), cudaMemcpyHostToDevice, st));
            if (from_crops) {
                k_crop_gather_store<<<dim3(nblk((int64_t)S * S), B), 256, 0, st>>>(n->crops, dspec, crop, n->x0,
                                                                                   n->target);
                GX_LAUNCHED(c);
            } else {
                k_crop_scale<<<B, 1024, 0, st>>>(n->pairs, c->N, dspec, dscale);
                GX_LAUNCHED(c);
                k_crop_gather<<<dim3(nblk((int64_t)S * S), B), 256, 0, st>>>(n->pairs, c->N, c->n[0], c->n[1], dspec,
                                                                               crop, dscale, n->x0, n->target);
                GX_LAUNCHED(c);
            }
            if ((rc = net_forward(c, B, S, S, 0, st))) return rc;
            const float inv_nout = 1.f / (3.f * crop * crop * B);
            k_loss<<<nblk((int64_t)B * S * S), 256, 0, st>>>(n->y, n->target, B, S, S, 4, 4, crop, crop, inv_nout,
                                                               n->d4, n->dsum + 1);
            GX_LAUNCHED(c);
            if ((rc = net_backward(c, B, S, S, 0, 1.f, st))) return rc;
            ++n->adam_t;
            const float c1 = 1.f - std::pow(b1, (float)n->adam_t), c2 = 1.f - std::pow(b2, (float)n->adam_t);
            // cosine decay of the step size over the call, down to lr / 20
            const double prog = (double)(step_i++) / std::max(1, total_steps - 1);
            const float lr_t = (float)(lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(3.141592653589793 * prog))));
            k_adam<<<nblk(P), 256, 0, st>>>(n->params, n->grad, n->m1, n->m2, P, lr_t, b1, b2, eps, c1, c2);
            GX_LAUNCHED(c);
            if ((rc = net_refresh(c, st))) return rc;
        }
        double L = 0;
        GX_CHECK(c, cudaMemcpyAsync(&L, n->dsum + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
        GX_CHECK(c, cudaStreamSynchronize(st));
        if (loss_out) loss_out[ep] = (float)(L / nb);
    }
    cudaFree(dspec);
    cudaFree(dscale);
    return GX_OK;
}

int gx_precond_forward(gx_ctx *c, int H, int W, const float *in, float *out, void *stream) {
    if (!c || H < 1 || W < 1 || !in || !out) return GX_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = net_alloc(c);
    if (rc) return rc;
    Net *n = c->net;
    if (!n->have_weights && (rc = net_refresh(c, st))) return rc;
    if ((rc = net_reserve(c, 1, H, W))) return rc;
    k_pack_input<float><<<nblk((int64_t)H * W), 256, 0, st>>>(in, H, W, 1.0, 1, n->x0);
    GX_LAUNCHED(c);
    if ((rc = net_forward(c, 1, H, W, 1, st))) return rc;
    k_f32_to_chw3<<<nblk((int64_t)H * W), 256, 0, st>>>(n->y, (int64_t)H * W, out);
    GX_LAUNCHED(c);
    GX_CHECK(c, cudaStreamSynchronize(st));
    return GX_OK;
}

int gx_precond_apply(gx_ctx *c, const double *v, double *z, void *stream) {
    if (!c || !v || !z || v == z) return GX_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t N = c->N;
    const int pc = c->cfg.precond;
    if (pc == GX_PRECOND_NONE) {
        GX_CHECK(c, cudaMemcpyAsync(z, v, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
        GX_CHECK(c, cudaStreamSynchronize(st));
        return GX_OK;
    }
    int rc = pc == GX_PRECOND_JACOBI ? gx_build_jacobi(c, st) : gx_build_jacobi32(c, st);
    if (rc) return rc;
    if (pc == GX_PRECOND_JACOBI) {
        if ((rc = gx_apply_jacobi(c, v, z, st))) return rc;
        GX_CHECK(c, cudaStreamSynchronize(st));
        return GX_OK;
    }
    NetSolverArgs nn;
    if ((rc = gx_net_solver_args(c, &nn, st))) return rc;
    const double vn = gx_norm_host(c, v, 3 * N, st, &rc);
    if (rc) return rc;
    if (vn == 0.0) {
        GX_CHECK(c, cudaMemsetAsync(z, 0, 3 * N * sizeof(double), st));
        GX_CHECK(c, cudaStreamSynchronize(st));
        return GX_OK;
    }
    const double s = vn / std::sqrt(3.0 * (double)N);
    const int H = c->n[1], W = c->n[0];
    gxn::PipeArgs p;
    p.in[0] = static_cast<const bf16 *>(nn.x0);
    p.in[1] = static_cast<const bf16 *>(nn.h1);
    p.in[2] = static_cast<const bf16 *>(nn.h2);
    p.in[3] = static_cast<const bf16 *>(nn.h3);
    p.out[0] = static_cast<bf16 *>(nn.h1);
    p.out[1] = static_cast<bf16 *>(nn.h2);
    p.out[2] = static_cast<bf16 *>(nn.h3);
    for (int l = 0; l < kNL; ++l) {
        p.w[l] = static_cast<const bf16 *>(nn.w[l]);
        p.bias[l] = nn.b[l];
    }
    p.v = v;
    p.jd = c->jdiag32;
    p.z = z;
    p.s = (float)s;
    p.flags = nn.flags;
    p.err = &c->dflags->timeout;
    p.H = H;
    p.W = W;
    constexpr int smem = gxn::kSmemBytes + 128;
    static int grid = 0;
    if (!grid) {
        int dev = 0, nsm = 0, per = 0;
        GX_CHECK(c, cudaGetDevice(&dev));
        GX_CHECK(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        GX_CHECK(c, cudaFuncSetAttribute((const void *)k_net_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        GX_CHECK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)k_net_apply, 2 * gxv::kThreads,
                                                                  smem));
        grid = std::max(1, std::min(per, 1) * nsm);   // one CTA per SM: its tensor memory
    }
    bf16 *x0 = static_cast<bf16 *>(nn.x0);
    float inv_s = (float)(1.0 / s);
    void *kargs[] = {&p, &x0, &inv_s};
    GX_CHECK(c, cudaLaunchCooperativeKernel((const void *)k_net_apply, dim3(grid), dim3(2 * gxv::kThreads), kargs, smem,
                                            st));
    GX_LAUNCHED(c);
    GX_CHECK(c, cudaStreamSynchronize(st));
    return GX_OK;
}

int gx_precond_loss_grad(gx_ctx *c, int H, int W, const float *in, const float *target, float *loss, float *grad,
                         void *stream) {
    if (!c || H < 1 || W < 1 || !in || !target || !grad) return GX_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = net_alloc(c);
    if (rc) return rc;
    Net *n = c->net;
    if (!n->have_weights && (rc = net_refresh(c, st))) return rc;
    if ((rc = net_reserve(c, 1, H, W))) return rc;
    const int64_t HW = (int64_t)H * W;
    k_pack_input<float><<<nblk(HW), 256, 0, st>>>(in, H, W, 1.0, 0, n->x0);
    GX_LAUNCHED(c);
    k_chw3_to_target<<<nblk(HW), 256, 0, st>>>(target, HW, n->target);
    GX_LAUNCHED(c);
    if ((rc = net_forward(c, 1, H, W, 0, st))) return rc;
    GX_CHECK(c, cudaMemsetAsync(n->dsum + 1, 0, sizeof(double), st));
    k_loss<<<nblk(HW), 256, 0, st>>>(n->y, n->target, 1, H, W, 0, 0, H, W, 1.f / (3.f * HW), n->d4, n->dsum + 1);
    GX_LAUNCHED(c);
    if ((rc = net_backward(c, 1, H, W, 0, 1.f, st))) return rc;
    GX_CHECK(c, cudaMemcpyAsync(grad, n->grad, param_count() * sizeof(float), cudaMemcpyDeviceToDevice, st));
    double L = 0;
    GX_CHECK(c, cudaMemcpyAsync(&L, n->dsum + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    GX_CHECK(c, cudaStreamSynchronize(st));
    if (loss) *loss = (float)L;
    return GX_OK;
}

}  // extern "C"
