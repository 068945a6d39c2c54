// gx_convtc.cuh -- the 3x3 convolution of the learned preconditioner on the
// fifth-generation tensor cores (tcgen05.mma kind::f16, BF16 operands, FP32
// accumulation in tensor memory), fed by TMA bulk copies.
//
// Implicit GEMM with the three kernel rows folded into N: one MMA per (input
// row rho, kernel column kx, 16 input channels),
//     D[128 pixels][3 NB] += A_{rho,kx}[128 pixels][16] * W_kx[3 NB][16]^T,
// where W_kx stacks the weights of kernel rows ky = 2, 1, 0 (NB output
// channels each).  D starts at the accumulator block of output row rho - 2,
// so its three NB-column blocks land on output rows rho - 2, rho - 1, rho with
// ky = 2, 1, 0 -- exactly the contributions of input row rho -- and tensor
// memory adds them up across rows.  A unit of R rows takes 3 (R + 2) CIN / 16
// MMAs instead of 9 R CIN / 16 (the tensor core accepts a narrow MMA no
// faster than a wide one).  Accumulators start at zero: the epilogue clears
// each output row's block after reading it (the two blocks on either side of
// the unit receive out-of-unit terms and are never read).
// Activations live in global memory as channel-blocked BF16 images with a
// one-pixel halo ring, [B][C/8][H + 2][W + 2][8]: the producer of a layer
// writes every edge pixel a second time into the ring (its periodic image, or
// zero for zero padding), so a tile needs no index arithmetic.  A unit of
// work is R image rows x 128 columns; its input tile, (R + 2) rows x 130
// columns, arrives in shared memory as C/8 channel slabs -- slab g holds
// channels 8g .. 8g + 7 of every tile pixel, one 16-byte chunk per pixel,
// pixels in row-major order.  In the blocked layout one tile row of one slab
// is 130 x 16 = 2080 contiguous bytes, so the tile is (R + 2) * C/8 bulk
// copies (TMA, cp.async.bulk), one per lane of the producer warp.  The A
// operand of tap (ky, kx) for output row r is then the 128 consecutive chunks
// starting at tile pixel (r + ky) * 130 + kx: one descriptor with a start
// moved by whole chunks (no im2col copy), LBO = slab size (next 8 channels),
// SBO = 128 bytes.  The weights come pre-packed in the same form (slab = 8
// input channels of one tap for all N outputs) by one more bulk copy.
//
// Warp roles of the 256-thread CTA, synchronised by mbarriers only:
//   warp 0:        producer (bulk copies), a ring of kStages tiles;
//   warp 1 lane 0: MMA issuer, 3 (R + 2) CIN / 16 MMAs per unit into one of
//                  two accumulator sets, then commits (stage free, accumulators full);
//   warps 4..7:    epilogue, warp w reading TMEM lane quarter w % 4 (pixels
//                  32 (w % 4) .. + 31 of the unit's 128 columns), row by row,
//                  clearing each row's block, then releasing the set.  A
//                  512-thread CTA has a second epilogue group, warps 12..15,
//                  and the two groups take alternate rows.
// So tile loads, MMAs and epilogue stores of consecutive units overlap.
//
// Epilogues: ReLU to BF16 (halo ring included), FP32 without halo (padded
// output channels), the ReLU mask of the data gradient, and -- inside the
// solver -- the preconditioned vector z = D^-1 v + s N(v / s), evaluated in
// FP32 (a preconditioner needs no FP64: FGMRES judges the FP64 residual) and
// stored as FP64.
#pragma once

#include <cuda_bf16.h>

#include "gx_tc.cuh"

namespace gxv {

typedef __nv_bfloat16 bf16;

constexpr int kTW = 128;            // output columns of a unit (the MMA's M)
constexpr int kTileRow = kTW + 2;   // tile row with its halo (pixels)
constexpr int kThreads = 256;       // eight warps: one role group (a CTA may run 1 or 2 groups)
constexpr int kStages = 2;          // tiles in flight
constexpr int kWaitLimit = 1 << 22; // mbarrier polls before a wait gives up

enum { EPI_RELU = 0, EPI_F32 = 1, EPI_MASK = 2, EPI_Z = 3 };

struct Args {
    const bf16 *wtc;      // weights packed [3 kx][CIN / 8][3 N (ky = 2, 1, 0)][8] (zero rows beyond COUTG)
    const float *bias;    // [COUTG] or null
    void *out;            // EPI_RELU / EPI_MASK: bf16 [B][N/8][H+2][W+2][8]; EPI_F32: float [B][H][W][COUTG]
    const bf16 *mask;     // EPI_MASK: bf16 [B][N/8][H+2][W+2][8], keep where > 0
    const double *v;      // EPI_Z: Krylov vector [3][H*W] (B = 1)
    const float *jd;      // EPI_Z: block-Jacobi inverse [H*W][9], FP32
    double *z;            // EPI_Z: [3][H*W]
    double s;             // EPI_Z: output scale s
    int *err;             // set when a bounded wait gives up
    int B, H, W, periodic;
};

template <int CIN, int N, int R>   // N: output channels of one row block (NB)
struct Shape {
    static_assert(CIN % 16 == 0 && N % 16 == 0 && N <= 32 && R >= 1 && R <= 4, "supported shapes");
    static constexpr int kSlabBytes = (R + 2) * kTileRow * 16;
    static constexpr int kTileBytes = (CIN / 8) * kSlabBytes;
    static constexpr int kLoads = (CIN / 8) * (R + 2);                   // bulk copies per tile (one row of one slab)
    static_assert(kLoads <= 32, "one copy per lane of the producer warp");
    static constexpr int kWSlabBytes = 3 * N * 16;                       // 8 input channels x 3 NB rows of W_kx
    static constexpr int kWBytes = 3 * (CIN / 8) * kWSlabBytes;
    static constexpr int kAccCols = (R + 4) * N;                         // blocks of output rows -2 .. R+1
    static constexpr int kTmemCols = 2 * kAccCols <= 128 ? 128 : 2 * kAccCols <= 256 ? 256 : 512;
    static_assert(2 * kAccCols <= 512, "two accumulator sets in tensor memory");
    // [weights][kStages tiles][bias 32 floats][barriers][tmem address, abort flag, units issued]
    // (tile pixels beyond the padded image are never written: they feed no valid output)
    static constexpr int kBiasOff = kWBytes + kStages * kTileBytes;
    static constexpr int kBarOff = kBiasOff + 4 * 32;
    static constexpr int kNumBars = 1 + 2 * kStages + 4;                 // weights, full/empty, acc full/empty
    static constexpr int kMiscOff = kBarOff + 8 * kNumBars;
    static constexpr int kSmemBytes = kMiscOff + 16;
};

// shared memory a conv of this shape needs (bytes, from a 128-byte aligned base)
template <int CIN, int N, int R>
__host__ __device__ constexpr int smem_bytes() { return Shape<CIN, N, R>::kSmemBytes; }

// decode a unit index into (image, first row, first column)
template <int R>
__device__ __forceinline__ void unit_pos(int u, int nseg, int nblk, int &b, int &y0, int &x0) {
    const int t = u / nseg;
    x0 = (u - t * nseg) * kTW;
    b = t / nblk;
    y0 = (t - b * nblk) * R;
}

// offset (elements) of the 8-channel chunk g of pixel (b, y, x) of a
// channel-blocked image with a halo ring and G chunks per pixel; y in
// [-1, H], x in [-1, W]
__host__ __device__ __forceinline__ int64_t blk_off(int b, int g, int y, int x, int H, int W, int G) {
    return ((((int64_t)b * G + g) * (H + 2) + (y + 1)) * (W + 2) + (x + 1)) * 8;
}

// store the C-channel value `val` (C/8 uint4) of pixel (b, y, x) into an image
// with a halo ring, and into the ring positions that image the pixel (its
// periodic copies, or zeros for zero padding); every ring position images
// exactly one pixel, so each is written once
template <int C>
__device__ __forceinline__ void store_with_halo(bf16 *img, int b, int y, int x, int H, int W, int periodic,
                                                const uint4 (&val)[C / 8]) {
    const uint4 zero = make_uint4(0, 0, 0, 0);
    auto put = [&](int yy, int xx, bool copy) {
#pragma unroll
        for (int g = 0; g < C / 8; ++g)
            *reinterpret_cast<uint4 *>(img + blk_off(b, g, yy, xx, H, W, C / 8)) = copy ? val[g] : zero;
    };
    put(y, x, true);
    const bool p = periodic != 0;
    const int ey = y == 0 ? H : (y == H - 1 ? -1 : -2);      // ring row imaging this pixel, or none
    const int ex = x == 0 ? W : (x == W - 1 ? -1 : -2);
    if (ey != -2) put(ey, x, p);
    if (ex != -2) put(y, ex, p);
    if (ey != -2 && ex != -2) put(ey, ex, p);
    // a one-row or one-column image is its own neighbour on both sides
    if (H == 1) {
        put(-1, x, p);
        if (ex != -2) put(-1, ex, p);
    }
    if (W == 1) {
        put(y, -1, p);
        if (ey != -2) put(ey, -1, p);
        if (H == 1) put(-1, -1, p);
    }
}

// out = epilogue(conv3x3(in, w) + bias) over the units cta, cta + ncta, ...
// Every thread of the CTA calls it (blockDim.x == 256 or 512); sm: smem_bytes()
// bytes, 128-byte aligned; in: the input image [B][CIN/8][H+2][W+2][8].  N: MMA
// width (output channels padded to 16 or 32); COUTG: output channels of w /
// bias (<= N).
template <int CIN, int N, int COUTG, int R, int EPI>
__device__ void conv_tc(const Args &args, const bf16 *in, unsigned char *sm, int cta, int ncta) {
    using namespace gxt;
    // register copies of the arguments: the inline assembly below clobbers
    // memory, which would otherwise force a reload of every field after it
    const int H = args.H, W = args.W, periodic = args.periodic;
    const bf16 *const wtc = args.wtc, *const mask = args.mask;
    const float *const bias = args.bias;
    void *const out = args.out;
    const double *const vz = args.v;
    const float *const jd = args.jd;
    double *const z = args.z;
    const double s_out = args.s;
    int *const err = args.err;
    using S = Shape<CIN, N, R>;
    static_assert(COUTG <= N && (EPI != EPI_Z || COUTG >= 3), "output channels");
    unsigned char *sW = sm;
    float *sBias = reinterpret_cast<float *>(sm + S::kBiasOff);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + S::kBarOff);
    uint64_t *wfull = bars, *full = bars + 1, *empty = bars + 1 + kStages, *accfull = bars + 1 + 2 * kStages,
             *accempty = accfull + 2;
    uint32_t *sTm = reinterpret_cast<uint32_t *>(sm + S::kMiscOff);
    volatile int *abort = reinterpret_cast<volatile int *>(sm + S::kMiscOff + 4);
    volatile int *s_issued = reinterpret_cast<volatile int *>(sm + S::kMiscOff + 8);   // units the MMA thread issued
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ngroups = blockDim.x >> 8, group = warp >> 3;    // epilogue groups, this warp's

    const int nseg = (W + kTW - 1) / kTW, nblk = (H + R - 1) / R;
    const int nunits = args.B * nblk * nseg;
    if (cta >= nunits) return;
    const int nmine = (nunits - 1 - cta) / ncta + 1;    // units of this CTA

    if (tid < 32) sBias[tid] = (bias && tid < COUTG) ? bias[tid] : 0.f;
    if (tid == 0) {
        for (int i = 0; i < S::kNumBars; ++i) mbar_init(&bars[i], i >= 1 + 2 * kStages + 2 ? 4 * 32 * ngroups : 1);
        *abort = 0;
        *s_issued = 0;
    }
    __syncwarp();
    if (warp == 0) tmem_alloc<S::kTmemCols>(sTm);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = *sTm;

    int nloaded = 0;    // (producer warp)
    if (warp == 0) {
        // ---- producer: lane 0 waits for the stage and announces the bytes, lanes issue the row copies
        if (lane == 0) {
            mbar_arrive_expect_tx(wfull, S::kWBytes);
            bulk_load(smem_addr(sW), wtc, S::kWBytes, wfull);
        }
        int i = 0;
        for (; i < nmine; ++i) {
            const int st = i % kStages, n = i / kStages;
            int b, y0, x0;
            unit_pos<R>(cta + i * ncta, nseg, nblk, b, y0, x0);
            // rows y0-1 .. y0+R of the padded image that exist (up to row H), and the
            // pixels of each from padded column x0 (= image column x0 - 1) that exist
            const int rows = min(R + 2, H + 2 - y0), npx = min(kTileRow, W + 2 - x0);
            int ok = 1;
            if (lane == 0) {
                if (n > 0) ok = mbar_wait_or_abort(&empty[st], (n - 1) & 1, kWaitLimit, abort);
                if (ok) mbar_arrive_expect_tx(&full[st], (uint32_t)(rows * (CIN / 8) * npx * 16));
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            if (lane < S::kLoads) {
                const int r = lane % (R + 2), g = lane / (R + 2);
                if (r < rows)
                    bulk_load(smem_addr(sm + S::kWBytes + st * S::kTileBytes + g * S::kSlabBytes + r * kTileRow * 16),
                              in + blk_off(b, g, y0 - 1 + r, x0 - 1, H, W, CIN / 8), npx * 16, &full[st]);
            }
        }
        nloaded = i;
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            constexpr uint32_t idesc = idesc_bf16_f32(kTW, 3 * N);
            const uint64_t bdesc = sdesc(smem_addr(sW), S::kWSlabBytes, 128);
            bool ok = mbar_wait_or_abort(wfull, 0, kWaitLimit, abort);
            int i = 0;
            for (; ok && i < nmine; ++i) {
                const int st = i % kStages, n = i / kStages, k = i & 1, m = i >> 1;
                if (!mbar_wait_or_abort(&full[st], n & 1, kWaitLimit, abort)) break;
                if (!mbar_wait_or_abort(&accempty[k], m & 1, kWaitLimit, abort)) break;
                tc_fence_after();
                const uint64_t ad = sdesc(smem_addr(sm + S::kWBytes + st * S::kTileBytes), S::kSlabBytes, 128);
                const uint32_t dacc = tm + k * S::kAccCols;
#pragma unroll
                for (int rho = 0; rho < R + 2; ++rho) {
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
                        for (int kc = 0; kc < CIN / 16; ++kc) {
                            const uint32_t aoff = (rho * kTileRow + kx) + 2 * kc * (S::kSlabBytes / 16);
                            const uint32_t boff = (kx * (CIN / 8) + 2 * kc) * (S::kWSlabBytes / 16);
                            mma_bf16(dacc + rho * N, ad + aoff, bdesc + boff, idesc, true);
                        }
                    }
                }
                mma_commit(&empty[st]);
                mma_commit(&accfull[k]);
            }
            *s_issued = i;
        }
    } else if ((warp & 7) >= 4) {
        // ---- epilogue
        const int q4 = warp & 3;
        const uint32_t lane_base = tm + ((uint32_t)(32 * q4) << 16);
        float bz[N];                   // the bias, in registers for the whole call
#pragma unroll
        for (int c = 0; c < N; ++c) bz[c] = sBias[c];
        // both accumulator sets start at zero (output-row blocks 2 .. R+1)
#pragma unroll 1
        for (int k = 0; k < 2; ++k) {
            for (int r = group; r < R; r += ngroups)
                for (int c = 0; c < N; c += 16) tmem_zero16(lane_base + k * S::kAccCols + (r + 2) * N + c);
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(&accempty[k]);
        }
        for (int i = 0; i < nmine; ++i) {
            const int k = i & 1, m = i >> 1;
            // one lane polls; the warp reads tensor memory together (.sync.aligned)
            int ok = 0;
            if (lane == 0) ok = mbar_wait_or_abort(&accfull[k], m & 1, kWaitLimit, abort);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            int b, y0, x0;
            unit_pos<R>(cta + i * ncta, nseg, nblk, b, y0, x0);
            const int xx = x0 + 32 * q4 + lane;
#pragma unroll 1
            for (int r = group; r < R; r += ngroups) {
                const int yy = y0 + r;
                const uint32_t blk = lane_base + k * S::kAccCols + (r + 2) * N;
                float acc[N];
#pragma unroll
                for (int j = 0; j < N / 16; ++j) tmem_ld16(blk + 16 * j, *reinterpret_cast<float(*)[16]>(&acc[16 * j]));
#pragma unroll
                for (int j = 0; j < N / 16; ++j) tmem_zero16(blk + 16 * j);
                if (yy >= H || xx >= W) continue;
                if (EPI == EPI_RELU || EPI == EPI_MASK) {
                    uint4 packed[N / 8];
                    uint32_t *pw = reinterpret_cast<uint32_t *>(packed);
                    if (EPI == EPI_MASK) {
#pragma unroll
                        for (int c8 = 0; c8 < N / 8; ++c8) {
                            const uint4 m4 =
                                *reinterpret_cast<const uint4 *>(mask + blk_off(b, c8, yy, xx, H, W, N / 8));
                            const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162 *>(&mw[h]);
                                const int c = 8 * c8 + 2 * h;
                                const float v0 = __bfloat162float(m2.x) > 0.f ? acc[c] : 0.f;
                                const float v1 = __bfloat162float(m2.y) > 0.f ? acc[c + 1] : 0.f;
                                const __nv_bfloat162 o = __floats2bfloat162_rn(v0, v1);
                                pw[c / 2] = *reinterpret_cast<const uint32_t *>(&o);
                            }
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < N; c += 2) {
                            const __nv_bfloat162 o = __floats2bfloat162_rn(fmaxf(acc[c] + bz[c], 0.f),
                                                                           fmaxf(acc[c + 1] + bz[c + 1], 0.f));
                            pw[c / 2] = *reinterpret_cast<const uint32_t *>(&o);
                        }
                    }
                    store_with_halo<N>(static_cast<bf16 *>(out), b, yy, xx, H, W, periodic, packed);
                } else if (EPI == EPI_F32) {
                    const int64_t pix = ((int64_t)b * H + yy) * W + xx;
                    float4 *o4 = reinterpret_cast<float4 *>(static_cast<float *>(out) + pix * COUTG);
#pragma unroll
                    for (int c = 0; c < COUTG; c += 4)
                        o4[c / 4] = make_float4(acc[c] + bz[c], acc[c + 1] + bz[c + 1],
                                                acc[c + 2] + bz[c + 2], acc[c + 3] + bz[c + 3]);
                } else {   // EPI_Z: z = D^-1 v + s y  (B = 1)
                    const int64_t HW = (int64_t)H * W, q = (int64_t)yy * W + xx;
                    const float v0 = (float)__ldcg(vz + q), v1 = (float)__ldcg(vz + HW + q),
                                v2 = (float)__ldcg(vz + 2 * HW + q);
                    const float *o = jd + q * 9, s = (float)s_out;
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        z[c * HW + q] =
                            (double)fmaf(s, acc[c] + bz[c], o[3 * c] * v0 + o[3 * c + 1] * v1 + o[3 * c + 2] * v2);
                }
            }
            // this set's output blocks are read and cleared: hand it back to the MMA thread
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(&accempty[k]);
        }
    }
    __syncthreads();
    if (tid == 0) {
        // drain before the barriers and buffers are reused: every copy issued
        // has landed and every MMA issued has completed (normally all consumed
        // already; after an abort these are the operations still in flight)
        const int nissued = *s_issued;
        for (int j = nloaded > kStages ? nloaded - kStages : 0; j < nloaded; ++j) {
            mbar_wait(&full[j % kStages], (j / kStages) & 1, kWaitLimit);
            if (j < nissued) mbar_wait(&empty[j % kStages], (j / kStages) & 1, kWaitLimit);
        }
        if (*abort && err) atomicExch(err, 1);
    }
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc<S::kTmemCols>(tm);
    }
    __syncthreads();     // shared memory (barriers included) is reused by the caller's next step
}

}  // namespace gxv
