// gx_netpipe.cuh -- the whole learned-preconditioner network (four 3x3
// convolutions, 16/32 -> 32 channels, ReLU, last layer adding s N(v / s) to
// the block-Jacobi image) as ONE persistent pipeline per CTA: the same
// tcgen05 convolution as gx_convtc.cuh (kernel rows folded into N = 96, A
// tiles addressed by moving descriptors, accumulators in tensor memory,
// bulk-copy tiles of channel-blocked halo images), but with the weights of all
// four layers resident in shared memory, the barriers and tensor memory set up
// once, and no grid barrier between layers.
//
// Every CTA walks the items (layer l, unit u) for l = 0..3 and its units u =
// cta, cta + ncta, ...  A tile of layer l >= 1 needs the layer l-1 outputs of
// its unit and of the 8 units around it (rows and columns wrap: periodic
// field), so before copying it the producer waits for their completion flags
// (ld.acquire, bounded); once a named barrier has ordered the epilogue's
// stores of a unit, a publisher warp fences them and releases the unit's flag
// (st.release), off the epilogue's path.  Waits only point to earlier layers, and
// every item of an earlier layer completes without outside help once it is
// loaded, so the walk cannot deadlock; all waits are bounded anyway, and an
// expired wait aborts the CTA's pipeline (the error flag is set, copies and
// MMAs in flight are drained, tensor memory is freed).
//
// The caller packs the layer-0 input, clears the CTA's flags and runs a grid
// barrier before the call (so that all flags start at zero and the input is
// complete), and another one after it (before z is read).
#pragma once

#include "gx_convtc.cuh"

namespace gxn {

using namespace gxv;

constexpr int kR = 4;                    // rows per unit
constexpr int kNB = 32;                  // output channels of one row block (all layers)
constexpr int kLayers = 4;
constexpr int kUnitRows = kR;

__host__ __device__ constexpr int layer_cin(int l) { return l == 0 ? 16 : 32; }
__host__ __device__ constexpr int wbytes(int l) { return 3 * (layer_cin(l) / 8) * 3 * kNB * 16; }
__host__ __device__ constexpr int woff(int l) { return l == 0 ? 0 : wbytes(0) + (l - 1) * wbytes(1); }
constexpr int kWTotal = woff(kLayers);
constexpr int kSlabBytes = (kR + 2) * kTileRow * 16;
constexpr int kTileBytes = 4 * kSlabBytes;                    // 32 channels (layer 0 uses half)
constexpr int kStagesP = 2;
constexpr int kTileOff = kWTotal;
constexpr int kBiasOff = kTileOff + kStagesP * kTileBytes;
constexpr int kBarOff = kBiasOff + kLayers * kNB * 4;
constexpr int kNumBars = 1 + 2 * kStagesP + 4;
constexpr int kMiscOff = kBarOff + 8 * kNumBars;
constexpr int kSmemBytes = kMiscOff + 16;
constexpr int kAccCols = (kR + 4) * kNB;                      // one accumulator set
constexpr int kTmemCols = 512;
static_assert(2 * kAccCols <= kTmemCols, "two accumulator sets");
constexpr int kFlagLimit = 1 << 20;                           // polls of a neighbour flag before giving up

struct PipeArgs {
    const bf16 *in[kLayers];     // layer inputs: x0 (16 ch), h1, h2, h3 (32 ch), blocked halo images
    bf16 *out[kLayers - 1];      // h1, h2, h3
    const bf16 *w[kLayers];      // weights packed [kx][cin/8][3 x 32][8]
    const float *bias[kLayers];  // [>= 3 or 32]: layers 0..2 have 32, layer 3 has 3 (then zero)
    const double *v;             // Krylov vector [3][H*W]
    const float *jd;             // FP32 block-Jacobi inverse [H*W][9]
    double *z;                   // output [3][H*W]
    float s;                     // output scale
    unsigned *flags;             // [3][units] completion flags of layers 0..2
    int *err;
    int H, W;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// generic-proxy global writes <-> asynchronous-proxy (bulk copy) reads
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// units of a H x W field (rows of kR image rows x 128 columns)
__host__ __device__ __forceinline__ int pipe_units(int H, int W) { return ((H + kR - 1) / kR) * ((W + kTW - 1) / kTW); }

// clear the completion flags of this CTA's units (before the grid barrier that precedes the pipeline)
__device__ __forceinline__ void pipe_clear_flags(unsigned *flags, int H, int W, int cta, int ncta) {
    const int nunits = pipe_units(H, W);
    for (int u = cta + ncta * (int)threadIdx.x; u < nunits; u += ncta * (int)blockDim.x)
        for (int l = 0; l < kLayers - 1; ++l) flags[l * nunits + u] = 0;
}

// one unit's MMAs of a layer with CIN input channels (fully unrolled: the
// tensor core then sees them back to back)
template <int CIN>
__device__ __forceinline__ void issue_unit(uint32_t dacc, uint64_t ad, uint64_t bd) {
    constexpr uint32_t idesc = gxt::idesc_bf16_f32(kTW, 3 * kNB);
    constexpr uint32_t kWSlab16 = 3 * kNB;                 // one 8-channel slab of W_kx, in 16-byte units
#pragma unroll
    for (int rho = 0; rho < kR + 2; ++rho)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx)
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc)
                gxt::mma_bf16(dacc + rho * kNB, ad + (uint32_t)(rho * kTileRow + kx + 2 * kc * (kSlabBytes / 16)),
                              bd + (uint32_t)((kx * (CIN / 8) + 2 * kc) * kWSlab16), idesc, true);
}

// unit of item t: layer l walks the CTA's units cta + i ncta for i = l, l + 1,
// ..., nmine - 1, 0, ..., l - 1.  On the periodic field any walk has a seam
// where its first units neighbour its last ones; starting each layer one unit
// further on puts the units that neighbour the previous layer's late units at
// the end of the layer, so a layer's first units depend only on units the
// previous layer finished early
__device__ __forceinline__ int item_unit(int t, int nmine, int cta, int ncta) {
    const int l = t / nmine, i = (t % nmine + l) % nmine;
    return cta + i * ncta;
}

// the four layers over this CTA's units (every thread of the CTA calls it;
// blockDim.x == 512: two epilogue groups of four warps, two rows each; sm:
// kSmemBytes bytes, 128-byte aligned)
static __device__ void net_pipeline(const PipeArgs &args, unsigned char *sm, int cta, int ncta) {
    using namespace gxt;
    // register copies of the arguments (the inline assembly clobbers memory)
    const int H = args.H, W = args.W;
    unsigned *const flags = args.flags;
    bf16 *const out0 = args.out[0], *const out1 = args.out[1], *const out2 = args.out[2];
    const bf16 *const in0 = args.in[0], *const in1 = args.in[1], *const in2 = args.in[2], *const in3 = args.in[3];
    const double *const vin = args.v;
    const float *const jd = args.jd;
    double *const zout = args.z;
    const float s_out = args.s;
    float *sBias = reinterpret_cast<float *>(sm + kBiasOff);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kBarOff);
    uint64_t *wfull = bars, *full = bars + 1, *empty = bars + 1 + kStagesP, *accfull = bars + 1 + 2 * kStagesP,
             *accempty = accfull + 2;
    uint32_t *sTm = reinterpret_cast<uint32_t *>(sm + kMiscOff);
    volatile int *abort = reinterpret_cast<volatile int *>(sm + kMiscOff + 4);
    volatile int *s_issued = reinterpret_cast<volatile int *>(sm + kMiscOff + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ngroups = blockDim.x >> 8, group = warp >> 3;

    const int nseg = (W + kTW - 1) / kTW, nblk = (H + kR - 1) / kR, nunits = nblk * nseg;
    if (cta >= nunits) return;
    if (ngroups != 2) {    // launch-configuration error: report it, touch nothing
        if (tid == 0 && args.err) atomicExch(args.err, 1);
        return;
    }
    const int nmine = (nunits - 1 - cta) / ncta + 1;
    const int nitems = kLayers * nmine;     // item t: layer t / nmine, unit cta + (t % nmine) ncta

    for (int i = tid; i < kLayers * kNB; i += blockDim.x) {
        const int l = i / kNB, c = i % kNB;
        const float *b = args.bias[l];
        sBias[i] = (b && c < (l == kLayers - 1 ? 3 : kNB)) ? b[c] : 0.f;
    }
    if (tid == 0) {
        for (int i = 0; i < kNumBars; ++i) mbar_init(&bars[i], i >= 1 + 2 * kStagesP + 2 ? 4 * 32 * ngroups : 1);
        *abort = 0;
        *s_issued = 0;
    }
    __syncwarp();
    if (warp == 0) tmem_alloc<kTmemCols>(sTm);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = *sTm;

    int nloaded = 0;    // (producer warp)
    if (warp == 0) {
        // ---- producer: all weights once, then the tiles; lane 0 waits, the lanes copy rows
        if (lane == 0) {
            mbar_arrive_expect_tx(wfull, kWTotal);
            for (int l = 0; l < kLayers; ++l) bulk_load(smem_addr(sm + woff(l)), args.w[l], wbytes(l), wfull);
        }
        int t = 0;
        for (; t < nitems; ++t) {
            const int l = t / nmine, u = item_unit(t, nmine, cta, ncta);
            const int st = t % kStagesP, n = t / kStagesP, cin = layer_cin(l);
            int b, y0, x0;
            unit_pos<kR>(u, nseg, nblk, b, y0, x0);
            const int rows = min(kR + 2, H + 2 - y0), npx = min(kTileRow, W + 2 - x0);
            int ok = 1;
            if (lane == 0 && n > 0) ok = mbar_wait_or_abort(&empty[st], (n - 1) & 1, kWaitLimit, abort);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (ok && l > 0) {
                // the 3 x 3 units around u must have finished layer l - 1: lanes 0..8 watch one each
                const int rb = y0 / kR, sg = x0 / kTW;
                const unsigned *fp = flags + (l - 1) * nunits +
                                     ((rb + lane / 3 - 1 + nblk) % nblk) * nseg + (sg + lane % 3 - 1 + nseg) % nseg;
                for (int polls = 0;; ++polls) {
                    const unsigned v = lane < 9 ? ld_acquire(fp) : 1u;
                    if (__all_sync(0xffffffffu, v != 0u)) break;
                    // give up together (a vote, so that the warp leaves the loop as one)
                    if (__any_sync(0xffffffffu, *abort != 0) || polls > kFlagLimit) {
                        if (lane == 0) *abort = 1;
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
                fence_proxy_async_global();
            }
            if (lane == 0 && ok) mbar_arrive_expect_tx(&full[st], (uint32_t)(rows * (cin / 8) * npx * 16));
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            if (lane < (cin / 8) * (kR + 2)) {
                const int r = lane % (kR + 2), g = lane / (kR + 2);
                if (r < rows)
                    bulk_load(smem_addr(sm + kTileOff + st * kTileBytes + g * kSlabBytes + r * kTileRow * 16),
                              (l == 0 ? in0 : l == 1 ? in1 : l == 2 ? in2 : in3) + blk_off(b, g, y0 - 1 + r, x0 - 1, H, W, cin / 8),
                              npx * 16, &full[st]);
            }
        }
        nloaded = t;
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            constexpr uint32_t kWSlab = 3 * kNB * 16;          // bytes of one 8-channel slab of W_kx
            bool ok = mbar_wait_or_abort(wfull, 0, kWaitLimit, abort);
            int t = 0;
            for (; ok && t < nitems; ++t) {
                const int l = t / nmine, st = t % kStagesP, n = t / kStagesP, k = t & 1, m = t >> 1;
                if (!mbar_wait_or_abort(&full[st], n & 1, kWaitLimit, abort)) break;
                if (!mbar_wait_or_abort(&accempty[k], m & 1, kWaitLimit, abort)) break;
                tc_fence_after();
                const uint64_t ad = sdesc(smem_addr(sm + kTileOff + st * kTileBytes), kSlabBytes, 128);
                const uint64_t bd = sdesc(smem_addr(sm + woff(l)), kWSlab, 128);
                if (l == 0)
                    issue_unit<16>(tm + k * kAccCols, ad, bd);
                else
                    issue_unit<32>(tm + k * kAccCols, ad, bd);
                mma_commit(&empty[st]);
                mma_commit(&accfull[k]);
            }
            *s_issued = t;
        }
    } else if (warp == 2) {
        // ---- publisher: once the epilogue has stored a unit of layers 0..2 (named
        // barrier: their stores are ordered before it), one gpu-scope fence and a
        // release store of the unit's completion flag
        const int nepi = 4 * 32 * ngroups;
        for (int t = 0; t < nitems; ++t) {
            const int l = t / nmine;
            if (l >= kLayers - 1) break;
            named_sync(1, nepi + 32);
            if (lane == 0 && !*abort) {
                __threadfence();
                fence_proxy_async_global();
                st_release(flags + l * nunits + item_unit(t, nmine, cta, ncta), 1u);
            }
            __syncwarp();
        }
    } else if ((warp & 7) >= 4) {
        // ---- epilogue: groups of four warps (TMEM lane quarters), alternate rows
        const int q4 = warp & 3;
        const int nepi = 4 * 32 * ngroups;
        const uint32_t lane_base = tm + ((uint32_t)(32 * q4) << 16);
#pragma unroll 1
        for (int k = 0; k < 2; ++k) {
            for (int r = group; r < kR; r += ngroups)
                for (int c = 0; c < kNB; c += 16) tmem_zero16(lane_base + k * kAccCols + (r + 2) * kNB + c);
            tmem_wait_st();
            tc_fence_before();
            mbar_arrive(&accempty[k]);
        }
        float bz[kNB];
        int lcur = -1;
        for (int t = 0; t < nitems; ++t) {
            const int l = t / nmine, u = item_unit(t, nmine, cta, ncta), k = t & 1, m = t >> 1;
            if (l != lcur) {
#pragma unroll
                for (int c = 0; c < kNB; ++c) bz[c] = sBias[l * kNB + c];
                lcur = l;
            }
            // lane 0 polls (returns at once after an abort); the warp reads tensor memory together
            int ok = 0;
            if (lane == 0) ok = mbar_wait_or_abort(&accfull[k], m & 1, kWaitLimit, abort);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (ok) {
                tc_fence_after();
                int b, y0, x0;
                unit_pos<kR>(u, nseg, nblk, b, y0, x0);
                const int xx = x0 + 32 * q4 + lane;
#pragma unroll 1
                for (int r = group; r < kR; r += 2) {
                    const int yy = y0 + r;
                    const uint32_t blk = lane_base + k * kAccCols + (r + 2) * kNB;
                    float acc[kNB];
                    tmem_ld16(blk, *reinterpret_cast<float(*)[16]>(&acc[0]));
                    tmem_ld16(blk + 16, *reinterpret_cast<float(*)[16]>(&acc[16]));
                    tmem_zero16(blk);
                    tmem_zero16(blk + 16);
                    if (yy >= H || xx >= W) continue;
                    if (l < kLayers - 1) {
                        uint4 packed[kNB / 8];
                        uint32_t *pw = reinterpret_cast<uint32_t *>(packed);
#pragma unroll
                        for (int c = 0; c < kNB; c += 2) {
                            const __nv_bfloat162 o = __floats2bfloat162_rn(fmaxf(acc[c] + bz[c], 0.f),
                                                                           fmaxf(acc[c + 1] + bz[c + 1], 0.f));
                            pw[c / 2] = *reinterpret_cast<const uint32_t *>(&o);
                        }
                        store_with_halo<kNB>(l == 0 ? out0 : (l == 1 ? out1 : out2), 0, yy, xx, H, W, 1, packed);
                    } else {   // z = D^-1 v + s y
                        const int64_t HW = (int64_t)H * W, q = (int64_t)yy * W + xx;
                        const float v0 = (float)__ldcg(vin + q), v1 = (float)__ldcg(vin + HW + q),
                                    v2 = (float)__ldcg(vin + 2 * HW + q);
                        const float *o = jd + q * 9;
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            zout[c * HW + q] = (double)fmaf(s_out, acc[c] + bz[c],
                                                            o[3 * c] * v0 + o[3 * c + 1] * v1 + o[3 * c + 2] * v2);
                    }
                }
                tmem_wait_st();
                tc_fence_before();
                mbar_arrive(&accempty[k]);
            }
            // hand the unit to the publisher (warp 2), which then fences and releases
            // it while the epilogue goes on (both sides synchronise at every item,
            // also after an abort, so the barrier's phases never mix)
            if (l < kLayers - 1) named_sync(1, nepi + 32);
        }
    }
    __syncthreads();
    if (tid == 0) {
        // drain before the barriers and buffers are reused (see gx_convtc.cuh)
        const int nissued = *s_issued;
        for (int j = nloaded > kStagesP ? nloaded - kStagesP : 0; j < nloaded; ++j) {
            mbar_wait(&full[j % kStagesP], (j / kStagesP) & 1, kWaitLimit);
            if (j < nissued) mbar_wait(&empty[j % kStagesP], (j / kStagesP) & 1, kWaitLimit);
        }
        if (*abort && args.err) atomicExch(args.err, 1);
    }
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc<kTmemCols>(tm);
    }
    __syncthreads();
}

}  // namespace gxn
