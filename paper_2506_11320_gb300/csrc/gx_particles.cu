// gx_particles.cu -- particle kernels of the GL-ECSIM hot path (2D).
//
// k_pd<true> (the fused push) does, for every particle of a species, in one
// pass over the cell bins:
//   1. the theta-implicit mover of Sec. 2.1 (Eq. 29-30 and the ECSIM update):
//      vbar = alpha (v^n + beta_s E^{n+theta}), v^{n+1} = 2 vbar - v^n,
//      x^{n+3/2} = x^{n+1/2} + dt v^{n+1}, alpha from B^n (Eq. 30);
//   2. the deposit of step n+1 for the particles that stay in their cell, with
//      alpha from B^{n+1}: charge, mass and momentum weights, the current
//      alpha (v - u_ref) and the mass-matrix sums alpha W_g W_g' (Eq. 33-35);
//   3. re-binning into the other copy of the particle arrays: a cell's stayers
//      fill its new bin from the bottom in order, particles that leave take
//      slots at the top of their new cell's bin (see bin_front / bin_back).
// k_pd<false> deposits without moving: the whole state (the deposit before
// the first step), or, right after the push, only the particles that arrived
// in each cell (the back segments of the new bins), added to the records the
// push wrote with fire-and-forget atomic adds (one add per record entry, so
// the sum is the same as adding the two records).
//
// Particle layout: one 32-byte slot per particle, two float4
// (ox, oy, vx, vy) and (vz, w, id bits, 0); cell c's bin is slots
// [c cap, (c+1) cap).  A staged chunk of a bin is one contiguous bulk copy, a
// particle that leaves its cell is one 32-byte sector written, and the
// stayers of a chunk go out as contiguous runs of whole lines.
//
// Work decomposition (GB300-first): a persistent grid, one CTA of 8 warps per
// SM; each warp is split into 4 groups of 8 lanes and a group owns one cell at
// a time (32 consecutive cells per CTA batch).  A cell's bin is streamed into
// shared memory in 64-particle chunks by the bulk-copy (TMA) engine, double
// buffered per group and signalled through mbarriers (bounded waits), so the
// next chunk's loads overlap the current chunk's arithmetic.  The mover and
// the stayer deposit run with no warp collectives; each lane accumulates its
// particles' 109 partial sums in registers and at the end of the cell the 8
// lanes are reduced through shared memory and the record is stored with plain
// stores.  The FP32 particle arithmetic stays on the CUDA cores: it is a
// scatter, not a dense contraction.
#include <cub/cub.cuh>

#include "gx_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kGroup = 8;                         // lanes per cell group
constexpr int kGroups = kThreads / kGroup;        // 32 cells per CTA batch
constexpr int kChunk = 64;                        // particles per staged chunk
constexpr int kPerLane = kChunk / kGroup;         // 8
constexpr int kScr = 56 * 33;                     // reduction scratch floats per warp
constexpr unsigned kFull = 0xffffffffu;
constexpr long long kSpinLimit = 1LL << 24;       // bounded mbarrier wait

struct P2 {
    int nx, ny;
    int64_t N;
    int cap;
    int nbatch;
    float dtdx, dtdy;
    float beta;                  // q dt / (2 m)
    float bc;                    // beta / c
    const float4 *in;            // current copy: 2 float4 per slot
    const int *cnt_in;
    float4 *out;                 // other copy
    int *cnt_out;
    const float4 *mE, *mB;       // mover: E^{n+theta}, B^n (node averaged)
    const float4 *dB, *dU;       // deposit: B for alpha, reference velocity u_ref
    float *rec;                  // [112][N] for this species
    DevFlags *flags;
    int arrivals;                // deposit only the back segments (the particles that arrived)
    int wall_ci;                 // x index of the last cell before a reflecting wall, or -1
};

// dynamic shared memory: mbarriers, staging [group][buffer][slot][2] float4,
// destination codes [group][slot], compaction maps [group][slot] (the slot of
// the t-th stayer), reduction scratch [warp][kScr]
// The per-group strides are padded (16 bytes, 4 bytes) so that the 4 groups of
// a warp, which touch the same slot positions of their own buffers, land on
// different shared-memory banks.
constexpr int kGroupBuf = 2 * kChunk * 2 + 1;     // float4 per group: 2 buffers of 64 slots + pad
constexpr int kCodeStride = kChunk + 1;
constexpr size_t kBarBytes = ((size_t)kGroups * 2 * sizeof(uint64_t) + 127) / 128 * 128;   // 2 mbarriers per group
constexpr size_t kBufBytes = (size_t)kGroups * kGroupBuf * sizeof(float4);
constexpr size_t kCodeBytes = (size_t)kGroups * kCodeStride * sizeof(int);
constexpr size_t kMapBytes = (size_t)kGroups * kChunk;
constexpr size_t kScrBytes = (size_t)(kThreads / 32) * kScr * sizeof(float);
// leaver counts per group and direction (8 neighbours)
constexpr size_t kDirBytes = (size_t)kGroups * 8 * sizeof(int);
size_t pd_smem_bytes() { return kBarBytes + kBufBytes + kCodeBytes + kMapBytes + kScrBytes + kDirBytes; }

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 1D bulk copy global -> shared (TMA engine), completion counted on an mbarrier
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// wait with an iteration limit; false if it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase) {
    for (long long it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

// one 32-byte particle slot written with a single 256-bit store (dst 32-byte aligned)
__device__ __forceinline__ void st_slot(float4 *dst, float4 a, float4 b) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(dst), "f"(a.x), "f"(a.y), "f"(a.z),
                 "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}

// ------------------------------------------------------------ deposit math
// alpha (Eq. 30) with b = beta B / c, row-major: alpha a = (a + a x b + (a.b) b)/(1 + b.b)
__device__ __forceinline__ void alpha_tensor(float bx, float by, float bz, float al[9]) {
    const float inv = __frcp_rn(1.0f + bx * bx + by * by + bz * bz);
    al[0] = (1.0f + bx * bx) * inv; al[1] = (bz + bx * by) * inv; al[2] = (bx * bz - by) * inv;
    al[3] = (by * bx - bz) * inv;   al[4] = (1.0f + by * by) * inv; al[5] = (bx + by * bz) * inv;
    al[6] = (by + bz * bx) * inv;   al[7] = (bz * by - bx) * inv; al[8] = (1.0f + bz * bz) * inv;
}

// The 109 partial sums of one lane, held as 55 register pairs so that the
// deposit can use the paired FP32 FMA (two rounded FMAs per instruction,
// bit-identical to two fmaf):
//   p[0..1]    RHO corner pairs (a0,a1), (a2,a3)
//   p[2..7]    MV  [component][corner pair]
//   p[8..13]   J   [component][corner pair]
//   p[14..49]  M   [pair class j][alpha entries (0,1) (2,3) (4,5) (6,7)]
//   p[50..54]  M   alpha entry 8 for pair classes (0,1) (2,3) (4,5) (6,7) (8,-)
struct RegAcc {
    float2 p[55];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < 55; ++k) p[k] = make_float2(0.f, 0.f);
    }
    // record entry k (Rec<2> layout); k is a compile-time constant after unrolling
    __device__ __forceinline__ float get(int k) const {
        int idx, comp;
        if (k < Rec<2>::MV) { idx = k >> 1; comp = k & 1; }
        else if (k < Rec<2>::J) { const int t = k - Rec<2>::MV, a = t / 3, c = t % 3; idx = 2 + 2 * c + (a >> 1); comp = a & 1; }
        else if (k < Rec<2>::M) { const int t = k - Rec<2>::J, a = t / 3, c = t % 3; idx = 8 + 2 * c + (a >> 1); comp = a & 1; }
        else if (k < Rec<2>::USED) {
            const int t = k - Rec<2>::M, j = t / 9, e = t % 9;
            if (e < 8) { idx = 14 + 4 * j + (e >> 1); comp = e & 1; }
            else { idx = 50 + (j >> 1); comp = j & 1; }
        } else {
            return 0.f;
        }
        return comp ? p[idx].y : p[idx].x;
    }
};

__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

// Deposit of one particle at cell-local offsets (x, y) with the corner values
// of B (for alpha) and u_ref: the partial sums of the record layout Rec<2>.
__device__ __forceinline__ void deposit_one(RegAcc &acc, float x, float y, float vx, float vy, float vz, float w,
                                            const float4 cB[4], const float4 cU[4], float bc) {
    const float wx0 = 1.0f - x, wx1 = x, wy0 = 1.0f - y, wy1 = y;
    const float W[4] = {wx0 * wy0, wx1 * wy0, wx0 * wy1, wx1 * wy1};
    float bx = 0.f, by = 0.f, bz = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        bx = fmaf(W[a], cB[a].x, bx); by = fmaf(W[a], cB[a].y, by); bz = fmaf(W[a], cB[a].z, bz);
        ux = fmaf(W[a], cU[a].x, ux); uy = fmaf(W[a], cU[a].y, uy); uz = fmaf(W[a], cU[a].z, uz);
    }
    float al[9];
    alpha_tensor(bc * bx, bc * by, bc * bz, al);
    const float dx_ = vx - ux, dy_ = vy - uy, dz_ = vz - uz;
    const float jx = w * (al[0] * dx_ + al[1] * dy_ + al[2] * dz_);
    const float jy = w * (al[3] * dx_ + al[4] * dy_ + al[5] * dz_);
    const float jz = w * (al[6] * dx_ + al[7] * dy_ + al[8] * dz_);
    const float wv[3] = {w * vx, w * vy, w * vz};
    const float jv[3] = {jx, jy, jz};
    const float2 W01 = make_float2(W[0], W[1]), W23 = make_float2(W[2], W[3]);
    acc.p[0] = __ffma2_rn(dup2(w), W01, acc.p[0]);
    acc.p[1] = __ffma2_rn(dup2(w), W23, acc.p[1]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc.p[2 + 2 * c] = __ffma2_rn(dup2(wv[c]), W01, acc.p[2 + 2 * c]);
        acc.p[3 + 2 * c] = __ffma2_rn(dup2(wv[c]), W23, acc.p[3 + 2 * c]);
        acc.p[8 + 2 * c] = __ffma2_rn(dup2(jv[c]), W01, acc.p[8 + 2 * c]);
        acc.p[9 + 2 * c] = __ffma2_rn(dup2(jv[c]), W23, acc.p[9 + 2 * c]);
    }
    const float X[3] = {w * wx0 * wx0, w * wx0 * wx1, w * wx1 * wx1};
    const float Y[3] = {wy0 * wy0, wy0 * wy1, wy1 * wy1};
    float pw[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) pw[j] = X[j % 3] * Y[j / 3];
    const float2 al2[4] = {make_float2(al[0], al[1]), make_float2(al[2], al[3]), make_float2(al[4], al[5]),
                           make_float2(al[6], al[7])};
#pragma unroll
    for (int j = 0; j < 9; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc.p[14 + 4 * j + q] = __ffma2_rn(dup2(pw[j]), al2[q], acc.p[14 + 4 * j + q]);
#pragma unroll
    for (int j = 0; j < 8; j += 2)
        acc.p[50 + j / 2] = __ffma2_rn(make_float2(pw[j], pw[j + 1]), dup2(al[8]), acc.p[50 + j / 2]);
    acc.p[54].x = fmaf(pw[8], al[8], acc.p[54].x);
}

// Sum the 8 lanes of every group of the warp through the warp's shared scratch
// (stride 33: conflict-free writes and column sums) and store the record of
// the group's cell (or add it, without reading it back, when `add`).
__device__ __forceinline__ void group_reduce_store(const RegAcc &acc, float *scr, int lane, int lig, int gshift,
                                                   float *dst, int64_t stride, bool active, bool add) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int k = 0; k < 56; ++k) scr[k * 33 + lane] = acc.get(h * 56 + k);
        __syncwarp();
        if (active) {
#pragma unroll
            for (int t = 0; t < 7; ++t) {
                const int k = lig * 7 + t;
                const float *c = scr + k * 33 + gshift;
                const float s = ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
                if (add) atomicAdd(dst + (size_t)(h * 56 + k) * stride, s);
                else dst[(size_t)(h * 56 + k) * stride] = s;
            }
        }
        __syncwarp();
    }
}

__device__ __forceinline__ void corner_nodes(int ci, int cj, int nx, int ny, int64_t nd[4]) {
    const int ip = ci + 1 == nx ? 0 : ci + 1, jp = cj + 1 == ny ? 0 : cj + 1;
    nd[0] = ci + (int64_t)nx * cj;
    nd[1] = ip + (int64_t)nx * cj;
    nd[2] = ci + (int64_t)nx * jp;
    nd[3] = ip + (int64_t)nx * jp;
}

// bottom slot of chunk ch of a bin whose front holds nf and back nb particles:
// front chunks are [64 ch, 64 ch + 64), back chunks count down from the top
__device__ __forceinline__ int chunk_base(int ch, int nf, int cap) {
    const int nchf = (nf + kChunk - 1) / kChunk;
    return ch < nchf ? ch * kChunk : cap - (ch - nchf + 1) * kChunk;
}
__device__ __forceinline__ int bin_chunks(int word) {
    return (bin_front(word) + kChunk - 1) / kChunk + (bin_back(word) + kChunk - 1) / kChunk;
}
// clamp a (possibly overflowed) count word to the capacity
__device__ __forceinline__ int clamp_word(int w, int cap) {
    int f = bin_front(w), b = bin_back(w);
    b = min(b, cap);
    f = min(f, cap - b);
    return f | (b << 16);
}
// the segments a pass visits: the whole bin, or only the arrivals (back)
__device__ __forceinline__ int seg_word(int w, int cap, int arrivals_only) {
    const int c = clamp_word(w, cap);
    return arrivals_only ? (int)((unsigned)c & 0xffff0000u) : c;
}

// ------------------------------------------------------------ open boundaries
// Philox4x64-10 (Salmon, Moraes, Dror and Shaw, SC 2011): ten rounds of
// (x0, x1, x2, x3) <- (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)),
// the key bumped by the Weyl constants between rounds.  The host-side test
// code implements the same generator, so both inject identical particles.
__device__ __forceinline__ void philox4x64(uint64_t k0, uint64_t k1, uint64_t x[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        const uint64_t hi0 = __umul64hi(M0, x[0]), lo0 = M0 * x[0];
        const uint64_t hi1 = __umul64hi(M1, x[2]), lo1 = M1 * x[2];
        const uint64_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
        x[0] = y0; x[1] = lo1; x[2] = y2; x[3] = lo0;
    }
}

// Particle k of cell `cell` in the draw of `step`: key (seed, species), counter
// (step, cell, k, 0); offsets in the cell from the top 24 bits of words 0 and 1,
// three normals by the Box-Muller transform of 24-bit uniforms of words 2 and 3;
// v = u + vth n.  Step 0 is the device-side initialisation, steps >= 1 the
// boundary refill after each push.
__device__ __forceinline__ void draw_particle(uint64_t seed, int species, uint64_t step, int64_t cell, int k, int ny,
                                              float ux, float uy, float uz, float vth, float &ox, float &oy,
                                              float &vx, float &vy, float &vz) {
    uint64_t x[4] = {step, (uint64_t)cell, (uint64_t)k, 0ull};
    philox4x64(seed, (uint64_t)species, x);
    const float s24 = 1.0f / 16777216.0f;
    ox = (float)(x[0] >> 40) * s24;
    oy = ny > 1 ? (float)(x[1] >> 40) * s24 : 0.f;
    const float u1 = (float)((x[2] >> 40) + 1) * s24, u2 = (float)((x[2] >> 16) & 0xffffffu) * s24;
    const float u3 = (float)((x[3] >> 40) + 1) * s24, u4 = (float)((x[3] >> 16) & 0xffffffu) * s24;
    const float ra = sqrtf(-2.f * logf(u1)), rb = sqrtf(-2.f * logf(u3));
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    vx = ux + vth * ra * cs;
    vy = uy + vth * ra * sn;
    vz = uz + vth * rb * cospif(2.f * u4);
}

// Device-side drifting Maxwellian species: ppc draws of step 0 in every cell,
// written straight into the cell's bin (one CTA per cell).
__global__ void k_maxwellian(int nx, int ny, int64_t N, int cap, int ppc, uint64_t seed, int species, float ux,
                             float uy, float uz, float vth, float w, int track, float4 *bins, int *cnt) {
    for (int64_t cell = blockIdx.x; cell < N; cell += gridDim.x) {
        for (int k = threadIdx.x; k < ppc; k += blockDim.x) {
            float ox, oy, vx, vy, vz;
            draw_particle(seed, species, 0ull, cell, k, ny, ux, uy, uz, vth, ox, oy, vx, vy, vz);
            const size_t o = (size_t)cell * cap + k;
            bins[2 * o] = make_float4(ox, oy, vx, vy);
            bins[2 * o + 1] = make_float4(vz, w, __int_as_float(track ? (int)(cell * ppc + k) : 0), 0.f);
        }
        if (threadIdx.x == 0) cnt[cell] = ppc;
    }
    (void)nx;
}

struct BcArgs {
    int nx, ny, G, cap;
    int64_t N;
    uint64_t seed, step;
    int species, track;
    float bc;                    // beta / c of the species (alpha)
    int nsides;                  // 2, or 1 with a reflecting wall on the high side (no refill there)
    int ppc[2];                  // per side (0: low x, 1: high x)
    float w[2], vth[2], u[2][3];
    float4 *bins;                // the current copy (after the push)
    int *cnt;
    float *rec;                  // [112][N] of the species
    const float4 *dB, *dU;       // node B^{n+1} and u_ref of the deposit
};

// One CTA per boundary cell: replace its particles by the side's fresh draws
// (key (seed, species), counter (step, cell, k, 0); offsets from the top 24
// bits of words 0 and 1, three normals by Box-Muller from 24-bit uniforms of
// words 2 and 3), deposit them with the push's deposit arithmetic and
// overwrite the cell's record and count.
__global__ void __launch_bounds__(128) k_bc_refill(BcArgs a) {
    __shared__ float red[4][Rec<2>::SIZE];
    const int t = blockIdx.x, G2c = a.nsides * a.G;
    const int j = t / G2c, r = t % G2c;
    const int side = r < a.G ? 0 : 1;
    const int i = r < a.G ? r : a.nx - G2c + r;
    const int64_t cell = (int64_t)j * a.nx + i;
    int64_t nd[4];
    corner_nodes(i, j, a.nx, a.ny, nd);
    float4 cB[4], cU[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) { cB[c] = a.dB[nd[c]]; cU[c] = a.dU[nd[c]]; }
    const int ppc = a.ppc[side];
    const float w = a.w[side], vth = a.vth[side];
    RegAcc acc;
    acc.zero();
    for (int k = threadIdx.x; k < ppc; k += blockDim.x) {
        float ox, oy, vx, vy, vz;
        draw_particle(a.seed, a.species, a.step, cell, k, a.ny, a.u[side][0], a.u[side][1], a.u[side][2], vth, ox, oy,
                      vx, vy, vz);
        const size_t o = (size_t)cell * a.cap + k;
        a.bins[2 * o] = make_float4(ox, oy, vx, vy);
        a.bins[2 * o + 1] = make_float4(vz, w, __int_as_float(a.track ? -1 : 0), 0.f);
        deposit_one(acc, ox, oy, vx, vy, vz, w, cB, cU, a.bc);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < Rec<2>::SIZE; ++k) {
        float v = acc.get(k);
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < Rec<2>::SIZE; k += blockDim.x)
        a.rec[(size_t)k * a.N + cell] = (red[0][k] + red[1][k]) + (red[2][k] + red[3][k]);
    if (threadIdx.x == 0) a.cnt[cell] = ppc;          // front segment only
}

// ------------------------------------------------------------ fused kernel
// WALL: the push reflects particles at the high-x face of cell x index
// p.wall_ci (a reflecting wall); a separate instantiation, so that the push
// without a wall compiles exactly as it would without the feature
template <bool PUSH, bool WALL = false>
__global__ void __launch_bounds__(kThreads, 1) k_pd(P2 p) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);                         // [groups][2]
    float4 *bufs = reinterpret_cast<float4 *>(smem + kBarBytes);                  // [groups][2][kChunk][2]
    int *codes = reinterpret_cast<int *>(smem + kBarBytes + kBufBytes);           // [groups][kChunk + 1]
    unsigned char *maps = smem + kBarBytes + kBufBytes + kCodeBytes;             // [groups][kChunk]
    float *scr_all = reinterpret_cast<float *>(smem + kBarBytes + kBufBytes + kCodeBytes + kMapBytes);  // [warps][kScr]
    int *dircnt = reinterpret_cast<int *>(smem + kBarBytes + kBufBytes + kCodeBytes + kMapBytes + kScrBytes);

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int g = tid / kGroup, lig = tid % kGroup;
    const int gshift = (lane / kGroup) * kGroup;
    float4 *mybuf = bufs + (size_t)g * kGroupBuf;
    int *mycode = codes + g * kCodeStride;
    unsigned char *mymap = maps + g * kChunk;
    uint64_t *mybar = bars + 2 * g;
    float *scr = scr_all + (size_t)warp * kScr;
    int *mydir = dircnt + g * 8;

    if (lig == 0) {
        mbar_init(&mybar[0], 1);
        mbar_init(&mybar[1], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();

    // producer state of this group (lane 0): next chunk to stream = chunk
    // `ich` of the cell of batch `ib`
    int ib = blockIdx.x, ich = 0, inch = -1, iword = 0;
    int issued = 0, cons = 0;
    auto find_next = [&]() -> bool {
        while (ib < p.nbatch) {
            if (inch < 0) {
                const int64_t cell = (int64_t)ib * kGroups + g;
                iword = cell < p.N ? seg_word(p.cnt_in[cell], p.cap, p.arrivals) : 0;
                inch = bin_chunks(iword);
            }
            if (ich < inch) return true;
            ib += gridDim.x;
            ich = 0;
            inch = -1;
        }
        return false;
    };
    // stream chunk `ich` of the cell: only the slots of its own segment (whole
    // 32-byte slots are 16-byte aligned), into the same positions of the
    // staging buffer
    auto issue = [&]() {
        const int slot = issued & 1;
        const int64_t cell = (int64_t)ib * kGroups + g;
        const int fr = bin_front(iword), sbase = chunk_base(ich, fr, p.cap);
        int lo = 0, hi = kChunk;
        if (ich < (fr + kChunk - 1) / kChunk) hi = min(kChunk, fr - sbase);
        else lo = max(0, p.cap - bin_back(iword) - sbase);
        const uint32_t bytes = (uint32_t)((hi - lo) * 2 * sizeof(float4));
        const float4 *src = p.in + 2 * ((size_t)cell * p.cap + sbase + lo);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&mybar[slot], bytes);
        bulk_g2s(mybuf + (size_t)(slot * kChunk + lo) * 2, src, bytes, &mybar[slot]);
        ++issued;
        ++ich;
    };
    if (lig == 0) {
        if (find_next()) issue();
        if (find_next()) issue();
    }

    bool abort = false;
    for (int b = blockIdx.x; b < p.nbatch; b += gridDim.x) {
        const int64_t cell = (int64_t)b * kGroups + g;
        const bool valid = cell < p.N;
        const int word = valid ? seg_word(p.cnt_in[cell], p.cap, p.arrivals) : 0;
        const int nch = bin_chunks(word);
        const int nchf = (bin_front(word) + kChunk - 1) / kChunk;
        const int wmax = __reduce_max_sync(kFull, nch);
        const int ci = valid ? (int)(cell % p.nx) : 0, cj = valid ? (int)(cell / p.nx) : 0;
        const bool wallc = WALL && PUSH && ci == p.wall_ci;      // the wall is this cell's high-x face
        int64_t nd[4];
        corner_nodes(ci, cj, p.nx, p.ny, nd);
        float4 cB[4], cU[4], mE[4], mB[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            cB[a] = __ldg(p.dB + nd[a]);
            cU[a] = __ldg(p.dU + nd[a]);
            if (PUSH) { mE[a] = __ldg(p.mE + nd[a]); mB[a] = __ldg(p.mB + nd[a]); }
        }
        RegAcc acc;
        acc.zero();
        int fbase = 0;                      // stayers written to this cell's new bin so far

        for (int ch = 0; ch < wmax; ++ch) {
            const bool has = ch < nch;
            const int slot = cons & 1;
            bool ok = true;
            if (has) ok = mbar_wait_bounded(&mybar[slot], (uint32_t)((cons >> 1) & 1));
            if (__any_sync(kFull, !ok)) { abort = true; break; }
            float4 *cbuf = mybuf + (size_t)slot * kChunk * 2;
            const int sbase = has ? chunk_base(ch, bin_front(word), p.cap) : 0;
            // particles of this chunk: slots of its own segment only
            unsigned long long vmask = 0ull;
            if (has) {
                const int lo = ch < nchf ? 0 : max(0, p.cap - bin_back(word) - sbase);
                const int hi = ch < nchf ? min(kChunk, bin_front(word) - sbase) : kChunk;
                if (hi > lo) vmask = (hi - lo == 64 ? ~0ull : ((1ull << (hi - lo)) - 1ull)) << lo;
            }
            unsigned long long smask = vmask;   // stayers (all of them without the push)
            int old[kPerLane];                  // ranks of this lane's leavers within their (group, neighbour)
            int ddest = 0, dbase = 0;           // lane d: neighbour d's cell and its count word before the run
            if (PUSH) {
                // ---- A1: mover.  New state written back into the staged chunk,
                // the destination cell of each leaver into the code row.
                unsigned long long lv = 0ull;
#pragma unroll 2
                for (int k = 0; k < kPerLane; ++k) {
                    const int j = k * kGroup + lig;
                    bool leave = false;
                    if ((vmask >> j) & 1ull) {
                        const float4 s0 = cbuf[2 * j];
                        float x = s0.x, y = s0.y, vx = s0.z, vy = s0.w;
                        float vz = reinterpret_cast<const float *>(cbuf + 2 * j + 1)[0];
                        const float wx0 = 1.f - x, wy0 = 1.f - y;
                        const float W0 = wx0 * wy0, W1 = x * wy0, W2 = wx0 * y, W3 = x * y;
                        const float ex = W0 * mE[0].x + W1 * mE[1].x + W2 * mE[2].x + W3 * mE[3].x;
                        const float ey = W0 * mE[0].y + W1 * mE[1].y + W2 * mE[2].y + W3 * mE[3].y;
                        const float ez = W0 * mE[0].z + W1 * mE[1].z + W2 * mE[2].z + W3 * mE[3].z;
                        const float bx = p.bc * (W0 * mB[0].x + W1 * mB[1].x + W2 * mB[2].x + W3 * mB[3].x);
                        const float by = p.bc * (W0 * mB[0].y + W1 * mB[1].y + W2 * mB[2].y + W3 * mB[3].y);
                        const float bz = p.bc * (W0 * mB[0].z + W1 * mB[1].z + W2 * mB[2].z + W3 * mB[3].z);
                        // a = v + beta E ; vbar = (a + a x b + (a.b) b) / (1 + b.b)
                        const float ax = fmaf(p.beta, ex, vx), ay = fmaf(p.beta, ey, vy), az = fmaf(p.beta, ez, vz);
                        const float inv = __frcp_rn(1.0f + bx * bx + by * by + bz * bz);
                        const float ab = ax * bx + ay * by + az * bz;
                        const float vbx = (ax + (ay * bz - az * by) + ab * bx) * inv;
                        const float vby = (ay + (az * bx - ax * bz) + ab * by) * inv;
                        const float vbz = (az + (ax * by - ay * bx) + ab * bz) * inv;
                        vx = 2.f * vbx - vx; vy = 2.f * vby - vy; vz = 2.f * vbz - vz;
                        x = fmaf(vx, p.dtdx, x);
                        if (WALL && wallc && x >= 1.f) { x = 2.f - x; vx = -vx; }   // specular reflection
                        y = fmaf(vy, p.dtdy, y);
                        float fx = floorf(x), fy = floorf(y);
                        x -= fx; y -= fy;
                        if (x >= 1.f) { x -= 1.f; fx += 1.f; }
                        if (y >= 1.f) { y -= 1.f; fy += 1.f; }
                        int sx = (int)fx, sy = (int)fy;
                        if (sx < -1 || sx > 1 || sy < -1 || sy > 1) {
                            atomicExch(&p.flags->cfl, 1);
                            sx = max(-1, min(1, sx)); sy = max(-1, min(1, sy));
                        }
                        if (p.ny == 1) { sy = 0; y = 0.f; }
                        leave = sx != 0 || sy != 0;
                        const int code = (sx + 1) + 3 * (sy + 1);          // 4 = stays
                        cbuf[2 * j] = make_float4(x, y, vx, vy);
                        reinterpret_cast<float *>(cbuf + 2 * j + 1)[0] = vz;
                        mycode[j] = code < 4 ? code : code - 1;            // neighbour 0..7
                    }
                    if (leave) lv |= 1ull << j;
                }
                // gather the group's leaver bits (each lane knows its own slots)
                unsigned long long all = lv;
#pragma unroll
                for (int o = 1; o < kGroup; o <<= 1) all |= __shfl_xor_sync(kFull, all, o);
                smask = vmask & ~all;
                __syncwarp();
                // ---- B1: reserve the leavers' slots at the top of their new
                // bins: each leaver takes a rank within its (group, neighbour)
                // from a shared-memory counter, then lane d reserves the whole
                // run of neighbour d with one global atomic (results used only
                // after the deposit)
                mydir[lig] = 0;
                __syncwarp();
#pragma unroll
                for (int k = 0; k < kPerLane; ++k) {
                    const int j = k * kGroup + lig;
                    old[k] = (lv >> j) & 1ull ? atomicAdd(&mydir[mycode[j]], 1) : 0;
                }
                __syncwarp();
                {
                    const int cntd = mydir[lig];
                    const int code = lig < 4 ? lig : lig + 1;
                    int dxg = ci + code % 3 - 1, dyg = cj + code / 3 - 1;
                    dxg = dxg < 0 ? dxg + p.nx : (dxg >= p.nx ? dxg - p.nx : dxg);
                    dyg = dyg < 0 ? dyg + p.ny : (dyg >= p.ny ? dyg - p.ny : dyg);
                    ddest = dxg + p.nx * dyg;
                    dbase = cntd > 0 ? atomicAdd(&p.cnt_out[ddest], cntd << 16) : 0;
                }
            }
            // ---- A2: deposit of the stayers (compacted, no idle lanes).  With
            // the push the stayers are scattered over the chunk: each lane
            // enters its own slots in the group's compaction map first.
            const int ns = __popcll(smask);
            const int vlo = vmask ? __ffsll((long long)vmask) - 1 : 0;
            if (PUSH) {
#pragma unroll
                for (int k = 0; k < kPerLane; ++k) {
                    const int j = k * kGroup + lig;
                    if ((smask >> j) & 1ull) mymap[__popcll(smask & ((1ull << j) - 1ull))] = (unsigned char)j;
                }
                __syncwarp();
            }
            for (int t = lig; t < ns; t += kGroup) {
                const int j = PUSH ? (int)mymap[t] : vlo + t;
                const float4 s0 = cbuf[2 * j];
                const float2 s1 = reinterpret_cast<const float2 *>(cbuf + 2 * j + 1)[0];
                deposit_one(acc, s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, cB, cU, p.bc);
            }
            // ---- B2: write the chunk into the other copy
            if (PUSH) {
                // stayers: bottom of this cell's new bin, in order.  The warp
                // writes one group's run at a time, 16 slots (512 contiguous
                // bytes) per store instruction.
                const int boff = (int)(cbuf - bufs);
                const int moff = (int)(mymap - maps);
#pragma unroll
                for (int gi = 0; gi < 4; ++gi) {
                    const int src = gi * kGroup;
                    const int ns_g = __shfl_sync(kFull, ns, src);
                    if (ns_g == 0) continue;
                    const int base_g = __shfl_sync(kFull, fbase, src);
                    const long long cell_g = __shfl_sync(kFull, (long long)cell, src);
                    const float4 *gbuf = bufs + __shfl_sync(kFull, boff, src);
                    const unsigned char *gmap = maps + __shfl_sync(kFull, moff, src);
                    float4 *dst = p.out + 2 * ((size_t)cell_g * p.cap + base_g);
                    // 32 slots (1 KB contiguous) per round, one 256-bit store per lane
                    for (int r0 = 0; r0 < ns_g; r0 += 32) {
                        const int t = r0 + lane;
                        if (t < ns_g) {
                            const int j = gmap[t];
                            st_slot(dst + 2 * t, gbuf[2 * j], gbuf[2 * j + 1]);
                        }
                    }
                }
                // leavers: the slot reserved in B1 (one 32-byte sector each)
#pragma unroll
                for (int k = 0; k < kPerLane; ++k) {
                    const int j = k * kGroup + lig;
                    const bool lvj = ((vmask >> j) & 1ull) && !((smask >> j) & 1ull);
                    const int d = lvj ? mycode[j] : 0;
                    const int dest = __shfl_sync(kFull, ddest, gshift + d);
                    const int w0 = __shfl_sync(kFull, dbase, gshift + d);
                    if (lvj) {
                        const int back = bin_back(w0) + old[k];
                        if (back < p.cap) {
                            const size_t o = (size_t)dest * p.cap + p.cap - 1 - back;
                            st_slot(p.out + 2 * o, cbuf[2 * j], cbuf[2 * j + 1]);
                        } else {
                            atomicExch(&p.flags->overflow, 1);
                        }
                    }
                }
                fbase += ns;
            }
            __syncwarp();
            if (has) {
                ++cons;
                if (lig == 0 && find_next()) issue();       // refill the buffer just consumed
            }
        }
        if (abort) break;
        // the stayers' count (the bottom segment) of this cell's new bin
        if (PUSH && valid && lig == 0 && fbase > 0) atomicAdd(&p.cnt_out[cell], fbase);
        group_reduce_store(acc, scr, lane, lig, gshift, p.rec + cell, p.N, valid && (!p.arrivals || nch > 0),
                           p.arrivals != 0);
    }
    if (abort) {
        if (lane == 0) atomicExch(&p.flags->timeout, 1);
        // drain this group's copies still in flight before the CTA exits
        if (lig == 0)
            for (int k = cons; k < issued; ++k) mbar_wait_bounded(&mybar[k & 1], (uint32_t)((k >> 1) & 1));
    }
}

// largest bin count after a push; a bin whose two segments met has lost
// particles (stayers and arrivals wrote over each other)
__global__ void k_max_count(const int *cnt, int64_t n, int cap, DevFlags *f) {
    int m = 0;
    bool over = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = bin_count(cnt[i]);
        m = max(m, c);
        over |= cap > 0 && c > cap;
    }
    m = __reduce_max_sync(kFull, m);
    if ((threadIdx.x & 31) == 0) atomicMax(&f->maxcount, m);
    if (over) atomicExch(&f->overflow, 1);
}

__global__ void k_counts(const int *cnt, int64_t n, int cap, int *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = bin_count(clamp_word(cnt[i], cap));
}

// ---------------------------------------------------------------- binning
// cell and in-cell offsets of every particle; positions scaled by the inverse
// cell widths (no FP64 division or fmod: both run on the slow FP64 pipe), the
// cell index wrapped in integers (positions within +-2^31 cells)
__global__ void k_locate(int64_t n, const double *x, const double *y, int nx, int ny, double idx, double idy,
                         int *cell, float *ox, float *oy, int *count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double sx = x[i] * idx, sy = (ny > 1) ? y[i] * idy : 0.0;
        double fx = floor(sx), fy = floor(sy);
        double rx = sx - fx, ry = sy - fy;
        const long long lx = (long long)fx, ly = (long long)fy;
        int cx = (lx >= 0 && lx < nx) ? (int)lx : (int)(((lx % nx) + nx) % nx);   // inside the box: no division
        int cy = ny == 1 ? 0 : ((ly >= 0 && ly < ny) ? (int)ly : (int)(((ly % ny) + ny) % ny));
        float fxo = (float)rx, fyo = (float)ry;
        if (fxo >= 1.f) { fxo = 0.f; cx = wrap_idx(cx + 1, nx); }
        if (fyo >= 1.f) { fyo = 0.f; cy = wrap_idx(cy + 1, ny); }
        if (ny == 1) fyo = 0.f;
        const int c = cx + nx * cy;
        cell[i] = c;
        ox[i] = fxo;
        oy[i] = fyo;
        atomicAdd(&count[c], 1);
    }
}

__global__ void k_scatter(int64_t n, const int *cell, const float *ox, const float *oy, const float *vx,
                          const float *vy, const float *vz, const float *w, const int32_t *id, int cap,
                          int *cursor, float4 *out, int track, DevFlags *f) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = cell[i];
        const int slot = atomicAdd(&cursor[c], 1);
        if (slot >= cap) { atomicExch(&f->overflow, 1); continue; }
        const size_t o = (size_t)c * cap + slot;
        const int idv = track ? (id ? id[i] : (int32_t)i) : 0;
        out[2 * o] = make_float4(ox[i], oy[i], vx[i], vy[i]);
        out[2 * o + 1] = make_float4(vz[i], w[i], __int_as_float(idv), 0.f);
    }
}

// copy bins into bins of a new capacity (both segments into the new front)
__global__ void k_rebin_copy(int64_t ncell, int oldcap, int newcap, const int *cnt, int *newcnt, const float4 *src,
                             float4 *dst) {
    const int64_t c = blockIdx.x;
    if (c >= ncell) return;
    const int word = clamp_word(cnt[c], oldcap);
    const int m = min(bin_count(word), newcap);
    for (int i = threadIdx.x; i < 2 * m; i += blockDim.x) {
        const size_t s = (size_t)c * oldcap + bin_slot(word, i >> 1, oldcap);
        dst[2 * ((size_t)c * newcap + (i >> 1)) + (i & 1)] = src[2 * s + (i & 1)];
    }
    if (threadIdx.x == 0) newcnt[c] = m;
}

__global__ void k_gather_out(int64_t ncell, int cap, const int *cnt, const int *offs, const float4 *src, int nx,
                             int ny, double dx, double dy, double *x, double *y, double *z, float *vx, float *vy,
                             float *vz, float *w, int32_t *id) {
    const int64_t c = blockIdx.x;
    if (c >= ncell) return;
    const int word = clamp_word(cnt[c], cap);
    const int m = bin_count(word);
    const int cx = (int)(c % nx), cy = (int)(c / nx);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const size_t s = (size_t)c * cap + bin_slot(word, i, cap);
        const float4 a = src[2 * s], b = src[2 * s + 1];
        const int o = offs[c] + i;
        if (x) x[o] = (cx + (double)a.x) * dx;
        if (y) y[o] = ny > 1 ? (cy + (double)a.y) * dy : 0.0;
        if (z) z[o] = 0.0;
        if (vx) vx[o] = a.z;
        if (vy) vy[o] = a.w;
        if (vz) vz[o] = b.x;
        if (w) w[o] = b.y;
        if (id) id[o] = __float_as_int(b.z);
    }
}

int grid_for(int64_t n, int block = 256) {
    int64_t g = (n + block - 1) / block;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

int alloc_bins(gx_ctx *c, int s, int cap) {
    Species &S = c->sp[s];
    const size_t nslot = (size_t)c->N * cap;
    for (int b = 0; b < 2; ++b) {
        S.p[b] = nullptr;
        GX_CHECK(c, cudaMalloc(&S.p[b], nslot * 2 * sizeof(float4)));
        GX_CHECK(c, cudaMalloc(&S.cnt[b], c->N * sizeof(int)));
        GX_CHECK(c, cudaMemset(S.cnt[b], 0, c->N * sizeof(int)));
    }
    S.cap = cap;
    return GX_OK;
}

void free_bins(Species &S) {
    for (int b = 0; b < 2; ++b) {
        if (S.p[b]) cudaFree(S.p[b]);
        S.p[b] = nullptr;
        if (S.cnt[b]) cudaFree(S.cnt[b]);
        S.cnt[b] = nullptr;
    }
}

// bin capacity: a multiple of the 64-particle chunk (staged chunks stay inside
// their bin) and below 2^15 (the packed count word)
int round_cap(double v) {
    int cap = (int)ceil(v);
    cap = (cap + kChunk - 1) / kChunk * kChunk;
    return cap < kChunk ? kChunk : cap;
}

}  // namespace

// --------------------------------------------------------------- binning
int gx_bin_particles(gx_ctx *c, int s, int64_t n, const double *x, const double *y, const double *z,
                     const float *vx, const float *vy, const float *vz, const float *w, const int32_t *id,
                     cudaStream_t st) {
    (void)z;
    Species &S = c->sp[s];
    int *cell = nullptr, *count = nullptr;
    float *ox = nullptr, *oy = nullptr;
    GX_CHECK(c, cudaMalloc(&cell, (n + 1) * sizeof(int)));
    GX_CHECK(c, cudaMalloc(&ox, (n + 1) * sizeof(float)));
    GX_CHECK(c, cudaMalloc(&oy, (n + 1) * sizeof(float)));
    GX_CHECK(c, cudaMalloc(&count, c->N * sizeof(int)));
    GX_CHECK(c, cudaMemsetAsync(count, 0, c->N * sizeof(int), st));
    if (n > 0) {
        k_locate<<<grid_for(n), 256, 0, st>>>(n, x, y, c->n[0], c->n[1], 1.0 / c->cfg.dx[0], 1.0 / c->cfg.dx[1], cell, ox,
                                               oy, count);
        GX_LAUNCHED(c);
    }
    DevFlags *dmax = nullptr;
    GX_CHECK(c, cudaMalloc(&dmax, sizeof(DevFlags)));
    GX_CHECK(c, cudaMemsetAsync(dmax, 0, sizeof(DevFlags), st));
    k_max_count<<<grid_for(c->N), 256, 0, st>>>(count, c->N, 0, dmax);
    GX_LAUNCHED(c);
    DevFlags hf{};
    GX_CHECK(c, cudaMemcpyAsync(&hf, dmax, sizeof(DevFlags), cudaMemcpyDeviceToHost, st));
    GX_CHECK(c, cudaStreamSynchronize(st));
    const double slack = c->cfg.bin_slack > 1.2 ? c->cfg.bin_slack : 1.2;
    const int cap = round_cap(std::max(64.0, hf.maxcount * slack));
    GX_CHECK(c, cudaFree(dmax));
    if (cap >= 32768) { c->err = "more than 32767 particles per cell bin"; return GX_EINVAL; }
    int rc = alloc_bins(c, s, cap);
    if (rc) return rc;
    GX_CHECK(c, cudaMemsetAsync(S.cnt[c->cur], 0, c->N * sizeof(int), st));
    if (n > 0) {
        k_scatter<<<grid_for(n), 256, 0, st>>>(n, cell, ox, oy, vx, vy, vz, w, id, cap, S.cnt[c->cur], S.p[c->cur],
                                                c->cfg.track_ids, c->dflags);
        GX_LAUNCHED(c);
    }
    GX_CHECK(c, cudaStreamSynchronize(st));
    cudaFree(cell); cudaFree(ox); cudaFree(oy); cudaFree(count);
    return GX_OK;
}

int gx_species_maxwellian_init(gx_ctx *c, int s, int ppc, double n0, const double u[3], double vth,
                               cudaStream_t st) {
    const double slack = c->cfg.bin_slack > 1.2 ? c->cfg.bin_slack : 1.2;
    const int cap = round_cap(std::max(64.0, ppc * slack));
    if (cap >= 32768) { c->err = "more than 32767 particles per cell bin"; return GX_EINVAL; }
    int rc = alloc_bins(c, s, cap);
    if (rc) return rc;
    const double dV = c->cfg.dx[0] * c->cfg.dx[1] * c->cfg.dx[2];
    const unsigned grid = (unsigned)std::min<int64_t>(c->N, 152 * 64);
    k_maxwellian<<<grid, 128, 0, st>>>(c->n[0], c->n[1], c->N, cap, ppc, c->cfg.seed, s, (float)u[0], (float)u[1],
                                       (float)u[2], (float)vth, (float)(n0 * dV / ppc), c->cfg.track_ids,
                                       c->sp[s].p[c->cur], c->sp[s].cnt[c->cur]);
    GX_LAUNCHED(c);
    GX_CHECK(c, cudaStreamSynchronize(st));
    return GX_OK;
}

int gx_regrow_bins(gx_ctx *c, int s, int newcap, cudaStream_t st) {
    newcap = round_cap(newcap);
    if (newcap >= 32768) { c->err = "more than 32767 particles per cell bin"; return GX_EOVERFLOW; }
    Species &S = c->sp[s];
    Species old = S;
    int rc = alloc_bins(c, s, newcap);
    if (rc) return rc;
    k_rebin_copy<<<(unsigned)c->N, 128, 0, st>>>(c->N, old.cap, newcap, old.cnt[c->cur], S.cnt[c->cur],
                                                  old.p[c->cur], S.p[c->cur]);
    GX_LAUNCHED(c);
    GX_CHECK(c, cudaStreamSynchronize(st));
    free_bins(old);
    return GX_OK;
}

// ------------------------------------------------------------ hot path
static int launch_pd(gx_ctx *c, bool push, cudaStream_t st) {
    static bool configured = false;
    if (!configured) {
        GX_CHECK(c, cudaFuncSetAttribute(k_pd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pd_smem_bytes()));
        GX_CHECK(c, cudaFuncSetAttribute(k_pd<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pd_smem_bytes()));
        GX_CHECK(c, cudaFuncSetAttribute(k_pd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pd_smem_bytes()));
        configured = true;
    }
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int nbatch = (int)((c->N + kGroups - 1) / kGroups);
    const int grid = std::max(1, std::min(nbatch, nsm));
    const int nxt = 1 - c->cur;
    for (int s = 0; s < c->nspecies; ++s) {
        Species &S = c->sp[s];
        P2 p{};
        p.nx = c->n[0]; p.ny = c->n[1]; p.N = c->N;
        p.cap = S.cap;
        p.nbatch = nbatch;
        p.dtdx = (float)(c->cfg.dt / c->cfg.dx[0]);
        p.dtdy = (float)(c->cfg.dt / c->cfg.dx[1]);
        const double beta = S.q * c->cfg.dt / (2.0 * S.m);
        p.beta = (float)beta;
        p.bc = (float)(beta / c->cfg.c);
        p.in = S.p[c->cur];
        p.out = S.p[nxt];
        p.cnt_in = S.cnt[c->cur];
        p.cnt_out = S.cnt[nxt];
        p.rec = c->rec + (size_t)s * c->N * Rec<2>::SIZE;
        p.flags = c->dflags;
        p.wall_ci = (c->cfg.bc_cells > 0 && c->cfg.bc_wall) ? c->n[0] - c->cfg.bc_cells - 1 : -1;
        if (push) {
            p.mE = c->nE; p.mB = c->nB; p.dB = c->nBnext; p.dU = c->nUref;
            GX_CHECK(c, cudaMemsetAsync(S.cnt[nxt], 0, c->N * sizeof(int), st));
            cudaEvent_t e0 = gx_ev_get(c), e1 = gx_ev_get(c);
            GX_CHECK(c, cudaEventRecord(e0, st));
            if (p.wall_ci >= 0) k_pd<true, true><<<grid, kThreads, pd_smem_bytes(), st>>>(p);
            else k_pd<true><<<grid, kThreads, pd_smem_bytes(), st>>>(p);
            GX_LAUNCHED(c);
            GX_CHECK(c, cudaEventRecord(e1, st));
            gx_ev_push(c, GX_T_PDK, e0, e1);
            c->n_pdk++;
            // the particles that arrived in each cell: the same pipelined
            // deposit over the back segments of the new bins, added to the
            // records the push just wrote
            P2 q = p;
            q.arrivals = 1;
            q.in = p.out;
            q.cnt_in = p.cnt_out;
            q.mE = nullptr; q.mB = nullptr;
            k_pd<false><<<grid, kThreads, pd_smem_bytes(), st>>>(q);
            GX_LAUNCHED(c);
            if (c->cfg.bc_cells > 0) {
                // open boundaries: the boundary cells' particles are replaced
                BcArgs b{};
                b.nx = c->n[0]; b.ny = c->n[1]; b.G = c->cfg.bc_cells; b.cap = S.cap; b.N = c->N;
                b.seed = c->cfg.seed; b.step = (uint64_t)(c->npush + 1); b.species = s;
                b.track = c->cfg.track_ids;
                b.bc = p.bc;
                const double dV = c->cfg.dx[0] * c->cfg.dx[1] * c->cfg.dx[2];
                b.nsides = c->cfg.bc_wall ? 1 : 2;
                for (int sd = 0; sd < b.nsides; ++sd) {
                    const BcSource &src = c->bsrc[sd][s];
                    if (src.ppc < 1) { c->err = "open boundaries need gx_boundary_source for every species"; return GX_ESTATE; }
                    if (src.ppc > S.cap) { c->err = "boundary ppc above the bin capacity"; return GX_EOVERFLOW; }
                    b.ppc[sd] = src.ppc;
                    b.w[sd] = (float)(src.n * dV / src.ppc);
                    b.vth[sd] = (float)src.vth;
                    for (int d = 0; d < 3; ++d) b.u[sd][d] = (float)src.u[d];
                }
                b.bins = p.out; b.cnt = p.cnt_out; b.rec = p.rec; b.dB = p.dB; b.dU = p.dU;
                k_bc_refill<<<(unsigned)(b.nsides * b.G * b.ny), 128, 0, st>>>(b);
                GX_LAUNCHED(c);
            }
        } else {
            p.mE = nullptr; p.mB = nullptr; p.dB = c->nB; p.dU = c->nUref;
            k_pd<false><<<grid, kThreads, pd_smem_bytes(), st>>>(p);
            GX_LAUNCHED(c);
        }
    }
    if (push) {
        c->cur = nxt;
        c->npush++;
        GX_CHECK(c, cudaMemsetAsync(&c->dflags->maxcount, 0, sizeof(int), st));
        for (int s = 0; s < c->nspecies; ++s) {
            k_max_count<<<grid_for(c->N), 256, 0, st>>>(c->sp[s].cnt[c->cur], c->N, c->sp[s].cap, c->dflags);
            GX_LAUNCHED(c);
        }
    }
    return GX_OK;
}

int gx_run_deposit(gx_ctx *c, cudaStream_t st) { return launch_pd(c, false, st); }
int gx_run_push_deposit(gx_ctx *c, cudaStream_t st) { return launch_pd(c, true, st); }

int gx_particles_out(gx_ctx *c, int s, double *x, double *y, double *z, float *vx, float *vy, float *vz, float *w,
                     int32_t *id, cudaStream_t st) {
    Species &S = c->sp[s];
    int *offs = nullptr, *counts = nullptr;
    void *tmp = nullptr;
    size_t tmpb = 0;
    GX_CHECK(c, cudaMalloc(&offs, (c->N + 1) * sizeof(int)));
    GX_CHECK(c, cudaMalloc(&counts, (c->N + 1) * sizeof(int)));
    k_counts<<<grid_for(c->N), 256, 0, st>>>(S.cnt[c->cur], c->N, S.cap, counts);
    GX_LAUNCHED(c);
    cub::DeviceScan::ExclusiveSum(nullptr, tmpb, counts, offs, (int)c->N, st);
    GX_CHECK(c, cudaMalloc(&tmp, tmpb + 16));
    GX_CHECK(c, cub::DeviceScan::ExclusiveSum(tmp, tmpb, counts, offs, (int)c->N, st));
    k_gather_out<<<(unsigned)c->N, 128, 0, st>>>(c->N, S.cap, S.cnt[c->cur], offs, S.p[c->cur], c->n[0], c->n[1],
                                                  c->cfg.dx[0], c->cfg.dx[1], x, y, z, vx, vy, vz, w, id);
    GX_LAUNCHED(c);
    GX_CHECK(c, cudaStreamSynchronize(st));
    cudaFree(offs); cudaFree(counts); cudaFree(tmp);
    return GX_OK;
}

void gx_free_bins(gx_ctx *c) {
    for (int s = 0; s < c->nspecies; ++s) free_bins(c->sp[s]);
}
