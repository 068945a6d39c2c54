// gx_particles.cu -- particle kernels of the GL-ECSIM hot path (2D).
//
// The fused kernel k_push_deposit does, for every particle of a species, in one
// pass over the cell bins:
//   1. the theta-implicit mover of Sec. 2.1 (Eq. 29-30 and the ECSIM update):
//      vbar = alpha (v^n + beta_s E^{n+theta}), v^{n+1} = 2 vbar - v^n,
//      x^{n+3/2} = x^{n+1/2} + dt v^{n+1}, with alpha from B^n (Eq. 30);
//   2. re-binning: the particle is written to its new cell's bin in the other
//      copy of the particle arrays (slot reserved with one warp-aggregated
//      atomic per destination cell);
//   3. the deposit of step n+1 at the new position with alpha from B^{n+1}:
//      charge, mass and momentum weights, the current alpha (v - u_ref) and
//      the mass-matrix sums alpha W_g W_g' (Eq. 33-35).
// k_deposit is the same kernel without steps 1-2 (moments of the current state).
//
// Work decomposition (GB300-first): one CTA per tile of TX x TY cells, 8 warps,
// each warp split into 4 groups of 8 lanes; a group owns one cell at a time.
// Particles are processed in chunks of 64 per group: the mover pass keeps 8
// particles per lane in flight (coalesced 32-byte segments per group), writes
// the new state and stages it in shared memory, compacted into particles that
// stay in the cell and particles that leave it.  Stayers are accumulated in
// per-lane registers (109 partial sums), reduced across the group through
// shared memory and added to the cell's record; leavers (about a tenth) add
// their contributions with shared-memory atomics to the record of their new
// cell, which may be in the one-cell ring around the tile.  At the end the tile
// records are stored to global memory (ring records to a per-tile buffer that a
// small kernel folds into the neighbours).  The FP32 particle arithmetic stays on
// the CUDA cores: it is a scatter, not a dense contraction.
#include <cub/cub.cuh>

#include "gx_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kGroup = 8;                         // lanes per cell group
constexpr int kGroups = kThreads / kGroup;        // 32 groups per CTA
constexpr int kPerLane = 8;                       // particles per lane per chunk
constexpr int kChunk = kGroup * kPerLane;         // 64 particles per group chunk
constexpr unsigned kFull = 0xffffffffu;

struct PDParams {
    int n[3];
    int T[3];
    int ntile[3];
    int LD[3];          // local cell dims incl. ring (T+2 on active axes)
    int NLD[3];         // local node dims (T+3 on active axes)
    int local;          // local cells incl. ring
    int ring;
    int cap;
    float dtdx[3];      // dt / dx per axis
    float beta;         // q dt / (2 m)
    float bc;           // beta / c
    int track;
    // particle bins
    const float *in[PF_COUNT];
    const int *cnt_in;
    float *out[PF_COUNT];
    int *cnt_out;
    // node fields (float4 per node)
    const float4 *mE, *mB;       // mover: E^{n+theta}, B^n
    const float4 *dB, *dU;       // deposit: B for alpha, reference velocity
    // outputs
    float *rec;                  // [N][112] for this species
    float *ring_out;             // [ntiles][ring][112]
    const int *ring_slot;        // [local] -> ring slot or -1 (interior)
    DevFlags *flags;
};

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// alpha (Eq. 30) with b = beta B / c, row-major: alpha a = (a + a x b + (a.b) b)/(1 + b.b)
__device__ __forceinline__ void alpha_tensor(float bx, float by, float bz, float al[9]) {
    float inv = 1.0f / (1.0f + bx * bx + by * by + bz * bz);
    al[0] = (1.0f + bx * bx) * inv; al[1] = (bz + bx * by) * inv; al[2] = (bx * bz - by) * inv;
    al[3] = (by * bx - bz) * inv;   al[4] = (1.0f + by * by) * inv; al[5] = (bx + by * bz) * inv;
    al[6] = (by + bz * bx) * inv;   al[7] = (bz * by - bx) * inv; al[8] = (1.0f + bz * bz) * inv;
}

struct RegAcc {
    float v[Rec<2>::SIZE];
    __device__ __forceinline__ void add(int k, float x) { v[k] += x; }
};
struct SmemAcc {
    float *base;
    __device__ __forceinline__ void add(int k, float x) { atomicAdd(base + k, x); }
};

// Deposit of one particle at cell-local offsets (x, y): weights of the four
// corners, B and u_ref interpolated from the corner values, alpha, then the
// partial sums of the record layout Rec<2>.
template <class A>
__device__ __forceinline__ void deposit_one(A &acc, float x, float y, float vx, float vy, float vz, float w,
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
    const float wvx = w * vx, wvy = w * vy, wvz = w * vz;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        acc.add(Rec<2>::RHO + a, w * W[a]);
        acc.add(Rec<2>::MV + 3 * a + 0, wvx * W[a]);
        acc.add(Rec<2>::MV + 3 * a + 1, wvy * W[a]);
        acc.add(Rec<2>::MV + 3 * a + 2, wvz * W[a]);
        acc.add(Rec<2>::J + 3 * a + 0, jx * W[a]);
        acc.add(Rec<2>::J + 3 * a + 1, jy * W[a]);
        acc.add(Rec<2>::J + 3 * a + 2, jz * W[a]);
    }
    const float X[3] = {w * wx0 * wx0, w * wx0 * wx1, w * wx1 * wx1};
    const float Y[3] = {wy0 * wy0, wy0 * wy1, wy1 * wy1};
#pragma unroll
    for (int jy_ = 0; jy_ < 3; ++jy_)
#pragma unroll
        for (int jx_ = 0; jx_ < 3; ++jx_) {
            const float pw = X[jx_] * Y[jy_];
#pragma unroll
            for (int e = 0; e < 9; ++e) acc.add(Rec<2>::M + 9 * (jx_ + 3 * jy_) + e, pw * al[e]);
        }
}

__device__ __forceinline__ int node_local(const PDParams &p, int lx, int ly) {
    return (lx + 1) + p.NLD[0] * (ly + 1);
}
__device__ __forceinline__ int cell_local(const PDParams &p, int lx, int ly) {
    return (lx + 1) + p.LD[0] * (ly + 1);
}

template <bool PUSH>
__global__ void __launch_bounds__(kThreads, 1) k_push_deposit(PDParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int NL = p.NLD[0] * p.NLD[1];
    float4 *sE = reinterpret_cast<float4 *>(smem);          // mover E^{n+theta}
    float4 *sB = sE + NL;                                    // mover B^n
    float4 *sDB = sB + NL;                                   // deposit B
    float4 *sDU = sDB + NL;                                  // deposit u_ref
    float *sRec = reinterpret_cast<float *>(sDU + NL);       // [local][112]
    float4 *sStage = reinterpret_cast<float4 *>(sRec + (size_t)p.local * Rec<2>::SIZE);  // [groups][64][2]

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int grp = tid / kGroup, lig = tid % kGroup;        // group and lane in group
    const int gshift = (lane / kGroup) * kGroup;             // first lane of my group in the warp
    const int tile = blockIdx.x;
    const int tx = tile % p.ntile[0], ty = tile / p.ntile[0];
    const int x0 = tx * p.T[0], y0 = ty * p.T[1];

    // stage node fields of the tile and its ring (+1 node) into shared memory
    for (int i = tid; i < NL; i += kThreads) {
        const int lx = i % p.NLD[0] - 1, ly = i / p.NLD[0] - 1;
        const int g = wrap_idx(x0 + lx, p.n[0]) + p.n[0] * wrap_idx(y0 + ly, p.n[1]);
        if (PUSH) { sE[i] = p.mE[g]; sB[i] = p.mB[g]; }
        sDB[i] = p.dB[g];
        sDU[i] = p.dU[g];
    }
    for (int i = tid; i < p.local * Rec<2>::SIZE; i += kThreads) sRec[i] = 0.f;
    __syncthreads();

    float4 *myStage = sStage + (size_t)grp * kChunk * 2;
    const int ncell_tile = p.T[0] * p.T[1];

    for (int c0 = 0; c0 < ncell_tile; c0 += kGroups) {
        const int lc = c0 + grp;
        const bool valid = lc < ncell_tile;
        const int lx = valid ? lc % p.T[0] : 0, ly = valid ? lc / p.T[0] : 0;
        const int gcell = (x0 + lx) + p.n[0] * (y0 + ly);
        int cnt = valid ? min(p.cnt_in[gcell], p.cap) : 0;
        const int wmax = __reduce_max_sync(kFull, cnt);
        const size_t binbase = (size_t)gcell * p.cap;
        const int homeL = cell_local(p, lx, ly);
        // corner nodes of the home cell
        const int n00 = node_local(p, lx, ly), n10 = n00 + 1, n01 = n00 + p.NLD[0], n11 = n01 + 1;

        for (int start = 0; start < wmax; start += kChunk) {
            // ---------------- pass 1: load, move, re-bin, stage
            float px[kPerLane], py[kPerLane], pvx[kPerLane], pvy[kPerLane], pvz[kPerLane], pw[kPerLane];
            int pid[kPerLane];
#pragma unroll
            for (int k = 0; k < kPerLane; ++k) {
                const int i = start + k * kGroup + lig;
                if (i < cnt) {
                    const size_t s = binbase + i;
                    px[k] = p.in[PF_OX][s]; py[k] = p.in[PF_OY][s];
                    pvx[k] = p.in[PF_VX][s]; pvy[k] = p.in[PF_VY][s]; pvz[k] = p.in[PF_VZ][s];
                    pw[k] = p.in[PF_W][s];
                    pid[k] = p.track ? __float_as_int(p.in[PF_ID][s]) : 0;
                }
            }
            int nstay = 0, nleave = 0;       // group-uniform
#pragma unroll
            for (int k = 0; k < kPerLane; ++k) {
                const int i = start + k * kGroup + lig;
                const bool act = i < cnt;
                float x = 0.f, y = 0.f, vx = 0.f, vy = 0.f, vz = 0.f, w = 0.f;
                int sx = 0, sy = 0;
                if (act) {
                    x = px[k]; y = py[k]; vx = pvx[k]; vy = pvy[k]; vz = pvz[k]; w = pw[k];
                    if (PUSH) {
                        const float wx0 = 1.f - x, wy0 = 1.f - y;
                        const float W0 = wx0 * wy0, W1 = x * wy0, W2 = wx0 * y, W3 = x * y;
                        const float4 e0 = sE[n00], e1 = sE[n10], e2 = sE[n01], e3 = sE[n11];
                        const float4 b0 = sB[n00], b1 = sB[n10], b2 = sB[n01], b3 = sB[n11];
                        const float ex = W0 * e0.x + W1 * e1.x + W2 * e2.x + W3 * e3.x;
                        const float ey = W0 * e0.y + W1 * e1.y + W2 * e2.y + W3 * e3.y;
                        const float ez = W0 * e0.z + W1 * e1.z + W2 * e2.z + W3 * e3.z;
                        const float bx = p.bc * (W0 * b0.x + W1 * b1.x + W2 * b2.x + W3 * b3.x);
                        const float by = p.bc * (W0 * b0.y + W1 * b1.y + W2 * b2.y + W3 * b3.y);
                        const float bz = p.bc * (W0 * b0.z + W1 * b1.z + W2 * b2.z + W3 * b3.z);
                        // a = v + beta E ; vbar = (a + a x b + (a.b) b) / (1 + b.b)
                        const float ax = fmaf(p.beta, ex, vx), ay = fmaf(p.beta, ey, vy), az = fmaf(p.beta, ez, vz);
                        const float inv = 1.0f / (1.0f + bx * bx + by * by + bz * bz);
                        const float ab = ax * bx + ay * by + az * bz;
                        const float vbx = (ax + (ay * bz - az * by) + ab * bx) * inv;
                        const float vby = (ay + (az * bx - ax * bz) + ab * by) * inv;
                        const float vbz = (az + (ax * by - ay * bx) + ab * bz) * inv;
                        vx = 2.f * vbx - vx; vy = 2.f * vby - vy; vz = 2.f * vbz - vz;
                        x = fmaf(vx, p.dtdx[0], x);
                        y = fmaf(vy, p.dtdx[1], y);
                        float fx = floorf(x), fy = floorf(y);
                        x -= fx; y -= fy;
                        if (x >= 1.f) { x -= 1.f; fx += 1.f; }
                        if (y >= 1.f) { y -= 1.f; fy += 1.f; }
                        sx = (int)fx; sy = (int)fy;
                        if (sx < -1 || sx > 1 || sy < -1 || sy > 1) {
                            atomicExch(&p.flags->cfl, 1);
                            sx = max(-1, min(1, sx)); sy = max(-1, min(1, sy));
                        }
                        if (p.n[1] == 1) { sy = 0; y = 0.f; }
                    }
                }
                // re-bin into the other copy: one atomic per destination cell per warp
                if (PUSH) {
                    const int dxg = wrap_idx(x0 + lx + sx, p.n[0]);
                    const int dyg = wrap_idx(y0 + ly + sy, p.n[1]);
                    const int dest = act ? dxg + p.n[0] * dyg : -1;
                    const unsigned peers = __match_any_sync(kFull, dest);
                    const int leader = __ffs(peers) - 1;
                    int base = 0;
                    if (act && lane == leader) base = atomicAdd(&p.cnt_out[dest], __popc(peers));
                    base = __shfl_sync(kFull, base, leader);
                    const int slot = base + __popc(peers & lanemask_lt());
                    if (act) {
                        if (slot < p.cap) {
                            const size_t o = (size_t)dest * p.cap + slot;
                            p.out[PF_OX][o] = x; p.out[PF_OY][o] = y;
                            p.out[PF_VX][o] = vx; p.out[PF_VY][o] = vy; p.out[PF_VZ][o] = vz;
                            p.out[PF_W][o] = w;
                            if (p.track) p.out[PF_ID][o] = __int_as_float(pid[k]);
                        } else {
                            atomicExch(&p.flags->overflow, 1);
                        }
                    }
                }
                // stage, compacted: stayers from the front, leavers from the back
                const bool stay = act && sx == 0 && sy == 0;
                const bool leave = act && !stay;
                const unsigned bs = (__ballot_sync(kFull, stay) >> gshift) & 0xffu;
                const unsigned bl = (__ballot_sync(kFull, leave) >> gshift) & 0xffu;
                const unsigned below = (1u << lig) - 1u;
                if (stay) {
                    const int pos = nstay + __popc(bs & below);
                    myStage[2 * pos] = make_float4(x, y, vx, vy);
                    myStage[2 * pos + 1] = make_float4(vz, w, 0.f, 0.f);
                } else if (leave) {
                    const int pos = kChunk - 1 - (nleave + __popc(bl & below));
                    myStage[2 * pos] = make_float4(x, y, vx, vy);
                    myStage[2 * pos + 1] = make_float4(vz, w, __int_as_float(cell_local(p, lx + sx, ly + sy)), 0.f);
                }
                nstay += __popc(bs);
                nleave += __popc(bl);
            }
            __syncwarp();

            // ---------------- pass 2: stayers, register accumulation
            RegAcc acc;
#pragma unroll
            for (int k = 0; k < Rec<2>::SIZE; ++k) acc.v[k] = 0.f;
            {
                const float4 cB[4] = {sDB[n00], sDB[n10], sDB[n01], sDB[n11]};
                const float4 cU[4] = {sDU[n00], sDU[n10], sDU[n01], sDU[n11]};
                const int smax = __reduce_max_sync(kFull, nstay);
                for (int j = lig; j < smax; j += kGroup) {
                    if (j < nstay) {
                        const float4 a = myStage[2 * j], b = myStage[2 * j + 1];
                        deposit_one(acc, a.x, a.y, a.z, a.w, b.x, b.y, cB, cU, p.bc);
                    }
                }
            }
            // ---------------- pass 3: leavers, shared-memory atomics into the
            // record of their new cell (interior or ring)
            if (PUSH) {
                const int lmax = __reduce_max_sync(kFull, nleave);
                for (int j = lig; j < lmax; j += kGroup) {
                    if (j < nleave) {
                        const float4 a = myStage[2 * (kChunk - 1 - j)], b = myStage[2 * (kChunk - 1 - j) + 1];
                        const int dl = __float_as_int(b.z);
                        const int dlx = dl % p.LD[0] - 1, dly = dl / p.LD[0] - 1;
                        const int m00 = node_local(p, dlx, dly), m10 = m00 + 1, m01 = m00 + p.NLD[0], m11 = m01 + 1;
                        const float4 cB[4] = {sDB[m00], sDB[m10], sDB[m01], sDB[m11]};
                        const float4 cU[4] = {sDU[m00], sDU[m10], sDU[m01], sDU[m11]};
                        SmemAcc sacc{sRec + (size_t)dl * Rec<2>::SIZE};
                        deposit_one(sacc, a.x, a.y, a.z, a.w, b.x, b.y, cB, cU, p.bc);
                    }
                }
            }
            __syncwarp();
            // ---------------- group reduction of the stayer sums through the
            // warp's (now free) stage buffer: two halves of 56 values; the
            // stride-33 layout keeps both the writes and the column sums free of
            // bank conflicts.
            if (__reduce_or_sync(kFull, nstay > 0 ? 1u : 0u) != 0u) {
                float *scratch = reinterpret_cast<float *>(sStage + (size_t)(warp * 4) * kChunk * 2);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
#pragma unroll
                    for (int k = 0; k < 56; ++k) scratch[k * 33 + lane] = acc.v[h * 56 + k];
                    __syncwarp();
                    if (nstay > 0) {
#pragma unroll
                        for (int t = 0; t < 7; ++t) {
                            const int k = lig * 7 + t;
                            float sum = 0.f;
#pragma unroll
                            for (int l = 0; l < kGroup; ++l) sum += scratch[k * 33 + gshift + l];
                            if (h * 56 + k < Rec<2>::USED) atomicAdd(&sRec[homeL * Rec<2>::SIZE + h * 56 + k], sum);
                        }
                    }
                    __syncwarp();
                }
            }
        }
    }
    __syncthreads();

    // store the tile records: interior cells to their global record, ring cells
    // to this tile's ring buffer
    const int nvec = Rec<2>::SIZE / 4;
    for (int i = tid; i < p.local * nvec; i += kThreads) {
        const int l = i / nvec, k = i % nvec;
        const float4 v = reinterpret_cast<const float4 *>(sRec)[i];
        const int rs = p.ring_slot[l];
        if (rs < 0) {
            const int lx = l % p.LD[0] - 1, ly = l / p.LD[0] - 1;
            const int g = (x0 + lx) + p.n[0] * (y0 + ly);
            reinterpret_cast<float4 *>(p.rec + (size_t)g * Rec<2>::SIZE)[k] = v;
        } else if (PUSH) {
            reinterpret_cast<float4 *>(p.ring_out + ((size_t)tile * p.ring + rs) * Rec<2>::SIZE)[k] = v;
        }
    }
}

// Fold ring buffers into the records of the cells they belong to.
__global__ void k_fold_rings(float *rec, const float *ring, const int *ring_lidx, int ring_n, int ntiles,
                             int ntx, int Tx, int Ty, int LDx, int nx, int ny) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= ntiles * ring_n) return;
    const int tile = warp / ring_n, rs = warp % ring_n;
    const int l = ring_lidx[rs];
    const int lx = l % LDx - 1, ly = l / LDx - 1;
    const int tx = tile % ntx, ty = tile / ntx;
    const int g = wrap_idx(tx * Tx + lx, nx) + nx * wrap_idx(ty * Ty + ly, ny);
    const float *src = ring + (size_t)warp * Rec<2>::SIZE;
    float *dst = rec + (size_t)g * Rec<2>::SIZE;
    for (int k = lane; k < Rec<2>::USED; k += 32) {
        const float v = src[k];
        if (v != 0.f) atomicAdd(dst + k, v);
    }
}

__global__ void k_max_count(const int *cnt, int64_t n, DevFlags *f) {
    int m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, cnt[i]);
    m = __reduce_max_sync(kFull, m);
    if ((threadIdx.x & 31) == 0) atomicMax(&f->maxcount, m);
}

// ---------------------------------------------------------------- binning
__global__ void k_locate(int64_t n, const double *x, const double *y, int nx, int ny, double dx, double dy,
                         int *cell, float *ox, float *oy, int *count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double sx = x[i] / dx, sy = (ny > 1) ? y[i] / dy : 0.0;
        double fx = floor(sx), fy = floor(sy);
        double rx = sx - fx, ry = sy - fy;
        int cx = wrap_idx((int)fmod(fx, (double)nx), nx);
        int cy = ny > 1 ? wrap_idx((int)fmod(fy, (double)ny), ny) : 0;
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
                          int *cursor, float *const *out, int track, DevFlags *f) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = cell[i];
        const int slot = atomicAdd(&cursor[c], 1);
        if (slot >= cap) { atomicExch(&f->overflow, 1); continue; }
        const size_t o = (size_t)c * cap + slot;
        out[PF_OX][o] = ox[i]; out[PF_OY][o] = oy[i];
        out[PF_VX][o] = vx[i]; out[PF_VY][o] = vy[i]; out[PF_VZ][o] = vz[i];
        out[PF_W][o] = w[i];
        if (track) out[PF_ID][o] = __int_as_float(id ? id[i] : (int32_t)i);
    }
}

// copy bins (old capacity) into bins of a new capacity
__global__ void k_rebin_copy(int64_t ncell, int oldcap, int newcap, const int *cnt, float *const *src,
                             float *const *dst, int nf) {
    const int64_t c = blockIdx.x;
    if (c >= ncell) return;
    const int m = min(cnt[c], min(oldcap, newcap));
    for (int f = 0; f < nf; ++f) {
        if (!src[f]) continue;
        for (int i = threadIdx.x; i < m; i += blockDim.x) dst[f][(size_t)c * newcap + i] = src[f][(size_t)c * oldcap + i];
    }
}

__global__ void k_gather_out(int64_t ncell, int cap, const int *cnt, const int *offs, float *const *src, int nx,
                             int ny, double dx, double dy, double *x, double *y, double *z, float *vx, float *vy,
                             float *vz, float *w, int32_t *id) {
    const int64_t c = blockIdx.x;
    if (c >= ncell) return;
    const int m = min(cnt[c], cap);
    const int cx = (int)(c % nx), cy = (int)(c / nx);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const size_t s = (size_t)c * cap + i;
        const int o = offs[c] + i;
        if (x) x[o] = (cx + (double)src[PF_OX][s]) * dx;
        if (y) y[o] = ny > 1 ? (cy + (double)src[PF_OY][s]) * dy : 0.0;
        if (z) z[o] = 0.0;
        if (vx) vx[o] = src[PF_VX][s];
        if (vy) vy[o] = src[PF_VY][s];
        if (vz) vz[o] = src[PF_VZ][s];
        if (w) w[o] = src[PF_W][s];
        if (id && src[PF_ID]) id[o] = __float_as_int(src[PF_ID][s]);
    }
}

int grid_for(int64_t n, int block = 256) {
    int64_t g = (n + block - 1) / block;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

size_t pd_smem_bytes(const gx_ctx *c) {
    const int NL = (c->tg.T[0] + 3) * (c->tg.T[1] + 3);
    return (size_t)4 * NL * sizeof(float4) + (size_t)c->tg.local * Rec<2>::SIZE * sizeof(float) +
           (size_t)kGroups * kChunk * 2 * sizeof(float4);
}

int alloc_bins(gx_ctx *c, int s, int cap) {
    Species &S = c->sp[s];
    const size_t nslot = (size_t)c->N * cap;
    for (int b = 0; b < 2; ++b) {
        for (int f = 0; f < PF_COUNT; ++f) {
            S.f[b][f] = nullptr;
            if (f == PF_OZ) continue;                          // 2D: no z offset
            if (f == PF_ID && !c->cfg.track_ids) continue;
            GX_CHECK(c, cudaMalloc(&S.f[b][f], nslot * sizeof(float)));
        }
        GX_CHECK(c, cudaMalloc(&S.cnt[b], c->N * sizeof(int)));
        GX_CHECK(c, cudaMemset(S.cnt[b], 0, c->N * sizeof(int)));
    }
    S.cap = cap;
    return GX_OK;
}

void free_bins(Species &S) {
    for (int b = 0; b < 2; ++b) {
        for (int f = 0; f < PF_COUNT; ++f) {
            if (S.f[b][f]) cudaFree(S.f[b][f]);
            S.f[b][f] = nullptr;
        }
        if (S.cnt[b]) cudaFree(S.cnt[b]);
        S.cnt[b] = nullptr;
    }
}

int round_cap(double v) {
    int cap = (int)ceil(v);
    cap = (cap + 31) / 32 * 32;
    return cap < 32 ? 32 : cap;
}

}  // namespace

// ------------------------------------------------------------------ tiles
int gx_choose_tiles(gx_ctx *c) {
    if (c->dim != 2) {
        c->err = "the particle kernels of this build handle the 2D (x-y) configuration";
        return GX_ENOTIMPL;
    }
    const int nx = c->n[0], ny = c->n[1];
    const int cx[] = {16, 8, 4, 2, 1}, cy[] = {8, 4, 2, 1};
    // prefer at least two waves of CTAs over the 152 SMs with the largest tile
    // (the ring costs relatively less on large tiles); otherwise the most tiles
    int bx = 1, by = 1;
    int64_t best_tiles = -1;
    int best_area = -1;
    bool best_two_waves = false;
    for (int a : cx) {
        if (nx % a) continue;
        for (int b : cy) {
            if (ny % b) continue;
            const int64_t tiles = (int64_t)(nx / a) * (ny / b);
            const int area = a * b;
            const bool two = tiles >= 304;
            bool better;
            if (two != best_two_waves) better = two;
            else if (two) better = area > best_area;
            else better = tiles > best_tiles || (tiles == best_tiles && area > best_area);
            if (best_tiles < 0 || better) { bx = a; by = b; best_tiles = tiles; best_area = area; best_two_waves = two; }
        }
    }
    TileGeom &t = c->tg;
    t.T[0] = bx; t.T[1] = by; t.T[2] = 1;
    t.ntile[0] = nx / bx; t.ntile[1] = ny / by; t.ntile[2] = 1;
    t.ntiles = t.ntile[0] * t.ntile[1];
    t.local = (bx + 2) * (by + 2);
    t.ring = t.local - bx * by;
    // ring-slot tables: local cell -> ring slot (-1 interior) and back
    const int LDx = bx + 2, LDy = by + 2;
    std::vector<int> sol(LDx * LDy, -1), los;
    for (int ly = 0; ly < LDy; ++ly)
        for (int lx = 0; lx < LDx; ++lx) {
            const bool interior = lx >= 1 && lx <= bx && ly >= 1 && ly <= by;
            if (!interior) { sol[lx + LDx * ly] = (int)los.size(); los.push_back(lx + LDx * ly); }
        }
    if (c->ring_slot_of_local) cudaFree(c->ring_slot_of_local);
    if (c->ring_local_of_slot) cudaFree(c->ring_local_of_slot);
    c->ring_slot_of_local = c->ring_local_of_slot = nullptr;
    GX_CHECK(c, cudaMalloc(&c->ring_slot_of_local, sol.size() * sizeof(int)));
    GX_CHECK(c, cudaMalloc(&c->ring_local_of_slot, los.size() * sizeof(int)));
    GX_CHECK(c, cudaMemcpy(c->ring_slot_of_local, sol.data(), sol.size() * sizeof(int), cudaMemcpyHostToDevice));
    GX_CHECK(c, cudaMemcpy(c->ring_local_of_slot, los.data(), los.size() * sizeof(int), cudaMemcpyHostToDevice));
    return GX_OK;
}

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
        k_locate<<<grid_for(n), 256, 0, st>>>(n, x, y, c->n[0], c->n[1], c->cfg.dx[0], c->cfg.dx[1], cell, ox, oy, count);
        GX_LAUNCHED(c);
    }
    int *dmax = nullptr;
    GX_CHECK(c, cudaMalloc(&dmax, sizeof(DevFlags)));
    GX_CHECK(c, cudaMemsetAsync(dmax, 0, sizeof(DevFlags), st));
    k_max_count<<<grid_for(c->N), 256, 0, st>>>(count, c->N, reinterpret_cast<DevFlags *>(dmax));
    GX_LAUNCHED(c);
    DevFlags hf{};
    GX_CHECK(c, cudaMemcpyAsync(&hf, dmax, sizeof(DevFlags), cudaMemcpyDeviceToHost, st));
    GX_CHECK(c, cudaStreamSynchronize(st));
    const double slack = c->cfg.bin_slack > 1.2 ? c->cfg.bin_slack : 1.2;
    const int cap = round_cap(std::max(32.0, hf.maxcount * slack));
    GX_CHECK(c, cudaFree(dmax));
    int rc = alloc_bins(c, s, cap);
    if (rc) return rc;
    // counts of the current copy = final cursor values
    float **dout = nullptr;
    GX_CHECK(c, cudaMalloc(&dout, PF_COUNT * sizeof(float *)));
    GX_CHECK(c, cudaMemcpyAsync(dout, S.f[c->cur], PF_COUNT * sizeof(float *), cudaMemcpyHostToDevice, st));
    GX_CHECK(c, cudaMemsetAsync(S.cnt[c->cur], 0, c->N * sizeof(int), st));
    if (n > 0) {
        k_scatter<<<grid_for(n), 256, 0, st>>>(n, cell, ox, oy, vx, vy, vz, w, id, cap, S.cnt[c->cur], dout,
                                                c->cfg.track_ids, c->dflags);
        GX_LAUNCHED(c);
    }
    GX_CHECK(c, cudaStreamSynchronize(st));
    cudaFree(dout); cudaFree(cell); cudaFree(ox); cudaFree(oy); cudaFree(count);
    return GX_OK;
}

int gx_regrow_bins(gx_ctx *c, int s, int newcap, cudaStream_t st) {
    Species &S = c->sp[s];
    Species old = S;
    int rc = alloc_bins(c, s, newcap);
    if (rc) return rc;
    float **dsrc = nullptr, **ddst = nullptr;
    GX_CHECK(c, cudaMalloc(&dsrc, PF_COUNT * sizeof(float *)));
    GX_CHECK(c, cudaMalloc(&ddst, PF_COUNT * sizeof(float *)));
    GX_CHECK(c, cudaMemcpyAsync(dsrc, old.f[c->cur], PF_COUNT * sizeof(float *), cudaMemcpyHostToDevice, st));
    GX_CHECK(c, cudaMemcpyAsync(ddst, S.f[c->cur], PF_COUNT * sizeof(float *), cudaMemcpyHostToDevice, st));
    k_rebin_copy<<<(unsigned)c->N, 128, 0, st>>>(c->N, old.cap, newcap, old.cnt[c->cur], dsrc, ddst, PF_COUNT);
    GX_LAUNCHED(c);
    GX_CHECK(c, cudaMemcpyAsync(S.cnt[c->cur], old.cnt[c->cur], c->N * sizeof(int), cudaMemcpyDeviceToDevice, st));
    GX_CHECK(c, cudaStreamSynchronize(st));
    cudaFree(dsrc); cudaFree(ddst);
    free_bins(old);
    return GX_OK;
}

// ------------------------------------------------------------ hot path
static int launch_pd(gx_ctx *c, bool push, cudaStream_t st) {
    const size_t smem = pd_smem_bytes(c);
    static size_t configured[2] = {0, 0};
    if (configured[push] < smem) {
        if (push) GX_CHECK(c, cudaFuncSetAttribute(k_push_deposit<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        else GX_CHECK(c, cudaFuncSetAttribute(k_push_deposit<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured[push] = smem;
    }
    const int nxt = 1 - c->cur;
    for (int s = 0; s < c->nspecies; ++s) {
        Species &S = c->sp[s];
        PDParams p{};
        for (int d = 0; d < 3; ++d) {
            p.n[d] = c->n[d];
            p.T[d] = c->tg.T[d];
            p.ntile[d] = c->tg.ntile[d];
            p.dtdx[d] = (float)(c->cfg.dt / c->cfg.dx[d]);
        }
        p.LD[0] = c->tg.T[0] + 2; p.LD[1] = c->tg.T[1] + 2; p.LD[2] = 1;
        p.NLD[0] = c->tg.T[0] + 3; p.NLD[1] = c->tg.T[1] + 3; p.NLD[2] = 1;
        p.local = c->tg.local;
        p.ring = c->tg.ring;
        p.cap = S.cap;
        const double beta = S.q * c->cfg.dt / (2.0 * S.m);
        p.beta = (float)beta;
        p.bc = (float)(beta / c->cfg.c);
        p.track = c->cfg.track_ids;
        for (int f = 0; f < PF_COUNT; ++f) {
            p.in[f] = S.f[c->cur][f];
            p.out[f] = S.f[nxt][f];
        }
        p.cnt_in = S.cnt[c->cur];
        p.cnt_out = S.cnt[nxt];
        if (push) {
            p.mE = c->nE; p.mB = c->nB; p.dB = c->nBnext; p.dU = c->nUref;
            GX_CHECK(c, cudaMemsetAsync(S.cnt[nxt], 0, c->N * sizeof(int), st));
        } else {
            p.mE = nullptr; p.mB = nullptr; p.dB = c->nB; p.dU = c->nUref;
        }
        p.rec = c->rec + (size_t)s * c->N * Rec<2>::SIZE;
        p.ring_out = c->ring + (size_t)s * c->tg.ntiles * c->tg.ring * Rec<2>::SIZE;
        p.ring_slot = c->ring_slot_of_local;
        p.flags = c->dflags;
        if (push) k_push_deposit<true><<<c->tg.ntiles, kThreads, smem, st>>>(p);
        else k_push_deposit<false><<<c->tg.ntiles, kThreads, smem, st>>>(p);
        GX_LAUNCHED(c);
        if (push) {
            const int64_t warps = (int64_t)c->tg.ntiles * c->tg.ring;
            k_fold_rings<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
                p.rec, p.ring_out, c->ring_local_of_slot, c->tg.ring, c->tg.ntiles, c->tg.ntile[0], c->tg.T[0],
                c->tg.T[1], c->tg.T[0] + 2, c->n[0], c->n[1]);
            GX_LAUNCHED(c);
        }
    }
    if (push) {
        c->cur = nxt;
        GX_CHECK(c, cudaMemsetAsync(&c->dflags->maxcount, 0, sizeof(int), st));
        for (int s = 0; s < c->nspecies; ++s) {
            k_max_count<<<grid_for(c->N), 256, 0, st>>>(c->sp[s].cnt[c->cur], c->N, c->dflags);
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
    int *offs = nullptr;
    void *tmp = nullptr;
    size_t tmpb = 0;
    GX_CHECK(c, cudaMalloc(&offs, (c->N + 1) * sizeof(int)));
    cub::DeviceScan::ExclusiveSum(nullptr, tmpb, S.cnt[c->cur], offs, (int)c->N, st);
    GX_CHECK(c, cudaMalloc(&tmp, tmpb + 16));
    GX_CHECK(c, cub::DeviceScan::ExclusiveSum(tmp, tmpb, S.cnt[c->cur], offs, (int)c->N, st));
    float **dsrc = nullptr;
    GX_CHECK(c, cudaMalloc(&dsrc, PF_COUNT * sizeof(float *)));
    GX_CHECK(c, cudaMemcpyAsync(dsrc, S.f[c->cur], PF_COUNT * sizeof(float *), cudaMemcpyHostToDevice, st));
    k_gather_out<<<(unsigned)c->N, 128, 0, st>>>(c->N, S.cap, S.cnt[c->cur], offs, dsrc, c->n[0], c->n[1],
                                                  c->cfg.dx[0], c->cfg.dx[1], x, y, z, vx, vy, vz, w, id);
    GX_LAUNCHED(c);
    GX_CHECK(c, cudaStreamSynchronize(st));
    cudaFree(offs); cudaFree(tmp); cudaFree(dsrc);
    return GX_OK;
}

size_t gx_pd_smem_bytes(const gx_ctx *c) { return pd_smem_bytes(c); }
void gx_free_bins(gx_ctx *c) {
    for (int s = 0; s < c->nspecies; ++s) free_bins(c->sp[s]);
}
