// gx_particles.cu -- particle kernels of the GL-ECSIM hot path (2D and 3D).
//
// k_pd<DIM, true> (the fused push) does, for every particle of a species, in
// one pass over the cell bins:
//   1. the theta-implicit mover of Sec. 2.1 (Eq. 29-30 and the ECSIM update):
//      vbar = alpha (v^n + beta_s E^{n+theta}), v^{n+1} = 2 vbar - v^n,
//      x^{n+3/2} = x^{n+1/2} + dt v^{n+1}, alpha from B^n (Eq. 30);
//   2. the deposit of step n+1 for the particles that stay in their cell, with
//      alpha from B^{n+1}: charge, mass and momentum weights, the current
//      alpha (v - u_ref) and the mass-matrix sums alpha W_g W_g' (Eq. 33-35);
//   3. re-binning into the other copy of the particle arrays: a cell's stayers
//      fill its new bin from the bottom in order, particles that leave take
//      slots at the top of their new cell's bin (see bin_front / bin_back).
// k_pd<DIM, false> deposits without moving: the whole state (the deposit
// before the first step), or, right after the push, only the particles that
// arrived in each cell (the back segments of the new bins), added to the
// records the push wrote with fire-and-forget atomic adds.
//
// Particle layout: per species and copy, cell bins of `cap` slots, each bin a
// small structure of arrays: field f of slot s of cell c at
// p[(c cap + s) ... ] = p[c cap nf + f cap + s], fields (o_0 .. o_{d-1}, v_x,
// v_y, v_z, w[, id]) with o the cell-local offsets in [0, 1).  A warp reads 32
// consecutive slots of a field as one coalesced 128-byte line.
//
// Work decomposition (GB300-first): one warp per cell, cells strided over all
// warps of a persistent grid.  The 32 lanes move 32 particles of the cell at a
// time.  The deposit is output-stationary with register blocking: every lane
// that deposits writes its particle's factors into the warp's shared table,
// the 2^d x 2^d corner-pair weights w X_jx Y_jy (Z_jz) (9 pair classes in 2D,
// 27 in 3D) and 16 columns (the nine entries of alpha, 1, v and
// alpha (v - u_ref)).  The warp's lanes form particle groups; within a group
// each lane owns a block of 9 pair classes x NCB columns (sums in registers,
// kept over all chunks of the cell) and walks the group's particles, so each
// particle's factors are read from shared memory by few lanes (2D: 4 groups of
// 8 lanes with 9 x 2 blocks; 3D: 2 groups of 12 with 9 x 4).  At the end of
// the cell the groups' sums are added, and the cell's record follows from the
// 16 sums per pair class: the mass-matrix sums are the alpha columns, and the
// charge, momentum and current weights of corner a are the sums of the 2^d pair
// classes whose product makes up W_a (for linear weights (1-o) = X_0 + X_1 and
// o = X_1 + X_2 per axis).  A lane holds 18 (2D) or 36 (3D) sums instead of the
// record's 109 or 299, so many warps fit an SM, and the same kernel serves both
// dimensions.  The FP32
// particle arithmetic stays on the CUDA cores: it is a scatter, not a dense
// contraction.
#include <cub/cub.cuh>

#include "gx_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarpsPerCta = kThreads / 32;
constexpr int kCols = 16;                         // alpha[9], 1, v[3], alpha (v - u_ref) [3]
constexpr unsigned kFull = 0xffffffffu;

// NC corners; ROWS pair classes in groups of 9; factor table of TSTR floats
// per particle (group g's 9 weights at 12 g, the 16 columns at COLOFF); NCB
// columns per lane block; LK lanes per particle group (row sets x 16 / NCB
// column blocks), KG groups; CTAS resident CTAs per SM
template <int DIM> struct Geo;
template <> struct Geo<2> {
    static constexpr int NC = 4, ROWS = 9, TSTR = 28, COLOFF = 12, NCB = 2, LK = 8, KG = 4, CENTER = 4, CTAS = 3;
};
template <> struct Geo<3> {
    static constexpr int NC = 8, ROWS = 27, TSTR = 52, COLOFF = 36, NCB = 4, LK = 12, KG = 2, CENTER = 13, CTAS = 2;
};
// shared floats per warp: the cell's interpolation coefficients [4][NC] float4,
// then the factor table [32][TSTR], which at the end of a cell holds the groups'
// sums [KG][ROWS][16] followed by their totals [ROWS][16]; after the warps, the
// CTA's record-tile stages (pd_stages)
template <int DIM>
__host__ __device__ constexpr int table_floats() {
    return 32 * Geo<DIM>::TSTR > (Geo<DIM>::KG + 1) * Geo<DIM>::ROWS * kCols
               ? 32 * Geo<DIM>::TSTR
               : (Geo<DIM>::KG + 1) * Geo<DIM>::ROWS * kCols;
}
template <int DIM>
__host__ __device__ constexpr int warp_floats() {
    return 16 * Geo<DIM>::NC + table_floats<DIM>();
}
// record-tile stages, double-buffered: in 2D four tiles are staged between CTA
// barriers (one barrier per four tiles, so a warp's cells of four tiles even
// out); in 3D one (the larger shared footprint cost more than the barrier saved)
template <int DIM>
__host__ __device__ constexpr int pd_stages() { return DIM == 2 ? 8 : 2; }
// in 2D a warp's leavers wait in shared memory (kLeaverCap of them) until the
// next chunk's might not fit, and to the end of the kernel: per leaver its
// offsets, velocity, weight, id and destination cell (leaver_stride floats).
// In 3D each chunk writes its own leavers after its deposit, which hides the
// reservation's latency (a buffer there cost 12 % at 64 particles per cell).
template <int DIM>
__host__ __device__ constexpr int leaver_stride() { return DIM == 2 ? 8 : 12; }
constexpr int kLeaverCap = 64;
template <int DIM>
__host__ __device__ constexpr bool leaver_buffer() { return DIM == 2; }
template <int DIM>
__host__ __device__ constexpr int leaver_floats() { return leaver_buffer<DIM>() ? kLeaverCap * leaver_stride<DIM>() : 0; }
template <int DIM>
constexpr size_t pd_smem_bytes() {
    return ((size_t)kWarpsPerCta * (warp_floats<DIM>() + leaver_floats<DIM>()) +
            pd_stages<DIM>() * (size_t)Rec<DIM>::SIZE * kRecTile) *
           sizeof(float);
}
static_assert(kWarpsPerCta == kRecTile, "one warp per cell of a record tile");

// field indices of a slot
template <int DIM> struct PF {
    static constexpr int V = DIM, W = DIM + 3, ID = DIM + 4;
};

struct PD {
    int n[3];
    int64_t N;
    int cap, nf;                 // bin capacity, fields stored per slot
    float dtd[3];                // dt / dx_d
    float beta;                  // q dt / (2 m)
    float bc;                    // beta / c
    const float *in;             // current copy
    const int *cnt_in;
    float *out;                  // other copy
    int *cnt_out;
    const float4 *mE, *mB;       // mover: E^{n+theta}, B^n (node averaged)
    const float4 *dB, *dU;       // deposit: B for alpha, reference velocity u_ref
    float *rec;                  // this species' tile-major records (rec_index)
    DevFlags *flags;
    int arrivals;                // deposit only the back segments (the particles that arrived)
    int wall_ci;                 // x index of the last cell before a reflecting wall, or -1
    int glon;                    // Gauss's-law correction: phi in the .w of the mover's E corners
    float gl[3];                 // its step per axis in cell units: gamma eps q / dx_d^2
};

// ------------------------------------------------------------ helpers
// 1 / x for 1 <= x < 2^126: the PTX approximate reciprocal (rcp.approx.ftz,
// within about 1 ulp) refined by one Newton-Raphson step r + r (1 - x r), which
// squares its relative error, so the result is within about 1 ulp of 1 / x.
// The mover's v^{n+1} feeds the comoving current alpha (v - u_ref), a small
// difference of large terms, so an unrefined approximation shows there.
__device__ __forceinline__ float recip_nr(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}

// alpha (Eq. 30) with b = beta B / c, row-major: alpha a = (a + a x b + (a.b) b)/(1 + b.b)
__device__ __forceinline__ void alpha_tensor(float bx, float by, float bz, float al[9]) {
    const float inv = recip_nr(fmaf(bx, bx, fmaf(by, by, fmaf(bz, bz, 1.0f))));
    al[0] = (1.0f + bx * bx) * inv; al[1] = (bz + bx * by) * inv; al[2] = (bx * bz - by) * inv;
    al[3] = (by * bx - bz) * inv;   al[4] = (1.0f + by * by) * inv; al[5] = (bx + by * bz) * inv;
    al[6] = (by + bz * bx) * inv;   al[7] = (bz * by - bx) * inv; al[8] = (1.0f + bz * bz) * inv;
}

// clamp a (possibly overflowed) count word to the capacity
__host__ __device__ __forceinline__ int clamp_word(int w, int cap) {
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

// linear weights of the 2^DIM corners at cell-local offsets o (corner a: bit d
// of a selects o_d, else 1 - o_d)
template <int DIM>
__device__ __forceinline__ void corner_weights(const float o[3], float W[Geo<DIM>::NC]) {
    const float x0 = 1.f - o[0], y0 = 1.f - o[1];
    W[0] = x0 * y0; W[1] = o[0] * y0; W[2] = x0 * o[1]; W[3] = o[0] * o[1];
    if constexpr (DIM == 3) {
        const float z0 = 1.f - o[2];
#pragma unroll
        for (int a = 0; a < 4; ++a) { W[a + 4] = W[a] * o[2]; W[a] *= z0; }
    }
}

// sum of a corner field at the particle: returns (x, y, z) of sum_a W_a f_a
template <int DIM>
__device__ __forceinline__ void gather(const float4 *f, const float W[Geo<DIM>::NC], float out[3]) {
    out[0] = out[1] = out[2] = 0.f;
#pragma unroll
    for (int a = 0; a < Geo<DIM>::NC; ++a) {
        const float4 v = f[a];
        out[0] = fmaf(W[a], v.x, out[0]);
        out[1] = fmaf(W[a], v.y, out[1]);
        out[2] = fmaf(W[a], v.z, out[2]);
    }
}

// The multilinear interpolant sum_a W_a(o) f_a of a cell's corner values, as
// the polynomial sum_S c_S prod_{d in S} o_d over the subsets S of the axes
// (c_S the coefficient of corner index S: c_0 = f_0, c_1 = f_1 - f_0, ...,
// the Moebius transform of the corner values over the bits of the corner
// index).  interp evaluates its x, y, z components by Horner steps, grad_w the
// gradient of its w component with respect to o.
template <int DIM>
__device__ __forceinline__ void interp(const float4 *c, const float o[3], float out[3]) {
    const float4 c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3];
    out[0] = fmaf(o[1], fmaf(o[0], c3.x, c2.x), fmaf(o[0], c1.x, c0.x));
    out[1] = fmaf(o[1], fmaf(o[0], c3.y, c2.y), fmaf(o[0], c1.y, c0.y));
    out[2] = fmaf(o[1], fmaf(o[0], c3.z, c2.z), fmaf(o[0], c1.z, c0.z));
    if constexpr (DIM == 3) {
        const float4 c4 = c[4], c5 = c[5], c6 = c[6], c7 = c[7];
        out[0] = fmaf(o[2], fmaf(o[1], fmaf(o[0], c7.x, c6.x), fmaf(o[0], c5.x, c4.x)), out[0]);
        out[1] = fmaf(o[2], fmaf(o[1], fmaf(o[0], c7.y, c6.y), fmaf(o[0], c5.y, c4.y)), out[1]);
        out[2] = fmaf(o[2], fmaf(o[1], fmaf(o[0], c7.z, c6.z), fmaf(o[0], c5.z, c4.z)), out[2]);
    }
}
template <int DIM>
__device__ __forceinline__ void grad_w(const float4 *c, const float o[3], float g[3]) {
    if constexpr (DIM == 2) {
        g[0] = fmaf(o[1], c[3].w, c[1].w);
        g[1] = fmaf(o[0], c[3].w, c[2].w);
        g[2] = 0.f;
    } else {
        g[0] = fmaf(o[2], fmaf(o[1], c[7].w, c[5].w), fmaf(o[1], c[3].w, c[1].w));
        g[1] = fmaf(o[2], fmaf(o[0], c[7].w, c[6].w), fmaf(o[0], c[3].w, c[2].w));
        g[2] = fmaf(o[1], fmaf(o[0], c[7].w, c[6].w), fmaf(o[0], c[5].w, c[4].w));
    }
}

// corner a's coefficient from the corner values held by the lanes of its array
// (lanes a ^ (1 << d) within the NC-lane group); every lane of the warp calls it
template <int DIM>
__device__ __forceinline__ float4 to_coef(float4 v, int a) {
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const float qx = __shfl_xor_sync(kFull, v.x, 1 << d), qy = __shfl_xor_sync(kFull, v.y, 1 << d);
        const float qz = __shfl_xor_sync(kFull, v.z, 1 << d), qw = __shfl_xor_sync(kFull, v.w, 1 << d);
        if ((a >> d) & 1) { v.x -= qx; v.y -= qy; v.z -= qz; v.w -= qw; }
    }
    return v;
}

__device__ __forceinline__ int64_t node_of(const int n[3], int i, int j, int k) {
    i = i >= n[0] ? i - n[0] : i;
    j = j >= n[1] ? j - n[1] : j;
    k = k >= n[2] ? k - n[2] : k;
    return (int64_t)i + (int64_t)n[0] * ((int64_t)j + (int64_t)n[1] * k);
}

// lane < 4 NC: corner a = lane % NC of array lane / NC (mover E, mover B,
// deposit B, u_ref) of cell (ci, cj, ck); the deposit pass needs arrays 2, 3 only
template <int DIM, bool PUSH>
__device__ __forceinline__ float4 load_corner(const PD &p, int lane, int ci, int cj, int ck) {
    constexpr int NC = Geo<DIM>::NC;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    const int arr = lane / NC, a = lane % NC;
    if (lane < 4 * NC && (PUSH || arr >= 2)) {
        const int64_t nd = node_of(p.n, ci + (a & 1), cj + ((a >> 1) & 1), ck + ((a >> 2) & 1));
        const float4 *src = arr == 0 ? p.mE : arr == 1 ? p.mB : arr == 2 ? p.dB : p.dU;
        v = __ldg(src + nd);
    }
    return v;
}

// record entry k of a cell from the group-summed pair-class sums Gs[j][16]
// (pair class j, column c: alpha 0..8, 1, v 10..12, alpha (v - u_ref) 13..15)
template <int DIM>
__device__ __forceinline__ float record_value(const float *Gs, int k) {
    using R = Rec<DIM>;
    using G = Geo<DIM>;
    if (k >= R::USED) return 0.f;
    if (k >= R::M) {                                          // M entry (j, e): the alpha column e
        const int t = k - R::M, j = t / 9, e = t - 9 * j;
        return Gs[j * kCols + e];
    }
    int a, col;
    if (k < R::MV) { a = k; col = 9; }
    else if (k < R::J) { const int t = k - R::MV; a = t / 3; col = 10 + t - 3 * a; }
    else { const int t = k - R::J; a = t / 3; col = 13 + t - 3 * a; }
    // W_a = prod_d (X_0 + X_1 or X_1 + X_2): the 2^d pair classes j0 + (bits of t)
    const int j0 = (a & 1) + 3 * ((a >> 1) & 1) + 9 * ((a >> 2) & 1);
    float s = 0.f;
#pragma unroll
    for (int t = 0; t < G::NC; ++t) s += Gs[(j0 + (t & 1) + 3 * ((t >> 1) & 1) + 9 * ((t >> 2) & 1)) * kCols + col];
    return s;
}

// ------------------------------------------------------------ fused kernel
// A CTA's 8 warps take the 8 cells of a record tile (one cell each), tiles
// strided over the persistent grid; the tile's records are staged in shared
// memory and written (or, for the arrivals, added) as one contiguous block.
// Every warp prefetches the next tile's cell: its count and corner values at the
// start of a cell, its first chunk of particles with the last chunk of the cell.
// WALL: the push reflects particles at the high-x face of cell x index
// p.wall_ci (a reflecting wall); a separate instantiation, so that the push
// without a wall compiles exactly as it would without the feature
template <int DIM, bool PUSH, bool WALL = false>
__global__ void __launch_bounds__(kThreads, Geo<DIM>::CTAS) k_pd(const __grid_constant__ PD p) {
    using G = Geo<DIM>;
    using R = Rec<DIM>;
    constexpr int NC = G::NC;
    constexpr int TILE = R::SIZE * kRecTile;                 // floats of a tile's record block
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *ws = smem + (size_t)warp * warp_floats<DIM>();
    float4 *cor = reinterpret_cast<float4 *>(ws);            // [4][NC] coefficients: mover E, mover B, deposit B, u_ref
    float *T = ws + 16 * NC;                                  // factor table [32][TSTR]; at a cell's end the sums
    float *stage = smem + (size_t)kWarpsPerCta * warp_floats<DIM>();   // [pd_stages][TILE]
    constexpr int NST = pd_stages<DIM>(), TPB = NST / 2;     // stages, tiles per CTA barrier
    const unsigned lt = (1u << lane) - 1u;
    // this lane's block and particle group: group kg walks the particles
    // KG s + pg; in 2D the two groups of a quarter warp take particles 4 apart,
    // which puts their table reads in different banks
    const int kg = lane / G::LK, lk = lane % G::LK;
    const bool role = kg < G::KG;
    const int pg = kg;
    constexpr int NCB = G::NCB, NQ = kCols / NCB;             // columns of a lane's block, blocks per row set
    static_assert(NCB == 1 || NCB == 2 || NCB == 4, "lane blocks of 1, 2 or 4 columns");
    const int roff = 12 * (lk / NQ), coff = G::COLOFF + NCB * (lk % NQ);
    const bool res[3] = {p.n[0] > 1, p.n[1] > 1, DIM == 3 && p.n[2] > 1};
    const int64_t ntiles = (p.N + kRecTile - 1) / kRecTile;
    const int64_t cstride = (int64_t)p.cap * p.nf;           // floats per bin
    // this warp's cell in its first tile and its coordinates, stepped by the warp's
    // cell stride without divisions (cells < 2^31)
    const unsigned nx = (unsigned)p.n[0], ny = (unsigned)p.n[1];
    const unsigned cs = gridDim.x * (unsigned)kRecTile;
    int64_t cell = (int64_t)blockIdx.x * kRecTile + warp;
    int ci, cj, ck;
    {
        const unsigned c0u = (unsigned)cell;
        ci = (int)(c0u % nx); cj = (int)((c0u / nx) % ny); ck = (int)(c0u / nx / ny);
    }
    const int si = (int)(cs % nx), sj = (int)((cs / nx) % ny), sk = (int)(cs / nx / ny);
    // scale of this lane's corner array: beta E (w: phi), beta / c B, beta / c B, u_ref
    const int carr = lane / NC, ca = lane % NC;
    const float csc = carr == 0 ? p.beta : (carr == 3 ? 1.f : p.bc);

    int wcur = cell < p.N ? seg_word(__ldg(p.cnt_in + cell), p.cap, p.arrivals) : 0;
    float4 ccur = cell < p.N ? load_corner<DIM, PUSH>(p, lane, ci, cj, ck) : make_float4(0.f, 0.f, 0.f, 0.f);

    // the next chunk's fields (registers): loaded one chunk ahead, across cells
    float po[DIM], pv[3], pw = 0.f, pid = 0.f;
    auto fetch = [&](const float *bin, int word, int c0) {
        const int nf_ = bin_front(word), nb_ = bin_back(word);
        const int i = c0 + lane;
#pragma unroll
        for (int d = 0; d < DIM; ++d) po[d] = 0.5f;
        pv[0] = pv[1] = pv[2] = 0.f;
        pw = 0.f;
        if (i < nf_ + nb_) {
            const float *q = bin + (i < nf_ ? i : p.cap - nb_ + (i - nf_));
#pragma unroll
            for (int d = 0; d < DIM; ++d) po[d] = __ldcs(q + (size_t)d * p.cap);
#pragma unroll
            for (int d = 0; d < 3; ++d) pv[d] = __ldcs(q + (size_t)(PF<DIM>::V + d) * p.cap);
            pw = __ldcs(q + (size_t)PF<DIM>::W * p.cap);
            if (PUSH && p.nf > PF<DIM>::ID) pid = __ldcs(q + (size_t)PF<DIM>::ID * p.cap);
        }
    };
    if (cell < p.N) fetch(p.in + cell * cstride, wcur, 0);

    // leavers wait in this warp's shared buffer (kLeaverCap entries of LVS floats:
    // offsets, velocity, weight, id, destination cell) and are written out at the
    // start of a chunk when more than 32 are pending, and at the end: one atomic
    // per destination and round of 32 reserves a run at the top of the
    // destination bin (its back segment), and each leaver takes its rank within
    // the run
    constexpr int LVS = leaver_stride<DIM>();
    constexpr bool LB = leaver_buffer<DIM>();
    float *lbuf = stage + (size_t)NST * TILE + (size_t)warp * leaver_floats<DIM>();
    int lpend = 0;                                            // leavers in lbuf (warp-uniform)
    auto flush_leavers = [&]() {
        __syncwarp();
        for (int b0 = 0; b0 < lpend; b0 += 32) {
            const int k = min(32, lpend - b0);
            const unsigned mk = k >= 32 ? kFull : ((1u << k) - 1u);
            if (lane < k) {
                const float *e = lbuf + (b0 + lane) * LVS;
                const float4 e0 = *reinterpret_cast<const float4 *>(e);
                const float4 e1 = *reinterpret_cast<const float4 *>(e + 4);
                float lo[3], lv[3], lw, lid;
                int dcell;
                if (DIM == 2) {
                    lo[0] = e0.x; lo[1] = e0.y; lo[2] = 0.f;
                    lv[0] = e0.z; lv[1] = e0.w; lv[2] = e1.x;
                    lw = e1.y; lid = e1.z; dcell = __float_as_int(e1.w);
                } else {
                    lo[0] = e0.x; lo[1] = e0.y; lo[2] = e0.z;
                    lv[0] = e0.w; lv[1] = e1.x; lv[2] = e1.y;
                    lw = e1.z; lid = e1.w; dcell = __float_as_int(e[8]);
                }
                const int64_t dest = dcell;
                const unsigned peers = __match_any_sync(mk, dcell);
                const int leader = __ffs(peers) - 1;
                int lold = 0;
                if (lane == leader) lold = atomicAdd(p.cnt_out + dest, __popc(peers) << 16);
                const int back = bin_back(__shfl_sync(peers, lold, leader)) + __popc(peers & lt);
                if (back < p.cap) {
                    float *dst = p.out + dest * cstride + (p.cap - 1 - back);
#pragma unroll
                    for (int d = 0; d < DIM; ++d) __stcs(dst + (size_t)d * p.cap, lo[d]);
#pragma unroll
                    for (int d = 0; d < 3; ++d) __stcs(dst + (size_t)(PF<DIM>::V + d) * p.cap, lv[d]);
                    __stcs(dst + (size_t)PF<DIM>::W * p.cap, lw);
                    if (p.nf > PF<DIM>::ID) __stcs(dst + (size_t)PF<DIM>::ID * p.cap, lid);
                } else {
                    atomicExch(&p.flags->overflow, 1);
                }
            }
        }
        __syncwarp();
        lpend = 0;
    };

    int it = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        // the next tile's cell of this warp: count and corners now, first chunk later
        const int64_t ncell = cell + cs;
        int nci = ci + si, ncj = cj + sj, nck = ck + sk;
        if (nci >= p.n[0]) { nci -= p.n[0]; ++ncj; }
        if (ncj >= p.n[1]) { ncj -= p.n[1]; ++nck; }
        const bool has_next = ncell < p.N;
        const int wnext = has_next ? seg_word(__ldg(p.cnt_in + ncell), p.cap, p.arrivals) : 0;
        const float4 cnext =
            has_next ? load_corner<DIM, PUSH>(p, lane, nci, ncj, nck) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float *bin_nx = p.in + ncell * cstride;

        const int nfr = bin_front(wcur), nbk = bin_back(wcur), n = nfr + nbk;
        __syncwarp();                                         // the previous cell's reads of cor and T are done
        {
            float4 v = ccur;
            v.x *= csc; v.y *= csc; v.z *= csc;
            v = to_coef<DIM>(v, ca);
            if (lane < 4 * NC) cor[lane] = v;
        }
        __syncwarp();
        float2 accp[NCB][4];                                  // [column][row pair]: rows 0..7 of the block
        float acc8[NCB];                                      // row 8
#pragma unroll
        for (int c = 0; c < NCB; ++c) {
            acc8[c] = 0.f;
#pragma unroll
            for (int r = 0; r < 4; ++r) accp[c][r] = make_float2(0.f, 0.f);
        }
        float *bin_out = PUSH ? p.out + cell * cstride : nullptr;
        const bool wallc = WALL && PUSH && ci == p.wall_ci;   // the wall is this cell's high-x face
        int fbase = 0;                                        // stayers written to this cell's new bin so far

        for (int c0 = 0; c0 < n; c0 += 32) {
            if (PUSH && LB && lpend > kLeaverCap - 32) flush_leavers();   // room for this chunk's leavers
            const int i = c0 + lane;
            const bool valid = i < n;
            float o[3] = {0.5f, 0.5f, 0.5f}, v[3] = {pv[0], pv[1], pv[2]}, w = pw, idb = pid;
#pragma unroll
            for (int d = 0; d < DIM; ++d) o[d] = po[d];
            if (c0 + 32 < n) fetch(p.in + cell * cstride, wcur, c0 + 32);
            else if (has_next) fetch(bin_nx, wnext, 0);
            if (DIM == 2) o[2] = 0.f;
            bool dep = valid;
            // 3D: a leaver's reservation (destination, its run's lanes and leader, the
            // leader's atomic), used after the chunk's deposit
            bool leaver = false;
            unsigned peers = 0u;
            int leader = 0, lold = 0;
            int64_t dest = 0;
            if (PUSH) {
                // ---- mover (Eq. 29-30, ECSIM update): e = beta E^{n+theta}, b = beta B^n / c
                float e3[3], b3[3];
                interp<DIM>(cor, o, e3);
                interp<DIM>(cor + NC, o, b3);
                const float bx = b3[0], by = b3[1], bz = b3[2];
                // a = v + beta E ; vbar = (a + a x b + (a.b) b) / (1 + b.b)
                const float ax = v[0] + e3[0], ay = v[1] + e3[1], az = v[2] + e3[2];
                const float inv = recip_nr(fmaf(bx, bx, fmaf(by, by, fmaf(bz, bz, 1.0f))));
                const float ab = ax * bx + ay * by + az * bz;
                const float vbx = (ax + (ay * bz - az * by) + ab * bx) * inv;
                const float vby = (ay + (az * bx - ax * bz) + ab * by) * inv;
                const float vbz = (az + (ax * by - ay * bx) + ab * bz) * inv;
                v[0] = 2.f * vbx - v[0]; v[1] = 2.f * vby - v[1]; v[2] = 2.f * vbz - v[2];
                // Gauss's-law correction: gamma eps q w grad phi at x^{n+1/2}, in cell units
                float gd[3] = {0.f, 0.f, 0.f};
                if (p.glon) {
                    grad_w<DIM>(cor, o, gd);
#pragma unroll
                    for (int d = 0; d < 3; ++d) gd[d] *= p.gl[d] * w;
                }
                int s[3] = {0, 0, 0};
                bool cfl = false;
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    o[d] = fmaf(v[d], p.dtd[d], o[d]) + gd[d];
                    if (WALL && d == 0 && wallc && o[0] >= 1.f) { o[0] = 2.f - o[0]; v[0] = -v[0]; }   // specular reflection
                    float f = floorf(o[d]);
                    o[d] -= f;
                    if (o[d] >= 1.f) { o[d] -= 1.f; f += 1.f; }
                    s[d] = (int)f;
                    if (s[d] < -1 || s[d] > 1) { cfl = true; s[d] = max(-1, min(1, s[d])); }
                    if (!res[d]) { s[d] = 0; o[d] = 0.f; }
                }
                if (valid && cfl) atomicExch(&p.flags->cfl, 1);
                const int code = (s[0] + 1) + 3 * (s[1] + 1) + (DIM == 3 ? 9 * (s[2] + 1) : 0);
                const bool stay = code == G::CENTER;
                // ---- re-bin: stayers to the bottom of this cell's new bin, in order
                const unsigned ms = __ballot_sync(kFull, valid && stay);
                const unsigned ml = __ballot_sync(kFull, valid && !stay);
                if (valid && stay) {
                    float *dst = bin_out + fbase + __popc(ms & lt);
#pragma unroll
                    for (int d = 0; d < DIM; ++d) __stcs(dst + (size_t)d * p.cap, o[d]);
#pragma unroll
                    for (int d = 0; d < 3; ++d) __stcs(dst + (size_t)(PF<DIM>::V + d) * p.cap, v[d]);
                    __stcs(dst + (size_t)PF<DIM>::W * p.cap, w);
                    if (p.nf > PF<DIM>::ID) __stcs(dst + (size_t)PF<DIM>::ID * p.cap, idb);
                } else if (!LB && valid) {
                    // ---- leavers: one atomic per (warp, destination) reserves a run at the
                    // top of the destination bin; each leaver takes its rank within the run
                    leaver = true;
                    int di = ci + s[0], dj = cj + s[1], dk = ck + s[2];
                    di = di < 0 ? di + p.n[0] : (di >= p.n[0] ? di - p.n[0] : di);
                    dj = dj < 0 ? dj + p.n[1] : (dj >= p.n[1] ? dj - p.n[1] : dj);
                    if (DIM == 3) dk = dk < 0 ? dk + p.n[2] : (dk >= p.n[2] ? dk - p.n[2] : dk);
                    dest = (int64_t)(di + p.n[0] * (dj + p.n[1] * dk));
                    peers = __match_any_sync(ml, code);
                    leader = __ffs(peers) - 1;
                    if (lane == leader) lold = atomicAdd(p.cnt_out + dest, __popc(peers) << 16);
                }
                if constexpr (LB) {
                    // ---- leavers: into the warp's buffer with their destination cell, written
                    // out at a chunk's start when the buffer might not hold its leavers
                    const int nl = __popc(ml);
                    if (nl > 0) {                             // warp-uniform
                        if (valid && !stay) {
                            int di = ci + s[0], dj = cj + s[1], dk = ck + s[2];
                            di = di < 0 ? di + p.n[0] : (di >= p.n[0] ? di - p.n[0] : di);
                            dj = dj < 0 ? dj + p.n[1] : (dj >= p.n[1] ? dj - p.n[1] : dj);
                            if (DIM == 3) dk = dk < 0 ? dk + p.n[2] : (dk >= p.n[2] ? dk - p.n[2] : dk);
                            const int dcell = di + p.n[0] * (dj + p.n[1] * dk);
                            float *e = lbuf + (lpend + __popc(ml & lt)) * LVS;
                            if (DIM == 2) {
                                *reinterpret_cast<float4 *>(e) = make_float4(o[0], o[1], v[0], v[1]);
                                *reinterpret_cast<float4 *>(e + 4) = make_float4(v[2], w, idb, __int_as_float(dcell));
                            } else {
                                *reinterpret_cast<float4 *>(e) = make_float4(o[0], o[1], o[2], v[0]);
                                *reinterpret_cast<float4 *>(e + 4) = make_float4(v[1], v[2], w, idb);
                                e[8] = __int_as_float(dcell);
                            }
                        }
                        lpend += nl;
                    }
                }
                fbase += __popc(ms);
                dep = valid && stay;
            }
            // ---- deposit factors of this lane's particle: in 2D written (if it deposits) as
            // row `its rank among the depositing lanes`, so that the rows [0, nrows) are
            // dense; in 3D as row `lane`, zero weights if it does not deposit (compacting
            // spilled registers there): b = beta B^{n+1} / c and u_ref at the particle
            constexpr bool CR = DIM == 2;
            const unsigned md = CR ? __ballot_sync(kFull, dep) : 0u;
            const int nrows = CR ? __popc(md) : min(32, n - c0);
            {
                float b3[3], U3[3], al[9];
                interp<DIM>(cor + 2 * NC, o, b3);
                interp<DIM>(cor + 3 * NC, o, U3);
                alpha_tensor(b3[0], b3[1], b3[2], al);
                const float d0 = v[0] - U3[0], d1 = v[1] - U3[1], d2 = v[2] - U3[2];
                const float wd = CR || dep ? w : 0.f;
                float X[3][3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float a0 = 1.f - o[d];
                    X[d][0] = a0 * a0; X[d][1] = a0 * o[d]; X[d][2] = o[d] * o[d];
                }
                float *tp = T + (CR ? __popc(md & lt) : lane) * G::TSTR;
                float *col = tp + G::COLOFF;
                if (!CR || dep) {
                    *reinterpret_cast<float4 *>(col) = make_float4(al[0], al[1], al[2], al[3]);
                    *reinterpret_cast<float4 *>(col + 4) = make_float4(al[4], al[5], al[6], al[7]);
                    *reinterpret_cast<float4 *>(col + 8) = make_float4(al[8], 1.f, v[0], v[1]);
                    *reinterpret_cast<float4 *>(col + 12) =
                        make_float4(v[2], fmaf(al[0], d0, fmaf(al[1], d1, al[2] * d2)),
                                    fmaf(al[3], d0, fmaf(al[4], d1, al[5] * d2)), fmaf(al[6], d0, fmaf(al[7], d1, al[8] * d2)));
#pragma unroll
                    for (int jz = 0; jz < (DIM == 3 ? 3 : 1); ++jz) {
                        float rw[9];
#pragma unroll
                        for (int jy = 0; jy < 3; ++jy) {
                            const float wyz = DIM == 3 ? wd * X[1][jy] * X[2][jz] : wd * X[1][jy];
#pragma unroll
                            for (int jx = 0; jx < 3; ++jx) rw[jx + 3 * jy] = wyz * X[0][jx];
                        }
                        float *rp = tp + 12 * jz;
                        *reinterpret_cast<float4 *>(rp) = make_float4(rw[0], rw[1], rw[2], rw[3]);
                        *reinterpret_cast<float4 *>(rp + 4) = make_float4(rw[4], rw[5], rw[6], rw[7]);
                        rp[8] = rw[8];
                    }
                }
            }
            __syncwarp();
            // ---- output-stationary accumulation: this lane adds, over its group's
            // particles, its 9 pair classes x NCB columns
            auto accumulate = [&](int pp) {
                const float *tp = T + pp * G::TSTR;
                const float4 r03 = *reinterpret_cast<const float4 *>(tp + roff);
                const float4 r47 = *reinterpret_cast<const float4 *>(tp + roff + 4);
                const float r8 = tp[roff + 8];
                float cc[NCB];
                if constexpr (NCB == 4) {
                    const float4 cv = *reinterpret_cast<const float4 *>(tp + coff);
                    cc[0] = cv.x; cc[1] = cv.y; cc[2] = cv.z; cc[3] = cv.w;
                } else if constexpr (NCB == 2) {
                    const float2 cv = *reinterpret_cast<const float2 *>(tp + coff);
                    cc[0] = cv.x; cc[1] = cv.y;
                } else {
                    cc[0] = tp[coff];
                }
#pragma unroll
                for (int c = 0; c < NCB; ++c) {
                    const float2 d = make_float2(cc[c], cc[c]);
                    accp[c][0] = __ffma2_rn(make_float2(r03.x, r03.y), d, accp[c][0]);
                    accp[c][1] = __ffma2_rn(make_float2(r03.z, r03.w), d, accp[c][1]);
                    accp[c][2] = __ffma2_rn(make_float2(r47.x, r47.y), d, accp[c][2]);
                    accp[c][3] = __ffma2_rn(make_float2(r47.z, r47.w), d, accp[c][3]);
                    acc8[c] = fmaf(r8, cc[c], acc8[c]);
                }
            };
            if (role) {
                if constexpr (DIM == 3) {
                    // a fixed trip count (the warp-uniform break skips the iterations past
                    // the last row): faster in 3D only
#pragma unroll
                    for (int si = 0; si < 32 / G::KG; ++si) {
                        if (G::KG * si >= nrows) break;
                        accumulate(pg + G::KG * si);   // rows past the chunk's end are zero
                    }
                } else {
                    // two particles per trip (the loop overhead and the table loads of
                    // both in flight together)
#pragma unroll 2
                    for (int pp = pg; pp < nrows; pp += G::KG) accumulate(pp);
                }
            }
            // ---- 3D leavers: the slot their run reserved
            if (PUSH && !LB && leaver) {
                const int back = bin_back(__shfl_sync(peers, lold, leader)) + __popc(peers & lt);
                if (back < p.cap) {
                    float *dst = p.out + dest * cstride + (p.cap - 1 - back);
#pragma unroll
                    for (int d = 0; d < DIM; ++d) __stcs(dst + (size_t)d * p.cap, o[d]);
#pragma unroll
                    for (int d = 0; d < 3; ++d) __stcs(dst + (size_t)(PF<DIM>::V + d) * p.cap, v[d]);
                    __stcs(dst + (size_t)PF<DIM>::W * p.cap, w);
                    if (p.nf > PF<DIM>::ID) __stcs(dst + (size_t)PF<DIM>::ID * p.cap, idb);
                } else {
                    atomicExch(&p.flags->overflow, 1);
                }
            }
            __syncwarp();                                    // the table is rewritten by the next chunk
        }
        if (n == 0 && has_next) fetch(bin_nx, wnext, 0);
        // the stayers' count (the bottom segment) of this cell's new bin
        if (PUSH && lane == 0 && fbase > 0) atomicAdd(p.cnt_out + cell, fbase);
        float *st = stage + (size_t)(it & (NST - 1)) * TILE;
        if (n > 0) {
            // the groups' sums: S[kg][pair class][column], this lane's 9 x 4 block
            if (role) {
                float *sd = T + (kg * G::ROWS + 9 * (lk / NQ)) * kCols + NCB * (lk % NQ);
#pragma unroll
                for (int ip = 0; ip < 4; ++ip)
#pragma unroll
                    for (int c = 0; c < NCB; ++c) {
                        sd[(2 * ip) * kCols + c] = accp[c][ip].x;
                        sd[(2 * ip + 1) * kCols + c] = accp[c][ip].y;
                    }
#pragma unroll
                for (int c = 0; c < NCB; ++c) sd[8 * kCols + c] = acc8[c];
            }
            __syncwarp();
            // totals over the groups, Gs[pair class][column], one column quad per lane and item
            float *Gs = T + G::KG * G::ROWS * kCols;
            for (int item = lane; item < G::ROWS * 4; item += 32) {
                const int j = item >> 2, q = item & 3;
                float4 s4 = *reinterpret_cast<const float4 *>(T + j * kCols + 4 * q);
#pragma unroll
                for (int g = 1; g < G::KG; ++g) {
                    const float4 u = *reinterpret_cast<const float4 *>(T + (g * G::ROWS + j) * kCols + 4 * q);
                    s4.x += u.x; s4.y += u.y; s4.z += u.z; s4.w += u.w;
                }
                *reinterpret_cast<float4 *>(Gs + j * kCols + 4 * q) = s4;
            }
            __syncwarp();
            for (int k = lane; k < R::SIZE; k += 32) st[k * kRecTile + warp] = record_value<DIM>(Gs, k);
        } else {
            for (int k = lane; k < R::SIZE; k += 32) st[k * kRecTile + warp] = 0.f;
        }
        // ---- the record blocks of the tiles staged since the last barrier: written whole
        // (or added, for the arrivals) after one CTA barrier
        if (it % TPB == TPB - 1 || t + gridDim.x >= ntiles) {
            __syncthreads();
            for (int h = it % TPB; h >= 0; --h) {
                const float4 *src = reinterpret_cast<const float4 *>(stage + (size_t)((it - h) & (NST - 1)) * TILE);
                float4 *dst = reinterpret_cast<float4 *>(p.rec + (size_t)(t - (int64_t)h * gridDim.x) * TILE);
                for (int i = threadIdx.x; i < TILE / 4; i += kThreads) {
                    const float4 v = src[i];
                    if (p.arrivals) {
                        if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) atomicAdd(dst + i, v);
                    } else {
                        dst[i] = v;
                    }
                }
            }
        }
        cell = ncell; ci = nci; cj = ncj; ck = nck;
        wcur = wnext;
        ccur = cnext;
    }
    if (PUSH && LB && lpend > 0) flush_leavers();
}

// ------------------------------------------------------------ arrivals deposit
// The particles that arrived in a cell during the push (the back segment of its
// new bin) are few, about the fraction of particles that cross a face in a step,
// so their deposit uses an entry-stationary scheme without a per-cell
// reduction: lane l owns the record entries k = l + 32 i, each a sum over the
// arrivals of a product a_k b_k of two per-particle factors (pair weight x
// alpha entry, or w W_a x (1, v_c, (alpha (v - u_ref))_c)).  The factors sit in
// a field-major table [field][particle], read as particle pairs: one packed FMA
// adds two particles' products.  A warp takes CPW consecutive cells at once: their
// arrivals share the 32-lane chunks, each cell's run padded to an even count
// (padding slots carry w = 0), so the factor pass and the per-cell set-up are
// spread over several cells' particles.  A CTA's 8 warps cover CPW record tiles,
// staged in shared memory and added to the records with 16-byte atomic adds.
template <int DIM> struct AF;   // factor table fields: pair weights, alpha, w W_a, v, alpha (v - u_ref), 1
template <> struct AF<2> { static constexpr int R = 0, AL = 9, WW = 18, V = 22, AD = 25, ONE = 28, NF = 29, E = 4, CPW = 4; };
template <> struct AF<3> { static constexpr int R = 0, AL = 27, WW = 36, V = 44, AD = 47, ONE = 50, NF = 51, E = 10, CPW = 2; };
// AF::CPW cells per warp on large grids; one on grids too small to fill the GPU that way
constexpr int kArrStride = 34;   // floats per table field: 32 particles + 2, which spreads the fields over the banks

// per warp: the CPW cells' coefficients [CPW][2 NC + 1] float4 (the +1 puts the cells
// in different banks), then the factor table
template <int DIM, int CPW>
__host__ __device__ constexpr int arr_cor_floats() { return CPW * (2 * Geo<DIM>::NC + 1) * 4; }
template <int DIM, int CPW>
__host__ __device__ constexpr int arr_warp_floats() {
    return arr_cor_floats<DIM, CPW>() + (AF<DIM>::NF * kArrStride + 3) / 4 * 4;
}
template <int DIM, int CPW>
constexpr size_t arr_smem_bytes() {
    return ((size_t)kWarpsPerCta * arr_warp_floats<DIM, CPW>() + 2 * (size_t)CPW * Rec<DIM>::SIZE * kRecTile) *
           sizeof(float);
}

// the two table fields whose product makes record entry k
template <int DIM>
__device__ __forceinline__ void arr_entry(int k, int &ia, int &ib) {
    using R = Rec<DIM>;
    using F = AF<DIM>;
    if (k >= R::M) {
        const int t = k - R::M, j = t / 9;
        ia = F::R + min(j, R::NPAIR - 1); ib = F::AL + t - 9 * j;
    } else if (k >= R::J) {
        const int t = k - R::J, a = t / 3;
        ia = F::WW + a; ib = F::AD + t - 3 * a;
    } else if (k >= R::MV) {
        const int t = k - R::MV, a = t / 3;
        ia = F::WW + a; ib = F::V + t - 3 * a;
    } else {
        ia = F::WW + k; ib = F::ONE;
    }
}

template <int DIM, int CPW>
__global__ void __launch_bounds__(kThreads, DIM == 2 ? 3 : 2) k_arr(const __grid_constant__ PD p) {
    using G = Geo<DIM>;
    using R = Rec<DIM>;
    using F = AF<DIM>;
    constexpr int NC = G::NC;
    constexpr int TILE = R::SIZE * kRecTile;
    constexpr int E = F::E;
    constexpr int SUP = kWarpsPerCta * CPW;                   // cells per CTA (CPW record tiles)
    static_assert(CPW * 2 * NC <= 32, "at most one corner value per lane");
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *ws = smem + (size_t)warp * arr_warp_floats<DIM, CPW>();
    float4 *cor = reinterpret_cast<float4 *>(ws);            // [CPW][2 NC + 1]: deposit B (beta / c), u_ref
    float *T = ws + arr_cor_floats<DIM, CPW>();               // [NF][kArrStride]
    float *stage = smem + (size_t)kWarpsPerCta * arr_warp_floats<DIM, CPW>();   // [2][CPW TILE]
    int oa[E], ob[E];                                         // table offsets of this lane's entries' factors
#pragma unroll
    for (int i = 0; i < E; ++i) {
        int a, b;
        arr_entry<DIM>(min(lane + 32 * i, R::SIZE - 1), a, b);
        oa[i] = a * kArrStride;
        ob[i] = b * kArrStride;
    }
    const int64_t nsup = (p.N + SUP - 1) / SUP;
    const int64_t ntiles = (p.N + kRecTile - 1) / kRecTile;
    const int64_t cstride = (int64_t)p.cap * p.nf;
    const unsigned nx = (unsigned)p.n[0], ny = (unsigned)p.n[1];
    // this lane's corner value: cell lc of the warp's CPW, array larr (0: B, 1: u_ref), corner la
    const int lc = lane / (2 * NC), larr = (lane / NC) & 1, la = lane % NC;
    const float lsc = larr == 0 ? p.bc : 1.f;

    int it = 0;
    for (int64_t st = blockIdx.x; st < nsup; st += gridDim.x, ++it) {
        const int64_t cell0 = st * SUP + (int64_t)warp * CPW;
        int nbl = 0;
        if (lane < CPW && cell0 + lane < p.N) nbl = bin_back(seg_word(__ldg(p.cnt_in + cell0 + lane), p.cap, 1));
        float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
        {
            const int64_t mc = cell0 + lc;
            if (lc < CPW && mc < p.N) {
                const unsigned u = (unsigned)mc;
                const int ci = (int)(u % nx), cj = (int)((u / nx) % ny), ck = (int)(u / nx / ny);
                const int64_t nd = node_of(p.n, ci + (la & 1), cj + ((la >> 1) & 1), ck + ((la >> 2) & 1));
                v4 = __ldg((larr == 0 ? p.dB : p.dU) + nd);
            }
        }
        // the cells' arrival counts and their even-padded offsets in the warp's chunk space
        int nb[CPW], ps[CPW + 1];
        ps[0] = 0;
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
            nb[c] = __shfl_sync(kFull, nbl, c);
            ps[c + 1] = ps[c] + ((nb[c] + 1) & ~1);
        }
        const int total = ps[CPW];
        float2 acc[CPW][E];
#pragma unroll
        for (int c = 0; c < CPW; ++c)
#pragma unroll
            for (int i = 0; i < E; ++i) acc[c][i] = make_float2(0.f, 0.f);
        if (total > 0) {
            __syncwarp();                                     // the previous cells' reads of cor are done
            v4.x *= lsc; v4.y *= lsc; v4.z *= lsc;
            v4 = to_coef<DIM>(v4, la);
            if (lc < CPW) cor[lc * (2 * NC + 1) + larr * NC + la] = v4;
            __syncwarp();
        }
        for (int c0 = 0; c0 < total; c0 += 32) {
            // ---- this lane's slot: cell c, arrival j (or padding)
            const int g = c0 + lane;
            int c = 0;
#pragma unroll
            for (int cc = 1; cc < CPW; ++cc) c = g >= ps[cc] ? cc : c;
            int nbc = nb[0], psc = ps[0];
#pragma unroll
            for (int cc = 1; cc < CPW; ++cc)
                if (c == cc) { nbc = nb[cc]; psc = ps[cc]; }
            const int j = g - psc;
            const bool valid = g < total && j < nbc;
            float o[3] = {0.5f, 0.5f, 0.f}, v[3] = {0.f, 0.f, 0.f}, w = 0.f;
            if (valid) {
                const float *q = p.in + (cell0 + c) * cstride + (p.cap - nbc + j);
#pragma unroll
                for (int d = 0; d < DIM; ++d) o[d] = __ldcs(q + (size_t)d * p.cap);
#pragma unroll
                for (int d = 0; d < 3; ++d) v[d] = __ldcs(q + (size_t)(PF<DIM>::V + d) * p.cap);
                w = __ldcs(q + (size_t)PF<DIM>::W * p.cap);
            }
            // ---- this lane's factors into column `lane` of the table
            {
                const float4 *cc4 = cor + c * (2 * NC + 1);
                float b3[3], U3[3], al[9], W[NC];
                interp<DIM>(cc4, o, b3);
                interp<DIM>(cc4 + NC, o, U3);
                alpha_tensor(b3[0], b3[1], b3[2], al);
                corner_weights<DIM>(o, W);
                const float d0 = v[0] - U3[0], d1 = v[1] - U3[1], d2 = v[2] - U3[2];
                float X[3][3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float a0 = 1.f - o[d];
                    X[d][0] = a0 * a0; X[d][1] = a0 * o[d]; X[d][2] = o[d] * o[d];
                }
                float *tc = T + lane;
#pragma unroll
                for (int jz = 0; jz < (DIM == 3 ? 3 : 1); ++jz)
#pragma unroll
                    for (int jy = 0; jy < 3; ++jy) {
                        const float wyz = DIM == 3 ? w * X[1][jy] * X[2][jz] : w * X[1][jy];
#pragma unroll
                        for (int jx = 0; jx < 3; ++jx) tc[(F::R + jx + 3 * jy + 9 * jz) * kArrStride] = wyz * X[0][jx];
                    }
#pragma unroll
                for (int e = 0; e < 9; ++e) tc[(F::AL + e) * kArrStride] = al[e];
#pragma unroll
                for (int a = 0; a < NC; ++a) tc[(F::WW + a) * kArrStride] = w * W[a];
#pragma unroll
                for (int d = 0; d < 3; ++d) tc[(F::V + d) * kArrStride] = v[d];
                tc[(F::AD + 0) * kArrStride] = fmaf(al[0], d0, fmaf(al[1], d1, al[2] * d2));
                tc[(F::AD + 1) * kArrStride] = fmaf(al[3], d0, fmaf(al[4], d1, al[5] * d2));
                tc[(F::AD + 2) * kArrStride] = fmaf(al[6], d0, fmaf(al[7], d1, al[8] * d2));
                tc[F::ONE * kArrStride] = 1.f;
            }
            __syncwarp();
            // ---- every cell's entries over its (even-aligned) slots of this chunk
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) {
                const int lo = max(ps[cc], c0), hi = min(ps[cc + 1], c0 + 32);
                for (int pp = lo - c0; pp < hi - c0; pp += 2) {
#pragma unroll
                    for (int i = 0; i < E; ++i) {
                        const float2 a2 = *reinterpret_cast<const float2 *>(T + oa[i] + pp);
                        const float2 b2 = *reinterpret_cast<const float2 *>(T + ob[i] + pp);
                        acc[cc][i] = __ffma2_rn(a2, b2, acc[cc][i]);
                    }
                }
            }
            __syncwarp();                                    // the table is rewritten by the next chunk
        }
        // ---- the cells' records into the stage, then the CTA's record tiles
        float *stg = stage + (size_t)(it & 1) * CPW * TILE;
#pragma unroll
        for (int cc = 0; cc < CPW; ++cc) {
            const int sc = warp * CPW + cc;
            float *dstc = stg + (sc / kRecTile) * TILE + sc % kRecTile;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int k = lane + 32 * i;
                if (k < R::SIZE) dstc[k * kRecTile] = k < R::USED ? acc[cc][i].x + acc[cc][i].y : 0.f;
            }
        }
        __syncthreads();
        {
            const float4 *src = reinterpret_cast<const float4 *>(stg);
            float4 *dst = reinterpret_cast<float4 *>(p.rec + (size_t)st * CPW * TILE);
            for (int i = threadIdx.x; i < CPW * TILE / 4; i += kThreads) {
                if (st * CPW + (4 * i) / TILE >= ntiles) break;   // record tiles past the grid
                const float4 vv = src[i];
                if (vv.x != 0.f || vv.y != 0.f || vv.z != 0.f || vv.w != 0.f) atomicAdd(dst + i, vv);
            }
        }
    }
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
// (step, cell, k, 0); offsets in the cell from the top 24 bits of words 0 and 1
// (and, along a resolved z, bits 16..39 of word 0), three normals by the
// Box-Muller transform of 24-bit uniforms of words 2 and 3; v = u + vth n.
// Step 0 is the device-side initialisation, steps >= 1 the boundary refill
// after each push.
__device__ __forceinline__ void draw_particle(uint64_t seed, int species, uint64_t step, int64_t cell, int k, int ny,
                                              int nz, float ux, float uy, float uz, float vth, float o[3], float v[3]) {
    uint64_t x[4] = {step, (uint64_t)cell, (uint64_t)k, 0ull};
    philox4x64(seed, (uint64_t)species, x);
    const float s24 = 1.0f / 16777216.0f;
    o[0] = (float)(x[0] >> 40) * s24;
    o[1] = ny > 1 ? (float)(x[1] >> 40) * s24 : 0.f;
    o[2] = nz > 1 ? (float)((x[0] >> 16) & 0xffffffu) * s24 : 0.f;
    const float u1 = (float)((x[2] >> 40) + 1) * s24, u2 = (float)((x[2] >> 16) & 0xffffffu) * s24;
    const float u3 = (float)((x[3] >> 40) + 1) * s24, u4 = (float)((x[3] >> 16) & 0xffffffu) * s24;
    const float ra = sqrtf(-2.f * logf(u1)), rb = sqrtf(-2.f * logf(u3));
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    v[0] = ux + vth * ra * cs;
    v[1] = uy + vth * ra * sn;
    v[2] = uz + vth * rb * cospif(2.f * u4);
}

// store particle (o, v, w, id) in slot `slot` of cell `cell`
template <int DIM>
__device__ __forceinline__ void put_particle(float *bins, int cap, int nf, int64_t cell, int slot, const float o[3],
                                             const float v[3], float w, float idb) {
    float *q = bins + (size_t)cell * cap * nf + slot;
#pragma unroll
    for (int d = 0; d < DIM; ++d) q[(size_t)d * cap] = o[d];
#pragma unroll
    for (int d = 0; d < 3; ++d) q[(size_t)(PF<DIM>::V + d) * cap] = v[d];
    q[(size_t)PF<DIM>::W * cap] = w;
    if (nf > PF<DIM>::ID) q[(size_t)PF<DIM>::ID * cap] = idb;
}

// Device-side drifting Maxwellian species: ppc draws of step 0 in every cell,
// written straight into the cell's bin (one CTA per cell).
template <int DIM>
__global__ void k_maxwellian(int ny, int nz, int64_t N, int cap, int nf, int ppc, uint64_t seed, int species,
                             float ux, float uy, float uz, float vth, float w, float *bins, int *cnt) {
    for (int64_t cell = blockIdx.x; cell < N; cell += gridDim.x) {
        for (int k = threadIdx.x; k < ppc; k += blockDim.x) {
            float o[3], v[3];
            draw_particle(seed, species, 0ull, cell, k, ny, nz, ux, uy, uz, vth, o, v);
            put_particle<DIM>(bins, cap, nf, cell, k, o, v, w, __int_as_float((int)(cell * ppc + k)));
        }
        if (threadIdx.x == 0) cnt[cell] = ppc;
    }
}

// The 109 sums of the 2D record held per thread (register accumulation; used by
// the boundary refill, whose few particles per cell are spread over a CTA)
struct RegAcc {
    float v[Rec<2>::SIZE];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < Rec<2>::SIZE; ++k) v[k] = 0.f;
    }
};

// the 2D record sums of one particle at offsets (x, y) with corner values of
// B (for alpha) and u_ref, in the layout Rec<2>
__device__ __forceinline__ void deposit_one(RegAcc &acc, float x, float y, float vx, float vy, float vz, float w,
                                            const float4 cB[4], const float4 cU[4], float bc) {
    const float o[3] = {x, y, 0.f};
    float W[4], B3[3], U3[3], al[9];
    corner_weights<2>(o, W);
    gather<2>(cB, W, B3);
    gather<2>(cU, W, U3);
    alpha_tensor(bc * B3[0], bc * B3[1], bc * B3[2], al);
    const float d[3] = {vx - U3[0], vy - U3[1], vz - U3[2]};
    const float vv[3] = {vx, vy, vz};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        acc.v[Rec<2>::RHO + a] = fmaf(w, W[a], acc.v[Rec<2>::RHO + a]);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float jr = fmaf(al[3 * r], d[0], fmaf(al[3 * r + 1], d[1], al[3 * r + 2] * d[2]));
            acc.v[Rec<2>::MV + 3 * a + r] = fmaf(w * vv[r], W[a], acc.v[Rec<2>::MV + 3 * a + r]);
            acc.v[Rec<2>::J + 3 * a + r] = fmaf(w * jr, W[a], acc.v[Rec<2>::J + 3 * a + r]);
        }
    }
    const float X[3] = {w * (1.f - x) * (1.f - x), w * x * (1.f - x), w * x * x};
    const float Y[3] = {(1.f - y) * (1.f - y), y * (1.f - y), y * y};
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const float pw = X[j % 3] * Y[j / 3];
#pragma unroll
        for (int e = 0; e < 9; ++e) acc.v[Rec<2>::M + 9 * j + e] = fmaf(pw, al[e], acc.v[Rec<2>::M + 9 * j + e]);
    }
}

struct BcArgs {
    int nx, ny, G, cap, nf;
    int64_t N;
    uint64_t seed, step;
    int species, track;
    float bc;                    // beta / c of the species (alpha)
    int nsides;                  // 2, or 1 with a reflecting wall on the high side (no refill there)
    int ppc[2];                  // per side (0: low x, 1: high x)
    float w[2], vth[2], u[2][3];
    float *bins;                 // the current copy (after the push)
    int *cnt;
    float *rec;                  // the species' tile-major records (rec_index)
    const float4 *dB, *dU;       // node B^{n+1} and u_ref of the deposit
};

// One CTA per boundary cell: replace its particles by the side's fresh draws
// (key (seed, species), counter (step, cell, k, 0)), deposit them with the
// deposit's arithmetic and overwrite the cell's record and count (2D).
__global__ void __launch_bounds__(128) k_bc_refill(BcArgs a) {
    __shared__ float red[4][Rec<2>::SIZE];
    const int t = blockIdx.x, G2c = a.nsides * a.G;
    const int j = t / G2c, r = t % G2c;
    const int side = r < a.G ? 0 : 1;
    const int i = r < a.G ? r : a.nx - G2c + r;
    const int64_t cell = (int64_t)j * a.nx + i;
    const int n3[3] = {a.nx, a.ny, 1};
    float4 cB[4], cU[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int64_t nd = node_of(n3, i + (c & 1), j + (c >> 1), 0);
        cB[c] = a.dB[nd];
        cU[c] = a.dU[nd];
    }
    const int ppc = a.ppc[side];
    const float w = a.w[side], vth = a.vth[side];
    RegAcc acc;
    acc.zero();
    for (int k = threadIdx.x; k < ppc; k += blockDim.x) {
        float o[3], v[3];
        draw_particle(a.seed, a.species, a.step, cell, k, a.ny, 1, a.u[side][0], a.u[side][1], a.u[side][2], vth, o, v);
        put_particle<2>(a.bins, a.cap, a.nf, cell, k, o, v, w, __int_as_float(a.track ? -1 : 0));
        deposit_one(acc, o[0], o[1], v[0], v[1], v[2], w, cB, cU, a.bc);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < Rec<2>::SIZE; ++k) {
        float v = acc.v[k];
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(kFull, v, m);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < Rec<2>::SIZE; k += blockDim.x)
        a.rec[rec_index(Rec<2>::SIZE, k, cell)] = (red[0][k] + red[1][k]) + (red[2][k] + red[3][k]);
    if (threadIdx.x == 0) a.cnt[cell] = ppc;          // front segment only
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
__device__ __forceinline__ int cell_along(double pos, double inv_dx, int n, float &off) {
    if (n == 1) { off = 0.f; return 0; }
    const double sx = pos * inv_dx, fx = floor(sx);
    const long long lx = (long long)fx;
    int cx = (lx >= 0 && lx < n) ? (int)lx : (int)(((lx % n) + n) % n);   // inside the box: no division
    off = (float)(sx - fx);
    if (off >= 1.f) { off = 0.f; cx = wrap_idx(cx + 1, n); }
    return cx;
}

__global__ void k_locate(int64_t n, const double *x, const double *y, const double *z, int nx, int ny, int nz,
                         double idx, double idy, double idz, int64_t *cell, float *ox, float *oy, float *oz,
                         int *count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float fx, fy, fz;
        const int cx = cell_along(x[i], idx, nx, fx);
        const int cy = cell_along(ny > 1 ? y[i] : 0.0, idy, ny, fy);
        const int cz = cell_along(nz > 1 ? z[i] : 0.0, idz, nz, fz);
        const int64_t c = cx + (int64_t)nx * (cy + (int64_t)ny * cz);
        cell[i] = c;
        ox[i] = fx;
        oy[i] = fy;
        oz[i] = fz;
        atomicAdd(&count[c], 1);
    }
}

template <int DIM>
__global__ void k_scatter(int64_t n, const int64_t *cell, const float *ox, const float *oy, const float *oz,
                          const float *vx, const float *vy, const float *vz, const float *w, const int32_t *id,
                          int cap, int nf, int *cursor, float *out, DevFlags *f) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = cell[i];
        const int slot = atomicAdd(&cursor[c], 1);
        if (slot >= cap) { atomicExch(&f->overflow, 1); continue; }
        const int idv = id ? id[i] : (int32_t)i;
        const float o[3] = {ox[i], oy[i], oz[i]}, v[3] = {vx[i], vy[i], vz[i]};
        put_particle<DIM>(out, cap, nf, c, slot, o, v, w[i], __int_as_float(idv));
    }
}

// copy bins into bins of a new capacity (both segments into the new front)
__global__ void k_rebin_copy(int64_t ncell, int oldcap, int newcap, int nf, const int *cnt, int *newcnt,
                             const float *src, float *dst) {
    const int64_t c = blockIdx.x;
    if (c >= ncell) return;
    const int word = clamp_word(cnt[c], oldcap);
    const int m = min(bin_count(word), newcap);
    const float *s = src + (size_t)c * oldcap * nf;
    float *d = dst + (size_t)c * newcap * nf;
    for (int t = threadIdx.x; t < m * nf; t += blockDim.x) {
        const int f = t / m, i = t % m;
        d[(size_t)f * newcap + i] = s[(size_t)f * oldcap + bin_slot(word, i, oldcap)];
    }
    if (threadIdx.x == 0) newcnt[c] = m;
}

template <int DIM>
__global__ void k_gather_out(int64_t ncell, int cap, int nf, const int *cnt, const int *offs, const float *src,
                             int nx, int ny, double dx, double dy, double dz, double *x, double *y, double *z,
                             float *vx, float *vy, float *vz, float *w, int32_t *id) {
    const int64_t c = blockIdx.x;
    if (c >= ncell) return;
    const int word = clamp_word(cnt[c], cap);
    const int m = bin_count(word);
    const int cx = (int)(c % nx), cy = (int)((c / nx) % ny), cz = (int)(c / ((int64_t)nx * ny));
    const float *b = src + (size_t)c * cap * nf;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const float *q = b + bin_slot(word, i, cap);
        const int o = offs[c] + i;
        if (x) x[o] = (cx + (double)q[0]) * dx;
        if (y) y[o] = ny > 1 ? (cy + (double)q[(size_t)cap]) * dy : 0.0;
        if (z) z[o] = DIM == 3 ? (cz + (double)q[(size_t)2 * cap]) * dz : 0.0;
        if (vx) vx[o] = q[(size_t)PF<DIM>::V * cap];
        if (vy) vy[o] = q[(size_t)(PF<DIM>::V + 1) * cap];
        if (vz) vz[o] = q[(size_t)(PF<DIM>::V + 2) * cap];
        if (w) w[o] = q[(size_t)PF<DIM>::W * cap];
        if (id) id[o] = __float_as_int(q[(size_t)PF<DIM>::ID * cap]);
    }
}

int grid_for(int64_t n, int block = 256) {
    int64_t g = (n + block - 1) / block;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

int alloc_bins(gx_ctx *c, int s, int cap) {
    Species &S = c->sp[s];
    S.nf = c->dim + 4 + (c->cfg.track_ids ? 1 : 0);
    const size_t nfl = (size_t)c->N * cap * S.nf;
    for (int b = 0; b < 2; ++b) {
        S.p[b] = nullptr;
        GX_CHECK(c, cudaMalloc(&S.p[b], nfl * sizeof(float)));
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

// bin capacity: a multiple of 32 (a warp's chunk of the front segment is one
// aligned line per field) and below 2^15 (the packed count word)
int round_cap(double v) {
    int cap = (int)ceil(v);
    cap = (cap + 31) / 32 * 32;
    return cap < 32 ? 32 : cap;
}

template <int DIM>
int configure_pd(gx_ctx *c) {
    static bool done = false;
    if (done) return GX_OK;
    const int sm = (int)pd_smem_bytes<DIM>();
    GX_CHECK(c, cudaFuncSetAttribute(k_pd<DIM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    GX_CHECK(c, cudaFuncSetAttribute(k_pd<DIM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    if constexpr (DIM == 2)
        GX_CHECK(c, cudaFuncSetAttribute(k_pd<DIM, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    GX_CHECK(c, cudaFuncSetAttribute(k_arr<DIM, AF<DIM>::CPW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)arr_smem_bytes<DIM, AF<DIM>::CPW>()));
    GX_CHECK(c, cudaFuncSetAttribute(k_arr<DIM, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)arr_smem_bytes<DIM, 1>()));
    done = true;
    return GX_OK;
}

// persistent grid: as many CTAs as fit on the device at once
template <int DIM>
int pd_grid(gx_ctx *c, int64_t ncell) {
    static int per_sm = 0;
    if (!per_sm) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pd<DIM, true>, kThreads, pd_smem_bytes<DIM>()) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (ncell + kWarpsPerCta - 1) / kWarpsPerCta;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)nsm * per_sm));
}

// the arrivals deposit: AF::CPW cells per warp where that still gives every CTA slot
// of the GPU at least two CTAs' work, else one; a persistent grid
template <int DIM, int CPW>
int arr_slots() {
    static int per_sm = 0;
    if (!per_sm) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arr<DIM, CPW>, kThreads,
                                                          arr_smem_bytes<DIM, CPW>()) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm * per_sm;
}
template <int DIM>
void launch_arr(const PD &q, int64_t ncell, cudaStream_t st) {
    constexpr int CPW = AF<DIM>::CPW;
    const int64_t big = (ncell + kWarpsPerCta * CPW - 1) / (kWarpsPerCta * CPW);
    const int slots = arr_slots<DIM, CPW>();
    if (big >= 2 * (int64_t)slots) {
        k_arr<DIM, CPW><<<(unsigned)std::min<int64_t>(big, slots), kThreads, arr_smem_bytes<DIM, CPW>(), st>>>(q);
    } else {
        const int64_t one = (ncell + kWarpsPerCta - 1) / kWarpsPerCta;
        const int s1 = arr_slots<DIM, 1>();
        k_arr<DIM, 1><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(one, s1)), kThreads, arr_smem_bytes<DIM, 1>(),
                        st>>>(q);
    }
}

template <int DIM>
int launch_pd(gx_ctx *c, bool push, cudaStream_t st) {
    int rc = configure_pd<DIM>(c);
    if (rc) return rc;
    const int grid = pd_grid<DIM>(c, c->N);
    const size_t smem = pd_smem_bytes<DIM>();
    const int nxt = 1 - c->cur;
    for (int s = 0; s < c->nspecies; ++s) {
        Species &S = c->sp[s];
        PD p{};
        for (int d = 0; d < 3; ++d) {
            p.n[d] = c->n[d];
            p.dtd[d] = (float)(c->cfg.dt / c->cfg.dx[d]);
        }
        p.N = c->N;
        p.cap = S.cap;
        p.nf = S.nf;
        const double beta = S.q * c->cfg.dt / (2.0 * S.m);
        p.beta = (float)beta;
        p.bc = (float)(beta / c->cfg.c);
        p.in = S.p[c->cur];
        p.out = S.p[nxt];
        p.cnt_in = S.cnt[c->cur];
        p.cnt_out = S.cnt[nxt];
        p.rec = c->rec + (size_t)s * rec_block(c->rec_size, c->N);
        p.flags = c->dflags;
        p.wall_ci = (c->cfg.bc_cells > 0 && c->cfg.bc_wall) ? c->n[0] - c->cfg.bc_cells - 1 : -1;
        if (push && c->cfg.gl_gamma > 0) {
            // eps = 1 / (Q2 sum_d 4 / dx_d^2), Q2 = sum_p (q_s w_p)^2 / V
            double Q2 = 0.0, lap = 0.0;
            for (int t = 0; t < c->nspecies; ++t) Q2 += c->sp[t].q * c->sp[t].q * c->sp[t].w2;
            Q2 /= (double)c->N * c->dV;
            for (int d = 0; d < 3; ++d)
                if (c->n[d] > 1) lap += 4.0 / (c->cfg.dx[d] * c->cfg.dx[d]);
            const double eps = (Q2 > 0 && lap > 0) ? 1.0 / (Q2 * lap) : 0.0;
            p.glon = eps > 0;
            for (int d = 0; d < 3; ++d)
                p.gl[d] = c->n[d] > 1 ? (float)(c->cfg.gl_gamma * eps * S.q / (c->cfg.dx[d] * c->cfg.dx[d])) : 0.f;
        }
        if (push) {
            p.mE = c->nE; p.mB = c->nB; p.dB = c->nBnext; p.dU = c->nUref;
            GX_CHECK(c, cudaMemsetAsync(S.cnt[nxt], 0, c->N * sizeof(int), st));
            cudaEvent_t e0 = gx_ev_get(c), e1 = gx_ev_get(c);
            GX_CHECK(c, cudaEventRecord(e0, st));
            if constexpr (DIM == 2) {
                if (p.wall_ci >= 0) k_pd<DIM, true, true><<<grid, kThreads, smem, st>>>(p);
                else k_pd<DIM, true><<<grid, kThreads, smem, st>>>(p);
            } else {
                k_pd<DIM, true><<<grid, kThreads, smem, st>>>(p);
            }
            GX_LAUNCHED(c);
            GX_CHECK(c, cudaEventRecord(e1, st));
            gx_ev_push(c, GX_T_PDK, e0, e1);
            c->n_pdk++;
            // the particles that arrived in each cell: the same deposit over the
            // back segments of the new bins, added to the records the push just wrote
            PD q = p;
            q.arrivals = 1;
            q.in = p.out;
            q.cnt_in = p.cnt_out;
            q.mE = nullptr; q.mB = nullptr;
            launch_arr<DIM>(q, c->N, st);
            GX_LAUNCHED(c);
            if (DIM == 2 && c->cfg.bc_cells > 0) {
                // open boundaries: the boundary cells' particles are replaced
                BcArgs b{};
                b.nx = c->n[0]; b.ny = c->n[1]; b.G = c->cfg.bc_cells; b.cap = S.cap; b.nf = S.nf; b.N = c->N;
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
            k_pd<DIM, false><<<grid, kThreads, smem, st>>>(p);
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

}  // namespace

// --------------------------------------------------------------- binning
int gx_bin_particles(gx_ctx *c, int s, int64_t n, const double *x, const double *y, const double *z,
                     const float *vx, const float *vy, const float *vz, const float *w, const int32_t *id,
                     cudaStream_t st) {
    Species &S = c->sp[s];
    int64_t *cell = nullptr;
    int *count = nullptr;
    float *ox = nullptr, *oy = nullptr, *oz = nullptr;
    GX_CHECK(c, cudaMalloc(&cell, (n + 1) * sizeof(int64_t)));
    GX_CHECK(c, cudaMalloc(&ox, (n + 1) * sizeof(float)));
    GX_CHECK(c, cudaMalloc(&oy, (n + 1) * sizeof(float)));
    GX_CHECK(c, cudaMalloc(&oz, (n + 1) * sizeof(float)));
    GX_CHECK(c, cudaMalloc(&count, c->N * sizeof(int)));
    GX_CHECK(c, cudaMemsetAsync(count, 0, c->N * sizeof(int), st));
    if (n > 0) {
        k_locate<<<grid_for(n), 256, 0, st>>>(n, x, y, z, c->n[0], c->n[1], c->n[2], 1.0 / c->cfg.dx[0],
                                               1.0 / c->cfg.dx[1], 1.0 / c->cfg.dx[2], cell, ox, oy, oz, count);
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
    const int cap = round_cap(std::max(32.0, hf.maxcount * slack));
    GX_CHECK(c, cudaFree(dmax));
    if (cap >= 32768) { c->err = "more than 32767 particles per cell bin"; return GX_EINVAL; }
    int rc = alloc_bins(c, s, cap);
    if (rc) return rc;
    GX_CHECK(c, cudaMemsetAsync(S.cnt[c->cur], 0, c->N * sizeof(int), st));
    if (n > 0) {
        if (c->dim == 3)
            k_scatter<3><<<grid_for(n), 256, 0, st>>>(n, cell, ox, oy, oz, vx, vy, vz, w, id, cap, S.nf,
                                                      S.cnt[c->cur], S.p[c->cur], c->dflags);
        else
            k_scatter<2><<<grid_for(n), 256, 0, st>>>(n, cell, ox, oy, oz, vx, vy, vz, w, id, cap, S.nf,
                                                      S.cnt[c->cur], S.p[c->cur], c->dflags);
        GX_LAUNCHED(c);
    }
    GX_CHECK(c, cudaStreamSynchronize(st));
    cudaFree(cell); cudaFree(ox); cudaFree(oy); cudaFree(oz); cudaFree(count);
    return GX_OK;
}

int gx_species_maxwellian_init(gx_ctx *c, int s, int ppc, double n0, const double u[3], double vth,
                               cudaStream_t st) {
    const double slack = c->cfg.bin_slack > 1.2 ? c->cfg.bin_slack : 1.2;
    const int cap = round_cap(std::max(32.0, ppc * slack));
    if (cap >= 32768) { c->err = "more than 32767 particles per cell bin"; return GX_EINVAL; }
    int rc = alloc_bins(c, s, cap);
    if (rc) return rc;
    const double dV = c->cfg.dx[0] * c->cfg.dx[1] * c->cfg.dx[2];
    const unsigned grid = (unsigned)std::min<int64_t>(c->N, 152 * 64);
    const float wgt = (float)(n0 * dV / ppc);
    Species &S = c->sp[s];
    if (c->dim == 3)
        k_maxwellian<3><<<grid, 128, 0, st>>>(c->n[1], c->n[2], c->N, cap, S.nf, ppc, c->cfg.seed, s, (float)u[0],
                                              (float)u[1], (float)u[2], (float)vth, wgt, S.p[c->cur], S.cnt[c->cur]);
    else
        k_maxwellian<2><<<grid, 128, 0, st>>>(c->n[1], 1, c->N, cap, S.nf, ppc, c->cfg.seed, s, (float)u[0],
                                              (float)u[1], (float)u[2], (float)vth, wgt, S.p[c->cur], S.cnt[c->cur]);
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
    k_rebin_copy<<<(unsigned)c->N, 128, 0, st>>>(c->N, old.cap, newcap, S.nf, old.cnt[c->cur], S.cnt[c->cur],
                                                  old.p[c->cur], S.p[c->cur]);
    GX_LAUNCHED(c);
    GX_CHECK(c, cudaStreamSynchronize(st));
    free_bins(old);
    return GX_OK;
}

// ------------------------------------------------------------ hot path
int gx_run_deposit(gx_ctx *c, cudaStream_t st) {
    return c->dim == 3 ? launch_pd<3>(c, false, st) : launch_pd<2>(c, false, st);
}
int gx_run_push_deposit(gx_ctx *c, cudaStream_t st) {
    return c->dim == 3 ? launch_pd<3>(c, true, st) : launch_pd<2>(c, true, st);
}

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
    if (c->dim == 3)
        k_gather_out<3><<<(unsigned)c->N, 128, 0, st>>>(c->N, S.cap, S.nf, S.cnt[c->cur], offs, S.p[c->cur], c->n[0],
                                                        c->n[1], c->cfg.dx[0], c->cfg.dx[1], c->cfg.dx[2], x, y, z, vx,
                                                        vy, vz, w, id);
    else
        k_gather_out<2><<<(unsigned)c->N, 128, 0, st>>>(c->N, S.cap, S.nf, S.cnt[c->cur], offs, S.p[c->cur], c->n[0],
                                                        c->n[1], c->cfg.dx[0], c->cfg.dx[1], c->cfg.dx[2], x, y, z, vx,
                                                        vy, vz, w, id);
    GX_LAUNCHED(c);
    GX_CHECK(c, cudaStreamSynchronize(st));
    cudaFree(offs); cudaFree(counts); cudaFree(tmp);
    return GX_OK;
}

void gx_free_bins(gx_ctx *c) {
    for (int s = 0; s < c->nspecies; ++s) free_bins(c->sp[s]);
}
