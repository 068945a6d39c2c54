// gx_noalloc.cu -- particle gather that allocates no memory.
//
// gx_get_particles sizes its scratch (per-cell counts and offsets, the scan's
// temporary storage) to the grid and allocates it on every call.  Some callers cannot allocate at that point: a diagnostics or
// checkpoint hook running while the particle arrays already fill the device,
// a code path that must not synchronise the device (cudaMalloc and cudaFree
// can), or a host thread that holds a memory budget of its own.  This variant
// keeps its only scratch, the per-cell output offsets, in a fixed file-scope
// device array, so it calls no allocating routine of CUDA, of a library or of
// PyTorch.
//
// Limits and rules:
//   * at most kMaxCells cells (the scratch holds one int per cell, 1 MiB);
//     larger grids get GX_EINVAL;
//   * the scratch address is looked up with cudaGetSymbolAddress once per
//     device, with that device current, and the module holding the scratch and
//     the two kernels is loaded, when gx_create makes a context on the device
//     (gx_noalloc_prepare): CUDA loads modules lazily, and loading one
//     allocates device memory and can synchronise, so this happens at context
//     creation and never inside gx_get_particles_noalloc;
//   * the scratch is shared by every context on the device: calls that overlap
//     in time (two streams, two host threads) race on it;
//   * every offset the gather reads is written by the scan of the same call,
//     so nothing has to be cleared between calls.
#include <mutex>

#include "gx_internal.cuh"

namespace {

constexpr int kMaxCells = 1 << 18;
constexpr int kMaxDevices = 64;
constexpr int kScanThreads = 1024;

__device__ __align__(256) int g_offs[kMaxCells];

std::mutex g_mu;
int *g_ptr[kMaxDevices] = {};

__device__ __forceinline__ int na_count(int w, int cap) {
    // occupancy of a bin word clipped to the capacity (a bin that overflowed
    // holds at most cap particles)
    int f = bin_front(w), b = bin_back(w);
    b = min(b, cap);
    f = min(f, cap - b);
    return f + b;
}

// exclusive prefix sum of the per-cell counts into offs, one CTA
__global__ void __launch_bounds__(kScanThreads) k_na_scan(const int *__restrict__ cnt, int n, int cap, int *offs) {
    __shared__ int warp_tot[kScanThreads / 32];
    const int per = (n + kScanThreads - 1) / kScanThreads;
    const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += na_count(cnt[i], cap);
    // inclusive scan of the thread sums: within the warp, then across warps
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int v = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int t = warp_tot[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    int base = v - s + (warp > 0 ? warp_tot[warp - 1] : 0);
    for (int i = lo; i < hi; ++i) {
        offs[i] = base;
        base += na_count(cnt[i], cap);
    }
}

// one CTA per cell: copy the cell's particles (front segment, then back) to
// positions offs[c] .. offs[c] + count - 1; a bin holds nf fields of cap slots
// each, (o_0 .. o_{dim-1}, v_x, v_y, v_z, w, id)
__global__ void k_na_gather(int64_t ncell, int cap, int nf, int dim, const int *__restrict__ cnt,
                            const int *__restrict__ offs, const float *__restrict__ P, int nx, int ny, double dx,
                            double dy, double dz, double *x, double *y, double *z, float *vx, float *vy, float *vz,
                            float *w, int32_t *id) {
    const int64_t c = blockIdx.x;
    if (c >= ncell) return;
    const int word = cnt[c];
    int f = bin_front(word), b = bin_back(word);
    b = min(b, cap);
    f = min(f, cap - b);
    const int m = f + b;
    const int cx = (int)(c % nx), cy = (int)((c / nx) % ny), cz = (int)(c / ((int64_t)nx * ny));
    const float *bin = P + (size_t)c * cap * nf;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const float *q = bin + (i < f ? i : cap - b + (i - f));
        const int o = offs[c] + i;
        if (x) x[o] = (cx + (double)q[0]) * dx;
        if (y) y[o] = ny > 1 ? (cy + (double)q[(size_t)cap]) * dy : 0.0;
        if (z) z[o] = dim == 3 ? (cz + (double)q[(size_t)2 * cap]) * dz : 0.0;
        if (vx) vx[o] = q[(size_t)dim * cap];
        if (vy) vy[o] = q[(size_t)(dim + 1) * cap];
        if (vz) vz[o] = q[(size_t)(dim + 2) * cap];
        if (w) w[o] = q[(size_t)(dim + 3) * cap];
        if (id) id[o] = __float_as_int(q[(size_t)(dim + 4) * cap]);
    }
}

// address of this device's scratch, looked up on the first call per device
int scratch_for_current_device(gx_ctx *c, int **out) {
    int dev = -1;
    GX_CHECK(c, cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        c->err = "gx_get_particles_noalloc: device ordinal out of range";
        return GX_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_offs);
        if (e != cudaSuccess || !p) {
            c->err = std::string("gx_get_particles_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return GX_ECUDA;
        }
        g_ptr[dev] = static_cast<int *>(p);
    }
    *out = g_ptr[dev];
    return GX_OK;
}

}  // namespace

// Called by gx_create with the context's device current: look the scratch up
// and load the module of this file (its kernels) now, so that the gather
// itself never triggers a lazy module load.
int gx_noalloc_prepare(gx_ctx *c) {
    int *p = nullptr;
    int rc = scratch_for_current_device(c, &p);
    if (rc) return rc;
    cudaFuncAttributes fa;
    GX_CHECK(c, cudaFuncGetAttributes(&fa, k_na_scan));
    GX_CHECK(c, cudaFuncGetAttributes(&fa, k_na_gather));
    return GX_OK;
}

extern "C" int gx_noalloc_max_cells(void) { return kMaxCells; }

extern "C" int gx_get_particles_noalloc(gx_ctx *c, int s, double *x, double *y, double *z, float *vx, float *vy,
                                        float *vz, float *w, int32_t *id, void *stream) {
    if (!c) return GX_EINVAL;
    if (s < 0 || s >= c->nspecies) { c->err = "gx_get_particles_noalloc: bad species"; return GX_EINVAL; }
    if (id && !c->cfg.track_ids) { c->err = "ids need track_ids"; return GX_EINVAL; }
    if (c->N > kMaxCells) {
        c->err = "gx_get_particles_noalloc: the grid has " + std::to_string(c->N) + " cells, more than the " +
                 std::to_string(kMaxCells) + " its fixed scratch holds";
        return GX_EINVAL;
    }
    int *offs = nullptr;
    int rc = scratch_for_current_device(c, &offs);   // set up by gx_create: a table lookup here
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const Species &S = c->sp[s];
    const int *cnt = S.cnt[c->cur];
    k_na_scan<<<1, kScanThreads, 0, st>>>(cnt, (int)c->N, S.cap, offs);
    GX_LAUNCHED(c);
    k_na_gather<<<(unsigned)c->N, 128, 0, st>>>(c->N, S.cap, S.nf, c->dim, cnt, offs, S.p[c->cur], c->n[0],
                                                c->n[1], c->cfg.dx[0], c->cfg.dx[1], c->cfg.dx[2], x, y, z, vx, vy,
                                                vz, w, id);
    GX_LAUNCHED(c);
    return GX_OK;
}
