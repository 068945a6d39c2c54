// gx_gmres.cu -- FP64 flexible GMRES for the implicit field equation.
//
// The paper names no linear solver; its field operator (Eq. 7 with the mass
// term of Eq. 35 and the LF term of Eq. 19) is non-symmetric because the
// rotation tensor is, so a Krylov method for general matrices is used:
// restarted FGMRES(m) with right preconditioning (identity, 3x3 block Jacobi,
// or the learned network, which is nonlinear and therefore needs the flexible
// variant that stores the preconditioned vectors).  Orthogonalisation is
// classical Gram-Schmidt applied twice; every inner product and norm is FP64.
//
// GB300-first design: the whole solve is one cooperative persistent kernel.
// Each thread owns a fixed set of nodes for every vector operation, so
// node-local steps need no synchronisation; a grid-wide barrier separates the
// steps that read other nodes (the matrix-vector product reads the 3x3
// neighbourhood) or need a global sum.  Global sums: every CTA writes its
// partial, and after the barrier every CTA adds all partials in the same
// order, so all CTAs hold bit-identical sums and take identical decisions (the
// Givens rotations, the convergence test) without another barrier.  An
// Arnoldi step costs four barriers.  The true residual ||b - A x|| / ||b|| is
// recomputed at every restart and decides convergence.  The learned
// preconditioner also runs inside the kernel: the thread that forms a Krylov
// column also packs it to BF16 for the network, the four convolution layers
// run on the fifth-generation tensor cores (tcgen05 fed by TMA bulk copies,
// accumulators in tensor memory) over the whole grid with a barrier before
// each layer, and the last adds the correction to the block-Jacobi image, so a
// solve is one launch with every preconditioner.
#include <cooperative_groups.h>
#include <type_traits>

#include "gx_netpipe.cuh"
#include "gx_op.cuh"

namespace cg = cooperative_groups;

constexpr int kMaxM = 64;

struct GmState {
    int j;             // current Krylov column
    int done;          // the current cycle has ended (a restart is due)
    int finished;      // the solve has ended
    int conv;          // converged (true residual <= tol)
    int total;         // Arnoldi steps (matrix-vector products on Krylov vectors) so far
    int jend;          // last column of the ended cycle
    int breakdown;
    int pad;
    double bnorm, beta, relres, est;
    double H[(kMaxM + 1) * kMaxM];     // rotated Hessenberg (upper triangular R), row-major [i][col]
    double cs[kMaxM], sn[kMaxM], g[kMaxM + 1];
};

namespace {

constexpr int kB = 256;               // threads per CTA (plain / block Jacobi: two CTAs per SM)
constexpr int kBNet = 512;            // with the network: one CTA per SM (its shared and tensor memory)
constexpr int kWarps = kB / 32;
constexpr int kMaxWarps = kBNet / 32;
constexpr int kMaxGrid = 152 * 8;
constexpr int kPartStride = kMaxM + 2;

struct CoArgs {
    OpArgs op;
    const double *b;
    double *x;          // solution (initial guess on entry)
    double *V;          // Krylov basis [(m+1)][3N]
    double *Z;          // preconditioned vectors [m][3N] (== V without a preconditioner)
    double *w, *r;      // [3N]
    const double *jd;   // block-Jacobi inverse [N][9], or null
    const float *jd32;  // the same in FP32 (the learned preconditioner's base)
    GmState *st;
    double *part;       // [2][kMaxGrid][kPartStride] CTA partial sums
    int64_t N;
    int m, maxit;
    double tol;
    int net;            // apply the learned preconditioner (the fields below)
    NetSolverArgs nn;
    double ns;          // its scale s = 1 / sqrt(3 N) (the Krylov columns have unit norm)
    float inv_ns;       // 1 / s
    int *err;           // set when a bounded wait of the network's tensor-core steps gives up
};

// in-kernel network: shared memory of the pipeline (+ alignment slack)
constexpr int kNetSmemBytes = gxn::kSmemBytes + 128;
static_assert(kBNet % gxv::kThreads == 0 && kBNet / gxv::kThreads <= 2, "the convolution's role groups");

// every thread's node set: q = tid, tid + nthreads, ...
#define NODE_LOOP(q) \
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x)

// CTA sums of kk <= 8 thread values -> dst[0..kk) (global partial row).  AT is the
// type of the thread and warp sums: double, or float for the mixed-precision cycles
// (whose vectors are FP32); the sums across warps and CTAs are FP64 either way.
template <typename AT>
__device__ __forceinline__ void cta_partials(AT acc[8], int kk, double *sred, double *dst) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i >= kk) break;                                   // kk is the same for the whole CTA
        AT v = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sred[warp * 8 + i] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < kk) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sred[w * 8 + threadIdx.x];
        dst[threadIdx.x] = s;
    }
    __syncthreads();
}

// sum over all CTAs of partial rows [0, k) -> out (shared), same order in every CTA
__device__ __forceinline__ void grid_sums(const double *part, int k, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < k; i += (int)(blockDim.x >> 5)) {
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(part + (size_t)b * kPartStride + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[i] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ double *prow(const CoArgs &a, int ph) {
    return a.part + ((size_t)(ph & 1) * kMaxGrid + blockIdx.x) * kPartStride;
}
__device__ __forceinline__ const double *pbuf(const CoArgs &a, int ph) {
    return a.part + (size_t)(ph & 1) * kMaxGrid * kPartStride;
}

// z = D^-1 v at node q from the FP32 inverse (the mixed-precision cycles)
__device__ __forceinline__ void jacobi_node(const float *jd, const float *v, float *z, int64_t N, int64_t q) {
    const float *o = jd + (size_t)q * 9;
    const float x0 = v[q], x1 = v[N + q], x2 = v[2 * N + q];
    z[q] = o[0] * x0 + o[1] * x1 + o[2] * x2;
    z[N + q] = o[3] * x0 + o[4] * x1 + o[5] * x2;
    z[2 * N + q] = o[6] * x0 + o[7] * x1 + o[8] * x2;
}

// z = D^-1 v at node q (3x3 block)
__device__ __forceinline__ void jacobi_node(const double *jd, const double *v, double *z, int64_t N, int64_t q) {
    const double *o = jd + (size_t)q * 9;
    const double x0 = v[q], x1 = v[N + q], x2 = v[2 * N + q];
    z[q] = o[0] * x0 + o[1] * x1 + o[2] * x2;
    z[N + q] = o[3] * x0 + o[4] * x1 + o[5] * x2;
    z[2 * N + q] = o[6] * x0 + o[7] * x1 + o[8] * x2;
}

// the network input of node q: (V_j at q) / s in BF16, 16 channels, into the
// halo-ring image x0 (periodic copies included); written by the thread that
// computes V_j at q, so the layer-1 tiles see it after the next grid barrier
__device__ __forceinline__ void net_pack_node(const CoArgs &a, int64_t q, double v0, double v1, double v2) {
    const float inv = a.inv_ns;
    const __nv_bfloat162 p01 = __floats2bfloat162_rn((float)v0 * inv, (float)v1 * inv);
    const __nv_bfloat162 p2 = __floats2bfloat162_rn((float)v2 * inv, 0.f);
    const uint4 val[2] = {make_uint4(*reinterpret_cast<const uint32_t *>(&p01), *reinterpret_cast<const uint32_t *>(&p2),
                                     0, 0),
                          make_uint4(0, 0, 0, 0)};
    const int W = a.op.g.nx;
    gxv::store_with_halo<16>(static_cast<gxv::bf16 *>(a.nn.x0), 0, (int)(q / W), (int)(q % W), a.op.g.ny, W, 1, val);
}

// Z_j = D^-1 V_j + s N(V_j / s), every CTA of the cooperative grid taking part:
// the four layers as one persistent tensor-core pipeline (gx_netpipe.cuh),
// after a grid barrier that completes the packed input V_j / s and the
// clearing of the pipeline's completion flags; the last layer writes Z_j
// itself (the caller's barrier follows)
__device__ void net_apply(const CoArgs &a, cg::grid_group &grid, int j, unsigned char *sm) {
    const int64_t n = 3 * a.N;
    const int H = a.op.g.ny, W = a.op.g.nx;
    gxn::pipe_clear_flags(a.nn.flags, H, W, blockIdx.x, gridDim.x);
    grid.sync();
    gxn::PipeArgs p;
    p.in[0] = static_cast<const gxv::bf16 *>(a.nn.x0);
    p.in[1] = static_cast<const gxv::bf16 *>(a.nn.h1);
    p.in[2] = static_cast<const gxv::bf16 *>(a.nn.h2);
    p.in[3] = static_cast<const gxv::bf16 *>(a.nn.h3);
    p.out[0] = static_cast<gxv::bf16 *>(a.nn.h1);
    p.out[1] = static_cast<gxv::bf16 *>(a.nn.h2);
    p.out[2] = static_cast<gxv::bf16 *>(a.nn.h3);
    for (int l = 0; l < 4; ++l) {
        p.w[l] = static_cast<const gxv::bf16 *>(a.nn.w[l]);
        p.bias[l] = a.nn.b[l];
    }
    p.v = a.V + (size_t)j * n;
    p.jd = a.jd32;
    p.z = a.Z + (size_t)j * n;
    p.s = (float)a.ns;
    p.flags = a.nn.flags;
    p.err = a.err;
    p.H = H;
    p.W = W;
    gxn::net_pipeline(p, sm, blockIdx.x, gridDim.x);
}

// NET: the learned preconditioner is applied in the kernel (the plain and
// Jacobi instantiation is smaller and fits two CTAs per SM).
// MIX: mixed-precision iterative refinement (Carson and Higham, SIAM J. Sci.
// Comput. 40, 2018): every restart computes the true residual b - A x and
// updates x in FP64; the Arnoldi cycle between restarts keeps its basis, the
// preconditioned vectors and w in FP32 and applies the operator from FP32 copies
// of M and kappa (3D: of the assembled blocks), while its inner products and
// norms accumulate in FP64.  A cycle stops once its residual estimate has
// fallen by kCycleDrop (well above the FP32 floor of the Arnoldi relation), and
// the next restart judges the FP64 true residual, so the solve still ends at
// the requested tolerance (the FP32 correction of a cycle is accurate to about
// kappa(A) 6e-8 of the residual it corrects, far below kCycleDrop for these
// operators, which are the identity plus positive semi-definite terms scaled by
// (c theta dt)^2 and the plasma's mass matrix).  GB300 runs FP64 at 1/64 of the FP32 rate: the cycle
// is where the FP64 solve spent it.
constexpr double kCycleDrop = 1e-4;
template <bool NET, int DIM = 2, bool MIX = false>
__global__ void __launch_bounds__(NET ? kBNet : kB, NET ? 1 : 2) k_fgmres(const __grid_constant__ CoArgs a) {
    using VT = typename std::conditional<MIX, float, double>::type;   // Krylov storage and arithmetic
    extern __shared__ __align__(128) unsigned char gsm_raw[];
    unsigned char *gsm = gsm_raw + ((128 - (gxt::smem_addr(gsm_raw) & 127)) & 127);
    cg::grid_group grid = cg::this_grid();
    __shared__ double sred[kMaxWarps * 8];
    __shared__ double hs[2][kMaxM + 2];
    __shared__ double s_cs[kMaxM], s_sn[kMaxM], s_g[kMaxM + 1], s_y[kMaxM];
    __shared__ double s_scalar[2];
    GmState *st = a.st;
    const int64_t N = a.N, n = 3 * N;
    const int m = a.m;
    const bool flex = a.Z != a.V;
    VT *const V = reinterpret_cast<VT *>(a.V);
    VT *const Z = reinterpret_cast<VT *>(a.Z);
    VT *const w = reinterpret_cast<VT *>(a.w);
    int j = st->j, done = st->done, total = st->total, breakdown = st->breakdown;
    double bnorm = st->bnorm;
    double ctol = a.tol;                            // this cycle's target for the residual estimate
    if (st->finished) return;
    for (int i = threadIdx.x; i < kMaxM; i += blockDim.x) { s_cs[i] = st->cs[i]; s_sn[i] = st->sn[i]; }
    for (int i = threadIdx.x; i <= kMaxM; i += blockDim.x) s_g[i] = st->g[i];
    int ph = 0;
    __syncthreads();
    const bool writer = blockIdx.x == 0 && threadIdx.x == 0;

    if (bnorm < 0.0) {                              // first launch of a solve: ||b||
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        NODE_LOOP(q) {
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[0] += a.b[c * N + q] * a.b[c * N + q];
        }
        cta_partials(acc, 1, sred, prow(a, ph));
        grid.sync();
        grid_sums(pbuf(a, ph), 1, s_scalar);
        ++ph;
        bnorm = sqrt(s_scalar[0]);
        if (writer) st->bnorm = bnorm;
    }
    if (bnorm == 0.0) {
        // b = 0: the operator is nonsingular, so the solution is exactly 0 (the
        // starting guess is not kept: its residual could not be judged relative to ||b||)
        NODE_LOOP(q) {
#pragma unroll
            for (int c = 0; c < 3; ++c) a.x[c * N + q] = 0.0;
        }
        if (writer) {
            st->beta = 0.0;
            st->relres = 0.0;
            st->finished = 1;
            st->conv = 1;
            st->done = 1;
            st->total = total;
        }
        return;
    }

    for (;;) {
        if (done) {
            // ---- restart: r = b - A x, beta = ||r||, convergence on the true residual
            double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            NODE_LOOP(q) {
                double ax[3];
                gx_apply_node<DIM, true>(a.op, a.x, q, ax);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double rv = a.b[c * N + q] - ax[c];
                    a.r[c * N + q] = rv;
                    acc[0] += rv * rv;
                }
            }
            cta_partials(acc, 1, sred, prow(a, ph));
            grid.sync();
            grid_sums(pbuf(a, ph), 1, s_scalar);
            ++ph;
            const double beta = sqrt(s_scalar[0]);
            const double relres = bnorm > 0.0 ? beta / bnorm : 0.0;
            if (writer) { st->beta = beta; st->relres = relres; }
            if (relres <= a.tol || total >= a.maxit || breakdown) {
                if (writer) {
                    st->finished = 1;
                    st->conv = relres <= a.tol;
                    st->done = 1;
                    st->total = total;
                }
                return;
            }
            j = 0;
            done = 0;
            if (MIX) ctol = fmax(a.tol, relres * kCycleDrop);
            for (int i = threadIdx.x; i <= kMaxM; i += blockDim.x) s_g[i] = i == 0 ? beta : 0.0;
            const double inv = 1.0 / beta;
            NODE_LOOP(q) {
#pragma unroll
                for (int c = 0; c < 3; ++c) V[c * N + q] = (VT)(a.r[c * N + q] * inv);
                if constexpr (MIX) {
                    if (a.jd) jacobi_node(a.jd32, V, Z, N, q);
                } else {
                    if (a.jd && !NET) jacobi_node(a.jd, V, Z, N, q);
                    if (NET) net_pack_node(a, q, V[q], V[N + q], V[2 * N + q]);
                }
            }
            __syncthreads();
            if (writer) {
                st->j = 0; st->done = 0; st->jend = -1;
                for (int i = 0; i <= kMaxM; ++i) st->g[i] = i == 0 ? beta : 0.0;
            }
            if (NET) net_apply(a, grid, 0, gsm);
            grid.sync();
        }

        // ---- Arnoldi step j: w = A z_j, two classical Gram-Schmidt passes
        const int k = j + 1;
        const VT *zj = (flex ? Z : V) + (size_t)j * n;
        // pass 1: w = A z_j, partial h0_i = V_i . w
        for (int i0 = 0; i0 < k; i0 += 8) {
            VT acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            NODE_LOOP(q) {
                VT wq[3];
                if (i0 == 0) {
                    gx_apply_node<DIM, true, VT>(a.op, zj, q, wq);
#pragma unroll
                    for (int c = 0; c < 3; ++c) w[c * N + q] = wq[c];
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) wq[c] = w[c * N + q];
                }
#pragma unroll
                for (int ii = 0; ii < 8; ++ii)
                    if (i0 + ii < k) {
                        const VT *vi = V + (size_t)(i0 + ii) * n;
                        acc[ii] += vi[q] * wq[0] + vi[N + q] * wq[1] + vi[2 * N + q] * wq[2];
                    }
            }
            cta_partials(acc, min(8, k - i0), sred, prow(a, ph) + i0);
        }
        grid.sync();
        grid_sums(pbuf(a, ph), k, hs[0]);
        ++ph;
        // pass 2: w -= sum h0_i V_i, partial h1_i = V_i . w
        NODE_LOOP(q) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                VT v = w[c * N + q];
                for (int i = 0; i < k; ++i) v -= (VT)hs[0][i] * V[(size_t)i * n + c * N + q];
                w[c * N + q] = v;
            }
        }
        for (int i0 = 0; i0 < k; i0 += 8) {
            VT acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            NODE_LOOP(q) {
                const VT w0 = w[q], w1 = w[N + q], w2 = w[2 * N + q];
#pragma unroll
                for (int ii = 0; ii < 8; ++ii)
                    if (i0 + ii < k) {
                        const VT *vi = V + (size_t)(i0 + ii) * n;
                        acc[ii] += vi[q] * w0 + vi[N + q] * w1 + vi[2 * N + q] * w2;
                    }
            }
            cta_partials(acc, min(8, k - i0), sred, prow(a, ph) + i0);
        }
        grid.sync();
        grid_sums(pbuf(a, ph), k, hs[1]);
        ++ph;
        // pass 3: w -= sum h1_i V_i, partial ||w||^2
        {
            VT acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            NODE_LOOP(q) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    VT v = w[c * N + q];
                    for (int i = 0; i < k; ++i) v -= (VT)hs[1][i] * V[(size_t)i * n + c * N + q];
                    w[c * N + q] = v;
                    acc[0] += v * v;
                }
            }
            cta_partials(acc, 1, sred, prow(a, ph));
        }
        grid.sync();
        grid_sums(pbuf(a, ph), 1, s_scalar);
        ++ph;
        const double hn = sqrt(s_scalar[0]);
        // Givens update of column j (identical in every CTA)
        if (threadIdx.x == 0) {
            double col[kMaxM + 1];
            for (int i = 0; i <= j; ++i) col[i] = hs[0][i] + hs[1][i];
            col[j + 1] = hn;
            for (int i = 0; i < j; ++i) {
                const double p = col[i], q2 = col[i + 1];
                col[i] = s_cs[i] * p + s_sn[i] * q2;
                col[i + 1] = -s_sn[i] * p + s_cs[i] * q2;
            }
            const double p = col[j], q2 = col[j + 1];
            const double den = sqrt(p * p + q2 * q2);
            const double cj = den == 0.0 ? 1.0 : p / den, sj = den == 0.0 ? 0.0 : q2 / den;
            s_cs[j] = cj;
            s_sn[j] = sj;
            col[j] = cj * p + sj * q2;
            s_g[j + 1] = -sj * s_g[j];
            s_g[j] = cj * s_g[j];
            s_scalar[1] = fabs(s_g[j + 1]) / bnorm;
            if (blockIdx.x == 0) {
                for (int i = 0; i <= j; ++i) st->H[i * kMaxM + j] = col[i];
                st->cs[j] = cj;
                st->sn[j] = sj;
                st->g[j] = s_g[j];
                st->g[j + 1] = s_g[j + 1];
            }
        }
        __syncthreads();
        total += 1;
        if (hn == 0.0) breakdown = 1;
        const double est = s_scalar[1];
        const bool ended = est <= ctol || total >= a.maxit || hn == 0.0 || j + 1 == m;
        if (writer) { st->total = total; st->est = est; st->breakdown = breakdown; }
        if (!ended) {
            // V_{j+1} = w / hn (and its block-Jacobi image)
            const VT inv = (VT)(1.0 / hn);
            VT *v1 = V + (size_t)(j + 1) * n;
            NODE_LOOP(q) {
#pragma unroll
                for (int c = 0; c < 3; ++c) v1[c * N + q] = w[c * N + q] * inv;
                if constexpr (MIX) {
                    if (a.jd) jacobi_node(a.jd32, v1, Z + (size_t)(j + 1) * n, N, q);
                } else {
                    if (a.jd && !NET) jacobi_node(a.jd, v1, Z + (size_t)(j + 1) * n, N, q);
                    if (NET) net_pack_node(a, q, v1[q], v1[N + q], v1[2 * N + q]);
                }
            }
            ++j;
            if (writer) st->j = j;
            if (NET) net_apply(a, grid, j, gsm);
            grid.sync();
            continue;
        }
        // ---- cycle end: y = R^-1 g, x += sum y_i z_i
        grid.sync();                                // R columns written by CTA 0
        if (threadIdx.x == 0) {
            for (int i = j; i >= 0; --i) {
                double s = s_g[i];
                for (int kk = i + 1; kk <= j; ++kk) s -= __ldcg(&st->H[i * kMaxM + kk]) * s_y[kk];
                s_y[i] = s / __ldcg(&st->H[i * kMaxM + i]);
            }
        }
        __syncthreads();
        const VT *Zb = flex ? Z : V;
        NODE_LOOP(q) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double v = a.x[c * N + q];
                for (int i = 0; i <= j; ++i) v += s_y[i] * (double)Zb[(size_t)i * n + c * N + q];
                a.x[c * N + q] = v;
            }
        }
        done = 1;
        if (writer) { st->done = 1; st->jend = j; }
        grid.sync();                                // x complete before the restart reads it
    }
}

__global__ void k_gm_init(GmState *st) {
    if (threadIdx.x == 0) {
        st->j = 0; st->done = 1; st->finished = 0; st->conv = 0; st->total = 0; st->jend = -1;
        st->breakdown = 0;
        st->bnorm = -1.0;
        for (int i = 0; i < kMaxM; ++i) { st->cs[i] = 1.0; st->sn[i] = 0.0; }
        for (int i = 0; i <= kMaxM; ++i) st->g[i] = 0.0;
    }
}

__global__ void k_norm2(const double *__restrict__ x, int64_t n, double *out) {
    __shared__ double sh[kWarps];
    double s = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        s += x[t] * x[t];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += sh[w];
        atomicAdd(out, t);
    }
}

__global__ void k_sub(const double *__restrict__ b, const double *__restrict__ ax, double *r, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        r[t] = b[t] - ax[t];
}

inline int nblocks(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kB - 1) / kB, 152 * 4));
}

}  // namespace

size_t gx_gm_state_bytes() { return sizeof(GmState); }
size_t gx_gm_partial_count() { return (size_t)2 * kMaxGrid * kPartStride; }
int gx_gm_max_restart() { return kMaxM; }

// ||x||_2 computed on the device, read back (synchronises st)
double gx_norm_host(gx_ctx *c, const double *x, int64_t n, cudaStream_t st, int *status) {
    *status = GX_OK;
    double *acc = c->gpart;
    double h = 0;
    if (cudaMemsetAsync(acc, 0, sizeof(double), st) != cudaSuccess) { *status = GX_ECUDA; return 0; }
    k_norm2<<<nblocks(n), kB, 0, st>>>(x, n, acc);
    c->launches += 1;
    if (cudaMemcpyAsync(&h, acc, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        *status = GX_ECUDA;
        c->err = "norm: CUDA error";
        return 0;
    }
    return sqrt(h);
}

// Solve A x = rhs for x = Eth (the starting point already in Eth).
int gx_fgmres(gx_ctx *c, cudaStream_t st) {
    const int64_t n = 3 * c->N;
    const int pc = c->cfg.precond;
    int rc;
    if (c->dim == 3 && (rc = gx3_build_op(c, st))) return rc;   // the operator's blocks for this solve
    // the learned preconditioner reads only the FP32 inverse; pair collection and the
    // Jacobi preconditioner need the FP64 one
    if (pc == GX_PRECOND_JACOBI || (pc == GX_PRECOND_NET && gx_net_collecting(c))) {
        rc = gx_build_jacobi(c, st);
        if (rc) return rc;
    } else if (pc == GX_PRECOND_NET) {
        rc = gx_build_jacobi32(c, st);
        if (rc) return rc;
    }
    const bool use_net = pc == GX_PRECOND_NET;
    const size_t smem = use_net ? (size_t)kNetSmemBytes : 0;
    const bool mix = c->cfg.gmres_mixed && !use_net;
    static int grids[5] = {0, 0, 0, 0, 0};
    const int kind = use_net ? 1 : (c->dim == 3 ? (mix ? 4 : 2) : (mix ? 3 : 0));
    int &grid = grids[kind];
    const void *kfns[5] = {(const void *)k_fgmres<false>, (const void *)k_fgmres<true>,
                           (const void *)k_fgmres<false, 3>, (const void *)k_fgmres<false, 2, true>,
                           (const void *)k_fgmres<false, 3, true>};
    const void *kfn = kfns[kind];
    if (!grid) {
        int dev = 0, nsm = 0, per = 0;
        GX_CHECK(c, cudaGetDevice(&dev));
        GX_CHECK(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        if (smem > 0)
            GX_CHECK(c, cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        GX_CHECK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kfn, use_net ? kBNet : kB, smem));
        grid = std::max(1, std::min(per * nsm, kMaxGrid));
    }
    CoArgs a{};
    a.op = gx_opargs(c);   // with gmres_mixed, its FP32 copies were written with M, kappa and the 3D blocks
    a.b = c->rhs;
    a.x = c->Eth;
    a.V = c->V;
    a.Z = pc == GX_PRECOND_NONE ? c->V : c->Z;
    a.w = c->w;
    a.r = c->r;
    a.jd = pc == GX_PRECOND_NONE ? nullptr : c->jdiag;
    a.jd32 = c->jdiag32;
    a.st = c->gm;
    a.part = c->gpart;
    a.N = c->N;
    a.m = c->cfg.gmres_restart;
    a.maxit = c->cfg.gmres_maxit;
    a.tol = c->cfg.gmres_tol;
    a.net = use_net;
    if (use_net) {
        if ((rc = gx_net_solver_args(c, &a.nn, st))) return rc;
        a.ns = 1.0 / std::sqrt(3.0 * (double)c->N);
        a.inv_ns = (float)std::sqrt(3.0 * (double)c->N);
        a.err = &c->dflags->timeout;
    }
    if (gx_net_collecting(c)) {
        // training pair of this solve: r0 = b - A E^n, so that A (E^{n+theta} - E^n) = r0
        if ((rc = gx_apply_A(c, c->E, c->w, st))) return rc;
        k_sub<<<nblocks(n), kB, 0, st>>>(c->rhs, c->w, c->r, n);
        GX_LAUNCHED(c);
        if ((rc = gx_net_pair_begin(c, c->r, st))) return rc;
    }
    k_gm_init<<<1, 32, 0, st>>>(c->gm);
    GX_LAUNCHED(c);
    void *args[] = {&a};
    // small grids: no more CTAs than one node per thread, so that the grid barriers
    // of every Arnoldi step synchronise few CTAs (the network path keeps its grid)
    const int ngrid = use_net ? grid : (int)std::max<int64_t>(1, std::min<int64_t>(grid, (c->N + kB - 1) / kB));
    GX_CHECK(c, cudaLaunchCooperativeKernel(kfn, dim3(ngrid), dim3(use_net ? kBNet : kB), args, smem, st));
    c->launches++;
    struct Flags { int j, done, finished, conv, total; };
    Flags *hf = reinterpret_cast<Flags *>(c->hpin);
    double tail[4];
    GX_CHECK(c, cudaMemcpyAsync(hf, c->gm, sizeof(Flags), cudaMemcpyDeviceToHost, st));
    GX_CHECK(c, cudaMemcpyAsync(tail, &c->gm->bnorm, sizeof(tail), cudaMemcpyDeviceToHost, st));
    GX_CHECK(c, cudaStreamSynchronize(st));
    if (!hf->finished) { c->err = "FGMRES: the solve did not finish"; return GX_ECUDA; }
    c->last.iters = hf->total;
    c->last.relres = tail[2];
    c->last.converged = hf->conv;
    if ((rc = gx_net_pair_end(c, hf->conv, std::min(hf->total, a.m), st))) return rc;
    if (!hf->conv) {
        c->err = "GMRES reached gmres_maxit without converging (best iterate kept)";
        return GX_ENOCONV;
    }
    return GX_OK;
}
