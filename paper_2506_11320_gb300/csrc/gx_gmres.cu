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
// The iteration is driven from the device: the Krylov column index, the
// Hessenberg matrix, the Givens rotations and the residual estimate live in a
// device-side state; reductions finish in the last CTA to arrive (no memsets,
// no host round trip); every kernel of an iteration returns at once when the
// state says the cycle is done.  The host enqueues iterations in batches and
// looks at the state only between batches and at restarts, so a solve costs a
// few host synchronisations instead of one per iteration.  The true residual
// ||b - A x|| / ||b|| is recomputed at every restart and decides convergence.
#include "gx_internal.cuh"

constexpr int kMaxM = 64;

struct GmState {
    int j;             // current Krylov column
    int done;          // the current cycle has ended
    int finished;      // the solve has ended
    int conv;          // converged (true residual <= tol)
    int total;         // matrix-vector products so far
    int jend;          // last column of the ended cycle
    int breakdown;
    int pad;
    unsigned cnt[4];   // last-CTA counters of the reductions
    double bnorm, beta, relres, hn2, est;
    double h[2][kMaxM + 2];
    double H[(kMaxM + 1) * kMaxM];
    double cs[kMaxM], sn[kMaxM], g[kMaxM + 1], y[kMaxM];
};

namespace {

constexpr int kB = 256;
constexpr int kRedBlocks = 152 * 2;
constexpr int kPartStride = kMaxM + 2;

inline int nblocks(int64_t n) {
    int64_t b = (n + kB - 1) / kB;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, kRedBlocks));
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;   // valid in thread 0
}

// true in every thread of the last CTA to finish (after its partials were
// published); resets the counter for the next use
__device__ __forceinline__ bool last_block(unsigned *counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
        if (last) *counter = 0;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// sum of the CTA partials of k values, by the last CTA
__device__ __forceinline__ void finish_sums(const double *partial, int k, double *out) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) s += partial[(size_t)b * kPartStride + i];
        out[i] = s;
    }
}

__global__ void k_gm_init(GmState *st) {
    if (threadIdx.x == 0) {
        st->j = 0; st->done = 1; st->finished = 0; st->conv = 0; st->total = 0; st->jend = -1;
        st->breakdown = 0;
        for (int i = 0; i < 4; ++i) st->cnt[i] = 0;
    }
}

// ||b||
__global__ void k_gm_bnorm(const double *__restrict__ b, int64_t n, GmState *st, double *partial) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        s += b[t] * b[t];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * kPartStride] = s;
    if (last_block(&st->cnt[0]) && threadIdx.x == 0) {
        double v = 0.0;
        for (int k = 0; k < (int)gridDim.x; ++k) v += partial[(size_t)k * kPartStride];
        st->bnorm = sqrt(v);
    }
}

// r = b - Ax (r holds Ax on entry); start a cycle or finish the solve
__global__ void k_gm_restart(const double *__restrict__ b, double *r, int64_t n, GmState *st, double *partial,
                             double tol, int maxit) {
    __shared__ double sh[32];
    if (st->finished) return;
    double s = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double v = b[t] - r[t];
        r[t] = v;
        s += v * v;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * kPartStride] = s;
    if (last_block(&st->cnt[0]) && threadIdx.x == 0) {
        double v = 0.0;
        for (int k = 0; k < (int)gridDim.x; ++k) v += partial[(size_t)k * kPartStride];
        const double beta = sqrt(v);
        st->beta = beta;
        st->relres = st->bnorm > 0.0 ? beta / st->bnorm : 0.0;
        if (st->relres <= tol) { st->finished = 1; st->conv = 1; st->done = 1; }
        else if (st->total >= maxit || st->breakdown) { st->finished = 1; st->done = 1; }
        else {
            st->done = 0;
            st->j = 0;
            st->jend = -1;
            for (int i = 0; i <= kMaxM; ++i) st->g[i] = 0.0;
            st->g[0] = beta;
        }
    }
}

// V_0 = r / beta
__global__ void k_gm_v0(const double *__restrict__ r, double *V, int64_t n, const GmState *st) {
    if (st->done) return;
    const double inv = 1.0 / st->beta;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        V[t] = r[t] * inv;
}

// h[pass][i] = V_i . w for i <= j
__global__ void k_gm_mdot(const double *__restrict__ V, int64_t n, const double *__restrict__ w, GmState *st,
                          double *partial, int pass) {
    __shared__ double sh[32];
    if (st->done) return;
    const int k = st->j + 1;
    for (int i = 0; i < k; ++i) {
        const double *v = V + (size_t)i * n;
        double s = 0.0;
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
            s += v[t] * w[t];
        s = block_sum(s, sh);
        if (threadIdx.x == 0) partial[(size_t)blockIdx.x * kPartStride + i] = s;
    }
    if (last_block(&st->cnt[1])) finish_sums(partial, k, st->h[pass]);
}

// w -= sum_i h[pass][i] V_i; for the second pass also ||w||^2 and the update
// of the Hessenberg column with Givens rotations (by the last CTA)
__global__ void k_gm_axpy(const double *__restrict__ V, int64_t n, double *w, GmState *st, double *partial, int pass,
                          int m, double tol, int maxit) {
    __shared__ double sh[32];
    __shared__ double coef[kMaxM + 2];
    if (st->done) return;
    const int k = st->j + 1;
    for (int i = threadIdx.x; i < k; i += blockDim.x) coef[i] = st->h[pass][i];
    __syncthreads();
    double s = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double acc = w[t];
        for (int i = 0; i < k; ++i) acc -= coef[i] * V[(size_t)i * n + t];
        w[t] = acc;
        s += acc * acc;
    }
    if (pass == 0) return;
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * kPartStride] = s;
    if (last_block(&st->cnt[2]) && threadIdx.x == 0) {
        double v = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) v += partial[(size_t)b * kPartStride];
        const int j = st->j;
        const double hn = sqrt(v);
        st->hn2 = v;
        double *H = st->H;
        for (int i = 0; i <= j; ++i) H[i * kMaxM + j] = st->h[0][i] + st->h[1][i];
        H[(j + 1) * kMaxM + j] = hn;
        for (int i = 0; i < j; ++i) {
            const double a = H[i * kMaxM + j], bb = H[(i + 1) * kMaxM + j];
            H[i * kMaxM + j] = st->cs[i] * a + st->sn[i] * bb;
            H[(i + 1) * kMaxM + j] = -st->sn[i] * a + st->cs[i] * bb;
        }
        const double a = H[j * kMaxM + j], bb = H[(j + 1) * kMaxM + j];
        const double den = sqrt(a * a + bb * bb);
        const double c = den == 0.0 ? 1.0 : a / den, sn = den == 0.0 ? 0.0 : bb / den;
        st->cs[j] = c;
        st->sn[j] = sn;
        H[j * kMaxM + j] = c * a + sn * bb;
        H[(j + 1) * kMaxM + j] = 0.0;
        st->g[j + 1] = -sn * st->g[j];
        st->g[j] = c * st->g[j];
        st->total += 1;
        st->est = fabs(st->g[j + 1]) / st->bnorm;
        if (hn == 0.0) st->breakdown = 1;
        if (st->est <= tol || st->total >= maxit || hn == 0.0 || j + 1 == m) {
            st->done = 1;
            st->jend = j;
        } else {
            st->j = j + 1;
        }
    }
}

// V_j = w / ||w|| (j already advanced by the Hessenberg update)
__global__ void k_gm_normalize(const double *__restrict__ w, double *V, int64_t n, const GmState *st) {
    if (st->done) return;
    const double inv = 1.0 / sqrt(st->hn2);
    double *v = V + (size_t)st->j * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        v[t] = w[t] * inv;
}

// y = H^{-1} g (upper triangular, jend+1 columns)
__global__ void k_gm_solve(GmState *st) {
    if (threadIdx.x != 0 || st->finished) return;
    const int je = st->jend;
    for (int i = je; i >= 0; --i) {
        double s = st->g[i];
        for (int k = i + 1; k <= je; ++k) s -= st->H[i * kMaxM + k] * st->y[k];
        st->y[i] = s / st->H[i * kMaxM + i];
    }
}

// x += sum_{i <= jend} y_i Z_i
__global__ void k_gm_xupdate(const double *__restrict__ Z, int64_t n, double *x, const GmState *st) {
    __shared__ double y[kMaxM];
    if (st->finished) return;
    const int k = st->jend + 1;
    for (int i = threadIdx.x; i < k; i += blockDim.x) y[i] = st->y[i];
    __syncthreads();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double acc = x[t];
        for (int i = 0; i < k; ++i) acc += y[i] * Z[(size_t)i * n + t];
        x[t] = acc;
    }
}

// staging of column j for preconditioners that take plain pointers
__global__ void k_gm_get_col(const double *__restrict__ V, int64_t n, const GmState *st, double *out) {
    if (st->done) return;
    const double *v = V + (size_t)st->j * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = v[t];
}
__global__ void k_gm_put_col(const double *__restrict__ in, double *Z, int64_t n, const GmState *st) {
    if (st->done) return;
    double *z = Z + (size_t)st->j * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        z[t] = in[t];
}

__global__ void k_gm_jacobi_col(const double *__restrict__ jd, const double *__restrict__ V, double *Z, int64_t N,
                                const GmState *st) {
    if (st->done) return;
    const double *v = V + (size_t)st->j * 3 * N;
    double *z = Z + (size_t)st->j * 3 * N;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        const double *o = jd + (size_t)q * 9;
        const double x0 = v[q], x1 = v[N + q], x2 = v[2 * N + q];
        z[q] = o[0] * x0 + o[1] * x1 + o[2] * x2;
        z[N + q] = o[3] * x0 + o[4] * x1 + o[5] * x2;
        z[2 * N + q] = o[6] * x0 + o[7] * x1 + o[8] * x2;
    }
}

}  // namespace

size_t gx_gm_state_bytes() { return sizeof(GmState); }
size_t gx_gm_partial_count() { return (size_t)kRedBlocks * kPartStride; }
int gx_gm_max_restart() { return kMaxM; }

// ||x||_2 computed on the device, read back (synchronises st)
double gx_norm_host(gx_ctx *c, const double *x, int64_t n, cudaStream_t st, int *status) {
    *status = GX_OK;
    k_gm_init<<<1, 32, 0, st>>>(c->gm);
    k_gm_bnorm<<<nblocks(n), kB, 0, st>>>(x, n, c->gm, c->gpart);
    c->launches += 2;
    double h = 0;
    if (cudaMemcpyAsync(&h, &c->gm->bnorm, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        *status = GX_ECUDA;
        c->err = "norm: CUDA error";
        return 0;
    }
    return h;
}

// Solve A x = rhs for x = Eth (initial guess already in Eth).
int gx_fgmres(gx_ctx *c, cudaStream_t st) {
    const int64_t n = 3 * c->N;
    const int m = c->cfg.gmres_restart;
    const int maxit = c->cfg.gmres_maxit;
    const double tol = c->cfg.gmres_tol;
    const int pc = c->cfg.precond;
    const bool flex = pc != GX_PRECOND_NONE;
    double *x = c->Eth, *b = c->rhs, *w = c->w, *r = c->r;
    double *V = c->V, *Z = flex ? c->Z : c->V;
    GmState *gs = c->gm;
    const int nb = nblocks(n);
    int rc;
    if (pc == GX_PRECOND_JACOBI || pc == GX_PRECOND_NET) { rc = gx_build_jacobi(c, st); if (rc) return rc; }
    k_gm_init<<<1, 32, 0, st>>>(gs);
    GX_LAUNCHED(c);
    k_gm_bnorm<<<nb, kB, 0, st>>>(b, n, gs, c->gpart);
    GX_LAUNCHED(c);
    struct Flags { int j, done, finished, conv, total; };
    Flags *hf = reinterpret_cast<Flags *>(c->hpin);
    auto read_flags = [&]() -> int {
        GX_CHECK(c, cudaMemcpyAsync(hf, gs, sizeof(Flags), cudaMemcpyDeviceToHost, st));
        GX_CHECK(c, cudaStreamSynchronize(st));
        return GX_OK;
    };
    auto enqueue_iteration = [&]() -> int {
        if (pc == GX_PRECOND_JACOBI) {
            k_gm_jacobi_col<<<nblocks(c->N), kB, 0, st>>>(c->jdiag, V, Z, c->N, gs);
            GX_LAUNCHED(c);
        } else if (pc == GX_PRECOND_NET) {
            k_gm_get_col<<<nb, kB, 0, st>>>(V, n, gs, c->vbuf);
            GX_LAUNCHED(c);
            int r2 = gx_net_apply(c, c->vbuf, c->zbuf, st);
            if (r2) return r2;
            k_gm_put_col<<<nb, kB, 0, st>>>(c->zbuf, Z, n, gs);
            GX_LAUNCHED(c);
        }
        int r2 = gx_apply_A_j(c, Z, n, &gs->j, &gs->done, w, st);
        if (r2) return r2;
        k_gm_mdot<<<nb, kB, 0, st>>>(V, n, w, gs, c->gpart, 0);
        GX_LAUNCHED(c);
        k_gm_axpy<<<nb, kB, 0, st>>>(V, n, w, gs, c->gpart, 0, m, tol, maxit);
        GX_LAUNCHED(c);
        k_gm_mdot<<<nb, kB, 0, st>>>(V, n, w, gs, c->gpart, 1);
        GX_LAUNCHED(c);
        k_gm_axpy<<<nb, kB, 0, st>>>(V, n, w, gs, c->gpart, 1, m, tol, maxit);
        GX_LAUNCHED(c);
        k_gm_normalize<<<nb, kB, 0, st>>>(w, V, n, gs);
        GX_LAUNCHED(c);
        return GX_OK;
    };
    // first batch sized by the previous solve (consecutive steps need similar
    // iteration counts), so most solves need one look at the device state
    int batch = std::max(2, std::min(16, c->last.iters > 0 ? c->last.iters : 4));
    for (int cycle = 0;; ++cycle) {
        // r = b - A x, decide, V_0 = r / beta
        rc = gx_apply_A(c, x, r, st);
        if (rc) return rc;
        k_gm_restart<<<nb, kB, 0, st>>>(b, r, n, gs, c->gpart, tol, maxit);
        GX_LAUNCHED(c);
        k_gm_v0<<<nb, kB, 0, st>>>(r, V, n, gs);
        GX_LAUNCHED(c);
        if (cycle == 0 && (rc = gx_net_pair_begin(c, r, st))) return rc;
        // iterate in batches until the cycle ends (kernels are no-ops after)
        for (;;) {
            for (int k = 0; k < batch; ++k)
                if ((rc = enqueue_iteration())) return rc;
            if ((rc = read_flags())) return rc;
            if (hf->done) break;
            batch = std::min(2 * batch, 16);
        }
        if (hf->finished) break;
        k_gm_solve<<<1, 32, 0, st>>>(gs);
        GX_LAUNCHED(c);
        k_gm_xupdate<<<nb, kB, 0, st>>>(Z, n, x, gs);
        GX_LAUNCHED(c);
        if (cycle > maxit + 2) break;
    }
    double tail[3];
    GX_CHECK(c, cudaMemcpyAsync(tail, &gs->relres, sizeof(double), cudaMemcpyDeviceToHost, st));
    GX_CHECK(c, cudaStreamSynchronize(st));
    c->last.iters = hf->total;
    c->last.relres = tail[0];
    c->last.converged = hf->conv;
    if ((rc = gx_net_pair_end(c, hf->conv, std::min(hf->total, m), st))) return rc;
    if (!hf->conv) {
        c->err = "GMRES reached gmres_maxit without converging (best iterate kept)";
        return GX_ENOCONV;
    }
    return GX_OK;
}
