// gx_gmres.cu -- FP64 flexible GMRES for the implicit field equation.
//
// The paper names no linear solver; its field operator (Eq. 7 with the mass
// term of Eq. 35 and the LF term of Eq. 19) is non-symmetric because the
// rotation tensor is, so a Krylov method for general matrices is used:
// restarted FGMRES(m) with right preconditioning (identity, 3x3 block Jacobi,
// or the learned network, which is nonlinear and therefore needs the flexible
// variant that stores the preconditioned vectors).  Orthogonalisation is
// classical Gram-Schmidt applied twice; every inner product and norm is FP64
// and reduced on the device.  Convergence is judged on the relative residual;
// the true residual ||b - A x|| / ||b|| is recomputed at every restart and at
// exit.
#include "gx_internal.cuh"

namespace {

constexpr int kB = 256;

inline int nblocks(int64_t n) {
    int64_t b = (n + kB - 1) / kB;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;
}

// out[i] += sum_t V_i[t] w[t] for i < k (out zeroed by the caller)
__global__ void k_mdot(const double *__restrict__ V, int64_t ldv, int k, const double *__restrict__ w, int64_t n,
                       double *out) {
    __shared__ double sh[32];
    for (int i = 0; i < k; ++i) {
        const double *v = V + (size_t)i * ldv;
        double s = 0.0;
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
            s += v[t] * w[t];
        s = block_sum(s, sh);
        if (threadIdx.x == 0) atomicAdd(out + i, s);
    }
}

// w[t] -= sum_i coef[i] V_i[t];  nrm2 += w[t]^2 (if nrm2)
__global__ void k_maxpy(const double *__restrict__ V, int64_t ldv, int k, const double *__restrict__ coef, double *w,
                        int64_t n, double *nrm2) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double acc = w[t];
        for (int i = 0; i < k; ++i) acc -= coef[i] * V[(size_t)i * ldv + t];
        w[t] = acc;
        s += acc * acc;
    }
    if (nrm2) {
        s = block_sum(s, sh);
        if (threadIdx.x == 0) atomicAdd(nrm2, s);
    }
}

// y = x / sqrt(*nrm2)
__global__ void k_normalize(const double *__restrict__ x, double *y, int64_t n, const double *nrm2) {
    const double inv = 1.0 / sqrt(*nrm2);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        y[t] = x[t] * inv;
}

// r = b - r;  nrm2 += r^2
__global__ void k_residual(const double *__restrict__ b, double *r, int64_t n, double *nrm2) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double v = b[t] - r[t];
        r[t] = v;
        s += v * v;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) atomicAdd(nrm2, s);
}

__global__ void k_nrm2(const double *__restrict__ x, int64_t n, double *nrm2) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        s += x[t] * x[t];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) atomicAdd(nrm2, s);
}

int precondition(gx_ctx *c, const double *v, double *z, cudaStream_t st) {
    switch (c->cfg.precond) {
        case GX_PRECOND_JACOBI: return gx_apply_jacobi(c, v, z, st);
        case GX_PRECOND_NET: return gx_net_apply(c, v, z, st);
        default: return GX_OK;
    }
}

}  // namespace

// ||x||_2 computed on the device, read back (synchronises st)
double gx_norm_host(gx_ctx *c, const double *x, int64_t n, cudaStream_t st, int *status) {
    *status = GX_OK;
    if (cudaMemsetAsync(c->dred, 0, sizeof(double), st) != cudaSuccess) { *status = GX_ECUDA; return 0; }
    k_nrm2<<<nblocks(n), kB, 0, st>>>(x, n, c->dred);
    c->launches++;
    double h = 0;
    if (cudaMemcpyAsync(&h, c->dred, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        *status = GX_ECUDA;
        c->err = "norm: CUDA error";
        return 0;
    }
    return sqrt(h);
}

// Solve A x = rhs for x = Eth (initial guess already in Eth).
int gx_fgmres(gx_ctx *c, cudaStream_t st) {
    const int64_t n = 3 * c->N;
    const int m = c->cfg.gmres_restart;
    const bool flex = c->cfg.precond != GX_PRECOND_NONE;
    double *x = c->Eth, *b = c->rhs, *w = c->w, *r = c->r;
    double *V = c->V, *Z = flex ? c->Z : c->V;
    double *dh = c->hcol;          // [m+2]: dot products of the current column
    double *dn = c->dred;          // scalar accumulators
    int rc;
    if (c->cfg.precond == GX_PRECOND_JACOBI) { rc = gx_build_jacobi(c, st); if (rc) return rc; }
    int status = GX_OK;
    const double bnorm = gx_norm_host(c, b, n, st, &status);
    if (status) return status;
    c->last = gx_solve_stats{};
    if (bnorm == 0.0) {
        GX_CHECK(c, cudaMemsetAsync(x, 0, n * sizeof(double), st));
        c->last.converged = 1;
        return GX_OK;
    }
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    int total = 0;
    bool conv = false;
    double relres = 1.0;
    for (;;) {
        // r = b - A x
        rc = gx_apply_A(c, x, r, st);
        if (rc) return rc;
        GX_CHECK(c, cudaMemsetAsync(dn, 0, sizeof(double), st));
        k_residual<<<nblocks(n), kB, 0, st>>>(b, r, n, dn);
        GX_LAUNCHED(c);
        double beta2 = 0;
        GX_CHECK(c, cudaMemcpyAsync(&beta2, dn, sizeof(double), cudaMemcpyDeviceToHost, st));
        GX_CHECK(c, cudaStreamSynchronize(st));
        const double beta = sqrt(beta2);
        relres = beta / bnorm;
        if (relres <= c->cfg.gmres_tol) { conv = true; break; }
        if (total >= c->cfg.gmres_maxit) break;
        k_normalize<<<nblocks(n), kB, 0, st>>>(r, V, n, dn);
        GX_LAUNCHED(c);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int jend = -1;
        for (int j = 0; j < m; ++j) {
            double *vj = V + (size_t)j * n;
            double *zj = Z + (size_t)j * n;
            if (flex) { rc = precondition(c, vj, zj, st); if (rc) return rc; }
            rc = gx_apply_A(c, zj, w, st);
            if (rc) return rc;
            // classical Gram-Schmidt, twice
            GX_CHECK(c, cudaMemsetAsync(dh, 0, 2 * (m + 2) * sizeof(double), st));
            k_mdot<<<nblocks(n), kB, 0, st>>>(V, n, j + 1, w, n, dh);
            GX_LAUNCHED(c);
            k_maxpy<<<nblocks(n), kB, 0, st>>>(V, n, j + 1, dh, w, n, nullptr);
            GX_LAUNCHED(c);
            k_mdot<<<nblocks(n), kB, 0, st>>>(V, n, j + 1, w, n, dh + (m + 2));
            GX_LAUNCHED(c);
            GX_CHECK(c, cudaMemsetAsync(dn, 0, sizeof(double), st));
            k_maxpy<<<nblocks(n), kB, 0, st>>>(V, n, j + 1, dh + (m + 2), w, n, dn);
            GX_LAUNCHED(c);
            k_normalize<<<nblocks(n), kB, 0, st>>>(w, V + (size_t)(j + 1) * n, n, dn);
            GX_LAUNCHED(c);
            GX_CHECK(c, cudaMemcpyAsync(c->hpin, dh, 2 * (m + 2) * sizeof(double), cudaMemcpyDeviceToHost, st));
            double hn2 = 0;
            GX_CHECK(c, cudaMemcpyAsync(&hn2, dn, sizeof(double), cudaMemcpyDeviceToHost, st));
            GX_CHECK(c, cudaStreamSynchronize(st));
            ++total;
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = c->hpin[i] + c->hpin[(m + 2) + i];
            const double hn = sqrt(hn2);
            H[(size_t)(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * H[(size_t)i * m + j] + sn[i] * H[(size_t)(i + 1) * m + j];
                H[(size_t)(i + 1) * m + j] = -sn[i] * H[(size_t)i * m + j] + cs[i] * H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = t;
            }
            const double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
            const double den = sqrt(a * a + bb * bb);
            cs[j] = den == 0.0 ? 1.0 : a / den;
            sn[j] = den == 0.0 ? 0.0 : bb / den;
            H[(size_t)j * m + j] = cs[j] * a + sn[j] * bb;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            jend = j;
            if (std::fabs(g[j + 1]) / bnorm <= c->cfg.gmres_tol || total >= c->cfg.gmres_maxit || hn == 0.0) break;
        }
        // y = H^{-1} g, x += Z y
        for (int i = jend; i >= 0; --i) {
            double s = g[i];
            for (int k = i + 1; k <= jend; ++k) s -= H[(size_t)i * m + k] * y[k];
            y[i] = s / H[(size_t)i * m + i];
        }
        for (int i = 0; i <= jend; ++i) c->hpin[i] = -y[i];
        GX_CHECK(c, cudaMemcpyAsync(dh, c->hpin, (jend + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
        k_maxpy<<<nblocks(n), kB, 0, st>>>(Z, n, jend + 1, dh, x, n, nullptr);
        GX_LAUNCHED(c);
    }
    c->last.iters = total;
    c->last.relres = relres;
    c->last.converged = conv ? 1 : 0;
    if (!conv) {
        c->err = "GMRES reached gmres_maxit without converging (best iterate kept)";
        return GX_ENOCONV;
    }
    return GX_OK;
}
