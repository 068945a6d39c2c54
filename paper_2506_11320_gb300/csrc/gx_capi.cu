// gx_capi.cu -- the C ABI of include/gx.h: context life cycle, argument
// checking, host orchestration of one GL-ECSIM step and read-back.
//
// One step (Sec. 1.1, 1.2, 2.1, 2.2 of the paper) is
//   gx_field_solve:      LF coefficients from E^n, right-hand side, FGMRES for
//                        E^{n+theta}, then B^{n+1} and E^{n+1};
//   gx_push_and_deposit: fused mover + re-bin + deposit of step n+1, then the
//                        grid-side assembly of rho, u, J and M.
// All device work is enqueued on the caller's stream.
#include <cstdio>
#include <cstring>
#include <initializer_list>

#include "gx_internal.cuh"

int gx_copy_uref(gx_ctx *c, int zero, cudaStream_t st);
void gx_free_bins(gx_ctx *c);

namespace {

cudaStream_t S(void *p) { return reinterpret_cast<cudaStream_t>(p); }

template <class T>
int dalloc(gx_ctx *c, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) return GX_OK;
    cudaError_t e = cudaMalloc(p, count * sizeof(T));
    if (e != cudaSuccess) {
        c->err = std::string("cudaMalloc failed: ") + cudaGetErrorString(e);
        return GX_ENOMEM;
    }
    return GX_OK;
}

#define TRY(x)                       \
    do {                             \
        int rc_ = (x);               \
        if (rc_ != GX_OK) return rc_; \
    } while (0)

int copy_in(gx_ctx *c, void *dst, const void *src, size_t bytes, int is_dev, cudaStream_t st) {
    GX_CHECK(c, cudaMemcpyAsync(dst, src, bytes, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    return GX_OK;
}
int copy_out(gx_ctx *c, void *dst, const void *src, size_t bytes, int is_dev, cudaStream_t st) {
    GX_CHECK(c, cudaMemcpyAsync(dst, src, bytes, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    return GX_OK;
}

thread_local std::string g_create_err;

// any non-finite value among n entries -> *bad = 1 (input validation of the
// host or device arrays a caller passes in)
template <class T>
__global__ void k_nonfinite(int64_t n, const T *__restrict__ a, int *bad) {
    bool b = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b |= !isfinite(a[i]);
    if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) atomicExch(bad, 1);
}

__global__ void k_sum_sq(int64_t n, const float *__restrict__ a, double *out) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)a[i] * (double)a[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// 1 if any of the arrays (device copies) holds a NaN or an infinity
template <class T>
int any_nonfinite(gx_ctx *c, std::initializer_list<std::pair<const T *, int64_t>> arrays, cudaStream_t st, int *out) {
    int *bad = &c->dflags->invalid;
    GX_CHECK(c, cudaMemsetAsync(bad, 0, sizeof(int), st));
    for (auto &a : arrays) {
        if (!a.first || a.second <= 0) continue;
        const int64_t blocks = std::min<int64_t>((a.second + 255) / 256, 152 * 8);
        k_nonfinite<T><<<(unsigned)blocks, 256, 0, st>>>(a.second, a.first, bad);
        GX_LAUNCHED(c);
    }
    GX_CHECK(c, cudaMemcpyAsync(&c->hflags->invalid, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    GX_CHECK(c, cudaStreamSynchronize(st));
    *out = c->hflags->invalid;
    return GX_OK;
}

// CUDA-event timing on the launching stream.  Start/stop pairs are recorded
// without synchronising and resolved later (gx_timers, or when many pile up),
// so timing adds no host round trip to a step.
cudaEvent_t ev_get(gx_ctx *c) {
    if (!c->evpool.empty()) {
        cudaEvent_t e = c->evpool.back();
        c->evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void ev_resolve(gx_ctx *c) {
    double *acc[4] = {&c->t_push, &c->t_mom, &c->t_solve, &c->t_pdk};
    for (int k = 0; k < 4; ++k) {
        for (auto &pr : c->evpend[k]) {
            cudaEventSynchronize(pr.second);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, pr.first, pr.second);
            *acc[k] += ms;
            c->evpool.push_back(pr.first);
            c->evpool.push_back(pr.second);
        }
        c->evpend[k].clear();
    }
}

struct EvTimer {
    gx_ctx *c;
    cudaStream_t st;
    int cat;
    cudaEvent_t a;
    EvTimer(gx_ctx *c_, cudaStream_t s, int k) : c(c_), st(s), cat(k), a(ev_get(c_)) { cudaEventRecord(a, st); }
    void stop() {
        cudaEvent_t b = ev_get(c);
        cudaEventRecord(b, st);
        c->evpend[cat].push_back({a, b});
        if (c->evpend[cat].size() > 512) ev_resolve(c);
    }
    // stop and return this interval's time now (synchronises on the event)
    double stop_now() {
        cudaEvent_t b = ev_get(c);
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        c->evpool.push_back(a);
        c->evpool.push_back(b);
        return ms;
    }
};

// Deposit of the current state.  With the comoving current the bulk velocity
// is needed first (Sec. 2.1): a first deposit with u_ref = 0 gives rho_m and P,
// hence u; the second deposit subtracts u at every particle, so the current is
// summed from small deviations.
int deposit_now(gx_ctx *c, cudaStream_t st) {
    TRY(gx_node_fields(c, nullptr, c->B, nullptr, c->nB, st));
    if (c->cfg.comoving) {
        TRY(gx_copy_uref(c, 1, st));
        TRY(gx_run_deposit(c, st));
        TRY(gx_assemble_moments(c, st));          // u from this pass; uref <- u
    } else {
        TRY(gx_copy_uref(c, 1, st));
    }
    TRY(gx_run_deposit(c, st));
    TRY(gx_assemble_moments(c, st));
    c->moments_valid = 1;
    return GX_OK;
}

int check_flags(gx_ctx *c, cudaStream_t st) {
    GX_CHECK(c, cudaMemcpyAsync(c->hflags, c->dflags, sizeof(DevFlags), cudaMemcpyDeviceToHost, st));
    GX_CHECK(c, cudaStreamSynchronize(st));
    if (c->hflags->overflow || c->hflags->cfl || c->hflags->timeout) {
        // report once: clear the device flags so the context stays usable
        GX_CHECK(c, cudaMemsetAsync(c->dflags, 0, 3 * sizeof(int), st));
    }
    if (c->hflags->timeout) {
        c->err = "a bounded device wait (bulk copy or tensor-core step) gave up";
        return GX_ETIMEOUT;
    }
    if (c->hflags->overflow) {
        c->err = "a cell bin overflowed: particles were lost (raise bin_slack)";
        return GX_EOVERFLOW;
    }
    if (c->hflags->cfl) {
        c->err = "a particle moved more than one cell in one step (reduce dt)";
        return GX_ECFL;
    }
    return GX_OK;
}

}  // namespace

cudaEvent_t gx_ev_get(gx_ctx *c) { return ev_get(c); }

int gx_sum_squares(gx_ctx *c, const float *a, int64_t n, cudaStream_t st, double *out) {
    double *acc = c->dred;
    GX_CHECK(c, cudaMemsetAsync(acc, 0, sizeof(double), st));
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_sum_sq<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, st>>>(n, a, acc);
    GX_LAUNCHED(c);
    GX_CHECK(c, cudaMemcpyAsync(out, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
    GX_CHECK(c, cudaStreamSynchronize(st));
    return GX_OK;
}
void gx_ev_push(gx_ctx *c, int cat, cudaEvent_t a, cudaEvent_t b) {
    c->evpend[cat].push_back({a, b});
    if (c->evpend[cat].size() > 512) ev_resolve(c);
}

extern "C" {

const char *gx_status_string(int s) {
    switch (s) {
        case GX_OK: return "ok";
        case GX_EINVAL: return "invalid argument";
        case GX_ENOMEM: return "out of memory";
        case GX_ECUDA: return "CUDA error";
        case GX_ENOCONV: return "GMRES did not converge";
        case GX_ECFL: return "particle moved more than one cell";
        case GX_ETIMEOUT: return "device wait timed out";
        case GX_ENOTIMPL: return "not implemented";
        case GX_EOVERFLOW: return "particle bin overflow";
        case GX_ESTATE: return "call out of order";
        default: return "unknown status";
    }
}

const char *gx_last_error(gx_ctx *c) { return c ? c->err.c_str() : g_create_err.c_str(); }

void gx_destroy(gx_ctx *c) {
    if (!c) return;
    gx_net_free(c);
    gx_free_bins(c);
    double **dp[] = {&c->E, &c->B, &c->Eth, &c->Enew, &c->Bnew, &c->rho, &c->rho_m, &c->P, &c->u, &c->J,
                     &c->M, &c->tmp3, &c->uref64, &c->kappa, &c->rhs, &c->EM, &c->jdiag, &c->V, &c->Z,
                     &c->w, &c->r, &c->dred, &c->hcol, &c->dBlf, &c->A3};
    for (auto p : dp)
        if (*p) cudaFree(*p);
    if (c->jdiag32) cudaFree(c->jdiag32);
    float **f32[] = {&c->M32, &c->kappa32, &c->A3f};
    for (auto p : f32)
        if (*p) cudaFree(*p);
    if (c->phi) cudaFree(c->phi);
    float4 **fp[] = {&c->nE, &c->nB, &c->nBnext, &c->nUref};
    for (auto p : fp)
        if (*p) cudaFree(*p);
    if (c->rec) cudaFree(c->rec);
    if (c->gm) cudaFree(c->gm);
    if (c->gpart) cudaFree(c->gpart);
    if (c->dflags) cudaFree(c->dflags);
    if (c->hflags) cudaFreeHost(c->hflags);
    if (c->hpin) cudaFreeHost(c->hpin);
    for (auto &v : c->evpend)
        for (auto &pr : v) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (auto e : c->evpool) cudaEventDestroy(e);
    delete c;
}

int gx_create(const gx_config *cfg, gx_ctx **out) {
    if (!cfg || !out) return GX_EINVAL;
    *out = nullptr;
    gx_ctx *c = new gx_ctx();
    c->cfg = *cfg;
    g_create_err.clear();
    auto fail = [&](int rc, const char *msg) {
        if (msg) c->err = msg;
        g_create_err = c->err;
        gx_destroy(c);
        return rc;
    };
    for (int d = 0; d < 3; ++d) {
        if (cfg->n[d] < 1) return fail(GX_EINVAL, "n[d] must be >= 1");
        if (!(cfg->dx[d] > 0)) return fail(GX_EINVAL, "dx[d] must be > 0");
        c->n[d] = cfg->n[d];
    }
    if ((int64_t)cfg->n[0] * cfg->n[1] > (int64_t)1 << 31 ||
        (int64_t)cfg->n[0] * cfg->n[1] * cfg->n[2] > (int64_t)1 << 31)
        return fail(GX_EINVAL, "at most 2^31 cells");
    const bool three = cfg->n[2] > 1;
    if (three && (cfg->bc_cells > 0 || cfg->bc_wall || cfg->divb_clean || cfg->precond == GX_PRECOND_NET))
        return fail(GX_ENOTIMPL, "a 3D grid runs periodic, without divb_clean and without the learned preconditioner");
    if (!(cfg->c > 0) || !(cfg->dt > 0)) return fail(GX_EINVAL, "c and dt must be > 0");
    if (!(cfg->theta >= 0.5 && cfg->theta <= 1.0)) return fail(GX_EINVAL, "theta must be in [0.5, 1]");
    if (cfg->gmres_restart < 1 || cfg->gmres_restart > gx_gm_max_restart())
        return fail(GX_EINVAL, "gmres_restart must be in [1, 64]");
    if (cfg->gmres_maxit < 1) return fail(GX_EINVAL, "gmres_maxit must be >= 1");
    if (!(cfg->gmres_tol > 0)) return fail(GX_EINVAL, "gmres_tol must be > 0");
    if (cfg->precond < 0 || cfg->precond > 2) return fail(GX_EINVAL, "precond must be 0, 1 or 2");
    if (cfg->nsmooth_u < 0 || cfg->ns_j < 0 || cfg->nsmooth_e < 0)
        return fail(GX_EINVAL, "smoothing passes must be >= 0");
    if (cfg->nsmooth_e > 10) return fail(GX_EINVAL, "nsmooth_e must be <= 10");
    if (cfg->bc_cells < 0 || (cfg->bc_cells > 0 && (cfg->bc_cells < 8 || 2 * cfg->bc_cells >= cfg->n[0])))
        return fail(GX_EINVAL, "bc_cells must be 0 or >= 8 with 2 bc_cells < nx");
    if (cfg->bc_cells > 0 && cfg->divb_clean) return fail(GX_EINVAL, "open boundaries without divb_clean");
    if (cfg->bc_wall && cfg->bc_cells <= 0) return fail(GX_EINVAL, "a reflecting wall needs bc_cells > 0");
    if (cfg->bc_cells > 0 && cfg->nsmooth_e > 0)   // the filter would move the held boundary E
        return fail(GX_EINVAL, "open boundaries without nsmooth_e");
    if (cfg->lf_on && !(cfg->lf_beta >= 0 && cfg->lf_beta < 1e300)) return fail(GX_EINVAL, "lf_beta must be >= 0");
    if (!(cfg->gl_gamma >= 0 && cfg->gl_gamma <= 1)) return fail(GX_EINVAL, "gl_gamma must be in [0, 1]");
    if (cfg->gmres_mixed != 0 && cfg->gmres_mixed != 1) return fail(GX_EINVAL, "gmres_mixed must be 0 or 1");
    if (cfg->gmres_mixed && cfg->precond == GX_PRECOND_NET)
        return fail(GX_EINVAL, "gmres_mixed is not combined with the learned preconditioner");
    if (cfg->gl_gamma > 0 && cfg->bc_cells > 0) return fail(GX_EINVAL, "gl_gamma needs a periodic grid (no bc_cells)");
    if (!(cfg->c < 1e300) || !(cfg->dt < 1e300) || !(cfg->gmres_tol < 1e300) || !(cfg->bin_slack == cfg->bin_slack))
        return fail(GX_EINVAL, "c, dt, gmres_tol and bin_slack must be finite");
    for (int d = 0; d < 3; ++d)
        if (!(cfg->dx[d] < 1e300)) return fail(GX_EINVAL, "dx[d] must be finite");
    c->dim = three ? 3 : 2;
    c->N = (int64_t)c->n[0] * c->n[1] * c->n[2];
    c->dV = cfg->dx[0] * cfg->dx[1] * cfg->dx[2];
    c->noff = three ? 27 : 9;
    const int64_t N = c->N;
    const int m = cfg->gmres_restart;
    int rc = GX_OK;
    double **vec3[] = {&c->E, &c->B, &c->Eth, &c->Enew, &c->Bnew, &c->P, &c->u, &c->J, &c->tmp3, &c->uref64,
                       &c->rhs, &c->EM, &c->w, &c->r};
    for (auto p : vec3)
        if ((rc = dalloc(c, p, 3 * N))) return fail(rc, nullptr);
    const int nax = three ? 3 : 2;
    if ((rc = dalloc(c, &c->rho, N)) || (rc = dalloc(c, &c->rho_m, N)) || (rc = dalloc(c, &c->M, (size_t)c->noff * 9 * N)) ||
        (rc = dalloc(c, &c->kappa, (size_t)nax * 3 * N)) || (three && (rc = dalloc(c, &c->A3, (size_t)243 * N))) || (rc = dalloc(c, &c->jdiag, 9 * N)) || (rc = dalloc(c, &c->jdiag32, 9 * N)) ||
        (rc = dalloc(c, &c->V, (size_t)(m + 1) * 3 * N)) || (rc = dalloc(c, &c->dred, 64)) ||
        (rc = dalloc(c, &c->hcol, 2 * (m + 2))) || (rc = dalloc(c, &c->dflags, 1)))
        return fail(rc, nullptr);
    if (cfg->precond != GX_PRECOND_NONE && (rc = dalloc(c, &c->Z, (size_t)m * 3 * N))) return fail(rc, nullptr);
    if (cfg->gmres_mixed &&
        (three ? (rc = dalloc(c, &c->A3f, (size_t)243 * N))
               : ((rc = dalloc(c, &c->M32, (size_t)c->noff * 9 * N)) || (rc = dalloc(c, &c->kappa32, (size_t)nax * 3 * N)))))
        return fail(rc, nullptr);
    if (cfg->lf_on && (rc = dalloc(c, &c->dBlf, (size_t)(6 + 3 * nax) * N))) return fail(rc, nullptr);   // D, B~, face fluxes
    if (cfg->divb_clean) {
        if ((rc = dalloc(c, &c->phi, N))) return fail(rc, nullptr);
        if (cudaMemset(c->phi, 0, N * sizeof(double)) != cudaSuccess) return fail(GX_ECUDA, "cudaMemset failed");
    }
    {
        char *gm = nullptr;
        if ((rc = dalloc(c, &gm, gx_gm_state_bytes())) || (rc = dalloc(c, &c->gpart, gx_gm_partial_count())))
            return fail(rc, nullptr);
        c->gm = reinterpret_cast<GmState *>(gm);
        if (cudaMemset(gm, 0, gx_gm_state_bytes()) != cudaSuccess) return fail(GX_ECUDA, "cudaMemset failed");
    }
    float4 **nodes[] = {&c->nE, &c->nB, &c->nBnext, &c->nUref};
    for (auto p : nodes)
        if ((rc = dalloc(c, p, N))) return fail(rc, nullptr);
    if (cudaMallocHost(&c->hpin, 2 * (m + 2) * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->hflags, sizeof(DevFlags)) != cudaSuccess)
        return fail(GX_ENOMEM, "pinned host allocation failed");
    std::memset(c->hflags, 0, sizeof(DevFlags));
    c->rec_size = c->dim == 3 ? Rec<3>::SIZE : Rec<2>::SIZE;
    if ((rc = dalloc(c, &c->rec, (size_t)GX_MAX_SPECIES * rec_block(c->rec_size, N)))) return fail(rc, nullptr);
    double *zero3[] = {c->E, c->B, c->Eth, c->Enew, c->Bnew, c->u, c->J, c->uref64};
    for (auto p : zero3)
        if (cudaMemset(p, 0, 3 * N * sizeof(double)) != cudaSuccess) return fail(GX_ECUDA, "cudaMemset failed");
    if (cudaMemset(c->M, 0, (size_t)c->noff * 9 * N * sizeof(double)) != cudaSuccess ||
        cudaMemset(c->rho, 0, N * sizeof(double)) != cudaSuccess ||
        cudaMemset(c->kappa, 0, (size_t)nax * 3 * N * sizeof(double)) != cudaSuccess ||
        cudaMemset(c->dflags, 0, sizeof(DevFlags)) != cudaSuccess ||
        cudaMemset(c->nUref, 0, N * sizeof(float4)) != cudaSuccess ||
        (c->M32 && cudaMemset(c->M32, 0, (size_t)c->noff * 9 * N * sizeof(float)) != cudaSuccess) ||
        (c->kappa32 && cudaMemset(c->kappa32, 0, (size_t)nax * 3 * N * sizeof(float)) != cudaSuccess) ||
        (c->A3f && cudaMemset(c->A3f, 0, (size_t)243 * N * sizeof(float)) != cudaSuccess) ||
        cudaDeviceSynchronize() != cudaSuccess)
        return fail(GX_ECUDA, "initialisation failed");
    if ((rc = gx_noalloc_prepare(c))) return fail(rc, nullptr);
    *out = c;
    return GX_OK;
}

int gx_species_add(gx_ctx *c, double q, double m, int64_t n, const double *x, const double *y, const double *z,
                   const float *vx, const float *vy, const float *vz, const float *w, int ptr_is_device,
                   int *species_id) {
    if (!c) return GX_EINVAL;
    if (c->nspecies >= GX_MAX_SPECIES) { c->err = "at most 4 species"; return GX_EINVAL; }
    if (!(m > 0) || q == 0.0 || n < 0 || n > (int64_t)2000000000) { c->err = "need q != 0, m > 0, 0 <= n < 2^31"; return GX_EINVAL; }
    if (n > 0 && (!x || !y || !vx || !vy || !vz || !w || (c->dim == 3 && !z))) {
        c->err = "null particle array";
        return GX_EINVAL;
    }
    cudaStream_t st = 0;
    const int s = c->nspecies;
    c->sp[s].q = q;
    c->sp[s].m = m;
    double *dx_ = nullptr, *dy_ = nullptr, *dz_ = nullptr;
    float *dvx = nullptr, *dvy = nullptr, *dvz = nullptr, *dw = nullptr;
    const double *px = x, *py = y, *pz = c->dim == 3 ? z : nullptr;
    const float *pvx = vx, *pvy = vy, *pvz = vz, *pw = w;
    if (!ptr_is_device && n > 0) {
        TRY(dalloc(c, &dx_, n)); TRY(dalloc(c, &dy_, n));
        TRY(dalloc(c, &dvx, n)); TRY(dalloc(c, &dvy, n)); TRY(dalloc(c, &dvz, n)); TRY(dalloc(c, &dw, n));
        TRY(copy_in(c, dx_, x, n * sizeof(double), 0, st)); TRY(copy_in(c, dy_, y, n * sizeof(double), 0, st));
        TRY(copy_in(c, dvx, vx, n * sizeof(float), 0, st)); TRY(copy_in(c, dvy, vy, n * sizeof(float), 0, st));
        TRY(copy_in(c, dvz, vz, n * sizeof(float), 0, st)); TRY(copy_in(c, dw, w, n * sizeof(float), 0, st));
        if (pz) {
            TRY(dalloc(c, &dz_, n));
            TRY(copy_in(c, dz_, z, n * sizeof(double), 0, st));
            pz = dz_;
        }
        px = dx_; py = dy_; pvx = dvx; pvy = dvy; pvz = dvz; pw = dw;
    }
    int rc = GX_OK, bad = 0;
    if (n > 0) {
        // a NaN or an infinity would bin a particle nowhere in particular: refuse the species
        rc = any_nonfinite<double>(c, {{px, n}, {py, n}, {pz, pz ? n : 0}}, st, &bad);
        if (!rc && !bad) rc = any_nonfinite<float>(c, {{pvx, n}, {pvy, n}, {pvz, n}, {pw, n}}, st, &bad);
        if (!rc && bad) { c->err = "gx_species_add: a position, velocity or weight is not finite"; rc = GX_EINVAL; }
    }
    if (!rc) rc = gx_bin_particles(c, s, n, px, py, pz, pvx, pvy, pvz, pw, nullptr, st);
    c->sp[s].w2 = 0.0;
    if (!rc && n > 0) rc = gx_sum_squares(c, pw, n, st, &c->sp[s].w2);
    if (dx_) { cudaFree(dx_); cudaFree(dy_); cudaFree(dvx); cudaFree(dvy); cudaFree(dvz); cudaFree(dw); }
    if (dz_) cudaFree(dz_);
    if (rc) return rc;
    TRY(check_flags(c, st));
    c->nspecies++;
    c->np_total += n;
    c->moments_valid = 0;
    c->pending = 0;
    if (species_id) *species_id = s;
    return GX_OK;
}

int gx_species_maxwellian(gx_ctx *c, double q, double m, int ppc, double n0, const double *u, double vth,
                          int *species_id) {
    if (!c) return GX_EINVAL;
    if (c->nspecies >= GX_MAX_SPECIES) { c->err = "at most 4 species"; return GX_EINVAL; }
    if (!(m > 0) || q == 0.0 || !u || ppc < 1 || ppc > 4096 || !(n0 >= 0.0) || !(vth >= 0.0) ||
        (int64_t)ppc * c->N > (int64_t)2000000000) {
        c->err = "gx_species_maxwellian: q != 0, m > 0, 1 <= ppc <= 4096, n0 >= 0, vth >= 0, under 2^31 particles";
        return GX_EINVAL;
    }
    const int s = c->nspecies;
    c->sp[s].q = q;
    c->sp[s].m = m;
    TRY(gx_species_maxwellian_init(c, s, ppc, n0, u, vth, 0));
    const double wm = (double)(float)(n0 * c->dV / ppc);          // every particle's FP32 weight
    c->sp[s].w2 = (double)ppc * (double)c->N * wm * wm;
    c->nspecies++;
    c->np_total += (int64_t)ppc * c->N;
    c->moments_valid = 0;
    c->pending = 0;
    if (species_id) *species_id = s;
    return GX_OK;
}

int gx_fields_set(gx_ctx *c, const double *E, const double *B, int ptr_is_device) {
    if (!c) return GX_EINVAL;
    const size_t bytes = 3 * c->N * sizeof(double);
    // validate in the scratch vectors first, so that refused fields leave E^n and B^n as they were
    if (E) TRY(copy_in(c, c->w, E, bytes, ptr_is_device, 0));
    if (B) TRY(copy_in(c, c->r, B, bytes, ptr_is_device, 0));
    int bad = 0;
    TRY(any_nonfinite<double>(c, {{E ? c->w : nullptr, 3 * c->N}, {B ? c->r : nullptr, 3 * c->N}}, 0, &bad));
    if (bad) { c->err = "gx_fields_set: E or B holds a value that is not finite"; return GX_EINVAL; }
    if (E) TRY(copy_in(c, c->E, c->w, bytes, 1, 0));
    if (B) TRY(copy_in(c, c->B, c->r, bytes, 1, 0));
    if (B && c->phi) GX_CHECK(c, cudaMemsetAsync(c->phi, 0, c->N * sizeof(double), 0));
    GX_CHECK(c, cudaStreamSynchronize(0));
    c->moments_valid = 0;
    c->pending = 0;
    c->have_eth = 0;
    return GX_OK;
}

int gx_boundary_source(gx_ctx *c, int side, int species, double n, const double *u, double vth, int ppc) {
    if (!c) return GX_EINVAL;
    if (c->cfg.bc_cells <= 0) { c->err = "gx_boundary_source needs cfg.bc_cells > 0"; return GX_EINVAL; }
    if (side < 0 || side > 1 || species < 0 || species >= c->nspecies || !u || !(n >= 0.0) || !(vth >= 0.0) ||
        ppc < 1 || ppc > 4096) {
        c->err = "gx_boundary_source: side 0/1, an existing species, n >= 0, vth >= 0, 1 <= ppc <= 4096";
        return GX_EINVAL;
    }
    BcSource &b = c->bsrc[side][species];
    b.n = n;
    b.u[0] = u[0]; b.u[1] = u[1]; b.u[2] = u[2];
    b.vth = vth;
    b.ppc = ppc;
    // the refilled bins must hold ppc particles
    if (ppc > c->sp[species].cap) TRY(gx_regrow_bins(c, species, ppc + ppc / 2, 0));
    return GX_OK;
}

int gx_deposit(gx_ctx *c, void *stream) {
    if (!c) return GX_EINVAL;
    cudaStream_t st = S(stream);
    EvTimer t(c, st, 1);
    TRY(deposit_now(c, st));
    t.stop();
    return GX_OK;
}

int gx_field_solve(gx_ctx *c, void *stream, gx_solve_stats *stats) {
    if (!c) return GX_EINVAL;
    cudaStream_t st = S(stream);
    if (!c->moments_valid) {
        EvTimer t(c, st, 1);
        TRY(deposit_now(c, st));
        t.stop();
    }
    EvTimer t(c, st, 2);
    TRY(gx_build_kappa(c, st));
    TRY(gx_build_rhs(c, st));
    TRY(gx_initial_guess(c, st));
    int rc = gx_fgmres(c, st);
    if (rc != GX_OK && rc != GX_ENOCONV) return rc;
    TRY(gx_advance(c, st));
    TRY(gx_node_fields(c, c->Eth, c->Bnew, c->nE, c->nBnext, st));
    const double ms = t.stop_now();
    c->t_solve += ms;
    c->last.ms = ms;
    if (stats) *stats = c->last;
    c->pending = 1;
    return rc;
}

int gx_push_and_deposit(gx_ctx *c, void *stream) {
    if (!c) return GX_EINVAL;
    if (!c->pending) { c->err = "gx_push_and_deposit needs a preceding gx_field_solve"; return GX_ESTATE; }
    if (c->cfg.bc_cells > 0)      // refuse before anything is launched
        for (int s = 0; s < c->nspecies; ++s)
            for (int sd = 0; sd < (c->cfg.bc_wall ? 1 : 2); ++sd)
                if (c->bsrc[sd][s].ppc < 1) {
                    c->err = "open boundaries need gx_boundary_source for every species on both sides";
                    return GX_ESTATE;
                }
    cudaStream_t st = S(stream);
    // grow a species' bins when the last step left one above 90 % of capacity
    if (c->hflags->maxcount > 0) {
        for (int s = 0; s < c->nspecies; ++s)
            if (c->hflags->maxcount > 0.9 * c->sp[s].cap)
                TRY(gx_regrow_bins(c, s, ((int)(c->hflags->maxcount * 1.5) + 31) / 32 * 32, st));
    }
    {
        EvTimer t(c, st, 0);
        if (c->cfg.gl_gamma > 0) TRY(c->dim == 3 ? gx3_gl_potential(c, st) : gx_gl_potential(c, st));
        TRY(gx_run_push_deposit(c, st));
        t.stop();
    }
    std::swap(c->E, c->Enew);
    std::swap(c->B, c->Bnew);
    std::swap(c->nB, c->nBnext);
    c->have_eth = 1;
    {
        EvTimer t(c, st, 1);
        TRY(gx_assemble_moments(c, st));
        t.stop();
    }
    c->moments_valid = 1;
    c->pending = 0;
    return check_flags(c, st);
}

int gx_step(gx_ctx *c, int nsteps, void *stream, gx_solve_stats *last) {
    if (!c || nsteps < 0) return GX_EINVAL;
    int status = GX_OK;
    for (int k = 0; k < nsteps; ++k) {
        int rc = gx_field_solve(c, stream, last);
        if (rc == GX_ENOCONV) status = rc;
        else if (rc) return rc;
        rc = gx_push_and_deposit(c, stream);
        if (rc) return rc;
    }
    return status;
}

int gx_get_fields(gx_ctx *c, double *E, double *B, int ptr_is_device) {
    if (!c) return GX_EINVAL;
    const size_t bytes = 3 * c->N * sizeof(double);
    if (E) TRY(copy_out(c, E, c->E, bytes, ptr_is_device, 0));
    if (B) TRY(copy_out(c, B, c->B, bytes, ptr_is_device, 0));
    GX_CHECK(c, cudaStreamSynchronize(0));
    return GX_OK;
}

int gx_get_solution(gx_ctx *c, double *Eth, int ptr_is_device) {
    if (!c || !Eth) return GX_EINVAL;
    TRY(copy_out(c, Eth, c->Eth, 3 * c->N * sizeof(double), ptr_is_device, 0));
    GX_CHECK(c, cudaStreamSynchronize(0));
    return GX_OK;
}

int gx_get_moments(gx_ctx *c, double *rho, double *J, double *M, double *u, int ptr_is_device) {
    if (!c) return GX_EINVAL;
    if (!c->moments_valid) TRY(deposit_now(c, 0));
    const int64_t N = c->N;
    if (rho) TRY(copy_out(c, rho, c->rho, N * sizeof(double), ptr_is_device, 0));
    if (J) TRY(copy_out(c, J, c->J, 3 * N * sizeof(double), ptr_is_device, 0));
    if (u) TRY(copy_out(c, u, c->u, 3 * N * sizeof(double), ptr_is_device, 0));
    if (M) {
        // device rows are [noff * 9][N] (entry o*9 + e); node-major 27-offset layout
        // for the caller (in 2D the 9 in-plane offsets are oz = 0: offset + 9)
        const int rows = c->noff * 9, base = c->dim == 3 ? 0 : 81;
        std::vector<double> h((size_t)rows * N), full((size_t)243 * N, 0.0);
        GX_CHECK(c, cudaMemcpy(h.data(), c->M, (size_t)rows * N * sizeof(double), cudaMemcpyDeviceToHost));
        for (int64_t q = 0; q < N; ++q)
            for (int k = 0; k < rows; ++k) full[(size_t)q * 243 + base + k] = h[(size_t)k * N + q];
        if (ptr_is_device) GX_CHECK(c, cudaMemcpy(M, full.data(), 243 * N * sizeof(double), cudaMemcpyHostToDevice));
        else std::memcpy(M, full.data(), 243 * N * sizeof(double));
    }
    GX_CHECK(c, cudaStreamSynchronize(0));
    return GX_OK;
}

int64_t gx_species_count(gx_ctx *c, int s) {
    if (!c || s < 0 || s >= c->nspecies) return -1;
    std::vector<int> h(c->N);
    if (cudaMemcpy(h.data(), c->sp[s].cnt[c->cur], c->N * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    int64_t t = 0;
    for (int v : h) t += std::min(bin_count(v), c->sp[s].cap);
    return t;
}

int gx_get_particles(gx_ctx *c, int s, double *x, double *y, double *z, float *vx, float *vy, float *vz, float *w,
                     int32_t *id, int ptr_is_device) {
    if (!c || s < 0 || s >= c->nspecies) return GX_EINVAL;
    if (id && !c->cfg.track_ids) { c->err = "ids need track_ids"; return GX_EINVAL; }
    const int64_t n = gx_species_count(c, s);
    if (n < 0) return GX_ECUDA;
    if (ptr_is_device) return gx_particles_out(c, s, x, y, z, vx, vy, vz, w, id, 0);
    double *dx_ = nullptr, *dy_ = nullptr, *dz_ = nullptr;
    float *dvx = nullptr, *dvy = nullptr, *dvz = nullptr, *dw = nullptr;
    int32_t *did = nullptr;
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    if (x) TRY(dalloc(c, &dx_, nn));
    if (y) TRY(dalloc(c, &dy_, nn));
    if (z) TRY(dalloc(c, &dz_, nn));
    if (vx) TRY(dalloc(c, &dvx, nn));
    if (vy) TRY(dalloc(c, &dvy, nn));
    if (vz) TRY(dalloc(c, &dvz, nn));
    if (w) TRY(dalloc(c, &dw, nn));
    if (id) TRY(dalloc(c, &did, nn));
    int rc = gx_particles_out(c, s, dx_, dy_, dz_, dvx, dvy, dvz, dw, did, 0);
    if (!rc) {
        if (x) rc |= cudaMemcpy(x, dx_, n * sizeof(double), cudaMemcpyDeviceToHost);
        if (y) rc |= cudaMemcpy(y, dy_, n * sizeof(double), cudaMemcpyDeviceToHost);
        if (z) rc |= cudaMemcpy(z, dz_, n * sizeof(double), cudaMemcpyDeviceToHost);
        if (vx) rc |= cudaMemcpy(vx, dvx, n * sizeof(float), cudaMemcpyDeviceToHost);
        if (vy) rc |= cudaMemcpy(vy, dvy, n * sizeof(float), cudaMemcpyDeviceToHost);
        if (vz) rc |= cudaMemcpy(vz, dvz, n * sizeof(float), cudaMemcpyDeviceToHost);
        if (w) rc |= cudaMemcpy(w, dw, n * sizeof(float), cudaMemcpyDeviceToHost);
        if (id) rc |= cudaMemcpy(id, did, n * sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (rc) { c->err = "particle copy-out failed"; rc = GX_ECUDA; }
    }
    void *ps[] = {dx_, dy_, dz_, dvx, dvy, dvz, dw, did};
    for (void *p : ps)
        if (p) cudaFree(p);
    return rc;
}

int gx_diagnostics(gx_ctx *c, void *stream, gx_diag *out) {
    if (!c || !out) return GX_EINVAL;
    cudaStream_t st = S(stream);
    if (!c->moments_valid && c->nspecies > 0) TRY(deposit_now(c, st));
    return gx_diag_run(c, out, st);
}

int gx_timers(gx_ctx *c, double *push_ms, double *moments_ms, double *solve_ms, int64_t *launches, int reset) {
    if (!c) return GX_EINVAL;
    ev_resolve(c);
    if (push_ms) *push_ms = c->t_push;
    if (moments_ms) *moments_ms = c->t_mom;
    if (solve_ms) *solve_ms = c->t_solve;
    if (launches) *launches = c->launches;
    if (reset) { c->t_push = c->t_mom = c->t_solve = 0; c->launches = 0; }
    return GX_OK;
}

int gx_kernel_timer(gx_ctx *c, double *pd_ms, int64_t *pd_launches, int reset) {
    if (!c) return GX_EINVAL;
    ev_resolve(c);
    if (pd_ms) *pd_ms = c->t_pdk;
    if (pd_launches) *pd_launches = c->n_pdk;
    if (reset) { c->t_pdk = 0; c->n_pdk = 0; }
    return GX_OK;
}

}  // extern "C"
