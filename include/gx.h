/*
 * gx.h -- C ABI of the GB300 GL-ECSIM hot-path library (libgx.so).
 *
 * The library implements one time step of the semi-implicit particle-in-cell
 * method of Chen, Zhou & Toth, "Suppressing spurious oscillations and particle
 * noise in particle-in-cell simulations" (arXiv 2506.11320): the theta-implicit
 * particle mover, the particle-to-grid moments it feeds (charge density, the
 * comoving-frame current, the ECSIM mass matrices), and the implicit field solve
 * with the limited Lax-Friedrichs terms.  Section and equation numbers below
 * refer to that paper: Sec. 1.1 "Discretization of Maxwell's equations", Sec. 1.2
 * "Suppressing spurious oscillations", Sec. 1.4 (the digital filter), Sec. 2.1
 * "Calculating current in the comoving frame", Sec. 2.2 "Smoothing the current".
 *
 * Conventions shared by every entry point:
 *   - Every function returns a status (GX_OK == 0) and never aborts or exits.
 *     On failure gx_last_error() describes the cause; the context stays usable
 *     unless the status is GX_ECUDA (a CUDA error: the device may need a reset).
 *   - Pointers are borrowed: the library copies data in and out during the call
 *     and keeps no caller pointer afterwards.  `ptr_is_device` says whether the
 *     caller's arrays live in host memory (0, pageable or pinned) or device
 *     memory of the context's GPU (1).  The library owns all of its device state.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued on it; calls that return host-visible results
 *     synchronise it before returning.
 *   - Units are Gaussian with an explicit speed of light c (Ampere's law
 *     dE/dt = c curl B - 4 pi J, Lorentz force q (E + v x B / c)).
 *   - Mesh (Sec. 1.1): collocated staggered grid, E at nodes, B at cell centres,
 *     periodic in every axis.  Node (i,j,k) sits at (i dx, j dy, k dz); cell
 *     (i,j,k) spans [i,i+1] x [j,j+1] x [k,k+1] cell widths.  Node and cell
 *     (i,j,k) share the flat index g = i + nx (j + ny k).  Vector fields are
 *     component-major FP64 arrays [3][nz][ny][nx].  n[2] == 1 selects the 2D
 *     (x-y, three velocity components) path; 3D needs every n[d] >= 2.
 */
#ifndef GX_H
#define GX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- statuses */
enum {
    GX_OK = 0,
    GX_EINVAL = 1,     /* bad argument or configuration */
    GX_ENOMEM = 2,     /* device or host allocation failed */
    GX_ECUDA = 3,      /* a CUDA runtime call or kernel failed */
    GX_ENOCONV = 4,    /* GMRES stopped at gmres_maxit; the best iterate is kept */
    GX_ECFL = 5,       /* a particle moved more than one cell in one step */
    GX_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
    GX_ENOTIMPL = 7,   /* feature not available for this configuration (e.g. 3D with divb_clean) */
    GX_EOVERFLOW = 8,  /* a cell's particle bin overflowed (particles were lost) */
    GX_ESTATE = 9      /* call out of order (e.g. push before a field solve) */
};

enum { GX_PRECOND_NONE = 0, GX_PRECOND_JACOBI = 1, GX_PRECOND_NET = 2 };

typedef struct gx_ctx gx_ctx;

/* Problem statement.  The method switches follow the paper:
 *   comoving   1: the current is computed in the comoving frame (Sec. 2.1,
 *                 Eq. 33-35): bulk velocity u first (mass-weighted plasma
 *                 velocity smoothed by nsmooth_u passes of the digital filter of
 *                 Eq. 26 with phi = 0.5 and strides 1,2,1,2,...), then the
 *                 deposit of the deviations v - u(x_p).
 *   lf_on      1: limited Lax-Friedrichs diffusion on B (explicit, Eq. 17-18)
 *                 and E (implicit, Eq. 19-20) with the MC limiter of Eq. 21,
 *                 parameter lf_beta; diffusion speed a = |u| (lf_speed_c = 0) or
 *                 a = c (lf_speed_c = 1, vacuum tests).
 *   ns_j          passes of the digital filter (phi = 0.5, d = 1) on the
 *                 comoving current (Sec. 2.2).
 *   theta         time centring of the theta scheme (Eq. 5-8), in [0.5, 1].
 *   gmres_*       FGMRES(restart) on the field equation, stopping at relative
 *                 residual gmres_tol or gmres_maxit matrix-vector products.
 *                 The solve starts from E^{n+theta} extrapolated linearly from
 *                 the previous step's solution and E^n (from E^n on the first
 *                 step and after gx_fields_set); the result does not depend on
 *                 the starting point beyond the tolerance.
 *   precond       GX_PRECOND_*: right preconditioner of the field solve.
 *   track_ids     1: carry a 32-bit particle id through the bins (testing).
 *   divb_clean 1: hyperbolic/parabolic cleaning of div B (Sec. 1.3): a scalar
 *                 phi at cell centres with d phi/dt + c_h^2 div B = -(c_h^2 /
 *                 c_p^2) phi and dB/dt = ... - grad phi, c_h = 0.8 dx/dt (dx:
 *                 the smaller cell width), dt c_h^2/c_p^2 = 0.1 (the paper's
 *                 settings).  Discretisation (the paper cites it from elsewhere):
 *                 central differences over neighbouring cells for div and grad,
 *                 B^{n+1} -= dt grad phi^n after the field advance, then
 *                 phi^{n+1} = exp(-0.1) (phi^n - dt c_h^2 div B^{n+1}).  phi
 *                 starts at zero and is reset by gx_fields_set.
 *   nsmooth_e     passes of the digital filter of Eq. 26 (phi = 0.5, strides
 *                 1, 2, 1, ...) on E^{n+1} after every step, in place of the
 *                 implicit LF term on E (the comparison of Sec. 3.1); the LF
 *                 term on B stays as lf_on says.  0: off.  At most 10 passes.
 *   bin_slack     capacity of a cell's particle bin relative to the largest
 *                 initial count (>= 1.2; the bins grow automatically when a
 *                 step finds one filled above 90 %).
 *   bc_cells      0: periodic along x.  G >= 8: open x boundaries (the shock
 *                 runs of Sec. 3.3): the G cells at each end hold a fixed
 *                 plasma state.  E at the nodes whose two x-neighbouring cells
 *                 are boundary cells and B in boundary cells keep their values
 *                 (Dirichlet rows in the E solve); after every push the
 *                 particles of every boundary cell are replaced by ppc fresh
 *                 particles per species drawn from that side's source (see
 *                 gx_boundary_source).  y stays periodic.  Not with divb_clean;
 *                 2 G < nx.  Not with nsmooth_e (the filter would move the held
 *                 boundary E).
 *   bc_wall       with bc_cells: 1 turns the high-x boundary cells into a
 *                 reflecting perfect conductor at rest (the shock-by-reflection
 *                 setup): they hold no particles and get no refill, E is held
 *                 (at its initial value, 0 for a conductor) from the wall face
 *                 x_w = (nx - G) dx on, B is held, and a particle crossing x_w
 *                 is reflected specularly (x -> 2 x_w - x, v_x -> -v_x).  Only
 *                 side 0 then needs gx_boundary_source.
 *   lf_rhs_printed with lf_on: 1 makes the right-hand side of the E solve curl
 *                 B^n, as Eq. 7 prints it; 0 (default) curls B^n + theta D, D
 *                 the LF increment that B^{n+1} receives (Eq. 17-18), the
 *                 B^{n+theta} that Eq. 7 comes from.  At theta = 1/2 and
 *                 c dt / dx >> 1 the printed form lets the shortest light modes
 *                 grow by about 1 + 2 a dt / dx per step.
 *   gl_gamma      > 0: the Gauss's-law position correction of GL-ECSIM (the
 *                 paper names it by citation; this library's reading): with
 *                 R_c = (div_C E^n)_c / (4 pi) - rhobar_c the Gauss residual of
 *                 cell c (rhobar the mean of the deposited charge density over
 *                 the cell's corner nodes) and phi_g the mean of R over the
 *                 cells around node g, every particle's position update of the
 *                 push gains dx_p = gl_gamma eps q_s w_p grad phi(x_p^{n+1/2}),
 *                 eps = 1 / (Q2 sum_d 4 / dx_d^2), Q2 = sum_p (q_s w_p)^2 / V:
 *                 one steepest-descent step on (dV / 2) sum_c R_c^2, which damps
 *                 every residual mode for 0 < gl_gamma <= 1.  0 (default): off.
 *                 Periodic grids only (not with bc_cells).
 *   gmres_mixed   1: mixed-precision FGMRES (iterative refinement).  Every
 *                 restart computes the true residual b - A x and updates x in
 *                 FP64; the Arnoldi cycles between restarts keep the Krylov
 *                 basis in FP32 and apply FP32 copies of the operator's
 *                 coefficients, with FP64 inner products, and each cycle stops
 *                 once its residual estimate has dropped by 1e-4.  The solve
 *                 still ends when the FP64 true residual reaches gmres_tol (the
 *                 relres of gx_solve_stats).  Costs 4 bytes per coefficient more
 *                 device memory; not with precond GX_PRECOND_NET.  0 (default):
 *                 all-FP64 FGMRES.
 *   seed          key of the context's counter-based draws (Philox4x64-10 with
 *                 key (seed, species)): the device-side Maxwellian species
 *                 (gx_species_maxwellian, counter (0, cell, particle, 0)) and the
 *                 boundary refill after push t (counter (t, cell, particle, 0)). */
typedef struct {
    int32_t n[3];
    int32_t comoving;
    int32_t lf_on;
    int32_t lf_speed_c;
    int32_t ns_j;
    int32_t nsmooth_u;
    int32_t gmres_restart;
    int32_t gmres_maxit;
    int32_t precond;
    int32_t track_ids;
    double dx[3];
    double c;
    double theta;
    double dt;
    double lf_beta;
    double gmres_tol;
    double bin_slack;
    int32_t divb_clean;
    int32_t nsmooth_e;
    int32_t bc_cells;
    int32_t bc_wall;
    uint64_t seed;
    int32_t lf_rhs_printed;
    double gl_gamma;
    int32_t gmres_mixed;
} gx_config;

typedef struct {
    int32_t iters;        /* matrix-vector products of the last solve */
    int32_t converged;    /* 1 if the relative residual reached gmres_tol */
    double relres;        /* true relative residual ||b - A E|| / ||b||, FP64 */
    double ms;            /* device time of the solve (CUDA events) */
} gx_solve_stats;

typedef struct {
    double energy_E;      /* dV sum_nodes |E|^2 / 8 pi */
    double energy_B;      /* dV sum_cells |B|^2 / 8 pi */
    double kinetic;       /* sum_p m_p |v_p|^2 / 2 */
    double momentum[3];   /* sum_p m_p v_p */
    double charge;        /* sum_g rho_g dV of the current deposit */
    double gauss_l2;      /* || div_C E - 4 pi rho_C ||_2 over cells (rho averaged to cells) */
    double divB_l2;       /* || div_N B ||_2 over nodes */
    int64_t n_particles;
} gx_diag;

/* ---------------------------------------------------------- life cycle */

/* Create a context on the current CUDA device.  Validates cfg (GX_EINVAL with
 * a message), allocates the field and solver state and sets E = B = 0. */
int gx_create(const gx_config *cfg, gx_ctx **out);

/* Free every device and host resource of ctx (NULL is ignored). */
void gx_destroy(gx_ctx *ctx);

const char *gx_status_string(int status);

/* Description of the last failure on ctx (empty string if none); the pointer
 * stays valid until the next call on ctx. */
const char *gx_last_error(gx_ctx *ctx);

/* ------------------------------------------------------------- set-up */

/* Add a species of n macro-particles with charge q and mass m per unit weight
 * (a particle of weight w carries q w and m w).  x, y, z are global positions
 * (FP64; z is ignored in 2D) wrapped into the periodic box; vx, vy, vz, w are
 * FP32.  Positions are x^{n+1/2} and velocities v^n of the ECSIM staggering.
 * The particles are copied into cell-sorted bins.  *species_id receives the
 * index of the new species (0, 1, ...; at most 4 species). */
int gx_species_add(gx_ctx *ctx, double q, double m, int64_t n,
                   const double *x, const double *y, const double *z,
                   const float *vx, const float *vy, const float *vz, const float *w,
                   int ptr_is_device, int *species_id);

/* Add a species generated on the device: ppc particles in every cell, drifting
 * Maxwellian with bulk velocity u[3] and per-component thermal speed vth,
 * density n0 (weights n0 dV / ppc), charge q and mass m per unit weight.
 * Particle k of cell (i, j) takes the four Philox4x64-10 words r of key
 * (cfg.seed, species index) and counter (0, j nx + i, k, 0): offsets in the
 * cell (r0 >> 40) 2^-24 and (r1 >> 40) 2^-24 (0 along y in 1D) and
 * v = u + vth (n0, n1, n2) from the Box-Muller transform of the 24-bit uniforms
 * ((r2 >> 40) + 1) 2^-24, ((r2 >> 16) & 0xffffff) 2^-24 (n0, n1) and the same
 * of r3 (n2) -- the draws of gx_boundary_source at step 0.  No host data is
 * involved.  1 <= ppc <= 4096; *species_id as for gx_species_add. */
int gx_species_maxwellian(gx_ctx *ctx, double q, double m, int ppc, double n0, const double *u, double vth,
                          int *species_id);

/* Set E (nodes) and B (cell centres), each FP64 [3][nz][ny][nx]. */
int gx_fields_set(gx_ctx *ctx, const double *E, const double *B, int ptr_is_device);

/* Plasma state of an open boundary (cfg.bc_cells > 0): side 0 is low x, side
 * 1 high x; for species `species` (already added): density n (particles of
 * weight n dV / ppc), bulk velocity u[3], per-component thermal speed vth, and
 * ppc particles per boundary cell (1 <= ppc <= 4096).  Every species needs a
 * source on both sides before the first push (GX_ESTATE otherwise).  The draw
 * of particle k of cell (i, j) after push number t (1, 2, ...) takes the four
 * Philox words r of counter (t, j nx + i, k, 0): cell offsets (r0 >> 40) 2^-24
 * and (r1 >> 40) 2^-24 (0 along y in 1D), and v = u + vth (n0, n1, n2) from the
 * Box-Muller transform of the 24-bit uniforms ((r2 >> 40) + 1) 2^-24,
 * ((r2 >> 16) & 0xffffff) 2^-24 (n0, n1) and the same of r3 (n2). */
int gx_boundary_source(gx_ctx *ctx, int side, int species, double n, const double *u, double vth, int ppc);

/* ------------------------------------------------------------- hot path */

/* Deposit the moments of the current particle state (positions x^{n+1/2},
 * velocities v^n, B^n): charge density, mass-weighted bulk velocity u
 * (Sec. 2.1), the current (comoving, Eq. 34, or standard) smoothed by ns_j
 * passes (Sec. 2.2), and the mass matrices M_gg' = sum_s beta_s sum_p q_p
 * alpha_p W_pg W_pg' (Eq. 33) with alpha from Eq. 30.  Called implicitly by
 * gx_field_solve when the moments are stale. */
int gx_deposit(gx_ctx *ctx, void *stream);

/* Solve the implicit field equation (Eq. 7 with the mass term and comoving
 * right-hand side of Eq. 35 and the implicit LF term of Eq. 19) for
 * E^{n+theta}, then form B^{n+1} = B^n - c dt curl E^{n+theta} (+ limited LF,
 * Eq. 17-18) and E^{n+1} = (E^{n+theta} - (1-theta) E^n) / theta (Eq. 10).
 * The new fields become current only at the next gx_push_and_deposit.
 * Returns GX_ENOCONV (best iterate kept) if gmres_maxit was reached.
 * stats may be NULL. */
int gx_field_solve(gx_ctx *ctx, void *stream, gx_solve_stats *stats);

/* Push every particle with the theta-implicit mover (Sec. 2.1, Eq. 29-30):
 * vbar = alpha (v^n + beta_s E^{n+theta}(x^{n+1/2})), v^{n+1} = 2 vbar - v^n,
 * x^{n+3/2} = x^{n+1/2} + dt v^{n+1} (periodic wrap), re-bin them by cell, and
 * in the same pass deposit the moments of step n+1 with alpha built from
 * B^{n+1}.  Requires a preceding gx_field_solve (GX_ESTATE otherwise); makes
 * E^{n+1}, B^{n+1} current.  GX_ECFL if a particle moved more than one cell. */
int gx_push_and_deposit(gx_ctx *ctx, void *stream);

/* nsteps x (gx_field_solve + gx_push_and_deposit).  last (may be NULL)
 * receives the statistics of the final solve. */
int gx_step(gx_ctx *ctx, int nsteps, void *stream, gx_solve_stats *last);

/* ------------------------------------------------------------- read-back */

/* Current E (nodes) and B (cells), FP64 [3][nz][ny][nx]; either may be NULL. */
int gx_get_fields(gx_ctx *ctx, double *E, double *B, int ptr_is_device);

/* E^{n+theta} of the last solve (FP64 [3][nz][ny][nx]). */
int gx_get_solution(gx_ctx *ctx, double *Etheta, int ptr_is_device);

/* Moments of the current deposit (FP64): rho [nz][ny][nx] (charge density),
 * J [3][nz][ny][nx] (comoving or standard current after ns_j smoothing passes),
 * M [nz][ny][nx][27][3][3] (mass matrix block coupling node g to its
 * neighbour at offset o = (ox+1) + 3 (oy+1) + 9 (oz+1); in 2D only oz = 0
 * blocks are non-zero), u [3][nz][ny][nx] (smoothed bulk velocity).  Any
 * pointer may be NULL. */
int gx_get_moments(gx_ctx *ctx, double *rho, double *J, double *M, double *u, int ptr_is_device);

/* Number of particles currently held by a species (-1 on a bad id). */
int64_t gx_species_count(gx_ctx *ctx, int species);

/* Copy a species' particles out in bin order: global positions (FP64),
 * velocities and weights (FP32), ids (int32, only with track_ids, else may be
 * NULL).  Each array holds gx_species_count() entries. */
int gx_get_particles(gx_ctx *ctx, int species, double *x, double *y, double *z,
                     float *vx, float *vy, float *vz, float *w, int32_t *id, int ptr_is_device);

/* FP64 diagnostics of the current state (synchronises the stream). */
int gx_diagnostics(gx_ctx *ctx, void *stream, gx_diag *out);

/* Accumulated device time (CUDA events on the launching stream) of the fused
 * push-and-deposit kernels, of the grid-side moment assembly, and of the
 * field solves since the last reset, in ms; plus the number of library kernel
 * launches.  reset != 0 clears the counters after reading. */
int gx_timers(gx_ctx *ctx, double *push_ms, double *moments_ms, double *solve_ms,
              int64_t *launches, int reset);

/* Accumulated device time (CUDA events on the launching stream, recorded
 * around each launch) of the fused mover + re-bin + deposit kernel alone, and
 * its number of launches (one per species and step); for roofline accounting.
 * reset != 0 clears both after reading. */
int gx_kernel_timer(gx_ctx *ctx, double *pd_ms, int64_t *pd_launches, int reset);

/* ------------------------------------------- learned GMRES preconditioner
 * An addition of this project (the paper has no learned preconditioner): a
 * 2D convolutional network N with four 3x3 layers (3 -> 32 -> 32 -> 32 -> 3
 * channels, ReLU between, periodic padding), BF16 weights and activations
 * with FP32 accumulation, used as the right preconditioner of FGMRES as a
 * learned correction of the 3x3 block-Jacobi preconditioner D^-1:
 * z = D^-1 r + s N(r / s), s = ||r||_2 / sqrt(3 N).  D^-1 carries what varies
 * from node to node (the local plasma response); the network learns the
 * translation-invariant remainder A^-1 r - D^-1 r.  2D only. */

/* Number of FP32 parameters of the network (weights [Cout][Cin][3][3] then
 * biases [Cout], per layer). */
int64_t gx_precond_param_count(void);

/* Load FP32 parameters (host or device); kept as an FP32 master copy and a
 * BF16 inference copy. */
int gx_precond_set_weights(gx_ctx *ctx, const float *params, int64_t n, int ptr_is_device);
int gx_precond_get_weights(gx_ctx *ctx, float *params, int64_t n, int ptr_is_device);

/* Keep up to `capacity` (residual, error) pairs (a ring: the newest replace
 * the oldest) from the converged solves that follow.  Each solve contributes
 * r0 = b - A E^n with e = E^{n+theta} - E^n (A e = r0 to the solver
 * tolerance), and (A V_j, V_j) for its first Krylov basis vectors V_j (up to
 * 6, one matrix-vector product each), which resemble what the preconditioner
 * is applied to.  capacity = 0 stops collecting. */
int gx_precond_collect(gx_ctx *ctx, int capacity);

/* Collect the same pairs as crops: every pair the following converged solves
 * produce is cut into `per_pair` windows of (crop + 8)^2 nodes (a crop x crop
 * training window with its 4-node halo, periodic wrap) at positions drawn by a
 * counter-based hash of `seed`, stored in FP32 already divided by the pair's
 * scale s = ||r||_2 / sqrt(3 N), as [2][3][crop+8][crop+8] (r / s, then
 * (e - D^-1 r) / s), with s; up to `capacity` crops (a ring).  About 6 (crop+8)^2
 * x 4 bytes a crop (38 KB at crop 32), so tens of thousands of training pairs fit
 * where whole fields would take 12.6 MB each at 1024 x 512.  With gmres_mixed
 * (FP32 Krylov basis) only (r0, e) is kept per solve.  gx_precond_train then
 * samples these crops (its `crop` must equal this one) and gx_precond_pairs
 * counts them.  capacity = 0 stops collecting; crop >= 8, crop + 8 <= nx, ny. */
int gx_precond_collect_crops(gx_ctx *ctx, int capacity, int crop, int per_pair, uint64_t seed);

/* Copy crop k (0 <= k < gx_precond_pairs) of the crop store to host memory:
 * out [2][3][crop+8][crop+8] FP32 as stored, *scale its s.  For tests. */
int gx_precond_crop(gx_ctx *ctx, int k, float *out, float *scale);

/* Number of training pairs kept: field pairs, or crops after gx_precond_collect_crops. */
int gx_precond_pairs(gx_ctx *ctx);

/* Train the network on the device with Adam (lr, beta1 0.9, beta2 0.999,
 * eps 1e-8, on an FP32 master copy) for `epochs` passes of `npairs` samples
 * each, in batches of `batch`.  A sample is a crop x crop window (crop >= 8) at
 * a random position (seeded by `seed`) of a random collected pair, cut from the
 * periodic grid with a 4-node halo so that the four 3x3 layers see exactly the
 * values they would see on the whole grid.  With s = ||r||_2 / sqrt(3 N) of the
 * pair (the scale the solver applies), the network learns the remainder over
 * block Jacobi: loss = sum over the crop of (N(r/s) - (e - D^-1 r)/s)^2 /
 * (2 * 3 crop^2 * batch), D^-1 that of the pair's own solve.
 * Forward, backward (data and weight gradients) and the update run in this
 * library's kernels.  loss_out (may be NULL) receives the mean batch loss of
 * each epoch.  GX_ESTATE if no pair has been collected. */
int gx_precond_train(gx_ctx *ctx, int npairs, int crop, int batch, int epochs, float lr,
                     uint64_t seed, float *loss_out, void *stream);

/* One forward pass of the network on a [3][H][W] FP32 input with periodic
 * padding: out = N(in), without the s-scaling.  H, W >= 1 are free (they need
 * not match the context's grid).  Device pointers; synchronises `stream`.
 * For tests. */
int gx_precond_forward(gx_ctx *ctx, int H, int W, const float *in, float *out, void *stream);

/* Apply the context's field-solve preconditioner to v ([3][N] FP64, device)
 * exactly as FGMRES applies it to a Krylov column: z = v (none), z = D^-1 v
 * (block Jacobi), z = D^-1 v + s N(v / s) with s = ||v||_2 / sqrt(3 N) (the
 * network on the tensor cores, its last layer adding its output to the block
 * Jacobi image).  D^-1 is rebuilt from the current operator (moments and LF
 * coefficients of the last solve).  z must not alias v.  Synchronises
 * `stream` (the norm is read back).  For tests. */
int gx_precond_apply(gx_ctx *ctx, const double *v, double *z, void *stream);

/* Loss and gradients of one [3][H][W] sample with zero padding:
 * *loss = sum (N(in) - target)^2 / (2 * 3 H W), grad (param_count FP32, the
 * layout of gx_precond_set_weights) = dloss/dparams.  Device pointers;
 * synchronises `stream`.  For tests. */
int gx_precond_loss_grad(gx_ctx *ctx, int H, int W, const float *in, const float *target,
                         float *loss, float *grad, void *stream);

/* ------------------------------------------- gather without allocation
 * The paper has no counterpart: this is a service of the library.  Same output
 * as gx_get_particles with ptr_is_device = 1 (bin order, the same values), for
 * callers that must not allocate device memory at that point (for instance a
 * diagnostics hook while the particle arrays fill the device, or a path that
 * must not synchronise).  It allocates nothing: its only scratch, the per-cell
 * output offsets, lives in a fixed device array of gx_noalloc_max_cells()
 * ints (262144, 1 MiB); larger grids get GX_EINVAL.  gx_create looks that
 * array up (once per device, with the context's device current) and loads the
 * code of this call then, so the call itself triggers no lazy module load
 * (which would allocate and could synchronise).  The array is shared by every context
 * on the device, so calls that overlap in time race.  Output pointers are
 * device arrays of gx_species_count() entries (NULL to skip a field; id only
 * with track_ids); the call enqueues two kernels on `stream` and does not
 * synchronise. */
int gx_noalloc_max_cells(void);
int gx_get_particles_noalloc(gx_ctx *ctx, int species, double *x, double *y, double *z,
                             float *vx, float *vy, float *vz, float *w, int32_t *id, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GX_H */
