/*
 * gx_oracle.c -- plain, slow, FP64 CPU oracle of the GL-ECSIM hot path.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm load this library.  The product path
 * (the CUDA library under paper_2506_11320_gb300/) never calls it, and the two
 * share no code, header, table or constant.
 *
 * It follows Chen, Zhou & Toth, "Suppressing spurious oscillations and particle
 * noise in particle-in-cell simulations" (arXiv 2506.11320), cited below by
 * section and equation.  Sections are numbered as in the paper's source:
 * Sec. 1.1 "Discretization of Maxwell's equations", Sec. 1.2 "Suppressing
 * spurious oscillations", Sec. 1.4 "From smoothing fields to the Lax-Friedrichs
 * diffusion", Sec. 2.1 "Calculating current in the comoving frame", Sec. 2.2
 * "Smoothing the current".
 *
 * Everything is written at the level of the definitions: direct loops over
 * particles and grid points, the mass matrix stored in full (every node keeps
 * all 27 neighbour blocks, no symmetry used), the comoving current done in two
 * passes (bulk velocity first, then the deposit of deviations from it), textbook
 * restarted GMRES with modified Gram-Schmidt, and dense Gaussian elimination as
 * a second solver for tiny grids.
 *
 * Mesh (Sec. 1.1): collocated staggered grid, E at nodes, B at cell centres.
 * Node (i,j,k) sits at (i dx, j dy, k dz); cell (i,j,k) spans
 * [i,i+1]x[j,j+1]x[k,k+1] cell widths.  All axes are periodic (with bc_cells,
 * x has open ends held at fixed plasma states: see bcell/bnode).  An axis with a
 * single cell is "collapsed": the periodic wrap makes node i+1 the same node as
 * node i, so derivatives along it vanish and averages along it are the identity,
 * and the same code covers 1D, 2D and 3D.  Positions along a collapsed axis are
 * not advanced and carry no weight.
 *
 * Units are Gaussian with an explicit speed of light c: Ampere's law
 * dE/dt = c curl B - 4 pi J (Eq. 1), Faraday's law dB/dt = -c curl E (Eq. 2) and
 * the Lorentz force q (E + v x B / c).
 *
 * Readings taken where the paper is silent or garbled (each is repeated at the
 * routine that uses it):
 *   - the shape function W is linear (cloud-in-cell) on the 2^d corner nodes;
 *   - B is averaged from cell centres to nodes (mean of the 2^d adjacent
 *     cells) before it is interpolated to particles with the same W as E;
 *   - the mover is the ECSIM one: positions live at half steps,
 *     v^{n+1} = 2 vbar - v^n, x^{n+3/2} = x^{n+1/2} + dt v^{n+1};
 *   - the mass-term prefactor printed as 4 pi/(c dV) in Eq. 35 is read as
 *     4 pi theta dt / dV (what substituting Jbar into Eq. 7 gives);
 *   - Eq. 8's "c theta dt" is read as "c dt" (Eq. 5 and Eq. 13 agree);
 *   - the implicit Lax-Friedrichs term on E (Eq. 19) enters with a minus sign
 *     (diffusive); with the printed plus sign it would be anti-diffusive;
 *   - the E limiter and diffusion speed are frozen at E^n, which keeps the
 *     field equation linear;
 *   - the 1D diffusion and filter are applied per axis and per component;
 *   - the diffusion speed a is |u| (the smoothed bulk velocity) averaged over
 *     the face / edge, or c for vacuum tests;
 *   - "plasma velocity" is mass weighted over all species, 0 where no mass;
 *   - a smoothness ratio with a zero denominator is taken as 0;
 *   - the E solve curls B^n + theta D, D the LF increment B^{n+1} receives
 *     (B^{n+theta} of Eq. 7 holds it);
 *   - div B cleaning (Sec. 1.3): phi at cell centres, central differences,
 *     B^{n+1} -= dt grad phi^n, then phi^{n+1} = exp(-0.1)(phi^n - dt c_h^2 div B^{n+1});
 *   - the E-field filter of the Sec. 3.1 comparison acts on E^{n+1} in place
 *     of the LF term on E;
 *   - open boundaries (the shock runs of Sec. 3.3-3.4): Dirichlet rows for E at
 *     boundary nodes, B held in boundary cells, boundary cells refilled after
 *     every push from Philox4x64-10 draws (or_bc_sample).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* Grid and method parameters.  Layout must match oracle/__init__.py. */
typedef struct {
    int32_t n[3];          /* cells per axis (1 = collapsed axis) */
    int32_t comoving;      /* 1: comoving-frame current (Sec. 2.1) */
    int32_t lf_on;         /* 1: limited Lax-Friedrichs diffusion on E and B (Sec. 1.2) */
    int32_t lf_speed_c;    /* 1: diffusion speed a = c; 0: a = |u| */
    int32_t ns_j;          /* passes of the digital filter on the current (Sec. 2.2) */
    int32_t nsmooth_u;     /* passes of the digital filter on the bulk velocity (Sec. 2.1) */
    int32_t gmres_restart;
    int32_t gmres_maxit;
    int32_t divb_clean;    /* 1: hyperbolic/parabolic divergence cleaning of B (Sec. 1.3) */
    int32_t nsmooth_e;     /* passes of the digital filter on E^{n+1} instead of LF on E (Sec. 3.1) */
    double dx[3];
    double c;              /* speed of light */
    double theta;          /* time centring of the theta scheme (Eq. 5-6) */
    double dt;
    double lf_beta;        /* MC limiter parameter beta (Eq. 21) */
    double gmres_tol;      /* relative residual target */
    int32_t bc_cells;      /* open x boundaries: cells per end held at a fixed plasma state (0: periodic) */
    int32_t bc_wall;       /* 1: the high-x boundary cells are a reflecting conducting wall instead */
    int32_t lf_rhs_printed; /* 1: the E solve curls B^n as Eq. 7 prints it, without theta D */
    double gl_gamma;       /* > 0: Gauss's-law position correction of GL-ECSIM, step fraction (see or_gl_displacement) */
} or_cfg;

/* ---------------------------------------------------------------- indexing */

static inline int64_t n_nodes(const or_cfg *g) { return (int64_t)g->n[0] * g->n[1] * g->n[2]; }

static inline int wrapi(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/* Linear index of node (or cell) (i,j,k) with periodic wrap. */
static inline int64_t ix(const or_cfg *g, int i, int j, int k) {
    return (int64_t)wrapi(i, g->n[0]) +
           (int64_t)g->n[0] * ((int64_t)wrapi(j, g->n[1]) + (int64_t)g->n[1] * wrapi(k, g->n[2]));
}

static inline void unix3(const or_cfg *g, int64_t idx, int *i, int *j, int *k) {
    *i = (int)(idx % g->n[0]);
    *j = (int)((idx / g->n[0]) % g->n[1]);
    *k = (int)(idx / ((int64_t)g->n[0] * g->n[1]));
}

static inline double cell_volume(const or_cfg *g) { return g->dx[0] * g->dx[1] * g->dx[2]; }

/* Open boundaries along x (the shock runs of Sec. 3.3; the paper does not print
 * the boundary treatment, this is the reading): bc_cells = G cells at each end
 * hold a fixed plasma state.  Boundary cells: i < G or i >= nx - G.  Boundary
 * nodes: i <= G - 1 or i >= nx - G + 1, the nodes whose two x-neighbouring
 * cells are both boundary cells.  E at boundary nodes and B in boundary cells
 * keep their values; the particles of boundary cells are replaced after every
 * push (or_bc_sample).  Everything else keeps the periodic indexing: with
 * G >= 8 no stencil or filter of an interior node reaches across the seam. */
static inline int bcell(const or_cfg *g, int i) {
    return g->bc_cells > 0 && (i < g->bc_cells || i >= g->n[0] - g->bc_cells);
}
static inline int bnode(const or_cfg *g, int i) {
    return g->bc_cells > 0 && (i <= g->bc_cells - 1 || i >= g->n[0] - g->bc_cells + (g->bc_wall ? 0 : 1));
}
/* With bc_wall the high-x boundary cells are a perfect conductor at rest (the
 * reflecting wall of the shock setups): no particles, E held (at 0 from the
 * initial fields) from the wall face x_w = (nx - G) dx on, B held, and a
 * particle that crosses x_w is reflected specularly: x -> 2 x_w - x, v_x -> -v_x. */

/* ----------------------------------------------------------- shape function */

/* Interpolation function W of Eq. 27, read as the linear (cloud-in-cell) shape:
 * the particle's cell (lowest corner node) and the weight of each of the 8
 * corners a = ax + 2 ay + 4 az.  Collapsed axes put all weight on corner 0. */
static void shape(const or_cfg *g, const double pos[3], int cell[3], double w[8]) {
    double f[3];
    for (int d = 0; d < 3; ++d) {
        double s = pos[d] / g->dx[d];
        double fl = floor(s);
        cell[d] = (int)fl;
        f[d] = (g->n[d] == 1) ? 0.0 : s - fl;
    }
    for (int a = 0; a < 8; ++a) {
        int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
        w[a] = (ax ? f[0] : 1.0 - f[0]) * (ay ? f[1] : 1.0 - f[1]) * (az ? f[2] : 1.0 - f[2]);
    }
}

static inline int64_t corner_node(const or_cfg *g, const int cell[3], int a) {
    return ix(g, cell[0] + (a & 1), cell[1] + ((a >> 1) & 1), cell[2] + ((a >> 2) & 1));
}

/* Interpolate a 3-component node field F[3][Nn] to a particle. */
static void gather3(const or_cfg *g, const double *F, const int cell[3], const double w[8], double out[3]) {
    int64_t N = n_nodes(g);
    out[0] = out[1] = out[2] = 0.0;
    for (int a = 0; a < 8; ++a) {
        int64_t nd = corner_node(g, cell, a);
        for (int c = 0; c < 3; ++c) out[c] += w[a] * F[c * N + nd];
    }
}

/* ------------------------------------------------------------ alpha tensor */

/* Rotation tensor of Sec. 2.1, Eq. 30, with b = beta_s B / c (Gaussian units put
 * the 1/c of the Lorentz force here).  Row-major 3x3 acting on a column vector:
 * alpha a = (a + a x b + (a.b) b) / (1 + b.b).
 * The dyadic form -beta I x B applied to a gives beta a x B, hence the + a x b. */
void or_alpha(const double b[3], double al[9]) {
    double D = 1.0 + b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    al[0] = 1.0 + b[0] * b[0]; al[1] = b[2] + b[0] * b[1];  al[2] = -b[1] + b[0] * b[2];
    al[3] = -b[2] + b[1] * b[0]; al[4] = 1.0 + b[1] * b[1]; al[5] = b[0] + b[1] * b[2];
    al[6] = b[1] + b[2] * b[0];  al[7] = -b[0] + b[2] * b[1]; al[8] = 1.0 + b[2] * b[2];
    for (int i = 0; i < 9; ++i) al[i] /= D;
}

static void matvec3(const double A[9], const double v[3], double out[3]) {
    for (int i = 0; i < 3; ++i) out[i] = A[3 * i] * v[0] + A[3 * i + 1] * v[1] + A[3 * i + 2] * v[2];
}

/* ---------------------------------------------------------- grid averaging */

/* B from cell centres to nodes: the mean of the 8 cells around each node
 * (reading: the paper keeps B at cell centres and does not say how it reaches
 * the particles; it is averaged to nodes and then interpolated with W). */
void or_node_avg(const or_cfg *g, const double *Bc, double *Bn) {
    int64_t N = n_nodes(g);
    for (int64_t nd = 0; nd < N; ++nd) {
        int i, j, k;
        unix3(g, nd, &i, &j, &k);
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int a = 0; a < 8; ++a)
                s += Bc[c * N + ix(g, i - 1 + (a & 1), j - 1 + ((a >> 1) & 1), k - 1 + ((a >> 2) & 1))];
            Bn[c * N + nd] = s / 8.0;
        }
    }
}

/* ------------------------------------------------------------ digital filter */

/* One pass of the digital filter of Sec. 1.4, Eq. 26,
 * v*_i = phi v_i + (1-phi)/2 (v_{i-d} + v_{i+d}), on a node field of ncomp
 * components.  Its multi-dimensional form is not stated; it is applied along
 * x, then y, then z, each sweep acting on the result of the previous one. */
void or_filter(const or_cfg *g, double *f, int ncomp, int d, double phi) {
    int64_t N = n_nodes(g);
    double *tmp = (double *)malloc(sizeof(double) * N);
    for (int c = 0; c < ncomp; ++c) {
        double *v = f + c * N;
        for (int ax = 0; ax < 3; ++ax) {
            if (g->n[ax] == 1) continue;
            for (int64_t nd = 0; nd < N; ++nd) {
                int i, j, k;
                unix3(g, nd, &i, &j, &k);
                int p[3] = {i, j, k}, m[3] = {i, j, k};
                p[ax] += d;
                m[ax] -= d;
                tmp[nd] = phi * v[nd] + 0.5 * (1.0 - phi) * (v[ix(g, m[0], m[1], m[2])] + v[ix(g, p[0], p[1], p[2])]);
            }
            memcpy(v, tmp, sizeof(double) * N);
        }
    }
    free(tmp);
}

/* ------------------------------------------------------- particle moments */

/* Mass density and momentum density at nodes (numerators of the plasma
 * velocity of Sec. 2.1): rho_m = sum m_p W_pg, P = sum m_p v_p W_pg over all
 * species.  Reading: the "plasma velocity" is mass weighted. */
void or_bulk_moments(const or_cfg *g, const double *qs, const double *ms, int64_t np,
                     const int32_t *sp, const double *x, const double *y, const double *z,
                     const double *vx, const double *vy, const double *vz, const double *w,
                     double *rho_m, double *P) {
    (void)qs;
    int64_t N = n_nodes(g);
    memset(rho_m, 0, sizeof(double) * N);
    memset(P, 0, sizeof(double) * 3 * N);
    for (int64_t p = 0; p < np; ++p) {
        double pos[3] = {x[p], y[p], z[p]}, W[8];
        int cell[3];
        shape(g, pos, cell, W);
        double mp = ms[sp[p]] * w[p];
        for (int a = 0; a < 8; ++a) {
            int64_t nd = corner_node(g, cell, a);
            rho_m[nd] += mp * W[a];
            P[nd] += mp * vx[p] * W[a];
            P[N + nd] += mp * vy[p] * W[a];
            P[2 * N + nd] += mp * vz[p] * W[a];
        }
    }
}

/* Comoving-frame velocity u(x) of Sec. 2.1: the plasma velocity P / rho_m
 * (0 at nodes without mass), smoothed by nsmooth_u passes of Eq. 26 with
 * phi = 0.5 and the stride alternating d = 1, 2, 1, 2, ... */
void or_bulk_velocity(const or_cfg *g, const double *rho_m, const double *P, double *u) {
    int64_t N = n_nodes(g);
    for (int64_t nd = 0; nd < N; ++nd)
        for (int c = 0; c < 3; ++c)
            u[c * N + nd] = rho_m[nd] != 0.0 ? P[c * N + nd] / rho_m[nd] : 0.0;
    for (int pass = 0; pass < g->nsmooth_u; ++pass) or_filter(g, u, 3, (pass % 2 == 0) ? 1 : 2, 0.5);
}

/* Moments the implicit field solve needs (Sec. 2.1):
 *   rho_g = (1/dV) sum_p q_p W_pg                                   (charge density)
 *   J_g   = (1/dV) sum_p q_p alpha_p (v_p - u(x_p)) W_pg            (Eq. 34, comoving)
 *         = (1/dV) sum_p q_p alpha_p v_p W_pg                       (u == NULL: standard)
 *   M_g,g' = sum_s beta_s sum_p q_p alpha_p W_pg W_pg'              (mass matrix, Eq. 33)
 * with u(x_p) = sum_g W_pg u_g and alpha_p built from B^n at the particle.
 * M is stored in full: M[((g * 27 + o) * 3 + i) * 3 + j], o = (ox+1) + 3 (oy+1) +
 * 9 (oz+1) the offset of g' from g in corner steps. */
void or_deposit(const or_cfg *g, const double *qs, const double *ms, int64_t np, const int32_t *sp,
                const double *x, const double *y, const double *z,
                const double *vx, const double *vy, const double *vz, const double *w,
                const double *Bn, const double *u, double *rho, double *J, double *M) {
    int64_t N = n_nodes(g);
    double dV = cell_volume(g);
    memset(rho, 0, sizeof(double) * N);
    memset(J, 0, sizeof(double) * 3 * N);
    memset(M, 0, sizeof(double) * N * 27 * 9);
    for (int64_t p = 0; p < np; ++p) {
        int s = sp[p];
        double beta = qs[s] * g->dt / (2.0 * ms[s]);
        double qp = qs[s] * w[p];
        double pos[3] = {x[p], y[p], z[p]}, W[8], Bp[3], b[3], al[9];
        int cell[3];
        shape(g, pos, cell, W);
        gather3(g, Bn, cell, W, Bp);
        for (int c = 0; c < 3; ++c) b[c] = beta * Bp[c] / g->c;
        or_alpha(b, al);
        double dv[3] = {vx[p], vy[p], vz[p]};
        if (u) {
            double up[3];
            gather3(g, u, cell, W, up);
            for (int c = 0; c < 3; ++c) dv[c] -= up[c];
        }
        double adv[3];
        matvec3(al, dv, adv);
        for (int a = 0; a < 8; ++a) {
            if (W[a] == 0.0) continue;
            int64_t na = corner_node(g, cell, a);
            rho[na] += qp * W[a] / dV;
            for (int c = 0; c < 3; ++c) J[c * N + na] += qp * adv[c] * W[a] / dV;
            for (int bb = 0; bb < 8; ++bb) {
                if (W[bb] == 0.0) continue;
                int o = ((bb & 1) - (a & 1) + 1) + 3 * (((bb >> 1) & 1) - ((a >> 1) & 1) + 1) +
                        9 * (((bb >> 2) & 1) - ((a >> 2) & 1) + 1);
                double f = beta * qp * W[a] * W[bb];
                double *blk = M + ((na * 27 + o) * 9);
                for (int e = 0; e < 9; ++e) blk[e] += f * al[e];
            }
        }
    }
}

/* ns_j passes of the digital filter (Eq. 26, phi = 0.5, d = 1) on the current,
 * Sec. 2.2. */
void or_smooth_current(const or_cfg *g, double *J, int ns_j) {
    for (int pass = 0; pass < ns_j; ++pass) or_filter(g, J, 3, 1, 0.5);
}

/* ------------------------------------------------------ discrete operators */

/* Derivative along axis d of a node field, evaluated at cell (i,j,k): the mean
 * of the 4 nodes on the cell's +d face minus the mean on its -d face, over dx_d.
 * (Collocated staggered mesh of Sec. 1.1.) */
static double dC(const or_cfg *g, const double *f, int i, int j, int k, int d) {
    double s = 0.0;
    for (int a = 0; a < 8; ++a) {
        int o[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
        double sgn = o[d] ? 1.0 : -1.0;
        s += sgn * f[ix(g, i + o[0], j + o[1], k + o[2])];
    }
    return s / (4.0 * g->dx[d]);
}

/* Derivative along axis d of a cell field, evaluated at node (i,j,k): the mean
 * of the 4 cells on the node's +d side minus the mean on its -d side, over dx_d. */
static double dN(const or_cfg *g, const double *f, int i, int j, int k, int d) {
    double s = 0.0;
    for (int a = 0; a < 8; ++a) {
        int o[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
        double sgn = o[d] ? 1.0 : -1.0;
        s += sgn * f[ix(g, i - 1 + o[0], j - 1 + o[1], k - 1 + o[2])];
    }
    return s / (4.0 * g->dx[d]);
}

/* curl of a node vector field, at cell centres. */
void or_curl_C(const or_cfg *g, const double *E, double *out) {
    int64_t N = n_nodes(g);
    const double *Ex = E, *Ey = E + N, *Ez = E + 2 * N;
    for (int64_t c = 0; c < N; ++c) {
        int i, j, k;
        unix3(g, c, &i, &j, &k);
        out[c] = dC(g, Ez, i, j, k, 1) - dC(g, Ey, i, j, k, 2);
        out[N + c] = dC(g, Ex, i, j, k, 2) - dC(g, Ez, i, j, k, 0);
        out[2 * N + c] = dC(g, Ey, i, j, k, 0) - dC(g, Ex, i, j, k, 1);
    }
}

/* curl of a cell vector field, at nodes. */
void or_curl_N(const or_cfg *g, const double *B, double *out) {
    int64_t N = n_nodes(g);
    const double *Bx = B, *By = B + N, *Bz = B + 2 * N;
    for (int64_t nd = 0; nd < N; ++nd) {
        int i, j, k;
        unix3(g, nd, &i, &j, &k);
        out[nd] = dN(g, Bz, i, j, k, 1) - dN(g, By, i, j, k, 2);
        out[N + nd] = dN(g, Bx, i, j, k, 2) - dN(g, Bz, i, j, k, 0);
        out[2 * N + nd] = dN(g, By, i, j, k, 0) - dN(g, Bx, i, j, k, 1);
    }
}

/* divergence of a node vector field, at cells. */
void or_div_C(const or_cfg *g, const double *E, double *out) {
    int64_t N = n_nodes(g);
    for (int64_t c = 0; c < N; ++c) {
        int i, j, k;
        unix3(g, c, &i, &j, &k);
        out[c] = dC(g, E, i, j, k, 0) + dC(g, E + N, i, j, k, 1) + dC(g, E + 2 * N, i, j, k, 2);
    }
}

/* divergence of a cell vector field, at nodes. */
void or_div_N(const or_cfg *g, const double *B, double *out) {
    int64_t N = n_nodes(g);
    for (int64_t nd = 0; nd < N; ++nd) {
        int i, j, k;
        unix3(g, nd, &i, &j, &k);
        out[nd] = dN(g, B, i, j, k, 0) + dN(g, B + N, i, j, k, 1) + dN(g, B + 2 * N, i, j, k, 2);
    }
}

/* gradient of a cell scalar, at nodes. */
void or_grad_N(const or_cfg *g, const double *f, double *out) {
    int64_t N = n_nodes(g);
    for (int64_t nd = 0; nd < N; ++nd) {
        int i, j, k;
        unix3(g, nd, &i, &j, &k);
        for (int d = 0; d < 3; ++d) out[d * N + nd] = dN(g, f, i, j, k, d);
    }
}

/* gradient of a node scalar, at cells. */
void or_grad_C(const or_cfg *g, const double *f, double *out) {
    int64_t N = n_nodes(g);
    for (int64_t c = 0; c < N; ++c) {
        int i, j, k;
        unix3(g, c, &i, &j, &k);
        for (int d = 0; d < 3; ++d) out[d * N + c] = dC(g, f, i, j, k, d);
    }
}

/* ------------------------------------------------------------ the limiter */

/* Generalised MC limiter of Sec. 1.2, Eq. 21: phi(r, beta) =
 * max(0, min(beta r, (1+r)/2, beta)). */
double or_mc_limiter(double r, double beta) {
    double v = fmin(fmin(beta * r, 0.5 * (1.0 + r)), beta);
    return v > 0.0 ? v : 0.0;
}

/* Smoothness ratio of Eq. 22 / Eq. 23; a zero denominator gives r = 0 (the flux
 * it scales multiplies that zero difference anyway). */
static double ratio(double prev, double cur) { return cur == 0.0 ? 0.0 : prev / cur; }

static double umag(const or_cfg *g, const double *u, int64_t nd) {
    int64_t N = n_nodes(g);
    return sqrt(u[nd] * u[nd] + u[N + nd] * u[N + nd] + u[2 * N + nd] * u[2 * N + nd]);
}

/* Diffusion coefficients kappa = (1 - phi_E) a / 2 of the implicit
 * Lax-Friedrichs term on E (Sec. 1.2, Eq. 19-20), on every edge from node g to
 * its +d neighbour, for each component: kappa[(d * 3 + comp) * Nn + g].
 * Readings: phi_E and a are frozen at E^n (keeps the solve linear); the 1D term
 * is applied per axis and component, with r taken along that axis (Eq. 23 with
 * the paper's left-biased stencil); a = |u| averaged over the edge's two nodes,
 * or c. */
void or_lf_kappa_E(const or_cfg *g, const double *En, const double *u, double *kappa) {
    int64_t N = n_nodes(g);
    memset(kappa, 0, sizeof(double) * 9 * N);
    for (int d = 0; d < 3; ++d) {
        if (g->n[d] == 1) continue;
        for (int comp = 0; comp < 3; ++comp) {
            const double *E = En + comp * N;
            for (int64_t nd = 0; nd < N; ++nd) {
                int i, j, k;
                unix3(g, nd, &i, &j, &k);
                int p[3] = {i, j, k}, m[3] = {i, j, k};
                p[d] += 1;
                m[d] -= 1;
                int64_t np_ = ix(g, p[0], p[1], p[2]), nm = ix(g, m[0], m[1], m[2]);
                double r = ratio(E[nd] - E[nm], E[np_] - E[nd]);
                double phi = or_mc_limiter(r, g->lf_beta);
                double a = g->lf_speed_c ? g->c : 0.5 * (umag(g, u, nd) + umag(g, u, np_));
                kappa[(d * 3 + comp) * N + nd] = (1.0 - phi) * a / 2.0;
            }
        }
    }
}

/* The implicit field operator of Sec. 1.2 and Sec. 2.1 (Eq. 7 with the mass
 * term of Eq. 35 and the diffusion of Eq. 19):
 *   A E = E + (c theta dt)^2 curl_N curl_C E + (4 pi theta dt / dV) M E
 *         - theta dt sum_d (1/dx_d) [kappa_+ (E_+ - E) - kappa_- (E - E_-)]
 * curl_N curl_C equals grad(div) - lap on this mesh.  kappa == NULL: no
 * diffusion term.  M == NULL: vacuum. */
void or_apply_A(const or_cfg *g, const double *M, const double *kappa, const double *E, double *out) {
    int64_t N = n_nodes(g);
    double *cC = (double *)malloc(sizeof(double) * 3 * N);
    double *cc = (double *)malloc(sizeof(double) * 3 * N);
    or_curl_C(g, E, cC);
    or_curl_N(g, cC, cc);
    double ct = g->c * g->theta * g->dt;
    double mfac = 4.0 * OR_PI * g->theta * g->dt / cell_volume(g);
    for (int64_t q = 0; q < 3 * N; ++q) out[q] = E[q] + ct * ct * cc[q];
    if (M) {
        for (int64_t nd = 0; nd < N; ++nd) {
            int i, j, k;
            unix3(g, nd, &i, &j, &k);
            for (int o = 0; o < 27; ++o) {
                int64_t nb = ix(g, i + (o % 3) - 1, j + (o / 3) % 3 - 1, k + o / 9 - 1);
                const double *blk = M + (nd * 27 + o) * 9;
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c) out[r * N + nd] += mfac * blk[3 * r + c] * E[c * N + nb];
            }
        }
    }
    if (kappa) {
        for (int d = 0; d < 3; ++d) {
            if (g->n[d] == 1) continue;
            double f = g->theta * g->dt / g->dx[d];
            for (int comp = 0; comp < 3; ++comp) {
                const double *Ec = E + comp * N;
                const double *kp = kappa + (d * 3 + comp) * N;
                for (int64_t nd = 0; nd < N; ++nd) {
                    int i, j, k;
                    unix3(g, nd, &i, &j, &k);
                    int p[3] = {i, j, k}, m[3] = {i, j, k};
                    p[d] += 1;
                    m[d] -= 1;
                    int64_t np_ = ix(g, p[0], p[1], p[2]), nm = ix(g, m[0], m[1], m[2]);
                    out[comp * N + nd] -= f * (kp[nd] * (Ec[np_] - Ec[nd]) - kp[nm] * (Ec[nd] - Ec[nm]));
                }
            }
        }
    }
    free(cC);
    free(cc);
    if (g->bc_cells) {           /* Dirichlet rows: E stays at its boundary value */
        for (int64_t nd = 0; nd < N; ++nd) {
            int i, j, k;
            unix3(g, nd, &i, &j, &k);
            if (bnode(g, i))
                for (int c = 0; c < 3; ++c) out[c * N + nd] = E[c * N + nd];
        }
    }
}

void or_lf_b_increment(const or_cfg *g, const double *Bc, const double *u, double *D);

/* Right-hand side of the E solve (Eq. 7; comoving form Eq. 35):
 *   b = E^n + c theta dt [curl_N B~ - (4 pi / c)(J - (1/dV) M E_M)]
 * with J the comoving current and E_M = -u x B^n / c the motional field at
 * nodes (B^n node averaged) when comoving != 0, and J the standard predicted-
 * current part without the E_M term otherwise.  B~ = B^n, or with lf_on
 * B^n + theta D, D the LF increment that B^{n+1} receives (Eq. 17-18):
 * Eq. 7 comes from substituting B^{n+theta} = (1-theta) B^n + theta B^{n+1}
 * into Eq. 6, and B^{n+1} carries D besides - c dt curl E^{n+theta}.
 * (Left out, the explicit D at level n amplifies the modes that the theta = 1/2
 * scheme flips in sign every step when c dt / dx >> 1.) */
void or_rhs(const or_cfg *g, const double *En, const double *Bc, const double *J, const double *M,
            const double *u, const double *Bn, double *b) {
    int64_t N = n_nodes(g);
    double *cn = (double *)malloc(sizeof(double) * 3 * N);
    if (g->lf_on && !g->lf_rhs_printed) {
        /* B^{n+theta} = (1 - theta) B^n + theta B^{n+1} holds the LF increment D
         * of B^{n+1} too, so the curl on the right acts on B^n + theta D */
        double *Bt = (double *)malloc(sizeof(double) * 3 * N);
        or_lf_b_increment(g, Bc, u, Bt);
        for (int64_t q = 0; q < 3 * N; ++q) Bt[q] = Bc[q] + g->theta * Bt[q];
        or_curl_N(g, Bt, cn);
        free(Bt);
    } else {
        or_curl_N(g, Bc, cn);
    }
    double ct = g->c * g->theta * g->dt;
    double jf = 4.0 * OR_PI * g->theta * g->dt;
    for (int64_t q = 0; q < 3 * N; ++q) b[q] = En[q] + ct * cn[q] - jf * J[q];
    if (g->comoving && M) {
        double *EM = (double *)malloc(sizeof(double) * 3 * N);
        for (int64_t nd = 0; nd < N; ++nd) {
            double ux = u[nd], uy = u[N + nd], uz = u[2 * N + nd];
            double bx = Bn[nd], by = Bn[N + nd], bz = Bn[2 * N + nd];
            EM[nd] = -(uy * bz - uz * by) / g->c;
            EM[N + nd] = -(uz * bx - ux * bz) / g->c;
            EM[2 * N + nd] = -(ux * by - uy * bx) / g->c;
        }
        double mf = jf / cell_volume(g);
        for (int64_t nd = 0; nd < N; ++nd) {
            int i, j, k;
            unix3(g, nd, &i, &j, &k);
            for (int o = 0; o < 27; ++o) {
                int64_t nb = ix(g, i + (o % 3) - 1, j + (o / 3) % 3 - 1, k + o / 9 - 1);
                const double *blk = M + (nd * 27 + o) * 9;
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c) b[r * N + nd] += mf * blk[3 * r + c] * EM[c * N + nb];
            }
        }
        free(EM);
    }
    free(cn);
    if (g->bc_cells) {           /* Dirichlet rows of the operator: b = E^n there */
        for (int64_t nd = 0; nd < N; ++nd) {
            int i, j, k;
            unix3(g, nd, &i, &j, &k);
            if (bnode(g, i))
                for (int c = 0; c < 3; ++c) b[c * N + nd] = En[c * N + nd];
        }
    }
}

/* ------------------------------------------------------------------ solvers */

static double dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Restarted GMRES(m) with modified Gram-Schmidt and Givens rotations (the
 * paper names no solver; the field equation is non-symmetric because alpha is).
 * x holds the initial guess on entry and the solution on exit.  Stops when the
 * relative residual ||b - A x|| / ||b|| reaches gmres_tol or after gmres_maxit
 * matrix-vector products.  Returns 0 if converged, 1 otherwise; writes the true
 * final relative residual and the number of products. */
int or_gmres(const or_cfg *g, const double *M, const double *kappa, const double *b, double *x,
             double *relres, int *iters) {
    int64_t n = 3 * n_nodes(g);
    int m = g->gmres_restart;
    double *V = (double *)malloc(sizeof(double) * n * (m + 1));
    double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
    double *cs = (double *)malloc(sizeof(double) * m), *sn = (double *)malloc(sizeof(double) * m);
    double *gg = (double *)malloc(sizeof(double) * (m + 1)), *y = (double *)malloc(sizeof(double) * m);
    double *r = (double *)malloc(sizeof(double) * n);
    double bnorm = sqrt(dot(n, b, b));
    int total = 0, conv = 0;
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        *relres = 0.0;
        *iters = 0;
        free(V); free(H); free(cs); free(sn); free(gg); free(y); free(r);
        return 0;
    }
    for (;;) {
        or_apply_A(g, M, kappa, x, r);
        for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
        double beta = sqrt(dot(n, r, r));
        if (beta / bnorm <= g->gmres_tol) { conv = 1; break; }
        if (total >= g->gmres_maxit) break;
        for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
        memset(gg, 0, sizeof(double) * (m + 1));
        gg[0] = beta;
        int jend = -1;
        for (int j = 0; j < m; ++j) {
            double *w = V + (int64_t)(j + 1) * n;
            or_apply_A(g, M, kappa, V + (int64_t)j * n, w);
            ++total;
            for (int i = 0; i <= j; ++i) {
                double h = dot(n, w, V + (int64_t)i * n);
                H[i * m + j] = h;
                for (int64_t q = 0; q < n; ++q) w[q] -= h * V[(int64_t)i * n + q];
            }
            double hn = sqrt(dot(n, w, w));
            H[(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (int64_t q = 0; q < n; ++q) w[q] /= hn;
            for (int i = 0; i < j; ++i) {
                double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
                H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
                H[i * m + j] = t;
            }
            double a = H[j * m + j], bb = H[(j + 1) * m + j];
            double den = sqrt(a * a + bb * bb);
            cs[j] = den == 0.0 ? 1.0 : a / den;
            sn[j] = den == 0.0 ? 0.0 : bb / den;
            H[j * m + j] = cs[j] * a + sn[j] * bb;
            H[(j + 1) * m + j] = 0.0;
            gg[j + 1] = -sn[j] * gg[j];
            gg[j] = cs[j] * gg[j];
            jend = j;
            if (fabs(gg[j + 1]) / bnorm <= g->gmres_tol || total >= g->gmres_maxit || hn == 0.0) break;
        }
        for (int i = jend; i >= 0; --i) {
            double s = gg[i];
            for (int k = i + 1; k <= jend; ++k) s -= H[i * m + k] * y[k];
            y[i] = s / H[i * m + i];
        }
        for (int i = 0; i <= jend; ++i)
            for (int64_t q = 0; q < n; ++q) x[q] += y[i] * V[(int64_t)i * n + q];
    }
    or_apply_A(g, M, kappa, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    *relres = sqrt(dot(n, r, r)) / bnorm;
    *iters = total;
    free(V); free(H); free(cs); free(sn); free(gg); free(y); free(r);
    return conv ? 0 : 1;
}

/* Second solver for tiny grids: assemble A column by column and solve by
 * Gaussian elimination with partial pivoting.  Returns 1 if singular. */
int or_dense_solve(const or_cfg *g, const double *M, const double *kappa, const double *b, double *x) {
    int64_t n = 3 * n_nodes(g);
    double *A = (double *)malloc(sizeof(double) * n * n);
    double *e = (double *)calloc((size_t)n, sizeof(double)), *col = (double *)malloc(sizeof(double) * n);
    for (int64_t j = 0; j < n; ++j) {
        e[j] = 1.0;
        or_apply_A(g, M, kappa, e, col);
        e[j] = 0.0;
        for (int64_t i = 0; i < n; ++i) A[i * n + j] = col[i];
    }
    memcpy(x, b, sizeof(double) * n);
    int sing = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t piv = k;
        for (int64_t i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > fabs(A[piv * n + k])) piv = i;
        if (A[piv * n + k] == 0.0) { sing = 1; break; }
        if (piv != k) {
            for (int64_t j = 0; j < n; ++j) { double t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
            double t = x[k]; x[k] = x[piv]; x[piv] = t;
        }
        for (int64_t i = k + 1; i < n; ++i) {
            double f = A[i * n + k] / A[k * n + k];
            if (f == 0.0) continue;
            for (int64_t j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
            x[i] -= f * x[k];
        }
    }
    if (!sing)
        for (int64_t i = n - 1; i >= 0; --i) {
            double s = x[i];
            for (int64_t j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
            x[i] = s / A[i * n + i];
        }
    free(A); free(e); free(col);
    return sing;
}

/* ---------------------------------------------------------- field advance */

/* Increment of the limited LF diffusion on B over one step (Eq. 17-18), per
 * component along every resolved axis:
 *   D_c = dt/dx_d (F_{c+1/2} - F_{c-1/2}),  F = (1 - phi_B) a / 2 (B_{c+1} - B_c),
 * phi_B = MC(r, beta) with r = (B_c - B_{c-1}) / (B_{c+1} - B_c) (Eq. 22),
 * a = |u| averaged over the face's 4 nodes (or c).  D = 0 without lf_on.  u may
 * be NULL when lf_speed_c != 0.  D [3][N]. */
void or_lf_b_increment(const or_cfg *g, const double *Bc, const double *u, double *D) {
    int64_t N = n_nodes(g);
    memset(D, 0, sizeof(double) * 3 * N);
    if (!g->lf_on) return;
    double *F = (double *)malloc(sizeof(double) * N);
    for (int d = 0; d < 3; ++d) {
        if (g->n[d] == 1) continue;
        double f = g->dt / g->dx[d];
        for (int comp = 0; comp < 3; ++comp) {
            const double *B = Bc + comp * N;
            for (int64_t c = 0; c < N; ++c) {
                int i, j, k;
                unix3(g, c, &i, &j, &k);
                int p[3] = {i, j, k}, m[3] = {i, j, k};
                p[d] += 1;
                m[d] -= 1;
                int64_t cp = ix(g, p[0], p[1], p[2]), cm = ix(g, m[0], m[1], m[2]);
                double r = ratio(B[c] - B[cm], B[cp] - B[c]);
                double phi = or_mc_limiter(r, g->lf_beta);
                double a;
                if (g->lf_speed_c) {
                    a = g->c;
                } else {
                    /* face between cell c and c+e_d: nodes with index_d = c_d + 1 */
                    double s = 0.0;
                    for (int t = 0; t < 4; ++t) {
                        int o[3] = {0, 0, 0};
                        int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
                        o[d] = 1;
                        o[e1] = t & 1;
                        o[e2] = (t >> 1) & 1;
                        s += umag(g, u, ix(g, i + o[0], j + o[1], k + o[2]));
                    }
                    a = s / 4.0;
                }
                F[c] = (1.0 - phi) * a / 2.0 * (B[cp] - B[c]);
            }
            for (int64_t c = 0; c < N; ++c) {
                int i, j, k;
                unix3(g, c, &i, &j, &k);
                int m[3] = {i, j, k};
                m[d] -= 1;
                D[comp * N + c] += f * (F[c] - F[ix(g, m[0], m[1], m[2])]);
            }
        }
    }
    free(F);
    if (g->bc_cells) {           /* boundary cells keep B: no increment there */
        for (int64_t c = 0; c < N; ++c) {
            int i, j, k;
            unix3(g, c, &i, &j, &k);
            if (bcell(g, i))
                for (int comp = 0; comp < 3; ++comp) D[comp * N + c] = 0.0;
        }
    }
}

/* B^{n+1} = B^n - c dt curl_C E^{n+theta} + D (Eq. 5 read with c dt, not
 * c theta dt, see Eq. 8; D the LF increment of or_lf_b_increment, Eq. 17-18),
 * and E^{n+1} = (E^{n+theta} - (1-theta) E^n) / theta (Eq. 10). */
void or_advance_fields(const or_cfg *g, const double *En, const double *Bc, const double *Eth,
                       const double *u, double *Enew, double *Bnew) {
    int64_t N = n_nodes(g);
    double *cc = (double *)malloc(sizeof(double) * 3 * N);
    double *D = (double *)malloc(sizeof(double) * 3 * N);
    or_curl_C(g, Eth, cc);
    or_lf_b_increment(g, Bc, u, D);
    for (int64_t q = 0; q < 3 * N; ++q) Bnew[q] = Bc[q] - g->c * g->dt * cc[q] + D[q];
    if (g->bc_cells) {           /* boundary cells keep their B */
        for (int64_t c = 0; c < N; ++c) {
            int i, j, k;
            unix3(g, c, &i, &j, &k);
            if (bcell(g, i))
                for (int comp = 0; comp < 3; ++comp) Bnew[comp * N + c] = Bc[comp * N + c];
        }
    }
    for (int64_t q = 0; q < 3 * N; ++q) Enew[q] = (Eth[q] - (1.0 - g->theta) * En[q]) / g->theta;
    free(cc);
    free(D);
}

/* ------------------------------------------------------ div B correction */

/* Hyperbolic/parabolic divergence cleaning (Sec. 1.3, "div B correction",
 * after Dedner et al.): a scalar phi at the cell centres with
 *   d phi / dt + c_h^2 div B = -(c_h^2 / c_p^2) phi,   dB/dt = -c curl E - grad phi,
 * c_h = 0.8 dx / dt and dt c_h^2 / c_p^2 = 0.1 (the paper's settings; dx is the
 * smallest cell width of the non-collapsed axes).  The paper takes its
 * discretisation from a reference that is not available here; reading: B and
 * phi at cell centres, divergence and gradient as central differences over the
 * neighbouring cells (so that grad = -div^T), and within a step
 *   B^{n+1} = (B^{n+1} of the field advance) - dt grad phi^n,
 *   phi^{n+1} = exp(-dt c_h^2 / c_p^2) (phi^n - dt c_h^2 div B^{n+1}),
 * the damping integrated exactly.  In place on Bnew [3][N] and phi [N]. */
void or_divb_clean(const or_cfg *g, double *Bnew, double *phi) {
    int64_t N = n_nodes(g);
    double dxmin = 0.0;
    for (int d = 0; d < 3; ++d)
        if (g->n[d] > 1 && (dxmin == 0.0 || g->dx[d] < dxmin)) dxmin = g->dx[d];
    if (dxmin == 0.0) return;                       /* no resolved axis: nothing to clean */
    const double ch = 0.8 * dxmin / g->dt;
    const double decay = exp(-0.1);
    for (int64_t c = 0; c < N; ++c) {
        int i, j, k;
        unix3(g, c, &i, &j, &k);
        for (int d = 0; d < 3; ++d) {
            if (g->n[d] == 1) continue;
            int p[3] = {i, j, k}, m[3] = {i, j, k};
            p[d] += 1;
            m[d] -= 1;
            Bnew[d * N + c] -= g->dt * (phi[ix(g, p[0], p[1], p[2])] - phi[ix(g, m[0], m[1], m[2])]) / (2.0 * g->dx[d]);
        }
    }
    double *div = (double *)malloc(sizeof(double) * N);
    for (int64_t c = 0; c < N; ++c) {
        int i, j, k;
        unix3(g, c, &i, &j, &k);
        double s = 0.0;
        for (int d = 0; d < 3; ++d) {
            if (g->n[d] == 1) continue;
            int p[3] = {i, j, k}, m[3] = {i, j, k};
            p[d] += 1;
            m[d] -= 1;
            s += (Bnew[d * N + ix(g, p[0], p[1], p[2])] - Bnew[d * N + ix(g, m[0], m[1], m[2])]) / (2.0 * g->dx[d]);
        }
        div[c] = s;
    }
    for (int64_t c = 0; c < N; ++c) phi[c] = decay * (phi[c] - g->dt * ch * ch * div[c]);
    free(div);
}

/* ------------------------------------------------------------------- mover */

/* theta-implicit mover (Sec. 2.1, Eq. 29-30 and the ECSIM update they cite):
 * vbar = alpha (v^n + beta_s E^{n+theta}(x^{n+1/2})), v^{n+1} = 2 vbar - v^n,
 * x^{n+3/2} = x^{n+1/2} + dt v^{n+1}, periodic wrap.  alpha uses the same
 * node-averaged B^n as the deposit.  vbar_out (3*np, may be NULL) receives vbar.
 * Returns the largest displacement in cell widths. */
double or_mover(const or_cfg *g, const double *qs, const double *ms, int64_t np, const int32_t *sp,
                double *x, double *y, double *z, double *vx, double *vy, double *vz,
                const double *Eth, const double *Bn, double *vbar_out) {
    double maxdisp = 0.0;
    for (int64_t p = 0; p < np; ++p) {
        int s = sp[p];
        double beta = qs[s] * g->dt / (2.0 * ms[s]);
        double pos[3] = {x[p], y[p], z[p]}, W[8], Ep[3], Bp[3], b[3], al[9];
        int cell[3];
        shape(g, pos, cell, W);
        gather3(g, Eth, cell, W, Ep);
        gather3(g, Bn, cell, W, Bp);
        for (int c = 0; c < 3; ++c) b[c] = beta * Bp[c] / g->c;
        or_alpha(b, al);
        double a[3] = {vx[p] + beta * Ep[0], vy[p] + beta * Ep[1], vz[p] + beta * Ep[2]}, vb[3];
        matvec3(al, a, vb);
        double vn[3] = {2.0 * vb[0] - vx[p], 2.0 * vb[1] - vy[p], 2.0 * vb[2] - vz[p]};
        if (vbar_out) { vbar_out[3 * p] = vb[0]; vbar_out[3 * p + 1] = vb[1]; vbar_out[3 * p + 2] = vb[2]; }
        vx[p] = vn[0]; vy[p] = vn[1]; vz[p] = vn[2];
        double *xs[3] = {x + p, y + p, z + p};
        for (int d = 0; d < 3; ++d) {
            if (g->n[d] == 1) continue;
            double disp = g->dt * vn[d];
            double L = g->n[d] * g->dx[d];
            double xn = *xs[d] + disp;
            if (d == 0 && g->bc_cells > 0 && g->bc_wall) {
                const double xw = (g->n[0] - g->bc_cells) * g->dx[0];
                if (xn >= xw) { xn = 2.0 * xw - xn; vx[p] = -vx[p]; }
            }
            xn = fmod(xn, L);
            if (xn < 0.0) xn += L;
            if (xn >= L) xn -= L;
            *xs[d] = xn;
            double dc = fabs(disp) / g->dx[d];
            if (dc > maxdisp) maxdisp = dc;
        }
    }
    return maxdisp;
}

/* ------------------------------------------------ Gauss's-law correction */

/* Particle-position correction for Gauss's law, the "GL" of GL-ECSIM (the
 * paper names the method by citation only; this is the reading used here).
 * With R_c = (div_C E)_c / (4 pi) - rhobar_c the Gauss residual of cell c,
 * rhobar_c the mean over the cell's 8 corner nodes of the particles' CIC
 * charge density rho, and
 *   F(x_1, ..., x_np) = (dV / 2) sum_c R_c^2,
 * the derivative of F with respect to a particle position is
 *   dF/dx_p = -q_p grad phi(x_p),  phi_g = mean of R over the 8 cells around node g,
 * phi interpolated with the particles' own linear weights (q_p = q_s w_p).  The
 * correction is one steepest-descent step,
 *   dx_p = gamma eps q_p grad phi(x_p),  eps = 1 / (Q2 sum_d 4 / dx_d^2),  Q2 = sum_p q_p^2 / V,
 * V the domain volume and the sum over resolved axes: for a uniform plasma the
 * linearised step multiplies a residual mode by about 1 - gamma eps Q2 k^2,
 * with k^2 <= sum_d 4 / dx_d^2 on the grid, so 0 < gamma <= 1 damps every mode.
 * Writes the displacements and, in F_out (may be NULL), F at the given positions.
 * Collapsed axes get no displacement. */
void or_gl_displacement(const or_cfg *g, const double *qs, int64_t np, const int32_t *sp,
                        const double *x, const double *y, const double *z, const double *w,
                        const double *E, double gamma, double *dx, double *dy, double *dz, double *F_out) {
    int64_t N = n_nodes(g);
    double dV = cell_volume(g);
    double *rho = (double *)calloc((size_t)N, sizeof(double));
    double *div = (double *)malloc(sizeof(double) * N);
    double *R = (double *)malloc(sizeof(double) * N);
    double *phi = (double *)malloc(sizeof(double) * N);
    double Q2 = 0.0;
    for (int64_t p = 0; p < np; ++p) {
        double qp = qs[sp[p]] * w[p];
        double pos[3] = {x[p], y[p], z[p]}, W[8];
        int cell[3];
        shape(g, pos, cell, W);
        for (int a = 0; a < 8; ++a) rho[corner_node(g, cell, a)] += qp * W[a] / dV;
        Q2 += qp * qp;
    }
    Q2 /= (double)N * dV;
    or_div_C(g, E, div);
    for (int64_t c = 0; c < N; ++c) {
        int i, j, k;
        unix3(g, c, &i, &j, &k);
        double rb = 0.0;
        for (int a = 0; a < 8; ++a) rb += rho[ix(g, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1))];
        R[c] = div[c] / (4.0 * OR_PI) - rb / 8.0;
    }
    double F = 0.0;
    for (int64_t c = 0; c < N; ++c) F += 0.5 * dV * R[c] * R[c];
    for (int64_t nd = 0; nd < N; ++nd) {
        int i, j, k;
        unix3(g, nd, &i, &j, &k);
        double s = 0.0;
        for (int a = 0; a < 8; ++a) s += R[ix(g, i - 1 + (a & 1), j - 1 + ((a >> 1) & 1), k - 1 + ((a >> 2) & 1))];
        phi[nd] = s / 8.0;
    }
    double lap = 0.0;
    for (int d = 0; d < 3; ++d)
        if (g->n[d] > 1) lap += 4.0 / (g->dx[d] * g->dx[d]);
    const double eps = (Q2 > 0.0 && lap > 0.0) ? 1.0 / (Q2 * lap) : 0.0;
    for (int64_t p = 0; p < np; ++p) {
        double qp = qs[sp[p]] * w[p];
        double pos[3] = {x[p], y[p], z[p]}, f[3];
        int cell[3];
        for (int d = 0; d < 3; ++d) {
            double sd = pos[d] / g->dx[d], fl = floor(sd);
            cell[d] = (int)fl;
            f[d] = (g->n[d] == 1) ? 0.0 : sd - fl;
        }
        double grad[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 8; ++a) {
            int ab[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
            double ph = phi[corner_node(g, cell, a)];
            for (int d = 0; d < 3; ++d) {
                if (g->n[d] == 1) continue;
                /* d W_a / d x_d: the derivative of the linear factor along d times the other two factors */
                double t = (ab[d] ? 1.0 : -1.0) / g->dx[d];
                for (int e = 0; e < 3; ++e)
                    if (e != d) t *= ab[e] ? f[e] : 1.0 - f[e];
                grad[d] += t * ph;
            }
        }
        dx[p] = gamma * eps * qp * grad[0];
        dy[p] = gamma * eps * qp * grad[1];
        dz[p] = gamma * eps * qp * grad[2];
    }
    if (F_out) *F_out = F;
    free(rho); free(div); free(R); free(phi);
}

/* -------------------------------------------------------------- diagnostics */

/* out[0] = electric energy dV sum |E|^2 / 8 pi, out[1] = magnetic energy,
 * out[2] = kinetic energy sum m_p |v|^2 / 2, out[3..5] = particle momentum. */
void or_energy(const or_cfg *g, const double *ms, int64_t np, const int32_t *sp,
               const double *vx, const double *vy, const double *vz, const double *w,
               const double *E, const double *Bc, double *out) {
    int64_t N = n_nodes(g);
    double dV = cell_volume(g);
    double we = 0.0, wb = 0.0, ke = 0.0, px = 0.0, py = 0.0, pz = 0.0;
    for (int64_t q = 0; q < 3 * N; ++q) { we += E[q] * E[q]; wb += Bc[q] * Bc[q]; }
    for (int64_t p = 0; p < np; ++p) {
        double mp = ms[sp[p]] * w[p];
        ke += 0.5 * mp * (vx[p] * vx[p] + vy[p] * vy[p] + vz[p] * vz[p]);
        px += mp * vx[p]; py += mp * vy[p]; pz += mp * vz[p];
    }
    out[0] = we * dV / (8.0 * OR_PI);
    out[1] = wb * dV / (8.0 * OR_PI);
    out[2] = ke;
    out[3] = px; out[4] = py; out[5] = pz;
}

/* ------------------------------------------------------------ one time step */

/* One full step (Sec. 1.1, 1.2, 2.1, 2.2) from (x^{n+1/2}, v^n, E^n, B^n):
 *  1. B^n averaged to nodes;
 *  2. bulk velocity u (needed for the comoving current and for a = |u|);
 *  3. deposit rho, J (comoving or standard), M with alpha from B^n;
 *  4. ns_j filter passes on J;
 *  5. LF coefficients from E^n (skipped with nsmooth_e > 0);
 *  6. right-hand side, GMRES from x0 = E^n -> E^{n+theta};
 *  7. B^{n+1}, E^{n+1}; with divb_clean, the divergence cleaning of B^{n+1}
 *     and of the cell-centred phi (in/out, may be NULL without it);
 *     with nsmooth_e, nsmooth_e filter passes on E^{n+1} (strides 1, 2, 1, ...);
 *  8. mover with E^{n+theta} and B^n.
 * E and B are updated in place; particles too.  Optional outputs (may be NULL):
 * Eth_out (3 Nn), J_out (3 Nn), M_out (Nn 27 9), u_out (3 Nn), vbar_out (3 np).
 * stats[0] = GMRES products, stats[1] = final relative residual,
 * stats[2] = max displacement in cells.  Returns 0 or 1 (GMRES not converged). */
int or_step(const or_cfg *g, const double *qs, const double *ms, int64_t np, const int32_t *sp,
            double *x, double *y, double *z, double *vx, double *vy, double *vz, const double *w,
            double *E, double *Bc, double *phi, double *Eth_out, double *J_out, double *M_out, double *u_out,
            double *vbar_out, double *stats) {
    int64_t N = n_nodes(g);
    double *Bn = (double *)malloc(sizeof(double) * 3 * N);
    double *u = (double *)calloc((size_t)(3 * N), sizeof(double));
    double *rho = (double *)malloc(sizeof(double) * N), *J = (double *)malloc(sizeof(double) * 3 * N);
    double *M = (double *)malloc(sizeof(double) * N * 27 * 9);
    double *kappa = (double *)malloc(sizeof(double) * 9 * N);
    double *b = (double *)malloc(sizeof(double) * 3 * N), *Eth = (double *)malloc(sizeof(double) * 3 * N);
    double *En1 = (double *)malloc(sizeof(double) * 3 * N), *Bn1 = (double *)malloc(sizeof(double) * 3 * N);
    or_node_avg(g, Bc, Bn);
    int need_u = g->comoving || (g->lf_on && !g->lf_speed_c);
    if (need_u) {
        double *rm = (double *)malloc(sizeof(double) * N), *P = (double *)malloc(sizeof(double) * 3 * N);
        or_bulk_moments(g, qs, ms, np, sp, x, y, z, vx, vy, vz, w, rm, P);
        or_bulk_velocity(g, rm, P, u);
        free(rm); free(P);
    }
    or_deposit(g, qs, ms, np, sp, x, y, z, vx, vy, vz, w, Bn, g->comoving ? u : NULL, rho, J, M);
    or_smooth_current(g, J, g->ns_j);
    /* with nsmooth_e > 0 the digital filter on E replaces the implicit LF term
     * on E; the LF term on B stays as lf_on says (the comparison of Sec. 3.1) */
    const int lf_e = g->lf_on && g->nsmooth_e == 0;
    if (lf_e) or_lf_kappa_E(g, E, u, kappa);
    or_rhs(g, E, Bc, J, M, u, Bn, b);
    memcpy(Eth, E, sizeof(double) * 3 * N);
    double relres = 0.0;
    int iters = 0;
    int rc = or_gmres(g, M, lf_e ? kappa : NULL, b, Eth, &relres, &iters);
    or_advance_fields(g, E, Bc, Eth, u, En1, Bn1);
    if (g->divb_clean && phi) or_divb_clean(g, Bn1, phi);
    /* E^{n+1} smoothed by nsmooth_e passes of Eq. 26, phi = 0.5, strides 1, 2, 1, ... */
    for (int pass = 0; pass < g->nsmooth_e; ++pass) or_filter(g, En1, 3, (pass % 2 == 0) ? 1 : 2, 0.5);
    /* GL correction (or_gl_displacement): the displacement of x^{n+1/2} from E^n and
     * the particles' own charge, added to the mover's update of the positions */
    double *gdx = NULL, *gdy = NULL, *gdz = NULL;
    if (g->gl_gamma > 0.0) {
        gdx = (double *)malloc(sizeof(double) * (np > 0 ? np : 1));
        gdy = (double *)malloc(sizeof(double) * (np > 0 ? np : 1));
        gdz = (double *)malloc(sizeof(double) * (np > 0 ? np : 1));
        or_gl_displacement(g, qs, np, sp, x, y, z, w, E, g->gl_gamma, gdx, gdy, gdz, NULL);
    }
    double md = or_mover(g, qs, ms, np, sp, x, y, z, vx, vy, vz, Eth, Bn, vbar_out);
    if (gdx) {
        double *xs[3] = {x, y, z}, *ds[3] = {gdx, gdy, gdz};
        for (int d = 0; d < 3; ++d) {
            if (g->n[d] == 1) continue;
            double L = g->n[d] * g->dx[d];
            for (int64_t p = 0; p < np; ++p) {
                double xn = fmod(xs[d][p] + ds[d][p], L);
                if (xn < 0.0) xn += L;
                if (xn >= L) xn -= L;
                xs[d][p] = xn;
            }
        }
        free(gdx); free(gdy); free(gdz);
    }
    memcpy(E, En1, sizeof(double) * 3 * N);
    memcpy(Bc, Bn1, sizeof(double) * 3 * N);
    if (Eth_out) memcpy(Eth_out, Eth, sizeof(double) * 3 * N);
    if (J_out) memcpy(J_out, J, sizeof(double) * 3 * N);
    if (M_out) memcpy(M_out, M, sizeof(double) * N * 27 * 9);
    if (u_out) memcpy(u_out, u, sizeof(double) * 3 * N);
    if (stats) { stats[0] = iters; stats[1] = relres; stats[2] = md; }
    free(Bn); free(u); free(rho); free(J); free(M); free(kappa); free(b); free(Eth); free(En1); free(Bn1);
    return rc;
}

/* ------------------------------------------------ boundary particle source */

/* Philox4x64-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC 2011): a counter-based generator, the same on the host
 * and the device, so that both inject identical particles.  Ten rounds of
 *   (x0, x1, x2, x3) <- (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0))
 * with the key bumped by the Weyl constants between rounds. */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    const uint64_t a0 = a & 0xffffffffu, a1 = a >> 32, b0 = b & 0xffffffffu, b1 = b >> 32;
    const uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
    const uint64_t mid = (p00 >> 32) + (p01 & 0xffffffffu) + (p10 & 0xffffffffu);
    *lo = a * b;
    *hi = p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
}

void or_philox4x64(const uint64_t key[2], const uint64_t ctr[4], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x0, &hi0, &lo0);
        mulhilo64(M1, x2, &hi1, &lo1);
        const uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The ppc particles that refill boundary cell (i, j) after the push of step
 * `step` (reading of the open boundaries): key (seed, species), counter
 * (step, cell index j nx + i, particle k, 0).  From the four 64-bit words:
 * offsets in the cell ox = (r0 >> 40) 2^-24, oy = (r1 >> 40) 2^-24 (exact in
 * FP32), and three normals by the Box-Muller transform of the 24-bit uniforms
 * u1 = ((r2 >> 40) + 1) 2^-24, u2 = ((r2 >> 16) & 0xffffff) 2^-24,
 * u3 = ((r3 >> 40) + 1) 2^-24, u4 = ((r3 >> 16) & 0xffffff) 2^-24:
 *   n0 = sqrt(-2 ln u1) cos(2 pi u2), n1 = sqrt(-2 ln u1) sin(2 pi u2),
 *   n2 = sqrt(-2 ln u3) cos(2 pi u4);
 * v = u + vth (n0, n1, n2).  Positions are global: x = (i + ox) dx, y = (j + oy) dy. */
void or_bc_sample(const or_cfg *g, uint64_t seed, int species, int64_t step, int i, int j, int ppc,
                  const double u[3], double vth, double *x, double *y, double *vx, double *vy, double *vz) {
    const uint64_t key[2] = {seed, (uint64_t)species};
    const double s24 = 1.0 / 16777216.0, twopi = 2.0 * OR_PI;
    for (int k = 0; k < ppc; ++k) {
        const uint64_t ctr[4] = {(uint64_t)step, (uint64_t)j * (uint64_t)g->n[0] + (uint64_t)i, (uint64_t)k, 0};
        uint64_t r[4];
        or_philox4x64(key, ctr, r);
        const double ox = (double)(r[0] >> 40) * s24, oy = (double)(r[1] >> 40) * s24;
        const double u1 = (double)((r[2] >> 40) + 1) * s24, u2 = (double)((r[2] >> 16) & 0xffffffu) * s24;
        const double u3 = (double)((r[3] >> 40) + 1) * s24, u4 = (double)((r[3] >> 16) & 0xffffffu) * s24;
        const double ra = sqrt(-2.0 * log(u1)), rb = sqrt(-2.0 * log(u3));
        x[k] = (i + ox) * g->dx[0];
        y[k] = g->n[1] > 1 ? (j + oy) * g->dx[1] : 0.0;
        vx[k] = u[0] + vth * ra * cos(twopi * u2);
        vy[k] = u[1] + vth * ra * sin(twopi * u2);
        vz[k] = u[2] + vth * rb * cos(twopi * u4);
    }
}

/* The ppc draws of cell (i, j, k) in the draw of `step` on a grid with a
 * resolved z axis: as or_bc_sample, with the counter's cell word the flat cell
 * index i + nx (j + ny k) and the z offset from bits 16..39 of word 0 (the
 * device-side Maxwellian species of a 3D grid draws its particles so). */
void or_cell_sample3(const or_cfg *g, uint64_t seed, int species, int64_t step, int i, int j, int k, int ppc,
                     const double u[3], double vth, double *x, double *y, double *z, double *vx, double *vy,
                     double *vz) {
    const uint64_t key[2] = {seed, (uint64_t)species};
    const double s24 = 1.0 / 16777216.0, twopi = 2.0 * OR_PI;
    const uint64_t cell = (uint64_t)i + (uint64_t)g->n[0] * ((uint64_t)j + (uint64_t)g->n[1] * (uint64_t)k);
    for (int p = 0; p < ppc; ++p) {
        const uint64_t ctr[4] = {(uint64_t)step, cell, (uint64_t)p, 0};
        uint64_t r[4];
        or_philox4x64(key, ctr, r);
        const double ox = (double)(r[0] >> 40) * s24, oy = (double)(r[1] >> 40) * s24;
        const double oz = (double)((r[0] >> 16) & 0xffffffu) * s24;
        const double u1 = (double)((r[2] >> 40) + 1) * s24, u2 = (double)((r[2] >> 16) & 0xffffffu) * s24;
        const double u3 = (double)((r[3] >> 40) + 1) * s24, u4 = (double)((r[3] >> 16) & 0xffffffu) * s24;
        const double ra = sqrt(-2.0 * log(u1)), rb = sqrt(-2.0 * log(u3));
        x[p] = (i + ox) * g->dx[0];
        y[p] = g->n[1] > 1 ? (j + oy) * g->dx[1] : 0.0;
        z[p] = g->n[2] > 1 ? (k + oz) * g->dx[2] : 0.0;
        vx[p] = u[0] + vth * ra * cos(twopi * u2);
        vy[p] = u[1] + vth * ra * sin(twopi * u2);
        vz[p] = u[2] + vth * rb * cos(twopi * u4);
    }
}

/* ------------------------------------------------- learned preconditioner net */

/* The convolutional correction network of the learned GMRES preconditioner (an
 * addition of this project; the paper has no such network).  Four 3x3
 * convolutions with channel counts 3 -> 32 -> 32 -> 32 -> 3 and ReLU between
 * them, on a 2D grid of H rows and W columns, channel-major tensors
 * x[C][H][W].  params: for each layer l, the weights Wl[Cout][Cin][3][3] then
 * the bias bl[Cout].  Padding is a periodic wrap (periodic != 0) or zeros. */
static const int NET_C[5] = {3, 32, 32, 32, 3};

int64_t or_net_param_count(void) {
    int64_t n = 0;
    for (int l = 0; l < 4; ++l) n += (int64_t)NET_C[l + 1] * NET_C[l] * 9 + NET_C[l + 1];
    return n;
}

/* Size of the activation buffer or_net_forward needs: for layers 1-3 the
 * pre-activation values, 3 * 32 * H * W doubles. */
int64_t or_net_act_count(int H, int W) { return (int64_t)3 * 32 * H * W; }

static double pad_at(const double *x, int H, int W, int periodic, int i, int j) {
    if (periodic) return x[wrapi(i, H) * W + wrapi(j, W)];
    if (i < 0 || i >= H || j < 0 || j >= W) return 0.0;
    return x[i * W + j];
}

static void conv3x3(int H, int W, int periodic, int cin, int cout, const double *Wt, const double *bias,
                    const double *x, double *y) {
    for (int co = 0; co < cout; ++co)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                double s = bias[co];
                for (int ci = 0; ci < cin; ++ci)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx)
                            s += Wt[((co * cin + ci) * 3 + ky) * 3 + kx] *
                                 pad_at(x + (int64_t)ci * H * W, H, W, periodic, i + ky - 1, j + kx - 1);
                y[((int64_t)co * H + i) * W + j] = s;
            }
}

/* Forward pass: y = N(x).  acts (or_net_act_count doubles, may be NULL)
 * receives the pre-activation outputs of layers 1-3. */
void or_net_forward(int H, int W, int periodic, const double *params, const double *x, double *y, double *acts) {
    int64_t HW = (int64_t)H * W;
    double *a = (double *)malloc(sizeof(double) * 32 * HW), *h = (double *)malloc(sizeof(double) * 32 * HW);
    const double *in = x;
    const double *p = params;
    for (int l = 0; l < 4; ++l) {
        int cin = NET_C[l], cout = NET_C[l + 1];
        const double *Wt = p, *bias = p + (int64_t)cout * cin * 9;
        p = bias + cout;
        if (l < 3) {
            conv3x3(H, W, periodic, cin, cout, Wt, bias, in, a);   /* reads in (x or h), writes a */
            if (acts) memcpy(acts + (int64_t)l * 32 * HW, a, sizeof(double) * 32 * HW);
            for (int64_t q = 0; q < (int64_t)cout * HW; ++q) h[q] = a[q] > 0.0 ? a[q] : 0.0;
            in = h;
        } else {
            conv3x3(H, W, periodic, cin, cout, Wt, bias, in, y);
        }
    }
    free(a); free(h);
}

/* Loss L = (1/(2 Nout)) sum (N(x) - t)^2 with Nout = 3 H W, and its gradient
 * with respect to every parameter (grad_params, same layout as params) and to
 * the input (grad_x, may be NULL).  Returns L. */
double or_net_loss_backward(int H, int W, int periodic, const double *params, const double *x,
                            const double *target, double *grad_params, double *grad_x) {
    int64_t HW = (int64_t)H * W;
    double *acts = (double *)malloc(sizeof(double) * or_net_act_count(H, W));
    double *y = (double *)malloc(sizeof(double) * 3 * HW);
    or_net_forward(H, W, periodic, params, x, y, acts);
    double nout = 3.0 * (double)HW, L = 0.0;
    double *gy = (double *)malloc(sizeof(double) * 32 * HW);
    for (int64_t q = 0; q < 3 * HW; ++q) {
        double d = y[q] - target[q];
        L += d * d;
        gy[q] = d / nout;
    }
    L /= 2.0 * nout;
    const double *Wl[4], *bl[4];
    double *gW[4], *gb[4];
    {
        const double *p = params;
        double *gp = grad_params;
        for (int l = 0; l < 4; ++l) {
            int cin = NET_C[l], cout = NET_C[l + 1];
            Wl[l] = p; bl[l] = p + (int64_t)cout * cin * 9; p = bl[l] + cout;
            gW[l] = gp; gb[l] = gp + (int64_t)cout * cin * 9; gp = gb[l] + cout;
        }
        memset(grad_params, 0, sizeof(double) * or_net_param_count());
    }
    double *gin = (double *)malloc(sizeof(double) * 32 * HW);
    double *hin = (double *)malloc(sizeof(double) * 32 * HW);
    for (int l = 3; l >= 0; --l) {
        int cin = NET_C[l], cout = NET_C[l + 1];
        /* the layer's input: x for l == 0, relu(pre-activation of layer l-1) otherwise */
        if (l == 0) memcpy(hin, x, sizeof(double) * 3 * HW);
        else
            for (int64_t q = 0; q < (int64_t)cin * HW; ++q) {
                double a = acts[(int64_t)(l - 1) * 32 * HW + q];
                hin[q] = a > 0.0 ? a : 0.0;
            }
        memset(gin, 0, sizeof(double) * (int64_t)cin * HW);
        for (int co = 0; co < cout; ++co)
            for (int i = 0; i < H; ++i)
                for (int j = 0; j < W; ++j) {
                    double d = gy[((int64_t)co * H + i) * W + j];
                    if (d == 0.0) continue;
                    gb[l][co] += d;
                    for (int ci = 0; ci < cin; ++ci)
                        for (int ky = 0; ky < 3; ++ky)
                            for (int kx = 0; kx < 3; ++kx) {
                                int ii = i + ky - 1, jj = j + kx - 1;
                                int64_t widx = ((co * cin + ci) * 3 + ky) * 3 + kx;
                                if (periodic) { ii = wrapi(ii, H); jj = wrapi(jj, W); }
                                else if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                                gW[l][widx] += d * hin[((int64_t)ci * H + ii) * W + jj];
                                gin[((int64_t)ci * H + ii) * W + jj] += d * Wl[l][widx];
                            }
                }
        if (l > 0) {
            for (int64_t q = 0; q < (int64_t)cin * HW; ++q)
                gy[q] = acts[(int64_t)(l - 1) * 32 * HW + q] > 0.0 ? gin[q] : 0.0;
        } else if (grad_x) {
            memcpy(grad_x, gin, sizeof(double) * 3 * HW);
        }
    }
    free(acts); free(y); free(gy); free(gin); free(hin);
    return L;
}
