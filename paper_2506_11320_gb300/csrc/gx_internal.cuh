// gx_internal.cuh -- internal declarations of the GB300 GL-ECSIM library.
//
// Data layout in HBM (2D = x-y with three velocity components; 3D = x-y-z):
//   * fields: FP64, component-major [3][N] with N = nx ny nz; E at nodes, B at
//     cell centres (collocated staggered mesh, Sec. 1.1 of the paper);
//   * particles: per species, cell bins of fixed capacity `cap` (a multiple of
//     32); each bin is a small structure of arrays of FP32 fields (o_0 ..
//     o_{d-1}, v_x, v_y, v_z, w[, id]), o the cell-local offsets in [0,1):
//     field f of slot s of cell c at p[(c cap) nf + f cap + s].  A bin holds a
//     bottom and a top segment (see bin_front / bin_back).  Two copies: the
//     push reads one and writes the other, then they swap;
//   * deposit records: per species and cell, FP32 partial sums over the cell's
//     particles (see Rec below), tile-major: entry k of cell c at
//     rec_index(size, k, c) = ((c / 8) size + k) 8 + c % 8 within the
//     species' block of ceil(N / 8) 8 size floats; written by the particle
//     kernels and folded into the FP64 node moments by the grid kernels;
//   * mass matrix: FP64 rows [o*9 + e][N], o over the 9 neighbour offsets
//     (o = (ox+1) + 3 (oy+1)), e the alpha component.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/gx.h"

#define GX_MAX_SPECIES 4
#define GX_PI 3.14159265358979323846

// --------------------------------------------------------------- records
// Per species s and cell c, sums over the particles p of s in c with cell-local
// linear weights W_a (corner a = ax + 2 ay (+ 4 az)) and pair weights
// P_j = X_jx Y_jy (Z_jz), X_0 = (1-ox)^2, X_1 = ox (1-ox), X_2 = ox^2:
//   [REC_RHO + a]            sum w W_a
//   [REC_MV + 3a + i]        sum w v_i W_a
//   [REC_J + 3a + i]         sum w (alpha (v - u_ref(x_p)))_i W_a
//   [REC_M + 9 j + e]        sum w alpha_e P_j          (alpha row-major, e = 3 r + c)
// The species factors q_s, m_s, beta_s are applied when the records are folded.
// Tile-major record layout: the kRecTile = 8 consecutive cells of a tile share
// each entry's 32-byte sector, and a tile's records are one contiguous block of
// size x 32 bytes.  The particle kernel works on the 8 cells of a tile at once
// (one warp each) and writes the block as whole sectors; the grid kernels'
// threads, one per node, read consecutive cells' entries as whole sectors.
constexpr int kRecTile = 8;
__host__ __device__ inline size_t rec_index(int size, int k, int64_t cell) {
    return ((size_t)(cell >> 3) * size + k) * kRecTile + (size_t)(cell & 7);
}
__host__ __device__ inline size_t rec_block(int size, int64_t N) {
    return (size_t)((N + kRecTile - 1) / kRecTile) * size * kRecTile;
}

template <int DIM> struct Rec;
template <> struct Rec<2> {
    static constexpr int NC = 4, NPAIR = 9;
    static constexpr int RHO = 0, MV = 4, J = 16, M = 28, USED = 109, SIZE = 112;
};
template <> struct Rec<3> {
    static constexpr int NC = 8, NPAIR = 27;
    static constexpr int RHO = 0, MV = 8, J = 32, M = 56, USED = 299, SIZE = 300;
};

// ------------------------------------------------------------- particles
// Per-bin structure of arrays: fields (o_0 .. o_{d-1}, v_x, v_y, v_z, w[, id
// bits]) of 4 bytes, nf = d + 4 (+1 with track_ids) of them per slot.

// A cell's bin holds two segments: particles that stayed in the cell during
// the last push fill slots [0, front) from the bottom, particles that arrived
// from a neighbour fill [cap - back, cap) from the top.  Both counts live in one
// 32-bit word (front in the low, back in the high 16 bits) so that a single
// atomicAdd reserves slots and sees the exact occupancy.
__host__ __device__ inline int bin_front(int w) { return w & 0xffff; }
__host__ __device__ inline int bin_back(int w) { return (int)((unsigned)w >> 16); }
__host__ __device__ inline int bin_count(int w) { return bin_front(w) + bin_back(w); }
// slot of the i-th particle of a bin (front first, then back)
__host__ __device__ inline int bin_slot(int w, int i, int cap) {
    const int f = bin_front(w);
    return i < f ? i : cap - bin_back(w) + (i - f);
}

struct Species {
    double q = 0, m = 0;
    int cap = 0;                        // bin capacity (particles per cell)
    int nf = 0;                         // FP32 fields stored per particle
    float *p[2] = {};                   // [copy]: [cell][field][cap]
    int *cnt[2] = {};                   // particles per cell, per copy
    double w2 = 0;                      // sum of the squared weights (the Gauss's-law correction's step)
};

struct BcSource {                       // plasma state of an open boundary, per species
    double n = 0, u[3] = {0, 0, 0}, vth = 0;
    int ppc = 0;
};

struct DevFlags {                       // written by kernels, read by the host
    int cfl;                            // a particle moved more than one cell
    int overflow;                       // a bin overflowed (particle dropped)
    int timeout;                        // a bounded device wait gave up
    int maxcount;                       // largest bin count after the last push
    int invalid;                        // an input array held a NaN or an infinity
};

// --------------------------------------------------------------- context
struct gx_ctx {
    gx_config cfg{};
    int dim = 2;
    int n[3] = {1, 1, 1};
    int64_t N = 0;
    double dV = 1;
    int noff = 9;                       // neighbour offsets per node (9 / 27)
    std::string err;

    // fields (FP64)
    double *E = nullptr, *B = nullptr;          // E^n (nodes), B^n (cells)
    double *phi = nullptr;                      // div B cleaning potential (cells), with divb_clean
    double *dBlf = nullptr;                     // with lf_on: D [3][N] (LF increment of B), B^n + theta D [3][N], fluxes [2][3][N]
    double *Eth = nullptr, *Enew = nullptr, *Bnew = nullptr;
    int pending = 0;                            // a solve is waiting for the push
    int have_eth = 0;                           // Eth holds E^{n-1+theta} of the step that produced E

    // FP32 node copies used by the particle kernels (float4: x, y, z, pad)
    float4 *nE = nullptr;        // E^{n+theta}
    float4 *nB = nullptr;        // B^n averaged to nodes
    float4 *nBnext = nullptr;    // B^{n+1} averaged to nodes
    float4 *nUref = nullptr;     // reference velocity subtracted in the deposit

    // particles
    int nspecies = 0;
    Species sp[GX_MAX_SPECIES];
    BcSource bsrc[2][GX_MAX_SPECIES];           // open-boundary states [side][species]
    int64_t npush = 0;                          // pushes done: the counter of the boundary draws
    int cur = 0;                                // which copy is current
    int64_t np_total = 0;

    // deposit records
    int rec_size = 112;
    float *rec = nullptr;                       // [S] blocks of rec_block(rec_size, N) floats

    // node moments (FP64)
    double *rho = nullptr, *rho_m = nullptr;    // [N]
    double *P = nullptr, *u = nullptr;          // [3][N]
    double *J = nullptr;                        // [3][N]
    double *M = nullptr;                        // [noff * 9][N] (offset o, alpha entry e at row o * 9 + e)
    double *A3 = nullptr;                       // 3D: the implicit operator as 27 blocks per node [243][N]
    float *M32 = nullptr;                       // gmres_mixed: FP32 copies of M (2D), kappa (2D) and A3 (3D)
    float *kappa32 = nullptr;
    float *A3f = nullptr;
    double *tmp3 = nullptr;                     // [3][N] scratch for filters
    double *uref64 = nullptr;                   // [3][N] FP64 copy of nUref values
    int moments_valid = 0;
    int have_u = 0;                             // u of a previous deposit exists

    // field solve
    double *kappa = nullptr;                    // [dim][3][N] LF-E coefficients
    double *rhs = nullptr, *EM = nullptr;       // [3][N]
    double *jdiag = nullptr;                    // [N][9] inverse 3x3 block diagonal
    float *jdiag32 = nullptr;                   // the same in FP32 (applied with the learned correction)
    double *V = nullptr, *Z = nullptr;          // Krylov bases [(m+1)][3N], [m][3N]
    double *w = nullptr, *r = nullptr;          // [3N]
    double *dred = nullptr;                     // reduction scratch
    int red_blocks = 0;
    double *hcol = nullptr;                     // [m+2] device column
    double *hpin = nullptr;                     // pinned host mirror of hcol
    struct GmState *gm = nullptr;               // device-side FGMRES state
    double *gpart = nullptr;                    // block partial sums
    gx_solve_stats last{};

    // learned preconditioner (allocated on demand)
    struct Net *net = nullptr;

    // flags, timers
    DevFlags *dflags = nullptr;
    DevFlags *hflags = nullptr;                 // pinned
    std::vector<cudaEvent_t> evpool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evpend[4];   // push, moments, solve, push kernel
    double t_push = 0, t_mom = 0, t_solve = 0;
    double t_pdk = 0;                           // the fused push kernel's launches alone
    int64_t n_pdk = 0;
    int64_t launches = 0;
};

// ------------------------------------------------------- shared helpers
#define GX_CHECK(ctx, call)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);             \
            return GX_ECUDA;                                                             \
        }                                                                                \
    } while (0)

#define GX_LAUNCHED(ctx)                                                                 \
    do {                                                                                 \
        cudaError_t e_ = cudaGetLastError();                                             \
        (ctx)->launches++;                                                               \
        if (e_ != cudaSuccess) {                                                         \
            (ctx)->err = std::string("kernel launch: ") + cudaGetErrorString(e_);        \
            return GX_ECUDA;                                                             \
        }                                                                                \
    } while (0)

__host__ __device__ inline int wrap_idx(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// event timing without host round trips (gx_capi.cu): an interval between two
// events recorded on the launching stream, resolved later into a category's sum
enum { GX_T_PUSH = 0, GX_T_MOM = 1, GX_T_SOLVE = 2, GX_T_PDK = 3 };
cudaEvent_t gx_ev_get(gx_ctx *c);
void gx_ev_push(gx_ctx *c, int cat, cudaEvent_t a, cudaEvent_t b);

// ------------------------------------------------ entry points per module
// particles (gx_particles.cu)
int gx_bin_particles(gx_ctx *c, int s, int64_t n, const double *x, const double *y, const double *z,
                     const float *vx, const float *vy, const float *vz, const float *w, const int32_t *id,
                     cudaStream_t st);
int gx_run_deposit(gx_ctx *c, cudaStream_t st);              // records from the current copy
int gx_run_push_deposit(gx_ctx *c, cudaStream_t st);         // mover + re-bin + records
int gx_particles_out(gx_ctx *c, int s, double *x, double *y, double *z, float *vx, float *vy, float *vz,
                     float *w, int32_t *id, cudaStream_t st);
int gx_regrow_bins(gx_ctx *c, int s, int newcap, cudaStream_t st);
// a drifting Maxwellian species drawn on the device straight into new bins of species s
int gx_species_maxwellian_init(gx_ctx *c, int s, int ppc, double n0, const double u[3], double vth,
                               cudaStream_t st);

// grid (gx_grid.cu)
int gx_node_fields(gx_ctx *c, const double *Eth, const double *Bcur, float4 *outE, float4 *outB,
                   cudaStream_t st);
int gx_assemble_moments(gx_ctx *c, cudaStream_t st);         // records -> rho, u, J, M
int gx_build_rhs(gx_ctx *c, cudaStream_t st);
int gx_build_kappa(gx_ctx *c, cudaStream_t st);
int gx_apply_A(gx_ctx *c, const double *x, double *y, cudaStream_t st);
int gx_apply_A_j(gx_ctx *c, const double *base, int64_t stride, const int *jptr, const int *doneptr, double *y,
                 cudaStream_t st);
int gx_build_jacobi(gx_ctx *c, cudaStream_t st);
// only the FP32 inverse (the learned preconditioner's base), inverted in FP32
int gx_build_jacobi32(gx_ctx *c, cudaStream_t st);
int gx_apply_jacobi(gx_ctx *c, const double *x, double *y, cudaStream_t st);
int gx_advance(gx_ctx *c, cudaStream_t st);                  // Enew, Bnew from Eth
int gx_initial_guess(gx_ctx *c, cudaStream_t st);            // Eth <- starting point of the solve
int gx_diag_run(gx_ctx *c, gx_diag *out, cudaStream_t st);

// Gauss's-law correction: the potential phi of the Gauss residual of E^n and the
// current deposit, into the .w of the node copy nE that the push reads
int gx_gl_potential(gx_ctx *c, cudaStream_t st);
int gx3_gl_potential(gx_ctx *c, cudaStream_t st);
// sum of squares of n device floats (FP64), read back (synchronises st)
int gx_sum_squares(gx_ctx *c, const float *a, int64_t n, cudaStream_t st, double *out);

// 3D grid (gx_grid3.cu): the same steps on a grid with a resolved z axis
int gx3_node_fields(gx_ctx *c, const double *Eth, const double *Bcur, float4 *outE, float4 *outB, cudaStream_t st);
int gx3_assemble_moments(gx_ctx *c, cudaStream_t st);
int gx3_build_rhs(gx_ctx *c, cudaStream_t st);
int gx3_build_kappa(gx_ctx *c, cudaStream_t st);
int gx3_build_op(gx_ctx *c, cudaStream_t st);            // assemble the operator blocks A3 for this solve
int gx3_apply_A(gx_ctx *c, const double *x, double *y, cudaStream_t st);
int gx3_build_jacobi(gx_ctx *c, bool fp64, cudaStream_t st);
int gx3_advance(gx_ctx *c, cudaStream_t st);
int gx3_filter(gx_ctx *c, double *f, int passes, bool alternate, cudaStream_t st);
int gx3_diag_grid(gx_ctx *c, double *acc, cudaStream_t st);

// solver (gx_gmres.cu)
int gx_fgmres(gx_ctx *c, cudaStream_t st);
size_t gx_gm_state_bytes();
size_t gx_gm_partial_count();
int gx_gm_max_restart();
double gx_norm_host(gx_ctx *c, const double *x, int64_t n, cudaStream_t st, int *status);

// allocation-free particle gather (gx_noalloc.cu): scratch lookup and module
// load at context creation
int gx_noalloc_prepare(gx_ctx *c);

// network (gx_net.cu)
// device pointers the solver kernel needs to apply the network itself: BF16
// forward weights [coutP][9][cinP] and FP32 biases of the 4 layers, the NHWC
// BF16 activation buffers (16, 32, 32, 32 channels) and the FP32 output [pix][8]
struct NetSolverArgs {
    const void *w[4];       // weights in the tensor-core operand layout
    const float *b[4];
    void *x0, *h1, *h2, *h3; // layer inputs: channel-blocked images with a halo ring
    unsigned *flags;        // per-unit completion flags of the network pipeline
};
int gx_net_solver_args(gx_ctx *c, NetSolverArgs *out, cudaStream_t st);
int gx_net_collecting(const gx_ctx *c);
int gx_net_pair_begin(gx_ctx *c, const double *r0, cudaStream_t st);
int gx_net_pair_end(gx_ctx *c, int converged, int nbasis, cudaStream_t st);
void gx_net_free(gx_ctx *c);
