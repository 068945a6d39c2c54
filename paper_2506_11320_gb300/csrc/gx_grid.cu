// gx_grid.cu -- grid kernels of the GL-ECSIM step (2D, FP64 fields).
//
// Mesh (Sec. 1.1): E at nodes, B at cell centres; node (i,j) at (i dx, j dy),
// cell (i,j) spans [i,i+1] x [j,j+1]; periodic.  Derivatives of a node field at
// a cell are differences of the face-averaged corner values, derivatives of a
// cell field at a node are differences of the side-averaged neighbouring cells,
// so that curl_N and curl_C are adjoint and div_C curl_N = 0 exactly.
//
// Layouts (component-major so that neighbouring threads touch neighbouring
// addresses): vector fields [3][N], mass-matrix rows [81][N] (entry o*9 + e:
// neighbour offset o = (ox+1) + 3 (oy+1), alpha component e), deposit records
// tile-major per species (rec_index).
#include "gx_op.cuh"

namespace {

constexpr int kB = 256;
// CTAs per SM the register budget of the heavier one-thread-per-node kernels
// must allow (64 registers a thread): a 512 x 256 node grid is then one wave
// of 512 CTAs over 152 SMs instead of 1.7 waves at two CTAs per SM
constexpr int kNodeCtas = 4;


// threads and CTAs of the one-thread-per-node kernels: 256-thread CTAs once the
// grid gives every SM two of them; on smaller grids (the narrow shock grids)
// smaller CTAs, down to one warp, so that the nodes still spread over all SMs
inline int node_threads(int64_t n) {
    int t = kB;
    while (t > 32 && (n + t - 1) / t < 2 * 152) t >>= 1;
    return t;
}
inline int node_blocks(int64_t n) {
    const int t = node_threads(n);
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, (int64_t)152 * 32 * (kB / t)));
}

#define GRID_LOOP(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ------------------------------------------------------ FP32 node copies
// E^{n+theta} as float4 per node; B averaged from the 4 cells around a node.
__global__ void k_node_fields(G2 g, const double *__restrict__ E, const double *__restrict__ B, float4 *outE,
                              float4 *outB) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
        if (outE) outE[q] = make_float4((float)E[q], (float)E[N + q], (float)E[2 * N + q], 0.f);
        if (outB) {
            const int64_t c0 = g.id(i - 1, j - 1), c1 = g.id(i, j - 1), c2 = g.id(i - 1, j), c3 = q;
            double b[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) b[k] = 0.25 * (B[k * N + c0] + B[k * N + c1] + B[k * N + c2] + B[k * N + c3]);
            outB[q] = make_float4((float)b[0], (float)b[1], (float)b[2], 0.f);
        }
    }
}

// ------------------------------------------------------ moment assembly
struct SpecK {
    int ns;
    double q[GX_MAX_SPECIES], m[GX_MAX_SPECIES], bq[GX_MAX_SPECIES];   // bq = beta_s q_s
    float bqf[GX_MAX_SPECIES];
};

// Record value of species s, row k, cell (FP32, as the particle kernels wrote it).
struct Recs {
    const float *a;           // species blocks of the tile-major records
    int64_t N;
    __device__ __forceinline__ float get(int s, int k, int64_t cell) const {
        return a[(size_t)s * rec_block(Rec<2>::SIZE, N) + rec_index(Rec<2>::SIZE, k, cell)];
    }
};

// rho, mass density, momentum and the raw plasma velocity at every node from
// the per-species cell records of the 4 cells around it.  The cell sums of
// one species are FP32 (the records are FP32 partial sums); species are
// combined in FP64.
__global__ void __launch_bounds__(kB, kNodeCtas) k_assemble_bulk(G2 g, SpecK sk, Recs R, double inv_dV, double *rho, double *rho_m, double *P,
                                double *u) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
        int64_t cell[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) cell[a] = g.id(i - (a & 1), j - (a >> 1));   // corner a of that cell is this node
        double r = 0, rm = 0, p[3] = {0, 0, 0};
        for (int s = 0; s < sk.ns; ++s) {
            float w = 0.f, mv[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                w += R.get(s, Rec<2>::RHO + a, cell[a]);
#pragma unroll
                for (int k = 0; k < 3; ++k) mv[k] += R.get(s, Rec<2>::MV + 3 * a + k, cell[a]);
            }
            r += sk.q[s] * (double)w;
            rm += sk.m[s] * (double)w;
#pragma unroll
            for (int k = 0; k < 3; ++k) p[k] += sk.m[s] * (double)mv[k];
        }
        rho[q] = r * inv_dV;
        rho_m[q] = rm;
        const double irm = rm != 0.0 ? 1.0 / rm : 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            P[k * N + q] = p[k];
            u[k * N + q] = p[k] * irm;
        }
    }
}

// All passes of the digital filter (Sec. 1.4, Eq. 26: v* = phi v + (1-phi)/2
// (v_{-d} + v_{+d}), phi = 0.5) on a 3-component node field, one 32x32 tile per
// CTA (32 x 8 threads, one component each) with a halo of sum(d) nodes loaded once, every sweep
// done in shared memory (x then y within each pass).  Strides alternate
// 1, 2, 1, ... when `alternate`, else all 1.  The sweeps run in FP32 (three
// operations per node and sweep, a few 1e-7 of the smoothed value after five
// passes); input and output stay FP64.
constexpr int kFT = 32;
constexpr int kFHaloMax = 16;
__device__ __forceinline__ int wrap_any(int i, int n) {
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
}
__global__ void __launch_bounds__(256) k_filter_fused(G2 g, const double *__restrict__ in, double *out, int npass,
                                                      int alternate) {
    extern __shared__ float fsh[];
    int halo = 0;
    for (int p = 0; p < npass; ++p) halo += (alternate && (p & 1)) ? 2 : 1;
    const int hx = g.nx > 1 ? halo : 0, hy = g.ny > 1 ? halo : 0;
    const int W = kFT + 2 * hx, H = kFT + 2 * hy;
    float *a = fsh, *b = fsh + W * H;
    const int x0 = blockIdx.x * kFT, y0 = blockIdx.y * kFT;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t N = g.N();
    {
        const int comp = blockIdx.z;       // one component per CTA layer
        const double *src = in + comp * N;
        for (int ly = ty; ly < H; ly += 8) {
            const int64_t row = (int64_t)g.nx * wrap_any(y0 + ly - hy, g.ny);
            for (int lx = tx; lx < W; lx += 32) a[ly * W + lx] = (float)src[row + wrap_any(x0 + lx - hx, g.nx)];
        }
        __syncthreads();
        for (int p = 0; p < npass; ++p) {
            const int d = (alternate && (p & 1)) ? 2 : 1;
            for (int axis = 0; axis < 2; ++axis) {
                if ((axis == 0 && g.nx == 1) || (axis == 1 && g.ny == 1)) continue;
                const int step = axis == 0 ? d : d * W;
                for (int ly = ty; ly < H; ly += 8)
                    for (int lx = tx; lx < W; lx += 32) {
                        const int t = ly * W + lx;
                        const bool inside = axis == 0 ? (lx >= d && lx < W - d) : (ly >= d && ly < H - d);
                        b[t] = inside ? fmaf(0.5f, a[t], 0.25f * (a[t - step] + a[t + step])) : a[t];
                    }
                __syncthreads();
                float *tmp = a; a = b; b = tmp;
            }
        }
        for (int ly = ty; ly < kFT; ly += 8)
            for (int lx = tx; lx < kFT; lx += 32) {
                const int gx = x0 + lx, gy = y0 + ly;
                if (gx < g.nx && gy < g.ny) out[comp * N + gx + (int64_t)g.nx * gy] = (double)a[(lx + hx) + W * (ly + hy)];
            }
    }
}

// FP32 -> FP64 widening written from the IEEE-754 binary32/binary64 layouts:
// sign kept, exponent rebiased (127 -> 1023, i.e. + 896), the 23 mantissa bits
// moved to the top of the 52.  Exact, and on the integer pipe: the hardware
// conversion runs at the FP64 rate (1/64 of FP32 on this part).  Zeros,
// infinities and NaNs map directly; subnormal inputs take the hardware path.
__device__ __forceinline__ double widen_f32(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu, sign = u & 0x80000000u;
    if (e == 0u && m != 0u) return (double)f;
    const uint32_t hi = e == 0u ? sign : (sign | ((e == 0xffu ? 0x7ffu : e + 896u) << 20) | (m >> 3));
    return __hiloint2double((int)hi, (int)(m << 29));
}

// Comoving current and mass-matrix rows at every node (Sec. 2.1, Eq. 33-35).
// J: the records hold sum w alpha (v - u_ref); the comoving current subtracts
// the plasma velocity u of this deposit, so the difference u - u_ref is
// removed through the mass-matrix sums (exactly: alpha is linear in the
// velocity), J_C = sum_s q_s [sum w alpha (v - u_ref) W - sum_b M_b (u - u_ref)_b].
// M: block o = (ox,oy) of node g collects every cell holding both g and g + o.
// Along x: ox = 0 -> cells -1 (pair class 2) and 0 (class 0); ox = +1 -> cell 0
// (class 1); ox = -1 -> cell -1 (class 1); the same in y.  Cell sums of one
// species are FP32 (the records are FP32 partial sums); the current's species
// are combined in FP64, the mass matrix (all species add with beta_s q_s > 0)
// in FP32 and stored as FP64.
__global__ void __launch_bounds__(kB, kNodeCtas) k_assemble_main(G2 g, SpecK sk, Recs R, double inv_dV, int comoving, const double *__restrict__ u,
                                const double *__restrict__ uref, double *J, double *M, float *M32) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
        double jc[3] = {0, 0, 0};
        float du[3][3][3];          // (u - u_ref) at the 3x3 nodes around q: [dy+1][dx+1][k]
        if (comoving) {
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const int64_t nb = g.id(i + dx, j + dy);
#pragma unroll
                    for (int k = 0; k < 3; ++k) du[dy + 1][dx + 1][k] = (float)(u[k * N + nb] - uref[k * N + nb]);
                }
        }
        // the raw current: the J entries of the 4 cells (corner a of each is this node)
        float js[GX_MAX_SPECIES][3];
#pragma unroll
        for (int s = 0; s < GX_MAX_SPECIES; ++s) js[s][0] = js[s][1] = js[s][2] = 0.f;
#pragma unroll
        for (int s = 0; s < GX_MAX_SPECIES; ++s) {
            if (s >= sk.ns) break;
#pragma unroll
            for (int cy = -1; cy <= 0; ++cy)
#pragma unroll
                for (int cx = -1; cx <= 0; ++cx) {
                    const int64_t cell = g.id(i + cx, j + cy);
                    const int a = -cx + 2 * (-cy);
#pragma unroll
                    for (int k = 0; k < 3; ++k) js[s][k] += R.get(s, Rec<2>::J + 3 * a + k, cell);
                }
        }
        // the mass-matrix blocks; the comoving correction -M^0 (u - u_ref) reads the same
        // record entries (block o of this node pairs it with node q + o, whose u - u_ref
        // the entries multiply), so it is accumulated here, each entry loaded once
#pragma unroll
        for (int o = 0; o < 9; ++o) {
            const int ox = o % 3 - 1, oy = o / 3 - 1;
            const float *d = du[oy + 1][ox + 1];
            float blk[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) blk[e] = 0.f;
            const int ncx = ox == 0 ? 2 : 1, ncy = oy == 0 ? 2 : 1;
#pragma unroll
            for (int tyy = 0; tyy < ncy; ++tyy) {
                const int cy = oy == 0 ? -tyy : (oy > 0 ? 0 : -1);
                const int jy = oy == 0 ? (cy == -1 ? 2 : 0) : 1;
#pragma unroll
                for (int txx = 0; txx < ncx; ++txx) {
                    const int cx = ox == 0 ? -txx : (ox > 0 ? 0 : -1);
                    const int jx = ox == 0 ? (cx == -1 ? 2 : 0) : 1;
                    const int64_t cell = g.id(i + cx, j + cy);
                    const int mrow = Rec<2>::M + 9 * (jx + 3 * jy);
#pragma unroll
                    for (int s = 0; s < GX_MAX_SPECIES; ++s) {
                        if (s >= sk.ns) break;
                        const float f = sk.bqf[s];
                        float mv[9];
#pragma unroll
                        for (int e = 0; e < 9; ++e) {
                            mv[e] = R.get(s, mrow + e, cell);
                            blk[e] = fmaf(f, mv[e], blk[e]);
                        }
                        if (comoving) {
#pragma unroll
                            for (int r = 0; r < 3; ++r)
                                js[s][r] -= mv[3 * r] * d[0] + mv[3 * r + 1] * d[1] + mv[3 * r + 2] * d[2];
                        }
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 9; ++e) M[(size_t)(o * 9 + e) * N + q] = widen_f32(blk[e]);
            if (M32)   // the FP32 copy the mixed-precision Krylov cycles apply
#pragma unroll
                for (int e = 0; e < 9; ++e) M32[(size_t)(o * 9 + e) * N + q] = blk[e];
        }
#pragma unroll
        for (int s = 0; s < GX_MAX_SPECIES; ++s)
            if (s < sk.ns)
#pragma unroll
                for (int k = 0; k < 3; ++k) jc[k] += sk.q[s] * (double)js[s][k];
#pragma unroll
        for (int k = 0; k < 3; ++k) J[k * N + q] = jc[k] * inv_dV;
    }
}

// starting point of the field solve: E^{n+theta} extrapolated linearly from
// E^{n-1+theta} (the previous solution, in x) and E^n:
// x = E^n + theta/(1-theta) (E^n - x), or E^n itself when there is no previous solution
__global__ void k_guess(int64_t n, const double *__restrict__ E, double *x, double f) {
    GRID_LOOP(t, n) { x[t] = f != 0.0 ? E[t] + f * (E[t] - x[t]) : E[t]; }
}

__global__ void k_copy_uref(int64_t N, const double *__restrict__ u, float4 *nU, double *u64, int zero) {
    GRID_LOOP(q, N) {
        float4 v = zero ? make_float4(0.f, 0.f, 0.f, 0.f)
                        : make_float4((float)u[q], (float)u[N + q], (float)u[2 * N + q], 0.f);
        nU[q] = v;
        u64[q] = v.x; u64[N + q] = v.y; u64[2 * N + q] = v.z;
    }
}

// ------------------------------------------------------------- operators
// derivatives of a cell field at node (i,j)
__device__ __forceinline__ double dNx(const G2 &g, const double *f, int i, int j) {
    return ((f[g.id(i, j - 1)] + f[g.id(i, j)]) - (f[g.id(i - 1, j - 1)] + f[g.id(i - 1, j)])) * g.hx;
}
__device__ __forceinline__ double dNy(const G2 &g, const double *f, int i, int j) {
    return ((f[g.id(i - 1, j)] + f[g.id(i, j)]) - (f[g.id(i - 1, j - 1)] + f[g.id(i, j - 1)])) * g.hy;
}
// derivatives of a node field at cell (i,j)
__device__ __forceinline__ double dCx(const G2 &g, const double *f, int i, int j) {
    return ((f[g.id(i + 1, j)] + f[g.id(i + 1, j + 1)]) - (f[g.id(i, j)] + f[g.id(i, j + 1)])) * g.hx;
}
__device__ __forceinline__ double dCy(const G2 &g, const double *f, int i, int j) {
    return ((f[g.id(i, j + 1)] + f[g.id(i + 1, j + 1)]) - (f[g.id(i, j)] + f[g.id(i + 1, j)])) * g.hy;
}

__global__ void k_matvec(OpArgs a, const double *__restrict__ x, double *__restrict__ y, const int *jptr,
                         int64_t stride, const int *doneptr) {
    // device-indexed operand (Krylov column j of a basis) and early exit once
    // the solver flagged the cycle done
    if (doneptr && *doneptr) return;
    if (jptr) x += (int64_t)(*jptr) * stride;
    const int64_t N = a.g.N();
    GRID_LOOP(q, N) {
        double out[3];
        gx_apply_A_node(a, x, q, out);
        y[q] = out[0];
        y[N + q] = out[1];
        y[2 * N + q] = out[2];
    }
}

// div B cleaning (Sec. 1.3): phi = decay (phi - dtch2 div B), the central
// divergence of the cell-centred B^{n+1} over neighbouring cells
__global__ void k_divb_phi(G2 g, const double *__restrict__ B, double dtch2, double decay, double *phi) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
        double d = 0.0;
        if (g.nx > 1) d += (B[g.id(i + 1, j)] - B[g.id(i - 1, j)]) * g.hx;
        if (g.ny > 1) d += (B[N + g.id(i, j + 1)] - B[N + g.id(i, j - 1)]) * g.hy;
        phi[q] = decay * (phi[q] - dtch2 * d);
    }
}

// Gauss residual of cell (i,j): R = (div_C E) / (4 pi) - rhobar, rhobar the mean
// of rho over the cell's 4 corner nodes (the Gauss's-law correction)
__global__ void k_gl_residual(G2 g, const double *__restrict__ E, const double *__restrict__ rho, double *R) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
        const double divE = dCx(g, E, i, j) + dCy(g, E + N, i, j);
        const double rb = 0.25 * (rho[q] + rho[g.id(i + 1, j)] + rho[g.id(i, j + 1)] + rho[g.id(i + 1, j + 1)]);
        R[q] = divE * (0.25 / GX_PI) - rb;
    }
}
// phi at node (i,j): the mean of R over the 4 cells around it, into nE[q].w
__global__ void k_gl_phi(G2 g, const double *__restrict__ R, float4 *nE) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
        nE[q].w = (float)(0.25 * (R[g.id(i - 1, j - 1)] + R[g.id(i, j - 1)] + R[g.id(i - 1, j)] + R[q]));
    }
}

// 3x3 diagonal block of A at every node, inverted (block-Jacobi preconditioner),
// in FP64 and in FP32
__global__ void k_jacobi(OpArgs a, double *jd, float *jd32) {
    const G2 &g = a.g;
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        // self-coupling of curl_N curl_C on this mesh: 1/dy^2 for x, 1/dx^2 for
        // y and their sum for z (2D, averaged second differences)
        const double sx = g.nx > 1 ? 1.0 / (g.dx * g.dx) : 0.0;
        const double sy = g.ny > 1 ? 1.0 / (g.dy * g.dy) : 0.0;
        double A[9] = {1 + a.ct2 * sy, 0, 0, 0, 1 + a.ct2 * sx, 0, 0, 0, 1 + a.ct2 * (sx + sy)};
        if (a.M) {
#pragma unroll
            for (int e = 0; e < 9; ++e) A[e] += a.mfac * a.M[(size_t)(4 * 9 + e) * N + q];   // centre offset
        }
        if (a.kappa) {
            const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
            const int64_t xm = g.id(i - 1, j), ym = g.id(i, j - 1);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double d = 0;
                if (g.nx > 1) d += a.lfx * (a.kappa[(0 * 3 + c) * N + q] + a.kappa[(0 * 3 + c) * N + xm]);
                if (g.ny > 1) d += a.lfy * (a.kappa[(1 * 3 + c) * N + q] + a.kappa[(1 * 3 + c) * N + ym]);
                A[4 * c] += d;
            }
        }
        if (g.bnode((int)q - (int)((unsigned)q / (unsigned)g.nx) * g.nx)) {   // Dirichlet row of an open boundary: the identity
#pragma unroll
            for (int e = 0; e < 9; ++e) A[e] = (e % 4 == 0) ? 1.0 : 0.0;
        }
        if (!jd) {
            // FP32 inverse only (the learned preconditioner's base): the block is
            // assembled in FP64 and inverted at the FP32 rate
            float F[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) F[e] = (float)A[e];
            const float f00 = F[4] * F[8] - F[5] * F[7], f01 = F[5] * F[6] - F[3] * F[8], f02 = F[3] * F[7] - F[4] * F[6];
            const float fid = 1.0f / (F[0] * f00 + F[1] * f01 + F[2] * f02);
            float *o32 = jd32 + (size_t)q * 9;
            o32[0] = f00 * fid; o32[1] = (F[2] * F[7] - F[1] * F[8]) * fid; o32[2] = (F[1] * F[5] - F[2] * F[4]) * fid;
            o32[3] = f01 * fid; o32[4] = (F[0] * F[8] - F[2] * F[6]) * fid; o32[5] = (F[2] * F[3] - F[0] * F[5]) * fid;
            o32[6] = f02 * fid; o32[7] = (F[1] * F[6] - F[0] * F[7]) * fid; o32[8] = (F[0] * F[4] - F[1] * F[3]) * fid;
            continue;
        }
        const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
        const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
        const double id = 1.0 / det;
        double *o = jd + (size_t)q * 9;
        o[0] = c00 * id; o[1] = (A[2] * A[7] - A[1] * A[8]) * id; o[2] = (A[1] * A[5] - A[2] * A[4]) * id;
        o[3] = c01 * id; o[4] = (A[0] * A[8] - A[2] * A[6]) * id; o[5] = (A[2] * A[3] - A[0] * A[5]) * id;
        o[6] = c02 * id; o[7] = (A[1] * A[6] - A[0] * A[7]) * id; o[8] = (A[0] * A[4] - A[1] * A[3]) * id;
        if (jd32) {
            float *o32 = jd32 + (size_t)q * 9;
#pragma unroll
            for (int e = 0; e < 9; ++e) o32[e] = (float)o[e];
        }
    }
}

__global__ void k_apply_jacobi(int64_t N, const double *__restrict__ jd, const double *__restrict__ x, double *y) {
    GRID_LOOP(q, N) {
        const double *o = jd + (size_t)q * 9;
        const double x0 = x[q], x1 = x[N + q], x2 = x[2 * N + q];
        y[q] = o[0] * x0 + o[1] * x1 + o[2] * x2;
        y[N + q] = o[3] * x0 + o[4] * x1 + o[5] * x2;
        y[2 * N + q] = o[6] * x0 + o[7] * x1 + o[8] * x2;
    }
}

// E_M = -u x B^n / c at nodes (B averaged to nodes), the motional field of Sec. 2.1.
__global__ void k_motional(G2 g, const double *__restrict__ u, const double *__restrict__ B, double c, double *EM) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
        const int64_t c0 = g.id(i - 1, j - 1), c1 = g.id(i, j - 1), c2 = g.id(i - 1, j), c3 = q;
        double b[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) b[k] = 0.25 * (B[k * N + c0] + B[k * N + c1] + B[k * N + c2] + B[k * N + c3]);
        const double ux = u[q], uy = u[N + q], uz = u[2 * N + q];
        const double ic = 1.0 / c;     // uniform: folded by the compiler into one division per thread
        EM[q] = -(uy * b[2] - uz * b[1]) * ic;
        EM[N + q] = -(uz * b[0] - ux * b[2]) * ic;
        EM[2 * N + q] = -(ux * b[1] - uy * b[0]) * ic;
    }
}

// b = E^n + c theta dt [curl_N B^n - (4 pi / c)(J - (1/dV) M E_M)]   (Eq. 35)
__global__ void __launch_bounds__(kB, kNodeCtas) k_rhs(G2 g, const double *__restrict__ E, const double *__restrict__ B, const double *__restrict__ J,
                      const double *__restrict__ M, const double *__restrict__ EM, double ctd, double jf, double mf,
                      double *b) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
        if (g.bnode(i)) {   // Dirichlet row of an open boundary: b = E^n
#pragma unroll
            for (int c = 0; c < 3; ++c) b[c * N + q] = E[c * N + q];
            continue;
        }
        const double *Bx = B, *By = B + N, *Bz = B + 2 * N;
        double cn[3];
        cn[0] = dNy(g, Bz, i, j);
        cn[1] = -dNx(g, Bz, i, j);
        cn[2] = dNx(g, By, i, j) - dNy(g, Bx, i, j);
        double out[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) out[k] = E[k * N + q] + ctd * cn[k] - jf * J[k * N + q];
        if (EM) {
            double m[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int o = 0; o < 9; ++o) {
                const int64_t nb = g.id(i + (o % 3) - 1, j + (o / 3) - 1);
                const double e[3] = {EM[nb], EM[N + nb], EM[2 * N + nb]};
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int k = 0; k < 3; ++k) m[r] = fma(M[(size_t)(o * 9 + 3 * r + k) * N + q], e[k], m[r]);
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) out[r] = fma(mf, m[r], out[r]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) b[k * N + q] = out[k];
    }
}

// The limiter's switch (Eq. 21) and the diffusion speed are evaluated in FP32
// (GB300 runs FP32 at 64x the FP64 rate): the differences are taken in FP64,
// the ratio r, phi(r) and |u| in FP32, and the flux products in FP64.  phi is
// continuous in r, so the FP32 rounding moves the flux by ~1e-7 of itself.
__device__ __forceinline__ float mc_limiter(float r, float beta) {
    const float v = fminf(fminf(beta * r, 0.5f * (1.0f + r)), beta);
    return v > 0.f ? v : 0.f;
}
__device__ __forceinline__ float ratio(double prev, double cur) {
    return cur == 0.0 ? 0.f : (float)prev / (float)cur;
}
__device__ __forceinline__ float umag(const double *u, int64_t N, int64_t q) {
    const float a = (float)u[q], b = (float)u[N + q], d = (float)u[2 * N + q];
    return sqrtf(a * a + b * b + d * d);
}

// kappa = (1 - phi_E) a / 2 on the edge from node g to g + e_d (Eq. 19-21),
// phi_E from E^n (frozen, keeps the solve linear), a = |u| averaged over the
// edge's two nodes or a = c.
__global__ void k_kappa(G2 g, const double *__restrict__ E, const double *__restrict__ u, double beta, int speed_c,
                        double c, double *kappa, float *kappa32) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
        for (int d = 0; d < 2; ++d) {
            const int64_t p = d == 0 ? g.id(i + 1, j) : g.id(i, j + 1);
            const int64_t m = d == 0 ? g.id(i - 1, j) : g.id(i, j - 1);
            const double a = speed_c ? c : 0.5 * (double)(umag(u, N, q) + umag(u, N, p));
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                const double *Ec = E + comp * N;
                const float r = ratio(Ec[q] - Ec[m], Ec[p] - Ec[q]);
                const double kv = (double)(1.0f - mc_limiter(r, (float)beta)) * a * 0.5;
                kappa[(d * 3 + comp) * N + q] = kv;
                if (kappa32) kappa32[(d * 3 + comp) * N + q] = (float)kv;
            }
        }
    }
}

// B^{n+1} = B^n - c dt curl_C E^{n+theta} + dt/dx_d (F_{c+1/2} - F_{c-1/2}),
// F = (1 - phi_B) a / 2 (B_{c+1} - B_c)  (Eq. 5, 17, 18, 22);  E^{n+1} from Eq. 10.
// Limited LF flux of B through the +x and +y faces of every cell (Eq. 17-18),
// each face once: F = dt/dx (1 - phi_B) a / 2 (B_{c+1} - B_c) per component,
// phi_B = MC(r, beta), r = (B_c - B_{c-1}) / (B_{c+1} - B_c), a = |u| averaged
// over the face (or c).  Ff [2][3][N]: axis, component, cell.
__global__ void k_lf_flux(G2 g, const double *__restrict__ B, const double *__restrict__ u, double c, double dt,
                          double beta, int speed_c, double *Ff) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            if ((d == 0 && g.nx == 1) || (d == 1 && g.ny == 1)) continue;
            const double f = dt * 2.0 * (d == 0 ? g.hx : g.hy);
            const int64_t cp = d == 0 ? g.id(i + 1, j) : g.id(i, j + 1);
            const int64_t cm = d == 0 ? g.id(i - 1, j) : g.id(i, j - 1);
            double a;
            if (speed_c) {
                a = c;
            } else {
                const int64_t n1 = g.id(i + 1, j + 1);
                a = 0.5 * (double)(umag(u, N, cp) + umag(u, N, n1));
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double *Bk = B + k * N;
                const double dp = Bk[cp] - Bk[q];
                const float r = ratio(Bk[q] - Bk[cm], dp);
                Ff[(d * 3 + k) * N + q] = f * ((double)(1.0f - mc_limiter(r, (float)beta)) * a * 0.5 * dp);
            }
        }
    }
}

// Increment of the limited LF diffusion on B over one step, D = F_{c+1/2} -
// F_{c-1/2} along every resolved axis (0 in boundary cells), and B~ = B^n +
// theta D, the part of B^{n+theta} the E solve curls: B^{n+1} receives D.
__global__ void __launch_bounds__(kB, kNodeCtas) k_lf_b(G2 g, const double *__restrict__ B, const double *__restrict__ Ff, double theta, double *D,
                       double *Bt) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
        const int64_t xm = g.id(i - 1, j), ym = g.id(i, j - 1);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double dn = 0.0;
            if (g.nx > 1) dn += Ff[(0 * 3 + k) * N + q] - Ff[(0 * 3 + k) * N + xm];
            if (g.ny > 1) dn += Ff[(1 * 3 + k) * N + q] - Ff[(1 * 3 + k) * N + ym];
            if (g.bcell(i)) dn = 0.0;   // boundary cells keep B
            D[k * N + q] = dn;
            Bt[k * N + q] = B[k * N + q] + theta * dn;
        }
    }
}

// B^{n+1} = B^n - c dt curl_C E^{n+theta} (+ the LF increment D, - dt grad phi^n)
// and E^{n+1} = (E^{n+theta} - (1 - theta) E^n) / theta
__global__ void k_advance(G2 g, const double *__restrict__ E, const double *__restrict__ B,
                          const double *__restrict__ Eth, double c, double dt, double theta,
                          const double *__restrict__ D, const double *__restrict__ phi, double *Enew, double *Bnew) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
        const int64_t Nq = N;
        double cu[3];
        cu[0] = dCy(g, Eth + 2 * Nq, i, j);
        cu[1] = -dCx(g, Eth + 2 * Nq, i, j);
        cu[2] = dCx(g, Eth + Nq, i, j) - dCy(g, Eth, i, j);
        double bn[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) bn[k] = B[k * N + q] - c * dt * cu[k];
        if (D) {
#pragma unroll
            for (int k = 0; k < 3; ++k) bn[k] += D[k * N + q];
        }
        if (phi) {   // div B cleaning (Sec. 1.3): - dt grad phi^n, central over cells (hx = 1 / (2 dx))
            if (g.nx > 1) bn[0] -= dt * (phi[g.id(i + 1, j)] - phi[g.id(i - 1, j)]) * g.hx;
            if (g.ny > 1) bn[1] -= dt * (phi[g.id(i, j + 1)] - phi[g.id(i, j - 1)]) * g.hy;
        }
        if (g.bcell(i)) {   // open boundary: B keeps its value
#pragma unroll
            for (int k = 0; k < 3; ++k) bn[k] = B[k * N + q];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Bnew[k * N + q] = bn[k];
            Enew[k * N + q] = (Eth[k * N + q] - (1.0 - theta) * E[k * N + q]) / theta;
        }
    }
}

// ------------------------------------------------------------ diagnostics
__global__ void k_diag_grid(G2 g, const double *__restrict__ E, const double *__restrict__ B,
                            const double *__restrict__ rho, double *acc) {
    const int64_t N = g.N();
    double we = 0, wb = 0, ch = 0, gl = 0, db = 0;
    GRID_LOOP(q, N) {
        const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
        for (int k = 0; k < 3; ++k) {
            we += E[k * N + q] * E[k * N + q];
            wb += B[k * N + q] * B[k * N + q];
        }
        ch += rho ? rho[q] : 0.0;
        // Gauss residual at cell (i,j): div_C E - 4 pi (rho averaged to the cell)
        const double divE = dCx(g, E, i, j) + dCy(g, E + N, i, j);
        const double rc = rho ? 0.25 * (rho[g.id(i, j)] + rho[g.id(i + 1, j)] + rho[g.id(i, j + 1)] + rho[g.id(i + 1, j + 1)]) : 0.0;
        const double gr = divE - 4.0 * GX_PI * rc;
        gl += gr * gr;
        const double divB = dNx(g, B, i, j) + dNy(g, B + N, i, j);
        db += divB * divB;
    }
    double v[5] = {we, wb, ch, gl, db};
    for (int k = 0; k < 5; ++k) {
        double s = v[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(acc + k, s);
    }
}

// Kinetic energy, momentum and count of one species.  The per-particle terms
// w v_i v_i and w v_i come from the FP32 particle state and are formed in FP32;
// each thread sums them over 16 cells in FP32 (about 16 terms) and adds those
// partial sums into FP64 accumulators, which take the species mass at the end
// (FP64 on this part runs at 1/64 of the FP32 rate, so FP64 per particle
// would make this pass ten times slower than its memory traffic).
__global__ void k_diag_particles(int64_t ncell, int cap, int nf, int dim, const int *cnt, const float *P, double mass,
                                 double *acc) {
    double ke = 0, px = 0, py = 0, pz = 0;
    double np = 0;
    float fk = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
    int since = 0;
    for (int64_t c = blockIdx.x; c < ncell; c += gridDim.x) {
        const int word = cnt[c];
        const int m = min(bin_count(word), cap);
        if (threadIdx.x == 0) np += m;
        const float *b = P + (size_t)c * cap * nf;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const float *q = b + bin_slot(word, i, cap);
            const float vx = q[(size_t)dim * cap], vy = q[(size_t)(dim + 1) * cap], vz = q[(size_t)(dim + 2) * cap];
            const float w = q[(size_t)(dim + 3) * cap], wa = w * vx, wb = w * vy, wd = w * vz;
            fk = fmaf(wa, vx, fmaf(wb, vy, fmaf(wd, vz, fk)));
            fx += wa; fy += wb; fz += wd;
        }
        if (++since == 16) {
            ke += fk; px += fx; py += fy; pz += fz;
            fk = fx = fy = fz = 0.f;
            since = 0;
        }
    }
    ke += fk; px += fx; py += fy; pz += fz;
    double v[5] = {0.5 * mass * ke, mass * px, mass * py, mass * pz, np};
    for (int k = 0; k < 5; ++k) {
        double s = v[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(acc + k, s);
    }
}

G2 geom(const gx_ctx *c) {
    return G2{c->n[0], c->n[1], c->cfg.dx[0], c->cfg.dx[1], 0.5 / c->cfg.dx[0], 0.5 / c->cfg.dx[1], c->cfg.bc_cells,
              c->cfg.bc_cells > 0 ? c->cfg.bc_wall : 0};
}

SpecK speck(const gx_ctx *c) {
    SpecK sk{};
    sk.ns = c->nspecies;
    for (int s = 0; s < c->nspecies; ++s) {
        sk.q[s] = c->sp[s].q;
        sk.m[s] = c->sp[s].m;
        sk.bq[s] = c->sp[s].q * c->cfg.dt / (2.0 * c->sp[s].m) * c->sp[s].q;
        sk.bqf[s] = (float)sk.bq[s];
    }
    return sk;
}

OpArgs opargs(const gx_ctx *c) {
    OpArgs a{};
    a.g = geom(c);
    const double ct = c->cfg.c * c->cfg.theta * c->cfg.dt;
    a.ct2 = ct * ct;
    a.mfac = 4.0 * GX_PI * c->cfg.theta * c->cfg.dt / c->dV;
    a.lfx = c->cfg.theta * c->cfg.dt / c->cfg.dx[0];
    a.lfy = c->cfg.theta * c->cfg.dt / c->cfg.dx[1];
    a.M = c->nspecies > 0 ? c->M : nullptr;
    a.kappa = (c->cfg.lf_on && c->cfg.nsmooth_e == 0) ? c->kappa : nullptr;   // the E filter replaces LF on E
    if (c->dim == 3) {
        a.g3 = G3{c->n[0], c->n[1], c->n[2], c->cfg.dx[0], c->cfg.dx[1], c->cfg.dx[2]};
        a.A3 = c->A3;
    }
    a.M32 = c->M32;
    a.kappa32 = c->kappa32;
    a.A3f = c->A3f;
    return a;
}

// all filter passes in one launch (result written to tmp3, then back to f)
int filter_passes(gx_ctx *c, double *f, int passes, bool alternate, cudaStream_t st) {
    if (passes <= 0) return GX_OK;
    const G2 g = geom(c);
    int halo = 0;
    for (int p = 0; p < passes; ++p) halo += (alternate && (p & 1)) ? 2 : 1;
    if (halo > kFHaloMax) { c->err = "too many filter passes"; return GX_EINVAL; }
    const int hx = g.nx > 1 ? halo : 0, hy = g.ny > 1 ? halo : 0;
    const size_t smem = 2 * (size_t)(kFT + 2 * hx) * (kFT + 2 * hy) * sizeof(float);
    static size_t configured = 0;
    if (smem > configured) {
        GX_CHECK(c, cudaFuncSetAttribute(k_filter_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = smem;
    }
    dim3 grid((g.nx + kFT - 1) / kFT, (g.ny + kFT - 1) / kFT, 3);
    k_filter_fused<<<grid, dim3(32, 8), smem, st>>>(g, f, c->tmp3, passes, alternate ? 1 : 0);
    GX_LAUNCHED(c);
    GX_CHECK(c, cudaMemcpyAsync(f, c->tmp3, 3 * c->N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return GX_OK;
}

}  // namespace

OpArgs gx_opargs(const gx_ctx *c) { return opargs(c); }

int gx_node_fields(gx_ctx *c, const double *Eth, const double *Bcur, float4 *outE, float4 *outB, cudaStream_t st) {
    if (c->dim == 3) return gx3_node_fields(c, Eth, Bcur, outE, outB, st);
    k_node_fields<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(geom(c), Eth, Bcur, outE, outB);
    GX_LAUNCHED(c);
    return GX_OK;
}

// records -> rho, u (smoothed), J (comoving or standard, smoothed), M; then
// the reference velocity of the next deposit becomes this u.
int gx_assemble_moments(gx_ctx *c, cudaStream_t st) {
    if (c->dim == 3) return gx3_assemble_moments(c, st);
    const G2 g = geom(c);
    const SpecK sk = speck(c);
    const Recs R{c->rec, c->N};
    k_assemble_bulk<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(g, sk, R, 1.0 / c->dV, c->rho, c->rho_m, c->P, c->u);
    GX_LAUNCHED(c);
    int rc = filter_passes(c, c->u, c->cfg.nsmooth_u, true, st);
    if (rc) return rc;
    k_assemble_main<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(g, sk, R, 1.0 / c->dV, c->cfg.comoving, c->u, c->uref64, c->J,
                                                       c->M, c->M32);
    GX_LAUNCHED(c);
    rc = filter_passes(c, c->J, c->cfg.ns_j, false, st);
    if (rc) return rc;
    // reference velocity of the next deposit: this u (comoving) or 0
    k_copy_uref<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(c->N, c->u, c->nUref, c->uref64, c->cfg.comoving ? 0 : 1);
    GX_LAUNCHED(c);
    c->have_u = 1;
    return GX_OK;
}

int gx_build_rhs(gx_ctx *c, cudaStream_t st) {
    if (c->dim == 3) return gx3_build_rhs(c, st);
    const G2 g = geom(c);
    const bool cm = c->cfg.comoving && c->nspecies > 0;
    if (cm) {
        k_motional<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(g, c->u, c->B, c->cfg.c, c->EM);
        GX_LAUNCHED(c);
    }
    const double ctd = c->cfg.c * c->cfg.theta * c->cfg.dt;
    const double jf = 4.0 * GX_PI * c->cfg.theta * c->cfg.dt;
    // with LF on B, the right-hand side curls B~ = B^n + theta D (D: the LF increment
    // B^{n+1} receives), held in dBlf + 3N; the fluxes go to dBlf + 6N
    const double *Bc = c->B;
    if (c->cfg.lf_on) {
        double *D = c->dBlf, *Bt = c->dBlf + 3 * c->N, *Ff = c->dBlf + 6 * c->N;
        k_lf_flux<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(g, c->B, c->u, c->cfg.c, c->cfg.dt, c->cfg.lf_beta,
                                                   c->cfg.lf_speed_c, Ff);
        GX_LAUNCHED(c);
        k_lf_b<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(g, c->B, Ff, c->cfg.theta, D, Bt);
        GX_LAUNCHED(c);
        if (!c->cfg.lf_rhs_printed) Bc = Bt;   // the printed Eq. 7 curls B^n alone
    }
    k_rhs<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(g, c->E, Bc, c->J, c->M, cm ? c->EM : nullptr, ctd, jf, jf / c->dV,
                                           c->rhs);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx_build_kappa(gx_ctx *c, cudaStream_t st) {
    if (c->dim == 3) return gx3_build_kappa(c, st);
    if (!c->cfg.lf_on || c->cfg.nsmooth_e > 0) return GX_OK;
    k_kappa<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(geom(c), c->E, c->u, c->cfg.lf_beta, c->cfg.lf_speed_c, c->cfg.c,
                                              c->kappa, c->kappa32);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx_apply_A(gx_ctx *c, const double *x, double *y, cudaStream_t st) {
    if (c->dim == 3) return gx3_apply_A(c, x, y, st);
    k_matvec<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(opargs(c), x, y, nullptr, 0, nullptr);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx_apply_A_j(gx_ctx *c, const double *base, int64_t stride, const int *jptr, const int *doneptr, double *y,
                 cudaStream_t st) {
    k_matvec<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(opargs(c), base, y, jptr, stride, doneptr);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx_build_jacobi(gx_ctx *c, cudaStream_t st) {
    if (c->dim == 3) return gx3_build_jacobi(c, true, st);
    k_jacobi<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(opargs(c), c->jdiag, c->jdiag32);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx_build_jacobi32(gx_ctx *c, cudaStream_t st) {
    if (c->dim == 3) return gx3_build_jacobi(c, false, st);
    k_jacobi<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(opargs(c), nullptr, c->jdiag32);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx_apply_jacobi(gx_ctx *c, const double *x, double *y, cudaStream_t st) {
    k_apply_jacobi<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(c->N, c->jdiag, x, y);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx_initial_guess(gx_ctx *c, cudaStream_t st) {
    const double th = c->cfg.theta;
    const double f = (c->have_eth && th < 1.0) ? th / (1.0 - th) : 0.0;
    k_guess<<<node_blocks(3 * c->N), node_threads(3 * c->N), 0, st>>>(3 * c->N, c->E, c->Eth, f);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx_advance(gx_ctx *c, cudaStream_t st) {
    if (c->dim == 3) return gx3_advance(c, st);
    // the LF increment D was computed from B^n and u when the right-hand side was built
    k_advance<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(geom(c), c->E, c->B, c->Eth, c->cfg.c, c->cfg.dt, c->cfg.theta,
                                               c->cfg.lf_on ? c->dBlf : nullptr, c->phi, c->Enew, c->Bnew);
    GX_LAUNCHED(c);
    if (c->phi) {
        // phi^{n+1} = exp(-dt c_h^2 / c_p^2) (phi^n - dt c_h^2 div B^{n+1}), c_h = 0.8 dx / dt
        const double dxmin = std::min(c->n[0] > 1 ? c->cfg.dx[0] : 1e300, c->n[1] > 1 ? c->cfg.dx[1] : 1e300);
        if (dxmin < 1e300) {
            const double ch = 0.8 * dxmin / c->cfg.dt;
            k_divb_phi<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(geom(c), c->Bnew, c->cfg.dt * ch * ch, std::exp(-0.1), c->phi);
            GX_LAUNCHED(c);
        }
    }
    // E^{n+1} smoothed by nsmooth_e filter passes (strides 1, 2, 1, ...) in place of LF on E
    return filter_passes(c, c->Enew, c->cfg.nsmooth_e, true, st);
}

int gx_gl_potential(gx_ctx *c, cudaStream_t st) {
    k_gl_residual<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(geom(c), c->E, c->rho, c->tmp3);
    GX_LAUNCHED(c);
    k_gl_phi<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(geom(c), c->tmp3, c->nE);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx_copy_uref(gx_ctx *c, int zero, cudaStream_t st);
int gx_copy_uref(gx_ctx *c, int zero, cudaStream_t st) {
    k_copy_uref<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(c->N, c->u, c->nUref, c->uref64, zero);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx_diag_run(gx_ctx *c, gx_diag *out, cudaStream_t st) {
    double *acc = c->dred;
    GX_CHECK(c, cudaMemsetAsync(acc, 0, 16 * sizeof(double), st));
    if (c->dim == 3) {
        int rc = gx3_diag_grid(c, acc, st);
        if (rc) return rc;
    } else {
        k_diag_grid<<<node_blocks(c->N), node_threads(c->N), 0, st>>>(geom(c), c->E, c->B, c->moments_valid ? c->rho : nullptr, acc);
        GX_LAUNCHED(c);
    }
    for (int s = 0; s < c->nspecies; ++s) {
        const Species &S = c->sp[s];
        k_diag_particles<<<(unsigned)std::min<int64_t>(c->N, 152 * 8), 128, 0, st>>>(
            c->N, S.cap, S.nf, c->dim, S.cnt[c->cur], S.p[c->cur], S.m, acc + 5);
        GX_LAUNCHED(c);
    }
    double h[16];
    GX_CHECK(c, cudaMemcpyAsync(h, acc, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
    GX_CHECK(c, cudaStreamSynchronize(st));
    out->energy_E = h[0] * c->dV / (8.0 * GX_PI);
    out->energy_B = h[1] * c->dV / (8.0 * GX_PI);
    out->charge = h[2] * c->dV;
    out->gauss_l2 = sqrt(h[3]);
    out->divB_l2 = sqrt(h[4]);
    out->kinetic = h[5];
    out->momentum[0] = h[6]; out->momentum[1] = h[7]; out->momentum[2] = h[8];
    out->n_particles = (int64_t)llround(h[9]);
    return GX_OK;
}
