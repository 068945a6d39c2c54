// gx_grid3.cu -- grid kernels of the GL-ECSIM step on a 3D grid (FP64 fields).
//
// Mesh (Sec. 1.1): E at nodes, B at cell centres; node (i,j,k) at
// (i dx, j dy, k dz), cell (i,j,k) spans [i,i+1] x [j,j+1] x [k,k+1]; periodic.
// A derivative along d of a node field at a cell is the mean of the 4 nodes of
// the cell's +d face minus the mean of its -d face, over dx_d; of a cell field
// at a node, the mean of the 4 cells on the node's +d side minus the 4 on its
// -d side.  So curl_N and curl_C are adjoint and div_C curl_N = 0 exactly, as
// in 2D.  The mass matrix couples a node with its 27 neighbours (Sec. 2.1,
// M_gg' = sum_p q alpha W_pg W_pg'), rows [o*9 + e][N], o = (ox+1) + 3 (oy+1)
// + 9 (oz+1).
//
// The implicit operator (Eq. 7 with the mass term of Eq. 35 and the diffusive
// LF term of Eq. 19) is assembled once per solve into 27 3x3 blocks per node,
//   A_o(q) = delta_o0 I + (c theta dt)^2 K_o + (4 pi theta dt / dV) M_o(q)
//            - LF(kappa),
// K_o the curl_N curl_C stencil: along an axis the composition of the two
// averaged differences is [1,-2,1]/dx^2 (same axis) or [-1,0,1]/(2 dx) (mixed),
// and [1,2,1]/4 across, so (curl curl x)_i = sum_{j != i} (D_j D_i x_j -
// D_j D_j x_i).  A matrix-vector product is then 27 block products per node,
// read once from memory (a 3D node has three times the 2D neighbours, and the
// expanded curl-curl would triple the FP64 work of every Krylov step).
#include "gx_op.cuh"

namespace {

constexpr int kB = 256;

inline int blocks_for(int64_t n) {
    int64_t b = (n + kB - 1) / kB;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

#define GRID_LOOP(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

struct H4 {
    double v[3];          // 1 / (4 dx_d): the face means' factor over dx_d
};

struct SpecK3 {
    int ns;
    double q[GX_MAX_SPECIES], m[GX_MAX_SPECIES];
    float bqf[GX_MAX_SPECIES];   // beta_s q_s
    float qf[GX_MAX_SPECIES];    // q_s
};

struct Recs3 {
    const float *a;       // species blocks of the tile-major records
    int64_t N;
    __device__ __forceinline__ float get(int s, int k, int64_t cell) const {
        return a[(size_t)s * rec_block(Rec<3>::SIZE, N) + rec_index(Rec<3>::SIZE, k, cell)];
    }
};

struct K3 {
    double k[27][9];      // (c theta dt)^2 times the curl_N curl_C stencil, [offset][3 row + col]
};

// derivative along d of a node field at cell (i,j,k)
__device__ __forceinline__ double dC3(const G3 &g, const H4 &h, const double *f, int i, int j, int k, int d) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int o0 = a & 1, o1 = (a >> 1) & 1, o2 = (a >> 2) & 1;
        const int od = d == 0 ? o0 : (d == 1 ? o1 : o2);
        const double v = f[g.id(i + o0, j + o1, k + o2)];
        s += od ? v : -v;
    }
    return s * h.v[d];
}
// derivative along d of a cell field at node (i,j,k)
__device__ __forceinline__ double dN3(const G3 &g, const H4 &h, const double *f, int i, int j, int k, int d) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int o0 = a & 1, o1 = (a >> 1) & 1, o2 = (a >> 2) & 1;
        const int od = d == 0 ? o0 : (d == 1 ? o1 : o2);
        const double v = f[g.id(i - 1 + o0, j - 1 + o1, k - 1 + o2)];
        s += od ? v : -v;
    }
    return s * h.v[d];
}
// mean of a cell field over the 8 cells around node (i,j,k)
__device__ __forceinline__ double cell_mean(const G3 &g, const double *f, int i, int j, int k) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) s += f[g.id(i - 1 + (a & 1), j - 1 + ((a >> 1) & 1), k - 1 + ((a >> 2) & 1))];
    return 0.125 * s;
}

// ------------------------------------------------------ FP32 node copies
__global__ void k3_node_fields(G3 g, const double *__restrict__ E, const double *__restrict__ B, float4 *outE,
                               float4 *outB) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        if (outE) outE[q] = make_float4((float)E[q], (float)E[N + q], (float)E[2 * N + q], 0.f);
        if (outB) {
            int i, j, k;
            g.ijk(q, i, j, k);
            outB[q] = make_float4((float)cell_mean(g, B, i, j, k), (float)cell_mean(g, B + N, i, j, k),
                                  (float)cell_mean(g, B + 2 * N, i, j, k), 0.f);
        }
    }
}

// ------------------------------------------------------ moment assembly
// rho, mass density, momentum and the raw plasma velocity at every node from
// the records of the 8 cells around it (corner a of cell q - a is node q)
__global__ void k3_assemble_bulk(G3 g, SpecK3 sk, Recs3 R, double inv_dV, double *rho, double *rho_m, double *P,
                                 double *u) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        int i, j, k;
        g.ijk(q, i, j, k);
        double r = 0, rm = 0, p[3] = {0, 0, 0};
        for (int s = 0; s < sk.ns; ++s) {
            float w = 0.f, mv[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const int64_t cell = g.id(i - (a & 1), j - ((a >> 1) & 1), k - ((a >> 2) & 1));
                w += R.get(s, Rec<3>::RHO + a, cell);
#pragma unroll
                for (int c = 0; c < 3; ++c) mv[c] += R.get(s, Rec<3>::MV + 3 * a + c, cell);
            }
            r += sk.q[s] * (double)w;
            rm += sk.m[s] * (double)w;
#pragma unroll
            for (int c = 0; c < 3; ++c) p[c] += sk.m[s] * (double)mv[c];
        }
        rho[q] = r * inv_dV;
        rho_m[q] = rm;
        const double irm = rm != 0.0 ? 1.0 / rm : 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            P[c * N + q] = p[c];
            u[c * N + q] = p[c] * irm;
        }
    }
}

// comoving current and the 27 mass-matrix blocks at every node (Sec. 2.1,
// Eq. 33-35).  J: the records hold sum w alpha (v - u_ref) W; the plasma
// velocity u of this deposit replaces u_ref through the mass-matrix sums
// (alpha is linear in the velocity): J_C(q) = sum_s q_s [sum_cells J records
// - sum_o Mraw_s,o(q) (u - u_ref)(q + o)] / dV, Mraw_s,o the unweighted pair
// sums of block o.  M: block o of node q collects every cell holding both q
// and q + o; per axis: o_d = 0 -> cells -1 (pair class 2) and 0 (class 0),
// o_d = +1 -> cell 0 (class 1), o_d = -1 -> cell -1 (class 1).  One pass over
// the blocks reads each (cell, class) record row once for both: weighted by
// beta_s q_s into M, by q_s into the current's correction.
__global__ void k3_assemble_main(G3 g, SpecK3 sk, Recs3 R, double inv_dV, int comoving,
                                 const double *__restrict__ u, const double *__restrict__ uref, double *J,
                                 double *M) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        int i, j, k;
        g.ijk(q, i, j, k);
        float jc[3] = {0.f, 0.f, 0.f};                       // comoving correction, summed over species
        double jr[3] = {0, 0, 0};                            // current records, species combined in FP64
        for (int s = 0; s < sk.ns; ++s) {
            float js[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const int64_t cell = g.id(i - (a & 1), j - ((a >> 1) & 1), k - ((a >> 2) & 1));
#pragma unroll
                for (int c = 0; c < 3; ++c) js[c] += R.get(s, Rec<3>::J + 3 * a + c, cell);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) jr[c] += sk.q[s] * (double)js[c];
        }
        for (int o = 0; o < 27; ++o) {
            const int oo[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
            float blk[9], blq[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) { blk[e] = 0.f; blq[e] = 0.f; }
            const int nt = (oo[0] == 0 ? 2 : 1) * (oo[1] == 0 ? 2 : 1) * (oo[2] == 0 ? 2 : 1);
            for (int t = 0; t < nt; ++t) {
                int cof[3], cls[3], tt = t;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (oo[d] == 0) {
                        const int pick = tt & 1;
                        tt >>= 1;
                        cof[d] = -pick;
                        cls[d] = pick ? 2 : 0;
                    } else {
                        cof[d] = oo[d] > 0 ? 0 : -1;
                        cls[d] = 1;
                    }
                }
                const int64_t cell = g.id(i + cof[0], j + cof[1], k + cof[2]);
                const int mrow = Rec<3>::M + 9 * (cls[0] + 3 * cls[1] + 9 * cls[2]);
                for (int s = 0; s < sk.ns; ++s) {
                    const float f = sk.bqf[s], fq = sk.qf[s];
#pragma unroll
                    for (int e = 0; e < 9; ++e) {
                        const float r = R.get(s, mrow + e, cell);
                        blk[e] = fmaf(f, r, blk[e]);
                        blq[e] = fmaf(fq, r, blq[e]);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < 9; ++e) M[(size_t)(o * 9 + e) * N + q] = (double)blk[e];
            if (comoving) {
                const int64_t nb = g.id(i + oo[0], j + oo[1], k + oo[2]);
                float d[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) d[c] = (float)(u[c * N + nb] - uref[c * N + nb]);
#pragma unroll
                for (int r = 0; r < 3; ++r) jc[r] += blq[3 * r] * d[0] + blq[3 * r + 1] * d[1] + blq[3 * r + 2] * d[2];
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) J[c * N + q] = (jr[c] - (double)jc[c]) * inv_dV;
    }
}

// one sweep of the digital filter (Sec. 1.4, Eq. 26, phi = 0.5) along `axis`
// with stride `st` on a 3-component node field: v* = v/2 + (v_- + v_+)/4
__global__ void k3_filter_sweep(G3 g, const double *__restrict__ in, double *out, int axis, int st) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        int i, j, k;
        g.ijk(q, i, j, k);
        const int64_t m = axis == 0 ? g.id(i - st, j, k) : (axis == 1 ? g.id(i, j - st, k) : g.id(i, j, k - st));
        const int64_t p = axis == 0 ? g.id(i + st, j, k) : (axis == 1 ? g.id(i, j + st, k) : g.id(i, j, k + st));
#pragma unroll
        for (int c = 0; c < 3; ++c) out[c * N + q] = 0.5 * in[c * N + q] + 0.25 * (in[c * N + m] + in[c * N + p]);
    }
}

// E_M = -u x B^n / c at nodes (B averaged to nodes), the motional field of Sec. 2.1
__global__ void k3_motional(G3 g, const double *__restrict__ u, const double *__restrict__ B, double c, double *EM) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        int i, j, k;
        g.ijk(q, i, j, k);
        const double b0 = cell_mean(g, B, i, j, k), b1 = cell_mean(g, B + N, i, j, k), b2 = cell_mean(g, B + 2 * N, i, j, k);
        const double ux = u[q], uy = u[N + q], uz = u[2 * N + q];
        const double ic = 1.0 / c;
        EM[q] = -(uy * b2 - uz * b1) * ic;
        EM[N + q] = -(uz * b0 - ux * b2) * ic;
        EM[2 * N + q] = -(ux * b1 - uy * b0) * ic;
    }
}

// b = E^n + c theta dt [curl_N B~ - (4 pi / c)(J - (1/dV) M E_M)]   (Eq. 35)
__global__ void k3_rhs(G3 g, H4 h, const double *__restrict__ E, const double *__restrict__ B,
                       const double *__restrict__ J, const double *__restrict__ M, const double *__restrict__ EM,
                       double ctd, double jf, double mf, double *b) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        int i, j, k;
        g.ijk(q, i, j, k);
        const double *Bx = B, *By = B + N, *Bz = B + 2 * N;
        double cn[3];
        cn[0] = dN3(g, h, Bz, i, j, k, 1) - dN3(g, h, By, i, j, k, 2);
        cn[1] = dN3(g, h, Bx, i, j, k, 2) - dN3(g, h, Bz, i, j, k, 0);
        cn[2] = dN3(g, h, By, i, j, k, 0) - dN3(g, h, Bx, i, j, k, 1);
        double out[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) out[c] = E[c * N + q] + ctd * cn[c] - jf * J[c * N + q];
        if (EM) {
            double m[3] = {0.0, 0.0, 0.0};
            for (int o = 0; o < 27; ++o) {
                const int64_t nb = g.id(i + o % 3 - 1, j + (o / 3) % 3 - 1, k + o / 9 - 1);
                const double e[3] = {EM[nb], EM[N + nb], EM[2 * N + nb]};
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) m[r] = fma(M[(size_t)(o * 9 + 3 * r + c) * N + q], e[c], m[r]);
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) out[r] = fma(mf, m[r], out[r]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) b[c * N + q] = out[c];
    }
}

// The limiter's switch (Eq. 21) and the diffusion speed in FP32, the
// differences and flux products in FP64 (as on the 2D grid)
__device__ __forceinline__ float mc_limiter3(float r, float beta) {
    const float v = fminf(fminf(beta * r, 0.5f * (1.0f + r)), beta);
    return v > 0.f ? v : 0.f;
}
__device__ __forceinline__ float ratio3(double prev, double cur) { return cur == 0.0 ? 0.f : (float)prev / (float)cur; }
__device__ __forceinline__ float umag3(const double *u, int64_t N, int64_t q) {
    const float a = (float)u[q], b = (float)u[N + q], d = (float)u[2 * N + q];
    return sqrtf(a * a + b * b + d * d);
}
__device__ __forceinline__ int64_t shift(const G3 &g, int i, int j, int k, int d, int s) {
    return d == 0 ? g.id(i + s, j, k) : (d == 1 ? g.id(i, j + s, k) : g.id(i, j, k + s));
}

// kappa = (1 - phi_E) a / 2 on the edge from node q to q + e_d (Eq. 19-21), phi_E
// from E^n, a = |u| averaged over the edge's two nodes or a = c
__global__ void k3_kappa(G3 g, const double *__restrict__ E, const double *__restrict__ u, double beta, int speed_c,
                         double c, double *kappa) {
    const int64_t N = g.N();
    const int n3[3] = {g.nx, g.ny, g.nz};
    GRID_LOOP(q, N) {
        int i, j, k;
        g.ijk(q, i, j, k);
        for (int d = 0; d < 3; ++d) {
            if (n3[d] == 1) continue;
            const int64_t p = shift(g, i, j, k, d, 1), m = shift(g, i, j, k, d, -1);
            const double a = speed_c ? c : 0.5 * (double)(umag3(u, N, q) + umag3(u, N, p));
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                const double *Ec = E + comp * N;
                const float r = ratio3(Ec[q] - Ec[m], Ec[p] - Ec[q]);
                kappa[(d * 3 + comp) * N + q] = (double)(1.0f - mc_limiter3(r, (float)beta)) * a * 0.5;
            }
        }
    }
}

// limited LF flux of B through the +d face of every cell (Eq. 17-18), each face
// once: F = dt/dx_d (1 - phi_B) a / 2 (B_{c+1} - B_c), a = |u| averaged over
// the face's 4 nodes (index c_d + 1 along d) or c.  Ff [3][3][N].
__global__ void k3_lf_flux(G3 g, const double *__restrict__ B, const double *__restrict__ u, double c, double dt,
                           double beta, int speed_c, double *Ff) {
    const int64_t N = g.N();
    const int n3[3] = {g.nx, g.ny, g.nz};
    const double dx3[3] = {g.dx, g.dy, g.dz};
    GRID_LOOP(q, N) {
        int i, j, k;
        g.ijk(q, i, j, k);
        for (int d = 0; d < 3; ++d) {
            if (n3[d] == 1) continue;
            const double f = dt / dx3[d];
            const int64_t cp = shift(g, i, j, k, d, 1), cm = shift(g, i, j, k, d, -1);
            double a;
            if (speed_c) {
                a = c;
            } else {
                float s = 0.f;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    int o[3];
                    o[d] = 1;
                    o[(d + 1) % 3] = t & 1;
                    o[(d + 2) % 3] = (t >> 1) & 1;
                    s += umag3(u, N, g.id(i + o[0], j + o[1], k + o[2]));
                }
                a = 0.25 * (double)s;
            }
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                const double *Bc = B + comp * N;
                const double dp = Bc[cp] - Bc[q];
                const float r = ratio3(Bc[q] - Bc[cm], dp);
                Ff[(d * 3 + comp) * N + q] = f * ((double)(1.0f - mc_limiter3(r, (float)beta)) * a * 0.5 * dp);
            }
        }
    }
}

// LF increment of B over one step, D = sum_d (F_{c+1/2} - F_{c-1/2}), and
// B~ = B^n + theta D, the part of B^{n+theta} the E solve curls
__global__ void k3_lf_b(G3 g, const double *__restrict__ B, const double *__restrict__ Ff, double theta, double *D,
                        double *Bt) {
    const int64_t N = g.N();
    const int n3[3] = {g.nx, g.ny, g.nz};
    GRID_LOOP(q, N) {
        int i, j, k;
        g.ijk(q, i, j, k);
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            double dn = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (n3[d] > 1) dn += Ff[(d * 3 + comp) * N + q] - Ff[(d * 3 + comp) * N + shift(g, i, j, k, d, -1)];
            D[comp * N + q] = dn;
            Bt[comp * N + q] = B[comp * N + q] + theta * dn;
        }
    }
}

// B^{n+1} = B^n - c dt curl_C E^{n+theta} (+ D), E^{n+1} = (E^{n+theta} - (1 - theta) E^n) / theta
__global__ void k3_advance(G3 g, H4 h, const double *__restrict__ E, const double *__restrict__ B,
                           const double *__restrict__ Eth, double c, double dt, double theta,
                           const double *__restrict__ D, double *Enew, double *Bnew) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        int i, j, k;
        g.ijk(q, i, j, k);
        const double *Ex = Eth, *Ey = Eth + N, *Ez = Eth + 2 * N;
        double cu[3];
        cu[0] = dC3(g, h, Ez, i, j, k, 1) - dC3(g, h, Ey, i, j, k, 2);
        cu[1] = dC3(g, h, Ex, i, j, k, 2) - dC3(g, h, Ez, i, j, k, 0);
        cu[2] = dC3(g, h, Ey, i, j, k, 0) - dC3(g, h, Ex, i, j, k, 1);
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            double bn = B[comp * N + q] - c * dt * cu[comp];
            if (D) bn += D[comp * N + q];
            Bnew[comp * N + q] = bn;
            Enew[comp * N + q] = (Eth[comp * N + q] - (1.0 - theta) * E[comp * N + q]) / theta;
        }
    }
}

// the 27 blocks of the operator at every node (see the file comment); LF: the
// diffusive term -theta dt / dx_d [kappa_+ (x_+ - x) - kappa_- (x - x_-)] per
// resolved axis and component.  A3f (or null): the same blocks rounded to FP32
// for the mixed-precision Krylov cycles.
__global__ void k3_assemble_A(G3 g, K3 K, double mfac, const double *__restrict__ M,
                              const double *__restrict__ kappa, double lfx, double lfy, double lfz, double *A3,
                              float *A3f) {
    const int64_t N = g.N();
    const int n3[3] = {g.nx, g.ny, g.nz};
    const double lf[3] = {lfx, lfy, lfz};
    GRID_LOOP(q, N) {
        int i, j, k;
        g.ijk(q, i, j, k);
        double kp[3][3], km[3][3];   // [axis][component]: kappa on the edges to q + e_d and from q - e_d
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const bool on = kappa && n3[d] > 1;
                kp[d][c] = on ? kappa[(d * 3 + c) * N + q] : 0.0;
                km[d][c] = on ? kappa[(d * 3 + c) * N + shift(g, i, j, k, d, -1)] : 0.0;
            }
        for (int o = 0; o < 27; ++o) {
            double blk[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) {
                blk[e] = K.k[o][e];
                if (M) blk[e] = fma(mfac, M[(size_t)(o * 9 + e) * N + q], blk[e]);
            }
            if (o == 13) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double s = 1.0;
#pragma unroll
                    for (int d = 0; d < 3; ++d) s += lf[d] * (kp[d][c] + km[d][c]);
                    blk[4 * c] += s;
                }
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int stride = d == 0 ? 1 : (d == 1 ? 3 : 9);
                if (o == 13 + stride)
#pragma unroll
                    for (int c = 0; c < 3; ++c) blk[4 * c] -= lf[d] * kp[d][c];
                if (o == 13 - stride)
#pragma unroll
                    for (int c = 0; c < 3; ++c) blk[4 * c] -= lf[d] * km[d][c];
            }
#pragma unroll
            for (int e = 0; e < 9; ++e) A3[(size_t)(o * 9 + e) * N + q] = blk[e];
            if (A3f)
#pragma unroll
                for (int e = 0; e < 9; ++e) A3f[(size_t)(o * 9 + e) * N + q] = (float)blk[e];
        }
    }
}

__global__ void k3_matvec(OpArgs a, const double *__restrict__ x, double *__restrict__ y) {
    const int64_t N = a.g3.N();
    GRID_LOOP(q, N) {
        double out[3];
        gx_apply_A3_node(a, x, q, out);
        y[q] = out[0];
        y[N + q] = out[1];
        y[2 * N + q] = out[2];
    }
}

// inverse of the centre block of the assembled operator (block-Jacobi
// preconditioner), FP64 and FP32
__global__ void k3_jacobi(int64_t N, const double *__restrict__ A3, double *jd, float *jd32) {
    GRID_LOOP(q, N) {
        double A[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) A[e] = A3[(size_t)(13 * 9 + e) * N + q];
        const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
        const double id = 1.0 / (A[0] * c00 + A[1] * c01 + A[2] * c02);
        double o[9];
        o[0] = c00 * id; o[1] = (A[2] * A[7] - A[1] * A[8]) * id; o[2] = (A[1] * A[5] - A[2] * A[4]) * id;
        o[3] = c01 * id; o[4] = (A[0] * A[8] - A[2] * A[6]) * id; o[5] = (A[2] * A[3] - A[0] * A[5]) * id;
        o[6] = c02 * id; o[7] = (A[1] * A[6] - A[0] * A[7]) * id; o[8] = (A[0] * A[4] - A[1] * A[3]) * id;
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            if (jd) jd[(size_t)q * 9 + e] = o[e];
            if (jd32) jd32[(size_t)q * 9 + e] = (float)o[e];
        }
    }
}

// field sums: |E|^2, |B|^2, rho, Gauss residual (div_C E - 4 pi rho averaged to
// the cell)^2 over cells, (div_N B)^2 over nodes
__global__ void k3_diag_grid(G3 g, H4 h, const double *__restrict__ E, const double *__restrict__ B,
                             const double *__restrict__ rho, double *acc) {
    const int64_t N = g.N();
    double we = 0, wb = 0, ch = 0, gl = 0, db = 0;
    GRID_LOOP(q, N) {
        int i, j, k;
        g.ijk(q, i, j, k);
        for (int c = 0; c < 3; ++c) {
            we += E[c * N + q] * E[c * N + q];
            wb += B[c * N + q] * B[c * N + q];
        }
        ch += rho ? rho[q] : 0.0;
        const double divE = dC3(g, h, E, i, j, k, 0) + dC3(g, h, E + N, i, j, k, 1) + dC3(g, h, E + 2 * N, i, j, k, 2);
        double rc = 0.0;
        if (rho) {
#pragma unroll
            for (int a = 0; a < 8; ++a) rc += rho[g.id(i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1))];
            rc *= 0.125;
        }
        const double gr = divE - 4.0 * GX_PI * rc;
        gl += gr * gr;
        const double divB = dN3(g, h, B, i, j, k, 0) + dN3(g, h, B + N, i, j, k, 1) + dN3(g, h, B + 2 * N, i, j, k, 2);
        db += divB * divB;
    }
    double v[5] = {we, wb, ch, gl, db};
    for (int c = 0; c < 5; ++c) {
        double s = v[c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(acc + c, s);
    }
}

// Gauss residual of cell (i,j,k) and its mean over the cells around a node (the
// Gauss's-law correction), as in 2D with 8 corners and 8 cells
__global__ void k3_gl_residual(G3 g, H4 h, const double *__restrict__ E, const double *__restrict__ rho, double *R) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        int i, j, k;
        g.ijk(q, i, j, k);
        const double divE = dC3(g, h, E, i, j, k, 0) + dC3(g, h, E + N, i, j, k, 1) + dC3(g, h, E + 2 * N, i, j, k, 2);
        double rb = 0.0;
#pragma unroll
        for (int a = 0; a < 8; ++a) rb += rho[g.id(i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1))];
        R[q] = divE * (0.25 / GX_PI) - 0.125 * rb;
    }
}
__global__ void k3_gl_phi(G3 g, const double *__restrict__ R, float4 *nE) {
    const int64_t N = g.N();
    GRID_LOOP(q, N) {
        int i, j, k;
        g.ijk(q, i, j, k);
        nE[q].w = (float)cell_mean(g, R, i, j, k);
    }
}

G3 geom3(const gx_ctx *c) {
    return G3{c->n[0], c->n[1], c->n[2], c->cfg.dx[0], c->cfg.dx[1], c->cfg.dx[2]};
}
H4 h4(const gx_ctx *c) {
    H4 h;
    for (int d = 0; d < 3; ++d) h.v[d] = 0.25 / c->cfg.dx[d];
    return h;
}
SpecK3 speck3(const gx_ctx *c) {
    SpecK3 sk{};
    sk.ns = c->nspecies;
    for (int s = 0; s < c->nspecies; ++s) {
        sk.q[s] = c->sp[s].q;
        sk.m[s] = c->sp[s].m;
        sk.bqf[s] = (float)(c->sp[s].q * c->cfg.dt / (2.0 * c->sp[s].m) * c->sp[s].q);
        sk.qf[s] = (float)c->sp[s].q;
    }
    return sk;
}

// (c theta dt)^2 curl_N curl_C as a 27-point block stencil: along axis d the
// weights of offset t in {-1, 0, 1} are s(t) = [1,2,1]/4 (average of averages),
// d2(t) = [1,-2,1] / dx^2 (difference of differences) and t / (2 dx) for a
// difference composed with an average
K3 curlcurl(const gx_ctx *c, double ct2) {
    K3 K{};
    const double *dx = c->cfg.dx;
    auto s = [](int t) { return t == 0 ? 0.5 : 0.25; };
    auto d2 = [](int t) { return t == 0 ? -2.0 : 1.0; };
    for (int o = 0; o < 27; ++o) {
        const int t[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double v = 0.0;
                if (i == j) {
                    for (int jj = 0; jj < 3; ++jj) {
                        if (jj == i) continue;
                        const int kk = 3 - i - jj;
                        v -= d2(t[jj]) / (dx[jj] * dx[jj]) * s(t[i]) * s(t[kk]);
                    }
                } else {
                    const int kk = 3 - i - j;
                    v = (double)(t[i] * t[j]) / (4.0 * dx[i] * dx[j]) * s(t[kk]);
                }
                K.k[o][3 * i + j] = ct2 * v;
            }
    }
    return K;
}

}  // namespace

int gx3_node_fields(gx_ctx *c, const double *Eth, const double *Bcur, float4 *outE, float4 *outB, cudaStream_t st) {
    k3_node_fields<<<blocks_for(c->N), kB, 0, st>>>(geom3(c), Eth, Bcur, outE, outB);
    GX_LAUNCHED(c);
    return GX_OK;
}

// all passes of the digital filter on a 3-component node field: per pass the
// sweeps along x, y and z (strides 1, 2, 1, ... when alternate), in FP64
int gx3_filter(gx_ctx *c, double *f, int passes, bool alternate, cudaStream_t st) {
    const G3 g = geom3(c);
    for (int p = 0; p < passes; ++p) {
        const int stride = (alternate && (p & 1)) ? 2 : 1;
        for (int axis = 0; axis < 3; ++axis) {
            if (c->n[axis] == 1) continue;      // a collapsed axis: the sweep is the identity
            k3_filter_sweep<<<blocks_for(c->N), kB, 0, st>>>(g, f, c->tmp3, axis, stride);
            GX_LAUNCHED(c);
            GX_CHECK(c, cudaMemcpyAsync(f, c->tmp3, 3 * c->N * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
    }
    return GX_OK;
}

int gx_copy_uref(gx_ctx *c, int zero, cudaStream_t st);

int gx3_assemble_moments(gx_ctx *c, cudaStream_t st) {
    const G3 g = geom3(c);
    const SpecK3 sk = speck3(c);
    const Recs3 R{c->rec, c->N};
    k3_assemble_bulk<<<blocks_for(c->N), kB, 0, st>>>(g, sk, R, 1.0 / c->dV, c->rho, c->rho_m, c->P, c->u);
    GX_LAUNCHED(c);
    int rc = gx3_filter(c, c->u, c->cfg.nsmooth_u, true, st);
    if (rc) return rc;
    k3_assemble_main<<<blocks_for(c->N), kB, 0, st>>>(g, sk, R, 1.0 / c->dV, c->cfg.comoving, c->u, c->uref64,
                                                       c->J, c->M);
    GX_LAUNCHED(c);
    rc = gx3_filter(c, c->J, c->cfg.ns_j, false, st);
    if (rc) return rc;
    rc = gx_copy_uref(c, c->cfg.comoving ? 0 : 1, st);
    if (rc) return rc;
    c->have_u = 1;
    return GX_OK;
}

int gx3_build_rhs(gx_ctx *c, cudaStream_t st) {
    const G3 g = geom3(c);
    const bool cm = c->cfg.comoving && c->nspecies > 0;
    if (cm) {
        k3_motional<<<blocks_for(c->N), kB, 0, st>>>(g, c->u, c->B, c->cfg.c, c->EM);
        GX_LAUNCHED(c);
    }
    const double ctd = c->cfg.c * c->cfg.theta * c->cfg.dt;
    const double jf = 4.0 * GX_PI * c->cfg.theta * c->cfg.dt;
    const double *Bc = c->B;
    if (c->cfg.lf_on) {
        double *D = c->dBlf, *Bt = c->dBlf + 3 * c->N, *Ff = c->dBlf + 6 * c->N;
        k3_lf_flux<<<blocks_for(c->N), kB, 0, st>>>(g, c->B, c->u, c->cfg.c, c->cfg.dt, c->cfg.lf_beta,
                                                    c->cfg.lf_speed_c, Ff);
        GX_LAUNCHED(c);
        k3_lf_b<<<blocks_for(c->N), kB, 0, st>>>(g, c->B, Ff, c->cfg.theta, D, Bt);
        GX_LAUNCHED(c);
        if (!c->cfg.lf_rhs_printed) Bc = Bt;   // the printed Eq. 7 curls B^n alone
    }
    k3_rhs<<<blocks_for(c->N), kB, 0, st>>>(g, h4(c), c->E, Bc, c->J, c->M, cm ? c->EM : nullptr, ctd, jf,
                                            jf / c->dV, c->rhs);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx3_build_kappa(gx_ctx *c, cudaStream_t st) {
    if (!c->cfg.lf_on || c->cfg.nsmooth_e > 0) return GX_OK;
    k3_kappa<<<blocks_for(c->N), kB, 0, st>>>(geom3(c), c->E, c->u, c->cfg.lf_beta, c->cfg.lf_speed_c, c->cfg.c,
                                               c->kappa);
    GX_LAUNCHED(c);
    return GX_OK;
}

// the operator's 27 blocks per node for this solve (M, kappa and the step's parameters)
int gx3_build_op(gx_ctx *c, cudaStream_t st) {
    const double ct = c->cfg.c * c->cfg.theta * c->cfg.dt;
    const double mfac = 4.0 * GX_PI * c->cfg.theta * c->cfg.dt / c->dV;
    const bool lfe = c->cfg.lf_on && c->cfg.nsmooth_e == 0;
    const double f = c->cfg.theta * c->cfg.dt;
    k3_assemble_A<<<blocks_for(c->N), kB, 0, st>>>(geom3(c), curlcurl(c, ct * ct), mfac,
                                                    c->nspecies > 0 ? c->M : nullptr, lfe ? c->kappa : nullptr,
                                                    f / c->cfg.dx[0], f / c->cfg.dx[1], f / c->cfg.dx[2], c->A3,
                                                    c->cfg.gmres_mixed ? c->A3f : nullptr);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx3_apply_A(gx_ctx *c, const double *x, double *y, cudaStream_t st) {
    k3_matvec<<<blocks_for(c->N), kB, 0, st>>>(gx_opargs(c), x, y);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx3_build_jacobi(gx_ctx *c, bool fp64, cudaStream_t st) {
    k3_jacobi<<<blocks_for(c->N), kB, 0, st>>>(c->N, c->A3, fp64 ? c->jdiag : nullptr, c->jdiag32);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx3_advance(gx_ctx *c, cudaStream_t st) {
    k3_advance<<<blocks_for(c->N), kB, 0, st>>>(geom3(c), h4(c), c->E, c->B, c->Eth, c->cfg.c, c->cfg.dt,
                                                c->cfg.theta, c->cfg.lf_on ? c->dBlf : nullptr, c->Enew, c->Bnew);
    GX_LAUNCHED(c);
    return gx3_filter(c, c->Enew, c->cfg.nsmooth_e, true, st);
}

int gx3_gl_potential(gx_ctx *c, cudaStream_t st) {
    k3_gl_residual<<<blocks_for(c->N), kB, 0, st>>>(geom3(c), h4(c), c->E, c->rho, c->tmp3);
    GX_LAUNCHED(c);
    k3_gl_phi<<<blocks_for(c->N), kB, 0, st>>>(geom3(c), c->tmp3, c->nE);
    GX_LAUNCHED(c);
    return GX_OK;
}

int gx3_diag_grid(gx_ctx *c, double *acc, cudaStream_t st) {
    k3_diag_grid<<<blocks_for(c->N), kB, 0, st>>>(geom3(c), h4(c), c->E, c->B, c->moments_valid ? c->rho : nullptr,
                                                  acc);
    GX_LAUNCHED(c);
    return GX_OK;
}
