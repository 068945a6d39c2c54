// gx_op.cuh -- the implicit field operator of the GL-ECSIM step (2D), shared
// by the grid kernels and the solver.
//
//   A x = x + (c theta dt)^2 curl_N curl_C x + (4 pi theta dt / dV) M x
//         - theta dt sum_d (1/dx_d) [kappa_+ (x_+ - x) - kappa_- (x - x_-)]
//
// (Eq. 7 with the mass term of Eq. 35 and the diffusive LF term of Eq. 19.)
// Mesh (Sec. 1.1): E at nodes, B at cell centres, periodic.  With the cell
// curl taken from face-averaged corner differences and the node curl from
// side-averaged cell differences, curl_N curl_C acts on the 3x3 node
// neighbourhood v[r][s] (row r along y, column s along x, centre (1,1)) as
//   (curl curl x)_x = hy^2 Dyy(x_x) + hx hy Dxy(x_y)
//   (curl curl x)_y = hx hy Dxy(x_x) + hx^2 Dxx(x_y)
//   (curl curl x)_z = hx^2 Dxx(x_z) + hy^2 Dyy(x_z)
// with hx = 1/(2 dx), hy = 1/(2 dy), Sx(r) = v[r][0] + 2 v[r][1] + v[r][2],
// Sy(s) = v[0][s] + 2 v[1][s] + v[2][s],
//   Dyy = 2 Sx(1) - Sx(0) - Sx(2),  Dxx = 2 Sy(1) - Sy(0) - Sy(2),
//   Dxy = v[0][0] - v[0][2] - v[2][0] + v[2][2]
// (the composition of the two averaged differences, expanded once).
#pragma once

#include "gx_internal.cuh"

// periodic index for small offsets (|off| < n): no integer division
__device__ __forceinline__ int gx_wr(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

struct G2 {
    int nx, ny;
    double dx, dy;
    double hx, hy;          // 1 / (2 dx), 1 / (2 dy): the averaged differences' factors
    int bc;                 // open x boundaries: cells per end held fixed (0: periodic)
    int wall;               // 1: the high-x boundary cells are a reflecting conductor
    __device__ __forceinline__ int64_t id(int i, int j) const {
        return (int64_t)gx_wr(i, nx) + (int64_t)nx * gx_wr(j, ny);
    }
    __device__ __forceinline__ int64_t N() const { return (int64_t)nx * ny; }
    // boundary cells: i < bc or i >= nx - bc; boundary nodes: both x-neighbouring cells are
    // boundary cells (i <= bc - 1 or i >= nx - bc + 1), and with the wall also its face node nx - bc
    __device__ __forceinline__ bool bcell(int i) const { return bc > 0 && (i < bc || i >= nx - bc); }
    __device__ __forceinline__ bool bnode(int i) const {
        return bc > 0 && (i <= bc - 1 || i >= nx - bc + (wall ? 0 : 1));
    }
};

// 3D geometry (all axes periodic; an axis of one cell collapses through the wrap)
struct G3 {
    int nx, ny, nz;
    double dx, dy, dz;
    __device__ __forceinline__ int64_t id(int i, int j, int k) const {
        return (int64_t)gx_wr(i, nx) + (int64_t)nx * ((int64_t)gx_wr(j, ny) + (int64_t)ny * gx_wr(k, nz));
    }
    __device__ __forceinline__ int64_t N() const { return (int64_t)nx * ny * nz; }
    // node coordinates (grids hold fewer than 2^31 nodes: 32-bit division)
    __device__ __forceinline__ void ijk(int64_t q, int &i, int &j, int &k) const {
        const unsigned u = (unsigned)q, r = u / (unsigned)nx;
        i = (int)(u - r * (unsigned)nx);
        k = (int)(r / (unsigned)ny);
        j = (int)(r - (unsigned)k * (unsigned)ny);
    }
};

struct OpArgs {
    G2 g;
    G3 g3;                 // 3D: the geometry, and
    const double *A3;      // the operator assembled as 27 node blocks [27 * 9][N] (or null in 2D)
    // FP32 copies for the mixed-precision Krylov cycles (null when not kept)
    const float *M32;      // 2D: M [81][N]
    const float *kappa32;  // 2D: kappa [2][3][N]
    const float *A3f;      // 3D: A3 [243][N]
    double ct2;            // (c theta dt)^2
    double mfac;           // 4 pi theta dt / dV
    double lfx, lfy;       // theta dt / dx, theta dt / dy
    const double *M;       // [81][N] or null
    const double *kappa;   // [2][3][N] or null
};

// operator arguments of a context (its current M, kappa and step parameters)
OpArgs gx_opargs(const gx_ctx *c);

// (A x) at node q, x component-major [3][N].  With CG the neighbourhood of x
// is read through L2 only (x was written by other CTAs of the same launch).  T
// = double is the operator; T = float the same operator from the FP32 copies of
// M and kappa (the mixed-precision Krylov cycles).
template <bool CG = false, typename T = double>
__device__ __forceinline__ void gx_apply_A_node(const OpArgs &a, const T *__restrict__ x, int64_t q, T out[3]) {
    constexpr bool F32 = sizeof(T) == 4;
    const G2 &g = a.g;
    const int64_t N = g.N();
    const int j = (int)((unsigned)q / (unsigned)g.nx), i = (int)q - j * g.nx;
    const int im = gx_wr(i - 1, g.nx), ip = gx_wr(i + 1, g.nx), jm = gx_wr(j - 1, g.ny), jp = gx_wr(j + 1, g.ny);
    const int xs[3] = {im, i, ip};
    const int64_t ys[3] = {(int64_t)jm * g.nx, (int64_t)j * g.nx, (int64_t)jp * g.nx};
    T v[3][3][3];   // [comp][row y][col x]
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int s = 0; s < 3; ++s) v[c][r][s] = CG ? __ldcg(x + c * N + ys[r] + xs[s]) : x[c * N + ys[r] + xs[s]];
    const T hx = (T)g.hx, hy = (T)g.hy;
    const T hxx = hx * hx, hyy = hy * hy, hxy = hx * hy;
    const T two = (T)2;
    auto Dyy = [&](int c) {
        const T s0 = v[c][0][0] + two * v[c][0][1] + v[c][0][2];
        const T s1 = v[c][1][0] + two * v[c][1][1] + v[c][1][2];
        const T s2 = v[c][2][0] + two * v[c][2][1] + v[c][2][2];
        return two * s1 - s0 - s2;
    };
    auto Dxx = [&](int c) {
        const T s0 = v[c][0][0] + two * v[c][1][0] + v[c][2][0];
        const T s1 = v[c][0][1] + two * v[c][1][1] + v[c][2][1];
        const T s2 = v[c][0][2] + two * v[c][1][2] + v[c][2][2];
        return two * s1 - s0 - s2;
    };
    auto Dxy = [&](int c) { return (v[c][0][0] - v[c][0][2]) - (v[c][2][0] - v[c][2][2]); };
    const T ct2 = (T)a.ct2;
    out[0] = v[0][1][1] + ct2 * (hyy * Dyy(0) + hxy * Dxy(1));
    out[1] = v[1][1][1] + ct2 * (hxy * Dxy(0) + hxx * Dxx(1));
    out[2] = v[2][1][1] + ct2 * (hxx * Dxx(2) + hyy * Dyy(2));
    const T *Mp = nullptr;
    if constexpr (F32) Mp = a.M ? a.M32 : nullptr;
    else Mp = a.M;
    if (Mp) {
        T m[3] = {0, 0, 0};
#pragma unroll
        for (int o = 0; o < 9; ++o) {
            const int ox = o % 3, oy = o / 3;
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int e = 0; e < 3; ++e) m[r] = fma(Mp[(size_t)(o * 9 + 3 * r + e) * N + q], v[e][oy][ox], m[r]);
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) out[r] = fma((T)a.mfac, m[r], out[r]);
    }
    const T *Kp = nullptr;
    if constexpr (F32) Kp = a.kappa ? a.kappa32 : nullptr;
    else Kp = a.kappa;
    if (Kp) {
        const int64_t xm = ys[1] + im, ym = ys[0] + i;
        const T lfx = (T)a.lfx, lfy = (T)a.lfy;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T *kx = Kp + (0 * 3 + c) * N, *ky = Kp + (1 * 3 + c) * N;
            if (g.nx > 1)
                out[c] -= lfx * (kx[q] * (v[c][1][2] - v[c][1][1]) - kx[xm] * (v[c][1][1] - v[c][1][0]));
            if (g.ny > 1)
                out[c] -= lfy * (ky[q] * (v[c][2][1] - v[c][1][1]) - ky[ym] * (v[c][1][1] - v[c][0][1]));
        }
    }
    if (g.bnode(i)) {   // Dirichlet row of an open boundary: E stays at its value
#pragma unroll
        for (int c = 0; c < 3; ++c) out[c] = v[c][1][1];
    }
}

// 3D: (A x) at node q from the assembled blocks, (A x)_r = sum_o sum_c
// A3[(o 9 + 3 r + c) N + q] x_c(q + o), o = (ox+1) + 3 (oy+1) + 9 (oz+1).
template <bool CG = false, typename T = double>
__device__ __forceinline__ void gx_apply_A3_node(const OpArgs &a, const T *__restrict__ x, int64_t q, T out[3]) {
    const G3 &g = a.g3;
    const int64_t N = g.N();
    int i, j, k;
    g.ijk(q, i, j, k);
    out[0] = out[1] = out[2] = 0;
    const T *A = nullptr;
    if constexpr (sizeof(T) == 4) A = a.A3f;
    else A = a.A3;
#pragma unroll 1
    for (int o = 0; o < 27; ++o) {
        const int64_t nb = g.id(i + o % 3 - 1, j + (o / 3) % 3 - 1, k + o / 9 - 1);
        T xv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) xv[c] = CG ? __ldcg(x + c * N + nb) : x[c * N + nb];
        const T *blk = A + (size_t)o * 9 * N + q;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) out[r] = fma(blk[(size_t)(3 * r + c) * N], xv[c], out[r]);
    }
}

// the operator of a DIM-dimensional grid at node q (T = float: from the FP32 copies)
template <int DIM, bool CG = false, typename T = double>
__device__ __forceinline__ void gx_apply_node(const OpArgs &a, const T *__restrict__ x, int64_t q, T out[3]) {
    if constexpr (DIM == 3) gx_apply_A3_node<CG, T>(a, x, q, out);
    else gx_apply_A_node<CG, T>(a, x, q, out);
}
