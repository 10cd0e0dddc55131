// lbm_internal.cuh -- device-side tables, storage traits and launch structs
// shared by the CUDA translation units of the solver (bulk.cu, boundary.cu,
// api.cu).  Nothing here is visible through the C ABI.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace lbmgb {

// ---------------------------------------------------------------------------
// Velocity sets (Appendix B).  The GPU orders each set as the rest velocity
// followed by opposite pairs (i, i+1) with c_{i+1} = -c_i, so the equilibrium
// can be evaluated once per pair (even and odd parts in c.u).
// ---------------------------------------------------------------------------

enum { D2Q9 = 0, D2Q37 = 1 };

template <int LAT>
struct Lat;

// D2Q9, Tab. d2q9: c_s^2 = 1/3, M = 1; isothermal second-order equilibrium.
template <>
struct Lat<D2Q9> {
    static constexpr int Q = 9, M = 1, NCLS = 3;
    static constexpr bool THERMAL = false;
    static constexpr double CS2 = 1.0 / 3.0;
    __host__ __device__ static constexpr int cx(int i)
    {
        constexpr int v[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
        return v[i];
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        constexpr int v[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
        return v[i];
    }
    // symmetry class of velocity i; |c|^2 of each class
    __host__ __device__ static constexpr int cls(int i) { return i == 0 ? 0 : (i < 5 ? 1 : 2); }
    __host__ __device__ static constexpr int c2cls(int k)
    {
        constexpr int v[3] = {0, 1, 2};
        return v[k];
    }
    __host__ __device__ static constexpr double wcls(int k)
    {
        constexpr double v[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
        return v[k];
    }
    __host__ __device__ static constexpr double w(int i) { return wcls(cls(i)); }
};

// D2Q37, Tab. d2q37 velocity classes (0,0) (1,0) (1,1) (2,0) (2,1) (2,2) (3,0)
// (3,1); M = 3.  c_s^2 and the class weights solve the Gauss-Hermite
// isotropy conditions through eighth order (the weights agree with the
// printed 14-decimal values; the printed c_s formula does not).
template <>
struct Lat<D2Q37> {
    static constexpr int Q = 37, M = 3, NCLS = 8;
    static constexpr bool THERMAL = true;
    static constexpr double CS2 = 0.6979533220196830882384091;
    __host__ __device__ static constexpr int cx(int i)
    {
        constexpr int v[37] = {0,
                               1, -1, 0, 0,                              // (1,0)
                               1, -1, 1, -1,                             // (1,1)
                               2, -2, 0, 0,                              // (2,0)
                               2, -2, 2, -2, 1, -1, 1, -1,               // (2,1)
                               2, -2, 2, -2,                             // (2,2)
                               3, -3, 0, 0,                              // (3,0)
                               3, -3, 3, -3, 1, -1, 1, -1};              // (3,1)
        return v[i];
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        constexpr int v[37] = {0,
                               0, 0, 1, -1,
                               1, -1, -1, 1,
                               0, 0, 2, -2,
                               1, -1, -1, 1, 2, -2, -2, 2,
                               2, -2, -2, 2,
                               0, 0, 3, -3,
                               1, -1, -1, 1, 3, -3, -3, 3};
        return v[i];
    }
    __host__ __device__ static constexpr int cls(int i)
    {
        return i == 0 ? 0 : i < 5 ? 1 : i < 9 ? 2 : i < 13 ? 3 : i < 21 ? 4 : i < 25 ? 5 : i < 29 ? 6 : 7;
    }
    __host__ __device__ static constexpr int c2cls(int k)
    {
        constexpr int v[8] = {0, 1, 2, 4, 5, 8, 9, 10};
        return v[k];
    }
    __host__ __device__ static constexpr double wcls(int k)
    {
        constexpr double v[8] = {0.23315066913235250229, 0.10730609154221900241,
                                 0.05766785988879488203, 0.014208216158450750265,
                                 0.0053530490005137752327, 0.0010119375926735754754,
                                 0.00024530102775771734547, 0.0002834142529941982174};
        return v[k];
    }
    __host__ __device__ static constexpr double w(int i) { return wcls(cls(i)); }
};

// ---------------------------------------------------------------------------
// Storage traits.  Populations are stored shifted, g = f - w rho0.  F16 keeps
// g / w so that every velocity uses the same half-precision range.
// ---------------------------------------------------------------------------

template <typename S>
struct Store;

template <>
struct Store<double> {
    using C = double;                       // arithmetic type of the bulk kernel
    static constexpr bool SCALED = false;
    __device__ static double load(const double* p) { return __ldg(p); }
    __device__ static void put(double* p, double v) { *p = v; }
};

template <>
struct Store<float> {
    using C = float;
    static constexpr bool SCALED = false;
    __device__ static float load(const float* p) { return __ldg(p); }
    __device__ static void put(float* p, float v) { *p = v; }
};

template <>
struct Store<__half> {
    using C = float;
    static constexpr bool SCALED = true;
    __device__ static float load(const __half* p) { return __half2float(__ldg(p)); }
    __device__ static void put(__half* p, float v) { *p = __float2half_rn(v); }
};

// ---------------------------------------------------------------------------
// Equilibrium and moments (shared by the bulk and boundary kernels)
// ---------------------------------------------------------------------------

// Coefficients of the shifted Hermite equilibrium as a polynomial in
// p = c.u / c_s^2 for one velocity class with xi^2 = |c|^2 / c_s^2:
//   f^eq / (w rho) - 1 = a0 + a1 p + a2 p^2 + a3 p^3 + a4 p^4.
// Thermal (Eq. feq-4, fourth-order Hermite in xi = c/c_s, u~ = u/c_s,
// theta - 1 = dT, with the (xi^2 - 6) coefficient of the (u.c)^2 (T-1)
// term): a3 = 1/6, a4 = 1/24.  Isothermal D2Q9: second order.
template <int LAT, typename C>
__device__ __forceinline__ void eq_coef(C u2, C dT, C* a0, C* a1, C* a2)
{
    using L = Lat<LAT>;
    constexpr C ics2 = C(1.0 / L::CS2);
#pragma unroll
    for (int k = 0; k < L::NCLS; ++k) {
        const C xi2 = C(L::c2cls(k)) * ics2;
        if (L::THERMAL) {
            a0[k] = C(0.5) * (dT * (xi2 - C(2)) - u2) +
                    C(1.0 / 24.0) * (C(3) * u2 * u2 + C(6) * dT * u2 * (C(4) - xi2) +
                                     C(3) * dT * dT * (xi2 * xi2 - C(8) * xi2 + C(8)));
            a1[k] = C(1) - C(0.5) * u2 + C(0.5) * dT * (xi2 - C(4));
            a2[k] = C(0.5) - C(0.25) * u2 + C(0.25) * dT * (xi2 - C(6));
        } else {
            a0[k] = C(-0.5) * u2;
            a1[k] = C(1);
            a2[k] = C(0.5);
        }
    }
}

template <int LAT, typename C>
struct Moments {
    C s0, ux, uy, dT, rho;
};

// Eq. macro on shifted populations (sum_i w_i c_i = 0, sum_i w_i |c_i|^2 =
// 2 c_s^2): rho = rho0 + sum g, rho u = sum g c, and
// theta - 1 = (sum g |c|^2 - rho |u|^2 - 2 c_s^2 (rho - rho0)) / (2 rho c_s^2).
template <int LAT, typename C>
__device__ __forceinline__ Moments<LAT, C> moments(const C* g, C rho0)
{
    using L = Lat<LAT>;
    C s0 = 0, sx = 0, sy = 0, se = 0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        s0 += g[i];
        if (L::cx(i)) sx += C(L::cx(i)) * g[i];
        if (L::cy(i)) sy += C(L::cy(i)) * g[i];
        if (L::THERMAL && i) se += C(L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i)) * g[i];
    }
    Moments<LAT, C> m;
    m.s0 = s0;
    m.rho = rho0 + s0;
    const C irho = C(1) / m.rho;
    m.ux = sx * irho;
    m.uy = sy * irho;
    m.dT = C(0);
    if (L::THERMAL)
        m.dT = (se - m.rho * (m.ux * m.ux + m.uy * m.uy) - C(2.0 * L::CS2) * s0) * irho *
               C(0.5 / L::CS2);
    return m;
}

// Shifted equilibrium of all velocities (g^eq = f^eq - w rho0).
template <int LAT, typename C>
__device__ __forceinline__ void equilibrium(const Moments<LAT, C>& m, C* geq)
{
    using L = Lat<LAT>;
    constexpr C ics2 = C(1.0 / L::CS2);
    constexpr C a3 = L::THERMAL ? C(1.0 / 6.0) : C(0);
    constexpr C a4 = L::THERMAL ? C(1.0 / 24.0) : C(0);
    C a0[L::NCLS], a1[L::NCLS], a2[L::NCLS];
    eq_coef<LAT, C>((m.ux * m.ux + m.uy * m.uy) * ics2, m.dT, a0, a1, a2);
    geq[0] = C(L::w(0)) * (m.s0 + m.rho * a0[0]);
#pragma unroll
    for (int i = 1; i < L::Q; i += 2) {
        const int k = L::cls(i);
        const C p = (C(L::cx(i)) * m.ux + C(L::cy(i)) * m.uy) * ics2;
        const C p2 = p * p;
        const C ev = a0[k] + p2 * (a2[k] + p2 * a4);
        const C od = p * (a1[k] + p2 * a3);
        geq[i] = C(L::w(i)) * (m.s0 + m.rho * (ev + od));
        geq[i + 1] = C(L::w(i)) * (m.s0 + m.rho * (ev - od));
    }
}

// ---------------------------------------------------------------------------
// Launch structs
// ---------------------------------------------------------------------------

enum { SIDE_PERIODIC = 0, SIDE_CBC = 1, SIDE_INFLOW = 2, SIDE_ZG = 3 };
enum { SCH_LODI = 0, SCH_LODI_RELAX = 1, SCH_CBC = 2, SCH_CBC_RELAX = 3 };
enum { VIS_MESO = 0, VIS_FD = 1, VIS_OFF = 2 };

// Grid geometry.  Populations are SoA planes f[i][y][x] with row pitch nxp.
struct Geom {
    int nx, ny, nxp, M;
    int perx, pery;
    int bx0, bx1, by0, by1;     // bulk nodes: [bx0, bx1) x [by0, by1)
    long long plane;            // ny * nxp
    double tau, rho0;
};

// One side of the grid (W = 0, E = 1, S = 2, N = 3).
struct Side {
    int kind, scheme;
    int L;                      // nodes along the side (ny for W/E, nx for S/N)
    int lo, hi;                 // tangential range of the side's own layers
    int tper;                   // tangential axis periodic
    int base;                   // first characteristic unknown of the side
    long long offU, offN;       // offsets of the side's strips (doubles)
    int ebase;                  // first node of the side in the extras list
};

// Characteristic boundary state and the near-boundary strips the bulk kernel
// exports: macros U (4 doubles) and non-equilibrium moments N = sigma'_xx,
// sigma'_xy, sigma'_yy, q_x, q_y (5 doubles) at depths d = 0, 1, 2 inside
// the boundary layers, for two time levels (parity of the step).
struct Band {
    Side s[4];
    int any_cbc;
    int n_side_unk, n_unk;      // unknowns of the boundary ODE (sides + corners)
    int corner_kind;            // kind of the four M x M corner blocks (or -1)
    int n_extra;                // zero-gradient / inflow nodes (sides, then corners)
    int n_extra_side;           // of which on the sides
    int viscous, dirichlet;
    double alpha_T, beta_P, t_inf;
    double pdev[4];             // P_inf - c_s^2 rho0 per side
    double Uin[4];              // inflow state (drho, ux, uy, dT)
    double *Ub, *Ya, *Yb, *acc, *V;
    int* mask;
    double *stripU, *stripN;
};

// Row-major index of the strip entries.
__host__ __device__ inline long long strip_u_index(const Side& S, int par, int d, int p)
{
    return S.offU + ((long long)(par * 3 + d) * S.L + p) * 4;
}
__host__ __device__ inline long long strip_n_index(const Side& S, int par, int d, int p)
{
    return S.offN + ((long long)(par * 3 + d) * S.L + p) * 5;
}

// Outward normal and tangent of each side, and the outward diagonal of each
// corner block (SW = 0, SE = 1, NW = 2, NE = 3).
__host__ __device__ inline int side_nx(int s) { return s == 0 ? -1 : (s == 1 ? 1 : 0); }
__host__ __device__ inline int side_ny(int s) { return s == 2 ? -1 : (s == 3 ? 1 : 0); }
__host__ __device__ inline int side_tx(int s) { return s < 2 ? 0 : 1; }
__host__ __device__ inline int side_ty(int s) { return s < 2 ? 1 : 0; }
__host__ __device__ inline int corner_sx(int c) { return (c & 1) ? 1 : -1; }
__host__ __device__ inline int corner_sy(int c) { return (c & 2) ? 1 : -1; }

// Node x_f (layer 0) of side s at tangential position p.
__host__ __device__ inline void side_xf(int s, int p, int nx, int ny, int M, int& x, int& y)
{
    if (s == 0) { x = M; y = p; }
    else if (s == 1) { x = nx - 1 - M; y = p; }
    else if (s == 2) { x = p; y = M; }
    else { x = p; y = ny - 1 - M; }
}

// ---------------------------------------------------------------------------
// Host-side launchers (defined in bulk.cu / boundary.cu)
// ---------------------------------------------------------------------------

int launch_init(int lat, int storage, const Geom& G, const Band& B, const double* rho,
                const double* ux, const double* uy, const double* T, void* f, cudaStream_t st);
int launch_bulk(int lat, int storage, const Geom& G, const Band& B, const void* fin, void* fout,
                int par_new, cudaStream_t st);
int launch_macros(int lat, int storage, const Geom& G, const void* f, double* rho, double* ux,
                  double* uy, double* T, int* flag, cudaStream_t st);
int launch_boundary(int lat, int storage, const Geom& G, const Band& B, void* fnew, int par_t,
                    cudaStream_t st);

}  // namespace lbmgb
