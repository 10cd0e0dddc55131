// lbm_internal.cuh -- device-side tables, storage traits and launch structs
// shared by the CUDA translation units of the solver (bulk.cu, boundary.cu,
// api.cu).  Nothing here is visible through the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace lbmgb {

// ---------------------------------------------------------------------------
// Velocity sets (Appendix B).  The GPU orders each set as the rest velocity
// followed by opposite pairs (i, i+1) with c_{i+1} = -c_i, so the equilibrium
// can be evaluated once per pair (even and odd parts in c.u).
// ---------------------------------------------------------------------------

enum { D2Q9 = 0, D2Q37 = 1, D2Q17 = 2 };

template <int LAT>
struct Lat;

// D2Q9, Tab. d2q9: c_s^2 = 1/3, M = 1; isothermal second-order equilibrium.
template <>
struct Lat<D2Q9> {
    static constexpr int Q = 9, M = 1, NCLS = 3;
    static constexpr bool THERMAL = false;
    static constexpr int ORDER = 2;         // Hermite order of the equilibrium
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
    // Population planes are stored grouped by c_y (groups c_y = 0, 1, -1)
    // so that one tensor copy fetches every population with a common source row.
    static constexpr int NG = 3;
    __host__ __device__ static constexpr int plane_of(int i)
    {
        constexpr int v[9] = {0, 1, 2, 3, 6, 4, 7, 8, 5};
        return v[i];
    }
    __host__ __device__ static constexpr int gcy(int g)
    {
        constexpr int v[3] = {0, 1, -1};
        return v[g];
    }
    __host__ __device__ static constexpr int gstart(int g)
    {
        constexpr int v[3] = {0, 3, 6};
        return v[g];
    }
    __host__ __device__ static constexpr int gcount(int g)
    {
        constexpr int v[3] = {3, 3, 3};
        return v[g];
    }
};

// D2Q37, Tab. d2q37 velocity classes (0,0) (1,0) (1,1) (2,0) (2,1) (2,2) (3,0)
// (3,1); M = 3.  c_s^2 and the class weights solve the Gauss-Hermite
// isotropy conditions through eighth order (the weights agree with the
// printed 14-decimal values; the printed c_s formula does not).
template <>
struct Lat<D2Q37> {
    static constexpr int Q = 37, M = 3, NCLS = 8;
    static constexpr bool THERMAL = true;
    static constexpr int ORDER = 4;
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
    // planes grouped by c_y = 0, 1, -1, 2, -2, 3, -3
    static constexpr int NG = 7;
    __host__ __device__ static constexpr int plane_of(int i)
    {
        constexpr int v[37] = {0,  1,  2,  7,  14, 8,  15, 16, 9,  3,  4,  21, 26,
                               10, 17, 18, 11, 22, 27, 28, 23, 24, 29, 30, 25, 5,
                               6,  31, 34, 12, 19, 20, 13, 32, 35, 36, 33};
        return v[i];
    }
    __host__ __device__ static constexpr int gcy(int g)
    {
        constexpr int v[7] = {0, 1, -1, 2, -2, 3, -3};
        return v[g];
    }
    __host__ __device__ static constexpr int gstart(int g)
    {
        constexpr int v[7] = {0, 7, 14, 21, 26, 31, 34};
        return v[g];
    }
    __host__ __device__ static constexpr int gcount(int g)
    {
        constexpr int v[7] = {7, 7, 7, 5, 5, 3, 3};
        return v[g];
    }
};

// D2Q17, Tab. d2q17 velocity classes (0,0) (1,0) (1,1) (2,2) (3,0); M = 3;
// third-order equilibrium (Eq. feq-3).  The class weights are the printed
// closed forms (a + b sqrt 193) / d; c_s^2 = 72 / (5 (25 + sqrt 193)), which
// is sum_i w_i c_ix^2 of those weights (the printed c_s formula gives its
// reciprocal).
template <>
struct Lat<D2Q17> {
    static constexpr int Q = 17, M = 3, NCLS = 5;
    static constexpr bool THERMAL = true;
    static constexpr int ORDER = 3;
    static constexpr double CS2 = 0.3702518670183398497189151;
    __host__ __device__ static constexpr int cx(int i)
    {
        constexpr int v[17] = {0, 1, -1, 0, 0, 1, -1, 1, -1, 2, -2, 2, -2, 3, -3, 0, 0};
        return v[i];
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        constexpr int v[17] = {0, 0, 0, 1, -1, 1, -1, -1, 1, 2, -2, -2, 2, 0, 0, 3, -3};
        return v[i];
    }
    __host__ __device__ static constexpr int cls(int i)
    {
        return i == 0 ? 0 : i < 5 ? 1 : i < 9 ? 2 : i < 13 ? 3 : 4;
    }
    __host__ __device__ static constexpr int c2cls(int k)
    {
        constexpr int v[5] = {0, 1, 2, 8, 9};
        return v[k];
    }
    __host__ __device__ static constexpr double wcls(int k)
    {
        constexpr double v[5] = {0.4020051469091126259416644, 0.1161548664977815438740355,
                                 0.0330063536229869139497538, 0.0000790786021659181312371,
                                 0.0002584145497874675595575};
        return v[k];
    }
    __host__ __device__ static constexpr double w(int i) { return wcls(cls(i)); }
    // planes grouped by c_y = 0, 1, -1, 2, -2, 3, -3
    static constexpr int NG = 7;
    __host__ __device__ static constexpr int plane_of(int i)
    {
        constexpr int v[17] = {0, 1, 2, 5, 8, 6, 9, 10, 7, 11, 13, 14, 12, 3, 4, 15, 16};
        return v[i];
    }
    __host__ __device__ static constexpr int gcy(int g)
    {
        constexpr int v[7] = {0, 1, -1, 2, -2, 3, -3};
        return v[g];
    }
    __host__ __device__ static constexpr int gstart(int g)
    {
        constexpr int v[7] = {0, 5, 8, 11, 13, 15, 16};
        return v[g];
    }
    __host__ __device__ static constexpr int gcount(int g)
    {
        constexpr int v[7] = {5, 3, 3, 2, 2, 1, 1};
        return v[g];
    }
};

// Group of velocity i (its plane lies in [gstart, gstart + gcount)).
template <int LAT>
__host__ __device__ constexpr int group_of(int i)
{
    int g = 0;
    while (!(Lat<LAT>::plane_of(i) >= Lat<LAT>::gstart(g) &&
             Lat<LAT>::plane_of(i) < Lat<LAT>::gstart(g) + Lat<LAT>::gcount(g)))
        ++g;
    return g;
}

// ---------------------------------------------------------------------------
// Storage traits.  Populations are stored shifted, g = f - w rho0.  F16 keeps
// g / w so that every velocity uses the same half-precision range.
// ---------------------------------------------------------------------------

// load(): read-only GLOBAL memory only (the non-coherent load path rejects
// any other address space); value(): the arithmetic value of a stored
// element already read (e.g. from shared memory); put(): any address space.
template <typename S>
struct Store;

template <>
struct Store<double> {
    using C = double;                       // arithmetic type of the bulk kernel
    static constexpr bool SCALED = false;
    __device__ static double load(const double* p) { return __ldg(p); }
    __device__ static double value(double v) { return v; }
    __device__ static void put(double* p, double v) { *p = v; }
};

template <>
struct Store<float> {
    using C = float;
    static constexpr bool SCALED = false;
    __device__ static float load(const float* p) { return __ldg(p); }
    __device__ static float value(float v) { return v; }
    __device__ static void put(float* p, float v) { *p = v; }
};

template <>
struct Store<__half> {
    using C = float;
    static constexpr bool SCALED = true;
    __device__ static float load(const __half* p) { return __half2float(__ldg(p)); }
    __device__ static float value(__half v) { return __half2float(v); }
    __device__ static void put(__half* p, float v) { *p = __float2half_rn(v); }
};

// ---------------------------------------------------------------------------
// Equilibrium and moments (shared by the bulk and boundary kernels)
// ---------------------------------------------------------------------------

// Coefficients of the shifted Hermite equilibrium as a polynomial in
// p = c.u / c_s^2 for a velocity class with xi^2 = |c|^2 / c_s^2:
//   f^eq / (w rho) - 1 = a0 + a1 p + a2 p^2 + a3 p^3 + a4 p^4,
// and each a_k as a polynomial in xi^2:
//   a0 = A0 + xi^2 (B0 + C0 xi^2),  a1 = A1 + B1 xi^2,  a2 = A2 + B2 xi^2.
// D2Q37: Eq. feq-4, the fourth-order Hermite expansion in xi = c/c_s,
// u~ = u/c_s, theta - 1 = t, read with the coefficient (xi^2 - 6) in the
// (u.c)^2 (T-1) term; then a3 = 1/6, a4 = 1/24.
// D2Q17: Eq. feq-3, the third-order expansion in the same variables;
// a3 = 1/6, a4 = 0.
// Isothermal D2Q9: second order, a0 = -u2/2, a1 = 1, a2 = 1/2.
template <typename C>
struct EqPoly {
    C A0, B0, C0, A1, B1, A2, B2;
};

template <int LAT, typename C>
__device__ __forceinline__ EqPoly<C> eq_poly(C u2, C t)
{
    EqPoly<C> e;
    if (Lat<LAT>::ORDER == 3) {
        // Eq. feq-3: even part -u2/2 - t + (t/2) xi^2 + p^2/2, odd part
        // p (1 - u2/2 - 2t + (t/2) xi^2) + p^3/6
        e.A0 = C(-0.5) * u2 - t;
        e.B0 = C(0.5) * t;
        e.C0 = C(0);
        e.A1 = C(1) - C(0.5) * u2 - C(2) * t;
        e.B1 = C(0.5) * t;
        e.A2 = C(0.5);
        e.B2 = C(0);
    } else if (Lat<LAT>::THERMAL) {
        e.A0 = C(-0.5) * u2 - t + C(0.125) * u2 * u2 + t * u2 + t * t;
        e.B0 = C(0.5) * t - C(0.25) * t * u2 - t * t;
        e.C0 = C(0.125) * t * t;
        e.A1 = C(1) - C(0.5) * u2 - C(2) * t;
        e.B1 = C(0.5) * t;
        e.A2 = C(0.5) - C(0.25) * u2 - C(1.5) * t;
        e.B2 = C(0.25) * t;
    } else {
        e.A0 = C(-0.5) * u2;
        e.B0 = e.C0 = e.B1 = e.B2 = C(0);
        e.A1 = C(1);
        e.A2 = C(0.5);
    }
    return e;
}

// Populations stored relative to a reference equilibrium f^eq(rho0, U, T0)
// (the mean flow; "ref"): the equilibrium of a node is then needed as the
// difference f^eq(rho, u, theta) - f^eq(rho0, U, 0), formed without
// cancellation from the deviations s = rho - rho0, v = u - U, theta.  Its
// coefficient differences dA_k = A_k(u2, t) - A_k(U2, 0) in d = u2 - U2 =
// (2 U.v + |v|^2) / c_s^2 (the B and C coefficients vanish at t = 0, so
// theirs are the values themselves), and the reference values A1r, A2r.
template <typename C>
struct EqDelta {
    C A0, A1, A2, A1r, A2r;
};

template <int LAT, typename C>
__device__ __forceinline__ EqDelta<C> eq_delta(C U2, C d, C t)
{
    EqDelta<C> e;
    if (Lat<LAT>::ORDER == 3) {
        e.A0 = C(-0.5) * d - t;
        e.A1 = C(-0.5) * d - C(2) * t;
        e.A2 = C(0);
        e.A1r = C(1) - C(0.5) * U2;
        e.A2r = C(0.5);
    } else if (Lat<LAT>::THERMAL) {
        e.A0 = C(-0.5) * d - t + C(0.125) * (C(2) * U2 + d) * d + t * (U2 + d) + t * t;
        e.A1 = C(-0.5) * d - C(2) * t;
        e.A2 = C(-0.25) * d - C(1.5) * t;
        e.A1r = C(1) - C(0.5) * U2;
        e.A2r = C(0.5) - C(0.25) * U2;
    } else {
        e.A0 = C(-0.5) * d;
        e.A1 = C(0);
        e.A2 = C(0);
        e.A1r = C(1);
        e.A2r = C(0.5);
    }
    return e;
}

// One opposite pair (+c, -c) of velocity class xi2 relative to the
// reference: g^eq_(+-) / w = Ev +- Od with
//   Ev = s (1 + ev) + rho0 dE,  Od = s od + rho0 dO,
// ev, od the even and odd parts at (u, theta) (as eq_poly's pair loop), and
// dE, dO their differences from the reference's, in q = c.v / c_s^2 and
// P = c.U / c_s^2 (p = P + q):
//   dE = da0 + da2 p^2 + a2r (p^2 - P^2) + a4 (p^2 - P^2)(p^2 + P^2)
//   dO = da1 p + a1r q + a3 q (p^2 + p P + P^2),  p^2 - P^2 = q (p + P).
template <int LAT, typename C>
__device__ __forceinline__ void eq_pair_ref(const EqPoly<C>& e, const EqDelta<C>& de, C xi2, C P, C q, C s,
                                            C rho0, C& Ev, C& Od)
{
    constexpr C a3 = Lat<LAT>::ORDER >= 3 ? C(1.0 / 6.0) : C(0);
    constexpr C a4 = Lat<LAT>::ORDER >= 4 ? C(1.0 / 24.0) : C(0);
    const C bc = e.B0 + e.C0 * xi2;
    const C a0 = e.A0 + xi2 * bc, a1 = e.A1 + e.B1 * xi2, a2 = e.A2 + e.B2 * xi2;
    const C da0 = de.A0 + xi2 * bc, da1 = de.A1 + e.B1 * xi2, da2 = de.A2 + e.B2 * xi2;
    const C p = P + q, p2 = p * p, P2 = P * P, dp2 = q * (p + P);
    const C ev = a0 + p2 * (a2 + p2 * a4);
    const C od = p * (a1 + p2 * a3);
    const C dE = da0 + da2 * p2 + de.A2r * dp2 + a4 * dp2 * (p2 + P2);
    const C dO = da1 * p + de.A1r * q + a3 * q * (p2 + p * P + P2);
    Ev = s * (C(1) + ev) + rho0 * dE;
    Od = s * od + rho0 * dO;
}

template <int LAT, typename C>
__device__ __forceinline__ void eq_coef(C u2, C dT, C* a0, C* a1, C* a2)
{
    using L = Lat<LAT>;
    constexpr C ics2 = C(1.0 / L::CS2);
    const EqPoly<C> e = eq_poly<LAT, C>(u2, dT);
#pragma unroll
    for (int k = 0; k < L::NCLS; ++k) {
        const C xi2 = C(L::c2cls(k)) * ics2;
        a0[k] = e.A0 + xi2 * (e.B0 + e.C0 * xi2);
        a1[k] = e.A1 + e.B1 * xi2;
        a2[k] = e.A2 + e.B2 * xi2;
    }
}

template <int LAT, typename C>
struct Moments {
    C s0, ux, uy, dT, rho;
    C sx, sy, se;   // sum g c_x, sum g c_y, sum g |c|^2
    // ref: populations held relative to f^eq(rho0, U, T0); U and v = u - U
    int ref = 0;
    C Ux = C(0), Uy = C(0), vx = C(0), vy = C(0);
};

// Eq. macro on shifted populations (sum_i w_i c_i = 0, sum_i w_i |c_i|^2 =
// 2 c_s^2): rho = rho0 + sum g, rho u = sum g c, and
// theta - 1 = (sum g |c|^2 - rho |u|^2 - 2 c_s^2 (rho - rho0)) / (2 rho c_s^2).
// The same from the sums s0 = sum g, (sx, sy) = sum g c, se = sum g |c|^2.
// With a reference (ref, U = (Ux, Uy)) the sums are of g = f - f^eq(rho0,
// U, 0): rho u = sum g c + rho0 U and sum f |c|^2 = sum g |c|^2 + rho0 (|U|^2
// + 2 c_s^2), formed as v = (sum g c - s U) / rho and
// theta = (sum g |c|^2 - 2 c_s^2 s - s |U|^2 - 2 rho U.v - rho |v|^2) / (2 rho c_s^2).
template <int LAT, typename C>
__device__ __forceinline__ Moments<LAT, C> moments_of_sums(C s0, C sx, C sy, C se, C rho0, int ref = 0,
                                                           C Ux = C(0), C Uy = C(0))
{
    using L = Lat<LAT>;
    Moments<LAT, C> m;
    m.s0 = s0;
    m.sx = sx;
    m.sy = sy;
    m.se = se;
    m.rho = rho0 + s0;
    const C irho = C(1) / m.rho;
    m.dT = C(0);
    if (!ref) {
        m.ux = sx * irho;
        m.uy = sy * irho;
        m.vx = m.ux;
        m.vy = m.uy;
        if (L::THERMAL)
            m.dT = (se - m.rho * (m.ux * m.ux + m.uy * m.uy) - C(2.0 * L::CS2) * s0) * irho *
                   C(0.5 / L::CS2);
        return m;
    }
    m.ref = 1;
    m.Ux = Ux;
    m.Uy = Uy;
    m.vx = (sx - s0 * Ux) * irho;
    m.vy = (sy - s0 * Uy) * irho;
    m.ux = Ux + m.vx;
    m.uy = Uy + m.vy;
    if (L::THERMAL)
        m.dT = (se - C(2.0 * L::CS2) * s0 - s0 * (Ux * Ux + Uy * Uy) -
                m.rho * (C(2) * (Ux * m.vx + Uy * m.vy) + m.vx * m.vx + m.vy * m.vy)) *
               irho * C(0.5 / L::CS2);
    return m;
}

template <int LAT, typename C>
__device__ __forceinline__ Moments<LAT, C> moments(const C* g, C rho0, int ref = 0, C Ux = C(0), C Uy = C(0))
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
    return moments_of_sums<LAT, C>(s0, sx, sy, se, rho0, ref, Ux, Uy);
}

// Moments of given macros (drho, u, theta - 1), with the reference's
// deviation v = u - U formed from vx = ux - Ux (the caller's values).
template <int LAT, typename C>
__device__ __forceinline__ Moments<LAT, C> moments_of_macros(C s0, C ux, C uy, C dT, C rho0, int ref = 0,
                                                             C Ux = C(0), C Uy = C(0))
{
    Moments<LAT, C> m;
    m.s0 = s0;
    m.rho = rho0 + s0;
    m.ux = ux;
    m.uy = uy;
    m.dT = Lat<LAT>::THERMAL ? dT : C(0);
    m.sx = m.sy = m.se = C(0);
    m.ref = ref;
    m.Ux = ref ? Ux : C(0);
    m.Uy = ref ? Uy : C(0);
    m.vx = ux - m.Ux;
    m.vy = uy - m.Uy;
    return m;
}

// Shifted equilibrium of all velocities (g^eq = f^eq - w rho0).
template <int LAT, typename C>
__device__ __forceinline__ void equilibrium(const Moments<LAT, C>& m, C* geq)
{
    using L = Lat<LAT>;
    constexpr C ics2 = C(1.0 / L::CS2);
    constexpr C a3 = L::ORDER >= 3 ? C(1.0 / 6.0) : C(0);
    constexpr C a4 = L::ORDER >= 4 ? C(1.0 / 24.0) : C(0);
    if (m.ref) {
        // relative to the reference equilibrium (eq_pair_ref)
        const C U2 = (m.Ux * m.Ux + m.Uy * m.Uy) * ics2;
        const C d = (C(2) * (m.Ux * m.vx + m.Uy * m.vy) + m.vx * m.vx + m.vy * m.vy) * ics2;
        const EqPoly<C> e = eq_poly<LAT, C>((m.ux * m.ux + m.uy * m.uy) * ics2, m.dT);
        const EqDelta<C> de = eq_delta<LAT, C>(U2, d, m.dT);
        const C rho0 = m.rho - m.s0;
        geq[0] = C(L::w(0)) * (m.s0 * (C(1) + e.A0) + rho0 * de.A0);
#pragma unroll
        for (int i = 1; i < L::Q; i += 2) {
            const C cx = C(L::cx(i)), cy = C(L::cy(i));
            const C P = (cx * m.Ux + cy * m.Uy) * ics2, q = (cx * m.vx + cy * m.vy) * ics2;
            C Ev, Od;
            eq_pair_ref<LAT, C>(e, de, C(L::c2cls(L::cls(i))) * ics2, P, q, m.s0, rho0, Ev, Od);
            geq[i] = C(L::w(i)) * (Ev + Od);
            geq[i + 1] = C(L::w(i)) * (Ev - Od);
        }
        return;
    }
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

// Grid geometry.  Populations are SoA planes f[i][y][x] with row pitch nxp;
// a node's offset inside a plane is y * nxp + x.
struct Geom {
    int nx, ny, nxp, M;
    int perx, pery;
    int bx0, bx1, by0, by1;     // bulk nodes: [bx0, bx1) x [by0, by1)
    long long plane;            // ny * nxp
    double tau, rho0, omega;    // omega = 1 / tau
    float omega_f, rho0_f, tau_f;
    unsigned long long wait_ns; // limit of the bulk kernel's first wait for a tensor copy
    // populations held relative to f^eq(rho0, uref, T0) (ref != 0) instead
    // of w rho0; uref rounded to float for float-valued arithmetic
    int ref;
    double uref[2];
    float uref_f[2];
};


// A rectangle of bulk nodes [x0, x1) x [y0, y1).
struct Region {
    int x0, x1, y0, y1;
};

// Tensor maps of one population buffer: box depths 7, 5, 3, 2 and 1 planes
// (the c_y group sizes of the three lattices).
struct Maps {
    CUtensorMap m7, m5, m3, m2, m1;
};

// Most runs one persistent bulk launch takes.
constexpr int kMaxBatchRuns = 256;

// One run of the persistent bulk kernel, in device memory: tensor maps and
// pointers of its two population buffers, geometry, the bulk region and
// the first of its work items (one item = one 128-node row segment).
struct BulkRun {
    Maps maps[2];
    void* f[2];
    int* status;
    Geom G;
    Region R;
    int seg0, nseg, first, pad;
};


// Offsets (in elements) of the pull sources and of the output planes, used
// by the bulk kernel away from periodic wrap-around: source of velocity i is
// node + ld[i] = i * plane - c_iy * nxp - c_ix, its output is node + st[i].
struct Offsets {
    int ld[37];
    int st[37];
};

// Near-boundary strips of each characteristic side, written by the band
// kernel for the next step: macros U = (drho, ux, uy, dT) and
// non-equilibrium moments N = (sigma'_xx, sigma'_xy, sigma'_yy, q_x, q_y)
// of the bulk nodes at depths d = 0 .. ND - 1 inside the boundary layers
// (x_f - d n), for two time levels.  Depths 0, 1, 2 serve the stencils of
// the boundary solver; with the mesoscopic viscous vector ND = M + 3 and
// depths M, M + 1, M + 2 serve its one-sided stencil, which starts at the
// first node none of whose populations was streamed from a boundary layer
// (N is kept there only).  Slot of (side s, depth d, position p) =
// offS[s] + d L[s] + p; arrays are [parity][slot][4] and [parity][slot][5].
struct Export {
    int cbc[4];
    int offS[4];
    int L[4];
    int ND;          // strip depths per side: 3, or M + 3 with the mesoscopic viscous vector
    int nslots;
    int sesize;      // bytes per strip value: 8 with FP64 storage, else 4 (StripReal)
    void* stripU;
    void* stripN;
};

// Shared-memory address of a generic pointer, and the global nanosecond
// timer (for bounded waits).
__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Arithmetic type of the strips and of the band kernel's stencils,
// transversal and viscous terms: FP64 with FP64 storage, FP32 otherwise.
template <typename S>
struct StripReal {
    using T = float;
};
template <>
struct StripReal<double> {
    using T = double;
};

// One unknown of the boundary ODE: layer j of a characteristic side at one
// tangential position, or the innermost node of a corner block.  Every
// neighbour the right-hand side needs is resolved when the solver is
// created: ref >= 0 is another unknown, ref < 0 is strip slot -(ref + 1)
// (a bulk node, interpolated in time between t and t + 1).
struct UDesc {
    int kind;        // side 0..3 (W, E, S, N) or 4 + corner (SW, SE, NW, NE)
    int j;           // layer 1..M (sides)
    int tmode;       // tangential stencil of the viscous terms: 0 central, 1 backward, -1 forward
    int wslot;       // strip slot of the NEEP source node (its macros at t + 1)
    int nb[6];       // +n, -n, -2n, -3n, +t, -t (corners: nb[0] = c - s, nb[1] = c - 2s)
    int vs[5];       // strip slots of the mesoscopic viscous terms: depths M, M + 1, M + 2 at p,
                     // then two tangential neighbours at depth M
    int wsrc;        // grid offset of the NEEP source node
    int wnode;       // grid offset of the node written (corner: block origin)
    int wdx, wdy;    // corner block: grid-offset steps along x and y
    int gid;         // tile tables: the unknown's global index (boundary state row)
    int level;       // tile tables: 0 owned, l > 0 halo computing 4 - l stages
    int pad;
};

// Unknowns per tile of the fused band kernel (its block size).
constexpr int kTileUnknowns = 128;

// A bulk node next to a characteristic side (a strip node) that a band tile
// reads or writes.  The bulk kernel updates it; the tile pulls it again for
// its macros (and non-equilibrium moments) at t + 1 and, for Eq. NEEP
// sources, its post-collision populations.
enum {
    kSNLoadT = 1,    // the tile reads its strip values of time t (stencils at stage 0, viscous terms)
    kSNPull = 2,     // the tile pulls it: macros of t + 1, Eq. NEEP copy, strips of t + 1
    kSNNeq = 4,      // the strips of t + 1 the tile writes include its non-equilibrium moments
};
struct StripNode {
    int x, y;
    int tslot;   // a strip slot of the node: its macros and moments of time t
    int fx;      // index of its population copy in shared memory (Eq. NEEP source), or -1
    int gslot;   // strip slot this tile writes for t + 1 (own side, owned position), or -1
    int flags;   // kSN* bits
};

enum { FFK_TINF = 0, FFK_AT, FFK_BP, FFK_1MAT, FFK_ATTI, FFK_1MAV, FFK_KR, FFK_SIXTH, FFK_N };

// The float-float split of the wave constants, from the double parameters
// already in B (host).
template <typename BandT>
inline void set_ffk(BandT& B)
{
    const double v[FFK_N] = {B.t_inf, B.alpha_T, B.beta_P, 1.0 - B.alpha_T, B.alpha_T * B.t_inf, 1.0 - B.alpha_V,
                             B.kR, 1.0 / 6.0};
    for (int q = 0; q < FFK_N; ++q) {
        const float h = float(v[q]);
        B.ffk[q][0] = h;
        B.ffk[q][1] = float(v[q] - double(h));
    }
}

struct Band {
    int n_unk;       // unknowns of the boundary ODE
    int n_zg;        // zero-gradient nodes (copied every step)
    int M;
    int viscous, dirichlet;
    int scheme[4];
    double alpha_T, beta_P, t_inf;
    double alpha_V;  // relaxation of the viscous term towards 0 (Eq. CBC-Relax extended)
    double pdev[4];  // P_inf - c_s^2 rho0 per side
    double kA;       // 1 / sqrt(8 c_s^2)
    double kB;       // sqrt(2 c_s^2)
    double kC;       // 1 / (2 sqrt 2): one-sided diagonal difference
    double kR;       // 1 / sqrt 2: corner frame
    double cs;       // c_s (isothermal system)
    double ihcs;     // 1 / (2 c_s)
    // the same constants rounded to float, for arithmetic in float-valued
    // types (no double-to-float conversion, an FP64-pipe instruction, per use)
    float kA_f, kB_f, kC_f, kR_f, cs_f, ihcs_f;
    float pdev_f[4];
    // float-float (hi, lo) forms of the wave constants (FFK_*)
    float ffk[FFK_N][2];
    const UDesc* ud;
    const int2* zg;  // (node, source) grid offsets
    // Tiles of the band kernel: tile t holds local descriptors
    // ld[t * kTileUnknowns + l] (padding: level 99) and strip nodes
    // sn[t * max_nodes + k] (padding: x = -1).  In ld, refs >= 0 index the
    // tile's unknowns and refs < 0 its strip nodes (-(k + 1)); vs[] and
    // wslot are strip-node indices, wsrc the strip node's population copy
    // (fx).
    int n_tiles;
    int max_nodes, max_fx;   // per tile, to size shared memory
    int grid;                // CTAs of the one-CTA band launch; CTA c takes tiles c, c + grid, ...
    const UDesc* ld;
    const StripNode* sn;
    double* Ub;      // boundary state [parity][n_unk][4] (the fused kernel); [n_unk][4]
                     // in the allocation-free path
    int* status;     // kernel status bits (bit 2: a cluster exchange timed out)
    double *Ya, *Yb, *acc, *V;   // stage scratch of the allocation-free path
    int* mask;
};

// ---------------------------------------------------------------------------
// Host-side launchers (defined in bulk.cu / boundary.cu)
// ---------------------------------------------------------------------------

// Launch with or without programmatic stream serialization: with it the
// kernel may start as soon as every CTA of the kernel before it in the
// stream has signalled (griddepcontrol.launch_dependents); it never waits on
// that kernel's results, so it must not read what that kernel writes.  Work
// issued after it in the stream still waits for both.
template <typename... K, typename... A>
inline int launch_ex(void (*kern)(K...), dim3 grd, dim3 blk, size_t smem, cudaStream_t st, bool early, A... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grd;
    cfg.blockDim = blk;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = early ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...) == cudaSuccess ? 0 : -1;
}

// The same with thread-block clusters of `cluster` CTAs along x (1: none).
template <typename... K, typename... A>
inline int launch_ex_cl(void (*kern)(K...), dim3 grd, dim3 blk, size_t smem, cudaStream_t st, bool early,
                        int cluster, A... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grd;
    cfg.blockDim = blk;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    int n = 0;
    if (early) {
        at[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[n].val.programmaticStreamSerializationAllowed = 1;
        ++n;
    }
    if (cluster > 1) {
        at[n].id = cudaLaunchAttributeClusterDimension;
        at[n].val.clusterDim.x = unsigned(cluster);
        at[n].val.clusterDim.y = 1;
        at[n].val.clusterDim.z = 1;
        ++n;
    }
    cfg.attrs = at;
    cfg.numAttrs = n;
    return cudaLaunchKernelEx(&cfg, kern, args...) == cudaSuccess ? 0 : -1;
}


// Initial populations f^eq(U0) into f, strips of time 0, boundary state.
int launch_init(int lat, int storage, const Geom& G, const Export& E, const Band& B,
                const double* rho, const double* ux, const double* uy, const double* T, void* f,
                cudaStream_t st);
// Fixed inflow equilibrium at the listed nodes of one population buffer.
int launch_inflow(int lat, int storage, const Geom& G, const int* nodes, int n, const double Uin[4],
                  void* f, cudaStream_t st);
// One bulk step fin -> fout over the nodes of region R; tmaps[0..4] describe
// fin for the tensor copies (box depths 7, 5, 3, 2, 1 planes); *status gets bit 1
// if a copy never completed.  early: programmatic stream serialization (the
// launch may start while the kernel before it in the stream runs, once that
// kernel's CTAs have signalled; it must not read what that kernel writes).
int launch_bulk(int lat, int storage, const Geom& G, const Offsets& O, const Region& R,
                const CUtensorMap* tmaps, const void* fin, void* fout, int* status,
                cudaStream_t st, bool early = false);
int launch_macros(int lat, int storage, const Geom& G, const void* f, double* rho, double* ux,
                  double* uy, double* T, int* flag, cudaStream_t st);
// The band of one step fin -> fnew: strip nodes, RK4 of the characteristic
// boundary state, Dirichlet populations.
int launch_boundary(int lat, int storage, const Geom& G, const Offsets& O, const Export& E,
                    const Band& B, const void* fin, void* fnew, int par_t,
                    cudaStream_t st);
// One grid of the batched band kernel, in device memory.
struct BandRun {
    Geom G;
    Offsets O;
    Band B;
    Export E;
    void* f[2];
};
// Band tiles of many grids of one lattice and storage in one launch:
// tile_run[t] = (run, tile of that run); smem = the largest band_dynamic_smem.
int launch_band_batch(int lat, int storage, const BandRun* runs, const int2* tile_run, int n_tiles,
                      size_t smem, int par_t, cudaStream_t st, bool early = false);
int prepare_band_batch(int lat, int storage, size_t smem);
// Dynamic shared memory the band kernel needs per CTA (without padding).
size_t band_dynamic_smem(int lat, int storage, const Band& B);
// Persistent bulk step of n_runs runs of one lattice and storage (buffer
// par -> par ^ 1 of each) with `grid` CTAs taking the total work items from
// a queue (two unsigned words in device memory, zero before the first
// launch; each launch leaves them zero), a two-stage tensor-copy pipeline
// per CTA.  Launches sharing a queue must not overlap.
int launch_bulk_persistent(int lat, int storage, const BulkRun* runs, int n_runs, int total, int par,
                           int grid, unsigned* queue, cudaStream_t st, bool early = false);
// Opt the persistent bulk kernel in to its dynamic shared memory.
int prepare_bulk_persistent(int lat, int storage);
// Opt the band kernel in to its dynamic shared memory (once, at creation).
int prepare_boundary(int lat, int storage, const Band& B);

// Zero-gradient copies (Eq. zg-bc) in fnew, after the bulk update of x_f.
int launch_zg(int lat, int storage, const Geom& G, const Band& B, void* fnew, cudaStream_t st);

// State of the tangent-linear step (tangent.cu): derivatives along three
// directions in the space of the relaxation parameters theta = (alpha_T,
// beta_P, P_inf (all sides), alpha_V, t_inf): direction k is dirs[k][.]
// (by default the first three unit vectors).  Arrays are sized with
// tl_dual_bytes() per value (the largest element type used).
constexpr int kTLParams = 5;
struct TLState {
    void* t[2];      // derivative populations per parity: [3][Q][plane], storage type
    void* strip[2];  // strip macros per parity (t, then t + 1): [nslots][4], stage type
    void* stripN[2]; // strip non-equilibrium moments per parity: [nslots][5], stage type
                     // (mesoscopic viscous vector only)
    void* Ud;        // boundary state: [n_unk][4], FP64 value + FP32 derivatives
    void* Uf;        // the same in the stage type
    void *Ya, *Yb;   // RK4 stage values: [n_unk][4], stage type
    void* acc;       // RK4 sum: [n_unk][4], as Ud
    int* mask;       // incoming waves at t: [n_unk]
    void* Vv;        // "-FD" viscous vector of time t: [n_unk][4], stage type
    double* sums;    // J and its derivatives along the three directions
    double dirs[3][kTLParams];
};
size_t tl_dual_bytes();
// One tangent-linear step f[par] -> f[par ^ 1] (FP64 or FP32 storage; the
// handle's checks exclude NEEP and inflow / zero-gradient sides), adding the loss over the bulk nodes (the nodes off the boundary
// layers) against dPref ([ny][nx] of P_ref - c_s^2 rho0, or null for 0) to
// T.sums.
int launch_tl_step(int lat, int storage, const TLState& T, const Geom& G, const Export& E,
                   const Band& B, const Region& bulk, void* const f[2], int par, const double* dPref,
                   cudaStream_t st);
// Seed the strip macros of parity par from f[par] and T.Ud / T.Uf with the
// boundary state of parity par (the derivatives as T holds them: zero after
// lbm_grad_begin's clear).
int launch_tl_seed(int lat, int storage, const TLState& T, const Geom& G, const Export& E, const Band& B,
                   void* const f[2], int par, cudaStream_t st);

// Reverse-mode (adjoint) sweep (adjoint.cu).  History of one recomputed
// segment (index k = step - first step of the segment) and the adjoint
// variables; element type C = the storage's arithmetic (populations) and R =
// StripReal (boundary solver inputs), except where stated.
// RK4 stage fields of one step at the unknowns, with the viscous vector and
// the incoming waves frozen at its stage 0.
struct StageSet {
    void* Y[4];       // [n_unk][4] (R): Y[0] = U_b(t), Y[s + 1] = U_b(t) + h_s k_s
    void* V;          // [n_unk][4] (R)
    int* mask;        // [n_unk]
};

struct AdjState {
    int K;            // checkpoint interval: steps per segment
    void* Mh;         // [K][ny * nx][4] (R): drho, ux, uy, dT of the bulk nodes after step k
                      // of a segment (two buffers: recompute beside the reverse steps)
    double* Ubh;      // [steps + 1][n_unk][4]: boundary state before step k of the run
    void* stUh;       // [steps + 1][nslots][4] (R): strip macros of the time before step k
    void* stNh;       // [steps + 1][nslots][5] (R): strip non-equilibrium moments, same time
    void* lpre[2];    // [Q][plane] (C): adjoint of the pulled (pre-collision) populations,
                      // by parity of their time
    double* lU;       // [n_unk][4]: adjoint of the boundary state
    void* lUr;        // [n_unk][4] (R): its rounding, read by the stage kernels
    StageSet sets[2]; // stage fields by parity of the step index within the run; the
                      // reverse step of t computes those of t - 1 beside its own adjoint
    void* Y[4];       // [n_unk][4] (R): RK4 stage fields at the unknowns (Y[0] = U_b(t)),
                      // the current set's
    void* lY[4];      // [n_unk][4] (R): their adjoints
    void* V;          // [n_unk][4] (R): viscous vector of the step (frozen), current set
    void* lV;         // [n_unk][4] (R): its adjoint
    int* mask;        // [n_unk]: incoming waves of the step, current set
    void* lSt;        // [nslots][4] (R): adjoint of the strip macros of time t
    void* lSt1;       // [nslots][4] (R): adjoint of the strip macros of time t + 1
    void* lN;         // [nslots][5] (R): adjoint of the strip moments of time t
    void* ext[2];     // [nslots][9] (R): what the strips add to the adjoint of the pulled
                      // populations of a strip node, by parity of the time: 4 moment
                      // coefficients, 5 weights of the non-equilibrium moments
    double* sums;     // [7]: J, dJ / d(alpha_T, beta_P, P_inf, alpha_V, t_inf), J again
    double* cpart;    // [4][4][M * M - 1]: corner blocks' Dirichlet shares (one step)
    // alpha_T, beta_P, t_inf, alpha_V, P_inf - c_s^2 rho0 per side, rounded
    // to float and as double (the stage kernels take their arithmetic's)
    float relax_f[8];
    double relax_d[8];
};
// Loss of the state in f (populations after a step) against dPref (or 0):
// sums[0] += sum over the bulk nodes of (P - c_s^2 rho0 - dPref)^2 (skipped
// if sums is null); the bulk nodes' moments into Mout ([ny * nx][4] of the
// strip type; skipped if null); it also copies the record rec.
// A history record copied by the loss kernel beside its work: the boundary
// state (n_ub doubles) and the strips' macros and moments (n_su, n_sn values
// of the strip type) of the time the loss is taken at (counts 0: none).
struct AdjRecord {
    const double* ub;
    double* ubh;
    long long n_ub;
    const void* su;
    void* suh;
    long long n_su;
    const void* sn;
    void* snh;
    long long n_sn;
};
int launch_adj_loss(int lat, int storage, const Geom& G, const Region& bulk, const void* f,
                    const double* dPref, double* sums, void* Mout, const AdjRecord& rec, cudaStream_t st);
// The Dirichlet write of a step (equilibrium form) from the boundary state
// Ub1 ([n_unk][4]) into the populations f.
int launch_adj_dwrite(int lat, int storage, const Geom& G, const Band& B, const double* Ub1, void* f,
                      cudaStream_t st);
// One reverse step for the forward step t -> t + 1 (see adjoint.cu):
// Ub, Ub1: the boundary state at t and t + 1; stU, stN: strips of t; stU1:
// strip macros of t + 1; Mh1: macros at t + 1; dPref1: the loss reference at
// t + 1 (or null); par: parity of t.  The boundary kernels go on st, the
// bulk kernel on sw (after what sw already waits for), joined on st through
// ev_bulk before the step's last kernel.  Stage set `set` (the parity of t's
// index within the run) holds t's stage fields if `pre` (computed by the
// reverse step of t + 1); with `nxt` this step computes those of t - 1 into
// the other set from Ubm = U_b(t - 1) and the strips stUm, stNm of t - 1.
int launch_adj_step(int lat, int storage, const Geom& G, const Export& E, const Band& B,
                    const Region& bulk, const AdjState& A, const double* Ub, const double* Ub1,
                    const void* stU, const void* stN, const void* stU1, const void* Mh1,
                    const double* dPref1, int par, int set, int pre, int nxt, const double* Ubm,
                    const void* stUm, const void* stNm, cudaStream_t st, cudaStream_t sw, cudaEvent_t ev_bulk);

}  // namespace lbmgb
