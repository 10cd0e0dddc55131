// charsys.cuh -- the characteristic system of the boundary solver (Sec. 3):
// frames, neighbour fetches, the decomposition and incoming-wave choice,
// the viscous vectors and the right-hand side of one boundary unknown.
// Used by the allocation-free boundary step and the tangent-linear step;
// the fused band kernel (boundary.cu) has its own cluster-split form of the
// same arithmetic.
#pragma once
#include "collide.cuh"

#include <type_traits>

namespace lbmgb {

// Lab <-> local frame.  Sides: n the outward normal, t = +y (W, E) or +x
// (S, N).  Corners: n = (sx, sy)/sqrt(2), t = n rotated by +90 degrees.
template <typename R>
__device__ __forceinline__ void to_local(int kind, R r, const R* U, R* Lc)
{
    Lc[0] = U[0];
    Lc[3] = U[3];
    switch (kind) {
    case 0: Lc[1] = -U[1]; Lc[2] = U[2]; break;
    case 1: Lc[1] = U[1]; Lc[2] = U[2]; break;
    case 2: Lc[1] = -U[2]; Lc[2] = U[1]; break;
    case 3: Lc[1] = U[2]; Lc[2] = U[1]; break;
    default: {
        const int c = kind - 4;
        const R n0 = (c & 1) ? r : -r, n1 = (c & 2) ? r : -r;
        Lc[1] = U[1] * n0 + U[2] * n1;
        Lc[2] = -U[1] * n1 + U[2] * n0;
    }
    }
}

template <typename R>
__device__ __forceinline__ void to_lab(int kind, R r, const R* Lc, R* U)
{
    U[0] = Lc[0];
    U[3] = Lc[3];
    switch (kind) {
    case 0: U[1] = -Lc[1]; U[2] = Lc[2]; break;
    case 1: U[1] = Lc[1]; U[2] = Lc[2]; break;
    case 2: U[2] = -Lc[1]; U[1] = Lc[2]; break;
    case 3: U[2] = Lc[1]; U[1] = Lc[2]; break;
    default: {
        const int c = kind - 4;
        const R n0 = (c & 1) ? r : -r, n1 = (c & 2) ? r : -r;
        U[1] = Lc[1] * n0 - Lc[2] * n1;
        U[2] = Lc[1] * n1 + Lc[2] * n0;
    }
    }
}

// A constant of the boundary solver in arithmetic type T: its float
// rounding for float-valued T (the same value the conversion would give),
// the double otherwise.
template <typename T>
__device__ __forceinline__ T bconst(double d, float f)
{
    if constexpr (sizeof(typename DualTraits<T>::Value) == 4) return T(f);
    else return T(d);
}

// Where a right-hand side reads its neighbours, in arithmetic type R.
template <typename R>
struct CtxT {
    const R* Y;     // stage values of the unknowns
    const R* St;    // strip macros at t
    const R* St1;   // strip macros at t + 1
    R frac;         // stage time fraction in [0, 1]
};
using Ctx = CtxT<double>;

template <typename R>
__device__ __forceinline__ void fetch(const CtxT<R>& X, int ref, R* U)
{
    if (ref >= 0) {
        if constexpr (std::is_same<R, double>::value) {
            const double2* p = reinterpret_cast<const double2*>(X.Y + 4LL * ref);
            const double2 a = p[0], b = p[1];
            U[0] = a.x; U[1] = a.y; U[2] = b.x; U[3] = b.y;
        } else if constexpr (std::is_same<R, float>::value) {
            const float4 a = *reinterpret_cast<const float4*>(X.Y + 4LL * ref);
            U[0] = a.x; U[1] = a.y; U[2] = a.z; U[3] = a.w;
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) U[c] = X.Y[4LL * ref + c];
        }
    } else {
        const long long s = 4LL * (-ref - 1);
        const R w0 = R(1) - X.frac, w1 = X.frac;
#pragma unroll
        for (int c = 0; c < 4; ++c) U[c] = w0 * X.St[s + c] + w1 * X.St1[s + c];
    }
}

template <typename R>
__device__ __forceinline__ void fetch_local(const CtxT<R>& X, int ref, int kind, R r, R* Lc)
{
    R U[4];
    fetch(X, ref, U);
    to_local(kind, r, U, Lc);
}

// ---------------------------------------------------------------------------
// Characteristic system in the local frame (Sec. 3.1)
// ---------------------------------------------------------------------------
// Thermal, U = (drho, u_n, u_t, dT), theta = 1 + dT, T~ = c_s^2 theta:
//   S rows: (-r/2, 0, 0, 1/2), (0, 0, 1, 0), (r/4, -a, 0, 1/4), (r/4, a, 0, 1/4)
//   S^-1 rows: (-1/r, 0, 1/r, 1/r), (0, 0, -b, b), (0, 1, 0, 0), (1, 0, 1, 1)
//   with r = T~/(rho c_s^2) = theta/rho, a = sqrt(T~/(8 c_s^4)),
//   b = sqrt(2 c_s^4 / T~) and Lambda = (u_n, u_n, u_n - c, u_n + c),
//   c = sqrt(2 T~).
// Isothermal D2Q9, U = (drho, u_n, u_t):
//   S rows: (1/2, -h, 0), (0, 0, 1), (1/2, h, 0) with h = rho/(2 c_s),
//   S^-1 rows: (1, 0, 1), (-c_s/rho, 0, c_s/rho), (0, 1, 0),
//   Lambda = (u_n - c_s, u_n, u_n + c_s).
// Everything below is templated on the arithmetic type T (double, or a
// Dual number for the tangent-linear step).
template <typename T>
struct CharSys {
    T rho, irho, r, ir, a, b, h, csr;
    T lam[4];
};

// The relaxation parameters of the incoming waves (Eqs. LODI-Relax,
// CBC-Relax): alpha_T on the transversal terms, beta_P on P - P_inf,
// the target transversal term t_inf, alpha_V on the viscous term (towards
// 0; 0 is the paper's equation), and P_inf - c_s^2 rho0 per side.
template <typename T>
struct Relax {
    T alpha_T, beta_P, t_inf, alpha_V;
    T pdev[4];
};

template <typename T>
__device__ __forceinline__ Relax<T> relax_of(const Band& B)
{
    Relax<T> P;
    P.alpha_T = T(B.alpha_T);
    P.beta_P = T(B.beta_P);
    P.t_inf = T(B.t_inf);
    P.alpha_V = T(B.alpha_V);
#pragma unroll
    for (int s = 0; s < 4; ++s) P.pdev[s] = T(B.pdev[s]);
    return P;
}

template <bool TH, typename T>
__device__ __forceinline__ CharSys<T> char_sys_r(const Band& B, const T& rho0, const T* U)
{
    CharSys<T> C;
    C.rho = rho0 + U[0];
    C.irho = T(1) / C.rho;
    if (TH) {
        const T th = T(1) + U[3];
        const T sth = sqrt(th);
        const T isth = T(1) / sth;
        C.r = th * C.irho;
        C.ir = C.rho * isth * isth;
        C.a = sth * bconst<T>(B.kA, B.kA_f);
        C.b = isth * bconst<T>(B.kB, B.kB_f);
        const T c = sth * bconst<T>(B.kB, B.kB_f);
        C.lam[0] = U[1];
        C.lam[1] = U[1];
        C.lam[2] = U[1] - c;
        C.lam[3] = U[1] + c;
        C.h = C.csr = T(0);
    } else {
        C.h = C.rho * bconst<T>(B.ihcs, B.ihcs_f);
        C.csr = bconst<T>(B.cs, B.cs_f) * C.irho;
        C.lam[0] = U[1] - bconst<T>(B.cs, B.cs_f);
        C.lam[1] = U[1];
        C.lam[2] = U[1] + bconst<T>(B.cs, B.cs_f);
        C.lam[3] = T(0);
        C.r = C.ir = C.a = C.b = T(0);
    }
    return C;
}

template <bool TH, typename T>
__device__ __forceinline__ CharSys<T> char_sys(const Band& B, double rho0, const T* U)
{
    return char_sys_r<TH, T>(B, T(rho0), U);
}

template <bool TH, typename T>
__device__ __forceinline__ void apply_S(const CharSys<T>& C, const T* v, T* o)
{
    if (TH) {
        const T rv = T(0.25) * C.r * v[0], q = T(0.25) * v[3], av = C.a * v[1];
        o[0] = T(-2) * rv + T(2) * q;
        o[1] = v[2];
        o[2] = rv - av + q;
        o[3] = rv + av + q;
    } else {
        const T hv = C.h * v[1];
        o[0] = T(0.5) * v[0] - hv;
        o[1] = v[2];
        o[2] = T(0.5) * v[0] + hv;
        o[3] = T(0);
    }
}

template <bool TH, typename T>
__device__ __forceinline__ int incoming_mask(const CharSys<T>& C)
{
    int m = 0;
#pragma unroll
    for (int i = 0; i < (TH ? 4 : 3); ++i)
        if (C.lam[i] < 0.0) m |= 1 << i;
    return m;
}

// dU/dt = -S^-1 Lbar (+ T + V for the CBC schemes): Lbar_i = L_i =
// Lambda_i (S dU/dn)_i for outgoing waves (Eq. thermal_WAV); for incoming
// waves Eq. PNR (LODI), Eq. LODI-Relax, Eq. CBC-PNR (CBC) or Eq. CBC-Relax,
// with beta (Z - Z_inf) on the incoming acoustic waves.
template <bool TH, typename T>
__device__ __forceinline__ void char_rhs(const CharSys<T>& C, const Relax<T>& P, const T* dUn,
                                         const T* TT, const T* VV, int mask, const T& dP, int scheme,
                                         T* k)
{
    T sd[4], st[4], sv[4], w[4];
    apply_S<TH>(C, dUn, sd);
    apply_S<TH>(C, TT, st);
    apply_S<TH>(C, VV, sv);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!TH && i == 3) { w[i] = T(0); continue; }
        if (!((mask >> i) & 1)) {
            w[i] = C.lam[i] * sd[i];
            continue;
        }
        const bool acoustic = TH ? (i >= 2) : (i != 1);
        const T relaxP = acoustic ? P.beta_P * dP : T(0);
        if (scheme == SCH_LODI) w[i] = T(0);
        else if (scheme == SCH_LODI_RELAX) w[i] = P.alpha_T * (P.t_inf - st[i]) + relaxP;
        else if (scheme == SCH_CBC) w[i] = st[i] + sv[i];
        else w[i] = st[i] + sv[i] + P.alpha_T * (P.t_inf - st[i]) + P.alpha_V * (T(0) - sv[i]) + relaxP;
    }
    T o[4];
    if (TH) {
        o[0] = (w[2] + w[3] - w[0]) * C.ir;
        o[1] = C.b * (w[3] - w[2]);
        o[2] = w[1];
        o[3] = w[0] + w[2] + w[3];
    } else {
        o[0] = w[0] + w[2];
        o[1] = C.csr * (w[2] - w[0]);
        o[2] = w[1];
        o[3] = T(0);
    }
    const bool cbc = scheme == SCH_CBC || scheme == SCH_CBC_RELAX;
#pragma unroll
    for (int m = 0; m < 4; ++m) k[m] = cbc ? -o[m] + (TT[m] + VV[m]) : -o[m];
}

// ---------------------------------------------------------------------------
// Viscous vectors, frozen at time t
// ---------------------------------------------------------------------------

// Mesoscopic form (Eqs. LaplaceU, LaplaceT) with the stencil starting M
// nodes below x_f (the first node none of whose populations came from a
// boundary layer): normal derivatives one-sided into the bulk
// (Eq. FD-dx-bw), tangential ones central (Eq. FD-dx-center) or one-sided
// inward next to a boundary node:
//   V = (0, (1/rho) d_j s'_jn, (1/rho) d_j s'_jt,
//        -div q / (rho c_s^2) + (nu / c_s^2) ((d_n u_n - d_t u_t)^2 + (d_n u_t + d_t u_n)^2)).
template <bool TH, typename T>
__device__ void vis_meso(const Geom& G, const T* SU, int su, const T* SN, int sn_, const UDesc& D,
                         double cs2, T* V)
{
    // SU, SN: macros (drho, ux, uy, ...) and non-equilibrium moments
    // (sigma'_xx, sigma'_xy, sigma'_yy, q_x, q_y) of time t, node k at
    // SU + su * k and SN + sn_ * k, indexed by D.vs[]; arithmetic T (FP64,
    // or Dual numbers in the tangent-linear step)
    const int s = D.kind;
    const int an = s < 2 ? 0 : 1, at = 1 - an;     // axes of n and t
    const T sn = T((s == 0 || s == 2) ? -1.0 : 1.0);
    T h[5][7];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const T* n = SN + (long long)sn_ * D.vs[k];
        const T* u = SU + (long long)su * D.vs[k];
        const T sxx = n[0], sxy = n[1], syy = n[2];
        h[k][0] = an == 0 ? sxx : syy;              // sigma'_nn
        h[k][1] = sn * sxy;                         // sigma'_nt
        h[k][2] = an == 0 ? syy : sxx;              // sigma'_tt
        h[k][3] = sn * n[3 + an];                   // q_n
        h[k][4] = n[3 + at];                        // q_t
        h[k][5] = sn * u[1 + an];                   // u_n
        h[k][6] = u[1 + at];                        // u_t
    }
    T dn[7], dt[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) {
        dn[m] = T(0.5) * (T(3) * h[0][m] - T(4) * h[1][m] + h[2][m]);
        if (D.tmode == 0) dt[m] = T(0.5) * (h[3][m] - h[4][m]);
        else dt[m] = T(float(D.tmode)) * T(0.5) * (T(3) * h[0][m] - T(4) * h[3][m] + h[4][m]);
    }
    const T irho = T(1) / (bconst<T>(G.rho0, G.rho0_f) + SU[(long long)su * D.vs[0]]);
    V[0] = T(0);
    V[1] = (dn[0] + dt[1]) * irho;
    V[2] = (dn[1] + dt[2]) * irho;
    V[3] = T(0);
    if (TH) {
        const T nu = T((G.tau - 0.5) * cs2);
        const T e1 = dn[5] - dt[6], e2 = dn[6] + dt[5];
        V[3] = -(dn[3] + dt[4]) * irho * T(1.0 / cs2) + nu * T(1.0 / cs2) * (e1 * e1 + e2 * e2);
    }
}

// "-FD" form (Sec. 4.2) at layer j from the macros of time t: 4-point
// one-sided second derivative at j = M, 3-point central elsewhere.  In the
// context's arithmetic R (FP64, or Dual numbers in the tangent-linear step).
template <bool TH, typename R>
__device__ void vis_fd(const Geom& G, const Band& B, const CtxT<R>& X0, const UDesc& D, int u,
                       double cs2, R* V)
{
    const int kind = D.kind;
    R U[4], A[4], Bv[4], Cv[4], Tp[4], Tm[4], dnn[4], d1n[4];
    fetch_local(X0, u, kind, R(0), U);
    fetch_local(X0, D.nb[1], kind, R(0), Bv);
    fetch_local(X0, D.nb[4], kind, R(0), Tp);
    fetch_local(X0, D.nb[5], kind, R(0), Tm);
    if (D.j == B.M) {
        fetch_local(X0, D.nb[2], kind, R(0), A);
        fetch_local(X0, D.nb[3], kind, R(0), Cv);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            dnn[m] = R(2) * U[m] - R(5) * Bv[m] + R(4) * A[m] - Cv[m];
            d1n[m] = R(0.5) * (R(3) * U[m] - R(4) * Bv[m] + A[m]);
        }
    } else {
        fetch_local(X0, D.nb[0], kind, R(0), A);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            dnn[m] = A[m] - R(2) * U[m] + Bv[m];
            d1n[m] = R(0.5) * (A[m] - Bv[m]);
        }
    }
    const R nu = R((G.tau - 0.5) * cs2);
    V[0] = R(0);
    V[1] = nu * (dnn[1] + (Tp[1] - R(2) * U[1] + Tm[1]));
    V[2] = nu * (dnn[2] + (Tp[2] - R(2) * U[2] + Tm[2]));
    V[3] = R(0);
    if (TH) {
        const R d1t1 = R(0.5) * (Tp[1] - Tm[1]), d1t2 = R(0.5) * (Tp[2] - Tm[2]);
        const R e1 = d1n[1] - d1t2, e2 = d1n[2] + d1t1;
        V[3] = R(2) * nu * (dnn[3] + (Tp[3] - R(2) * U[3] + Tm[3])) + nu * R(1.0 / cs2) * (e1 * e1 + e2 * e2);
    }
}

// ---------------------------------------------------------------------------
// Right-hand side of one unknown
// ---------------------------------------------------------------------------

template <int LAT, typename T>
__device__ void unknown_rhs(const Geom& G, const Band& B, const Relax<T>& P, const CtxT<T>& X,
                            const UDesc& D, int u, const T* V, int mask, T* k)
{
    using L = Lat<LAT>;
    constexpr bool TH = L::THERMAL;
    const int kind = D.kind;
    const T r = bconst<T>(B.kR, B.kR_f);
    T U[4], A[4], Bv[4], dUn[4];
    fetch_local(X, u, kind, r, U);
    if (kind >= 4) {
        // Corner: LODI (Eq. PNR) along the outward diagonal, one-sided
        // difference of spacing sqrt(2) through the two diagonal bulk nodes.
        fetch_local(X, D.nb[0], kind, r, A);
        fetch_local(X, D.nb[1], kind, r, Bv);
#pragma unroll
        for (int m = 0; m < 4; ++m) dUn[m] = (T(3) * U[m] - T(4) * A[m] + Bv[m]) * bconst<T>(B.kC, B.kC_f);
        const T zero[4] = {T(0), T(0), T(0), T(0)};
        const CharSys<T> C = char_sys_r<TH, T>(B, bconst<T>(G.rho0, G.rho0_f), U);
        T kl[4];
        char_rhs<TH>(C, P, dUn, zero, zero, mask, T(0), SCH_LODI, kl);
        to_lab(kind, r, kl, k);
        return;
    }
    if (D.j == B.M) {            // Eq. FD-dx-bw at the outermost layer
        fetch_local(X, D.nb[1], kind, r, A);
        fetch_local(X, D.nb[2], kind, r, Bv);
#pragma unroll
        for (int m = 0; m < 4; ++m) dUn[m] = T(0.5) * (T(3) * U[m] - T(4) * A[m] + Bv[m]);
    } else {                     // Eq. FD-dx-center at inner layers
        fetch_local(X, D.nb[0], kind, r, A);
        fetch_local(X, D.nb[1], kind, r, Bv);
#pragma unroll
        for (int m = 0; m < 4; ++m) dUn[m] = T(0.5) * (A[m] - Bv[m]);
    }
    // transversal vector T (Sec. 3.1) from central differences along the side
    T Up[4], Um[4];
    fetch_local(X, D.nb[4], kind, r, Up);
    fetch_local(X, D.nb[5], kind, r, Um);
    const T rho0 = bconst<T>(G.rho0, G.rho0_f), cs2 = T(L::CS2);
    const CharSys<T> C = char_sys_r<TH, T>(B, rho0, U);
    const T ut = U[2];
    const T d_rhout = T(0.5) * ((rho0 + Up[0]) * Up[2] - (rho0 + Um[0]) * Um[2]);
    const T d_un = T(0.5) * (Up[1] - Um[1]);
    const T d_ut = T(0.5) * (Up[2] - Um[2]);
    // P_inf - c_s^2 rho0 of this side (selected, not indexed: no stack)
    const T pdev = kind == 0 ? P.pdev[0] : kind == 1 ? P.pdev[1] : kind == 2 ? P.pdev[2] : P.pdev[3];
    T TT[4], dP;
    if (TH) {
        // rho T - rho0 = drho + rho0 dT + drho dT
        const T d_rhoT = T(0.5) * ((Up[0] + rho0 * Up[3] + Up[0] * Up[3]) -
                                   (Um[0] + rho0 * Um[3] + Um[0] * Um[3]));
        const T d_Tut = T(0.5) * ((T(1) + Up[3]) * Up[2] - (T(1) + Um[3]) * Um[2]);
        TT[0] = -d_rhout;
        TT[1] = -ut * d_un;
        TT[2] = -cs2 * C.irho * d_rhoT - ut * d_ut;
        TT[3] = -d_Tut;
        dP = cs2 * (U[0] + rho0 * U[3] + U[0] * U[3]) - pdev;
    } else {
        TT[0] = -d_rhout;
        TT[1] = -ut * d_un;
        TT[2] = -cs2 * C.irho * T(0.5) * (Up[0] - Um[0]) - ut * d_ut;
        TT[3] = T(0);
        dP = cs2 * U[0] - pdev;
    }
    T kl[4];
    char_rhs<TH>(C, P, dUn, TT, V, mask, dP, B.scheme[kind], kl);
    to_lab(kind, r, kl, k);
}

// Mesoscopic Dirichlet condition for the new boundary state, stored
// post-collision: f^eq(Unew) and, for Eq. NEEP, the non-equilibrium part of
// the bulk neighbour after its collision, f*(x_f) - f^eq(U(x_f, t+1)), or
// (dirichlet 2) that part projected onto the Hermite polynomials of orders 2
// and 3 (a regularised scheme, named by the paper as future work).
// Computed in the arithmetic type of the storage.
template <int LAT, typename S, typename R, bool REF = true>
__device__ void dirichlet(const Geom& G, const Band& B, S* f, const R* Us, const S* fsrc,
                          const UDesc& D, const R* Unew, bool dry = false)
{
    // dry: the same instructions without the stores (instruction-cache
    // warm-up)
    // Us: macros of x_f at t + 1; fsrc: its stored post-collision
    // populations, indexed by velocity (both read only for Eq. NEEP)
    using L = Lat<LAT>;
    using Cm = typename Store<S>::C;
    Moments<LAT, Cm> m;
    m.s0 = Cm(Unew[0]);
    m.rho = Cm(G.rho0) + m.s0;
    m.ux = Cm(Unew[1]);
    m.uy = Cm(Unew[2]);
    m.dT = L::THERMAL ? Cm(Unew[3]) : Cm(0);
    if (REF && G.ref) {
        m.ref = 1;
        m.Ux = Cm(stored_ref<S>(G, 0));
        m.Uy = Cm(stored_ref<S>(G, 1));
        m.vx = Cm(double(Unew[1]) - stored_ref<S>(G, 0));
        m.vy = Cm(double(Unew[2]) - stored_ref<S>(G, 1));
    }
    Cm ge[L::Q];
    equilibrium<LAT, Cm>(m, ge);
    if (B.dirichlet >= 1) {             // Eq. NEEP, or its regularised form
        Moments<LAT, Cm> ms;
        ms.s0 = Cm(Us[0]);
        ms.rho = Cm(G.rho0) + ms.s0;
        ms.ux = Cm(Us[1]);
        ms.uy = Cm(Us[2]);
        ms.dT = L::THERMAL ? Cm(Us[3]) : Cm(0);
        if (REF && G.ref) {
            ms.ref = 1;
            ms.Ux = Cm(stored_ref<S>(G, 0));
            ms.Uy = Cm(stored_ref<S>(G, 1));
            ms.vx = Cm(double(Us[1]) - stored_ref<S>(G, 0));
            ms.vy = Cm(double(Us[2]) - stored_ref<S>(G, 1));
        }
        Cm gs[L::Q];
        equilibrium<LAT, Cm>(ms, gs);
        Cm gn[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            Cm v = Cm(Store<S>::value(fsrc[i]));     // fsrc is in shared memory
            if (Store<S>::SCALED) v *= Cm(L::w(i));
            gn[i] = v - gs[i];
        }
        if (B.dirichlet == 2) {
            // Regularised form: the Hermite projection of f^neq onto orders 2
            // (and 3 on the thermal lattices),
            // w_i [H2_i : a2 / (2 c_s^4) + H3_i : a3 / (6 c_s^6)], a_n = sum H_n f^neq
            constexpr Cm cs2 = Cm(L::CS2);
            Cm a2xx = 0, a2xy = 0, a2yy = 0, a3xxx = 0, a3xxy = 0, a3xyy = 0, a3yyy = 0;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const Cm cx = Cm(L::cx(i)), cy = Cm(L::cy(i));
                a2xx += (cx * cx - cs2) * gn[i];
                a2xy += cx * cy * gn[i];
                a2yy += (cy * cy - cs2) * gn[i];
                if (L::ORDER >= 3) {
                    a3xxx += (cx * cx * cx - Cm(3) * cs2 * cx) * gn[i];
                    a3xxy += (cx * cx * cy - cs2 * cy) * gn[i];
                    a3xyy += (cx * cy * cy - cs2 * cx) * gn[i];
                    a3yyy += (cy * cy * cy - Cm(3) * cs2 * cy) * gn[i];
                }
            }
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const Cm cx = Cm(L::cx(i)), cy = Cm(L::cy(i));
                const Cm h2 = (cx * cx - cs2) * a2xx + Cm(2) * cx * cy * a2xy + (cy * cy - cs2) * a2yy;
                Cm h = h2 / (Cm(2) * cs2 * cs2);
                if (L::ORDER >= 3) {
                    const Cm h3 = (cx * cx * cx - Cm(3) * cs2 * cx) * a3xxx +
                                  Cm(3) * (cx * cx * cy - cs2 * cy) * a3xxy +
                                  Cm(3) * (cx * cy * cy - cs2 * cx) * a3xyy +
                                  (cy * cy * cy - Cm(3) * cs2 * cy) * a3yyy;
                    h += h3 / (Cm(6) * cs2 * cs2 * cs2);
                }
                gn[i] = Cm(L::w(i)) * h;
            }
        }
#pragma unroll
        for (int i = 0; i < L::Q; ++i) ge[i] += gn[i];
    }
    const int nb = D.kind >= 4 ? G.M : 1;
    for (int a = 0; a < nb; ++a)
        for (int b = 0; b < nb; ++b) {
            const long long node = D.wnode + a * D.wdx + b * D.wdy;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                Cm v = ge[i];
                if (Store<S>::SCALED) v *= Cm(1.0 / L::w(i));
                if (!dry) Store<S>::put(f + L::plane_of(i) * G.plane + node, v);
            }
        }
}

}  // namespace lbmgb
