// boundary.cu -- boundary conditions of one time step.
//
//  k_stage   one classical RK4 stage (Sec. 3.3, "Time integration") of the
//            boundary ODE on every characteristic unknown: layer j = 1..M
//            of every CBC side position (Sec. 3.3, "Multi-speed LBM") and the
//            innermost node of every corner block.  Stage 0 freezes the
//            viscous vector and the incoming-wave mask of time t; stage 3
//            ends the step, writes the mesoscopic Dirichlet populations
//            (equilibrium or Eq. NEEP) post-collision into the new buffer,
//            and copies the zero-gradient nodes (Eq. zg-bc).
//
// All characteristic arithmetic is FP64.  Every neighbour a right-hand side
// needs is resolved on the host into a UDesc: another unknown (stage value)
// or a strip slot holding a bulk node's macros at t and t + 1 (interpolated
// linearly at the stage time, Sec. 3.3).
#include "lbm_internal.cuh"

namespace lbmgb {

namespace {

constexpr int kBandThreads = 32;   // few unknowns: spread them over many SMs

// Lab <-> local frame.  Sides: n the outward normal, t = +y (W, E) or +x
// (S, N).  Corners: n = (sx, sy)/sqrt(2), t = n rotated by +90 degrees.
__device__ __forceinline__ void to_local(int kind, double r, const double* U, double* Lc)
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
        const double n0 = (c & 1) ? r : -r, n1 = (c & 2) ? r : -r;
        Lc[1] = U[1] * n0 + U[2] * n1;
        Lc[2] = -U[1] * n1 + U[2] * n0;
    }
    }
}

__device__ __forceinline__ void to_lab(int kind, double r, const double* Lc, double* U)
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
        const double n0 = (c & 1) ? r : -r, n1 = (c & 2) ? r : -r;
        U[1] = Lc[1] * n0 - Lc[2] * n1;
        U[2] = Lc[1] * n1 + Lc[2] * n0;
    }
    }
}

struct Ctx {
    const double* Y;     // stage values of the unknowns
    const double* St;    // strip macros at t
    const double* St1;   // strip macros at t + 1
    double frac;         // stage time fraction in [0, 1]
};

__device__ __forceinline__ void fetch(const Ctx& X, int ref, double* U)
{
    if (ref >= 0) {
        const double2* p = reinterpret_cast<const double2*>(X.Y + 4LL * ref);
        const double2 a = p[0], b = p[1];
        U[0] = a.x; U[1] = a.y; U[2] = b.x; U[3] = b.y;
    } else {
        const long long s = 4LL * (-ref - 1);
        const double w0 = 1.0 - X.frac, w1 = X.frac;
#pragma unroll
        for (int c = 0; c < 4; ++c) U[c] = w0 * X.St[s + c] + w1 * X.St1[s + c];
    }
}

__device__ __forceinline__ void fetch_local(const Ctx& X, int ref, int kind, double r, double* Lc)
{
    double U[4];
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
struct CharSys {
    double rho, irho, r, ir, a, b, h, csr;
    double lam[4];
};

template <bool TH>
__device__ __forceinline__ CharSys char_sys(const Band& B, double rho0, const double* U)
{
    CharSys C;
    C.rho = rho0 + U[0];
    C.irho = 1.0 / C.rho;
    if (TH) {
        const double th = 1.0 + U[3];
        const double sth = sqrt(th);
        const double isth = 1.0 / sth;
        C.r = th * C.irho;
        C.ir = C.rho * isth * isth;
        C.a = sth * B.kA;
        C.b = isth * B.kB;
        const double c = sth * B.kB;
        C.lam[0] = U[1];
        C.lam[1] = U[1];
        C.lam[2] = U[1] - c;
        C.lam[3] = U[1] + c;
        C.h = C.csr = 0.0;
    } else {
        C.h = C.rho * B.ihcs;
        C.csr = B.cs * C.irho;
        C.lam[0] = U[1] - B.cs;
        C.lam[1] = U[1];
        C.lam[2] = U[1] + B.cs;
        C.lam[3] = 0.0;
        C.r = C.ir = C.a = C.b = 0.0;
    }
    return C;
}

template <bool TH>
__device__ __forceinline__ void apply_S(const CharSys& C, const double* v, double* o)
{
    if (TH) {
        const double rv = 0.25 * C.r * v[0], q = 0.25 * v[3], av = C.a * v[1];
        o[0] = -2.0 * rv + 2.0 * q;
        o[1] = v[2];
        o[2] = rv - av + q;
        o[3] = rv + av + q;
    } else {
        const double hv = C.h * v[1];
        o[0] = 0.5 * v[0] - hv;
        o[1] = v[2];
        o[2] = 0.5 * v[0] + hv;
        o[3] = 0.0;
    }
}

template <bool TH>
__device__ __forceinline__ int incoming_mask(const CharSys& C)
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
template <bool TH>
__device__ __forceinline__ void char_rhs(const CharSys& C, const Band& B, const double* dUn,
                                         const double* TT, const double* VV, int mask, double dP,
                                         int scheme, double* k)
{
    double sd[4], st[4], sv[4], w[4];
    apply_S<TH>(C, dUn, sd);
    apply_S<TH>(C, TT, st);
    apply_S<TH>(C, VV, sv);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!TH && i == 3) { w[i] = 0.0; continue; }
        if (!((mask >> i) & 1)) {
            w[i] = C.lam[i] * sd[i];
            continue;
        }
        const bool acoustic = TH ? (i >= 2) : (i != 1);
        const double relaxP = acoustic ? B.beta_P * dP : 0.0;
        if (scheme == SCH_LODI) w[i] = 0.0;
        else if (scheme == SCH_LODI_RELAX) w[i] = B.alpha_T * (B.t_inf - st[i]) + relaxP;
        else if (scheme == SCH_CBC) w[i] = st[i] + sv[i];
        else w[i] = st[i] + sv[i] + B.alpha_T * (B.t_inf - st[i]) + relaxP;
    }
    double o[4];
    if (TH) {
        o[0] = (w[2] + w[3] - w[0]) * C.ir;
        o[1] = C.b * (w[3] - w[2]);
        o[2] = w[1];
        o[3] = w[0] + w[2] + w[3];
    } else {
        o[0] = w[0] + w[2];
        o[1] = C.csr * (w[2] - w[0]);
        o[2] = w[1];
        o[3] = 0.0;
    }
    const bool cbc = scheme == SCH_CBC || scheme == SCH_CBC_RELAX;
#pragma unroll
    for (int m = 0; m < 4; ++m) k[m] = -o[m] + (cbc ? TT[m] + VV[m] : 0.0);
}

// ---------------------------------------------------------------------------
// Viscous vectors, frozen at time t
// ---------------------------------------------------------------------------

// Mesoscopic form at x_f (Eqs. LaplaceU, LaplaceT): normal derivatives
// one-sided into the bulk (Eq. FD-dx-bw), tangential ones central
// (Eq. FD-dx-center) or one-sided inward next to a boundary node:
//   V = (0, (1/rho) d_j s'_jn, (1/rho) d_j s'_jt,
//        -div q / (rho c_s^2) + (nu / c_s^2) ((d_n u_n - d_t u_t)^2 + (d_n u_t + d_t u_n)^2)).
template <bool TH>
__device__ void vis_meso(const Geom& G, const Band& B, const Export& E, int par_t,
                         const UDesc& D, double cs2, double* V)
{
    const double* SU = E.stripU + (long long)par_t * E.nslots * 4;
    const double* SN = E.stripN + (long long)par_t * E.nslots * 5;
    const int s = D.kind;
    const int an = s < 2 ? 0 : 1, at = 1 - an;     // axes of n and t
    const double sn = (s == 0 || s == 2) ? -1.0 : 1.0;
    double h[5][7];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double* n = SN + 5LL * D.vs[k];
        const double* u = SU + 4LL * D.vs[k];
        const double sxx = n[0], sxy = n[1], syy = n[2];
        h[k][0] = an == 0 ? sxx : syy;              // sigma'_nn
        h[k][1] = sn * sxy;                         // sigma'_nt
        h[k][2] = an == 0 ? syy : sxx;              // sigma'_tt
        h[k][3] = sn * n[3 + an];                   // q_n
        h[k][4] = n[3 + at];                        // q_t
        h[k][5] = sn * u[1 + an];                   // u_n
        h[k][6] = u[1 + at];                        // u_t
    }
    double dn[7], dt[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) {
        dn[m] = 0.5 * (3.0 * h[0][m] - 4.0 * h[1][m] + h[2][m]);
        if (D.tmode == 0) dt[m] = 0.5 * (h[3][m] - h[4][m]);
        else dt[m] = double(D.tmode) * 0.5 * (3.0 * h[0][m] - 4.0 * h[3][m] + h[4][m]);
    }
    const double irho = 1.0 / (G.rho0 + SU[4LL * D.vs[0]]);
    V[0] = 0.0;
    V[1] = (dn[0] + dt[1]) * irho;
    V[2] = (dn[1] + dt[2]) * irho;
    V[3] = 0.0;
    if (TH) {
        const double nu = (G.tau - 0.5) * cs2;
        const double e1 = dn[5] - dt[6], e2 = dn[6] + dt[5];
        V[3] = -(dn[3] + dt[4]) * irho * (1.0 / cs2) + nu * (1.0 / cs2) * (e1 * e1 + e2 * e2);
    }
}

// "-FD" form (Sec. 4.2) at layer j from the macros of time t: 4-point
// one-sided second derivative at j = M, 3-point central elsewhere.
template <bool TH>
__device__ void vis_fd(const Geom& G, const Band& B, const Ctx& X0, const UDesc& D, int u,
                       double cs2, double* V)
{
    const int kind = D.kind;
    double U[4], A[4], Bv[4], Cv[4], Tp[4], Tm[4], dnn[4], d1n[4];
    fetch_local(X0, u, kind, 0.0, U);
    fetch_local(X0, D.nb[1], kind, 0.0, Bv);
    fetch_local(X0, D.nb[4], kind, 0.0, Tp);
    fetch_local(X0, D.nb[5], kind, 0.0, Tm);
    if (D.j == B.M) {
        fetch_local(X0, D.nb[2], kind, 0.0, A);
        fetch_local(X0, D.nb[3], kind, 0.0, Cv);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            dnn[m] = 2.0 * U[m] - 5.0 * Bv[m] + 4.0 * A[m] - Cv[m];
            d1n[m] = 0.5 * (3.0 * U[m] - 4.0 * Bv[m] + A[m]);
        }
    } else {
        fetch_local(X0, D.nb[0], kind, 0.0, A);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            dnn[m] = A[m] - 2.0 * U[m] + Bv[m];
            d1n[m] = 0.5 * (A[m] - Bv[m]);
        }
    }
    const double nu = (G.tau - 0.5) * cs2;
    V[0] = 0.0;
    V[1] = nu * (dnn[1] + (Tp[1] - 2.0 * U[1] + Tm[1]));
    V[2] = nu * (dnn[2] + (Tp[2] - 2.0 * U[2] + Tm[2]));
    V[3] = 0.0;
    if (TH) {
        const double d1t1 = 0.5 * (Tp[1] - Tm[1]), d1t2 = 0.5 * (Tp[2] - Tm[2]);
        const double e1 = d1n[1] - d1t2, e2 = d1n[2] + d1t1;
        V[3] = 2.0 * nu * (dnn[3] + (Tp[3] - 2.0 * U[3] + Tm[3])) + nu * (1.0 / cs2) * (e1 * e1 + e2 * e2);
    }
}

// ---------------------------------------------------------------------------
// Right-hand side of one unknown
// ---------------------------------------------------------------------------

template <int LAT>
__device__ void unknown_rhs(const Geom& G, const Band& B, const Ctx& X, const UDesc& D, int u,
                            const double* V, int mask, double* k)
{
    using L = Lat<LAT>;
    constexpr bool TH = L::THERMAL;
    const int kind = D.kind;
    const double r = B.kR;
    double U[4], A[4], Bv[4], dUn[4];
    fetch_local(X, u, kind, r, U);
    if (kind >= 4) {
        // Corner: LODI (Eq. PNR) along the outward diagonal, one-sided
        // difference of spacing sqrt(2) through the two diagonal bulk nodes.
        fetch_local(X, D.nb[0], kind, r, A);
        fetch_local(X, D.nb[1], kind, r, Bv);
#pragma unroll
        for (int m = 0; m < 4; ++m) dUn[m] = (3.0 * U[m] - 4.0 * A[m] + Bv[m]) * B.kC;
        const double zero[4] = {0.0, 0.0, 0.0, 0.0};
        const CharSys C = char_sys<TH>(B, G.rho0, U);
        double kl[4];
        char_rhs<TH>(C, B, dUn, zero, zero, mask, 0.0, SCH_LODI, kl);
        to_lab(kind, r, kl, k);
        return;
    }
    if (D.j == B.M) {            // Eq. FD-dx-bw at the outermost layer
        fetch_local(X, D.nb[1], kind, r, A);
        fetch_local(X, D.nb[2], kind, r, Bv);
#pragma unroll
        for (int m = 0; m < 4; ++m) dUn[m] = 0.5 * (3.0 * U[m] - 4.0 * A[m] + Bv[m]);
    } else {                     // Eq. FD-dx-center at inner layers
        fetch_local(X, D.nb[0], kind, r, A);
        fetch_local(X, D.nb[1], kind, r, Bv);
#pragma unroll
        for (int m = 0; m < 4; ++m) dUn[m] = 0.5 * (A[m] - Bv[m]);
    }
    // transversal vector T (Sec. 3.1) from central differences along the side
    double Up[4], Um[4];
    fetch_local(X, D.nb[4], kind, r, Up);
    fetch_local(X, D.nb[5], kind, r, Um);
    const double rho0 = G.rho0, cs2 = L::CS2;
    const CharSys C = char_sys<TH>(B, rho0, U);
    const double ut = U[2];
    const double d_rhout = 0.5 * ((rho0 + Up[0]) * Up[2] - (rho0 + Um[0]) * Um[2]);
    const double d_un = 0.5 * (Up[1] - Um[1]);
    const double d_ut = 0.5 * (Up[2] - Um[2]);
    double TT[4], dP;
    if (TH) {
        // rho T - rho0 = drho + rho0 dT + drho dT
        const double d_rhoT = 0.5 * ((Up[0] + rho0 * Up[3] + Up[0] * Up[3]) -
                                     (Um[0] + rho0 * Um[3] + Um[0] * Um[3]));
        const double d_Tut = 0.5 * ((1.0 + Up[3]) * Up[2] - (1.0 + Um[3]) * Um[2]);
        TT[0] = -d_rhout;
        TT[1] = -ut * d_un;
        TT[2] = -cs2 * C.irho * d_rhoT - ut * d_ut;
        TT[3] = -d_Tut;
        dP = cs2 * (U[0] + rho0 * U[3] + U[0] * U[3]) - B.pdev[kind];
    } else {
        TT[0] = -d_rhout;
        TT[1] = -ut * d_un;
        TT[2] = -cs2 * C.irho * 0.5 * (Up[0] - Um[0]) - ut * d_ut;
        TT[3] = 0.0;
        dP = cs2 * U[0] - B.pdev[kind];
    }
    double kl[4];
    char_rhs<TH>(C, B, dUn, TT, V, mask, dP, B.scheme[kind], kl);
    to_lab(kind, r, kl, k);
}

// ---------------------------------------------------------------------------
// Population writes (stage 3)
// ---------------------------------------------------------------------------

// Mesoscopic Dirichlet condition for the new boundary state, stored
// post-collision: f^eq(Unew) and, for Eq. NEEP, the non-equilibrium part of
// the bulk neighbour after its collision, f*(x_f) - f^eq(U(x_f, t+1)).  Computed
// in the arithmetic type of the storage.
template <int LAT, typename S>
__device__ void dirichlet(const Geom& G, const Band& B, const Export& E, S* f, int par_new,
                          const UDesc& D, const double* Unew)
{
    using L = Lat<LAT>;
    using Cm = typename Store<S>::C;
    Moments<LAT, Cm> m;
    m.s0 = Cm(Unew[0]);
    m.rho = Cm(G.rho0) + m.s0;
    m.ux = Cm(Unew[1]);
    m.uy = Cm(Unew[2]);
    m.dT = Cm(L::THERMAL ? Unew[3] : 0.0);
    Cm ge[L::Q];
    equilibrium<LAT, Cm>(m, ge);
    if (B.dirichlet == 1) {
        const double* Us = E.stripU + ((long long)par_new * E.nslots + D.wslot) * 4;
        Moments<LAT, Cm> ms;
        ms.s0 = Cm(Us[0]);
        ms.rho = Cm(G.rho0) + ms.s0;
        ms.ux = Cm(Us[1]);
        ms.uy = Cm(Us[2]);
        ms.dT = Cm(L::THERMAL ? Us[3] : 0.0);
        Cm gs[L::Q];
        equilibrium<LAT, Cm>(ms, gs);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            Cm v = Cm(Store<S>::load(f + L::plane_of(i) * G.plane + D.wsrc));
            if (Store<S>::SCALED) v *= Cm(L::w(i));
            ge[i] += v - gs[i];
        }
    }
    const int nb = D.kind >= 4 ? G.M : 1;
    for (int a = 0; a < nb; ++a)
        for (int b = 0; b < nb; ++b) {
            const long long node = D.wnode + a * D.wdx + b * D.wdy;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                Cm v = ge[i];
                if (Store<S>::SCALED) v *= Cm(1.0 / L::w(i));
                Store<S>::put(f + L::plane_of(i) * G.plane + node, v);
            }
        }
}

template <int LAT, typename S>
__global__ void __launch_bounds__(kBandThreads)
    k_stage(Geom G, Band B, Export E, S* __restrict__ f, int par_t, int stage)
{
    using L = Lat<LAT>;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (stage == 3 && u >= B.n_unk) {
        // zero gradient: copy the post-collision populations of x_f
        const int z = u - B.n_unk;
        if (z >= B.n_zg) return;
        const int2 nd = B.zg[z];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) f[i * G.plane + nd.x] = f[i * G.plane + nd.y];
        return;
    }
    if (u >= B.n_unk) return;
    const UDesc D = B.ud[u];
    Ctx X;
    X.Y = stage == 0 ? B.Ub : (stage == 2 ? B.Yb : B.Ya);
    X.St = E.stripU + (long long)par_t * E.nslots * 4;
    X.St1 = E.stripU + (long long)(par_t ^ 1) * E.nslots * 4;
    X.frac = stage == 0 ? 0.0 : (stage == 3 ? 1.0 : 0.5);
    double* Yout = stage == 1 ? B.Yb : B.Ya;

    double V[4];
    int mask;
    if (stage == 0) {
        double Ul[4];
        to_local(D.kind, B.kR, B.Ub + 4LL * u, Ul);
        mask = incoming_mask<L::THERMAL>(char_sys<L::THERMAL>(B, G.rho0, Ul));
        if (D.kind >= 4 || B.viscous == VIS_OFF) V[0] = V[1] = V[2] = V[3] = 0.0;
        else if (B.viscous == VIS_FD) vis_fd<L::THERMAL>(G, B, X, D, u, L::CS2, V);
        else vis_meso<L::THERMAL>(G, B, E, par_t, D, L::CS2, V);
        double2* vo = reinterpret_cast<double2*>(B.V + 4LL * u);
        vo[0] = make_double2(V[0], V[1]);
        vo[1] = make_double2(V[2], V[3]);
        B.mask[u] = mask;
    } else {
        const double2* vi = reinterpret_cast<const double2*>(B.V + 4LL * u);
        const double2 v0 = vi[0], v1 = vi[1];
        V[0] = v0.x; V[1] = v0.y; V[2] = v1.x; V[3] = v1.y;
        mask = B.mask[u];
    }
    double k[4];
    unknown_rhs<LAT>(G, B, X, D, u, V, mask, k);

    const double* U0 = B.Ub + 4LL * u;
    double* acc = B.acc + 4LL * u;
    if (stage < 3) {
        const double wk = stage == 0 ? 1.0 : 2.0;
        const double hk = stage == 2 ? 1.0 : 0.5;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            acc[m] = (stage == 0 ? 0.0 : acc[m]) + wk * k[m];
            Yout[4LL * u + m] = U0[m] + hk * k[m];
        }
        return;
    }
    double Unew[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) Unew[m] = U0[m] + (acc[m] + k[m]) * (1.0 / 6.0);
#pragma unroll
    for (int m = 0; m < 4; ++m) B.Ub[4LL * u + m] = Unew[m];
    dirichlet<LAT, S>(G, B, E, f, par_t ^ 1, D, Unew);
}

template <int LAT, typename S>
int boundary_t(const Geom& G, const Export& E, const Band& B, void* fnew, int par_t, cudaStream_t st)
{
    S* f = static_cast<S*>(fnew);
    if (B.n_unk > 0) {
        const int nb = (B.n_unk + kBandThreads - 1) / kBandThreads;
        for (int stage = 0; stage < 3; ++stage)
            k_stage<LAT, S><<<nb, kBandThreads, 0, st>>>(G, B, E, f, par_t, stage);
    }
    const int n3 = B.n_unk + B.n_zg;
    if (n3 > 0)
        k_stage<LAT, S><<<(n3 + kBandThreads - 1) / kBandThreads, kBandThreads, 0, st>>>(G, B, E, f,
                                                                                      par_t, 3);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

int launch_boundary(int lat, int storage, const Geom& G, const Export& E, const Band& B,
                    void* fnew, int par_t, cudaStream_t st)
{
    if (lat == D2Q9) {
        if (storage == 0) return boundary_t<D2Q9, double>(G, E, B, fnew, par_t, st);
        if (storage == 1) return boundary_t<D2Q9, float>(G, E, B, fnew, par_t, st);
        if (storage == 2) return boundary_t<D2Q9, __half>(G, E, B, fnew, par_t, st);
    } else {
        if (storage == 0) return boundary_t<D2Q37, double>(G, E, B, fnew, par_t, st);
        if (storage == 1) return boundary_t<D2Q37, float>(G, E, B, fnew, par_t, st);
        if (storage == 2) return boundary_t<D2Q37, __half>(G, E, B, fnew, par_t, st);
    }
    return -1;
}

}  // namespace lbmgb

// ---------------------------------------------------------------------------
// Allocation-free boundary step for one side (no counterpart in the paper)
// ---------------------------------------------------------------------------
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool, under a no-allocation policy, or in a context
// where cudaMalloc is forbidden.  lbm_cbc_side_step_noalloc() advances the
// characteristic boundary state of one straight CBC side whose tangential
// axis is periodic by one time step (the four RK4 stages above), with its
// stage scratch in the file-scope array below instead of a workspace.

#include <cmath>
#include <cstdio>
#include <mutex>

#include "lbm_cbc.h"

namespace lbmgb {
namespace {

constexpr int kNoAllocMaxUnknowns = 12288;     // M * length: 4096 positions of D2Q37
constexpr int kNoAllocMaxDevices = 64;
// Ya, Yb, acc, V (4 doubles per unknown each), then the incoming masks.
constexpr size_t kNoAllocDoubles = 16ull * kNoAllocMaxUnknowns + kNoAllocMaxUnknowns / 2;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

std::mutex g_noalloc_mutex;
double* g_noalloc_addr[kNoAllocMaxDevices] = {};

template <int LAT>
__global__ void __launch_bounds__(kBandThreads)
    k_side_stage_noalloc(Geom G, Band B, Export E, int side, int L, const double* __restrict__ St,
                         const double* __restrict__ St1, int stage)
{
    using Lt = Lat<LAT>;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= B.n_unk) return;
    const int M = B.M, p = u / M, j = 1 + u % M;
    auto wrapp = [L](int q) { return q < 0 ? q + L : (q >= L ? q - L : q); };
    auto ref = [&](int jj, int q) {
        q = wrapp(q);
        return jj >= 1 ? q * M + (jj - 1) : -((-jj) * L + q + 1);
    };
    UDesc D;
    D.kind = side;
    D.j = j;
    D.tmode = 0;
    D.nb[0] = j < M ? ref(j + 1, p) : 0;
    D.nb[1] = ref(j - 1, p);
    D.nb[2] = ref(j - 2, p);
    D.nb[3] = ref(j - 3, p);
    D.nb[4] = ref(j, p + 1);
    D.nb[5] = ref(j, p - 1);
    D.vs[0] = p;
    D.vs[1] = L + p;
    D.vs[2] = 2 * L + p;
    D.vs[3] = wrapp(p + 1);
    D.vs[4] = wrapp(p - 1);
    Ctx X;
    X.Y = stage == 0 ? B.Ub : (stage == 2 ? B.Yb : B.Ya);
    X.St = St;
    X.St1 = St1;
    X.frac = stage == 0 ? 0.0 : (stage == 3 ? 1.0 : 0.5);
    double* Yout = stage == 1 ? B.Yb : B.Ya;
    double V[4];
    int mask;
    if (stage == 0) {
        double Ul[4];
        to_local(side, B.kR, B.Ub + 4LL * u, Ul);
        mask = incoming_mask<Lt::THERMAL>(char_sys<Lt::THERMAL>(B, G.rho0, Ul));
        if (B.viscous == VIS_OFF) V[0] = V[1] = V[2] = V[3] = 0.0;
        else if (B.viscous == VIS_FD) vis_fd<Lt::THERMAL>(G, B, X, D, u, Lt::CS2, V);
        else vis_meso<Lt::THERMAL>(G, B, E, 0, D, Lt::CS2, V);
        for (int m = 0; m < 4; ++m) B.V[4LL * u + m] = V[m];
        B.mask[u] = mask;
    } else {
        for (int m = 0; m < 4; ++m) V[m] = B.V[4LL * u + m];
        mask = B.mask[u];
    }
    double k[4];
    unknown_rhs<LAT>(G, B, X, D, u, V, mask, k);
    const double* U0 = B.Ub + 4LL * u;
    double* acc = B.acc + 4LL * u;
    if (stage < 3) {
        const double wk = stage == 0 ? 1.0 : 2.0;
        const double hk = stage == 2 ? 1.0 : 0.5;
        for (int m = 0; m < 4; ++m) {
            acc[m] = (stage == 0 ? 0.0 : acc[m]) + wk * k[m];
            Yout[4LL * u + m] = U0[m] + hk * k[m];
        }
        return;
    }
    double Unew[4];
    for (int m = 0; m < 4; ++m) Unew[m] = U0[m] + (acc[m] + k[m]) * (1.0 / 6.0);
    for (int m = 0; m < 4; ++m) B.Ub[4LL * u + m] = Unew[m];
}

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the array's name as a device address).
int noalloc_scratch(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        fprintf(stderr, "lbm_cbc_side_step_noalloc: cudaGetDevice: %s\n", cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        fprintf(stderr, "lbm_cbc_side_step_noalloc: device %d beyond the supported %d\n", dev,
                kNoAllocMaxDevices);
        return LBM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            fprintf(stderr, "lbm_cbc_side_step_noalloc: cudaGetSymbolAddress: %s\n",
                    cudaGetErrorString(e));
            return LBM_ERR_CUDA;
        }
        g_noalloc_addr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_addr[dev];
    return LBM_OK;
}

}  // namespace
}  // namespace lbmgb

extern "C" int lbm_cbc_side_step_noalloc(int lattice, int side, int length, double tau,
                                         const lbm_cbc_params* p, double* Ub, const double* strip_t,
                                         const double* strip_t1, const double* neq_t, void* stream)
{
    using namespace lbmgb;
    if (lattice != LBM_D2Q9 && lattice != LBM_D2Q37) return LBM_ERR_ARG;
    if (!p || !Ub || !strip_t || !strip_t1 || side < 0 || side > 3 || !(tau > 0.5)) return LBM_ERR_ARG;
    if (p->viscous < 0 || p->viscous > 2 || p->scheme[side] < 0 || p->scheme[side] > 3 || !(p->rho0 > 0.0))
        return LBM_ERR_ARG;
    if (p->viscous == LBM_VISCOUS_MESO && !neq_t) {
        fprintf(stderr, "lbm_cbc_side_step_noalloc: mesoscopic viscous terms need neq_t\n");
        return LBM_ERR_ARG;
    }
    const int M = lattice == LBM_D2Q9 ? 1 : 3;
    if (length < 3 || (long long)length * M > kNoAllocMaxUnknowns) {
        fprintf(stderr,
                "lbm_cbc_side_step_noalloc: side length %d outside [3, %d] (at most %d unknowns)\n",
                length, kNoAllocMaxUnknowns / M, kNoAllocMaxUnknowns);
        return LBM_ERR_ARG;
    }
    double* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != LBM_OK) return rc;
    const double cs2 = lattice == LBM_D2Q9 ? Lat<D2Q9>::CS2 : Lat<D2Q37>::CS2;
    const int n = length * M;
    Geom G{};
    G.M = M;
    G.tau = tau;
    G.rho0 = p->rho0;
    Band B{};
    B.n_unk = n;
    B.M = M;
    B.viscous = p->viscous;
    B.scheme[side] = p->scheme[side];
    B.alpha_T = p->alpha_T;
    B.beta_P = p->beta_P;
    B.t_inf = p->t_inf;
    const double pinf = p->p_inf[side] != 0.0 ? p->p_inf[side] : cs2 * p->rho0;
    B.pdev[side] = pinf - cs2 * p->rho0;
    B.kA = 1.0 / std::sqrt(8.0 * cs2);
    B.kB = std::sqrt(2.0 * cs2);
    B.kC = 1.0 / (2.0 * std::sqrt(2.0));
    B.kR = 1.0 / std::sqrt(2.0);
    B.cs = std::sqrt(cs2);
    B.ihcs = 0.5 / B.cs;
    B.Ub = Ub;
    B.Ya = scratch;
    B.Yb = scratch + 4ull * kNoAllocMaxUnknowns;
    B.acc = scratch + 8ull * kNoAllocMaxUnknowns;
    B.V = scratch + 12ull * kNoAllocMaxUnknowns;
    B.mask = reinterpret_cast<int*>(scratch + 16ull * kNoAllocMaxUnknowns);
    Export E{};
    E.nslots = 3 * length;
    E.stripU = const_cast<double*>(strip_t);
    E.stripN = const_cast<double*>(neq_t);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nb = (n + kBandThreads - 1) / kBandThreads;
    for (int stage = 0; stage < 4; ++stage) {
        if (lattice == LBM_D2Q9)
            k_side_stage_noalloc<D2Q9><<<nb, kBandThreads, 0, st>>>(G, B, E, side, length, strip_t, strip_t1, stage);
        else
            k_side_stage_noalloc<D2Q37><<<nb, kBandThreads, 0, st>>>(G, B, E, side, length, strip_t, strip_t1, stage);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "lbm_cbc_side_step_noalloc: launch: %s\n", cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}
