// boundary.cu -- boundary conditions of one time step.
//
//  k_cbc_stage  one RK4 stage (Sec. 3.3, "Time integration") of the boundary
//               ODE on every characteristic unknown: each of the M layers of
//               every CBC side position and the innermost node of each corner
//               block.  Stage 0 also freezes the viscous vector and the
//               incoming-wave mask of time t; stage 3 finishes the step and
//               writes the mesoscopic Dirichlet populations (equilibrium or
//               Eq. NEEP), post-collision, into the new population buffer.
//  k_extras     zero gradient (Eq. zg-bc) and inflow-equilibrium nodes.
//
// All boundary arithmetic is FP64: the characteristic decomposition works on
// small gradients of O(1) states.  Bulk macros at stage times come from the
// strips the bulk kernel exported (time t and t+1), interpolated linearly.
#include "lbm_internal.cuh"

namespace lbmgb {

namespace {

constexpr int kBandThreads = 32;   // few unknowns: spread them over many SMs

struct Frame {
    double n0, n1, t0, t1;
};

__device__ inline Frame frame_of_side(int s)
{
    return Frame{double(side_nx(s)), double(side_ny(s)), double(side_tx(s)), double(side_ty(s))};
}

// Corner blocks: outward diagonal n = (sx, sy)/sqrt(2), t = n rotated by +90.
__device__ inline Frame frame_of_corner(int c)
{
    const double r = 1.0 / sqrt(2.0);
    const double n0 = corner_sx(c) * r, n1 = corner_sy(c) * r;
    return Frame{n0, n1, -n1, n0};
}

__device__ inline void to_local(const double* U, const Frame& F, double* Lc)
{
    Lc[0] = U[0];
    Lc[1] = U[1] * F.n0 + U[2] * F.n1;
    Lc[2] = U[1] * F.t0 + U[2] * F.t1;
    Lc[3] = U[3];
}

__device__ inline void to_lab(const double* Lc, const Frame& F, double* U)
{
    U[0] = Lc[0];
    U[1] = Lc[1] * F.n0 + Lc[2] * F.t0;
    U[2] = Lc[1] * F.n1 + Lc[2] * F.t1;
    U[3] = Lc[3];
}

// Corner block met at the low / high tangential end of a side.
__device__ inline int lo_corner(int s) { return s == 3 ? 2 : (s == 1 ? 1 : 0); }
__device__ inline int hi_corner(int s) { return s == 2 ? 1 : (s == 0 ? 2 : 3); }

// Stage value of layer j (j >= 1: boundary unknown; j <= 0: bulk node at
// depth -j, interpolated between t and t+1) at tangential position p.
__device__ inline void fetch(const Geom& G, const Band& B, const double* Y, int par_t, double frac,
                             int s, int j, int p, double U[4])
{
    const Side& S = B.s[s];
    if (S.tper) {
        p %= S.L;
        if (p < 0) p += S.L;
    }
    if (j >= 1) {
        const double* src;
        if (p < S.lo) src = Y + 4LL * (B.n_side_unk + lo_corner(s));
        else if (p > S.hi) src = Y + 4LL * (B.n_side_unk + hi_corner(s));
        else src = Y + 4LL * (S.base + (p - S.lo) * G.M + (j - 1));
#pragma unroll
        for (int c = 0; c < 4; ++c) U[c] = src[c];
    } else {
        const double* a = B.stripU + strip_u_index(S, par_t, -j, p);
        const double* b = B.stripU + strip_u_index(S, par_t ^ 1, -j, p);
#pragma unroll
        for (int c = 0; c < 4; ++c) U[c] = (1.0 - frac) * a[c] + frac * b[c];
    }
}

__device__ inline void fetch_local(const Geom& G, const Band& B, const double* Y, int par_t,
                                   double frac, int s, int j, int p, const Frame& F, double Lc[4])
{
    double U[4];
    fetch(G, B, Y, par_t, frac, s, j, p, U);
    to_local(U, F, Lc);
}

// ---------------------------------------------------------------------------
// Characteristic right-hand side in the local frame (Sec. 3.1, 3.2)
// ---------------------------------------------------------------------------

// Thermal system, U = (drho, u_n, u_t, dT), T~ = c_s^2 (1 + dT):
//   S = [[-T~/(2 rho c_s^2), 0, 0, 1/2], [0, 0, 1, 0],
//        [T~/(4 rho c_s^2), -sqrt(T~/(8 c_s^4)), 0, 1/4],
//        [T~/(4 rho c_s^2),  sqrt(T~/(8 c_s^4)), 0, 1/4]],
//   Lambda = (u_n, u_n, u_n - sqrt(2 T~), u_n + sqrt(2 T~)).
// The isothermal D2Q9 system for (drho, u_n, u_t) has
//   S = [[1/2, -rho/(2 c_s), 0], [0, 0, 1], [1/2, rho/(2 c_s), 0]],
//   Lambda = (u_n - c_s, u_n, u_n + c_s).
struct CharSys {
    bool th;
    double r, a, b, cs, rho;
    double lam[4];
};

__device__ inline CharSys char_sys(bool th, double cs2, double rho0, const double U[4])
{
    CharSys C;
    C.th = th;
    C.rho = rho0 + U[0];
    if (th) {
        const double theta = 1.0 + U[3];
        C.r = theta / C.rho;                      // T~ / (rho c_s^2)
        C.a = sqrt(theta / (8.0 * cs2));          // sqrt(T~ / (8 c_s^4))
        C.b = sqrt(2.0 * cs2 / theta);            // sqrt(2 c_s^4 / T~)
        const double c = sqrt(2.0 * cs2 * theta); // sqrt(2 T~)
        C.lam[0] = U[1];
        C.lam[1] = U[1];
        C.lam[2] = U[1] - c;
        C.lam[3] = U[1] + c;
        C.cs = 0.0;
    } else {
        C.cs = sqrt(cs2);
        C.r = C.a = C.b = 0.0;
        C.lam[0] = U[1] - C.cs;
        C.lam[1] = U[1];
        C.lam[2] = U[1] + C.cs;
        C.lam[3] = 0.0;
    }
    return C;
}

__device__ inline void apply_S(const CharSys& C, const double v[4], double o[4])
{
    if (C.th) {
        o[0] = -0.5 * C.r * v[0] + 0.5 * v[3];
        o[1] = v[2];
        o[2] = 0.25 * C.r * v[0] - C.a * v[1] + 0.25 * v[3];
        o[3] = 0.25 * C.r * v[0] + C.a * v[1] + 0.25 * v[3];
    } else {
        const double h = C.rho / (2.0 * C.cs);
        o[0] = 0.5 * v[0] - h * v[1];
        o[1] = v[2];
        o[2] = 0.5 * v[0] + h * v[1];
        o[3] = 0.0;
    }
}

__device__ inline void apply_Sinv(const CharSys& C, const double w[4], double o[4])
{
    if (C.th) {
        o[0] = (w[2] + w[3] - w[0]) / C.r;
        o[1] = C.b * (w[3] - w[2]);
        o[2] = w[1];
        o[3] = w[0] + w[2] + w[3];
    } else {
        o[0] = w[0] + w[2];
        o[1] = C.cs / C.rho * (w[2] - w[0]);
        o[2] = w[1];
        o[3] = 0.0;
    }
}

__device__ inline int incoming_mask(const CharSys& C)
{
    const int n = C.th ? 4 : 3;
    int m = 0;
    for (int i = 0; i < n; ++i)
        if (C.lam[i] < 0.0) m |= 1 << i;
    return m;
}

// dU/dt = -S^-1 Lbar (+ T + V for the CBC schemes) with Lbar_i = L_i =
// Lambda_i (S dU/dn)_i for outgoing waves (Eq. thermal_WAV) and, for
// incoming waves, Eq. PNR (LODI), Eq. LODI-Relax, Eq. CBC-PNR (CBC) or
// Eq. CBC-Relax.  beta (Z - Z_inf) acts on incoming acoustic waves.
__device__ inline void char_rhs(const CharSys& C, const Band& B, const double dUn[4],
                                const double TT[4], const double VV[4], int mask, double dP,
                                int scheme, double k[4])
{
    double sd[4], st[4], sv[4], w[4];
    apply_S(C, dUn, sd);
    apply_S(C, TT, st);
    apply_S(C, VV, sv);
    const int n = C.th ? 4 : 3;
    for (int i = 0; i < 4; ++i) w[i] = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!((mask >> i) & 1)) {
            w[i] = C.lam[i] * sd[i];
            continue;
        }
        const bool acoustic = C.th ? (i >= 2) : (i != 1);
        const double relaxP = acoustic ? B.beta_P * dP : 0.0;
        if (scheme == SCH_LODI) w[i] = 0.0;
        else if (scheme == SCH_LODI_RELAX) w[i] = B.alpha_T * (B.t_inf - st[i]) + relaxP;
        else if (scheme == SCH_CBC) w[i] = st[i] + sv[i];
        else w[i] = st[i] + sv[i] + B.alpha_T * (B.t_inf - st[i]) + relaxP;
    }
    double o[4];
    apply_Sinv(C, w, o);
    const bool cbc = scheme == SCH_CBC || scheme == SCH_CBC_RELAX;
    for (int m = 0; m < 4; ++m) k[m] = -o[m] + (cbc ? TT[m] + VV[m] : 0.0);
}

// ---------------------------------------------------------------------------
// Viscous vectors (frozen at time t)
// ---------------------------------------------------------------------------

// Mesoscopic form at x_f of side s, position p, from the non-equilibrium
// moments the bulk kernel exported: normal derivatives one-sided into the
// bulk (Eq. FD-dx-bw), tangential ones central (Eq. FD-dx-center), and
// one-sided inward where the tangential neighbour is a boundary node.
//   V = (0, (1/rho) d_j s'_jn, (1/rho) d_j s'_jt,
//        (-div q + heating) / (rho c_s^2)),
//   heating = rho nu ((d_n u_n - d_t u_t)^2 + (d_n u_t + d_t u_n)^2).
template <int LAT>
__device__ void vis_meso(const Geom& G, const Band& B, int par_t, int s, int p, double V[4])
{
    constexpr double cs2 = Lat<LAT>::CS2;
    const Side& S = B.s[s];
    const Frame F = frame_of_side(s);
    auto H = [&](int d, int pp, double h[7]) {
        if (S.tper) {
            pp %= S.L;
            if (pp < 0) pp += S.L;
        }
        const double* n = B.stripN + strip_n_index(S, par_t, d, pp);
        const double* u = B.stripU + strip_u_index(S, par_t, d, pp);
        const double sn0 = n[0] * F.n0 + n[1] * F.n1, sn1 = n[1] * F.n0 + n[2] * F.n1;
        const double st0 = n[0] * F.t0 + n[1] * F.t1, st1 = n[1] * F.t0 + n[2] * F.t1;
        h[0] = F.n0 * sn0 + F.n1 * sn1;
        h[1] = F.t0 * sn0 + F.t1 * sn1;
        h[2] = F.t0 * st0 + F.t1 * st1;
        h[3] = n[3] * F.n0 + n[4] * F.n1;
        h[4] = n[3] * F.t0 + n[4] * F.t1;
        h[5] = u[1] * F.n0 + u[2] * F.n1;
        h[6] = u[1] * F.t0 + u[2] * F.t1;
    };
    int tmode = 0;
    if (!S.tper) {
        if (p == S.hi) tmode = 1;
        else if (p == S.lo) tmode = -1;
    }
    double h0[7], h1[7], h2[7], ha[7], hb[7];
    H(0, p, h0);
    H(1, p, h1);
    H(2, p, h2);
    if (tmode == 0) {
        H(0, p + 1, ha);
        H(0, p - 1, hb);
    } else if (tmode == 1) {
        H(0, p - 1, ha);
        H(0, p - 2, hb);
    } else {
        H(0, p + 1, ha);
        H(0, p + 2, hb);
    }
    double dn[7], dt[7];
    for (int m = 0; m < 7; ++m) {
        dn[m] = 0.5 * (3.0 * h0[m] - 4.0 * h1[m] + h2[m]);
        if (tmode == 0) dt[m] = 0.5 * (ha[m] - hb[m]);
        else if (tmode == 1) dt[m] = 0.5 * (3.0 * h0[m] - 4.0 * ha[m] + hb[m]);
        else dt[m] = -0.5 * (3.0 * h0[m] - 4.0 * ha[m] + hb[m]);
    }
    const double rho = G.rho0 + B.stripU[strip_u_index(S, par_t, 0, p)];
    V[0] = 0.0;
    V[1] = (dn[0] + dt[1]) / rho;
    V[2] = (dn[1] + dt[2]) / rho;
    V[3] = 0.0;
    if (Lat<LAT>::THERMAL) {
        const double nu = (G.tau - 0.5) * cs2;
        const double e1 = dn[5] - dt[6], e2 = dn[6] + dt[5];
        V[3] = -(dn[3] + dt[4]) / (rho * cs2) + nu / cs2 * (e1 * e1 + e2 * e2);
    }
}

// "-FD" form (Sec. 4.2) at layer j: second derivatives of the macros of time
// t, 4-point one-sided at j = M, 3-point central elsewhere and along the side.
template <int LAT>
__device__ void vis_fd(const Geom& G, const Band& B, int par_t, int s, int j, int p, double V[4])
{
    constexpr double cs2 = Lat<LAT>::CS2;
    const Frame F = frame_of_side(s);
    const double* Y = B.Ub;
    double U[4], A[4], Bv[4], Cv[4], Tp[4], Tm[4];
    fetch_local(G, B, Y, par_t, 0.0, s, j, p, F, U);
    fetch_local(G, B, Y, par_t, 0.0, s, j - 1, p, F, Bv);
    fetch_local(G, B, Y, par_t, 0.0, s, j, p + 1, F, Tp);
    fetch_local(G, B, Y, par_t, 0.0, s, j, p - 1, F, Tm);
    double dnn[4], d1n[4];
    if (j == G.M) {
        fetch_local(G, B, Y, par_t, 0.0, s, j - 2, p, F, A);
        fetch_local(G, B, Y, par_t, 0.0, s, j - 3, p, F, Cv);
        for (int m = 0; m < 4; ++m) {
            dnn[m] = 2.0 * U[m] - 5.0 * Bv[m] + 4.0 * A[m] - Cv[m];
            d1n[m] = 0.5 * (3.0 * U[m] - 4.0 * Bv[m] + A[m]);
        }
    } else {
        fetch_local(G, B, Y, par_t, 0.0, s, j + 1, p, F, A);
        for (int m = 0; m < 4; ++m) {
            dnn[m] = A[m] - 2.0 * U[m] + Bv[m];
            d1n[m] = 0.5 * (A[m] - Bv[m]);
        }
    }
    double dtt[4], d1t[4];
    for (int m = 0; m < 4; ++m) {
        dtt[m] = Tp[m] - 2.0 * U[m] + Tm[m];
        d1t[m] = 0.5 * (Tp[m] - Tm[m]);
    }
    const double nu = (G.tau - 0.5) * cs2;
    V[0] = 0.0;
    V[1] = nu * (dnn[1] + dtt[1]);
    V[2] = nu * (dnn[2] + dtt[2]);
    V[3] = 0.0;
    if (Lat<LAT>::THERMAL) {
        const double e1 = d1n[1] - d1t[2], e2 = d1n[2] + d1t[1];
        V[3] = 2.0 * nu * (dnn[3] + dtt[3]) + nu / cs2 * (e1 * e1 + e2 * e2);
    }
}

// ---------------------------------------------------------------------------
// Right-hand sides of the boundary ODE
// ---------------------------------------------------------------------------

template <int LAT>
__device__ void side_rhs(const Geom& G, const Band& B, const double* Y, int par_t, double frac,
                         int s, int j, int p, const double V[4], int mask, double k[4])
{
    using L = Lat<LAT>;
    const Frame F = frame_of_side(s);
    double U[4], A[4], Bv[4], dUn[4], Up[4], Um[4];
    fetch_local(G, B, Y, par_t, frac, s, j, p, F, U);
    if (j == G.M) {                 // Eq. FD-dx-bw at the outermost layer
        fetch_local(G, B, Y, par_t, frac, s, j - 1, p, F, A);
        fetch_local(G, B, Y, par_t, frac, s, j - 2, p, F, Bv);
        for (int m = 0; m < 4; ++m) dUn[m] = 0.5 * (3.0 * U[m] - 4.0 * A[m] + Bv[m]);
    } else {                        // Eq. FD-dx-center at inner layers
        fetch_local(G, B, Y, par_t, frac, s, j + 1, p, F, A);
        fetch_local(G, B, Y, par_t, frac, s, j - 1, p, F, Bv);
        for (int m = 0; m < 4; ++m) dUn[m] = 0.5 * (A[m] - Bv[m]);
    }
    // transversal vector T (Sec. 3.1), central differences along the side
    fetch_local(G, B, Y, par_t, frac, s, j, p + 1, F, Up);
    fetch_local(G, B, Y, par_t, frac, s, j, p - 1, F, Um);
    const double rho0 = G.rho0, cs2 = L::CS2;
    const double rho = rho0 + U[0], ut = U[2];
    const double d_rhout = 0.5 * ((rho0 + Up[0]) * Up[2] - (rho0 + Um[0]) * Um[2]);
    const double d_un = 0.5 * (Up[1] - Um[1]);
    const double d_ut = 0.5 * (Up[2] - Um[2]);
    double TT[4], dP;
    if (L::THERMAL) {
        // rho T - rho0 = drho + rho0 dT + drho dT
        const double d_rhoT = 0.5 * ((Up[0] + rho0 * Up[3] + Up[0] * Up[3]) -
                                     (Um[0] + rho0 * Um[3] + Um[0] * Um[3]));
        const double d_Tut = 0.5 * ((1.0 + Up[3]) * Up[2] - (1.0 + Um[3]) * Um[2]);
        TT[0] = -d_rhout;
        TT[1] = -ut * d_un;
        TT[2] = -(cs2 / rho) * d_rhoT - ut * d_ut;
        TT[3] = -d_Tut;
        dP = cs2 * (U[0] + rho0 * U[3] + U[0] * U[3]) - B.pdev[s];
    } else {
        TT[0] = -d_rhout;
        TT[1] = -ut * d_un;
        TT[2] = -(cs2 / rho) * 0.5 * (Up[0] - Um[0]) - ut * d_ut;
        TT[3] = 0.0;
        dP = cs2 * U[0] - B.pdev[s];
    }
    const CharSys C = char_sys(L::THERMAL, cs2, rho0, U);
    double kl[4];
    char_rhs(C, B, dUn, TT, V, mask, dP, B.s[s].scheme, kl);
    to_lab(kl, F, k);
}

// Corner: LODI (Eq. PNR) along the outward diagonal at the innermost corner
// node, with a one-sided difference of spacing sqrt(2) into the bulk.
template <int LAT>
__device__ void corner_rhs(const Geom& G, const Band& B, const double* Y, int par_t, double frac,
                           int c, int mask, double k[4])
{
    using L = Lat<LAT>;
    const Frame F = frame_of_corner(c);
    const int sx = corner_sx(c), sy = corner_sy(c);
    const int sW = sx < 0 ? 0 : 1;
    const int yc = sy < 0 ? G.M - 1 : G.ny - G.M;
    double U[4], U1[4], U2[4], dUn[4];
    to_local(Y + 4LL * (B.n_side_unk + c), F, U);
    fetch_local(G, B, Y, par_t, frac, sW, 0, yc - sy, F, U1);
    fetch_local(G, B, Y, par_t, frac, sW, -1, yc - 2 * sy, F, U2);
    const double h = 2.0 * sqrt(2.0);
    for (int m = 0; m < 4; ++m) dUn[m] = (3.0 * U[m] - 4.0 * U1[m] + U2[m]) / h;
    const double zero[4] = {0.0, 0.0, 0.0, 0.0};
    const CharSys C = char_sys(L::THERMAL, L::CS2, G.rho0, U);
    double kl[4];
    char_rhs(C, B, dUn, zero, zero, mask, 0.0, SCH_LODI, kl);
    to_lab(kl, F, k);
}

// ---------------------------------------------------------------------------
// Population writes
// ---------------------------------------------------------------------------

template <int LAT, typename S>
__device__ inline void load_g(const Geom& G, const S* f, int x, int y, double* g)
{
    using L = Lat<LAT>;
    const S* in = f + (long long)y * G.nxp + x;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        double v = double(Store<S>::load(in + (long long)i * G.plane));
        if (Store<S>::SCALED) v *= L::w(i);
        g[i] = v;
    }
}

template <int LAT, typename S>
__device__ inline void put_g(const Geom& G, S* f, int x, int y, const double* g)
{
    using L = Lat<LAT>;
    S* out = f + (long long)y * G.nxp + x;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        double v = g[i];
        if (Store<S>::SCALED) v *= 1.0 / L::w(i);
        Store<S>::put(out + (long long)i * G.plane, typename Store<S>::C(v));
    }
}

template <int LAT>
__device__ inline void geq_of(double rho0, const double U[4], double* ge)
{
    Moments<LAT, double> m;
    m.s0 = U[0];
    m.rho = rho0 + U[0];
    m.ux = U[1];
    m.uy = U[2];
    m.dT = Lat<LAT>::THERMAL ? U[3] : 0.0;
    equilibrium<LAT, double>(m, ge);
}

// Mesoscopic Dirichlet condition for the boundary state Unew, stored
// post-collision: f^eq(Unew), plus for Eq. NEEP the non-equilibrium part of
// the bulk neighbour x_f after its collision, f*(x_f) - f^eq(U(x_f)).
template <int LAT, typename S>
__device__ void dirichlet(const Geom& G, const Band& B, S* f, int par_new, const double Unew[4],
                          int xs, int ys, const double* Usrc, int x0, int y0, int nbx, int nby,
                          int dx, int dy)
{
    using L = Lat<LAT>;
    double ge[L::Q];
    geq_of<LAT>(G.rho0, Unew, ge);
    if (B.dirichlet == 1) {
        double gs[L::Q], gf[L::Q];
        load_g<LAT, S>(G, f, xs, ys, gs);
        geq_of<LAT>(G.rho0, Usrc, gf);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) ge[i] += gs[i] - gf[i];
    }
    for (int a = 0; a < nbx; ++a)
        for (int b = 0; b < nby; ++b) put_g<LAT, S>(G, f, x0 + a * dx, y0 + b * dy, ge);
    (void)par_new;
}

template <int LAT, typename S>
__global__ void __launch_bounds__(kBandThreads)
    k_cbc_stage(Geom G, Band B, S* __restrict__ f, int par_t, int stage)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= B.n_unk) return;
    const double frac = stage == 0 ? 0.0 : (stage == 3 ? 1.0 : 0.5);
    const double* Yin = stage == 0 ? B.Ub : (stage == 2 ? B.Yb : B.Ya);
    double* Yout = stage == 1 ? B.Yb : B.Ya;
    const bool corner = u >= B.n_side_unk;
    int s = 0, p = 0, j = 0, c = 0;
    if (corner) {
        c = u - B.n_side_unk;
    } else {
        while (s < 3 && !(B.s[s].kind == SIDE_CBC && u >= B.s[s].base &&
                          u < B.s[s].base + (B.s[s].hi - B.s[s].lo + 1) * G.M))
            ++s;
        const int r = u - B.s[s].base;
        p = B.s[s].lo + r / G.M;
        j = 1 + r % G.M;
    }
    double V[4];
    int mask;
    if (stage == 0) {
        const Frame F = corner ? frame_of_corner(c) : frame_of_side(s);
        double Ul[4];
        to_local(B.Ub + 4LL * u, F, Ul);
        mask = incoming_mask(char_sys(Lat<LAT>::THERMAL, Lat<LAT>::CS2, G.rho0, Ul));
        if (corner || B.viscous == VIS_OFF) {
            V[0] = V[1] = V[2] = V[3] = 0.0;
        } else if (B.viscous == VIS_FD) {
            vis_fd<LAT>(G, B, par_t, s, j, p, V);
        } else {
            vis_meso<LAT>(G, B, par_t, s, p, V);
        }
        for (int m = 0; m < 4; ++m) B.V[4LL * u + m] = V[m];
        B.mask[u] = mask;
    } else {
        for (int m = 0; m < 4; ++m) V[m] = B.V[4LL * u + m];
        mask = B.mask[u];
    }
    double k[4];
    if (corner) corner_rhs<LAT>(G, B, Yin, par_t, frac, c, mask, k);
    else side_rhs<LAT>(G, B, Yin, par_t, frac, s, j, p, V, mask, k);

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
    for (int m = 0; m < 4; ++m) Unew[m] = U0[m] + (acc[m] + k[m]) / 6.0;
    for (int m = 0; m < 4; ++m) B.Ub[4LL * u + m] = Unew[m];

    const int par_new = par_t ^ 1;
    if (corner) {
        const int sx = corner_sx(c), sy = corner_sy(c);
        const int sW = sx < 0 ? 0 : 1;
        const int xc = sx < 0 ? G.M - 1 : G.nx - G.M;
        const int yc = sy < 0 ? G.M - 1 : G.ny - G.M;
        const double* Us = B.stripU + strip_u_index(B.s[sW], par_new, 0, yc - sy);
        const int x0 = sx < 0 ? 0 : G.nx - 1, y0 = sy < 0 ? 0 : G.ny - 1;
        dirichlet<LAT, S>(G, B, f, par_new, Unew, xc - sx, yc - sy, Us, x0, y0, G.M, G.M,
                          sx < 0 ? 1 : -1, sy < 0 ? 1 : -1);
    } else {
        int xf, yf;
        side_xf(s, p, G.nx, G.ny, G.M, xf, yf);
        const double* Us = B.stripU + strip_u_index(B.s[s], par_new, 0, p);
        dirichlet<LAT, S>(G, B, f, par_new, Unew, xf, yf, Us, xf + j * side_nx(s),
                          yf + j * side_ny(s), 1, 1, 0, 0);
    }
}

// Zero gradient (Eq. zg-bc: copy of the post-collision populations of x_f)
// and inflow equilibrium nodes; corner blocks copy the diagonal bulk node.
template <int LAT, typename S>
__global__ void k_extras(Geom G, Band B, S* __restrict__ f)
{
    using L = Lat<LAT>;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B.n_extra) return;
    int kind, x, y, xs, ys;
    if (e < B.n_extra_side) {
        int s = 0;
        while (s < 3 && !(B.s[s].kind >= SIDE_INFLOW && e >= B.s[s].ebase &&
                          e < B.s[s].ebase + (B.s[s].hi - B.s[s].lo + 1) * G.M))
            ++s;
        const int r = e - B.s[s].ebase;
        const int p = B.s[s].lo + r / G.M, j = 1 + r % G.M;
        side_xf(s, p, G.nx, G.ny, G.M, xs, ys);
        x = xs + j * side_nx(s);
        y = ys + j * side_ny(s);
        kind = B.s[s].kind;
    } else {
        const int r = e - B.n_extra_side, MM = G.M * G.M;
        const int c = r / MM, a = (r % MM) / G.M, b = r % G.M;
        const int sx = corner_sx(c), sy = corner_sy(c);
        x = sx < 0 ? a : G.nx - 1 - a;
        y = sy < 0 ? b : G.ny - 1 - b;
        const int xc = sx < 0 ? G.M - 1 : G.nx - G.M, yc = sy < 0 ? G.M - 1 : G.ny - G.M;
        xs = xc - sx;
        ys = yc - sy;
        kind = B.corner_kind;
    }
    double g[L::Q];
    if (kind == SIDE_ZG) load_g<LAT, S>(G, f, xs, ys, g);
    else geq_of<LAT>(G.rho0, B.Uin, g);
    put_g<LAT, S>(G, f, x, y, g);
}

template <int LAT, typename S>
int boundary_t(const Geom& G, const Band& B, void* fnew, int par_t, cudaStream_t st)
{
    S* f = static_cast<S*>(fnew);
    if (B.n_extra > 0) k_extras<LAT, S><<<(B.n_extra + 127) / 128, 128, 0, st>>>(G, B, f);
    if (B.n_unk > 0) {
        const int nb = (B.n_unk + kBandThreads - 1) / kBandThreads;
        for (int stage = 0; stage < 4; ++stage)
            k_cbc_stage<LAT, S><<<nb, kBandThreads, 0, st>>>(G, B, f, par_t, stage);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

int launch_boundary(int lat, int storage, const Geom& G, const Band& B, void* fnew, int par_t,
                    cudaStream_t st)
{
    if (lat == D2Q9) {
        if (storage == 0) return boundary_t<D2Q9, double>(G, B, fnew, par_t, st);
        if (storage == 1) return boundary_t<D2Q9, float>(G, B, fnew, par_t, st);
        if (storage == 2) return boundary_t<D2Q9, __half>(G, B, fnew, par_t, st);
    } else {
        if (storage == 0) return boundary_t<D2Q37, double>(G, B, fnew, par_t, st);
        if (storage == 1) return boundary_t<D2Q37, float>(G, B, fnew, par_t, st);
        if (storage == 2) return boundary_t<D2Q37, __half>(G, B, fnew, par_t, st);
    }
    return -1;
}

}  // namespace lbmgb
