// collide.cuh -- the per-node update shared by the bulk kernels (bulk.cu)
// and the band kernel (boundary.cu): plain pull, moments, BGK collision.
#pragma once
#include "dual.cuh"
#include "lbm_internal.cuh"

namespace lbmgb {

// 1/tau and rho0 in the precision of arithmetic type C (float-based types
// take the float-rounded values).
template <typename C>
__device__ __forceinline__ C omega_of(const Geom& G)
{
    if constexpr (sizeof(typename DualTraits<C>::Value) == 4) return C(G.omega_f);
    else return C(G.omega);
}
template <typename C>
__device__ __forceinline__ C rho0_of(const Geom& G)
{
    if constexpr (sizeof(typename DualTraits<C>::Value) == 4) return C(G.rho0_f);
    else return C(G.rho0);
}

// The reference velocity of the stored populations in the precision of C.
template <typename C>
__device__ __forceinline__ C uref_of(const Geom& G, int k)
{
    if constexpr (sizeof(typename DualTraits<C>::Value) == 4) return C(G.uref_f[k]);
    else return C(G.uref[k]);
}

// The reference velocity the populations of storage S are held against, as
// a double: the value in the storage's arithmetic (float-rounded for FP32
// and FP16), so that every kernel shifts by the same equilibrium.
template <typename S>
__host__ __device__ __forceinline__ double stored_ref(const Geom& G, int k)
{
    if constexpr (sizeof(typename Store<S>::C) == 4) return double(G.uref_f[k]);
    else return G.uref[k];
}

// Moments of the stored populations g of a node (the grid's reference; REF =
// false compiles the plain shift only, for kernels instantiated per form).
template <int LAT, typename C, bool REF = true>
__device__ __forceinline__ Moments<LAT, C> moments_G(const Geom& G, const C* g)
{
    return moments<LAT, C>(g, rho0_of<C>(G), REF ? G.ref : 0, uref_of<C>(G, 0), uref_of<C>(G, 1));
}

// Viscous stress sigma' = -(1 - 1/(2 tau)) sum c c (f - f^eq) (Eq. LaplaceU)
// and heat flux q = (1 - 1/(2 tau)) 1/2 sum (f - f^eq) |c-u|^2 (c-u)
// (Eqs. heatflux, LaplaceT; the equilibrium part of the central third
// moment vanishes on D2Q37).
template <int LAT, typename C, typename T>
__device__ __forceinline__ void neq_moments(const C* g, const Moments<LAT, C>& m, T fac, T* N)
{
    using L = Lat<LAT>;
    C geq[L::Q];
    equilibrium<LAT, C>(m, geq);
    C pxx = 0, pxy = 0, pyy = 0, qx = 0, qy = 0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const C d = g[i] - geq[i];
        const C cx = C(L::cx(i)), cy = C(L::cy(i));
        pxx += cx * cx * d;
        pxy += cx * cy * d;
        pyy += cy * cy * d;
        if (L::THERMAL) {
            const C ex = cx - m.ux, ey = cy - m.uy;
            const C h = C(0.5) * d * (ex * ex + ey * ey);
            qx += h * ex;
            qy += h * ey;
        }
    }
    N[0] = -fac * T(pxx);
    N[1] = -fac * T(pxy);
    N[2] = -fac * T(pyy);
    N[3] = fac * T(qx);
    N[4] = fac * T(qy);
}

// Plain pull of node (x, y) with periodic wrap-around of the sources.
template <int LAT, typename S, typename C>
__device__ __forceinline__ void pull_plain(const Geom& G, const Offsets& O,
                                           const S* __restrict__ fin, int x, int y, C* g)
{
    using L = Lat<LAT>;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        int xs = x - L::cx(i), ys = y - L::cy(i);
        if (L::cx(i) && G.perx) xs = xs < 0 ? xs + G.nx : (xs >= G.nx ? xs - G.nx : xs);
        if (L::cy(i) && G.pery) ys = ys < 0 ? ys + G.ny : (ys >= G.ny ? ys - G.ny : ys);
        g[i] = C(Store<S>::load(fin + (O.st[i] + ys * G.nxp + xs)));
    }
}

// The same with the plane offsets computed from the plane size (for kernels
// that serve several grids in one launch).
template <int LAT, typename S, typename C>
__device__ __forceinline__ void pull_plain_planes(const Geom& G, const S* __restrict__ fin, int x,
                                                  int y, C* g)
{
    using L = Lat<LAT>;
    const int plane = int(G.plane);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        int xs = x - L::cx(i), ys = y - L::cy(i);
        if (L::cx(i) && G.perx) xs = xs < 0 ? xs + G.nx : (xs >= G.nx ? xs - G.nx : xs);
        if (L::cy(i) && G.pery) ys = ys < 0 ? ys + G.ny : (ys >= G.ny ? ys - G.ny : ys);
        g[i] = C(Store<S>::load(fin + (L::plane_of(i) * plane + ys * G.nxp + xs)));
    }
}

// Moments (Eq. macro) and BGK collision (Eq. bgk) of one node whose pulled
// populations are in g (already multiplied by w for scaled storage).  The
// post-collision value of velocity i goes to put(i, value); the moments of
// the pulled populations are returned.
// BGK collision of a node whose moments m are known; gi(i) gives the
// pre-collision population i (read as the pair loop needs it).
template <int LAT, typename C, typename Get, typename Put>
__device__ __forceinline__ void collide_given(const Geom& G, const Moments<LAT, C>& m, Get&& gi, Put&& put)
{
    using L = Lat<LAT>;
    constexpr int Q = L::Q;

    // BGK collide (Eq. bgk), one opposite pair at a time:
    // g^eq_{+-} = w (rho - rho0) + w rho (even +- odd) in p = c.u / c_s^2,
    // or, relative to a reference equilibrium (m.ref), w (Ev +- Od) of
    // eq_pair_ref.
    constexpr C ics2 = C(1.0 / L::CS2);
    constexpr C a3 = L::ORDER >= 3 ? C(1.0 / 6.0) : C(0);
    constexpr C a4 = L::ORDER >= 4 ? C(1.0 / 24.0) : C(0);
    const C uxs = m.ux * ics2, uys = m.uy * ics2;
    const EqPoly<C> e = eq_poly<LAT, C>(m.ux * uxs + m.uy * uys, m.dT);
    const C om = omega_of<C>(G);
    const bool ref = m.ref != 0;
    EqDelta<C> de;
    C rho0r = C(0), Uxs = C(0), Uys = C(0), vxs = C(0), vys = C(0);
    if (ref) {
        Uxs = m.Ux * ics2;
        Uys = m.Uy * ics2;
        vxs = m.vx * ics2;
        vys = m.vy * ics2;
        de = eq_delta<LAT, C>(m.Ux * Uxs + m.Uy * Uys, C(2) * (m.Ux * vxs + m.Uy * vys) + m.vx * vxs + m.vy * vys,
                              m.dT);
        rho0r = m.rho - m.s0;
    }
    // g^eq of the pair (i, i + 1) of class k
    auto pair = [&](int i, C& gp, C& gm) {
        const int k = L::cls(i);
        const C xi2 = C(L::c2cls(k)) * ics2;
        if (ref) {
            const C P = C(L::cx(i)) * Uxs + C(L::cy(i)) * Uys, q = C(L::cx(i)) * vxs + C(L::cy(i)) * vys;
            C Ev, Od;
            eq_pair_ref<LAT, C>(e, de, xi2, P, q, m.s0, rho0r, Ev, Od);
            gp = C(L::w(i)) * (Ev + Od);
            gm = C(L::w(i)) * (Ev - Od);
            return;
        }
        const C a0 = e.A0 + xi2 * (e.B0 + e.C0 * xi2);
        const C a1 = e.A1 + e.B1 * xi2;
        const C a2 = e.A2 + e.B2 * xi2;
        C p;
        if (L::cx(i) == 0) p = C(L::cy(i)) * uys;
        else if (L::cy(i) == 0) p = C(L::cx(i)) * uxs;
        else p = C(L::cx(i)) * uxs + C(L::cy(i)) * uys;
        const C p2 = p * p;
        const C ev = a0 + p2 * (a2 + p2 * a4);
        const C od = p * (a1 + p2 * a3);
        const C ws0 = C(L::w(i)) * m.s0, wr = C(L::w(i)) * m.rho;
        gp = ws0 + wr * (ev + od);
        gm = ws0 + wr * (ev - od);
    };
    if (sizeof(typename DualTraits<C>::Value) == 8) {
        {
            const C geq = ref ? C(L::w(0)) * (m.s0 * (C(1) + e.A0) + rho0r * de.A0)
                              : C(L::w(0)) * (m.s0 + m.rho * e.A0);
            { const C g_ = gi(0); put(0, g_ + om * (geq - g_)); }
        }
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            C gp, gm;
            pair(i, gp, gm);
            { const C g_ = gi(i); put(i, g_ + om * (gp - g_)); }
            { const C g_ = gi(i + 1); put(i + 1, g_ + om * (gm - g_)); }
        }
    } else {
        // FP32 arithmetic.  Float-rounded weights and c_s^2 miss the discrete
        // moment identities by ~1e-8, which would make each collision leak
        // mass, momentum and energy at that relative rate.  The equilibrium
        // is therefore closed on the conserved moments: the |c| = 1 pairs
        // take the momentum and energy remainders and the rest velocity the
        // mass remainder (corrections of float-rounding size).
        C M0 = 0, Mx = 0, My = 0, Me = 0;
#pragma unroll
        for (int i = 5; i < Q; i += 2) {
            const int k = L::cls(i);
            C gp, gm;
            pair(i, gp, gm);
            const C sum = gp + gm, dif = gp - gm;
            M0 += sum;
            if (L::cx(i)) Mx += C(L::cx(i)) * dif;
            if (L::cy(i)) My += C(L::cy(i)) * dif;
            if (L::THERMAL) Me += C(L::c2cls(k)) * sum;
            { const C g_ = gi(i); put(i, g_ + om * (gp - g_)); }
            { const C g_ = gi(i + 1); put(i + 1, g_ + om * (gm - g_)); }
        }
        // |c| = 1 class: (1,0) and (-1,0) are velocities 1, 2; (0,1), (0,-1) are 3, 4
        C ex, ey;
        if (ref) {
            C Ev, Od;
            eq_pair_ref<LAT, C>(e, de, ics2, Uxs, vxs, m.s0, rho0r, Ev, Od);
            ex = C(L::w(1)) * Ev;
            eq_pair_ref<LAT, C>(e, de, ics2, Uys, vys, m.s0, rho0r, Ev, Od);
            ey = C(L::w(1)) * Ev;
        } else {
            const C a0 = e.A0 + ics2 * (e.B0 + e.C0 * ics2);
            const C a2 = e.A2 + e.B2 * ics2;
            const C px2 = uxs * uxs, py2 = uys * uys;
            const C ws0 = C(L::w(1)) * m.s0, wr = C(L::w(1)) * m.rho;
            ex = ws0 + wr * (a0 + px2 * (a2 + px2 * a4));
            ey = ws0 + wr * (a0 + py2 * (a2 + py2 * a4));
        }
        if (L::THERMAL) {
            const C d = C(0.25) * (m.se - Me - C(2) * (ex + ey));
            ex += d;
            ey += d;
        }
        const C ox = C(0.5) * (m.sx - Mx), oy = C(0.5) * (m.sy - My);
        { const C g_ = gi(1); put(1, g_ + om * (ex + ox - g_)); }
        { const C g_ = gi(2); put(2, g_ + om * (ex - ox - g_)); }
        { const C g_ = gi(3); put(3, g_ + om * (ey + oy - g_)); }
        { const C g_ = gi(4); put(4, g_ + om * (ey - oy - g_)); }
        const C geq0 = m.s0 - M0 - C(2) * (ex + ey);
        { const C g_ = gi(0); put(0, g_ + om * (geq0 - g_)); }
    }

}

// The same collision for storage that holds h_i = g_i / w_i (FP16), done in
// those scaled variables so that no population is multiplied by w_i on the
// way in or divided by it on the way out: the moments are sums of w_i h_i
// (w_i c_i folded into one constant), and h^eq_i = g^eq_i / w_i =
// (rho - rho0) + rho (even +- odd) carries no weight.  FP32 arithmetic, with
// the conserved-moment closure of the FP32 path above (the closure sums take
// w_i back in).  put(i, value) receives h*_i.
template <int LAT, bool REF, typename Put>
__device__ __forceinline__ void collide_scaled(const Geom& G, const float* h, Put&& put)
{
    using L = Lat<LAT>;
    using C = float;
    constexpr int Q = L::Q;
    C s0 = 0, sx = 0, sy = 0, se = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        s0 += C(L::w(i)) * h[i];
        if (L::cx(i)) sx += C(L::w(i) * L::cx(i)) * h[i];
        if (L::cy(i)) sy += C(L::w(i) * L::cy(i)) * h[i];
        if (L::THERMAL && i) se += C(L::w(i) * (L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i))) * h[i];
    }
    const Moments<LAT, C> m = moments_of_sums<LAT, C>(s0, sx, sy, se, rho0_of<C>(G), REF ? G.ref : 0,
                                                      uref_of<C>(G, 0), uref_of<C>(G, 1));
    constexpr C ics2 = C(1.0 / L::CS2);
    constexpr C a3 = L::ORDER >= 3 ? C(1.0 / 6.0) : C(0);
    constexpr C a4 = L::ORDER >= 4 ? C(1.0 / 24.0) : C(0);
    const C uxs = m.ux * ics2, uys = m.uy * ics2;
    const EqPoly<C> e = eq_poly<LAT, C>(m.ux * uxs + m.uy * uys, m.dT);
    const C om = omega_of<C>(G);
    const bool ref = m.ref != 0;
    EqDelta<C> de;
    C rho0r = C(0), Uxs = C(0), Uys = C(0), vxs = C(0), vys = C(0);
    if (ref) {
        Uxs = m.Ux * ics2;
        Uys = m.Uy * ics2;
        vxs = m.vx * ics2;
        vys = m.vy * ics2;
        de = eq_delta<LAT, C>(m.Ux * Uxs + m.Uy * Uys, C(2) * (m.Ux * vxs + m.Uy * vys) + m.vx * vxs + m.vy * vys,
                              m.dT);
        rho0r = m.rho - m.s0;
    }
    C M0 = 0, Mx = 0, My = 0, Me = 0;
#pragma unroll
    for (int i = 5; i < Q; i += 2) {
        const int k = L::cls(i);
        const C xi2 = C(L::c2cls(k)) * ics2;
        C hp, hm;
        if (ref) {
            const C P = C(L::cx(i)) * Uxs + C(L::cy(i)) * Uys, q = C(L::cx(i)) * vxs + C(L::cy(i)) * vys;
            C Ev, Od;
            eq_pair_ref<LAT, C>(e, de, xi2, P, q, m.s0, rho0r, Ev, Od);
            hp = Ev + Od;
            hm = Ev - Od;
        } else {
            const C a0 = e.A0 + xi2 * (e.B0 + e.C0 * xi2);
            const C a1 = e.A1 + e.B1 * xi2;
            const C a2 = e.A2 + e.B2 * xi2;
            C p;
            if (L::cx(i) == 0) p = C(L::cy(i)) * uys;
            else if (L::cy(i) == 0) p = C(L::cx(i)) * uxs;
            else p = C(L::cx(i)) * uxs + C(L::cy(i)) * uys;
            const C p2 = p * p;
            const C ev = a0 + p2 * (a2 + p2 * a4);
            const C od = p * (a1 + p2 * a3);
            hp = m.s0 + m.rho * (ev + od);
            hm = m.s0 + m.rho * (ev - od);
        }
        const C sum = hp + hm, dif = hp - hm;
        M0 += C(L::w(i)) * sum;
        if (L::cx(i)) Mx += C(L::w(i) * L::cx(i)) * dif;
        if (L::cy(i)) My += C(L::w(i) * L::cy(i)) * dif;
        if (L::THERMAL) Me += C(L::w(i) * L::c2cls(k)) * sum;
        put(i, h[i] + om * (hp - h[i]));
        put(i + 1, h[i + 1] + om * (hm - h[i + 1]));
    }
    // |c| = 1 class and the rest velocity close the conserved moments, in
    // unscaled units, then scaled
    C ex, ey;
    if (ref) {
        C Ev, Od;
        eq_pair_ref<LAT, C>(e, de, ics2, Uxs, vxs, m.s0, rho0r, Ev, Od);
        ex = C(L::w(1)) * Ev;
        eq_pair_ref<LAT, C>(e, de, ics2, Uys, vys, m.s0, rho0r, Ev, Od);
        ey = C(L::w(1)) * Ev;
    } else {
        const C a0 = e.A0 + ics2 * (e.B0 + e.C0 * ics2);
        const C a2 = e.A2 + e.B2 * ics2;
        const C px2 = uxs * uxs, py2 = uys * uys;
        const C ws0 = C(L::w(1)) * m.s0, wr = C(L::w(1)) * m.rho;
        ex = ws0 + wr * (a0 + px2 * (a2 + px2 * a4));
        ey = ws0 + wr * (a0 + py2 * (a2 + py2 * a4));
    }
    if (L::THERMAL) {
        const C d = C(0.25) * (m.se - Me - C(2) * (ex + ey));
        ex += d;
        ey += d;
    }
    const C ox = C(0.5) * (m.sx - Mx), oy = C(0.5) * (m.sy - My);
    constexpr C iw1 = C(1.0 / L::w(1));
    put(1, h[1] + om * ((ex + ox) * iw1 - h[1]));
    put(2, h[2] + om * ((ex - ox) * iw1 - h[2]));
    put(3, h[3] + om * ((ey + oy) * iw1 - h[3]));
    put(4, h[4] + om * ((ey - oy) * iw1 - h[4]));
    const C geq0 = m.s0 - M0 - C(2) * (ex + ey);
    put(0, h[0] + om * (geq0 * C(1.0 / L::w(0)) - h[0]));
}

template <int LAT, typename C, bool REF = false, typename Put>
__device__ __forceinline__ Moments<LAT, C> collide(const Geom& G, const C* g, Put&& put)
{
    const Moments<LAT, C> m = moments_G<LAT, C, REF>(G, g);
    collide_given<LAT, C>(G, m, [&](int i) -> const C& { return g[i]; }, put);
    return m;
}

}  // namespace lbmgb
