// bulk.cu -- bulk kernels of the thermal lattice Boltzmann step.
//
//  k_bulk     fused pull-stream + moments + BGK collide on the interior
//             bulk nodes (Eqs. lbe, macro, bgk with the equilibria of
//             Eqs. feq-3/feq-4).
//  k_rim      the same update on the rim: bands of width max(M, 3) next to
//             the non-periodic sides, whose pulls reach nodes the boundary
//             phase writes; it also exports the macros and non-equilibrium
//             moments of the three bulk columns/rows next to each
//             characteristic side (used by the boundary solver of
//             Sec. 3.3).  The interior is independent of the boundary phase
//             of the same step, so the two can run concurrently.
//  k_init     f = f^eq(U0) on every node and the strips of time 0.
//  k_inflow   the fixed inflow equilibrium on the inflow nodes of a buffer.
//  k_init_band  boundary ODE state of time 0.
//  k_macros   macroscopic fields of the stored populations (Eq. macro).
//
// Populations are stored post-collision and shifted, g = f* - w rho0, in SoA
// planes [Q][ny][nxp].  A bulk node pulls g*_i(x - c_i) for every i.  Away
// from periodic wrap-around the 37 shifted source rows of a 128-node row
// segment are staged through shared memory by tensor copies (TMA); stores
// go straight to global memory at fixed plane offsets (Offsets, in the
// kernel parameter bank).  The FP32/FP16 paths do all of their arithmetic in
// FP32; the FP64 path in FP64.
#include "lbm_internal.cuh"

#include <utility>

namespace lbmgb {

namespace {

constexpr int kBulkThreads = 128;   // one CTA = one row segment of 128 nodes

// TMA staging.  For population i a CTA needs the source row segment
// [x0 - c_ix, x0 + 127 - c_ix] of row y - c_iy.  Planes are stored grouped by
// c_y, so one 3D tensor copy brings, for every population of a group, the
// 16-byte-aligned box [x0 - H, x0 + 128 + H) of its source row into shared
// memory (H = 4 elements for 4- and 8-byte storage, 8 for 2-byte storage,
// >= max |c_x| = 3); each thread then reads its shifted values there.
// Group boxes start 128-byte aligned.
template <int LAT, typename S>
struct Stage {
    static constexpr int H = sizeof(S) == 2 ? 8 : 4;
    static constexpr int W = kBulkThreads + 2 * H;                 // elements per row box
    static constexpr int ROWB = W * int(sizeof(S));                // bytes per row box
    __host__ __device__ static constexpr int gbytes(int g) { return Lat<LAT>::gcount(g) * ROWB; }
    __host__ __device__ static constexpr int gofs(int g)           // byte offset of group g
    {
        int o = 0;
        for (int k = 0; k < g; ++k) o += (gbytes(k) + 127) / 128 * 128;
        return o;
    }
    static constexpr int TOTAL = gofs(Lat<LAT>::NG);
    static constexpr int TX = Lat<LAT>::Q * ROWB;                  // bytes per tile
    // element index of velocity i's row box inside the staging buffer
    __host__ __device__ static constexpr int elem(int i)
    {
        return gofs(group_of<LAT>(i)) / int(sizeof(S)) +
               (Lat<LAT>::plane_of(i) - Lat<LAT>::gstart(group_of<LAT>(i))) * W;
    }
};

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

// Wait for the transaction barrier (phase 0) with a 1 s limit; on timeout
// record it in *status and wait once more (again bounded) for copies still
// in flight before giving up.
__device__ bool wait_tx(unsigned long long* bar, int* status)
{
    const unsigned a = smem_u32(bar);
    for (int attempt = 0; attempt < 2; ++attempt) {
        const unsigned long long t0 = global_ns();
        for (;;) {
            unsigned ok;
            asm volatile(
                "{\n .reg .pred p;\n"
                " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                " selp.u32 %0, 1, 0, p;\n}"
                : "=r"(ok)
                : "r"(a), "r"(0u)
                : "memory");
            if (ok) return attempt == 0;
            if (global_ns() - t0 > 1000000000ull) break;
        }
        if (attempt == 0) atomicOr(status, 2);
    }
    return false;
}

template <typename C>
__device__ __forceinline__ C omega_of(const Geom& G);
template <>
__device__ __forceinline__ float omega_of<float>(const Geom& G) { return G.omega_f; }
template <>
__device__ __forceinline__ double omega_of<double>(const Geom& G) { return G.omega; }
template <typename C>
__device__ __forceinline__ C rho0_of(const Geom& G);
template <>
__device__ __forceinline__ float rho0_of<float>(const Geom& G) { return G.rho0_f; }
template <>
__device__ __forceinline__ double rho0_of<double>(const Geom& G) { return G.rho0; }

// Viscous stress sigma' = -(1 - 1/(2 tau)) sum c c (f - f^eq) (Eq. LaplaceU)
// and heat flux q = (1 - 1/(2 tau)) 1/2 sum (f - f^eq) |c-u|^2 (c-u)
// (Eqs. heatflux, LaplaceT; the equilibrium part of the central third
// moment vanishes on D2Q37).
template <int LAT, typename C>
__device__ __forceinline__ void neq_moments(const C* g, const Moments<LAT, C>& m, double fac,
                                         double* N)
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
    N[0] = -fac * double(pxx);
    N[1] = -fac * double(pxy);
    N[2] = -fac * double(pyy);
    N[3] = fac * double(qx);
    N[4] = fac * double(qy);
}

// Strip export of one bulk node next to a characteristic side (a few
// columns/rows of the grid): macros and non-equilibrium moments of its
// pulled (pre-collision) populations g with moments m.
template <int LAT, typename C>
__device__ __forceinline__ void export_from(const Geom& G, const Export& E, const C* g,
                                            const Moments<LAT, C>& m, int x, int y, int par_new)
{
    const int dd[4] = {x - G.M, G.nx - 1 - G.M - x, y - G.M, G.ny - 1 - G.M - y};
    double N[5];
    neq_moments<LAT, C>(g, m, 1.0 - 0.5 / G.tau, N);
    const double U[4] = {double(m.s0), double(m.ux), double(m.uy), double(m.dT)};
    for (int s = 0; s < 4; ++s) {
        if (!E.cbc[s] || dd[s] < 0 || dd[s] > 2) continue;
        const int p = s < 2 ? y : x;
        const long long slot = (long long)par_new * E.nslots + E.offS[s] + dd[s] * E.L[s] + p;
        double* u = E.stripU + slot * 4;
        double* n = E.stripN + slot * 5;
        for (int c = 0; c < 4; ++c) u[c] = U[c];
        for (int c = 0; c < 5; ++c) n[c] = N[c];
    }
}

// Tensor maps of the input buffer: box depths 7, 5 and 3 planes.
struct Maps {
    CUtensorMap m7, m5, m3;
};

// One 3D tensor copy per c_y group; every offset, coordinate shift and map
// choice is a template constant so nothing is looked up at run time.
template <int LAT, typename S, int GI>
__device__ __forceinline__ void issue_group(const Maps& tm, unsigned char* smem, int x0, int y,
                                            unsigned bar)
{
    using L = Lat<LAT>;
    using BX = Stage<LAT, S>;
    constexpr int cnt = L::gcount(GI);
    static_assert(cnt == 7 || cnt == 5 || cnt == 3, "group depth without a tensor map");
    constexpr int ofs = BX::gofs(GI);
    constexpr int dy = L::gcy(GI);
    constexpr int z0 = L::gstart(GI);
    const CUtensorMap* m = cnt == 7 ? &tm.m7 : (cnt == 5 ? &tm.m5 : &tm.m3);
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(smem + ofs)), "l"(m), "r"(x0 - BX::H), "r"(y - dy), "r"(z0), "r"(bar)
        : "memory");
}

template <int LAT, typename S, int... GI>
__device__ __forceinline__ void issue_copies(const Maps& tm, unsigned char* smem, int x0, int y,
                                             unsigned bar, std::integer_sequence<int, GI...>)
{
    (issue_group<LAT, S, GI>(tm, smem, x0, y, bar), ...);
}

// g_i = staged source row of velocity i at column t - c_ix (offsets folded).
template <int LAT, typename S, typename C, int... I>
__device__ __forceinline__ void gather_staged(C* g, const S* sb, int t,
                                              std::integer_sequence<int, I...>)
{
    using BX = Stage<LAT, S>;
    ((g[I] = C(sb[std::integral_constant<int, BX::elem(I) + BX::H - Lat<LAT>::cx(I)>::value + t])),
     ...);
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

// Moments, BGK collision (Eq. bgk) and post-collision store of one node
// whose pulled populations are in g, plus (EXPORT) the strip export next to
// the characteristic sides.  Only rim nodes export: the interior lies at
// least max(M, 3) >= 3 nodes inside every characteristic side.
template <int LAT, typename S, typename C, bool EXPORT>
__device__ __forceinline__ void collide_store(const Geom& G, const Offsets& O, const Export& E,
                                              const S* __restrict__ fin, S* __restrict__ fout,
                                              int x, int y, int par_new, C* g)
{
    using L = Lat<LAT>;
    constexpr int Q = L::Q;
    const int node = y * G.nxp + x;
    if (Store<S>::SCALED) {
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] *= C(L::w(i));
    }

    const Moments<LAT, C> m = moments<LAT, C>(g, rho0_of<C>(G));

    // BGK collide (Eq. bgk), one opposite pair at a time:
    // g^eq_{+-} = w (rho - rho0) + w rho (even +- odd) in p = c.u / c_s^2.
    constexpr C ics2 = C(1.0 / L::CS2);
    constexpr C a3 = L::THERMAL ? C(1.0 / 6.0) : C(0);
    constexpr C a4 = L::THERMAL ? C(1.0 / 24.0) : C(0);
    const C uxs = m.ux * ics2, uys = m.uy * ics2;
    const EqPoly<C> e = eq_poly<LAT, C>(m.ux * uxs + m.uy * uys, m.dT);
    const C om = omega_of<C>(G);
    S* out = fout + node;
    auto put = [&](int i, C v) {
        if (Store<S>::SCALED) v *= C(1.0 / L::w(i));
        Store<S>::put(out + O.st[i], v);
    };
    if (sizeof(C) == 8) {
        {
            const C geq = C(L::w(0)) * (m.s0 + m.rho * e.A0);
            put(0, g[0] + om * (geq - g[0]));
        }
#pragma unroll
        for (int i = 1; i < Q; i += 2) {
            const int k = L::cls(i);
            const C xi2 = C(L::c2cls(k)) * ics2;
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
            const C gp = ws0 + wr * (ev + od);
            const C gm = ws0 + wr * (ev - od);
            put(i, g[i] + om * (gp - g[i]));
            put(i + 1, g[i + 1] + om * (gm - g[i + 1]));
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
            const C xi2 = C(L::c2cls(k)) * ics2;
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
            const C gp = ws0 + wr * (ev + od);
            const C gm = ws0 + wr * (ev - od);
            const C sum = gp + gm, dif = gp - gm;
            M0 += sum;
            if (L::cx(i)) Mx += C(L::cx(i)) * dif;
            if (L::cy(i)) My += C(L::cy(i)) * dif;
            if (L::THERMAL) Me += C(L::c2cls(k)) * sum;
            put(i, g[i] + om * (gp - g[i]));
            put(i + 1, g[i + 1] + om * (gm - g[i + 1]));
        }
        // |c| = 1 class: (1,0) and (-1,0) are velocities 1, 2; (0,1), (0,-1) are 3, 4
        const C a0 = e.A0 + ics2 * (e.B0 + e.C0 * ics2);
        const C a2 = e.A2 + e.B2 * ics2;
        const C px2 = uxs * uxs, py2 = uys * uys;
        const C ws0 = C(L::w(1)) * m.s0, wr = C(L::w(1)) * m.rho;
        C ex = ws0 + wr * (a0 + px2 * (a2 + px2 * a4));
        C ey = ws0 + wr * (a0 + py2 * (a2 + py2 * a4));
        if (L::THERMAL) {
            const C d = C(0.25) * (m.se - Me - C(2) * (ex + ey));
            ex += d;
            ey += d;
        }
        const C ox = C(0.5) * (m.sx - Mx), oy = C(0.5) * (m.sy - My);
        put(1, g[1] + om * (ex + ox - g[1]));
        put(2, g[2] + om * (ex - ox - g[2]));
        put(3, g[3] + om * (ey + oy - g[3]));
        put(4, g[4] + om * (ey - oy - g[4]));
        const C geq0 = m.s0 - M0 - C(2) * (ex + ey);
        put(0, g[0] + om * (geq0 - g[0]));
    }

    // Strip export for the characteristic boundary solver.
    const bool near = (E.cbc[0] && x - G.M <= 2) || (E.cbc[1] && G.nx - 1 - G.M - x <= 2) ||
                      (E.cbc[2] && y - G.M <= 2) || (E.cbc[3] && G.ny - 1 - G.M - y <= 2);
    if (EXPORT && near) export_from<LAT, C>(G, E, g, m, x, y, par_new);
}

template <int LAT, typename S>
__global__ void __launch_bounds__(kBulkThreads)
    k_bulk(const __grid_constant__ Maps tm, Geom G, Offsets O, Export E, Region R,
           const S* __restrict__ fin, S* __restrict__ fout, int par_new, int* status)
{
    using L = Lat<LAT>;
    using C = typename Store<S>::C;
    using BX = Stage<LAT, S>;
    constexpr int Q = L::Q;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar;
    const int x0 = (R.x0 / kBulkThreads + blockIdx.x) * kBulkThreads;   // tiles aligned to 128
    const int x = x0 + threadIdx.x;
    const int y = R.y0 + blockIdx.y;
    const bool valid = x >= R.x0 && x < R.x1;

    // Pull stream (Eq. lbe): g_i(x) = g*_i(x - c_i).  Segments whose sources
    // wrap around a periodic axis use plain loads; all others stage the 37
    // shifted source rows through shared memory with tensor copies.
    const bool wrap = (G.pery && (y < L::M || y >= G.ny - L::M)) ||
                      (G.perx && (x0 - L::M < 0 || x0 + kBulkThreads + L::M > G.nx));
    C g[Q];
    if (!wrap) {
        S* sb = reinterpret_cast<S*>(smem_raw);
        if (threadIdx.x == 0) {
            const unsigned b = smem_u32(&bar);
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         ::"r"(b), "r"(BX::TX) : "memory");
            issue_copies<LAT, S>(tm, smem_raw, x0, y, b, std::make_integer_sequence<int, L::NG>{});
        }
        __syncthreads();
        if (!wait_tx(&bar, status) || !valid) return;
        gather_staged<LAT, S, C>(g, sb, threadIdx.x, std::make_integer_sequence<int, Q>{});
    } else {
        if (!valid) return;
        pull_plain<LAT, S, C>(G, O, fin, x, y, g);
    }
    collide_store<LAT, S, C, false>(G, O, E, fin, fout, x, y, par_new, g);   // never near a side
}

// The rim bands: one thread per node, plain loads (the bands are a few
// nodes wide, too narrow for row-segment staging).
template <int LAT, typename S>
__global__ void __launch_bounds__(kBulkThreads)
    k_rim(Geom G, Offsets O, Export E, Rim RM, const S* __restrict__ fin, S* __restrict__ fout,
          int par_new)
{
    using C = typename Store<S>::C;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= RM.total) return;
    // band of node k, selected with constant indices (no local copy of RM)
    int bx0 = RM.r[0].x0, bw = RM.r[0].x1 - RM.r[0].x0, by0 = RM.r[0].y0, b0 = 0;
#pragma unroll
    for (int j = 1; j < 4; ++j)
        if (j < RM.n && k >= RM.start[j]) {
            bx0 = RM.r[j].x0;
            bw = RM.r[j].x1 - RM.r[j].x0;
            by0 = RM.r[j].y0;
            b0 = RM.start[j];
        }
    const int l = k - b0;
    const int x = bx0 + l % bw, y = by0 + l / bw;
    C g[Lat<LAT>::Q];
    pull_plain<LAT, S, C>(G, O, fin, x, y, g);
    collide_store<LAT, S, C, true>(G, O, E, fin, fout, x, y, par_new, g);
}

template <int LAT, typename S>
__global__ void k_init(Geom G, Export E, const double* __restrict__ rho,
                       const double* __restrict__ ux, const double* __restrict__ uy,
                       const double* __restrict__ T, S* __restrict__ f)
{
    using L = Lat<LAT>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    const long long n = (long long)y * G.nx + x;
    Moments<LAT, double> m;
    m.s0 = rho[n] - G.rho0;
    m.rho = rho[n];
    m.ux = ux[n];
    m.uy = uy[n];
    m.dT = L::THERMAL ? T[n] - 1.0 : 0.0;
    double geq[L::Q];
    equilibrium<LAT, double>(m, geq);
    S* out = f + (long long)y * G.nxp + x;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        double v = geq[i];
        if (Store<S>::SCALED) v *= 1.0 / L::w(i);
        Store<S>::put(out + (long long)L::plane_of(i) * G.plane, typename Store<S>::C(v));
    }
    // strips of time 0 (parity 0): U0 and zero non-equilibrium moments
    const int dd[4] = {x - G.M, G.nx - 1 - G.M - x, y - G.M, G.ny - 1 - G.M - y};
    const bool inbx = (G.perx || (x >= G.M && x < G.nx - G.M));
    const bool inby = (G.pery || (y >= G.M && y < G.ny - G.M));
    if (!(inbx && inby)) return;
    const double U[4] = {m.s0, m.ux, m.uy, m.dT};
    for (int s = 0; s < 4; ++s) {
        if (!E.cbc[s] || dd[s] < 0 || dd[s] > 2) continue;
        const int p = s < 2 ? y : x;
        const long long slot = E.offS[s] + dd[s] * E.L[s] + p;
        double* u = E.stripU + slot * 4;
        double* nn = E.stripN + slot * 5;
        for (int c = 0; c < 4; ++c) u[c] = U[c];
        for (int c = 0; c < 5; ++c) nn[c] = 0.0;
    }
}

template <int LAT, typename S>
__global__ void k_inflow(Geom G, const int* __restrict__ nodes, int n, double d0, double d1,
                         double d2, double d3, S* __restrict__ f)
{
    using L = Lat<LAT>;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    Moments<LAT, double> m;
    m.s0 = d0;
    m.rho = G.rho0 + d0;
    m.ux = d1;
    m.uy = d2;
    m.dT = L::THERMAL ? d3 : 0.0;
    double geq[L::Q];
    equilibrium<LAT, double>(m, geq);
    const long long node = nodes[k];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        double v = geq[i];
        if (Store<S>::SCALED) v *= 1.0 / L::w(i);
        Store<S>::put(f + L::plane_of(i) * G.plane + node, typename Store<S>::C(v));
    }
}

__global__ void k_init_band(Geom G, Band B, const double* __restrict__ rho,
                            const double* __restrict__ ux, const double* __restrict__ uy,
                            const double* __restrict__ T, int thermal)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= B.n_unk) return;
    const UDesc& D = B.ud[u];
    // the written node of a side layer, the innermost node of a corner block
    int node = D.wnode;
    if (D.kind >= 4) node += (G.M - 1) * (D.wdx + D.wdy);
    const int y = node / G.nxp, x = node - y * G.nxp;
    const long long n = (long long)y * G.nx + x;
    double* U = B.Ub + 4 * (long long)u;
    U[0] = rho[n] - G.rho0;
    U[1] = ux[n];
    U[2] = uy[n];
    U[3] = thermal ? T[n] - 1.0 : 0.0;
}

template <int LAT, typename S>
__global__ void k_macros(Geom G, const S* __restrict__ f, double* __restrict__ rho,
                         double* __restrict__ ux, double* __restrict__ uy, double* __restrict__ T,
                         int* flag)
{
    using L = Lat<LAT>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    const S* in = f + (long long)y * G.nxp + x;
    double g[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        double v = double(Store<S>::load(in + (long long)L::plane_of(i) * G.plane));
        if (Store<S>::SCALED) v *= L::w(i);
        g[i] = v;
    }
    const Moments<LAT, double> m = moments<LAT, double>(g, G.rho0);
    const long long n = (long long)y * G.nx + x;
    rho[n] = G.rho0 + m.s0;
    ux[n] = m.ux;
    uy[n] = m.uy;
    T[n] = 1.0 + m.dT;
    if (!isfinite(m.s0) || !isfinite(m.ux) || !isfinite(m.uy) || !isfinite(m.dT)) atomicOr(flag, 1);
}

template <int LAT, typename S>
int init_t(const Geom& G, const Export& E, const Band& B, const double* rho, const double* ux,
           const double* uy, const double* T, void* f, cudaStream_t st)
{
    dim3 blk(128), grd((G.nx + 127) / 128, G.ny);
    k_init<LAT, S><<<grd, blk, 0, st>>>(G, E, rho, ux, uy, T, static_cast<S*>(f));
    if (B.n_unk > 0)
        k_init_band<<<(B.n_unk + 127) / 128, 128, 0, st>>>(G, B, rho, ux, uy, T, Lat<LAT>::THERMAL);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int LAT, typename S>
int inflow_t(const Geom& G, const int* nodes, int n, const double U[4], void* f, cudaStream_t st)
{
    if (n <= 0) return 0;
    k_inflow<LAT, S><<<(n + 127) / 128, 128, 0, st>>>(G, nodes, n, U[0], U[1], U[2], U[3],
                                                     static_cast<S*>(f));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int LAT, typename S>
int bulk_t(const Geom& G, const Offsets& O, const Export& E, const Region& R,
           const CUtensorMap* tmaps, const void* fin, void* fout, int par_new, int* status,
           cudaStream_t st)
{
    const int h = R.y1 - R.y0;
    if (R.x1 <= R.x0 || h <= 0) return 0;
    const int t0 = R.x0 / kBulkThreads, t1 = (R.x1 + kBulkThreads - 1) / kBulkThreads;
    const size_t smem = Stage<LAT, S>::TOTAL;
    Maps tm;
    tm.m7 = tmaps[0];
    tm.m5 = tmaps[1];
    tm.m3 = tmaps[2];
    dim3 blk(kBulkThreads), grd(t1 - t0, h);
    k_bulk<LAT, S><<<grd, blk, smem, st>>>(tm, G, O, E, R, static_cast<const S*>(fin),
                                           static_cast<S*>(fout), par_new, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int LAT, typename S>
int rim_t(const Geom& G, const Offsets& O, const Export& E, const Rim& RM, const void* fin,
          void* fout, int par_new, cudaStream_t st)
{
    const int n = RM.total;
    if (n <= 0) return 0;
    k_rim<LAT, S><<<(n + kBulkThreads - 1) / kBulkThreads, kBulkThreads, 0, st>>>(
        G, O, E, RM, static_cast<const S*>(fin), static_cast<S*>(fout), par_new);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int LAT, typename S>
int macros_t(const Geom& G, const void* f, double* rho, double* ux, double* uy, double* T,
             int* flag, cudaStream_t st)
{
    dim3 blk(128), grd((G.nx + 127) / 128, G.ny);
    k_macros<LAT, S><<<grd, blk, 0, st>>>(G, static_cast<const S*>(f), rho, ux, uy, T, flag);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

#define LBM_DISPATCH(lat, storage, CALL)                                   \
    do {                                                                   \
        if (lat == D2Q9) {                                                 \
            if (storage == 0) return CALL(D2Q9, double);                   \
            if (storage == 1) return CALL(D2Q9, float);                    \
            if (storage == 2) return CALL(D2Q9, __half);                   \
        } else {                                                           \
            if (storage == 0) return CALL(D2Q37, double);                  \
            if (storage == 1) return CALL(D2Q37, float);                   \
            if (storage == 2) return CALL(D2Q37, __half);                  \
        }                                                                  \
        return -1;                                                         \
    } while (0)

int launch_init(int lat, int storage, const Geom& G, const Export& E, const Band& B,
                const double* rho, const double* ux, const double* uy, const double* T, void* f,
                cudaStream_t st)
{
#define CALL(L, S) init_t<L, S>(G, E, B, rho, ux, uy, T, f, st)
    LBM_DISPATCH(lat, storage, CALL);
#undef CALL
}

int launch_inflow(int lat, int storage, const Geom& G, const int* nodes, int n, const double Uin[4],
                  void* f, cudaStream_t st)
{
#define CALL(L, S) inflow_t<L, S>(G, nodes, n, Uin, f, st)
    LBM_DISPATCH(lat, storage, CALL);
#undef CALL
}

int launch_bulk(int lat, int storage, const Geom& G, const Offsets& O, const Export& E,
                const Region& R, const CUtensorMap* tmaps, const void* fin, void* fout,
                int par_new, int* status, cudaStream_t st)
{
#define CALL(L, S) bulk_t<L, S>(G, O, E, R, tmaps, fin, fout, par_new, status, st)
    LBM_DISPATCH(lat, storage, CALL);
#undef CALL
}

int launch_rim(int lat, int storage, const Geom& G, const Offsets& O, const Export& E,
               const Rim& RM, const void* fin, void* fout, int par_new, cudaStream_t st)
{
#define CALL(L, S) rim_t<L, S>(G, O, E, RM, fin, fout, par_new, st)
    LBM_DISPATCH(lat, storage, CALL);
#undef CALL
}

int launch_macros(int lat, int storage, const Geom& G, const void* f, double* rho, double* ux,
                  double* uy, double* T, int* flag, cudaStream_t st)
{
#define CALL(L, S) macros_t<L, S>(G, f, rho, ux, uy, T, flag, st)
    LBM_DISPATCH(lat, storage, CALL);
#undef CALL
}

}  // namespace lbmgb
