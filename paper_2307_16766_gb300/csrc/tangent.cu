// tangent.cu -- the tangent-linear step: one time step of the method (the
// same strip macros, characteristic boundary solver, Dirichlet write and
// fused pull-stream + BGK collide) evaluated on Dual numbers, so that the
// populations, the boundary state and a pressure loss carry their
// derivatives along three directions in the space of the incoming-wave
// relaxation parameters (Eqs. LODI-Relax, CBC-Relax): alpha_T, beta_P, P_inf,
// alpha_V (the viscous term's relaxation) and t_inf.
//
//   k_tl_strip     macros of the strip nodes at t (the first step's seed)
//   k_tl_bulk      (first) pull-stream + BGK collide of every bulk node, one
//                  derivative direction at a time, the macros of t + 1 of
//                  the strip nodes (Eq. lbe, Eq. macro), and the loss of the
//                  node: J += (P - P_ref)^2 and its derivatives,
//                  P - c_s^2 rho0 = c_s^2 (drho + rho0 dT + drho dT)
//   k_tl_stage     one RK4 stage of every boundary unknown (Sec. 3.3),
//                  right-hand side from charsys.cuh on Dual numbers of the
//                  storage's arithmetic, state and RK4 sum with FP64 values
//   k_tl_dirichlet f^eq of the new boundary state on the band nodes
//                  (equilibrium Dirichlet condition)
//
//   k_tl_neq       (mesoscopic viscous vector) non-equilibrium moments of
//                  the strip nodes at t + 1 (Eqs. LaplaceU, LaplaceT)
//
// Supported: FP64 and FP32 storage, equilibrium Dirichlet condition, any
// viscous vector (frozen at time t, as in the ordinary step),
// characteristic and periodic sides (checked on the host).
#include "charsys.cuh"

#include <type_traits>

namespace lbmgb {

namespace {

constexpr int kTD = 3;                      // derivative directions

// Boundary state and RK4 sum: FP64 value (the state accumulates over the
// steps, as in the ordinary step) with FP32 derivatives.  Only the linear
// RK4 bookkeeping is done on it.
struct TS {
    double v;
    float d[kTD];
};

template <typename C>
__device__ __forceinline__ TS ts_axpy(const TS& a, double w, const C& k)
{
    // a + w k
    TS r;
    r.v = a.v + w * double(k.v);
#pragma unroll
    for (int q = 0; q < kTD; ++q) r.d[q] = a.d[q] + float(w) * float(k.d[q]);
    return r;
}
// arithmetic of the strips, stage values and right-hand sides: the
// storage's (FP32 inputs around an FP64 state with FP32 storage)
template <typename S>
using TB = Dual<typename Store<S>::C, kTD>;

template <typename To, typename From>
__device__ __forceinline__ To dcast(const From& a)
{
    // element types by value (an element expression's decltype is a
    // reference, and casting to it would reinterpret the source's bytes)
    using V = std::remove_cv_t<std::remove_reference_t<decltype(To{}.v)>>;
    using E = std::remove_cv_t<std::remove_reference_t<decltype(To{}.d[0])>>;
    To r;
    r.v = static_cast<V>(a.v);
#pragma unroll
    for (int k = 0; k < kTD; ++k) r.d[k] = static_cast<E>(a.d[k]);
    return r;
}

// Populations (value and derivative planes) of node `off` as Dual numbers.
template <int LAT, typename S, typename C>
__device__ __forceinline__ void load_node(const Geom& G, const S* f, const S* t, long long off, C* g)
{
    using L = Lat<LAT>;
    const long long dstride = (long long)L::Q * G.plane;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const long long o = (long long)L::plane_of(i) * G.plane + off;
        g[i].v = f[o];
#pragma unroll
        for (int k = 0; k < kTD; ++k) g[i].d[k] = t[k * dstride + o];
    }
}

// Source offset of velocity i's pull (Eq. lbe) at node (x, y), periodic
// wrap-around.
template <int LAT>
__device__ __forceinline__ long long pull_src(const Geom& G, int i, int x, int y)
{
    using L = Lat<LAT>;
    int xs = x - L::cx(i), ys = y - L::cy(i);
    if (L::cx(i) && G.perx) xs = xs < 0 ? xs + G.nx : (xs >= G.nx ? xs - G.nx : xs);
    if (L::cy(i) && G.pery) ys = ys < 0 ? ys + G.ny : (ys >= G.ny ? ys - G.ny : ys);
    return (long long)L::plane_of(i) * G.plane + (long long)ys * G.nxp + xs;
}

template <int LAT, typename S, typename C>
__device__ __forceinline__ void pull_node(const Geom& G, const S* f, const S* t, int x, int y, C* g)
{
    using L = Lat<LAT>;
    const long long dstride = (long long)L::Q * G.plane;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const long long o = pull_src<LAT>(G, i, x, y);
        g[i].v = f[o];
#pragma unroll
        for (int k = 0; k < kTD; ++k) g[i].d[k] = t[k * dstride + o];
    }
}

// The node of strip slot q, or false if it is not a bulk node (no unknown
// reads those slots).
__device__ __forceinline__ bool slot_node(const Geom& G, const Export& E, int q, int& x, int& y)
{
    int s = -1;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (E.cbc[k] && q >= E.offS[k] && q < E.offS[k] + E.ND * E.L[k]) s = k;
    if (s < 0) return false;
    const int r = q - E.offS[s], d = r / E.L[s], p = r % E.L[s];
    const int M = G.M;
    if (s == 0) { x = M + d; y = p; }
    else if (s == 1) { x = G.nx - 1 - M - d; y = p; }
    else if (s == 2) { x = p; y = M + d; }
    else { x = p; y = G.ny - 1 - M - d; }
    const bool inbx = G.perx || (x >= M && x < G.nx - M);
    const bool inby = G.pery || (y >= M && y < G.ny - M);
    return inbx && inby;
}

// Strip macros of time t from the stored (post-collision) populations,
// which carry the macros of t (the collision keeps them): the seed of the
// first tangent-linear step; later steps take them from the bulk pass of the
// step before.
template <int LAT, typename S>
__global__ void k_tl_strip(Geom G, Export E, const S* __restrict__ f, const S* __restrict__ t,
                           TB<S>* __restrict__ St)
{
    using L = Lat<LAT>;
    using C = TB<S>;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= E.nslots) return;
    int x = 0, y = 0;
    C* a = St + 4LL * q;
    if (!slot_node(G, E, q, x, y)) {
#pragma unroll
        for (int c = 0; c < 4; ++c) a[c] = C(0);
        return;
    }
    C g[L::Q];
    load_node<LAT, S, C>(G, f, t, (long long)y * G.nxp + x, g);
    const Moments<LAT, C> m = moments<LAT, C>(g, rho0_of<C>(G));
    a[0] = m.s0; a[1] = m.ux; a[2] = m.uy; a[3] = m.dT;
}

// Non-equilibrium moments (sigma', q) of the strip nodes at t + 1, from
// their pulled (pre-collision) populations, for the mesoscopic viscous
// vector of the next step; the same arithmetic as the ordinary step's strip
// phase, on Dual numbers.
template <int LAT, typename S>
__global__ void k_tl_neq(Geom G, Export E, const S* __restrict__ f, const S* __restrict__ t,
                         TB<S>* __restrict__ StN1)
{
    using L = Lat<LAT>;
    using C = TB<S>;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= E.nslots) return;
    int x = 0, y = 0;
    C* a = StN1 + 5LL * q;
    if (!slot_node(G, E, q, x, y)) {
#pragma unroll
        for (int c = 0; c < 5; ++c) a[c] = C(0);
        return;
    }
    // one derivative direction at a time (Dual<., 1>), as in the bulk pass
    using C1 = Dual<typename Store<S>::C, 1>;
    const long long dstride = (long long)L::Q * G.plane;
#pragma unroll 1
    for (int k = 0; k < kTD; ++k) {
        C1 g[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const long long o = pull_src<LAT>(G, i, x, y);
            g[i].v = f[o];
            g[i].d[0] = t[k * dstride + o];
        }
        const Moments<LAT, C1> m = moments<LAT, C1>(g, rho0_of<C1>(G));
        C1 N[5];
        neq_moments<LAT, C1, C1>(g, m, C1(1) - C1(0.5) * omega_of<C1>(G), N);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            if (k == 0) a[c].v = N[c].v;
            a[c].d[k] = N[c].d[0];
        }
    }
}

// The strips' non-equilibrium moments of time t from the handle's own
// strips (values), with zero derivatives: the first tangent-linear step's
// seed.
template <typename S>
__global__ void k_tl_seed_neq(Export E, const typename StripReal<S>::T* __restrict__ SN, TB<S>* StN)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= E.nslots) return;
#pragma unroll
    for (int c = 0; c < 5; ++c) StN[5LL * q + c] = TB<S>(typename Store<S>::C(SN[5LL * q + c]));
}

// One RK4 stage of every boundary unknown.  Ud, acc: state and sum of k
// (FP64); Uf: the state in the stage type, for the neighbours' stencils;
// Ya, Yb: stage values; mask: incoming waves at t.
template <int LAT, typename S>
__global__ void k_tl_stage(Geom G, Band B, Relax<TB<S>> P, const TB<S>* __restrict__ St,
                           const TB<S>* __restrict__ St1, const TB<S>* __restrict__ StN, TS* Ud,
                           TB<S>* Uf, TB<S>* Ya, TB<S>* Yb, TS* acc, int* mask, TB<S>* Vv, int stage)
{
    using Lt = Lat<LAT>;
    using T = TB<S>;
    // stage 0 reads only time t: the bulk pass launched after it for early
    // start (it writes only t + 1) may begin now
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // stages 2 and 3 start early behind the stage before them: wait for it
    // (and its memory) before reading what it wrote
    if (stage >= 2) asm volatile("griddepcontrol.wait;" ::: "memory");
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= B.n_unk) return;
    const UDesc D = B.ud[u];
    CtxT<T> X;
    X.Y = stage == 0 ? Uf : (stage == 2 ? Yb : Ya);
    X.St = St;
    X.St1 = St1;
    X.frac = stage == 0 ? T(0) : (stage == 3 ? T(1) : T(0.5));
    T* Yout = stage == 1 ? Yb : Ya;
    // viscous vector: of time t at stage 0, then frozen for the later
    // stages (corners take none)
    T V[4] = {T(0), T(0), T(0), T(0)};
    if (B.viscous != VIS_OFF && D.kind < 4) {
        T* Vu = Vv + 4LL * u;
        if (stage == 0) {
            if (B.viscous == VIS_FD) vis_fd<Lt::THERMAL>(G, B, X, D, u, Lt::CS2, V);
            else vis_meso<Lt::THERMAL>(G, St, 4, StN, 5, D, Lt::CS2, V);
#pragma unroll
            for (int m = 0; m < 4; ++m) Vu[m] = V[m];
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) V[m] = Vu[m];
        }
    }
    int mk;
    if (stage == 0) {
        T Ul[4];
        to_local(D.kind, T(B.kR), Uf + 4LL * u, Ul);
        mk = incoming_mask<Lt::THERMAL>(char_sys<Lt::THERMAL>(B, G.rho0, Ul));
        mask[u] = mk;
    } else {
        mk = mask[u];
    }
    T k[4];
    unknown_rhs<LAT, T>(G, B, P, X, D, u, V, mk, k);
    TS* U0 = Ud + 4LL * u;
    TS* ac = acc + 4LL * u;
    if (stage < 3) {
        const double wk = stage == 0 ? 1.0 : 2.0;
        const double hk = stage == 2 ? 1.0 : 0.5;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            ac[m] = ts_axpy(stage == 0 ? TS{0.0, {0.f, 0.f, 0.f}} : ac[m], wk, k[m]);
            Yout[4LL * u + m] = dcast<T>(ts_axpy(U0[m], hk, k[m]));
        }
    } else {
        // RK4: U(t + 1) = U(t) + (k1 + 2 k2 + 2 k3 + k4) / 6
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            TS s = ts_axpy(ac[m], 1.0, k[m]);
            U0[m] = ts_axpy(U0[m], 1.0 / 6.0, s);
            Uf[4LL * u + m] = dcast<T>(U0[m]);
        }
    }
}

// Equilibrium Dirichlet condition of the new boundary state: f^eq on the
// unknown's band node (corner: its M x M block), value and derivatives, in
// the storage's arithmetic.  Thread (u, k) takes derivative direction k of
// unknown u on Dual<., 1> numbers (direction 0 also writes the values):
// three short chains per unknown instead of one long one.
template <int LAT, typename S>
__global__ void k_tl_dirichlet(Geom G, Band B, const TB<S>* __restrict__ Uf, S* __restrict__ f,
                               S* __restrict__ t)
{
    using L = Lat<LAT>;
    using C1 = Dual<typename Store<S>::C, 1>;
    // launched early behind the last stage: wait for it
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (u >= B.n_unk) return;
    const UDesc D = B.ud[u];
    const TB<S>* U = Uf + 4LL * u;
    C1 Uk[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        Uk[c].v = U[c].v;
        Uk[c].d[0] = U[c].d[k];
    }
    Moments<LAT, C1> m;
    m.s0 = Uk[0];
    m.rho = rho0_of<C1>(G) + m.s0;
    m.ux = Uk[1];
    m.uy = Uk[2];
    m.dT = L::THERMAL ? Uk[3] : C1(0);
    C1 ge[L::Q];
    equilibrium<LAT, C1>(m, ge);
    const long long dstride = (long long)L::Q * G.plane;
    const int nb = D.kind >= 4 ? G.M : 1;
    for (int a = 0; a < nb; ++a)
        for (int b = 0; b < nb; ++b) {
            const long long node = D.wnode + a * D.wdx + b * D.wdy;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const long long o = (long long)L::plane_of(i) * G.plane + node;
                if (k == 0) f[o] = S(ge[i].v);
                t[k * dstride + o] = S(ge[i].d[0]);
            }
        }
}

// Pull-stream + BGK collide of every bulk node, one derivative direction
// at a time (Dual<C, 1>: the three passes share the pulled values), and the
// loss of the node: the bulk nodes are the nodes off the boundary layers,
// and the collision keeps the macros, so the pulled populations' moments
// give P at t + 1.
// Threads of a bulk-pass CTA: the pulled populations of one direction are
// staged in shared memory, a column per thread (37 x 128 FP32 Dual numbers
// or 37 x 64 FP64 ones: 37 KB), rather than held in registers, and the
// registers are capped so that four FP32 CTAs share an SM (the collision's
// working set then spills a few words; at two CTAs per SM, uncapped, the
// pass ran 1.2x slower).
template <typename S>
constexpr int tl_bulk_threads() { return sizeof(typename Store<S>::C) == 8 ? 64 : 128; }
template <typename S>
constexpr int tl_bulk_min_blocks() { return sizeof(typename Store<S>::C) == 8 ? 1 : 4; }

template <int LAT, typename S>
__global__ void __launch_bounds__(tl_bulk_threads<S>(), tl_bulk_min_blocks<S>())
    k_tl_bulk(Geom G, Region R, Export E, const S* __restrict__ f, const S* __restrict__ t,
              S* __restrict__ fo, S* __restrict__ to, TB<S>* __restrict__ St1,
              const double* __restrict__ dPref, double* sums)
{
    using L = Lat<LAT>;
    using C1 = Dual<typename Store<S>::C, 1>;
    constexpr int NT = tl_bulk_threads<S>();
    __shared__ C1 sg[L::Q][NT];
    const int l = threadIdx.x;
    const int x = R.x0 + blockIdx.x * NT + l;
    const int y = R.y0 + blockIdx.y;
    double acc[kTD + 1] = {0.0, 0.0, 0.0, 0.0};
    if (x < R.x1) {
        const long long node = (long long)y * G.nxp + x;
        const long long dstride = (long long)L::Q * G.plane;
        // strip slots of this node (depth 0 .. ND - 1 inside a
        // characteristic side; on a small grid a node can lie in the strips
        // of all four sides): its macros at t + 1
        int slot[4] = {-1, -1, -1, -1}, ns = 0;
        {
            const int dd[4] = {x - G.M, G.nx - 1 - G.M - x, y - G.M, G.ny - 1 - G.M - y};
#pragma unroll
            for (int s = 0; s < 4; ++s)
                if (E.cbc[s] && dd[s] >= 0 && dd[s] < E.ND)
                    slot[ns++] = E.offS[s] + dd[s] * E.L[s] + (s < 2 ? y : x);
        }
        double e = 0.0;
#pragma unroll 1
        for (int k = 0; k < kTD; ++k) {
            // offsets inside one buffer fit in 32 bits (the grid check keeps
            // Q x plane below 2^31); direction k's planes start at tk / tok
            const S* tk = t + k * dstride;
            S* tok = to + k * dstride;
            // pull (Eq. lbe) into the thread's column, summing the moments
            // as moments() does
            C1 s0 = 0, sx = 0, sy = 0, se = 0;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const int o = int(pull_src<LAT>(G, i, x, y));
                C1 g;
                g.v = f[o];
                g.d[0] = tk[o];
                sg[i][l] = g;
                s0 += g;
                if (L::cx(i)) sx += C1(L::cx(i)) * g;
                if (L::cy(i)) sy += C1(L::cy(i)) * g;
                if (L::THERMAL && i) se += C1(L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i)) * g;
            }
            // read the column back below rather than keeping it in registers
            asm volatile("" ::: "memory");
            const Moments<LAT, C1> m = moments_of_sums<LAT, C1>(s0, sx, sy, se, rho0_of<C1>(G));
            const int nd = int(node);
            collide_given<LAT, C1>(G, m, [&](int i) -> C1 { return sg[i][l]; }, [&](int i, const C1& v) {
                const int o = L::plane_of(i) * int(G.plane) + nd;
                if (k == 0) fo[o] = v.v;
                tok[o] = v.d[0];
            });
            asm volatile("" ::: "memory");
            for (int q = 0; q < ns; ++q) {
                TB<S>* a = St1 + 4LL * slot[q];
                const C1 mc[4] = {m.s0, m.ux, m.uy, m.dT};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (k == 0) a[c].v = mc[c].v;
                    a[c].d[k] = mc[c].d[0];
                }
            }
            // P - c_s^2 rho0 = c_s^2 (drho + rho0 dT + drho dT)
            const double s0v = double(m.s0.v), dT = double(m.dT.v);
            const double s0d = double(m.s0.d[0]), dTd = double(m.dT.d[0]);
            if (k == 0) {
                const double dP = L::THERMAL ? L::CS2 * (s0v + G.rho0 * dT + s0v * dT) : L::CS2 * s0v;
                e = dP - (dPref ? dPref[(long long)y * G.nx + x] : 0.0);
                acc[0] = e * e;
            }
            const double dPd = L::THERMAL ? L::CS2 * (s0d + G.rho0 * dTd + s0d * dT + s0v * dTd) : L::CS2 * s0d;
            acc[k + 1] = 2.0 * e * dPd;
        }
    }
    constexpr int NW = NT / 32;
    __shared__ double red[kTD + 1][NW];
#pragma unroll
    for (int c = 0; c < kTD + 1; ++c) {
        double a = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if ((l & 31) == 0) red[c][l >> 5] = a;
    }
    __syncthreads();
    if (l < kTD + 1) {
        double a = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) a += red[l][w];
        atomicAdd(sums + l, a);
    }
}

template <int LAT, typename S>
int tl_step_t(const TLState& T, const Geom& G, const Export& E, const Band& B, const Region& bulk,
              void* const f[2], int par, const double* dPref, cudaStream_t st)
{
    using R = TB<S>;
    const S* fi = static_cast<const S*>(f[par]);
    S* fo = static_cast<S*>(f[par ^ 1]);
    const S* ti = static_cast<const S*>(T.t[par]);
    S* to = static_cast<S*>(T.t[par ^ 1]);
    R* St = static_cast<R*>(T.strip[par]);
    R* St1 = static_cast<R*>(T.strip[par ^ 1]);
    // the parameters as Dual numbers seeded with the three directions
    Relax<R> P;
    P.alpha_T = R(B.alpha_T);
    P.beta_P = R(B.beta_P);
    P.alpha_V = R(B.alpha_V);
    P.t_inf = R(B.t_inf);
    for (int s = 0; s < 4; ++s) P.pdev[s] = R(B.pdev[s]);
    using Ed = typename Store<S>::C;
    for (int k = 0; k < kTD; ++k) {
        P.alpha_T.d[k] = Ed(T.dirs[k][0]);
        P.beta_P.d[k] = Ed(T.dirs[k][1]);
        for (int s = 0; s < 4; ++s) P.pdev[s].d[k] = Ed(T.dirs[k][2]);
        P.alpha_V.d[k] = Ed(T.dirs[k][3]);
        P.t_inf.d[k] = Ed(T.dirs[k][4]);
    }
    // RK4 stage 0 (time t only) and, beside it by programmatic launch, the
    // bulk pass, which also gives the strip macros of t + 1 that stages 1-3
    // read; stages 1-3 and the Dirichlet write follow in stream order
    const int nb = (B.n_unk + 127) / 128;
    auto stage = [&](int k, bool early) {
        return launch_ex(k_tl_stage<LAT, S>, dim3(nb), dim3(128), 0, st, early, G, B, P,
                         static_cast<const R*>(St), static_cast<const R*>(St1),
                         static_cast<const R*>(T.stripN[par]), static_cast<TS*>(T.Ud),
                         static_cast<R*>(T.Uf), static_cast<R*>(T.Ya), static_cast<R*>(T.Yb),
                         static_cast<TS*>(T.acc), T.mask, static_cast<R*>(T.Vv), k);
    };
    bool first = true;
    if (B.n_unk > 0) {
        if (stage(0, false)) return -1;
        first = false;
    }
    if (bulk.x1 > bulk.x0 && bulk.y1 > bulk.y0) {
        constexpr int NT = tl_bulk_threads<S>();
        dim3 grd((bulk.x1 - bulk.x0 + NT - 1) / NT, bulk.y1 - bulk.y0);
        if (launch_ex(k_tl_bulk<LAT, S>, grd, dim3(NT), 0, st, !first, G, bulk, E, fi, ti, fo, to, St1, dPref,
                      T.sums))
            return -1;
    }
    if (B.n_unk > 0) {
        for (int k = 1; k < 4; ++k)
            if (stage(k, k >= 2)) return -1;
        if (launch_ex(k_tl_dirichlet<LAT, S>, dim3(nb, kTD), dim3(128), 0, st, true, G, B,
                      static_cast<const R*>(T.Uf), fo, to))
            return -1;
    }
    if (B.viscous == VIS_MESO && E.nslots > 0)
        k_tl_neq<LAT, S><<<(E.nslots + 127) / 128, 128, 0, st>>>(G, E, fi, ti, static_cast<R*>(T.stripN[par ^ 1]));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int LAT, typename S>
int tl_seed_strips_t(const TLState& T, const Geom& G, const Export& E, void* const f[2], int par,
                     cudaStream_t st)
{
    if (E.nslots == 0) return 0;
    const int nb = (E.nslots + 127) / 128;
    k_tl_strip<LAT, S><<<nb, 128, 0, st>>>(
        G, E, static_cast<const S*>(f[par]), static_cast<const S*>(T.t[par]), static_cast<TB<S>*>(T.strip[par]));
    using SR = typename StripReal<S>::T;
    k_tl_seed_neq<S><<<nb, 128, 0, st>>>(E, static_cast<const SR*>(E.stripN) + (long long)par * E.nslots * 5,
                                         static_cast<TB<S>*>(T.stripN[par]));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// boundary state of parity par -> Ud (and its copy Uf in the stage type)
template <typename S>
__global__ void k_tl_seed(Band B, TS* Ud, TB<S>* Uf, int par)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= B.n_unk) return;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        Ud[4LL * u + m] = TS{B.Ub[((long long)par * B.n_unk + u) * 4 + m], {0.f, 0.f, 0.f}};
        Uf[4LL * u + m] = dcast<TB<S>>(Ud[4LL * u + m]);
    }
}

#define TL_DISPATCH(lat, storage, CALL)                                    \
    do {                                                                   \
        if (storage == 0) {                                                \
            if (lat == D2Q9) return CALL(D2Q9, double);                    \
            if (lat == D2Q17) return CALL(D2Q17, double);                  \
            return CALL(D2Q37, double);                                    \
        }                                                                  \
        if (storage == 1) {                                                \
            if (lat == D2Q9) return CALL(D2Q9, float);                     \
            if (lat == D2Q17) return CALL(D2Q17, float);                   \
            return CALL(D2Q37, float);                                     \
        }                                                                  \
        return -1;                                                         \
    } while (0)

}  // namespace

size_t tl_dual_bytes() { return sizeof(TS) > sizeof(TB<double>) ? sizeof(TS) : sizeof(TB<double>); }

int launch_tl_step(int lat, int storage, const TLState& T, const Geom& G, const Export& E,
                   const Band& B, const Region& bulk, void* const f[2], int par, const double* dPref,
                   cudaStream_t st)
{
#define CALL(L, S) tl_step_t<L, S>(T, G, E, B, bulk, f, par, dPref, st)
    TL_DISPATCH(lat, storage, CALL);
#undef CALL
}

int launch_tl_seed(int lat, int storage, const TLState& T, const Geom& G, const Export& E, const Band& B,
                   void* const f[2], int par, cudaStream_t st)
{
    {
        const int rc = [&]() -> int {
#define CALL(L, S) tl_seed_strips_t<L, S>(T, G, E, f, par, st)
            TL_DISPATCH(lat, storage, CALL);
#undef CALL
        }();
        if (rc) return rc;
    }
    if (B.n_unk == 0) return 0;
    const int nb = (B.n_unk + 127) / 128;
    if (storage == 0)
        k_tl_seed<double><<<nb, 128, 0, st>>>(B, static_cast<TS*>(T.Ud), static_cast<TB<double>*>(T.Uf), par);
    else
        k_tl_seed<float><<<nb, 128, 0, st>>>(B, static_cast<TS*>(T.Ud), static_cast<TB<float>*>(T.Uf), par);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lbmgb
