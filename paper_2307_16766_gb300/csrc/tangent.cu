// tangent.cu -- the tangent-linear step: one time step of the method (the
// same strip macros, characteristic boundary solver, Dirichlet write and
// fused pull-stream + BGK collide) evaluated on Dual numbers, so that the
// populations, the boundary state and a pressure loss carry their
// derivatives with respect to the three parameters of the incoming-wave
// relaxation (Eqs. LODI-Relax, CBC-Relax): alpha_T, beta_P and P_inf.
//
//   k_tl_strip     macros of the strip nodes at t (their populations) and
//                  at t + 1 (pulled, Eq. lbe), value and derivatives
//   k_tl_stage     one RK4 stage of every boundary unknown (Sec. 3.3),
//                  right-hand side from charsys.cuh on Dual<double, 3>
//   k_tl_dirichlet f^eq of the new boundary state on the band nodes
//   k_tl_bulk      pull-stream + BGK collide of every bulk node on
//                  Dual<C, 3> (C the storage's arithmetic type)
//   k_tl_loss      J += sum over the loss region of (P - P_ref)^2 and its
//                  derivatives, P - c_s^2 rho0 = c_s^2 (drho + rho0 dT + drho dT)
//
// Supported: FP64 and FP32 storage, equilibrium Dirichlet condition, no
// viscous vector, characteristic and periodic sides (checked on the host).
#include "charsys.cuh"

namespace lbmgb {

namespace {

constexpr int kTD = 3;                      // derivative directions
using TD = Dual<double, kTD>;               // boundary solver type

template <typename C>
__device__ __forceinline__ TD to_td(const C& a)
{
    TD r;
    r.v = double(a.v);
#pragma unroll
    for (int k = 0; k < kTD; ++k) r.d[k] = double(a.d[k]);
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

// Pull (Eq. lbe) of node (x, y) as Dual numbers, periodic wrap-around.
template <int LAT, typename S, typename C>
__device__ __forceinline__ void pull_node(const Geom& G, const S* f, const S* t, int x, int y, C* g)
{
    using L = Lat<LAT>;
    const long long dstride = (long long)L::Q * G.plane;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        int xs = x - L::cx(i), ys = y - L::cy(i);
        if (L::cx(i) && G.perx) xs = xs < 0 ? xs + G.nx : (xs >= G.nx ? xs - G.nx : xs);
        if (L::cy(i) && G.pery) ys = ys < 0 ? ys + G.ny : (ys >= G.ny ? ys - G.ny : ys);
        const long long o = (long long)L::plane_of(i) * G.plane + (long long)ys * G.nxp + xs;
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
        if (E.cbc[k] && q >= E.offS[k] && q < E.offS[k] + 3 * E.L[k]) s = k;
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

template <int LAT, typename S>
__global__ void k_tl_strip(Geom G, Export E, const S* __restrict__ f, const S* __restrict__ t,
                           TD* __restrict__ St, TD* __restrict__ St1)
{
    using L = Lat<LAT>;
    using C = Dual<typename Store<S>::C, kTD>;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= E.nslots) return;
    int x = 0, y = 0;
    TD* a = St + 4LL * q;
    TD* b = St1 + 4LL * q;
    if (!slot_node(G, E, q, x, y)) {
#pragma unroll
        for (int c = 0; c < 4; ++c) a[c] = b[c] = TD(0);
        return;
    }
    C g[L::Q];
    // time t: the stored (post-collision) populations carry the macros of t
    load_node<LAT, S, C>(G, f, t, (long long)y * G.nxp + x, g);
    Moments<LAT, C> m = moments<LAT, C>(g, rho0_of<C>(G));
    a[0] = to_td(m.s0); a[1] = to_td(m.ux); a[2] = to_td(m.uy); a[3] = to_td(m.dT);
    // time t + 1: pulled
    pull_node<LAT, S, C>(G, f, t, x, y, g);
    m = moments<LAT, C>(g, rho0_of<C>(G));
    b[0] = to_td(m.s0); b[1] = to_td(m.ux); b[2] = to_td(m.uy); b[3] = to_td(m.dT);
}

// One RK4 stage of every boundary unknown: Y (stage values), acc (sum of
// k), U (state, updated in place at stage 3), mask (incoming waves at t).
template <int LAT>
__global__ void k_tl_stage(Geom G, Band B, Relax<TD> P, const TD* __restrict__ St,
                           const TD* __restrict__ St1, TD* Ud, TD* Ya, TD* Yb, TD* acc, int* mask,
                           int stage)
{
    using Lt = Lat<LAT>;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= B.n_unk) return;
    const UDesc D = B.ud[u];
    CtxT<TD> X;
    X.Y = stage == 0 ? Ud : (stage == 2 ? Yb : Ya);
    X.St = St;
    X.St1 = St1;
    X.frac = stage == 0 ? TD(0) : (stage == 3 ? TD(1) : TD(0.5));
    TD* Yout = stage == 1 ? Yb : Ya;
    const TD V[4] = {TD(0), TD(0), TD(0), TD(0)};
    int mk;
    if (stage == 0) {
        TD Ul[4];
        to_local(D.kind, TD(B.kR), Ud + 4LL * u, Ul);
        mk = incoming_mask<Lt::THERMAL>(char_sys<Lt::THERMAL>(B, G.rho0, Ul));
        mask[u] = mk;
    } else {
        mk = mask[u];
    }
    TD k[4];
    unknown_rhs<LAT, TD>(G, B, P, X, D, u, V, mk, k);
    TD* U0 = Ud + 4LL * u;
    TD* ac = acc + 4LL * u;
    if (stage < 3) {
        const double wk = stage == 0 ? 1.0 : 2.0;
        const double hk = stage == 2 ? 1.0 : 0.5;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            ac[m] = (stage == 0 ? TD(0) : ac[m]) + TD(wk) * k[m];
            Yout[4LL * u + m] = U0[m] + TD(hk) * k[m];
        }
        return;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) U0[m] = U0[m] + (ac[m] + k[m]) * TD(1.0 / 6.0);
}

// Equilibrium Dirichlet condition: f^eq(U_b(t + 1)) on the unknown's band
// node (corner: its M x M block), value and derivatives.
template <int LAT, typename S>
__global__ void k_tl_dirichlet(Geom G, Band B, const TD* __restrict__ Ud, S* __restrict__ f,
                               S* __restrict__ t)
{
    using L = Lat<LAT>;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= B.n_unk) return;
    const UDesc D = B.ud[u];
    const TD* U = Ud + 4LL * u;
    Moments<LAT, TD> m;
    m.s0 = U[0];
    m.rho = TD(G.rho0) + U[0];
    m.ux = U[1];
    m.uy = U[2];
    m.dT = L::THERMAL ? U[3] : TD(0);
    TD ge[L::Q];
    equilibrium<LAT, TD>(m, ge);
    const long long dstride = (long long)L::Q * G.plane;
    const int nb = D.kind >= 4 ? G.M : 1;
    for (int a = 0; a < nb; ++a)
        for (int b = 0; b < nb; ++b) {
            const long long node = D.wnode + a * D.wdx + b * D.wdy;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const long long o = (long long)L::plane_of(i) * G.plane + node;
                f[o] = S(ge[i].v);
#pragma unroll
                for (int k = 0; k < kTD; ++k) t[k * dstride + o] = S(ge[i].d[k]);
            }
        }
}

template <int LAT, typename S>
__global__ void __launch_bounds__(128) k_tl_bulk(Geom G, Region R, const S* __restrict__ f,
                                                 const S* __restrict__ t, S* __restrict__ fo,
                                                 S* __restrict__ to)
{
    using L = Lat<LAT>;
    using C = Dual<typename Store<S>::C, kTD>;
    const int x = R.x0 + blockIdx.x * blockDim.x + threadIdx.x;
    const int y = R.y0 + blockIdx.y;
    if (x >= R.x1) return;
    C g[L::Q];
    pull_node<LAT, S, C>(G, f, t, x, y, g);
    const long long node = (long long)y * G.nxp + x;
    const long long dstride = (long long)L::Q * G.plane;
    collide<LAT, C>(G, g, [&](int i, const C& v) {
        const long long o = (long long)L::plane_of(i) * G.plane + node;
        fo[o] = v.v;
#pragma unroll
        for (int k = 0; k < kTD; ++k) to[k * dstride + o] = v.d[k];
    });
}

// J += sum (dP - dP_ref)^2 and dJ_k += sum 2 (dP - dP_ref) dP'_k over the
// loss region; sums[0] = J, sums[1..3] = dJ.  dP_ref: [ny][nx] or null.
template <int LAT, typename S>
__global__ void __launch_bounds__(128) k_tl_loss(Geom G, Region R, const S* __restrict__ f,
                                                 const S* __restrict__ t,
                                                 const double* __restrict__ dPref, double* sums)
{
    using L = Lat<LAT>;
    using C = Dual<typename Store<S>::C, kTD>;
    const int x = R.x0 + blockIdx.x * blockDim.x + threadIdx.x;
    const int y = R.y0 + blockIdx.y;
    double v[kTD + 1] = {0.0, 0.0, 0.0, 0.0};
    if (x < R.x1) {
        C g[L::Q];
        load_node<LAT, S, C>(G, f, t, (long long)y * G.nxp + x, g);
        const Moments<LAT, C> m = moments<LAT, C>(g, rho0_of<C>(G));
        const TD s0 = to_td(m.s0), dT = to_td(m.dT);
        const TD dP = L::THERMAL ? TD(L::CS2) * (s0 + TD(G.rho0) * dT + s0 * dT) : TD(L::CS2) * s0;
        const double e = dP.v - (dPref ? dPref[(long long)y * G.nx + x] : 0.0);
        v[0] = e * e;
#pragma unroll
        for (int k = 0; k < kTD; ++k) v[k + 1] = 2.0 * e * dP.d[k];
    }
    __shared__ double red[kTD + 1][4];
#pragma unroll
    for (int c = 0; c < kTD + 1; ++c) {
        double a = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = a;
    }
    __syncthreads();
    if (threadIdx.x < kTD + 1) {
        const double a = red[threadIdx.x][0] + red[threadIdx.x][1] + red[threadIdx.x][2] + red[threadIdx.x][3];
        atomicAdd(sums + threadIdx.x, a);
    }
}

template <int LAT, typename S>
int tl_step_t(const TLState& T, const Geom& G, const Export& E, const Band& B, const Region& bulk,
              const Region& loss, void* const f[2], int par, const double* dPref, cudaStream_t st)
{
    const S* fi = static_cast<const S*>(f[par]);
    S* fo = static_cast<S*>(f[par ^ 1]);
    const S* ti = static_cast<const S*>(T.t[par]);
    S* to = static_cast<S*>(T.t[par ^ 1]);
    TD* St = static_cast<TD*>(T.St);
    TD* St1 = static_cast<TD*>(T.St1);
    TD* Ud = static_cast<TD*>(T.Ud);
    Relax<TD> P;
    P.alpha_T = TD(B.alpha_T);
    P.alpha_T.d[0] = 1.0;                       // direction 0: alpha_T
    P.beta_P = TD(B.beta_P);
    P.beta_P.d[1] = 1.0;                        // direction 1: beta_P
    P.t_inf = TD(B.t_inf);
    for (int s = 0; s < 4; ++s) {
        P.pdev[s] = TD(B.pdev[s]);
        P.pdev[s].d[2] = 1.0;                   // direction 2: P_inf (all sides)
    }
    if (B.n_unk > 0) {
        if (E.nslots > 0)
            k_tl_strip<LAT, S><<<(E.nslots + 127) / 128, 128, 0, st>>>(G, E, fi, ti, St, St1);
        for (int stage = 0; stage < 4; ++stage)
            k_tl_stage<LAT><<<(B.n_unk + 127) / 128, 128, 0, st>>>(
                G, B, P, St, St1, Ud, static_cast<TD*>(T.Ya), static_cast<TD*>(T.Yb),
                static_cast<TD*>(T.acc), T.mask, stage);
        k_tl_dirichlet<LAT, S><<<(B.n_unk + 127) / 128, 128, 0, st>>>(G, B, Ud, fo, to);
    }
    if (bulk.x1 > bulk.x0 && bulk.y1 > bulk.y0) {
        dim3 grd((bulk.x1 - bulk.x0 + 127) / 128, bulk.y1 - bulk.y0);
        k_tl_bulk<LAT, S><<<grd, 128, 0, st>>>(G, bulk, fi, ti, fo, to);
    }
    if (loss.x1 > loss.x0 && loss.y1 > loss.y0) {
        dim3 grd((loss.x1 - loss.x0 + 127) / 128, loss.y1 - loss.y0);
        k_tl_loss<LAT, S><<<grd, 128, 0, st>>>(G, loss, fo, to, dPref, T.sums);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int LAT>
__global__ void k_tl_seed(Band B, TD* Ud, int par)
{
    // boundary state of the current parity with zero derivatives
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= B.n_unk) return;
#pragma unroll
    for (int m = 0; m < 4; ++m) Ud[4LL * u + m] = TD(B.Ub[((long long)par * B.n_unk + u) * 4 + m]);
}

template <int LAT>
__global__ void k_tl_unseed(Band B, const TD* Ud, int par)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= B.n_unk) return;
#pragma unroll
    for (int m = 0; m < 4; ++m) B.Ub[((long long)par * B.n_unk + u) * 4 + m] = Ud[4LL * u + m].v;
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

size_t tl_dual_bytes() { return sizeof(TD); }

int launch_tl_step(int lat, int storage, const TLState& T, const Geom& G, const Export& E,
                   const Band& B, const Region& bulk, const Region& loss, void* const f[2], int par,
                   const double* dPref, cudaStream_t st)
{
#define CALL(L, S) tl_step_t<L, S>(T, G, E, B, bulk, loss, f, par, dPref, st)
    TL_DISPATCH(lat, storage, CALL);
#undef CALL
}

int launch_tl_seed(const TLState& T, const Band& B, int par, bool back, cudaStream_t st)
{
    if (B.n_unk == 0) return 0;
    TD* Ud = static_cast<TD*>(T.Ud);
    if (back) k_tl_unseed<D2Q37><<<(B.n_unk + 127) / 128, 128, 0, st>>>(B, Ud, par);
    else k_tl_seed<D2Q37><<<(B.n_unk + 127) / 128, 128, 0, st>>>(B, Ud, par);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lbmgb
