// bulk.cu -- bulk kernels of the thermal lattice Boltzmann step.
//
//  k_bulk    fused pull-stream + moments + BGK collide on every bulk node
//            (Eqs. lbe, macro, bgk with the equilibria of Eqs. feq-3/feq-4),
//            plus the export of macros and non-equilibrium moments on the
//            three bulk columns/rows next to each characteristic boundary
//            (used by the boundary solver of Sec. 3.3).
//  k_init    f = f^eq(U0) on every node, the strips of time 0.
//  k_init_band  boundary ODE state of time 0.
//  k_macros  macroscopic fields of the stored populations (Eq. macro).
//
// Populations are stored post-collision and shifted, g = f* - w rho0, in
// SoA planes [Q][ny][nxp].  A bulk node pulls g*_i(x - c_i) for every i.
#include "lbm_internal.cuh"

namespace lbmgb {

namespace {

constexpr int kBulkThreads = 128;

// Viscous stress sigma' = -(1 - 1/(2 tau)) sum c c (f - f^eq) (Eq. LaplaceU)
// and heat flux q = (1 - 1/(2 tau)) 1/2 sum (f - f^eq) |c-u|^2 (c-u)
// (Eqs. heatflux, LaplaceT; the equilibrium part of the central third
// moment vanishes on D2Q37).
template <int LAT, typename C>
__device__ __forceinline__ void neq_moments(const C* g, const Moments<LAT, C>& m, double fac,
                                            double N[5])
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

template <int LAT, typename S>
__global__ void __launch_bounds__(kBulkThreads)
    k_bulk(Geom G, Band B, const S* __restrict__ fin, S* __restrict__ fout, int par_new)
{
    using L = Lat<LAT>;
    using C = typename Store<S>::C;
    constexpr int Q = L::Q;
    const int x = G.bx0 + blockIdx.x * blockDim.x + threadIdx.x;
    const int y = G.by0 + blockIdx.y;
    if (x >= G.bx1) return;

    // Pull stream (Eq. lbe): g_i(x) = g*_i(x - c_i), periodic axes wrap.
    C g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int xs = x - L::cx(i), ys = y - L::cy(i);
        if (L::cx(i) && G.perx) xs = xs < 0 ? xs + G.nx : (xs >= G.nx ? xs - G.nx : xs);
        if (L::cy(i) && G.pery) ys = ys < 0 ? ys + G.ny : (ys >= G.ny ? ys - G.ny : ys);
        C v = Store<S>::load(fin + (long long)i * G.plane + (long long)ys * G.nxp + xs);
        if (Store<S>::SCALED) v *= C(L::w(i));
        g[i] = v;
    }

    const Moments<LAT, C> m = moments<LAT, C>(g, C(G.rho0));

    // BGK collide (Eq. bgk) with the shifted equilibrium, one opposite pair
    // at a time: f^eq_{+-} = w rho (1 + even +- odd) in p = c.u / c_s^2.
    constexpr C ics2 = C(1.0 / L::CS2);
    constexpr C a3 = L::THERMAL ? C(1.0 / 6.0) : C(0);
    constexpr C a4 = L::THERMAL ? C(1.0 / 24.0) : C(0);
    C a0[L::NCLS], a1[L::NCLS], a2[L::NCLS];
    eq_coef<LAT, C>((m.ux * m.ux + m.uy * m.uy) * ics2, m.dT, a0, a1, a2);
    const C om = C(1.0 / G.tau);
    S* out = fout + (long long)y * G.nxp + x;
    {
        const C geq = C(L::w(0)) * (m.s0 + m.rho * a0[0]);
        C v = g[0] + om * (geq - g[0]);
        if (Store<S>::SCALED) v *= C(1.0 / L::w(0));
        Store<S>::put(out, v);
    }
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const int k = L::cls(i);
        const C p = (C(L::cx(i)) * m.ux + C(L::cy(i)) * m.uy) * ics2;
        const C p2 = p * p;
        const C ev = a0[k] + p2 * (a2[k] + p2 * a4);
        const C od = p * (a1[k] + p2 * a3);
        const C wr = C(L::w(i));
        const C gp = wr * (m.s0 + m.rho * (ev + od));
        const C gm = wr * (m.s0 + m.rho * (ev - od));
        C vp = g[i] + om * (gp - g[i]);
        C vm = g[i + 1] + om * (gm - g[i + 1]);
        if (Store<S>::SCALED) {
            vp *= C(1.0 / L::w(i));
            vm *= C(1.0 / L::w(i));
        }
        Store<S>::put(out + (long long)i * G.plane, vp);
        Store<S>::put(out + (long long)(i + 1) * G.plane, vm);
    }

    // Near-boundary export for the characteristic boundary solver.
    if (B.any_cbc) {
        const int dW = x - G.M, dE = G.nx - 1 - G.M - x;
        const int dS = y - G.M, dN = G.ny - 1 - G.M - y;
        const bool inW = B.s[0].kind == SIDE_CBC && dW >= 0 && dW <= 2;
        const bool inE = B.s[1].kind == SIDE_CBC && dE >= 0 && dE <= 2;
        const bool inS = B.s[2].kind == SIDE_CBC && dS >= 0 && dS <= 2;
        const bool inN = B.s[3].kind == SIDE_CBC && dN >= 0 && dN <= 2;
        if (inW || inE || inS || inN) {
            double N[5];
            neq_moments<LAT, C>(g, m, 1.0 - 0.5 / G.tau, N);
            const double U[4] = {double(m.s0), double(m.ux), double(m.uy), double(m.dT)};
            const int dd[4] = {dW, dE, dS, dN};
            const bool in[4] = {inW, inE, inS, inN};
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (!in[s]) continue;
                const int p = s < 2 ? y : x;
                double* u = B.stripU + strip_u_index(B.s[s], par_new, dd[s], p);
                double* n = B.stripN + strip_n_index(B.s[s], par_new, dd[s], p);
#pragma unroll
                for (int c = 0; c < 4; ++c) u[c] = U[c];
#pragma unroll
                for (int c = 0; c < 5; ++c) n[c] = N[c];
            }
        }
    }
}

template <int LAT, typename S>
__global__ void k_init(Geom G, Band B, const double* __restrict__ rho, const double* __restrict__ ux,
                       const double* __restrict__ uy, const double* __restrict__ T, S* __restrict__ f)
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
        Store<S>::put(out + (long long)i * G.plane, typename Store<S>::C(v));
    }
    // strips of time 0 (parity 0): U0 and zero non-equilibrium moments
    if (B.any_cbc) {
        const int dd[4] = {x - G.M, G.nx - 1 - G.M - x, y - G.M, G.ny - 1 - G.M - y};
        const double U[4] = {m.s0, m.ux, m.uy, m.dT};
        for (int s = 0; s < 4; ++s) {
            const Side& S_ = B.s[s];
            const int p = s < 2 ? y : x;
            if (S_.kind != SIDE_CBC || dd[s] < 0 || dd[s] > 2 || p < S_.lo || p > S_.hi) continue;
            double* u = B.stripU + strip_u_index(S_, 0, dd[s], p);
            double* nn = B.stripN + strip_n_index(S_, 0, dd[s], p);
            for (int c = 0; c < 4; ++c) u[c] = U[c];
            for (int c = 0; c < 5; ++c) nn[c] = 0.0;
        }
    }
}

// Node of characteristic unknown u: side layers in (side, p, j) order, then
// the innermost node of each corner block.
__device__ inline void unknown_node(const Geom& G, const Band& B, int u, int& x, int& y)
{
    if (u < B.n_side_unk) {
        int s = 0;
        while (s < 3 && !(B.s[s].kind == SIDE_CBC && u >= B.s[s].base &&
                          u < B.s[s].base + (B.s[s].hi - B.s[s].lo + 1) * G.M))
            ++s;
        const int r = u - B.s[s].base;
        const int p = B.s[s].lo + r / G.M, j = 1 + r % G.M;
        side_xf(s, p, G.nx, G.ny, G.M, x, y);
        x += j * side_nx(s);
        y += j * side_ny(s);
    } else {
        const int c = u - B.n_side_unk;
        x = corner_sx(c) < 0 ? G.M - 1 : G.nx - G.M;
        y = corner_sy(c) < 0 ? G.M - 1 : G.ny - G.M;
    }
}

__global__ void k_init_band(Geom G, Band B, const double* __restrict__ rho,
                            const double* __restrict__ ux, const double* __restrict__ uy,
                            const double* __restrict__ T, int thermal)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= B.n_unk) return;
    int x, y;
    unknown_node(G, B, u, x, y);
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
        double v = double(Store<S>::load(in + (long long)i * G.plane));
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
int init_t(const Geom& G, const Band& B, const double* rho, const double* ux, const double* uy,
           const double* T, void* f, cudaStream_t st)
{
    dim3 blk(128), grd((G.nx + 127) / 128, G.ny);
    k_init<LAT, S><<<grd, blk, 0, st>>>(G, B, rho, ux, uy, T, static_cast<S*>(f));
    if (B.n_unk > 0)
        k_init_band<<<(B.n_unk + 127) / 128, 128, 0, st>>>(G, B, rho, ux, uy, T, Lat<LAT>::THERMAL);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int LAT, typename S>
int bulk_t(const Geom& G, const Band& B, const void* fin, void* fout, int par_new, cudaStream_t st)
{
    const int w = G.bx1 - G.bx0, h = G.by1 - G.by0;
    if (w <= 0 || h <= 0) return 0;
    dim3 blk(kBulkThreads), grd((w + kBulkThreads - 1) / kBulkThreads, h);
    k_bulk<LAT, S><<<grd, blk, 0, st>>>(G, B, static_cast<const S*>(fin), static_cast<S*>(fout),
                                        par_new);
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

int launch_init(int lat, int storage, const Geom& G, const Band& B, const double* rho,
                const double* ux, const double* uy, const double* T, void* f, cudaStream_t st)
{
#define CALL(L, S) init_t<L, S>(G, B, rho, ux, uy, T, f, st)
    LBM_DISPATCH(lat, storage, CALL);
#undef CALL
}

int launch_bulk(int lat, int storage, const Geom& G, const Band& B, const void* fin, void* fout,
                int par_new, cudaStream_t st)
{
#define CALL(L, S) bulk_t<L, S>(G, B, fin, fout, par_new, st)
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
