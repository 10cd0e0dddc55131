// adjoint.cu -- the reverse-mode (adjoint) sweep of the method's time step,
// for gradients of the pressure loss
//     J = sum over steps n and bulk nodes x of (P_n(x) - c_s^2 rho0 - dP_ref,n(x))^2
// with respect to the relaxation parameters of the incoming waves
// (Eqs. LODI-Relax, CBC-Relax): alpha_T, beta_P, P_inf, alpha_V, t_inf --
// all five in one backward pass.
//
// The forward step t -> t + 1 (Fig. flowchart-lbm-algo, Sec. 3.3) is read as
//   f^pre_{t+1}(x, i) = f*_t(x - c_i, i)                  pull (Eq. lbe), bulk x
//   f*_{t+1}(x)       = C(f^pre_{t+1}(x))                 BGK collision (Eq. bgk)
//   U_b(t+1)          = RK4(U_b(t); strips, V, theta)     the boundary ODE
//   f*_{t+1}(b)       = f^eq(U_b(t+1))                    equilibrium Dirichlet write
// where the strips are moments of pulled populations of strip nodes:
// macros U(t) = m(f^pre_t), U(t+1) = m(f^pre_{t+1}) and, for the mesoscopic
// viscous vector, the non-equilibrium moments N(t) = neq(f^pre_t) of the
// nodes of its stencil.  The adjoint runs this backwards, one kernel set per
// step (launch_adj_step), with the adjoint of the pulled populations,
// lambda^pre, as the state carried from step to step:
//
//   k_adj_band       the boundary part, one cooperative launch whose phases
//                    are separated by grid-wide barriers:
//                    - lambda of U_b(t+1) from the populations the Dirichlet
//                      write set, gathered from lambda^pre_{t+2} (f*_{t+1}(b, i)
//                      is pulled by the bulk node b + c_i);
//                    - the RK4 stage fields of step t recomputed from U_b(t);
//                    - each RK4 stage backwards: lambda^T dF at the stage
//                      field, from forward derivatives of the right-hand side
//                      (charsys.cuh) along its 29 inputs, two per thread;
//                    - the frozen viscous vector backwards;
//                    - lambda of U_b(t), and what the strips of t add to
//                      lambda^pre at their nodes (moment and
//                      non-equilibrium-moment weights)
//   k_adj_bulk       lambda^pre_{t+1} at every bulk node: the collision's
//                    adjoint (through the equilibrium's dependence on the
//                    moments), the loss at t + 1 and the strips' shares, from
//                    lambda*_{t+1}(x, i) = lambda^pre_{t+2}(x + c_i, i); on
//                    a second stream, beside the boundary kernels
//   k_adj_strip1     the share of the strip macros of t + 1, afterwards
//
// The host (api.cu) runs the forward steps with checkpoints and, segment by
// segment from the last, recomputes the steps (storing the macros, boundary
// state and strips of every step) and runs these kernels backwards.
// Supported: FP64 and FP32 storage, the equilibrium Dirichlet condition,
// characteristic and periodic sides, every viscous form.
#include "charsys.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace cg = cooperative_groups;

namespace lbmgb {

namespace {

template <typename S>
using CT = typename Store<S>::C;          // population arithmetic
template <typename S>
using RT = typename StripReal<S>::T;      // boundary solver inputs

constexpr int kAdjThreads = 128;
// The cooperative boundary kernel: two CTAs of six warps per SM (at most 170
// registers a thread), so that one stage's derivative items (eight per
// unknown) and the next step's stage items run in one pass of the grid.
constexpr int kBandThreads = 192;
// Forward derivative directions per evaluation: four, so that one boundary
// unknown's right-hand side is differentiated by eight threads within the
// register cap of kBandThreads (eight directions per thread spilled and ran
// 4x slower; two needed two passes of the grid per stage).
constexpr int kChunk = 4;
constexpr int kRhsInputs = 29;            // 5 stage-field neighbours x 4, V (4), theta (5)
constexpr int kRhsChunks = (kRhsInputs + kChunk - 1) / kChunk;
constexpr int kMesoInputs = 36;           // 5 stencil nodes x (5 moments, u_x, u_y), drho of node 0
constexpr int kMesoChunks = (kMesoInputs + kChunk - 1) / kChunk;
constexpr int kFdInputs = 24;             // 6 neighbours x 4
constexpr int kFdChunks = kFdInputs / kChunk;

// A node of a periodic axis wrapped into the grid; true if it is a bulk node
// (a pull target of the bulk update).
__device__ __forceinline__ bool wrap_bulk(const Geom& G, int& x, int& y)
{
    if (G.perx) x = x < 0 ? x + G.nx : (x >= G.nx ? x - G.nx : x);
    if (G.pery) y = y < 0 ? y + G.ny : (y >= G.ny ? y - G.ny : y);
    return x >= G.bx0 && x < G.bx1 && y >= G.by0 && y < G.by1;
}

// a[k] = sum_i lam(i) d g^eq_i / d m_k at the moments m = (drho, u_x, u_y,
// theta - 1): the equilibrium (Eqs. feq-3, feq-4, pairwise as equilibrium()
// evaluates it) on forward derivatives along the four moments.
template <int LAT, typename C, typename Lam>
__device__ __forceinline__ void eq_vjp(C s0, C ux, C uy, C dT, C rho0, Lam&& lam, C a[4])
{
    using L = Lat<LAT>;
    using D4 = Dual<C, 4>;
    D4 m0(s0), mx(ux), my(uy), mt(L::THERMAL ? dT : C(0));
    m0.d[0] = C(1);
    mx.d[1] = C(1);
    my.d[2] = C(1);
    if (L::THERMAL) mt.d[3] = C(1);
    const D4 rho = D4(rho0) + m0;
    constexpr C ics2 = C(1.0 / L::CS2);
    constexpr C a3 = L::ORDER >= 3 ? C(1.0 / 6.0) : C(0);
    constexpr C a4 = L::ORDER >= 4 ? C(1.0 / 24.0) : C(0);
    const D4 uxs = mx * ics2, uys = my * ics2;
    const EqPoly<D4> e = eq_poly<LAT, D4>(mx * uxs + my * uys, mt);
    C acc[4] = {C(0), C(0), C(0), C(0)};
    auto add = [&](C l, const D4& g) {
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += l * g.d[k];
    };
    {
        const D4 g0 = C(L::w(0)) * (m0 + rho * e.A0);
        add(lam(0), g0);
    }
#pragma unroll
    for (int i = 1; i < L::Q; i += 2) {
        const int k = L::cls(i);
        const C xi2 = C(L::c2cls(k)) * ics2;
        const D4 A0 = e.A0 + xi2 * (e.B0 + e.C0 * xi2);
        const D4 A1 = e.A1 + e.B1 * xi2;
        const D4 A2 = e.A2 + e.B2 * xi2;
        D4 p;
        if (L::cx(i) == 0) p = C(L::cy(i)) * uys;
        else if (L::cy(i) == 0) p = C(L::cx(i)) * uxs;
        else p = C(L::cx(i)) * uxs + C(L::cy(i)) * uys;
        const D4 p2 = p * p;
        const D4 ev = A0 + p2 * (A2 + p2 * a4);
        const D4 od = p * (A1 + p2 * a3);
        const D4 ws0 = C(L::w(i)) * m0, wr = C(L::w(i)) * rho;
        add(lam(i), ws0 + wr * (ev + od));
        add(lam(i + 1), ws0 + wr * (ev - od));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = acc[k];
}

// Pull-back of a covector mu on the moments m = (drho, u_x, u_y, theta - 1)
// to the population sums S = (sum g, sum g c_x, sum g c_y, sum g |c|^2)
// (Eq. macro): b_s = sum_k mu_k dm_k/dS_s; then d/dg_i = b_0 + b_1 c_ix +
// b_2 c_iy + b_3 |c_i|^2.
template <int LAT, typename C>
__device__ __forceinline__ void moment_pullback(C s0, C ux, C uy, C dT, C rho0, const C mu[4], C b[4])
{
    using L = Lat<LAT>;
    const C ir = C(1) / (rho0 + s0);
    b[0] = mu[0] - (mu[1] * ux + mu[2] * uy) * ir;
    b[1] = mu[1] * ir;
    b[2] = mu[2] * ir;
    b[3] = C(0);
    if (L::THERMAL) {
        // theta - 1 = (S_3 - (S_1^2 + S_2^2) / rho - 2 c_s^2 S_0) / (2 rho c_s^2)
        const C h = ir * C(0.5 / L::CS2);
        b[0] += mu[3] * ((ux * ux + uy * uy - C(2.0 * L::CS2)) * h - dT * ir);
        b[1] -= mu[3] * C(2) * ux * h;
        b[2] -= mu[3] * C(2) * uy * h;
        b[3] = mu[3] * h;
    }
}

// Weight of non-equilibrium moment n on velocity c at flow velocity u:
// sigma'_xx, sigma'_xy, sigma'_yy: c_x c_x, c_x c_y, c_y c_y; q_x, q_y:
// |c - u|^2 (c - u) / 2 (Eqs. LaplaceU, LaplaceT).
template <typename C>
__device__ __forceinline__ C neq_weight(int n, C cx, C cy, C ux, C uy)
{
    if (n == 0) return cx * cx;
    if (n == 1) return cx * cy;
    if (n == 2) return cy * cy;
    const C ex = cx - ux, ey = cy - uy, h = C(0.5) * (ex * ex + ey * ey);
    return n == 3 ? h * ex : h * ey;
}

// The relaxation parameters (alpha_T, beta_P, t_inf, alpha_V, P_inf - c_s^2
// rho0 per side) in arithmetic type R, rounded on the host.
template <typename R>
__device__ __forceinline__ R relax_value(const AdjState& A, int q)
{
    if constexpr (sizeof(R) == 4) return A.relax_f[q];
    else return A.relax_d[q];
}

// Block sum of v[0..NV) added to sums[0..NV) (one double atomic per block
// and value); every thread of the block must call it.
template <int NV, int NT = kAdjThreads>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sums)
{
    __shared__ double part[NV][NT / 32];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if ((threadIdx.x & 31) == 0) part[k][threadIdx.x >> 5] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double a = 0.0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) a += part[threadIdx.x][w];
        if (a != 0.0) atomicAdd(sums + threadIdx.x, a);
    }
}

// ---------------------------------------------------------------------------
// Loss of one state (forward pass)
// ---------------------------------------------------------------------------

// The moments (drho, u_x, u_y, theta - 1) of every bulk node of the state f
// (the collision keeps them: those of its pulled populations) into Mout
// ([ny * nx][4], type R; skipped if null), and, if sums is not null, the
// loss sums[0] += (P - c_s^2 rho0 - dPref)^2 over them.
template <int LAT, typename S>
__global__ void __launch_bounds__(kAdjThreads)
    k_adj_loss(Geom G, Region R, const S* __restrict__ f, const double* __restrict__ dPref, double* sums,
               RT<S>* __restrict__ Mout, AdjRecord rec)
{
    using L = Lat<LAT>;
    using C = CT<S>;
    using Rt = RT<S>;
    {
        // the history record, one value per thread of the grid
        const long long nrec = rec.n_ub + rec.n_su + rec.n_sn;
        const long long nthr = (long long)gridDim.x * gridDim.y * kAdjThreads;
        for (long long i = ((long long)blockIdx.y * gridDim.x + blockIdx.x) * kAdjThreads + threadIdx.x; i < nrec;
             i += nthr) {
            if (i < rec.n_ub) rec.ubh[i] = rec.ub[i];
            else if (i < rec.n_ub + rec.n_su) {
                const long long j = i - rec.n_ub;
                static_cast<Rt*>(rec.suh)[j] = static_cast<const Rt*>(rec.su)[j];
            } else {
                const long long j = i - rec.n_ub - rec.n_su;
                static_cast<Rt*>(rec.snh)[j] = static_cast<const Rt*>(rec.sn)[j];
            }
        }
    }
    const int x = R.x0 + blockIdx.x * kAdjThreads + threadIdx.x, y = R.y0 + blockIdx.y;
    double v[1] = {0.0};
    if (x < R.x1 && y < R.y1) {
        C g[L::Q];
        const long long node = (long long)y * G.nxp + x;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) g[i] = C(f[L::plane_of(i) * G.plane + node]);
        const Moments<LAT, C> m = moments_G<LAT, C>(G, g);
        const long long idx = (long long)y * G.nx + x;
        if (Mout) {
            Rt* o = Mout + 4 * idx;
            o[0] = Rt(m.s0);
            o[1] = Rt(m.ux);
            o[2] = Rt(m.uy);
            o[3] = Rt(m.dT);
        }
        if (sums) {
            const double s0 = double(m.s0), dT = double(m.dT);
            const double dP = L::THERMAL ? L::CS2 * (s0 + G.rho0 * dT + s0 * dT) : L::CS2 * s0;
            const double e = dP - (dPref ? dPref[idx] : 0.0);
            v[0] = e * e;
        }
    }
    if (sums) block_sum<1>(v, sums);
}

// ---------------------------------------------------------------------------
// Boundary: the Dirichlet write, the RK4 stages and the viscous vector
// ---------------------------------------------------------------------------

// lambda_U(t+1)[u] += sum over the nodes b the unknown writes and the
// velocities i of lambda*_{t+1}(b, i) d f^eq_i / dU at U_b(t+1): per node,
// sum_i lambda*_i dg^eq_i/dU_k of one node the Dirichlet write of unknown u
// set (node q of a corner's M x M block, row-major; the node itself for a
// side unknown), lambda*_i = lambda^pre_{t+2}(node + c_i, i), U = U_b(t+1).
template <int LAT, typename S>
__device__ __forceinline__ CT<S> dirichlet_part(const Geom& G, const UDesc& D, const double* __restrict__ U,
                                                const CT<S>* __restrict__ lnext, int k, int q)
{
    using L = Lat<LAT>;
    using C = CT<S>;
    using D1 = Dual<C, 1>;
    const int a = q / G.M, b = q % G.M;
    const long long node = D.wnode + (D.kind >= 4 ? a * D.wdx + b * D.wdy : 0);
    const int x = int(node % G.nxp), y = int(node / G.nxp);
    C lam[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        int xs = x + L::cx(i), ys = y + L::cy(i);
        lam[i] = wrap_bulk(G, xs, ys) ? lnext[L::plane_of(i) * G.plane + (long long)ys * G.nxp + xs] : C(0);
    }
    Moments<LAT, D1> m;
    m.s0 = D1(U[0]);
    m.ux = D1(U[1]);
    m.uy = D1(U[2]);
    m.dT = D1(L::THERMAL ? U[3] : 0.0);
    (k == 0 ? m.s0 : k == 1 ? m.ux : k == 2 ? m.uy : m.dT).d[0] = C(1);
    m.rho = D1(G.rho0) + m.s0;
    D1 ge[L::Q];
    equilibrium<LAT, D1>(m, ge);
    C s = C(0);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) s += lam[i] * ge[i].d[0];
    return s;
}

// The Dirichlet write's adjoint, thread (u, k): lambda_U(t+1)_k of unknown
// u gains the share of the node it writes (of the first node of a corner's
// block; the other M^2 - 1 nodes of the four corner blocks are items of
// adj_corner_item, folded in by the next phase in a fixed order), by
// forward derivatives of the equilibrium along moment k; thread (u, 0)
// also sets the stage-0 field Y0[u] = U_b(t).
template <int LAT, typename S>
__device__ __forceinline__ void adj_dirichlet_item(const Geom& G, const Band& B, const double* __restrict__ Ub,
                                                   const double* __restrict__ Ub1, const CT<S>* __restrict__ lnext,
                                                   double* lU, RT<S>* lUr, RT<S>* Y0, int tid)
{
    using L = Lat<LAT>;
    const int u = tid >> 2, k = tid & 3;
    if (u >= B.n_unk) return;
    if (k == 0) {
#pragma unroll
        for (int m = 0; m < 4; ++m) Y0[4LL * u + m] = RT<S>(Ub[4LL * u + m]);
    }
    if (!L::THERMAL && k == 3) return;
    const double v = lU[4LL * u + k] + double(dirichlet_part<LAT, S>(G, B.ud[u], Ub1 + 4LL * u, lnext, k, 0));
    lU[4LL * u + k] = v;
    lUr[4LL * u + k] = RT<S>(v);
}

// Item (c, k, q) of the corner blocks: node q + 1 of corner c's block.
template <int LAT, typename S>
__device__ __forceinline__ void adj_corner_item(const Geom& G, const Band& B, const AdjState& A,
                                                const double* __restrict__ Ub1, const CT<S>* __restrict__ lnext,
                                                int tid)
{
    using L = Lat<LAT>;
    const int per = G.M * G.M - 1;
    const int c = tid / (4 * per), k = (tid / per) % 4, q = tid % per;
    const int u = B.n_unk - 4 + c;
    A.cpart[tid] = (!L::THERMAL && k == 3)
                       ? 0.0
                       : double(dirichlet_part<LAT, S>(G, B.ud[u], Ub1 + 4LL * u, lnext, k, q + 1));
}

// The other nodes' shares of corner unknown u's block (component k), in
// order: the reverse step's first stage phase and its last phase add them.
__device__ __forceinline__ double corner_share(const Geom& G, const Band& B, const AdjState& A, int u, int k)
{
    const int per = G.M * G.M - 1, c = u - (B.n_unk - 4);
    double v = 0.0;
    for (int q = 0; q < per; ++q) v += A.cpart[(c * 4 + k) * per + q];
    return v;
}

// Stage `stage` (0, 1, 2) of step t recomputed: Y[stage + 1] = U_b(t) + h k;
// stage 0 also freezes the viscous vector and the incoming waves.
template <int LAT, typename S>
__device__ __forceinline__ void adj_fwd_item(const Geom& G, const Band& B, const AdjState& A, const StageSet& Z,
                                             const RT<S>* __restrict__ stU, const RT<S>* __restrict__ stN,
                                             const RT<S>* __restrict__ stU1, int stage, int u)
{
    using Lt = Lat<LAT>;
    using R = RT<S>;
    if (u >= B.n_unk) return;
    const UDesc D = B.ud[u];
    CtxT<R> X;
    X.Y = static_cast<const R*>(Z.Y[stage]);
    X.St = stU;
    X.St1 = stU1;
    X.frac = stage == 0 ? R(0) : R(0.5);
    R V[4] = {R(0), R(0), R(0), R(0)};
    R* Vu = static_cast<R*>(Z.V) + 4LL * u;
    int mk;
    if (stage == 0) {
        if (B.viscous != VIS_OFF && D.kind < 4) {
            if (B.viscous == VIS_FD) vis_fd<Lt::THERMAL>(G, B, X, D, u, Lt::CS2, V);
            else vis_meso<Lt::THERMAL>(G, stU, 4, stN, 5, D, Lt::CS2, V);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) Vu[m] = V[m];
        R Ul[4];
        to_local(D.kind, R(B.kR), X.Y + 4LL * u, Ul);
        mk = incoming_mask<Lt::THERMAL>(char_sys<Lt::THERMAL>(B, G.rho0, Ul));
        Z.mask[u] = mk;
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) V[m] = Vu[m];
        mk = Z.mask[u];
    }
    Relax<R> P;
    P.alpha_T = relax_value<R>(A, 0);
    P.beta_P = relax_value<R>(A, 1);
    P.t_inf = relax_value<R>(A, 2);
    P.alpha_V = relax_value<R>(A, 3);
#pragma unroll
    for (int q = 0; q < 4; ++q) P.pdev[q] = relax_value<R>(A, 4 + q);
    R k[4];
    unknown_rhs<LAT, R>(G, B, P, X, D, u, V, mk, k);
    const R h = stage == 2 ? R(1) : R(0.5);
    R* Yo = static_cast<R*>(Z.Y[stage + 1]) + 4LL * u;
#pragma unroll
    for (int m = 0; m < 4; ++m) Yo[m] = static_cast<const R*>(Z.Y[0])[4LL * u + m] + h * k[m];
}

// lambda of one strip macro or stage value: the stage field at a reference
// (Sec. 3.3: a strip node at stage time fraction frac is (1 - frac) U(t) +
// frac U(t + 1)).
template <typename R>
__device__ __forceinline__ void scatter_ref(const AdjState& A, R* lY, int ref, int m, R frac, R g)
{
    if (ref >= 0) {
        atomicAdd(lY + 4LL * ref + m, g);
        return;
    }
    const long long s = 4LL * (-ref - 1) + m;
    if (frac != R(1)) atomicAdd(static_cast<R*>(A.lSt) + s, (R(1) - frac) * g);
    if (frac != R(0)) atomicAdd(static_cast<R*>(A.lSt1) + s, frac * g);
}


// One RK4 stage backwards.  Thread (u, c) evaluates the right-hand side of
// unknown u (unknown_rhs, charsys.cuh) at the stage field on Dual numbers
// seeded along inputs 2c, 2c + 1 of: the stage-field values it reads (own,
// then the two normal and two tangential neighbours; 4 components each),
// the viscous vector (4) and theta = (alpha_T, beta_P, P_inf - c_s^2 rho0 of
// its side, alpha_V, t_inf), and adds lambda_k^T dk/dinput to the adjoint of
// each input.  lambda_k of stage s: U(t+1) = U + (k0 + 2 k1 + 2 k2 + k3)/6,
// Y1 = U + k0/2, Y2 = U + k1/2, Y3 = U + k2.
template <int LAT, typename S>
__device__ __forceinline__ void adj_vjp_item(const Geom& G, const Band& B, const AdjState& A,
                                             const RT<S>* __restrict__ stU, const RT<S>* __restrict__ stU1,
                                             int stage, int tid, double (&th)[5])
{
    using R = RT<S>;
    using T8 = Dual<R, kChunk>;
    const int u = tid / kRhsChunks, c = tid % kRhsChunks;
    if (u < B.n_unk) {
        const UDesc D = B.ud[u];
        const bool corner = D.kind >= 4;
        UDesc Dl = D;
        int ref[5] = {u, 0, 0, 0, 0}, nr;
        if (corner) {
            ref[1] = D.nb[0]; ref[2] = D.nb[1];
            Dl.nb[0] = 1; Dl.nb[1] = 2;
            nr = 3;
        } else {
            if (D.j == B.M) {
                ref[1] = D.nb[1]; ref[2] = D.nb[2];
                Dl.nb[1] = 1; Dl.nb[2] = 2;
            } else {
                ref[1] = D.nb[0]; ref[2] = D.nb[1];
                Dl.nb[0] = 1; Dl.nb[1] = 2;
            }
            ref[3] = D.nb[4]; ref[4] = D.nb[5];
            Dl.nb[4] = 3; Dl.nb[5] = 4;
            nr = 5;
        }
        const R frac = stage == 0 ? R(0) : (stage == 3 ? R(1) : R(0.5));
        CtxT<R> Xr;
        Xr.Y = static_cast<const R*>(A.Y[stage]);
        Xr.St = stU;
        Xr.St1 = stU1;
        Xr.frac = frac;
        auto seed = [&](T8& v, int j) {
            if (j / kChunk == c) v.d[j % kChunk] = R(1);
        };
        T8 Yl[20];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            R v[4] = {R(0), R(0), R(0), R(0)};
            if (k < nr) fetch(Xr, ref[k], v);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                Yl[4 * k + m] = T8(v[m]);
                seed(Yl[4 * k + m], 4 * k + m);
            }
        }
        T8 Vd[4];
        const R* Vu = static_cast<const R*>(A.V) + 4LL * u;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            Vd[m] = T8(Vu[m]);
            seed(Vd[m], 20 + m);
        }
        Relax<T8> P;
        P.alpha_T = T8(relax_value<R>(A, 0));
        P.beta_P = T8(relax_value<R>(A, 1));
        P.t_inf = T8(relax_value<R>(A, 2));
        P.alpha_V = T8(relax_value<R>(A, 3));
#pragma unroll
        for (int q = 0; q < 4; ++q) P.pdev[q] = T8(relax_value<R>(A, 4 + q));
        seed(P.alpha_T, 24);
        seed(P.beta_P, 25);
        if (!corner) {
            T8& pd = D.kind == 0 ? P.pdev[0] : D.kind == 1 ? P.pdev[1] : D.kind == 2 ? P.pdev[2] : P.pdev[3];
            seed(pd, 26);
        }
        seed(P.alpha_V, 27);
        seed(P.t_inf, 28);
        CtxT<T8> Xl;
        Xl.Y = Yl;
        Xl.St = Xl.St1 = nullptr;
        Xl.frac = T8(frac);
        T8 k[4];
        unknown_rhs<LAT, T8>(G, B, P, Xl, Dl, 0, Vd, A.mask[u], k);
        const R cs = (stage == 0 || stage == 3) ? R(1.0 / 6.0) : R(1.0 / 3.0);
        const R ch = stage == 2 ? R(1) : R(0.5);
        R lk[4];
        R* lUr = static_cast<R*>(A.lUr) + 4LL * u;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            R lu = lUr[m];
            if (stage == 3 && corner && G.M > 1) {
                // the corner block's other nodes (adj_corner_item) join here;
                // the stages after this one read the rounded sum
                lu = R(A.lU[4LL * u + m] + corner_share(G, B, A, u, m));
                if (c == 0) lUr[m] = lu;
            }
            lk[m] = cs * lu;
            if (stage < 3) lk[m] += ch * static_cast<const R*>(A.lY[stage + 1])[4LL * u + m];
        }
        R* lY = static_cast<R*>(A.lY[stage]);
#pragma unroll
        for (int d = 0; d < kChunk; ++d) {
            const int j = kChunk * c + d;
            if (j >= kRhsInputs) break;
            R g = R(0);
#pragma unroll
            for (int m = 0; m < 4; ++m) g += lk[m] * k[m].d[d];
            if (g == R(0)) continue;
            if (j < 20) {
                if (j / 4 < nr) scatter_ref<R>(A, lY, ref[j / 4], j % 4, frac, g);
            } else if (j < 24) {
                static_cast<R*>(A.lV)[4LL * u + (j - 20)] += g;      // one thread per (u, j)
            } else {
                th[j - 24] += double(g);
            }
        }
    }
}

// The mesoscopic viscous vector of side unknown u (vis_meso, Eqs. LaplaceU,
// LaplaceT) backwards to its stencil's strip values of time t: thread (u, c)
// takes inputs 2c, 2c + 1 of (5 moments, u_x, u_y) per stencil node, then
// drho of the first node.
template <int LAT, typename S>
__device__ __forceinline__ void adj_vis_meso_item(const Geom& G, const Band& B, const AdjState& A,
                                                  const RT<S>* __restrict__ stU, const RT<S>* __restrict__ stN, int tid)
{
    using Lt = Lat<LAT>;
    using R = RT<S>;
    using T8 = Dual<R, kChunk>;
    const int u = tid / kMesoChunks, c = tid % kMesoChunks;
    if (u >= B.n_unk) return;
    const UDesc D = B.ud[u];
    if (D.kind >= 4) return;
    const R* lV = static_cast<const R*>(A.lV) + 4LL * u;
    if (lV[0] == R(0) && lV[1] == R(0) && lV[2] == R(0) && lV[3] == R(0)) return;
    T8 SU[5 * 4], SN[5 * 5];
    UDesc Dl = D;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int sl = D.vs[k];
        Dl.vs[k] = k;
#pragma unroll
        for (int m = 0; m < 4; ++m) SU[4 * k + m] = T8(stU[4LL * sl + m]);
#pragma unroll
        for (int m = 0; m < 5; ++m) SN[5 * k + m] = T8(stN[5LL * sl + m]);
    }
#pragma unroll
    for (int d = 0; d < kChunk; ++d) {
        const int j = kChunk * c + d;
        if (j >= kMesoInputs) break;
        if (j == 35) { SU[0].d[d] = R(1); continue; }
        const int k = j / 7, m = j % 7;
        if (m < 5) SN[5 * k + m].d[d] = R(1);
        else SU[4 * k + (m - 4)].d[d] = R(1);   // m = 5: u_x, m = 6: u_y
    }
    T8 Vo[4];
    vis_meso<Lt::THERMAL, T8>(G, SU, 4, SN, 5, Dl, Lt::CS2, Vo);
#pragma unroll
    for (int d = 0; d < kChunk; ++d) {
        const int j = kChunk * c + d;
        if (j >= kMesoInputs) break;
        R g = R(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) g += lV[m] * Vo[m].d[d];
        if (g == R(0)) continue;
        if (j == 35) {
            atomicAdd(static_cast<R*>(A.lSt) + 4LL * D.vs[0], g);
            continue;
        }
        const int k = j / 7, m = j % 7, sl = D.vs[k];
        if (m < 5) atomicAdd(static_cast<R*>(A.lN) + 5LL * sl + m, g);
        else atomicAdd(static_cast<R*>(A.lSt) + 4LL * sl + (m - 4), g);
    }
}

// The "-FD" viscous vector of side unknown u (vis_fd, Sec. 4.2) backwards to
// the stage-0 field: its own value and the neighbours -n, +t, -t and +n (or,
// at the outermost layer, -2n and -3n).
template <int LAT, typename S>
__device__ __forceinline__ void adj_vis_fd_item(const Geom& G, const Band& B, const AdjState& A,
                                                const RT<S>* __restrict__ stU, int tid)
{
    using Lt = Lat<LAT>;
    using R = RT<S>;
    using T8 = Dual<R, kChunk>;
    const int u = tid / kFdChunks, c = tid % kFdChunks;
    if (u >= B.n_unk) return;
    const UDesc D = B.ud[u];
    if (D.kind >= 4) return;
    const R* lV = static_cast<const R*>(A.lV) + 4LL * u;
    if (lV[0] == R(0) && lV[1] == R(0) && lV[2] == R(0) && lV[3] == R(0)) return;
    UDesc Dl = D;
    int ref[6] = {u, D.nb[1], D.nb[4], D.nb[5], 0, 0}, nr;
    Dl.nb[1] = 1; Dl.nb[4] = 2; Dl.nb[5] = 3;
    if (D.j == B.M) {
        ref[4] = D.nb[2]; ref[5] = D.nb[3];
        Dl.nb[2] = 4; Dl.nb[3] = 5;
        nr = 6;
    } else {
        ref[4] = D.nb[0];
        Dl.nb[0] = 4;
        nr = 5;
    }
    CtxT<R> X0;
    X0.Y = static_cast<const R*>(A.Y[0]);
    X0.St = stU;
    X0.St1 = stU;
    X0.frac = R(0);
    T8 Yl[24];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        R v[4] = {R(0), R(0), R(0), R(0)};
        if (k < nr) fetch(X0, ref[k], v);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            Yl[4 * k + m] = T8(v[m]);
            const int j = 4 * k + m;
            if (j / kChunk == c) Yl[4 * k + m].d[j % kChunk] = R(1);
        }
    }
    CtxT<T8> Xl;
    Xl.Y = Yl;
    Xl.St = Xl.St1 = nullptr;
    Xl.frac = T8(0);
    T8 Vo[4];
    vis_fd<Lt::THERMAL, T8>(G, B, Xl, Dl, 0, Lt::CS2, Vo);
    R* lY0 = static_cast<R*>(A.lY[0]);
#pragma unroll
    for (int d = 0; d < kChunk; ++d) {
        const int j = kChunk * c + d;
        if (j / 4 >= nr) break;
        R g = R(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) g += lV[m] * Vo[m].d[d];
        if (g != R(0)) scatter_ref<R>(A, lY0, ref[j / 4], j % 4, R(0), g);
    }
}

// The strips' adjoints as additions to lambda^pre at their nodes.  The strip
// macros of t + 1 and of t are moments of pulled populations: their
// adjoints are coefficients on the moments (ext[0..3]).  The
// non-equilibrium moments N(t) = (sigma', q) of a node of the mesoscopic
// stencil give, per pulled population i,
//   d(lambda_N . N)/dg_i = sum_n c_n w_n(c_i; u) + sum_k nu_k dm_k/dg_i,
// c = (1 - 1/(2 tau)) (-lambda_sigma', +lambda_q) (ext[4..8]) and
// nu_k = -sum_i (sum_n c_n w_n(c_i)) dg^eq_i/dm_k (the equilibrium inside
// f^neq) + sum_a lambda_q_a sigma'_ab for k = u_b (the velocity inside the
// heat flux's weights, with sum f^neq (c - u)(c - u) = Pi^neq = -sigma' /
// (1 - 1/(2 tau)) and a traceless Pi^neq on the thermal lattices).
// Thread q also folds unknown q: lambda_U(t) = lambda_U(t+1) + the adjoints
// of the four stage fields at q (Y0 = U, Y_s = U + h k_{s-1}).
template <int LAT, typename S>
__device__ __forceinline__ void adj_extras_item(const Geom& G, const Export& E, const Band& B, const AdjState& A,
                                                const RT<S>* __restrict__ stU, const RT<S>* __restrict__ stN,
                                                int par, int q)
{
    using L = Lat<LAT>;
    using R = RT<S>;
    if (q < B.n_unk) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            double sum = 0.0;
#pragma unroll
            for (int r = 0; r < 4; ++r) sum += double(static_cast<const R*>(A.lY[r])[4LL * q + m]);
            if (q >= B.n_unk - 4 && B.ud[q].kind >= 4 && G.M > 1) sum += corner_share(G, B, A, q, m);
            const double v = A.lU[4LL * q + m] + sum;
            A.lU[4LL * q + m] = v;
            static_cast<R*>(A.lUr)[4LL * q + m] = R(v);
        }
    }
    if (q >= E.nslots) return;
    R* lSt = static_cast<R*>(A.lSt) + 4LL * q;
    R* lSt1 = static_cast<R*>(A.lSt1) + 4LL * q;
    R* Et = static_cast<R*>(A.ext[par]) + 9LL * q;
    (void)lSt1;     // the strip macros of t + 1: k_adj_strip1, after the bulk kernel
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        Et[k] += lSt[k];
        lSt[k] = R(0);
    }
    if (B.viscous != VIS_MESO) return;
    R* lN = static_cast<R*>(A.lN) + 5LL * q;
    R lam[5];
    bool any = false;
#pragma unroll
    for (int n = 0; n < 5; ++n) {
        lam[n] = lN[n];
        lN[n] = R(0);
        any = any || lam[n] != R(0);
    }
    if (!any) return;
    const R fac = R(1) - R(0.5) * R(G.omega);
    R cw[5] = {-fac * lam[0], -fac * lam[1], -fac * lam[2], fac * lam[3], fac * lam[4]};
    if (!L::THERMAL) cw[3] = cw[4] = R(0);
    const R* U = stU + 4LL * q;
    const R* N = stN + 5LL * q;
    const R ux = U[1], uy = U[2];
    R nu[4];
    eq_vjp<LAT, R>(U[0], ux, uy, U[3], R(G.rho0),
                   [&](int i) {
                       const R cx = R(L::cx(i)), cy = R(L::cy(i));
                       R phi = R(0);
#pragma unroll
                       for (int n = 0; n < 5; ++n) phi += cw[n] * neq_weight<R>(n, cx, cy, ux, uy);
                       return -phi;
                   },
                   nu);
    if (L::THERMAL) {
        nu[1] += lam[3] * N[0] + lam[4] * N[1];
        nu[2] += lam[3] * N[1] + lam[4] * N[2];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) Et[k] += nu[k];
#pragma unroll
    for (int n = 0; n < 5; ++n) Et[4 + n] += cw[n];
}

// The boundary part of one reverse step in one cooperative launch (its CTAs
// all resident): the phases above in order, each over all its items
// (thread-strided), separated by grid-wide barriers -- the Dirichlet write's
// adjoint (and the stage adjoints zeroed), the three stage fields unless the
// previous reverse step computed them (`pre`), the four stages backwards,
// the viscous vector, then lambda_U(t) and the strips' shares.  Beside the
// first three stage phases (items after the stage adjoint's) run the three
// stage fields of step t - 1 into the other stage set Zn (`nxt`), from
// U_b(t - 1) = Ubm and the strips of t - 1 and t; they depend on nothing the
// adjoint computes.  The parameter sums of the stages are reduced per block
// at the end.
template <int LAT, typename S>
__global__ void __launch_bounds__(kBandThreads, 2)
    k_adj_band(Geom G, Export E, Band B, AdjState A, StageSet Zn, const double* __restrict__ Ub,
               const double* __restrict__ Ub1, const double* __restrict__ Ubm, const CT<S>* __restrict__ lnext,
               const RT<S>* __restrict__ stU, const RT<S>* __restrict__ stN, const RT<S>* __restrict__ stU1,
               const RT<S>* __restrict__ stUm, const RT<S>* __restrict__ stNm, int par, int pre, int nxt)
{
    using R = RT<S>;
    cg::grid_group grid = cg::this_grid();
    const int nth = int(gridDim.x * blockDim.x), t0 = int(blockIdx.x * blockDim.x + threadIdx.x);
    const int nu = B.n_unk;
    StageSet Z;
#pragma unroll
    for (int q = 0; q < 4; ++q) Z.Y[q] = A.Y[q];
    Z.V = A.V;
    Z.mask = A.mask;
    // the corner unknowns, if any, are the last four
    const int ncp = (nu >= 4 && B.ud[nu - 4].kind == 4) ? 16 * (G.M * G.M - 1) : 0;
    for (int i = t0; i < 4 * nu + ncp; i += nth) {
        if (i < 4 * nu) {
            if (nxt && (i & 3) == 1) {
                R* y = static_cast<R*>(Zn.Y[0]) + 4LL * (i >> 2);
#pragma unroll
                for (int m = 0; m < 4; ++m) y[m] = R(Ubm[4LL * (i >> 2) + m]);
            }
            adj_dirichlet_item<LAT, S>(G, B, Ub, Ub1, lnext, A.lU, static_cast<R*>(A.lUr), static_cast<R*>(A.Y[0]), i);
        } else {
            adj_corner_item<LAT, S>(G, B, A, Ub1, lnext, i - 4 * nu);
        }
    }
    {
        R* z = static_cast<R*>(A.lY[0]);     // lY[0..3] and lV, contiguous
        for (long long i = t0; i < 20LL * nu; i += nth) z[i] = R(0);
    }
    grid.sync();
    if (!pre) {
        for (int s = 0; s < 3; ++s) {
            for (int u = t0; u < nu; u += nth) adj_fwd_item<LAT, S>(G, B, A, Z, stU, stN, stU1, s, u);
            grid.sync();
        }
    }
    double th[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int s = 3; s >= 0; --s) {
        const int nv = nu * kRhsChunks, nf = (nxt && s > 0) ? nu : 0;
        for (int i = t0; i < nv + nf; i += nth) {
            if (i < nv) adj_vjp_item<LAT, S>(G, B, A, stU, stU1, s, i, th);
            else adj_fwd_item<LAT, S>(G, B, A, Zn, stUm, stNm, stU, 3 - s, i - nv);
        }
        grid.sync();
    }
    if (B.viscous == VIS_MESO) {
        for (int i = t0; i < nu * kMesoChunks; i += nth) adj_vis_meso_item<LAT, S>(G, B, A, stU, stN, i);
    } else if (B.viscous == VIS_FD) {
        for (int i = t0; i < nu * kFdChunks; i += nth) adj_vis_fd_item<LAT, S>(G, B, A, stU, i);
    }
    grid.sync();
    const int nq = nu > E.nslots ? nu : E.nslots;
    for (int q = t0; q < nq; q += nth) adj_extras_item<LAT, S>(G, E, B, A, stU, stN, par, q);
    block_sum<5, kBandThreads>(th, A.sums + 1);
}

// ---------------------------------------------------------------------------
// Bulk: the collision, the pull, the loss and the strips' shares backwards
// ---------------------------------------------------------------------------

// The strip macros of t + 1 this step's boundary solver read are moments of
// the pulled populations at t + 1: their adjoint lambda_St1 adds
// pullback(lambda_St1)_i to lambda^pre_{t+1} of the strip node (atomically:
// a node can be the strip node of two sides).  Runs after k_adj_bulk.
template <int LAT, typename S>
__global__ void k_adj_strip1(Geom G, Export E, AdjState A, const RT<S>* __restrict__ Mh1, CT<S>* lcur)
{
    using L = Lat<LAT>;
    using C = CT<S>;
    using R = RT<S>;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= E.nslots) return;
    R* l1 = static_cast<R*>(A.lSt1) + 4LL * q;
    C mu[4];
    bool any = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        mu[k] = C(l1[k]);
        l1[k] = R(0);
        any = any || mu[k] != C(0);
    }
    if (!any) return;
    int s = 0;
    while (!(E.cbc[s] && q >= E.offS[s] && q < E.offS[s] + E.ND * E.L[s])) ++s;
    const int r = q - E.offS[s], d = r / E.L[s], p = r % E.L[s];
    int x, y;
    if (s == 0) { x = G.M + d; y = p; }
    else if (s == 1) { x = G.nx - 1 - G.M - d; y = p; }
    else if (s == 2) { x = p; y = G.M + d; }
    else { x = p; y = G.ny - 1 - G.M - d; }
    const R* mh = Mh1 + 4 * ((long long)y * G.nx + x);
    C b[4];
    moment_pullback<LAT, C>(C(mh[0]), C(mh[1]), C(mh[2]), L::THERMAL ? C(mh[3]) : C(0), C(G.rho0), mu, b);
    const long long node = (long long)y * G.nxp + x;
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
        atomicAdd(lcur + L::plane_of(i) * G.plane + node,
                  b[0] + b[1] * C(L::cx(i)) + b[2] * C(L::cy(i)) + b[3] * C(L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i)));
}

// lambda^pre_{t+1}(x) at every bulk node x:
//   lambda*_i   = lambda^pre_{t+2}(x + c_i, i) if x + c_i is a bulk node, else 0
//   mu          = omega a + (the loss at t + 1) + (the strips' moment coefficients),
//                 a_k = sum_i lambda*_i dg^eq_i/dm_k
//   lambda^pre_i = (1 - omega) lambda*_i + pullback(mu)_i (+ the strips' weights)
// (Eq. bgk: g* = g + omega (g^eq(m(g)) - g)); the moments m_{t+1}(x) come
// from the recomputed macros (the collision keeps them).
template <int LAT, typename S>
__global__ void __launch_bounds__(kAdjThreads)
    k_adj_bulk(Geom G, Region Rg, Export E, AdjState A, const CT<S>* __restrict__ lnext, CT<S>* __restrict__ lcur,
               const RT<S>* __restrict__ Mh1, const double* __restrict__ dPref1, int par1)
{
    using L = Lat<LAT>;
    using C = CT<S>;
    using R = RT<S>;
    const int x = Rg.x0 + blockIdx.x * kAdjThreads + threadIdx.x, y = Rg.y0 + blockIdx.y;
    double v[1] = {0.0};
    if (x < Rg.x1) {
        const long long node = (long long)y * G.nxp + x;
        C lam[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            int xs = x + L::cx(i), ys = y + L::cy(i);
            lam[i] = wrap_bulk(G, xs, ys) ? lnext[L::plane_of(i) * G.plane + (long long)ys * G.nxp + xs] : C(0);
        }
        const long long idx = (long long)y * G.nx + x;
        const R* mh = Mh1 + 4 * idx;
        const double s0d = double(mh[0]), uxd = double(mh[1]), uyd = double(mh[2]);
        const double dTd = L::THERMAL ? double(mh[3]) : 0.0;
        const C s0 = C(s0d), ux = C(uxd), uy = C(uyd), dT = C(dTd), rho0 = C(G.rho0);
        C a[4];
        eq_vjp<LAT, C>(s0, ux, uy, dT, rho0, [&](int i) { return lam[i]; }, a);
        // the loss at t + 1: (dP - dP_ref)^2, dP = c_s^2 (drho + rho0 dT + drho dT)
        const double dP = L::THERMAL ? L::CS2 * (s0d + G.rho0 * dTd + s0d * dTd) : L::CS2 * s0d;
        const double e = dP - (dPref1 ? dPref1[idx] : 0.0);
        v[0] = e * e;
        const C om = C(G.omega);
        C mu[4];
        mu[0] = om * a[0] + C(2.0 * e * L::CS2 * (L::THERMAL ? 1.0 + dTd : 1.0));
        mu[1] = om * a[1];
        mu[2] = om * a[2];
        mu[3] = om * a[3] + (L::THERMAL ? C(2.0 * e * L::CS2 * (G.rho0 + s0d)) : C(0));
        // the strips' shares at this node (a strip node of up to four sides)
        C cw[5] = {C(0), C(0), C(0), C(0), C(0)};
        bool strip = false;
        {
            const int dd[4] = {x - G.M, G.nx - 1 - G.M - x, y - G.M, G.ny - 1 - G.M - y};
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (!E.cbc[s] || dd[s] < 0 || dd[s] >= E.ND) continue;
                R* Es = static_cast<R*>(A.ext[par1]) + 9LL * (E.offS[s] + dd[s] * E.L[s] + (s < 2 ? y : x));
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    mu[k] += C(Es[k]);
                    Es[k] = R(0);
                }
#pragma unroll
                for (int n = 0; n < 5; ++n) {
                    cw[n] += C(Es[4 + n]);
                    Es[4 + n] = R(0);
                }
                strip = true;
            }
        }
        C b[4];
        moment_pullback<LAT, C>(s0, ux, uy, dT, rho0, mu, b);
        const C keep = C(1) - om;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const C cx = C(L::cx(i)), cy = C(L::cy(i));
            C r = keep * lam[i] + b[0] + b[1] * cx + b[2] * cy + b[3] * C(L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i));
            if (strip) {
#pragma unroll
                for (int n = 0; n < 5; ++n) r += cw[n] * neq_weight<C>(n, cx, cy, ux, uy);
            }
            lcur[L::plane_of(i) * G.plane + node] = r;
        }
    }
    block_sum<1>(v, A.sums + 6);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------

template <int LAT, typename S>
int adj_loss_t(const Geom& G, const Region& bulk, const void* f, const double* dPref, double* sums, void* Mout,
               const AdjRecord& rec, cudaStream_t st)
{
    // one block at least: the record is copied even without bulk nodes
    dim3 grd(std::max(1, (bulk.x1 - bulk.x0 + kAdjThreads - 1) / kAdjThreads), std::max(1, bulk.y1 - bulk.y0));
    k_adj_loss<LAT, S><<<grd, kAdjThreads, 0, st>>>(G, bulk, static_cast<const S*>(f), dPref, sums,
                                                    static_cast<RT<S>*>(Mout), rec);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// The populations the Dirichlet write of a step set, from the recorded
// boundary state U_b(t + 1): thread u writes unknown u's nodes exactly as the
// band kernel does (dirichlet(), equilibrium form, the state rounded to the
// strip type first).
template <int LAT, typename S>
__global__ void k_adj_dwrite(Geom G, Band B, const double* __restrict__ Ub1, S* __restrict__ f)
{
    using R = RT<S>;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= B.n_unk) return;
    const R Unew[4] = {R(Ub1[4LL * u]), R(Ub1[4LL * u + 1]), R(Ub1[4LL * u + 2]), R(Ub1[4LL * u + 3])};
    dirichlet<LAT, S, R>(G, B, f, nullptr, nullptr, B.ud[u], Unew);
}

template <int LAT, typename S>
int adj_dwrite_t(const Geom& G, const Band& B, const double* Ub1, void* f, cudaStream_t st)
{
    if (B.n_unk <= 0) return 0;
    k_adj_dwrite<LAT, S><<<(B.n_unk + kAdjThreads - 1) / kAdjThreads, kAdjThreads, 0, st>>>(G, B, Ub1,
                                                                                             static_cast<S*>(f));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <int LAT, typename S>
int adj_step_t(const Geom& G, const Export& E, const Band& B, const Region& bulk, const AdjState& A0,
               const double* Ub, const double* Ub1, const void* stU_, const void* stN_, const void* stU1_,
               const void* Mh1_, const double* dPref1, int par, int set, int pre, int nxt, const double* Ubm,
               const void* stUm_, const void* stNm_, cudaStream_t st, cudaStream_t sw, cudaEvent_t ev_bulk)
{
    using R = RT<S>;
    using C = CT<S>;
    AdjState A = A0;        // the current stage set
#pragma unroll
    for (int q = 0; q < 4; ++q) A.Y[q] = A0.sets[set].Y[q];
    A.V = A0.sets[set].V;
    A.mask = A0.sets[set].mask;
    StageSet Zn = A0.sets[set ^ 1];
    const R* stU = static_cast<const R*>(stU_);
    const R* stN = static_cast<const R*>(stN_);
    const R* stU1 = static_cast<const R*>(stU1_);
    const R* stUm = static_cast<const R*>(stUm_);
    const R* stNm = static_cast<const R*>(stNm_);
    const R* Mh1 = static_cast<const R*>(Mh1_);
    const C* lnext = static_cast<const C*>(A.lpre[par]);      // lambda^pre_{t+2}
    C* lcur = static_cast<C*>(A.lpre[par ^ 1]);               // lambda^pre_{t+1}
    auto blocks = [](long long n) { return int((n + kAdjThreads - 1) / kAdjThreads); };
    // the bulk (every node but the strip macros' share of t + 1) on sw,
    // beside the boundary chain on st
    if (bulk.x1 > bulk.x0 && bulk.y1 > bulk.y0) {
        dim3 grd((bulk.x1 - bulk.x0 + kAdjThreads - 1) / kAdjThreads, bulk.y1 - bulk.y0);
        k_adj_bulk<LAT, S><<<grd, kAdjThreads, 0, sw>>>(G, bulk, E, A, lnext, lcur, Mh1, dPref1, par ^ 1);
    }
    if (cudaEventRecord(ev_bulk, sw) != cudaSuccess) return -1;
    if (B.n_unk > 0 || E.nslots > 0) {
        static int grid_ctas = 0;     // per instantiation: resident CTAs of the cooperative kernel
        if (grid_ctas == 0) {
            int per_sm = 0, sms = 0, dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_band<LAT, S>, kBandThreads, 0) != cudaSuccess ||
                per_sm < 1)
                return -1;
            // two CTAs per SM at most: more measured slower (longer grid
            // barriers, less room for the kernels on the other streams)
            grid_ctas = std::min(per_sm, 2) * sms;
        }
        const double* a_Ub = Ub;
        const double* a_Ub1 = Ub1;
        const double* a_Ubm = Ubm;
        void* args[] = {const_cast<Geom*>(&G), const_cast<Export*>(&E), const_cast<Band*>(&B), &A, &Zn,
                        &a_Ub, &a_Ub1, &a_Ubm, &lnext, &stU, &stN, &stU1, &stUm, &stNm, &par, &pre, &nxt};
        if (cudaLaunchCooperativeKernel((const void*)k_adj_band<LAT, S>, dim3(grid_ctas), dim3(kBandThreads), args, 0,
                                        st) != cudaSuccess)
            return -1;
    }
    if (cudaStreamWaitEvent(st, ev_bulk, 0) != cudaSuccess) return -1;
    if (E.nslots > 0) k_adj_strip1<LAT, S><<<blocks(E.nslots), kAdjThreads, 0, st>>>(G, E, A, Mh1, lcur);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

#define ADJ_DISPATCH(lat, storage, CALL)                                   \
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

int launch_adj_loss(int lat, int storage, const Geom& G, const Region& bulk, const void* f,
                    const double* dPref, double* sums, void* Mout, const AdjRecord& rec, cudaStream_t st)
{
#define CALL(L, S) adj_loss_t<L, S>(G, bulk, f, dPref, sums, Mout, rec, st)
    ADJ_DISPATCH(lat, storage, CALL);
#undef CALL
}

int launch_adj_dwrite(int lat, int storage, const Geom& G, const Band& B, const double* Ub1, void* f,
                      cudaStream_t st)
{
#define CALL(L, S) adj_dwrite_t<L, S>(G, B, Ub1, f, st)
    ADJ_DISPATCH(lat, storage, CALL);
#undef CALL
}

int launch_adj_step(int lat, int storage, const Geom& G, const Export& E, const Band& B,
                    const Region& bulk, const AdjState& A, const double* Ub, const double* Ub1,
                    const void* stU, const void* stN, const void* stU1, const void* Mh1,
                    const double* dPref1, int par, int set, int pre, int nxt, const double* Ubm,
                    const void* stUm, const void* stNm, cudaStream_t st, cudaStream_t sw, cudaEvent_t ev_bulk)
{
#define CALL(L, S)                                                                                              \
    adj_step_t<L, S>(G, E, B, bulk, A, Ub, Ub1, stU, stN, stU1, Mh1, dPref1, par, set, pre, nxt, Ubm, stUm, stNm, \
                     st, sw, ev_bulk)
    ADJ_DISPATCH(lat, storage, CALL);
#undef CALL
}

}  // namespace lbmgb
