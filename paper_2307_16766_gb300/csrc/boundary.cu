// boundary.cu -- boundary conditions of one time step.
//
//  k_band    the characteristic boundary condition (Sec. 3) of one step in
//            one launch: each CTA takes a tile of a characteristic side,
//            updates the strip nodes next to it, integrates the boundary
//            ODE of its layers j = 1..M (and corner) over the four RK4
//            stages in shared memory, and writes the mesoscopic Dirichlet
//            populations (equilibrium or Eq. NEEP) post-collision.
//  k_zg      zero-gradient copies (Eq. zg-bc), after the bulk update.
//
// The characteristic decomposition and the RK4 update are FP64; with FP32
// or FP16 storage the fused kernel forms their inputs (stencils,
// transversal and viscous terms, strip macros) in FP32.  Every neighbour a
// right-hand side needs is resolved on the host into a UDesc: another
// unknown (stage value) or a strip node holding a bulk node's macros at t
// and t + 1 (interpolated linearly at the stage time, Sec. 3.3).
#include "charsys.cuh"

#include <algorithm>
#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace lbmgb {

namespace {

constexpr int kBandThreads = 32;   // allocation-free path: one thread per unknown
// Fused band kernel: a group of kTileThreads threads per characteristic
// component, one thread per local unknown of the tile.
constexpr int kTileThreads = kTileUnknowns;
constexpr int kCluster = 4;         // groups per band tile: one per characteristic component

// A band tile is, with FP32 / FP16 storage (MONO), one CTA of kCluster
// groups (the whole tile on one SM), and with FP64 storage a cluster of
// kCluster CTAs of one group each (one SM per characteristic component).
template <bool MONO>
constexpr int band_threads() { return MONO ? kCluster * kTileThreads : kTileThreads; }

// ---------------------------------------------------------------------------
// The band kernel: four component groups per tile
// ---------------------------------------------------------------------------
// Group r owns component / wave r of every unknown of the tile.  With FP64
// storage (one warp instruction of FP64 per 64 cycles on each SM
// sub-partition) the groups are the four CTAs of a cluster on four SMs,
// exchanging their shares through distributed shared memory; with FP32 /
// FP16 storage the wave arithmetic is float-float and the four groups share
// one CTA and its shared memory.

// Share c of the mesoscopic viscous vector (see vis_meso), in arithmetic
// type R: V1 for c = 1, V2 for c = 2; V3 is split, its conductive part for
// c = 0 and its viscous-heating part for c = 3 (V0 = 0).
template <bool TH, typename R>
__device__ R vis_meso_c(int c, const Geom& G, const R* SU, const R* SN, const UDesc& D, R cs2)
{
    if (!TH && (c == 0 || c == 3)) return R(0);
    const int s = D.kind;
    const int an = s < 2 ? 0 : 1, at = 1 - an;
    const R sn = (s == 0 || s == 2) ? R(-1) : R(1);
    auto h = [&](int k, int m) -> R {
        const R* n = SN + 5LL * D.vs[k];
        const R* u = SU + 4LL * D.vs[k];
        switch (m) {
        case 0: return an == 0 ? n[0] : n[2];
        case 1: return sn * n[1];
        case 2: return an == 0 ? n[2] : n[0];
        case 3: return sn * n[3 + an];
        case 4: return n[3 + at];
        case 5: return sn * u[1 + an];
        default: return u[1 + at];
        }
    };
    auto dn = [&](int m) { return R(0.5) * (R(3) * h(0, m) - R(4) * h(1, m) + h(2, m)); };
    auto dt = [&](int m) {
        if (D.tmode == 0) return R(0.5) * (h(3, m) - h(4, m));
        return R(D.tmode) * R(0.5) * (R(3) * h(0, m) - R(4) * h(3, m) + h(4, m));
    };
    if (c == 3) {
        const R nu = (bconst<R>(G.tau, G.tau_f) - R(0.5)) * cs2;
        const R e1 = dn(5) - dt(6), e2 = dn(6) + dt(5);
        return nu * (R(1) / cs2) * (e1 * e1 + e2 * e2);
    }
    const R irho = R(1) / (rho0_of<R>(G) + SU[4LL * D.vs[0]]);
    if (c == 1) return (dn(0) + dt(1)) * irho;
    if (c == 2) return (dn(1) + dt(2)) * irho;
    return -(dn(3) + dt(4)) * irho * (R(1) / cs2);
}

// Share c of the "-FD" viscous vector (see vis_fd), split as vis_meso_c:
// V3 = (c = 0 part) + (c = 3 part).
template <bool TH, typename R>
__device__ R vis_fd_c(int c, const Geom& G, const Band& B, const CtxT<R>& X0, const UDesc& D, int u,
                      R cs2)
{
    if (!TH && (c == 0 || c == 3)) return R(0);
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
    const R nu = (bconst<R>(G.tau, G.tau_f) - R(0.5)) * cs2;
    if (c == 1) return nu * (dnn[1] + (Tp[1] - R(2) * U[1] + Tm[1]));
    if (c == 2) return nu * (dnn[2] + (Tp[2] - R(2) * U[2] + Tm[2]));
    if (c == 0) return R(2) * nu * (dnn[3] + (Tp[3] - R(2) * U[3] + Tm[3]));
    const R d1t1 = R(0.5) * (Tp[1] - Tm[1]), d1t2 = R(0.5) * (Tp[2] - Tm[2]);
    const R e1 = d1n[1] - d1t2, e2 = d1n[2] + d1t1;
    return nu * (R(1) / cs2) * (e1 * e1 + e2 * e2);
}

// Lab component m of a local-frame vector (m = 1, 2 need k1 and k2).
__device__ __forceinline__ double lab_component(int m, int kind, double r, double k0, double k1,
                                                double k2, double k3)
{
    if (m == 0) return k0;
    if (m == 3) return k3;
    switch (kind) {
    case 0: return m == 1 ? -k1 : k2;
    case 1: return m == 1 ? k1 : k2;
    case 2: return m == 1 ? k2 : -k1;
    case 3: return m == 1 ? k2 : k1;
    default: {
        const int c = kind - 4;
        const double n0 = (c & 1) ? r : -r, n1 = (c & 2) ? r : -r;
        return m == 1 ? k1 * n0 - k2 * n1 : k1 * n1 + k2 * n0;
    }
    }
}

// The band kernel forms the inputs of the characteristic system (stencils,
// transversal and viscous terms, strip-node macros) in StripReal<S>: FP64
// with FP64 storage, FP32 otherwise.  The characteristic decomposition
// (projection on the waves, wave amplitudes with their relaxation towards
// the targets, and back to the lab frame) and the RK4 update of the
// boundary state are FP64 with FP64 storage and float-float (below)
// otherwise; the boundary state is kept in FP64 between steps.

// Exchanges inside a cluster without a cluster barrier: a CTA stores a
// value into the shared memory of every CTA of its cluster with st.async,
// which counts the bytes on the receiving CTA's transaction barrier; each
// CTA expects the bytes of one exchange on its own barrier and waits for
// them (bounded).
__device__ __forceinline__ unsigned cluster_map(unsigned a, unsigned q)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(q));
    return r;
}

__device__ __forceinline__ void put_async(unsigned a, double v, unsigned bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];"
                 ::"r"(a), "l"(__double_as_longlong(v)), "r"(bar) : "memory");
}

// Unevaluated sums hi + lo of two floats ("float-float"), built from the
// error-free transformations TwoSum (Knuth) and TwoProduct (by FMA): about
// 48 significant bits at FP32 issue cost.  The band kernel forms the wave
// amplitudes and the right-hand side with FP32 and FP16 storage in them
// instead of FP64 (one FP64 warp instruction per 64 cycles on each SM
// sub-partition; with the four components of a tile on one SM the FP64
// work would queue there): their projections S dU/dn cancel (an acoustic
// wave has a small entropy part), and plain FP32 lost accuracy there.
struct FF {
    float h, l;
};
__device__ __forceinline__ FF ff_fast(float a, float b)      // |a| >= |b|
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ FF ff_two_sum(float a, float b)
{
    const float s = a + b, z = s - a;
    return {s, (a - (s - z)) + (b - z)};
}
__device__ __forceinline__ FF ff_prod(float a, float b)
{
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ FF ff_add(FF x, FF y)
{
    const FF s = ff_two_sum(x.h, y.h), t = ff_two_sum(x.l, y.l);
    const FF u = ff_fast(s.h, s.l + t.h);
    return ff_fast(u.h, u.l + t.l);
}
__device__ __forceinline__ FF ff_neg(FF x) { return {-x.h, -x.l}; }
__device__ __forceinline__ FF ff_mul(FF x, float b)
{
    const FF p = ff_prod(x.h, b);
    return ff_fast(p.h, fmaf(x.l, b, p.l));
}
__device__ __forceinline__ FF ff_mul(FF x, FF y)
{
    const FF p = ff_prod(x.h, y.h);
    return ff_fast(p.h, fmaf(x.h, y.l, fmaf(x.l, y.h, p.l)));
}
__device__ __forceinline__ double ff_to_double(FF x) { return double(x.h) + double(x.l); }
__device__ __forceinline__ double ff_pack(FF x)
{
    return __hiloint2double(__float_as_int(x.h), __float_as_int(x.l));
}
__device__ __forceinline__ FF ff_unpack(double v)
{
    return {__int_as_float(__double2hiint(v)), __int_as_float(__double2loint(v))};
}
__device__ __forceinline__ FF ff_const(const float (&c)[2]) { return {c[0], c[1]}; }
__device__ __forceinline__ FF ff_scale(FF x, float p2) { return {x.h * p2, x.l * p2}; }   // p2: a power of 2
__device__ __forceinline__ FF ff_split(double d)
{
    const float h = float(d);
    return {h, float(d - double(h))};
}

// v into slot p of every CTA of the cluster, counted on barrier `bar` there
template <typename T>
__device__ __forceinline__ void put_cluster(T* p, T v, unsigned long long* bar)
{
    const unsigned a = smem_u32(p), b = smem_u32(bar);
#pragma unroll
    for (unsigned q = 0; q < kCluster; ++q) put_async(cluster_map(a, q), v, cluster_map(b, q));
}

__device__ __forceinline__ void expect_bytes(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Wait for phase `parity` of an exchange barrier, at most 1 s; a timeout is
// recorded as bit 2 of *status (the values read after it are not valid) and
// returns false.
__device__ __forceinline__ bool wait_exchange(unsigned long long* bar, unsigned parity, int* status)
{
    const unsigned b = smem_u32(bar);
    const unsigned long long t0 = global_ns();
    for (;;) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n"
            " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(b), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > 1000000000ull) {
            atomicOr(status, 4);
            return false;
        }
    }
}

__device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }

// One tile of the boundary band: a run of positions of one characteristic
// side (all M layers, and the corner next to it on a W/E side), plus the
// halo its four RK4 stages need (Sec. 3.3).  Four groups of 128 threads
// (MONO: one CTA; FP64: a cluster of four CTAs), group r forming wave r and
// lab component r of every local unknown.
//
// 1. Strip nodes: the tile pulls the bulk nodes at depths 0..2 next to the
//    side that its stencils read (Eq. lbe) for their macros at t + 1
//    (Eq. macro), and keeps them with the stored macros and moments of t in
//    shared memory (every CTA of a cluster); for its own positions it also
//    writes the macros and non-equilibrium moments of t + 1 for the next
//    step.  (The bulk kernel updates the populations of these nodes.)
// 2. RK4 (Sec. 3.3, "Time integration"): the local table lists the tile's
//    unknowns by level: level 0 are owned, level l computes the first 4 - l
//    stages, level 4 only supplies U(t).  Per stage, the inputs of the
//    characteristic system (1/rho, sqrt(theta), 1/sqrt(theta), P - P_inf
//    and the transversal terms; in type R), then wave r, then lab component
//    r of the right-hand side and of the stage value (float-float with
//    FP32 / FP16 storage, FP64 with FP64 storage; stage values are shared in
//    type R).  Stage 0 freezes the viscous vector and the incoming-wave
//    mask of time t.
// 3. The owners write U(t + 1) and the mesoscopic Dirichlet populations
//    (equilibrium or Eq. NEEP), shared out over the four groups.
template <int LAT, typename S, bool REF, bool MONO>
__device__ __forceinline__ void band_tile(const Geom& G, const Offsets& O, const Band& B,
                                          const Export& E, const S* __restrict__ fin,
                                          S* __restrict__ f, int par_t, int tile)
{
    using L = Lat<LAT>;
    using C = typename Store<S>::C;
    using R = typename StripReal<S>::T;
    constexpr bool TH = L::THERMAL;
    // a kernel launched after this one for early start (the bulk update,
    // which reads only the old buffer) may begin now
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // MONO (FP32 / FP16 storage): one CTA of four 128-thread groups per
    // tile, group r in the role of cluster rank r, exchanging through its
    // own shared memory (the tile then holds one SM and leaves the others to
    // the bulk kernel); FP64 storage: a cluster of four 128-thread CTAs.
    static_assert(!MONO || sizeof(S) < 8, "FP64 storage keeps the cluster form");
    const int grp = MONO ? int(threadIdx.x / kTileThreads) : int(cg::this_cluster().block_rank());
    const int l = int(threadIdx.x % kTileThreads);
    // MONO: groups 0 and 1 do the strip phase for the tile; meanwhile the
    // eight warps of groups 2 and 3 run one stage and the Dirichlet write
    // without effect (no stores, no waits), each warp one part of that code
    // with its lanes in all four roles, so that the code is in the SM's
    // instruction caches when the tile reaches it (measured: the first
    // stage otherwise waits several microseconds on instruction fetch under
    // the bulk kernel's traffic, and one warp fetching it all in sequence
    // takes longer than the strip phase).
    const bool puller = !MONO || grp < 2;
    __shared__ __align__(16) R Ys[kTileThreads * 4];        // stage values, lab frame
    __shared__ __align__(16) R Xp[kTileThreads * 8];        // shares of the system's inputs
    __shared__ __align__(16) double Xw[kTileThreads * 4];   // wave amplitudes
    __shared__ __align__(16) R Xv[kTileThreads * 4];        // viscous vector (local frame, frozen)
    // exchange barriers: waves of even / odd stages, stage values of even /
    // odd stages
    __shared__ __align__(8) unsigned long long xbar[4];
    extern __shared__ __align__(16) unsigned char dyn_raw[];
    R* SUt = reinterpret_cast<R*>(dyn_raw);        // [max_nodes][4] macros of t
    R* SUt1 = SUt + 4 * B.max_nodes;               // [max_nodes][4] macros of t + 1
    R* SNt = SUt1 + 4 * B.max_nodes;               // [max_nodes][5] moments of t
    S* Fx = reinterpret_cast<S*>(SNt + 5 * B.max_nodes);   // [max_fx][Q], node k in CTA k % 4
    auto bcast = [&](auto* p, auto v) {
        if constexpr (MONO) {
            *p = v;
        } else {
            cg::cluster_group cl = cg::this_cluster();
#pragma unroll
            for (int q = 0; q < kCluster; ++q) *cl.map_shared_rank(p, q) = v;
        }
    };
    auto sync_all = [&]() {
        if constexpr (MONO) __syncthreads();
        else cg::this_cluster().sync();
    };
    // the stage exchanges: a value into slot p of every group, then the wait
    // for all of them
    auto xput = [&](auto* p, auto v, unsigned long long* bar) {
        if constexpr (MONO) *p = v;
        else put_cluster(p, v, bar);
    };
    auto xwait = [&](unsigned long long* bar, unsigned parity) -> bool {
        if constexpr (MONO) {
            __syncthreads();
            return true;
        } else {
            return wait_exchange(bar, parity, B.status);
        }
    };
    // Descriptors first, all at once: under a saturated memory system each
    // dependent global round trip costs microseconds.
    const int ns = B.max_nodes;
    const StripNode* snt = B.sn + (long long)tile * ns;
    // the strip node this thread pulls: node k goes to CTA k % 4 (MONO:
    // group k % 2), and the nodes of a CTA (group) are dealt round its four
    // warps
    constexpr int kPullStride = MONO ? 2 * kTileThreads : kCluster * kTileThreads;
    const int kp = MONO ? (grp & 1) + 2 * (4 * (l % 32) + l / 32) : grp + kCluster * (4 * (l % 32) + l / 32);
    // the time-t slots this thread loads: nodes tl, tl + tstride, ...
    // (descriptors of the first kLT issued here, the rest in a loop); every
    // CTA of a cluster loads all of them into its own shared memory
    constexpr int kLT = 3;
    constexpr int tstride = MONO ? 2 * kTileThreads : kTileThreads;
    const int tl = MONO ? int(threadIdx.x) : l;
    auto load_desc = [&](StripNode& Nb, int* tsl) {
        Nb = StripNode{-1, -1, 0, -1, -1, 0};
        if (puller && kp < ns) Nb = snt[kp];
#pragma unroll
        for (int j = 0; j < kLT; ++j) {
            const int k = tl + j * tstride;
            tsl[j] = -1;
            if (puller && k < ns) {
                const StripNode& N = snt[k];
                if (N.x >= 0 && (N.flags & kSNLoadT)) tsl[j] = N.tslot;
            }
        }
    };
    // the cluster form issues them before its cluster barrier; the one-CTA
    // form at the start of the strip phase (they are dead after it)
    StripNode NbC;
    int tslC[kLT];
    if constexpr (!MONO) load_desc(NbC, tslC);
    const UDesc D = B.ld[(long long)tile * kTileUnknowns + l];
    int nc0 = 0, nc1 = 0, nc2 = 0, nc3 = 0;
    if constexpr (!MONO) {
        if (l == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&xbar[k])));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        // unknowns that compute stage s (the same in every CTA of the cluster)
        nc0 = __syncthreads_count(D.level <= 3);
        nc1 = __syncthreads_count(D.level <= 2);
        nc2 = __syncthreads_count(D.level <= 1);
        nc3 = __syncthreads_count(D.level <= 0);
    }
    if constexpr (!MONO) sync_all();    // every CTA of the cluster runs before any remote store

    // 1. strip nodes: macros of t and moments of t for every CTA; macros of
    //    t + 1 (pull and Eq. macro) by CTA k % kCluster (MONO: group k % 2)
    //    for node k, shared out; post-collision populations of Eq. NEEP
    //    sources kept locally
    const R* gU = static_cast<const R*>(E.stripU) + (long long)par_t * E.nslots * 4;
    const R* gN = static_cast<const R*>(E.stripN) + (long long)par_t * E.nslots * 5;
    const bool meso = B.viscous == VIS_MESO;
    auto load_t = [&](int k, int ts) {
#pragma unroll
        for (int c = 0; c < 4; ++c) SUt[4 * k + c] = gU[4LL * ts + c];
        if (meso) {
#pragma unroll
            for (int c = 0; c < 5; ++c) SNt[5 * k + c] = gN[5LL * ts + c];
        }
    };
    auto pull_t1 = [&](int k, const StripNode& N) {
        C g[L::Q];
        pull_plain<LAT, S, C>(G, O, fin, N.x, N.y, g);
        if (Store<S>::SCALED) {
#pragma unroll
            for (int i = 0; i < L::Q; ++i) g[i] *= C(L::w(i));
        }
        Moments<LAT, C> m;
        if (N.fx >= 0) {
            S* fx = Fx + N.fx * L::Q;
            m = collide<LAT, C, REF>(G, g, [&](int i, C v) {
                if (Store<S>::SCALED) v *= C(1.0 / L::w(i));
                Store<S>::put(fx + i, v);
            });
        } else {
            m = moments_G<LAT, C, REF>(G, g);
        }
        const R U1[4] = {R(m.s0), R(m.ux), R(m.uy), R(m.dT)};
#pragma unroll
        for (int c = 0; c < 4; ++c) bcast(SUt1 + 4 * k + c, U1[c]);
        if (N.gslot >= 0) {             // the strips of t + 1, for the next step
            R* u = static_cast<R*>(E.stripU) + ((long long)(par_t ^ 1) * E.nslots + N.gslot) * 4;
#pragma unroll
            for (int c = 0; c < 4; ++c) u[c] = U1[c];
            if (N.flags & kSNNeq) {     // a node of the mesoscopic stencil
                R N1[5];
                neq_moments<LAT, C, R>(g, m, R(1) - R(0.5) * omega_of<R>(G), N1);
                R* q = static_cast<R*>(E.stripN) + ((long long)(par_t ^ 1) * E.nslots + N.gslot) * 5;
#pragma unroll
                for (int c = 0; c < 5; ++c) q[c] = N1[c];
            }
        }
    };
    // U(t) of the tile's unknowns, loaded with the strip's own loads: in the
    // cluster form by every CTA, which keeps its component grp (u0g); in
    // the one-CTA form by group 0, which leaves it in shared memory for all
    // groups (Ys in R, U0s in FP64)
    const int lev = D.level;            // > 4: no unknown on this thread
    __shared__ __align__(16) double U0s[MONO ? 4 * kTileThreads : 1];
    double u0g = 0.0;
    auto strip = [&](const StripNode& Nb, const int* tsl) {
        double U0[4] = {0.0, 0.0, 0.0, 0.0};
        if (lev <= 4 && (!MONO || grp == 0)) {
            const double2* p = reinterpret_cast<const double2*>(B.Ub + ((long long)par_t * B.n_unk + D.gid) * 4);
            const double2 a = p[0], b = p[1];
            U0[0] = a.x; U0[1] = a.y; U0[2] = b.x; U0[3] = b.y;
        }
#pragma unroll
        for (int j = 0; j < kLT; ++j)
            if (tsl[j] >= 0) load_t(tl + j * tstride, tsl[j]);
        if (Nb.x >= 0 && (Nb.flags & kSNPull)) pull_t1(kp, Nb);
        for (int k = tl + kLT * tstride; k < ns; k += tstride) {
            const StripNode N = snt[k];
            if (N.x >= 0 && (N.flags & kSNLoadT)) load_t(k, N.tslot);
        }
        for (int k = kp + kPullStride; k < ns; k += kPullStride) {
            const StripNode N = snt[k];
            if (N.x >= 0 && (N.flags & kSNPull)) pull_t1(k, N);
        }
        if (lev <= 4 && (!MONO || grp == 0)) {
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                Ys[4 * l + m] = R(U0[m]);
                if constexpr (MONO) U0s[4 * l + m] = U0[m];
            }
        }
        if constexpr (!MONO) u0g = grp == 0 ? U0[0] : grp == 1 ? U0[1] : grp == 2 ? U0[2] : U0[3];
    };
    if constexpr (!MONO) {
        strip(NbC, tslC);
        sync_all();
    }

    // 2. RK4, component rank of every unknown, and 3. the Dirichlet write
    // (pass 1).  MONO: pass 0 is the strip phase in groups 0 and 1 and the
    // warm-up in groups 2 and 3, which runs the one copy of this code.
    static_assert(!MONO || sizeof(R) == 4, "the one-CTA form keeps every input local");
#pragma unroll 1
    for (int pass = MONO ? 0 : 1; pass < 2; ++pass) {
      const bool dry = pass == 0;
      if (dry && puller) {
        StripNode Nb;
        int tsl[kLT];
        load_desc(Nb, tsl);
        strip(Nb, tsl);
      } else {
        // warm-up: eight warps, one code part each (0: A's stencils and
        // inputs, 1: A's viscous vector, 2: B, 3 and 4: C in roles 0-1 and
        // 2-3, 5: the Dirichlet write, 6 and 7: none) with their lanes in
        // every role of the part; the real pass: part 8, all of it
        const int part = dry ? int(threadIdx.x / 32) % 8 : 8;
        const int rank = !dry ? grp
                       : part == 3 ? int(threadIdx.x % 2)
                       : part == 4 ? 2 + int(threadIdx.x % 2) : int(threadIdx.x % 4);
        CtxT<R> X;
        X.Y = Ys;
        X.St = SUt;
        X.St1 = SUt1;
        const R rho0r = rho0_of<R>(G), cs2r = R(L::CS2), kr = bconst<R>(B.kR, B.kR_f);
        const R kAr = bconst<R>(B.kA, B.kA_f), kBr = bconst<R>(B.kB, B.kB_f), ihcsr = bconst<R>(B.ihcs, B.ihcs_f),
                csr_ = bconst<R>(B.cs, B.cs_f);
        const bool corner = lev <= 4 && D.kind >= 4;
        const int scheme = corner ? SCH_LODI : (lev <= 4 ? B.scheme[D.kind] : 0);
        const bool cbc = scheme == SCH_CBC || scheme == SCH_CBC_RELAX;
        double acc = 0.0, kc = 0.0;         // lab component rank of sum k and of the last k
        const double u0r = [&] {            // component grp of U(t)
            if constexpr (MONO) return U0s[4 * l + grp];
            else return u0g;
        }();
        FF accf{0.0f, 0.0f};                // the same sum in float-float (FP32 / FP16 storage)
        const FF u0f = ff_split(u0r);
        bool incoming = false;              // wave rank incoming at time t
        // In FP32 every CTA forms all inputs of the system itself; in FP64 each
        // CTA forms a share and the shares are exchanged (FP64 issue is slow).
        constexpr bool kLocal = sizeof(R) == 4;
        R xs[8] = {0, 0, 0, 0, 0, 0, 0, 0}; // the inputs, kLocal
        R Vs[4] = {0, 0, 0, 0};             // viscous vector (local frame, frozen), kLocal
        bool xok = true;                    // every exchange so far completed in time
        for (int stage = 0; stage < (dry ? 1 : 4); ++stage) {
            const bool comp = lev <= 3 - stage;
            if (!MONO && l == 0) {          // bytes of this stage's two exchanges
                const unsigned ncomp = unsigned(stage == 0 ? nc0 : stage == 1 ? nc1 : stage == 2 ? nc2 : nc3);
                expect_bytes(&xbar[stage & 1], unsigned(kCluster * sizeof(double)) * ncomp);
                expect_bytes(&xbar[2 + (stage & 1)], unsigned(kCluster * sizeof(R)) * ncomp);
            }
            X.frac = stage == 0 ? R(0) : (stage == 3 ? R(1) : R(0.5));
            R Ul[4] = {0, 0, 0, 0}, dUn[4] = {0, 0, 0, 0};
            R d_ut = 0;
            // A: inputs of the system, type R: 1/rho, the transversal terms,
            // sqrt(theta), 1/sqrt(theta), P - P_inf and d(rho T)/dt (thermal) or
            // d rho/dt (isothermal)
            if (comp && (part == 8 || part <= 1)) {
                const int kind = D.kind;
                R A[4], Bv[4], Up[4], Um[4];
                if (part != 1) {             // (the warm-up's part 1: the viscous vector only)
                    fetch_local(X, l, kind, kr, Ul);
                    if (corner) {
                        // LODI along the outward diagonal, one-sided difference of
                        // spacing sqrt(2) through the two diagonal bulk nodes
                        fetch_local(X, D.nb[0], kind, kr, A);
                        fetch_local(X, D.nb[1], kind, kr, Bv);
                        const R kC = bconst<R>(B.kC, B.kC_f);
#pragma unroll
                        for (int m = 0; m < 4; ++m) dUn[m] = (R(3) * Ul[m] - R(4) * A[m] + Bv[m]) * kC;
#pragma unroll
                        for (int m = 0; m < 4; ++m) Up[m] = Um[m] = R(0);
                    } else {
                        if (D.j == B.M) {        // Eq. FD-dx-bw at the outermost layer
                            fetch_local(X, D.nb[1], kind, kr, A);
                            fetch_local(X, D.nb[2], kind, kr, Bv);
#pragma unroll
                            for (int m = 0; m < 4; ++m) dUn[m] = R(0.5) * (R(3) * Ul[m] - R(4) * A[m] + Bv[m]);
                        } else {                 // Eq. FD-dx-center at inner layers
                            fetch_local(X, D.nb[0], kind, kr, A);
                            fetch_local(X, D.nb[1], kind, kr, Bv);
#pragma unroll
                            for (int m = 0; m < 4; ++m) dUn[m] = R(0.5) * (A[m] - Bv[m]);
                        }
                        fetch_local(X, D.nb[4], kind, kr, Up);
                        fetch_local(X, D.nb[5], kind, kr, Um);
                    }
                    d_ut = R(0.5) * (Up[2] - Um[2]);
                }
                // share q of the inputs (q = 0..3: entries {0,1}, {2,3},
                // {4,5,6 isothermal}, {6,7 thermal})
                auto input = [&](int i) -> R {
                    switch (i) {
                    case 0: return R(1) / (rho0r + Ul[0]);
                    case 1: return corner ? R(0) : R(-0.5) * ((rho0r + Up[0]) * Up[2] - (rho0r + Um[0]) * Um[2]);
                    case 2: return TH ? sqrt_r(R(1) + Ul[3]) : R(0);
                    case 3: return corner ? R(0) : -Ul[2] * (R(0.5) * (Up[1] - Um[1]));
                    case 4: return TH ? rsqrt_r(R(1) + Ul[3]) : R(0);
                    case 5: {
                        const R dP = TH ? cs2r * (Ul[0] + rho0r * Ul[3] + Ul[0] * Ul[3]) : cs2r * Ul[0];
                        return corner ? R(0) : dP - bconst<R>(B.pdev[kind], B.pdev_f[kind]);
                    }
                    case 6:
                        // rho T - rho0 = drho + rho0 dT + drho dT
                        return TH ? R(0.5) * ((Up[0] + rho0r * Up[3] + Up[0] * Up[3]) -
                                              (Um[0] + rho0r * Um[3] + Um[0] * Um[3]))
                                  : R(0.5) * (Up[0] - Um[0]);
                    default:
                        return (TH && !corner) ? R(-0.5) * ((R(1) + Up[3]) * Up[2] - (R(1) + Um[3]) * Um[2]) : R(0);
                    }
                };
                if constexpr (kLocal) {
                    if (part != 1) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) xs[i] = input(i);
                    }
                    if (stage == 0 && !corner && part != 0) {
                        if (B.viscous == VIS_FD) {
#pragma unroll
                            for (int c = 0; c < 4; ++c) Vs[c] = vis_fd_c<TH, R>(c, G, B, X, D, l, cs2r);
                        } else if (B.viscous == VIS_MESO) {
#pragma unroll
                            for (int c = 0; c < 4; ++c) Vs[c] = vis_meso_c<TH, R>(c, G, SUt, SNt, D, cs2r);
                        }
                    }
                } else {
                    R* xp = Xp + 8 * l;
                    if (rank == 0) {
                        bcast(xp + 0, input(0));
                        bcast(xp + 1, input(1));
                    } else if (rank == 1) {
                        if (TH) bcast(xp + 2, input(2));
                        bcast(xp + 3, input(3));
                    } else if (rank == 2) {
                        if (TH) bcast(xp + 4, input(4));
                        bcast(xp + 5, input(5));
                        if (!TH) bcast(xp + 6, input(6));
                    } else if (TH) {
                        bcast(xp + 6, input(6));
                        bcast(xp + 7, input(7));
                    }
                    if (stage == 0) {
                        R v = R(0);
                        if (!corner && B.viscous == VIS_FD) v = vis_fd_c<TH, R>(rank, G, B, X, D, l, cs2r);
                        else if (!corner && B.viscous == VIS_MESO) v = vis_meso_c<TH, R>(rank, G, SUt, SNt, D, cs2r);
                        bcast(Xv + 4 * l + rank, v);
                    }
                }
            }
            if constexpr (!kLocal) sync_all();
            // B: wave rank, FP64.  Row rank of S (see apply_S) applied to dU/dn,
            // T and V, with Lambda_rank.
            auto XP = [&](int i) -> R {
                if constexpr (kLocal) return xs[i];
                else return Xp[8 * l + i];
            };
            R TTr[4] = {0, 0, 0, 0};        // transversal terms, local frame
            R Vr[4] = {0, 0, 0, 0};
            if (comp && (part == 8 || part == 2)) {
                if (!corner) {
                    TTr[0] = XP(1);
                    TTr[1] = XP(3);
                    TTr[2] = -cs2r * XP(0) * XP(6) - Ul[2] * d_ut;
                    TTr[3] = TH ? XP(7) : R(0);
                }
                if constexpr (kLocal) {
                    Vr[1] = Vs[1];
                    Vr[2] = Vs[2];
                    Vr[3] = TH ? Vs[0] + Vs[3] : R(0);      // V0 = 0; V3 from two shares
                } else {
                    const R* xv = Xv + 4 * l;
                    Vr[1] = xv[1];
                    Vr[2] = xv[2];
                    Vr[3] = TH ? xv[0] + xv[3] : R(0);
                }
                // Row `rank` of S (see apply_S) and Lambda_rank.  Their entries
                // are formed from the inputs in type R (the inputs' own
                // precision) and only the non-zero ones enter the FP64
                // projections: thermal rows (-r/2, 0, 0, 1/2), (0, 0, 1, 0),
                // (r/4, -+a, 0, 1/4); isothermal rows (1/2, -+h, 0), (0, 0, 1).
                R c0 = R(0), c1 = R(0), c3 = R(0), lamr = Ul[1];
                bool acoustic = false;
                if (TH) {
                    const R rr = (R(1) + Ul[3]) * XP(0);
                    if (rank == 0) {
                        c0 = R(-0.5) * rr;
                        c3 = R(0.5);
                    } else if (rank >= 2) {
                        const R sg = rank == 2 ? R(-1) : R(1);
                        c0 = R(0.25) * rr;
                        c1 = sg * XP(2) * kAr;
                        c3 = R(0.25);
                        lamr = Ul[1] + sg * XP(2) * kBr;
                        acoustic = true;
                    }
                } else if (rank == 0 || rank == 2) {
                    const R sg = rank == 0 ? R(-1) : R(1);
                    c0 = R(0.5);
                    c1 = sg * (rho0r + Ul[0]) * ihcsr;
                    lamr = Ul[1] + sg * csr_;
                    acoustic = true;
                }
                double w = 0.0;
                if constexpr (kLocal) {
                    // the wave in float-float; every product of two inputs is
                    // exact in it, as in FP64
                    auto srow = [&](const R* v) -> FF {
                        if (rank == 1) return FF{v[2], 0.0f};
                        if (TH) {
                            const FF sr = ff_add(ff_prod(c0, v[0]), ff_prod(c3, v[3]));
                            return rank == 0 ? sr : ff_add(sr, ff_prod(c1, v[1]));
                        }
                        return ff_add(ff_prod(c0, v[0]), ff_prod(c1, v[1]));
                    };
                    if (stage == 0) incoming = lamr < R(0);
                    FF wf{0.0f, 0.0f};
                    if (TH || rank != 3) {
                        if (!incoming) {
                            wf = ff_mul(srow(dUn), lamr);
                        } else if (scheme != SCH_LODI) {
                            const FF st = srow(TTr);
                            const FF relaxP = acoustic ? ff_mul(ff_const(B.ffk[FFK_BP]), XP(5)) : FF{0.0f, 0.0f};
                            if (scheme == SCH_LODI_RELAX) {
                                wf = ff_add(ff_mul(ff_add(ff_const(B.ffk[FFK_TINF]), ff_neg(st)),
                                                   ff_const(B.ffk[FFK_AT])),
                                            relaxP);
                            } else if (scheme == SCH_CBC) {
                                wf = B.viscous != VIS_OFF ? ff_add(st, srow(Vr)) : st;
                            } else {
                                // Eq. CBC-Relax; the viscous term relaxed towards 0
                                // at rate alpha_V (0: the paper's equation)
                                wf = ff_add(ff_mul(st, ff_const(B.ffk[FFK_1MAT])), ff_const(B.ffk[FFK_ATTI]));
                                if (B.viscous != VIS_OFF) wf = ff_add(wf, ff_mul(srow(Vr), ff_const(B.ffk[FFK_1MAV])));
                                wf = ff_add(wf, relaxP);
                            }
                        }
                    }
                    w = ff_pack(wf);
                } else {
                    const double d0 = double(c0), d1 = double(c1), d3 = double(c3);
                    auto srow = [&](const R* v) -> double {
                        if (rank == 1) return double(v[2]);
                        if (TH) {
                            const double sr = d0 * double(v[0]) + d3 * double(v[3]);
                            return rank == 0 ? sr : sr + d1 * double(v[1]);
                        }
                        return d0 * double(v[0]) + d1 * double(v[1]);
                    };
                    const double lam = double(lamr);
                    if (stage == 0) incoming = lam < 0.0;
                    if (TH || rank != 3) {
                        if (!incoming) {
                            w = lam * srow(dUn);
                        } else if (scheme != SCH_LODI) {
                            const double st = srow(TTr);
                            const double relaxP = acoustic ? B.beta_P * double(XP(5)) : 0.0;
                            if (scheme == SCH_LODI_RELAX) w = B.alpha_T * (B.t_inf - st) + relaxP;
                            // the viscous projection (none when the viscous vector is off)
                            else if (scheme == SCH_CBC) w = st + (B.viscous != VIS_OFF ? srow(Vr) : 0.0);
                            else {
                                // Eq. CBC-Relax; the viscous term relaxed towards 0
                                // at rate alpha_V (0: the paper's equation)
                                const double sv = B.viscous != VIS_OFF ? srow(Vr) : 0.0;
                                w = (1.0 - B.alpha_T) * st + (1.0 - B.alpha_V) * sv + B.alpha_T * B.t_inf + relaxP;
                            }
                        }
                    }
                }
                if (!dry) xput(Xw + 4 * l + rank, w, &xbar[stage & 1]);
                // the transversal and viscous terms this CTA adds in step C
                if (cbc) {
                    if (rank == 3) {
                        TTr[3] += Vr[3];
                    } else if (rank != 0) {         // V0 = 0
                        TTr[1] += Vr[1];
                        TTr[2] += Vr[2];
                    }
                }
            }
            if (xok && !dry) xok = xwait(&xbar[stage & 1], (stage >> 1) & 1);
            // C: lab component rank of the right-hand side (S^-1 of the waves,
            // with r^-1 = rho / theta, b = sqrt(2 c_s^4 / T~) formed in type R);
            // RK4 update (FP64).  A side unknown's lab component 1 or 2 needs
            // one local component only.
            if (comp && (part == 8 || part == 3 || part == 4)) {
                if constexpr (kLocal) {
                    // float-float from the waves to the lab component; one
                    // conversion to FP64 for the RK4 sum
                    const double* wp = Xw + 4 * l;
                    const FF w0 = ff_unpack(wp[0]), w1 = ff_unpack(wp[1]), w2 = ff_unpack(wp[2]),
                             w3 = ff_unpack(wp[3]);
                    const FF zero{0.0f, 0.0f};
                    FF kl1 = zero, kl2 = zero, klr = zero;
                    if (rank == 0) {
                        if (TH) {
                            const R irr = (rho0r + Ul[0]) * XP(4) * XP(4);
                            klr = ff_neg(ff_mul(ff_add(ff_add(w2, w3), ff_neg(w0)), irr));
                        } else {
                            klr = ff_neg(ff_add(w0, w2));
                        }
                        if (cbc) klr = ff_add(klr, FF{TTr[0], 0.0f});
                    } else if (rank == 3) {
                        klr = TH ? ff_neg(ff_add(ff_add(w0, w2), w3)) : zero;
                        if (cbc && TH) klr = ff_add(klr, FF{TTr[3], 0.0f});
                    } else {
                        const bool sideW = D.kind < 2;
                        const bool need1 = corner || ((rank == 1) == sideW);
                        const bool need2 = corner || ((rank == 1) != sideW);
                        if (need1) {
                            const R bf = TH ? XP(4) * kBr : csr_ * XP(0);
                            kl1 = ff_neg(ff_mul(TH ? ff_add(w3, ff_neg(w2)) : ff_add(w2, ff_neg(w0)), bf));
                            if (cbc) kl1 = ff_add(kl1, FF{TTr[1], 0.0f});
                        }
                        if (need2) {
                            kl2 = ff_neg(w1);
                            if (cbc) kl2 = ff_add(kl2, FF{TTr[2], 0.0f});
                        }
                    }
                    // lab component (lab_component's selection, in float-float)
                    FF kf;
                    if (rank == 0 || rank == 3) {
                        kf = klr;
                    } else if (D.kind < 4) {
                        const int kind = D.kind;
                        kf = kind == 0 ? (rank == 1 ? ff_neg(kl1) : kl2)
                           : kind == 1 ? (rank == 1 ? kl1 : kl2)
                           : kind == 2 ? (rank == 1 ? kl2 : ff_neg(kl1))
                                       : (rank == 1 ? kl2 : kl1);
                    } else {
                        const int c = D.kind - 4;
                        const FF r = ff_const(B.ffk[FFK_KR]);
                        const FF n0 = (c & 1) ? r : ff_neg(r), n1 = (c & 2) ? r : ff_neg(r);
                        kf = rank == 1 ? ff_add(ff_mul(kl1, n0), ff_neg(ff_mul(kl2, n1)))
                                       : ff_add(ff_mul(kl1, n1), ff_mul(kl2, n0));
                    }
                    // RK4 (sum and stage value) in float-float as well: no
                    // FP64 instruction in the stage loop
                    if (stage < 3) {
                        const FF k2 = stage == 0 ? kf : ff_scale(kf, 2.0f);
                        accf = stage == 0 ? k2 : ff_add(accf, k2);
                        const FF y = ff_add(u0f, ff_scale(kf, stage == 2 ? 1.0f : 0.5f));
                        if (!dry) xput(Ys + 4 * l + rank, y.h, &xbar[2 + (stage & 1)]);
                    } else {
                        // RK4: U(t + 1) = U(t) + (k1 + 2 k2 + 2 k3 + k4) / 6
                        const FF un = ff_add(u0f, ff_mul(ff_add(accf, kf), ff_const(B.ffk[FFK_SIXTH])));
                        if (!dry) {
                            B.Ub[((long long)(par_t ^ 1) * B.n_unk + D.gid) * 4 + rank] = ff_to_double(un);
                            xput(Ys + 4 * l + rank, un.h, &xbar[2 + (stage & 1)]);
                        }
                    }
                } else {
                    const double* w = Xw + 4 * l;
                    double kl1 = 0.0, kl2 = 0.0, klr = 0.0;
                    if (rank == 0) {
                        if (TH) {
                            const R irr = (rho0r + Ul[0]) * XP(4) * XP(4);
                            klr = -((w[2] + w[3] - w[0]) * double(irr));
                        } else {
                            klr = -(w[0] + w[2]);
                        }
                        if (cbc) klr += double(TTr[0]);
                    } else if (rank == 3) {
                        klr = TH ? -(w[0] + w[2] + w[3]) : 0.0;
                        if (cbc && TH) klr += double(TTr[3]);
                    } else {
                        const bool sideW = D.kind < 2;
                        const bool need1 = corner || ((rank == 1) == sideW);
                        const bool need2 = corner || ((rank == 1) != sideW);
                        if (need1) {
                            const R bf = TH ? XP(4) * kBr : csr_ * XP(0);
                            kl1 = -(double(bf) * (TH ? w[3] - w[2] : w[2] - w[0]));
                            if (cbc) kl1 += double(TTr[1]);
                        }
                        if (need2) {
                            kl2 = -w[1];
                            if (cbc) kl2 += double(TTr[2]);
                        }
                    }
                    kc = lab_component(rank, D.kind, B.kR, klr, kl1, kl2, klr);
                    if (stage < 3) {
                        const double wk = stage == 0 ? 1.0 : 2.0;
                        const double hk = stage == 2 ? 1.0 : 0.5;
                        acc = (stage == 0 ? 0.0 : acc) + wk * kc;
                        if (!dry) xput(Ys + 4 * l + rank, R(u0r + hk * kc), &xbar[2 + (stage & 1)]);
                    } else {
                        // RK4: U(t + 1) = U(t) + (k1 + 2 k2 + 2 k3 + k4) / 6
                        const double un = u0r + (acc + kc) * (1.0 / 6.0);
                        if (!dry) {
                            B.Ub[((long long)(par_t ^ 1) * B.n_unk + D.gid) * 4 + rank] = un;
                            xput(Ys + 4 * l + rank, R(un), &xbar[2 + (stage & 1)]);
                        }
                    }
                }
            }
            if (xok && !dry) xok = xwait(&xbar[2 + (stage & 1)], (stage >> 1) & 1);
        }

        // 3. Dirichlet populations of unknown l, on CTA l % kCluster
        if (lev == 0 && l % kCluster == rank && (part == 8 || part == 5)) {
            const R Unew[4] = {Ys[4 * l], Ys[4 * l + 1], Ys[4 * l + 2], Ys[4 * l + 3]};
            const bool neep = B.dirichlet >= 1;     // needs x_f: NEEP or regularised NEEP
            const S* fs = nullptr;
            if (neep) {
                if constexpr (MONO) fs = Fx + D.wsrc * L::Q;
                else fs = cg::this_cluster().map_shared_rank(Fx + D.wsrc * L::Q, D.wslot % kCluster);
            }
            dirichlet<LAT, S, R, REF>(G, B, f, neep ? SUt1 + 4 * D.wslot : nullptr, fs, D, Unew, dry);
        }
      }
      if (dry) sync_all();              // the strip phase (and the warm-up) are complete
    }
    if constexpr (!MONO) cg::this_cluster().sync();   // no CTA leaves while its Fx may be read
}

// The tile form by storage.  FP32 / FP16: one 512-thread CTA per tile, at
// most 128 registers a thread (the whole register file of its SM, which
// then holds no bulk CTA: the bulk kernel runs undisturbed on the other
// SMs).  FP64: a cluster of four 128-thread CTAs (launched with the cluster
// attribute), its FP64 wave arithmetic spread over four SMs.
template <typename S>
constexpr bool band_mono() { return sizeof(S) < 8; }

template <int LAT, typename S, bool REF, bool MONO>
__global__ void __launch_bounds__(band_threads<MONO>(), 1)
    k_band(Geom G, Offsets O, Band B, Export E, const S* __restrict__ fin, S* __restrict__ f,
           int par_t)
{
    if constexpr (MONO) {
        for (int t = blockIdx.x; t < B.n_tiles; t += gridDim.x) {
            band_tile<LAT, S, REF, MONO>(G, O, B, E, fin, f, par_t, t);
            __syncthreads();            // the next tile reuses the shared memory
        }
    } else {
        band_tile<LAT, S, REF, MONO>(G, O, B, E, fin, f, par_t, blockIdx.x / kCluster);
    }
}

// Band tiles of many grids in one launch: CTA (cluster) t takes tile
// tile_run[t].y of run tile_run[t].x, whose structures it copies to shared
// memory first; the tile form as in k_band.
template <int LAT, typename S>
__global__ void __launch_bounds__(band_threads<band_mono<S>()>(), 1)
    k_band_batch(const BandRun* __restrict__ runs, const int2* __restrict__ tile_run, int par_t)
{
    constexpr bool MONO = band_mono<S>();
    __shared__ __align__(16) BandRun R;
    const int2 tr = tile_run[MONO ? blockIdx.x : blockIdx.x / kCluster];
    {
        const int* src = reinterpret_cast<const int*>(runs + tr.x);
        int* dst = reinterpret_cast<int*>(&R);
        for (int k = threadIdx.x; k < int(sizeof(BandRun) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    band_tile<LAT, S, false, MONO>(R.G, R.O, R.B, R.E, static_cast<const S*>(R.f[par_t]),
                      static_cast<S*>(R.f[par_t ^ 1]), par_t, tr.y);
}

// Zero gradient (Eq. zg-bc): the post-collision populations of x_f.
template <int LAT, typename S>
__global__ void k_zg(Geom G, Band B, S* __restrict__ f)
{
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= B.n_zg) return;
    const int2 nd = B.zg[z];
#pragma unroll
    for (int i = 0; i < Lat<LAT>::Q; ++i) f[i * G.plane + nd.x] = f[i * G.plane + nd.y];
}

template <int LAT, typename S>
size_t band_smem(const Band& B)
{
    return (size_t)B.max_nodes * 13 * sizeof(typename StripReal<S>::T) +
           (size_t)B.max_fx * Lat<LAT>::Q * sizeof(S);
}

template <int LAT, typename S>
int boundary_t(const Geom& G, const Offsets& O, const Export& E, const Band& B, const void* fin,
               void* fnew, int par_t, cudaStream_t st)
{
    if (B.n_tiles == 0) return 0;
    const size_t smem = band_smem<LAT, S>(B);
    const S* fi = static_cast<const S*>(fin);
    S* fo = static_cast<S*>(fnew);
    constexpr bool mono = band_mono<S>();
    constexpr int ncl = mono ? 1 : kCluster;
    const dim3 grd(mono ? std::max(1, std::min(B.grid, B.n_tiles)) : B.n_tiles * ncl), blk(band_threads<mono>());
    if (G.ref)
        return launch_ex_cl(k_band<LAT, S, true, mono>, grd, blk, smem, st, false, ncl, G, O, B, E, fi, fo, par_t);
    return launch_ex_cl(k_band<LAT, S, false, mono>, grd, blk, smem, st, false, ncl, G, O, B, E, fi, fo, par_t);
}

template <int LAT, typename S>
int band_batch_t(const BandRun* runs, const int2* tile_run, int n_tiles, size_t smem, int par_t,
                 cudaStream_t st, bool early)
{
    if (n_tiles == 0) return 0;
    constexpr bool mono = band_mono<S>();
    return launch_ex_cl(k_band_batch<LAT, S>, dim3(mono ? n_tiles : n_tiles * kCluster),
                        dim3(band_threads<mono>()), smem, st, early, mono ? 1 : kCluster, runs, tile_run, par_t);
}

template <int LAT, typename S>
int prepare_batch_t(size_t smem)
{
    return cudaFuncSetAttribute(k_band_batch<LAT, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(smem)) == cudaSuccess ? 0 : -1;
}

template <int LAT, typename S>
int prepare_t(const Band& B)
{
    // the 48 KB default covers static + dynamic shared memory: always opt in
    const size_t smem = band_smem<LAT, S>(B);
    auto set = [&](const void* k) {
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) == cudaSuccess;
    };
    constexpr bool mono = band_mono<S>();
    const bool ok = set((const void*)k_band<LAT, S, false, mono>) && set((const void*)k_band<LAT, S, true, mono>);
    return ok ? 0 : -1;
}

template <int LAT, typename S>
int zg_t(const Geom& G, const Band& B, void* fnew, cudaStream_t st)
{
    if (B.n_zg == 0) return 0;
    k_zg<LAT, S><<<(B.n_zg + 127) / 128, 128, 0, st>>>(G, B, static_cast<S*>(fnew));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

#define BAND_DISPATCH(lat, storage, CALL)                                  \
    do {                                                                   \
        if (lat == D2Q9) {                                                 \
            if (storage == 0) return CALL(D2Q9, double);                   \
            if (storage == 1) return CALL(D2Q9, float);                    \
            if (storage == 2) return CALL(D2Q9, __half);                   \
        } else if (lat == D2Q17) {                                         \
            if (storage == 0) return CALL(D2Q17, double);                  \
            if (storage == 1) return CALL(D2Q17, float);                   \
            if (storage == 2) return CALL(D2Q17, __half);                  \
        } else {                                                           \
            if (storage == 0) return CALL(D2Q37, double);                  \
            if (storage == 1) return CALL(D2Q37, float);                   \
            if (storage == 2) return CALL(D2Q37, __half);                  \
        }                                                                  \
    } while (0)

int launch_boundary(int lat, int storage, const Geom& G, const Offsets& O, const Export& E,
                    const Band& B, const void* fin, void* fnew, int par_t, cudaStream_t st)
{
#define CALL(L, S) boundary_t<L, S>(G, O, E, B, fin, fnew, par_t, st)
    BAND_DISPATCH(lat, storage, CALL);
#undef CALL
    return -1;
}

size_t band_dynamic_smem(int lat, int storage, const Band& B)
{
#define CALL(L, S) band_smem<L, S>(B)
    BAND_DISPATCH(lat, storage, CALL);
#undef CALL
    return 0;
}

int prepare_boundary(int lat, int storage, const Band& B)
{
#define CALL(L, S) prepare_t<L, S>(B)
    BAND_DISPATCH(lat, storage, CALL);
#undef CALL
    return -1;
}

int launch_band_batch(int lat, int storage, const BandRun* runs, const int2* tile_run, int n_tiles,
                      size_t smem, int par_t, cudaStream_t st, bool early)
{
#define CALL(L, S) band_batch_t<L, S>(runs, tile_run, n_tiles, smem, par_t, st, early)
    BAND_DISPATCH(lat, storage, CALL);
#undef CALL
    return -1;
}

int prepare_band_batch(int lat, int storage, size_t smem)
{
#define CALL(L, S) prepare_batch_t<L, S>(smem)
    BAND_DISPATCH(lat, storage, CALL);
#undef CALL
    return -1;
}

int launch_zg(int lat, int storage, const Geom& G, const Band& B, void* fnew, cudaStream_t st)
{
#define CALL(L, S) zg_t<L, S>(G, B, fnew, st)
    BAND_DISPATCH(lat, storage, CALL);
#undef CALL
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

// Address of the scratch array per CUDA context: a module is loaded once per
// context, so another context on the same device (a driver-API context, or
// the primary context recreated after a reset) holds its own copy.
struct NoallocAddr {
    void* ctx;
    double* addr;
};
std::mutex g_noalloc_mutex;
NoallocAddr g_noalloc_addr[kNoAllocMaxDevices] = {};
int g_noalloc_n = 0;

// The current context (cuCtxGetCurrent, looked up through the runtime), or
// null if the driver does not provide it.
void* current_context()
{
    using Fn = int (*)(void**);
    static Fn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(p);
    }
    void* ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

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
        // the caller's deep strip: 5 moments then the 4 macros per node
        else vis_meso<Lt::THERMAL>(G, static_cast<const double*>(E.stripN) + 5, 9,
                                   static_cast<const double*>(E.stripN), 9, D, Lt::CS2, V);
        for (int m = 0; m < 4; ++m) B.V[4LL * u + m] = V[m];
        B.mask[u] = mask;
    } else {
        for (int m = 0; m < 4; ++m) V[m] = B.V[4LL * u + m];
        mask = B.mask[u];
    }
    double k[4];
    unknown_rhs<LAT, double>(G, B, relax_of<double>(B), X, D, u, V, mask, k);
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

// Device address of the scratch array in the current context, looked up
// once per context (host code cannot use the array's name as a device
// address).
int noalloc_scratch(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);     // makes the device's primary context current if none is
    if (e != cudaSuccess) {
        fprintf(stderr, "lbm_cbc_side_step_noalloc: cudaGetDevice: %s\n", cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    void* ctx = current_context();
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    for (int k = 0; k < g_noalloc_n; ++k)
        if (ctx && g_noalloc_addr[k].ctx == ctx) {
            *out = g_noalloc_addr[k].addr;
            return LBM_OK;
        }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        fprintf(stderr, "lbm_cbc_side_step_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    if (ctx && g_noalloc_n < kNoAllocMaxDevices) g_noalloc_addr[g_noalloc_n++] = NoallocAddr{ctx, static_cast<double*>(p)};
    *out = static_cast<double*>(p);
    return LBM_OK;
}

}  // namespace
}  // namespace lbmgb

extern "C" int lbm_cbc_side_step_noalloc(int lattice, int side, int length, double tau,
                                         const lbm_cbc_params* p, double* Ub, const double* strip_t,
                                         const double* strip_t1, const double* neq_t, void* stream)
{
    using namespace lbmgb;
    if (lattice != LBM_D2Q9 && lattice != LBM_D2Q37 && lattice != LBM_D2Q17) return LBM_ERR_ARG;
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
    const double cs2 = lattice == LBM_D2Q9 ? Lat<D2Q9>::CS2
                     : lattice == LBM_D2Q17 ? Lat<D2Q17>::CS2 : Lat<D2Q37>::CS2;
    const int n = length * M;
    Geom G{};
    G.M = M;
    G.tau = tau;
    G.rho0 = p->rho0;
    G.rho0_f = float(p->rho0);
    G.tau_f = float(tau);
    G.wait_ns = 1000000000ull;
    G.omega = 1.0 / tau;
    G.omega_f = float(G.omega);
    Band B{};
    B.n_unk = n;
    B.M = M;
    B.viscous = p->viscous;
    B.scheme[side] = p->scheme[side];
    B.alpha_T = p->alpha_T;
    B.beta_P = p->beta_P;
    B.t_inf = p->t_inf;
    B.alpha_V = p->alpha_V;
    const double pinf = p->p_inf[side] != 0.0 ? p->p_inf[side] : cs2 * p->rho0;
    B.pdev[side] = pinf - cs2 * p->rho0;
    B.pdev_f[side] = float(B.pdev[side]);
    B.kA = 1.0 / std::sqrt(8.0 * cs2);
    B.kB = std::sqrt(2.0 * cs2);
    B.kC = 1.0 / (2.0 * std::sqrt(2.0));
    B.kR = 1.0 / std::sqrt(2.0);
    B.cs = std::sqrt(cs2);
    B.ihcs = 0.5 / B.cs;
    B.kA_f = float(B.kA);
    B.kB_f = float(B.kB);
    B.kC_f = float(B.kC);
    B.kR_f = float(B.kR);
    B.cs_f = float(B.cs);
    B.ihcs_f = float(B.ihcs);
    set_ffk(B);
    B.Ub = Ub;
    B.Ya = scratch;
    B.Yb = scratch + 4ull * kNoAllocMaxUnknowns;
    B.acc = scratch + 8ull * kNoAllocMaxUnknowns;
    B.V = scratch + 12ull * kNoAllocMaxUnknowns;
    B.mask = reinterpret_cast<int*>(scratch + 16ull * kNoAllocMaxUnknowns);
    Export E{};
    E.nslots = 3 * length;
    E.sesize = 8;
    E.stripU = const_cast<double*>(strip_t);
    E.stripN = const_cast<double*>(neq_t);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nb = (n + kBandThreads - 1) / kBandThreads;
    for (int stage = 0; stage < 4; ++stage) {
        if (lattice == LBM_D2Q9)
            k_side_stage_noalloc<D2Q9><<<nb, kBandThreads, 0, st>>>(G, B, E, side, length, strip_t, strip_t1, stage);
        else if (lattice == LBM_D2Q17)
            k_side_stage_noalloc<D2Q17><<<nb, kBandThreads, 0, st>>>(G, B, E, side, length, strip_t, strip_t1, stage);
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
