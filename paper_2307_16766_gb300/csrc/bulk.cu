// bulk.cu -- bulk kernels of the thermal lattice Boltzmann step.
//
//  k_bulk     fused pull-stream + moments + BGK collide (Eqs. lbe, macro,
//             bgk with the equilibria of Eqs. feq-3/feq-4) on every bulk node.
//  k_init     f = f^eq(U0) on every node and the strips of time 0.
//  k_inflow   the fixed inflow equilibrium on the inflow nodes of a buffer.
//  k_init_band  boundary ODE state of time 0.
//  k_macros   macroscopic fields of the stored populations (Eq. macro).
//
// Populations are stored post-collision and shifted, g = f* - w rho0, in SoA
// planes [Q][ny][nxp].  A bulk node pulls g*_i(x - c_i) for every i.  Away
// from periodic wrap-around the 37 shifted source rows of a 128-node row
// segment are staged through shared memory by tensor copies (TMA), two row
// segments per CTA with FP32 / FP16 storage (one with the reference
// equilibrium and with FP64 storage); stores
// go straight to global memory at fixed plane offsets (Offsets, in the
// kernel parameter bank).  The FP32/FP16 paths do all of their arithmetic in
// FP32; the FP64 path in FP64.
#include "collide.cuh"

#include <utility>

namespace lbmgb {

namespace {

constexpr int kBulkThreads = 128;   // a thread per node of a 128-node row segment

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

// Wait for phase `parity` of a transaction barrier for at most limit_ns (the
// handle's wait limit, 1 s by default; 0: one non-blocking test, as
// try_wait may itself suspend the thread for longer than the copies take);
// on timeout record it in *status and wait once more, for at most 1 s, for
// the copies still in flight, so that none lands in the shared memory of a
// CTA that has left.
__device__ bool wait_tx(unsigned long long* bar, int* status, unsigned long long limit_ns, unsigned parity = 0)
{
    const unsigned a = smem_u32(bar);
    for (int attempt = 0; attempt < 2; ++attempt) {
        const unsigned long long t0 = global_ns(), lim = attempt == 0 ? limit_ns : 1000000000ull;
        for (;;) {
            unsigned ok;
            if (lim == 0)
                asm volatile(
                    "{\n .reg .pred p;\n"
                    " mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                    " selp.u32 %0, 1, 0, p;\n}"
                    : "=r"(ok)
                    : "r"(a), "r"(parity)
                    : "memory");
            else
                asm volatile(
                    "{\n .reg .pred p;\n"
                    " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                    " selp.u32 %0, 1, 0, p;\n}"
                    : "=r"(ok)
                    : "r"(a), "r"(parity)
                    : "memory");
            if (ok) return attempt == 0;
            if (global_ns() - t0 > lim) break;
        }
        if (attempt == 0) atomicOr(status, 2);
    }
    return false;
}


// One 3D tensor copy per c_y group; every offset, coordinate shift and map
// choice is a template constant so nothing is looked up at run time.
template <int LAT, typename S, int GI>
__device__ __forceinline__ void issue_group(const Maps& tm, unsigned char* smem, int x0, int y,
                                            unsigned bar)
{
    using L = Lat<LAT>;
    using BX = Stage<LAT, S>;
    constexpr int cnt = L::gcount(GI);
    static_assert(cnt == 7 || cnt == 5 || cnt == 3 || cnt == 2 || cnt == 1,
                  "group depth without a tensor map");
    constexpr int ofs = BX::gofs(GI);
    constexpr int dy = L::gcy(GI);
    constexpr int z0 = L::gstart(GI);
    const CUtensorMap* m = cnt == 7 ? &tm.m7 : cnt == 5 ? &tm.m5 : cnt == 3 ? &tm.m3
                         : cnt == 2 ? &tm.m2 : &tm.m1;
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

// Pull-stream result g of node (x, y) -> moments, BGK collision (Eq. bgk)
// and post-collision store.
template <int LAT, typename S, typename C, bool REF>
__device__ __forceinline__ void collide_store(const Geom& G, const Offsets& O, S* __restrict__ fout,
                                              int x, int y, C* g)
{
    S* out = fout + (y * G.nxp + x);
    if constexpr (Store<S>::SCALED) {
        collide_scaled<LAT, REF>(G, g, [&](int i, C v) { Store<S>::put(out + O.st[i], v); });
    } else {
        collide<LAT, C, REF>(G, g, [&](int i, C v) { Store<S>::put(out + O.st[i], v); });
    }
}

// Row segments per CTA of k_bulk: the tensor copies of every row are issued
// at once (one transaction barrier each), so the copies of later rows land
// while earlier rows are computed.  Plain FP32 and FP16: two rows, a CTA
// keeping 40 KB (FP32) in flight with the registers of one row (measured
// beside the one-CTA band tiles: FP32 1024x512 step 31.9-32.3 us against
// 33.0 with one row; FP16 4096^2 36.5k against 32.1k MLUPS).  With the
// reference equilibrium (89 registers) one row measured faster (1024x512:
// 12.1k -> 13.2k MLUPS); FP64 storage (ALU-bound on GB300, twice the
// staging) keeps one row.
template <typename S, bool REF>
constexpr int bulk_rows() { return (sizeof(S) <= 4 && !REF) ? 2 : 1; }

template <int LAT, typename S, bool REF>
__device__ __forceinline__ void bulk_body(const Maps& tm, const Geom& G, const Offsets& O, const Region& R,
                                          const S* __restrict__ fin, S* __restrict__ fout, int* status)
{
    constexpr int ROWS = bulk_rows<S, REF>();
    using L = Lat<LAT>;
    using C = typename Store<S>::C;
    using BX = Stage<LAT, S>;
    constexpr int Q = L::Q;
    extern __shared__ __align__(128) unsigned char smem_raw[];   // ROWS x BX::TOTAL
    __shared__ __align__(8) unsigned long long bar[ROWS];
    const int x0 = (R.x0 / kBulkThreads + blockIdx.x) * kBulkThreads;   // tiles aligned to 128
    const int x = x0 + threadIdx.x;
    const int yb = R.y0 + blockIdx.y * ROWS;
    const bool valid = x >= R.x0 && x < R.x1;

    // Pull stream (Eq. lbe): g_i(x) = g*_i(x - c_i).  Rows whose sources
    // wrap around a periodic axis use plain loads; all others stage the 37
    // shifted source rows through shared memory with tensor copies.
    const bool xwrap = G.perx && (x0 - L::M < 0 || x0 + kBulkThreads + L::M > G.nx);
    auto staged = [&](int y) {
        return y < R.y1 && !xwrap && !(G.pery && (y < L::M || y >= G.ny - L::M));
    };
    if (threadIdx.x == 0) {
#pragma unroll
        for (int r = 0; r < ROWS; ++r)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[r])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            if (!staged(yb + r)) continue;
            const unsigned b = smem_u32(&bar[r]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         ::"r"(b), "r"(BX::TX) : "memory");
            issue_copies<LAT, S>(tm, smem_raw + r * BX::TOTAL, x0, yb + r, b,
                                 std::make_integer_sequence<int, L::NG>{});
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int r = 0; r < ROWS; ++r) {
        const int y = yb + r;
        if (y >= R.y1) break;
        C g[Q];
        if (staged(y)) {
            if (!wait_tx(&bar[r], status, G.wait_ns)) {
                // timed out (status set): let the later rows' copies land
                // (bounded) before the CTA's shared memory goes away
                for (int q = r + 1; q < ROWS; ++q)
                    if (staged(yb + q)) wait_tx(&bar[q], status, G.wait_ns);
                return;
            }
            if (!valid) continue;
            gather_staged<LAT, S, C>(g, reinterpret_cast<const S*>(smem_raw + r * BX::TOTAL), threadIdx.x,
                                     std::make_integer_sequence<int, Q>{});
        } else {
            if (!valid) continue;
            pull_plain<LAT, S, C>(G, O, fin, x, y, g);
        }
        collide_store<LAT, S, C, REF>(G, O, fout, x, y, g);
    }
}

template <int LAT, typename S>
__global__ void __launch_bounds__(kBulkThreads)
    k_bulk(const __grid_constant__ Maps tm, Geom G, Offsets O, Region R, const S* __restrict__ fin,
           S* __restrict__ fout, int* status)
{
    bulk_body<LAT, S, false>(tm, G, O, R, fin, fout, status);
}

// With a reference equilibrium: about twice the equilibrium arithmetic per
// node (89 registers with FP32 storage; capping them at the plain form's 72
// spilled and measured slower).
template <int LAT, typename S>
__global__ void __launch_bounds__(kBulkThreads)
    k_bulk_ref(const __grid_constant__ Maps tm, Geom G, Offsets O, Region R, const S* __restrict__ fin,
               S* __restrict__ fout, int* status)
{
    bulk_body<LAT, S, true>(tm, G, O, R, fin, fout, status);
}

// Persistent form of k_bulk for one or many grids of one lattice and
// storage: `grid` CTAs take the work items (run, row, 128-node segment) of
// the runs from a queue, and each CTA keeps the tensor copies of its next
// item in flight while it computes the current one (two staging buffers,
// one transaction barrier each).  The arithmetic per node is that of k_bulk.
template <int LAT, typename S>
__global__ void __launch_bounds__(kBulkThreads)
    k_bulk_persistent(const BulkRun* __restrict__ runs, int n_runs, int total, int par, unsigned* queue)
{
    using L = Lat<LAT>;
    using C = typename Store<S>::C;
    using BX = Stage<LAT, S>;
    extern __shared__ __align__(128) unsigned char smem_raw[];   // 2 x BX::TOTAL
    __shared__ __align__(8) unsigned long long bar[2];
    __shared__ int s_first[kMaxBatchRuns + 1];
    // the next group's kernel of a batched step (other grids) may begin now
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    for (int k = threadIdx.x; k <= n_runs; k += blockDim.x) s_first[k] = k < n_runs ? runs[k].first : total;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    // work item w -> run, segment origin x0, row y; staged unless its
    // sources wrap around a periodic axis
    struct Item {
        int run, x0, y;
        bool staged;
    };
    auto locate = [&](int w) {
        int lo = 0, hi = n_runs - 1;
        while (lo < hi) {                   // last run whose first item is <= w
            const int mid = (lo + hi + 1) >> 1;
            if (s_first[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        const BulkRun& R = runs[lo];
        const int local = w - s_first[lo];
        Item it;
        it.run = lo;
        it.x0 = (R.seg0 + local % R.nseg) * kBulkThreads;
        it.y = R.R.y0 + local / R.nseg;
        it.staged = !((R.G.pery && (it.y < L::M || it.y >= R.G.ny - L::M)) ||
                      (R.G.perx && (it.x0 - L::M < 0 || it.x0 + kBulkThreads + L::M > R.G.nx)));
        return it;
    };
    auto issue = [&](const Item& it, int stage) {
        if (threadIdx.x != 0 || !it.staged) return;
        const unsigned b = smem_u32(&bar[stage]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(BX::TX)
                     : "memory");
        issue_copies<LAT, S>(runs[it.run].maps[par], smem_raw + stage * BX::TOTAL, it.x0, it.y, b,
                             std::make_integer_sequence<int, L::NG>{});
    };

    // Work items are taken from a queue (queue[0]: next item) as CTAs free
    // up, so that CTAs on SMs that hold other kernels' CTAs (the band
    // kernel beside this one) take fewer items.  The last CTA to finish
    // (queue[1] counts them) resets the queue for the next launch.
    __shared__ int s_w[2];
    auto grab = [&]() { return int(atomicAdd(&queue[0], 1u)); };
    unsigned phase0 = 0u, phase1 = 0u;      // next phase of each stage's barrier
    int stage = 0;
    if (threadIdx.x == 0) s_w[0] = grab();
    __syncthreads();
    int w = s_w[0];
    Item cur{0, 0, 0, false};
    if (w < total) {
        cur = locate(w);
        issue(cur, 0);
    }
    while (w < total) {
        if (threadIdx.x == 0) s_w[stage ^ 1] = grab();
        __syncthreads();
        const int wn = s_w[stage ^ 1];
        Item nxt{0, 0, 0, false};
        if (wn < total) {                   // the buffer of stage ^ 1 was released last iteration
            nxt = locate(wn);
            issue(nxt, stage ^ 1);
        }
        const BulkRun& R = runs[cur.run];
        const int x = cur.x0 + threadIdx.x;
        const bool valid = x >= R.R.x0 && x < R.R.x1;
        bool ok = true;
        C g[L::Q];
        if (cur.staged) {
            ok = wait_tx(&bar[stage], R.status, R.G.wait_ns, stage ? phase1 : phase0);
            if (stage) phase1 ^= 1u;
            else phase0 ^= 1u;
            ok = __syncthreads_and(ok);     // one decision for the whole CTA
            if (ok && valid)
                gather_staged<LAT, S, C>(g, reinterpret_cast<const S*>(smem_raw + stage * BX::TOTAL),
                                         threadIdx.x, std::make_integer_sequence<int, L::Q>{});
        } else if (valid) {
            pull_plain_planes<LAT, S, C>(R.G, static_cast<const S*>(R.f[par]), x, cur.y, g);
        }
        if (!ok) {
            // a copy never completed: wait (bounded) for the one in flight
            // for the next item, then leave
            if (wn < total && nxt.staged) wait_tx(&bar[stage ^ 1], R.status, R.G.wait_ns, stage ? phase0 : phase1);
            break;
        }
        if (valid) {
            S* out = static_cast<S*>(R.f[par ^ 1]) + (cur.y * R.G.nxp + x);
            const int plane = int(R.G.plane);
            auto put = [&](int i, C v) { Store<S>::put(out + L::plane_of(i) * plane, v); };
            // runs of a batch hold the plain shift (lbm_batch_create)
            if constexpr (Store<S>::SCALED) collide_scaled<LAT, false>(R.G, g, put);
            else collide<LAT, C, false>(R.G, g, put);
        }
        __syncthreads();                    // stage buffer read by all before its reuse
        w = wn;
        cur = nxt;
        stage ^= 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&queue[1], 1u) == gridDim.x - 1) {   // every CTA has taken its last item
            queue[0] = 0u;
            queue[1] = 0u;
            __threadfence();
        }
    }
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
    // the equilibrium in the storage's arithmetic (as the bulk update
    // evaluates it), from the deviations formed in FP64
    using C = typename Store<S>::C;
    Moments<LAT, C> mc;
    mc.s0 = C(m.s0);
    mc.rho = C(m.rho);
    mc.ux = C(m.ux);
    mc.uy = C(m.uy);
    mc.dT = C(m.dT);
    if (G.ref) {                        // the deviation from the reference, in FP64
        mc.ref = 1;
        mc.Ux = uref_of<C>(G, 0);
        mc.Uy = uref_of<C>(G, 1);
        mc.vx = C(m.ux - stored_ref<S>(G, 0));
        mc.vy = C(m.uy - stored_ref<S>(G, 1));
    }
    C geq[L::Q];
    equilibrium<LAT, C>(mc, geq);
    S* out = f + (long long)y * G.nxp + x;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        C v = geq[i];
        if (Store<S>::SCALED) v *= C(1.0 / L::w(i));
        Store<S>::put(out + (long long)L::plane_of(i) * G.plane, v);
    }
    // strips of time 0 (parity 0): U0 and zero non-equilibrium moments
    const int dd[4] = {x - G.M, G.nx - 1 - G.M - x, y - G.M, G.ny - 1 - G.M - y};
    const bool inbx = (G.perx || (x >= G.M && x < G.nx - G.M));
    const bool inby = (G.pery || (y >= G.M && y < G.ny - G.M));
    if (!(inbx && inby)) return;
    using R = typename StripReal<S>::T;
    const R U[4] = {R(m.s0), R(m.ux), R(m.uy), R(m.dT)};
    for (int s = 0; s < 4; ++s) {
        if (!E.cbc[s] || dd[s] < 0 || dd[s] >= E.ND) continue;
        const int p = s < 2 ? y : x;
        const long long slot = E.offS[s] + dd[s] * E.L[s] + p;
        R* u = static_cast<R*>(E.stripU) + slot * 4;
        R* nn = static_cast<R*>(E.stripN) + slot * 5;
        for (int c = 0; c < 4; ++c) u[c] = U[c];
        for (int c = 0; c < 5; ++c) nn[c] = R(0);
    }
}

template <int LAT, typename S>
__global__ void k_inflow(Geom G, const int* __restrict__ nodes, int n, double d0, double d1,
                         double d2, double d3, S* __restrict__ f)
{
    using L = Lat<LAT>;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const Moments<LAT, double> m =
        moments_of_macros<LAT, double>(d0, d1, d2, d3, G.rho0, G.ref, stored_ref<S>(G, 0), stored_ref<S>(G, 1));
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
    const Moments<LAT, double> m = moments<LAT, double>(g, G.rho0, G.ref, stored_ref<S>(G, 0), stored_ref<S>(G, 1));
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
int bulk_t(const Geom& G, const Offsets& O, const Region& R, const CUtensorMap* tmaps,
           const void* fin, void* fout, int* status, cudaStream_t st, bool early)
{
    const int h = R.y1 - R.y0;
    if (R.x1 <= R.x0 || h <= 0) return 0;
    const int t0 = R.x0 / kBulkThreads, t1 = (R.x1 + kBulkThreads - 1) / kBulkThreads;
    Maps tm;
    tm.m7 = tmaps[0];
    tm.m5 = tmaps[1];
    tm.m3 = tmaps[2];
    tm.m2 = tmaps[3];
    tm.m1 = tmaps[4];
    const dim3 blk(kBulkThreads);
    if (G.ref) {
        constexpr int ROWS = bulk_rows<S, true>();
        constexpr size_t smem = ROWS * Stage<LAT, S>::TOTAL;
        static_assert(smem <= 48 * 1024, "bulk staging above the default dynamic shared memory");
        return launch_ex(k_bulk_ref<LAT, S>, dim3(t1 - t0, (h + ROWS - 1) / ROWS), blk, smem, st, early, tm, G, O,
                         R, static_cast<const S*>(fin), static_cast<S*>(fout), status);
    }
    constexpr int ROWS = bulk_rows<S, false>();
    constexpr size_t smem = ROWS * Stage<LAT, S>::TOTAL;
    static_assert(smem <= 48 * 1024, "bulk staging above the default dynamic shared memory");
    return launch_ex(k_bulk<LAT, S>, dim3(t1 - t0, (h + ROWS - 1) / ROWS), blk, smem, st, early, tm, G, O, R,
                     static_cast<const S*>(fin), static_cast<S*>(fout), status);
}

template <int LAT, typename S>
int bulk_persistent_t(const BulkRun* runs, int n_runs, int total, int par, int grid, unsigned* queue,
                      cudaStream_t st, bool early)
{
    if (total <= 0) return 0;
    if (n_runs > kMaxBatchRuns) return -1;
    return launch_ex(k_bulk_persistent<LAT, S>, dim3(grid), dim3(kBulkThreads), 2 * Stage<LAT, S>::TOTAL, st,
                     early, runs, n_runs, total, par, queue);
}

template <int LAT, typename S>
int prepare_persistent_t()
{
    return cudaFuncSetAttribute(k_bulk_persistent<LAT, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                2 * Stage<LAT, S>::TOTAL) == cudaSuccess ? 0 : -1;
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
        } else if (lat == D2Q17) {                                         \
            if (storage == 0) return CALL(D2Q17, double);                  \
            if (storage == 1) return CALL(D2Q17, float);                   \
            if (storage == 2) return CALL(D2Q17, __half);                  \
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

int launch_bulk(int lat, int storage, const Geom& G, const Offsets& O, const Region& R,
                const CUtensorMap* tmaps, const void* fin, void* fout, int* status,
                cudaStream_t st, bool early)
{
#define CALL(L, S) bulk_t<L, S>(G, O, R, tmaps, fin, fout, status, st, early)
    LBM_DISPATCH(lat, storage, CALL);
#undef CALL
}


int launch_bulk_persistent(int lat, int storage, const BulkRun* runs, int n_runs, int total, int par,
                           int grid, unsigned* queue, cudaStream_t st, bool early)
{
#define CALL(L, S) bulk_persistent_t<L, S>(runs, n_runs, total, par, grid, queue, st, early)
    LBM_DISPATCH(lat, storage, CALL);
#undef CALL
}

int prepare_bulk_persistent(int lat, int storage)
{
#define CALL(L, S) prepare_persistent_t<L, S>()
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
