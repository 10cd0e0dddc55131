// api.cu -- host runtime behind the C ABI of include/lbm_cbc.h.
//
// A handle owns (or borrows, with lbm_create_in) one device workspace carved
// into: the two population buffers (ping-pong by step parity), the
// near-boundary strips exported by the bulk kernel, the boundary ODE state
// and RK4 stage buffers, a macro buffer and a status flag.  Every launch goes
// to the handle's stream.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include <sys/stat.h>

#include <cudaTypedefs.h>

#include "lbm_cbc.h"
#include "lbm_internal.cuh"

using namespace lbmgb;

struct lbm_handle {
    int lattice = 0, nx = 0, ny = 0, M = 0, Q = 0, storage = 0;
    double tau = 0;
    lbm_cbc_params P{};
    Geom G{};
    Offsets O{};
    Export E{};
    Band B{};
    size_t esize = 0, f_bytes = 0;
    void* f[2] = {nullptr, nullptr};
    int* inflow_nodes = nullptr;
    int n_inflow = 0;
    bool inflow_done[2] = {false, false};   // buffer already holds the inflow equilibrium
    double Uin[4] = {0, 0, 0, 0};
    double* macro = nullptr;
    int* flag = nullptr;     // [0]: non-finite macros seen, [1]: kernel status bits
    CUtensorMap tmap[2][5];  // tensor-copy descriptors of the two buffers, box depths 7, 5, 3, 2, 1
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool owns_ws = false;
    cudaStream_t stream = nullptr;
    Region bulk{};           // nodes of the bulk kernel
    BulkRun* brun = nullptr; // its run descriptor (workspace)
    int bulk_items = 0;      // its work items (row segments)
    cudaStream_t aux = nullptr;              // internal stream: the bulk beside the band, when timed
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t kev[5] = {};  // caller's timing events (see lbm_set_kernel_events)
    long long steps = 0;
    bool initialized = false;
    bool bulk_pending = false;   // phase 0 issued, phase 1 not yet
    // tangent-linear steps (lbm_grad_*): their state, and whether they
    // advanced the populations past the strips and boundary state of the
    // ordinary step (which then needs lbm_init_fields or lbm_set_state)
    TLState tl{};
    void* tl_mem = nullptr;
    bool grad_stale = false;
    // reverse-mode gradients (lbm_adj_*): history and adjoint buffers, and the
    // checkpoints of the forward pass (every adj_K steps, then the end state)
    void* adj_mem = nullptr;
    AdjState adj{};
    int adj_max = 0, adj_n = 0;
    long long adj_start = 0;
    const double* adj_ref = nullptr;
    long long adj_ref_stride = 0;
    char* adj_ckpt = nullptr;
    size_t adj_ckpt_bytes = 0;
    size_t adj_hist_bytes = 0;          // one of the two history buffers (by segment parity)
    bool adj_fwd_done = false;
    cudaStream_t adj_sv = nullptr, adj_sw = nullptr;   // reverse steps: boundary, bulk
    cudaEvent_t adj_ev[4] = {};         // step done, bulk done, segment recomputed, segment reversed
    std::string err;
};

namespace {
const char* const kGradStale =
    "gradient steps advanced this handle past its boundary strips: call lbm_init_fields or "
    "lbm_set_state before stepping it again";
}  // namespace

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Plan {
    Geom G{};
    Offsets O{};
    Export E{};
    Band B{};
    int Q = 0;
    size_t esize = 0, f_bytes = 0, stripU_n = 0, stripN_n = 0;
    Region bulk{};
    std::vector<StripNode> sn;   // strip nodes of the tiles
    std::vector<int> sbeg;
    std::vector<UDesc> ldp;      // ld and sn at a fixed stride per tile (device copies)
    std::vector<StripNode> snp;
    std::vector<UDesc> ud;
    std::vector<UDesc> ld;       // tile tables of the fused band kernel
    std::vector<int> tbeg;
    std::vector<int2> zg;
    std::vector<int> inflow;
    double Uin[4] = {0, 0, 0, 0};
    size_t off_f0 = 0, off_f1 = 0, off_sU = 0, off_sN = 0, off_Ub = 0, off_ud = 0, off_ld = 0,
           off_sn = 0, off_brun = 0, off_zg = 0, off_in = 0, off_macro = 0, off_flag = 0,
           total = 0;
};

std::string fmt(const char* f, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, f);
    vsnprintf(buf, sizeof buf, f, ap);
    va_end(ap);
    return buf;
}

double lattice_cs2(int lattice)
{
    return lattice == LBM_D2Q9 ? Lat<D2Q9>::CS2 : lattice == LBM_D2Q17 ? Lat<D2Q17>::CS2 : Lat<D2Q37>::CS2;
}

int lattice_cx(int lattice, int i)
{
    return lattice == LBM_D2Q9 ? Lat<D2Q9>::cx(i) : lattice == LBM_D2Q17 ? Lat<D2Q17>::cx(i) : Lat<D2Q37>::cx(i);
}
int lattice_cy(int lattice, int i)
{
    return lattice == LBM_D2Q9 ? Lat<D2Q9>::cy(i) : lattice == LBM_D2Q17 ? Lat<D2Q17>::cy(i) : Lat<D2Q37>::cy(i);
}
int lattice_plane(int lattice, int i)
{
    return lattice == LBM_D2Q9 ? Lat<D2Q9>::plane_of(i)
         : lattice == LBM_D2Q17 ? Lat<D2Q17>::plane_of(i) : Lat<D2Q37>::plane_of(i);
}

// Side geometry (W = 0, E = 1, S = 2, N = 3): outward normal and the layer-0
// node x_f at tangential position p (Fig. Layer-Multispeed-BC).
const int kSN[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};

void side_xf(int s, int p, int nx, int ny, int M, int& x, int& y)
{
    if (s == 0) { x = M; y = p; }
    else if (s == 1) { x = nx - 1 - M; y = p; }
    else if (s == 2) { x = p; y = M; }
    else { x = p; y = ny - 1 - M; }
}

// Validate a configuration, lay out the workspace and resolve the boundary
// descriptors.
int make_plan(int lattice, int nx, int ny, double tau, const lbm_cbc_params* p, Plan& pl,
              std::string& err)
{
    if (!p) { err = "params is NULL"; return LBM_ERR_ARG; }
    if (lattice != LBM_D2Q9 && lattice != LBM_D2Q37 && lattice != LBM_D2Q17) {
        err = fmt("unknown lattice %d", lattice);
        return LBM_ERR_ARG;
    }
    if (!(tau > 0.5) || !std::isfinite(tau)) { err = fmt("tau must exceed 1/2 (got %g)", tau); return LBM_ERR_ARG; }
    if (p->storage < LBM_F64 || p->storage > LBM_F16) { err = fmt("unknown storage %d", p->storage); return LBM_ERR_ARG; }
    if (!(p->rho0 > 0.0)) { err = "rho0 must be positive"; return LBM_ERR_ARG; }
    if (p->viscous < 0 || p->viscous > 2) { err = "unknown viscous mode"; return LBM_ERR_ARG; }
    if (p->dirichlet < 0 || p->dirichlet > 2) { err = "unknown Dirichlet mode"; return LBM_ERR_ARG; }
    if (!std::isfinite(p->alpha_T) || !std::isfinite(p->beta_P) || !std::isfinite(p->t_inf) ||
        !std::isfinite(p->alpha_V)) {
        err = "relaxation parameters must be finite";
        return LBM_ERR_ARG;
    }
    if (p->band_ctas < 0) { err = "band_ctas must be >= 0"; return LBM_ERR_ARG; }
    {
        const double ur2 = p->u_ref[0] * p->u_ref[0] + p->u_ref[1] * p->u_ref[1];
        if (!std::isfinite(ur2) || !(ur2 < lattice_cs2(lattice))) {
            err = "u_ref must be finite and slower than c_s";
            return LBM_ERR_ARG;
        }
    }
    for (int s = 0; s < 4; ++s) {
        if (p->side[s] < 0 || p->side[s] > 3) { err = fmt("unknown kind %d of side %d", p->side[s], s); return LBM_ERR_ARG; }
        if (p->scheme[s] < 0 || p->scheme[s] > 3) { err = fmt("unknown scheme of side %d", s); return LBM_ERR_ARG; }
    }
    const int perx = p->side[0] == LBM_SIDE_PERIODIC, pery = p->side[2] == LBM_SIDE_PERIODIC;
    if (perx != (p->side[1] == LBM_SIDE_PERIODIC) || pery != (p->side[3] == LBM_SIDE_PERIODIC)) {
        err = "a periodic side needs a periodic opposite side";
        return LBM_ERR_ARG;
    }
    const int M = lattice == LBM_D2Q9 ? 1 : 3;
    const int Q = lattice == LBM_D2Q9 ? 9 : lattice == LBM_D2Q17 ? 17 : 37;
    const int nmin_b = 2 * M + 3;
    if (nx < 1 || ny < 1 || nx > (1 << 20) || ny > 65535) { err = fmt("grid %d x %d out of range", nx, ny); return LBM_ERR_ARG; }
    if ((!perx && nx < nmin_b) || (!pery && ny < nmin_b)) {
        err = fmt("non-periodic axes need at least %d nodes", nmin_b);
        return LBM_ERR_ARG;
    }
    if ((perx && nx < M) || (pery && ny < M)) { err = fmt("periodic axes need at least %d nodes", M); return LBM_ERR_ARG; }
    if (!perx && !pery) {
        int ncbc = 0;
        for (int s = 0; s < 4; ++s) ncbc += p->side[s] == LBM_SIDE_CBC;
        if (ncbc != 0 && ncbc != 4) { err = "with four open sides, either all or none must be CBC"; return LBM_ERR_ARG; }
    }
    if (p->viscous == LBM_VISCOUS_MESO) {
        // the mesoscopic stencil's deepest node, x_f - (M + 2) n, must be a
        // bulk node: 3 M + 3 nodes on an axis with a characteristic side
        const int nmin_v = 3 * M + 3;
        if (((p->side[0] == LBM_SIDE_CBC || p->side[1] == LBM_SIDE_CBC) && nx < nmin_v) ||
            ((p->side[2] == LBM_SIDE_CBC || p->side[3] == LBM_SIDE_CBC) && ny < nmin_v)) {
            err = fmt("the mesoscopic viscous terms need at least %d nodes across a characteristic side",
                      nmin_v);
            return LBM_ERR_ARG;
        }
    }
    const int nxp = (nx + 63) / 64 * 64;
    if ((double)Q * ny * nxp >= 2147483647.0) { err = "grid too large (more than 2^31 population values)"; return LBM_ERR_ARG; }

    Geom& G = pl.G;
    G.nx = nx;
    G.ny = ny;
    G.M = M;
    G.nxp = nxp;
    G.perx = perx;
    G.pery = pery;
    G.bx0 = perx ? 0 : M;
    G.bx1 = perx ? nx : nx - M;
    G.by0 = pery ? 0 : M;
    G.by1 = pery ? ny : ny - M;
    G.plane = (long long)ny * G.nxp;

    // The bulk kernel updates every bulk node; the band kernel of the same
    // step writes only boundary nodes, reads only the old buffer, so the two
    // run concurrently.
    pl.bulk = Region{G.bx0, G.bx1, G.by0, G.by1};
    G.tau = tau;
    G.rho0 = p->rho0;
    G.omega = 1.0 / tau;
    G.omega_f = float(1.0 / tau);
    G.rho0_f = float(p->rho0);
    G.tau_f = float(tau);
    G.wait_ns = 1000000000ull;
    G.ref = p->u_ref[0] != 0.0 || p->u_ref[1] != 0.0;
    for (int k = 0; k < 2; ++k) {
        G.uref[k] = p->u_ref[k];
        G.uref_f[k] = float(p->u_ref[k]);
    }
    for (int i = 0; i < Q; ++i) {
        const int plane_i = lattice_plane(lattice, i);
        pl.O.st[i] = int(plane_i * G.plane);
        pl.O.ld[i] = int(plane_i * G.plane) - lattice_cy(lattice, i) * nxp - lattice_cx(lattice, i);
    }

    // strips: slots (side, depth, position) of the characteristic sides
    Export& E = pl.E;
    const bool meso = p->viscous == LBM_VISCOUS_MESO;
    // depths 0..2 for the stencils; M..M+2 for the mesoscopic viscous terms
    E.ND = 3 + (meso ? M : 0);
    int L[4], lo[4], hi[4], tper[4];
    for (int s = 0; s < 4; ++s) {
        L[s] = s < 2 ? ny : nx;
        tper[s] = s < 2 ? pery : perx;
        lo[s] = tper[s] ? 0 : M;
        hi[s] = tper[s] ? L[s] - 1 : L[s] - 1 - M;
        E.cbc[s] = p->side[s] == LBM_SIDE_CBC;
        E.L[s] = L[s];
        E.offS[s] = E.nslots;
        if (E.cbc[s]) E.nslots += E.ND * L[s];
    }
    auto slot = [&](int s, int d, int pp) {
        if (tper[s]) pp = ((pp % L[s]) + L[s]) % L[s];
        return E.offS[s] + d * L[s] + pp;
    };
    auto goff = [&](int x, int y) { return y * nxp + x; };

    Band& B = pl.B;
    B.M = M;
    const double cs2 = lattice_cs2(lattice);
    int corner_kind = -1;
    if (!perx && !pery) {
        if (p->side[0] == LBM_SIDE_CBC) corner_kind = SIDE_CBC;
        else if (p->side[0] == LBM_SIDE_INFLOW || p->side[1] == LBM_SIDE_INFLOW ||
                 p->side[2] == LBM_SIDE_INFLOW || p->side[3] == LBM_SIDE_INFLOW)
            corner_kind = SIDE_INFLOW;
        else corner_kind = SIDE_ZG;
    }
    // unknown index of side s, layer j, position pp (pp already in range):
    // layer-major, so that the threads of a warp share j (one stencil
    // branch, neighbours of one kind) and the RK4 stages do not diverge
    int base[4] = {0, 0, 0, 0}, npos[4] = {0, 0, 0, 0}, n_side = 0;
    for (int s = 0; s < 4; ++s)
        if (E.cbc[s]) {
            base[s] = n_side;
            npos[s] = hi[s] - lo[s] + 1;
            n_side += npos[s] * M;
        }
    const int lo_corner[4] = {0, 1, 0, 2}, hi_corner[4] = {2, 3, 1, 3};
    auto ref = [&](int s, int j, int pp) -> int {
        if (tper[s]) pp = ((pp % L[s]) + L[s]) % L[s];
        if (j <= 0) return -(slot(s, -j, pp) + 1);
        if (pp < lo[s]) return n_side + lo_corner[s];
        if (pp > hi[s]) return n_side + hi_corner[s];
        return base[s] + (j - 1) * npos[s] + (pp - lo[s]);
    };
    for (int s = 0; s < 4; ++s) {
        if (!E.cbc[s]) continue;
        for (int j = 1; j <= M; ++j)
            for (int pp = lo[s]; pp <= hi[s]; ++pp) {
                UDesc D;
                std::memset(&D, 0, sizeof D);
                D.kind = s;
                D.j = j;
                D.nb[0] = j < M ? ref(s, j + 1, pp) : 0;
                D.nb[1] = ref(s, j - 1, pp);
                D.nb[2] = ref(s, j - 2, pp);
                D.nb[3] = j - 3 >= -2 ? ref(s, j - 3, pp) : 0;
                D.nb[4] = ref(s, j, pp + 1);
                D.nb[5] = ref(s, j, pp - 1);
                D.tmode = tper[s] ? 0 : (pp == hi[s] ? 1 : (pp == lo[s] ? -1 : 0));
                if (meso) {
                    // Sec. 3.3, "Evaluation of viscous terms": the one-sided
                    // stencil starts M nodes below x_f, at the first node none
                    // of whose populations came from a boundary layer
                    D.vs[0] = slot(s, M, pp);
                    D.vs[1] = slot(s, M + 1, pp);
                    D.vs[2] = slot(s, M + 2, pp);
                    if (D.tmode == 0) { D.vs[3] = slot(s, M, pp + 1); D.vs[4] = slot(s, M, pp - 1); }
                    else if (D.tmode == 1) { D.vs[3] = slot(s, M, pp - 1); D.vs[4] = slot(s, M, pp - 2); }
                    else { D.vs[3] = slot(s, M, pp + 1); D.vs[4] = slot(s, M, pp + 2); }
                }
                int x, y;
                side_xf(s, pp, nx, ny, M, x, y);
                D.wsrc = goff(x, y);
                D.wslot = slot(s, 0, pp);
                D.wnode = goff(x + j * kSN[s][0], y + j * kSN[s][1]);
                pl.ud.push_back(D);
            }
    }
    if (corner_kind == SIDE_CBC)
        for (int c = 0; c < 4; ++c) {
            UDesc D;
            std::memset(&D, 0, sizeof D);
            const int sx = (c & 1) ? 1 : -1, sy = (c & 2) ? 1 : -1;
            const int sW = sx < 0 ? 0 : 1;
            const int xc = sx < 0 ? M - 1 : nx - M, yc = sy < 0 ? M - 1 : ny - M;
            D.kind = 4 + c;
            D.nb[0] = -(slot(sW, 0, yc - sy) + 1);
            D.nb[1] = -(slot(sW, 1, yc - 2 * sy) + 1);
            D.wsrc = goff(xc - sx, yc - sy);
            D.wslot = slot(sW, 0, yc - sy);
            D.wnode = goff(sx < 0 ? 0 : nx - 1, sy < 0 ? 0 : ny - 1);
            D.wdx = sx < 0 ? 1 : -1;
            D.wdy = (sy < 0 ? 1 : -1) * nxp;
            pl.ud.push_back(D);
        }
    // zero-gradient and inflow nodes
    for (int s = 0; s < 4; ++s) {
        if (p->side[s] != LBM_SIDE_ZG && p->side[s] != LBM_SIDE_INFLOW) continue;
        for (int pp = lo[s]; pp <= hi[s]; ++pp)
            for (int j = 1; j <= M; ++j) {
                int x, y;
                side_xf(s, pp, nx, ny, M, x, y);
                const int node = goff(x + j * kSN[s][0], y + j * kSN[s][1]);
                if (p->side[s] == LBM_SIDE_ZG) pl.zg.push_back(make_int2(node, goff(x, y)));
                else pl.inflow.push_back(node);
            }
    }
    if (corner_kind == SIDE_ZG || corner_kind == SIDE_INFLOW)
        for (int c = 0; c < 4; ++c) {
            const int sx = (c & 1) ? 1 : -1, sy = (c & 2) ? 1 : -1;
            const int xc = sx < 0 ? M - 1 : nx - M, yc = sy < 0 ? M - 1 : ny - M;
            for (int a = 0; a < M; ++a)
                for (int b = 0; b < M; ++b) {
                    const int x = sx < 0 ? a : nx - 1 - a, y = sy < 0 ? b : ny - 1 - b;
                    if (corner_kind == SIDE_ZG) pl.zg.push_back(make_int2(goff(x, y), goff(xc - sx, yc - sy)));
                    else pl.inflow.push_back(goff(x, y));
                }
        }
    B.n_unk = int(pl.ud.size());
    B.n_zg = int(pl.zg.size());

    // Tiles of the fused band kernel: runs of P positions of one
    // characteristic side with all M layers owned (each corner owned by the
    // W/E tile next to it), closed over the neighbours the RK4 stages read:
    // level l + 1 holds the unknowns level l reads that are not yet in the
    // tile, up to level 4 (U(t) only).
    {
        const int P = kTileUnknowns / M - 8;
        auto used_refs = [&](const UDesc& D, int* r) {
            int n = 0;
            if (D.kind >= 4) return 0;                  // corners read strips only
            r[n++] = D.j < M ? D.nb[0] : D.nb[2];       // normal stencil
            r[n++] = D.nb[1];
            r[n++] = D.nb[4];                           // tangential stencil
            r[n++] = D.nb[5];
            if (p->viscous == LBM_VISCOUS_FD) {
                if (D.j == M) r[n++] = D.nb[3];
                else r[n++] = D.nb[0];
            }
            return n;
        };
        std::vector<int> g2l(pl.ud.size(), -1);
        // grid node of strip slot sl: side s, depth d, position pp
        auto slot_side = [&](int sl) {
            int s = 0;
            while (!(E.cbc[s] && sl >= E.offS[s] && sl < E.offS[s] + E.ND * L[s])) ++s;
            return s;
        };
        auto slot_x = [&](int sl) {
            const int s = slot_side(sl), d = (sl - E.offS[s]) / L[s], pp = (sl - E.offS[s]) % L[s];
            int x, y;
            side_xf(s, pp, nx, ny, M, x, y);
            return x - d * kSN[s][0];
        };
        auto slot_y = [&](int sl) {
            const int s = slot_side(sl), d = (sl - E.offS[s]) / L[s], pp = (sl - E.offS[s]) % L[s];
            int x, y;
            side_xf(s, pp, nx, ny, M, x, y);
            return y - d * kSN[s][1];
        };
        B.max_nodes = 0;
        B.max_fx = 0;
        for (int s = 0; s < 4; ++s) {
            if (!E.cbc[s]) continue;
            for (int a = lo[s]; a <= hi[s]; a += P) {
                const int b = std::min(a + P - 1, hi[s]);
                std::vector<int> list, level;
                auto add = [&](int g, int lev) {
                    if (g2l[g] >= 0) return;
                    g2l[g] = int(list.size());
                    list.push_back(g);
                    level.push_back(lev);
                };
                for (int j = 1; j <= M; ++j)
                    for (int pp = a; pp <= b; ++pp) add(ref(s, j, pp), 0);
                if (corner_kind == SIDE_CBC && s < 2)
                    for (int c = s; c < 4; c += 2)           // corners on this W/E side
                        if ((c < 2 && a == lo[s]) || (c >= 2 && b == hi[s])) add(n_side + c, 0);
                size_t f0 = 0;
                for (int lev = 0; lev < 4; ++lev) {
                    const size_t f1 = list.size();
                    for (size_t q = f0; q < f1; ++q) {
                        int r[6];
                        const int nr = used_refs(pl.ud[list[q]], r);
                        for (int k = 0; k < nr; ++k)
                            if (r[k] >= 0) add(r[k], lev + 1);
                    }
                    f0 = f1;
                }
                if ((int)list.size() > kTileUnknowns) {
                    err = fmt("internal: boundary tile of %zu unknowns", list.size());
                    return LBM_ERR_ARG;
                }
                // strip nodes the tile reads or owns; node key = grid offset;
                // `use` adds kSN* bits to the node's flags
                std::vector<StripNode> nodes;
                std::unordered_map<int, int> n2l, fxl;
                auto node_of = [&](int sl, int use) {
                    const int x = slot_x(sl), y = slot_y(sl), key = goff(x, y);
                    auto it = n2l.find(key);
                    if (it != n2l.end()) {
                        nodes[it->second].flags |= use;
                        return it->second;
                    }
                    n2l[key] = int(nodes.size());
                    nodes.push_back(StripNode{x, y, sl, -1, -1, use});
                    return int(nodes.size()) - 1;
                };
                // the strips of the tile's own positions: pulled and written
                // by the tile (with the non-equilibrium moments at the depths
                // of the mesoscopic stencil)
                for (int d = 0; d < E.ND; ++d)
                    for (int pp = a; pp <= b; ++pp) {
                        const int sl = slot(s, d, pp);
                        nodes[node_of(sl, kSNPull | (meso && d >= M ? kSNNeq : 0))].gslot = sl;
                    }
                pl.tbeg.push_back(int(pl.ld.size()));
                for (size_t q = 0; q < list.size(); ++q) {
                    UDesc D = pl.ud[list[q]];
                    const UDesc Dg = D;
                    const bool comp = level[q] <= 3;
                    for (int k = 0; k < 6; ++k) {
                        if (D.nb[k] >= 0) D.nb[k] = g2l[D.nb[k]] >= 0 ? g2l[D.nb[k]] : 0;
                        else D.nb[k] = comp ? -(node_of(-Dg.nb[k] - 1, kSNLoadT | kSNPull) + 1) : -1;
                    }
                    for (int k = 0; k < 5; ++k)
                        D.vs[k] = comp && D.kind < 4 && meso ? node_of(Dg.vs[k], kSNLoadT) : 0;
                    if (level[q] == 0 && p->dirichlet != LBM_DIRICHLET_EQ) {
                        const int nl = node_of(Dg.wslot, kSNPull);
                        D.wslot = nl;
                        auto it = fxl.find(nl);
                        if (it == fxl.end()) {
                            const int fi = int(fxl.size());
                            fxl[nl] = fi;
                            nodes[nl].fx = fi;
                            D.wsrc = fi;
                        } else {
                            D.wsrc = it->second;
                        }
                    } else {
                        D.wslot = 0;
                        D.wsrc = 0;
                    }
                    D.gid = list[q];
                    D.level = level[q];
                    pl.ld.push_back(D);
                }
                for (int g : list) g2l[g] = -1;
                pl.sbeg.push_back(int(pl.sn.size()));
                pl.sn.insert(pl.sn.end(), nodes.begin(), nodes.end());
                B.max_nodes = std::max(B.max_nodes, int(nodes.size()));
                B.max_fx = std::max(B.max_fx, int(fxl.size()));
            }
        }
        pl.tbeg.push_back(int(pl.ld.size()));
        pl.sbeg.push_back(int(pl.sn.size()));
        B.n_tiles = int(pl.tbeg.size()) - 1;
        // device tables at a fixed stride per tile (kTileUnknowns unknowns,
        // max_nodes strip nodes), so the kernel reads no offsets first;
        // padding: level 99 (no unknown), x = -1 (no node)
        UDesc pad_u;
        std::memset(&pad_u, 0, sizeof pad_u);
        pad_u.level = 99;
        pl.ldp.assign((size_t)B.n_tiles * kTileUnknowns, pad_u);
        pl.snp.assign((size_t)B.n_tiles * B.max_nodes, StripNode{-1, -1, 0, -1, -1, 0});
        for (int t = 0; t < B.n_tiles; ++t) {
            std::copy(pl.ld.begin() + pl.tbeg[t], pl.ld.begin() + pl.tbeg[t + 1],
                      pl.ldp.begin() + (size_t)t * kTileUnknowns);
            std::copy(pl.sn.begin() + pl.sbeg[t], pl.sn.begin() + pl.sbeg[t + 1],
                      pl.snp.begin() + (size_t)t * B.max_nodes);
        }
    }
    B.viscous = p->viscous;
    B.dirichlet = p->dirichlet;
    for (int s = 0; s < 4; ++s) {
        B.scheme[s] = p->scheme[s];
        const double pinf = p->p_inf[s] != 0.0 ? p->p_inf[s] : cs2 * p->rho0;
        B.pdev[s] = pinf - cs2 * p->rho0;
        B.pdev_f[s] = float(B.pdev[s]);
    }
    B.alpha_T = p->alpha_T;
    B.beta_P = p->beta_P;
    B.t_inf = p->t_inf;
    B.alpha_V = p->alpha_V;
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
    pl.Uin[0] = p->inflow[0] - p->rho0;
    pl.Uin[1] = p->inflow[1];
    pl.Uin[2] = p->inflow[2];
    pl.Uin[3] = lattice != LBM_D2Q9 ? p->inflow[3] - 1.0 : 0.0;

    pl.Q = Q;
    pl.esize = p->storage == LBM_F64 ? 8 : (p->storage == LBM_F32 ? 4 : 2);
    // One-CTA band tiles hold whole SMs, which the bulk kernel beside them
    // then lacks.  The band launch gets as few CTAs as keep it, at ~25 us
    // per tile, within half the bulk kernel's time at ~6 TB/s; each CTA
    // takes every grid-th tile (measured on the 4096^2 pulse, 484 tiles:
    // 32 CTAs 22.5k MLUPS, 48 22.4k, 64 22.1k, 96 21.6k, one per tile 21.2k).
    if (p->band_ctas > 0) {
        B.grid = std::max(1, std::min(B.n_tiles, p->band_ctas));
    } else {
        const double bulk_us = double(G.bx1 - G.bx0) * double(G.by1 - G.by0) * 2.0 * Q * double(pl.esize) / 6.0e6;
        const double want = std::ceil(2.0 * 25.0 * B.n_tiles / std::max(bulk_us, 1.0));
        B.grid = std::max(1, std::min(B.n_tiles, int(std::min(want, 1.0e9))));
    }
    pl.f_bytes = (size_t)Q * (size_t)G.plane * pl.esize;
    pl.stripU_n = 2ull * E.nslots * 4;
    pl.stripN_n = 2ull * E.nslots * 5;
    const size_t nu = (size_t)B.n_unk;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + bytes); return at; };
    pl.off_f0 = take(pl.f_bytes);
    pl.off_f1 = take(pl.f_bytes);
    E.sesize = p->storage == LBM_F64 ? 8 : 4;
    pl.off_sU = take(pl.stripU_n * E.sesize);
    pl.off_sN = take(pl.stripN_n * E.sesize);
    pl.off_Ub = take(2 * nu * 32);
    pl.off_ud = take(nu * sizeof(UDesc));
    pl.off_ld = take(pl.ldp.size() * sizeof(UDesc));
    pl.off_sn = take(pl.snp.size() * sizeof(StripNode));
    pl.off_brun = take(sizeof(BulkRun));
    pl.off_zg = take(pl.zg.size() * sizeof(int2));
    pl.off_in = take(pl.inflow.size() * sizeof(int));
    pl.off_macro = take((size_t)4 * nx * ny * 8);
    pl.off_flag = take(2 * sizeof(int));
    pl.total = o;
    return LBM_OK;
}

template <typename T>
T* at(void* base, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(base) + off); }

int cuda_fail(lbm_handle* h, cudaError_t e, const char* what)
{
    if (h) h->err = fmt("%s: %s", what, cudaGetErrorString(e));
    return LBM_ERR_CUDA;
}

int check_launch(lbm_handle* h, int rc, const char* what)
{
    if (rc == 0) return LBM_OK;
    const cudaError_t e = cudaGetLastError();
    return cuda_fail(h, e == cudaSuccess ? cudaErrorLaunchFailure : e, what);
}

// cuTensorMapEncodeTiled from the driver, looked up through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3D view [Q][ny][nxp] of a population buffer; box = one padded row segment
// of 128 + 2H elements in `depth` consecutive planes (the bulk kernel's
// tensor copies of one c_y group).
int encode_population_map(lbm_handle* h, void* base, int depth, CUtensorMap* map)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) {
        h->err = "cuTensorMapEncodeTiled is not available from the driver";
        return LBM_ERR_CUDA;
    }
    const int es = int(h->esize);
    const int halo = es == 2 ? 8 : 4;
    const CUtensorMapDataType dt = es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                 : es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                           : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    cuuint64_t dims[3] = {cuuint64_t(h->G.nxp), cuuint64_t(h->ny), cuuint64_t(h->Q)};
    cuuint64_t strides[2] = {cuuint64_t(h->G.nxp) * es, cuuint64_t(h->G.plane) * es};
    cuuint32_t box[3] = {cuuint32_t(128 + 2 * halo), 1, cuuint32_t(depth)};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        h->err = fmt("cuTensorMapEncodeTiled failed (%d)", int(r));
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

int setup(lbm_handle* h, int lattice, int nx, int ny, double tau, const lbm_cbc_params* p,
          const Plan& pl, void* ws, size_t ws_bytes, bool owns)
{
    h->lattice = lattice;
    h->nx = nx;
    h->ny = ny;
    h->M = pl.G.M;
    h->Q = pl.Q;
    h->tau = tau;
    h->P = *p;
    h->storage = p->storage;
    h->G = pl.G;
    h->O = pl.O;
    h->E = pl.E;
    h->B = pl.B;
    h->bulk = pl.bulk;
    h->esize = pl.esize;
    h->f_bytes = pl.f_bytes;
    h->ws = ws;
    h->ws_bytes = ws_bytes;
    h->owns_ws = owns;
    h->f[0] = at<char>(ws, pl.off_f0);
    h->f[1] = at<char>(ws, pl.off_f1);
    h->E.stripU = at<char>(ws, pl.off_sU);
    h->E.stripN = at<char>(ws, pl.off_sN);
    h->B.Ub = at<double>(ws, pl.off_Ub);
    h->B.Ya = h->B.Yb = h->B.acc = h->B.V = nullptr;
    h->B.mask = nullptr;
    h->B.ud = at<UDesc>(ws, pl.off_ud);
    h->B.ld = at<UDesc>(ws, pl.off_ld);
    h->B.sn = at<StripNode>(ws, pl.off_sn);
    h->B.zg = at<int2>(ws, pl.off_zg);
    h->inflow_nodes = at<int>(ws, pl.off_in);
    h->n_inflow = int(pl.inflow.size());
    for (int c = 0; c < 4; ++c) h->Uin[c] = pl.Uin[c];
    h->macro = at<double>(ws, pl.off_macro);
    h->flag = at<int>(ws, pl.off_flag);
    h->B.status = h->flag + 1;
    const int depths[5] = {7, 5, 3, 2, 1};
    for (int b = 0; b < 2; ++b)
        for (int k = 0; k < 5; ++k) {
            const int rc = encode_population_map(h, h->f[b], depths[k] <= h->Q ? depths[k] : 1, &h->tmap[b][k]);
            if (rc != LBM_OK) return rc;
        }
    // Run descriptor of the persistent bulk kernel (this grid alone), which
    // a batch copies into its group's table.
    {
        BulkRun r;
        std::memset(&r, 0, sizeof r);
        CUtensorMap* dst[5] = {&r.maps[0].m7, &r.maps[0].m5, &r.maps[0].m3, &r.maps[0].m2, &r.maps[0].m1};
        CUtensorMap* dst1[5] = {&r.maps[1].m7, &r.maps[1].m5, &r.maps[1].m3, &r.maps[1].m2, &r.maps[1].m1};
        for (int k = 0; k < 5; ++k) {
            *dst[k] = h->tmap[0][k];
            *dst1[k] = h->tmap[1][k];
        }
        r.f[0] = h->f[0];
        r.f[1] = h->f[1];
        r.status = h->flag + 1;
        r.G = h->G;
        r.R = h->bulk;
        r.seg0 = h->bulk.x0 / 128;
        r.nseg = (h->bulk.x1 + 127) / 128 - r.seg0;
        r.first = 0;
        h->bulk_items = h->bulk.x1 > h->bulk.x0 ? r.nseg * (h->bulk.y1 - h->bulk.y0) : 0;
        h->brun = at<BulkRun>(ws, pl.off_brun);
        const cudaError_t e0 = cudaMemcpyAsync(h->brun, &r, sizeof r, cudaMemcpyHostToDevice, h->stream);
        if (e0 != cudaSuccess) return cuda_fail(h, e0, "bulk run descriptor");
    }
    // Band CTAs share their SMs with bulk CTAs (reserving whole SMs for the
    // band through its shared-memory request measured slower: the bulk loses
    // more than the band gains).
    if (h->B.n_tiles > 0 && prepare_boundary(h->lattice, h->storage, h->B) != 0)
        return cuda_fail(h, cudaGetLastError(), "band kernel shared memory");
    cudaError_t e = cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream set-up");
    // Zero the population buffers (the row padding x >= nx is never written,
    // and a saved state then holds no leftover bytes of the workspace), the
    // strips (positions no kernel writes stay finite) and the status words,
    // and upload the boundary tables.
    e = cudaMemsetAsync(h->f[0], 0, h->f_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->f[1], 0, h->f_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->E.stripU, 0, pl.stripU_n * h->E.sesize, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->flag, 0, 2 * sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->E.stripN, 0, pl.stripN_n * h->E.sesize, h->stream);
    if (e == cudaSuccess && !pl.ud.empty())
        e = cudaMemcpyAsync(const_cast<UDesc*>(h->B.ud), pl.ud.data(), pl.ud.size() * sizeof(UDesc),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && !pl.ldp.empty())
        e = cudaMemcpyAsync(const_cast<UDesc*>(h->B.ld), pl.ldp.data(), pl.ldp.size() * sizeof(UDesc),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && !pl.snp.empty())
        e = cudaMemcpyAsync(const_cast<StripNode*>(h->B.sn), pl.snp.data(), pl.snp.size() * sizeof(StripNode),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && !pl.zg.empty())
        e = cudaMemcpyAsync(const_cast<int2*>(h->B.zg), pl.zg.data(), pl.zg.size() * sizeof(int2),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && !pl.inflow.empty())
        e = cudaMemcpyAsync(h->inflow_nodes, pl.inflow.data(), pl.inflow.size() * sizeof(int),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "workspace set-up");
    return LBM_OK;
}

int mark(lbm_handle* h, int k, cudaStream_t st)
{
    if (!h->kev[k]) return LBM_OK;
    const cudaError_t e = cudaEventRecord(h->kev[k], st);
    return e == cudaSuccess ? LBM_OK : cuda_fail(h, e, "timing event");
}

// Bulk update of step (parity par) on stream st, bracketed by the caller's
// timing events 0 and 1 when set; early: start beside the band kernel just
// launched on st (programmatic stream serialization).
int bulk(lbm_handle* h, int par, cudaStream_t st, bool early = false)
{
    int rc = mark(h, 0, st);
    if (rc != LBM_OK) return rc;
    rc = launch_bulk(h->lattice, h->storage, h->G, h->O, h->bulk, h->tmap[par], h->f[par],
                     h->f[par ^ 1], h->flag + 1, st, early);
    if (rc) return check_launch(h, rc, "bulk kernel");
    return mark(h, 1, st);
}

// Inflow equilibrium (once per buffer) and the band kernel of step (parity
// par) on stream st, bracketed by timing events 3 and 4.
int band(lbm_handle* h, int par, cudaStream_t st)
{
    int rc = mark(h, 3, st);
    if (rc != LBM_OK) return rc;
    // Inflow nodes carry a fixed equilibrium, imposed after streaming like
    // every boundary condition; each buffer gets it once, the first time a
    // step writes that buffer.
    if (h->n_inflow > 0 && !h->inflow_done[par ^ 1]) {
        rc = launch_inflow(h->lattice, h->storage, h->G, h->inflow_nodes, h->n_inflow, h->Uin,
                           h->f[par ^ 1], st);
        if (rc) return check_launch(h, rc, "inflow kernel");
        h->inflow_done[par ^ 1] = true;
    }
    rc = launch_boundary(h->lattice, h->storage, h->G, h->O, h->E, h->B, h->f[par], h->f[par ^ 1],
                         par, st);
    if (rc) return check_launch(h, rc, "band kernel");
    return mark(h, 4, st);
}


// Zero-gradient copies of step (parity par), after the bulk update.
int zero_gradient(lbm_handle* h, int par, cudaStream_t st)
{
    const int rc = launch_zg(h->lattice, h->storage, h->G, h->B, h->f[par ^ 1], st);
    return rc ? check_launch(h, rc, "zero-gradient kernel") : LBM_OK;
}

void release_streams(lbm_handle* h)
{
    if (h->aux) cudaStreamSynchronize(h->aux);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->aux) cudaStreamDestroy(h->aux);
    h->aux = nullptr;
    h->ev_fork = h->ev_join = nullptr;
}

int create_common(int lattice, int nx, int ny, double tau, const lbm_cbc_params* p, void* ws,
                  size_t ws_bytes, lbm_handle** out)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    Plan pl;
    std::string err;
    int rc = make_plan(lattice, nx, ny, tau, p, pl, err);
    if (rc != LBM_OK) {
        fprintf(stderr, "lbm_create: %s\n", err.c_str());
        return rc;
    }
    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) return LBM_ERR_ALLOC;
    bool owns = false;
    if (ws) {
        if (ws_bytes < pl.total || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) {
            fprintf(stderr, "lbm_create_in: workspace of %zu bytes at %p is too small or misaligned (%zu needed)\n",
                    ws_bytes, ws, pl.total);
            delete h;
            return LBM_ERR_ARG;
        }
    } else {
        const cudaError_t e = cudaMalloc(&ws, pl.total);
        if (e != cudaSuccess) {
            fprintf(stderr, "lbm_create: cudaMalloc(%zu): %s\n", pl.total, cudaGetErrorString(e));
            delete h;
            return LBM_ERR_ALLOC;
        }
        ws_bytes = pl.total;
        owns = true;
    }
    rc = setup(h, lattice, nx, ny, tau, p, pl, ws, ws_bytes, owns);
    if (rc != LBM_OK) {
        fprintf(stderr, "lbm_create: %s\n", h->err.c_str());
        release_streams(h);
        if (owns) cudaFree(ws);
        delete h;
        return rc;
    }
    *out = h;
    return LBM_OK;
}

}  // namespace

// FP64 FMA throughput (the roof of ALU-bound FP64 work): every thread runs
// kFmaChains independent chains x <- x a + b on registers, enough to hide the
// FMA latency at the FP64 issue rate; no memory traffic inside the loop.  The
// chains start at x >= 0 and a, b > 0 keep them there, so the sum never
// equals the negative `never` argument and nothing is stored; the test keeps
// the chains live.
constexpr int kFmaChains = 8, kFmaThreads = 256, kFmaCtasPerSm = 8;

__global__ void __launch_bounds__(kFmaThreads) k_fp64_fma(double* out, int iters, double never)
{
    double x[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
    const double a = 0.9999999, b = 1e-7;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += x[c];
    if (s == never) out[blockIdx.x] = s;
}

extern "C" {

int lbm_params_default(lbm_cbc_params* p)
{
    if (!p) return LBM_ERR_ARG;
    std::memset(p, 0, sizeof *p);
    for (int s = 0; s < 4; ++s) {
        p->side[s] = LBM_SIDE_PERIODIC;
        p->scheme[s] = LBM_CBC_RELAX;
        p->p_inf[s] = 0.0;
    }
    p->viscous = LBM_VISCOUS_MESO;
    p->dirichlet = LBM_DIRICHLET_EQ;
    p->inflow[0] = 1.0;
    p->inflow[3] = 1.0;
    p->storage = LBM_F32;
    p->rho0 = 1.0;
    return LBM_OK;
}

int lbm_workspace_bytes(int lattice, int nx, int ny, const lbm_cbc_params* p, size_t* bytes)
{
    if (!bytes) return LBM_ERR_ARG;
    Plan pl;
    std::string err;
    const int rc = make_plan(lattice, nx, ny, 0.75, p, pl, err);
    if (rc != LBM_OK) return rc;
    *bytes = pl.total;
    return LBM_OK;
}

int lbm_create(int lattice, int nx, int ny, double tau, const lbm_cbc_params* p, lbm_handle** out)
{
    return create_common(lattice, nx, ny, tau, p, nullptr, 0, out);
}

int lbm_create_in(int lattice, int nx, int ny, double tau, const lbm_cbc_params* p,
                  void* dev_workspace, size_t workspace_bytes, lbm_handle** out)
{
    if (!dev_workspace) return LBM_ERR_ARG;
    return create_common(lattice, nx, ny, tau, p, dev_workspace, workspace_bytes, out);
}

int lbm_set_stream(lbm_handle* h, void* stream)
{
    if (!h) return LBM_ERR_ARG;
    h->stream = static_cast<cudaStream_t>(stream);
    return LBM_OK;
}

int lbm_init_fields(lbm_handle* h, const double* rho, const double* ux, const double* uy,
                    const double* T, int on_device)
{
    if (!h) return LBM_ERR_ARG;
    if (!rho || !ux || !uy || (!T && h->lattice != LBM_D2Q9)) {
        h->err = "NULL field";
        return LBM_ERR_ARG;
    }
    const size_t n = (size_t)h->nx * h->ny;
    const double *dr = rho, *du = ux, *dv = uy, *dt = T;
    if (!on_device) {
        double* m = h->macro;
        const double* src[4] = {rho, ux, uy, T ? T : rho};
        for (int c = 0; c < 4; ++c) {
            const cudaError_t e = cudaMemcpyAsync(m + c * n, src[c], n * 8, cudaMemcpyHostToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "copy of initial fields");
        }
        dr = m;
        du = m + n;
        dv = m + 2 * n;
        dt = m + 3 * n;
    } else if (!dt) {
        dt = dr;   // unused by the isothermal lattice
    }
    int rc = launch_init(h->lattice, h->storage, h->G, h->E, h->B, dr, du, dv, dt, h->f[0], h->stream);
    if (rc) return check_launch(h, rc, "init kernels");
    h->inflow_done[0] = h->inflow_done[1] = false;
    cudaError_t e = cudaMemsetAsync(h->flag, 0, 2 * sizeof(int), h->stream);   // a fresh state, no status
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "init");
    h->steps = 0;
    h->initialized = true;
    h->bulk_pending = false;
    h->grad_stale = false;
    return LBM_OK;
}

int lbm_step_phase(lbm_handle* h, int phase)
{
    if (!h) return LBM_ERR_ARG;
    if (!h->initialized) {
        h->err = "lbm_step before lbm_init_fields";
        return LBM_ERR_STATE;
    }
    if (h->grad_stale) { h->err = kGradStale; return LBM_ERR_STATE; }
    const int par = int(h->steps & 1);
    if (phase == 0) {
        if (h->bulk_pending) { h->err = "bulk phase issued twice"; return LBM_ERR_STATE; }
        int rc = mark(h, 2, h->stream);
        if (rc == LBM_OK) rc = bulk(h, par, h->stream);
        if (rc != LBM_OK) return rc;
        h->bulk_pending = true;
        return LBM_OK;
    }
    if (phase == 1) {
        if (!h->bulk_pending) { h->err = "boundary phase before bulk phase"; return LBM_ERR_STATE; }
        int rc = band(h, par, h->stream);
        if (rc == LBM_OK) rc = zero_gradient(h, par, h->stream);
        if (rc != LBM_OK) return rc;
        h->bulk_pending = false;
        h->steps++;
        return LBM_OK;
    }
    h->err = fmt("unknown phase %d", phase);
    return LBM_ERR_ARG;
}

int lbm_step(lbm_handle* h, int n)
{
    if (!h || n < 0) return LBM_ERR_ARG;
    if (!h->initialized) {
        h->err = "lbm_step before lbm_init_fields";
        return LBM_ERR_STATE;
    }
    if (h->bulk_pending) { h->err = "lbm_step in the middle of a phased step"; return LBM_ERR_STATE; }
    if (h->grad_stale) { h->err = kGradStale; return LBM_ERR_STATE; }
    for (int i = 0; i < n; ++i) {
        const int par = int(h->steps & 1);
        int rc = mark(h, 2, h->stream);
        if (rc != LBM_OK) return rc;
        if (h->B.n_tiles == 0) {
            // no characteristic side: bulk, inflow and zero gradient in order
            rc = bulk(h, par, h->stream);
            if (rc == LBM_OK) rc = band(h, par, h->stream);
            if (rc == LBM_OK) rc = zero_gradient(h, par, h->stream);
            if (rc != LBM_OK) return rc;
            h->steps++;
            continue;
        }
        // The band kernel and the bulk kernel write disjoint nodes of the
        // new buffer and read only the old one, so they run side by side:
        // the band first (its few CTAs take their SMs before the bulk's),
        // then the bulk on the same stream with early start, which the band
        // kernel allows at once; the zero-gradient copies and the next step
        // wait for both.
        if (!h->kev[0] && !h->kev[3]) {
            rc = band(h, par, h->stream);
            if (rc == LBM_OK) rc = bulk(h, par, h->stream, true);
            if (rc == LBM_OK) rc = zero_gradient(h, par, h->stream);
            if (rc != LBM_OK) return rc;
            h->steps++;
            continue;
        }
        // With the caller's timing events between the launches: fork the
        // bulk kernel and the zero-gradient copies onto the internal stream
        // and join before the next step.
        cudaError_t e = cudaEventRecord(h->ev_fork, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->aux, h->ev_fork, 0);
        if (e != cudaSuccess) return cuda_fail(h, e, "fork");
        rc = band(h, par, h->stream);
        if (rc == LBM_OK) rc = bulk(h, par, h->aux);
        if (rc == LBM_OK) rc = zero_gradient(h, par, h->aux);
        if (rc != LBM_OK) return rc;
        e = cudaEventRecord(h->ev_join, h->aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_join, 0);
        if (e != cudaSuccess) return cuda_fail(h, e, "join");
        h->steps++;
    }
    return LBM_OK;
}

int lbm_set_wait_limit(lbm_handle* h, double seconds)
{
    if (!h) return LBM_ERR_ARG;
    if (!(seconds >= 0.0) || !(seconds <= 60.0)) {
        h->err = "wait limit must be in [0, 60] seconds";
        return LBM_ERR_ARG;
    }
    h->G.wait_ns = (unsigned long long)(seconds * 1e9);
    BulkRun* r = h->brun;   // the batch copy of this run's geometry, as well
    const cudaError_t e = cudaMemcpyAsync(&r->G.wait_ns, &h->G.wait_ns, sizeof h->G.wait_ns,
                                          cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(h, e, "wait limit");
}

int lbm_set_kernel_events(lbm_handle* h, void* const* events, int n)
{
    if (!h) return LBM_ERR_ARG;
    if (!(n == 0 || n == 2 || n == 5) || (n > 0 && !events)) {
        h->err = "lbm_set_kernel_events takes 0, 2 or 5 events";
        return LBM_ERR_ARG;
    }
    for (int k = 0; k < n; ++k)
        if (!events[k]) { h->err = "NULL event"; return LBM_ERR_ARG; }
    for (int k = 0; k < 5; ++k) h->kev[k] = k < n ? static_cast<cudaEvent_t>(events[k]) : nullptr;
    return LBM_OK;
}

int lbm_get_macros(lbm_handle* h, double* rho, double* ux, double* uy, double* T, int on_device)
{
    if (!h) return LBM_ERR_ARG;
    if (!h->initialized) { h->err = "lbm_get_macros before lbm_init_fields"; return LBM_ERR_STATE; }
    if (h->bulk_pending) { h->err = "lbm_get_macros in the middle of a step"; return LBM_ERR_STATE; }
    if (!rho || !ux || !uy || !T) { h->err = "NULL output"; return LBM_ERR_ARG; }
    const size_t n = (size_t)h->nx * h->ny;
    double* d[4];
    if (on_device) {
        d[0] = rho; d[1] = ux; d[2] = uy; d[3] = T;
    } else {
        for (int c = 0; c < 4; ++c) d[c] = h->macro + c * n;
    }
    cudaError_t e = cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream);   // status word kept
    if (e != cudaSuccess) return cuda_fail(h, e, "flag reset");
    const int rc = launch_macros(h->lattice, h->storage, h->G, h->f[h->steps & 1], d[0], d[1], d[2], d[3],
                                 h->flag, h->stream);
    if (rc) return check_launch(h, rc, "macros kernel");
    if (!on_device) {
        double* dst[4] = {rho, ux, uy, T};
        for (int c = 0; c < 4; ++c) {
            e = cudaMemcpyAsync(dst[c], d[c], n * 8, cudaMemcpyDeviceToHost, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "copy of macros");
        }
    }
    int flag[2] = {0, 0};
    e = cudaMemcpyAsync(flag, h->flag, sizeof flag, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "macros");
    if (flag[1]) {
        h->err = (flag[1] & 2) ? "a tensor copy of the bulk kernel did not complete in time"
                               : "a cluster exchange of the band kernel did not complete in time";
        return LBM_ERR_TIMEOUT;
    }
    if (flag[0]) {
        h->err = "non-finite macroscopic values";
        return LBM_ERR_NUMERICAL;
    }
    return LBM_OK;
}

namespace {
struct StateHeader {
    char magic[8];
    int lattice, nx, ny, storage, n_unk;
    long long steps;
    unsigned long long f_bytes, stripU_n, stripN_n;
    double u_ref[2];    // the reference the populations are held against
};
}  // namespace

int lbm_state_bytes(const lbm_handle* h, size_t* bytes)
{
    if (!h || !bytes) return LBM_ERR_ARG;
    *bytes = sizeof(StateHeader) + h->f_bytes + 18ull * h->E.nslots * h->E.sesize + 32ull * h->B.n_unk;
    return LBM_OK;
}

int lbm_get_state(lbm_handle* h, void* buf, size_t bytes)
{
    size_t need = 0;
    if (lbm_state_bytes(h, &need) != LBM_OK || !buf) return LBM_ERR_ARG;
    if (bytes < need) { h->err = fmt("state buffer needs %zu bytes", need); return LBM_ERR_ARG; }
    if (!h->initialized || h->bulk_pending) { h->err = "no complete state to save"; return LBM_ERR_STATE; }
    if (h->grad_stale) { h->err = kGradStale; return LBM_ERR_STATE; }
    StateHeader hd{};
    std::memcpy(hd.magic, "LBMCBC03", 8);
    hd.lattice = h->lattice; hd.nx = h->nx; hd.ny = h->ny; hd.storage = h->storage; hd.n_unk = h->B.n_unk;
    hd.steps = h->steps; hd.f_bytes = h->f_bytes; hd.stripU_n = 8ull * h->E.nslots; hd.stripN_n = 10ull * h->E.nslots;
    hd.u_ref[0] = h->G.ref ? h->G.uref[0] : 0.0;
    hd.u_ref[1] = h->G.ref ? h->G.uref[1] : 0.0;
    char* p = static_cast<char*>(buf);
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    cudaError_t e = cudaMemcpyAsync(p, h->f[h->steps & 1], h->f_bytes, cudaMemcpyDeviceToHost, h->stream);
    p += h->f_bytes;
    const size_t su = 8ull * h->E.nslots * h->E.sesize, sn = 10ull * h->E.nslots * h->E.sesize;
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, h->E.stripU, su, cudaMemcpyDeviceToHost, h->stream);
    p += su;
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, h->E.stripN, sn, cudaMemcpyDeviceToHost, h->stream);
    p += sn;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p, h->B.Ub + (h->steps & 1) * 4ull * h->B.n_unk, 32ull * h->B.n_unk,
                            cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "state copy");
    return LBM_OK;
}

int lbm_set_state(lbm_handle* h, const void* buf, size_t bytes)
{
    size_t need = 0;
    if (lbm_state_bytes(h, &need) != LBM_OK || !buf) return LBM_ERR_ARG;
    if (bytes < need) { h->err = "state buffer too small"; return LBM_ERR_ARG; }
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    if (std::memcmp(hd.magic, "LBMCBC03", 8) != 0 || hd.lattice != h->lattice || hd.nx != h->nx ||
        hd.ny != h->ny || hd.storage != h->storage || hd.n_unk != h->B.n_unk || hd.f_bytes != h->f_bytes ||
        hd.stripU_n != 8ull * h->E.nslots || hd.stripN_n != 10ull * h->E.nslots ||
        hd.u_ref[0] != (h->G.ref ? h->G.uref[0] : 0.0) || hd.u_ref[1] != (h->G.ref ? h->G.uref[1] : 0.0)) {
        h->err = "state was saved from a different configuration";
        return LBM_ERR_ARG;
    }
    const char* p = static_cast<const char*>(buf) + sizeof hd;
    cudaError_t e = cudaMemcpyAsync(h->f[hd.steps & 1], p, h->f_bytes, cudaMemcpyHostToDevice, h->stream);
    p += h->f_bytes;
    const size_t su = 8ull * h->E.nslots * h->E.sesize, sn = 10ull * h->E.nslots * h->E.sesize;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->E.stripU, p, su, cudaMemcpyHostToDevice, h->stream);
    p += su;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->E.stripN, p, sn, cudaMemcpyHostToDevice, h->stream);
    p += sn;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->B.Ub + (hd.steps & 1) * 4ull * h->B.n_unk, p, 32ull * h->B.n_unk,
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "state restore");
    h->steps = hd.steps;
    h->initialized = true;
    h->bulk_pending = false;
    h->grad_stale = false;
    h->inflow_done[0] = h->inflow_done[1] = false;
    return LBM_OK;
}

long long lbm_steps_done(const lbm_handle* h) { return h ? h->steps : -1; }

// ---------------------------------------------------------------------------
// Gradients with respect to the relaxation parameters (tangent-linear steps)
// ---------------------------------------------------------------------------

int lbm_grad_begin(lbm_handle* h) { return lbm_grad_begin_along(h, nullptr); }

int lbm_grad_begin_along(lbm_handle* h, const double* dirs)
{
    if (!h) return LBM_ERR_ARG;
    if (dirs)
        for (int i = 0; i < 3 * kTLParams; ++i)
            if (!std::isfinite(dirs[i])) { h->err = "gradient directions must be finite"; return LBM_ERR_ARG; }
    if (!h->initialized || h->bulk_pending) { h->err = "lbm_grad_begin before a complete step state"; return LBM_ERR_STATE; }
    if (h->tl_mem) { h->err = "gradient steps already begun"; return LBM_ERR_STATE; }
    if (h->G.ref) { h->err = "gradient steps need u_ref = (0, 0)"; return LBM_ERR_ARG; }
    if (h->storage != LBM_F64 && h->storage != LBM_F32) {
        h->err = "gradient steps need FP64 or FP32 storage";
        return LBM_ERR_ARG;
    }
    if (h->B.n_unk > 0 && h->B.dirichlet != 0) {
        h->err = "gradient steps need the equilibrium Dirichlet condition";
        return LBM_ERR_ARG;
    }
    if (h->n_inflow > 0 || h->B.n_zg > 0) {
        h->err = "gradient steps support characteristic and periodic sides only";
        return LBM_ERR_ARG;
    }
    const size_t dual = tl_dual_bytes();
    const size_t tbytes = 3 * h->f_bytes;
    const size_t sbytes = (size_t)std::max(1, h->E.nslots) * 4 * dual;
    const size_t nbytes = (size_t)std::max(1, h->E.nslots) * 5 * dual;
    const size_t ubytes = (size_t)std::max(1, h->B.n_unk) * 4 * dual;
    size_t o = 0;
    auto take = [&](size_t b) { const size_t at = o; o = align_up(o + b); return at; };
    const size_t o_t0 = take(tbytes), o_t1 = take(tbytes), o_st = take(sbytes), o_st1 = take(sbytes),
                 o_sn = take(nbytes), o_sn1 = take(nbytes),
                 o_ud = take(ubytes), o_uf = take(ubytes), o_ya = take(ubytes), o_yb = take(ubytes),
                 o_acc = take(ubytes), o_vv = take(ubytes),
                 o_mask = take((size_t)std::max(1, h->B.n_unk) * sizeof(int)), o_sums = take(4 * sizeof(double));
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, o);
    if (e != cudaSuccess) return cuda_fail(h, e, "gradient state allocation");
    TLState& T = h->tl;
    T.t[0] = at<char>(mem, o_t0);
    T.t[1] = at<char>(mem, o_t1);
    T.strip[0] = at<char>(mem, o_st);
    T.strip[1] = at<char>(mem, o_st1);
    T.stripN[0] = at<char>(mem, o_sn);
    T.stripN[1] = at<char>(mem, o_sn1);
    T.Ud = at<char>(mem, o_ud);
    T.Uf = at<char>(mem, o_uf);
    T.Ya = at<char>(mem, o_ya);
    T.Yb = at<char>(mem, o_yb);
    T.acc = at<char>(mem, o_acc);
    T.mask = at<int>(mem, o_mask);
    T.Vv = at<char>(mem, o_vv);
    T.sums = at<double>(mem, o_sums);
    for (int k = 0; k < 3; ++k)
        for (int q = 0; q < kTLParams; ++q) T.dirs[k][q] = dirs ? dirs[k * kTLParams + q] : (q == k ? 1.0 : 0.0);
    h->tl_mem = mem;
    // the initial fields do not depend on the parameters: zero derivatives
    e = cudaMemsetAsync(mem, 0, o, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "gradient state");
    if (launch_tl_seed(h->lattice, h->storage, T, h->G, h->E, h->B, h->f, int(h->steps & 1), h->stream))
        return check_launch(h, -1, "gradient seed kernel");
    h->grad_stale = true;
    return LBM_OK;
}

int lbm_grad_step(lbm_handle* h, int n, const double* dP_ref, long long ref_stride)
{
    if (!h || n < 0) return LBM_ERR_ARG;
    if (!h->tl_mem) { h->err = "lbm_grad_step before lbm_grad_begin"; return LBM_ERR_STATE; }
    for (int i = 0; i < n; ++i) {
        const int par = int(h->steps & 1);
        const double* ref = dP_ref ? dP_ref + (long long)i * ref_stride : nullptr;
        if (launch_tl_step(h->lattice, h->storage, h->tl, h->G, h->E, h->B, h->bulk, h->f, par, ref,
                           h->stream))
            return check_launch(h, -1, "tangent-linear step");
        h->steps++;
    }
    return LBM_OK;
}

int lbm_grad_result(lbm_handle* h, double* J, double* dJ)
{
    if (!h || !J || !dJ) return LBM_ERR_ARG;
    if (!h->tl_mem) { h->err = "lbm_grad_result before lbm_grad_begin"; return LBM_ERR_STATE; }
    double v[4];
    cudaError_t e = cudaMemcpyAsync(v, h->tl.sums, sizeof v, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "gradient result");
    *J = v[0];
    for (int k = 0; k < 3; ++k) dJ[k] = v[k + 1];
    return LBM_OK;
}

int lbm_grad_end(lbm_handle* h)
{
    if (!h) return LBM_ERR_ARG;
    if (!h->tl_mem) return LBM_OK;
    cudaError_t e = h->stream ? cudaStreamSynchronize(h->stream) : cudaDeviceSynchronize();
    cudaFree(h->tl_mem);
    h->tl_mem = nullptr;
    h->tl = TLState{};
    return e == cudaSuccess ? LBM_OK : cuda_fail(h, e, "gradient state release");
}

// ---------------------------------------------------------------------------
// Reverse-mode gradients with segment checkpointing (adjoint.cu)
// ---------------------------------------------------------------------------

namespace {

// Bytes of one checkpoint: the populations of the current parity, both
// parities of the strips and of the boundary state.
size_t adj_ckpt_layout(const lbm_handle* h, size_t* o_su, size_t* o_sn, size_t* o_ub)
{
    size_t o = align_up(h->f_bytes);
    *o_su = o;
    o = align_up(o + 8ull * h->E.nslots * h->E.sesize);
    *o_sn = o;
    o = align_up(o + 10ull * h->E.nslots * h->E.sesize);
    *o_ub = o;
    return align_up(o + 64ull * h->B.n_unk);
}

int adj_copy_state(lbm_handle* h, int idx, bool save)
{
    size_t o_su, o_sn, o_ub;
    adj_ckpt_layout(h, &o_su, &o_sn, &o_ub);
    char* c = h->adj_ckpt + (size_t)idx * h->adj_ckpt_bytes;
    const size_t su = 8ull * h->E.nslots * h->E.sesize, sn = 10ull * h->E.nslots * h->E.sesize;
    void* f = h->f[h->steps & 1];
    auto cp = [&](void* ck, void* live, size_t n) {
        if (n == 0) return cudaSuccess;
        return save ? cudaMemcpyAsync(ck, live, n, cudaMemcpyDeviceToDevice, h->stream)
                    : cudaMemcpyAsync(live, ck, n, cudaMemcpyDeviceToDevice, h->stream);
    };
    cudaError_t e = cp(c, f, h->f_bytes);
    if (e == cudaSuccess) e = cp(c + o_su, h->E.stripU, su);
    if (e == cudaSuccess) e = cp(c + o_sn, h->E.stripN, sn);
    if (e == cudaSuccess) e = cp(c + o_ub, h->B.Ub, 64ull * h->B.n_unk);
    return e == cudaSuccess ? LBM_OK : cuda_fail(h, e, save ? "checkpoint" : "checkpoint restore");
}

// Bulk-macro history buffer b (0 or 1) of the adjoint state.
AdjState adj_hist(const lbm_handle* h, int b)
{
    AdjState A = h->adj;
    A.Mh = static_cast<char*>(A.Mh) + (size_t)b * h->adj_hist_bytes;
    return A;
}

// The boundary state and the strips of the current time into slot k (the
// step index within the run) of the history.
int adj_snapshot(lbm_handle* h, const AdjState& A, int k)
{
    const int par = int(h->steps & 1);
    const size_t nu = (size_t)h->B.n_unk, ns = (size_t)h->E.nslots, es = h->E.sesize;
    cudaError_t e = cudaSuccess;
    if (nu) e = cudaMemcpyAsync(A.Ubh + (size_t)k * nu * 4, h->B.Ub + par * nu * 4, nu * 32,
                                cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && ns)
        e = cudaMemcpyAsync(static_cast<char*>(A.stUh) + (size_t)k * ns * 4 * es,
                            static_cast<char*>(h->E.stripU) + par * ns * 4 * es, ns * 4 * es,
                            cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && ns)
        e = cudaMemcpyAsync(static_cast<char*>(A.stNh) + (size_t)k * ns * 5 * es,
                            static_cast<char*>(h->E.stripN) + par * ns * 5 * es, ns * 5 * es,
                            cudaMemcpyDeviceToDevice, h->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(h, e, "history snapshot");
}

}  // namespace

int lbm_adj_begin(lbm_handle* h, int checkpoint_every, int max_steps)
{
    if (!h) return LBM_ERR_ARG;
    if (checkpoint_every < 1 || max_steps < 1) {
        h->err = "checkpoint interval and step count must be positive";
        return LBM_ERR_ARG;
    }
    if (!h->initialized || h->bulk_pending) { h->err = "lbm_adj_begin before a complete step state"; return LBM_ERR_STATE; }
    if (h->grad_stale || h->tl_mem) { h->err = "tangent-linear gradient steps in use"; return LBM_ERR_STATE; }
    if (h->adj_mem) { h->err = "reverse-mode gradients already begun"; return LBM_ERR_STATE; }
    if (h->G.ref) { h->err = "reverse-mode gradients need u_ref = (0, 0)"; return LBM_ERR_ARG; }
    if (h->storage != LBM_F64 && h->storage != LBM_F32) {
        h->err = "reverse-mode gradients need FP64 or FP32 storage";
        return LBM_ERR_ARG;
    }
    if (h->B.n_unk > 0 && h->B.dirichlet != 0) {
        h->err = "reverse-mode gradients need the equilibrium Dirichlet condition";
        return LBM_ERR_ARG;
    }
    if (h->n_inflow > 0 || h->B.n_zg > 0) {
        h->err = "reverse-mode gradients support characteristic and periodic sides only";
        return LBM_ERR_ARG;
    }
    const int K = std::min(checkpoint_every, max_steps);
    const size_t N = (size_t)h->nx * h->ny, nu = (size_t)std::max(1, h->B.n_unk),
                 ns = (size_t)std::max(1, h->E.nslots), es = h->E.sesize;
    const int nckpt = (max_steps + K - 1) / K + 1;
    size_t o_su, o_sn, o_ub;
    h->adj_ckpt_bytes = adj_ckpt_layout(h, &o_su, &o_sn, &o_ub);
    size_t o = 0;
    auto take = [&](size_t b) { const size_t at = o; o = align_up(o + b); return at; };
    // the bulk macros of a segment in two buffers (the recompute of one
    // segment runs beside the reverse steps of the next); the boundary state
    // and the strips of every step of the run, recorded by the forward pass
    const size_t o_mh = take((size_t)K * 4 * N * es);
    h->adj_hist_bytes = o;
    o += h->adj_hist_bytes;
    const size_t o_ubh = take((size_t)(max_steps + 1) * nu * 32),
                 o_suh = take((size_t)(max_steps + 1) * ns * 4 * es),
                 o_snh = take((size_t)(max_steps + 1) * ns * 5 * es);
    const size_t o_l0 = take(h->f_bytes), o_l1 = take(h->f_bytes), o_lu = take(nu * 32), o_lur = take(nu * 4 * es),
                 o_y = take(2 * 4 * nu * 4 * es), o_ly = take(5 * nu * 4 * es),   // lY[0..3], then lV
                 o_v = take(2 * nu * 4 * es), o_mask = take(2 * nu * sizeof(int)), o_lst = take(ns * 4 * es),
                 o_lst1 = take(ns * 4 * es), o_ln = take(ns * 5 * es), o_e0 = take(ns * 9 * es),
                 o_e1 = take(ns * 9 * es), o_sums = take(8 * sizeof(double)), o_cp = take(16 * 9 * sizeof(double)),
                 o_ck = take((size_t)nckpt * h->adj_ckpt_bytes);
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, o);
    if (e != cudaSuccess) return cuda_fail(h, e, "reverse-mode gradient allocation");
    AdjState& A = h->adj;
    A = AdjState{};
    A.K = K;
    A.Mh = at<char>(mem, o_mh);
    A.Ubh = at<double>(mem, o_ubh);
    A.stUh = at<char>(mem, o_suh);
    A.stNh = at<char>(mem, o_snh);
    A.lpre[0] = at<char>(mem, o_l0);
    A.lpre[1] = at<char>(mem, o_l1);
    A.lU = at<double>(mem, o_lu);
    A.lUr = at<char>(mem, o_lur);
    const double rl[8] = {h->B.alpha_T, h->B.beta_P, h->B.t_inf, h->B.alpha_V,
                          h->B.pdev[0], h->B.pdev[1], h->B.pdev[2], h->B.pdev[3]};
    for (int q = 0; q < 8; ++q) {
        A.relax_d[q] = rl[q];
        A.relax_f[q] = float(rl[q]);
    }
    for (int b = 0; b < 2; ++b) {
        for (int q = 0; q < 4; ++q) A.sets[b].Y[q] = at<char>(mem, o_y + (b * 4 + q) * nu * 4 * es);
        A.sets[b].V = at<char>(mem, o_v + b * nu * 4 * es);
        A.sets[b].mask = at<int>(mem, o_mask + b * nu * sizeof(int));
    }
    for (int q = 0; q < 4; ++q) {
        A.Y[q] = A.sets[0].Y[q];
        A.lY[q] = at<char>(mem, o_ly + q * nu * 4 * es);
    }
    A.lV = at<char>(mem, o_ly + 4 * nu * 4 * es);
    A.V = A.sets[0].V;
    A.mask = A.sets[0].mask;
    A.lSt = at<char>(mem, o_lst);
    A.lSt1 = at<char>(mem, o_lst1);
    A.lN = at<char>(mem, o_ln);
    A.ext[0] = at<char>(mem, o_e0);
    A.ext[1] = at<char>(mem, o_e1);
    A.sums = at<double>(mem, o_sums);
    A.cpart = at<double>(mem, o_cp);
    h->adj_ckpt = at<char>(mem, o_ck);
    h->adj_mem = mem;
    h->adj_max = max_steps;
    h->adj_fwd_done = false;
    e = cudaStreamCreateWithFlags(&h->adj_sv, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->adj_sw, cudaStreamNonBlocking);
    for (int q = 0; q < 4 && e == cudaSuccess; ++q) e = cudaEventCreateWithFlags(&h->adj_ev[q], cudaEventDisableTiming);
    // everything but the checkpoints starts at zero
    if (e == cudaSuccess) e = cudaMemsetAsync(mem, 0, o_ck, h->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(h, e, "reverse-mode gradient state");
}

int lbm_adj_forward(lbm_handle* h, int n, const double* dP_ref, long long ref_stride, double* J)
{
    if (!h || !J) return LBM_ERR_ARG;
    if (!h->adj_mem) { h->err = "lbm_adj_forward before lbm_adj_begin"; return LBM_ERR_STATE; }
    if (n < 1 || n > h->adj_max) { h->err = fmt("step count %d outside [1, %d]", n, h->adj_max); return LBM_ERR_ARG; }
    if (h->bulk_pending) { h->err = "lbm_adj_forward in the middle of a step"; return LBM_ERR_STATE; }
    const int K = h->adj.K;
    cudaError_t e = cudaMemsetAsync(h->adj.sums, 0, 8 * sizeof(double), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "loss reset");
    h->adj_start = h->steps;
    const size_t nu = (size_t)h->B.n_unk, ns = (size_t)h->E.nslots, es = h->E.sesize;
    int rc = adj_copy_state(h, 0, true);
    if (rc == LBM_OK) rc = adj_snapshot(h, h->adj, 0);
    for (int i = 0; i < n && rc == LBM_OK; ++i) {
        if (i > 0 && i % K == 0) rc = adj_copy_state(h, i / K, true);
        if (rc == LBM_OK) rc = lbm_step(h, 1);
        // the loss after step i, and the boundary history of that time
        const int par = int(h->steps & 1);
        AdjRecord rec{h->B.Ub + par * nu * 4, h->adj.Ubh + (size_t)(i + 1) * nu * 4, (long long)(nu * 4),
                      static_cast<char*>(h->E.stripU) + par * ns * 4 * es,
                      static_cast<char*>(h->adj.stUh) + (size_t)(i + 1) * ns * 4 * es, (long long)(ns * 4),
                      static_cast<char*>(h->E.stripN) + par * ns * 5 * es,
                      static_cast<char*>(h->adj.stNh) + (size_t)(i + 1) * ns * 5 * es, (long long)(ns * 5)};
        if (rc == LBM_OK &&
            launch_adj_loss(h->lattice, h->storage, h->G, h->bulk, h->f[par],
                            dP_ref ? dP_ref + (long long)i * ref_stride : nullptr, h->adj.sums, nullptr, rec,
                            h->stream))
            rc = check_launch(h, -1, "loss kernel");
    }
    if (rc != LBM_OK) return rc;
    rc = adj_copy_state(h, (n + K - 1) / K, true);       // the end state
    if (rc != LBM_OK) return rc;
    h->adj_n = n;
    h->adj_ref = dP_ref;
    h->adj_ref_stride = ref_stride;
    h->adj_fwd_done = true;
    e = cudaMemcpyAsync(J, h->adj.sums, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? LBM_OK : cuda_fail(h, e, "loss");
}

int lbm_adj_backward(lbm_handle* h, double* dJ)
{
    if (!h || !dJ) return LBM_ERR_ARG;
    if (!h->adj_mem || !h->adj_fwd_done) { h->err = "lbm_adj_backward before lbm_adj_forward"; return LBM_ERR_STATE; }
    AdjState& A = h->adj;
    const int K = A.K, n = h->adj_n, nseg = (n + K - 1) / K;
    const size_t N = (size_t)h->nx * h->ny, nu = (size_t)std::max(1, h->B.n_unk),
                 ns = (size_t)std::max(1, h->E.nslots), es = h->E.sesize;
    // adjoint variables start at zero
    cudaError_t e = cudaSuccess;
    void* zero[] = {A.lpre[0], A.lpre[1], A.lU, A.lUr, A.lSt, A.lSt1, A.lN, A.ext[0], A.ext[1]};
    const size_t zbytes[] = {h->f_bytes, h->f_bytes, nu * 32, nu * 4 * es, ns * 4 * es, ns * 4 * es, ns * 5 * es,
                             ns * 9 * es, ns * 9 * es};
    for (int q = 0; q < 9 && e == cudaSuccess; ++q) e = cudaMemsetAsync(zero[q], 0, zbytes[q], h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.sums + 1, 0, 7 * sizeof(double), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint reset");
    cudaStream_t sr = h->stream, sv = h->adj_sv, sw = h->adj_sw;
    cudaEvent_t ev_step = h->adj_ev[0], ev_bulk = h->adj_ev[1], ev_rc = h->adj_ev[2], ev_rev = h->adj_ev[3];
    // the reverse streams start after the resets
    e = cudaEventRecord(ev_step, sr);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sv, ev_step, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint streams");
    const size_t ub = nu * 4, su = ns * 4 * es, sn = ns * 5 * es;
    // Recompute the populations of segment seg from its checkpoint (on the
    // handle's stream) and keep the bulk macros of every step in history
    // buffer seg & 1: the bulk kernel of the ordinary step, then the
    // Dirichlet write from the recorded boundary state (the boundary ODE is
    // not solved again: its states and strips were recorded by the forward
    // pass).
    auto recompute = [&](int seg) -> int {
        const AdjState H = adj_hist(h, seg & 1);
        const int L = std::min(K, n - seg * K);
        h->steps = h->adj_start + (long long)seg * K;
        int rc = adj_copy_state(h, seg, false);
        for (int k = 0; k < L && rc == LBM_OK; ++k) {
            const int par = int(h->steps & 1);
            rc = bulk(h, par, sr);
            if (rc == LBM_OK &&
                launch_adj_dwrite(h->lattice, h->storage, h->G, h->B, A.Ubh + (size_t)(seg * K + k + 1) * nu * 4,
                                  h->f[par ^ 1], sr))
                rc = check_launch(h, -1, "Dirichlet write");
            if (rc == LBM_OK && launch_adj_loss(h->lattice, h->storage, h->G, h->bulk, h->f[par ^ 1], nullptr,
                                                nullptr, static_cast<char*>(H.Mh) + (size_t)k * 4 * N * es,
                                                AdjRecord{}, sr))
                rc = check_launch(h, -1, "macros kernel");
            h->steps++;
        }
        return rc;
    };
    int rc = recompute(nseg - 1);
    for (int seg = nseg - 1; seg >= 0 && rc == LBM_OK; --seg) {
        // the reverse steps of seg wait for its recompute
        e = cudaEventRecord(ev_rc, sr);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sv, ev_rc, 0);
        if (e != cudaSuccess) { rc = cuda_fail(h, e, "adjoint streams"); break; }
        const AdjState H = adj_hist(h, seg & 1);
        const long long t0 = h->adj_start + (long long)seg * K;
        const int L = std::min(K, n - seg * K);
        for (int k = L - 1; k >= 0 && rc == LBM_OK; --k) {
            const long long t = t0 + k;
            const size_t r = (size_t)seg * K + k;      // the step within the run
            const double* ref = h->adj_ref ? h->adj_ref + (t - h->adj_start) * h->adj_ref_stride : nullptr;
            e = cudaEventRecord(ev_step, sv);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(sw, ev_step, 0);
            if (e != cudaSuccess) { rc = cuda_fail(h, e, "adjoint streams"); break; }
            // the stage fields of step r were computed by the reverse step of
            // r + 1 unless r is the last step; those of r - 1 are computed now
            const int pre = r + 1 < (size_t)n, nxt = r > 0;
            const size_t rm = nxt ? r - 1 : r;
            if (launch_adj_step(h->lattice, h->storage, h->G, h->E, h->B, h->bulk, A, A.Ubh + r * ub,
                                A.Ubh + (r + 1) * ub, static_cast<char*>(A.stUh) + r * su,
                                static_cast<char*>(A.stNh) + r * sn, static_cast<char*>(A.stUh) + (r + 1) * su,
                                static_cast<char*>(H.Mh) + (size_t)k * 4 * N * es, ref, int(t & 1), int(r & 1),
                                pre, nxt, A.Ubh + rm * ub, static_cast<char*>(A.stUh) + rm * su,
                                static_cast<char*>(A.stNh) + rm * sn, sv, sw, ev_bulk))
                rc = check_launch(h, -1, "reverse step");
        }
        // meanwhile the previous segment's recompute, into the other buffer
        // once the reverse steps that read it (segment seg + 1) are done
        if (rc == LBM_OK && seg > 0) {
            e = cudaStreamWaitEvent(sr, ev_rev, 0);
            if (e != cudaSuccess) { rc = cuda_fail(h, e, "adjoint streams"); break; }
            rc = recompute(seg - 1);
        }
        if (rc == LBM_OK) {
            e = cudaEventRecord(ev_rev, sv);
            if (e != cudaSuccess) rc = cuda_fail(h, e, "adjoint streams");
        }
    }
    // back to the state after the forward pass, after the last reverse step
    if (rc == LBM_OK) {
        e = cudaEventRecord(ev_step, sv);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sr, ev_step, 0);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "adjoint streams");
    }
    h->steps = h->adj_start + n;
    if (rc == LBM_OK) rc = adj_copy_state(h, nseg, false);
    if (rc != LBM_OK) {
        cudaStreamSynchronize(sv);
        cudaStreamSynchronize(sw);
        return rc;
    }
    double v[8];
    e = cudaMemcpyAsync(v, A.sums, sizeof v, cudaMemcpyDeviceToHost, sr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sr);
    if (e != cudaSuccess) return cuda_fail(h, e, "reverse sweep");
    for (int k = 0; k < kTLParams; ++k) dJ[k] = v[1 + k];
    return LBM_OK;
}

namespace {
void adj_release(lbm_handle* h)
{
    if (h->adj_sv) cudaStreamSynchronize(h->adj_sv);
    if (h->adj_sw) cudaStreamSynchronize(h->adj_sw);
    for (int q = 0; q < 4; ++q)
        if (h->adj_ev[q]) cudaEventDestroy(h->adj_ev[q]);
    if (h->adj_sv) cudaStreamDestroy(h->adj_sv);
    if (h->adj_sw) cudaStreamDestroy(h->adj_sw);
    h->adj_sv = h->adj_sw = nullptr;
    for (int q = 0; q < 4; ++q) h->adj_ev[q] = nullptr;
}
}  // namespace

int lbm_adj_end(lbm_handle* h)
{
    if (!h) return LBM_ERR_ARG;
    if (!h->adj_mem) return LBM_OK;
    cudaError_t e = h->stream ? cudaStreamSynchronize(h->stream) : cudaDeviceSynchronize();
    adj_release(h);
    cudaFree(h->adj_mem);
    h->adj_mem = nullptr;
    h->adj = AdjState{};
    h->adj_ckpt = nullptr;
    h->adj_fwd_done = false;
    return e == cudaSuccess ? LBM_OK : cuda_fail(h, e, "reverse-mode gradient release");
}

const char* lbm_last_error(const lbm_handle* h) { return h ? h->err.c_str() : "NULL handle"; }

void lbm_destroy(lbm_handle* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    release_streams(h);
    if (h->tl_mem) cudaFree(h->tl_mem);
    if (h->adj_mem) {
        adj_release(h);
        cudaFree(h->adj_mem);
    }
    if (h->owns_ws && h->ws) cudaFree(h->ws);
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many independent runs stepped together
// ---------------------------------------------------------------------------

struct lbm_batch {
    int n = 0;
    std::vector<lbm_handle*> runs;
    struct Group {
        int lattice = 0, storage = 0;
        std::vector<int> members;          // run indices
        BulkRun* bulk = nullptr;           // device: one per member
        int total_items = 0, grid = 0, ctas_per_sm = 0;
        BandRun* band = nullptr;           // device: one per member
        int2* tile_run = nullptr;          // device: (member, tile) per band tile
        unsigned* queue = nullptr;         // device: work queue of the persistent bulk kernel
        int n_tiles = 0;
        size_t band_smem = 0;
    };
    std::vector<Group> groups;
    void* dev = nullptr;                   // the groups' descriptor arrays
    cudaStream_t stream = nullptr, cap = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool tuned = false;
    int nsm = 0;
    long long steps = 0;
    std::string err;
};

namespace {

int batch_fail(lbm_batch* b, cudaError_t e, const char* what)
{
    b->err = fmt("%s: %s", what, cudaGetErrorString(e));
    return LBM_ERR_CUDA;
}

// Autotuned CTAs per SM of the persistent bulk kernel, cached in a text file
// (LBM_AUTOTUNE_CACHE, default ~/.cache/lbm_cbc_autotune.txt; empty = off):
// one line "device lattice storage bucket ctas_per_sm" per tuned case, the
// bucket being log2 of the group's work items.
std::string autotune_path()
{
    const char* p = getenv("LBM_AUTOTUNE_CACHE");
    if (p) return p;
    const char* home = getenv("HOME");
    return home ? std::string(home) + "/.cache/lbm_cbc_autotune.txt" : std::string();
}

std::string autotune_key(int lattice, int storage, int items)
{
    int dev = 0;
    cudaDeviceProp prop;
    std::memset(&prop, 0, sizeof prop);
    if (cudaGetDevice(&dev) == cudaSuccess) cudaGetDeviceProperties(&prop, dev);
    std::string name = prop.name;
    for (char& c : name)
        if (c == ' ') c = '_';
    int bucket = 0;
    while ((1 << bucket) < items) ++bucket;
    return fmt("%s %d %d %d", name.c_str(), lattice, storage, bucket);
}

int autotune_lookup(const std::string& key)
{
    const std::string path = autotune_path();
    if (path.empty()) return 0;
    FILE* fp = fopen(path.c_str(), "r");
    if (!fp) return 0;
    char line[512];
    int found = 0;
    while (fgets(line, sizeof line, fp)) {
        std::string l(line);
        const size_t sp = l.find_last_of(' ');
        if (sp == std::string::npos) continue;
        if (l.compare(0, sp, key) == 0) found = atoi(l.c_str() + sp + 1);   // last entry wins
    }
    fclose(fp);
    return found >= 1 && found <= 8 ? found : 0;
}

void autotune_store(const std::string& key, int value)
{
    const std::string path = autotune_path();
    if (path.empty()) return;
    const size_t slash = path.find_last_of('/');
    if (slash != std::string::npos) {
        const std::string dir = path.substr(0, slash);
        for (size_t i = 1; i <= dir.size(); ++i)        // mkdir -p
            if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
    }
    FILE* fp = fopen(path.c_str(), "a");
    if (!fp) return;
    fprintf(fp, "%s %d\n", key.c_str(), value);
    fclose(fp);
}

// One step of every run: per group one batched band launch and one
// persistent bulk launch, then the zero-gradient copies, on the batch's
// stream.
int batch_issue_step(lbm_batch* b, int par, cudaStream_t s0, bool with_inflow)
{
    // All on one stream: the band kernels of the groups, then their bulk
    // kernels, each after the first with early start (every kernel here
    // signals its dependents at once; none reads what another writes), so
    // all run side by side; the zero-gradient copies and the next step
    // wait for all of them.
    // inflow equilibria (once per buffer) ahead of the fork, so that every
    // kernel of the step comes after them
    if (with_inflow)
        for (lbm_handle* h : b->runs)
            if (h->n_inflow > 0 && !h->inflow_done[par ^ 1]) {
                if (launch_inflow(h->lattice, h->storage, h->G, h->inflow_nodes, h->n_inflow, h->Uin,
                                  h->f[par ^ 1], s0))
                    return batch_fail(b, cudaGetLastError(), "inflow kernel");
                h->inflow_done[par ^ 1] = true;
            }
    bool first = true;
    for (auto& g : b->groups) {
        if (g.n_tiles == 0) continue;
        if (launch_band_batch(g.lattice, g.storage, g.band, g.tile_run, g.n_tiles, g.band_smem, par, s0,
                              !first))
            return batch_fail(b, cudaGetLastError(), "batched band kernel");
        first = false;
    }
    for (auto& g : b->groups) {
        if (launch_bulk_persistent(g.lattice, g.storage, g.bulk, int(g.members.size()), g.total_items, par,
                                   g.grid, g.queue, s0, !first))
            return batch_fail(b, cudaGetLastError(), "persistent bulk kernel");
        first = false;
    }
    for (lbm_handle* h : b->runs)
        if (h->B.n_zg > 0 && launch_zg(h->lattice, h->storage, h->G, h->B, h->f[par ^ 1], s0))
            return batch_fail(b, cudaGetLastError(), "zero-gradient kernel");
    return LBM_OK;
}

// Pick the persistent bulk kernel's CTAs per SM for each group: the fastest
// of 1..5 over three timed launches each (the launches rewrite the new
// buffer from the current one, which the following step rewrites again).
int batch_autotune(lbm_batch* b)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return batch_fail(b, e, "autotune events");
    const int par = int(b->steps & 1);
    for (auto& g : b->groups) {
        const std::string key = autotune_key(g.lattice, g.storage, g.total_items);
        int best = autotune_lookup(key);
        if (!best) {
            float best_ms = 1e30f;
            for (int m = 1; m <= 5; ++m) {
                const int grid = b->nsm * m;
                launch_bulk_persistent(g.lattice, g.storage, g.bulk, int(g.members.size()), g.total_items, par,
                                       grid, g.queue, b->stream);        // warm-up
                cudaEventRecord(e0, b->stream);
                for (int r = 0; r < 3; ++r)
                    launch_bulk_persistent(g.lattice, g.storage, g.bulk, int(g.members.size()), g.total_items,
                                           par, grid, g.queue, b->stream);
                cudaEventRecord(e1, b->stream);
                e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return batch_fail(b, e, "autotune");
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_ms) { best_ms = ms; best = m; }
            }
            autotune_store(key, best);
        }
        g.ctas_per_sm = best;
        g.grid = b->nsm * best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuned = true;
    return LBM_OK;
}

void batch_release(lbm_batch* b)
{
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    for (int k = 0; k < 2; ++k)
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->dev) cudaFree(b->dev);
    for (lbm_handle* h : b->runs) lbm_destroy(h);
    delete b;
}

}  // namespace

extern "C" {

int lbm_batch_create(int n, const int* lattice, const int* nx, const int* ny, const double* tau,
                     const lbm_cbc_params* params, lbm_batch** out)
{
    if (!out || n < 1 || !lattice || !nx || !ny || !tau || !params) return LBM_ERR_ARG;
    *out = nullptr;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_ALLOC;
    b->n = n;
    for (int r = 0; r < n; ++r) {
        lbm_handle* h = nullptr;
        if (params[r].u_ref[0] != 0.0 || params[r].u_ref[1] != 0.0) {
            fprintf(stderr, "lbm_batch_create: run %d has u_ref != 0 (batches hold the plain shift)\n", r);
            batch_release(b);
            return LBM_ERR_ARG;
        }
        const int rc = lbm_create(lattice[r], nx[r], ny[r], tau[r], params + r, &h);
        if (rc != LBM_OK) {
            fprintf(stderr, "lbm_batch_create: run %d rejected\n", r);
            batch_release(b);
            return rc;
        }
        b->runs.push_back(h);
    }
    // groups by lattice and storage
    for (int r = 0; r < n; ++r) {
        lbm_handle* h = b->runs[r];
        lbm_batch::Group* g = nullptr;
        for (auto& x : b->groups)
            if (x.lattice == h->lattice && x.storage == h->storage) g = &x;
        if (!g) {
            b->groups.emplace_back();
            g = &b->groups.back();
            g->lattice = h->lattice;
            g->storage = h->storage;
        }
        g->members.push_back(r);
    }
    // descriptor arrays (host copies, then one device allocation)
    std::vector<std::vector<BulkRun>> bulk(b->groups.size());
    std::vector<std::vector<BandRun>> band(b->groups.size());
    std::vector<std::vector<int2>> tiles(b->groups.size());
    size_t bytes = 0;
    std::vector<size_t> off_bulk, off_band, off_tiles, off_queue;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        auto& g = b->groups[gi];
        if ((int)g.members.size() > kMaxBatchRuns) {
            fprintf(stderr, "lbm_batch_create: more than %d runs of one lattice and storage\n", kMaxBatchRuns);
            batch_release(b);
            return LBM_ERR_ARG;
        }
        int first = 0;
        for (size_t k = 0; k < g.members.size(); ++k) {
            lbm_handle* h = b->runs[g.members[k]];
            BulkRun r;
            const cudaError_t e = cudaMemcpy(&r, h->brun, sizeof r, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                fprintf(stderr, "lbm_batch_create: %s\n", cudaGetErrorString(e));
                batch_release(b);
                return LBM_ERR_CUDA;
            }
            r.first = first;
            first += h->bulk_items;
            bulk[gi].push_back(r);
            BandRun br;
            std::memset(&br, 0, sizeof br);
            br.G = h->G;
            br.O = h->O;
            br.B = h->B;
            br.E = h->E;
            br.f[0] = h->f[0];
            br.f[1] = h->f[1];
            band[gi].push_back(br);
            for (int t = 0; t < h->B.n_tiles; ++t) tiles[gi].push_back(make_int2(int(k), t));
            g.band_smem = std::max(g.band_smem, band_dynamic_smem(h->lattice, h->storage, h->B));
        }
        g.total_items = first;
        g.n_tiles = int(tiles[gi].size());
        off_bulk.push_back(bytes);
        bytes = align_up(bytes + bulk[gi].size() * sizeof(BulkRun));
        off_band.push_back(bytes);
        bytes = align_up(bytes + band[gi].size() * sizeof(BandRun));
        off_tiles.push_back(bytes);
        bytes = align_up(bytes + std::max<size_t>(1, tiles[gi].size()) * sizeof(int2));
        off_queue.push_back(bytes);
        bytes = align_up(bytes + 2 * sizeof(unsigned));
    }
    cudaError_t e = cudaMalloc(&b->dev, bytes);
    for (size_t gi = 0; e == cudaSuccess && gi < b->groups.size(); ++gi) {
        auto& g = b->groups[gi];
        g.bulk = at<BulkRun>(b->dev, off_bulk[gi]);
        g.band = at<BandRun>(b->dev, off_band[gi]);
        g.tile_run = at<int2>(b->dev, off_tiles[gi]);
        g.queue = at<unsigned>(b->dev, off_queue[gi]);
        e = cudaMemcpy(g.bulk, bulk[gi].data(), bulk[gi].size() * sizeof(BulkRun), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(g.band, band[gi].data(), band[gi].size() * sizeof(BandRun), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(g.queue, 0, 2 * sizeof(unsigned));
        if (e == cudaSuccess && !tiles[gi].empty())
            e = cudaMemcpy(g.tile_run, tiles[gi].data(), tiles[gi].size() * sizeof(int2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && prepare_bulk_persistent(g.lattice, g.storage)) e = cudaGetLastError();
        if (e == cudaSuccess && prepare_band_batch(g.lattice, g.storage, g.band_smem)) e = cudaGetLastError();
    }
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    for (auto& g : b->groups) g.grid = b->nsm * 4;               // until tuned

    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        fprintf(stderr, "lbm_batch_create: %s\n", cudaGetErrorString(e));
        batch_release(b);
        return LBM_ERR_CUDA;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_run(lbm_batch* b, int run, lbm_handle** h)
{
    if (!b || !h || run < 0 || run >= b->n) return LBM_ERR_ARG;
    *h = b->runs[run];
    return LBM_OK;
}

int lbm_batch_set_stream(lbm_batch* b, void* stream)
{
    if (!b) return LBM_ERR_ARG;
    b->stream = static_cast<cudaStream_t>(stream);
    for (lbm_handle* h : b->runs) h->stream = b->stream;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int n)
{
    if (!b || n < 0) return LBM_ERR_ARG;
    for (lbm_handle* h : b->runs) {
        if (!h->initialized) { b->err = "lbm_batch_step before every run's lbm_init_fields"; return LBM_ERR_STATE; }
        if (h->steps != b->runs[0]->steps) { b->err = "runs of a batch stepped apart"; return LBM_ERR_STATE; }
        if (h->grad_stale) { b->err = kGradStale; return LBM_ERR_STATE; }
    }
    b->steps = b->runs[0]->steps;
    if (n > 0 && !b->tuned) {
        const int rc = batch_autotune(b);
        if (rc != LBM_OK) return rc;
    }
    for (int i = 0; i < n; ++i) {
        const int par = int(b->steps & 1);
        bool eager = false;
        for (lbm_handle* h : b->runs)
            if (h->n_inflow > 0 && !(h->inflow_done[0] && h->inflow_done[1])) eager = true;
        if (eager) {
            const int rc = batch_issue_step(b, par, b->stream, true);
            if (rc != LBM_OK) return rc;
        } else {
            if (!b->graph[par]) {
                // capture this parity's step once on an internal stream
                cudaGraph_t gr = nullptr;
                cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) return batch_fail(b, e, "capture");
                const int rc = batch_issue_step(b, par, b->cap, false);
                e = cudaStreamEndCapture(b->cap, &gr);
                if (rc != LBM_OK) return rc;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[par], gr, 0);
                if (gr) cudaGraphDestroy(gr);
                if (e != cudaSuccess) return batch_fail(b, e, "graph");
            }
            const cudaError_t e = cudaGraphLaunch(b->graph[par], b->stream);
            if (e != cudaSuccess) return batch_fail(b, e, "graph launch");
        }
        b->steps++;
        for (lbm_handle* h : b->runs) h->steps++;
    }
    return LBM_OK;
}

int lbm_batch_ctas_per_sm(const lbm_batch* b, int lattice, int storage)
{
    if (!b) return LBM_ERR_ARG;
    for (const auto& g : b->groups)
        if (g.lattice == lattice && g.storage == storage) return g.ctas_per_sm;
    return 0;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : "NULL batch"; }

int lbm_fp64_fma_rate(int iters, void* stream, double* flops_per_s)
{
    if (!flops_per_s || iters < 1 || iters > (1 << 24)) return LBM_ERR_ARG;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = sms * kFmaCtasPerSm;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    float ms = 0.0f;
    if (e == cudaSuccess) {
        k_fp64_fma<<<grid, kFmaThreads, 0, st>>>(nullptr, 64, -1.0);   // warm-up
        cudaEventRecord(ev[0], st);
        k_fp64_fma<<<grid, kFmaThreads, 0, st>>>(nullptr, iters, -1.0);
        cudaEventRecord(ev[1], st);
        e = cudaEventSynchronize(ev[1]);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess || !(ms > 0.0f)) return LBM_ERR_CUDA;
    *flops_per_s = 2.0 * kFmaChains * double(grid) * kFmaThreads * iters / (ms * 1e-3);
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b)
{
    if (b) batch_release(b);
}

}  // extern "C"
