// a8: batched ensembles of uneven Navier-Stokes runs in one set of launches.
//
// Every member is built like a single problem (its own stencil size,
// polynomial degree, spacing, time step and boundary systems).  The members'
// states are concatenated as node-major records.  One RK4 stage for the
// whole ensemble is three launches: the merged ghost residual, the merged
// ghost solve, and one stage kernel whose thread blocks each read a block
// descriptor (the member's operand arrays, its slice of nodes, its operand
// width and its dt): a SELL-C layout with one slice per block.  Members are
// ordered by descending step count, so the members still running at any
// global step form a prefix of the blocks and of the ghost rows; the
// ensemble runs in phases of constant active prefix, each replayed from a
// captured CUDA graph.  No device-side waits are involved.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "problem.cuh"
#include "records.cuh"

namespace rbf {

namespace {

template <class T>
struct BlockDesc {
    const int32_t *pidx;
    const T *wx, *wz, *wd, *wh;
    const T *pibar;
    const unsigned char *flags;
    const int32_t *lcls, *loff;   // member's lattice storage (null: per-node rows only)
    const T *lw;
    int64_t n_prog;   // member's prognostic nodes (operand stride, node bound)
    int64_t rec0;     // member's first record in the concatenated state
    int32_t node0;    // first member node of this block
    int32_t SLQ;      // operand vectors per lane
    int32_t n_cls;    // member's lattice classes
    double dt;
};

template <class T>
struct EnsArgs {
    const T *Uin, *Un;
    T *Uout, *K;      // K indexed by state record
    int stage;
    double cA, cB;    // RK4 stage coefficients, scaled by each member's dt
    T cp, g_over_tb, theta_bar, dpibar, rd_cv;
};

template <class T>
struct VecE;
template <>
struct VecE<float> {
    static constexpr int V = 4;
    using W = float4;
    using I = int4;
    __device__ static float at(const float4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
    __device__ static int at(const int4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
    __device__ static int4 shift(const int4 &v, int d) { return make_int4(v.x + d, v.y + d, v.z + d, v.w + d); }
};
template <>
struct VecE<double> {
    static constexpr int V = 2;
    using W = double2;
    using I = int2;
    __device__ static double at(const double2 &v, int k) { return k == 0 ? v.x : v.y; }
    __device__ static int at(const int2 &v, int k) { return k == 0 ? v.x : v.y; }
    __device__ static int2 shift(const int2 &v, int d) { return make_int2(v.x + d, v.y + d); }
};

// The stage kernel of Eqs. (uEq)-(piEq) with the RK4 update, for a block of
// one ensemble member (same arithmetic and operand order as the single-problem
// stage kernel with streamed operands).  LAT: members with lattice storage
// take a class node's operands from the member's class table.
template <class T, int G, bool DIFF, bool LAT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 3) ens_stage_kernel(const BlockDesc<T> *__restrict__ descs, EnsArgs<T> a) {
    using VT = VecE<T>;
    using W = typename VT::W;
    using I = typename VT::I;
    constexpr int V = VT::V;
    const BlockDesc<T> d = descs[blockIdx.x];
    const int g = threadIdx.x % G;
    int64_t i = d.node0 + threadIdx.x / G;
    const bool live = i < d.n_prog;
    if (!live) i = d.n_prog - 1;
    const int64_t stride = d.n_prog * G;
    const int64_t off0 = i * G + g;
    const I *pidx = reinterpret_cast<const I *>(d.pidx);
    const W *wx = reinterpret_cast<const W *>(d.wx), *wz = reinterpret_cast<const W *>(d.wz);
    const W *wd = reinterpret_cast<const W *>(d.wd), *wh = reinterpret_cast<const W *>(d.wh);
    grid_dep_wait();
    grid_dep_launch();
    const T *U = a.Uin + d.rec0 * 4;   // member-local record indices from here on
    Rec<T> fi = {0, 0, 0, 0};
    if (DIFF) fi = load_rec(U, i);
    T ux = 0, uz = 0, ud = 0, wx_ = 0, wz_ = 0, wd_ = 0, tx = 0, tz = 0, td = 0, px = 0, pz = 0, ph = 0;
    auto vec = [&](const I &jv, const W &cx, const W &cz, const W &cd, const W &ch) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            Rec<T> r = load_rec(U, VT::at(jv, v));
            if (DIFF) { r.u -= fi.u; r.w -= fi.w; r.t -= fi.t; r.p -= fi.p; }
            const T x = VT::at(cx, v), z = VT::at(cz, v), dd = VT::at(cd, v), h = VT::at(ch, v);
            ux += x * r.u; uz += z * r.u; ud += dd * r.u;
            wx_ += x * r.w; wz_ += z * r.w; wd_ += dd * r.w;
            tx += x * r.t; tz += z * r.t; td += dd * r.t;
            px += x * r.p; pz += z * r.p; ph += h * r.p;
        }
    };
    const int cl = (LAT && d.lcls) ? __ldg(d.lcls + i) : -1;
    if (LAT && cl >= 0) {
        const I *lo = reinterpret_cast<const I *>(d.loff);
        const W *lw = reinterpret_cast<const W *>(d.lw);
        const int64_t ls = (int64_t)d.n_cls * d.SLQ * G;   // in vectors, between operators
        int64_t off = (int64_t)cl * d.SLQ * G + g;
#pragma unroll 2
        for (int q = 0; q < d.SLQ; ++q, off += G)
            vec(VT::shift(__ldg(lo + off), (int)i), __ldg(lw + off), __ldg(lw + ls + off), __ldg(lw + 2 * ls + off),
                __ldg(lw + 3 * ls + off));
    } else {
        int64_t off = off0;
#pragma unroll 2
        for (int q = 0; q < d.SLQ; ++q, off += stride)
            vec(__ldg(pidx + off), __ldg(wx + off), __ldg(wz + off), __ldg(wd + off), __ldg(wh + off));
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        ux += __shfl_xor_sync(0xffffffffu, ux, o, G);
        uz += __shfl_xor_sync(0xffffffffu, uz, o, G);
        ud += __shfl_xor_sync(0xffffffffu, ud, o, G);
        wx_ += __shfl_xor_sync(0xffffffffu, wx_, o, G);
        wz_ += __shfl_xor_sync(0xffffffffu, wz_, o, G);
        wd_ += __shfl_xor_sync(0xffffffffu, wd_, o, G);
        tx += __shfl_xor_sync(0xffffffffu, tx, o, G);
        tz += __shfl_xor_sync(0xffffffffu, tz, o, G);
        td += __shfl_xor_sync(0xffffffffu, td, o, G);
        px += __shfl_xor_sync(0xffffffffu, px, o, G);
        pz += __shfl_xor_sync(0xffffffffu, pz, o, G);
        ph += __shfl_xor_sync(0xffffffffu, ph, o, G);
    }
    if (!live) return;
    const Rec<T> c = DIFF ? fi : load_rec(U, i);
    const unsigned char fl = d.flags[i];
    const T cpth = a.cp * (a.theta_bar + c.t);
    T k[4];
    k[0] = -c.u * ux - c.w * uz - cpth * px + ud;
    k[1] = -c.u * wx_ - c.w * wz_ - cpth * pz + a.g_over_tb * c.t + wd_;
    k[2] = -c.u * tx - c.w * tz + td;
    k[3] = -c.u * px - c.w * (a.dpibar + pz) - a.rd_cv * (d.pibar[i] + c.p) * (ux + wz_) + ph;
    if (fl & 1) k[1] = 0;
    if (fl & 2) k[0] = 0;
    const T an = (T)(a.cA * d.dt), bs = (T)(a.cB * d.dt);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (f % G != g) continue;
        const T kf = k[f];
        const int64_t e = (d.rec0 + i) * 4 + f;
        const T un = a.Un[e];
        if (a.stage == 0) {
            a.K[e] = bs * kf;
            a.Uout[e] = un + an * kf;
        } else if (a.stage < 3) {
            a.K[e] += bs * kf;
            a.Uout[e] = un + an * kf;
        } else {
            a.Uout[e] = un + (a.K[e] + bs * kf);
        }
    }
}

const double kA[4] = {0.5, 0.5, 1.0, 0.0};
const double kB[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

template <class T>
void fill_descs(Problem &pb) {
    EnsembleState &E = *pb.ens;
    const int C = 256 / pb.G;
    std::vector<BlockDesc<T>> h;
    E.blocks_before.assign(1, 0);
    for (int oi : E.order) {
        Problem &m = *E.members[oi];
        const int64_t total = (int64_t)m.SL * m.G * m.n_prog;
        const T *pw = (const T *)m.pw.p;
        for (int64_t n0 = 0; n0 < m.n_prog; n0 += C) {
            BlockDesc<T> d{};
            d.pidx = m.pidx.p;
            d.wx = pw;
            d.wz = pw + total;
            d.wd = pw + 2 * total;
            d.wh = pw + 3 * total;
            d.pibar = (const T *)m.pibar.p;
            d.flags = m.flags.p;
            if (m.lat.enabled) {
                d.lcls = m.lat.cls.p;
                d.loff = m.lat.loff.p;
                d.lw = (const T *)m.lat.lw.p;
                d.n_cls = m.lat.n_cls;
            }
            d.n_prog = m.n_prog;
            d.rec0 = E.rec0[oi];
            d.node0 = (int32_t)n0;
            d.SLQ = m.SLQ;
            d.dt = E.dt[oi];
            h.push_back(d);
        }
        E.blocks_before.push_back((int64_t)h.size());
    }
    E.descs.alloc(h.size() * sizeof(BlockDesc<T>));
    RBF_CUDA(cudaMemcpyAsync(E.descs.p, h.data(), E.descs.bytes(), cudaMemcpyHostToDevice, pb.st));
    RBF_CUDA(cudaStreamSynchronize(pb.st));
}

template <class T, int G>
void launch_ens(Problem &pb, const EnsArgs<T> &a, int64_t nblocks, cudaStream_t s, bool pdl) {
    constexpr bool kDiff = sizeof(T) == 4;
    if (pb.lat.enabled)
        launch_kernel(ens_stage_kernel<T, G, kDiff, true>, dim3((unsigned)nblocks), dim3(256), s, pdl,
                      (const BlockDesc<T> *)pb.ens->descs.p, a);
    else
        launch_kernel(ens_stage_kernel<T, G, kDiff, false>, dim3((unsigned)nblocks), dim3(256), s, pdl,
                      (const BlockDesc<T> *)pb.ens->descs.p, a);
}

template <class T>
void ens_step(Problem &pb, T *U, cudaStream_t s, bool rec, int step) {
    EnsembleState &E = *pb.ens;
    const int64_t nb = E.blocks_before[E.active_members];
    pb.gh.rows = E.rows_before[E.active_members];
    EnsArgs<T> a{};
    T *S0 = (T *)pb.S0.p, *S1 = (T *)pb.S1.p;
    T *in[4] = {U, S0, S1, S0};
    T *out[4] = {S0, S1, S0, U};
    a.Un = U;
    a.K = (T *)pb.K.p;
    a.cp = (T)pb.cp;
    a.g_over_tb = (T)(pb.g / pb.theta_bar);
    a.theta_bar = (T)pb.theta_bar;
    a.dpibar = (T)(-pb.g / (pb.cp * pb.theta_bar));
    a.rd_cv = (T)(pb.rd / pb.cv);
    for (int st = 0; st < 4; ++st) {
        enqueue_ghost_fill(pb, in[st], s);
        a.Uin = in[st];
        a.Uout = out[st];
        a.stage = st;
        a.cA = kA[st];
        a.cB = kB[st];
        if (rec) RBF_CUDA(cudaEventRecordWithFlags(pb.rhs_ev[(step * 4 + st) * 2], s, cudaEventRecordExternal));
        const bool pdl = pb.pdl && !rec;
        switch (pb.G) {
            case 1: launch_ens<T, 1>(pb, a, nb, s, pdl); break;
            case 2: launch_ens<T, 2>(pb, a, nb, s, pdl); break;
            case 4: launch_ens<T, 4>(pb, a, nb, s, pdl); break;
            default: RBF_FAIL(RBF_E_ARG, "ensemble threads per node %d not in {1,2,4}", pb.G);
        }
        if (rec) RBF_CUDA(cudaEventRecordWithFlags(pb.rhs_ev[(step * 4 + st) * 2 + 1], s, cudaEventRecordExternal));
    }
}

// Concatenates the members' ghost plans (in run order) into pb.gh, with
// state records shifted by each member's record offset.
template <class T>
void merge_ghosts(Problem &pb) {
    EnsembleState &E = *pb.ens;
    GhostPlan &M = pb.gh;
    int npad = 0;
    int64_t ng = 0, ninv = 0;
    int nc = 0, ncl = -1;
    int fcl[4] = {0, 0, 0, 0};
    for (int oi : E.order) {
        GhostPlan &g = E.members[oi]->gh;
        RBF_REQUIRE(g.n_ghost > 0, "ensemble member %d has no ghost nodes", oi);
        npad = std::max(npad, g.npad);
        ng += g.n_ghost;
        nc += g.n_comp;
        ninv += (int64_t)(g.inv.bytes() / sizeof(T));
        if (ncl < 0) {
            ncl = g.n_class;
            memcpy(fcl, g.field_class, sizeof(fcl));
        }
        RBF_REQUIRE(ncl == g.n_class && !memcmp(fcl, g.field_class, sizeof(fcl)),
                    "ensemble members need the same boundary-operator classes");
    }
    std::vector<int32_t> gidx((size_t)ng * npad), owner(ng), pos(ng), comp_of(ng);
    std::vector<T> gw((size_t)4 * ng * npad, (T)0);
    std::vector<unsigned char> tb(ng);
    std::vector<int64_t> grec(ng), cstart(nc + 1), inv_off((size_t)ncl * nc);
    M.inv.alloc(ninv * sizeof(T));
    E.rows_before.assign(1, 0);
    int64_t r0 = 0, c0 = 0, i0 = 0;
    for (int oi : E.order) {
        Problem &m = *E.members[oi];
        GhostPlan &g = m.gh;
        const int64_t gn = g.n_ghost, rec0 = E.rec0[oi];
        const int gp = g.npad, gc = g.n_comp;
        std::vector<int32_t> hidx((size_t)gn * gp), how(gn), hpos(gn), hcomp(gn);
        std::vector<T> hw((size_t)4 * gn * gp);
        std::vector<unsigned char> htb(gn);
        std::vector<int64_t> hgrec(gn), hcs(gc + 1), hio((size_t)ncl * gc);
        RBF_CUDA(cudaMemcpy(hidx.data(), g.gidx.p, hidx.size() * 4, cudaMemcpyDeviceToHost));
        RBF_CUDA(cudaMemcpy(hw.data(), g.gw.p, hw.size() * sizeof(T), cudaMemcpyDeviceToHost));
        RBF_CUDA(cudaMemcpy(how.data(), g.owner.p, gn * 4, cudaMemcpyDeviceToHost));
        RBF_CUDA(cudaMemcpy(htb.data(), g.tb.p, gn, cudaMemcpyDeviceToHost));
        RBF_CUDA(cudaMemcpy(hpos.data(), g.pos.p, gn * 4, cudaMemcpyDeviceToHost));
        RBF_CUDA(cudaMemcpy(hcomp.data(), g.comp_of.p, gn * 4, cudaMemcpyDeviceToHost));
        RBF_CUDA(cudaMemcpy(hgrec.data(), g.grec.p, gn * 8, cudaMemcpyDeviceToHost));
        RBF_CUDA(cudaMemcpy(hcs.data(), g.comp_start.p, (gc + 1) * 8, cudaMemcpyDeviceToHost));
        RBF_CUDA(cudaMemcpy(hio.data(), g.inv_off.p, hio.size() * 8, cudaMemcpyDeviceToHost));
        RBF_REQUIRE(rec0 + m.n_all < ((int64_t)1 << 31), "ensemble exceeds int32 record indexing");
        for (int64_t r = 0; r < gn; ++r) {
            for (int k = 0; k < npad; ++k) {
                const bool in = k < gp;
                gidx[(size_t)(r0 + r) * npad + k] = (int32_t)(rec0 + (in ? hidx[(size_t)r * gp + k] : how[r]));
                for (int f = 0; f < 4; ++f)
                    gw[((size_t)f * ng + r0 + r) * npad + k] = in ? hw[((size_t)f * gn + r) * gp + k] : (T)0;
            }
            owner[r0 + r] = (int32_t)(rec0 + how[r]);
            tb[r0 + r] = htb[r];
            pos[r0 + r] = (int32_t)(r0 + hpos[r]);
        }
        for (int64_t q = 0; q < gn; ++q) {
            comp_of[r0 + q] = (int32_t)(c0 + hcomp[q]);
            grec[r0 + q] = rec0 + hgrec[q];
        }
        for (int c = 0; c < gc; ++c) cstart[c0 + c] = r0 + hcs[c];
        for (int cl = 0; cl < ncl; ++cl)
            for (int c = 0; c < gc; ++c) inv_off[(size_t)cl * nc + c0 + c] = i0 + hio[(size_t)cl * gc + c];
        const int64_t mi = (int64_t)(g.inv.bytes() / sizeof(T));
        RBF_CUDA(cudaMemcpy((T *)M.inv.p + i0, g.inv.p, mi * sizeof(T), cudaMemcpyDeviceToDevice));
        r0 += gn;
        c0 += gc;
        i0 += mi;
        E.rows_before.push_back(r0);
    }
    cstart[nc] = ng;
    M.n_ghost = ng;
    M.rows = ng;
    M.n_comp = nc;
    M.n_class = ncl;
    M.npad = npad;
    memcpy(M.field_class, fcl, sizeof(fcl));
    M.gidx.alloc(gidx.size());
    M.gw.alloc(gw.size() * sizeof(T));
    M.owner.alloc(ng);
    M.tb.alloc(ng);
    M.pos.alloc(ng);
    M.comp_of.alloc(ng);
    M.grec.alloc(ng);
    M.comp_start.alloc(nc + 1);
    M.inv_off.alloc(inv_off.size());
    M.res.alloc((size_t)4 * ng * sizeof(T));
    RBF_CUDA(cudaMemcpy(M.gidx.p, gidx.data(), gidx.size() * 4, cudaMemcpyHostToDevice));
    RBF_CUDA(cudaMemcpy(M.gw.p, gw.data(), gw.size() * sizeof(T), cudaMemcpyHostToDevice));
    RBF_CUDA(cudaMemcpy(M.owner.p, owner.data(), ng * 4, cudaMemcpyHostToDevice));
    RBF_CUDA(cudaMemcpy(M.tb.p, tb.data(), ng, cudaMemcpyHostToDevice));
    RBF_CUDA(cudaMemcpy(M.pos.p, pos.data(), ng * 4, cudaMemcpyHostToDevice));
    RBF_CUDA(cudaMemcpy(M.comp_of.p, comp_of.data(), ng * 4, cudaMemcpyHostToDevice));
    RBF_CUDA(cudaMemcpy(M.grec.p, grec.data(), ng * 8, cudaMemcpyHostToDevice));
    RBF_CUDA(cudaMemcpy(M.comp_start.p, cstart.data(), (nc + 1) * 8, cudaMemcpyHostToDevice));
    RBF_CUDA(cudaMemcpy(M.inv_off.p, inv_off.data(), inv_off.size() * 8, cudaMemcpyHostToDevice));
    build_ghost_bands(M, sizeof(T) == 8 ? 64 : 32, pb.st);
    // the members' own ghost plans are no longer needed
    for (auto &m : E.members) m->gh = GhostPlan();
}

void set_ens_threads(Problem &pb, int G) {
    EnsembleState &E = *pb.ens;
    pb.G = G;
    for (auto &m : E.members) {
        m->G = G;
        m->pf = 0;
        pack_operators(*m);
    }
    if (pb.precision == 64) fill_descs<double>(pb);
    else fill_descs<float>(pb);
}

// Autotuner: lanes per node (and with it nodes per CTA = 256 / lanes and the
// SELL slice width) for the whole ensemble, timed on full RK4 steps.
void autotune_ensemble(Problem &pb) {
    EnsembleState &E = *pb.ens;
    E.active_members = (int)E.members.size();
    DevBuf<unsigned char> U((size_t)E.total_records * 4 * pb.tsize());
    RBF_CUDA(cudaMemsetAsync(U.p, 0, U.bytes(), pb.st));
    cudaEvent_t e0, e1;
    RBF_CUDA(cudaEventCreate(&e0));
    RBF_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bestG = 2;
    for (int G : {1, 2, 4}) {
        set_ens_threads(pb, G);
        float ms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            RBF_CUDA(cudaEventRecord(e0, pb.st));
            for (int it = 0; it < 2; ++it) enqueue_ens_step(pb, 0.0, U.p, pb.st, false, 0);
            RBF_CUDA(cudaEventRecord(e1, pb.st));
            RBF_CUDA(cudaEventSynchronize(e1));
            float t = 0.f;
            RBF_CUDA(cudaEventElapsedTime(&t, e0, e1));
            ms = std::min(ms, t);
        }
        if (ms < best) { best = ms; bestG = G; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_ens_threads(pb, bestG);
}

}  // namespace

void enqueue_ens_step(Problem &pb, double, void *U, cudaStream_t s, bool rec, int step) {
    if (pb.precision == 64) ens_step<double>(pb, (double *)U, s, rec, step);
    else ens_step<float>(pb, (float *)U, s, rec, step);
}

void build_ensemble(Problem &pb, const rbf_ns_params &common, int n, const rbf_ens_member *mem, const double *x,
                    const double *z, const int32_t *kind, const int32_t *owner, void *stream) {
    RBF_REQUIRE(n >= 1, "an ensemble needs at least one member");
    RBF_REQUIRE(common.precision == 32 || common.precision == 64, "precision must be 64 or 32");
    RBF_REQUIRE(x && z && kind && owner && mem, "null argument");
    RBF_REQUIRE(common.threads_per_node == 0 || common.threads_per_node == 1 || common.threads_per_node == 2 ||
                    common.threads_per_node == 4,
                "ensemble threads per node must be 0 (autotune), 1, 2 or 4");
    pb.kind = kEnsemble;
    pb.F = 4;
    pb.precision = common.precision;
    pb.st = as_stream(stream);
    RBF_CUDA(cudaStreamCreateWithFlags(&pb.cap, cudaStreamNonBlocking));
    pb.tdev.alloc(1);
    pb.theta_bar = common.theta_bar;
    pb.g = common.g;
    pb.cp = common.cp;
    pb.cv = common.cv;
    pb.rd = common.rd;
    pb.diff = pb.precision == 32 ? 1 : 0;
    RBF_REQUIRE(common.storage == RBF_STORE_PER_NODE || common.storage == RBF_STORE_LATTICE, "unknown storage mode %d",
                common.storage);
    pb.lat.enabled = common.storage == RBF_STORE_LATTICE;   // each member keeps its own class table
    pb.ens.reset(new EnsembleState());
    EnsembleState &E = *pb.ens;
    int64_t off_all = 0, off_prog = 0, off_ghost = 0;
    cudaEvent_t e0, e1;
    RBF_CUDA(cudaEventCreate(&e0));
    RBF_CUDA(cudaEventCreate(&e1));
    RBF_CUDA(cudaEventRecord(e0, pb.st));
    for (int r = 0; r < n; ++r) {
        const rbf_ens_member &mr = mem[r];
        RBF_REQUIRE(mr.n_prog >= 1 && mr.n_all > mr.n_prog, "member %d needs prognostic and ghost nodes", r);
        RBF_REQUIRE(mr.dt > 0.0 && std::isfinite(mr.dt) && mr.n_steps >= 0, "member %d: bad dt or step count", r);
        rbf_ns_params p = common;
        p.n_sten = mr.n_sten;
        p.poly_l = mr.poly_l;
        p.period_x = mr.period_x;
        // each member's own gamma: its own constant (or the common one) with
        // the member's spacing, or the member's gamma as given
        RBF_REQUIRE(std::isfinite(mr.gamma_c) && mr.gamma_c >= 0.0, "member %d: gamma_c must be >= 0", r);
        p.gamma = resolve_gamma(mr.gamma, mr.gamma_c > 0.0 ? mr.gamma_c : common.gamma_c, mr.spacing, common.hv_k);
        p.gamma_c = 0.0;
        p.threads_per_node = 2;
        std::unique_ptr<Problem> m(new Problem());
        build_ns(*m, p, x + off_all, z + off_all, mr.n_prog, mr.n_all, kind + off_prog, owner + off_ghost, stream,
                 false);
        E.rec0.push_back(off_all);
        E.dt.push_back(mr.dt);
        E.n_steps.push_back(mr.n_steps);
        E.members.push_back(std::move(m));
        off_all += mr.n_all;
        off_prog += mr.n_prog;
        off_ghost += mr.n_all - mr.n_prog;
    }
    E.total_records = off_all;
    E.total_nodes = off_prog;
    pb.n_prog = off_prog;
    pb.n_all = off_all;
    E.order.resize(n);
    std::iota(E.order.begin(), E.order.end(), 0);
    std::stable_sort(E.order.begin(), E.order.end(), [&](int a, int b) { return E.n_steps[a] > E.n_steps[b]; });
    if (pb.precision == 64) merge_ghosts<double>(pb);
    else merge_ghosts<float>(pb);
    // RK4 buffers over all records; the accumulator is indexed by record too
    const size_t bytes = (size_t)E.total_records * 4 * pb.tsize();
    pb.S0.alloc(bytes);
    pb.S1.alloc(bytes);
    pb.K.alloc(bytes);
    RBF_CUDA(cudaMemsetAsync(pb.S0.p, 0, bytes, pb.st));
    RBF_CUDA(cudaMemsetAsync(pb.S1.p, 0, bytes, pb.st));
    RBF_CUDA(cudaMemsetAsync(pb.K.p, 0, bytes, pb.st));
    RBF_CUDA(cudaEventRecord(e1, pb.st));
    RBF_CUDA(cudaEventSynchronize(e1));
    RBF_CUDA(cudaEventElapsedTime(&pb.weight_build_ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (auto &m : E.members) pb.ghost_setup_ms += m->ghost_setup_ms;
    if (common.threads_per_node == 0) autotune_ensemble(pb);
    else set_ens_threads(pb, common.threads_per_node);
    // FP64 weights and raw stencils were only needed to build and repack
    for (auto &m : E.members) {
        m->w64.release();
        m->idx.release();
        m->x.release();
        m->z.release();
    }
    pb.n = E.members[0]->n;
    pb.n_slots = 0;
    for (auto &m : E.members) pb.n_slots = std::max(pb.n_slots, m->n_slots);
    RBF_CUDA(cudaStreamSynchronize(pb.st));
}

namespace {

// One pass of a whole-run graph's loop: the WHILE node that repeats a phase's
// chunk of steps stops once its counter reaches zero.
__global__ void count_down(unsigned *counter, cudaGraphConditionalHandle h) {
    if (threadIdx.x == 0) {
        const unsigned v = *counter - 1;
        *counter = v;
        if (v == 0) cudaGraphSetConditional(h, 0);
    }
}

constexpr int kRunChunk = 16;   // steps per loop pass of a phase

// Captures a whole run of `total` global steps as one graph: per phase of
// constant active prefix (members leave it as they reach their end), a memset
// that arms the phase's counter, a WHILE node whose body is kRunChunk steps of
// the active members and the count-down kernel, then the phase's leftover
// steps.  The loop bodies hold plain kernel launches (no programmatic
// dependent launch edges).
void build_run_graph(Problem &pb, int64_t total, void *U) {
    EnsembleState &E = *pb.ens;
    if (pb.graph) cudaGraphExecDestroy(pb.graph);
    pb.graph = nullptr;
    std::vector<std::pair<int, int64_t>> phases;   // (active members, steps)
    for (int64_t t = 0; t < total;) {
        int active = 0;
        while (active < (int)E.order.size() && E.n_steps[E.order[active]] > t) ++active;
        const int64_t phase_end = std::min(total, E.n_steps[E.order[active - 1]]);
        phases.emplace_back(active, phase_end - t);
        t = phase_end;
    }
    if (E.wcount.n < phases.size()) E.wcount.alloc(phases.size());
    const bool pdl0 = pb.pdl;
    pb.pdl = false;
    cudaGraph_t g = nullptr;
    RBF_CUDA(cudaGraphCreate(&g, 0));
    bool capturing = false;
    try {
        std::vector<cudaGraphNode_t> deps;
        for (size_t p = 0; p < phases.size(); ++p) {
            E.active_members = phases[p].first;
            const int64_t steps = phases[p].second;
            const int chunk = (int)std::min<int64_t>(steps, kRunChunk);
            const int64_t passes = steps / chunk, rem = steps - passes * chunk;
            cudaMemsetParams mp = {};
            mp.dst = E.wcount.p + p;
            mp.value = (unsigned)passes;
            mp.elementSize = 4;
            mp.width = 1;
            mp.height = 1;
            cudaGraphNode_t arm;
            RBF_CUDA(cudaGraphAddMemsetNode(&arm, g, deps.data(), deps.size(), &mp));
            cudaGraphConditionalHandle h;
            RBF_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t loop;
            RBF_CUDA(cudaGraphAddNode(&loop, g, &arm, nullptr, 1, &cp));
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            RBF_CUDA(cudaStreamBeginCaptureToGraph(pb.cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            capturing = true;
            for (int q = 0; q < chunk; ++q) enqueue_ens_step(pb, 0.0, U, pb.cap, false, q);
            count_down<<<1, 32, 0, pb.cap>>>(E.wcount.p + p, h);
            RBF_CHECK_LAUNCH();
            cudaGraph_t out = nullptr;
            capturing = false;
            RBF_CUDA(cudaStreamEndCapture(pb.cap, &out));
            deps.assign(1, loop);
            if (rem > 0) {
                RBF_CUDA(cudaStreamBeginCaptureToGraph(pb.cap, g, deps.data(), nullptr, deps.size(),
                                                       cudaStreamCaptureModeThreadLocal));
                capturing = true;
                for (int q = 0; q < rem; ++q) enqueue_ens_step(pb, 0.0, U, pb.cap, false, q);
                cudaStreamCaptureStatus cs;
                const cudaGraphNode_t *tail = nullptr;
                size_t nt = 0;
                RBF_CUDA(cudaStreamGetCaptureInfo(pb.cap, &cs, nullptr, nullptr, &tail, nullptr, &nt));
                std::vector<cudaGraphNode_t> next(tail, tail + nt);
                capturing = false;
                RBF_CUDA(cudaStreamEndCapture(pb.cap, &out));
                deps = next;
            }
        }
        RBF_CUDA(cudaGraphInstantiate(&pb.graph, g, 0));
    } catch (...) {
        if (capturing) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(pb.cap, &junk);
        }
        cudaGraphDestroy(g);
        pb.pdl = pdl0;
        throw;
    }
    cudaGraphDestroy(g);
    pb.pdl = pdl0;
    pb.graph_U = U;
    pb.graph_steps = (int)std::min<int64_t>(total, INT32_MAX);
    E.whole_run = true;
}

}  // namespace

// Steps every member min(max_steps, its n_steps) steps (max_steps < 0: all).
// The whole run is one graph launch (build_run_graph, rebuilt when the state
// or the step count changes); with stage timing on, phases are replayed from
// one-step graphs that carry the timing events instead.
void run_ensemble(Problem &pb, int64_t max_steps, void *U) {
    EnsembleState &E = *pb.ens;
    RBF_REQUIRE(U != nullptr, "null state");
    const int64_t longest = E.n_steps[E.order[0]];
    const int64_t total = max_steps < 0 ? longest : std::min(max_steps, longest);
    cudaEvent_t ev;
    RBF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    RBF_CUDA(cudaEventRecord(ev, pb.st));
    RBF_CUDA(cudaStreamWaitEvent(pb.cap, ev, 0));
    if (!pb.record_rhs_events && total > 0) {
        if (!pb.graph || !E.whole_run || pb.graph_U != U || pb.graph_steps != (int)std::min<int64_t>(total, INT32_MAX))
            build_run_graph(pb, total, U);
        RBF_CUDA(cudaGraphLaunch(pb.graph, pb.cap));
    }
    int64_t t = pb.record_rhs_events ? 0 : total;
    while (t < total) {
        int active = 0;
        while (active < (int)E.order.size() && E.n_steps[E.order[active]] > t) ++active;
        const int64_t phase_end = std::min(total, E.n_steps[E.order[active - 1]]);
        const int64_t steps = phase_end - t;
        const int chunk = (int)std::min<int64_t>(steps, pb.record_rhs_events ? 1 : 16);
        if (!pb.graph || E.whole_run || pb.graph_U != U || pb.graph_steps != chunk || E.active_members != active) {
            if (pb.graph) cudaGraphExecDestroy(pb.graph);
            pb.graph = nullptr;
            E.whole_run = false;
            E.active_members = active;
            if (pb.record_rhs_events) {
                for (cudaEvent_t e : pb.rhs_ev) cudaEventDestroy(e);
                pb.rhs_ev.assign(8 * chunk, nullptr);
                for (auto &e : pb.rhs_ev) RBF_CUDA(cudaEventCreate(&e));
            }
            cudaGraph_t g = nullptr;
            RBF_CUDA(cudaStreamBeginCapture(pb.cap, cudaStreamCaptureModeThreadLocal));
            try {
                for (int q = 0; q < chunk; ++q) enqueue_ens_step(pb, 0.0, U, pb.cap, pb.record_rhs_events, q);
            } catch (...) {
                cudaStreamEndCapture(pb.cap, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            RBF_CUDA(cudaStreamEndCapture(pb.cap, &g));
            cudaError_t e = cudaGraphInstantiate(&pb.graph, g, 0);
            cudaGraphDestroy(g);
            RBF_CUDA(e);
            pb.graph_U = U;
            pb.graph_steps = chunk;
        }
        int64_t done = 0;
        while (done + chunk <= steps) {
            RBF_CUDA(cudaGraphLaunch(pb.graph, pb.cap));
            done += chunk;
        }
        for (; done < steps; ++done) enqueue_ens_step(pb, 0.0, U, pb.cap, false, 0);
        t = phase_end;
    }
    RBF_CUDA(cudaEventRecord(ev, pb.cap));
    RBF_CUDA(cudaStreamWaitEvent(pb.st, ev, 0));
    cudaEventDestroy(ev);
}

// Node updates (prognostic nodes x RK4 steps) of run_ensemble(max_steps).
double ensemble_node_updates(const Problem &pb, int64_t max_steps) {
    const EnsembleState &E = *pb.ens;
    double s = 0.0;
    for (size_t r = 0; r < E.members.size(); ++r) {
        const int64_t st = max_steps < 0 ? E.n_steps[r] : std::min(max_steps, E.n_steps[r]);
        s += (double)E.members[r]->n_prog * (double)st;
    }
    return s;
}

}  // namespace rbf

extern "C" int rbf_ens_create(rbf_problem **out, const rbf_ns_params *common, int32_t n_members,
                              const rbf_ens_member *members, const double *x, const double *z, const int32_t *kind,
                              const int32_t *ghost_owner, void *stream) {
    return rbf::guarded([&] {
        RBF_REQUIRE(out && common, "null argument");
        *out = nullptr;
        auto *h = new rbf_problem();
        try {
            rbf::build_ensemble(h->impl, *common, n_members, members, x, z, kind, ghost_owner, stream);
            *out = h;
        } catch (...) {
            delete h;
            throw;
        }
    });
}

extern "C" int rbf_ens_run(rbf_problem *h, int64_t max_steps, void *U) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && h->impl.kind == rbf::kEnsemble, "not an ensemble problem");
        rbf::run_ensemble(h->impl, max_steps, U);
    });
}

extern "C" int rbf_ens_node_updates(const rbf_problem *h, int64_t max_steps, double *out) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && out && h->impl.kind == rbf::kEnsemble, "not an ensemble problem");
        *out = rbf::ensemble_node_updates(h->impl, max_steps);
    });
}
