// a3 + a5 + a6 + a7: packed operators and the fused right-hand side + RK4
// stage kernels of the Navier-Stokes (Sec. 6.2, Eqs. (uEq)-(piEq)) and the
// scalar advection (Sec. 6.1) problems.
//
// Packed layout (SELL with one slice per node group): neighbour slot t of
// node i goes to lane g = t % G, step s = t / G, and is stored at
// [s][i][g].  A warp covers 32/G nodes x G lanes, so every weight and index
// load of a step is one contiguous 128-byte (FP32) or 256-byte (FP64)
// segment.  The G lanes of a node reduce their partial sums with xor
// shuffles and then split the four fields' epilogues between them.
//
// FP32 mode uses the difference form sum_j w_ij (f_j - f_i) (every operator
// here annihilates constants: the p_0 = 1 constraint row of Eq. (weights)),
// which drops the centre slot and keeps cancellation errors relative to the
// local variation.  FP64 mode keeps the plain product sum_j w_ij f_j.
//
// Each stage kernel evaluates all 12 stencil sums of a node (d/dx, d/dz of
// the four fields, the dissipation mu Lap + hyperviscosity on u, w, theta',
// hyperviscosity on pi'), the tendencies of Eqs. (uEq)-(piEq), and the
// classical RK4 update in its epilogue, so one RK4 stage is one pass.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "problem.cuh"
#include "records.cuh"

namespace rbf {

namespace {

template <class T>
struct NSArgs {
    const T *Uin;     // [n_all][4] stage input (node-major records), ghosts filled
    const T *Un;      // [n_all][4] state at the start of the step
    T *Uout;          // [n_all][4] stage output (prognostic records)
    T *K;             // [n_prog][4] RK4 accumulator
    T *dUdt;          // [n_prog][4] tendency (stage < 0)
    const int32_t *pidx;
    const T *wx, *wz, *wd, *wh;
    const T *pibar;
    const unsigned char *flags;
    // split stage launches: each of the two launches takes its nodes from
    // nlist (n_list of them; null: every node, one launch per stage)
    const int32_t *nlist;
    int64_t n_list;
    // lattice storage (csrc/lattice.cu): class of each node (-1: per-node
    // operators), and per class the relative index and the packed operators
    // of every slot, [4][n_cls][SLQ][G][V] (null: per-node storage only)
    const int32_t *lcls, *loff;
    const T *lw;
    int n_cls;
    int64_t n_prog, n_all;
    int SLQ;          // operand vectors per lane
    int stage;
    T a_next, b_stage;
    T cp, g_over_tb, theta_bar, dpibar, rd_cv;
};

// 16-byte operand vectors: 4 FP32 or 2 FP64 slots, with matching index vectors.
template <class T>
struct Vec;
template <>
struct Vec<float> {
    static constexpr int V = 4;
    using W = float4;
    using I = int4;
    __device__ static float at(const float4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
    __device__ static int at(const int4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
    __device__ static int4 shift(const int4 &v, int d) { return make_int4(v.x + d, v.y + d, v.z + d, v.w + d); }
};
template <>
struct Vec<double> {
    static constexpr int V = 2;
    using W = double2;
    using I = int2;
    __device__ static double at(const double2 &v, int k) { return k == 0 ? v.x : v.y; }
    __device__ static int at(const int2 &v, int k) { return k == 0 ? v.x : v.y; }
    __device__ static int2 shift(const int2 &v, int d) { return make_int2(v.x + d, v.y + d); }
};

constexpr int kPrefetchVec = 3;   // operand vectors per lane held in registers (prefetch variant)

// One RK4 stage (or the bare right-hand side when stage < 0) for G lanes per
// node.  Each lane reads its operands as 16-byte vectors (V slots each) and
// gathers one node record per neighbour.  PF > 0: the lane's operand vectors
// (constant data) are loaded into registers before grid_dep_wait(), so they
// stream in while the preceding ghost kernels finish; PF == 0 streams them.
// LAT: a node of a lattice class takes its operand vectors from the class
// table (neighbour = node + offset); the lanes of a warp whose nodes share a
// class read the same table entries, which stay in L1.
template <class T, int G, bool DIFF, int PF, bool LAT>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && PF == 0) ? 4 : 1) ns_stage_kernel(NSArgs<T> a) {
    using VT = Vec<T>;
    using W = typename VT::W;
    using I = typename VT::I;
    constexpr int V = VT::V;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int g = (int)(tid % G);
    int64_t i = tid / G;
    bool live;
    if (a.nlist) {
        live = i < a.n_list;
        i = __ldg(a.nlist + (live ? i : a.n_list - 1));
    } else {
        live = i < a.n_prog;
        if (!live) i = a.n_prog - 1;   // keep the lanes of the warp in the shuffles
    }
    // lanes without a node leave unless a warp shuffle still needs them
    if (G == 1 ? !live : !__any_sync(0xffffffffu, live)) return;
    const int64_t stride = a.n_prog * G;   // in vectors, between consecutive q
    const int64_t off0 = i * G + g;
    const I *pidx = reinterpret_cast<const I *>(a.pidx);
    const W *wx = reinterpret_cast<const W *>(a.wx), *wz = reinterpret_cast<const W *>(a.wz);
    const W *wd = reinterpret_cast<const W *>(a.wd), *wh = reinterpret_cast<const W *>(a.wh);
    constexpr int R = PF > 0 ? PF : 1;
    I jr[R];
    W rx[R], rz[R], rd[R], rh[R];
    if (PF > 0) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (q < a.SLQ) {
                const int64_t off = off0 + q * stride;
                jr[q] = __ldg(pidx + off);
                rx[q] = __ldg(wx + off);
                rz[q] = __ldg(wz + off);
                rd[q] = __ldg(wd + off);
                rh[q] = __ldg(wh + off);
            }
        }
    }
    grid_dep_wait();     // the stage input (and its ghosts) come from earlier kernels
    grid_dep_launch();
    const T *U = a.Uin;
    Rec<T> fi = {0, 0, 0, 0};
    if (DIFF) fi = load_rec(U, i);
    T ux = 0, uz = 0, ud = 0, wx_ = 0, wz_ = 0, wd_ = 0, tx = 0, tz = 0, td = 0, px = 0, pz = 0, ph = 0;
    auto vec = [&](const I &jv, const W &cx, const W &cz, const W &cd, const W &ch) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            Rec<T> r = load_rec(U, VT::at(jv, v));
            if (DIFF) { r.u -= fi.u; r.w -= fi.w; r.t -= fi.t; r.p -= fi.p; }
            const T x = VT::at(cx, v), z = VT::at(cz, v), d = VT::at(cd, v), h = VT::at(ch, v);
            ux += x * r.u; uz += z * r.u; ud += d * r.u;
            wx_ += x * r.w; wz_ += z * r.w; wd_ += d * r.w;
            tx += x * r.t; tz += z * r.t; td += d * r.t;
            px += x * r.p; pz += z * r.p; ph += h * r.p;
        }
    };
    if (PF > 0) {
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (q < a.SLQ) vec(jr[q], rx[q], rz[q], rd[q], rh[q]);
    } else if (LAT && __ldg(a.lcls + i) >= 0) {
        const int c = __ldg(a.lcls + i);
        const I *lo = reinterpret_cast<const I *>(a.loff);
        const W *lw = reinterpret_cast<const W *>(a.lw);
        const int64_t ls = (int64_t)a.n_cls * a.SLQ * G;   // in vectors, between operators
        int64_t off = (int64_t)c * a.SLQ * G + g;
#pragma unroll 2
        for (int q = 0; q < a.SLQ; ++q, off += G)
            vec(VT::shift(__ldg(lo + off), (int)i), __ldg(lw + off), __ldg(lw + ls + off), __ldg(lw + 2 * ls + off),
                __ldg(lw + 3 * ls + off));
    } else {
        int64_t off = off0;
#pragma unroll 2
        for (int q = 0; q < a.SLQ; ++q, off += stride)
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
    const unsigned char fl = a.flags[i];
    const T cpth = a.cp * (a.theta_bar + c.t);
    T k[4];
    k[0] = -c.u * ux - c.w * uz - cpth * px + ud;
    k[1] = -c.u * wx_ - c.w * wz_ - cpth * pz + a.g_over_tb * c.t + wd_;
    k[2] = -c.u * tx - c.w * tz + td;
    k[3] = -c.u * px - c.w * (a.dpibar + pz) - a.rd_cv * (a.pibar[i] + c.p) * (ux + wz_) + ph;
    if (fl & 1) k[1] = 0;   // w = 0 held on bottom/top walls
    if (fl & 2) k[0] = 0;   // u = 0 held on left/right walls
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (f % G != g) continue;   // lanes split the four fields' epilogues
        const T kf = k[f];
        const int64_t e = i * 4 + f;
        if (a.stage < 0) {
            a.dUdt[e] = kf;
        } else {
            const T un = a.Un[e];
            if (a.stage == 0) {
                a.K[e] = a.b_stage * kf;
                a.Uout[e] = un + a.a_next * kf;
            } else if (a.stage < 3) {
                a.K[e] += a.b_stage * kf;
                a.Uout[e] = un + a.a_next * kf;
            } else {
                a.Uout[e] = un + (a.K[e] + a.b_stage * kf);
            }
        }
    }
}

// Velocity u(x, t) = sum_k c_k(t) (U_k, V_k)(x) with c_k(t) = fa_k + fb_k
// cos(fm_k pi t / T): one separable part for the deformational flow, two for
// the vortex flow of Sec. 6.1.  Packed block k holds part k's flux-form
// weights; the hyperviscosity block follows the parts.
template <class T>
struct AdvArgs {
    const T *Uin, *Un;
    T *Uout, *K, *dUdt;
    const int32_t *pidx;
    const T *wa, *wa2, *wh;
    int64_t n_prog;
    int SL, stage;
    T a_next, b_stage;
    const double *tdev;   // device time (graph replays) or nullptr
    double t_host, t_frac_dt, period_T;
    double fa[2], fb[2], fm[2];
};

__device__ __forceinline__ double flow_factor(double a, double b, double m, double t, double T) {
    return b == 0.0 ? a : a + b * cos(m * 3.141592653589793 * t / T);
}

template <class T, int G, int NP>
__global__ void __launch_bounds__(256) adv_stage_kernel(AdvArgs<T> a) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int g = (int)(tid % G);
    int64_t i = tid / G;
    const bool live = i < a.n_prog;
    if (!live) i = a.n_prog - 1;
    grid_dep_wait();
    grid_dep_launch();
    T sa = 0, sb = 0, sh = 0;
    const int64_t stride = a.n_prog * G;
    int64_t off = i * G + g;
#pragma unroll 4
    for (int s = 0; s < a.SL; ++s, off += stride) {
        const int j = __ldg(a.pidx + off);
        const T v = a.Uin[j];
        sa += __ldg(a.wa + off) * v;
        if (NP == 2) sb += __ldg(a.wa2 + off) * v;
        sh += __ldg(a.wh + off) * v;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o, G);
        if (NP == 2) sb += __shfl_xor_sync(0xffffffffu, sb, o, G);
        sh += __shfl_xor_sync(0xffffffffu, sh, o, G);
    }
    if (!live || g != 0) return;
    // velocity time factors at this stage's time
    double t = (a.tdev ? *a.tdev : a.t_host) + a.t_frac_dt;
    T kf = (T)flow_factor(a.fa[0], a.fb[0], a.fm[0], t, a.period_T) * sa + sh;
    if (NP == 2) kf += (T)flow_factor(a.fa[1], a.fb[1], a.fm[1], t, a.period_T) * sb;
    if (a.stage < 0) {
        a.dUdt[i] = kf;
    } else {
        const T un = a.Un[i];
        if (a.stage == 0) {
            a.K[i] = a.b_stage * kf;
            a.Uout[i] = un + a.a_next * kf;
        } else if (a.stage < 3) {
            a.K[i] += a.b_stage * kf;
            a.Uout[i] = un + a.a_next * kf;
        } else {
            a.Uout[i] = un + (a.K[i] + a.b_stage * kf);
        }
    }
}

__global__ void advance_time(double *t, double dt) {
    grid_dep_wait();
    *t += dt;
}

// Packs FP64 weights [ops][n_prog][n] into [n_packed][SLQ][n_prog][G][V] of T
// (slot t = (q G + g) V + v of node i) and the indices alike.
// comb[q][o]: coefficient of weight block o in packed operator q.
template <class T>
__global__ void pack_kernel(const double *__restrict__ w64, const int32_t *__restrict__ idx, int64_t n_prog,
                            int n, int nops, int first, int n_slots, int SLQ, int G, int V, int n_packed,
                            const double *__restrict__ comb, T *__restrict__ pw, int32_t *__restrict__ pidx) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int per = SLQ * G * V;
    int64_t total = (int64_t)per * n_prog;
    if (t >= total) return;
    int64_t i = t / per;
    int slot = (int)(t - i * per);
    int v = slot % V, gq = slot / V;
    int g = gq % G, q = gq / G;
    int64_t dst = (((int64_t)q * n_prog + i) * G + g) * V + v;
    if (slot < n_slots) {
        int k = slot + first;
        pidx[dst] = idx[i * n + k];
        for (int p = 0; p < n_packed; ++p) {
            double val = 0.0;
            for (int o = 0; o < nops; ++o) {
                double c = comb[p * nops + o];
                if (c != 0.0) val += c * w64[((int64_t)o * n_prog + i) * n + k];
            }
            pw[(int64_t)p * total + dst] = (T)val;
        }
    } else {
        pidx[dst] = (int32_t)i;
        for (int p = 0; p < n_packed; ++p) pw[(int64_t)p * total + dst] = (T)0;
    }
}

// Advection: packed block k < NP = flux-form weights of velocity part k,
// -(Dx_ij U_k(x_j) + Dy_ij V_k(x_j)); block NP = (-1)^(k+1) gamma Delta^k
// weights; columns folded onto the source node of reflected nodes
// (Sec. 6.1).  Weight blocks in w64: Dx, Dy, Delta^k.  vel holds
// [NP][U, V][n_all].
template <class T>
__global__ void pack_adv_kernel(const double *__restrict__ w64, const int32_t *__restrict__ idx, int64_t n_prog,
                                int64_t n_all, int n, int has_hv, double hvc, const double *__restrict__ vel, int NP,
                                const int32_t *__restrict__ src, int SL, int G, T *__restrict__ pw,
                                int32_t *__restrict__ pidx) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = (int64_t)SL * G * n_prog;
    if (t >= total) return;
    int64_t i = t / ((int64_t)SL * G);
    int slot = (int)(t - i * SL * G);
    int s = slot / G, g = slot - s * G;
    int64_t dst = ((int64_t)s * n_prog + i) * G + g;
    if (slot < n) {
        int j = idx[i * n + slot];
        pidx[dst] = src[j];
        double dx = w64[((int64_t)0 * n_prog + i) * n + slot];
        double dy = w64[((int64_t)1 * n_prog + i) * n + slot];
        for (int k = 0; k < NP; ++k)
            pw[k * total + dst] = (T)(-(dx * vel[(2 * k) * n_all + j] + dy * vel[(2 * k + 1) * n_all + j]));
        pw[NP * total + dst] = has_hv ? (T)(hvc * w64[((int64_t)2 * n_prog + i) * n + slot]) : (T)0;
    } else {
        pidx[dst] = (int32_t)i;
        for (int k = 0; k <= NP; ++k) pw[k * total + dst] = (T)0;
    }
}

template <class T>
__global__ void minmax_kernel(const T *U, int64_t n_prog, int F, double *out, int *bad) {
    // node-major records U[i * F + f]; out[f*2+0] min, out[f*2+1] max via
    // ordered-int atomics on doubles
    for (int f = 0; f < F; ++f) {
        double lo = INFINITY, hi = -INFINITY;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_prog; i += (int64_t)gridDim.x * blockDim.x) {
            double v = (double)U[i * F + f];
            if (!isfinite(v)) atomicExch(bad, 1);
            lo = fmin(lo, v);
            hi = fmax(hi, v);
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if ((threadIdx.x & 31) == 0) {
            // monotone map of doubles to signed 64-bit integers
            long long l = __double_as_longlong(lo), h = __double_as_longlong(hi);
            l = l < 0 ? (long long)(0x8000000000000000ULL - (unsigned long long)l) : l;
            h = h < 0 ? (long long)(0x8000000000000000ULL - (unsigned long long)h) : h;
            atomicMin((long long *)&out[f * 2], l);
            atomicMax((long long *)&out[f * 2 + 1], h);
        }
    }
}

template <class T, int G, int PF>
void launch_ns_g(const NSArgs<T> &a, cudaStream_t s, bool pdl, int prio) {
    constexpr bool kDiff = sizeof(T) == 4;   // FP32: difference form; FP64: plain sums
    const dim3 grid(div_up((a.nlist ? a.n_list : a.n_prog) * G, 256)), blk(256);
    if (a.lcls) {
        if (PF == 0) launch_kernel_prio(ns_stage_kernel<T, G, kDiff, 0, true>, grid, blk, s, pdl, prio, a);
        else RBF_FAIL(RBF_E_ARG, "the lattice storage has no prefetch variant");
    } else {
        launch_kernel_prio(ns_stage_kernel<T, G, kDiff, PF, false>, grid, blk, s, pdl, prio, a);
    }
}

template <class T>
void launch_ns(const NSArgs<T> &a, int G, int pf, cudaStream_t s, bool pdl, int prio = 0) {
    if (pf > 0 && a.SLQ > kPrefetchVec)
        RBF_FAIL(RBF_E_ARG, "prefetch variant needs <= %d operand vectors per lane", kPrefetchVec);
    switch (G * 2 + (pf > 0)) {
        case 2: launch_ns_g<T, 1, 0>(a, s, pdl, prio); break;
        case 3: launch_ns_g<T, 1, kPrefetchVec>(a, s, pdl, prio); break;
        case 4: launch_ns_g<T, 2, 0>(a, s, pdl, prio); break;
        case 5: launch_ns_g<T, 2, kPrefetchVec>(a, s, pdl, prio); break;
        case 8: launch_ns_g<T, 4, 0>(a, s, pdl, prio); break;
        case 9: launch_ns_g<T, 4, kPrefetchVec>(a, s, pdl, prio); break;
        case 16: launch_ns_g<T, 8, 0>(a, s, pdl, prio); break;
        case 17: launch_ns_g<T, 8, kPrefetchVec>(a, s, pdl, prio); break;
        default: RBF_FAIL(RBF_E_ARG, "threads per node %d not in {1,2,4,8}", G);
    }
}

template <class T, int NP>
void launch_adv_np(const AdvArgs<T> &a, int G, cudaStream_t s, bool pdl) {
    const dim3 grid(div_up(a.n_prog * G, 256)), blk(256);
    switch (G) {
        case 1: launch_kernel(adv_stage_kernel<T, 1, NP>, grid, blk, s, pdl, a); break;
        case 2: launch_kernel(adv_stage_kernel<T, 2, NP>, grid, blk, s, pdl, a); break;
        case 4: launch_kernel(adv_stage_kernel<T, 4, NP>, grid, blk, s, pdl, a); break;
        case 8: launch_kernel(adv_stage_kernel<T, 8, NP>, grid, blk, s, pdl, a); break;
        default: RBF_FAIL(RBF_E_ARG, "threads per node %d not in {1,2,4,8}", G);
    }
}

template <class T>
void launch_adv(const AdvArgs<T> &a, int G, cudaStream_t s, bool pdl) {
    if (a.wa2) launch_adv_np<T, 2>(a, G, s, pdl);
    else launch_adv_np<T, 1>(a, G, s, pdl);
}

template <class T>
NSArgs<T> ns_args(Problem &pb) {
    NSArgs<T> a{};
    const int64_t total = (int64_t)pb.SLQ * pb.V * pb.G * pb.n_prog;
    const T *pw = (const T *)pb.pw.p;
    a.pidx = pb.pidx.p;
    a.wx = pw;
    a.wz = pw + total;
    a.wd = pw + 2 * total;
    a.wh = pw + 3 * total;
    a.pibar = (const T *)pb.pibar.p;
    a.flags = pb.flags.p;
    if (pb.lat.enabled) {
        a.lcls = pb.lat.cls.p;
        a.loff = pb.lat.loff.p;
        a.lw = (const T *)pb.lat.lw.p;
        a.n_cls = pb.lat.n_cls;
    }
    a.n_prog = pb.n_prog;
    a.n_all = pb.n_all;
    a.SLQ = pb.SLQ;
    a.cp = (T)pb.cp;
    a.g_over_tb = (T)(pb.g / pb.theta_bar);
    a.theta_bar = (T)pb.theta_bar;
    a.dpibar = (T)(-pb.g / (pb.cp * pb.theta_bar));
    a.rd_cv = (T)(pb.rd / pb.cv);
    return a;
}

template <class T>
AdvArgs<T> adv_args(Problem &pb) {
    AdvArgs<T> a{};
    const int64_t total = (int64_t)pb.SL * pb.G * pb.n_prog;
    const T *pw = (const T *)pb.pw.p;
    a.pidx = pb.pidx.p;
    a.wa = pw;
    a.wa2 = pb.n_vparts == 2 ? pw + total : nullptr;
    a.wh = pw + pb.n_vparts * total;
    a.n_prog = pb.n_prog;
    a.SL = pb.SL;
    a.period_T = pb.period_T;
    for (int k = 0; k < 2; ++k) {
        a.fa[k] = pb.vpart[k][0];
        a.fb[k] = pb.vpart[k][1];
        a.fm[k] = pb.vpart[k][2];
    }
    return a;
}

// RK4 coefficients: stage s writes U_n + a[s] dt k_s and accumulates b[s] dt k_s
const double kA[4] = {0.5, 0.5, 1.0, 0.0};
const double kB[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

// One RK4 step on stream s.  With the split (pb.split, not while recording
// stage events), each stage runs as two launches: the nodes off the wall set
// on the side stream, the wall set (nodes whose records feed a ghost residual
// or whose stencils read a ghost) on s after the stage's ghost fill.  The
// ghost fill of stage st + 1 needs only the wall set of stage st, so it runs
// while the side stream finishes stage st.  Event pairs alternate by stage
// parity: ev_w[st & 1] marks stage st's wall set, ev_r[st & 1] the rest.
// `first` = false continues a step sequence whose side stream is still open
// (the previous call passed `last` = false); `last` joins the side stream
// back into s.
template <class T>
void rk4_ns(Problem &pb, double dt, T *U, cudaStream_t s, bool rec, int step, bool first, bool last) {
    NSArgs<T> a = ns_args<T>(pb);
    T *S0 = (T *)pb.S0.p, *S1 = (T *)pb.S1.p;
    T *in[4] = {U, S0, S1, S0};
    T *out[4] = {S0, S1, S0, U};
    a.Un = U;
    a.K = (T *)pb.K.p;
    const bool split = pb.split && !rec;
    if (split) {
        RBF_CUDA(cudaEventRecord(pb.ev_fork, s));
        RBF_CUDA(cudaStreamWaitEvent(pb.side, pb.ev_fork, 0));
    }
    for (int st = 0; st < 4; ++st) {
        a.Uin = in[st];
        a.Uout = out[st];
        a.stage = st;
        a.a_next = (T)(kA[st] * dt);
        a.b_stage = (T)(kB[st] * dt);
        if (split) {
            NSArgs<T> ar = a;   // every node off the wall set
            ar.nlist = pb.rlist.p;
            ar.n_list = pb.n_prog - pb.n_wall;
            if (st > 0) RBF_CUDA(cudaStreamWaitEvent(pb.side, pb.ev_w[(st - 1) & 1], 0));
            launch_ns<T>(ar, pb.G, pb.pf, pb.side, pb.pdl);
            RBF_CUDA(cudaEventRecord(pb.ev_r[st & 1], pb.side));
            enqueue_ghost_fill(pb, in[st], s, pb.prio_hi);   // ahead of the other launch's blocks
            if (st > 0 || !first) RBF_CUDA(cudaStreamWaitEvent(s, pb.ev_r[(st + 3) & 1], 0));
            NSArgs<T> aw = a;   // the wall set, ahead of the other launch
            aw.nlist = pb.wlist.p;
            aw.n_list = pb.n_wall;
            launch_ns<T>(aw, pb.G, pb.pf, s, pb.pdl, pb.prio_hi);
            RBF_CUDA(cudaEventRecord(pb.ev_w[st & 1], s));
            continue;
        }
        enqueue_ghost_fill(pb, in[st], s);
        if (rec) RBF_CUDA(cudaEventRecordWithFlags(pb.rhs_ev[(step * 4 + st) * 2], s, cudaEventRecordExternal));
        launch_ns<T>(a, pb.G, pb.pf, s, pb.pdl && !rec);
        if (rec) RBF_CUDA(cudaEventRecordWithFlags(pb.rhs_ev[(step * 4 + st) * 2 + 1], s, cudaEventRecordExternal));
    }
    if (split && last) RBF_CUDA(cudaStreamWaitEvent(s, pb.ev_r[1], 0));
}

template <class T>
void rk4_adv(Problem &pb, double t, double dt, T *U, cudaStream_t s, bool use_tdev, bool rec, int step) {
    AdvArgs<T> a = adv_args<T>(pb);
    T *S0 = (T *)pb.S0.p, *S1 = (T *)pb.S1.p;
    T *in[4] = {U, S0, S1, S0};
    T *out[4] = {S0, S1, S0, U};
    const double frac[4] = {0.0, 0.5, 0.5, 1.0};
    a.Un = U;
    a.K = (T *)pb.K.p;
    a.tdev = use_tdev ? pb.tdev.p : nullptr;
    a.t_host = t;
    for (int st = 0; st < 4; ++st) {
        a.Uin = in[st];
        a.Uout = out[st];
        a.stage = st;
        a.a_next = (T)(kA[st] * dt);
        a.b_stage = (T)(kB[st] * dt);
        a.t_frac_dt = frac[st] * dt;
        if (rec) RBF_CUDA(cudaEventRecordWithFlags(pb.rhs_ev[(step * 4 + st) * 2], s, cudaEventRecordExternal));
        launch_adv<T>(a, pb.G, s, pb.pdl && !rec);
        if (rec) RBF_CUDA(cudaEventRecordWithFlags(pb.rhs_ev[(step * 4 + st) * 2 + 1], s, cudaEventRecordExternal));
    }
    if (use_tdev) {
        launch_kernel(advance_time, dim3(1), dim3(1), s, pb.pdl && !rec, pb.tdev.p, dt);
    }
}

}  // namespace

void pack_operators(Problem &pb) {
    const int nops = (int)pb.ops.size();
    pb.n_slots = pb.diff ? pb.n - 1 : pb.n;
    // NS: 16-byte operand vectors; advection: one slot per load
    pb.V = pb.kind == kNS ? (int)(16 / pb.tsize()) : 1;
    pb.SLQ = div_up(pb.n_slots, pb.G * pb.V);
    pb.SL = pb.SLQ * pb.V;
    const int64_t total = (int64_t)pb.SL * pb.G * pb.n_prog;
    pb.pidx.alloc(total);
    if (pb.kind == kAdvection) {
        pb.n_packed = pb.n_vparts + 1;
        pb.pw.alloc((size_t)pb.n_packed * total * pb.tsize());
        const int has_hv = nops > 2;
        if (pb.precision == 64)
            pack_adv_kernel<double><<<div_up(total, 256), 256, 0, pb.st>>>(
                pb.w64.p, pb.idx.p, pb.n_prog, pb.n_all, pb.n, has_hv, pb.hvc, pb.vel.p, pb.n_vparts, pb.src.p,
                pb.SL, pb.G, (double *)pb.pw.p, pb.pidx.p);
        else
            pack_adv_kernel<float><<<div_up(total, 256), 256, 0, pb.st>>>(
                pb.w64.p, pb.idx.p, pb.n_prog, pb.n_all, pb.n, has_hv, pb.hvc, pb.vel.p, pb.n_vparts, pb.src.p,
                pb.SL, pb.G, (float *)pb.pw.p, pb.pidx.p);
        RBF_CHECK_LAUNCH();
        RBF_CUDA(cudaStreamSynchronize(pb.st));
        return;
    }
    // Navier-Stokes: packed operators as combinations of the FP64 weight blocks
    auto slot = [&](int op) {
        for (int i = 0; i < nops; ++i)
            if (pb.ops[i] == op) return i;
        RBF_FAIL(RBF_E_ARG, "operator %d was not built", op);
    };
    std::vector<double> comb(4 * nops, 0.0);
    pb.n_packed = 4;
    comb[0 * nops + slot(RBF_OP_DX)] = 1.0;
    comb[1 * nops + slot(RBF_OP_DZ)] = 1.0;
    comb[2 * nops + slot(RBF_OP_LAP)] = pb.mu;
    if (pb.hv_k > 0) {
        comb[2 * nops + slot(RBF_OP_HV)] += pb.hvc;
        comb[3 * nops + slot(RBF_OP_HV)] = pb.hvc;
    }
    DevBuf<double> dcomb(comb.size());
    RBF_CUDA(cudaMemcpyAsync(dcomb.p, comb.data(), dcomb.bytes(), cudaMemcpyHostToDevice, pb.st));
    pb.pw.alloc((size_t)pb.n_packed * total * pb.tsize());
    if (pb.precision == 64)
        pack_kernel<double><<<div_up(total, 256), 256, 0, pb.st>>>(pb.w64.p, pb.idx.p, pb.n_prog, pb.n, nops, pb.diff,
                                                                   pb.n_slots, pb.SLQ, pb.G, pb.V, pb.n_packed,
                                                                   dcomb.p, (double *)pb.pw.p, pb.pidx.p);
    else
        pack_kernel<float><<<div_up(total, 256), 256, 0, pb.st>>>(pb.w64.p, pb.idx.p, pb.n_prog, pb.n, nops, pb.diff,
                                                                  pb.n_slots, pb.SLQ, pb.G, pb.V, pb.n_packed,
                                                                  dcomb.p, (float *)pb.pw.p, pb.pidx.p);
    RBF_CHECK_LAUNCH();
    RBF_CUDA(cudaStreamSynchronize(pb.st));
    if (pb.lat.enabled) pack_lattice(pb, comb, nops);
}

void enqueue_rk4_step(Problem &pb, double t, double dt, void *U, cudaStream_t s, bool rec, int step, bool first,
                      bool last) {
    const bool tdev = (s == pb.cap);
    if (pb.kind == kNS) {
        if (pb.precision == 64) rk4_ns<double>(pb, dt, (double *)U, s, rec, step, first, last);
        else rk4_ns<float>(pb, dt, (float *)U, s, rec, step, first, last);
    } else {
        if (pb.precision == 64) rk4_adv<double>(pb, t, dt, (double *)U, s, tdev, rec, step);
        else rk4_adv<float>(pb, t, dt, (float *)U, s, tdev, rec, step);
    }
}

void enqueue_rhs(Problem &pb, double t, void *U, void *dUdt, cudaStream_t s) {
    if (pb.kind == kNS) {
        enqueue_ghost_fill(pb, U, s);
        if (pb.precision == 64) {
            NSArgs<double> a = ns_args<double>(pb);
            a.Uin = (const double *)U;
            a.dUdt = (double *)dUdt;
            a.stage = -1;
            launch_ns<double>(a, pb.G, pb.pf, s, false);
        } else {
            NSArgs<float> a = ns_args<float>(pb);
            a.Uin = (const float *)U;
            a.dUdt = (float *)dUdt;
            a.stage = -1;
            launch_ns<float>(a, pb.G, pb.pf, s, false);
        }
    } else {
        if (pb.precision == 64) {
            AdvArgs<double> a = adv_args<double>(pb);
            a.Uin = (const double *)U;
            a.dUdt = (double *)dUdt;
            a.stage = -1;
            a.t_host = t;
            launch_adv<double>(a, pb.G, s, false);
        } else {
            AdvArgs<float> a = adv_args<float>(pb);
            a.Uin = (const float *)U;
            a.dUdt = (float *)dUdt;
            a.stage = -1;
            a.t_host = t;
            launch_adv<float>(a, pb.G, s, false);
        }
    }
}

// Autotuner: for every (threads per node, register prefetch) choice it
// repacks the operators and times whole RK4 steps through the real launch
// path (ghost kernels, programmatic launches) on a zero state, then keeps the
// fastest; a problem with a wall set then times its steps with split stage
// launches on and off.  The advection problem times its right-hand side per
// lane count.
void autotune_threads_per_node(Problem &pb) {
    const int cands[4] = {1, 2, 4, 8};
    float best = 1e30f;
    int bestG = 4, bestPf = 0;
    cudaEvent_t e0, e1;
    RBF_CUDA(cudaEventCreate(&e0));
    RBF_CUDA(cudaEventCreate(&e1));
    const size_t ts = pb.tsize();
    const int64_t rows = pb.kind == kNS ? pb.n_all : pb.n_prog;
    DevBuf<unsigned char> U((size_t)pb.F * rows * ts);
    DevBuf<unsigned char> D((size_t)pb.F * pb.n_prog * ts);
    RBF_CUDA(cudaMemsetAsync(U.p, 0, U.bytes(), pb.st));
    for (int G : cands) {
        pb.G = G;
        pack_operators(pb);
        for (int pf : {0, kPrefetchVec}) {
            if (pf > 0 && (pb.kind != kNS || pb.SLQ > kPrefetchVec || pb.lat.enabled)) continue;
            pb.pf = pf;
            float ms = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                RBF_CUDA(cudaEventRecord(e0, pb.st));
                for (int it = 0; it < 4; ++it) {
                    if (pb.kind == kNS) enqueue_rk4_step(pb, 0.0, 1e-3, U.p, pb.st, false, 0);
                    else enqueue_rhs(pb, 0.0, U.p, D.p, pb.st);
                }
                RBF_CUDA(cudaEventRecord(e1, pb.st));
                RBF_CUDA(cudaEventSynchronize(e1));
                float t = 0.f;
                RBF_CUDA(cudaEventElapsedTime(&t, e0, e1));
                ms = std::min(ms, t);
            }
            if (ms < best) { best = ms; bestG = G; bestPf = pf; }
        }
    }
    pb.G = bestG;
    pb.pf = bestPf;
    pack_operators(pb);
    if (pb.kind == kNS && pb.wlist.p) {
        // split stage launches, on or off, timed the same way
        float t[2] = {1e30f, 1e30f};
        for (int on = 0; on < 2; ++on) {
            pb.split = on != 0;
            for (int rep = 0; rep < 3; ++rep) {
                RBF_CUDA(cudaEventRecord(e0, pb.st));
                for (int it = 0; it < 4; ++it) enqueue_rk4_step(pb, 0.0, 1e-3, U.p, pb.st, false, 0);
                RBF_CUDA(cudaEventRecord(e1, pb.st));
                RBF_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                RBF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                t[on] = std::min(t[on], ms);
            }
        }
        pb.split = t[1] < t[0];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

void minmax(Problem &pb, const void *U, double *out) {
    DevBuf<double> d(2 * pb.F);
    DevBuf<int> bad(1);
    std::vector<long long> init(2 * pb.F);
    for (int f = 0; f < pb.F; ++f) {
        init[2 * f] = 0x7fffffffffffffffLL;
        init[2 * f + 1] = (long long)0x8000000000000000ULL;
    }
    RBF_CUDA(cudaMemcpyAsync(d.p, init.data(), d.bytes(), cudaMemcpyHostToDevice, pb.st));
    RBF_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), pb.st));
    // an ensemble's records interleave members' ghosts: scan every record
    const int64_t rows = pb.kind == kEnsemble ? pb.n_all : pb.n_prog;
    if (pb.precision == 64) minmax_kernel<double><<<128, 256, 0, pb.st>>>((const double *)U, rows, pb.F, d.p, bad.p);
    else minmax_kernel<float><<<128, 256, 0, pb.st>>>((const float *)U, rows, pb.F, d.p, bad.p);
    RBF_CHECK_LAUNCH();
    std::vector<long long> h(2 * pb.F);
    int hb = 0;
    RBF_CUDA(cudaMemcpyAsync(h.data(), d.p, d.bytes(), cudaMemcpyDeviceToHost, pb.st));
    RBF_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, pb.st));
    RBF_CUDA(cudaStreamSynchronize(pb.st));
    for (int q = 0; q < 2 * pb.F; ++q) {
        long long v = h[q];
        if (v < 0) v = (long long)(0x8000000000000000ULL - (unsigned long long)v);
        double dv;
        memcpy(&dv, &v, 8);
        out[q] = dv;
    }
    if (hb) RBF_FAIL(RBF_E_NONFINITE, "non-finite value in the state");
}

}  // namespace rbf
