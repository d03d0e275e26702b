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

namespace rbf {

namespace {

template <class T>
struct NSArgs {
    const T *Uin;     // [4][n_all] stage input, ghosts filled
    const T *Un;      // [4][n_all] state at the start of the step
    T *Uout;          // [4][n_all] stage output (prognostic entries)
    T *K;             // [4][n_prog] RK4 accumulator
    T *dUdt;          // [4][n_prog] tendency (stage < 0)
    const int32_t *pidx;
    const T *wx, *wz, *wd, *wh;
    const T *pibar;
    const unsigned char *flags;
    int64_t n_prog, n_all;
    int SL;
    int stage;
    T a_next, b_stage;
    T cp, g_over_tb, theta_bar, dpibar, rd_cv;
};

constexpr int kPrefetch = 10;   // neighbour slots per lane held in registers (prefetch variant)

// One RK4 stage (or the bare right-hand side when stage < 0) for G lanes per
// node.  PF > 0: the lane's packed weights and indices (constant data) are
// loaded into registers before grid_dep_wait(), so they stream in while the
// preceding ghost kernels finish; PF == 0 streams them inside the loop.
template <class T, int G, bool DIFF, int PF>
__global__ void __launch_bounds__(256) ns_stage_kernel(NSArgs<T> a) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int g = (int)(tid % G);
    int64_t i = tid / G;
    const bool live = i < a.n_prog;
    if (!live) i = a.n_prog - 1;   // keep the lanes of the warp in the shuffles
    const int64_t N = a.n_all;
    const int64_t stride = a.n_prog * G;
    const int64_t off0 = i * G + g;
    constexpr int R = PF > 0 ? PF : 1;
    int jr[R];
    T rx[R], rz[R], rd[R], rh[R];
    if (PF > 0) {
#pragma unroll
        for (int s = 0; s < R; ++s) {
            if (s < a.SL) {
                const int64_t off = off0 + s * stride;
                jr[s] = __ldg(a.pidx + off);
                rx[s] = __ldg(a.wx + off);
                rz[s] = __ldg(a.wz + off);
                rd[s] = __ldg(a.wd + off);
                rh[s] = __ldg(a.wh + off);
            }
        }
    }
    grid_dep_wait();     // the stage input (and its ghosts) come from earlier kernels
    grid_dep_launch();
    const T *U = a.Uin;
    T fi0 = 0, fi1 = 0, fi2 = 0, fi3 = 0;
    if (DIFF) { fi0 = U[i]; fi1 = U[N + i]; fi2 = U[2 * N + i]; fi3 = U[3 * N + i]; }
    T ux = 0, uz = 0, ud = 0, wx_ = 0, wz_ = 0, wd_ = 0, tx = 0, tz = 0, td = 0, px = 0, pz = 0, ph = 0;
    auto accumulate = [&](int j, T cx, T cz, T cd, T ch) {
        T u = U[j], w = U[N + j], t = U[2 * N + j], p = U[3 * N + j];
        if (DIFF) { u -= fi0; w -= fi1; t -= fi2; p -= fi3; }
        ux += cx * u; uz += cz * u; ud += cd * u;
        wx_ += cx * w; wz_ += cz * w; wd_ += cd * w;
        tx += cx * t; tz += cz * t; td += cd * t;
        px += cx * p; pz += cz * p; ph += ch * p;
    };
    if (PF > 0) {
#pragma unroll
        for (int s = 0; s < R; ++s)
            if (s < a.SL) accumulate(jr[s], rx[s], rz[s], rd[s], rh[s]);
    } else {
        int64_t off = off0;
#pragma unroll 4
        for (int s = 0; s < a.SL; ++s, off += stride)
            accumulate(__ldg(a.pidx + off), __ldg(a.wx + off), __ldg(a.wz + off), __ldg(a.wd + off),
                       __ldg(a.wh + off));
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
    const T u = U[i], w = U[N + i], th = U[2 * N + i], pi = U[3 * N + i];
    const unsigned char fl = a.flags[i];
    const T cpth = a.cp * (a.theta_bar + th);
    T k[4];
    k[0] = -u * ux - w * uz - cpth * px + ud;
    k[1] = -u * wx_ - w * wz_ - cpth * pz + a.g_over_tb * th + wd_;
    k[2] = -u * tx - w * tz + td;
    k[3] = -u * px - w * (a.dpibar + pz) - a.rd_cv * (a.pibar[i] + pi) * (ux + wz_) + ph;
    if (fl & 1) k[1] = 0;   // w = 0 held on bottom/top walls
    if (fl & 2) k[0] = 0;   // u = 0 held on left/right walls
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (f % G != g) continue;   // lanes split the four fields' epilogues
        const T kf = k[f];
        if (a.stage < 0) {
            a.dUdt[f * a.n_prog + i] = kf;
        } else {
            const T un = a.Un[f * N + i];
            T *kp = a.K + f * a.n_prog + i;
            if (a.stage == 0) {
                *kp = a.b_stage * kf;
                a.Uout[f * N + i] = un + a.a_next * kf;
            } else if (a.stage < 3) {
                *kp += a.b_stage * kf;
                a.Uout[f * N + i] = un + a.a_next * kf;
            } else {
                a.Uout[f * N + i] = un + (*kp + a.b_stage * kf);
            }
        }
    }
}

template <class T>
struct AdvArgs {
    const T *Uin, *Un;
    T *Uout, *K, *dUdt;
    const int32_t *pidx;
    const T *wa, *wh;
    int64_t n_prog;
    int SL, stage;
    T a_next, b_stage;
    const double *tdev;   // device time (graph replays) or nullptr
    double t_host, t_frac_dt, period_T;
};

template <class T, int G>
__global__ void __launch_bounds__(256) adv_stage_kernel(AdvArgs<T> a) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int g = (int)(tid % G);
    int64_t i = tid / G;
    const bool live = i < a.n_prog;
    if (!live) i = a.n_prog - 1;
    grid_dep_wait();
    grid_dep_launch();
    T sa = 0, sh = 0;
    const int64_t stride = a.n_prog * G;
    int64_t off = i * G + g;
#pragma unroll 4
    for (int s = 0; s < a.SL; ++s, off += stride) {
        const int j = __ldg(a.pidx + off);
        const T v = a.Uin[j];
        sa += __ldg(a.wa + off) * v;
        sh += __ldg(a.wh + off) * v;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o, G);
        sh += __shfl_xor_sync(0xffffffffu, sh, o, G);
    }
    if (!live || g != 0) return;
    // velocity time factor c(t) = cos(pi t / T) at this stage's time
    double t = (a.tdev ? *a.tdev : a.t_host) + a.t_frac_dt;
    const T c = (T)cos(3.141592653589793 * t / a.period_T);
    const T kf = c * sa + sh;
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

// Packs FP64 weights [ops][n_prog][n] into [n_packed][SL][n_prog][G] of T.
// comb[q][o]: coefficient of weight block o in packed operator q.
template <class T>
__global__ void pack_kernel(const double *__restrict__ w64, const int32_t *__restrict__ idx, int64_t n_prog,
                            int n, int nops, int first, int n_slots, int SL, int G, int n_packed,
                            const double *__restrict__ comb, T *__restrict__ pw, int32_t *__restrict__ pidx) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t total = (int64_t)SL * G * n_prog;
    if (t >= total) return;
    int64_t i = t / ((int64_t)SL * G);
    int slot = (int)(t - i * SL * G);
    int s = slot / G, g = slot - s * G;
    int64_t dst = ((int64_t)s * n_prog + i) * G + g;
    if (slot < n_slots) {
        int k = slot + first;
        pidx[dst] = idx[i * n + k];
        for (int q = 0; q < n_packed; ++q) {
            double v = 0.0;
            for (int o = 0; o < nops; ++o) {
                double c = comb[q * nops + o];
                if (c != 0.0) v += c * w64[((int64_t)o * n_prog + i) * n + k];
            }
            pw[(int64_t)q * total + dst] = (T)v;
        }
    } else {
        pidx[dst] = (int32_t)i;
        for (int q = 0; q < n_packed; ++q) pw[(int64_t)q * total + dst] = (T)0;
    }
}

// Advection: packed block 0 = flux-form weights -(Dx_ij U(x_j) + Dy_ij V(x_j)),
// block 1 = (-1)^(k+1) gamma Delta^k weights; columns folded onto the source
// node of reflected nodes (Sec. 6.1).  Weight blocks in w64: Dx, Dy, Delta^k.
template <class T>
__global__ void pack_adv_kernel(const double *__restrict__ w64, const int32_t *__restrict__ idx, int64_t n_prog,
                                int n, int has_hv, double hvc, const double *__restrict__ Uv,
                                const double *__restrict__ Vv, const int32_t *__restrict__ src, int SL, int G,
                                T *__restrict__ pw, int32_t *__restrict__ pidx) {
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
        pw[dst] = (T)(-(dx * Uv[j] + dy * Vv[j]));
        pw[total + dst] = has_hv ? (T)(hvc * w64[((int64_t)2 * n_prog + i) * n + slot]) : (T)0;
    } else {
        pidx[dst] = (int32_t)i;
        pw[dst] = (T)0;
        pw[total + dst] = (T)0;
    }
}

template <class T>
__global__ void minmax_kernel(const T *U, int64_t n_all, int64_t n_prog, int F, double *out, int *bad) {
    // out[f*2+0] min, out[f*2+1] max via ordered-int atomics on doubles
    for (int f = 0; f < F; ++f) {
        double lo = INFINITY, hi = -INFINITY;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_prog; i += (int64_t)gridDim.x * blockDim.x) {
            double v = (double)U[f * n_all + i];
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
void launch_ns_g(const NSArgs<T> &a, cudaStream_t s, bool pdl) {
    constexpr bool kDiff = sizeof(T) == 4;   // FP32: difference form; FP64: plain sums
    const dim3 grid(div_up(a.n_prog * G, 256)), blk(256);
    launch_kernel(ns_stage_kernel<T, G, kDiff, PF>, grid, blk, s, pdl, a);
}

template <class T>
void launch_ns(const NSArgs<T> &a, int G, int pf, cudaStream_t s, bool pdl) {
    if (pf > 0 && a.SL > kPrefetch) RBF_FAIL(RBF_E_ARG, "prefetch variant needs <= %d slots per lane", kPrefetch);
    switch (G * 2 + (pf > 0)) {
        case 2: launch_ns_g<T, 1, 0>(a, s, pdl); break;
        case 3: launch_ns_g<T, 1, kPrefetch>(a, s, pdl); break;
        case 4: launch_ns_g<T, 2, 0>(a, s, pdl); break;
        case 5: launch_ns_g<T, 2, kPrefetch>(a, s, pdl); break;
        case 8: launch_ns_g<T, 4, 0>(a, s, pdl); break;
        case 9: launch_ns_g<T, 4, kPrefetch>(a, s, pdl); break;
        case 16: launch_ns_g<T, 8, 0>(a, s, pdl); break;
        case 17: launch_ns_g<T, 8, kPrefetch>(a, s, pdl); break;
        default: RBF_FAIL(RBF_E_ARG, "threads per node %d not in {1,2,4,8}", G);
    }
}

template <class T>
void launch_adv(const AdvArgs<T> &a, int G, cudaStream_t s, bool pdl) {
    const dim3 grid(div_up(a.n_prog * G, 256)), blk(256);
    switch (G) {
        case 1: launch_kernel(adv_stage_kernel<T, 1>, grid, blk, s, pdl, a); break;
        case 2: launch_kernel(adv_stage_kernel<T, 2>, grid, blk, s, pdl, a); break;
        case 4: launch_kernel(adv_stage_kernel<T, 4>, grid, blk, s, pdl, a); break;
        case 8: launch_kernel(adv_stage_kernel<T, 8>, grid, blk, s, pdl, a); break;
        default: RBF_FAIL(RBF_E_ARG, "threads per node %d not in {1,2,4,8}", G);
    }
}

template <class T>
NSArgs<T> ns_args(Problem &pb) {
    NSArgs<T> a{};
    const int64_t total = (int64_t)pb.SL * pb.G * pb.n_prog;
    const T *pw = (const T *)pb.pw.p;
    a.pidx = pb.pidx.p;
    a.wx = pw;
    a.wz = pw + total;
    a.wd = pw + 2 * total;
    a.wh = pw + 3 * total;
    a.pibar = (const T *)pb.pibar.p;
    a.flags = pb.flags.p;
    a.n_prog = pb.n_prog;
    a.n_all = pb.n_all;
    a.SL = pb.SL;
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
    a.wh = pw + total;
    a.n_prog = pb.n_prog;
    a.SL = pb.SL;
    a.period_T = pb.period_T;
    return a;
}

// RK4 coefficients: stage s writes U_n + a[s] dt k_s and accumulates b[s] dt k_s
const double kA[4] = {0.5, 0.5, 1.0, 0.0};
const double kB[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

template <class T>
void rk4_ns(Problem &pb, double dt, T *U, cudaStream_t s, bool rec, int step) {
    NSArgs<T> a = ns_args<T>(pb);
    T *S0 = (T *)pb.S0.p, *S1 = (T *)pb.S1.p;
    T *in[4] = {U, S0, S1, S0};
    T *out[4] = {S0, S1, S0, U};
    a.Un = U;
    a.K = (T *)pb.K.p;
    for (int st = 0; st < 4; ++st) {
        enqueue_ghost_fill(pb, in[st], s);
        a.Uin = in[st];
        a.Uout = out[st];
        a.stage = st;
        a.a_next = (T)(kA[st] * dt);
        a.b_stage = (T)(kB[st] * dt);
        if (rec) RBF_CUDA(cudaEventRecordWithFlags(pb.rhs_ev[(step * 4 + st) * 2], s, cudaEventRecordExternal));
        launch_ns<T>(a, pb.G, pb.pf, s, pb.pdl && !rec);
        if (rec) RBF_CUDA(cudaEventRecordWithFlags(pb.rhs_ev[(step * 4 + st) * 2 + 1], s, cudaEventRecordExternal));
    }
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
    pb.SL = div_up(pb.n_slots, pb.G);
    const int64_t total = (int64_t)pb.SL * pb.G * pb.n_prog;
    pb.pidx.alloc(total);
    if (pb.kind == kAdvection) {
        pb.n_packed = 2;
        pb.pw.alloc((size_t)2 * total * pb.tsize());
        const int has_hv = nops > 2;
        if (pb.precision == 64)
            pack_adv_kernel<double><<<div_up(total, 256), 256, 0, pb.st>>>(
                pb.w64.p, pb.idx.p, pb.n_prog, pb.n, has_hv, pb.hvc, pb.vel.p, pb.vel.p + pb.n_all, pb.src.p, pb.SL,
                pb.G, (double *)pb.pw.p, pb.pidx.p);
        else
            pack_adv_kernel<float><<<div_up(total, 256), 256, 0, pb.st>>>(
                pb.w64.p, pb.idx.p, pb.n_prog, pb.n, has_hv, pb.hvc, pb.vel.p, pb.vel.p + pb.n_all, pb.src.p, pb.SL,
                pb.G, (float *)pb.pw.p, pb.pidx.p);
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
                                                                   pb.n_slots, pb.SL, pb.G, pb.n_packed, dcomb.p,
                                                                   (double *)pb.pw.p, pb.pidx.p);
    else
        pack_kernel<float><<<div_up(total, 256), 256, 0, pb.st>>>(pb.w64.p, pb.idx.p, pb.n_prog, pb.n, nops, pb.diff,
                                                                  pb.n_slots, pb.SL, pb.G, pb.n_packed, dcomb.p,
                                                                  (float *)pb.pw.p, pb.pidx.p);
    RBF_CHECK_LAUNCH();
    RBF_CUDA(cudaStreamSynchronize(pb.st));
}

void enqueue_rk4_step(Problem &pb, double t, double dt, void *U, cudaStream_t s, bool rec, int step) {
    const bool tdev = (s == pb.cap);
    if (pb.kind == kNS) {
        if (pb.precision == 64) rk4_ns<double>(pb, dt, (double *)U, s, rec, step);
        else rk4_ns<float>(pb, dt, (float *)U, s, rec, step);
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

// Autotuner: times the stage kernel for every (threads per node, register
// prefetch) choice on the problem's own operators, repacking for each lane
// count, and keeps the fastest.  NS only; advection picks G the same way.
void autotune_threads_per_node(Problem &pb) {
    const int cands[4] = {1, 2, 4, 8};
    float best = 1e30f;
    int bestG = 4, bestPf = 0;
    cudaEvent_t e0, e1;
    RBF_CUDA(cudaEventCreate(&e0));
    RBF_CUDA(cudaEventCreate(&e1));
    const size_t ts = pb.tsize();
    DevBuf<unsigned char> U((size_t)pb.F * (pb.kind == kNS ? pb.n_all : pb.n_prog) * ts);
    DevBuf<unsigned char> D((size_t)pb.F * pb.n_prog * ts);
    RBF_CUDA(cudaMemsetAsync(U.p, 0, U.bytes(), pb.st));
    for (int G : cands) {
        pb.G = G;
        pack_operators(pb);
        for (int pf : {0, kPrefetch}) {
            if (pf > 0 && (pb.kind != kNS || pb.SL > kPrefetch)) continue;
            pb.pf = pf;
            float ms = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                RBF_CUDA(cudaEventRecord(e0, pb.st));
                for (int it = 0; it < 10; ++it) {
                    if (pb.kind == kNS) {
                        if (pb.precision == 64) {
                            NSArgs<double> a = ns_args<double>(pb);
                            a.Uin = (const double *)U.p; a.dUdt = (double *)D.p; a.stage = -1;
                            launch_ns<double>(a, G, pf, pb.st, false);
                        } else {
                            NSArgs<float> a = ns_args<float>(pb);
                            a.Uin = (const float *)U.p; a.dUdt = (float *)D.p; a.stage = -1;
                            launch_ns<float>(a, G, pf, pb.st, false);
                        }
                    } else {
                        enqueue_rhs(pb, 0.0, U.p, D.p, pb.st);
                    }
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
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pb.G = bestG;
    pb.pf = bestPf;
    pack_operators(pb);
}

void minmax(Problem &pb, const void *U, double *out) {
    const int64_t stride = pb.kind == kNS ? pb.n_all : pb.n_prog;
    DevBuf<double> d(2 * pb.F);
    DevBuf<int> bad(1);
    std::vector<long long> init(2 * pb.F);
    for (int f = 0; f < pb.F; ++f) {
        init[2 * f] = 0x7fffffffffffffffLL;
        init[2 * f + 1] = (long long)0x8000000000000000ULL;
    }
    RBF_CUDA(cudaMemcpyAsync(d.p, init.data(), d.bytes(), cudaMemcpyHostToDevice, pb.st));
    RBF_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), pb.st));
    if (pb.precision == 64) minmax_kernel<double><<<128, 256, 0, pb.st>>>((const double *)U, stride, pb.n_prog, pb.F, d.p, bad.p);
    else minmax_kernel<float><<<128, 256, 0, pb.st>>>((const float *)U, stride, pb.n_prog, pb.F, d.p, bad.p);
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
