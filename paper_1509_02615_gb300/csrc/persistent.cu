// a4 + a5 + a7 in one launch: a whole rbf_run (n_steps classical RK4 steps,
// four stages each, the ghost solve of Sec. 5.2 before every stage) as one
// cooperative kernel, for problems small enough that all their nodes fit one
// co-resident grid (one CTA per SM).
//
// Each CTA owns `chunk` consecutive nodes.  Every record its nodes' stencils
// read is listed once per CTA (its halo: own nodes first, then the others in
// index order), and the packed slots refer to positions in that list.  Per
// stage a CTA copies its halo records into shared memory with one round of
// independent L2 loads, then evaluates the fused right-hand side of
// Eqs. (uEq)-(piEq) with every gather served from shared memory.  With
// R > 0 a lane also keeps its packed operators (R 16-byte vectors of each
// of the four weight blocks and of the halo positions) in registers for the
// whole run; the step-start state U_n and the RK4 accumulator of its node
// live in registers too.
//
// Phases of one stage, separated by grid barriers:
//   A  ghost residuals b - W_I u_I - W_B u_B (8 lanes per wall row),
//   B  ghost values u_G = W_G^{-1} r (one warp per class and position),
//   C  halo copy, stencil sums, tendencies and the RK4 update.
// The arithmetic of each phase (operand order, lane reductions, epilogue)
// is that of the launch-per-phase kernels with the same lane count, so both
// run modes give the same numbers.
//
// Every barrier wait is bounded: after spin_limit polls a CTA raises the
// abort flag; every other CTA leaves at its next barrier, the launch ends,
// and the host reports RBF_E_TIMEOUT.  No wait can outlive the launch.
#include <algorithm>
#include <cstring>
#include <vector>

#include "problem.cuh"
#include "records.cuh"

namespace rbf {

namespace {

template <class T>
struct PV;
template <>
struct PV<float> {
    static constexpr int V = 4;
    using W = float4;
    using L = ushort4;
    __device__ static float at(const float4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
    __device__ static int at(const ushort4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
};
template <>
struct PV<double> {
    static constexpr int V = 2;
    using W = double2;
    using L = ushort2;
    __device__ static double at(const double2 &v, int k) { return k == 0 ? v.x : v.y; }
    __device__ static int at(const ushort2 &v, int k) { return k == 0 ? v.x : v.y; }
};

// Records written during the launch are read through L2 (.cg), never through
// the non-coherent path.
__device__ __forceinline__ Rec<float> ld_rec_cg(const float *U, int64_t j) {
    const float4 v = __ldcg(reinterpret_cast<const float4 *>(U) + j);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Rec<double> ld_rec_cg(const double *U, int64_t j) {
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(U) + 2 * j);
    const double2 b = __ldcg(reinterpret_cast<const double2 *>(U) + 2 * j + 1);
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st_rec(float *U, int64_t j, const Rec<float> &r) {
    reinterpret_cast<float4 *>(U)[j] = make_float4(r.u, r.w, r.t, r.p);
}
__device__ __forceinline__ void st_rec(double *U, int64_t j, const Rec<double> &r) {
    reinterpret_cast<double2 *>(U)[2 * j] = make_double2(r.u, r.w);
    reinterpret_cast<double2 *>(U)[2 * j + 1] = make_double2(r.t, r.p);
}
__device__ __forceinline__ Rec<float> sh_rec(const float *S, int j) {
    const float4 v = reinterpret_cast<const float4 *>(S)[j];
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Rec<double> sh_rec(const double *S, int j) {
    const double2 a = reinterpret_cast<const double2 *>(S)[2 * j];
    const double2 b = reinterpret_cast<const double2 *>(S)[2 * j + 1];
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void sh_store(float *S, int j, const Rec<float> &r) {
    reinterpret_cast<float4 *>(S)[j] = make_float4(r.u, r.w, r.t, r.p);
}
__device__ __forceinline__ void sh_store(double *S, int j, const Rec<double> &r) {
    reinterpret_cast<double2 *>(S)[2 * j] = make_double2(r.u, r.w);
    reinterpret_cast<double2 *>(S)[2 * j + 1] = make_double2(r.t, r.p);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(int *p, int v) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier with a bounded wait.  `target` counts the arrivals expected
// so far (gridDim.x per barrier on top of the counter's value at launch; the
// comparison tolerates wrap-around, so the counter is never reset between
// launches).
// Returns false if this or another CTA gave up; the caller then returns.
__device__ bool grid_barrier(unsigned *arrive, int *abort, unsigned &target, long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        __threadfence();
        red_release_add(arrive, 1u);
        int ok = 1;
        long long polls = 0;
        while ((int)(ld_acquire(arrive) - target) < 0) {
            if (ld_relaxed(abort)) { ok = 0; break; }
            if (++polls > limit) {
                st_relaxed(abort, 1);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        if (ok && ld_relaxed(abort)) ok = 0;
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class T>
struct PArgs {
    T *U, *S0, *S1;                 // node-major records [n_all][4]
    const T *pw;                    // [4][SLQ][n_prog][G][V]
    const uint16_t *lidx;           // [SLQ][n_prog][G][V]
    const int32_t *hoff, *hlist;
    const T *pibar;
    const unsigned char *flags;
    int64_t n_prog, total;          // total = SLQ * n_prog * G * V
    int SLQ, chunk;
    // ghost systems (GhostPlan)
    int64_t ng, rows;
    int npad, n_comp, n_class;
    const int32_t *gidx, *owner, *pos, *comp_of;
    const T *gw, *inv;
    T *res;
    const unsigned char *tb;
    const int64_t *comp_start, *inv_off, *grec;
    int4 cls_fields;
    T cp_tb2, gconst;
    // tendencies and RK4
    T cp, g_over_tb, theta_bar, dpibar, rd_cv;
    T an0, an1, an2, bs0, bs1, bs2, bs3;
    int64_t n_steps;
    unsigned *arrive;               // monotone arrival counter (wraps)
    unsigned base;                  // its value when this launch starts
    int *abort;
    long long spin_limit;
};

constexpr int kRowLanes = 8;   // lanes per wall row (phase A), as the ghost kernels

template <class T, int G, int R, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) rk4_persistent(const __grid_constant__ PArgs<T> a) {
    using P = PV<T>;
    using W = typename P::W;
    using L = typename P::L;
    constexpr int V = P::V;
    constexpr bool DIFF = sizeof(T) == 4;   // FP32: difference form (self slot dropped)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *halo = reinterpret_cast<T *>(smem_raw);

    const int c = blockIdx.x;
    const int h0 = a.hoff[c], nh = a.hoff[c + 1] - h0;
    const int64_t n0 = (int64_t)c * a.chunk;
    const int cnt = (int)min((int64_t)a.chunk, a.n_prog - n0);
    const int li = threadIdx.x / G, g = threadIdx.x % G;
    const bool live = li < cnt;
    const int64_t i = live ? n0 + li : n0;   // idle lanes mirror the first node
    const int self = live ? li : 0;          // own nodes open the halo list
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);

    const int64_t stride = a.n_prog * G;     // in vectors, between consecutive q
    const int64_t off0 = i * G + g;
    const W *wx = reinterpret_cast<const W *>(a.pw);
    const W *wz = reinterpret_cast<const W *>(a.pw + a.total);
    const W *wd = reinterpret_cast<const W *>(a.pw + 2 * a.total);
    const W *wh = reinterpret_cast<const W *>(a.pw + 3 * a.total);
    const L *lx = reinterpret_cast<const L *>(a.lidx);
    constexpr int RR = R > 0 ? R : 1;
    L jr[RR];
    W rx[RR], rz[RR], rd[RR], rh[RR];
    if (R > 0) {
#pragma unroll
        for (int q = 0; q < RR; ++q) {
            if (q < a.SLQ) {
                const int64_t off = off0 + q * stride;
                jr[q] = __ldg(lx + off);
                rx[q] = __ldg(wx + off);
                rz[q] = __ldg(wz + off);
                rd[q] = __ldg(wd + off);
                rh[q] = __ldg(wh + off);
            }
        }
    }
    const T pib = __ldg(a.pibar + i);
    const unsigned char fl = __ldg(a.flags + i);
    T un[4], K[4] = {0, 0, 0, 0};
    {
        const Rec<T> r0 = ld_rec_cg(a.U, i);
        un[0] = r0.u; un[1] = r0.w; un[2] = r0.t; un[3] = r0.p;
    }
    unsigned target = a.base;

    for (int64_t step = 0; step < a.n_steps; ++step) {
        for (int st = 0; st < 4; ++st) {
            T *Uin = st == 0 ? a.U : st == 2 ? a.S1 : a.S0;
            T *Uout = st == 0 ? a.S0 : st == 1 ? a.S1 : st == 2 ? a.S0 : a.U;
            if (a.rows > 0) {
                // ---- A: ghost residuals, all four fields per row -------------
                const int per = a.npad / kRowLanes;
                for (int64_t e = gwarp * 32 + lane; e < ((a.rows * kRowLanes + 31) & ~(int64_t)31);
                     e += nwarps * 32) {
                    int64_t r = e / kRowLanes;
                    const int ln = (int)(e % kRowLanes);
                    const bool rl = r < a.rows;
                    if (!rl) r = a.rows - 1;
                    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
                    for (int t = 0; t < per; ++t) {
                        const int64_t o = r * a.npad + ln + kRowLanes * t;
                        const Rec<T> v = ld_rec_cg(Uin, __ldg(a.gidx + o));
                        a0 += __ldg(a.gw + o) * v.u;
                        a1 += __ldg(a.gw + a.ng * a.npad + o) * v.w;
                        a2 += __ldg(a.gw + 2 * a.ng * a.npad + o) * v.t;
                        a3 += __ldg(a.gw + 3 * a.ng * a.npad + o) * v.p;
                    }
#pragma unroll
                    for (int o = kRowLanes / 2; o > 0; o >>= 1) {
                        a0 += __shfl_xor_sync(0xffffffffu, a0, o, kRowLanes);
                        a1 += __shfl_xor_sync(0xffffffffu, a1, o, kRowLanes);
                        a2 += __shfl_xor_sync(0xffffffffu, a2, o, kRowLanes);
                        a3 += __shfl_xor_sync(0xffffffffu, a3, o, kRowLanes);
                    }
                    if (rl && ln < 4) {
                        const T acc = ln == 0 ? a0 : ln == 1 ? a1 : ln == 2 ? a2 : a3;
                        T b = 0;
                        if (ln == 3 && __ldg(a.tb + r)) {
                            // pi'_z = g theta' / (c_p theta_bar (theta_bar + theta')) at the wall node
                            const T th = __ldcg(Uin + (int64_t)__ldg(a.owner + r) * 4 + 2);
                            b = a.gconst * th / (a.cp_tb2 + a.cp_tb2 / a.theta_bar * th);
                        }
                        a.res[ln * a.ng + __ldg(a.pos + r)] = b - acc;
                    }
                }
                if (!grid_barrier(a.arrive, a.abort, target, a.spin_limit)) return;
                // ---- B: ghost values, one warp per (class, position) ---------
                for (int64_t w = gwarp; w < (int64_t)a.n_class * a.rows; w += nwarps) {
                    const int cls = (int)(w / a.rows);
                    const int64_t q = w - (int64_t)cls * a.rows;
                    const int cc = __ldg(a.comp_of + q);
                    const int64_t s0 = __ldg(a.comp_start + cc);
                    const int m = (int)(__ldg(a.comp_start + cc + 1) - s0);
                    const int row = (int)(q - s0);
                    const T *Ainv = a.inv + __ldg(a.inv_off + cls * a.n_comp + cc) + (int64_t)row * m;
                    const int fm = cls == 0 ? a.cls_fields.x : cls == 1 ? a.cls_fields.y
                                 : cls == 2 ? a.cls_fields.z : a.cls_fields.w;
                    const int64_t rec = __ldg(a.grec + q);
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        if (!(fm & (1 << f))) continue;
                        const T *rr = a.res + f * a.ng + s0;
                        T s = 0;
                        for (int j = lane; j < m; j += 32) s += __ldg(Ainv + j) * __ldcg(rr + j);
                        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                        if (lane == 0) Uin[rec * 4 + f] = s;
                    }
                }
                if (!grid_barrier(a.arrive, a.abort, target, a.spin_limit)) return;
            }
            // ---- C: halo copy, stencil sums, tendencies, RK4 update ----------
            for (int h = threadIdx.x; h < nh; h += blockDim.x)
                sh_store(halo, h, ld_rec_cg(Uin, __ldg(a.hlist + h0 + h)));
            __syncthreads();
            Rec<T> fi = {0, 0, 0, 0};
            if (DIFF) fi = sh_rec(halo, self);
            T ux = 0, uz = 0, ud = 0, wx_ = 0, wz_ = 0, wd_ = 0, tx = 0, tz = 0, td = 0, px = 0, pz = 0, ph = 0;
            auto vec = [&](const L &jv, const W &cx, const W &cz, const W &cd, const W &ch) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    Rec<T> r = sh_rec(halo, P::at(jv, v));
                    if (DIFF) { r.u -= fi.u; r.w -= fi.w; r.t -= fi.t; r.p -= fi.p; }
                    const T x = P::at(cx, v), z = P::at(cz, v), d = P::at(cd, v), hh = P::at(ch, v);
                    ux += x * r.u; uz += z * r.u; ud += d * r.u;
                    wx_ += x * r.w; wz_ += z * r.w; wd_ += d * r.w;
                    tx += x * r.t; tz += z * r.t; td += d * r.t;
                    px += x * r.p; pz += z * r.p; ph += hh * r.p;
                }
            };
            if (R > 0) {
#pragma unroll
                for (int q = 0; q < RR; ++q)
                    if (q < a.SLQ) vec(jr[q], rx[q], rz[q], rd[q], rh[q]);
            } else {
                int64_t off = off0;
#pragma unroll 2
                for (int q = 0; q < a.SLQ; ++q, off += stride)
                    vec(__ldg(lx + off), __ldg(wx + off), __ldg(wz + off), __ldg(wd + off), __ldg(wh + off));
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
            const Rec<T> cr = DIFF ? fi : sh_rec(halo, self);
            const T cpth = a.cp * (a.theta_bar + cr.t);
            T k[4];
            k[0] = -cr.u * ux - cr.w * uz - cpth * px + ud;
            k[1] = -cr.u * wx_ - cr.w * wz_ - cpth * pz + a.g_over_tb * cr.t + wd_;
            k[2] = -cr.u * tx - cr.w * tz + td;
            k[3] = -cr.u * px - cr.w * (a.dpibar + pz) - a.rd_cv * (pib + cr.p) * (ux + wz_) + ph;
            if (fl & 1) k[1] = 0;   // w = 0 held on bottom/top walls
            if (fl & 2) k[0] = 0;   // u = 0 held on left/right walls
            const T an = st == 0 ? a.an0 : st == 1 ? a.an1 : a.an2;
            const T bs = st == 0 ? a.bs0 : st == 1 ? a.bs1 : st == 2 ? a.bs2 : a.bs3;
            T o4[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const T kf = k[f];
                if (st == 0) {
                    K[f] = bs * kf;
                    o4[f] = un[f] + an * kf;
                } else if (st < 3) {
                    K[f] += bs * kf;
                    o4[f] = un[f] + an * kf;
                } else {
                    o4[f] = un[f] + (K[f] + bs * kf);
                }
            }
            if (st == 3) {
#pragma unroll
                for (int f = 0; f < 4; ++f) un[f] = o4[f];
            }
            if (live && g == 0) st_rec(Uout, i, Rec<T>{o4[0], o4[1], o4[2], o4[3]});
            const bool last = step + 1 == a.n_steps && st == 3;
            if (!last && !grid_barrier(a.arrive, a.abort, target, a.spin_limit)) return;
        }
    }
}

// Kernel variants: (lanes per node, operand vectors held in registers,
// thread limit).  The register variant covers FP32 stencils of up to 36
// packed slots with one lane per node (255 registers, no spills); the others
// read their operands each stage.
struct Variant {
    int G, R, maxt;
    void *fn;
};

template <class T>
std::vector<Variant> variants() {
    if constexpr (sizeof(T) == 4) {
        return {{1, 9, 256, (void *)rk4_persistent<float, 1, 9, 256>},
                {1, 0, 1024, (void *)rk4_persistent<float, 1, 0, 1024>},
                {2, 0, 1024, (void *)rk4_persistent<float, 2, 0, 1024>},
                {4, 0, 1024, (void *)rk4_persistent<float, 4, 0, 1024>}};
    } else {
        return {{1, 0, 512, (void *)rk4_persistent<double, 1, 0, 512>},
                {2, 0, 512, (void *)rk4_persistent<double, 2, 0, 512>},
                {4, 0, 1024, (void *)rk4_persistent<double, 4, 0, 1024>}};
    }
}

template <class T>
PArgs<T> pargs(Problem &pb, T *U, double dt, int64_t n_steps) {
    const PersistPlan &ps = pb.ps;
    const GhostPlan &gh = pb.gh;
    PArgs<T> a{};
    a.U = U;
    a.S0 = (T *)pb.S0.p;
    a.S1 = (T *)pb.S1.p;
    a.pw = (const T *)ps.pw.p;
    a.lidx = ps.lidx.p;
    a.hoff = ps.hoff.p;
    a.hlist = ps.hlist.p;
    a.pibar = (const T *)pb.pibar.p;
    a.flags = pb.flags.p;
    a.n_prog = pb.n_prog;
    a.total = (int64_t)ps.SLQ * pb.n_prog * ps.G * ps.V;
    a.SLQ = ps.SLQ;
    a.chunk = ps.chunk;
    a.ng = gh.n_ghost;
    a.rows = gh.n_ghost > 0 ? gh.rows : 0;
    a.npad = gh.npad;
    a.n_comp = gh.n_comp;
    a.n_class = gh.n_class;
    a.gidx = gh.gidx.p;
    a.owner = gh.owner.p;
    a.pos = gh.pos.p;
    a.comp_of = gh.comp_of.p;
    a.gw = (const T *)gh.gw.p;
    a.inv = (const T *)gh.inv.p;
    a.res = (T *)gh.res.p;
    a.tb = gh.tb.p;
    a.comp_start = gh.comp_start.p;
    a.inv_off = gh.inv_off.p;
    a.grec = gh.grec.p;
    int fields[4] = {0, 0, 0, 0};
    for (int f = 0; f < 4; ++f) fields[gh.field_class[f]] |= 1 << f;
    a.cls_fields = make_int4(fields[0], fields[1], fields[2], fields[3]);
    a.cp_tb2 = (T)(pb.cp * pb.theta_bar * pb.theta_bar);
    a.gconst = (T)pb.g;
    a.cp = (T)pb.cp;
    a.g_over_tb = (T)(pb.g / pb.theta_bar);
    a.theta_bar = (T)pb.theta_bar;
    a.dpibar = (T)(-pb.g / (pb.cp * pb.theta_bar));
    a.rd_cv = (T)(pb.rd / pb.cv);
    // RK4 coefficients: stage s writes U_n + a[s] dt k_s, accumulates b[s] dt k_s
    a.an0 = (T)(0.5 * dt);
    a.an1 = (T)(0.5 * dt);
    a.an2 = (T)(1.0 * dt);
    a.bs0 = (T)(1.0 / 6.0 * dt);
    a.bs1 = (T)(1.0 / 3.0 * dt);
    a.bs2 = (T)(1.0 / 3.0 * dt);
    a.bs3 = (T)(1.0 / 6.0 * dt);
    a.n_steps = n_steps;
    a.arrive = ps.arrive.p;
    a.base = ps.base;
    a.abort = ps.abort.p;
    a.spin_limit = ps.spin_limit;
    return a;
}

void *variant_fn(const PersistPlan &ps, int precision) {
    const std::vector<Variant> v = precision == 64 ? variants<double>() : variants<float>();
    for (const Variant &x : v)
        if (x.G == ps.G && x.R == ps.R && x.maxt == ps.maxt) return x.fn;
    return nullptr;
}

}  // namespace

bool persistent_plan(Problem &pb, int G) {
    PersistPlan &ps = pb.ps;
    ps.ready = false;
    if (pb.kind != kNS) return false;
    int dev = 0, coop = 0, smem_optin = 0;
    RBF_CUDA(cudaGetDevice(&dev));
    RBF_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    RBF_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (!coop) return false;
    const int nsm = sm_count();
    const int chunk = div_up(pb.n_prog, nsm);
    const int threads = div_up((int64_t)chunk * G, 32) * 32;
    if (threads > 1024) return false;

    // operators packed for G lanes, kept beside the launch-per-stage packing
    const int G0 = pb.G, pf0 = pb.pf, SLQ0 = pb.SLQ, SL0 = pb.SL, V0 = pb.V;
    DevBuf<int32_t> pidx0 = std::move(pb.pidx);
    DevBuf<unsigned char> pw0 = std::move(pb.pw);
    auto restore = [&] {
        pb.pidx = std::move(pidx0);
        pb.pw = std::move(pw0);
        pb.G = G0; pb.pf = pf0; pb.SLQ = SLQ0; pb.SL = SL0; pb.V = V0;
    };
    std::vector<int32_t> hp;
    try {
        pb.G = G;
        pack_operators(pb);
        hp.resize(pb.pidx.n);
        RBF_CUDA(cudaMemcpy(hp.data(), pb.pidx.p, pb.pidx.bytes(), cudaMemcpyDeviceToHost));
    } catch (...) {
        restore();
        throw;
    }
    ps.pw = std::move(pb.pw);
    ps.G = G;
    ps.SLQ = pb.SLQ;
    ps.V = pb.V;
    restore();

    // halo lists: own nodes first, then every other record the CTA's
    // stencils read, ascending; slots refer to positions in the list
    const int grid = div_up(pb.n_prog, chunk);
    const int lanes = G * ps.V;            // slots of one node per operand vector
    std::vector<int32_t> hoff(grid + 1, 0), hlist;
    std::vector<uint16_t> lidx(hp.size());
    std::vector<int32_t> other;
    int halo_max = 0;
    for (int c = 0; c < grid; ++c) {
        const int64_t n0 = (int64_t)c * chunk, n1 = std::min<int64_t>(n0 + chunk, pb.n_prog);
        other.clear();
        for (int q = 0; q < ps.SLQ; ++q)
            for (int64_t i = n0; i < n1; ++i)
                for (int s = 0; s < lanes; ++s) {
                    const int32_t j = hp[((int64_t)q * pb.n_prog + i) * lanes + s];
                    if (j < n0 || j >= n1) other.push_back(j);
                }
        std::sort(other.begin(), other.end());
        other.erase(std::unique(other.begin(), other.end()), other.end());
        const int64_t nh = (n1 - n0) + (int64_t)other.size();
        if (nh > 65535) return false;
        halo_max = std::max<int>(halo_max, (int)nh);
        hoff[c] = (int32_t)hlist.size();
        for (int64_t i = n0; i < n1; ++i) hlist.push_back((int32_t)i);
        hlist.insert(hlist.end(), other.begin(), other.end());
        for (int q = 0; q < ps.SLQ; ++q)
            for (int64_t i = n0; i < n1; ++i)
                for (int s = 0; s < lanes; ++s) {
                    const int64_t e = ((int64_t)q * pb.n_prog + i) * lanes + s;
                    const int32_t j = hp[e];
                    const int64_t loc =
                        (j >= n0 && j < n1)
                            ? j - n0
                            : (n1 - n0) + (std::lower_bound(other.begin(), other.end(), j) - other.begin());
                    lidx[e] = (uint16_t)loc;
                }
    }
    hoff[grid] = (int32_t)hlist.size();
    const size_t smem = (size_t)halo_max * 4 * pb.tsize();
    if (smem > (size_t)smem_optin) return false;

    // kernel variant: operands in registers when they fit, else read each stage
    const std::vector<Variant> vs = pb.precision == 64 ? variants<double>() : variants<float>();
    int pick = -1;
    for (int k = 0; k < (int)vs.size(); ++k) {
        const Variant &v = vs[k];
        if (v.G != G || threads > v.maxt) continue;
        if (v.R > 0 && ps.SLQ > v.R) continue;
        if (pick < 0 || (v.R > 0 && vs[pick].R == 0)) pick = k;
    }
    if (pick < 0) return false;
    RBF_CUDA(cudaFuncSetAttribute(vs[pick].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    RBF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vs[pick].fn, threads, smem));
    if ((int64_t)per_sm * nsm < grid) return false;

    ps.R = vs[pick].R;
    ps.maxt = vs[pick].maxt;
    ps.chunk = chunk;
    ps.threads = threads;
    ps.grid = grid;
    ps.halo_max = halo_max;
    ps.halo_total = (int64_t)hlist.size();
    ps.smem = smem;
    ps.hoff.alloc(hoff.size());
    ps.hlist.alloc(hlist.size());
    ps.lidx.alloc(lidx.size());
    RBF_CUDA(cudaMemcpy(ps.hoff.p, hoff.data(), ps.hoff.bytes(), cudaMemcpyHostToDevice));
    RBF_CUDA(cudaMemcpy(ps.hlist.p, hlist.data(), ps.hlist.bytes(), cudaMemcpyHostToDevice));
    RBF_CUDA(cudaMemcpy(ps.lidx.p, lidx.data(), ps.lidx.bytes(), cudaMemcpyHostToDevice));
    RBF_CUDA(cudaStreamSynchronize(pb.st));
    if (ps.arrive.n == 0) ps.arrive.alloc(1);
    RBF_CUDA(cudaMemset(ps.arrive.p, 0, sizeof(unsigned)));
    ps.base = 0;
    if (ps.abort.n == 0) {
        ps.abort.alloc(1);
        RBF_CUDA(cudaMemset(ps.abort.p, 0, sizeof(int)));
    }
    ps.ready = true;
    return true;
}

void persistent_run(Problem &pb, double dt, int64_t n_steps, void *U, cudaStream_t s) {
    PersistPlan &ps = pb.ps;
    RBF_REQUIRE(ps.ready, "no persistent plan for this problem");
    if (n_steps <= 0) return;
    void *fn = variant_fn(ps, pb.precision);
    RBF_REQUIRE(fn != nullptr, "persistent kernel variant missing");
    if (pb.precision == 64) {
        PArgs<double> a = pargs<double>(pb, (double *)U, dt, n_steps);
        void *args[] = {&a};
        RBF_CUDA(cudaLaunchCooperativeKernel(fn, dim3(ps.grid), dim3(ps.threads), args, ps.smem, s));
    } else {
        PArgs<float> a = pargs<float>(pb, (float *)U, dt, n_steps);
        void *args[] = {&a};
        RBF_CUDA(cudaLaunchCooperativeKernel(fn, dim3(ps.grid), dim3(ps.threads), args, ps.smem, s));
    }
    // barriers of this launch: 3 per stage with ghosts, 1 without, minus the last
    const int64_t per_stage = pb.gh.n_ghost > 0 && pb.gh.rows > 0 ? 3 : 1;
    ps.base += (unsigned)((uint64_t)ps.grid * (uint64_t)(4 * per_stage * n_steps - 1));
}

void persistent_check(Problem &pb) {
    if (pb.ps.abort.n == 0) return;
    int v = 0;
    RBF_CUDA(cudaMemcpy(&v, pb.ps.abort.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (v) {
        // an aborted launch left the arrival count unknown: restart it
        RBF_CUDA(cudaMemset(pb.ps.arrive.p, 0, sizeof(unsigned)));
        pb.ps.base = 0;
        RBF_CUDA(cudaMemset(pb.ps.abort.p, 0, sizeof(int)));
        RBF_FAIL(RBF_E_TIMEOUT,
                 "a grid barrier of the persistent kernel gave up after %lld polls; the state is partially "
                 "updated",
                 pb.ps.spin_limit);
    }
}

}  // namespace rbf
