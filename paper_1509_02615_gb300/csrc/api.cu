// extern "C" entry points of librbffd (declared in include/rbffd.h): problem
// construction, stepping, graph replay and queries.  Every call is guarded:
// library failures become RBF_E_* codes with a message in rbf_last_error().
#include <cmath>
#include <cstring>

#include "problem.cuh"

namespace rbf {

namespace {
thread_local std::string g_last_error;
}

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

const char *last_error() { return g_last_error.c_str(); }

int sm_count() {
    int dev = 0, n = 0;
    RBF_CUDA(cudaGetDevice(&dev));
    RBF_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    return n;
}

Problem::~Problem() {
    if (graph) cudaGraphExecDestroy(graph);
    for (cudaEvent_t e : rhs_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : {ev_fork, ev_w[0], ev_w[1], ev_r[0], ev_r[1]})
        if (e) cudaEventDestroy(e);
    if (side) cudaStreamDestroy(side);
    if (cap) cudaStreamDestroy(cap);
}

namespace {

template <class T>
__global__ void pibar_kernel(const double *z, int64_t n_prog, double g, double cp, double theta_bar, T *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n_prog) out[i] = (T)(1.0 - g * z[i] / (cp * theta_bar));   // Sec. 6.3 background Exner
}

__global__ void set_time(double *t, double v) { *t = v; }

void common_setup(Problem &pb, const double *x, const double *z, int64_t n_prog, int64_t n_all, void *stream) {
    RBF_REQUIRE(n_prog >= 1 && n_all >= n_prog, "need 1 <= n_prog <= n_all (got %lld, %lld)", (long long)n_prog,
                (long long)n_all);
    RBF_REQUIRE(n_all < ((int64_t)1 << 31), "n_all exceeds int32 indexing");
    RBF_REQUIRE(x && z, "null coordinates");
    for (int64_t i = 0; i < n_all; ++i)
        RBF_REQUIRE(std::isfinite(x[i]) && std::isfinite(z[i]), "non-finite coordinate at node %lld", (long long)i);
    int ndev = 0;
    RBF_CUDA(cudaGetDeviceCount(&ndev));
    RBF_REQUIRE(ndev > 0, "no CUDA device");
    pb.st = as_stream(stream);
    pb.n_prog = n_prog;
    pb.n_all = n_all;
    RBF_CUDA(cudaStreamCreateWithFlags(&pb.cap, cudaStreamNonBlocking));
    pb.x.alloc(n_all);
    pb.z.alloc(n_all);
    RBF_CUDA(cudaMemcpyAsync(pb.x.p, x, n_all * 8, cudaMemcpyHostToDevice, pb.st));
    RBF_CUDA(cudaMemcpyAsync(pb.z.p, z, n_all * 8, cudaMemcpyHostToDevice, pb.st));
    pb.tdev.alloc(1);
}

}  // namespace

void alloc_scratch(Problem &pb) {
    const int64_t stride = pb.kind == kNS ? pb.n_all : pb.n_prog;
    const size_t ts = pb.tsize();
    pb.S0.alloc((size_t)pb.F * stride * ts);
    pb.S1.alloc((size_t)pb.F * stride * ts);
    pb.K.alloc((size_t)pb.F * pb.n_prog * ts);
    // ghost entries of the stage buffers are written by the ghost fill; zero
    // them once so that nothing uninitialised is ever read
    RBF_CUDA(cudaMemsetAsync(pb.S0.p, 0, pb.S0.bytes(), pb.st));
    RBF_CUDA(cudaMemsetAsync(pb.S1.p, 0, pb.S1.bytes(), pb.st));
}

namespace {

void choose_threads(Problem &pb, int requested) {
    if (requested == 0) {
        autotune_threads_per_node(pb);
    } else {
        RBF_REQUIRE(requested == 1 || requested == 2 || requested == 4 || requested == 8,
                    "threads_per_node must be 0, 1, 2, 4 or 8");
        pb.G = requested;
        pack_operators(pb);
        // registers hold the operands when they fit (per-node storage only)
        pb.pf = (pb.kind == kNS && pb.SLQ <= 3 && !pb.lat.enabled) ? 3 : 0;
    }
}

}  // namespace

// Algorithmic bytes of one Navier-Stokes node-RHS of the stage kernel.
// Per-node storage: packed weights (4 operators) + index per slot, the
// node's own values, U_n, the RK4 accumulator read+write, the stage output,
// pibar and the flag byte.  Lattice storage: class nodes read a class id
// instead of their operators, irregular nodes read both, and the class table
// is read once per launch.
double ns_rhs_bytes(const Problem &pb) {
    const double ts = (double)pb.tsize(), slots = pb.n_slots;
    const double rest = 4 * ts + 4 * ts + 8 * ts + 4 * ts + ts + 1;
    const double ops = slots * (4 * ts + 4);
    if (!pb.lat.enabled) return ops + rest;
    const double cn = (double)pb.lat.class_nodes, N = (double)pb.n_prog;
    const double table = (double)pb.lat.n_cls * pb.SLQ * pb.G * pb.V * (4 * ts + 4);
    return 4 + rest + (N - cn) / N * ops + table / N;
}

namespace {

void invalidate_graph(Problem &pb) {
    if (pb.graph) cudaGraphExecDestroy(pb.graph);
    pb.graph = nullptr;
    pb.graph_U = nullptr;
    pb.graph_steps = 0;
}

// Captures `steps` RK4 steps on the private stream into an executable graph.
void capture(Problem &pb, void *U, double dt, int steps) {
    invalidate_graph(pb);
    if (pb.record_rhs_events) {
        for (cudaEvent_t e : pb.rhs_ev) cudaEventDestroy(e);
        pb.rhs_ev.assign(8 * steps, nullptr);
        for (auto &e : pb.rhs_ev) RBF_CUDA(cudaEventCreate(&e));
    }
    cudaGraph_t g = nullptr;
    RBF_CUDA(cudaStreamBeginCapture(pb.cap, cudaStreamCaptureModeThreadLocal));
    try {
        for (int s = 0; s < steps; ++s)
            enqueue_rk4_step(pb, 0.0, dt, U, pb.cap, pb.record_rhs_events, s, s == 0, s == steps - 1);
    } catch (...) {
        cudaStreamEndCapture(pb.cap, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    RBF_CUDA(cudaStreamEndCapture(pb.cap, &g));
    // node priorities: the split's wall-set launches go ahead of the others
    cudaError_t e = cudaGraphInstantiateWithFlags(&pb.graph, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    RBF_CUDA(e);
    pb.graph_U = U;
    pb.graph_dt = dt;
    pb.graph_steps = steps;
}

void run(Problem &pb, double t0, double dt, int64_t n_steps, void *U) {
    RBF_REQUIRE(U != nullptr, "null state");
    RBF_REQUIRE((reinterpret_cast<uintptr_t>(U) & 15) == 0, "state must be 16-byte aligned (node-major records)");
    RBF_REQUIRE(n_steps >= 0, "n_steps < 0");
    RBF_REQUIRE(std::isfinite(dt) && std::isfinite(t0), "non-finite time or step");
    if (n_steps == 0) return;
    if (pb.kind == kAdvection && pb.run_mode == RBF_RUN_PERSISTENT && pb.ps.ready && !pb.record_rhs_events) {
        adv_persistent_run(pb, t0, dt, n_steps, U, pb.st);
        return;
    }
    if (pb.kind == kNS && pb.run_mode == RBF_RUN_PERSISTENT && pb.ps.ready && !pb.record_rhs_events) {
        // the equations are autonomous: t0 does not enter the launch
        persistent_run(pb, dt, n_steps, U, pb.st);
        return;
    }
    const int chunk = (int)std::min<int64_t>(n_steps, pb.record_rhs_events ? 1 : 16);
    if (!pb.graph || pb.graph_U != U || pb.graph_dt != dt || pb.graph_steps != chunk) capture(pb, U, dt, chunk);
    cudaEvent_t ev;
    RBF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    // order the private stream after the caller's stream
    RBF_CUDA(cudaEventRecord(ev, pb.st));
    RBF_CUDA(cudaStreamWaitEvent(pb.cap, ev, 0));
    set_time<<<1, 1, 0, pb.cap>>>(pb.tdev.p, t0);
    RBF_CHECK_LAUNCH();
    int64_t done = 0;
    while (done + chunk <= n_steps) {
        RBF_CUDA(cudaGraphLaunch(pb.graph, pb.cap));
        done += chunk;
    }
    // remainder steps go straight onto the private stream
    for (; done < n_steps; ++done) enqueue_rk4_step(pb, t0 + done * dt, dt, U, pb.cap, false, 0);
    RBF_CUDA(cudaEventRecord(ev, pb.cap));
    RBF_CUDA(cudaStreamWaitEvent(pb.st, ev, 0));
    cudaEventDestroy(ev);   // released once the recorded work completes
}

// Times `steps` RK4 steps of the current run mode on U (best of three).
float time_run(Problem &pb, void *U, int steps) {
    cudaEvent_t e0, e1;
    RBF_CUDA(cudaEventCreate(&e0));
    RBF_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    try {
        run(pb, 0.0, 1e-3, steps, U);   // warm-up (and graph capture)
        for (int rep = 0; rep < 3; ++rep) {
            RBF_CUDA(cudaEventRecord(e0, pb.st));
            run(pb, 0.0, 1e-3, steps, U);
            RBF_CUDA(cudaEventRecord(e1, pb.st));
            RBF_CUDA(cudaEventSynchronize(e1));
            float t = 0.f;
            RBF_CUDA(cudaEventElapsedTime(&t, e0, e1));
            best = std::min(best, t);
        }
        persistent_check(pb);
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

// Run-mode autotuner of an advection problem: graph replay (with the lanes
// per node it was packed for) against the persistent kernel for 2, 4 and 8
// lanes per node (operators repacked for each) and CTAs of 64, 128 and 256
// threads, on a zero state; keeps the fastest.  lanes > 0 restricts the
// persistent candidates to that lane count.
void choose_run_mode_adv(Problem &pb, int mode, int lanes, int ctas) {
    RBF_REQUIRE(mode == RBF_RUN_AUTO || mode == RBF_RUN_GRAPH || mode == RBF_RUN_PERSISTENT,
                "unknown run mode %d", mode);
    RBF_REQUIRE(lanes == 0 || lanes == 2 || lanes == 4 || lanes == 8,
                "lanes must be 0, 2, 4 or 8 for an advection problem");
    RBF_REQUIRE(ctas == 0, "the CTA count of an advection problem follows from its lanes and CTA size (ctas = 0)");
    invalidate_graph(pb);
    if (mode == RBF_RUN_GRAPH) {
        pb.run_mode = RBF_RUN_GRAPH;
        pb.ps.ready = false;
        return;
    }
    const int G0 = pb.G;
    const size_t bytes = (size_t)pb.n_prog * pb.tsize();
    DevBuf<unsigned char> U(bytes);
    RBF_CUDA(cudaMemsetAsync(U.p, 0, bytes, pb.st));
    const int steps = 8;
    float best = 1e30f;
    int bG = 0, bT = 0;
    if (mode == RBF_RUN_AUTO) {
        pb.run_mode = RBF_RUN_GRAPH;
        pb.ps.ready = false;
        best = time_run(pb, U.p, steps);
        invalidate_graph(pb);
    }
    for (int G : {2, 4, 8}) {
        if (lanes && G != lanes) continue;
        pb.G = G;
        pack_operators(pb);
        for (int threads : {64, 128, 256}) {
            if (!adv_persistent_plan(pb, threads)) continue;
            pb.run_mode = RBF_RUN_PERSISTENT;
            const float t = time_run(pb, U.p, steps);
            if (t < best) {
                best = t;
                bG = G;
                bT = threads;
            }
        }
    }
    pb.ps.ready = false;
    pb.run_mode = RBF_RUN_GRAPH;
    if (bG == 0) {
        pb.G = G0;
        pack_operators(pb);
        RBF_REQUIRE(mode == RBF_RUN_AUTO, "the persistent kernel does not fit this problem");
        return;
    }
    pb.G = bG;
    pack_operators(pb);
    RBF_REQUIRE(adv_persistent_plan(pb, bT), "persistent plan failed");
    pb.run_mode = RBF_RUN_PERSISTENT;
    RBF_CUDA(cudaStreamSynchronize(pb.st));
}

// Run-mode autotuner: graph replay against the persistent kernel for each
// (lanes per node, CTA count) that fits, on a zero state; keeps the fastest.
// lanes > 0 restricts the persistent candidates to that lane count, ctas > 0
// to that CTA count; with both given (RBF_RUN_PERSISTENT) nothing is timed.
void choose_run_mode(Problem &pb, int mode, int lanes, int ctas) {
    if (pb.kind == kAdvection) {
        choose_run_mode_adv(pb, mode, lanes, ctas);
        return;
    }
    RBF_REQUIRE(pb.kind == kNS, "run modes apply to Navier-Stokes and advection problems");
    RBF_REQUIRE(mode == RBF_RUN_AUTO || mode == RBF_RUN_GRAPH || mode == RBF_RUN_PERSISTENT,
                "unknown run mode %d", mode);
    RBF_REQUIRE(lanes == 0 || lanes == 1 || lanes == 2 || lanes == 4, "lanes must be 0, 1, 2 or 4");
    RBF_REQUIRE(ctas >= 0, "ctas must be >= 0");
    if (mode == RBF_RUN_GRAPH) {
        pb.run_mode = RBF_RUN_GRAPH;
        return;
    }
    const int nsm = sm_count();
    std::vector<std::pair<int, int>> cands;
    for (int G : {1, 2, 4}) {
        if (lanes && G != lanes) continue;
        if (ctas) {
            cands.emplace_back(G, ctas);
            continue;
        }
        // explicit lanes without a CTA count: one CTA per SM, untimed
        if (lanes && mode == RBF_RUN_PERSISTENT) {
            cands.emplace_back(G, nsm);
            continue;
        }
        for (int div : {1, 2, 4, 8}) {
            const int c = nsm / div;
            if (c >= 1 && (div == 1 || (int64_t)c * 8 <= pb.n_prog)) cands.emplace_back(G, c);
        }
    }
    const bool timing = mode == RBF_RUN_AUTO || cands.size() > 1;
    const size_t bytes = (size_t)pb.F * pb.n_all * pb.tsize();
    DevBuf<unsigned char> U(timing ? bytes : 0);
    if (timing) RBF_CUDA(cudaMemsetAsync(U.p, 0, bytes, pb.st));
    const int steps = 8;
    float best = 1e30f;
    std::pair<int, int> pick(0, 0);
    if (mode == RBF_RUN_AUTO) {
        pb.run_mode = RBF_RUN_GRAPH;
        best = time_run(pb, U.p, steps);
        invalidate_graph(pb);
    }
    for (auto &c : cands) {
        if (!persistent_plan(pb, c.first, c.second)) continue;
        if (!timing) {
            pick = c;
            break;
        }
        pb.run_mode = RBF_RUN_PERSISTENT;
        const float t = time_run(pb, U.p, steps);
        if (t < best) {
            best = t;
            pick = c;
        }
    }
    if (pick.first == 0) {
        pb.ps.ready = false;
        pb.run_mode = RBF_RUN_GRAPH;
        RBF_REQUIRE(mode == RBF_RUN_AUTO, "the persistent kernel does not fit this problem");
        return;
    }
    if (!pb.ps.ready || pb.ps.G != pick.first || pb.ps.grid != std::min<int64_t>(pick.second, pb.n_prog))
        persistent_plan(pb, pick.first, pick.second);
    RBF_REQUIRE(pb.ps.ready, "persistent plan failed");
    pb.run_mode = RBF_RUN_PERSISTENT;
    // zero the stage buffers the timing runs wrote (ghost records included)
    RBF_CUDA(cudaMemsetAsync(pb.S0.p, 0, pb.S0.bytes(), pb.st));
    RBF_CUDA(cudaMemsetAsync(pb.S1.p, 0, pb.S1.bytes(), pb.st));
    RBF_CUDA(cudaStreamSynchronize(pb.st));
}

}  // namespace

// Hyperviscosity coefficient of a problem (Sec. 5.3): gamma_c > 0 forms
// gamma = gamma_c h^(2k - 1) (the reading of the paper's resolution-independent
// constant; see rbf_hyperviscosity_gamma); gamma_c == 0 takes gamma as given.
double resolve_gamma(double gamma, double gamma_c, double spacing, int hv_k) {
    RBF_REQUIRE(std::isfinite(gamma_c) && gamma_c >= 0.0, "gamma_c must be >= 0");
    if (gamma_c == 0.0 || hv_k < 1) return gamma;
    RBF_REQUIRE(gamma == 0.0, "give either gamma or gamma_c, not both");
    RBF_REQUIRE(std::isfinite(spacing) && spacing > 0.0, "gamma_c needs a node spacing > 0");
    return gamma_c * std::pow(spacing, 2 * hv_k - 1);
}

// Builds a Navier-Stokes problem (stencils, weights, packing, ghost systems).
// with_scratch = false leaves out the RK4 stage buffers (ensemble members
// step in their ensemble's buffers).
void build_ns(Problem &pb, const rbf_ns_params &prm, const double *x, const double *z, int64_t n_prog,
          int64_t n_all, const int32_t *kind, const int32_t *ghost_owner, void *stream, bool with_scratch) {
    RBF_REQUIRE(prm.storage == RBF_STORE_PER_NODE || prm.storage == RBF_STORE_LATTICE, "unknown storage mode %d",
                prm.storage);
    RBF_REQUIRE(prm.precision == 64 || prm.precision == 32, "precision must be 64 or 32");
    RBF_REQUIRE(prm.n_sten >= 2, "stencil size must be >= 2");
    RBF_REQUIRE(prm.mu >= 0.0 && prm.gamma >= 0.0, "mu and gamma must be >= 0");
    const double gamma = resolve_gamma(prm.gamma, prm.gamma_c, prm.spacing, prm.hv_k);
    RBF_REQUIRE(prm.theta_bar > 0.0 && prm.cp > 0.0 && prm.cv > 0.0, "bad physical constants");
    RBF_REQUIRE(kind != nullptr, "null kind");
    RBF_REQUIRE(n_all == n_prog || ghost_owner != nullptr, "ghosts need ghost_owner");
    RBF_REQUIRE(with_scratch || prm.threads_per_node != 0, "autotuning needs the stage buffers");
    pb.kind = rbf::kNS;
    pb.F = 4;
    rbf::common_setup(pb, x, z, n_prog, n_all, stream);
    pb.precision = prm.precision;
    pb.n = prm.n_sten;
    pb.p = prm.phs_p;
    pb.l = prm.poly_l;
    pb.hv_k = prm.hv_k;
    pb.hv_p = prm.hv_p;
    pb.period_x = prm.period_x;
    pb.mu = prm.mu;
    pb.gamma = gamma;
    pb.hvc = prm.hv_k > 0 ? ((prm.hv_k % 2 == 1) ? 1.0 : -1.0) * gamma : 0.0;  // (-1)^(k+1) gamma
    pb.theta_bar = prm.theta_bar;
    pb.g = prm.g;
    pb.cp = prm.cp;
    pb.cv = prm.cv;
    pb.rd = prm.rd;
    pb.diff = pb.precision == 32 ? 1 : 0;
    for (int64_t i = 0; i < n_prog; ++i)
        RBF_REQUIRE(kind[i] >= 0 && kind[i] <= 4, "kind[%lld]=%d not in [0, 4]", (long long)i, kind[i]);

    cudaEvent_t e0, e1;
    RBF_CUDA(cudaEventCreate(&e0));
    RBF_CUDA(cudaEventCreate(&e1));
    RBF_CUDA(cudaEventRecord(e0, pb.st));
    pb.idx.alloc((size_t)n_prog * pb.n);
    rbf::build_stencils(pb.x.p, pb.z.p, n_all, n_prog, pb.n, pb.period_x, pb.idx.p, pb.st);
    pb.ops = {RBF_OP_DX, RBF_OP_DZ, RBF_OP_LAP, RBF_OP_DXX, RBF_OP_DZZ};
    const int nbase = (int)pb.ops.size();
    if (pb.hv_k > 0) pb.ops.push_back(RBF_OP_HV);
    pb.w64.alloc(pb.ops.size() * (size_t)n_prog * pb.n);
    if (pb.hv_k > 0 && pb.hv_p == pb.p) {
        // one augmented system serves every operator: one LU, six right-hand sides
        rbf::build_weights(pb.x.p, pb.z.p, pb.n_all, pb.idx.p, n_prog, pb.n, pb.period_x, pb.p, pb.l, pb.hv_k,
                           pb.ops.data(), (int)pb.ops.size(), pb.w64.p, pb.st);
    } else {
        rbf::build_weights(pb.x.p, pb.z.p, pb.n_all, pb.idx.p, n_prog, pb.n, pb.period_x, pb.p, pb.l, 0,
                           pb.ops.data(), nbase, pb.w64.p, pb.st);
        if (pb.hv_k > 0) {
            int hv = RBF_OP_HV;
            rbf::build_weights(pb.x.p, pb.z.p, pb.n_all, pb.idx.p, n_prog, pb.n, pb.period_x, pb.hv_p, pb.l,
                               pb.hv_k, &hv, 1, pb.w64.p + (size_t)nbase * n_prog * pb.n, pb.st);
        }
    }
    RBF_CUDA(cudaEventRecord(e1, pb.st));
    RBF_CUDA(cudaEventSynchronize(e1));
    RBF_CUDA(cudaEventElapsedTime(&pb.weight_build_ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);

    // per-node background Exner pressure and Dirichlet flags
    pb.pibar.alloc((size_t)n_prog * pb.tsize());
    if (pb.precision == 64)
        rbf::pibar_kernel<double><<<rbf::div_up(n_prog, 256), 256, 0, pb.st>>>(pb.z.p, n_prog, pb.g, pb.cp,
                                                                             pb.theta_bar, (double *)pb.pibar.p);
    else
        rbf::pibar_kernel<float><<<rbf::div_up(n_prog, 256), 256, 0, pb.st>>>(pb.z.p, n_prog, pb.g, pb.cp,
                                                                            pb.theta_bar, (float *)pb.pibar.p);
    RBF_CHECK_LAUNCH();
    std::vector<unsigned char> fl(n_prog);
    for (int64_t i = 0; i < n_prog; ++i)
        fl[i] = (kind[i] == 1 || kind[i] == 2) ? 1 : (kind[i] == 3 || kind[i] == 4) ? 2 : 0;
    pb.flags.alloc(n_prog);
    RBF_CUDA(cudaMemcpyAsync(pb.flags.p, fl.data(), n_prog, cudaMemcpyHostToDevice, pb.st));

    rbf::build_ghost_plan(pb, kind, ghost_owner);
    if (with_scratch) rbf::build_wall_set(pb);
    if (with_scratch) rbf::alloc_scratch(pb);
    pb.lat.enabled = prm.storage == RBF_STORE_LATTICE;
    rbf::choose_threads(pb, prm.threads_per_node);
    if (with_scratch && prm.threads_per_node == 0) rbf::choose_run_mode(pb, RBF_RUN_AUTO, 0, 0);
    RBF_CUDA(cudaStreamSynchronize(pb.st));
}

}  // namespace rbf

using rbf::Problem;

extern "C" {

const char *rbf_last_error(void) { return rbf::last_error(); }

int rbf_ns_create(rbf_problem **out, const rbf_ns_params *prm, const double *x, const double *z, int64_t n_prog,
                  int64_t n_all, const int32_t *kind, const int32_t *ghost_owner, void *stream) {
    return rbf::guarded([&] {
        RBF_REQUIRE(out && prm, "null argument");
        *out = nullptr;
        auto *h = new rbf_problem();
        try {
            rbf::build_ns(h->impl, *prm, x, z, n_prog, n_all, kind, ghost_owner, stream, true);
            *out = h;
        } catch (...) {
            delete h;
            throw;
        }
    });
}

int rbf_adv_create(rbf_problem **out, const rbf_adv_params *prm, const double *x, const double *z, int64_t n_prog,
                   int64_t n_all, const int32_t *src, const double *U, const double *V, void *stream) {
    // the deformational flow: one part with c(t) = cos(pi t / T)
    const rbf_flow_part part = {0.0, 1.0, 1.0};
    return rbf_adv_create_flow(out, prm, x, z, n_prog, n_all, src, 1, U, V, &part, stream);
}

int rbf_adv_create_flow(rbf_problem **out, const rbf_adv_params *prm, const double *x, const double *z,
                        int64_t n_prog, int64_t n_all, const int32_t *src, int32_t n_parts, const double *U,
                        const double *V, const rbf_flow_part *parts, void *stream) {
    return rbf::guarded([&] {
        RBF_REQUIRE(out && prm && src && U && V && parts, "null argument");
        *out = nullptr;
        RBF_REQUIRE(n_parts == 1 || n_parts == 2, "n_parts must be 1 or 2, got %d", n_parts);
        for (int k = 0; k < n_parts; ++k)
            RBF_REQUIRE(std::isfinite(parts[k].a) && std::isfinite(parts[k].b) && std::isfinite(parts[k].m),
                        "flow part %d has a non-finite coefficient", k);
        RBF_REQUIRE(prm->precision == 64 || prm->precision == 32, "precision must be 64 or 32");
        RBF_REQUIRE(prm->period_T > 0.0 && prm->gamma >= 0.0, "period_T must be > 0 and gamma >= 0");
        const double gamma = rbf::resolve_gamma(prm->gamma, prm->gamma_c, prm->spacing, prm->hv_k);
        for (int64_t j = 0; j < n_all; ++j)
            RBF_REQUIRE(src[j] >= 0 && src[j] < n_prog && (j >= n_prog || src[j] == j),
                        "src[%lld]=%d invalid", (long long)j, src[j]);
        auto *h = new rbf_problem();
        try {
            Problem &pb = h->impl;
            pb.kind = rbf::kAdvection;
            pb.F = 1;
            rbf::common_setup(pb, x, z, n_prog, n_all, stream);
            pb.precision = prm->precision;
            pb.n = prm->n_sten;
            pb.p = prm->phs_p;
            pb.l = prm->poly_l;
            pb.hv_k = prm->hv_k;
            pb.hv_p = prm->hv_p;
            pb.gamma = gamma;
            pb.hvc = prm->hv_k > 0 ? ((prm->hv_k % 2 == 1) ? 1.0 : -1.0) * gamma : 0.0;
            pb.period_T = prm->period_T;
            pb.diff = 0;
            pb.n_vparts = n_parts;
            for (int k = 0; k < n_parts; ++k) {
                pb.vpart[k][0] = parts[k].a;
                pb.vpart[k][1] = parts[k].b;
                pb.vpart[k][2] = parts[k].m;
            }
            pb.vel.alloc(2 * (size_t)n_parts * n_all);
            pb.src.alloc(n_all);
            for (int k = 0; k < n_parts; ++k) {
                RBF_CUDA(cudaMemcpyAsync(pb.vel.p + (2 * k) * n_all, U + k * n_all, n_all * 8,
                                         cudaMemcpyHostToDevice, pb.st));
                RBF_CUDA(cudaMemcpyAsync(pb.vel.p + (2 * k + 1) * n_all, V + k * n_all, n_all * 8,
                                         cudaMemcpyHostToDevice, pb.st));
            }
            RBF_CUDA(cudaMemcpyAsync(pb.src.p, src, n_all * 4, cudaMemcpyHostToDevice, pb.st));

            cudaEvent_t e0, e1;
            RBF_CUDA(cudaEventCreate(&e0));
            RBF_CUDA(cudaEventCreate(&e1));
            RBF_CUDA(cudaEventRecord(e0, pb.st));
            pb.idx.alloc((size_t)n_prog * pb.n);
            rbf::build_stencils(pb.x.p, pb.z.p, n_all, n_prog, pb.n, 0.0, pb.idx.p, pb.st);
            pb.ops = {RBF_OP_DX, RBF_OP_DZ};
            if (pb.hv_k > 0) pb.ops.push_back(RBF_OP_HV);
            pb.w64.alloc(pb.ops.size() * (size_t)n_prog * pb.n);
            if (pb.hv_k > 0 && pb.hv_p == pb.p) {
                rbf::build_weights(pb.x.p, pb.z.p, pb.n_all, pb.idx.p, n_prog, pb.n, 0.0, pb.p, pb.l, pb.hv_k,
                                   pb.ops.data(), (int)pb.ops.size(), pb.w64.p, pb.st);
            } else {
                rbf::build_weights(pb.x.p, pb.z.p, pb.n_all, pb.idx.p, n_prog, pb.n, 0.0, pb.p, pb.l, 0, pb.ops.data(),
                                   2, pb.w64.p, pb.st);
                if (pb.hv_k > 0) {
                    int hv = RBF_OP_HV;
                    rbf::build_weights(pb.x.p, pb.z.p, pb.n_all, pb.idx.p, n_prog, pb.n, 0.0, pb.hv_p, pb.l, pb.hv_k,
                                       &hv, 1, pb.w64.p + 2 * (size_t)n_prog * pb.n, pb.st);
                }
            }
            RBF_CUDA(cudaEventRecord(e1, pb.st));
            RBF_CUDA(cudaEventSynchronize(e1));
            RBF_CUDA(cudaEventElapsedTime(&pb.weight_build_ms, e0, e1));
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            rbf::alloc_scratch(pb);
            rbf::choose_threads(pb, 0);
            rbf::choose_run_mode(pb, RBF_RUN_AUTO, 0, 0);
            RBF_CUDA(cudaStreamSynchronize(pb.st));
            *out = h;
        } catch (...) {
            delete h;
            throw;
        }
    });
}

int rbf_rhs(rbf_problem *h, double t, void *U, void *dUdt) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && U && dUdt, "null argument");
        RBF_REQUIRE(((reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(dUdt)) & 15) == 0,
                    "state and tendency must be 16-byte aligned (node-major records)");
        RBF_REQUIRE(h->impl.kind != rbf::kEnsemble, "ensembles step with rbf_ens_run");
        rbf::enqueue_rhs(h->impl, t, U, dUdt, h->impl.st);
    });
}

int rbf_rk4_step(rbf_problem *h, double t, double dt, void *U) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && U, "null argument");
        RBF_REQUIRE((reinterpret_cast<uintptr_t>(U) & 15) == 0, "state must be 16-byte aligned (node-major records)");
        RBF_REQUIRE(std::isfinite(dt) && std::isfinite(t), "non-finite time or step");
        RBF_REQUIRE(h->impl.kind != rbf::kEnsemble, "ensembles step with rbf_ens_run");
        rbf::enqueue_rk4_step(h->impl, t, dt, U, h->impl.st, false, 0);
    });
}

int rbf_run(rbf_problem *h, double t0, double dt, int64_t n_steps, void *U) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h, "null problem");
        RBF_REQUIRE(h->impl.kind != rbf::kEnsemble, "ensembles step with rbf_ens_run");
        rbf::run(h->impl, t0, dt, n_steps, U);
    });
}

int rbf_run_host(rbf_problem *h, double t0, double dt, int64_t n_steps, void *U_host) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && U_host, "null argument");
        Problem &pb = h->impl;
        const int64_t stride = pb.kind == rbf::kNS ? pb.n_all : pb.n_prog;
        const size_t bytes = (size_t)pb.F * stride * pb.tsize();
        // the problem keeps one device copy of the state for repeated calls
        if (pb.host_state.bytes() < bytes) pb.host_state.alloc(bytes);
        RBF_CUDA(cudaMemcpyAsync(pb.host_state.p, U_host, bytes, cudaMemcpyHostToDevice, pb.st));
        rbf::run(pb, t0, dt, n_steps, pb.host_state.p);
        RBF_CUDA(cudaMemcpyAsync(U_host, pb.host_state.p, bytes, cudaMemcpyDeviceToHost, pb.st));
        RBF_CUDA(cudaStreamSynchronize(pb.st));
        rbf::persistent_check(pb);
    });
}

int rbf_sync(rbf_problem *h) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h, "null problem");
        RBF_CUDA(cudaStreamSynchronize(h->impl.st));
        RBF_CUDA(cudaStreamSynchronize(h->impl.cap));
        rbf::persistent_check(h->impl);
    });
}

int rbf_set_run_mode(rbf_problem *h, int32_t mode, int32_t lanes, int32_t ctas) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h, "null problem");
        Problem &pb = h->impl;
        RBF_CUDA(cudaStreamSynchronize(pb.st));
        RBF_CUDA(cudaStreamSynchronize(pb.cap));
        rbf::choose_run_mode(pb, mode, lanes, ctas);
    });
}

int rbf_set_stage_split(rbf_problem *h, int32_t enable) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h, "null problem");
        Problem &pb = h->impl;
        RBF_REQUIRE(pb.kind == rbf::kNS, "stage splitting applies to Navier-Stokes problems");
        RBF_REQUIRE(!enable || (pb.side && pb.wlist.p), "the problem has no wall set to split");
        RBF_CUDA(cudaStreamSynchronize(pb.st));
        RBF_CUDA(cudaStreamSynchronize(pb.cap));
        rbf::invalidate_graph(pb);
        pb.split = enable != 0;
    });
}

int rbf_set_operator_storage(rbf_problem *h, int32_t mode, int32_t threads_per_node, int64_t *class_nodes,
                             int32_t *n_classes) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h, "null problem");
        Problem &pb = h->impl;
        RBF_REQUIRE(pb.kind == rbf::kNS,
                    "operator storage is switched on Navier-Stokes problems (an ensemble's is set at creation)");
        RBF_REQUIRE(mode == RBF_STORE_PER_NODE || mode == RBF_STORE_LATTICE, "unknown storage mode %d", mode);
        RBF_REQUIRE(threads_per_node == 0 || threads_per_node == 1 || threads_per_node == 2 ||
                        threads_per_node == 4 || threads_per_node == 8,
                    "threads_per_node must be 0, 1, 2, 4 or 8");
        RBF_CUDA(cudaStreamSynchronize(pb.st));
        RBF_CUDA(cudaStreamSynchronize(pb.cap));
        rbf::invalidate_graph(pb);
        pb.lat.enabled = mode == RBF_STORE_LATTICE;
        if (threads_per_node == 0) RBF_REQUIRE(pb.S0.p, "autotuning needs the stage buffers");
        rbf::choose_threads(pb, threads_per_node);
        if (class_nodes) *class_nodes = pb.lat.enabled ? pb.lat.class_nodes : 0;
        if (n_classes) *n_classes = pb.lat.enabled ? pb.lat.n_cls : 0;
    });
}

int rbf_set_spin_limit(rbf_problem *h, int64_t polls) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h, "null problem");
        RBF_REQUIRE(polls >= 0, "spin limit must be >= 0");
        h->impl.ps.spin_limit = polls;
    });
}

int rbf_minmax(rbf_problem *h, const void *U, double *out) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && U && out, "null argument");
        rbf::minmax(h->impl, U, out);
    });
}

int rbf_get_info(const rbf_problem *h, rbf_info *out) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && out, "null argument");
        const Problem &pb = h->impl;
        memset(out, 0, sizeof(*out));
        out->n_prog = pb.n_prog;
        out->n_all = pb.n_all;
        out->n_ghost = pb.gh.n_ghost;
        out->n_fields = pb.F;
        out->precision = pb.precision;
        out->n_sten = pb.n;
        out->threads_per_node = pb.G;
        out->slots = pb.SL * pb.G;
        const bool ghosts = pb.kind != rbf::kAdvection && pb.gh.n_ghost > 0;
        out->launches_per_step = 4 * (ghosts ? (pb.split ? 4 : 3) : 1) + (pb.kind == rbf::kAdvection ? 1 : 0);
        out->stage_split = pb.split ? 1 : 0;
        out->n_components = pb.gh.n_comp;
        out->n_ghost_classes = pb.gh.n_class;
        out->prefetch = pb.pf > 0 ? 1 : 0;
        out->run_mode = pb.kind == rbf::kEnsemble ? RBF_RUN_GRAPH : pb.run_mode;
        if (pb.ps.ready) {
            out->persist_lanes = pb.ps.G;
            out->persist_regs = pb.ps.R > 0 ? 1 : 0;
            out->persist_chunk = pb.ps.chunk;
            out->persist_halo_max = pb.ps.halo_max;
            out->persist_ctas = pb.ps.grid;
        }
        out->weight_build_ms = pb.weight_build_ms;
        out->ghost_setup_ms = pb.ghost_setup_ms;
        const double ts = (double)pb.tsize();
        double slots = pb.n_slots;   // algorithmic, without padding
        if (pb.kind == rbf::kEnsemble) {   // node-weighted mean over the members
            double s = 0.0;
            for (auto &m : pb.ens->members) s += (double)m->n_slots * (double)m->n_prog;
            slots = s / (double)pb.n_prog;
        }
        if (pb.kind != rbf::kAdvection) {
            if (pb.kind == rbf::kEnsemble) {   // node-weighted mean over the members
                double b = 0.0;
                for (auto &m : pb.ens->members) b += rbf::ns_rhs_bytes(*m) * (double)m->n_prog;
                out->rhs_bytes_per_node = b / (double)pb.n_prog;
            } else {
                out->rhs_bytes_per_node = rbf::ns_rhs_bytes(pb);
            }
            out->rhs_flops_per_node = slots * (12 * 2 + (pb.diff ? 4 : 0)) + 40 + 4 * 4;
        } else {
            // packed weights (velocity parts + hyperviscosity) + index per
            // slot, the node's value, U_n, the accumulator read+write, the
            // stage output
            out->rhs_bytes_per_node = slots * ((pb.n_vparts + 1) * ts + 4) + ts + ts + 2 * ts + ts;
            out->rhs_flops_per_node = slots * 2 * (pb.n_vparts + 1) + 10 + 4 * (pb.n_vparts - 1);
        }
    });
}

int rbf_get_weights(const rbf_problem *h, int32_t op, double *out, int32_t *out_idx) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && out, "null argument");
        const Problem &pb = h->impl;
        int slot = -1;
        for (size_t i = 0; i < pb.ops.size(); ++i)
            if (pb.ops[i] == op) slot = (int)i;
        RBF_REQUIRE(slot >= 0, "operator %d not built for this problem", op);
        const size_t cnt = (size_t)pb.n_prog * pb.n;
        RBF_CUDA(cudaMemcpy(out, pb.w64.p + slot * cnt, cnt * 8, cudaMemcpyDeviceToHost));
        if (out_idx) RBF_CUDA(cudaMemcpy(out_idx, pb.idx.p, cnt * 4, cudaMemcpyDeviceToHost));
    });
}

int rbf_destroy(rbf_problem *h) {
    return rbf::guarded([&] {
        if (!h) return;
        cudaStreamSynchronize(h->impl.st);
        cudaStreamSynchronize(h->impl.cap);
        delete h;
    });
}

// Kernel timing for measurement: when enabled, rbf_run captures one step per
// graph with timing events around the four fused stage kernels; afterwards
// rbf_stage_kernel_ms returns their summed device time of the last step.
int rbf_set_stage_timing(rbf_problem *h, int32_t enable) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h, "null problem");
        h->impl.record_rhs_events = enable != 0;
        rbf::invalidate_graph(h->impl);
    });
}

int rbf_stage_kernel_ms(rbf_problem *h, double *ms) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && ms, "null argument");
        Problem &pb = h->impl;
        RBF_REQUIRE(pb.record_rhs_events && !pb.rhs_ev.empty(), "stage timing not enabled or no step run");
        RBF_CUDA(cudaStreamSynchronize(pb.cap));
        double total = 0.0;
        for (size_t q = 0; q + 1 < pb.rhs_ev.size(); q += 2) {
            float t = 0.f;
            RBF_CUDA(cudaEventElapsedTime(&t, pb.rhs_ev[q], pb.rhs_ev[q + 1]));
            total += t;
        }
        *ms = total;
    });
}

}  // extern "C"

int rbf_hyperviscosity_gamma(double c, double h, int32_t k, double *gamma) {
    return rbf::guarded([&] {
        RBF_REQUIRE(gamma, "null output");
        RBF_REQUIRE(std::isfinite(c) && c >= 0.0, "c must be >= 0");
        RBF_REQUIRE(std::isfinite(h) && h > 0.0, "h must be > 0");
        RBF_REQUIRE(k >= 1, "k must be >= 1");
        *gamma = c * std::pow(h, 2 * k - 1);
    });
}
