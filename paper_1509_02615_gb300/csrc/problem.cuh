// Internal layout of an rbf_problem: the packed operators, ghost systems, RK4
// scratch and captured graphs of one Navier-Stokes or advection problem.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "common.cuh"

namespace rbf {

enum ProblemKind { kNS = 0, kAdvection = 1, kEnsemble = 2 };

struct Problem;

// a8: members of a batched ensemble and their launch geometry.
struct EnsembleState {
    std::vector<std::unique_ptr<Problem>> members;   // caller order
    std::vector<int64_t> rec0;          // first state record of each member (caller order)
    std::vector<double> dt;
    std::vector<int64_t> n_steps;
    std::vector<int> order;             // members by descending n_steps
    std::vector<int64_t> blocks_before; // [n+1] stage blocks of the first k members in that order
    std::vector<int64_t> rows_before;   // [n+1] ghost rows of the first k members in that order
    DevBuf<unsigned char> descs;        // one block descriptor per stage block
    int64_t total_records = 0, total_nodes = 0;
    int active_members = 0;             // launch geometry of the captured graph
    bool whole_run = false;             // the captured graph is a whole run (loop nodes)
    DevBuf<unsigned> wcount;            // loop counters of the whole-run graph, one per phase
};

struct GhostPlan {
    int64_t n_ghost = 0;         // ghost rows in the layout
    int64_t rows = 0;            // ghost rows processed per fill (active prefix)
    int n_comp = 0;
    int n_class = 0;
    int npad = 0;                // stencil slots per wall row, padded to 8
    int field_class[4] = {0, 0, 0, 0};
    DevBuf<int32_t> gidx;        // [n_ghost][npad] owner-stencil node per slot
    DevBuf<unsigned char> gw;    // [F][n_ghost][npad] T: BC weights, zero on ghosts
    DevBuf<int32_t> owner;       // [n_ghost] state record of each row's wall node
    DevBuf<unsigned char> tb;    // [n_ghost] 1 if the owner is a bottom/top node
    DevBuf<int32_t> pos;         // [n_ghost] position of ghost row in component order
    DevBuf<int64_t> grec;        // [n_ghost] state record of the ghost at each position
    DevBuf<int32_t> comp_of;     // [n_ghost] component of each position
    DevBuf<int64_t> comp_start;  // [n_comp + 1] first position of each component
    DevBuf<int64_t> inv_off;     // [n_class][n_comp] offset of each inverse block
    DevBuf<unsigned char> inv;   // T [sum over class, comp of m^2]
    DevBuf<unsigned char> res;   // T [F][n_ghost] residual b - W_I u_I - W_B u_B
    // banded inverse rows: row (class, position) keeps the entries of its
    // W_G^{-1} row above 2^-8 eps of the row's largest (CSR)
    DevBuf<int64_t> brow;        // [n_class * n_ghost + 1]
    DevBuf<int32_t> bcol;        // position of each kept entry
    DevBuf<unsigned char> bval;  // T value of each kept entry
    int64_t band_nnz = 0;
};

// Time factor c_k(t) = a + b cos(m pi t / T) of a separable velocity part
// (advection, Sec. 6.1), as the persistent advection kernel evaluates it.  It
// is the same expression as the stage kernel's flow_factor (csrc/ns.cu), so
// the two run modes agree bit for bit (tests/test_gpu_adv_persistent.py).
__device__ __forceinline__ double velocity_time_factor(double a, double b, double m, double t, double T) {
    return b == 0.0 ? a : a + b * cos(m * 3.141592653589793 * t / T);
}

// flags bit of the wall set (split stage launches)
constexpr unsigned char kWallSetFlag = 4;

// Builds gh.brow / bcol / bval from the dense inverse blocks.
void build_ghost_bands(GhostPlan &gh, int precision, cudaStream_t st);

// Persistent run mode: one cooperative launch runs all the steps of an
// rbf_run (csrc/persistent.cu).  The nodes are split into compact blocks,
// one per CTA; each block's list of the records its stencils read (own
// nodes first), its lane operators packed in block order, and the constant
// data of the ghost rows and ghost values it solves for itself.
struct PersistPlan {
    bool ready = false;
    int G = 0;                   // lanes per node
    int R = 0;                   // operand vectors held in registers (0: read each stage)
    int maxt = 0;                // thread limit of the kernel variant
    int SLQ = 0, V = 0;          // packing of pw / lidx (as Problem::SLQ, V)
    int chunk = 0;               // largest block (nodes per CTA)
    int threads = 0, grid = 0;
    int halo_max = 0;            // largest record list
    int rows_max = 0;            // most ghost rows one CTA solves
    size_t smem = 0;
    DevBuf<unsigned char> pw;    // T [4][SLQ][grid * chunk][G][V]
    DevBuf<uint16_t> lidx;       // [SLQ][grid * chunk][G][V] list position of each slot
    DevBuf<int32_t> hlist;       // record lists of all CTAs
    DevBuf<unsigned char> cta;   // per-CTA layout records
    DevBuf<unsigned char> blob;  // per-CTA ghost-row and ghost-value data
    DevBuf<unsigned int> arrive; // barrier arrivals, monotone across launches
    unsigned base = 0;           // its value when the next launch starts
    DevBuf<int> abort;           // set when a barrier wait gives up (sticky until rbf_sync)
    // owned-rows mode (FP64): each wall row's residual is formed once, by the
    // CTA that owns its wall node, and read back from global memory by the
    // CTAs that solve ghosts after a barrier among those CTAs only
    bool own_rows = false;
    int wall_ctas = 0;           // CTAs that solve ghosts (the barrier's members)
    DevBuf<unsigned char> resg;  // T [4][ghost rows] residuals of the stage
    DevBuf<unsigned int> arrive2;   // their barrier's arrivals
    unsigned base2 = 0;
    long long spin_limit = 1LL << 21;   // polls per barrier wait (about a second)
};

struct Problem {
    ProblemKind kind = kNS;
    cudaStream_t st = nullptr;    // caller's stream
    cudaStream_t cap = nullptr;   // private stream for graph capture
    int precision = 64;
    bool pdl = true;              // programmatic dependent launch between kernels
    int F = 4;
    int64_t n_prog = 0, n_all = 0;
    int n = 0;                    // stencil size
    int G = 4;                    // threads per node
    int pf = 0;                   // > 0: stage kernel holds its operands in registers
    int diff = 0;                 // 1: difference form (self slot dropped)
    int n_slots = 0;              // neighbour slots per node before padding
    int SL = 0;                   // slots per lane (padded)
    int V = 1;                    // slots per operand vector (16 bytes for NS)
    int SLQ = 0;                  // operand vectors per lane
    // NS physics
    double mu = 0, gamma = 0, hvc = 0, theta_bar = 300, g = 9.81, cp = 1004, cv = 717, rd = 287;
    double period_x = 0;
    int p = 7, l = 4, hv_k = 0, hv_p = 7;
    // advection
    double period_T = 1.0;
    int n_vparts = 1;             // separable velocity parts (1 or 2)
    double vpart[2][3] = {{0.0, 1.0, 1.0}, {0.0, 0.0, 0.0}};   // c_k(t) = a + b cos(m pi t / T)
    DevBuf<double> vel;           // [n_vparts][2][n_all] spatial velocity factors U_k, V_k
    DevBuf<int32_t> src;          // [n_all] source node of each node

    // FP64 setup products (kept for rbf_get_weights)
    std::vector<int> ops;         // operator code of each weight block
    DevBuf<double> x, z;
    DevBuf<int32_t> idx;          // [n_prog][n]
    DevBuf<double> w64;           // [ops][n_prog][n]

    // packed operators, precision T
    int n_packed = 4;
    DevBuf<int32_t> pidx;         // [SLQ][n_prog][G][V]
    DevBuf<unsigned char> pw;     // T [n_packed][SLQ][n_prog][G][V]
    DevBuf<unsigned char> pibar;  // T [n_prog]
    DevBuf<unsigned char> flags;  // [n_prog]: bit0 w Dirichlet, bit1 u Dirichlet, bit2 wall set

    // Split stage launches (graph and step modes of problems with ghosts):
    // the wall set, the nodes whose records feed a ghost residual or whose
    // stencils read a ghost, runs as its own launch per stage, so that the
    // next stage's ghost fill overlaps the launch of the other nodes.
    bool split = false;
    DevBuf<int32_t> wlist;        // [n_wall] wall-set nodes, ascending
    DevBuf<int32_t> rlist;        // [n_prog - n_wall] the other nodes, ascending
    int64_t n_wall = 0;
    int prio_hi = 0;              // scheduling priority of the wall-set launches
    cudaStream_t side = nullptr;  // stream of the other nodes' launches
    cudaEvent_t ev_fork = nullptr, ev_w[2] = {nullptr, nullptr}, ev_r[2] = {nullptr, nullptr};

    GhostPlan gh;

    // RK4 scratch, precision T, node-major records [rows][F]
    DevBuf<unsigned char> S0, S1, K;
    DevBuf<double> tdev;          // device time for graph replays (advection)
    DevBuf<unsigned char> host_state;  // device copy used by rbf_run_host

    // graph cache
    cudaGraphExec_t graph = nullptr;
    void *graph_U = nullptr;
    double graph_dt = 0.0;
    int graph_steps = 0;
    bool record_rhs_events = false;
    std::vector<cudaEvent_t> rhs_ev;   // [2 * 4 * graph_steps] when recording

    int run_mode = 1;             // RBF_RUN_GRAPH or RBF_RUN_PERSISTENT
    PersistPlan ps;

    // Lattice operator storage (csrc/lattice.cu): one packed operator row per
    // class of translated stencils, used by the stage kernels when enabled.
    struct Lattice {
        bool enabled = false, classified = false;
        int min_members = 32;
        int32_t n_cls = 0;
        int64_t class_nodes = 0;      // nodes in classes (the rest keep per-node operators)
        std::vector<int32_t> cls_host;
        std::vector<int64_t> rep;     // first member of each class
        std::vector<int32_t> rep_idx; // [n_cls][n] its stencil
        std::vector<double> rep_w;    // [nops][n_cls][n] its FP64 weights
        DevBuf<int32_t> cls;          // [n_prog] class of each node, -1: per-node operators
        DevBuf<int32_t> loff;         // [n_cls][SLQ][G][V] relative index of each slot
        DevBuf<unsigned char> lw;     // T [4][n_cls][SLQ][G][V] packed operators
    } lat;

    float weight_build_ms = 0.f, ghost_setup_ms = 0.f;
    std::unique_ptr<EnsembleState> ens;

    size_t tsize() const { return precision == 64 ? 8 : 4; }
    ~Problem();
};

// Launches one RK4 step (4 stages, ghost fill before each) on stream s.
// With split stage launches, a sequence of steps may leave the side stream
// open between them: first = false continues such a sequence, last = false
// leaves it open (the sequence's last step must pass last = true).
void enqueue_rk4_step(Problem &pb, double t, double dt, void *U, cudaStream_t s, bool record_events, int step_in_graph,
                      bool first = true, bool last = true);
void enqueue_rhs(Problem &pb, double t, void *U, void *dUdt, cudaStream_t s);
void autotune_threads_per_node(Problem &pb);
void pack_operators(Problem &pb);
void pack_lattice(Problem &pb, const std::vector<double> &comb, int nops);
double ns_rhs_bytes(const Problem &pb);
// gamma of Sec. 5.3 from a problem's gamma or (gamma_c, spacing) (api.cu)
double resolve_gamma(double gamma, double gamma_c, double spacing, int hv_k);
int32_t lattice_classes(const int32_t *idx, const double *x, const double *z, int64_t n_prog, int n,
                        double period_x, double h, int min_members, int32_t *cls);
void build_ghost_plan(Problem &pb, const int32_t *kind_host, const int32_t *owner_host);
// Ghost residual and banded ghost solve of the state U on stream s; prio != 0
// is the kernels' scheduling priority (see launch_kernel_prio).
void enqueue_ghost_fill(Problem &pb, void *U, cudaStream_t s, int prio = 0);
void minmax(Problem &pb, const void *U, double *out);
// Split stage launches of a problem with ghosts: marks the wall set in
// pb.flags, lists it and the other nodes in pb.wlist / pb.rlist and creates
// the side stream and its events; the split itself stays off until the
// autotuner or rbf_set_stage_split turns it on (csrc/ghost.cu).
void build_wall_set(Problem &pb);
void build_ns(Problem &pb, const rbf_ns_params &prm, const double *x, const double *z, int64_t n_prog,
              int64_t n_all, const int32_t *kind, const int32_t *ghost_owner, void *stream, bool with_scratch);
void alloc_scratch(Problem &pb);
void enqueue_ens_step(Problem &pb, double dt_unused, void *U, cudaStream_t s, bool rec, int step);
void build_ensemble(Problem &pb, const rbf_ns_params &common, int n, const rbf_ens_member *mem, const double *x,
                    const double *z, const int32_t *kind, const int32_t *owner, void *stream);
void run_ensemble(Problem &pb, int64_t max_steps, void *U);
double ensemble_node_updates(const Problem &pb, int64_t max_steps);
// Builds the persistent plan for G lanes per node on `ctas` CTAs (0: one per
// SM); false if the problem does not fit one co-resident launch (pb.ps.ready
// tells the same).
bool persistent_plan(Problem &pb, int G, int ctas);
void persistent_run(Problem &pb, double dt, int64_t n_steps, void *U, cudaStream_t s);
// Advection (a6 + a7) in one cooperative launch: the plan for the problem's
// current packing (pb.G lanes per node, operators in registers) with CTAs of
// `threads` threads (64, 128 or 256); false if it does not fit.
bool adv_persistent_plan(Problem &pb, int threads);
void adv_persistent_run(Problem &pb, double t0, double dt, int64_t n_steps, void *U, cudaStream_t s);

// a9 fused into the persistent run: the learned correction's network (BF16
// weights, FP32 biases and scales) and its per-field strengths.
struct MlpView {
    const void *Pb;                 // __nv_bfloat16 parameters
    const float *P;                 // FP32 parameters (biases)
    int64_t oW1, ob1, oW2, ob2, oW3, ob3;
    const float *scales;            // [12]: feature, output, own-value scales
    float alpha[4];
    int n_in;
    unsigned long long *bad;        // non-finite corrections skipped
};
// True if a learned run can go through the persistent kernel (FP32 problem in
// persistent mode with a variant that holds the network).
bool persistent_mlp_ready(const Problem &pb);
void persistent_run_mlp(Problem &pb, double dt, int64_t n_steps, void *U, cudaStream_t s, const MlpView &mv);
// Persistent plan for corrected runs: times short corrected runs on a zero
// state for each lane count and CTA count, keeps the fastest plan that holds
// the network and puts the problem in persistent mode; false if none fits.
bool persistent_tune_mlp(Problem &pb, const MlpView &mv);
// RBF_E_TIMEOUT (and clears the flag) if a persistent launch gave up a wait.
void persistent_check(Problem &pb);

}  // namespace rbf

struct rbf_problem {
    rbf::Problem impl;
};
