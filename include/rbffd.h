/*
 * rbffd.h -- C ABI of the GB300 (sm_103a) PHS RBF-FD library.
 *
 * The method (Barnett, Flyer & Wicker, "An RBF-FD polynomial method based on
 * polyharmonic splines for the Navier-Stokes equations"):
 *   Sec. 3, Eq. (weights): per node, solve the augmented system
 *       [A P; P^T 0] [w; lambda] = [L phi; L p]   at x_c,
 *   A_ij = ||x_i - x_j||^p (odd PHS), P = 2D monomials of degree <= l,
 *   giving one row of a sparse differentiation matrix (only nonzeros kept).
 *   Sec. 5.2, Eq. (bcEqn): ghost values u_G = -W_G^{-1}(W_I u_I + W_B u_B).
 *   Sec. 5.3, Eq. (laplacian): hyperviscosity (-1)^(k+1) gamma Delta^k.
 *   Sec. 6.1: flux-form scalar advection with reflected boundary nodes.
 *   Sec. 6.2, Eqs. (uEq)-(piEq): 2D compressible Navier-Stokes in
 *   perturbation form, fields [u, w, theta', pi'], stepped with RK4.
 *
 * Conventions (every entry point):
 *   - Return value: RBF_OK (0) or one of the RBF_E_* codes; the message of
 *     the last failure on the calling thread is in rbf_last_error().
 *     No C++ exception crosses the ABI.
 *   - "device" pointers are CUDA global-memory pointers on the current
 *     device; "host" pointers are ordinary CPU memory.  The caller owns every
 *     buffer it passes; the library never frees them.
 *   - Node arrays list the prognostic nodes [0, n_prog) first, then ghost or
 *     reflected nodes [n_prog, n_all).
 *   - Field arrays are node-major records: U[i * F + f], the F fields of node
 *     i contiguous (F = 4: u, w, theta', pi' for Navier-Stokes; F = 1 for
 *     advection), 16-byte aligned.
 *   - stream: a cudaStream_t (NULL = legacy default stream).  Setup calls
 *     (rbf_build_*, rbf_*_create) return after their work completes; the
 *     stepping calls (rbf_rhs, rbf_rk4_step, rbf_run) only enqueue work.
 *   - There is no CPU fallback: without a usable GPU every call returns
 *     RBF_E_CUDA.
 */
#ifndef RBFFD_H
#define RBFFD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define RBF_OK 0
#define RBF_E_ARG 1          /* invalid argument (message says which)        */
#define RBF_E_SINGULAR 2     /* a weight or ghost system has a zero pivot    */
#define RBF_E_NONFINITE 3    /* NaN or Inf found by rbf_check_finite         */
#define RBF_E_TIMEOUT 4      /* a bounded device-side wait gave up           */
#define RBF_E_CUDA 5         /* CUDA runtime error (message has the string)  */
#define RBF_E_OOM 6          /* device allocation failed                     */

/* ---- operators L of Eq. (weights) -------------------------------------- */
#define RBF_OP_DX 0   /* d/dx                                              */
#define RBF_OP_DZ 1   /* d/dz (the second coordinate, y in Sec. 6.1)       */
#define RBF_OP_LAP 2  /* Laplacian, Eq. (laplacian)                        */
#define RBF_OP_HV 3   /* Delta^k, Eq. (laplacian) applied k times          */
#define RBF_OP_DXX 4  /* d2/dx2                                            */
#define RBF_OP_DZZ 5  /* d2/dz2                                            */

/* Message of the last failing call on this thread ("" if none). */
const char *rbf_last_error(void);

/*
 * a1  Stencil selection (Sec. 6: the n nearest nodes; Appendix A).
 * For each centre c in [0, n_centers) (centres are nodes 0..n_centers-1),
 * writes the n nearest of all n_all nodes, ordered by squared distance
 * (FP64, dx*dx + dz*dz without fused multiply-add), ties by node index.
 * With period_x > 0, dx is taken to the minimum image in x.
 *   x, z      device, double [n_all]
 *   idx       device, int32 [n_centers][n] (output; idx[c][0] == c)
 * Errors: RBF_E_ARG for n < 1, n > n_all, n > 128, non-finite coordinates or
 * a node density so uneven that a search window holds > 2048 candidates.
 */
int rbf_build_stencils(const double *x, const double *z, int64_t n_all, int64_t n_centers,
                       int32_t n, double period_x, int32_t *idx, void *stream);

/*
 * Allocation-free form of rbf_build_stencils (the paper has no counterpart;
 * this is a service for callers).  Some callers may not allocate device
 * memory: a framework whose memory pool owns the whole GPU (a cudaMalloc
 * would bypass its accounting or fail), a process with a fixed device-memory
 * budget, or a loop that cannot afford cudaMalloc/cudaFree's implicit device
 * synchronisation.  This entry point calls no cudaMalloc, cudaFree or other
 * allocating routine: its binning grid and counters live in one static
 * device array of about 5 MB (kept by every GPU that loads the library until
 * the process exits).  Arguments, output and ordering are those of
 * rbf_build_stencils; the caller still provides x, z and idx.
 *   Limits: n_all <= 262144 nodes and a binning grid of <= 262144 cells
 *   (about n_all / 2); larger inputs return RBF_E_ARG with a message.
 *   Set-up: every call looks up the array's device address
 *   (cudaGetSymbolAddress) on the current device, so the address stays valid
 *   across a device reset or a new context; the first call on a device also
 *   loads the library's device code there.
 *   Sharing: every call on a device uses the same array.  Calls whose work
 *   overlaps on the GPU (other streams or threads) race; serialise them.
 *   Counters are cleared at the start of every call.
 */
int rbf_build_stencils_static(const double *x, const double *z, int64_t n_all, int64_t n_centers,
                              int32_t n, double period_x, int32_t *idx, void *stream);

/*
 * a2  RBF-FD weights (Sec. 3, Eq. (weights); Sec. 5.3, Eq. (laplacian)).
 * One augmented solve per stencil with PHS r^p (p odd, 1 <= p <= 15) and all
 * monomials of degree <= l (0 <= l <= 8), in coordinates shifted to the
 * centre and scaled by the stencil radius; LU with partial pivoting in FP64.
 * RBF_OP_HV uses Delta^hv_k and needs p >= 2*hv_k + 1.
 *   x, z      device, double [n_all]
 *   idx       device, int32 [n_centers][n], centre first (rbf_build_stencils)
 *   ops       host, int32 [n_ops], RBF_OP_* codes (1 <= n_ops <= 6)
 *   w         device, double [n_ops][n_centers][n] (output, physical units)
 * Errors: RBF_E_ARG for bad sizes or codes, n + (l+1)(l+2)/2 > 160;
 * RBF_E_SINGULAR if a pivot vanishes (node id in the message).
 */
int rbf_build_weights(const double *x, const double *z, int64_t n_all, const int32_t *idx,
                      int64_t n_centers, int32_t n, double period_x, int32_t p, int32_t l,
                      int32_t hv_k, const int32_t *ops, int32_t n_ops, double *w, void *stream);

/*
 * Hyperviscosity coefficient of Sec. 5.3 (host only, no GPU needed).  The
 * paper asks for one constant c "regardless of the resolution" and prints
 * gamma = c h^(-2k), which cannot be dimensionally right; this library reads
 * it as gamma = c h^(2k - 1): with dt proportional to h (the paper's time
 * steps), dt * gamma * rho(Delta^k) is then the same at every resolution.
 * The term added to the right-hand side is (-1)^(k+1) gamma Delta^k, which
 * damps.  *gamma = c * h^(2k - 1).
 * Errors: RBF_E_ARG for c < 0, h <= 0, k < 1 or a null output.
 */
int rbf_hyperviscosity_gamma(double c, double h, int32_t k, double *gamma);

/* ---- problems: a stepping context built once, stepped many times -------- */
typedef struct rbf_problem rbf_problem;

/* Parameters of the Navier-Stokes problem (Sec. 6.2-6.3). */
/* Operator storage of the stage kernels (rbf_ns_params.storage,
 * rbf_set_operator_storage). */
#define RBF_STORE_PER_NODE 0
#define RBF_STORE_LATTICE 1

typedef struct rbf_ns_params {
    int32_t n_sten;     /* stencil size n (37 in Sec. 6)                      */
    int32_t phs_p;      /* PHS exponent of d/dx, d/dz, Lap, BC operators (7)   */
    int32_t poly_l;     /* polynomial degree l (4)                            */
    int32_t hv_k;       /* hyperviscosity Laplacian power k (3); 0 = none     */
    int32_t hv_p;       /* PHS exponent of the Delta^k weights (>= 2k+1)      */
    int32_t precision;  /* 64: FP64 storage and arithmetic; 32: FP64-built
                           weights stored in FP32, FP32 RHS and RK4           */
    int32_t threads_per_node; /* 0 = autotuned (lanes per node and register
                                 prefetch); else 1, 2, 4 or 8 lanes        */
    int32_t storage;    /* RBF_STORE_PER_NODE (0, Sec. 3's rows) or
                           RBF_STORE_LATTICE (1, one row per class of
                           translated stencils; see rbf_set_operator_storage);
                           the only way to choose it for an ensemble         */
    double period_x;    /* > 0: periodic in x with this period (m)            */
    double mu;          /* viscosity (m^2/s)                                  */
    double gamma;       /* hyperviscosity coefficient gamma >= 0, used as
                           given when gamma_c = 0                            */
    double theta_bar;   /* background potential temperature T_s (300 K)      */
    double g, cp, cv, rd; /* 9.81, 1004, 717, 287                             */
    double gamma_c;     /* > 0: the library forms gamma = gamma_c *
                           spacing^(2 hv_k - 1) (rbf_hyperviscosity_gamma;
                           gamma must then be 0); 0: gamma as given          */
    double spacing;     /* node spacing h in the case's length unit (m) for
                           gamma_c; ensembles take it per member             */
} rbf_ns_params;

/*
 * Build a Navier-Stokes problem: stencils (a1), weights (a2) for d/dx, d/dz,
 * Lap, d2/dx2, d2/dz2 and Delta^k, the packed operators (a3) and the ghost
 * systems of Sec. 5.2 (a4: inverted once, applied every stage).
 *   x, z         host, double [n_all]
 *   kind         host, int32 [n_prog]: 0 interior, 1 bottom, 2 top, 3 left,
 *                4 right wall (corner nodes belong to bottom/top)
 *   ghost_owner  host, int32 [n_all - n_prog]: the wall node of each ghost
 * Boundary conditions (Sec. 6.3, 6.4): bottom/top u_z = 0, w = w_zz = 0,
 * theta'_z = 0, pi'_z = g theta'/(c_p theta_bar (theta_bar + theta'));
 * left/right u = u_xx = 0, w_x = 0, theta'_x = 0, pi'_x = 0.
 * The problem keeps the stream for all its work.
 */
int rbf_ns_create(rbf_problem **out, const rbf_ns_params *prm, const double *x, const double *z,
                  int64_t n_prog, int64_t n_all, const int32_t *kind, const int32_t *ghost_owner,
                  void *stream);

/* Parameters of the scalar-advection problem (Sec. 6.1). */
typedef struct rbf_adv_params {
    int32_t n_sten;     /* 37                                                 */
    int32_t phs_p;      /* PHS exponent of d/dx, d/dy (7)                     */
    int32_t poly_l;     /* 4                                                  */
    int32_t hv_k;       /* 4                                                  */
    int32_t hv_p;       /* 9 (Delta^4 r^7 is singular at r = 0)               */
    int32_t precision;  /* 64 or 32                                           */
    double gamma;       /* hyperviscosity coefficient (used when gamma_c = 0) */
    double period_T;    /* velocity time factor cos(pi t / T)                 */
    double gamma_c;     /* > 0: gamma = gamma_c * spacing^(2 hv_k - 1)        */
    double spacing;     /* node spacing h (unit square: 1 / (m - 1))          */
} rbf_adv_params;

/*
 * Build a flux-form advection problem psi_t = -(u psi)_x - (v psi)_y with
 * u = U(x,y) cos(pi t/T), v = V(x,y) cos(pi t/T).  Nodes [n_prog, n_all) are
 * reflections of prognostic nodes (src gives the source); their values are
 * their sources' values and U, V are sampled at their own positions.
 *   x, z, U, V   host, double [n_all];  src  host, int32 [n_all]
 */
int rbf_adv_create(rbf_problem **out, const rbf_adv_params *prm, const double *x, const double *z,
                   int64_t n_prog, int64_t n_all, const int32_t *src, const double *U,
                   const double *V, void *stream);

/*
 * One time-separable part of an advecting velocity: the flow is
 * u(x, t) = sum_k c_k(t) U_k(x), v(x, t) = sum_k c_k(t) V_k(x) with
 * c_k(t) = a + b cos(m pi t / T), T = rbf_adv_params.period_T.
 */
typedef struct rbf_flow_part {
    double a, b, m;
} rbf_flow_part;

/*
 * Flux-form advection (Sec. 6.1) in a velocity field made of n_parts (1 or 2)
 * time-separable parts.  The vortex flow of Sec. 6.1,
 * u = u_theta(r, t) sin(theta), v = -u_theta(r, t) cos(theta) with
 * u_theta = (4 pi r / T) [1 - cos(2 pi t / T) (1 - (4r)^6) / (1 + (4r)^6)],
 * is two parts: the solid-body rotation with c_1 = 1 ({1, 0, 0}) and the
 * same rotation scaled by (1 - (4r)^6) / (1 + (4r)^6) with
 * c_2 = -cos(2 pi t / T) ({0, -1, 2}).  rbf_adv_create is this call with one
 * part {0, 1, 1}.
 *   U, V    host, double [n_parts][n_all]: part k's spatial factors sampled
 *           at every node's own position (reflected nodes included)
 *   parts   host [n_parts]
 * Other arguments, ownership and errors as rbf_adv_create; RBF_E_ARG for
 * n_parts outside {1, 2} or a non-finite coefficient.  Each extra part adds
 * one packed weight block (n_sten weights per node) to the stage kernel's
 * stream.
 */
int rbf_adv_create_flow(rbf_problem **out, const rbf_adv_params *prm, const double *x, const double *z,
                        int64_t n_prog, int64_t n_all, const int32_t *src, int32_t n_parts, const double *U,
                        const double *V, const rbf_flow_part *parts, void *stream);

/* One member of a batched ensemble (a8). */
typedef struct rbf_ens_member {
    int64_t n_prog, n_all;  /* member's prognostic nodes and all nodes (ghosts last) */
    int32_t n_sten;         /* its stencil size                                   */
    int32_t poly_l;         /* its polynomial degree                              */
    double period_x;        /* > 0: periodic in x                                 */
    double gamma;           /* its hyperviscosity coefficient (common.gamma_c = 0) */
    double dt;              /* its RK4 time step                                  */
    int64_t n_steps;        /* steps to its end time                              */
    double spacing;         /* its node spacing h: with common.gamma_c > 0 its
                               gamma is common.gamma_c * spacing^(2 hv_k - 1)    */
    double gamma_c;         /* > 0: its own hyperviscosity constant in place of
                               common.gamma_c (0: the common one)                */
} rbf_ens_member;

/*
 * a8  Batched ensemble of Navier-Stokes runs of uneven size (no counterpart
 * in the paper, which runs one case at a time; each member is the method of
 * Secs. 3, 5.2, 5.3 and 6.2-6.3 with its own nodes, stencil size, degree,
 * spacing and dt).  common supplies the physics, PHS exponents, hyperviscosity
 * power and precision; its n_sten, poly_l, period_x and gamma are replaced
 * per member.  x, z are the members' node arrays concatenated (host, double);
 * kind concatenates the members' prognostic kinds and ghost_owner their ghost
 * owners (member-local indices), as for rbf_ns_create.  The state is the
 * members' node-major records concatenated in the same order
 * ([sum n_all][4]).  common.threads_per_node = 0 autotunes the lanes per node
 * for the whole ensemble; 1, 2 or 4 fixes them (RBF_E_ARG otherwise).
 */
int rbf_ens_create(rbf_problem **out, const rbf_ns_params *common, int32_t n_members,
                   const rbf_ens_member *members, const double *x, const double *z, const int32_t *kind,
                   const int32_t *ghost_owner, void *stream);

/*
 * Advances every member by min(max_steps, its n_steps) RK4 steps of its own
 * dt (max_steps < 0: to each member's end); members that finish drop out of
 * the launches.  Asynchronous on the problem's stream.
 */
int rbf_ens_run(rbf_problem *pb, int64_t max_steps, void *U);

/* Node updates (prognostic nodes x steps) that rbf_ens_run(max_steps) performs. */
int rbf_ens_node_updates(const rbf_problem *pb, int64_t max_steps, double *out);

/* ---- a9: learned tendency correction ----------------------------------------
 * The paper has no learned component; this is a small per-node MLP that
 * corrects coarse runs of the method.  Features of node i: the stencil
 * differences U_f(x_j) - U_f(x_i) of the four fields over the n - 1
 * non-centre nodes of i's stencil divided by per-field scales s_in
 * (field-major order, 4 (n - 1) values), then the node's own four values
 * divided by s_own (4 values).  Network: f(x) = h2 W3 + b3 with
 * h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2), width 64, BF16 weights, FP32
 * accumulation; y = f(x) - f(0), so a locally uniform state gets no
 * correction.  Output: delta_f = y_f s_out[f] (y clipped to [-4, 4] when
 * applied), added as dt * delta after each coarse RK4 step (Dirichlet
 * components excluded).
 * Parameters (FP32 master copy, flat): W1 [4(n-1)+4][64], b1 [64], W2 [64][64],
 * b2 [64], W3 [64][4], b3 [4].  Data sets: states [n_runs][n_snap][n_all][4]
 * FP32 (ghosts filled), targets [n_runs][n_snap-1][n_prog][4] FP32.
 */
typedef struct rbf_mlp rbf_mlp;

/* MLP bound to a coarse Navier-Stokes problem (its stencils and flags); the
 * problem must outlive the MLP.  Weights start at zero: set them. */
int rbf_mlp_create(rbf_mlp **out, rbf_problem *coarse, void *stream);
int rbf_mlp_n_params(const rbf_mlp *m, int64_t *out);
/* host float [n_params]; also refreshes the BF16 copy and resets Adam */
int rbf_mlp_set_params(rbf_mlp *m, const float *params);
int rbf_mlp_get_params(const rbf_mlp *m, float *params);
/* host float [12]: s_in[4], s_out[4], s_own[4] (all > 0) */
int rbf_mlp_set_scales(rbf_mlp *m, const float *scales);
int rbf_mlp_get_scales(const rbf_mlp *m, float *scales);
/* scales = root mean squares of the differences, targets and values of a data set (device) */
int rbf_mlp_fit_scales(rbf_mlp *m, const float *states, const float *targets, int64_t n_runs, int64_t n_snap);
/*
 * Loss (mean over samples and outputs of (y - target/s_out)^2, y unclipped) and its
 * gradient for a given batch: samples device int64 [batch][2] (target index
 * k in [0, n_runs (n_snap-1)), node i); grad_host float [n_params].
 */
int rbf_mlp_grad(rbf_mlp *m, const float *states, const float *targets, int64_t n_runs, int64_t n_snap,
                 const int64_t *samples, int32_t batch, float *grad_host, float *loss_host);
/* iters Adam steps on random batches (seeded on the device); loss_host [iters] or NULL */
int rbf_mlp_train(rbf_mlp *m, const float *states, const float *targets, int64_t n_runs, int64_t n_snap,
                  int64_t iters, int32_t batch, float lr, uint64_t seed, float *loss_host);
/* delta [n_prog][4] for a state U [n_all][4] whose ghosts are filled (device) */
int rbf_mlp_forward(rbf_mlp *m, const void *U, void *delta);
/*
 * n_steps corrected coarse steps: ghost fill, delta = MLP(U), RK4 step,
 * U_f += alpha[f] * dt * delta_f (alpha: host double [4], each >= 0; all
 * zero is the uncorrected solver).
 * A non-finite delta is skipped (the uncorrected step is kept) and counted
 * in *n_fallback (host, optional).  Synchronous.
 */
int rbf_learned_run(rbf_mlp *m, double t0, double dt, int64_t n_steps, const double *alpha, void *U,
                    int64_t *n_fallback);
/*
 * Chooses the coarse problem's persistent plan (lanes per node, CTAs) for
 * corrected runs: times short corrected runs of the fused persistent kernel
 * on a zero state for lanes 1, 2, 4 and one CTA per SM, per 2, 4 or 8 SMs,
 * and keeps the fastest.  The problem's run mode becomes persistent with that
 * plan (rbf_run uses it too; rbf_get_info reports it).  Synchronous.
 * Errors: RBF_E_ARG if no persistent kernel holding the network fits the
 * problem (FP64 problems, or too many nodes for one co-resident grid).
 */
int rbf_mlp_tune_run(rbf_mlp *m);
int rbf_mlp_destroy(rbf_mlp *m);
/*
 * Restriction by injection (device): for e < n_map, record
 * (e / block_records) * block_stride + e % block_records of dst takes record
 * map[e] of src (node-major records of 4 fields; precisions 32 or 64).
 */
int rbf_restrict(const void *src, int32_t src_precision, const int64_t *map, int64_t n_map, void *dst,
                 int32_t dst_precision, int64_t block_records, int64_t block_stride, void *stream);
/*
 * Weighted restriction (device): dst record of entry e (placed as in
 * rbf_restrict) = sum over q < m of w[e][q] * src record idx[e][q];
 * idx int64 [n_map][m], w double [n_map][m]; dst FP32.
 */
int rbf_restrict_weighted(const void *src, int32_t src_precision, const int64_t *idx, const double *w, int32_t m,
                          int64_t n_map, float *dst, int64_t block_records, int64_t block_stride, void *stream);
/* The ghost solve of Sec. 5.2 alone: fills the ghost records of U (device). */
int rbf_fill_ghosts(rbf_problem *pb, void *U);
/*
 * Training targets of a data set: target (r, k) = (state (r, k+1) -
 * one coarse RK4 step from state (r, k)) / dt.  FP32 problem; device arrays.
 */
int rbf_mlp_targets(rbf_problem *pb, const float *states, int64_t n_runs, int64_t n_snap, double dt, float *targets);

/*
 * a4+a5(+a6)  Right-hand side at time t.
 *   U     device, FP64 or FP32 per the problem's precision:
 *         NS [n_all][4] (ghost records are overwritten with the solved
 *         ghost values); advection [n_prog][1]
 *   dUdt  device, same precision, [n_prog][F]
 */
int rbf_rhs(rbf_problem *pb, double t, void *U, void *dUdt);

/*
 * a7  One classical RK4 step of size dt from time t, in place on U
 * (layout as for rbf_rhs).  Dirichlet components (w on bottom/top walls,
 * u on left/right walls) keep their values.
 */
int rbf_rk4_step(rbf_problem *pb, double t, double dt, void *U);

/*
 * n_steps RK4 steps from t0, in the problem's run mode (rbf_set_run_mode):
 * replayed from a captured CUDA graph of the per-stage kernels, or one
 * persistent cooperative launch for all steps.  Asynchronous on the
 * problem's stream; rbf_sync reports a persistent launch that gave up.
 */
int rbf_run(rbf_problem *pb, double t0, double dt, int64_t n_steps, void *U);

/*
 * Run modes of rbf_run for Navier-Stokes and scalar advection problems.
 *   RBF_RUN_GRAPH       ghost residual, ghost solve and fused stage kernels
 *                       per stage (advection: the stage kernel alone),
 *                       captured once and replayed as a graph.
 *   RBF_RUN_PERSISTENT  one cooperative launch runs every step: one CTA per
 *                       SM owns a contiguous slice of nodes, copies the
 *                       records its stencils read into shared memory each
 *                       stage, and grid barriers separate the ghost
 *                       residual, ghost solve and stage phases (Sec. 5.2,
 *                       Eqs. (uEq)-(piEq), RK4).  Results equal the graph
 *                       mode's with the same lanes per node.  Available when
 *                       every node fits one co-resident grid.
 *                       Advection problems (Sec. 6.1, RK4): every lane
 *                       keeps its packed slots in registers, each stage
 *                       gathers the stage input through L2 and the CTAs
 *                       meet at a grid barrier; results equal the graph
 *                       mode's bit for bit with the same lanes per node.
 *   RBF_RUN_AUTO        time both on a zero state and keep the faster
 *                       (done at creation when threads_per_node is 0, and
 *                       always for advection problems).
 * lanes: lanes per node of the persistent kernel (Navier-Stokes 1, 2 or 4;
 *        advection 2, 4 or 8, which also become the lanes of the graph
 *        mode; 0 = fastest).
 * ctas:  CTAs of the persistent kernel (0: fastest of 1, 1/2, 1/4, 1/8 per
 *        SM; with lanes > 0 and RBF_RUN_PERSISTENT, one per SM untimed).
 *        Advection problems take 0: their CTA count follows from the lanes
 *        and the fastest CTA size (64, 128 or 256 threads).
 * Errors: RBF_E_ARG if the mode or an argument is out of range, the problem
 * is an ensemble, or RBF_RUN_PERSISTENT does not fit.
 */
#define RBF_RUN_AUTO 0
#define RBF_RUN_GRAPH 1
#define RBF_RUN_PERSISTENT 2
int rbf_set_run_mode(rbf_problem *pb, int32_t mode, int32_t lanes, int32_t ctas);

/*
 * Split stage launches of the graph mode and of rbf_rk4_step (Sec. 5.2,
 * Eq. (bcEqn); Sec. 6.2).  The wall set is every node whose record a ghost
 * residual reads (the wall nodes' stencils) and every node whose stencil
 * reads a ghost.  With enable = 1 each stage runs as two launches: the other
 * nodes on a private stream, the wall set after the stage's ghost fill.  The
 * next stage's ghost residual and ghost solve need only the wall set, so
 * they run while the other launch finishes.  Each node's arithmetic is
 * unchanged, so the results are bitwise those of enable = 0.  It pays where
 * the ghost fill is a large share of a stage (small problems) and costs a
 * little where the stage kernel dominates, so a problem created with
 * threads_per_node = 0 times both and keeps the faster; otherwise it is off
 * until this call turns it on.  Stage timing (rbf_set_stage_timing) runs
 * unsplit.
 * Errors: RBF_E_ARG if pb is not a Navier-Stokes problem, or enable = 1 and
 * the problem has no wall set to split (no ghosts, or every node in it).
 */
int rbf_set_stage_split(rbf_problem *pb, int32_t enable);

/*
 * The node blocks of the persistent run mode, as a service for callers that
 * want the same decomposition: recursive coordinate bisection of the n points
 * (x, z) into `parts` blocks of equal size (+-1 node), each cut across the
 * longer extent of the points being split, ties by index.
 *   x, z      host, double [n]
 *   block_of  host, int32 [n] (out): block of each point, 0 .. parts-1
 * Host-only (no device call).  Errors: RBF_E_ARG for null pointers, n < 1,
 * parts outside [1, n] or non-finite coordinates.
 */
int rbf_partition_blocks(const double *x, const double *z, int64_t n, int32_t parts, int32_t *block_of);

/*
 * f4 (beyond the paper): how the graph-mode stage kernels store their
 * operators.  RBF_STORE_PER_NODE (the default) keeps one packed row of every
 * differentiation matrix per node, as Sec. 3 builds them.  RBF_STORE_LATTICE
 * groups nodes whose stencils are translates of each other -- the same
 * relative index offsets and relative positions, as on the interior and the
 * wall rows of Cartesian and hexagonal lattices -- into classes of at least
 * 32 members.  Each class keeps the packed operators of its first member,
 * and the stage kernel reads them from a table of a few tens of kB; the
 * other nodes keep their own rows.  The weights of a class's members agree
 * with its first member's up to rounding (identical augmented systems of
 * Eq. (weights)).  threads_per_node: 0 re-runs the autotuner with the new
 * storage, else 1, 2, 4 or 8.  class_nodes, n_classes (nullable, host)
 * receive the number of nodes in classes and of classes (0 for per-node
 * storage).  rbf_get_info's rhs_bytes_per_node follows the storage.  The
 * persistent run mode keeps its own operators and is not affected.
 * Synchronises the problem's stream.  RBF_E_ARG for an advection problem, an
 * ensemble (whose storage is chosen at creation, rbf_ns_params.storage) or
 * an unknown mode.
 */
int rbf_set_operator_storage(rbf_problem *pb, int32_t mode, int32_t threads_per_node, int64_t *class_nodes,
                             int32_t *n_classes);

/*
 * Host-only: the lattice classes of rbf_set_operator_storage for given
 * stencils.  idx [n_prog][n_sten] (host, int32, indices into the n_all
 * nodes), x, z [n_all] (host); period_x > 0 for a periodic x; h is the unit
 * of the position keys (relative positions are compared at h / 2^20).
 * cls [n_prog] (host) receives each node's class in the order of the
 * classes' first members, or -1 for nodes whose class has fewer than
 * min_members members; *n_classes the number of classes.  RBF_E_ARG for
 * null pointers, indices outside [0, n_all), non-finite coordinates or
 * h <= 0.
 */
int rbf_lattice_classes(const int32_t *idx, const double *x, const double *z, int64_t n_prog, int64_t n_all,
                        int32_t n_sten, double period_x, double h, int32_t min_members, int32_t *cls,
                        int32_t *n_classes);

/*
 * Bound on the polls of each grid-barrier wait of the persistent kernel
 * (default 2^21, about a second).  When a wait runs out, that CTA raises an
 * abort flag, every CTA leaves at its next barrier, the launch ends with the
 * state partially updated, and the next rbf_sync (or rbf_run_host) returns
 * RBF_E_TIMEOUT and clears the flag.  polls >= 0; 0 gives up at the first
 * wait that is not already complete (used by the tests of that path).
 */
int rbf_set_spin_limit(rbf_problem *pb, int64_t polls);

/*
 * End-to-end form of rbf_run on a HOST state: copies U_host to the device,
 * runs n_steps, copies the result back and waits.  U_host should be pinned.
 */
int rbf_run_host(rbf_problem *pb, double t0, double dt, int64_t n_steps, void *U_host);

/*
 * Waits for the problem's stream; returns RBF_E_CUDA on an asynchronous
 * fault and RBF_E_TIMEOUT if a persistent launch gave up a barrier wait.
 */
int rbf_sync(rbf_problem *pb);

/*
 * Per-field minimum and maximum over the prognostic nodes of U (device,
 * layout as for rbf_rhs), written to host out_minmax [F][2] (min, max).  Returns
 * RBF_E_NONFINITE if any prognostic value is NaN or Inf.  Synchronous.
 */
int rbf_minmax(rbf_problem *pb, const void *U, double *out_minmax);

/* Facts about a problem, for tests and measurement. */
typedef struct rbf_info {
    int64_t n_prog, n_all, n_ghost;
    int32_t n_fields, precision, n_sten, threads_per_node;
    int32_t slots;              /* packed neighbour slots per node          */
    int32_t launches_per_step;  /* kernel launches in one RK4 step of the
                                   graph mode (a persistent run is one launch) */
    int32_t n_components;       /* independent ghost systems                */
    int32_t n_ghost_classes;    /* distinct ghost matrices per component    */
    int32_t prefetch;           /* 1: stage kernel holds operands in registers */
    int32_t run_mode;           /* RBF_RUN_GRAPH or RBF_RUN_PERSISTENT       */
    double weight_build_ms;     /* GPU time of stencils + weights + pack    */
    double ghost_setup_ms;      /* GPU time of the ghost inverses           */
    double rhs_bytes_per_node;  /* algorithmic HBM bytes of one RHS stage   */
    double rhs_flops_per_node;  /* arithmetic of one RHS stage              */
    int32_t persist_lanes;      /* persistent kernel: lanes per node (0: none) */
    int32_t persist_regs;       /* 1: it keeps its operands in registers    */
    int32_t persist_chunk;      /* nodes per CTA                            */
    int32_t persist_halo_max;   /* largest per-CTA record list (0 for
                                   advection, which gathers through L2)      */
    int32_t persist_ctas;       /* CTAs of the persistent launch            */
    int32_t stage_split;        /* 1: split stage launches (rbf_set_stage_split) */
} rbf_info;
int rbf_get_info(const rbf_problem *pb, rbf_info *out);

/*
 * Copies of the problem's FP64 weights, for parity tests:
 *   op = RBF_OP_*; out host double [n_prog][n_sten] and (optional) out_idx
 *   host int32 [n_prog][n_sten].  RBF_E_ARG if the problem has no such op.
 */
int rbf_get_weights(const rbf_problem *pb, int32_t op, double *out, int32_t *out_idx);

/*
 * Stage-kernel timing for measurement.  With enable != 0, rbf_run captures
 * one RK4 step per graph and records CUDA events around each of the four
 * fused right-hand-side + RK4 stage kernels; rbf_stage_kernel_ms then waits
 * and returns (host double) their summed device time in the last replayed
 * step.  RBF_E_ARG if timing is off or no step has run.
 */
int rbf_set_stage_timing(rbf_problem *pb, int32_t enable);
int rbf_stage_kernel_ms(rbf_problem *pb, double *ms);

/* Destroys the problem and frees its device memory (after a sync). */
int rbf_destroy(rbf_problem *pb);

#ifdef __cplusplus
}
#endif
#endif /* RBFFD_H */
