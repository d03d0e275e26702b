// a2: RBF-FD weights from the augmented PHS + polynomial system
// (Sec. 3, Eq. (weights); hyperviscosity by the PHS Laplacian recursion of
// Sec. 5.3, Eq. (laplacian)).
//
// GPU design: one CTA of four warps per stencil.  The S x (S + K) augmented
// matrix (S = n + (l+1)(l+2)/2 unknowns, K right-hand sides = operators) lives
// in shared memory.  The CTA runs Gaussian elimination with partial pivoting,
// one barrier per step: warp 0 looks one column ahead (update, pivot,
// multipliers) while the other three warps update the trailing block.  A
// column-oriented back substitution follows.  All arithmetic is FP64: the
// systems' conditioning grows with the PHS order (Sec. 2), and the work is
// FP64-ALU bound (about (2/3) S^3 flops per node), not a dense GEMM.
#include <climits>
#include <cmath>

#include "common.cuh"

namespace rbf {

namespace {

constexpr int kMaxOps = 6;
constexpr int kMaxS = 160;   // largest system size

struct WeightJob {
    int n, M, S, ld;       // stencil size, monomials, system size, leading dim
    int p, l, k;           // PHS exponent, degree, Delta power
    int nops;
    int ops[kMaxOps];
    int order[kMaxOps];    // derivative order of each operator (for rescaling)
    double period;
    int64_t n_all;         // bound of the stencil indices
};

// r^e for odd e >= -1, given r2 = r^2 and r = sqrt(r2), r > 0.
__device__ __forceinline__ double rpow_odd(double r2, double r, int e) {
    if (e == -1) return 1.0 / r;
    double v = r;
    for (int t = 0; t < (e - 1) / 2; ++t) v *= r2;
    return v;
}

// L applied to ||x - x_j||^p at the centre, with (dx, dz) = x_c - x_j.
__device__ double phs_rhs(int op, int p, int k, double dx, double dz) {
    double r2 = dx * dx + dz * dz;
    if (r2 == 0.0) return 0.0;
    double r = sqrt(r2);
    switch (op) {
        case RBF_OP_DX: return p * rpow_odd(r2, r, p - 2) * dx;
        case RBF_OP_DZ: return p * rpow_odd(r2, r, p - 2) * dz;
        case RBF_OP_LAP: return (double)(p * p) * rpow_odd(r2, r, p - 2);
        case RBF_OP_DXX: return p * rpow_odd(r2, r, p - 2) + (double)(p * (p - 2)) * rpow_odd(r2, r, p - 4) * dx * dx;
        case RBF_OP_DZZ: return p * rpow_odd(r2, r, p - 2) + (double)(p * (p - 2)) * rpow_odd(r2, r, p - 4) * dz * dz;
        case RBF_OP_HV: {
            // Delta r^q = q^2 r^(q-2) in two dimensions, applied k times
            double c = 1.0;
            int q = p;
            for (int t = 0; t < k; ++t) { c *= (double)q * q; q -= 2; }
            return c * rpow_odd(r2, r, q);
        }
    }
    return 0.0;
}

__device__ __forceinline__ double factorial(int m) {
    double f = 1.0;
    for (int i = 2; i <= m; ++i) f *= i;
    return f;
}

// L applied to xi^a eta^b at the origin.
__device__ double poly_rhs(int op, int k, int a, int b) {
    switch (op) {
        case RBF_OP_DX: return (a == 1 && b == 0) ? 1.0 : 0.0;
        case RBF_OP_DZ: return (a == 0 && b == 1) ? 1.0 : 0.0;
        case RBF_OP_LAP: return ((a == 2 && b == 0) || (a == 0 && b == 2)) ? 2.0 : 0.0;
        case RBF_OP_DXX: return (a == 2 && b == 0) ? 2.0 : 0.0;
        case RBF_OP_DZZ: return (a == 0 && b == 2) ? 2.0 : 0.0;
        case RBF_OP_HV: {
            // Delta^k = sum_i C(k, i) d^2i/dx^2i d^2(k-i)/dz^2(k-i)
            if ((a & 1) || (b & 1) || a + b != 2 * k) return 0.0;
            int i = a / 2;
            double comb = factorial(k) / (factorial(i) * factorial(k - i));
            return comb * factorial(a) * factorial(b);
        }
    }
    return 0.0;
}

// Look-ahead step of weights_kernel, run by one warp: the pivot of column
// col among logical rows col.. (permutation pc), the permutation with the
// pivot row moved to col (pn; pn == pc allowed), the pivot, its failure flag
// (by the step's parity) and the multipliers of the rows below it.
__device__ __forceinline__ void pivot_step(double *A, int ld, int S, int col, const int *pc, int *pn, double *mvn,
                                           double *diag, int *s_bad, int lane) {
    const long long kTiny = __double_as_longlong(1e-14);
    const long long kInf = 0x7ff0000000000000LL;
    long long best = -1;
    int bi = col;
    for (int i = col + lane; i < S; i += 32) {
        const long long v = __double_as_longlong(A[pc[i] * ld + col]) & 0x7fffffffffffffffLL;
        if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    const bool bad = !(best > kTiny) || best >= kInf;   // tiny, inf or NaN pivot
    const int rc = pc[col], rb = pc[bi];
    const double piv = A[rb * ld + col];
    __syncwarp();
    if (pn != pc)   // entries from col - 1 on: pn then holds every settled entry
        for (int i = col - 1 + lane; i < S; i += 32) pn[i] = pc[i];
    __syncwarp();
    if (lane == 0) {
        pn[col] = rb;
        pn[bi] = rc;
        diag[col] = piv;
        s_bad[col & 1] = bad;
    }
    __syncwarp();
    const double inv = bad ? 0.0 : 1.0 / piv;
    for (int i = col + 1 + lane; i < S; i += 32) mvn[i] = A[pn[i] * ld + col] * inv;
}

// One CTA of NT threads per stencil, one barrier per elimination step.  Rows
// are addressed through a permutation (logical row -> shared-memory row)
// instead of being swapped.  In step kk, warp 0 updates column kk+1, finds the
// pivot of step kk+1 and writes the next permutation and multipliers (both
// double-buffered), while the other warps update columns kk+2.. of the
// trailing block with the current ones.  The results are the same bits as a
// plain elimination with row swaps: every entry sees the same operations.
template <int NT>
__global__ void __launch_bounds__(NT) weights_kernel(const double *__restrict__ x, const double *__restrict__ z,
                                                     const int32_t *__restrict__ idx, int64_t n_centers,
                                                     WeightJob job, double *__restrict__ w,
                                                     int *__restrict__ bad_node) {
    extern __shared__ double sm[];
    __shared__ double s_red[NT / 32];
    __shared__ int s_bad[2];        // pivot failure flags, by the parity of the step they belong to
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t c = blockIdx.x;
    if (c >= n_centers) return;
    const int n = job.n, S = job.S, ld = job.ld, K = job.nops, W = S + K;
    double *A = sm;                 // S x ld, row-major, rows in shared-memory order
    double *xi = A + S * ld;        // n shifted, scaled coordinates
    double *eta = xi + n;
    double *const mv0 = eta + n, *const mv1 = mv0 + S;   // multipliers, double-buffered by step
    double *const diag = mv1 + S;                         // S pivots (the diagonal of U)
    int *const pm0 = reinterpret_cast<int *>(diag + S), *const pm1 = pm0 + S;   // permutations, likewise

    const int32_t *row = idx + c * n;
    const double xc = x[c], zc = z[c];
    double smax = 0.0;
    int bad_idx = 0;
    for (int j = tid; j < n; j += NT) {
        int q = row[j];
        if (q < 0 || q >= job.n_all) { bad_idx = 1; q = (int)c; }
        double dx = x[q] - xc;
        if (job.period > 0.0) {
            if (dx > 0.5 * job.period) dx -= job.period;
            else if (dx < -0.5 * job.period) dx += job.period;
        }
        double dz = z[q] - zc;
        xi[j] = dx;
        eta[j] = dz;
        smax = fmax(smax, sqrt(dx * dx + dz * dz));
    }
    for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    if (lane == 0) s_red[warp] = smax;
    if (__syncthreads_or(bad_idx)) {
        if (tid == 0) atomicMin(bad_node, (int)c);
        return;
    }
    smax = s_red[0];
    for (int q = 1; q < NT / 32; ++q) smax = fmax(smax, s_red[q]);
    const double inv_s = 1.0 / smax;
    for (int j = tid; j < n; j += NT) { xi[j] *= inv_s; eta[j] *= inv_s; }
    for (int i = tid; i < S; i += NT) { pm0[i] = i; pm1[i] = i; }
    __syncthreads();

    {
        int i = 0, j = tid;
        while (i < n && j >= n) { j -= n - i - 1; ++i; }
        for (; i < n;) {
            double dx = xi[i] - xi[j], dz = eta[i] - eta[j];
            double r2 = dx * dx + dz * dz;
            const double v = (r2 == 0.0) ? 0.0 : rpow_odd(r2, sqrt(r2), job.p);
            A[i * ld + j] = v;
            A[j * ld + i] = v;
            j += NT;
            while (i < n && j >= n) { j -= n - i - 1; ++i; }
        }
    }
    for (int i = tid; i < n; i += NT) {
        int m = 0;
        for (int d = 0; d <= job.l; ++d) {
            for (int b = 0; b <= d; ++b, ++m) {
                int a = d - b;
                double v = 1.0;
                for (int t = 0; t < a; ++t) v *= xi[i];
                for (int t = 0; t < b; ++t) v *= eta[i];
                A[i * ld + n + m] = v;
                A[(n + m) * ld + i] = v;
            }
        }
        for (int o = 0; o < K; ++o) A[i * ld + S + o] = phs_rhs(job.ops[o], job.p, job.k, -xi[i], -eta[i]);
    }
    for (int e = tid; e < job.M * job.M; e += NT) {
        int r = e / job.M, q = e - r * job.M;
        A[(n + r) * ld + n + q] = 0.0;
    }
    if (tid < job.M) {
        int m = 0;
        for (int d = 0; d <= job.l; ++d)
            for (int b = 0; b <= d; ++b, ++m)
                if (m == tid)
                    for (int o = 0; o < K; ++o) A[(n + m) * ld + S + o] = poly_rhs(job.ops[o], job.k, d - b, b);
    }
    __syncthreads();

    if (warp == 0) pivot_step(A, ld, S, 0, pm0, pm0, mv0, diag, s_bad, lane);
    __syncthreads();
    int cur = 0;
    int failed = s_bad[0];
    if (!failed) {
        for (int kk = 0; kk < S; ++kk) {
            const int *pc = cur ? pm1 : pm0;
            const double *mc = cur ? mv1 : mv0;
            const double *prow = A + pc[kk] * ld;
            if (warp == 0) {
                if (kk + 1 < S) {
                    const double pk = prow[kk + 1];
                    for (int i = kk + 1 + lane; i < S; i += 32) A[pc[i] * ld + kk + 1] -= mc[i] * pk;
                    __syncwarp();
                    pivot_step(A, ld, S, kk + 1, pc, cur ? pm0 : pm1, cur ? mv0 : mv1, diag, s_bad, lane);
                }
            } else {
                // A[i][j] -= m_i p_j, logical rows i > kk, columns j >= kk+2,
                // entries NT-32 apart in row-major order, two per pass
                constexpr int NB = NT - 32;
                const int wcols = W - kk - 2, rows = S - kk - 1;
                if (wcols > 0 && rows > 0) {
                    const int qi = NB / wcols, qj = NB - qi * wcols;
                    const int t = tid - 32;
                    int i = t / wcols, j = t - i * wcols;
                    const int *prm = pc + kk + 1;
                    const double *mrow = mc + kk + 1;
                    const double *pr = prow + kk + 2;
                    while (i < rows) {
                        int i2 = i + qi, j2 = j + qj;
                        if (j2 >= wcols) { j2 -= wcols; ++i2; }
                        double *r0 = A + prm[i] * ld + kk + 2;
                        const double m0 = mrow[i], p0 = pr[j], a0 = r0[j];
                        const bool two = i2 < rows;
                        double m1 = 0.0, p1 = 0.0, a1 = 0.0;
                        double *r1 = r0;
                        if (two) { r1 = A + prm[i2] * ld + kk + 2; m1 = mrow[i2]; p1 = pr[j2]; a1 = r1[j2]; }
                        r0[j] = a0 - m0 * p0;
                        if (two) r1[j2] = a1 - m1 * p1;
                        i = i2 + qi;
                        j = j2 + qj;
                        if (j >= wcols) { j -= wcols; ++i; }
                    }
                }
            }
            __syncthreads();
            if (kk + 1 < S) {
                if (s_bad[(kk + 1) & 1]) { failed = 1; break; }   // the pivot of step kk+1 (uniform)
                cur ^= 1;
            }
        }
    }
    if (failed) {
        if (tid == 0) atomicMin(bad_node, (int)c);
        return;
    }
    const int *P = cur ? pm1 : pm0;   // the last step's permutation: every entry settled
    for (int i = S - 1; i >= 0; --i) {
        if (tid < K) A[P[i] * ld + S + tid] /= diag[i];
        __syncthreads();
        const double *xr = A + P[i] * ld + S;
        for (int e = tid; e < i * K; e += NT) {
            const int j = e / K, o = e - j * K;
            double *rj = A + P[j] * ld;
            rj[S + o] -= rj[i] * xr[o];
        }
        __syncthreads();
    }
    for (int o = 0; o < K; ++o) {
        double scale = 1.0;
        for (int t = 0; t < job.order[o]; ++t) scale *= inv_s;
        for (int j = tid; j < n; j += NT) w[((int64_t)o * n_centers + c) * n + j] = A[P[j] * ld + S + o] * scale;
    }
}

int op_order(int op, int k) {
    switch (op) {
        case RBF_OP_DX: case RBF_OP_DZ: return 1;
        case RBF_OP_LAP: case RBF_OP_DXX: case RBF_OP_DZZ: return 2;
        case RBF_OP_HV: return 2 * k;
    }
    return -1;
}

}  // namespace

void build_weights(const double *x, const double *z, int64_t n_all, const int32_t *idx, int64_t n_centers, int n,
                   double period_x, int p, int l, int hv_k, const int *ops, int n_ops, double *w,
                   cudaStream_t st) {
    RBF_REQUIRE(n >= 1 && n <= 128, "stencil size n=%d must be in [1, 128]", n);
    RBF_REQUIRE(p >= 1 && p <= 15 && (p & 1), "PHS exponent p=%d must be odd in [1, 15]", p);
    RBF_REQUIRE(l >= 0 && l <= 8, "polynomial degree l=%d must be in [0, 8]", l);
    RBF_REQUIRE(n_ops >= 1 && n_ops <= kMaxOps, "n_ops=%d must be in [1, %d]", n_ops, kMaxOps);
    RBF_REQUIRE(period_x >= 0.0, "period_x must be >= 0");
    WeightJob job{};
    job.n = n;
    job.M = (l + 1) * (l + 2) / 2;
    job.S = n + job.M;
    RBF_REQUIRE(job.S <= kMaxS, "system size n + (l+1)(l+2)/2 = %d exceeds %d", job.S, kMaxS);
    RBF_REQUIRE(job.M <= n, "need at least (l+1)(l+2)/2 = %d stencil nodes, have %d", job.M, n);
    job.p = p;
    job.l = l;
    job.k = hv_k;
    job.nops = n_ops;
    job.period = period_x;
    job.n_all = n_all;
    for (int o = 0; o < n_ops; ++o) {
        int op = ops[o];
        RBF_REQUIRE(op >= 0 && op <= 5, "unknown operator code %d", op);
        job.ops[o] = op;
        job.order[o] = op_order(op, hv_k);
        if (op == RBF_OP_HV) RBF_REQUIRE(hv_k >= 1 && p >= 2 * hv_k + 1, "Delta^%d needs p >= %d (p=%d)", hv_k, 2 * hv_k + 1, p);
        if (op == RBF_OP_DXX || op == RBF_OP_DZZ || op == RBF_OP_LAP) RBF_REQUIRE(p >= 3, "second derivatives need p >= 3");
    }
    if (n_centers == 0) return;
    RBF_REQUIRE(x && z && idx && w, "null pointer argument");
    RBF_REQUIRE(n_centers <= INT_MAX, "at most %d centres per call", INT_MAX);
    job.ld = (job.S + n_ops) | 1;   // odd leading dimension: fewer bank conflicts
    const size_t smem = ((size_t)job.S * job.ld + 2 * n + 4 * job.S + 8) * sizeof(double);
    int max_smem = 0, dev = 0;
    RBF_CUDA(cudaGetDevice(&dev));
    RBF_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    RBF_REQUIRE(smem + 1024 <= (size_t)max_smem, "weight system too large for shared memory");
    constexpr int kThreads = 128;   // four warps per system: one look-ahead, three on the trailing block
    RBF_CUDA(cudaFuncSetAttribute(weights_kernel<kThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DevBuf<int> bad(1);
    int init = INT_MAX;
    RBF_CUDA(cudaMemcpyAsync(bad.p, &init, sizeof(int), cudaMemcpyHostToDevice, st));
    weights_kernel<kThreads><<<(unsigned)n_centers, kThreads, smem, st>>>(x, z, idx, n_centers, job, w, bad.p);
    RBF_CHECK_LAUNCH();
    int hb = INT_MAX;
    RBF_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaStreamSynchronize(st));
    if (hb != INT_MAX)
        RBF_FAIL(RBF_E_SINGULAR, "singular weight system (or stencil index outside [0, n_all)) at node %d", hb);
}

}  // namespace rbf

extern "C" int rbf_build_weights(const double *x, const double *z, int64_t n_all, const int32_t *idx,
                                 int64_t n_centers, int32_t n, double period_x, int32_t p, int32_t l,
                                 int32_t hv_k, const int32_t *ops, int32_t n_ops, double *w, void *stream) {
    return rbf::guarded([&] {
        RBF_REQUIRE(n_centers >= 0 && n_centers <= n_all, "n_centers out of range");
        RBF_REQUIRE(ops != nullptr, "null ops");
        int o[6] = {0, 0, 0, 0, 0, 0};
        RBF_REQUIRE(n_ops >= 1 && n_ops <= 6, "n_ops=%d must be in [1, 6]", n_ops);
        for (int i = 0; i < n_ops; ++i) o[i] = ops[i];
        rbf::build_weights(x, z, n_all, idx, n_centers, n, period_x, p, l, hv_k, o, n_ops, w, rbf::as_stream(stream));
    });
}
