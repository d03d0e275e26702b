// a2: RBF-FD weights from the augmented PHS + polynomial system
// (Sec. 3, Eq. (weights); hyperviscosity by the PHS Laplacian recursion of
// Sec. 5.3, Eq. (laplacian)).
//
// GPU design: one warp per stencil.  The S x (S + K) augmented matrix
// (S = n + (l+1)(l+2)/2 unknowns, K right-hand sides = operators) lives in
// shared memory; the warp runs Gaussian elimination with partial pivoting
// (lanes own columns, the elimination walks the rows), then a column-oriented
// back substitution (lanes own rows).  All arithmetic is FP64: the systems'
// conditioning grows with the PHS order (Sec. 2), and the work is FP64-ALU
// bound (about (2/3) S^3 flops per node), not a dense GEMM.
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

__global__ void weights_kernel(const double *__restrict__ x, const double *__restrict__ z,
                               const int32_t *__restrict__ idx, int64_t n_centers, WeightJob job,
                               double *__restrict__ w, int *__restrict__ bad_node) {
    extern __shared__ double sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp;
    if (c >= n_centers) return;
    const int n = job.n, S = job.S, ld = job.ld, K = job.nops;
    double *A = sm + (size_t)warp * (S * ld + 2 * n + 8);
    double *xi = A + S * ld;
    double *eta = xi + n;

    // shifted coordinates and stencil radius s = max_j ||x_j - x_c||
    const int32_t *row = idx + c * n;
    const double xc = x[c], zc = z[c];
    double smax = 0.0;
    bool bad_idx = false;
    for (int j = lane; j < n; j += 32) {
        int q = row[j];
        if (q < 0 || q >= job.n_all) { bad_idx = true; q = (int)c; }
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
    if (__any_sync(0xffffffffu, bad_idx)) {   // index outside [0, n_all): report, skip
        if (lane == 0) atomicMin(bad_node, (int)c);
        return;
    }
    const double inv_s = 1.0 / smax;
    __syncwarp();
    for (int j = lane; j < n; j += 32) { xi[j] *= inv_s; eta[j] *= inv_s; }
    __syncwarp();

    // assemble [A P | rhs; P^T 0 | rhs]; the PHS block is symmetric, so each
    // pair (i <= j) is evaluated once (entries of the upper triangle walked
    // row by row, 32 apart per lane)
    {
        int i = 0, j = lane;
        while (i < n && j >= n) { j -= n - i - 1; ++i; }   // j - i counts from the diagonal
        for (; i < n;) {
            double dx = xi[i] - xi[j], dz = eta[i] - eta[j];
            double r2 = dx * dx + dz * dz;
            const double v = (r2 == 0.0) ? 0.0 : rpow_odd(r2, sqrt(r2), job.p);
            A[i * ld + j] = v;
            A[j * ld + i] = v;
            j += 32;
            while (i < n && j >= n) { j -= n - i - 1; ++i; }
        }
    }
    for (int i = lane; i < n; i += 32) {
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
    for (int e = lane; e < job.M * job.M; e += 32) {
        int r = e / job.M, q = e - r * job.M;
        A[(n + r) * ld + n + q] = 0.0;
    }
    if (lane < job.M) {
        int m = 0;
        for (int d = 0; d <= job.l; ++d)
            for (int b = 0; b <= d; ++b, ++m)
                if (m == lane)
                    for (int o = 0; o < K; ++o) A[(n + m) * ld + S + o] = poly_rhs(job.ops[o], job.k, d - b, b);
    }
    __syncwarp();

    // Gaussian elimination with partial pivoting on the S x (S + K) block.
    // The pivot search compares |a| through its bit pattern (for non-negative
    // doubles the integer order is the numeric order), keeping the compares off
    // the FP64 pipe; the rank-1 update of the trailing block spreads its entries
    // over all 32 lanes.
    const int W = S + K;
    bool singular = false;
    const long long kTiny = __double_as_longlong(1e-14);
    const long long kInf = 0x7ff0000000000000LL;
    for (int kk = 0; kk < S; ++kk) {
        long long best = -1;
        int bi = kk;
        for (int i = kk + lane; i < S; i += 32) {
            const long long v = __double_as_longlong(A[i * ld + kk]) & 0x7fffffffffffffffLL;
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (!(best > kTiny) || best >= kInf) { singular = true; break; }   // tiny, inf or NaN pivot
        if (bi != kk)
            for (int j = kk + lane; j < W; j += 32) {
                double t = A[kk * ld + j];
                A[kk * ld + j] = A[bi * ld + j];
                A[bi * ld + j] = t;
            }
        __syncwarp();
        // multipliers of the rows below the pivot, kept in the pivot column
        const double inv = 1.0 / A[kk * ld + kk];
        for (int i = kk + 1 + lane; i < S; i += 32) A[i * ld + kk] *= inv;
        __syncwarp();
        // A[i][j] -= m_i p_j over the (S-kk-1) x (W-kk-1) trailing block, its
        // entries walked row by row, 32 apart per lane, two per pass
        const int w = W - kk - 1;
        if (w > 0) {
            int i = kk + 1, j = kk + 1 + lane;
            while (j >= W && i < S) { j -= w; ++i; }
            while (i < S) {
                int i2 = i, j2 = j + 32;
                while (j2 >= W && i2 < S) { j2 -= w; ++i2; }
                const double m0 = A[i * ld + kk], p0 = A[kk * ld + j], a0 = A[i * ld + j];
                const bool two = i2 < S;
                double m1 = 0.0, p1 = 0.0, a1 = 0.0;
                if (two) { m1 = A[i2 * ld + kk]; p1 = A[kk * ld + j2]; a1 = A[i2 * ld + j2]; }
                A[i * ld + j] = a0 - m0 * p0;
                if (two) A[i2 * ld + j2] = a1 - m1 * p1;
                i = i2;
                j = j2 + 32;
                while (j >= W && i < S) { j -= w; ++i; }
            }
        }
        __syncwarp();
    }
    if (singular) {
        if (lane == 0) atomicMin(bad_node, (int)c);
        return;
    }
    // back substitution, column-oriented: x_i = b_i / u_ii, then b_j -= u_ji x_i
    for (int i = S - 1; i >= 0; --i) {
        if (lane < K) A[i * ld + S + lane] /= A[i * ld + i];
        __syncwarp();
        for (int j = lane; j < i; j += 32) {
            double u = A[j * ld + i];
            for (int o = 0; o < K; ++o) A[j * ld + S + o] -= u * A[i * ld + S + o];
        }
        __syncwarp();
    }
    for (int o = 0; o < K; ++o) {
        double scale = 1.0;
        for (int t = 0; t < job.order[o]; ++t) scale *= inv_s;
        for (int j = lane; j < n; j += 32) w[((int64_t)o * n_centers + c) * n + j] = A[j * ld + S + o] * scale;
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
    job.ld = (job.S + n_ops) | 1;   // odd leading dimension: fewer bank conflicts
    size_t per_warp = ((size_t)job.S * job.ld + 2 * n + 8) * sizeof(double);
    // as many systems per CTA (one CTA per SM) as the 227 KB of shared memory
    // a CTA may hold, up to 8: the SM's four sub-partitions each have their
    // own share of the FP64 pipe, so fewer than four warps leave part of it
    // idle (S = 77: 52 KB per system, 4 warps)
    int max_smem = 0, dev = 0;
    RBF_CUDA(cudaGetDevice(&dev));
    RBF_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    int warps = (int)std::min<size_t>(8, (size_t)max_smem / per_warp);
    RBF_REQUIRE(warps >= 1, "weight system too large for shared memory");
    RBF_CUDA(cudaFuncSetAttribute(weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(warps * per_warp)));
    DevBuf<int> bad(1);
    int init = INT_MAX;
    RBF_CUDA(cudaMemcpyAsync(bad.p, &init, sizeof(int), cudaMemcpyHostToDevice, st));
    weights_kernel<<<div_up(n_centers, warps), warps * 32, warps * per_warp, st>>>(x, z, idx, n_centers, job, w, bad.p);
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
