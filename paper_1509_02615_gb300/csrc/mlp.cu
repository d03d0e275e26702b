// a9: learned tendency correction for coarse runs (no counterpart in the
// paper; the paper's method is the solver it corrects).
//
// Per coarse node: features = the stencil differences of the four fields,
// scaled per field (4 (n-1) values, the node's own RBF-FD stencil); a 3-layer
// MLP f (width 64, tanh, BF16 weights, FP32 accumulation) gives the tendency
// correction delta = (f(x) - f(0)) s_out, added as dt * delta after each
// coarse RK4 step.  Subtracting f(0) makes a locally uniform state (all
// differences zero), where fine and coarse steps agree, uncorrected.
//
// Kernels (CUDA cores: the per-node contraction is ~14k MACs on a few
// thousand nodes, latency-bound, not a tensor-core sized GEMM):
//   mlp_infer_kernel  fused gather + forward, one thread per node, weights in
//                     shared memory as BF16
//   mlp_train_kernel  fused gather + forward + backward for 128 samples per
//                     block; per-block weight gradients (H^T dH products over
//                     the block's samples) are added to FP32 gradients
//   mlp_adam_kernel   Adam on FP32 master weights, refreshes the BF16 copy
#include <cuda_bf16.h>

#include <cmath>
#include <vector>
#include <cstring>

#include "problem.cuh"
#include "records.cuh"

namespace rbf {

constexpr int kWidth = 64;
constexpr int kTrainBlock = 128;
constexpr int kScaleWarps = 2048;   // warps of the scale-sum launch (256 blocks of 256 threads)
constexpr float kClip = 4.f;   // |y| <= 4 (in output-scale units) when the correction is applied

struct Mlp {
    int n = 0, slots = 0, n_in = 0;
    int64_t n_params = 0;
    int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
    cudaStream_t st = nullptr;
    DevBuf<float> P, Gr, M, V, scales, loss;
    DevBuf<float> Gp, Lp;     // per-block gradient and loss partials of a training launch
    DevBuf<__nv_bfloat16> Pb;
    DevBuf<double> acc;       // scale sums
    DevBuf<unsigned long long> bad;
    int64_t t = 0;
};

namespace {

struct Offs {   // parameter offsets: W1 [n_in][64], b1, W2 [64][64], b2, W3 [64][4], b3
    int64_t oW1, ob1, oW2, ob2, oW3, ob3;
};

Offs offs_of(const Mlp &m) { return {m.oW1, m.ob1, m.oW2, m.ob2, m.oW3, m.ob3}; }

// state of target sample k: runs hold n_snap states and n_snap - 1 targets
__device__ __forceinline__ int64_t state_of(int64_t k, int64_t n_snap) {
    return (k / (n_snap - 1)) * n_snap + k % (n_snap - 1);
}

struct Net {
    const __nv_bfloat16 *W1, *W2, *W3;
    const float *b1, *b2, *b3;
};

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// shared-memory image of the network: BF16 weights, FP32 biases
__device__ Net load_net(unsigned char *sm, const __nv_bfloat16 *Pb, const float *P, int n_in, const Offs o) {
    const int64_t oW1 = o.oW1, ob1 = o.ob1, oW2 = o.oW2, ob2 = o.ob2, oW3 = o.oW3, ob3 = o.ob3;
    __nv_bfloat16 *w1 = reinterpret_cast<__nv_bfloat16 *>(sm);
    __nv_bfloat16 *w2 = w1 + n_in * kWidth;
    __nv_bfloat16 *w3 = w2 + kWidth * kWidth;
    float *b = reinterpret_cast<float *>(w3 + kWidth * 4);
    for (int e = threadIdx.x; e < n_in * kWidth; e += blockDim.x) w1[e] = Pb[oW1 + e];
    for (int e = threadIdx.x; e < kWidth * kWidth; e += blockDim.x) w2[e] = Pb[oW2 + e];
    for (int e = threadIdx.x; e < kWidth * 4; e += blockDim.x) w3[e] = Pb[oW3 + e];
    for (int e = threadIdx.x; e < kWidth; e += blockDim.x) {
        b[e] = P[ob1 + e];
        b[kWidth + e] = P[ob2 + e];
    }
    if (threadIdx.x < 4) b[2 * kWidth + threadIdx.x] = P[ob3 + threadIdx.x];
    __syncthreads();
    return {w1, w2, w3, b, b + kWidth, b + 2 * kWidth};
}

// f(0) of the network (the output for all-zero features), and its hidden
// activations, computed by the first 64 threads of the block into z1, z2, y0.
__device__ void zero_branch(const Net &net, float *z1, float *z2, float *y0) {
    const int t = threadIdx.x;
    if (t < kWidth) z1[t] = tanhf(net.b1[t]);
    __syncthreads();
    if (t < kWidth) {
        float a = net.b2[t];
        for (int m = 0; m < kWidth; ++m) a += z1[m] * bf(net.W2[m * kWidth + t]);
        z2[t] = tanhf(a);
    }
    __syncthreads();
    if (t < 4) {
        float a = net.b3[t];
        for (int m = 0; m < kWidth; ++m) a += z2[m] * bf(net.W3[m * 4 + t]);
        y0[t] = a;
    }
    __syncthreads();
}

__host__ __device__ __forceinline__ size_t net_bytes(int n_in) {
    return (size_t)(n_in * kWidth + kWidth * kWidth + kWidth * 4) * 2 + (2 * kWidth + 4) * 4;
}

// h1 += x (row r of W1) for the features of one neighbour (4 fields)
__device__ __forceinline__ void layer1_row(float *h, const __nv_bfloat16 *w1, int row, float x) {
    const __nv_bfloat162 *w = reinterpret_cast<const __nv_bfloat162 *>(w1 + row * kWidth);
#pragma unroll
    for (int j = 0; j < kWidth / 2; ++j) {
        const float2 v = __bfloat1622float2(w[j]);
        h[2 * j] += x * v.x;
        h[2 * j + 1] += x * v.y;
    }
}

// out = tanh(in W + b), 64 x 64
__device__ __forceinline__ void layer2(const float *in, const __nv_bfloat16 *w2, const float *b, float *out) {
#pragma unroll
    for (int j = 0; j < kWidth; ++j) out[j] = b[j];
    for (int m = 0; m < kWidth; ++m) {
        const float x = in[m];
        const __nv_bfloat162 *w = reinterpret_cast<const __nv_bfloat162 *>(w2 + m * kWidth);
#pragma unroll
        for (int j = 0; j < kWidth / 2; ++j) {
            const float2 v = __bfloat1622float2(w[j]);
            out[2 * j] += x * v.x;
            out[2 * j + 1] += x * v.y;
        }
    }
#pragma unroll
    for (int j = 0; j < kWidth; ++j) out[j] = tanhf(out[j]);
}

// Fused gather + forward pass: delta[i] = MLP(features of node i) * s_out.
template <class T>
__global__ void __launch_bounds__(128) mlp_infer_kernel(const T *__restrict__ U, const int32_t *__restrict__ idx, int n,
                                                        int64_t n_prog, const __nv_bfloat16 *__restrict__ Pb,
                                                        const float *__restrict__ P, Offs m_off, const float *scales,
                                                        const unsigned char *__restrict__ flags, T *__restrict__ delta) {
    extern __shared__ unsigned char sm[];
    const int n_in = 4 * (n - 1) + 4;
    const Net net = load_net(sm, Pb, P, n_in, m_off);
    __shared__ float z1[kWidth], z2[kWidth], y0[4];
    zero_branch(net, z1, z2, y0);
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_prog) return;
    const float is0 = 1.f / scales[0], is1 = 1.f / scales[1], is2 = 1.f / scales[2], is3 = 1.f / scales[3];
    const Rec<T> own = load_rec(U, i);
    float h[kWidth];
#pragma unroll
    for (int j = 0; j < kWidth; ++j) h[j] = net.b1[j];
    const int slots = n - 1;
    for (int k = 1; k < n; ++k) {
        const Rec<T> r = load_rec(U, idx[i * n + k]);
        layer1_row(h, net.W1, 0 * slots + k - 1, (float)(r.u - own.u) * is0);
        layer1_row(h, net.W1, 1 * slots + k - 1, (float)(r.w - own.w) * is1);
        layer1_row(h, net.W1, 2 * slots + k - 1, (float)(r.t - own.t) * is2);
        layer1_row(h, net.W1, 3 * slots + k - 1, (float)(r.p - own.p) * is3);
    }
    // the node's own values
    layer1_row(h, net.W1, 4 * slots + 0, (float)own.u / scales[8]);
    layer1_row(h, net.W1, 4 * slots + 1, (float)own.w / scales[9]);
    layer1_row(h, net.W1, 4 * slots + 2, (float)own.t / scales[10]);
    layer1_row(h, net.W1, 4 * slots + 3, (float)own.p / scales[11]);
#pragma unroll
    for (int j = 0; j < kWidth; ++j) h[j] = tanhf(h[j]);
    float h2[kWidth];
    layer2(h, net.W2, net.b2, h2);
    float y[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) y[c] = net.b3[c];
#pragma unroll
    for (int m = 0; m < kWidth; ++m)
#pragma unroll
        for (int c = 0; c < 4; ++c) y[c] += h2[m] * bf(net.W3[m * 4 + c]);
    const unsigned char fl = flags[i];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        // y = f(x) - f(0); a safeguard clips the correction at 4 output scales
        float d = fminf(fmaxf(y[c] - y0[c], -kClip), kClip) * scales[4 + c];
        if ((c == 1 && (fl & 1)) || (c == 0 && (fl & 2))) d = 0.f;   // Dirichlet components stay fixed
        delta[i * 4 + c] = (T)d;
    }
}

// U += dt * delta on prognostic records; a non-finite delta is skipped
// (the node falls back to the uncorrected step) and counted.
template <class T>
__global__ void mlp_apply_kernel(T *U, const T *delta, int64_t n_prog, T dt, float4 alpha, unsigned long long *bad) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_prog * 4) return;
    const int f = (int)(e & 3);
    const T a = (T)(f == 0 ? alpha.x : f == 1 ? alpha.y : f == 2 ? alpha.z : alpha.w);
    const T d = delta[e];
    if (isfinite((double)d)) U[e] += a * dt * d;
    else atomicAdd(bad, 1ull);
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

struct TrainArgs {
    const float *S;       // states [n_runs][n_snap][n_all][4] (ghosts filled)
    const float *Tg;      // targets [n_runs][n_snap - 1][n_prog][4] (raw tendencies)
    int64_t n_states;     // targets: n_runs (n_snap - 1)
    int64_t n_snap;
    int64_t n_all, n_prog;
    const int32_t *idx;
    int n;
    const int64_t *samples;   // optional [B][2] (state, node); else drawn from seed
    unsigned long long seed;
    long long iter;
    int B;
    const __nv_bfloat16 *Pb;
    const float *P;
    const float *scales;
    float *Gp;            // [blocks][n_params]: this block's weight gradients
    int64_t n_params;
    float *Lp;            // [blocks]: this block's loss
};

// Fused gather + forward + backward for one block of 128 samples; the block's
// weight gradients (X^T dH1, H1^T dH2, H2^T dY and bias sums) and loss go to
// its own partials, which mlp_reduce_kernel sums over the blocks in block
// order (so training is deterministic).
__global__ void __launch_bounds__(kTrainBlock) mlp_train_kernel(TrainArgs a, Offs m_off) {
    extern __shared__ unsigned char sm[];
    float *const gp = a.Gp + blockIdx.x * a.n_params;
    const int n_in = 4 * (a.n - 1) + 4;
    const int xs = n_in + 1;                 // padded row strides (bank spread)
    const int hs = kWidth + 1;
    const Net net = load_net(sm, a.Pb, a.P, n_in, m_off);
    __shared__ float z1[kWidth], z2[kWidth], y0[4], dz[4], dz2[kWidth], dz1[kWidth];
    zero_branch(net, z1, z2, y0);
    float *X = reinterpret_cast<float *>(sm + ((net_bytes(n_in) + 15) & ~size_t(15)));
    float *H1 = X + kTrainBlock * xs;
    float *H2 = H1 + kTrainBlock * hs;
    float *DY = H2 + kTrainBlock * hs;
    __shared__ float red[kTrainBlock];
    const int t = threadIdx.x;
    const int s = blockIdx.x * kTrainBlock + t;
    const bool live = s < a.B;
    int64_t k = 0, i = 0;
    if (live) {
        if (a.samples) {
            k = a.samples[2 * (int64_t)s];
            i = a.samples[2 * (int64_t)s + 1];
        } else {
            const unsigned long long h = splitmix64(a.seed ^ splitmix64((unsigned long long)a.iter * 0x100000001ull + s));
            k = (int64_t)(h % (unsigned long long)a.n_states);
            i = (int64_t)((h >> 32) % (unsigned long long)a.n_prog);
        }
    }
    // features
    const float *Uk = a.S + state_of(k, a.n_snap) * a.n_all * 4;
    const Rec<float> own = load_rec(Uk, i);
    const float is0 = 1.f / a.scales[0], is1 = 1.f / a.scales[1], is2 = 1.f / a.scales[2], is3 = 1.f / a.scales[3];
    const int slots = a.n - 1;
    float *x = X + t * xs;
    float h[kWidth];
#pragma unroll
    for (int j = 0; j < kWidth; ++j) h[j] = net.b1[j];
    for (int q = 1; q < a.n; ++q) {
        const Rec<float> r = load_rec(Uk, a.idx[i * a.n + q]);
        const float f0 = live ? (r.u - own.u) * is0 : 0.f, f1 = live ? (r.w - own.w) * is1 : 0.f;
        const float f2 = live ? (r.t - own.t) * is2 : 0.f, f3 = live ? (r.p - own.p) * is3 : 0.f;
        x[q - 1] = f0;
        x[slots + q - 1] = f1;
        x[2 * slots + q - 1] = f2;
        x[3 * slots + q - 1] = f3;
        layer1_row(h, net.W1, q - 1, f0);
        layer1_row(h, net.W1, slots + q - 1, f1);
        layer1_row(h, net.W1, 2 * slots + q - 1, f2);
        layer1_row(h, net.W1, 3 * slots + q - 1, f3);
    }
    {
        // the node's own values
        const float o0 = live ? own.u / a.scales[8] : 0.f, o1 = live ? own.w / a.scales[9] : 0.f;
        const float o2 = live ? own.t / a.scales[10] : 0.f, o3 = live ? own.p / a.scales[11] : 0.f;
        x[4 * slots + 0] = o0;
        x[4 * slots + 1] = o1;
        x[4 * slots + 2] = o2;
        x[4 * slots + 3] = o3;
        layer1_row(h, net.W1, 4 * slots + 0, o0);
        layer1_row(h, net.W1, 4 * slots + 1, o1);
        layer1_row(h, net.W1, 4 * slots + 2, o2);
        layer1_row(h, net.W1, 4 * slots + 3, o3);
    }
#pragma unroll
    for (int j = 0; j < kWidth; ++j) {
        h[j] = tanhf(h[j]);
        H1[t * hs + j] = h[j];
    }
    float h2[kWidth];
    layer2(h, net.W2, net.b2, h2);
#pragma unroll
    for (int j = 0; j < kWidth; ++j) H2[t * hs + j] = h2[j];
    float y[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) y[c] = net.b3[c] - y0[c];
#pragma unroll
    for (int m = 0; m < kWidth; ++m)
#pragma unroll
        for (int c = 0; c < 4; ++c) y[c] += h2[m] * bf(net.W3[m * 4 + c]);
    float lsum = 0.f;
    const float inv = 1.f / (4.f * (float)a.B);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float d = 0.f;
        if (live) {
            const float tgt = a.Tg[(k * a.n_prog + i) * 4 + c] / a.scales[4 + c];
            const float r = y[c] - tgt;
            lsum += r * r * inv;
            d = 2.f * r * inv;
        }
        DY[t * 4 + c] = d;
    }
    red[t] = lsum;
    __syncthreads();
    for (int w = kTrainBlock / 2; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    if (t == 0) a.Lp[blockIdx.x] = red[0];
    // the f(0) branch enters y with the opposite sign: its output gradient is
    // dz = -sum dY over the block, propagated back through z2 and z1
    if (t < 4) {
        float acc = 0.f;
        for (int q = 0; q < kTrainBlock; ++q) acc += DY[q * 4 + t];
        dz[t] = -acc;
    }
    __syncthreads();
    if (t < kWidth) {
        float g = 0.f;
        for (int c = 0; c < 4; ++c) g += bf(net.W3[t * 4 + c]) * dz[c];
        dz2[t] = g * (1.f - z2[t] * z2[t]);
    }
    __syncthreads();
    if (t < kWidth) {
        float g = 0.f;
        for (int j = 0; j < kWidth; ++j) g += bf(net.W2[t * kWidth + j]) * dz2[j];
        dz1[t] = g * (1.f - z1[t] * z1[t]);
    }
    __syncthreads();
    // dW3 = H2^T dY + z2 dz^T, db3 = sum dY + dz
    for (int o = t; o < kWidth * 4 + 4; o += kTrainBlock) {
        float acc = 0.f;
        if (o < kWidth * 4) {
            const int m = o >> 2, c = o & 3;
            for (int q = 0; q < kTrainBlock; ++q) acc += H2[q * hs + m] * DY[q * 4 + c];
            gp[m_off.oW3 + o] = acc + z2[m] * dz[c];
        } else {
            const int c = o - kWidth * 4;
            for (int q = 0; q < kTrainBlock; ++q) acc += DY[q * 4 + c];
            gp[m_off.ob3 + c] = acc + dz[c];
        }
    }
    __syncthreads();
    // dH2 = (dY W3^T) o (1 - h2^2), written over this thread's H2 row
#pragma unroll
    for (int m = 0; m < kWidth; ++m) {
        float g = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) g += DY[t * 4 + c] * bf(net.W3[m * 4 + c]);
        H2[t * hs + m] = g * (1.f - h2[m] * h2[m]);
    }
    __syncthreads();
    // dW2 = H1^T dH2 + z1 dz2^T, db2 = sum dH2 + dz2
    for (int o = t; o < kWidth * kWidth + kWidth; o += kTrainBlock) {
        float acc = 0.f;
        if (o < kWidth * kWidth) {
            const int m = o / kWidth, j = o % kWidth;
            for (int q = 0; q < kTrainBlock; ++q) acc += H1[q * hs + m] * H2[q * hs + j];
            gp[m_off.oW2 + o] = acc + z1[m] * dz2[j];
        } else {
            const int j = o - kWidth * kWidth;
            for (int q = 0; q < kTrainBlock; ++q) acc += H2[q * hs + j];
            gp[m_off.ob2 + j] = acc + dz2[j];
        }
    }
    __syncthreads();
    // dH1 = (dH2 W2^T) o (1 - h1^2), written over this thread's H1 row
    for (int m = 0; m < kWidth; ++m) {
        float g = 0.f;
        const __nv_bfloat162 *w = reinterpret_cast<const __nv_bfloat162 *>(net.W2 + m * kWidth);
#pragma unroll
        for (int j = 0; j < kWidth / 2; ++j) {
            const float2 v = __bfloat1622float2(w[j]);
            g += H2[t * hs + 2 * j] * v.x + H2[t * hs + 2 * j + 1] * v.y;
        }
        const float hm = H1[t * hs + m];
        // each thread rewrites only its own row, after every thread has read
        // all rows of H1 in the dW2 product above
        h[m] = g * (1.f - hm * hm);
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kWidth; ++m) H1[t * hs + m] = h[m];
    __syncthreads();
    // dW1 = X^T dH1, db1 = sum dH1
    for (int o = t; o < n_in * kWidth + kWidth; o += kTrainBlock) {
        float acc = 0.f;
        if (o < n_in * kWidth) {
            const int r = o / kWidth, j = o % kWidth;
            for (int q = 0; q < kTrainBlock; ++q) acc += X[q * xs + r] * H1[q * hs + j];
            gp[m_off.oW1 + o] = acc;
        } else {
            const int j = o - n_in * kWidth;
            for (int q = 0; q < kTrainBlock; ++q) acc += H1[q * hs + j];
            gp[m_off.ob1 + j] = acc + dz1[j];
        }
    }
}

// G = sum over the blocks of their gradient partials, and the iteration's
// loss = sum of the blocks' losses, both in block order.
__global__ void mlp_reduce_kernel(const float *Gp, const float *Lp, int nb, int64_t n_params, float *G,
                                  float *loss) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n_params) {
        float g = 0.f;
        for (int b = 0; b < nb; ++b) g += Gp[b * n_params + p];
        G[p] = g;
    }
    if (p == 0) {
        float l = 0.f;
        for (int b = 0; b < nb; ++b) l += Lp[b];
        *loss = l;
    }
}

__global__ void mlp_adam_kernel(float *P, __nv_bfloat16 *Pb, float *G, float *M, float *V, int64_t n, float lr,
                                float b1t, float b2t) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float g = G[p];
    const float m = 0.9f * M[p] + 0.1f * g;
    const float v = 0.999f * V[p] + 0.001f * g * g;
    M[p] = m;
    V[p] = v;
    const float w = P[p] - lr * (m / (1.f - b1t)) / (sqrtf(v / (1.f - b2t)) + 1e-8f);
    P[p] = w;
    Pb[p] = __float2bfloat16_rn(w);
    G[p] = 0.f;
}

__global__ void to_bf16(const float *P, __nv_bfloat16 *Pb, int64_t n) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) Pb[p] = __float2bfloat16_rn(P[p]);
}

// sums for the scales, one row of 12 per warp (the host adds the rows in warp
// order, so the scales do not depend on the warps' timing): [f] squared
// stencil differences of field f, [4+f] squared targets, [8+f] squared own values
__global__ void mlp_scale_sums(const float *S, const float *Tg, int64_t n_states, int64_t n_snap, int64_t n_all,
                               int64_t n_prog, const int32_t *idx, int n, double *acc) {
    double a[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t total = n_states * n_prog;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / n_prog, i = e - k * n_prog;
        const float *Uk = S + state_of(k, n_snap) * n_all * 4;
        const Rec<float> own = load_rec(Uk, i);
        for (int q = 1; q < n; ++q) {
            const Rec<float> r = load_rec(Uk, idx[i * n + q]);
            const float d0 = r.u - own.u, d1 = r.w - own.w, d2 = r.t - own.t, d3 = r.p - own.p;
            a[0] += d0 * d0; a[1] += d1 * d1; a[2] += d2 * d2; a[3] += d3 * d3;
        }
        const float *tg = Tg + e * 4;
        for (int c = 0; c < 4; ++c) a[4 + c] += (double)tg[c] * tg[c];
        a[8] += (double)own.u * own.u; a[9] += (double)own.w * own.w;
        a[10] += (double)own.t * own.t; a[11] += (double)own.p * own.p;
    }
    for (int c = 0; c < 12; ++c) {
        double v = a[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) acc[((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 12 + c] = v;
    }
}

template <class S_, class D_>
__global__ void restrict_kernel(const S_ *src, const int64_t *map, int64_t n_map, D_ *dst, int64_t block_records,
                                int64_t block_stride) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_map) return;
    const int64_t r = e / block_records, loc = e - r * block_records;
    const int64_t s = map[e], d = r * block_stride + loc;
#pragma unroll
    for (int c = 0; c < 4; ++c) dst[d * 4 + c] = (D_)src[s * 4 + c];
}

// dst record of entry e = sum_q w[e][q] src[idx[e][q]] (weighted restriction)
template <class S_>
__global__ void restrict_avg_kernel(const S_ *src, const int64_t *idx, const double *w, int m, int64_t n_map,
                                    float *dst, int64_t block_records, int64_t block_stride) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_map) return;
    double a[4] = {0, 0, 0, 0};
    for (int q = 0; q < m; ++q) {
        const double wq = w[e * m + q];
        const int64_t s = idx[e * m + q];
#pragma unroll
        for (int c = 0; c < 4; ++c) a[c] += wq * (double)src[s * 4 + c];
    }
    const int64_t r = e / block_records, loc = e - r * block_records;
    const int64_t d = r * block_stride + loc;
#pragma unroll
    for (int c = 0; c < 4; ++c) dst[d * 4 + c] = (float)a[c];
}

// targets = (next - step(this)) / dt on prognostic records
__global__ void target_kernel(const float *next, const float *stepped, float *tg, int64_t n_prog, float inv_dt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n_prog * 4) tg[e] = (next[e] - stepped[e]) * inv_dt;
}

size_t train_smem(int n_in) {
    return ((net_bytes(n_in) + 15) & ~size_t(15)) + (size_t)kTrainBlock * ((n_in + 1) + 2 * (kWidth + 1) + 4) * 4;
}

void mlp_launch_infer(Mlp &m, Problem &pb, const void *U, void *delta, cudaStream_t s) {
    const size_t smem = net_bytes(m.n_in);
    const dim3 grid(div_up(pb.n_prog, 128)), blk(128);
    if (pb.precision == 64)
        mlp_infer_kernel<double><<<grid, blk, smem, s>>>((const double *)U, pb.idx.p, m.n, pb.n_prog, m.Pb.p, m.P.p, offs_of(m),
                                                         m.scales.p, pb.flags.p, (double *)delta);
    else
        mlp_infer_kernel<float><<<grid, blk, smem, s>>>((const float *)U, pb.idx.p, m.n, pb.n_prog, m.Pb.p, m.P.p, offs_of(m),
                                                        m.scales.p, pb.flags.p, (float *)delta);
    RBF_CHECK_LAUNCH();
}

void mlp_launch_train(Mlp &m, Problem &pb, const float *S, const float *Tg, int64_t n_runs, int64_t n_snap,
                      const int64_t *samples, int B, unsigned long long seed, long long iter, float *loss) {
    TrainArgs a{};
    a.S = S;
    a.Tg = Tg;
    a.n_states = n_runs * (n_snap - 1);
    a.n_snap = n_snap;
    a.n_all = pb.n_all;
    a.n_prog = pb.n_prog;
    a.idx = pb.idx.p;
    a.n = m.n;
    a.samples = samples;
    a.seed = seed;
    a.iter = iter;
    a.B = B;
    a.Pb = m.Pb.p;
    a.P = m.P.p;
    a.scales = m.scales.p;
    const int nb = div_up(B, kTrainBlock);
    if (m.Gp.n < (size_t)nb * m.n_params) m.Gp.alloc((size_t)nb * m.n_params);
    if (m.Lp.n < (size_t)nb) m.Lp.alloc(nb);
    a.Gp = m.Gp.p;
    a.n_params = m.n_params;
    a.Lp = m.Lp.p;
    mlp_train_kernel<<<nb, kTrainBlock, train_smem(m.n_in), m.st>>>(a, offs_of(m));
    RBF_CHECK_LAUNCH();
    mlp_reduce_kernel<<<div_up(m.n_params, 256), 256, 0, m.st>>>(m.Gp.p, m.Lp.p, nb, m.n_params, m.Gr.p, loss);
    RBF_CHECK_LAUNCH();
}

}  // namespace

void mlp_init(Mlp &m, Problem &pb, void *stream) {
    RBF_REQUIRE(pb.kind == kNS, "the learned correction needs a Navier-Stokes problem");
    RBF_REQUIRE(pb.idx.p != nullptr, "the coarse problem's stencils were released");
    m.st = as_stream(stream);
    m.n = pb.n;
    m.slots = pb.n - 1;
    m.n_in = 4 * m.slots + 4;
    RBF_REQUIRE(train_smem(m.n_in) <= 227 * 1024, "stencil of %d nodes too large for the training kernel", pb.n);
    m.oW1 = 0;
    m.ob1 = m.oW1 + (int64_t)m.n_in * kWidth;
    m.oW2 = m.ob1 + kWidth;
    m.ob2 = m.oW2 + kWidth * kWidth;
    m.oW3 = m.ob2 + kWidth;
    m.ob3 = m.oW3 + kWidth * 4;
    m.n_params = m.ob3 + 4;
    m.P.alloc(m.n_params);
    m.Gr.alloc(m.n_params);
    m.M.alloc(m.n_params);
    m.V.alloc(m.n_params);
    m.Pb.alloc(m.n_params);
    m.scales.alloc(12);
    m.acc.alloc(12 * kScaleWarps);
    m.bad.alloc(1);
    RBF_CUDA(cudaMemsetAsync(m.P.p, 0, m.P.bytes(), m.st));
    RBF_CUDA(cudaMemsetAsync(m.Gr.p, 0, m.Gr.bytes(), m.st));
    RBF_CUDA(cudaMemsetAsync(m.M.p, 0, m.M.bytes(), m.st));
    RBF_CUDA(cudaMemsetAsync(m.V.p, 0, m.V.bytes(), m.st));
    const float ones[12] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
    RBF_CUDA(cudaMemcpyAsync(m.scales.p, ones, sizeof(ones), cudaMemcpyHostToDevice, m.st));
    RBF_CUDA(cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)train_smem(m.n_in)));
    RBF_CUDA(cudaStreamSynchronize(m.st));
}

}  // namespace rbf

struct rbf_mlp {
    rbf::Mlp impl;
    rbf_problem *coarse = nullptr;
};

using rbf::Mlp;

extern "C" {

int rbf_mlp_create(rbf_mlp **out, rbf_problem *coarse, void *stream) {
    return rbf::guarded([&] {
        RBF_REQUIRE(out && coarse, "null argument");
        *out = nullptr;
        auto *h = new rbf_mlp();
        try {
            h->coarse = coarse;
            rbf::mlp_init(h->impl, coarse->impl, stream);
            *out = h;
        } catch (...) {
            delete h;
            throw;
        }
    });
}

int rbf_mlp_n_params(const rbf_mlp *h, int64_t *out) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && out, "null argument");
        *out = h->impl.n_params;
    });
}

int rbf_mlp_set_params(rbf_mlp *h, const float *params) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && params, "null argument");
        Mlp &m = h->impl;
        RBF_CUDA(cudaMemcpyAsync(m.P.p, params, m.P.bytes(), cudaMemcpyHostToDevice, m.st));
        rbf::to_bf16<<<rbf::div_up(m.n_params, 256), 256, 0, m.st>>>(m.P.p, m.Pb.p, m.n_params);
        RBF_CHECK_LAUNCH();
        RBF_CUDA(cudaMemsetAsync(m.M.p, 0, m.M.bytes(), m.st));
        RBF_CUDA(cudaMemsetAsync(m.V.p, 0, m.V.bytes(), m.st));
        RBF_CUDA(cudaMemsetAsync(m.Gr.p, 0, m.Gr.bytes(), m.st));
        m.t = 0;
        RBF_CUDA(cudaStreamSynchronize(m.st));
    });
}

int rbf_mlp_get_params(const rbf_mlp *h, float *params) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && params, "null argument");
        const Mlp &m = h->impl;
        RBF_CUDA(cudaStreamSynchronize(m.st));
        RBF_CUDA(cudaMemcpy(params, m.P.p, m.P.bytes(), cudaMemcpyDeviceToHost));
    });
}

int rbf_mlp_set_scales(rbf_mlp *h, const float *scales) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && scales, "null argument");
        for (int c = 0; c < 12; ++c) RBF_REQUIRE(scales[c] > 0.f && std::isfinite(scales[c]), "scales must be > 0");
        RBF_CUDA(cudaMemcpyAsync(h->impl.scales.p, scales, 12 * sizeof(float), cudaMemcpyHostToDevice, h->impl.st));
        RBF_CUDA(cudaStreamSynchronize(h->impl.st));
    });
}

int rbf_mlp_get_scales(const rbf_mlp *h, float *scales) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && scales, "null argument");
        RBF_CUDA(cudaStreamSynchronize(h->impl.st));
        RBF_CUDA(cudaMemcpy(scales, h->impl.scales.p, 12 * sizeof(float), cudaMemcpyDeviceToHost));
    });
}

int rbf_mlp_fit_scales(rbf_mlp *h, const float *states, const float *targets, int64_t n_runs, int64_t n_snap) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && states && targets && n_runs > 0 && n_snap >= 2, "bad argument");
        const int64_t n_states = n_runs * (n_snap - 1);
        Mlp &m = h->impl;
        rbf::Problem &pb = h->coarse->impl;
        rbf::mlp_scale_sums<<<rbf::kScaleWarps / 8, 256, 0, m.st>>>(states, targets, n_states, n_snap, pb.n_all,
                                                                   pb.n_prog, pb.idx.p, m.n, m.acc.p);
        RBF_CHECK_LAUNCH();
        std::vector<double> rows(12 * rbf::kScaleWarps);
        RBF_CUDA(cudaMemcpyAsync(rows.data(), m.acc.p, rows.size() * sizeof(double), cudaMemcpyDeviceToHost, m.st));
        RBF_CUDA(cudaStreamSynchronize(m.st));
        double s[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < rbf::kScaleWarps; ++w)
            for (int c = 0; c < 12; ++c) s[c] += rows[(size_t)w * 12 + c];
        float sc[12];
        const double cnt_in = (double)n_states * pb.n_prog * (m.n - 1), cnt_out = (double)n_states * pb.n_prog;
        for (int c = 0; c < 4; ++c) {
            sc[c] = (float)std::sqrt(std::max(s[c] / cnt_in, 1e-30));
            sc[4 + c] = (float)std::sqrt(std::max(s[4 + c] / cnt_out, 1e-30));
            sc[8 + c] = (float)std::sqrt(std::max(s[8 + c] / cnt_out, 1e-30));
        }
        RBF_CUDA(cudaMemcpyAsync(m.scales.p, sc, sizeof(sc), cudaMemcpyHostToDevice, m.st));
        RBF_CUDA(cudaStreamSynchronize(m.st));
    });
}

int rbf_mlp_grad(rbf_mlp *h, const float *states, const float *targets, int64_t n_runs, int64_t n_snap,
                 const int64_t *samples, int32_t batch, float *grad_host, float *loss_host) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && states && targets && samples && batch > 0 && n_runs > 0 && n_snap >= 2, "bad argument");
        Mlp &m = h->impl;
        rbf::DevBuf<float> loss(1);
        RBF_CUDA(cudaMemsetAsync(loss.p, 0, sizeof(float), m.st));
        RBF_CUDA(cudaMemsetAsync(m.Gr.p, 0, m.Gr.bytes(), m.st));
        rbf::mlp_launch_train(m, h->coarse->impl, states, targets, n_runs, n_snap, samples, batch, 0, 0, loss.p);
        if (grad_host) RBF_CUDA(cudaMemcpyAsync(grad_host, m.Gr.p, m.Gr.bytes(), cudaMemcpyDeviceToHost, m.st));
        if (loss_host) RBF_CUDA(cudaMemcpyAsync(loss_host, loss.p, sizeof(float), cudaMemcpyDeviceToHost, m.st));
        RBF_CUDA(cudaMemsetAsync(m.Gr.p, 0, m.Gr.bytes(), m.st));
        RBF_CUDA(cudaStreamSynchronize(m.st));
    });
}

int rbf_mlp_train(rbf_mlp *h, const float *states, const float *targets, int64_t n_runs, int64_t n_snap,
                  int64_t iters, int32_t batch, float lr, uint64_t seed, float *loss_host) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && states && targets && n_runs > 0 && n_snap >= 2 && iters >= 0 && batch > 0, "bad argument");
        RBF_REQUIRE(lr > 0.f && std::isfinite(lr), "lr must be > 0");
        Mlp &m = h->impl;
        m.loss.alloc(std::max<int64_t>(iters, 1));
        RBF_CUDA(cudaMemsetAsync(m.loss.p, 0, m.loss.bytes(), m.st));
        for (int64_t it = 0; it < iters; ++it) {
            rbf::mlp_launch_train(m, h->coarse->impl, states, targets, n_runs, n_snap, nullptr, batch, seed, it,
                                  m.loss.p + it);
            m.t += 1;
            // cosine decay of the step size over the run
            const float lr_t = lr * 0.5f * (1.f + std::cos(3.14159265358979f * (float)it / (float)iters));
            rbf::mlp_adam_kernel<<<rbf::div_up(m.n_params, 256), 256, 0, m.st>>>(
                m.P.p, m.Pb.p, m.Gr.p, m.M.p, m.V.p, m.n_params, lr_t, std::pow(0.9f, (float)m.t),
                std::pow(0.999f, (float)m.t));
            RBF_CHECK_LAUNCH();
        }
        if (loss_host) RBF_CUDA(cudaMemcpyAsync(loss_host, m.loss.p, iters * sizeof(float), cudaMemcpyDeviceToHost, m.st));
        RBF_CUDA(cudaStreamSynchronize(m.st));
    });
}

int rbf_mlp_forward(rbf_mlp *h, const void *U, void *delta) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && U && delta, "null argument");
        rbf::mlp_launch_infer(h->impl, h->coarse->impl, U, delta, h->impl.st);
    });
}

// The network as the persistent kernel reads it, with strengths alpha.
static rbf::MlpView mlp_view(Mlp &m, const double *alpha) {
    rbf::MlpView mv{};
    mv.Pb = m.Pb.p;
    mv.P = m.P.p;
    mv.oW1 = m.oW1; mv.ob1 = m.ob1; mv.oW2 = m.oW2; mv.ob2 = m.ob2; mv.oW3 = m.oW3; mv.ob3 = m.ob3;
    mv.scales = m.scales.p;
    for (int f = 0; f < 4; ++f) mv.alpha[f] = (float)alpha[f];
    mv.n_in = m.n_in;
    mv.bad = m.bad.p;
    return mv;
}

int rbf_mlp_tune_run(rbf_mlp *h) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h, "null argument");
        Mlp &m = h->impl;
        rbf::Problem &pb = h->coarse->impl;
        RBF_CUDA(cudaStreamSynchronize(pb.st));
        RBF_CUDA(cudaStreamSynchronize(pb.cap));
        const double ones[4] = {1.0, 1.0, 1.0, 1.0};
        RBF_REQUIRE(rbf::persistent_tune_mlp(pb, mlp_view(m, ones)),
                    "no persistent kernel with the network fits this problem");
    });
}

int rbf_learned_run(rbf_mlp *h, double t0, double dt, int64_t n_steps, const double *alpha, void *U,
                    int64_t *n_fallback) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && U && alpha && n_steps >= 0, "bad argument");
        RBF_REQUIRE((reinterpret_cast<uintptr_t>(U) & 15) == 0, "state must be 16-byte aligned (node-major records)");
        for (int f = 0; f < 4; ++f) RBF_REQUIRE(alpha[f] >= 0.0 && std::isfinite(alpha[f]), "alpha must be >= 0");
        const float4 al = make_float4((float)alpha[0], (float)alpha[1], (float)alpha[2], (float)alpha[3]);
        Mlp &m = h->impl;
        rbf::Problem &pb = h->coarse->impl;
        RBF_CUDA(cudaMemsetAsync(m.bad.p, 0, sizeof(unsigned long long), pb.st));
        if (pb.run_mode == RBF_RUN_PERSISTENT && rbf::persistent_mlp_ready(pb)) {
            // the whole corrected run in one persistent launch (network evaluated
            // at stage 0 of every step from the records in shared memory)
            const rbf::MlpView mv = mlp_view(m, alpha);
            rbf::persistent_run_mlp(pb, dt, n_steps, U, pb.st, mv);
            unsigned long long bad = 0;
            RBF_CUDA(cudaMemcpyAsync(&bad, m.bad.p, sizeof(bad), cudaMemcpyDeviceToHost, pb.st));
            RBF_CUDA(cudaStreamSynchronize(pb.st));
            rbf::persistent_check(pb);
            if (n_fallback) *n_fallback = (int64_t)bad;
            return;
        }
        rbf::DevBuf<unsigned char> delta((size_t)pb.n_prog * 4 * pb.tsize());
        for (int64_t s = 0; s < n_steps; ++s) {
            // features need the ghosts of the current state; then step and add dt * delta
            rbf::enqueue_ghost_fill(pb, U, pb.st);
            rbf::mlp_launch_infer(m, pb, U, delta.p, pb.st);
            rbf::enqueue_rk4_step(pb, t0 + s * dt, dt, U, pb.st, false, 0);
            if (pb.precision == 64)
                rbf::mlp_apply_kernel<double><<<rbf::div_up(pb.n_prog * 4, 256), 256, 0, pb.st>>>(
                    (double *)U, (const double *)delta.p, pb.n_prog, dt, al, m.bad.p);
            else
                rbf::mlp_apply_kernel<float><<<rbf::div_up(pb.n_prog * 4, 256), 256, 0, pb.st>>>(
                    (float *)U, (const float *)delta.p, pb.n_prog, (float)dt, al, m.bad.p);
            RBF_CHECK_LAUNCH();
        }
        unsigned long long bad = 0;
        RBF_CUDA(cudaMemcpyAsync(&bad, m.bad.p, sizeof(bad), cudaMemcpyDeviceToHost, pb.st));
        RBF_CUDA(cudaStreamSynchronize(pb.st));
        if (n_fallback) *n_fallback = (int64_t)bad;
    });
}

int rbf_mlp_destroy(rbf_mlp *h) {
    return rbf::guarded([&] {
        if (!h) return;
        cudaStreamSynchronize(h->impl.st);
        delete h;
    });
}

int rbf_restrict(const void *src, int32_t src_precision, const int64_t *map, int64_t n_map, void *dst,
                 int32_t dst_precision, int64_t block_records, int64_t block_stride, void *stream) {
    return rbf::guarded([&] {
        RBF_REQUIRE(src && map && dst && n_map >= 0 && block_records > 0 && block_stride >= block_records,
                    "bad argument");
        RBF_REQUIRE((src_precision == 32 || src_precision == 64) && (dst_precision == 32 || dst_precision == 64),
                    "precision must be 32 or 64");
        if (n_map == 0) return;
        cudaStream_t s = rbf::as_stream(stream);
        const int grid = rbf::div_up(n_map, 256);
        if (src_precision == 64 && dst_precision == 32)
            rbf::restrict_kernel<double, float><<<grid, 256, 0, s>>>((const double *)src, map, n_map, (float *)dst,
                                                                     block_records, block_stride);
        else if (src_precision == 64)
            rbf::restrict_kernel<double, double><<<grid, 256, 0, s>>>((const double *)src, map, n_map, (double *)dst,
                                                                      block_records, block_stride);
        else if (dst_precision == 32)
            rbf::restrict_kernel<float, float><<<grid, 256, 0, s>>>((const float *)src, map, n_map, (float *)dst,
                                                                    block_records, block_stride);
        else
            rbf::restrict_kernel<float, double><<<grid, 256, 0, s>>>((const float *)src, map, n_map, (double *)dst,
                                                                     block_records, block_stride);
        RBF_CHECK_LAUNCH();
    });
}

int rbf_restrict_weighted(const void *src, int32_t src_precision, const int64_t *idx, const double *w, int32_t m,
                          int64_t n_map, float *dst, int64_t block_records, int64_t block_stride, void *stream) {
    return rbf::guarded([&] {
        RBF_REQUIRE(src && idx && w && dst && m >= 1 && n_map >= 0 && block_records > 0 &&
                        block_stride >= block_records, "bad argument");
        RBF_REQUIRE(src_precision == 32 || src_precision == 64, "precision must be 32 or 64");
        if (n_map == 0) return;
        cudaStream_t s = rbf::as_stream(stream);
        const int grid = rbf::div_up(n_map, 256);
        if (src_precision == 64)
            rbf::restrict_avg_kernel<double><<<grid, 256, 0, s>>>((const double *)src, idx, w, m, n_map, dst,
                                                                  block_records, block_stride);
        else
            rbf::restrict_avg_kernel<float><<<grid, 256, 0, s>>>((const float *)src, idx, w, m, n_map, dst,
                                                                 block_records, block_stride);
        RBF_CHECK_LAUNCH();
    });
}

int rbf_fill_ghosts(rbf_problem *h, void *U) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && U && h->impl.kind == rbf::kNS, "needs a Navier-Stokes problem and a state");
        RBF_REQUIRE((reinterpret_cast<uintptr_t>(U) & 15) == 0, "state must be 16-byte aligned (node-major records)");
        rbf::enqueue_ghost_fill(h->impl, U, h->impl.st);
    });
}

int rbf_mlp_targets(rbf_problem *h, const float *states, int64_t n_runs, int64_t n_snap, double dt, float *targets) {
    return rbf::guarded([&] {
        RBF_REQUIRE(h && states && targets && n_runs > 0 && n_snap >= 2, "bad argument");
        rbf::Problem &pb = h->impl;
        RBF_REQUIRE(pb.kind == rbf::kNS && pb.precision == 32, "targets need an FP32 Navier-Stokes problem");
        const int64_t rec = pb.n_all * 4;
        rbf::DevBuf<float> tmp(rec);
        for (int64_t r = 0; r < n_runs; ++r)
            for (int64_t k = 0; k + 1 < n_snap; ++k) {
                const float *cur = states + (r * n_snap + k) * rec;
                RBF_CUDA(cudaMemcpyAsync(tmp.p, cur, rec * 4, cudaMemcpyDeviceToDevice, pb.st));
                rbf::enqueue_rk4_step(pb, 0.0, dt, tmp.p, pb.st, false, 0);
                rbf::target_kernel<<<rbf::div_up(pb.n_prog * 4, 256), 256, 0, pb.st>>>(
                    cur + rec, tmp.p, targets + (r * (n_snap - 1) + k) * pb.n_prog * 4, pb.n_prog, (float)(1.0 / dt));
                RBF_CHECK_LAUNCH();
            }
        RBF_CUDA(cudaStreamSynchronize(pb.st));
    });
}

}  // extern "C"
