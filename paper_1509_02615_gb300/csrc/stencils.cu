// a1: stencil selection -- the n nearest nodes of every centre (Sec. 6 uses
// n = 37, complete rings on Cartesian and hexagonal lattices, Appendix A).
//
// GPU design: nodes are binned into a uniform grid (about two nodes per cell,
// counting sort by cell).  One warp serves one centre: it gathers every node
// in a (2R+1)^2 window of cells into shared memory, ranks the candidates by
// (squared distance, node index) and keeps the first n.  The window is
// accepted only when the n-th distance is strictly inside the radius that
// the window is guaranteed to cover; otherwise R grows.  The result equals a
// brute-force sort over all nodes.
#include <cfloat>
#include <cmath>

#include "common.cuh"

namespace rbf {

namespace {

constexpr int kMaxCand = 2048;   // candidates per window held in shared memory
constexpr int kWarpsPerBlock = 4;

struct Grid {
    double x0, z0, cw, ch;   // origin and cell size
    int ncx, ncz;
    double period;           // > 0: periodic in x
};

__global__ void bbox_kernel(const double *x, const double *z, int64_t n, double *out, int *bad) {
    // out: [xmin, xmax, zmin, zmax] reduced with atomics on the ordered-int image
    __shared__ double s[4][256];
    double v[4] = {DBL_MAX, -DBL_MAX, DBL_MAX, -DBL_MAX};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double a = x[i], b = z[i];
        if (!isfinite(a) || !isfinite(b)) atomicExch(bad, 1);
        v[0] = fmin(v[0], a); v[1] = fmax(v[1], a);
        v[2] = fmin(v[2], b); v[3] = fmax(v[3], b);
    }
    for (int k = 0; k < 4; ++k) s[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s[0][threadIdx.x] = fmin(s[0][threadIdx.x], s[0][threadIdx.x + w]);
            s[1][threadIdx.x] = fmax(s[1][threadIdx.x], s[1][threadIdx.x + w]);
            s[2][threadIdx.x] = fmin(s[2][threadIdx.x], s[2][threadIdx.x + w]);
            s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x * 4 + 0] = s[0][0], out[blockIdx.x * 4 + 1] = s[1][0],
                          out[blockIdx.x * 4 + 2] = s[2][0], out[blockIdx.x * 4 + 3] = s[3][0];
}

__device__ __forceinline__ int cell_x(const Grid &g, double x) {
    int c = (int)floor((x - g.x0) / g.cw);
    if (g.period > 0.0) {
        c %= g.ncx;
        if (c < 0) c += g.ncx;
    } else {
        c = min(max(c, 0), g.ncx - 1);
    }
    return c;
}
__device__ __forceinline__ int cell_z(const Grid &g, double z) {
    int c = (int)floor((z - g.z0) / g.ch);
    return min(max(c, 0), g.ncz - 1);
}

__global__ void count_kernel(const double *x, const double *z, int64_t n, Grid g, int *cell, int *count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cell_z(g, z[i]) * g.ncx + cell_x(g, x[i]);
    cell[i] = c;
    atomicAdd(&count[c], 1);
}

// Exclusive scan of count[0..m) into start[0..m] by one block of 1024 threads.
__global__ void scan_kernel(const int *count, int m, int *start) {
    __shared__ int part[1024];
    int t = threadIdx.x;
    int chunk = (m + blockDim.x - 1) / blockDim.x;
    int b = t * chunk, e = min(b + chunk, m);
    int s = 0;
    for (int i = b; i < e; ++i) s += count[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < blockDim.x; off <<= 1) {
        int v = (t >= off) ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;
    for (int i = b; i < e; ++i) {
        start[i] = run;
        run += count[i];
    }
    if (t == blockDim.x - 1) start[m] = part[t];
}

__global__ void scatter_kernel(const int *cell, int64_t n, const int *start, int *cursor, int *sorted) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cell[i];
    int pos = start[c] + atomicAdd(&cursor[c], 1);
    sorted[pos] = (int)i;
}

// Squared distance as the oracle defines it: minimum image in x, then
// dx*dx + dz*dz with each operation rounded (no contraction into FMA).
__device__ __forceinline__ double sqdist(double xc, double zc, double xj, double zj, double period) {
    double dx = __dsub_rn(xj, xc);
    if (period > 0.0) {
        double half = 0.5 * period;
        if (dx > half) dx = __dsub_rn(dx, period);
        else if (dx < -half) dx = __dadd_rn(dx, period);
    }
    double dz = __dsub_rn(zj, zc);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dz, dz));
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
knn_kernel(const double *__restrict__ x, const double *__restrict__ z, int64_t n_centers, int n, Grid g,
           const int *__restrict__ start, const int *__restrict__ sorted, int R0, int Rmax,
           int32_t *__restrict__ idx, int *__restrict__ status) {
    extern __shared__ unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *cd2 = reinterpret_cast<double *>(smem) + warp * kMaxCand;
    int *cid = reinterpret_cast<int *>(reinterpret_cast<double *>(smem) + kWarpsPerBlock * kMaxCand) + warp * kMaxCand;
    __shared__ double nth_d2[kWarpsPerBlock];

    const int64_t c = blockIdx.x * (int64_t)kWarpsPerBlock + warp;
    if (c >= n_centers) return;
    const double xc = x[c], zc = z[c];
    const int cx = cell_x(g, xc), cz = cell_z(g, zc);

    for (int R = R0; R <= Rmax; ++R) {
        // x columns of the window (all columns once if the window wraps onto itself)
        bool all_x = (2 * R + 1 >= g.ncx);
        int xa = all_x ? 0 : cx - R, xb = all_x ? g.ncx - 1 : cx + R;
        int za = max(cz - R, 0), zb = min(cz + R, g.ncz - 1);
        bool all_z = (cz - R <= 0) && (cz + R >= g.ncz - 1);
        if (g.period <= 0.0) {
            all_x = all_x || ((cx - R <= 0) && (cx + R >= g.ncx - 1));
            xa = max(xa, 0);
            xb = min(xb, g.ncx - 1);
        }
        int m = 0;
        bool overflow = false;
        for (int rz = za; rz <= zb && !overflow; ++rz) {
            // up to two contiguous column ranges (wrap-around in periodic x)
            int ranges[2][2];
            int nr = 0;
            if (g.period > 0.0 && !all_x) {
                int a = xa, b = xb;
                if (a < 0) { ranges[nr][0] = a + g.ncx; ranges[nr][1] = g.ncx - 1; ++nr; a = 0; }
                if (b >= g.ncx) { ranges[nr][0] = 0; ranges[nr][1] = b - g.ncx; ++nr; b = g.ncx - 1; }
                ranges[nr][0] = a; ranges[nr][1] = b; ++nr;
            } else {
                ranges[0][0] = xa; ranges[0][1] = xb; nr = 1;
            }
            for (int q = 0; q < nr; ++q) {
                int p0 = start[rz * g.ncx + ranges[q][0]];
                int p1 = start[rz * g.ncx + ranges[q][1] + 1];
                for (int base = p0; base < p1; base += 32) {
                    int p = base + lane;
                    bool has = p < p1;
                    unsigned mask = __ballot_sync(0xffffffffu, has);
                    int pos = m + __popc(mask & ((1u << lane) - 1u));
                    int cnt = __popc(mask);
                    if (m + cnt > kMaxCand) { overflow = true; break; }
                    if (has) {
                        int j = sorted[p];
                        cd2[pos] = sqdist(xc, zc, x[j], z[j], g.period);
                        cid[pos] = j;
                    }
                    m += cnt;
                }
                if (overflow) break;
            }
        }
        if (overflow) {
            if (lane == 0) atomicCAS(status, 0, 2);
            return;
        }
        __syncwarp();
        if (m < n) continue;
        // rank every candidate by (d2, index); ranks are a permutation
        for (int i = lane; i < m; i += 32) {
            double di = cd2[i];
            int ii = cid[i];
            int rank = 0;
            for (int j = 0; j < m; ++j) {
                double dj = cd2[j];
                rank += (dj < di) || (dj == di && cid[j] < ii);
            }
            if (rank < n) idx[c * n + rank] = ii;
            if (rank == n - 1) nth_d2[warp] = di;
        }
        __syncwarp();
        double guard = DBL_MAX;
        if (!all_x) guard = fmin(guard, R * g.cw);
        if (!all_z) guard = fmin(guard, R * g.ch);
        guard *= (1.0 - 1e-9);
        if (nth_d2[warp] < guard * guard) return;   // the window provably holds the n nearest
        __syncwarp();
    }
    if (lane == 0) atomicCAS(status, 0, 3);
}

}  // namespace

void build_stencils(const double *x, const double *z, int64_t n_all, int64_t n_centers, int n,
                    double period_x, int32_t *idx, cudaStream_t st) {
    RBF_REQUIRE(n >= 1 && n <= 128, "stencil size n=%d must be in [1, 128]", n);
    RBF_REQUIRE(n_all >= n, "n_all=%lld smaller than the stencil size %d", (long long)n_all, n);
    RBF_REQUIRE(n_centers >= 0 && n_centers <= n_all, "n_centers=%lld out of range", (long long)n_centers);
    RBF_REQUIRE(n_all < (int64_t)1 << 31, "n_all=%lld exceeds int32 indexing", (long long)n_all);
    RBF_REQUIRE(period_x >= 0.0 && std::isfinite(period_x), "period_x must be finite and >= 0");
    if (n_centers == 0) return;
    RBF_REQUIRE(x && z && idx, "null pointer argument");

    const int nb = 64;
    DevBuf<double> part(nb * 4);
    DevBuf<int> bad(1);
    RBF_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    bbox_kernel<<<nb, 256, 0, st>>>(x, z, n_all, part.p, bad.p);
    RBF_CHECK_LAUNCH();
    std::vector<double> hp(nb * 4);
    int hbad = 0;
    RBF_CUDA(cudaMemcpyAsync(hp.data(), part.p, part.bytes(), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaStreamSynchronize(st));
    RBF_REQUIRE(!hbad, "non-finite node coordinates");
    double xmin = DBL_MAX, xmax = -DBL_MAX, zmin = DBL_MAX, zmax = -DBL_MAX;
    for (int b = 0; b < nb; ++b) {
        xmin = std::fmin(xmin, hp[b * 4 + 0]); xmax = std::fmax(xmax, hp[b * 4 + 1]);
        zmin = std::fmin(zmin, hp[b * 4 + 2]); zmax = std::fmax(zmax, hp[b * 4 + 3]);
    }
    Grid g;
    g.period = period_x;
    double W = period_x > 0.0 ? period_x : (xmax - xmin);
    double H = zmax - zmin;
    double area = std::fmax(W, 1e-300) * std::fmax(H, 1e-300);
    if (W <= 0.0 || H <= 0.0) area = std::fmax(W, H) * std::fmax(W, H) / (double)n_all;
    double cell = std::sqrt(2.0 * area / (double)n_all);
    if (!(cell > 0.0)) cell = 1.0;
    g.x0 = xmin;
    g.z0 = zmin;
    g.ncx = (int)std::fmax(1.0, std::fmin(std::floor(W / cell), 1e6));
    g.ncz = (int)std::fmax(1.0, std::fmin(std::ceil(H / cell), 1e6));
    if (period_x <= 0.0 && W / g.ncx > 0) g.ncx = (int)std::fmax(1.0, std::ceil(W / cell));
    g.cw = W > 0.0 ? W / g.ncx : cell;
    g.ch = H > 0.0 ? H / g.ncz : cell;
    int64_t ncell = (int64_t)g.ncx * g.ncz;
    RBF_REQUIRE(ncell < ((int64_t)1 << 30), "binning grid too large");

    DevBuf<int> cellof(n_all), count(ncell), start(ncell + 1), cursor(ncell), sorted(n_all);
    DevBuf<int> status(1);
    RBF_CUDA(cudaMemsetAsync(count.p, 0, count.bytes(), st));
    RBF_CUDA(cudaMemsetAsync(cursor.p, 0, cursor.bytes(), st));
    RBF_CUDA(cudaMemsetAsync(status.p, 0, sizeof(int), st));
    count_kernel<<<div_up(n_all, 256), 256, 0, st>>>(x, z, n_all, g, cellof.p, count.p);
    RBF_CHECK_LAUNCH();
    scan_kernel<<<1, 1024, 0, st>>>(count.p, (int)ncell, start.p);
    RBF_CHECK_LAUNCH();
    scatter_kernel<<<div_up(n_all, 256), 256, 0, st>>>(cellof.p, n_all, start.p, cursor.p, sorted.p);
    RBF_CHECK_LAUNCH();

    // first window: about 2.5 n candidates at two nodes per cell
    int R0 = (int)std::ceil(std::sqrt(2.5 * n / (4.0 * 2.0)));
    R0 = R0 < 1 ? 1 : R0;
    int Rmax = std::max(g.ncx, g.ncz);
    size_t smem = (size_t)kWarpsPerBlock * kMaxCand * (sizeof(double) + sizeof(int));
    RBF_CUDA(cudaFuncSetAttribute(knn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    knn_kernel<<<div_up(n_centers, kWarpsPerBlock), kWarpsPerBlock * 32, smem, st>>>(
        x, z, n_centers, n, g, start.p, sorted.p, R0, Rmax, idx, status.p);
    RBF_CHECK_LAUNCH();
    int hs = 0;
    RBF_CUDA(cudaMemcpyAsync(&hs, status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaStreamSynchronize(st));
    RBF_REQUIRE(hs == 0, "stencil search failed (%s)",
                hs == 2 ? "more than 2048 candidates in a search window: node density too uneven"
                        : "no window holds n nodes");
}

// ---- allocation-free variant (rbf_build_stencils_static) --------------------
// The same kernels as rbf_build_stencils, with every scratch buffer carved out
// of one file-scope device array instead of cudaMalloc.  The array lives on
// every GPU that loads this library until the process exits.
namespace {

constexpr int64_t kStaticMaxNodes = 262144;   // n_all limit of the static variant
constexpr int64_t kStaticMaxCells = 262144;   // binning cells limit
constexpr int kBboxBlocks = 64;

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffPart = 0;
constexpr size_t kOffBad = kOffPart + align256(kBboxBlocks * 4 * sizeof(double));
constexpr size_t kOffStatus = kOffBad + 256;
constexpr size_t kOffCellOf = kOffStatus + 256;
constexpr size_t kOffSorted = kOffCellOf + align256(kStaticMaxNodes * sizeof(int));
constexpr size_t kOffCount = kOffSorted + align256(kStaticMaxNodes * sizeof(int));
constexpr size_t kOffCursor = kOffCount + align256(kStaticMaxCells * sizeof(int));
constexpr size_t kOffStart = kOffCursor + align256(kStaticMaxCells * sizeof(int));
constexpr size_t kStaticScratchBytes = kOffStart + align256((kStaticMaxCells + 1) * sizeof(int));  // ~5 MB

static __device__ __align__(256) unsigned char g_stencil_scratch[kStaticScratchBytes];

// Device address of the scratch array on the current device.  In host code
// the symbol is only a stand-in, so the address is looked up with the device
// current -- on every call, not cached: after a device reset or in a new
// context the module is loaded again and the array moves.  The lookup is
// cheap next to the call's own two stream synchronisations.
unsigned char *static_scratch() {
    void *ptr = nullptr;
    RBF_CUDA(cudaGetSymbolAddress(&ptr, g_stencil_scratch));
    return static_cast<unsigned char *>(ptr);
}

}  // namespace

void build_stencils_static(const double *x, const double *z, int64_t n_all, int64_t n_centers, int n,
                           double period_x, int32_t *idx, cudaStream_t st) {
    RBF_REQUIRE(n >= 1 && n <= 128, "stencil size n=%d must be in [1, 128]", n);
    RBF_REQUIRE(n_all >= n, "n_all=%lld smaller than the stencil size %d", (long long)n_all, n);
    RBF_REQUIRE(n_all <= kStaticMaxNodes, "n_all=%lld exceeds the static scratch limit of %lld nodes",
                (long long)n_all, (long long)kStaticMaxNodes);
    RBF_REQUIRE(n_centers >= 0 && n_centers <= n_all, "n_centers=%lld out of range", (long long)n_centers);
    RBF_REQUIRE(period_x >= 0.0 && std::isfinite(period_x), "period_x must be finite and >= 0");
    if (n_centers == 0) return;
    RBF_REQUIRE(x && z && idx, "null pointer argument");
    unsigned char *base = static_scratch();
    double *part = reinterpret_cast<double *>(base + kOffPart);
    int *bad = reinterpret_cast<int *>(base + kOffBad);
    int *status = reinterpret_cast<int *>(base + kOffStatus);
    int *cellof = reinterpret_cast<int *>(base + kOffCellOf);
    int *sorted = reinterpret_cast<int *>(base + kOffSorted);
    int *count = reinterpret_cast<int *>(base + kOffCount);
    int *cursor = reinterpret_cast<int *>(base + kOffCursor);
    int *start = reinterpret_cast<int *>(base + kOffStart);

    // bounding box (the array keeps the previous call's contents: clear flags)
    RBF_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
    bbox_kernel<<<kBboxBlocks, 256, 0, st>>>(x, z, n_all, part, bad);
    RBF_CHECK_LAUNCH();
    double hp[kBboxBlocks * 4];
    int hbad = 0;
    RBF_CUDA(cudaMemcpyAsync(hp, part, sizeof(hp), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaStreamSynchronize(st));
    RBF_REQUIRE(!hbad, "non-finite node coordinates");
    double xmin = DBL_MAX, xmax = -DBL_MAX, zmin = DBL_MAX, zmax = -DBL_MAX;
    for (int b = 0; b < kBboxBlocks; ++b) {
        xmin = std::fmin(xmin, hp[b * 4 + 0]); xmax = std::fmax(xmax, hp[b * 4 + 1]);
        zmin = std::fmin(zmin, hp[b * 4 + 2]); zmax = std::fmax(zmax, hp[b * 4 + 3]);
    }
    // binning grid: the same rule as the allocating entry point
    Grid g;
    g.period = period_x;
    double W = period_x > 0.0 ? period_x : (xmax - xmin);
    double H = zmax - zmin;
    double area = std::fmax(W, 1e-300) * std::fmax(H, 1e-300);
    if (W <= 0.0 || H <= 0.0) area = std::fmax(W, H) * std::fmax(W, H) / (double)n_all;
    double cell = std::sqrt(2.0 * area / (double)n_all);
    if (!(cell > 0.0)) cell = 1.0;
    g.x0 = xmin;
    g.z0 = zmin;
    g.ncx = (int)std::fmax(1.0, std::fmin(std::floor(W / cell), 1e6));
    g.ncz = (int)std::fmax(1.0, std::fmin(std::ceil(H / cell), 1e6));
    if (period_x <= 0.0 && W / g.ncx > 0) g.ncx = (int)std::fmax(1.0, std::ceil(W / cell));
    g.cw = W > 0.0 ? W / g.ncx : cell;
    g.ch = H > 0.0 ? H / g.ncz : cell;
    const int64_t ncell = (int64_t)g.ncx * g.ncz;
    RBF_REQUIRE(ncell <= kStaticMaxCells, "binning grid of %lld cells exceeds the static scratch limit of %lld",
                (long long)ncell, (long long)kStaticMaxCells);

    RBF_CUDA(cudaMemsetAsync(count, 0, ncell * sizeof(int), st));
    RBF_CUDA(cudaMemsetAsync(cursor, 0, ncell * sizeof(int), st));
    RBF_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
    count_kernel<<<div_up(n_all, 256), 256, 0, st>>>(x, z, n_all, g, cellof, count);
    RBF_CHECK_LAUNCH();
    scan_kernel<<<1, 1024, 0, st>>>(count, (int)ncell, start);
    RBF_CHECK_LAUNCH();
    scatter_kernel<<<div_up(n_all, 256), 256, 0, st>>>(cellof, n_all, start, cursor, sorted);
    RBF_CHECK_LAUNCH();
    int R0 = (int)std::ceil(std::sqrt(2.5 * n / (4.0 * 2.0)));
    R0 = R0 < 1 ? 1 : R0;
    const int Rmax = std::max(g.ncx, g.ncz);
    const size_t smem = (size_t)kWarpsPerBlock * kMaxCand * (sizeof(double) + sizeof(int));
    RBF_CUDA(cudaFuncSetAttribute(knn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    knn_kernel<<<div_up(n_centers, kWarpsPerBlock), kWarpsPerBlock * 32, smem, st>>>(
        x, z, n_centers, n, g, start, sorted, R0, Rmax, idx, status);
    RBF_CHECK_LAUNCH();
    int hs = 0;
    RBF_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(cudaStreamSynchronize(st));
    RBF_REQUIRE(hs == 0, "stencil search failed (%s)",
                hs == 2 ? "more than 2048 candidates in a search window: node density too uneven"
                        : "no window holds n nodes");
}

}  // namespace rbf

extern "C" int rbf_build_stencils(const double *x, const double *z, int64_t n_all, int64_t n_centers,
                                  int32_t n, double period_x, int32_t *idx, void *stream) {
    return rbf::guarded([&] {
        rbf::build_stencils(x, z, n_all, n_centers, n, period_x, idx, rbf::as_stream(stream));
    });
}

extern "C" int rbf_build_stencils_static(const double *x, const double *z, int64_t n_all, int64_t n_centers,
                                         int32_t n, double period_x, int32_t *idx, void *stream) {
    return rbf::guarded([&] {
        rbf::build_stencils_static(x, z, n_all, n_centers, n, period_x, idx, rbf::as_stream(stream));
    });
}
