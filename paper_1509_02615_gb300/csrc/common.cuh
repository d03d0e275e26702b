// Shared host-side plumbing of librbffd: error reporting, checked CUDA calls,
// device buffers.  No method arithmetic lives here.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "../../include/rbffd.h"

namespace rbf {

// Message of the last failure on this thread (rbf_last_error).
void set_error(const char *fmt, ...);
const char *last_error();

// Thrown inside the library, caught at every extern "C" boundary.
struct Failure {
    int code;
};

[[noreturn]] inline void fail(int code) { throw Failure{code}; }

#define RBF_FAIL(code, ...)          \
    do {                             \
        ::rbf::set_error(__VA_ARGS__); \
        ::rbf::fail(code);           \
    } while (0)

#define RBF_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            int c_ = (e_ == cudaErrorMemoryAllocation) ? RBF_E_OOM : RBF_E_CUDA;          \
            RBF_FAIL(c_, "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
        }                                                                                 \
    } while (0)

#define RBF_CHECK_LAUNCH() RBF_CUDA(cudaGetLastError())

#define RBF_REQUIRE(cond, ...)                   \
    do {                                         \
        if (!(cond)) RBF_FAIL(RBF_E_ARG, __VA_ARGS__); \
    } while (0)

// Runs f, converting library failures into return codes.
template <class F>
int guarded(F &&f) {
    try {
        f();
        return RBF_OK;
    } catch (const Failure &e) {
        return e.code;
    } catch (const std::exception &e) {
        set_error("internal error: %s", e.what());
        return RBF_E_ARG;
    } catch (...) {
        set_error("internal error");
        return RBF_E_ARG;
    }
}

// Owning device buffer (cudaMalloc / cudaFree).
template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    explicit DevBuf(size_t count) { alloc(count); }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count) {
        release();
        n = count;
        if (count) RBF_CUDA(cudaMalloc((void **)&p, count * sizeof(T)));
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
};

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Number of SMs of the current device (cached per call site by callers).
int sm_count();

// Programmatic dependent launch (sm_90+): a kernel launched with
// programmatic stream serialization may start while its predecessor is still
// running.  It must call grid_dep_wait() before touching memory that an
// earlier kernel writes or reads-after-us; work on constant inputs (weights,
// indices) can go before the wait.  grid_dep_launch() lets the next kernel
// be scheduled.  Both are no-ops for ordinary launches.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// prio != 0: the launch's scheduling priority (lower is more urgent; in a
// captured graph it becomes the kernel node's priority, which graphs
// instantiated with cudaGraphInstantiateFlagUseNodePriority honour).
template <typename... KArgs, typename... Args>
void launch_kernel_prio(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, bool pdl, int prio,
                        Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    int na = 0;
    if (pdl) {
        at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    if (prio != 0) {
        at[na].id = cudaLaunchAttributePriority;
        at[na].val.priority = prio;
        ++na;
    }
    cfg.attrs = na ? at : nullptr;
    cfg.numAttrs = na;
    RBF_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

template <typename... KArgs, typename... Args>
void launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, bool pdl, Args &&...args) {
    launch_kernel_prio(kernel, grid, block, s, pdl, 0, std::forward<Args>(args)...);
}

// ---- internal entry points shared between translation units ----------------
// a1: stencils of nodes [0, n_centers) among all n_all (device arrays).
void build_stencils(const double *x, const double *z, int64_t n_all, int64_t n_centers, int n,
                    double period_x, int32_t *idx, cudaStream_t st);
// a2: weights [n_ops][n_centers][n] (device), FP64.  Writes the first failing
// node into *bad_node (host) or -1.
void build_weights(const double *x, const double *z, int64_t n_all, const int32_t *idx, int64_t n_centers, int n,
                   double period_x, int p, int l, int hv_k, const int *ops, int n_ops, double *w,
                   cudaStream_t st);

}  // namespace rbf
