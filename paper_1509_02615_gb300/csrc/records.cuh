// Node-major state records: the four prognostic fields [u, w, theta', pi']
// of one node are contiguous (16 bytes in FP32, 32 bytes in FP64), so a
// stencil gather is one or two 16-byte loads per neighbour.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rbf {

template <class T>
struct Rec {
    T u, w, t, p;
};

// Read-only (non-coherent) load of record j; valid for data that no thread
// of the running kernel writes.
__device__ __forceinline__ Rec<float> load_rec(const float *U, int64_t j) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(U) + j);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Rec<double> load_rec(const double *U, int64_t j) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(U) + 2 * j);
    const double2 b = __ldg(reinterpret_cast<const double2 *>(U) + 2 * j + 1);
    return {a.x, a.y, b.x, b.y};
}

}  // namespace rbf
