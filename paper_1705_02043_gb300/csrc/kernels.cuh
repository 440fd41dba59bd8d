// Free-space kernels of Eq. (kexamples) on the device, accumulated into
// per-thread registers.  r = x - y; coincident points (r = 0) contribute
// nothing (the excluded self term).
#pragma once
#include <cuda_runtime.h>

namespace pk {

__device__ __forceinline__ double inv_sqrt(double r2) { return r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0; }
__device__ __forceinline__ float inv_sqrt(float r2) { return r2 > 0.0f ? rsqrtf(r2) : 0.0f; }

template <typename T, int K>
struct Kern;

// Laplace 1/r
template <typename T>
struct Kern<T, 1> {
    static __device__ __forceinline__ void add(T *acc, T dx, T dy, T dz, const T *phi) {
        T ir = inv_sqrt(dx * dx + dy * dy + dz * dz);
        acc[0] += ir * phi[0];
    }
};

// Stokes velocity (1/8pi)(I/r + r r^T/r^3)
template <typename T>
struct Kern<T, 3> {
    static __device__ __forceinline__ void add(T *acc, T dx, T dy, T dz, const T *f) {
        T ir = inv_sqrt(dx * dx + dy * dy + dz * dz);
        const T c = (T)0.039788735772973836;  // 1/(8 pi)
        T cir = c * ir;
        T fr = (f[0] * dx + f[1] * dy + f[2] * dz) * cir * ir * ir;
        acc[0] += f[0] * cir + dx * fr;
        acc[1] += f[1] * cir + dy * fr;
        acc[2] += f[2] * cir + dz * fr;
    }
};

}  // namespace pk
