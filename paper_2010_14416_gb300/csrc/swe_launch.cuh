// swe_launch.cuh -- definitions of the per-precision launchers; included by
// exactly one translation unit per precision (swe_step_f32.cu, swe_step_f64.cu).
#pragma once

#include "swe_kernels.cuh"

namespace swe {

template <typename T>
static inline unsigned grid_for(long long n, int block) {
    return (unsigned)((n + block - 1) / block);
}

template <typename T>
cudaError_t Launch<T>::step(const StepArgs<T>& a, int block, cudaStream_t st) {
    const long long n = a.n;
    switch (block) {
        case 128: step_kernel<T, 128><<<grid_for<T>(n, 128), 128, 0, st>>>(a); break;
        case 256: step_kernel<T, 256><<<grid_for<T>(n, 256), 256, 0, st>>>(a); break;
        case 512: step_kernel<T, 512><<<grid_for<T>(n, 512), 512, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::dt(const V4<T>* s, const V4<T>* geoB, long long n, T g, T h_dry,
                          unsigned long long* dt_write, cudaStream_t st) {
    dt_kernel<T, 256><<<grid_for<T>(n, 256), 256, 0, st>>>(s, geoB, n, g, h_dry, dt_write);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::pack(const T* h, const T* hu, const T* hv, const long long* perm, const T* z,
                            V4<T>* s, long long n, cudaStream_t st) {
    pack_state_kernel<T><<<grid_for<T>(n, 256), 256, 0, st>>>(h, hu, hv, perm, z, s, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::unpack(const V4<T>* s, const long long* perm, T* h, T* hu, T* hv, long long n,
                              cudaStream_t st) {
    unpack_state_kernel<T><<<grid_for<T>(n, 256), 256, 0, st>>>(s, perm, h, hu, hv, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::riemann(long long n, const T* hL, const T* unL, const T* utL, const T* hR,
                               const T* unR, const T* utR, T g, T h_dry, T* G1, T* G2, T* G3, T* S,
                               cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    riemann_batch_kernel<T><<<grid_for<T>(n, 256), 256, 0, st>>>(n, hL, unL, utL, hR, unR, utR, g, h_dry,
                                                                   G1, G2, G3, S);
    return cudaGetLastError();
}

}  // namespace swe
