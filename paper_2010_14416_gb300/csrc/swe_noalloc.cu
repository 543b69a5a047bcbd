// swe_noalloc.cu -- an allocation-free CFL time step (swe_cfl_dt_noalloc).
//
// Some callers cannot call cudaMalloc: code that owns every byte of device
// memory through its own arena or pool, code running while a CUDA graph is
// being captured (where allocation is not allowed), and embedders that forbid
// the library from taking memory behind their back.  For them this entry
// point computes the CFL time step of a state without allocating anything.
// Its scratch (one partial minimum per thread block) lives in the file-scope
// device array below, which every GPU that loads this library holds until
// the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "swe_internal.h"

namespace swe {
namespace {

constexpr int kNoallocBlock = 256;
constexpr int kNoallocMaxBlocks = 65536;  // 512 KiB of scratch

// per-block minima of R_i / (sqrt(g h_i) + |u_i|); every call rewrites the
// slots of the blocks it launches, so nothing has to be cleared between calls
static __device__ __align__(256) double g_noalloc_scratch[kNoallocMaxBlocks];

template <typename T>
__global__ void __launch_bounds__(kNoallocBlock)
cfl_partial_kernel(const T* __restrict__ h, const T* __restrict__ hu, const T* __restrict__ hv,
                   const T* __restrict__ rin, long long n, T g, T h_dry, double* __restrict__ partial) {
    using A = Ar<T>;
    __shared__ double warp_min[kNoallocBlock / 32];
    const long long i = (long long)blockIdx.x * kNoallocBlock + threadIdx.x;
    double cand = __longlong_as_double((long long)kInfBits);
    if (i < n) {
        const T hi = h[i];
        if (hi > h_dry) {
            const T r = A::rcp_(hi);
            const T u = hu[i] * r, v = hv[i] * r;
            cand = (double)A::div_(rin[i], A::sqrt_(g * hi) + A::sqrt_(u * u + v * v));
        }
    }
    for (int o = 16; o > 0; o >>= 1) cand = fmin(cand, __shfl_xor_sync(0xffffffffu, cand, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_min[wid] = cand;
    __syncthreads();
    if (wid == 0) {
        double v = lane < kNoallocBlock / 32 ? warp_min[lane] : __longlong_as_double((long long)kInfBits);
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) partial[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(1024)
cfl_final_kernel(const double* __restrict__ partial, int n_blocks, double cfl, double* __restrict__ dt_out) {
    __shared__ double warp_min[32];
    double v = __longlong_as_double((long long)kInfBits);
    for (int b = threadIdx.x; b < n_blocks; b += 1024) v = fmin(v, partial[b]);
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_min[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = warp_min[lane];
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) *dt_out = cfl * v;
    }
}

// Device address of the scratch array on the current device.  The array's
// name in host code is only a host-side stand-in, so the address is asked for
// on every call (the lookup allocates nothing): a cached address would point
// at freed memory once cudaDeviceReset has replaced the device's context.
// The first lookup on a device loads this library's device code there.
int scratch_address(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        set_error(std::string("swe_cfl_dt_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return SWE_ECUDA;
    }
    *out = (double*)p;
    return SWE_OK;
}

}  // namespace
}  // namespace swe

using namespace swe;

extern "C" int swe_cfl_dt_noalloc(int precision, int64_t n, const void* h, const void* hu, const void* hv,
                                  const void* rin, double g, double h_dry, double cfl, double* dt_out,
                                  void* stream) {
    if (n < 1 || !h || !hu || !hv || !rin || !dt_out || !(g > 0.0) || !(h_dry > 0.0) || !(cfl > 0.0) ||
        !std::isfinite(cfl)) {
        set_error("swe_cfl_dt_noalloc: bad arguments");
        return SWE_EINVAL;
    }
    if (n > (int64_t)kNoallocMaxBlocks * kNoallocBlock) {
        set_error("swe_cfl_dt_noalloc: " + std::to_string(n) + " cells exceed the allocation-free limit of " +
                  std::to_string((int64_t)kNoallocMaxBlocks * kNoallocBlock) + " cells");
        return SWE_EINVAL;
    }
    if (precision != SWE_FP64 && precision != SWE_FP32) {
        set_error("swe_cfl_dt_noalloc: bad precision");
        return SWE_EINVAL;
    }
    double* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    const int nb = (int)((n + kNoallocBlock - 1) / kNoallocBlock);
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == SWE_FP32)
        cfl_partial_kernel<float><<<nb, kNoallocBlock, 0, st>>>(
            (const float*)h, (const float*)hu, (const float*)hv, (const float*)rin, (long long)n, (float)g,
            (float)h_dry, scratch);
    else
        cfl_partial_kernel<double><<<nb, kNoallocBlock, 0, st>>>(
            (const double*)h, (const double*)hu, (const double*)hv, (const double*)rin, (long long)n, g, h_dry,
            scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        cfl_final_kernel<<<1, 1024, 0, st>>>(scratch, nb, cfl, dt_out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error(std::string("swe_cfl_dt_noalloc: launch: ") + cudaGetErrorString(e));
        return SWE_ECUDA;
    }
    return SWE_OK;
}
