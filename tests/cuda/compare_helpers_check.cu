// Standalone GPU check of the FP64 comparison helpers of swe_kernels.cuh
// (gt_pos, le_pos, lt_pos, abs_lt_pos, gt_zero, ge_zero, le_zero, lt_zero,
// max_zero, min_nonneg, max_finite): each must return exactly what the
// plain IEEE expression it replaces returns, for every pair of values in a
// set of special values (signed zeros, denormals, the extremes of the finite
// range, infinities, quiet NaNs of both signs, the dry threshold and its
// neighbours) and seeded random bit patterns and magnitudes.  Prints one line
// per helper with its mismatch count and exits 0 when all are zero.
//
// It also checks inv_cbrt_newton (the FP64 friction's h^(-1/3)) against
// CUDA's double cube root over depths from 1e-6 to 1e5 m: the largest
// relative errors of r, r^3 (= 1/h) and r^7 (= h^(-7/3)), in units of 2^-52,
// printed as "ulps_r", "ulps_r3", "ulps_r7"; the run fails above 4, 8 and 16.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "swe_kernels.cuh"

using namespace swe;

constexpr int kChecks = 11;

__device__ bool same_bits(double a, double b) { return __double_as_longlong(a) == __double_as_longlong(b); }

__global__ void check(const double* xs, int n, const double* cs, int nc, unsigned long long* bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = xs[i];
    for (int j = 0; j < n; ++j) {
        const double y = xs[j];
        if (isfinite(x) && isfinite(y) && !same_bits(max_finite(x, y), x > y ? x : y)) atomicAdd(bad + 0, 1ULL);
        const bool nonneg = !signbit(x) && !signbit(y) && !isnan(x) && !isnan(y);
        if (nonneg && !same_bits(min_nonneg(x, y), x < y ? x : y)) atomicAdd(bad + 1, 1ULL);
    }
    for (int j = 0; j < nc; ++j) {
        const double c = cs[j];
        if (gt_pos(x, c) != (x > c)) atomicAdd(bad + 2, 1ULL);
        if (le_pos(x, c) != (x <= c)) atomicAdd(bad + 3, 1ULL);
        if (lt_pos(x, c) != (x < c)) atomicAdd(bad + 4, 1ULL);
        if (abs_lt_pos(x, c) != (fabs(x) < c)) atomicAdd(bad + 5, 1ULL);
    }
    if (gt_zero(x) != (x > 0.0)) atomicAdd(bad + 6, 1ULL);
    if (ge_zero(x) != (x >= 0.0)) atomicAdd(bad + 7, 1ULL);
    if (le_zero(x) != (x <= 0.0)) atomicAdd(bad + 8, 1ULL);
    if (lt_zero(x) != (x < 0.0)) atomicAdd(bad + 9, 1ULL);
    if (!same_bits(max_zero(x), 0.0 > x ? 0.0 : x)) atomicAdd(bad + 10, 1ULL);
}

__global__ void check_cbrt(int n, double* worst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double h = exp(log(1e-6) + (log(1e5) - log(1e-6)) * (i + 0.5) / n);   // log-spaced depths
    const double r = inv_cbrt_newton(h), r3 = r * r * r, r7 = r3 * r3 * r;
    const double c = cbrt(h);
    const double e[3] = {fabs(r * c - 1.0), fabs(r3 * h - 1.0), fabs(r7 * (h * h * c) - 1.0)};
    for (int k = 0; k < 3; ++k)   // non-negative doubles order like their bit patterns
        atomicMax((unsigned long long*)&worst[k], (unsigned long long)__double_as_longlong(e[k] / 2.220446049250313e-16));
}

static double from_bits(unsigned long long b) {
    double v;
    std::memcpy(&v, &b, sizeof v);
    return v;
}

int main() {
    std::vector<double> xs = {0.0, -0.0, 1.0, -1.0, INFINITY, -INFINITY, from_bits(0x7FF8000000000000ULL),
                              from_bits(0xFFF8000000000000ULL), from_bits(0x7FF0000000000001ULL),
                              from_bits(0x0000000000000001ULL), from_bits(0x8000000000000001ULL),
                              from_bits(0x000FFFFFFFFFFFFFULL), from_bits(0x0010000000000000ULL),
                              from_bits(0x7FEFFFFFFFFFFFFFULL), from_bits(0xFFEFFFFFFFFFFFFFULL),
                              1e-6, -1e-6, std::nextafter(1e-6, 1.0), std::nextafter(1e-6, 0.0), 3.0e38, -3.0e38,
                              std::nextafter(3.0e38, 0.0), std::nextafter(3.0e38, 1e300), 0.5, 2.0, 10.0, -10.0};
    unsigned long long s = 0x9E3779B97F4A7C15ULL;   // xorshift64 seed
    for (int k = 0; k < 3000; ++k) {
        s ^= s << 13;
        s ^= s >> 7;
        s ^= s << 17;
        if (k % 3 == 0) xs.push_back(from_bits(s));   // any bit pattern, NaNs included
        else xs.push_back((double)(s >> 11) / 9007199254740992.0 * std::pow(10.0, (int)(s % 19) - 9) *
                          ((s >> 7) & 1 ? -1.0 : 1.0));
    }
    const double cs[] = {1e-6, std::nextafter(1e-6, 1.0), 3.0e38, 0.5, 2.0, 10.0, from_bits(1ULL),
                         from_bits(0x7FEFFFFFFFFFFFFFULL)};
    const int n = (int)xs.size(), nc = (int)(sizeof cs / sizeof cs[0]);
    double *dx = nullptr, *dc = nullptr;
    unsigned long long* dbad = nullptr;
    if (cudaMalloc(&dx, n * sizeof(double)) != cudaSuccess || cudaMalloc(&dc, nc * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dbad, kChecks * sizeof(unsigned long long)) != cudaSuccess) {
        std::printf("device allocation failed\n");
        return 2;
    }
    cudaMemcpy(dx, xs.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(dc, cs, nc * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemset(dbad, 0, kChecks * sizeof(unsigned long long));
    check<<<(n + 127) / 128, 128>>>(dx, n, dc, nc, dbad);
    unsigned long long bad[kChecks];
    const cudaError_t e = cudaMemcpy(bad, dbad, sizeof bad, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        std::printf("cuda error: %s\n", cudaGetErrorString(e));
        return 2;
    }
    const char* names[kChecks] = {"max_finite", "min_nonneg", "gt_pos", "le_pos", "lt_pos", "abs_lt_pos",
                                  "gt_zero", "ge_zero", "le_zero", "lt_zero", "max_zero"};
    int failed = 0;
    for (int k = 0; k < kChecks; ++k) {
        std::printf("%s %llu\n", names[k], bad[k]);
        failed += bad[k] != 0;
    }
    std::printf("values %d\n", n);
    double* dworst = nullptr;
    const int nh = 1 << 20;
    double worst[3] = {0.0, 0.0, 0.0};
    if (cudaMalloc(&dworst, sizeof worst) != cudaSuccess) return 2;
    cudaMemcpy(dworst, worst, sizeof worst, cudaMemcpyHostToDevice);
    check_cbrt<<<nh / 256, 256>>>(nh, dworst);
    if (cudaMemcpy(worst, dworst, sizeof worst, cudaMemcpyDeviceToHost) != cudaSuccess) return 2;
    cudaFree(dworst);
    std::printf("ulps_r %.2f\nulps_r3 %.2f\nulps_r7 %.2f\n", worst[0], worst[1], worst[2]);
    failed += !(worst[0] <= 4.0) + !(worst[1] <= 8.0) + !(worst[2] <= 16.0);
    cudaFree(dx);
    cudaFree(dc);
    cudaFree(dbad);
    return failed ? 1 : 0;
}
