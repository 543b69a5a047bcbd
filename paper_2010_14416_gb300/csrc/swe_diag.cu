// swe_diag.cu -- diagnostics of a mesh's state (swe_diagnostics) and a
// steady-state driver (swe_run_to_steady).
//
// The paper computes inflow and outflow rates during its runs and copies
// them to the host on a side stream (Section 5.3.2), and it first runs to a
// stabilised solution before the production runs (Section 6.3.2).  Here:
//   - cell reductions (stored volume, largest depth change over the last step,
//     largest depth and speed, wet cells) in per-block partials on a fixed
//     grid, summed by one block: deterministic;
//   - the outward discharge through each boundary group, evaluated with the
//     step kernel's own boundary flux on the current state (the mass that
//     leaves through those edges in the next step per unit time), one value
//     per boundary edge, summed per group on the host in a fixed order.
// Interior fluxes cancel, so volume^{n+1} - volume^n = -dt_n * sum of the
// discharges evaluated on U^n.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "swe_internal.h"

using namespace swe;

namespace {

constexpr int kDiagBlock = 256;
constexpr int kDiagMaxBlocks = 1024;
constexpr int kDiagWords = 5;  // volume, dh_max, h_max, speed_max, n_wet

template <typename T>
__global__ void __launch_bounds__(kDiagBlock)
diag_cells_kernel(const V4<T>* __restrict__ cur, const V4<T>* __restrict__ prev, const V4<T>* __restrict__ geoB,
                  long long n, double h_dry, int have_prev, double* __restrict__ partial) {
    double vol = 0.0, dh = 0.0, hmax = 0.0, spd = 0.0, wet = 0.0;
    for (long long i = (long long)blockIdx.x * kDiagBlock + threadIdx.x; i < n; i += (long long)gridDim.x * kDiagBlock) {
        const V4<T> c = cur[i];
        const double h = (double)c.x;
        vol += h / (double)geoB[i].z;
        if (have_prev) dh = fmax(dh, fabs(h - (double)prev[i].x));
        hmax = fmax(hmax, h);
        if (h > h_dry) {
            wet += 1.0;
            const double u = (double)c.y / h, v = (double)c.z / h;
            spd = fmax(spd, sqrt(u * u + v * v));
        }
    }
    __shared__ double red[kDiagWords][kDiagBlock];
    red[0][threadIdx.x] = vol; red[1][threadIdx.x] = dh; red[2][threadIdx.x] = hmax;
    red[3][threadIdx.x] = spd; red[4][threadIdx.x] = wet;
    __syncthreads();
    for (int s = kDiagBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + s]);
            red[2][threadIdx.x] = fmax(red[2][threadIdx.x], red[2][threadIdx.x + s]);
            red[3][threadIdx.x] = fmax(red[3][threadIdx.x], red[3][threadIdx.x + s]);
            red[4][threadIdx.x] += red[4][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x < kDiagWords) partial[blockIdx.x * kDiagWords + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void diag_final_kernel(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    if (threadIdx.x == 0) {
        double vol = 0.0, dh = 0.0, hmax = 0.0, spd = 0.0, wet = 0.0;
        for (int b = 0; b < nb; ++b) {
            vol += partial[b * kDiagWords];
            dh = fmax(dh, partial[b * kDiagWords + 1]);
            hmax = fmax(hmax, partial[b * kDiagWords + 2]);
            spd = fmax(spd, partial[b * kDiagWords + 3]);
            wet += partial[b * kDiagWords + 4];
        }
        out[0] = vol; out[1] = dh; out[2] = hmax; out[3] = spd; out[4] = wet;
    }
}

// one boundary edge per thread: L * (outward mass flux) with the step's
// boundary treatment (Section 3.1)
template <typename T>
__global__ void diag_boundary_kernel(const V4<T>* __restrict__ cur, const V4<T>* __restrict__ geoA,
                                     const V4<T>* __restrict__ geoB, const V4<T>* __restrict__ geoR,
                                     const long long* __restrict__ slots,
                                     const int* __restrict__ groups, long long nb, BcTable bc, T g, T h_dry,
                                     int hll, double* __restrict__ q) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const long long s = slots[k];
    const long long i = s / 3;
    const int j = (int)(s % 3);
    const V4<T> c = cur[i];
    const V4<T> gA = geoA[i], gB = geoB[i];
    const T lx = j == 0 ? gA.x : (j == 1 ? gA.z : gB.x);
    const T ly = j == 0 ? gA.y : (j == 1 ? gA.w : gB.y);
    const T l2 = edge_l2(lx, ly);
    T pre = T(0);
    if constexpr (sizeof(T) == 8) {
        const V4<T> gR = geoR[i];
        pre = j == 0 ? gR.x : (j == 1 ? gR.y : gR.z);
    }
    const T rl = edge_rl<T>(pre, l2);   // the step's own edge scale
    const T len = l2 * rl;
    T ui, vi;
    cell_velocity<T>(c.x, c.y, c.z, h_dry, ui, vi);
    const int grp = groups[k];
    T F0, F1, F2;
    edge_boundary<T>(bc.kind[grp], bc.value[grp], c.x, ui, vi, c.w, lx * rl, ly * rl, g, h_dry, F0, F1, F2, hll != 0);
    q[k] = (double)len * (double)F0;
}

int dfail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return SWE_ECUDA;
}

struct DiagDeviceGuard {
    int prev = -1;
    explicit DiagDeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DiagDeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
int diagnostics_t(swe_mesh* m, swe_diag* out) {
    const int64_t n = m->hm.n_cells;
    cudaStream_t st = m->stream;
    // boundary edges in a fixed order (internal cell, local edge)
    std::vector<long long> slots;
    std::vector<int> groups;
    for (int64_t s = 0; s < 3 * n; ++s)
        if (m->hm.code[s] < 0) {
            slots.push_back(s);
            groups.push_back(-1 - m->hm.code[s]);
        }
    const long long nb = (long long)slots.size();
    const int nblk = (int)std::min<long long>(kDiagMaxBlocks, (n + kDiagBlock - 1) / kDiagBlock);
    void *partial = nullptr, *res = nullptr, *dslots = nullptr, *dgroups = nullptr, *dq = nullptr;
    cudaError_t e = cudaMalloc(&partial, (size_t)nblk * kDiagWords * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&res, kDiagWords * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dslots, std::max<long long>(nb, 1) * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&dgroups, std::max<long long>(nb, 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&dq, std::max<long long>(nb, 1) * sizeof(double));
    std::vector<double> q(nb), r(kDiagWords);
    unsigned long long sm[kSmallWords];
    if (e == cudaSuccess && nb)
        e = cudaMemcpyAsync(dslots, slots.data(), nb * sizeof(long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && nb)
        e = cudaMemcpyAsync(dgroups, groups.data(), nb * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const V4<T>* cur = (const V4<T>*)m->state[m->nstep % 2];
        const V4<T>* prev = (const V4<T>*)m->state[(m->nstep + 1) % 2];
        diag_cells_kernel<T><<<nblk, kDiagBlock, 0, st>>>(cur, prev, (const V4<T>*)m->geoB, n, m->cfg.h_dry,
                                                         m->nstep > 0 ? 1 : 0, (double*)partial);
        diag_final_kernel<<<1, 32, 0, st>>>((const double*)partial, nblk, (double*)res);
        if (nb)
            diag_boundary_kernel<T><<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(
                cur, (const V4<T>*)m->geoA, (const V4<T>*)m->geoB, (const V4<T>*)m->geoR, (const long long*)dslots,
                (const int*)dgroups, nb,
                m->bc, (T)m->cfg.g, (T)m->cfg.h_dry, m->cfg.flux == SWE_FLUX_HLL ? 1 : 0, (double*)dq);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.data(), res, kDiagWords * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && nb) e = cudaMemcpyAsync(q.data(), dq, nb * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sm, m->small, sizeof sm, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (void* p : {partial, res, dslots, dgroups, dq})
        if (p) cudaFree(p);
    if (e != cudaSuccess) return dfail(e, "swe_diagnostics");
    std::memset(out, 0, sizeof *out);
    out->volume = r[0];
    out->dh_max = r[1];
    out->h_max = r[2];
    out->speed_max = r[3];
    out->n_wet = (int64_t)r[4];
    out->n_groups = m->n_groups;
    for (long long k = 0; k < nb; ++k) out->discharge[groups[k]] += q[k];
    std::memcpy(&out->t, &sm[kSlotT], sizeof(double));
    if (m->nstep > 0) std::memcpy(&out->dt_last, &sm[kSlotDtLast], sizeof(double));
    return SWE_OK;
}

}  // namespace

extern "C" {

int swe_diagnostics(swe_mesh* m, swe_diag* out) {
    if (!m || !out) { set_error("swe_diagnostics: bad arguments"); return SWE_EINVAL; }
    if (!m->have_state) { set_error("swe_diagnostics: no state set"); return SWE_EINVAL; }
    DiagDeviceGuard dg(m->cfg.device);
    int rc = flush_mesh_bc(m);
    if (rc) return rc;
    return m->cfg.precision == SWE_FP32 ? diagnostics_t<float>(m, out) : diagnostics_t<double>(m, out);
}

int swe_run_to_steady(swe_mesh* m, double cfl, double tol, int64_t check_every, int64_t max_steps,
                      int64_t* steps_done, int* converged, double* t_out) {
    NvtxRange nvtx_range("swe_run_to_steady");
    if (!m || !(tol > 0.0) || check_every < 1 || max_steps < 0) {
        set_error("swe_run_to_steady: bad arguments");
        return SWE_EINVAL;
    }
    int64_t done = 0;
    int conv = 0;
    swe_diag d;
    while (done < max_steps) {
        const int64_t k = std::min(check_every, max_steps - done);
        double t;
        int rc = swe_step(m, k, cfl, &t);
        if (rc) return rc;
        done += k;
        rc = swe_diagnostics(m, &d);
        if (rc) return rc;
        if (d.dt_last > 0.0 && d.dh_max / d.dt_last < tol) { conv = 1; break; }
    }
    if (steps_done) *steps_done = done;
    if (converged) *converged = conv;
    if (t_out) {
        swe_info info;
        int rc = swe_get_info(m, &info);
        if (rc) return rc;
        *t_out = info.t;
    }
    return SWE_OK;
}

}  // extern "C"
