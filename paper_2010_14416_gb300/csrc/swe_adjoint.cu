// swe_adjoint.cu -- discrete adjoint of the FP64 step (swe_adjoint), frozen-dt
// stepping (swe_step_dt) and parameter updates (swe_set_fields).
//
// The loss is L = sum_g (h_g^N - target_g)^2 after N steps with the step
// sizes frozen at the forward run's values.  With U^{n+1} = F(U^n; z, m) the
// adjoint state lambda^n = (dF/dU^n)^T lambda^{n+1} runs backwards from
// lambda^N = dL/dU^N, accumulating dL/dz and dL/dm on the way.  Cell i's
// update is U_i + Phi(U_i, m_i, R_i), R_i = (1/|Omega_i|) sum_e E_ie, where
// E_ie is the edge's flux-and-bed-source contribution (Eq 13, 30, 37).  One
// reverse step is two gathers, no atomics:
//   phase 1 (cell i): recompute R_i; differentiate Phi on 7-component duals
//     (h, hu, hv, g m^2, R) -> own term a_i, dL/dm_i, nu_i = (dPhi/dR)^T lambda / |Omega_i|
//   phase 2 (cell j): differentiate each edge term E_je and the neighbour's
//     E_ie on 4-component duals (h_j, hu_j, hv_j, z_j):
//     lambda^n_j = a_j + sum_e (dE_je)^T nu_j + (dE_ie)^T nu_i,  dL/dz_j likewise.
// Both phases run the forward's own templated edge and friction functions,
// so the derivatives are those of the branches the forward takes.
// States are recomputed segment by segment from checkpoints taken every k
// steps of the forward run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "swe_dual.cuh"
#include "swe_internal.h"

using namespace swe;

namespace {

using D4 = Dual<4>;
using D7 = Dual<7>;

struct AdjArgs {
    const V4<double>* __restrict__ U;     // state U^n, internal order
    const V4<double>* __restrict__ geoA;
    const V4<double>* __restrict__ geoB;
    const V4<double>* __restrict__ geoR;  // 1/|L n| of the three edges (the forward's)
    const int4* __restrict__ topo;
    const double* __restrict__ gm2;
    V4<double>* __restrict__ lam;         // lambda (h, hu, hv, -)
    V4<double>* __restrict__ aw;          // own term of phase 1
    V4<double>* __restrict__ nu;          // (dPhi/dR)^T lambda / |Omega|
    double* __restrict__ gm;              // dL/d(g m^2), accumulated
    double* __restrict__ gz;              // dL/dz, accumulated
    long long n;
    double dt, g, h_dry;
    int hll;
    BcTable bc;
    // phase 1 with the edge pass: the interior fluxes of U^n from edge_flux_kernel
    const V4<double>* __restrict__ eflux;
    const double* __restrict__ esrc;
    const int4* __restrict__ eidx;
};

// the forward's unit normal and length of an edge, from its 1/|L n|
__device__ __forceinline__ void unit_normal(double lx, double ly, double rl, double& n1, double& n2, double& len) {
    const double l2 = lx * lx + ly * ly;
    len = l2 * rl;
    n1 = lx * rl;
    n2 = ly * rl;
}

__device__ __forceinline__ void edge_ln(const V4<double>& gA, const V4<double>& gB, int j, double& lx, double& ly) {
    lx = j == 0 ? gA.x : (j == 1 ? gA.z : gB.x);
    ly = j == 0 ? gA.y : (j == 1 ? gA.w : gB.y);
}

// EDGES reads R_i's interior fluxes from the edge pass (the forward's own
// edge-pass arithmetic) instead of evaluating them; R_i is the same bit for bit.
template <bool EDGES>
__global__ void __launch_bounds__(128) adj_phase1_kernel(const AdjArgs a) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const double g = a.g, h_dry = a.h_dry;
    const V4<double> own = a.U[i];
    const V4<double> gA = a.geoA[i], gB = a.geoB[i], gR = a.geoR[i];
    const int4 tp = a.topo[i];
    const int code[3] = {tp.x, tp.y, tp.z};
    const double hi = own.x, zi = own.w;
    double ui, vi;
    cell_velocity<double>(hi, own.y, own.z, h_dry, ui, vi);
    // the forward's explicit right-hand side R_i
    double f0 = 0.0, f1 = 0.0, f2 = 0.0, sx = 0.0, sy = 0.0;
    int4 ei = make_int4(-1, -1, -1, 0);
    if constexpr (EDGES) ei = a.eidx[i];
    for (int j = 0; j < 3; ++j) {
        double lx, ly, n1, n2, len;
        edge_ln(gA, gB, j, lx, ly);
        unit_normal(lx, ly, j == 0 ? gR.x : (j == 1 ? gR.y : gR.z), n1, n2, len);
        double F0, F1, F2;
        const int c = code[j];
        if (c >= 0) {
            const V4<double> o = a.U[c & kNbrMask];
            double src;
            if constexpr (EDGES) {
                if (!(hi > h_dry) && !(o.x > h_dry)) {
                    const double zs = tmax(zi, o.w);
                    const double hsi = tmax(0.0, hi + zi - zs);
                    F0 = 0.0; F1 = 0.0; F2 = 0.0;
                    src = 0.5 * g * (hsi * hsi - hi * hi);
                } else {
                    const int e = j == 0 ? ei.x : (j == 1 ? ei.y : ei.z);
                    const V4<double> fl = a.eflux[e];
                    if (c & kFlipBit) {
                        F0 = -fl.x; F1 = -fl.y; F2 = -fl.z;
                        src = a.esrc[e];
                    } else {
                        F0 = fl.x; F1 = fl.y; F2 = fl.z;
                        src = fl.w;
                    }
                }
            } else {
                edge_interior<double>(hi, ui, vi, zi, o.x, o.y, o.z, o.w, n1, n2, (c & kFlipBit) != 0, g, h_dry, F0,
                                      F1, F2, src, a.hll != 0);
            }
            sx += src * lx;
            sy += src * ly;
        } else {
            const int grp = -1 - c;
            edge_boundary<double>(a.bc.kind[grp], a.bc.value[grp], hi, ui, vi, zi, n1, n2, g, h_dry, F0, F1, F2,
                                  a.hll != 0);
        }
        f0 += len * F0;
        f1 += len * F1;
        f2 += len * F2;
    }
    const double ia = gB.z;
    const double Rh = -f0 * ia, Rx = (sx - f1) * ia, Ry = (sy - f2) * ia;
    // Phi on duals: seeds h, hu, hv, g m^2, Rh, Rx, Ry
    D7 dh, dqx, dqy;
    friction_update<D7>(D7::seed(hi, 0), D7::seed(own.y, 1), D7::seed(own.z, 2), D7::seed(a.gm2[i], 3),
                        D7::seed(Rh, 4), D7::seed(Rx, 5), D7::seed(Ry, 6), D7(a.dt), D7(h_dry), dh, dqx, dqy);
    // the forward's clamps: h < 0 zeroes the cell, h <= h_dry zeroes momentum
    const V4<double> L = a.lam[i];
    double lh = L.x, lx_ = L.y, ly_ = L.z;
    const double hn = hi + dh.v;
    if (hn < 0.0) { lh = 0.0; lx_ = 0.0; ly_ = 0.0; }
    else if (hn <= h_dry) { lx_ = 0.0; ly_ = 0.0; }
    double w[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) w[k] = lh * dh.d[k] + lx_ * dqx.d[k] + ly_ * dqy.d[k];
    V4<double> own_term;
    own_term.x = lh + w[0];
    own_term.y = lx_ + w[1];
    own_term.z = ly_ + w[2];
    own_term.w = 0.0;
    a.aw[i] = own_term;
    a.gm[i] += w[3];
    V4<double> nu;
    nu.x = w[4] * ia;
    nu.y = w[5] * ia;
    nu.z = w[6] * ia;
    nu.w = 0.0;
    a.nu[i] = nu;
}

__global__ void __launch_bounds__(128) adj_phase2_kernel(const AdjArgs a) {
    const long long jc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (jc >= a.n) return;
    const double g = a.g, h_dry = a.h_dry;
    const V4<double> own = a.U[jc];
    const V4<double> gA = a.geoA[jc], gB = a.geoB[jc], gR = a.geoR[jc];
    const int4 tp = a.topo[jc];
    const int code[3] = {tp.x, tp.y, tp.z};
    const V4<double> nuj = a.nu[jc];
    const D4 H = D4::seed(own.x, 0), QX = D4::seed(own.y, 1), QY = D4::seed(own.z, 2), Z = D4::seed(own.w, 3);
    D4 U, V;
    cell_velocity<D4>(H, QX, QY, D4(h_dry), U, V);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 1
    for (int j = 0; j < 3; ++j) {
        double lx, ly, n1, n2, len;
        edge_ln(gA, gB, j, lx, ly);
        unit_normal(lx, ly, j == 0 ? gR.x : (j == 1 ? gR.y : gR.z), n1, n2, len);
        const int c = code[j];
        D4 F0, F1, F2;
        if (c >= 0) {
            const long long i = c & kNbrMask;
            const V4<double> o = a.U[i];
            D4 src;
            edge_interior<D4>(H, U, V, Z, D4(o.x), D4(o.y), D4(o.z), D4(o.w), D4(n1), D4(n2), (c & kFlipBit) != 0,
                              D4(g), D4(h_dry), F0, F1, F2, src, a.hll != 0);
            // this cell's term E_je = (-len F0, -len F1 + src lx, -len F2 + src ly)
            // the neighbour's E_ie = (len F0, len F1 - src_i lx, len F2 - src_i ly),
            // src_i = (g/2)(h**_i^2 - h_i^2) with z* = max(z_i, z_j) as the neighbour forms it
            const D4 zs_i = tmax(D4(o.w), Z);
            const D4 hs_i = tmax(D4(0.0), D4(o.x) + D4(o.w) - zs_i);
            const D4 src_i = D4(0.5 * g) * (hs_i * hs_i - D4(o.x * o.x));
            const V4<double> nui = a.nu[i];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double e0 = -len * F0.d[k];
                const double e1 = -len * F1.d[k] + src.d[k] * lx;
                const double e2 = -len * F2.d[k] + src.d[k] * ly;
                const double o0 = len * F0.d[k];
                const double o1 = len * F1.d[k] - src_i.d[k] * lx;
                const double o2 = len * F2.d[k] - src_i.d[k] * ly;
                acc[k] += nuj.x * e0 + nuj.y * e1 + nuj.z * e2 + nui.x * o0 + nui.y * o1 + nui.z * o2;
            }
        } else {
            const int grp = -1 - c;
            edge_boundary<D4>(a.bc.kind[grp], a.bc.value[grp], H, U, V, Z, D4(n1), D4(n2), D4(g), D4(h_dry), F0, F1,
                              F2, a.hll != 0);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                acc[k] += -len * (nuj.x * F0.d[k] + nuj.y * F1.d[k] + nuj.z * F2.d[k]);
        }
    }
    const V4<double> aw = a.aw[jc];
    V4<double> out;
    out.x = aw.x + acc[0];
    out.y = aw.y + acc[1];
    out.z = aw.z + acc[2];
    out.w = 0.0;
    a.lam[jc] = out;
    a.gz[jc] += acc[3];
}

// loss += sum_g (h_g - target_g)^2 for one observation (one thread: fixed order)
__global__ void adj_loss_kernel(const V4<double>* __restrict__ U, const long long* __restrict__ gauges,
                                const double* __restrict__ target, int n_gauges, double* __restrict__ loss) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double L = *loss;
        for (int k = 0; k < n_gauges; ++k) {
            const double r = U[gauges[k]].x - target[k];
            L += r * r;
        }
        *loss = L;
    }
}

// lambda^n += d(observation)/dU^n: 2 (h_g - target_g) on the gauges' depths
__global__ void adj_inject_kernel(const V4<double>* __restrict__ U, const long long* __restrict__ gauges,
                                  const double* __restrict__ target, int n_gauges, V4<double>* __restrict__ lam) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int k = 0; k < n_gauges; ++k) {
            const long long c = gauges[k];
            lam[c].x += 2.0 * (U[c].x - target[k]);
        }
    }
}

// caller-order gradients: dL/dm = dL/d(g m^2) * 2 g m, dL/dz as is
__global__ void adj_output_kernel(const double* __restrict__ gm, const double* __restrict__ gz,
                                  const double* __restrict__ gm2, const long long* __restrict__ perm, double g,
                                  double* __restrict__ out_m, double* __restrict__ out_z, long long n) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) {
        const long long o = perm[c];
        // g m = sqrt(g * g m^2) for m >= 0
        if (out_m) out_m[o] = gm[c] * 2.0 * sqrt(g * gm2[c]);
        if (out_z) out_z[o] = gz[c];
    }
}

template <typename T>
__global__ void set_z_kernel(V4<T>* __restrict__ s0, V4<T>* __restrict__ s1, const T* __restrict__ z, long long n) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) {
        s0[c].w = z[c];
        s1[c].w = z[c];
    }
}

int afail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return SWE_ECUDA;
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

struct AdjDeviceGuard {
    int prev = -1;
    explicit AdjDeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~AdjDeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

__global__ void small_init_kernel(unsigned long long* small) {
    if (threadIdx.x < kSmallWords) small[threadIdx.x] = threadIdx.x < 3 ? kInfBits : 0ULL;
}

// Observations every obs_every steps (obs_every divides nsteps); targets:
// [nsteps / obs_every][n_gauges].
int adjoint_impl(swe_mesh* m, int64_t nsteps, double cfl, const int32_t* gauge_cells, int n_gauges,
                 const double* targets, int64_t obs_every, int checkpoint_every, double* loss,
                 double* grad_manning, double* grad_bathy, int where, double* dts_out) {
    if (!m || nsteps < 1 || !(cfl > 0.0) || !gauge_cells || n_gauges < 1 || !targets || !loss ||
        (where != SWE_HOST && where != SWE_DEVICE) || checkpoint_every < 0 || obs_every < 1 ||
        nsteps % obs_every != 0) {
        set_error("swe_adjoint: bad arguments");
        return SWE_EINVAL;
    }
    const int64_t n_obs = nsteps / obs_every;
    if (m->cfg.precision != SWE_FP64) { set_error("swe_adjoint: the adjoint runs on FP64 meshes"); return SWE_EINVAL; }
    if (!m->have_state) { set_error("swe_adjoint: no state set"); return SWE_EINVAL; }
    const int64_t n = m->hm.n_cells;
    std::vector<long long> gint(n_gauges);
    for (int k = 0; k < n_gauges; ++k) {
        if (gauge_cells[k] < 0 || gauge_cells[k] >= n) { set_error("swe_adjoint: gauge cell out of range"); return SWE_EINVAL; }
        gint[k] = m->hm.inv[gauge_cells[k]];
    }
    const int K = checkpoint_every > 0 ? checkpoint_every : 50;
    const int64_t nseg = (nsteps + K - 1) / K;
    AdjDeviceGuard dg(m->cfg.device);
    int rc = flush_mesh_bc(m);
    if (rc) return rc;
    cudaStream_t st = m->stream;
    const size_t sb = (size_t)n * sizeof(V4<double>);
    DevBuf ckpt, seg, dtlog, small, lam, aw, nu, gmv, gzv, dg_idx, dtarget, dloss;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](DevBuf& b, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(&b.p, bytes ? bytes : 16);
    };
    alloc(ckpt, nseg * sb);
    alloc(seg, (size_t)K * sb);
    alloc(dtlog, nsteps * sizeof(double));
    alloc(small, kSmallWords * sizeof(unsigned long long));
    alloc(lam, sb);
    alloc(aw, sb);
    alloc(nu, sb);
    alloc(gmv, n * sizeof(double));
    alloc(gzv, n * sizeof(double));
    alloc(dg_idx, n_gauges * sizeof(long long));
    alloc(dtarget, (size_t)n_obs * n_gauges * sizeof(double));
    alloc(dloss, sizeof(double));
    if (e != cudaSuccess) {
        set_error(std::string("swe_adjoint: device allocation failed: ") + cudaGetErrorString(e));
        return SWE_ENOMEM;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(dloss.p, 0, sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dg_idx.p, gint.data(), n_gauges * sizeof(long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtarget.p, targets, (size_t)n_obs * n_gauges * sizeof(double), cudaMemcpyHostToDevice, st);
    const long long* gi = (const long long*)dg_idx.p;
    const double* tg = (const double*)dtarget.p;
    // forward run: checkpoints every K steps, step sizes logged, loss summed
    // over the observations
    for (int64_t s = 0; s < nsteps && e == cudaSuccess; ++s) {
        void* cur = m->state[m->nstep % 2];
        void* nxt = m->state[(m->nstep + 1) % 2];
        if (s % K == 0) e = cudaMemcpyAsync((char*)ckpt.p + (s / K) * sb, cur, sb, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = launch_step_raw(m, cur, nxt, m->small, m->nstep, cfl, nullptr, (double*)dtlog.p + s, st);
        ++m->nstep;
        m->act_valid = false;   // stepped without the activity bytes
        if (e == cudaSuccess && (s + 1) % obs_every == 0) {
            adj_loss_kernel<<<1, 32, 0, st>>>((const V4<double>*)nxt, gi, tg + ((s + 1) / obs_every - 1) * n_gauges,
                                             n_gauges, (double*)dloss.p);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) return afail(e, "swe_adjoint: forward");
    std::vector<double> dts(nsteps);
    std::vector<unsigned long long> fstat(kSmallWords);
    e = cudaMemcpyAsync(dts.data(), dtlog.p, nsteps * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fstat.data(), m->small, kSmallWords * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return afail(e, "swe_adjoint: forward");
    if (fstat[kSlotStatus] & kStatusNonFinite) { set_error("swe_adjoint: forward run is not finite"); return SWE_ENONFINITE; }
    for (double d : dts)
        if (!std::isfinite(d)) { set_error("swe_adjoint: forward run went dry"); return SWE_EDRY; }
    if (dts_out) std::memcpy(dts_out, dts.data(), nsteps * sizeof(double));
    // lambda^N = d(last observation)/dU^N
    e = cudaMemsetAsync(lam.p, 0, sb, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(gmv.p, 0, n * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(gzv.p, 0, n * sizeof(double), st);
    if (e == cudaSuccess) {
        adj_inject_kernel<<<1, 32, 0, st>>>((const V4<double>*)m->state[m->nstep % 2], gi,
                                           tg + (n_obs - 1) * n_gauges, n_gauges, (V4<double>*)lam.p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) { small_init_kernel<<<1, 32, 0, st>>>((unsigned long long*)small.p); e = cudaGetLastError(); }
    if (e != cudaSuccess) return afail(e, "swe_adjoint: loss");
    AdjArgs a;
    a.geoA = (const V4<double>*)m->geoA;
    a.geoB = (const V4<double>*)m->geoB;
    a.geoR = (const V4<double>*)m->geoR;
    a.topo = m->topo;
    a.gm2 = (const double*)m->gm2;
    a.lam = (V4<double>*)lam.p;
    a.aw = (V4<double>*)aw.p;
    a.nu = (V4<double>*)nu.p;
    a.gm = (double*)gmv.p;
    a.gz = (double*)gzv.p;
    a.n = n;
    a.g = m->cfg.g;
    a.h_dry = m->cfg.h_dry;
    a.hll = m->cfg.flux == SWE_FLUX_HLL ? 1 : 0;
    a.bc = m->bc;
    // with the edge pass, phase 1 takes R's interior fluxes from one evaluation per edge
    const bool edges = m->plain.edges && m->eflux;
    a.eflux = edges ? (const V4<double>*)m->eflux : nullptr;
    a.esrc = edges ? (const double*)m->esrc : nullptr;
    a.eidx = edges ? m->eidx : nullptr;
    StepArgs<double> ea{};
    if (edges) {
        ea.ecells = m->ecells;
        ea.eln = (const double*)m->eln;
        ea.erl = (const double*)m->erl;
        ea.eflux = (V4<double>*)m->eflux;
        ea.esrc = (double*)m->esrc;
        ea.n_edges = m->n_edges;
        ea.g = m->cfg.g;
        ea.h_dry = m->cfg.h_dry;
        ea.hll = a.hll;
    }
    const unsigned grid = (unsigned)((n + 127) / 128);
    // reverse sweep, segment by segment
    for (int64_t sgi = nseg - 1; sgi >= 0 && e == cudaSuccess; --sgi) {
        const int64_t n0 = sgi * K, n1 = std::min<int64_t>(n0 + K, nsteps);
        char* segp = (char*)seg.p;
        e = cudaMemcpyAsync(segp, (char*)ckpt.p + sgi * sb, sb, cudaMemcpyDeviceToDevice, st);
        for (int64_t k = 0; k + 1 < n1 - n0 && e == cudaSuccess; ++k)
            e = launch_step_raw(m, segp + k * sb, segp + (k + 1) * sb, (unsigned long long*)small.p, k, cfl,
                                (const double*)dtlog.p + n0 + k, nullptr, st);
        for (int64_t k = n1 - n0 - 1; k >= 0 && e == cudaSuccess; --k) {
            a.U = (const V4<double>*)(segp + k * sb);
            a.dt = dts[n0 + k];
            if (edges) {
                ea.s_in = a.U;
                e = Launch<double>::edge_flux(ea, st);
                if (e != cudaSuccess) break;
                adj_phase1_kernel<true><<<grid, 128, 0, st>>>(a);
            } else {
                adj_phase1_kernel<false><<<grid, 128, 0, st>>>(a);
            }
            adj_phase2_kernel<<<grid, 128, 0, st>>>(a);
            const int64_t nn = n0 + k;  // lambda now holds lambda^nn
            if (nn > 0 && nn % obs_every == 0)
                adj_inject_kernel<<<1, 32, 0, st>>>(a.U, gi, tg + (nn / obs_every - 1) * n_gauges, n_gauges, a.lam);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) return afail(e, "swe_adjoint: reverse sweep");
    // outputs
    if (where == SWE_DEVICE) {
        adj_output_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const double*)gmv.p, (const double*)gzv.p,
                                                                       (const double*)m->gm2, m->perm, m->cfg.g,
                                                                       grad_manning, grad_bathy, n);
        e = cudaGetLastError();
    } else {
        DevBuf om, oz;
        alloc(om, n * sizeof(double));
        alloc(oz, n * sizeof(double));
        if (e == cudaSuccess) {
            adj_output_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const double*)gmv.p, (const double*)gzv.p,
                                                                           (const double*)m->gm2, m->perm, m->cfg.g,
                                                                           (double*)om.p, (double*)oz.p, n);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && grad_manning)
            e = cudaMemcpyAsync(grad_manning, om.p, n * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && grad_bathy)
            e = cudaMemcpyAsync(grad_bathy, oz.p, n * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, dloss.p, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return afail(e, "swe_adjoint: output");
    return SWE_OK;
}

}  // namespace

extern "C" {

int swe_adjoint(swe_mesh* m, int64_t nsteps, double cfl, const int32_t* gauge_cells, int n_gauges,
                const double* target_h, int checkpoint_every, double* loss, double* grad_manning,
                double* grad_bathy, int where, double* dts_out) {
    NvtxRange nvtx_range("swe_adjoint");
    return adjoint_impl(m, nsteps, cfl, gauge_cells, n_gauges, target_h, nsteps, checkpoint_every, loss,
                        grad_manning, grad_bathy, where, dts_out);
}

int swe_adjoint_series(swe_mesh* m, int64_t nsteps, double cfl, const int32_t* gauge_cells, int n_gauges,
                       const double* targets, int64_t obs_every, int checkpoint_every, double* loss,
                       double* grad_manning, double* grad_bathy, int where, double* dts_out) {
    NvtxRange nvtx_range("swe_adjoint_series");
    return adjoint_impl(m, nsteps, cfl, gauge_cells, n_gauges, targets, obs_every, checkpoint_every, loss,
                        grad_manning, grad_bathy, where, dts_out);
}

int swe_step_dt(swe_mesh* m, int64_t nsteps, const double* dts, double* t_out) {
    NvtxRange nvtx_range("swe_step_dt");
    if (!m || nsteps < 0 || (nsteps > 0 && !dts)) { set_error("swe_step_dt: bad arguments"); return SWE_EINVAL; }
    if (!m->have_state) { set_error("swe_step_dt: no state set"); return SWE_EINVAL; }
    for (int64_t s = 0; s < nsteps; ++s)
        if (!(dts[s] > 0.0) || !std::isfinite(dts[s])) { set_error("swe_step_dt: step sizes must be > 0"); return SWE_EINVAL; }
    AdjDeviceGuard dg(m->cfg.device);
    int rc = flush_mesh_bc(m);
    if (rc) return rc;
    cudaStream_t st = m->stream;
    DevBuf d;
    cudaError_t e = cudaMalloc(&d.p, (nsteps ? nsteps : 1) * sizeof(double));
    if (e == cudaSuccess && nsteps)
        e = cudaMemcpyAsync(d.p, dts, nsteps * sizeof(double), cudaMemcpyHostToDevice, st);
    for (int64_t s = 0; s < nsteps && e == cudaSuccess; ++s) {
        e = launch_step_raw(m, m->state[m->nstep % 2], m->state[(m->nstep + 1) % 2], m->small, m->nstep, 1.0,
                            (const double*)d.p + s, (double*)(m->small + kSlotDtLast), st);
        ++m->nstep;
        m->act_valid = false;   // stepped without the activity bytes
    }
    unsigned long long sm[kSmallWords];
    if (e == cudaSuccess) e = cudaMemcpyAsync(sm, m->small, sizeof sm, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return afail(e, "swe_step_dt");
    if (t_out) std::memcpy(t_out, &sm[kSlotT], sizeof(double));
    if (sm[kSlotStatus] & kStatusNonFinite) { set_error("swe_step_dt: non-finite state"); return SWE_ENONFINITE; }
    return SWE_OK;
}

int swe_set_fields(swe_mesh* m, const double* bathy, const double* manning) {
    if (!m) { set_error("swe_set_fields: NULL mesh"); return SWE_EINVAL; }
    const int64_t n = m->hm.n_cells;
    if (manning)
        for (int64_t c = 0; c < n; ++c)
            if (!(manning[c] >= 0.0) || !std::isfinite(manning[c])) {
                set_error("swe_set_fields: negative or non-finite Manning coefficient");
                return SWE_EINVAL;
            }
    if (bathy)
        for (int64_t c = 0; c < n; ++c)
            if (!std::isfinite(bathy[c])) { set_error("swe_set_fields: non-finite bed"); return SWE_EINVAL; }
    AdjDeviceGuard dg(m->cfg.device);
    cudaStream_t st = m->stream;
    cudaError_t e = cudaStreamSynchronize(st);
    for (int64_t c = 0; c < n; ++c) {
        const int64_t o = m->hm.perm[c];
        if (bathy) m->hm.z[c] = bathy[o];
        if (manning) m->hm.m[c] = manning[o];
    }
    const bool f32 = m->cfg.precision == SWE_FP32;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (e == cudaSuccess && bathy) {
        if (f32) {
            std::vector<float> zt(n);
            for (int64_t c = 0; c < n; ++c) zt[c] = (float)m->hm.z[c];
            e = cudaMemcpy(m->zdev, zt.data(), n * sizeof(float), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) {
                set_z_kernel<float><<<grid, 256, 0, st>>>((V4<float>*)m->state[0], (V4<float>*)m->state[1],
                                                         (const float*)m->zdev, n);
                e = cudaGetLastError();
            }
        } else {
            e = cudaMemcpy(m->zdev, m->hm.z.data(), n * sizeof(double), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) {
                set_z_kernel<double><<<grid, 256, 0, st>>>((V4<double>*)m->state[0], (V4<double>*)m->state[1],
                                                          (const double*)m->zdev, n);
                e = cudaGetLastError();
            }
        }
    }
    if (e == cudaSuccess && manning) {
        if (f32) {
            std::vector<float> g(n);
            for (int64_t c = 0; c < n; ++c) g[c] = (float)(m->cfg.g * m->hm.m[c] * m->hm.m[c]);
            e = cudaMemcpy(m->gm2, g.data(), n * sizeof(float), cudaMemcpyHostToDevice);
            m->topo_dirty = true;  // topo.w carries g m^2 in FP32
        } else {
            std::vector<double> g(n);
            for (int64_t c = 0; c < n; ++c) g[c] = m->cfg.g * m->hm.m[c] * m->hm.m[c];
            e = cudaMemcpy(m->gm2, g.data(), n * sizeof(double), cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return afail(e, "swe_set_fields");
    return flush_mesh_bc(m);
}

}  // extern "C"
