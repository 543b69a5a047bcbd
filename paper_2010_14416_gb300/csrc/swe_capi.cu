// swe_capi.cu -- the C ABI of libswe (declared in include/swe.h).
//
// Device layout of one mesh (n cells, precision T, internal locality order):
//   state[2]  V4<T>[n]   (h, hu, hv, z) ping-pong pair
//   geoA      V4<T>[n]   L n of edges 0 and 1
//   geoB      V4<T>[n]   L n of edge 2, 1/|Omega|, inscribed radius
//   topo      int4[n]    neighbour codes
//   gm2       T[n]       g m^2
//   perm      int64[n]   internal -> caller index
//   small     u64[8]     dt slots 0..2 (double bits), t, status, clamp count
// Step n reads state[n % 2] and dt slot n % 3, writes state[(n+1) % 2] and
// slot (n+1) % 3, and clears slot (n+2) % 3, so a graph of a multiple of six
// steps replays from any step index that is a multiple of six.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "swe_internal.h"

namespace swe {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

namespace {

constexpr int kDefaultGraphSteps = 48;

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return SWE_ECUDA;
}

__global__ void init_small_kernel(unsigned long long* small, double t) {
    if (threadIdx.x == 0) {
        small[0] = kInfBits; small[1] = kInfBits; small[2] = kInfBits;
        small[kSlotT] = (unsigned long long)__double_as_longlong(t);
        small[kSlotStatus] = 0ULL;
        small[kSlotClamp] = 0ULL;
        small[6] = 0ULL; small[7] = 0ULL;
    }
}

}  // namespace
}  // namespace swe

using namespace swe;


namespace {

int dev_alloc(swe_mesh* m, void** p, size_t bytes, const char* what) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error(std::string("device allocation failed for ") + what + ": " + cudaGetErrorString(e));
        return SWE_ENOMEM;
    }
    m->device_bytes += (int64_t)bytes;
    return SWE_OK;
}

void drop_graph(swe_mesh* m) {
    if (m->graph) cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
    m->graph_len = 0;
    m->graph_cfl = -1.0;
}

// topo[c] = (neighbour codes, and for FP32 the bits of g m^2 in .w)
std::vector<int4> make_topo(const swe_mesh* m) {
    const HostMesh& H = m->hm;
    const int64_t n = H.n_cells;
    std::vector<int4> topo(n);
    for (int64_t c = 0; c < n; ++c) {
        int w = 0;
        if (m->esz == 4) {
            const float gm2 = (float)(m->cfg.g * H.m[c] * H.m[c]);
            std::memcpy(&w, &gm2, sizeof w);
        }
        // static activity: an inflow or fixed-stage edge keeps the cell out of the quiet path
        bool fixed = false;
        for (int j = 0; j < 3; ++j) {
            const int32_t code = H.code[3 * c + j];
            if (code < 0) {
                const int kind = m->bc.kind[-1 - code];
                fixed = fixed || kind == kBcInflow || kind == kBcStage;
            }
        }
        if (fixed) w |= kStaticBit;
        topo[c] = make_int4(H.code[3 * c], H.code[3 * c + 1], H.code[3 * c + 2], w);
    }
    return topo;
}

template <typename T>
int upload_static(swe_mesh* m) {
    const HostMesh& H = m->hm;
    const int64_t n = H.n_cells;
    if (sizeof(T) == 8) {
        std::vector<V4<double>> R(n);
        for (int64_t c = 0; c < n; ++c) {
            R[c].x = host_edge_rl(H.ln[6 * c + 0], H.ln[6 * c + 1]);
            R[c].y = host_edge_rl(H.ln[6 * c + 2], H.ln[6 * c + 3]);
            R[c].z = host_edge_rl(H.ln[6 * c + 4], H.ln[6 * c + 5]);
            R[c].w = 0.0;
        }
        cudaError_t e = cudaMemcpy(m->geoR, R.data(), n * sizeof(V4<double>), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "swe_mesh_create: upload");
    }
    std::vector<V4<T>> A(n), B(n);
    std::vector<T> gm2(n), zt(n);
    const std::vector<int4> topo = make_topo(m);
    for (int64_t c = 0; c < n; ++c) {
        A[c].x = (T)H.ln[6 * c + 0]; A[c].y = (T)H.ln[6 * c + 1];
        A[c].z = (T)H.ln[6 * c + 2]; A[c].w = (T)H.ln[6 * c + 3];
        B[c].x = (T)H.ln[6 * c + 4]; B[c].y = (T)H.ln[6 * c + 5];
        B[c].z = (T)H.inv_area[c]; B[c].w = (T)H.rin[c];
        gm2[c] = (T)(m->cfg.g * H.m[c] * H.m[c]);
        zt[c] = (T)H.z[c];
    }
    cudaError_t e;
    if ((e = cudaMemcpy(m->geoA, A.data(), n * sizeof(V4<T>), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->geoB, B.data(), n * sizeof(V4<T>), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->gm2, gm2.data(), n * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->zdev, zt.data(), n * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->topo, topo.data(), n * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->perm, H.perm.data(), n * sizeof(long long), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "swe_mesh_create: upload");
    return SWE_OK;
}

int flush_topo(swe_mesh* m) {
    if (!m->topo_dirty) return SWE_OK;
    const int64_t n = m->hm.n_cells;
    const std::vector<int4> topo = make_topo(m);
    cudaError_t e = cudaMemcpyAsync(m->topo, topo.data(), n * sizeof(int4), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "swe_set_bc: upload");
    for (int gI = 0; gI < m->n_groups; ++gI) {
        if (m->bc.kind[gI] == kBcInflow)
            m->bc.value[gI] = m->group_len[gI] > 0.0 ? m->group_value[gI] / m->group_len[gI] : 0.0;
        else
            m->bc.value[gI] = m->group_value[gI];
    }
    m->topo_dirty = false;
    m->act_valid = false;   // static activity may have changed
    drop_graph(m);
    return SWE_OK;
}

template <typename T>
StepArgs<T> make_args(swe_mesh* m, int64_t step_index, double cfl) {
    StepArgs<T> a;
    const int p2 = (int)(step_index % 2), p3 = (int)(step_index % 3);
    a.s_in = (const V4<T>*)m->state[p2];
    a.s_out = (V4<T>*)m->state[1 - p2];
    a.geoA = (const V4<T>*)m->geoA;
    a.geoB = (const V4<T>*)m->geoB;
    a.geoR = (const V4<T>*)m->geoR;
    a.topo = m->topo;
    a.gm2 = (const T*)m->gm2;
    a.dt_read = (const double*)(m->small + p3);
    a.dt_write = m->small + (p3 + 1) % 3;
    a.dt_reset = m->small + (p3 + 2) % 3;
    a.t = (double*)(m->small + kSlotT);
    a.status = (unsigned*)(m->small + kSlotStatus);
    a.n_clamped = m->small + kSlotClamp;
    a.n_active = m->small + kSlotActive;
    a.n = m->hm.n_cells;
    a.grid = m->grid;
    a.cfl = cfl;
    a.hll = m->cfg.flux == SWE_FLUX_HLL ? 1 : 0;
    a.dt_fixed = nullptr;
    a.dt_log = (double*)(m->small + kSlotDtLast);  // size of the last step, for diagnostics
    a.ecells = nullptr;
    a.eln = nullptr;
    a.erl = (const T*)m->erl;
    a.eflux = nullptr;
    a.esrc = nullptr;
    a.eidx = nullptr;
    a.n_edges = 0;
    if (m->cfg.edge_pass && m->eflux) {
        a.ecells = m->ecells;
        a.eln = (const T*)m->eln;
        a.eflux = (V4<T>*)m->eflux;
        a.esrc = (T*)m->esrc;
        a.eidx = m->eidx;
        a.n_edges = m->n_edges;
    }
    a.act_in = nullptr;
    a.act_next = nullptr;
    a.act_clear = nullptr;
    if (m->cfg.activity && m->act[0]) {
        a.act_in = m->act[p3];
        a.act_next = m->act[(p3 + 1) % 3];
        a.act_clear = m->act[(p3 + 2) % 3];
    }
    a.g = (T)m->cfg.g;
    a.h_dry = (T)m->cfg.h_dry;
    a.bc = m->bc;
    a.debug = m->cfg.debug_checks;
    a.n_groups = m->n_groups;
    return a;
}

template <typename T>
cudaError_t launch_one(swe_mesh* m, int64_t step_index, double cfl, cudaStream_t st) {
    if (m->cfg.cell_pairs)
        return Launch<T>::step_pair(make_args<T>(m, step_index, cfl), m->cfg.block_size, m->cfg.min_blocks,
                                    m->cfg.geometry_early, m->cfg.stages, st);
    return Launch<T>::step(make_args<T>(m, step_index, cfl), m->cfg.block_size, m->cfg.min_blocks,
                           m->cfg.stages, m->cfg.geometry_early, st);
}

template <typename T>
int capture_graph(swe_mesh* m, int len, double cfl) {
    drop_graph(m);
    cudaError_t e = cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "swe_step: begin capture");
    cudaError_t le = cudaSuccess;
    for (int s = 0; s < len && le == cudaSuccess; ++s) le = launch_one<T>(m, s, cfl, m->cap_stream);
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(m->cap_stream, &gr);
    if (le != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return cuda_fail(le, "swe_step: capture launch"); }
    if (e != cudaSuccess) return cuda_fail(e, "swe_step: end capture");
    e = cudaGraphInstantiate(&m->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) { m->graph = nullptr; return cuda_fail(e, "swe_step: instantiate"); }
    m->graph_len = len;
    m->graph_cfl = cfl;
    return SWE_OK;
}

template <typename T>
int run_steps(swe_mesh* m, int64_t nsteps, double cfl) {
    if (m->cfg.activity) {
        if (!m->act_valid) {
            int rc = init_activity(m);
            if (rc) return rc;
        }
    } else {
        m->act_valid = false;   // steps without activity bytes do not maintain them
    }
    int64_t left = nsteps;
    const int gsteps = m->cfg.graph_steps;
    // singles until the step index is a multiple of six
    while (left > 0 && (m->nstep % 6 != 0 || gsteps <= 0 || left < gsteps)) {
        cudaError_t e = launch_one<T>(m, m->nstep, cfl, m->stream);
        if (e != cudaSuccess) return cuda_fail(e, "swe_step: launch");
        ++m->nstep;
        --left;
        if (m->nstep % 6 == 0 && gsteps > 0 && left >= gsteps) break;
    }
    if (left >= gsteps && gsteps > 0) {
        if (!m->graph || m->graph_len != gsteps || m->graph_cfl != cfl) {
            int rc = capture_graph<T>(m, gsteps, cfl);
            if (rc) return rc;
        }
        while (left >= gsteps) {
            cudaError_t e = cudaGraphLaunch(m->graph, m->stream);
            if (e != cudaSuccess) return cuda_fail(e, "swe_step: graph launch");
            m->nstep += gsteps;
            left -= gsteps;
        }
    }
    while (left > 0) {
        cudaError_t e = launch_one<T>(m, m->nstep, cfl, m->stream);
        if (e != cudaSuccess) return cuda_fail(e, "swe_step: launch");
        ++m->nstep;
        --left;
    }
    return SWE_OK;
}

int read_small(swe_mesh* m, unsigned long long out[kSmallWords]) {
    cudaError_t e = cudaMemcpyAsync(out, m->small, sizeof(unsigned long long) * kSmallWords,
                                    cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "swe: reading the status block");
    return SWE_OK;
}

int status_code(unsigned long long st) {
    if (st & kStatusBadIndex) {
        set_error("swe_step: a neighbour index, edge index or boundary group out of range (debug checks)");
        return SWE_EMESH;
    }
    if (st & kStatusNonFinite) { set_error("swe_step: non-finite state"); return SWE_ENONFINITE; }
    if (st & kStatusDry) { set_error("swe_step: every cell is dry, no CFL time step"); return SWE_EDRY; }
    return SWE_OK;
}

double bits_to_double(unsigned long long b) {
    double d;
    std::memcpy(&d, &b, sizeof d);
    return d;
}

int ensure_stage(swe_mesh* m) {
    for (int k = 0; k < 3; ++k) {
        if (!m->stage[k]) {
            int rc = dev_alloc(m, &m->stage[k], m->hm.n_cells * m->esz, "staging");
            if (rc) return rc;
        }
    }
    return SWE_OK;
}

template <typename T>
int set_state_t(swe_mesh* m, const void* h, const void* hu, const void* hv, int where, double t) {
    const int64_t n = m->hm.n_cells;
    const T* src[3] = {(const T*)h, (const T*)hu, (const T*)hv};
    cudaError_t e;
    if (where == SWE_HOST) {
        int rc = ensure_stage(m);
        if (rc) return rc;
        for (int k = 0; k < 3; ++k) {
            e = cudaMemcpyAsync(m->stage[k], src[k], n * sizeof(T), cudaMemcpyHostToDevice, m->stream);
            if (e != cudaSuccess) return cuda_fail(e, "swe_set_state: copy");
            src[k] = (const T*)m->stage[k];
        }
    }
    // z rides in the state record (copied from the static z array)
    e = Launch<T>::pack(src[0], src[1], src[2], m->perm, (const T*)m->zdev, (V4<T>*)m->state[0], n, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->state[1], m->state[0], n * sizeof(V4<T>),
                                              cudaMemcpyDeviceToDevice, m->stream);
    if (e == cudaSuccess) { init_small_kernel<<<1, 32, 0, m->stream>>>(m->small, t); e = cudaGetLastError(); }
    if (e == cudaSuccess)
        e = Launch<T>::dt((const V4<T>*)m->state[0], (const V4<T>*)m->geoB, n, (T)m->cfg.g, (T)m->cfg.h_dry,
                          m->small + 0, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "swe_set_state");
    m->have_state = true;
    m->nstep = 0;
    m->act_valid = false;
    return SWE_OK;
}

template <typename T>
int get_state_t(swe_mesh* m, void* h, void* hu, void* hv, int where) {
    const int64_t n = m->hm.n_cells;
    const V4<T>* cur = (const V4<T>*)m->state[m->nstep % 2];
    cudaError_t e;
    if (where == SWE_DEVICE) {
        e = Launch<T>::unpack(cur, m->perm, (T*)h, (T*)hu, (T*)hv, n, m->stream);
        if (e != cudaSuccess) return cuda_fail(e, "swe_get_state");
        return SWE_OK;
    }
    int rc = ensure_stage(m);
    if (rc) return rc;
    e = Launch<T>::unpack(cur, m->perm, (T*)m->stage[0], (T*)m->stage[1], (T*)m->stage[2], n, m->stream);
    void* dst[3] = {h, hu, hv};
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(dst[k], m->stage[k], n * sizeof(T), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "swe_get_state");
    return SWE_OK;
}

}  // namespace

namespace swe {

template <typename T>
cudaError_t launch_raw_t(swe_mesh* m, const void* in, void* out, unsigned long long* small, int64_t step_index,
                         double cfl, const double* dt_fixed, double* dt_log, cudaStream_t st, bool with_activity,
                         void* eflux_out, void* esrc_out) {
    StepArgs<T> a = make_args<T>(m, step_index, cfl);
    a.s_in = (const V4<T>*)in;
    a.s_out = (V4<T>*)out;
    const int p3 = (int)(step_index % 3);
    a.dt_read = (const double*)(small + p3);
    a.dt_write = small + (p3 + 1) % 3;
    a.dt_reset = small + (p3 + 2) % 3;
    a.t = (double*)(small + kSlotT);
    a.status = (unsigned*)(small + kSlotStatus);
    a.n_clamped = small + kSlotClamp;
    a.n_active = small + kSlotActive;
    a.dt_fixed = dt_fixed;
    a.dt_log = dt_log;
    if (with_activity && a.act_in)
        return Launch<T>::step(a, m->cfg.block_size, m->cfg.min_blocks, m->cfg.stages, m->cfg.geometry_early, st);
    a.act_in = nullptr;
    a.act_next = nullptr;
    a.act_clear = nullptr;
    const bool edges = m->plain.edges && m->eflux;
    a.ecells = edges ? m->ecells : nullptr;
    a.eln = edges ? (const T*)m->eln : nullptr;
    a.eflux = edges ? (V4<T>*)(eflux_out ? eflux_out : m->eflux) : nullptr;
    a.esrc = edges ? (T*)(esrc_out ? esrc_out : m->esrc) : nullptr;
    a.eidx = edges ? m->eidx : nullptr;
    a.n_edges = edges ? m->n_edges : 0;
    a.grid = m->plain.grid;
    if (m->plain.pairs)
        return Launch<T>::step_pair(a, m->plain.block, m->plain.min_blocks, m->plain.geo, m->plain.stages, st);
    return Launch<T>::step(a, m->plain.block, m->plain.min_blocks, m->plain.stages, m->plain.geo, st);
}

// One step of mesh m from buffer `in` to buffer `out` with the given status
// block and step index (dt slot rotation), taking dt from *dt_fixed when set.
cudaError_t launch_step_raw(swe_mesh* m, const void* in, void* out, unsigned long long* small, int64_t step_index,
                            double cfl, const double* dt_fixed, double* dt_log, cudaStream_t st, bool with_activity,
                            void* eflux_out, void* esrc_out) {
    return m->cfg.precision == SWE_FP32
               ? launch_raw_t<float>(m, in, out, small, step_index, cfl, dt_fixed, dt_log, st, with_activity,
                                     eflux_out, esrc_out)
               : launch_raw_t<double>(m, in, out, small, step_index, cfl, dt_fixed, dt_log, st, with_activity,
                                      eflux_out, esrc_out);
}

double host_edge_rl(double lx, double ly) { return 1.0 / std::sqrt(std::fma(lx, lx, ly * ly)); }

void append_edges(const HostMesh& H, int64_t base, std::vector<int2>& cells, std::vector<double>& ln, int4* eidx,
                  std::vector<double>* rl) {
    const int64_t n = H.n_cells;
    for (int64_t c = 0; c < n; ++c) eidx[c] = make_int4(-1, -1, -1, 0);
    for (int64_t c = 0; c < n; ++c)
        for (int j = 0; j < 3; ++j) {
            const int32_t code = H.code[3 * c + j];
            if (code >= 0 && !(code & kFlipBit)) {
                const int e = (int)cells.size();
                const int k = code & kNbrMask;
                cells.push_back(make_int2((int)(base + c), (int)(base + k)));
                ln.push_back(H.ln[6 * c + 2 * j]);
                ln.push_back(H.ln[6 * c + 2 * j + 1]);
                if (rl) rl->push_back(host_edge_rl(H.ln[6 * c + 2 * j], H.ln[6 * c + 2 * j + 1]));
                (j == 0 ? eidx[c].x : (j == 1 ? eidx[c].y : eidx[c].z)) = e;
                for (int jk = 0; jk < 3; ++jk)
                    if ((H.code[3 * k + jk] & kNbrMask) == (int32_t)c && H.code[3 * k + jk] >= 0)
                        (jk == 0 ? eidx[k].x : (jk == 1 ? eidx[k].y : eidx[k].z)) = e;
            }
        }
}

int build_edges(swe_mesh* m) {
    if (m->eflux) return SWE_OK;
    const HostMesh& H = m->hm;
    const int64_t n = H.n_cells;
    std::vector<int2> cells;
    std::vector<double> ln, rl;
    std::vector<int4> eidx(n);
    cells.reserve(3 * n / 2 + 1);
    ln.reserve(3 * n + 2);
    append_edges(H, 0, cells, ln, eidx.data(), m->esz == 8 ? &rl : nullptr);
    const int64_t E = (int64_t)cells.size();
    const size_t esz = m->esz;
    std::vector<char> lnt(2 * E * esz);
    for (int64_t q = 0; q < 2 * E; ++q) {
        if (esz == 4) { const float v = (float)ln[q]; std::memcpy(&lnt[q * 4], &v, 4); }
        else std::memcpy(&lnt[q * 8], &ln[q], 8);
    }
    const size_t Eb = (size_t)std::max<int64_t>(E, 1);
    cudaError_t e = cudaMalloc((void**)&m->ecells, Eb * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&m->eln, 2 * Eb * esz);
    if (e == cudaSuccess) e = cudaMalloc(&m->eflux, Eb * 4 * esz);
    if (e == cudaSuccess) e = cudaMalloc(&m->esrc, Eb * esz);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->eidx, (size_t)n * sizeof(int4));
    if (e == cudaSuccess && esz == 8) e = cudaMalloc(&m->erl, Eb * esz);
    if (e != cudaSuccess) {
        void* bufs[] = {m->ecells, m->eln, m->eflux, m->esrc, m->eidx, m->erl};
        for (void* b : bufs)
            if (b) cudaFree(b);
        m->ecells = nullptr; m->eln = nullptr; m->eflux = nullptr; m->esrc = nullptr; m->eidx = nullptr;
        m->erl = nullptr;
        set_error("edge pass: device allocation failed");
        return SWE_ENOMEM;
    }
    if (E) e = cudaMemcpy(m->ecells, cells.data(), E * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && E) e = cudaMemcpy(m->eln, lnt.data(), 2 * E * esz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->eidx, eidx.data(), n * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && esz == 8 && E) e = cudaMemcpy(m->erl, rl.data(), E * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "edge pass: upload");
    m->n_edges = E;
    m->device_bytes += (int64_t)(Eb * (sizeof(int2) + 7 * esz) + n * sizeof(int4));
    return SWE_OK;
}

int init_activity(swe_mesh* m) {
    const int64_t n = m->hm.n_cells;
    cudaError_t e = cudaSuccess;
    if (!m->act[0]) {
        const int64_t len = (n + 31) / 32 * 32 + 32;
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            e = cudaMalloc((void**)&m->act[k], len);
            if (e == cudaSuccess) e = cudaMemsetAsync(m->act[k], 0, len, m->stream);
        }
        if (e != cudaSuccess) {
            for (auto& p : m->act) {
                if (p) cudaFree(p);
                p = nullptr;
            }
            set_error("activity bytes: device allocation failed");
            return SWE_ENOMEM;
        }
        m->act_len = len;
        m->device_bytes += 3 * len;
    }
    const int p3 = (int)(m->nstep % 3);
    e = cudaMemsetAsync(m->act[p3], 2, m->act_len, m->stream);   // bit 1: rebuilt (act_init_kernel)
    if (e == cudaSuccess) e = cudaMemsetAsync(m->act[(p3 + 1) % 3], 0, m->act_len, m->stream);
    // the previous step's bytes: all 1, so the next step writes every cell's
    // state (its output buffer holds no step's result yet)
    if (e == cudaSuccess) e = cudaMemsetAsync(m->act[(p3 + 2) % 3], 1, m->act_len, m->stream);
    if (e == cudaSuccess)
        e = m->cfg.precision == SWE_FP32
                ? Launch<float>::act_init((const V4<float>*)m->state[m->nstep % 2], m->topo, n, (float)m->cfg.h_dry,
                                          m->act[p3], m->stream)
                : Launch<double>::act_init((const V4<double>*)m->state[m->nstep % 2], m->topo, n, m->cfg.h_dry,
                                           m->act[p3], m->stream);
    if (e != cudaSuccess) return cuda_fail(e, "activity bytes: initialisation");
    m->act_valid = true;
    return SWE_OK;
}

int flush_mesh_bc(swe_mesh* m) { return flush_topo(m); }

void drop_mesh_graph(swe_mesh* m) { drop_graph(m); }

}  // namespace swe

extern "C" {

void swe_config_default(swe_config* cfg) {
    if (!cfg) return;
    cfg->precision = SWE_FP64;
    cfg->g = 9.81;
    cfg->h_dry = 1e-6;
    cfg->reorder = SWE_REORDER_HILBERT;
    cfg->block_size = 0;
    cfg->graph_steps = 0;
    cfg->device = 0;
    cfg->min_blocks = 0;
    cfg->stages = 0;
    cfg->geometry_early = 0;
    cfg->activity = 0;
    cfg->edge_pass = 0;
    cfg->grid = 0;
    cfg->debug_checks = 0;
    cfg->cell_pairs = 0;
    cfg->flux = SWE_FLUX_HLLC;
}

const char* swe_last_error(void) { return g_last_error.c_str(); }

int swe_debug_code_ok(int32_t code, int64_t n_cells, int n_groups) {
    return code_ok(code, (long long)n_cells, n_groups) ? 1 : 0;
}

void swe_mesh_destroy(swe_mesh* m) {
    if (!m) return;
    DeviceGuard dg(m->cfg.device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    drop_graph(m);
    void* bufs[] = {m->state[0], m->state[1], m->geoA, m->geoB, m->topo, m->gm2, m->zdev, m->perm,
                    m->stage[0], m->stage[1], m->stage[2], m->small, m->act[0], m->act[1], m->act[2],
                    m->ecells, m->eln, m->eflux, m->esrc, m->eidx, m->geoR, m->erl};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    delete m;
}

int swe_mesh_create(const double* nodes, int64_t n_nodes, const int32_t* tris, int64_t n_tris,
                    const double* bathy, const double* manning, const swe_config* cfg, swe_mesh** out) {
    if (!out) { set_error("swe_mesh_create: out is NULL"); return SWE_EINVAL; }
    *out = nullptr;
    swe_config c;
    swe_config_default(&c);
    if (cfg) c = *cfg;
    if (c.precision != SWE_FP64 && c.precision != SWE_FP32) { set_error("swe_mesh_create: bad precision"); return SWE_EINVAL; }
    if (!(c.g > 0.0) || !(c.h_dry > 0.0) || !std::isfinite(c.g) || !std::isfinite(c.h_dry)) {
        set_error("swe_mesh_create: g and h_dry must be finite and > 0");
        return SWE_EINVAL;
    }
    if (c.h_dry < (double)FLT_MIN) {
        // a wet depth must stay a normal float: FP32 kernels hold it as one, and the
        // FP64 friction term starts its h^(-1/3) iteration from the float reciprocal cube root
        set_error("swe_mesh_create: h_dry must be at least FLT_MIN (1.18e-38)");
        return SWE_EINVAL;
    }
    if (c.flux != SWE_FLUX_HLLC && c.flux != SWE_FLUX_HLL) { set_error("swe_mesh_create: unknown flux"); return SWE_EINVAL; }
    if (c.geometry_early != 0 && c.geometry_early != 1) {
        set_error("swe_mesh_create: geometry_early must be 0 or 1");
        return SWE_EINVAL;
    }
    if (c.activity != 0 && c.activity != 1) {
        set_error("swe_mesh_create: activity must be 0 or 1");
        return SWE_EINVAL;
    }
    if (c.edge_pass != 0 && c.edge_pass != 1) {
        set_error("swe_mesh_create: edge_pass must be 0 or 1");
        return SWE_EINVAL;
    }
    if (c.grid < 0) {
        set_error("swe_mesh_create: grid must be >= 0");
        return SWE_EINVAL;
    }
    if (c.debug_checks != 0 && c.debug_checks != 1) {
        set_error("swe_mesh_create: debug_checks must be 0 or 1");
        return SWE_EINVAL;
    }

    if (c.cell_pairs != 0 && c.cell_pairs != 1) {
        set_error("swe_mesh_create: cell_pairs must be 0 or 1");
        return SWE_EINVAL;
    }
    if (c.cell_pairs && (c.precision != SWE_FP32 || c.activity || c.edge_pass)) {
        set_error("swe_mesh_create: cell_pairs needs FP32, without activity or edge_pass");
        return SWE_EINVAL;
    }
    if (c.edge_pass && c.activity) {
        set_error("swe_mesh_create: edge_pass and activity exclude each other");
        return SWE_EINVAL;
    }
    if (c.block_size == 0) c.block_size = c.precision == SWE_FP32 ? 256 : 128;
    if (c.block_size != 128 && c.block_size != 256 && c.block_size != 512) {
        set_error("swe_mesh_create: block_size must be 128, 256 or 512");
        return SWE_EINVAL;
    }
    if (c.min_blocks == 0)
        c.min_blocks = c.precision == SWE_FP32 ? Launch<float>::default_min_blocks(c.block_size)
                                               : Launch<double>::default_min_blocks(c.block_size);
    if (c.stages == 0) c.stages = (c.precision == SWE_FP32 || c.activity) && !c.cell_pairs ? 3 : 1;
    if (c.graph_steps == 0) c.graph_steps = kDefaultGraphSteps;
    if (c.graph_steps > 0) c.graph_steps = std::max(6, (c.graph_steps / 6) * 6);
    if (c.activity && n_tris >= kActivityMaxCells) {
        set_error("swe_mesh_create: activity needs fewer than 2^29 cells");
        return SWE_EINVAL;
    }
    swe_mesh* m = new (std::nothrow) swe_mesh();
    if (!m) { set_error("swe_mesh_create: out of host memory"); return SWE_ENOMEM; }
    m->cfg = c;
    m->esz = c.precision == SWE_FP32 ? 4 : 8;
    std::string err;
    int rc;
    try {
        rc = build_host_mesh(nodes, n_nodes, tris, n_tris, bathy, manning, c.reorder, c.precision == SWE_FP32, m->hm,
                             err);
    } catch (const std::bad_alloc&) {
        rc = SWE_ENOMEM;
        err = "swe_mesh_create: out of host memory";
    }
    if (rc) { set_error(err); delete m; return rc; }
    DeviceGuard dg(c.device);
    if (!dg.ok) { set_error("swe_mesh_create: cannot select the device"); delete m; return SWE_ECUDA; }
    cudaError_t e = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete m; return cuda_fail(e, "swe_mesh_create: stream"); }
    const int64_t n = n_tris;
    const size_t v4 = 4 * m->esz;
    if ((rc = dev_alloc(m, &m->state[0], n * v4, "state")) || (rc = dev_alloc(m, &m->state[1], n * v4, "state")) ||
        (rc = dev_alloc(m, &m->geoA, n * v4, "geometry")) || (rc = dev_alloc(m, &m->geoB, n * v4, "geometry")) ||
        (c.precision == SWE_FP64 && (rc = dev_alloc(m, &m->geoR, n * v4, "geometry"))) ||
        (rc = dev_alloc(m, (void**)&m->topo, n * sizeof(int4), "topology")) ||
        (rc = dev_alloc(m, &m->gm2, n * m->esz, "manning")) ||
        (rc = dev_alloc(m, &m->zdev, n * m->esz, "bed")) ||
        (rc = dev_alloc(m, (void**)&m->perm, n * sizeof(long long), "permutation")) ||
        (rc = dev_alloc(m, (void**)&m->small, kSmallWords * sizeof(unsigned long long), "status"))) {
        swe_mesh_destroy(m);
        return rc;
    }
    rc = c.precision == SWE_FP32 ? upload_static<float>(m) : upload_static<double>(m);
    if (rc) { swe_mesh_destroy(m); return rc; }
    if (c.edge_pass) {
        rc = build_edges(m);
        if (rc) { swe_mesh_destroy(m); return rc; }
    }
    {
        int per_sm = 0, sms = 0;
        e = c.cell_pairs ? Launch<float>::pair_resident_blocks(c.block_size, c.min_blocks, c.geometry_early, c.stages,
                                                               &per_sm)
            : c.precision == SWE_FP32
                ? Launch<float>::resident_blocks(c.block_size, c.min_blocks, c.stages, c.geometry_early, c.activity,
                                                 c.edge_pass, &per_sm)
                : Launch<double>::resident_blocks(c.block_size, c.min_blocks, c.stages, c.geometry_early, c.activity,
                                                  c.edge_pass, &per_sm);
        if (e == cudaErrorInvalidValue) {
            swe_mesh_destroy(m);
            set_error("swe_mesh_create: no compiled step kernel for this block_size / min_blocks / stages / "
                      "geometry_early / activity / edge_pass / cell_pairs");
            return SWE_EINVAL;
        }
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device);
        if (e != cudaSuccess) { swe_mesh_destroy(m); return cuda_fail(e, "swe_mesh_create: occupancy"); }
        const long long units = c.cell_pairs ? (n + 1) / 2 : n;   // a thread's work item: a cell or a pair
        const long long need = (units + c.block_size - 1) / c.block_size;
        const long long wave = (long long)std::max(per_sm, 1) * std::max(sms, 1);
        m->grid = (unsigned)std::min(need, c.grid > 0 ? (long long)c.grid : wave);
        // launches without activity bytes: the same shape, or the default one
        // when the configured shape exists only as an activity kernel
        m->plain = LaunchShape{c.block_size, c.min_blocks, c.stages, c.geometry_early, c.edge_pass, m->grid,
                               c.cell_pairs};
        if (c.activity) {
            LaunchShape d;
            d.block = c.precision == SWE_FP32 ? 256 : 128;
            d.min_blocks = c.precision == SWE_FP32 ? Launch<float>::default_min_blocks(d.block)
                                                   : Launch<double>::default_min_blocks(d.block);
            d.stages = c.precision == SWE_FP32 ? 3 : 1;
            d.geo = 0;
            int pb = 0;
            e = c.precision == SWE_FP32
                    ? Launch<float>::resident_blocks(d.block, d.min_blocks, d.stages, 0, 0, 0, &pb)
                    : Launch<double>::resident_blocks(d.block, d.min_blocks, d.stages, 0, 0, 0, &pb);
            if (e != cudaSuccess) { swe_mesh_destroy(m); return cuda_fail(e, "swe_mesh_create: occupancy"); }
            d.grid = (unsigned)std::min((long long)((n + d.block - 1) / d.block), (long long)std::max(pb, 1) * std::max(sms, 1));
            m->plain = d;
        }
    }
    m->bc.kind[0] = kBcWall;
    m->bc.value[0] = 0.0;
    m->group_len.assign(1, 0.0);
    m->group_value.assign(1, 0.0);
    for (int64_t s = 0; s < 3 * n; ++s)
        if (m->hm.code[s] < 0) m->group_len[0] += m->hm.len[s];
    *out = m;
    return SWE_OK;
}

int swe_set_bc(swe_mesh* m, const int32_t* pairs, int64_t n, int kind, double value) {
    if (!m || (!pairs && n > 0) || n < 0) { set_error("swe_set_bc: bad arguments"); return SWE_EINVAL; }
    if (kind < SWE_BC_WALL || kind > SWE_BC_STAGE) { set_error("swe_set_bc: unknown kind"); return SWE_EINVAL; }
    if (m->n_groups >= kMaxGroups - 1) { set_error("swe_set_bc: too many boundary groups"); return SWE_EINVAL; }
    if (!std::isfinite(value)) { set_error("swe_set_bc: non-finite value"); return SWE_EINVAL; }
    HostMesh& H = m->hm;
    const int grp = m->n_groups;
    std::vector<int64_t> slots;
    slots.reserve(n);
    for (int64_t e = 0; e < n; ++e) {
        const int32_t a = pairs[2 * e], b = pairs[2 * e + 1];
        const uint64_t key = ((uint64_t)std::min(a, b) << 32) | (uint64_t)std::max(a, b);
        auto it = std::lower_bound(H.bkey.begin(), H.bkey.end(), key);
        if (it == H.bkey.end() || *it != key) {
            set_error("swe_set_bc: node pair " + std::to_string(a) + "," + std::to_string(b) +
                      " is not a boundary edge");
            return SWE_EINVAL;
        }
        slots.push_back(H.bslot[it - H.bkey.begin()]);
    }
    double total = 0.0;
    for (int64_t s : slots) {
        const int old = -1 - H.code[s];
        if (old == grp) continue;
        m->group_len[old] -= H.len[s];
        total += H.len[s];
        H.code[s] = -1 - grp;
    }
    m->group_len.push_back(total);
    m->group_value.push_back(value);
    m->bc.kind[grp] = kind;
    m->n_groups = grp + 1;
    m->topo_dirty = true;
    DeviceGuard dg(m->cfg.device);
    return flush_topo(m);
}

int swe_set_stream(swe_mesh* m, void* stream) {
    if (!m) { set_error("swe_set_stream: NULL mesh"); return SWE_EINVAL; }
    m->stream = (cudaStream_t)stream;
    return SWE_OK;
}

int swe_set_state(swe_mesh* m, const void* h, const void* hu, const void* hv, int where, double t) {
    if (!m || !h || !hu || !hv || (where != SWE_HOST && where != SWE_DEVICE) || !std::isfinite(t)) {
        set_error("swe_set_state: bad arguments");
        return SWE_EINVAL;
    }
    DeviceGuard dg(m->cfg.device);
    int rc = flush_topo(m);
    if (rc) return rc;
    return m->cfg.precision == SWE_FP32 ? set_state_t<float>(m, h, hu, hv, where, t)
                                        : set_state_t<double>(m, h, hu, hv, where, t);
}

int swe_step(swe_mesh* m, int64_t nsteps, double cfl, double* t_out) {
    NvtxRange nvtx_range("swe_step");
    if (!m || nsteps < 0 || !(cfl > 0.0) || !std::isfinite(cfl)) { set_error("swe_step: bad arguments"); return SWE_EINVAL; }
    if (!m->have_state) { set_error("swe_step: no state set"); return SWE_EINVAL; }
    DeviceGuard dg(m->cfg.device);
    int rc = flush_topo(m);
    if (rc) return rc;
    rc = m->cfg.precision == SWE_FP32 ? run_steps<float>(m, nsteps, cfl) : run_steps<double>(m, nsteps, cfl);
    if (rc) return rc;
    if (t_out) {
        unsigned long long s[kSmallWords];
        rc = read_small(m, s);
        if (rc) return rc;
        *t_out = bits_to_double(s[kSlotT]);
        return status_code(s[kSlotStatus]);
    }
    return SWE_OK;
}

int swe_get_state(swe_mesh* m, void* h, void* hu, void* hv, int where) {
    if (!m || !h || !hu || !hv || (where != SWE_HOST && where != SWE_DEVICE)) {
        set_error("swe_get_state: bad arguments");
        return SWE_EINVAL;
    }
    if (!m->have_state) { set_error("swe_get_state: no state set"); return SWE_EINVAL; }
    DeviceGuard dg(m->cfg.device);
    return m->cfg.precision == SWE_FP32 ? get_state_t<float>(m, h, hu, hv, where)
                                        : get_state_t<double>(m, h, hu, hv, where);
}

int swe_synchronize(swe_mesh* m) {
    if (!m) { set_error("swe_synchronize: NULL mesh"); return SWE_EINVAL; }
    DeviceGuard dg(m->cfg.device);
    unsigned long long s[kSmallWords];
    int rc = read_small(m, s);
    if (rc) return rc;
    return status_code(s[kSlotStatus]);
}

int swe_get_info(swe_mesh* m, swe_info* info) {
    if (!m || !info) { set_error("swe_get_info: bad arguments"); return SWE_EINVAL; }
    DeviceGuard dg(m->cfg.device);
    std::memset(info, 0, sizeof *info);
    info->n_cells = m->hm.n_cells;
    info->precision = m->cfg.precision;
    info->device_bytes = m->device_bytes;
    info->n_steps = m->nstep;
    if (!m->have_state) {
        info->dt_next = INFINITY;
        return SWE_OK;
    }
    unsigned long long s[kSmallWords];
    int rc = read_small(m, s);
    if (rc) return rc;
    info->t = bits_to_double(s[kSlotT]);
    // the slot holds min_i R_i / (c_i + |u_i|); the CFL number of the next
    // swe_step call multiplies it
    info->dt_next = bits_to_double(s[m->nstep % 3]);
    info->n_clamped = (int64_t)s[kSlotClamp];
    info->n_active = (int64_t)s[kSlotActive];
    info->status = s[kSlotStatus] & kStatusBadIndex    ? SWE_EMESH
                   : s[kSlotStatus] & kStatusNonFinite ? SWE_ENONFINITE
                   : (s[kSlotStatus] & kStatusDry ? SWE_EDRY : SWE_OK);
    return SWE_OK;
}

int swe_get_permutation(swe_mesh* m, int64_t* perm) {
    if (!m || !perm) { set_error("swe_get_permutation: bad arguments"); return SWE_EINVAL; }
    std::memcpy(perm, m->hm.perm.data(), sizeof(int64_t) * m->hm.n_cells);
    return SWE_OK;
}

int swe_mesh_preprocess(const double* nodes, int64_t n_nodes, const int32_t* tris, int64_t n_tris, int reorder,
                        int precision, int64_t* perm, int32_t* code, double* ln, double* inv_area, double* rin) {
    if (n_tris < 1) { set_error("swe_mesh_preprocess: empty mesh"); return SWE_EINVAL; }
    if (precision != SWE_FP32 && precision != SWE_FP64) { set_error("swe_mesh_preprocess: bad precision"); return SWE_EINVAL; }
    HostMesh H;
    std::string err;
    int rc;
    try {
        std::vector<double> zeros((size_t)n_tris, 0.0);
        rc = build_host_mesh(nodes, n_nodes, tris, n_tris, zeros.data(), zeros.data(), reorder, precision == SWE_FP32, H,
                             err);
    } catch (const std::bad_alloc&) {
        rc = SWE_ENOMEM;
        err = "swe_mesh_preprocess: out of host memory";
    }
    if (rc) { set_error(err); return rc; }
    const size_t n = (size_t)n_tris;
    if (perm) std::memcpy(perm, H.perm.data(), n * sizeof(int64_t));
    if (code) std::memcpy(code, H.code.data(), 3 * n * sizeof(int32_t));
    if (ln) std::memcpy(ln, H.ln.data(), 6 * n * sizeof(double));
    if (inv_area) std::memcpy(inv_area, H.inv_area.data(), n * sizeof(double));
    if (rin) std::memcpy(rin, H.rin.data(), n * sizeof(double));
    return SWE_OK;
}

int swe_riemann_flux(int precision, int64_t n, const void* hL, const void* unL, const void* utL,
                     const void* hR, const void* unR, const void* utR, double g, double h_dry, void* G1,
                     void* G2, void* G3, void* S, void* stream) {
    return swe_riemann_flux_kind(precision, SWE_FLUX_HLLC, n, hL, unL, utL, hR, unR, utR, g, h_dry, G1, G2, G3, S,
                                 stream);
}

int swe_riemann_flux_kind(int precision, int flux, int64_t n, const void* hL, const void* unL, const void* utL,
                          const void* hR, const void* unR, const void* utR, double g, double h_dry, void* G1,
                          void* G2, void* G3, void* S, void* stream) {
    if (flux != SWE_FLUX_HLLC && flux != SWE_FLUX_HLL) { set_error("swe_riemann_flux: unknown flux"); return SWE_EINVAL; }
    const int hll = flux == SWE_FLUX_HLL ? 1 : 0;
    if (n < 0 || (n > 0 && (!hL || !unL || !utL || !hR || !unR || !utR || !G1 || !G2 || !G3))) {
        set_error("swe_riemann_flux: bad arguments");
        return SWE_EINVAL;
    }
    cudaError_t e;
    if (precision == SWE_FP32)
        e = Launch<float>::riemann(n, (const float*)hL, (const float*)unL, (const float*)utL, (const float*)hR,
                                   (const float*)unR, (const float*)utR, (float)g, (float)h_dry, (float*)G1,
                                   (float*)G2, (float*)G3, (float*)S, hll, (cudaStream_t)stream);
    else if (precision == SWE_FP64)
        e = Launch<double>::riemann(n, (const double*)hL, (const double*)unL, (const double*)utL,
                                    (const double*)hR, (const double*)unR, (const double*)utR, g, h_dry,
                                    (double*)G1, (double*)G2, (double*)G3, (double*)S, hll, (cudaStream_t)stream);
    else {
        set_error("swe_riemann_flux: bad precision");
        return SWE_EINVAL;
    }
    if (e != cudaSuccess) return cuda_fail(e, "swe_riemann_flux");
    return SWE_OK;
}

}  // extern "C"
