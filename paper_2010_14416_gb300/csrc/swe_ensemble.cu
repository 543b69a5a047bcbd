// swe_ensemble.cu -- batched ensemble of meshes advanced together
// (swe_ensemble_* in include/swe.h).
//
// The members' device arrays are copied into one concatenated layout, each
// member padded to a whole multiple of kEnsPad cells.  Padding cells are dry
// cells with three wall edges: they take the quiet path and never change.
// Neighbour codes are offset to the concatenated numbering and boundary
// groups to one global table (group 0 = wall).  Every member keeps its own
// status block (dt slots, time, status, clamps) and CFL number, so each member
// takes exactly the steps the plain solver would take on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "swe_internal.h"

using namespace swe;

struct swe_ensemble {
    int precision = SWE_FP64;
    int device = 0;
    size_t esz = 8;
    int n_members = 0;
    double g = 9.81, h_dry = 1e-6;
    int hll = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<int64_t> base, n_cells, first_tile;
    int64_t n_total = 0, n_tiles = 0;    // n_tiles counts kEnsPad-cell spans
    int n_groups = 1;                    // global boundary groups
    int debug = 0;                       // debug checks (any member created with them)
    void* state[2] = {nullptr, nullptr};
    void* geoA = nullptr;
    void* geoB = nullptr;
    void* geoR = nullptr;             // FP64: 1/|L n| of the three edges
    int4* topo = nullptr;
    void* gm2 = nullptr;
    long long* perm = nullptr;        // per member, relative to the member's base
    int* tile_member = nullptr;
    long long* member_first_tile = nullptr;
    double* cfl = nullptr;
    unsigned long long* small = nullptr;
    unsigned long long* n_active = nullptr;
    int* kind = nullptr;
    double* value = nullptr;
    void* stage[3] = {nullptr, nullptr, nullptr};
    int64_t stage_cells = 0;
    // launch shape (autotuned by swe_ensemble_autotune; none changes the results)
    int block = 256, min_blocks = 1, stages = 1, geo_early = 0, chunk_log2 = 5, activity = 0;
    // activity bytes over the concatenated layout (activity mode)
    unsigned char* act[3] = {nullptr, nullptr, nullptr};
    int64_t act_len = 0;
    bool act_valid = false;
    // edge pass (FP64 ensembles): the members' interior edges, concatenated
    int edges = 0;
    int64_t n_edges = 0;
    // dynamic chunks: three rotating per-step counters
    int dynamic = 0;
    // split step (FP32): the members mostly wet at creation come first in the
    // layout (pair_spans kEnsPad-cell spans) and run on the cell-pair kernel,
    // the others on the kernel of the shape above, in the same step
    int split = 0;
    // activity kernel with per-warp queues of the cells that run the flux path
    int queue = 0;
    int64_t pair_spans = 0;
    int pair_minb = 8, pair_geo = 1;
    unsigned pair_grid = 0;
    unsigned* sched = nullptr;
    int2* ecells = nullptr;
    void* eln = nullptr;
    void* erl = nullptr;
    void* eflux = nullptr;
    void* esrc = nullptr;
    int4* eidx = nullptr;
    unsigned grid = 0;
    int64_t nstep = 0;
    std::vector<double> cfl_host;
    // graphs keyed by (start step mod 6, length)
    std::map<std::pair<int, int64_t>, cudaGraphExec_t> graphs;
    int64_t device_bytes = 0;
};

namespace {

int efail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return SWE_ECUDA;
}

struct EnsDeviceGuard {
    int prev = -1;
    explicit EnsDeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~EnsDeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int ens_alloc(swe_ensemble* E, void** p, size_t bytes, const char* what) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error(std::string("swe_ensemble_create: device allocation failed for ") + what);
        return SWE_ENOMEM;
    }
    E->device_bytes += (int64_t)bytes;
    return SWE_OK;
}

void drop_graphs(swe_ensemble* E) {
    for (auto& kv : E->graphs) cudaGraphExecDestroy(kv.second);
    E->graphs.clear();
}

__global__ void ens_init_small_kernel(unsigned long long* small, const unsigned long long* first_slot,
                                      const double* t0, int n_members) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n_members) {
        unsigned long long* s = small + 8 * (long long)k;
        s[0] = first_slot[k];
        s[1] = kInfBits;
        s[2] = kInfBits;
        s[3] = (unsigned long long)__double_as_longlong(t0[k]);
        s[4] = 0ULL; s[5] = 0ULL; s[6] = 0ULL; s[7] = 0ULL;
    }
}

// Cells of a member's state deeper than h_dry (the split step's placement).
template <typename T>
__global__ void count_wet_kernel(const V4<T>* __restrict__ s, long long n, T h_dry, unsigned long long* out) {
    unsigned c = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        c += s[i].x > h_dry ? 1u : 0u;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, (unsigned long long)c);
}

template <typename T>
__global__ void ens_unpack_kernel(const V4<T>* __restrict__ s, const long long* __restrict__ perm, long long base,
                                  T* __restrict__ h, T* __restrict__ hu, T* __restrict__ hv, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const long long o = perm[base + i];
        const V4<T> v = s[base + i];
        h[o] = v.x; hu[o] = v.y; hv[o] = v.z;
    }
}

template <typename T>
EnsArgs<T> ens_args(swe_ensemble* E, int64_t step_index) {
    EnsArgs<T> a;
    const int p2 = (int)(step_index % 2), p3 = (int)(step_index % 3);
    a.s_in = (const V4<T>*)E->state[p2];
    a.s_out = (V4<T>*)E->state[1 - p2];
    a.geoA = (const V4<T>*)E->geoA;
    a.geoB = (const V4<T>*)E->geoB;
    a.geoR = (const V4<T>*)E->geoR;
    a.erl = (const T*)E->erl;
    a.topo = E->topo;
    a.gm2 = (const T*)E->gm2;
    a.tile_member = E->tile_member;
    a.member_first_tile = E->member_first_tile;
    a.cfl = E->cfl;
    a.small = E->small;
    a.kind_ = E->kind;
    a.value_ = E->value;
    a.n_active = E->n_active;
    a.n_total = E->n_total;
    a.cell_lo = 0;
    a.pair_spans = 0;
    a.chunk_log2 = E->chunk_log2;
    a.sched = E->sched;
    a.sched_slot = p3;
    a.sched_reset = (p3 + 2) % 3;
    a.ecells = nullptr;
    a.eln = nullptr;
    a.eflux = nullptr;
    a.esrc = nullptr;
    a.eidx = nullptr;
    a.n_edges = 0;
    if (E->edges && E->eflux) {
        a.ecells = E->ecells;
        a.eln = (const T*)E->eln;
        a.eflux = (V4<T>*)E->eflux;
        a.esrc = (T*)E->esrc;
        a.eidx = E->eidx;
        a.n_edges = E->n_edges;
    }
    a.act_in = nullptr;
    a.act_next = nullptr;
    a.act_clear = nullptr;
    if (E->activity && E->act[0]) {
        a.act_in = E->act[p3];
        a.act_next = E->act[(p3 + 1) % 3];
        a.act_clear = E->act[(p3 + 2) % 3];
    }
    a.slot_read = p3;
    a.slot_write = (p3 + 1) % 3;
    a.slot_reset = (p3 + 2) % 3;
    a.hll = E->hll;
    a.g = (T)9.81;
    a.h_dry = (T)1e-6;
    a.debug = E->debug;
    a.n_groups = E->n_groups;
    return a;
}

struct EnsPhysics {
    double g, h_dry;
};

template <typename T>
cudaError_t ens_launch(swe_ensemble* E, int64_t step_index, const EnsPhysics& ph, cudaStream_t st) {
    EnsArgs<T> a = ens_args<T>(E, step_index);
    a.g = (T)ph.g;
    a.h_dry = (T)ph.h_dry;
    if (E->split && E->pair_spans > 0) {   // the paired members, then the others from cell_lo on
        a.pair_spans = (unsigned)E->pair_spans;
        const cudaError_t e = Launch<T>::ensemble_step_pair(a, E->pair_minb, E->pair_geo, E->pair_grid, st);
        if (e != cudaSuccess) return e;
        a.cell_lo = E->pair_spans * kEnsPad;
    }
    if (a.act_in)
        return Launch<T>::ensemble_step_act(a, E->block, E->min_blocks, E->geo_early, E->grid, st, E->dynamic,
                                            E->queue);
    if (E->dynamic) return Launch<T>::ensemble_step_dyn(a, E->block, E->min_blocks, E->geo_early, E->grid, st);
    return Launch<T>::ensemble_step(a, E->block, E->min_blocks, E->stages, E->geo_early, E->grid, st);
}

// blocks of one resident wave of the given ensemble kernel shape
template <typename T>
cudaError_t ens_wave(swe_ensemble* E, int block, int min_blocks, int stages, int geo_early, long long* wave) {
    int per_sm = 0, sms = 0;
    cudaError_t e = Launch<T>::ensemble_resident_blocks(block, min_blocks, stages, geo_early, &per_sm);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, E->device);
    *wave = (long long)std::max(per_sm, 1) * std::max(sms, 1);
    return e;
}

template <typename T>
int ens_build(swe_ensemble* E, swe_mesh* const* M) {
    const int nm = E->n_members;
    const size_t v4 = sizeof(V4<T>);
    // FP32: the members with at least half their cells wet now come first in
    // the layout (the split step's cell-pair kernel takes them); otherwise the
    // members' order.  The placement changes no member's arithmetic.
    std::vector<int> order(nm);
    std::iota(order.begin(), order.end(), 0);
    std::vector<char> wet_member(nm, 0);
    if (sizeof(T) == 4) {
        unsigned long long* d_cnt = nullptr;
        cudaError_t e = cudaMalloc(&d_cnt, nm * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, nm * sizeof(unsigned long long), E->stream);
        for (int k = 0; k < nm && e == cudaSuccess; ++k) {
            const long long n = M[k]->hm.n_cells;
            const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, 1024);
            count_wet_kernel<T><<<grid, 256, 0, E->stream>>>((const V4<T>*)M[k]->state[M[k]->nstep % 2], n,
                                                              (T)E->h_dry, d_cnt + k);
            e = cudaGetLastError();
        }
        std::vector<unsigned long long> cnt(nm, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cnt.data(), d_cnt, nm * sizeof(unsigned long long), cudaMemcpyDeviceToHost, E->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(E->stream);
        if (d_cnt) cudaFree(d_cnt);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_create: wet cells");
        for (int k = 0; k < nm; ++k) wet_member[k] = 2 * cnt[k] >= (unsigned long long)M[k]->hm.n_cells;
        std::stable_partition(order.begin(), order.end(), [&](int k) { return wet_member[k] != 0; });
    }
    // offsets in layout order, padded to whole tiles
    E->base.resize(nm);
    E->n_cells.resize(nm);
    E->first_tile.resize(nm);
    int64_t off = 0;
    E->pair_spans = 0;
    for (int k : order) {
        E->base[k] = off;
        E->n_cells[k] = M[k]->hm.n_cells;
        E->first_tile[k] = off / kEnsPad;
        off += (M[k]->hm.n_cells + kEnsPad - 1) / kEnsPad * kEnsPad;
        if (wet_member[k]) E->pair_spans = off / kEnsPad;
    }
    E->n_total = off;
    E->n_tiles = off / kEnsPad;
    if (E->n_total >= (int64_t)kNbrMask) { set_error("swe_ensemble_create: too many cells in total"); return SWE_EINVAL; }
    int rc;
    if ((rc = ens_alloc(E, &E->state[0], off * v4, "state")) || (rc = ens_alloc(E, &E->state[1], off * v4, "state")) ||
        (rc = ens_alloc(E, &E->geoA, off * v4, "geometry")) || (rc = ens_alloc(E, &E->geoB, off * v4, "geometry")) ||
        (sizeof(T) == 8 && (rc = ens_alloc(E, &E->geoR, off * v4, "geometry"))) ||
        (rc = ens_alloc(E, (void**)&E->topo, off * sizeof(int4), "topology")) ||
        (rc = ens_alloc(E, &E->gm2, off * sizeof(T), "manning")) ||
        (rc = ens_alloc(E, (void**)&E->perm, off * sizeof(long long), "permutation")) ||
        (rc = ens_alloc(E, (void**)&E->tile_member, E->n_tiles * sizeof(int), "tiles")) ||
        (rc = ens_alloc(E, (void**)&E->member_first_tile, nm * sizeof(long long), "tiles")) ||
        (rc = ens_alloc(E, (void**)&E->cfl, nm * sizeof(double), "cfl")) ||
        (rc = ens_alloc(E, (void**)&E->small, nm * 8 * sizeof(unsigned long long), "status")) ||
        (rc = ens_alloc(E, (void**)&E->n_active, sizeof(unsigned long long), "status")) ||
        (rc = ens_alloc(E, (void**)&E->sched, 3 * sizeof(unsigned), "status")))
        return rc;
    cudaStream_t st = E->stream;
    cudaError_t e = cudaSuccess;
    // zero everything that padding cells read (state, topology filled below)
    for (void* p : {E->state[0], E->state[1], E->geoA, E->geoB, E->geoR, E->gm2})
        if (e == cudaSuccess && p) e = cudaMemsetAsync(p, 0, p == E->gm2 ? off * sizeof(T) : off * v4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(E->n_active, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(E->sched, 0, 3 * sizeof(unsigned), st);
    if (e != cudaSuccess) return efail(e, "swe_ensemble_create: clear");
    // global boundary groups: 0 = wall, then each member's groups
    std::vector<int> kinds{kBcWall};
    std::vector<double> values{0.0};
    std::vector<int> gbase(nm);
    for (int k = 0; k < nm; ++k) {
        gbase[k] = (int)kinds.size();
        for (int gI = 0; gI < M[k]->n_groups; ++gI) {
            kinds.push_back(M[k]->bc.kind[gI]);
            values.push_back(M[k]->bc.value[gI]);
        }
    }
    if ((rc = ens_alloc(E, (void**)&E->kind, kinds.size() * sizeof(int), "boundary groups")) ||
        (rc = ens_alloc(E, (void**)&E->value, values.size() * sizeof(double), "boundary groups")))
        return rc;
    e = cudaMemcpy(E->kind, kinds.data(), kinds.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(E->value, values.data(), values.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return efail(e, "swe_ensemble_create: boundary groups");
    E->n_groups = (int)kinds.size();
    for (int k = 0; k < nm; ++k) E->debug = E->debug || M[k]->cfg.debug_checks;
    // per-member device copies and host-built topology / tile tables
    std::vector<int4> topo(off);
    std::vector<long long> perm(off, 0);
    std::vector<int> tile_member(E->n_tiles);
    const int wall_code = -1;  // global group 0
    for (int k = 0; k < nm; ++k) {
        const swe_mesh* m = M[k];
        const int64_t b = E->base[k], n = E->n_cells[k];
        const void* cur = m->state[m->nstep % 2];
        e = cudaMemcpyAsync((char*)E->state[0] + b * v4, cur, n * v4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync((char*)E->geoA + b * v4, m->geoA, n * v4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync((char*)E->geoB + b * v4, m->geoB, n * v4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && sizeof(T) == 8)
            e = cudaMemcpyAsync((char*)E->geoR + b * v4, m->geoR, n * v4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync((char*)E->gm2 + b * sizeof(T), m->gm2, n * sizeof(T),
                                                  cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_create: copy");
        for (int64_t c = 0; c < n; ++c) {
            int code[3];
            for (int j = 0; j < 3; ++j) {
                const int32_t v = m->hm.code[3 * c + j];
                code[j] = v >= 0 ? (int)((v & kNbrMask) + b) | (v & kFlipBit) : -1 - (gbase[k] + (-1 - v));
            }
            int w = 0;
            if (sizeof(T) == 4) {
                const float gm2 = (float)(m->cfg.g * m->hm.m[c] * m->hm.m[c]);
                std::memcpy(&w, &gm2, sizeof w);
            }
            // static activity: an inflow or fixed-stage edge
            for (int j = 0; j < 3; ++j)
                if (code[j] < 0 && (kinds[-1 - code[j]] == kBcInflow || kinds[-1 - code[j]] == kBcStage))
                    w |= kStaticBit;
            topo[b + c] = make_int4(code[0], code[1], code[2], w);
            perm[b + c] = m->hm.perm[c];
        }
        for (int64_t c = n; c < (E->n_cells[k] + kEnsPad - 1) / kEnsPad * kEnsPad; ++c)
            topo[b + c] = make_int4(wall_code, wall_code, wall_code, 0);
        const int64_t t0 = E->first_tile[k];
        const int64_t t1 = (b + (n + kEnsPad - 1) / kEnsPad * kEnsPad) / kEnsPad;
        for (int64_t t = t0; t < t1; ++t) tile_member[t] = k;
    }
    std::vector<long long> mft(E->first_tile.begin(), E->first_tile.end());
    e = cudaMemcpyAsync(E->topo, topo.data(), off * sizeof(int4), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E->perm, perm.data(), off * sizeof(long long), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E->tile_member, tile_member.data(), E->n_tiles * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(E->member_first_tile, mft.data(), nm * sizeof(long long), cudaMemcpyHostToDevice, st);
    // each member's status block starts from its current CFL minimum and time
    std::vector<unsigned long long> first(nm);
    std::vector<double> t0(nm);
    for (int k = 0; k < nm && e == cudaSuccess; ++k) {
        unsigned long long s[kSmallWords];
        e = cudaMemcpy(s, M[k]->small, sizeof s, cudaMemcpyDeviceToHost);
        first[k] = s[M[k]->nstep % 3];
        std::memcpy(&t0[k], &s[kSlotT], sizeof(double));
    }
    unsigned long long* d_first = nullptr;
    double* d_t0 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d_first, nm * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&d_t0, nm * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(d_first, first.data(), nm * sizeof(unsigned long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_t0, t0.data(), nm * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        ens_init_small_kernel<<<(nm + 127) / 128, 128, 0, st>>>(E->small, d_first, d_t0, nm);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(E->state[1], E->state[0], off * v4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (d_first) cudaFree(d_first);
    if (d_t0) cudaFree(d_t0);
    if (e != cudaSuccess) return efail(e, "swe_ensemble_create: upload");
    Launch<T>::ensemble_default(&E->block, &E->min_blocks, &E->stages, &E->geo_early);
    long long wave = 0;
    e = ens_wave<T>(E, E->block, E->min_blocks, E->stages, E->geo_early, &wave);
    if (e != cudaSuccess) return efail(e, "swe_ensemble_create: occupancy");
    E->grid = (unsigned)std::min<long long>((long long)(E->n_total / E->block), wave);
    if (sizeof(T) == 4) {   // the split step's cell-pair kernel: one resident wave
        int per_sm = 0, sms = 0;
        e = Launch<T>::ensemble_pair_resident_blocks(E->pair_minb, E->pair_geo, &per_sm);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, E->device);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_create: occupancy");
        E->pair_grid = (unsigned)std::max<long long>(
            1, std::min<long long>(E->pair_spans, (long long)std::max(per_sm, 1) * std::max(sms, 1)));
    }
    E->cfl_host.assign(nm, -1.0);
    // FP64: the members' interior edges for the edge pass (the FP64 pipe bounds
    // the step, so evaluating each edge once pays; FP32 steps are bound by memory)
    if (sizeof(T) == 8) {
        std::vector<int2> cells;
        std::vector<double> ln, rl;
        std::vector<int4> eidx(off, make_int4(-1, -1, -1, 0));
        for (int k = 0; k < nm; ++k) append_edges(M[k]->hm, E->base[k], cells, ln, eidx.data() + E->base[k], &rl);
        const int64_t ne = (int64_t)cells.size();
        const size_t nb = (size_t)std::max<int64_t>(ne, 1);
        if ((rc = ens_alloc(E, (void**)&E->ecells, nb * sizeof(int2), "edges")) ||
            (rc = ens_alloc(E, &E->eln, 2 * nb * sizeof(T), "edges")) ||
            (rc = ens_alloc(E, &E->erl, nb * sizeof(T), "edges")) ||
            (rc = ens_alloc(E, &E->eflux, nb * sizeof(V4<T>), "edges")) ||
            (rc = ens_alloc(E, &E->esrc, nb * sizeof(T), "edges")) ||
            (rc = ens_alloc(E, (void**)&E->eidx, off * sizeof(int4), "edges")))
            return rc;
        if (ne) e = cudaMemcpy(E->ecells, cells.data(), ne * sizeof(int2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && ne) e = cudaMemcpy(E->eln, ln.data(), 2 * ne * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && ne) e = cudaMemcpy(E->erl, rl.data(), ne * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(E->eidx, eidx.data(), off * sizeof(int4), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_create: edges");
        E->n_edges = ne;
    }
    return SWE_OK;
}

// Activity bytes of the ensemble's current state (allocated once).
template <typename T>
int ens_init_activity(swe_ensemble* E) {
    cudaError_t e = cudaSuccess;
    if (!E->act[0]) {
        const int64_t len = (E->n_total + 31) / 32 * 32 + 32;
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            e = cudaMalloc((void**)&E->act[k], len);
            if (e == cudaSuccess) e = cudaMemsetAsync(E->act[k], 0, len, E->stream);
        }
        if (e != cudaSuccess) {
            for (auto& p : E->act) {
                if (p) cudaFree(p);
                p = nullptr;
            }
            set_error("swe_ensemble: no device memory for the activity bytes");
            return SWE_ENOMEM;
        }
        E->act_len = len;
        E->device_bytes += 3 * len;
    }
    const int p3 = (int)(E->nstep % 3);
    e = cudaMemsetAsync(E->act[p3], 2, E->act_len, E->stream);   // bit 1: rebuilt (act_init_kernel)
    if (e == cudaSuccess) e = cudaMemsetAsync(E->act[(p3 + 1) % 3], 0, E->act_len, E->stream);
    // the previous step's bytes: all 1, so the next step writes every cell's state
    if (e == cudaSuccess) e = cudaMemsetAsync(E->act[(p3 + 2) % 3], 1, E->act_len, E->stream);
    if (e == cudaSuccess)
        e = Launch<T>::act_init((const V4<T>*)E->state[E->nstep % 2], E->topo, E->n_total, (T)E->h_dry, E->act[p3],
                                E->stream);
    if (e != cudaSuccess) return efail(e, "swe_ensemble: activity bytes");
    E->act_valid = true;
    return SWE_OK;
}

template <typename T>
int ens_capture(swe_ensemble* E, int64_t start, int64_t len, const EnsPhysics& ph, cudaGraphExec_t* out) {
    cudaError_t e = cudaStreamBeginCapture(E->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return efail(e, "swe_ensemble_step: begin capture");
    cudaError_t le = cudaSuccess;
    for (int64_t s = 0; s < len && le == cudaSuccess; ++s) le = ens_launch<T>(E, start + s, ph, E->cap_stream);
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(E->cap_stream, &gr);
    if (le != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return efail(le, "swe_ensemble_step: capture launch"); }
    if (e != cudaSuccess) return efail(e, "swe_ensemble_step: end capture");
    e = cudaGraphInstantiate(out, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return efail(e, "swe_ensemble_step: instantiate");
    return SWE_OK;
}

template <typename T>
int ens_get_state(swe_ensemble* E, int k, void* h, void* hu, void* hv, int where) {
    const int64_t n = E->n_cells[k];
    const V4<T>* cur = (const V4<T>*)E->state[E->nstep % 2];
    cudaError_t e;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (where == SWE_DEVICE) {
        ens_unpack_kernel<T><<<grid, 256, 0, E->stream>>>(cur, E->perm, E->base[k], (T*)h, (T*)hu, (T*)hv, n);
        e = cudaGetLastError();
        return e == cudaSuccess ? SWE_OK : efail(e, "swe_ensemble_get_state");
    }
    if (E->stage_cells < n) {
        for (int j = 0; j < 3; ++j) {
            if (E->stage[j]) cudaFree(E->stage[j]);
            E->stage[j] = nullptr;
            e = cudaMalloc(&E->stage[j], n * sizeof(T));
            if (e != cudaSuccess) { E->stage_cells = 0; return efail(e, "swe_ensemble_get_state: staging"); }
        }
        E->stage_cells = n;
    }
    ens_unpack_kernel<T><<<grid, 256, 0, E->stream>>>(cur, E->perm, E->base[k], (T*)E->stage[0], (T*)E->stage[1],
                                                      (T*)E->stage[2], n);
    e = cudaGetLastError();
    void* dst[3] = {h, hu, hv};
    for (int j = 0; j < 3 && e == cudaSuccess; ++j)
        e = cudaMemcpyAsync(dst[j], E->stage[j], n * sizeof(T), cudaMemcpyDeviceToHost, E->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E->stream);
    return e == cudaSuccess ? SWE_OK : efail(e, "swe_ensemble_get_state");
}

// ---- launch-shape autotuner (swe_ensemble_autotune) --------------------------------
// Trial steps read the current state and write a scratch state buffer, a
// scratch copy of the members' status blocks and a scratch activity counter:
// nothing the ensemble holds changes.  First every compiled (block,
// min_blocks, stages, geometry early) shape with every chunk size at one
// resident wave, then
// grids of half, one and two waves for the best of those.

struct EnsShape {
    int block, min_blocks, stages, geo_early, chunk_log2;
    unsigned grid;
    int activity;
    int edges;
    int dynamic;
    // split step: the cell-pair kernel's (min_blocks, geometry early, grid) first
    int split = 0;
    int pair_minb = 8, pair_geo = 1;
    unsigned pair_grid = 0;
    int queue = 0;   // activity kernel with per-warp queues (FP32)
};

template <typename T>
int ens_time_shapes(swe_ensemble* E, const std::vector<EnsShape>& cand, int trial_steps, void* scratch,
                    unsigned long long* small, unsigned long long* act, std::vector<double>& ms) {
    cudaStream_t st = E->stream;
    const int rounds = 2;
    std::vector<cudaEvent_t> ev(2 * rounds * cand.size(), nullptr);
    // the dynamic kernels' counters rotate per trial launch, as per step
    cudaError_t e = cudaMemsetAsync(E->sched, 0, 3 * sizeof(unsigned), st);
    int launch_no = 0;
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    for (int r = 0; r < rounds && e == cudaSuccess; ++r)
        for (size_t c = 0; c < cand.size() && e == cudaSuccess; ++c) {
            EnsArgs<T> a = ens_args<T>(E, E->nstep);
            a.s_out = (V4<T>*)scratch;
            a.small = small;
            a.n_active = act;
            a.chunk_log2 = cand[c].chunk_log2;
            a.g = (T)E->g;
            a.h_dry = (T)E->h_dry;
            const EnsShape& sh = cand[c];
            // activity trials read the current bytes and rewrite the next buffer with
            // exactly the bytes the next real step writes there
            const int p3 = (int)(E->nstep % 3);
            if (!sh.edges) {
                a.ecells = nullptr; a.eln = nullptr; a.eflux = nullptr; a.esrc = nullptr; a.eidx = nullptr;
                a.n_edges = 0;
            } else {
                a.ecells = E->ecells; a.eln = (const T*)E->eln; a.eflux = (V4<T>*)E->eflux; a.esrc = (T*)E->esrc;
                a.eidx = E->eidx; a.n_edges = E->n_edges;
            }
            a.act_in = sh.activity ? E->act[p3] : nullptr;
            a.act_next = sh.activity ? E->act[(p3 + 1) % 3] : nullptr;
            a.act_clear = sh.activity ? E->act[(p3 + 2) % 3] : nullptr;
            auto launch = [&]() {
                a.sched_slot = launch_no % 3;
                a.sched_reset = (launch_no + 2) % 3;
                ++launch_no;
                a.cell_lo = 0;
                a.pair_spans = 0;
                if (sh.split && E->pair_spans > 0) {
                    a.pair_spans = (unsigned)E->pair_spans;
                    const cudaError_t pe = Launch<T>::ensemble_step_pair(a, sh.pair_minb, sh.pair_geo, sh.pair_grid, st);
                    if (pe != cudaSuccess) return pe;
                    a.cell_lo = E->pair_spans * kEnsPad;
                }
                if (sh.activity)
                    return Launch<T>::ensemble_step_act(a, sh.block, sh.min_blocks, sh.geo_early, sh.grid, st,
                                                        sh.dynamic, sh.queue);
                if (sh.dynamic)
                    return Launch<T>::ensemble_step_dyn(a, sh.block, sh.min_blocks, sh.geo_early, sh.grid, st);
                return Launch<T>::ensemble_step(a, sh.block, sh.min_blocks, sh.stages, sh.geo_early, sh.grid, st);
            };
            e = launch();  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(ev[2 * (r * cand.size() + c)], st);
            for (int s = 0; s < trial_steps && e == cudaSuccess; ++s) e = launch();
            if (e == cudaSuccess) e = cudaEventRecord(ev[2 * (r * cand.size() + c) + 1], st);
        }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    ms.assign(cand.size(), 1e300);
    for (int r = 0; r < rounds && e == cudaSuccess; ++r)
        for (size_t c = 0; c < cand.size() && e == cudaSuccess; ++c) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ev[2 * (r * cand.size() + c)], ev[2 * (r * cand.size() + c) + 1]);
            ms[c] = std::min(ms[c], (double)t / trial_steps);
        }
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    return e == cudaSuccess ? SWE_OK : efail(e, "swe_ensemble_autotune: trial steps");
}

template <typename T>
int ens_autotune_t(swe_ensemble* E, int trial_steps, swe_tune* out) {
    const EnsShape before{E->block, E->min_blocks, E->stages, E->geo_early, E->chunk_log2, E->grid,
                          E->activity, E->edges, E->dynamic, E->split, E->pair_minb, E->pair_geo, E->pair_grid,
                          E->queue};
    std::vector<EnsShape> cand{before};
    const bool with_act = E->n_total < kActivityMaxCells;
    if (with_act) {
        const int rc = ens_init_activity<T>(E);
        if (rc) return rc;
    }
    int v[32][4];
    const int nv = std::min(Launch<T>::ensemble_variants(v, 32), 32);
    for (int k = 0; k < nv; ++k) {
        long long wave = 0;
        cudaError_t e = ens_wave<T>(E, v[k][0], v[k][1], v[k][2], v[k][3], &wave);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_autotune: occupancy");
        const unsigned gr = (unsigned)std::max(1LL, std::min((long long)(E->n_total / v[k][0]), wave));
        for (int cl2 = 2; cl2 <= 6; ++cl2) {
            const EnsShape sh{v[k][0], v[k][1], v[k][2], v[k][3], cl2, gr, 0, 0, 0};
            if (!(sh.block == before.block && sh.min_blocks == before.min_blocks && sh.stages == before.stages &&
                  sh.geo_early == before.geo_early && sh.chunk_log2 == before.chunk_log2 && sh.grid == before.grid &&
                  !before.activity && !before.edges && !before.dynamic && !before.split))
                cand.push_back(sh);
        }
    }
    int w[16][3];
    const int nw = with_act ? std::min(Launch<T>::ensemble_act_variants(w, 16), 16) : 0;
    for (int k = 0; k < nw; ++k) {
        int per_sm = 0, sms = 0;
        cudaError_t e = Launch<T>::ensemble_act_resident_blocks(w[k][0], w[k][1], w[k][2], &per_sm);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, E->device);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_autotune: occupancy");
        const long long wave = (long long)std::max(per_sm, 1) * std::max(sms, 1);
        const unsigned gr = (unsigned)std::max(1LL, std::min((long long)(E->n_total / w[k][0]), wave));
        for (int cl2 = 2; cl2 <= 6; ++cl2) cand.push_back({w[k][0], w[k][1], 3, w[k][2], cl2, gr, 1, 0, 0});
        // and with dynamically taken chunks (at least 4 tiles each)
        int per_sm_d = 0;
        e = Launch<T>::ensemble_act_resident_blocks(w[k][0], w[k][1], w[k][2], &per_sm_d, 1);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_autotune: occupancy");
        const long long wave_d = (long long)std::max(per_sm_d, 1) * std::max(sms, 1);
        const unsigned gr_d = (unsigned)std::max(1LL, std::min((long long)(E->n_total / w[k][0]), wave_d));
        for (int cl2 = 2; cl2 <= 5; ++cl2) cand.push_back({w[k][0], w[k][1], 3, w[k][2], cl2, gr_d, 1, 0, 1});
    }
    // FP32: the activity kernel with per-warp queues of the cells that run the
    // flux path, round-robin and dynamic chunks
    int wq[8][3];
    const int nwq = with_act ? std::min(Launch<T>::ensemble_actq_variants(wq, 8), 8) : 0;
    for (int k = 0; k < nwq; ++k) {
        int sms = 0;
        cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, E->device);
        for (int dyn = 0; dyn <= 1 && e == cudaSuccess; ++dyn) {
            int per_sm = 0;
            e = Launch<T>::ensemble_act_resident_blocks(wq[k][0], wq[k][1], wq[k][2], &per_sm, dyn, 1);
            if (e != cudaSuccess) break;
            const long long wave = (long long)std::max(per_sm, 1) * std::max(sms, 1);
            const unsigned gr = (unsigned)std::max(1LL, std::min((long long)(E->n_total / wq[k][0]), wave));
            for (int cl2 = 2; cl2 <= (dyn ? 5 : 6); ++cl2) {
                EnsShape sh{wq[k][0], wq[k][1], 3, wq[k][2], cl2, gr, 1, 0, dyn};
                sh.queue = 1;
                cand.push_back(sh);
            }
        }
        if (e != cudaSuccess) return efail(e, "swe_ensemble_autotune: occupancy");
    }
    int y[16][3];
    const int ny = std::min(Launch<T>::ensemble_dyn_variants(y, 16), 16);
    for (int k = 0; k < ny; ++k) {
        int per_sm = 0, sms = 0;
        cudaError_t e = Launch<T>::ensemble_dyn_resident_blocks(y[k][0], y[k][1], y[k][2], &per_sm);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, E->device);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_autotune: occupancy");
        const long long wave = (long long)std::max(per_sm, 1) * std::max(sms, 1);
        const unsigned gr = (unsigned)std::max(1LL, std::min((long long)(E->n_total / y[k][0]), wave));
        for (int cl2 = 0; cl2 <= 5; ++cl2) cand.push_back({y[k][0], y[k][1], 1, y[k][2], cl2, gr, 0, 0, 1});
    }
    int x[16][4];
    const int nx = E->eflux ? std::min(Launch<T>::ensemble_edge_variants(x, 16), 16) : 0;
    for (int k = 0; k < nx; ++k) {
        int per_sm = 0, sms = 0;
        cudaError_t e = Launch<T>::ensemble_edge_resident_blocks(x[k][0], x[k][1], x[k][2], x[k][3], &per_sm);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, E->device);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_autotune: occupancy");
        const long long wave = (long long)std::max(per_sm, 1) * std::max(sms, 1);
        const unsigned gr = (unsigned)std::max(1LL, std::min((long long)(E->n_total / x[k][0]), wave));
        for (int cl2 = 2; cl2 <= 6; ++cl2) cand.push_back({x[k][0], x[k][1], x[k][2], x[k][3], cl2, gr, 0, 1, 0});
    }
    // FP32 with members placed for the cell-pair kernel: every activity and
    // dynamically scheduled shape also as the second kernel of a split step
    int pq[8][2];
    const int npq = E->pair_spans > 0 ? std::min(Launch<T>::ensemble_pair_variants(pq, 8), 8) : 0;
    std::vector<unsigned> pair_wave(npq, 0);
    for (int q = 0; q < npq; ++q) {
        int per_sm = 0, sms = 0;
        cudaError_t e = Launch<T>::ensemble_pair_resident_blocks(pq[q][0], pq[q][1], &per_sm);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, E->device);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_autotune: occupancy");
        pair_wave[q] = (unsigned)std::max<long long>(
            1, std::min<long long>(E->pair_spans, (long long)std::max(per_sm, 1) * std::max(sms, 1)));
    }
    if (npq > 0) {
        const size_t n0 = cand.size();
        for (size_t c = 1; c < n0; ++c)
            if (cand[c].activity || cand[c].dynamic) {
                EnsShape sh = cand[c];
                sh.split = 1;
                sh.pair_minb = pq[0][0];
                sh.pair_geo = pq[0][1];
                sh.pair_grid = pair_wave[0];
                cand.push_back(sh);
            }
    }
    void* scratch = nullptr;
    unsigned long long *small = nullptr, *act = nullptr;
    const size_t small_bytes = 8 * (size_t)E->n_members * sizeof(unsigned long long);
    if (cudaMalloc(&scratch, (size_t)E->n_total * sizeof(V4<T>)) != cudaSuccess ||
        cudaMalloc(&small, small_bytes) != cudaSuccess || cudaMalloc(&act, sizeof(unsigned long long)) != cudaSuccess) {
        for (void* p : {scratch, (void*)small, (void*)act})
            if (p) cudaFree(p);
        set_error("swe_ensemble_autotune: no device memory for the scratch state");
        return SWE_ENOMEM;
    }
    cudaError_t e = cudaMemcpyAsync(small, E->small, small_bytes, cudaMemcpyDeviceToDevice, E->stream);
    int rc = e == cudaSuccess ? SWE_OK : efail(e, "swe_ensemble_autotune: status copy");
    std::vector<double> ms;
    if (!rc) rc = ens_time_shapes<T>(E, cand, trial_steps, scratch, small, act, ms);
    size_t best = 0;
    std::vector<EnsShape> cand2;
    std::vector<double> ms2;
    if (!rc) {
        // runoff, as for a mesh: the shape in use and the (at most four)
        // candidates within 5 % of the fastest, timed again over at least 32
        // steps; the first of them in candidate order within 1 % of the fastest
        // there is kept (stable from run to run)
        const double fastest = *std::min_element(ms.begin(), ms.end());
        std::vector<size_t> close;
        for (size_t c = 0; c < cand.size(); ++c)
            if (ms[c] <= fastest * 1.05) close.push_back(c);
        std::stable_sort(close.begin(), close.end(), [&](size_t x, size_t y) { return ms[x] < ms[y]; });
        if (close.size() > 4) close.resize(4);
        if (std::find(close.begin(), close.end(), (size_t)0) == close.end()) close.push_back(0);
        std::sort(close.begin(), close.end());
        if (close.size() > 1) {
            std::vector<EnsShape> rc_cand;
            for (size_t c : close) rc_cand.push_back(cand[c]);
            std::vector<double> rc_ms;
            rc = ens_time_shapes<T>(E, rc_cand, std::max(32, 4 * trial_steps), scratch, small, act, rc_ms);
            if (!rc)
                for (size_t k = 0; k < close.size(); ++k) ms[close[k]] = rc_ms[k];
        }
        double fast2 = 1e300;
        for (size_t c : close) fast2 = std::min(fast2, ms[c]);
        best = close[0];
        for (size_t c : close)
            if (ms[c] <= fast2 * 1.01) { best = c; break; }
    }
    if (!rc) {
        long long wave = 0;
        const EnsShape b = cand[best];
        if (b.activity || b.edges || b.dynamic) {
            int per_sm = 0, sms = 0;
            e = b.activity  ? Launch<T>::ensemble_act_resident_blocks(b.block, b.min_blocks, b.geo_early, &per_sm,
                                                                      b.dynamic, b.queue)
                : b.dynamic ? Launch<T>::ensemble_dyn_resident_blocks(b.block, b.min_blocks, b.geo_early, &per_sm)
                            : Launch<T>::ensemble_edge_resident_blocks(b.block, b.min_blocks, b.stages, b.geo_early,
                                                                       &per_sm);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, E->device);
            wave = (long long)std::max(per_sm, 1) * std::max(sms, 1);
        } else {
            e = ens_wave<T>(E, b.block, b.min_blocks, b.stages, b.geo_early, &wave);
        }
        if (e != cudaSuccess) rc = efail(e, "swe_ensemble_autotune: occupancy");
        const long long tiles = (long long)(E->n_total / b.block);
        for (long long gsz : {wave / 2, 2 * wave}) {
            const unsigned gr = (unsigned)std::max(1LL, std::min(tiles, gsz));
            if (!rc && gr != b.grid) {
                EnsShape sh = b;
                sh.grid = gr;
                cand2.push_back(sh);
            }
        }
        // a split step: the other cell-pair kernel shapes, and two waves of the first
        if (!rc && b.split) {
            for (int q = 1; q < npq; ++q) {
                EnsShape sh = b;
                sh.pair_minb = pq[q][0];
                sh.pair_geo = pq[q][1];
                sh.pair_grid = pair_wave[q];
                cand2.push_back(sh);
            }
            EnsShape sh = b;
            sh.pair_grid = (unsigned)std::min<long long>(E->pair_spans, 2LL * pair_wave[0]);
            if (sh.pair_grid != b.pair_grid) cand2.push_back(sh);
        }
        // grids of half and two waves for the kept shape, timed as long as the runoff
        if (!rc && !cand2.empty())
            rc = ens_time_shapes<T>(E, cand2, std::max(32, 4 * trial_steps), scratch, small, act, ms2);
    }
    for (void* p : {scratch, (void*)small, (void*)act}) cudaFree(p);
    // the trials consumed the dynamic kernels' counters: the steps start from zero
    if (!rc) {
        const cudaError_t ze = cudaMemsetAsync(E->sched, 0, 3 * sizeof(unsigned), E->stream);
        if (ze != cudaSuccess) rc = efail(ze, "swe_ensemble_autotune: counters");
    }
    if (rc) return rc;
    EnsShape pick = cand[best];
    double ms_pick = ms[best];
    for (size_t c = 0; c < cand2.size(); ++c)
        if (ms2[c] * 1.02 < ms_pick) { pick = cand2[c]; ms_pick = ms2[c]; }
    E->block = pick.block;
    E->min_blocks = pick.min_blocks;
    E->stages = pick.stages;
    E->geo_early = pick.geo_early;
    E->activity = pick.activity;
    E->edges = pick.edges;
    E->dynamic = pick.dynamic;
    E->split = pick.split;
    E->queue = pick.queue;
    E->pair_minb = pick.pair_minb;
    E->pair_geo = pick.pair_geo;
    E->pair_grid = pick.pair_grid;
    // the activity bytes are rebuilt from the state before the next step: trials
    // of split steps leave the paired members' next bytes unwritten
    E->act_valid = false;
    E->chunk_log2 = pick.chunk_log2;
    E->grid = pick.grid;
    drop_graphs(E);
    if (out) {
        out->block_size = pick.block;
        out->min_blocks = pick.min_blocks;
        out->stages = pick.stages;
        out->geometry_early = pick.geo_early;
        out->activity = pick.activity;
        out->edge_pass = pick.edges;
        out->dynamic = pick.dynamic;
        out->chunk = 1 << pick.chunk_log2;
        out->grid = pick.grid;
        out->cells_per_thread = (double)E->n_total / ((double)pick.grid * pick.block);
        out->ms_best = ms_pick;
        out->ms_before = ms[0];
        out->n_candidates = (int)(cand.size() + cand2.size());
        out->cell_pairs = pick.split;
        out->queue = pick.queue;
    }
    return SWE_OK;
}

}  // namespace

extern "C" {

void swe_ensemble_destroy(swe_ensemble* E) {
    if (!E) return;
    EnsDeviceGuard dg(E->device);
    if (E->stream) cudaStreamSynchronize(E->stream);
    drop_graphs(E);
    void* bufs[] = {E->state[0], E->state[1], E->geoA, E->geoB, E->topo, E->gm2, E->perm, E->tile_member,
                    E->member_first_tile, E->cfl, E->small, E->n_active, E->kind, E->value,
                    E->stage[0], E->stage[1], E->stage[2], E->act[0], E->act[1], E->act[2],
                    E->ecells, E->eln, E->eflux, E->esrc, E->eidx, E->geoR, E->erl, E->sched};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (E->cap_stream) cudaStreamDestroy(E->cap_stream);
    delete E;
}

int swe_ensemble_create(swe_mesh* const* members, int n_members, swe_ensemble** out) {
    if (!out) { set_error("swe_ensemble_create: out is NULL"); return SWE_EINVAL; }
    *out = nullptr;
    if (!members || n_members < 1) { set_error("swe_ensemble_create: no members"); return SWE_EINVAL; }
    for (int k = 0; k < n_members; ++k) {
        const swe_mesh* m = members[k];
        if (!m) { set_error("swe_ensemble_create: NULL member"); return SWE_EINVAL; }
        if (!m->have_state) { set_error("swe_ensemble_create: member " + std::to_string(k) + " has no state"); return SWE_EINVAL; }
        if (m->cfg.precision != members[0]->cfg.precision || m->cfg.device != members[0]->cfg.device ||
            m->cfg.g != members[0]->cfg.g || m->cfg.h_dry != members[0]->cfg.h_dry ||
            m->cfg.flux != members[0]->cfg.flux) {
            set_error("swe_ensemble_create: members differ in precision, device, flux, g or h_dry");
            return SWE_EINVAL;
        }
        if (m->topo_dirty) { set_error("swe_ensemble_create: member boundary groups not applied"); return SWE_EINVAL; }
    }
    swe_ensemble* E = new (std::nothrow) swe_ensemble();
    if (!E) { set_error("swe_ensemble_create: out of host memory"); return SWE_ENOMEM; }
    E->precision = members[0]->cfg.precision;
    E->device = members[0]->cfg.device;
    E->esz = E->precision == SWE_FP32 ? 4 : 8;
    E->n_members = n_members;
    E->g = members[0]->cfg.g;
    E->h_dry = members[0]->cfg.h_dry;
    E->hll = members[0]->cfg.flux == SWE_FLUX_HLL ? 1 : 0;
    E->stream = members[0]->stream;
    EnsDeviceGuard dg(E->device);
    for (int k = 0; k < n_members; ++k) {
        cudaError_t e = cudaStreamSynchronize(members[k]->stream);
        if (e != cudaSuccess) { swe_ensemble_destroy(E); return efail(e, "swe_ensemble_create: member stream"); }
    }
    cudaError_t e = cudaStreamCreateWithFlags(&E->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { swe_ensemble_destroy(E); return efail(e, "swe_ensemble_create: stream"); }
    int rc;
    try {
        rc = E->precision == SWE_FP32 ? ens_build<float>(E, members) : ens_build<double>(E, members);
    } catch (const std::bad_alloc&) {
        set_error("swe_ensemble_create: out of host memory");
        rc = SWE_ENOMEM;
    }
    if (rc) { swe_ensemble_destroy(E); return rc; }
    *out = E;
    return SWE_OK;
}

int swe_ensemble_set_stream(swe_ensemble* E, void* stream) {
    if (!E) { set_error("swe_ensemble_set_stream: NULL ensemble"); return SWE_EINVAL; }
    E->stream = (cudaStream_t)stream;
    return SWE_OK;
}

int swe_ensemble_step(swe_ensemble* E, int64_t nsteps, const double* cfl, double* t_out) {
    NvtxRange nvtx_range("swe_ensemble_step");
    if (!E || nsteps < 0) { set_error("swe_ensemble_step: bad arguments"); return SWE_EINVAL; }
    EnsDeviceGuard dg(E->device);
    std::vector<double> c(E->n_members, 0.9);
    if (cfl)
        for (int k = 0; k < E->n_members; ++k) {
            if (!(cfl[k] > 0.0) || !std::isfinite(cfl[k])) { set_error("swe_ensemble_step: bad cfl"); return SWE_EINVAL; }
            c[k] = cfl[k];
        }
    cudaError_t e;
    if (c != E->cfl_host) {
        e = cudaMemcpyAsync(E->cfl, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, E->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(E->stream);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_step: cfl");
        E->cfl_host = c;
    }
    const EnsPhysics ph{E->g, E->h_dry};
    if (nsteps > 0 && E->activity && !E->act_valid) {
        int rc = E->precision == SWE_FP32 ? ens_init_activity<float>(E) : ens_init_activity<double>(E);
        if (rc) return rc;
    }
    if (nsteps > 0) {
        // the whole call is one CUDA graph: nsteps step kernels over all members
        const auto key = std::make_pair((int)(E->nstep % 6), nsteps);
        auto it = E->graphs.find(key);
        cudaGraphExec_t ge = nullptr;
        if (it == E->graphs.end()) {
            if (E->graphs.size() >= 8) drop_graphs(E);
            int rc = E->precision == SWE_FP32 ? ens_capture<float>(E, E->nstep % 6, nsteps, ph, &ge)
                                              : ens_capture<double>(E, E->nstep % 6, nsteps, ph, &ge);
            if (rc) return rc;
            E->graphs[key] = ge;
        } else {
            ge = it->second;
        }
        e = cudaGraphLaunch(ge, E->stream);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_step: graph launch");
        E->nstep += nsteps;
    }
    if (t_out) {
        std::vector<unsigned long long> s(8 * (size_t)E->n_members);
        e = cudaMemcpyAsync(s.data(), E->small, s.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                            E->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(E->stream);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_step: status");
        int rc = SWE_OK;
        for (int k = 0; k < E->n_members; ++k) {
            std::memcpy(&t_out[k], &s[8 * k + kSlotT], sizeof(double));
            if ((s[8 * k + kSlotStatus] & kStatusBadIndex) && !rc) {
                set_error("swe_ensemble_step: member " + std::to_string(k) +
                          ": an index or boundary group out of range (debug checks)");
                rc = SWE_EMESH;
            } else if ((s[8 * k + kSlotStatus] & kStatusNonFinite) && !rc) {
                set_error("swe_ensemble_step: member " + std::to_string(k) + " has a non-finite state");
                rc = SWE_ENONFINITE;
            } else if ((s[8 * k + kSlotStatus] & kStatusDry) && !rc) {
                set_error("swe_ensemble_step: member " + std::to_string(k) + " is completely dry");
                rc = SWE_EDRY;
            }
        }
        return rc;
    }
    return SWE_OK;
}

int swe_ensemble_set_shape(swe_ensemble* E, const swe_tune* shape) {
    if (!E || !shape || (shape->activity != 0 && shape->activity != 1) || (shape->edge_pass != 0 && shape->edge_pass != 1) ||
        (shape->dynamic != 0 && shape->dynamic != 1) || shape->activity + shape->edge_pass > 1 ||
        shape->edge_pass + shape->dynamic > 1 || (shape->edge_pass && !E->eflux) ||
        (shape->activity && shape->dynamic && shape->chunk < 4) ||
        shape->chunk < 1 || (shape->chunk & (shape->chunk - 1)) || shape->chunk > 4096 || shape->grid < 0) {
        set_error("swe_ensemble_set_shape: bad arguments");
        return SWE_EINVAL;
    }
    if (shape->activity && E->n_total >= kActivityMaxCells) {
        set_error("swe_ensemble_set_shape: activity needs fewer than 2^29 cells");
        return SWE_EINVAL;
    }
    if ((shape->cell_pairs != 0 && shape->cell_pairs != 1) ||
        (shape->cell_pairs && (E->precision != SWE_FP32 || shape->edge_pass))) {
        set_error("swe_ensemble_set_shape: cell_pairs (a split step) needs FP32 and no edge pass");
        return SWE_EINVAL;
    }
    if ((shape->queue != 0 && shape->queue != 1) ||
        (shape->queue && (E->precision != SWE_FP32 || !shape->activity))) {
        set_error("swe_ensemble_set_shape: queue needs FP32 and activity");
        return SWE_EINVAL;
    }
    EnsDeviceGuard dg(E->device);
    int per_sm = 0, sms = 0;
    cudaError_t e;
    const int B = shape->block_size, M = shape->min_blocks, S = shape->stages, Gx = shape->geometry_early;
    if (E->precision == SWE_FP32) {
        if (shape->activity)
            e = Launch<float>::ensemble_act_resident_blocks(B, M, Gx, &per_sm, shape->dynamic, shape->queue);
        else if (shape->dynamic) e = Launch<float>::ensemble_dyn_resident_blocks(B, M, Gx, &per_sm);
        else e = Launch<float>::ensemble_resident_blocks(B, M, S, Gx, &per_sm);
    } else {
        if (shape->activity) e = Launch<double>::ensemble_act_resident_blocks(B, M, Gx, &per_sm, shape->dynamic);
        else if (shape->dynamic) e = Launch<double>::ensemble_dyn_resident_blocks(B, M, Gx, &per_sm);
        else if (shape->edge_pass) e = Launch<double>::ensemble_edge_resident_blocks(B, M, S, Gx, &per_sm);
        else e = Launch<double>::ensemble_resident_blocks(B, M, S, Gx, &per_sm);
    }
    if (e == cudaErrorInvalidValue) {
        set_error("swe_ensemble_set_shape: no compiled ensemble kernel of this shape");
        return SWE_EINVAL;
    }
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, E->device);
    if (e != cudaSuccess) return efail(e, "swe_ensemble_set_shape: occupancy");
    const long long tiles = (long long)(E->n_total / shape->block_size);
    const long long wave = (long long)std::max(per_sm, 1) * std::max(sms, 1);
    long long cl2 = 0;
    while ((1LL << cl2) < shape->chunk) ++cl2;
    E->block = shape->block_size;
    E->min_blocks = shape->min_blocks;
    E->stages = shape->activity ? 3 : (shape->dynamic ? 1 : shape->stages);
    E->geo_early = shape->geometry_early;
    E->chunk_log2 = (int)cl2;
    E->grid = (unsigned)std::max(1LL, std::min(tiles, shape->grid > 0 ? (long long)shape->grid : wave));
    if (E->activity != shape->activity || E->split != shape->cell_pairs) E->act_valid = false;
    E->activity = shape->activity;
    E->edges = shape->edge_pass;
    E->dynamic = shape->dynamic;
    E->split = shape->cell_pairs;   // the cell-pair kernel keeps its shape and one-wave grid
    E->queue = shape->queue;
    if (E->dynamic) {   // counters from zero (earlier steps may have left them used)
        e = cudaMemsetAsync(E->sched, 0, 3 * sizeof(unsigned), E->stream);
        if (e != cudaSuccess) return efail(e, "swe_ensemble_set_shape: counters");
    }
    drop_graphs(E);
    return SWE_OK;
}

int swe_ensemble_autotune(swe_ensemble* E, int trial_steps, swe_tune* out) {
    NvtxRange nvtx_range("swe_ensemble_autotune");
    if (!E || trial_steps < 0) { set_error("swe_ensemble_autotune: bad arguments"); return SWE_EINVAL; }
    if (trial_steps == 0) trial_steps = 4;
    EnsDeviceGuard dg(E->device);
    return E->precision == SWE_FP32 ? ens_autotune_t<float>(E, trial_steps, out)
                                    : ens_autotune_t<double>(E, trial_steps, out);
}

int swe_ensemble_get_state(swe_ensemble* E, int member, void* h, void* hu, void* hv, int where) {
    if (!E || member < 0 || member >= E->n_members || !h || !hu || !hv || (where != SWE_HOST && where != SWE_DEVICE)) {
        set_error("swe_ensemble_get_state: bad arguments");
        return SWE_EINVAL;
    }
    EnsDeviceGuard dg(E->device);
    return E->precision == SWE_FP32 ? ens_get_state<float>(E, member, h, hu, hv, where)
                                    : ens_get_state<double>(E, member, h, hu, hv, where);
}

int swe_ensemble_get_info(swe_ensemble* E, int member, swe_info* info) {
    if (!E || !info || member < 0 || member >= E->n_members) {
        set_error("swe_ensemble_get_info: bad arguments");
        return SWE_EINVAL;
    }
    EnsDeviceGuard dg(E->device);
    unsigned long long s[8];
    unsigned long long act = 0;
    cudaError_t e = cudaMemcpyAsync(s, E->small + 8 * (size_t)member, sizeof s, cudaMemcpyDeviceToHost, E->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&act, E->n_active, sizeof act, cudaMemcpyDeviceToHost, E->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E->stream);
    if (e != cudaSuccess) return efail(e, "swe_ensemble_get_info");
    std::memset(info, 0, sizeof *info);
    info->n_cells = E->n_cells[member];
    info->n_steps = E->nstep;
    info->n_clamped = (int64_t)s[kSlotClamp];
    std::memcpy(&info->t, &s[kSlotT], sizeof(double));
    std::memcpy(&info->dt_next, &s[E->nstep % 3], sizeof(double));
    info->precision = E->precision;
    info->status = (s[kSlotStatus] & kStatusBadIndex)     ? SWE_EMESH
                   : (s[kSlotStatus] & kStatusNonFinite) ? SWE_ENONFINITE
                   : ((s[kSlotStatus] & kStatusDry) ? SWE_EDRY : SWE_OK);
    info->device_bytes = E->device_bytes;
    info->n_active = (int64_t)act;  // all members together
    return SWE_OK;
}

}  // extern "C"
