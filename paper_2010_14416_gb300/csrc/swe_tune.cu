// swe_tune.cu -- launch-shape autotuner of the step kernel (swe_autotune).
//
// The paper fixes one thread per cell (Section 5.3.2) and no block size; here
// the shape of the fused step kernel is a measured choice per mesh: every
// compiled (block, min_blocks, stages, geometry early) shape of the step
// kernel, every (block, min_blocks, geometry early) shape of the cell-pair
// step (FP32) and of the activity kernel, each with several grid sizes (one or two resident waves looping
// over the cells, or 1, 2 or 4 cells per thread), is timed with CUDA events
// on the mesh's current state.  The trial steps read the current state and
// write a scratch state buffer and a scratch copy of the status block; trials
// of the activity kernel also write the mesh's next activity buffers, with
// exactly the bytes the next real step writes there.  Every shape evaluates
// the same arithmetic on every cell, so the choice changes speed only, never
// results (the GPU tests check this bit for bit).  A runoff then times the
// shape in use and the (at most four) candidates within 5 % of the fastest
// again over at least 32 steps, and keeps the first of them in the fixed
// candidate order within 1 % of the fastest there: short trials blur
// differences of a few percent, and a tie keeps the same choice from run to
// run.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "swe_internal.h"

using namespace swe;

namespace {

constexpr double kTuneTolerance = 1.02;    // first pass: ties within 2 %
constexpr double kRunoffWindow = 1.05;     // candidates within 5 % of the fastest go to the runoff
constexpr int kRunoffMax = 4;              // at most this many
constexpr double kRunoffTolerance = 1.01;  // runoff: ties within 1 %

struct Shape {
    int block, min_blocks, stages, geo_early, activity, edges;
    unsigned grid;
    int pairs;
};

bool same_shape(const Shape& a, const Shape& b) {
    return a.block == b.block && a.min_blocks == b.min_blocks && a.stages == b.stages && a.geo_early == b.geo_early &&
           a.activity == b.activity && a.edges == b.edges && a.grid == b.grid && a.pairs == b.pairs;
}

int tfail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return SWE_ECUDA;
}

struct TuneDeviceGuard {
    int prev = -1;
    explicit TuneDeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~TuneDeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
int candidate_shapes(const swe_mesh* m, std::vector<Shape>& cand) {
    const long long n = m->hm.n_cells;
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->cfg.device);
    if (e != cudaSuccess) return tfail(e, "swe_autotune: device attribute");
    // the shape in use first
    cand.push_back({m->cfg.block_size, m->cfg.min_blocks, m->cfg.stages, m->cfg.geometry_early, m->cfg.activity,
                    m->cfg.edge_pass, m->grid, m->cfg.cell_pairs});
    auto add = [&](int block, int minb, int stages, int geo, int act, int edges, int pairs = 0) -> int {
        int per_sm = 0;
        cudaError_t er = pairs ? Launch<T>::pair_resident_blocks(block, minb, geo, stages, &per_sm)
                               : Launch<T>::resident_blocks(block, minb, stages, geo, act, edges, &per_sm);
        if (er != cudaSuccess) return tfail(er, "swe_autotune: occupancy");
        const long long units = pairs ? (n + 1) / 2 : n;
        const long long need = (units + block - 1) / block;
        const long long wave = (long long)std::max(per_sm, 1) * std::max(sms, 1);
        const long long grids[] = {wave, 2 * wave, need, (need + 1) / 2, (need + 3) / 4};
        for (long long gsz : grids) {
            const Shape sh{block, minb, stages, geo, act, edges,
                           (unsigned)std::max(1LL, std::min(gsz, need)), pairs};
            bool seen = false;
            for (const Shape& c : cand) seen = seen || same_shape(c, sh);
            if (!seen) cand.push_back(sh);
        }
        return SWE_OK;
    };
    int v[64][4];
    const int nv = std::min(Launch<T>::step_variants(v, 64), 64);
    for (int k = 0; k < nv; ++k) {
        const int rc = add(v[k][0], v[k][1], v[k][2], v[k][3], 0, 0);
        if (rc) return rc;
    }
    const int ne = std::min(Launch<T>::edge_variants(v, 64), 64);
    for (int k = 0; k < ne; ++k) {
        const int rc = add(v[k][0], v[k][1], v[k][2], v[k][3], 0, 1);
        if (rc) return rc;
    }
    int q[64][4];
    const int nq = std::min(Launch<T>::pair_variants(q, 64), 64);
    for (int k = 0; k < nq; ++k) {
        const int rc = add(q[k][0], q[k][1], q[k][3], q[k][2], 0, 0, 1);
        if (rc) return rc;
    }
    int w[64][4];
    const int nw = n < kActivityMaxCells ? std::min(Launch<T>::act_variants(w, 64), 64) : 0;
    for (int k = 0; k < nw; ++k) {
        const int rc = add(w[k][0], w[k][1], w[k][3], w[k][2], 1, 0);
        if (rc) return rc;
    }
    return SWE_OK;
}

void apply_shape(swe_mesh* m, const Shape& sh) {
    m->cfg.block_size = sh.block;
    m->cfg.min_blocks = sh.min_blocks;
    m->cfg.stages = sh.stages;
    m->cfg.geometry_early = sh.geo_early;
    m->cfg.activity = sh.activity;
    m->cfg.edge_pass = sh.edges;
    m->cfg.cell_pairs = sh.pairs;
    m->grid = sh.grid;
    if (!sh.activity)
        m->plain = LaunchShape{sh.block, sh.min_blocks, sh.stages, sh.geo_early, sh.edges, sh.grid, sh.pairs};
}

template <typename T>
int autotune_t(swe_mesh* m, int trial_steps, swe_tune* out) {
    const int64_t n = m->hm.n_cells;
    std::vector<Shape> cand;
    int rc = candidate_shapes<T>(m, cand);
    if (rc) return rc;
    const Shape before = cand[0];
    const LaunchShape plain_before = m->plain;
    cudaStream_t st = m->stream;
    // the edge list for the edge-pass trials, and the activity bytes of the
    // current state for the activity-kernel trials
    rc = build_edges(m);
    if (rc) return rc;
    if (n < kActivityMaxCells) {
        rc = init_activity(m);
        if (rc) return rc;
    }
    void* scratch = nullptr;
    unsigned long long* small = nullptr;
    cudaError_t e = cudaMalloc(&scratch, (size_t)n * sizeof(V4<T>));
    if (e != cudaSuccess) {
        set_error("swe_autotune: no device memory for the scratch state");
        return SWE_ENOMEM;
    }
    e = cudaMalloc(&small, kSmallWords * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFree(scratch);
        set_error("swe_autotune: no device memory for the scratch status block");
        return SWE_ENOMEM;
    }
    const int rounds = 2;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(small, m->small, kSmallWords * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
    const void* cur = m->state[m->nstep % 2];
    // time the listed candidates over `steps` steps each, `rounds` times in
    // turn; ms[c] = the best round's time per step
    std::vector<double> ms(cand.size(), 1e300);
    auto time_candidates = [&](const std::vector<size_t>& which, int steps) {
        std::vector<cudaEvent_t> ev(2 * rounds * which.size(), nullptr);
        for (auto& x : ev)
            if (e == cudaSuccess) e = cudaEventCreate(&x);
        for (int r = 0; r < rounds && e == cudaSuccess; ++r) {
            for (size_t w = 0; w < which.size() && e == cudaSuccess; ++w) {
                apply_shape(m, cand[which[w]]);
                e = launch_step_raw(m, cur, scratch, small, m->nstep, 0.9, nullptr, nullptr, st, true);  // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(ev[2 * (r * which.size() + w)], st);
                for (int k = 0; k < steps && e == cudaSuccess; ++k)
                    e = launch_step_raw(m, cur, scratch, small, m->nstep, 0.9, nullptr, nullptr, st, true);
                if (e == cudaSuccess) e = cudaEventRecord(ev[2 * (r * which.size() + w) + 1], st);
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        for (size_t w = 0; w < which.size(); ++w) ms[which[w]] = 1e300;
        for (int r = 0; r < rounds && e == cudaSuccess; ++r)
            for (size_t w = 0; w < which.size() && e == cudaSuccess; ++w) {
                float t = 0.f;
                e = cudaEventElapsedTime(&t, ev[2 * (r * which.size() + w)], ev[2 * (r * which.size() + w) + 1]);
                ms[which[w]] = std::min(ms[which[w]], (double)t / steps);
            }
        for (auto& x : ev)
            if (x) cudaEventDestroy(x);
    };
    std::vector<size_t> all(cand.size());
    for (size_t c = 0; c < cand.size(); ++c) all[c] = c;
    time_candidates(all, trial_steps);
    // the first candidate (in the fixed order above) within a tolerance of the
    // fastest of a set: timings within noise of each other then give the same
    // choice from run to run
    auto first_within = [&](const std::vector<size_t>& which, double tol, bool plain_only) {
        double fastest = 1e300;
        for (size_t c : which)
            if (!plain_only || !cand[c].activity) fastest = std::min(fastest, ms[c]);
        for (size_t c : which)
            if ((!plain_only || !cand[c].activity) && ms[c] <= fastest * tol) return c;
        return cand.size();
    };
    size_t best = 0, best_plain = cand.size();
    if (e == cudaSuccess) {
        best_plain = first_within(all, kTuneTolerance, true);
        // runoff: the candidates within kRunoffWindow of the fastest (at most
        // kRunoffMax, the fastest first) timed again over runs long enough for
        // the differences of a few percent that short trials blur
        double fastest = 1e300;
        for (size_t c : all) fastest = std::min(fastest, ms[c]);
        std::vector<size_t> close;
        for (size_t c : all)
            if (ms[c] <= fastest * kRunoffWindow) close.push_back(c);
        std::stable_sort(close.begin(), close.end(), [&](size_t x, size_t y) { return ms[x] < ms[y]; });
        if (close.size() > (size_t)kRunoffMax) close.resize(kRunoffMax);
        // the shape in use runs too: it is kept unless another is faster in the runoff
        if (std::find(close.begin(), close.end(), (size_t)0) == close.end()) close.push_back(0);
        std::sort(close.begin(), close.end());   // back to the fixed candidate order
        if (close.size() > 1) time_candidates(close, std::max(32, 4 * trial_steps));
        best = e == cudaSuccess ? first_within(close, kRunoffTolerance, false) : 0;
    }
    cudaFree(scratch);
    cudaFree(small);
    const Shape pick = e == cudaSuccess ? cand[best] : before;
    // launches without activity bytes take the fastest shape of the plain kernel
    if (e == cudaSuccess && best_plain < cand.size()) apply_shape(m, cand[best_plain]);
    else m->plain = plain_before;
    apply_shape(m, pick);
    // the activity bytes are rebuilt before the next step: the trials cleared the
    // previous step's bytes, which tell the next step whose state it may leave
    m->act_valid = false;
    drop_mesh_graph(m);
    if (e != cudaSuccess) return tfail(e, "swe_autotune: trial steps");
    if (out) {
        out->block_size = pick.block;
        out->min_blocks = pick.min_blocks;
        out->stages = pick.stages;
        out->geometry_early = pick.geo_early;
        out->activity = pick.activity;
        out->edge_pass = pick.edges;
        out->dynamic = 0;
        out->chunk = 0;
        out->grid = pick.grid;
        out->cells_per_thread = (double)n / ((double)pick.grid * pick.block);
        out->ms_best = ms[best];
        out->ms_before = ms[0];
        out->n_candidates = (int)cand.size();
        out->cell_pairs = pick.pairs;
        out->queue = 0;
    }
    return SWE_OK;
}

}  // namespace

extern "C" {

int swe_autotune(swe_mesh* m, int trial_steps, swe_tune* out) {
    NvtxRange nvtx_range("swe_autotune");
    if (!m || trial_steps < 0) { set_error("swe_autotune: bad arguments"); return SWE_EINVAL; }
    if (!m->have_state) { set_error("swe_autotune: no state set"); return SWE_EINVAL; }
    if (trial_steps == 0) trial_steps = 8;
    TuneDeviceGuard dg(m->cfg.device);
    int rc = flush_mesh_bc(m);
    if (rc) return rc;
    return m->cfg.precision == SWE_FP32 ? autotune_t<float>(m, trial_steps, out)
                                        : autotune_t<double>(m, trial_steps, out);
}

}  // extern "C"
