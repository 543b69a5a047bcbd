// swe_internal.h -- host-side structures shared by the mesh preprocessing and
// the C ABI of libswe.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/swe.h"
#include "swe_kernels.cuh"

namespace swe {

// A named NVTX range over a public call (swe_step, swe_adjoint, ...), for
// timeline tools; a no-op costing a few nanoseconds when none is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Result of the host preprocessing (Section 3.1 geometry, neighbours across
// shared edges, locality order), in the internal cell order.
struct HostMesh {
    int64_t n_cells = 0, n_nodes = 0;
    std::vector<int64_t> perm;      // perm[new] = caller index
    std::vector<int64_t> inv;       // inv[caller] = new
    std::vector<int32_t> tri;       // [n][3] counter-clockwise, internal order
    std::vector<double> ln;         // [n][3][2] L_ij n_ij (outward, times edge length)
    std::vector<double> inv_area;   // 1/|Omega_i|
    std::vector<double> rin;        // inscribed radius 2|Omega|/perimeter
    std::vector<double> z, m;       // bed elevation, Manning n
    std::vector<int32_t> code;      // [n][3] neighbour code: k | flip bit, or -1 - group
    std::vector<double> len;        // [n][3] edge length (FP64, for BC group lengths)
    std::vector<int64_t> bslot;     // boundary half-edge slots (3 i + j), sorted by node key
    std::vector<uint64_t> bkey;     // matching sorted keys (min node << 32 | max node)
};

// Builds the host mesh; returns SWE_OK or an error code with a message.
int build_host_mesh(const double* nodes, int64_t n_nodes, const int32_t* tris, int64_t n_tris,
                    const double* bathy, const double* manning, int reorder, bool pair_cells,
                    HostMesh& out, std::string& err);

// Locality orderings of the cells; each returns order[new] = old.
std::vector<int64_t> order_hilbert(const std::vector<double>& cx, const std::vector<double>& cy);
std::vector<int64_t> order_rcm(int64_t n, const std::vector<int64_t>& nbr /* [n][3], -1 = none */);
// A matching of adjacent cells: a greedy pass along `along` (order[new] =
// old) matches each unmatched cell with its unmatched neighbour that comes
// soonest after it, at most 256 places later; mate[c] = the partner of cell c
// (caller numbering) or -1, rot[c] = the local edge of c (counter-clockwise
// nodes t) that it shares with its partner, 0 when unmatched.  Deterministic.
void match_cells(const std::vector<int64_t>& along, const std::vector<int64_t>& nbr, const std::vector<int32_t>& t,
                 std::vector<int64_t>& mate, std::vector<int>& rot);
// A locality order rearranged so that positions (2p, 2p+1) hold matched
// pairs, each at its first cell's place; unmatched cells go in segments of 64
// of their own, kept near their place, so that a warp's 32 pairs are all
// matched or all unmatched.
std::vector<int64_t> place_pairs(const std::vector<int64_t>& order, const std::vector<int64_t>& mate);

// Thread-local error message of the C ABI.
void set_error(const std::string& msg);

// A launch shape of the step kernel.
struct LaunchShape {
    int block = 0, min_blocks = 0, stages = 0, geo = 0, edges = 0;
    unsigned grid = 0;
    int pairs = 0;   // the cell-pair kernel (FP32): grid blocks over (n + 1) / 2 pairs
};

// Words of a mesh's device status block.
constexpr int kSmallWords = 8;
constexpr int kSlotT = 3, kSlotStatus = 4, kSlotClamp = 5, kSlotActive = 6, kSlotDtLast = 7;

}  // namespace swe

struct swe_mesh;

namespace swe {
// One step of mesh m from state buffer `in` to `out` (see swe_capi.cu).  With
// with_activity (and the mesh's activity mode on) the step reads and maintains
// the mesh's activity bytes: only for `in` = the mesh's current state.
// With the edge pass, eflux_out / esrc_out (when set) receive the step's edge
// fluxes instead of the mesh's own buffers.
cudaError_t launch_step_raw(swe_mesh* m, const void* in, void* out, unsigned long long* small, int64_t step_index,
                            double cfl, const double* dt_fixed, double* dt_log, cudaStream_t st,
                            bool with_activity = false, void* eflux_out = nullptr, void* esrc_out = nullptr);
// Allocates (once) and fills the activity bytes of m's current state.
int init_activity(swe_mesh* m);
// Builds (once) the interior-edge list of the edge-pass step.
int build_edges(swe_mesh* m);
// Appends the interior edges of H, its cells numbered from `base`, in canonical
// orientation (each once, from its left cell, in the order of that cell):
// (left, right), the left cell's L n, and into eidx[0 .. H.n_cells) each
// cell's edge per local edge (-1 on the boundary).
void append_edges(const HostMesh& H, int64_t base, std::vector<int2>& cells, std::vector<double>& ln, int4* eidx,
                  std::vector<double>* rl = nullptr);
// 1/|L n| of an edge as every FP64 kernel takes it: 1/sqrt(fma(lx, lx, ly ly)),
// formed on the host with one rounding per operation (the same on every host).
double host_edge_rl(double lx, double ly);
// The activity kernel indexes cells with 32 bits: meshes below this size.
constexpr int64_t kActivityMaxCells = int64_t(1) << 29;
// Applies pending boundary-group changes of m to the device.
int flush_mesh_bc(swe_mesh* m);
// Drops m's captured CUDA graph (after a change of launch shape).
void drop_mesh_graph(swe_mesh* m);
}  // namespace swe

// One mesh: host preprocessing result, device arrays and stepping state.
struct swe_mesh {
    swe_config cfg{};
    swe::HostMesh hm;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    size_t esz = 8;                    // sizeof(T)
    void* state[2] = {nullptr, nullptr};
    void* geoA = nullptr;
    void* geoB = nullptr;
    void* geoR = nullptr;              // FP64: V4<double> 1/|L n| of the three edges
    int4* topo = nullptr;
    void* gm2 = nullptr;
    void* zdev = nullptr;
    long long* perm = nullptr;
    void* stage[3] = {nullptr, nullptr, nullptr};
    unsigned long long* small = nullptr;
    swe::BcTable bc{};
    std::vector<double> group_len;     // total edge length per group
    std::vector<double> group_value;   // Q or eta_s as given
    int n_groups = 1;
    bool topo_dirty = false;
    bool have_state = false;
    int64_t nstep = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_len = 0;
    double graph_cfl = -1.0;
    int64_t device_bytes = 0;
    unsigned grid = 0;                 // blocks of the step kernel (about one resident wave)
    // activity bytes (cfg.activity): three rotating buffers of act_len bytes;
    // act_valid says that the one step nstep reads describes the current state
    unsigned char* act[3] = {nullptr, nullptr, nullptr};
    int64_t act_len = 0;
    bool act_valid = false;
    // shape of the steps that run without activity bytes (launch_step_raw for
    // other buffers: adjoint, frozen time steps); equals the cfg shape when
    // activity is off
    swe::LaunchShape plain;
    // edge pass (cfg.edge_pass): interior edges in canonical orientation
    int64_t n_edges = 0;
    int2* ecells = nullptr;            // (left, right)
    void* eln = nullptr;               // [E][2] T, L n outward from the left cell
    void* erl = nullptr;               // FP64: [E] 1/|L n|
    void* eflux = nullptr;             // V4<T>[E]
    void* esrc = nullptr;              // T[E]
    int4* eidx = nullptr;              // per cell, the edge of each local edge (-1: boundary)
    // reverse step of swe_adjoint: SWE_ADJOINT_TRANSPOSE or SWE_ADJOINT_DUAL
    int adjoint_method = SWE_ADJOINT_TRANSPOSE;
};


