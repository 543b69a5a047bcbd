// swe_launch.cuh -- definitions of the per-precision launchers; included by
// exactly one translation unit per precision (swe_step_f32.cu, swe_step_f64.cu).
#pragma once

#include "swe_kernels.cuh"

namespace swe {

template <typename T>
static inline unsigned grid_for(long long n, int block) {
    return (unsigned)((n + block - 1) / block);
}

// Compiled (block, min blocks per SM, stages, geometry early) variants of
// the step kernel.  FP32 variants trade registers for occupancy; FP64 keeps
// its registers (its FP64 pipe, not memory latency, is the limit).  Every
// FP32 variant stays within the 48 KB of static shared memory a block may
// declare.  Geometry-early variants suit wet meshes (one memory round trip
// fewer per active cell), the others mostly dry ones (no geometry traffic for
// quiet cells); the autotuner chooses.
#define SWE_STEP_VARIANTS_F32(X)                                                                       \
    X(128, 1, 1, 0) X(256, 1, 1, 0) X(512, 1, 1, 0) X(128, 8, 1, 0) X(256, 4, 1, 0) X(256, 5, 1, 0)    \
    X(512, 2, 1, 0) X(256, 4, 2, 0) X(256, 4, 3, 0) X(256, 4, 4, 0) X(128, 8, 3, 0) X(128, 8, 4, 0)    \
    X(256, 4, 1, 1) X(256, 4, 3, 1) X(128, 8, 1, 1) X(128, 8, 3, 1)
#define SWE_STEP_VARIANTS_F64(X) \
    X(128, 1, 1, 0) X(256, 1, 1, 0) X(512, 1, 1, 0) X(128, 1, 2, 0) X(256, 1, 2, 0) X(128, 1, 1, 1) X(256, 1, 1, 1)

// (block, min blocks per SM, stages, geometry early) shapes of the cell pass of
// the edge-pass step (edge_flux_kernel runs before it with 256-thread blocks)
#define SWE_EDGE_VARIANTS_F32(X) X(256, 4, 1, 0) X(128, 8, 1, 0)
#define SWE_EDGE_VARIANTS_F64(X) X(128, 1, 1, 0) X(256, 1, 1, 0)
constexpr int kEdgeBlock = 256;

// (block, min blocks per SM, geometry early, stages) shapes of the activity
// kernel; stages = the state's prefetch distance + 1.  Shared memory per
// thread: `stages` state records and activity bytes, 2 topology records.
#define SWE_ACT_VARIANTS_F32(X)                                                                     \
    X(128, 8, 0, 3) X(256, 4, 0, 3) X(512, 2, 0, 3) X(128, 8, 1, 3) X(256, 4, 1, 3) X(128, 8, 1, 4) \
    X(128, 8, 1, 5) X(256, 4, 1, 4) X(128, 8, 0, 4)
#define SWE_ACT_VARIANTS_F64(X) X(128, 1, 0, 3) X(256, 1, 0, 3) X(128, 1, 1, 3) X(128, 1, 0, 4)

template <typename T>
int Launch<T>::default_min_blocks(int block) {
    if (sizeof(T) == 8) return 1;
    return block == 128 ? 8 : (block == 256 ? 4 : 2);
}

template <typename T>
cudaError_t Launch<T>::step(const StepArgs<T>& a, int block, int min_blocks, int stages, int geo_early,
                            cudaStream_t st) {
    const unsigned grid = a.grid;
    if (grid == 0) return cudaErrorInvalidValue;
    if (a.act_in) {
#define SWE_LAUNCH_ACT(B, M, G, S) \
    if (block == B && min_blocks == M && geo_early == G && stages == S) {         \
        step_kernel_act<T, B, M, G != 0, S - 1><<<grid, B, 0, st>>>(a);          \
        return cudaGetLastError();                                                \
    }
        if constexpr (sizeof(T) == 4) {
            SWE_ACT_VARIANTS_F32(SWE_LAUNCH_ACT)
        } else {
            SWE_ACT_VARIANTS_F64(SWE_LAUNCH_ACT)
        }
#undef SWE_LAUNCH_ACT
        return cudaErrorInvalidValue;
    }
    if (a.eflux) {
        cudaError_t e = edge_flux(a, st);
        if (e != cudaSuccess) return e;
#define SWE_LAUNCH_EDGE(B, M, S, G) \
    if (block == B && min_blocks == M && stages == S && geo_early == G) {        \
        step_kernel<T, B, M, S, G != 0, true><<<grid, B, 0, st>>>(a);            \
        return cudaGetLastError();                                                \
    }
        if constexpr (sizeof(T) == 4) {
            SWE_EDGE_VARIANTS_F32(SWE_LAUNCH_EDGE)
        } else {
            SWE_EDGE_VARIANTS_F64(SWE_LAUNCH_EDGE)
        }
#undef SWE_LAUNCH_EDGE
        return cudaErrorInvalidValue;
    }
#define SWE_LAUNCH(B, M, S, G) \
    if (block == B && min_blocks == M && stages == S && geo_early == G) {        \
        step_kernel<T, B, M, S, G != 0><<<grid, B, 0, st>>>(a);                  \
        return cudaGetLastError();                                                \
    }
    if constexpr (sizeof(T) == 4) {
        SWE_STEP_VARIANTS_F32(SWE_LAUNCH)
    } else {
        SWE_STEP_VARIANTS_F64(SWE_LAUNCH)
    }
#undef SWE_LAUNCH
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Launch<T>::resident_blocks(int block, int min_blocks, int stages, int geo_early, int activity,
                                       int edges, int* per_sm) {
    if (edges) {
#define SWE_OCC_EDGE(B, M, S, G) \
    if (block == B && min_blocks == M && stages == S && geo_early == G)          \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_kernel<T, B, M, S, G != 0, true>, B, 0);
        if constexpr (sizeof(T) == 4) {
            SWE_EDGE_VARIANTS_F32(SWE_OCC_EDGE)
        } else {
            SWE_EDGE_VARIANTS_F64(SWE_OCC_EDGE)
        }
#undef SWE_OCC_EDGE
        return cudaErrorInvalidValue;
    }
    if (activity) {
#define SWE_OCC_ACT(B, M, G, S) \
    if (block == B && min_blocks == M && geo_early == G && stages == S)           \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_kernel_act<T, B, M, G != 0, S - 1>, B, 0);
        if constexpr (sizeof(T) == 4) {
            SWE_ACT_VARIANTS_F32(SWE_OCC_ACT)
        } else {
            SWE_ACT_VARIANTS_F64(SWE_OCC_ACT)
        }
#undef SWE_OCC_ACT
        return cudaErrorInvalidValue;
    }
#define SWE_OCC(B, M, S, G) \
    if (block == B && min_blocks == M && stages == S && geo_early == G)          \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_kernel<T, B, M, S, G != 0>, B, 0);
    if constexpr (sizeof(T) == 4) {
        SWE_STEP_VARIANTS_F32(SWE_OCC)
    } else {
        SWE_STEP_VARIANTS_F64(SWE_OCC)
    }
#undef SWE_OCC
    return cudaErrorInvalidValue;
}

template <typename T>
int Launch<T>::step_variants(int (*out)[4], int max) {
    int k = 0;
#define SWE_LIST(B, M, S, G) \
    if (k < max) { out[k][0] = B; out[k][1] = M; out[k][2] = S; out[k][3] = G; } \
    ++k;
    if constexpr (sizeof(T) == 4) {
        SWE_STEP_VARIANTS_F32(SWE_LIST)
    } else {
        SWE_STEP_VARIANTS_F64(SWE_LIST)
    }
#undef SWE_LIST
    return k;
}

// (block, min blocks per SM, geometry early, stages) shapes of the cell-pair
// step (FP32); stages is 1 (records read directly).  On the fully wet 13M
// river (0.270 ms per step at 256 x 4) a cp.async pipeline of pair records
// measured slower (2 or 3 pairs ahead: 0.285-0.353 ms, spilling at 64
// registers), and so did copying the second cell's records, or those and the
// next pair's first, into shared memory during the first cell's update
// (0.272 and 0.280 ms), and so did an L2 bulk prefetch of each warp's records
// one or two grid-stride iterations ahead (0.275 and 0.282 against 0.265 ms at
// 256 x 4): the pair kernel has none.
#define SWE_PAIR_VARIANTS_F32(X) X(256, 4, 0, 1) X(256, 4, 1, 1) X(128, 8, 1, 1) X(128, 8, 0, 1) X(256, 3, 1, 1)

template <typename T>
cudaError_t Launch<T>::step_pair(const StepArgs<T>& a, int block, int min_blocks, int geo_early, int stages,
                                 cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (a.grid == 0) return cudaErrorInvalidValue;
#define SWE_LAUNCH_PAIR(B, M, G, S) \
    if (block == B && min_blocks == M && geo_early == G && stages == S) {      \
        step_kernel_pair<B, M, G != 0><<<a.grid, B, 0, st>>>(a);            \
        return cudaGetLastError();                                              \
    }
        SWE_PAIR_VARIANTS_F32(SWE_LAUNCH_PAIR)
#undef SWE_LAUNCH_PAIR
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Launch<T>::pair_resident_blocks(int block, int min_blocks, int geo_early, int stages, int* per_sm) {
    if constexpr (sizeof(T) == 4) {
#define SWE_OCC_PAIR(B, M, G, S) \
    if (block == B && min_blocks == M && geo_early == G && stages == S)        \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_kernel_pair<B, M, G != 0>, B, 0);
        SWE_PAIR_VARIANTS_F32(SWE_OCC_PAIR)
#undef SWE_OCC_PAIR
    }
    return cudaErrorInvalidValue;
}

template <typename T>
int Launch<T>::pair_variants(int (*out)[4], int max) {
    int k = 0;
    if constexpr (sizeof(T) == 4) {
#define SWE_LIST(B, M, G, S) \
    if (k < max) { out[k][0] = B; out[k][1] = M; out[k][2] = G; out[k][3] = S; } \
    ++k;
        SWE_PAIR_VARIANTS_F32(SWE_LIST)
#undef SWE_LIST
    }
    return k;
}

template <typename T>
cudaError_t Launch<T>::edge_flux(const StepArgs<T>& a, cudaStream_t st) {
    if (a.n_edges <= 0) return cudaSuccess;
    const long long eb = (a.n_edges + kEdgeBlock - 1) / kEdgeBlock;
    const unsigned egrid = (unsigned)(eb < 65536 ? eb : 65536);
    edge_flux_kernel<T, kEdgeBlock><<<egrid, kEdgeBlock, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
int Launch<T>::edge_variants(int (*out)[4], int max) {
    int k = 0;
#define SWE_LIST(B, M, S, G) \
    if (k < max) { out[k][0] = B; out[k][1] = M; out[k][2] = S; out[k][3] = G; } \
    ++k;
    if constexpr (sizeof(T) == 4) {
        SWE_EDGE_VARIANTS_F32(SWE_LIST)
    } else {
        SWE_EDGE_VARIANTS_F64(SWE_LIST)
    }
#undef SWE_LIST
    return k;
}

template <typename T>
int Launch<T>::act_variants(int (*out)[4], int max) {
    int k = 0;
#define SWE_LIST(B, M, G, S) \
    if (k < max) { out[k][0] = B; out[k][1] = M; out[k][2] = G; out[k][3] = S; } \
    ++k;
    if constexpr (sizeof(T) == 4) {
        SWE_ACT_VARIANTS_F32(SWE_LIST)
    } else {
        SWE_ACT_VARIANTS_F64(SWE_LIST)
    }
#undef SWE_LIST
    return k;
}

template <typename T>
cudaError_t Launch<T>::act_init(const V4<T>* s, const int4* topo, long long n, T h_dry, unsigned char* act,
                                cudaStream_t st) {
    act_init_kernel<T><<<grid_for<T>(n, 256), 256, 0, st>>>(s, topo, n, h_dry, act);
    return cudaGetLastError();
}

// Compiled (block, min blocks per SM, stages, geometry early) shapes of the
// ensemble kernel; the first of each list is the default.  Blocks divide the
// 256-cell padding.
#define SWE_ENS_VARIANTS_F32(X)                                                                    \
    X(256, 4, 3, 0) X(256, 4, 1, 0) X(256, 4, 2, 0) X(128, 8, 3, 0) X(128, 8, 1, 0) X(256, 4, 3, 1) \
    X(256, 4, 1, 1) X(128, 8, 3, 1) X(128, 8, 1, 1)
#define SWE_ENS_VARIANTS_F64(X) \
    X(256, 1, 1, 0) X(128, 1, 1, 0) X(256, 1, 2, 0) X(128, 1, 2, 0) X(256, 1, 1, 1) X(128, 1, 1, 1)

template <typename T>
void Launch<T>::ensemble_default(int* block, int* min_blocks, int* stages, int* geo_early) {
    int v[1][4];
    ensemble_variants(v, 1);
    *block = v[0][0];
    *min_blocks = v[0][1];
    *stages = v[0][2];
    *geo_early = v[0][3];
}

template <typename T>
int Launch<T>::ensemble_variants(int (*out)[4], int max) {
    int k = 0;
#define SWE_LIST(B, M, S, G) \
    if (k < max) { out[k][0] = B; out[k][1] = M; out[k][2] = S; out[k][3] = G; } \
    ++k;
    if constexpr (sizeof(T) == 4) {
        SWE_ENS_VARIANTS_F32(SWE_LIST)
    } else {
        SWE_ENS_VARIANTS_F64(SWE_LIST)
    }
#undef SWE_LIST
    return k;
}

// (block, min blocks per SM, stages, geometry early) shapes of the ensemble's
// edge-pass cell kernel (FP64 only: the edge pass pays where the FP64 pipe bounds the step)
#define SWE_ENS_EDGE_VARIANTS_F32(X)
#define SWE_ENS_EDGE_VARIANTS_F64(X) X(256, 1, 1, 0) X(128, 1, 1, 0)

template <typename T>
int Launch<T>::ensemble_edge_variants(int (*out)[4], int max) {
    int k = 0;
#define SWE_LIST(B, M, S, G) \
    if (k < max) { out[k][0] = B; out[k][1] = M; out[k][2] = S; out[k][3] = G; } \
    ++k;
    if constexpr (sizeof(T) == 4) {
        SWE_ENS_EDGE_VARIANTS_F32(SWE_LIST)
    } else {
        SWE_ENS_EDGE_VARIANTS_F64(SWE_LIST)
    }
#undef SWE_LIST
    return k;
}

template <typename T>
cudaError_t Launch<T>::ensemble_edge_resident_blocks(int block, int min_blocks, int stages, int geo_early,
                                                     int* per_sm) {
#define SWE_OCC(B, M, S, G) \
    if (block == B && min_blocks == M && stages == S && geo_early == G)          \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, ensemble_step_kernel<T, B, M, S, G != 0, true>, \
                                                             B, 0);
    if constexpr (sizeof(T) == 4) {
        SWE_ENS_EDGE_VARIANTS_F32(SWE_OCC)
    } else {
        SWE_ENS_EDGE_VARIANTS_F64(SWE_OCC)
    }
#undef SWE_OCC
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Launch<T>::ensemble_step(const EnsArgs<T>& a, int block, int min_blocks, int stages, int geo_early,
                                     unsigned grid, cudaStream_t st) {
    if (grid == 0) return cudaErrorInvalidValue;
    if (a.eflux) {
        StepArgs<T> ea{};
        ea.s_in = a.s_in;
        ea.ecells = a.ecells;
        ea.eln = a.eln;
        ea.erl = a.erl;
        ea.eflux = a.eflux;
        ea.esrc = a.esrc;
        ea.n_edges = a.n_edges;
        ea.g = a.g;
        ea.h_dry = a.h_dry;
        ea.hll = a.hll;
        ea.n = a.n_total;
        ea.debug = a.debug;
        ea.n_groups = a.n_groups;
        ea.status = (unsigned*)(a.small + 4);   // a bad edge is reported through the first member
        cudaError_t e = edge_flux(ea, st);
        if (e != cudaSuccess) return e;
#define SWE_LAUNCH_EDGE(B, M, S, G) \
    if (block == B && min_blocks == M && stages == S && geo_early == G) {        \
        ensemble_step_kernel<T, B, M, S, G != 0, true><<<grid, B, 0, st>>>(a);   \
        return cudaGetLastError();                                                \
    }
        if constexpr (sizeof(T) == 4) {
            SWE_ENS_EDGE_VARIANTS_F32(SWE_LAUNCH_EDGE)
        } else {
            SWE_ENS_EDGE_VARIANTS_F64(SWE_LAUNCH_EDGE)
        }
#undef SWE_LAUNCH_EDGE
        return cudaErrorInvalidValue;
    }
#define SWE_LAUNCH(B, M, S, G) \
    if (block == B && min_blocks == M && stages == S && geo_early == G) {        \
        ensemble_step_kernel<T, B, M, S, G != 0><<<grid, B, 0, st>>>(a);         \
        return cudaGetLastError();                                                \
    }
    if constexpr (sizeof(T) == 4) {
        SWE_ENS_VARIANTS_F32(SWE_LAUNCH)
    } else {
        SWE_ENS_VARIANTS_F64(SWE_LAUNCH)
    }
#undef SWE_LAUNCH
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Launch<T>::ensemble_resident_blocks(int block, int min_blocks, int stages, int geo_early,
                                                int* per_sm) {
#define SWE_OCC(B, M, S, G) \
    if (block == B && min_blocks == M && stages == S && geo_early == G)          \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, ensemble_step_kernel<T, B, M, S, G != 0>, B, 0);
    if constexpr (sizeof(T) == 4) {
        SWE_ENS_VARIANTS_F32(SWE_OCC)
    } else {
        SWE_ENS_VARIANTS_F64(SWE_OCC)
    }
#undef SWE_OCC
    return cudaErrorInvalidValue;
}

// (block, min blocks per SM, geometry early) shapes of the ensemble's activity kernel
#define SWE_ENS_ACT_VARIANTS_F32(X) X(128, 8, 1) X(128, 8, 0) X(256, 4, 1) X(256, 4, 0) X(128, 7, 1)
#define SWE_ENS_ACT_VARIANTS_F64(X) X(256, 1, 0) X(128, 1, 0)

// (block, min blocks per SM, geometry early) shapes of the ensemble's activity
// kernel with per-warp queues of the cells that run the flux path (FP32); at
// 8 blocks of 128 (64 registers) the queue's state spills 40-60 B
#define SWE_ENS_ACTQ_VARIANTS_F32(X) X(128, 7, 1) X(128, 7, 0) X(128, 6, 1)

template <typename T>
cudaError_t Launch<T>::ensemble_step_act(const EnsArgs<T>& a, int block, int min_blocks, int geo_early,
                                         unsigned grid, cudaStream_t st, int dynamic, int queue) {
    if (grid == 0 || !a.act_in || (dynamic && (!a.sched || a.chunk_log2 < 2))) return cudaErrorInvalidValue;
    if (queue) {
        if constexpr (sizeof(T) == 4) {
#define SWE_LAUNCH(B, M, G) \
    if (block == B && min_blocks == M && geo_early == G) {                                       \
        if (dynamic) ensemble_step_kernel_act<T, B, M, G != 0, true, true><<<grid, B, 0, st>>>(a); \
        else ensemble_step_kernel_act<T, B, M, G != 0, false, true><<<grid, B, 0, st>>>(a);     \
        return cudaGetLastError();                                                               \
    }
            SWE_ENS_ACTQ_VARIANTS_F32(SWE_LAUNCH)
#undef SWE_LAUNCH
        }
        return cudaErrorInvalidValue;
    }
#define SWE_LAUNCH(B, M, G) \
    if (block == B && min_blocks == M && geo_early == G) {                        \
        if (dynamic) ensemble_step_kernel_act<T, B, M, G != 0, true><<<grid, B, 0, st>>>(a); \
        else ensemble_step_kernel_act<T, B, M, G != 0><<<grid, B, 0, st>>>(a);   \
        return cudaGetLastError();                                                \
    }
    if constexpr (sizeof(T) == 4) {
        SWE_ENS_ACT_VARIANTS_F32(SWE_LAUNCH)
    } else {
        SWE_ENS_ACT_VARIANTS_F64(SWE_LAUNCH)
    }
#undef SWE_LAUNCH
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Launch<T>::ensemble_act_resident_blocks(int block, int min_blocks, int geo_early, int* per_sm,
                                                    int dynamic, int queue) {
    if (queue) {
        if constexpr (sizeof(T) == 4) {
#define SWE_OCC(B, M, G) \
    if (block == B && min_blocks == M && geo_early == G)                                         \
        return dynamic ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(                           \
                             per_sm, ensemble_step_kernel_act<T, B, M, G != 0, true, true>, B, 0)  \
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(                           \
                             per_sm, ensemble_step_kernel_act<T, B, M, G != 0, false, true>, B, 0);
            SWE_ENS_ACTQ_VARIANTS_F32(SWE_OCC)
#undef SWE_OCC
        }
        return cudaErrorInvalidValue;
    }
#define SWE_OCC(B, M, G) \
    if (block == B && min_blocks == M && geo_early == G)                          \
        return dynamic ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(             \
                             per_sm, ensemble_step_kernel_act<T, B, M, G != 0, true>, B, 0) \
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(             \
                             per_sm, ensemble_step_kernel_act<T, B, M, G != 0>, B, 0);
    if constexpr (sizeof(T) == 4) {
        SWE_ENS_ACT_VARIANTS_F32(SWE_OCC)
    } else {
        SWE_ENS_ACT_VARIANTS_F64(SWE_OCC)
    }
#undef SWE_OCC
    return cudaErrorInvalidValue;
}

template <typename T>
int Launch<T>::ensemble_actq_variants(int (*out)[3], int max) {
    int k = 0;
    if constexpr (sizeof(T) == 4) {
#define SWE_LIST(B, M, G) \
    if (k < max) { out[k][0] = B; out[k][1] = M; out[k][2] = G; } \
    ++k;
        SWE_ENS_ACTQ_VARIANTS_F32(SWE_LIST)
#undef SWE_LIST
    }
    return k;
}

template <typename T>
int Launch<T>::ensemble_act_variants(int (*out)[3], int max) {
    int k = 0;
#define SWE_LIST(B, M, G) \
    if (k < max) { out[k][0] = B; out[k][1] = M; out[k][2] = G; } \
    ++k;
    if constexpr (sizeof(T) == 4) {
        SWE_ENS_ACT_VARIANTS_F32(SWE_LIST)
    } else {
        SWE_ENS_ACT_VARIANTS_F64(SWE_LIST)
    }
#undef SWE_LIST
    return k;
}

// (block, min blocks per SM, geometry early) shapes of the dynamically scheduled ensemble kernel
#define SWE_ENS_DYN_VARIANTS_F32(X) X(128, 8, 0) X(128, 8, 1) X(256, 4, 0) X(128, 7, 1) X(128, 6, 1)
#define SWE_ENS_DYN_VARIANTS_F64(X) X(128, 1, 0) X(256, 1, 0)

template <typename T>
cudaError_t Launch<T>::ensemble_step_dyn(const EnsArgs<T>& a, int block, int min_blocks, int geo_early,
                                         unsigned grid, cudaStream_t st) {
    if (grid == 0 || !a.sched) return cudaErrorInvalidValue;
#define SWE_LAUNCH(B, M, G) \
    if (block == B && min_blocks == M && geo_early == G) {                        \
        ensemble_step_kernel_dyn<T, B, M, G != 0><<<grid, B, 0, st>>>(a);        \
        return cudaGetLastError();                                                \
    }
    if constexpr (sizeof(T) == 4) {
        SWE_ENS_DYN_VARIANTS_F32(SWE_LAUNCH)
    } else {
        SWE_ENS_DYN_VARIANTS_F64(SWE_LAUNCH)
    }
#undef SWE_LAUNCH
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Launch<T>::ensemble_dyn_resident_blocks(int block, int min_blocks, int geo_early, int* per_sm) {
#define SWE_OCC(B, M, G) \
    if (block == B && min_blocks == M && geo_early == G)                          \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, ensemble_step_kernel_dyn<T, B, M, G != 0>, B, 0);
    if constexpr (sizeof(T) == 4) {
        SWE_ENS_DYN_VARIANTS_F32(SWE_OCC)
    } else {
        SWE_ENS_DYN_VARIANTS_F64(SWE_OCC)
    }
#undef SWE_OCC
    return cudaErrorInvalidValue;
}

template <typename T>
int Launch<T>::ensemble_dyn_variants(int (*out)[3], int max) {
    int k = 0;
#define SWE_LIST(B, M, G) \
    if (k < max) { out[k][0] = B; out[k][1] = M; out[k][2] = G; } \
    ++k;
    if constexpr (sizeof(T) == 4) {
        SWE_ENS_DYN_VARIANTS_F32(SWE_LIST)
    } else {
        SWE_ENS_DYN_VARIANTS_F64(SWE_LIST)
    }
#undef SWE_LIST
    return k;
}

// (min blocks per SM, geometry early) shapes of the split ensemble's
// cell-pair kernel (128-thread blocks: 128 pairs are one kEnsPad span)
#define SWE_ENS_PAIR_VARIANTS_F32(X) X(8, 1) X(8, 0) X(7, 1)

template <typename T>
cudaError_t Launch<T>::ensemble_step_pair(const EnsArgs<T>& a, int min_blocks, int geo_early, unsigned grid,
                                          cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (grid == 0) return cudaErrorInvalidValue;
        if (a.pair_spans == 0) return cudaSuccess;
#define SWE_LAUNCH(M, G) \
    if (min_blocks == M && geo_early == G) {                                             \
        ensemble_step_kernel_pair<128, M, G != 0><<<grid, 128, 0, st>>>(a);             \
        return cudaGetLastError();                                                       \
    }
        SWE_ENS_PAIR_VARIANTS_F32(SWE_LAUNCH)
#undef SWE_LAUNCH
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Launch<T>::ensemble_pair_resident_blocks(int min_blocks, int geo_early, int* per_sm) {
    if constexpr (sizeof(T) == 4) {
#define SWE_OCC(M, G) \
    if (min_blocks == M && geo_early == G)                                               \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, ensemble_step_kernel_pair<128, M, G != 0>, 128, 0);
        SWE_ENS_PAIR_VARIANTS_F32(SWE_OCC)
#undef SWE_OCC
    }
    return cudaErrorInvalidValue;
}

template <typename T>
int Launch<T>::ensemble_pair_variants(int (*out)[2], int max) {
    int k = 0;
    if constexpr (sizeof(T) == 4) {
#define SWE_LIST(M, G) \
    if (k < max) { out[k][0] = M; out[k][1] = G; } \
    ++k;
        SWE_ENS_PAIR_VARIANTS_F32(SWE_LIST)
#undef SWE_LIST
    }
    return k;
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
                               int hll, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    riemann_batch_kernel<T><<<grid_for<T>(n, 256), 256, 0, st>>>(n, hL, unL, utL, hR, unR, utR, g, h_dry,
                                                                   G1, G2, G3, S, hll);
    return cudaGetLastError();
}

}  // namespace swe
