/*
 * swe.h -- C ABI of libswe, a single-GPU (GB300, sm_103a) time-explicit
 * finite-volume solver for the 2D shallow-water equations on unstructured
 * triangular meshes.
 *
 * The method is the one of Delmas & Soulaimani, "Multi-GPU implementation of
 * a time-explicit finite volume solver for the Shallow-Water Equations using
 * CUDA and a CUDA-Aware version of OpenMPI", Sections 2-3:
 *   U = (h, hu, hv) cell averages on triangles (Eq 1-11), edge fluxes by the
 *   HLLC Riemann solver in the edge-normal frame (Eq 12-14, 17-26), bed slope
 *   by hydrostatic reconstruction (Eq 28-30), semi-implicit Manning friction
 *   (Eq 31-37), explicit Euler with the CFL step on the inscribed radius
 *   (Eq 15-16), boundary conditions of Section 3.1.
 *
 * Conventions for every call:
 *   - Return value: SWE_OK (0) or one of the SWE_E* codes below.  A message
 *     for the last failure of the calling thread is in swe_last_error().
 *     No C++ exception crosses this interface.
 *   - Arrays are dense, C order, in the caller's own cell/node numbering.
 *     The library keeps an internal locality ordering of the cells and never
 *     exposes it except through swe_get_permutation().
 *   - The library copies every input array; no caller pointer is retained
 *     after a call returns.
 *   - Floating-point state arrays are double for SWE_FP64 meshes and float for
 *     SWE_FP32 meshes (FP32 state, FP64 time step and time).
 *   - Device pointers (where = SWE_DEVICE) must be on the mesh's device and
 *     are used in stream order on the mesh's stream.
 *   - Calls on one mesh are not thread-safe; distinct meshes are independent.
 */
#ifndef SWE_H
#define SWE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SWE_API __attribute__((visibility("default")))
#else
#define SWE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SWE_OK 0
#define SWE_EINVAL 1     /* bad argument */
#define SWE_EMESH 2      /* malformed mesh: bad index, zero area, edge shared by > 2 cells */
#define SWE_ENOMEM 3     /* host or device allocation failed */
#define SWE_ECUDA 4      /* a CUDA runtime call failed */
#define SWE_ENONFINITE 5 /* a step produced a non-finite state */
#define SWE_EDRY 6       /* every cell is dry: the CFL step (Eq 15) does not exist */
#define SWE_ETIMEOUT 7   /* a bounded device-side wait gave up; reserved: no kernel of this
                            library waits on another block or device (each step is one
                            or two kernel launches, ordered by the stream) */

/* ---- enums ---- */
#define SWE_FP64 0
#define SWE_FP32 1

#define SWE_REORDER_NONE 0
#define SWE_REORDER_RCM 1     /* reverse Cuthill-McKee on the cell adjacency graph */
#define SWE_REORDER_HILBERT 2 /* Hilbert curve through the cell centroids */

#define SWE_BC_WALL 0         /* Section 3.1: inflow with Q = 0, G~ = (0, g h^2/2, 0) */
#define SWE_BC_INFLOW 1       /* Section 3.1: G~ = (-q, q^2/h + g h^2/2, 0), q = Q / group length */
#define SWE_BC_TRANSMISSIVE 2 /* Section 3.1: Riemann problem with U_R = U_L */
#define SWE_BC_STAGE 3        /* fixed free surface eta_s: ghost depth max(0, eta_s - z) */

#define SWE_HOST 0
#define SWE_DEVICE 1

#define SWE_FLUX_HLLC 0       /* Eq 17-25 with the HLLC third component (Eq 24), the paper's scheme */
#define SWE_FLUX_HLL 1        /* Eq 17-18 for all three components (the HLL flux the paper starts from) */

#define SWE_ADJOINT_TRANSPOSE 0 /* reverse step by hand-written transposes, each interior edge once */
#define SWE_ADJOINT_DUAL 1      /* reverse step on forward-mode dual numbers, each edge from both cells */

typedef struct swe_mesh swe_mesh;

typedef struct swe_config {
    int precision;    /* SWE_FP64 (default) or SWE_FP32 */
    double g;         /* gravitational acceleration, default 9.81 m/s^2; finite and > 0 */
    double h_dry;     /* wet/dry threshold, default 1e-6 m; finite and >= FLT_MIN (1.18e-38): a wet
                         depth is then a normal float, which the FP32 kernels and the FP64 friction
                         term's h^(-1/3) iteration (started from the float cube root) need */
    int reorder;      /* SWE_REORDER_*, default SWE_REORDER_HILBERT.  FP32 meshes: with RCM or
                         HILBERT the cells of the order are then arranged in pairs (2p, 2p+1)
                         that share an edge, made the local edge 0 of both, wherever a greedy
                         matching along the Hilbert order finds one (cell_pairs uses them);
                         FP64 meshes keep the caller's local edge numbering */
    int block_size;   /* threads per block of the step kernel; 0 = library default */
    int graph_steps;  /* steps captured per CUDA graph; 0 = default, < 0 = no graphs */
    int device;       /* CUDA device ordinal, default 0 */
    int min_blocks;   /* resident blocks per SM the step kernel is compiled for; 0 = default.
                         0 = default (FP32: 2048 / (2 block_size), FP64: 1) */
    int stages;       /* depth of the per-thread cp.async pipeline that stages the next cells'
                         state and topology records in shared memory; 1 = direct loads;
                         0 = default (FP32: 3, FP64: 1).  Compiled (block_size, min_blocks,
                         stages): FP32 (128|256|512, 1, 1), (128, 8, 1), (256, 4|5, 1),
                         (512, 2, 1), (256, 4, 2|3|4), (128, 8, 3|4); FP64 (128|256|512, 1, 1),
                         (128|256, 1, 2); others give SWE_EINVAL */
    int flux;         /* SWE_FLUX_HLLC (default) or SWE_FLUX_HLL */
    int geometry_early; /* 1: a cell's geometry is loaded together with its neighbours' states
                           (one memory round trip fewer on wet meshes); 0 (default): only
                           after the test that skips dry cells among dry neighbours (no
                           geometry traffic for those).  Compiled with 1: FP32 (256, 4, 1|3),
                           (128, 8, 1|3); FP64 (128|256, 1, 1).  Results do not depend on it */
    int activity;     /* 1: keep one activity byte per cell (three rotating buffers, 3 bytes per
                         cell of device memory): a cell is active when it or a neighbour is wet
                         or it has an inflow/stage edge, and an inactive cell takes its update
                         (h, 0, 0) without reading its topology or its neighbours, and with no
                         store when it was inactive in the previous step too (the state in the
                         output buffer, two steps old, is then already the new one); each step
                         marks the cells that the next one must treat as active, and the two
                         steps after a change from outside (set_state, set_bc, the tuner)
                         store every state.  0 (default):
                         every cell tests its neighbours.  With activity, stages is the
                         prefetch distance of the streamed state plus one (default 3).
                         Compiled (block_size, min_blocks, geometry_early, stages) with 1:
                         FP32 (128, 8, 0, 3|4), (256, 4, 0, 3), (512, 2, 0, 3),
                         (128, 8, 1, 3|4|5), (256, 4, 1, 3|4); FP64 (128, 1, 0, 3|4),
                         (256, 1, 0, 3), (128, 1, 1, 3).  Results do not depend on it */
    int edge_pass;    /* 1: each step first evaluates every interior edge's flux once (one thread
                         per edge, from its left cell), then updates the cells from those
                         fluxes; 0 (default): each cell evaluates its own three edges, so every
                         interior flux is evaluated twice.  The edge pass halves the flux
                         arithmetic for more memory traffic: it pays where the arithmetic
                         bounds the step (FP64).  Compiled cell passes: FP32 (256, 4, 1),
                         (128, 8, 1); FP64 (128|256, 1, 1), all with geometry_early 0.  Not
                         with activity.  Results do not depend on it */
    int grid;         /* blocks launched per step by the step kernel (each block loops over its
                         share of the cells); 0 = default, one resident wave; larger values are
                         clamped to one cell per thread.  Results do not depend on it */
    int debug_checks; /* 1: every step, ensemble and adjoint kernel checks each neighbour index,
                         edge index and boundary group it is about to use against the mesh's
                         sizes (swe_debug_code_ok) before the access; an out-of-range one is not
                         used (the edge is taken as a wall) and sets a bit of the device status
                         word, which the next synchronising call returns as SWE_EMESH.  A stand-in
                         for a memory checker on the library's own index tables; it costs one
                         branch per cell when off.  0 (default): no checks.  Results of a valid
                         mesh do not depend on it */
    int cell_pairs;   /* FP32 only, not with activity or edge_pass.  1: each thread of the step
                         kernel updates the cell pair (2p, 2p+1); when the two share their local
                         edge 0, its flux is evaluated once for both (five Riemann problems per
                         pair instead of six).  stages must then be 0 or 1 (records read
                         directly).  Compiled (block_size, min_blocks, geometry_early): (256, 4,
                         0|1), (128, 8, 0|1), (256, 3, 1).  0 (default): one cell per thread.
                         Results do not depend on it */
} swe_config;

/* Fills *cfg with the defaults listed above. */
SWE_API void swe_config_default(swe_config* cfg);

/*
 * The check that swe_config.debug_checks applies to each neighbour code
 * before it is used (the paper keeps each cell's neighbours in a table,
 * Section 4.2; here a code >= 0 names a neighbour cell, bit 30 marking the
 * edge's right side, and a code < 0 names boundary group -1 - code).
 * Returns 1 when the code can be used on a mesh of n_cells cells with
 * n_groups boundary groups: an interior code whose cell index (bits 0-29) is
 * below n_cells, or a boundary code whose group is below n_groups; else 0.
 * Host-callable, touches no device.
 */
SWE_API int swe_debug_code_ok(int32_t code, int64_t n_cells, int n_groups);

/*
 * Builds a mesh (Section 3.1): orients every triangle counter-clockwise, finds
 * the neighbour across each edge, computes |Omega_i|, L_ij n_ij (Eq 9) and the
 * inscribed radius 2|Omega_i|/perimeter (Eq 15), reorders the cells for
 * locality and uploads everything to the device.  Every boundary edge starts
 * as a wall.
 *   nodes   [n_nodes][2] double, metres
 *   tris    [n_tris][3] int32, 0-based node indices, either orientation
 *   bathy   [n_tris] double, cell-centred bed elevation z (m), finite
 *   manning [n_tris] double, Manning coefficient m (s m^-1/3), finite and >= 0
 *   cfg     NULL for defaults
 *   out     receives the new mesh (owned by the caller; free with swe_mesh_destroy)
 * Errors: SWE_EINVAL (NULL pointers, n < 1, n_tris >= 2^30, a negative or
 * non-finite Manning coefficient, a non-finite bed),
 * SWE_EMESH, SWE_ENOMEM, SWE_ECUDA.
 */
SWE_API int swe_mesh_create(const double* nodes, int64_t n_nodes, const int32_t* tris, int64_t n_tris,
                    const double* bathy, const double* manning, const swe_config* cfg,
                    swe_mesh** out);

/* Releases the mesh and all its host and device memory.  NULL is ignored. */
SWE_API void swe_mesh_destroy(swe_mesh* mesh);

/*
 * Puts the boundary edges given as node pairs into a new boundary group of
 * the given kind (Section 3.1).  value is the discharge Q (m^3/s) for
 * SWE_BC_INFLOW, spread uniformly over the group's total edge length, the
 * free-surface elevation eta_s (m) for SWE_BC_STAGE, and ignored otherwise.
 * An edge already in another group moves to the new one.
 *   node_pairs [n][2] int32 node indices of boundary edges, either order
 * Errors: SWE_EINVAL (a pair that is not a boundary edge, more than 63 groups).
 */
SWE_API int swe_set_bc(swe_mesh* mesh, const int32_t* node_pairs, int64_t n, int kind, double value);

/* Sets the CUDA stream (a cudaStream_t, NULL = legacy default stream) used by
 * all later calls on this mesh. */
SWE_API int swe_set_stream(swe_mesh* mesh, void* cuda_stream);

/*
 * Sets the state U = (h, hu, hv) and the time t, then computes the first CFL
 * step from it (Eq 15).  h, hu, hv: [n_tris] arrays of the mesh precision, on
 * the host (where = SWE_HOST; copied before return) or on the device
 * (SWE_DEVICE; read in stream order).  h must be >= 0 and finite.
 * Errors: SWE_EINVAL, SWE_ECUDA.
 */
SWE_API int swe_set_state(swe_mesh* mesh, const void* h, const void* hu, const void* hv, int where,
                  double t);

/*
 * Advances nsteps explicit Euler steps (Eq 37) with the time step recomputed
 * after every update as cfl * min_i R_i / (sqrt(g h_i) + |u_i|) over wet cells
 * (Eq 15).  Each step is one fused kernel: edge fluxes with hydrostatic
 * reconstruction and HLLC, boundary fluxes, semi-implicit friction, update,
 * and the next step's min-reduction.  Launches are asynchronous on the mesh
 * stream and replayed from CUDA graphs.  If t_out is not NULL the call waits
 * for the steps, checks the device status word and stores the time reached.
 * Errors: SWE_EINVAL (no state set, cfl <= 0), SWE_ECUDA; with t_out also
 * SWE_ENONFINITE and SWE_EDRY.
 */
SWE_API int swe_step(swe_mesh* mesh, int64_t nsteps, double cfl, double* t_out);

/*
 * Copies the current state out, in the caller's cell numbering, to host
 * (waits for completion) or device (stream-ordered) arrays of the mesh
 * precision.  Errors: SWE_EINVAL, SWE_ECUDA.
 */
SWE_API int swe_get_state(swe_mesh* mesh, void* h, void* hu, void* hv, int where);

/* Waits for the mesh stream and reports the device status word: SWE_OK,
 * SWE_ENONFINITE or SWE_EDRY. */
SWE_API int swe_synchronize(swe_mesh* mesh);

typedef struct swe_info {
    int64_t n_cells;
    int64_t n_steps;        /* steps taken since the last swe_set_state */
    int64_t n_clamped;      /* cells whose depth was clamped from < 0 to 0 */
    double t;               /* time reached */
    double dt_next;         /* CFL step for the next update (+inf if all dry) */
    int precision;
    int status;             /* device status word mapped to an SWE_* code */
    int64_t device_bytes;   /* device memory held by the mesh */
    int64_t n_active;       /* cell updates since swe_set_state that ran the full flux path
                               (the others were dry cells among dry neighbours: no flux) */
} swe_info;

/* Waits for the mesh stream and fills *info. */
SWE_API int swe_get_info(swe_mesh* mesh, swe_info* info);

/* perm[new] = caller's index of the cell stored at internal position new
 * (the locality ordering).  perm: [n_tris] int64 host array. */
SWE_API int swe_get_permutation(swe_mesh* mesh, int64_t* perm);

/* ---- diagnostics and steady state ---- */

typedef struct swe_diag {
    double t;               /* time of the state */
    double dt_last;         /* size of the last step (0 before the first) */
    double volume;          /* stored water, sum_i |Omega_i| h_i (m^3) */
    double dh_max;          /* max_i |h_i^n - h_i^{n-1}| over the last step (m) */
    double h_max;           /* largest depth (m) */
    double speed_max;       /* largest |u| over wet cells (m/s) */
    int64_t n_wet;          /* cells with h > h_dry */
    int n_groups;           /* boundary groups, group 0 = the default wall */
    double discharge[64];   /* outward discharge through each group (m^3/s) for the current
                               state: what leaves through those edges in the next step per
                               unit time (an inflow group of discharge Q gives -Q) */
} swe_diag;

/*
 * Diagnostics of the current state: stored volume, depth change over the last
 * step, extremes, wet cells, and the inflow/outflow rates of Section 5.3.2
 * (per boundary group, with the step's own boundary fluxes of Section 3.1).
 * Since interior fluxes cancel, volume after a step minus volume before it
 * equals -dt times the sum of the discharges of the state before it.
 * Deterministic; waits for the mesh stream.  Errors: SWE_EINVAL, SWE_ECUDA.
 */
SWE_API int swe_diagnostics(swe_mesh* mesh, swe_diag* out);

/*
 * Runs until the state is steady (the paper's first phase, a stabilised
 * solution before production runs, Section 6.3.2): steps of check_every,
 * stopping when max_i |h_i^{n+1} - h_i^n| / dt < tol (m/s) or after
 * max_steps.  steps_done, converged (1/0) and t_out may be NULL.
 */
SWE_API int swe_run_to_steady(swe_mesh* mesh, double cfl, double tol, int64_t check_every, int64_t max_steps,
                              int64_t* steps_done, int* converged, double* t_out);

/* ---- discrete adjoint (inverse analysis) ---- */

/*
 * Gradient of a gauge misfit with respect to the per-cell Manning coefficient
 * and bed elevation, by the discrete adjoint of the FP64 step (Eq 37 and
 * everything it calls).  The paper motivates inverse analysis (Section 1) but
 * gives no adjoint; this is the adjoint of the discrete map as implemented.
 *
 * From the mesh's current state U^0, runs nsteps forward steps with the CFL
 * number cfl (the mesh state advances to U^N exactly as swe_step would move
 * it), then
 *   loss = sum_k (h[gauge_cells[k]]^N - target_h[k])^2
 * and its gradient with the step sizes held at the forward run's values
 * (the dt sequence is not differentiated; dts_out, if not NULL, receives it:
 * [nsteps] host doubles).  States are checkpointed every checkpoint_every
 * steps (0 = 50) and recomputed segment by segment in the reverse sweep.
 *   gauge_cells [n_gauges] caller cell indices; target_h [n_gauges] (host)
 *   loss        one host double
 *   grad_manning, grad_bathy: [n_tris] doubles in the caller's cell order, on
 *               the host (where = SWE_HOST) or device (SWE_DEVICE); either may be NULL
 * Each reverse step recomputes the forward right-hand side, transposes the
 * cell update (friction solve, Eq 33-37) and then every interior edge's flux
 * and bed source terms (Eq 12-30) once per edge for both of its cells
 * (swe_adjoint_method).
 * Device memory: about (nsteps/checkpoint_every + checkpoint_every + 4) x 32 B per cell,
 * plus 64 B per interior edge.
 * Errors: SWE_EINVAL (FP32 mesh, no state, bad gauge), SWE_ENOMEM, SWE_ECUDA,
 * SWE_ENONFINITE, SWE_EDRY, SWE_EMESH (debug checks).
 */
SWE_API int swe_adjoint(swe_mesh* mesh, int64_t nsteps, double cfl, const int32_t* gauge_cells, int n_gauges,
                        const double* target_h, int checkpoint_every, double* loss, double* grad_manning,
                        double* grad_bathy, int where, double* dts_out);

/*
 * Chooses how swe_adjoint and swe_adjoint_series form each reverse step's
 * edge terms (not in the paper, which gives no adjoint):
 *   SWE_ADJOINT_TRANSPOSE (default): one pass over the interior edges runs
 *     each edge's flux forward once and then backwards through its
 *     operations (hand-written transposes of Eq 12-30), giving the adjoints
 *     of both cells' states and beds; a cell pass adds them up in a fixed
 *     order.
 *   SWE_ADJOINT_DUAL: every cell differentiates its own and its neighbours'
 *     edge terms by running the forward's device functions on
 *     four-component forward-mode dual numbers (each edge from both sides);
 *     slower, and kept as an independent check of the transposes.
 * Both give the gradient of the same discrete map (to rounding).
 * Errors: SWE_EINVAL (NULL mesh, unknown method).
 */
SWE_API int swe_adjoint_method(swe_mesh* mesh, int method);

/*
 * Same as swe_adjoint for a time-series misfit: observations every obs_every
 * steps (obs_every must divide nsteps),
 *   loss = sum_{o=1..nsteps/obs_every} sum_k (h[gauge_cells[k]]^{o obs_every} - targets[o-1][k])^2,
 *   targets: [nsteps/obs_every][n_gauges] host doubles.
 * The adjoint adds each observation's residual to the adjoint state as the
 * reverse sweep passes its step.  swe_adjoint is the case obs_every = nsteps.
 */
SWE_API int swe_adjoint_series(swe_mesh* mesh, int64_t nsteps, double cfl, const int32_t* gauge_cells,
                               int n_gauges, const double* targets, int64_t obs_every, int checkpoint_every,
                               double* loss, double* grad_manning, double* grad_bathy, int where,
                               double* dts_out);

/* Advances nsteps steps with prescribed step sizes dts[nsteps] (host array,
 * each > 0) instead of the CFL step: the frozen-dt map that swe_adjoint
 * differentiates.  t_out (nullable) receives the time reached; waits. */
SWE_API int swe_step_dt(swe_mesh* mesh, int64_t nsteps, const double* dts, double* t_out);

/* Replaces the bed elevation and/or Manning coefficients ([n_tris] host
 * doubles in the caller's order; NULL keeps the current field).  The state's
 * h, hu, hv are kept.  Waits for the mesh stream.  Errors: SWE_EINVAL (a
 * non-finite bed, a negative or non-finite Manning coefficient). */
SWE_API int swe_set_fields(swe_mesh* mesh, const double* bathy, const double* manning);

/* ---- batched ensemble (uncertainty propagation: many runs of the same solver) ---- */

typedef struct swe_ensemble swe_ensemble;

/*
 * Builds an ensemble from n_members meshes that all have a state (and the
 * same precision, device, g and h_dry).  The members' device arrays are
 * copied into one concatenated layout; the member meshes are not modified and
 * may be destroyed afterwards.  Each member keeps its own CFL time step and
 * time, continuing from its current state, and receives exactly the updates
 * the plain solver (swe_step) would give it.  FP32 ensembles place the
 * members with at least half their cells wet (h > h_dry) at creation first in
 * the layout, for the split step (swe_tune.cell_pairs); the placement changes
 * no member's results.  The ensemble uses the first member's stream until
 * swe_ensemble_set_stream.
 * Errors: SWE_EINVAL, SWE_ENOMEM, SWE_ECUDA.
 */
SWE_API int swe_ensemble_create(swe_mesh* const* members, int n_members, swe_ensemble** out);

/* Releases the ensemble.  NULL is ignored. */
SWE_API void swe_ensemble_destroy(swe_ensemble* ens);

/* Sets the CUDA stream of all later ensemble calls. */
SWE_API int swe_ensemble_set_stream(swe_ensemble* ens, void* cuda_stream);

/*
 * Advances every member nsteps steps (Eq 37, each with its own CFL step of
 * Eq 15) as one CUDA-graph launch: each step is one kernel over all members'
 * cells.  cfl: [n_members] host array, or NULL for 0.9.  t_out: NULL, or a
 * [n_members] host array that receives each member's time (the call then
 * waits and reports SWE_ENONFINITE / SWE_EDRY for the first failing member).
 */
SWE_API int swe_ensemble_step(swe_ensemble* ens, int64_t nsteps, const double* cfl, double* t_out);

/* Copies member `member`'s state out in that member's caller cell order
 * (host arrays: waits; device arrays: stream-ordered). */
SWE_API int swe_ensemble_get_state(swe_ensemble* ens, int member, void* h, void* hu, void* hv, int where);

/* Fills *info for one member (n_active counts all members together). */
SWE_API int swe_ensemble_get_info(swe_ensemble* ens, int member, swe_info* info);

/*
 * Evaluates the edge Riemann flux of the step kernel on n independent
 * normal-frame states (Eq 17-26, with the readings of the step kernel):
 * G~(U_L, U_R) with U_K = (h_K, h_K un_K, h_K ut_K).  All twelve pointers are
 * device arrays of n elements of the given precision, used on `cuda_stream`.
 * G1..G3 receive the flux, S (may be NULL) receives [n][3] = S_L, S_R, S*.
 * Errors: SWE_EINVAL, SWE_ECUDA.
 */
SWE_API int swe_riemann_flux(int precision, int64_t n, const void* hL, const void* unL, const void* utL,
                     const void* hR, const void* unR, const void* utR, double g, double h_dry,
                     void* G1, void* G2, void* G3, void* S, void* cuda_stream);

/*
 * Runs only the host preprocessing of swe_mesh_create (validation,
 * orientation, neighbours, geometry, locality order, and for SWE_FP32 the
 * cell pairs) for a mesh of the given precision and returns its result in the
 * internal order, without touching a GPU.  Any output may be NULL.
 *   perm     [n_tris] int64: caller index of internal cell c
 *   code     [n_tris][3] int32: per local edge j (edge from vertex j to j+1 of
 *            the counter-clockwise triangle), the internal index of the
 *            neighbour, with bit 0x40000000 set when the neighbour has the
 *            lower caller index (it is the edge's left state), or -1 on the
 *            boundary
 *   ln       [n_tris][3][2] double: L_ij n_ij, outward normal times length
 *   inv_area [n_tris] double: 1/|Omega_i|;  rin [n_tris] double: 2|Omega_i|/perimeter
 * Errors: as swe_mesh_create, without SWE_ECUDA.
 */
SWE_API int swe_mesh_preprocess(const double* nodes, int64_t n_nodes, const int32_t* tris, int64_t n_tris,
                                int reorder, int precision, int64_t* perm, int32_t* code, double* ln,
                                double* inv_area, double* rin);

/*
 * Allocation-free CFL time step.  The paper has no counterpart: this entry
 * point exists for callers that cannot let the library call cudaMalloc (code
 * that owns all device memory through its own arena, or that runs while a
 * CUDA graph is being captured, where allocation is not allowed).
 *
 * Writes to *dt_out (a device double) cfl * min_i R_i / (sqrt(g h_i) + |u_i|)
 * over the cells with h_i > h_dry (Eq 15), or +inf when every cell is dry --
 * the same value swe_set_state computes for its first step.  It allocates
 * nothing and calls no allocating routine.
 *   precision  SWE_FP64 (double arrays) or SWE_FP32 (float arrays)
 *   n          number of cells, 1 <= n <= 16,777,216 (larger n: SWE_EINVAL)
 *   h, hu, hv  [n] device arrays of the state, any cell order
 *   rin        [n] device array of inscribed radii 2|Omega_i|/perimeter, same order
 *   dt_out     one device double; written in stream order on `cuda_stream`
 * Runs on the calling thread's current device.  Its scratch is a 512 KiB
 * static device array that every GPU loading the library holds until the
 * process exits.  Every call looks up that array's address on the current
 * device (which allocates nothing, and stays right after a cudaDeviceReset);
 * the first call on a device also loads the library's device code there, so
 * make the first call on a device before any stream capture.
 * All calls share the array: calls that overlap on the GPU (for instance on
 * two streams) race and may return wrong values.
 * Errors: SWE_EINVAL, SWE_ECUDA.
 */
SWE_API int swe_cfl_dt_noalloc(int precision, int64_t n, const void* h, const void* hu, const void* hv,
                               const void* rin, double g, double h_dry, double cfl, double* dt_out,
                               void* cuda_stream);

/* swe_riemann_flux with a choice of flux (SWE_FLUX_HLLC or SWE_FLUX_HLL). */
SWE_API int swe_riemann_flux_kind(int precision, int flux, int64_t n, const void* hL, const void* unL,
                                  const void* utL, const void* hR, const void* unR, const void* utR, double g,
                                  double h_dry, void* G1, void* G2, void* G3, void* S, void* cuda_stream);

/* ---- launch-shape autotuner ---- */

typedef struct swe_tune {
    int block_size;          /* chosen threads per block */
    int min_blocks;          /* chosen resident-block target the kernel is compiled for */
    int stages;              /* chosen cp.async staging depth (1 = direct loads) */
    int geometry_early;      /* chosen geometry load placement (swe_config.geometry_early) */
    int activity;            /* chosen activity mode (swe_config.activity) */
    int edge_pass;           /* chosen edge-pass mode (swe_config.edge_pass) */
    int dynamic;             /* ensembles: 1 = blocks take chunks from a per-step counter as they
                                finish, 0 = fixed round-robin chunks; 0 for a mesh */
    int chunk;               /* ensembles: tiles per chunk (round-robin or taken dynamically);
                                0 for a mesh */
    int64_t grid;            /* blocks launched per step */
    double cells_per_thread; /* cells each thread updates per step: cells / (grid * block_size) */
    double ms_best;          /* measured time per step of the chosen shape (ms; from the runoff
                                when one ran) */
    double ms_before;        /* measured time per step of the shape in use before the call (ms;
                                from the runoff, which always includes it, when one ran) */
    int n_candidates;        /* shapes timed */
    int cell_pairs;          /* meshes: chosen pair mode (swe_config.cell_pairs); FP32 ensembles:
                                1 = split step: the members placed first (mostly wet at
                                creation) are updated by a cell-pair kernel (128-thread blocks,
                                one pair of cells per thread, one resident wave), the others by
                                the kernel of this shape, in the same step */
    int queue;               /* FP32 ensembles with activity: 1 = each warp gathers the cells that
                                run the flux path into a queue in shared memory and updates them
                                32 at a time (full warps where wet cells are scattered), the
                                quiet cells at once; compiled (block_size, min_blocks,
                                geometry_early): (128, 7, 0|1), (128, 6, 1); 0 otherwise */
} swe_tune;

/*
 * Chooses the step kernel's launch shape for this mesh by measurement: every
 * compiled (block_size, min_blocks, stages, geometry_early, activity,
 * edge_pass) shape (see swe_config) with several
 * grid sizes -- one or two resident waves looping over the cells, or 1, 2 or 4
 * cells per thread -- is timed with CUDA events over trial_steps steps
 * (>= 1; 0 = 8), twice; the shape in use and the (at most four) shapes within
 * 5 % of the fastest are then timed again over max(32, 4 trial_steps) steps,
 * and the first of them (in a fixed order, the shape in use first) within 1 %
 * of the fastest there is kept for all later steps.  The
 * paper fixes no launch shape; every shape evaluates the same arithmetic on
 * every cell, so the choice changes the speed only: states, times and time
 * steps are bit for bit the same whatever is chosen.  The trial steps read the
 * current state and write scratch copies of the state and status block, so
 * the mesh's state, time and step count do not change.  Allocates one state
 * buffer for the duration of the call and waits for the mesh stream.
 * out may be NULL.  Errors: SWE_EINVAL (no state set), SWE_ENOMEM, SWE_ECUDA.
 */
SWE_API int swe_autotune(swe_mesh* mesh, int trial_steps, swe_tune* out);

/*
 * The same for an ensemble's batched step: its compiled (block_size,
 * min_blocks, stages, geometry_early) shapes (FP32: (256, 4, 3|1|2, 0),
 * (128, 8, 3|1, 0), (256, 4, 3|1, 1), (128, 8, 3|1, 1); FP64: (256|128, 1,
 * 1|2, 0), (256|128, 1, 1, 1)) and its activity-mode shapes (activity 1,
 * stages 3: FP32 (128, 8) and (256, 4) with geometry_early 0|1; FP64
 * (256|128, 1) with 0), and for FP64 ensembles its edge-pass shapes
 * (edge_pass 1: (256|128, 1, 1, 0)), times chunks of 4 to 64 tiles; and its
 * dynamically scheduled shapes (dynamic 1, stages 1: FP32 (128, 8) with
 * geometry_early 0|1, (256, 4) with 0; FP64 (128|256, 1) with 0) with chunks
 * of 1 to 32 tiles; and the activity-mode shapes with dynamically taken
 * chunks (activity 1, dynamic 1) of 4 to 32 tiles; for FP32 ensembles the
 * activity shapes with per-warp queues (queue 1) with either chunk order; for
 * FP32 ensembles with
 * members placed for the split step, every activity or dynamically scheduled
 * shape also as the second kernel of a split step (cell_pairs 1); each over
 * trial_steps steps, twice; then, as for a mesh,
 * a runoff of the shape in use and the (at most four) shapes within 5 % of the
 * fastest over max(32, 4 trial_steps) steps, keeping the first within 1 % of
 * the fastest there; then grids of half and two resident waves for the kept
 * shape (and for a split step, the cell-pair kernel's other shapes and two
 * waves of it), over as many steps, one of which replaces it when 2 % faster.
 * Members' states, times and steps are unchanged by the call and by the
 * choice.  trial_steps 0 = 4.
 */
SWE_API int swe_ensemble_autotune(swe_ensemble* ens, int trial_steps, swe_tune* out);

/*
 * Sets an ensemble's launch shape directly (for instance one that
 * swe_ensemble_autotune chose earlier): block_size, min_blocks, stages,
 * geometry_early, activity, edge_pass and dynamic must name a compiled shape
 * (listed above; stages is ignored with activity; edge_pass only for FP64
 * ensembles; edge_pass excludes activity and dynamic; activity with dynamic
 * needs chunks of at least 4 tiles), chunk a power of
 * two up to 4096 tiles,
 * grid the blocks to launch (0 = one resident wave), cell_pairs 0 or 1 (a
 * split step, FP32 without edge_pass; its cell-pair kernel runs one resident
 * wave of (128, 8) blocks with geometry_early 1), queue 0 or 1 (FP32 with
 * activity); other fields are
 * ignored.  Results do not depend on the shape.  Errors: SWE_EINVAL.
 */
SWE_API int swe_ensemble_set_shape(swe_ensemble* ens, const swe_tune* shape);

/* Message of the last failed call on this thread ("" if none). */
SWE_API const char* swe_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SWE_H */
