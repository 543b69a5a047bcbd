// swe_kernels.cuh -- device code of the fused shallow-water step (sm_103a).
//
// One thread owns one cell (in the locality order chosen at mesh build time)
// and gathers its three neighbours, so every cell's sum of edge fluxes is
// formed in a fixed order without atomics.  Each interior edge has a
// canonical orientation: the cell with the lower caller index is the left
// state and its outward normal is the edge normal.  Both cells of an edge
// evaluate the same device function on the same operands (the right cell
// passes them swapped back into canonical order) and apply the result with
// opposite signs, so the two contributions cancel (exactly, as long as the
// compiler emits the same instruction sequence for each unrolled edge slot),
// and the result does not depend on the cell ordering.
//
// Method: Delmas & Soulaimani, Sections 2-3 (Eq 12-37); readings of the
// garbled equations are the same as the oracle's and are listed where used.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "swe_f32.cuh"

namespace swe {

constexpr int kMaxGroups = 64;
constexpr int kNbrMask = 0x3FFFFFFF;   // neighbour index bits
constexpr int kFlipBit = 0x40000000;   // set when this cell is the right side of the edge
constexpr int kStaticBit = (int)0x80000000;  // in topo.w: the cell has an inflow or fixed-stage edge
constexpr unsigned long long kInfBits = 0x7FF0000000000000ULL;  // +inf as double bits

// status word bits
constexpr unsigned kStatusNonFinite = 1u;
constexpr unsigned kStatusDry = 2u;
constexpr unsigned kStatusBadIndex = 4u;   // debug checks: an index or boundary group out of range

// Debug checks: whether a neighbour code can be used on a mesh of n cells with
// n_groups boundary groups -- an interior code (>= 0) whose cell index is below
// n, or a boundary code (< 0) whose group -1 - code is below n_groups.
__host__ __device__ __forceinline__ bool code_ok(int code, long long n, int n_groups) {
    if (code >= 0) return (long long)(code & 0x3FFFFFFF) < n;
    return -1 - (long long)code < (long long)n_groups;
}

constexpr int kBcWall = 0, kBcInflow = 1, kBcTransmissive = 2, kBcStage = 3;

constexpr int kEnsPad = 256;  // ensemble members are padded to whole multiples of this many cells

template <typename T>
struct alignas(4 * sizeof(T)) V4 {
    T x, y, z, w;
};

// Boundary groups: for group g, kind[g] and value[g] = q (m^2/s, inflow per
// unit length) or eta_s (m, stage).
struct BcTable {
    int kind[kMaxGroups];
    double value[kMaxGroups];
};

template <typename T>
struct StepArgs {
    const V4<T>* __restrict__ s_in;    // (h, hu, hv, z) per cell
    V4<T>* __restrict__ s_out;
    const V4<T>* __restrict__ geoA;    // (L n)_0 x, y, (L n)_1 x, y : outward normals times length
    const V4<T>* __restrict__ geoB;    // (L n)_2 x, y, 1/|Omega|, inscribed radius
    const V4<T>* __restrict__ geoR;    // FP64: 1/|L n| of the three edges (x, y, z)
    const int4* __restrict__ topo;     // neighbour codes of the 3 edges; .w = g m^2 bits (FP32)
    const T* __restrict__ gm2;         // g m^2 per cell (Manning factor of Eq 32), FP64 only
    const double* dt_read;             // min_i R_i/(c_i+|u_i|) of the current state
    unsigned long long* dt_write;      // same quantity for the new state (atomicMin on bits)
    unsigned long long* dt_reset;      // slot cleared to +inf for the step after next
    double* t;                         // simulated time
    unsigned* status;                  // kStatus* bits
    unsigned long long* n_clamped;     // cells clamped from h < 0
    unsigned long long* n_active;      // cells that ran the full flux path (diagnostic)
    long long n;                       // number of cells
    unsigned grid;                     // blocks launched (grid-stride)
    double cfl;
    int hll;                           // 1: HLL flux for all components, 0: HLLC
    const double* dt_fixed;            // if set: the step size to take (frozen time steps)
    double* dt_log;                    // if set: receives the step size taken
    // activity bytes (step_kernel_act only): read, marked for the next step,
    // cleared for the step after next
    const unsigned char* act_in;
    unsigned char* act_next;
    unsigned char* act_clear;
    // edge pass (step_kernel with EDGES): interior edges in canonical orientation,
    // evaluated once per step by edge_flux_kernel before the cell pass
    const int2* ecells;                // (left, right) cell of each interior edge
    const T* eln;                      // [E][2] L n of the edge, outward from the left cell
    const T* erl;                      // FP64: 1/|L n| of the edge
    V4<T>* eflux;                      // (F0, F1, F2, bed source factor of the left cell) per edge
    T* esrc;                           // bed source factor of the right cell per edge
    const int4* eidx;                  // per cell: the interior edge of each local edge (x, y, z)
    long long n_edges;
    T g, h_dry;
    BcTable bc;
    int debug;                         // 1: check indices and groups before use (kStatusBadIndex)
    int n_groups;                      // boundary groups in use
    __device__ __forceinline__ int bc_kind(int grp) const { return bc.kind[grp]; }
    __device__ __forceinline__ double bc_value(int grp) const { return bc.value[grp]; }
    __device__ __forceinline__ long long cell_bound() const { return n; }
};

// Arguments of the batched ensemble step: the members' cells are concatenated,
// each member padded to a whole multiple of kEnsPad cells (padding cells are
// dry and walled in, so they take the quiet path).  A block works on tiles of
// BLOCK cells (BLOCK divides kEnsPad), so every tile belongs to one member.
template <typename T>
struct EnsArgs {
    const V4<T>* __restrict__ s_in;
    V4<T>* __restrict__ s_out;
    const V4<T>* __restrict__ geoA;
    const V4<T>* __restrict__ geoB;
    const V4<T>* __restrict__ geoR;    // FP64: 1/|L n| of the three edges
    const int4* __restrict__ topo;     // neighbour codes offset to the concatenated numbering
    const T* __restrict__ gm2;         // FP64 only
    const int* __restrict__ tile_member;               // member of each kEnsPad-cell span
    const long long* __restrict__ member_first_tile;   // first kEnsPad-cell span of each member
    const double* __restrict__ cfl;    // per member
    unsigned long long* small;         // per member: 8 words (dt slots 0..2, t, status, clamps, -, -)
    const int* __restrict__ kind_;     // global boundary groups (0 = wall)
    const double* __restrict__ value_;
    unsigned long long* n_active;      // all members (diagnostic)
    long long n_total;                 // cells of the padded layout (a multiple of kEnsPad)
    // split step: the first pair_spans kEnsPad-cell spans belong to the members
    // the cell-pair kernel updates; the other kernels then update the cells
    // from cell_lo = pair_spans * kEnsPad on (otherwise both are 0)
    long long cell_lo;
    unsigned pair_spans;
    int chunk_log2;                    // tiles per round-robin chunk = 2^chunk_log2
    // dynamic chunks (ensemble_step_kernel_dyn): three rotating counters; the
    // step takes chunks from sched[sched_slot] and zeroes sched[sched_reset]
    unsigned* sched;
    int sched_slot, sched_reset;
    // activity bytes over the concatenated layout (ensemble_step_kernel_act)
    const unsigned char* act_in;
    unsigned char* act_next;
    unsigned char* act_clear;
    // edge pass over the concatenated members (ensemble_step_kernel with EDGES)
    const int2* ecells;
    const T* eln;
    const T* erl;
    V4<T>* eflux;
    T* esrc;
    const int4* eidx;
    long long n_edges;
    int slot_read, slot_write, slot_reset;
    int hll;
    T g, h_dry;
    int debug;                         // 1: check indices and groups before use (kStatusBadIndex)
    int n_groups;                      // global boundary groups in use
    __device__ __forceinline__ int bc_kind(int grp) const { return kind_[grp]; }
    __device__ __forceinline__ double bc_value(int grp) const { return value_[grp]; }
    __device__ __forceinline__ long long cell_bound() const { return n_total; }
};

// ---- precision-specific arithmetic ------------------------------------------------
// The FP32 instantiation is compiled with fast-math: division, reciprocal and
// square root map to the hardware approximations (a few ulp), which the
// 1e-4 FP32 tolerance absorbs.  The FP64 instantiation keeps IEEE division
// and square root.
template <typename T> struct Ar;
template <> struct Ar<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float rcp_(float x) { return __fdividef(1.0f, x); }
    // h^(-7/3) through the hardware base-2 exp/log pair
    static __device__ __forceinline__ float pow_m73(float h) { return exp2f(-7.0f / 3.0f * __log2f(h)); }
};
template <> struct Ar<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
    static __device__ __forceinline__ double div_(double a, double b) { return a / b; }
    static __device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double pow_m73(double h) { return 1.0 / (h * h * cbrt(h)); }
};

template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <typename T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }

// FP64 (the double instantiation only): where the paper's formulas divide by
// several quantities in turn, one division by their product and
// multiplications replace them.  A double division or square root is an
// iteration of several operations on the FP64 unit, which bounds that path;
// the products stay far inside the double range for depths of 1e-6 to 1e4 m.
// Results move by a few ulps.  FP32 divisions are single hardware
// approximations, and the adjoint's duals keep the formulas as written.
template <typename T>
constexpr bool kOneDivision = std::is_same<T, double>::value;

// h^(-1/3) in double without a division or a double cube root, for the
// friction factor h^(-7/3) = r^7 and 1/h = r^3 (Eq 33-35): Newton's iteration
// for r^-3 = h, r <- r (4 - h r^3) / 3, started from the FP32 reciprocal cube
// root (relative error about 2^-22) and taken twice (the error squares each
// time, to the rounding of the last step).  For positive normal h in the FP32
// range; friction calls it for wet cells only (h > h_dry).
__device__ __forceinline__ double inv_cbrt_newton(double h) {
    double r = (double)rcbrtf((float)h);
    r = r * fma(-h, r * r * r, 4.0) * (1.0 / 3.0);
    r = r * fma(-h, r * r * r, 4.0) * (1.0 / 3.0);
    return r;
}

// ---- comparisons of the flux path ------------------------------------------------
// On GB300 the FP64 unit (2 operations per clock per SM) executes compares and
// min/max of doubles as well as their arithmetic, and it bounds the FP64 step.
// For doubles each helper below forms exactly the IEEE result of its
// comparison (NaN, infinities and signed zeros included) from the bit
// patterns, with 64-bit integer operations, which the FP64 kernels leave
// idle; the selects return the same operand the plain expression returns, so
// results are bit for bit those of the plain operators.  Other scalars (float,
// the adjoint's dual numbers) use the plain operators.
namespace cmp {
constexpr unsigned long long kPosInf = 0x7FF0000000000000ULL;   // bits of +inf
constexpr unsigned long long kNegZero = 0x8000000000000000ULL;  // bits of -0
__device__ __forceinline__ unsigned long long bits(double x) { return (unsigned long long)__double_as_longlong(x); }
template <typename T>
constexpr bool kInt = std::is_same<T, double>::value;
}  // namespace cmp

// x > c for c finite and > 0
template <typename T>
__device__ __forceinline__ bool gt_pos(T x, T c) {
    if constexpr (cmp::kInt<T>) {
        const unsigned long long xb = cmp::bits(x), cb = cmp::bits(c);
        return xb - cb - 1ULL < cmp::kPosInf - cb;          // c < x <= +inf
    } else {
        return x > c;
    }
}
// x <= c for c finite and > 0
template <typename T>
__device__ __forceinline__ bool le_pos(T x, T c) {
    if constexpr (cmp::kInt<T>) {
        const unsigned long long xb = cmp::bits(x), cb = cmp::bits(c);
        return xb <= cb || xb - cmp::kNegZero <= cmp::kPosInf;   // +0 <= x <= c, or -inf <= x <= -0
    } else {
        return x <= c;
    }
}
// x < c for c finite and > 0
template <typename T>
__device__ __forceinline__ bool lt_pos(T x, T c) {
    if constexpr (cmp::kInt<T>) {
        const unsigned long long xb = cmp::bits(x), cb = cmp::bits(c);
        return xb < cb || xb - cmp::kNegZero <= cmp::kPosInf;
    } else {
        return x < c;
    }
}
// |x| < c for c finite and > 0
template <typename T>
__device__ __forceinline__ bool abs_lt_pos(T x, T c) {
    if constexpr (cmp::kInt<T>) {
        return (cmp::bits(x) & ~cmp::kNegZero) < cmp::bits(c);
    } else {
        return fabs(x) < c;
    }
}
template <typename T>
__device__ __forceinline__ bool gt_zero(T x) {
    if constexpr (cmp::kInt<T>) return cmp::bits(x) - 1ULL < cmp::kPosInf;            // smallest denormal .. +inf
    else return x > T(0);
}
template <typename T>
__device__ __forceinline__ bool ge_zero(T x) {
    if constexpr (cmp::kInt<T>) {
        const unsigned long long xb = cmp::bits(x);
        return xb <= cmp::kPosInf || xb == cmp::kNegZero;
    } else {
        return x >= T(0);
    }
}
template <typename T>
__device__ __forceinline__ bool le_zero(T x) {
    if constexpr (cmp::kInt<T>) {
        const unsigned long long xb = cmp::bits(x);
        return xb == 0ULL || xb - cmp::kNegZero <= cmp::kPosInf;
    } else {
        return x <= T(0);
    }
}
template <typename T>
__device__ __forceinline__ bool lt_zero(T x) {
    if constexpr (cmp::kInt<T>) return cmp::bits(x) - (cmp::kNegZero + 1ULL) < cmp::kPosInf;  // -inf .. -denormal
    else return x < T(0);
}
// tmax(0, x)
template <typename T>
__device__ __forceinline__ T max_zero(T x) {
    if constexpr (cmp::kInt<T>) return lt_zero(x) ? T(0) : x;
    else return tmax(T(0), x);
}
// tmin(a, b) for a, b >= +0 (or +inf), e.g. CFL candidates and depths
template <typename T>
__device__ __forceinline__ T min_nonneg(T a, T b) {
    if constexpr (cmp::kInt<T>) return cmp::bits(a) < cmp::bits(b) ? a : b;
    else return tmin(a, b);
}
// tmax(a, b) for finite a, b (bed elevations)
template <typename T>
__device__ __forceinline__ T max_finite(T a, T b) {
    if constexpr (cmp::kInt<T>) {
        // the sign-magnitude bits, turned into a two's-complement key, order
        // finite doubles except that -0 sorts below +0, where IEEE has a tie
        const long long ab = __double_as_longlong(a), bb = __double_as_longlong(b);
        const long long ka = ab ^ ((ab >> 63) & 0x7FFFFFFFFFFFFFFFLL), kb = bb ^ ((bb >> 63) & 0x7FFFFFFFFFFFFFFFLL);
        const bool both_zero = (((unsigned long long)ab | (unsigned long long)bb) << 1) == 0ULL;
        return (ka > kb && !both_zero) ? a : b;
    } else {
        return tmax(a, b);
    }
}

// 1/|L n| of an edge.  FP64 takes it precomputed (the host forms
// 1/sqrt(fma(lx, lx, ly ly)) once per cell edge, the same on every host): the
// square root and division are a quarter of the flux pass's FP64 work, and the
// FP64 pipe bounds that path.  FP32 forms it with the hardware reciprocal
// square root, since memory bounds that path.
template <typename T>
__device__ __forceinline__ T edge_rl(T pre, T l2) {
    if constexpr (sizeof(T) == 8) return pre;
    else return Ar<T>::rsqrt_(l2);
}

// |L n|^2 of an edge, written as one fused multiply-add so that every kernel
// (and both cells of an edge, whose L n differ only in sign) forms the same
// value.
template <typename T>
__device__ __forceinline__ T edge_l2(T lx, T ly) { return fma(lx, lx, ly * ly); }

// ---- Riemann flux in the edge-normal frame (Eq 14, 17-26) -------------------------
// Input U_K = (h_K, h_K un_K, h_K ut_K) given as depth and normal/tangential
// velocity.  Readings: Eq 20 p_K = sqrt(h*(h*+h_K)/2)/h_K; Eq 21-22 use the
// normal velocity jump; the two-rarefaction base is clamped at 0; Eq 24 is
// upwinded (ut_L when S* >= 0); Eq 26 line 2 is the right-dry case; both dry
// gives no flux.
// With hll_only the third component is the HLL flux of U_3 = h ut (Eq 18
// applied to it) instead of the HLLC upwinding of Eq 24.
template <typename T>
__device__ __forceinline__ void riemann_hllc(T hL, T unL, T utL, T hR, T unR, T utR, T g, T h_dry,
                                             T& G1, T& G2, T& G3, T* speeds = nullptr, bool hll_only = false) {
    if constexpr (std::is_same<T, float>::value) {   // FP32: swe_f32.cuh, branch-free and explicitly rounded
        f32::riemann<float>(hL, unL, utL, hR, unR, utR, g, f32::mul(0.5f, g), h_dry, G1, G2, G3, speeds, hll_only);
        return;
    }
    using A = Ar<T>;
    const bool wetL = gt_pos(hL, h_dry), wetR = gt_pos(hR, h_dry);
    if (!wetL && !wetR) {
        G1 = T(0); G2 = T(0); G3 = T(0);
        if (speeds) { speeds[0] = T(0); speeds[1] = T(0); speeds[2] = T(0); }
        return;
    }
    const T aL = A::sqrt_(g * hL), aR = A::sqrt_(g * hR);
    T SL, SR, Ss;
    if (!wetL) {
        SL = unR - T(2) * aR; SR = unR + aR; Ss = SL;
    } else if (!wetR) {
        SL = unL - aL; SR = unL + T(2) * aL; Ss = SR;
    } else {
        const T hsum = hL + hR;
        const T h0 = T(0.5) * hsum - T(0.25) * A::div_((unR - unL) * hsum, aL + aR);  // Eq 21
        T hs;
        if (le_pos(h0, min_nonneg(hL, hR))) {                                      // Eq 22
            const T b = max_zero(T(0.5) * (aL + aR) + T(0.25) * (unL - unR));
            hs = A::div_(b * b, g);
        } else if constexpr (!kOneDivision<T>) {                                    // Eq 23
            const T r2h0 = A::rcp_(T(2) * h0);
            const T gL = A::sqrt_(g * (h0 + hL) * r2h0 * A::rcp_(hL));
            const T gR = A::sqrt_(g * (h0 + hR) * r2h0 * A::rcp_(hR));
            hs = A::div_(hL * gL + hR * gR + unL - unR, gL + gR);
        } else {
            // one division gives 1/(2 h0 h_L) and 1/(2 h0 h_R) (h0 > min(h_L, h_R) > 0 here)
            const T h02 = T(2) * h0;
            const T inv = A::rcp_(h02 * hL * hR);
            const T gL = A::sqrt_(g * (h0 + hL) * (hR * inv));
            const T gR = A::sqrt_(g * (h0 + hR) * (hL * inv));
            hs = A::div_(hL * gL + hR * gR + unL - unR, gL + gR);
        }
        T pL = T(1), pR = T(1);                                                     // Eq 20
        if constexpr (!kOneDivision<T>) {
            if (gt_pos(hs, hL)) pL = A::div_(A::sqrt_(T(0.5) * hs * (hs + hL)), hL);
            if (gt_pos(hs, hR)) pR = A::div_(A::sqrt_(T(0.5) * hs * (hs + hR)), hR);
        } else {
            // sqrt(h*(h*+h_K)/2)/h_K = sqrt(h*(h*+h_K)/(2 h_K^2)); both shocks share a division
            const bool shL = gt_pos(hs, hL), shR = gt_pos(hs, hR);
            if (shL && shR) {
                const T inv = A::rcp_(hL * hR);
                pL = A::sqrt_(T(0.5) * hs * (hs + hL)) * (hR * inv);
                pR = A::sqrt_(T(0.5) * hs * (hs + hR)) * (hL * inv);
            } else if (shL) {
                pL = A::div_(A::sqrt_(T(0.5) * hs * (hs + hL)), hL);
            } else if (shR) {
                pR = A::div_(A::sqrt_(T(0.5) * hs * (hs + hR)), hR);
            }
        }
        SL = unL - aL * pL;                                                          // Eq 19
        SR = unR + aR * pR;
        const T mL = hL * (unL - SL), mR = hR * (unR - SR);
        Ss = A::div_(SL * mR - SR * mL, mR - mL);                                    // Eq 25
    }
    const T qL = hL * unL, qR = hR * unR;
    const T PL = qL * unL + T(0.5) * g * hL * hL;
    const T PR = qR * unR + T(0.5) * g * hR * hR;
    if (ge_zero(SL)) {                                                               // Eq 17
        G1 = qL; G2 = PL;
        if (hll_only) G3 = qL * utL;
    } else if (le_zero(SR)) {
        G1 = qR; G2 = PR;
        if (hll_only) G3 = qR * utR;
    } else {                                                                         // Eq 18
        const T r = A::rcp_(SR - SL);
        const T ss = SR * SL;
        G1 = (SR * qL - SL * qR + ss * (hR - hL)) * r;
        G2 = (SR * PL - SL * PR + ss * (qR - qL)) * r;
        if (hll_only) G3 = (SR * (qL * utL) - SL * (qR * utR) + ss * (hR * utR - hL * utL)) * r;
    }
    if (!hll_only) G3 = G1 * (ge_zero(Ss) ? utL : utR);                              // Eq 24
    if (speeds) { speeds[0] = SL; speeds[1] = SR; speeds[2] = Ss; }
}

template <typename T>
__device__ __forceinline__ T inf_of();
template <>
__device__ __forceinline__ float inf_of<float>() { return __int_as_float(0x7F800000); }
template <>
__device__ __forceinline__ double inf_of<double>() { return __longlong_as_double((long long)kInfBits); }

// ---- the step size, formed once per warp ------------------------------------------
// dt = cfl * (min of the previous state) in double, and its rounding to the
// state precision, made by lane 0 and broadcast (all 32 lanes must call):
// FP32 kernels then run no FP64 instruction per thread for it.  dt is
// non-negative or +inf, so "has a step" is an integer compare of its bits.
template <typename T>
struct WarpDt {
    double d;
    T t;
    bool have;
};
template <typename T>
__device__ __forceinline__ WarpDt<T> warp_step_dt(double cfl, const double* dt_read, const double* dt_fixed) {
    double v = 0.0;
    T vt = T(0);
    if ((threadIdx.x & 31) == 0) {
        v = dt_fixed ? *dt_fixed : cfl * (*dt_read);
        vt = T(v);
    }
    WarpDt<T> r;
    r.d = __shfl_sync(0xffffffffu, v, 0);
    r.t = __shfl_sync(0xffffffffu, vt, 0);
    r.have = (unsigned long long)__double_as_longlong(r.d) < kInfBits;
    return r;
}

// ---- block min of a non-negative candidate, published with one atomicMin ----------
// The minimum is taken in the candidate's own precision and widened to double
// once (exact and monotone, so the result equals a double minimum): an FP32
// kernel keeps its reduction off the FP64 pipe.  Non-negative doubles order
// like their bit patterns, so the 64-bit atomicMin is exact.  Optionally also
// sums a per-thread counter into *count_dst (one atomicAdd per block).
template <int BLOCK, typename T>
__device__ __forceinline__ void block_min_publish(T cand, unsigned long long* dst, unsigned cnt = 0u,
                                                  unsigned long long* count_dst = nullptr) {
    __shared__ T warp_min[BLOCK / 32];
    __shared__ unsigned warp_cnt[BLOCK / 32];
    for (int o = 16; o > 0; o >>= 1) cand = tmin(cand, __shfl_xor_sync(0xffffffffu, cand, o));
    if (count_dst) cnt = __reduce_add_sync(0xffffffffu, cnt);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { warp_min[wid] = cand; warp_cnt[wid] = cnt; }
    __syncthreads();
    if (wid == 0) {
        T v = lane < BLOCK / 32 ? warp_min[lane] : inf_of<T>();
        unsigned c = lane < BLOCK / 32 ? warp_cnt[lane] : 0u;
        for (int o = 16; o > 0; o >>= 1) v = tmin(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (count_dst) c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0 && v < inf_of<T>())
            atomicMin(dst, (unsigned long long)__double_as_longlong((double)v));
        if (lane == 0 && count_dst && c) atomicAdd(count_dst, (unsigned long long)c);
    }
}

// ---- Manning factor g m^2: packed in topo.w (FP32) or its own array (FP64) --------
// (the sign bit of topo.w is the static-activity flag; g m^2 >= 0 leaves it free)
template <typename Args>
__device__ __forceinline__ float load_gm2(const Args&, long long, const int4& tp, float) {
    return __int_as_float(tp.w & 0x7FFFFFFF);
}
template <typename Args>
__device__ __forceinline__ double load_gm2(const Args& a, long long i, const int4&, double) {
    return a.gm2[i];
}

// ---- asynchronous global -> shared copies (cp.async, 16 B, L2 only) ------------------
// Each thread stages its own future cells' records; it alone reads them back,
// so the per-thread wait_group is the only synchronisation needed.
template <int BYTES>
__device__ __forceinline__ void cp_async_record(void* smem_dst, const void* gmem_src) {
    static_assert(BYTES % 16 == 0, "records are whole 16-byte chunks");
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
#pragma unroll
    for (int b = 0; b < BYTES; b += 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + b),
                     "l"((const char*)gmem_src + b)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// ---- pieces of one cell update, shared by the step kernels and the adjoint ----------
// Templated on the scalar so the discrete adjoint can run them on forward-mode
// dual numbers: it then differentiates exactly the arithmetic, and takes
// exactly the branches, of the forward step.

template <typename T>
__device__ __forceinline__ void cell_velocity(T h, T hu, T hv, T h_dry, T& u, T& v) {
    u = T(0);
    v = T(0);
    if (gt_pos(h, h_dry)) { const T r = Ar<T>::rcp_(h); u = hu * r; v = hv * r; }
}

// Flux leaving cell i through an interior edge (per unit length, x-y frame)
// and the edge's bed source factor (g/2)(h**_i^2 - h_i^2) (Eq 30 with 1/2).
// (n1, n2) is cell i's outward unit normal; flip says cell i is the right
// state of the edge's canonical orientation.
template <typename T>
__device__ __forceinline__ void edge_interior(T hi, T ui, T vi, T zi, T hk, T huk, T hvk, T zk, T n1, T n2,
                                              bool flip, T g, T h_dry, T& F0, T& F1, T& F2, T& src,
                                              bool hll_only = false, T* src_k = nullptr) {
    if constexpr (std::is_same<T, float>::value) {   // FP32: swe_f32.cuh
        f32::edge_interior<float>(hi, ui, vi, zi, hk, huk, hvk, zk, n1, n2, flip, g, f32::mul(0.5f, g), h_dry, F0, F1,
                                  F2, src, hll_only, src_k);
        return;
    }
    T uk, vk;
    cell_velocity<T>(hk, huk, hvk, h_dry, uk, vk);
    // hydrostatic reconstruction (Eq 28): z* = max(z_i, z_k)
    const T zs = max_finite(zi, zk);
    const T hsi = max_zero(hi + zi - zs);
    const T hsk = max_zero(hk + zk - zs);
    // canonical orientation: left = lower caller index
    const T hL = flip ? hsk : hsi, hR = flip ? hsi : hsk;
    const T uL = flip ? uk : ui, vL = flip ? vk : vi;
    const T uR = flip ? ui : uk, vR = flip ? vi : vk;
    const T c1 = flip ? -n1 : n1, c2 = flip ? -n2 : n2;
    // rotate into the edge frame (Eq 12)
    const T unL = uL * c1 + vL * c2, utL = vL * c1 - uL * c2;
    const T unR = uR * c1 + vR * c2, utR = vR * c1 - uR * c2;
    T G1, G2, G3;
    riemann_hllc<T>(hL, unL, utL, hR, unR, utR, g, h_dry, G1, G2, G3, nullptr, hll_only);
    // back to (x, y) (Eq 12 inverse), as the flux leaving this cell
    const T s = flip ? T(-1) : T(1);
    F0 = s * G1;
    F1 = s * (G2 * c1 - G3 * c2);
    F2 = s * (G2 * c2 + G3 * c1);
    src = T(0.5) * g * (hsi * hsi - hi * hi);
    if (src_k) *src_k = T(0.5) * g * (hsk * hsk - hk * hk);   // the other cell's bed source factor
}

// Flux leaving cell i through a boundary edge of the given kind (Section 3.1).
template <typename T>
__device__ __forceinline__ void edge_boundary(int kind, double value, T hi, T ui, T vi, T zi, T n1, T n2, T g,
                                              T h_dry, T& F0, T& F1, T& F2, bool hll_only = false) {
    if constexpr (std::is_same<T, float>::value) {   // FP32: swe_f32.cuh
        f32::edge_boundary(kind, value, hi, ui, vi, zi, n1, n2, g, f32::mul(0.5f, g), h_dry, F0, F1, F2, hll_only);
        return;
    }
    const T un = ui * n1 + vi * n2, ut = vi * n1 - ui * n2;
    T G1, G2, G3;
    if (kind == kBcWall) {
        G1 = T(0); G2 = T(0.5) * g * hi * hi; G3 = T(0);
    } else if (kind == kBcInflow) {
        const T q = T(value);
        G1 = -q;
        G2 = T(0.5) * g * hi * hi + (gt_pos(hi, h_dry) ? Ar<T>::div_(q * q, hi) : T(0));
        G3 = T(0);
    } else {
        T hg = hi;
        if (kind == kBcStage) hg = max_zero(T(value) - zi);
        riemann_hllc<T>(hi, un, ut, hg, un, ut, g, h_dry, G1, G2, G3, nullptr, hll_only);
    }
    F0 = G1;
    F1 = G2 * n1 - G3 * n2;
    F2 = G2 * n2 + G3 * n1;
}

// Semi-implicit friction (Eq 33-37): dU solving [I - dt/2 J_f] dU = dt (R + S_f)
// with R = (Rh, Rx, Ry) the explicit right-hand side per unit area.
template <typename T>
__device__ __forceinline__ void friction_update(T hi, T qx, T qy, T gm2, T Rh, T Rx, T Ry, T dt, T h_dry, T& dh,
                                                T& dqx, T& dqy) {
    using A = Ar<T>;
    dh = dt * Rh;
    dqx = dt * Rx;
    dqy = dt * Ry;
    if (gt_pos(hi, h_dry) && gt_zero(gm2)) {
        const T qq = qx * qx + qy * qy;
        if (gt_zero(qq)) {
            const T qn = A::sqrt_(qq);
            T cf, rh;                                       // c = g m^2 h^(-7/3), 1/h
            if constexpr (kOneDivision<T>) {
                const T r = inv_cbrt_newton(hi), r3 = r * r * r;   // h^(-1/3), 1/h
                cf = gm2 * (r3 * r3 * r);                            // h^(-7/3) = r^7
                rh = r3;
            } else {
                cf = gm2 * A::pow_m73(hi);
                rh = A::rcp_(hi);
            }
            const T al = T(0.5) * dt * cf;                  // alpha = dt c / 2
            // rhs: dt (R_q + S_f) + dt/2 J_qh dh, with S_f = -c|q|q and
            // J_qh = (7/3) c |q| q / h
            const T k = dt * cf * qn * (T(7.0 / 6.0) * dh * rh - T(1));
            const T bx = dqx + k * qx, by = dqy + k * qy;
            // (1 + a|q|) I + a q q^T/|q| has eigenvalue 1 + 2a|q| along q
            // and 1 + a|q| across it
            const T d1 = T(1) + al * qn, d2 = d1 + al * qn;
            T rqd2, rd1;                                    // 1/(|q| d2), 1/d1
            if constexpr (kOneDivision<T>) {
                const T qd2 = qn * d2, inv = A::rcp_(qd2 * d1);
                rqd2 = d1 * inv;
                rd1 = qd2 * inv;
            } else {
                rqd2 = A::rcp_(qn * d2);
                rd1 = A::rcp_(d1);
            }
            const T proj = (bx * qx + by * qy) * al * rqd2;
            dqx = (bx - proj * qx) * rd1;
            dqy = (by - proj * qy) * rd1;
        }
    }
}

// ---- the end of one cell update -----------------------------------------------------
// From the summed edge terms (f = sum of L_ij F_ij, s = sum of the bed source
// factors times L_ij n_ij) to the new state (Eq 37 with friction, Eq 33-36),
// its checks, and the cell's next CFL candidate R_i/(sqrt(g h)+|u|) (Eq 15;
// +inf when the new state is dry).  Every cell kernel ends here, so their
// arithmetic is the same.
template <typename T, typename Args>
__device__ __forceinline__ T finish_cell(const Args& a, long long i, const V4<T>& own, T f0, T f1, T f2, T sx, T sy,
                                         T ia, T rin, T gm2, T dt, unsigned long long* n_clamped, unsigned* status) {
    using A = Ar<T>;
    const T g = a.g, h_dry = a.h_dry;
    const T hi = own.x;
    V4<T> out;
    out.w = own.w;
    const T Rh = -f0 * ia;
    const T Rx = (sx - f1) * ia;
    const T Ry = (sy - f2) * ia;
    const T qx = own.y, qy = own.z;
    T dh, dqx, dqy;
    friction_update<T>(hi, qx, qy, gm2, Rh, Rx, Ry, dt, h_dry, dh, dqx, dqy);
    out.x = hi + dh;
    out.y = qx + dqx;
    out.z = qy + dqy;
    if (lt_zero(out.x)) {
        out.x = T(0); out.y = T(0); out.z = T(0);
        atomicAdd(n_clamped, 1ULL);
    } else if (le_pos(out.x, h_dry)) {
        out.y = T(0); out.z = T(0);
    }
    const T big = T(3.0e38);
    if (!lt_pos(out.x, big) || !abs_lt_pos(out.y, big) || !abs_lt_pos(out.z, big))
        atomicOr(status, kStatusNonFinite);
    a.s_out[i] = out;
    // next CFL candidate (Eq 15), R_i / (sqrt(g h) + |u|) on the new state
    T cand = inf_of<T>();
    if (gt_pos(out.x, h_dry)) {
        if constexpr (kOneDivision<T>) {
            // R h / (h sqrt(g h) + |q|): the velocity's division folded into the candidate's
            const T qm = A::sqrt_(out.y * out.y + out.z * out.z);
            cand = A::div_(rin * out.x, out.x * A::sqrt_(g * out.x) + qm);
        } else {
            const T r = A::rcp_(out.x);
            const T u = out.y * r, v = out.z * r;
            const T den = A::sqrt_(g * out.x) + A::sqrt_(u * u + v * v);
            cand = A::div_(rin, den);
        }
    }
    return cand;
}

// ---- one FP32 cell of the fused step -------------------------------------------------
// update_cell for FP32: the same loads, quiet test and edge loop, with the
// arithmetic of swe_f32.cuh, every operation explicitly rounded, so that every
// FP32 kernel and launch shape gives the same bits.
// Pairs of cells sharing their local edge 0 (step_kernel_pair): with PAIR 1
// the first cell hands the flux of that edge to the second (pmode kPairGive ->
// kPairGiven, pe = the flux leaving the first cell); with PAIR 2 the second
// takes its negative (pmode kPairTake) instead of evaluating the edge.
struct PairEdge { float F0, F1, F2; };
constexpr int kPairNone = 0, kPairGive = 1, kPairGiven = 2, kPairTake = 3;

template <bool GEO_EARLY, bool EDGES, int PAIR = 0, typename Args>
__device__ __forceinline__ float update_cell_f32(const Args& a, long long i, const V4<float>& own, const int4& tp,
                                                 float dt, unsigned& active, unsigned long long* n_clamped,
                                                 unsigned* status, int* pmode = nullptr,
                                                 volatile PairEdge* pe = nullptr) {
    const float g = a.g, h_dry = a.h_dry, g2 = f32::mul(0.5f, g);
    const float hi = own.x, zi = own.w;
    int code[3] = {tp.x, tp.y, tp.z};
    if (a.debug) {   // an unusable code is flagged and taken as a wall (group 0)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (!code_ok(code[j], a.cell_bound(), a.n_groups)) {
                atomicOr(status, kStatusBadIndex);
                code[j] = -1;
            }
    }
    V4<float> nb[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) nb[j] = code[j] >= 0 ? a.s_in[code[j] & kNbrMask] : own;
    V4<float> gA, gB;
    float gm2;
    if constexpr (GEO_EARLY) {
        gA = a.geoA[i];
        gB = a.geoB[i];
        gm2 = load_gm2(a, i, tp, 0.0f);
    }
    bool quiet = !(hi > h_dry);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (code[j] >= 0) {
            quiet = quiet && !(nb[j].x > h_dry);
        } else {
            const int kind = a.bc_kind(-1 - code[j]);
            quiet = quiet && (kind == kBcWall || kind == kBcTransmissive);
        }
    }
    V4<float> out;
    out.w = zi;
    if (quiet) {
        out.x = hi; out.y = 0.0f; out.z = 0.0f;
        a.s_out[i] = out;
        return inf_of<float>();
    }
    active += 1u;
    if constexpr (!GEO_EARLY) {
        gA = a.geoA[i];
        gB = a.geoB[i];
        gm2 = load_gm2(a, i, tp, 0.0f);
    }
    float ui, vi;
    f32::velocity(hi, own.y, own.z, h_dry, ui, vi);
    float f0 = 0.0f, f1 = 0.0f, f2 = 0.0f, sx = 0.0f, sy = 0.0f;
    int4 ei = make_int4(-1, -1, -1, 0);
    if constexpr (EDGES) ei = a.eidx[i];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int c = j == 0 ? code[0] : (j == 1 ? code[1] : code[2]);
        const V4<float> o = j == 0 ? nb[0] : (j == 1 ? nb[1] : nb[2]);
        const float lx = j == 0 ? gA.x : (j == 1 ? gA.z : gB.x);
        const float ly = j == 0 ? gA.y : (j == 1 ? gA.w : gB.y);
        const float l2 = edge_l2(lx, ly);
        const float rl = rsqrtf(l2);
        const float len = f32::mul(l2, rl);
        const float n1 = f32::mul(lx, rl), n2 = f32::mul(ly, rl);   // this cell's outward unit normal
        float F0, F1, F2;
        if (c >= 0) {
            float src;
            if constexpr (EDGES) {
                if (!(hi > h_dry) && !(o.x > h_dry)) {
                    const float zs = f32::vmax(zi, o.w);
                    const float hsi = f32::max0(f32::sub(f32::add(hi, zi), zs));
                    F0 = 0.0f; F1 = 0.0f; F2 = 0.0f;
                    f32::bed_src(hsi, hi, g2, src);
                } else {
                    int e = j == 0 ? ei.x : (j == 1 ? ei.y : ei.z);
                    if (a.debug && !(e >= 0 && e < a.n_edges)) {
                        atomicOr(status, kStatusBadIndex);
                        e = 0;
                    }
                    const V4<float> fl = a.eflux[e];
                    if (c & kFlipBit) {
                        F0 = -fl.x; F1 = -fl.y; F2 = -fl.z;
                        src = a.esrc[e];
                    } else {
                        F0 = fl.x; F1 = fl.y; F2 = fl.z;
                        src = fl.w;
                    }
                }
            } else if (PAIR == 2 && j == 0 && *pmode == kPairTake) {
                // the first cell's evaluation of this edge, seen from this side;
                // the bed source factor is this cell's own (Eq 30)
                const float zs = f32::vmax(zi, o.w);
                const float hsi = f32::max0(f32::sub(f32::add(hi, zi), zs));
                f32::bed_src(hsi, hi, g2, src);
                F0 = -pe->F0; F1 = -pe->F1; F2 = -pe->F2;
            } else {
                f32::edge_interior<float>(hi, ui, vi, zi, o.x, o.y, o.z, o.w, n1, n2, (c & kFlipBit) != 0, g, g2,
                                          h_dry, F0, F1, F2, src, a.hll != 0);
                if (PAIR == 1 && j == 0 && *pmode == kPairGive) {
                    pe->F0 = F0; pe->F1 = F1; pe->F2 = F2;
                    *pmode = kPairGiven;
                }
            }
            sx = f32::fma(src, lx, sx);
            sy = f32::fma(src, ly, sy);
        } else {
            const int grp = -1 - c;
            f32::edge_boundary(a.bc_kind(grp), a.bc_value(grp), hi, ui, vi, zi, n1, n2, g, g2, h_dry, F0, F1, F2,
                               a.hll != 0);
        }
        f0 = f32::fma(len, F0, f0);
        f1 = f32::fma(len, F1, f1);
        f2 = f32::fma(len, F2, f2);
    }
    bool clamped, nonfinite;
    const float cand = f32::finish<float>(hi, f32::rcp_(hi), own.y, own.z, f0, f1, f2, sx, sy, gB.z, gB.w, gm2, dt, g,
                                          h_dry, out.x, out.y, out.z, clamped, nonfinite);
    if (clamped) atomicAdd(n_clamped, 1ULL);
    if (nonfinite) atomicOr(status, kStatusNonFinite);
    a.s_out[i] = out;
    return cand;
}

// ---- one cell of the fused step -----------------------------------------------------
// Returns the cell's CFL candidate R_i/(sqrt(g h)+|u|) of the new state (+inf
// when the new state is dry); sets `active` when the full flux path ran.
//
// A dry cell whose neighbours are all dry and whose boundary edges are walls
// or transmissive is "quiet": every mass flux it sees is exactly +-0 (both
// sides dry give G = 0; walls carry no mass), so its depth is unchanged, and
// its momentum is set to zero by the dry-cell rule after the update.  Its new
// state is therefore (h, 0, 0) bit for bit whatever the momentum terms were,
// and the edge loop, geometry and friction are skipped.
//
// GEO_EARLY issues the cell's geometry loads together with the neighbour
// gathers (one memory round trip fewer for a cell that runs the flux path,
// at the price of geometry traffic for quiet cells too); otherwise they are
// issued after the quiet test.  Both give the same results.
//
// EDGES takes the interior fluxes from the edge pass (edge_flux_kernel, the
// same edge_interior arithmetic evaluated once per edge from the left cell)
// instead of evaluating them here; an edge with both cells dry has no flux and
// its bed source factor is formed inline, as edge_interior would form it.
template <typename T, bool GEO_EARLY, bool EDGES = false, typename Args>
__device__ __forceinline__ T update_cell(const Args& a, long long i, const V4<T>& own, const int4& tp, T dt,
                                         unsigned& active, unsigned long long* n_clamped, unsigned* status) {
    if constexpr (std::is_same<T, float>::value) {
        return update_cell_f32<GEO_EARLY, EDGES>(a, i, own, tp, dt, active, n_clamped, status);
    } else {
    using A = Ar<T>;
    const T g = a.g, h_dry = a.h_dry;
    const T hi = own.x, zi = own.w;
    int code[3] = {tp.x, tp.y, tp.z};
    if (a.debug) {   // an unusable code is flagged and taken as a wall (group 0)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (!code_ok(code[j], a.cell_bound(), a.n_groups)) {
                atomicOr(status, kStatusBadIndex);
                code[j] = -1;
            }
    }
    // issue the three neighbour gathers before any arithmetic
    V4<T> nb[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) nb[j] = code[j] >= 0 ? a.s_in[code[j] & kNbrMask] : own;
    V4<T> gA, gB, gR;
    T gm2;
    if constexpr (GEO_EARLY) {
        gA = a.geoA[i];
        gB = a.geoB[i];
        if constexpr (sizeof(T) == 8) gR = a.geoR[i];
        gm2 = load_gm2(a, i, tp, T(0));
    }
    bool quiet = !gt_pos(hi, h_dry);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (code[j] >= 0) {
            quiet = quiet && !gt_pos(nb[j].x, h_dry);
        } else {
            const int kind = a.bc_kind(-1 - code[j]);
            quiet = quiet && (kind == kBcWall || kind == kBcTransmissive);
        }
    }
    V4<T> out;
    out.w = zi;
    if (quiet) {
        out.x = hi; out.y = T(0); out.z = T(0);
        a.s_out[i] = out;
        return inf_of<T>();
    }
    active += 1u;
    if constexpr (!GEO_EARLY) {
        gA = a.geoA[i];
        gB = a.geoB[i];
        if constexpr (sizeof(T) == 8) gR = a.geoR[i];
        gm2 = load_gm2(a, i, tp, T(0));
    }
    if constexpr (sizeof(T) != 8) gR = gA;   // unused: FP32 forms 1/|L n| itself
    T ui, vi;
    cell_velocity<T>(hi, own.y, own.z, h_dry, ui, vi);
    T f0 = T(0), f1 = T(0), f2 = T(0), sx = T(0), sy = T(0);
    int4 ei = make_int4(-1, -1, -1, 0);
    if constexpr (EDGES) ei = a.eidx[i];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int c = j == 0 ? code[0] : (j == 1 ? code[1] : code[2]);
        const V4<T> o = j == 0 ? nb[0] : (j == 1 ? nb[1] : nb[2]);
        const T lx = j == 0 ? gA.x : (j == 1 ? gA.z : gB.x);
        const T ly = j == 0 ? gA.y : (j == 1 ? gA.w : gB.y);
        const T l2 = edge_l2(lx, ly);
        const T rl = edge_rl<T>(j == 0 ? gR.x : (j == 1 ? gR.y : gR.z), l2);
        const T len = l2 * rl;
        const T n1 = lx * rl, n2 = ly * rl;     // this cell's outward unit normal
        T F0, F1, F2;
        if (c >= 0) {
            T src;
            if constexpr (EDGES) {
                if (!gt_pos(hi, h_dry) && !gt_pos(o.x, h_dry)) {
                    const T zs = max_finite(zi, o.w);
                    const T hsi = max_zero(hi + zi - zs);
                    F0 = T(0); F1 = T(0); F2 = T(0);
                    src = T(0.5) * g * (hsi * hsi - hi * hi);
                } else {
                    int e = j == 0 ? ei.x : (j == 1 ? ei.y : ei.z);
                    if (a.debug && !(e >= 0 && e < a.n_edges)) {
                        atomicOr(status, kStatusBadIndex);
                        e = 0;
                    }
                    const V4<T> fl = a.eflux[e];
                    if (c & kFlipBit) {
                        F0 = -fl.x; F1 = -fl.y; F2 = -fl.z;
                        src = a.esrc[e];
                    } else {
                        F0 = fl.x; F1 = fl.y; F2 = fl.z;
                        src = fl.w;
                    }
                }
            } else {
                edge_interior<T>(hi, ui, vi, zi, o.x, o.y, o.z, o.w, n1, n2, (c & kFlipBit) != 0, g, h_dry, F0, F1,
                                 F2, src, a.hll != 0);
            }
            sx += src * lx;
            sy += src * ly;
        } else {
            const int grp = -1 - c;
            edge_boundary<T>(a.bc_kind(grp), a.bc_value(grp), hi, ui, vi, zi, n1, n2, g, h_dry, F0, F1, F2,
                             a.hll != 0);
        }
        f0 += len * F0;
        f1 += len * F1;
        f2 += len * F2;
    }
    return finish_cell<T>(a, i, own, f0, f1, f2, sx, sy, gB.z, gB.w, gm2, dt, n_clamped, status);
    }
}

// ---- the fused step: fluxes + bed source + BCs + friction + update + next dt ------
// Grid-stride over cells with about one resident wave of blocks, so the block
// reduction (and its barrier) runs once per block.  With STAGES > 1 each
// thread keeps its next STAGES-1 cells' state and topology records in flight
// through cp.async into its own shared-memory slots.
template <typename T, int BLOCK, int MINB, int STAGES, bool GEO_EARLY, bool EDGES = false>
__global__ void __launch_bounds__(BLOCK, MINB) step_kernel(const StepArgs<T> a) {
    const WarpDt<T> wdt = warp_step_dt<T>(a.cfl, a.dt_read, a.dt_fixed);
    const double dt_d = wdt.d;
    const bool have_dt = wdt.have;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.dt_reset = kInfBits;
        if (have_dt) *a.t += dt_d;
        else atomicOr(a.status, kStatusDry);
        if (a.dt_log) *a.dt_log = dt_d;
    }
    T cand = inf_of<T>();
    unsigned active = 0u;
    const long long stride = (long long)gridDim.x * BLOCK;
    long long i = (long long)blockIdx.x * BLOCK + threadIdx.x;
    if (!have_dt) {
        for (; i < a.n; i += stride) a.s_out[i] = a.s_in[i];
    } else if constexpr (STAGES <= 1) {
        const T dt = wdt.t;
        for (; i < a.n; i += stride) {
            const V4<T> own = a.s_in[i];
            const int4 tp = a.topo[i];
            cand = min_nonneg(cand, update_cell<T, GEO_EARLY, EDGES>(a, i, own, tp, dt, active, a.n_clamped, a.status));
        }
    } else {
        __shared__ V4<T> st_own[STAGES][BLOCK];
        __shared__ int4 st_topo[STAGES][BLOCK];
        const T dt = wdt.t;
        const int tid = threadIdx.x;
#pragma unroll
        for (int s = 0; s < STAGES - 1; ++s) {
            const long long c = i + (long long)s * stride;
            if (c < a.n) {
                cp_async_record<sizeof(V4<T>)>(&st_own[s][tid], &a.s_in[c]);
                cp_async_record<16>(&st_topo[s][tid], &a.topo[c]);
            }
            cp_async_commit();
        }
        int slot = 0;
        for (; i < a.n; i += stride) {
            const long long c = i + (long long)(STAGES - 1) * stride;
            const int fill = slot == 0 ? STAGES - 1 : slot - 1;
            if (c < a.n) {
                cp_async_record<sizeof(V4<T>)>(&st_own[fill][tid], &a.s_in[c]);
                cp_async_record<16>(&st_topo[fill][tid], &a.topo[c]);
            }
            cp_async_commit();
            cp_async_wait<STAGES - 1>();
            const V4<T> own = st_own[slot][tid];
            const int4 tp = st_topo[slot][tid];
            cand = min_nonneg(cand, update_cell<T, GEO_EARLY, EDGES>(a, i, own, tp, dt, active, a.n_clamped, a.status));
            slot = slot == STAGES - 1 ? 0 : slot + 1;
        }
        cp_async_wait<0>();
    }
    block_min_publish<BLOCK>(cand, a.dt_write, active, a.n_active);
}

// ---- the fused step over pairs of adjacent cells (FP32) -----------------------------
// Thread work item p is the cell pair (2p, 2p+1).  The mesh's pairing order
// puts two cells that share an edge at such positions, with that edge as
// local edge 0 of both, for most cells.  The edge's flux is then evaluated
// once, by the first cell, and the second takes its negative: bit for bit
// what it would evaluate itself (the edge's canonical evaluation, rotated with
// the exactly opposite normal), while each cell still sums its edges in local
// order, so the results equal the one-cell kernels'.  Five Riemann problems
// per pair instead of six.  Unmatched cells come in whole warps of their own.
template <int BLOCK, int MINB, bool GEO_EARLY>
__global__ void __launch_bounds__(BLOCK, MINB) step_kernel_pair(const StepArgs<float> a) {
    const WarpDt<float> wdt = warp_step_dt<float>(a.cfl, a.dt_read, a.dt_fixed);
    const bool have_dt = wdt.have;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.dt_reset = kInfBits;
        if (have_dt) *a.t += wdt.d;
        else atomicOr(a.status, kStatusDry);
        if (a.dt_log) *a.dt_log = wdt.d;
    }
    float cand = inf_of<float>();
    unsigned active = 0u;
    // 32-bit pair indices (a mesh has fewer than 2^30 cells): fewer live registers
    const unsigned stride = gridDim.x * BLOCK;
    const unsigned np = (unsigned)((a.n + 1) >> 1);
    unsigned p = blockIdx.x * BLOCK + threadIdx.x;
    __shared__ PairEdge slot[BLOCK];
    volatile PairEdge* pe = &slot[threadIdx.x];
    if (!have_dt) {
        for (long long i = p; i < a.n; i += (long long)gridDim.x * BLOCK) a.s_out[i] = a.s_in[i];
    } else {
        const float dt = wdt.t;
        for (; p < np; p += stride) {
            const long long iA = 2 * (long long)p, iB = iA + 1;
            const bool hasB = iB < a.n;
            const V4<float> ownA = a.s_in[iA];
            const int4 tpA = a.topo[iA];
            const int cB = hasB ? __ldg(&a.topo[iB].x) : -1;
            const bool shared = tpA.x >= 0 && cB >= 0 && (long long)(tpA.x & kNbrMask) == iB &&
                                (long long)(cB & kNbrMask) == iA;
            // the first cell gives its edge 0; the handed-over flux waits in shared
            // memory, not in registers, through the first cell's other edges
            int mode = shared ? kPairGive : kPairNone;
            cand = min_nonneg(cand, update_cell_f32<GEO_EARLY, false, 1>(a, iA, ownA, tpA, dt, active, a.n_clamped,
                                                                         a.status, &mode, pe));
            if (hasB) {
                // the second cell's records are read after the first cell's update
                // (fewer live registers)
                const V4<float> ownB = a.s_in[iB];
                const int4 tpB = a.topo[iB];
                int modeB = mode == kPairGiven ? kPairTake : kPairNone;
                cand = min_nonneg(cand, update_cell_f32<GEO_EARLY, false, 2>(a, iB, ownB, tpB, dt, active,
                                                                             a.n_clamped, a.status, &modeB, pe));
            }
        }
    }
    block_min_publish<BLOCK>(cand, a.dt_write, active, a.n_active);
}

// ---- edge pass: each interior edge's flux once per step ----------------------------
// The canonical evaluation of an interior edge (from its left cell, Eq 12-30)
// is the one both of its cells make in step_kernel; here one thread makes it
// and stores the flux leaving the left cell and both cells' bed source
// factors, which the cell pass (step_kernel with EDGES) applies with the
// left/right sign.  Edges with both cells dry are skipped: the cells form
// them inline.  Worth it where the flux arithmetic, not memory, bounds the
// step (the FP64 pipe).
template <typename T, int BLOCK>
__global__ void __launch_bounds__(BLOCK) edge_flux_kernel(const StepArgs<T> a) {
    const T g = a.g, h_dry = a.h_dry;
    const long long stride = (long long)gridDim.x * BLOCK;
    for (long long e = (long long)blockIdx.x * BLOCK + threadIdx.x; e < a.n_edges; e += stride) {
        const int2 lr = a.ecells[e];
        if (a.debug && !(lr.x >= 0 && lr.x < a.n && lr.y >= 0 && lr.y < a.n)) {
            atomicOr(a.status, kStatusBadIndex);
            continue;
        }
        const V4<T> L = a.s_in[lr.x], R = a.s_in[lr.y];
        if (!gt_pos(L.x, h_dry) && !gt_pos(R.x, h_dry)) continue;
        const T lx = a.eln[2 * e], ly = a.eln[2 * e + 1];
        const T l2 = edge_l2(lx, ly);
        T pre = T(0);
        if constexpr (sizeof(T) == 8) pre = a.erl[e];
        const T rl = edge_rl<T>(pre, l2);
        const T n1 = lx * rl, n2 = ly * rl;
        T ui, vi;
        cell_velocity<T>(L.x, L.y, L.z, h_dry, ui, vi);
        T F0, F1, F2, sl, sr;
        edge_interior<T>(L.x, ui, vi, L.w, R.x, R.y, R.z, R.w, n1, n2, false, g, h_dry, F0, F1, F2, sl, a.hll != 0,
                         &sr);
        V4<T> f;
        f.x = F0; f.y = F1; f.z = F2; f.w = sl;
        a.eflux[e] = f;
        a.esrc[e] = sr;
    }
}

// ---- the fused step with activity bytes ------------------------------------------
// One byte per cell in three rotating buffers.  In the buffer a step reads, a
// cell's byte is non-zero exactly when the cell is not quiet: it is wet, or a
// neighbour is wet, or it has an inflow or fixed-stage edge.  The step marks
// in the next buffer (plain stores of 1, so concurrent marks of one byte
// agree) every cell that is wet after its update together with its
// neighbours, and every cell with an inflow/stage edge; and it clears each
// cell's byte in the third buffer, which the step after next fills.  A cell
// whose byte is 0 takes the quiet update (h, 0, 0) without its topology
// record or its neighbours' states -- the same result the neighbour test of
// update_cell gives, bit for bit.
//
// Per-thread cp.async pipeline over the thread's cells c_k = i0 + k stride:
// iteration k issues the topology of c_{k+1} (only if its byte is set), then
// the activity bytes of c_{k+PF+1} (8 lanes copy the warp's 32 bytes) and the
// state record of c_{k+PF}; it then processes c_k.  PF (the prefetch
// distance of the streamed state, >= 2) is a compiled shape parameter.
template <typename T, int BLOCK, int MINB, bool GEO_EARLY, int PF>
__global__ void __launch_bounds__(BLOCK, MINB) step_kernel_act(const StepArgs<T> a) {
    static_assert(BLOCK % 32 == 0, "warps of whole cells");
    static_assert(PF >= 2, "the wait counts below assume a prefetch distance of at least two cells");
    constexpr int NS = PF + 1;  // state and activity slots
    const WarpDt<T> wdt = warp_step_dt<T>(a.cfl, a.dt_read, a.dt_fixed);
    const double dt_d = wdt.d;
    const bool have_dt = wdt.have;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.dt_reset = kInfBits;
        if (have_dt) *a.t += dt_d;
        else atomicOr(a.status, kStatusDry);
        if (a.dt_log) *a.dt_log = dt_d;
    }
    T cand = inf_of<T>();
    unsigned active = 0u;
    // 32-bit cell indices: the host allows this kernel only for n < 2^29, so
    // c + (PF + 1) stride < 2^32 with stride <= n + BLOCK and PF <= 5
    const unsigned stride = gridDim.x * BLOCK;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned i0 = blockIdx.x * BLOCK + tid;
    const unsigned n = (unsigned)a.n;
    if (!have_dt) {
        // no step: the state and its activity carry over unchanged
        for (unsigned c = i0; c < n; c += stride) {
            a.s_out[c] = a.s_in[c];
            a.act_next[c] = a.act_in[c];
            a.act_clear[c] = 0;
        }
    } else {
        static_assert(PF <= 5, "32-bit indices");
        __shared__ V4<T> st_own[NS][BLOCK];
        __shared__ int4 st_topo[2][BLOCK];
        __shared__ unsigned st_act[NS][BLOCK / 4];  // 32 activity bytes per warp per stage
        __shared__ unsigned st_prev[NS][BLOCK / 4]; // and the previous step's (act_clear) bytes
        const T dt = wdt.t;
        // warp w of the block owns st_act[.][8 w .. 8 w + 7]; lanes 0..7 copy 4 bytes each
        auto act_copy = [&](int slot, unsigned c) {
            const unsigned base = c - lane;
            if (lane < 8 && base < n) {
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(
                                 (unsigned)__cvta_generic_to_shared(&st_act[slot][warp * 8 + lane])),
                             "l"(a.act_in + base + 4 * lane)
                             : "memory");
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(
                                 (unsigned)__cvta_generic_to_shared(&st_prev[slot][warp * 8 + lane])),
                             "l"(a.act_clear + base + 4 * lane)
                             : "memory");
            }
        };
        // bit 0: the cell runs the flux path in this step (bit 0 of its byte);
        // bit 1: the previous step's byte is not 0 (the cell ran the flux path
        // then, or the bytes were rebuilt less than two steps ago)
        auto act_byte = [&](int slot) -> unsigned {
            return (((const unsigned char*)&st_act[slot][warp * 8])[lane] & 1u) |
                   (((const unsigned char*)&st_prev[slot][warp * 8])[lane] ? 2u : 0u);
        };
        // prologue: activity of c_0 .. c_PF and states of c_0 .. c_{PF-1}; then topology of c_0
#pragma unroll
        for (int q = 0; q <= PF; ++q) act_copy(q, i0 + q * stride);
#pragma unroll
        for (int q = 0; q < PF; ++q)
            if (i0 + q * stride < n) cp_async_record<sizeof(V4<T>)>(&st_own[q][tid], &a.s_in[i0 + q * stride]);
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
        unsigned f_cur = act_byte(0);
        if ((f_cur & 1u) && i0 < n) cp_async_record<16>(&st_topo[0][tid], &a.topo[i0]);
        cp_async_commit();                                       // T_{-1}
        cp_async_commit();                                       // H_{-1} (empty: its copies were in the first group)
        int ks = 0, k2 = 0;  // k mod NS, k mod 2
        for (unsigned c = i0; c - lane < n; c += stride) {
            const int ks1 = ks + 1 == NS ? 0 : ks + 1;          // slot of c_{k+1}
            const int ksp = ks == 0 ? NS - 1 : ks - 1;          // slot of c_{k+PF} (c_{k-1}'s, consumed)
            // groups so far: ..., T_{k-1}, H_{k-1}; H_{k-PF} and older (activity of
            // c_{k+1}, state of c_k) must be complete, which H_{k-2} implies
            cp_async_wait<2>();
            __syncwarp();
            const unsigned f_next = act_byte(ks1);
            const unsigned c1 = c + stride, cp = c + PF * stride, cp1 = c + (PF + 1) * stride;
            if ((f_next & 1u) && c1 < n) cp_async_record<16>(&st_topo[k2 ^ 1][tid], &a.topo[c1]);
            cp_async_commit();                                   // T_k
            __syncwarp();                                        // every lane has read slot ks before it refills
            act_copy(ks, cp1);
            if (cp < n) cp_async_record<sizeof(V4<T>)>(&st_own[ksp][tid], &a.s_in[cp]);
            cp_async_commit();                                   // H_k
            cp_async_wait<3>();                                  // T_{k-1}: the topology of c_k
            if (c < n) {
                const V4<T> own = st_own[ks][tid];
                if (!(f_cur & 1u)) {
                    // quiet: the new state is (h, 0, 0); if the cell was quiet in the
                    // previous step too, the output buffer (the state of two steps
                    // ago, itself dry at rest with the same h) holds it already
                    if (f_cur & 2u) {
                        V4<T> out;
                        out.x = own.x; out.y = T(0); out.z = T(0); out.w = own.w;
                        a.s_out[c] = out;
                    }
                } else {
                    const T r = update_cell<T, GEO_EARLY>(a, c, own, st_topo[k2][tid], dt, active, a.n_clamped,
                                                          a.status);
                    cand = min_nonneg(cand, r);
                    const bool wet = r < inf_of<T>();
                    // the topology record is read again from shared memory rather than kept
                    // live in registers across the update
                    const volatile int* tv = (const volatile int*)&st_topo[k2][tid];
                    if (wet || (tv[3] & kStaticBit)) a.act_next[c] = 1;
                    if (wet) {
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            const int code = tv[j];
                            if (code >= 0 && (!a.debug || code_ok(code, a.n, a.n_groups)))
                                a.act_next[code & kNbrMask] = 1;
                        }
                    }
                }
                a.act_clear[c] = 0;
            }
            f_cur = f_next;
            ks = ks1;
            k2 ^= 1;
        }
        cp_async_wait<0>();
    }
    block_min_publish<BLOCK>(cand, a.dt_write, active, a.n_active);
}

// Activity bytes of a state (into a buffer filled with 2): a wet cell marks
// itself and its neighbours, a cell with an inflow/stage edge marks itself.
// Bit 0 says that the cell runs the flux path; bit 1, set in every rebuilt
// byte, keeps the step after next from leaving a quiet state in place (its
// output buffer holds the state that was set, not a step's result).
template <typename T>
__global__ void act_init_kernel(const V4<T>* __restrict__ s, const int4* __restrict__ topo, long long n, T h_dry,
                                unsigned char* __restrict__ act) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const bool wet = s[c].x > h_dry;
    const int4 tp = topo[c];
    if (wet || (tp.w & kStaticBit)) act[c] = 3;
    if (wet) {   // (an out-of-range index is skipped here; the step's debug checks report it)
        if (tp.x >= 0 && (tp.x & kNbrMask) < n) act[tp.x & kNbrMask] = 3;
        if (tp.y >= 0 && (tp.y & kNbrMask) < n) act[tp.y & kNbrMask] = 3;
        if (tp.z >= 0 && (tp.z & kNbrMask) < n) act[tp.z & kNbrMask] = 3;
    }
}

// ---- batched ensemble step -------------------------------------------------------
// Members advance together, each with its own CFL step: one launch covers every
// member's cells.  When a block moves on to another member, its warps publish
// the finished member's CFL minimum (warp shuffle, one atomicMin per warp, no
// barrier).
// The warp minimum is taken in the state precision and widened once (exact:
// widening is monotone), which keeps FP32 kernels off the FP64 pipe.
template <typename T>
__device__ __forceinline__ void warp_min_publish(T cand, unsigned long long* dst) {
    for (int o = 16; o > 0; o >>= 1) cand = tmin(cand, __shfl_xor_sync(0xffffffffu, cand, o));
    if ((threadIdx.x & 31) == 0 && cand < inf_of<T>())
        atomicMin(dst, (unsigned long long)__double_as_longlong((double)cand));
}

// Tiles are dealt to blocks in round-robin chunks of 2^chunk_log2 tiles,
// which balances wet (expensive) and dry (cheap) members across the GPU while
// the member still changes only at chunk or member boundaries.  The chunk
// size, the tile size BLOCK and the grid are launch shapes chosen by the
// autotuner; none of them changes any cell's arithmetic.
__device__ __forceinline__ long long ens_tile_of(long long k, long long nchunk_stride, long long b, int cl2) {
    const long long mask = (1LL << cl2) - 1;
    return ((b + (k >> cl2) * nchunk_stride) << cl2) + (k & mask);
}

template <typename T, int BLOCK, int MINB, int STAGES, bool GEO_EARLY, bool EDGES = false>
__global__ void __launch_bounds__(BLOCK, MINB) ensemble_step_kernel(const EnsArgs<T> a) {
    static_assert(kEnsPad % BLOCK == 0, "a tile must not straddle two members");
    const long long G = gridDim.x, b = blockIdx.x;
    const int cl2 = a.chunk_log2;
    const long long t_lo = a.cell_lo / BLOCK;              // tiles from cell_lo on
    const long long n_tiles = (a.n_total - a.cell_lo) / BLOCK;
    const long long n_chunks = (n_tiles + (1LL << cl2) - 1) >> cl2;
    // this block's chunks: b, b + G, b + 2G, ... ; k counts its tiles
    const long long my_chunks = b < n_chunks ? (n_chunks - 1 - b) / G + 1 : 0;
    const long long k_end = my_chunks << cl2;
    const int tid = threadIdx.x;
    int member = -1;
    unsigned long long* sm = nullptr;
    bool have_dt = false;
    T dt = T(0);
    T cand = inf_of<T>();
    unsigned active = 0u;
    __shared__ V4<T> st_own[STAGES > 1 ? STAGES : 1][BLOCK];
    __shared__ int4 st_topo[STAGES > 1 ? STAGES : 1][BLOCK];
    if constexpr (STAGES > 1) {
#pragma unroll
        for (int s = 0; s < STAGES - 1; ++s) {
            const long long tile = ens_tile_of(s, G, b, cl2);
            if (s < k_end && tile < n_tiles) {
                const long long c = (tile + t_lo) * BLOCK + tid;
                cp_async_record<sizeof(V4<T>)>(&st_own[s][tid], &a.s_in[c]);
                cp_async_record<16>(&st_topo[s][tid], &a.topo[c]);
            }
            cp_async_commit();
        }
    }
    int slot = 0;
    for (long long k = 0; k < k_end; ++k) {
        const long long tile = ens_tile_of(k, G, b, cl2);
        if (tile >= n_tiles) break;                        // ragged last chunk
        const long long cell0 = (tile + t_lo) * BLOCK;
        const int mk = a.tile_member[cell0 / kEnsPad];     // uniform across the block
        if (mk != member) {
            if (member >= 0) warp_min_publish<T>(cand, sm + a.slot_write);
            cand = inf_of<T>();
            member = mk;
            sm = a.small + 8 * (long long)mk;
            // mk is uniform across the block, so every lane is here
            const WarpDt<T> wdt = warp_step_dt<T>(a.cfl[mk], (const double*)(sm + a.slot_read), nullptr);
            const double dt_d = wdt.d;
            have_dt = wdt.have;
            dt = wdt.t;
            if (cell0 == a.member_first_tile[mk] * kEnsPad && tid == 0) {
                sm[a.slot_reset] = kInfBits;
                if (have_dt) *(double*)(sm + 3) += dt_d;
                else atomicOr((unsigned*)(sm + 4), kStatusDry);
            }
        }
        const long long i = cell0 + tid;
        V4<T> own;
        int4 tp;
        if constexpr (STAGES > 1) {
            const long long kn = k + STAGES - 1;
            const long long nt = ens_tile_of(kn, G, b, cl2);
            const int fill = slot == 0 ? STAGES - 1 : slot - 1;
            if (kn < k_end && nt < n_tiles) {
                const long long c = (nt + t_lo) * BLOCK + tid;
                cp_async_record<sizeof(V4<T>)>(&st_own[fill][tid], &a.s_in[c]);
                cp_async_record<16>(&st_topo[fill][tid], &a.topo[c]);
            }
            cp_async_commit();
            cp_async_wait<STAGES - 1>();
            own = st_own[slot][tid];
            tp = st_topo[slot][tid];
            slot = slot == STAGES - 1 ? 0 : slot + 1;
        } else {
            own = a.s_in[i];
            tp = a.topo[i];
        }
        if (have_dt)
            cand = min_nonneg(cand, update_cell<T, GEO_EARLY, EDGES>(a, i, own, tp, dt, active, sm + 5, (unsigned*)(sm + 4)));
        else
            a.s_out[i] = own;
    }
    if constexpr (STAGES > 1) cp_async_wait<0>();
    if (member >= 0) warp_min_publish<T>(cand, sm + a.slot_write);
    active = __reduce_add_sync(0xffffffffu, active);
    if ((tid & 31) == 0 && active) atomicAdd(a.n_active, (unsigned long long)active);
}

// ---- batched ensemble step with dynamically taken chunks ------------------------------
// Each block takes its next chunk of 2^chunk_log2 tiles from a per-step
// counter (one atomicAdd per chunk, taken one chunk ahead), so blocks that
// drew cheap (dry) chunks take more of them and the grid finishes together.
// Which block updates a cell changes nothing in the cell's arithmetic, and the
// per-member minimum and the counters are order-independent: the results are
// those of the static schedule bit for bit.
template <typename T, int BLOCK, int MINB, bool GEO_EARLY>
__global__ void __launch_bounds__(BLOCK, MINB) ensemble_step_kernel_dyn(const EnsArgs<T> a) {
    static_assert(kEnsPad % BLOCK == 0, "a tile must not straddle two members");
    const int cl2 = a.chunk_log2;
    const long long t_lo = a.cell_lo / BLOCK;              // tiles from cell_lo on
    const long long n_tiles = (a.n_total - a.cell_lo) / BLOCK;
    const unsigned n_chunks = (unsigned)((n_tiles + (1LL << cl2) - 1) >> cl2);
    const int tid = threadIdx.x;
    __shared__ unsigned s_chunk[2];
    if (blockIdx.x == 0 && tid == 0) a.sched[a.sched_reset] = 0u;   // the counter of the step after next
    if (tid == 0) s_chunk[0] = atomicAdd(&a.sched[a.sched_slot], 1u);
    __syncthreads();
    int member = -1;
    unsigned long long* sm = nullptr;
    bool have_dt = false;
    T dt = T(0);
    T cand = inf_of<T>();
    unsigned active = 0u;
    unsigned chunk = s_chunk[0];
    for (int it = 0; chunk < n_chunks; ++it) {
        if (tid == 0) s_chunk[(it + 1) & 1] = atomicAdd(&a.sched[a.sched_slot], 1u);   // the next chunk, ahead
        const long long t0 = (long long)chunk << cl2;
        for (int q = 0; q < (1 << cl2); ++q) {
            const long long tile = t0 + q;
            if (tile >= n_tiles) break;                    // ragged last chunk
            const long long cell0 = (tile + t_lo) * BLOCK;
            const int mk = a.tile_member[cell0 / kEnsPad];  // uniform across the block
            if (mk != member) {
                if (member >= 0) warp_min_publish<T>(cand, sm + a.slot_write);
                cand = inf_of<T>();
                member = mk;
                sm = a.small + 8 * (long long)mk;
                const WarpDt<T> wdt = warp_step_dt<T>(a.cfl[mk], (const double*)(sm + a.slot_read), nullptr);
                have_dt = wdt.have;
                dt = wdt.t;
                if (cell0 == a.member_first_tile[mk] * kEnsPad && tid == 0) {
                    sm[a.slot_reset] = kInfBits;
                    if (have_dt) *(double*)(sm + 3) += wdt.d;
                    else atomicOr((unsigned*)(sm + 4), kStatusDry);
                }
            }
            const long long i = cell0 + tid;
            const V4<T> own = a.s_in[i];
            const int4 tp = a.topo[i];
            if (have_dt)
                cand = min_nonneg(cand, update_cell<T, GEO_EARLY>(a, i, own, tp, dt, active, sm + 5, (unsigned*)(sm + 4)));
            else
                a.s_out[i] = own;
        }
        __syncthreads();   // the next chunk's index is visible, and every thread has read this one
        chunk = s_chunk[(it + 1) & 1];
    }
    if (member >= 0) warp_min_publish<T>(cand, sm + a.slot_write);
    active = __reduce_add_sync(0xffffffffu, active);
    if ((tid & 31) == 0 && active) atomicAdd(a.n_active, (unsigned long long)active);
}

// ---- batched ensemble step with activity bytes ----------------------------------------
// The activity mode of step_kernel_act over the concatenated members: the same
// bytes, marks and per-thread cp.async pipeline, with the thread's cells taken
// tile by tile in the ensemble's round-robin chunk order.  Tiles are whole
// (members are padded), so a tile is valid for every lane or for none.  Cells
// are indexed with 32 bits (the host allows this kernel below 2^29 cells).
//
// DYN takes the chunks dynamically, as ensemble_step_kernel_dyn does: the
// block's j-th chunk is s_ch[j mod 3], drawn from the step's counter two
// chunks ahead by thread 0 at the start of chunk j - 2 and published by the
// barrier that starts chunk j - 1, so the pipeline's look-ahead of three
// cells (into chunk j + 1 at most, chunks being at least 4 tiles) always
// finds its tile.  The slot refilled at the start of chunk j held chunk
// j - 1, which nothing reads after that barrier.
template <typename T, int BLOCK, int MINB, bool GEO_EARLY, bool DYN = false, bool QUEUE = false>
__global__ void __launch_bounds__(BLOCK, MINB) ensemble_step_kernel_act(const EnsArgs<T> a) {
    static_assert(kEnsPad % BLOCK == 0, "a tile must not straddle two members");
    constexpr unsigned kNone = 0xFFFFFFFFu;
    const unsigned G = gridDim.x, b = blockIdx.x;
    const int cl2 = a.chunk_log2;                   // >= 2 with DYN (the host checks)
    const unsigned t_lo = (unsigned)(a.cell_lo / BLOCK);           // tiles from cell_lo on
    const unsigned n_tiles = (unsigned)((a.n_total - a.cell_lo) / BLOCK);
    const unsigned n_chunks = (n_tiles + (1u << cl2) - 1) >> cl2;
    const unsigned my_chunks = b < n_chunks ? (n_chunks - 1 - b) / G + 1 : 0;
    const unsigned k_end = DYN ? kNone : my_chunks << cl2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ unsigned s_ch[3];
    if constexpr (DYN) {
        if (b == 0 && tid == 0) a.sched[a.sched_reset] = 0u;   // the counter of the step after next
        if (tid == 0) {
            s_ch[0] = atomicAdd(&a.sched[a.sched_slot], 1u);
            s_ch[1] = atomicAdd(&a.sched[a.sched_slot], 1u);
        }
        __syncthreads();
    }
    // this thread's cell in the block's k-th tile (kNone past the end)
    auto cell_of = [&](unsigned k) -> unsigned {
        if constexpr (DYN) {
            const unsigned ch = s_ch[(k >> cl2) % 3];
            if (ch >= n_chunks) return kNone;
            const unsigned t = (ch << cl2) + (k & ((1u << cl2) - 1));
            return t < n_tiles ? (t + t_lo) * BLOCK + tid : kNone;
        } else {
            if (k >= k_end) return kNone;
            const unsigned t = ((b + (k >> cl2) * G) << cl2) + (k & ((1u << cl2) - 1));
            return t < n_tiles ? (t + t_lo) * BLOCK + tid : kNone;
        }
    };
    __shared__ V4<T> st_own[3][BLOCK];
    __shared__ int4 st_topo[QUEUE ? 1 : 2][BLOCK];
    // QUEUE: each warp's cells that run the flux path, a ring of 64 slots
    __shared__ unsigned s_q[QUEUE ? BLOCK / 32 : 1][64];
    unsigned qh = 0u, qt = 0u;                               // warp-uniform head and tail
    // per warp: the 32 activity bytes of its cells in 3 stages (lanes 0..7 copy
    // 4 each).  Unlike step_kernel_act, this kernel writes every quiet state:
    // leaving those quiet in two steps in place measured slower here (the
    // kernel is bound by instruction issue, not by its bytes).
    __shared__ unsigned st_act[3][BLOCK / 4];
    auto act_copy = [&](int slot, unsigned c) {
        if (lane < 8 && c != kNone)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(
                             (unsigned)__cvta_generic_to_shared(&st_act[slot][warp * 8 + lane])),
                         "l"(a.act_in + (c - lane) + 4 * lane)
                         : "memory");
    };
    // whether the cell runs the flux path (bit 0 of its byte)
    auto act_byte = [&](int slot) -> unsigned {
        return ((const unsigned char*)&st_act[slot][warp * 8])[lane] & 1u;
    };
    int member = -1;
    unsigned long long* sm = nullptr;
    bool have_dt = false;
    T dt = T(0);
    T cand = inf_of<T>();
    unsigned active = 0u;
    // QUEUE: the full update of one queued cell (topology read here), its marks
    auto run_queued = [&](unsigned cq) {
        const V4<T> own = a.s_in[cq];
        const int4 tp = a.topo[cq];
        const T r = update_cell<T, GEO_EARLY>(a, cq, own, tp, dt, active, sm + 5, (unsigned*)(sm + 4));
        cand = min_nonneg(cand, r);
        const bool wet = r < inf_of<T>();
        if (wet || (tp.w & kStaticBit)) a.act_next[cq] = 1;
        if (wet) {
            const int code[3] = {tp.x, tp.y, tp.z};
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (code[j] >= 0 && (!a.debug || code_ok(code[j], a.n_total, a.n_groups)))
                    a.act_next[code[j] & kNbrMask] = 1;
        }
    };
    // QUEUE: the queued cells left, on as many lanes (warp-uniform call)
    auto flush = [&]() {
        if constexpr (QUEUE) {
            const unsigned nq = qh - qt;
            if (lane < nq) run_queued(s_q[warp][(qt + lane) & 63]);
            qt = qh;
            __syncwarp();
        }
    };
    {
        const unsigned c0 = cell_of(0), c1 = cell_of(1), c2 = cell_of(2);
        act_copy(0, c0);
        act_copy(1, c1);
        act_copy(2, c2);
        if (c0 != kNone) cp_async_record<sizeof(V4<T>)>(&st_own[0][tid], &a.s_in[c0]);
        if (c1 != kNone) cp_async_record<sizeof(V4<T>)>(&st_own[1][tid], &a.s_in[c1]);
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
    }
    unsigned f_cur = act_byte(0);
    {
        const unsigned c0 = cell_of(0);
        if (!QUEUE && f_cur && c0 != kNone) cp_async_record<16>(&st_topo[0][tid], &a.topo[c0]);
    }
    cp_async_commit();                                           // T_{-1}
    cp_async_commit();                                           // H_{-1} (empty)
    int k3 = 0, k2 = 0;
    for (unsigned k = 0; k < k_end; ++k) {
        if constexpr (DYN) {
            if ((k & ((1u << cl2) - 1)) == 0) {                  // a chunk starts (block-uniform)
                if (k) __syncthreads();
                if (tid == 0) s_ch[((k >> cl2) + 2) % 3] = atomicAdd(&a.sched[a.sched_slot], 1u);
            }
        }
        const unsigned c = cell_of(k);
        if (c == kNone) break;                                   // ragged last chunk (block-uniform)
        const int mk = a.tile_member[(c - tid) / kEnsPad];       // uniform across the block
        if (mk != member) {
            if (member >= 0) {
                flush();   // with the member's own step and status block
                warp_min_publish<T>(cand, sm + a.slot_write);
            }
            cand = inf_of<T>();
            member = mk;
            sm = a.small + 8 * (long long)mk;
            const WarpDt<T> wdt = warp_step_dt<T>(a.cfl[mk], (const double*)(sm + a.slot_read), nullptr);
            have_dt = wdt.have;
            dt = wdt.t;
            if ((long long)(c - tid) == a.member_first_tile[mk] * kEnsPad && tid == 0) {
                sm[a.slot_reset] = kInfBits;
                if (have_dt) *(double*)(sm + 3) += wdt.d;
                else atomicOr((unsigned*)(sm + 4), kStatusDry);
            }
        }
        const int k3n = k3 == 2 ? 0 : k3 + 1, k3nn = k3n == 2 ? 0 : k3n + 1;
        cp_async_wait<2>();
        __syncwarp();
        const unsigned f_next = act_byte(k3n);
        const unsigned c1 = cell_of(k + 1), c2 = cell_of(k + 2), c3 = cell_of(k + 3);
        if (!QUEUE && f_next && c1 != kNone) cp_async_record<16>(&st_topo[k2 ^ 1][tid], &a.topo[c1]);
        cp_async_commit();                                       // T_k
        __syncwarp();
        act_copy(k3, c3);
        if (c2 != kNone) cp_async_record<sizeof(V4<T>)>(&st_own[k3nn][tid], &a.s_in[c2]);
        cp_async_commit();                                       // H_k
        cp_async_wait<3>();                                      // T_{k-1}: the topology of c_k
        const V4<T> own = st_own[k3][tid];
        if (!have_dt) {
            a.s_out[c] = own;
            a.act_next[c] = (unsigned char)f_cur;
        } else if constexpr (QUEUE) {
            // quiet cells now; the others join the warp's queue, which runs
            // whenever it holds a full warp of cells
            if (!f_cur) {
                V4<T> out;
                out.x = own.x; out.y = T(0); out.z = T(0); out.w = own.w;
                a.s_out[c] = out;
            }
            const bool runs = f_cur != 0u;
            const unsigned m = __ballot_sync(0xffffffffu, runs);
            if (runs) s_q[warp][(qh + __popc(m & ((1u << lane) - 1u))) & 63] = c;
            qh += __popc(m);
            __syncwarp();
            if (qh - qt >= 32u) {
                const unsigned cq = s_q[warp][(qt + lane) & 63];
                qt += 32u;
                __syncwarp();   // read before later appends reuse the slot
                run_queued(cq);
            }
        } else if (!f_cur) {
            V4<T> out;
            out.x = own.x; out.y = T(0); out.z = T(0); out.w = own.w;
            a.s_out[c] = out;
        } else {
            const T r = update_cell<T, GEO_EARLY>(a, c, own, st_topo[k2][tid], dt, active, sm + 5,
                                                  (unsigned*)(sm + 4));
            cand = min_nonneg(cand, r);
            const bool wet = r < inf_of<T>();
            const volatile int* tv = (const volatile int*)&st_topo[k2][tid];
            if (wet || (tv[3] & kStaticBit)) a.act_next[c] = 1;
            if (wet) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int code = tv[j];
                    if (code >= 0 && (!a.debug || code_ok(code, a.n_total, a.n_groups)))
                        a.act_next[code & kNbrMask] = 1;
                }
            }
        }
        a.act_clear[c] = 0;
        f_cur = f_next;
        k3 = k3n;
        k2 ^= 1;
    }
    cp_async_wait<0>();
    if (member >= 0) {
        flush();
        warp_min_publish<T>(cand, sm + a.slot_write);
    }
    active = __reduce_add_sync(0xffffffffu, active);
    if ((tid & 31) == 0 && active) atomicAdd(a.n_active, (unsigned long long)active);
}

// ---- batched ensemble step over cell pairs (FP32) ------------------------------------
// A split ensemble places the members that are mostly wet at creation first in
// its layout; this kernel updates their spans [0, pair_spans), and one of the
// other ensemble kernels the rest (from cell_lo on) in the same step.  A block
// takes a contiguous run of spans (the wet members cost about the same per
// cell, so equal runs balance, and a block changes member rarely); its thread
// t updates the pair (2t, 2t+1) of the span (BLOCK pairs = kEnsPad cells)
// exactly as step_kernel_pair does, so the members' results are those of the
// plain solver bit for bit.
template <int BLOCK, int MINB, bool GEO_EARLY>
__global__ void __launch_bounds__(BLOCK, MINB) ensemble_step_kernel_pair(const EnsArgs<float> a) {
    static_assert(2 * BLOCK == kEnsPad, "a block's pairs are one span");
    const unsigned ns = a.pair_spans;
    const unsigned lo = (unsigned)((unsigned long long)ns * blockIdx.x / gridDim.x);
    const unsigned hi = (unsigned)((unsigned long long)ns * (blockIdx.x + 1) / gridDim.x);
    const int tid = threadIdx.x;
    __shared__ PairEdge slot[BLOCK];
    volatile PairEdge* pe = &slot[tid];
    unsigned active = 0u;
    // runs of spans of one member: the member's step size, then its spans; the
    // member's status block is addressed from its index where used
    for (unsigned t = lo; t < hi;) {
        const int mk = a.tile_member[t];       // uniform across the block
        unsigned long long* sm = a.small + 8 * mk;
        const WarpDt<float> wdt = warp_step_dt<float>(a.cfl[mk], (const double*)(sm + a.slot_read), nullptr);
        if ((long long)t == a.member_first_tile[mk] && tid == 0) {
            sm[a.slot_reset] = kInfBits;
            if (wdt.have) *(double*)(sm + 3) += wdt.d;
            else atomicOr((unsigned*)(sm + 4), kStatusDry);
        }
        if (!wdt.have) {
            for (; t < hi && a.tile_member[t] == mk; ++t) {
                const unsigned iA = t * kEnsPad + 2 * tid;
                a.s_out[iA] = a.s_in[iA];
                a.s_out[iA + 1] = a.s_in[iA + 1];
            }
            continue;
        }
        const float dt = wdt.t;
        float cand = inf_of<float>();
        for (; t < hi && a.tile_member[t] == mk; ++t) {
            const unsigned iA = t * kEnsPad + 2 * tid, iB = iA + 1;
            const V4<float> ownA = a.s_in[iA];
            const int4 tpA = a.topo[iA];
            const int cB = __ldg(&a.topo[iB].x);
            const bool shared = tpA.x >= 0 && cB >= 0 && (unsigned)(tpA.x & kNbrMask) == iB &&
                                (unsigned)(cB & kNbrMask) == iA;
            int mode = shared ? kPairGive : kPairNone;
            cand = min_nonneg(cand, update_cell_f32<GEO_EARLY, false, 1>(a, iA, ownA, tpA, dt, active,
                                                                         a.small + 8 * mk + 5,
                                                                         (unsigned*)(a.small + 8 * mk + 4), &mode,
                                                                         pe));
            const V4<float> ownB = a.s_in[iB];
            const int4 tpB = a.topo[iB];
            int modeB = mode == kPairGiven ? kPairTake : kPairNone;
            cand = min_nonneg(cand, update_cell_f32<GEO_EARLY, false, 2>(a, iB, ownB, tpB, dt, active,
                                                                         a.small + 8 * mk + 5,
                                                                         (unsigned*)(a.small + 8 * mk + 4), &modeB,
                                                                         pe));
        }
        warp_min_publish<float>(cand, a.small + 8 * mk + a.slot_write);
    }
    active = __reduce_add_sync(0xffffffffu, active);
    if ((tid & 31) == 0 && active) atomicAdd(a.n_active, (unsigned long long)active);
}

// ---- CFL min of a given state (used after swe_set_state) --------------------------
template <typename T, int BLOCK>
__global__ void __launch_bounds__(BLOCK) dt_kernel(const V4<T>* __restrict__ s, const V4<T>* __restrict__ geoB,
                                                   long long n, T g, T h_dry, unsigned long long* dt_write) {
    using A = Ar<T>;
    const long long i = (long long)blockIdx.x * BLOCK + threadIdx.x;
    T cand = inf_of<T>();
    if (i < n) {
        const V4<T> c = s[i];
        if (c.x > h_dry) {
            const T r = A::rcp_(c.x);
            const T u = c.y * r, v = c.z * r;
            cand = A::div_(geoB[i].w, A::sqrt_(g * c.x) + A::sqrt_(u * u + v * v));
        }
    }
    block_min_publish<BLOCK>(cand, dt_write);
}

// ---- layout conversion between caller arrays and the packed internal state --------
// pack: s[new] = (h[perm[new]], hu[..], hv[..], z[new])
template <typename T>
__global__ void pack_state_kernel(const T* __restrict__ h, const T* __restrict__ hu, const T* __restrict__ hv,
                                  const long long* __restrict__ perm, const T* __restrict__ z,
                                  V4<T>* __restrict__ s, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const long long o = perm[i];
        V4<T> v;
        v.x = h[o]; v.y = hu[o]; v.z = hv[o]; v.w = z[i];
        s[i] = v;
    }
}

template <typename T>
__global__ void unpack_state_kernel(const V4<T>* __restrict__ s, const long long* __restrict__ perm,
                                    T* __restrict__ h, T* __restrict__ hu, T* __restrict__ hv, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const long long o = perm[i];
        const V4<T> v = s[i];
        h[o] = v.x; hu[o] = v.y; hv[o] = v.z;
    }
}

// ---- batched Riemann flux (parity entry point) --------------------------------------
template <typename T>
__global__ void riemann_batch_kernel(long long n, const T* __restrict__ hL, const T* __restrict__ unL,
                                     const T* __restrict__ utL, const T* __restrict__ hR,
                                     const T* __restrict__ unR, const T* __restrict__ utR, T g, T h_dry,
                                     T* __restrict__ G1, T* __restrict__ G2, T* __restrict__ G3, T* __restrict__ S,
                                     int hll) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        T a, b, c, sp[3];
        riemann_hllc<T>(hL[i], unL[i], utL[i], hR[i], unR[i], utR[i], g, h_dry, a, b, c, sp, hll != 0);
        G1[i] = a; G2[i] = b; G3[i] = c;
        if (S) { S[3 * i] = sp[0]; S[3 * i + 1] = sp[1]; S[3 * i + 2] = sp[2]; }
    }
}

// ---- host-side launchers, one set per precision ------------------------------------
template <typename T>
struct Launch {
    // (block, min_blocks) pairs with a compiled kernel; see step_variants()
    // with a.act_in set, the activity kernel (stages ignored) runs
    static cudaError_t step(const StepArgs<T>& a, int block, int min_blocks, int stages, int geo_early,
                            cudaStream_t st);
    // with a.eflux set (and a.act_in not), the edge pass then the cell pass run
    static cudaError_t resident_blocks(int block, int min_blocks, int stages, int geo_early, int activity,
                                       int edges, int* per_sm);
    // compiled (block, min_blocks, stages, geo_early) shapes of the cell pass of the edge-pass step
    static int edge_variants(int (*out)[4], int max);
    // the edge pass alone (interior fluxes of a.s_in into a.eflux, a.esrc)
    static cudaError_t edge_flux(const StepArgs<T>& a, cudaStream_t st);
    // compiled (block, min_blocks, geo_early, stages = prefetch distance + 1) shapes of the activity kernel
    static int act_variants(int (*out)[4], int max);
    static cudaError_t act_init(const V4<T>* s, const int4* topo, long long n, T h_dry, unsigned char* act,
                                cudaStream_t st);
    // compiled (block, min_blocks, stages, geo_early) shapes of the step kernel; returns their number
    static int step_variants(int (*out)[4], int max);
    // the step over cell pairs (FP32 only; cudaErrorInvalidValue otherwise) with one of its
    // compiled (block, min_blocks, geo_early, stages) shapes; a.grid blocks of `block` threads,
    // each thread a pair at a time
    static cudaError_t step_pair(const StepArgs<T>& a, int block, int min_blocks, int geo_early, int stages,
                                 cudaStream_t st);
    static cudaError_t pair_resident_blocks(int block, int min_blocks, int geo_early, int stages, int* per_sm);
    static int pair_variants(int (*out)[4], int max);
    // batched ensemble step with one of its compiled (block, min_blocks, stages, geo_early) shapes
    static cudaError_t ensemble_step(const EnsArgs<T>& a, int block, int min_blocks, int stages, int geo_early,
                                     unsigned grid, cudaStream_t st);
    static cudaError_t ensemble_resident_blocks(int block, int min_blocks, int stages, int geo_early, int* per_sm);
    static int ensemble_variants(int (*out)[4], int max);
    // activity kernel of the ensemble: compiled (block, min_blocks, geo_early) shapes,
    // with round-robin (dynamic 0) or dynamically taken (dynamic 1) chunks
    // (queue 1, FP32: the cells that run the flux path are gathered per warp into
    // full warps first; compiled shapes from ensemble_actq_variants)
    static cudaError_t ensemble_step_act(const EnsArgs<T>& a, int block, int min_blocks, int geo_early,
                                         unsigned grid, cudaStream_t st, int dynamic = 0, int queue = 0);
    static cudaError_t ensemble_act_resident_blocks(int block, int min_blocks, int geo_early, int* per_sm,
                                                    int dynamic = 0, int queue = 0);
    static int ensemble_act_variants(int (*out)[3], int max);
    static int ensemble_actq_variants(int (*out)[3], int max);
    // edge pass of the ensemble (a.eflux set): edge kernel, then the cell pass of
    // one of its compiled (block, min_blocks, stages, geo_early) shapes
    static int ensemble_edge_variants(int (*out)[4], int max);
    // dynamically scheduled ensemble kernel: compiled (block, min_blocks, geo_early) shapes
    static cudaError_t ensemble_step_dyn(const EnsArgs<T>& a, int block, int min_blocks, int geo_early,
                                         unsigned grid, cudaStream_t st);
    static cudaError_t ensemble_dyn_resident_blocks(int block, int min_blocks, int geo_early, int* per_sm);
    static int ensemble_dyn_variants(int (*out)[3], int max);
    static cudaError_t ensemble_edge_resident_blocks(int block, int min_blocks, int stages, int geo_early,
                                                     int* per_sm);
    // cell-pair kernel of a split ensemble (FP32 only): 128-thread blocks, compiled
    // (min_blocks, geo_early) shapes
    static cudaError_t ensemble_step_pair(const EnsArgs<T>& a, int min_blocks, int geo_early, unsigned grid,
                                          cudaStream_t st);
    static cudaError_t ensemble_pair_resident_blocks(int min_blocks, int geo_early, int* per_sm);
    static int ensemble_pair_variants(int (*out)[2], int max);
    static void ensemble_default(int* block, int* min_blocks, int* stages, int* geo_early);
    static int default_min_blocks(int block);
    static cudaError_t dt(const V4<T>* s, const V4<T>* geoB, long long n, T g, T h_dry,
                          unsigned long long* dt_write, cudaStream_t st);
    static cudaError_t pack(const T* h, const T* hu, const T* hv, const long long* perm, const T* z,
                            V4<T>* s, long long n, cudaStream_t st);
    static cudaError_t unpack(const V4<T>* s, const long long* perm, T* h, T* hu, T* hv, long long n,
                              cudaStream_t st);
    static cudaError_t riemann(long long n, const T* hL, const T* unL, const T* utL, const T* hR,
                               const T* unR, const T* utR, T g, T h_dry, T* G1, T* G2, T* G3, T* S,
                               int hll, cudaStream_t st);
};

}  // namespace swe
