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
    long long n_edges;
    // phase 2 on transposes: the interior edges (canonical orientation), their
    // L n and 1/|L n|, and per edge the adjoints of its two cells' states
    const int2* __restrict__ ecells;
    const double* __restrict__ eln;
    const double* __restrict__ erl;
    V4<double>* __restrict__ ed;
    // debug checks: neighbour codes and edge indices are checked before use
    int debug;
    int n_groups;
    unsigned* status;
};

// a neighbour code of cell i checked before use when debug checks are on: an
// unusable one is flagged and taken as a wall (group 0)
__device__ __forceinline__ int adj_code(const AdjArgs& a, int c) {
    if (a.debug && !code_ok(c, a.n, a.n_groups)) {
        atomicOr(a.status, kStatusBadIndex);
        return -1;
    }
    return c;
}

// the forward's unit normal and length of an edge, from its 1/|L n|
__device__ __forceinline__ void unit_normal(double lx, double ly, double rl, double& n1, double& n2, double& len) {
    const double l2 = edge_l2(lx, ly);
    len = l2 * rl;
    n1 = lx * rl;
    n2 = ly * rl;
}

__device__ __forceinline__ void edge_ln(const V4<double>& gA, const V4<double>& gB, int j, double& lx, double& ly) {
    lx = j == 0 ? gA.x : (j == 1 ? gA.z : gB.x);
    ly = j == 0 ? gA.y : (j == 1 ? gA.w : gB.y);
}

// Reverse of the semi-implicit friction update (friction_update, Eq 33-37,
// the literal formulas) at (h, qx, qy, g m^2, Rh, Rx, Ry): for the adjoints
// (bdh, bdqx, bdqy) of (dh, dqx, dqy), the adjoints w[0..6] of the seven
// inputs, in the order of the dual-number seeds.
__device__ void friction_rev(double hi, double qx, double qy, double gm2, double Rh, double Rx, double Ry, double dt,
                             double h_dry, double bdh, double bdqx, double bdqy, double w[7]) {
    const double dh = dt * Rh, dqx0 = dt * Rx, dqy0 = dt * Ry;
    const double qq = qx * qx + qy * qy;
    const bool act = gt_pos(hi, h_dry) && gt_zero(gm2) && gt_zero(qq);
#pragma unroll
    for (int k = 0; k < 7; ++k) w[k] = 0.0;
    if (!act) {
        w[4] = bdh * dt; w[5] = bdqx * dt; w[6] = bdqy * dt;
        return;
    }
    // forward
    const double qn = sqrt(qq);
    const double p = 1.0 / (hi * hi * cbrt(hi));                // h^(-7/3)
    const double cf = gm2 * p, rh = 1.0 / hi;
    const double al = 0.5 * dt * cf;
    const double P = 7.0 / 6.0 * dh * rh - 1.0;
    const double k = dt * cf * qn * P;
    const double bx = dqx0 + k * qx, by = dqy0 + k * qy;
    const double d1 = 1.0 + al * qn, d2 = d1 + al * qn;
    const double rqd2 = 1.0 / (qn * d2), rd1 = 1.0 / d1;
    const double S = bx * qx + by * qy;
    const double proj = S * al * rqd2;
    // reverse: dq = (b - proj q) / d1
    const double b_rd1 = bdqx * (bx - proj * qx) + bdqy * (by - proj * qy);
    double b_bx = bdqx * rd1, b_by = bdqy * rd1;
    const double b_proj = -(bdqx * qx + bdqy * qy) * rd1;
    double b_qx = -bdqx * proj * rd1, b_qy = -bdqy * proj * rd1;
    // proj = S al / (|q| d2)
    const double b_S = b_proj * al * rqd2;
    double b_al = b_proj * S * rqd2;
    const double b_rqd2 = b_proj * S * al;
    b_bx += b_S * qx; b_qx += b_S * bx;
    b_by += b_S * qy; b_qy += b_S * by;
    double b_qn = -b_rqd2 * rqd2 * rqd2 * d2;
    const double b_d2 = -b_rqd2 * rqd2 * rqd2 * qn;
    double b_d1 = -b_rd1 * rd1 * rd1 + b_d2;
    b_al += b_d2 * qn + b_d1 * qn;
    b_qn += b_d2 * al + b_d1 * al;
    // b = dt R_q + k q
    const double b_k = b_bx * qx + b_by * qy;
    b_qx += b_bx * k; b_qy += b_by * k;
    // k = dt c |q| P, P = (7/6) dh / h - 1
    double b_cf = b_k * dt * qn * P + b_al * 0.5 * dt;
    b_qn += b_k * dt * cf * P;
    const double b_P = b_k * dt * cf * qn;
    const double b_dh = bdh + b_P * 7.0 / 6.0 * rh;
    const double b_rh = b_P * 7.0 / 6.0 * dh;
    // c = g m^2 h^(-7/3), 1/h, |q| = sqrt(qx^2 + qy^2)
    const double b_h = -b_rh * rh * rh - b_cf * gm2 * (7.0 / 3.0) * p * rh;
    const double b_gm2 = b_cf * p;
    const double b_qq = b_qn / (2.0 * qn);
    b_qx += 2.0 * b_qq * qx;
    b_qy += 2.0 * b_qq * qy;
    w[0] = b_h; w[1] = b_qx; w[2] = b_qy; w[3] = b_gm2;
    w[4] = b_dh * dt; w[5] = b_bx * dt; w[6] = b_by * dt;
}

// EDGES reads R_i's interior fluxes from the edge pass (the forward's own
// edge-pass arithmetic) instead of evaluating them; R_i is the same bit for bit.
// TRANSPOSE transposes the friction update by hand (friction_rev) instead of
// running it on seven-component duals.
template <bool EDGES, bool TRANSPOSE>
__global__ void __launch_bounds__(128) adj_phase1_kernel(const AdjArgs a) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const double g = a.g, h_dry = a.h_dry;
    const V4<double> own = a.U[i];
    const V4<double> gA = a.geoA[i], gB = a.geoB[i], gR = a.geoR[i];
    const int4 tp = a.topo[i];
    const int code[3] = {adj_code(a, tp.x), adj_code(a, tp.y), adj_code(a, tp.z)};
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
                    int e = j == 0 ? ei.x : (j == 1 ? ei.y : ei.z);
                    if (a.debug && !(e >= 0 && e < a.n_edges)) {
                        atomicOr(a.status, kStatusBadIndex);
                        e = 0;
                    }
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
    const V4<double> L = a.lam[i];
    double lh = L.x, lx_ = L.y, ly_ = L.z;
    double w[7];
    if constexpr (TRANSPOSE) {
        // the forward's clamps (h < 0 zeroes the cell, h <= h_dry zeroes momentum) on
        // the new depth, then the friction update's transpose
        const double hn = hi + a.dt * Rh;
        if (hn < 0.0) { lh = 0.0; lx_ = 0.0; ly_ = 0.0; }
        else if (hn <= h_dry) { lx_ = 0.0; ly_ = 0.0; }
        friction_rev(hi, own.y, own.z, a.gm2[i], Rh, Rx, Ry, a.dt, h_dry, lh, lx_, ly_, w);
    } else {
        // Phi on duals: seeds h, hu, hv, g m^2, Rh, Rx, Ry
        D7 dh, dqx, dqy;
        friction_update<D7>(D7::seed(hi, 0), D7::seed(own.y, 1), D7::seed(own.z, 2), D7::seed(a.gm2[i], 3),
                            D7::seed(Rh, 4), D7::seed(Rx, 5), D7::seed(Ry, 6), D7(a.dt), D7(h_dry), dh, dqx, dqy);
        // the forward's clamps: h < 0 zeroes the cell, h <= h_dry zeroes momentum
        const double hn = hi + dh.v;
        if (hn < 0.0) { lh = 0.0; lx_ = 0.0; ly_ = 0.0; }
        else if (hn <= h_dry) { lx_ = 0.0; ly_ = 0.0; }
#pragma unroll
        for (int k = 0; k < 7; ++k) w[k] = lh * dh.d[k] + lx_ * dqx.d[k] + ly_ * dqy.d[k];
    }
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
    const int code[3] = {adj_code(a, tp.x), adj_code(a, tp.y), adj_code(a, tp.z)};
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

// ---- hand-written transposes of the edge flux (the default reverse step) ----------
// The reverse of one interior edge's contribution to both of its cells:
// with E_L = (-len F0, -len F1 + src_L lx, -len F2 + src_L ly) the edge's term
// in the left cell's (-f0, sx - f1, sy - f2) and E_R the right cell's
// (its flux is -F, its L n is -(lx, ly)), the step's adjoint needs
// d(nu_L . E_L + nu_R . E_R) / d(h, hu, hv, z) of both cells.  One forward
// evaluation of the edge and one reverse sweep through it give both, where
// the dual-number kernels evaluate the edge from each side on four-component
// duals.  The forward is recomputed here with the literal formulas of
// Eq 12-30 (the ones the dual-number kernels differentiate) and every branch
// is taken as the forward takes it; the derivative of a max at a tie is that
// of the operand the forward returns.

// Reverse of riemann_hllc (Eq 17-26) at (hL, unL, utL, hR, unR, utR): adds
// the adjoints of the six inputs for the flux adjoints (bG1, bG2, bG3).
__device__ void riemann_rev(double hL, double unL, double utL, double hR, double unR, double utR, double g,
                            double h_dry, bool hll_only, double bG1, double bG2, double bG3, double& bhL,
                            double& bunL, double& butL, double& bhR, double& bunR, double& butR) {
    const bool wetL = gt_pos(hL, h_dry), wetR = gt_pos(hR, h_dry);
    if (!wetL && !wetR) return;   // no flux on either side
    // ---- forward values
    const double aL = sqrt(g * hL), aR = sqrt(g * hR);
    double SL, SR, Ss, h0 = 0.0, hs = 0.0, pL = 1.0, pR = 1.0, gL = 0.0, gR = 0.0, b = 0.0;
    const double hsum = hL + hR, asum = aL + aR, du = unR - unL;
    bool rare = false, shL = false, shR = false, base_pos = false;
    if (!wetL) {
        SL = unR - 2.0 * aR; SR = unR + aR; Ss = SL;
    } else if (!wetR) {
        SL = unL - aL; SR = unL + 2.0 * aL; Ss = SR;
    } else {
        h0 = 0.5 * hsum - 0.25 * du * hsum / asum;                              // Eq 21
        rare = le_pos(h0, min_nonneg(hL, hR));
        if (rare) {                                                            // Eq 22
            const double base = 0.5 * asum + 0.25 * (unL - unR);
            base_pos = !lt_zero(base);
            b = base_pos ? base : 0.0;
            hs = b * b / g;
        } else {                                                               // Eq 23
            gL = sqrt(g * (h0 + hL) / (2.0 * h0 * hL));
            gR = sqrt(g * (h0 + hR) / (2.0 * h0 * hR));
            hs = (hL * gL + hR * gR + unL - unR) / (gL + gR);
        }
        shL = gt_pos(hs, hL);                                                  // Eq 20
        shR = gt_pos(hs, hR);
        if (shL) pL = sqrt(0.5 * hs * (hs + hL)) / hL;
        if (shR) pR = sqrt(0.5 * hs * (hs + hR)) / hR;
        SL = unL - aL * pL;                                                    // Eq 19
        SR = unR + aR * pR;
        const double mL = hL * (unL - SL), mR = hR * (unR - SR);
        Ss = (SL * mR - SR * mL) / (mR - mL);                                  // Eq 25
    }
    const double qL = hL * unL, qR = hR * unR;
    const double PL = qL * unL + 0.5 * g * hL * hL, PR = qR * unR + 0.5 * g * hR * hR;
    const bool supL = ge_zero(SL), supR = !supL && le_zero(SR);              // Eq 17
    const double D = SR - SL;
    double G1;
    if (supL) G1 = qL;
    else if (supR) G1 = qR;
    else G1 = (SR * qL - SL * qR + SR * SL * (hR - hL)) / D;
    // ---- reverse
    double bSL = 0.0, bSR = 0.0, bqL = 0.0, bqR = 0.0, bPL = 0.0, bPR = 0.0;
    if (!hll_only) {                                                           // Eq 24
        const bool up = ge_zero(Ss);
        bG1 += bG3 * (up ? utL : utR);
        if (up) butL += bG3 * G1;
        else butR += bG3 * G1;
    } else if (supL) {
        bqL += bG3 * utL; butL += bG3 * qL;
    } else if (supR) {
        bqR += bG3 * utR; butR += bG3 * qR;
    } else {
        const double N3 = SR * qL * utL - SL * qR * utR + SR * SL * (hR * utR - hL * utL);
        const double bN3 = bG3 / D;
        const double dh = hR * utR - hL * utL;
        bSR += bN3 * (qL * utL + SL * dh) - bG3 * N3 / (D * D);
        bSL += bN3 * (-qR * utR + SR * dh) + bG3 * N3 / (D * D);
        bqL += bN3 * SR * utL;
        bqR -= bN3 * SL * utR;
        butL += bN3 * (SR * qL - SR * SL * hL);
        butR += bN3 * (-SL * qR + SR * SL * hR);
        bhR += bN3 * SR * SL * utR;
        bhL -= bN3 * SR * SL * utL;
    }
    if (supL) {                                                                // Eq 17-18
        bqL += bG1; bPL += bG2;
    } else if (supR) {
        bqR += bG1; bPR += bG2;
    } else {
        const double G2 = (SR * PL - SL * PR + SR * SL * (qR - qL)) / D;
        const double bN1 = bG1 / D, bN2 = bG2 / D, bD = -(bG1 * G1 + bG2 * G2) / D;
        bSR += bN1 * (qL + SL * (hR - hL)) + bN2 * (PL + SL * (qR - qL)) + bD;
        bSL += bN1 * (-qR + SR * (hR - hL)) + bN2 * (-PR + SR * (qR - qL)) - bD;
        bqL += bN1 * SR - bN2 * SR * SL;
        bqR += -bN1 * SL + bN2 * SR * SL;
        bPL += bN2 * SR;
        bPR -= bN2 * SL;
        bhR += bN1 * SR * SL;
        bhL -= bN1 * SR * SL;
    }
    // P_K = q_K un_K + g h_K^2 / 2, q_K = h_K un_K
    bqL += bPL * unL; bunL += bPL * qL; bhL += bPL * g * hL;
    bqR += bPR * unR; bunR += bPR * qR; bhR += bPR * g * hR;
    bhL += bqL * unL; bunL += bqL * hL;
    bhR += bqR * unR; bunR += bqR * hR;
    double baL = 0.0, baR = 0.0;
    if (!wetL) {                                                               // Eq 26
        bunR += bSL + bSR; baR += -2.0 * bSL + bSR;
    } else if (!wetR) {
        bunL += bSL + bSR; baL += -bSL + 2.0 * bSR;
    } else {
        bunL += bSL; baL -= bSL * pL;
        bunR += bSR; baR += bSR * pR;
        const double bpL = -bSL * aL, bpR = bSR * aR;
        double bhs = 0.0;
        if (shL) {   // p_L = r / h_L, r = sqrt(h* (h* + h_L) / 2)
            const double r = pL * hL;
            bhs += bpL * (hs + 0.5 * hL) / (2.0 * r * hL);
            bhL += bpL * (hs / (4.0 * r * hL) - pL / hL);
        }
        if (shR) {
            const double r = pR * hR;
            bhs += bpR * (hs + 0.5 * hR) / (2.0 * r * hR);
            bhR += bpR * (hs / (4.0 * r * hR) - pR / hR);
        }
        if (rare) {
            if (base_pos) {
                const double bb = bhs * 2.0 * b / g;
                baL += 0.5 * bb; baR += 0.5 * bb;
                bunL += 0.25 * bb; bunR -= 0.25 * bb;
            }
        } else {
            // h* = N / (g_L + g_R), N = h_L g_L + h_R g_R + un_L - un_R
            const double Dg = gL + gR;
            const double bN = bhs / Dg, bDg = -bhs * hs / Dg;
            bhL += bN * gL; bhR += bN * gR;
            bunL += bN; bunR -= bN;
            const double bgL = bN * hL + bDg, bgR = bN * hR + bDg;
            // g_K = sqrt(X_K), X_K = g (h0 + h_K) / (2 h0 h_K) = (g/2)(1/h_K + 1/h0)
            const double bXL = bgL / (2.0 * gL), bXR = bgR / (2.0 * gR);
            const double bh0 = -(bXL + bXR) * 0.5 * g / (h0 * h0);
            bhL -= bXL * 0.5 * g / (hL * hL);
            bhR -= bXR * 0.5 * g / (hR * hR);
            // h0 = hsum/2 - du hsum / (4 asum)
            const double bhsum = bh0 * (0.5 - 0.25 * du / asum);
            const double bdu = -bh0 * 0.25 * hsum / asum;
            const double basum = bh0 * 0.25 * du * hsum / (asum * asum);
            bhL += bhsum; bhR += bhsum;
            bunR += bdu; bunL -= bdu;
            baL += basum; baR += basum;
        }
    }
    if (aL > 0.0) bhL += baL * g / (2.0 * aL);                                 // a_K = sqrt(g h_K)
    if (aR > 0.0) bhR += baR * g / (2.0 * aR);
}

// Reverse of one interior edge in canonical orientation (left cell L, its
// outward unit normal (n1, n2)): for the adjoints (wF0, wF1, wF2) of the flux
// leaving L and (sL, sR) of the two cells' bed source factors, adds the
// adjoints of (h, hu, hv, z) of L to dL and of R to dR.
__device__ void edge_interior_rev(const V4<double>& L, const V4<double>& R, double n1, double n2, double g,
                                  double h_dry, bool hll_only, double wF0, double wF1, double wF2, double sL,
                                  double sR, V4<double>& dL, V4<double>& dR) {
    // forward: velocities (R9), hydrostatic reconstruction (Eq 28), rotation (Eq 12)
    const bool wL = gt_pos(L.x, h_dry), wR = gt_pos(R.x, h_dry);
    const double rL = wL ? 1.0 / L.x : 0.0, rR = wR ? 1.0 / R.x : 0.0;
    const double uL = L.y * rL, vL = L.z * rL, uR = R.y * rR, vR = R.z * rR;
    const bool zleft = L.w > R.w;   // z* = max(z_L, z_R); a tie takes z_R, as the forward
    const double zs = zleft ? L.w : R.w;
    const double xL = L.x + L.w - zs, xR = R.x + R.w - zs;
    const bool pL = !lt_zero(xL), pR = !lt_zero(xR);
    const double hL = pL ? xL : 0.0, hR = pR ? xR : 0.0;
    const double unL = uL * n1 + vL * n2, utL = vL * n1 - uL * n2;
    const double unR = uR * n1 + vR * n2, utR = vR * n1 - uR * n2;
    // reverse: back from (x, y) (Eq 12 inverse)
    const double bG1 = wF0, bG2 = wF1 * n1 + wF2 * n2, bG3 = -wF1 * n2 + wF2 * n1;
    double bhL = 0.0, bunL = 0.0, butL = 0.0, bhR = 0.0, bunR = 0.0, butR = 0.0;
    riemann_rev(hL, unL, utL, hR, unR, utR, g, h_dry, hll_only, bG1, bG2, bG3, bhL, bunL, butL, bhR, bunR, butR);
    // bed source factors (Eq 30 with 1/2): src_K = (g/2)(h**_K^2 - h_K^2)
    bhL += sL * g * hL;
    bhR += sR * g * hR;
    double bh0L = -sL * g * L.x, bh0R = -sR * g * R.x;
    // rotation
    const double buL = bunL * n1 - butL * n2, bvL = bunL * n2 + butL * n1;
    const double buR = bunR * n1 - butR * n2, bvR = bunR * n2 + butR * n1;
    double bqxL = 0.0, bqyL = 0.0, bqxR = 0.0, bqyR = 0.0;
    if (wL) { bqxL = buL * rL; bqyL = bvL * rL; bh0L -= (buL * uL + bvL * vL) * rL; }
    if (wR) { bqxR = buR * rR; bqyR = bvR * rR; bh0R -= (buR * uR + bvR * vR) * rR; }
    // reconstruction
    double bzL = 0.0, bzR = 0.0, bzs = 0.0;
    if (pL) { bh0L += bhL; bzL += bhL; bzs -= bhL; }
    if (pR) { bh0R += bhR; bzR += bhR; bzs -= bhR; }
    if (zleft) bzL += bzs;
    else bzR += bzs;
    dL.x += bh0L; dL.y += bqxL; dL.z += bqyL; dL.w += bzL;
    dR.x += bh0R; dR.y += bqxR; dR.z += bqyR; dR.w += bzR;
}

// Phase 2, edges: each interior edge once, the adjoints of both cells' states
// through it, into ed[2 e] (left cell) and ed[2 e + 1] (right cell).
__global__ void __launch_bounds__(128) adj_edge_kernel(const AdjArgs a) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < a.n_edges; e += stride) {
        int2 lr = a.ecells[e];
        V4<double> dl, dr;
        dl.x = dl.y = dl.z = dl.w = 0.0;
        dr.x = dr.y = dr.z = dr.w = 0.0;
        if (a.debug && !(lr.x >= 0 && lr.x < a.n && lr.y >= 0 && lr.y < a.n)) {
            atomicOr(a.status, kStatusBadIndex);
            a.ed[2 * e] = dl;
            a.ed[2 * e + 1] = dr;
            continue;
        }
        const V4<double> L = a.U[lr.x], R = a.U[lr.y];
        const double lx = a.eln[2 * e], ly = a.eln[2 * e + 1];
        double n1, n2, len;
        unit_normal(lx, ly, a.erl[e], n1, n2, len);
        const V4<double> nl = a.nu[lr.x], nr = a.nu[lr.y];
        const double sL = nl.y * lx + nl.z * ly, sR = -(nr.y * lx + nr.z * ly);
        edge_interior_rev(L, R, n1, n2, a.g, a.h_dry, a.hll != 0, len * (nr.x - nl.x), len * (nr.y - nl.y),
                          len * (nr.z - nl.z), sL, sR, dl, dr);
        a.ed[2 * e] = dl;
        a.ed[2 * e + 1] = dr;
    }
}

// Phase 2, cells: lambda^n_j = own term + the contributions of j's interior
// edges (in local edge order) + its boundary edges' (on duals, own state
// only); dL/dz_j likewise.
__global__ void __launch_bounds__(128) adj_cell_kernel(const AdjArgs a) {
    const long long jc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (jc >= a.n) return;
    const int4 tp = a.topo[jc];
    const int code[3] = {adj_code(a, tp.x), adj_code(a, tp.y), adj_code(a, tp.z)};
    const int4 ei = a.eidx[jc];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    bool any_boundary = false;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int c = code[j];
        if (c >= 0) {
            int e = j == 0 ? ei.x : (j == 1 ? ei.y : ei.z);
            if (a.debug && !(e >= 0 && e < a.n_edges)) {
                atomicOr(a.status, kStatusBadIndex);
                continue;
            }
            const V4<double> d = a.ed[2 * (long long)e + ((c & kFlipBit) ? 1 : 0)];
            acc[0] += d.x; acc[1] += d.y; acc[2] += d.z; acc[3] += d.w;
        } else {
            any_boundary = true;
        }
    }
    if (any_boundary) {
        const double g = a.g, h_dry = a.h_dry;
        const V4<double> own = a.U[jc];
        const V4<double> gA = a.geoA[jc], gB = a.geoB[jc], gR = a.geoR[jc];
        const V4<double> nuj = a.nu[jc];
        const D4 H = D4::seed(own.x, 0), QX = D4::seed(own.y, 1), QY = D4::seed(own.z, 2), Z = D4::seed(own.w, 3);
        D4 U, V;
        cell_velocity<D4>(H, QX, QY, D4(h_dry), U, V);
        for (int j = 0; j < 3; ++j) {
            const int c = code[j];
            if (c >= 0) continue;
            double lx, ly, n1, n2, len;
            edge_ln(gA, gB, j, lx, ly);
            unit_normal(lx, ly, j == 0 ? gR.x : (j == 1 ? gR.y : gR.z), n1, n2, len);
            const int grp = -1 - c;
            D4 F0, F1, F2;
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
    DevBuf ckpt, seg, dtlog, small, lam, aw, nu, gmv, gzv, dg_idx, dtarget, dloss, ed;
    const bool transposes = m->adjoint_method == SWE_ADJOINT_TRANSPOSE;
    if (transposes) {   // the interior edge list of the edge-by-edge reverse step
        rc = build_edges(m);
        if (rc) return rc;
    }
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
    if (transposes) alloc(ed, (size_t)std::max<int64_t>(m->n_edges, 1) * 2 * sizeof(V4<double>));
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
    // With the edge pass, the recomputation of a segment keeps each step's edge
    // fluxes (64 B per interior edge and step), so phase 1 reads the fluxes of
    // U^n that the recomputed step n -> n+1 formed instead of running the edge
    // pass again; without room for them, phase 1 runs it.
    const bool edges = m->plain.edges && m->eflux;
    DevBuf segflux, segsrc;
    const size_t Eb = (size_t)std::max<int64_t>(m->n_edges, 1);
    bool keep = edges && transposes;
    if (keep) {
        keep = cudaMalloc(&segflux.p, (size_t)K * Eb * sizeof(V4<double>)) == cudaSuccess &&
               cudaMalloc(&segsrc.p, (size_t)K * Eb * sizeof(double)) == cudaSuccess;
        if (!keep) (void)cudaGetLastError();   // clear the failed allocation's error
    }
    V4<double>* const sflux = (V4<double>*)segflux.p;
    double* const ssrc = (double*)segsrc.p;
    // forward run: checkpoints every K steps, step sizes logged, loss summed
    // over the observations.  The last segment's states (and, with the edge
    // pass, the fluxes its steps form) are kept as the reverse sweep's segment
    // buffer: recomputing them would give the same bits (the same kernels and
    // step sizes), so the reverse sweep starts without a recomputation.
    const int64_t last0 = (nseg - 1) * K;   // first step of the last segment
    char* const segp = (char*)seg.p;
    for (int64_t s = 0; s < nsteps && e == cudaSuccess; ++s) {
        void* cur = m->state[m->nstep % 2];
        void* nxt = m->state[(m->nstep + 1) % 2];
        if (s % K == 0) e = cudaMemcpyAsync((char*)ckpt.p + (s / K) * sb, cur, sb, cudaMemcpyDeviceToDevice, st);
        const bool in_last = s >= last0;
        if (e == cudaSuccess && in_last)
            e = cudaMemcpyAsync(segp + (s - last0) * sb, cur, sb, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = launch_step_raw(m, cur, nxt, m->small, m->nstep, cfl, nullptr, (double*)dtlog.p + s, st, false,
                                keep && in_last ? (void*)(sflux + (s - last0) * Eb) : nullptr,
                                keep && in_last ? (void*)(ssrc + (s - last0) * Eb) : nullptr);
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
    if (fstat[kSlotStatus] & kStatusBadIndex) {
        set_error("swe_adjoint: an index or boundary group out of range in the forward run (debug checks)");
        return SWE_EMESH;
    }
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
    a.n_edges = m->n_edges;
    a.debug = m->cfg.debug_checks;
    a.n_groups = m->n_groups;
    a.status = (unsigned*)((unsigned long long*)small.p + kSlotStatus);
    // with the edge pass, phase 1 takes R's interior fluxes from one evaluation per edge
    a.eflux = edges ? (const V4<double>*)m->eflux : nullptr;
    a.esrc = edges ? (const double*)m->esrc : nullptr;
    a.eidx = m->eidx;
    a.ecells = m->ecells;
    a.eln = (const double*)m->eln;
    a.erl = (const double*)m->erl;
    a.ed = (V4<double>*)ed.p;
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
        ea.n = n;
        ea.debug = a.debug;
        ea.n_groups = a.n_groups;
        ea.status = a.status;
    }
    const unsigned egrid = (unsigned)std::min<int64_t>((std::max<int64_t>(m->n_edges, 1) + 127) / 128, 65535);
    const unsigned grid = (unsigned)((n + 127) / 128);
    // reverse sweep, segment by segment
    for (int64_t sgi = nseg - 1; sgi >= 0 && e == cudaSuccess; --sgi) {
        const int64_t n0 = sgi * K, n1 = std::min<int64_t>(n0 + K, nsteps);
        const bool from_forward = sgi == nseg - 1;   // the forward run kept this segment
        if (!from_forward)
            e = cudaMemcpyAsync(segp, (char*)ckpt.p + sgi * sb, sb, cudaMemcpyDeviceToDevice, st);
        for (int64_t k = 0; !from_forward && k + 1 < n1 - n0 && e == cudaSuccess; ++k)
            e = launch_step_raw(m, segp + k * sb, segp + (k + 1) * sb, (unsigned long long*)small.p, k, cfl,
                                (const double*)dtlog.p + n0 + k, nullptr, st, false,
                                keep ? (void*)(sflux + k * Eb) : nullptr, keep ? (void*)(ssrc + k * Eb) : nullptr);
        if (keep && !from_forward && e == cudaSuccess) {   // the segment's last state has no recomputed step
            const int64_t k = n1 - n0 - 1;
            ea.s_in = (const V4<double>*)(segp + k * sb);
            ea.eflux = sflux + k * Eb;
            ea.esrc = ssrc + k * Eb;
            e = Launch<double>::edge_flux(ea, st);
        }
        for (int64_t k = n1 - n0 - 1; k >= 0 && e == cudaSuccess; --k) {
            a.U = (const V4<double>*)(segp + k * sb);
            a.dt = dts[n0 + k];
            if (keep) {
                a.eflux = sflux + k * Eb;
                a.esrc = ssrc + k * Eb;
                adj_phase1_kernel<true, true><<<grid, 128, 0, st>>>(a);
            } else if (edges) {
                ea.s_in = a.U;
                e = Launch<double>::edge_flux(ea, st);
                if (e != cudaSuccess) break;
                if (transposes) adj_phase1_kernel<true, true><<<grid, 128, 0, st>>>(a);
                else adj_phase1_kernel<true, false><<<grid, 128, 0, st>>>(a);
            } else {
                if (transposes) adj_phase1_kernel<false, true><<<grid, 128, 0, st>>>(a);
                else adj_phase1_kernel<false, false><<<grid, 128, 0, st>>>(a);
            }
            if (transposes) {
                adj_edge_kernel<<<egrid, 128, 0, st>>>(a);
                adj_cell_kernel<<<grid, 128, 0, st>>>(a);
            } else {
                adj_phase2_kernel<<<grid, 128, 0, st>>>(a);
            }
            const int64_t nn = n0 + k;  // lambda now holds lambda^nn
            if (nn > 0 && nn % obs_every == 0)
                adj_inject_kernel<<<1, 32, 0, st>>>(a.U, gi, tg + (nn / obs_every - 1) * n_gauges, n_gauges, a.lam);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) return afail(e, "swe_adjoint: reverse sweep");
    if (m->cfg.debug_checks) {
        unsigned long long rs[kSmallWords];
        e = cudaMemcpyAsync(rs, small.p, sizeof rs, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return afail(e, "swe_adjoint: reverse sweep status");
        if (rs[kSlotStatus] & kStatusBadIndex) {
            set_error("swe_adjoint: an index or boundary group out of range in the reverse sweep (debug checks)");
            return SWE_EMESH;
        }
    }
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
    if (sm[kSlotStatus] & kStatusBadIndex) {
        set_error("swe_step_dt: an index or boundary group out of range (debug checks)");
        return SWE_EMESH;
    }
    if (sm[kSlotStatus] & kStatusNonFinite) { set_error("swe_step_dt: non-finite state"); return SWE_ENONFINITE; }
    return SWE_OK;
}

int swe_adjoint_method(swe_mesh* m, int method) {
    if (!m) { set_error("swe_adjoint_method: NULL mesh"); return SWE_EINVAL; }
    if (method != SWE_ADJOINT_TRANSPOSE && method != SWE_ADJOINT_DUAL) {
        set_error("swe_adjoint_method: unknown method");
        return SWE_EINVAL;
    }
    m->adjoint_method = method;
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
