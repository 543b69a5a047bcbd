// swe_f32.cuh -- the FP32 arithmetic of one cell update (Eq 12-37).
//
// Every product, sum and fused multiply-add is written out with a rounded
// operation that the compiler may not fuse or reorder (mul, add, sub, fma
// below), so that every FP32 kernel and launch shape that inlines these
// functions rounds each cell identically: the kernels differ in how they
// load and schedule cells, and their results agree bit for bit.  (Left to
// itself, the compiler fuses multiply-adds differently under different
// register limits.)  Square roots and reciprocals are the hardware
// approximations (the FP32 step is compiled with fast-math intrinsics).
// The functions are written on a lane type V (float) with its mask type, and
// decisions in the Riemann solver are selects.
//
// Readings of the garbled equations are those of riemann_hllc and the oracle.
#pragma once

#include <cuda_runtime.h>

namespace swe {
namespace f32 {

// ---- lanes and masks -----------------------------------------------------------------
__device__ __forceinline__ bool any(bool m) { return m; }
__device__ __forceinline__ bool all(bool m) { return m; }
__device__ __forceinline__ bool mand(bool a, bool b) { return a && b; }
__device__ __forceinline__ bool mor(bool a, bool b) { return a || b; }
__device__ __forceinline__ bool mnot(bool a) { return !a; }

template <typename V> struct Mask;
template <> struct Mask<float> { using type = bool; };
template <typename V> using MaskT = typename Mask<V>::type;

template <typename V> __device__ __forceinline__ V splat(float c);
template <> __device__ __forceinline__ float splat<float>(float c) { return c; }

// ---- rounded operations (never fused, never reordered) ------------------------------
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float neg(float a) { return -a; }
// a - b = a + (-b) exactly (IEEE subtraction), signed zeros included
__device__ __forceinline__ float sub(float a, float b) { return __fadd_rn(a, -b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// hardware approximations
__device__ __forceinline__ float sqrt_(float a) { return sqrtf(a); }
__device__ __forceinline__ float rsqrt_(float a) { return rsqrtf(a); }
__device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float rcp_(float a) { return __fdividef(1.0f, a); }
// h^(-7/3) through the hardware base-2 exponential and logarithm
__device__ __forceinline__ float pow_m73(float h) { return exp2f(-7.0f / 3.0f * __log2f(h)); }
// comparisons (plain IEEE: false with a NaN operand) and selects
__device__ __forceinline__ bool gt(float a, float b) { return a > b; }
__device__ __forceinline__ bool ge(float a, float b) { return a >= b; }
__device__ __forceinline__ bool le(float a, float b) { return a <= b; }
__device__ __forceinline__ bool lt(float a, float b) { return a < b; }
__device__ __forceinline__ float sel(bool m, float a, float b) { return m ? a : b; }
// max(0, x), min and max on the min/max unit (one instruction each): a NaN
// operand gives the other operand (IEEE maxNum/minNum).  A NaN depth or
// momentum still reaches its own cell's new state, which the non-finite
// check reads, since the cell's update adds to its own h and q.
template <typename V>
__device__ __forceinline__ V max0(V x) { return fmaxf(x, splat<V>(0.0f)); }
template <typename V>
__device__ __forceinline__ V vmin(V a, V b) { return fminf(a, b); }
template <typename V>
__device__ __forceinline__ V vmax(V a, V b) { return fmaxf(a, b); }

// Wave speeds of two wet sides (Eq 19-25): the star depth by Eq 22 or Eq 23 as
// Eq 21's h0 decides, the shock factors of Eq 20, and S* as the quotient
// num / den of Eq 25.  Here m_L = h_L (un_L - S_L) > 0 > m_R = h_R (un_R - S_R),
// so den = m_R - m_L < 0 and S* >= 0 exactly when num <= 0: the flux needs
// only that sign (Eq 24), and the quotient is formed only on request.
template <typename V>
__device__ __forceinline__ void wet_speeds(V hL, V unL, V hR, V unR, V aL, V aR, V g, V g2, V& SL, V& SR, V& num,
                                           V& den) {
    const V one = splat<V>(1.0f);
    const V rhL = rcp_(hL), rhR = rcp_(hR);
    const V hsum = add(hL, hR), asum = add(aL, aR);
    // du = un_R - un_L; un_L - un_R is exactly -du (rounding is symmetric in sign)
    const V du = sub(unR, unL);
    const V h0 = mul(hsum, fma(mul(splat<V>(-0.25f), du), rcp_(asum), splat<V>(0.5f)));                // Eq 21
    const V b = max0(fma(splat<V>(-0.25f), du, mul(splat<V>(0.5f), asum)));                            // Eq 22
    const V hs_rare = div_(mul(b, b), g);
    const V rh0 = rcp_(h0);                                                                           // Eq 23
    const V gL = sqrt_(mul(g2, add(rh0, rhL))), gR = sqrt_(mul(g2, add(rh0, rhR)));
    const V hs_shock = div_(fma(hL, gL, fma(hR, gR, neg(du))), add(gL, gR));
    const V hs = sel(le(h0, vmin(hL, hR)), hs_rare, hs_shock);
    const V half_hs = mul(splat<V>(0.5f), hs);
    const V pL = sel(gt(hs, hL), mul(sqrt_(mul(half_hs, add(hs, hL))), rhL), one);                   // Eq 20
    const V pR = sel(gt(hs, hR), mul(sqrt_(mul(half_hs, add(hs, hR))), rhR), one);
    SL = fma(neg(aL), pL, unL);                                                                       // Eq 19
    SR = fma(aR, pR, unR);
    const V mL = mul(hL, sub(unL, SL)), mR = mul(hR, sub(unR, SR));
    num = fma(SL, mR, neg(mul(SR, mL)));                                                              // Eq 25
    den = sub(mR, mL);
}

// ---- Riemann flux in the edge-normal frame (Eq 14, 17-26) ------------------------------
// Readings: Eq 20 p_K = sqrt(h*(h*+h_K)/2)/h_K; Eq 21-22 use the normal
// velocity jump; the two-rarefaction base is clamped at 0; Eq 24 is upwinded
// (ut_L when S* >= 0); Eq 26 line 2 is the right-dry case; both dry gives no
// flux.  Lanes of one warp take different sides of the star-depth choice
// (Eq 22 or Eq 23, by the sign of h0 - min(h_L, h_R)) in most flows, so both
// estimates, both shock factors (Eq 20) and the star-region HLL flux (Eq 18)
// are formed and the decisions are selects; a value formed on a rejected
// side may be infinite or NaN and is never passed on.  Both sides wet is the
// one branch; the one-dry speed cases (Eq 26) are selects within the other.  Eq 23's g_K = sqrt(g (h0 + h_K)/(2 h0 h_K)) is formed as
// sqrt(g/2 (1/h0 + 1/h_K)), and 1/h_K is shared with Eq 20.  With hll_only the
// third component is the HLL flux of U_3 = h ut (Eq 18 applied to it).
template <typename V>
__device__ __forceinline__ void riemann(V hL, V unL, V utL, V hR, V unR, V utR, V g, V g2, V h_dry, V& G1, V& G2,
                                        V& G3, V* speeds, bool hll_only) {
    const V zero = splat<V>(0.0f);
    const bool wetL = gt(hL, h_dry), wetR = gt(hR, h_dry);
    const V aL = sqrt_(mul(g, hL)), aR = sqrt_(mul(g, hR));
    V SL, SR, Ss;
    bool upL;   // S* >= 0: the tangential velocity of the left side (Eq 24)
    if (wetL && wetR) {
        V num, den;
        wet_speeds(hL, unL, hR, unR, aL, aR, g, g2, SL, SR, num, den);
        upL = le(num, zero);
        if (speeds) Ss = div_(num, den);
    } else {
        if (!wetL && !wetR) {                                                 // both dry: no flux
            G1 = zero; G2 = zero; G3 = zero;
            if (speeds) { speeds[0] = zero; speeds[1] = zero; speeds[2] = zero; }
            return;
        }
        // one side dry (Eq 26)
        const V SLl = fma(splat<V>(-2.0f), aR, unR), SRl = add(unR, aR);     // left dry
        const V SLr = sub(unL, aL), SRr = fma(splat<V>(2.0f), aL, unL);      // right dry
        SL = sel(wetL, SLr, SLl);
        SR = sel(wetL, SRr, SRl);
        Ss = sel(wetL, SRr, SLl);
        upL = ge(Ss, zero);
    }
    const V qL = mul(hL, unL), qR = mul(hR, unR);
    const V PL = fma(qL, unL, mul(mul(g2, hL), hL));
    const V PR = fma(qR, unR, mul(mul(g2, hR), hR));
    const V r = rcp_(sub(SR, SL)), ss = mul(SR, SL);                                                  // Eq 18
    const bool supL = ge(SL, zero), supR = le(SR, zero);                                              // Eq 17
    const V G1s = mul(fma(SR, qL, fma(neg(SL), qR, mul(ss, sub(hR, hL)))), r);
    const V G2s = mul(fma(SR, PL, fma(neg(SL), PR, mul(ss, sub(qR, qL)))), r);
    G1 = sel(supL, qL, sel(supR, qR, G1s));
    G2 = sel(supL, PL, sel(supR, PR, G2s));
    if (hll_only) {
        const V qtL = mul(qL, utL), qtR = mul(qR, utR);
        const V G3s = mul(fma(SR, qtL, fma(neg(SL), qtR, mul(ss, sub(mul(hR, utR), mul(hL, utL))))), r);
        G3 = sel(supL, qtL, sel(supR, qtR, G3s));
    } else {
        G3 = mul(G1, sel(upL, utL, utR));                                                             // Eq 24
    }
    if (speeds) { speeds[0] = SL; speeds[1] = SR; speeds[2] = Ss; }
}

// ---- one interior edge (Eq 12, 28, 30) ---------------------------------------------------
// The flux leaving cell i (per unit length, x-y frame) and the edge's bed
// source factor (g/2)(h**_i^2 - h_i^2) (Eq 30 with 1/2); src_k, if given,
// receives the other cell's factor.  (n1, n2) is cell i's outward unit
// normal; flip says cell i is the right state of the edge's canonical
// orientation (left = lower caller index).  Both states are rotated into
// cell i's frame; for the right cell the canonical frame is that frame turned
// by pi, which negates the normal and tangential components, so both cells
// evaluate the same Riemann problem bit for bit, and the right cell's flux is
// the left cell's with only the mass flux's sign changed in the x-y frame.
template <typename V>
__device__ __forceinline__ void bed_src(V hs, V h, V g2, V& src) { src = mul(g2, fma(hs, hs, neg(mul(h, h)))); }

template <typename V>
__device__ __forceinline__ void velocity(V h, V hu, V hv, V h_dry, V& u, V& v) {
    const auto wet = gt(h, h_dry);
    const V r = rcp_(h);
    u = sel(wet, mul(hu, r), splat<V>(0.0f));
    v = sel(wet, mul(hv, r), splat<V>(0.0f));
}

template <typename V>
__device__ __forceinline__ void edge_interior(V hi, V ui, V vi, V zi, V hk, V huk, V hvk, V zk, V n1, V n2,
                                              MaskT<V> flip, V g, V g2, V h_dry, V& F0, V& F1, V& F2, V& src,
                                              bool hll_only, V* src_k = nullptr) {
    V uk, vk;
    velocity(hk, huk, hvk, h_dry, uk, vk);
    // hydrostatic reconstruction (Eq 28): z* = max(z_i, z_k)
    const V zs = vmax(zi, zk);
    const V hsi = max0(sub(add(hi, zi), zs));
    const V hsk = max0(sub(add(hk, zk), zs));
    // both sides in cell i's edge frame (Eq 12): normal n, tangent (-n2, n1)
    const V uni = fma(ui, n1, mul(vi, n2)), uti = fma(vi, n1, neg(mul(ui, n2)));
    const V unk = fma(uk, n1, mul(vk, n2)), utk = fma(vk, n1, neg(mul(uk, n2)));
    // the canonical orientation
    const V hL = sel(flip, hsk, hsi), hR = sel(flip, hsi, hsk);
    const V unL = sel(flip, neg(unk), uni), utL = sel(flip, neg(utk), uti);
    const V unR = sel(flip, neg(uni), unk), utR = sel(flip, neg(uti), utk);
    V G1, G2, G3;
    riemann(hL, unL, utL, hR, unR, utR, g, g2, h_dry, G1, G2, G3, (V*)nullptr, hll_only);
    // back to (x, y) (Eq 12 inverse), as the flux leaving cell i
    F0 = sel(flip, neg(G1), G1);
    F1 = fma(G2, n1, neg(mul(G3, n2)));
    F2 = fma(G2, n2, mul(G3, n1));
    bed_src(hsi, hi, g2, src);
    if (src_k) bed_src(hsk, hk, g2, *src_k);
}

// ---- one boundary edge (Section 3.1), one cell --------------------------------------------
__device__ __forceinline__ void edge_boundary(int kind, double value, float hi, float ui, float vi, float zi,
                                              float n1, float n2, float g, float g2, float h_dry, float& F0,
                                              float& F1, float& F2, bool hll_only) {
    const float un = fma(ui, n1, mul(vi, n2)), ut = fma(vi, n1, neg(mul(ui, n2)));
    const float p = mul(mul(g2, hi), hi);                                   // g h^2 / 2
    float G1, G2, G3;
    if (kind == 0) {                                                         // wall
        G1 = 0.0f; G2 = p; G3 = 0.0f;
    } else if (kind == 1) {                                                  // inflow, q per unit length
        const float q = (float)value;
        G1 = -q;
        G2 = hi > h_dry ? add(p, div_(mul(q, q), hi)) : p;
        G3 = 0.0f;
    } else {                                                                 // transmissive, fixed stage
        const float hg = kind == 3 ? max0(sub((float)value, zi)) : hi;
        riemann(hi, un, ut, hg, un, ut, g, g2, h_dry, G1, G2, G3, (float*)nullptr, hll_only);
    }
    F0 = G1;
    F1 = fma(G2, n1, neg(mul(G3, n2)));
    F2 = fma(G2, n2, mul(G3, n1));
}

// ---- semi-implicit friction (Eq 33-37) ---------------------------------------------------
// dU solving [I - dt/2 J_f] dU = dt (R + S_f), R = (Rh, Rx, Ry) per unit area,
// for cells with h > h_dry, g m^2 > 0 and |q| > 0 (else dU = dt R).  ri is
// 1/h (the cell's own velocity already formed it).  (1 + a|q|) I + a q q^T/|q|
// has eigenvalue 1 + 2a|q| along q and 1 + a|q| across it; one reciprocal
// gives 1/(|q| d2) and 1/d1.
template <typename V>
__device__ __forceinline__ void friction(V hi, V ri, V qx, V qy, V gm2, V Rh, V Rx, V Ry, V dt, V h_dry, V& dh,
                                         V& dqx, V& dqy) {
    dh = mul(dt, Rh);
    dqx = mul(dt, Rx);
    dqy = mul(dt, Ry);
    const V zero = splat<V>(0.0f);
    const V qq = fma(qx, qx, mul(qy, qy));
    const auto act = mand(mand(gt(hi, h_dry), gt(gm2, zero)), gt(qq, zero));
    if (!any(act)) return;
    const V qn = sqrt_(qq);
    const V cf = mul(gm2, pow_m73(hi));                                      // c = g m^2 h^(-7/3)
    const V dtcf = mul(dt, cf);
    const V al = mul(splat<V>(0.5f), dtcf);                                  // alpha = dt c / 2
    // rhs: dt (R_q + S_f) + dt/2 J_qh dh, S_f = -c|q|q, J_qh = (7/3) c |q| q / h
    const V k = mul(mul(dtcf, qn), fma(mul(splat<V>(7.0f / 6.0f), dh), ri, splat<V>(-1.0f)));
    const V bx = fma(k, qx, dqx), by = fma(k, qy, dqy);
    const V d1 = fma(al, qn, splat<V>(1.0f));
    const V d2 = fma(al, qn, d1);
    const V qd2 = mul(qn, d2);
    const V inv = rcp_(mul(qd2, d1));
    const V proj = mul(mul(fma(bx, qx, mul(by, qy)), al), mul(d1, inv));
    const V rd1 = mul(qd2, inv);
    dqx = sel(act, mul(fma(neg(proj), qx, bx), rd1), dqx);
    dqy = sel(act, mul(fma(neg(proj), qy, by), rd1), dqy);
}

// ---- the end of one cell update (Eq 37, the checks, Eq 15) --------------------------------
// From the summed edge terms (f = sum of L F, s = sum of the bed source
// factors times L n) to the new state, the clamps (a negative depth becomes
// a dry cell at rest; a dry cell's momentum is zero), and the next CFL
// candidate R h / (h sqrt(g h) + |q|) = R / (sqrt(g h) + |u|) (Eq 15; +inf
// when dry).  Returns the candidate; sets clamped / nonfinite per lane.
template <typename V>
__device__ __forceinline__ V finish(V hi, V ri, V qx, V qy, V f0, V f1, V f2, V sx, V sy, V ia, V rin, V gm2, V dt,
                                    V g, V h_dry, V& oh, V& ou, V& ov, MaskT<V>& clamped, MaskT<V>& nonfinite) {
    const V zero = splat<V>(0.0f);
    const V Rh = mul(neg(f0), ia);
    const V Rx = mul(sub(sx, f1), ia);
    const V Ry = mul(sub(sy, f2), ia);
    V dh, dqx, dqy;
    friction(hi, ri, qx, qy, gm2, Rh, Rx, Ry, dt, h_dry, dh, dqx, dqy);
    V h = add(hi, dh), u = add(qx, dqx), v = add(qy, dqy);
    clamped = lt(h, zero);
    const auto dry = le(h, h_dry);
    h = sel(clamped, zero, h);
    u = sel(dry, zero, u);
    v = sel(dry, zero, v);
    const V big = splat<V>(3.0e38f);
    // finite and below 3e38 in magnitude (NaN fails every comparison)
    const auto okh = lt(h, big);
    const auto oku = lt(fabsf(u), big);
    const auto okv = lt(fabsf(v), big);
    nonfinite = mnot(mand(okh, mand(oku, okv)));
    oh = h; ou = u; ov = v;
    const V qm = sqrt_(fma(u, u, mul(v, v)));
    const V cand = div_(mul(rin, h), fma(h, sqrt_(mul(g, h)), qm));
    return sel(gt(h, h_dry), cand, splat<V>(__int_as_float(0x7F800000)));
}

}  // namespace f32
}  // namespace swe
