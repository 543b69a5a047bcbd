"""Reference gradient of the gauge-misfit loss (test infrastructure).

TEST INFRASTRUCTURE ONLY.  A second, vectorised statement of the oracle's
step (Sections 2-3, Eq 12-37, the same readings as ``swe_oracle.c``) in plain
PyTorch CPU FP64 ops, differentiated by autograd.  It is built on the C
oracle's own geometry (areas, lengths, normals, neighbours, boundary groups),
so it shares nothing with the CUDA library.  Its forward values are pinned to
the C oracle, its gradient to central differences of the C oracle and to
forward-mode (jvp) directional derivatives.

The loss is L = sum_g (h_g^N - target_g)^2 over gauge cells after N steps
with the time-step sequence frozen at given values (the gradient of the
discrete map with dt held fixed).  Unsafe operations (square roots at 0,
divisions by dry depths) are evaluated on sanitised inputs so that
branches not taken contribute exact zeros to the gradient.
"""
from __future__ import annotations

import numpy as np
import torch
from torch.utils.checkpoint import checkpoint

import oracle

BC_WALL, BC_INFLOW, BC_TRANSMISSIVE, BC_STAGE = 0, 1, 2, 3


def _safe(mask, x, fill=1.0):
    return torch.where(mask, x, torch.full_like(x, fill))


def hllc(hL, unL, utL, hR, unR, utR, g, h_dry):
    """Vectorised HLLC flux (Eq 17-26) in the edge-normal frame."""
    wetL, wetR = hL > h_dry, hR > h_dry
    any_wet = wetL | wetR
    both = wetL & wetR
    aL = torch.sqrt(g * _safe(hL > 0, hL))
    aL = torch.where(hL > 0, aL, torch.zeros_like(aL))
    aR = torch.sqrt(g * _safe(hR > 0, hR))
    aR = torch.where(hR > 0, aR, torch.zeros_like(aR))
    # both wet: adaptive h* (Eq 21-23), p_k (Eq 20), speeds (Eq 19), S* (Eq 25)
    hsum = hL + hR
    h0 = 0.5 * hsum - 0.25 * (unR - unL) * hsum / _safe(both, aL + aR)
    rare = h0 <= torch.minimum(hL, hR)
    base = torch.clamp(0.5 * (aL + aR) + 0.25 * (unL - unR), min=0.0)
    hs_rare = base * base / g
    shock = both & ~rare
    h0s = _safe(shock, h0)
    hLs, hRs = _safe(shock, hL), _safe(shock, hR)
    gL = torch.sqrt(g * (h0s + hLs) / (2.0 * h0s * hLs))
    gR = torch.sqrt(g * (h0s + hRs) / (2.0 * h0s * hRs))
    hs_shock = (hLs * gL + hRs * gR + unL - unR) / (gL + gR)
    hs = torch.where(rare, hs_rare, hs_shock)
    upL = both & (hs > hL)
    upR = both & (hs > hR)
    hsL = _safe(upL, hs)
    pL = torch.where(upL, torch.sqrt(0.5 * hsL * (hsL + _safe(upL, hL))) / _safe(upL, hL), torch.ones_like(hs))
    hsR = _safe(upR, hs)
    pR = torch.where(upR, torch.sqrt(0.5 * hsR * (hsR + _safe(upR, hR))) / _safe(upR, hR), torch.ones_like(hs))
    SL_w = unL - aL * pL
    SR_w = unR + aR * pR
    mL = hL * (unL - SL_w)
    mR = hR * (unR - SR_w)
    Ss_w = (SL_w * mR - SR_w * mL) / _safe(both, mR - mL)
    # dry-bed speeds (Eq 26)
    SL = torch.where(both, SL_w, torch.where(~wetL, unR - 2.0 * aR, unL - aL))
    SR = torch.where(both, SR_w, torch.where(~wetL, unR + aR, unL + 2.0 * aL))
    Ss = torch.where(both, Ss_w, torch.where(~wetL, SL, SR))
    # HLL (Eq 17-18)
    qL, qR = hL * unL, hR * unR
    PL = qL * unL + 0.5 * g * hL * hL
    PR = qR * unR + 0.5 * g * hR * hR
    star = (SL < 0) & (SR > 0) & any_wet
    r = 1.0 / _safe(star, SR - SL)
    G1s = (SR * qL - SL * qR + SR * SL * (hR - hL)) * r
    G2s = (SR * PL - SL * PR + SR * SL * (qR - qL)) * r
    G1 = torch.where(SL >= 0, qL, torch.where(SR <= 0, qR, G1s))
    G2 = torch.where(SL >= 0, PL, torch.where(SR <= 0, PR, G2s))
    G3 = G1 * torch.where(Ss >= 0, utL, utR)                          # Eq 24
    zero = torch.zeros_like(G1)
    return (torch.where(any_wet, G1, zero), torch.where(any_wet, G2, zero), torch.where(any_wet, G3, zero))


class TorchStep:
    """One explicit Euler step (Eq 37) on the C oracle's mesh, in torch ops."""

    def __init__(self, M: "oracle.Mesh"):
        geo = M.geometry()
        kind, value, glen = M.groups()
        n = M.n_cells
        self.n = n
        self.g, self.h_dry = M.g, M.h_dry
        self.area = torch.tensor(geo["area"])
        self.L = torch.tensor(geo["len"])
        self.n1 = torch.tensor(geo["nx"])
        self.n2 = torch.tensor(geo["ny"])
        nbr = torch.tensor(geo["nbr"])
        self.interior = nbr >= 0
        own = torch.arange(n).unsqueeze(1).expand(n, 3)
        self.k = torch.where(self.interior, nbr, own)
        grp = torch.where(self.interior, torch.zeros_like(nbr), -1 - nbr)
        kind_t = torch.tensor(kind.astype(np.int64))
        q = np.where(kind == BC_INFLOW, value / np.where(glen > 0, glen, 1.0), value)
        self.kind = torch.where(self.interior, torch.full_like(nbr, -1), kind_t[grp])
        self.bval = torch.tensor(q)[grp]

    def step(self, h, hu, hv, z, m, dt):
        g, h_dry = self.g, self.h_dry
        wet = h > h_dry
        hs_ = _safe(wet, h)
        u = torch.where(wet, hu / hs_, torch.zeros_like(h))
        v = torch.where(wet, hv / hs_, torch.zeros_like(h))
        hi, zi, ui, vi = h[:, None], z[:, None], u[:, None], v[:, None]
        hk, zk, uk, vk = h[self.k], z[self.k], u[self.k], v[self.k]
        n1, n2 = self.n1, self.n2
        # interior edges: hydrostatic reconstruction (Eq 28), rotation (Eq 12)
        zs = torch.maximum(zi.expand_as(zk), zk)
        hLs = torch.clamp(hi + zi - zs, min=0.0)
        hRs = torch.clamp(hk + zk - zs, min=0.0)
        unL, utL = ui * n1 + vi * n2, -ui * n2 + vi * n1
        unR, utR = uk * n1 + vk * n2, -uk * n2 + vk * n1
        G1i, G2i, G3i = hllc(hLs, unL, utL, hRs, unR, utR, g, h_dry)
        src = 0.5 * g * (hLs * hLs - hi * hi)                          # Eq 30 with 1/2
        # boundary edges (Section 3.1)
        hb = hi.expand_as(zk)
        unB, utB = unL, utL
        ghost = torch.where(self.kind == BC_STAGE, torch.clamp(self.bval - zi, min=0.0), hb)
        G1r, G2r, G3r = hllc(hb, unB, utB, ghost, unB, utB, g, h_dry)
        qb = self.bval
        hbs = _safe(hb > h_dry, hb)
        G2in = 0.5 * g * hb * hb + torch.where(hb > h_dry, qb * qb / hbs, torch.zeros_like(hb))
        zero = torch.zeros_like(hb)
        G1b = torch.where(self.kind == BC_WALL, zero, torch.where(self.kind == BC_INFLOW, -qb, G1r))
        G2b = torch.where(self.kind == BC_WALL, 0.5 * g * hb * hb, torch.where(self.kind == BC_INFLOW, G2in, G2r))
        G3b = torch.where((self.kind == BC_WALL) | (self.kind == BC_INFLOW), zero, G3r)
        I = self.interior
        G1 = torch.where(I, G1i, G1b)
        G2 = torch.where(I, G2i, G2b)
        G3 = torch.where(I, G3i, G3b)
        src = torch.where(I, src, zero)
        F0 = G1
        F1 = G2 * n1 - G3 * n2
        F2 = G2 * n2 + G3 * n1
        L = self.L
        A = self.area
        Rh = -(L * F0).sum(1) / A
        Rx = (-(L * F1).sum(1) + (L * src * n1).sum(1)) / A
        Ry = (-(L * F2).sum(1) + (L * src * n2).sum(1)) / A
        # semi-implicit friction (Eq 33-37), Cramer's rule on the 2x2 block
        dh = dt * Rh
        fr = wet & (m > 0)
        hf = _safe(fr, h)
        c = g * m * m * hf ** (-7.0 / 3.0)
        qq = hu * hu + hv * hv
        pos = fr & (qq > 0)
        qn = torch.where(pos, torch.sqrt(_safe(pos, qq)), torch.zeros_like(qq))
        qns = _safe(pos, qn)
        Sx, Sy = -c * qn * hu, -c * qn * hv
        Jxh = (7.0 / 3.0) * c * qn * hu / hf
        Jyh = (7.0 / 3.0) * c * qn * hv / hf
        Jxx = torch.where(pos, -c * (qn + hu * hu / qns), torch.zeros_like(qq))
        Jxy = torch.where(pos, -c * (hu * hv / qns), torch.zeros_like(qq))
        Jyy = torch.where(pos, -c * (qn + hv * hv / qns), torch.zeros_like(qq))
        A11, A12 = 1.0 - 0.5 * dt * Jxx, -0.5 * dt * Jxy
        A21, A22 = -0.5 * dt * Jxy, 1.0 - 0.5 * dt * Jyy
        b1 = dt * (Rx + Sx) + 0.5 * dt * Jxh * dh
        b2 = dt * (Ry + Sy) + 0.5 * dt * Jyh * dh
        det = A11 * A22 - A12 * A21
        dqx = torch.where(fr, (b1 * A22 - A12 * b2) / det, dt * Rx)
        dqy = torch.where(fr, (A11 * b2 - b1 * A21) / det, dt * Ry)
        h1 = h + dh
        hu1 = hu + dqx
        hv1 = hv + dqy
        neg = h1 < 0
        dry1 = h1 <= h_dry
        zf = torch.zeros_like(h1)
        h1 = torch.where(neg, zf, h1)
        hu1 = torch.where(neg | dry1, zf, hu1)
        hv1 = torch.where(neg | dry1, zf, hv1)
        return h1, hu1, hv1


def run(step: TorchStep, h, hu, hv, z, m, dts, segment=20):
    """Steps with the given dt sequence; recomputes segments in the backward."""
    def seg(h_, hu_, hv_, z_, m_, d):
        for dt in d:
            h_, hu_, hv_ = step.step(h_, hu_, hv_, z_, m_, float(dt))
        return h_, hu_, hv_
    for s in range(0, len(dts), segment):
        d = list(dts[s:s + segment])
        if torch.is_grad_enabled() and (z.requires_grad or m.requires_grad or h.requires_grad):
            h, hu, hv = checkpoint(seg, h, hu, hv, z, m, d, use_reentrant=False)
        else:
            h, hu, hv = seg(h, hu, hv, z, m, d)
    return h, hu, hv


def loss_and_gradient(M: "oracle.Mesh", h0, hu0, hv0, dts, gauges, target, segment=20):
    """L = sum_g (h_g^N - target_g)^2 and its gradient w.r.t. (manning, bathy)."""
    step = TorchStep(M)
    z = torch.tensor(M.z, requires_grad=True)
    m = torch.tensor(M.m, requires_grad=True)
    h, hu, hv = (torch.tensor(np.asarray(a, np.float64)) for a in (h0, hu0, hv0))
    hN, _, _ = run(step, h, hu, hv, z, m, dts, segment)
    gi = torch.tensor(np.asarray(gauges, np.int64))
    L = ((hN[gi] - torch.tensor(np.asarray(target, np.float64))) ** 2).sum()
    gz, gm = torch.autograd.grad(L, [z, m])
    return float(L.detach()), gm.numpy(), gz.numpy()


def loss_and_gradient_series(M: "oracle.Mesh", h0, hu0, hv0, dts, gauges, targets, obs_every, segment=None):
    """Time-series misfit sum_o sum_g (h_g^{o k} - targets[o-1, g])^2 with
    observations every k = obs_every steps, and its gradient w.r.t.
    (manning, bathy)."""
    step = TorchStep(M)
    z = torch.tensor(M.z, requires_grad=True)
    m = torch.tensor(M.m, requires_grad=True)
    h, hu, hv = (torch.tensor(np.asarray(a, np.float64)) for a in (h0, hu0, hv0))
    gi = torch.tensor(np.asarray(gauges, np.int64))
    tg = torch.tensor(np.asarray(targets, np.float64))
    L = torch.zeros((), dtype=torch.float64)
    for o in range(len(dts) // obs_every):
        d = dts[o * obs_every:(o + 1) * obs_every]
        h, hu, hv = run(step, h, hu, hv, z, m, d, segment or obs_every)
        L = L + ((h[gi] - tg[o]) ** 2).sum()
    gz, gm = torch.autograd.grad(L, [z, m])
    return float(L.detach()), gm.numpy(), gz.numpy()


def loss_only(M: "oracle.Mesh", h0, hu0, hv0, dts, gauges, target, z=None, m=None):
    step = TorchStep(M)
    zz = torch.tensor(M.z if z is None else z)
    mm = torch.tensor(M.m if m is None else m)
    with torch.no_grad():
        h, hu, hv = (torch.tensor(np.asarray(a, np.float64)) for a in (h0, hu0, hv0))
        hN, _, _ = run(step, h, hu, hv, zz, mm, dts)
    return float(((hN[torch.tensor(np.asarray(gauges, np.int64))] - torch.tensor(target)) ** 2).sum())
