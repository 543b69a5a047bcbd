"""Exact solutions of the 1D dam-break Riemann problem (test infrastructure).

The paper validates its solver on a one-dimensional dam break (Section 6.3)
and calls the result classic, pointing to Toro (2001).  These are the
textbook exact solutions used as pins for the oracle:

* wet bed (Stoker): left rarefaction, right shock; the star depth solves
  f_L(h*) + f_R(h*) + (u_R - u_L) = 0 with
  f_K(h) = 2 (sqrt(g h) - sqrt(g h_K))                    for h <= h_K,
  f_K(h) = (h - h_K) sqrt(g (h + h_K) / (2 h h_K))         for h >  h_K;
* dry bed (Ritter): h = (2 c0 - x/t)^2 / (9 g) on -c0 <= x/t <= 2 c0.

Only ``tests/`` and the bench's CPU leg use this module.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(h, hk, g):
    if h <= hk:
        return 2.0 * (math.sqrt(g * h) - math.sqrt(g * hk))
    return (h - hk) * math.sqrt(0.5 * g * (h + hk) / (h * hk))


def star_state(hL, hR, g=9.81):
    """Star depth and velocity for a dam break with zero initial velocity."""
    if hR <= 0.0:
        return 0.0, 2.0 * math.sqrt(g * hL)
    lo, hi = hR, hL
    for _ in range(200):  # bisection: f is monotone increasing in h
        mid = 0.5 * (lo + hi)
        if _fk(mid, hL, g) + _fk(mid, hR, g) > 0.0:
            hi = mid
        else:
            lo = mid
    hs = 0.5 * (lo + hi)
    us = 0.5 * (_fk(hs, hR, g) - _fk(hs, hL, g))
    return hs, us


def dam_break(x, t, hL, hR, x0=0.0, g=9.81):
    """Depth and velocity at positions x and time t > 0 for the dam break
    with the discontinuity at x0 (left state hL, right state hR, u = 0)."""
    x = np.asarray(x, dtype=np.float64)
    xi = (x - x0) / t
    cL = math.sqrt(g * hL)
    h = np.empty_like(xi)
    u = np.empty_like(xi)
    if hR <= 0.0:
        # Ritter: rarefaction directly into the dry bed
        left = xi <= -cL
        fan = (xi > -cL) & (xi < 2.0 * cL)
        h[left] = hL
        u[left] = 0.0
        h[fan] = (2.0 * cL - xi[fan]) ** 2 / (9.0 * g)
        u[fan] = 2.0 * (cL + xi[fan]) / 3.0
        dry = xi >= 2.0 * cL
        h[dry] = 0.0
        u[dry] = 0.0
        return h, u
    hs, us = star_state(hL, hR, g)
    cs = math.sqrt(g * hs)
    shock = us * hs / (hs - hR)  # mass balance across the shock
    head, tail = -cL, us - cs
    left = xi <= head
    fan = (xi > head) & (xi < tail)
    star = (xi >= tail) & (xi < shock)
    right = xi >= shock
    h[left], u[left] = hL, 0.0
    h[fan] = (2.0 * cL - xi[fan]) ** 2 / (9.0 * g)
    u[fan] = 2.0 * (cL + xi[fan]) / 3.0
    h[star], u[star] = hs, us
    h[right], u[right] = hR, 0.0
    return h, u


def wave_speeds(hL, hR, g=9.81):
    """(rarefaction head, rarefaction tail, shock speed) for the wet-bed case."""
    hs, us = star_state(hL, hR, g)
    return -math.sqrt(g * hL), us - math.sqrt(g * hs), us * hs / (hs - hR)
