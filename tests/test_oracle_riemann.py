"""Pins for the oracle's Riemann solver (Eq 17-26) against the mathematics:
closed-form values, consistency, conservation symmetry and the exact
Riemann solution of the textbook dam break."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import analytic

G = 9.81
GOLD = os.path.join(os.path.dirname(__file__), "golden", "hstar_10_1.txt")


def _golden():
    vals = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


def test_hstar_two_shock_closed_form():
    gv = _golden()
    hs, h0 = oracle.hstar(gv["hL"], 0.0, gv["hR"], 0.0)
    assert h0 == pytest.approx(gv["h0"], abs=1e-14)
    assert hs == pytest.approx(gv["hstar"], abs=5e-12)


def test_exact_solver_matches_published_star_state():
    # the analytic module is itself pinned to textbook exact values
    gv = _golden()
    hs, us = analytic.star_state(10.0, 1.0)
    head, tail, shock = analytic.wave_speeds(10.0, 1.0)
    assert hs == pytest.approx(gv["exact_hstar"], abs=1e-10)
    assert us == pytest.approx(gv["exact_ustar"], abs=1e-10)
    assert shock == pytest.approx(gv["exact_shock"], abs=1e-9)
    assert head == pytest.approx(gv["exact_head"], abs=1e-9)
    assert tail == pytest.approx(gv["exact_tail"], abs=1e-9)


def test_wave_speed_estimates_against_exact_dam_break():
    # Eq 19-20: S_L is the exact rarefaction head (p_L = 1 since h* < h_L);
    # S_R with the shock factor p_R is within 0.5% of the exact shock speed.
    gv = _golden()
    _, S = oracle.hllc(10.0, 0.0, 0.0, 1.0, 0.0, 0.0)
    assert S[0] == pytest.approx(gv["exact_head"], abs=1e-9)
    assert abs(S[1] - gv["exact_shock"]) / gv["exact_shock"] < 5e-3


@pytest.mark.parametrize("h,u", [(1.0, 0.5), (3.0, 1.0), (0.2, 0.3)])
def test_two_rarefaction_estimate_is_exact(h, u):
    # symmetric diverging flow: the two-rarefaction estimate (Eq 22) is the
    # exact star depth, which the exact solver finds from f_L + f_R + du = 0
    hs, h0 = oracle.hstar(h, -u, h, u)
    assert h0 <= h
    a = math.sqrt(G * h)
    exact = (a - 0.5 * u) ** 2 / G      # 2 rarefactions: 2(a* - a) = -u ... a* = a - u/2
    # independent check by bisection on the exact-solver residual
    lo, hi = 0.0, h
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        r = 2 * (2 * (math.sqrt(G * mid) - a)) + 2 * u
        lo, hi = (mid, hi) if r < 0 else (lo, mid)
    assert exact == pytest.approx(lo, rel=1e-10)
    assert hs == pytest.approx(lo, rel=1e-10)


def test_vacuum_clamps_hstar_to_zero():
    hs, _ = oracle.hstar(1.0, -20.0, 1.0, 20.0)
    assert hs == 0.0


def _phys(h, un, ut):
    return np.array([h * un, h * un * un + 0.5 * G * h * h, h * un * ut])


def test_consistency_random_states():
    rng = np.random.default_rng(3)
    for _ in range(500):
        h = rng.uniform(1e-3, 20)
        un = rng.uniform(-30, 30)
        ut = rng.uniform(-5, 5)
        Gf, _ = oracle.hllc(h, un, ut, h, un, ut)
        ref = _phys(h, un, ut)
        assert np.allclose(Gf, ref, rtol=1e-12, atol=1e-12 * (1 + np.abs(ref).max()))


def test_conservation_symmetry_random_states():
    # Flux seen from the other cell (L<->R, n -> -n) must be -F (Eq 9):
    # G1' = -G1, G2' = G2, G3' = G3 in the respective frames.
    rng = np.random.default_rng(4)
    for _ in range(500):
        hL, hR = rng.uniform(1e-3, 10, 2)
        unL, unR, utL, utR = rng.uniform(-8, 8, 4)
        Gf, S = oracle.hllc(hL, unL, utL, hR, unR, utR)
        Gb, Sb = oracle.hllc(hR, -unR, -utR, hL, -unL, -utL)
        if abs(S[2]) < 1e-9:
            continue  # upwind tie at S* = 0
        assert Gb[0] == pytest.approx(-Gf[0], rel=1e-11, abs=1e-11)
        assert Gb[1] == pytest.approx(Gf[1], rel=1e-11, abs=1e-11)
        assert Gb[2] == pytest.approx(Gf[2], rel=1e-11, abs=1e-11)
        assert Sb[0] == pytest.approx(-S[1], rel=1e-12, abs=1e-12)


def test_dry_dry_is_zero():
    Gf, _ = oracle.hllc(0.0, 1.0, 2.0, 5e-7, -1.0, 0.0)
    assert np.all(Gf == 0.0)


def test_dry_bed_speeds():
    # Eq 26: left dry -> S_L = un_R - 2 a_R, S_R = un_R + a_R, S* = S_L
    hR, unR = 4.0, 0.7
    aR = math.sqrt(G * hR)
    _, S = oracle.hllc(0.0, 0.0, 0.0, hR, unR, 0.0)
    assert S == pytest.approx([unR - 2 * aR, unR + aR, unR - 2 * aR], rel=1e-14)
    hL, unL = 2.0, -0.4
    aL = math.sqrt(G * hL)
    _, S = oracle.hllc(hL, unL, 0.0, 0.0, 0.0, 0.0)
    assert S == pytest.approx([unL - aL, unL + 2 * aL, unL + 2 * aL], rel=1e-14)


def test_dry_bed_dam_site_flux_closed_form():
    # right side dry, water at rest on the left: S_L = -c0, S_R = 2 c0 (Eq 26),
    # so Eq 18 reduces by hand to G1 = 2 c0 h0 / 3 and G2 = g h0^2 / 3
    h0 = 10.0
    c0 = math.sqrt(G * h0)
    Gf, _ = oracle.hllc(h0, 0.0, 0.0, 0.0, 0.0, 0.0)
    assert Gf[0] == pytest.approx(2 * c0 * h0 / 3, rel=1e-14)
    assert Gf[1] == pytest.approx(G * h0 * h0 / 3, rel=1e-14)
    assert Gf[2] == 0.0


def test_hllc_shear_is_upwinded():
    # isolated shear wave carried by un > 0: the exact flux of the tangential
    # momentum at x/t = 0 is h un ut_L (Eq 24 read as upwind)
    Gf, S = oracle.hllc(1.0, 1.0, 2.0, 1.0, 1.0, -3.0)
    assert S[2] > 0
    assert Gf[0] == pytest.approx(1.0, rel=1e-14)
    assert Gf[2] == pytest.approx(2.0, rel=1e-14)
    Gf, S = oracle.hllc(1.0, -1.0, 2.0, 1.0, -1.0, -3.0)
    assert S[2] < 0
    assert Gf[2] == pytest.approx(-1.0 * -3.0, rel=1e-14)


def test_supersonic_branches():
    # S_L >= 0 gives the left physical flux, S_R <= 0 the right one (Eq 17)
    Gf, S = oracle.hllc(1.0, 12.0, 0.5, 2.0, 11.0, -0.5)
    assert S[0] >= 0
    assert np.allclose(Gf, _phys(1.0, 12.0, 0.5), rtol=1e-14)
    Gf, S = oracle.hllc(1.0, -12.0, 0.5, 2.0, -13.0, -0.5)
    assert S[1] <= 0
    assert np.allclose(Gf, _phys(2.0, -13.0, -0.5), rtol=1e-14)


def test_hll_third_component_closed_form():
    # a shear wave with equal depth and normal velocity u (subsonic): S_L = u - a,
    # S_R = u + a (p = 1), and Eq 18 applied to h ut gives by hand
    # h [ (u+a) u ut_L - (u-a) u ut_R + (u^2 - a^2)(ut_R - ut_L) ] / (2a)
    h, u, utl, utr = 2.0, 0.7, 1.5, -0.5
    a = math.sqrt(G * h)
    Gf = oracle.hll(h, u, utl, h, u, utr)
    expect = h * ((u + a) * u * utl - (u - a) * u * utr + (u * u - a * a) * (utr - utl)) / (2 * a)
    assert Gf[2] == pytest.approx(expect, rel=1e-13)
    # components 1-2 equal HLLC's; consistency and the supersonic branch
    Gc, _ = oracle.hllc(h, u, utl, h, u, utr)
    assert np.allclose(Gf[:2], Gc[:2], rtol=0, atol=0)
    assert np.allclose(oracle.hll(1.3, 0.4, 0.9, 1.3, 0.4, 0.9), _phys(1.3, 0.4, 0.9), rtol=1e-12)
    assert np.allclose(oracle.hll(1.0, 12.0, 0.5, 2.0, 11.0, -0.5), _phys(1.0, 12.0, 0.5), rtol=1e-14)


def test_hll_conservation_symmetry():
    rng = np.random.default_rng(8)
    for _ in range(300):
        hL, hR = rng.uniform(1e-3, 10, 2)
        unL, unR, utL, utR = rng.uniform(-8, 8, 4)
        Gf = oracle.hll(hL, unL, utL, hR, unR, utR)
        Gb = oracle.hll(hR, -unR, -utR, hL, -unL, -utL)
        assert Gb[0] == pytest.approx(-Gf[0], rel=1e-11, abs=1e-11)
        assert Gb[1] == pytest.approx(Gf[1], rel=1e-11, abs=1e-11)
        assert Gb[2] == pytest.approx(Gf[2], rel=1e-11, abs=1e-11)


# ---------------------------------------------------------------------------
# Eq 19-25 worked by hand on asymmetric wet states (tests/golden/sstar_asym.txt)
# ---------------------------------------------------------------------------

from tests.golden_cases import read_cases  # noqa: E402

SSTAR = read_cases("sstar_asym.txt")


@pytest.mark.parametrize("name", sorted(SSTAR))
def test_hllc_speeds_and_flux_match_hand_worked_asymmetric_states(name):
    c = SSTAR[name]
    hs, h0 = oracle.hstar(c["hL"], c["unL"], c["hR"], c["unR"])
    assert h0 == pytest.approx(c["h0"], rel=1e-13)
    assert hs == pytest.approx(c["hstar"], rel=1e-13)
    G, S = oracle.hllc(c["hL"], c["unL"], c["utL"], c["hR"], c["unR"], c["utR"])
    assert S[0] == pytest.approx(c["SL"], rel=1e-13)
    assert S[1] == pytest.approx(c["SR"], rel=1e-13)
    assert S[2] == pytest.approx(c["Sstar"], rel=1e-12)
    for k in range(3):
        assert G[k] == pytest.approx(c[f"G{k + 1}"], rel=1e-12)


def test_hand_worked_states_cover_both_contact_sides_and_both_estimates():
    # the golden cases exercise S* of either sign, a shock on either side and
    # both star-depth estimates (Eq 22 and Eq 23)
    signs = {math.copysign(1.0, c["Sstar"]) for c in SSTAR.values()}
    assert signs == {1.0, -1.0}
    assert any(c["pL"] > 1 for c in SSTAR.values()) and any(c["pR"] > 1 for c in SSTAR.values())
    two_rare = [c for c in SSTAR.values() if c["h0"] <= min(c["hL"], c["hR"])]
    assert two_rare and len(two_rare) < len(SSTAR)
    for c in SSTAR.values():
        assert c["hL"] != c["hR"] and c["unL"] != c["unR"]
