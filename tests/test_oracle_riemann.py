"""Pins of the exact Euler Riemann solver used as the Sod reference (Sec. 3.1, Fig. 7)."""
import math
import os

import numpy as np
import pytest

from oracle import exact_riemann as ER

GOLD = os.path.join(os.path.dirname(__file__), "golden", "sod_star_state.txt")


def _gold():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    return [float(x) for x in rows[0]]


def test_sod_star_matches_textbook_table():
    ps, us, rl, rr = ER.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    for got, ref in zip((ps, us, rl, rr), _gold()):
        assert abs(got - ref) <= 6e-6, (got, ref)


@pytest.mark.parametrize("case", [
    (1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4),       # shock right, rarefaction left
    (1.0, -2.0, 0.4, 1.0, 2.0, 0.4, 1.4),        # two rarefactions
    (1.0, 0.0, 1000.0, 1.0, 0.0, 0.01, 1.4),     # strong shock
    (5.99924, 19.5975, 460.894, 5.99242, -6.19633, 46.095, 1.4),  # two shocks
    (1.0, 0.3, 2.0, 0.5, -0.1, 0.3, 5.0 / 3.0),
])
def test_star_state_satisfies_wave_relations(case):
    """Each side of the star region obeys Rankine-Hugoniot (shock) or isentropy+invariant."""
    rL, uL, pL, rR, uR, pR, g = case
    ps, us, rsL, rsR = ER.star_state(*case)
    for side, (r, u, p, rs, sgn) in enumerate([(rL, uL, pL, rsL, -1), (rR, uR, pR, rsR, +1)]):
        if ps > p:
            # shock speed from mass conservation, then momentum and energy fluxes must match
            S = (rs * us - r * u) / (rs - r)
            m1, m2 = r * (u - S), rs * (us - S)
            assert abs(m1 - m2) <= 1e-9 * max(1.0, abs(m1))
            assert abs((m1 * u + p) - (m2 * us + ps)) <= 1e-9 * max(1.0, abs(p), abs(ps))
            h1 = g / (g - 1) * p / r + 0.5 * (u - S) ** 2
            h2 = g / (g - 1) * ps / rs + 0.5 * (us - S) ** 2
            assert abs(h1 - h2) <= 1e-9 * max(1.0, abs(h1))
        else:
            # isentropic: p / rho^gamma constant; Riemann invariant u -/+ 2a/(g-1) constant
            assert abs(ps / rs ** g - p / r ** g) <= 1e-10 * p / r ** g
            a, as_ = math.sqrt(g * p / r), math.sqrt(g * ps / rs)
            J = u - sgn * 2 * a / (g - 1)
            Js = us - sgn * 2 * as_ / (g - 1)
            assert abs(J - Js) <= 1e-10 * max(1.0, abs(J))


def test_sample_recovers_states_far_away():
    r, u, p = ER.sample(np.array([-100.0, 100.0]), 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    assert np.allclose(r, [1.0, 0.125]) and np.allclose(p, [1.0, 0.1]) and np.allclose(u, 0.0)


def test_sample_is_continuous_inside_rarefaction():
    xs = np.linspace(-1.2, 0.0, 2001)
    r, u, p = ER.sample(xs, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    assert np.max(np.abs(np.diff(r))) < 2e-3 and np.max(np.abs(np.diff(p))) < 2e-3
