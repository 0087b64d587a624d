"""Host-side set-up of the paper's validation runs (paper_1303_2470_gb300/validation.py) on
CPU: the Taylor-Aris sweep's flow gives the Peclet numbers asked for, and at those numbers
every link probability of the slit flow stays non-negative (so the sweep needs no
negative-probability override)."""
import itertools

import numpy as np
import pytest


@pytest.fixture(scope="module")
def validation():
    from paper_1303_2470_gb300 import build as b
    b.build()
    from paper_1303_2470_gb300 import validation as v
    return v


@pytest.mark.parametrize("L,D_b", [(100, 0.01), (32, 0.02), (17, 0.05)])
def test_poiseuille_u_max_gives_the_requested_peclet_number(validation, L, D_b):
    from paper_1303_2470_gb300 import media
    for Pe in (1.0, 10.0, 30.0, 60.0, 120.0):
        u_max = validation.poiseuille_u_max(L, D_b, Pe)
        vbar = media.poiseuille_profile(L, u_max)[1:L + 1].mean()          # mean over the L fluid planes
        assert L * vbar / D_b == pytest.approx(Pe, rel=1e-12)


def test_sweep_link_probabilities_are_non_negative_up_to_pe_120(validation):
    from paper_1303_2470_gb300 import media
    L, D_b = 100, 0.01
    half_lambda = 6.0 * D_b                                                  # lambda = 12 D_b
    links = [c for c in itertools.product((-1, 0, 1), repeat=3) if 1 <= sum(map(abs, c)) <= 2]
    for Pe in (10.0, 30.0, 60.0, 120.0):
        prof = media.poiseuille_profile(L, validation.poiseuille_u_max(L, D_b, Pe)).astype(np.float32)
        u = prof.astype(np.float64)
        for c in links:
            cu = c[0] * u                                                    # flow along x
            w = 1 / 18 if sum(map(abs, c)) == 1 else 1 / 36
            p = w * (half_lambda + 3 * cu + 4.5 * cu ** 2 - 1.5 * u ** 2)
            assert p.min() > 0.0, (Pe, c)
    # and the margin closes beyond: at Pe = 150 the upstream face link at the centre turns negative
    u = validation.poiseuille_u_max(L, D_b, 150.0)
    assert half_lambda - 3 * u + 3 * u ** 2 < 0.0
