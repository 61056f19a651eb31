"""Pins of the bond-basis gauge builder (App. A; a builder variant that changes q).

- The vertical split reproduces the bond weight: B T = W entry by entry.
- At exact chi nothing is truncated: Z~ = Z and q = pi for every state (enumeration).
- beta = 0: q is uniform.
- At a truncating chi q is a normalised distribution different from pi and from the
  spin-basis q; both are valid MH proposals, compared by their exact stationary
  acceptance (enumeration).
"""
import math

import numpy as np
import pytest

from oracle import exact, tnmc
from paper_2104_13264_gb300 import instances


def test_vertical_split_reproduces_the_bond_weight():
    for J in (1.0, -0.7, 0.0, 2.3):
        for beta in (0.3, 1.0):
            B, T = tnmc.vertical_split(J, beta)
            W = np.exp(beta * J * np.outer([-1.0, 1.0], [-1.0, 1.0]))
            np.testing.assert_allclose(B @ T, W, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("inst", [instances.random_small(4, 4, 0.9, 8, seed=2), instances.ea_pm(3, 5, 1.0, 8, seed=4),
                                  instances.random_small(4, 3, 0.7, 8, seed=5)])
def test_exact_chi_gives_pi(inst):
    env = tnmc.build_env_bond(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    S, logZ, pi, _ = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    assert env.logZ == pytest.approx(logZ, abs=1e-10)
    q = np.exp(tnmc.logq(env, S)[1])
    np.testing.assert_allclose(q, pi, rtol=1e-9, atol=1e-15)


def test_beta_zero_is_uniform():
    inst = instances.random_small(4, 5, 0.0, 2, seed=3)
    env = tnmc.build_env_bond(inst.Jh, inst.Jv, inst.h, 0.0, 2)
    _, lq, _, _ = tnmc.sample(env, 50, seed=1)
    np.testing.assert_allclose(lq, -20 * math.log(2), atol=1e-12)


def test_truncated_bond_gauge_is_a_different_valid_proposal():
    inst = instances.random_small(4, 4, 1.1, 2, seed=7, hscale=0.2)
    S, _, pi, _ = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    qb = np.exp(tnmc.logq(tnmc.build_env_bond(inst.Jh, inst.Jv, inst.h, inst.beta, 2), S)[1])
    qs = np.exp(tnmc.logq(tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 2), S)[1])
    assert qb.sum() == pytest.approx(1.0, abs=1e-12)
    assert exact.tv_distance(pi, qb) > 1e-4 and exact.tv_distance(qb, qs) > 1e-6
    ab, a_s = exact.independence_acceptance(pi, qb), exact.independence_acceptance(pi, qs)
    assert 0.0 < ab < 1.0 and 0.0 < a_s < 1.0
