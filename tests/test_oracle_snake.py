"""Pins of the snake site order (odd rows right to left; App. A leaves the labelling open).

- Exact chi: q = pi by enumeration in snake order too.
- Truncating chi: the same q as raster order wherever no weight is clamped.  Row r's
  conditionals are exact marginals of one distribution over the row, f env_r normalised
  (the row MPS is contracted without truncation), so the order inside a row cannot change
  its law; only clamped negative weights could.  Each order still draws different spins
  from the same random words.  Sampled log q equals forced log q, draws follow q (chi^2).
- A single row is the same in both orders (row 0 runs left to right).
"""
import math

import numpy as np
import pytest

from oracle import exact, tnmc
from paper_2104_13264_gb300 import instances


def _env(inst, chi, order):
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, chi)
    env.order = order
    return env


@pytest.mark.parametrize("inst", [instances.random_small(4, 4, 0.9, 8, seed=2), instances.ea_pm(3, 5, 1.0, 8, seed=4)])
def test_exact_chi_gives_pi_in_snake_order(inst):
    S, _, pi, _ = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    q = np.exp(tnmc.logq(_env(inst, inst.chi, "snake"), S)[1])
    np.testing.assert_allclose(q, pi, rtol=1e-9, atol=1e-15)


def test_truncated_snake_q_equals_raster_q_and_draws_differ():
    inst = instances.random_small(4, 5, 1.1, 2, seed=7, hscale=0.2)
    S, _, pi, _ = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    qs = np.exp(tnmc.logq(_env(inst, 2, "snake"), S)[1])
    qr = np.exp(tnmc.logq(_env(inst, 2, "raster"), S)[1])
    assert qs.sum() == pytest.approx(1.0, abs=1e-12)
    assert exact.tv_distance(qr, pi) > 1e-3                   # truncation is active
    np.testing.assert_allclose(qs, qr, rtol=1e-9, atol=1e-18)
    env = _env(inst, 2, "snake")
    sp, lq, E, _ = tnmc.sample(env, 200, seed=3)
    spr = tnmc.sample(_env(inst, 2, "raster"), 200, seed=3)[0]
    assert np.mean(np.all(sp.reshape(200, -1) == spr.reshape(200, -1), axis=1)) < 0.9
    _, lqf, Ef, _ = tnmc.logq(env, sp)
    np.testing.assert_allclose(lq, lqf, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(E, Ef, rtol=1e-13, atol=1e-13)


def test_snake_draw_frequencies_follow_q():
    inst = instances.random_small(3, 3, 0.8, 1, seed=5)
    env = _env(inst, 1, "snake")
    S, _, _, _ = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    q = np.exp(tnmc.logq(env, S)[1])
    n = 40000
    sp = tnmc.sample(env, n, seed=11)[0]
    bits = ((sp.reshape(n, -1) > 0).astype(np.int64) << np.arange(9)[None]).sum(axis=1)
    counts = np.bincount(bits, minlength=512)
    expc = n * q
    keep = expc > 5
    chi2 = float(((counts[keep] - expc[keep]) ** 2 / expc[keep]).sum())
    dof = int(keep.sum()) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)


def test_single_row_is_the_same_in_both_orders():
    inst = instances.random_small(1, 9, 0.8, 2, seed=6)
    sp = tnmc.sample(_env(inst, 2, "raster"), 50, seed=1)[0]
    np.testing.assert_array_equal(tnmc.logq(_env(inst, 2, "snake"), sp)[1], tnmc.logq(_env(inst, 2, "raster"), sp)[1])
