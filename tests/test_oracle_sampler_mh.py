"""Pins of the oracle's sampler, evaluator and MH chain (Sec. 2, Algorithm 1) -- no GPU."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import exact, philox, tnmc
from paper_2104_13264_gb300 import instances


def test_q_normalised_at_truncated_chi():
    """Each conditional is normalised, so sum_sigma q(sigma) = 1 for any environment."""
    for chi in (1, 2, 4):
        inst = instances.random_small(4, 4, 0.9, chi, seed=11)
        env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, chi)
        S = exact.all_states(4, 4)
        _, lq, _, fl = tnmc.logq(env, S)
        assert np.all(fl == 0)
        assert np.exp(lq).sum() == pytest.approx(1.0, abs=1e-12)


def test_q_equals_pi_at_exact_chi():
    inst = instances.ea_gauss(4, 4, 1.3, 4, seed=2, hscale=0.4)
    S, logZ, pi, E = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 4)
    _, lq, Eo, _ = tnmc.logq(env, S)
    assert np.max(np.abs(np.exp(lq) / pi - 1)) < 1e-10
    assert np.array_equal(Eo, E) or np.max(np.abs(Eo - E)) < 1e-12
    # MH then accepts every proposal: Delta = 0 up to rounding
    d = -inst.beta * (E[1:] - E[:-1]) + (lq[:-1] - lq[1:])
    assert np.max(np.abs(d)) < 1e-9


def test_sampler_frequencies_match_q():
    """Chi^2 of proposal frequencies against forced q over all 512 states of a 3x3 lattice."""
    inst = instances.random_small(3, 3, 0.8, 2, seed=5)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 2)
    B = 400000
    sp, lq, _, fl = tnmc.sample(env, B, seed=21)
    assert np.all(fl == 0)
    bits = ((sp.reshape(B, 9) > 0).astype(np.int64) << np.arange(9)).sum(axis=1)
    counts = np.bincount(bits, minlength=512)
    S = exact.all_states(3, 3)
    _, lq_all, _, _ = tnmc.logq(env, S)
    e = B * np.exp(lq_all)
    chi2 = ((counts - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi2, 511) > 1e-3
    # the log q returned with each draw is the forced log q of that draw
    assert np.allclose(lq, lq_all[bits], atol=1e-13)


def test_sample_offset_shards_reproduce_one_launch():
    inst = instances.random_small(3, 4, 0.8, 2, seed=6)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 2)
    a = tnmc.sample(env, 64, seed=9)
    b1 = tnmc.sample(env, 40, seed=9, sample_offset=0)
    b2 = tnmc.sample(env, 24, seed=9, sample_offset=40)
    assert np.array_equal(a[0], np.concatenate([b1[0], b2[0]]))
    assert np.array_equal(a[1], np.concatenate([b1[1], b2[1]]))


def test_draw_rule_thresholds():
    x = np.array([0, 1, 2 ** 63 - 1, 2 ** 63, 2 ** 64 - 1], dtype=np.uint64)
    assert tnmc.threshold_plus(np.full(5, 0.5), x).tolist() == [True, True, True, False, False]
    assert tnmc.threshold_plus(np.full(5, 1.0), x).all()
    assert not tnmc.threshold_plus(np.zeros(5), x).any()


def _transition_matrix(pi, q):
    """T(w -> w') = q(w') min(1, q(w) pi(w') / (q(w') pi(w))) for w' != w (eq. mh-acc)."""
    N = pi.size
    T = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            if i != j:
                T[i, j] = q[j] * min(1.0, q[i] * pi[j] / (q[j] * pi[i]))
        T[i, i] = 1.0 - T[i].sum()
    return T


def test_detailed_balance_by_enumeration():
    """pi(w) T(w -> w') is symmetric for an approximate q (Sec. 2, property iv)."""
    inst = instances.random_small(2, 3, 1.1, 1, seed=8)
    S, logZ, pi, E = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 1)
    _, lq, _, _ = tnmc.logq(env, S)
    q = np.exp(lq)
    assert abs(q.sum() - 1) < 1e-12 and exact.tv_distance(pi, q) > 1e-3
    T = _transition_matrix(pi, q)
    F = pi[:, None] * T
    assert np.max(np.abs(F - F.T)) < 1e-15
    # the rule used by the oracle's scan equals min(1, ratio) in probability
    i, j = 3, 17
    ratio = q[i] * pi[j] / (q[j] * pi[i])
    u = np.linspace(0, 1, 100001)[:-1]
    acc = tnmc.mh_accept(inst.beta, np.full(u.size, lq[j]), np.full(u.size, E[j]), lq[i], E[i], u)
    assert acc.mean() == pytest.approx(min(1.0, ratio), abs=2e-5)


def test_mh_rejects_invalid_proposals():
    u = np.array([0.0, 0.0, 0.0, 0.0])
    a = tnmc.mh_accept(1.0, np.array([-np.inf, np.nan, -np.inf, np.nan]), np.zeros(4),
                       np.array([-1.0, -1.0, -np.inf, -np.inf]), np.zeros(4), u)
    assert a.tolist() == [False, False, False, False]


def test_mh_leaves_a_start_outside_the_support():
    """A start with log q = -inf accepts the first valid proposal whatever u and the
    energies are; a start with finite log q follows the ordinary rule."""
    u = np.array([0.999999, 0.5, 0.999999])
    a = tnmc.mh_accept(1.0, np.array([-1.0, -3.0, -1.0]), np.array([50.0, 0.0, 50.0]),
                       np.array([-np.inf, -np.inf, -2.0]), np.array([0.0, 0.0, 0.0]), u)
    assert a.tolist() == [True, True, False]


def _batch_means(x, nb=20):
    x = np.asarray(x, dtype=np.float64)
    m = x.size // nb
    bm = x[: m * nb].reshape(nb, m).mean(axis=1)
    return bm.mean(), bm.std(ddof=1) / math.sqrt(nb)


def test_chain_samples_pi_with_poor_q():
    """chi = 1 gives a poor q; the MH chain still samples pi (Sec. 2, property iv).

    Compares chain averages of the energy and of every spin with their exact
    Boltzmann values, using the spread of independent chains as the error.
    """
    inst = instances.random_small(3, 3, 0.4, 1, seed=0, hscale=0.5)
    S, logZ, pi, E = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 1)
    q = np.exp(tnmc.logq(env, S)[1])
    assert exact.tv_distance(pi, q) > 0.3
    C, T, burn = 256, 400, 100
    sp, lq, Ep, fl = tnmc.sample(env, C * T, seed=4)
    cs, clq, cE = tnmc.init_chains(env, C, seed=4)
    acc, _, _, _ = tnmc.mh_scan(inst.beta, C, T, sp, lq, Ep, cs, clq, cE, seed=4)
    a2 = acc.reshape(C, T)
    curE = cE.copy()
    curS = cs.reshape(C, 9).astype(np.float64)
    sumE = np.zeros(C)
    sumS = np.zeros((C, 9))
    props = sp.reshape(C, T, 9).astype(np.float64)
    for j in range(T):
        curE = np.where(a2[:, j], Ep.reshape(C, T)[:, j], curE)
        curS = np.where(a2[:, j, None], props[:, j], curS)
        if j >= burn:
            sumE += curE
            sumS += curS
    mE = sumE / (T - burn)
    mS = sumS / (T - burn)
    Sf = S.reshape(-1, 9).astype(np.float64)
    exE, exS = float(pi @ E), pi @ Sf
    qE = float(q @ E)
    seE = mE.std(ddof=1) / math.sqrt(C)
    assert abs(mE.mean() - exE) < 4 * seE
    assert abs(qE - exE) > 10 * seE          # the test can tell q from pi
    seS = mS.std(axis=0, ddof=1) / math.sqrt(C)
    assert np.all(np.abs(mS.mean(axis=0) - exS) < 4.5 * seS)


def test_chain_acceptance_matches_exact_value():
    """Measured acceptance agrees with the exact stationary acceptance within 3 sigma."""
    inst = instances.random_small(4, 4, 0.9, 2, seed=12)
    S, logZ, pi, E = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 1)
    q = np.exp(tnmc.logq(env, S)[1])
    a_exact = exact.independence_acceptance(pi, q)
    C, T = 200, 400
    sp, lq, Ep, _ = tnmc.sample(env, C * T, seed=13)
    cs, clq, cE = tnmc.init_chains(env, C, seed=13)
    acc, _, _, _ = tnmc.mh_scan(inst.beta, C, T, sp, lq, Ep, cs, clq, cE, seed=13)
    per_chain = acc.reshape(C, T)[:, 50:].mean(axis=1)
    m, se = per_chain.mean(), per_chain.std(ddof=1) / math.sqrt(C)
    assert abs(m - a_exact) < 3 * se + 1e-3
    assert a_exact < 0.99


def test_independence_acceptance_brute_force():
    rng = np.random.default_rng(0)
    pi = rng.random(40); pi /= pi.sum()
    q = rng.random(40); q /= q.sum()
    q[[3, 7]] = q[[5, 5]]                  # ties in pi/q are handled
    pi[3] = pi[5]
    a = sum(min(pi[i] * q[j], pi[j] * q[i]) for i in range(40) for j in range(40))
    assert exact.independence_acceptance(pi, q) == pytest.approx(a, rel=1e-12)


def test_config1_chain_observables(golden):
    """8x8 ferromagnet chain (chi = 8, 10^4 steps, random start) vs the transfer matrix."""
    inst = instances.config1()
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    T = 10000
    sp, lq, Ep, fl = tnmc.sample(env, T, seed=0)
    assert np.all(fl == 0)
    cs, clq, cE = tnmc.init_chains(env, 1, seed=0)
    acc, _, _, _ = tnmc.mh_scan(inst.beta, 1, T, sp, lq, Ep, cs, clq, cE, seed=0)
    assert acc.mean() > 0.5
    idx = np.maximum.accumulate(np.where(acc, np.arange(T), -1))
    burn = 100
    states_E = np.where(idx >= 0, Ep[np.maximum(idx, 0)], cE[0])[burn:]
    absm = np.abs(np.where(idx[:, None] >= 0, sp[np.maximum(idx, 0)].reshape(T, -1),
                           cs.reshape(1, -1)).mean(axis=1))[burn:]
    mE, sE = _batch_means(states_E / 64)
    mm, sm = _batch_means(absm)
    ref = golden["ferro8x8_b044"]
    assert abs(mE - ref["E_per_spin"]) < 3 * sE + 2e-3
    assert abs(mm - ref["abs_m"]) < 3 * sm + 2e-3


def test_init_chain_bits():
    sp = philox.init_bits(5, 300, np.arange(4))
    assert set(np.unique(sp)) <= {-1, 1}
    assert 0.4 < (sp > 0).mean() < 0.6


def test_flagged_samples_keep_their_draw_probability():
    """Signed tensors make both weights of some conditionals clamp to zero; such a site is
    drawn with p = 1/2.  q must remain the exact law of the procedure: summed over every
    configuration it is 1 including the flagged ones, and the sampler's draws follow it."""
    Ly, Lx = 2, 3
    shapes = [(tnmc.bond_dim(2, Lx, Ly, r, c), 2, tnmc.bond_dim(2, Lx, Ly, r, c + 1))
              for r in range(Ly) for c in range(Lx)]
    ts = instances.random_tensors(shapes, seed=3, positive=False)
    inst = instances.random_small(Ly, Lx, 0.7, 2, seed=4)
    env = tnmc.Env(Lx, Ly, inst.beta, 2, inst.Jh, inst.Jv, inst.h)
    env.M = [[ts[r * Lx + c] for c in range(Lx)] for r in range(Ly)]
    S = exact.all_states(Ly, Lx)
    _, lq, _, fl = tnmc.logq(env, S)
    assert fl.any() and (fl == 0).any()
    assert np.exp(lq).sum() == pytest.approx(1.0, abs=1e-12)
    sp, lq2, _, fl2 = tnmc.sample(env, 200_000, seed=5)
    idx = ((sp.reshape(len(sp), -1) > 0).astype(np.int64) << np.arange(Ly * Lx)).sum(axis=1)
    counts = np.bincount(idx, minlength=len(S))
    np.testing.assert_allclose(lq2, lq[idx], rtol=0, atol=1e-12)
    e = len(sp) * np.exp(lq)
    keep = e > 5
    assert stats.chi2.sf(((counts[keep] - e[keep]) ** 2 / e[keep]).sum(), keep.sum() - 1) > 1e-3
