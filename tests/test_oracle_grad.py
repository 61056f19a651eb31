"""Pins of the oracle's reverse-mode gradient of log q -- no GPU."""
import numpy as np
import pytest

from oracle import exact, tnmc
from paper_2104_13264_gb300 import instances


@pytest.fixture(scope="module")
def case():
    inst = instances.villain(4, 5, 1.5, 2)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 2)
    sp, lq, _, fl = tnmc.sample(env, 40, seed=3)
    w = np.random.default_rng(1).random(40)
    lq2, G = tnmc.logq_grad(env, sp, w)
    return inst, env, sp, w, lq2, G


def test_matches_central_differences(case):
    inst, env, sp, w, _, G = case
    for r, c in ((0, 0), (0, 4), (1, 2), (2, 1), (3, 3)):
        fd = tnmc.finite_diff_grad(env, sp, w, r, c)
        scale = max(np.abs(fd).max(), 1e-3)
        assert np.abs(G[r][c] - fd).max() < 1e-6 * scale + 1e-9, (r, c)


def test_degree_zero_homogeneity(case):
    """log q is invariant under M_c -> lambda M_c, hence <G_c, M_c> = 0."""
    _, env, _, _, _, G = case
    for r in range(env.Ly):
        for c in range(env.Lx):
            assert abs(np.sum(G[r][c] * env.M[r][c])) < 1e-10 * (1 + np.abs(G[r][c]).sum())


def test_gauge_invariance(case):
    """Inserting X X^-1 on a bond leaves q unchanged: <G_c, M_c X> = <G_{c+1}, X M_{c+1}>."""
    _, env, _, _, _, G = case
    rng = np.random.default_rng(4)
    for r in range(env.Ly):
        for c in range(env.Lx - 1):
            d = env.M[r][c].shape[2]
            X = rng.standard_normal((d, d))
            lhs = np.sum(G[r][c] * np.einsum("asb,bk->ask", env.M[r][c], X))
            rhs = np.sum(G[r][c + 1] * np.einsum("kb,bsc->ksc", X, env.M[r][c + 1]))
            assert lhs == pytest.approx(rhs, abs=1e-10 * (1 + abs(lhs)))


def test_log_q_unchanged_by_gauge_transform(case):
    _, env, sp, _, lq, _ = case
    rng = np.random.default_rng(6)
    r, c = 2, 1
    d = env.M[r][c].shape[2]
    X = rng.standard_normal((d, d)) + 3 * np.eye(d)
    M0, M1 = env.M[r][c], env.M[r][c + 1]
    try:
        env.M[r][c] = np.einsum("asb,bk->ask", M0, X)
        env.M[r][c + 1] = np.einsum("kb,bsc->ksc", np.linalg.inv(X), M1)
        lq2 = tnmc.logq(env, sp)[1]
    finally:
        env.M[r][c], env.M[r][c + 1] = M0, M1
    assert np.allclose(lq, lq2, atol=1e-12)


def test_exact_chi_gradient_has_closed_form():
    """At exact chi, log q = log pi - the row-local part; a perturbation along M_c
    that keeps the environment exact changes nothing, and the gradient of
    sum_sigma q(sigma) = 1 vanishes."""
    inst = instances.random_small(3, 3, 0.8, 2, seed=2)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 2)
    S = exact.all_states(3, 3)
    lq = tnmc.logq(env, S)[1]
    q = np.exp(lq)
    # d/dM sum_sigma q(sigma) = sum_sigma q(sigma) d log q(sigma) = 0 (normalisation)
    _, G = tnmc.logq_grad(env, S, q)
    for r in range(3):
        for c in range(3):
            assert np.abs(G[r][c]).max() < 1e-12
