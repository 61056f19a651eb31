"""Pins of the two-site variational compression (App. A: the alternative to successive SVD).

What fixes it other than itself:
- Eckart-Young: with one truncated bond (the others at their exact rank), the best
  approximation is the rank-k SVD of the dense vector cut at that bond, computed here
  by numpy's SVD of the contracted vector.
- The objective: no sweep increases ||X - e^ls Y|| (dense vectors, 2^Lx entries), and
  on generic rows the sweeps improve on successive SVD.
- Stationarity: after many sweeps the gradient of ||X - Y||^2 with respect to every
  site tensor, built element by element from dense contractions, vanishes.
- Exact chi: q = pi by enumeration; a truncating chi gives a normalised q.
"""
import math

import numpy as np
import pytest

from oracle import exact, tnmc
from paper_2104_13264_gb300 import instances


def dense(tensors):
    """The 2^Lx vector of an MPS, site 0 the most significant index."""
    v = np.ones((1, 1))
    for t in tensors:
        v = np.einsum("na,asb->nsb", v, t).reshape(-1, t.shape[2])
    return v[:, 0]


def random_mps(Lx, D, seed):
    g = np.random.default_rng(seed)
    dims = [1] + [min(D, 2 ** min(c, Lx - c)) for c in range(1, Lx)] + [1]
    return [g.standard_normal((dims[c], 2, dims[c + 1])) * (1 + 0.2 * c) for c in range(Lx)]


def approx_error(X, Y, ls):
    x = dense(X)
    return float(np.linalg.norm(x - math.exp(ls) * dense(Y)) / np.linalg.norm(x))


def test_one_truncated_bond_is_the_eckart_young_optimum():
    # Lx = 4, chi = 2: bonds 1 and 3 have exact rank <= 2, only bond 2 (rank 4) is cut
    for seed in range(4):
        X = random_mps(4, 4, seed)
        Y, ls = tnmc.truncate_row_variational(X, 2, 4, 40, 0, sweeps=2)
        U, S, Vh = np.linalg.svd(dense(X).reshape(4, 4))
        best = (U[:, :2] * S[:2]) @ Vh[:2]
        np.testing.assert_allclose(math.exp(ls) * dense(Y), best.ravel(), rtol=1e-10, atol=1e-12 * S[0])


@pytest.mark.parametrize("seed", range(3))
def test_sweeps_never_increase_the_error_and_improve_on_successive_svd(seed):
    Lx, chi = 8, 2
    X = random_mps(Lx, 8, seed)
    Y0, l0 = tnmc.truncate_row(X, chi, Lx, 40, 0)
    errs = [approx_error(X, Y0, l0)]
    for sw in (1, 2, 4):
        Y, ls = tnmc.truncate_row_variational(X, chi, Lx, 40, 0, sweeps=sw)
        errs.append(approx_error(X, Y, ls))
    assert all(b <= a * (1 + 1e-10) for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < errs[0] * (1 - 1e-4), errs


def test_ising_row_improves_on_successive_svd():
    inst = instances.ea_gauss(6, 9, 1.5, 2, seed=11, hscale=0.3)
    X = tnmc.apply_row_mpo(tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 2).M[3], inst.Jh, inst.Jv, inst.h,
                           inst.beta, 2)
    Y0, l0 = tnmc.truncate_row(X, 2, 9, 6, 2)
    Y1, l1 = tnmc.truncate_row_variational(X, 2, 9, 6, 2, sweeps=3)
    e0, e1 = approx_error(X, Y0, l0), approx_error(X, Y1, l1)
    assert e1 < e0 * (1 - 1e-4), (e0, e1)


def test_converged_sweeps_are_stationary():
    Lx, chi = 6, 2
    X = random_mps(Lx, 8, 5)
    Y, ls = tnmc.truncate_row_variational(X, chi, Lx, 40, 0, sweeps=60)
    x = dense(X)
    y = math.exp(ls) * dense(Y)
    scale = np.linalg.norm(x)
    for c in range(Lx):
        # d/dY_c of ||x - y||^2 element by element: y is linear in Y_c
        grad = np.zeros(Y[c].size)
        bound = 0.0
        for i in range(Y[c].size):
            Ei = np.zeros(Y[c].size)
            Ei[i] = 1.0
            T = list(Y)
            T[c] = Ei.reshape(Y[c].shape)
            t = math.exp(ls) * dense(T)
            grad[i] = 2.0 * t @ (y - x)
            bound = max(bound, 2.0 * np.linalg.norm(t) * scale)
        assert np.abs(grad).max() < 1e-8 * bound, (c, np.abs(grad).max(), bound)


@pytest.mark.parametrize("inst", [instances.random_small(4, 4, 0.9, 8, seed=2), instances.ea_pm(3, 5, 1.0, 8, seed=4)])
def test_exact_chi_gives_pi(inst):
    env = tnmc.build_env_variational(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi, sweeps=2)
    S, logZ, pi, _ = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    assert env.logZ == pytest.approx(logZ, abs=1e-10)
    q = np.exp(tnmc.logq(env, S)[1])
    np.testing.assert_allclose(q, pi, rtol=1e-9, atol=1e-15)


def test_truncating_chi_is_a_normalised_proposal():
    inst = instances.random_small(4, 5, 1.1, 2, seed=7, hscale=0.2)
    S, _, pi, _ = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    qv = np.exp(tnmc.logq(tnmc.build_env_variational(inst.Jh, inst.Jv, inst.h, inst.beta, 2, sweeps=2), S)[1])
    qs = np.exp(tnmc.logq(tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 2), S)[1])
    assert qv.sum() == pytest.approx(1.0, abs=1e-12)
    assert exact.tv_distance(qv, qs) > 1e-8
    av, a_s = exact.independence_acceptance(pi, qv), exact.independence_acceptance(pi, qs)
    assert 0.0 < av < 1.0 and 0.0 < a_s < 1.0
