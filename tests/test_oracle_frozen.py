"""Pins of the oracle's frozen-line move for closed lattices (App. B).

- The cut: on a torus, H(sigma) = H_open(free spins; fields from the frozen ones) +
  H(frozen spins alone), by brute-force energies of eq. ising.
- The move keeps the Boltzmann distribution of the closed lattice invariant: exact
  samples on a 3 x 4 torus (enumeration) pushed through one move stay distributed as pi
  (chi^2), with a poor q (chi = 1) so that the MH step does the work; a planted mistake
  (the frozen spins' fields dropped) fails it.
"""
import numpy as np
from scipy import stats

from oracle import tnmc

rng = np.random.default_rng(12)


def _torus(L, beta, seed, hscale=0.3):
    r = np.random.default_rng(seed)
    return r.standard_normal((L, L)), r.standard_normal((L, L)), hscale * r.standard_normal((L, L)), beta


def test_cut_energy_decomposition():
    Jh, Jv, h, beta = _torus(5, 1.0, 1)
    sp = rng.choice([-1, 1], size=(40, 5, 5)).astype(np.int8)
    for px, py in ((True, True), (True, False), (False, True)):
        for kr, kc in ((0, 0), (2, 4), (4, 1)):
            rows, cols, Jh_e, Jv_e, h_e = tnmc.frozen_cut(Jh, Jv, h, sp, kr, kc, px, py)
            Eo = np.array([tnmc.energy(Jh_e, Jv_e, h_e[b], sp[b][np.ix_(rows, cols)][None])[0] for b in range(40)])
            Ef = tnmc.energy_periodic(Jh, Jv, h, sp, px, py) - Eo
            # the remainder depends on the frozen spins only: flipping free spins leaves it
            sp2 = sp.copy()
            for i, r in enumerate(rows):
                for j, c in enumerate(cols):
                    if (i + j) % 3 == 0:
                        sp2[:, r, c] *= -1
            rows2, cols2, Jh2, Jv2, h2 = tnmc.frozen_cut(Jh, Jv, h, sp2, kr, kc, px, py)
            Eo2 = np.array([tnmc.energy(Jh2, Jv2, h2[b], sp2[b][np.ix_(rows2, cols2)][None])[0] for b in range(40)])
            np.testing.assert_allclose(tnmc.energy_periodic(Jh, Jv, h, sp2, px, py) - Eo2, Ef, atol=1e-12)


def _move_pvalue():
    Ly, Lx = 3, 4
    r = np.random.default_rng(5)
    Jh, Jv, h = r.standard_normal((Ly, Lx)), r.standard_normal((Ly, Lx)), 0.4 * r.standard_normal((Ly, Lx))
    beta = 1.3
    n_sites = Ly * Lx
    k = np.arange(2 ** n_sites)[:, None]
    S = (2 * ((k >> np.arange(n_sites)[None]) & 1) - 1).astype(np.int8).reshape(-1, Ly, Lx)
    E = tnmc.energy_periodic(Jh, Jv, h, S, True, True)
    w = np.exp(-beta * (E - E.min()))
    pi = w / w.sum()
    n = 60000
    idx = np.random.default_rng(3).choice(len(pi), size=n, p=pi)
    out, acc = tnmc.frozen_line_step(Jh, Jv, h, beta, 1, S[idx], kr=1, kc=2, px=True, py=True, seed=4, step=0, T=2)
    assert 0.05 < acc.mean() < 0.9, acc.mean()
    bits = (out.reshape(n, -1) > 0).astype(np.int64)
    counts = np.bincount((bits << np.arange(n_sites)).sum(axis=1), minlength=len(pi))
    e = n * pi
    keep = e > 5
    chi2 = ((counts[keep] - e[keep]) ** 2 / e[keep]).sum()
    return stats.chi2.sf(chi2, keep.sum() - 1)


def test_frozen_line_move_keeps_pi():
    assert _move_pvalue() > 1e-3


def test_planted_mistake_is_caught(monkeypatch):
    real = tnmc.frozen_cut

    def no_fields(Jh, Jv, h, spins, kr, kc, px, py):
        rows, cols, Jh_e, Jv_e, h_e = real(Jh, Jv, h, spins, kr, kc, px, py)
        return rows, cols, Jh_e, Jv_e, np.broadcast_to(np.asarray(h)[np.ix_(rows, cols)], h_e.shape).copy()

    monkeypatch.setattr(tnmc, "frozen_cut", no_fields)
    assert _move_pvalue() < 1e-6
