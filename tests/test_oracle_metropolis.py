"""Pins of the oracle's single-spin-flip Metropolis sweeps and of the link-overlap
diagnostic (Sec. 3, "Equilibration", eq. Delta).

- A checkerboard sweep must leave the Boltzmann distribution invariant: exact
  samples of pi (drawn by enumeration) pushed through one oracle sweep are still
  distributed as pi (chi^2).  A planted mistake in the local field fails it.
- The local field is checked against energy differences of eq. ising computed by
  brute force (oracle.exact.energy_loops).
- The paper's identity: for Gaussian couplings the disorder average of
  (1/|V|)(<H> + beta (|E| - sum <s_i s_j>^2)) vanishes.  It is checked with exact
  thermal averages (enumeration) over many 3x3 disorder samples, which pins the
  estimator's signs and normalisation; the chain estimator (replica pairs) agrees
  with the exact per-instance value within its statistical error.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import exact, tnmc
from paper_2104_13264_gb300 import instances


def _exact_samples(inst, n, seed):
    S, _, pi, _ = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    idx = np.random.default_rng(seed).choice(len(pi), size=n, p=pi)
    return S, pi, idx


def _state_index(spins):
    bits = (np.asarray(spins).reshape(spins.shape[0], -1) > 0).astype(np.int64)
    return (bits << np.arange(bits.shape[1])).sum(axis=1)


def _sweep_chi2_pvalue(inst, n=400_000):
    S, pi, idx = _exact_samples(inst, n, seed=3)
    out = tnmc.metropolis_sweeps(inst.Jh, inst.Jv, inst.h, inst.beta, S[idx], seed=9, sweep_offset=0, sweeps=1,
                                 chain_ids=np.arange(n))
    counts = np.bincount(_state_index(out), minlength=len(pi))
    e = n * pi
    keep = e > 5
    chi2 = ((counts[keep] - e[keep]) ** 2 / e[keep]).sum()
    return stats.chi2.sf(chi2, keep.sum() - 1)


def test_sweep_leaves_boltzmann_invariant():
    inst = instances.random_small(2, 3, 0.8, 1, seed=5, hscale=0.5)
    assert _sweep_chi2_pvalue(inst) > 1e-3


def test_planted_mistake_breaks_invariance(monkeypatch):
    """Dropping the neighbours from the local field (a plausible slip) must be caught."""
    inst = instances.random_small(2, 3, 0.8, 1, seed=5, hscale=0.5)
    monkeypatch.setattr(tnmc, "local_field", lambda Jh, Jv, h, spins: np.broadcast_to(
        np.asarray(h, dtype=np.float64), np.asarray(spins).shape).copy())
    assert _sweep_chi2_pvalue(inst) < 1e-6


def test_local_field_is_half_the_flip_energy():
    inst = instances.random_small(3, 4, 1.0, 1, seed=2, hscale=0.7)
    rng = np.random.default_rng(1)
    sp = rng.choice([-1, 1], size=(5, 3, 4)).astype(np.int8)
    f = tnmc.local_field(inst.Jh, inst.Jv, inst.h, sp)
    for b in range(5):
        E0 = exact.energy_loops(inst.Jh, inst.Jv, inst.h, sp[b])
        for r in range(3):
            for c in range(4):
                s2 = sp[b].copy()
                s2[r, c] = -s2[r, c]
                dE = exact.energy_loops(inst.Jh, inst.Jv, inst.h, s2) - E0
                assert dE == pytest.approx(2.0 * sp[b, r, c] * f[b, r, c], abs=1e-12)


def test_sweep_counters_shard_and_compose():
    inst = instances.ea_gauss(4, 5, 1.5, 1, seed=3)
    sp = np.random.default_rng(2).choice([-1, 1], size=(10, 4, 5)).astype(np.int8)
    ids = np.arange(100, 110)
    two = tnmc.metropolis_sweeps(inst.Jh, inst.Jv, inst.h, inst.beta, sp, 7, 40, 2, ids)
    one = tnmc.metropolis_sweeps(inst.Jh, inst.Jv, inst.h, inst.beta, sp, 7, 40, 1, ids)
    one = tnmc.metropolis_sweeps(inst.Jh, inst.Jv, inst.h, inst.beta, one, 7, 41, 1, ids)
    assert np.array_equal(two, one)
    part = tnmc.metropolis_sweeps(inst.Jh, inst.Jv, inst.h, inst.beta, sp[3:7], 7, 40, 2, ids[3:7])
    assert np.array_equal(two[3:7], part)
    assert not np.array_equal(two, sp)


def _exact_delta(inst):
    S, _, pi, E = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    s = S.astype(np.float64)
    corr = []
    if inst.Lx > 1:
        corr.append((pi[:, None, None] * s[:, :, :-1] * s[:, :, 1:]).sum(axis=0).ravel())
    if inst.Ly > 1:
        corr.append((pi[:, None, None] * s[:, :-1, :] * s[:, 1:, :]).sum(axis=0).ravel())
    q = float(np.sum(np.concatenate(corr) ** 2))
    return tnmc.delta_instance(inst.beta, inst.Lx, inst.Ly, float(pi @ E), q)


def test_delta_vanishes_on_the_gaussian_disorder_average():
    """Integration by parts over N(0, 1) couplings: [<H>] = -beta sum (1 - [<s_i s_j>^2])."""
    d = np.array([_exact_delta(instances.ea_gauss(3, 3, 1.3, 1, seed=1000 + k, float32=False)) for k in range(3000)])
    assert abs(d.mean()) < 3 * d.std(ddof=1) / np.sqrt(d.size), (d.mean(), d.std())
    # a single instance is not zero: the identity is a statement about the average
    assert np.abs(d).mean() > 10 * d.std(ddof=1) / np.sqrt(d.size)


def test_delta_from_replica_pairs_estimates_the_instance_value():
    inst = instances.ea_gauss(3, 4, 1.1, 1, seed=7, float32=False)
    S, pi, idx = _exact_samples(inst, 200_000, seed=11)
    sp = S[idx]
    E = tnmc.energy(inst.Jh, inst.Jv, inst.h, sp)
    est = tnmc.delta_from_chains(inst.beta, inst.Lx, inst.Ly, sp, E)
    q = tnmc.link_overlap(None, None, sp[0::2], sp[1::2])
    err = np.sqrt(np.var(E) / E.size + inst.beta ** 2 * np.var(q) / q.size) / (inst.Lx * inst.Ly)
    assert est == pytest.approx(_exact_delta(inst), abs=4 * err)
