"""Pins of the three-dimensional oracle (Sec. 3D; App. A, three-dimensional paragraph).

What fixes it other than itself:
- The energy against explicit loops over sites and bonds of the cubic lattice.
- Exact D and chi (no truncation anywhere): q = pi by enumeration, on lattices where
  every bond direction and both boundary MPS are non-trivial.
- Lattices one site thick (Ly = 1 or Lx = 1) are planar: the layer PEPS is an MPS, the
  layer boundaries are trivial or exact, and at any truncating D the 3D q must equal
  the two-dimensional oracle's q with chi = D on the same planar lattice (itself pinned).
- At truncating D and chi: q sums to 1 over all states (the forced evaluator is
  prefix-consistent), sampled log q equals forced log q, draw frequencies follow q (chi^2).
"""
import math

import numpy as np
import pytest

from oracle import peps3d, tnmc


def random3d(Lz, Ly, Lx, seed, hs=0.3):
    g = np.random.default_rng(seed)
    return (g.normal(size=(Lz, Ly, Lx - 1)), g.normal(size=(Lz, Ly - 1, Lx)), g.normal(size=(Lz - 1, Ly, Lx)),
            hs * g.normal(size=(Lz, Ly, Lx)))


def all_states3d(Lz, Ly, Lx):
    n = Lz * Ly * Lx
    k = np.arange(2 ** n, dtype=np.int64)[:, None]
    return (2 * ((k >> np.arange(n)[None]) & 1) - 1).reshape(-1, Lz, Ly, Lx).astype(np.int8)


def energy_loops3d(Jx, Jy, Jz, h, s):
    Lz, Ly, Lx = s.shape
    E = 0.0
    for z in range(Lz):
        for y in range(Ly):
            for x in range(Lx):
                E -= h[z][y][x] * s[z][y][x]
                if x + 1 < Lx:
                    E -= Jx[z][y][x] * s[z][y][x] * s[z][y][x + 1]
                if y + 1 < Ly:
                    E -= Jy[z][y][x] * s[z][y][x] * s[z][y + 1][x]
                if z + 1 < Lz:
                    E -= Jz[z][y][x] * s[z][y][x] * s[z + 1][y][x]
    return E


def boltzmann3d(Jx, Jy, Jz, h, beta):
    S = all_states3d(*h.shape)
    E = np.array([energy_loops3d(Jx, Jy, Jz, h, s) for s in S])
    a = -beta * E
    lz = a.max() + math.log(np.exp(a - a.max()).sum())
    return S, np.exp(a - lz)


def test_energy_matches_loops():
    Jx, Jy, Jz, h = random3d(3, 2, 4, 1)
    S = (2 * np.random.default_rng(2).integers(0, 2, size=(300, 3, 2, 4)) - 1).astype(np.int8)
    np.testing.assert_allclose(peps3d.energy3d(Jx, Jy, Jz, h, S),
                               [energy_loops3d(Jx, Jy, Jz, h, s) for s in S], rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("shape", [(3, 2, 2), (2, 2, 3), (2, 3, 2), (2, 2, 4)])
def test_exact_bonds_give_pi(shape):
    Jx, Jy, Jz, h = random3d(*shape, seed=sum(shape))
    env = peps3d.build_env3d(Jx, Jy, Jz, h, 0.7, 64, 512)
    S, pi = boltzmann3d(Jx, Jy, Jz, h, 0.7)
    _, lq, E, fl = peps3d.logq3d(env, S)
    assert np.all(fl == 0)
    np.testing.assert_allclose(np.exp(lq), pi, rtol=1e-9, atol=1e-15)


def _planar(Jx, Jy, Jz, h, axis):
    """The 2D lattice of a one-site-thick 3D lattice: rows = layers z, columns = the
    remaining in-layer direction."""
    if axis == "y":      # Ly = 1
        return Jx[:, 0, :], Jz[:, 0, :], h[:, 0, :]
    return Jy[:, :, 0], Jz[:, :, 0], h[:, :, 0]     # Lx = 1


@pytest.mark.parametrize("shape,axis", [((5, 1, 6), "y"), ((6, 5, 1), "x"), ((4, 1, 7), "y")])
def test_one_site_thick_lattices_reduce_to_two_dimensions(shape, axis):
    Jx, Jy, Jz, h = random3d(*shape, seed=3 + shape[0])
    beta, D = 0.9, 2
    env3 = peps3d.build_env3d(Jx, Jy, Jz, h, beta, D, 2)
    Jh, Jv, h2 = _planar(Jx, Jy, Jz, h, axis)
    env2 = tnmc.build_env(Jh, Jv, h2, beta, D)
    sp3, lq3, E3, _ = peps3d.sample3d(env3, 200, seed=4, sample_offset=9)
    sp2 = sp3.reshape(200, h2.shape[0], h2.shape[1])
    _, lq2, E2, _ = tnmc.logq(env2, sp2)
    np.testing.assert_allclose(lq3, lq2, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(E3, E2, rtol=1e-12, atol=1e-12)
    # and the draws are the 2D sampler's (same Philox words: site z Ly Lx + y Lx + x)
    osp2 = tnmc.sample(env2, 200, seed=4, sample_offset=9)[0]
    assert np.mean(np.all(osp2.reshape(200, -1) == sp3.reshape(200, -1), axis=1)) >= 0.99


def test_truncated_q_is_normalised_and_consistent():
    Jx, Jy, Jz, h = random3d(2, 3, 2, 8)
    env = peps3d.build_env3d(Jx, Jy, Jz, h, 1.1, 2, 1)
    S, pi = boltzmann3d(Jx, Jy, Jz, h, 1.1)
    q = np.exp(peps3d.logq3d(env, S)[1])
    assert q.sum() == pytest.approx(1.0, abs=1e-12)
    assert 0.5 * np.abs(q - pi).sum() > 1e-3          # truncation is active
    sp, lq, E, fl = peps3d.sample3d(env, 300, seed=2)
    _, lqf, Ef, _ = peps3d.logq3d(env, sp)
    np.testing.assert_allclose(lq, lqf, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(E, Ef, rtol=1e-12, atol=1e-12)


def test_draw_frequencies_follow_q():
    Jx, Jy, Jz, h = random3d(2, 2, 2, 5)
    env = peps3d.build_env3d(Jx, Jy, Jz, h, 0.8, 1, 1)
    S = all_states3d(2, 2, 2)
    q = np.exp(peps3d.logq3d(env, S)[1])
    n = 40000
    sp = peps3d.sample3d(env, n, seed=11)[0]
    bits = ((sp.reshape(n, -1) > 0).astype(np.int64) << np.arange(8)[None]).sum(axis=1)
    counts = np.bincount(bits, minlength=256)
    exp = n * q
    keep = exp > 5
    chi2 = float(((counts[keep] - exp[keep]) ** 2 / exp[keep]).sum())
    dof = int(keep.sum()) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)


# ---- the bond basis (vertical bonds split W = B T) ----

@pytest.mark.parametrize("shape", [(3, 2, 2), (2, 2, 3), (2, 3, 2)])
def test_bond_basis_exact_bonds_give_pi(shape):
    Jx, Jy, Jz, h = random3d(*shape, seed=7 + sum(shape))
    env = peps3d.build_env3d_bond(Jx, Jy, Jz, h, 0.7, 64, 512)
    S, pi = boltzmann3d(Jx, Jy, Jz, h, 0.7)
    np.testing.assert_allclose(np.exp(peps3d.logq3d(env, S)[1]), pi, rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("shape", [(5, 1, 6), (4, 1, 7)])
def test_bond_basis_one_row_layers_reduce_to_the_2d_bond_gauge(shape):
    """Ly = 1: each layer is a row, the layer PEPS an MPS compressed by successive SVD, and
    the 3D bond basis is the 2D bond gauge of the planar lattice with chi = D."""
    Jx, Jy, Jz, h = random3d(*shape, seed=11 + shape[0])
    beta, D = 0.9, 2
    env3 = peps3d.build_env3d_bond(Jx, Jy, Jz, h, beta, D, 2)
    Jh, Jv, h2 = _planar(Jx, Jy, Jz, h, "y")
    env2 = tnmc.build_env_bond(Jh, Jv, h2, beta, D)
    sp3, lq3, _, _ = peps3d.sample3d(env3, 150, seed=4, sample_offset=9)
    _, lq2, _, _ = tnmc.logq(env2, sp3.reshape(150, h2.shape[0], h2.shape[1]))
    np.testing.assert_allclose(lq3, lq2, rtol=1e-10, atol=1e-10)


def test_bond_basis_truncated_q_is_normalised_and_better_than_spin_basis():
    Jx, Jy, Jz, h = random3d(2, 3, 2, 8)
    S, pi = boltzmann3d(Jx, Jy, Jz, h, 1.1)
    qb = np.exp(peps3d.logq3d(peps3d.build_env3d_bond(Jx, Jy, Jz, h, 1.1, 1, 1), S)[1])
    qs = np.exp(peps3d.logq3d(peps3d.build_env3d(Jx, Jy, Jz, h, 1.1, 1, 1), S)[1])
    assert qb.sum() == pytest.approx(1.0, abs=1e-12)
    assert 0.5 * np.abs(qb - pi).sum() > 1e-3
    print("TV to pi: bond %.4f, spin %.4f" % (0.5 * np.abs(qb - pi).sum(), 0.5 * np.abs(qs - pi).sum()))
