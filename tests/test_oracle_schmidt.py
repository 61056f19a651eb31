"""Pins of the oracle builder's singular-value record (App. A, "successive SVD").

At every SVD step of the right-to-left sweep the oracle records the kept
singular values divided by the 2-norm of all of them (`env.sv`) and the
discarded squared-weight fraction (`env.discarded`); the CUDA builder is
compared with both.  They are pinned here against a computation that shares
nothing with the builder: the exact row-weight vector psi_r, enumerated over
all configurations of rows r..Ly-1 (oracle.exact.row_weight_vector), cut
between sites c-1 and c and put through an SVD.

- When nothing below (r, c) in the build order was truncated, the site matrix of
  that SVD step is psi_r in mixed canonical form, so its normalised singular
  values are psi_r's Schmidt coefficients.  At exact chi that holds at every
  bond of every row.
- At the first truncated bond of the build (rows from Ly-1 up, bonds from Lx-1
  down) the discarded fraction is psi_r's Schmidt tail weight there.
A normalisation by the largest instead of the 2-norm, squared values, or a
wrong kept count each fail one of these.
"""
import numpy as np
import pytest

from oracle import exact, tnmc
from paper_2104_13264_gb300 import instances


def _exact_rank(Lx, Ly, r, c):
    return min(1 << c, 1 << (Lx - c), 1 << (Ly - r))


@pytest.mark.parametrize("inst", [instances.random_small(3, 5, 0.8, 4, seed=11),
                                  instances.random_small(4, 4, 0.9, 4, seed=12),
                                  instances.ea_pm(4, 4, 1.0, 4, seed=13)])
def test_sv_equal_schmidt_coefficients_at_exact_chi(inst):
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    assert len(env.sv) == inst.Ly * (inst.Lx - 1)
    for r in range(inst.Ly):
        psi = exact.row_weight_vector(inst.Jh, inst.Jv, inst.h, inst.beta, r)
        for c in range(1, inst.Lx):
            lam = exact.schmidt_values(psi, inst.Lx, c)
            k = tnmc.bond_dim(inst.chi, inst.Lx, inst.Ly, r, c)
            assert k == _exact_rank(inst.Lx, inst.Ly, r, c)
            np.testing.assert_allclose(env.sv[(r, c)], lam[:k], rtol=0, atol=1e-12)
            assert env.discarded[(r, c)] == pytest.approx(float(np.sum(lam[k:] ** 2)), abs=1e-24)


@pytest.mark.parametrize("inst", [instances.random_small(3, 5, 0.8, 2, seed=21),
                                  instances.random_small(4, 4, 0.9, 2, seed=22),
                                  instances.ea_gauss(4, 5, 1.2, 2, seed=23),
                                  instances.random_small(4, 6, 0.7, 3, seed=24)])
def test_first_truncation_discards_the_schmidt_tail(inst):
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    Lx, Ly = inst.Lx, inst.Ly
    order = [(r, c) for r in range(Ly - 1, -1, -1) for c in range(Lx - 1, 0, -1)]
    first = next((r, c) for r, c in order
                 if tnmc.bond_dim(inst.chi, Lx, Ly, r, c) < _exact_rank(Lx, Ly, r, c))
    r0, c0 = first
    psi = exact.row_weight_vector(inst.Jh, inst.Jv, inst.h, inst.beta, r0)
    # every bond before it in the build order is exact: Schmidt coefficients there
    for r, c in order[:order.index(first)]:
        lam = exact.schmidt_values(exact.row_weight_vector(inst.Jh, inst.Jv, inst.h, inst.beta, r), Lx, c)
        k = env.sv[(r, c)].size
        np.testing.assert_allclose(env.sv[(r, c)], lam[:k], atol=1e-12)
    lam = exact.schmidt_values(psi, Lx, c0)
    k = tnmc.bond_dim(inst.chi, Lx, Ly, r0, c0)
    tail = float(np.sum(lam[k:] ** 2))
    assert tail > 1e-10                     # a real truncation
    # squared singular values carry ~1e-16 of the total weight in absolute error
    assert env.discarded[(r0, c0)] == pytest.approx(tail, rel=1e-6, abs=1e-15)
    np.testing.assert_allclose(env.sv[(r0, c0)], lam[:k], atol=1e-12)


def test_row_weight_vector_sums_to_Z():
    """sum_sigma_0 psi_0 = Z (rows above row 0: none), by enumeration both ways."""
    inst = instances.random_small(3, 4, 0.7, 4, seed=3)
    psi = exact.row_weight_vector(inst.Jh, inst.Jv, inst.h, inst.beta, 0)
    _, logZ, _, _ = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    assert np.log(psi.sum()) == pytest.approx(logZ, abs=1e-12)
