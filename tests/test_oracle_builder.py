"""Pins of the oracle's boundary-MPS builder (App. A) -- no GPU."""
import math

import numpy as np
import pytest

from oracle import exact, tnmc
from paper_2104_13264_gb300 import instances


def _arrays(case):
    return (np.asarray(case[k], dtype=np.float64) for k in ("Jh", "Jv", "h"))


def test_exact_chi_reproduces_enumerated_Z(golden):
    """With chi >= 2^floor(min(Lx, Ly...)/2) nothing is truncated and Z~ = Z."""
    for case in golden["small"]:
        Jh, Jv, h = _arrays(case)
        chi = 2 ** (case["Lx"] // 2)
        env = tnmc.build_env(Jh, Jv, h, case["beta"], chi)
        assert env.logZ == pytest.approx(case["logZ"], abs=1e-11), case["name"]
        assert max(env.discarded.values()) < 1e-24


def test_transfer_matrix_matches_enumeration(golden):
    for case in golden["small"]:
        Jh, Jv, h = _arrays(case)
        logZ, E, _ = exact.transfer_matrix(Jh, Jv, h, case["beta"])
        assert logZ == pytest.approx(case["logZ"], abs=1e-11)
        assert E == pytest.approx(case["E_mean"], abs=1e-10)


def test_ferro8x8_exact_at_chi16(golden):
    inst = instances.config1()
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 16)
    assert env.logZ == pytest.approx(golden["ferro8x8_b044"]["logZ"], abs=1e-10)
    env8 = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 8)
    # truncated: Z~ close to but not equal to Z
    assert abs(env8.logZ - golden["ferro8x8_b044"]["logZ"]) < 1e-3
    assert max(env8.discarded.values()) > 0


def test_beta_zero_is_uniform():
    inst = instances.random_small(4, 5, 0.0, 2, seed=4)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, 0.0, 2)
    n = inst.Lx * inst.Ly
    assert env.logZ == pytest.approx(n * math.log(2), abs=1e-12)
    S = np.random.default_rng(0).choice([-1, 1], size=(30, 4, 5)).astype(np.int8)
    _, lq, _, fl = tnmc.logq(env, S)
    assert np.all(fl == 0)
    assert np.allclose(lq, -n * math.log(2), atol=1e-12)


def test_zero_couplings_product_state():
    rng = np.random.default_rng(3)
    Ly, Lx = 4, 6
    h = rng.standard_normal((Ly, Lx))
    beta = 0.8
    env = tnmc.build_env(np.zeros((Ly, Lx - 1)), np.zeros((Ly - 1, Lx)), h, beta, 1)
    assert env.logZ == pytest.approx(float(np.sum(np.log(2 * np.cosh(beta * h)))), abs=1e-12)


def test_single_row_and_ladder_closed_form():
    rng = np.random.default_rng(5)
    Lx = 9
    J = rng.standard_normal(Lx - 1)
    beta = 0.9
    env = tnmc.build_env(J[None], np.zeros((0, Lx)), np.zeros((1, Lx)), beta, 2)
    z1 = math.log(2) + float(np.sum(np.log(2 * np.cosh(beta * J))))
    assert env.logZ == pytest.approx(z1, abs=1e-12)
    # 2 x Lx ladder is exact at chi = 4 (= 2^(Ly - r) bound); compare with the transfer matrix
    Jh = rng.standard_normal((2, Lx - 1))
    Jv = rng.standard_normal((1, Lx))
    env = tnmc.build_env(Jh, Jv, np.zeros((2, Lx)), beta, 4)
    logZ, _, _ = exact.transfer_matrix(Jh, Jv, np.zeros((2, Lx)), beta)
    assert env.logZ == pytest.approx(logZ, abs=1e-11)


def test_bond_dimensions_follow_static_rule():
    inst = instances.random_small(5, 7, 0.7, 3, seed=9)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    for r in range(inst.Ly):
        for c in range(inst.Lx):
            a, two, b = env.M[r][c].shape
            assert two == 2
            assert a == tnmc.bond_dim(inst.chi, inst.Lx, inst.Ly, r, c)
            assert b == tnmc.bond_dim(inst.chi, inst.Lx, inst.Ly, r, c + 1)


def test_right_canonical_form():
    """After the right-to-left SVD sweep every site c >= 1 is right-orthonormal."""
    inst = instances.ea_gauss(6, 6, 1.2, 4, seed=1)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    for r in range(inst.Ly):
        for c in range(1, inst.Lx):
            M = env.M[r][c]
            A = M.reshape(M.shape[0], -1)
            assert np.allclose(A @ A.T, np.eye(M.shape[0]), atol=1e-12)
        assert np.linalg.norm(env.M[r][0]) == pytest.approx(1.0, abs=1e-14)


def test_truncation_error_decreases_with_chi(golden):
    inst = instances.config1()
    ref = golden["ferro8x8_b044"]["logZ"]
    errs = [abs(tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, chi).logZ - ref) for chi in (1, 2, 4, 8)]
    assert errs[0] > errs[1] > errs[2] > errs[3]


def test_onsager_trend(golden):
    """log Z~ / n approaches -beta f of the infinite lattice as L grows (Sec. 3 cites the exact results)."""
    beta = 0.3
    target = golden["onsager_minus_beta_f"]["0.3"]
    gaps = []
    for L in (8, 16, 24):
        inst = instances.ferromagnet(L, L, beta, 8)
        env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, beta, 8)
        gaps.append(target - env.logZ / (L * L))
    # open boundaries cost free energy: positive gap shrinking roughly like 1/L
    assert gaps[0] > gaps[1] > gaps[2] > 0
    assert gaps[2] * 24 == pytest.approx(gaps[1] * 16, rel=0.15)


def test_onsager_closed_forms(golden):
    g = golden["onsager_minus_beta_f_at_beta_c"]
    assert g["value"] == pytest.approx(g["closed_form"], abs=1e-12)
    # energy per spin tends to -sqrt(2) at beta_c from both sides
    bc = exact.BETA_C
    for d in (1e-6, -1e-6):
        assert exact.onsager_energy_per_spin(bc + d) == pytest.approx(-math.sqrt(2), abs=5e-4)
    assert exact.yang_magnetisation(0.3) == 0.0
    assert 0.9 < golden["yang_m_beta_0.6"] < 1.0
