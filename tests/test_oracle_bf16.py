"""Pins of the oracle's BF16 helpers (the operand rounding of the tensor-core path).

bfloat16 keeps float32's sign and 8 exponent bits and the top 7 of its 23
fraction bits; values are rounded to nearest, ties to even.  The checks use an
independent bit-level formula on float32 patterns, exactly representable values,
and the tie cases.
"""
import numpy as np

from oracle import tnmc
from paper_2104_13264_gb300 import instances


def _bf16_from_f32_bits(x32):
    """Round-to-nearest-even of float32 values to bfloat16 on their bit patterns."""
    b = np.asarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_representable_values_unchanged():
    v = np.array([0.0, 1.0, -1.0, 1.5, -3.0, 2.0 ** -100, 2.0 ** 100, 1.0 + 2.0 ** -7, 255.0 / 128.0])
    assert np.array_equal(tnmc.round_bf16(v), v)


def test_ties_to_even():
    v = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 2.0 + 2.0 ** -7])
    want = np.array([1.0, 1.0 + 2.0 ** -6, -1.0, 2.0])
    assert np.array_equal(tnmc.round_bf16(v), want)


def test_matches_bit_level_rounding_of_float32_values():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(200000) * np.exp(rng.uniform(-30, 30, 200000))).astype(np.float32)
    assert np.array_equal(tnmc.round_bf16(x.astype(np.float64)), _bf16_from_f32_bits(x))


def test_split_carries_sixteen_bits():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))
    hi = tnmc.round_bf16(x)
    s = tnmc.split_bf16(x)
    assert np.array_equal(s - hi, tnmc.round_bf16(x - hi))
    rel = np.abs(s - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -16
    assert np.abs(hi - x).max() > 0          # the lo part is needed


def test_env_bf16_replaces_every_tensor():
    from paper_2104_13264_gb300 import instances
    inst = instances.random_small(3, 4, 0.8, 2, seed=1)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    e2 = tnmc.env_bf16(env)
    for r in range(inst.Ly):
        for c in range(inst.Lx):
            assert e2.M[r][c].shape == env.M[r][c].shape
            assert np.array_equal(e2.M[r][c], tnmc.split_bf16(env.M[r][c]))
    assert e2.logZ == env.logZ


def test_field_combined_right_sweep_is_the_same_recursion():
    """R_c = sum_sigma f(sigma) M[:, sigma, :] R_{c+1} and R_c = Mt^(u) R_{c+1} (the field
    of the spin above applied to the tensor first) are one recursion: in FP64 with
    unrounded Mt the oracle's draws and log q are unchanged."""
    inst = instances.random_small(5, 7, 0.9, 4, seed=3)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    sp, lq, E, fl = tnmc.sample(env, 300, seed=4)
    env.Mr = [[tnmc.field_combined(env, r, c) for c in range(inst.Lx)] for r in range(inst.Ly)]
    sp2, lq2, E2, fl2 = tnmc.sample(env, 300, seed=4)
    assert np.array_equal(sp, sp2) and np.array_equal(fl, fl2)
    np.testing.assert_allclose(lq2, lq, rtol=0, atol=1e-12)
    # the combination itself, entry by entry from the definition of f
    r, c = 3, 2
    Mt = tnmc.field_combined(env, r, c)
    M = env.M[r][c]
    for u, su in enumerate((-1.0, 1.0)):
        ref = sum(np.exp(inst.beta * inst.Jv[r - 1, c] * su * ss) * M[:, k, :] for k, ss in enumerate((-1.0, 1.0)))
        np.testing.assert_allclose(Mt[u], ref, rtol=1e-15, atol=1e-300)
    Mt0 = tnmc.field_combined(env, 0, 2)
    np.testing.assert_array_equal(Mt0[0], env.M[0][2][:, 0, :] + env.M[0][2][:, 1, :])


def test_env_bf16_rounds_the_right_sweep_tensors():
    inst = instances.random_small(4, 5, 0.8, 4, seed=6)
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    e2 = tnmc.env_bf16(env)
    for r in range(inst.Ly):
        for c in range(inst.Lx):
            exact_t = tnmc.field_combined(env, r, c)
            np.testing.assert_array_equal(e2.Mr[r][c], tnmc.split_bf16(exact_t))
            assert np.abs(e2.Mr[r][c] - exact_t).max() <= 2.0 ** -15 * np.abs(exact_t).max()
