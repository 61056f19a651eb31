"""Statistical agreement of GPU chains with exact values (needs a GB300).

The MH step makes the chain's stationary law exactly pi whatever q is (Sec. 2,
property iv, Algorithm 1); the acceptance rate of the independence sampler is a
fixed functional of (pi, q).  Here chains run entirely through the C ABI and are
compared with values that do not come from the GPU:

- 8 x 8 ferromagnet at beta = 0.44, chi = 8, 10^4 proposals in one chain (the
  first workload): <E>/n and <|m|> within 3 sigma (batch means) of the row
  transfer matrix values stored in tests/golden.
- 4 x 4 lattice at chi = 1 (a poor q): the measured acceptance within 3 sigma of
  the exact stationary acceptance computed from the oracle's q and pi by
  enumeration (oracle.exact.independence_acceptance).
- The lower-precision forms keep the acceptance of the plain FP64 form within 1 %
  (relative), on the 256-wide chi = 64 strip and on a +-J glass at chi = 4 whose
  acceptance is about 0.95 (rejections there are q's own error, so a precision loss
  would show; 2.6e5 proposals put 1 % at about 15 standard errors).
"""
import math

import numpy as np
import pytest

from oracle import exact, tnmc
from paper_2104_13264_gb300 import instances

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_13264_gb300 import binding
    binding.lib()
    return binding


def _chain_trace(B, env, C, T, seed, precision):
    """Run C chains of T proposals each through the C ABI; return the accept flags
    [C, T] and, per chain, the index of the proposal that is the state after each step
    (-1: still the start)."""
    sp, lq, E, fl = B.sample(env, C * T, seed=seed, precision=precision)
    chain = B.init_chains(env, C, seed=seed + 1, precision=precision)
    acc = B.mh_step(env, C, T, (sp, lq, E), chain, seed=seed + 2)
    torch.cuda.synchronize()
    a = acc.cpu().numpy().astype(bool).reshape(C, T)
    idx = np.where(a, np.arange(C * T).reshape(C, T), -1)
    state = np.maximum.accumulate(idx, axis=1)
    return a, state, sp, E


def _batch_means(x, nb):
    x = np.asarray(x, dtype=np.float64)
    m = x.size // nb
    bm = x[:m * nb].reshape(nb, m).mean(axis=1)
    return bm.mean(), bm.std(ddof=1) / math.sqrt(nb)


def test_config1_chain_observables_vs_transfer_matrix(B, golden):
    inst = instances.config1()
    ref = golden["ferro8x8_b044"]
    env = B.Env.from_instance(inst)
    a, state, sp, E = _chain_trace(B, env, 1, 10000, seed=0, precision="f64")
    keep = state[0] >= 0
    st = state[0][keep]
    n = inst.Lx * inst.Ly
    e = E.cpu().numpy()[st] / n
    m = np.abs(sp.view(10000, -1).double().mean(dim=1).cpu().numpy())[st]
    em, es = _batch_means(e[100:], 20)
    mm, ms = _batch_means(m[100:], 20)
    print("8x8: <E>/n %.5f +- %.5f (exact %.5f); <|m|> %.5f +- %.5f (exact %.5f); acceptance %.4f"
          % (em, es, ref["E_per_spin"], mm, ms, ref["abs_m"], a.mean()))
    assert abs(em - ref["E_per_spin"]) < 3 * es
    assert abs(mm - ref["abs_m"]) < 3 * ms


def test_chi1_acceptance_vs_exact_stationary_value(B):
    inst = instances.random_small(4, 4, 0.9, 1, seed=31)
    S, _, pi, _ = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    oenv = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, 1)
    q = np.exp(tnmc.logq(oenv, S)[1])
    a_exact = exact.independence_acceptance(pi, q)
    env = B.Env.from_instance(inst)
    # an independence sampler with a poor q leaves a random start slowly (states with a
    # large pi / q hold it), so the chains are long and the first 256 steps are dropped
    C, T, burn = 256, 2048, 256
    a, _, _, _ = _chain_trace(B, env, C, T, seed=5, precision="f64")
    per_chain = a[:, burn:].mean(axis=1)
    am, sd = per_chain.mean(), per_chain.std(ddof=1) / math.sqrt(C)
    print("4x4 chi=1: acceptance %.4f +- %.4f, exact %.4f" % (am, sd, a_exact))
    assert a_exact < 0.95                       # q is far from pi: the test has teeth
    assert abs(am - a_exact) < 3 * sd


def _acceptance(B, env, C, T, seed, precision):
    a, _, _, _ = _chain_trace(B, env, C, T, seed, precision)
    return a[:, 4:].mean()


@pytest.mark.parametrize("case", ["strip_chi64", "pm16_chi4"])
def test_low_precision_acceptance_within_one_percent_of_fp64(B, case):
    if case == "strip_chi64":
        inst = instances.config5_strip(16)
        C, T, precs = 64, 64, ("f32", "bf16")
    else:
        # +-J glass at chi = 4: q visibly away from pi (acceptance ~0.95)
        inst = instances.ea_pm(16, 16, 1.0, 4, seed=7)
        C, T, precs = 1024, 256, ("f32", "bf16")
    env = B.Env.from_instance(inst, precisions=("f64",) + precs)
    a64 = _acceptance(B, env, C, T, 11, "f64")
    if case == "pm16_chi4":
        assert a64 < 0.99
    for p in precs:
        ap = _acceptance(B, env, C, T, 11, p)
        print("%s: acceptance f64 %.5f, %s %.5f (rel diff %.4f)" % (case, a64, p, ap, abs(ap - a64) / a64))
        assert abs(ap - a64) <= 0.01 * a64
    env.free()
