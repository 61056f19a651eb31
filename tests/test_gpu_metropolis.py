"""Metropolis sweeps between proposals and the Delta diagnostic through the C ABI (needs a GB300).

- tnmc_metropolis: the oracle's checkerboard sweeps from the same Philox stream, spin
  for spin (the flip rule compares a 53-bit uniform with exp in FP64 on both sides);
  energies against the oracle's; log q equal to a forced evaluation of the new states.
- tnmc_link_overlap: exact integer counts against the oracle's.
- Batched forms: per instance identical to the single-instance calls.
- The paper's chain (TNMH moves + Metropolis sweeps, Sec. 3, Table hb) on a batch of
  4 x 4 Gaussian instances: after burn-in its Delta estimate agrees, within 3 sigma, with
  the exact per-instance values averaged over the batch (enumeration in the oracle).
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


@pytest.mark.parametrize("inst", [instances.ea_gauss(12, 10, 2.0, 4, seed=3), instances.ea_pm(9, 16, 1.0, 4, seed=2),
                                  instances.random_small(5, 7, 1.2, 3, seed=4, hscale=0.5),
                                  instances.ferromagnet(1, 9, 0.7, 2)])
def test_metropolis_matches_oracle(B, inst):
    env = B.Env.from_instance(inst)
    C = 64
    cs, clq, cE = B.init_chains(env, C, seed=1)
    start = cs.cpu().numpy()
    B.metropolis(env, (cs, clq, cE), seed=11, chain_offset=5, sweep_offset=7, sweeps=3)
    torch.cuda.synchronize()
    ref = tnmc.metropolis_sweeps(inst.Jh, inst.Jv, inst.h, inst.beta, start, seed=11, sweep_offset=7, sweeps=3,
                                 chain_ids=5 + np.arange(C))
    got = cs.cpu().numpy()
    assert np.array_equal(got, ref)
    assert not np.array_equal(got, start)
    oE = tnmc.energy(inst.Jh, inst.Jv, inst.h, ref)
    np.testing.assert_allclose(cE.cpu().numpy(), oE, rtol=1e-12, atol=1e-12)
    lq2, E2, _ = B.logq(env, cs)
    torch.cuda.synchronize()
    assert torch.equal(clq, lq2) and torch.equal(cE, E2)


def test_link_overlap_matches_oracle(B):
    inst = instances.ea_gauss(11, 13, 1.0, 2, seed=5)
    env = B.Env.from_instance(inst)
    cs = B.init_chains(env, 10, seed=3)[0]
    q = B.link_overlap(env, cs).cpu().numpy()
    sp = cs.cpu().numpy()
    assert np.array_equal(q, tnmc.link_overlap(None, None, sp[0::2], sp[1::2]))


def test_batched_metropolis_equals_single(B):
    from paper_2104_13264_gb300 import batched
    insts = [instances.ea_gauss(8, 8, 2.0, 4, seed=k) for k in range(3)] + [instances.ea_gauss(6, 10, 2.0, 8, seed=9)]
    envs = B.build_envs_batched(insts, precisions=("f64",))
    C = 6
    run = batched.BatchRunner(envs, 4 * C, chains=C, precision="f64", tile=64, order="cost", tune=False,
                              seed=4, sweeps=2)
    run.plan.set_step(4, 3)
    before = [run.plan.view(run.chain[0], i, chains=True).clone() for i in range(len(insts))]
    run.plan.metropolis(run.chain, 2)
    q = run.plan.link_overlap(run.chain[0])
    torch.cuda.synchronize()
    for i, e in enumerate(envs):
        ch = (before[i].clone(), torch.empty(C, dtype=torch.float64, device="cuda"),
              torch.empty(C, dtype=torch.float64, device="cuda"))
        B.metropolis(e, ch, seed=4, chain_offset=i * C, sweep_offset=3 * 2, sweeps=2)
        torch.cuda.synchronize()
        assert torch.equal(ch[0], run.plan.view(run.chain[0], i, chains=True))
        assert torch.equal(ch[1], run.plan.rows(run.chain[1], i, chains=True))
        assert torch.equal(ch[2], run.plan.rows(run.chain[2], i, chains=True))
        assert torch.equal(q[i], B.link_overlap(e, ch[0]))


def _exact_delta(inst):
    S, _, pi, E = exact.boltzmann(inst.Jh, inst.Jv, inst.h, inst.beta)
    s = S.astype(np.float64)
    corr = np.concatenate([(pi[:, None, None] * s[:, :, :-1] * s[:, :, 1:]).sum(axis=0).ravel(),
                           (pi[:, None, None] * s[:, :-1, :] * s[:, 1:, :]).sum(axis=0).ravel()])
    return tnmc.delta_instance(inst.beta, inst.Lx, inst.Ly, float(pi @ E), float(np.sum(corr ** 2)))


def test_tnmh_plus_metropolis_reaches_the_exact_delta(B):
    from paper_2104_13264_gb300 import batched
    insts = [instances.ea_gauss(4, 4, 2.0, 2, seed=200 + k) for k in range(48)]
    envs = B.build_envs_batched(insts, precisions=("f64",))
    C = 64
    run = batched.BatchRunner(envs, 2 * C, chains=C, precision="f64", tile=64, order="cost", tune=False,
                              seed=7, sweeps=1)
    d0, _ = run.delta()
    vals = []
    for it in range(60):
        run.step_eager()
        if it >= 20:
            vals.append(run.delta()[1].cpu().numpy())
    v = np.array(vals)                            # [iterations, instances]
    exact_i = np.array([_exact_delta(i) for i in insts])
    # per-instance estimation errors are independent across instances (iterations within
    # one instance are correlated, so each instance contributes its time average)
    dev = v.mean(axis=0) - exact_i
    err = dev.std(ddof=1) / math.sqrt(dev.size)
    est, ref = float(v.mean()), float(exact_i.mean())
    print("Delta: start %.4f, chain estimate %.5f +- %.5f, exact %.5f" % (d0, est, err, ref))
    assert abs(d0 - ref) > 10 * err               # the start is far from equilibrium
    assert abs(dev.mean()) < 3 * err
