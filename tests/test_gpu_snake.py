"""Snake site order through the C ABI (tnmc_env_set_order; needs a GB300).

- FP64: draws equal to the oracle's snake-order draws but at a CDF edge, log q within
  1e-9, energies to rounding; forced evaluation equals sampling bit for bit.
- FP32: log q within 1e-4 relative of the oracle's forced evaluation.
- The batched plan of snake-order envs equals the single-instance calls.
- Exact chi: MH accepts every proposal.  BF16 and the backward reject snake order.
"""
import numpy as np
import pytest

from oracle import tnmc
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


CASES = [instances.random_small(6, 7, 0.9, 2, seed=1), instances.ea_pm(9, 11, 1.0, 4, seed=2),
         instances.ea_gauss(7, 20, 1.5, 8, seed=3, hscale=0.4), instances.random_small(5, 1, 0.8, 2, seed=5),
         instances.ferromagnet(12, 40, 0.4407, 16, hfield=0.05)]


def _oracle(inst):
    env = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    env.order = "snake"
    return env


@pytest.mark.parametrize("idx", range(len(CASES)))
def test_snake_fp64_and_fp32_match_oracle(B, idx):
    inst = CASES[idx]
    ref = _oracle(inst)
    env = B.Env.from_instance(inst, precisions=("f64", "f32")).set_order("snake")
    n = 301
    sp, lq, E, fl = B.sample(env, n, seed=7, sample_offset=3)
    torch.cuda.synchronize()
    osp, olq, oE, _ = tnmc.sample(ref, n, seed=7, sample_offset=3)
    sp_h = sp.cpu().numpy()
    same = np.all(sp_h.reshape(n, -1) == osp.reshape(n, -1), axis=1)
    assert same.mean() >= 0.98
    np.testing.assert_allclose(lq.cpu().numpy()[same], olq[same], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(E.cpu().numpy(), tnmc.energy(inst.Jh, inst.Jv, inst.h, sp_h), rtol=1e-12, atol=1e-12)
    if not same.all():
        np.testing.assert_allclose(lq.cpu().numpy()[~same], tnmc.logq(ref, sp_h[~same])[1], rtol=1e-9, atol=1e-9)
    lq2, E2, _ = B.logq(env, sp)
    torch.cuda.synchronize()
    assert torch.equal(lq, lq2) and torch.equal(E, E2)
    sp3, lq3, _, fl3 = B.sample(env, 200, seed=9, precision="f32")
    torch.cuda.synchronize()
    _, olq3, _, _ = tnmc.logq(ref, sp3.cpu().numpy())
    np.testing.assert_allclose(lq3.cpu().numpy(), olq3, rtol=1e-4)


def test_snake_batched_equals_single(B):
    from paper_2104_13264_gb300 import batched
    insts = [instances.ea_gauss(8, 8, 2.0, 4, seed=k) for k in range(3)] + [instances.ea_gauss(6, 10, 2.0, 8, seed=9)]
    envs = B.build_envs_batched(insts, precisions=("f64",))
    for e in envs:
        e.set_order("snake")
    run = batched.BatchRunner(envs, 64, chains=8, precision="f64", tile=64, order="cost", tune=False, seed=4)
    run.plan.set_step(4, 0)
    prop = run.plan.alloc_proposals()
    run.plan.sample(prop)
    torch.cuda.synchronize()
    for i, (e, inst) in enumerate(zip(envs, insts)):
        sp, lq, E, fl = B.sample(e, 64, seed=4, sample_offset=(i << 40))
        torch.cuda.synchronize()
        assert torch.equal(run.plan.view(prop[0], i), sp)
        assert torch.equal(run.plan.rows(prop[1], i), lq)


def test_snake_exact_chi_accepts_everything_and_unsupported_paths(B):
    inst = instances.ea_gauss(4, 4, 1.0, 4, seed=4, hscale=0.3)
    env = B.Env.from_instance(inst, precisions=("f64", "f32", "bf16")).set_order("snake")
    C, T = 64, 32
    prop = B.sample(env, C * T, seed=2)[:3]
    chain = B.init_chains(env, C, seed=2)
    acc = B.mh_step(env, C, T, prop, chain, seed=3)
    assert acc.float().mean().item() > 0.999
    with pytest.raises(B.TnmcError):
        B.sample(env, 16, precision="bf16")
    with pytest.raises(B.TnmcError):
        B.logq_backward(env, prop[0][:8], torch.ones(8, device="cuda"))
