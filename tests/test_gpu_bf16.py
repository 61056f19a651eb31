"""BF16 tensor-core sampler (tcgen05) vs the oracle through the C-ABI (needs a GB300).

The BF16 path contracts BF16 hi + lo pairs of both operands (environment and
vectors) on the tensor cores with FP32 accumulation.  Its q is the q of the
environment rounded to those pairs: the oracle replaces its own FP64 tensors by
their hi + lo pairs (oracle.tnmc.env_bf16) and evaluates the GPU's draws in FP64.
Bar: log q within 1e-4 relative; energies exact for integer couplings, FP64 otherwise.
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


CASES = [
    instances.random_small(6, 20, 0.9, 16, seed=1),     # 3 segments of the left sweep, ragged
    instances.ea_pm(16, 16, 1.0, 16, seed=2),
    instances.config1(),                                 # Lx < checkpoint stride
    instances.random_small(9, 1, 0.8, 2, seed=5),       # one column: no right sweep
    instances.random_small(1, 9, 0.8, 2, seed=6),       # one row
    instances.random_small(5, 23, 0.8, 8, seed=3),      # last segment of length 7
    instances.random_small(4, 17, 0.8, 8, seed=8),      # last segment of length 1
    instances.ferromagnet(12, 48, 0.4407, 16),
    instances.villain(8, 24, 1.5, 32),
]


@pytest.mark.parametrize("idx", range(len(CASES)))
def test_bf16_logq_vs_oracle(B, idx):
    inst = CASES[idx]
    ref = tnmc.env_bf16(tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi))
    env = B.Env.from_instance(inst, precisions=("f64", "bf16"))
    n = 333
    sp, lq, E, fl = B.sample(env, n, seed=3 + idx, sample_offset=11, precision="bf16")
    lq2, E2, fl2 = B.logq(env, sp, precision="bf16")
    torch.cuda.synchronize()
    assert torch.equal(lq, lq2) and torch.equal(E, E2) and torch.equal(fl, fl2)   # forced == sampled
    spn = sp.cpu().numpy()
    assert set(np.unique(spn)) <= {-1, 1}
    _, olq, oE, ofl = tnmc.logq(ref, spn)
    assert np.all(fl.cpu().numpy() == 0) and np.all(ofl == 0)
    np.testing.assert_allclose(lq.cpu().numpy(), olq, rtol=1e-4)
    if inst.integer_couplings:
        assert np.array_equal(E.cpu().numpy(), oE)
    else:
        # FP64 sums in another order than the oracle's
        np.testing.assert_allclose(E.cpu().numpy(), oE, rtol=1e-12, atol=1e-12)


def test_bf16_draws_follow_q(B):
    """Chi^2 of BF16 draw frequencies against the BF16 q itself (3x3, all 512 states)."""
    from scipy import stats

    from oracle import exact
    inst = instances.random_small(3, 3, 0.8, 2, seed=5)
    env = B.Env.from_instance(inst, precisions=("f64", "bf16"))
    n = 1 << 20
    sp, lq, _, _ = B.sample(env, n, seed=21, precision="bf16")
    bits = ((sp.view(n, 9) > 0).long() << torch.arange(9, device="cuda")).sum(dim=1)
    counts = torch.bincount(bits, minlength=512).cpu().numpy()
    S = torch.from_numpy(exact.all_states(3, 3)).cuda()
    lq_all = B.logq(env, S, precision="bf16")[0].cpu().numpy()
    assert abs(np.exp(lq_all).sum() - 1) < 1e-5
    e = n * np.exp(lq_all)
    chi2 = ((counts - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi2, 511) > 1e-4


def test_bf16_shards_bit_exact(B):
    inst = instances.random_small(5, 19, 0.8, 8, seed=9)
    env = B.Env.from_instance(inst, precisions=("f64", "bf16"))
    full = B.sample(env, 700, seed=5, precision="bf16")
    a = B.sample(env, 300, seed=5, sample_offset=0, precision="bf16")
    b = B.sample(env, 400, seed=5, sample_offset=300, precision="bf16")
    for x, y, z in zip(full, a, b):
        assert torch.equal(x, torch.cat([y, z]))


def test_bf16_exact_chi_acceptance(B):
    """Exact chi: q equals pi up to the hi + lo rounding of the operands (~2^-16), so
    the MH acceptance is 1 to within a per-mille."""
    inst = instances.ea_gauss(4, 4, 1.0, 4, seed=4, hscale=0.3)
    env = B.Env.from_instance(inst, precisions=("f64", "bf16"))
    C, T = 64, 64
    prop = B.sample(env, C * T, seed=2, precision="bf16")[:3]
    chain = B.init_chains(env, C, seed=2, precision="bf16")
    acc = B.mh_step(env, C, T, prop, chain, seed=3)
    assert acc.float().mean().item() > 0.999


def test_bf16_wait_timeout_is_reported_and_context_survives(B, monkeypatch):
    """The tensor-core sampler's mbarrier waits are bounded.  With the in-loop poll limit
    set to 0 (test hook) every such wait gives up at once: the call must return, the env's
    status word must read TNMC_E_TIMEOUT, the kernel must have drained its copies and freed
    its TMEM, and a following normal call must still match the oracle."""
    inst = instances.random_small(4, 9, 0.8, 4, seed=2)
    ref = tnmc.env_bf16(tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi))
    env = B.Env.from_instance(inst, precisions=("f64", "bf16"))
    assert env.status() == 0
    monkeypatch.setenv("TNMC_DEBUG_POLL_LIMIT", "0")
    B.sample(env, 300, seed=1, precision="bf16")
    torch.cuda.synchronize()
    monkeypatch.delenv("TNMC_DEBUG_POLL_LIMIT")
    assert env.status() == 5                      # TNMC_E_TIMEOUT (kept: the first error)
    for _ in range(2):                            # TMEM was freed: further launches allocate it
        sp, lq, E, fl = B.sample(env, 300, seed=4, precision="bf16")
        torch.cuda.synchronize()
        _, olq, oE, ofl = tnmc.logq(ref, sp.cpu().numpy())
        assert np.all(fl.cpu().numpy() == 0)
        np.testing.assert_allclose(lq.cpu().numpy(), olq, rtol=1e-4)


def test_bf16_wide_lattice_vs_oracle(B):
    """A 448-column lattice (14 spin-bit words per sample, the right stack 447 deep)."""
    inst = instances.ea_pm(3, 448, 1.0, 8, seed=4)
    ref = tnmc.env_bf16(tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi))
    env = B.Env.from_instance(inst, precisions=("f64", "bf16"))
    sp, lq, E, fl = B.sample(env, 333, seed=3, sample_offset=11, precision="bf16")
    lq2, E2, fl2 = B.logq(env, sp, precision="bf16")
    torch.cuda.synchronize()
    assert torch.equal(lq, lq2) and torch.equal(E, E2) and torch.equal(fl, fl2)
    _, olq, oE, ofl = tnmc.logq(ref, sp.cpu().numpy())
    assert np.all(fl.cpu().numpy() == 0) and np.all(ofl == 0)
    np.testing.assert_allclose(lq.cpu().numpy(), olq, rtol=1e-4)
    assert np.array_equal(E.cpu().numpy(), oE)
