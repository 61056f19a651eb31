"""The MH decision u < exp(min(0, Delta)) at its edges, through tnmc_mh_step (needs a GB300).

The scan decides most proposals with two integer compares against a band precomputed
around the threshold weight, and the rest with the FP64 rule (which itself skips the FP64
exp in certain cases and behind an FP32 exp with a guard band). Here every chain gets one proposal whose Delta sits a chosen distance from
log u, where u is the chain's own MH uniform (computed by the oracle's Philox): the
decisions must equal the oracle's rule, evaluated with the FP64 exp, proposal by proposal.
The distances cover both sides of the guard band, tiny ones (exp rounding) being avoided.
"""
import numpy as np
import pytest

from oracle import philox, tnmc
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


@pytest.mark.parametrize("offset,reps", [(0.0, 256), (1e5, 256), (-3e4, 256), (0.0, 2300)])
def test_mh_decisions_at_the_edges_match_the_fp64_rule(B, offset, reps):
    """offset shifts both states' weights a = -beta E - log q by the same amount (the scan's
    integer bands scale their margin 1e-12 (1 + |theta|) with it); reps = 2300 gives more
    than 65536 chains, the thread-per-chain form of the scan."""
    inst = instances.ferromagnet(2, 3, 0.5, 2)
    env = B.Env.from_instance(inst)
    m = 1e-12 * (1.0 + abs(offset))
    deltas = np.array([-0.5, -1e-2, -1e-4, -2e-5, -1e-5, -5e-6, -2e-6, -1e-6, -1e-8, -1e-11, -1e-13,
                       1e-13, 1e-11, 1e-8, 1e-6, 2e-6, 5e-6, 1e-5, 2e-5, 1e-4, 1e-2, 0.5]
                      + [k * m for k in (-3.0, -1.5, -1.2, -0.5, 0.5, 1.2, 1.5, 3.0)])
    C = deltas.size * reps
    seed, off = 11, 3
    u = philox.mh_uniform(seed, np.uint64(off), np.arange(C))          # T = 1: step offset + 0
    d = np.log(np.maximum(u, 1e-300)) + np.repeat(deltas, reps)           # Delta = log u + delta
    d = np.concatenate([d, [-50.0, -45.0, 0.0, 3.0]])                     # far below, zero, positive
    C = d.size
    u = philox.mh_uniform(seed, np.uint64(off), np.arange(C))
    # chain: lq = 0, E = -offset / beta (a = offset); proposal: E = 0, lq = -(offset + Delta)
    E_cur = np.full(C, -offset / inst.beta)
    lq_prop = -(offset + d)
    dev = torch.device("cuda")
    prop = (torch.ones((C, inst.Ly, inst.Lx), dtype=torch.int8, device=dev),
            torch.from_numpy(lq_prop).to(dev), torch.zeros(C, dtype=torch.float64, device=dev))
    chain = (-torch.ones((C, inst.Ly, inst.Lx), dtype=torch.int8, device=dev),
             torch.zeros(C, dtype=torch.float64, device=dev), torch.from_numpy(E_cur).to(dev))
    acc = B.mh_step(env, C, 1, prop, chain, seed=seed, step_offset=off).cpu().numpy().astype(bool)
    ref = tnmc.mh_accept(inst.beta, lq_prop, np.zeros(C), np.zeros(C), E_cur, u)
    assert np.array_equal(acc, ref), np.nonzero(acc != ref)[0][:10]
    # both sides occur, and the band around the threshold is exercised
    assert acc.any() and (~acc).any()
    # the chains that accepted carry the proposal's log q and energy, the others their own
    np.testing.assert_array_equal(chain[1].cpu().numpy(), np.where(ref, lq_prop, 0.0))
    np.testing.assert_array_equal(chain[2].cpu().numpy(), np.where(ref, 0.0, E_cur))
