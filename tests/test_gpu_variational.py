"""The two-site variational builder (tnmc_build_env_variational, App. A) through the C ABI
(needs a GB300).

- Builder: log Z~, log-scales, singular-value record and bond dims against the oracle's
  build_env_variational.
- Samplers on it: FP64 draws equal to the oracle's (from its own build) but at a CDF
  edge, log q within 1e-9; FP32 and BF16 log q within 1e-4 relative of the oracle's
  forced evaluation (on the BF16-rounded tensors for BF16).
- Exact chi: q = pi, so MH accepts every proposal.
- At equal chi the variational and successive-SVD environments are different valid
  proposals; their GPU chain acceptances are reported side by side.
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


CASES = [(instances.random_small(6, 7, 0.9, 2, seed=1), 2), (instances.ea_pm(8, 9, 1.0, 4, seed=2), 1),
         (instances.ea_gauss(7, 10, 1.5, 3, seed=3, hscale=0.4), 3), (instances.random_small(9, 2, 0.8, 1, seed=5), 2),
         (instances.ea_gauss(6, 40, 1.2, 8, seed=8, hscale=0.3), 2)]


@pytest.mark.parametrize("idx", range(len(CASES)))
def test_variational_builder_and_fp64_sampler(B, idx):
    inst, sweeps = CASES[idx]
    ref = tnmc.build_env_variational(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi, sweeps=sweeps)
    env = B.Env.from_instance(inst, precisions=("f64", "f32", "bf16"), sweeps=sweeps)
    assert env.status() == 0
    ex = env.export()
    assert ex["logZ"] == pytest.approx(ref.logZ, rel=1e-10, abs=1e-10)
    np.testing.assert_allclose(ex["log_scale"], ref.log_scale, rtol=1e-10, atol=1e-9)
    for (r, c), sv in ref.sv.items():
        np.testing.assert_allclose(ex["sv"][r, c, :sv.size], sv, atol=1e-9)
        assert ex["discarded"][r, c] == pytest.approx(ref.discarded[(r, c)], abs=1e-12)
    for r in range(inst.Ly):
        for c in range(inst.Lx + 1):
            assert ex["bond_dims"][r, c] == (ref.M[r][c].shape[0] if c < inst.Lx else 1)
    n = 301
    sp, lq, E, fl = B.sample(env, n, seed=7, sample_offset=3)
    torch.cuda.synchronize()
    osp, olq, oE, _ = tnmc.sample(ref, n, seed=7, sample_offset=3)
    sp = sp.cpu().numpy()
    same = np.all(sp.reshape(n, -1) == osp.reshape(n, -1), axis=1)
    assert same.mean() >= 0.98
    for b in np.nonzero(~same)[0]:
        site = int(np.argmax(osp[b].reshape(-1) != sp[b].reshape(-1)))
        x = philox.draw_words(7, site, np.array([3 + b], dtype=np.uint64))[0]
        r, c = divmod(site, inst.Lx)
        wraw = tnmc.run(ref, 1, forced=osp[b:b + 1], keep=True)[4][r][3][0, c]
        w = np.maximum(wraw, 0.0)
        assert abs(float(x) / 2.0 ** 64 - w[1] / w.sum()) < 1e-6, (b, site)
    np.testing.assert_allclose(lq.cpu().numpy()[same], olq[same], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(E.cpu().numpy()[same], oE[same], rtol=1e-12, atol=1e-12)
    for prec, oref in (("f32", ref), ("bf16", tnmc.env_bf16(ref))):
        sp2, lq2, E2, fl2 = B.sample(env, 200, seed=9, precision=prec)
        torch.cuda.synchronize()
        _, olq2, oE2, ofl2 = tnmc.logq(oref, sp2.cpu().numpy())
        assert np.all(fl2.cpu().numpy() == 0) and np.all(ofl2 == 0)
        np.testing.assert_allclose(lq2.cpu().numpy(), olq2, rtol=1e-4)


def test_variational_exact_chi_accepts_everything(B):
    inst = instances.ea_gauss(4, 4, 1.0, 4, seed=4, hscale=0.3)
    env = B.Env.from_instance(inst, sweeps=2)
    C, T = 64, 32
    prop = B.sample(env, C * T, seed=2)[:3]
    chain = B.init_chains(env, C, seed=2)
    acc = B.mh_step(env, C, T, prop, chain, seed=3)
    assert acc.float().mean().item() > 0.999


def test_variational_rejects_the_bond_basis(B):
    inst = instances.ea_gauss(4, 4, 1.0, 2, seed=4)
    with pytest.raises(Exception):
        B.Env.from_instance(inst, gauge="bond", sweeps=1)


@pytest.mark.parametrize("inst", [instances.ea_pm(16, 16, 1.0, 2, seed=7), instances.villain(16, 16, 1.5, 2),
                                  instances.ea_gauss(16, 16, 2.0, 4, seed=9, hscale=0.2)])
def test_variational_and_svd_acceptance_at_equal_chi(B, inst):
    acc = {}
    for sweeps in (0, 2):
        env = B.Env.from_instance(inst, sweeps=sweeps)
        C, T = 256, 256
        prop = B.sample(env, C * T, seed=5)[:3]
        chain = B.init_chains(env, C, seed=6)
        acc[sweeps] = B.mh_step(env, C, T, prop, chain, seed=7).view(C, T)[:, 16:].float().mean().item()
    print("%s %dx%d chi=%d: acceptance successive SVD %.4f, variational (2 sweeps) %.4f"
          % (inst.name, inst.Ly, inst.Lx, inst.chi, acc[0], acc[2]))
    assert 0.0 < acc[0] < 1.0 and 0.0 < acc[2] < 1.0
