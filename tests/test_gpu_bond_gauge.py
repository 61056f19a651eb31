"""The bond-basis gauge builder (tnmc_build_env_bond, App. A) through the C ABI (needs a GB300).

- Builder: log Z~, the log-scales and the singular-value record of the truncated
  bond-basis boundary MPS against the oracle's build_env_bond.
- Samplers on it: FP64 draws equal to the oracle's (from its own build) but at a CDF
  edge, log q within 1e-9 relative; FP32 and BF16 log q within 1e-4 relative of the
  oracle's forced evaluation (on the BF16-rounded tensors for BF16).
- Exact chi: q = pi, so MH accepts every proposal.
- At equal truncation chi the bond gauge (sampled from 2 chi bonds) and the spin basis
  are different valid proposals; their GPU chain acceptances are reported side by side.
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


CASES = [instances.random_small(6, 7, 0.9, 2, seed=1), instances.ea_pm(8, 9, 1.0, 4, seed=2),
         instances.ferromagnet(10, 12, 0.4407, 8), instances.ea_gauss(7, 5, 1.5, 3, seed=3, hscale=0.4),
         instances.random_small(9, 1, 0.8, 2, seed=5), instances.random_small(1, 9, 0.8, 2, seed=6)]


@pytest.mark.parametrize("idx", range(len(CASES)))
def test_bond_gauge_builder_and_fp64_sampler(B, idx):
    inst = CASES[idx]
    ref = tnmc.build_env_bond(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    env = B.Env.from_instance(inst, precisions=("f64", "f32", "bf16"), gauge="bond")
    assert env.status() == 0
    ex = env.export()
    assert ex["logZ"] == pytest.approx(ref.logZ, rel=1e-10, abs=1e-10)
    np.testing.assert_allclose(ex["log_scale"][1:], ref.log_scale[1:], rtol=1e-10, atol=1e-9)
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
        r, c = divmod(site, inst.Lx)
        x = philox.draw_words(7, site, np.array([3 + b], dtype=np.uint64))[0]
        assert abs(float(x) / 2.0 ** 64 - _oracle_pplus(ref, osp[b:b + 1], r, c)) < 1e-6, (b, site)
    lqn = lq.cpu().numpy()
    np.testing.assert_allclose(lqn[same], olq[same], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(E.cpu().numpy()[same], oE[same], rtol=1e-12, atol=1e-12)
    for prec, oref in (("f32", ref), ("bf16", tnmc.env_bf16(ref))):
        sp2, lq2, E2, fl2 = B.sample(env, 200, seed=9, precision=prec)
        torch.cuda.synchronize()
        _, olq2, oE2, ofl2 = tnmc.logq(oref, sp2.cpu().numpy())
        assert np.all(fl2.cpu().numpy() == 0) and np.all(ofl2 == 0)
        np.testing.assert_allclose(lq2.cpu().numpy(), olq2, rtol=1e-4)


def _oracle_pplus(env, spins, r, c):
    """Oracle conditional p_+ at (r, c) given the spins before it (FP64)."""
    f = tnmc.row_fields(env, spins, r)
    M = env.M[r]
    R = np.ones((1, 1))
    for cc in range(env.Lx - 1, c, -1):
        Y = np.einsum("asb,nb->nas", M[cc], R)
        R = Y[:, :, 0] * f[:, cc, 0:1] + Y[:, :, 1] * f[:, cc, 1:2]
        R = R / np.abs(R).max()
    Lam = np.ones((1, 1))
    for cc in range(c):
        s = int(spins[0, r, cc] > 0)
        Lam = np.einsum("na,ab->nb", Lam, M[cc][:, s, :]) * f[0, cc, s]
        Lam = Lam / np.abs(Lam).max()
    U = np.einsum("na,asb->nsb", Lam, M[c])
    w = np.maximum(np.einsum("nsb,nb->ns", U, R)[0] * f[0, c], 0)
    return w[1] / w.sum()


def test_bond_gauge_exact_chi_accepts_everything(B):
    inst = instances.ea_gauss(4, 4, 1.0, 4, seed=4, hscale=0.3)
    env = B.Env.from_instance(inst, gauge="bond")
    C, T = 64, 32
    prop = B.sample(env, C * T, seed=2)[:3]
    chain = B.init_chains(env, C, seed=2)
    acc = B.mh_step(env, C, T, prop, chain, seed=3)
    assert acc.float().mean().item() > 0.999


@pytest.mark.parametrize("inst", [instances.ea_pm(16, 16, 1.0, 2, seed=7), instances.villain(16, 16, 1.5, 2),
                                  instances.ferromagnet(16, 16, 0.4407, 2)])
def test_bond_and_spin_gauge_acceptance_at_equal_chi(B, inst):
    acc = {}
    for gauge in ("spin", "bond"):
        env = B.Env.from_instance(inst, gauge=gauge)
        C, T = 256, 256
        prop = B.sample(env, C * T, seed=5)[:3]
        chain = B.init_chains(env, C, seed=6)
        acc[gauge] = B.mh_step(env, C, T, prop, chain, seed=7).view(C, T)[:, 16:].float().mean().item()
    print("%s %dx%d chi=%d: acceptance spin %.4f, bond %.4f" % (inst.name, inst.Ly, inst.Lx, inst.chi, acc["spin"],
                                                               acc["bond"]))
    assert 0.0 < acc["spin"] < 1.0 and 0.0 < acc["bond"] < 1.0
