"""Three-dimensional TNMH through the C ABI (Sec. 3D; App. A; needs a GB300).

- Builder: the per-layer log-scales and the bond dims of the compressed layer PEPS
  against the oracle's build_env3d (both are invariant under the orthogonal bond gauges
  in which the two QR routines may differ).
- FP64 sampler: draws equal to the oracle's (from its own build) but at a CDF edge, log q
  within 1e-9, energies to rounding; a sample that differs is checked to be a valid draw
  (its forced log q matches the oracle's).
- FP32 sampler: forced log q of its draws within 1e-5 relative of the oracle's.
- Forced evaluation equals sampling, bit for bit, in both precisions.
- Exact (D, chi): q = pi, so MH accepts every proposal; the MH scan equals the oracle's.
"""
import numpy as np
import pytest

from oracle import peps3d, tnmc
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


CASES = [instances.cubic_random(3, 4, 5, 0.6, 2, 3, seed=1), instances.cubic_random(2, 5, 3, 0.8, 3, 4, seed=2),
         instances.cubic_random(4, 3, 3, 0.5, 2, 2, seed=3, hscale=0.5), instances.cubic_random(2, 1, 7, 0.9, 2, 2, seed=4),
         instances.cubic_random(3, 6, 1, 0.7, 2, 3, seed=5), instances.cubic_random(3, 3, 4, 0.4, 4, 8, seed=6)]


def _oracle_env(inst):
    return peps3d.build_env3d(inst.Jx, inst.Jy, inst.Jz, inst.h, inst.beta, inst.D, inst.chi)


@pytest.mark.parametrize("idx", range(len(CASES)))
def test_builder_matches_oracle(B, idx):
    inst = CASES[idx]
    ref = _oracle_env(inst)
    env = B.Env3D.from_instance(inst)
    assert env.status() == 0
    ex = env.export()
    np.testing.assert_allclose(ex["log_scale"], ref.log_scale, rtol=1e-10, atol=1e-9)
    for z in range(inst.shape[0]):
        for y in range(inst.shape[1]):
            for x in range(inst.shape[2]):
                assert tuple(ex["dims"][z, y, x]) == ref.A[z][y][x].shape[1:], (z, y, x)


@pytest.mark.parametrize("idx", range(len(CASES)))
def test_fp64_sampler_matches_oracle(B, idx):
    inst = CASES[idx]
    ref = _oracle_env(inst)
    env = B.Env3D.from_instance(inst)
    n = 301
    sp, lq, E, fl = B.sample3d(env, n, seed=7, sample_offset=5)
    torch.cuda.synchronize()
    osp, olq, oE, ofl = peps3d.sample3d(ref, n, seed=7, sample_offset=5)
    sp_h = sp.cpu().numpy()
    assert np.all(fl.cpu().numpy() == 0) and np.all(ofl == 0)
    same = np.all(sp_h.reshape(n, -1) == osp.reshape(n, -1), axis=1)
    assert same.mean() >= 0.98, same.mean()
    np.testing.assert_allclose(lq.cpu().numpy()[same], olq[same], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(E.cpu().numpy(), peps3d.energy3d(inst.Jx, inst.Jy, inst.Jz, inst.h, sp_h), rtol=1e-12,
                               atol=1e-12)
    if not same.all():
        _, olq_d, _, _ = peps3d.logq3d(ref, sp_h[~same])
        np.testing.assert_allclose(lq.cpu().numpy()[~same], olq_d, rtol=1e-9, atol=1e-9)
    # forced evaluation of the draws reproduces the sampled log q bit for bit
    lq2, E2, _ = B.logq3d(env, sp)
    torch.cuda.synchronize()
    assert torch.equal(lq, lq2) and torch.equal(E, E2)


@pytest.mark.parametrize("idx", [0, 2, 5])
def test_fp32_sampler_vs_oracle(B, idx):
    inst = CASES[idx]
    ref = _oracle_env(inst)
    env = B.Env3D.from_instance(inst)
    sp, lq, E, fl = B.sample3d(env, 256, seed=9, precision="f32")
    lq2, _, _ = B.logq3d(env, sp, precision="f32")
    torch.cuda.synchronize()
    assert torch.equal(lq, lq2)
    assert np.all(fl.cpu().numpy() == 0)
    _, olq, _, ofl = peps3d.logq3d(ref, sp.cpu().numpy())
    assert np.all(ofl == 0)
    err = np.abs(lq.cpu().numpy() - olq) / np.abs(olq)
    print("3D FP32 log q: max relative error %.2e" % err.max())
    assert err.max() < 1e-5


def test_exact_bonds_accept_everything_and_mh_matches_oracle(B):
    inst = instances.cubic_random(2, 3, 2, 0.6, 8, 8, seed=4)
    env = B.Env3D.from_instance(inst)
    C, T = 64, 16
    prop = B.sample3d(env, C * T, seed=2)[:3]
    chain = B.init_chains3d(env, C, seed=3)
    start = [c.clone() for c in chain]
    acc = B.mh_step3d(env, C, T, prop, chain, seed=4)
    torch.cuda.synchronize()
    assert acc.float().mean().item() > 0.999
    ps, plq, pE = (t.cpu().numpy() for t in prop)
    cs, clq, cE = (t.cpu().numpy() for t in start)
    n = inst.h.size
    ref = tnmc.mh_scan(inst.beta, C, T, ps.reshape(C * T, 1, n), plq, pE, cs.reshape(C, 1, n), clq, cE, seed=4)
    np.testing.assert_array_equal(acc.cpu().numpy().astype(bool), ref[0])
    np.testing.assert_array_equal(chain[0].cpu().numpy().reshape(C, 1, n), ref[1])


def test_truncated_instance_acceptance_is_below_one(B):
    inst = instances.cubic_random(3, 3, 3, 1.2, 1, 1, seed=8)
    env = B.Env3D.from_instance(inst)
    C, T = 128, 32
    prop = B.sample3d(env, C * T, seed=2)[:3]
    chain = B.init_chains3d(env, C, seed=3)
    acc = B.mh_step3d(env, C, T, prop, chain, seed=4).view(C, T)[:, 8:].float().mean().item()
    assert 0.0 < acc < 0.999


# ---- the bond basis (tnmc3d_build_env_bond) ----

BOND_CASES = [instances.cubic_random(3, 4, 5, 0.6, 2, 3, seed=1), instances.cubic_random(2, 5, 3, 0.8, 2, 4, seed=2),
              instances.cubic_random(4, 3, 3, 0.5, 1, 2, seed=3, hscale=0.5), instances.cubic_random(3, 3, 4, 0.4, 4, 8, seed=6)]


@pytest.mark.parametrize("idx", range(len(BOND_CASES)))
def test_bond_basis_matches_oracle(B, idx):
    inst = BOND_CASES[idx]
    ref = peps3d.build_env3d_bond(inst.Jx, inst.Jy, inst.Jz, inst.h, inst.beta, inst.D, inst.chi)
    env = B.Env3D.from_instance(inst, gauge="bond")
    assert env.status() == 0
    ex = env.export()
    for z in range(inst.shape[0]):
        for y in range(inst.shape[1]):
            for x in range(inst.shape[2]):
                assert tuple(ex["dims"][z, y, x]) == ref.A[z][y][x].shape[1:], (z, y, x)
    n = 301
    sp, lq, E, fl = B.sample3d(env, n, seed=7, sample_offset=5)
    torch.cuda.synchronize()
    osp, olq, _, ofl = peps3d.sample3d(ref, n, seed=7, sample_offset=5)
    sp_h = sp.cpu().numpy()
    assert np.all(fl.cpu().numpy() == 0) and np.all(ofl == 0)
    same = np.all(sp_h.reshape(n, -1) == osp.reshape(n, -1), axis=1)
    assert same.mean() >= 0.98, same.mean()
    np.testing.assert_allclose(lq.cpu().numpy()[same], olq[same], rtol=1e-9, atol=1e-9)
    if not same.all():
        np.testing.assert_allclose(lq.cpu().numpy()[~same], peps3d.logq3d(ref, sp_h[~same])[1], rtol=1e-9, atol=1e-9)
    sp2, lq2, _, _ = B.sample3d(env, 200, seed=9, precision="f32")
    torch.cuda.synchronize()
    olq2 = peps3d.logq3d(ref, sp2.cpu().numpy())[1]
    err = np.abs(lq2.cpu().numpy() - olq2) / np.abs(olq2)
    print("3D bond basis FP32 log q: max relative error %.2e" % err.max())
    assert err.max() < 1e-5


def test_bond_basis_exact_bonds_accept_everything(B):
    inst = instances.cubic_random(2, 3, 2, 0.6, 8, 4, seed=4)
    env = B.Env3D.from_instance(inst, gauge="bond")
    C, T = 64, 16
    prop = B.sample3d(env, C * T, seed=2)[:3]
    chain = B.init_chains3d(env, C, seed=3)
    acc = B.mh_step3d(env, C, T, prop, chain, seed=4)
    assert acc.float().mean().item() > 0.999


@pytest.mark.parametrize("gauge,D,chi", [("spin", 2, 2), ("bond", 1, 1)])
def test_3d_chain_energy_matches_enumeration(B, gauge, D, chi):
    """MH with truncated 3D proposals is exact: the chains' mean energy agrees with the
    Boltzmann average (enumeration of the 2^18 states) within 3 sigma (batch means).  The
    truncations keep max pi/q small (1.5 and 7.9 here), so the independence chains mix
    within the run; the spin basis at (1, 1) has max pi/q = 8e9 on this instance and its
    chains stay near <E>_q for any feasible run length."""
    inst = instances.cubic_random(2, 3, 3, 0.7, D, chi, seed=12, hscale=0.4)
    S = (2 * ((np.arange(2 ** 18)[:, None] >> np.arange(18)[None]) & 1) - 1).reshape(-1, 2, 3, 3).astype(np.int8)
    Eall = peps3d.energy3d(inst.Jx, inst.Jy, inst.Jz, inst.h, S)
    a = -inst.beta * Eall
    w = np.exp(a - a.max())
    exact_E = float((w * Eall).sum() / w.sum())
    env = B.Env3D.from_instance(inst, gauge=gauge)
    C, T, steps, burn = 256, 4, 40, 10
    chain = B.init_chains3d(env, C, seed=5)
    means, acc = [], []
    for k in range(steps):
        prop = B.sample3d(env, C * T, seed=9, sample_offset=k * C * T)[:3]
        acc.append(B.mh_step3d(env, C, T, prop, chain, seed=10, step_offset=k * T).float().mean().item())
        if k >= burn:
            means.append(chain[2].cpu().numpy())
    per_chain = np.mean(np.array(means), axis=0)          # time average of each chain
    est = float(per_chain.mean())
    err = float(per_chain.std(ddof=1) / np.sqrt(C))
    print("3D %s chains: <E> %.4f +- %.4f, exact %.4f, acceptance %.3f" % (gauge, est, err, exact_E, np.mean(acc)))
    assert 0.0 < np.mean(acc) < 1.0
    assert abs(est - exact_E) < 3 * err + 1e-9
