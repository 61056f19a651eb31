"""Closed lattices by frozen lines (App. B) through the C ABI (needs a GB300).

- One move of 16 chains on a 6 x 6 torus (and a 5 x 7 cylinder) against the oracle's
  frozen-line move: new spins bit for bit, the same accept decisions (FP64).
- Exactness of the chain: 3 x 4 torus, a poor q (chi = 1).  20000 exact samples of the
  closed lattice's Boltzmann law (enumeration) stay distributed as that law after 6
  random-cut moves on the GPU (chi^2 over the states).  (From a random start this q mixes
  slowly; the oracle's chains show the same distance from pi move for move.)
"""
import numpy as np
import pytest
from scipy import stats

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


@pytest.mark.parametrize("Ly,Lx,px,py", [(6, 6, True, True), (5, 7, True, False)])
def test_frozen_line_move_matches_oracle(B, Ly, Lx, px, py):
    from paper_2104_13264_gb300 import frozen
    r = np.random.default_rng([Ly, Lx])
    Jh, Jv, h = r.standard_normal((Ly, Lx)), r.standard_normal((Ly, Lx)), 0.3 * r.standard_normal((Ly, Lx))
    beta, chi, C, T = 1.2, 4, 16, 3
    start = r.choice([-1, 1], size=(C, Ly, Lx)).astype(np.int8)
    ch = frozen.FrozenLineChains(Jh, Jv, h, beta, chi, start, px=px, py=py, precision="f64", proposals=T, seed=5)
    ref = start
    for k, cut in enumerate([(2, 3), (0, Lx - 1)]):
        acc = ch.step(cut).cpu().numpy().astype(bool)
        ref, oacc = tnmc.frozen_line_step(Jh, Jv, h, beta, chi, ref, cut[0], cut[1], px, py, seed=5, step=k, T=T)
        assert np.array_equal(acc[0], oacc)
        assert np.array_equal(ch.spins[0].cpu().numpy(), ref)
    E = ch.energy()[0].cpu().numpy()
    np.testing.assert_allclose(E, tnmc.energy_periodic(Jh, Jv, h, ref, px, py), rtol=1e-12, atol=1e-12)


def test_several_disorders_in_one_move(B):
    """Three disorder samples of a 5 x 5 torus, 4 chains each, in one batched move: each
    disorder's chains equal the oracle's move with the plan's instance numbering."""
    from paper_2104_13264_gb300 import frozen
    r = np.random.default_rng(7)
    D, C, L, T = 3, 4, 5, 2
    Jh, Jv, h = r.standard_normal((D, L, L)), r.standard_normal((D, L, L)), np.zeros((D, L, L))
    start = r.choice([-1, 1], size=(D, C, L, L)).astype(np.int8)
    ch = frozen.FrozenLineChains(Jh, Jv, h, [1.0, 1.5, 2.0], 4, start, proposals=T, seed=3)
    acc = ch.step((3, 1)).cpu().numpy().astype(bool)
    for d in range(D):
        ref, oacc = tnmc.frozen_line_step(Jh[d], Jv[d], h[d], [1.0, 1.5, 2.0][d], 4, start[d], 3, 1, True, True,
                                          seed=3, step=0, T=T, instance_offset=d * C)
        assert np.array_equal(acc[d], oacc)
        assert np.array_equal(ch.spins[d].cpu().numpy(), ref)
    # Delta of the closed lattices: energies and link overlaps as the oracle computes them
    dm, dd = ch.delta()
    sp = ch.spins.cpu().numpy()
    for d in range(D):
        E = tnmc.energy_periodic(Jh[d], Jv[d], h[d], sp[d], True, True)
        q = sum(((sp[d][a] * np.roll(sp[d][a], -1, 1)) * (sp[d][a + 1] * np.roll(sp[d][a + 1], -1, 1))).sum()
                + ((sp[d][a] * np.roll(sp[d][a], -1, 0)) * (sp[d][a + 1] * np.roll(sp[d][a + 1], -1, 0))).sum()
                for a in range(0, C, 2)) / (C // 2)
        beta = [1.0, 1.5, 2.0][d]
        assert dd[d].item() == pytest.approx((E.mean() + beta * (2 * L * L - q)) / (L * L), abs=1e-12)


def test_frozen_line_chains_sample_the_torus_boltzmann_law(B):
    from paper_2104_13264_gb300 import frozen
    Ly, Lx = 3, 4
    r = np.random.default_rng(5)
    Jh, Jv, h = r.standard_normal((Ly, Lx)), r.standard_normal((Ly, Lx)), 0.4 * r.standard_normal((Ly, Lx))
    beta = 1.3
    n = Ly * Lx
    k = np.arange(2 ** n)[:, None]
    S = (2 * ((k >> np.arange(n)[None]) & 1) - 1).astype(np.int8).reshape(-1, Ly, Lx)
    E = tnmc.energy_periodic(Jh, Jv, h, S, True, True)
    w = np.exp(-beta * (E - E.min()))
    pi = w / w.sum()
    C = 20000
    start = S[np.random.default_rng(6).choice(len(pi), size=C, p=pi)]
    ch = frozen.FrozenLineChains(Jh, Jv, h, beta, 1, start, proposals=1, seed=8)
    accs = [ch.step().float().mean().item() for _ in range(6)]
    assert 0.05 < np.mean(accs) < 0.95
    bits = (ch.spins[0].reshape(C, -1) > 0).long().cpu().numpy()
    counts = np.bincount((bits << np.arange(n)).sum(axis=1), minlength=len(pi))
    e = C * pi
    keep = e > 5
    chi2 = ((counts[keep] - e[keep]) ** 2 / e[keep]).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-3, (np.mean(accs), chi2)
