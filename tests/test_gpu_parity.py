"""CUDA path vs the FP64 oracle through the C-ABI (needs a GB300)."""
import math

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


def _cases():
    return [
        instances.random_small(4, 4, 0.9, 2, seed=1),
        instances.random_small(4, 4, 0.7, 4, seed=2),            # exact chi
        instances.random_small(5, 7, 1.1, 3, seed=3),            # odd sizes, chi not a power of 2
        instances.random_small(3, 17, 0.8, 8, seed=4),           # wide, ragged P padding
        instances.random_small(9, 1, 0.8, 2, seed=5),            # one column
        instances.random_small(1, 9, 0.8, 2, seed=6),            # one row
        instances.random_small(6, 6, 0.9, 1, seed=7),            # chi = 1
        instances.ea_pm(8, 8, 1.0, 4, seed=1),
        instances.villain(6, 6, 1.5, 4),
        instances.config1(),
        instances.ea_gauss(12, 12, 2.0, 8, seed=3),
    ]


def _oracle_env(inst):
    return tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)


@pytest.mark.parametrize("idx", range(11))
def test_builder_gauge_invariants(B, idx):
    inst = _cases()[idx]
    ref = _oracle_env(inst)
    env = B.Env.from_instance(inst, precisions=("f64", "f32"))
    ex = env.export()
    assert env.status() == 0
    assert ex["logZ"] == pytest.approx(ref.logZ, abs=1e-9 * max(1.0, abs(ref.logZ)))
    for r in range(inst.Ly):
        for c in range(inst.Lx):
            assert ex["bond_dims"][r, c] == tnmc.bond_dim(inst.chi, inst.Lx, inst.Ly, r, c)
        assert ex["log_scale"][r] == pytest.approx(ref.log_scale[r], abs=1e-9 * max(1.0, abs(ref.log_scale[r])))
    for (r, c), s in ref.sv.items():
        k = s.size
        np.testing.assert_allclose(ex["sv"][r, c, :k], s, atol=1e-9)
        assert ex["discarded"][r, c] == pytest.approx(ref.discarded[(r, c)], abs=1e-12)
    # sites c >= 1 are right-orthonormal; kept directions at the rounding level are
    # stored as zero rows (they carry no weight)
    T = ex["tensors"]
    for r in range(inst.Ly):
        for c in range(1, inst.Lx):
            a = ex["bond_dims"][r, c]
            b = ex["bond_dims"][r, c + 1]
            A = T[r, c, :a, :, :b].reshape(a, -1)
            nz = np.linalg.norm(A, axis=1) > 0.5
            G = A[nz] @ A[nz].T
            np.testing.assert_allclose(G, np.eye(G.shape[0]), atol=1e-10)
            assert np.all(np.linalg.norm(A[~nz], axis=1) == 0)


@pytest.mark.parametrize("idx", range(11))
def test_fp64_sampler_matches_oracle(B, idx):
    inst = _cases()[idx]
    ref = _oracle_env(inst)
    env = B.Env.from_instance(inst, precisions=("f64",))
    n = 301 if idx % 2 else 256          # ragged tail vs whole tiles
    sp, lq, E, fl = B.sample(env, n, seed=11 + idx, sample_offset=5)
    torch.cuda.synchronize()
    osp, olq, oE, ofl = tnmc.sample(ref, n, seed=11 + idx, sample_offset=5)
    sp = sp.cpu().numpy()
    assert np.array_equal(sp, osp), "spins differ"
    np.testing.assert_allclose(lq.cpu().numpy(), olq, rtol=0, atol=1e-9)
    if inst.integer_couplings:
        assert np.array_equal(E.cpu().numpy(), oE)
    else:
        np.testing.assert_allclose(E.cpu().numpy(), oE, rtol=1e-13, atol=1e-12)
    assert np.array_equal(fl.cpu().numpy(), ofl)


def test_forced_mode_equals_sampling_mode(B):
    inst = instances.ea_pm(10, 10, 1.0, 8, seed=2)
    for prec in ("f64", "f32"):
        env = B.Env.from_instance(inst, precisions=("f64", "f32"))
        sp, lq, E, fl = B.sample(env, 500, seed=3, precision=prec)
        lq2, E2, fl2 = B.logq(env, sp, precision=prec)
        assert torch.equal(lq, lq2) and torch.equal(E, E2) and torch.equal(fl, fl2)


def test_sample_offset_shards_bit_exact(B):
    inst = instances.random_small(6, 5, 0.8, 4, seed=8)
    env = B.Env.from_instance(inst, precisions=("f64", "f32"))
    for prec in ("f64", "f32"):
        full = B.sample(env, 700, seed=5, precision=prec)
        a = B.sample(env, 300, seed=5, sample_offset=0, precision=prec)
        b = B.sample(env, 400, seed=5, sample_offset=300, precision=prec)
        for x, y, z in zip(full, a, b):
            assert torch.equal(x, torch.cat([y, z]))


def test_fp32_sampler_vs_oracle(B):
    """FP32 sampler: log q of its draws within 1e-4 relative of the oracle's forced
    log q; draws equal to the oracle's apart from those at a CDF edge."""
    inst = instances.config2()
    ref = _oracle_env(inst)
    env = B.Env.from_instance(inst, precisions=("f64", "f32"))
    n = 513
    sp, lq, E, fl = B.sample(env, n, seed=0, precision="f32")
    sp = sp.cpu().numpy()
    lq = lq.cpu().numpy()
    _, olq_forced, oE, ofl = tnmc.logq(ref, sp)
    assert np.all(ofl == 0) and np.all(fl.cpu().numpy() == 0)
    np.testing.assert_allclose(lq, olq_forced, rtol=1e-4)
    assert np.array_equal(E.cpu().numpy(), oE)
    osp, olq, _, _ = tnmc.sample(ref, n, seed=0)
    same = np.all(osp.reshape(n, -1) == sp.reshape(n, -1), axis=1)
    assert same.mean() > 0.9
    # every differing sample must first differ at a site whose draw sat at the CDF edge
    for b in np.nonzero(~same)[0]:
        site = int(np.argmax(osp[b].reshape(-1) != sp[b].reshape(-1)))
        r, c = divmod(site, inst.Lx)
        # oracle conditional at that site given the shared prefix
        pre = osp[b:b + 1].copy()
        pplus = _oracle_pplus(ref, pre, r, c)
        x = philox.draw_words(0, site, np.array([b], dtype=np.uint64))[0]
        assert abs(float(x) / 2.0 ** 64 - pplus) < 1e-5, (b, site)


def _oracle_pplus(env, spins, r, c):
    """Oracle conditional p_+ at (r, c) given spins before it (FP64)."""
    Lx = env.Lx
    f = tnmc.row_fields(env, spins, r)
    M = env.M[r]
    R = np.ones((1, 1))
    for cc in range(Lx - 1, c, -1):
        Y = np.einsum("asb,nb->nas", M[cc], R)
        R = Y[:, :, 0] * f[:, cc, 0:1] + Y[:, :, 1] * f[:, cc, 1:2]
    Lam = np.ones((1, 1))
    for cc in range(c):
        s = int(spins[0, r, cc] > 0)
        Lam = np.einsum("na,ab->nb", Lam, M[cc][:, s, :]) * f[0, cc, s]
    U = np.einsum("na,asb->nsb", Lam, M[c])
    w = np.maximum(np.einsum("nsb,nb->ns", U, R)[0] * f[0, c], 0)
    return w[1] / w.sum()


def test_init_chains_and_mh_match_oracle(B):
    inst = instances.config1()
    ref = _oracle_env(inst)
    env = B.Env.from_instance(inst)
    C, T = 16, 64
    cs, clq, cE = B.init_chains(env, C, seed=9)
    ocs, oclq, ocE = tnmc.init_chains(ref, C, seed=9)
    assert np.array_equal(cs.cpu().numpy(), ocs)
    np.testing.assert_allclose(clq.cpu().numpy(), oclq, atol=1e-9)
    # identical proposal inputs on both sides -> identical decisions
    osp, olq, oE, _ = tnmc.sample(ref, C * T, seed=10)
    prop = (torch.from_numpy(osp).cuda(), torch.from_numpy(olq).cuda(), torch.from_numpy(oE).cuda())
    chain = (torch.from_numpy(ocs).cuda(), torch.from_numpy(oclq).cuda(), torch.from_numpy(ocE).cuda())
    nacc = torch.zeros(1, dtype=torch.int64, device="cuda")
    acc = B.mh_step(env, C, T, prop, chain, seed=12, step_offset=3, n_accepted=nacc)
    oacc, osp2, olq2, oE2 = tnmc.mh_scan(inst.beta, C, T, osp, olq, oE, ocs, oclq, ocE, seed=12, step_offset=3)
    assert np.array_equal(acc.cpu().numpy().astype(bool), oacc)
    assert int(nacc.item()) == int(oacc.sum())
    assert np.array_equal(chain[0].cpu().numpy(), osp2)
    assert np.array_equal(chain[1].cpu().numpy(), olq2)
    assert np.array_equal(chain[2].cpu().numpy(), oE2)


def test_mh_rejects_flagged_proposals(B):
    inst = instances.config1()
    env = B.Env.from_instance(inst)
    C, T = 4, 8
    sp = torch.ones((C * T, 8, 8), dtype=torch.int8, device="cuda")
    lq = torch.full((C * T,), -math.inf, dtype=torch.float64, device="cuda")
    lq[1::2] = float("nan")
    E = torch.zeros(C * T, dtype=torch.float64, device="cuda")
    chain = (torch.ones((C, 8, 8), dtype=torch.int8, device="cuda"), torch.zeros(C, dtype=torch.float64, device="cuda"),
             torch.zeros(C, dtype=torch.float64, device="cuda"))
    acc = B.mh_step(env, C, T, (sp, lq, E), chain, seed=1)
    assert int(acc.sum()) == 0


def test_mh_start_outside_support_matches_oracle(B):
    """Chains whose start has log q = -inf take their first valid proposal (same rule as
    the oracle's scan); later decisions follow the ordinary ratio."""
    inst = instances.ea_pm(6, 6, 1.0, 2, seed=3)
    ref = _oracle_env(inst)
    env = B.Env.from_instance(inst)
    C, T = 8, 16
    sp, lq, E, fl = B.sample(env, C * T, seed=4)
    lq[::5] = -math.inf                       # a few invalid proposals too
    cs, clq, cE = B.init_chains(env, C, seed=5)
    clq[::2] = -math.inf
    ocs, oclq, ocE = cs.cpu().numpy().copy(), clq.cpu().numpy().copy(), cE.cpu().numpy().copy()
    acc = B.mh_step(env, C, T, (sp, lq, E), (cs, clq, cE), seed=6, step_offset=3)
    oacc, osp, olq, oE = tnmc.mh_scan(inst.beta, C, T, sp.cpu().numpy(), lq.cpu().numpy(), E.cpu().numpy(),
                                      ocs, oclq, ocE, seed=6, step_offset=3)
    assert np.array_equal(acc.cpu().numpy().astype(bool), oacc)
    assert np.array_equal(cs.cpu().numpy(), osp)
    assert np.array_equal(clq.cpu().numpy(), olq) and np.array_equal(cE.cpu().numpy(), oE)
    first_valid = [next(j for j in range(T) if (i * T + j) % 5) for i in range(0, C, 2)]
    assert all(oacc[i * T + j] for i, j in zip(range(0, C, 2), first_valid))
    assert bool(torch.isfinite(clq).all())


def test_exact_chi_gives_acceptance_one(B):
    """At exact chi q = pi, so Delta = 0 and every proposal is accepted (Sec. 2)."""
    inst = instances.ea_gauss(4, 4, 1.0, 4, seed=4, hscale=0.3)
    env = B.Env.from_instance(inst)
    C, T = 64, 32
    prop = B.sample(env, C * T, seed=2)[:3]
    chain = B.init_chains(env, C, seed=2)
    acc = B.mh_step(env, C, T, prop, chain, seed=3)
    # the first step of each chain leaves a random start (q != pi there is impossible: exact)
    assert acc.float().mean().item() > 0.999


def test_beta_zero_uniform_q(B):
    inst = instances.random_small(7, 5, 0.0, 4, seed=2)
    env = B.Env.from_instance(inst)
    sp, lq, E, fl = B.sample(env, 200, seed=1)
    np.testing.assert_allclose(lq.cpu().numpy(), -35 * math.log(2), atol=1e-12)


def test_empty_batch_is_noop(B):
    env = B.Env.from_instance(instances.config1())
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    B.sample(env, 0, out=(torch.empty((0, 8, 8), dtype=torch.int8, device="cuda"), e, e,
                          torch.empty(0, dtype=torch.int32, device="cuda")))
    torch.cuda.synchronize()


def test_missing_precision_is_rejected(B):
    env = B.Env.from_instance(instances.config1(), precisions=("f64",))
    with pytest.raises(B.TnmcError, match="status 6"):
        B.sample(env, 4, precision="f32")


def test_config2_full_launch_sampled(B):
    """Config-2 launch (B = 65536, FP32, the benchmark's shape): 48 sampled outputs
    checked one by one against the oracle's forced evaluation."""
    inst = instances.config2()
    ref = _oracle_env(inst)
    env = B.Env.from_instance(inst, precisions=("f64", "f32"))
    n = 65536
    sp, lq, E, fl = B.sample(env, n, seed=0, precision="f32")
    torch.cuda.synchronize()
    assert int(fl.sum().item()) == 0
    idx = np.random.default_rng(0).choice(n, 48, replace=False)
    spn = sp[torch.from_numpy(idx).cuda()].cpu().numpy()
    _, olq, oE, _ = tnmc.logq(ref, spn)
    np.testing.assert_allclose(lq.cpu().numpy()[idx], olq, rtol=1e-4)
    assert np.array_equal(E.cpu().numpy()[idx], oE)
    # the oracle's own draws for those sample indices agree on most samples
    osp, _, _, _ = tnmc.sample(ref, 48, seed=0, samples=idx)
    same = np.all(osp.reshape(48, -1) == spn.reshape(48, -1), axis=1)
    assert same.mean() > 0.8


@pytest.mark.parametrize("inst", [instances.ea_pm(8, 9, 1.0, 4, seed=5), instances.villain(6, 7, 1.5, 8),
                                  instances.ferromagnet(5, 12, 0.0, 4)])
def test_z2_builder_equals_dense_builder(B, inst, monkeypatch):
    """With h = 0 the library builds in parity sectors; the dense builder (forced) must
    give the same gauge-invariant environment and the same q."""
    env_z2 = B.Env.from_instance(inst)
    ex_z2 = env_z2.export()
    monkeypatch.setenv("TNMC_DENSE_BUILDER", "1")
    env_d = B.Env.from_instance(inst)
    ex_d = env_d.export()
    monkeypatch.delenv("TNMC_DENSE_BUILDER")
    assert ex_z2["logZ"] == pytest.approx(ex_d["logZ"], abs=1e-10 * max(1.0, abs(ex_d["logZ"])))
    np.testing.assert_allclose(ex_z2["sv"], ex_d["sv"], atol=1e-10)
    np.testing.assert_allclose(ex_z2["log_scale"], ex_d["log_scale"], atol=1e-9)
    assert np.array_equal(ex_z2["bond_dims"], ex_d["bond_dims"])
    sp, lq, E, fl = B.sample(env_z2, 257, seed=4)
    lq2, E2, fl2 = B.logq(env_d, sp)
    np.testing.assert_allclose(lq.cpu().numpy(), lq2.cpu().numpy(), atol=1e-9)
