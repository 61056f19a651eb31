"""Batched persistent form vs the single-instance path and the oracle (needs a GB300).

Each instance of a batch follows the single-instance definitions exactly, so
the batched outputs must equal the single-instance calls at the same sample
indices bit for bit, and (FP64) the oracle's draws and log q.
"""
import numpy as np
import pytest

from oracle import philox, tnmc
from paper_2104_13264_gb300 import instances

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHIFT = 40


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_13264_gb300 import binding
    binding.lib()
    return binding


def _mixed():
    """Uneven sizes and bond dimensions, with and without fields (both builders)."""
    return [
        instances.ea_gauss(8, 8, 2.0, 8, seed=1),
        instances.random_small(5, 7, 1.1, 3, seed=3),
        instances.ea_gauss(16, 16, 2.0, 16, seed=2),
        instances.random_small(9, 1, 0.8, 2, seed=5),
        instances.ea_pm(12, 20, 1.0, 8, seed=4),
        instances.random_small(1, 9, 0.8, 2, seed=6),
        instances.ea_gauss(24, 24, 2.0, 32, seed=7, hscale=0.2),
    ]


@pytest.fixture(scope="module")
def mixed(B):
    insts = _mixed()
    envs_b = B.build_envs_batched(insts, precisions=("f64", "f32"))
    envs_s = [B.Env.from_instance(i, precisions=("f64", "f32")) for i in insts]
    return insts, envs_b, envs_s


def test_batched_build_equals_single(B, mixed):
    insts, envs_b, envs_s = mixed
    for inst, eb, es in zip(insts, envs_b, envs_s):
        xb, xs = eb.export(), es.export()
        assert eb.status() == 0
        for k in ("tensors", "log_scale", "sv", "discarded", "bond_dims"):
            assert np.array_equal(xb[k], xs[k]), k
        assert xb["logZ"] == xs["logZ"]
    ref = tnmc.build_env(insts[1].Jh, insts[1].Jv, insts[1].h, insts[1].beta, insts[1].chi)
    assert envs_b[1].export()["logZ"] == pytest.approx(ref.logZ, abs=1e-9 * abs(ref.logZ))


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("tile,order", [(64, "instance"), (128, "cost"), (64, "cost"), (128, "instance")])
def test_batched_sample_equals_single(B, mixed, precision, tile, order):
    insts, envs, _ = mixed
    Bs = [130, 64, 200, 0, 77, 5, 129]          # ragged tails, an empty instance
    plan = B.Batch(envs, Bs, chains=1, precision=precision, tile=tile, order=order)
    out = plan.alloc_proposals()
    seed = 11
    for k in range(2):
        plan.set_step(seed, k)
        plan.sample(out)
        for i, e in enumerate(envs):
            ref = B.sample(e, Bs[i], seed=seed, sample_offset=(i << SHIFT) + k * Bs[i], precision=precision)
            assert torch.equal(plan.view(out[0], i), ref[0])
            for a, b in zip(out[1:], ref[1:]):
                assert torch.equal(plan.rows(a, i), b)
        # forced evaluation of the whole arena reproduces log q and energy
        lq, E, fl = plan.logq(out[0])
        assert torch.equal(lq, out[1]) and torch.equal(E, out[2]) and torch.equal(fl, out[3])


def _oracle_on_export(inst, env):
    """The oracle's sampler on the GPU-built tensors (separates the sampler's arithmetic
    from the two builders' different SVD routines)."""
    ex = env.export()
    ref = tnmc.Env(inst.Lx, inst.Ly, inst.beta, inst.chi, inst.Jh, inst.Jv, inst.h)
    bd = ex["bond_dims"]
    ref.M = [[ex["tensors"][r, c, :bd[r, c], :, :bd[r, c + 1]].copy() for c in range(inst.Lx)]
             for r in range(inst.Ly)]
    return ref


def test_batched_f64_vs_oracle(B, mixed):
    insts, envs, _ = mixed
    Bs = [40, 33, 24, 8, 20, 16, 12]
    plan = B.Batch(envs, Bs, chains=1, precision="f64", tile=64, order="cost")
    out = plan.alloc_proposals()
    seed, k = 5, 3
    plan.set_step(seed, k)
    plan.sample(out)
    for i, inst in enumerate(insts):
        offs = (i << SHIFT) + k * Bs[i]
        got_sp = plan.view(out[0], i).cpu().numpy()
        got_lq = plan.rows(out[1], i).cpu().numpy()
        # the same tensors: draws bit-exact, log q within 1e-9 absolute
        sp, lq, E, fl = tnmc.sample(_oracle_on_export(inst, envs[i]), Bs[i], seed=seed, sample_offset=offs)
        assert np.array_equal(got_sp, sp)
        np.testing.assert_allclose(got_lq, lq, rtol=0, atol=1e-9)
        if inst.integer_couplings:
            assert np.array_equal(plan.rows(out[2], i).cpu().numpy(), E)
        else:
            np.testing.assert_allclose(plan.rows(out[2], i).cpu().numpy(), E, rtol=1e-13, atol=1e-12)
        # the oracle's own environment (its own SVD routine): same draws, log q within 1e-9 relative
        ref = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
        sp2, lq2, _, _ = tnmc.sample(ref, Bs[i], seed=seed, sample_offset=offs)
        assert np.array_equal(got_sp, sp2)
        np.testing.assert_allclose(got_lq, lq2, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batched_init_and_mh_equal_single(B, mixed, precision):
    insts, envs, _ = mixed
    C = 4
    Bs = [C * t for t in (8, 3, 16, 1, 5, 2, 6)]
    plan = B.Batch(envs, Bs, chains=C, precision=precision, tile=64, order="cost")
    seed = 9
    chain = plan.init_chains(seed)
    for i, e in enumerate(envs):
        n = e.Lx * e.Ly
        ids = (np.uint64(i) << np.uint64(32)) + np.arange(C, dtype=np.uint64)
        want = philox.init_bits(seed, n, ids).reshape(C, e.Ly, e.Lx)
        got = plan.view(chain[0], i, chains=True)
        assert np.array_equal(got.cpu().numpy(), want)
        lq, E, _ = B.logq(e, got, precision=precision)
        assert torch.equal(plan.rows(chain[1], i, chains=True), lq)
        assert torch.equal(plan.rows(chain[2], i, chains=True), E)
    singles = [tuple(t.clone() for t in (plan.view(chain[0], i, chains=True), plan.rows(chain[1], i, chains=True),
                                         plan.rows(chain[2], i, chains=True))) for i in range(len(envs))]
    out = plan.alloc_proposals()
    acc = torch.zeros(out[1].numel(), dtype=torch.uint8, device="cuda")
    nacc = torch.zeros(len(envs), dtype=torch.int64, device="cuda")
    total = 0
    for k in range(3):
        plan.set_step(seed, k)
        plan.sample(out)
        plan.mh(out, chain, acc, nacc)
        total += int(acc.sum())
        for i, e in enumerate(envs):
            T = Bs[i] // C
            prop = tuple(t.clone() for t in (plan.view(out[0], i), plan.rows(out[1], i), plan.rows(out[2], i)))
            a1 = B.mh_step(e, C, T, prop, singles[i], seed=seed, step_offset=(i << SHIFT) + k * T)
            assert torch.equal(plan.rows(acc, i), a1)
            assert torch.equal(plan.view(chain[0], i, chains=True), singles[i][0])
            assert torch.equal(plan.rows(chain[1], i, chains=True), singles[i][1])
            assert torch.equal(plan.rows(chain[2], i, chains=True), singles[i][2])
    assert int(nacc.sum()) == total


def test_graph_runner_equals_eager(B, mixed, tmp_path):
    from paper_2104_13264_gb300 import batched
    insts, envs, _ = mixed
    Bs = [64 * 4] * len(envs)
    g = batched.BatchRunner(envs, Bs, chains=4, precision="f32", seed=3, cache_path=str(tmp_path / "t.json"))
    e = batched.BatchRunner(envs, Bs, chains=4, precision="f32", tile=g.plan.tile, order=g.plan.order, seed=3)
    for _ in range(3):
        g.step()
        e.step_eager()
    torch.cuda.synchronize()
    for a, b in zip(g.chain, e.chain):
        assert torch.equal(a, b)
    assert torch.equal(g.n_accepted, e.n_accepted)
    assert torch.equal(g.accepted, e.accepted)
    assert int(g.n_accepted.sum()) > 0
    import json
    cache = json.loads((tmp_path / "t.json").read_text())
    (entry,) = cache.values()
    assert (entry["tile"], entry["order"]) in batched.CANDIDATES and len(entry["candidates"]) == 4


def test_config3_full_size_sampled(B):
    """256 Gaussian EA instances, L in {16..64}, chi in {8,16,32}, 4096 proposals each, one
    persistent launch; sampled instances equal their single-instance calls."""
    from paper_2104_13264_gb300 import batched
    insts = instances.config3()
    envs = B.build_envs_batched(insts, precisions=("f32",))
    for e in envs[:3]:
        assert e.status() == 0
    run = batched.BatchRunner(envs, 4096, chains=16, precision="f32", tune=False, seed=1)
    run.step()
    run.step()
    torch.cuda.synchronize()
    plan = run.plan
    assert plan.info()["items"] == 256 * 4096 // plan.tile
    # the step counter is now 2: re-draw step 1 for a few instances through tnmc_sample
    for i in (0, 17, 128, 255):
        ref = B.sample(envs[i], 4096, seed=1, sample_offset=(i << SHIFT) + 1 * 4096, precision="f32")
        assert torch.equal(plan.view(run.prop[0], i), ref[0])
        assert torch.equal(plan.rows(run.prop[1], i), ref[1])
    # FP32 at beta = 2 may lose a conditional to rounding (both weights clamp to 0): such
    # proposals are flagged and drawn with p = 1/2 at that site, which their finite log q
    # records, so they stay in the chain's exact proposal law
    lq, fl = run.prop[1], run.prop[3]
    assert bool(torch.isfinite(lq).all())
    frac = float((fl != 0).double().mean())
    bad = sorted({i for i in range(plan.n) if bool((plan.rows(fl, i) != 0).any())})
    print("flagged fraction %.3g in %d instances %s" % (frac, len(bad), bad[:20]))
    assert frac < 1e-2
    assert int(run.n_accepted.sum()) > 0


def test_batch_balance_is_a_fraction(B):
    from paper_2104_13264_gb300 import batched
    insts = [instances.ea_gauss(8 + 4 * (k % 3), 8 + 4 * (k % 3), 2.0, 4, seed=k) for k in range(12)]
    envs = B.build_envs_batched(insts, precisions=("f32",))
    run = batched.BatchRunner(envs, 256, chains=8, precision="f32", tile=64, order="cost", tune=False, seed=1)
    run.plan.set_step(1, 0)
    run.plan.sample(run.prop)
    eff, span = run.plan.balance()
    assert 0.0 < eff <= 1.0 and span > 0.0


def test_mixed_runner_matches_single_instance_calls(B):
    """The per-chi-class runner: its tensor-core instances evolve exactly as the
    single-instance BF16 sample + MH calls with the documented counters, and its FP32
    instances as their own persistent plan."""
    from paper_2104_13264_gb300 import batched
    insts = [instances.ea_gauss(8, 8, 2.0, 4, seed=1), instances.ea_gauss(10, 10, 2.0, 32, seed=2),
             instances.ea_gauss(6, 9, 2.0, 8, seed=3), instances.ea_gauss(12, 12, 2.0, 32, seed=4)]
    run = batched.MixedRunner(insts, 256, 8, tc_chi=32, seed=5, tune=False)
    assert run.big_idx == [1, 3] and run.small_idx == [0, 2]
    start = [tuple(t.clone() for t in ch) for ch in run.big_chain]
    for _ in range(2):
        run.step()
    torch.cuda.synchronize()
    for j, i in enumerate(run.big_idx):
        e = run.big_envs[j]
        ch = start[j]
        idx = len(run.small_idx) + j
        for k in range(2):
            sp, lq, E, _ = B.sample(e, 256, seed=5, sample_offset=(idx << 40) + k * 256, precision="bf16")
            B.mh_step(e, 8, 32, (sp, lq, E), ch, seed=5, step_offset=(idx << 40) + k * 32)
        torch.cuda.synchronize()
        assert torch.equal(ch[0], run.big_chain[j][0]) and torch.equal(ch[1], run.big_chain[j][1])
    assert run.n_accepted() > 0
