"""Parity at the headline shape: the 256-wide critical ferromagnet at chi = 64 (needs a GB300).

The 256 x 256, chi = 64, B = 2^20 workload is too large for the oracle to build, so its
shape is checked on the 16-row strip of the same lattice (Lx = 256, beta = 0.4407,
chi = 64, bond dimensions reaching 64 for rows r <= 10): the same kernels, the same
K = 64 contraction with no zero padding, the same 255-deep right stack per row and
eight spin-bit words per sample, in the launch configuration the benchmark uses.

- Builder (Z2 sectors, and the dense path): gauge-invariant outputs against the
  oracle's FP64 build (App. A).
- BF16 tensor-core sampler: the oracle evaluates the GPU's draws in FP64 on the
  environment rounded to the BF16 hi + lo pairs (oracle.tnmc.env_bf16); log q within
  1e-4 relative, forced == sampled, exact integer energies, no flags.
- The plain FP64 form on both builds: draws equal to the oracle's except at a CDF
  edge, log q within 1e-9 relative (two SVD routines agree to ~1e-11 per tensor).
- All three samplers on identical tensors (seeded positive tensors with the strip's
  bond dimensions, given to both sides): FP64 spins bit-exact and log q within 1e-9
  absolute; FP32 and BF16 within 1e-4 relative.
- |log q| near 10^4 (128 x 256 at chi = 16): the BF16 bar at the largest n the oracle
  evaluates in seconds; the measured error is printed beside the bar.
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


@pytest.fixture(scope="module")
def strip(B):
    inst = instances.config5_strip(16)
    ref = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    env = B.Env.from_instance(inst, precisions=("f64", "f32", "bf16"))
    assert env.status() == 0
    return inst, ref, env


def _check_builder(ex, ref, inst):
    assert ex["logZ"] == pytest.approx(ref.logZ, rel=1e-11)
    np.testing.assert_allclose(ex["log_scale"], ref.log_scale, rtol=1e-11, atol=1e-9)
    worst_sv, worst_d = 0.0, 0.0
    for (r, c), s in ref.sv.items():
        k = s.size
        assert ex["bond_dims"][r, c] == k
        worst_sv = max(worst_sv, float(np.abs(ex["sv"][r, c, :k] - s).max()))
        worst_d = max(worst_d, abs(ex["discarded"][r, c] - ref.discarded[(r, c)]))
    assert worst_sv < 1e-9 and worst_d < 1e-12, (worst_sv, worst_d)
    T = ex["tensors"]
    for r in range(inst.Ly):
        for c in range(1, inst.Lx):
            a, b = ex["bond_dims"][r, c], ex["bond_dims"][r, c + 1]
            A = T[r, c, :a, :, :b].reshape(a, -1)
            nz = np.linalg.norm(A, axis=1) > 0.5
            np.testing.assert_allclose(A[nz] @ A[nz].T, np.eye(int(nz.sum())), atol=1e-10)
            assert np.all(np.linalg.norm(A[~nz], axis=1) == 0)
    # chi = 64 is reached, below the exact Schmidt rank (up to 2^16 here); the weight it
    # discards on this strip is at the rounding level (the spectrum decays fast)
    assert ex["bond_dims"].max() == 64
    assert any(ex["bond_dims"][r, c] < min(1 << c, 1 << (inst.Lx - c), 1 << (inst.Ly - r))
               for r in range(inst.Ly) for c in range(1, inst.Lx))
    print("strip build: max |sv - oracle| %.3g, max |discarded - oracle| %.3g, max discarded %.3g"
          % (worst_sv, worst_d, max(ref.discarded.values())))


def test_strip_builder_chi64_z2(strip):
    inst, ref, env = strip
    _check_builder(env.export(), ref, inst)


def test_strip_builder_chi64_dense(B, strip, monkeypatch):
    inst, ref, _ = strip
    monkeypatch.setenv("TNMC_DENSE_BUILDER", "1")
    env = B.Env.from_instance(inst, precisions=("f64",))
    monkeypatch.delenv("TNMC_DENSE_BUILDER")
    assert env.status() == 0
    _check_builder(env.export(), ref, inst)
    env.free()


def _bf16_vs_oracle(B, env, ref, n, seed, offset):
    sp, lq, E, fl = B.sample(env, n, seed=seed, sample_offset=offset, precision="bf16")
    lq2, E2, fl2 = B.logq(env, sp, precision="bf16")
    torch.cuda.synchronize()
    assert torch.equal(lq, lq2) and torch.equal(E, E2) and torch.equal(fl, fl2)   # forced == sampled
    spn = sp.cpu().numpy()
    assert set(np.unique(spn)) <= {-1, 1}
    _, olq, oE, ofl = tnmc.logq(tnmc.env_bf16(ref), spn)
    assert np.all(fl.cpu().numpy() == 0) and np.all(ofl == 0)
    assert np.array_equal(E.cpu().numpy(), oE)
    rel = np.abs(lq.cpu().numpy() - olq) / np.abs(olq)
    return rel, olq


def test_strip_bf16_sampler_vs_oracle(B, strip):
    inst, ref, env = strip
    rel, olq = _bf16_vs_oracle(B, env, ref, 300, seed=17, offset=1 << 20)   # 2 tiles + a ragged 44
    print("strip BF16: max rel err of log q %.3g (bar 1e-4), |log q| ~ %.0f" % (rel.max(), np.abs(olq).mean()))
    assert rel.max() < 1e-4


def test_strip_fp64_plain_form_vs_oracle(B, strip):
    inst, ref, env = strip
    n = 200
    sp, lq, E, fl = B.sample(env, n, seed=23, sample_offset=77, precision="f64")
    torch.cuda.synchronize()
    osp, olq, oE, ofl = tnmc.sample(ref, n, seed=23, sample_offset=77)
    sp = sp.cpu().numpy()
    same = np.all(sp.reshape(n, -1) == osp.reshape(n, -1), axis=1)
    assert same.mean() >= 0.98, same.mean()
    for b in np.nonzero(~same)[0]:
        site = int(np.argmax(osp[b].reshape(-1) != sp[b].reshape(-1)))
        r, c = divmod(site, inst.Lx)
        pplus = _oracle_pplus(ref, osp[b:b + 1], r, c)
        x = philox.draw_words(23, site, np.array([77 + b], dtype=np.uint64))[0]
        assert abs(float(x) / 2.0 ** 64 - pplus) < 1e-6, (b, site)
    lqn = lq.cpu().numpy()
    err = np.abs(lqn[same] - olq[same]) / np.abs(olq[same])
    print("strip FP64 (two builders): max rel err of log q %.3g (bar 1e-9), %d/%d draws equal"
          % (err.max(), same.sum(), n))
    assert err.max() < 1e-9
    assert np.array_equal(E.cpu().numpy()[same], oE[same])
    assert np.all(fl.cpu().numpy() == 0)


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


def test_strip_samplers_on_shared_tensors(B):
    """Identical seeded tensors on both sides (inputs, not builder output)."""
    inst = instances.config5_strip(16)
    shapes = [(tnmc.bond_dim(64, inst.Lx, inst.Ly, r, c), 2, tnmc.bond_dim(64, inst.Lx, inst.Ly, r, c + 1))
              for r in range(inst.Ly) for c in range(inst.Lx)]
    ts = instances.random_tensors(shapes, seed=5)
    oenv = tnmc.Env(inst.Lx, inst.Ly, inst.beta, inst.chi, inst.Jh, inst.Jv, inst.h)
    oenv.M = [[ts[r * inst.Lx + c] for c in range(inst.Lx)] for r in range(inst.Ly)]
    env = B.Env.from_instance(inst, precisions=("f64", "f32", "bf16"))
    P = env.info()["pad"]
    flat = np.zeros((inst.Ly, inst.Lx, P, 2, P))
    for r in range(inst.Ly):
        for c in range(inst.Lx):
            t = ts[r * inst.Lx + c]
            flat[r, c, :t.shape[0], :, :t.shape[2]] = t
    B.set_tensors(env, torch.from_numpy(flat.reshape(-1)).cuda())
    n = 200
    # FP64: the oracle's own draws from the shared Philox stream, bit for bit
    sp, lq, E, fl = B.sample(env, n, seed=31, sample_offset=9, precision="f64")
    torch.cuda.synchronize()
    osp, olq, oE, ofl = tnmc.sample(oenv, n, seed=31, sample_offset=9)
    assert np.array_equal(sp.cpu().numpy(), osp)
    err = np.abs(lq.cpu().numpy() - olq).max()
    print("shared tensors FP64: max abs err of log q %.3g (bar 1e-9)" % err)
    assert err < 1e-9
    assert np.array_equal(E.cpu().numpy(), oE) and np.array_equal(fl.cpu().numpy(), ofl)
    # FP32 and BF16: the oracle evaluates their draws (on the BF16 pairs for BF16)
    for prec, oref in (("f32", oenv), ("bf16", tnmc.env_bf16(oenv))):
        sp, lq, E, fl = B.sample(env, n, seed=37, precision=prec)
        torch.cuda.synchronize()
        _, olq, oE, ofl = tnmc.logq(oref, sp.cpu().numpy())
        rel = np.abs(lq.cpu().numpy() - olq) / np.abs(olq)
        print("shared tensors %s: max rel err of log q %.3g (bar 1e-4)" % (prec, rel.max()))
        assert rel.max() < 1e-4
        assert np.array_equal(E.cpu().numpy(), oE)
    env.free()


def test_bf16_logq_near_1e4(B):
    """128 x 256 ferromagnet at beta = 0.4407, chi = 16: |log q| ~ 10^4 over 32768 sites."""
    inst = instances.ferromagnet(128, 256, 0.4407, 16)
    ref = tnmc.build_env(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi)
    env = B.Env.from_instance(inst, precisions=("f64", "bf16"))
    rel, olq = _bf16_vs_oracle(B, env, ref, 129, seed=41, offset=0)
    print("128x256 chi=16 BF16: max rel err of log q %.3g (bar 1e-4), mean |log q| %.0f"
          % (rel.max(), np.abs(olq).mean()))
    assert np.abs(olq).mean() > 8e3
    assert rel.max() < 1e-4
    env.free()
