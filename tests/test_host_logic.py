"""Host-side logic that needs no GPU: residence weights of the tuning loop and the
reference arm's JSON line of bench.py."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_residence_weights_by_hand():
    from paper_2104_13264_gb300.tuning import residence_weights
    acc = torch.tensor([[0, 1, 0, 0, 1, 0],
                        [0, 0, 0, 0, 0, 0],
                        [1, 1, 1, 1, 1, 1],
                        [1, 0, 0, 0, 0, 0]], dtype=torch.uint8)
    w_acc, w_held = residence_weights(acc)
    assert w_acc.tolist() == [[0, 3, 0, 0, 2, 0], [0] * 6, [1] * 6, [6, 0, 0, 0, 0, 0]]
    assert w_held.tolist() == [1, 6, 0, 0]


def test_residence_weights_sum_to_T():
    from paper_2104_13264_gb300.tuning import residence_weights
    g = torch.Generator().manual_seed(0)
    acc = (torch.rand(50, 37, generator=g) < 0.3).to(torch.uint8)
    w_acc, w_held = residence_weights(acc)
    assert torch.equal(w_acc.sum(dim=1) + w_held, torch.full((50,), 37))
    assert bool(((w_acc > 0) == acc.bool()).all())


def test_reference_arm_prints_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "c1",
                        "--steps", "1", "--warmup", "0", "--cpu-batch", "64"],
                       capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["workload"] == "c1"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_open_instances_match_the_oracle_cut():
    """The frozen-line driver's open instances (couplings and fields from the frozen spins)
    are the oracle's, for the three closed geometries and several cuts."""
    import numpy as np

    from oracle import tnmc
    from paper_2104_13264_gb300 import frozen
    r = np.random.default_rng(4)
    for Ly, Lx in ((5, 6), (2, 3), (3, 2)):
        Jh, Jv, h = r.standard_normal((Ly, Lx)), r.standard_normal((Ly, Lx)), r.standard_normal((Ly, Lx))
        sp = r.choice([-1, 1], size=(7, Ly, Lx)).astype(np.int8)
        for px, py in ((True, True), (True, False), (False, True)):
            for kr, kc in ((0, 0), (Ly - 1, 1), (1, Lx - 1)):
                a = frozen.open_instances(Jh, Jv, h, sp, kr, kc, px, py)
                b = tnmc.frozen_cut(Jh, Jv, h, sp, kr, kc, px, py)
                assert list(a[0]) == list(b[0]) and list(a[1]) == list(b[1])
                for x, y in zip(a[2:], b[2:]):
                    np.testing.assert_allclose(x, y, rtol=0, atol=1e-13)


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("gauge", ["spin", "bond"])
def test_roofline_flop_count_uses_the_built_bond_dimensions(gauge):
    """The roofline's algorithmic FLOPs per sample (8 chi_c chi_{c+1} per site, 4 on row 0)
    model the sampling bonds as min(chi, 2^min(c, Lx - c, Ly - r)) (doubled in the bond
    basis). They must equal the same sum over the bonds of the environments the oracle
    actually builds, on random instances whose bonds saturate in some rows and not in others."""
    from types import SimpleNamespace

    import numpy as np

    from oracle import tnmc
    bench = _bench_module()
    r = np.random.default_rng(0)
    build = tnmc.build_env if gauge == "spin" else tnmc.build_env_bond
    for Ly, Lx, chi in ((6, 7, 4), (5, 9, 3), (4, 4, 16), (3, 10, 2), (2, 1, 4)):
        Jh, Jv = r.standard_normal((Ly, Lx - 1)), r.standard_normal((Ly - 1, Lx))
        h = 0.3 * r.standard_normal((Ly, Lx))
        env = build(Jh, Jv, h, 0.7, chi)
        built = sum((8 if row > 0 else 4) * env.M[row][c].shape[0] * env.M[row][c].shape[2]
                    for row in range(Ly) for c in range(Lx))
        model = bench.algorithmic_flops(SimpleNamespace(Lx=Lx, Ly=Ly, chi=chi), gauge=gauge)
        assert model == built, (Ly, Lx, chi, model, built)


def test_mh_band_margin_is_sound():
    """The MH scan's integer bands (order-preserving int64 keys of the weights a; accept on
    key(a) <= max(key(theta - m), key(a')), reject on key(a) >= key(theta + m), with
    theta = a' - log u and m = 1e-12 (1 + |theta|)) never contradict the rule
    u < exp(min(0, a' - a)) evaluated in FP64, here with numpy's log and exp, for current
    weights placed at chosen multiples of m from theta and weights of magnitude 1 to 1e7.
    This checks the margin argument; the kernels themselves are compared with the oracle's
    rule on the GPU."""
    import numpy as np
    i64max = np.int64(2 ** 63 - 1)

    def key(x):
        b = np.asarray(x, dtype=np.float64).view(np.int64)
        return np.where(b >= 0, b, b ^ i64max)

    rng = np.random.default_rng(1)
    n = 250_000
    decided = 0
    for scale in (1.0, 1e3, 1e5, 1e7):
        u = rng.integers(1, 2 ** 53, n) * 2.0 ** -53
        u[:10] = 1 - 2.0 ** -53
        u[10:20] = 2.0 ** -53
        wt = rng.normal(0.0, scale, n)
        theta = wt - np.log(u)
        m = 1e-12 * (1.0 + np.abs(theta))
        k = rng.choice([-5, -2, -1.01, -1, -0.5, 0, 0.5, 1, 1.01, 2, 5, 1e6, -1e6], n)
        wc = theta + k * m
        lo = np.maximum(key(theta - m), key(wt))
        hi = key(theta + m)
        kc = key(wc)
        acc, rej = kc <= lo, (kc >= hi) & ~(kc <= lo)
        with np.errstate(over="ignore"):
            d = wt - wc
            rule = (d >= 0) | (u < np.exp(np.minimum(d, 0.0)))
        assert not np.any(acc & ~rule), scale
        assert not np.any(rej & rule), scale
        decided += int(np.sum(acc | rej))
    assert decided > 0.7 * 4 * n       # most placements fall outside the band
