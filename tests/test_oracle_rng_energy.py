"""Pins of the oracle's Philox stream and Ising energy (no GPU)."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import exact, philox, tnmc
from paper_2104_13264_gb300 import instances

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_philox_matches_triton_interpreter():
    """Triton's Philox4x32-10 (run by its CPU interpreter) is an independent implementation."""
    pytest.importorskip("triton")
    code = textwrap.dedent("""
        import os, json
        os.environ["TRITON_INTERPRET"] = "1"
        import torch, triton, triton.language as tl
        @triton.jit
        def k(out, seed, c0p, c1p, c2p, c3p, N: tl.constexpr):
            o = tl.arange(0, N)
            a, b, c, d = tl.philox(seed, tl.load(c0p + o), tl.load(c1p + o), tl.load(c2p + o), tl.load(c3p + o))
            tl.store(out + o * 4 + 0, a); tl.store(out + o * 4 + 1, b)
            tl.store(out + o * 4 + 2, c); tl.store(out + o * 4 + 3, d)
        N = 8
        g = torch.Generator().manual_seed(5)
        cs = [torch.randint(-2**31, 2**31 - 1, (N,), dtype=torch.int64, generator=g).to(torch.int32) for _ in range(4)]
        res = {}
        for seed in (0, 12345, 0xFFFFFFFF, 0x123456789ABCDEF):
            out = torch.zeros(N * 4, dtype=torch.int32)
            k[(1,)](out, seed, *cs, N=N)
            res[str(seed)] = [x & 0xFFFFFFFF for x in out.tolist()]
        print(json.dumps({"c": [[x & 0xFFFFFFFF for x in c.tolist()] for c in cs], "out": res}))
    """)
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr[-300:])
    import json
    d = json.loads(p.stdout.strip().splitlines()[-1])
    c = [np.array(x, dtype=np.uint64) for x in d["c"]]
    for seed, words in d["out"].items():
        s = int(seed)
        w = philox.philox4x32_10(c[0], c[1], c[2], c[3], s & 0xFFFFFFFF, s >> 32)
        got = np.stack(w, axis=1).reshape(-1)
        assert got.tolist() == words, seed


def test_philox_uniformity():
    """Chi^2 of the 64-bit draws' top 8 bits and of MH uniforms over 256 bins."""
    x = philox.draw_words(7, 5, np.arange(200000, dtype=np.uint64))
    counts = np.bincount((x >> np.uint64(56)).astype(np.int64), minlength=256)
    e = x.size / 256
    chi2 = ((counts - e) ** 2 / e).sum()
    assert 180 < chi2 < 340          # 255 dof, ~ +-4.5 sigma
    u = philox.mh_uniform(7, np.arange(200000, dtype=np.uint64), 3)
    assert u.min() >= 0 and u.max() < 1
    counts = np.bincount((u * 256).astype(np.int64), minlength=256)
    chi2 = ((counts - e) ** 2 / e).sum()
    assert 180 < chi2 < 340


def test_streams_are_distinct():
    a = philox.draw_words(1, 0, np.arange(64, dtype=np.uint64))
    b = philox.draw_words(1, 1, np.arange(64, dtype=np.uint64))
    c = philox.draw_words(2, 0, np.arange(64, dtype=np.uint64))
    assert len(set(a.tolist()) | set(b.tolist()) | set(c.tolist())) == 192


def test_energy_matches_loops():
    for inst in (instances.random_small(3, 4, 1.0, 2, seed=1), instances.villain(4, 5, 1.0, 2),
                 instances.ea_pm(5, 3, 1.0, 2, seed=2)):
        rng = np.random.default_rng(0)
        S = rng.choice([-1, 1], size=(20, inst.Ly, inst.Lx)).astype(np.int8)
        E = tnmc.energy(inst.Jh, inst.Jv, inst.h, S)
        for b in range(20):
            assert E[b] == pytest.approx(exact.energy_loops(inst.Jh, inst.Jv, inst.h, S[b]), abs=1e-12)


def test_energy_integer_and_ground_state():
    L = 6
    inst = instances.ferromagnet(L, L, 1.0, 2)
    up = np.ones((1, L, L), dtype=np.int8)
    assert tnmc.energy(inst.Jh, inst.Jv, inst.h, up)[0] == -2 * L * (L - 1)
    pm = instances.ea_pm(L, L, 1.0, 2, seed=3)
    S = np.random.default_rng(1).choice([-1, 1], size=(50, L, L)).astype(np.int8)
    E = tnmc.energy(pm.Jh, pm.Jv, pm.h, S)
    assert np.all(E == np.round(E))


def test_villain_every_plaquette_frustrated():
    inst = instances.villain(6, 8, 1.0, 2)
    for r in range(5):
        for c in range(7):
            prod = inst.Jh[r, c] * inst.Jh[r + 1, c] * inst.Jv[r, c] * inst.Jv[r, c + 1]
            assert prod == -1
