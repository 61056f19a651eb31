"""tnmc_sample_noalloc through the C ABI (needs a GB300).

The entry point serves callers that cannot let the library allocate device
memory (a fixed budget owned by another allocator, or loops where an
allocation or the synchronisation of a cudaFree is not acceptable).  It must
give the same proposals as tnmc_sample, and it must not allocate: a counting
device-memory hook (tnmc_set_allocator) sees every allocation the library makes,
and none may happen during the call.  Two calls in a row check that the shared
fixed scratch carries nothing from one call into the next.  This file is
collected last so a failure here comes after every other test has run.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _call_noalloc(L, env, prec, n, seed, offset):
    dev = torch.device("cuda")
    sp = torch.empty((n, env.Ly, env.Lx), dtype=torch.int8, device=dev)
    lq = torch.empty(n, dtype=torch.float64, device=dev)
    E = torch.empty(n, dtype=torch.float64, device=dev)
    fl = torch.empty(n, dtype=torch.int32, device=dev)
    st = L.tnmc_sample_noalloc(env.handle, prec, n, seed, offset, ctypes.c_void_p(sp.data_ptr()),
                               ctypes.c_void_p(lq.data_ptr()), ctypes.c_void_p(E.data_ptr()),
                               ctypes.c_void_p(fl.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, L.tnmc_last_error()
    return sp, lq, E, fl


@pytest.mark.parametrize("prec_name", ["f64", "f32"])
def test_noalloc_matches_sample_twice(prec_name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_13264_gb300 import binding, instances
    L = binding.lib()
    prec = binding.PRECISIONS[prec_name]
    inst = instances.ea_pm(20, 24, 1.0, 16, seed=3)
    env = binding.Env.from_instance(inst, precisions=("f64", "f32"))
    for call, (n, seed, offset) in enumerate([(3001, 5, 0), (1777, 6, 12345)]):
        got = _call_noalloc(L, env, prec, n, seed, offset)
        ref = binding.sample(env, n, seed=seed, sample_offset=offset, precision=prec_name)
        torch.cuda.synchronize()
        assert torch.equal(got[0], ref[0]), "spins differ on call %d" % call
        assert torch.allclose(got[1], ref[1], rtol=0, atol=1e-9), "log q differs on call %d" % call
        assert torch.equal(got[2], ref[2]) and torch.equal(got[3], ref[3])
    env.free()


def test_noalloc_makes_no_allocation():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_13264_gb300 import binding, instances
    L = binding.lib()
    calls = {"alloc": 0, "free": 0}

    def _alloc(nbytes, stream, ctx):
        calls["alloc"] += 1
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        except Exception:  # noqa: BLE001 -- out of memory: the library reports it
            return None

    def _free(ptr, nbytes, stream, ctx):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    hooks = (binding.ALLOC_FN(_alloc), binding.FREE_FN(_free))
    assert L.tnmc_set_allocator(ctypes.cast(hooks[0], ctypes.c_void_p), ctypes.cast(hooks[1], ctypes.c_void_p), None) == 0
    try:
        inst = instances.ea_pm(20, 24, 1.0, 16, seed=4)
        env = binding.Env.from_instance(inst, precisions=("f64", "f32"))
        torch.cuda.synchronize()
        assert calls["alloc"] > 0                      # the hook does see the library's allocations
        ref = binding.sample(env, 2049, seed=9, precision="f32")   # grows the env's own scratch
        torch.cuda.synchronize()
        before = dict(calls)
        got = _call_noalloc(L, env, binding.PRECISIONS["f32"], 2049, 9, 0)
        torch.cuda.synchronize()
        assert calls == before, (before, calls)
        assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])
        env.free()
    finally:
        assert L.tnmc_set_allocator(None, None, None) == 0
