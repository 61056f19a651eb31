"""The device-memory hook (tnmc_set_allocator) with PyTorch's caching allocator (needs a GB300).

Results must not depend on who owns the memory: an env built and sampled with every
allocation in torch's caching allocator equals one built with the default allocator,
bit for bit, and every byte goes back to torch when the objects are freed.
"""
import numpy as np
import pytest

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


def test_torch_caching_allocator_hook(B):
    inst = instances.random_small(6, 9, 0.9, 4, seed=4)
    precs = ("f64", "f32", "bf16")
    ref_env = B.Env.from_instance(inst, precisions=precs)
    ref = [B.sample(ref_env, 300, seed=2, precision=p) for p in precs]
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    B.use_torch_allocator()
    try:
        env = B.Env.from_instance(inst, precisions=precs)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() - before >= env.info()["bytes"]
        assert np.array_equal(env.export()["tensors"], ref_env.export()["tensors"])
        for p, r in zip(precs, ref):
            out = B.sample(env, 300, seed=2, precision=p)
            for x, y in zip(out, r):
                assert torch.equal(x, y)
            lq, E, fl = B.logq(env, out[0], precision=p)
            assert torch.equal(lq, out[1])
        # the MH scan's temporary and a batch plan allocate through the hook as well
        chain = B.init_chains(env, 4, seed=1)
        acc = B.mh_step(env, 4, 75, out[:3], chain, seed=3)
        plan = B.Batch([env], [256], chains=4, precision="f32", tile=128, order="cost")
        props = plan.alloc_proposals()
        plan.set_step(1, 0)
        plan.sample(props)
        single = B.sample(env, 256, seed=1, sample_offset=0, precision="f32")
        assert torch.equal(plan.view(props[0], 0), single[0])
        torch.cuda.synchronize()
        del chain, acc, props, single, out, lq, E, fl
        plan.free()
        env.free()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() - before < (1 << 20)
    finally:
        B.use_default_allocator()
    # objects created afterwards use the default allocator again
    env2 = B.Env.from_instance(inst, precisions=("f64",))
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() - before < (1 << 20)
    assert torch.equal(B.sample(env2, 300, seed=2)[1], ref[0][1])
    env2.free()
