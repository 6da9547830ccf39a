"""Failures made on the host, with the GPU left healthy: a forced device
allocation failure (fire_debug_fail_alloc) is reported as FIRE_ENOMEM and
leaves the context usable."""
import numpy as np
import pytest

from paper_1701_03549_gb300 import synth, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("after", [0, 1])
def test_forced_allocation_failure_leaves_the_context_usable(after):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1701_03549_gb300 import fire

    wl = workloads.single_fire_128(replicates=8)
    ref_ctx = fire.Context(0)
    ref_m = ref_ctx.landscape_upload(wl.land)
    want, _ = ref_m.simulate_batch(wl.params, wl.ignitions, wl.seeds)
    # fresh, with the state in global memory: its first host-pointer call
    # grows two buffers (argument staging, then the state buffers)
    ctx = fire.Context(0)
    ctx.set_launch(4, 0, 0, fire.STATE_GLOBAL)
    m = ctx.landscape_upload(wl.land)
    ctx.debug_fail_alloc(after)
    with pytest.raises(fire.FireError) as e:
        m.simulate_batch(wl.params, wl.ignitions, wl.seeds)
    assert e.value.code == fire.FIRE_ENOMEM
    assert "fire_debug_fail_alloc" in str(e.value)
    got, _ = m.simulate_batch(wl.params, wl.ignitions, wl.seeds)
    assert np.array_equal(got, want)
    got2, _ = m.simulate_batch(wl.params, wl.ignitions, wl.seeds)
    assert np.array_equal(got2, want)
    m.free()
    ctx.close()
    ref_m.free()
    ref_ctx.close()
