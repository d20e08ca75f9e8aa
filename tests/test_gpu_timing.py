"""The encode's device time (aqmp_last_device_ms): CUDA events the library
records around its kernels, on the stream that runs them.  It is positive
after an encode, no longer than the caller's own events around the same
call (which also hold the call's host work), and it covers the kernels: at
least the sum of their profiled launch times."""
import numpy as np
import pytest

from paper_2605_09190_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2605_09190_gb300 import aqmp, build_lib
    build_lib.build()
    aqmp.load_library()
    assert torch.cuda.is_available()
    return aqmp


def test_device_time_lies_within_the_call_and_covers_its_kernels(lib):
    planes = [torch.from_numpy(synthetic.gradient_scene(512, 512, seed=s)).cuda() for s in range(3)]
    stream = torch.cuda.current_stream()
    for graphs in range(4):                      # the first calls run eagerly, later ones replay a graph
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        code = lib.aqmp_encode_planes(planes, 2.0)
        e1.record(stream)
        dev = lib.aqmp_last_device_ms()
        e1.synchronize()
        caller = e0.elapsed_time(e1)
        code.free()
        assert 0.0 < dev <= caller * (1 + 1e-3) + 1e-3, (graphs, dev, caller)
    lib.aqmp_profile_reset()
    lib.aqmp_profile_enable(True)
    code = lib.aqmp_encode_planes(planes, 2.0)
    dev = lib.aqmp_last_device_ms()
    code.free()
    lib.aqmp_profile_enable(False)
    prof = lib.aqmp_profile_read()
    kernels_ms = sum(v[1] for v in prof.values())
    assert kernels_ms > 0.0
    assert dev >= 0.98 * kernels_ms, (dev, kernels_ms)
    assert np.isfinite(dev)
