"""Failure detection on the GPU without faulting it: a bounded device wait
is made to run out (a barrier nothing arrives on) and must come back as
AQMP_E_TIMEOUT with the device still usable; host-made overflows and bad
arguments come back as error codes."""
import time

import numpy as np
import pytest

import oracle
from paper_2605_09190_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2605_09190_gb300 import aqmp, build_lib
    build_lib.build()
    assert torch.cuda.is_available()
    return aqmp


def test_bounded_wait_times_out_and_the_device_stays_usable(lib):
    t0 = time.perf_counter()
    rc = lib.aqmp_selftest_wait(50)
    dt = time.perf_counter() - t0
    assert rc == -7, lib.load_library().aqmp_last_error()
    assert 0.04 <= dt < 5.0
    # the context still works: an encode right after matches the oracle
    img = synthetic.gradient_scene(64, 64, seed=3)
    leaves, atoms, _ = lib.aqmp_encode_planes([torch.from_numpy(img).cuda()], [1.5]).copy()
    enc = oracle.encode([img], [1.5])
    assert np.array_equal(atoms["j"].astype(np.int64), enc.atom_j.astype(np.int64))


def test_argument_errors_leave_no_result(lib):
    img = torch.zeros((64, 96), dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.AqmpError) as e:
        lib.aqmp_encode_planes([img], [2.0])
    assert e.value.code == -2
