"""Failure detection without a GPU fault: the convolution's device waits are
bounded (1 s of wall time), and a wait that gives up sets the handle's device
error word, which sbim_check_device reports as SBIM_ERR_TIMEOUT.  The self-test
entry point makes such a wait run out on purpose (a barrier nothing completes);
the handle then keeps stepping correctly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CS, CP, RHO = 3464.0, 6000.0, 2670.0


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_bounded_wait_reports_and_handle_recovers():
    import time
    from paper_2102_08756_gb300 import sbim as B
    from paper_2102_08756_gb300.sbim import SBIM
    n, n_cut, dt = 32, 12, 0.3 * 100.0 / CP
    g = torch.Generator(device="cuda").manual_seed(9)
    x = [torch.randn((3, n, n), device="cuda", generator=g) * 1e-3 for _ in range(20)]
    a = SBIM(n, n, n * 100.0, n * 100.0, CS, CP, RHO, dt, n_cut, 1, "fp32", True)
    ref = SBIM(n, n, n * 100.0, n * 100.0, CS, CP, RHO, dt, n_cut, 1, "fp32", True)
    for m in range(8):
        a.step(x[m], x[m + 1])
        ref.step(x[m], x[m + 1])
    t0 = time.perf_counter()
    B.sbim_selftest_wait_timeout(a.h)        # raises unless the timeout was reported
    took = time.perf_counter() - t0
    assert 0.9 < took < 30.0, took           # the wait gave up after its 1 s limit
    a.check()                                # the error word is clear again
    for m in range(8, 18):                   # the handle keeps working, bit for bit
        assert torch.equal(a.step(x[m], x[m + 1]), ref.step(x[m], x[m + 1]))
    a.check()
    ref.check()
