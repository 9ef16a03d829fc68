"""Failure detection without a GPU fault: a bounded mbarrier wait that nothing completes gives up
on its own, the kernel records it in a device flag and exits, the host reports CS_ERR_TIMEOUT,
and the context stays usable (a later library computation still matches the oracle bit for bit).
Host-side failures (bad arguments, NaN inputs) are covered with the operators and solvers."""
import numpy as np
import pytest

from oracle import philox

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from tests._gpu import ensure_built
    ensure_built()


def test_bounded_wait_gives_up_and_context_survives():
    import paper_2305_06482_gb300 as cs
    L = cs.lib()
    assert L.cs_wait_selftest(1, 1 << 16, None) == cs.CS_OK           # the barrier completes
    rc = L.cs_wait_selftest(0, 1 << 12, None)                         # nothing ever arrives
    assert rc == 6, rc                                                # CS_ERR_TIMEOUT
    assert b"gave up" in L.cs_last_error()
    assert L.cs_wait_selftest(0, 0, None) == 1                        # bad limit refused on the host
    # the flag was cleared and the context works: a completed wait and a device computation
    assert L.cs_wait_selftest(1, 1 << 16, None) == cs.CS_OK
    got = cs.sketch_draw(99, 0, 2, 12, 3, 4).cpu().numpy()
    want = philox.sketch_draw(99, 0, 2, 12, 3, 4)
    assert np.array_equal(got, want)
    cs.device_status()
