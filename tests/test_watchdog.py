"""The host-side watchdog on stream completion (binding.wait): the failure is
made on the host with a fake event (no GPU, nothing hangs): a stream that never
completes raises DG_E_TIMEOUT after the limit, one that completes after a few
polls returns."""
import time

import pytest


class FakeEvent:
    def __init__(self, done_after):
        self.polls, self.done_after = 0, done_after

    def query(self):
        self.polls += 1
        return self.done_after is not None and self.polls > self.done_after


@pytest.fixture(scope="module")
def B():
    from paper_1806_02343_gb300 import build, binding
    build.build()
    return binding


def test_wait_times_out_on_a_stream_that_never_completes(B):
    ev = FakeEvent(None)
    t0 = time.monotonic()
    with pytest.raises(B.DGError) as e:
        B.wait(timeout_s=0.05, poll_s=1e-3, event=ev)
    assert e.value.code == B.DG_E_TIMEOUT == -6
    assert 0.05 <= time.monotonic() - t0 < 2.0 and ev.polls > 3
    assert str(e.value).endswith("(-6)")


def test_wait_returns_once_the_stream_completes(B):
    ev = FakeEvent(3)
    B.wait(timeout_s=5.0, poll_s=1e-4, event=ev)
    assert ev.polls == 4
