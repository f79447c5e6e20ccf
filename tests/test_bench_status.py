"""bench.py withholds a timed leg whose kernels recorded a device timeout
(a bounded wait that ran out): the status word is read after every timed
region, and such a leg reports no value.  CPU only: torch's CUDA calls are
replaced by a stand-in that records nothing, and the status word by a stub."""
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Event:
    def __init__(self, enable_timing=False):
        self.t = 0.0

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 1.5


def fake_torch():
    cuda = types.SimpleNamespace(Event=_Event, synchronize=lambda: None,
                                 current_stream=lambda: None)
    return types.SimpleNamespace(cuda=cuda)


@pytest.fixture
def status(monkeypatch):
    state = {"err": None, "reads": 0}

    def reader():
        state["reads"] += 1
        err, state["err"] = state["err"], None   # reading clears it, as the library does
        return err

    monkeypatch.setattr(bench, "STATUS_READER", reader)
    return state


def test_clean_leg_reports_its_time(status):
    total, kms = bench.time_steps(fake_torch(), lambda kev: None, 4, 3, None)
    assert total == 1.5 and kms is None
    assert status["reads"] == 1


def test_leg_with_device_timeout_is_withheld(status):
    def step(kev):
        status["err"] = "qadic status 7: bounded wait expired (site 3)"

    with pytest.raises(bench.LegWithheld):
        bench.time_steps(fake_torch(), step, 4, 3, None)
    rec = bench.guarded(bench.time_steps, fake_torch(), step, 4, 3, None)
    assert rec["status"] == "device_timeout" and rec["value"] is None
    assert "bounded wait" in rec["error"]


def test_timeout_in_warmup_also_withholds(status):
    calls = {"n": 0}

    def step(kev):
        calls["n"] += 1
        if calls["n"] == 1:          # first warm-up step only
            status["err"] = "qadic status 7: expired"

    rec = bench.guarded(bench.time_steps, fake_torch(), step, 2, 3, None)
    assert rec["status"] == "device_timeout"


def test_guarded_passes_results_through(status):
    assert bench.guarded(lambda a, b=0: {"value": a + b}, 1, b=2) == {"value": 3}


def test_library_reader_maps_timeout_only():
    class Err(RuntimeError):
        def __init__(self, st):
            super().__init__(f"status {st}")
            self.status = st

    def fake_q(st):
        def sync_status():
            if st:
                raise Err(st)
        return types.SimpleNamespace(sync_status=sync_status, QadicError=Err,
                                     E_DEVICE_TIMEOUT=7)

    assert bench.library_status_reader(fake_q(0))() is None
    assert "7" in bench.library_status_reader(fake_q(7))()
    with pytest.raises(Err):           # any other error is not a timeout: it propagates
        bench.library_status_reader(fake_q(6))()


def test_plane_kernel_label_follows_the_dispatch_rule():
    """The roofline names the kernel that runs: CTA pairs for GF(101^2) at
    n = 4096 (K = 4096 within one exact chunk of 6656), one CTA per tile for
    GF(251^2) at n = 16384 (chunk of 1073 K elements) and for one tile row."""
    assert bench.plane_kernel(101, 4096) == "gemm_planes_pair_kernel<2,128,false>"
    assert bench.plane_kernel(251, 16384) == "gemm_planes_tc_kernel<2,128,false>"
    assert bench.plane_kernel(101, 128) == "gemm_planes_tc_kernel<2,128,false>"
    assert bench.plane_kernel(101, 6656) == "gemm_planes_pair_kernel<2,128,false>"
    assert bench.plane_kernel(101, 6657) == "gemm_planes_tc_kernel<2,128,false>"
