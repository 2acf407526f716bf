"""fibar_queue_counts_noalloc against fibar_debug_state (collected last on purpose: it must
pass after the other GPU tests as well as alone in a fresh process)."""
import ctypes as C

import numpy as np
import pytest

import eventsim

pytestmark = pytest.mark.gpu


def _handle(W, H, **params):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_20071_gb300 import Fibar
    return torch, Fibar(W, H, c_on=0.2, c_off=0.2, **params)


@pytest.mark.parametrize("mode", [dict(spatial_filter=1, blur_mode=1), dict(spatial_filter=1, blur_mode=0),
                                  dict(spatial_filter=0)])
def test_counts_match_debug_state_twice(mode):
    from paper_2510_20071_gb300 import binding
    W, H = 240, 180
    torch, f = _handle(W, H, **mode)
    ev = eventsim.make_config("sine_checker_240x180_1M", n_events=300_000, device="cuda")
    dev_out = torch.full((H, W), -1, dtype=torch.int32, device="cuda")
    host_out = np.full(W * H, 0xFFFFFFFF, dtype=np.uint32)
    for lo, hi in [(0, 120_000), (120_000, 300_000)]:
        f.push(ev[lo:hi])
        f.readout(int(ev[hi - 1, 1].item()), torch.empty((H, W), dtype=torch.float32, device="cuda"))
        ref = f.state()["cnt"]
        # two calls in a row, device and host output, through the C ABI
        for _ in range(2):
            rc = binding.fibar_queue_counts_noalloc(f.h, dev_out.data_ptr(), 1, f._s)
            assert rc == 0, binding.fibar_last_error(f.h)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(dev_out.cpu().numpy().reshape(-1).view(np.uint32), ref)
            rc = binding.fibar_queue_counts_noalloc(f.h, host_out.ctypes.data, 0, f._s)
            assert rc == 0, binding.fibar_last_error(f.h)
            np.testing.assert_array_equal(host_out, ref)
        if mode.get("spatial_filter", 1):
            assert int(ref.sum()) == f.state()["q"] > 0
    f.close()


def test_rejects_sensors_beyond_the_buffer():
    from paper_2510_20071_gb300 import binding
    torch, f = _handle(1280, 1024, spatial_filter=1, blur_mode=1)  # 1,310,720 pixels > 2^20
    out = torch.empty(1280 * 1024, dtype=torch.int32, device="cuda")
    rc = binding.fibar_queue_counts_noalloc(f.h, out.data_ptr(), 1, f._s)
    assert rc == binding.FIBAR_EINVAL
    assert "exceeds its fixed buffer" in binding.fibar_last_error(f.h)
    f.close()
