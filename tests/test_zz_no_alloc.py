"""fibar_queue_counts_noalloc against fibar_debug_state (collected last on purpose: it must
pass after the other GPU tests as well as alone in a fresh process).

The entry point serves callers that cannot allocate device memory once they run: it
counts into a fixed buffer built into the library.  The test calls it on a fresh handle
before anything else has allocated the debug counters, checks that device memory stays
unchanged over the later calls, and compares the counts with fibar_debug_state's."""
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
    img = torch.empty((H, W), dtype=torch.float32, device="cuda")
    for step, (lo, hi) in enumerate([(0, 120_000), (120_000, 300_000)]):
        f.push(ev[lo:hi])
        f.readout(int(ev[hi - 1, 1].item()), img)
        got = []
        # calls in a row, device and host output, through the C ABI; on the fresh handle
        # they come before any fibar_debug_state call
        for i in range(3):
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            rc = binding.fibar_queue_counts_noalloc(f.h, dev_out.data_ptr(), 1, f._s)
            assert rc == 0, binding.fibar_last_error(f.h)
            torch.cuda.synchronize()
            got.append(dev_out.cpu().numpy().reshape(-1).view(np.uint32).copy())
            rc = binding.fibar_queue_counts_noalloc(f.h, host_out.ctypes.data, 0, f._s)
            assert rc == 0, binding.fibar_last_error(f.h)
            got.append(host_out.copy())
            if i > 0 or step > 0:
                # the first call may load the library's device code; later ones allocate nothing
                assert torch.cuda.mem_get_info()[0] == free0
        ref = f.state()["cnt"]
        for g in got:
            np.testing.assert_array_equal(g, ref)
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
