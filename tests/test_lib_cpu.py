"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, exports every
symbol include/fibar.h declares, its structs match the binding, and host-side argument
validation rejects bad input before any CUDA call."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fibar.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(fibar_\w+)\s*\(", src, re.M)))


def test_header_declarations_match_binding():
    from paper_2510_20071_gb300 import EXPORTED
    assert declared_functions() == sorted(EXPORTED)


def test_library_builds_and_exports_every_symbol():
    from paper_2510_20071_gb300 import build
    lib = build.build()
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib]).decode()
    syms = set(re.findall(r" T (\w+)", out))
    for name in declared_functions():
        assert name in syms, name
    C.CDLL(lib)  # loads


def test_struct_layouts_match_header(tmp_path):
    from paper_2510_20071_gb300 import FibarParams, FibarStateView, FibarStats
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "fibar.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(fibar_event_t), sizeof(fibar_params_t),
         sizeof(fibar_stats_t), sizeof(fibar_state_view_t), offsetof(fibar_params_t, max_pending),
         offsetof(fibar_state_view_t, n_at));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = list(map(int, subprocess.check_output([str(exe)]).split()))
    assert vals == [16, C.sizeof(FibarParams), C.sizeof(FibarStats), C.sizeof(FibarStateView),
                    FibarParams.max_pending.offset, FibarStateView.n_at.offset]


def test_defaults_and_host_validation():
    import paper_2510_20071_gb300 as fb
    p = fb.fibar_default_params()
    assert p.t_cut == 40.0 and p.fill_num == 1 and p.fill_den == 2
    assert p.c_on == 1.0 and p.c_off == 1.0 and p.spatial_filter == 1 and p.blur_mode == 0
    # rejected by parameter checks, before any CUDA call
    for (W, H, over) in [(0, 8, {}), (8, 0, {}), (5000, 5000, {}), (8, 8, dict(t_cut=3.0)),
                         (8, 8, dict(fill_num=0)), (8, 8, dict(fill_den=300)), (8, 8, dict(c_on=0.0)),
                         (8, 8, dict(blur_mode=3)), (8, 8, dict(q_min=65)), (8, 8, dict(q_min=4, q_init=2)),
                         (8, 8, dict(max_pending=1 << 28))]:
        q = fb.fibar_default_params()
        for k, v in over.items():
            setattr(q, k, v)
        rc, h = fb.fibar_create(W, H, q)
        assert rc == fb.FIBAR_EINVAL and not h.value


def test_binding_refuses_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2510_20071_gb300 as fb
    with pytest.raises(fb.FibarError):
        fb.Fibar(8, 8)


def test_group_and_batch_entry_points_reject_bad_arguments_without_a_device():
    """The serving entry points check their arguments before any CUDA call."""
    import array
    import paper_2510_20071_gb300 as fb
    lib = fb.load_library()
    rc, g = fb.fibar_group_create([])
    assert rc == fb.FIBAR_EINVAL and not g.value
    out = C.c_void_p()
    assert lib.fibar_group_create(None, 1, C.byref(out)) == fb.FIBAR_EINVAL
    assert lib.fibar_group_create((C.c_void_p * 1)(None), 1025, C.byref(out)) == fb.FIBAR_EINVAL
    assert lib.fibar_group_create((C.c_void_p * 1)(None), 1, None) == fb.FIBAR_EINVAL
    assert fb.fibar_group_readout(None, 0, 0, 0, 1, None, None, 0) == fb.FIBAR_EINVAL
    assert fb.fibar_group_join(None, 0) == fb.FIBAR_EINVAL
    assert fb.fibar_group_latency(None, 0, 0, 0) == fb.FIBAR_EINVAL
    assert fb.fibar_group_stats(None, fb.FibarGroupStats()) == fb.FIBAR_EINVAL
    assert fb.fibar_group_last_error(None) == "null group"
    fb.fibar_group_destroy(None)
    assert fb.fibar_set_grid_share(None, 8) == fb.FIBAR_EINVAL
    # batched pushes: nothing to do, missing arrays, and a NULL handle per entry
    assert fb.fibar_push_batch(0, 0, 0, 0, 1, None, 0) == fb.FIBAR_OK
    assert fb.fibar_push_batch(0, 0, 0, 2, 1, None, 0) == fb.FIBAR_EINVAL
    hs, ptrs, ns = array.array("Q", [0, 0]), array.array("Q", [16, 32]), array.array("Q", [1, 1])
    status = array.array("i", [7, 7])
    rc = fb.fibar_push_batch(hs.buffer_info()[0], ptrs.buffer_info()[0], ns.buffer_info()[0], 2, 1,
                             status.buffer_info()[0], 0)
    assert rc == fb.FIBAR_EINVAL and list(status) == [fb.FIBAR_EINVAL, fb.FIBAR_EINVAL]
    # batched read-outs: nothing to do, then missing arrays
    assert fb.fibar_readout_batch([], [], [], None, None, 0) == fb.FIBAR_OK
    assert lib.fibar_readout_batch(None, None, None, 1, None, None, None) == fb.FIBAR_EINVAL


def test_group_stats_layout_matches_header(tmp_path):
    from paper_2510_20071_gb300 import FibarGroupStats
    prog = tmp_path / "gl.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "fibar.h"
int main(void) {
  printf("%zu %zu\\n", sizeof(fibar_group_stats_t), offsetof(fibar_group_stats_t, programmatic_edges));
  return 0;
}
""")
    exe = tmp_path / "gl"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = list(map(int, subprocess.check_output([str(exe)]).split()))
    assert vals == [C.sizeof(FibarGroupStats), FibarGroupStats.programmatic_edges.offset]
