"""ccl_label_static: the entry point for callers that cannot allocate device memory (a
framework that owns all device memory through its own pool, a real-time loop that must
not stall in the allocator, a process with a fixed memory budget).  It keeps its scratch
in a fixed 16 MiB device array inside the library instead of allocating a workspace.

The test calls it through the C ABI twice in a row, on two different images, and checks
each result against the regular ccl_label (labels are integers: the bar is equality),
then checks that an image too large for the fixed scratch is refused.  It lives in a
file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _label_both(lib, img):
    import torch

    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    h, w = img.shape
    dimg = torch.from_numpy(img).cuda()
    ref = torch.full((h, w), -1, dtype=torch.int32, device="cuda")
    k_ref = ctypes.c_int32(-1)
    assert lib.ccl_label(dimg.data_ptr(), h, w, dimg.stride(0), 8, ref.data_ptr(), ctypes.byref(k_ref), s) == 0
    out = torch.full((h, w), -1, dtype=torch.int32, device="cuda")
    k_dev = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rc = lib.ccl_label_static(dimg.data_ptr(), h, w, dimg.stride(0), 8, out.data_ptr(), k_dev.data_ptr(), s)
    assert rc == 0, rc
    torch.cuda.synchronize()
    return ref.cpu().numpy(), k_ref.value, out.cpu().numpy(), int(k_dev.item())


def test_static_scratch_matches_regular_entry_point_twice():
    import paper_1606_05973_gb300 as ccl

    lib = ccl.lib()
    first = synth.bernoulli(1024, 1024, 0.5, 1)
    second = synth.bernoulli(777, 1500, 0.62, 2)  # different shape: the scratch is reused
    for img in (first, second):
        ref, k_ref, got, k = _label_both(lib, img)
        assert k == k_ref
        assert np.array_equal(got, ref)


def test_static_scratch_refuses_images_that_do_not_fit():
    import torch

    import paper_1606_05973_gb300 as ccl

    lib = ccl.lib()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    h, w = 4096, 4096  # workspace ~38 MiB > 16 MiB
    dimg = torch.zeros((h, w), dtype=torch.uint8, device="cuda")
    out = torch.zeros((h, w), dtype=torch.int32, device="cuda")
    rc = lib.ccl_label_static(dimg.data_ptr(), h, w, w, 8, out.data_ptr(), None, s)
    assert rc == 8  # CCL_ERR_TOO_LARGE
    assert "16 MiB" in ccl.ccl_status_string(rc)
