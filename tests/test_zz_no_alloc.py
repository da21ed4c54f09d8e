"""ccl_label_static: the entry point for callers that cannot allocate device memory (a
framework that owns all device memory through its own pool, a real-time loop that must
not stall in the allocator, a process with a fixed memory budget).  It keeps its scratch
in a fixed 16 MiB device array inside the library instead of allocating a workspace.

The tests call it through the C ABI and compare each result with the regular ccl_label
(labels are integers: the bar is equality): twice in a row on two different images, under
4-connectivity, with K left in the scratch (NULL num_components_dev), and on the largest
image that fits the scratch, whose one-row-taller neighbour is refused.  The status word
of the scratch is read (and cleared) without allocating after each call.  This file is
collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOO_LARGE = 8


def _static_status(lib, s):
    flags = ctypes.c_int32(-1)
    assert lib.ccl_label_static_status(s, ctypes.byref(flags)) == 0
    return flags.value


def _label_both(lib, img, conn=8, with_k=True):
    import torch

    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    h, w = img.shape
    dimg = torch.from_numpy(img).cuda()
    ref = torch.full((h, w), -1, dtype=torch.int32, device="cuda")
    k_ref = ctypes.c_int32(-1)
    assert lib.ccl_label(dimg.data_ptr(), h, w, dimg.stride(0), conn, ref.data_ptr(), ctypes.byref(k_ref), s) == 0
    out = torch.full((h, w), -1, dtype=torch.int32, device="cuda")
    k_dev = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rc = lib.ccl_label_static(dimg.data_ptr(), h, w, dimg.stride(0), conn, out.data_ptr(),
                              k_dev.data_ptr() if with_k else None, s)
    assert rc == 0, rc
    torch.cuda.synchronize()
    assert _static_status(lib, s) == 0
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


def test_static_scratch_four_connectivity_and_k_in_scratch():
    import paper_1606_05973_gb300 as ccl

    lib = ccl.lib()
    img = synth.bernoulli(901, 1333, 0.55, 5)
    ref, k_ref, got, k = _label_both(lib, img, conn=4)
    assert k == k_ref and np.array_equal(got, ref)
    ref, _, got, k = _label_both(lib, img, conn=8, with_k=False)  # K goes to the scratch header
    assert k == -1 and np.array_equal(got, ref)


def test_static_scratch_size_limit_from_both_sides():
    """The largest height that fits at width 2048 is found by asking the entry point; that
    image is labelled exactly, and one row more is refused with nothing launched."""
    import torch

    import paper_1606_05973_gb300 as ccl

    lib = ccl.lib()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    w = 2048
    dimg = torch.zeros((4096, w), dtype=torch.uint8, device="cuda")
    out = torch.zeros((4096, w), dtype=torch.int32, device="cuda")

    def fits(h):
        rc = lib.ccl_label_static(dimg.data_ptr(), h, w, w, 8, out.data_ptr(), None, s)
        assert rc in (0, TOO_LARGE), rc
        return rc == 0

    lo, hi = 1, 4096  # fits(lo), not fits(hi)
    assert fits(lo) and not fits(hi)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if fits(mid):
            lo = mid
        else:
            hi = mid
    torch.cuda.synchronize()
    assert _static_status(lib, s) == 0
    img = synth.bernoulli(lo, w, 0.5, 7)
    ref, k_ref, got, k = _label_both(lib, img)
    assert k == k_ref and np.array_equal(got, ref)
    assert not fits(lo + 1)


def test_static_scratch_refuses_images_that_do_not_fit():
    import torch

    import paper_1606_05973_gb300 as ccl

    lib = ccl.lib()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    h, w = 4096, 4096  # workspace ~38 MiB > 16 MiB
    dimg = torch.zeros((h, w), dtype=torch.uint8, device="cuda")
    out = torch.zeros((h, w), dtype=torch.int32, device="cuda")
    rc = lib.ccl_label_static(dimg.data_ptr(), h, w, w, 8, out.data_ptr(), None, s)
    assert rc == TOO_LARGE
    assert "16 MiB" in ccl.ccl_status_string(rc)
