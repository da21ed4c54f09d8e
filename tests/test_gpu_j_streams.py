"""The fan-out batch form (every image labelled as by ccl_label_async on one of three library
streams joined back to the caller's stream), forced with ccl_set_launch_mode(3) or chosen by
ccl_set_streams_min_px, against the oracle element by element: uneven images under every
tile policy, more images than streams, two calls in a row, 4-connectivity, multi-class and
threshold batches, K left out, the launch counts, and replay from a CUDA graph (the fork and
join captured)."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture
def ccl():
    import paper_1606_05973_gb300 as ccl

    lib = ccl.lib()
    yield ccl
    lib.ccl_set_launch_mode(0)
    lib.ccl_set_tile_policy(0)
    lib.ccl_set_tuning(None, 0, 0, 0, 0, 0)  # the built-in table and its streams_min_px


def _status(ccl, stream=None):
    import torch

    flags = ctypes.c_int32(0)
    s = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    assert ccl.lib().ccl_device_status(s, ctypes.byref(flags)) == 0
    return flags.value


def _uneven():
    # sizes across several tiles in both directions with ragged edges, one image that fills
    # no whole tile, and contents below, at and above the percolation threshold
    return [synth.bernoulli(700, 1300, 0.6, 1), synth.serpentine(515, 999), synth.bernoulli(64, 512, 0.45, 2),
            synth.bernoulli(37, 41, 0.5, 3),
            synth.make_batch_image({"h": 900, "w": 1030, "kind": "blobs", "seed": 4, "p": 0.5, "sigma": 4.0}),
            synth.bernoulli(1500, 257, 0.3, 5)]


def _check(imgs, outs, ks, conn=8, prep=None):
    for im, o, k in zip(imgs, outs, ks.cpu().numpy()):
        ref, rk = oracle.cclremsp(prep(im) if prep else im, conn)
        assert k == rk and np.array_equal(o.cpu().numpy(), ref), im.shape


@pytest.mark.parametrize("policy", [0, 1, 2, 3])
def test_fanout_matches_oracle_every_tile_policy(ccl, policy):
    import torch

    lib = ccl.lib()
    assert lib.ccl_set_launch_mode(3) == 0 and lib.ccl_set_tile_policy(policy) == 0
    imgs = _uneven()
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    ccl.ccl_profile_reset()
    ccl.ccl_profile_enable(1)
    outs, ks = ccl.label_batch(dev)
    torch.cuda.synchronize()
    ccl.ccl_profile_enable(0)
    kt = ccl.kernel_times()
    n = len(imgs)  # three kernels per image, none over the batch
    assert kt["tile_local"][0] == n and kt["global_merge_flatten"][0] == n and kt["final_labels"][0] == n
    assert kt["persistent"][0] == 0
    assert _status(ccl) == 0
    _check(imgs, outs, ks)


def test_fanout_two_calls_in_a_row_other_sizes(ccl):
    """The library streams and their workspaces are reused by the next call on the same
    stream, here with larger images on some streams (the workspaces grow)."""
    import torch

    lib = ccl.lib()
    assert lib.ccl_set_launch_mode(3) == 0
    first = [synth.bernoulli(300, 400, 0.5, 6), synth.bernoulli(200, 300, 0.6, 7)]
    second = [synth.bernoulli(900, 1100, 0.55, 8), synth.serpentine(800, 600), synth.bernoulli(333, 777, 0.4, 9),
              synth.bernoulli(1200, 1000, 0.62, 10)]
    for imgs in (first, second):
        dev = [torch.from_numpy(im).cuda() for im in imgs]
        outs, ks = ccl.label_batch(dev)
        _check(imgs, outs, ks)
    assert _status(ccl) == 0


def test_fanout_chosen_by_smallest_image(ccl):
    """Under launch mode 0 the threshold is the smallest image's pixel count."""
    import torch

    lib = ccl.lib()
    imgs = [synth.bernoulli(600, 700, 0.55, 11), synth.bernoulli(300, 900, 0.5, 12)]
    dev = [torch.from_numpy(im).cuda() for im in imgs]

    def tile_launches(min_px):
        assert lib.ccl_set_streams_min_px(min_px) == 0
        ccl.ccl_profile_reset()
        ccl.ccl_profile_enable(1)
        outs, ks = ccl.label_batch(dev)
        torch.cuda.synchronize()
        ccl.ccl_profile_enable(0)
        _check(imgs, outs, ks)
        return ccl.kernel_times()["tile_local"][0]

    assert tile_launches(300 * 900) == 2      # the smaller image reaches it: one per image
    assert tile_launches(300 * 900 + 1) != 2  # one pixel short: another form
    assert tile_launches(-1) != 2
    assert _status(ccl) == 0


def test_fanout_four_connectivity_classes_threshold(ccl):
    import torch

    lib = ccl.lib()
    assert lib.ccl_set_launch_mode(3) == 0
    imgs = _uneven()[:4]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    outs, ks = ccl.label_batch(dev, connectivity=4)
    _check(imgs, outs, ks, conn=4)
    rng = np.random.default_rng(21)
    cls = [rng.integers(0, 4, size=s, dtype=np.uint8) for s in ((300, 500), (129, 257), (64, 64))]
    dcls = [torch.from_numpy(im).cuda() for im in cls]
    for conn in (8, 4):
        outs, ks = ccl.label_batch(dcls, connectivity=conn, classes=True)
        for im, o, k in zip(cls, outs, ks.cpu().numpy()):
            ref, rk = oracle.classes(im, conn)
            assert k == rk and np.array_equal(o.cpu().numpy(), ref), conn
    grey = [rng.integers(0, 256, size=s, dtype=np.uint8) for s in ((400, 333), (250, 700))]
    dgrey = [torch.from_numpy(im).cuda() for im in grey]
    outs, ks = ccl.label_batch(dgrey, threshold=140)
    _check(grey, outs, ks, prep=lambda im: oracle.binarize(im, 140))
    assert _status(ccl) == 0


def test_fanout_without_k_and_graph_replay(ccl):
    import torch

    lib = ccl.lib()
    assert lib.ccl_set_launch_mode(3) == 0 and lib.ccl_set_tile_policy(3) == 0  # big tiles
    imgs = [synth.bernoulli(1100, 1500, 0.6, 31), synth.serpentine(700, 1600), synth.bernoulli(513, 1025, 0.5, 32),
            synth.bernoulli(260, 1900, 0.45, 33)]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    refs = [oracle.cclremsp(im) for im in imgs]
    outs = [torch.full(im.shape, -3, dtype=torch.int32, device="cuda") for im in imgs]
    descs = (ccl.ImageDesc * len(imgs))()
    for i, (d, o) in enumerate(zip(dev, outs)):
        descs[i].img, descs[i].H, descs[i].W = d.data_ptr(), d.shape[0], d.shape[1]
        descs[i].pitch_bytes, descs[i].labels = d.stride(0), o.data_ptr()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    sp = ctypes.c_void_p(s.cuda_stream)
    assert lib.ccl_label_batch(descs, len(imgs), 8, None, sp) == 0  # K left out; sizes the workspaces
    s.synchronize()
    for o, (ref, _) in zip(outs, refs):
        assert np.array_equal(o.cpu().numpy(), ref)
        o.fill_(-1)
    torch.cuda.synchronize()
    kd = torch.full((len(imgs),), -1, dtype=torch.int32, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert lib.ccl_label_batch(descs, len(imgs), 8, ctypes.c_void_p(kd.data_ptr()), sp) == 0
    g.replay()
    torch.cuda.synchronize()
    for o, k, (ref, rk) in zip(outs, kd.cpu().numpy(), refs):
        assert k == rk and np.array_equal(o.cpu().numpy(), ref)
    assert _status(ccl, s) == 0
