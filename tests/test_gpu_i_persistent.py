"""The persistent single-launch path (one cooperative kernel for the tile pass, the boundary
merge, flatten and the labelling pass; forced with ccl_set_launch_mode(2)) against the
oracle and against the three-kernel path, element by element: single images, batches of
uneven images under every tile policy and under each density class of the tuning table's
probe, 4-connectivity, multi-class, and replay from a CUDA graph."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture
def lib():
    import paper_1606_05973_gb300 as ccl

    h = ccl.lib()
    yield h
    h.ccl_set_launch_mode(0)
    h.ccl_set_tile_policy(0)


def _label(lib, img, conn=8, mode=0):
    import torch

    import paper_1606_05973_gb300 as ccl

    assert lib.ccl_set_launch_mode(mode) == 0
    lab, k = ccl.label(torch.from_numpy(img).cuda(), connectivity=conn)
    flags = ctypes.c_int32(0)
    lib.ccl_device_status(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(flags))
    assert flags.value == 0
    return lab.cpu().numpy(), k


SHAPES = [(1, 1), (1, 300), (300, 1), (63, 255), (64, 256), (65, 257), (129, 1000), (700, 333), (1024, 1024),
          (2048, 2048)]


@pytest.mark.parametrize("h,w", SHAPES)
@pytest.mark.parametrize("p", [0.1, 0.45, 0.9])
def test_single_images_persistent_equals_three_kernels_and_oracle(lib, h, w, p):
    img = synth.bernoulli(h, w, p, h * 7 + w)
    ref, rk = oracle.cclremsp(img)
    a, ka = _label(lib, img, mode=2)
    b, kb = _label(lib, img, mode=1)
    assert ka == kb == rk
    assert np.array_equal(a, ref) and np.array_equal(b, ref)


@pytest.mark.parametrize("conn", [4, 8])
def test_single_serpentine_and_blobs(lib, conn):
    for img in (synth.serpentine(999, 1501), synth.blobs(1200, 900, 6.0, 3)):
        ref, rk = oracle.cclremsp(img, conn)
        got, k = _label(lib, img, conn=conn, mode=2)
        assert k == rk and np.array_equal(got, ref)


def _batch(lib, imgs, conn=8, classes=False):
    import torch

    import paper_1606_05973_gb300 as ccl

    assert lib.ccl_set_launch_mode(2) == 0
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    labs, kd = ccl.label_batch(dev, connectivity=conn, classes=classes)
    torch.cuda.synchronize()
    flags = ctypes.c_int32(0)
    lib.ccl_device_status(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(flags))
    assert flags.value == 0
    return [x.cpu().numpy() for x in labs], kd.cpu().tolist()


@pytest.mark.parametrize("policy", [0, 1, 2])
def test_batch_every_tile_policy(lib, policy):
    specs = synth.batch_specs(n=40, seed=5 + policy, lo=8, hi=1500)
    imgs = [synth.make_batch_image(s) for s in specs]
    assert lib.ccl_set_tile_policy(policy) == 0
    labs, ks = _batch(lib, imgs)
    for im, lab, k in zip(imgs, labs, ks):
        ref, rk = oracle.cclremsp(im)
        assert k == rk and np.array_equal(lab, ref)


@pytest.mark.parametrize("p", [0.05, 0.5, 0.95])
def test_batch_in_each_density_class(lib, p):
    """A tuning table (ccl_set_tuning) whose density classes take different tile shapes,
    so the on-device probe decides: three 576 x 576 images at a density in each class."""
    import paper_1606_05973_gb300 as ccl

    rows = (ccl.TuneRow * 1)()
    rows[0].max_px = -1
    rows[0].shape[0], rows[0].shape[1], rows[0].shape[2] = 0, 1, 0
    rows[0].ctas_per_sm = 6
    rows[0].persistent = 1
    assert lib.ccl_set_tuning(rows, 1, 300, 700, 64, 0) == 0
    try:
        imgs = [synth.bernoulli(576, 576, p, 60 + i) for i in range(3)]
        labs, ks = _batch(lib, imgs)
    finally:
        assert lib.ccl_set_tuning(None, 0, 0, 0, 0, 0) == 0
    for im, lab, k in zip(imgs, labs, ks):
        ref, rk = oracle.cclremsp(im)
        assert k == rk and np.array_equal(lab, ref)


def test_batch_four_connectivity_and_classes(lib):
    imgs = [synth.bernoulli(300 + 37 * i, 200 + 91 * i, 0.5, 70 + i) for i in range(6)]
    labs, ks = _batch(lib, imgs, conn=4)
    for im, lab, k in zip(imgs, labs, ks):
        ref, rk = oracle.cclremsp(im, 4)
        assert k == rk and np.array_equal(lab, ref)
    rng = np.random.Generator(np.random.PCG64(3))
    cls = [(im * rng.integers(1, 5, im.shape)).astype(np.uint8) for im in imgs]
    labs, ks = _batch(lib, cls, conn=8, classes=True)
    for im, lab, k in zip(cls, labs, ks):
        ref, rk = oracle.classes(im, 8)
        assert k == rk and np.array_equal(lab, ref)


def test_batch_graph_replay_persistent(lib):
    import torch

    import paper_1606_05973_gb300 as ccl

    specs = synth.batch_specs(n=64, seed=9, lo=16, hi=700)
    imgs = [synth.make_batch_image(s) for s in specs]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.full(im.shape, -1, dtype=torch.int32, device="cuda") for im in imgs]
    kd = torch.full((len(imgs),), -1, dtype=torch.int32, device="cuda")
    assert lib.ccl_set_launch_mode(2) == 0
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        ccl.label_batch(dev, outs=outs, stream=st, k_out=kd)  # sizes the workspace
        st.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            ccl.label_batch(dev, outs=outs, stream=st, k_out=kd)
        for o in outs:
            o.fill_(-1)
        kd.fill_(-1)
        for _ in range(3):
            g.replay()
    torch.cuda.synchronize()
    for im, o, k in zip(imgs, outs, kd.cpu().tolist()):
        ref, rk = oracle.cclremsp(im)
        assert k == rk and np.array_equal(o.cpu().numpy(), ref)
