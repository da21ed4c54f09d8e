"""The continuous-batching server: results in a mix of concurrent requests are the same as
labelling each image alone (bit-exact), requests share one memory pool (a request larger
than a lane's even share of the cap is served; requests larger than the whole cap are
refused), launches on different lanes are in flight together, and the statistics add up."""
import ctypes
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone():
    import torch

    import paper_1606_05973_gb300 as ccl

    specs = synth.batch_specs(n=48, seed=21, lo=8, hi=1200)
    imgs = [synth.make_batch_image(s) for s in specs]
    imgs.append(np.zeros((0, 4), np.uint8))
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    alone = [ccl.label(t) for t in dev]
    torch.cuda.synchronize()
    outs = [torch.full(tuple(t.shape), -1, dtype=torch.int32, device="cuda") for t in dev]
    ks = [None] * len(dev)
    with ccl.Server(mem_cap_bytes=1 << 30, lanes=3, max_batch=8) as srv:
        def client(lo):
            ids = [(i, srv.submit(dev[i], outs[i])) for i in range(lo, len(dev), 4)]
            for i, rid in ids:
                ks[i] = srv.wait(rid)

        th = [threading.Thread(target=client, args=(c,)) for c in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        st = srv.stats()
    torch.cuda.synchronize()
    for i, im in enumerate(imgs):
        ref, rk = oracle.cclremsp(im)
        assert ks[i] == rk == alone[i][1], i
        assert np.array_equal(outs[i].cpu().numpy(), alone[i][0].cpu().numpy()), i
        assert np.array_equal(outs[i].cpu().numpy(), ref), i
    assert st["completed"] == len(imgs)
    assert st["launches"] >= 1 and st["mean_batch"] >= 1.0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_server_refuses_what_does_not_fit_and_keeps_going():
    import torch

    import paper_1606_05973_gb300 as ccl

    big = torch.ones((4096, 4096), dtype=torch.uint8, device="cuda")
    big_out = torch.empty((4096, 4096), dtype=torch.int32, device="cuda")
    small = torch.from_numpy(synth.bernoulli(300, 400, 0.5, 3)).cuda()
    small_out = torch.empty((300, 400), dtype=torch.int32, device="cuda")
    with ccl.Server(mem_cap_bytes=16 << 20, lanes=2, max_batch=4) as srv:  # 4096^2 needs > 16 MiB
        rid = srv.submit(big, big_out)
        with pytest.raises(ccl.CCLError) as e:
            srv.wait(rid)
        assert e.value.status == 8  # CCL_ERR_TOO_LARGE
        k = srv.wait(srv.submit(small, small_out))
    ref, rk = oracle.cclremsp(synth.bernoulli(300, 400, 0.5, 3))
    assert k == rk and np.array_equal(small_out.cpu().numpy(), ref)


def test_request_larger_than_an_even_share_is_served():
    """The pool is shared: with a 64 MiB cap over four lanes (16 MiB each if split evenly) a
    3000 x 3000 image, whose workspace is over 16 MiB, is served and exact."""
    import torch

    import paper_1606_05973_gb300 as ccl

    img = synth.bernoulli(3000, 3000, 0.55, 31)
    need = ctypes.c_int64(0)
    assert ccl.lib().ccl_workspace_bytes(3000, 3000, ctypes.byref(need)) == 0
    assert need.value > (64 << 20) // 4
    d = torch.from_numpy(img).cuda()
    out = torch.full((3000, 3000), -1, dtype=torch.int32, device="cuda")
    with ccl.Server(mem_cap_bytes=64 << 20, lanes=4, max_batch=2) as srv:
        k = srv.wait(srv.submit(d, out), timeout_ms=60000)
    ref, rk = oracle.cclremsp(img)
    assert k == rk
    assert np.array_equal(out.cpu().numpy(), ref)


def test_lanes_run_together_and_results_stay_exact():
    """Twelve requests submitted at once, one per launch: several lanes are in flight
    together (peak_busy_lanes), and every result equals the oracle's."""
    import torch

    import paper_1606_05973_gb300 as ccl

    imgs = [synth.bernoulli(1024, 1536, 0.3 + 0.04 * i, 40 + i) for i in range(12)]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.full(im.shape, -1, dtype=torch.int32, device="cuda") for im in imgs]
    with ccl.Server(mem_cap_bytes=1 << 30, lanes=3, max_batch=1) as srv:
        ids = [srv.submit(d, o) for d, o in zip(dev, outs)]
        ks = [srv.wait(r, timeout_ms=60000) for r in ids]
        st = srv.stats()
    assert st["launches"] == 12 and st["completed"] == 12
    assert st["peak_busy_lanes"] >= 2
    assert st["peak_inflight_bytes"] > 0
    for im, k, o in zip(imgs, ks, outs):
        ref, rk = oracle.cclremsp(im)
        assert k == rk
        assert np.array_equal(o.cpu().numpy(), ref)
