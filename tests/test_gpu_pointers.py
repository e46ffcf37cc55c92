"""Where the caller's buffers live.  Inputs and outputs may each be host or
device memory, in any mix, and give the same graph bit for bit; another
device's memory is refused before anything is launched.  With one GPU the
test hook KNNG_TEST_FOREIGN_DEVICE makes the library classify pointers as if
another device were current, so every device pointer looks foreign while host
memory stays usable."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2112_06630_gb300 as knng  # noqa: E402

N, D, K = 600, 24, 10
ARGS = dict(rho=0.5, delta=0.001, max_iters=6, seed=3)


def _x():
    return workloads.gaussian_mixture(N, D, 12, seed=11)


def _np(t):
    return t.cpu().numpy() if torch.is_tensor(t) else t


def test_host_device_and_mixed_outputs_give_the_same_graph():
    x = _x()
    xd = torch.from_numpy(x).cuda()
    ri, rd, _ = knng.knng_build(xd, K, **ARGS)
    ri, rd = _np(ri), _np(rd)
    hi, hd, _ = knng.knng_build(x, K, **ARGS)
    np.testing.assert_array_equal(hi, ri)
    np.testing.assert_array_equal(hd, rd)
    for src in (x, xd):
        # ids on the device with dists on the host, and the other way round
        for dev_ids in (True, False):
            ids = torch.full((N, K), -1, dtype=torch.int32, device="cuda") if dev_ids else np.full((N, K), -1, np.int32)
            dists = np.full((N, K), -1, np.float32) if dev_ids else torch.full((N, K), -1.0, device="cuda")
            knng.knng_build(src, K, out=(ids, dists), **ARGS)
            np.testing.assert_array_equal(_np(ids), ri)
            np.testing.assert_array_equal(_np(dists), rd)
    # brute force: device input with host outputs equals the device outputs
    bi, bd = knng.knng_bruteforce(xd, K)
    lib = knng.load()
    hi2 = np.empty((N, K), np.int32)
    hd2 = np.empty((N, K), np.float32)
    assert lib.knng_bruteforce(xd.data_ptr(), N, D, K, None, 0, hi2.ctypes.data, hd2.ctypes.data,
                               torch.cuda.current_stream().cuda_stream) == 0
    np.testing.assert_array_equal(hi2, _np(bi))
    np.testing.assert_array_equal(hd2, _np(bd))


def test_foreign_device_memory_refused_before_any_launch(monkeypatch):
    x = _x()
    xd = torch.from_numpy(x).cuda()
    lib = knng.load()
    stream = torch.cuda.current_stream().cuda_stream
    monkeypatch.setenv("KNNG_TEST_FOREIGN_DEVICE", "1")

    def refused(fn, *a, **kw):
        with pytest.raises(knng.KnngError) as ei:
            fn(*a, **kw)
        assert ei.value.code == -1

    refused(knng.knng_build, xd, K, **ARGS)
    # a device output alone is refused as well, and nothing is written to it
    guard = torch.full((N, K), -7.0, device="cuda")
    refused(knng.knng_build, x, K, out=(np.empty((N, K), np.int32), guard), **ARGS)
    assert bool((guard == -7.0).all())
    refused(knng.knng_bruteforce, xd, 5)
    refused(knng.knng_bruteforce, x, 5, rows=torch.arange(10, device="cuda"))
    refused(knng.knng_build_batched, [x, xd], 5)
    refused(knng.knng_build_batched_ex, [dict(data=xd, K=5, rho=0.5, delta=0.001, max_iters=5, seed=0)])
    refused(knng.Context, xd, K)
    # a starting graph on the device: refused, and *out is left NULL
    gi = torch.from_numpy(workloads.random_graph(N, K, seed=2)[0]).to(torch.int32).cuda()
    gn = np.ones((N, K), np.uint8)
    h = ctypes.c_void_p(0x1234)
    assert lib.knng_init_from_graph(ctypes.byref(h), x.ctypes.data, N, D, K, 0.5, 0.001, 0, 0, stream,
                                    gi.data_ptr(), gn.ctypes.data, 0) == -1
    assert h.value is None
    # host memory stays usable: the same graph as without the hook
    with knng.Context(x, K, rho=ARGS["rho"], delta=ARGS["delta"], seed=ARGS["seed"]) as c:
        c.run(ARGS["max_iters"])
        refused(c.get, device=True)
        hi, hd = c.get(device=False)
    monkeypatch.delenv("KNNG_TEST_FOREIGN_DEVICE")
    ri, rd, _ = knng.knng_build(x, K, **ARGS)
    np.testing.assert_array_equal(hi, ri)
    np.testing.assert_array_equal(hd, rd)
