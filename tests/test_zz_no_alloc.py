"""knng_bruteforce_noalloc: the brute-force K-NNG for callers that cannot
allocate device memory (stream capture in global mode, programs whose device
memory belongs to their own pool, real-time code that must not allocate after
start-up).  Its scratch is a static device array, so its results must equal
those of knng_bruteforce on the same device buffers, call after call.

Collected last on purpose (file name), so a stop-at-first-failure run has
already run every other test when it gets here; it also passes alone.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2112_06630_gb300 as knng  # noqa: E402

SCRATCH_BYTES = 8 << 20


@pytest.fixture(scope="module")
def noalloc():
    lib = knng.load()
    fn = lib.knng_bruteforce_noalloc
    P = ctypes.c_void_p
    fn.restype = ctypes.c_int
    fn.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P, ctypes.c_int64, P, P, P]
    return fn


def _call(fn, xd, K, rows=None):
    n, d = xd.shape
    nq = n if rows is None else rows.shape[0]
    ids = torch.full((nq, K), -1, dtype=torch.int32, device=xd.device)
    dists = torch.full((nq, K), -1.0, dtype=torch.float32, device=xd.device)
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(xd.data_ptr(), n, d, K, 0 if rows is None else rows.data_ptr(), nq, ids.data_ptr(),
            dists.data_ptr(), stream)
    torch.cuda.synchronize()
    return rc, ids.cpu().numpy(), dists.cpu().numpy()


def _same_up_to_ties(gi, gd, ri, rd, rtol=1e-5):
    np.testing.assert_allclose(gd, rd, rtol=rtol, atol=1e-7)
    mism = gi != ri
    if mism.any():
        assert np.allclose(gd[mism], rd[mism], rtol=rtol, atol=1e-7)


def test_noalloc_matches_bruteforce_two_calls_in_a_row(noalloc):
    # call 1: all rows of a mixture; call 2: a different size, d not a multiple
    # of 4 and a subset of query rows, reusing the same scratch
    x1 = workloads.gaussian_mixture(6000, 16, 30, seed=1)
    x2 = workloads.uniform(3001, 7, seed=2)
    rows2 = torch.tensor([0, 3000, 17, 1500, 2999, 42], dtype=torch.int64, device="cuda")
    for x, K, rows in ((x1, 20, None), (x2, 10, rows2)):
        xd = torch.from_numpy(x).cuda()
        rc, gi, gd = _call(noalloc, xd, K, rows)
        assert rc == 0
        ri, rd = knng.knng_bruteforce(xd, K, rows=rows)
        _same_up_to_ties(gi, gd, ri.cpu().numpy(), rd.cpu().numpy())


def test_noalloc_rejects_oversize_and_host_pointers(noalloc):
    d = 16
    n = SCRATCH_BYTES // (4 * d) + 1
    xd = torch.zeros((n, d), dtype=torch.float32, device="cuda")
    rc, _, _ = _call(noalloc, xd, 4)
    assert rc == -1
    xh = np.zeros((100, 4), np.float32)
    ids = np.zeros((100, 4), np.int32)
    dists = np.zeros((100, 4), np.float32)
    assert noalloc(xh.ctypes.data, 100, 4, 4, None, 100, ids.ctypes.data, dists.ctypes.data, None) == -1


def test_noalloc_scratch_exactly_full_and_just_under(noalloc):
    """The size limit at its edge: a padded copy that fills the array exactly
    (16 floats x 131,072 rows = 8 MiB) is taken, and so is a row width that
    is not a multiple of 4 just under it (7 floats pad to 8: 262,143 rows);
    one row more is refused.  Query rows keep the runs short."""
    g = np.random.default_rng(5)
    for n, d in ((SCRATCH_BYTES // (4 * 16), 16), (SCRATCH_BYTES // (4 * 8) - 1, 7)):
        x = workloads.gaussian_mixture(n, d, 64, seed=d)
        xd = torch.from_numpy(x).cuda()
        rows = torch.from_numpy(np.sort(g.choice(n, 40, replace=False)).astype(np.int64)).cuda()
        rc, gi, gd = _call(noalloc, xd, 12, rows)
        assert rc == 0
        ri, rd = knng.knng_bruteforce(xd, 12, rows=rows)
        _same_up_to_ties(gi, gd, ri.cpu().numpy(), rd.cpu().numpy())
    big = torch.zeros((SCRATCH_BYTES // (4 * 8) + 1, 7), dtype=torch.float32, device="cuda")
    rc, _, _ = _call(noalloc, big, 4, torch.zeros(1, dtype=torch.int64, device="cuda"))
    assert rc == -1


def test_noalloc_refuses_foreign_device_memory(noalloc, monkeypatch):
    """Memory of another device is refused before any launch.  With one GPU
    the test hook makes the library check the pointers as if another device
    were current: every device pointer then belongs to a foreign device."""
    xd = torch.from_numpy(workloads.uniform(300, 8, seed=3)).cuda()
    monkeypatch.setenv("KNNG_TEST_NOALLOC_FOREIGN_DEVICE", "1")
    rc, gi, _ = _call(noalloc, xd, 5)
    assert rc == -1 and (gi == -1).all()
    monkeypatch.delenv("KNNG_TEST_NOALLOC_FOREIGN_DEVICE")
    rc, gi, _ = _call(noalloc, xd, 5)
    assert rc == 0 and (gi >= 0).all()


def test_noalloc_inside_global_mode_capture(noalloc):
    """The case the entry point exists for: calls recorded while a stream is
    captured in global mode (where an allocation would fail the capture).
    One eager call first does the per-context set-up; the captured calls then
    use other K classes and row paths than that call (K 20 over 64-float rows,
    whose tiles need more than 48 KB of shared memory, and K 30 over 7-float
    rows).  The replayed graph gives knng_bruteforce's answers."""
    warm = torch.from_numpy(workloads.uniform(500, 8, seed=4)).cuda()
    assert _call(noalloc, warm, 4)[0] == 0
    cases = [(workloads.gaussian_mixture(3000, 64, 20, seed=6), 20), (workloads.uniform(2500, 7, seed=7), 30)]
    ins, outs = [], []
    for x, K in cases:
        xd = torch.from_numpy(x).cuda()
        ins.append((xd, K))
        outs.append((torch.full((x.shape[0], K), -1, dtype=torch.int32, device="cuda"),
                     torch.full((x.shape[0], K), -1.0, dtype=torch.float32, device="cuda")))
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    rcs = []
    with torch.cuda.graph(graph, capture_error_mode="global"):
        s = torch.cuda.current_stream().cuda_stream
        for (xd, K), (ids, dists) in zip(ins, outs):
            rcs.append(noalloc(xd.data_ptr(), xd.shape[0], xd.shape[1], K, None, xd.shape[0], ids.data_ptr(),
                               dists.data_ptr(), s))
    assert rcs == [0, 0]
    assert all((ids == -1).all() for ids, _ in outs)  # captured, not yet run
    graph.replay()
    torch.cuda.synchronize()
    for (xd, K), (ids, dists) in zip(ins, outs):
        ri, rd = knng.knng_bruteforce(xd, K)
        _same_up_to_ties(ids.cpu().numpy(), dists.cpu().numpy(), ri.cpu().numpy(), rd.cpu().numpy())
