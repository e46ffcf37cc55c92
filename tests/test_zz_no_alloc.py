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
