"""Failure detection on the GPU without a fault: a bounded device wait that
runs out must come back as an error status that the host reads, and the
library and the GPU must stay usable afterwards.

A test hook (KNNG_TEST_HOLD_LOCKS=h) starts the locks of the first h lists
held, and a one-run proposal pool (KNNG_TEST_BUCKET_POOL_CHUNKS=1), with the
join in one pass (KNNG_TEST_JOIN_PASSES=1), sends proposals past full buckets
to the locked insertion; an insertion into a held
list spins a bounded number of times (about half a second), gives up, raises
the timeout counter, and the call returns KNNG_ERR_TIMEOUT.  Nothing traps,
faults or hangs.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2112_06630_gb300 as knng  # noqa: E402

KNNG_ERR_TIMEOUT = -4


def _case():
    n, d, K, rho = 1800, 3, 16, 0.5
    g = np.random.default_rng(n)
    x = g.integers(0, 6, size=(n, d)).astype(np.float32)
    ids0, new0 = workloads.random_graph(n, K, seed=n + 1, p_new=0.6)
    return x, ids0, new0, K, rho


def test_held_locks_time_out_and_the_library_recovers(monkeypatch):
    x, ids0, new0, K, rho = _case()
    xd = torch.from_numpy(x).cuda()
    monkeypatch.setenv("KNNG_TEST_BUCKET_POOL_CHUNKS", "1")
    monkeypatch.setenv("KNNG_TEST_JOIN_PASSES", "1")
    monkeypatch.setenv("KNNG_TEST_HOLD_LOCKS", "4")
    with knng.Context(xd, K, rho=rho, seed=11, graph=(ids0, new0), iter=0) as c:
        with pytest.raises(knng.KnngError) as err:
            c.iterate()
        assert err.value.code == KNNG_ERR_TIMEOUT
        st = c.stats()
        assert st["lock_timeouts"] > 0 and st["bucket_overflow"] > 0
    # the GPU and the library are fine: the same iteration without held
    # locks matches the oracle bit for bit
    monkeypatch.delenv("KNNG_TEST_HOLD_LOCKS")
    with knng.Context(xd, K, rho=rho, seed=11, graph=(ids0, new0), iter=0) as c:
        conv, ch = c.iterate()
        gi, gd, gf = c.state()
        assert c.stats()["lock_timeouts"] == 0
    st = oracle.State(x, K, rho, seed=11)
    st.init_graph(ids0, new0, 0)
    r = st.iterate()
    oi, od, of = st.state()
    assert (gi == oi).all() and (gd == od).all() and (gf == of).all()
    assert ch == r["changes"]


def test_timeout_reported_by_the_one_shot_build(monkeypatch):
    x, _, _, K, rho = _case()
    monkeypatch.setenv("KNNG_TEST_BUCKET_POOL_CHUNKS", "1")
    monkeypatch.setenv("KNNG_TEST_JOIN_PASSES", "1")
    monkeypatch.setenv("KNNG_TEST_HOLD_LOCKS", "4")
    with pytest.raises(knng.KnngError) as err:
        knng.knng_build(torch.from_numpy(x).cuda(), K, rho, 0.001, 2, seed=3)
    assert err.value.code == KNNG_ERR_TIMEOUT
