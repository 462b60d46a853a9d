"""Host logic of the serving loop's admission policy (no GPU needed)."""
import collections
from types import SimpleNamespace

from paper_1703_00443_gb300.serving import Admission


def _q(sizes):
    return collections.deque(SimpleNamespace(nbytes=s, name=i) for i, s in enumerate(sizes))


def test_fifo_batches_respect_budget_and_cap():
    adm = Admission(budget_bytes=100, max_batch=3)
    q = _q([30, 30, 30, 30, 50])
    b1, rej, t1 = adm.take(q)
    assert [r.name for r in b1] == [0, 1, 2] and not rej and t1 == 90   # cap of 3
    b2, rej, t2 = adm.take(q)
    assert b2 == [] and adm.reserved == 90                              # budget exhausted
    adm.release(t1)
    b3, rej, t3 = adm.take(q)
    assert [r.name for r in b3] == [3, 4] and t3 == 80


def test_oversized_request_is_rejected_not_blocking():
    adm = Admission(budget_bytes=100, max_batch=8)
    q = _q([150, 20, 20])
    b, rej, t = adm.take(q)
    assert [r.name for r in rej] == [0]
    assert [r.name for r in b] == [1, 2] and t == 40


def test_staging_cap_splits_batches_but_admits_a_large_request_alone():
    adm = Admission(budget_bytes=1000, max_batch=8, max_stage_bytes=100)
    q = collections.deque(SimpleNamespace(nbytes=10, stage_bytes=sb, name=i)
                          for i, sb in enumerate([40, 40, 40, 150, 30]))
    b1, _, _ = adm.take(q)
    assert [r.name for r in b1] == [0, 1]            # a third would pass the 100-byte cap
    b2, _, _ = adm.take(q)
    assert [r.name for r in b2] == [2]               # the next one is 150 on its own
    b3, _, _ = adm.take(q)
    assert [r.name for r in b3] == [3]               # larger than the cap: admitted alone
    b4, _, _ = adm.take(q)
    assert [r.name for r in b4] == [4]


def test_fifo_order_is_kept_when_head_does_not_fit():
    adm = Admission(budget_bytes=100, max_batch=8)
    adm.reserved = 70
    q = _q([50, 10])
    b, rej, t = adm.take(q)
    assert b == [] and len(q) == 2      # the head waits; nothing overtakes it


def test_scheduler_failure_fails_pending_requests_instead_of_hanging():
    """If the scheduling thread raises, every queued and in-flight request's future gets the
    error, and later submissions are refused (host logic only, no GPU)."""
    import collections
    import concurrent.futures
    import threading

    from paper_1703_00443_gb300.serving import QPServer, Request

    srv = QPServer.__new__(QPServer)
    srv.queues = [collections.deque(), collections.deque()]
    srv.inflight = []
    srv.cv = threading.Condition()
    srv._error = None
    mk = lambda: Request((), None, 0.0, concurrent.futures.Future())  # noqa: E731
    queued, running = [mk(), mk()], [mk()]
    srv.queues[0].append(queued[0])
    srv.queues[1].append(queued[1])
    srv.inflight.append({"reqs": running})

    def boom():
        raise ValueError("planted scheduler fault")

    srv._schedule = boom
    try:
        srv._loop()
    except ValueError:
        pass
    for r in queued + running:
        assert isinstance(r.future.exception(timeout=1), RuntimeError)
    assert not any(srv.queues) and not srv.inflight
    try:
        srv.submit(None, None, None, None, None, None, None)
        raise AssertionError("submit after a scheduler failure must raise")
    except RuntimeError:
        pass


def test_submit_routes_requests_by_size_class():
    """submit() queues a request in the class of its n (thresholds size_classes) and records
    its host addresses once (host logic only, no GPU)."""
    import collections
    import threading

    import numpy as np
    import torch

    from paper_1703_00443_gb300.serving import QPServer

    srv = QPServer.__new__(QPServer)
    srv.dtype = torch.float32
    srv.size_classes = (32, 192)
    srv.queues = [collections.deque() for _ in range(3)]
    srv.cv = threading.Condition()
    srv._error = None
    for n in (8, 31, 32, 100, 192, 300):
        data = (np.eye(n), np.zeros(n), np.ones((n, n)), np.ones(n), np.zeros((0, n)), np.zeros(0))
        srv.submit(*data, np.zeros(n))
    assert [[r.dims[0] for r in q] for q in srv.queues] == [[8, 31], [32, 100], [192, 300]]
    r = srv.queues[2][1]
    assert len(r.ptrs) == 7 and r.ptrs[0] == r.data[0].__array_interface__["data"][0]
    assert all(x.dtype == np.float32 and x.flags.c_contiguous for x in r.data)


def test_sections_are_aligned_and_disjoint():
    from paper_1703_00443_gb300.serving import _sections
    offs, total = _sections([0, 5, 64, 65, 1])
    assert all(o % 64 == 0 for o in offs)
    ends = [o + max(k, 1) for o, k in zip(offs, [0, 5, 64, 65, 1])]
    assert all(e <= nxt for e, nxt in zip(ends, offs[1:] + [total]))


def test_stage_bytes_bound_a_batch_staging():
    """The admission's staging cap is sound: for batches of mixed sizes, the input and result
    staging the scheduler lays out (sections per field, each 64-element aligned, plus the
    descriptors after the inputs) never exceeds the sum of the requests' stage_bytes plus the
    64 KB margin the server keeps."""
    import ctypes

    import numpy as np
    import torch

    from paper_1703_00443_gb300 import _lib, inputs
    from paper_1703_00443_gb300.serving import _sections, stage_bytes
    lib = _lib.load()
    for seed in range(5):
        sizes = inputs.serve_sizes(40, seed=seed, n_hi=256 if seed % 2 else 512)
        dims = np.array(sizes, dtype=np.int32)
        B = len(sizes)
        desc = (_lib.QPInstanceDesc * B)()
        sz = _lib.QPPackedSizes()
        assert lib.qp_packed_plan_ex(None, 0, B, dims.ctypes.data_as(ctypes.c_void_p), None, None,
                                     desc, ctypes.byref(sz)) == 0
        dbytes = B * ctypes.sizeof(_lib.QPInstanceDesc)
        _, n_in = _sections([sz.nQ, sz.nq, sz.nG, sz.nh, sz.nA, sz.nb, sz.nq, (dbytes + 3) // 4])
        _, n_out = _sections([sz.nq, sz.nh, sz.nb, sz.nQ, sz.nq, sz.nG, sz.nh, sz.nA, sz.nb])
        budget = sum(stage_bytes(s, torch.float32) for s in sizes) + (64 << 10)
        assert 4 * n_in <= budget and 4 * n_out <= budget
