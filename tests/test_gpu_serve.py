"""Serving loop: every request's count equals the count of the same graph
alone (exact integers, tolerance zero), with requests overlapping on the
device; admission limits, unknown ids and injected failures are reported
as statuses, never as hangs."""
import time

import pytest

import graphgen as gg
import oracle
from tests import pins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch
    torch.cuda.init()
    import paper_2210_00389_gb300 as tc
    return tc


def drain(tc, s, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        assert time.time() - t0 < timeout, "requests did not finish in time"
        for t in tickets:
            if t in out:
                continue
            done, c, st = tc.tc_serve_poll(s, t)
            if done:
                out[t] = (c, st)
        time.sleep(0.002)
    return [out[t] for t in tickets]


@pytest.mark.parametrize("borrow", [False, True])
def test_serve_mix_equals_alone(tc, borrow):
    resident = gg.rmat(15, 16, seed=81, relabel_seed=82)
    one_shot = pins.random_small_graphs() + [c[0] for c in pins.closed_form_cases()][:12]
    one_shot += [gg.rmat(s, 8, seed=90 + s) for s in (8, 10, 12)]
    one_shot += [gg.rmat(17, 4, seed=95)]  # large one-shot (n > the batch limit)
    # borrowed views: the arrays in one_shot stay alive until drained
    s = tc.tc_serve_create(8 << 30, slots=16, queue_capacity=1024, wait_limit_ms=60000,
                           borrow_views=borrow)
    try:
        gid = tc.tc_serve_register(s, resident.offsets, resident.cols)
        tickets, want = [], []
        for i, g in enumerate(one_shot):
            mode = tc.TC_MODE_COVER if i % 2 == 0 else tc.TC_MODE_PLAIN
            tickets.append(tc.tc_serve_submit(s, (g.offsets, g.cols), 0, mode))
            want.append(oracle.cetc(g)["T"])
            if i % 5 == 0:
                tickets.append(tc.tc_serve_submit(s, None, gid, tc.TC_MODE_COVER))
                want.append(None)
        res = drain(tc, s, tickets)
    finally:
        tc.tc_serve_destroy(s)
    T_res = oracle.plain_count(resident)
    for (c, st), w in zip(res, want):
        assert st == tc.TC_OK
        assert c == (T_res if w is None else w)


def test_serve_rejections_and_statuses(tc):
    g = gg.complete(10)
    s = tc.tc_serve_create(1 << 20, slots=2, queue_capacity=8, wait_limit_ms=5000)
    try:
        big = gg.rmat(14, 16, seed=3)
        with pytest.raises(tc.TCError) as e:
            tc.tc_serve_submit(s, (big.offsets, big.cols), 0, tc.TC_MODE_COVER)
        assert e.value.status == tc.TC_ERR_OOM
        with pytest.raises(tc.TCError) as e:
            tc.tc_serve_submit(s, None, 12345, tc.TC_MODE_COVER)
        assert e.value.status == tc.TC_ERR_NOT_FOUND
        with pytest.raises(tc.TCError) as e:
            tc.tc_serve_poll(s, 999999)
        assert e.value.status == tc.TC_ERR_NOT_FOUND
        bad = g.cols.copy()
        bad[0] = 55
        t_bad = tc.tc_serve_submit(s, (g.offsets, bad), 0, tc.TC_MODE_COVER)
        t_ok = tc.tc_serve_submit(s, (g.offsets, g.cols), 0, tc.TC_MODE_COVER)
        (c_bad, st_bad), (c_ok, st_ok) = drain(tc, s, [t_bad, t_ok])
        assert st_bad == tc.TC_ERR_INVALID_GRAPH and st_ok == tc.TC_OK and c_ok == 120
    finally:
        tc.tc_serve_destroy(s)


def test_serve_injected_failure_is_isolated(tc):
    gs = [gg.complete(k) for k in (5, 6, 7, 8)]
    s = tc.tc_serve_create(1 << 30, slots=1, queue_capacity=16, wait_limit_ms=20000,
                           fail_request=2)
    try:
        ts = [tc.tc_serve_submit(s, (g.offsets, g.cols), 0, tc.TC_MODE_COVER) for g in gs]
        res = drain(tc, s, ts)
    finally:
        tc.tc_serve_destroy(s)
    assert [st for _, st in res] == [tc.TC_OK, tc.TC_ERR_OOM, tc.TC_OK, tc.TC_OK]
    assert [c for c, _ in res] == [10, 0, 35, 56]


def test_serve_shutdown_with_pending_requests(tc):
    g = gg.rmat(16, 16, seed=5)
    s = tc.tc_serve_create(4 << 30, slots=1, queue_capacity=64, wait_limit_ms=20000)
    for _ in range(20):
        tc.tc_serve_submit(s, (g.offsets, g.cols), 0, tc.TC_MODE_COVER)
    t0 = time.time()
    tc.tc_serve_destroy(s)  # cancels what is queued, finishes what runs
    assert time.time() - t0 < 60
