"""The serving runtime (impact_server_*) through the C ABI (needs a GPU).

Requests of different dimensions and grid sizes arrive from a client thread
at random times while others are on the device; each result must be bitwise
the same as the build run alone (the mix-invariance of continuous batching),
and the memory budget must hold requests back rather than fail them."""

import random
import threading
import time

import numpy as np
import pytest
import torch

from paper_2401_03555_gb300 import impact, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.fail("the GPU tests need a CUDA device")
    impact.load()


def mix(count, seed):
    rng = random.Random(seed)
    pool = [lambda: W.robot_2d(cells_per_dim=7), lambda: W.room_5d(cells_per_dim=4),
            lambda: W.unicycle_3d(nx=9, ny=9, nth=7), lambda: W.building_7d(cells_per_dim=3),
            lambda: W.bas_4d(eta_scale=1.0)]
    out = []
    for i in range(count):
        if rng.random() < 0.5:
            out.append(W.random_linear(rng.randrange(256), min_cells=300, max_cells=3000))
        else:
            out.append(rng.choice(pool)())
    return out


def host(csr):
    t = lambda x: x.cpu().numpy()
    return (t(csr.row_ptr), t(csr.col), t(csr.lo), t(csr.up), t(csr.sink_lo), t(csr.sink_up),
            t(csr.trunc), t(csr.row_flags))


def same(a, b):
    return all(x.shape == y.shape and np.array_equal(x.view(np.uint8), y.view(np.uint8))
               for x, y in zip(host(a), host(b)))


def serve(server, probs, seed, max_gap_s=0.004):
    """Submit from a client thread at random gaps; returns the tickets."""
    tickets = [None] * len(probs)
    rng = random.Random(seed)

    def client():
        for i, p in enumerate(probs):
            time.sleep(rng.random() * max_gap_s)
            tickets[i] = server.submit(p)

    th = threading.Thread(target=client)
    th.start()
    th.join()
    return tickets


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_results_equal_alone_and_in_the_mix(precision):
    probs = mix(16, seed=7)
    alone = [impact.build(p, precision) for p in probs]
    with impact.Server(precision, max_batch=6, streams=2) as srv:
        tickets = serve(srv, probs, seed=1)
        for t, p, ref in zip(tickets, probs, alone):
            done, lat = srv.poll(t, wait=True)
            assert done and lat > 0
            got = srv.result(t)
            assert same(got, ref), f"{p.name}: served result differs from the build alone"
            srv.release(t)
        st = srv.stats()
        assert st["completed"] == len(probs)
        assert st["pairs"] == sum(r.nnz for r in alone)
        assert st["groups"] >= 2


def test_memory_budget_holds_requests_back():
    probs = [W.room_5d(cells_per_dim=5) for _ in range(6)]
    one = impact.build(probs[0], "fp32")
    ws = impact.workspace_bytes(probs[0], "fp32")
    # room for about two requests in flight at a time
    budget = 2 * (ws + one.nbytes()) + (4 << 20)
    with impact.Server("fp32", memory_budget=budget, max_batch=4) as srv:
        tickets = serve(srv, probs, seed=3, max_gap_s=0.0)
        for t in tickets:
            assert srv.poll(t, wait=True)[0]
            assert same(srv.result(t), one)
            srv.release(t)
        st = srv.stats()
        assert st["completed"] == len(probs) and st["groups"] >= 3
        for _ in range(200):   # released groups are freed by the scheduler thread
            if srv.stats()["bytes_in_use"] == 0:
                break
            time.sleep(0.01)
        assert srv.stats()["bytes_in_use"] == 0


def test_request_larger_than_the_budget_fails_cleanly():
    with impact.Server("fp32", memory_budget=1 << 20) as srv:
        t = srv.submit(W.room_5d(cells_per_dim=6))
        with pytest.raises(impact.ImpactError) as ei:
            srv.poll(t, wait=True)
        assert ei.value.status == impact.IMPACT_ERR_OOM
        srv.release(t)
        t2 = srv.submit(W.robot_2d(cells_per_dim=3))   # still serves what fits
        assert srv.poll(t2, wait=True)[0]
        srv.release(t2)


def test_cancel_withdraws_a_waiting_request():
    """A kept result holds the budget, so the next request waits; cancelling
    it keeps it off the device, and the server goes on serving."""
    prob = W.room_5d(cells_per_dim=5)
    one = impact.build(prob, "fp32")
    ws = impact.workspace_bytes(prob, "fp32")
    budget = ws + one.nbytes() + (256 << 10)        # one request at a time (rows: 1 MB)
    with impact.Server("fp32", memory_budget=budget) as srv:
        t1 = srv.submit(prob)
        assert srv.poll(t1, wait=True)[0]            # finished, result kept
        t2 = srv.submit(prob)
        time.sleep(0.05)
        assert srv.stats()["waiting"] == 1
        srv.cancel(t2)
        assert srv.stats()["waiting"] == 0
        with pytest.raises(impact.ImpactError) as ei:
            srv.poll(t2, wait=True)
        assert ei.value.status == impact.IMPACT_ERR_CANCELLED
        with pytest.raises(impact.ImpactError):       # only waiting requests cancel
            srv.cancel(t1)
        srv.release(t2)
        with pytest.raises(impact.ImpactError):       # released: unknown
            srv.cancel(t2)
        assert same(srv.result(t1), one)
        srv.release(t1)
        t3 = srv.submit(prob)                         # the budget is free again
        assert srv.poll(t3, wait=True)[0]
        assert same(srv.result(t3), one)
        srv.release(t3)
        assert srv.stats()["completed"] == 2
