"""Failure paths of the C ABI, each made to fire without faulting a GPU.

* Row checks (Def. 3.1's row conditions): a fault-injection knob makes one
  row's check see an impossible lower-bound sum; the call must return
  IMPACT_ERR_UNSOUND with exactly that row flagged.
* Emit mismatch: impact_emit with one interior row boundary moved by one
  (row_ptr stays monotone and inside the capacity, so every store stays in
  the caller's arrays); the two rows concerned disagree with their ranges.
* Bounded waits: one row never publishes its pair count, so the rows after it
  give up their offset look-back after a short spin limit; the call returns
  IMPACT_ERR_TIMEOUT and the next build on the same device is correct.
* Capacity: the one-pass build into arrays one pair too short.
* Out of memory: the n-th allocation of an entry point is made to fail on the
  host (impact_debug_fail_alloc) for every n until the call succeeds; each
  failure returns IMPACT_ERR_OOM and leaves no library memory behind.
"""

import ctypes
import dataclasses

import numpy as np
import pytest
import torch

from paper_2401_03555_gb300 import impact, workloads as W

pytestmark = pytest.mark.gpu


def small():
    return W.room_5d(cells_per_dim=5)


def csr_of(rb, pb, nnz, precision="fp32"):
    return impact.CSR(precision, rb["row_ptr"], pb["col"][:nnz], pb["lo"][:nnz], pb["up"][:nnz],
                      rb["sink_lo"], rb["sink_up"], rb["trunc"], rb["row_flags"])


def assert_same(a, b):
    for f in ("row_ptr", "col", "lo", "up", "sink_lo", "sink_up", "trunc", "row_flags"):
        assert torch.equal(getattr(a, f), getattr(b, f)), f


@pytest.mark.parametrize("mode", ["count", "build", "one_pass"])
def test_row_check_fires_on_exactly_the_faulted_row(mode):
    prob = small()
    ref = impact.build(prob, "fp32")
    bad = 17
    b = impact.Batch([prob], "fp32",
                     tune=impact.tuning(fault_row=bad, one_pass=mode == "one_pass"))
    rb = impact.alloc_rows(b.rows)
    with pytest.raises(impact.ImpactError) as e:
        if mode == "count":
            b.count(rb)
        else:
            pb = impact.alloc_pairs(ref.nnz, "fp32")
            b.build_into(rb, pb, ref.nnz)
    assert e.value.status == impact.IMPACT_ERR_UNSOUND
    flags = rb["row_flags"].cpu().numpy()
    assert np.flatnonzero(flags).tolist() == [bad]
    assert flags[bad] == 0x1                            # IMPACT_ROW_LO_SUM_ABOVE_ONE
    # everything else is the unfaulted build
    assert torch.equal(rb["row_ptr"], ref.row_ptr)
    assert torch.equal(rb["trunc"], ref.trunc) and torch.equal(rb["sink_up"], ref.sink_up)


def test_emit_reports_a_row_pointer_that_does_not_match():
    prob = small()
    ref = impact.build(prob, "fp32")
    rp = ref.row_ptr.clone()
    counts = (rp[1:] - rp[:-1]).cpu().numpy()
    nz = np.flatnonzero(counts[1:] > 0) + 1
    k = int(nz[len(nz) // 2])                     # an interior row with a pair
    rp[k] += 1                                    # row k-1 one longer, row k one shorter
    rb = impact.alloc_rows(prob.rows)
    rb["row_ptr"].copy_(rp)
    pb = impact.alloc_pairs(ref.nnz, "fp32")
    a = impact._Args(prob)
    c = impact._csr_struct(rb, pb, capacity=ref.nnz)
    lib = impact.load()
    st = lib.impact_emit(ctypes.byref(a.sys), ctypes.byref(a.grid), ctypes.byref(a.inp),
                         a.sigma_ptr, a.cutoff, impact.FP32_SOUND, ctypes.byref(c), None)
    assert st == impact.IMPACT_ERR_CUDA
    assert "disagreed" in lib.impact_last_error().decode()
    # rows other than k-1 and k are written exactly as in the reference
    torch.cuda.synchronize()
    ok = torch.ones(ref.nnz, dtype=torch.bool, device="cuda")
    ok[int(rp[k - 1]):int(rp[k + 1])] = False
    assert torch.equal(pb["col"][ok], ref.col[ok]) and torch.equal(pb["up"][ok], ref.up[ok])


@pytest.mark.parametrize("mode", ["count", "build"])
def test_a_spent_step_guard_is_an_internal_error_and_the_library_recovers(mode):
    """The walk's step guard bounds every row's depth-first loop; when it runs
    out (a broken invariant) the row is reported, not looped on."""
    prob = small()
    ref = impact.build(prob, "fp32")
    b = impact.Batch([prob], "fp32", tune=impact.tuning(guard_row=prob.rows // 3))
    rb = impact.alloc_rows(b.rows)
    with pytest.raises(impact.ImpactError) as e:
        if mode == "count":
            b.count(rb)
        else:
            pb = impact.alloc_pairs(ref.nnz, "fp32")
            b.build_into(rb, pb, ref.nnz)
    assert e.value.status == impact.IMPACT_ERR_CUDA
    assert "step guard" in str(e.value)
    assert_same(impact.build(prob, "fp32"), ref)


def test_a_caller_image_wider_than_the_window_cap_is_refused():
    """Caller-supplied images are not bounded by the planner: one row whose
    image spans 135 cells of a dimension (the cap is 128) makes the setup
    kernel report the overflow, and the call fails with IMPACT_ERR_ARG."""
    # cutoff 1e-8: a point image's window is about 2 x 32 noise cells wide
    base = dataclasses.replace(W.robot_2d(cells_per_dim=150), cutoff=1e-8)
    rng = np.random.default_rng(9)
    pts = rng.uniform(-9.0, 9.0, size=(base.rows, 2))
    img = np.stack([pts, pts], axis=2)
    img[base.rows // 2, 0] = (-9.0, 9.0)
    prob = W.with_images(base, img)
    with pytest.raises(impact.ImpactError) as e:
        impact.build(prob, "fp32")
    assert e.value.status == impact.IMPACT_ERR_ARG
    assert "window" in str(e.value)
    img[base.rows // 2, 0] = (-1.0, 1.0)               # 15 cells: builds
    assert impact.build(W.with_images(base, img), "fp32").nnz > 0


def test_look_back_wait_times_out_and_the_device_stays_usable():
    """The one-pass build (caller arrays): each row waits, boundedly, for the
    pair counts of the rows before it."""
    prob = small()
    ref = impact.build(prob, "fp32")
    b = impact.Batch([prob], "fp32", tune=impact.tuning(stall_row=prob.rows // 2,
                                                        spin_limit=2000, one_pass=True))
    rb = impact.alloc_rows(b.rows)
    pb = impact.alloc_pairs(ref.nnz, "fp32")
    with pytest.raises(impact.ImpactError) as e:
        b.build_into(rb, pb, ref.nnz)
    assert e.value.status == impact.IMPACT_ERR_TIMEOUT
    # same context, same library: the next builds are complete and identical
    again = impact.build(prob, "fp32")
    assert_same(again, ref)
    nnz = impact.Batch([prob], "fp32").build_into(rb, pb, ref.nnz)
    assert nnz == ref.nnz
    assert_same(csr_of(rb, pb, nnz), ref)


@pytest.mark.parametrize("one_pass", [False, True])
def test_build_into_short_capacity_reports_the_needed_pairs(one_pass):
    prob = small()
    ref = impact.build(prob, "fp32")
    b = impact.Batch([prob], "fp32", tune=impact.tuning(one_pass=one_pass))
    rb = impact.alloc_rows(b.rows)
    pb = impact.alloc_pairs(ref.nnz - 1, "fp32")
    pb["col"].fill_(-7)
    c = impact._csr_struct(rb, pb, capacity=ref.nnz - 1)
    st = impact.load().impact_batch_build(b.reqs, 1, b.prec, b._tp(),
                                          ctypes.byref(c), None)
    assert st == impact.IMPACT_ERR_CAPACITY
    assert int(c.nnz) == ref.nnz                       # the needed count comes back
    assert torch.equal(rb["row_ptr"], ref.row_ptr)     # row pointers and terms are valid
    assert torch.equal(rb["trunc"], ref.trunc)
    col = pb["col"].cpu()
    if one_pass:   # the rows that fit are written
        fit = int(np.searchsorted(ref.row_ptr.cpu().numpy(), ref.nnz - 1, side="right")) - 1
        end = int(ref.row_ptr[fit])
        assert torch.equal(col[:end], ref.col[:end].cpu())
    else:          # the emit pass saw the short capacity and wrote nothing
        assert bool((col == -7).all())


def _oom_sweep(call, check=None, limit=40):
    """Fails allocation n = 1, 2, ... of `call` until it succeeds."""
    torch.cuda.synchronize()
    base = impact.live_bytes()
    for n in range(1, limit):
        impact.fail_alloc(n)
        try:
            res = call()
        except impact.ImpactError as e:
            impact.fail_alloc(0)
            assert e.status == impact.IMPACT_ERR_OOM, (n, e)
            torch.cuda.synchronize()
            assert impact.live_bytes() == base, n      # everything taken was given back
            continue
        impact.fail_alloc(0)
        if check:
            check(res)
        return n
    impact.fail_alloc(0)
    raise AssertionError("the call never succeeded")


def test_out_of_memory_paths_release_everything():
    prob = small()
    ref = impact.build(prob, "fp32")
    rb = impact.alloc_rows(prob.rows)
    pb = impact.alloc_pairs(ref.nnz, "fp32")

    # every sweep below reaches the call's own allocations (n >= 2 means at
    # least one allocation was made to fail on the way)
    def lib_owned():
        return impact.build_library_owned(prob, "fp32")
    assert _oom_sweep(lib_owned, lambda r: r[1] == ref.nnz) >= 2

    def count_scratch():   # impact_batch_count with the library's own workspace
        return impact.Batch([prob, W.robot_2d(cells_per_dim=7)], "fp32").count(rb)
    assert _oom_sweep(count_scratch) >= 2

    def build_into_scratch():   # impact_batch_build into caller arrays, library workspace
        return impact.Batch([prob], "fp32").build_into(rb, pb, ref.nnz)
    assert _oom_sweep(build_into_scratch, lambda n: n == ref.nnz) >= 2

    def graph():
        g = impact.Batch([prob], "fp32").graph(rb, pb, ref.nnz)
        g.launch()
        torch.cuda.synchronize()
        n = g.result()
        g.close()
        return n
    assert _oom_sweep(graph, lambda n: n == ref.nnz) >= 2
    robot = W.robot_2d(cells_per_dim=9)
    imdp = impact.build(robot, "fp64")
    labels = impact.label_cells(robot, target=[([3.0, 3.0], [7.0, 7.0])])
    assert _oom_sweep(lambda: impact.synthesize(imdp, robot, labels, max_iters=50)) >= 2
    assert _oom_sweep(lambda: impact.region_vectors(robot,
                                                    target=[([3.0, 3.0], [7.0, 7.0])])) >= 2
    draws = np.random.default_rng(0).standard_normal((64, robot.n)) * 0.5
    assert _oom_sweep(lambda: impact.build_mc(robot, draws, "fp64")) >= 2


def test_server_request_fails_cleanly_under_an_allocation_failure():
    prob = small()
    ref = impact.build(prob, "fp32")
    with impact.Server("fp32") as srv:
        impact.fail_alloc(1)                          # the next group's first allocation
        t = srv.submit(prob)
        with pytest.raises(impact.ImpactError) as e:
            srv.poll(t, wait=True)
        impact.fail_alloc(0)
        assert e.value.status == impact.IMPACT_ERR_OOM
        srv.release(t)
        t2 = srv.submit(prob)                         # the server carries on
        srv.poll(t2, wait=True)
        assert_same(srv.result(t2), ref)
        srv.release(t2)
