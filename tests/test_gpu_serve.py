"""Continuous-batching server: requests of mixed size and storage arrive over
time, share the GPU in batches, and each result equals (bitwise) the result
of running that request alone. Admission respects the memory budget."""
import numpy as np
import pytest

import inputs
from paper_1708_01613_gb300.serve import FoamServer, Request, footprint_bytes, run_one_at_a_time, summarize



def requests():
    spec = [(256, 256, "f16", 48, 0.000), (192, 128, "f32", 30, 0.002), (320, 64, "f16", 75, 0.004),
            (512, 512, "f32", 40, 0.010), (128, 128, "f16", 61, 0.015), (256, 192, "f32", 22, 0.020)]
    out = []
    for i, (nx, ny, storage, steps, t) in enumerate(spec):
        bub = inputs.poisson_disk_bubbles(nx, ny, 3, 5.0, 0.15 * min(nx, ny), 2.0, seed=500 + i)
        out.append(Request(i, t, nx, ny, bub, steps, storage, inputs.RHO_LIQ_G55, inputs.RHO_GAS_G55, True, 4))
    return out


@pytest.mark.gpu
def test_served_results_equal_lone_runs_and_budget_holds():
    reqs = requests()
    # room for the two largest boxes at most: the rest queue behind them
    budget = sorted(footprint_bytes(r) for r in reqs)[-1] + sorted(footprint_bytes(r) for r in reqs)[-2]
    server = FoamServer(memory_budget_bytes=budget, max_boxes=4, quantum_updates=2e6, keep_pops=True)
    served = {r.rid: r for r in server.run(reqs)}
    assert sorted(served) == [r.rid for r in reqs]
    assert server.stats["peak_bytes"] <= budget
    assert server.stats["batch_rebuilds"] >= 3
    alone, _ = run_one_at_a_time(reqs, keep_pops=True)
    for a in alone:
        s = served[a.rid]
        assert np.array_equal(s.pops, a.pops), a.rid
        assert s.mass == a.mass and s.n_bubbles == a.n_bubbles
        assert s.latency_s >= 0 and s.done_s >= s.admit_s >= s.arrival_s - 1e-9
    summ = summarize(list(served.values()), server.stats["makespan_s"])
    assert summ["requests"] == 6 and summ["p99_s"] >= summ["p50_s"] > 0


def test_fair_steps_water_filling():
    """Pure host logic: equal shares of the update budget, small jobs finish
    inside their share and hand the rest on, everybody moves."""
    from paper_1708_01613_gb300.serve import _Job, fair_steps

    def job(rid, nx, ny, rem):
        return _Job(Request(rid, 0.0, nx, ny, np.zeros((0, 3)), rem), None, rem, 0.0, 0)

    jobs = [job(0, 100, 100, 50), job(1, 1000, 1000, 1000), job(2, 1000, 100, 1000), job(3, 10, 10, 10**6)]
    s = fair_steps(jobs, 4e6)
    # by remaining work: job 0 (5e5 updates) fits its 1e6 share; jobs 2 and 3
    # (1e8 each) split 3.5e6 three ways, then 2.4e6 two ways; job 1 gets the rest
    assert s == {0: 50, 2: 11, 3: 12000, 1: 1}
    assert sum(s[j.req.rid] * j.cells for j in jobs) <= 4e6 + 1e6
    assert all(v >= 1 for v in fair_steps(jobs, 1.0).values())
    assert fair_steps(jobs, 1e12) == {0: 50, 1: 1000, 2: 1000, 3: 10**6}


def test_time_share_and_lockstep_plans():
    from paper_1708_01613_gb300.serve import _Job, fair_time_steps, lockstep_steps

    def job(rid, cells, rem):
        return _Job(Request(rid, 0.0, cells, 1, np.zeros((0, 3)), rem), None, rem, 0.0, 0)

    jobs = [job(0, 100, 1000), job(1, 10**6, 1000)]
    # step costs 1e-5 + 1e-9 * cells: 1.01e-5 s and 1.01e-3 s; budget 0.02 s
    # -> job 0 wants 1000 * 1.01e-5 = 0.0101 s > 0.01 s share: 990 steps,
    #    job 1 gets the rest: (0.02 - 990 * 1.01e-5) / 1.01e-3 -> 9 steps
    assert fair_time_steps(jobs, 0.02, 1e-5, 1e-9) == {0: 990, 1: 9}
    # lockstep: each launch costs 1e-5 + 1e-9 * 1000100 = 1.0101e-3 s -> 19 launches
    assert lockstep_steps(jobs, 0.02, 1e-5, 1e-9) == {0: 19, 1: 19}
    # short job ends after 5 launches, the rest are cheaper
    jobs = [job(0, 10**6, 5), job(1, 100, 10**5)]
    t5 = 5 * (1e-5 + 1e-9 * 1000100)
    more = int((0.02 - t5) // (1e-5 + 1e-7))
    assert lockstep_steps(jobs, 0.02, 1e-5, 1e-9) == {0: 5, 1: 5 + more}
    assert lockstep_steps(jobs, 0.0, 1e-5, 1e-9) == {0: 1, 1: 1}


def test_tiered_plan():
    from paper_1708_01613_gb300.serve import _Job, tiered_steps

    def job(rid, t, cells, rem):
        return _Job(Request(rid, t, cells, 1, np.zeros((0, 3)), rem), None, rem, 0.0, 0)

    jobs = [job(0, 0.2, 100, 10), job(1, 0.1, 10**6, 1000), job(2, 0.0, 10**6, 500), job(3, 0.3, 1000, 10**4)]
    s = tiered_steps(jobs, 4e6, big_updates=1e8)
    # small jobs 0 and 3 share half the budget (job 0 needs 1e3 updates, job 3
    # gets the rest of 2e6); big job 2 arrived first and takes the remainder;
    # big job 1 waits
    assert s[0] == 10 and s[3] == int((2e6 - 1e3) // 1000)
    assert s[2] == int((4e6 - 1e3 - s[3] * 1000) // 10**6) and s[1] == 0
    only_small = tiered_steps(jobs[:1] + jobs[3:], 4e6, big_updates=1e8)
    assert only_small == {0: 10, 3: int((4e6 - 1e3) // 1000)}
    # a big job past its slowdown bound: the small ones move one step, the
    # big one takes the rest of the quantum
    late = tiered_steps(jobs, 4e6, big_updates=1e8, small_share=0.0)
    assert late[0] == 1 and late[3] == 1 and late[1] == 0
    assert late[2] == int((4e6 - 100 - 1000) // 10**6)


def test_ordered_fill_plans():
    """Pure host logic of the "fifo" and "srpt" policies: jobs take all their
    remaining steps in the given order until the update budget runs out; the
    first job in the order always moves; the rest wait."""
    from paper_1708_01613_gb300.serve import _Job, ordered_steps

    def job(rid, t, cells, rem):
        return _Job(Request(rid, t, cells, 1, np.zeros((0, 3)), rem), None, rem, 0.0, 0)

    jobs = [job(0, 0.2, 100, 10), job(1, 0.1, 10**6, 1000), job(2, 0.0, 10**6, 3), job(3, 0.3, 1000, 10**4)]
    fifo = ordered_steps(jobs, 4e6, key=lambda j: (j.req.arrival_s, j.req.rid))
    # job 2 (first) takes its 3 steps (3e6 updates), job 1 the one step that
    # fits the last 1e6; jobs 0 and 3 wait
    assert fifo == {2: 3, 1: 1, 0: 0, 3: 0}
    srpt = ordered_steps(jobs, 4e6, key=lambda j: j.remaining * j.cells)
    # by remaining work: job 0 (1e3), job 2 (3e6), job 3 (1e7: 999 steps of
    # the 999000 left), job 1 nothing
    assert srpt == {0: 10, 2: 3, 3: 999, 1: 0}
    assert ordered_steps(jobs, 0.0, key=lambda j: j.req.rid) == {0: 1, 1: 0, 2: 0, 3: 0}
    assert sum(srpt[j.req.rid] * j.cells for j in jobs) <= 4e6


def test_order_keys_of_the_ordered_policies():
    """Pure host logic: the orders "fifo", "express", "srpt" and "hrrn" put
    the jobs where their definitions say, at one time of the stream."""
    from paper_1708_01613_gb300.serve import _Job, order_key

    def job(rid, t, cells, rem):
        return _Job(Request(rid, t, cells, 1, np.zeros((0, 3)), rem), None, rem, 0.0, 0)

    # at now = 10 s with 1e-9 s per update: remaining GPU time 1e-3, 5.0, 2.0, 0.01 s;
    # waited 9, 8, 2, 1 s
    jobs = [job(0, 1.0, 10**4, 100), job(1, 2.0, 10**6, 5000), job(2, 8.0, 10**6, 2000), job(3, 9.0, 10**5, 100)]
    order = lambda pol, **kw: [j.req.rid for j in sorted(jobs, key=order_key(pol, 10.0, 1e-9, **kw))]
    assert order("fifo") == [0, 1, 2, 3]
    assert order("express", big_s=0.02) == [0, 3, 1, 2]
    # srpt: remaining - w * waited: w = 0: 0.001, 5, 2, 0.01; w = 1: -8.999, -3, 0, -0.99
    assert order("srpt", age_weight=0.0) == [0, 3, 2, 1]
    assert order("srpt", age_weight=1.0) == [0, 1, 3, 2]
    # hrrn: waited / remaining = 9000, 1.6, 1, 100
    assert order("hrrn") == [0, 3, 1, 2]
    with pytest.raises(ValueError):
        order_key("tiered", 0.0, 1e-9)


@pytest.mark.gpu
def test_request_larger_than_budget_is_refused():
    r = requests()[3]
    with pytest.raises(ValueError):
        FoamServer(memory_budget_bytes=footprint_bytes(r) - 1).run([r])


@pytest.mark.gpu
def test_served_results_match_oracle():
    """A served mix (FP32 and FP16 deviation storage, barrier on, K = 4,
    staggered arrivals, queueing under a memory budget) against one FP64
    oracle run per request, from the same initial density: FP32 populations
    within 1e-5, FP16 within 2e-3 on rho."""
    import oracle as O

    reqs = requests()
    budget = sorted(footprint_bytes(r) for r in reqs)[-1] + sorted(footprint_bytes(r) for r in reqs)[-2]
    server = FoamServer(memory_budget_bytes=budget, max_boxes=4, quantum_updates=2e6, keep_pops=True)
    served = {r.rid: r for r in server.run(reqs)}
    for r in reqs:
        P = O.make_params(r.nx, r.ny, barrier=True, relabel_every=4)
        ref = O.OracleSim(P)
        ref.init_density(O.init_bubbles(P, r.bubbles, r.rho_l, r.rho_g, 4.0))
        ref.step(r.steps)
        got = served[r.rid]
        if r.storage == "f32":
            err = float(np.max(np.abs(got.pops - ref.f)) / np.max(np.abs(ref.f)))
            tol = 1e-5
        else:
            f16 = got.pops.astype(np.float64)
            rho = ref.f.sum(0)
            err = float(np.max(np.abs(f16.sum(0) - rho)) / np.max(np.abs(rho)))
            tol = 2e-3
        print(f"served {r.rid} {r.nx}x{r.ny} {r.storage} {r.steps} steps: rel err {err:.3e}")
        assert err < tol, (r.rid, err)
