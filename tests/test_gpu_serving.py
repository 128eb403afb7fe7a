"""Serving runtime on the GPU: queued solves admitted as slots and the HBM
budget allow, overlapping on the device, with each result equal to the same
solve run alone."""
import time

import numpy as np
import pytest

from oracle import pf_oracle as O
from paper_1711_10579_gb300 import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1711_10579_gb300 import pf as _pf

    return _pf


def _wait(pf, ctx, tickets, slots, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            r = pf.pf_poll(ctx, t, slots[t])
            if r is not None:
                out[t] = r
        assert time.time() - t0 < timeout, "served requests did not finish"
        time.sleep(0.001)
    return out


def _requests(rng, pool, n_req):
    reqs = []
    for k in range(n_req):
        ci = int(rng.integers(0, len(pool)))
        case = pool[ci][0]
        if isinstance(case, cases.SinglePhaseCase):
            pl, ql, pg = cases.scenario_loads(case, 1, seed=int(rng.integers(1 << 30)), sigma=0.1)
            reqs.append((ci, pl[0], ql[0], pg[0]))
        else:
            pl, ql = cases.feeder_scenario_loads(case, 1, seed=int(rng.integers(1 << 30)), sigma=0.1)
            reqs.append((ci, pl[0].reshape(-1), ql[0].reshape(-1), None))
    return reqs


def test_served_results_equal_standalone_solves(pf):
    ctx = pf.pf_ctx_create(0)
    try:
        pool = []
        # the last two run on 4-CTA clusters (16,000 buses, 5,000 feeder nodes and more)
        for case in (cases.transmission_case(800, 1080, 160, 1), cases.case_2000bus(3),
                     cases.feeder_case(600, 2), cases.transmission_case(5000, 6750, 1000, 4),
                     cases.transmission_case(17000, 22950, 3400, 5), cases.feeder_case(5200, 6)):
            pool.append((case, pf.pf_create_case(ctx, case)))
        rng = np.random.default_rng(0)
        reqs = _requests(rng, pool, 48)
        opts = pf.make_opts(warm_start=0)
        tickets, slots = [], {}
        for ci, pl, ql, pg in reqs:
            t = pf.pf_submit(ctx, pool[ci][1], pl, ql, pg, opts)
            tickets.append(t)
            slots[t] = pool[ci][1].slots
        res = _wait(pf, ctx, tickets, slots)
        # the requests overlapped on the GPU: several of them in one launch
        # of cases of different sizes, and several on the GPU at once
        st = pf.pf_serve_get_stats(ctx)
        assert st["requests"] == len(reqs)
        assert st["max_group"] > 1 and st["peak_running"] > 1
        assert st["group_launches"] < len(reqs)
        for k, (ci, pl, ql, pg) in enumerate(reqs):
            vm, va, info = res[tickets[k]]
            assert info["status"] == 0 and info["mismatch"] <= 1e-8, info
            h = pool[ci][1]
            vm1, va1, info1 = pf.pf_solve_batch(h, pl[None], ql[None],
                                                None if pg is None else pg[None], opts)
            # the same launch alone: identical result
            assert np.max(np.abs(vm - vm1[0])) <= 1e-12
            assert np.max(np.abs(va - va1[0])) <= 1e-12
        # a sample against the oracle
        for k in range(0, len(reqs), 12):
            ci, pl, ql, pg = reqs[k]
            case = pool[ci][0]
            vm, va, _ = res[tickets[k]]
            if pg is not None:
                ref = O.newton_polar(case.with_loads(pl, ql, pg))
                assert np.max(np.abs(vm - ref["vm"])) <= 1e-6
                assert np.max(np.abs(va - ref["va"])) <= 1e-6
            else:
                ref = O.newton_cim(case.with_loads(pl.reshape(-1, 3), ql.reshape(-1, 3)))
                assert np.max(np.abs(vm - np.abs(ref["V"]))) <= 1e-6
        for _, h in pool:
            pf.pf_destroy_case(h)
    finally:
        pf.pf_ctx_destroy(ctx)


def test_warm_started_serving_matches_cold_within_tolerance(pf):
    ctx = pf.pf_ctx_create(0)
    try:
        case = cases.case_2000bus(5)
        h = pf.pf_create_case(ctx, case)
        pl, ql, pg = cases.scenario_loads(case, 8, seed=3, sigma=0.05)
        warm = pf.make_opts(warm_start=1)
        tickets = [pf.pf_submit(ctx, h, pl[k], ql[k], pg[k], warm) for k in range(8)]
        res = _wait(pf, ctx, tickets, {t: h.slots for t in tickets})
        for k, t in enumerate(tickets):
            vm, va, info = res[t]
            assert info["status"] == 0
            vm1, va1, _ = pf.pf_solve_batch(h, pl[k:k + 1], ql[k:k + 1], pg[k:k + 1],
                                            pf.make_opts(warm_start=0))
            assert np.max(np.abs(vm - vm1[0])) <= 1e-6
            assert np.max(np.abs(va - va1[0])) <= 1e-6
        pf.pf_destroy_case(h)
    finally:
        pf.pf_ctx_destroy(ctx)


def test_admission_by_hbm_budget(pf):
    # a budget that holds the resident cases plus about one request at a time
    probe = pf.pf_ctx_create(0)
    case = cases.case_2000bus(6)
    h = pf.pf_create_case(probe, case)
    per_req = pf.pf_case_get_stats(h)["bytes_per_scenario"]
    pf.pf_destroy_case(h)
    pf.pf_ctx_destroy(probe)
    ctx = pf.pf_ctx_create(0, int(1.5 * per_req))
    try:
        h = pf.pf_create_case(ctx, case)
        pl, ql, pg = cases.scenario_loads(case, 6, seed=4, sigma=0.05)
        tickets = [pf.pf_submit(ctx, h, pl[k], ql[k], pg[k]) for k in range(6)]
        res = _wait(pf, ctx, tickets, {t: h.slots for t in tickets})
        assert all(r[2]["status"] == 0 for r in res.values())
        # larger than the whole budget: refused with PF_ERR_NOMEM, not hung
        big = cases.case_10000bus(0)
        hb = pf.pf_create_case(ctx, big)
        t = pf.pf_submit(ctx, hb, None, None, None)
        r = _wait(pf, ctx, [t], {t: hb.slots})[t]
        assert r[2]["status"] == pf.PF_ERR_NOMEM
        pf.pf_destroy_case(hb)
        pf.pf_destroy_case(h)
    finally:
        pf.pf_ctx_destroy(ctx)


def test_serving_errors_are_reported_on_the_host(pf):
    ctx = pf.pf_ctx_create(0)
    try:
        with pytest.raises(pf.PfError) as e:
            pf.pf_poll(ctx, 123456789, 1)
        assert e.value.code == pf.PF_ERR_INVALID
        case = cases.case_10000bus(1)
        h = pf.pf_create_case(ctx, case)
        t = pf.pf_submit(ctx, h)
        # an immediate drain with no time left reports the pending request
        try:
            pf.pf_drain(ctx, 0)
        except pf.PfError as err:
            assert err.code == pf.PF_ERR_TIMEOUT
        pf.pf_drain(ctx, 60_000)
        r = pf.pf_poll(ctx, t, h.slots)
        assert r is not None and r[2]["status"] == 0
        pf.pf_destroy_case(h)
    finally:
        pf.pf_ctx_destroy(ctx)


def test_served_solves_enforce_reactive_limits(pf):
    """Requests with opts.q_limits on cases with limits (single phase and a
    three-phase feeder with PV nodes) give the oracle's switched solutions."""
    ctx = pf.pf_ctx_create(0)
    try:
        c1 = cases.with_q_limits(cases.transmission_case(300, 405, 60, 2), 1)
        c3 = cases.with_phase_q_limits(cases.with_pv_nodes(cases.feeder_case(400, 3), 8, 3), 1)
        h1, h3 = pf.pf_create_case(ctx, c1), pf.pf_create_case(ctx, c3)
        o = pf.make_opts(q_limits=1)
        tickets, slots = [], {}
        for k in range(3):
            t = pf.pf_submit(ctx, h1, c1.p_load, c1.q_load, c1.p_gen, o)
            tickets.append(t)
            slots[t] = h1.slots
            t = pf.pf_submit(ctx, h3, c3.p_load.reshape(-1), c3.q_load.reshape(-1), None, o)
            tickets.append(t)
            slots[t] = h3.slots
        out = _wait(pf, ctx, tickets, slots)
        r1 = O.newton_polar_qlim(c1)
        r3 = O.newton_cim_qlim(c3)
        for t in tickets:
            vm, va, info = out[t]
            assert info["status"] == 0 and info["q_switched"] > 0
            if slots[t] == h1.slots:
                assert info["q_switched"] == int(r1["switched"].sum())
                assert np.max(np.abs(vm - r1["vm"])) <= 1e-6
                assert np.max(np.abs(va - r1["va"])) <= 1e-6
            else:
                assert info["q_switched"] == int(r3["switched"].sum())
                assert np.max(np.abs(vm - np.abs(r3["V"]))) <= 1e-6
        pf.pf_destroy_case(h1)
        pf.pf_destroy_case(h3)
    finally:
        pf.pf_ctx_destroy(ctx)


def test_served_fp64_and_newton_krylov_requests(pf):
    """FP64 Newton-Raphson requests (group launches in FP64, one CTA and a
    4-CTA cluster) equal the same solves run alone; Newton-Krylov requests
    (one launch each) match the oracle, and one that does not converge falls
    back to Newton-Raphson; all kinds mixed in one stream."""
    ctx = pf.pf_ctx_create(0)
    try:
        small = cases.case_2000bus(2)
        large = cases.transmission_case(17000, 22950, 3400, 7)
        hs, hl = pf.pf_create_case(ctx, small), pf.pf_create_case(ctx, large)
        f64 = pf.make_opts(precision=pf.PF_FP64)
        nk = pf.make_opts(method=pf.PF_NK)
        jobs = []
        for k in range(6):
            case, h = (small, hs) if k % 2 == 0 else (large, hl)
            pl, ql, pg = cases.scenario_loads(case, 1, seed=40 + k, sigma=0.1)
            o = nk if k in (2, 4) else f64
            jobs.append((case, h, pl, ql, pg, o, pf.pf_submit(ctx, h, pl[0], ql[0], pg[0], o)))
        # a Newton-Krylov request that GMRES cannot finish (2 inner iterations
        # per Newton step) is solved again with Newton-Raphson, as pf_solve does
        starved = pf.make_opts(method=pf.PF_NK, gmres_max_iter=2)
        pl, ql, pg = cases.scenario_loads(large, 1, seed=60, sigma=0.1)
        jobs.append((large, hl, pl, ql, pg, starved, pf.pf_submit(ctx, hl, pl[0], ql[0], pg[0],
                                                                  starved)))
        res = _wait(pf, ctx, [j[-1] for j in jobs], {j[-1]: j[1].slots for j in jobs})
        assert res[jobs[-1][-1]][2]["fallback"] == 1
        for case, h, pl, ql, pg, o, t in jobs:
            vm, va, info = res[t]
            assert info["status"] == 0 and info["mismatch"] <= 1e-8, info
            if o.method == pf.PF_NR:
                vm1, va1, _ = pf.pf_solve_batch(h, pl, ql, pg, o)
                assert np.max(np.abs(vm - vm1[0])) <= 1e-12
                assert np.max(np.abs(va - va1[0])) <= 1e-12
            else:
                ref = O.newton_polar(case.with_loads(pl[0], ql[0], pg[0]))
                assert np.max(np.abs(vm - ref["vm"])) <= 1e-6
                assert np.max(np.abs(va - ref["va"])) <= 1e-6
        pf.pf_destroy_case(hs)
        pf.pf_destroy_case(hl)
    finally:
        pf.pf_ctx_destroy(ctx)


def test_queued_requests_of_one_case_coalesce_into_a_batch(pf):
    """Requests of one case queued together (pf_submit_batch) run as one
    batched solve instead of one CTA each: every result equals pf_solve_batch
    of the same loads (the same kernels and launch), a request of the case
    with other options in the same burst runs on its own, and a sample
    matches the oracle."""
    ctx = pf.pf_ctx_create(0)
    try:
        case = cases.case_2000bus(2)
        h = pf.pf_create_case(ctx, case)
        B = 40
        pl, ql, pg = cases.scenario_loads(case, B, seed=17)
        opts = pf.make_opts()
        tickets = pf.pf_submit_batch(ctx, h, pl, ql, pg, opts)
        other = pf.make_opts(tol=1e-10)
        t_other = pf.pf_submit(ctx, h, pl[0], ql[0], pg[0], other)
        slots = {t: h.slots for t in tickets + [t_other]}
        res = _wait(pf, ctx, tickets + [t_other], slots)
        st = pf.pf_serve_get_stats(ctx)
        assert st["batch_launches"] == 1 and st["max_batch"] == B
        assert st["requests"] == B + 1
        vm_b, va_b, inf_b = pf.pf_solve_batch(h, pl, ql, pg, opts)
        for k, t in enumerate(tickets):
            vm, va, info = res[t]
            assert info["status"] == 0 and info["mismatch"] <= 1e-8, info
            assert info["iterations"] == inf_b["iterations"][k]
            assert np.max(np.abs(vm - vm_b[k])) <= 1e-12
            assert np.max(np.abs(va - va_b[k])) <= 1e-12
        vm, va, info = res[t_other]
        assert info["status"] == 0 and info["mismatch"] <= 1e-10, info
        for k in (0, B - 1):
            ref = O.newton_polar(case.with_loads(pl[k], ql[k], pg[k]))
            vm, va, _ = res[tickets[k]]
            assert np.max(np.abs(vm - ref["vm"])) <= 1e-6
            assert np.max(np.abs(va - ref["va"])) <= 1e-6
        pf.pf_destroy_case(h)
    finally:
        pf.pf_ctx_destroy(ctx)
