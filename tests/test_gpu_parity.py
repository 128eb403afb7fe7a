"""GPU parity: every step of the Newton iteration, through the C ABI, against
the FP64 oracle on the same seeded inputs.

Tolerances: mismatch and Jacobian entries are FP64 arithmetic on both sides
(rectangular form on the GPU, trigonometric form in the oracle), so they
agree to ~1e-12 relative; a converged solve must match the oracle within
|dV| <= 1e-6 pu and |dtheta| <= 1e-6 rad at a mismatch <= 1e-8 pu.
"""
import numpy as np
import pytest

from oracle import pf_oracle as O
from paper_1711_10579_gb300 import cases

pytestmark = pytest.mark.gpu

V_TOL = 1e-6
A_TOL = 1e-6


@pytest.fixture(scope="module")
def pf():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1711_10579_gb300 import pf as _pf

    return _pf


@pytest.fixture(scope="module")
def ctx(pf):
    h = pf.pf_ctx_create(0)
    yield h
    pf.pf_ctx_destroy(h)


def _zip_case(case, seed):
    import dataclasses as dc

    z = np.random.default_rng(seed).dirichlet([1, 1, 1], case.n_bus)
    return dc.replace(case, zip=z)


def _rand_v(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.9, 1.1, n), rng.uniform(-0.3, 0.3, n)


def _oracle_blocks(case, Y, vm, va):
    """Oracle Jacobian (Eq. 10) regrouped into 2x2 blocks on the Ybus pattern."""
    J = O.jacobian_polar(case, Y, vm, va).tocsr()
    pvpq, pq = O.unknowns_polar(case)
    n = case.n_bus
    ip = np.full(n, -1)
    ip[pvpq] = np.arange(pvpq.size)
    iq = np.full(n, -1)
    iq[pq] = pvpq.size + np.arange(pq.size)
    Yc = Y.tocsr()
    Yc.sort_indices()
    out = np.zeros((Yc.nnz, 2, 2))
    for i in range(n):
        for p in range(Yc.indptr[i], Yc.indptr[i + 1]):
            j = Yc.indices[p]
            rows = (ip[i], iq[i])
            cols = (ip[j], iq[j])
            for a in range(2):
                for b in range(2):
                    if rows[a] >= 0 and cols[b] >= 0:
                        out[p, a, b] = J[rows[a], cols[b]]
                    elif i == j and a == b:
                        out[p, a, b] = 1.0
    return out


def _gpu_mis_to_oracle_order(case, mis):
    pvpq, pq = O.unknowns_polar(case)
    return np.concatenate([mis[pvpq, 0], mis[pq, 1]])


# ----------------------------------------------------------------------------
# single phase, step by step
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["14", "300zip", "2000"])
def test_mismatch_and_jacobian_single_phase(pf, ctx, name):
    case = {"14": cases.case_14bus(0),
            "300zip": _zip_case(cases.transmission_case(300, 405, 60, 2), 2),
            "2000": cases.case_2000bus(0)}[name]
    Y = O.ybus_single(case)
    c = pf.pf_create_case(ctx, case)
    try:
        for seed in range(3):
            vm, va = _rand_v(case.n_bus, seed)
            mis = pf.pf_eval_mismatch(c, vm, va)
            ref = O.mismatch_polar(case, Y, vm, va)
            got = _gpu_mis_to_oracle_order(case, mis)
            assert np.max(np.abs(got - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))
            # rows without an equation are exactly zero
            assert np.all(mis[case.bus_type == cases.SLACK] == 0)
            assert np.all(mis[case.bus_type == cases.PV, 1] == 0)
            st = pf.pf_case_get_stats(c)
            blocks = pf.pf_eval_jacobian(c, vm, va, st["nnz_y"])
            ref_b = _oracle_blocks(case, Y, vm, va)
            scale = max(1.0, np.max(np.abs(ref_b)))
            assert np.max(np.abs(blocks - ref_b)) <= 1e-11 * scale
    finally:
        pf.pf_destroy_case(c)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
@pytest.mark.parametrize("name", ["300zip", "2000"])
def test_newton_step_matches_oracle_solve(pf, ctx, name, prec, tol):
    case = {"300zip": _zip_case(cases.transmission_case(300, 405, 60, 2), 2),
            "2000": cases.case_2000bus(0)}[name]
    Y = O.ybus_single(case)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va = O.flat_start_polar(case)
        vm = vm + np.where(case.bus_type == cases.PQ, 0.01 * np.sin(np.arange(case.n_bus)), 0)
        va = va + np.where(case.bus_type != cases.SLACK, 0.02 * np.cos(np.arange(case.n_bus)), 0)
        p = pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED
        dx, _ = pf.pf_newton_step(c, vm, va, pf.make_opts(precision=p, refine_steps=2))
        F = O.mismatch_polar(case, Y, vm, va)
        ref = O.solve_linear(O.jacobian_polar(case, Y, vm, va), F, "splu")
        got = _gpu_mis_to_oracle_order(case, dx)
        assert np.max(np.abs(got - ref)) <= tol * max(1.0, np.max(np.abs(ref)))
        assert np.all(dx[case.bus_type == cases.SLACK] == 0)
        assert np.all(dx[case.bus_type == cases.PV, 1] == 0)
    finally:
        pf.pf_destroy_case(c)


# ----------------------------------------------------------------------------
# single phase, full solves
# ----------------------------------------------------------------------------

def _check_solve(case, vm, va, info, ref):
    assert info["status"] == 0, info
    assert info["mismatch"] <= 1e-8
    assert np.max(np.abs(vm - ref["vm"])) <= V_TOL
    assert np.max(np.abs(va - ref["va"])) <= A_TOL


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["14", "300zip", "2000", "10000"])
def test_solve_single_phase_matches_oracle(pf, ctx, name, prec):
    case = {"14": cases.case_14bus(0),
            "300zip": _zip_case(cases.transmission_case(300, 405, 60, 2), 2),
            "2000": cases.case_2000bus(0), "10000": cases.case_10000bus(0)}[name]
    ref = O.newton_polar(case)
    assert ref["converged"]
    c = pf.pf_create_case(ctx, case)
    try:
        p = pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED
        vm, va, info = pf.pf_solve(c, pf.make_opts(precision=p))
        _check_solve(case, vm, va, info, ref)
        assert info["iterations"] <= ref["iterations"] + 2
        assert info["solve_us"] > 0
    finally:
        pf.pf_destroy_case(c)


@pytest.mark.parametrize("cluster,threads", [(1, 1024), (2, 512), (8, 256), (16, 1024), (4, 128)])
def test_launch_shapes_agree(pf, ctx, cluster, threads):
    case = cases.case_2000bus(1)
    ref = O.newton_polar(case)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve(c, pf.make_opts(cluster_size=cluster, block_threads=threads))
        _check_solve(case, vm, va, info, ref)
    finally:
        pf.pf_destroy_case(c)


def test_warm_start_reuses_the_last_solution(pf, ctx):
    case = cases.case_2000bus(2)
    ref = O.newton_polar(case)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve(c)
        _check_solve(case, vm, va, info, ref)
        vm2, va2, info2 = pf.pf_solve(c, pf.make_opts(warm_start=1))
        _check_solve(case, vm2, va2, info2, ref)
        assert info2["iterations"] <= 1
    finally:
        pf.pf_destroy_case(c)


def test_edge_cases(pf, ctx):
    one = cases.SinglePhaseCase(
        n_bus=1, bus_type=np.array([0], np.int32), v_set=np.array([1.02]), p_gen=np.zeros(1),
        q_gen=np.zeros(1), p_load=np.zeros(1), q_load=np.zeros(1), zip=np.array([[1.0, 0, 0]]),
        br_from=np.zeros(0, np.int32), br_to=np.zeros(0, np.int32), br_r=np.zeros(0),
        br_x=np.zeros(0), br_b=np.zeros(0))
    c = pf.pf_create_case(ctx, one)
    vm, va, info = pf.pf_solve(c)
    assert info["status"] == 0 and info["iterations"] == 0 and vm[0] == 1.02
    pf.pf_destroy_case(c)
    # two-bus closed form through the GPU
    tb = cases.two_bus_case(0.9, 0.3, 0.02, 0.15)
    ref = O.newton_polar(tb)
    c = pf.pf_create_case(ctx, tb)
    vm, va, info = pf.pf_solve(c, pf.make_opts(precision=pf.PF_FP64))
    _check_solve(tb, vm, va, info, ref)
    # no iteration allowed: reports MAXITER with the flat-start mismatch
    vm, va, info = pf.pf_solve(c, pf.make_opts(max_iter=0))
    assert info["status"] == pf.PF_ERR_MAXITER and info["iterations"] == 0
    pf.pf_destroy_case(c)
    # far beyond the nose of the PV curve: no solution exists
    bad = cases.two_bus_case(50.0, 20.0, 0.02, 0.15)
    c = pf.pf_create_case(ctx, bad)
    vm, va, info = pf.pf_solve(c, pf.make_opts(max_iter=20))
    assert info["status"] in (pf.PF_ERR_MAXITER, pf.PF_ERR_DIVERGED, pf.PF_ERR_SINGULAR)
    pf.pf_destroy_case(c)


# ----------------------------------------------------------------------------
# batches of scenarios
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("B,S", [(37, 2), (64, 4), (100, 32), (512, 0)])
def test_batch_matches_oracle_and_single(pf, ctx, B, S):
    case = cases.case_2000bus(0)
    p_load, q_load, p_gen = cases.scenario_loads(case, B, seed=11)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve_batch(c, p_load, q_load, p_gen, pf.make_opts(scen_per_cta=S))
        assert np.all(info["status"] == 0), info["status"]
        assert np.all(info["mismatch"] <= 1e-8)
        for b in sorted({0, B // 2, B - 1}):
            ref = O.newton_polar(case.with_loads(p_load[b], q_load[b], p_gen[b]))
            assert np.max(np.abs(vm[b] - ref["vm"])) <= V_TOL
            assert np.max(np.abs(va[b] - ref["va"])) <= A_TOL
            # the same scenario solved alone
            c1 = pf.pf_create_case(ctx, case.with_loads(p_load[b], q_load[b], p_gen[b]))
            vm1, va1, _ = pf.pf_solve(c1)
            pf.pf_destroy_case(c1)
            assert np.max(np.abs(vm[b] - vm1)) <= 1e-9
            assert np.max(np.abs(va[b] - va1)) <= 1e-9
    finally:
        pf.pf_destroy_case(c)


def test_device_entry_point_matches_host_entry_point(pf, ctx):
    torch = pytest.importorskip("torch")
    case = cases.case_2000bus(3)
    B = 16
    p_load, q_load, p_gen = cases.scenario_loads(case, B, seed=5)
    c = pf.pf_create_case(ctx, case)
    try:
        vm_h, va_h, info_h = pf.pf_solve_batch(c, p_load, q_load, p_gen)
        dev = torch.device("cuda:0")
        t = [torch.tensor(a, device=dev) for a in (p_load, q_load, p_gen)]
        vm_d = torch.zeros((B, case.n_bus), dtype=torch.float64, device=dev)
        va_d = torch.zeros_like(vm_d)
        info_d = torch.zeros((B, pf.INFO_DTYPE.itemsize), dtype=torch.uint8, device=dev)
        stream = torch.cuda.current_stream()
        pf.pf_solve_batch_device(c, B, t[0], t[1], t[2], pf.make_opts(), vm_d, va_d, info_d,
                                 stream.cuda_stream)
        torch.cuda.synchronize()
        info = np.frombuffer(info_d.cpu().numpy().tobytes(), dtype=pf.INFO_DTYPE)
        assert np.all(info["status"] == 0)
        assert np.max(np.abs(vm_d.cpu().numpy() - vm_h)) <= 1e-12
        assert np.max(np.abs(va_d.cpu().numpy() - va_h)) <= 1e-12
    finally:
        pf.pf_destroy_case(c)


def test_pinned_host_buffers_are_read_and_written_in_place(pf, ctx):
    """pf_solve_batch on pinned host buffers runs the batch reading the inputs
    and writing the results in place over the host link (no staging copies):
    on a ragged batch its results equal those of pageable buffers (staged
    copies) bit for bit, with the same per-scenario records."""
    torch = pytest.importorskip("torch")
    case = cases.case_2000bus(3)
    B = 37
    p_load, q_load, p_gen = cases.scenario_loads(case, B, seed=6)
    c = pf.pf_create_case(ctx, case)
    try:
        vm_p, va_p, info_p = pf.pf_solve_batch(c, p_load, q_load, p_gen)

        def pinned(shape, dtype=torch.float64):
            return torch.zeros(shape, dtype=dtype, pin_memory=True).numpy()

        h = [pinned(a.shape) for a in (p_load, q_load, p_gen)]
        for dst, src in zip(h, (p_load, q_load, p_gen)):
            dst[...] = src
        vm, va = pinned((B, case.n_bus)), pinned((B, case.n_bus))
        info = pinned((B * pf.INFO_DTYPE.itemsize,), torch.uint8).view(pf.INFO_DTYPE)
        pf.pf_solve_batch(c, h[0], h[1], h[2], out=(vm, va, info))
        assert np.all(info["status"] == 0) and np.all(info["mismatch"] <= 1e-8)
        assert np.array_equal(vm, vm_p) and np.array_equal(va, va_p)
        for k in ("status", "iterations", "linear_iterations", "mismatch", "max_step"):
            assert np.array_equal(info[k], info_p[k]), k
    finally:
        pf.pf_destroy_case(c)


# ----------------------------------------------------------------------------
# three phase (current injection)
# ----------------------------------------------------------------------------

def test_mismatch_over_the_whole_angle_range(pf, ctx):
    """Bus voltages are formed from angles by a table of sin / cos at
    multiples of 2^-7 rad plus a short Taylor series, with sincos() beyond
    |angle| = 4 rad; the mismatch must match the oracle's (numpy sin / cos)
    over the table's range, at its edges and past them."""
    case = cases.case_2000bus(0)
    Y = O.ybus_single(case)
    rng = np.random.default_rng(11)
    n = case.n_bus
    edges = np.array([0.0, 4.0, -4.0, 4.0 - 2.0**-9, -(4.0 - 2.0**-9), 2.0**-8, -2.0**-8,
                      3 * 2.0**-8, 4.0 + 1e-12, -4.0 - 1e-12, 7.5, -12.0, np.pi, -np.pi])
    c = pf.pf_create_case(ctx, case)
    try:
        for seed in range(3):
            vm = rng.uniform(0.9, 1.1, n)
            va = rng.uniform(-6.0, 6.0, n)
            va[: edges.size] = edges
            rng.shuffle(va)
            mis = pf.pf_eval_mismatch(c, vm, va)
            ref = O.mismatch_polar(case, Y, vm, va)
            got = _gpu_mis_to_oracle_order(case, mis)
            assert np.max(np.abs(got - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))
    finally:
        pf.pf_destroy_case(c)


def _rand_v3(case, seed):
    rng = np.random.default_rng(seed)
    V = O.cim_flat_start(case)
    V = V * rng.uniform(0.92, 1.05, V.size) * np.exp(1j * rng.uniform(-0.1, 0.1, V.size))
    return np.abs(V), np.where(np.abs(V) > 0, np.angle(V), 0.0), V


@pytest.mark.parametrize("n", [12, 300])
def test_mismatch_and_jacobian_three_phase(pf, ctx, n):
    case = cases.feeder_case(n, 3, reduced_p=0.5, max_drop=0.08)
    Y = O.ybus_three_phase(case)
    c = pf.pf_create_case(ctx, case)
    try:
        for seed in range(2):
            vm, va, V = _rand_v3(case, seed)
            V = vm * np.exp(1j * va)  # same rounding as the GPU input
            mis = pf.pf_eval_mismatch(c, vm, va)
            ref = O.cim_mismatch(case, Y, V).reshape(n, 6)
            assert np.max(np.abs(mis - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))
            st = pf.pf_case_get_stats(c)
            blocks = pf.pf_eval_jacobian(c, vm, va, st["nnz_y"])
            J = O.cim_jacobian(case, Y, V).toarray()
            rp, col = pf.pf_case_pattern(c, st["nnz_y"])
            free = np.concatenate([O.cim_free_slots(case).reshape(n, 3)] * 2, 1)
            for i in range(n):
                for p in range(rp[i], rp[i + 1]):
                    j = col[p]
                    rb = J[6 * i:6 * i + 6, 6 * j:6 * j + 6].copy()
                    rb[~free[i], :] = 0
                    rb[:, ~free[j]] = 0
                    if i == j:
                        rb[~free[i], ~free[i]] = 1
                    assert np.max(np.abs(blocks[p] - rb)) <= 1e-10 * max(1, np.max(np.abs(rb)))
    finally:
        pf.pf_destroy_case(c)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [200, 8000])
def test_solve_three_phase_matches_oracle(pf, ctx, n, prec):
    case = cases.case_feeder8000(0) if n == 8000 else cases.feeder_case(n, 1)
    ref = O.newton_cim(case)
    assert ref["converged"]
    c = pf.pf_create_case(ctx, case)
    try:
        p = pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED
        vm, va, info = pf.pf_solve(c, pf.make_opts(precision=p))
        assert info["status"] == 0 and info["mismatch"] <= 1e-8, info
        assert np.max(np.abs(vm - np.abs(ref["V"]))) <= V_TOL
        rv = np.where(np.abs(ref["V"]) > 0, np.angle(ref["V"]), 0.0)
        d = np.angle(np.exp(1j * (va - rv)))
        assert np.max(np.abs(d)) <= A_TOL
    finally:
        pf.pf_destroy_case(c)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_newton_step_three_phase_matches_oracle_solve(pf, ctx, prec, tol):
    """One Newton step of the 8,000-node feeder (6x6 blocks; 66 of its 100
    factor levels hold at most 32 items, which a single FP64 solve factors a
    warp per item) against the oracle's sparse direct solve of Eq. 22-23 on
    the free unknowns; absent phases take no step."""
    case = cases.case_feeder8000(0)
    Y = O.ybus_three_phase(case)
    vm, va, _ = _rand_v3(case, 5)
    V = vm * np.exp(1j * va)  # same rounding as the GPU input
    c = pf.pf_create_case(ctx, case)
    try:
        p = pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED
        dx, _ = pf.pf_newton_step(c, vm, va, pf.make_opts(precision=p, refine_steps=2))
        idx = O.cim_unknowns(case)
        F = O.cim_mismatch(case, Y, V)[idx]
        J = O.cim_jacobian(case, Y, V)[idx][:, idx].tocsr()
        full = np.zeros(6 * case.n_node)
        full[idx] = O.solve_linear(J, F, "splu")
        ref = full.reshape(case.n_node, 6)
        assert np.max(np.abs(dx - ref)) <= tol * max(1.0, np.max(np.abs(ref)))
    finally:
        pf.pf_destroy_case(c)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_graph_matches_kernel_by_kernel(pf, ctx, prec):
    """The batch as one CUDA graph (device-driven loop) and launched kernel by
    kernel run the same kernels on the same data: identical results.  The
    graph is built once and reused by later calls with other inputs; a
    scenario that cannot converge within max_iter ends the loop on its own."""
    case = cases.case_2000bus(1)
    B = 40
    p = pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED
    c = pf.pf_create_case(ctx, case)
    try:
        for seed in (3, 4):
            pl, ql, pg = cases.scenario_loads(case, B, seed=seed)
            vm_g, va_g, inf_g = pf.pf_solve_batch(c, pl, ql, pg, pf.make_opts(precision=p))
            vm_k, va_k, inf_k = pf.pf_solve_batch(c, pl, ql, pg,
                                                  pf.make_opts(precision=p, kernel_by_kernel=1))
            assert np.all(inf_g["status"] == 0)
            assert np.array_equal(vm_g, vm_k) and np.array_equal(va_g, va_k)
            for k in ("status", "iterations", "linear_iterations", "mismatch", "max_step"):
                assert np.array_equal(inf_g[k], inf_k[k]), k
        # an iteration limit below what the scenarios need: every one stops at it
        pl, ql, pg = cases.scenario_loads(case, B, seed=5)
        _, _, inf = pf.pf_solve_batch(c, pl, ql, pg, pf.make_opts(precision=p, max_iter=2))
        assert np.all(inf["status"] == pf.PF_ERR_MAXITER) and np.all(inf["iterations"] == 2)
    finally:
        pf.pf_destroy_case(c)


def test_three_phase_batch_matches_single(pf, ctx):
    case = cases.feeder_case(500, 2)
    B = 9
    pl, ql = cases.feeder_scenario_loads(case, B, seed=3)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve_batch(c, pl, ql, None, pf.make_opts(scen_per_cta=2))
        assert np.all(info["status"] == 0)
        for b in (0, B - 1):
            ref = O.newton_cim(case.with_loads(pl[b], ql[b]))
            assert np.max(np.abs(vm[b] - np.abs(ref["V"]))) <= V_TOL
    finally:
        pf.pf_destroy_case(c)


# ----------------------------------------------------------------------------
# Newton-Krylov: GMRES(m) + ILU(0)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["14", "300zip", "2000", "10000"])
def test_newton_krylov_matches_oracle(pf, ctx, name, prec):
    case = {"14": cases.case_14bus(0),
            "300zip": _zip_case(cases.transmission_case(300, 405, 60, 2), 2),
            "2000": cases.case_2000bus(0), "10000": cases.case_10000bus(0)}[name]
    ref = O.newton_polar(case)
    c = pf.pf_create_case(ctx, case)
    try:
        p = pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED
        vm, va, info = pf.pf_solve(c, pf.make_opts(method=pf.PF_NK, precision=p))
        _check_solve(case, vm, va, info, ref)
        assert info["linear_iterations"] >= info["iterations"] > 0
        # NR and NK reach the same voltages
        vm2, va2, info2 = pf.pf_solve(c, pf.make_opts(method=pf.PF_NR, precision=p))
        assert np.max(np.abs(vm - vm2)) <= V_TOL and np.max(np.abs(va - va2)) <= A_TOL
    finally:
        pf.pf_destroy_case(c)


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_gmres_step_meets_its_residual_bound(pf, ctx, prec, rtol):
    case = _zip_case(cases.transmission_case(300, 405, 60, 2), 2)
    Y = O.ybus_single(case)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va = O.flat_start_polar(case)
        vm = vm + np.where(case.bus_type == cases.PQ, 0.01 * np.sin(np.arange(case.n_bus)), 0)
        va = va + np.where(case.bus_type != cases.SLACK, 0.02 * np.cos(np.arange(case.n_bus)), 0)
        p = pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED
        dx, _ = pf.pf_newton_step(c, vm, va, pf.make_opts(method=pf.PF_NK, precision=p,
                                                        gmres_rtol=rtol, gmres_max_iter=2000))
        F = O.mismatch_polar(case, Y, vm, va)
        J = O.jacobian_polar(case, Y, vm, va)
        got = _gpu_mis_to_oracle_order(case, dx)
        # FP32 products add rounding on top of the GMRES bound
        slack = 1.5 if prec == "fp64" else 20.0
        assert np.linalg.norm(F - J @ got) <= slack * rtol * np.linalg.norm(F)
        ref = O.solve_linear(J, F, "splu")
        assert np.max(np.abs(got - ref)) <= 1e4 * slack * rtol * np.max(np.abs(ref))
    finally:
        pf.pf_destroy_case(c)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_newton_krylov_three_phase(pf, ctx, prec):
    case = cases.feeder_case(400, 5)
    ref = O.newton_cim(case)
    c = pf.pf_create_case(ctx, case)
    try:
        p = pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED
        vm, va, info = pf.pf_solve(c, pf.make_opts(method=pf.PF_NK, precision=p))
        assert info["status"] == 0 and info["mismatch"] <= 1e-8, info
        assert np.max(np.abs(vm - np.abs(ref["V"]))) <= V_TOL
    finally:
        pf.pf_destroy_case(c)


def test_newton_krylov_batch_matches_single(pf, ctx):
    case = cases.case_2000bus(4)
    B = 12
    p_load, q_load, p_gen = cases.scenario_loads(case, B, seed=8)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve_batch(c, p_load, q_load, p_gen,
                                         pf.make_opts(method=pf.PF_NK, scen_per_cta=4))
        assert np.all(info["status"] == 0), info
        for b in (0, B - 1):
            ref = O.newton_polar(case.with_loads(p_load[b], q_load[b], p_gen[b]))
            assert np.max(np.abs(vm[b] - ref["vm"])) <= V_TOL
            assert np.max(np.abs(va[b] - ref["va"])) <= A_TOL
    finally:
        pf.pf_destroy_case(c)


# ----------------------------------------------------------------------------
# branch flows (Sec. I outputs), a post-step over solved voltages
# ----------------------------------------------------------------------------

def test_branch_flows_match_oracle_single_phase(pf, ctx):
    case = cases.case_2000bus(2)
    B = 5
    pl, ql, pg = cases.scenario_loads(case, B, seed=6)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve_batch(c, pl, ql, pg)
        assert np.all(info["status"] == 0)
        rng = np.random.default_rng(1)
        vm[1] = rng.uniform(0.9, 1.1, case.n_bus)  # an arbitrary voltage too
        va[1] = rng.uniform(-0.5, 0.5, case.n_bus)
        got = pf.pf_branch_flows(c, vm, va, case.n_branch)
        for b in range(B):
            ref = O.branch_flows(case, vm[b], va[b])
            scale = max(1.0, np.max(np.abs(ref[0])))
            for k, key in enumerate(("p_from", "q_from", "p_to", "q_to")):
                assert np.max(np.abs(got[key][b] - ref[k])) <= 1e-12 * scale, key
            assert abs(got["loss"][b, 0] - ref[4][0]) <= 1e-10 * scale
            assert abs(got["loss"][b, 1] - ref[4][1]) <= 1e-10 * scale
        # at a solution the losses are the net specified injection plus slack
        Y = O.ybus_single(case)
        V = vm[0] * np.exp(1j * va[0])
        assert abs(got["loss"][0, 0] - (V * np.conj(Y @ V)).real.sum()) < 1e-9
    finally:
        pf.pf_destroy_case(c)


def test_branch_flows_match_oracle_three_phase(pf, ctx):
    case = cases.feeder_case(400, 3)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve(c)
        assert info["status"] == 0
        got = pf.pf_branch_flows(c, vm, va, case.n_branch)
        ref = O.branch_flows(case, vm, va)
        scale = max(1.0, np.max(np.abs(ref[0])))
        for k, key in enumerate(("p_from", "q_from", "p_to", "q_to")):
            assert np.max(np.abs(got[key][0] - ref[k].reshape(-1))) <= 1e-12 * scale, key
        assert abs(got["loss"][0, 0] - ref[4][0]) <= 1e-10 * scale
    finally:
        pf.pf_destroy_case(c)


def test_newton_krylov_falls_back_to_newton_raphson(pf, ctx):
    """NK starved of inner iterations cannot converge; with nk_fallback (the
    default) the scenarios are redone with NR and match the oracle, alone and
    in a batch; without it they report the failure."""
    case = cases.case_2000bus(5)
    starve = dict(method=pf.PF_NK, gmres_max_iter=1, max_iter=8)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve(c, pf.make_opts(nk_fallback=0, **starve))
        assert info["status"] != 0 and info["fallback"] == 0
        vm, va, info = pf.pf_solve(c, pf.make_opts(**starve))
        assert info["fallback"] == 1
        _check_solve(case, vm, va, info, O.newton_polar(case))
        B = 6
        pl, ql, pg = cases.scenario_loads(case, B, seed=9)
        vm, va, inf = pf.pf_solve_batch(c, pl, ql, pg, pf.make_opts(scen_per_cta=2, **starve))
        assert np.all(inf["status"] == 0) and np.all(inf["fallback"] == 1)
        for b in (0, B - 1):
            ref = O.newton_polar(case.with_loads(pl[b], ql[b], pg[b]))
            assert np.max(np.abs(vm[b] - ref["vm"])) <= V_TOL
            assert np.max(np.abs(va[b] - ref["va"])) <= A_TOL
        # a converging NK batch is left alone
        vm, va, inf = pf.pf_solve_batch(c, pl, ql, pg, pf.make_opts(method=pf.PF_NK,
                                                                    scen_per_cta=2))
        assert np.all(inf["status"] == 0) and np.all(inf["fallback"] == 0)
    finally:
        pf.pf_destroy_case(c)


# ----------------------------------------------------------------------------
# Newton-Krylov with BiCGSTAB (the paper's Krylov method, Sec. III.B)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["300zip", "2000", "10000"])
def test_newton_krylov_bicgstab_matches_oracle(pf, ctx, name, prec):
    case = {"300zip": _zip_case(cases.transmission_case(300, 405, 60, 2), 2),
            "2000": cases.case_2000bus(0), "10000": cases.case_10000bus(0)}[name]
    ref = O.newton_polar(case)
    c = pf.pf_create_case(ctx, case)
    try:
        p = pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED
        vm, va, info = pf.pf_solve(c, pf.make_opts(method=pf.PF_NK, krylov=1, precision=p,
                                                   nk_fallback=0, gmres_max_iter=2000))
        _check_solve(case, vm, va, info, ref)
        assert info["linear_iterations"] > 0 and info["fallback"] == 0
    finally:
        pf.pf_destroy_case(c)


@pytest.mark.parametrize("prec,rtol,slack", [("fp64", 1e-10, 10.0), ("mixed", 1e-5, 50.0)])
def test_bicgstab_step_meets_its_residual_bound(pf, ctx, prec, rtol, slack):
    case = _zip_case(cases.transmission_case(300, 405, 60, 2), 2)
    Y = O.ybus_single(case)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va = O.flat_start_polar(case)
        vm = vm + np.where(case.bus_type == cases.PQ, 0.01 * np.sin(np.arange(case.n_bus)), 0)
        va = va + np.where(case.bus_type != cases.SLACK, 0.02 * np.cos(np.arange(case.n_bus)), 0)
        p = pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED
        dx, _ = pf.pf_newton_step(c, vm, va, pf.make_opts(method=pf.PF_NK, krylov=1,
                                                        precision=p, gmres_rtol=rtol,
                                                        gmres_max_iter=2000))
        F = O.mismatch_polar(case, Y, vm, va)
        J = O.jacobian_polar(case, Y, vm, va)
        got = _gpu_mis_to_oracle_order(case, dx)
        # the recursively updated BiCGSTAB residual drifts from the true one
        # by rounding; the bound allows for that
        assert np.linalg.norm(F - J @ got) <= slack * rtol * np.linalg.norm(F)
    finally:
        pf.pf_destroy_case(c)


def test_newton_krylov_bicgstab_batch_matches_oracle(pf, ctx):
    case = cases.case_2000bus(4)
    B = 8
    p_load, q_load, p_gen = cases.scenario_loads(case, B, seed=12)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve_batch(c, p_load, q_load, p_gen,
                                         pf.make_opts(method=pf.PF_NK, krylov=1, scen_per_cta=4,
                                                      nk_fallback=0, gmres_max_iter=2000))
        assert np.all(info["status"] == 0), info
        for b in (0, B - 1):
            ref = O.newton_polar(case.with_loads(p_load[b], q_load[b], p_gen[b]))
            assert np.max(np.abs(vm[b] - ref["vm"])) <= V_TOL
            assert np.max(np.abs(va[b] - ref["va"])) <= A_TOL
    finally:
        pf.pf_destroy_case(c)


def test_bicgstab_needs_its_work_vectors(pf, ctx):
    case = cases.case_14bus(0)
    c = pf.pf_create_case(ctx, case)
    try:
        with pytest.raises(pf.PfError):
            pf.pf_solve(c, pf.make_opts(method=pf.PF_NK, krylov=1, gmres_restart=4))
    finally:
        pf.pf_destroy_case(c)


# ----------------------------------------------------------------------------
# three phase with PV nodes (dVr = -(Vi/Vr) dVi substitution on the GPU,
# augmented system in the oracle)
# ----------------------------------------------------------------------------

def _check_cim_solve(case, vm, va, info, ref):
    assert info["status"] == 0, info
    assert info["mismatch"] <= 1e-8
    Vref = ref["V"]
    assert np.max(np.abs(vm - np.abs(Vref))) <= V_TOL
    present = np.abs(Vref) > 0
    dang = np.angle(np.exp(1j * (va - np.angle(Vref))))
    assert np.max(np.abs(dang[present])) <= A_TOL


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_three_phase_pv_solve_matches_oracle(pf, ctx, prec):
    case = cases.with_pv_nodes(cases.feeder_case(600, 4), 8, 3)
    ref = O.newton_cim(case)
    assert ref["converged"]
    c = pf.pf_create_case(ctx, case)
    try:
        p = pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED
        vm, va, info = pf.pf_solve(c, pf.make_opts(precision=p))
        _check_cim_solve(case, vm, va, info, ref)
        pv = O.cim_pv_slots(case)
        assert np.max(np.abs(vm[pv] - np.repeat(case.v_set, 3)[pv])) <= 1e-12
        # Newton-Krylov on the same system
        vm, va, info = pf.pf_solve(c, pf.make_opts(method=pf.PF_NK, precision=p, nk_fallback=0,
                                                   gmres_max_iter=2000))
        _check_cim_solve(case, vm, va, info, ref)
    finally:
        pf.pf_destroy_case(c)


def test_three_phase_pv_batch_matches_oracle(pf, ctx):
    case = cases.with_pv_nodes(cases.feeder_case(500, 6), 6, 1)
    B = 6
    pl, ql = cases.feeder_scenario_loads(case, B, seed=5, sigma=0.1)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve_batch(c, pl, ql, None, pf.make_opts(scen_per_cta=2))
        assert np.all(info["status"] == 0), info
        for b in (0, B - 1):
            ref = O.newton_cim(case.with_loads(pl[b], ql[b]))
            _check_cim_solve(case, vm[b], va[b], info[b], ref)
    finally:
        pf.pf_destroy_case(c)


def test_three_phase_pv_two_node_closed_form(pf, ctx):
    """A PV node behind a lossless line from the balanced source: each phase
    is the two-bus PV problem (delta2 = asin(P x / (V1 V2)))."""
    import dataclasses as dc

    pg, x, vset = 0.3, 0.1, 1.02
    base = np.zeros((3, 3), dtype=np.complex128)
    np.fill_diagonal(base, 1j * x)
    case = cases.ThreePhaseCase(
        n_node=2, source=0, phases=np.array([7, 7], np.uint8), p_load=np.zeros((2, 3)),
        q_load=np.zeros((2, 3)), zip=np.tile([1.0, 0.0, 0.0], (2, 1)),
        br_from=np.array([0], np.int32), br_to=np.array([1], np.int32),
        br_phases=np.array([7], np.uint8), br_z=base[None])
    case = dc.replace(case, node_type=np.array([cases.PQ, cases.PV], np.int32),
                      v_set=np.array([1.0, vset]), p_gen=np.array([[0, 0, 0], [pg, pg, pg]], float))
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve(c, pf.make_opts(precision=pf.PF_FP64))
        assert info["status"] == 0
        d = np.arcsin(pg * x / vset)
        rot = np.angle(np.exp(-2j * np.pi / 3 * np.arange(3)))
        assert np.max(np.abs(vm[3:] - vset)) <= 1e-12
        assert np.max(np.abs(np.angle(np.exp(1j * (va[3:] - rot - d))))) <= 1e-9
    finally:
        pf.pf_destroy_case(c)


# ----------------------------------------------------------------------------
# reactive limits of PV buses (rounds of PV -> PQ switching)
# ----------------------------------------------------------------------------

def _gpu_switched(case, vm):
    """PV buses the GPU switched: a PV bus keeps |V| = v_set exactly (its |V|
    is no unknown), a switched one does not."""
    pv = case.bus_type == cases.PV
    return pv & (vm != case.v_set)


def _check_qlim(case, vm, va, info, ref):
    assert info["status"] == 0, info
    assert info["mismatch"] <= 1e-8
    assert np.array_equal(_gpu_switched(case, vm), ref["switched"])
    assert info["q_switched"] == int(ref["switched"].sum())
    assert info["q_rounds"] == ref["rounds"]
    assert np.max(np.abs(vm - ref["vm"])) <= V_TOL
    assert np.max(np.abs(va - ref["va"])) <= A_TOL


@pytest.mark.parametrize("method", ["nr", "nk"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,seed", [("300", 1), ("2000", 2), ("10000", 1)])
def test_q_limits_single_matches_oracle(pf, ctx, name, seed, prec, method):
    base = {"300": cases.transmission_case(300, 405, 60, 2), "2000": cases.case_2000bus(0),
            "10000": cases.case_10000bus(0)}[name]
    case = cases.with_q_limits(base, seed)
    ref = O.newton_polar_qlim(case)
    assert ref["converged"] and ref["switched"].any()
    c = pf.pf_create_case(ctx, case)
    try:
        p = pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED
        m = pf.PF_NR if method == "nr" else pf.PF_NK
        vm, va, info = pf.pf_solve(c, pf.make_opts(precision=p, method=m, q_limits=1,
                                                   nk_fallback=0))
        _check_qlim(case, vm, va, info, ref)
        assert info["iterations"] >= ref["rounds"] - 1
    finally:
        pf.pf_destroy_case(c)


def test_q_limits_batch_matches_oracle(pf, ctx):
    base = cases.case_2000bus(1)
    case = cases.with_q_limits(base, 3)
    B = 40
    p_load, q_load, p_gen = cases.scenario_loads(case, B, seed=21)
    c = pf.pf_create_case(ctx, case)
    try:
        for opts in (pf.make_opts(q_limits=1), pf.make_opts(q_limits=1, kernel_by_kernel=1),
                     pf.make_opts(q_limits=1, method=pf.PF_NK, nk_fallback=0)):
            vm, va, info = pf.pf_solve_batch(c, p_load, q_load, p_gen, opts)
            counts = set()
            for b in (0, 7, 19, B - 1):
                ref = O.newton_polar_qlim(case.with_loads(p_load[b], q_load[b], p_gen[b]))
                assert ref["converged"]
                _check_qlim(case, vm[b], va[b], info[b], ref)
                counts.add(int(info[b]["q_switched"]))
            assert np.all(info["status"] == 0)
            # the rounds are per scenario: a scenario with nothing left to
            # switch stops at once
            assert len(counts) > 1 or max(counts) > 0
    finally:
        pf.pf_destroy_case(c)


def test_q_limits_two_bus_closed_form(pf, ctx):
    """Two-bus PV past q_max becomes PQ at q_max: the PQ closed form."""
    import dataclasses as dc
    import math

    pg, x, vset, pl, ql, qmax = 0.3, 0.1, 1.02, 0.1, 0.05, 0.15
    case = cases.two_bus_case(pg, 0.0, 0.0, x, pv=True, v2=vset)
    case = dc.replace(case, p_load=np.array([0.0, pl]), q_load=np.array([0.0, ql]),
                      q_min=np.array([-9.0, -1.0]), q_max=np.array([9.0, qmax]))
    # PQ closed form: u = |V2|^2 solves u^2 - (2 Q x + 1) u + (P^2 + Q^2) x^2 = 0
    # for the net injection P + jQ through a lossless line x (larger root)
    P, Q = pg - pl, qmax - ql
    u = ((2 * Q * x + 1) + math.sqrt((2 * Q * x + 1) ** 2 - 4 * (P * P + Q * Q) * x * x)) / 2
    v2 = math.sqrt(u)
    d2 = math.asin(P * x / v2)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve(c, pf.make_opts(precision=pf.PF_FP64, q_limits=1, tol=1e-12))
        assert info["status"] == 0 and info["q_switched"] == 1 and info["q_rounds"] == 2
        assert abs(vm[1] - v2) < 1e-10 and abs(va[1] - d2) < 1e-10
        vm0, _, info0 = pf.pf_solve(c, pf.make_opts(precision=pf.PF_FP64, tol=1e-12))
        assert info0["q_switched"] == 0 and vm0[1] == vset
    finally:
        pf.pf_destroy_case(c)


def test_q_limits_wide_limits_change_nothing(pf, ctx):
    base = cases.case_2000bus(0)
    case = cases.with_q_limits(base, 1, q_range=(50.0, 60.0))
    B = 16
    p_load, q_load, p_gen = cases.scenario_loads(case, B, seed=4)
    c = pf.pf_create_case(ctx, case)
    try:
        vm0, va0, i0 = pf.pf_solve_batch(c, p_load, q_load, p_gen)
        vm1, va1, i1 = pf.pf_solve_batch(c, p_load, q_load, p_gen, pf.make_opts(q_limits=1))
        assert np.all(i1["q_switched"] == 0) and np.all(i1["q_rounds"] == 1)
        assert np.array_equal(vm0, vm1) and np.array_equal(va0, va1)
        assert np.array_equal(i0["iterations"], i1["iterations"])
    finally:
        pf.pf_destroy_case(c)


# ----------------------------------------------------------------------------
# FP64 refinement on demand (mixed Newton-Raphson)
# ----------------------------------------------------------------------------

def test_refinement_on_demand(pf, ctx):
    """refine_stall = 0 refines every step below refine_below; a tiny
    refine_stall refines the same steps (any reduction counts as a stall);
    the default refines only steps that cut the mismatch by less than 10x.
    All reach the oracle's solution."""
    case = cases.case_2000bus(3)
    ref = O.newton_polar(case)
    B = 24
    p_load, q_load, p_gen = cases.scenario_loads(case, B, seed=31)
    refs = [O.newton_polar(case.with_loads(p_load[b], q_load[b], p_gen[b])) for b in (0, B - 1)]
    c = pf.pf_create_case(ctx, case)
    try:
        res = {}
        for name, rs in (("always", 0.0), ("tiny", 1e-12), ("default", None)):
            o = pf.make_opts() if rs is None else pf.make_opts(refine_stall=rs)
            vm, va, info = pf.pf_solve(c, o)
            _check_solve(case, vm, va, info, ref)
            vmb, vab, ib = pf.pf_solve_batch(c, p_load, q_load, p_gen, o)
            assert np.all(ib["status"] == 0)
            for k, b in enumerate((0, B - 1)):
                _check_solve(case, vmb[b], vab[b], ib[b], refs[k])
            res[name] = (info, ib)
        # refinement passes are the linear iterations beyond one per step
        extra = lambda i: np.asarray(i["linear_iterations"]) - np.asarray(i["iterations"])
        assert np.all(extra(res["always"][1]) > 0)
        assert np.array_equal(extra(res["always"][1]), extra(res["tiny"][1]))
        assert np.all(extra(res["default"][1]) <= extra(res["always"][1]))
        assert pf.make_opts().refine_stall == 0.1
    finally:
        pf.pf_destroy_case(c)


# ----------------------------------------------------------------------------
# reactive limits of three-phase PV slots
# ----------------------------------------------------------------------------

def _check_cim_qlim(case, vm, va, info, ref):
    _check_cim_solve(case, vm, va, info, ref)
    pv = O.cim_pv_slots(case)
    vset = np.repeat(case.v_set, 3)
    held = pv & (np.abs(vm - vset) > 1e-9)
    assert np.array_equal(held, ref["switched"])
    assert info["q_switched"] == int(ref["switched"].sum())
    assert info["q_rounds"] == ref["rounds"]


@pytest.mark.parametrize("method", ["nr", "nk"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_three_phase_q_limits_match_oracle(pf, ctx, prec, method):
    base = cases.with_pv_nodes(cases.feeder_case(600, 4), 8, 3)
    case = cases.with_phase_q_limits(base, 1)
    ref = O.newton_cim_qlim(case)
    assert ref["converged"] and ref["switched"].any()
    c = pf.pf_create_case(ctx, case)
    try:
        p = pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED
        m = pf.PF_NR if method == "nr" else pf.PF_NK
        vm, va, info = pf.pf_solve(c, pf.make_opts(precision=p, method=m, q_limits=1,
                                                   nk_fallback=0, gmres_max_iter=2000))
        _check_cim_qlim(case, vm, va, info, ref)
    finally:
        pf.pf_destroy_case(c)


def test_three_phase_q_limits_batch_matches_oracle(pf, ctx):
    base = cases.with_pv_nodes(cases.feeder_case(500, 6), 8, 1)
    case = cases.with_phase_q_limits(base, 2)
    B = 8
    pl, ql = cases.feeder_scenario_loads(case, B, seed=5, sigma=0.1)
    c = pf.pf_create_case(ctx, case)
    try:
        for opts in (pf.make_opts(q_limits=1), pf.make_opts(q_limits=1, kernel_by_kernel=1)):
            vm, va, info = pf.pf_solve_batch(c, pl, ql, None, opts)
            assert np.all(info["status"] == 0), info
            for b in (0, 3, B - 1):
                ref = O.newton_cim_qlim(case.with_loads(pl[b], ql[b]))
                _check_cim_qlim(case, vm[b], va[b], info[b], ref)
    finally:
        pf.pf_destroy_case(c)


def test_three_phase_q_limit_two_node_closed_form(pf, ctx):
    """The lossless two-node line with q_max below the injection that holds
    v_set: every phase is held at q_max, the two-bus PQ closed form."""
    import dataclasses as dc
    import math

    pg, x, vset, qmax = 0.3, 0.1, 1.02, 0.1
    base = np.zeros((3, 3), dtype=np.complex128)
    np.fill_diagonal(base, 1j * x)
    case = cases.ThreePhaseCase(
        n_node=2, source=0, phases=np.array([7, 7], np.uint8), p_load=np.zeros((2, 3)),
        q_load=np.zeros((2, 3)), zip=np.tile([1.0, 0.0, 0.0], (2, 1)),
        br_from=np.array([0], np.int32), br_to=np.array([1], np.int32),
        br_phases=np.array([7], np.uint8), br_z=base[None])
    case = dc.replace(case, node_type=np.array([cases.PQ, cases.PV], np.int32),
                      v_set=np.array([1.0, vset]), p_gen=np.array([[0, 0, 0], [pg, pg, pg]], float),
                      q_min=np.full((2, 3), -1.0), q_max=np.full((2, 3), qmax))
    P, Q = pg, qmax
    u = ((2 * Q * x + 1) + math.sqrt((2 * Q * x + 1) ** 2 - 4 * (P * P + Q * Q) * x * x)) / 2
    v2 = math.sqrt(u)
    d2 = math.asin(P * x / v2)
    rot = np.angle(np.exp(-2j * np.pi / 3 * np.arange(3)))
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve(c, pf.make_opts(precision=pf.PF_FP64, q_limits=1, tol=1e-12))
        assert info["status"] == 0 and info["q_switched"] == 3 and info["q_rounds"] == 2
        assert np.max(np.abs(vm[3:] - v2)) <= 1e-10
        assert np.max(np.abs(np.angle(np.exp(1j * (va[3:] - rot - d2))))) <= 1e-10
    finally:
        pf.pf_destroy_case(c)


def test_heavy_loading_mixed_precision(pf, ctx):
    """The 10,000-bus grid loaded 5.3 times as heavily as the benchmark grid
    (DC angle target 1.6 rad: lowest |V| about 0.36 pu, near the nose of the
    loading curve; load spread lognormal(0, 0.1)).  Mixed precision (FP32
    factors) needs exactly as many Newton steps as FP64 and matches the oracle;
    its steps still cut the mismatch by more than tenfold, so the on-demand
    FP64 refinement is not taken, while refinement of every step below
    refine_below (refine_stall = 0) is taken and also matches the oracle."""
    case = cases.transmission_case(10_000, 13_500, 2_000, 0, max_angle=1.6)
    B = 64
    pl, ql, pg = cases.scenario_loads(case, B, seed=31, sigma=0.1)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = pf.pf_solve_batch(c, pl, ql, pg)
        _, _, i64 = pf.pf_solve_batch(c, pl, ql, pg, pf.make_opts(precision=pf.PF_FP64))
        vr, ar, ir = pf.pf_solve_batch(c, pl, ql, pg, pf.make_opts(refine_stall=0.0))
        for inf in (info, i64, ir):
            assert np.all(inf["status"] == 0) and np.all(inf["mismatch"] <= 1e-8)
        assert np.array_equal(info["iterations"], i64["iterations"])
        assert np.array_equal(info["linear_iterations"], info["iterations"])
        assert np.all(ir["linear_iterations"] > ir["iterations"])
        for b in (0, B // 2, B - 1):
            ref = O.newton_polar(case.with_loads(pl[b], ql[b], pg[b]))
            assert ref["converged"]
            for v, a in ((vm, va), (vr, ar)):
                assert np.max(np.abs(v[b] - ref["vm"])) <= V_TOL
                assert np.max(np.abs(a[b] - ref["va"])) <= A_TOL
    finally:
        pf.pf_destroy_case(c)


# ----------------------------------------------------------------------------
# the benchmark's own workload at full size
# ----------------------------------------------------------------------------

def test_full_size_batch_in_the_benchmark_launch_shape(pf, ctx):
    """The 10,000-bus grid x 9,728 scenarios, autotuned as the benchmark runs
    it (mixed NR, graph): every scenario converges with its PV magnitudes and
    the slack untouched; sampled scenarios match the oracle; and a random
    scenario's power mismatch, recomputed by the oracle from the GPU's
    voltages, is below the tolerance."""
    case = cases.case_10000bus(0)
    B = 9728
    pl, ql, pg = cases.scenario_loads(case, B, seed=21, sigma=0.2)
    c = pf.pf_create_case(ctx, case)
    try:
        pf.pf_autotune(c, B, pf.make_opts())
        vm, va, info = pf.pf_solve_batch(c, pl, ql, pg)
        assert np.all(info["status"] == 0)
        assert np.all(info["mismatch"] <= 1e-8)
        pv = case.bus_type == cases.PV
        slack = case.bus_type == cases.SLACK
        assert np.all(vm[:, pv] == case.v_set[pv]) and np.all(vm[:, slack] == case.v_set[slack])
        assert np.all(va[:, slack] == 0.0)
        Y = O.ybus_single(case)
        rng = np.random.default_rng(2)
        for b in [0, B - 1] + list(rng.integers(1, B - 1, 2)):
            sc = case.with_loads(pl[b], ql[b], pg[b])
            ref = O.newton_polar(sc)
            assert np.max(np.abs(vm[b] - ref["vm"])) <= V_TOL
            assert np.max(np.abs(va[b] - ref["va"])) <= A_TOL
            F = O.mismatch_polar(sc, Y, vm[b], va[b])
            assert np.max(np.abs(F)) <= 1e-8
    finally:
        pf.pf_destroy_case(c)

