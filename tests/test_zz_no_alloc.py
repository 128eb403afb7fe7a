"""pf_solve_noalloc: the Newton-Raphson solve for callers that cannot
allocate device memory while running (fixed-latency control loops, host
applications that own the GPU's memory).  Its workspace is a fixed array
compiled into the library; here its results are checked against the
allocating device entry point, on two calls in a row: both run the same
kernel in the same launch shape on the same inputs, so the results must be
identical bit for bit (stale contents of the shared array would show).
Collected last on purpose, and independent of the other test files."""
import numpy as np
import pytest

from paper_1711_10579_gb300 import cases

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1711_10579_gb300 import pf

    ctx = pf.pf_ctx_create(0)
    yield pf, torch, ctx
    pf.pf_ctx_destroy(ctx)


def _buffers(pf, torch, n, slots):
    dev = torch.device("cuda:0")
    vm = torch.zeros(slots, dtype=torch.float64, device=dev)
    va = torch.zeros_like(vm)
    info = torch.zeros(pf.INFO_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    return vm, va, info


def _info(pf, t):
    return np.frombuffer(t.cpu().numpy().tobytes(), dtype=pf.INFO_DTYPE)[0]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["mesh2000", "mesh10000", "feeder2000"])
def test_noalloc_matches_the_allocating_entry_point(env, name, prec):
    pf, torch, ctx = env
    case = {"mesh2000": cases.case_2000bus(1), "mesh10000": cases.case_10000bus(2),
            "feeder2000": cases.feeder_case(2000, 4)}[name]
    c = pf.pf_create_case(ctx, case)
    try:
        opts = pf.make_opts(precision=pf.PF_FP64 if prec == "fp64" else pf.PF_MIXED)
        dev = torch.device("cuda:0")
        stream = torch.cuda.current_stream().cuda_stream
        if isinstance(case, cases.SinglePhaseCase):
            pl, ql, pg = cases.scenario_loads(case, 2, seed=17, sigma=0.1)
        else:
            pl, ql = cases.feeder_scenario_loads(case, 2, seed=17, sigma=0.1)
            pl, ql, pg = pl.reshape(2, -1), ql.reshape(2, -1), None
        for k in range(2):  # two calls in a row share the scratch array
            d = [None if a is None else torch.tensor(a[k], device=dev) for a in (pl, ql, pg)]
            vm0, va0, in0 = _buffers(pf, torch, case, c.slots)
            pf.pf_solve_batch_device(c, 1, d[0], d[1], d[2], opts, vm0, va0, in0, stream)
            vm1, va1, in1 = _buffers(pf, torch, case, c.slots)
            pf.pf_solve_noalloc(c, opts, d[0], d[1], d[2], vm1, va1, in1, stream)
            torch.cuda.synchronize()
            i0, i1 = _info(pf, in0), _info(pf, in1)
            assert i0["status"] == 0 and i1["status"] == 0, (i0, i1)
            assert i1["mismatch"] <= 1e-8
            assert torch.equal(vm1, vm0) and torch.equal(va1, va0)
            for key in ("iterations", "linear_iterations", "mismatch", "max_step"):
                assert i0[key] == i1[key], key
    finally:
        pf.pf_destroy_case(c)


def test_noalloc_call_allocates_nothing(env):
    """After a first call, another call leaves the device's free memory
    unchanged (every buffer of the test exists before the measurement)."""
    pf, torch, ctx = env
    case = cases.case_2000bus(3)
    c = pf.pf_create_case(ctx, case)
    try:
        dev = torch.device("cuda:0")
        stream = torch.cuda.current_stream().cuda_stream
        pl, ql, pg = cases.scenario_loads(case, 1, seed=5, sigma=0.1)
        d = [torch.tensor(a[0], device=dev) for a in (pl, ql, pg)]
        vm, va, info = _buffers(pf, torch, case, c.slots)
        pf.pf_solve_noalloc(c, pf.make_opts(), d[0], d[1], d[2], vm, va, info, stream)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        pf.pf_solve_noalloc(c, pf.make_opts(), d[0], d[1], d[2], vm, va, info, stream)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert _info(pf, info)["status"] == 0
    finally:
        pf.pf_destroy_case(c)


def test_noalloc_rejects_a_case_beyond_its_scratch(env):
    pf, torch, ctx = env
    # a 200,000-bus radial line needs more than the fixed array holds
    n = 200_000
    line = cases.SinglePhaseCase(
        n_bus=n, bus_type=np.r_[0, np.full(n - 1, 2)].astype(np.int32), v_set=np.ones(n),
        p_gen=np.zeros(n), q_gen=np.zeros(n), p_load=np.full(n, 1e-6), q_load=np.zeros(n),
        zip=np.tile([1.0, 0.0, 0.0], (n, 1)), br_from=np.arange(n - 1, dtype=np.int32),
        br_to=np.arange(1, n, dtype=np.int32), br_r=np.full(n - 1, 1e-4),
        br_x=np.full(n - 1, 1e-3), br_b=np.zeros(n - 1))
    c = pf.pf_create_case(ctx, line)
    try:
        vm, va, info = _buffers(pf, torch, line, c.slots)
        with pytest.raises(pf.PfError) as e:
            pf.pf_solve_noalloc(c, pf.make_opts(), None, None, None, vm, va, info,
                                torch.cuda.current_stream().cuda_stream)
        assert e.value.code == pf.PF_ERR_INVALID and "scratch" in str(e.value)
    finally:
        pf.pf_destroy_case(c)


def test_noalloc_refuses_reactive_limits(env):
    pf, torch, ctx = env
    case = cases.with_q_limits(cases.case_14bus(0), 1)
    c = pf.pf_create_case(ctx, case)
    try:
        vm, va, info = _buffers(pf, torch, case, c.slots)
        with pytest.raises(pf.PfError) as e:
            pf.pf_solve_noalloc(c, pf.make_opts(q_limits=1), None, None, None, vm, va, info,
                                torch.cuda.current_stream().cuda_stream)
        assert e.value.code == pf.PF_ERR_UNSUPPORTED and "reactive" in str(e.value)
    finally:
        pf.pf_destroy_case(c)
