"""The benchmark's algorithmic byte counts, pinned on the CPU: the scalar
non-zeros of the polar Jacobian it counts from the branch list and bus types
equal those of the oracle's Jacobian of Eq. 10 at a generic voltage."""
import numpy as np
import pytest

import bench
from oracle import pf_oracle as O
from paper_1711_10579_gb300 import cases


@pytest.mark.parametrize("case", [cases.case_14bus(0), cases.transmission_case(300, 405, 60, 2),
                                  cases.case_2000bus(1)], ids=["14", "300", "2000"])
def test_jacobian_nonzeros_match_the_oracle(case):
    rng = np.random.default_rng(3)
    vm = 1.0 + 0.05 * rng.standard_normal(case.n_bus)
    va = 0.1 * rng.standard_normal(case.n_bus)
    J = O.jacobian_polar(case, O.ybus_single(case), vm, va).tocsr()
    J.eliminate_zeros()
    assert bench.jacobian_nnz(case) == J.nnz


def test_scope_bytes_per_unit():
    """The per-unit bytes follow the counts they are built from."""
    case = cases.case_14bus(0)
    st = {"n_bus": 14, "nnz_y": 54, "n_unknowns": 22, "nnz_lu": 60}
    b = bench.scope_bytes(case, st, B=1)
    assert b["k_factor"] == 60 * 4 * 2 * 4
    assert b["k_solve"] == 60 * 4 * 4 + 3 * 22 * 4
    assert b["k_update"] == 14 * 40
    assert b["k_mismatch"] == 54 * 20 + 4 * 15 + 14 * 48 + bench.jacobian_nnz(case) * 4


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores, one
    bounded sample per step) prints one JSON line with the keys the driver
    reads, on the workload and metric of the GPU arm."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "solves/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] >= 3
    assert f"x {bench.B_MAIN} load scenarios" in line["config"]["workload"]
    for k in ("cpu_baseline", "e2e"):
        assert k in line
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
