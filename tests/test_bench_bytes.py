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
