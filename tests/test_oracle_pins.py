"""Pins of the FP64 oracle to facts other than itself.

Each test ties one part of the oracle to a closed form, a physical identity,
a brute-force or library computation, or an invariant, chosen so that a
dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them.  CPU only.
"""
import math

import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

from oracle import pf_oracle as O
from paper_1711_10579_gb300 import cases


# -----------------------------------------------------------------------------
# single phase
# -----------------------------------------------------------------------------

def two_bus_pq_closed_form(P, Q, r, x, v1=1.0):
    """|V2| and angle of a load P + jQ fed through z = r + jx from v1 at 0.

    From v1 = V2 + z conj(S / V2): with u = |V2|^2, a = rP + xQ, c = xP - rQ,
    u^2 + (2a - v1^2) u + (r^2 + x^2)(P^2 + Q^2) = 0; the operable root is the
    larger one, and delta2 = -atan2(c, u + a).
    """
    a = r * P + x * Q
    c = x * P - r * Q
    disc = (v1 * v1 - 2 * a) ** 2 - 4 * (r * r + x * x) * (P * P + Q * Q)
    assert disc > 0, "load beyond the nose of the PV curve"
    u = ((v1 * v1 - 2 * a) + math.sqrt(disc)) / 2
    return math.sqrt(u), -math.atan2(c, u + a)


@pytest.mark.parametrize("P,Q,r,x", [
    (0.5, 0.2, 0.01, 0.1), (1.0, 0.3, 0.02, 0.2), (0.05, -0.3, 0.005, 0.04),
    (1.5, 0.0, 0.05, 0.15)])
@pytest.mark.parametrize("linear", ["dense", "splu", "gmres"])
def test_two_bus_pq_closed_form(P, Q, r, x, linear):
    case = cases.two_bus_case(P, Q, r, x)
    res = O.newton_polar(case, tol=1e-12, linear=linear)
    assert res["converged"]
    vm2, va2 = two_bus_pq_closed_form(P, Q, r, x)
    assert abs(res["vm"][1] - vm2) < 1e-10
    assert abs(res["va"][1] - va2) < 1e-10
    assert res["vm"][0] == 1.0 and res["va"][0] == 0.0


@pytest.mark.parametrize("P,x,v2", [(0.8, 0.2, 1.02), (-0.5, 0.1, 0.98), (1.5, 0.3, 1.05)])
def test_two_bus_lossless_pv_closed_form(P, x, v2):
    case = cases.two_bus_case(P, 0.0, 0.0, x, pv=True, v2=v2)
    res = O.newton_polar(case, tol=1e-12)
    assert res["converged"]
    # lossless line: P = V1 V2 sin(delta2 - delta1) / x
    assert abs(res["va"][1] - math.asin(P * x / (1.0 * v2))) < 1e-11
    assert res["vm"][1] == v2


def _two_bus_pv_with_load(pg, x, vset, pl, ql, qmin, qmax):
    import dataclasses as dc

    case = cases.two_bus_case(pg, 0.0, 0.0, x, pv=True, v2=vset)
    return dc.replace(case, p_load=np.array([0.0, pl]), q_load=np.array([0.0, ql]),
                      q_min=np.array([-9.0, qmin]), q_max=np.array([9.0, qmax]))


@pytest.mark.parametrize("vset,qmin,qmax,side", [(1.02, -1.0, 0.15, "max"),
                                                 (0.98, -0.1, 1.0, "min"),
                                                 (1.02, -1.0, 1.0, None)])
def test_two_bus_pv_reactive_limit_closed_form(vset, qmin, qmax, side):
    """A generator with a local load behind a lossless line: held at v_set
    its reactive output is (v^2 - v cos delta)/x + q_load with
    v sin delta = (p_gen - p_load) x; past a limit the bus is PQ with net
    injection (p_gen - p_load) + j (limit - q_load), the PQ closed form."""
    pg, x, pl, ql = 0.3, 0.1, 0.1, 0.05
    case = _two_bus_pv_with_load(pg, x, vset, pl, ql, qmin, qmax)
    res = O.newton_polar_qlim(case, tol=1e-12)
    assert res["converged"]
    d = math.asin((pg - pl) * x / vset)
    q_free = (vset * vset - vset * math.cos(d)) / x + ql
    if side is None:
        assert not res["switched"].any() and res["rounds"] == 1
        assert abs(res["qg"][1] - q_free) < 1e-10
        assert abs(res["va"][1] - d) < 1e-11 and res["vm"][1] == vset
        return
    lim = qmax if side == "max" else qmin
    assert (q_free > qmax) if side == "max" else (q_free < qmin)
    assert res["switched"][1] and res["rounds"] == 2
    vm2, va2 = two_bus_pq_closed_form(-(pg - pl), -(lim - ql), 0.0, x)
    assert abs(res["vm"][1] - vm2) < 1e-10
    assert abs(res["va"][1] - va2) < 1e-10
    assert abs(res["qg"][1] - lim) < 1e-10


@pytest.mark.parametrize("zip_frac", [(0.2, 0.3, 0.5), (0.0, 0.0, 1.0), (0.0, 1.0, 0.0)])
def test_generator_q_with_zip_load_closed_form(zip_frac):
    """Two-bus PV with a ZIP load at the generator's bus: at |V| = v_set the
    load is (p, q) x (zp + zi v + zz v^2), so the generator's reactive output
    is (v^2 - v cos delta)/x + q (zp + zi v + zz v^2) with
    v sin delta = (p_gen - p shape) x."""
    import dataclasses as dc

    pg, x, v, pl, ql = 0.3, 0.1, 1.04, 0.1, 0.05
    case = _two_bus_pv_with_load(pg, x, v, pl, ql, -9.0, 9.0)
    case = dc.replace(case, zip=np.array([[1.0, 0.0, 0.0], list(zip_frac)]))
    res = O.newton_polar_qlim(case, tol=1e-12)
    shape = zip_frac[0] + zip_frac[1] * v + zip_frac[2] * v * v
    d = math.asin((pg - pl * shape) * x / v)
    assert abs(res["va"][1] - d) < 1e-11
    assert abs(res["qg"][1] - ((v * v - v * math.cos(d)) / x + ql * shape)) < 1e-10


@pytest.mark.parametrize("name,seed", [("300", 1), ("2000", 2)])
def test_reactive_limits_hold_at_the_solution(name, seed):
    """After the rounds: the mismatch of the switched system is below tol,
    every remaining PV bus is inside its limits, every switched bus was PV
    and sits exactly at the limit it crossed with |V| off its set point;
    wide limits give the plain solve."""
    base = {"300": cases.transmission_case(300, 405, 60, 2), "2000": cases.case_2000bus(0)}[name]
    case = cases.with_q_limits(base, seed)
    res = O.newton_polar_qlim(case)
    assert res["converged"] and res["switched"].any()
    Y = O.ybus_single(case)
    sw = res["switched"]
    assert np.all(case.bus_type[sw] == cases.PV)
    assert np.all(res["case"].bus_type[sw] == cases.PQ)
    F = O.mismatch_polar(res["case"], Y, res["vm"], res["va"])
    assert np.max(np.abs(F)) <= 1e-8
    qg = O.generator_q(case, Y, res["vm"], res["va"])
    at = np.where(qg[sw] > 0, case.q_max[sw], case.q_min[sw])
    assert np.max(np.abs(qg[sw] - at)) <= 1e-8
    assert np.min(np.abs(res["vm"][sw] - case.v_set[sw])) > 1e-6
    pv = res["case"].bus_type == cases.PV
    assert np.all(qg[pv] <= case.q_max[pv] + 1e-9) and np.all(qg[pv] >= case.q_min[pv] - 1e-9)
    wide = cases.with_q_limits(base, seed, q_range=(50.0, 60.0))
    r2 = O.newton_polar_qlim(wide)
    r0 = O.newton_polar(base)
    assert r2["rounds"] == 1 and not r2["switched"].any()
    assert np.array_equal(r2["vm"], r0["vm"]) and np.array_equal(r2["va"], r0["va"])


def _random_voltage(n, rng):
    return rng.uniform(0.9, 1.1, n), rng.uniform(-0.3, 0.3, n)


def test_power_balance_identity_single_phase():
    """Tellegen: total injection = series I^2 z losses - charging Q, any V."""
    rng = np.random.default_rng(3)
    case = cases.case_14bus(1)
    Y = O.ybus_single(case)
    for _ in range(5):
        vm, va = _random_voltage(case.n_bus, rng)
        P, Q = O.power_polar(Y, vm, va)
        V = vm * np.exp(1j * va)
        f, t = case.br_from, case.br_to
        i_series = (V[f] - V[t]) / (case.br_r + 1j * case.br_x)
        loss_p = np.sum(case.br_r * np.abs(i_series) ** 2)
        loss_q = (np.sum(case.br_x * np.abs(i_series) ** 2)
                  - np.sum(case.br_b / 2 * (np.abs(V[f]) ** 2 + np.abs(V[t]) ** 2)))
        assert abs(P.sum() - loss_p) < 1e-11 * max(1, loss_p)
        assert abs(Q.sum() - loss_q) < 1e-11 * max(1, abs(loss_q))


def test_power_balance_at_solution():
    """At convergence the specified injections plus slack output equal losses."""
    case = cases.case_14bus(0)
    res = O.newton_polar(case, tol=1e-12)
    Y = O.ybus_single(case)
    V = res["vm"] * np.exp(1j * res["va"])
    f, t = case.br_from, case.br_to
    i_series = (V[f] - V[t]) / (case.br_r + 1j * case.br_x)
    loss_p = np.sum(case.br_r * np.abs(i_series) ** 2)
    P, _ = O.power_polar(Y, res["vm"], res["va"])
    Psp, _ = O.specified_power(case, res["vm"])
    nonslack = case.bus_type != cases.SLACK
    total = Psp[nonslack].sum() + P[~nonslack].sum()
    assert abs(total - loss_p) < 1e-10


def _zip_case(seed):
    case = cases.case_14bus(seed)
    rng = np.random.default_rng(seed + 100)
    z = rng.dirichlet([1, 1, 1], case.n_bus)
    return case.__class__(**{**case.__dict__, "zip": z})


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_jacobian_matches_central_differences(seed):
    case = _zip_case(seed)
    Y = O.ybus_single(case)
    rng = np.random.default_rng(seed)
    vm, va = _random_voltage(case.n_bus, rng)
    pvpq, pq = O.unknowns_polar(case)
    J = O.jacobian_polar(case, Y, vm, va).toarray()
    h = 1e-6
    cols = []
    for k in range(pvpq.size + pq.size):
        vp, ap = vm.copy(), va.copy()
        vmn, van = vm.copy(), va.copy()
        if k < pvpq.size:
            ap[pvpq[k]] += h
            van[pvpq[k]] -= h
        else:
            vp[pq[k - pvpq.size]] += h
            vmn[pq[k - pvpq.size]] -= h
        # J is the derivative of the calculated power, i.e. of -mismatch
        d = -(O.mismatch_polar(case, Y, vp, ap) - O.mismatch_polar(case, Y, vmn, van)) / (2 * h)
        cols.append(d)
    Jfd = np.array(cols).T
    assert np.max(np.abs(J - Jfd)) <= 1e-6 * max(1.0, np.max(np.abs(J)))


def test_newton_matches_generic_root_finder():
    """A derivative-free root finder reaches the same fixed point."""
    case = _zip_case(4)
    Y = O.ybus_single(case)
    pvpq, pq = O.unknowns_polar(case)
    vm0, va0 = O.flat_start_polar(case)

    def F(z):
        vm, va = vm0.copy(), va0.copy()
        va[pvpq] = z[:pvpq.size]
        vm[pq] = z[pvpq.size:]
        return O.mismatch_polar(case, Y, vm, va)

    z0 = np.concatenate([va0[pvpq], vm0[pq]])
    sol = so.root(F, z0, method="hybr", options={"xtol": 1e-13})
    assert np.max(np.abs(F(sol.x))) < 1e-11
    res = O.newton_polar(case, tol=1e-12)
    assert res["converged"]
    assert np.max(np.abs(res["va"][pvpq] - sol.x[:pvpq.size])) < 1e-9
    assert np.max(np.abs(res["vm"][pq] - sol.x[pvpq.size:])) < 1e-9


def test_quadratic_convergence():
    for seed in range(3):
        res = O.newton_polar(cases.case_14bus(seed), tol=1e-13)
        h = res["history"]
        assert res["converged"] and len(h) >= 4
        # once in the basin: e_{k+1} <= C e_k^2
        for a, b in zip(h[1:-1], h[2:]):
            if a < 1e-1 and b > 1e-13:
                assert b <= 50.0 * a * a


def test_permutation_invariance():
    case = cases.case_14bus(5)
    res = O.newton_polar(case, tol=1e-12)
    perm = np.random.default_rng(9).permutation(case.n_bus)
    res2 = O.newton_polar(case.relabel(perm), tol=1e-12)
    assert np.max(np.abs(res2["vm"] - res["vm"][perm])) < 1e-11
    assert np.max(np.abs(res2["va"] - res["va"][perm])) < 1e-11


def test_newton_raphson_and_newton_krylov_agree():
    """NR (SuperLU, dense LU) and NK (GMRES + ILU(0)) reach the same V."""
    for seed in range(3):
        case = _zip_case(seed)
        out = [O.newton_polar(case, tol=1e-11, linear=lin) for lin in ("dense", "splu", "gmres")]
        for r in out:
            assert r["converged"]
        for r in out[1:]:
            assert np.max(np.abs(r["vm"] - out[0]["vm"])) < 1e-9
            assert np.max(np.abs(r["va"] - out[0]["va"])) < 1e-9


def test_medium_grid_converges_with_both_sparse_solvers():
    case = cases.case_2000bus(0)
    r1 = O.newton_polar(case, linear="splu")
    assert r1["converged"] and r1["iterations"] <= 8
    # the 14-bus case is the spec'd load level; larger meshes are scaled
    assert cases.case_14bus(0).load_scale == 1.0
    assert 0 < case.load_scale < 1.0


def test_flat_start_zero_load_needs_no_iteration():
    case = cases.two_bus_case(0.0, 0.0, 0.01, 0.1)
    res = O.newton_polar(case)
    assert res["converged"] and res["iterations"] == 0


# -----------------------------------------------------------------------------
# Krylov pieces
# -----------------------------------------------------------------------------

def test_ilu0_is_exact_lu_without_fill():
    """A tridiagonal matrix has no fill, so ILU(0) is its LU factorisation."""
    rng = np.random.default_rng(0)
    n = 40
    A = sp.diags([rng.uniform(-1, 1, n - 1), rng.uniform(4, 5, n), rng.uniform(-1, 1, n - 1)],
                 [-1, 0, 1], format="csr")
    L, U = O.ilu0(A)
    assert np.max(np.abs((L @ U - A).toarray())) < 1e-13
    # against a dense Doolittle elimination without pivoting
    M = A.toarray()
    for k in range(n):
        M[k + 1:, k] /= M[k, k]
        M[k + 1:, k + 1:] -= np.outer(M[k + 1:, k], M[k, k + 1:])
    assert np.max(np.abs(np.triu(M) - U.toarray())) < 1e-13
    assert np.max(np.abs(np.tril(M, -1) + np.eye(n) - L.toarray())) < 1e-13


def test_ilu0_matches_matrix_on_pattern():
    rng = np.random.default_rng(1)
    n = 60
    A = sp.random(n, n, density=0.08, random_state=2, format="csr")
    A = A + A.T + sp.eye(n) * 6.0
    A.data += rng.uniform(-0.2, 0.2, A.data.size)
    A = A.tocsr()
    L, U = O.ilu0(A)
    LU = (L @ U).toarray()
    Ad = A.toarray()
    mask = Ad != 0
    assert np.max(np.abs(LU[mask] - Ad[mask])) < 1e-12
    # and ILU(0) is not the exact factorisation (fill was dropped)
    assert np.max(np.abs(LU - Ad)) > 1e-8
    # the factors keep the pattern of A
    assert not np.any((L.toarray() != 0) & ~mask & ~np.eye(n, dtype=bool))
    assert not np.any((U.toarray() != 0) & ~mask)


def test_gmres_with_full_restart_solves_exactly():
    rng = np.random.default_rng(2)
    n = 25
    A = sp.csr_matrix(rng.standard_normal((n, n)) + 8 * np.eye(n))
    b = rng.standard_normal(n)
    x, it = O.gmres(A, b, restart=n, tol=1e-13)
    assert np.max(np.abs(x - np.linalg.solve(A.toarray(), b))) < 1e-11
    assert it <= n


def test_bicgstab_solves_like_a_direct_solver():
    """BiCGSTAB (unpreconditioned and with ILU(0)) reaches the dense LU
    solution of a nonsymmetric Jacobian; with M = A exactly (ILU(0) of a
    matrix without fill) it converges in one iteration."""
    case = cases.case_14bus(2)
    Y = O.ybus_single(case)
    vm, va = O.flat_start_polar(case)
    J = O.jacobian_polar(case, Y, vm + 0.01, va + 0.02).tocsr()
    rng = np.random.default_rng(4)
    b = rng.standard_normal(J.shape[0])
    ref = np.linalg.solve(J.toarray(), b)
    x, it = O.bicgstab(J, b, tol=1e-13, max_iter=500)
    assert np.max(np.abs(x - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref)))
    L, U = O.ilu0(J)
    x2, it2 = O.bicgstab(J, b, L, U, tol=1e-13, max_iter=500)
    assert np.max(np.abs(x2 - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref)))
    assert it2 <= it
    T = sp.diags([np.full(30, 4.0), np.full(29, -1.0), np.full(29, -2.0)], [0, 1, -1]).tocsr()
    Lt, Ut = O.ilu0(T)  # tridiagonal: no fill, ILU(0) = LU
    bt = rng.standard_normal(30)
    xt, itt = O.bicgstab(T, bt, Lt, Ut, tol=1e-12)
    assert itt == 1 and np.max(np.abs(T @ xt - bt)) <= 1e-10


def test_newton_with_bicgstab_matches_direct():
    case = cases.transmission_case(300, 405, 60, 7)
    a = O.newton_polar(case, linear="splu")
    b = O.newton_polar(case, linear="bicgstab")
    assert a["converged"] and b["converged"]
    assert np.max(np.abs(a["vm"] - b["vm"])) <= 1e-9
    assert np.max(np.abs(a["va"] - b["va"])) <= 1e-9


def test_gmres_restarted_with_ilu0():
    rng = np.random.default_rng(3)
    n = 120
    A = sp.random(n, n, density=0.05, random_state=4, format="csr") + sp.eye(n) * 3.0
    b = rng.standard_normal(n)
    L, U = O.ilu0(A)
    x, _ = O.gmres(A, b, L, U, restart=5, tol=1e-12, max_restarts=500)
    assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b)


# -----------------------------------------------------------------------------
# three phase, current injection
# -----------------------------------------------------------------------------

def _line_feeder(n, zs, zm, p, q, zip_frac=(1.0, 0.0, 0.0), phases=None,
                 br_phases=None):
    """Chain 0 - 1 - ... - n-1 with identical branches and loads."""
    base = np.full((3, 3), zm, dtype=np.complex128)
    np.fill_diagonal(base, zs)
    ph = np.full(n, 7, dtype=np.uint8) if phases is None else np.asarray(phases, np.uint8)
    bph = ph[1:].copy() if br_phases is None else np.asarray(br_phases, np.uint8)
    pl = np.zeros((n, 3))
    ql = np.zeros((n, 3))
    for k in range(1, n):
        for s in range(3):
            if (ph[k] >> s) & 1:
                pl[k, s] = p[k - 1][s] if np.ndim(p) else p
                ql[k, s] = q[k - 1][s] if np.ndim(q) else q
    return cases.ThreePhaseCase(
        n_node=n, source=0, phases=ph, p_load=pl, q_load=ql,
        zip=np.tile(np.asarray(zip_frac, float), (n, 1)),
        br_from=np.arange(n - 1, dtype=np.int32), br_to=np.arange(1, n, dtype=np.int32),
        br_phases=bph, br_z=np.repeat(base[None], n - 1, axis=0))


ROT = np.exp(-2j * np.pi / 3 * np.arange(3))


@pytest.mark.parametrize("zm", [0.0, 0.004 + 0.015j])
def test_cim_balanced_constant_power_is_two_bus_closed_form(zm):
    """Balanced loads on a transposed line see the positive-sequence z1 = zs - zm."""
    zs = 0.02 + 0.06j
    P, Q = 0.8, 0.3
    case = _line_feeder(2, zs, zm, P, Q)
    res = O.newton_cim(case, tol=1e-13)
    assert res["converged"]
    z1 = zs - zm
    vm2, va2 = two_bus_pq_closed_form(P, Q, z1.real, z1.imag)
    V2 = res["V"][3:6]
    assert np.max(np.abs(V2 - vm2 * np.exp(1j * va2) * ROT)) < 1e-10


def test_cim_constant_impedance_closed_form():
    """Constant-Z load S = S_Z |V|^2 is the admittance conj(S_Z): a divider."""
    zs, zm = 0.03 + 0.08j, 0.01 + 0.03j
    P, Q = 0.9, 0.4
    case = _line_feeder(2, zs, zm, P, Q, zip_frac=(0.0, 0.0, 1.0))
    res = O.newton_cim(case, tol=1e-13)
    assert res["converged"]
    V2 = 1.0 / (1.0 + (zs - zm) * np.conj(P + 1j * Q))
    assert np.max(np.abs(res["V"][3:6] - V2 * ROT)) < 1e-11


def test_cim_single_phase_lateral_is_two_bus_closed_form():
    """A one-phase lateral has no mutual coupling: plain two-bus form, rotated."""
    zs, zm = 0.02 + 0.06j, 0.005 + 0.02j
    P, Q = 0.4, 0.1
    case = _line_feeder(2, zs, zm, P, Q, phases=[7, 2])  # phase b only
    res = O.newton_cim(case, tol=1e-13)
    vm2, va2 = two_bus_pq_closed_form(P, Q, zs.real, zs.imag)
    assert abs(res["V"][4] - vm2 * np.exp(1j * va2) * ROT[1]) < 1e-10
    assert res["V"][3] == 0 and res["V"][5] == 0


def _cim_random_case(seed, n=12):
    return cases.feeder_case(n, seed, lateral_p=0.5, reduced_p=0.6, max_drop=0.08)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cim_jacobian_matches_central_differences(seed):
    case = _cim_random_case(seed)
    Y = O.ybus_three_phase(case)
    rng = np.random.default_rng(seed)
    V = O.cim_flat_start(case)
    V = V * rng.uniform(0.9, 1.05, V.size) * np.exp(1j * rng.uniform(-0.1, 0.1, V.size))
    idx = O.cim_unknowns(case)
    J = O.cim_jacobian(case, Y, V).toarray()[np.ix_(idx, idx)]
    n = case.n_node
    h = 1e-6
    cols = []
    for k in idx:
        node, slot = divmod(int(k), 6)
        dv = np.zeros(3 * n, dtype=np.complex128)
        dv[3 * node + slot % 3] = h if slot < 3 else 1j * h
        fp = O.cim_mismatch(case, Y, V + dv)[idx]
        fm = O.cim_mismatch(case, Y, V - dv)[idx]
        cols.append(-(fp - fm) / (2 * h))  # J = d(Y V - I_sp)/dV
    Jfd = np.array(cols).T
    assert np.max(np.abs(J - Jfd)) <= 1e-6 * max(1.0, np.max(np.abs(J)))


def test_cim_power_balance_identity():
    """Total injected complex power equals the series losses of all branches."""
    case = _cim_random_case(4, n=30)
    Y = O.ybus_three_phase(case)
    rng = np.random.default_rng(1)
    V = O.cim_flat_start(case) * rng.uniform(0.9, 1.1, 3 * case.n_node)
    S = V * np.conj(Y @ V)
    loss = 0.0
    for e in range(case.n_branch):
        ph = [s for s in range(3) if (case.br_phases[e] >> s) & 1]
        f, t = case.br_from[e], case.br_to[e]
        dV = V[3 * f + np.array(ph)] - V[3 * t + np.array(ph)]
        Z = case.br_z[e][np.ix_(ph, ph)]
        i_series = np.linalg.solve(Z, dV)
        loss += np.conj(i_series) @ (Z @ i_series)  # I^H Z I
    assert abs(S.sum() - loss) < 1e-10 * max(1.0, abs(loss))


def test_cim_matches_generic_root_finder():
    case = _cim_random_case(7)
    Y = O.ybus_three_phase(case)
    idx = O.cim_unknowns(case)
    V0 = O.cim_flat_start(case)
    n = case.n_node

    def unpack(z):
        full = np.zeros(6 * n)
        full[idx] = z
        full = full.reshape(n, 6)
        return V0 * np.where(O.cim_free_slots(case), 0.0, 1.0) + (full[:, :3] + 1j * full[:, 3:]).reshape(-1)

    V0c = O.cim_flat_start(case).copy()
    z0 = np.stack([V0c.real.reshape(n, 3), V0c.imag.reshape(n, 3)], 1).reshape(n, 6).reshape(-1)[idx]
    F = lambda z: O.cim_mismatch(case, Y, unpack(z))[idx]  # noqa: E731
    sol = so.root(F, z0, method="hybr", options={"xtol": 1e-13})
    assert np.max(np.abs(F(sol.x))) < 1e-11
    res = O.newton_cim(case, tol=1e-12)
    assert res["converged"]
    assert np.max(np.abs(res["V"] - unpack(sol.x))) < 1e-9


def test_cim_solvers_agree_on_generated_feeder():
    case = cases.feeder_case(300, 3)
    out = [O.newton_cim(case, tol=1e-11, linear=lin) for lin in ("dense", "splu", "gmres")]
    for r in out:
        assert r["converged"]
    for r in out[1:]:
        assert np.max(np.abs(r["V"] - out[0]["V"])) < 1e-9


# -----------------------------------------------------------------------------
# branch flows (Sec. I: voltages and branch power flows are the outputs)
# -----------------------------------------------------------------------------

def _bus_sums(case, pf_, qf, pt, qt, slots, width):
    """Power leaving each bus (slot) into its branches."""
    S = np.zeros(slots, dtype=np.complex128)
    for k in range(case.n_branch):
        f, t = int(case.br_from[k]), int(case.br_to[k])
        for a in range(width):
            S[width * f + a] += pf_[k] + 1j * qf[k] if width == 1 else pf_[k, a] + 1j * qf[k, a]
            S[width * t + a] += pt[k] + 1j * qt[k] if width == 1 else pt[k, a] + 1j * qt[k, a]
    return S


@pytest.mark.parametrize("seed", [0, 3])
def test_branch_flows_sum_to_nodal_injections(seed):
    """Kirchhoff at every bus: the powers leaving a bus into its branches add
    up to V_i conj((Y V)_i), with Y assembled independently (Eq. 2-3)."""
    rng = np.random.default_rng(seed)
    case = cases.case_14bus(seed)
    Y = O.ybus_single(case)
    for _ in range(3):
        vm, va = _random_voltage(case.n_bus, rng)
        pf_, qf, pt, qt, loss = O.branch_flows(case, vm, va)
        V = vm * np.exp(1j * va)
        S = _bus_sums(case, pf_, qf, pt, qt, case.n_bus, 1)
        ref = V * np.conj(Y @ V)
        assert np.max(np.abs(S - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))
        assert abs(loss[0] + 1j * loss[1] - ref.sum()) < 1e-11


def test_branch_flows_three_phase_sum_to_nodal_injections():
    case = _cim_random_case(5, n=25)
    Y = O.ybus_three_phase(case)
    rng = np.random.default_rng(2)
    V = O.cim_flat_start(case) * rng.uniform(0.9, 1.1, 3 * case.n_node) * np.exp(
        1j * rng.uniform(-0.05, 0.05, 3 * case.n_node))
    vm, va = np.abs(V), np.where(np.abs(V) > 0, np.angle(V), 0.0)
    pf_, qf, pt, qt, loss = O.branch_flows(case, vm, va)
    S = _bus_sums(case, pf_, qf, pt, qt, 3 * case.n_node, 3)
    ref = V * np.conj(Y @ V)
    assert np.max(np.abs(S - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_branch_flow_of_two_bus_closed_form():
    """A load P + jQ at the end of one line: the line carries P_to = -P,
    Q_to = -Q at the load end and loses r |S|^2 / |V2|^2 (with |V2| from the
    closed form above)."""
    P, Q, r, x = 0.6, 0.25, 0.03, 0.12
    case = cases.two_bus_case(P, Q, r, x)
    res = O.newton_polar(case, tol=1e-12)
    pf_, qf, pt, qt, loss = O.branch_flows(case, res["vm"], res["va"])
    v2, _ = two_bus_pq_closed_form(P, Q, r, x)
    assert abs(pt[0] + P) < 1e-10 and abs(qt[0] + Q) < 1e-10
    assert abs(loss[0] - r * (P * P + Q * Q) / v2 ** 2) < 1e-10
    assert abs(loss[1] - x * (P * P + Q * Q) / v2 ** 2) < 1e-10


# -----------------------------------------------------------------------------
# three phase with PV nodes (augmented CIM Newton)
# -----------------------------------------------------------------------------

def _pv_line(x, pg, vset, n=2):
    import dataclasses as dc

    case = _line_feeder(n, 1j * x, 0.0, 0.0, 0.0)
    node_type = np.full(n, cases.PQ, dtype=np.int32)
    node_type[n - 1] = cases.PV
    v = np.ones(n)
    v[n - 1] = vset
    p_gen = np.zeros((n, 3))
    p_gen[n - 1] = pg
    return dc.replace(case, node_type=node_type, v_set=v, p_gen=p_gen)


@pytest.mark.parametrize("pg,x,vset", [(0.3, 0.1, 1.02), (-0.2, 0.2, 0.97)])
def test_cim_pv_node_is_two_bus_pv_closed_form(pg, x, vset):
    """A lossless line (z = jx, no mutual coupling) from the balanced source
    to a PV node: each phase is the two-bus PV problem, delta2 = asin(P x /
    (V1 V2)) from the phase's source angle, and the generator's reactive
    injection Q = (V2^2 - V1 V2 cos delta2) / x."""
    case = _pv_line(x, pg, vset)
    res = O.newton_cim(case, tol=1e-12)
    assert res["converged"]
    d = math.asin(pg * x / vset)
    q = (vset * vset - vset * math.cos(d)) / x
    for s in range(3):
        v2 = res["V"][3 + s]
        assert abs(abs(v2) - vset) < 1e-12
        assert abs(np.angle(v2 / ROT[s]) - d) < 1e-10
        assert abs(res["Qg"][3 + s] - q) < 1e-10


def test_cim_pv_converges_quadratically_and_balances_power():
    """The augmented Jacobian is exact: the mismatch falls quadratically, and
    at the solution the generation (with the solved Q_g) minus the loads
    equals the series losses of all branches."""
    case = cases.with_pv_nodes(cases.feeder_case(120, 5), 3, 2)
    res = O.newton_cim(case, tol=1e-13)
    h = res["history"]
    assert res["converged"]
    for k in range(1, len(h) - 1):
        if h[k] < 1e-3 and h[k + 1] > 1e-12:
            assert h[k + 1] <= 50.0 * h[k] ** 2
    Y = O.ybus_three_phase(case)
    V, Qg = res["V"], res["Qg"]
    S = V * np.conj(Y @ V)  # injected into the network
    free = O.cim_free_slots(case)
    Ssp = O.cim_specified_power(case, V, Qg)
    assert np.max(np.abs((S - Ssp)[free])) < 1e-11
    pv = O.cim_pv_slots(case)
    assert np.max(np.abs(np.abs(V[pv]) - np.repeat(case.v_set, 3)[pv])) < 1e-12


@pytest.mark.parametrize("seed", [0, 3])
def test_cim_pv_augmented_jacobian_matches_central_differences(seed):
    """Every column of the augmented system (Re V, Im V and Q_g unknowns;
    current and magnitude rows) against central differences of
    G = [Y V - I_sp, |V|^2 - v_set^2], at a point with non-zero Q_g."""
    case = cases.with_pv_nodes(cases.feeder_case(40, 7 + seed), 4, seed)
    Y = O.ybus_three_phase(case)
    rng = np.random.default_rng(seed)
    V = O.cim_flat_start(case)
    V = V * rng.uniform(0.92, 1.05, V.size) * np.exp(1j * rng.uniform(-0.1, 0.1, V.size))
    pvs = np.flatnonzero(O.cim_pv_slots(case))
    assert pvs.size > 0
    Qg = np.zeros(3 * case.n_node)
    Qg[pvs] = rng.uniform(-0.2, 0.2, pvs.size)
    Fa, Ja = O.cim_pv_system(case, Y, V, Qg)
    Ja = Ja.toarray()
    idx = O.cim_unknowns(case)
    n = case.n_node
    h = 1e-6

    def G(V_, Q_):
        return -O.cim_pv_system(case, Y, V_, Q_)[0]

    cols = []
    for k in idx:
        node, slot = divmod(int(k), 6)
        dv = np.zeros(3 * n, dtype=np.complex128)
        dv[3 * node + slot % 3] = h if slot < 3 else 1j * h
        cols.append((G(V + dv, Qg) - G(V - dv, Qg)) / (2 * h))
    for s in pvs:
        dq = np.zeros(3 * n)
        dq[s] = h
        cols.append((G(V, Qg + dq) - G(V, Qg - dq)) / (2 * h))
    Jfd = np.array(cols).T
    assert Ja.shape == Jfd.shape
    assert np.max(np.abs(Ja - Jfd)) <= 1e-6 * max(1.0, np.max(np.abs(Ja)))
    # the Q_g columns are non-zero only in the PV node's own two rows
    qcols = Ja[:, idx.size:]
    assert np.all(np.count_nonzero(qcols, axis=0) <= 2)


# three phase: reactive limits of PV phase slots (rounds of switching)

@pytest.mark.parametrize("pg,x,vset,qmax", [(0.3, 0.1, 1.02, 0.1), (0.1, 0.2, 1.03, 0.05)])
def test_cim_reactive_limit_two_node_closed_form(pg, x, vset, qmax):
    """The lossless two-node line of the PV closed form with q_max below the
    reactive injection that holds v_set: every phase is held at q_max, a
    two-bus PQ problem with injection pg + j q_max per phase."""
    import dataclasses as dc

    case = _pv_line(x, pg, vset)
    d = math.asin(pg * x / vset)
    q_free = (vset * vset - vset * math.cos(d)) / x
    assert q_free > qmax
    case = dc.replace(case, q_min=np.full((2, 3), -1.0), q_max=np.full((2, 3), qmax))
    res = O.newton_cim_qlim(case, tol=1e-12)
    assert res["converged"] and res["rounds"] == 2
    assert res["switched"][3:].all() and not res["switched"][:3].any()
    vm2, va2 = two_bus_pq_closed_form(-pg, -qmax, 0.0, x)
    for s in range(3):
        v2 = res["V"][3 + s]
        assert abs(abs(v2) - vm2) < 1e-10
        assert abs(np.angle(v2 / ROT[s]) - va2) < 1e-10
        assert abs(res["Qg"][3 + s] - qmax) < 1e-12


@pytest.mark.parametrize("n,seed", [(400, 3), (600, 4)])
def test_cim_reactive_limits_hold_at_the_solution(n, seed):
    """After the rounds: the power mismatch is below tol, every PV slot still
    free is inside its limits at |V| = v_set, every held slot sits at the
    limit it crossed with |V| off v_set; wide limits give the plain solve."""
    import dataclasses as dc

    base = cases.with_pv_nodes(cases.feeder_case(n, seed), 8, 3)
    case = cases.with_phase_q_limits(base, 1)
    res = O.newton_cim_qlim(case)
    assert res["converged"] and res["switched"].any() and res["rounds"] >= 2
    Y = O.ybus_three_phase(case)
    V, Qg, sw = res["V"], res["Qg"], res["switched"]
    dS = O.cim_power_mismatch(case, Y, V, Qg)
    assert max(np.max(np.abs(dS.real)), np.max(np.abs(dS.imag))) <= 1e-8
    pv = O.cim_pv_slots(case)
    assert not (sw & ~pv).any()
    qmin, qmax = case.q_min.reshape(-1), case.q_max.reshape(-1)
    free = pv & ~sw
    assert np.all(Qg[free] <= qmax[free] + 1e-12) and np.all(Qg[free] >= qmin[free] - 1e-12)
    vset = np.repeat(case.v_set, 3)
    assert np.max(np.abs(np.abs(V[free]) - vset[free])) < 1e-12
    at = np.minimum(np.abs(Qg[sw] - qmax[sw]), np.abs(Qg[sw] - qmin[sw]))
    assert np.max(at) == 0.0
    assert np.min(np.abs(np.abs(V[sw]) - vset[sw])) > 1e-7
    wide = dc.replace(case, q_min=np.full((case.n_node, 3), -10.0),
                      q_max=np.full((case.n_node, 3), 10.0))
    r2 = O.newton_cim_qlim(wide)
    r0 = O.newton_cim(base)
    assert r2["rounds"] == 1 and not r2["switched"].any()
    assert np.array_equal(r2["V"], r0["V"])
