"""Host-side logic of the library, CPU only: symbol exports, validation,
admittance assembly and the symbolic analysis (no GPU calls)."""
import ctypes
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pf_oracle as O
from paper_1711_10579_gb300 import build as B
from paper_1711_10579_gb300 import cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pf():
    B.build()
    from paper_1711_10579_gb300 import pf as _pf

    _pf.lib()
    return _pf


def test_library_exports_every_declared_symbol(pf):
    header = open(os.path.join(ROOT, "include", "pf.h")).read()
    header = re.sub(r"/\*.*?\*/", "", header, flags=re.S)
    declared = set(re.findall(r"\b(pf_[a-z_]+)\s*\(", header))
    assert len(declared) >= 20
    lib = ctypes.CDLL(pf.LIB_PATH)
    missing = [s for s in sorted(declared) if not hasattr(lib, s)]
    assert not missing, missing


def test_ybus_matches_oracle_single_phase(pf):
    for seed in range(3):
        case = cases.transmission_case(300, 405, 60, seed)
        rp, col, val = pf.pf_ybus(case)
        Y = sp.csr_matrix((val, col, rp), shape=(case.n_bus,) * 2)
        assert abs(Y - O.ybus_single(case)).max() < 1e-10


def test_ybus_matches_oracle_three_phase(pf):
    f = cases.feeder_case(120, 4, reduced_p=0.6)
    rp, col, val = pf.pf_ybus(f)
    n = f.n_node
    Yd = np.zeros((3 * n, 3 * n), complex)
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            Yd[3 * i:3 * i + 3, 3 * col[p]:3 * col[p] + 3] = val[p]
    assert np.max(np.abs(Yd - O.ybus_three_phase(f).toarray())) < 1e-9


def _brute_fill(n, edges, perm):
    """Filled graph of symmetric elimination in the order perm (brute force)."""
    inv = np.empty(n, int)
    inv[perm] = np.arange(n)
    adj = [set() for _ in range(n)]
    for a, b in edges:
        adj[inv[a]].add(inv[b])
        adj[inv[b]].add(inv[a])
    filled = set()
    for k in range(n):
        higher = sorted(v for v in adj[k] if v > k)
        for i in higher:
            filled.add((i, k))
            filled.add((k, i))
        for a in higher:
            for b in higher:
                if a != b:
                    adj[a].add(b)
    return filled | {(i, i) for i in range(n)}


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_symbolic_lu_pattern_is_the_exact_fill(pf, seed):
    case = cases.transmission_case(60, 90, 10, seed)
    perm, rp, col, fl, bl = pf.pf_symbolic(case, pf.PF_NR)
    n = case.n_bus
    assert sorted(perm) == list(range(n))
    got = {(i, int(col[p])) for i in range(n) for p in range(rp[i], rp[i + 1])}
    want = _brute_fill(n, zip(case.br_from, case.br_to), perm)
    assert got == want


@pytest.mark.parametrize("method", ["NR", "NK"])
def test_level_sets_respect_dependencies(pf, method):
    case = cases.transmission_case(500, 680, 100, 3)
    m = pf.PF_NR if method == "NR" else pf.PF_NK
    perm, rp, col, fl, bl = pf.pf_symbolic(case, m)
    n = case.n_bus
    for i in range(n):
        cols = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cols) > 0) and i in cols
        lower, upper = cols[cols < i], cols[cols > i]
        assert np.all(fl[lower] < fl[i]) and (lower.size == 0 or fl[i] == fl[lower].max() + 1)
        assert np.all(bl[upper] < bl[i]) and (upper.size == 0 or bl[i] == bl[upper].max() + 1)


def test_ilu_pattern_is_ybus_pattern(pf):
    case = cases.transmission_case(400, 540, 80, 5)
    perm, rp, col, _, _ = pf.pf_symbolic(case, pf.PF_NK)
    yr, yc, _ = pf.pf_ybus(case)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    got = {(i, int(c)) for i in range(case.n_bus) for c in col[rp[i]:rp[i + 1]]}
    want = {(int(inv[i]), int(inv[c])) for i in range(case.n_bus) for c in yc[yr[i]:yr[i + 1]]}
    assert got == want


def test_rcm_reduces_bandwidth(pf):
    case = cases.transmission_case(2000, 2700, 400, 7)
    perm, rp, col, _, _ = pf.pf_symbolic(case, pf.PF_NK)
    rows = np.repeat(np.arange(case.n_bus), np.diff(rp))
    bw_rcm = np.max(np.abs(rows - col))
    yr, yc, _ = pf.pf_ybus(case)
    rows0 = np.repeat(np.arange(case.n_bus), np.diff(yr))
    assert bw_rcm < np.max(np.abs(rows0 - yc)) / 5


def test_tree_feeder_has_no_fill(pf):
    st = pf.pf_analyze(cases.feeder_case(2000, 1))
    assert st["nnz_lu"] == st["nnz_y"]
    assert st["block_size"] == 6


def test_stats_of_the_10000_bus_case(pf):
    st = pf.pf_analyze(cases.case_10000bus(0))
    assert st["n_unknowns"] == 2 * 7999 + 2000
    assert st["nnz_y"] == 10_000 + 2 * 13_500
    assert st["nnz_y"] <= st["nnz_lu"] <= 3 * st["nnz_y"]
    assert st["levels_factor"] < 200


def _invalid(pf, case, match):
    with pytest.raises(pf.PfError) as e:
        pf.pf_analyze(case)
    assert e.value.code == pf.PF_ERR_INVALID
    assert re.search(match, str(e.value)), str(e.value)


def test_validation_errors(pf):
    import dataclasses as dc

    base = cases.case_14bus(0)
    bt = base.bus_type.copy()
    bt[0] = cases.PQ
    _invalid(pf, dc.replace(base, bus_type=bt), "exactly one slack")
    bt = base.bus_type.copy()
    bt[3] = cases.SLACK
    _invalid(pf, dc.replace(base, bus_type=bt), "exactly one slack")
    f = base.br_from.copy()
    f[2] = 99
    _invalid(pf, dc.replace(base, br_from=f), "out of range")
    t = base.br_to.copy()
    t[0] = base.br_from[0]
    _invalid(pf, dc.replace(base, br_to=t), "self loop")
    r, x = base.br_r.copy(), base.br_x.copy()
    r[1] = x[1] = 0.0
    _invalid(pf, dc.replace(base, br_r=r, br_x=x), "zero impedance")
    pl = base.p_load.copy()
    pl[5] = np.nan
    _invalid(pf, dc.replace(base, p_load=pl), "non-finite")
    # drop every branch of bus 13: disconnected
    keep = (base.br_from != 13) & (base.br_to != 13)
    _invalid(pf, dc.replace(base, br_from=base.br_from[keep], br_to=base.br_to[keep],
                            br_r=base.br_r[keep], br_x=base.br_x[keep], br_b=base.br_b[keep]),
             "not connected")
    fd = cases.feeder_case(30, 0)
    ph = fd.phases.copy()
    ph[5] = 0
    _invalid(pf, dc.replace(fd, phases=ph), "phase mask")
    bp = fd.br_phases.copy()
    bp[:] = 7
    ph = fd.phases.copy()
    ph[fd.br_to[4]] = 1
    _invalid(pf, dc.replace(fd, phases=ph, br_phases=bp), "phases missing")


def test_single_bus_case_is_valid(pf):
    one = cases.SinglePhaseCase(
        n_bus=1, bus_type=np.array([0], np.int32), v_set=np.ones(1), p_gen=np.zeros(1),
        q_gen=np.zeros(1), p_load=np.zeros(1), q_load=np.zeros(1), zip=np.array([[1.0, 0, 0]]),
        br_from=np.zeros(0, np.int32), br_to=np.zeros(0, np.int32), br_r=np.zeros(0),
        br_x=np.zeros(0), br_b=np.zeros(0))
    st = pf.pf_analyze(one)
    assert st["n_unknowns"] == 0 and st["nnz_lu"] == 1


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1711_10579_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"(import\s+oracle|from\s+oracle|pf_oracle)", src), f


def test_reactive_limit_validation(pf):
    import dataclasses as dc

    base = cases.with_q_limits(cases.case_14bus(0), 1)
    pf.pf_analyze(base)  # valid
    qmin = base.q_min.copy()
    qmin[3] = base.q_max[3] + 0.1
    _invalid(pf, dc.replace(base, q_min=qmin), "not an interval")
    qmin[3] = np.nan
    _invalid(pf, dc.replace(base, q_min=qmin), "not an interval")
    # infinite limits are an interval
    pf.pf_analyze(dc.replace(base, q_min=np.full(base.n_bus, -np.inf),
                             q_max=np.full(base.n_bus, np.inf)))
    d = pf.make_desc(base)
    d.desc.q_max = None  # one without the other
    with pytest.raises(pf.PfError) as e:
        st = pf.pf_case_stats()
        pf._check(pf.lib().pf_analyze(pf.C.byref(d.desc), pf.C.byref(st)))
    assert "go together" in str(e.value)


def test_info_and_opts_layout(pf):
    """The Python mirrors of pf_info / pf_opts end with the reactive-limit
    fields, and the defaults leave the limits off."""
    assert [f for f, _ in pf.pf_info._fields_][-2:] == ["q_switched", "q_rounds"]
    assert pf.INFO_DTYPE.itemsize == pf.C.sizeof(pf.pf_info) == 48
    assert pf.make_opts().q_limits == 0


def _c_struct_fields(header, name):
    """Field names of `typedef struct { ... } name;` in a C header, in order."""
    import re as _re

    end = _re.search(r"\}\s*" + name + r";", header).start()
    body = header[header.rfind("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = _re.sub(r"/\*.*?\*/", "", body, flags=_re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "int a, b" or "const double* x"
        head, *rest = decl.split(",")
        fields.append(_re.findall(r"[A-Za-z_]\w*", head)[-1])
        fields += [_re.findall(r"[A-Za-z_]\w*", r)[-1] for r in rest]
    return fields


@pytest.mark.parametrize("cname,pyname", [("pf_opts", "pf_opts"), ("pf_info", "pf_info"),
                                          ("pf_case_desc", "pf_case_desc"),
                                          ("pf_case_stats", "pf_case_stats"),
                                          ("pf_serve_stats", "pf_serve_stats")])
def test_binding_structs_mirror_the_header(pf, cname, pyname):
    """The ctypes mirrors list the header's fields in the header's order (a
    field added to one side only, or reordered, shifts every later field)."""
    import os

    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "pf.h")).read()
    assert [f for f, _ in getattr(pf, pyname)._fields_] == _c_struct_fields(hdr, cname)


def _run_schedule(sch, col, rowptr, A):
    """Executes the packed factor records level by level the way the kernels
    do, every step reading the state before the step (so an item that reads
    what another item of its own step writes gives a wrong factor), and
    returns (factor blocks, inverse diagonal blocks)."""
    FF = 1 << 30
    LU = A.copy()
    n, bs = rowptr.size - 1, A.shape[1]
    uinv = np.zeros((n, bs, bs))
    for l in range(sch["fac_ptr"].size - 1):
        before = LU.copy()
        for e, k, dg, _ in sch["fac_rec"][sch["fac_ptr"][l]:sch["fac_ptr"][l + 1]]:
            inv = np.linalg.inv(before[dg])
            if e == dg:
                uinv[k] = inv
            else:
                LU[e] = before[e] @ inv
        before = LU.copy()
        for x, le, ue, rest in sch["tgt_rec"][sch["tgt_ptr"][l]:sch["tgt_ptr"][l + 1]]:
            e = x & ~FF
            if x & FF:
                assert np.all(before[e] == 0.0)  # a fill entry's first update
            c = np.zeros((bs, bs)) if x & FF else before[e].copy()
            c -= before[le] @ before[ue]
            q = rest
            while q >= 0 and sch["con"][q][0] >= 0:
                c -= before[sch["con"][q][0]] @ before[sch["con"][q][1]]
                q += 1
            LU[e] = c
    return LU, uinv


@pytest.mark.parametrize("name,method", [("14", 0), ("300", 0), ("feeder", 0), ("300", 1)])
def test_packed_schedule_factors_and_solves(pf, name, method):
    """The fan-out records the kernels run (pf_schedule), executed level by
    level on the CPU with every step reading the state before it: Newton-
    Raphson's records give the exact block LU of a random matrix on the
    factor pattern (L U = A, fill entries starting from zero), Newton-
    Krylov's the ILU(0) factor ((L U)_ij = A_ij on the pattern); the sweep
    records, level by level, solve L U x = b."""
    meth = pf.PF_NR if method == 0 else pf.PF_NK
    case = {"14": cases.case_14bus(0), "300": cases.transmission_case(300, 405, 60, 2),
            "feeder": cases.feeder_case(60, 3)}[name]
    bs = 2 if isinstance(case, cases.SinglePhaseCase) else 6
    perm, rowptr, col, _, _ = pf.pf_symbolic(case, meth)
    sch = pf.pf_schedule(case, meth)
    n = rowptr.size - 1
    # the Ybus pattern in the new numbering: the entries that are not fill
    import ctypes as C

    st = pf.pf_analyze(case)
    yrp = np.zeros(n + 1, np.int32)
    ycol = np.zeros(st["nnz_y"], np.int32)
    d = pf.make_desc(case)
    nz = C.c_int64()
    vals = np.zeros(st["nnz_y"] * (2 if bs == 2 else 18))
    pf.lib().pf_ybus(C.byref(d.desc), C.byref(nz), yrp.ctypes.data_as(C.POINTER(C.c_int32)),
                     ycol.ctypes.data_as(C.POINTER(C.c_int32)),
                     vals.ctypes.data_as(C.POINTER(C.c_double)))
    inv = np.empty(n, int)
    inv[perm] = np.arange(n)
    ypat = {(inv[i], inv[j]) for i in range(n) for j in ycol[yrp[i]:yrp[i + 1]]}
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    rng = np.random.default_rng(3)
    A = rng.uniform(-1, 1, (col.size, bs, bs))
    for e in range(col.size):
        if (rows[e], col[e]) not in ypat:
            A[e] = 0.0  # fill
        elif rows[e] == col[e]:
            A[e] += 4.0 * bs * np.eye(bs)
    LU, uinv = _run_schedule(sch, col, rowptr, A)
    Ad = np.zeros((n * bs, n * bs))
    Ld = np.eye(n * bs)
    Ud = np.zeros((n * bs, n * bs))
    for e in range(col.size):
        i, j = rows[e], col[e]
        blk = (slice(i * bs, i * bs + bs), slice(j * bs, j * bs + bs))
        Ad[blk] = A[e]
        if j < i:
            Ld[blk] = LU[e]
        else:
            Ud[blk] = LU[e]
    for k in range(n):
        dk = rowptr[k] + np.flatnonzero(col[rowptr[k]:rowptr[k + 1]] == k)[0]
        assert np.allclose(uinv[k] @ LU[dk], np.eye(bs), atol=1e-12)
    P = Ld @ Ud
    if meth == pf.PF_NR:
        assert np.max(np.abs(P - Ad)) <= 1e-11 * np.max(np.abs(Ad))
    else:
        mask = np.zeros_like(Ad, dtype=bool)
        for e in range(col.size):
            i, j = rows[e], col[e]
            mask[i * bs:i * bs + bs, j * bs:j * bs + bs] = True
        assert np.max(np.abs((P - Ad)[mask])) <= 1e-11 * np.max(np.abs(Ad))
    # the sweeps, level by level, each level reading the vector before it
    b = rng.uniform(-1, 1, (n, bs))
    y = b.copy()
    for l in range(sch["flev_ptr"].size - 1):
        before = y.copy()
        for i, p0, p1, _ in sch["fwd_rec"][sch["flev_ptr"][l]:sch["flev_ptr"][l + 1]]:
            y[i] = before[i] - sum((LU[p] @ before[col[p]] for p in range(p0, p1)), np.zeros(bs))
    for l in range(sch["blev_ptr"].size - 1):
        before = y.copy()
        for i, p0, p1, _ in sch["bwd_rec"][sch["blev_ptr"][l]:sch["blev_ptr"][l + 1]]:
            acc = before[i] - sum((LU[p] @ before[col[p]] for p in range(p0, p1)), np.zeros(bs))
            y[i] = uinv[i] @ acc
    x = y.reshape(-1)
    assert np.max(np.abs(P @ x - b.reshape(-1))) <= 1e-10
