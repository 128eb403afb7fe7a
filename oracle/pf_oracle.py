"""Plain FP64 CPU oracle for the Newton power-flow iteration.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
link this module: only the test suite, the smoke check and the CPU-baseline leg
of the benchmark use it.  It shares no code with the CUDA library; the only
common input is the seeded case description drawn by the case generators.

What it computes, in the paper's notation (arXiv 1711.10579):

* ``ybus_single``        nodal admittance matrix, Eq. 2-3, pi-model branches.
* ``power_polar``        P_i, Q_i in polar form, Eq. 6-7 (term by term).
* ``mismatch_polar``     Delta P, Delta Q, Eq. 8-9 (with ZIP loads, Eq. 14-15).
* ``jacobian_polar``     [J1 J2; J3 J4] of Eq. 10, first derivatives of Eq. 6-7.
* ``newton_polar``       single-phase Newton-Raphson (Sec. II.A algorithm box).
* ``generator_q`` / ``newton_polar_qlim``  reactive output of PV generators and
                         the rounds of PV -> PQ switching at their limits.
* ``ybus_three_phase``   3x3 complex block admittance matrix, Eq. 11.
* ``cim_mismatch``       current mismatch Delta I, Eq. 12-19.
* ``cim_jacobian``       6x6 real blocks of Eq. 21-23.
* ``newton_cim``         three-phase current-injection Newton (Sec. II.B box),
                         with PV nodes through ``cim_pv_system`` (augmented
                         with reactive injections and |V| equations).
* ``newton_cim_qlim``    the same with the reactive limits of PV phase slots
                         enforced by rounds of switching.
* ``ilu0`` / ``gmres``   ILU(0) and restarted, right-preconditioned GMRES used
                         by the Newton-Krylov variant (Sec. III.B).
* ``bicgstab``           right-preconditioned BiCGSTAB, the Krylov method the
                         paper used (Sec. III.B).
* ``branch_flows``       power into each branch at both ends and the losses
                         (the "power flows" output of the problem statement,
                         Sec. I), single and three phase, from the branch
                         models of Eq. 2-3 and Eq. 11.

Readings of points the paper leaves open (the same list is kept with the
design notes):

* line charging: pi model, total charging b split b/2 to each end (Eq. 2 sums
  over j = 0, the ground);
* theta_ij is the angle of Y_ij and delta_i the angle of bus i (the only way
  Eq. 6-7 are consistent);
* unknowns: angles of PV and PQ buses, magnitudes of PQ buses; the slack is
  fixed (Eq. 10);
* stop test: infinity norm of the power mismatch <= tol (default 1e-8 pu),
  checked before each solve, in place of the unnamed step thresholds;
* ZIP coefficients are the load at |V| = 1 pu split by fractions
  (constant power, constant current, constant impedance), Eq. 14-15;
* three-phase: every node has three phase slots; absent phases and the
  source node carry no unknowns; the source is an ideal balanced source;
  loads are wye-connected; a PV node (deferred by Sec. II.B) injects a given
  P and a free Q per phase and holds |V| = v_set on every phase present;
* reactive limits of PV buses: after a converged solve every PV bus (three
  phase: every PV phase slot) whose generator Q is outside [q_min, q_max]
  is held at that limit (|V| free) and the solve is repeated from the last
  voltages, until nothing violates; a held bus or slot stays held;
* the diagonal adjustments a, b, c, d of Eq. 23 are the derivatives of the
  specified current (Eq. 17) with respect to the real and imaginary voltage,
  so that J is the exact Jacobian of Y V - I_sp in the ordering of Eq. 19-20;
* flat start: |V| = set point or 1 pu, angle 0 (three-phase: balanced
  1 pu at 0, -120, +120 degrees).
"""
from __future__ import annotations

import math
from dataclasses import replace

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

SLACK, PV, PQ = 0, 1, 2


# =============================================================================
# single phase, polar form (Sec. II.A)
# =============================================================================

def ybus_single(case) -> sp.csr_matrix:
    """Eq. 2-3: Y_ii = sum of admittances at bus i (incl. ground), Y_ij = -y_ij.

    Each branch is a pi model: series admittance y = 1/(r + jx) and half of
    the total line charging j b/2 to ground at each end.
    """
    n = case.n_bus
    rows, cols, vals = [], [], []
    for f, t, r, x, b in zip(case.br_from, case.br_to, case.br_r, case.br_x,
                             case.br_b):
        y = 1.0 / complex(r, x)
        sh = complex(0.0, b / 2.0)
        rows += [f, t, f, t]
        cols += [f, t, t, f]
        vals += [y + sh, y + sh, -y, -y]
    Y = sp.coo_matrix((np.asarray(vals, dtype=np.complex128),
                       (np.asarray(rows), np.asarray(cols))), shape=(n, n))
    return Y.tocsr()  # duplicates are summed


def specified_power(case, vm):
    """Eq. 12-15: specified injection = generation - ZIP load at |V|."""
    zp, zi, zz = case.zip[:, 0], case.zip[:, 1], case.zip[:, 2]
    shape = zp + zi * vm + zz * vm * vm
    return case.p_gen - case.p_load * shape, case.q_gen - case.q_load * shape


def specified_power_dvm(case, vm):
    """Derivative of the specified power (Eq. 12-15) with respect to |V_i|."""
    zi, zz = case.zip[:, 1], case.zip[:, 2]
    dshape = zi + 2.0 * zz * vm
    return -case.p_load * dshape, -case.q_load * dshape


def power_polar(Y, vm, va):
    """Eq. 6-7: P_i and Q_i summed over the nonzeros of row i of Y."""
    Yc = Y.tocoo()
    i, j = Yc.row, Yc.col
    mag = np.abs(Yc.data)
    th = np.angle(Yc.data)
    ang = th - va[i] + va[j]
    n = vm.size
    P = np.bincount(i, weights=vm[i] * vm[j] * mag * np.cos(ang), minlength=n)
    Q = -np.bincount(i, weights=vm[i] * vm[j] * mag * np.sin(ang), minlength=n)
    return P, Q


def unknowns_polar(case):
    """Rows/columns of Eq. 10: angle of every PV and PQ bus, |V| of every PQ."""
    pvpq = np.flatnonzero(case.bus_type != SLACK)
    pq = np.flatnonzero(case.bus_type == PQ)
    return pvpq, pq


def mismatch_polar(case, Y, vm, va):
    """Eq. 8-9 stacked as [Delta P (PV, PQ); Delta Q (PQ)]."""
    pvpq, pq = unknowns_polar(case)
    P, Q = power_polar(Y, vm, va)
    Psp, Qsp = specified_power(case, vm)
    return np.concatenate([(Psp - P)[pvpq], (Qsp - Q)[pq]])


def jacobian_polar(case, Y, vm, va) -> sp.csr_matrix:
    """Eq. 10: derivatives of P_calc - P_sp and Q_calc - Q_sp (Eq. 6-9).

    Off-diagonal entries (j != i), with a = theta_ij - delta_i + delta_j:
        dP_i/d delta_j = -|V_i||V_j||Y_ij| sin a
        dQ_i/d delta_j = -|V_i||V_j||Y_ij| cos a
        dP_i/d |V_j|  =  |V_i||Y_ij| cos a
        dQ_i/d |V_j|  = -|V_i||Y_ij| sin a
    Diagonal entries collect the j != i terms of the same derivatives taken
    with respect to bus i plus the j = i term of Eq. 6-7, and subtract the
    derivative of the ZIP load (Eq. 14-15).
    """
    n = case.n_bus
    Yc = Y.tocoo()
    i, j = Yc.row, Yc.col
    mag = np.abs(Yc.data)
    th = np.angle(Yc.data)
    ang = th - va[i] + va[j]
    off = i != j
    io, jo, mo, ao = i[off], j[off], mag[off], ang[off]

    # off-diagonal derivatives
    dP_dd = -vm[io] * vm[jo] * mo * np.sin(ao)
    dQ_dd = -vm[io] * vm[jo] * mo * np.cos(ao)
    dP_dv = vm[io] * mo * np.cos(ao)
    dQ_dv = -vm[io] * mo * np.sin(ao)

    # diagonal derivatives
    d = ~off
    yii = np.zeros(n)
    th_ii = np.zeros(n)
    yii[i[d]] = mag[d]
    th_ii[i[d]] = th[d]
    dPi_ddi = np.bincount(io, weights=vm[io] * vm[jo] * mo * np.sin(ao), minlength=n)
    dQi_ddi = np.bincount(io, weights=vm[io] * vm[jo] * mo * np.cos(ao), minlength=n)
    dPi_dvi = (np.bincount(io, weights=vm[jo] * mo * np.cos(ao), minlength=n)
               + 2.0 * vm * yii * np.cos(th_ii))
    dQi_dvi = (-np.bincount(io, weights=vm[jo] * mo * np.sin(ao), minlength=n)
               - 2.0 * vm * yii * np.sin(th_ii))
    dPsp, dQsp = specified_power_dvm(case, vm)
    dPi_dvi = dPi_dvi - dPsp
    dQi_dvi = dQi_dvi - dQsp

    # full 2n x 2n matrix in (delta, |V|) x (P, Q) order, then select Eq. 10
    rows = np.concatenate([io, io, n + io, n + io,
                           np.arange(n), np.arange(n), n + np.arange(n), n + np.arange(n)])
    cols = np.concatenate([jo, n + jo, jo, n + jo,
                           np.arange(n), n + np.arange(n), np.arange(n), n + np.arange(n)])
    vals = np.concatenate([dP_dd, dP_dv, dQ_dd, dQ_dv,
                           dPi_ddi, dPi_dvi, dQi_ddi, dQi_dvi])
    J = sp.coo_matrix((vals, (rows, cols)), shape=(2 * n, 2 * n)).tocsr()
    pvpq, pq = unknowns_polar(case)
    sel = np.concatenate([pvpq, n + pq])
    return J[sel][:, sel].tocsr()


def flat_start_polar(case):
    """Initial guess: set-point magnitudes (1 pu for PQ), zero angles."""
    vm = np.where(case.bus_type == PQ, 1.0, case.v_set).astype(np.float64)
    return vm, np.zeros(case.n_bus)


def newton_polar(case, tol=1e-8, max_iter=30, linear="splu", vm0=None,
                 va0=None, gmres_restart=30, gmres_tol=1e-10, Y=None):
    """Single-phase Newton-Raphson, Sec. II.A algorithm box.

    Each iteration evaluates the mismatch (Eq. 8-9), stops when its infinity
    norm is <= ``tol``, otherwise builds the Jacobian (Eq. 10), solves for
    (Delta delta, Delta |V|) and updates the angles of PV/PQ buses and the
    magnitudes of PQ buses.  ``linear`` picks the solve of Eq. 10:
    ``"splu"`` SuperLU with COLAMD ordering (Sec. III.A, the paper's solver),
    ``"dense"`` LAPACK partial-pivoting LU, ``"gmres"`` restarted GMRES with an
    ILU(0) preconditioner on a bandwidth-reducing ordering (Sec. III.B),
    ``"bicgstab"`` BiCGSTAB with the same preconditioner (the paper's).

    Returns dict(vm, va, iterations, mismatch, history, steps, converged).
    """
    if Y is None:
        Y = ybus_single(case)
    vm, va = flat_start_polar(case)
    if vm0 is not None:
        vm = np.array(vm0, dtype=np.float64)
    if va0 is not None:
        va = np.array(va0, dtype=np.float64)
    pvpq, pq = unknowns_polar(case)
    npvpq = pvpq.size
    history, steps = [], []
    k = 0
    converged = False
    while True:
        F = mismatch_polar(case, Y, vm, va)
        norm = float(np.max(np.abs(F))) if F.size else 0.0
        history.append(norm)
        if not np.isfinite(norm):
            break
        if norm <= tol:
            converged = True
            break
        if k >= max_iter:
            break
        k += 1
        J = jacobian_polar(case, Y, vm, va)
        dx = solve_linear(J, F, linear, gmres_restart, gmres_tol)
        va[pvpq] += dx[:npvpq]
        vm[pq] += dx[npvpq:]
        steps.append(float(np.max(np.abs(dx))) if dx.size else 0.0)
    return dict(vm=vm, va=va, iterations=k, mismatch=history[-1],
                history=history, steps=steps, converged=converged)


def generator_q(case, Y, vm, va):
    """Reactive output of the generator at every bus: the injection Q_i of
    Eq. 7 plus the bus's own reactive load at |V_i| (Eq. 12-15)."""
    _, Q = power_polar(Y, vm, va)
    zp, zi, zz = case.zip[:, 0], case.zip[:, 1], case.zip[:, 2]
    return Q + case.q_load * (zp + zi * vm + zz * vm * vm)


def newton_polar_qlim(case, tol=1e-8, max_iter=30, linear="splu", max_rounds=50,
                      gmres_restart=30, gmres_tol=1e-10):
    """Newton-Raphson with the reactive limits [q_min, q_max] of PV buses
    enforced by type switching (the PV rule of Sec. II.A holds |V| by free
    reactive output; a generator at its limit can no longer do so).

    Rounds: solve (newton_polar) from the last voltages; take the reactive
    output of every PV bus (generator_q); every PV bus outside its limits
    becomes a PQ bus whose generation is the limit it crossed; stop after a
    round with no violation.  A switched bus stays PQ.  Returns
    newton_polar's dict with the iterations of all rounds summed, plus
    ``switched`` (bool per bus), ``rounds``, ``qg`` (reactive generation at
    the solution) and ``case`` (the switched case)."""
    Y = ybus_single(case)
    cur = case
    switched = np.zeros(case.n_bus, dtype=bool)
    vm0 = va0 = None
    total = 0
    rounds = 0
    while True:
        rounds += 1
        res = newton_polar(cur, tol, max_iter, linear, vm0, va0, gmres_restart, gmres_tol, Y=Y)
        total += res["iterations"]
        qg = generator_q(cur, Y, res["vm"], res["va"])
        if not res["converged"] or case.q_max is None or rounds >= max_rounds:
            break
        pv = cur.bus_type == PV
        hi = pv & (qg > case.q_max)
        lo = pv & (qg < case.q_min)
        if not (hi | lo).any():
            break
        bt = cur.bus_type.copy()
        bt[hi | lo] = PQ
        q_gen = cur.q_gen.copy()
        q_gen[hi] = case.q_max[hi]
        q_gen[lo] = case.q_min[lo]
        cur = replace(cur, bus_type=bt, q_gen=q_gen)
        switched |= hi | lo
        vm0, va0 = res["vm"], res["va"]
    res = dict(res)
    res.update(iterations=total, switched=switched, rounds=rounds, qg=qg, case=cur)
    return res


def solve_linear(J, F, linear="splu", restart=30, tol=1e-10):
    """Solve J dx = F with the chosen method (see ``newton_polar``)."""
    if F.size == 0:
        return F.copy()
    if linear == "dense":
        return np.linalg.solve(J.toarray(), F)
    if linear == "splu":
        return spla.splu(J.tocsc(), permc_spec="COLAMD").solve(F)
    if linear in ("gmres", "bicgstab"):
        from scipy.sparse.csgraph import reverse_cuthill_mckee
        p = reverse_cuthill_mckee(J.tocsr(), symmetric_mode=False)
        Jp = J.tocsr()[p][:, p].tocsr()
        L, U = ilu0(Jp)
        if linear == "gmres":
            y, _ = gmres(Jp, F[p], L, U, restart=restart, tol=tol, max_restarts=200)
        else:
            y, _ = bicgstab(Jp, F[p], L, U, tol=tol, max_iter=20000)
        dx = np.empty_like(y)
        dx[p] = y
        return dx
    raise ValueError(linear)


# =============================================================================
# Krylov pieces for the Newton-Krylov variant (Sec. III.B)
# =============================================================================

def ilu0(A):
    """ILU(0): unit-lower L and upper U restricted to the pattern of A.

    Row-by-row elimination where an update a_ij -= l_ik u_kj is kept only if
    (i, j) is already a nonzero of A, so that (L U)_ij = A_ij on the pattern.
    Plain Python loops over the sparse rows: for small and medium matrices.
    """
    A = A.tocsr().astype(np.float64)
    A.sort_indices()
    n = A.shape[0]
    indptr, indices = A.indptr, A.indices
    vals = A.data.copy()
    pos = [dict(zip(indices[indptr[i]:indptr[i + 1]].tolist(),
                    range(indptr[i], indptr[i + 1]))) for i in range(n)]
    diag = np.array([pos[i][i] for i in range(n)])
    for i in range(n):
        row = pos[i]
        for p in range(indptr[i], indptr[i + 1]):
            k = indices[p]
            if k >= i:
                break
            vals[p] /= vals[diag[k]]
            lik = vals[p]
            for q in range(diag[k] + 1, indptr[k + 1]):
                j = indices[q]
                t = row.get(j)
                if t is not None:
                    vals[t] -= lik * vals[q]
    LU = sp.csr_matrix((vals, indices.copy(), indptr.copy()), shape=A.shape)
    L = sp.tril(LU, k=-1, format="csr") + sp.eye(n, format="csr")
    U = sp.triu(LU, k=0, format="csr")
    return L.tocsr(), U.tocsr()


def bicgstab(A, b, L=None, U=None, tol=1e-10, max_iter=1000):
    """BiCGSTAB (van der Vorst 1992; the Krylov method of Sec. III.B) with
    right preconditioning M = L U: solves A M^-1 u = b, x = M^-1 u, from
    x = 0, stopping when ||b - A x|| <= tol ||b||.  Returns (x, iterations).
    """
    from scipy.sparse.linalg import spsolve_triangular

    def apply_minv(v):
        if L is None:
            return v
        y = spsolve_triangular(L, v, lower=True, unit_diagonal=True)
        return spsolve_triangular(U, y, lower=False)

    n = b.size
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0
    r = b.copy()
    r_hat = b.copy()
    rho_prev = alpha = omega = 1.0
    v = np.zeros(n)
    p = np.zeros(n)
    for it in range(1, max_iter + 1):
        rho = r_hat @ r
        if rho == 0.0:
            return x, it - 1
        beta = (rho / rho_prev) * (alpha / omega)
        p = r + beta * (p - omega * v)
        p_hat = apply_minv(p)
        v = A @ p_hat
        alpha = rho / (r_hat @ v)
        s = r - alpha * v
        if np.linalg.norm(s) <= tol * bnorm:
            return x + alpha * p_hat, it
        s_hat = apply_minv(s)
        t = A @ s_hat
        omega = (t @ s) / (t @ t)
        x = x + alpha * p_hat + omega * s_hat
        r = s - omega * t
        if np.linalg.norm(r) <= tol * bnorm or omega == 0.0:
            return x, it
        rho_prev = rho
    return x, max_iter


def gmres(A, b, L=None, U=None, restart=30, tol=1e-10, max_restarts=100,
          x0=None):
    """Restarted GMRES(m) with right preconditioning M = L U.

    Arnoldi with modified Gram-Schmidt, Givens rotations on the Hessenberg
    matrix, stop when the residual norm <= tol * ||b||.  Returns (x, iters).
    """
    from scipy.sparse.linalg import spsolve_triangular

    def apply_minv(v):
        if L is None:
            return v
        y = spsolve_triangular(L, v, lower=True, unit_diagonal=True)
        return spsolve_triangular(U, y, lower=False)

    n = b.size
    x = np.zeros(n) if x0 is None else x0.astype(np.float64).copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), 0
    total = 0
    for _ in range(max_restarts):
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            break
        m = restart
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(m):
            w = A @ apply_minv(V[k])
            for i in range(k + 1):
                H[i, k] = V[i] @ w
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0.0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = math.hypot(H[k, k], H[k + 1, k])
            cs[k] = H[k, k] / den
            sn[k] = H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            k_used = k + 1
            total += 1
            if abs(g[k + 1]) <= tol * bnorm:
                break
        y = np.zeros(k_used)
        for i in range(k_used - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k_used] @ y[i + 1:]) / H[i, i]
        x = x + apply_minv(V[:k_used].T @ y)
    return x, total


# =============================================================================
# three phase, current injection method (Sec. II.B)
# =============================================================================

def _phase_list(mask):
    return [s for s in range(3) if (int(mask) >> s) & 1]


def ybus_three_phase(case) -> sp.csr_matrix:
    """Eq. 11: 3x3 complex blocks; phase s of node i sits at row 3 i + s.

    A branch's admittance is the inverse of the submatrix of its series
    impedance over the phases present on that branch.
    """
    n = case.n_node
    rows, cols, vals = [], [], []
    for e in range(case.n_branch):
        f, t = int(case.br_from[e]), int(case.br_to[e])
        ph = _phase_list(case.br_phases[e])
        Zs = case.br_z[e][np.ix_(ph, ph)]
        Yb = np.linalg.inv(Zs)
        for a, pa in enumerate(ph):
            for c, pc in enumerate(ph):
                y = Yb[a, c]
                rows += [3 * f + pa, 3 * t + pa, 3 * f + pa, 3 * t + pa]
                cols += [3 * f + pc, 3 * t + pc, 3 * t + pc, 3 * f + pc]
                vals += [y, y, -y, -y]
    Y = sp.coo_matrix((np.asarray(vals, dtype=np.complex128),
                       (np.asarray(rows), np.asarray(cols))), shape=(3 * n, 3 * n))
    return Y.tocsr()


def cim_free_slots(case):
    """Phase slots that carry unknowns: present phases of non-source nodes."""
    mask = np.zeros(3 * case.n_node, dtype=bool)
    for i in range(case.n_node):
        if i == case.source:
            continue
        for s in _phase_list(case.phases[i]):
            mask[3 * i + s] = True
    return mask


def cim_flat_start(case):
    """Balanced v_source at 0, -120, +120 degrees on every present phase."""
    rot = np.exp(-2j * np.pi / 3 * np.arange(3))
    V = np.zeros(3 * case.n_node, dtype=np.complex128)
    for i in range(case.n_node):
        for s in _phase_list(case.phases[i]):
            V[3 * i + s] = case.v_source * rot[s]
    return V


def cim_pv_slots(case):
    """Phase slots of PV nodes (present phases; the reading beyond the paper:
    a PV node's generator injects P_g per phase and holds |V| at v_set)."""
    mask = np.zeros(3 * case.n_node, dtype=bool)
    pv = case.pv_mask() if hasattr(case, "pv_mask") else np.zeros(case.n_node, bool)
    for i in np.flatnonzero(pv):
        for s in _phase_list(case.phases[i]):
            mask[3 * i + s] = True
    return mask


def cim_specified_power(case, V, Qg=None):
    """Eq. 12-15 per phase slot: S_sp = generation - ZIP load at |V|; the
    generation is P_g + j Qg on PV slots (Qg, [3 n], the reactive injection
    of the iterate) and zero elsewhere."""
    vm = np.abs(V)
    zp = np.repeat(case.zip[:, 0], 3)
    zi = np.repeat(case.zip[:, 1], 3)
    zz = np.repeat(case.zip[:, 2], 3)
    shape = zp + zi * vm + zz * vm * vm
    S = -(case.p_load.reshape(-1) * shape) - 1j * (case.q_load.reshape(-1) * shape)
    pv = cim_pv_slots(case)
    if pv.any():
        q = np.zeros(3 * case.n_node) if Qg is None else np.asarray(Qg, dtype=float)
        S = S + np.where(pv, case.p_gen.reshape(-1) + 1j * q, 0.0)
    return S


def cim_specified_current(case, V, Qg=None):
    """Eq. 17: I_sp = conj(S_sp / V) on free slots, 0 elsewhere."""
    free = cim_free_slots(case)
    S = cim_specified_power(case, V, Qg)
    I = np.zeros_like(V)
    I[free] = np.conj(S[free] / V[free])
    return I


def cim_mismatch(case, Y, V, Qg=None):
    """Eq. 16, 18, 19: Delta I = I_sp - Y V, per node as [Im a,b,c, Re a,b,c].

    Returns the full 6 n vector; entries of absent phases and of the source
    are zero.
    """
    free = cim_free_slots(case)
    dI = cim_specified_current(case, V, Qg) - Y @ V
    dI = np.where(free, dI, 0.0)
    n = case.n_node
    out = np.empty((n, 6))
    d3 = dI.reshape(n, 3)
    out[:, :3] = d3.imag
    out[:, 3:] = d3.real
    return out.reshape(-1)


def cim_power_mismatch(case, Y, V, Qg=None):
    """Delta S = V conj(Delta I) = S_sp - V conj(Y V) on free slots."""
    free = cim_free_slots(case)
    dS = cim_specified_power(case, V, Qg) - V * np.conj(Y @ V)
    return np.where(free, dS, 0.0)


def cim_load_derivatives(case, V, Qg=None):
    """a, b, c, d of Eq. 23 per phase slot.

    With S_sp = P + jQ a function of m = |V| (Eq. 14-15) and
    I_sp = conj(S_sp) V / m^2 (Eq. 17):
        Re I_sp = (P Vr + Q Vi) / m^2,  Im I_sp = (P Vi - Q Vr) / m^2.
    a = d Im/d Vr, b = d Im/d Vi, c = d Re/d Vr, d = d Re/d Vi by the product
    rule, using dm/dVr = Vr/m, dm/dVi = Vi/m.
    """
    Vr, Vi = V.real, V.imag
    m = np.abs(V)
    zp = np.repeat(case.zip[:, 0], 3)
    zi = np.repeat(case.zip[:, 1], 3)
    zz = np.repeat(case.zip[:, 2], 3)
    pl = case.p_load.reshape(-1)
    ql = case.q_load.reshape(-1)
    P = -pl * (zp + zi * m + zz * m * m)
    Q = -ql * (zp + zi * m + zz * m * m)
    pv = cim_pv_slots(case)
    if pv.any():  # a PV generator injects constant P_g + j Qg
        P = P + np.where(pv, case.p_gen.reshape(-1), 0.0)
        Q = Q + np.where(pv, 0.0 if Qg is None else np.asarray(Qg, dtype=float), 0.0)
    dP = -pl * (zi + 2.0 * zz * m)  # dP/dm
    dQ = -ql * (zi + 2.0 * zz * m)
    free = cim_free_slots(case)
    safe_m = np.where(free, m, 1.0)
    g = 1.0 / safe_m ** 2
    dg = -2.0 / safe_m ** 3
    dm_dr = np.where(free, Vr / safe_m, 0.0)
    dm_di = np.where(free, Vi / safe_m, 0.0)
    re_num = P * Vr + Q * Vi
    im_num = P * Vi - Q * Vr
    c = g * (P + (dP * Vr + dQ * Vi) * dm_dr) + re_num * dg * dm_dr
    d = g * (Q + (dP * Vr + dQ * Vi) * dm_di) + re_num * dg * dm_di
    a = g * (-Q + (dP * Vi - dQ * Vr) * dm_dr) + im_num * dg * dm_dr
    b = g * (P + (dP * Vi - dQ * Vr) * dm_di) + im_num * dg * dm_di
    z = ~free
    for arr in (a, b, c, d):
        arr[z] = 0.0
    return a, b, c, d


def cim_jacobian(case, Y, V, Qg=None) -> sp.csr_matrix:
    """Eq. 21-23 as a 6n x 6n real matrix.

    Node-pair block (rows [Im a,b,c; Re a,b,c], columns [Re a,b,c; Im a,b,c]):
    [[B, G], [G, -B]] with G + jB the 3x3 block of Y (Eq. 21); on the
    diagonal a, b, c, d are subtracted (Eq. 23).
    """
    n = case.n_node
    Yc = Y.tocoo()
    r, c_, v = Yc.row, Yc.col, Yc.data
    ni, si = r // 3, r % 3
    nj, sj = c_ // 3, c_ % 3
    G, B = v.real, v.imag
    rows = np.concatenate([6 * ni + si, 6 * ni + si, 6 * ni + 3 + si, 6 * ni + 3 + si])
    cols = np.concatenate([6 * nj + sj, 6 * nj + 3 + sj, 6 * nj + sj, 6 * nj + 3 + sj])
    vals = np.concatenate([B, G, G, -B])
    a, b, c, d = cim_load_derivatives(case, V, Qg)
    k = np.arange(3 * n)
    nk, sk = k // 3, k % 3
    rows = np.concatenate([rows, 6 * nk + sk, 6 * nk + sk, 6 * nk + 3 + sk, 6 * nk + 3 + sk])
    cols = np.concatenate([cols, 6 * nk + sk, 6 * nk + 3 + sk, 6 * nk + sk, 6 * nk + 3 + sk])
    vals = np.concatenate([vals, -a, -b, -c, -d])
    return sp.coo_matrix((vals, (rows, cols)), shape=(6 * n, 6 * n)).tocsr()


def cim_unknowns(case):
    """Indices into the 6n ordering of Eq. 20 that are free unknowns."""
    free = cim_free_slots(case).reshape(case.n_node, 3)
    mask = np.concatenate([free, free], axis=1).reshape(-1)
    return np.flatnonzero(mask)


def newton_cim(case, tol=1e-8, max_iter=30, linear="splu", V0=None,
               gmres_restart=30, gmres_tol=1e-10, Y=None):
    """Three-phase current-injection Newton, Sec. II.B algorithm box.

    Each iteration forms Delta I (Eq. 12-20), stops when the power mismatch
    V conj(Delta I) has infinity norm (over real and imaginary parts) <= tol,
    otherwise solves J Delta V = Delta I (Eq. 22-23) on the free unknowns,
    adds Delta V to the rectangular voltages and forms the complex V again.
    """
    if Y is None:
        Y = ybus_three_phase(case)
    V = cim_flat_start(case) if V0 is None else np.array(V0, dtype=np.complex128)
    if cim_pv_slots(case).any():
        return _newton_cim_pv(case, Y, V, tol, max_iter, linear, gmres_restart, gmres_tol)
    idx = cim_unknowns(case)
    n = case.n_node
    history, steps = [], []
    k = 0
    converged = False
    while True:
        dS = cim_power_mismatch(case, Y, V)
        norm = float(max(np.max(np.abs(dS.real)), np.max(np.abs(dS.imag))))
        history.append(norm)
        if not np.isfinite(norm):
            break
        if norm <= tol:
            converged = True
            break
        if k >= max_iter:
            break
        k += 1
        F = cim_mismatch(case, Y, V)[idx]
        J = cim_jacobian(case, Y, V)[idx][:, idx].tocsr()
        dx = solve_linear(J, F, linear, gmres_restart, gmres_tol)
        full = np.zeros(6 * n)
        full[idx] = dx
        full = full.reshape(n, 6)
        V = V + (full[:, :3] + 1j * full[:, 3:]).reshape(-1)
        steps.append(float(np.max(np.abs(dx))) if dx.size else 0.0)
    return dict(V=V, iterations=k, mismatch=history[-1], history=history,
                steps=steps, converged=converged)


def newton_cim_qlim(case, tol=1e-8, max_iter=30, linear="splu", max_rounds=50,
                    gmres_restart=30, gmres_tol=1e-10):
    """Three-phase Newton with the reactive limits [q_min, q_max] of every
    PV phase slot enforced by switching, the rounds of newton_polar_qlim per
    slot: after a converged solve every PV slot whose reactive injection Q_g
    is outside its limits is held at the limit it crossed (a given
    injection, |V| free) and the solve repeats from the last voltages; stop
    after a round with no violation.  Returns newton_cim's dict with the
    iterations summed, ``switched`` (bool [3 n]) and ``rounds``."""
    Y = ybus_three_phase(case)
    n = case.n_node
    V = cim_flat_start(case)
    pv = cim_pv_slots(case)
    switched = np.zeros(3 * n, dtype=bool)
    Qg = np.zeros(3 * n)
    total = 0
    rounds = 0
    while True:
        rounds += 1
        res = _newton_cim_pv(case, Y, V, tol, max_iter, linear, gmres_restart, gmres_tol,
                             switched, Qg)
        total += res["iterations"]
        if not res["converged"] or case.q_max is None or rounds >= max_rounds:
            break
        qg = res["Qg"]
        qmax = np.asarray(case.q_max, dtype=float).reshape(-1)
        qmin = np.asarray(case.q_min, dtype=float).reshape(-1)
        act = pv & ~switched
        hi = act & (qg > qmax)
        lo = act & (qg < qmin)
        if not (hi | lo).any():
            break
        Qg = qg.copy()
        Qg[hi] = qmax[hi]
        Qg[lo] = qmin[lo]
        switched |= hi | lo
        V = res["V"]
    res = dict(res)
    res.update(iterations=total, switched=switched, rounds=rounds)
    return res


# ---------------------------------------------------------------------------
# branch flows (Sec. I problem statement: voltages and branch power flows)
# ---------------------------------------------------------------------------

def branch_flows(case, vm, va):
    """Power leaving each end of each branch into it, and the total loss.

    Single phase, branch k from f to t (pi model of Eq. 2): series current
    i_s = (V_f - V_t) / (r + jx), charging current j (b/2) V at each end, so
    the power leaving bus f is S_f = V_f conj(i_s + j (b/2) V_f) and leaving
    bus t is S_t = V_t conj(-i_s + j (b/2) V_t).  Three phase (Eq. 11): the
    series currents over the branch's phases are Z^-1 (V_f - V_t), with Z the
    branch's impedance restricted to its phases, and no charging.  vm, va as
    the solvers return them (three phase: [3 n], slot 3 i + s).  Returns
    (p_from, q_from, p_to, q_to) per branch (three phase: [m, 3], zero on
    absent phases) and the total loss (P, Q) = sum of S_f + S_t.
    """
    V = np.asarray(vm, dtype=float) * np.exp(1j * np.asarray(va, dtype=float))
    m = case.n_branch
    if hasattr(case, "n_bus"):
        Sf = np.zeros(m, dtype=np.complex128)
        St = np.zeros(m, dtype=np.complex128)
        for k in range(m):
            f, t = int(case.br_from[k]), int(case.br_to[k])
            i_s = (V[f] - V[t]) / complex(case.br_r[k], case.br_x[k])
            ch = 1j * case.br_b[k] / 2.0
            Sf[k] = V[f] * np.conj(i_s + ch * V[f])
            St[k] = V[t] * np.conj(-i_s + ch * V[t])
    else:
        Sf = np.zeros((m, 3), dtype=np.complex128)
        St = np.zeros((m, 3), dtype=np.complex128)
        for k in range(m):
            f, t = int(case.br_from[k]), int(case.br_to[k])
            ph = _phase_list(case.br_phases[k])
            Z = case.br_z[k][np.ix_(ph, ph)]
            dv = V[3 * f + np.asarray(ph)] - V[3 * t + np.asarray(ph)]
            i_s = np.linalg.solve(Z, dv)
            for a, s in enumerate(ph):
                Sf[k, s] = V[3 * f + s] * np.conj(i_s[a])
                St[k, s] = V[3 * t + s] * np.conj(-i_s[a])
    loss = (Sf + St).sum()
    return Sf.real, Sf.imag, St.real, St.imag, (loss.real, loss.imag)


def cim_pv_system(case, Y, V, Qg, switched=None):
    """Right-hand side and Jacobian of the augmented CIM system with PV slots.
    Unknowns: the CIM unknowns (cim_unknowns order) then Q_g of every PV slot
    (cim_pv_slots order).  Equations: the current mismatch rows, then
    |V|^2 - v_set^2 per PV slot.  Returns (Fa, Ja) with Ja the derivative of
    G = [Y V - I_sp, |V|^2 - v_set^2] and Fa = -G, so that Ja dx = Fa is the
    Newton step.  The Q_g column of the current rows is
    d(Y V - I_sp)/dQ_g = j V / |V|^2 (I_sp = conj(S_sp) V / |V|^2 with S_sp
    containing j Q_g); the magnitude row is (2 Re V, 2 Im V).  Slots in
    ``switched`` (held at a reactive limit) keep their Q_g as a given
    injection and have neither unknown nor magnitude equation."""
    idx = cim_unknowns(case)
    act = cim_pv_slots(case)
    if switched is not None:
        act = act & ~switched
    pvs = np.flatnonzero(act)
    npv = pvs.size
    vset = np.repeat(np.asarray(case.v_set, dtype=float), 3)
    pos = {int(k): p for p, k in enumerate(idx)}
    F = cim_mismatch(case, Y, V, Qg)[idx]
    J = cim_jacobian(case, Y, V, Qg)[idx][:, idx].tocsr()
    nu = idx.size
    rows, cols, vals = [], [], []
    for t, slot in enumerate(pvs):
        node, ph = divmod(int(slot), 3)
        v = V[slot]
        w = 1j * v / abs(v) ** 2
        r_im, r_re = pos[6 * node + ph], pos[6 * node + 3 + ph]
        rows += [r_im, r_re, nu + t, nu + t]
        cols += [nu + t, nu + t, r_im, r_re]
        vals += [w.imag, w.real, 2.0 * v.real, 2.0 * v.imag]
    Jq = sp.coo_matrix((vals, (rows, cols)), shape=(nu + npv, nu + npv)).tocsr()
    Ja = sp.bmat([[J, None], [None, sp.csr_matrix((npv, npv))]]).tocsr() + Jq
    cons = np.abs(V[pvs]) ** 2 - vset[pvs] ** 2
    return np.concatenate([F, -cons]), Ja


def _newton_cim_pv(case, Y, V, tol, max_iter, linear, gmres_restart, gmres_tol,
                   switched=None, Qg0=None):
    """CIM Newton with PV nodes, augmented form: the reactive injection Q_g of
    every PV slot is an extra unknown and |V|^2 = v_set^2 an extra equation
    per PV slot (linearised: 2 Vr dVr + 2 Vi dVi = v_set^2 - |V|^2).  The
    Q_g column of the current equations is d(Y V - I_sp)/dQ_g = j V / |V|^2
    (I_sp = conj(S_sp) V / |V|^2 with S_sp containing j Q_g).  The start
    puts PV slots at v_set on the flat-start angles with Q_g = 0."""
    n = case.n_node
    pv = cim_pv_slots(case)
    if switched is not None:
        pv = pv & ~switched
    vset = np.repeat(np.asarray(case.v_set, dtype=float), 3)
    V = np.where(pv, V / np.where(np.abs(V) > 0, np.abs(V), 1.0) * vset, V)
    Qg = np.zeros(3 * n) if Qg0 is None else np.array(Qg0, dtype=float)
    idx = cim_unknowns(case)
    pvs = np.flatnonzero(pv)
    npv = pvs.size
    history, steps = [], []
    k = 0
    converged = False
    while True:
        dS = cim_power_mismatch(case, Y, V, Qg)
        cons = np.abs(V[pvs]) ** 2 - vset[pvs] ** 2
        norm = float(max(np.max(np.abs(dS.real)), np.max(np.abs(dS.imag)),
                         np.max(np.abs(cons)) if npv else 0.0))
        history.append(norm)
        if not np.isfinite(norm):
            break
        if norm <= tol:
            converged = True
            break
        if k >= max_iter:
            break
        k += 1
        Fa, Ja = cim_pv_system(case, Y, V, Qg, switched)
        nu = idx.size
        dx = solve_linear(Ja, Fa, linear, gmres_restart, gmres_tol)
        full = np.zeros(6 * n)
        full[idx] = dx[:nu]
        full = full.reshape(n, 6)
        V = V + (full[:, :3] + 1j * full[:, 3:]).reshape(-1)
        Qg[pvs] += dx[nu:]
        steps.append(float(np.max(np.abs(dx))) if dx.size else 0.0)
    return dict(V=V, iterations=k, mismatch=history[-1], history=history,
                steps=steps, converged=converged, Qg=Qg)
