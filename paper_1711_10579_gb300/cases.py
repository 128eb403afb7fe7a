"""Seeded synthetic power-flow inputs shaped like the paper's workloads.

The paper benchmarks replicated IEEE-30 transmission grids (Sec. IV) and a
replicated IEEE 906 LV three-phase feeder (Sec. IV, Table 1).  Neither data set
is used here; these generators build random grids of the same kind instead:

* ``transmission_case``  single-phase meshed grid: a random geometric spanning
  tree plus extra nearest-neighbour edges, one slack, PV and PQ buses.
* ``feeder_case``        three-phase unbalanced radial feeder with 1- and
  2-phase laterals and ZIP loads per phase.
* ``scenario_loads``     per-scenario lognormal load multipliers for batches.
* ``serving_stream``     Poisson arrivals of mixed transmission/feeder requests.

This module only draws numbers.  It holds none of the method's arithmetic (no
admittance matrix, no power-flow equation), so both the FP64 oracle and the
CUDA library consume its output independently.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SLACK, PV, PQ = 0, 1, 2
PHASE_A, PHASE_B, PHASE_C = 1, 2, 4


@dataclasses.dataclass
class SinglePhaseCase:
    """Single-phase (balanced) grid data in per unit.

    ``p_gen``/``q_gen`` are generator injections, ``p_load``/``q_load`` the
    load at |V| = 1 pu; the specified net injection is gen - load (Eq. 12-13).
    ``zip`` holds per-bus load fractions (constant power, constant current,
    constant impedance) in the order of Eq. 14-15; rows sum to one.
    Branches use the pi model: series r + jx, total line charging b.
    """

    n_bus: int
    bus_type: np.ndarray  # int32 [n]: 0 slack, 1 PV, 2 PQ
    v_set: np.ndarray  # float64 [n]: |V| set point (slack, PV); 1.0 for PQ
    p_gen: np.ndarray  # float64 [n]
    q_gen: np.ndarray  # float64 [n] (used for PQ buses only)
    p_load: np.ndarray  # float64 [n]
    q_load: np.ndarray  # float64 [n]
    zip: np.ndarray  # float64 [n, 3]
    br_from: np.ndarray  # int32 [m]
    br_to: np.ndarray  # int32 [m]
    br_r: np.ndarray  # float64 [m]
    br_x: np.ndarray  # float64 [m]
    br_b: np.ndarray  # float64 [m]
    name: str = ""
    seed: int = 0
    load_scale: float = 1.0
    q_min: np.ndarray | None = None  # float64 [n]: reactive generation limits
    q_max: np.ndarray | None = None  # of PV buses (pu); None = no limits

    @property
    def n_branch(self) -> int:
        return int(self.br_from.shape[0])

    def with_loads(self, p_load, q_load, p_gen=None) -> "SinglePhaseCase":
        """Copy of the case with other loads (and optionally generation)."""
        return dataclasses.replace(
            self,
            p_load=np.ascontiguousarray(p_load, dtype=np.float64),
            q_load=np.ascontiguousarray(q_load, dtype=np.float64),
            p_gen=self.p_gen.copy() if p_gen is None
            else np.ascontiguousarray(p_gen, dtype=np.float64))

    def relabel(self, perm: np.ndarray) -> "SinglePhaseCase":
        """Same grid with bus ``perm[k]`` renamed to ``k``."""
        perm = np.asarray(perm)
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        return dataclasses.replace(
            self,
            bus_type=self.bus_type[perm].copy(), v_set=self.v_set[perm].copy(),
            p_gen=self.p_gen[perm].copy(), q_gen=self.q_gen[perm].copy(),
            p_load=self.p_load[perm].copy(), q_load=self.q_load[perm].copy(),
            zip=self.zip[perm].copy(),
            q_min=None if self.q_min is None else self.q_min[perm].copy(),
            q_max=None if self.q_max is None else self.q_max[perm].copy(),
            br_from=inv[self.br_from].astype(np.int32),
            br_to=inv[self.br_to].astype(np.int32))


@dataclasses.dataclass
class ThreePhaseCase:
    """Three-phase unbalanced radial feeder in per unit (Sec. II.B).

    Every node owns three phase slots (a, b, c); ``phases`` is a bit mask of
    the slots that exist.  ``br_z`` is each branch's full 3x3 series impedance
    matrix; only the rows and columns of the phases present on the branch are
    meaningful.  Loads are wye-connected per phase, ZIP fractions in the order
    (constant power, constant current, constant impedance) of Eq. 14-15.
    Node ``source`` is an ideal balanced source of magnitude ``v_source``.
    """

    n_node: int
    source: int
    phases: np.ndarray  # uint8 [n] bit mask a=1, b=2, c=4
    p_load: np.ndarray  # float64 [n, 3]
    q_load: np.ndarray  # float64 [n, 3]
    zip: np.ndarray  # float64 [n, 3]
    br_from: np.ndarray  # int32 [m] (parent)
    br_to: np.ndarray  # int32 [m] (child)
    br_phases: np.ndarray  # uint8 [m]
    br_z: np.ndarray  # complex128 [m, 3, 3]
    v_source: float = 1.0
    load_scale: float = 1.0
    name: str = ""
    seed: int = 0
    # PV nodes (a reading beyond the paper, which defers them): generators
    # holding |V| of each present phase at v_set with injection p_gen
    node_type: np.ndarray | None = None  # int32 [n]: 1 PV, 2 PQ; None = all PQ
    v_set: np.ndarray | None = None  # float64 [n]: |V| of a PV node's phases
    p_gen: np.ndarray | None = None  # float64 [n, 3]: P injected per phase
    q_min: np.ndarray | None = None  # float64 [n, 3]: reactive limits of PV
    q_max: np.ndarray | None = None  # nodes' phases (pu); None = no limits

    @property
    def n_branch(self) -> int:
        return int(self.br_from.shape[0])

    def pv_mask(self) -> np.ndarray:
        """bool [n]: PV nodes."""
        if self.node_type is None:
            return np.zeros(self.n_node, dtype=bool)
        return np.asarray(self.node_type) == PV

    def with_loads(self, p_load, q_load) -> "ThreePhaseCase":
        return dataclasses.replace(
            self, p_load=np.ascontiguousarray(p_load, dtype=np.float64),
            q_load=np.ascontiguousarray(q_load, dtype=np.float64))


# ----------------------------------------------------------------------------
# topology helpers
# ----------------------------------------------------------------------------

def _geometric_spanning_tree(pos: np.ndarray, order: np.ndarray):
    """Each bus, in ``order``, links to its nearest already-placed bus.

    A uniform grid of cells keeps the nearest-neighbour search local, so this
    stays fast for 10^5 buses.
    """
    n = pos.shape[0]
    g = max(1, int(math.ceil(math.sqrt(n / 2.0))))
    cells: dict = {}
    edges = []
    for rank, b in enumerate(order):
        x, y = pos[b]
        cx, cy = min(int(x * g), g - 1), min(int(y * g), g - 1)
        if rank > 0:
            best, bestd = -1, np.inf
            ring = 0
            while True:
                for i in range(cx - ring, cx + ring + 1):
                    for j in range(cy - ring, cy + ring + 1):
                        if max(abs(i - cx), abs(j - cy)) != ring:
                            continue
                        for c in cells.get((i, j), ()):
                            d = (pos[c, 0] - x) ** 2 + (pos[c, 1] - y) ** 2
                            if d < bestd:
                                best, bestd = c, d
                # every unseen cell is at least ``ring / g`` away
                if best >= 0 and (ring / g) ** 2 >= bestd:
                    break
                ring += 1
                if ring > 2 * g + 2:
                    break
            edges.append((best, b))
        cells.setdefault((cx, cy), []).append(b)
    return edges


def mesh_topology(n: int, m: int, rng: np.random.Generator, k_near: int = 4):
    """Random geometric mesh: spanning tree + extra nearest-neighbour edges.

    Returns an int32 array [m, 2] of undirected edges (no duplicates, no
    self loops).  Extra edges are drawn without replacement from the pairs
    linking a bus to one of its ``k_near`` nearest neighbours.
    """
    if m < n - 1:
        raise ValueError("a connected grid needs m >= n - 1 branches")
    pos = rng.random((n, 2))
    order = rng.permutation(n)
    tree = _geometric_spanning_tree(pos, order)
    have = {(min(a, b), max(a, b)) for a, b in tree}
    from scipy.spatial import cKDTree  # spatial index only

    k = min(k_near + 1, n)
    _, nb = cKDTree(pos).query(pos, k=k)
    cand = set()
    for i in range(n):
        for j in nb[i, 1:]:
            j = int(j)
            e = (min(i, j), max(i, j))
            if e not in have:
                cand.add(e)
    cand = sorted(cand)
    need = m - (n - 1)
    if need > len(cand):
        raise ValueError(f"only {len(cand)} candidate extra edges for {need}")
    pick = rng.choice(len(cand), size=need, replace=False) if need else []
    edges = [(a, b) for a, b in tree] + [cand[i] for i in sorted(pick)]
    return np.asarray(edges, dtype=np.int32).reshape(-1, 2), pos


# ----------------------------------------------------------------------------
# single-phase transmission grids
# ----------------------------------------------------------------------------

def _dc_angle_spread(n, f, t, x, p_net):
    """Largest |theta_f - theta_t| of the linear (DC) estimate B' theta = P.

    Only sizes the load level of a drawn grid; the slack (bus 0) angle is 0.
    """
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    w = 1.0 / x
    B = sp.coo_matrix((np.r_[w, w, -w, -w], (np.r_[f, t, f, t], np.r_[f, t, t, f])),
                      shape=(n, n)).tocsc()
    th = np.zeros(n)
    if n > 1:
        th[1:] = spla.spsolve(B[1:, 1:], p_net[1:])
    return float(np.max(np.abs(th[f] - th[t])))


def transmission_case(n: int, m: int, n_pv: int, seed: int,
                      name: str = "", pv_share: float = 1.05,
                      max_angle: float = 0.3) -> SinglePhaseCase:
    """Meshed single-phase grid with the distributions of the 14-bus case.

    r ~ U[0.002, 0.02], x = r * U[5, 15], b ~ U[0, 0.05]; bus 0 is the slack
    at 1.0 pu; ``n_pv`` random PV buses with |V| ~ U[0.98, 1.05] and no load;
    every other bus is PQ with P ~ U[0.05, 0.5], Q = P * U[0.2, 0.5].  PV
    generation (weights U[0.5, 1.5]) sums to ``pv_share`` x the total load.

    On large meshes that load level has no power-flow solution (the slack
    alone absorbs the 5% surplus of thousands of buses), so loads and
    generation are scaled by one factor s <= 1 chosen so that a linear (DC)
    estimate of the largest angle across a branch is at most ``max_angle``
    radians; s is recorded in ``load_scale`` (it is 1 for the 14-bus case).
    Line charging is capped so that its total (at 1 pu) does not exceed the
    total reactive load: on a lightly loaded large grid the drawn charging
    lifts voltages (1.3 pu and more) beyond the reach of a flat-start Newton
    iteration, while normally loaded grids (the 14-bus case) keep it as drawn.
    """
    rng = np.random.default_rng(seed)
    edges, _ = mesh_topology(n, m, rng)
    r = rng.uniform(0.002, 0.02, m)
    x = r * rng.uniform(5.0, 15.0, m)
    b = rng.uniform(0.0, 0.05, m)
    bus_type = np.full(n, PQ, dtype=np.int32)
    bus_type[0] = SLACK
    pv = rng.choice(np.arange(1, n), size=n_pv, replace=False)
    bus_type[pv] = PV
    v_set = np.ones(n)
    v_set[pv] = rng.uniform(0.98, 1.05, n_pv)
    p_load = np.zeros(n)
    q_load = np.zeros(n)
    pq = np.flatnonzero(bus_type == PQ)
    p_load[pq] = rng.uniform(0.05, 0.5, pq.size)
    q_load[pq] = p_load[pq] * rng.uniform(0.2, 0.5, pq.size)
    w = rng.uniform(0.5, 1.5, n_pv)
    p_gen = np.zeros(n)
    p_gen[pv] = pv_share * p_load.sum() * w / w.sum()
    zipf = np.zeros((n, 3))
    zipf[:, 0] = 1.0
    spread = _dc_angle_spread(n, edges[:, 0], edges[:, 1], x, p_gen - p_load)
    scale = min(1.0, max_angle / spread) if spread > 0 else 1.0
    b_scale = min(1.0, scale * q_load.sum() / b.sum()) if b.sum() > 0 else 1.0
    return SinglePhaseCase(
        n_bus=n, bus_type=bus_type, v_set=v_set, p_gen=p_gen * scale,
        q_gen=np.zeros(n), p_load=p_load * scale, q_load=q_load * scale,
        zip=zipf, br_from=edges[:, 0].copy(), br_to=edges[:, 1].copy(),
        br_r=r, br_x=x, br_b=b * b_scale, name=name or f"mesh{n}", seed=seed,
        load_scale=scale)


def case_14bus(seed: int = 0) -> SinglePhaseCase:
    """14 buses, 20 branches (spanning tree + 7 extra edges), 4 PV, 9 PQ."""
    return transmission_case(14, 20, 4, seed, name="mesh14")


def case_10000bus(seed: int = 0) -> SinglePhaseCase:
    """10,000 buses, 13,500 branches (average degree 2.7), 2,000 PV."""
    return transmission_case(10_000, 13_500, 2_000, seed, name="mesh10000")


def case_2000bus(seed: int = 0) -> SinglePhaseCase:
    """2,000 buses, 2,700 branches, 400 PV: the batched-scenario topology."""
    return transmission_case(2_000, 2_700, 400, seed, name="mesh2000")


def scenario_loads(case: SinglePhaseCase, n_scen: int, seed: int,
                   sigma: float = 0.2, pv_share: float = 1.05):
    """Per-scenario loads: every bus load x lognormal(0, sigma).

    PV generation is rescaled per scenario so that it again sums to
    ``pv_share`` x that scenario's total load.  Returns (p_load, q_load,
    p_gen), each float64 [n_scen, n_bus].
    """
    rng = np.random.default_rng(seed)
    mult = rng.lognormal(0.0, sigma, (n_scen, case.n_bus))
    p_load = case.p_load[None, :] * mult
    q_load = case.q_load[None, :] * mult
    pv = case.bus_type == PV
    w = np.where(pv, case.p_gen, 0.0)
    w = w / w.sum()
    p_gen = np.where(pv[None, :], pv_share * p_load.sum(1, keepdims=True) * w[None, :],
                     case.p_gen[None, :])
    return (np.ascontiguousarray(p_load), np.ascontiguousarray(q_load),
            np.ascontiguousarray(p_gen))


def two_bus_case(p: float, q: float, r: float, x: float, b: float = 0.0,
                 pv: bool = False, v2: float = 1.0, v1: float = 1.0,
                 zip_frac=(1.0, 0.0, 0.0)) -> SinglePhaseCase:
    """Slack bus 0 feeding bus 1 through one branch.

    PQ form: bus 1 consumes p + jq.  PV form: bus 1 injects p at |V| = v2.
    """
    bt = np.array([SLACK, PV if pv else PQ], dtype=np.int32)
    return SinglePhaseCase(
        n_bus=2, bus_type=bt, v_set=np.array([v1, v2 if pv else 1.0]),
        p_gen=np.array([0.0, p if pv else 0.0]), q_gen=np.zeros(2),
        p_load=np.array([0.0, 0.0 if pv else p]),
        q_load=np.array([0.0, 0.0 if pv else q]),
        zip=np.array([[1.0, 0.0, 0.0], list(zip_frac)], dtype=np.float64),
        br_from=np.array([0], dtype=np.int32), br_to=np.array([1], dtype=np.int32),
        br_r=np.array([r]), br_x=np.array([x]), br_b=np.array([b]),
        name="two-bus")


# ----------------------------------------------------------------------------
# three-phase distribution feeders
# ----------------------------------------------------------------------------

def _phase_count(mask: int) -> int:
    return (mask & 1) + ((mask >> 1) & 1) + ((mask >> 2) & 1)


def feeder_case(n: int, seed: int, lateral_p: float = 0.2,
                reduced_p: float = 0.3, max_drop: float = 0.05,
                zip_frac=(0.5, 0.3, 0.2), name: str = "") -> ThreePhaseCase:
    """Seeded radial three-phase feeder with unbalanced laterals.

    Node k attaches to node k-1 (continuing the lateral, same phases) with
    probability 1 - ``lateral_p``; otherwise it starts a new lateral.  A new
    lateral is reduced with probability ``reduced_p``: it branches off a
    uniform earlier node and keeps a random 1- or 2-phase subset of that
    node's phases.  Otherwise it is three-phase and branches off a uniform
    earlier three-phase node.  Branch impedance: self
    (0.02+0.06j), mutual (0.005+0.02j), both times a length U[0.1, 1].
    Loads: P ~ U[0, 0.05], Q = P * U[0.2, 0.5] per present phase, ZIP
    fractions (P, I, Z) = ``zip_frac``.  The paper's literal load level has no
    solution on an 8,000-node tree, so all loads are scaled by one factor
    chosen so that a linear (DistFlow-style, self impedance only) estimate of
    the largest voltage drop equals ``max_drop``; the factor is recorded.
    """
    rng = np.random.default_rng(seed)
    parent = np.full(n, -1, dtype=np.int64)
    phases = np.zeros(n, dtype=np.uint8)
    phases[0] = 7
    three = [0]  # nodes carrying all three phases
    for k in range(1, n):
        if rng.random() >= lateral_p:
            p = k - 1
            ph = int(phases[p])
        elif rng.random() >= reduced_p:
            # new three-phase lateral: branch off a three-phase node
            p = int(three[int(rng.integers(0, len(three)))])
            ph = 7
        else:
            # new reduced lateral: a 1- or 2-phase subset of any node's phases
            p = int(rng.integers(0, k))
            present = [bit for bit in (1, 2, 4) if int(phases[p]) & bit]
            size = min(int(rng.integers(1, 3)), len(present))
            if size == len(present) and len(present) > 1:
                size = len(present) - 1
            chosen = rng.choice(present, size=size, replace=False)
            ph = int(sum(int(c) for c in chosen))
        parent[k] = p
        phases[k] = ph
        if ph == 7:
            three.append(k)
    m = n - 1
    br_from = parent[1:].astype(np.int32)
    br_to = np.arange(1, n, dtype=np.int32)
    ell = rng.uniform(0.1, 1.0, m)
    zs, zm = 0.02 + 0.06j, 0.005 + 0.02j
    base = np.full((3, 3), zm, dtype=np.complex128)
    np.fill_diagonal(base, zs)
    br_z = ell[:, None, None] * base[None, :, :]
    br_ph = phases[1:].copy()
    pl = np.zeros((n, 3))
    ql = np.zeros((n, 3))
    for s in range(3):
        has = (phases >> s) & 1
        has[0] = 0
        draw = rng.uniform(0.0, 0.05, n)
        pl[:, s] = np.where(has == 1, draw, 0.0)
        ql[:, s] = pl[:, s] * rng.uniform(0.2, 0.5, n)
    # linear drop estimate: downstream load sums along the tree, per phase
    down_p = pl.copy()
    down_q = ql.copy()
    for k in range(n - 1, 0, -1):
        down_p[parent[k]] += down_p[k]
        down_q[parent[k]] += down_q[k]
    drop = np.zeros((n, 3))
    for k in range(1, n):
        e = k - 1
        rr = ell[e] * zs.real
        xx = ell[e] * zs.imag
        drop[k] = drop[parent[k]] + rr * down_p[k] + xx * down_q[k]
    worst = float(drop.max())
    scale = max_drop / worst if worst > 0 else 1.0
    zipf = np.tile(np.asarray(zip_frac, dtype=np.float64), (n, 1))
    return ThreePhaseCase(
        n_node=n, source=0, phases=phases, p_load=pl * scale, q_load=ql * scale,
        zip=zipf, br_from=br_from, br_to=br_to, br_phases=br_ph, br_z=br_z,
        v_source=1.0, load_scale=scale, name=name or f"feeder{n}", seed=seed)


def with_pv_nodes(case: ThreePhaseCase, count: int, seed: int, p_range=(0.005, 0.02),
                  v_set: float = 1.0) -> ThreePhaseCase:
    """The feeder with ``count`` three-phase nodes (not the source) turned
    into PV generators: P per phase ~ U[p_range] (times the load scale),
    |V| held at ``v_set`` on every phase."""
    rng = np.random.default_rng(seed)
    cand = np.flatnonzero((case.phases == 7) & (np.arange(case.n_node) != case.source))
    pick = rng.choice(cand, size=min(count, cand.size), replace=False)
    node_type = np.full(case.n_node, PQ, dtype=np.int32)
    node_type[pick] = PV
    vset = np.ones(case.n_node)
    vset[pick] = v_set
    pg = np.zeros((case.n_node, 3))
    pg[pick] = rng.uniform(p_range[0], p_range[1], (pick.size, 3)) * case.load_scale * 20.0
    return dataclasses.replace(case, node_type=node_type, v_set=vset, p_gen=pg,
                               name=case.name + f"_pv{pick.size}")


def with_q_limits(case: SinglePhaseCase, seed: int, q_range=(0.5, 3.0)) -> SinglePhaseCase:
    """The grid with reactive generation limits at every bus (read at PV
    buses only): q_max ~ U[q_range] and q_min = -U[q_range] pu, drawn
    independently."""
    rng = np.random.default_rng(seed)
    qmax = rng.uniform(q_range[0], q_range[1], case.n_bus)
    qmin = -rng.uniform(q_range[0], q_range[1], case.n_bus)
    return dataclasses.replace(case, q_min=qmin, q_max=qmax, name=case.name + "_qlim")


def with_phase_q_limits(case: ThreePhaseCase, seed: int, q_max_range=(0.01, 0.08),
                        q_min_range=(0.0, 0.004)) -> ThreePhaseCase:
    """The feeder with reactive limits on every phase slot (read at PV
    nodes only), in units of the load scale x 20 (the scale of the PV
    generation of with_pv_nodes): q_max ~ U[q_max_range], q_min ~
    -U[q_min_range], drawn independently."""
    rng = np.random.default_rng(seed)
    unit = case.load_scale * 20.0
    qmax = rng.uniform(q_max_range[0], q_max_range[1], (case.n_node, 3)) * unit
    qmin = -rng.uniform(q_min_range[0], q_min_range[1], (case.n_node, 3)) * unit
    return dataclasses.replace(case, q_min=qmin, q_max=qmax, name=case.name + "_qlim")


def case_feeder8000(seed: int = 0) -> ThreePhaseCase:
    """8,000 nodes (24,000 phase slots), 30% reduced-phase laterals."""
    return feeder_case(8_000, seed, name="feeder8000")


def feeder_scenario_loads(case: ThreePhaseCase, n_scen: int, seed: int,
                          sigma: float = 0.2):
    """Per-scenario three-phase loads: each node's load x lognormal(0, sigma)."""
    rng = np.random.default_rng(seed)
    mult = rng.lognormal(0.0, sigma, (n_scen, case.n_node, 1))
    return (np.ascontiguousarray(case.p_load[None] * mult),
            np.ascontiguousarray(case.q_load[None] * mult))


# ----------------------------------------------------------------------------
# serving stream
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Request:
    t_arrive: float  # seconds from stream start
    kind: str  # "transmission" or "feeder"
    topo: int  # index into the pool of that kind
    load_seed: int  # seed of this request's per-bus load multipliers


def topology_pool(kind: str, count: int, seed: int, n_min: int, n_max: int):
    """``count`` seeded cases with log-uniform sizes in [n_min, n_max]."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), count))
    out = []
    for i, s in enumerate(sizes.astype(int)):
        if kind == "transmission":
            n = int(s)
            out.append(transmission_case(n, int(round(1.35 * n)), n // 5,
                                         seed * 1000 + i))
        else:
            out.append(feeder_case(int(s), seed * 1000 + i))
    return out


def serving_stream(seed: int, rate: float = 2000.0, duration: float = 60.0,
                   share_transmission: float = 0.7, pool_size: int = 64):
    """Poisson arrivals: (time, kind, pool index, load seed) per request."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        kind = "transmission" if rng.random() < share_transmission else "feeder"
        out.append(Request(t, kind, int(rng.integers(0, pool_size)),
                           int(rng.integers(0, 2**31 - 1))))
    return out
