/*
 * pf.h -- C ABI of a GB300-native Newton power-flow library.
 *
 * The library implements the hot path of the ExaGridPF method (Wang, Bachan,
 * Chan, arXiv 1711.10579): the Newton iteration of AC power flow.
 *
 *   single phase (Sec. II.A): polar Newton-Raphson.  Each iteration forms the
 *     power mismatch Delta P, Delta Q (Eq. 8-9) from I = Y V (Eq. 1) and
 *     S = V conj(I) (the quantity of Eq. 5-7), assembles the Jacobian of
 *     Eq. 10 and solves for (Delta delta, Delta |V|);
 *   three phase (Sec. II.B): current-injection Newton.  Each iteration forms
 *     Delta I = I_sp - Y V (Eq. 12-19) and solves the 6x6-block system of
 *     Eq. 21-23 for the rectangular voltage correction (Eq. 20).
 *
 * The Newton correction is solved either by a numeric sparse LU
 * refactorisation on a symbolic pattern computed once per topology plus
 * level-scheduled triangular solves (Newton-Raphson, Sec. III.A) or by
 * restarted GMRES with an ILU(0) preconditioner (Newton-Krylov, Sec. III.B).
 * Every step of the iteration runs in this library's own CUDA kernels on one
 * GPU; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *  - The return value is a pf_status; negative values are errors.  No call
 *    aborts or throws across the ABI.  pf_last_error() returns a message for
 *    the last failing call of the calling thread.
 *  - Pointers named h_* or without prefix are HOST memory owned by the caller;
 *    the library copies inputs during the call and writes outputs only before
 *    returning.  Pointers named d_* are DEVICE memory on the context's GPU,
 *    owned by the caller; calls taking d_* pointers and a stream are
 *    asynchronous on that stream.
 *  - Arrays are dense, C order, float64 unless stated.  "Per bus" arrays have
 *    n_bus entries in the caller's bus numbering; three-phase "per slot"
 *    arrays have 3 * n_bus entries, slot 3*i + s for phase s (a=0, b=1, c=2)
 *    of node i, the phase indexing of Sec. II.B.
 *  - Units are per unit (pu) and radians.
 */
#ifndef PF_H
#define PF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pf_ctx_s* pf_ctx;   /* one GPU, its streams and serving runtime */
typedef struct pf_case_s* pf_case; /* one topology: Ybus, symbolic patterns, warm start */
typedef uint64_t pf_ticket;        /* handle of a submitted (served) solve */

enum pf_status {
  PF_OK = 0,
  PF_PENDING = 1,         /* pf_poll: the solve has not finished yet */
  PF_ERR_INVALID = -1,    /* bad argument or case description */
  PF_ERR_NOMEM = -2,      /* device or host allocation failed / over budget */
  PF_ERR_MAXITER = -3,    /* Newton stopped at max_iter above tolerance */
  PF_ERR_DIVERGED = -4,   /* mismatch became non-finite or exploded */
  PF_ERR_SINGULAR = -5,   /* zero or non-finite pivot block in the factorisation */
  PF_ERR_TIMEOUT = -6,    /* a bounded wait ran out */
  PF_ERR_BUSY = -7,       /* serving queue full; retry later */
  PF_ERR_CUDA = -8,       /* a CUDA runtime call failed */
  PF_ERR_UNSUPPORTED = -9 /* valid request the library does not implement */
};

enum pf_bus_type { PF_SLACK = 0, PF_PV = 1, PF_PQ = 2 };
enum pf_method { PF_NR = 0, PF_NK = 1 };
enum pf_precision { PF_FP64 = 0, PF_MIXED = 1 };
enum pf_kind { PF_SINGLE_PHASE = 1, PF_THREE_PHASE = 3 };

/*
 * Case description (problem statement of Sec. II: P and Q drawn or injected
 * per bus and phase, V magnitude and angle per bus and phase out).
 *
 * kind == PF_SINGLE_PHASE:
 *   bus_type[n]   pf_bus_type; exactly one PF_SLACK.
 *   v_set[n]      |V| set point of the slack and PV buses (ignored for PQ).
 *   p_gen[n], q_gen[n]    generation (q_gen used for PQ buses only).
 *   p_load[n], q_load[n]  load at |V| = 1 pu.
 *   zip[n][3]     load fractions (constant power, constant current,
 *                 constant impedance) of Eq. 14-15; NULL = constant power.
 *                 Specified injection = gen - load(|V|)  (Eq. 12-15).
 *   br_from/br_to[m], br_r/br_x/br_b[m]: pi-model branches, series r + jx,
 *                 total line charging b split b/2 per end (Eq. 2-3).
 *   q_min[n], q_max[n]  optional reactive generation limits of PV buses
 *                 (enforced with pf_opts.q_limits).
 * kind == PF_THREE_PHASE (Sec. II.B; PV nodes are a reading beyond the
 * paper, which defers them):
 *   phases[n]     uint8 bit mask of present phases (a=1, b=2, c=4).
 *   bus_type[n]   optional: PF_PV marks a node whose generator holds |V| of
 *                 every present phase at v_set[n] while injecting
 *                 p_gen[n][3] per phase (its reactive injection is solved
 *                 for); other nodes PF_PQ.  NULL = no PV nodes.
 *   source        index of the ideal balanced source node (slack).
 *   v_source      its magnitude; phase angles 0, -120, +120 degrees.
 *   p_load[3n], q_load[3n]  wye load per slot at |V| = 1 pu.
 *   zip[n][3]     ZIP fractions per node (NULL = constant power).
 *   br_from/br_to[m], br_phases[m] (mask of phases on the branch, a subset
 *                 of both end nodes' phases), br_z[m][3][3][2] the series
 *                 impedance matrix (re, im); the branch admittance is the
 *                 inverse of its submatrix over the branch's phases (Eq. 11).
 *   q_min[3n], q_max[3n]  optional reactive limits per phase slot of PV
 *                 nodes (enforced with pf_opts.q_limits).
 * Unused fields may be NULL.
 */
typedef struct {
  int kind;
  int n_bus;
  int n_branch;
  const int32_t* bus_type;
  const double* v_set;
  const double* p_gen;
  const double* q_gen;
  const double* p_load;
  const double* q_load;
  const double* zip;
  const int32_t* br_from;
  const int32_t* br_to;
  const double* br_r;
  const double* br_x;
  const double* br_b;
  const uint8_t* phases;
  int source;
  double v_source;
  const uint8_t* br_phases;
  const double* br_z;
  /* optional reactive generation limits (pu; both or neither; q_min <= q_max;
     read when pf_opts.q_limits is set): single phase per bus [n], read at
     PV buses; three phase per node and phase [n][3], read at PV nodes */
  const double* q_min;
  const double* q_max;
} pf_case_desc;

typedef struct {
  int method;         /* pf_method, default PF_NR */
  int precision;      /* pf_precision, default PF_MIXED */
  double tol;         /* stop when the power-mismatch infinity norm <= tol (pu); default 1e-8 */
  int max_iter;       /* Newton iterations; default 30 */
  int refine_steps;   /* NR + PF_MIXED: FP64 iterative-refinement steps per solve; default 1 */
  double refine_below; /* ... applied once the mismatch norm is <= this (pu); default 1e-3 */
  int gmres_restart;  /* NK: Krylov subspace size m of GMRES(m); default 30 */
  int gmres_max_iter; /* NK: inner iterations per Newton step; default 300 */
  double gmres_rtol;  /* NK: inner relative-residual floor; default 1e-6 */
  int warm_start;     /* 1 = start from the case's last converged voltages */
  int cluster_size;   /* single-solve launch: CTAs per cluster (0 = autotuned) */
  int block_threads;  /* threads per CTA (0 = autotuned) */
  int scen_per_cta;   /* batched launch: scenarios per CTA (0 = autotuned) */
  int nk_fallback;    /* PF_NK through pf_solve / pf_solve_batch: redo every
                         scenario that ends without convergence (max_iter,
                         divergence, singular preconditioner) with PF_NR from
                         a flat start, as Sec. III.B warns NK may fail;
                         default 1 */
  int kernel_by_kernel; /* batched PF_NR: 1 = launch the phase kernels one by one
                           instead of as one CUDA graph (for profilers, which
                           cannot look inside a graph with a conditional node);
                           default 0 */
  int krylov;         /* PF_NK inner solver: 0 = restarted GMRES(gmres_restart)
                         (default), 1 = BiCGSTAB (the method of Sec. III.B;
                         needs gmres_restart >= 7 for its work vectors) */
  int q_limits;       /* cases with q_min/q_max: 1 = enforce the reactive limits.
                         After a converged solve every PV bus whose generator Q
                         (Q_i of Eq. 7 plus its own reactive load) -- three
                         phase: every PV phase slot whose reactive injection
                         Q_g -- is outside [q_min, q_max] is held at the limit
                         it crossed (|V| free), and the scenario is solved again
                         from its last voltages; rounds end when nothing
                         violates (held buses and slots stay held; at most 64
                         rounds, then PF_ERR_MAXITER).  The block pattern is the
                         same either way, so no symbolic step is repeated.
                         The call waits for the device between rounds.
                         Default 0 (limits ignored) */
  double refine_stall; /* NR + PF_MIXED: the FP64 refinement of a step is taken
                          only where the FP32 factors hold convergence back:
                          the mismatch is <= refine_below and the last Newton
                          step cut it by less than 1 / refine_stall (norm_k >
                          refine_stall x norm_(k-1)).  0 = whenever the
                          mismatch is <= refine_below.  Default 0.1 */
} pf_opts;

typedef struct {
  int status;            /* pf_status of this solve */
  int iterations;        /* Newton iterations performed (solves of Eq. 10 / 22) */
  int linear_iterations; /* NK: total GMRES iterations; NR batch (B >= 2):
                            triangular-solve passes (one per Newton step
                            plus one per FP64 refinement) */
  int fallback;          /* 1: a PF_NK solve that ended without convergence
                            was redone with PF_NR (opts.nk_fallback) */
  double mismatch;       /* final infinity norm of the power mismatch (pu) */
  double max_step;       /* infinity norm of the last Newton correction */
  double solve_us;       /* device time of the solve, microseconds */
  int q_switched;        /* opts.q_limits: PV buses (three phase: PV phase
                            slots) held at a reactive limit */
  int q_rounds;          /* opts.q_limits: solves the scenario needed (1 + the
                            last round that switched one of its buses) */
} pf_info;

/* Sizes produced by the symbolic phase (per method's ordering). */
typedef struct {
  int kind, n_bus, block_size, n_unknowns;
  long long nnz_y;        /* block entries of Ybus (incl. diagonal) */
  long long nnz_lu;       /* block entries of L+U (NR, after fill) */
  long long n_updates;    /* block multiply-subtracts of one NR factorisation */
  int levels_factor;      /* level sets of the NR factorisation / forward solve */
  int levels_backward;    /* level sets of the NR backward solve */
  int levels_ilu;         /* level sets of ILU(0) (NK ordering) */
  int levels_ilu_backward;
  long long device_bytes; /* device memory held by the case (symbolic data) */
  long long bytes_per_scenario; /* workspace per solved scenario */
} pf_case_stats;

/*
 * Host-only analysis (no GPU needed): validates the description, assembles
 * Ybus and runs the symbolic phase exactly as pf_create_case does, and fills
 * *out (device_bytes = what pf_create_case would hold).  Lets a caller size a
 * case before creating it.  Errors: PF_ERR_INVALID.
 */
int pf_analyze(const pf_case_desc* desc, pf_case_stats* out);
/*
 * Host-only: Ybus of Eq. 2-3 / Eq. 11 in the caller's numbering as block CSR.
 * Call with rowptr == NULL to get *nnz only; otherwise rowptr[n+1],
 * col[nnz], val[nnz][2*ybs*ybs] (re, im interleaved, ybs = 1 or 3) are
 * filled.
 */
int pf_ybus(const pf_case_desc* desc, int64_t* nnz, int32_t* rowptr, int32_t* col,
            double* val);
/*
 * Host-only: symbolic pattern of a method (PF_NR: minimum-degree ordering
 * with LU fill; PF_NK: reverse Cuthill-McKee ordering, Ybus pattern for
 * ILU(0)).  perm[n] maps new to caller numbering; rowptr[n+1], col[nnz] is
 * the factor's block pattern in the new numbering (nnz = nnz_lu or nnz_y of
 * pf_analyze); flevel[n] / blevel[n] the level of each new row in the
 * factorisation / forward schedule and in the backward schedule.
 */
int pf_symbolic(const pf_case_desc* desc, int method, int32_t* perm, int32_t* rowptr,
                int32_t* col, int32_t* flevel, int32_t* blevel);

/*
 * Host-only: the packed schedule the kernels run for a method's symbolic
 * pattern (in the new numbering of pf_symbolic; entries index its col[]),
 * for tests and diagnostics.  sizes[6] = {n, factor levels L, backward
 * levels, factor items F, targets T, con pairs C}; with any array NULL only
 * what is given is written.  fac_ptr[L+1] / tgt_ptr[L+1]: items and targets
 * of level l; fac_rec[F][4] = {entry, pivot k, diagonal entry of k, 0}
 * (Sec. III.A fan-out step 1: U_kk^-1, or L_ik = A_ik U_kk^-1);
 * tgt_rec[T][4] = {entry | 2^30 when a fill entry starts from zero, first L
 * entry, first U entry, start of its other (L, U) pairs in con or -1}
 * (step 2: A -= sum L U); con[C][2], lists ended by (-1, -1);
 * flev_ptr[L+1] / fwd_rec[n][4] = {row, first entry, diagonal entry, 0} of
 * the forward sweep by level; blev_ptr / bwd_rec[n][4] = {row, first U entry,
 * end, 0} of the backward sweep.
 */
int pf_schedule(const pf_case_desc* desc, int method, int64_t* sizes, int32_t* fac_ptr,
                int32_t* fac_rec, int32_t* tgt_ptr, int32_t* tgt_rec, int32_t* con,
                int32_t* flev_ptr, int32_t* fwd_rec, int32_t* blev_ptr, int32_t* bwd_rec);

/* Fill *opts with the defaults listed in pf_opts. */
void pf_opts_default(pf_opts* opts);
/* Message of the last failing call on this thread ("" if none). */
const char* pf_last_error(void);
/* Name of a pf_status value. */
const char* pf_status_str(int status);

/*
 * Context on CUDA device `device`.  hbm_budget_bytes bounds the device memory
 * the serving runtime admits requests into (0 = 80% of free memory).
 */
int pf_ctx_create(int device, size_t hbm_budget_bytes, pf_ctx* out);
int pf_ctx_destroy(pf_ctx ctx);

/*
 * Copies and validates the description, assembles Ybus (Eq. 2-3 or 11),
 * computes orderings (minimum degree for the LU of Sec. III.A; reverse
 * Cuthill-McKee for the Krylov solver, Sec. III.B), the block fill pattern,
 * level sets and update lists, and uploads them.  Errors: PF_ERR_INVALID
 * (no or several slack buses, indices out of range, disconnected grid,
 * non-finite values, PV in three phase, zero impedance), PF_ERR_NOMEM,
 * PF_ERR_CUDA.
 */
int pf_create_case(pf_ctx ctx, const pf_case_desc* desc, pf_case* out);
int pf_destroy_case(pf_case c);
int pf_case_get_stats(pf_case c, pf_case_stats* out);

/*
 * One solve of the case as described (flat start or warm start).
 * vmag, vang: per bus (single phase) or per slot (three phase), host.
 * info: host.  Returns PF_OK if the solve ran (its own outcome is in
 * info->status) or an error if it could not run.
 */
int pf_solve(pf_case c, const pf_opts* opts, double* vmag, double* vang,
             pf_info* info);

/*
 * B scenarios of one topology solved together over the shared symbolic
 * pattern (Newton-Raphson: phase kernels in one CUDA graph whose loop ends on
 * the device when no scenario runs; Newton-Krylov: one persistent launch).
 * Scenario b uses p_load[b][*], q_load[b][*] (per bus or per slot; a load
 * scale per bus and scenario is these arrays scaled) and, single phase
 * only, p_gen[b][n]; NULL = the case's own values.  Outputs vmag[b][*],
 * vang[b][*], info[b].  Host arrays; the call blocks until done.
 */
int pf_solve_batch(pf_case c, int B, const double* p_load, const double* q_load,
                   const double* p_gen, const pf_opts* opts, double* vmag,
                   double* vang, pf_info* info);

/*
 * Device-resident form of pf_solve_batch, asynchronous on `stream`
 * (a cudaStream_t, NULL = legacy default stream).  d_info receives B pf_info
 * records in device memory.  B = 1 runs the single-solve cluster launch.
 * The device arrays must stay valid until the stream passes this call.
 */
int pf_solve_batch_device(pf_case c, int B, const double* d_p_load,
                          const double* d_q_load, const double* d_p_gen,
                          const pf_opts* opts, double* d_vmag, double* d_vang,
                          pf_info* d_info, void* stream);

/*
 * Serving: queue one solve of case c with its own loads (host arrays as in
 * pf_solve_batch with B = 1; NULL = the case's own).  The runtime admits
 * queued requests onto the GPU as job slots and device memory (the context's
 * budget) allow, so requests overlap on the device (several cases of
 * different sizes in one group launch; see pf_serve_get_stats).  Warm start
 * from the case's last result if opts->warm_start: a served solve reads the
 * case's warm-start voltages only while no other served solve of the case
 * writes them, and writes them only when it is the case's only served solve
 * on the GPU.  A Newton-Krylov request that ends without convergence is
 * solved again with Newton-Raphson when opts->nk_fallback (info.fallback = 1),
 * as in pf_solve.  Sixteen or more queued Newton-Raphson requests of one case
 * with the same tol, max_iter, precision and refinement options and their own
 * p_load and q_load (and all or none p_gen) are coalesced into one batched
 * solve of up to 4,864 scenarios (the pf_solve_batch kernels; a flat start,
 * warm_start ignored).  PF_ERR_BUSY if the queue is full.  Thread safe.
 */
int pf_submit(pf_ctx ctx, pf_case c, const double* p_load, const double* q_load,
              const double* p_gen, const pf_opts* opts, pf_ticket* out);
/*
 * B requests of case c at once, queued together (so that they can be
 * coalesced into one batched solve): request k has the loads
 * p_load[k][...], q_load[k][...], p_gen[k][...] (host arrays laid out as in
 * pf_solve_batch; NULL = the case's own) and the ticket out[k].  Either all
 * B are queued or none (PF_ERR_BUSY when the queue cannot take them).
 * Thread safe.
 */
int pf_submit_batch(pf_ctx ctx, pf_case c, int B, const double* p_load, const double* q_load,
                    const double* p_gen, const pf_opts* opts, pf_ticket* out);
/*
 * PF_PENDING while the request is queued or running; otherwise copies the
 * result into vmag/vang/info (host, may be NULL), releases the ticket and
 * returns PF_OK.  PF_ERR_INVALID for an unknown ticket.  Thread safe.
 */
int pf_poll(pf_ctx ctx, pf_ticket t, double* vmag, double* vang, pf_info* info);
/* Block until every submitted request has finished (bounded by timeout_ms). */
int pf_drain(pf_ctx ctx, int timeout_ms);
/*
 * Counters of the context's serving runtime since it started (all zero before
 * the first pf_submit).  Newton-Raphson requests (no reactive limits, default
 * launch shape) run as group launches: one launch solves several queued
 * requests of any cases and sizes, one CTA each (a cluster of 2 CTAs for
 * grids of 4,000 buses or feeders of 2,000 nodes and more, of 4 CTAs from
 * 16,000 buses or 5,000 nodes, of 8 CTAs from 40,000 buses or 12,000 nodes),
 * and each request retires when its own solve ends.  Runs of queued requests of one case are coalesced into batched
 * solves (pf_submit).  Newton-Krylov requests and requests with reactive
 * limits run as one launch each.
 */
typedef struct {
  uint64_t requests;        /* requests finished on the GPU */
  uint64_t group_launches;  /* group launches issued */
  int max_group;            /* most requests in one group launch */
  int peak_running;         /* most requests on the GPU at the same time */
  uint64_t batch_launches;  /* coalesced batched solves issued */
  int max_batch;            /* most requests in one coalesced batch */
} pf_serve_stats;
int pf_serve_get_stats(pf_ctx ctx, pf_serve_stats* out);

/*
 * Inspection entry points: single steps of the iteration on the GPU, for
 * parity tests and diagnostics.  vmag, vang: host, per bus / per slot.
 *
 * pf_eval_mismatch: single phase mis[n][2] = (Delta P, Delta Q) of Eq. 8-9
 *   (0 where the bus has no such equation: slack both, PV Delta Q);
 *   three phase mis[n][6] = Delta I of Eq. 16-19 in the order
 *   [Im a, b, c, Re a, b, c] (0 on absent phases and the source).
 */
int pf_eval_mismatch(pf_case c, const double* vmag, const double* vang,
                     double* mis);
/*
 * pf_eval_jacobian: Jacobian blocks on the Ybus block pattern returned by
 * pf_case_pattern (caller's numbering, rows = equations of bus i, columns =
 * unknowns of bus j, row-major bs x bs, bs = 2 or 6).  Single phase block =
 * [[dP/d delta, dP/d|V|], [dQ/d delta, dQ/d|V|]] (Eq. 10); three phase
 * block = Eq. 21 / 23.  Rows and columns without an unknown (slack, PV |V|,
 * absent phase, source) are zero except a 1 on the diagonal.
 */
int pf_eval_jacobian(pf_case c, const double* vmag, const double* vang,
                     double* blocks);
/* Block pattern of Ybus in the caller's numbering: rowptr[n+1], col[nnz_y]. */
int pf_case_pattern(pf_case c, int32_t* rowptr, int32_t* col);
/*
 * pf_newton_step: one solve J dx = F at the given voltage with the method and
 * precision of opts; dx[n][bs] per bus in the unknown order of Eq. 10
 * (delta, |V|) or Eq. 20 (Re a,b,c, Im a,b,c), 0 where no unknown.
 * info->linear_iterations reports GMRES iterations for PF_NK.
 */
int pf_newton_step(pf_case c, const pf_opts* opts, const double* vmag,
                   const double* vang, double* dx, pf_info* info);

/*
 * Newton-Raphson solve of one scenario that allocates nothing.  (The paper
 * has no counterpart: this entry point exists for callers of the library.)
 *
 * Some callers cannot allocate device memory once they are running: a
 * real-time grid-control loop with a fixed latency budget must not call
 * cudaMalloc / cudaFree, which can block on the whole device, and a host
 * application that owns the GPU's memory through its own pool may forbid any
 * other allocation.  For them this call takes its workspace from a fixed
 * array in device memory compiled into the library (32 MiB, held by every
 * GPU that loads the library until the process exits), and calls no
 * cudaMalloc, cudaFree or other allocating routine.  The case must have been
 * created beforehand (pf_create_case allocates).
 *
 * Arguments as pf_solve_batch_device with B = 1: d_p_load, d_q_load,
 * d_p_gen (NULL = the case's own), d_vmag, d_vang, d_info are device
 * pointers; the call is asynchronous on `stream`.  opts->method must be
 * PF_NR and block_threads / scen_per_cta 0; opts->q_limits on a case with
 * reactive limits is PF_ERR_UNSUPPORTED (the rounds wait for the device and
 * keep per-scenario state).  A case whose workspace does not
 * fit the array is rejected with PF_ERR_INVALID and a message giving both
 * sizes (with the LU values, about 230 bytes per bus in mixed precision and
 * 350 in FP64 on grids as dense as the 10,000-bus test grid).  The lane
 * tables of the launch are uploaded by pf_create_case, so a call makes no
 * host-to-device copy.
 *
 * Like pf_solve, a converged call stores its voltages in the case as the warm
 * start that later calls with opts->warm_start read.  That state is shared
 * with pf_solve and with served requests of the same case: warm-started
 * solves of one case that overlap on the GPU may start from a mix of two
 * solutions, so a caller that warm-starts must not let them overlap.
 *
 * The first call on a device also looks up the array's device address (a
 * host-side query, cached for later calls).  Every call shares the array and the
 * kernel writes all it later reads, so a call does not depend on what an
 * earlier call left there; calls that overlap on the GPU (other streams, or
 * other host threads) race on it and must be serialised by the caller.
 */
int pf_solve_noalloc(pf_case c, const pf_opts* opts, const double* d_p_load,
                     const double* d_q_load, const double* d_p_gen, double* d_vmag,
                     double* d_vang, pf_info* d_info, void* stream);

/*
 * Branch power flows of given bus voltages (the problem statement of Sec. I
 * asks for voltages and branch flows).  Branch models as in Ybus: Eq. 2-3
 * (pi model: series y = 1/(r + jx), half the line charging j b/2 at each end)
 * and Eq. 11 (three phase: y = inverse of the series impedance over the
 * branch's phases).  For scenario b and branch k (the case's branch order),
 * the power leaving the from bus into the branch, s_from = V_f conj(I_f),
 * I_f = y (V_f - V_t) + j b/2 V_f, and leaving the to bus, s_to likewise;
 * s_from + s_to is the branch loss.  vmag, vang: [B][n] (single phase) or
 * [B][n][3] (three phase) as pf_solve_batch writes them.  Outputs [B][m]
 * or [B][m][3] (p_from, q_from, p_to, q_to, pu) and loss[B][2] (total P and
 * Q loss of the scenario, summed on the device in a fixed order).  Host
 * arrays, caller-owned; blocking; PF_ERR_INVALID on null arguments.  Not
 * in the Newton iteration: a post-step over solved voltages.
 */
int pf_branch_flows(pf_case c, int B, const double* vmag, const double* vang, double* p_from,
                    double* q_from, double* p_to, double* q_to, double* loss);

/*
 * Autotuner for batched solves (B >= 2): runs B copies of the case's own
 * scenario with each candidate launch shape (scenarios per CTA 1, 2, 4, 8,
 * and 16 for PF_NR when B >= 32; threads per CTA 128, 256, 512), times them
 * with CUDA events and stores the fastest in the case for (B, method,
 * precision).  A PF_NR batch runs its factorisation and its triangular
 * sweeps as separate launches; each gets the shape with the least time of
 * its own phase.  Later batch solves of that B with scen_per_cta == 0 and
 * block_threads == 0 use the stored shapes; *opts (in: method, precision;
 * out: the chosen shape, for PF_NR that of the factorisation, which alone
 * also applies to the sweeps when passed back explicitly).  Without tuning,
 * a batch uses about one CTA per SM (at most 8 scenarios per CTA).
 * Blocking; allocates the batch workspace.
 */
int pf_autotune(pf_case c, int B, pf_opts* opts);

/*
 * Launch shape a solve of B scenarios with these options would use:
 * grid CTAs, CTAs per cluster, threads per CTA, scenarios per cluster.
 */
int pf_launch_config(pf_case c, const pf_opts* opts, int B, int* grid, int* cluster,
                     int* threads, int* scen_per_cluster);

/*
 * A solve of B copies of the case's own scenario with per-phase device timers
 * (diagnostics).  phase_us[8] (host) receives microseconds spent in: set-up,
 * mismatch + Jacobian, stop test, factorisation, triangular solves,
 * right-hand sides and refinement residuals, voltage update, output -- as
 * seen by one thread of the first CTA of the launch between its barriers,
 * summed over the Newton iterations.  info: B records (host, may be NULL).
 */
int pf_profile_solve(pf_case c, int B, const pf_opts* opts, double* phase_us, pf_info* info);

#ifdef __cplusplus
}
#endif

#endif /* PF_H */
