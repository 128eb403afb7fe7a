// Views of device-resident data shared by the host driver and the kernels.
#pragma once

#include <cstdint>

#include "../../include/pf.h"

namespace pf {

// Running status of a scenario inside a solve.
constexpr int kRunning = PF_PENDING;
// Scenario bus type of a PV bus switched to PQ at a reactive limit.
constexpr int kPQLimit = 3;
// Krylov basis vectors per GMRES cycle (restart m <= kMaxJ - 1).
constexpr int kMaxJ = 64;
// Half width of the sine / cosine table: angles j 2^-7 for |j| <= kTrigHalf.
// A target record whose entry index carries this bit is the first update of
// a fill entry of the factor: it starts from zero (no Jacobian value is
// written there and none is read).
constexpr int kFillFirst = 1 << 30;
constexpr int kTrigHalf = 512;  // = fx::kHalf (fixtrig.h)
// Size of the fixed scratch array used by pf_solve_noalloc.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;

// Symbolic structure and bus data of one case for one ordering (device
// pointers, new numbering).  Shared by every scenario of the case.
struct DevSys {
  int kind;  // PF_SINGLE_PHASE or PF_THREE_PHASE
  int n;     // buses / nodes
  // Ybus: complex scalars (single phase) or 3x3 complex blocks, (re, im)
  const int* y_rowptr;
  const int* y_col;
  const double* y_val;
  const float2* y32;  // single phase: FP32 copy of y_val for the Jacobian
  const long long* trig;  // (cos jh, sin jh) x 2^62, h = 2^-7, j = -kTrigHalf..kTrigHalf
  const float* zip32;   // single phase: FP32 copy of zip for the Jacobian
  // factor pattern (L, diagonal, U per row) and its maps
  const int* lu_rowptr;
  const int* lu_col;
  const int* lu_diag;
  const int* lu2y;
  // fan-out factorisation schedule (see Symbolic)
  const int* fac_ptr;
  const int* fac_items;
  const int* tgt_ptr;
  const int* tgt_entry;
  const int* tgt_cptr;
  const int* con_l;
  const int* con_u;
  // level schedules, and lanes per row for the launch's shape
  const int* flev_ptr;
  const int* flev_rows;
  int nflev;
  const int* blev_ptr;
  const int* blev_rows;
  int nblev;
  int fac_solo_from;  // factor levels >= this run in CTA 0 alone (single solves)
  // packed records: forward / backward rows {i, first, end} of the L / U
  // part per level position; factor items {e, k, diag(k)}; targets {entry,
  // L entry, U entry of the first contribution, start in `con` of the other
  // contributions or -1}; contributions {L entry, U entry}, each target's
  // list ended by {-1, -1}
  const int4* fwd_rec;
  const int4* bwd_rec;
  const int4* fac_rec;
  const int4* tgt_rec;
  const int2* con;
  const int8_t* g_fwd;
  const int8_t* g_bwd;
  // bus data: single phase type 0/1/2; three phase phase mask | 8 at the
  // source | 16 at a PV node (v_set its |V|, p_gen3 its generation)
  const int8_t* btype;
  const double* v_set;
  const double* q_gen;
  const double* zip;     // 3 per bus / node
  const double* p_gen0;  // case's own generation (single phase)
  const double* p_gen3;  // three phase: generation per slot of PV nodes (btype & 16)
  const double* q_min;   // single phase, optional: reactive limits of PV buses
  const double* q_max;
  const double* p_load0; // case's own loads (per bus or per slot)
  const double* q_load0;
  const int* perm;       // new -> caller numbering
  const int* iperm;      // caller -> new numbering
  double v_source;
};

// Per-solve state for B scenarios, interleaved as [entry][scenario].
struct DevWork {
  int B;  // scenario stride
  // inputs in caller numbering (NULL = the case's own)
  const double* in_p_load;
  const double* in_q_load;
  const double* in_p_gen;
  const double* in_vm;  // optional start voltage (inspection calls)
  const double* in_va;
  // outputs in caller numbering
  double* out_vm;
  double* out_va;
  pf_info* out_info;
  // warm start (new numbering, scenario 0 only): read if warm_in, written
  // after a converged solve if warm_out
  double* warm_vm;
  double* warm_va;
  double2* warm_V;
  int warm_in, warm_out;
  // state
  double* spec;   // single: (p_load, q_load, p_gen); three: (p_load, q_load) x 3
  double* vm;     // single phase
  double* va;
  double2* V;     // 1 or 3 per row
  double2* U;     // single phase, FP64 solves: V / |V| (null in mixed precision)
  double2* dV;    // refinement: voltage change of the step
  double* abcd;   // three phase: Eq. 23 adjustments, 12 per row
  double* F;      // mismatch, bs per row
  double* dx;     // Newton step, bs per row
  double* r;      // refinement residual, bs per row
  double* qg;     // three phase: reactive injection of PV slots, 3 per row
  void* lu;       // factor values, bs*bs per entry
  void* uinv;     // inverse diagonal blocks, bs*bs per row
  void* y;        // triangular-solve vector, bs per row
  // Newton-Krylov (factor precision): the Jacobian for products, the Krylov
  // basis [m+1][rows][B][bs], work vectors and reduction slots
  // [2][cluster][B][kMaxJ]
  void* jm;
  void* vb;
  void* wv;
  void* zg;
  void* xg;
  void* gred;
  unsigned long long* norm;  // [2][B] max |mismatch| (bit pattern of a double)
  unsigned long long* step;  // [2][B] max |step|
  int* flag;                 // [B] singular pivot seen
  // batched phase kernels: per-scenario state between launches
  int* status;               // [B] kRunning or the final pf_status
  int* refine;               // [B] this iteration takes the FP64 refinement
  int* iter;                 // [B] index of the scenario's latest mismatch
  unsigned long long* t0;    // start time of the launch sequence (ns)
  int* anyref;               // the last stop test left a scenario refining
  struct CallArgs* call;     // this call's inputs and outputs
  // reactive limits of PV buses (single phase; null when not enforced)
  int8_t* bt;                // [row][B] bus type of the scenario (kPQLimit:
                             // PQ at a limit, generation qsw)
  double* qsw;               // [row][B] reactive generation of a switched bus
  int* qdone;                // [B] 1: the scenario failed in an earlier round
  int* qcnt;                 // [B] switched buses
  int* qit;                  // [2][B] Newton and linear iterations of the rounds
  double* qus;               // [B] device time of the rounds
  pf_info* qinfo;            // [B] result of a scenario that failed
  int* nsw;                  // buses switched by the last check (one counter)
};

// Inputs and outputs of one batched call, read by the phase kernels from
// device memory (so that a captured graph of them serves every call).
struct CallArgs {
  const double* p_load;
  const double* q_load;
  const double* p_gen;
  const double* vm0;  // optional start voltages, the caller's [scenario][bus] order
  const double* va0;
  double* vm;
  double* va;
  pf_info* info;
};

struct DevOpts {
  double tol;
  int max_iter;
  int refine;   // FP64 refinement steps (mixed NR)
  double refine_below;  // ... taken once the mismatch norm is at most this
  double refine_stall;  // ... and the last step cut it by less than 1 / this (0: always)
  int S;        // scenarios per cluster
  int mode;     // 0 solve, 1 evaluate mismatch + Jacobian, 2 one Newton step
  unsigned long long* prof;  // optional per-phase device time (ns), kProfPhases
  int y_in_smem;             // the solve vector lives in dynamic shared memory
  int m;                     // Newton-Krylov: GMRES restart length
  int max_lin;               // ... inner iterations per Newton step
  double rtol;               // ... inner relative-residual floor
  int krylov;                // Newton-Krylov inner solver: 0 GMRES, 1 BiCGSTAB
  int ring;                  // batches of 2x2 blocks: the factorisation stages
                             // its gathers in dynamic shared memory
};

size_t dynamic_smem_bytes(int bs, size_t tf, bool nk, int n, const DevOpts& o, int threads);

// One single-CTA solve of a group launch (several cases of different sizes
// in one launch): its case, workspace and options, and the flag the CTA
// raises (1) once its results are written.
struct GroupJob {
  DevSys S;
  DevWork w;
  DevOpts o;
  int* done;
};
constexpr int kGroupMax = 160;  // jobs of one group launch
// The jobs of a launch: CTA b runs desc[job[b]].
struct GroupList {
  int n;
  int job[kGroupMax];
};

// Phases timed by the optional profile (cluster 0, CTA 0, between barriers).
enum ProfPhase { kProfSetup = 0, kProfMismatch, kProfStop, kProfFactor, kProfSolve,
                 kProfResidual, kProfUpdate, kProfOutput, kProfPhases };

}  // namespace pf
