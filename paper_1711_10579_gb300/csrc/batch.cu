// Batched Newton-Raphson as a sequence of phase kernels on one stream.
//
// A batch of B load scenarios of one topology has no step that couples
// scenarios, so the iteration of Sec. II.A (single phase) or Sec. II.B (three
// phase) runs as separate launches, each shaped for its own step:
//
//   setup, mismatch + Jacobian (Eq. 1-10 / 12-23), dV, FP64 residual,
//   update and output are independent per (row, scenario): a wide grid in
//   which the 32 lanes of a warp serve 32 scenarios of one row, so every
//   load of the [entry][scenario] arrays is one contiguous segment, and in
//   which many small CTAs per SM hide the latency of the neighbour gathers;
//   the stop test is one CTA over all scenarios;
//   the block LU refactorisation (Sec. III.A) and the triangular sweeps
//   are level-synchronous: one CTA per S scenarios, as in the persistent
//   kernel, with the registers and shared memory of the whole SM.
//
// Every launch reads the per-scenario status left by the previous ones and
// skips finished scenarios.  The sequence is one CUDA graph: the set-up and
// first stop test, then a conditional WHILE node whose body is one Newton
// iteration and whose stop test sets the loop condition (any scenario still
// running), then the results.  The device decides when to stop; the host
// neither waits nor issues iterations that have nothing left to do.  The
// graph is built once per launch shape and workspace; a call passes its own
// inputs and outputs through a small record in device memory.

#include "api_internal.h"
#include "kernels.cuh"

#include <array>
#include <cstring>
#include <vector>

namespace pf {

namespace {

constexpr int kRowThreads = 256;  // threads of a row-parallel CTA
constexpr int kRowsPerThread = 8;

// Row-parallel tiling: a CTA serves sb scenarios (lanes) x rb rows; thread
// (lane, r) takes scenario x sb + lane and rows r, r + rb, ... of the CTA's
// row range.
struct RowTile {
  int gs, i, di, iend;
};

__device__ __forceinline__ bool row_tile(int B, int n, int sb, RowTile& t) {
  const int lane = threadIdx.x & (sb - 1), r = threadIdx.x / sb, rb = blockDim.x / sb;
  t.gs = blockIdx.x * sb + lane;
  t.i = blockIdx.y * rb * kRowsPerThread + r;
  t.di = rb;
  t.iend = min(n, (int)(blockIdx.y + 1) * rb * kRowsPerThread);
  return t.gs < B;
}

// The largest value per scenario: the lanes of a warp with the same scenario
// sit sb apart; one atomic per warp and scenario.
__device__ __forceinline__ void commit_max(unsigned long long m, int sb, bool on,
                                           unsigned long long* dst) {
  for (int off = sb; off < 32; off <<= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
  if (on && (int)(threadIdx.x & 31) < sb && m != 0ull) atomicMax(dst, m);
}

// The workspace view of this call: its inputs and outputs from w.call.
__device__ __forceinline__ DevWork with_call(DevWork w) {
  const CallArgs* c = w.call;
  w.in_p_load = c->p_load;
  w.in_q_load = c->q_load;
  w.in_p_gen = c->p_gen;
  w.in_vm = c->vm0;
  w.in_va = c->va0;
  w.out_vm = c->vm;
  w.out_va = c->va;
  w.out_info = c->info;
  return w;
}

__device__ __forceinline__ void put_info(const DevWork& w, int gs, int st, int it, double nrm,
                                         double step) {
  pf_info* out = w.call->info;
  if (!out) return;
  pf_info inf;
  inf.status = st;
  inf.iterations = it;
  // triangular-solve passes: one per Newton step and one per refinement
  inf.linear_iterations = it + (w.refine[gs] >> 1);
  inf.fallback = 0;
  inf.mismatch = nrm;
  inf.max_step = step;
  inf.solve_us = 0.0;
  inf.q_switched = 0;
  inf.q_rounds = 1;
  out[gs] = inf;
}

// This call's inputs and outputs (one thread; launched before the sequence).
__global__ void k_args(CallArgs* dst, CallArgs a) { *dst = a; }

template <int BS>
__global__ void __launch_bounds__(kRowThreads) k_setup(DevSys S, DevWork w, int sb) {
  RowTile t;
  if (!row_tile(w.B, S.n, sb, t)) return;
  const DevWork wc = with_call(w);
  for (int i = t.i; i < t.iend; i += t.di) setup_row<BS == 6>(S, wc, i, t.gs);
  if (blockIdx.y == 0 && t.i == 0) {
    w.status[t.gs] = kRunning;
    w.refine[t.gs] = 0;
    w.iter[t.gs] = 0;
  }
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *w.t0 = global_ns();
}

// Single-phase set-up through 32 x 32 tiles (buses in the caller's order x
// scenarios) staged in shared memory: the caller's [scenario][bus] inputs
// are read along buses and the [bus][scenario] state written along
// scenarios, both contiguous.
__global__ void __launch_bounds__(256) k_setup_tile(DevSys S, DevWork w) {
  __shared__ double tp[3][32][33];
  const int n = S.n, B = w.B;
  const int o0 = blockIdx.x * 32, g0 = blockIdx.y * 32, tx = threadIdx.x;
  const CallArgs* c = w.call;
  const DevWork wc = with_call(w);
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int gs = g0 + r, oi = o0 + tx;
    if (gs < B && oi < n) {
      const size_t src = (size_t)gs * n + oi;
      const int i = S.iperm[oi];
      tp[0][r][tx] = c->p_load ? c->p_load[src] : S.p_load0[i];
      tp[1][r][tx] = c->q_load ? c->q_load[src] : S.q_load0[i];
      tp[2][r][tx] = c->p_gen ? c->p_gen[src] : S.p_gen0[i];
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int oi = o0 + r, gs = g0 + tx;
    if (oi >= n || gs >= B) continue;
    const int i = S.iperm[oi];
    setup_1ph(S, wc, i, gs, tp[0][tx][r], tp[1][tx][r], tp[2][tx][r]);
    if (i == 0) {
      setup_scenario(w, gs);
      w.status[gs] = kRunning;
      w.refine[gs] = 0;
      w.iter[gs] = 0;
      if (gs == 0) *w.t0 = global_ns();
    }
  }
}

// Step A: mismatch, its norm and the Jacobian (iteration w.iter[gs]).  The
// mixed-precision single-phase kernel is bound by the FP64 pipe: 5 CTAs per
// SM (48 registers) hide its neighbour gathers better than 4 (2.6% faster,
// with a few bytes of spills).
template <int BS, typename TF>
__global__ void __launch_bounds__(kRowThreads, (BS == 2 && sizeof(TF) == 4) ? 5 : 1)
    k_mismatch(DevSys S, DevWork w, int sb) {
  RowTile t;
  const bool on = row_tile(w.B, S.n, sb, t) && w.status[t.gs] == kRunning;
  unsigned long long m = 0ull;
  int it = 0;
  if (on) {
    it = w.iter[t.gs];
    for (int i = t.i; i < t.iend; i += t.di) {
      double nrm;
      if constexpr (BS == 6) {
        mismatch_jacobian_3ph<TF>(S, w, i, t.gs, nrm, nullptr);
      } else {
        mismatch_jacobian_1ph<TF>(S, w, i, t.gs, nrm, nullptr);
      }
      m = max(m, abs_bits(nrm));
    }
  }
  commit_max(m, sb, on, w.norm + (size_t)(it & 1) * w.B + t.gs);
}

// Stop test (the decisions of the persistent kernel, with the refinement
// chosen per scenario), one CTA over all scenarios.  A running scenario
// advances its iteration index.  When a graph's loop condition is given, it
// is set to whether any scenario still runs.
__global__ void __launch_bounds__(1024) k_stop(DevWork w, DevOpts o, int has_cond,
                                               cudaGraphConditionalHandle cond) {
  const int B = w.B;
  int running = 0, refining = 0;
  for (int gs = threadIdx.x; gs < B; gs += blockDim.x) {
    if (w.status[gs] != kRunning) continue;
    const int it = w.iter[gs];
    const double nrm =
        __longlong_as_double((long long)__ldcg(w.norm + (size_t)(it & 1) * B + gs));
    int st = kRunning;
    if (!(nrm <= 1e12)) st = PF_ERR_DIVERGED;
    else if (nrm <= o.tol) st = PF_OK;
    else if (it >= o.max_iter) st = PF_ERR_MAXITER;
    w.status[gs] = st;
    int rf = w.refine[gs] & ~1;  // refinement count << 1
    if (st == kRunning) {
      // the previous iteration's norm (its buffer is cleared below)
      const double prev =
          __longlong_as_double((long long)__ldcg(w.norm + (size_t)((it + 1) & 1) * B + gs));
      if (o.refine > 0 && refine_now(o, it, nrm, prev)) {
        rf += 3;  // flag, and one more
        refining = 1;
      }
      w.refine[gs] = rf;
      w.iter[gs] = it + 1;
      ++running;
    } else {
      w.refine[gs] = rf;
      const double step =
          it > 0
              ? __longlong_as_double((long long)__ldcg(w.step + (size_t)((it - 1) & 1) * B + gs))
              : 0.0;
      put_info(w, gs, st, it, nrm, step);
    }
    // the buffers of the next iteration (read last one iteration ago)
    w.norm[(size_t)((it + 1) & 1) * B + gs] = 0ull;
    w.step[(size_t)((it + 1) & 1) * B + gs] = 0ull;
  }
  running = __syncthreads_or(running);
  refining = __syncthreads_or(refining);
  if (threadIdx.x == 0) *w.anyref = refining;
  if (has_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, running ? 1u : 0u);
}

// Inside a graph: whether this iteration's refinement launches run at all.
__global__ void k_rflag(const int* anyref, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, *anyref ? 1u : 0u);
}

// The team of one level-synchronous CTA: scenarios [blockIdx.x S, + S),
// those still running (and, for a refinement pass, refining).
__device__ __forceinline__ bool level_team(const DevWork& w, const DevOpts& o, bool refining,
                                           Team& tm) {
  __shared__ unsigned sh_act;
  tm.tid = threadIdx.x;
  tm.nthr = blockDim.x;
  tm.S = o.S;
  tm.s0 = blockIdx.x * o.S;
  tm.ns = min(o.S, w.B - tm.s0);
  if (threadIdx.x == 0) {
    unsigned act = 0;
    for (int s = 0; s < tm.ns; ++s) {
      const int gs = tm.s0 + s;
      if (w.status[gs] == kRunning && (!refining || (w.refine[gs] & 1))) act |= 1u << s;
    }
    sh_act = act;
  }
  __syncthreads();
  tm.act = sh_act;
  return tm.act != 0;
}

// Step B: numeric block LU refactorisation; a singular pivot ends its
// scenario.
template <int BS, typename TF>
__global__ void __launch_bounds__(BS == 2 ? 512 : 256) k_factor(DevSys S, DevWork w, DevOpts o) {
  Team tm;
  if (!level_team(w, o, false, tm)) return;
  extern __shared__ __align__(16) unsigned char dsm[];
  factor_levels<BS, TF, false>(S, w, tm, 0, S.nflev, o.ring ? dsm : nullptr);
  __syncthreads();
  const int s = threadIdx.x;
  if (s < tm.ns && ((tm.act >> s) & 1u) && __ldcg(w.flag + tm.s0 + s)) {
    const int gs = tm.s0 + s;
    const int it = w.iter[gs] - 1;  // the stop test advanced it
    w.status[gs] = PF_ERR_SINGULAR;
    put_info(w, gs, PF_ERR_SINGULAR, it,
             __longlong_as_double((long long)__ldcg(w.norm + (size_t)(it & 1) * w.B + gs)), 0.0);
  }
}

// Step C: forward and backward sweeps on F (pass 0) or on the FP64 residual
// (pass > 0, scenarios that refine), writing or adding to dx.
template <int BS, typename TF>
__global__ void __launch_bounds__(BS == 2 ? 512 : 256) k_solve(DevSys S, DevWork w, DevOpts o,
                                                               int pass) {
  Team tm;
  if (!level_team(w, o, pass > 0, tm)) return;
  extern __shared__ __align__(16) unsigned char dsm[];
  BSweep<TF> a;
  a.lu = reinterpret_cast<const TF*>(w.lu);
  a.uinv = reinterpret_cast<const TF*>(w.uinv);
  a.col = S.lu_col;
  a.y = reinterpret_cast<TF*>(w.y);
  a.rhs = (pass == 0) ? w.F : w.r;
  a.dx = nullptr;
  a.accumulate = 0;
  a.B = w.B;
  a.lev_ptr = S.flev_ptr;
  a.rec = S.fwd_rec;
  a.nlev = S.nflev;
  a.gsz = S.g_fwd;
  a.red = reinterpret_cast<TF*>(dsm);
  a.refine = nullptr;
  // the staged records after the lanes' partial sums (16-byte aligned)
  a.srec = reinterpret_cast<int4*>(dsm + (((size_t)blockDim.x * BS * sizeof(TF) + 15) & ~(size_t)15));
  sweep_batch<BS, TF, true>(a, tm);
  a.rhs = nullptr;
  a.dx = w.dx;
  a.accumulate = (pass == 0) ? 0 : 1;
  // single phase, first pass: the step of a scenario that takes no
  // refinement stays in y (k_update reads it there)
  a.refine = (BS == 2 && pass == 0) ? w.refine : nullptr;
  a.lev_ptr = S.blev_ptr;
  a.rec = S.bwd_rec;
  a.nlev = S.nblev;
  a.gsz = S.g_bwd;
  sweep_batch<BS, TF, false>(a, tm);
}

// Step R: voltage change of the step, then the FP64 residual r = F - J dx.
template <int BS>
__global__ void __launch_bounds__(kRowThreads) k_dv(DevSys S, DevWork w, int sb) {
  RowTile t;
  if (!row_tile(w.B, S.n, sb, t) || w.status[t.gs] != kRunning || !(w.refine[t.gs] & 1)) return;
  for (int i = t.i; i < t.iend; i += t.di) dv_row<BS == 6>(S, w, i, t.gs);
}

template <int BS>
__global__ void __launch_bounds__(kRowThreads) k_resid(DevSys S, DevWork w, int sb) {
  RowTile t;
  if (!row_tile(w.B, S.n, sb, t) || w.status[t.gs] != kRunning || !(w.refine[t.gs] & 1)) return;
  for (int i = t.i; i < t.iend; i += t.di) resid_row<BS == 6>(S, w, i, t.gs);
}

// Step E: voltage update and the norm of the step.  Single phase: the step
// of a scenario that refined is in dx, of the others in y (FP32 in mixed
// precision: 8 bytes per bus read instead of 16, and 16 not written).
template <int BS, typename TF>
__global__ void __launch_bounds__(kRowThreads) k_update(DevSys S, DevWork w, int sb) {
  RowTile t;
  const bool on = row_tile(w.B, S.n, sb, t) && w.status[t.gs] == kRunning;
  unsigned long long m = 0ull;
  int it = 0;
  if (on) {
    it = w.iter[t.gs] - 1;  // the stop test advanced it
    const TF* y = (BS == 2 && !(w.refine[t.gs] & 1)) ? reinterpret_cast<const TF*>(w.y) : nullptr;
    for (int i = t.i; i < t.iend; i += t.di)
      m = max(m, abs_bits(update_row<BS == 6, TF>(S, w, i, t.gs, y)));
  }
  commit_max(m, sb, on, w.step + (size_t)(it & 1) * w.B + t.gs);
}

// Results in the caller's numbering, and the device time of the sequence.
template <int BS>
__global__ void __launch_bounds__(kRowThreads) k_output(DevSys S, DevWork w, int sb) {
  RowTile t;
  if (!row_tile(w.B, S.n, sb, t)) return;
  const DevWork wc = with_call(w);
  const bool ok = w.status[t.gs] == PF_OK;
  for (int i = t.i; i < t.iend; i += t.di) output_row<BS == 6>(S, wc, i, t.gs, ok);
  if (blockIdx.y == 0 && t.i == 0 && wc.out_info)
    wc.out_info[t.gs].solve_us = (double)(global_ns() - __ldcg(w.t0)) * 1e-3;
}

// Single-phase results through 32 x 32 tiles (the transpose of the set-up):
// |V| and angle in the caller's [scenario][bus] order, and the device time.
__global__ void __launch_bounds__(256) k_output_tile(DevSys S, DevWork w) {
  __shared__ double tv[2][32][33];
  const int n = S.n, B = w.B;
  const int o0 = blockIdx.x * 32, g0 = blockIdx.y * 32, tx = threadIdx.x;
  const CallArgs* c = w.call;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int oi = o0 + r, gs = g0 + tx;
    if (oi >= n || gs >= B) continue;
    const int i = S.iperm[oi];
    const size_t b = (size_t)i * B + gs;
    tv[0][r][tx] = __ldcg(w.vm + b);
    tv[1][r][tx] = __ldcg(w.va + b);
    if (i == 0 && c->info) c->info[gs].solve_us = (double)(global_ns() - __ldcg(w.t0)) * 1e-3;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int gs = g0 + r, oi = o0 + tx;
    if (gs >= B || oi >= n) continue;
    const size_t dst = (size_t)gs * n + oi;
    if (c->vm) c->vm[dst] = tv[0][tx][r];
    if (c->va) c->va[dst] = tv[1][tx][r];
  }
}

// ---------------------------------------------------------------------------
// host side: the launch sequence, direct or as one CUDA graph
// ---------------------------------------------------------------------------

// One kernel launch of the sequence: function, shape and arguments.
struct Launch {
  const void* fn;
  dim3 grid, block;
  size_t smem;
  std::vector<void*> args;
};

// The sequence of one batched solve, as a list of launches: prologue
// (set-up, first mismatch and stop test), the body of one Newton iteration
// (factor, sweeps, refinement, update, next mismatch and stop test) and the
// epilogue (results).  Argument storage lives in the Plan.
template <int BS, typename TF>
struct Plan {
  DevSys S;
  DevWork w;
  DevOpts of, os;
  int sb, pass0 = 0, pass1 = 1, has_cond = 0;
  cudaGraphConditionalHandle cond = 0, rcond = 0;
  const int* anyref = nullptr;
  // the loop body: pre, refinement, post (body = all three, in order)
  std::vector<Launch> pro, body, pre, ref, post, epi;
  dim3 rows, blk;
  int threads_f, threads_s;
  size_t red, ring;

  void build(int refine) {
    const int B = w.B, n = S.n;
    sb = 1;
    while (sb < 32 && sb < B) sb <<= 1;
    const int rb = kRowThreads / sb;
    rows = dim3((B + sb - 1) / sb, (n + rb * kRowsPerThread - 1) / (rb * kRowsPerThread));
    blk = dim3(kRowThreads);
    const dim3 gf((B + of.S - 1) / of.S), gsv((B + os.S - 1) / os.S);
    red = (((size_t)threads_s * BS * sizeof(TF) + 15) & ~(size_t)15) + (size_t)kSweepStage * 16;
    ring = !of.ring ? 0
                    : (size_t)threads_f * (of.S == 32 && BS == 2 ? FactorWarp<TF>::bytes
                                                                  : FactorPipe<TF>::bytes);
    auto rowk = [&](const void* fn) {
      return Launch{fn, rows, blk, 0, {&S, &w, &sb}};
    };
    const Launch stop{(const void*)k_stop, dim3(1), dim3(1024), 0, {&w, &of, &has_cond, &cond}};
    const dim3 tiles((n + 31) / 32, (B + 31) / 32), tblk(32, 8);
    Launch setup, output;
    if constexpr (BS == 2) {
      setup = Launch{(const void*)k_setup_tile, tiles, tblk, 0, {&S, &w}};
      output = Launch{(const void*)k_output_tile, tiles, tblk, 0, {&S, &w}};
    } else {
      setup = rowk((const void*)k_setup<BS>);
      output = rowk((const void*)k_output<BS>);
    }
    pro = {setup, rowk((const void*)k_mismatch<BS, TF>), stop};
    pre = {Launch{(const void*)k_factor<BS, TF>, gf, dim3(threads_f), ring, {&S, &w, &of}},
           Launch{(const void*)k_solve<BS, TF>, gsv, dim3(threads_s), red, {&S, &w, &os, &pass0}}};
    ref.clear();
    for (int p = 0; p < refine; ++p) {
      ref.push_back(rowk((const void*)k_dv<BS>));
      ref.push_back(rowk((const void*)k_resid<BS>));
      ref.push_back(
          Launch{(const void*)k_solve<BS, TF>, gsv, dim3(threads_s), red, {&S, &w, &os, &pass1}});
    }
    post = {rowk((const void*)k_update<BS, TF>), rowk((const void*)k_mismatch<BS, TF>), stop};
    body = pre;
    body.insert(body.end(), ref.begin(), ref.end());
    body.insert(body.end(), post.begin(), post.end());
    anyref = w.anyref;
    epi = {output};
  }
};

// Optional per-phase device time: events between launches, summed per phase.
struct PhaseClock {
  cudaStream_t st;
  unsigned long long* out;  // host, kProfPhases entries (ns), or null
  std::vector<cudaEvent_t> ev;
  std::vector<int> phase;
  cudaError_t mark(int ph) {
    if (!out) return cudaSuccess;
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    ev.push_back(e);
    phase.push_back(ph);
    return cudaEventRecord(e, st);
  }
  cudaError_t finish() {
    cudaError_t r = cudaSuccess;
    if (out && !ev.empty()) {
      r = cudaEventSynchronize(ev.back());
      for (size_t k = 1; r == cudaSuccess && k < ev.size(); ++k) {
        float ms = 0.f;
        r = cudaEventElapsedTime(&ms, ev[k - 1], ev[k]);
        out[phase[k]] += (unsigned long long)(ms * 1e6);
      }
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
    return r;
  }
};

template <int BS, typename TF>
cudaError_t set_smem(const Plan<BS, TF>& p) {
  cudaError_t e = cudaSuccess;
  if (p.ring > 48 * 1024)
    e = cudaFuncSetAttribute(k_factor<BS, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)p.ring);
  if (e == cudaSuccess && p.red > 48 * 1024)
    e = cudaFuncSetAttribute(k_solve<BS, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)p.red);
  return e;
}

// Direct launches, max_iter bodies (finished scenarios make them no-ops),
// with events between launches when a profile is asked for.
template <int BS, typename TF>
cudaError_t run_direct(Plan<BS, TF>& p, cudaStream_t st, unsigned long long* prof) {
  PhaseClock clk{st, prof, {}, {}};
  cudaError_t e = clk.mark(kProfSetup);
  auto go = [&](const Launch& l, int ph) {
    if (e == cudaSuccess)
      e = cudaLaunchKernel(l.fn, l.grid, l.block, const_cast<void**>(l.args.data()), l.smem, st);
    if (e == cudaSuccess) e = clk.mark(ph);
  };
  const void* fsolve = (const void*)k_solve<BS, TF>;
  const void* ffac = (const void*)k_factor<BS, TF>;
  const void* fmis = (const void*)k_mismatch<BS, TF>;
  auto phase = [&](const Launch& l) {
    if (l.fn == fsolve) return (int)kProfSolve;
    if (l.fn == ffac) return (int)kProfFactor;
    if (l.fn == fmis) return (int)kProfMismatch;
    if (l.fn == (const void*)k_stop) return (int)kProfStop;
    if (l.fn == (const void*)k_update<BS, TF>) return (int)kProfUpdate;
    if (l.fn == (const void*)k_setup<BS> || l.fn == (const void*)k_setup_tile)
      return (int)kProfSetup;
    if (l.fn == (const void*)k_output<BS> || l.fn == (const void*)k_output_tile)
      return (int)kProfOutput;
    return (int)kProfResidual;
  };
  for (const Launch& l : p.pro) go(l, phase(l));
  for (int it = 0; it < p.of.max_iter && e == cudaSuccess; ++it)
    for (const Launch& l : p.body) go(l, phase(l));
  for (const Launch& l : p.epi) go(l, phase(l));
  const cudaError_t e2 = clk.finish();
  return e != cudaSuccess ? e : e2;
}

// Adds the launches as a chain of kernel nodes after `dep` (may be null).
static cudaError_t add_chain(cudaGraph_t g, const std::vector<Launch>& ls, cudaGraphNode_t* dep) {
  for (const Launch& l : ls) {
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void*>(l.fn);
    kp.gridDim = l.grid;
    kp.blockDim = l.block;
    kp.sharedMemBytes = (unsigned)l.smem;
    kp.kernelParams = const_cast<void**>(l.args.data());
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphAddKernelNode(&node, g, *dep ? dep : nullptr, *dep ? 1 : 0, &kp);
    if (e != cudaSuccess) return e;
    *dep = node;
  }
  return cudaSuccess;
}

// The whole solve as one graph: prologue, a WHILE node whose body is one
// Newton iteration (its stop test sets the loop condition: any scenario
// still running), epilogue.  Rebuilt when the key changes.
template <int BS, typename TF>
cudaError_t run_graph(Plan<BS, TF>& p, cudaStream_t st, BatchGraph* g, int refine) {
  const DevOpts& o = p.of;
  std::array<long long, 17> key = {
      (long long)(uintptr_t)p.w.spec, (long long)(uintptr_t)p.S.lu_col, p.w.B, BS,
      (long long)sizeof(TF), o.S, p.threads_f, p.os.S, p.threads_s, o.max_iter, refine, o.ring,
      (long long)(uintptr_t)p.S.g_fwd, 0, 0, (long long)(uintptr_t)p.w.bt, 0};
  std::memcpy(&key[13], &o.tol, 8);
  std::memcpy(&key[14], &o.refine_below, 8);
  std::memcpy(&key[16], &o.refine_stall, 8);
  if (!g->exec || g->key != key) {
    g->reset();
    cudaError_t e = cudaGraphCreate(&g->graph, 0);
    if (e != cudaSuccess) return e;
    e = cudaGraphConditionalHandleCreate(&p.cond, g->graph, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    p.has_cond = 1;
    cudaGraphNode_t dep = nullptr;
    e = add_chain(g->graph, p.pro, &dep);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = p.cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    e = cudaGraphAddNode(&loop, g->graph, &dep, nullptr, 1, &cp);
    if (e != cudaSuccess) return e;
    cudaGraph_t bg = cp.conditional.phGraph_out[0];
    cudaGraphNode_t bdep = nullptr;
    // the refinement launches sit in an IF node, skipped in the iterations
    // where no scenario refines (its flag is set inside the body)
    const bool nested =
        !p.ref.empty() && cudaGraphConditionalHandleCreate(&p.rcond, bg, 0, 0) == cudaSuccess;
    cudaGetLastError();
    if (nested) {
      std::vector<Launch> flag = {
          Launch{(const void*)k_rflag, dim3(1), dim3(1), 0, {&p.anyref, &p.rcond}}};
      e = add_chain(bg, flag, &bdep);
      if (e == cudaSuccess) e = add_chain(bg, p.pre, &bdep);
      if (e != cudaSuccess) return e;
      cudaGraphNodeParams ip = {};
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = p.rcond;
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      cudaGraphNode_t ifn;
      e = cudaGraphAddNode(&ifn, bg, &bdep, nullptr, 1, &ip);
      if (e != cudaSuccess) return e;
      cudaGraphNode_t rdep = nullptr;
      e = add_chain(ip.conditional.phGraph_out[0], p.ref, &rdep);
      if (e != cudaSuccess) return e;
      bdep = ifn;
      e = add_chain(bg, p.post, &bdep);
    } else {
      e = add_chain(bg, p.body, &bdep);
    }
    if (e != cudaSuccess) return e;
    dep = loop;
    e = add_chain(g->graph, p.epi, &dep);
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
      g->reset();
      return e;
    }
    g->key = key;
  }
  return cudaGraphLaunch(g->exec, st);
}

template <int BS, typename TF>
cudaError_t run_batch_t(const DevSys& S, const DevWork& w, const DevOpts& of, int threads_f,
                        const DevOpts& os, int threads_s, cudaStream_t st, BatchGraph* g,
                        unsigned long long* prof) {
  Plan<BS, TF> p;
  p.S = S;
  p.w = w;
  p.of = of;
  p.os = os;
  p.threads_f = threads_f;
  p.threads_s = threads_s;
  p.build(of.refine);
  cudaError_t e = set_smem(p);
  if (e != cudaSuccess) return e;
  // this call's inputs and outputs
  CallArgs a{w.in_p_load, w.in_q_load, w.in_p_gen, w.in_vm, w.in_va, w.out_vm, w.out_va, w.out_info};
  k_args<<<1, 1, 0, st>>>(w.call, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (g && !prof) return run_graph(p, st, g, of.refine);
  return run_direct(p, st, prof);
}

}  // namespace

cudaError_t launch_batch_nr(int bs, bool fp32, const DevSys& S, const DevWork& w,
                            const DevOpts& of, int threads_f, const DevOpts& os, int threads_s,
                            cudaStream_t st, BatchGraph* g, unsigned long long* prof) {
  if (bs == 2) return fp32 ? run_batch_t<2, float>(S, w, of, threads_f, os, threads_s, st, g, prof)
                           : run_batch_t<2, double>(S, w, of, threads_f, os, threads_s, st, g, prof);
  return fp32 ? run_batch_t<6, float>(S, w, of, threads_f, os, threads_s, st, g, prof)
              : run_batch_t<6, double>(S, w, of, threads_f, os, threads_s, st, g, prof);
}

}  // namespace pf
