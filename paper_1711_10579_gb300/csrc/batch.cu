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
//   the stop test is one thread per scenario;
//   the block LU refactorisation (Sec. III.A) and the triangular sweeps
//   are level-synchronous: one CTA per S scenarios, as in the persistent
//   kernel, with the registers and shared memory of the whole SM.
//
// Every launch reads the per-scenario status left by the previous ones and
// skips finished scenarios, so the host issues the whole sequence up to the
// iteration limit without waiting for the device.

#include "kernels.cuh"

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

__device__ __forceinline__ void put_info(const DevWork& w, int gs, int st, int it, double nrm,
                                         double step) {
  if (!w.out_info) return;
  pf_info inf;
  inf.status = st;
  inf.iterations = it;
  inf.linear_iterations = 0;
  inf.reserved = 0;
  inf.mismatch = nrm;
  inf.max_step = step;
  inf.solve_us = 0.0;
  w.out_info[gs] = inf;
}

template <int BS>
__global__ void __launch_bounds__(kRowThreads) k_setup(DevSys S, DevWork w, int sb) {
  RowTile t;
  if (!row_tile(w.B, S.n, sb, t)) return;
  for (int i = t.i; i < t.iend; i += t.di) setup_row<BS == 6>(S, w, i, t.gs);
  if (blockIdx.y == 0 && t.i == 0) {
    w.status[t.gs] = kRunning;
    w.refine[t.gs] = 0;
  }
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *w.t0 = global_ns();
}

// Step A of iteration it: mismatch, its norm and the Jacobian.
template <int BS, typename TF>
__global__ void __launch_bounds__(kRowThreads) k_mismatch(DevSys S, DevWork w, int sb, int it) {
  RowTile t;
  const bool on = row_tile(w.B, S.n, sb, t) && w.status[t.gs] == kRunning;
  unsigned long long m = 0ull;
  if (on) {
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

// Stop test of iteration it, one thread per scenario (the decisions of the
// persistent kernel, with the refinement chosen per scenario).
__global__ void k_stop(DevWork w, DevOpts o, int it) {
  const int gs = blockIdx.x * blockDim.x + threadIdx.x;
  const int B = w.B;
  if (gs >= B) return;
  w.refine[gs] = 0;
  if (w.status[gs] != kRunning) return;
  const double nrm = __longlong_as_double((long long)__ldcg(w.norm + (size_t)(it & 1) * B + gs));
  int st = kRunning;
  if (!(nrm <= 1e12)) st = PF_ERR_DIVERGED;
  else if (nrm <= o.tol) st = PF_OK;
  else if (it >= o.max_iter) st = PF_ERR_MAXITER;
  w.status[gs] = st;
  if (st == kRunning) {
    w.refine[gs] = (o.refine > 0 && nrm <= o.refine_below) ? 1 : 0;
  } else {
    const double step =
        it > 0 ? __longlong_as_double((long long)__ldcg(w.step + (size_t)((it - 1) & 1) * B + gs))
               : 0.0;
    put_info(w, gs, st, it, nrm, step);
  }
  // the buffers of the next iteration (read last one iteration ago)
  w.norm[(size_t)((it + 1) & 1) * B + gs] = 0ull;
  w.step[(size_t)((it + 1) & 1) * B + gs] = 0ull;
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
      if (w.status[gs] == kRunning && (!refining || w.refine[gs])) act |= 1u << s;
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
__global__ void __launch_bounds__(BS == 2 ? 512 : 256) k_factor(DevSys S, DevWork w, DevOpts o,
                                                                int it) {
  Team tm;
  if (!level_team(w, o, false, tm)) return;
  extern __shared__ __align__(16) unsigned char dsm[];
  factor_levels<BS, TF, false>(S, w, tm, 0, S.nflev, o.ring ? dsm : nullptr);
  __syncthreads();
  const int s = threadIdx.x;
  if (s < tm.ns && ((tm.act >> s) & 1u) && __ldcg(w.flag + tm.s0 + s)) {
    const int gs = tm.s0 + s;
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
  sweep_batch<BS, TF, true>(a, tm);
  a.rhs = nullptr;
  a.dx = w.dx;
  a.accumulate = (pass == 0) ? 0 : 1;
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
  if (!row_tile(w.B, S.n, sb, t) || w.status[t.gs] != kRunning || !w.refine[t.gs]) return;
  for (int i = t.i; i < t.iend; i += t.di) dv_row<BS == 6>(S, w, i, t.gs);
}

template <int BS>
__global__ void __launch_bounds__(kRowThreads) k_resid(DevSys S, DevWork w, int sb) {
  RowTile t;
  if (!row_tile(w.B, S.n, sb, t) || w.status[t.gs] != kRunning || !w.refine[t.gs]) return;
  for (int i = t.i; i < t.iend; i += t.di) resid_row<BS == 6>(S, w, i, t.gs);
}

// Step E: voltage update and the norm of the step.
template <int BS>
__global__ void __launch_bounds__(kRowThreads) k_update(DevSys S, DevWork w, int sb, int it) {
  RowTile t;
  const bool on = row_tile(w.B, S.n, sb, t) && w.status[t.gs] == kRunning;
  unsigned long long m = 0ull;
  if (on) {
    for (int i = t.i; i < t.iend; i += t.di) m = max(m, abs_bits(update_row<BS == 6>(S, w, i, t.gs)));
  }
  commit_max(m, sb, on, w.step + (size_t)(it & 1) * w.B + t.gs);
}

// Results in the caller's numbering, and the device time of the sequence.
template <int BS>
__global__ void __launch_bounds__(kRowThreads) k_output(DevSys S, DevWork w, int sb) {
  RowTile t;
  if (!row_tile(w.B, S.n, sb, t)) return;
  const bool ok = w.status[t.gs] == PF_OK;
  for (int i = t.i; i < t.iend; i += t.di) output_row<BS == 6>(S, w, i, t.gs, ok);
  if (blockIdx.y == 0 && t.i == 0 && w.out_info)
    w.out_info[t.gs].solve_us = (double)(global_ns() - __ldcg(w.t0)) * 1e-3;
}

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
cudaError_t run_batch_t(const DevSys& S, const DevWork& w, const DevOpts& o, int threads,
                        cudaStream_t st, unsigned long long* prof) {
  const int B = w.B, n = S.n;
  int sb = 1;
  while (sb < 32 && sb < B) sb <<= 1;
  const int rb = kRowThreads / sb;
  const dim3 rows((B + sb - 1) / sb, (n + rb * kRowsPerThread - 1) / (rb * kRowsPerThread));
  const dim3 blk(kRowThreads);
  const int groups = (B + o.S - 1) / o.S;
  const size_t red = (size_t)threads * BS * sizeof(TF);
  const size_t ring = o.ring ? (size_t)threads * FactorPipe<TF>::bytes : 0;
  cudaError_t e = cudaSuccess;
  if (ring > 48 * 1024)
    e = cudaFuncSetAttribute(k_factor<BS, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ring);
  if (e == cudaSuccess && red > 48 * 1024)
    e = cudaFuncSetAttribute(k_solve<BS, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)red);
  if (e != cudaSuccess) return e;
  PhaseClock clk{st, prof, {}, {}};
  auto check = [&](int ph) {
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = clk.mark(ph);
  };
  check(kProfSetup);
  k_setup<BS><<<rows, blk, 0, st>>>(S, w, sb);
  check(kProfSetup);
  for (int it = 0; e == cudaSuccess; ++it) {
    k_mismatch<BS, TF><<<rows, blk, 0, st>>>(S, w, sb, it);
    check(kProfMismatch);
    k_stop<<<(B + 127) / 128, 128, 0, st>>>(w, o, it);
    check(kProfStop);
    if (it >= o.max_iter) break;
    k_factor<BS, TF><<<groups, threads, ring, st>>>(S, w, o, it);
    check(kProfFactor);
    for (int pass = 0; pass <= o.refine && e == cudaSuccess; ++pass) {
      if (pass > 0) {
        k_dv<BS><<<rows, blk, 0, st>>>(S, w, sb);
        k_resid<BS><<<rows, blk, 0, st>>>(S, w, sb);
        check(kProfResidual);
      }
      k_solve<BS, TF><<<groups, threads, red, st>>>(S, w, o, pass);
      check(kProfSolve);
    }
    k_update<BS><<<rows, blk, 0, st>>>(S, w, sb, it);
    check(kProfUpdate);
  }
  if (e == cudaSuccess) {
    k_output<BS><<<rows, blk, 0, st>>>(S, w, sb);
    check(kProfOutput);
  }
  const cudaError_t e2 = clk.finish();
  return e != cudaSuccess ? e : e2;
}

}  // namespace

cudaError_t launch_batch_nr(int bs, bool fp32, const DevSys& S, const DevWork& w, const DevOpts& o,
                            int threads, cudaStream_t st, unsigned long long* prof) {
  if (bs == 2) return fp32 ? run_batch_t<2, float>(S, w, o, threads, st, prof)
                           : run_batch_t<2, double>(S, w, o, threads, st, prof);
  return fp32 ? run_batch_t<6, float>(S, w, o, threads, st, prof)
              : run_batch_t<6, double>(S, w, o, threads, st, prof);
}

}  // namespace pf
