// Solve dispatch: launch configuration, result transfer and the inspection
// entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "api_internal.h"

namespace pf {

namespace {

int check_opts(const pf_opts& o) {
  if (o.method != PF_NR && o.method != PF_NK)
    return set_error(PF_ERR_INVALID, "opts.method must be PF_NR or PF_NK");
  if (o.precision != PF_FP64 && o.precision != PF_MIXED)
    return set_error(PF_ERR_INVALID, "opts.precision must be PF_FP64 or PF_MIXED");
  if (!(o.tol > 0.0)) return set_error(PF_ERR_INVALID, "opts.tol must be positive");
  if (o.max_iter < 0 || o.max_iter > 1000)
    return set_error(PF_ERR_INVALID, "opts.max_iter must be in [0, 1000]");
  if (!(o.refine_below >= 0.0))
    return set_error(PF_ERR_INVALID, "opts.refine_below must be >= 0");
  if (!(o.refine_stall >= 0.0))
    return set_error(PF_ERR_INVALID, "opts.refine_stall must be >= 0");
  if (o.refine_steps < 0 || o.refine_steps > 10)
    return set_error(PF_ERR_INVALID, "opts.refine_steps must be in [0, 10]");
  if (o.cluster_size < 0 || o.cluster_size > 16 || (o.cluster_size & (o.cluster_size - 1)))
    return set_error(PF_ERR_INVALID, "opts.cluster_size must be 0 or a power of two <= 16");
  if (o.block_threads < 0 || o.block_threads > 1024 || (o.block_threads % 32))
    return set_error(PF_ERR_INVALID, "opts.block_threads must be 0 or a multiple of 32 <= 1024");
  if (o.scen_per_cta < 0 || o.scen_per_cta > 32 || (o.scen_per_cta & (o.scen_per_cta - 1)))
    return set_error(PF_ERR_INVALID, "opts.scen_per_cta must be 0 or a power of two <= 32");
  if (o.kernel_by_kernel != 0 && o.kernel_by_kernel != 1)
    return set_error(PF_ERR_INVALID, "opts.kernel_by_kernel must be 0 or 1");
  if (o.nk_fallback != 0 && o.nk_fallback != 1)
    return set_error(PF_ERR_INVALID, "opts.nk_fallback must be 0 or 1");
  if (o.krylov != 0 && o.krylov != 1)
    return set_error(PF_ERR_INVALID, "opts.krylov must be 0 (GMRES) or 1 (BiCGSTAB)");
  if (o.q_limits != 0 && o.q_limits != 1)
    return set_error(PF_ERR_INVALID, "opts.q_limits must be 0 or 1");
  if (o.method == PF_NK && o.krylov == 1 && o.gmres_restart < 7)
    return set_error(PF_ERR_INVALID, "BiCGSTAB needs opts.gmres_restart >= 7 (work vectors)");
  if (o.method == PF_NK) {
    if (o.gmres_restart < 1 || o.gmres_restart >= kMaxJ)
      return set_error(PF_ERR_INVALID, "opts.gmres_restart must be in [1, 63]");
    if (o.gmres_max_iter < 1) return set_error(PF_ERR_INVALID, "opts.gmres_max_iter must be >= 1");
    if (!(o.gmres_rtol > 0.0 && o.gmres_rtol < 1.0))
      return set_error(PF_ERR_INVALID, "opts.gmres_rtol must be in (0, 1)");
    if (o.scen_per_cta > 8)
      return set_error(PF_ERR_INVALID, "opts.scen_per_cta must be <= 8 for PF_NK");
  }
  return PF_OK;
}

struct ClusterKey {
  int bs, fp32, nk, threads;
  bool operator<(const ClusterKey& k) const {
    return std::tie(bs, fp32, nk, threads) < std::tie(k.bs, k.fp32, k.nk, k.threads);
  }
};

int cached_max_cluster(int bs, bool fp32, bool nk, int threads) {
  static std::mutex mu;
  static std::map<ClusterKey, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  ClusterKey k{bs, fp32 ? 1 : 0, nk ? 1 : 0, threads};
  auto it = cache.find(k);
  if (it != cache.end()) return it->second;
  int c = max_cluster(bs, fp32, nk, threads);
  cache[k] = c;
  return c;
}

}  // namespace

void launch_shape(pf_case c, const pf_opts& o, int B, bool fp32, int* grid, int* cluster,
                  int* threads, int* S) {
  const int bs = c->bs;
  // 2x2 blocks: 512 threads (128 registers each); 6x6 blocks and the
  // Newton-Krylov kernels: 256
  const int max_threads = (bs == 2 && o.method != PF_NK) ? 512 : 256;
  if (B == 1) {
    *threads = o.block_threads ? std::min(o.block_threads, max_threads) : max_threads;
    *cluster = o.cluster_size ? o.cluster_size
                              : cached_max_cluster(bs, fp32, o.method == PF_NK, *threads);
    *S = 1;
    *grid = *cluster;
  } else {
    int tS = 0, tth = 0;
    if (!o.scen_per_cta && !o.block_threads) {
      std::lock_guard<std::mutex> lk(c->tuned_mu);
      auto it = c->tuned.find({B, o.method, o.precision});
      if (it != c->tuned.end()) {
        tS = it->second[0];
        tth = it->second[1];
      }
    }
    // default: about one CTA per SM, up to 8 scenarios per CTA
    int dS = 1;
    while (dS < 8 && (long long)B >= 2LL * dS * c->ctx->num_sms) dS <<= 1;
    if (o.method == PF_NK) dS = std::min(dS, 8);
    *threads = o.block_threads ? std::min(o.block_threads, max_threads)
                               : (tth ? tth : max_threads);
    *cluster = 1;
    *S = o.scen_per_cta ? o.scen_per_cta : (tS ? tS : dS);
    *grid = (B + *S - 1) / *S;
  }
}

int run_solve(pf_case c, const pf_opts& o, int B, const double* d_p_load, const double* d_q_load,
              const double* d_p_gen, Workspace* ws, cudaStream_t st, RunMode mode, double* out_vm,
              double* out_va, pf_info* out_info, unsigned long long* prof, const double* d_vm0,
              const double* d_va0, bool qlim, bool warm_write) {
  int rc = check_opts(o);
  if (rc != PF_OK) return rc;
  const bool nk = o.method == PF_NK;
  const int kind = c->data.kind, n = c->data.n, bs = c->bs;
  rc = ws->ensure(kind, n, std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu()), B,
                  nk ? o.gmres_restart : 0);
  if (rc != PF_OK) return rc;
  SysBuf& sb = nk ? c->nk : c->nr;
  // inspection of the Jacobian reads the factor array as FP64
  const bool fp32 = (o.precision == PF_MIXED) && mode != RunMode::Eval;
  int threads, cluster, S, grid;
  launch_shape(c, o, B, fp32, &grid, &cluster, &threads, &S);
  // a batch of Newton-Raphson solves runs its sweeps in a shape of their own
  const bool phased = B > 1 && !nk && mode == RunMode::Solve;
  int S_s = S, threads_s = threads;
  if (phased && !o.scen_per_cta && !o.block_threads) {
    std::lock_guard<std::mutex> lk(c->tuned_mu);
    auto it = c->tuned.find({B, o.method, o.precision});
    if (it != c->tuned.end() && it->second[2] > 0) {
      S_s = it->second[2];
      threads_s = it->second[3];
    }
  }
  DevSys sys;
  rc = sb.lanes_for(threads_s, S_s, sys);
  if (rc != PF_OK) return rc;
  DevWork w = ws->w;
  w.B = B;
  if (fp32) w.U = nullptr;  // the mixed-precision Jacobian reads V alone
  w.in_p_load = d_p_load;
  w.in_q_load = d_q_load;
  w.in_p_gen = d_p_gen;
  w.in_vm = nullptr;
  w.in_va = nullptr;
  w.out_vm = out_vm ? out_vm : ws->st_vm;
  w.out_va = out_va ? out_va : ws->st_va;
  w.out_info = out_info ? out_info : ws->st_info;
  w.warm_vm = c->warm_vm;
  w.warm_va = c->warm_va;
  w.warm_V = c->warm_V;
  w.warm_in = (o.warm_start && c->warm_valid && B == 1 && mode == RunMode::Solve) ? 1 : 0;
  w.warm_out = (B == 1 && mode == RunMode::Solve && warm_write) ? 1 : 0;
  if (mode != RunMode::Solve) {
    w.in_vm = ws->st_p_load;  // staged start voltage of an inspection call
    w.in_va = ws->st_q_load;
    w.in_p_load = w.in_q_load = w.in_p_gen = nullptr;
  } else if (d_vm0) {
    w.in_vm = d_vm0;  // the rounds of reactive limits restart from the last voltages
    w.in_va = d_va0;
    w.warm_in = 0;
  }
  if (!qlim || mode != RunMode::Solve) w.bt = nullptr;
  DevOpts d;
  d.tol = o.tol;
  d.max_iter = o.max_iter;
  d.refine = fp32 && o.method == PF_NR ? o.refine_steps : 0;
  d.refine_below = o.refine_below;
  d.refine_stall = o.refine_stall;
  d.S = S;
  d.mode = mode == RunMode::Solve ? 0 : (mode == RunMode::Eval ? 1 : 2);
  d.prof = prof;
  d.m = nk ? o.gmres_restart : 0;
  d.max_lin = o.gmres_max_iter;
  d.rtol = o.gmres_rtol;
  d.krylov = o.krylov;
  // single solves keep the triangular-solve vector in shared memory when it fits
  const size_t tf = fp32 ? 4 : 8;
  d.y_in_smem = 0;
  d.ring = 0;
  const size_t extra = dynamic_smem_bytes(bs, tf, nk, n, d, threads);
  d.y_in_smem = (B == 1 && (size_t)n * bs * tf + extra <= 200 * 1024) ? 1 : 0;
  if (phased) {
    // a batch of Newton-Raphson solves: phase kernels; the factorisation of
    // 2x2 blocks stages its gathers in shared memory
    d.ring = (S > 1 && bs == 2) ? 1 : 0;
    DevOpts ds = d;
    ds.S = S_s;
    unsigned long long hprof[kProfPhases] = {};
    cudaError_t e = launch_batch_nr(bs, fp32, sys, w, d, threads, ds, threads_s, st,
                                    o.kernel_by_kernel ? nullptr : &ws->graph,
                                    prof ? hprof : nullptr);
    if (e == cudaSuccess && prof) {
      // the launches have finished (the profile waited for its last event)
      unsigned long long cur[kProfPhases];
      e = cudaMemcpy(cur, prof, sizeof(cur), cudaMemcpyDeviceToHost);
      for (int k = 0; k < kProfPhases; ++k) cur[k] += hprof[k];
      if (e == cudaSuccess) e = cudaMemcpy(prof, cur, sizeof(cur), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return cuda_error(e, "launching the batched Newton kernels");
    return PF_OK;
  }
  // the persistent kernel: a batch of Newton-Krylov solves of 2x2 blocks
  // stages the factorisation's gathers in shared memory when that fits
  if (S > 1 && bs == 2) {
    d.ring = 1;
    if (dynamic_smem_bytes(bs, tf, nk, n, d, threads) > 200 * 1024) d.ring = 0;
  }
  cudaError_t e = launch_newton(bs, fp32, nk, sys, w, d, grid, cluster, threads, st);
  if (e != cudaSuccess) return cuda_error(e, "launching the Newton kernel");
  return PF_OK;
}

// Reactive limits of PV buses: rounds of solves.  Each round solves every
// scenario (the first from the usual start, the later ones from the last
// voltages, so that a scenario with nothing switched stops at once), then
// one check switches every PV bus whose generator Q is outside its limits
// to PQ at that limit, in that scenario only.  The rounds end when a check
// switches nothing; a bus switches at most once, so at most nPV + 1 rounds
// are needed (capped at 64).
int run_solve_q(pf_case c, const pf_opts& o, int B, const double* d_p_load, const double* d_q_load,
                const double* d_p_gen, Workspace* ws, cudaStream_t st, double* out_vm,
                double* out_va, pf_info* out_info, bool warm_write) {
  const CaseData& cd = c->data;
  if (!o.q_limits || cd.q_max.empty())
    return run_solve(c, o, B, d_p_load, d_q_load, d_p_gen, ws, st, RunMode::Solve, out_vm,
                     out_va, out_info, nullptr, nullptr, nullptr, false, warm_write);
  int rc = check_opts(o);
  if (rc != PF_OK) return rc;
  const bool nk = o.method == PF_NK;
  rc = ws->ensure(cd.kind, cd.n, std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu()), B,
                  nk ? o.gmres_restart : 0);
  if (rc != PF_OK) return rc;
  double* vm = out_vm ? out_vm : ws->st_vm;
  double* va = out_va ? out_va : ws->st_va;
  pf_info* info = out_info ? out_info : ws->st_info;
  const DevSys& sys = (nk ? c->nk : c->nr).view;
  DevWork w = ws->w;
  w.B = B;
  const bool three = cd.kind != PF_SINGLE_PHASE;
  int npv = 0;  // buses, or phase slots, that can switch
  for (size_t i = 0; i < cd.bus_type.size(); ++i)
    if (cd.bus_type[i] == PF_PV)
      npv += three ? ((cd.phases[i] & 1) + ((cd.phases[i] >> 1) & 1) + ((cd.phases[i] >> 2) & 1))
                   : 1;
  const int cap = std::min(npv + 1, 64);
  cudaError_t e = launch_qlim_init(sys, w, three, st);
  if (e != cudaSuccess) return cuda_error(e, "launching the reactive-limit set-up");
  int round = 0, pending = 0;
  for (;;) {
    ++round;
    rc = run_solve(c, o, B, d_p_load, d_q_load, d_p_gen, ws, st, RunMode::Solve, vm, va, info,
                   nullptr, round > 1 ? vm : nullptr, round > 1 ? va : nullptr, true, warm_write);
    if (rc != PF_OK) return rc;
    e = cudaMemsetAsync(w.nsw, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_qlim_check(sys, w, info, round, three, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&pending, w.nsw, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "checking reactive limits");
    if (pending == 0 || round >= cap) break;
  }
  e = launch_qlim_final(w, info, round, pending > 0 ? 1 : 0, st);
  if (e != cudaSuccess) return cuda_error(e, "launching the reactive-limit summary");
  return PF_OK;
}

int fetch_results(pf_case c, Workspace* ws, int B, double* vmag, double* vang, pf_info* info,
                  cudaStream_t st) {
  const size_t per = (size_t)c->data.n * (c->data.kind == PF_SINGLE_PHASE ? 1 : 3);
  std::vector<pf_info> inf(B);
  cudaError_t e = cudaSuccess;
  if (vmag) e = cudaMemcpyAsync(vmag, ws->st_vm, per * B * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && vang)
    e = cudaMemcpyAsync(vang, ws->st_va, per * B * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(inf.data(), ws->st_info, B * sizeof(pf_info), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "running the solve");
  if (info) std::copy(inf.begin(), inf.end(), info);
  if (B == 1 && inf[0].status == PF_OK) c->warm_valid = true;
  return PF_OK;
}

int inspect(pf_case c, InspectKind k, const pf_opts* po, const double* vmag, const double* vang,
            double* out, pf_info* info) {
  pf_opts o;
  if (po) o = *po; else pf_opts_default(&o);
  cudaSetDevice(c->ctx->device);
  cudaStream_t st = c->ctx->stream;
  Workspace* ws = &c->ws1;
  const int kind = c->data.kind, n = c->data.n, bs = c->bs;
  int rc = ws->ensure(kind, n, std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu()), 1,
                      o.method == PF_NK ? o.gmres_restart : 0);
  if (rc != PF_OK) return rc;
  const size_t per = (size_t)n * (kind == PF_SINGLE_PHASE ? 1 : 3);
  cudaError_t e = cudaMemcpyAsync(ws->st_p_load, vmag, per * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws->st_q_load, vang, per * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "copying the voltage");
  RunMode mode = (k == InspectKind::Step) ? RunMode::Step : RunMode::Eval;
  if (k != InspectKind::Step) {
    o.precision = PF_FP64;
    o.method = PF_NR;
  }
  rc = run_solve(c, o, 1, nullptr, nullptr, nullptr, ws, st, mode, nullptr, nullptr);
  if (rc != PF_OK) return rc;
  const Symbolic& s = (k == InspectKind::Step && o.method == PF_NK) ? c->nk.sym : c->nr.sym;
  if (k == InspectKind::Jacobian) {
    const int bb = bs * bs;
    std::vector<double> lu((size_t)s.nnz_lu() * bb);
    e = cudaMemcpyAsync(lu.data(), ws->w.lu, lu.size() * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "evaluating the Jacobian");
    for (int q = 0; q < s.nnz_lu(); ++q) {
      const int ye = s.lu2y[q];
      if (ye < 0) continue;
      std::copy(lu.begin() + (size_t)q * bb, lu.begin() + (size_t)(q + 1) * bb,
                out + (size_t)s.y_src[ye] * bb);
    }
    return PF_OK;
  }
  std::vector<double> v((size_t)n * bs);
  const double* src = (k == InspectKind::Mismatch) ? ws->w.F : ws->w.dx;
  e = cudaMemcpyAsync(v.data(), src, v.size() * 8, cudaMemcpyDeviceToHost, st);
  pf_info inf{};
  if (e == cudaSuccess && k == InspectKind::Step)
    e = cudaMemcpyAsync(&inf, ws->st_info, sizeof(pf_info), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "running the inspection kernel");
  for (int i = 0; i < n; ++i)
    for (int t = 0; t < bs; ++t) out[(size_t)s.perm[i] * bs + t] = v[(size_t)i * bs + t];
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = PF_OK;
  }
  return PF_OK;
}

// Newton-Raphson single solve whose workspace is carved out of the fixed
// scratch array instead of allocated: no cudaMalloc, no cudaFree, no host
// heap.  Everything the kernel reads from the workspace is written by the
// kernel first (its set-up zeroes the norm, step and pivot-flag slots), so
// the contents left by an earlier call do not matter; calls that overlap on
// the GPU share the array and race.
int solve_noalloc(pf_case c, const pf_opts& o, const double* d_p_load, const double* d_q_load,
                  const double* d_p_gen, double* d_vmag, double* d_vang, pf_info* d_info,
                  cudaStream_t st) {
  int rc = check_opts(o);
  if (rc != PF_OK) return rc;
  if (o.method != PF_NR)
    return set_error(PF_ERR_UNSUPPORTED, "pf_solve_noalloc runs Newton-Raphson only");
  if (o.q_limits && !c->data.q_max.empty())
    return set_error(PF_ERR_UNSUPPORTED, "pf_solve_noalloc does not enforce reactive limits");
  if (o.block_threads || o.scen_per_cta)
    return set_error(PF_ERR_INVALID, "pf_solve_noalloc uses the default CTA shape");
  const int kind = c->data.kind, n = c->data.n, bs = c->bs;
  const int nsl = kind == PF_SINGLE_PHASE ? 1 : 3;
  const bool fp32 = o.precision == PF_MIXED;
  const size_t tf = fp32 ? 4 : 8;
  const Symbolic& sy = c->nr.sym;
  const int threads = noalloc_threads(bs);
  int cluster = o.cluster_size;
  if (!cluster) cluster = max_cluster(bs, fp32, false, threads);
  // the lane tables of this launch shape, uploaded when the case was created
  DevSys sys;
  rc = c->nr.lanes_cached(threads, 1, sys);
  if (rc != PF_OK) return rc;
  // carve the workspace (256-byte aligned pieces)
  const size_t nb = (size_t)n;
  enum { kSpec, kVm, kVa, kV, kU, kDV, kAbcd, kF, kDx, kR, kLu, kUinv, kY, kNorm, kStep, kFlag,
         kQg, kPieces };
  size_t sizes[kPieces];
  sizes[kSpec] = nb * (kind == PF_SINGLE_PHASE ? 3 : 6) * 8;
  sizes[kVm] = kind == PF_SINGLE_PHASE ? nb * 8 : 0;
  sizes[kVa] = kind == PF_SINGLE_PHASE ? nb * 8 : 0;
  sizes[kV] = nb * nsl * 16;
  sizes[kU] = kind == PF_SINGLE_PHASE && !fp32 ? nb * 16 : 0;  // FP64 solves only
  sizes[kDV] = nb * nsl * 16;
  sizes[kAbcd] = kind == PF_THREE_PHASE ? nb * 12 * 8 : 0;
  sizes[kF] = nb * bs * 8;
  sizes[kDx] = nb * bs * 8;
  sizes[kR] = nb * bs * 8;
  sizes[kLu] = (size_t)sy.nnz_lu() * bs * bs * tf;
  sizes[kUinv] = nb * bs * bs * tf;
  sizes[kY] = nb * bs * tf;
  sizes[kNorm] = 2 * 8;
  sizes[kStep] = 2 * 8;
  sizes[kFlag] = 8;
  sizes[kQg] = kind == PF_THREE_PHASE ? nb * 3 * 8 : 0;  // PV reactive injections
  size_t offs[kPieces], off = 0;
  for (int q = 0; q < kPieces; ++q) {
    offs[q] = off;
    off += (sizes[q] + 255) & ~size_t(255);
  }
  if (off > kNoAllocScratchBytes) {
    char msg[160];
    snprintf(msg, sizeof(msg),
             "this case needs %zu bytes of scratch; pf_solve_noalloc has %zu", off,
             kNoAllocScratchBytes);
    return set_error(PF_ERR_INVALID, msg);
  }
  void* base = nullptr;
  cudaError_t e = noalloc_scratch(&base);
  if (e != cudaSuccess) return cuda_error(e, "looking up the scratch array");
  auto at = [&](int q) -> void* {
    return sizes[q] ? static_cast<void*>(static_cast<unsigned char*>(base) + offs[q]) : nullptr;
  };
  DevWork w{};
  w.B = 1;
  w.in_p_load = d_p_load;
  w.in_q_load = d_q_load;
  w.in_p_gen = d_p_gen;
  w.out_vm = d_vmag;
  w.out_va = d_vang;
  w.out_info = d_info;
  w.warm_vm = c->warm_vm;
  w.warm_va = c->warm_va;
  w.warm_V = c->warm_V;
  w.warm_in = (o.warm_start && c->warm_valid) ? 1 : 0;
  w.warm_out = 1;
  w.spec = (double*)at(kSpec);
  w.vm = (double*)at(kVm);
  w.va = (double*)at(kVa);
  w.V = (double2*)at(kV);
  w.U = (double2*)at(kU);
  w.dV = (double2*)at(kDV);
  w.abcd = (double*)at(kAbcd);
  w.F = (double*)at(kF);
  w.dx = (double*)at(kDx);
  w.r = (double*)at(kR);
  w.lu = at(kLu);
  w.uinv = at(kUinv);
  w.y = at(kY);
  w.norm = (unsigned long long*)at(kNorm);
  w.step = (unsigned long long*)at(kStep);
  w.flag = (int*)at(kFlag);
  w.qg = (double*)at(kQg);
  DevOpts d{};
  d.tol = o.tol;
  d.max_iter = o.max_iter;
  d.refine = fp32 ? o.refine_steps : 0;
  d.refine_below = o.refine_below;
  d.refine_stall = o.refine_stall;
  d.S = 1;
  d.mode = 0;
  d.prof = nullptr;
  d.m = 0;
  d.max_lin = o.gmres_max_iter;
  d.rtol = o.gmres_rtol;
  d.y_in_smem = ((size_t)n * bs * tf <= 200 * 1024) ? 1 : 0;
  e = launch_newton(bs, fp32, false, sys, w, d, cluster, cluster, threads, st);
  if (e != cudaSuccess) return cuda_error(e, "launching the Newton kernel");
  return PF_OK;
}

int autotune(pf_case c, int B, pf_opts* io) {
  if (B < 2) return set_error(PF_ERR_INVALID, "autotuning is for batches (B >= 2)");
  pf_opts o = *io;
  int rc = check_opts(o);
  if (rc != PF_OK) return rc;
  cudaSetDevice(c->ctx->device);
  cudaStream_t st = c->ctx->stream;
  Workspace* ws = &c->wsB;
  const bool nr = o.method == PF_NR;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_error(e, "creating timing events");
  // Newton-Raphson batches: the factorisation and the sweeps are separate
  // launches whose times (per-phase profile) do not depend on each other's
  // shape, so each gets its own fastest shape
  unsigned long long* d_prof = nullptr;
  if (nr) e = cudaMalloc(&d_prof, kProfPhases * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cuda_error(e, "allocating the profile counters");
  }
  const int max_threads = (c->bs == 2 && nr) ? 512 : 256;
  float best = 1e30f, best_f = 1e30f, best_s = 1e30f;
  int bestS = 0, bestT = 0, bestS_s = 0, bestT_s = 0;
  for (int S : {1, 2, 4, 8, 16, 32}) {
    if (S > 8 && (!nr || 2 * S > B)) continue;
    for (int T : {128, 256, 512}) {
      if (T > max_threads) continue;
      pf_opts t = o;
      t.scen_per_cta = S;
      t.block_threads = T;
      float ms = 1e30f;
      unsigned long long h[kProfPhases] = {};
      for (int rep = 0; rep < 2 && rc == PF_OK; ++rep) {
        if (nr) e = cudaMemsetAsync(d_prof, 0, kProfPhases * sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess)
          rc = run_solve(c, t, B, nullptr, nullptr, nullptr, ws, st, RunMode::Solve, nullptr,
                         nullptr, nullptr, (nr && rep > 0) ? d_prof : nullptr);
        if (rc == PF_OK && e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (rc == PF_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
        float x = 0;
        if (rc == PF_OK && e == cudaSuccess) e = cudaEventElapsedTime(&x, e0, e1);
        if (rc == PF_OK && e == cudaSuccess && nr && rep > 0)
          e = cudaMemcpy(h, d_prof, sizeof(h), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_error(e, "timing a candidate shape");
        if (rep > 0) ms = x;  // the first run warms up
      }
      if (rc != PF_OK) break;
      if (!nr && ms < best) {
        best = ms;
        bestS = S;
        bestT = T;
      }
      if (nr) {
        const float f = (float)h[kProfFactor], sv = (float)h[kProfSolve];
        if (f < best_f) {
          best_f = f;
          bestS = S;
          bestT = T;
        }
        if (sv < best_s) {
          best_s = sv;
          bestS_s = S;
          bestT_s = T;
        }
      }
    }
    if (rc != PF_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (d_prof) cudaFree(d_prof);
  if (rc != PF_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(c->tuned_mu);
    c->tuned[{B, o.method, o.precision}] = {bestS, bestT, bestS_s, bestT_s};
  }
  io->scen_per_cta = bestS;
  io->block_threads = bestT;
  return PF_OK;
}

int profile_solve(pf_case c, int B, const pf_opts& o, double* phase_us, pf_info* info) {
  cudaSetDevice(c->ctx->device);
  cudaStream_t st = c->ctx->stream;
  Workspace* ws = (B == 1) ? &c->ws1 : &c->wsB;
  int rc = ws->ensure(c->data.kind, c->data.n,
                      std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu()), B,
                      o.method == PF_NK ? o.gmres_restart : 0);
  if (rc != PF_OK) return rc;
  unsigned long long* d_prof = nullptr;
  cudaError_t e = cudaMalloc(&d_prof, kProfPhases * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_error(e, "allocating the profile counters");
  e = cudaMemsetAsync(d_prof, 0, kProfPhases * sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    rc = run_solve(c, o, B, nullptr, nullptr, nullptr, ws, st, RunMode::Solve, nullptr, nullptr,
                   nullptr, d_prof);
    unsigned long long h[kProfPhases];
    if (rc == PF_OK) rc = fetch_results(c, ws, B, nullptr, nullptr, info, st);
    if (rc == PF_OK) {
      e = cudaMemcpy(h, d_prof, sizeof(h), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) rc = cuda_error(e, "reading the profile counters");
      else
        for (int k = 0; k < kProfPhases; ++k) phase_us[k] = 1e-3 * (double)h[k];
    }
  } else {
    rc = cuda_error(e, "clearing the profile counters");
  }
  cudaFree(d_prof);
  return rc;
}

}  // namespace pf
