// Internal state behind the opaque handles of pf.h.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "device.h"
#include "host.h"

namespace pf {

int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* what);

// A set of cudaMalloc'ed blocks released together.
struct DevBuffer {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  ~DevBuffer();
  void release();
  cudaError_t alloc(void** out, size_t nbytes);
};

// One ordering of a case: host symbolic analysis plus its device copy.
struct SysBuf {
  Symbolic sym;
  DevSys view{};
  DevBuffer mem;
  std::map<int, std::array<const int8_t*, 2>> g_cache;
  std::mutex g_mu;  // the serving thread and callers share g_cache
  int build(const CaseData& c, const Ybus& y, Ordering ord, bool fill);
  // The view with the lane tables of a launch shape (uploaded on first use
  // and cached); lanes_cached only looks them up and fails if absent.
  int lanes_for(int threads, int S, DevSys& out);
  int lanes_cached(int threads, int S, DevSys& out);

 private:
  void finish_view(const std::array<const int8_t*, 2>& g, int threads, DevSys& out) const;
};

// Threads per CTA of the entry point without allocation (its lane tables are
// uploaded when the case is created).
inline int noalloc_threads(int bs) { return bs == 2 ? 512 : 256; }

// Per-solve device state for up to `cap` scenarios plus staging buffers.
// A batched Newton-Raphson solve as one CUDA graph (batch.cu): its key is
// the launch configuration and workspace it was built for.
struct BatchGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::array<long long, 17> key{};
  BatchGraph() = default;
  BatchGraph(const BatchGraph&) {}  // a copy starts empty
  BatchGraph& operator=(const BatchGraph&) {
    reset();
    return *this;
  }
  ~BatchGraph() { reset(); }
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    key = {};
  }
};

struct Workspace {
  // capacity the buffers were sized for: scenarios, Krylov restart length,
  // case kind, rows and factor block entries
  int cap = 0;
  int cap_m = -1;
  int cap_kind = 0;
  int cap_n = 0;
  long long cap_nnz = 0;
  DevWork w{};
  DevBuffer mem;
  double *st_p_load = nullptr, *st_q_load = nullptr, *st_p_gen = nullptr;
  double *st_vm = nullptr, *st_va = nullptr;
  pf_info* st_info = nullptr;
  BatchGraph graph;  // batched Newton-Raphson launch sequence
  int ensure(int kind, int n, long long nnz_lu, int B, int m = 0);
  static size_t bytes_for(int kind, int n, long long nnz_lu, int B, int m = 0);
};

struct Server;

}  // namespace pf

struct pf_ctx_s {
  int device = 0;
  int num_sms = 0;
  size_t budget = 0;
  // largest case created in this context per kind (single phase, three
  // phase): rows and factor block entries (serving sizes its job slots once)
  std::atomic<int> max_n[2] = {0, 0};
  std::atomic<long long> max_nnz[2] = {0, 0};
  cudaStream_t stream = nullptr;
  pf::Server* server = nullptr;  // owned; released by serve_shutdown
  std::mutex server_mu;
};

struct pf_case_s {
  pf_ctx ctx = nullptr;
  pf::CaseData data;
  pf::Ybus y;
  int bs = 2;
  pf::SysBuf nr;  // minimum degree + fill (LU)
  pf::SysBuf nk;  // reverse Cuthill-McKee, Ybus pattern (ILU(0))
  pf::Workspace ws1, wsB;
  pf::DevBuffer mem;
  double* warm_vm = nullptr;
  double* warm_va = nullptr;
  double2* warm_V = nullptr;
  bool warm_valid = false;
  std::mutex mu;
  // autotuned batch shapes: (B, method, precision) -> (scenarios per CTA,
  // threads) of the factorisation (Newton-Krylov: the whole launch), then of
  // the triangular sweeps of a Newton-Raphson batch
  std::map<std::array<int, 3>, std::array<int, 4>> tuned;
  std::mutex tuned_mu;
};

namespace pf {

enum class RunMode { Solve, Eval, Step };
enum class InspectKind { Mismatch, Jacobian, Step };

// Launches one solve of B scenarios on `ws` (asynchronous on `st`).
// Outputs go to out_vm / out_va / out_info when given, else to the
// workspace's staging buffers.
int run_solve(pf_case c, const pf_opts& o, int B, const double* d_p_load,
              const double* d_q_load, const double* d_p_gen, Workspace* ws,
              cudaStream_t st, RunMode mode, double* out_vm, double* out_va,
              pf_info* out_info = nullptr, unsigned long long* prof = nullptr,
              const double* d_vm0 = nullptr, const double* d_va0 = nullptr, bool qlim = false,
              bool warm_write = true);
// run_solve of a Solve with the reactive limits of PV buses enforced when
// o.q_limits is set and the case has them (rounds of solves, waiting for the
// device between rounds); otherwise run_solve.  warm_write false: a single
// solve leaves the case's warm-start voltages alone.
int run_solve_q(pf_case c, const pf_opts& o, int B, const double* d_p_load,
                const double* d_q_load, const double* d_p_gen, Workspace* ws, cudaStream_t st,
                double* out_vm, double* out_va, pf_info* out_info, bool warm_write = true);
// Reactive-limit checks (qlim.cu).
cudaError_t launch_qlim_init(const DevSys& S, const DevWork& w, bool three, cudaStream_t st);
cudaError_t launch_qlim_check(const DevSys& S, const DevWork& w, const pf_info* info, int round,
                              bool three, cudaStream_t st);
cudaError_t launch_qlim_final(const DevWork& w, pf_info* info, int round, int capped,
                              cudaStream_t st);
void launch_shape(pf_case c, const pf_opts& o, int B, bool fp32, int* grid, int* cluster,
                  int* threads, int* S);
int profile_solve(pf_case c, int B, const pf_opts& o, double* phase_us, pf_info* info);
int autotune(pf_case c, int B, pf_opts* o);
// Copies staged results of the last run_solve on ws to host arrays.
int fetch_results(pf_case c, Workspace* ws, int B, double* vmag, double* vang,
                  pf_info* info, cudaStream_t st);
int inspect(pf_case c, InspectKind k, const pf_opts* o, const double* vmag,
            const double* vang, double* out, pf_info* info);

// Launchers in newton.cu (kernels in newton.cuh) and batch.cu.
cudaError_t launch_newton(int bs, bool fp32, bool nk, const DevSys& S, const DevWork& w,
                          const DevOpts& o, int grid, int cluster, int threads,
                          cudaStream_t st);
int max_cluster(int bs, bool fp32, bool nk, int threads);
// Group launch (newton.cu, kernel in newton.cuh): list.n clusters of `cluster` CTAs (1-8), cluster
// b solving desc[list.job[b]] with smem bytes of dynamic shared memory per CTA.
cudaError_t launch_newton_group(int bs, bool fp32, const GroupJob* desc, const GroupList& list,
                                size_t smem, int cluster, cudaStream_t st);
// Branch flows and losses (flows.cu); device arrays, ph = 1 or 3.
cudaError_t launch_branch_flows(int ph, const int2* ft, const double* yb, const double* sh, int n,
                                int m, int B, const double* vm, const double* va, double* pf_,
                                double* qf, double* pt, double* qt, double* loss,
                                cudaStream_t st);
// Batched Newton-Raphson as phase kernels (batch.cu); prof, if given, is a
// host array of kProfPhases device times (ns) to add to.
cudaError_t launch_batch_nr(int bs, bool fp32, const DevSys& S, const DevWork& w,
                            const DevOpts& of, int threads_f, const DevOpts& os, int threads_s,
                            cudaStream_t st, BatchGraph* g, unsigned long long* prof);
cudaError_t noalloc_scratch(void** ptr);
int solve_noalloc(pf_case c, const pf_opts& o, const double* d_p_load, const double* d_q_load,
                  const double* d_p_gen, double* d_vmag, double* d_vang, pf_info* d_info,
                  cudaStream_t st);

// Serving runtime (serve.cpp).
void serve_shutdown(pf_ctx ctx);
void serve_forget_case(pf_ctx ctx, pf_case c);

}  // namespace pf
