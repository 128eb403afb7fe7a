// Serving runtime: continuous admission of queued solves onto the GPU.
//
// Each context owns one dispatcher thread.  Requests wait in a FIFO queue.
// Newton-Raphson requests run as group launches: one launch takes every
// queued request that fits (free job slots and the context's HBM budget),
// of any cases and sizes, and each of its CTAs solves one request on its own
// (newton.cuh: newton_group_kernel); the largest requests run in separate
// group launches of 2-, 4- and 8-CTA clusters, one cluster per request.  A job's
// descriptor, inputs and outputs
// live in pinned host memory; the CTA raises the job's done flag when its
// results are written, so every request retires as soon as its own solve
// ends, while the other CTAs of its launch still run.  New requests form the
// next group at once, on the next of several streams, so requests that
// arrive while others are on the GPU start as job slots free up and their
// work overlaps on the device.  Newton-Krylov requests and requests with
// reactive limits (rounds that wait for the device between solves) run as
// per-request launches on a few stream slots of their own.
//
// Warm starts: the case's warm-start voltages are read by a job only while
// no job of that case that writes them is in flight, and written only by a
// job that is the case's only one in flight, so no job starts from a mix of
// two solutions.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.h"

namespace pf {

namespace {

constexpr int kJobs = kGroupMax;  // single-CTA solves on the GPU at once (about one per SM)
constexpr int kGroupStreams = 64;  // group launches in flight at once (each on its own stream)
constexpr int kSlots = 8;         // per-request launches (Newton-Krylov, reactive limits)
constexpr size_t kMaxQueue = 1 << 20;
constexpr size_t kGroupSmemMax = 200 * 1024;  // a job's solve vector in shared memory up to this
// Requests of at least this many rows (buses; nodes of a feeder) run on a
// cluster of CTAs instead of one CTA: their single-CTA solve is the tail of
// the latency (a 63,000-bus grid: 65 ms on one CTA, 37 ms on 4).  Tiers:
// kMidCluster CTAs from kMidRows*, kBigCluster from kBigRows*, kHugeCluster
// from kHugeRows*.
constexpr int kMidRows1ph = 4000, kMidRows3ph = 2000, kMidCluster = 2;
constexpr int kBigRows1ph = 16000, kBigRows3ph = 5000, kBigCluster = 4;
constexpr int kHugeRows1ph = 40000, kHugeRows3ph = 12000, kHugeCluster = 8;
constexpr int kTierCluster[4] = {1, kMidCluster, kBigCluster, kHugeCluster};

// Coalesced batches: kBatchMin or more queued Newton-Raphson requests of one
// case with the same solve options and their own loads run as one batched
// solve (the phase kernels of batch.cu in one CUDA graph, flat start) of at
// most kBatchMax scenarios (and kBatchDoubles staged doubles per vector),
// on one of kBatchSlots streams.
constexpr int kBatchMin = 16, kBatchMax = 4864, kBatchSlots = 2;
constexpr size_t kBatchDoubles = size_t(1) << 26;

struct Request {
  pf_ticket id = 0;
  pf_case c = nullptr;
  pf_opts o{};
  std::vector<double> p_load, q_load, p_gen;  // empty = the case's own
  std::vector<double> vm, va;
  pf_info info{};
  int state = 0;  // 0 queued, 1 running, 2 done
  size_t footprint = 0;
  int nk_lin = -1;  // Newton-Krylov inner iterations before a Newton-Raphson redo
};

bool grouped(const Request& r) {
  return r.o.method == PF_NR && !(r.o.q_limits && !r.c->data.q_max.empty()) &&
         !r.o.block_threads && !r.o.scen_per_cta && !r.o.cluster_size;
}

// The cluster size of a request is kTierCluster[size_tier].
int size_tier(const Request& r) {
  const bool one = r.c->data.kind == PF_SINGLE_PHASE;
  const int n = r.c->data.n;
  if (n >= (one ? kHugeRows1ph : kHugeRows3ph)) return 3;
  if (n >= (one ? kBigRows1ph : kBigRows3ph)) return 2;
  return n >= (one ? kMidRows1ph : kMidRows3ph) ? 1 : 0;
}

size_t slots_of(const Request& r) {
  return (size_t)r.c->data.n * (r.c->data.kind == PF_SINGLE_PHASE ? 1 : 3);
}

// Pinned host staging of one request: inputs (3 vectors) and results (2).
struct Staging {
  double* h_in = nullptr;
  double* h_out = nullptr;
  size_t cap = 0;  // doubles per vector
  int ensure(size_t per) {
    if (per <= cap) return PF_OK;
    if (h_in) cudaFreeHost(h_in);
    if (h_out) cudaFreeHost(h_out);
    h_in = h_out = nullptr;
    cap = 0;
    cudaError_t e = cudaMallocHost(&h_in, 3 * per * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&h_out, 2 * per * sizeof(double));
    if (e != cudaSuccess) return cuda_error(e, "allocating pinned staging");
    cap = per;
    return PF_OK;
  }
  ~Staging() {
    if (h_in) cudaFreeHost(h_in);
    if (h_out) cudaFreeHost(h_out);
  }
};

// One single-CTA solve slot of the group launches.  One workspace per case
// kind, grown to the largest request they have run (cudaFree would
// synchronise the device, so they are never shrunk).
struct Job {
  Workspace ws1ph, ws3ph;
  Staging io;
  Request* req = nullptr;
  int stream = -1;
  bool warm_in = false, warm_out = false;
  int want_n = 0;  // sizes to grow the buffers to (largest case of the kind seen)
  long long want_nnz = 0;
  size_t want_per = 0;
};

// One coalesced batch in flight: its stream, workspace and pinned staging
// ([3][B][per] inputs, [2][B][per] results, [B] records), grown as needed.
struct BatchSlot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  Workspace ws;
  double* h_in = nullptr;
  double* h_out = nullptr;
  pf_info* h_info = nullptr;
  size_t cap = 0;  // doubles per [B][per] vector
  int cap_B = 0;
  std::vector<Request*> reqs;
  size_t per = 0;
  int ensure(size_t need, int B) {
    if (need <= cap && B <= cap_B) return PF_OK;
    release();
    const size_t c = std::max(need, 2 * cap);
    const int b = std::max(B, 2 * cap_B);
    cudaError_t e = cudaMallocHost(&h_in, 3 * c * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&h_out, 2 * c * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&h_info, (size_t)b * sizeof(pf_info));
    if (e != cudaSuccess) {
      release();
      return cuda_error(e, "allocating pinned batch staging");
    }
    cap = c;
    cap_B = b;
    return PF_OK;
  }
  void release() {
    if (h_in) cudaFreeHost(h_in);
    if (h_out) cudaFreeHost(h_out);
    if (h_info) cudaFreeHost(h_info);
    h_in = h_out = nullptr;
    h_info = nullptr;
    cap = 0;
    cap_B = 0;
  }
  ~BatchSlot() { release(); }
};

// Runs fn(k) for k in [0, B) on up to 8 host threads when the work is large
// (copies of a coalesced batch's inputs and results), else on this thread.
template <class Fn>
void parallel_for(int B, size_t bytes, Fn fn) {
  const int T = bytes >= (size_t(64) << 20) ? std::min(8, B) : 1;
  if (T <= 1) {
    for (int k = 0; k < B; ++k) fn(k);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < T; ++t)
    th.emplace_back([&, t] {
      for (int k = t; k < B; k += T) fn(k);
    });
  for (auto& x : th) x.join();
}

// Requests that one coalesced batch can hold together: same case, options
// that change the solve, and the same inputs given.
bool batchable(const Request& r) {
  return grouped(r) && !r.p_load.empty() && !r.q_load.empty() &&
         (r.c->data.kind == PF_SINGLE_PHASE || r.p_gen.empty());
}

bool same_batch(const Request& a, const Request& b) {
  return a.c == b.c && a.o.precision == b.o.precision && a.o.tol == b.o.tol &&
         a.o.max_iter == b.o.max_iter && a.o.refine_steps == b.o.refine_steps &&
         a.o.refine_below == b.o.refine_below && a.o.refine_stall == b.o.refine_stall &&
         a.p_gen.empty() == b.p_gen.empty();
}

// One per-request launch slot: a stream with its own workspaces.
struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  Workspace ws1ph, ws3ph;
  Staging io;
  pf_info* h_info = nullptr;
  Request* req = nullptr;
};

}  // namespace

struct Server {
  pf_ctx ctx = nullptr;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<Request*> queue;
  std::unordered_map<pf_ticket, std::unique_ptr<Request>> all;
  Job jobs[kJobs];
  GroupJob* h_desc = nullptr;  // pinned: the jobs' descriptors
  pf_info* h_info = nullptr;   // pinned: the jobs' result records
  int* h_done = nullptr;       // pinned: the jobs' done flags
  cudaStream_t gst[kGroupStreams] = {};
  int gnext = 0;
  int ginflight[kGroupStreams] = {};
  Slot slots[kSlots];
  BatchSlot batches[kBatchSlots];
  std::unordered_map<pf_case, int> warm_readers, warm_writers;
  // largest case seen per kind (single phase, three phase): rows, factor
  // entries and staged doubles per vector
  int max_n[2] = {0, 0};
  long long max_nnz[2] = {0, 0};
  size_t max_per[2] = {0, 0};
  size_t used = 0;  // device bytes of running requests
  int running = 0;
  bool stop = false;
  pf_ticket next = 1;
  std::string fatal;  // a CUDA failure that stopped the dispatcher
  pf_serve_stats stats{};

  size_t footprint(const Request& r) const {
    const pf_case c = r.c;
    return Workspace::bytes_for(c->data.kind, c->data.n,
                                std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu()), 1,
                                r.o.method == PF_NK ? r.o.gmres_restart : 0);
  }

  void begin(Request* r) {
    r->state = 1;
    used += r->footprint;
    ++running;
    stats.peak_running = std::max(stats.peak_running, running);
  }

  void end(Request* r) {
    r->state = 2;
    used -= r->footprint;
    --running;
    ++stats.requests;
  }

  void fail(Request* r, int code) {
    std::memset(&r->info, 0, sizeof(r->info));
    r->info.status = code;
    r->state = 2;
  }

  // ---- group launches ----

  // Claims job k for request r (lock held): the warm-start roles.
  void claim(int k, Request* r) {
    Job& J = jobs[k];
    pf_case c = r->c;
    // warm start: read while no writer of the case is in flight; written by
    // the case's only job in flight
    const bool writer = warm_writers[c] > 0;
    J.warm_in = r->o.warm_start && c->warm_valid && !writer;
    J.warm_out = !writer && warm_readers[c] == 0;
    if (J.warm_in) ++warm_readers[c];
    if (J.warm_out) ++warm_writers[c];
    // the slot's buffers are grown to the largest case of the kind created
    // in the context (so that a slot is allocated once)
    const int ki = c->data.kind == PF_SINGLE_PHASE ? 0 : 1;
    J.want_n = std::max(max_n[ki], ctx->max_n[ki].load());
    J.want_nnz = std::max(max_nnz[ki], ctx->max_nnz[ki].load());
    J.want_per = std::max(max_per[ki], (size_t)J.want_n * (ki == 0 ? 1 : 3));
    h_done[k] = 0;
    J.req = r;
    begin(r);
  }

  // Undoes claim() for a job that never ran (lock held).
  void unclaim(int k, int code) {
    Job& J = jobs[k];
    Request* r = J.req;
    if (J.warm_in) --warm_readers[r->c];
    if (J.warm_out) --warm_writers[r->c];
    J.req = nullptr;
    J.stream = -1;
    end(r);
    fail(r, code);
  }

  // Stages job k (dispatcher thread, lock not held: it may allocate): its
  // workspace, pinned inputs and descriptor; returns the dynamic shared
  // memory its solve needs.
  int stage(int k, size_t* smem) {
    Job& J = jobs[k];
    Request* r = J.req;
    pf_case c = r->c;
    const int kind = c->data.kind, n = c->data.n, bs = c->bs;
    const bool fp32 = r->o.precision == PF_MIXED;
    const size_t per = slots_of(*r), tf = fp32 ? 4 : 8;
    Workspace& ws = kind == PF_SINGLE_PHASE ? J.ws1ph : J.ws3ph;
    // grown at once to the largest case of the kind seen so far (claim), so
    // that job slots are rarely reallocated (cudaFree synchronises the device)
    const long long nnz = std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu());
    int rc = ws.ensure(kind, std::max(n, J.want_n), std::max(nnz, J.want_nnz), 1, 0);
    if (rc == PF_OK) rc = J.io.ensure(std::max(per, J.want_per));
    GroupJob& g = h_desc[k];
    if (rc == PF_OK) rc = c->nr.lanes_cached(noalloc_threads(bs), 1, g.S);
    if (rc != PF_OK) return rc;
    const std::vector<double>* src[3] = {&r->p_load, &r->q_load, &r->p_gen};
    const double* in[3] = {nullptr, nullptr, nullptr};
    for (int q = 0; q < 3; ++q) {
      if (src[q]->empty()) continue;
      std::memcpy(J.io.h_in + q * per, src[q]->data(), per * sizeof(double));
      in[q] = J.io.h_in + q * per;
    }
    DevWork w = ws.w;
    w.B = 1;
    if (fp32) w.U = nullptr;
    w.in_p_load = in[0];
    w.in_q_load = in[1];
    w.in_p_gen = in[2];
    w.in_vm = w.in_va = nullptr;
    w.out_vm = J.io.h_out;
    w.out_va = J.io.h_out + per;
    w.out_info = h_info + k;
    w.warm_vm = c->warm_vm;
    w.warm_va = c->warm_va;
    w.warm_V = c->warm_V;
    w.warm_in = J.warm_in ? 1 : 0;
    w.warm_out = J.warm_out ? 1 : 0;
    w.bt = nullptr;
    DevOpts d{};
    d.tol = r->o.tol;
    d.max_iter = r->o.max_iter;
    d.refine = fp32 ? r->o.refine_steps : 0;
    d.refine_below = r->o.refine_below;
    d.refine_stall = r->o.refine_stall;
    d.S = 1;
    d.mode = 0;
    d.prof = nullptr;
    d.y_in_smem = ((size_t)n * bs * tf <= kGroupSmemMax) ? 1 : 0;
    d.max_lin = r->o.gmres_max_iter;
    d.rtol = r->o.gmres_rtol;
    g.w = w;
    g.o = d;
    g.done = h_done + k;
    h_done[k] = 0;
    *smem = d.y_in_smem ? (size_t)n * bs * tf : 0;
    return PF_OK;
  }

  void retire(int k) {
    Job& J = jobs[k];
    Request* r = J.req;
    const size_t per = slots_of(*r);
    r->vm.assign(J.io.h_out, J.io.h_out + per);
    r->va.assign(J.io.h_out + per, J.io.h_out + 2 * per);
    r->info = h_info[k];
    if (r->nk_lin >= 0) {  // a Newton-Krylov request solved again by Newton-Raphson
      r->info.fallback = 1;
      r->info.linear_iterations = r->nk_lin;
    }
    if (J.warm_in) --warm_readers[r->c];
    if (J.warm_out) {
      --warm_writers[r->c];
      if (r->info.status == PF_OK) r->c->warm_valid = true;
    }
    --ginflight[J.stream];
    J.req = nullptr;
    J.stream = -1;
    end(r);
  }

  // Admits queued Newton-Raphson requests into one group launch per (case
  // kind, precision): the jobs are claimed with the lock held, staged and
  // launched without it (staging may allocate), and failures are settled
  // with the lock held again.  Returns whether anything was admitted.
  bool admit_groups(std::unique_lock<std::mutex>& lk) {
    // a new group goes to a stream with nothing in flight; with none free,
    // arrivals wait in the queue and form a larger group when one frees up
    int idle = 0;
    for (int q = 0; q < kGroupStreams; ++q) idle += ginflight[q] == 0;
    if (idle == 0) return false;
    std::vector<int> claimed;
    int free_job = 0;
    bool any = false;
    for (auto it = queue.begin(); it != queue.end();) {
      Request* r = *it;
      if (!grouped(*r)) {
        ++it;
        continue;
      }
      while (free_job < kJobs && jobs[free_job].req) ++free_job;
      if (free_job >= kJobs) break;
      if (used + r->footprint > ctx->budget) {
        if (running > 0) break;  // wait for memory to free up (FIFO order)
        it = queue.erase(it);    // can never fit, even alone
        fail(r, PF_ERR_NOMEM);
        any = true;
        continue;
      }
      it = queue.erase(it);
      claim(free_job, r);
      claimed.push_back(free_job);
      any = true;
    }
    if (claimed.empty()) return any;
    struct Group {
      GroupList list;
      size_t smem = 0;
      int bs = 2;
      bool fp32 = true;
      int cluster = 1;
    };
    Group grp[16];
    for (Group& g : grp) g.list.n = 0;
    std::vector<std::pair<int, int>> failed;  // (job, status)
    lk.unlock();
    for (int k : claimed) {
      Request* r = jobs[k].req;
      size_t smem = 0;
      const int rc = stage(k, &smem);
      if (rc != PF_OK) {
        failed.push_back({k, rc});
        continue;
      }
      const int tier = size_tier(*r);
      Group& g = grp[(r->c->bs == 2 ? 0 : 2) + (r->o.precision == PF_MIXED ? 0 : 1) + 4 * tier];
      g.bs = r->c->bs;
      g.fp32 = r->o.precision == PF_MIXED;
      g.cluster = kTierCluster[tier];
      g.smem = std::max(g.smem, smem);
      g.list.job[g.list.n++] = k;
    }
    std::string err;
    for (Group& g : grp) {
      if (g.list.n == 0) continue;
      // the next idle stream (round robin), else the next one
      int sidx = gnext;
      for (int q = 0; q < kGroupStreams; ++q) {
        const int c = (gnext + q) % kGroupStreams;
        if (ginflight[c] == 0) {
          sidx = c;
          break;
        }
      }
      gnext = (sidx + 1) % kGroupStreams;
      const cudaError_t e =
          launch_newton_group(g.bs, g.fp32, h_desc, g.list, g.smem, g.cluster, gst[sidx]);
      for (int q = 0; q < g.list.n; ++q) {
        if (e == cudaSuccess) jobs[g.list.job[q]].stream = sidx;
        else failed.push_back({g.list.job[q], PF_ERR_CUDA});
      }
      if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        continue;
      }
      ginflight[sidx] += g.list.n;
      ++stats.group_launches;
      stats.max_group = std::max(stats.max_group, g.list.n);
    }
    lk.lock();
    if (!err.empty()) fatal = err;
    for (auto& f : failed) unclaim(f.first, f.second);
    return any;
  }

  // ---- coalesced batches ----

  // Takes the oldest run of kBatchMin or more batchable queued requests of
  // one case and options into a free batch slot (lock held), stages and
  // launches it without the lock.  Returns whether anything was admitted.
  bool admit_batches(std::unique_lock<std::mutex>& lk) {
    BatchSlot* bs = nullptr;
    for (BatchSlot& b : batches)
      if (b.reqs.empty()) {
        bs = &b;
        break;
      }
    if (!bs) return false;
    // the oldest request whose case has kBatchMin batchable requests queued
    std::unordered_map<pf_case, int> per_case;
    for (Request* r : queue)
      if (batchable(*r)) ++per_case[r->c];
    Request* head = nullptr;
    for (Request* r : queue) {
      if (batchable(*r) && per_case[r->c] >= kBatchMin) {
        head = r;
        break;
      }
    }
    if (!head) return false;
    std::vector<Request*> pick;
    const size_t per = slots_of(*head);
    const int cap = (int)std::min<size_t>(kBatchMax, std::max<size_t>(1, kBatchDoubles / per));
    size_t need = 0;
    for (Request* q : queue) {
      if ((int)pick.size() >= cap) break;
      if (!batchable(*q) || !same_batch(*head, *q)) continue;
      if (used + need + q->footprint > ctx->budget) break;
      pick.push_back(q);
      need += q->footprint;
    }
    if ((int)pick.size() < kBatchMin) return false;  // other options, or wait for memory
    for (Request* q : pick) begin(q);  // state 1: running
    queue.erase(std::remove_if(queue.begin(), queue.end(), [](const Request* q) { return q->state == 1; }),
                queue.end());
    bs->reqs = pick;
    bs->per = per;
    const int B = (int)pick.size();
    ++stats.batch_launches;
    stats.max_batch = std::max(stats.max_batch, B);
    lk.unlock();
    const int rc = launch_batch(*bs, B);
    lk.lock();
    if (rc != PF_OK) {
      for (Request* q : bs->reqs) {
        end(q);
        fail(q, rc);
      }
      bs->reqs.clear();
    }
    return true;
  }

  // Stages the batch's inputs, runs the batched solve and queues the copies
  // of its results (dispatcher thread, lock not held).
  int launch_batch(BatchSlot& bs, int B) {
    Request* r0 = bs.reqs[0];
    pf_case c = r0->c;
    const size_t per = bs.per, nb = per * (size_t)B;
    int rc = bs.ensure(nb, B);
    if (rc != PF_OK) return rc;
    rc = bs.ws.ensure(c->data.kind, c->data.n, std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu()),
                      B, 0);
    if (rc != PF_OK) return rc;
    const bool gen = !r0->p_gen.empty();
    parallel_for(B, nb * (gen ? 3 : 2) * sizeof(double), [&](int k) {
      const Request* r = bs.reqs[k];
      std::memcpy(bs.h_in + k * per, r->p_load.data(), per * sizeof(double));
      std::memcpy(bs.h_in + nb + k * per, r->q_load.data(), per * sizeof(double));
      if (gen) std::memcpy(bs.h_in + 2 * nb + k * per, r->p_gen.data(), per * sizeof(double));
    });
    cudaError_t e = cudaMemcpyAsync(bs.ws.st_p_load, bs.h_in, nb * sizeof(double),
                                    cudaMemcpyHostToDevice, bs.st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bs.ws.st_q_load, bs.h_in + nb, nb * sizeof(double),
                          cudaMemcpyHostToDevice, bs.st);
    if (e == cudaSuccess && gen)
      e = cudaMemcpyAsync(bs.ws.st_p_gen, bs.h_in + 2 * nb, nb * sizeof(double),
                          cudaMemcpyHostToDevice, bs.st);
    if (e != cudaSuccess) return cuda_error(e, "staging batch inputs");
    pf_opts o = r0->o;
    o.warm_start = 0;
    rc = run_solve(c, o, B, bs.ws.st_p_load, bs.ws.st_q_load, gen ? bs.ws.st_p_gen : nullptr,
                   &bs.ws, bs.st, RunMode::Solve, nullptr, nullptr, nullptr);
    if (rc != PF_OK) return rc;
    e = cudaMemcpyAsync(bs.h_out, bs.ws.st_vm, nb * sizeof(double), cudaMemcpyDeviceToHost, bs.st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bs.h_out + nb, bs.ws.st_va, nb * sizeof(double),
                          cudaMemcpyDeviceToHost, bs.st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bs.h_info, bs.ws.st_info, (size_t)B * sizeof(pf_info),
                          cudaMemcpyDeviceToHost, bs.st);
    if (e == cudaSuccess) e = cudaEventRecord(bs.ev, bs.st);
    return e == cudaSuccess ? PF_OK : cuda_error(e, "launching a coalesced batch");
  }

  // Hands each request of a finished batch its results: copied without the
  // lock (the requests are running, so nothing else touches their results),
  // retired with it.
  void finish_batch(BatchSlot& bs, std::unique_lock<std::mutex>& lk) {
    const int B = (int)bs.reqs.size();
    const size_t per = bs.per, nb = per * (size_t)B;
    lk.unlock();
    parallel_for(B, 2 * nb * sizeof(double), [&](int k) {
      Request* r = bs.reqs[k];
      r->vm.assign(bs.h_out + k * per, bs.h_out + (k + 1) * per);
      r->va.assign(bs.h_out + nb + k * per, bs.h_out + nb + (k + 1) * per);
      r->info = bs.h_info[k];
    });
    lk.lock();
    for (Request* r : bs.reqs) end(r);
    bs.reqs.clear();
  }

  // ---- per-request launches ----

  int start(Request* r, Slot& s) {
    pf_case c = r->c;
    const size_t per = slots_of(*r);
    int rc = s.io.ensure(per);
    if (rc != PF_OK) return rc;
    if (!s.h_info) {
      cudaError_t e = cudaMallocHost(&s.h_info, sizeof(pf_info));
      if (e != cudaSuccess) return cuda_error(e, "allocating pinned staging");
    }
    Workspace& ws = (c->data.kind == PF_SINGLE_PHASE) ? s.ws1ph : s.ws3ph;
    rc = ws.ensure(c->data.kind, c->data.n, std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu()), 1,
                   r->o.method == PF_NK ? r->o.gmres_restart : 0);
    if (rc != PF_OK) return rc;
    const double* d_in[3] = {nullptr, nullptr, nullptr};
    double* dst[3] = {ws.st_p_load, ws.st_q_load, ws.st_p_gen};
    const std::vector<double>* src[3] = {&r->p_load, &r->q_load, &r->p_gen};
    for (int k = 0; k < 3; ++k) {
      if (src[k]->empty()) continue;
      std::memcpy(s.io.h_in + k * per, src[k]->data(), per * sizeof(double));
      cudaError_t e = cudaMemcpyAsync(dst[k], s.io.h_in + k * per, per * sizeof(double),
                                      cudaMemcpyHostToDevice, s.st);
      if (e != cudaSuccess) return cuda_error(e, "staging request inputs");
      d_in[k] = dst[k];
    }
    pf_opts o = r->o;
    // these solves read the warm start only while no job of the case writes
    // it, and never write it
    if (!c->warm_valid || warm_writers[c] > 0) o.warm_start = 0;
    // per-request solves run on 8-CTA clusters so that every slot fits
    if (!o.cluster_size) o.cluster_size = 8;
    rc = run_solve_q(c, o, 1, d_in[0], d_in[1], d_in[2], &ws, s.st, nullptr, nullptr, nullptr,
                     /*warm_out=*/false);
    if (rc != PF_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(s.io.h_out, ws.st_vm, per * sizeof(double),
                                    cudaMemcpyDeviceToHost, s.st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s.io.h_out + per, ws.st_va, per * sizeof(double),
                          cudaMemcpyDeviceToHost, s.st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s.h_info, ws.st_info, sizeof(pf_info), cudaMemcpyDeviceToHost, s.st);
    if (e == cudaSuccess) e = cudaEventRecord(s.ev, s.st);
    if (e != cudaSuccess) return cuda_error(e, "launching a served solve");
    s.req = r;
    begin(r);
    return PF_OK;
  }

  void finish(Slot& s) {
    Request* r = s.req;
    const size_t per = slots_of(*r);
    s.req = nullptr;
    if (s.h_info->status != PF_OK && r->o.method == PF_NK && r->o.nk_fallback) {
      // Newton-Krylov ended without convergence: the request is solved again
      // with Newton-Raphson from a flat start, as pf_solve does
      r->nk_lin = s.h_info->linear_iterations;
      used -= r->footprint;
      --running;
      r->o.method = PF_NR;
      r->o.cluster_size = r->o.block_threads = r->o.scen_per_cta = 0;
      r->o.warm_start = 0;
      r->footprint = footprint(*r);
      r->state = 0;
      queue.push_front(r);
      return;
    }
    r->vm.assign(s.io.h_out, s.io.h_out + per);
    r->va.assign(s.io.h_out + per, s.io.h_out + 2 * per);
    r->info = *s.h_info;
    if (r->nk_lin >= 0) {
      r->info.fallback = 1;
      r->info.linear_iterations = r->nk_lin;
    }
    end(r);
  }

  bool admit_slots() {
    bool any = false;
    for (auto it = queue.begin(); it != queue.end();) {
      Request* r = *it;
      if (grouped(*r)) {
        ++it;
        continue;
      }
      Slot* free_slot = nullptr;
      for (Slot& s : slots)
        if (!s.req) {
          free_slot = &s;
          break;
        }
      if (!free_slot) break;
      if (used + r->footprint > ctx->budget) {
        if (running > 0) break;
        it = queue.erase(it);
        fail(r, PF_ERR_NOMEM);
        any = true;
        continue;
      }
      it = queue.erase(it);
      int rc = start(r, *free_slot);
      if (rc != PF_OK) fail(r, rc);
      any = true;
    }
    return any;
  }

  void loop() {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      bool progressed = false;
      for (int k = 0; k < kJobs; ++k) {
        if (jobs[k].req && __atomic_load_n(h_done + k, __ATOMIC_ACQUIRE) != 0) {
          retire(k);
          progressed = true;
        }
      }
      // a failed group launch: its jobs never raise their flags
      for (int q = 0; q < kGroupStreams; ++q) {
        if (ginflight[q] == 0) continue;
        const cudaError_t e = cudaStreamQuery(gst[q]);
        if (e == cudaSuccess || e == cudaErrorNotReady) continue;
        fatal = cudaGetErrorString(e);
        for (int k = 0; k < kJobs; ++k) {
          if (!jobs[k].req || jobs[k].stream != q) continue;
          --ginflight[q];
          unclaim(k, PF_ERR_CUDA);
        }
        progressed = true;
      }
      for (BatchSlot& b : batches) {
        if (b.reqs.empty()) continue;
        const cudaError_t q = cudaEventQuery(b.ev);
        if (q == cudaSuccess) {
          finish_batch(b, lk);
          progressed = true;
        } else if (q != cudaErrorNotReady) {
          fatal = cudaGetErrorString(q);
          for (Request* r : b.reqs) {
            end(r);
            fail(r, PF_ERR_CUDA);
          }
          b.reqs.clear();
          progressed = true;
        }
      }
      for (Slot& s : slots) {
        if (!s.req) continue;
        cudaError_t q = cudaEventQuery(s.ev);
        if (q == cudaSuccess) {
          finish(s);
          progressed = true;
        } else if (q != cudaErrorNotReady) {
          fatal = cudaGetErrorString(q);
          Request* r = s.req;
          s.req = nullptr;
          end(r);
          fail(r, PF_ERR_CUDA);
          progressed = true;
        }
      }
      if (!queue.empty()) {
        if (admit_slots()) progressed = true;
        if (admit_batches(lk)) progressed = true;
        if (!queue.empty() && admit_groups(lk)) progressed = true;
      }
      if (progressed) done_cv.notify_all();
      if (stop && queue.empty() && running == 0) break;
      if (running == 0 && queue.empty()) {
        cv.wait(lk);
      } else {
        // short sleeps keep the dispatcher cheap while kernels run
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(progressed ? 0 : 20));
        lk.lock();
      }
    }
  }

  int init(pf_ctx c) {
    ctx = c;
    cudaError_t e = cudaMallocHost(&h_desc, kJobs * sizeof(GroupJob));
    if (e == cudaSuccess) e = cudaMallocHost(&h_info, kJobs * sizeof(pf_info));
    if (e == cudaSuccess) e = cudaMallocHost(&h_done, kJobs * sizeof(int));
    if (e != cudaSuccess) return cuda_error(e, "allocating the serving descriptors");
    std::memset(h_done, 0, kJobs * sizeof(int));
    for (cudaStream_t& st : gst) {
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_error(e, "creating serving streams");
    }
    for (Slot& s : slots) {
      e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_error(e, "creating serving streams");
    }
    for (BatchSlot& b : batches) {
      e = cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_error(e, "creating serving streams");
    }
    th = std::thread([this] { loop(); });
    return PF_OK;
  }

  ~Server() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv.notify_all();
    if (th.joinable()) th.join();
    for (cudaStream_t st : gst)
      if (st) cudaStreamSynchronize(st);
    for (cudaStream_t st : gst)
      if (st) cudaStreamDestroy(st);
    for (Slot& s : slots) {
      if (s.st) cudaStreamDestroy(s.st);
      if (s.ev) cudaEventDestroy(s.ev);
      if (s.h_info) cudaFreeHost(s.h_info);
    }
    for (BatchSlot& b : batches) {
      if (b.st) cudaStreamSynchronize(b.st);
      if (b.st) cudaStreamDestroy(b.st);
      if (b.ev) cudaEventDestroy(b.ev);
    }
    if (h_desc) cudaFreeHost(h_desc);
    if (h_info) cudaFreeHost(h_info);
    if (h_done) cudaFreeHost(h_done);
  }
};

static Server* server_of(pf_ctx ctx, int* rc) {
  std::lock_guard<std::mutex> lk(ctx->server_mu);
  *rc = PF_OK;
  if (!ctx->server) {
    auto s = std::make_unique<Server>();
    *rc = s->init(ctx);
    if (*rc != PF_OK) return nullptr;
    ctx->server = s.release();
  }
  return ctx->server;
}

void serve_shutdown(pf_ctx ctx) {
  std::lock_guard<std::mutex> lk(ctx->server_mu);
  delete ctx->server;
  ctx->server = nullptr;
}

void serve_forget_case(pf_ctx ctx, pf_case c) {
  Server* sv;
  {
    std::lock_guard<std::mutex> lk(ctx->server_mu);
    sv = ctx->server;
  }
  if (!sv) return;
  std::unique_lock<std::mutex> lk(sv->mu);
  // drop queued requests of the case, wait for its running ones
  for (auto it = sv->queue.begin(); it != sv->queue.end();) {
    if ((*it)->c == c) {
      sv->fail(*it, PF_ERR_INVALID);
      it = sv->queue.erase(it);
    } else {
      ++it;
    }
  }
  sv->done_cv.wait(lk, [&] {
    for (Slot& s : sv->slots)
      if (s.req && s.req->c == c) return false;
    for (BatchSlot& b : sv->batches)
      if (!b.reqs.empty() && b.reqs[0]->c == c) return false;
    for (Job& j : sv->jobs)
      if (j.req && j.req->c == c) return false;
    return true;
  });
  sv->warm_readers.erase(c);
  sv->warm_writers.erase(c);
  for (auto& kv : sv->all)
    if (kv.second->c == c) kv.second->c = nullptr;
}

}  // namespace pf

using namespace pf;

extern "C" {

int pf_submit_batch(pf_ctx ctx, pf_case c, int B, const double* p_load, const double* q_load,
                    const double* p_gen, const pf_opts* opts, pf_ticket* out) {
  if (!ctx || !c || !out || B < 1) return set_error(PF_ERR_INVALID, "null argument or B < 1");
  if (c->ctx != ctx) return set_error(PF_ERR_INVALID, "the case belongs to another context");
  if (p_gen && c->data.kind != PF_SINGLE_PHASE)
    return set_error(PF_ERR_INVALID, "p_gen is for single-phase cases only");
  int rc;
  Server* sv = server_of(ctx, &rc);
  if (!sv) return rc;
  const size_t per = (size_t)c->data.n * (c->data.kind == PF_SINGLE_PHASE ? 1 : 3);
  std::vector<std::unique_ptr<Request>> rs(B);
  for (auto& r : rs) r = std::make_unique<Request>();
  const int given = (p_load != nullptr) + (q_load != nullptr) + (p_gen != nullptr);
  parallel_for(B, (size_t)given * per * B * sizeof(double), [&](int k) {
    Request* r = rs[k].get();
    r->c = c;
    if (opts) r->o = *opts; else pf_opts_default(&r->o);
    if (p_load) r->p_load.assign(p_load + k * per, p_load + (k + 1) * per);
    if (q_load) r->q_load.assign(q_load + k * per, q_load + (k + 1) * per);
    if (p_gen) r->p_gen.assign(p_gen + k * per, p_gen + (k + 1) * per);
  });
  std::lock_guard<std::mutex> lk(sv->mu);
  if (!sv->fatal.empty()) return set_error(PF_ERR_CUDA, "serving stopped: " + sv->fatal);
  if (sv->queue.size() + B > kMaxQueue) return set_error(PF_ERR_BUSY, "serving queue is full");
  {
    const int ki = c->data.kind == PF_SINGLE_PHASE ? 0 : 1;
    sv->max_n[ki] = std::max(sv->max_n[ki], c->data.n);
    sv->max_nnz[ki] = std::max(sv->max_nnz[ki], (long long)std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu()));
    sv->max_per[ki] = std::max(sv->max_per[ki], per);
  }
  // all B queued under one lock: the dispatcher sees them together
  for (int k = 0; k < B; ++k) {
    auto& r = rs[k];
    r->footprint = sv->footprint(*r);
    r->id = sv->next++;
    out[k] = r->id;
    sv->queue.push_back(r.get());
    sv->all.emplace(r->id, std::move(r));
  }
  sv->cv.notify_all();
  return PF_OK;
}

int pf_submit(pf_ctx ctx, pf_case c, const double* p_load, const double* q_load,
              const double* p_gen, const pf_opts* opts, pf_ticket* out) {
  return pf_submit_batch(ctx, c, 1, p_load, q_load, p_gen, opts, out);
}

int pf_poll(pf_ctx ctx, pf_ticket t, double* vmag, double* vang, pf_info* info) {
  if (!ctx) return set_error(PF_ERR_INVALID, "null context");
  int rc;
  Server* sv = server_of(ctx, &rc);
  if (!sv) return rc;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(t);
  if (it == sv->all.end()) return set_error(PF_ERR_INVALID, "unknown ticket");
  Request* r = it->second.get();
  if (r->state != 2) return PF_PENDING;
  if (vmag && !r->vm.empty()) std::copy(r->vm.begin(), r->vm.end(), vmag);
  if (vang && !r->va.empty()) std::copy(r->va.begin(), r->va.end(), vang);
  if (info) *info = r->info;
  sv->all.erase(it);
  return PF_OK;
}

int pf_serve_get_stats(pf_ctx ctx, pf_serve_stats* out) {
  if (!ctx || !out) return set_error(PF_ERR_INVALID, "null argument");
  std::memset(out, 0, sizeof(*out));
  Server* sv;
  {
    std::lock_guard<std::mutex> lk(ctx->server_mu);
    sv = ctx->server;
  }
  if (!sv) return PF_OK;
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->stats;
  return PF_OK;
}

int pf_drain(pf_ctx ctx, int timeout_ms) {
  if (!ctx) return set_error(PF_ERR_INVALID, "null context");
  Server* sv;
  {
    std::lock_guard<std::mutex> lk(ctx->server_mu);
    sv = ctx->server;
  }
  if (!sv) return PF_OK;
  std::unique_lock<std::mutex> lk(sv->mu);
  const bool ok = sv->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                       [&] { return sv->queue.empty() && sv->running == 0; });
  return ok ? PF_OK : set_error(PF_ERR_TIMEOUT, "requests still pending");
}

}  // extern "C"
