// Serving runtime: continuous admission of queued solves onto the GPU.
//
// Each context owns one dispatcher thread and a set of slots.  A slot is a
// CUDA stream with its own solve workspace and pinned host staging.  Requests
// wait in a FIFO queue; the dispatcher admits the head of the queue whenever a
// slot is free and the request's device footprint fits the context's HBM
// budget, launches its persistent Newton kernel on the slot's stream, and
// retires it when the stream's event completes.  Requests of different cases
// and sizes therefore run concurrently on different SMs, and a request that
// arrives while others are on the GPU starts as soon as a slot frees up.
#include <cuda_runtime.h>

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

constexpr int kSlots = 16;
constexpr size_t kMaxQueue = 1 << 20;

double now_us() {
  using namespace std::chrono;
  return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  pf_ticket id = 0;
  pf_case c = nullptr;
  pf_opts o{};
  std::vector<double> p_load, q_load, p_gen;  // empty = the case's own
  std::vector<double> vm, va;
  pf_info info{};
  int state = 0;  // 0 queued, 1 running, 2 done
  size_t footprint = 0;
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  // one workspace per case kind, so alternating single- and three-phase
  // requests do not reallocate (cudaFree would synchronise the device)
  Workspace ws1ph, ws3ph;
  Request* req = nullptr;
  double* h_in = nullptr;  // pinned: p_load, q_load, p_gen (3 * cap)
  double* h_out = nullptr; // pinned: vm, va (2 * cap)
  pf_info* h_info = nullptr;
  size_t cap = 0;          // doubles per staged vector
};

}  // namespace

struct Server {
  pf_ctx ctx = nullptr;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<Request*> queue;
  std::unordered_map<pf_ticket, std::unique_ptr<Request>> all;
  Slot slots[kSlots];
  size_t used = 0;  // device bytes of running requests
  int running = 0;
  bool stop = false;
  pf_ticket next = 1;
  std::string fatal;  // a CUDA failure that stopped the dispatcher

  size_t footprint(const Request& r) const {
    const pf_case c = r.c;
    return Workspace::bytes_for(c->data.kind, c->data.n,
                                std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu()), 1,
                                r.o.method == PF_NK ? r.o.gmres_restart : 0);
  }

  // Launch r on slot s (dispatcher thread, lock held).
  int start(Request* r, Slot& s) {
    pf_case c = r->c;
    const size_t per = (size_t)c->data.n * (c->data.kind == PF_SINGLE_PHASE ? 1 : 3);
    if (per > s.cap) {
      if (s.h_in) cudaFreeHost(s.h_in);
      if (s.h_out) cudaFreeHost(s.h_out);
      s.h_in = s.h_out = nullptr;
      s.cap = 0;
      cudaError_t e = cudaMallocHost(&s.h_in, 3 * per * sizeof(double));
      if (e == cudaSuccess) e = cudaMallocHost(&s.h_out, 2 * per * sizeof(double));
      if (e != cudaSuccess) return cuda_error(e, "allocating pinned staging");
      s.cap = per;
    }
    if (!s.h_info) {
      cudaError_t e = cudaMallocHost(&s.h_info, sizeof(pf_info));
      if (e != cudaSuccess) return cuda_error(e, "allocating pinned staging");
    }
    Workspace& ws = (c->data.kind == PF_SINGLE_PHASE) ? s.ws1ph : s.ws3ph;
    int rc = ws.ensure(c->data.kind, c->data.n,
                       std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu()), 1,
                       r->o.method == PF_NK ? r->o.gmres_restart : 0);
    if (rc != PF_OK) return rc;
    const double* d_in[3] = {nullptr, nullptr, nullptr};
    double* dst[3] = {ws.st_p_load, ws.st_q_load, ws.st_p_gen};
    const std::vector<double>* src[3] = {&r->p_load, &r->q_load, &r->p_gen};
    for (int k = 0; k < 3; ++k) {
      if (src[k]->empty()) continue;
      std::memcpy(s.h_in + k * per, src[k]->data(), per * sizeof(double));
      cudaError_t e = cudaMemcpyAsync(dst[k], s.h_in + k * per, per * sizeof(double),
                                      cudaMemcpyHostToDevice, s.st);
      if (e != cudaSuccess) return cuda_error(e, "staging request inputs");
      d_in[k] = dst[k];
    }
    pf_opts o = r->o;
    if (!c->warm_valid) o.warm_start = 0;
    // served solves run on 8-CTA clusters so that every slot fits on the GPU
    if (!o.cluster_size) o.cluster_size = 8;
    rc = run_solve_q(c, o, 1, d_in[0], d_in[1], d_in[2], &ws, s.st, nullptr, nullptr, nullptr);
    if (rc != PF_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(s.h_out, ws.st_vm, per * sizeof(double),
                                    cudaMemcpyDeviceToHost, s.st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s.h_out + per, ws.st_va, per * sizeof(double),
                          cudaMemcpyDeviceToHost, s.st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s.h_info, ws.st_info, sizeof(pf_info), cudaMemcpyDeviceToHost, s.st);
    if (e == cudaSuccess) e = cudaEventRecord(s.ev, s.st);
    if (e != cudaSuccess) return cuda_error(e, "launching a served solve");
    r->state = 1;
    s.req = r;
    used += r->footprint;
    ++running;
    return PF_OK;
  }

  void finish(Slot& s) {
    Request* r = s.req;
    const size_t per = (size_t)r->c->data.n * (r->c->data.kind == PF_SINGLE_PHASE ? 1 : 3);
    r->vm.assign(s.h_out, s.h_out + per);
    r->va.assign(s.h_out + per, s.h_out + 2 * per);
    r->info = *s.h_info;
    if (r->info.status == PF_OK) r->c->warm_valid = true;
    r->state = 2;
    used -= r->footprint;
    --running;
    s.req = nullptr;
  }

  void fail(Request* r, int code) {
    std::memset(&r->info, 0, sizeof(r->info));
    r->info.status = code;
    r->state = 2;
  }

  void loop() {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      bool progressed = false;
      for (Slot& s : slots) {
        if (!s.req) continue;
        cudaError_t q = cudaEventQuery(s.ev);
        if (q == cudaSuccess) {
          finish(s);
          progressed = true;
        } else if (q != cudaErrorNotReady) {
          fatal = cudaGetErrorString(q);
          fail(s.req, PF_ERR_CUDA);
          used -= s.req->footprint;
          --running;
          s.req = nullptr;
          progressed = true;
        }
      }
      while (!queue.empty()) {
        Request* r = queue.front();
        Slot* free_slot = nullptr;
        for (Slot& s : slots)
          if (!s.req) {
            free_slot = &s;
            break;
          }
        if (!free_slot) break;
        if (used + r->footprint > ctx->budget) {
          if (running > 0) break;  // wait for memory to free up
          queue.pop_front();       // can never fit, even alone
          fail(r, PF_ERR_NOMEM);
          progressed = true;
          continue;
        }
        queue.pop_front();
        int rc = start(r, *free_slot);
        if (rc != PF_OK) fail(r, rc);
        progressed = true;
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
    for (Slot& s : slots) {
      cudaError_t e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
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
    for (Slot& s : slots) {
      if (s.st) cudaStreamDestroy(s.st);
      if (s.ev) cudaEventDestroy(s.ev);
      if (s.h_in) cudaFreeHost(s.h_in);
      if (s.h_out) cudaFreeHost(s.h_out);
      if (s.h_info) cudaFreeHost(s.h_info);
    }
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
    return true;
  });
  for (auto& kv : sv->all)
    if (kv.second->c == c) kv.second->c = nullptr;
}

}  // namespace pf

using namespace pf;

extern "C" {

int pf_submit(pf_ctx ctx, pf_case c, const double* p_load, const double* q_load,
              const double* p_gen, const pf_opts* opts, pf_ticket* out) {
  if (!ctx || !c || !out) return set_error(PF_ERR_INVALID, "null argument");
  if (c->ctx != ctx) return set_error(PF_ERR_INVALID, "the case belongs to another context");
  if (p_gen && c->data.kind != PF_SINGLE_PHASE)
    return set_error(PF_ERR_INVALID, "p_gen is for single-phase cases only");
  int rc;
  Server* sv = server_of(ctx, &rc);
  if (!sv) return rc;
  auto r = std::make_unique<Request>();
  r->c = c;
  if (opts) r->o = *opts; else pf_opts_default(&r->o);
  const size_t per = (size_t)c->data.n * (c->data.kind == PF_SINGLE_PHASE ? 1 : 3);
  if (p_load) r->p_load.assign(p_load, p_load + per);
  if (q_load) r->q_load.assign(q_load, q_load + per);
  if (p_gen) r->p_gen.assign(p_gen, p_gen + per);
  std::lock_guard<std::mutex> lk(sv->mu);
  if (!sv->fatal.empty()) return set_error(PF_ERR_CUDA, "serving stopped: " + sv->fatal);
  if (sv->queue.size() >= kMaxQueue) return set_error(PF_ERR_BUSY, "serving queue is full");
  r->footprint = sv->footprint(*r);
  r->id = sv->next++;
  *out = r->id;
  sv->queue.push_back(r.get());
  sv->all.emplace(r->id, std::move(r));
  sv->cv.notify_all();
  return PF_OK;
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
