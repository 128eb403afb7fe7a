// C ABI of the power-flow library: contexts, cases, solves and inspection
// calls.  Host code only; every numeric step runs in the CUDA kernels of
// newton.cuh (single solves, Newton-Krylov, served requests), batch.cu
// (batched Newton-Raphson), flows.cu and qlim.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "api_internal.h"

namespace pf {

thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return set_error(PF_ERR_CUDA, m);
}

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------

DevBuffer::~DevBuffer() { release(); }

void DevBuffer::release() {
  for (void* p : ptrs) cudaFree(p);
  ptrs.clear();
  bytes = 0;
}

cudaError_t DevBuffer::alloc(void** out, size_t nbytes) {
  *out = nullptr;
  if (nbytes == 0) nbytes = 16;
  nbytes = (nbytes + 255) & ~size_t(255);
  cudaError_t e = cudaMalloc(out, nbytes);
  if (e == cudaSuccess) {
    ptrs.push_back(*out);
    bytes += nbytes;
  }
  return e;
}

template <class T>
static cudaError_t upload(DevBuffer& buf, const std::vector<T>& v, const T** out) {
  void* p;
  cudaError_t e = buf.alloc(&p, v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  *out = static_cast<const T*>(p);
  return e;
}

// ---------------------------------------------------------------------------
// system upload
// ---------------------------------------------------------------------------

// The kernels' packed records of a symbolic analysis, one 16-byte load per
// item: forward / backward sweep rows {row, first entry, end, 0} in level
// order; factor items {entry, pivot k, diagonal entry of k, 0}; targets
// {entry (| kFillFirst when a fill entry gets its first update, which then
// starts from zero), first L entry, first U entry, start of the rest in
// `con` or -1}; `con` holds the other (L, U) pairs of a target, each list
// ended by (-1, -1) (most targets receive one update per level).
static void pack_records(const Symbolic& s, std::vector<int4>& fwd, std::vector<int4>& bwd,
                         std::vector<int4>& fac, std::vector<int4>& tgt, std::vector<int2>& con) {
  const int n = s.n;
  fwd.assign(n, make_int4(0, 0, 0, 0));
  bwd.assign(n, make_int4(0, 0, 0, 0));
  fac.assign(s.fac_items.size(), make_int4(0, 0, 0, 0));
  tgt.assign(s.tgt_entry.size(), make_int4(0, 0, 0, 0));
  for (int t = 0; t < n; ++t) {
    const int i = s.flev_rows[t], j = s.blev_rows[t];
    fwd[t] = make_int4(i, s.lu_rowptr[i], s.lu_diag[i], 0);
    bwd[t] = make_int4(j, s.lu_diag[j] + 1, s.lu_rowptr[j + 1], 0);
  }
  for (size_t t = 0; t < fac.size(); ++t) {
    const int e = s.fac_items[t], k = s.lu_col[e];
    fac[t] = make_int4(e, k, s.lu_diag[k], 0);
  }
  con.clear();
  std::vector<char> touched(s.nnz_lu(), 0);
  for (size_t t = 0; t < tgt.size(); ++t) {
    const int c0 = s.tgt_cptr[t], c1 = s.tgt_cptr[t + 1];
    const int te = s.tgt_entry[t];
    const bool fill_first = s.lu2y[te] < 0 && !touched[te];
    touched[te] = 1;
    int rest = -1;
    if (c1 - c0 > 1) {
      rest = (int)con.size();
      for (int c = c0 + 1; c < c1; ++c) con.push_back(make_int2(s.con_l[c], s.con_u[c]));
      con.push_back(make_int2(-1, -1));
    }
    tgt[t] = make_int4(te | (fill_first ? kFillFirst : 0), s.con_l[c0], s.con_u[c0], rest);
  }
  if (con.empty()) con.push_back(make_int2(-1, -1));
}

int SysBuf::build(const CaseData& c, const Ybus& y, Ordering ord, bool fill) {
  analyze(y, ord, fill, sym);
  const int n = c.n;
  const Symbolic& s = sym;
  DevSys& d = view;
  std::memset(&d, 0, sizeof(d));
  d.kind = c.kind;
  d.n = n;
  // Ybus values in the new numbering
  const int vb = 2 * y.ybs * y.ybs;
  std::vector<double> yv((size_t)s.nnz_y() * vb);
  for (int e = 0; e < s.nnz_y(); ++e)
    std::copy(y.val.begin() + (size_t)s.y_src[e] * vb, y.val.begin() + (size_t)(s.y_src[e] + 1) * vb,
              yv.begin() + (size_t)e * vb);
  std::vector<int8_t> bt(n);
  std::vector<double> vset(n, 1.0), qg(n, 0.0), zip(3 * (size_t)n), pg(n, 0.0);
  std::vector<double> pl, ql, pg3;
  if (c.kind != PF_SINGLE_PHASE) pg3.assign(3 * (size_t)n, 0.0);
  if (c.kind == PF_SINGLE_PHASE) {
    pl.assign(n, 0.0);
    ql.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
      int o = s.perm[i];
      bt[i] = c.bus_type[o];
      vset[i] = c.v_set[o];
      qg[i] = c.q_gen[o];
      pg[i] = c.p_gen[o];
      pl[i] = c.p_load[o];
      ql[i] = c.q_load[o];
      for (int k = 0; k < 3; ++k) zip[3 * (size_t)i + k] = c.zip[3 * (size_t)o + k];
    }
  } else {
    pl.assign(3 * (size_t)n, 0.0);
    ql.assign(3 * (size_t)n, 0.0);
    for (int i = 0; i < n; ++i) {
      int o = s.perm[i];
      const bool pv = !c.bus_type.empty() && c.bus_type[o] == PF_PV;
      bt[i] = (int8_t)((c.phases[o] & 7) | (o == c.source ? 8 : 0) | (pv ? 16 : 0));
      vset[i] = c.v_set.empty() ? 1.0 : c.v_set[o];
      for (int k = 0; k < 3; ++k) {
        zip[3 * (size_t)i + k] = c.zip[3 * (size_t)o + k];
        pl[3 * (size_t)i + k] = c.p_load3[3 * (size_t)o + k];
        ql[3 * (size_t)i + k] = c.q_load3[3 * (size_t)o + k];
        pg3[3 * (size_t)i + k] = c.p_gen3.empty() ? 0.0 : c.p_gen3[3 * (size_t)o + k];
      }
    }
    d.v_source = c.v_source;
  }
  cudaError_t e = cudaSuccess;
#define UP(vec, field) \
  if (e == cudaSuccess) e = upload(mem, vec, &d.field)
  UP(s.y_rowptr, y_rowptr);
  UP(s.y_col, y_col);
  UP(yv, y_val);
  std::vector<float2> y32;
  if (c.kind == PF_SINGLE_PHASE) {
    y32.resize(s.nnz_y());
    for (int e = 0; e < s.nnz_y(); ++e) y32[e] = make_float2((float)yv[2 * e], (float)yv[2 * e + 1]);
  }
  UP(y32, y32);
  std::vector<float> zip32(zip.size());
  for (size_t k = 0; k < zip.size(); ++k) zip32[k] = (float)zip[k];
  UP(zip32, zip32);
  // cos and sin of j 2^-7 as 2^62 fixed point (long double on the host)
  std::vector<long long> trig(2 * (2 * kTrigHalf + 1));
  for (int j = -kTrigHalf; j <= kTrigHalf; ++j) {
    const long double a = (long double)j / 128.0L;
    trig[2 * (j + kTrigHalf)] = llroundl(cosl(a) * 4611686018427387904.0L);
    trig[2 * (j + kTrigHalf) + 1] = llroundl(sinl(a) * 4611686018427387904.0L);
  }
  UP(trig, trig);
  UP(s.lu_rowptr, lu_rowptr);
  UP(s.lu_col, lu_col);
  UP(s.lu_diag, lu_diag);
  UP(s.lu2y, lu2y);
  UP(s.fac_ptr, fac_ptr);
  UP(s.fac_items, fac_items);
  UP(s.tgt_ptr, tgt_ptr);
  UP(s.tgt_entry, tgt_entry);
  UP(s.tgt_cptr, tgt_cptr);
  UP(s.con_l, con_l);
  UP(s.con_u, con_u);
  UP(s.flev_ptr, flev_ptr);
  UP(s.flev_rows, flev_rows);
  UP(s.blev_ptr, blev_ptr);
  UP(s.blev_rows, blev_rows);
  UP(bt, btype);
  UP(vset, v_set);
  UP(qg, q_gen);
  UP(zip, zip);
  UP(pg, p_gen0);
  UP(pg3, p_gen3);
  UP(pl, p_load0);
  UP(ql, q_load0);
  d.q_min = d.q_max = nullptr;
  if (!c.q_max.empty()) {  // per bus, or per node and phase
    const int per = c.kind == PF_SINGLE_PHASE ? 1 : 3;
    std::vector<double> qmin((size_t)per * n), qmax((size_t)per * n);
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < per; ++a) {
        qmin[(size_t)i * per + a] = c.q_min[(size_t)s.perm[i] * per + a];
        qmax[(size_t)i * per + a] = c.q_max[(size_t)s.perm[i] * per + a];
      }
    UP(qmin, q_min);
    UP(qmax, q_max);
  }
  UP(s.perm, perm);
  std::vector<int> iperm(s.perm.size());
  for (size_t k = 0; k < s.perm.size(); ++k) iperm[s.perm[k]] = (int)k;
  UP(iperm, iperm);
  // packed per-item records (one 16-byte load each) for the kernels' prefetch
  std::vector<int4> fwd, bwd, fac, tgt;
  std::vector<int2> con;
  pack_records(s, fwd, bwd, fac, tgt, con);
  UP(fwd, fwd_rec);
  UP(bwd, bwd_rec);
  UP(fac, fac_rec);
  UP(tgt, tgt_rec);
  UP(con, con);
#undef UP
  d.nflev = (int)s.flev_ptr.size() - 1;
  d.nblev = (int)s.blev_ptr.size() - 1;
  if (e != cudaSuccess) return cuda_error(e, "uploading the symbolic analysis");
  return PF_OK;
}

// Lanes-per-row tables for a given number of threads per cluster (cached).
// A single solve gives a row up to one warp of lanes; a batch of S scenarios
// per CTA has threads / S row slots and gives a long row up to 64 lanes
// (summed across warps through shared memory).
int SysBuf::lanes_for(int threads, int S, DevSys& out) {
  std::lock_guard<std::mutex> lk(g_mu);
  const int rows = S > 1 ? threads / S : threads;
  const int key = 2 * rows + (S > 1 ? 1 : 0);
  auto it = g_cache.find(key);
  if (it == g_cache.end()) {
    const int cap = S > 1 ? 64 : 32;
    auto gw = lanes_per_level(sym.flev_ptr, sym.flev_llen, rows, cap);
    auto gb = lanes_per_level(sym.blev_ptr, sym.blev_ulen, rows, cap);
    std::array<const int8_t*, 2> arr{};
    cudaError_t e = upload(mem, gw, &arr[0]);
    if (e == cudaSuccess) e = upload(mem, gb, &arr[1]);
    if (e != cudaSuccess) return cuda_error(e, "uploading lane tables");
    it = g_cache.emplace(key, arr).first;
  }
  finish_view(it->second, threads, out);
  return PF_OK;
}

int SysBuf::lanes_cached(int threads, int S, DevSys& out) {
  std::lock_guard<std::mutex> lk(g_mu);
  const int rows = S > 1 ? threads / S : threads;
  auto it = g_cache.find(2 * rows + (S > 1 ? 1 : 0));
  if (it == g_cache.end())
    return set_error(PF_ERR_INVALID, "no lane tables were uploaded for this launch shape");
  finish_view(it->second, threads, out);
  return PF_OK;
}

void SysBuf::finish_view(const std::array<const int8_t*, 2>& g, int threads, DevSys& out) const {
  out = view;
  out.g_fwd = g[0];
  out.g_bwd = g[1];
  // the suffix of factor levels narrow enough for one CTA of `threads`
  int solo = (int)sym.flev_ptr.size() - 1;
  while (solo > 0) {
    const int l = solo - 1;
    const int items = std::max(sym.fac_ptr[l + 1] - sym.fac_ptr[l], sym.tgt_ptr[l + 1] - sym.tgt_ptr[l]);
    if (items > threads) break;
    --solo;
  }
  out.fac_solo_from = solo;
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------

size_t Workspace::bytes_for(int kind, int n, long long nnz_lu, int B, int m) {
  const int bs = kind == PF_SINGLE_PHASE ? 2 : 6;
  const int nsl = kind == PF_SINGLE_PHASE ? 1 : 3;
  size_t nb = (size_t)n * B;
  size_t t = 0;
  t += nb * (kind == PF_SINGLE_PHASE ? 3 : 6) * 8;      // spec
  t += (kind == PF_SINGLE_PHASE ? 2 : 0) * nb * 8;      // vm, va
  t += 2 * nb * nsl * 16;                               // V, dV
  t += (kind == PF_SINGLE_PHASE ? 16 : 0) * nb;         // U (FP64 solves)
  t += (kind == PF_SINGLE_PHASE ? 0 : 15) * nb * 8;     // abcd, PV reactive injection
  t += 3 * nb * bs * 8;                                 // F, dx, r
  t += (size_t)nnz_lu * B * bs * bs * 8;                // lu
  t += nb * bs * bs * 8;                                // uinv
  t += nb * bs * 8;                                     // y
  t += (size_t)B * (2 * 8 + 2 * 8 + 4 + 12) + 16 + 64;  // norm, step, flag, status, t0, call
  t += 3 * nb * nsl * 8;                                // staged inputs
  t += 2 * nb * nsl * 8 + (size_t)B * sizeof(pf_info);  // staged outputs
  t += nb * (kind == PF_SINGLE_PHASE ? 9 : 1)          // reactive-limit rounds
       + (size_t)B * (5 * 4 + 8 + sizeof(pf_info)) + 4;
  if (m > 0) {                                          // Newton-Krylov (FP64 bound)
    t += (size_t)nnz_lu * B * bs * bs * 8;              // Jacobian copy
    t += (size_t)(m + 1 + 3) * nb * bs * 8;             // basis, w, z, x
    t += (size_t)2 * 16 * B * kMaxJ * 8;                // reduction slots
  }
  return t;
}

int Workspace::ensure(int kind, int n, long long nnz_lu, int B, int m) {
  if (kind == cap_kind && B <= cap && m <= cap_m && n <= cap_n && nnz_lu <= cap_nnz) return PF_OK;
  if (kind == cap_kind) {  // grow every dimension, never shrink
    B = std::max(B, cap);
    m = std::max(m, cap_m);
    n = std::max(n, cap_n);
    nnz_lu = std::max(nnz_lu, cap_nnz);
  }
  mem.release();
  graph.reset();
  cap = 0;
  cap_m = -1;
  cap_kind = 0;
  cap_n = 0;
  cap_nnz = 0;
  const int bs = kind == PF_SINGLE_PHASE ? 2 : 6;
  const int nsl = kind == PF_SINGLE_PHASE ? 1 : 3;
  size_t nb = (size_t)n * B;
  std::memset(&w, 0, sizeof(w));
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = mem.alloc(p, bytes);
  };
  A((void**)&w.spec, nb * (kind == PF_SINGLE_PHASE ? 3 : 6) * 8);
  if (kind == PF_SINGLE_PHASE) {
    A((void**)&w.vm, nb * 8);
    A((void**)&w.va, nb * 8);
  }
  A((void**)&w.V, nb * nsl * 16);
  if (kind == PF_SINGLE_PHASE) A((void**)&w.U, nb * 16);
  A((void**)&w.dV, nb * nsl * 16);
  if (kind == PF_THREE_PHASE) A((void**)&w.abcd, nb * 12 * 8);
  if (kind == PF_THREE_PHASE) A((void**)&w.qg, nb * 3 * 8);
  A((void**)&w.F, nb * bs * 8);
  A((void**)&w.dx, nb * bs * 8);
  A((void**)&w.r, nb * bs * 8);
  A(&w.lu, (size_t)nnz_lu * B * bs * bs * 8);
  A(&w.uinv, nb * bs * bs * 8);
  A(&w.y, nb * bs * 8);
  A((void**)&w.norm, (size_t)2 * B * 8);
  A((void**)&w.step, (size_t)2 * B * 8);
  A((void**)&w.flag, (size_t)B * 4);
  A((void**)&w.status, (size_t)B * 4);
  A((void**)&w.refine, (size_t)B * 4);
  A((void**)&w.iter, (size_t)B * 4);
  A((void**)&w.t0, 8);
  A((void**)&w.anyref, 8);
  A((void**)&w.call, sizeof(CallArgs));
  A((void**)&st_p_load, nb * nsl * 8);
  A((void**)&st_q_load, nb * nsl * 8);
  A((void**)&st_p_gen, nb * nsl * 8);
  A((void**)&st_vm, nb * nsl * 8);
  A((void**)&st_va, nb * nsl * 8);
  A((void**)&st_info, (size_t)B * sizeof(pf_info));
  {  // reactive-limit rounds (three phase: held phases in bt, values in qg)
    A((void**)&w.bt, nb);
    if (kind == PF_SINGLE_PHASE) A((void**)&w.qsw, nb * 8);
    A((void**)&w.qdone, (size_t)B * 4);
    A((void**)&w.qcnt, (size_t)B * 4);
    A((void**)&w.qit, (size_t)3 * B * 4);
    A((void**)&w.qus, (size_t)B * 8);
    A((void**)&w.qinfo, (size_t)B * sizeof(pf_info));
    A((void**)&w.nsw, 4);
  }
  if (m > 0) {
    A(&w.jm, (size_t)nnz_lu * B * bs * bs * 8);
    A(&w.vb, (size_t)(m + 1) * nb * bs * 8);
    A(&w.wv, nb * bs * 8);
    A(&w.zg, nb * bs * 8);
    A(&w.xg, nb * bs * 8);
    A(&w.gred, (size_t)2 * 16 * B * kMaxJ * 8);
  }
  if (e != cudaSuccess) {
    mem.release();
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      return set_error(PF_ERR_NOMEM, "device memory exhausted for the solve workspace");
    }
    return cuda_error(e, "allocating the solve workspace");
  }
  cap = B;
  cap_m = m;
  cap_kind = kind;
  cap_n = n;
  cap_nnz = nnz_lu;
  w.B = B;
  return PF_OK;
}

}  // namespace pf

using namespace pf;

static void fill_stats(const CaseData& d, const Symbolic& nr, const Symbolic& nk,
                       pf_case_stats* out) {
  std::memset(out, 0, sizeof(*out));
  out->kind = d.kind;
  out->n_bus = d.n;
  out->block_size = d.kind == PF_SINGLE_PHASE ? 2 : 6;
  int unknowns = 0;
  if (d.kind == PF_SINGLE_PHASE) {
    for (int8_t t : d.bus_type) unknowns += (t == PF_PQ) ? 2 : (t == PF_PV ? 1 : 0);
  } else {
    for (int i = 0; i < d.n; ++i)
      if (i != d.source)
        for (int a = 0; a < 3; ++a) unknowns += ((d.phases[i] >> a) & 1) * 2;
  }
  out->n_unknowns = unknowns;
  out->nnz_y = nr.nnz_y();
  out->nnz_lu = nr.nnz_lu();
  out->n_updates = nr.n_updates;
  out->levels_factor = (int)nr.flev_ptr.size() - 1;
  out->levels_backward = (int)nr.blev_ptr.size() - 1;
  out->levels_ilu = (int)nk.flev_ptr.size() - 1;
  out->levels_ilu_backward = (int)nk.blev_ptr.size() - 1;
  out->bytes_per_scenario = (long long)Workspace::bytes_for(d.kind, d.n, nr.nnz_lu(), 1);
}


// ---------------------------------------------------------------------------
// exported functions
// ---------------------------------------------------------------------------

extern "C" {

void pf_opts_default(pf_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->method = PF_NR;
  o->precision = PF_MIXED;
  o->tol = 1e-8;
  o->max_iter = 30;
  o->refine_steps = 1;
  o->refine_below = 1e-3;
  o->refine_stall = 0.1;
  o->gmres_restart = 30;
  o->gmres_max_iter = 300;
  o->gmres_rtol = 1e-6;
  o->warm_start = 0;
  o->nk_fallback = 1;
}

const char* pf_last_error(void) { return g_last_error.c_str(); }

const char* pf_status_str(int s) {
  switch (s) {
    case PF_OK: return "PF_OK";
    case PF_PENDING: return "PF_PENDING";
    case PF_ERR_INVALID: return "PF_ERR_INVALID";
    case PF_ERR_NOMEM: return "PF_ERR_NOMEM";
    case PF_ERR_MAXITER: return "PF_ERR_MAXITER";
    case PF_ERR_DIVERGED: return "PF_ERR_DIVERGED";
    case PF_ERR_SINGULAR: return "PF_ERR_SINGULAR";
    case PF_ERR_TIMEOUT: return "PF_ERR_TIMEOUT";
    case PF_ERR_BUSY: return "PF_ERR_BUSY";
    case PF_ERR_CUDA: return "PF_ERR_CUDA";
    case PF_ERR_UNSUPPORTED: return "PF_ERR_UNSUPPORTED";
    default: return "unknown status";
  }
}

int pf_ctx_create(int device, size_t budget, pf_ctx* out) {
  if (!out) return set_error(PF_ERR_INVALID, "null output pointer");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceCount");
  if (device < 0 || device >= count) return set_error(PF_ERR_INVALID, "no such CUDA device");
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceProperties");
  auto ctx = std::make_unique<pf_ctx_s>();
  ctx->device = device;
  ctx->num_sms = prop.multiProcessorCount;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemGetInfo");
    budget = (size_t)(0.8 * (double)fr);
  }
  ctx->budget = budget;
  e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamCreate");
  *out = ctx.release();
  return PF_OK;
}

int pf_ctx_destroy(pf_ctx ctx) {
  if (!ctx) return set_error(PF_ERR_INVALID, "null context");
  cudaSetDevice(ctx->device);
  serve_shutdown(ctx);
  cudaStreamSynchronize(ctx->stream);
  cudaStreamDestroy(ctx->stream);
  delete ctx;
  return PF_OK;
}

int pf_create_case(pf_ctx ctx, const pf_case_desc* desc, pf_case* out) {
  if (!ctx || !out) return set_error(PF_ERR_INVALID, "null context or output pointer");
  *out = nullptr;
  auto c = std::make_unique<pf_case_s>();
  c->ctx = ctx;
  std::string err;
  int rc = copy_case(desc, c->data, err);
  if (rc != PF_OK) return set_error(rc, err);
  rc = build_ybus(c->data, c->y, err);
  if (rc != PF_OK) return set_error(rc, err);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  c->bs = c->data.kind == PF_SINGLE_PHASE ? 2 : 6;
  rc = c->nr.build(c->data, c->y, Ordering::MinDegree, true);
  if (rc != PF_OK) return rc;
  {
    // the lane tables of the entry point without allocation (and of served
    // single-CTA solves), uploaded now
    DevSys unused;
    rc = c->nr.lanes_for(pf::noalloc_threads(c->bs), 1, unused);
    if (rc != PF_OK) return rc;
  }
  {
    const int ki = c->data.kind == PF_SINGLE_PHASE ? 0 : 1;
    const long long nnz = std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu());
    int cur = ctx->max_n[ki].load();
    while (cur < c->data.n && !ctx->max_n[ki].compare_exchange_weak(cur, c->data.n)) {
    }
    long long curz = ctx->max_nnz[ki].load();
    while (curz < nnz && !ctx->max_nnz[ki].compare_exchange_weak(curz, nnz)) {
    }
  }
  rc = c->nk.build(c->data, c->y, Ordering::RCM, false);
  if (rc != PF_OK) return rc;
  // warm-start storage (new numbering of the NR ordering)
  const int n = c->data.n;
  e = c->mem.alloc((void**)&c->warm_vm, (size_t)n * 8);
  if (e == cudaSuccess) e = c->mem.alloc((void**)&c->warm_va, (size_t)n * 8);
  if (e == cudaSuccess) e = c->mem.alloc((void**)&c->warm_V, (size_t)n * 3 * 16);
  if (e != cudaSuccess) return cuda_error(e, "allocating warm-start storage");
  *out = c.release();
  return PF_OK;
}

int pf_destroy_case(pf_case c) {
  if (!c) return set_error(PF_ERR_INVALID, "null case");
  cudaSetDevice(c->ctx->device);
  serve_forget_case(c->ctx, c);
  cudaDeviceSynchronize();
  delete c;
  return PF_OK;
}

int pf_case_get_stats(pf_case c, pf_case_stats* out) {
  if (!c || !out) return set_error(PF_ERR_INVALID, "null argument");
  fill_stats(c->data, c->nr.sym, c->nk.sym, out);
  out->device_bytes = (long long)(c->nr.mem.bytes + c->nk.mem.bytes + c->mem.bytes);
  return PF_OK;
}

// Options of the Newton-Raphson redo of Newton-Krylov solves that did not
// converge: same precision and stopping rule, Newton-Raphson's own launch
// shapes, flat start.
static pf_opts fallback_opts(const pf_opts& o) {
  pf_opts r = o;
  r.method = PF_NR;
  r.cluster_size = 0;
  r.block_threads = 0;
  r.scen_per_cta = 0;
  r.warm_start = 0;
  return r;
}

int pf_solve(pf_case c, const pf_opts* opts, double* vmag, double* vang, pf_info* info) {
  if (!c) return set_error(PF_ERR_INVALID, "null case");
  pf_opts o;
  if (opts) o = *opts; else pf_opts_default(&o);
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->ctx->device);
  cudaStream_t st = c->ctx->stream;
  int rc = run_solve_q(c, o, 1, nullptr, nullptr, nullptr, &c->ws1, st, nullptr, nullptr,
                       nullptr);
  if (rc != PF_OK) return rc;
  pf_info inf;
  rc = fetch_results(c, &c->ws1, 1, vmag, vang, &inf, st);
  if (rc == PF_OK && o.method == PF_NK && o.nk_fallback && inf.status != PF_OK) {
    const int lin = inf.linear_iterations;
    rc = run_solve_q(c, fallback_opts(o), 1, nullptr, nullptr, nullptr, &c->ws1, st, nullptr,
                     nullptr, nullptr);
    if (rc == PF_OK) rc = fetch_results(c, &c->ws1, 1, vmag, vang, &inf, st);
    inf.fallback = 1;
    inf.linear_iterations = lin;  // the GMRES iterations spent before the redo
  }
  if (info) *info = inf;
  return rc;
}

// The device address of a host buffer the GPU can reach directly (pinned
// memory), or null (pageable memory, or no buffer).
static void* device_view(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int pf_solve_batch(pf_case c, int B, const double* p_load, const double* q_load,
                   const double* p_gen, const pf_opts* opts, double* vmag, double* vang,
                   pf_info* info) {
  if (!c || B < 1) return set_error(PF_ERR_INVALID, "null case or B < 1");
  if (p_gen && c->data.kind != PF_SINGLE_PHASE)
    return set_error(PF_ERR_INVALID, "p_gen is for single-phase cases only");
  pf_opts o;
  if (opts) o = *opts; else pf_opts_default(&o);
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->ctx->device);
  cudaStream_t st = c->ctx->stream;
  Workspace* ws = (B == 1) ? &c->ws1 : &c->wsB;
  int rc = ws->ensure(c->data.kind, c->data.n, std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu()), B,
                      o.method == PF_NK ? o.gmres_restart : 0);
  if (rc != PF_OK) return rc;
  const size_t per = (size_t)c->data.n * (c->data.kind == PF_SINGLE_PHASE ? 1 : 3);
  // A Newton-Raphson batch whose host buffers are all pinned: the set-up
  // kernel reads the inputs and the result kernels write the outputs over the
  // host link directly, with no staging copies around the solve.
  if (B > 1 && o.method == PF_NR && !(o.q_limits && !c->data.q_max.empty())) {
    const void* hp[6] = {p_load, q_load, p_gen, vmag, vang, info};
    void* dp[6];
    bool direct = true;
    for (int k = 0; k < 6; ++k) {
      dp[k] = device_view(hp[k]);
      if (hp[k] && !dp[k]) direct = false;
    }
    if (direct) {
      rc = run_solve(c, o, B, (const double*)dp[0], (const double*)dp[1], (const double*)dp[2],
                     ws, st, RunMode::Solve, (double*)dp[3], (double*)dp[4], (pf_info*)dp[5]);
      if (rc != PF_OK) return rc;
      const cudaError_t e = cudaStreamSynchronize(st);
      return e == cudaSuccess ? PF_OK : cuda_error(e, "running the solve");
    }
  }
  cudaError_t e = cudaSuccess;
  if (p_load) e = cudaMemcpyAsync(ws->st_p_load, p_load, per * B * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && q_load)
    e = cudaMemcpyAsync(ws->st_q_load, q_load, per * B * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && p_gen)
    e = cudaMemcpyAsync(ws->st_p_gen, p_gen, per * B * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "copying scenario inputs");
  rc = run_solve_q(c, o, B, p_load ? ws->st_p_load : nullptr, q_load ? ws->st_q_load : nullptr,
                 p_gen ? ws->st_p_gen : nullptr, ws, st, nullptr, nullptr, nullptr);
  if (rc != PF_OK) return rc;
  std::vector<pf_info> inf(B);
  rc = fetch_results(c, ws, B, vmag, vang, inf.data(), st);
  if (rc == PF_OK && o.method == PF_NK && o.nk_fallback) {
    // redo the scenarios that did not converge with Newton-Raphson, as one
    // batch of their own inputs
    std::vector<int> bad;
    for (int b = 0; b < B; ++b)
      if (inf[b].status != PF_OK) bad.push_back(b);
    if (!bad.empty()) {
      const int R = (int)bad.size();
      auto gather = [&](const double* src) {
        std::vector<double> v;
        if (!src) return v;
        v.resize(per * R);
        for (int k = 0; k < R; ++k)
          std::copy(src + per * bad[k], src + per * (bad[k] + 1), v.begin() + per * k);
        return v;
      };
      std::vector<double> pl = gather(p_load), ql = gather(q_load), pg = gather(p_gen);
      std::vector<double> vm(per * R), va(per * R);
      std::vector<pf_info> ri(R);
      Workspace* ws2 = (R == 1) ? &c->ws1 : &c->wsB;
      const pf_opts fo = fallback_opts(o);
      rc = ws2->ensure(c->data.kind, c->data.n,
                       std::max(c->nr.sym.nnz_lu(), c->nk.sym.nnz_lu()), R, 0);
      if (rc != PF_OK) return rc;
      e = cudaSuccess;
      if (p_load) e = cudaMemcpyAsync(ws2->st_p_load, pl.data(), per * R * 8, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess && q_load)
        e = cudaMemcpyAsync(ws2->st_q_load, ql.data(), per * R * 8, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess && p_gen)
        e = cudaMemcpyAsync(ws2->st_p_gen, pg.data(), per * R * 8, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_error(e, "copying scenario inputs");
      rc = run_solve_q(c, fo, R, p_load ? ws2->st_p_load : nullptr, q_load ? ws2->st_q_load : nullptr,
                     p_gen ? ws2->st_p_gen : nullptr, ws2, st, nullptr, nullptr, nullptr);
      if (rc == PF_OK) rc = fetch_results(c, ws2, R, vm.data(), va.data(), ri.data(), st);
      if (rc != PF_OK) return rc;
      for (int k = 0; k < R; ++k) {
        const int b = bad[k];
        if (vmag) std::copy(vm.begin() + per * k, vm.begin() + per * (k + 1), vmag + per * b);
        if (vang) std::copy(va.begin() + per * k, va.begin() + per * (k + 1), vang + per * b);
        ri[k].linear_iterations = inf[b].linear_iterations;
        ri[k].fallback = 1;
        inf[b] = ri[k];
      }
    }
  }
  if (info) std::copy(inf.begin(), inf.end(), info);
  return rc;
}

int pf_solve_batch_device(pf_case c, int B, const double* d_p_load, const double* d_q_load,
                          const double* d_p_gen, const pf_opts* opts, double* d_vmag,
                          double* d_vang, pf_info* d_info, void* stream) {
  if (!c || B < 1) return set_error(PF_ERR_INVALID, "null case or B < 1");
  if (d_p_gen && c->data.kind != PF_SINGLE_PHASE)
    return set_error(PF_ERR_INVALID, "p_gen is for single-phase cases only");
  pf_opts o;
  if (opts) o = *opts; else pf_opts_default(&o);
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->ctx->device);
  Workspace* ws = (B == 1) ? &c->ws1 : &c->wsB;
  return run_solve_q(c, o, B, d_p_load, d_q_load, d_p_gen, ws, (cudaStream_t)stream, d_vmag,
                     d_vang, d_info);
}

int pf_analyze(const pf_case_desc* desc, pf_case_stats* out) {
  if (!out) return set_error(PF_ERR_INVALID, "null output pointer");
  CaseData d;
  Ybus y;
  std::string err;
  int rc = copy_case(desc, d, err);
  if (rc == PF_OK) rc = build_ybus(d, y, err);
  if (rc != PF_OK) return set_error(rc, err);
  Symbolic nr, nk;
  analyze(y, Ordering::MinDegree, true, nr);
  analyze(y, Ordering::RCM, false, nk);
  fill_stats(d, nr, nk, out);
  // what pf_create_case uploads: both systems' arrays and Ybus values
  long long b = 0;
  for (const Symbolic* s : {&nr, &nk}) {
    b += 4LL * ((long long)s->y_rowptr.size() + s->y_col.size() + s->lu_rowptr.size() +
                s->lu_col.size() + s->lu_diag.size() + s->lu2y.size() + s->fac_ptr.size() +
                s->fac_items.size() + s->tgt_ptr.size() + s->tgt_entry.size() +
                s->tgt_cptr.size() + s->con_l.size() + s->con_u.size() +
                s->flev_ptr.size() + s->flev_rows.size() +
                s->blev_ptr.size() + s->blev_rows.size() + s->perm.size());
    b += (long long)y.val.size() * 8 + (long long)d.n * (1 + 8 * 9);
  }
  out->device_bytes = b;
  return PF_OK;
}

int pf_ybus(const pf_case_desc* desc, int64_t* nnz, int32_t* rowptr, int32_t* col,
            double* val) {
  if (!nnz) return set_error(PF_ERR_INVALID, "null nnz pointer");
  CaseData d;
  Ybus y;
  std::string err;
  int rc = copy_case(desc, d, err);
  if (rc == PF_OK) rc = build_ybus(d, y, err);
  if (rc != PF_OK) return set_error(rc, err);
  *nnz = y.nnz();
  if (!rowptr) return PF_OK;
  if (!col || !val) return set_error(PF_ERR_INVALID, "col and val are required with rowptr");
  std::copy(y.rowptr.begin(), y.rowptr.end(), rowptr);
  std::copy(y.col.begin(), y.col.end(), col);
  std::copy(y.val.begin(), y.val.end(), val);
  return PF_OK;
}

int pf_symbolic(const pf_case_desc* desc, int method, int32_t* perm, int32_t* rowptr,
                int32_t* col, int32_t* flevel, int32_t* blevel) {
  if (method != PF_NR && method != PF_NK)
    return set_error(PF_ERR_INVALID, "method must be PF_NR or PF_NK");
  CaseData d;
  Ybus y;
  std::string err;
  int rc = copy_case(desc, d, err);
  if (rc == PF_OK) rc = build_ybus(d, y, err);
  if (rc != PF_OK) return set_error(rc, err);
  Symbolic s;
  if (method == PF_NR) analyze(y, Ordering::MinDegree, true, s);
  else analyze(y, Ordering::RCM, false, s);
  if (perm) std::copy(s.perm.begin(), s.perm.end(), perm);
  if (rowptr) std::copy(s.lu_rowptr.begin(), s.lu_rowptr.end(), rowptr);
  if (col) std::copy(s.lu_col.begin(), s.lu_col.end(), col);
  for (int l = 0; l + 1 < (int)s.flev_ptr.size(); ++l)
    for (int t = s.flev_ptr[l]; t < s.flev_ptr[l + 1]; ++t)
      if (flevel) flevel[s.flev_rows[t]] = l;
  for (int l = 0; l + 1 < (int)s.blev_ptr.size(); ++l)
    for (int t = s.blev_ptr[l]; t < s.blev_ptr[l + 1]; ++t)
      if (blevel) blevel[s.blev_rows[t]] = l;
  return PF_OK;
}

int pf_schedule(const pf_case_desc* desc, int method, int64_t* sizes, int32_t* fac_ptr,
                int32_t* fac_rec, int32_t* tgt_ptr, int32_t* tgt_rec, int32_t* con,
                int32_t* flev_ptr, int32_t* fwd_rec, int32_t* blev_ptr, int32_t* bwd_rec) {
  if (!sizes) return set_error(PF_ERR_INVALID, "null sizes");
  if (method != PF_NR && method != PF_NK)
    return set_error(PF_ERR_INVALID, "method must be PF_NR or PF_NK");
  CaseData d;
  Ybus y;
  std::string err;
  int rc = copy_case(desc, d, err);
  if (rc == PF_OK) rc = build_ybus(d, y, err);
  if (rc != PF_OK) return set_error(rc, err);
  Symbolic s;
  if (method == PF_NR) analyze(y, Ordering::MinDegree, true, s);
  else analyze(y, Ordering::RCM, false, s);
  std::vector<int4> fwd, bwd, fac, tgt;
  std::vector<int2> cn;
  pack_records(s, fwd, bwd, fac, tgt, cn);
  if (s.fac_ptr.size() != s.flev_ptr.size() || s.tgt_ptr.size() != s.flev_ptr.size())
    return set_error(PF_ERR_INVALID, "factor and forward schedules differ in levels");
  sizes[0] = s.n;
  sizes[1] = (int64_t)s.flev_ptr.size() - 1;
  sizes[2] = (int64_t)s.blev_ptr.size() - 1;
  sizes[3] = (int64_t)fac.size();
  sizes[4] = (int64_t)tgt.size();
  sizes[5] = (int64_t)cn.size();
  auto put4 = [](const std::vector<int4>& v, int32_t* out) {
    if (!out) return;
    for (size_t k = 0; k < v.size(); ++k) {
      out[4 * k] = v[k].x;
      out[4 * k + 1] = v[k].y;
      out[4 * k + 2] = v[k].z;
      out[4 * k + 3] = v[k].w;
    }
  };
  if (fac_ptr) std::copy(s.fac_ptr.begin(), s.fac_ptr.end(), fac_ptr);
  if (tgt_ptr) std::copy(s.tgt_ptr.begin(), s.tgt_ptr.end(), tgt_ptr);
  if (flev_ptr) std::copy(s.flev_ptr.begin(), s.flev_ptr.end(), flev_ptr);
  if (blev_ptr) std::copy(s.blev_ptr.begin(), s.blev_ptr.end(), blev_ptr);
  put4(fac, fac_rec);
  put4(tgt, tgt_rec);
  put4(fwd, fwd_rec);
  put4(bwd, bwd_rec);
  if (con)
    for (size_t k = 0; k < cn.size(); ++k) {
      con[2 * k] = cn[k].x;
      con[2 * k + 1] = cn[k].y;
    }
  return PF_OK;
}

int pf_case_pattern(pf_case c, int32_t* rowptr, int32_t* col) {
  if (!c || !rowptr || !col) return set_error(PF_ERR_INVALID, "null argument");
  std::copy(c->y.rowptr.begin(), c->y.rowptr.end(), rowptr);
  std::copy(c->y.col.begin(), c->y.col.end(), col);
  return PF_OK;
}

int pf_eval_mismatch(pf_case c, const double* vmag, const double* vang, double* mis) {
  if (!c || !vmag || !vang || !mis) return set_error(PF_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(c->mu);
  return inspect(c, InspectKind::Mismatch, nullptr, vmag, vang, mis, nullptr);
}

int pf_eval_jacobian(pf_case c, const double* vmag, const double* vang, double* blocks) {
  if (!c || !vmag || !vang || !blocks) return set_error(PF_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(c->mu);
  return inspect(c, InspectKind::Jacobian, nullptr, vmag, vang, blocks, nullptr);
}

int pf_newton_step(pf_case c, const pf_opts* opts, const double* vmag, const double* vang,
                   double* dx, pf_info* info) {
  if (!c || !vmag || !vang || !dx) return set_error(PF_ERR_INVALID, "null argument");
  pf_opts o;
  if (opts) o = *opts; else pf_opts_default(&o);
  std::lock_guard<std::mutex> lk(c->mu);
  return inspect(c, InspectKind::Step, &o, vmag, vang, dx, info);
}

int pf_branch_flows(pf_case c, int B, const double* vmag, const double* vang, double* p_from,
                    double* q_from, double* p_to, double* q_to, double* loss) {
  if (!c || B < 1 || !vmag || !vang || !p_from || !q_from || !p_to || !q_to || !loss)
    return set_error(PF_ERR_INVALID, "null argument or B < 1");
  std::lock_guard<std::mutex> lk(c->mu);
  const CaseData& d = c->data;
  const int ph = d.kind == PF_SINGLE_PHASE ? 1 : 3, n = d.n, m = d.m;
  std::vector<double> yb, sh;
  std::string err;
  int rc = branch_admittances(d, yb, sh, err);
  if (rc != PF_OK) return set_error(rc, err);
  std::vector<int2> ft(m);
  for (int e = 0; e < m; ++e) ft[e] = make_int2(d.br_from[e], d.br_to[e]);
  cudaSetDevice(c->ctx->device);
  cudaStream_t st = c->ctx->stream;
  DevBuffer buf;
  const size_t nv = (size_t)B * n * ph, nf = (size_t)B * m * ph;
  int2* d_ft = nullptr;
  double *d_yb = nullptr, *d_sh = nullptr, *d_vm = nullptr, *d_va = nullptr, *d_out = nullptr;
  cudaError_t e = buf.alloc((void**)&d_ft, sizeof(int2) * std::max(m, 1));
  if (e == cudaSuccess) e = buf.alloc((void**)&d_yb, 8 * std::max<size_t>(yb.size(), 1));
  if (e == cudaSuccess) e = buf.alloc((void**)&d_sh, 8 * std::max(m, 1));
  if (e == cudaSuccess) e = buf.alloc((void**)&d_vm, 8 * nv);
  if (e == cudaSuccess) e = buf.alloc((void**)&d_va, 8 * nv);
  if (e == cudaSuccess) e = buf.alloc((void**)&d_out, 8 * (4 * nf + 2 * (size_t)B));
  if (e == cudaSuccess && m > 0) {
    e = cudaMemcpyAsync(d_ft, ft.data(), sizeof(int2) * m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_yb, yb.data(), 8 * yb.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_sh, sh.data(), 8 * m, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_vm, vmag, 8 * nv, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_va, vang, 8 * nv, cudaMemcpyHostToDevice, st);
  double* o = d_out;
  if (e == cudaSuccess)
    e = launch_branch_flows(ph, d_ft, d_yb, d_sh, n, m, B, d_vm, d_va, o, o + nf, o + 2 * nf,
                            o + 3 * nf, o + 4 * nf, st);
  double* outs[4] = {p_from, q_from, p_to, q_to};
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    if (nf) e = cudaMemcpyAsync(outs[k], o + k * nf, 8 * nf, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(loss, o + 4 * nf, 16 * (size_t)B, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "computing branch flows");
  return PF_OK;
}

int pf_autotune(pf_case c, int B, pf_opts* opts) {
  if (!c || !opts) return set_error(PF_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(c->mu);
  return autotune(c, B, opts);
}

int pf_launch_config(pf_case c, const pf_opts* opts, int B, int* grid, int* cluster,
                     int* threads, int* scen) {
  if (!c || B < 1 || !grid || !cluster || !threads || !scen)
    return set_error(PF_ERR_INVALID, "null argument or B < 1");
  pf_opts o;
  if (opts) o = *opts; else pf_opts_default(&o);
  cudaSetDevice(c->ctx->device);
  launch_shape(c, o, B, o.precision == PF_MIXED, grid, cluster, threads, scen);
  return PF_OK;
}

int pf_solve_noalloc(pf_case c, const pf_opts* opts, const double* d_p_load,
                     const double* d_q_load, const double* d_p_gen, double* d_vmag,
                     double* d_vang, pf_info* d_info, void* stream) {
  if (!c) return set_error(PF_ERR_INVALID, "null case");
  pf_opts o;
  if (opts) o = *opts; else pf_opts_default(&o);
  std::lock_guard<std::mutex> lk(c->mu);
  cudaError_t e = cudaSetDevice(c->ctx->device);
  if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  return solve_noalloc(c, o, d_p_load, d_q_load, d_p_gen, d_vmag, d_vang, d_info,
                       (cudaStream_t)stream);
}

int pf_profile_solve(pf_case c, int B, const pf_opts* opts, double* phase_us, pf_info* info) {
  if (!c || !phase_us || B < 1) return set_error(PF_ERR_INVALID, "null argument or B < 1");
  pf_opts o;
  if (opts) o = *opts; else pf_opts_default(&o);
  std::lock_guard<std::mutex> lk(c->mu);
  return profile_solve(c, B, o, phase_us, info);
}

}  // extern "C"
