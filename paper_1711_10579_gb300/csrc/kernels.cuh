// Device building blocks of the Newton power-flow kernels for sm_103a:
// complex and block arithmetic, the fused mismatch + Jacobian of one row
// (Eq. 1-10 single phase, Eq. 12-23 three phase), the team helpers, the
// level-scheduled block LU refactorisation and triangular sweeps, the GMRES
// reductions, and the per-row steps of an iteration.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>
#include <mutex>

#include "device.h"
#include "fixtrig.h"

static_assert(pf::kTrigHalf == pf::fx::kHalf, "one sine / cosine table size");

namespace cg = cooperative_groups;

namespace pf {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // a conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) {
  return make_double2(a.x * s, a.y * s);
}
__device__ __forceinline__ double2 ldc(const double2* p) { return __ldcg(p); }

// Asynchronous 16-byte copies global -> shared (cp.async, L2 only): a copy
// holds no register while in flight, so a thread can keep many gathers
// outstanding.  Each thread waits for its own groups of copies.
__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// FP64 -> FP32 rounded toward zero by integer instructions (fixtrig.h).
__device__ __forceinline__ float to_f32_trunc(double v) { return fx::to_f32_trunc(v); }

// |v| as an ordered bit pattern: non-negative doubles order like their bits,
// and a NaN of either sign maps above +inf.  Integer work only.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

// sin a and cos a: the table method in 64-bit fixed point on the integer
// pipes (fixtrig.h; four FP64-free conversions and a dozen 64-bit integer
// products), sincos() beyond |a| <= 4.
__device__ __forceinline__ void sincos_tab(const long long* tab, double a, double* s, double* c) {
  if (!fx::sincos_q(tab, a, s, c)) sincos(a, s, c);
}

// The FP64 refinement of a mixed-precision Newton-Raphson step is taken
// where the FP32 factors hold convergence back: the mismatch norm is at
// most refine_below and (refine_stall > 0) the last step cut it by less
// than 1 / refine_stall.
__device__ __forceinline__ bool refine_now(const DevOpts& o, int it, double nrm, double prev) {
  if (!(nrm <= o.refine_below)) return false;
  return o.refine_stall <= 0.0 || it == 0 || !(prev > 0.0) || nrm > o.refine_stall * prev;
}

template <bool CL>
__device__ __forceinline__ void csync() {
  if constexpr (CL) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// dense bs x bs blocks (row-major) in registers
// ---------------------------------------------------------------------------

template <int BS, typename T>
__device__ __forceinline__ void blk_load(const T* p, T (&a)[BS * BS]) {
  static_assert((BS * BS * sizeof(T)) % 16 == 0, "block must be 16-byte sized");
  constexpr int NV = BS * BS * (int)sizeof(T) / 16;
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    float4 t = __ldcg(q + v);
    const T* tt = reinterpret_cast<const T*>(&t);
#pragma unroll
    for (int k = 0; k < 16 / (int)sizeof(T); ++k) a[v * (16 / sizeof(T)) + k] = tt[k];
  }
}

template <int BS, typename T>
__device__ __forceinline__ void blk_store(T* p, const T (&a)[BS * BS]) {
  constexpr int NV = BS * BS * (int)sizeof(T) / 16;
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    float4 t;
    T* tt = reinterpret_cast<T*>(&t);
#pragma unroll
    for (int k = 0; k < 16 / (int)sizeof(T); ++k) tt[k] = a[v * (16 / sizeof(T)) + k];
    q[v] = t;
  }
}

template <int BS, typename T>
__device__ __forceinline__ void blk_mul(const T (&a)[BS * BS], const T (&b)[BS * BS],
                                        T (&c)[BS * BS]) {
#pragma unroll
  for (int i = 0; i < BS; ++i)
#pragma unroll
    for (int j = 0; j < BS; ++j) {
      T s = 0;
#pragma unroll
      for (int k = 0; k < BS; ++k) s += a[i * BS + k] * b[k * BS + j];
      c[i * BS + j] = s;
    }
}

template <int BS, typename T>
__device__ __forceinline__ void blk_msub(T (&c)[BS * BS], const T (&a)[BS * BS],
                                         const T (&b)[BS * BS]) {
#pragma unroll
  for (int i = 0; i < BS; ++i)
#pragma unroll
    for (int j = 0; j < BS; ++j) {
      T s = c[i * BS + j];
#pragma unroll
      for (int k = 0; k < BS; ++k) s -= a[i * BS + k] * b[k * BS + j];
      c[i * BS + j] = s;
    }
}

// Inverse by Gauss-Jordan elimination with partial pivoting inside the block.
// Returns false for a zero or non-finite pivot.
template <int BS, typename T>
__device__ __forceinline__ bool blk_inv(T (&a)[BS * BS], T (&inv)[BS * BS]) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < BS * BS; ++i) inv[i] = (i % (BS + 1) == 0) ? T(1) : T(0);
#pragma unroll
  for (int c = 0; c < BS; ++c) {
    int piv = c;
    T best = a[c * BS + c] < 0 ? -a[c * BS + c] : a[c * BS + c];
#pragma unroll
    for (int r = c + 1; r < BS; ++r) {
      T v = a[r * BS + c] < 0 ? -a[r * BS + c] : a[r * BS + c];
      if (v > best) {
        best = v;
        piv = r;
      }
    }
    if (!(best > T(0)) || !isfinite(best)) ok = false;
    // swap rows c and piv (unrolled selects keep the arrays in registers)
#pragma unroll
    for (int r = c + 1; r < BS; ++r) {
      if (r == piv) {
#pragma unroll
        for (int j = 0; j < BS; ++j) {
          T t = a[c * BS + j];
          a[c * BS + j] = a[r * BS + j];
          a[r * BS + j] = t;
          t = inv[c * BS + j];
          inv[c * BS + j] = inv[r * BS + j];
          inv[r * BS + j] = t;
        }
      }
    }
    T d = T(1) / a[c * BS + c];
#pragma unroll
    for (int j = 0; j < BS; ++j) {
      a[c * BS + j] *= d;
      inv[c * BS + j] *= d;
    }
#pragma unroll
    for (int r = 0; r < BS; ++r) {
      if (r == c) continue;
      T f = a[r * BS + c];
#pragma unroll
      for (int j = 0; j < BS; ++j) {
        a[r * BS + j] -= f * a[c * BS + j];
        inv[r * BS + j] -= f * inv[c * BS + j];
      }
    }
  }
  return ok;
}

template <typename T>
__device__ __forceinline__ T group_sum(T v, int G, unsigned gmask) {
  for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o, G);
  return v;
}

// ---------------------------------------------------------------------------
// step A: mismatch + Jacobian, single phase (polar unknowns, 2x2 blocks)
// ---------------------------------------------------------------------------

// Rows: (P, Q) equations of bus i; columns: (delta, |V|) of bus j.  The slack
// has no unknown and PV buses no |V| unknown: their rows become identity rows
// and their columns zero, which keeps the system of Eq. 10 unchanged.  With
// reactive limits enforced the types are the scenario's (w.bt): a PV bus at
// its limit is PQ with generation w.qsw.
template <typename TF>
__device__ void mismatch_jacobian_1ph(const DevSys& S, const DevWork& w, int i, int gs,
                                      double& nrm, TF* jcopy) {
  const int B = w.B;
  const size_t b = (size_t)i * B + gs;
  const int8_t* tp = w.bt ? w.bt + gs : S.btype;
  const size_t ts = w.bt ? (size_t)B : 1;
  const double2 Vi = ldc(w.V + b);
  const double vmi = __ldcg(w.vm + b);
  const double pl = __ldcg(w.spec + b * 3), ql = __ldcg(w.spec + b * 3 + 1),
               pg = __ldcg(w.spec + b * 3 + 2);
  const double zp = S.zip[3 * i], zi = S.zip[3 * i + 1], zz = S.zip[3 * i + 2];
  const int t = tp[i * ts];
  const double2* Y = reinterpret_cast<const double2*>(S.y_val);
  // The Jacobian is formed in the factor's precision TF: it only feeds the
  // factorisation (the mismatch and the refinement residual stay FP64).
  TF* lu = reinterpret_cast<TF*>(w.lu);
  auto put = [&](int e, TF j00, TF j01, TF j10, TF j11) {
    TF blk[4] = {j00, j01, j10, j11};
    blk_store<2>(lu + ((size_t)e * B + gs) * 4, blk);
    if (jcopy) blk_store<2>(jcopy + ((size_t)e * B + gs) * 4, blk);
  };
  // FP64 mismatch of Eq. 8-9 from the current I = sum_j Y_ij V_j (four FMAs
  // per entry) and S = V conj(I)
  double2 I = make_double2(0.0, 0.0);
  auto mismatch = [&]() {
    const double2 Sc = cmulc(Vi, I);
    const double shape = fma(fma(zz, vmi, zi), vmi, zp);
    const double f0 = (t != PF_SLACK) ? fma(-pl, shape, pg) - Sc.x : 0.0;
    const double qgen = (t == kPQLimit) ? __ldcg(w.qsw + b) : S.q_gen[i];
    const double f1 = (t >= PF_PQ) ? fma(-ql, shape, qgen) - Sc.y : 0.0;
    w.F[b * 2] = f0;
    w.F[b * 2 + 1] = f1;
    // max(|f0|, |f1|) on the bit patterns (NaN above +inf), no FP64 instruction
    nrm = __longlong_as_double((long long)max(abs_bits(f0), abs_bits(f1)));
    return Sc;
  };
  if constexpr (sizeof(TF) == 4) {
#pragma unroll 4
    for (int e = S.y_rowptr[i]; e < S.y_rowptr[i + 1]; ++e) {
      const int j = S.y_col[e];
      const double2 y = Y[e], v = ldc(w.V + (size_t)j * B + gs);
      I.x = fma(y.x, v.x, I.x);
      I.x = fma(-y.y, v.y, I.x);
      I.y = fma(y.x, v.y, I.y);
      I.y = fma(y.y, v.x, I.y);
    }
    mismatch();
    // The FP32 Jacobian over the factor's row, from the same neighbour
    // voltages (now in L1): the FP32 operands are cut from the FP64 values by
    // integer bit operations (conversion instructions would occupy the FP64
    // pipe of this GPU), so the assembly executes no FP64 instruction.
    const float vix = to_f32_trunc(Vi.x), viy = to_f32_trunc(Vi.y);
    const float Ix = to_f32_trunc(I.x), Iy = to_f32_trunc(I.y);
    const float pl32 = to_f32_trunc(pl), ql32 = to_f32_trunc(ql), vm32 = to_f32_trunc(vmi);
    float ydx = 0.f, ydy = 0.f;
    int ed = -1;
#pragma unroll 1
    for (int e = S.lu_rowptr[i]; e < S.lu_rowptr[i + 1]; ++e) {
      const int yi = S.lu2y[e];
      if (yi < 0) continue;  // fill entry: the factor starts it from zero
      const int j = S.lu_col[e];
      const float2 y32 = S.y32[yi];
      if (j == i) {
        ed = e;
        ydx = y32.x;
        ydy = y32.y;
        continue;
      }
      float j00 = 0.f, j01 = 0.f, j10 = 0.f, j11 = 0.f;
      const int tj = tp[j * ts];
      if (t != PF_SLACK && tj != PF_SLACK) {
        // c = V_i conj(Y_ij V_j): dS_i/d delta_j = -j c, dS_i/d|V_j| = c / |V_j|
        const double2 v = ldc(w.V + (size_t)j * B + gs);
        const float vjx = to_f32_trunc(v.x), vjy = to_f32_trunc(v.y);
        const float yvx = y32.x * vjx - y32.y * vjy, yvy = y32.x * vjy + y32.y * vjx;
        const float cx = vix * yvx + viy * yvy, cy = viy * yvx - vix * yvy;
        j00 = cy;
        j10 = -cx;
        if (tj >= PF_PQ) {
          const float rv = rsqrtf(fmaf(vjx, vjx, vjy * vjy));
          j01 = cx * rv;
          j11 = cy * rv;
        }
        if (t == PF_PV) j10 = j11 = 0.f;
      }
      put(e, j00, j01, j10, j11);
    }
    if (ed >= 0) {
      float j00, j01, j10, j11;
      if (t == PF_SLACK) {
        j00 = j11 = 1.f;
        j01 = j10 = 0.f;
      } else {
        // dS_i/d delta_i = j (S_i - V_i conj(Y_ii V_i));
        // dS_i/d|V_i| = U_i conj(I_i + Y_ii V_i), plus the load's slope
        const float rvi = rsqrtf(fmaf(vix, vix, viy * viy));
        const float uix = vix * rvi, uiy = viy * rvi;
        const float yvx = ydx * vix - ydy * viy, yvy = ydx * viy + ydy * vix;  // Y_ii V_i
        const float scx = vix * Ix + viy * Iy, scy = viy * Ix - vix * Iy;  // V_i conj(I_i)
        const float dx = vix * yvx + viy * yvy, dy = viy * yvx - vix * yvy;
        const float ax = Ix + yvx, ay = Iy + yvy;
        const float ex = uix * ax + uiy * ay, ey = uiy * ax - uix * ay;
        const float dshape = fmaf(2.f * S.zip32[3 * i + 2], vm32, S.zip32[3 * i + 1]);
        j00 = -(scy - dy);
        j10 = scx - dx;
        j01 = fmaf(pl32, dshape, ex);
        j11 = fmaf(ql32, dshape, ey);
        if (t == PF_PV) {
          j01 = 0.f;
          j10 = 0.f;
          j11 = 1.f;
        }
      }
      put(ed, j00, j01, j10, j11);
    }
  } else {
#pragma unroll 4
    for (int e = S.y_rowptr[i]; e < S.y_rowptr[i + 1]; ++e) {
      const int j = S.y_col[e];
      const double2 y = Y[e], v = ldc(w.V + (size_t)j * B + gs);
      I.x = fma(y.x, v.x, I.x);
      I.x = fma(-y.y, v.y, I.x);
      I.y = fma(y.x, v.y, I.y);
      I.y = fma(y.y, v.x, I.y);
    }
    const double2 Sc = mismatch();
    // U = V / |V| per bus (kept by the update in FP64 solves) avoids divisions
    const double2 Ui = ldc(w.U + b);
    const double dshape = fma(2.0 * zz, vmi, zi);
#pragma unroll 2
    for (int e = S.lu_rowptr[i]; e < S.lu_rowptr[i + 1]; ++e) {
      const int j = S.lu_col[e];
      const int yi = S.lu2y[e];
      if (yi < 0) continue;  // fill entry: the factor starts it from zero
      double j00 = 0, j01 = 0, j10 = 0, j11 = 0;
      {
        const double yx = Y[yi].x, yy = Y[yi].y;
        if (j != i) {
          const int tj = tp[j * ts];
          if (t != PF_SLACK && tj != PF_SLACK) {
            const size_t bj = (size_t)j * B + gs;
            // dS_i/d|V_j| = V_i conj(Y_ij U_j); dS_i/d delta_j = -j |V_j| dS_i/d|V_j|
            const double2 Uj = ldc(w.U + bj);
            const double vmj = __ldcg(w.vm + bj);
            const double yux = yx * Uj.x - yy * Uj.y, yuy = yx * Uj.y + yy * Uj.x;
            const double cx = Vi.x * yux + Vi.y * yuy, cy = Vi.y * yux - Vi.x * yuy;
            j00 = vmj * cy;
            j10 = -vmj * cx;
            if (tj >= PF_PQ) {
              j01 = cx;
              j11 = cy;
            }
            if (t == PF_PV) j10 = j11 = 0.0;
          }
        } else if (t == PF_SLACK) {
          j00 = j11 = 1.0;
        } else {
          const double yvx = yx * Vi.x - yy * Vi.y, yvy = yx * Vi.y + yy * Vi.x;  // Y_ii V_i
          const double dx = Vi.x * yvx + Vi.y * yvy, dy = Vi.y * yvx - Vi.x * yvy;
          const double ax = I.x + yvx, ay = I.y + yvy;
          const double ex = Ui.x * ax + Ui.y * ay, ey = Ui.y * ax - Ui.x * ay;
          j00 = -(Sc.y - dy);
          j10 = Sc.x - dx;
          j01 = ex + pl * dshape;
          j11 = ey + ql * dshape;
          if (t == PF_PV) {
            j01 = 0.0;
            j10 = 0.0;
            j11 = 1.0;
          }
        }
      }
      put(e, (TF)j00, (TF)j01, (TF)j10, (TF)j11);
    }
  }
}

// ---------------------------------------------------------------------------
// step A: current mismatch + Jacobian, three phase (6x6 blocks)
// ---------------------------------------------------------------------------

// Derivatives of the specified current I = conj(S(m)) V / m^2 (Eq. 17 with
// the ZIP load of Eq. 14-15, m = |V|) with respect to Re V and Im V, formed
// in complex arithmetic: dI/dVr = [conj(S') (Vr/m) V + conj(S)] / m^2
// - 2 conj(S) V Vr / m^4 and dI/dVi likewise with j conj(S).
__device__ __forceinline__ void load_slope(double2 V, double pl, double ql, double zp,
                                           double zi, double zz, double2& Isp,
                                           double2& dIdr, double2& dIdi) {
  const double m2 = V.x * V.x + V.y * V.y;
  const double m = sqrt(m2);
  const double shape = zp + zi * m + zz * m2;
  const double dshape = zi + 2.0 * zz * m;
  const double2 cS = make_double2(-pl * shape, ql * shape);     // conj(S)
  const double2 cSp = make_double2(-pl * dshape, ql * dshape);  // conj(dS/dm)
  const double inv2 = 1.0 / m2;                                 // the one division
  const double2 cSV = cmul(cS, V);
  Isp = cscale(cSV, inv2);
  const double2 base = cscale(cmul(cSp, V), inv2 * inv2 * m);   // / m^3
  dIdr = csub(cadd(cscale(base, V.x), cscale(cS, inv2)), cscale(cSV, 2.0 * V.x * inv2 * inv2));
  const double2 jcS = make_double2(-cS.y, cS.x);
  dIdi = csub(cadd(cscale(base, V.y), cscale(jcS, inv2)), cscale(cSV, 2.0 * V.y * inv2 * inv2));
}

template <typename TF>
__device__ void mismatch_jacobian_3ph(const DevSys& S, const DevWork& w, int i, int gs,
                                      double& nrm, TF* jcopy) {
  const int B = w.B;
  const size_t b = (size_t)i * B + gs;
  const int mask = S.btype[i] & 7;
  const bool src = (S.btype[i] & 8) != 0;
  const bool pv = (S.btype[i] & 16) != 0;
  double2 Vi[3], I[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Vi[a] = ldc(w.V + b * 3 + a);
    I[a] = make_double2(0.0, 0.0);
  }
  const double2* Y = reinterpret_cast<const double2*>(S.y_val);
  for (int e = S.y_rowptr[i]; e < S.y_rowptr[i + 1]; ++e) {
    const size_t bj = ((size_t)S.y_col[e] * B + gs) * 3;
    double2 Vj[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) Vj[c] = ldc(w.V + bj + c);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) I[a] = cadd(I[a], cmul(Y[(size_t)e * 9 + a * 3 + c], Vj[c]));
  }
  nrm = 0.0;
  double adj[12];  // a[3], b[3], c[3], d[3] of Eq. 23
  const double zp = S.zip[3 * i], zi = S.zip[3 * i + 1], zz = S.zip[3 * i + 2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const bool freea = ((mask >> a) & 1) && !src;
    double fim = 0.0, fre = 0.0;
    adj[a] = adj[3 + a] = adj[6 + a] = adj[9 + a] = 0.0;
    if (freea) {
      const double pl = __ldcg(w.spec + b * 6 + a), ql = __ldcg(w.spec + b * 6 + 3 + a);
      double2 Isp, dr, di;
      load_slope(Vi[a], pl, ql, zp, zi, zz, Isp, dr, di);
      if (pv) {
        // the generator of a PV node: constant P_g + j Q_g (Q_g solved for)
        double2 Ig, gr, gi;
        load_slope(Vi[a], -S.p_gen3[(size_t)i * 3 + a], -__ldcg(w.qg + b * 3 + a), 1.0, 0.0,
                   0.0, Ig, gr, gi);
        Isp = cadd(Isp, Ig);
        dr = cadd(dr, gr);
        di = cadd(di, gi);
      }
      const double2 dI = csub(Isp, I[a]);
      fim = dI.y;
      fre = dI.x;
      const double2 dS = cmulc(Vi[a], dI);
      double v = fmax(fabs(dS.x), fabs(dS.y));
      if (!isfinite(v)) v = __longlong_as_double(0x7ff8000000000000ULL);
      nrm = fmax(nrm, v);
      adj[a] = dr.y;      // a = d Im I_sp / d Vr
      adj[3 + a] = di.y;  // b = d Im I_sp / d Vi
      adj[6 + a] = dr.x;  // c = d Re I_sp / d Vr
      adj[9 + a] = di.x;  // d = d Re I_sp / d Vi
    }
    w.F[b * 6 + a] = fim;
    w.F[b * 6 + 3 + a] = fre;
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) w.abcd[b * 12 + k] = adj[k];

  TF* lu = reinterpret_cast<TF*>(w.lu);
  for (int e = S.lu_rowptr[i]; e < S.lu_rowptr[i + 1]; ++e) {
    const int j = S.lu_col[e];
    const int yi = S.lu2y[e];
    if (yi < 0) continue;  // fill entry: the factor starts it from zero
    TF blk[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) blk[k] = TF(0);
    {
      const int maskj = S.btype[j] & 7;
      const bool srcj = (S.btype[j] & 8) != 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const bool fa = ((mask >> a) & 1) && !src;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const bool fc = ((maskj >> c) & 1) && !srcj;
          if (fa && fc) {
            const double2 y = Y[(size_t)yi * 9 + a * 3 + c];
            // Eq. 21: rows (Im, Re) of the current, columns (Re, Im) of V
            blk[a * 6 + c] = (TF)y.y;
            blk[a * 6 + 3 + c] = (TF)y.x;
            blk[(3 + a) * 6 + c] = (TF)y.x;
            blk[(3 + a) * 6 + 3 + c] = (TF)(-y.y);
          }
        }
      }
      if (j == i) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const bool fa = ((mask >> a) & 1) && !src;
          if (fa) {  // Eq. 23
            blk[a * 6 + a] -= (TF)adj[a];
            blk[a * 6 + 3 + a] -= (TF)adj[3 + a];
            blk[(3 + a) * 6 + a] -= (TF)adj[6 + a];
            blk[(3 + a) * 6 + 3 + a] -= (TF)adj[9 + a];
          } else {
            blk[a * 6 + a] = TF(1);
            blk[(3 + a) * 6 + 3 + a] = TF(1);
          }
        }
      }
      if ((S.btype[j] & 16) && !srcj) {
        // PV column node: its phase c keeps |V| by dVr = -(Vi/Vr) dVi, so
        // the unknowns are (dQ_c, dVi_c): column 3 + c becomes col(Vi) -
        // (Vi/Vr) col(Vr), and column c carries d(Y V - I_sp)/dQ_c = j V / |V|^2,
        // nonzero only in the node's own rows of phase c.  A phase held at a
        // reactive limit (w.bt) keeps its plain columns.
        const size_t bj3 = ((size_t)j * B + gs) * 3;
        const int heldj = w.bt ? w.bt[(size_t)j * B + gs] : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (!((maskj >> c) & 1) || ((heldj >> c) & 1)) continue;
          const double2 v = (j == i) ? Vi[c] : ldc(w.V + bj3 + c);
          const TF rho = (TF)(v.y / v.x);
#pragma unroll
          for (int r = 0; r < 6; ++r) {
            blk[r * 6 + 3 + c] -= rho * blk[r * 6 + c];
            blk[r * 6 + c] = TF(0);
          }
          if (j == i) {
            const double m2 = v.x * v.x + v.y * v.y;
            blk[c * 6 + c] = (TF)(v.x / m2);
            blk[(3 + c) * 6 + c] = (TF)(-v.y / m2);
          }
        }
      }
    }
    blk_store<6>(lu + ((size_t)e * B + gs) * 36, blk);
    if (jcopy) blk_store<6>(jcopy + ((size_t)e * B + gs) * 36, blk);
  }
}

// ---------------------------------------------------------------------------
// cluster-wide schedule helpers
// ---------------------------------------------------------------------------

struct Team {
  int tid;       // thread index within the cluster
  int nthr;      // threads in the cluster (a multiple of S)
  int S;         // scenario slots per cluster (a power of two)
  int s0;        // first scenario of the cluster
  int ns;        // scenarios of the cluster (<= S)
  unsigned act;  // active scenarios (bit s = scenario s0 + s)
};

// Every thread serves the fixed scenario slot tid % S.  Runs fn(item, gs)
// for items [0, count) and every active scenario, then a cluster barrier.
template <bool CL, class Fn>
__device__ void run_items(const Team& tm, int count, Fn fn) {
  const int s = tm.tid & (tm.S - 1);
  if (s < tm.ns && ((tm.act >> s) & 1u)) {
    for (int it = tm.tid / tm.S; it < count; it += tm.nthr / tm.S) fn(it, tm.s0 + s);
  }
  csync<CL>();
}

// Runs fn(i, gs) for every row and active scenario, then a cluster barrier.
template <bool CL, class Fn>
__device__ void run_rows(const Team& tm, int n, Fn fn) {
  run_items<CL>(tm, n, fn);
}

// Like run_rows for an fn that returns a non-negative value per row: the
// largest value of each scenario (NaN above +inf) goes to base[gs], with one
// atomic per warp and scenario slot instead of one per row.
template <bool CL, class Fn>
__device__ void run_rows_max(const Team& tm, int n, unsigned long long* base, Fn fn) {
  const int s = tm.tid & (tm.S - 1);
  unsigned long long m = 0ull;
  if (s < tm.ns && ((tm.act >> s) & 1u)) {
    for (int it = tm.tid / tm.S; it < n; it += tm.nthr / tm.S) {
      m = max(m, abs_bits(fn(it, tm.s0 + s)));
    }
  }
  // the lanes of a warp with the same slot sit S apart
  for (int off = tm.S; off < 32; off <<= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((int)(threadIdx.x & 31) < tm.S && m != 0ull) atomicMax(base + tm.s0 + s, m);
  csync<CL>();
}

// ---------------------------------------------------------------------------
// level sweeps with prefetch of the next level's static data
// ---------------------------------------------------------------------------

// A thread's share of one row of a triangular sweep, loaded ahead: the row,
// its first entry for this lane, that entry's column and (2x2 blocks) value,
// and for the backward sweep the inverse diagonal block.  Factor values and
// indices do not change during the sweeps, so all of this is loaded before
// the previous level's barrier; only the solve vector is read after it.
template <int BS, typename TF>
struct RowPref {
  static constexpr int NV = (BS == 2) ? 4 : 1;
  int i, p, pe, k;
  TF v[NV], d[NV];
};

template <int BS, typename TF, bool FWD>
__device__ __forceinline__ void sweep_pref(const DevSys& S, const DevWork& w, const int4* rec,
                                           int pos, bool have, int gs, int lane,
                                           RowPref<BS, TF>& P) {
  P.i = -1;
  P.p = P.pe = 0;
  if (!have) return;
  const int4 q = __ldg(rec + pos);
  P.i = q.x;
  P.p = q.y + lane;
  P.pe = q.z;
  const TF* lu = reinterpret_cast<const TF*>(w.lu);
  if (P.p < P.pe) {
    P.k = __ldg(S.lu_col + P.p);
    if constexpr (BS == 2) blk_load<2>(lu + ((size_t)P.p * w.B + gs) * 4, P.v);
  }
  if constexpr (!FWD && BS == 2) {
    if (lane == 0) blk_load<2>(reinterpret_cast<const TF*>(w.uinv) + ((size_t)P.i * w.B + gs) * 4, P.d);
  }
}

// Forward: y_i -= sum_k L_ik y_k.  Backward: y_i = U_ii^-1 (y_i - sum_j U_ij y_j).
template <int BS, typename TF, bool FWD>
__device__ __forceinline__ void sweep_row(const DevSys& S, const DevWork& w, TF* y,
                                          const RowPref<BS, TF>& P, int gs, int lane, int G,
                                          unsigned gmask) {
  constexpr int BB = BS * BS;
  const int B = w.B;
  const TF* lu = reinterpret_cast<const TF*>(w.lu);
  TF acc[BS];
#pragma unroll
  for (int c = 0; c < BS; ++c) acc[c] = TF(0);
  for (int p = P.p; p < P.pe; p += G) {
    TF L[BB];
    int k;
    if (p == P.p) {
      k = P.k;
      if constexpr (BS == 2) {
#pragma unroll
        for (int t = 0; t < 4; ++t) L[t] = P.v[t];
      } else {
        blk_load<BS>(lu + ((size_t)p * B + gs) * BB, L);
      }
    } else {
      k = __ldg(S.lu_col + p);
      blk_load<BS>(lu + ((size_t)p * B + gs) * BB, L);
    }
    const size_t bk = ((size_t)k * B + gs) * BS;
    TF yk[BS];
#pragma unroll
    for (int c = 0; c < BS; ++c) yk[c] = y[bk + c];
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
      for (int c = 0; c < BS; ++c) acc[r] += L[r * BS + c] * yk[c];
  }
  if (G > 1) {
#pragma unroll
    for (int c = 0; c < BS; ++c) acc[c] = group_sum(acc[c], G, gmask);
  }
  if (lane == 0) {
    const size_t bi = ((size_t)P.i * B + gs) * BS;
    if constexpr (FWD) {
#pragma unroll
      for (int c = 0; c < BS; ++c) y[bi + c] = y[bi + c] - acc[c];
    } else {
      TF t[BS], D[BB];
#pragma unroll
      for (int c = 0; c < BS; ++c) t[c] = y[bi + c] - acc[c];
      if constexpr (BS == 2) {
#pragma unroll
        for (int q = 0; q < 4; ++q) D[q] = P.d[q];
      } else {
        blk_load<BS>(reinterpret_cast<const TF*>(w.uinv) + ((size_t)P.i * B + gs) * BB, D);
      }
#pragma unroll
      for (int r = 0; r < BS; ++r) {
        TF sacc = TF(0);
#pragma unroll
        for (int c = 0; c < BS; ++c) sacc += D[r * BS + c] * t[c];
        y[bi + r] = sacc;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// batched triangular sweeps (one CTA, S scenarios per CTA)
// ---------------------------------------------------------------------------

// A thread's share of one row of a batched sweep, loaded before any result of
// its level is stored: the row, this lane's first entry (column and, for 2x2
// blocks, value) and, for lane 0, the row's own right-hand side and (backward,
// 2x2 blocks) its inverse diagonal block.
template <int BS, typename TF>
struct BRow {
  static constexpr int NV = (BS == 2) ? 4 : 1;
  int i, p, pe, k;
  TF v[NV], d[NV], own[BS];
};

// Pointers and sizes of one batched sweep.
template <typename TF>
struct BSweep {
  const TF* lu;        // factor values [entry][scenario][BS x BS]
  const TF* uinv;      // inverse diagonal blocks [row][scenario][BS x BS]
  const int* col;      // factor columns
  TF* y;               // solve vector [row][scenario][BS]
  const double* rhs;   // forward: right-hand side (else y holds it)
  double* dx;          // backward: also written here (else only y)
  int accumulate;      // backward: dx += y instead of dx = y
  int B;
  const int* lev_ptr;  // level schedule and its row records
  const int4* rec;
  int nlev;
  const int8_t* gsz;   // lanes per row for each level
  TF* red;             // shared memory for the partial sums of lanes
  int4* srec;          // shared memory for kSweepStage row records, or null
  const int* refine;   // backward, dx not accumulated: dx only for the
                       // scenarios with bit 0 set (the others' step stays
                       // in y, where the update reads it), or null = all
};

// Rows of a wide level whose records one batched sweep stages in shared
// memory at a time (16 bytes each).
constexpr int kSweepStage = 1024;

template <int BS, typename TF, bool FWD>
__device__ __forceinline__ void brow_from(BRow<BS, TF>& P, const BSweep<TF>& a, int4 q, int lane,
                                          int gs) {
  P.i = q.x;
  P.p = q.y + lane;
  P.pe = q.z;
  if (P.p < P.pe) {
    P.k = __ldg(a.col + P.p);
    if constexpr (BS == 2) blk_load<2>(a.lu + ((size_t)P.p * a.B + gs) * 4, P.v);
  }
  if (lane == 0) {
    const size_t bi = ((size_t)P.i * a.B + gs) * BS;
#pragma unroll
    for (int c = 0; c < BS; ++c) P.own[c] = (FWD && a.rhs) ? (TF)__ldcg(a.rhs + bi + c) : a.y[bi + c];
    if constexpr (!FWD && BS == 2) blk_load<2>(a.uinv + ((size_t)P.i * a.B + gs) * 4, P.d);
  }
}

template <int BS, typename TF, bool FWD>
__device__ __forceinline__ void brow_load(BRow<BS, TF>& P, const BSweep<TF>& a, int pos, bool have,
                                          int lane, int gs) {
  P.i = -1;
  P.p = P.pe = 0;
  if (!have) return;
  brow_from<BS, TF, FWD>(P, a, __ldg(a.rec + pos), lane, gs);
}

// Entry p of a row: its column and block (from the row's prefetch when p is
// the lane's first entry).
template <int BS, typename TF>
__device__ __forceinline__ void brow_entry(const BRow<BS, TF>& P, const BSweep<TF>& a, int p,
                                           int gs, int& k, TF (&L)[BS * BS]) {
  if (BS == 2 && p == P.p) {
    k = P.k;
#pragma unroll
    for (int t = 0; t < BS * BS; ++t) L[t] = P.v[(BS == 2) ? t : 0];
  } else {
    k = (p == P.p) ? P.k : __ldg(a.col + p);
    blk_load<BS>(a.lu + ((size_t)p * a.B + gs) * BS * BS, L);
  }
}

// Forward: y_i = b_i - acc.  Backward: y_i = U_ii^-1 (y_i - acc), and dx
// unless nodx.
template <int BS, typename TF, bool FWD>
__device__ __forceinline__ void brow_finish(const BRow<BS, TF>& P, const BSweep<TF>& a, int gs,
                                            const TF (&acc)[BS], bool nodx) {
  constexpr int BB = BS * BS;
  const size_t bi = ((size_t)P.i * a.B + gs) * BS;
  TF t[BS];
#pragma unroll
  for (int c = 0; c < BS; ++c) t[c] = P.own[c] - acc[c];
  if constexpr (!FWD) {
    TF D[BB];
    if constexpr (BS == 2) {
#pragma unroll
      for (int q = 0; q < 4; ++q) D[q] = P.d[q];
    } else {
      blk_load<BS>(a.uinv + ((size_t)P.i * a.B + gs) * BB, D);
    }
    TF u[BS];
#pragma unroll
    for (int r = 0; r < BS; ++r) {
      u[r] = TF(0);
#pragma unroll
      for (int c = 0; c < BS; ++c) u[r] += D[r * BS + c] * t[c];
    }
#pragma unroll
    for (int c = 0; c < BS; ++c) t[c] = u[c];
  }
#pragma unroll
  for (int c = 0; c < BS; ++c) a.y[bi + c] = t[c];
  if (!FWD && a.dx && !nodx) {
#pragma unroll
    for (int c = 0; c < BS; ++c)
      a.dx[bi + c] = a.accumulate ? __ldcg(a.dx + bi + c) + (double)t[c] : (double)t[c];
  }
}

// Batched triangular sweep.  Every thread serves the scenario slot tid % S;
// the nthr / S row slots take a level's rows with G = gsz[l] lanes per row
// (G from the level's width and its longest row), so the long rows near the
// top of the elimination tree are split across lanes instead of being walked
// by one thread.  Lanes in one warp are summed with shuffles, lanes in
// different warps through shared memory, in a fixed order.  Levels with one
// lane per row take R rows at a time and issue all their loads before any
// store.  Each thread's first row of level l+1 is loaded while level l runs.
// Not inlined: it has the registers to itself.
template <int BS, typename TF, bool FWD>
__device__ __noinline__ void sweep_batch(const BSweep<TF> a, const Team tm) {
  constexpr int BB = BS * BS;
  // one row in flight per thread (more measured no faster: the extra
  // registers spill)
  const int NS = tm.S;
  const int slot = tm.tid & (NS - 1);
  const bool on = slot < tm.ns && ((tm.act >> slot) & 1u);
  const int gs = tm.s0 + slot;
  const int q = tm.tid / NS, nq = tm.nthr / NS;
  const bool nodx = !FWD && a.refine != nullptr && on && !(a.refine[gs] & 1);
  auto pref = [&](int l, BRow<BS, TF>& P) {
    const int G = a.gsz[l], base = a.lev_ptr[l], width = a.lev_ptr[l + 1] - base;
    const int group = q / G;
    brow_load<BS, TF, FWD>(P, a, base + group, on && group < width, q & (G - 1), gs);
  };
  BRow<BS, TF> cur, nxt;
  if (a.nlev > 0) pref(0, cur);
  for (int l = 0; l < a.nlev; ++l) {
    const int G = a.gsz[l], base = a.lev_ptr[l], width = a.lev_ptr[l + 1] - base;
    if (l + 1 < a.nlev) pref(l + 1, nxt);
    if (G == 1) {
      // one lane per row: row r goes to row slot r % nq
      auto row = [&](const BRow<BS, TF>& P) {
        TF acc[BS];
#pragma unroll
        for (int c = 0; c < BS; ++c) acc[c] = TF(0);
        for (int p = P.p; p < P.pe; ++p) {
          int k;
          TF L[BB];
          brow_entry<BS, TF>(P, a, p, gs, k, L);
          const size_t bk = ((size_t)k * a.B + gs) * BS;
#pragma unroll
          for (int rr = 0; rr < BS; ++rr)
#pragma unroll
            for (int c = 0; c < BS; ++c) acc[rr] += L[rr * BS + c] * a.y[bk + c];
        }
        if (P.i >= 0) brow_finish<BS, TF, FWD>(P, a, gs, acc, nodx);
      };
      if (on && q < width) row(cur);  // its record came during the last level
      if (a.srec && width > nq) {
        // the other rows' records staged in shared memory, kSweepStage at a
        // time, so that a row's loads start one round trip earlier
        for (int c0 = nq; c0 < width; c0 += kSweepStage) {
          const int c1 = min(c0 + kSweepStage, width);
          __syncthreads();  // the last chunk's readers are done
          for (int t = tm.tid; t < c1 - c0; t += tm.nthr) a.srec[t] = __ldg(a.rec + base + c0 + t);
          __syncthreads();
          if (on)
            for (int r = c0 + q; r < c1; r += nq) {
              BRow<BS, TF> P;
              brow_from<BS, TF, FWD>(P, a, a.srec[r - c0], 0, gs);
              row(P);
            }
        }
      } else if (on) {
        for (int r = q + nq; r < width; r += nq) {
          BRow<BS, TF> P;
          brow_load<BS, TF, FWD>(P, a, base + r, true, 0, gs);
          row(P);
        }
      }
    } else {
      // one row per group of G lanes (G * width <= nq)
      const int lane = q & (G - 1), group = q / G;
      TF acc[BS];
#pragma unroll
      for (int c = 0; c < BS; ++c) acc[c] = TF(0);
      for (int pp = cur.p; pp < cur.pe; pp += G) {
        int k;
        TF L[BB];
        brow_entry<BS, TF>(cur, a, pp, gs, k, L);
        const size_t bk = ((size_t)k * a.B + gs) * BS;
#pragma unroll
        for (int rr = 0; rr < BS; ++rr)
#pragma unroll
          for (int c = 0; c < BS; ++c) acc[rr] += L[rr * BS + c] * a.y[bk + c];
      }
      // lanes of one (row, slot) sit S threads apart
      const int GW = min(G, 32 / NS);
      for (int off = NS; off < NS * GW; off <<= 1) {
#pragma unroll
        for (int c = 0; c < BS; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
      }
      const bool row = cur.i >= 0;
      if (G > GW) {
        const int NW = G / GW;
        if (row && (lane & (GW - 1)) == 0) {
#pragma unroll
          for (int c = 0; c < BS; ++c) a.red[((group * NW + lane / GW) * NS + slot) * BS + c] = acc[c];
        }
        __syncthreads();
        if (row && lane == 0) {
#pragma unroll
          for (int c = 0; c < BS; ++c) acc[c] = TF(0);
          for (int wp = 0; wp < NW; ++wp) {
#pragma unroll
            for (int c = 0; c < BS; ++c) acc[c] += a.red[((group * NW + wp) * NS + slot) * BS + c];
          }
        }
      }
      if (row && lane == 0) brow_finish<BS, TF, FWD>(cur, a, gs, acc, nodx);
    }
    __syncthreads();
    cur = nxt;
  }
}

// One triangular sweep over all levels.  A single-scenario team gives each
// row gsz[l] lanes; a batch team gives each (row, scenario) one thread.  The
// first row of each group for level l+1 is prefetched while level l runs.
template <int BS, typename TF, bool FWD, bool CL>
__device__ void sweep(const DevSys& S, const DevWork& w, TF* y, const Team& tm,
                      const int* lev_ptr, const int4* rec, int nlev, const int8_t* gsz,
                      TF* red) {
  if constexpr (!CL) {
    if (tm.S > 1) {
      BSweep<TF> a;
      a.lu = reinterpret_cast<const TF*>(w.lu);
      a.uinv = reinterpret_cast<const TF*>(w.uinv);
      a.col = S.lu_col;
      a.y = y;
      a.rhs = nullptr;
      a.dx = nullptr;
      a.accumulate = 0;
      a.B = w.B;
      a.lev_ptr = lev_ptr;
      a.rec = rec;
      a.nlev = nlev;
      a.gsz = gsz;
      a.red = red;
      a.srec = nullptr;
      sweep_batch<BS, TF, FWD>(a, tm);
      return;
    }
  }
  const bool single = (tm.S == 1);
  const int slot = single ? 0 : (tm.tid & (tm.S - 1));
  const bool on = slot < tm.ns && ((tm.act >> slot) & 1u);
  const int gs = tm.s0 + slot;
  auto geom = [&](int l, int& G, int& group, int& lane, int& ngroups) {
    if (single) {
      G = gsz[l];
      group = tm.tid / G;
      lane = tm.tid % G;
      ngroups = tm.nthr / G;
    } else {
      G = 1;
      group = tm.tid / tm.S;
      lane = 0;
      ngroups = tm.nthr / tm.S;
    }
  };
  RowPref<BS, TF> cur, nxt;
  {
    int G, group, lane, ngroups;
    geom(0, G, group, lane, ngroups);
    const int base = lev_ptr[0], width = lev_ptr[1] - base;
    sweep_pref<BS, TF, FWD>(S, w, rec, base + group, on && nlev > 0 && group < width, gs, lane, cur);
  }
  for (int l = 0; l < nlev; ++l) {
    int G, group, lane, ngroups;
    geom(l, G, group, lane, ngroups);
    const int base = lev_ptr[l], width = lev_ptr[l + 1] - base;
    if (l + 1 < nlev) {
      int G2, group2, lane2, ng2;
      geom(l + 1, G2, group2, lane2, ng2);
      const int b2 = lev_ptr[l + 1], w2 = lev_ptr[l + 2] - b2;
      sweep_pref<BS, TF, FWD>(S, w, rec, b2 + group2, on && group2 < w2, gs, lane2, nxt);
    }
    if (on) {
      const unsigned gmask =
          (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
      if (group < width) sweep_row<BS, TF, FWD>(S, w, y, cur, gs, lane, G, gmask);
      for (int r = group + ngroups; r < width; r += ngroups) {
        RowPref<BS, TF> P;
        sweep_pref<BS, TF, FWD>(S, w, rec, base + r, true, gs, lane, P);
        sweep_row<BS, TF, FWD>(S, w, y, P, gs, lane, G, gmask);
      }
    }
    csync<CL>();
    cur = nxt;
  }
}

// Fan-out (right-looking) block LU of levels [l0, l1), L with identity
// diagonal blocks.  Level l, step 1: every pivot k of the level inverts its
// diagonal block (U_kk^-1 is stored) and every L entry (i, k) of the pivot
// columns becomes L_ik = A_ik U_kk^-1 -- all these entries received their
// last update at an earlier level.  Step 2: every entry (i, j) the level's
// pivots touch gathers A_ij -= sum_k L_ik U_kj in a fixed order (so results
// are deterministic).  A thread takes R items of a step at a time so that
// their loads overlap; the first record of each step is loaded before the
// barrier that precedes the step.  Not inlined: it has the registers to
// itself.
template <typename TF>
struct FactorArgs {
  TF* lu;
  TF* uinv;
  int* flag;
  int B;
  const int* fac_ptr;
  const int4* fac_rec;
  const int* tgt_ptr;
  const int4* tgt_rec;
  const int2* con;
  unsigned char* ring;  // shared memory for factor_pipe (batches of 2x2 blocks)
};

template <int BS, typename TF, bool CL>
__device__ __noinline__ void factor_run(const FactorArgs<TF> S, const Team tm, int l0, int l1) {
  if (l0 >= l1) return;
  constexpr int BB = BS * BS;
  // items in flight per thread: more than one measured no faster (the
  // extra registers spill)
  constexpr int R = 1;
  const int slot = tm.tid & (tm.S - 1);
  const bool on = slot < tm.ns && ((tm.act >> slot) & 1u);
  const int gs = tm.s0 + slot;
  const int first = tm.tid / tm.S, stride = tm.nthr / tm.S;
  TF* lu = S.lu;
  auto blk = [&](int e) { return lu + ((size_t)e * S.B + gs) * BB; };
  const int4 none = make_int4(-1, 0, 0, -1);
  auto fac_first = [&](int l) {
    const int f0 = S.fac_ptr[l], nf = S.fac_ptr[l + 1] - f0;
    return (on && first < nf) ? __ldg(S.fac_rec + f0 + first) : none;
  };
  auto tgt_first = [&](int l) {
    const int t0 = S.tgt_ptr[l], nt = S.tgt_ptr[l + 1] - t0;
    return (on && first < nt) ? __ldg(S.tgt_rec + t0 + first) : none;
  };
  int4 fr = fac_first(l0);
  for (int l = l0; l < l1; ++l) {
    const int4 tr = tgt_first(l);  // for step 2, loaded ahead
    // step 1: r = {e, k, diag(k)}: U_kk^-1 for the diagonal, else L_ik = A_ik U_kk^-1
    if (on) {
      const int f0 = S.fac_ptr[l], nf = S.fac_ptr[l + 1] - f0;
      for (int t = first; t < nf; t += R * stride) {
        int4 r[R];
        TF d[R][BB], a[R][BB];
#pragma unroll
        for (int u = 0; u < R; ++u) {
          const int tu = t + u * stride;
          r[u] = (u == 0 && t == first) ? fr : (tu < nf ? __ldg(S.fac_rec + f0 + tu) : none);
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
          if (r[u].x >= 0) {
            blk_load<BS>(blk(r[u].z), d[u]);
            if (r[u].x != r[u].z) blk_load<BS>(blk(r[u].x), a[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
          if (r[u].x < 0) continue;
          TF di[BB];
          const bool ok = blk_inv<BS>(d[u], di);
          if (r[u].x == r[u].z) {
            if (!ok) S.flag[gs] = 1;
            blk_store<BS>(S.uinv + ((size_t)r[u].y * S.B + gs) * BB, di);
          } else {
            TF lk[BB];
            blk_mul<BS>(a[u], di, lk);
            blk_store<BS>(blk(r[u].x), lk);
          }
        }
      }
    }
    csync<CL>();
    fr = (l + 1 < l1) ? fac_first(l + 1) : none;  // for the next level's step 1
    // step 2: r = {e, L entry, U entry, rest}: A_e -= L U, then the rest
    const int t0 = S.tgt_ptr[l], nt = S.tgt_ptr[l + 1] - t0;
    if (nt > 0) {
      if (on) {
        for (int t = first; t < nt; t += R * stride) {
          int4 r[R];
          TF c[R][BB], lv[R][BB], uv[R][BB];
#pragma unroll
          for (int u = 0; u < R; ++u) {
            const int tu = t + u * stride;
            r[u] = (u == 0 && t == first) ? tr : (tu < nt ? __ldg(S.tgt_rec + t0 + tu) : none);
          }
#pragma unroll
          for (int u = 0; u < R; ++u) {
            if (r[u].x >= 0) {
              if (r[u].x & kFillFirst) {
                r[u].x &= ~kFillFirst;
#pragma unroll
                for (int q = 0; q < BB; ++q) c[u][q] = TF(0);
              } else {
                blk_load<BS>(blk(r[u].x), c[u]);
              }
              blk_load<BS>(blk(r[u].y), lv[u]);
              blk_load<BS>(blk(r[u].z), uv[u]);
            }
          }
#pragma unroll
          for (int u = 0; u < R; ++u) {
            if (r[u].x < 0) continue;
            blk_msub<BS>(c[u], lv[u], uv[u]);
            if (r[u].w >= 0) {
              for (int q = r[u].w;; ++q) {
                const int2 cq = __ldg(S.con + q);
                if (cq.x < 0) break;
                TF l2[BB], u2[BB];
                blk_load<BS>(blk(cq.x), l2);
                blk_load<BS>(blk(cq.y), u2);
                blk_msub<BS>(c[u], l2, u2);
              }
            }
            blk_store<BS>(blk(r[u].x), c[u]);
          }
        }
      }
      csync<CL>();
    }
  }
}

// Depth of factor_pipe's per-thread ring of items (2x2 blocks).
template <typename TF>
struct FactorPipe {
  static constexpr int D = sizeof(TF) == 4 ? 4 : 2;  // items in flight
  static constexpr int NV = 4 * (int)sizeof(TF) / 16;  // 16-byte pieces per block
  // bytes per thread: D slots of three blocks and 2 D records
  static constexpr int bytes = D * 3 * NV * 16 + 2 * D * 16;
};

// The factorisation of factor_run for a batch of 2x2 blocks (one CTA), with
// its gathers staged through shared memory: every thread keeps the blocks of
// its next D items and the records of the D after those in flight by
// cp.async while it computes the current item, so the wide levels are not
// bound by one load latency per item.  Shared memory is laid out [piece]
// [thread] in 16-byte units so that a warp's accesses do not conflict.  The
// next step's first records are requested before each barrier.
template <typename TF>
__device__ __noinline__ void factor_pipe(const FactorArgs<TF> S, const Team tm, int l0, int l1) {
  if (l0 >= l1) return;
  using P = FactorPipe<TF>;
  constexpr int D = P::D, NV = P::NV, BB = 4;
  const int slot = tm.tid & (tm.S - 1);
  const bool on = slot < tm.ns && ((tm.act >> slot) & 1u);
  const int gs = tm.s0 + slot;
  const int first = tm.tid / tm.S, stride = tm.nthr / tm.S;
  const int T = blockDim.x;
  uint4* R = reinterpret_cast<uint4*>(S.ring);
  // block c (0..2) of item slot d, piece v; record slot m (0..2D-1)
  auto blk_at = [&](int d, int c, int v) { return R + ((d * 3 + c) * NV + v) * T + threadIdx.x; };
  auto rec_at = [&](int m) { return R + (D * 3 * NV + m) * T + threadIdx.x; };
  auto gblk = [&](int e) { return S.lu + ((size_t)e * S.B + gs) * BB; };
  auto fetch_blk = [&](int d, int c, int e) {
#pragma unroll
    for (int v = 0; v < NV; ++v) cp16(blk_at(d, c, v), gblk(e) + v * (16 / sizeof(TF)));
  };
  auto read_blk = [&](int d, int c, TF (&a)[BB]) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const uint4 q = *blk_at(d, c, v);
      const TF* t = reinterpret_cast<const TF*>(&q);
#pragma unroll
      for (int k = 0; k < 16 / (int)sizeof(TF); ++k) a[v * (16 / sizeof(TF)) + k] = t[k];
    }
  };
  // items of one step: records rec[base + first + k * stride], k < K
  auto count = [&](int n) { return (on && first < n) ? (n - first + stride - 1) / stride : 0; };
  auto fetch_recs = [&](const int4* rec, int K) {
    for (int k = 0; k < D && k < K; ++k) cp16(rec_at(k), rec + first + k * stride);
    cp_commit();
  };
  // one step: fetch(d, r) requests the blocks of record r into item slot d,
  // work(d, r) computes the item and stores its result
  auto step = [&](const int4* rec, int K, auto fetch, auto work) {
    cp_wait<0>();  // this step's first records
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (k < K) {
        const int4 r = *reinterpret_cast<const int4*>(rec_at(k));
        fetch(k, r);
        if (k + D < K) cp16(rec_at(k + D), rec + first + (k + D) * stride);
      }
      cp_commit();
    }
    for (int k = 0; k < K; ++k) {
      cp_wait<D - 1>();
      const int4 r = *reinterpret_cast<const int4*>(rec_at(k % (2 * D)));
      work(k % D, r);
      const int k2 = k + D;
      if (k2 < K) {
        const int4 r2 = *reinterpret_cast<const int4*>(rec_at(k2 % (2 * D)));
        fetch(k % D, r2);
        if (k2 + D < K) cp16(rec_at(k % (2 * D)), rec + first + (k2 + D) * stride);
      }
      cp_commit();
    }
  };
  // step 1: r = {e, k, diag(k)}: U_kk^-1 for the diagonal, else L_ik = A_ik U_kk^-1
  auto fetch1 = [&](int d, int4 r) {
    fetch_blk(d, 0, r.z);
    if (r.x != r.z) fetch_blk(d, 1, r.x);
  };
  auto work1 = [&](int d, int4 r) {
    TF a[BB], di[BB];
    read_blk(d, 0, a);
    const bool ok = blk_inv<2>(a, di);
    if (r.x == r.z) {
      if (!ok) S.flag[gs] = 1;
      blk_store<2>(S.uinv + ((size_t)r.y * S.B + gs) * BB, di);
    } else {
      TF x[BB], lk[BB];
      read_blk(d, 1, x);
      blk_mul<2>(x, di, lk);
      blk_store<2>(gblk(r.x), lk);
    }
  };
  // step 2: r = {e, L entry, U entry, rest}: A_e -= L U, then the rest
  auto fetch2 = [&](int d, int4 r) {
    if (!(r.x & kFillFirst)) fetch_blk(d, 0, r.x);
    fetch_blk(d, 1, r.y);
    fetch_blk(d, 2, r.z);
  };
  auto work2 = [&](int d, int4 r) {
    TF c[BB], lv[BB], uv[BB];
    if (r.x & kFillFirst) {
#pragma unroll
      for (int q = 0; q < BB; ++q) c[q] = TF(0);
    } else {
      read_blk(d, 0, c);
    }
    read_blk(d, 1, lv);
    read_blk(d, 2, uv);
    blk_msub<2>(c, lv, uv);
    if (r.w >= 0) {
      for (int q = r.w;; ++q) {
        const int2 cq = __ldg(S.con + q);
        if (cq.x < 0) break;
        TF l2[BB], u2[BB];
        blk_load<2>(gblk(cq.x), l2);
        blk_load<2>(gblk(cq.y), u2);
        blk_msub<2>(c, l2, u2);
      }
    }
    blk_store<2>(gblk(r.x & ~kFillFirst), c);
  };
  fetch_recs(S.fac_rec + S.fac_ptr[l0], count(S.fac_ptr[l0 + 1] - S.fac_ptr[l0]));
  for (int l = l0; l < l1; ++l) {
    const int f0 = S.fac_ptr[l], nf = S.fac_ptr[l + 1] - f0;
    step(S.fac_rec + f0, count(nf), fetch1, work1);
    const int t0 = S.tgt_ptr[l], nt = S.tgt_ptr[l + 1] - t0;
    fetch_recs(S.tgt_rec + t0, count(nt));
    __syncthreads();
    if (nt > 0) {
      step(S.tgt_rec + t0, count(nt), fetch2, work2);
      if (l + 1 < l1) fetch_recs(S.fac_rec + S.fac_ptr[l + 1], count(S.fac_ptr[l + 2] - S.fac_ptr[l + 1]));
      __syncthreads();
    } else if (l + 1 < l1) {
      cp_wait<0>();
      fetch_recs(S.fac_rec + S.fac_ptr[l + 1], count(S.fac_ptr[l + 2] - S.fac_ptr[l + 1]));
    }
  }
  cp_wait<0>();
}

// Depth of factor_warp's per-thread ring of items (2x2 blocks) and its
// shared memory per thread: D slots of three blocks, no records.
template <typename TF>
struct FactorWarp {
  static constexpr int D = sizeof(TF) == 4 ? 8 : 4;    // items in flight per warp
  static constexpr int NV = 4 * (int)sizeof(TF) / 16;  // 16-byte pieces per block
  static constexpr int bytes = D * 3 * NV * 16;
};

// The factorisation of factor_pipe with the 32 lanes of a warp on 32
// scenarios of the same item (S = 32): every block load is one contiguous
// 32-scenario segment and the item records are the same for the whole warp.
// A warp takes the items w, w + W, ... of a step (W warps); lane j loads the
// record of the warp's item 32 b + j, and the record of any item in flight is
// broadcast from the two batches held in registers, so the shared-memory ring
// holds block data only and keeps D items per warp in flight.  The 2x2
// pivot block is inverted in closed form (adjugate over the determinant); a
// zero or non-finite determinant or inverse marks the scenario singular.
template <typename TF>
__device__ __noinline__ void factor_warp(const FactorArgs<TF> S, const Team tm, int l0, int l1) {
  if (l0 >= l1) return;
  using P = FactorWarp<TF>;
  constexpr int D = P::D, NV = P::NV, BB = 4;
  static_assert(D < 32, "an item in flight lies in one of two record batches");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool on = lane < tm.ns && ((tm.act >> lane) & 1u);
  const int gs = tm.s0 + lane;
  const int T = blockDim.x;
  uint4* R = reinterpret_cast<uint4*>(S.ring);
  auto at = [&](int d, int c, int v) { return R + ((d * 3 + c) * NV + v) * T + threadIdx.x; };
  auto gblk = [&](int e) { return S.lu + ((size_t)e * S.B + gs) * BB; };
  auto fetch_blk = [&](int d, int c, int e) {
#pragma unroll
    for (int v = 0; v < NV; ++v) cp16(at(d, c, v), gblk(e) + v * (16 / sizeof(TF)));
  };
  auto read_blk = [&](int d, int c, TF (&a)[BB]) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const uint4 q = *at(d, c, v);
      const TF* t = reinterpret_cast<const TF*>(&q);
#pragma unroll
      for (int k = 0; k < 16 / (int)sizeof(TF); ++k) a[v * (16 / sizeof(TF)) + k] = t[k];
    }
  };
  const int4 none = make_int4(-1, 0, 0, -1);
  // items of a step for this warp, and lane's record of batch b
  auto count = [&](int n) { return n > wid ? (n - wid + nw - 1) / nw : 0; };
  // Steps alternate their direction (step 1 forward, step 2 backward): a
  // step starts on the blocks the previous step touched last, the ones most
  // likely still in L2 (factor 15.4 -> 15.2 ms per 4,864-scenario step).
  int rev = 0, nstep = 0;
  auto batch = [&](const int4* rec, int K, int b) {
    const int k = 32 * b + lane;
    const int idx = wid + k * nw;
    return k < K ? __ldg(rec + (rev ? nstep - 1 - idx : idx)) : none;
  };
  auto bcast = [&](int4 x, int src) {
    return make_int4(__shfl_sync(0xffffffffu, x.x, src), __shfl_sync(0xffffffffu, x.y, src),
                     __shfl_sync(0xffffffffu, x.z, src), __shfl_sync(0xffffffffu, x.w, src));
  };
  // one step: fetch(d, r) requests the blocks of record r into slot d,
  // work(d, r) computes the item and stores its result; first = the
  // warp's first record batch, loaded before the barrier that precedes it
  auto step = [&](const int4* rec, int K, int4 first, auto fetch, auto work) {
    int4 ra = first, rb = K > 32 ? batch(rec, K, 1) : none;
    int base = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (k < K) {
        const int4 r = bcast(ra, k);
        if (on) fetch(k, r);
      }
      cp_commit();
    }
    for (int k = 0; k < K; ++k) {
      cp_wait<D - 1>();
      const int4 r = bcast(ra, k - base);
      if (on) work(k % D, r);
      const int k2 = k + D;
      if (k2 < K) {
        const int o = k2 - base;
        const int4 r2 = bcast(o < 32 ? ra : rb, o & 31);
        if (on) fetch(k % D, r2);
      }
      cp_commit();
      if (k + 1 - base == 32) {
        ra = rb;
        base += 32;
        rb = base + 32 < K ? batch(rec, K, base / 32 + 1) : none;
      }
    }
  };
  // step 1: r = {e, k, diag(k)}: U_kk^-1 for the diagonal, else L_ik = A_ik U_kk^-1
  auto fetch1 = [&](int d, int4 r) {
    fetch_blk(d, 0, r.z);
    if (r.x != r.z) fetch_blk(d, 1, r.x);
  };
  auto work1 = [&](int d, int4 r) {
    TF a[BB];
    read_blk(d, 0, a);
    const TF det = a[0] * a[3] - a[1] * a[2];
    const TF rd = TF(1) / det;
    TF di[BB] = {a[3] * rd, -a[1] * rd, -a[2] * rd, a[0] * rd};
    if (r.x == r.z) {
      if (!(det != TF(0)) || !isfinite(di[0]) || !isfinite(di[1]) || !isfinite(di[2]) ||
          !isfinite(di[3]))
        S.flag[gs] = 1;
      blk_store<2>(S.uinv + ((size_t)r.y * S.B + gs) * BB, di);
    } else {
      TF x[BB], lk[BB];
      read_blk(d, 1, x);
      blk_mul<2>(x, di, lk);
      blk_store<2>(gblk(r.x), lk);
    }
  };
  // step 2: r = {e, L entry, U entry, rest}: A_e -= L U, then the rest
  auto fetch2 = [&](int d, int4 r) {
    if (!(r.x & kFillFirst)) fetch_blk(d, 0, r.x);
    fetch_blk(d, 1, r.y);
    fetch_blk(d, 2, r.z);
  };
  auto work2 = [&](int d, int4 r) {
    TF c[BB], lv[BB], uv[BB];
    if (r.x & kFillFirst) {
#pragma unroll
      for (int q = 0; q < BB; ++q) c[q] = TF(0);
    } else {
      read_blk(d, 0, c);
    }
    read_blk(d, 1, lv);
    read_blk(d, 2, uv);
    blk_msub<2>(c, lv, uv);
    if (r.w >= 0) {
      for (int q = r.w;; ++q) {
        const int2 cq = __ldg(S.con + q);
        if (cq.x < 0) break;
        TF l2[BB], u2[BB];
        blk_load<2>(gblk(cq.x), l2);
        blk_load<2>(gblk(cq.y), u2);
        blk_msub<2>(c, l2, u2);
      }
    }
    blk_store<2>(gblk(r.x & ~kFillFirst), c);
  };
  int f0 = S.fac_ptr[l0], nf = S.fac_ptr[l0 + 1] - f0;
  nstep = nf;
  int4 first = batch(S.fac_rec + f0, count(nf), 0);
  for (int l = l0; l < l1; ++l) {
    rev = 0;
    nstep = nf;
    step(S.fac_rec + f0, count(nf), first, fetch1, work1);
    const int t0 = S.tgt_ptr[l], nt = S.tgt_ptr[l + 1] - t0;
    rev = 1;
    nstep = nt;
    first = batch(S.tgt_rec + t0, count(nt), 0);
    cp_wait<0>();
    __syncthreads();
    if (nt > 0) {
      step(S.tgt_rec + t0, count(nt), first, fetch2, work2);
      cp_wait<0>();
    }
    if (l + 1 < l1) {
      f0 = S.fac_ptr[l + 1];
      nf = S.fac_ptr[l + 2] - f0;
      rev = 0;
      nstep = nf;
      first = batch(S.fac_rec + f0, count(nf), 0);
    }
    if (nt > 0) __syncthreads();
  }
}

// One level of factor_run for one scenario (S = 1), a warp per item with the
// lanes on the entries of the block: lane t computes entries t and t + 32 of
// a product, and the rows of the augmented matrix [A | I] of blk_inv's
// Gauss-Jordan elimination are updated by all lanes at once.  Every entry
// goes through the same operations in the same order as in blk_inv /
// blk_mul / blk_msub, so results are bit for bit those of factor_run.
// This GPU's FP64 pipe takes a warp instruction per 64 cycles per SM
// sub-partition however many lanes are active, so a 6x6 FP64 item of ~1,000
// FP64 instructions in one thread holds a narrow level for ~30 us; spread
// over the lanes an item is ~150 warp instructions (more per item than 32
// items a warp, so wide levels stay a thread per item).  The warps of every
// CTA of the team take items (CL: a cluster).
template <int BS, typename TF>
struct FactorCoop {
  static constexpr int kWarps = 8;     // warps of a CTA that take items
  static constexpr int kMaxItems = 32;  // levels of at most this many items
  static constexpr int BB = BS * BS, AW = 2 * BS;
  static constexpr int words = BS * AW + 2 * BB;  // [A | I] (step 2: the target), two blocks
};

// The warps' scratch, one array for both team kinds of a kernel.
template <int BS, typename TF>
__device__ __forceinline__ TF* factor_coop_scratch() {
  __shared__ TF sh[FactorCoop<BS, TF>::kWarps * FactorCoop<BS, TF>::words];
  return sh;
}

template <int BS, typename TF, bool CL>
__device__ __noinline__ void factor_coop_level(const FactorArgs<TF> S, const Team tm, int l) {
  using P = FactorCoop<BS, TF>;
  constexpr int BB = P::BB, AW = P::AW;
  static_assert(BB <= 64 && (BS - 1) * AW <= 64 && AW <= 32, "two entries per lane at most");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = min(P::kWarps, (int)(blockDim.x >> 5));
  // CTAs of the team (S = 1: tid = threadIdx.x * csize + crank)
  const int csize = tm.nthr / (int)blockDim.x;
  const int crank = tm.tid - (int)threadIdx.x * csize;
  const int gw = wid * csize + crank, ngw = nw * csize;  // this warp, warps of the team
  const bool on = tm.ns > 0 && (tm.act & 1u) && wid < nw;
  const int gs = tm.s0;
  // BS rows of AW: [A | A^-1 in progress]
  TF* aug = factor_coop_scratch<BS, TF>() + (size_t)min(wid, P::kWarps - 1) * P::words;
  TF* X = aug + BS * AW;
  TF* Y = X + BB;
  TF* Z = aug;  // step 2's target block
  auto gblk = [&](int e) { return S.lu + ((size_t)e * S.B + gs) * BB; };
  auto load = [&](TF* dst, const TF* src) {
    for (int q = lane; q < BB; q += 32) dst[q] = __ldcg(src + q);
  };
  auto store = [&](TF* dst, const TF* src) {
    for (int q = lane; q < BB; q += 32) dst[q] = src[q];
  };
  // C -= A B on the lanes' entries (blk_msub's order of the k terms)
  auto msub = [&](TF* C, const TF* A, const TF* B) {
    for (int q = lane; q < BB; q += 32) {
      const int i = q / BS, j = q % BS;
      TF s = C[q];
#pragma unroll
      for (int k = 0; k < BS; ++k) s -= A[i * BS + k] * B[k * BS + j];
      C[q] = s;
    }
  };
  // step 1: r = {e, k, diag(k)}: U_kk^-1 for the diagonal, else L_ik = A_ik U_kk^-1
  const int f0 = S.fac_ptr[l], nf = S.fac_ptr[l + 1] - f0;
  if (on) {
    for (int t = gw; t < nf; t += ngw) {
      const int4 r = __ldg(S.fac_rec + f0 + t);
      const TF* d = gblk(r.z);
      for (int q = lane; q < BS * AW; q += 32) {
        const int i = q / AW, j = q % AW;
        aug[q] = j < BS ? __ldcg(d + i * BS + j) : (j - BS == i ? TF(1) : TF(0));
      }
      if (r.x != r.z) load(X, gblk(r.x));
      __syncwarp();
      bool ok = true;
      for (int c = 0; c < BS; ++c) {
        // pivot row: the first largest |a_rc|, r >= c (every lane alike)
        int piv = c;
        TF best = aug[c * AW + c] < 0 ? -aug[c * AW + c] : aug[c * AW + c];
        for (int rr = c + 1; rr < BS; ++rr) {
          const TF v = aug[rr * AW + c] < 0 ? -aug[rr * AW + c] : aug[rr * AW + c];
          if (v > best) {
            best = v;
            piv = rr;
          }
        }
        if (!(best > TF(0)) || !isfinite(best)) ok = false;
        if (piv != c && lane < AW) {
          const TF t0 = aug[c * AW + lane];
          aug[c * AW + lane] = aug[piv * AW + lane];
          aug[piv * AW + lane] = t0;
        }
        __syncwarp();
        const TF dv = TF(1) / aug[c * AW + c];
        __syncwarp();
        if (lane < AW) aug[c * AW + lane] *= dv;
        __syncwarp();
        // rows r != c: a_rj -= a_rc a_cj, with a_rc read before any write
        TF nv[2];
        int at[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = lane + 32 * h;
          at[h] = -1;
          if (q < (BS - 1) * AW) {
            int rr = q / AW;
            rr += rr >= c;
            const int j = q % AW;
            const TF f = aug[rr * AW + c];
            TF v = aug[rr * AW + j];
            v -= f * aug[c * AW + j];
            nv[h] = v;
            at[h] = rr * AW + j;
          }
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h)
          if (at[h] >= 0) aug[at[h]] = nv[h];
        __syncwarp();
      }
      if (r.x == r.z) {
        if (!ok && lane == 0) S.flag[gs] = 1;
        TF* u = S.uinv + ((size_t)r.y * S.B + gs) * BB;
        for (int q = lane; q < BB; q += 32) u[q] = aug[(q / BS) * AW + BS + q % BS];
      } else {
        TF* o = gblk(r.x);
        for (int q = lane; q < BB; q += 32) {
          const int i = q / BS, j = q % BS;
          TF s = 0;
#pragma unroll
          for (int k = 0; k < BS; ++k) s += X[i * BS + k] * aug[k * AW + BS + j];
          o[q] = s;
        }
      }
      __syncwarp();
    }
  }
  csync<CL>();
  // step 2: r = {e, L entry, U entry, rest}: A_e -= L U, then the rest
  const int t0 = S.tgt_ptr[l], nt = S.tgt_ptr[l + 1] - t0;
  if (nt == 0) return;
  if (on) {
    for (int t = gw; t < nt; t += ngw) {
      const int4 r = __ldg(S.tgt_rec + t0 + t);
      const int e = r.x & ~kFillFirst;
      if (r.x & kFillFirst) {
        for (int q = lane; q < BB; q += 32) Z[q] = TF(0);
      } else {
        load(Z, gblk(e));
      }
      load(X, gblk(r.y));
      load(Y, gblk(r.z));
      __syncwarp();
      msub(Z, X, Y);
      if (r.w >= 0) {
        for (int q = r.w;; ++q) {
          const int2 cq = __ldg(S.con + q);
          if (cq.x < 0) break;
          __syncwarp();
          load(X, gblk(cq.x));
          load(Y, gblk(cq.y));
          __syncwarp();
          msub(Z, X, Y);
        }
      }
      store(gblk(e), Z);
      __syncwarp();
    }
  }
  csync<CL>();
}

template <int BS, typename TF, bool CL>
__device__ __forceinline__ void factor_levels(const DevSys& S, const DevWork& w, const Team& tm,
                                              int l0, int l1, unsigned char* ring) {
  FactorArgs<TF> f;
  f.lu = reinterpret_cast<TF*>(w.lu);
  f.uinv = reinterpret_cast<TF*>(w.uinv);
  f.flag = w.flag;
  f.B = w.B;
  f.fac_ptr = S.fac_ptr;
  f.fac_rec = S.fac_rec;
  f.tgt_ptr = S.tgt_ptr;
  f.tgt_rec = S.tgt_rec;
  f.con = S.con;
  f.ring = ring;
  // a single solve of 6x6 FP64 blocks: the levels of few items a warp per
  // item, the others a thread per item
  if constexpr (BS == 6 && sizeof(TF) == 8) {
    if (tm.S == 1) {
      for (int l = l0; l < l1;) {
        auto items = [&](int q) {
          return max(S.fac_ptr[q + 1] - S.fac_ptr[q], S.tgt_ptr[q + 1] - S.tgt_ptr[q]);
        };
        if (items(l) <= FactorCoop<BS, TF>::kMaxItems) {
          factor_coop_level<BS, TF, CL>(f, tm, l);
          ++l;
        } else {
          int l2 = l + 1;
          while (l2 < l1 && items(l2) > FactorCoop<BS, TF>::kMaxItems) ++l2;
          factor_run<BS, TF, CL>(f, tm, l, l2);
          l = l2;
        }
      }
      return;
    }
  }
  if constexpr (BS == 2 && !CL) {
    if (tm.S == 32 && ring) {
      factor_warp<TF>(f, tm, l0, l1);
      return;
    }
    if (tm.S > 1 && ring) {
      factor_pipe<TF>(f, tm, l0, l1);
      return;
    }
  }
  factor_run<BS, TF, CL>(f, tm, l0, l1);
}

// ---------------------------------------------------------------------------
// Newton-Krylov: restarted GMRES(m), right-preconditioned by ILU(0)
// ---------------------------------------------------------------------------


// Team-wide sums of per-scenario partials.  part(j) is the calling thread's
// partial of index j for its scenario slot; every thread must call (inactive
// ones return 0).  Lanes of a slot are summed with shuffles, warps through
// shared memory, and the CTAs of a cluster through per-rank global slots read
// back after a cluster barrier -- a fixed order, so results are deterministic.
// Results: rs[j * S + slot], valid for every thread of the CTA on return.
template <bool CL, typename T, class Part>
__device__ void team_sum(const Team& tm, int J, Part part, T* redw, T* rs, T* gred, int par,
                         int csize, int crank, int B) {
  const int S = tm.S;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < J; ++j) {
    T v = part(j);
    for (int off = 16; off >= S; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane < S) redw[(warp * J + j) * S + lane] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < J * S; t += blockDim.x) {
    const int j = t / S, s = t - j * S;
    T a = T(0);
    for (int q = 0; q < nw; ++q) a += redw[(q * J + j) * S + s];
    if constexpr (CL) {
      if (s < tm.ns) gred[(((size_t)par * csize + crank) * B + tm.s0 + s) * kMaxJ + j] = a;
    } else {
      rs[j * S + s] = a;
    }
  }
  if constexpr (CL) {
    csync<CL>();
    for (int t = threadIdx.x; t < J * S; t += blockDim.x) {
      const int j = t / S, s = t - j * S;
      T a = T(0);
      if (s < tm.ns)
        for (int r = 0; r < csize; ++r)
          a += __ldcg(gred + (((size_t)par * csize + r) * B + tm.s0 + s) * kMaxJ + j);
      rs[j * S + s] = a;
    }
  }
  __syncthreads();
}

// Per-slot GMRES state kept by every CTA in shared memory (identical copies,
// updated from identical reduction results): H column-major with leading
// dimension m+1, Givens cosines / sines, the rotated right-hand side g and
// the coefficients y.
template <typename T>
struct GmresState {
  T* H;
  T* cs;
  T* sn;
  T* g;
  T* y;
  __device__ static int words(int m) { return (m + 1) * m + 4 * m + 1; }
  __device__ void bind(T* base, int m, int slot) {
    H = base + (size_t)slot * words(m);
    cs = H + (m + 1) * m;
    sn = cs + m;
    g = sn + m;
    y = g + m + 1;
  }
};

// ---------------------------------------------------------------------------
// per (row, scenario) steps shared by the persistent kernel and the batched
// phase kernels
// ---------------------------------------------------------------------------

// Set-up of bus i (single phase), scenario gs, from its specified load and
// generation: the injections and the start voltage.
__device__ __forceinline__ void setup_1ph(const DevSys& S, const DevWork& w, int i, int gs,
                                          double pl, double ql, double pg) {
  const size_t b = (size_t)i * w.B + gs;
  const int oi = S.perm[i];
  w.spec[b * 3] = pl;
  w.spec[b * 3 + 1] = ql;
  w.spec[b * 3 + 2] = pg;
  double vm, va;
  if (w.in_vm) {
    vm = w.in_vm[(size_t)gs * S.n + oi];
    va = w.in_va[(size_t)gs * S.n + oi];
  } else if (w.warm_in) {
    vm = w.warm_vm[oi];
    va = w.warm_va[oi];
  } else {
    vm = (S.btype[i] == PF_PQ) ? 1.0 : S.v_set[i];
    va = 0.0;
  }
  w.vm[b] = vm;
  w.va[b] = va;
  double sn, cs;
  sincos_tab(S.trig, va, &sn, &cs);
  if (w.U) w.U[b] = make_double2(cs, sn);
  w.V[b] = make_double2(vm * cs, vm * sn);
}

// The accumulators of scenario gs (once per scenario, with bus 0).
__device__ __forceinline__ void setup_scenario(const DevWork& w, int gs) {
  w.norm[gs] = 0ull;
  w.norm[w.B + gs] = 0ull;
  w.step[gs] = 0ull;
  w.step[w.B + gs] = 0ull;
  w.flag[gs] = 0;
}

// Set-up of row i, scenario gs: specified injections, start voltage and
// (row 0) the scenario's accumulators.
template <bool THREE>
__device__ __forceinline__ void setup_row(const DevSys& S, const DevWork& w, int i, int gs) {
  const int B = w.B, n = S.n;
  const size_t b = (size_t)i * B + gs;
  const int oi = S.perm[i];
  if (!THREE) {
    const size_t src = (size_t)gs * n + oi;
    setup_1ph(S, w, i, gs, w.in_p_load ? w.in_p_load[src] : S.p_load0[i],
              w.in_q_load ? w.in_q_load[src] : S.q_load0[i],
              w.in_p_gen ? w.in_p_gen[src] : S.p_gen0[i]);
  } else {
    const int mask = S.btype[i] & 7;
    for (int a = 0; a < 3; ++a) {
      const size_t src = ((size_t)gs * n + oi) * 3 + a;
      w.spec[b * 6 + a] = w.in_p_load ? w.in_p_load[src] : S.p_load0[(size_t)i * 3 + a];
      w.spec[b * 6 + 3 + a] = w.in_q_load ? w.in_q_load[src] : S.q_load0[(size_t)i * 3 + a];
      double2 v = make_double2(0.0, 0.0);
      if ((mask >> a) & 1) {
        if (w.in_vm) {
          double sn, cs;
          sincos(w.in_va[src], &sn, &cs);
          v = make_double2(w.in_vm[src] * cs, w.in_vm[src] * sn);
        } else if (w.warm_in) {
          v = w.warm_V[(size_t)oi * 3 + a];
        } else {
          // balanced source angles 0, -120, +120 degrees; PV nodes at v_set
          double sn, cs;
          sincos(-2.0943951023931954923 * a, &sn, &cs);
          const double m0 = (S.btype[i] & 16) ? S.v_set[i] : S.v_source;
          v = make_double2(m0 * cs, m0 * sn);
        }
      }
      w.V[b * 3 + a] = v;
      // the reactive injections carry over between rounds of reactive limits
      if (!(w.bt && w.in_vm)) w.qg[b * 3 + a] = 0.0;
    }
  }
  if (i == 0) setup_scenario(w, gs);
}

// Voltage change of the current step (complex), for J dx evaluated from Y
// and V in the FP64 refinement residual.
template <bool THREE>
__device__ __forceinline__ void dv_row(const DevSys& S, const DevWork& w, int i, int gs) {
  const int B = w.B;
  const size_t b = (size_t)i * B + gs;
  if constexpr (THREE) {
    const bool pv = (S.btype[i] & 16) != 0 && !(S.btype[i] & 8);
    const int held = w.bt ? w.bt[b] : 0;
    for (int a = 0; a < 3; ++a) {
      const double di = __ldcg(w.dx + b * 6 + 3 + a);
      double dr = __ldcg(w.dx + b * 6 + a);
      if (pv && ((S.btype[i] >> a) & 1) && !((held >> a) & 1)) {  // (dQ, dVi): dVr = -(Vi/Vr) dVi
        const double2 v = ldc(w.V + b * 3 + a);
        dr = -(v.y / v.x) * di;
      }
      w.dV[b * 3 + a] = make_double2(dr, di);
    }
  } else {
    // dV = j d_delta V + d|V| U = V (d|V| / |V| + j d_delta)
    const double2 V = ldc(w.V + b);
    const double dd = __ldcg(w.dx + b * 2), dm = __ldcg(w.dx + b * 2 + 1);
    const double sm = dm / __ldcg(w.vm + b);
    w.dV[b] = make_double2(sm * V.x - dd * V.y, sm * V.y + dd * V.x);
  }
}

// FP64 residual r = F - J dx of row i, matrix-free from Y, V and dV
// (single phase: dS = dV conj(I) + V conj(Y dV) plus the load's slope).
template <bool THREE>
__device__ __forceinline__ void resid_row(const DevSys& S, const DevWork& w, int i, int gs) {
  const int B = w.B;
  const size_t b = (size_t)i * B + gs;
  double* y = w.r;
  const double2* Y = reinterpret_cast<const double2*>(S.y_val);
  if constexpr (THREE) {
    double2 YdV[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    for (int e = S.y_rowptr[i]; e < S.y_rowptr[i + 1]; ++e) {
      const size_t bj = ((size_t)S.y_col[e] * B + gs) * 3;
      for (int c = 0; c < 3; ++c) {
        const double2 d = ldc(w.dV + bj + c);
        for (int a = 0; a < 3; ++a) YdV[a] = cadd(YdV[a], cmul(Y[(size_t)e * 9 + a * 3 + c], d));
      }
    }
    const int mask = S.btype[i] & 7;
    const bool src = (S.btype[i] & 8) != 0;
    const bool pv = (S.btype[i] & 16) != 0;
    const int held = w.bt ? w.bt[b] : 0;
    for (int a = 0; a < 3; ++a) {
      const bool fa = ((mask >> a) & 1) && !src;
      const double2 dv = ldc(w.dV + b * 3 + a);  // the step as a voltage change
      const double dr = dv.x, di = dv.y;
      double rim, rre;
      if (fa) {
        // J dV = [Im; Re](Y dV) - [a b; c d] dV   (Eq. 21-23)
        const double* ad = w.abcd + b * 12;
        double jim = YdV[a].y - (ad[a] * dr + ad[3 + a] * di);
        double jre = YdV[a].x - (ad[6 + a] * dr + ad[9 + a] * di);
        if (pv && !((held >> a) & 1)) {  // plus the dQ column j V / |V|^2
          const double2 v = ldc(w.V + b * 3 + a);
          const double dq = __ldcg(w.dx + b * 6 + a), m2 = v.x * v.x + v.y * v.y;
          jim += v.x / m2 * dq;
          jre -= v.y / m2 * dq;
        }
        rim = __ldcg(w.F + b * 6 + a) - jim;
        rre = __ldcg(w.F + b * 6 + 3 + a) - jre;
      } else {
        rim = -dr;
        rre = -di;
      }
      y[b * 6 + a] = rim;
      y[b * 6 + 3 + a] = rre;
    }
  } else {
    // Y dV and the current I = Y V of the step's start point
    double2 YdV = make_double2(0.0, 0.0), I = make_double2(0.0, 0.0);
#pragma unroll 2
    for (int e = S.y_rowptr[i]; e < S.y_rowptr[i + 1]; ++e) {
      const size_t bj = (size_t)S.y_col[e] * B + gs;
      const double2 y = Y[e], d = ldc(w.dV + bj), v = ldc(w.V + bj);
      YdV.x = fma(y.x, d.x, YdV.x);
      YdV.x = fma(-y.y, d.y, YdV.x);
      YdV.y = fma(y.x, d.y, YdV.y);
      YdV.y = fma(y.y, d.x, YdV.y);
      I.x = fma(y.x, v.x, I.x);
      I.x = fma(-y.y, v.y, I.x);
      I.y = fma(y.x, v.y, I.y);
      I.y = fma(y.y, v.x, I.y);
    }
    const double2 V = ldc(w.V + b), dV = ldc(w.dV + b);
    // dS = dV conj(I) + V conj(Y dV), plus the load's slope on |V|
    const double2 dS = cadd(cmulc(dV, I), cmulc(V, YdV));
    const double vmi = __ldcg(w.vm + b);
    const double dshape = S.zip[3 * i + 1] + 2.0 * S.zip[3 * i + 2] * vmi;
    const double dd = __ldcg(w.dx + b * 2), dm = __ldcg(w.dx + b * 2 + 1);
    const int t = w.bt ? w.bt[b] : S.btype[i];
    const double r0 = (t != PF_SLACK)
                          ? __ldcg(w.F + b * 2) - (dS.x + __ldcg(w.spec + b * 3) * dshape * dm)
                          : -dd;
    const double r1 = (t >= PF_PQ)
                          ? __ldcg(w.F + b * 2 + 1) - (dS.y + __ldcg(w.spec + b * 3 + 1) * dshape * dm)
                          : -dm;
    y[b * 2] = r0;
    y[b * 2 + 1] = r1;
  }
}

// Voltage update of row i (Sec. II.A box: delta += Delta delta, |V| +=
// Delta|V|; Sec. II.B box: V^c += Delta V^c).  Returns the largest step.
// Single phase: the step from dx, or (y non-null) from the solve vector y of
// the sweeps, which holds it when no refinement followed (the same values:
// dx = (double) y there).
template <bool THREE, typename TY = double>
__device__ __forceinline__ double update_row(const DevSys& S, const DevWork& w, int i, int gs,
                                             const TY* y = nullptr) {
  const int B = w.B;
  constexpr int NSL = THREE ? 3 : 1;
  const size_t b = (size_t)i * B + gs;
  double stp = 0.0;
  if constexpr (THREE) {
    const bool pv = (S.btype[i] & 16) != 0 && !(S.btype[i] & 8);
    const int held = w.bt ? w.bt[b] : 0;
    for (int a = 0; a < NSL; ++a) {
      double dr = __ldcg(w.dx + b * 6 + a);
      const double di = __ldcg(w.dx + b * 6 + 3 + a);
      stp = fmax(stp, fmax(fabs(dr), fabs(di)));
      const double2 v = ldc(w.V + b * 3 + a);
      if (pv && ((S.btype[i] >> a) & 1) && !((held >> a) & 1)) {
        // PV slot: the step is (dQ, dVi) with dVr = -(Vi/Vr) dVi; the new
        // voltage is put back on |V| = v_set
        w.qg[b * 3 + a] += dr;
        dr = -(v.y / v.x) * di;
        const double2 u = make_double2(v.x + dr, v.y + di);
        const double sc = S.v_set[i] / sqrt(u.x * u.x + u.y * u.y);
        w.V[b * 3 + a] = make_double2(u.x * sc, u.y * sc);
      } else {
        w.V[b * 3 + a] = make_double2(v.x + dr, v.y + di);
      }
    }
  } else {
    // (d angle, d|V|) with one vector load
    double dd, dm;
    if (y && sizeof(TY) == 4) {
      const float2 q = __ldcg(reinterpret_cast<const float2*>(y) + b);
      dd = (double)q.x;
      dm = (double)q.y;
    } else {
      const double2 q = __ldcg(reinterpret_cast<const double2*>(y ? (const void*)y : (const void*)w.dx) + b);
      dd = q.x;
      dm = q.y;
    }
    stp = __longlong_as_double((long long)max(abs_bits(dd), abs_bits(dm)));
    const double vm = __ldcg(w.vm + b) + dm, va = __ldcg(w.va + b) + dd;
    w.vm[b] = vm;
    w.va[b] = va;
    double sn, cs;
    sincos_tab(S.trig, va, &sn, &cs);
    if (w.U) w.U[b] = make_double2(cs, sn);
    w.V[b] = make_double2(vm * cs, vm * sn);
  }
  return stp;
}

// Result of row i in the caller's numbering (and the warm start).
template <bool THREE>
__device__ __forceinline__ void output_row(const DevSys& S, const DevWork& w, int i, int gs, bool ok) {
  const int B = w.B, n = S.n;
  const size_t b = (size_t)i * B + gs;
  const int oi = S.perm[i];
  if constexpr (THREE) {
    const int mask = S.btype[i] & 7;
    for (int a = 0; a < 3; ++a) {
      const double2 v = ldc(w.V + b * 3 + a);
      const bool pres = (mask >> a) & 1;
      const size_t dst = ((size_t)gs * n + oi) * 3 + a;
      if (w.out_vm) w.out_vm[dst] = pres ? hypot(v.x, v.y) : 0.0;
      if (w.out_va) w.out_va[dst] = pres ? atan2(v.y, v.x) : 0.0;
      if (w.warm_out && gs == 0 && ok) w.warm_V[(size_t)oi * 3 + a] = v;
    }
  } else {
    const size_t dst = (size_t)gs * n + oi;
    const double vm = __ldcg(w.vm + b), va = __ldcg(w.va + b);
    if (w.out_vm) w.out_vm[dst] = vm;
    if (w.out_va) w.out_va[dst] = va;
    if (w.warm_out && gs == 0 && ok) {
      w.warm_vm[oi] = vm;
      w.warm_va[oi] = va;
    }
  }
}

}  // namespace pf
