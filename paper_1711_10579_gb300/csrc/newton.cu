// Persistent Newton power-flow kernel for sm_103a.
//
// One launch runs complete Newton solves.  The grid is made of clusters of
// CTAs; cluster c owns scenarios [c*S, c*S + S) and iterates them to
// convergence on its own, so clusters never wait for one another.  Inside a
// cluster every step of an iteration is spread over all its threads and the
// steps are separated by cluster barriers:
//
//   A  mismatch + Jacobian assembly (fused): I = Y V (Eq. 1), S = V conj(I)
//      (the power of Eq. 5-7), Delta P / Delta Q (Eq. 8-9) and the Jacobian
//      blocks of Eq. 10 written straight into the factor's value array;
//      three phase: Delta I (Eq. 12-19) and the 6x6 blocks of Eq. 21-23.
//   stop test on the infinity norm of the power mismatch (per scenario);
//   B  numeric block LU refactorisation on the fixed symbolic pattern
//      (Sec. III.A), one level set at a time, rows of a level in parallel;
//   C  level-scheduled forward and backward block triangular solves;
//   R  (mixed precision) FP64 residual r = F - J dx evaluated matrix-free
//      from Y and V, then another FP32 solve, dx += correction;
//   E  voltage update (Sec. II.A box: delta += Delta delta, |V| += Delta|V|;
//      Sec. II.B box: V^c += Delta V^c).
//
// Single solves run one cluster of up to 16 CTAs; batches of scenarios run
// one CTA per S scenarios.  Values are interleaved as [entry][scenario] so
// that neighbouring threads of a batch read neighbouring memory.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "device.h"

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

__device__ __forceinline__ void atomic_max_pos(unsigned long long* p, double v) {
  // non-negative doubles order like their bit patterns; NaN maps above +inf
  if (!(v >= 0.0)) v = __longlong_as_double(0x7ff8000000000000ULL);
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
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
    if (!(best > T(0)) || !isfinite((double)best)) ok = false;
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
// and their columns zero, which keeps the system of Eq. 10 unchanged.
template <typename TF>
__device__ void mismatch_jacobian_1ph(const DevSys& S, const DevWork& w, int i, int gs,
                                      double& nrm) {
  const int B = w.B;
  const size_t b = (size_t)i * B + gs;
  const double2 Vi = ldc(w.V + b);
  double2 I = make_double2(0.0, 0.0);
  const double2* Y = reinterpret_cast<const double2*>(S.y_val);
  for (int e = S.y_rowptr[i]; e < S.y_rowptr[i + 1]; ++e) {
    const int j = S.y_col[e];
    I = cadd(I, cmul(Y[e], ldc(w.V + (size_t)j * B + gs)));
  }
  w.I[b] = I;
  const double vmi = __ldcg(w.vm + b);
  const double2 Sc = cmulc(Vi, I);
  const double pl = __ldcg(w.spec + b * 3), ql = __ldcg(w.spec + b * 3 + 1),
               pg = __ldcg(w.spec + b * 3 + 2);
  const double zp = S.zip[3 * i], zi = S.zip[3 * i + 1], zz = S.zip[3 * i + 2];
  const double shape = zp + zi * vmi + zz * vmi * vmi;
  const double dshape = zi + 2.0 * zz * vmi;
  const int t = S.btype[i];
  const double f0 = (t != PF_SLACK) ? (pg - pl * shape) - Sc.x : 0.0;
  const double f1 = (t == PF_PQ) ? (S.q_gen[i] - ql * shape) - Sc.y : 0.0;
  w.F[b * 2] = f0;
  w.F[b * 2 + 1] = f1;
  nrm = fmax(fabs(f0), fabs(f1));
  if (!isfinite(f0) || !isfinite(f1)) nrm = __longlong_as_double(0x7ff8000000000000ULL);

  TF* lu = reinterpret_cast<TF*>(w.lu);
  for (int e = S.lu_rowptr[i]; e < S.lu_rowptr[i + 1]; ++e) {
    const int j = S.lu_col[e];
    const int yi = S.lu2y[e];
    double j00 = 0, j01 = 0, j10 = 0, j11 = 0;
    if (yi >= 0) {
      const double2 Yij = Y[yi];
      if (j != i) {
        const int tj = S.btype[j];
        if (t != PF_SLACK && tj != PF_SLACK) {
          const size_t bj = (size_t)j * B + gs;
          // dS_i/d delta_j = -j V_i conj(Y_ij V_j); dS_i/d|V_j| = V_i conj(Y_ij V_j)/|V_j|
          const double2 c = cmulc(Vi, cmul(Yij, ldc(w.V + bj)));
          j00 = c.y;
          j10 = -c.x;
          if (tj == PF_PQ) {
            const double inv = 1.0 / __ldcg(w.vm + bj);
            j01 = c.x * inv;
            j11 = c.y * inv;
          }
          if (t == PF_PV) j10 = j11 = 0.0;
        }
      } else if (t == PF_SLACK) {
        j00 = j11 = 1.0;
      } else {
        // dS_i/d delta_i = j (S_i - V_i conj(Y_ii V_i));
        // dS_i/d|V_i| = (S_i + V_i conj(Y_ii V_i)) / |V_i|, minus the load's slope
        const double2 d = cmulc(Vi, cmul(Yij, Vi));
        j00 = -(Sc.y - d.y);
        j10 = Sc.x - d.x;
        j01 = (Sc.x + d.x) / vmi + pl * dshape;
        j11 = (Sc.y + d.y) / vmi + ql * dshape;
        if (t == PF_PV) {
          j01 = 0.0;
          j10 = 0.0;
          j11 = 1.0;
        }
      }
    }
    TF blk[4] = {(TF)j00, (TF)j01, (TF)j10, (TF)j11};
    blk_store<2>(lu + ((size_t)e * B + gs) * 4, blk);
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
  const double inv2 = 1.0 / m2;
  const double2 cSV = cmul(cS, V);
  Isp = cscale(cSV, inv2);
  const double2 base = cscale(cmul(cSp, V), inv2 / m);
  dIdr = csub(cadd(cscale(base, V.x), cscale(cS, inv2)), cscale(cSV, 2.0 * V.x * inv2 * inv2));
  const double2 jcS = make_double2(-cS.y, cS.x);
  dIdi = csub(cadd(cscale(base, V.y), cscale(jcS, inv2)), cscale(cSV, 2.0 * V.y * inv2 * inv2));
}

template <typename TF>
__device__ void mismatch_jacobian_3ph(const DevSys& S, const DevWork& w, int i, int gs,
                                      double& nrm) {
  const int B = w.B;
  const size_t b = (size_t)i * B + gs;
  const int mask = S.btype[i] & 7;
  const bool src = (S.btype[i] & 8) != 0;
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
    w.I[b * 3 + a] = I[a];
    const bool freea = ((mask >> a) & 1) && !src;
    double fim = 0.0, fre = 0.0;
    adj[a] = adj[3 + a] = adj[6 + a] = adj[9 + a] = 0.0;
    if (freea) {
      const double pl = __ldcg(w.spec + b * 6 + a), ql = __ldcg(w.spec + b * 6 + 3 + a);
      double2 Isp, dr, di;
      load_slope(Vi[a], pl, ql, zp, zi, zz, Isp, dr, di);
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
    TF blk[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) blk[k] = TF(0);
    if (yi >= 0) {
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
    }
    blk_store<6>(lu + ((size_t)e * B + gs) * 36, blk);
  }
}

// ---------------------------------------------------------------------------
// steps B, C: factorisation and triangular solves of one row
// ---------------------------------------------------------------------------

// Row i of the block LU (row-oriented, L with identity diagonal blocks):
// for each L entry (i, k) in increasing k: L_ik = A_ik U_kk^-1, then
// A_ij -= L_ik U_kj for the U entries of row k.  The G lanes of a group share
// the inner loop; rows of one level are independent.
template <int BS, typename TF>
__device__ void factor_row(const DevSys& S, const DevWork& w, int i, int gs, int lane, int G,
                           unsigned gmask) {
  const int B = w.B;
  TF* lu = reinterpret_cast<TF*>(w.lu);
  TF* uinv = reinterpret_cast<TF*>(w.uinv);
  constexpr int BB = BS * BS;
  const int rp = S.lu_rowptr[i], dg = S.lu_diag[i];
  for (int p = rp; p < dg; ++p) {
    const int k = S.lu_col[p];
    TF a[BB], u[BB], l[BB];
    blk_load<BS>(lu + ((size_t)p * B + gs) * BB, a);
    blk_load<BS>(uinv + ((size_t)k * B + gs) * BB, u);
    blk_mul<BS>(a, u, l);
    if (G > 1) __syncwarp(gmask);
    if (lane == 0) blk_store<BS>(lu + ((size_t)p * B + gs) * BB, l);
    const int kd = S.lu_diag[k], ke = S.lu_rowptr[k + 1], up = S.upd_ptr[p] - kd - 1;
    for (int q = kd + 1 + lane; q < ke; q += G) {
      const int pos = S.upd_pos[up + q];
      if (pos < 0) continue;  // dropped by ILU(0)
      TF c[BB], uu[BB];
      blk_load<BS>(lu + ((size_t)pos * B + gs) * BB, c);
      blk_load<BS>(lu + ((size_t)q * B + gs) * BB, uu);
      blk_msub<BS>(c, l, uu);
      blk_store<BS>(lu + ((size_t)pos * B + gs) * BB, c);
    }
    if (G > 1) __syncwarp(gmask);
  }
  if (lane == 0) {
    TF d[BB], di[BB];
    blk_load<BS>(lu + ((size_t)dg * B + gs) * BB, d);
    if (!blk_inv<BS>(d, di)) w.flag[gs] = 1;
    blk_store<BS>(uinv + ((size_t)i * B + gs) * BB, di);
  }
}

// Forward substitution, row i: y_i -= sum_k L_ik y_k.
template <int BS, typename TF>
__device__ void forward_row(const DevSys& S, const DevWork& w, int i, int gs, int lane, int G,
                            unsigned gmask) {
  const int B = w.B;
  const TF* lu = reinterpret_cast<const TF*>(w.lu);
  TF* y = reinterpret_cast<TF*>(w.y);
  constexpr int BB = BS * BS;
  TF acc[BS];
#pragma unroll
  for (int c = 0; c < BS; ++c) acc[c] = TF(0);
  const int rp = S.lu_rowptr[i], dg = S.lu_diag[i];
  for (int p = rp + lane; p < dg; p += G) {
    const size_t bk = ((size_t)S.lu_col[p] * B + gs) * BS;
    TF L[BB];
    blk_load<BS>(lu + ((size_t)p * B + gs) * BB, L);
    TF yk[BS];
#pragma unroll
    for (int c = 0; c < BS; ++c) yk[c] = __ldcg(y + bk + c);
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
    const size_t bi = ((size_t)i * B + gs) * BS;
#pragma unroll
    for (int c = 0; c < BS; ++c) y[bi + c] = __ldcg(y + bi + c) - acc[c];
  }
}

// Backward substitution, row i: x_i = U_ii^-1 (y_i - sum_j U_ij x_j).
template <int BS, typename TF>
__device__ void backward_row(const DevSys& S, const DevWork& w, int i, int gs, int lane, int G,
                             unsigned gmask) {
  const int B = w.B;
  const TF* lu = reinterpret_cast<const TF*>(w.lu);
  const TF* uinv = reinterpret_cast<const TF*>(w.uinv);
  TF* y = reinterpret_cast<TF*>(w.y);
  constexpr int BB = BS * BS;
  TF acc[BS];
#pragma unroll
  for (int c = 0; c < BS; ++c) acc[c] = TF(0);
  const int dg = S.lu_diag[i], re = S.lu_rowptr[i + 1];
  for (int q = dg + 1 + lane; q < re; q += G) {
    const size_t bj = ((size_t)S.lu_col[q] * B + gs) * BS;
    TF U[BB];
    blk_load<BS>(lu + ((size_t)q * B + gs) * BB, U);
    TF xj[BS];
#pragma unroll
    for (int c = 0; c < BS; ++c) xj[c] = __ldcg(y + bj + c);
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
      for (int c = 0; c < BS; ++c) acc[r] += U[r * BS + c] * xj[c];
  }
  if (G > 1) {
#pragma unroll
    for (int c = 0; c < BS; ++c) acc[c] = group_sum(acc[c], G, gmask);
  }
  if (lane == 0) {
    const size_t bi = ((size_t)i * B + gs) * BS;
    TF t[BS], Di[BB];
#pragma unroll
    for (int c = 0; c < BS; ++c) t[c] = __ldcg(y + bi + c) - acc[c];
    blk_load<BS>(uinv + ((size_t)i * B + gs) * BB, Di);
#pragma unroll
    for (int r = 0; r < BS; ++r) {
      TF s = TF(0);
#pragma unroll
      for (int c = 0; c < BS; ++c) s += Di[r * BS + c] * t[c];
      y[bi + r] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// cluster-wide schedule helpers
// ---------------------------------------------------------------------------

struct Team {
  int tid;    // thread index within the cluster
  int nthr;   // threads in the cluster
  int s0;     // first scenario of the cluster
  int ns;     // scenarios of the cluster
  unsigned act;  // active scenarios (bit s = scenario s0 + s)
};

// Runs `row(i, gs, lane, G, gmask)` for every row of every level in order,
// with a cluster barrier after each level.
template <bool CL, class RowFn>
__device__ void run_levels(const Team& tm, const int* lev_ptr, const int* lev_rows, int nlev,
                           const int8_t* gsz, bool reverse, RowFn row) {
  for (int t = 0; t < nlev; ++t) {
    const int l = reverse ? nlev - 1 - t : t;
    const int base = lev_ptr[l], width = lev_ptr[l + 1] - base;
    if (tm.ns == 1) {
      if (tm.act & 1u) {
        const int G = gsz[l];
        const int group = tm.tid / G, lane = tm.tid % G, ngroups = tm.nthr / G;
        const unsigned gmask =
            (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
        for (int r = group; r < width; r += ngroups) row(lev_rows[base + r], tm.s0, lane, G, gmask);
      }
    } else {
      const int items = width * tm.ns;
      for (int it = tm.tid; it < items; it += tm.nthr) {
        const int r = it / tm.ns, s = it - r * tm.ns;
        if ((tm.act >> s) & 1u) row(lev_rows[base + r], tm.s0 + s, 0, 1, 0u);
      }
    }
    csync<CL>();
  }
}

// Runs `fn(i, gs)` for every row and active scenario, then a cluster barrier.
template <bool CL, class Fn>
__device__ void run_rows(const Team& tm, int n, Fn fn) {
  const int items = n * tm.ns;
  for (int it = tm.tid; it < items; it += tm.nthr) {
    const int i = it / tm.ns, s = it - i * tm.ns;
    if ((tm.act >> s) & 1u) fn(i, tm.s0 + s);
  }
  csync<CL>();
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------

template <int BS, typename TF, bool CL>
__global__ void __launch_bounds__(BS == 2 ? 1024 : 256) newton_kernel(DevSys S, DevWork w, DevOpts o) {
  constexpr bool THREE = (BS == 6);
  constexpr int NSL = THREE ? 3 : 1;  // complex voltages per row
  const int csize = CL ? (int)cg::this_cluster().num_blocks() : 1;
  const int crank = CL ? (int)cg::this_cluster().block_rank() : 0;
  const int cid = blockIdx.x / csize;
  Team tm;
  tm.tid = crank * blockDim.x + threadIdx.x;
  tm.nthr = csize * blockDim.x;
  tm.s0 = cid * o.S;
  tm.ns = min(o.S, w.B - tm.s0);
  if (tm.ns <= 0) return;  // whole cluster exits together
  const int n = S.n, B = w.B;
  __shared__ int sh_status[32];
  __shared__ unsigned sh_act;
  __shared__ unsigned long long sh_t0;
  if (threadIdx.x == 0) {
    sh_t0 = global_ns();
    for (int s = 0; s < 32; ++s) sh_status[s] = kRunning;
    sh_act = (tm.ns >= 32) ? 0xffffffffu : ((1u << tm.ns) - 1u);
  }
  __syncthreads();
  tm.act = sh_act;

  // ---- set-up: specified injections, start voltage, accumulators ----
  run_rows<CL>(tm, n, [&](int i, int gs) {
    const size_t b = (size_t)i * B + gs;
    const int oi = S.perm[i];
    if (!THREE) {
      const size_t src = (size_t)gs * n + oi;
      w.spec[b * 3] = w.in_p_load ? w.in_p_load[src] : S.p_load0[i];
      w.spec[b * 3 + 1] = w.in_q_load ? w.in_q_load[src] : S.q_load0[i];
      w.spec[b * 3 + 2] = w.in_p_gen ? w.in_p_gen[src] : S.p_gen0[i];
      double vm, va;
      if (w.in_vm) {
        vm = w.in_vm[oi];
        va = w.in_va[oi];
      } else if (w.warm_in) {
        vm = w.warm_vm[i];
        va = w.warm_va[i];
      } else {
        vm = (S.btype[i] == PF_PQ) ? 1.0 : S.v_set[i];
        va = 0.0;
      }
      w.vm[b] = vm;
      w.va[b] = va;
      double sn, cs;
      sincos(va, &sn, &cs);
      w.V[b] = make_double2(vm * cs, vm * sn);
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
            sincos(w.in_va[(size_t)oi * 3 + a], &sn, &cs);
            v = make_double2(w.in_vm[(size_t)oi * 3 + a] * cs, w.in_vm[(size_t)oi * 3 + a] * sn);
          } else if (w.warm_in) {
            v = w.warm_V[(size_t)i * 3 + a];
          } else {
            // balanced source angles 0, -120, +120 degrees
            double sn, cs;
            sincos(-2.0943951023931954923 * a, &sn, &cs);
            v = make_double2(S.v_source * cs, S.v_source * sn);
          }
        }
        w.V[b * 3 + a] = v;
      }
    }
    if (i == 0) {
      w.norm[gs] = 0ull;
      w.norm[B + gs] = 0ull;
      w.step[gs] = 0ull;
      w.step[B + gs] = 0ull;
      w.flag[gs] = 0;
    }
  });

  int it = 0;
  for (;; ++it) {
    // ---- A: mismatch + Jacobian ----
    run_rows<CL>(tm, n, [&](int i, int gs) {
      double nrm;
      if constexpr (THREE) {
        mismatch_jacobian_3ph<TF>(S, w, i, gs, nrm);
      } else {
        mismatch_jacobian_1ph<TF>(S, w, i, gs, nrm);
      }
      atomic_max_pos(w.norm + (size_t)(it & 1) * B + gs, nrm);
    });
    if (o.mode == 1) return;  // inspection: F and J stay in the workspace

    // ---- stop test (every CTA decides identically from global values) ----
    if (threadIdx.x == 0) {
      unsigned act = 0;
      for (int s = 0; s < tm.ns; ++s) {
        const int gs = tm.s0 + s;
        if (sh_status[s] != kRunning) continue;
        const double nrm = __longlong_as_double((long long)__ldcg(w.norm + (size_t)(it & 1) * B + gs));
        int st = kRunning;
        if (!(nrm <= 1e12)) st = PF_ERR_DIVERGED;
        else if (o.mode == 0 && nrm <= o.tol) st = PF_OK;
        else if (o.mode == 0 && it >= o.max_iter) st = PF_ERR_MAXITER;
        sh_status[s] = st;
        if (st == kRunning) act |= 1u << s;
        if (crank == 0) {
          if (st != kRunning && w.out_info) {
            pf_info inf;
            inf.status = st;
            inf.iterations = it;
            inf.linear_iterations = 0;
            inf.reserved = 0;
            inf.mismatch = nrm;
            inf.max_step = it > 0 ? __longlong_as_double((long long)__ldcg(w.step + (size_t)((it - 1) & 1) * B + gs)) : 0.0;
            inf.solve_us = 0.0;
            w.out_info[gs] = inf;
          }
          // the buffers of the next iteration (read last one iteration ago)
          w.norm[(size_t)((it + 1) & 1) * B + gs] = 0ull;
          w.step[(size_t)((it + 1) & 1) * B + gs] = 0ull;
        }
      }
      sh_act = act;
    }
    __syncthreads();
    tm.act = sh_act;
    if (tm.act == 0) break;

    // ---- B: numeric factorisation ----
    run_levels<CL>(tm, S.flev_ptr, S.flev_rows, S.nflev, S.g_fac, false,
                   [&](int i, int gs, int lane, int G, unsigned gmask) {
                     factor_row<BS, TF>(S, w, i, gs, lane, G, gmask);
                   });
    if (threadIdx.x == 0) {
      unsigned act = tm.act;
      for (int s = 0; s < tm.ns; ++s) {
        const int gs = tm.s0 + s;
        if (((act >> s) & 1u) && __ldcg(w.flag + gs)) {
          act &= ~(1u << s);
          sh_status[s] = PF_ERR_SINGULAR;
          if (crank == 0 && w.out_info) {
            pf_info inf;
            inf.status = PF_ERR_SINGULAR;
            inf.iterations = it;
            inf.linear_iterations = 0;
            inf.reserved = 0;
            inf.mismatch = __longlong_as_double((long long)__ldcg(w.norm + (size_t)(it & 1) * B + gs));
            inf.max_step = 0.0;
            inf.solve_us = 0.0;
            w.out_info[gs] = inf;
          }
        }
      }
      sh_act = act;
    }
    __syncthreads();
    tm.act = sh_act;
    if (tm.act == 0) break;

    // ---- C: triangular solves, then FP64 refinement ----
    for (int pass = 0; pass <= o.refine; ++pass) {
      // right-hand side: F, or the FP64 residual of the current step
      if (pass == 0) {
        run_rows<CL>(tm, n, [&](int i, int gs) {
          const size_t b = (size_t)i * B + gs;
          TF* y = reinterpret_cast<TF*>(w.y);
          for (int c = 0; c < BS; ++c) y[b * BS + c] = (TF)__ldcg(w.F + b * BS + c);
        });
      } else {
        // voltage change of the step (complex), for J dx evaluated from Y and V
        run_rows<CL>(tm, n, [&](int i, int gs) {
          const size_t b = (size_t)i * B + gs;
          if constexpr (THREE) {
            for (int a = 0; a < 3; ++a)
              w.dV[b * 3 + a] = make_double2(__ldcg(w.dx + b * 6 + a), __ldcg(w.dx + b * 6 + 3 + a));
          } else {
            // dV = V (j d_delta + d|V| / |V|)
            const double2 V = ldc(w.V + b);
            const double dd = __ldcg(w.dx + b * 2), dm = __ldcg(w.dx + b * 2 + 1);
            const double2 f = make_double2(dm / __ldcg(w.vm + b), dd);
            w.dV[b] = cmul(V, f);
          }
        });
        run_rows<CL>(tm, n, [&](int i, int gs) {
          const size_t b = (size_t)i * B + gs;
          TF* y = reinterpret_cast<TF*>(w.y);
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
            for (int a = 0; a < 3; ++a) {
              const bool fa = ((mask >> a) & 1) && !src;
              const double dr = __ldcg(w.dx + b * 6 + a), di = __ldcg(w.dx + b * 6 + 3 + a);
              double rim, rre;
              if (fa) {
                // J dV = [Im; Re](Y dV) - [a b; c d] dV   (Eq. 21-23)
                const double* ad = w.abcd + b * 12;
                const double jim = YdV[a].y - (ad[a] * dr + ad[3 + a] * di);
                const double jre = YdV[a].x - (ad[6 + a] * dr + ad[9 + a] * di);
                rim = __ldcg(w.F + b * 6 + a) - jim;
                rre = __ldcg(w.F + b * 6 + 3 + a) - jre;
              } else {
                rim = -dr;
                rre = -di;
              }
              y[b * 6 + a] = (TF)rim;
              y[b * 6 + 3 + a] = (TF)rre;
            }
          } else {
            double2 YdV = make_double2(0.0, 0.0);
            for (int e = S.y_rowptr[i]; e < S.y_rowptr[i + 1]; ++e)
              YdV = cadd(YdV, cmul(Y[e], ldc(w.dV + (size_t)S.y_col[e] * B + gs)));
            const double2 V = ldc(w.V + b), I = ldc(w.I + b), dV = ldc(w.dV + b);
            // dS = dV conj(I) + V conj(Y dV), plus the load's slope on |V|
            const double2 dS = cadd(cmulc(dV, I), cmulc(V, YdV));
            const double vmi = __ldcg(w.vm + b);
            const double dshape = S.zip[3 * i + 1] + 2.0 * S.zip[3 * i + 2] * vmi;
            const double dd = __ldcg(w.dx + b * 2), dm = __ldcg(w.dx + b * 2 + 1);
            const int t = S.btype[i];
            const double r0 = (t != PF_SLACK)
                                  ? __ldcg(w.F + b * 2) - (dS.x + __ldcg(w.spec + b * 3) * dshape * dm)
                                  : -dd;
            const double r1 = (t == PF_PQ)
                                  ? __ldcg(w.F + b * 2 + 1) - (dS.y + __ldcg(w.spec + b * 3 + 1) * dshape * dm)
                                  : -dm;
            y[b * 2] = (TF)r0;
            y[b * 2 + 1] = (TF)r1;
          }
        });
      }
      run_levels<CL>(tm, S.flev_ptr, S.flev_rows, S.nflev, S.g_fwd, false,
                     [&](int i, int gs, int lane, int G, unsigned gmask) {
                       forward_row<BS, TF>(S, w, i, gs, lane, G, gmask);
                     });
      run_levels<CL>(tm, S.blev_ptr, S.blev_rows, S.nblev, S.g_bwd, false,
                     [&](int i, int gs, int lane, int G, unsigned gmask) {
                       backward_row<BS, TF>(S, w, i, gs, lane, G, gmask);
                     });
      run_rows<CL>(tm, n, [&](int i, int gs) {
        const size_t b = ((size_t)i * B + gs) * BS;
        const TF* y = reinterpret_cast<const TF*>(w.y);
        for (int c = 0; c < BS; ++c) {
          const double v = (double)__ldcg(y + b + c);
          w.dx[b + c] = (pass == 0) ? v : __ldcg(w.dx + b + c) + v;
        }
      });
    }

    if (o.mode == 2) return;  // inspection: the step stays in the workspace

    // ---- E: voltage update ----
    run_rows<CL>(tm, n, [&](int i, int gs) {
      const size_t b = (size_t)i * B + gs;
      double stp = 0.0;
      if constexpr (THREE) {
        for (int a = 0; a < NSL; ++a) {
          const double dr = __ldcg(w.dx + b * 6 + a), di = __ldcg(w.dx + b * 6 + 3 + a);
          stp = fmax(stp, fmax(fabs(dr), fabs(di)));
          const double2 v = ldc(w.V + b * 3 + a);
          w.V[b * 3 + a] = make_double2(v.x + dr, v.y + di);
        }
      } else {
        const double dd = __ldcg(w.dx + b * 2), dm = __ldcg(w.dx + b * 2 + 1);
        stp = fmax(fabs(dd), fabs(dm));
        const double vm = __ldcg(w.vm + b) + dm, va = __ldcg(w.va + b) + dd;
        w.vm[b] = vm;
        w.va[b] = va;
        double sn, cs;
        sincos(va, &sn, &cs);
        w.V[b] = make_double2(vm * cs, vm * sn);
      }
      atomic_max_pos(w.step + (size_t)(it & 1) * B + gs, stp);
    });
  }

  // ---- results in the caller's numbering ----
  tm.act = (tm.ns >= 32) ? 0xffffffffu : ((1u << tm.ns) - 1u);
  run_rows<CL>(tm, n, [&](int i, int gs) {
    const size_t b = (size_t)i * B + gs;
    const int oi = S.perm[i];
    const bool ok = sh_status[gs - tm.s0] == PF_OK;
    if constexpr (THREE) {
      const int mask = S.btype[i] & 7;
      for (int a = 0; a < 3; ++a) {
        const double2 v = ldc(w.V + b * 3 + a);
        const bool pres = (mask >> a) & 1;
        const size_t dst = ((size_t)gs * n + oi) * 3 + a;
        if (w.out_vm) w.out_vm[dst] = pres ? hypot(v.x, v.y) : 0.0;
        if (w.out_va) w.out_va[dst] = pres ? atan2(v.y, v.x) : 0.0;
        if (w.warm_out && gs == 0 && ok) w.warm_V[(size_t)i * 3 + a] = v;
      }
    } else {
      const size_t dst = (size_t)gs * n + oi;
      const double vm = __ldcg(w.vm + b), va = __ldcg(w.va + b);
      if (w.out_vm) w.out_vm[dst] = vm;
      if (w.out_va) w.out_va[dst] = va;
      if (w.warm_out && gs == 0 && ok) {
        w.warm_vm[i] = vm;
        w.warm_va[i] = va;
      }
    }
  });
  if (crank == 0 && threadIdx.x == 0 && w.out_info) {
    const double us = (double)(global_ns() - sh_t0) * 1e-3;
    for (int s = 0; s < tm.ns; ++s) w.out_info[tm.s0 + s].solve_us = us;
  }
}

// ---------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------

template <int BS, typename TF, bool CL>
static cudaError_t launch_t(const DevSys& S, const DevWork& w, const DevOpts& o, int grid,
                            int cluster, int threads, cudaStream_t st) {
  auto kern = newton_kernel<BS, TF, CL>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (CL) {
    if (cluster > 8) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, S, w, o);
}

// Maximum cluster size the device can co-schedule for this kernel.
template <int BS, typename TF>
static int max_cluster_t(int threads) {
  auto kern = newton_kernel<BS, TF, true>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int c = 16; c >= 1; c >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(threads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, kern, &cfg) == cudaSuccess && num > 0) return c;
    cudaGetLastError();
  }
  return 1;
}

cudaError_t launch_newton(int bs, bool fp32, const DevSys& S, const DevWork& w,
                          const DevOpts& o, int grid, int cluster, int threads,
                          cudaStream_t st) {
  const bool cl = cluster > 1;
  if (bs == 2) {
    if (fp32) return cl ? launch_t<2, float, true>(S, w, o, grid, cluster, threads, st)
                        : launch_t<2, float, false>(S, w, o, grid, cluster, threads, st);
    return cl ? launch_t<2, double, true>(S, w, o, grid, cluster, threads, st)
              : launch_t<2, double, false>(S, w, o, grid, cluster, threads, st);
  }
  if (fp32) return cl ? launch_t<6, float, true>(S, w, o, grid, cluster, threads, st)
                      : launch_t<6, float, false>(S, w, o, grid, cluster, threads, st);
  return cl ? launch_t<6, double, true>(S, w, o, grid, cluster, threads, st)
            : launch_t<6, double, false>(S, w, o, grid, cluster, threads, st);
}

int max_cluster(int bs, bool fp32, int threads) {
  if (bs == 2) return fp32 ? max_cluster_t<2, float>(threads) : max_cluster_t<2, double>(threads);
  return fp32 ? max_cluster_t<6, float>(threads) : max_cluster_t<6, double>(threads);
}

}  // namespace pf
