// Branch power flows and losses of solved (or any) bus voltages.
//
// The problem statement of the paper asks for the voltages and the power
// flows of the branches (Sec. I).  With the branch models that build Ybus
// (Eq. 2-3: pi model, series admittance y = 1/(r + jx) and half of the line
// charging at each end; Eq. 11: a three-phase branch's admittance is the
// inverse of its series impedance over the phases present), the current
// entering branch k at its from end is I_f = y (V_f - V_t) + j b/2 V_f and
// at its to end I_t = y (V_t - V_f) + j b/2 V_t (per phase, matrix y, no
// charging, for three phase).  The power leaving a bus into the branch is
// S = V conj(I); S_f + S_t is the branch loss.  One thread per (branch,
// scenario); the losses of a scenario are summed by one CTA in a fixed
// order (deterministic).

#include <cuda_runtime.h>

#include "device.h"

namespace pf {

namespace {

// Voltage of slot s of bus / node i, scenario gs, from the caller's polar
// [scenario][bus * ph] arrays.
__device__ __forceinline__ double2 volt(const double* vm, const double* va, size_t k) {
  double sn, cs;
  sincos(va[k], &sn, &cs);
  return make_double2(vm[k] * cs, vm[k] * sn);
}

__device__ __forceinline__ double2 cmul_(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// s = v conj(i)
__device__ __forceinline__ double2 vconj(double2 v, double2 i) {
  return make_double2(v.x * i.x + v.y * i.y, v.y * i.x - v.x * i.y);
}

template <int PH>
__global__ void __launch_bounds__(256) k_flows(const int2* ft, const double* yb, const double* sh,
                                               int n, int m, int B, const double* vm,
                                               const double* va, double* pf_, double* qf,
                                               double* pt, double* qt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x, gs = blockIdx.y;
  if (e >= m || gs >= B) return;
  const int2 b = __ldg(ft + e);
  const size_t base = (size_t)gs * n * PH;
  double2 Vf[PH], Vt[PH];
#pragma unroll
  for (int a = 0; a < PH; ++a) {
    Vf[a] = volt(vm, va, base + (size_t)b.x * PH + a);
    Vt[a] = volt(vm, va, base + (size_t)b.y * PH + a);
  }
  const double* y = yb + (size_t)e * 18;
#pragma unroll
  for (int a = 0; a < PH; ++a) {
    double2 If = make_double2(0.0, 0.0);
#pragma unroll
    for (int c = 0; c < PH; ++c) {
      const double2 yac = make_double2(y[2 * (3 * a + c)], y[2 * (3 * a + c) + 1]);
      const double2 d = make_double2(Vf[c].x - Vt[c].x, Vf[c].y - Vt[c].y);
      const double2 t = cmul_(yac, d);
      If.x += t.x;
      If.y += t.y;
    }
    double2 It = make_double2(-If.x, -If.y);
    if (PH == 1) {  // line charging j b/2 at each end
      const double h = sh[e];
      If.x -= h * Vf[0].y;
      If.y += h * Vf[0].x;
      It.x -= h * Vt[0].y;
      It.y += h * Vt[0].x;
    }
    const double2 Sf = vconj(Vf[a], If), St = vconj(Vt[a], It);
    const size_t o = ((size_t)gs * m + e) * PH + a;
    pf_[o] = Sf.x;
    qf[o] = Sf.y;
    pt[o] = St.x;
    qt[o] = St.y;
  }
}

// loss[gs] = (sum of P_f + P_t, sum of Q_f + Q_t) over the scenario's
// branch slots, one CTA per scenario, fixed order.
__global__ void __launch_bounds__(256) k_losses(int cnt, const double* pf_, const double* qf,
                                                const double* pt, const double* qt,
                                                double* loss) {
  __shared__ double sp[256], sq[256];
  const size_t base = (size_t)blockIdx.x * cnt;
  double p = 0.0, q = 0.0;
  for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
    p += pf_[base + k] + pt[base + k];
    q += qf[base + k] + qt[base + k];
  }
  sp[threadIdx.x] = p;
  sq[threadIdx.x] = q;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sp[threadIdx.x] += sp[threadIdx.x + s];
      sq[threadIdx.x] += sq[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    loss[2 * blockIdx.x] = sp[0];
    loss[2 * blockIdx.x + 1] = sq[0];
  }
}

}  // namespace

cudaError_t launch_branch_flows(int ph, const int2* ft, const double* yb, const double* sh, int n,
                                int m, int B, const double* vm, const double* va, double* pf_,
                                double* qf, double* pt, double* qt, double* loss,
                                cudaStream_t st) {
  if (m > 0) {
    const dim3 grid((m + 255) / 256, B);
    if (ph == 1)
      k_flows<1><<<grid, 256, 0, st>>>(ft, yb, sh, n, m, B, vm, va, pf_, qf, pt, qt);
    else
      k_flows<3><<<grid, 256, 0, st>>>(ft, yb, sh, n, m, B, vm, va, pf_, qf, pt, qt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_losses<<<B, 256, 0, st>>>(m * ph, pf_, qf, pt, qt, loss);
  return cudaGetLastError();
}

}  // namespace pf
