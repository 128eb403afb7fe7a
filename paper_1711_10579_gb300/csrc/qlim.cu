// Reactive limits of PV buses and of the phases of three-phase PV nodes:
// the checks between the rounds of solves.
//
// Sec. II.A holds the magnitude of a PV bus by letting its generator supply
// whatever reactive power that takes.  A real generator has limits
// [q_min, q_max]; one that would leave them can no longer hold |V| and is
// modelled as a PQ bus whose reactive generation is the limit it crossed.
// After a round of solves the generator Q of every PV bus of a converged
// scenario is Q_i of Eq. 7 (from I = Y V at the final voltages) plus the
// bus's own reactive load at |V_i| (Eq. 12-15); a bus outside its limits
// gets the scenario bus type kPQLimit and its limit as generation, which
// the mismatch (Eq. 8-9) and Jacobian (Eq. 10) read in the next round.
// Three phase: the reactive injection Q_g of a PV phase slot is an unknown
// of the current-injection Newton (w.qg); a slot outside [q_min, q_max] is
// held at the limit it crossed (w.qg fixed, its bit set in w.bt, |V| free)
// and keeps the plain columns of Eq. 21-23 in the next round.
// Rows are in the numbering of the solve's ordering; w.bt is [row][B].

#include <cuda_runtime.h>

#include "device.h"

namespace pf {

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_qlim_init(DevSys S, DevWork w, int three) {
  const size_t k = (size_t)blockIdx.x * kThreads + threadIdx.x;
  const int B = w.B;
  if (k >= (size_t)S.n * B) return;
  const int i = (int)(k / B), gs = (int)(k % B);
  if (three) {
    w.bt[k] = 0;  // no phase held
  } else {
    w.bt[k] = S.btype[i];
    w.qsw[k] = 0.0;
  }
  if (i == 0) {
    w.qdone[gs] = 0;
    w.qcnt[gs] = 0;
    w.qit[gs] = 0;
    w.qit[B + gs] = 0;
    w.qit[2 * B + gs] = 0;
    w.qus[gs] = 0.0;
  }
}

// One thread per (row, scenario).  The thread of row 0 also adds the
// round's counters to the scenario's totals and keeps the result of a
// scenario that failed (it takes no further part in the rounds).
__global__ void __launch_bounds__(kThreads) k_qlim_check(DevSys S, DevWork w, const pf_info* info,
                                                         int round, int three) {
  const size_t k = (size_t)blockIdx.x * kThreads + threadIdx.x;
  const int B = w.B;
  if (k >= (size_t)S.n * B) return;
  const int i = (int)(k / B), gs = (int)(k % B);
  const int status = info[gs].status;
  if (w.qdone[gs]) return;  // failed in an earlier round
  if (i == 0) {
    pf_info f = info[gs];
    w.qit[gs] += f.iterations;
    w.qit[B + gs] += f.linear_iterations;
    w.qus[gs] += f.solve_us;
    if (status != PF_OK) {
      f.iterations = w.qit[gs];
      f.linear_iterations = w.qit[B + gs];
      f.solve_us = w.qus[gs];
      f.q_rounds = round;
      w.qinfo[gs] = f;
      w.qdone[gs] = 1;
    }
  }
  if (status != PF_OK) return;
  if (three) {
    const int t = S.btype[i];
    if (!(t & 16) || (t & 8)) return;  // not a PV node, or the source
    int held = w.bt[k], add = 0;
    for (int a = 0; a < 3; ++a) {
      if (!((t >> a) & 1) || ((held >> a) & 1)) continue;
      const double q = w.qg[k * 3 + a], qmax = S.q_max[i * 3 + a], qmin = S.q_min[i * 3 + a];
      double lim;
      if (q > qmax) lim = qmax;
      else if (q < qmin) lim = qmin;
      else continue;
      w.qg[k * 3 + a] = lim;
      held |= 1 << a;
      ++add;
    }
    if (add) {
      w.bt[k] = (int8_t)held;
      atomicAdd(w.qcnt + gs, add);
      atomicAdd(w.nsw, add);
      w.qit[2 * B + gs] = round;
    }
    return;
  }
  if (w.bt[k] != PF_PV) return;
  // Q_i = Im(V_i conj(I_i)), I = Y V (Eq. 1, 7)
  const double2* Y = reinterpret_cast<const double2*>(S.y_val);
  double2 I = make_double2(0.0, 0.0);
  for (int e = S.y_rowptr[i]; e < S.y_rowptr[i + 1]; ++e) {
    const double2 y = Y[e], v = w.V[(size_t)S.y_col[e] * B + gs];
    I.x += y.x * v.x - y.y * v.y;
    I.y += y.x * v.y + y.y * v.x;
  }
  const double2 V = w.V[k];
  const double vm = w.vm[k];
  const double shape = S.zip[3 * i] + (S.zip[3 * i + 1] + S.zip[3 * i + 2] * vm) * vm;
  const double qg = (V.y * I.x - V.x * I.y) + w.spec[k * 3 + 1] * shape;
  double lim;
  if (qg > S.q_max[i]) lim = S.q_max[i];
  else if (qg < S.q_min[i]) lim = S.q_min[i];
  else return;
  w.bt[k] = (int8_t)kPQLimit;
  w.qsw[k] = lim;
  atomicAdd(w.qcnt + gs, 1);
  atomicAdd(w.nsw, 1);
  w.qit[2 * B + gs] = round;  // the last round that switched a bus of gs
}

// The scenario's result over all rounds: summed counters, the kept result
// of a failed scenario, and PF_ERR_MAXITER for one still switching when the
// rounds were capped.
__global__ void __launch_bounds__(kThreads) k_qlim_final(DevWork w, pf_info* info, int round,
                                                         int capped) {
  const int gs = blockIdx.x * kThreads + threadIdx.x, B = w.B;
  if (gs >= B) return;
  pf_info f = info[gs];
  if (w.qdone[gs]) {
    f = w.qinfo[gs];
  } else {
    f.iterations = w.qit[gs];
    f.linear_iterations = w.qit[B + gs];
    f.solve_us = w.qus[gs];
    if (capped && w.qit[2 * B + gs] == round) f.status = PF_ERR_MAXITER;
    // the scenario's own rounds: up to the one after its last switch
    f.q_rounds = min(w.qit[2 * B + gs] + 1, round);
  }
  f.q_switched = w.qcnt[gs];
  info[gs] = f;
}

}  // namespace

cudaError_t launch_qlim_init(const DevSys& S, const DevWork& w, bool three, cudaStream_t st) {
  const size_t tot = (size_t)S.n * w.B;
  k_qlim_init<<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, st>>>(S, w, three);
  return cudaGetLastError();
}

cudaError_t launch_qlim_check(const DevSys& S, const DevWork& w, const pf_info* info, int round,
                              bool three, cudaStream_t st) {
  const size_t tot = (size_t)S.n * w.B;
  k_qlim_check<<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, st>>>(S, w, info,
                                                                                  round, three);
  return cudaGetLastError();
}

cudaError_t launch_qlim_final(const DevWork& w, pf_info* info, int round, int capped,
                              cudaStream_t st) {
  k_qlim_final<<<(w.B + kThreads - 1) / kThreads, kThreads, 0, st>>>(w, info, round, capped);
  return cudaGetLastError();
}

}  // namespace pf
