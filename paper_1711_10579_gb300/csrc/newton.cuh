#pragma once
// Persistent Newton power-flow kernel for sm_103a (templates; each
// newton_<block size><precision>.cu instantiates one block size and one
// precision, so that the kernels compile in parallel).
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
// Single solves run one cluster of up to 16 CTAs; Newton-Krylov batches run
// one CTA per S scenarios (Newton-Raphson batches run as the phase kernels
// of batch.cu).  Values are interleaved as [entry][scenario] so that
// neighbouring threads of a batch read neighbouring memory.
#include "kernels.cuh"

namespace pf {

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------

// The solves of cluster (or, with CL false, CTA) number cid.
template <int BS, typename TF, bool CL, bool NK>
__device__ __forceinline__ void newton_solve(const DevSys& S, const DevWork& w, const DevOpts& o,
                                             int cid) {
  constexpr bool THREE = (BS == 6);
  constexpr int NSL = THREE ? 3 : 1;  // complex voltages per row
  const int csize = CL ? (int)cg::this_cluster().num_blocks() : 1;
  const int crank = CL ? (int)cg::this_cluster().block_rank() : 0;
  Team tm;
  // consecutive items go to different CTAs of the cluster (all SMs busy on
  // short loops); scenario slots stay in the low bits
  tm.tid = (threadIdx.x / o.S) * (o.S * csize) + crank * o.S + (threadIdx.x & (o.S - 1));
  tm.nthr = csize * blockDim.x;
  tm.S = o.S;
  tm.s0 = cid * o.S;
  tm.ns = min(o.S, w.B - tm.s0);
  if (tm.ns <= 0) return;  // whole cluster exits together
  const int n = S.n, B = w.B;
  // CTA 0 alone ("solo") runs the narrow levels and the triangular solves of a
  // single solve: __syncthreads instead of cluster barriers and their fences
  Team solo = tm;
  solo.tid = threadIdx.x;
  solo.nthr = blockDim.x;
  extern __shared__ __align__(16) unsigned char dsm[];
  TF* yv = o.y_in_smem ? reinterpret_cast<TF*>(dsm) : reinterpret_cast<TF*>(w.y);
  // Newton-Krylov shared memory after the solve vector: per-slot GMRES state,
  // per-warp reduction partials and reduction results
  TF* nk_state = reinterpret_cast<TF*>(dsm + (o.y_in_smem ? (size_t)n * BS * sizeof(TF) : 0));
  TF* nk_redw = nk_state + (NK ? (size_t)o.S * GmresState<TF>::words(o.m) : 0);
  TF* nk_rs = nk_redw + (NK ? (size_t)(blockDim.x / 32) * kMaxJ * o.S : 0);
  // batched sweeps: partial sums of a row's lanes in different warps; then
  // the batched factorisation's ring of in-flight items (16-byte aligned)
  TF* sw_red = nk_rs + (NK ? (size_t)kMaxJ * o.S : 0);
  unsigned char* sw_ring =
      o.ring ? reinterpret_cast<unsigned char*>(
                   ((reinterpret_cast<uintptr_t>(sw_red + (o.S > 1 ? (size_t)blockDim.x * BS : 0))) +
                    15) &
                   ~(uintptr_t)15)
             : nullptr;
  __shared__ int sh_lin[32];       // inner iterations, whole solve
  __shared__ int sh_lin_step[32];  // inner iterations, this Newton step
  __shared__ int sh_kk[32];
  __shared__ unsigned sh_inner;
  __shared__ TF sh_bnorm[32], sh_eta[32], sh_hk1[32];
  __shared__ TF sh_rho[32], sh_rho0[32], sh_alpha[32], sh_omega[32];  // BiCGSTAB
  __shared__ unsigned sh_sdone, sh_restart;
  __shared__ int sh_status[32];
  __shared__ double sh_prev[32];  // mismatch norm of the previous iteration
  __shared__ unsigned sh_act;
  __shared__ int sh_refine;
  __shared__ unsigned long long sh_t0;
  if (threadIdx.x == 0) {
    sh_t0 = global_ns();
    for (int s = 0; s < 32; ++s) {
      sh_status[s] = kRunning;
      sh_lin[s] = 0;
      sh_prev[s] = 0.0;
    }
    sh_act = (tm.ns >= 32) ? 0xffffffffu : ((1u << tm.ns) - 1u);
  }
  __syncthreads();
  tm.act = sh_act;
  // optional per-phase timing, kept by one thread of the first cluster
  const bool prof = o.prof != nullptr && cid == 0 && crank == 0 && threadIdx.x == 0;
  unsigned long long t_last = prof ? global_ns() : 0ull;
  auto tick = [&](int phase) {
    if (prof) {
      const unsigned long long t = global_ns();
      o.prof[phase] += t - t_last;
      t_last = t;
    }
  };

  // ---- set-up: specified injections, start voltage, accumulators ----
  run_rows<CL>(tm, n, [&](int i, int gs) {
    setup_row<THREE>(S, w, i, gs);
  });
  tick(kProfSetup);

  int it = 0;
  for (;; ++it) {
    // ---- A: mismatch + Jacobian ----
    run_rows_max<CL>(tm, n, w.norm + (size_t)(it & 1) * B, [&](int i, int gs) {
      double nrm;
      TF* jcopy = NK ? reinterpret_cast<TF*>(w.jm) : nullptr;
      if constexpr (THREE) {
        mismatch_jacobian_3ph<TF>(S, w, i, gs, nrm, jcopy);
      } else {
        mismatch_jacobian_1ph<TF>(S, w, i, gs, nrm, jcopy);
      }
      return nrm;
    });
    tick(kProfMismatch);
    if (o.mode == 1) return;  // inspection: F and J stay in the workspace

    // ---- stop test (every CTA decides identically from global values) ----
    if (threadIdx.x == 0) {
      unsigned act = 0;
      int refine = 0;
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
        if (st == kRunning && refine_now(o, it, nrm, sh_prev[s])) refine = 1;
        sh_prev[s] = nrm;
        if (crank == 0) {
          if (st != kRunning && w.out_info) {
            pf_info inf;
            inf.status = st;
            inf.iterations = it;
            inf.linear_iterations = sh_lin[s];
            inf.fallback = 0;
            inf.mismatch = nrm;
            inf.max_step = it > 0 ? __longlong_as_double((long long)__ldcg(w.step + (size_t)((it - 1) & 1) * B + gs)) : 0.0;
            inf.solve_us = 0.0;
            inf.q_switched = 0;
            inf.q_rounds = 1;
            w.out_info[gs] = inf;
          }
          // the buffers of the next iteration (read last one iteration ago)
          w.norm[(size_t)((it + 1) & 1) * B + gs] = 0ull;
          w.step[(size_t)((it + 1) & 1) * B + gs] = 0ull;
        }
      }
      sh_act = act;
      sh_refine = refine;
    }
    __syncthreads();
    tm.act = sh_act;
    const int n_refine = (sh_refine || o.mode == 2) ? o.refine : 0;
    tick(kProfStop);
    if (tm.act == 0) break;

    // ---- B: numeric factorisation, two parallel steps per level; the narrow
    // top levels of a single solve run in CTA 0 alone ----
    factor_levels<BS, TF, CL>(S, w, tm, 0, S.fac_solo_from, sw_ring);
    solo.act = tm.act;
    if (S.fac_solo_from < S.nflev) {
      if (crank == 0) factor_levels<BS, TF, false>(S, w, solo, S.fac_solo_from, S.nflev, sw_ring);
      csync<CL>();
    }
    tick(kProfFactor);
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
            inf.linear_iterations = sh_lin[s];
            inf.fallback = 0;
            inf.mismatch = __longlong_as_double((long long)__ldcg(w.norm + (size_t)(it & 1) * B + gs));
            inf.max_step = 0.0;
            inf.solve_us = 0.0;
            inf.q_switched = 0;
            inf.q_rounds = 1;
            w.out_info[gs] = inf;
          }
        }
      }
      sh_act = act;
    }
    __syncthreads();
    tm.act = sh_act;
    if (tm.act == 0) break;

    // ---- C (Newton-Krylov): GMRES(m) on J dx = F, right ILU(0) ----
    if constexpr (NK) {
      const int m = o.m;
      const int slot = tm.tid & (tm.S - 1);
      const int gs = tm.s0 + slot;
      TF* const V0 = reinterpret_cast<TF*>(w.vb);
      TF* const W = reinterpret_cast<TF*>(w.wv);
      TF* const Z = reinterpret_cast<TF*>(w.zg);
      TF* const X = reinterpret_cast<TF*>(w.xg);
      const TF* const JM = reinterpret_cast<const TF*>(w.jm);
      const size_t NV = (size_t)n * B * BS;
      const int first = tm.tid / tm.S, stride = tm.nthr / tm.S;
      int par = 0;
      auto slot_on = [&](unsigned bits) { return slot < tm.ns && ((bits >> slot) & 1u); };
      auto rs = [&](int j) { return nk_rs[j * tm.S + slot]; };
      auto tsum = [&](int J, auto part) {
        team_sum<CL, TF>(tm, J, part, nk_redw, nk_rs, reinterpret_cast<TF*>(w.gred), par, csize,
                         crank, B);
        par ^= 1;
      };
      // J u for row i (block SpMV on the Jacobian's own pattern)
      auto jrow = [&](int i, const TF* u, TF (&out)[BS]) {
#pragma unroll
        for (int c = 0; c < BS; ++c) out[c] = TF(0);
        for (int e = S.lu_rowptr[i]; e < S.lu_rowptr[i + 1]; ++e) {
          TF Jb[BS * BS];
          blk_load<BS>(JM + ((size_t)e * B + gs) * BS * BS, Jb);
          const size_t bj = ((size_t)S.lu_col[e] * B + gs) * BS;
          TF uj[BS];
#pragma unroll
          for (int c = 0; c < BS; ++c) uj[c] = __ldcg(u + bj + c);
#pragma unroll
          for (int r = 0; r < BS; ++r)
#pragma unroll
            for (int c = 0; c < BS; ++c) out[r] += Jb[r * BS + c] * uj[c];
        }
      };
      // z = M^-1 u by the ILU(0) sweeps in CTA 0 (u, z in global memory)
      auto precond = [&](const TF* u, TF* zout, bool accumulate, unsigned bits) {
        solo.act = bits;
        if (crank == 0) {
          run_rows<false>(solo, n, [&](int i, int g2) {
            const size_t bb = ((size_t)i * B + g2) * BS;
            for (int c = 0; c < BS; ++c) yv[bb + c] = __ldcg(u + bb + c);
          });
          sweep<BS, TF, true, false>(S, w, yv, solo, S.flev_ptr, S.fwd_rec, S.nflev, S.g_fwd, sw_red);
          sweep<BS, TF, false, false>(S, w, yv, solo, S.blev_ptr, S.bwd_rec, S.nblev, S.g_bwd, sw_red);
          run_rows<false>(solo, n, [&](int i, int g2) {
            const size_t bb = ((size_t)i * B + g2) * BS;
            for (int c = 0; c < BS; ++c) zout[bb + c] = accumulate ? zout[bb + c] + yv[bb + c] : yv[bb + c];
          });
        }
        csync<CL>();
      };
      // ||F||_2 and the inner tolerance eta = clamp(||F||_inf, rtol, 0.1)
      tsum(1, [&](int) {
        TF a = TF(0);
        if (slot_on(tm.act))
          for (int i = first; i < n; i += stride)
            for (int c = 0; c < BS; ++c) {
              const TF f = (TF)__ldcg(w.F + ((size_t)i * B + gs) * BS + c);
              a += f * f;
              X[((size_t)i * B + gs) * BS + c] = TF(0);
            }
        return a;
      });
      if (threadIdx.x < tm.ns) {
        const int t = threadIdx.x;
        sh_lin_step[t] = 0;
        const double ninf = __longlong_as_double((long long)__ldcg(w.norm + (size_t)(it & 1) * B + tm.s0 + t));
        sh_bnorm[t] = sqrt(nk_rs[t]);
        const double eta = (o.mode == 2) ? o.rtol : fmin(0.1, fmax(o.rtol, ninf));
        sh_eta[t] = (TF)eta;
      }
      __syncthreads();
      if (o.krylov == 1) {
        // BiCGSTAB (the Krylov method of Sec. III.B), right-preconditioned by
        // ILU(0): solves J M^-1 u = F with x = M^-1 u from x = 0.  Work
        // vectors borrow the first 8 GMRES basis slots.
        TF* const R = V0;
        TF* const RH = V0 + NV;
        TF* const P = V0 + 2 * NV;
        TF* const VV = V0 + 3 * NV;
        TF* const SV = V0 + 4 * NV;
        TF* const TV = V0 + 5 * NV;
        TF* const PH = V0 + 6 * NV;
        TF* const SH = V0 + 7 * NV;
        auto q_of = [&](int i, int c) { return ((size_t)i * B + gs) * BS + c; };
        if (slot_on(tm.act))
          for (int i = first; i < n; i += stride)
            for (int c = 0; c < BS; ++c) {
              const size_t q = q_of(i, c);
              const TF f = (TF)__ldcg(w.F + q);
              R[q] = f;
              RH[q] = f;
              P[q] = TF(0);
              VV[q] = TF(0);
            }
        if (threadIdx.x < tm.ns) {
          const int t = threadIdx.x;
          sh_rho[t] = sh_bnorm[t] * sh_bnorm[t];  // (r_hat, r) with r = r_hat = F
          sh_rho0[t] = TF(1);
          sh_alpha[t] = TF(1);
          sh_omega[t] = TF(1);
        }
        if (threadIdx.x == 0) {
          unsigned bits = 0;
          for (int t = 0; t < tm.ns; ++t)
            if (((tm.act >> t) & 1u) && sh_bnorm[t] > TF(0) && o.max_lin > 0) bits |= 1u << t;
          sh_inner = bits;
        }
        csync<CL>();
        unsigned inner = sh_inner;
        while (inner != 0) {
          // p = r + beta (p - omega v), beta = (rho / rho_prev)(alpha / omega)
          if (slot_on(inner)) {
            const TF beta = (sh_rho[slot] / sh_rho0[slot]) * (sh_alpha[slot] / sh_omega[slot]);
            const TF om = sh_omega[slot];
            for (int i = first; i < n; i += stride)
              for (int c = 0; c < BS; ++c) {
                const size_t q = q_of(i, c);
                P[q] = R[q] + beta * (P[q] - om * VV[q]);
              }
          }
          csync<CL>();
          precond(P, PH, false, inner);
          // v = J p_hat, alpha = rho / (r_hat, v)
          tsum(1, [&](int) {
            TF a = TF(0);
            if (slot_on(inner))
              for (int i = first; i < n; i += stride) {
                TF jv[BS];
                jrow(i, PH, jv);
                for (int c = 0; c < BS; ++c) {
                  const size_t q = q_of(i, c);
                  VV[q] = jv[c];
                  a += RH[q] * jv[c];
                }
              }
            return a;
          });
          if (threadIdx.x < tm.ns && ((inner >> threadIdx.x) & 1u)) {
            const TF d = nk_rs[threadIdx.x];
            sh_alpha[threadIdx.x] = (d != TF(0)) ? sh_rho[threadIdx.x] / d : TF(0);
          }
          __syncthreads();
          // s = r - alpha v
          tsum(1, [&](int) {
            TF a = TF(0);
            if (slot_on(inner)) {
              const TF al = sh_alpha[slot];
              for (int i = first; i < n; i += stride)
                for (int c = 0; c < BS; ++c) {
                  const size_t q = q_of(i, c);
                  const TF sv = R[q] - al * VV[q];
                  SV[q] = sv;
                  a += sv * sv;
                }
            }
            return a;
          });
          // slots whose s already meets the tolerance finish with x += alpha p_hat
          if (threadIdx.x == 0) {
            unsigned done = 0;
            for (int t = 0; t < tm.ns; ++t)
              if (((inner >> t) & 1u) &&
                  (sqrt(nk_rs[t]) <= sh_eta[t] * sh_bnorm[t] || sh_alpha[t] == TF(0)))
                done |= 1u << t;
            sh_sdone = done;
          }
          __syncthreads();
          const unsigned sdone = sh_sdone, go = inner & ~sdone;
          if (slot_on(sdone)) {
            const TF al = sh_alpha[slot];
            for (int i = first; i < n; i += stride)
              for (int c = 0; c < BS; ++c) X[q_of(i, c)] += al * PH[q_of(i, c)];
          }
          csync<CL>();
          if (go != 0) {
            precond(SV, SH, false, go);
            // t = J s_hat, omega = (t, s) / (t, t)
            if (slot_on(go))
              for (int i = first; i < n; i += stride) {
                TF jt[BS];
                jrow(i, SH, jt);
                for (int c = 0; c < BS; ++c) TV[q_of(i, c)] = jt[c];
              }
            tsum(2, [&](int j) {
              TF a = TF(0);
              if (slot_on(go))
                for (int i = first; i < n; i += stride)
                  for (int c = 0; c < BS; ++c) {
                    const size_t q = q_of(i, c);
                    a += TV[q] * (j == 0 ? SV[q] : TV[q]);
                  }
              return a;
            });
            if (threadIdx.x < tm.ns && ((go >> threadIdx.x) & 1u)) {
              const TF ts = nk_rs[threadIdx.x], tt = nk_rs[tm.S + threadIdx.x];
              sh_omega[threadIdx.x] = (tt > TF(0)) ? ts / tt : TF(0);
            }
            __syncthreads();
            // x += alpha p_hat + omega s_hat; r = s - omega t; ||r||^2, (r_hat, r)
            tsum(2, [&](int j) {
              TF a = TF(0);
              if (slot_on(go)) {
                const TF al = sh_alpha[slot], om = sh_omega[slot];
                for (int i = first; i < n; i += stride)
                  for (int c = 0; c < BS; ++c) {
                    const size_t q = q_of(i, c);
                    if (j == 0) {
                      X[q] += al * PH[q] + om * SH[q];
                      const TF r = SV[q] - om * TV[q];
                      R[q] = r;
                      a += r * r;
                    } else {
                      a += RH[q] * R[q];
                    }
                  }
              }
              return a;
            });
          }
          if (threadIdx.x == 0) {
            unsigned nxt = 0, rst = 0;
            for (int t = 0; t < tm.ns; ++t) {
              if (!((inner >> t) & 1u)) continue;
              sh_lin[t] += 1;
              sh_lin_step[t] += 1;
              if ((sdone >> t) & 1u) continue;
              const TF res = sqrt(nk_rs[t]), rho = nk_rs[tm.S + t];
              sh_rho0[t] = sh_rho[t];
              sh_rho[t] = rho;
              if (!(res <= sh_eta[t] * sh_bnorm[t]) && sh_lin_step[t] < o.max_lin &&
                  res > TF(0) && sh_omega[t] != TF(0)) {
                nxt |= 1u << t;
                // near breakdown, (r_hat, r) << |r_hat| |r| (r_hat = F, |F| =
                // bnorm; 1e-5 in FP32, 1e-10 in FP64): restart from the
                // current x with r_hat = r
                const TF brk = sizeof(TF) == 4 ? TF(1e-5) : TF(1e-10);
                if (!(fabs(rho) > brk * sh_bnorm[t] * res)) {
                  rst |= 1u << t;
                  sh_rho[t] = res * res;
                  sh_rho0[t] = TF(1);
                  sh_alpha[t] = TF(1);
                  sh_omega[t] = TF(1);
                }
              }
            }
            sh_inner = nxt;
            sh_restart = rst;
          }
          __syncthreads();
          inner = sh_inner;
          if (sh_restart != 0) {
            const unsigned rst = sh_restart;
            if (slot_on(rst))
              for (int i = first; i < n; i += stride)
                for (int c = 0; c < BS; ++c) {
                  const size_t q = q_of(i, c);
                  RH[q] = R[q];
                  P[q] = TF(0);
                  VV[q] = TF(0);
                }
            csync<CL>();
          }
        }
      } else
      for (int restart = 0;; ++restart) {
        // r = F - J x into V_0, and ||r||_2
        tsum(1, [&](int) {
          TF a = TF(0);
          if (slot_on(tm.act))
            for (int i = first; i < n; i += stride) {
              TF jx[BS];
              if (restart > 0) jrow(i, X, jx);
              for (int c = 0; c < BS; ++c) {
                const size_t q = ((size_t)i * B + gs) * BS + c;
                const TF r = (TF)__ldcg(w.F + q) - (restart > 0 ? jx[c] : TF(0));
                V0[q] = r;
                a += r * r;
              }
            }
          return a;
        });
        if (threadIdx.x == 0) {
          unsigned bits = 0;
          for (int t = 0; t < tm.ns; ++t) {
            sh_kk[t] = 0;
            if (!((tm.act >> t) & 1u)) continue;
            GmresState<TF> G;
            G.bind(nk_state, m, t);
            const TF beta = sqrt(nk_rs[t]);
            G.g[0] = beta;
            if (beta > sh_eta[t] * sh_bnorm[t] && sh_lin_step[t] < o.max_lin) bits |= 1u << t;
          }
          sh_inner = bits;
        }
        __syncthreads();
        unsigned inner = sh_inner;
        const unsigned started = inner;
        if (inner == 0) break;
        // v_0 = r / beta
        run_items<CL>(tm, n, [&](int i, int g2) {
          const int t = g2 - tm.s0;
          if (!((inner >> t) & 1u)) return;
          GmresState<TF> G;
          G.bind(nk_state, m, t);
          const TF inv = TF(1) / G.g[0];
          for (int c = 0; c < BS; ++c) V0[((size_t)i * B + g2) * BS + c] *= inv;
        });
        for (int k = 0; k < m; ++k) {
          // z = M^-1 v_k, then w = J z
          precond(V0 + (size_t)k * NV, Z, false, inner);
          if (slot_on(inner))
            for (int i = first; i < n; i += stride) {
              TF jz[BS];
              jrow(i, Z, jz);
              for (int c = 0; c < BS; ++c) W[((size_t)i * B + gs) * BS + c] = jz[c];
            }
          auto dots = [&](int j) {
            TF a = TF(0);
            if (slot_on(inner))
              for (int i = first; i < n; i += stride)
                for (int c = 0; c < BS; ++c) {
                  const size_t q = ((size_t)i * B + gs) * BS + c;
                  a += V0[(size_t)j * NV + q] * W[q];
                }
            return a;
          };
          auto orth = [&](const TF* hv) {  // w -= V_{0..k} hv (own rows)
            if (slot_on(inner))
              for (int i = first; i < n; i += stride)
                for (int c = 0; c < BS; ++c) {
                  const size_t q = ((size_t)i * B + gs) * BS + c;
                  TF v = W[q];
                  for (int j = 0; j <= k; ++j) v -= hv[j] * V0[(size_t)j * NV + q];
                  W[q] = v;
                }
          };
          const bool keeper = threadIdx.x < tm.ns && ((inner >> threadIdx.x) & 1u);
          GmresState<TF> G;
          G.bind(nk_state, m, keeper ? threadIdx.x : 0);
          TF* Hk = G.H + (size_t)k * (m + 1);
          // classical Gram-Schmidt, twice (CGS2)
          TF hv[kMaxJ];
          tsum(k + 1, dots);
          for (int j = 0; j <= k; ++j) hv[j] = rs(j);
          if (keeper)
            for (int j = 0; j <= k; ++j) Hk[j] = nk_rs[j * tm.S + threadIdx.x];
          orth(hv);
          tsum(k + 1, dots);
          for (int j = 0; j <= k; ++j) hv[j] = rs(j);
          if (keeper)
            for (int j = 0; j <= k; ++j) Hk[j] += nk_rs[j * tm.S + threadIdx.x];
          orth(hv);
          tsum(1, [&](int) {
            TF a = TF(0);
            if (slot_on(inner))
              for (int i = first; i < n; i += stride)
                for (int c = 0; c < BS; ++c) {
                  const TF v = W[((size_t)i * B + gs) * BS + c];
                  a += v * v;
                }
            return a;
          });
          // Hessenberg column k: apply the earlier rotations, make a new one
          if (keeper) {
            const int t = threadIdx.x;
            const TF hk1 = sqrt(nk_rs[t]);
            sh_hk1[t] = hk1;
            for (int j = 0; j < k; ++j) {
              const TF a0 = Hk[j], a1 = Hk[j + 1];
              Hk[j] = G.cs[j] * a0 + G.sn[j] * a1;
              Hk[j + 1] = -G.sn[j] * a0 + G.cs[j] * a1;
            }
            const TF den = sqrt(Hk[k] * Hk[k] + hk1 * hk1);
            bool stop = false;
            if (den > TF(0)) {
              G.cs[k] = Hk[k] / den;
              G.sn[k] = hk1 / den;
              Hk[k] = den;
              Hk[k + 1] = TF(0);
              G.g[k + 1] = -G.sn[k] * G.g[k];
              G.g[k] = G.cs[k] * G.g[k];
              sh_kk[t] = k + 1;
            } else {
              stop = true;  // breakdown with a zero column: keep the first k steps
            }
            sh_lin[t] += 1;
            sh_lin_step[t] += 1;
            const TF res = G.g[k + 1] < TF(0) ? -G.g[k + 1] : G.g[k + 1];
            if (stop || res <= sh_eta[t] * sh_bnorm[t] || sh_lin_step[t] >= o.max_lin ||
                !(hk1 > TF(0)))
              atomicAnd(&sh_inner, ~(1u << t));
          }
          __syncthreads();
          const unsigned nxt = sh_inner;
          // v_{k+1} = w / h_{k+1,k} for the slots that go on
          if (k + 1 < m && nxt != 0) {
            run_items<CL>(tm, n, [&](int i, int g2) {
              const int t = g2 - tm.s0;
              if (!((nxt >> t) & 1u)) return;
              const TF inv = TF(1) / sh_hk1[t];
              for (int c = 0; c < BS; ++c) {
                const size_t q = ((size_t)i * B + g2) * BS + c;
                V0[(size_t)(k + 1) * NV + q] = W[q] * inv;
              }
            });
          }
          inner = nxt;
          if (inner == 0) break;
        }
        // y = R^-1 g per slot; x += M^-1 (V y)
        if (threadIdx.x < tm.ns && ((started >> threadIdx.x) & 1u)) {
          const int t = threadIdx.x, kk = sh_kk[t];
          GmresState<TF> G;
          G.bind(nk_state, m, t);
          for (int j = kk - 1; j >= 0; --j) {
            TF v = G.g[j];
            for (int l = j + 1; l < kk; ++l) v -= G.H[j + (size_t)l * (m + 1)] * G.y[l];
            G.y[j] = v / G.H[j + (size_t)j * (m + 1)];
          }
        }
        __syncthreads();
        run_items<CL>(tm, n, [&](int i, int g2) {
          const int t = g2 - tm.s0;
          const size_t bq = ((size_t)i * B + g2) * BS;
          if (!((started >> t) & 1u)) {
            for (int c = 0; c < BS; ++c) W[bq + c] = TF(0);
            return;
          }
          GmresState<TF> G;
          G.bind(nk_state, m, t);
          const int kk = sh_kk[t];
          for (int c = 0; c < BS; ++c) {
            TF v = TF(0);
            for (int j = 0; j < kk; ++j) v += G.y[j] * V0[(size_t)j * NV + bq + c];
            W[bq + c] = v;
          }
        });
        precond(W, X, true, started);
      }
      // the Newton step
      run_rows<CL>(tm, n, [&](int i, int g2) {
        const size_t bq = ((size_t)i * B + g2) * BS;
        for (int c = 0; c < BS; ++c) w.dx[bq + c] = (double)__ldcg(X + bq + c);
      });
      tick(kProfSolve);
    } else {
    // ---- C: triangular solves, then FP64 refinement ----
    for (int pass = 0; pass <= n_refine; ++pass) {
      // right-hand side: F, or the FP64 residual of the current step
      if (pass > 0) {
        // voltage change of the step (complex), for J dx evaluated from Y and V
        run_rows<CL>(tm, n, [&](int i, int gs) {
          dv_row<THREE>(S, w, i, gs);
        });
        run_rows<CL>(tm, n, [&](int i, int gs) {
          resid_row<THREE>(S, w, i, gs);
        });
      }
      tick(kProfResidual);
      // forward and backward sweeps: CTA 0 alone for a single solve
      solo.act = tm.act;
      // (Newton-Raphson batches run as the phase kernels of batch.cu)
      if (crank == 0) {
        const double* rhs = (pass == 0) ? w.F : w.r;
        run_rows<false>(solo, n, [&](int i, int gs) {
          const size_t b = ((size_t)i * B + gs) * BS;
          for (int c = 0; c < BS; ++c) yv[b + c] = (TF)__ldcg(rhs + b + c);
        });
        sweep<BS, TF, true, false>(S, w, yv, solo, S.flev_ptr, S.fwd_rec, S.nflev, S.g_fwd, sw_red);
        sweep<BS, TF, false, false>(S, w, yv, solo, S.blev_ptr, S.bwd_rec, S.nblev, S.g_bwd, sw_red);
        run_rows<false>(solo, n, [&](int i, int gs) {
          const size_t b = ((size_t)i * B + gs) * BS;
          for (int c = 0; c < BS; ++c) {
            const double v = (double)yv[b + c];
            w.dx[b + c] = (pass == 0) ? v : w.dx[b + c] + v;
          }
        });
      }
      csync<CL>();
      tick(kProfSolve);
    }

    }
    if (o.mode == 2) return;  // inspection: the step stays in the workspace

    // ---- E: voltage update ----
    run_rows_max<CL>(tm, n, w.step + (size_t)(it & 1) * B, [&](int i, int gs) {
      return update_row<THREE>(S, w, i, gs);
    });
    tick(kProfUpdate);
  }

  // ---- results in the caller's numbering ----
  tm.act = (tm.ns >= 32) ? 0xffffffffu : ((1u << tm.ns) - 1u);
  run_rows<CL>(tm, n, [&](int i, int gs) {
    output_row<THREE>(S, w, i, gs, sh_status[gs - tm.s0] == PF_OK);
  });
  tick(kProfOutput);
  if (crank == 0 && threadIdx.x == 0 && w.out_info) {
    const double us = (double)(global_ns() - sh_t0) * 1e-3;
    for (int s = 0; s < tm.ns; ++s) w.out_info[tm.s0 + s].solve_us = us;
  }
}

template <int BS, typename TF, bool CL, bool NK>
__global__ void __launch_bounds__(BS == 2 ? 512 : 256) newton_kernel(DevSys S, DevWork w, DevOpts o) {
  const int csize = CL ? (int)cg::this_cluster().num_blocks() : 1;
  newton_solve<BS, TF, CL, NK>(S, w, o, blockIdx.x / csize);
}

// Several cases of different sizes in one launch: CTA (or, with CL, cluster)
// b solves the job list.job[b] of the descriptor array (its own case,
// workspace, inputs and outputs) as a single-scenario Newton-Raphson solve.
// Descriptors, inputs and outputs may live in pinned host memory.  When its
// results are written the CTA (cluster) raises the job's done flag, so every
// job can be retired on its own while the rest of the launch still runs.
template <int BS, typename TF, bool CL>
__global__ void __launch_bounds__(BS == 2 ? 512 : 256)
    newton_group_kernel(const GroupJob* desc, GroupList list) {
  const int csize = CL ? (int)cg::this_cluster().num_blocks() : 1;
  const int crank = CL ? (int)cg::this_cluster().block_rank() : 0;
  __shared__ GroupJob job;
  {
    const unsigned* src = reinterpret_cast<const unsigned*>(desc + list.job[blockIdx.x / csize]);
    unsigned* dst = reinterpret_cast<unsigned*>(&job);
    for (int k = threadIdx.x; k < (int)(sizeof(GroupJob) / 4); k += blockDim.x) dst[k] = src[k];
  }
  __syncthreads();
  newton_solve<BS, TF, CL, false>(job.S, job.w, job.o, 0);
  // the results (every thread's writes) reach the host before the flag
  __threadfence_system();
  csync<CL>();
  if (crank == 0 && threadIdx.x == 0) {
    __threadfence_system();
    *reinterpret_cast<volatile int*>(job.done) = 1;
  }
}

// ---------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------

template <int BS, typename TF, bool CL, bool NK>
cudaError_t launch_t(const DevSys& S, const DevWork& w, const DevOpts& o, int grid,
                            int cluster, int threads, cudaStream_t st) {
  auto kern = newton_kernel<BS, TF, CL, NK>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = dynamic_smem_bytes(BS, sizeof(TF), NK, S.n, o, threads);
  // (static + dynamic shared memory above 48 KB needs the opt-in)
  if (cfg.dynamicSmemBytes > 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cfg.dynamicSmemBytes);
    if (e != cudaSuccess) return e;
  }
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
template <int BS, typename TF, bool NK>
int max_cluster_t(int threads) {
  auto kern = newton_kernel<BS, TF, true, NK>;
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

template <int BS, typename TF, bool CL>
cudaError_t launch_group_t(const GroupJob* desc, const GroupList& list, size_t smem,
                                  int cluster, cudaStream_t st) {
  auto kern = newton_group_kernel<BS, TF, CL>;
  if (smem > 0) {  // (static + dynamic shared memory above 48 KB needs the opt-in)
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(list.n * cluster);
  cfg.blockDim = dim3(BS == 2 ? 512 : 256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (CL) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, desc, list);
}

// Entry points of one block size and precision (instantiated in
// newton_<block size><precision>.cu; dispatched by newton.cu).
template <int BS, typename TF>
cudaError_t launch_newton_as(bool nk, const DevSys& S, const DevWork& w, const DevOpts& o,
                             int grid, int cluster, int threads, cudaStream_t st) {
  const bool cl = cluster > 1;
  if (nk)
    return cl ? launch_t<BS, TF, true, true>(S, w, o, grid, cluster, threads, st)
              : launch_t<BS, TF, false, true>(S, w, o, grid, cluster, threads, st);
  return cl ? launch_t<BS, TF, true, false>(S, w, o, grid, cluster, threads, st)
            : launch_t<BS, TF, false, false>(S, w, o, grid, cluster, threads, st);
}

template <int BS, typename TF>
cudaError_t launch_group_as(const GroupJob* desc, const GroupList& list, size_t smem, int cluster,
                            cudaStream_t st) {
  return cluster > 1 ? launch_group_t<BS, TF, true>(desc, list, smem, cluster, st)
                     : launch_group_t<BS, TF, false>(desc, list, smem, cluster, st);
}

template <int BS, typename TF>
int max_cluster_as(bool nk, int threads) {
  return nk ? max_cluster_t<BS, TF, true>(threads) : max_cluster_t<BS, TF, false>(threads);
}

#define PF_NEWTON_INSTANTIATE(BSV, TFT)                                                          \
  template cudaError_t launch_newton_as<BSV, TFT>(bool, const DevSys&, const DevWork&,          \
                                                  const DevOpts&, int, int, int, cudaStream_t); \
  template cudaError_t launch_group_as<BSV, TFT>(const GroupJob*, const GroupList&, size_t,     \
                                                 int, cudaStream_t);                             \
  template int max_cluster_as<BSV, TFT>(bool, int);

}  // namespace pf
