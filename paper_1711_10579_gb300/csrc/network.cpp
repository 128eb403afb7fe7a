// Case validation and nodal admittance matrix assembly.
//
// Single phase: Eq. 2-3 of the paper, Y_ii = sum of the admittances at bus i
// (including the path to ground), Y_ij = -y_ij, with pi-model branches
// (series r + jx, half of the line charging b at each end).
// Three phase: Eq. 11, one 3x3 complex block per node pair; a branch's
// admittance is the inverse of its series impedance over the phases it
// carries.
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <sstream>

#include "host.h"

namespace pf {

namespace {

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

template <class T>
std::vector<T> copy_or(const T* p, size_t n, T dflt) {
  if (!p) return std::vector<T>(n, dflt);
  return std::vector<T>(p, p + n);
}

bool connected(int n, const std::vector<int>& f, const std::vector<int>& t,
               int root) {
  std::vector<std::vector<int>> adj(n);
  for (size_t e = 0; e < f.size(); ++e) {
    adj[f[e]].push_back(t[e]);
    adj[t[e]].push_back(f[e]);
  }
  std::vector<char> seen(n, 0);
  std::vector<int> stack{root};
  seen[root] = 1;
  int count = 1;
  while (!stack.empty()) {
    int v = stack.back();
    stack.pop_back();
    for (int u : adj[v])
      if (!seen[u]) {
        seen[u] = 1;
        ++count;
        stack.push_back(u);
      }
  }
  return count == n;
}

using cd = std::complex<double>;

// Inverse of a k x k complex matrix (k <= 3) by Gauss-Jordan elimination with
// partial pivoting.  Returns false when singular.
bool invert_small(int k, cd* a, cd* inv) {
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) inv[i * k + j] = (i == j) ? cd(1, 0) : cd(0, 0);
  for (int c = 0; c < k; ++c) {
    int piv = c;
    for (int r = c + 1; r < k; ++r)
      if (std::abs(a[r * k + c]) > std::abs(a[piv * k + c])) piv = r;
    if (!(std::abs(a[piv * k + c]) > 0.0)) return false;
    if (piv != c)
      for (int j = 0; j < k; ++j) {
        std::swap(a[c * k + j], a[piv * k + j]);
        std::swap(inv[c * k + j], inv[piv * k + j]);
      }
    cd d = a[c * k + c];
    for (int j = 0; j < k; ++j) {
      a[c * k + j] /= d;
      inv[c * k + j] /= d;
    }
    for (int r = 0; r < k; ++r) {
      if (r == c) continue;
      cd f = a[r * k + c];
      if (f == cd(0, 0)) continue;
      for (int j = 0; j < k; ++j) {
        a[r * k + j] -= f * a[c * k + j];
        inv[r * k + j] -= f * inv[c * k + j];
      }
    }
  }
  return true;
}

}  // namespace

// Optional reactive limits (per bus, or per node and phase): both or
// neither, each an interval (infinite ends allowed).
static int copy_q_limits(const pf_case_desc* d, size_t cnt, CaseData& c, std::string& err) {
  if ((d->q_min != nullptr) != (d->q_max != nullptr)) {
    err = "q_min and q_max go together";
    return PF_ERR_INVALID;
  }
  if (!d->q_min) return PF_OK;
  c.q_min.assign(d->q_min, d->q_min + cnt);
  c.q_max.assign(d->q_max, d->q_max + cnt);
  for (size_t k = 0; k < cnt; ++k)
    if (std::isnan(c.q_min[k]) || std::isnan(c.q_max[k]) || c.q_min[k] > c.q_max[k]) {
      std::ostringstream msg;
      msg << "slot " << k << " has reactive limits that are not an interval";
      err = msg.str();
      return PF_ERR_INVALID;
    }
  return PF_OK;
}

int copy_case(const pf_case_desc* d, CaseData& c, std::string& err) {
  std::ostringstream msg;
  if (!d) {
    err = "null case description";
    return PF_ERR_INVALID;
  }
  if (d->kind != PF_SINGLE_PHASE && d->kind != PF_THREE_PHASE) {
    err = "kind must be PF_SINGLE_PHASE (1) or PF_THREE_PHASE (3)";
    return PF_ERR_INVALID;
  }
  if (d->n_bus < 1 || d->n_branch < 0 || d->n_bus > (1 << 26) ||
      d->n_branch > (1 << 27)) {
    err = "n_bus must be >= 1 and n_branch >= 0 (and within int range)";
    return PF_ERR_INVALID;
  }
  const int n = d->n_bus, m = d->n_branch;
  c.kind = d->kind;
  c.n = n;
  c.m = m;
  if (m > 0 && (!d->br_from || !d->br_to)) {
    err = "br_from / br_to are required";
    return PF_ERR_INVALID;
  }
  c.br_from.assign(d->br_from, d->br_from + m);
  c.br_to.assign(d->br_to, d->br_to + m);
  for (int e = 0; e < m; ++e) {
    if (c.br_from[e] < 0 || c.br_from[e] >= n || c.br_to[e] < 0 ||
        c.br_to[e] >= n) {
      msg << "branch " << e << " has a bus index out of range";
      err = msg.str();
      return PF_ERR_INVALID;
    }
    if (c.br_from[e] == c.br_to[e]) {
      msg << "branch " << e << " is a self loop";
      err = msg.str();
      return PF_ERR_INVALID;
    }
  }
  c.zip = copy_or<double>(d->zip, (size_t)n * 3, 0.0);
  if (!d->zip)
    for (int i = 0; i < n; ++i) c.zip[3 * i] = 1.0;
  if (!finite_all(c.zip.data(), c.zip.size())) {
    err = "zip contains non-finite values";
    return PF_ERR_INVALID;
  }

  if (d->kind == PF_SINGLE_PHASE) {
    if (!d->bus_type || !d->br_r || !d->br_x) {
      err = "bus_type, br_r and br_x are required for a single-phase case";
      return PF_ERR_INVALID;
    }
    c.bus_type.resize(n);
    int slack = -1, nslack = 0;
    for (int i = 0; i < n; ++i) {
      int t = d->bus_type[i];
      if (t != PF_SLACK && t != PF_PV && t != PF_PQ) {
        msg << "bus " << i << " has an unknown type " << t;
        err = msg.str();
        return PF_ERR_INVALID;
      }
      c.bus_type[i] = (int8_t)t;
      if (t == PF_SLACK) {
        slack = i;
        ++nslack;
      }
    }
    if (nslack != 1) {
      msg << "a single-phase case needs exactly one slack bus (found " << nslack
          << ")";
      err = msg.str();
      return PF_ERR_INVALID;
    }
    c.v_set = copy_or<double>(d->v_set, n, 1.0);
    c.p_gen = copy_or<double>(d->p_gen, n, 0.0);
    c.q_gen = copy_or<double>(d->q_gen, n, 0.0);
    c.p_load = copy_or<double>(d->p_load, n, 0.0);
    c.q_load = copy_or<double>(d->q_load, n, 0.0);
    c.br_r.assign(d->br_r, d->br_r + m);
    c.br_x.assign(d->br_x, d->br_x + m);
    c.br_b = copy_or<double>(d->br_b, m, 0.0);
    for (auto* v : {&c.v_set, &c.p_gen, &c.q_gen, &c.p_load, &c.q_load, &c.br_r,
                    &c.br_x, &c.br_b})
      if (!finite_all(v->data(), v->size())) {
        err = "case data contain non-finite values";
        return PF_ERR_INVALID;
      }
    if (copy_q_limits(d, (size_t)n, c, err) != PF_OK) return PF_ERR_INVALID;
    for (int i = 0; i < n; ++i)
      if (c.bus_type[i] != PF_PQ && !(c.v_set[i] > 0.0)) {
        msg << "bus " << i << " needs a positive |V| set point";
        err = msg.str();
        return PF_ERR_INVALID;
      }
    for (int e = 0; e < m; ++e)
      if (c.br_r[e] == 0.0 && c.br_x[e] == 0.0) {
        msg << "branch " << e << " has zero impedance";
        err = msg.str();
        return PF_ERR_INVALID;
      }
    if (!connected(n, c.br_from, c.br_to, slack)) {
      err = "the grid is not connected (every bus must reach the slack)";
      return PF_ERR_INVALID;
    }
  } else {
    if (!d->phases || !d->br_phases || !d->br_z) {
      err = "phases, br_phases and br_z are required for a three-phase case";
      return PF_ERR_INVALID;
    }
    if (d->source < 0 || d->source >= n) {
      err = "source node out of range";
      return PF_ERR_INVALID;
    }
    // PV nodes (optional): bus_type PF_PV, |V| set point v_set[n], generation
    // p_gen[n][3] per phase
    c.bus_type.assign(n, (int8_t)PF_PQ);
    bool any_pv = false;
    if (d->bus_type) {
      for (int i = 0; i < n; ++i) {
        const int t = d->bus_type[i];
        if (t != PF_PV && t != PF_PQ && t != PF_SLACK) {
          msg << "node " << i << " has an unknown type " << t;
          err = msg.str();
          return PF_ERR_INVALID;
        }
        if (t == PF_PV) {
          if (i == d->source) {
            err = "the source node cannot be a PV node";
            return PF_ERR_INVALID;
          }
          c.bus_type[i] = (int8_t)PF_PV;
          any_pv = true;
        }
      }
    }
    if (any_pv && (!d->v_set || !d->p_gen)) {
      err = "PV nodes need v_set[n] and p_gen[n][3]";
      return PF_ERR_INVALID;
    }
    c.v_set = copy_or<double>(any_pv ? d->v_set : nullptr, n, 1.0);
    c.p_gen3 = copy_or<double>(any_pv ? d->p_gen : nullptr, (size_t)3 * n, 0.0);
    if (!finite_all(c.v_set.data(), c.v_set.size()) ||
        !finite_all(c.p_gen3.data(), c.p_gen3.size())) {
      err = "v_set or p_gen contain non-finite values";
      return PF_ERR_INVALID;
    }
    for (int i = 0; i < n; ++i)
      if (c.bus_type[i] == PF_PV && !(c.v_set[i] > 0.0)) {
        msg << "PV node " << i << " needs a positive |V| set point";
        err = msg.str();
        return PF_ERR_INVALID;
      }
    if (copy_q_limits(d, (size_t)3 * n, c, err) != PF_OK) return PF_ERR_INVALID;
    c.source = d->source;
    c.v_source = d->v_source > 0 ? d->v_source : 1.0;
    if (!std::isfinite(c.v_source)) {
      err = "v_source is not finite";
      return PF_ERR_INVALID;
    }
    c.phases.assign(d->phases, d->phases + n);
    for (int i = 0; i < n; ++i)
      if ((c.phases[i] & 7) == 0 || (c.phases[i] & ~7)) {
        msg << "node " << i << " has an invalid phase mask";
        err = msg.str();
        return PF_ERR_INVALID;
      }
    c.p_load3 = copy_or<double>(d->p_load, (size_t)3 * n, 0.0);
    c.q_load3 = copy_or<double>(d->q_load, (size_t)3 * n, 0.0);
    if (!finite_all(c.p_load3.data(), c.p_load3.size()) ||
        !finite_all(c.q_load3.data(), c.q_load3.size())) {
      err = "loads contain non-finite values";
      return PF_ERR_INVALID;
    }
    c.br_phases.assign(d->br_phases, d->br_phases + m);
    c.br_z.assign(d->br_z, d->br_z + (size_t)m * 18);
    if (!finite_all(c.br_z.data(), c.br_z.size())) {
      err = "br_z contains non-finite values";
      return PF_ERR_INVALID;
    }
    for (int e = 0; e < m; ++e) {
      uint8_t ph = c.br_phases[e];
      if ((ph & 7) == 0 || (ph & ~7) || (ph & ~c.phases[c.br_from[e]]) ||
          (ph & ~c.phases[c.br_to[e]])) {
        msg << "branch " << e
            << " carries phases missing at one of its ends (or none)";
        err = msg.str();
        return PF_ERR_INVALID;
      }
    }
    if (!connected(n, c.br_from, c.br_to, c.source)) {
      err = "the feeder is not connected to the source";
      return PF_ERR_INVALID;
    }
  }
  return PF_OK;
}

int build_ybus(const CaseData& c, Ybus& y, std::string& err) {
  const int n = c.n;
  y.n = n;
  y.ybs = (c.kind == PF_SINGLE_PHASE) ? 1 : 3;
  const int vb = 2 * y.ybs * y.ybs;  // doubles per block
  // pattern: diagonal plus both directions of every branch
  std::vector<std::vector<int>> cols(n);
  for (int i = 0; i < n; ++i) cols[i].push_back(i);
  for (int e = 0; e < c.m; ++e) {
    cols[c.br_from[e]].push_back(c.br_to[e]);
    cols[c.br_to[e]].push_back(c.br_from[e]);
  }
  y.rowptr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    auto& v = cols[i];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    y.rowptr[i + 1] = y.rowptr[i] + (int)v.size();
  }
  y.col.resize(y.rowptr[n]);
  for (int i = 0; i < n; ++i)
    std::copy(cols[i].begin(), cols[i].end(), y.col.begin() + y.rowptr[i]);
  y.val.assign((size_t)y.rowptr[n] * vb, 0.0);
  auto find = [&](int i, int j) {
    auto b = y.col.begin() + y.rowptr[i], e = y.col.begin() + y.rowptr[i + 1];
    return (int)(std::lower_bound(b, e, j) - y.col.begin());
  };
  if (c.kind == PF_SINGLE_PHASE) {
    for (int e = 0; e < c.m; ++e) {
      int f = c.br_from[e], t = c.br_to[e];
      cd ys = 1.0 / cd(c.br_r[e], c.br_x[e]);
      cd sh(0.0, c.br_b[e] / 2.0);
      auto add = [&](int i, int j, cd v) {
        int p = find(i, j);
        y.val[2 * p] += v.real();
        y.val[2 * p + 1] += v.imag();
      };
      add(f, f, ys + sh);
      add(t, t, ys + sh);
      add(f, t, -ys);
      add(t, f, -ys);
    }
  } else {
    for (int e = 0; e < c.m; ++e) {
      int f = c.br_from[e], t = c.br_to[e];
      int ph[3], k = 0;
      for (int s = 0; s < 3; ++s)
        if (c.br_phases[e] >> s & 1) ph[k++] = s;
      cd z[9], yb[9];
      for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
          const double* zz = &c.br_z[(size_t)e * 18 + 2 * (3 * ph[a] + ph[b])];
          z[a * k + b] = cd(zz[0], zz[1]);
        }
      if (!invert_small(k, z, yb)) {
        std::ostringstream msg;
        msg << "branch " << e << " has a singular impedance matrix";
        err = msg.str();
        return PF_ERR_INVALID;
      }
      auto add = [&](int i, int j, double sign) {
        int p = find(i, j);
        for (int a = 0; a < k; ++a)
          for (int b = 0; b < k; ++b) {
            size_t o = (size_t)p * vb + 2 * (3 * ph[a] + ph[b]);
            y.val[o] += sign * yb[a * k + b].real();
            y.val[o + 1] += sign * yb[a * k + b].imag();
          }
      };
      add(f, f, 1.0);
      add(t, t, 1.0);
      add(f, t, -1.0);
      add(t, f, -1.0);
    }
  }
  if (!finite_all(y.val.data(), y.val.size())) {
    err = "admittance matrix has non-finite entries";
    return PF_ERR_INVALID;
  }
  return PF_OK;
}

// Per-branch admittances for the branch-flow kernel: yb[e] a 3x3 complex
// matrix (row-major, (re, im) pairs; single phase: y = 1/(r + jx) at [0][0],
// three phase: the inverse of the series impedance over the branch's phases,
// zero elsewhere) and sh[e] = b/2 (single phase; 0 for three phase).
int branch_admittances(const CaseData& c, std::vector<double>& yb, std::vector<double>& sh,
                       std::string& err) {
  yb.assign((size_t)c.m * 18, 0.0);
  sh.assign(c.m, 0.0);
  for (int e = 0; e < c.m; ++e) {
    double* out = &yb[(size_t)e * 18];
    if (c.kind == PF_SINGLE_PHASE) {
      const cd y = 1.0 / cd(c.br_r[e], c.br_x[e]);
      out[0] = y.real();
      out[1] = y.imag();
      sh[e] = c.br_b[e] / 2.0;
      continue;
    }
    int ph[3], k = 0;
    for (int s = 0; s < 3; ++s)
      if (c.br_phases[e] >> s & 1) ph[k++] = s;
    cd z[9], y[9];
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) {
        const double* zz = &c.br_z[(size_t)e * 18 + 2 * (3 * ph[a] + ph[b])];
        z[a * k + b] = cd(zz[0], zz[1]);
      }
    if (!invert_small(k, z, y)) {
      err = "a branch has a singular impedance matrix";
      return PF_ERR_INVALID;
    }
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) {
        out[2 * (3 * ph[a] + ph[b])] = y[a * k + b].real();
        out[2 * (3 * ph[a] + ph[b]) + 1] = y[a * k + b].imag();
      }
  }
  return PF_OK;
}

}  // namespace pf
