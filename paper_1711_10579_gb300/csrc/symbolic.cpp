// Symbolic analysis of the block Newton system, computed once per topology.
//
// The Jacobian of Eq. 10 (grouped per bus into 2x2 blocks) and of Eq. 22
// (6x6 blocks per node) has the block pattern of Ybus.  The direct solver of
// Sec. III.A permutes the matrix with an approximate-minimum-degree ordering
// to limit fill; here a minimum-degree ordering of the bus graph is computed
// by explicit elimination, which yields the fill pattern of the LU factors at
// the same time.  The Krylov solver of Sec. III.B permutes the matrix to keep
// nonzeros near the diagonal; reverse Cuthill-McKee does that.
//
// From the pattern the analysis derives, for the GPU:
//  * level sets of the factorisation / forward solve (a row depends on the
//    rows of its L part) and of the backward solve (U part);
//  * a fan-out (right-looking) schedule of the numeric factorisation: at
//    level l every pivot of the level and every L entry of its column is
//    finalised in parallel, then every entry those pivots update gathers its
//    updates in parallel, so no row is walked sequentially and the critical
//    path is two parallel steps per level.
#include <algorithm>
#include <cstdint>
#include <deque>
#include <set>
#include <utility>

#include "host.h"

namespace pf {

namespace {

// Bus graph without self loops (adjacency sorted).
std::vector<std::vector<int>> bus_graph(const Ybus& y) {
  std::vector<std::vector<int>> adj(y.n);
  for (int i = 0; i < y.n; ++i)
    for (int p = y.rowptr[i]; p < y.rowptr[i + 1]; ++p)
      if (y.col[p] != i) adj[i].push_back(y.col[p]);
  return adj;
}

// Minimum-degree ordering by explicit elimination on the bus graph.  When a
// vertex is eliminated its remaining neighbours become a clique; the
// neighbour set at that moment is the structure of its column of L.  Ties go
// to the smallest vertex id, so the ordering is deterministic.
void min_degree(std::vector<std::vector<int>> adj, std::vector<int>& perm,
                std::vector<std::vector<int>>& lstruct) {
  const int n = (int)adj.size();
  std::set<std::pair<int, int>> queue;
  for (int v = 0; v < n; ++v) queue.insert({(int)adj[v].size(), v});
  perm.clear();
  lstruct.assign(n, {});
  std::vector<int> merged;
  while (!queue.empty()) {
    int v = queue.begin()->second;
    queue.erase(queue.begin());
    perm.push_back(v);
    std::vector<int> nb;
    nb.swap(adj[v]);
    for (int u : nb) {
      queue.erase({(int)adj[u].size(), u});
      // adj[u] := (adj[u] U nb) \ {u, v}
      merged.clear();
      std::set_union(adj[u].begin(), adj[u].end(), nb.begin(), nb.end(),
                     std::back_inserter(merged));
      auto& a = adj[u];
      a.clear();
      for (int w : merged)
        if (w != u && w != v) a.push_back(w);
      queue.insert({(int)a.size(), u});
    }
    lstruct[v] = std::move(nb);
  }
}

// Reverse Cuthill-McKee: breadth-first search from a pseudo-peripheral
// vertex, visiting neighbours by increasing degree, then reversed.
void rcm(const std::vector<std::vector<int>>& adj, std::vector<int>& perm) {
  const int n = (int)adj.size();
  std::vector<char> seen(n, 0);
  perm.clear();
  auto bfs_last = [&](int s, std::vector<int>& dist) {
    dist.assign(n, -1);
    std::deque<int> q{s};
    dist[s] = 0;
    int last = s;
    while (!q.empty()) {
      int v = q.front();
      q.pop_front();
      last = v;
      for (int u : adj[v])
        if (dist[u] < 0) {
          dist[u] = dist[v] + 1;
          q.push_back(u);
        }
    }
    return last;
  };
  std::vector<int> dist;
  for (int start = 0; start < n; ++start) {
    if (seen[start]) continue;
    // pseudo-peripheral vertex: repeat BFS from the farthest vertex
    int s = start, ecc = -1;
    for (int it = 0; it < 4; ++it) {
      int far = bfs_last(s, dist);
      if (dist[far] <= ecc) break;
      ecc = dist[far];
      s = far;
    }
    std::deque<int> q{s};
    seen[s] = 1;
    while (!q.empty()) {
      int v = q.front();
      q.pop_front();
      perm.push_back(v);
      std::vector<int> nb;
      for (int u : adj[v])
        if (!seen[u]) nb.push_back(u);
      std::sort(nb.begin(), nb.end(), [&](int a, int b) {
        return adj[a].size() != adj[b].size() ? adj[a].size() < adj[b].size()
                                              : a < b;
      });
      for (int u : nb) {
        seen[u] = 1;
        q.push_back(u);
      }
    }
  }
  std::reverse(perm.begin(), perm.end());
}

void build_levels(int n, const std::vector<int>& level, std::vector<int>& ptr,
                  std::vector<int>& rows) {
  int nl = 0;
  for (int v : level) nl = std::max(nl, v + 1);
  ptr.assign(nl + 1, 0);
  for (int v : level) ++ptr[v + 1];
  for (int l = 0; l < nl; ++l) ptr[l + 1] += ptr[l];
  rows.assign(n, 0);
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (int i = 0; i < n; ++i) rows[fill[level[i]]++] = i;
}

}  // namespace

void analyze(const Ybus& y, Ordering ord, bool with_fill, Symbolic& s) {
  const int n = y.n;
  s.n = n;
  auto adj = bus_graph(y);
  std::vector<std::vector<int>> lstruct;  // old ids; only with MinDegree
  if (ord == Ordering::MinDegree) {
    min_degree(adj, s.perm, lstruct);
  } else if (ord == Ordering::RCM) {
    rcm(adj, s.perm);
  } else {
    s.perm.resize(n);
    for (int i = 0; i < n; ++i) s.perm[i] = i;
  }
  s.iperm.assign(n, 0);
  for (int k = 0; k < n; ++k) s.iperm[s.perm[k]] = k;

  // Ybus pattern in the new numbering
  s.y_rowptr.assign(n + 1, 0);
  s.y_col.clear();
  s.y_src.clear();
  std::vector<std::pair<int, int>> row;
  for (int i = 0; i < n; ++i) {
    int o = s.perm[i];
    row.clear();
    for (int p = y.rowptr[o]; p < y.rowptr[o + 1]; ++p)
      row.push_back({s.iperm[y.col[p]], p});
    std::sort(row.begin(), row.end());
    for (auto& e : row) {
      s.y_col.push_back(e.first);
      s.y_src.push_back(e.second);
    }
    s.y_rowptr[i + 1] = (int)s.y_col.size();
  }

  // factor pattern (new numbering): strict upper part of row k = column
  // structure of L below k (symmetric pattern)
  std::vector<std::vector<int>> upper(n), lower(n);
  if (with_fill) {
    if (lstruct.empty()) {
      // symbolic elimination in the given order
      std::vector<std::vector<int>> g(n);
      for (int i = 0; i < n; ++i)
        for (int p = s.y_rowptr[i]; p < s.y_rowptr[i + 1]; ++p)
          if (s.y_col[p] > i) g[i].push_back(s.y_col[p]);
      for (int k = 0; k < n; ++k) {
        auto& st = g[k];
        std::sort(st.begin(), st.end());
        st.erase(std::unique(st.begin(), st.end()), st.end());
        if (!st.empty()) {
          int par = st[0];
          for (size_t t = 1; t < st.size(); ++t) g[par].push_back(st[t]);
        }
        upper[k] = st;
      }
    } else {
      for (int v = 0; v < n; ++v) {
        int k = s.iperm[v];
        for (int u : lstruct[v]) upper[k].push_back(s.iperm[u]);
        std::sort(upper[k].begin(), upper[k].end());
      }
    }
  } else {
    for (int i = 0; i < n; ++i)
      for (int p = s.y_rowptr[i]; p < s.y_rowptr[i + 1]; ++p)
        if (s.y_col[p] > i) upper[i].push_back(s.y_col[p]);
  }
  for (int k = 0; k < n; ++k)
    for (int i : upper[k]) lower[i].push_back(k);  // k increasing => sorted

  s.lu_rowptr.assign(n + 1, 0);
  s.lu_col.clear();
  s.lu_diag.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    for (int k : lower[i]) s.lu_col.push_back(k);
    s.lu_diag[i] = (int)s.lu_col.size();
    s.lu_col.push_back(i);
    for (int j : upper[i]) s.lu_col.push_back(j);
    s.lu_rowptr[i + 1] = (int)s.lu_col.size();
  }
  const int nnz = (int)s.lu_col.size();

  // factor entry -> Ybus entry (new numbering), -1 for fill
  s.lu2y.assign(nnz, -1);
  for (int i = 0; i < n; ++i) {
    int p = s.y_rowptr[i], pe = s.y_rowptr[i + 1];
    for (int q = s.lu_rowptr[i]; q < s.lu_rowptr[i + 1]; ++q) {
      while (p < pe && s.y_col[p] < s.lu_col[q]) ++p;
      if (p < pe && s.y_col[p] == s.lu_col[q]) s.lu2y[q] = p;
    }
  }

  // level sets
  std::vector<int> flev(n, 0), blev(n, 0);
  for (int i = 0; i < n; ++i) {
    int l = 0;
    for (int p = s.lu_rowptr[i]; p < s.lu_diag[i]; ++p)
      l = std::max(l, flev[s.lu_col[p]] + 1);
    flev[i] = l;
  }
  for (int i = n - 1; i >= 0; --i) {
    int l = 0;
    for (int q = s.lu_diag[i] + 1; q < s.lu_rowptr[i + 1]; ++q)
      l = std::max(l, blev[s.lu_col[q]] + 1);
    blev[i] = l;
  }
  build_levels(n, flev, s.flev_ptr, s.flev_rows);
  build_levels(n, blev, s.blev_ptr, s.blev_rows);
  const int nf = (int)s.flev_ptr.size() - 1, nb = (int)s.blev_ptr.size() - 1;
  s.flev_llen.assign(nf, 0);
  s.blev_ulen.assign(nb, 0);
  for (int l = 0; l < nf; ++l)
    for (int t = s.flev_ptr[l]; t < s.flev_ptr[l + 1]; ++t) {
      int i = s.flev_rows[t];
      s.flev_llen[l] = std::max(s.flev_llen[l], s.lu_diag[i] - s.lu_rowptr[i]);
    }
  for (int l = 0; l < nb; ++l)
    for (int t = s.blev_ptr[l]; t < s.blev_ptr[l + 1]; ++t) {
      int i = s.blev_rows[t];
      s.blev_ulen[l] = std::max(s.blev_ulen[l], s.lu_rowptr[i + 1] - s.lu_diag[i] - 1);
    }

  // fan-out schedule: L entries by column, then per level the finalised
  // entries and the gathered updates
  std::vector<int> rowof(nnz);
  std::vector<std::vector<int>> colL(n);
  for (int i = 0; i < n; ++i)
    for (int p = s.lu_rowptr[i]; p < s.lu_rowptr[i + 1]; ++p) {
      rowof[p] = i;
      if (p < s.lu_diag[i]) colL[s.lu_col[p]].push_back(p);
    }
  auto find = [&](int i, int j) {
    const int* b = s.lu_col.data() + s.lu_rowptr[i];
    const int* e = s.lu_col.data() + s.lu_rowptr[i + 1];
    const int* q = std::lower_bound(b, e, j);
    return (q != e && *q == j) ? (int)(q - s.lu_col.data()) : -1;
  };
  s.fac_ptr.assign(nf + 1, 0);
  s.tgt_ptr.assign(nf + 1, 0);
  s.fac_items.clear();
  s.tgt_entry.clear();
  s.tgt_cptr.assign(1, 0);
  s.con_l.clear();
  s.con_u.clear();
  s.n_updates = 0;
  struct Tri { int t, k, p, q; };
  std::vector<Tri> tri;
  for (int l = 0; l < nf; ++l) {
    tri.clear();
    for (int r = s.flev_ptr[l]; r < s.flev_ptr[l + 1]; ++r) {
      const int k = s.flev_rows[r];
      s.fac_items.push_back(s.lu_diag[k]);
      for (int p : colL[k]) {
        s.fac_items.push_back(p);
        const int i = rowof[p];
        for (int q = s.lu_diag[k] + 1; q < s.lu_rowptr[k + 1]; ++q) {
          const int t = find(i, s.lu_col[q]);
          if (t >= 0) tri.push_back({t, k, p, q});
        }
      }
    }
    std::sort(tri.begin(), tri.end(), [](const Tri& a, const Tri& b) {
      return a.t != b.t ? a.t < b.t : a.k < b.k;
    });
    for (size_t u = 0; u < tri.size(); ++u) {
      if (u == 0 || tri[u].t != tri[u - 1].t) {
        if (u > 0) s.tgt_cptr.push_back((int)s.con_l.size());
        s.tgt_entry.push_back(tri[u].t);
      }
      s.con_l.push_back(tri[u].p);
      s.con_u.push_back(tri[u].q);
    }
    if (!tri.empty()) s.tgt_cptr.push_back((int)s.con_l.size());
    s.n_updates += (long long)tri.size();
    s.fac_ptr[l + 1] = (int)s.fac_items.size();
    s.tgt_ptr[l + 1] = (int)s.tgt_entry.size();
  }
}

std::vector<int8_t> lanes_per_level(const std::vector<int>& lev_ptr,
                                    const std::vector<int>& longest,
                                    int threads, int cap) {
  const int nl = (int)lev_ptr.size() - 1;
  std::vector<int8_t> g(nl, 1);
  for (int l = 0; l < nl; ++l) {
    int width = lev_ptr[l + 1] - lev_ptr[l];
    int want = 1;
    while (want < cap && want < longest[l]) want <<= 1;
    // keep every row of the level in flight at once when possible
    while (want > 1 && (long long)want * width > threads) want >>= 1;
    g[l] = (int8_t)want;
  }
  return g;
}

}  // namespace pf
