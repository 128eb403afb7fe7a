// Host-side data structures of the power-flow library: the admittance
// matrix, the symbolic analysis of the Newton system and the level schedules.
// Everything here is plain C++ (no CUDA) so it can be built and exercised on
// a machine without a GPU.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pf.h"

namespace pf {

// Ybus in the caller's numbering as block CSR with sorted columns and every
// diagonal block present.  ybs = 1: complex scalars (single phase, Eq. 2-3);
// ybs = 3: 3x3 complex blocks (three phase, Eq. 11).  val holds 2*ybs*ybs
// doubles per entry, (re, im) interleaved, blocks row-major.
struct Ybus {
  int n = 0;
  int ybs = 1;
  std::vector<int> rowptr, col;
  std::vector<double> val;
  int nnz() const { return (int)col.size(); }
};

// Validated, copied case description (caller's numbering).
struct CaseData {
  int kind = PF_SINGLE_PHASE;
  int n = 0, m = 0;
  // single phase, per bus
  std::vector<int8_t> bus_type;
  std::vector<double> v_set, p_gen, q_gen, p_load, q_load, zip;  // zip: n*3
  std::vector<double> q_min, q_max;  // optional reactive limits (empty = none)
  // three phase: per node / per slot
  std::vector<uint8_t> phases;
  int source = 0;
  double v_source = 1.0;
  std::vector<double> p_load3, q_load3;  // 3n
  std::vector<double> p_gen3;            // 3n: generation of PV nodes (bus_type, v_set)
  // branches
  std::vector<int> br_from, br_to;
  std::vector<double> br_r, br_x, br_b;
  std::vector<uint8_t> br_phases;
  std::vector<double> br_z;  // m*18
};

// Copies and validates; returns PF_OK or PF_ERR_INVALID with a message.
int copy_case(const pf_case_desc* d, CaseData& out, std::string& err);
// Eq. 2-3 (pi-model branches) or Eq. 11 (3x3 blocks).
int build_ybus(const CaseData& c, Ybus& y, std::string& err);
// Per-branch admittances of the same models (for branch flows): yb[m][18] as
// 3x3 complex row-major, sh[m] the half line charging (single phase).
int branch_admittances(const CaseData& c, std::vector<double>& yb, std::vector<double>& sh,
                       std::string& err);

// Ordering of the bus graph.
enum class Ordering { MinDegree, RCM, Natural };

// Symbolic analysis of the block Newton system for one ordering.  All
// indices are in the new (permuted) numbering.
struct Symbolic {
  int n = 0;
  std::vector<int> perm, iperm;  // perm[new] = old, iperm[old] = new
  // Ybus pattern in the new numbering; y_src[e] = entry of the caller's CSR
  std::vector<int> y_rowptr, y_col, y_src;
  // block pattern of the factor (L strictly lower, diagonal, U strictly
  // upper) -- with fill for LU, equal to the Ybus pattern for ILU(0)
  std::vector<int> lu_rowptr, lu_col, lu_diag;
  std::vector<int> lu2y;  // factor entry -> new-order Ybus entry or -1 (fill)
  // fan-out factorisation schedule, per level l of the factor's level sets:
  //  fac_items[fac_ptr[l] .. fac_ptr[l+1]) are the factor entries finalised
  //    at level l: the diagonal block of each pivot k of the level and every
  //    L entry (i, k) of those pivot columns;
  //  targets t in [tgt_ptr[l], tgt_ptr[l+1]) are the entries tgt_entry[t]
  //    that the level's pivots update, A_t -= sum of L(con_l[c]) U(con_u[c])
  //    over c in [tgt_cptr[t], tgt_cptr[t+1]) (con_l an L entry (i, k),
  //    con_u a U entry (k, j) of a pivot k of the level).  ILU(0) drops the
  //    updates whose target is not in the pattern.
  std::vector<int> fac_ptr, fac_items, tgt_ptr, tgt_entry, tgt_cptr, con_l, con_u;
  long long n_updates = 0;
  // level sets: rows of level l are flev_rows[flev_ptr[l] .. flev_ptr[l+1])
  std::vector<int> flev_ptr, flev_rows;  // factor / forward solve (L deps)
  std::vector<int> blev_ptr, blev_rows;  // backward solve (U deps)
  // per level: the longest parallel inner loop (for choosing lanes per row)
  std::vector<int> flev_llen;  // forward: longest L part of a row
  std::vector<int> blev_ulen;  // backward: longest U part of a row
  int nnz_lu() const { return (int)lu_col.size(); }
  int nnz_y() const { return (int)y_col.size(); }
};

// Computes the ordering and, for MinDegree, the fill of the exact LU
// factorisation (with_fill = true) or the ILU(0) pattern (with_fill = false).
void analyze(const Ybus& y, Ordering ord, bool with_fill, Symbolic& s);

// Lanes per row (1, 2, 4, ..., cap, cap a power of two <= 64) for each level
// of a schedule, given the longest inner loop per level, the level widths and
// the threads (row slots) available.
std::vector<int8_t> lanes_per_level(const std::vector<int>& lev_ptr,
                                    const std::vector<int>& longest,
                                    int threads, int cap = 32);

}  // namespace pf
