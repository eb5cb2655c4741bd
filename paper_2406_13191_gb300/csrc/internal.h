// Internal declarations shared by the host setup code and the CUDA translation units.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "dcopf_dual.h"

namespace dcopf {

// Sparse LDL^T factor of the reduced Laplacian B_r = E^T Omega E (slack removed),
// in a minimum-degree elimination order.  Row/column indices are elimination
// positions 0..n-1.
struct SparseFactor {
  int n = 0;
  std::vector<int> bus_of_pos;  // position -> bus
  std::vector<int> pos_of_bus;  // bus -> position, -1 for the slack bus
  // strictly lower L, unit diagonal, by rows (row i holds columns k < i)
  std::vector<int> lrow_ptr, lrow_col;
  std::vector<double> lrow_val;
  // strictly lower L by columns (column k holds rows i > k) = rows of L^T
  std::vector<int> lcol_ptr, lcol_row;
  std::vector<double> lcol_val;
  std::vector<double> diag;
  // level schedules: rows listed level by level
  std::vector<int> fwd_rows, fwd_level_ptr;
  std::vector<int> bwd_rows, bwd_level_ptr;
  // The same rows in schedule order, ELL-packed: for the row at schedule position idx,
  // its first kEll entries at [a * n + idx] (a < kEll; unused slots the row itself with
  // value 0), the rest in a schedule-ordered CSR overflow (ptr [n + 1]).  Entries keep
  // the CSR (forward) / CSC (backward) order, so sums are the same as the plain walk's.
  static constexpr int kEll = 4;
  std::vector<int> fell_col, bell_col, fovf_ptr, fovf_col, bovf_ptr, bovf_col;
  std::vector<double> fell_val, bell_val, fovf_val, bovf_val;
  int64_t nnz() const { return (int64_t)lrow_col.size(); }
  // Packed copy for shared-memory staging (empty when indices do not fit 16 bits):
  // 16-byte aligned sections at the byte offsets below.
  std::vector<unsigned char> blob;
  int off_diag = 0, off_val = 0, off_rptr = 0, off_cptr = 0, off_rcol = 0, off_crow = 0,
      off_cmap = 0, off_frows = 0, off_brows = 0, off_flev = 0, off_blev = 0;
};

// Validated copy of the network plus everything derived from it on the host.
struct HostNet {
  int n_bus = 0, n_line = 0, n_gen = 0, slack = 0;
  bool qp = false;
  double S = 100.0;
  std::vector<int> line_from, line_to, gen_bus;
  std::vector<double> b, fmax, fmin, pmin, pmax, cost_lin, cost_quad;
  std::vector<uint8_t> bridge;
  // normalised generator data (Appendix A1): p = mid + sigma x, x in [-1, 1]
  std::vector<double> sigma, mid, ctil, mq, cconst;
  // bus -> incident lines (+1 from-bus, -1 to-bus), for E^T Omega eta
  std::vector<int> bus_line_ptr, bus_line_idx;
  // bus -> generators at it (ascending generator index), for sparse injections
  std::vector<int> bus_gen_ptr, bus_gen_idx;
  std::vector<double> bus_line_coef;  // +b_l or -b_l
  SparseFactor F;
  std::vector<double> phi;  // Phi~ = Phi diag(sigma), row-major [n_line][n_gen]
  std::vector<double> phim; // Phi mid, [n_line] (flows of the mid-box dispatch)
};

// Builds a HostNet from the C description (validation, ordering, factorisation,
// PTDF build).  Returns DCOPF_OK or an error with a message in *err.
dcopf_status build_host_net(const dcopf_network_desc* d, HostNet* out, std::string* err,
                            bool verbose, bool build_phi = true);

// Solves B_r theta = rhs in place (rhs indexed by elimination position).
void host_ldl_solve(const SparseFactor& F, double* x);

}  // namespace dcopf
