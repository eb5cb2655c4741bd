// Host-side network core: validation, bridges, minimum-degree ordering, sparse
// LDL^T of the reduced Laplacian and the FP64 PTDF at the generator buses.
//
// The PTDF is H = Omega E (E^T Omega E)^{-1} with E the reduced incidence matrix
// (Section 2, below problem (1)); H_a appends a zero slack column.  The hot path
// needs only Phi = H_a G (columns at generator buses), which is built here one
// generator bus at a time by sparse solves, and the normalised Phi~ = Phi diag(sigma)
// of Appendix A1.
#include <algorithm>
#include <cstring>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <queue>
#include <thread>

#include "internal.h"

namespace dcopf {

namespace {

bool finite(double v) { return std::isfinite(v); }

// Tarjan low-link bridges, iterative.
std::vector<uint8_t> find_bridges(int n_bus, const std::vector<int>& lf,
                                  const std::vector<int>& lt) {
  int nl = (int)lf.size();
  std::vector<std::vector<std::pair<int, int>>> adj(n_bus);
  for (int l = 0; l < nl; ++l) {
    adj[lf[l]].push_back({lt[l], l});
    adj[lt[l]].push_back({lf[l], l});
  }
  std::vector<int> disc(n_bus, -1), low(n_bus, 0);
  std::vector<uint8_t> br(nl, 0);
  int t = 0;
  struct Frame { int u, pl, it; };
  for (int r = 0; r < n_bus; ++r) {
    if (disc[r] >= 0) continue;
    disc[r] = low[r] = t++;
    std::vector<Frame> st{{r, -1, 0}};
    while (!st.empty()) {
      Frame& fr = st.back();
      if (fr.it < (int)adj[fr.u].size()) {
        auto [v, l] = adj[fr.u][fr.it++];
        if (l == fr.pl) continue;
        if (disc[v] < 0) {
          disc[v] = low[v] = t++;
          st.push_back({v, l, 0});
        } else {
          low[fr.u] = std::min(low[fr.u], disc[v]);
        }
      } else {
        Frame done = st.back();
        st.pop_back();
        if (!st.empty()) {
          int p = st.back().u;
          low[p] = std::min(low[p], low[done.u]);
          if (low[done.u] > disc[p]) br[done.pl] = 1;
        }
      }
    }
  }
  return br;
}

// Minimum-degree elimination on the explicit elimination graph.  Returns the order
// and, for each eliminated vertex, its neighbours at elimination time (the
// sparsity pattern of that column of L).
void min_degree(int n, std::vector<std::vector<int>> adj, std::vector<int>* order,
                std::vector<std::vector<int>>* colpat) {
  for (auto& a : adj) std::sort(a.begin(), a.end());
  std::vector<char> alive(n, 1);
  using E = std::pair<int, int>;
  std::priority_queue<E, std::vector<E>, std::greater<E>> pq;
  for (int i = 0; i < n; ++i) pq.push({(int)adj[i].size(), i});
  order->clear();
  colpat->assign(n, {});
  std::vector<int> tmp;
  while (!pq.empty()) {
    auto [d, v] = pq.top();
    pq.pop();
    if (!alive[v] || d != (int)adj[v].size()) continue;
    alive[v] = 0;
    order->push_back(v);
    std::vector<int> nb = adj[v];
    (*colpat)[v] = nb;
    for (int a : nb) {
      // adj[a] <- (adj[a] U nb) \ {a, v}
      tmp.clear();
      std::set_union(adj[a].begin(), adj[a].end(), nb.begin(), nb.end(), std::back_inserter(tmp));
      tmp.erase(std::remove_if(tmp.begin(), tmp.end(), [&](int x) { return x == a || x == v; }),
                tmp.end());
      adj[a].swap(tmp);
      pq.push({(int)adj[a].size(), a});
    }
  }
}

}  // namespace

void host_ldl_solve(const SparseFactor& F, double* x) {
  for (int i = 0; i < F.n; ++i) {
    double s = x[i];
    for (int p = F.lrow_ptr[i]; p < F.lrow_ptr[i + 1]; ++p) s -= F.lrow_val[p] * x[F.lrow_col[p]];
    x[i] = s;
  }
  for (int i = 0; i < F.n; ++i) x[i] /= F.diag[i];
  for (int i = F.n - 1; i >= 0; --i) {
    double s = x[i];
    for (int p = F.lcol_ptr[i]; p < F.lcol_ptr[i + 1]; ++p) s -= F.lcol_val[p] * x[F.lcol_row[p]];
    x[i] = s;
  }
}

dcopf_status build_host_net(const dcopf_network_desc* d, HostNet* H, std::string* err,
                            bool verbose, bool build_phi) {
  auto fail = [&](dcopf_status s, const std::string& m) {
    *err = m;
    return s;
  };
  if (!d) return fail(DCOPF_ERR_INVALID_ARG, "null network description");
  if (d->n_bus < 1 || d->n_line < 0 || d->n_gen < 1)
    return fail(DCOPF_ERR_INVALID_ARG, "n_bus and n_gen must be >= 1, n_line >= 0");
  if (d->n_bus > (1 << 24) || d->n_line > (1 << 26) || d->n_gen > (1 << 24))
    return fail(DCOPF_ERR_UNSUPPORTED, "network too large");
  if (d->n_line == 0)  // one bus: the dual has lambda only (merit order in closed form)
    return fail(DCOPF_ERR_UNSUPPORTED, "a network without lines has no flow constraints to dualise");
  if (d->slack_bus < 0 || d->slack_bus >= d->n_bus)
    return fail(DCOPF_ERR_INVALID_ARG, "slack_bus out of range");
  if ((d->n_line > 0 && (!d->line_from || !d->line_to || !d->line_b || !d->flow_max)) ||
      !d->gen_bus || !d->pmin || !d->pmax || !d->cost_lin)
    return fail(DCOPF_ERR_INVALID_ARG, "null array in network description");
  if (!(d->base_mva > 0) || !finite(d->base_mva))
    return fail(DCOPF_ERR_INVALID_ARG, "base_mva must be positive and finite");
  HostNet& h = *H;
  h.n_bus = d->n_bus;
  h.n_line = d->n_line;
  h.n_gen = d->n_gen;
  h.slack = d->slack_bus;
  h.S = d->base_mva;
  h.qp = d->cost_quad != nullptr;
  int nb = h.n_bus, nl = h.n_line, ng = h.n_gen;
  h.line_from.assign(d->line_from, d->line_from + nl);
  h.line_to.assign(d->line_to, d->line_to + nl);
  h.b.assign(d->line_b, d->line_b + nl);
  h.fmax.assign(d->flow_max, d->flow_max + nl);
  h.fmin.resize(nl);
  for (int l = 0; l < nl; ++l) h.fmin[l] = d->flow_min ? d->flow_min[l] : -d->flow_max[l];
  h.gen_bus.assign(d->gen_bus, d->gen_bus + ng);
  h.pmin.assign(d->pmin, d->pmin + ng);
  h.pmax.assign(d->pmax, d->pmax + ng);
  h.cost_lin.assign(d->cost_lin, d->cost_lin + ng);
  h.cost_quad.assign(ng, 0.0);
  if (h.qp) h.cost_quad.assign(d->cost_quad, d->cost_quad + ng);
  for (int l = 0; l < nl; ++l) {
    if (h.line_from[l] < 0 || h.line_from[l] >= nb || h.line_to[l] < 0 || h.line_to[l] >= nb)
      return fail(DCOPF_ERR_INVALID_ARG, "line endpoint out of range");
    if (h.line_from[l] == h.line_to[l]) return fail(DCOPF_ERR_NETWORK, "line is a self loop");
    if (!finite(h.b[l]) || !finite(h.fmax[l]) || !finite(h.fmin[l]))
      return fail(DCOPF_ERR_INVALID_ARG, "non-finite line data");
    if (!(h.b[l] > 0)) return fail(DCOPF_ERR_NETWORK, "line susceptance must be > 0");
    if (h.fmin[l] > h.fmax[l]) return fail(DCOPF_ERR_NETWORK, "flow_min > flow_max");
  }
  for (int j = 0; j < ng; ++j) {
    if (h.gen_bus[j] < 0 || h.gen_bus[j] >= nb)
      return fail(DCOPF_ERR_INVALID_ARG, "gen_bus out of range");
    if (!finite(h.pmin[j]) || !finite(h.pmax[j]) || !finite(h.cost_lin[j]) ||
        !finite(h.cost_quad[j]))
      return fail(DCOPF_ERR_INVALID_ARG, "non-finite generator data");
    if (h.pmin[j] > h.pmax[j]) return fail(DCOPF_ERR_NETWORK, "pmin > pmax");
    if (h.cost_quad[j] < 0) return fail(DCOPF_ERR_NETWORK, "cost_quad must be >= 0");
  }
  // connectivity (BFS from the slack)
  {
    std::vector<std::vector<int>> adj(nb);
    for (int l = 0; l < nl; ++l) {
      adj[h.line_from[l]].push_back(h.line_to[l]);
      adj[h.line_to[l]].push_back(h.line_from[l]);
    }
    std::vector<char> seen(nb, 0);
    std::vector<int> q{h.slack};
    seen[h.slack] = 1;
    for (size_t k = 0; k < q.size(); ++k)
      for (int v : adj[q[k]])
        if (!seen[v]) { seen[v] = 1; q.push_back(v); }
    if ((int)q.size() != nb) return fail(DCOPF_ERR_NETWORK, "network is islanded");
  }
  h.bridge = find_bridges(nb, h.line_from, h.line_to);

  // normalised generators (Appendix A1) and per-generator constants:
  // cost_j(mid + sigma x) = mq x^2 + ctil x + cconst
  double S = h.S;
  h.sigma.resize(ng); h.mid.resize(ng); h.ctil.resize(ng); h.mq.resize(ng); h.cconst.resize(ng);
  for (int j = 0; j < ng; ++j) {
    double s = 0.5 * (h.pmax[j] - h.pmin[j]), m = 0.5 * (h.pmax[j] + h.pmin[j]);
    double a = h.cost_quad[j], c = h.cost_lin[j];
    h.sigma[j] = s;
    h.mid[j] = m;
    h.ctil[j] = s * (c * S + 2.0 * a * S * S * m);
    h.mq[j] = a * S * S * s * s;
    h.cconst[j] = a * S * S * m * m + c * S * m;
  }
  // bus -> incident lines
  h.bus_line_ptr.assign(nb + 1, 0);
  for (int l = 0; l < nl; ++l) { h.bus_line_ptr[h.line_from[l] + 1]++; h.bus_line_ptr[h.line_to[l] + 1]++; }
  for (int i = 0; i < nb; ++i) h.bus_line_ptr[i + 1] += h.bus_line_ptr[i];
  h.bus_line_idx.resize(2 * nl);
  h.bus_line_coef.resize(2 * nl);
  {
    std::vector<int> fill(h.bus_line_ptr.begin(), h.bus_line_ptr.end() - 1);
    for (int l = 0; l < nl; ++l) {
      int p = fill[h.line_from[l]]++;
      h.bus_line_idx[p] = l; h.bus_line_coef[p] = h.b[l];
      p = fill[h.line_to[l]]++;
      h.bus_line_idx[p] = l; h.bus_line_coef[p] = -h.b[l];
    }
  }

  // bus -> generators (ascending index)
  h.bus_gen_ptr.assign(nb + 1, 0);
  for (int j = 0; j < ng; ++j) h.bus_gen_ptr[h.gen_bus[j] + 1]++;
  for (int i = 0; i < nb; ++i) h.bus_gen_ptr[i + 1] += h.bus_gen_ptr[i];
  h.bus_gen_idx.resize(ng);
  {
    std::vector<int> fill(h.bus_gen_ptr.begin(), h.bus_gen_ptr.end() - 1);
    for (int j = 0; j < ng; ++j) h.bus_gen_idx[fill[h.gen_bus[j]]++] = j;
  }

  // ---- reduced Laplacian, minimum-degree order, symbolic + numeric LDL^T
  SparseFactor& F = h.F;
  int n = nb - 1;
  F.n = n;
  std::vector<int> red(nb, -1), bus_of_red(n);
  for (int i = 0, k = 0; i < nb; ++i)
    if (i != h.slack) { red[i] = k; bus_of_red[k] = i; ++k; }
  std::vector<std::vector<int>> adj(n);
  std::vector<double> diagA(n, 0.0);
  // off-diagonal values of B_r keyed by (min,max) reduced index
  std::vector<std::vector<std::pair<int, double>>> offv(n);
  for (int l = 0; l < nl; ++l) {
    int u = red[h.line_from[l]], v = red[h.line_to[l]];
    if (u >= 0) diagA[u] += h.b[l];
    if (v >= 0) diagA[v] += h.b[l];
    if (u >= 0 && v >= 0) {
      adj[u].push_back(v);
      adj[v].push_back(u);
      offv[u].push_back({v, -h.b[l]});
      offv[v].push_back({u, -h.b[l]});
    }
  }
  for (auto& a : adj) { std::sort(a.begin(), a.end()); a.erase(std::unique(a.begin(), a.end()), a.end()); }
  std::vector<int> order;
  std::vector<std::vector<int>> colpat;
  min_degree(n, adj, &order, &colpat);
  std::vector<int> pos(n);
  for (int k = 0; k < n; ++k) pos[order[k]] = k;
  F.bus_of_pos.resize(n);
  F.pos_of_bus.assign(nb, -1);
  for (int k = 0; k < n; ++k) { F.bus_of_pos[k] = bus_of_red[order[k]]; F.pos_of_bus[bus_of_red[order[k]]] = k; }
  // column patterns in positions (all rows later than the column)
  std::vector<std::vector<int>> rows(n);
  for (int v = 0; v < n; ++v) {
    auto& r = rows[pos[v]];
    for (int a : colpat[v]) r.push_back(pos[a]);
    std::sort(r.begin(), r.end());
  }
  std::vector<std::vector<double>> vals(n);
  std::vector<double> dg(n);
  for (int k = 0; k < n; ++k) {
    vals[k].assign(rows[k].size(), 0.0);
    dg[k] = diagA[order[k]];
  }
  for (int v = 0; v < n; ++v) {
    int cv = pos[v];
    for (auto [u, val] : offv[v]) {
      int cu = pos[u];
      if (cu > cv) {  // entry (cu, cv) lives in column cv
        auto it = std::lower_bound(rows[cv].begin(), rows[cv].end(), cu);
        vals[cv][it - rows[cv].begin()] += val;
      }
    }
  }
  for (int k = 0; k < n; ++k) {
    double Dk = dg[k];
    if (!(Dk > 0) || !finite(Dk)) return fail(DCOPF_ERR_NETWORK, "Laplacian factorisation broke down");
    auto& rk = rows[k];
    auto& vk = vals[k];
    for (size_t a = 0; a < rk.size(); ++a) vk[a] /= Dk;  // now L_ik
    for (size_t a = 0; a < rk.size(); ++a) {
      int i = rk[a];
      double li = vk[a];
      dg[i] -= li * li * Dk;
      for (size_t c = 0; c < a; ++c) {
        int j = rk[c];  // j < i: update entry (i, j) in column j
        auto it = std::lower_bound(rows[j].begin(), rows[j].end(), i);
        vals[j][it - rows[j].begin()] -= li * Dk * vk[c];
      }
    }
  }
  F.diag = dg;
  // CSC of L (columns) and CSR of L (rows)
  F.lcol_ptr.assign(n + 1, 0);
  for (int k = 0; k < n; ++k) F.lcol_ptr[k + 1] = F.lcol_ptr[k] + (int)rows[k].size();
  F.lcol_row.resize(F.lcol_ptr[n]);
  F.lcol_val.resize(F.lcol_ptr[n]);
  F.lrow_ptr.assign(n + 1, 0);
  for (int k = 0; k < n; ++k) {
    std::copy(rows[k].begin(), rows[k].end(), F.lcol_row.begin() + F.lcol_ptr[k]);
    std::copy(vals[k].begin(), vals[k].end(), F.lcol_val.begin() + F.lcol_ptr[k]);
    for (int i : rows[k]) F.lrow_ptr[i + 1]++;
  }
  for (int i = 0; i < n; ++i) F.lrow_ptr[i + 1] += F.lrow_ptr[i];
  F.lrow_col.resize(F.lrow_ptr[n]);
  F.lrow_val.resize(F.lrow_ptr[n]);
  {
    std::vector<int> fill(F.lrow_ptr.begin(), F.lrow_ptr.end() - 1);
    for (int k = 0; k < n; ++k)
      for (size_t a = 0; a < rows[k].size(); ++a) {
        int p = fill[rows[k][a]]++;
        F.lrow_col[p] = k;
        F.lrow_val[p] = vals[k][a];
      }
  }
  // level schedules
  auto schedule = [&](bool fwd, std::vector<int>* lrows, std::vector<int>* lptr) {
    std::vector<int> lev(n, 0);
    int maxl = 0;
    if (fwd) {
      for (int i = 0; i < n; ++i) {
        int l = 0;
        for (int p = F.lrow_ptr[i]; p < F.lrow_ptr[i + 1]; ++p) l = std::max(l, lev[F.lrow_col[p]] + 1);
        lev[i] = l;
        maxl = std::max(maxl, l);
      }
    } else {
      for (int i = n - 1; i >= 0; --i) {
        int l = 0;
        for (int p = F.lcol_ptr[i]; p < F.lcol_ptr[i + 1]; ++p) l = std::max(l, lev[F.lcol_row[p]] + 1);
        lev[i] = l;
        maxl = std::max(maxl, l);
      }
    }
    int nlev = n > 0 ? maxl + 1 : 0;
    lptr->assign(nlev + 1, 0);
    for (int i = 0; i < n; ++i) (*lptr)[lev[i] + 1]++;
    for (int l = 0; l < nlev; ++l) (*lptr)[l + 1] += (*lptr)[l];
    lrows->resize(n);
    std::vector<int> fill(lptr->begin(), lptr->end() - 1);
    for (int i = 0; i < n; ++i) (*lrows)[fill[lev[i]]++] = i;
  };
  schedule(true, &F.fwd_rows, &F.fwd_level_ptr);
  schedule(false, &F.bwd_rows, &F.bwd_level_ptr);
  // ELL packing of the rows in schedule order (a row's entries load in one round trip)
  auto ell = [&](const std::vector<int>& order, const std::vector<int>& ptr, const std::vector<int>& idx_of,
                 const std::vector<double>& val, std::vector<int>* ecol, std::vector<double>* eval,
                 std::vector<int>* optr, std::vector<int>* ocol, std::vector<double>* oval) {
    const int K = SparseFactor::kEll;
    ecol->assign((size_t)K * n, 0);
    eval->assign((size_t)K * n, 0.0);
    optr->assign(n + 1, 0);
    ocol->clear();
    oval->clear();
    for (int q = 0; q < n; ++q) {
      const int i = order[q];
      for (int a = 0; a < K; ++a) (*ecol)[(size_t)a * n + q] = i;
      int a = 0;
      for (int p = ptr[i]; p < ptr[i + 1]; ++p, ++a) {
        if (a < K) {
          (*ecol)[(size_t)a * n + q] = idx_of[p];
          (*eval)[(size_t)a * n + q] = val[p];
        } else {
          ocol->push_back(idx_of[p]);
          oval->push_back(val[p]);
        }
      }
      (*optr)[q + 1] = (int)ocol->size();
    }
  };
  ell(F.fwd_rows, F.lrow_ptr, F.lrow_col, F.lrow_val, &F.fell_col, &F.fell_val, &F.fovf_ptr, &F.fovf_col,
      &F.fovf_val);
  ell(F.bwd_rows, F.lcol_ptr, F.lcol_row, F.lcol_val, &F.bell_col, &F.bell_val, &F.bovf_ptr, &F.bovf_col,
      &F.bovf_val);
  // packed factor for shared-memory staging: FP64 values stored once (CSR order),
  // the CSC walk reads them through a position map; indices in 16 bits
  if (n > 0 && n < 65535) {
    size_t nnz = F.lrow_col.size();
    size_t off = 0;
    auto sec = [&](size_t bytes) { size_t o = off; off = (off + bytes + 15) & ~(size_t)15; return (int)o; };
    F.off_diag = sec(8 * (size_t)n);
    F.off_val = sec(8 * nnz);
    F.off_rptr = sec(4 * (size_t)(n + 1));
    F.off_cptr = sec(4 * (size_t)(n + 1));
    F.off_cmap = sec(4 * nnz);
    F.off_rcol = sec(2 * nnz);
    F.off_crow = sec(2 * nnz);
    F.off_frows = sec(2 * (size_t)n);
    F.off_brows = sec(2 * (size_t)n);
    F.off_flev = sec(2 * F.fwd_level_ptr.size());
    F.off_blev = sec(2 * F.bwd_level_ptr.size());
    F.blob.assign(off, 0);
    unsigned char* B = F.blob.data();
    memcpy(B + F.off_diag, F.diag.data(), 8 * (size_t)n);
    memcpy(B + F.off_val, F.lrow_val.data(), 8 * nnz);
    for (int i = 0; i <= n; ++i) {
      ((uint32_t*)(B + F.off_rptr))[i] = (uint32_t)F.lrow_ptr[i];
      ((uint32_t*)(B + F.off_cptr))[i] = (uint32_t)F.lcol_ptr[i];
    }
    // position of each CSC entry in the CSR value array
    std::vector<int> fill(F.lrow_ptr.begin(), F.lrow_ptr.end() - 1);
    std::vector<uint32_t> cmap(nnz);
    for (int k = 0; k < n; ++k)
      for (int p = F.lcol_ptr[k]; p < F.lcol_ptr[k + 1]; ++p) {
        int i = F.lcol_row[p];
        // CSR row i lists its columns in increasing order, and columns k are visited in
        // increasing order here, so the next unused slot of row i is entry (i, k)
        cmap[p] = (uint32_t)fill[i]++;
      }
    memcpy(B + F.off_cmap, cmap.data(), 4 * nnz);
    for (size_t p = 0; p < nnz; ++p) {
      ((uint16_t*)(B + F.off_rcol))[p] = (uint16_t)F.lrow_col[p];
      ((uint16_t*)(B + F.off_crow))[p] = (uint16_t)F.lcol_row[p];
    }
    for (int i = 0; i < n; ++i) {
      ((uint16_t*)(B + F.off_frows))[i] = (uint16_t)F.fwd_rows[i];
      ((uint16_t*)(B + F.off_brows))[i] = (uint16_t)F.bwd_rows[i];
    }
    for (size_t l = 0; l < F.fwd_level_ptr.size(); ++l)
      ((uint16_t*)(B + F.off_flev))[l] = (uint16_t)F.fwd_level_ptr[l];
    for (size_t l = 0; l < F.bwd_level_ptr.size(); ++l)
      ((uint16_t*)(B + F.off_blev))[l] = (uint16_t)F.bwd_level_ptr[l];
  }

  // ---- Phi~ = H_a G diag(sigma), built one generator bus at a time (FP64); skipped
  // for a sparse-only handle
  if (build_phi) h.phi.assign((size_t)nl * ng, 0.0);
  std::vector<int> gens_order(ng);
  std::iota(gens_order.begin(), gens_order.end(), 0);
  unsigned nthreads = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if ((int64_t)ng * (F.nnz() + n) < 2000000) nthreads = 1;
  auto worker = [&](int t) {
    std::vector<double> x(n);
    for (int j = t; j < ng; j += (int)nthreads) {
      int bus = h.gen_bus[j];
      if (bus == h.slack || n == 0) continue;  // zero column of H_a
      std::fill(x.begin(), x.end(), 0.0);
      x[F.pos_of_bus[bus]] = 1.0;
      host_ldl_solve(F, x.data());
      for (int l = 0; l < nl; ++l) {
        int pf = F.pos_of_bus[h.line_from[l]], pt = F.pos_of_bus[h.line_to[l]];
        double th_f = pf >= 0 ? x[pf] : 0.0, th_t = pt >= 0 ? x[pt] : 0.0;
        h.phi[(size_t)l * ng + j] = h.b[l] * (th_f - th_t) * h.sigma[j];
      }
    }
  };
  if (build_phi) {
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nthreads; ++t) th.emplace_back(worker, (int)t);
    worker(0);
    for (auto& t : th) t.join();
  }
  // Phi mid = Phi~ diag(1/sigma) mid, computed from the unscaled columns
  h.phim.assign(nl, 0.0);
  {
    std::vector<double> inj(n, 0.0);
    for (int j = 0; j < ng; ++j) {
      int p = F.pos_of_bus[h.gen_bus[j]];
      if (p >= 0) inj[p] += h.mid[j];
    }
    if (n > 0) host_ldl_solve(F, inj.data());
    for (int l = 0; l < nl; ++l) {
      int pf = F.pos_of_bus[h.line_from[l]], pt = F.pos_of_bus[h.line_to[l]];
      h.phim[l] = h.b[l] * ((pf >= 0 ? inj[pf] : 0.0) - (pt >= 0 ? inj[pt] : 0.0));
    }
  }
  if (verbose)
    fprintf(stderr, "[dcopf] n_bus=%d n_line=%d n_gen=%d nnz(L)=%lld levels fwd=%zu bwd=%zu bridges=%d\n",
            nb, nl, ng, (long long)F.nnz(), F.fwd_level_ptr.size() - 1, F.bwd_level_ptr.size() - 1,
            (int)std::count(h.bridge.begin(), h.bridge.end(), 1));
  return DCOPF_OK;
}

}  // namespace dcopf
