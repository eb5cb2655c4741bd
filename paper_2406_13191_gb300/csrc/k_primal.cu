// Primal recovery: a feasible dispatch, and so an upper bound on gamma*, from a dual
// point.  The paper has no primal step.  Its Remarks 1-2 (Section 3) give the fact
// used here: every feasible dispatch costs at least every dual value, so the pair
// (certified lower bound, cost of a feasible dispatch) brackets gamma* without a
// stored optimum.
//
// One CTA per instance, FP64 throughout (normalised generators, Appendix A1:
// p = mid + sigma x, |x| <= 1):
//   k_primal_balance  (or, from a caller's candidate, its box clip moved towards a box
//                     corner until it meets the demand)
//                     w_j = ctil_j + sigma_j lambda + pi~_j from the FP64 adjoint; the
//                     closed-form minimiser x_j(w_j + sigma_j delta) for a uniform price
//                     shift delta (eq. (6) / eq. (16)); bisection on delta until the
//                     total dispatch brackets the demand between two adjacent shifts,
//                     then the convex combination of the two bracketing dispatches that
//                     meets it exactly.  Also the reference dispatch (the caller's,
//                     checked against the box and the balance, or the proportional one).
//   k_forward<double> flows of both (Phi~ in FP64, base flows f0)
//   k_primal_repair   outage correction, the reference's feasibility, and the smallest
//                     t in [0, 1] with (1 - t) x_bal + t x_ref inside every flow limit
//                     (the feasible set is convex)
//   k_forward<double> flows of the repaired dispatch, recomputed
//   k_primal_finish   largest violation (rounding only), cost (the upper bound),
//                     dispatch in p.u.
#include "dev.cuh"
#include "kernels.h"

namespace dcopf {

namespace {

constexpr double kTol = 1e-9;  // p.u.: reference box / balance / limits

__device__ __forceinline__ double reduced_cost(const DevNet& N, int j, double lam, double pi) {
  return N.ctil[j] + N.sigma[j] * lam + pi;
}

}  // namespace

__global__ void k_primal_balance(DevNet N, const double* __restrict__ lambda,
                                 const double* __restrict__ pit, const double* __restrict__ demand,
                                 const double* __restrict__ p_cand,
                                 const double* __restrict__ p_ref, double* __restrict__ xb,
                                 double* __restrict__ xr, int* __restrict__ pst) {
  __shared__ double red[32];
  const int b = blockIdx.x, ng = N.n_gen, tid = threadIdx.x, nt = blockDim.x;
  const double D = demand[b];
  double* xbb = xb + (size_t)b * ng;
  double* xrb = xr + (size_t)b * ng;
  double smin = 0.0, smax = 0.0;  // box totals
  for (int j = tid; j < ng; j += nt) {
    smin += N.mid[j] - N.sigma[j];
    smax += N.mid[j] + N.sigma[j];
  }
  smin = block_sum(smin, red);
  smax = block_sum(smax, red);
  if (D > smax || D < smin) {  // no dispatch in the box meets the demand
    for (int j = tid; j < ng; j += nt) { xbb[j] = 0.0; xrb[j] = 0.0; }
    if (tid == 0) pst[b] = 1;
    return;
  }
  if (p_cand) {
    // the caller's candidate, clipped to the box, moved towards pmax (total below the
    // demand) or pmin (above) until it meets the demand
    const double* pc = p_cand + (size_t)b * ng;
    double tot = 0.0;
    for (int j = tid; j < ng; j += nt) {
      const double m = N.mid[j], sg = N.sigma[j];
      tot += fmin(m + sg, fmax(m - sg, pc[j]));
    }
    tot = block_sum(tot, red);
    const bool up = tot < D;
    const double room = up ? smax - tot : tot - smin;
    const double phi = room > 0.0 ? fmin(1.0, (up ? D - tot : tot - D) / room) : 0.0;
    for (int j = tid; j < ng; j += nt) {
      const double m = N.mid[j], sg = N.sigma[j];
      double p = fmin(m + sg, fmax(m - sg, pc[j]));
      p = up ? p + phi * (m + sg - p) : p - phi * (p - (m - sg));
      xbb[j] = sg > 0.0 ? (p - m) / sg : 0.0;
    }
  } else {
    const double lam = lambda[b];
    const double* pi = pit + (size_t)b * ng;
    // the shifts beyond which every unit sits at pmax (below lo) or at pmin (above hi)
    double dlo = INFINITY, dhi = -INFINITY;
    for (int j = tid; j < ng; j += nt) {
      const double s = N.sigma[j];
      if (s > 0.0) {
        const double w = reduced_cost(N, j, lam, pi[j]);
        dlo = fmin(dlo, (-2.0 * N.mq[j] - w) / s);
        dhi = fmax(dhi, (2.0 * N.mq[j] - w) / s);
      }
    }
    dlo = -block_max(-dlo, red);
    dhi = block_max(dhi, red);
    auto x_at = [&](int j, double delta) {
      const double s = N.sigma[j];
      return s > 0.0 ? inner_x<double>(reduced_cost(N, j, lam, pi[j]) + s * delta, N.mq[j]) : 0.0;
    };
    auto total = [&](double delta) {
      double acc = 0.0;
      for (int j = tid; j < ng; j += nt) acc += N.mid[j] + N.sigma[j] * x_at(j, delta);
      return block_sum(acc, red);
    };
    double lo = 0.0, hi = 0.0;
    if (dlo <= dhi) {
      lo = dlo - 1.0;
      hi = dhi + 1.0;
      // total(lo) >= D >= total(hi) throughout; every thread takes the same branch
      for (int it = 0; it < 2000; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (total(mid) >= D) lo = mid;
        else hi = mid;
      }
    }
    const double P_lo = total(lo), P_hi = total(hi);
    double phi = P_lo > P_hi ? (D - P_hi) / (P_lo - P_hi) : 0.0;
    phi = fmin(1.0, fmax(0.0, phi));
    for (int j = tid; j < ng; j += nt) {
      const double x_lo = x_at(j, lo), x_hi = x_at(j, hi);
      xbb[j] = x_hi + phi * (x_lo - x_hi);
    }
  }
  // reference dispatch
  int bad = 0;
  if (p_ref) {
    const double* pr = p_ref + (size_t)b * ng;
    double s = 0.0;
    for (int j = tid; j < ng; j += nt) {
      const double p = pr[j], m = N.mid[j], sg = N.sigma[j];
      s += p;
      bad |= !(fabs(p - m) <= sg + kTol);  // outside the box (or NaN)
      xrb[j] = sg > 0.0 ? (p - m) / sg : 0.0;
    }
    s = block_sum(s, red);
    bad = __syncthreads_or(bad);
    if (!(fabs(s - D) <= kTol * fmax(1.0, D))) bad = 1;
  } else {
    // proportional: pmin + theta (pmax - pmin), i.e. x = 2 theta - 1
    const double theta = smax > smin ? (D - smin) / (smax - smin) : 0.0;
    for (int j = tid; j < ng; j += nt) xrb[j] = N.sigma[j] > 0.0 ? 2.0 * theta - 1.0 : 0.0;
  }
  if (tid == 0) pst[b] = bad ? 2 : 0;
}

// Outage correction of both flow sets (f' = f + u f_k, line k without limits), the
// reference's feasibility and the repair weight t; x_ub = (1 - t) x_bal + t x_ref.
__global__ void k_primal_repair(DevNet N, const int* __restrict__ outage, const double* __restrict__ u,
                                const double* __restrict__ fb, const double* __restrict__ fr,
                                const double* __restrict__ xb, const double* __restrict__ xr,
                                int* __restrict__ pst, double* __restrict__ tout,
                                double* __restrict__ xu) {
  __shared__ double red[32];
  const int b = blockIdx.x, nl = N.n_line, ng = N.n_gen, tid = threadIdx.x, nt = blockDim.x;
  const int st = pst[b];
  double* xub = xu + (size_t)b * ng;
  if (st != 0) {
    for (int j = tid; j < ng; j += nt) xub[j] = 0.0;
    if (tid == 0) tout[b] = NAN;
    return;
  }
  const int k = outage ? outage[b] : -1;
  const double* fbb = fb + (size_t)b * nl;
  const double* frb = fr + (size_t)b * nl;
  const double fbk = k >= 0 ? fbb[k] : 0.0, frk = k >= 0 ? frb[k] : 0.0;
  double vref = 0.0, t = 0.0;
  for (int i = tid; i < nl; i += nt) {
    if (i == k) continue;
    const double ui = k >= 0 ? u[(size_t)b * nl + i] : 0.0;
    const double f_b = fbb[i] + ui * fbk, f_r = frb[i] + ui * frk;
    const double hi = N.fmax[i], lo = N.fmin[i];
    vref = fmax(vref, fmax(f_r - hi, lo - f_r));
    if (f_b > hi) t = fmax(t, f_r < f_b ? (f_b - hi) / (f_b - f_r) : 1.0);
    if (f_b < lo) t = fmax(t, f_r > f_b ? (lo - f_b) / (f_r - f_b) : 1.0);
  }
  vref = block_max(vref, red);
  t = fmin(1.0, block_max(t, red));
  if (!(vref <= kTol)) {  // the reference breaks a limit: no bound
    for (int j = tid; j < ng; j += nt) xub[j] = 0.0;
    if (tid == 0) { pst[b] = 2; tout[b] = NAN; }
    return;
  }
  const double* xbb = xb + (size_t)b * ng;
  const double* xrb = xr + (size_t)b * ng;
  for (int j = tid; j < ng; j += nt) xub[j] = (1.0 - t) * xbb[j] + t * xrb[j];
  if (tid == 0) tout[b] = t;
}

// Largest flow violation of the repaired dispatch (its flows recomputed), its cost
// (the upper bound; +inf without a bound) and the dispatch in p.u.
__global__ void k_primal_finish(DevNet N, const int* __restrict__ outage, const double* __restrict__ u,
                                const double* __restrict__ f, const double* __restrict__ xu,
                                const int* __restrict__ pst, double* __restrict__ upper,
                                double* __restrict__ dispatch, double* __restrict__ maxviol) {
  __shared__ double red[32];
  const int b = blockIdx.x, nl = N.n_line, ng = N.n_gen, tid = threadIdx.x, nt = blockDim.x;
  const bool ok = pst[b] == 0;
  const double* xb = xu + (size_t)b * ng;
  if (dispatch)
    for (int j = tid; j < ng; j += nt)
      dispatch[(size_t)b * ng + j] = ok ? N.mid[j] + N.sigma[j] * xb[j] : NAN;
  if (!ok) {
    if (tid == 0) {
      upper[b] = INFINITY;
      if (maxviol) maxviol[b] = NAN;
    }
    return;
  }
  const int k = outage ? outage[b] : -1;
  const double* fb = f + (size_t)b * nl;
  const double fk = k >= 0 ? fb[k] : 0.0;
  double v = 0.0;
  for (int i = tid; i < nl; i += nt) {
    if (i == k) continue;
    const double fi = fb[i] + (k >= 0 ? u[(size_t)b * nl + i] * fk : 0.0);
    v = fmax(v, fmax(fi - N.fmax[i], N.fmin[i] - fi));
  }
  double c = 0.0;
  for (int j = tid; j < ng; j += nt) {
    const double x = xb[j];
    c += (N.mq[j] * x + N.ctil[j]) * x + N.cconst[j];
  }
  v = block_max(v, red);
  c = block_sum(c, red);
  if (tid == 0) {
    upper[b] = c;
    if (maxviol) maxviol[b] = v;
  }
}

dcopf_status run_primal(dcopf_dual* h, int B, const int* outage, const double* lambda,
                        const double* mh, const double* ml, const double* p_cand,
                        const double* p_ref, double* upper, int* pstatus, double* dispatch,
                        double* maxviol, cudaStream_t s) {
  const DevNet& N = h->dev;
  Workspace& w = h->ws;
  const int nl = N.n_line, ng = N.n_gen;
  PrimalBufs& pb = h->pb;
  if (B > pb.cap) {
    pb.cap = 0;  // reset unless every buffer below is allocated
    const size_t bg = (size_t)B * ng * 8, bl = (size_t)B * nl * 8;
    if (pb.xr.alloc(bg) != cudaSuccess || pb.xu.alloc(bg) != cudaSuccess ||
        pb.fr.alloc(bl) != cudaSuccess || pb.t.alloc((size_t)B * 8) != cudaSuccess ||
        pb.st.alloc((size_t)B * 4) != cudaSuccess) {
      cudaGetLastError();
      return DCOPF_ERR_OOM;
    }
    pb.cap = B;
  }
  int* pst = pstatus ? pstatus : pb.st.as<int>();
  if (!p_cand) launch_adjoint64(h, B, outage, mh, ml, s);
  k_primal_balance<<<B, 256, 0, s>>>(N, lambda, w.pit64.as<double>(), w.demand.as<double>(), p_cand,
                                     p_ref, w.x64.as<double>(), pb.xr.as<double>(), pst);
  launch_forward64(h, B, w.x64.as<double>(), w.f0.as<double>(), w.f.as<double>(), s);
  launch_forward64(h, B, pb.xr.as<double>(), w.f0.as<double>(), pb.fr.as<double>(), s);
  k_primal_repair<<<B, 256, 0, s>>>(N, outage, w.u64.as<double>(), w.f.as<double>(),
                                    pb.fr.as<double>(), w.x64.as<double>(), pb.xr.as<double>(), pst,
                                    pb.t.as<double>(), pb.xu.as<double>());
  launch_forward64(h, B, pb.xu.as<double>(), w.f0.as<double>(), w.f.as<double>(), s);
  k_primal_finish<<<B, 256, 0, s>>>(N, outage, w.u64.as<double>(), w.f.as<double>(),
                                    pb.xu.as<double>(), pst, upper, dispatch, maxviol);
  h->launches += 3;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { h->last_error = cudaGetErrorString(e); return DCOPF_ERR_CUDA; }
  return DCOPF_OK;
}

}  // namespace dcopf
