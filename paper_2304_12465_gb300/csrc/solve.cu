// Solve drivers: RPCholesky-preconditioned CG (Alg. 1) in float64 or with
// mixed-precision iterative refinement, and KRILL PCG (Alg. 2).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <vector>

#include "dense.cuh"
#include "kmv.cuh"
#include "krill.cuh"
#include "pcg.cuh"
#include "rpc.cuh"
#include "solve.cuh"

namespace krr {

template <typename T>
__global__ void scale_kernel(const T *__restrict__ in, T *__restrict__ out, int64_t n, double a) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (T)((double)in[e] * a);
}

template <typename T>
static krr_status scale(const T *in, T *out, int64_t n, double a, cudaStream_t s) {
  int64_t g = (n + 255) / 256;
  if (g > num_sms() * 8) g = num_sms() * 8;
  scale_kernel<T><<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(in, out, n, a);
  KRR_LAUNCH_CHECK();
  return KRR_OK;
}

// Relative tolerance floor of one inner float32 PCG solve.
constexpr double kInnerFloor = 1e-4;
// Share of the outer tolerance an inner solve aims at: the true residual
// after the correction follows the inner recursive one to within the float32
// products' rounding, so half the remaining need leaves a factor-2 margin.
constexpr double kInnerTarget = 0.5;

struct RefineStats {
  int iters = 0, outer = 0, products32 = 0, products64 = 0;
  double relres = 0.0;
  krr_status status = KRR_OK;
};

krr_status refine_solve(const PcgOps<float> &ops,
                        const std::function<krr_status(const double *, double *, cudaStream_t)>
                            &product64,
                        int64_t N, int m, const double *Y, double *alpha, double tol, int maxit,
                        cudaStream_t s, RefineStats *rs);

static double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

krr_status pcg_solve_device(const double *Xd, int64_t N, int d, int kern, double sigma,
                            const double *Y, int m, double mu, const krr_factor *F,
                            double tol, int maxit, int prec, double *alpha, cudaStream_t s,
                            krr_info *info) {
  const double lambda = mu * (double)N;
  auto t0 = std::chrono::steady_clock::now();
  pcg_counters_take(nullptr, nullptr);
  const NystromCore *core = nullptr;
  // the float-float path applies the float64 preconditioner
  const int core_prec = (prec == KRR_PREC_FLOAT_FLOAT) ? (int)KRR_PREC_FP64 : prec;
  if (F && F->rank > 0) KRR_TRY(nystrom_core(F, mu, core_prec, s, &core));
  const double t_build = core ? core->build_s : 0.0;
  auto t1 = std::chrono::steady_clock::now();
  (void)t0;
  std::vector<double> tolv(m, tol);
  double entries = 0.0;
  int outer = 0, iters_total = 0, escalated = 0;
  double relres = 0.0;
  krr_status final_status = KRR_OK;

  if (prec == KRR_PREC_FP64 || prec == KRR_PREC_FLOAT_FLOAT) {
    // float64 PCG; the products in float64, or (float-float) float64-accurate
    // products on the float32 pipes -- the same iterates up to rounding
    DevBuf<double> part;
    DevBuf<float> vsplit;
    PointsFF Pff;
    const bool ff = (prec == KRR_PREC_FLOAT_FLOAT);
    if (ff) KRR_TRY(prepare_points_ff(Xd, N, d, kern, sigma, s, Pff));
    auto product = [&](const double *in, double *out, cudaStream_t st) {
      if (ff) return kmv_ff(Pff, lambda, in, N, m, out, N, st, part, vsplit);
      return kmv_f64(Xd, N, d, kern, sigma, lambda, in, N, m, out, N, st, part);
    };
    PcgOps<double> ops;
    PrecondWs pws;
    ops.product = product;
    ops.precond = [&](const double *in, double *out, cudaStream_t st) {
      if (core) return nystrom_apply_f64(F, core, in, m, out, st, &pws);
      return scale<double>(in, out, N * m, 1.0 / lambda, st);
    };
    PcgStats stats;
    KRR_TRY(pcg_run<double>(ops, N, m, Y, alpha, tolv.data(), maxit, s, &stats));
    iters_total = stats.iters_max;
    entries += kmv_entries(N) * stats.products;
    if (stats.breakdown) final_status = KRR_EBREAKDOWN;
    else if (!stats.converged) final_status = KRR_ENOCONV;
    relres = stats.relres_max;
    if (info) {
      DevBuf<double> mx, r;
      KRR_TRY(mx.alloc((size_t)N * m, s));
      KRR_TRY(r.alloc((size_t)N * m, s));
      KRR_TRY(product(alpha, mx.p, s));
      entries += kmv_entries(N);
      KRR_TRY(residual_f64(Y, mx.p, r.p, N * m, s));
      std::vector<double> rn(m), yn(m);
      KRR_TRY(column_norms(r.p, N, m, rn.data(), s));
      KRR_TRY(column_norms(Y, N, m, yn.data(), s));
      relres = 0.0;
      for (int c = 0; c < m; ++c) relres = std::max(relres, yn[c] > 0 ? rn[c] / yn[c] : rn[c]);
    }
  } else {
    // iterative refinement: float64 outer loop around a float32 inner PCG
    PointsF32 P;
    KRR_TRY(prepare_points_f32(Xd, N, d, kern, sigma, s, P));
    KRR_TRY(prepare_points_tc(Xd, s, P));
    PointsFF Pff;
    KRR_TRY(prepare_points_ff(Xd, N, d, kern, sigma, s, Pff));
    DevBuf<float> part32, vsplit;
    DevBuf<double> part64;
    PcgOps<float> ops;
    const float lam32 = (float)lambda;
    ops.product = [&](const float *in, float *out, cudaStream_t st) {
      return kmv_f32(P, lam32, in, N, m, out, N, st, part32);
    };
    PrecondWs pws;
    ops.precond = [&](const float *in, float *out, cudaStream_t st) {
      if (core) return nystrom_apply_f32(F, core, in, m, out, st, &pws);
      return scale<float>(in, out, N * m, 1.0 / lambda, st);
    };
    auto product64 = [&](const double *in, double *out, cudaStream_t st) {
      return kmv_ff(Pff, lambda, in, N, m, out, N, st, part64, vsplit);
    };
    RefineStats rs;
    KRR_TRY(refine_solve(ops, product64, N, m, Y, alpha, tol, maxit, s, &rs));
    iters_total = rs.iters;
    outer = rs.outer;
    relres = rs.relres;
    final_status = rs.status;
    entries += kmv_entries(N) * (rs.products32 + rs.products64);
    if (final_status != KRR_OK && maxit - rs.iters > 0) {
      // the float32 inner iterations stalled: continue in higher precision
      DevBuf<double> r64, mx;
      KRR_TRY(r64.alloc((size_t)N * m, s));
      KRR_TRY(mx.alloc((size_t)N * m, s));
      Escalation e;
      e.Pff = &Pff;
      e.X = Xd;
      e.N = N;
      e.d = d;
      e.kern = kern;
      e.m = m;
      e.sigma = sigma;
      e.lambda = lambda;
      e.tol = tol;
      e.core = core;
      e.Y = Y;
      e.alpha = alpha;
      e.r64 = r64.p;
      e.mx = mx.p;
      e.yn.resize(m);
      e.rn.resize(m);
      KRR_TRY(column_norms(Y, N, m, e.yn.data(), s));
      KRR_TRY(kmv_ff(Pff, lambda, alpha, N, m, mx.p, N, s, part64, vsplit));
      KRR_TRY(residual_f64(Y, mx.p, r64.p, (int64_t)N * m, s));
      KRR_TRY(column_norms(r64.p, N, m, e.rn.data(), s));
      e.budget = maxit - rs.iters;
      e.iters = rs.iters;
      e.outer = rs.outer;
      e.entries = kmv_entries(N);
      e.ffpart = &part64;
      e.ffvsplit = &vsplit;
      KRR_TRY(escalate_refine(e, s));
      iters_total = e.iters;
      outer = e.outer;
      relres = e.relres;
      final_status = e.status;
      entries += e.entries;
      escalated = 1;
    }
  }
  KRR_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iters = iters_total;
    info->outer_refinements = outer;
    info->rank = F ? F->rank : 0;
    info->escalated = escalated;
    info->rel_residual = relres;
    info->kernel_entries = entries;
    info->t_build_s = t_build;
    info->t_solve_s = seconds_since(t1);
    pcg_counters_take(&info->graph_replays, &info->host_checks);
  }
  if (final_status == KRR_ENOCONV)
    set_error("PCG did not reach the tolerance (relative residual %.3e > %.3e)", relres, tol);
  if (final_status == KRR_EBREAKDOWN) set_error("PCG breakdown: p^T M p <= 0 or NaN");
  return final_status;
}

// Mixed-precision iterative refinement shared by the single and batched
// solves: x = 0, r = y; repeat { solve M d = r with the float32 PCG to a
// loose per-column tolerance; x += d; r = y - M x with the float64-accurate
// product } until every column's float64 relative residual is <= tol.
krr_status refine_solve(const PcgOps<float> &ops,
                        const std::function<krr_status(const double *, double *, cudaStream_t)>
                            &product64,
                        int64_t N, int m, const double *Y, double *alpha, double tol, int maxit,
                        cudaStream_t s, RefineStats *rs) {
  DevBuf<float> b32, d32;
  DevBuf<double> mx, r64;
  KRR_TRY(b32.alloc((size_t)N * m, s));
  KRR_TRY(d32.alloc((size_t)N * m, s));
  KRR_TRY(mx.alloc((size_t)N * m, s));
  KRR_TRY(r64.alloc((size_t)N * m, s));
  KRR_CUDA_TRY(cudaMemsetAsync(alpha, 0, sizeof(double) * N * m, s));
  KRR_CUDA_TRY(cudaMemcpyAsync(r64.p, Y, sizeof(double) * N * m, cudaMemcpyDeviceToDevice, s));
  std::vector<double> yn(m), rn(m);
  KRR_TRY(column_norms(Y, N, m, yn.data(), s));
  rn = yn;
  const int max_outer = 12;
  double prev_worst = 1e300;
  krr_status final_status = KRR_ENOCONV;
  int budget = maxit, outer = 0, iters = 0, prod32 = 0;
  double relres = 0.0;
  auto worst_rel = [&]() {
    double w = 0.0;
    for (int c = 0; c < m; ++c) w = std::max(w, yn[c] > 0 ? rn[c] / yn[c] : 0.0);
    return w;
  };
  while (true) {
    const double worst = worst_rel();
    relres = worst;
    if (worst <= tol) { final_status = KRR_OK; break; }
    if (outer >= max_outer || budget <= 0) break;
    if (outer > 0 && worst > 0.5 * prev_worst) break;  // refinement stagnated
    prev_worst = worst;
    // inner tolerances: aim below what the outer test needs (kInnerTarget), but
    // stop each float32 solve at kInnerFloor -- below that its recursive
    // residual keeps falling while the true residual is held up by float32
    // products, so the iterations are better spent after the next float64
    // residual
    std::vector<double> inner_tol(m);
    KRR_TRY(convert_f64_to_f32(r64.p, b32.p, N * m, s));
    for (int c = 0; c < m; ++c) {
      const double rel = (yn[c] > 0) ? rn[c] / yn[c] : 0.0;
      inner_tol[c] = (rel > tol) ? std::max(kInnerTarget * tol / rel, kInnerFloor) : 1.0;
      // columns already converged get a zero right-hand side (no work)
      if (!(rel > tol))
        KRR_CUDA_TRY(cudaMemsetAsync(b32.p + (int64_t)c * N, 0, sizeof(float) * N, s));
    }
    // one float32 inner solve may use at most half the iteration budget: one
    // that runs into this cap has stalled (see escalate_refine)
    const int limit = std::min(budget, std::max(1, maxit / 2));
    PcgStats st;
    KRR_TRY(pcg_run<float>(ops, N, m, b32.p, d32.p, inner_tol.data(), limit, s, &st));
    iters += st.iters_max;
    budget -= st.iters_max;
    prod32 += st.products;
    const bool capped = st.iters_max >= limit && !st.converged;
    KRR_TRY(add_f32_to_f64(alpha, d32.p, N * m, s));
    KRR_TRY(product64(alpha, mx.p, s));
    KRR_TRY(residual_f64(Y, mx.p, r64.p, N * m, s));
    KRR_TRY(column_norms(r64.p, N, m, rn.data(), s));
    ++outer;
    if (st.breakdown) { final_status = KRR_EBREAKDOWN; break; }
    if (capped && worst_rel() > tol) break;
  }
  if (final_status != KRR_OK && final_status != KRR_EBREAKDOWN) {
    relres = worst_rel();
    if (relres <= tol) final_status = KRR_OK;
  }
  rs->iters = iters;
  rs->outer = outer;
  rs->relres = relres;
  rs->status = final_status;
  rs->products32 = prod32;
  rs->products64 = outer;
  return KRR_OK;
}

// --------------------------------------------------------------- batched
__global__ void add_shift_kernel(double *__restrict__ out, const double *__restrict__ x,
                                 int64_t N, int m, const double *__restrict__ lam) {
  const int64_t total = N * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] += lam[e / N] * x[e];
}

krr_status pcg_solve_batched_device(const double *Xd, int64_t N, int d, int S,
                                    const int *kerns, const double *sigmas,
                                    const krr_factor *const *factors, int ms,
                                    const double *mus, const double *Y, double tol, int maxit,
                                    double *alpha, cudaStream_t s, krr_info *info) {
  auto t0 = std::chrono::steady_clock::now();
  pcg_counters_take(nullptr, nullptr);
  const int mt = S * ms;
  std::vector<double> lam(mt);
  std::vector<const NystromCore *> cores(mt, nullptr);
  double t_build = 0.0;
  for (int q = 0; q < S; ++q)
    for (int c = 0; c < ms; ++c) {
      lam[q * ms + c] = mus[c] * (double)N;
      if (factors && factors[q] && factors[q]->rank > 0) {
        KRR_TRY(nystrom_core(factors[q], mus[c], KRR_PREC_MIXED, s, &cores[q * ms + c]));
        t_build += cores[q * ms + c]->build_s;
      }
    }
  auto t1 = std::chrono::steady_clock::now();
  (void)t0;
  PointsF32 Pb;
  KRR_TRY(kmvb_prepare(Xd, N, d, s, Pb));
  std::vector<PointsFF> Pff(S);
  for (int q = 0; q < S; ++q) KRR_TRY(prepare_points_ff(Xd, N, d, kerns[q], sigmas[q], s, Pff[q]));
  std::vector<float> lam32(mt);
  for (int c = 0; c < mt; ++c) lam32[c] = (float)lam[c];
  DevBuf<float> lam_dev32, part32, vsplit;
  DevBuf<double> lam_dev, part64;
  KRR_TRY(lam_dev32.alloc(mt, s));
  KRR_TRY(lam_dev.alloc(mt, s));
  KRR_CUDA_TRY(cudaMemcpyAsync(lam_dev32.p, lam32.data(), sizeof(float) * mt,
                               cudaMemcpyHostToDevice, s));
  KRR_CUDA_TRY(cudaMemcpyAsync(lam_dev.p, lam.data(), sizeof(double) * mt,
                               cudaMemcpyHostToDevice, s));
  PcgOps<float> ops;
  ops.product = [&](const float *in, float *out, cudaStream_t st) {
    return kmv_batched_f32(Pb, S, kerns, sigmas, ms, lam_dev32.p, in, out, st, part32);
  };
  PrecondWs pws;
  ops.precond = [&](const float *in, float *out, cudaStream_t st) {
    for (int q = 0; q < S; ++q)
      for (int c = 0; c < ms; ++c) {
        const int col = q * ms + c;
        const float *r = in + (int64_t)col * N;
        float *z = out + (int64_t)col * N;
        if (cores[col]) KRR_TRY(nystrom_apply_f32(factors[q], cores[col], r, 1, z, st, &pws));
        else KRR_TRY(scale<float>(r, z, N, 1.0 / lam[col], st));
      }
    return KRR_OK;
  };
  auto product64 = [&](const double *in, double *out, cudaStream_t st) {
    // A_s x without the shift, per setting, then + lambda x per column
    for (int q = 0; q < S; ++q)
      KRR_TRY(kmv_ff(Pff[q], 0.0, in + (int64_t)q * ms * N, N, ms, out + (int64_t)q * ms * N,
                     N, st, part64, vsplit));
    int64_t g = (N * mt + 255) / 256;
    if (g > num_sms() * 8) g = num_sms() * 8;
    add_shift_kernel<<<(unsigned)g, 256, 0, st>>>(out, in, N, mt, lam_dev.p);
    KRR_LAUNCH_CHECK();
    return KRR_OK;
  };
  RefineStats rs;
  KRR_TRY(refine_solve(ops, product64, N, mt, Y, alpha, tol, maxit, s, &rs));
  KRR_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iters = rs.iters;
    info->outer_refinements = rs.outer;
    info->rank = 0;
    info->escalated = 0;
    for (int q = 0; q < S; ++q)
      if (factors && factors[q]) info->rank = std::max(info->rank, factors[q]->rank);
    info->rel_residual = rs.relres;
    info->kernel_entries = kmv_entries(N) * ((double)S * rs.products32 + (double)S * rs.products64);
    info->t_build_s = t_build;
    info->t_solve_s = seconds_since(t1);
    pcg_counters_take(&info->graph_replays, &info->host_checks);
  }
  if (rs.status == KRR_ENOCONV)
    set_error("batched PCG did not reach the tolerance (%.3e > %.3e)", rs.relres, tol);
  if (rs.status == KRR_EBREAKDOWN) set_error("batched PCG breakdown");
  return rs.status;
}

// --------------------------------------------------------------- KRILL
__global__ void axpy_sub_kernel(const double *__restrict__ b, const double *__restrict__ mx,
                                double *__restrict__ r, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    r[e] = b[e] - mx[e];
}

__global__ void add_f64_kernel(double *__restrict__ x, const double *__restrict__ d, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    x[e] += d[e];
}

krr_status krill_solve_device(const krill_precond *P, const double *Y, int m, double tol,
                              int maxit, double *beta, cudaStream_t s, krr_info *info) {
  auto t1 = std::chrono::steady_clock::now();
  pcg_counters_take(nullptr, nullptr);
  const int k = P->k;
  DevBuf<double> b, tmp, r, dx, mx, u64, v64;
  KRR_TRY(b.alloc((size_t)k * m, s));
  KRR_TRY(tmp.alloc((size_t)k * m, s));
  KRR_TRY(r.alloc((size_t)k * m, s));
  KRR_TRY(dx.alloc((size_t)k * m, s));
  KRR_TRY(mx.alloc((size_t)k * m, s));
  KrillFF Q;
  KRR_TRY(krill_points_ff(P, s, Q));
  KRR_TRY(krill_rhs(P, Q, Y, m, b.p, s));
  KrillTC5 T;
  KRR_TRY(krill_points_tc5(P, s, T));
  double entries = (double)P->N * k;
  DevBuf<float> u;
  DevBuf<double> v;
  PcgOps<double> ops;
  ops.product = [&](const double *in, double *out, cudaStream_t st) {
    return T.ok ? krill_product_tc5(P, T, in, m, out, st, u)
                : krill_product(P, in, m, out, st, u, v);
  };
  ops.precond = [&](const double *in, double *out, cudaStream_t st) {
    return krill_precond_apply(P, in, m, tmp.p, out, st);
  };
  KRR_CUDA_TRY(cudaMemsetAsync(beta, 0, sizeof(double) * k * m, s));
  KRR_CUDA_TRY(cudaMemcpyAsync(r.p, b.p, sizeof(double) * k * m, cudaMemcpyDeviceToDevice, s));
  std::vector<double> bn(m), rn(m);
  KRR_TRY(column_norms(b.p, k, m, bn.data(), s));
  rn = bn;
  int outer = 0, iters_total = 0, budget = maxit;
  double relres = 1.0, prev = 1e300;
  krr_status final_status = KRR_ENOCONV;
  bool breakdown = false;
  while (true) {
    double worst = 0.0;
    for (int c = 0; c < m; ++c) worst = std::max(worst, bn[c] > 0 ? rn[c] / bn[c] : 0.0);
    relres = worst;
    if (worst <= tol) { final_status = KRR_OK; break; }
    if (outer >= 12 || budget <= 0) break;
    if (outer > 0 && worst > 0.5 * prev) break;
    prev = worst;
    std::vector<double> itol(m);
    for (int c = 0; c < m; ++c) {
      const double rel = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
      itol[c] = (rel > tol) ? std::max(0.3 * tol / rel, 1e-5) : 1.0;
      if (!(rel > tol)) KRR_CUDA_TRY(cudaMemsetAsync(r.p + (int64_t)c * k, 0, sizeof(double) * k, s));
    }
    PcgStats st;
    KRR_TRY(pcg_run<double>(ops, k, m, r.p, dx.p, itol.data(), budget, s, &st));
    iters_total += st.iters_max;
    budget -= st.iters_max;
    entries += 2.0 * (double)P->N * k * st.products;
    add_f64_kernel<<<ceil_div((int64_t)k * m, 256), 256, 0, s>>>(beta, dx.p, (int64_t)k * m);
    KRR_LAUNCH_CHECK();
    KRR_TRY(krill_product64(P, Q, beta, m, mx.p, s, u64, v64));
    entries += 2.0 * (double)P->N * k;
    axpy_sub_kernel<<<ceil_div((int64_t)k * m, 256), 256, 0, s>>>(b.p, mx.p, r.p, (int64_t)k * m);
    KRR_LAUNCH_CHECK();
    KRR_TRY(column_norms(r.p, k, m, rn.data(), s));
    ++outer;
    if (st.breakdown) { breakdown = true; break; }
  }
  if (final_status != KRR_OK) {
    double worst = 0.0;
    for (int c = 0; c < m; ++c) worst = std::max(worst, bn[c] > 0 ? rn[c] / bn[c] : 0.0);
    relres = worst;
    if (worst <= tol) final_status = KRR_OK;
  }
  KRR_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iters = iters_total;
    info->outer_refinements = outer;
    info->rank = k;
    info->escalated = 0;
    info->rel_residual = relres;
    info->kernel_entries = entries;
    info->t_build_s = P->build_s;
    info->t_solve_s = seconds_since(t1);
    pcg_counters_take(&info->graph_replays, &info->host_checks);
  }
  if (breakdown && final_status != KRR_OK) {
    set_error("KRILL PCG breakdown");
    return KRR_EBREAKDOWN;
  }
  if (final_status != KRR_OK) {
    set_error("KRILL PCG did not reach the tolerance (%.3e > %.3e)", relres, tol);
    return KRR_ENOCONV;
  }
  return KRR_OK;
}

}  // namespace krr

namespace krr {

static double escalation_worst(const Escalation &e) {
  double w = 0.0;
  for (int c = 0; c < e.m; ++c) w = std::max(w, e.yn[c] > 0 ? e.rn[c] / e.yn[c] : 0.0);
  return w;
}

krr_status escalate_refine(Escalation &e, cudaStream_t s) {
  const int64_t N = e.N, nm = N * e.m;
  const int m = e.m;
  DevBuf<double> b64, d64, F64, X64, part64;
  KRR_TRY(b64.alloc((size_t)nm, s));
  KRR_TRY(d64.alloc((size_t)nm, s));
  // the float32 factor in float64 (exactly representable), consistent with
  // the mixed core W that was built from it
  krr_factor view;
  view.N = N;
  NystromCore identity;
  identity.lambda = e.lambda;
  const NystromCore *core = (e.core && e.core->rank > 0) ? e.core : &identity;
  if (core != &identity) {
    KRR_TRY(F64.alloc((size_t)N * core->rank, s));
    KRR_TRY(convert_f32_to_f64(core->F32, F64.p, N * core->rank, s));
    view.F = F64.p;
  }
  PcgOps<double> ops;
  ops.product = [&](const double *in, double *out, cudaStream_t st) {
    return kmv_ff(*e.Pff, e.lambda, in, N, m, out, N, st, *e.ffpart, *e.ffvsplit);
  };
  PrecondWs pws;
  ops.precond = [&](const double *in, double *out, cudaStream_t st) {
    return nystrom_apply_f64(&view, core, in, m, out, st, &pws);
  };
  // second stage: the float-float product's own rounding (about 2^-48 of
  // sum_j |a_ij x_j|) can reach the order of the residual; residuals then come
  // from the float64 product
  bool res64 = false;
  const double *Xdev = nullptr;
  auto residual = [&]() -> krr_status {
    if (res64)
      KRR_TRY(kmv_f64(Xdev, N, e.d, e.kern, e.sigma, e.lambda, e.alpha, N, m, e.mx, N, s,
                      part64));
    else
      KRR_TRY(kmv_ff(*e.Pff, e.lambda, e.alpha, N, m, e.mx, N, s, *e.ffpart, *e.ffvsplit));
    e.entries += kmv_entries(N);
    KRR_TRY(residual_f64(e.Y, e.mx, e.r64, nm, s));
    return column_norms(e.r64, N, m, e.rn.data(), s);
  };
  e.status = KRR_ENOCONV;
  double prev = 1e300;
  for (int outer = 0;; ++outer) {
    double worst = escalation_worst(e);
    e.relres = worst;
    if (worst <= e.tol) { e.status = KRR_OK; break; }
    if (outer >= 10 || e.budget <= 0) break;
    if (outer > 0 && worst > 0.5 * prev) {
      if (res64) break;
      res64 = true;
      KRR_TRY(device_view(e.X, (size_t)N * e.d, s, X64, &Xdev));
      KRR_TRY(residual());
      worst = escalation_worst(e);
      e.relres = worst;
      if (worst <= e.tol) { e.status = KRR_OK; break; }
    }
    prev = worst;
    std::vector<double> itol(m);
    KRR_CUDA_TRY(cudaMemcpyAsync(b64.p, e.r64, sizeof(double) * nm, cudaMemcpyDeviceToDevice, s));
    for (int c = 0; c < m; ++c) {
      const double rel = e.yn[c] > 0 ? e.rn[c] / e.yn[c] : 0.0;
      itol[c] = rel > e.tol ? std::max(0.3 * e.tol / rel, 1e-12) : 1.0;
      if (!(rel > e.tol))
        KRR_CUDA_TRY(cudaMemsetAsync(b64.p + (int64_t)c * N, 0, sizeof(double) * N, s));
    }
    PcgStats st;
    KRR_TRY(pcg_run<double>(ops, N, m, b64.p, d64.p, itol.data(), e.budget, s, &st));
    e.iters += st.iters_max;
    e.budget -= st.iters_max;
    e.entries += kmv_entries(N) * st.products;
    add_f64_kernel<<<ceil_div(nm, 256), 256, 0, s>>>(e.alpha, d64.p, nm);
    KRR_LAUNCH_CHECK();
    KRR_TRY(residual());
    e.outer += 1;
    if (st.breakdown) {
      e.status = KRR_EBREAKDOWN;
      break;
    }
  }
  if (e.status != KRR_OK) {
    e.relres = escalation_worst(e);
    if (e.relres <= e.tol) e.status = KRR_OK;
  }
  view.F = nullptr;
  return KRR_OK;
}

}  // namespace krr
