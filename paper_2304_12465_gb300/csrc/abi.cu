// The C ABI declared in include/krr.h: argument checks, host/device staging of
// caller arrays, and dispatch to the device implementations.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kmv.cuh"
#include "krill.cuh"
#include "pcg.cuh"
#include "rpc.cuh"
#include "solve.cuh"

namespace krr {

static thread_local std::string g_error;

void set_error(const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
}

void clear_error() { g_error.clear(); }

krr_status raise_smem_limit_ptr(const void *func, size_t bytes) {
  static std::mutex mtx;
  static std::vector<std::pair<const void *, size_t>> limits;
  std::lock_guard<std::mutex> lk(mtx);
  for (auto &e : limits) {
    if (e.first != func) continue;
    if (bytes <= e.second) return KRR_OK;
    KRR_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)bytes));
    e.second = bytes;
    return KRR_OK;
  }
  if (bytes > 48 * 1024)
    KRR_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)bytes));
  limits.emplace_back(func, bytes > 48 * 1024 ? bytes : 48 * 1024);
  return KRR_OK;
}

static thread_local cudaStream_t g_alloc_stream = nullptr;
void set_alloc_stream(cudaStream_t s) { g_alloc_stream = s; }
cudaStream_t alloc_stream() { return g_alloc_stream; }

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static std::atomic<unsigned long long> g_launches{0};
static thread_local bool g_count_launches = true;
void set_launch_counting(bool on) { g_count_launches = on; }
static thread_local CaptureLog *t_capture_log = nullptr;
void count_launch() {
  if (t_capture_log) {
    ++t_capture_log->launches;
    return;
  }
  if (g_count_launches) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int num_sms() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached = n > 0 ? n : 1;
  }
  return cached;
}

// -------------------------------------------------------------- profiling
static bool g_profiling = false;
static std::mutex g_prof_mtx;
struct ProfEvent {
  cudaEvent_t a, b;
  int tag;
};
static std::vector<ProfEvent> g_prof_events;
// launches timed inside replayed graphs, already converted to milliseconds
static double g_prof_done_ms[3] = {0.0, 0.0, 0.0};
static int g_prof_done_n[3] = {0, 0, 0};

bool profiling_on() { return g_profiling; }

void KmvTimer::begin(cudaStream_t s) {
  on = g_profiling;
  if (!on) return;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  if (t_capture_log) cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
  else cudaEventRecord(a, s);
}

void KmvTimer::end(cudaStream_t s) {
  if (!on) return;
  if (t_capture_log) {
    // an event node of the graph being captured: timed after each replay
    cudaEventRecordWithFlags(b, s, cudaEventRecordExternal);
    t_capture_log->timers.push_back({a, b, tag});
    return;
  }
  cudaEventRecord(b, s);
  std::lock_guard<std::mutex> lk(g_prof_mtx);
  g_prof_events.push_back({a, b, tag});
}

CaptureLog::~CaptureLog() {
  for (auto &t : timers) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
}

void capture_log_begin(CaptureLog *log) { t_capture_log = log; }

void capture_replayed(const CaptureLog &log) {
  count_launches(log.launches);
  if (log.timers.empty()) return;
  std::lock_guard<std::mutex> lk(g_prof_mtx);
  for (const auto &t : log.timers) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (t.tag >= 0 && t.tag < 3) {
      g_prof_done_ms[t.tag] += ms;
      g_prof_done_n[t.tag] += 1;
    }
  }
}

void kmv_profile_reset() {
  std::lock_guard<std::mutex> lk(g_prof_mtx);
  for (auto &e : g_prof_events) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  g_prof_events.clear();
  for (int t = 0; t < 3; ++t) {
    g_prof_done_ms[t] = 0.0;
    g_prof_done_n[t] = 0;
  }
}

void kmv_profile_collect(int tag, double *ms, int *launches) {
  std::lock_guard<std::mutex> lk(g_prof_mtx);
  double tot = 0.0;
  int n = 0;
  if (tag >= 0 && tag < 3) {
    tot = g_prof_done_ms[tag];
    n = g_prof_done_n[tag];
    g_prof_done_ms[tag] = 0.0;
    g_prof_done_n[tag] = 0;
  }
  std::vector<ProfEvent> keep;
  for (auto &e : g_prof_events) {
    if (e.tag != tag) {
      keep.push_back(e);
      continue;
    }
    float t = 0.f;
    cudaEventSynchronize(e.b);
    cudaEventElapsedTime(&t, e.a, e.b);
    tot += t;
    ++n;
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  *ms = tot;
  *launches = n;
  g_prof_events.swap(keep);
}

// Output staging: a device pointer is used directly; a host pointer gets a
// device buffer that is copied back by finish().
template <typename T>
struct OutView {
  T *user = nullptr;
  T *dev = nullptr;
  DevBuf<T> tmp;
  size_t count = 0;
  krr_status init(T *p, size_t n, cudaStream_t s) {
    user = p;
    count = n;
    if (p == nullptr || is_device_ptr(p)) {
      dev = p;
      return KRR_OK;
    }
    KRR_TRY(tmp.alloc(n, s));
    dev = tmp.p;
    return KRR_OK;
  }
  krr_status finish(cudaStream_t s) {
    if (user && dev != user && count) {
      KRR_CUDA_TRY(cudaMemcpyAsync(user, dev, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    }
    KRR_CUDA_TRY(cudaStreamSynchronize(s));
    return KRR_OK;
  }
};

static bool valid_kernel(int kern) {
  return kern == KRR_GAUSSIAN || kern == KRR_LAPLACE_L1 || kern == KRR_MATERN52;
}

#define KRR_CHECK_POINTS(X, N, d, kern, sigma)                                         \
  KRR_REQUIRE((X) != nullptr, "X is NULL");                                            \
  KRR_REQUIRE((N) >= 1, "N must be >= 1 (got %lld)", (long long)(N));                  \
  KRR_REQUIRE((d) >= 1 && (d) <= 32, "d must be in [1, 32] (got %d)", (int)(d));        \
  KRR_REQUIRE(valid_kernel(kern), "unknown kernel %d", (int)(kern));                   \
  KRR_REQUIRE((sigma) > 0 && std::isfinite(sigma), "sigma must be positive and finite")

void free_factor(krr_factor *f) {
  if (!f) return;
  dev_free(f->F, f->free_stream);
  dev_free(f->S, f->free_stream);
  dev_free(f->dres, f->free_stream);
  for (auto &c : f->cores) {
    dev_free(c.W, f->free_stream);
    dev_free(c.Wt, f->free_stream);
    dev_free(c.F32, f->free_stream);
  }
  delete f;
}

static void free_krill(krill_precond *P) {
  if (!P) return;
  cudaFree(P->X);
  cudaFree(P->S);
  cudaFree(P->H);
  cudaFree(P->Bsk);
  cudaFree(P->P);
  cudaFree(P->L);
  cudaFree(P->Winv);
  cudaFree(P->Winv_t);
  cudaFree(P->xt);
  cudaFree(P->cn);
  delete P;
}

}  // namespace krr

using namespace krr;

extern "C" {

const char *krr_last_error(void) { return g_error.c_str(); }

void krr_set_autotune(int on) { set_autotune(on != 0); }

void krr_set_pcg_graphs(int on) { set_pcg_graphs(on != 0); }

krr_status krr_check_bounded_wait(int64_t budget_cycles, void *stream) {
  clear_error();
  return tc5_wait_selftest((long long)budget_cycles, (cudaStream_t)stream);
}

krr_status krr_autotune_choice(krr_kernel kern, int d, int m, int64_t N, int *splits) {
  clear_error();
  KRR_REQUIRE(splits, "splits is NULL");
  KRR_REQUIRE(valid_kernel(kern), "unknown kernel %d", (int)kern);
  KRR_REQUIRE(d >= 1 && d <= 32 && m >= 1 && m <= 16 && N >= 1, "bad shape");
  const int M = m <= 1 ? 1 : m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : 16;
  *splits = tuned_splits((int)kern, (d + 3) / 4 * 4, M, N);
  return KRR_OK;
}

krr_status krr_set_product_path(int path) {
  clear_error();
  KRR_REQUIRE(path == KRR_PRODUCT_TENSOR || path == KRR_PRODUCT_FMA ||
                  path == KRR_PRODUCT_MMA_SYNC,
              "unknown product path %d", path);
  set_product_path(path);
  return KRR_OK;
}

krr_status krr_profile_collect(int which, double *ms, int *launches) {
  clear_error();
  KRR_REQUIRE(which >= 0 && which <= 2 && ms && launches, "bad profile query");
  kmv_profile_collect(which, ms, launches);
  return KRR_OK;
}

krr_status krr_set_product_variant(int variant) {
  clear_error();
  return set_tc5_variant(variant);
}

krr_status krr_autotune_variant(krr_kernel kern, int d, int m, int64_t N, int *variant,
                                float *ms) {
  clear_error();
  KRR_REQUIRE(variant, "variant is NULL");
  KRR_REQUIRE(valid_kernel(kern), "unknown kernel %d", (int)kern);
  KRR_REQUIRE(d >= 1 && d <= 32 && m >= 1 && m <= 16 && N >= 1, "bad shape");
  const int mg = m > 8 ? 8 : m;
  const int M = mg <= 2 ? 2 : mg <= 4 ? 4 : 8;
  int best = 0;
  float t[KRR_PRODUCT_VARIANTS] = {};
  if (!tc5_tuned((int)kern, d, M, N, &best, t)) best = 0;
  *variant = best;
  if (ms)
    for (int v = 0; v < KRR_PRODUCT_VARIANTS; ++v) ms[v] = t[v];
  return KRR_OK;
}

const char *krr_version(void) { return "krr-gb300 0.1 (sm_103a)"; }

uint64_t krr_launch_count(void) { return g_launches.load(); }

void krr_set_profiling(int on) {
  g_profiling = on != 0;
  kmv_profile_reset();
}

krr_status krr_kmatvec(const double *X, int64_t N, int d, krr_kernel kern, double sigma,
                       double lambda, const double *V, int m, double *Y, krr_precision prec,
                       void *stream) {
  clear_error();
  KRR_CHECK_POINTS(X, N, d, kern, sigma);
  KRR_REQUIRE(V && Y, "V and Y must not be NULL");
  KRR_REQUIRE(m >= 1 && m <= 16, "m must be in [1, 16]");
  KRR_REQUIRE(prec == KRR_PREC_FP64 || prec == KRR_PREC_MIXED || prec == KRR_PREC_FLOAT_FLOAT,
              "unknown precision");
  KRR_REQUIRE(std::isfinite(lambda), "lambda must be finite");
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf<double> tx, tv;
  const double *Xd, *Vd;
  KRR_TRY(device_view(X, (size_t)N * d, s, tx, &Xd));
  KRR_TRY(device_view(V, (size_t)N * m, s, tv, &Vd));
  OutView<double> out;
  KRR_TRY(out.init(Y, (size_t)N * m, s));
  if (prec == KRR_PREC_FP64) {
    DevBuf<double> part;
    KRR_TRY(kmv_f64(Xd, N, d, kern, sigma, lambda, Vd, N, m, out.dev, N, s, part));
  } else if (prec == KRR_PREC_FLOAT_FLOAT) {
    PointsFF P;
    KRR_TRY(prepare_points_ff(Xd, N, d, kern, sigma, s, P));
    DevBuf<double> part;
    DevBuf<float> vsplit;
    KRR_TRY(kmv_ff(P, lambda, Vd, N, m, out.dev, N, s, part, vsplit));
  } else {
    PointsF32 P;
    KRR_TRY(prepare_points_f32(Xd, N, d, kern, sigma, s, P));
    KRR_TRY(prepare_points_tc(Xd, s, P));
    DevBuf<float> v32, y32, part;
    KRR_TRY(v32.alloc((size_t)N * m, s));
    KRR_TRY(y32.alloc((size_t)N * m, s));
    KRR_TRY(convert_f64_to_f32(Vd, v32.p, N * m, s));
    KRR_TRY(kmv_f32(P, (float)lambda, v32.p, N, m, y32.p, N, s, part));
    KRR_TRY(tc5_check_fault(s));
    KRR_TRY(convert_f32_to_f64(y32.p, out.dev, N * m, s));
  }
  return out.finish(s);
}

krr_status krr_kmatvec_batched(const double *X, int64_t N, int d, int S, const int *kerns,
                               const double *sigmas, int ms, const double *lambdas,
                               const double *V, double *Y, void *stream) {
  clear_error();
  KRR_REQUIRE(X && kerns && sigmas && lambdas && V && Y, "NULL argument");
  KRR_REQUIRE(N >= 1, "N must be >= 1");
  KRR_REQUIRE(d >= 1 && d <= 32, "d must be in [1, 32]");
  KRR_REQUIRE(S >= 1 && S <= KRR_MAX_SETTINGS, "S must be in [1, %d]", KRR_MAX_SETTINGS);
  KRR_REQUIRE(ms == 1 || ms == 2, "ms must be 1 or 2");
  for (int q = 0; q < S; ++q) {
    KRR_REQUIRE(valid_kernel(kerns[q]), "unknown kernel %d in setting %d", kerns[q], q);
    KRR_REQUIRE(sigmas[q] > 0 && std::isfinite(sigmas[q]), "sigma of setting %d invalid", q);
  }
  for (int c = 0; c < S * ms; ++c)
    KRR_REQUIRE(std::isfinite(lambdas[c]), "lambda %d is not finite", c);
  cudaStream_t s = (cudaStream_t)stream;
  const int mt = S * ms;
  DevBuf<double> tx, tv;
  const double *Xd, *Vd;
  KRR_TRY(device_view(X, (size_t)N * d, s, tx, &Xd));
  KRR_TRY(device_view(V, (size_t)N * mt, s, tv, &Vd));
  OutView<double> out;
  KRR_TRY(out.init(Y, (size_t)N * mt, s));
  PointsF32 P;
  KRR_TRY(kmvb_prepare(Xd, N, d, s, P));
  std::vector<float> lam32(mt);
  for (int c = 0; c < mt; ++c) lam32[c] = (float)lambdas[c];
  DevBuf<float> lam, v32, y32, part;
  KRR_TRY(lam.alloc(mt, s));
  KRR_CUDA_TRY(cudaMemcpyAsync(lam.p, lam32.data(), sizeof(float) * mt, cudaMemcpyHostToDevice, s));
  KRR_TRY(v32.alloc((size_t)N * mt, s));
  KRR_TRY(y32.alloc((size_t)N * mt, s));
  KRR_TRY(convert_f64_to_f32(Vd, v32.p, N * mt, s));
  KRR_TRY(kmv_batched_f32(P, S, kerns, sigmas, ms, lam.p, v32.p, y32.p, s, part));
  KRR_TRY(convert_f32_to_f64(y32.p, out.dev, N * mt, s));
  return out.finish(s);
}

krr_status krr_predict(const double *Xtrain, int64_t N, int d, krr_kernel kern, double sigma,
                       const double *alpha, int m, const double *Xtest, int64_t Nt,
                       double *out, krr_precision prec, void *stream) {
  clear_error();
  KRR_CHECK_POINTS(Xtrain, N, d, kern, sigma);
  KRR_REQUIRE(alpha && Xtest && out, "alpha, Xtest and out must not be NULL");
  KRR_REQUIRE(Nt >= 1, "number of test points must be >= 1");
  KRR_REQUIRE(m >= 1 && m <= 16, "m must be in [1, 16]");
  KRR_REQUIRE(prec == KRR_PREC_FP64 || prec == KRR_PREC_MIXED, "unknown precision");
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf<double> tx, ta, tt;
  const double *Xd, *Ad, *Td;
  KRR_TRY(device_view(Xtrain, (size_t)N * d, s, tx, &Xd));
  KRR_TRY(device_view(alpha, (size_t)N * m, s, ta, &Ad));
  KRR_TRY(device_view(Xtest, (size_t)Nt * d, s, tt, &Td));
  OutView<double> o;
  KRR_TRY(o.init(out, (size_t)Nt * m, s));
  if (prec == KRR_PREC_FP64) {
    DevBuf<double> part;
    KRR_TRY(kcross_f64(Td, Nt, Xd, N, d, kern, sigma, Ad, N, m, o.dev, Nt, s, part));
  } else {
    PointsF32 P, R;
    KRR_TRY(prepare_points_f32(Xd, N, d, kern, sigma, s, P));
    KRR_TRY(prepare_points_f32(Td, Nt, d, kern, sigma, s, R, P.mean.p));
    // the tcgen05 rectangular product when both point sets have split operands
    bool tc5 = false;
    if (product_path() == 0) {
      int bad_p = 0, bad_r = 0;
      KRR_TRY(prepare_points_tc5(Xd, s, P, &bad_p));
      if (P.nh5 > 0) KRR_TRY(prepare_points_tc5(Td, s, R, &bad_r));
      tc5 = P.nh5 > 0 && R.nh5 > 0;
    }
    DevBuf<float> a32, y32, part;
    KRR_TRY(a32.alloc((size_t)N * m, s));
    KRR_TRY(y32.alloc((size_t)Nt * m, s));
    KRR_TRY(convert_f64_to_f32(Ad, a32.p, N * m, s));
    if (tc5) {
      KRR_TRY(kmv_tc5(R, P, 0.0f, false, a32.p, N, m, y32.p, Nt, s, part));
      KRR_TRY(tc5_check_fault(s));
    } else {
      KRR_TRY(kcross_f32(R, P, a32.p, N, m, y32.p, Nt, s, part));
    }
    KRR_TRY(convert_f32_to_f64(y32.p, o.dev, Nt * m, s));
  }
  return o.finish(s);
}

krr_status krr_rpc_sample(const double *dres, int64_t N, double dfloor, uint64_t seed,
                          uint64_t t, int ndraw, int64_t *draws, int *ndraw_out, void *stream) {
  clear_error();
  KRR_REQUIRE(dres && draws && ndraw_out, "NULL argument");
  KRR_REQUIRE(N >= 1, "N must be >= 1");
  KRR_REQUIRE(ndraw >= 1 && ndraw <= 1024, "ndraw must be in [1, 1024]");
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf<double> td;
  const double *dd;
  KRR_TRY(device_view(dres, (size_t)N, s, td, &dd));
  OutView<int64_t> out;
  KRR_TRY(out.init(draws, (size_t)ndraw, s));
  DevBuf<int64_t> cand;
  DevBuf<int> counts;
  KRR_TRY(cand.alloc(ndraw, s));
  KRR_TRY(counts.alloc(2, s));
  KRR_REQUIRE(!std::isnan(dfloor), "dfloor is NaN");
  KRR_TRY(rpc_sample_device(dd, N, dfloor, seed, t, ndraw, out.dev, cand.p, counts.p, s));
  int h[2];
  KRR_CUDA_TRY(cudaMemcpyAsync(h, counts.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  KRR_TRY(out.finish(s));
  *ndraw_out = h[0];
  return KRR_OK;
}

krr_status krr_rpcholesky(const double *X, int64_t N, int d, krr_kernel kern, double sigma,
                          int k, int block, uint64_t seed, void *stream, krr_factor **F_out) {
  return krr_pivoted_cholesky(X, N, d, kern, sigma, k, block, seed, KRR_PIVOT_RPCHOLESKY,
                              stream, F_out);
}

krr_status krr_pivoted_cholesky(const double *X, int64_t N, int d, krr_kernel kern,
                                double sigma, int k, int block, uint64_t seed,
                                krr_pivot_rule rule, void *stream, krr_factor **F_out) {
  clear_error();
  KRR_CHECK_POINTS(X, N, d, kern, sigma);
  KRR_REQUIRE(F_out, "F_out is NULL");
  *F_out = nullptr;
  KRR_REQUIRE(k >= 1 && k <= 4096 && k <= N, "k must be in [1, min(N, 4096)]");
  KRR_REQUIRE(rule == KRR_PIVOT_RPCHOLESKY || rule == KRR_PIVOT_UNIFORM ||
                  rule == KRR_PIVOT_GREEDY,
              "unknown pivot rule %d", (int)rule);
  if (block == 0 && rule == KRR_PIVOT_GREEDY) block = 1;
  if (block == 0) block = (k + 9) / 10 < 100 ? (k + 9) / 10 : 100;
  KRR_REQUIRE(block >= 1 && block <= RPC_MAX_BLOCK, "block must be in [1, %d]", RPC_MAX_BLOCK);
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf<double> tx;
  const double *Xd;
  KRR_TRY(device_view(X, (size_t)N * d, s, tx, &Xd));
  krr_factor *f = new (std::nothrow) krr_factor();
  if (!f) return KRR_ENOMEM;
  krr_status st = rpcholesky_device(Xd, N, d, kern, sigma, k, block, seed, s, f, (int)rule);
  if (st == KRR_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error("RPCholesky failed: %s", cudaGetErrorString(e));
      st = KRR_ECUDA;
    }
  }
  if (st != KRR_OK) {
    free_factor(f);
    return st;
  }
  *F_out = f;
  return KRR_OK;
}

krr_status krr_factor_info(const krr_factor *F, int64_t *N, int *rank, int *nblocks) {
  clear_error();
  KRR_REQUIRE(F, "factor is NULL");
  if (N) *N = F->N;
  if (rank) *rank = F->rank;
  if (nblocks) *nblocks = F->nblocks;
  return KRR_OK;
}

krr_status krr_factor_export(const krr_factor *F, double *F_out, int64_t *pivots, double *dres) {
  clear_error();
  KRR_REQUIRE(F, "factor is NULL");
  if (F_out)
    KRR_CUDA_TRY(cudaMemcpy(F_out, F->F, sizeof(double) * (size_t)F->N * F->rank,
                            cudaMemcpyDefault));
  if (pivots)
    KRR_CUDA_TRY(cudaMemcpy(pivots, F->S, sizeof(int64_t) * (size_t)F->rank, cudaMemcpyDefault));
  if (dres)
    KRR_CUDA_TRY(cudaMemcpy(dres, F->dres, sizeof(double) * (size_t)F->N, cudaMemcpyDefault));
  return KRR_OK;
}

void krr_factor_free(krr_factor *F) { free_factor(F); }

krr_status krr_precond_apply(const krr_factor *F, double mu, const double *R, int m, double *Z,
                             krr_precision prec, void *stream) {
  clear_error();
  KRR_REQUIRE(F && R && Z, "NULL argument");
  KRR_REQUIRE(m >= 1 && m <= 16, "m must be in [1, 16]");
  KRR_REQUIRE(mu > 0 && std::isfinite(mu), "mu must be positive");
  KRR_REQUIRE(prec == KRR_PREC_FP64 || prec == KRR_PREC_MIXED, "unknown precision");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = F->N;
  DevBuf<double> tr;
  const double *Rd;
  KRR_TRY(device_view(R, (size_t)N * m, s, tr, &Rd));
  OutView<double> out;
  KRR_TRY(out.init(Z, (size_t)N * m, s));
  const NystromCore *core = nullptr;
  NystromCore identity;  // rank 0: P = lambda I
  identity.mu = mu;
  identity.lambda = mu * (double)N;
  identity.prec = prec;
  if (F->rank > 0) KRR_TRY(nystrom_core(F, mu, prec, s, &core));
  else core = &identity;
  if (prec == KRR_PREC_FP64) {
    KRR_TRY(nystrom_apply_f64(F, core, Rd, m, out.dev, s));
  } else {
    DevBuf<float> r32, z32;
    KRR_TRY(r32.alloc((size_t)N * m, s));
    KRR_TRY(z32.alloc((size_t)N * m, s));
    KRR_TRY(convert_f64_to_f32(Rd, r32.p, N * m, s));
    KRR_TRY(nystrom_apply_f32(F, core, r32.p, m, z32.p, s));
    KRR_TRY(convert_f32_to_f64(z32.p, out.dev, N * m, s));
  }
  return out.finish(s);
}

krr_status krr_pcg_solve(const double *X, int64_t N, int d, krr_kernel kern, double sigma,
                         const double *Y, int m, double mu, const krr_factor *F, double tol,
                         int maxit, krr_precision prec, double *alpha_out, void *stream,
                         krr_info *info) {
  clear_error();
  KRR_CHECK_POINTS(X, N, d, kern, sigma);
  KRR_REQUIRE(Y && alpha_out, "Y and alpha_out must not be NULL");
  KRR_REQUIRE(m >= 1 && m <= 16, "m must be in [1, 16]");
  KRR_REQUIRE(mu > 0 && std::isfinite(mu), "mu must be positive and finite");
  KRR_REQUIRE(tol > 0 && tol < 1, "tol must be in (0, 1)");
  KRR_REQUIRE(prec == KRR_PREC_FP64 || prec == KRR_PREC_MIXED || prec == KRR_PREC_FLOAT_FLOAT,
              "unknown precision");
  KRR_REQUIRE(!F || F->N == N, "factor was built for N = %lld, not %lld", (long long)(F ? F->N : 0),
              (long long)N);
  if (maxit <= 0) maxit = 1000;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf<double> tx, ty;
  const double *Xd, *Yd;
  KRR_TRY(device_view(X, (size_t)N * d, s, tx, &Xd));
  KRR_TRY(device_view(Y, (size_t)N * m, s, ty, &Yd));
  OutView<double> out;
  KRR_TRY(out.init(alpha_out, (size_t)N * m, s));
  if (info) std::memset(info, 0, sizeof(*info));
  const bool prof = profiling_on();
  if (prof) kmv_profile_reset();
  krr_status st = pcg_solve_device(Xd, N, d, kern, sigma, Yd, m, mu, F, tol, maxit, prec, out.dev,
                                   s, info);
  if (st != KRR_OK && st != KRR_ENOCONV) return st;
  KRR_TRY(tc5_check_fault(s));   // a bounded wait of a tensor-core product gave up
  krr_status st2 = out.finish(s);
  if (st2 != KRR_OK) return st2;
  if (info && prof) {
    kmv_profile_collect(0, &info->kmv_ms, &info->kmv_launches);
    kmv_profile_collect(1, &info->kmv64_ms, &info->kmv64_launches);
    kmv_profile_collect(2, &info->kmvff_ms, &info->kmvff_launches);
  }
  return st;
}

krr_status krr_pcg_solve_batched(const double *X, int64_t N, int d, int S, const int *kerns,
                                 const double *sigmas, const krr_factor *const *factors,
                                 int ms, const double *mus, const double *Y, double tol,
                                 int maxit, double *alpha_out, void *stream, krr_info *info) {
  clear_error();
  KRR_REQUIRE(X && kerns && sigmas && mus && Y && alpha_out, "NULL argument");
  KRR_REQUIRE(N >= 1, "N must be >= 1");
  KRR_REQUIRE(d >= 1 && d <= 32, "d must be in [1, 32]");
  KRR_REQUIRE(S >= 1 && S <= KRR_MAX_SETTINGS, "S must be in [1, %d]", KRR_MAX_SETTINGS);
  KRR_REQUIRE(ms == 1 || ms == 2, "ms must be 1 or 2");
  KRR_REQUIRE(tol > 0 && tol < 1, "tol must be in (0, 1)");
  for (int q = 0; q < S; ++q) {
    KRR_REQUIRE(valid_kernel(kerns[q]), "unknown kernel %d in setting %d", kerns[q], q);
    KRR_REQUIRE(sigmas[q] > 0 && std::isfinite(sigmas[q]), "sigma of setting %d invalid", q);
    KRR_REQUIRE(!factors || !factors[q] || factors[q]->N == N, "factor %d has the wrong N", q);
  }
  for (int c = 0; c < ms; ++c)
    KRR_REQUIRE(mus[c] > 0 && std::isfinite(mus[c]), "mu %d must be positive", c);
  if (maxit <= 0) maxit = 1000;
  const int mt = S * ms;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf<double> tx, ty;
  const double *Xd, *Yd;
  KRR_TRY(device_view(X, (size_t)N * d, s, tx, &Xd));
  KRR_TRY(device_view(Y, (size_t)N * mt, s, ty, &Yd));
  OutView<double> out;
  KRR_TRY(out.init(alpha_out, (size_t)N * mt, s));
  if (info) std::memset(info, 0, sizeof(*info));
  const bool prof = profiling_on();
  if (prof) kmv_profile_reset();
  krr_status st = pcg_solve_batched_device(Xd, N, d, S, kerns, sigmas, factors, ms, mus, Yd, tol,
                                           maxit, out.dev, s, info);
  if (st != KRR_OK && st != KRR_ENOCONV) return st;
  krr_status st2 = out.finish(s);
  if (st2 != KRR_OK) return st2;
  if (info && prof) {
    kmv_profile_collect(0, &info->kmv_ms, &info->kmv_launches);
    kmv_profile_collect(2, &info->kmvff_ms, &info->kmvff_launches);
  }
  return st;
}

krr_status krr_sparse_sign(int64_t N, int s_rows, int zeta, uint64_t seed, int32_t *rows,
                           double *vals, void *stream) {
  clear_error();
  KRR_REQUIRE(rows && vals, "NULL argument");
  KRR_REQUIRE(N >= 1 && s_rows >= 1, "N and s must be >= 1");
  KRR_REQUIRE(zeta >= 1 && zeta <= 64 && zeta <= s_rows, "zeta must be in [1, min(s, 64)]");
  cudaStream_t s = (cudaStream_t)stream;
  OutView<int32_t> orow;
  OutView<double> oval;
  KRR_TRY(orow.init(rows, (size_t)N * zeta, s));
  KRR_TRY(oval.init(vals, (size_t)N * zeta, s));
  KRR_TRY(sparse_sign_device(N, s_rows, zeta, seed, orow.dev, nullptr, oval.dev, s));
  KRR_TRY(orow.finish(s));
  return oval.finish(s);
}

krr_status krill_build(const double *X, int64_t N, int d, krr_kernel kern, double sigma,
                       const int64_t *centers, int k, double mu, int sketch_rows, int zeta,
                       uint64_t seed, void *stream, krill_precond **P_out) {
  clear_error();
  KRR_CHECK_POINTS(X, N, d, kern, sigma);
  KRR_REQUIRE(centers && P_out, "NULL argument");
  *P_out = nullptr;
  KRR_REQUIRE(k >= 1 && k <= 8192 && k <= N, "k must be in [1, min(N, 8192)]");
  KRR_REQUIRE(mu > 0 && std::isfinite(mu), "mu must be positive and finite");
  if (sketch_rows == 0) sketch_rows = 2 * k;
  if (zeta == 0) zeta = (int)std::ceil(std::log((double)k + 1.0));
  if (zeta < 1) zeta = 1;
  KRR_REQUIRE(sketch_rows >= 1 && sketch_rows <= 65536, "sketch_rows must be in [1, 65536]");
  KRR_REQUIRE(zeta <= 64 && zeta <= sketch_rows, "zeta must be in [1, min(s, 64)]");
  KRR_REQUIRE((double)N * zeta < 2.0e9, "N * zeta too large");
  // centers: distinct and in range (checked on the host)
  std::vector<int64_t> hc(k);
  KRR_CUDA_TRY(cudaMemcpy(hc.data(), centers, sizeof(int64_t) * k, cudaMemcpyDefault));
  {
    std::vector<int64_t> sorted(hc);
    std::sort(sorted.begin(), sorted.end());
    for (int i = 0; i < k; ++i) {
      KRR_REQUIRE(sorted[i] >= 0 && sorted[i] < N, "center %lld out of range", (long long)sorted[i]);
      KRR_REQUIRE(i == 0 || sorted[i] != sorted[i - 1], "centers must be distinct");
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  krill_precond *P = new (std::nothrow) krill_precond();
  if (!P) return KRR_ENOMEM;
  P->N = N;
  P->d = d;
  P->kern = kern;
  P->sigma = sigma;
  P->k = k;
  P->s = sketch_rows;
  P->zeta = zeta;
  P->mu = mu;
  P->lambda = mu * (double)N;
  P->seed = seed;
  krr_status st = KRR_OK;
  auto fail = [&](krr_status e) {
    free_krill(P);
    return e;
  };
  if ((st = dev_alloc(&P->X, (size_t)N * d)) != KRR_OK) return fail(st);
  if (cudaMemcpyAsync(P->X, X, sizeof(double) * N * d, cudaMemcpyDefault, s) != cudaSuccess) {
    set_error("copy of X failed");
    return fail(KRR_ECUDA);
  }
  if ((st = dev_alloc(&P->S, (size_t)k)) != KRR_OK) return fail(st);
  if (cudaMemcpyAsync(P->S, hc.data(), sizeof(int64_t) * k, cudaMemcpyHostToDevice, s) !=
      cudaSuccess) {
    set_error("copy of centers failed");
    return fail(KRR_ECUDA);
  }
  if ((st = krill_build_device(P, s)) != KRR_OK) return fail(st);
  *P_out = P;
  return KRR_OK;
}

krr_status krill_export(const krill_precond *P, double *H, double *Bsk, double *Pm, double *Cu,
                        int *s_out) {
  clear_error();
  KRR_REQUIRE(P, "handle is NULL");
  const size_t kk = (size_t)P->k * P->k;
  if (H) KRR_CUDA_TRY(cudaMemcpy(H, P->H, sizeof(double) * kk, cudaMemcpyDefault));
  if (Bsk)
    KRR_CUDA_TRY(cudaMemcpy(Bsk, P->Bsk, sizeof(double) * (size_t)P->s * P->k, cudaMemcpyDefault));
  if (Pm) KRR_CUDA_TRY(cudaMemcpy(Pm, P->P, sizeof(double) * kk, cudaMemcpyDefault));
  if (Cu) {
    // upper factor C = L^T, column-major
    std::vector<double> L(kk), C(kk, 0.0);
    KRR_CUDA_TRY(cudaMemcpy(L.data(), P->L, sizeof(double) * kk, cudaMemcpyDeviceToHost));
    for (int j = 0; j < P->k; ++j)
      for (int i = 0; i <= j; ++i) C[i + (size_t)j * P->k] = L[j + (size_t)i * P->k];
    KRR_CUDA_TRY(cudaMemcpy(Cu, C.data(), sizeof(double) * kk, cudaMemcpyDefault));
  }
  if (s_out) *s_out = P->s;
  return KRR_OK;
}

krr_status krill_solve(const krill_precond *P, const double *Y, int m, double tol, int maxit,
                       double *beta_out, void *stream, krr_info *info) {
  clear_error();
  KRR_REQUIRE(P && Y && beta_out, "NULL argument");
  KRR_REQUIRE(m >= 1 && m <= 16, "m must be in [1, 16]");
  KRR_REQUIRE(tol > 0 && tol < 1, "tol must be in (0, 1)");
  if (maxit <= 0) maxit = 1000;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf<double> ty;
  const double *Yd;
  KRR_TRY(device_view(Y, (size_t)P->N * m, s, ty, &Yd));
  OutView<double> out;
  KRR_TRY(out.init(beta_out, (size_t)P->k * m, s));
  if (info) std::memset(info, 0, sizeof(*info));
  krr_status st = krill_solve_device(P, Yd, m, tol, maxit, out.dev, s, info);
  if (st != KRR_OK && st != KRR_ENOCONV) return st;
  KRR_TRY(tc5_check_fault(s));   // a bounded wait of a tensor-core product gave up
  krr_status st2 = out.finish(s);
  return st2 != KRR_OK ? st2 : st;
}

void krill_free(krill_precond *P) { free_krill(P); }

}  // extern "C"
