// C ABI of libpint (declarations and contracts in include/pint.h).
// Every entry point catches pint::Fail and converts it to a status code;
// nothing here aborts or prints.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstring>
#include <atomic>
#include <set>
#include <thread>

namespace pint {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

void* dalloc(Ctx* c, size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, std::max<size_t>(bytes, 16), c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Fail{PINT_ERR_OOM, std::string("device allocation of ") + std::to_string(bytes) + " bytes failed"};
  }
  c->allocs.push_back(p);
  return p;
}

void dfree(Ctx* c, void* p) {
  if (!p) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
  if (it != c->allocs.end()) {
    *it = c->allocs.back();
    c->allocs.pop_back();
  }
  cudaFreeAsync(p, c->stream);
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

const double* stage_in(Ctx* c, const double* p, size_t n, std::vector<void*>& tmp) {
  if (!p || is_device_ptr(p)) return p;
  double* d = (double*)dalloc(c, n * sizeof(double));
  tmp.push_back(d);
  PINT_CUDA(cudaMemcpyAsync(d, p, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  return d;
}

// output staging: device pointer used directly, host pointer through a temp
struct OutBuf {
  double* user = nullptr;
  double* dev = nullptr;
  size_t n = 0;
  bool host = false;
};
static OutBuf stage_out(Ctx* c, double* p, size_t n, std::vector<void*>& tmp) {
  OutBuf o;
  o.user = p;
  o.n = n;
  if (!p) return o;
  if (is_device_ptr(p)) {
    o.dev = p;
    return o;
  }
  o.host = true;
  o.dev = (double*)dalloc(c, n * sizeof(double));
  tmp.push_back(o.dev);
  return o;
}
static void finish_out(Ctx* c, const OutBuf& o) {
  if (o.host && o.user)
    PINT_CUDA(cudaMemcpyAsync(o.user, o.dev, o.n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
}
static void free_tmp(Ctx* c, std::vector<void*>& tmp) {
  for (void* p : tmp) dfree(c, p);
  tmp.clear();
}

template <typename F>
static pint_status guarded(Ctx* c, F&& f) {
  std::vector<void*> tmp;
  try {
    f(tmp);
    if (c) {
      free_tmp(c, tmp);
      PINT_CUDA(cudaStreamSynchronize(c->stream));
    }
    return PINT_OK;
  } catch (const Fail& e) {
    set_error(e.msg);
    if (c) {
      for (void* p : tmp) {
        auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
        if (it != c->allocs.end()) c->allocs.erase(it);
        cudaFreeAsync(p, c->stream);
      }
      cudaStreamSynchronize(c->stream);
    }
    return e.code;
  } catch (const std::exception& e) {
    set_error(std::string("host exception: ") + e.what());
    return PINT_ERR_BAD_ARG;
  }
}

// wall time of one setup stage (synchronised), accumulated into c->stage_ms[k]
template <typename F>
static void timed_stage(Ctx* c, int k, F&& f) {
  PINT_CUDA(cudaStreamSynchronize(c->stream));
  const auto t0 = std::chrono::steady_clock::now();
  f();
  PINT_CUDA(cudaStreamSynchronize(c->stream));
  c->stage_ms[k] += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Section 3.2: the splitting scheme is stable when
// Delta t lambda_max(A22, M22) <= 1 - gamma^2.  The final time picked for
// T <= 0 keeps 90% of that bound on the coarse step Delta t = T / N and is
// rounded down to two significant digits (so that it prints exactly).
static double stable_final_time(int N, double gamma, double lam22) {
  if (!(lam22 > 0) || !(gamma >= 0 && gamma < 1)) return 0.0;
  const double t = 0.9 * N * (1.0 - gamma * gamma) / lam22;
  if (!(t > 0) || !std::isfinite(t)) return 0.0;
  const double e = std::floor(std::log10(t)) - 1.0;
  const double scale = std::pow(10.0, e);
  return std::floor(t / scale) * scale;
}

static void fill_info(Ctx* c, pint_space_info* info, double ms) {
  if (!info) return;
  info->n_f = c->n_f;
  info->nc = c->nc;
  info->J = c->J;
  info->ell = c->ell;
  info->n_blocks = c->n_blocks;
  info->n_raw = c->n_raw;
  info->L = c->L;
  info->d1 = c->d1;
  info->d2 = c->d2;
  info->gamma = c->gamma;
  info->lambda_max22 = c->lam22;
  info->dt_max = c->dt_max;
  info->setup_ms = ms;
  info->T = c->have_time ? c->T : 0.0;
  info->Dt = c->have_time ? c->Dt : 0.0;
  info->dt = c->have_time ? c->dt : 0.0;
}

}  // namespace pint

using namespace pint;

extern "C" {

const char* pint_last_error(void) { return g_err.c_str(); }

pint_status pint_setup_fine_grid(pint_ctx** out, int n_f, const double* kappa_cells, void* stream) {
  if (!out) {
    set_error("out is NULL");
    return PINT_ERR_BAD_ARG;
  }
  *out = nullptr;
  if (n_f < 4 || n_f > 4096 || !kappa_cells) {
    set_error("n_f must be in [4, 4096] and kappa_cells non-NULL");
    return PINT_ERR_BAD_ARG;
  }
  Ctx* c = new Ctx();
  c->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    set_error("no CUDA device");
    return PINT_ERR_CUDA;
  }
  c->n_f = n_f;
  c->nn = (n_f + 1) * (n_f + 1);
  pint_status s = guarded(c, [&](std::vector<void*>& tmp) {
    size_t nk = (size_t)n_f * n_f;
    std::vector<double> hk(nk);
    if (is_device_ptr(kappa_cells)) {
      PINT_CUDA(cudaMemcpyAsync(hk.data(), kappa_cells, nk * 8, cudaMemcpyDeviceToHost, c->stream));
      PINT_CUDA(cudaStreamSynchronize(c->stream));
    } else {
      std::memcpy(hk.data(), kappa_cells, nk * 8);
    }
    for (double v : hk) PINT_REQUIRE(v > 0.0 && std::isfinite(v), PINT_ERR_BAD_ARG, "kappa must be finite and > 0");
    const double* dk = stage_in(c, kappa_cells, nk, tmp);
    build_fine(c, dk);
    c->have_grid = true;
  });
  if (s != PINT_OK) {
    pint_destroy((pint_ctx*)c);
    return s;
  }
  *out = (pint_ctx*)c;
  return PINT_OK;
}

pint_status pint_build_multiscale_spaces(pint_ctx* ctx, int nc, int J, int ell, pint_space_info* info) {
  Ctx* c = (Ctx*)ctx;
  if (!c) {
    set_error("ctx is NULL");
    return PINT_ERR_BAD_ARG;
  }
  return guarded(c, [&](std::vector<void*>&) {
    PINT_REQUIRE(c->have_grid, PINT_ERR_STATE, "pint_setup_fine_grid first");
    PINT_REQUIRE(!c->have_spaces, PINT_ERR_STATE, "spaces already built for this context");
    PINT_REQUIRE(nc >= 1 && c->n_f % nc == 0, PINT_ERR_BAD_ARG, "nc must divide n_f");
    PINT_REQUIRE(c->n_f / nc >= 2 && c->n_f / nc <= 48, PINT_ERR_BAD_ARG, "n_f/nc must be in [2, 48]");
    PINT_REQUIRE(J >= 0 && J <= 16, PINT_ERR_BAD_ARG, "J must be in [0, 16]");
    PINT_REQUIRE(ell >= 1 && ell <= 8, PINT_ERR_BAD_ARG, "ell must be in [1, 8]");
    cudaEvent_t e0, e1;
    PINT_CUDA(cudaEventCreate(&e0));
    PINT_CUDA(cudaEventCreate(&e1));
    PINT_CUDA(cudaEventRecord(e0, c->stream));
    c->nc = nc;
    c->J = J;
    c->ell = ell;
    c->bs = c->n_f / nc;
    c->nb = (c->bs + 1) * (c->bs + 1);
    c->n_blocks = nc * nc;
    timed_stage(c, 0, [&] { build_blocks(c); });
    timed_stage(c, 1, [&] { build_windows(c); });
    c->have_spaces = true;
    PINT_CUDA(cudaEventRecord(e1, c->stream));
    PINT_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    fill_info(c, info, ms);
  });
}

pint_status pint_assemble_reduced(pint_ctx* ctx, double T, int N, int P, double alpha, int precision,
                                  int flags, pint_space_info* info) {
  Ctx* c = (Ctx*)ctx;
  if (!c) {
    set_error("ctx is NULL");
    return PINT_ERR_BAD_ARG;
  }
  pint_status unstable = PINT_OK;
  pint_status s = guarded(c, [&](std::vector<void*>&) {
    PINT_REQUIRE(c->have_spaces, PINT_ERR_STATE, "pint_build_multiscale_spaces first");
    PINT_REQUIRE(std::isfinite(T), PINT_ERR_BAD_ARG, "T must be finite");
    PINT_REQUIRE(N >= 1 && N <= 4096, PINT_ERR_BAD_ARG, "N must be in [1, 4096]");
    PINT_REQUIRE(P >= 2 && P <= 64, PINT_ERR_BAD_ARG, "P must be in [2, 64]");
    PINT_REQUIRE(alpha > 0 && alpha < 1, PINT_ERR_BAD_ARG, "alpha must be in (0, 1)");
    PINT_REQUIRE(precision == PINT_FP64 || precision == PINT_MIXED || precision == PINT_MIXED_F32,
                 PINT_ERR_BAD_ARG, "unknown precision");
    PINT_REQUIRE(!(flags & PINT_CARRY_LAGS) || precision == PINT_FP64, PINT_ERR_BAD_ARG,
                 "PINT_CARRY_LAGS is an FP64 comparison mode");
    PINT_REQUIRE(!(flags & PINT_FINE_SEQUENTIAL) || precision == PINT_FP64, PINT_ERR_BAD_ARG,
                 "PINT_FINE_SEQUENTIAL is an FP64 comparison mode");
    // from here on the context's operators and time grid change: until this
    // call succeeds there is no time grid to solve on, and nothing derived
    // from the previous one (captured graphs, low-precision operator copies)
    // is reused
    c->have_time = false;
    c->graph_epoch++;
    cudaEvent_t e0, e1;
    PINT_CUDA(cudaEventCreate(&e0));
    PINT_CUDA(cudaEventCreate(&e1));
    PINT_CUDA(cudaEventRecord(e0, c->stream));
    if (!c->have_reduced) {
      timed_stage(c, 2, [&] { build_galerkin(c); });
      timed_stage(c, 3, [&] { build_reduced(c); });
      PINT_REQUIRE(c->d2 <= 4096, PINT_ERR_BAD_ARG, "dim V_H2 above 4096 (nc <= 63)");
      timed_stage(c, 4, [&] { build_spectral(c); });
      c->have_reduced = true;
    }
    if (T <= 0) T = stable_final_time(N, c->gamma, c->lam22);
    PINT_REQUIRE(T > 0 && std::isfinite(T), PINT_ERR_BAD_ARG,
                 "no stable final time: lambda_max(A22, M22) or gamma out of range");
    c->T = T;
    c->N = N;
    c->P = P;
    c->alpha = alpha;
    c->precision = precision;
    c->fine_seq = (flags & PINT_FINE_SEQUENTIAL) != 0;
    c->autotune = (flags & PINT_AUTOTUNE) != 0;
    c->coarse64 = (flags & PINT_COARSE_FP64) != 0;
    c->coarse_grid = (flags & PINT_COARSE_GRID) != 0;
    c->refine64 = (flags & PINT_REFINE_FP64) != 0;
    c->carry = (flags & PINT_CARRY_LAGS) != 0;
    c->adj_response = (flags & PINT_ADJOINT_RESPONSE) != 0;
    c->Dt = T / N;
    c->dt = c->Dt / P;
    timed_stage(c, 5, [&] { hot_prepare(c); });
    // graphs captured for the previous time grid hold its dt and alpha as
    // kernel arguments: never replay them after a re-assembly
    c->graph_epoch++;
    c->have_time = true;
    PINT_CUDA(cudaEventRecord(e1, c->stream));
    PINT_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    fill_info(c, info, ms);
    if (c->Dt > c->dt_max && !(flags & PINT_ALLOW_UNSTABLE)) unstable = PINT_ERR_UNSTABLE_DT;
  });
  if (s == PINT_OK && unstable != PINT_OK) {
    set_error("Delta t exceeds (1 - gamma^2) / lambda_max(A22, M22)");
    return unstable;
  }
  return s;
}

static pint_status solve_common(Ctx* c, const double* u0_nodes, const double* f_shape, const double* amp,
                                double eps, int k_max, double wr_tol, int wr_max, double* u_out,
                                double* coarse_out, pint_stats* stats, bool sequential) {
  if (!c) {
    set_error("ctx is NULL");
    return PINT_ERR_BAD_ARG;
  }
  if (stats) std::memset(stats, 0, sizeof(pint_stats));
  pint_status inner = PINT_OK;
  pint_status s = guarded(c, [&](std::vector<void*>& tmp) {
    PINT_REQUIRE(c->have_time, PINT_ERR_STATE, "pint_assemble_reduced first");
    PINT_REQUIRE(u0_nodes && f_shape, PINT_ERR_BAD_ARG, "u0_nodes and f_shape are required");
    PINT_REQUIRE(eps == eps && wr_tol == wr_tol, PINT_ERR_BAD_ARG, "eps and wr_tol must not be NaN");
    PINT_REQUIRE(k_max >= 1 && wr_max >= 1, PINT_ERR_BAD_ARG, "k_max and wr_max must be >= 1");
    const double* du0 = stage_in(c, u0_nodes, c->nn, tmp);
    const double* df = stage_in(c, f_shape, c->nn, tmp);
    const double* da = stage_in(c, amp, c->N, tmp);
    OutBuf ou = stage_out(c, u_out, (size_t)c->N * c->nn, tmp);
    OutBuf oc = stage_out(c, coarse_out, (size_t)(c->N + 1) * (c->d1 + c->d2), tmp);
    try {
      if (c->carry)
        solve_carry(c, du0, df, da, eps, k_max, ou.dev, oc.dev, stats, sequential);
      else if (c->precision != PINT_FP64 && !sequential)
        solve_mixed(c, du0, df, da, eps, k_max, wr_tol, wr_max, ou.dev, oc.dev, stats, 1);
      else
        solve_fp64(c, du0, df, da, eps, k_max, wr_tol, wr_max, ou.dev, oc.dev, stats, sequential);
    } catch (const Fail& f) {
      if (f.code != PINT_ERR_NOT_CONVERGED) throw;
      inner = f.code;
      set_error(f.msg);
    }
    finish_out(c, ou);
    finish_out(c, oc);
  });
  return s != PINT_OK ? s : inner;
}

pint_status pint_parareal_solve(pint_ctx* ctx, const double* u0_nodes, const double* f_shape,
                                const double* amp, double eps, int k_max, double wr_tol, int wr_max,
                                double* u_out, double* coarse_out, pint_stats* stats) {
  return solve_common((Ctx*)ctx, u0_nodes, f_shape, amp, eps, k_max, wr_tol, wr_max, u_out, coarse_out,
                      stats, false);
}

pint_status pint_batch_solve(pint_batch_item* items, int count, int workers) {
  if (count < 0 || (count > 0 && !items)) {
    set_error("items required, count >= 0");
    return PINT_ERR_BAD_ARG;
  }
  std::set<pint_ctx*> seen;
  for (int i = 0; i < count; ++i) {
    if (!items[i].ctx || !seen.insert(items[i].ctx).second) {
      set_error("item " + std::to_string(i) + ": NULL or repeated context");
      return PINT_ERR_BAD_ARG;
    }
  }
  if (count == 0) return PINT_OK;
  // longest first: fine unknowns x N x P (0 for a context without a time grid)
  std::vector<int> order(count);
  std::vector<double> work(count);
  for (int i = 0; i < count; ++i) {
    const Ctx* c = (const Ctx*)items[i].ctx;
    order[i] = i;
    work[i] = c->have_time ? (double)c->nn * c->N * c->P : 0.0;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
  if (workers <= 0) workers = std::min(count, 16);
  workers = std::min(workers, count);
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<std::string> msg(count);
  std::atomic<int> next{0};
  auto run = [&]() {
    cudaSetDevice(dev);
    for (int j = next.fetch_add(1); j < count; j = next.fetch_add(1)) {
      pint_batch_item& it = items[order[j]];
      it.status = pint_parareal_solve(it.ctx, it.u0_nodes, it.f_shape, it.amp, it.eps, it.k_max, it.wr_tol,
                                      it.wr_max, it.u_out, it.coarse_out, it.stats);
      if (it.status != PINT_OK) msg[order[j]] = pint_last_error();
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < workers; ++w) pool.emplace_back(run);
  run();  // the calling thread is one of the workers
  for (auto& t : pool) t.join();
  pint_status first = PINT_OK;
  int where = -1;
  for (int i = 0; i < count; ++i) {
    const pint_status s = items[i].status;
    if (s == PINT_OK) continue;
    if (first == PINT_OK || (first == PINT_ERR_NOT_CONVERGED && s != PINT_ERR_NOT_CONVERGED)) {
      first = s;
      where = i;
    }
  }
  if (where >= 0) set_error("item " + std::to_string(where) + ": " + msg[where]);
  return first;
}

pint_status pint_sequential_solve(pint_ctx* ctx, const double* u0_nodes, const double* f_shape,
                                  const double* amp, double* u_out, double* coarse_out) {
  return solve_common((Ctx*)ctx, u0_nodes, f_shape, amp, 0.0, 1, 0.0, 1, u_out, coarse_out, nullptr, true);
}

pint_status pint_adjoint(pint_ctx* ctx, const int* obs_nodes, int n_obs, const double* data,
                         const double* u0_nodes, const double* f_shape, const double* amp, double eps,
                         int k_max, double wr_tol, int wr_max, double* misfit, double* grad_u0,
                         double* grad_amp) {
  Ctx* c = (Ctx*)ctx;
  if (!c) {
    set_error("ctx is NULL");
    return PINT_ERR_BAD_ARG;
  }
  return guarded(c, [&](std::vector<void*>& tmp) {
    PINT_REQUIRE(c->have_time, PINT_ERR_STATE, "pint_assemble_reduced first");
    PINT_REQUIRE(obs_nodes && n_obs >= 1 && data && u0_nodes && f_shape, PINT_ERR_BAD_ARG,
                 "obs_nodes, n_obs >= 1, data, u0_nodes and f_shape are required");
    PINT_REQUIRE(eps >= 0 && wr_tol >= 0 && k_max >= 1 && wr_max >= 1, PINT_ERR_BAD_ARG,
                 "eps, wr_tol >= 0 and k_max, wr_max >= 1");
    // observation node ids: checked on the host, used on the device
    std::vector<int> h_obs(n_obs);
    const bool obs_dev = is_device_ptr(obs_nodes);
    if (obs_dev)
      PINT_CUDA(cudaMemcpyAsync(h_obs.data(), obs_nodes, (size_t)n_obs * 4, cudaMemcpyDeviceToHost, c->stream));
    else
      std::memcpy(h_obs.data(), obs_nodes, (size_t)n_obs * 4);
    PINT_CUDA(cudaStreamSynchronize(c->stream));
    for (int o = 0; o < n_obs; ++o)
      PINT_REQUIRE(h_obs[o] >= 0 && h_obs[o] < c->nn, PINT_ERR_BAD_ARG, "observation node id out of range");
    int* d_obs = (int*)dalloc(c, (size_t)n_obs * 4);
    tmp.push_back(d_obs);
    PINT_CUDA(cudaMemcpyAsync(d_obs, h_obs.data(), (size_t)n_obs * 4, cudaMemcpyHostToDevice, c->stream));
    const double* dd = stage_in(c, data, (size_t)c->N * n_obs, tmp);
    const double* du0 = stage_in(c, u0_nodes, c->nn, tmp);
    const double* df = stage_in(c, f_shape, c->nn, tmp);
    const double* da = stage_in(c, amp, c->N, tmp);
    OutBuf og = stage_out(c, grad_u0, c->nn, tmp);
    OutBuf oa = stage_out(c, grad_amp, c->N, tmp);
    adjoint_solve(c, d_obs, n_obs, dd, du0, df, da, eps, k_max, wr_tol, wr_max, misfit, og.dev, oa.dev);
    finish_out(c, og);
    finish_out(c, oa);
    PINT_CUDA(cudaStreamSynchronize(c->stream));
  });
}

pint_status pint_get_reduced(pint_ctx* ctx, int which, double* out, const double* aux) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !out) {
    set_error("ctx and out are required");
    return PINT_ERR_BAD_ARG;
  }
  return guarded(c, [&](std::vector<void*>& tmp) {
    PINT_REQUIRE(c->have_reduced, PINT_ERR_STATE, "pint_assemble_reduced first");
    const int d1 = c->d1, d2 = c->d2;
    const double* src = nullptr;
    size_t n = 0;
    switch (which) {
      case 0: src = c->M11; n = (size_t)d1 * d1; break;
      case 1: src = c->A11; n = (size_t)d1 * d1; break;
      case 2: src = c->M22; n = (size_t)d2 * d2; break;
      case 3: src = c->A22; n = (size_t)d2 * d2; break;
      case 4: src = c->M12; n = (size_t)d1 * d2; break;
      case 5: src = c->A12; n = (size_t)d1 * d2; break;
      case 7: src = c->GM; n = (size_t)c->n_raw * c->n_raw; break;
      case 6: {
        PINT_REQUIRE(aux, PINT_ERR_BAD_ARG, "which = 6 needs f_shape in aux");
        const double* df = stage_in(c, aux, c->nn, tmp);
        double* nodes = (double*)dalloc(c, (size_t)c->nn * 8);
        double* raw = (double*)dalloc(c, (size_t)c->n_raw * 8);
        double* v = (double*)dalloc(c, (size_t)(d1 + d2) * 8);
        tmp.push_back(nodes);
        tmp.push_back(raw);
        tmp.push_back(v);
        apply_stencil(c, c->stM, df, nodes, 1);
        raw_dot(c, nodes, 1, raw);
        to_reduced(c, raw, 1, v, v + d1);
        src = v;
        n = (size_t)(d1 + d2);
        break;
      }
      case 9: {  // setup stage wall times, ms (6 doubles)
        if (is_device_ptr(out))
          PINT_CUDA(cudaMemcpyAsync(out, c->stage_ms, sizeof(c->stage_ms), cudaMemcpyHostToDevice, c->stream));
        else
          std::memcpy(out, c->stage_ms, sizeof(c->stage_ms));
        PINT_CUDA(cudaStreamSynchronize(c->stream));
        return;
      }
      case 8: {
        std::vector<double> h(2 * (size_t)c->n_raw);
        for (int r = 0; r < c->n_raw; ++r) {
          h[2 * r] = c->kind[r];
          h[2 * r + 1] = c->owner[r];
        }
        if (is_device_ptr(out))
          PINT_CUDA(cudaMemcpyAsync(out, h.data(), h.size() * 8, cudaMemcpyHostToDevice, c->stream));
        else
          std::memcpy(out, h.data(), h.size() * 8);
        PINT_CUDA(cudaStreamSynchronize(c->stream));
        return;
      }
      default: PINT_REQUIRE(false, PINT_ERR_BAD_ARG, "unknown quantity");
    }
    PINT_CUDA(cudaMemcpyAsync(out, src, n * 8, cudaMemcpyDefault, c->stream));
    PINT_CUDA(cudaStreamSynchronize(c->stream));
  });
}

pint_status pint_prolong(pint_ctx* ctx, const double* coarse, int count, double* u_out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !coarse || !u_out || count < 1) {
    set_error("ctx, coarse, u_out and count >= 1 are required");
    return PINT_ERR_BAD_ARG;
  }
  return guarded(c, [&](std::vector<void*>& tmp) {
    PINT_REQUIRE(c->have_reduced, PINT_ERR_STATE, "pint_assemble_reduced first");
    const int d1 = c->d1, d2 = c->d2;
    const double* dc = stage_in(c, coarse, (size_t)count * (d1 + d2), tmp);
    double* u = (double*)dalloc(c, (size_t)count * d1 * 8);
    double* w = (double*)dalloc(c, (size_t)count * d2 * 8);
    tmp.push_back(u);
    tmp.push_back(w);
    PINT_CUDA(cudaMemcpy2DAsync(u, (size_t)d1 * 8, dc, (size_t)(d1 + d2) * 8, (size_t)d1 * 8, count,
                                cudaMemcpyDeviceToDevice, c->stream));
    PINT_CUDA(cudaMemcpy2DAsync(w, (size_t)d2 * 8, dc + d1, (size_t)(d1 + d2) * 8, (size_t)d2 * 8, count,
                                cudaMemcpyDeviceToDevice, c->stream));
    OutBuf o = stage_out(c, u_out, (size_t)count * c->nn, tmp);
    prolong_coeffs(c, u, w, count, o.dev);
    finish_out(c, o);
  });
}

pint_status pint_apply_G(pint_ctx* ctx, const double* in, int count, const double* f_shape, const double* amp,
                         double* out) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !in || !out || !f_shape || count < 1) {
    set_error("ctx, in, out, f_shape and count >= 1 are required");
    return PINT_ERR_BAD_ARG;
  }
  return guarded(c, [&](std::vector<void*>& tmp) {
    PINT_REQUIRE(c->have_time, PINT_ERR_STATE, "pint_assemble_reduced first");
    PINT_REQUIRE(count <= c->N, PINT_ERR_BAD_ARG, "count must be <= N");
    const size_t d = c->d1 + c->d2;
    const double* di = stage_in(c, in, count * d, tmp);
    const double* df = stage_in(c, f_shape, c->nn, tmp);
    const double* da = stage_in(c, amp, count, tmp);
    OutBuf o = stage_out(c, out, count * d, tmp);
    apply_G_dev(c, di, count, df, da, o.dev);
    finish_out(c, o);
  });
}

pint_status pint_apply_F(pint_ctx* ctx, const double* in, int count, const double* f_shape, const double* amp,
                         double wr_tol, int wr_max, double* out, int* wr_iters) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !in || !out || !f_shape || count < 1 || wr_max < 1) {
    set_error("ctx, in, out, f_shape, count >= 1 and wr_max >= 1 are required");
    return PINT_ERR_BAD_ARG;
  }
  return guarded(c, [&](std::vector<void*>& tmp) {
    PINT_REQUIRE(c->have_time, PINT_ERR_STATE, "pint_assemble_reduced first");
    PINT_REQUIRE(count <= c->N, PINT_ERR_BAD_ARG, "count must be <= N");
    const size_t d = c->d1 + c->d2;
    const double* di = stage_in(c, in, count * d, tmp);
    const double* df = stage_in(c, f_shape, c->nn, tmp);
    const double* da = stage_in(c, amp, count, tmp);
    OutBuf o = stage_out(c, out, count * d, tmp);
    apply_F_dev(c, di, count, df, da, wr_tol, wr_max, o.dev, wr_iters);
    finish_out(c, o);
  });
}

int pint_set_wait_limit(int spins) {
  const int old = wait_limit();
  set_wait_limit(spins);
  return old;
}

int pint_set_sweep_smem(int bytes) {
  const int old = sweep_smem();
  set_sweep_smem(bytes);
  return old;
}

int pint_tuning_count(void) { return umma_tuning_count(); }

pint_status pint_tuning_get(int* rows, float* us, int cap, int* count) {
  if (!rows || !count || cap < 0) {
    set_error("rows and count are required, cap >= 0");
    return PINT_ERR_BAD_ARG;
  }
  *count = umma_tuning_get(rows, us, cap);
  return PINT_OK;
}

pint_status pint_tuning_set(const int* rows, const float* us, int count) {
  if (count < 0 || (count > 0 && !rows)) {
    set_error("rows required, count >= 0");
    return PINT_ERR_BAD_ARG;
  }
  const int bad = umma_tuning_set(rows, us, count);
  if (bad >= 0) {
    set_error("tuning row " + std::to_string(bad) + " is not a valid (M, Kp, ncols, maxs, tn, s, pair)");
    return PINT_ERR_BAD_ARG;
  }
  return PINT_OK;
}

pint_status pint_tuning_clear(void) {
  umma_tuning_clear();
  return PINT_OK;
}

pint_status pint_get_info(pint_ctx* ctx, pint_space_info* info) {
  Ctx* c = (Ctx*)ctx;
  if (!c || !info) {
    set_error("ctx and info are required");
    return PINT_ERR_BAD_ARG;
  }
  fill_info(c, info, 0.0);
  return PINT_OK;
}

pint_status pint_destroy(pint_ctx* ctx) {
  Ctx* c = (Ctx*)ctx;
  if (!c) return PINT_OK;
  cudaStreamSynchronize(c->stream);
  for (void* p : c->allocs) cudaFreeAsync(p, c->stream);
  cudaStreamSynchronize(c->stream);
  hot_release(c);
  mixed_release(c);
  adjoint_release(c);
  delete c;
  cudaGetLastError();
  return PINT_OK;
}

}  // extern "C"
