// Adjoint (backward) parareal for an observation misfit.
//
// The paper does not treat differentiation.  The gradient is that of the map
// Algorithm 1 converges to (the fine scheme of eqs. (2.4)-(2.5) interval
// after interval, lags restarted at each coarse boundary), which is affine in
// the initial value and the per-interval source amplitudes:
//   x_0 = M_H^-1 [Psi1 Psi2]^T M_f u0,   x_{n+1} = Phi x_n + a_n s.
// For J = 1/2 sum_{n=1..N} ||O x_n - d_n||^2 (O: the prolongation at the
// observation nodes) the adjoint states solve the backward recurrence
//   lambda_N = O^T r_N,  lambda_n = Phi^T lambda_{n+1} + O^T r_n,  lambda_0 = Phi^T lambda_1,
// and dJ/da_n = <lambda_{n+1}, s>, dJ/du0 = M_f [Psi1 Psi2] M_H^-1 lambda_0.
//
// The recurrence is solved by parareal run backwards in time with the
// transposed propagators: Phi^T (the fine scheme's P steps transposed, on all
// intervals at once) and G^T (one transposed coarse step), with the update
//   lambda_n^{k+1} = G^T lambda_{n+1}^{k+1} + Phi^T lambda_{n+1}^k - G^T lambda_{n+1}^k + O^T r_n.
// At k = N it equals the backward recurrence exactly.  The only forward data
// the adjoint needs are the coarse states x_n (the checkpoints at the coarse
// boundaries): the map is linear, so nothing inside an interval is stored.
//
// Everything runs in the spectral coordinates of the forward solve
// (u = Q u~, w = Q2 w~).  One step of the scheme there, h = dt or Dt,
//   u1 = D (u - CM (w - wl) - h CA w + h F1),        D = (1 + h Lambda1)^-1
//   w1 = (1 - h Lambda2) w - CM^T (u - ul) - h CA^T u1 + h F2,
// has, for adjoint outputs (alpha, beta) of (u1, w1) and (gamma, delta) of
// the lag outputs (ul' = u, wl' = w), the adjoint inputs
//   a^ = D (alpha - h CA beta)
//   adj u  = a^ - CM beta + gamma,         adj ul = CM beta,
//   adj w  = -(CM + h CA)^T a^ + (1 - h Lambda2) beta + delta,   adj wl = CM^T a^.
// The interval start maps x to (u, w, u, w), so adj x = (adj u + adj ul, adj w + adj wl).
// T = double on the FP64 path, float on the low-precision path.
//
// Amplitude gradient, two routes.  Default: the fine adjoint is recomputed
// inside each interval from the boundary adjoint lambda_{n+1} (the coarse
// checkpoints), stepping the transposed fine scheme P times on all intervals
// at once, and dJ/da_n = sum_{p=0..P-1} <mu_p, c> with mu_0 = (lambda_{n+1}, 0),
// mu_{p+1} = S^T mu_p (S the one-step map) and c the step's source term for
// a unit amplitude from a zero state.  PINT_ADJOINT_RESPONSE: the shortcut
// <lambda_{n+1}, s> with s the interval's response to the unit source (equal
// in exact arithmetic: s = sum_p S^p c).
#include "common.cuh"

#include <algorithm>
#include <cmath>

namespace pint {

namespace {

inline unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// u rows (warp per row i) of one transposed step for column v = blockIdx.y:
// al <- adj u, ga <- adj ul, aD <- a^ (rows [cols][d1])
template <typename T>
__global__ void k_adjT_u(const T* __restrict__ CA, const T* __restrict__ CM, int d1, int d2,
                         const T* __restrict__ lam1, T h, T* __restrict__ al, const T* __restrict__ be,
                         T* __restrict__ ga, T* __restrict__ aD) {
  const int v = blockIdx.y;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= d1) return;
  const T* b = be + (size_t)v * d2;
  T tA = 0, tM = 0;
  for (int j = lane; j < d2; j += 32) {
    const T bj = b[j];
    tA += CA[(size_t)i * d2 + j] * bj;
    tM += CM[(size_t)i * d2 + j] * bj;
  }
  for (int o = 16; o > 0; o >>= 1) {
    tA += __shfl_xor_sync(0xffffffffu, tA, o);
    tM += __shfl_xor_sync(0xffffffffu, tM, o);
  }
  if (lane == 0) {
    const size_t k = (size_t)v * d1 + i;
    const T ah = (al[k] - h * tA) / (T(1) + h * lam1[i]);
    aD[k] = ah;
    al[k] = ah - tM + ga[k];
    ga[k] = tM;
  }
}

// w rows (warp per row j): be <- adj w, de <- adj wl
template <typename T>
__global__ void k_adjT_w(const T* __restrict__ CMt, const T* __restrict__ CAt, int d1, int d2,
                         const T* __restrict__ lam2, T h, T* __restrict__ be, T* __restrict__ de,
                         const T* __restrict__ aD) {
  const int v = blockIdx.y;
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (j >= d2) return;
  const T* a = aD + (size_t)v * d1;
  T s1 = 0, s2 = 0;
  for (int i = lane; i < d1; i += 32) {
    const T ai = a[i];
    s1 += CMt[(size_t)j * d1 + i] * ai;
    s2 += CAt[(size_t)j * d1 + i] * ai;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) {
    const size_t k = (size_t)v * d2 + j;
    be[k] = -s1 - h * s2 + (T(1) - h * lam2[j]) * be[k] + de[k];
    de[k] = s1;
  }
}

// start of a transposed sweep: (alpha, beta) = lambda rows, (gamma, delta) = 0
template <typename T>
__global__ void k_adj_load(const double* __restrict__ lu, const double* __restrict__ lw, int d1, int d2,
                           int cols, T* __restrict__ al, T* __restrict__ be, T* __restrict__ ga,
                           T* __restrict__ de) {
  const long long n1 = (long long)cols * d1, n2 = (long long)cols * d2;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n1 + n2;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < n1) {
      al[e] = (T)lu[e];
      ga[e] = 0;
    } else {
      be[e - n1] = (T)lw[e - n1];
      de[e - n1] = 0;
    }
  }
}

// end of a transposed sweep (interval start x -> (u, w, u, w)):
// out = (al + ga, be + de)
template <typename T>
__global__ void k_adj_store(const T* __restrict__ al, const T* __restrict__ be, const T* __restrict__ ga,
                            const T* __restrict__ de, int d1, int d2, int cols, double* __restrict__ ou,
                            double* __restrict__ ow) {
  const long long n1 = (long long)cols * d1, n2 = (long long)cols * d2;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n1 + n2;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < n1)
      ou[e] = (double)al[e] + (double)ga[e];
    else
      ow[e - n1] = (double)be[e - n1] + (double)de[e - n1];
  }
}

// acc[v] += <(al, be)_v, (cu, cw)> for every column v (block per column): one
// term of the recomputed amplitude gradient (the lag parts of c are zero)
template <typename T>
__global__ void k_amp_acc(const T* __restrict__ al, const T* __restrict__ be, const double* __restrict__ cu,
                          const double* __restrict__ cw, int d1, int d2, double* __restrict__ acc) {
  __shared__ double sh[64];
  const int v = blockIdx.x;
  const T* a = al + (size_t)v * d1;
  const T* b = be + (size_t)v * d2;
  double s = 0.0;
  for (int e = threadIdx.x; e < d1 + d2; e += blockDim.x)
    s += (e < d1) ? (double)a[e] * cu[e] : (double)b[e - d1] * cw[e - d1];
  s = pintd::block_sum(s, sh);
  if (threadIdx.x == 0) acc[v] += s;
}

// nodal indicators of the observation nodes, [n_obs][nn]
__global__ void k_indicators(const int* __restrict__ obs, int n_obs, int nn, double* __restrict__ E) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)n_obs * nn;
       e += (long long)gridDim.x * blockDim.x) {
    const int o = (int)(e / nn), k = (int)(e % nn);
    E[e] = (k == obs[o]) ? 1.0 : 0.0;
  }
}

// R <- R - data, and J += 1/2 sum R^2 (one double atomic per block)
__global__ void k_resid(double* __restrict__ R, const double* __restrict__ data, long long n,
                        double* __restrict__ J) {
  __shared__ double sh[64];
  double s = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double r = R[e] - data[e];
    R[e] = r;
    s += r * r;
  }
  s = pintd::block_sum(s, sh);
  if (threadIdx.x == 0) atomicAdd(J, 0.5 * s);
}

// parareal update of the backward sweep at time n:
// lam_n = g + Fh - Gold + src (first sweep: g + src); Gold <- g; jump^2 partial
__global__ void k_adj_update(const double* __restrict__ gu, const double* __restrict__ gw,
                             const double* __restrict__ fu, const double* __restrict__ fw,
                             double* __restrict__ Gu, double* __restrict__ Gw, const double* __restrict__ su,
                             const double* __restrict__ sw, double* __restrict__ lu, double* __restrict__ lw,
                             int d1, int d2, int first, double* __restrict__ jump2) {
  __shared__ double sh[64];
  double s = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d1 + d2; e += gridDim.x * blockDim.x) {
    if (e < d1) {
      const double g = gu[e];
      double v = first ? g : g + fu[e] - Gu[e];
      if (su) v += su[e];
      const double dv = v - lu[e];
      s += dv * dv;
      lu[e] = v;
      Gu[e] = g;
    } else {
      const int j = e - d1;
      const double g = gw[j];
      double v = first ? g : g + fw[j] - Gw[j];
      if (sw) v += sw[j];
      const double dv = v - lw[j];
      s += dv * dv;
      lw[j] = v;
      Gw[j] = g;
    }
  }
  s = pintd::block_sum(s, sh);
  if (threadIdx.x == 0) atomicAdd(jump2, s);
}

// dJ/da_n = <lambda_{n+1}, s> (block per n)
__global__ void k_amp_grad(const double* __restrict__ lu, const double* __restrict__ lw,
                           const double* __restrict__ su, const double* __restrict__ sw, int d1, int d2,
                           double* __restrict__ g) {
  __shared__ double sh[64];
  const int n = blockIdx.x;
  const double* a = lu + (size_t)(n + 1) * d1;
  const double* b = lw + (size_t)(n + 1) * d2;
  double s = 0.0;
  for (int e = threadIdx.x; e < d1 + d2; e += blockDim.x) s += (e < d1) ? a[e] * su[e] : b[e - d1] * sw[e - d1];
  s = pintd::block_sum(s, sh);
  if (threadIdx.x == 0) g[n] = s;
}

__global__ void k_norm2_rows(const double* __restrict__ lu, const double* __restrict__ lw, int d1, int d2,
                             double* __restrict__ out) {
  __shared__ double sh[64];
  const int n = blockIdx.x;
  double s = 0.0;
  for (int e = threadIdx.x; e < d1 + d2; e += blockDim.x) {
    const double v = (e < d1) ? lu[(size_t)n * d1 + e] : lw[(size_t)n * d2 + e - d1];
    s += v * v;
  }
  s = pintd::block_sum(s, sh);
  if (threadIdx.x == 0) out[n] = s;
}

template <typename T>
__global__ void k_cast(const double* __restrict__ x, long long n, T* __restrict__ y) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] = (T)x[e];
}

struct Adj {
  int N = 0, d1 = 0, d2 = 0, n_obs = 0, prec = -1;
  std::vector<void*> bufs;
  // observation operator, residuals, sources
  double *E = nullptr, *raw = nullptr, *t1 = nullptr, *t2 = nullptr, *Ou = nullptr, *Ow = nullptr;
  double *R = nullptr, *gu = nullptr, *gw = nullptr, *red = nullptr;
  // adjoint states and parareal bookkeeping (rows n = 0..N)
  double *Lu = nullptr, *Lw = nullptr, *Fu = nullptr, *Fw = nullptr, *Gu = nullptr, *Gw = nullptr;
  double *cu = nullptr, *cw = nullptr, *su = nullptr, *sw = nullptr, *yu = nullptr, *yw = nullptr;
  double *xu = nullptr, *xw = nullptr, *nodes = nullptr;
  // transposed-sweep work arrays (T), N columns
  void *al = nullptr, *be = nullptr, *ga = nullptr, *de = nullptr, *aD = nullptr;
  // couplings and spectra in T (float copies on the low-precision path)
  void *CA = nullptr, *CM = nullptr, *CAt = nullptr, *CMt = nullptr, *l1 = nullptr, *l2 = nullptr;
};

Adj& adj_get(Ctx* c, int n_obs) {
  if (!c->adj) c->adj = new Adj();
  Adj& A = *reinterpret_cast<Adj*>(c->adj);
  const int N = c->N, d1 = c->d1, d2 = c->d2, prec = c->precision == PINT_FP64 ? 0 : 1;
  if (A.N == N && A.d1 == d1 && A.d2 == d2 && A.n_obs == n_obs && A.prec == prec) return A;
  for (void* b : A.bufs) dfree(c, b);
  A = Adj();
  A.N = N;
  A.d1 = d1;
  A.d2 = d2;
  A.n_obs = n_obs;
  A.prec = prec;
  auto D = [&](size_t n) {
    A.bufs.push_back(dalloc(c, std::max<size_t>(n, 1) * 8));
    return (double*)A.bufs.back();
  };
  const size_t ts = prec ? 4 : 8;
  auto Tb = [&](size_t n) {
    A.bufs.push_back(dalloc(c, std::max<size_t>(n, 1) * ts));
    return A.bufs.back();
  };
  A.E = D((size_t)n_obs * c->nn);
  A.raw = D((size_t)n_obs * c->n_raw);
  A.t1 = D((size_t)n_obs * d1);
  A.t2 = D((size_t)n_obs * d2);
  A.Ou = D((size_t)n_obs * d1);
  A.Ow = D((size_t)n_obs * d2);
  A.R = D((size_t)N * n_obs);
  A.gu = D((size_t)N * d1);
  A.gw = D((size_t)N * d2);
  A.red = D(2 * (size_t)N + 8);
  A.Lu = D((size_t)(N + 1) * d1);
  A.Lw = D((size_t)(N + 1) * d2);
  A.Fu = D((size_t)N * d1);
  A.Fw = D((size_t)N * d2);
  A.Gu = D((size_t)N * d1);
  A.Gw = D((size_t)N * d2);
  A.cu = D(d1);
  A.cw = D(d2);
  A.su = D(d1);
  A.sw = D(d2);
  A.yu = D(d1);
  A.yw = D(d2);
  A.xu = D(d1);
  A.xw = D(d2);
  A.nodes = D(c->nn);
  A.al = Tb((size_t)N * d1);
  A.ga = Tb((size_t)N * d1);
  A.aD = Tb((size_t)N * d1);
  A.be = Tb((size_t)N * d2);
  A.de = Tb((size_t)N * d2);
  if (prec) {
    A.CA = Tb((size_t)d1 * d2);
    A.CM = Tb((size_t)d1 * d2);
    A.CAt = Tb((size_t)d1 * d2);
    A.CMt = Tb((size_t)d1 * d2);
    A.l1 = Tb(d1);
    A.l2 = Tb(d2);
  }
  return A;
}

// out rows = Phi^T (or G^T with one step) of the `cols` rows of (lu, lw)
// (acc, cu, cw given: acc[v] += <mu_p, c> before each step p, see above)
template <typename T>
void transposed_sweep(Ctx* c, Adj& A, const T* CA, const T* CM, const T* CAt, const T* CMt, const T* l1,
                      const T* l2, const double* lu, const double* lw, int cols, int steps, double h, double* ou,
                      double* ow, double* acc = nullptr, const double* cu = nullptr, const double* cw = nullptr) {
  const int d1 = c->d1, d2 = c->d2;
  T *al = (T*)A.al, *be = (T*)A.be, *ga = (T*)A.ga, *de = (T*)A.de, *aD = (T*)A.aD;
  const long long tot = (long long)cols * (d1 + d2);
  k_adj_load<T><<<std::min(nb(tot, 256), 4096u), 256, 0, c->stream>>>(lu, lw, d1, d2, cols, al, be, ga, de);
  for (int p = 0; p < steps; ++p) {
    if (acc) {
      k_amp_acc<T><<<cols, 256, 0, c->stream>>>(al, be, cu, cw, d1, d2, acc);
      c->launches++;
    }
    k_adjT_u<T><<<dim3(nb((long long)d1 * 32, 256), cols), 256, 0, c->stream>>>(CA, CM, d1, d2, l1, (T)h, al, be,
                                                                                 ga, aD);
    k_adjT_w<T><<<dim3(nb((long long)d2 * 32, 256), cols), 256, 0, c->stream>>>(CMt, CAt, d1, d2, l2, (T)h, be,
                                                                                 de, aD);
  }
  k_adj_store<T><<<std::min(nb(tot, 256), 4096u), 256, 0, c->stream>>>(al, be, ga, de, d1, d2, cols, ou, ow);
  PINT_LAUNCH_CHECK();
  c->launches += 2 + 2 * steps;
}

template <typename T>
void backward_parareal(Ctx* c, Adj& A, const T* CA, const T* CM, const T* CAt, const T* CMt, const T* l1,
                       const T* l2, int k_max, double rel_tol) {
  const int N = c->N, d1 = c->d1, d2 = c->d2, P = c->P;
  auto Lu = [&](int n) { return A.Lu + (size_t)n * d1; };
  auto Lw = [&](int n) { return A.Lw + (size_t)n * d2; };
  // sources O^T r_n for n = 1..N are rows n-1 of (gu, gw); none at n = 0
  auto src_u = [&](int n) { return n >= 1 ? A.gu + (size_t)(n - 1) * d1 : nullptr; };
  auto src_w = [&](int n) { return n >= 1 ? A.gw + (size_t)(n - 1) * d2 : nullptr; };
  const unsigned ub = nb(d1 + d2, 256);
  PINT_CUDA(cudaMemsetAsync(A.Lu, 0, (size_t)(N + 1) * d1 * 8, c->stream));
  PINT_CUDA(cudaMemsetAsync(A.Lw, 0, (size_t)(N + 1) * d2 * 8, c->stream));
  // k = 0: lambda_N = O^T r_N, then G^T sweep downwards
  PINT_CUDA(cudaMemcpyAsync(Lu(N), src_u(N), d1 * 8, cudaMemcpyDeviceToDevice, c->stream));
  PINT_CUDA(cudaMemcpyAsync(Lw(N), src_w(N), d2 * 8, cudaMemcpyDeviceToDevice, c->stream));
  for (int n = N - 1; n >= 0; --n) {
    transposed_sweep<T>(c, A, CA, CM, CAt, CMt, l1, l2, Lu(n + 1), Lw(n + 1), 1, 1, c->Dt, A.cu, A.cw);
    k_adj_update<<<ub, 256, 0, c->stream>>>(A.cu, A.cw, nullptr, nullptr, A.Gu + (size_t)n * d1,
                                            A.Gw + (size_t)n * d2, src_u(n), src_w(n), Lu(n), Lw(n), d1, d2, 1,
                                            A.red + 2 * N);
  }
  PINT_LAUNCH_CHECK();
  // scale of the adjoint states for the relative stopping test
  k_norm2_rows<<<N + 1, 256, 0, c->stream>>>(A.Lu, A.Lw, d1, d2, A.red);
  std::vector<double> nr(N + 1);
  PINT_CUDA(cudaMemcpyAsync(nr.data(), A.red, (N + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
  PINT_CUDA(cudaStreamSynchronize(c->stream));
  double scale = 0.0;
  for (double v : nr) scale = std::max(scale, std::sqrt(v));
  const double tol = rel_tol * std::max(scale, 1e-300);
  const int kcap = std::min(k_max, N);
  for (int k = 1; k <= kcap; ++k) {
    // Phi^T on the intervals whose input can still change: n = 0..N-k
    // (lambda_{n+1} is exact for n + 1 > N - k + 1 after sweep k - 1)
    const int nact = N - k + 1;
    transposed_sweep<T>(c, A, CA, CM, CAt, CMt, l1, l2, Lu(1), Lw(1), nact, P, c->dt, A.Fu, A.Fw);
    PINT_CUDA(cudaMemsetAsync(A.red, 0, 8, c->stream));
    for (int n = N - 1; n >= 0; --n) {
      transposed_sweep<T>(c, A, CA, CM, CAt, CMt, l1, l2, Lu(n + 1), Lw(n + 1), 1, 1, c->Dt, A.cu, A.cw);
      k_adj_update<<<ub, 256, 0, c->stream>>>(A.cu, A.cw, A.Fu + (size_t)n * d1, A.Fw + (size_t)n * d2,
                                              A.Gu + (size_t)n * d1, A.Gw + (size_t)n * d2, src_u(n), src_w(n),
                                              Lu(n), Lw(n), d1, d2, 0, A.red);
    }
    PINT_LAUNCH_CHECK();
    c->launches += N;
    double j2 = 0.0;
    PINT_CUDA(cudaMemcpyAsync(&j2, A.red, 8, cudaMemcpyDeviceToHost, c->stream));
    PINT_CUDA(cudaStreamSynchronize(c->stream));
    PINT_REQUIRE(std::isfinite(j2), PINT_ERR_NONFINITE, "non-finite adjoint state");
    // the summed squared change over all times bounds the largest one
    if (std::sqrt(j2) <= tol) break;
  }
}

}  // namespace

void adjoint_release(Ctx* c) {
  if (c->adj) {
    delete reinterpret_cast<Adj*>(c->adj);
    c->adj = nullptr;
  }
}

void adjoint_solve(Ctx* c, const int* obs, int n_obs, const double* data, const double* u0_nodes,
                   const double* f_nodes, const double* amp_dev, double eps, int k_max, double wr_tol, int wr_max,
                   double* misfit_host, double* grad_u0, double* grad_amp) {
  const int N = c->N, d1 = c->d1, d2 = c->d2;
  // forward solve: coarse states x_0..x_N (the checkpoints) in spectral coordinates
  if (c->precision != PINT_FP64)
    solve_mixed(c, u0_nodes, f_nodes, amp_dev, eps, k_max, wr_tol, wr_max, nullptr, nullptr, nullptr, 1);
  else
    solve_fp64(c, u0_nodes, f_nodes, amp_dev, eps, k_max, wr_tol, wr_max, nullptr, nullptr, nullptr, false);
  double *Xu = nullptr, *Xw = nullptr;
  hot_states(c, &Xu, &Xw);
  Adj& A = adj_get(c, n_obs);
  // observation operator rows in spectral coordinates: e_o^T Psi [Q, Q2]
  k_indicators<<<std::min(nb((long long)n_obs * c->nn, 256), 4096u), 256, 0, c->stream>>>(obs, n_obs, c->nn, A.E);
  PINT_LAUNCH_CHECK();
  raw_dot(c, A.E, n_obs, A.raw);
  to_reduced(c, A.raw, n_obs, A.t1, A.t2);
  dense_gemm(c, A.t1, c->Q, A.Ou, n_obs, d1, d1, false, false, 1.0, 0.0);
  dense_gemm(c, A.t2, c->Q2, A.Ow, n_obs, d2, d2, false, false, 1.0, 0.0);
  // residuals r_n = O x_n - d_n (n = 1..N) and the misfit
  dense_gemm(c, Xu + d1, A.Ou, A.R, N, n_obs, d1, false, true, 1.0, 0.0);
  dense_gemm(c, Xw + d2, A.Ow, A.R, N, n_obs, d2, false, true, 1.0, 1.0);
  double* dJ = A.red + 2 * N + 1;
  PINT_CUDA(cudaMemsetAsync(dJ, 0, 8, c->stream));
  k_resid<<<std::min(nb((long long)N * n_obs, 256), 1024u), 256, 0, c->stream>>>(A.R, data, (long long)N * n_obs,
                                                                                dJ);
  PINT_LAUNCH_CHECK();
  // adjoint sources O^T r_n as rows
  dense_gemm(c, A.R, A.Ou, A.gu, N, d1, n_obs, false, false, 1.0, 0.0);
  dense_gemm(c, A.R, A.Ow, A.gw, N, d2, n_obs, false, false, 1.0, 0.0);
  c->launches += 8;
  // backward parareal
  if (A.prec == 0) {
    backward_parareal<double>(c, A, c->CA, c->CM, c->CAt, c->CMt, c->lam1, c->lam2, N, 1e-14);
  } else {
    const long long nc = (long long)d1 * d2;
    k_cast<float><<<1024, 256, 0, c->stream>>>(c->CA, nc, (float*)A.CA);
    k_cast<float><<<1024, 256, 0, c->stream>>>(c->CM, nc, (float*)A.CM);
    k_cast<float><<<1024, 256, 0, c->stream>>>(c->CAt, nc, (float*)A.CAt);
    k_cast<float><<<1024, 256, 0, c->stream>>>(c->CMt, nc, (float*)A.CMt);
    k_cast<float><<<nb(d1, 256), 256, 0, c->stream>>>(c->lam1, d1, (float*)A.l1);
    k_cast<float><<<nb(d2, 256), 256, 0, c->stream>>>(c->lam2, d2, (float*)A.l2);
    PINT_LAUNCH_CHECK();
    backward_parareal<float>(c, A, (const float*)A.CA, (const float*)A.CM, (const float*)A.CAt,
                             (const float*)A.CMt, (const float*)A.l1, (const float*)A.l2, N, 1e-7);
  }
  if (grad_amp && c->adj_response) {
    // dJ/da_n = <lambda_{n+1}, s>
    unit_response(c, A.su, A.sw);
    k_amp_grad<<<N, 256, 0, c->stream>>>(A.Lu, A.Lw, A.su, A.sw, d1, d2, grad_amp);
    PINT_LAUNCH_CHECK();
  } else if (grad_amp) {
    // the fine adjoint recomputed inside every interval from lambda_{n+1}:
    // dJ/da_n = sum_p <mu_p, c>, all intervals at once
    step_source(c, A.su, A.sw);
    PINT_CUDA(cudaMemsetAsync(grad_amp, 0, (size_t)N * 8, c->stream));
    if (A.prec == 0)
      transposed_sweep<double>(c, A, c->CA, c->CM, c->CAt, c->CMt, c->lam1, c->lam2, A.Lu + d1, A.Lw + d2, N,
                               c->P, c->dt, A.Fu, A.Fw, grad_amp, A.su, A.sw);
    else
      transposed_sweep<float>(c, A, (const float*)A.CA, (const float*)A.CM, (const float*)A.CAt,
                              (const float*)A.CMt, (const float*)A.l1, (const float*)A.l2, A.Lu + d1, A.Lw + d2,
                              N, c->P, c->dt, A.Fu, A.Fw, grad_amp, A.su, A.sw);
  }
  // dJ/du0 = M_f Psi [Q, Q2] M_H~^-1 lambda_0, with M_H~ = [[I, CM], [CM^T, I]]
  if (grad_u0) {
    const double* l0u = A.Lu;
    const double* l0w = A.Lw;
    PINT_CUDA(cudaMemcpyAsync(A.yw, l0w, d2 * 8, cudaMemcpyDeviceToDevice, c->stream));
    dense_gemm(c, l0u, c->CM, A.yw, 1, d2, d1, false, false, -1.0, 1.0);        // g2 - CM^T g1
    dense_gemm(c, c->projInv, A.yw, A.xw, d2, 1, d2, false, false, 1.0, 0.0);  // (I - CM^T CM)^-1 (.)
    PINT_CUDA(cudaMemcpyAsync(A.xu, l0u, d1 * 8, cudaMemcpyDeviceToDevice, c->stream));
    dense_gemm(c, c->CM, A.xw, A.xu, d1, 1, d2, false, false, -1.0, 1.0);       // g1 - CM y_w
    dense_gemm(c, A.xu, c->Q, A.yu, 1, d1, d1, false, true, 1.0, 0.0);         // original coordinates
    dense_gemm(c, A.xw, c->Q2, A.yw, 1, d2, d2, false, true, 1.0, 0.0);
    prolong_coeffs(c, A.yu, A.yw, 1, A.nodes);
    apply_stencil(c, c->stM, A.nodes, grad_u0, 1);
    c->launches += 6;
  }
  if (misfit_host) {
    PINT_CUDA(cudaMemcpyAsync(misfit_host, dJ, 8, cudaMemcpyDeviceToHost, c->stream));
  }
  PINT_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace pint
