// Spectral bases of the reduced operators and the derived couplings.
//   A11 Q = M11 Q Lambda1, Q^T M11 Q = I;  A22 Q2 = M22 Q2 Lambda2, Q2^T M22 Q2 = I.
// In these coordinates the implicit V_H1 solves of eqs. (2.4) and (4.12)
// and the M22 solve of eq. (2.5) are diagonal, and the couplings become
//   CM = Q^T M12 Q2,  CA = Q^T A12 Q2.
// gamma of eq. (4.15) is the largest singular value of CM (the cosines of
// the principal angles between V_H1 and V_H2 in L2), and lambda_max(A22, M22)
// = max Lambda2 gives the time-step bound of Section 3.2.
#include "common.cuh"

#include <cmath>

namespace pint {

namespace {
__global__ void k_eye_minus(const double* G, int n, double* out) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  out[e] = ((e / n) == (e % n) ? 1.0 : 0.0) - G[e];
}
}  // namespace

void build_spectral(Ctx* c) {
  const int d1 = c->d1, d2 = c->d2;
  auto A = [&](size_t n) { return (double*)dalloc(c, n * 8); };
  if (!c->Q) {
    c->Q = A((size_t)d1 * d1);
    c->lam1 = A(d1);
    c->Q2 = A((size_t)d2 * d2);
    c->lam2 = A(d2);
    c->CM = A((size_t)d1 * d2);
    c->CA = A((size_t)d1 * d2);
    c->CMt = A((size_t)d1 * d2);
    c->CAt = A((size_t)d1 * d2);
    c->projL = A((size_t)d2 * d2);
  }
  dense_gen_eig(c, c->A11, c->M11, d1, c->Q, c->lam1);
  dense_gen_eig(c, c->A22, c->M22, d2, c->Q2, c->lam2);
  double* T = A((size_t)d1 * d2);
  dense_gemm(c, c->M12, c->Q2, T, d1, d2, d2, false, false, 1.0, 0.0);
  dense_gemm(c, c->Q, T, c->CM, d1, d2, d1, true, false, 1.0, 0.0);
  dense_gemm(c, c->A12, c->Q2, T, d1, d2, d2, false, false, 1.0, 0.0);
  dense_gemm(c, c->Q, T, c->CA, d1, d2, d1, true, false, 1.0, 0.0);
  dense_transpose(c, c->CM, d1, d2, c->CMt);
  dense_transpose(c, c->CA, d1, d2, c->CAt);
  double* G = A((size_t)d2 * d2);
  double* V = A((size_t)d2 * d2);
  double* ev = A(d2);
  dense_gemm(c, c->CM, c->CM, G, d2, d2, d1, true, false, 1.0, 0.0);
  k_eye_minus<<<(unsigned)(((long long)d2 * d2 + 255) / 256), 256, 0, c->stream>>>(G, d2, c->projL);
  PINT_LAUNCH_CHECK();
  dense_sym_eig(c, G, V, ev, d2);
  double gmax = 0, lmax = 0;
  PINT_CUDA(cudaMemcpyAsync(&gmax, ev + d2 - 1, 8, cudaMemcpyDeviceToHost, c->stream));
  PINT_CUDA(cudaMemcpyAsync(&lmax, c->lam2 + d2 - 1, 8, cudaMemcpyDeviceToHost, c->stream));
  PINT_CUDA(cudaStreamSynchronize(c->stream));
  c->gamma = std::sqrt(std::max(gmax, 0.0));
  c->lam22 = lmax;
  c->dt_max = (1.0 - c->gamma * c->gamma) / lmax;
  dense_cholesky(c, c->projL, d2);
  // explicit inverse (I - CM^T CM)^-1 for the initial projection
  if (!c->projInv) c->projInv = A((size_t)d2 * d2);
  PINT_CUDA(cudaMemsetAsync(G, 0, (size_t)d2 * d2 * 8, c->stream));
  k_eye_minus<<<(unsigned)(((long long)d2 * d2 + 255) / 256), 256, 0, c->stream>>>(G, d2, c->projInv);
  PINT_LAUNCH_CHECK();
  dense_trsm_lower(c, c->projL, c->projInv, d2, d2, false);
  dense_trsm_lower(c, c->projL, c->projInv, d2, d2, true);
  dfree(c, T);
  dfree(c, G);
  dfree(c, V);
  dfree(c, ev);
}

}  // namespace pint
