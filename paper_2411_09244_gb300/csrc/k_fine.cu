// Q1 fine-grid assembly (Section 2, eq. (2.2); M_f and A_f of Section 3.2)
// as 9-point stencils on all (n_f+1)^2 nodes, plus the kappa_tilde-weighted
// mass of the CEM inner product s(u, v) = int kappa H^-2 u v (eq. (3.1)).
// Stencil entry k = (dy+1)*3 + (dx+1) couples node (i, j) to (i+dx, j+dy).
#include "common.cuh"

namespace pint {

// One thread per node gathers the element contributions of its (up to 4)
// adjacent cells; no atomics, fixed summation order.
__global__ void k_assemble_stencils(int n_f, const double* __restrict__ kappa, double kt_scale,
                                    double* __restrict__ stA, double* __restrict__ stM,
                                    double* __restrict__ stS) {
  int nn1 = n_f + 1;
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nn1 * nn1) return;
  int i = node % nn1, j = node / nn1;
  double h2 = 1.0 / ((double)n_f * n_f);
  double a[9], m[9], s[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) a[k] = m[k] = s[k] = 0.0;
  for (int cj = j - 1; cj <= j; ++cj) {
    if (cj < 0 || cj >= n_f) continue;
    for (int ci = i - 1; ci <= i; ++ci) {
      if (ci < 0 || ci >= n_f) continue;
      double kap = kappa[cj * n_f + ci];
      int lx = i - ci, ly = j - cj;
      int ca = (ly == 0) ? (lx == 0 ? 0 : 1) : (lx == 1 ? 2 : 3);
      for (int cb = 0; cb < 4; ++cb) {
        int bx = ci + pintd::corner_x(cb), by = cj + pintd::corner_y(cb);
        int k = (by - j + 1) * 3 + (bx - i + 1);
        double ke = pintd::q1_stiff(ca, cb), me = pintd::q1_mass(ca, cb) * h2;
        a[k] += kap * ke;
        m[k] += me;
        s[k] += kap * kt_scale * me;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    stA[(size_t)node * 9 + k] = a[k];
    stM[(size_t)node * 9 + k] = m[k];
    stS[(size_t)node * 9 + k] = s[k];
  }
}

// y = St x on all nodes, for `count` stacked nodal vectors
__global__ void k_apply_stencil(int n_f, int count, const double* __restrict__ st,
                                const double* __restrict__ x, double* __restrict__ y) {
  int nn1 = n_f + 1, nn = nn1 * nn1;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nn * count) return;
  int v = (int)(t / nn), node = (int)(t % nn);
  int i = node % nn1, j = node / nn1;
  const double* xv = x + (size_t)v * nn;
  double acc = 0.0;
  for (int dy = -1; dy <= 1; ++dy) {
    int jj = j + dy;
    if (jj < 0 || jj > n_f) continue;
    for (int dx = -1; dx <= 1; ++dx) {
      int ii = i + dx;
      if (ii < 0 || ii > n_f) continue;
      acc += st[(size_t)node * 9 + (dy + 1) * 3 + (dx + 1)] * xv[jj * nn1 + ii];
    }
  }
  y[t] = acc;
}

void build_fine(Ctx* c, const double* kappa_dev) {
  int nn = c->nn;
  size_t sb = (size_t)nn * 9 * sizeof(double);
  c->stA = (double*)dalloc(c, sb);
  c->stM = (double*)dalloc(c, sb);
  c->stS = (double*)dalloc(c, sb);
  c->kappa = (double*)dalloc(c, (size_t)c->n_f * c->n_f * sizeof(double));
  PINT_CUDA(cudaMemcpyAsync(c->kappa, kappa_dev, (size_t)c->n_f * c->n_f * sizeof(double),
                            cudaMemcpyDeviceToDevice, c->stream));
  // kappa_tilde scale H^-2 is applied when the coarse grid is known; keep
  // stS = kappa-weighted mass here and rescale in build_blocks.
  k_assemble_stencils<<<(nn + 255) / 256, 256, 0, c->stream>>>(c->n_f, c->kappa, 1.0, c->stA,
                                                              c->stM, c->stS);
  PINT_LAUNCH_CHECK();
}

void apply_stencil(Ctx* c, const double* st, const double* x, double* y, int count) {
  long long tot = (long long)c->nn * count;
  k_apply_stencil<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(c->n_f, count, st, x, y);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

}  // namespace pint
