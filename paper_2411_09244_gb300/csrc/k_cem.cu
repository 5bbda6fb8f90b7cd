// Constraint energy minimising bases on the oversampled windows K_i^+
// (Section 3.1, eq. (3.2)), one window per coarse block, for every
// auxiliary function of that block at once.
//
// With A_w the fine stiffness on the window's interior nodes (zero Dirichlet
// data on the window boundary, which also carries the domain boundary) and
// C the constraint functionals of all auxiliary functions of the blocks in
// the window, eq. (3.2) is the saddle-point system
//     A_w phi + C^T mu = 0,   C phi = g,
// with g the s-Gram column of the target function.  It is solved by the
// Schur complement:  A_w = L L^T (banded Cholesky, bandwidth wx+1),
// Y = L^-1 C^T, S = Y^T Y (= C A_w^-1 C^T), S X = g, phi = L^-T (Y X).
// Columns of C^T are zero above the first node of their block, so Y's are
// too; the forward solve and the Schur products start there.
//
// S = Y^T Y squares the conditioning (cond(S) ~ 1e12 on a contrast-1e6
// window), so the plain Schur solve leaves forward errors ~1e-9 in phi.  One
// step of iterative refinement with the same factors removes them: with
// X = -mu, the residuals r1 = C^T X - A_w phi and r2 = g - C phi give
// z = L^-1 r1, dX = S^-1 (r2 - Y^T z), dphi = L^-T (z + Y dX).
#include "common.cuh"

#include <algorithm>

namespace pint {

namespace {

struct WinDev {
  int X0, Y0, wx, wy, nw, b, m, t0, kt, blk;
  int bx0, by0, nbx, nby;  // coarse blocks of the window (rectangle)
  long long lb_off, y_off, s_off, psi_off, col_off;
  long long bc_off;        // first constraint column of each window block (bcol table)
  long long r_off;         // refinement scratch: nw kt (r1, z, dphi) and m kt (r2, t)
};

// window-local constraint column of aux function qq of block (xb, yb), or -1
__device__ __forceinline__ int win_col(const WinDev& W, const int* __restrict__ bcol, int xb, int yb, int qq) {
  if (xb < W.bx0 || xb >= W.bx0 + W.nbx || yb < W.by0 || yb >= W.by0 + W.nby) return -1;
  return bcol[W.bc_off + (yb - W.by0) * W.nbx + (xb - W.bx0)] + qq;
}

// --- banded A_w from the 9-point stiffness stencil -------------------------
__global__ void k_win_assemble(const WinDev* __restrict__ wd, int w0, const double* __restrict__ stA,
                               int n_f, double* __restrict__ lb) {
  const WinDev W = wd[w0 + blockIdx.y];
  const int b = W.b, bw = b + 1;
  double* L = lb + W.lb_off;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)W.nw * bw;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / bw), k = (int)(e % bw);
    int j = i - b + k;  // column
    double v = 0.0;
    if (j >= 0) {
      int xi = i % W.wx, yi = i / W.wx, xj = j % W.wx, yj = j / W.wx;
      int dx = xj - xi, dy = yj - yi;
      if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) {
        int node = (W.Y0 + yi) * (n_f + 1) + (W.X0 + xi);
        v = stA[(size_t)node * 9 + (dy + 1) * 3 + (dx + 1)];
      }
    }
    L[e] = v;
  }
}

// --- right-looking banded Cholesky, one CTA per window ----------------------
// storage: row i, slot k <-> column i - b + k (k = b is the diagonal)
__global__ void __launch_bounds__(512) k_band_chol(const WinDev* __restrict__ wd, int w0,
                                                   double* __restrict__ lb, int* __restrict__ status) {
  const WinDev W = wd[w0 + blockIdx.x];
  const int b = W.b, bw = b + 1, n = W.nw;
  double* L = lb + W.lb_off;
  __shared__ double s_piv;
  __shared__ double col[1100];
  for (int k = 0; k < n; ++k) {
    int rem = min(b, n - 1 - k);
    if (threadIdx.x == 0) {
      double d = L[(size_t)k * bw + b];
      if (!(d > 0.0)) {
        status[w0 + blockIdx.x] = 1;
        d = 1.0;
      }
      s_piv = sqrt(d);
      L[(size_t)k * bw + b] = s_piv;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < rem; t += blockDim.x) {
      int i = k + 1 + t;
      double v = L[(size_t)i * bw + (k - i + b)] / s_piv;
      L[(size_t)i * bw + (k - i + b)] = v;
      col[t] = v;
    }
    __syncthreads();
    int tri = rem * (rem + 1) / 2;
    for (int t = threadIdx.x; t < tri; t += blockDim.x) {
      // t -> (ii, jj) with 0 <= jj <= ii < rem
      int ii = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
      while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
      while (ii * (ii + 1) / 2 > t) --ii;
      int jj = t - ii * (ii + 1) / 2;
      int i = k + 1 + ii, j = k + 1 + jj;
      L[(size_t)i * bw + (j - i + b)] -= col[ii] * col[jj];
    }
    __syncthreads();
  }
}

// --- C^T scattered into Y (row-major n_w x m): zero, then scatter -----------
__global__ void k_win_zero(const WinDev* __restrict__ wd, int w0, double* __restrict__ y) {
  const WinDev W = wd[w0 + blockIdx.y];
  double* Y = y + W.y_off;
  const long long tot = (long long)W.nw * W.m;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x)
    Y[e] = 0.0;
}

__global__ void k_win_scatter(const WinDev* __restrict__ wd, int w0, const int* __restrict__ colmap,
                              const double* __restrict__ con_rows, int kcap, int nb, int bs, int nc,
                              double* __restrict__ y) {
  const WinDev W = wd[w0 + blockIdx.y];
  double* Y = y + W.y_off;
  const long long tot2 = (long long)W.m * nb;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot2;
       e += (long long)gridDim.x * blockDim.x) {
    int c = (int)(e / nb), r = (int)(e % nb);
    int code = colmap[W.col_off + c];
    int blk = code / kcap, q = code % kcap;
    int bxb = blk % nc, byb = blk / nc;
    int gx = bxb * bs + r % (bs + 1), gy = byb * bs + r / (bs + 1);
    int lx = gx - W.X0, ly = gy - W.Y0;
    if (lx < 0 || lx >= W.wx || ly < 0 || ly >= W.wy) continue;
    Y[(size_t)(ly * W.wx + lx) * W.m + c] = con_rows[((size_t)blk * kcap + q) * nb + r];
  }
}

// --- Y = L^-1 Y, one thread per column, starting at the column's first row --
__global__ void k_band_fwd(const WinDev* __restrict__ wd, int w0, const double* __restrict__ lb,
                           const int* __restrict__ first, double* __restrict__ y) {
  const WinDev W = wd[w0 + blockIdx.y];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= W.m) return;
  const int b = W.b, bw = b + 1, m = W.m;
  const double* L = lb + W.lb_off;
  double* Y = y + W.y_off;
  const int i0 = first[W.col_off + c];
  for (int i = i0; i < W.nw; ++i) {
    double v = Y[(size_t)i * m + c];
    const double* Li = L + (size_t)i * bw;
    int k0 = max(i0, i - b);
    for (int k = k0; k < i; ++k) v -= Li[k - i + b] * Y[(size_t)k * m + c];
    Y[(size_t)i * m + c] = v / Li[b];
  }
}

// --- S = Y^T Y, 32x32 tiles, K range from the later first row of the tile ---
__global__ void __launch_bounds__(256) k_win_schur(const WinDev* __restrict__ wd, int w0,
                                                   const double* __restrict__ y,
                                                   const int* __restrict__ first,
                                                   double* __restrict__ sch) {
  const WinDev W = wd[w0 + blockIdx.z];
  const int m = W.m;
  const int ti = blockIdx.y * 32, tj = blockIdx.x * 32;
  if (ti >= m || tj >= m || tj > ti + 31) return;  // lower triangle of tiles only
  const double* Y = y + W.y_off;
  __shared__ double As[16][33], Bs[16][33];
  __shared__ int s_k0;
  if (threadIdx.x == 0) {
    int fa = 1 << 30, fb = 1 << 30;
    for (int t = 0; t < 32; ++t) {
      if (ti + t < m) fa = min(fa, first[W.col_off + ti + t]);
      if (tj + t < m) fb = min(fb, first[W.col_off + tj + t]);
    }
    s_k0 = max(fa, fb);
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // each thread 2x2 outputs
  double acc[2][2] = {{0, 0}, {0, 0}};
  for (int k0 = s_k0; k0 < W.nw; k0 += 16) {
    for (int t = threadIdx.x; t < 16 * 32; t += 256) {
      int kk = t / 32, cc = t % 32;
      int k = k0 + kk;
      As[kk][cc] = (k < W.nw && ti + cc < m) ? Y[(size_t)k * m + ti + cc] : 0.0;
      Bs[kk][cc] = (k < W.nw && tj + cc < m) ? Y[(size_t)k * m + tj + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a0 = As[kk][ty * 2], a1 = As[kk][ty * 2 + 1];
      double b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
  double* S = sch + W.s_off;
  for (int a = 0; a < 2; ++a)
    for (int bb = 0; bb < 2; ++bb) {
      int i = ti + ty * 2 + a, j = tj + tx * 2 + bb;
      if (i < m && j < m) {
        S[(size_t)i * m + j] = acc[a][bb];
        S[(size_t)j * m + i] = acc[a][bb];
      }
    }
}

// --- dense Cholesky of S and solve S X = g, one CTA per window ---------------
__global__ void __launch_bounds__(512) k_win_small(const WinDev* __restrict__ wd, int w0,
                                                   double* __restrict__ sch,
                                                   const double* __restrict__ gram, int kcap,
                                                   int* __restrict__ status) {
  const WinDev W = wd[w0 + blockIdx.x];
  const int m = W.m, kt = W.kt;
  double* S = sch + W.s_off;
  __shared__ double s_piv;
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      double d = S[(size_t)k * m + k];
      if (!(d > 0.0)) {
        status[w0 + blockIdx.x] = 2;
        d = 1.0;
      }
      s_piv = sqrt(d);
      S[(size_t)k * m + k] = s_piv;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) S[(size_t)i * m + k] /= s_piv;
    __syncthreads();
    int rem = m - k - 1;
    for (int t = threadIdx.x; t < rem * rem; t += blockDim.x) {
      int i = k + 1 + t / rem, j = k + 1 + t % rem;
      if (j <= i) S[(size_t)i * m + j] -= S[(size_t)i * m + k] * S[(size_t)j * m + k];
    }
    __syncthreads();
  }
  // X (m x kt) stored after S in the same buffer region: s_off + m*m
  double* Xw = S + (size_t)m * m;
  for (int q = threadIdx.x; q < kt; q += blockDim.x) {
    // forward: L z = g, g = gram_q e_{t0+q}
    for (int i = 0; i < m; ++i) {
      double v = (i == W.t0 + q) ? gram[(size_t)W.blk * kcap + q] : 0.0;
      for (int k = 0; k < i; ++k) v -= S[(size_t)i * m + k] * Xw[(size_t)k * kt + q];
      Xw[(size_t)i * kt + q] = v / S[(size_t)i * m + i];
    }
    // backward: L^T x = z
    for (int i = m - 1; i >= 0; --i) {
      double v = Xw[(size_t)i * kt + q];
      for (int k = i + 1; k < m; ++k) v -= S[(size_t)k * m + i] * Xw[(size_t)k * kt + q];
      Xw[(size_t)i * kt + q] = v / S[(size_t)i * m + i];
    }
  }
}

// Z <- L^-T Z for the kt columns of Z (column q at q n), whole CTA:
// column-oriented back substitution, x_i = z_i / L_ii, then z_k -= L_ik x_i
// for k in [i-b, i)
__device__ void band_back_cols(const double* __restrict__ L, double* __restrict__ Z, int n, int b, int kt) {
  const int bw = b + 1;
  for (int i = n - 1; i >= 0; --i) {
    const double* Li = L + (size_t)i * bw;
    if (threadIdx.x < kt) Z[(size_t)threadIdx.x * n + i] /= Li[b];
    __syncthreads();
    int k0 = max(0, i - b);
    int cnt = (i - k0) * kt;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      int k = k0 + t / kt, q = t % kt;
      Z[(size_t)q * n + k] -= Li[k - i + b] * Z[(size_t)q * n + i];
    }
    __syncthreads();
  }
}

// --- phi = L^-T (Y X), one CTA per window ------------------------------------
__global__ void __launch_bounds__(512) k_win_phi(const WinDev* __restrict__ wd, int w0,
                                                 const double* __restrict__ lb,
                                                 const double* __restrict__ y,
                                                 const double* __restrict__ sch,
                                                 double* __restrict__ psi) {
  const WinDev W = wd[w0 + blockIdx.x];
  const int m = W.m, kt = W.kt, n = W.nw;
  const double* Y = y + W.y_off;
  const double* Xw = sch + W.s_off + (size_t)m * m;
  double* Z = psi + W.psi_off;  // kt x n, column q at q*n
  for (long long e = threadIdx.x; e < (long long)n * kt; e += blockDim.x) {
    int i = (int)(e / kt), q = (int)(e % kt);
    double acc = 0.0;
    for (int c = 0; c < m; ++c) acc += Y[(size_t)i * m + c] * Xw[(size_t)c * kt + q];
    Z[(size_t)q * n + i] = acc;
  }
  __syncthreads();
  band_back_cols(lb + W.lb_off, Z, n, W.b, kt);
}

// --- refinement step 1: residuals of the saddle-point system -----------------
// r1[i][q] = (C^T X)_iq - (A_w phi)_iq on the window nodes; r2[c][q] =
// g_cq - (C phi)_cq on the constraints.  One CTA per window.
__global__ void __launch_bounds__(512) k_win_resid(const WinDev* __restrict__ wd, int w0,
                                                   const double* __restrict__ stA, int n_f,
                                                   const int* __restrict__ colmap, const int* __restrict__ bcol,
                                                   const int* __restrict__ blk_k, const double* __restrict__ con_rows,
                                                   const double* __restrict__ gram, int kcap, int nb, int bs, int nc,
                                                   const double* __restrict__ sch, const double* __restrict__ psi,
                                                   double* __restrict__ r1, double* __restrict__ r2) {
  const WinDev W = wd[w0 + blockIdx.x];
  const int m = W.m, kt = W.kt, n = W.nw;
  const double* Xw = sch + W.s_off + (size_t)m * m;  // [c][kt]
  const double* phi = psi + W.psi_off;                // [q][n]
  double* R1 = r1 + W.r_off;                          // [i][kt]
  double* R2 = r2 + W.r_off;                          // [c][kt]
  for (long long e = threadIdx.x; e < (long long)n * kt; e += blockDim.x) {
    const int i = (int)(e / kt), q = (int)(e % kt);
    const int lx = i % W.wx, ly = i / W.wx, gx = W.X0 + lx, gy = W.Y0 + ly;
    double acc = 0.0;
    // C^T X: the (up to 4) blocks whose closure holds node (gx, gy)
    for (int yb = max(0, (gy - 1) / bs); yb <= min(nc - 1, gy / bs); ++yb)
      for (int xb = max(0, (gx - 1) / bs); xb <= min(nc - 1, gx / bs); ++xb) {
        if (gx < xb * bs || gx > (xb + 1) * bs || gy < yb * bs || gy > (yb + 1) * bs) continue;
        const int b2 = yb * nc + xb, r = (gy - yb * bs) * (bs + 1) + (gx - xb * bs);
        for (int qq = 0; qq < blk_k[b2]; ++qq) {
          const int c = win_col(W, bcol, xb, yb, qq);
          if (c < 0) break;
          acc += con_rows[((size_t)b2 * kcap + qq) * nb + r] * Xw[(size_t)c * kt + q];
        }
      }
    // A_w phi (zero Dirichlet data outside the window)
    const int node = gy * (n_f + 1) + gx;
    double ap = 0.0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int x2 = lx + dx, y2 = ly + dy;
        if (x2 < 0 || x2 >= W.wx || y2 < 0 || y2 >= W.wy) continue;
        ap += stA[(size_t)node * 9 + (dy + 1) * 3 + (dx + 1)] * phi[(size_t)q * n + y2 * W.wx + x2];
      }
    R1[(size_t)i * kt + q] = acc - ap;
  }
  // r2: one warp per constraint column, lanes over the block's nodes
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int c = warp; c < m; c += nwarp) {
    const int code = colmap[W.col_off + c], b2 = code / kcap, qq = code % kcap;
    const int xb = b2 % nc, yb = b2 / nc;
    for (int q = 0; q < kt; ++q) {
      double acc = 0.0;
      for (int r = lane; r < nb; r += 32) {
        const int gx = xb * bs + r % (bs + 1), gy = yb * bs + r / (bs + 1);
        const int lx = gx - W.X0, ly = gy - W.Y0;
        if (lx < 0 || lx >= W.wx || ly < 0 || ly >= W.wy) continue;
        acc += con_rows[((size_t)b2 * kcap + qq) * nb + r] * phi[(size_t)q * n + ly * W.wx + lx];
      }
      acc = pintd::warp_sum(acc);
      if (lane == 0) {
        const double g = (c == W.t0 + q) ? gram[(size_t)W.blk * kcap + q] : 0.0;
        R2[(size_t)c * kt + q] = g - acc;
      }
    }
  }
}

// --- refinement step 2: z = L^-1 r1 in place, one warp per column -------------
__global__ void __launch_bounds__(256) k_win_fwd_cols(const WinDev* __restrict__ wd, int w0,
                                                      const double* __restrict__ lb, double* __restrict__ r1) {
  const WinDev W = wd[w0 + blockIdx.x];
  const int kt = W.kt, n = W.nw, b = W.b, bw = b + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const double* L = lb + W.lb_off;
  double* Z = r1 + W.r_off;  // [i][kt]
  for (int q = warp; q < kt; q += nwarp) {
    for (int i = 0; i < n; ++i) {
      const double* Li = L + (size_t)i * bw;
      double acc = 0.0;
      for (int k = max(0, i - b) + lane; k < i; k += 32) acc += Li[k - i + b] * Z[(size_t)k * kt + q];
      acc = pintd::warp_sum(acc);
      if (lane == 0) Z[(size_t)i * kt + q] = (Z[(size_t)i * kt + q] - acc) / Li[b];
      __syncwarp();
    }
  }
}

// --- refinement step 3: r2 <- r2 - Y^T z, threads over constraint columns ----
constexpr int RQ = 8;  // right-hand sides per pass
__global__ void __launch_bounds__(128) k_win_ytz(const WinDev* __restrict__ wd, int w0,
                                                 const double* __restrict__ y, const int* __restrict__ first,
                                                 const double* __restrict__ r1, double* __restrict__ r2) {
  const WinDev W = wd[w0 + blockIdx.y];
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= W.m) return;
  const int m = W.m, kt = W.kt, n = W.nw;
  const double* Y = y + W.y_off;
  const double* Z = r1 + W.r_off;
  double* R2 = r2 + W.r_off;
  const int i0 = first[W.col_off + c];
  for (int q0 = 0; q0 < kt; q0 += RQ) {
    double acc[RQ];
#pragma unroll
    for (int t = 0; t < RQ; ++t) acc[t] = 0.0;
    for (int i = i0; i < n; ++i) {
      const double yv = Y[(size_t)i * m + c];
#pragma unroll
      for (int t = 0; t < RQ; ++t)
        if (q0 + t < kt) acc[t] += yv * Z[(size_t)i * kt + q0 + t];
    }
#pragma unroll
    for (int t = 0; t < RQ; ++t)
      if (q0 + t < kt) R2[(size_t)c * kt + q0 + t] -= acc[t];
  }
}

// --- refinement step 4: dX = S^-1 r2 (Cholesky factor of S from k_win_small) --
__global__ void __launch_bounds__(256) k_win_small_rhs(const WinDev* __restrict__ wd, int w0,
                                                       const double* __restrict__ sch, double* __restrict__ r2) {
  const WinDev W = wd[w0 + blockIdx.x];
  const int m = W.m, kt = W.kt;
  const double* S = sch + W.s_off;
  double* X = r2 + W.r_off;  // [c][kt], overwritten by the solution
  for (int q = threadIdx.x; q < kt; q += blockDim.x) {
    for (int i = 0; i < m; ++i) {
      double v = X[(size_t)i * kt + q];
      for (int k = 0; k < i; ++k) v -= S[(size_t)i * m + k] * X[(size_t)k * kt + q];
      X[(size_t)i * kt + q] = v / S[(size_t)i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
      double v = X[(size_t)i * kt + q];
      for (int k = i + 1; k < m; ++k) v -= S[(size_t)k * m + i] * X[(size_t)k * kt + q];
      X[(size_t)i * kt + q] = v / S[(size_t)i * m + i];
    }
  }
}

// --- refinement step 5: phi += L^-T (z + Y dX), one CTA per window -----------
__global__ void __launch_bounds__(512) k_win_phi_corr(const WinDev* __restrict__ wd, int w0,
                                                      const double* __restrict__ lb, const double* __restrict__ y,
                                                      const double* __restrict__ r1, const double* __restrict__ r2,
                                                      double* __restrict__ dphi, double* __restrict__ psi) {
  const WinDev W = wd[w0 + blockIdx.x];
  const int m = W.m, kt = W.kt, n = W.nw;
  const double* Y = y + W.y_off;
  const double* Z = r1 + W.r_off;   // [i][kt]
  const double* dX = r2 + W.r_off;  // [c][kt]
  double* D = dphi + W.r_off;       // [q][n]
  for (long long e = threadIdx.x; e < (long long)n * kt; e += blockDim.x) {
    const int i = (int)(e / kt), q = (int)(e % kt);
    double acc = Z[(size_t)i * kt + q];
    for (int c = 0; c < m; ++c) acc += Y[(size_t)i * m + c] * dX[(size_t)c * kt + q];
    D[(size_t)q * n + i] = acc;
  }
  __syncthreads();
  band_back_cols(lb + W.lb_off, D, n, W.b, kt);
  double* phi = psi + W.psi_off;
  for (long long e = threadIdx.x; e < (long long)n * kt; e += blockDim.x) phi[e] += D[e];
}

}  // namespace

void build_windows(Ctx* c) {
  const int nc = c->nc, bs = c->bs, ell = c->ell, kcap = c->kmax;
  c->win.assign(c->n_blocks, WinDesc{});
  std::vector<WinDev> wd(c->n_blocks);
  std::vector<int> colmap, first, bcol;
  long long psi_tot = 0, col_tot = 0;
  for (int blk = 0; blk < c->n_blocks; ++blk) {
    int bx = blk % nc, by = blk / nc;
    WinDesc& W = c->win[blk];
    W.bx0 = std::max(0, bx - ell);
    W.bx1 = std::min(nc - 1, bx + ell);
    W.by0 = std::max(0, by - ell);
    W.by1 = std::min(nc - 1, by + ell);
    W.X0 = W.bx0 * bs + 1;
    W.Y0 = W.by0 * bs + 1;
    W.wx = (W.bx1 + 1) * bs - W.bx0 * bs - 1;
    W.wy = (W.by1 + 1) * bs - W.by0 * bs - 1;
    W.nw = W.wx * W.wy;
    W.m = 0;
    W.t0 = -1;
    WinDev& D = wd[blk];
    D.col_off = col_tot;
    D.bc_off = (long long)bcol.size();
    D.bx0 = W.bx0;
    D.by0 = W.by0;
    D.nbx = W.bx1 - W.bx0 + 1;
    D.nby = W.by1 - W.by0 + 1;
    for (int yb = W.by0; yb <= W.by1; ++yb)
      for (int xb = W.bx0; xb <= W.bx1; ++xb) {
        int b2 = yb * nc + xb;
        if (b2 == blk) W.t0 = W.m;
        bcol.push_back(W.m);
        // first window row touched by block b2 (its smallest interior node)
        int fx = std::max(xb * bs, W.X0) - W.X0, fy = std::max(yb * bs, W.Y0) - W.Y0;
        for (int q = 0; q < c->blk_k[b2]; ++q) {
          colmap.push_back(b2 * kcap + q);
          first.push_back(fy * W.wx + fx);
        }
        W.m += c->blk_k[b2];
      }
    col_tot += W.m;
    W.kt = c->blk_k[blk];
    W.psi_off = psi_tot;
    psi_tot += (long long)W.kt * W.nw;
    D.X0 = W.X0;
    D.Y0 = W.Y0;
    D.wx = W.wx;
    D.wy = W.wy;
    D.nw = W.nw;
    D.b = W.wx + 1;
    D.m = W.m;
    D.t0 = W.t0;
    D.kt = W.kt;
    D.blk = blk;
    D.psi_off = W.psi_off;
  }
  c->psi_total = psi_tot;
  c->psi = (double*)dalloc(c, (size_t)psi_tot * sizeof(double));
  int* d_colmap = (int*)dalloc(c, colmap.size() * sizeof(int));
  int* d_first = (int*)dalloc(c, first.size() * sizeof(int));
  int* d_bcol = (int*)dalloc(c, bcol.size() * sizeof(int));
  int* d_blk_k = (int*)dalloc(c, c->n_blocks * sizeof(int));
  PINT_CUDA(cudaMemcpyAsync(d_bcol, bcol.data(), bcol.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  PINT_CUDA(cudaMemcpyAsync(d_blk_k, c->blk_k.data(), c->n_blocks * sizeof(int), cudaMemcpyHostToDevice,
                            c->stream));
  PINT_CUDA(cudaMemcpyAsync(d_colmap, colmap.data(), colmap.size() * sizeof(int),
                            cudaMemcpyHostToDevice, c->stream));
  PINT_CUDA(cudaMemcpyAsync(d_first, first.data(), first.size() * sizeof(int),
                            cudaMemcpyHostToDevice, c->stream));
  int* d_status = (int*)dalloc(c, c->n_blocks * sizeof(int));
  PINT_CUDA(cudaMemsetAsync(d_status, 0, c->n_blocks * sizeof(int), c->stream));
  // batches under a scratch budget
  const long long budget = 24LL << 30;
  int w = 0;
  while (w < c->n_blocks) {
    long long lb = 0, yy = 0, ss = 0, rr = 0;
    int w1 = w;
    while (w1 < c->n_blocks) {
      const WinDev& D = wd[w1];
      long long nlb = (long long)D.nw * (D.b + 1), ny = (long long)D.nw * D.m,
                ns = (long long)D.m * D.m + (long long)D.m * D.kt,
                nr = (long long)std::max(D.nw, D.m) * D.kt;
      if (w1 > w && (lb + nlb + yy + ny + ss + ns + 3 * (rr + nr)) * 8 > budget) break;
      wd[w1].lb_off = lb;
      wd[w1].y_off = yy;
      wd[w1].s_off = ss;
      wd[w1].r_off = rr;
      lb += nlb;
      yy += ny;
      ss += ns;
      rr += nr;
      ++w1;
    }
    int nwin = w1 - w;
    WinDev* d_wd = (WinDev*)dalloc(c, sizeof(WinDev) * c->n_blocks);
    PINT_CUDA(cudaMemcpyAsync(d_wd, wd.data(), sizeof(WinDev) * c->n_blocks, cudaMemcpyHostToDevice,
                              c->stream));
    double* d_lb = (double*)dalloc(c, (size_t)lb * 8);
    double* d_y = (double*)dalloc(c, (size_t)yy * 8);
    double* d_s = (double*)dalloc(c, (size_t)ss * 8);
    int maxm = 0, maxb = 0;
    for (int t = w; t < w1; ++t) {
      maxm = std::max(maxm, wd[t].m);
      maxb = std::max(maxb, wd[t].b);
    }
    PINT_REQUIRE(maxb + 1 <= 1100, PINT_ERR_BAD_ARG, "window too wide for the band kernel");
    k_win_assemble<<<dim3(64, nwin), 256, 0, c->stream>>>(d_wd, w, c->stA, c->n_f, d_lb);
    PINT_LAUNCH_CHECK();
    k_band_chol<<<nwin, 512, 0, c->stream>>>(d_wd, w, d_lb, d_status);
    PINT_LAUNCH_CHECK();
    k_win_zero<<<dim3(64, nwin), 256, 0, c->stream>>>(d_wd, w, d_y);
    PINT_LAUNCH_CHECK();
    k_win_scatter<<<dim3(32, nwin), 256, 0, c->stream>>>(d_wd, w, d_colmap, c->con_rows, kcap,
                                                         c->nb, bs, nc, d_y);
    PINT_LAUNCH_CHECK();
    k_band_fwd<<<dim3((maxm + 127) / 128, nwin), 128, 0, c->stream>>>(d_wd, w, d_lb, d_first, d_y);
    PINT_LAUNCH_CHECK();
    int tiles = (maxm + 31) / 32;
    k_win_schur<<<dim3(tiles, tiles, nwin), 256, 0, c->stream>>>(d_wd, w, d_y, d_first, d_s);
    PINT_LAUNCH_CHECK();
    k_win_small<<<nwin, 512, 0, c->stream>>>(d_wd, w, d_s, c->con_gram, kcap, d_status);
    PINT_LAUNCH_CHECK();
    k_win_phi<<<nwin, 512, 0, c->stream>>>(d_wd, w, d_lb, d_y, d_s, c->psi);
    PINT_LAUNCH_CHECK();
    // one step of iterative refinement with the same factors
    double* d_r1 = (double*)dalloc(c, (size_t)rr * 8);
    double* d_r2 = (double*)dalloc(c, (size_t)rr * 8);
    double* d_dp = (double*)dalloc(c, (size_t)rr * 8);
    k_win_resid<<<nwin, 512, 0, c->stream>>>(d_wd, w, c->stA, c->n_f, d_colmap, d_bcol, d_blk_k, c->con_rows,
                                             c->con_gram, kcap, c->nb, bs, nc, d_s, c->psi, d_r1, d_r2);
    PINT_LAUNCH_CHECK();
    k_win_fwd_cols<<<nwin, 256, 0, c->stream>>>(d_wd, w, d_lb, d_r1);
    PINT_LAUNCH_CHECK();
    k_win_ytz<<<dim3((maxm + 127) / 128, nwin), 128, 0, c->stream>>>(d_wd, w, d_y, d_first, d_r1, d_r2);
    PINT_LAUNCH_CHECK();
    k_win_small_rhs<<<nwin, 256, 0, c->stream>>>(d_wd, w, d_s, d_r2);
    PINT_LAUNCH_CHECK();
    k_win_phi_corr<<<nwin, 512, 0, c->stream>>>(d_wd, w, d_lb, d_y, d_r1, d_r2, d_dp, c->psi);
    PINT_LAUNCH_CHECK();
    PINT_CUDA(cudaStreamSynchronize(c->stream));
    dfree(c, d_r1);
    dfree(c, d_r2);
    dfree(c, d_dp);
    dfree(c, d_lb);
    dfree(c, d_y);
    dfree(c, d_s);
    dfree(c, d_wd);
    w = w1;
  }
  std::vector<int> st(c->n_blocks);
  PINT_CUDA(cudaMemcpyAsync(st.data(), d_status, st.size() * sizeof(int), cudaMemcpyDeviceToHost,
                            c->stream));
  PINT_CUDA(cudaStreamSynchronize(c->stream));
  dfree(c, d_status);
  dfree(c, d_colmap);
  dfree(c, d_first);
  dfree(c, d_bcol);
  dfree(c, d_blk_k);
  for (int s : st) PINT_REQUIRE(s == 0, PINT_ERR_SINGULAR, "window saddle-point system singular");
}

}  // namespace pint
