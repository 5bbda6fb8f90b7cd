// Per coarse block K_i (Section 3): the continua of the NLMC construction
// (eqs. (3.4)-(3.5)), the auxiliary eigenproblem eq. (3.1) and the
// eigen-enrichment of the auxiliary space, ending in the constraint
// functionals nu -> s(phi, nu) of every auxiliary function of the block
// (the rows of the constraint operator of eq. (3.2)).
//
// One CTA per block, dense FP64 in a per-block global scratch:
//   S = L L^T (Cholesky), C = L^-1 A L^-T, C = Y diag(lam) Y^T by the
//   parallel cyclic Jacobi method (round-robin pairing, all n/2 rotations of
//   a round applied together), eigenvectors Phi = L^-T Y (s-orthonormal).
// Auxiliary functions of a block, in order: matrix indicator (if the block
// has background cells), one indicator per high-conductivity 4-connected
// component (ordered by smallest cell index), then the enrichment: the span
// of the J+1 smallest eigenfunctions (a tied next eigenvalue extends the
// set) projected s-orthogonally off the indicators, directions with
// projected s-norm^2 <= 1e-8 dropped, s-orthonormalised, rotated to the
// eigenvectors of the nodal weight w(x,y) = x + 0.6180339887 y + 0.3 x^2
// - 0.2 y^3 + 0.1 x y (block coordinates in [0,1]), ascending, and signed so
// that sum_nodes exp(x + 1.7 y) e(x, y) > 0.
#include "common.cuh"

namespace pint {

namespace {

constexpr int BT = 256;       // threads per block CTA
constexpr int KCAP = 64;      // aux functions per block (indicators + enrichment)

struct BlkArgs {
  int n_f, nc, bs, nb, J;
  double kappa_min, kt_scale, h2;
  const double* kappa;
  double* scratch;            // per block: 4 nb^2 + 2 nb doubles + ints
  long long scratch_stride;   // doubles per block
  double* con_rows;           // [block][KCAP][nb]
  double* con_gram;           // [block][KCAP]
  int* info;                  // [block][8]: k, has_matrix, n_frac, n_enr, status, sweeps
  int block0;
};

__device__ inline double q1s(int a, int b) { return pintd::q1_stiff(a, b); }
__device__ inline double q1m(int a, int b) { return pintd::q1_mass(a, b); }

// rotation (c, s) zeroing the (p,q) entry of [[a, b],[b, d]] under J^T A J,
// J = [[c, s], [-s, c]] on rows/columns (p, q)
__device__ inline void jacobi_rot(double a, double b, double d, double& c, double& s) {
  if (b == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
  double tau = (d - a) / (2.0 * b);
  double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  c = 1.0 / sqrt(1.0 + t * t);
  s = t * c;
}

// serial cyclic Jacobi for a small symmetric matrix (n <= KCAP), row-major
// lda = n; V receives the eigenvectors (columns), lam ascending.
__device__ void small_eig(double* A, double* V, double* lam, int n) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double v = A[i * n + j] * A[i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double c, s;
        jacobi_rot(A[p * n + p], A[p * n + q], A[q * n + q], c, s);
        if (s == 0.0) continue;
        for (int k = 0; k < n; ++k) {
          double x = A[p * n + k], y = A[q * n + k];
          A[p * n + k] = c * x - s * y;
          A[q * n + k] = s * x + c * y;
        }
        for (int k = 0; k < n; ++k) {
          double x = A[k * n + p], y = A[k * n + q];
          A[k * n + p] = c * x - s * y;
          A[k * n + q] = s * x + c * y;
        }
        for (int k = 0; k < n; ++k) {
          double x = V[k * n + p], y = V[k * n + q];
          V[k * n + p] = c * x - s * y;
          V[k * n + q] = s * x + c * y;
        }
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
  // selection sort ascending, columns of V follow
  for (int i = 0; i < n; ++i) {
    int m = i;
    for (int j = i + 1; j < n; ++j)
      if (lam[j] < lam[m]) m = j;
    if (m != i) {
      double t = lam[i];
      lam[i] = lam[m];
      lam[m] = t;
      for (int k = 0; k < n; ++k) {
        double u = V[k * n + i];
        V[k * n + i] = V[k * n + m];
        V[k * n + m] = u;
      }
    }
  }
}

// block-local node (a, b) -> id b*(bs+1) + a; cell (ci, cj) -> cj*bs + ci
__device__ inline double cell_kappa(const BlkArgs& g, int bx, int by, int ci, int cj) {
  return g.kappa[(size_t)(by * g.bs + cj) * g.n_f + (bx * g.bs + ci)];
}

// y = S_b x with S_b the block-local kappa_tilde mass (only this block's cells)
__device__ double apply_sb_row(const BlkArgs& g, int bx, int by, int r, const double* x) {
  int bs = g.bs, w = bs + 1;
  int a = r % w, b = r / w;
  double acc = 0.0;
  for (int cj = b - 1; cj <= b; ++cj) {
    if (cj < 0 || cj >= bs) continue;
    for (int ci = a - 1; ci <= a; ++ci) {
      if (ci < 0 || ci >= bs) continue;
      double kt = cell_kappa(g, bx, by, ci, cj) * g.kt_scale * g.h2;
      int lx = a - ci, ly = b - cj;
      int ca = (ly == 0) ? (lx == 0 ? 0 : 1) : (lx == 1 ? 2 : 3);
      for (int cb = 0; cb < 4; ++cb) {
        int col = (cj + pintd::corner_y(cb)) * w + ci + pintd::corner_x(cb);
        acc += kt * q1m(ca, cb) * x[col];
      }
    }
  }
  return acc;
}

// y = A_b x with A_b the block-local stiffness (only this block's cells)
__device__ double apply_ab_row(const BlkArgs& g, int bx, int by, int r, const double* x) {
  int bs = g.bs, w = bs + 1;
  int a = r % w, b = r / w;
  double acc = 0.0;
  for (int cj = b - 1; cj <= b; ++cj) {
    if (cj < 0 || cj >= bs) continue;
    for (int ci = a - 1; ci <= a; ++ci) {
      if (ci < 0 || ci >= bs) continue;
      double kap = cell_kappa(g, bx, by, ci, cj);
      int lx = a - ci, ly = b - cj;
      int ca = (ly == 0) ? (lx == 0 ? 0 : 1) : (lx == 1 ? 2 : 3);
      for (int cb = 0; cb < 4; ++cb) {
        int col = (cj + pintd::corner_y(cb)) * w + ci + pintd::corner_x(cb);
        acc += kap * q1s(ca, cb) * x[col];
      }
    }
  }
  return acc;
}

// ---------------------------------------------------------------------------
// Large blocks (nb > SI_MIN_NB nodes): the J + 1 smallest pairs of eq. (3.1)
// by shift-invert subspace iteration instead of the dense Jacobi (whose
// O(nb^3) sweeps dominate setup for 32-cell blocks).  K = A_b + sigma S_b is
// banded (9-point stencil, half-bandwidth bs + 2) and factored once, K = L L^T;
// each iteration solves K Y = S_b X for the m columns of X and runs
// Rayleigh-Ritz with the exact A_b and S_b, so the Ritz vectors come out
// S-orthonormal and sorted.  The iteration stops when the leading m - 2 pairs
// have residuals ||A x - theta S x|| below 1e-12 (||A x|| + |theta| ||S x||)
// + 1e-15 lambda_max ||S x||.  lambda_max (the cluster rule's absolute scale)
// is the element bound 24 (H/h)^2: kappa cancels between A_b and the
// kappa_tilde mass, so every cell's pencil has that largest eigenvalue, and a
// uniform block attains it.
// ---------------------------------------------------------------------------
constexpr int SI_MIN_NB = 400;
constexpr int SI_EXTRA = 6;      // Ritz vectors beyond the J + 1 wanted
constexpr int SI_MAXIT = 400;
constexpr double SI_SIGMA = 1.0; // the pencil's eigenvalues are O(pi^2 (a^2 + b^2)), bs-independent

__device__ inline double si_hash(int r, int j) {
  unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(r * 64 + j + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// returns the iterations done; Ritz values into th[0..m), vectors (S-orthonormal,
// ascending) into X (column j at j nb); sets *status = 1 for a non-positive pivot
__device__ int si_eigs(const BlkArgs& g, int bx, int by, int m, double* Kb, double* X, double* Y, double* Z,
                       double* AX, double* sm, double* th, double* sh, int* status) {
  const int nb = g.nb, bs = g.bs, w1 = bs + 1, hw = bs + 2, bw = hw + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = BT / 32;
  __shared__ double s_piv;
  __shared__ int s_done;
  double* Am = sm;             // m x m
  double* Sm = Am + KCAP * KCAP;
  double* Lm = Sm + KCAP * KCAP;
  double* Wm = Lm + KCAP * KCAP;
  double* Vm = Wm + KCAP * KCAP;
  // ---- banded K = A_b + sigma S_b (row r, slot k <-> column r - hw + k) ----
  for (int e = tid; e < nb * bw; e += BT) Kb[e] = 0.0;
  __syncthreads();
  for (int r = tid; r < nb; r += BT) {
    const int a = r % w1, b = r / w1;
    for (int cj = b - 1; cj <= b; ++cj) {
      if (cj < 0 || cj >= bs) continue;
      for (int ci = a - 1; ci <= a; ++ci) {
        if (ci < 0 || ci >= bs) continue;
        const double kap = cell_kappa(g, bx, by, ci, cj), kt = kap * g.kt_scale * g.h2;
        const int lx = a - ci, ly = b - cj;
        const int ca = (ly == 0) ? (lx == 0 ? 0 : 1) : (lx == 1 ? 2 : 3);
        for (int cb = 0; cb < 4; ++cb) {
          const int col = (cj + pintd::corner_y(cb)) * w1 + ci + pintd::corner_x(cb);
          if (col <= r) Kb[(size_t)r * bw + (col - r + hw)] += kap * q1s(ca, cb) + SI_SIGMA * kt * q1m(ca, cb);
        }
      }
    }
  }
  __syncthreads();
  // ---- banded Cholesky, right-looking -------------------------------------------
  for (int k = 0; k < nb; ++k) {
    if (tid == 0) {
      double d = Kb[(size_t)k * bw + hw];
      if (!(d > 0.0)) {
        *status = 1;
        d = 1.0;
      }
      s_piv = sqrt(d);
      Kb[(size_t)k * bw + hw] = s_piv;
    }
    __syncthreads();
    const int rem = min(hw, nb - 1 - k);
    for (int t = tid; t < rem; t += BT) Kb[(size_t)(k + 1 + t) * bw + (k - (k + 1 + t) + hw)] /= s_piv;
    __syncthreads();
    for (int t = tid; t < rem * rem; t += BT) {
      const int i = k + 1 + t / rem, j = k + 1 + t % rem;
      if (j <= i)
        Kb[(size_t)i * bw + (j - i + hw)] -= Kb[(size_t)i * bw + (k - i + hw)] * Kb[(size_t)j * bw + (k - j + hw)];
    }
    __syncthreads();
  }
  // ---- start: seeded pseudo-random columns ----------------------------------
  for (int e = tid; e < nb * m; e += BT) X[e] = si_hash(e % nb, e / nb);
  __syncthreads();
  const double lmax = 24.0 * bs * bs;
  const int need = m - 2;
  int it = 0;
  for (it = 1; it <= SI_MAXIT; ++it) {
    // Z = S X; Y = K^-1 Z (a warp per column: forward then backward, row by row)
    for (int e = tid; e < nb * m; e += BT) Z[e] = apply_sb_row(g, bx, by, e % nb, X + (size_t)(e / nb) * nb);
    __syncthreads();
    for (int j = warp; j < m; j += nwarp) {
      double* y = Y + (size_t)j * nb;
      const double* z = Z + (size_t)j * nb;
      for (int i = 0; i < nb; ++i) {
        const double* Li = Kb + (size_t)i * bw;
        double acc = 0.0;
        for (int k = max(0, i - hw) + lane; k < i; k += 32) acc += Li[k - i + hw] * y[k];
        acc = pintd::warp_sum(acc);
        if (lane == 0) y[i] = (z[i] - acc) / Li[hw];
        __syncwarp();
      }
      for (int i = nb - 1; i >= 0; --i) {
        double acc = 0.0;
        for (int k = i + 1 + lane; k <= min(nb - 1, i + hw); k += 32) acc += Kb[(size_t)k * bw + (i - k + hw)] * y[k];
        acc = pintd::warp_sum(acc);
        if (lane == 0) y[i] = (y[i] - acc) / Kb[(size_t)i * bw + hw];
        __syncwarp();
      }
    }
    __syncthreads();
    // Rayleigh-Ritz on span(Y): AX = A Y, Z = S Y, Am = Y^T A Y, Sm = Y^T S Y
    for (int e = tid; e < nb * m; e += BT) {
      const double* yc = Y + (size_t)(e / nb) * nb;
      AX[e] = apply_ab_row(g, bx, by, e % nb, yc);
      Z[e] = apply_sb_row(g, bx, by, e % nb, yc);
    }
    __syncthreads();
    for (int pq = warp; pq < m * m; pq += nwarp) {
      const int p = pq / m, q = pq % m;
      if (q < p) continue;
      double aa = 0.0, ss = 0.0;
      for (int r = lane; r < nb; r += 32) {
        const double yp = Y[(size_t)p * nb + r];
        aa += yp * AX[(size_t)q * nb + r];
        ss += yp * Z[(size_t)q * nb + r];
      }
      aa = pintd::warp_sum(aa);
      ss = pintd::warp_sum(ss);
      if (lane == 0) {
        Am[p * m + q] = Am[q * m + p] = aa;
        Sm[p * m + q] = Sm[q * m + p] = ss;
      }
    }
    __syncthreads();
    if (tid == 0) {
      // Sm = L L^T, C = L^-1 Am L^-T, C = W diag(th) W^T, V = L^-T W
      for (int k = 0; k < m; ++k) {
        double d = Sm[k * m + k];
        for (int t = 0; t < k; ++t) d -= Lm[k * m + t] * Lm[k * m + t];
        d = sqrt(fmax(d, 1e-300));
        Lm[k * m + k] = d;
        for (int i = k + 1; i < m; ++i) {
          double v = Sm[i * m + k];
          for (int t = 0; t < k; ++t) v -= Lm[i * m + t] * Lm[k * m + t];
          Lm[i * m + k] = v / d;
        }
        for (int i = 0; i < k; ++i) Lm[i * m + k] = 0.0;
      }
      for (int col = 0; col < m; ++col)  // Wm = L^-1 Am (column col)
        for (int i = 0; i < m; ++i) {
          double v = Am[i * m + col];
          for (int t = 0; t < i; ++t) v -= Lm[i * m + t] * Wm[t * m + col];
          Wm[i * m + col] = v / Lm[i * m + i];
        }
      for (int col = 0; col < m; ++col)  // C = L^-1 (L^-1 Am)^T, symmetric
        for (int i = 0; i < m; ++i) {
          double v = Wm[col * m + i];
          for (int t = 0; t < i; ++t) v -= Lm[i * m + t] * Am[t * m + col];
          Am[i * m + col] = v / Lm[i * m + i];
        }
      for (int i = 0; i < m; ++i)
        for (int j = i + 1; j < m; ++j) {
          const double v = 0.5 * (Am[i * m + j] + Am[j * m + i]);
          Am[i * m + j] = Am[j * m + i] = v;
        }
      small_eig(Am, Wm, th, m);
      for (int col = 0; col < m; ++col)  // V = L^-T W
        for (int i = m - 1; i >= 0; --i) {
          double v = Wm[i * m + col];
          for (int t = i + 1; t < m; ++t) v -= Lm[t * m + i] * Vm[t * m + col];
          Vm[i * m + col] = v / Lm[i * m + i];
        }
    }
    __syncthreads();
    // X = Y V; the residuals of the new Ritz pairs from A Y V and S Y V
    for (int e = tid; e < nb * m; e += BT) {
      const int r = e % nb, j = e / nb;
      double x = 0.0;
      for (int t = 0; t < m; ++t) x += Y[(size_t)t * nb + r] * Vm[t * m + j];
      X[e] = x;
    }
    if (tid == 0) s_done = 1;
    __syncthreads();
    for (int j = 0; j < need; ++j) {
      double rr = 0.0, a2 = 0.0, s2 = 0.0;
      for (int r = tid; r < nb; r += BT) {
        double ax = 0.0, sx = 0.0;
        for (int t = 0; t < m; ++t) {
          ax += AX[(size_t)t * nb + r] * Vm[t * m + j];
          sx += Z[(size_t)t * nb + r] * Vm[t * m + j];
        }
        const double res = ax - th[j] * sx;
        rr += res * res;
        a2 += ax * ax;
        s2 += sx * sx;
      }
      rr = pintd::block_sum(rr, sh);
      a2 = pintd::block_sum(a2, sh);
      s2 = pintd::block_sum(s2, sh);
      const double tol = 1e-12 * (sqrt(a2) + fabs(th[j]) * sqrt(s2)) + 1e-15 * lmax * sqrt(s2);
      if (tid == 0 && !(sqrt(rr) <= tol)) s_done = 0;
    }
    __syncthreads();
    if (s_done) break;
  }
  return min(it, SI_MAXIT);
}

__device__ inline int rr_player(int k, int r, int m) {
  // circle method: position k of round r (player 0 fixed)
  return k == 0 ? 0 : 1 + ((k - 1 + r) % (m - 1));
}

__global__ void __launch_bounds__(BT) k_block_setup(BlkArgs g) {
  const int blk = g.block0 + blockIdx.x;
  const int bx = blk % g.nc, by = blk / g.nc;
  const int nb = g.nb, bs = g.bs, w1 = bs + 1;
  const int tid = threadIdx.x;
  double* base = g.scratch + (size_t)blockIdx.x * g.scratch_stride;
  double* Cm = base;                   // A -> C
  double* Lm = Cm + (size_t)nb * nb;   // S -> L
  double* Vm = Lm + (size_t)nb * nb;   // Jacobi vectors
  double* Tm = Vm + (size_t)nb * nb;   // temp / Phi
  double* lam = Tm + (size_t)nb * nb;  // nb
  double* lsort = lam + nb;            // nb
  int* perm = (int*)(lsort + nb);      // nb
  int* label = perm + nb;              // bs*bs
  int* stack = label + bs * bs;        // bs*bs
  double* R = (double*)(stack + bs * bs + 2);  // KCAP * nb (aligned enough: +2 ints)
  R = (double*)(((uintptr_t)R + 7) & ~(uintptr_t)7);
  double* work = R + (size_t)KCAP * nb;        // small matrices: 4 * KCAP^2 + KCAP*nb*2
  __shared__ double sh[64];
  __shared__ double rc[1200], rs_[1200];
  __shared__ int rp[2400];
  __shared__ int s_nsel, s_kind, s_nfrac, s_hasm, s_ne, s_status;
  __shared__ double s_G[KCAP];
  __shared__ int s_keep[KCAP];

  if (tid == 0) s_status = 0;
  const bool use_si = nb > SI_MIN_NB;
  const int m_si = min(nb, g.J + 1 + SI_EXTRA);
  int sweeps = 0;
  if (use_si) {
    // ---- large block: shift-invert subspace iteration (see si_eigs) ---------
    if (g.J > 0) {
      double* X = Lm;
      double* Y = X + (size_t)nb * m_si;
      double* Z = Y + (size_t)nb * m_si;
      double* AXs = Z + (size_t)nb * m_si;
      sweeps = si_eigs(g, bx, by, m_si, Cm, X, Y, Z, AXs, Vm, lam, sh, &s_status);
      for (int e = tid; e < nb * m_si; e += BT) {
        const int r = e % nb, j = e / nb;
        Tm[(size_t)r * nb + j] = X[e];
      }
      for (int j = tid; j < m_si; j += BT) {
        perm[j] = j;
        lsort[j] = lam[j];
      }
    }
    __syncthreads();
  } else {
  // ---- assemble dense A_b and S_b (eq. (3.1)), one row per thread --------
  for (size_t e = tid; e < (size_t)nb * nb; e += BT) {
    Cm[e] = 0.0;
    Lm[e] = 0.0;
  }
  __syncthreads();
  for (int r = tid; r < nb; r += BT) {
    int a = r % w1, b = r / w1;
    for (int cj = b - 1; cj <= b; ++cj) {
      if (cj < 0 || cj >= bs) continue;
      for (int ci = a - 1; ci <= a; ++ci) {
        if (ci < 0 || ci >= bs) continue;
        double kap = cell_kappa(g, bx, by, ci, cj);
        double kt = kap * g.kt_scale * g.h2;
        int lx = a - ci, ly = b - cj;
        int ca = (ly == 0) ? (lx == 0 ? 0 : 1) : (lx == 1 ? 2 : 3);
        for (int cb = 0; cb < 4; ++cb) {
          int col = (cj + pintd::corner_y(cb)) * w1 + ci + pintd::corner_x(cb);
          Cm[(size_t)r * nb + col] += kap * q1s(ca, cb);
          Lm[(size_t)r * nb + col] += kt * q1m(ca, cb);
        }
      }
    }
  }
  __syncthreads();
  // ---- Cholesky S = L L^T (right-looking) -----------------------------------
  for (int k = 0; k < nb; ++k) {
    if (tid == 0) {
      double d = Lm[(size_t)k * nb + k];
      if (!(d > 0.0)) {
        s_status = 1;
        d = 1.0;
      }
      Lm[(size_t)k * nb + k] = sqrt(d);
    }
    __syncthreads();
    double piv = Lm[(size_t)k * nb + k];
    for (int i = k + 1 + tid; i < nb; i += BT) Lm[(size_t)i * nb + k] /= piv;
    __syncthreads();
    int rem = nb - k - 1;
    for (int idx = tid; idx < rem * rem; idx += BT) {
      int i = k + 1 + idx / rem, j = k + 1 + idx % rem;
      if (j <= i) Lm[(size_t)i * nb + j] -= Lm[(size_t)i * nb + k] * Lm[(size_t)j * nb + k];
    }
    __syncthreads();
  }
  // ---- C = L^-1 A L^-T: T = L^-1 A (columns), C = L^-1 T^T ------------------
  for (int j = tid; j < nb; j += BT) {
    for (int i = 0; i < nb; ++i) {
      double t = Cm[(size_t)i * nb + j];
      for (int k = 0; k < i; ++k) t -= Lm[(size_t)i * nb + k] * Tm[(size_t)k * nb + j];
      Tm[(size_t)i * nb + j] = t / Lm[(size_t)i * nb + i];
    }
  }
  __syncthreads();
  for (int j = tid; j < nb; j += BT) {
    for (int i = 0; i < nb; ++i) {
      double t = Tm[(size_t)j * nb + i];
      for (int k = 0; k < i; ++k) t -= Lm[(size_t)i * nb + k] * Cm[(size_t)k * nb + j];
      Cm[(size_t)i * nb + j] = t / Lm[(size_t)i * nb + i];
    }
  }
  __syncthreads();
  for (size_t e = tid; e < (size_t)nb * nb; e += BT) {
    int i = (int)(e / nb), j = (int)(e % nb);
    if (i < j) {
      double v = 0.5 * (Cm[(size_t)i * nb + j] + Cm[(size_t)j * nb + i]);
      Cm[(size_t)i * nb + j] = v;
      Cm[(size_t)j * nb + i] = v;
    }
    Vm[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // ---- parallel cyclic Jacobi ----------------------------------------------
  const int m = nb + (nb & 1);
  const int npair = m / 2;
  double prev_off = 1e300;
  for (; sweeps < 40; ++sweeps) {
    double off = 0.0, tot = 0.0;
    for (size_t e = tid; e < (size_t)nb * nb; e += BT) {
      double v = Cm[e] * Cm[e];
      tot += v;
      if (e / nb != e % nb) off += v;
    }
    off = pintd::block_sum(off, sh);
    tot = pintd::block_sum(tot, sh);
    // converged, or (once in the quadratic phase) stalled at the rounding floor
    if (off == 0.0 || off <= 1e-30 * tot || (off <= 1e-20 * tot && off > 0.25 * prev_off)) break;
    prev_off = off;
    for (int r = 0; r < m - 1; ++r) {
      for (int k = tid; k < npair; k += BT) {
        int x = rr_player(k, r, m), y = rr_player(m - 1 - k, r, m);
        int p = min(x, y), q = max(x, y);
        double c = 1.0, s = 0.0;
        if (q < nb)
          jacobi_rot(Cm[(size_t)p * nb + p], Cm[(size_t)p * nb + q], Cm[(size_t)q * nb + q], c, s);
        rc[k] = c;
        rs_[k] = s;
        rp[2 * k] = p;
        rp[2 * k + 1] = (q < nb) ? q : -1;
      }
      __syncthreads();
      // rows p, q of C
      for (int idx = tid; idx < npair * nb; idx += BT) {
        int k = idx / nb, j = idx % nb;
        int p = rp[2 * k], q = rp[2 * k + 1];
        if (q < 0 || rs_[k] == 0.0) continue;
        double c = rc[k], s = rs_[k];
        double xv = Cm[(size_t)p * nb + j], yv = Cm[(size_t)q * nb + j];
        Cm[(size_t)p * nb + j] = c * xv - s * yv;
        Cm[(size_t)q * nb + j] = s * xv + c * yv;
      }
      __syncthreads();
      // columns p, q of C and V
      for (int idx = tid; idx < npair * nb; idx += BT) {
        int k = idx / nb, i = idx % nb;
        int p = rp[2 * k], q = rp[2 * k + 1];
        if (q < 0 || rs_[k] == 0.0) continue;
        double c = rc[k], s = rs_[k];
        double xv = Cm[(size_t)i * nb + p], yv = Cm[(size_t)i * nb + q];
        Cm[(size_t)i * nb + p] = c * xv - s * yv;
        Cm[(size_t)i * nb + q] = s * xv + c * yv;
        xv = Vm[(size_t)i * nb + p];
        yv = Vm[(size_t)i * nb + q];
        Vm[(size_t)i * nb + p] = c * xv - s * yv;
        Vm[(size_t)i * nb + q] = s * xv + c * yv;
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < nb; i += BT) lam[i] = Cm[(size_t)i * nb + i];
  __syncthreads();
  // ---- Phi = L^-T V (back substitution per column), into Tm ------------------
  for (int j = tid; j < nb; j += BT) {
    for (int i = nb - 1; i >= 0; --i) {
      double t = Vm[(size_t)i * nb + j];
      for (int k = i + 1; k < nb; ++k) t -= Lm[(size_t)k * nb + i] * Tm[(size_t)k * nb + j];
      Tm[(size_t)i * nb + j] = t / Lm[(size_t)i * nb + i];
    }
  }
  // ---- sort eigenvalues ascending (rank sort) --------------------------------
  for (int i = tid; i < nb; i += BT) {
    double li = lam[i];
    int rk = 0;
    for (int j = 0; j < nb; ++j) {
      double lj = lam[j];
      rk += (lj < li) || (lj == li && j < i);
    }
    perm[rk] = i;
    lsort[rk] = li;
  }
  __syncthreads();
  }  // dense path
  // ---- selection with cluster completion; continua by flood fill ------------
  if (tid == 0) {
    // eigenpairs available to the rule: all (dense) or the converged Ritz pairs
    const int navail = use_si ? m_si - 2 : nb;
    int nsel = (g.J > 0) ? min(g.J + 1, navail) : 0;
    const double lmax = use_si ? 24.0 * bs * bs : fabs(lsort[nb - 1]);
    while (nsel > 0 && nsel < navail &&
           lsort[nsel] - lsort[nsel - 1] <= 1e-8 * fabs(lsort[nsel]) + 1e-12 * lmax)
      ++nsel;
    if (use_si && g.J > 0 && nsel >= navail) s_status = 3;  // a cluster wider than the Ritz pairs
    s_nsel = nsel;
    int hasm = 0;
    for (int c = 0; c < bs * bs; ++c) {
      double kap = cell_kappa(g, bx, by, c % bs, c / bs);
      bool mat = (kap == g.kappa_min);
      label[c] = mat ? 0 : -1;
      hasm |= mat ? 1 : 0;
    }
    int nfr = 0;
    for (int c0 = 0; c0 < bs * bs; ++c0) {
      if (label[c0] != -1) continue;
      int lab = hasm + nfr;
      ++nfr;
      int top = 0;
      stack[top++] = c0;
      label[c0] = lab;
      while (top > 0) {
        int c = stack[--top];
        int cx = c % bs, cy = c / bs;
        const int nx[4] = {cx, cx, cx - 1, cx + 1}, ny[4] = {cy - 1, cy + 1, cy, cy};
        for (int t = 0; t < 4; ++t) {
          if (nx[t] < 0 || nx[t] >= bs || ny[t] < 0 || ny[t] >= bs) continue;
          int cc = ny[t] * bs + nx[t];
          if (label[cc] == -1) {
            label[cc] = lab;
            stack[top++] = cc;
          }
        }
      }
    }
    // matrix cells were labelled 0 before fracture labels were assigned;
    // with no matrix the fracture labels start at 0 as well
    s_hasm = hasm;
    s_nfrac = nfr;
    s_kind = hasm + nfr;
    if (s_kind + nsel > KCAP) s_status = 2;
    for (int q = 0; q < KCAP; ++q) s_G[q] = 0.0;
    if (s_status == 0)
      for (int c = 0; c < bs * bs; ++c)
        s_G[label[c]] += cell_kappa(g, bx, by, c % bs, c / bs) * g.kt_scale * g.h2;
  }
  __syncthreads();
  if (s_status != 0) {
    if (tid == 0) {
      g.info[blk * 8 + 4] = s_status;
      g.info[blk * 8 + 0] = 0;
    }
    return;
  }
  const int kind = s_kind, nsel = s_nsel;
  // ---- indicator functionals r_C(node) = sum_{cells c in C at node} kt_c h^2/4
  for (int idx = tid; idx < kind * nb; idx += BT) {
    int q = idx / nb, r = idx % nb;
    int a = r % w1, b = r / w1;
    double acc = 0.0;
    for (int cj = b - 1; cj <= b; ++cj) {
      if (cj < 0 || cj >= bs) continue;
      for (int ci = a - 1; ci <= a; ++ci) {
        if (ci < 0 || ci >= bs) continue;
        if (label[cj * bs + ci] == q) acc += cell_kappa(g, bx, by, ci, cj) * g.kt_scale * g.h2 * 0.25;
      }
    }
    R[(size_t)q * nb + r] = acc;
  }
  __syncthreads();
  // ---- enrichment -----------------------------------------------------------
  double* RV = work;                        // kind x nsel
  double* Gp = RV + KCAP * KCAP;            // nsel x nsel
  double* U = Gp + KCAP * KCAP;             // nsel x nsel
  double* sig = U + KCAP * KCAP;            // KCAP
  double* C0 = sig + KCAP;                  // nsel x ne
  double* Rw = C0 + KCAP * KCAP;            // ne x ne
  double* E = Rw + KCAP * KCAP;             // ne x ne
  double* Vn = E + KCAP * KCAP;             // nb x ne (nodal parts)
  double* En = Vn + (size_t)KCAP * nb;      // nb x ne (final enrichment nodal)
  for (int idx = tid; idx < kind * nsel; idx += BT) {
    int q = idx / nsel, s = idx % nsel;
    int col = perm[s];
    double acc = 0.0;
    for (int r = 0; r < nb; ++r) acc += R[(size_t)q * nb + r] * Tm[(size_t)r * nb + col];
    RV[q * KCAP + s] = acc;
  }
  __syncthreads();
  if (tid == 0) {
    for (int a = 0; a < nsel; ++a)
      for (int b = 0; b < nsel; ++b) {
        double acc = (a == b) ? 1.0 : 0.0;
        for (int q = 0; q < kind; ++q) acc -= RV[q * KCAP + a] * RV[q * KCAP + b] / s_G[q];
        Gp[a * nsel + b] = acc;
      }
    for (int a = 0; a < nsel; ++a)
      for (int b = a + 1; b < nsel; ++b) {
        double v = 0.5 * (Gp[a * nsel + b] + Gp[b * nsel + a]);
        Gp[a * nsel + b] = Gp[b * nsel + a] = v;
      }
    small_eig(Gp, U, sig, nsel);
    int ne = 0;
    for (int a = 0; a < nsel; ++a)
      if (sig[a] > 1e-8) s_keep[ne++] = a;
    s_ne = ne;
    for (int a = 0; a < nsel; ++a)
      for (int e = 0; e < ne; ++e) C0[a * KCAP + e] = U[a * nsel + s_keep[e]] / sqrt(sig[s_keep[e]]);
  }
  __syncthreads();
  const int ne = s_ne;
  for (int idx = tid; idx < nb * ne; idx += BT) {
    int r = idx / ne, e = idx % ne;
    double acc = 0.0;
    for (int s = 0; s < nsel; ++s) acc += Tm[(size_t)r * nb + perm[s]] * C0[s * KCAP + e];
    Vn[(size_t)r * KCAP + e] = acc;
  }
  __syncthreads();
  for (int idx = tid; idx < ne * ne; idx += BT) {
    int a = idx / ne, b = idx % ne;
    double acc = 0.0;
    for (int r = 0; r < nb; ++r) {
      double xl = (double)(r % w1) / bs, yl = (double)(r / w1) / bs;
      double wgt = xl + 0.6180339887 * yl + 0.3 * xl * xl - 0.2 * yl * yl * yl + 0.1 * xl * yl;
      acc += Vn[(size_t)r * KCAP + a] * wgt * Vn[(size_t)r * KCAP + b];
    }
    Rw[a * ne + b] = acc;
  }
  __syncthreads();
  if (tid == 0 && ne > 0) {
    for (int a = 0; a < ne; ++a)
      for (int b = a + 1; b < ne; ++b) {
        double v = 0.5 * (Rw[a * ne + b] + Rw[b * ne + a]);
        Rw[a * ne + b] = Rw[b * ne + a] = v;
      }
    small_eig(Rw, E, sig, ne);
  }
  __syncthreads();
  for (int idx = tid; idx < nb * ne; idx += BT) {
    int r = idx / ne, e = idx % ne;
    double acc = 0.0;
    for (int f = 0; f < ne; ++f) acc += Vn[(size_t)r * KCAP + f] * E[f * ne + e];
    En[(size_t)r * KCAP + e] = acc;
  }
  __syncthreads();
  for (int e = 0; e < ne; ++e) {
    double acc = 0.0;
    for (int r = tid; r < nb; r += BT) {
      double xl = (double)(r % w1) / bs, yl = (double)(r / w1) / bs;
      acc += exp(xl + 1.7 * yl) * En[(size_t)r * KCAP + e];
    }
    acc = pintd::block_sum(acc, sh);
    if (acc < 0.0)
      for (int r = tid; r < nb; r += BT) En[(size_t)r * KCAP + e] = -En[(size_t)r * KCAP + e];
    __syncthreads();
  }
  // ---- constraint rows: indicators, then S_b e - sum_C a_C r_C -------------
  double* rows = g.con_rows + (size_t)blk * KCAP * nb;
  for (int idx = tid; idx < kind * nb; idx += BT) rows[idx] = R[idx];
  if (tid < KCAP) g.con_gram[(size_t)blk * KCAP + tid] = (tid < kind) ? s_G[tid] : (tid < kind + ne ? 1.0 : 0.0);
  __syncthreads();
  double* ecol = Vn;  // reuse: contiguous copy of one enrichment function
  for (int e = 0; e < ne; ++e) {
    for (int r = tid; r < nb; r += BT) ecol[r] = En[(size_t)r * KCAP + e];
    __syncthreads();
    // a_C = r_C . e / G_C
    for (int q = 0; q < kind; ++q) {
      double acc = 0.0;
      for (int r = tid; r < nb; r += BT) acc += R[(size_t)q * nb + r] * ecol[r];
      acc = pintd::block_sum(acc, sh);
      if (tid == 0) sig[q] = acc / s_G[q];
      __syncthreads();
    }
    for (int r = tid; r < nb; r += BT) {
      double v = apply_sb_row(g, bx, by, r, ecol);
      for (int q = 0; q < kind; ++q) v -= sig[q] * R[(size_t)q * nb + r];
      rows[(size_t)(kind + e) * nb + r] = v;
    }
    __syncthreads();
  }
  if (tid == 0) {
    int* inf = g.info + blk * 8;
    inf[0] = kind + ne;
    inf[1] = s_hasm;
    inf[2] = s_nfrac;
    inf[3] = ne;
    inf[4] = 0;
    inf[5] = sweeps;
    inf[6] = nsel;
  }
}

__global__ void k_scale(double* x, size_t n, double s) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= s;
}

// minimum of x (single CTA; every thread holds a finite partial minimum)
__global__ void k_min(const double* x, int n, double* out) {
  __shared__ double sh[1024];
  double m = 1e300;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmin(m, x[i]);
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

}  // namespace

void build_blocks(Ctx* c) {
  const int nb = c->nb;
  c->kmax = KCAP;
  PINT_REQUIRE(nb <= 2 * 1200 - 2, PINT_ERR_BAD_ARG, "coarse block too large (n_f/nc <= 48)");
  // s uses kappa_tilde = kappa H^-2: rescale the global s-stencil
  double kts = (double)c->nc * c->nc;
  size_t ns = (size_t)c->nn * 9;
  k_scale<<<(unsigned)((ns + 255) / 256), 256, 0, c->stream>>>(c->stS, ns, kts);
  PINT_LAUNCH_CHECK();
  double* dmin = (double*)dalloc(c, sizeof(double));
  k_min<<<1, 1024, 0, c->stream>>>(c->kappa, c->n_f * c->n_f, dmin);
  PINT_LAUNCH_CHECK();
  double kmin = 0;
  PINT_CUDA(cudaMemcpyAsync(&kmin, dmin, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PINT_CUDA(cudaStreamSynchronize(c->stream));
  dfree(c, dmin);

  c->con_rows = (double*)dalloc(c, (size_t)c->n_blocks * KCAP * nb * sizeof(double));
  c->con_gram = (double*)dalloc(c, (size_t)c->n_blocks * KCAP * sizeof(double));
  int* dinfo = (int*)dalloc(c, (size_t)c->n_blocks * 8 * sizeof(int));
  PINT_CUDA(cudaMemsetAsync(c->con_rows, 0, (size_t)c->n_blocks * KCAP * nb * sizeof(double), c->stream));
  PINT_CUDA(cudaMemsetAsync(dinfo, 0, (size_t)c->n_blocks * 8 * sizeof(int), c->stream));
  long long stride = 4LL * nb * nb + 2LL * nb + (nb + 2LL * c->bs * c->bs + 8) / 2 + 2 +
                     (long long)KCAP * nb + 8LL * KCAP * KCAP + 2LL * KCAP * nb + KCAP + 16;
  // batch so that scratch stays below ~8 GB
  long long per = stride * (long long)sizeof(double);
  int batch = (int)std::max<long long>(1, std::min<long long>(c->n_blocks, (8LL << 30) / per));
  double* scratch = (double*)dalloc(c, (size_t)per * batch);
  BlkArgs g;
  g.n_f = c->n_f;
  g.nc = c->nc;
  g.bs = c->bs;
  g.nb = nb;
  g.J = c->J;
  g.kappa_min = kmin;
  g.kt_scale = kts;
  g.h2 = 1.0 / ((double)c->n_f * c->n_f);
  g.kappa = c->kappa;
  g.scratch = scratch;
  g.scratch_stride = stride;
  g.con_rows = c->con_rows;
  g.con_gram = c->con_gram;
  g.info = dinfo;
  for (int b0 = 0; b0 < c->n_blocks; b0 += batch) {
    g.block0 = b0;
    int nblk = std::min(batch, c->n_blocks - b0);
    k_block_setup<<<nblk, BT, 0, c->stream>>>(g);
    PINT_LAUNCH_CHECK();
  }
  std::vector<int> info((size_t)c->n_blocks * 8);
  PINT_CUDA(cudaMemcpyAsync(info.data(), dinfo, info.size() * sizeof(int), cudaMemcpyDeviceToHost,
                            c->stream));
  PINT_CUDA(cudaStreamSynchronize(c->stream));
  dfree(c, scratch);
  dfree(c, dinfo);
  c->blk_k.assign(c->n_blocks, 0);
  c->blk_kind_off.assign(c->n_blocks, 0);
  c->kind.clear();
  c->owner.clear();
  c->L = 0;
  int off = 0;
  for (int b = 0; b < c->n_blocks; ++b) {
    const int* inf = &info[(size_t)b * 8];
    PINT_REQUIRE(inf[4] != 1, PINT_ERR_SINGULAR, "block s-mass matrix not positive definite");
    PINT_REQUIRE(inf[4] != 2, PINT_ERR_BAD_ARG, "too many continua + enrichment functions in a block");
    PINT_REQUIRE(inf[4] != 3, PINT_ERR_BAD_ARG,
                 "eigenvalue cluster of a block wider than its subspace iteration (raise J or use smaller blocks)");
    c->blk_k[b] = inf[0];
    c->blk_kind_off[b] = off;
    off += inf[0];
    if (inf[1]) {
      c->kind.push_back(0);
      c->owner.push_back(b);
    }
    for (int f = 0; f < inf[2]; ++f) {
      c->kind.push_back(1);
      c->owner.push_back(b);
    }
    for (int e = 0; e < inf[3]; ++e) {
      c->kind.push_back(2);
      c->owner.push_back(b);
    }
    c->L += inf[2];
  }
  c->n_raw = off;
}

}  // namespace pint
