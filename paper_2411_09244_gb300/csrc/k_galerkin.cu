// Galerkin projections of eq. (3.8) and the V_H1 / V_H2 split of eq. (3.7).
//
// Every raw basis (matrix, fracture or enrichment CEM basis) lives on its
// window's interior nodes.  The raw Gram matrices G_X = Psi_all^T X Psi_all,
// X in {M_f, A_f, s}, are formed window pair by window pair: X Psi_b is
// evaluated once on the closure of b's window (9-point stencils), then dotted
// with Psi_a over the overlap.  The split is a sparse change of basis of the
// raw bases,
//   V_H1: psi_tilde_r = psi_r - coef_r psi_bar  (fracture and enrichment r,
//         the last fracture basis dropped),
//   V_H2: psi_bar = sum_fracture psi_r / L, then the matrix bases,
// so M11 = T1^T G_M T1 etc. are evaluated with rank-one corrections.
#include "common.cuh"

#include <algorithm>
#include <mutex>

namespace pint {

namespace {

struct GWin {
  int X0, Y0, wx, wy, nw, kt, raw0, pad;
  long long psi_off, xpsi_off;
};

// X Psi_b on the closure (wx+2) x (wy+2) of b's window, for X = A, M, s
__global__ void k_xpsi(const GWin* __restrict__ gw, int n_f, const double* __restrict__ stA,
                       const double* __restrict__ stM, const double* __restrict__ stS,
                       const double* __restrict__ psi, double* __restrict__ xpsi,
                       long long xstride) {
  const GWin W = gw[blockIdx.y];
  const int cw = W.wx + 2, ch = W.wy + 2, ncl = cw * ch;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ncl * W.kt; e += gridDim.x * blockDim.x) {
    int q = e / ncl, l = e % ncl;
    int cx = l % cw, cy = l / cw;           // closure coords, interior starts at (1,1)
    int gx = W.X0 - 1 + cx, gy = W.Y0 - 1 + cy;
    double a = 0, m = 0, s = 0;
    if (gx >= 0 && gx <= n_f && gy >= 0 && gy <= n_f) {
      int node = gy * (n_f + 1) + gx;
      const double* ps = psi + W.psi_off + (size_t)q * W.nw;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int ix = cx - 1 + dx, iy = cy - 1 + dy;  // interior coords
          if (ix < 0 || ix >= W.wx || iy < 0 || iy >= W.wy) continue;
          double v = ps[iy * W.wx + ix];
          int k = (dy + 1) * 3 + (dx + 1);
          a += stA[(size_t)node * 9 + k] * v;
          m += stM[(size_t)node * 9 + k] * v;
          s += stS[(size_t)node * 9 + k] * v;
        }
    }
    size_t o = W.xpsi_off + (size_t)q * ncl + l;
    xpsi[o] = a;
    xpsi[o + xstride] = m;
    xpsi[o + 2 * xstride] = s;
  }
}

constexpr int KA = 24;  // max bases per window handled by the pair kernel

// G_X[raw_a][raw_b] for all a of window wa and one b of window wb
__global__ void __launch_bounds__(256) k_pair(const GWin* __restrict__ gw, const int2* __restrict__ pairs,
                                              const double* __restrict__ psi,
                                              const double* __restrict__ xpsi, long long xstride,
                                              int n_raw, double* __restrict__ GA,
                                              double* __restrict__ GM, double* __restrict__ GS) {
  const int2 pr = pairs[blockIdx.x];
  const GWin A = gw[pr.x], B = gw[pr.y];
  const int qb = blockIdx.y;
  if (qb >= B.kt) return;
  // overlap of A's interior with B's closure, in global node coords
  int x0 = max(A.X0, B.X0 - 1), x1 = min(A.X0 + A.wx - 1, B.X0 + B.wx);
  int y0 = max(A.Y0, B.Y0 - 1), y1 = min(A.Y0 + A.wy - 1, B.Y0 + B.wy);
  double acc[3][KA];
#pragma unroll
  for (int t = 0; t < KA; ++t) acc[0][t] = acc[1][t] = acc[2][t] = 0.0;
  const int ox = x1 - x0 + 1, oy = y1 - y0 + 1;
  const int cwB = B.wx + 2;
  const double* xb = xpsi + B.xpsi_off + (size_t)qb * cwB * (B.wy + 2);
  if (ox > 0 && oy > 0) {
    for (int e = threadIdx.x; e < ox * oy; e += blockDim.x) {
      int gx = x0 + e % ox, gy = y0 + e / ox;
      int lb = (gy - B.Y0 + 1) * cwB + (gx - B.X0 + 1);
      double va = xb[lb], vm = xb[lb + xstride], vs = xb[lb + 2 * xstride];
      int la = (gy - A.Y0) * A.wx + (gx - A.X0);
#pragma unroll
      for (int t = 0; t < KA; ++t) {
        if (t < A.kt) {
          double p = psi[A.psi_off + (size_t)t * A.nw + la];
          acc[0][t] += p * va;
          acc[1][t] += p * vm;
          acc[2][t] += p * vs;
        }
      }
    }
  }
  __shared__ double sh[64];
  for (int t = 0; t < A.kt; ++t) {
    double s0 = pintd::block_sum(acc[0][t], sh);
    double s1 = pintd::block_sum(acc[1][t], sh);
    double s2 = pintd::block_sum(acc[2][t], sh);
    if (threadIdx.x == 0) {
      size_t o = (size_t)(A.raw0 + t) * n_raw + (B.raw0 + qb);
      GA[o] = s0;
      GM[o] = s1;
      GS[o] = s2;
    }
  }
}

// out[v][raw] = sum_nodes psi_raw(node) vec_v(node).  Vectors go two at a
// time through one read of the basis function (the bases are the largest
// array read); each vector's sum keeps the same order either way.
__global__ void k_raw_dot(const GWin* __restrict__ gw, int n_f, const double* __restrict__ psi,
                          const double* __restrict__ vec, int count, int n_raw,
                          double* __restrict__ out) {
  const GWin W = gw[blockIdx.x];
  const int q = blockIdx.y;
  if (q >= W.kt) return;
  const int nn = (n_f + 1) * (n_f + 1);
  __shared__ double sh[64];
  for (int v = 0; v < count; v += 2) {
    const bool two = v + 1 < count;
    const double* x0 = vec + (size_t)v * nn;
    const double* x1 = two ? x0 + nn : x0;
    double a0 = 0.0, a1 = 0.0;
    for (int l = threadIdx.x; l < W.nw; l += blockDim.x) {
      const int gx = W.X0 + l % W.wx, gy = W.Y0 + l / W.wx, node = gy * (n_f + 1) + gx;
      const double p = psi[W.psi_off + (size_t)q * W.nw + l];
      a0 += p * x0[node];
      if (two) a1 += p * x1[node];
    }
    a0 = pintd::block_sum(a0, sh);
    if (threadIdx.x == 0) out[(size_t)v * n_raw + W.raw0 + q] = a0;
    if (two) {
      a1 = pintd::block_sum(a1, sh);
      if (threadIdx.x == 0) out[(size_t)(v + 1) * n_raw + W.raw0 + q] = a1;
    }
  }
}

// gb = G beta, with beta = 1/L on fracture raws
__global__ void k_gbeta(const double* __restrict__ G, const int* __restrict__ kind, int n_raw,
                        double invL, double* __restrict__ gb) {
  int r = blockIdx.x;
  __shared__ double sh[64];
  double acc = 0.0;
  for (int c = threadIdx.x; c < n_raw; c += blockDim.x)
    if (kind[c] == 1) acc += G[(size_t)r * n_raw + c] * invL;
  acc = pintd::block_sum(acc, sh);
  if (threadIdx.x == 0) gb[r] = acc;
}

// bGb = beta^T G beta and coef_r = (G_S beta)_r / (beta^T G_S beta)
__global__ void k_bgb(const double* __restrict__ gbM, const double* __restrict__ gbA,
                      const double* __restrict__ gbS, const int* __restrict__ kind, int n_raw,
                      double invL, double* __restrict__ scal, double* __restrict__ coef) {
  __shared__ double sh[64];
  double m = 0, a = 0, s = 0;
  for (int c = threadIdx.x; c < n_raw; c += blockDim.x)
    if (kind[c] == 1) {
      m += gbM[c] * invL;
      a += gbA[c] * invL;
      s += gbS[c] * invL;
    }
  m = pintd::block_sum(m, sh);
  a = pintd::block_sum(a, sh);
  s = pintd::block_sum(s, sh);
  if (threadIdx.x == 0) {
    scal[0] = m;
    scal[1] = a;
    scal[2] = s;
  }
  for (int c = threadIdx.x; c < n_raw; c += blockDim.x) coef[c] = (kind[c] >= 1) ? gbS[c] / s : 0.0;
}

// reduced blocks of X from G_X (see file header); has_bar selects the L > 0 form
__global__ void k_reduce(const double* __restrict__ G, const double* __restrict__ gb,
                         const double* __restrict__ scal, int which, const double* __restrict__ coef,
                         const int* __restrict__ h1, int d1, const int* __restrict__ h2m, int nm,
                         int has_bar, int n_raw, double* __restrict__ X11,
                         double* __restrict__ X12, double* __restrict__ X22) {
  const int d2 = nm + has_bar;
  const double bgb = has_bar ? scal[which] : 0.0;
  long long tot = (long long)d1 * d1 + (long long)d1 * d2 + (long long)d2 * d2;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < (long long)d1 * d1) {
      int i = (int)(e / d1), j = (int)(e % d1);
      int ri = h1[i], rj = h1[j];
      double v = G[(size_t)ri * n_raw + rj];
      if (has_bar)
        v += -gb[ri] * coef[rj] - coef[ri] * gb[rj] + bgb * coef[ri] * coef[rj];
      X11[e] = v;
    } else if (e < (long long)d1 * d1 + (long long)d1 * d2) {
      long long f = e - (long long)d1 * d1;
      int i = (int)(f / d2), j = (int)(f % d2);
      int ri = h1[i];
      double v;
      if (has_bar && j == 0) {
        v = gb[ri] - coef[ri] * bgb;
      } else {
        int rm = h2m[j - has_bar];
        v = G[(size_t)ri * n_raw + rm];
        if (has_bar) v -= coef[ri] * gb[rm];
      }
      X12[f] = v;
    } else {
      long long f = e - (long long)d1 * d1 - (long long)d1 * d2;
      int i = (int)(f / d2), j = (int)(f % d2);
      double v;
      if (has_bar && i == 0 && j == 0) v = bgb;
      else if (has_bar && i == 0) v = gb[h2m[j - 1]];
      else if (has_bar && j == 0) v = gb[h2m[i - 1]];
      else v = G[(size_t)h2m[i - has_bar] * n_raw + h2m[j - has_bar]];
      X22[f] = v;
    }
  }
}

// v1 = T1^T raw, v2 = T2^T raw for count raw vectors
__global__ void k_to_reduced(const double* __restrict__ raw, int count, int n_raw,
                             const int* __restrict__ kind, double invL, const double* __restrict__ coef,
                             const int* __restrict__ h1, int d1, const int* __restrict__ h2m, int nm,
                             int has_bar, double* __restrict__ v1, double* __restrict__ v2) {
  const int v = blockIdx.x;
  const double* r = raw + (size_t)v * n_raw;
  __shared__ double sh[64];
  double br = 0.0;
  if (has_bar) {
    for (int c = threadIdx.x; c < n_raw; c += blockDim.x)
      if (kind[c] == 1) br += r[c] * invL;
    br = pintd::block_sum(br, sh);
  }
  const int d2 = nm + has_bar;
  for (int i = threadIdx.x; i < d1; i += blockDim.x) v1[(size_t)v * d1 + i] = r[h1[i]] - coef[h1[i]] * br;
  for (int j = threadIdx.x; j < d2; j += blockDim.x)
    v2[(size_t)v * d2 + j] = (has_bar && j == 0) ? br : r[h2m[j - has_bar]];
}

// raw coefficients a = T1 u + T2 w, stored transposed: a[raw][v]
__global__ void k_from_reduced(const double* __restrict__ u, const double* __restrict__ w, int count,
                               int n_raw, const int* __restrict__ kind, double invL,
                               const double* __restrict__ coef, const int* __restrict__ h1, int d1,
                               const int* __restrict__ h2m, int nm, int has_bar,
                               double* __restrict__ a) {
  const int v = blockIdx.x;
  const int d2 = nm + has_bar;
  __shared__ double sh[64];
  double cu = 0.0;
  if (has_bar) {
    for (int i = threadIdx.x; i < d1; i += blockDim.x) cu += coef[h1[i]] * u[(size_t)v * d1 + i];
    cu = pintd::block_sum(cu, sh);
  }
  const double bar = has_bar ? (w[(size_t)v * d2] - cu) * invL : 0.0;
  for (int r = threadIdx.x; r < n_raw; r += blockDim.x) a[(size_t)r * count + v] = (kind[r] == 1) ? bar : 0.0;
  __syncthreads();
  for (int i = threadIdx.x; i < d1; i += blockDim.x) a[(size_t)h1[i] * count + v] += u[(size_t)v * d1 + i];
  for (int j = threadIdx.x; j < nm; j += blockDim.x)
    a[(size_t)h2m[j] * count + v] += w[(size_t)v * d2 + has_bar + j];
}

// out[v][node] = sum over windows containing node, bases q: a[raw][v] psi
__global__ void k_prolong(const GWin* __restrict__ gw, int n_f, int nc, int bs, int ell,
                          const double* __restrict__ psi, const double* __restrict__ a, int count,
                          double* __restrict__ out) {
  const int nn1 = n_f + 1, nn = nn1 * nn1;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nn * count) return;
  int v = (int)(t / nn), node = (int)(t % nn);
  int gx = node % nn1, gy = node / nn1;
  int cx = min(gx / bs, nc - 1), cy = min(gy / bs, nc - 1);
  double acc = 0.0;
  for (int by = max(0, cy - ell - 1); by <= min(nc - 1, cy + ell + 1); ++by)
    for (int bx = max(0, cx - ell - 1); bx <= min(nc - 1, cx + ell + 1); ++bx) {
      const GWin W = gw[by * nc + bx];
      int lx = gx - W.X0, ly = gy - W.Y0;
      if (lx < 0 || lx >= W.wx || ly < 0 || ly >= W.wy) continue;
      int l = ly * W.wx + lx;
      for (int q = 0; q < W.kt; ++q)
        acc += a[(size_t)(W.raw0 + q) * count + v] * psi[W.psi_off + (size_t)q * W.nw + l];
    }
  out[t] = acc;
}

// k_prolong in double-float arithmetic: thread per node, VB states per thread
// (the coefficient pairs of the VB states are contiguous), bases as FP32 pairs
// out[v][node] = sum over the windows containing node and their bases q of
// a[raw(q)][v] psi_q(node), in double-float arithmetic (bases and coefficients
// as FP32 pairs).  One CTA per (coarse block, group of VB times).  The block's nodes (the last node row / column joins the last
// block) share the candidate windows, whose descriptors are staged in shared
// memory once; every thread walks the same windows and bases (uniform control
// flow), its node's basis values are read once per time group, and the
// coefficient pairs of a basis are warp-uniform loads.
constexpr int PB_MAXW = 19 * 19;  // candidate windows of a block (ell <= 8)
template <int VB>
__global__ void __launch_bounds__(256) k_prolong_df_blk(const GWin* __restrict__ gw, int n_f, int nc, int bs,
                                                        int ell, const float* __restrict__ psih,
                                                        const float* __restrict__ psil,
                                                        const float2* __restrict__ a2, int count,
                                                        double* __restrict__ out) {
  __shared__ GWin sw[PB_MAXW];
  const int nn1 = n_f + 1, nn = nn1 * nn1;
  const int cx = blockIdx.x % nc, cy = blockIdx.x / nc;
  const int v0 = blockIdx.y * VB;
  const int bx0 = max(0, cx - ell - 1), bx1 = min(nc - 1, cx + ell + 1);
  const int by0 = max(0, cy - ell - 1), by1 = min(nc - 1, cy + ell + 1);
  const int nwx = bx1 - bx0 + 1, nwin = nwx * (by1 - by0 + 1);
  for (int e = threadIdx.x; e < nwin; e += blockDim.x) sw[e] = gw[(by0 + e / nwx) * nc + bx0 + e % nwx];
  __syncthreads();
  const int gx0 = cx * bs, gy0 = cy * bs;
  const int tw = bs + (cx == nc - 1 ? 1 : 0), th = bs + (cy == nc - 1 ? 1 : 0);
  for (int t = threadIdx.x; t < tw * th; t += blockDim.x) {
    const int gx = gx0 + t % tw, gy = gy0 + t / tw;
    float sh[VB], sl[VB];
#pragma unroll
    for (int v = 0; v < VB; ++v) sh[v] = sl[v] = 0.f;
    for (int wi = 0; wi < nwin; ++wi) {
      const GWin& W = sw[wi];
      const int lx = gx - W.X0, ly = gy - W.Y0;
      if (lx < 0 || lx >= W.wx || ly < 0 || ly >= W.wy) continue;
      const size_t pi0 = W.psi_off + (size_t)ly * W.wx + lx;
      const float2* ac = a2 + (size_t)W.raw0 * count + v0;
      for (int q = 0; q < W.kt; ++q) {
        const size_t pi = pi0 + (size_t)q * W.nw;
        const float ph = psih[pi], pl = psil[pi];
#pragma unroll
        for (int v = 0; v < VB; ++v)
          if (v0 + v < count) {
            const float2 c = ac[(size_t)q * count + v];
            pintd::df_fma(c.x, c.y, ph, pl, sh[v], sl[v]);
          }
      }
    }
    const int node = gy * nn1 + gx;
#pragma unroll
    for (int v = 0; v < VB; ++v)
      if (v0 + v < count) out[(size_t)(v0 + v) * nn + node] = (double)sh[v] + (double)sl[v];
  }
}

// x -> interleaved pairs (fl32(x), fl32(x - fl32(x)))
__global__ void k_split_pairs2(const double* __restrict__ x, long long n, float2* __restrict__ y) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double v = x[e];
    const float hv = (float)v;
    y[e] = make_float2(hv, (float)(v - (double)hv));
  }
}

__global__ void k_split_pairs(const double* __restrict__ x, long long n, float* __restrict__ h,
                              float* __restrict__ l) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double v = x[e];
    const float hv = (float)v;
    h[e] = hv;
    l[e] = (float)(v - (double)hv);
  }
}

}  // namespace

static GWin* make_gwin(Ctx* c) {
  std::vector<GWin> gw(c->n_blocks);
  long long xoff = 0;
  for (int b = 0; b < c->n_blocks; ++b) {
    const WinDesc& W = c->win[b];
    GWin& G = gw[b];
    G.X0 = W.X0;
    G.Y0 = W.Y0;
    G.wx = W.wx;
    G.wy = W.wy;
    G.nw = W.nw;
    G.kt = W.kt;
    G.raw0 = c->blk_kind_off[b];
    G.pad = 0;
    G.psi_off = W.psi_off;
    G.xpsi_off = xoff;
    xoff += (long long)W.kt * (W.wx + 2) * (W.wy + 2);
    c->win[b].xpsi_off = G.xpsi_off;
  }
  GWin* d = (GWin*)dalloc(c, sizeof(GWin) * gw.size());
  PINT_CUDA(cudaMemcpyAsync(d, gw.data(), sizeof(GWin) * gw.size(), cudaMemcpyHostToDevice, c->stream));
  c->d_windesc = (int*)d;
  return d;
}

void build_galerkin(Ctx* c) {
  GWin* d_gw = make_gwin(c);
  long long xtot = 0;
  for (const auto& W : c->win) xtot += (long long)W.kt * (W.wx + 2) * (W.wy + 2);
  double* xpsi = (double*)dalloc(c, (size_t)xtot * 3 * sizeof(double));
  k_xpsi<<<dim3(64, c->n_blocks), 256, 0, c->stream>>>(d_gw, c->n_f, c->stA, c->stM, c->stS, c->psi,
                                                       xpsi, xtot);
  PINT_LAUNCH_CHECK();
  // window pairs with A's interior meeting B's closure
  std::vector<int2> pairs;
  int maxkt = 0;
  for (int a = 0; a < c->n_blocks; ++a) {
    const WinDesc& A = c->win[a];
    maxkt = std::max(maxkt, A.kt);
    for (int b = 0; b < c->n_blocks; ++b) {
      const WinDesc& B = c->win[b];
      int x0 = std::max(A.X0, B.X0 - 1), x1 = std::min(A.X0 + A.wx - 1, B.X0 + B.wx);
      int y0 = std::max(A.Y0, B.Y0 - 1), y1 = std::min(A.Y0 + A.wy - 1, B.Y0 + B.wy);
      if (x0 <= x1 && y0 <= y1 && A.kt > 0 && B.kt > 0) pairs.push_back(make_int2(a, b));
    }
  }
  PINT_REQUIRE(maxkt <= KA, PINT_ERR_BAD_ARG, "too many bases per block for the Galerkin kernel");
  int2* d_pairs = (int2*)dalloc(c, pairs.size() * sizeof(int2));
  PINT_CUDA(cudaMemcpyAsync(d_pairs, pairs.data(), pairs.size() * sizeof(int2), cudaMemcpyHostToDevice,
                            c->stream));
  size_t g2 = (size_t)c->n_raw * c->n_raw;
  c->GM = (double*)dalloc(c, g2 * 8);
  c->GA = (double*)dalloc(c, g2 * 8);
  c->GS = (double*)dalloc(c, g2 * 8);
  PINT_CUDA(cudaMemsetAsync(c->GM, 0, g2 * 8, c->stream));
  PINT_CUDA(cudaMemsetAsync(c->GA, 0, g2 * 8, c->stream));
  PINT_CUDA(cudaMemsetAsync(c->GS, 0, g2 * 8, c->stream));
  for (size_t p0 = 0; p0 < pairs.size(); p0 += 65535) {
    unsigned np = (unsigned)std::min<size_t>(65535, pairs.size() - p0);
    k_pair<<<dim3(np, maxkt), 256, 0, c->stream>>>(d_gw, d_pairs + p0, c->psi, xpsi, xtot, c->n_raw,
                                                   c->GA, c->GM, c->GS);
    PINT_LAUNCH_CHECK();
  }
  PINT_CUDA(cudaStreamSynchronize(c->stream));
  dfree(c, xpsi);
  dfree(c, d_pairs);
}

namespace {
struct SplitDev {
  int* kind;
  int* h1;
  int* h2m;
};
SplitDev split_dev(Ctx* c) {
  // three int arrays packed after each other in d_h1 (allocated in build_reduced)
  int* base = reinterpret_cast<int*>(c->d_h1);
  return SplitDev{base, base + c->n_raw, base + c->n_raw + c->d1};
}
}  // namespace

void build_reduced(Ctx* c) {
  const int n_raw = c->n_raw;
  c->h1.clear();
  c->h2m.clear();
  int last_frac = -1;
  for (int r = 0; r < n_raw; ++r)
    if (c->kind[r] == 1) last_frac = r;
  for (int r = 0; r < n_raw; ++r) {
    if (c->kind[r] == 0) c->h2m.push_back(r);
    else if (r != last_frac) c->h1.push_back(r);
  }
  c->has_bar = c->L > 0;
  c->d1 = (int)c->h1.size();
  c->d2 = (int)c->h2m.size() + (c->has_bar ? 1 : 0);
  PINT_REQUIRE(c->d1 > 0 && c->d2 > 0, PINT_ERR_BAD_ARG, "empty V_H1 or V_H2");
  std::vector<int> packed;
  packed.insert(packed.end(), c->kind.begin(), c->kind.end());
  packed.insert(packed.end(), c->h1.begin(), c->h1.end());
  packed.insert(packed.end(), c->h2m.begin(), c->h2m.end());
  c->d_h1 = (double*)dalloc(c, packed.size() * sizeof(int));
  PINT_CUDA(cudaMemcpyAsync(c->d_h1, packed.data(), packed.size() * sizeof(int), cudaMemcpyHostToDevice,
                            c->stream));
  SplitDev sd = split_dev(c);
  const double invL = c->has_bar ? 1.0 / c->L : 0.0;
  double* gb = (double*)dalloc(c, 3 * (size_t)n_raw * 8);
  double* scal = (double*)dalloc(c, 4 * 8);
  c->coef = (double*)dalloc(c, (size_t)n_raw * 8);
  PINT_CUDA(cudaMemsetAsync(scal, 0, 32, c->stream));
  PINT_CUDA(cudaMemsetAsync(c->coef, 0, (size_t)n_raw * 8, c->stream));
  if (c->has_bar) {
    k_gbeta<<<n_raw, 128, 0, c->stream>>>(c->GM, sd.kind, n_raw, invL, gb);
    k_gbeta<<<n_raw, 128, 0, c->stream>>>(c->GA, sd.kind, n_raw, invL, gb + n_raw);
    k_gbeta<<<n_raw, 128, 0, c->stream>>>(c->GS, sd.kind, n_raw, invL, gb + 2 * n_raw);
    k_bgb<<<1, 256, 0, c->stream>>>(gb, gb + n_raw, gb + 2 * n_raw, sd.kind, n_raw, invL, scal, c->coef);
    PINT_LAUNCH_CHECK();
  }
  const int d1 = c->d1, d2 = c->d2, nm = (int)c->h2m.size();
  auto A = [&](size_t n) { return (double*)dalloc(c, n * 8); };
  c->M11 = A((size_t)d1 * d1);
  c->A11 = A((size_t)d1 * d1);
  c->M12 = A((size_t)d1 * d2);
  c->A12 = A((size_t)d1 * d2);
  c->M22 = A((size_t)d2 * d2);
  c->A22 = A((size_t)d2 * d2);
  k_reduce<<<512, 256, 0, c->stream>>>(c->GM, gb, scal, 0, c->coef, sd.h1, d1, sd.h2m, nm,
                                        c->has_bar, n_raw, c->M11, c->M12, c->M22);
  k_reduce<<<512, 256, 0, c->stream>>>(c->GA, gb + n_raw, scal, 1, c->coef, sd.h1, d1, sd.h2m, nm,
                                        c->has_bar, n_raw, c->A11, c->A12, c->A22);
  PINT_LAUNCH_CHECK();
  PINT_CUDA(cudaStreamSynchronize(c->stream));
  dfree(c, gb);
  dfree(c, scal);
}

void raw_dot(Ctx* c, const double* vec_nodes, int count, double* out_raw) {
  int maxkt = 0;
  for (const auto& W : c->win) maxkt = std::max(maxkt, W.kt);
  k_raw_dot<<<dim3(c->n_blocks, maxkt), 256, 0, c->stream>>>((const GWin*)c->d_windesc, c->n_f, c->psi,
                                                              vec_nodes, count, c->n_raw, out_raw);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

void to_reduced(Ctx* c, const double* raw, int count, double* v1, double* v2) {
  SplitDev sd = split_dev(c);
  k_to_reduced<<<count, 256, 0, c->stream>>>(raw, count, c->n_raw, sd.kind,
                                             c->has_bar ? 1.0 / c->L : 0.0, c->coef, sd.h1, c->d1,
                                             sd.h2m, (int)c->h2m.size(), c->has_bar, v1, v2);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

void prolong_coeffs(Ctx* c, const double* u, const double* w, int count, double* out_nodes) {
  SplitDev sd = split_dev(c);
  double* a = (double*)dalloc(c, (size_t)c->n_raw * count * 8);
  k_from_reduced<<<count, 256, 0, c->stream>>>(u, w, count, c->n_raw, sd.kind,
                                               c->has_bar ? 1.0 / c->L : 0.0, c->coef, sd.h1, c->d1,
                                               sd.h2m, (int)c->h2m.size(), c->has_bar, a);
  PINT_LAUNCH_CHECK();
  long long tot = (long long)c->nn * count;
  k_prolong<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(
      (const GWin*)c->d_windesc, c->n_f, c->nc, c->bs, c->ell, c->psi, a, count, out_nodes);
  PINT_LAUNCH_CHECK();
  c->launches += 2;
  dfree(c, a);
}

void prolong_coeffs_df(Ctx* c, const double* u, const double* w, int count, double* out_nodes, const float* psih,
                       const float* psil) {
  SplitDev sd = split_dev(c);
  const size_t na = (size_t)c->n_raw * count;
  double* a = (double*)dalloc(c, na * 8);
  float* ap = (float*)dalloc(c, na * 8);
  k_from_reduced<<<count, 256, 0, c->stream>>>(u, w, count, c->n_raw, sd.kind, c->has_bar ? 1.0 / c->L : 0.0,
                                               c->coef, sd.h1, c->d1, sd.h2m, (int)c->h2m.size(), c->has_bar, a);
  PINT_LAUNCH_CHECK();
  k_split_pairs2<<<(unsigned)std::min<size_t>((na + 255) / 256, 4096), 256, 0, c->stream>>>(
      a, (long long)na, reinterpret_cast<float2*>(ap));
  PINT_LAUNCH_CHECK();
  constexpr int VB = 17;  // 65 coarse times of a 64-interval solve in four groups
  const int per = (c->bs + 1) * (c->bs + 1);
  const int threads = std::min(256, (per + 31) / 32 * 32);
  PINT_REQUIRE((2 * c->ell + 3) * (2 * c->ell + 3) <= PB_MAXW, PINT_ERR_BAD_ARG, "oversampling too wide");
  const dim3 grid((unsigned)(c->nc * c->nc), (unsigned)((count + VB - 1) / VB));
  k_prolong_df_blk<VB><<<grid, threads, 0, c->stream>>>((const GWin*)c->d_windesc, c->n_f, c->nc, c->bs, c->ell,
                                                        psih, psil, reinterpret_cast<const float2*>(ap), count,
                                                        out_nodes);
  PINT_LAUNCH_CHECK();
  c->launches += 3;
  dfree(c, a);
  dfree(c, ap);
}

// FP64 bases -> FP32 pairs (for prolong_coeffs_df)
void split_bases(Ctx* c, float* psih, float* psil) {
  k_split_pairs<<<4096, 256, 0, c->stream>>>(c->psi, c->psi_total, psih, psil);
  PINT_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Allocation-free prolongation (pint_prolong_noalloc, declared in pint.h).
//
// Some callers cannot call cudaMalloc or any allocating routine: a host
// runtime that owns the device allocator and forbids other allocations, a
// real-time loop that must not touch the allocator, or a caller that has no
// allocator at all.  This entry point runs the same two kernels as
// pint_prolong but keeps the scratch it needs (the split u / w rows and the
// raw-basis coefficients) in the file-scope device array below, so the call
// itself allocates and frees nothing.  Limits and hazards:
//   * count * (d1 + d2 + n_raw) <= PINT_NOALLOC_SCRATCH_DOUBLES, else
//     PINT_ERR_BAD_ARG (8 MB per GPU that loads the library, held until exit);
//   * coarse and u_out must be device pointers (host staging would allocate);
//   * every call shares the one array: calls whose kernels overlap on the GPU
//     (two streams, two threads, two contexts on one device) race;
//   * each call writes every scratch element it reads before reading it, so
//     what an earlier call left there does not matter.
// Host code cannot use the array's name as a device address; the address is
// fetched with cudaGetSymbolAddress, once per device, by the first call made
// on that device.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t PINT_NOALLOC_SCRATCH_DOUBLES = (size_t)1 << 20;
static __device__ __align__(256) double g_noalloc_scratch[PINT_NOALLOC_SCRATCH_DOUBLES];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {nullptr};

// the scratch address on device `dev`, which must be the current device
double* noalloc_scratch_for_device(int dev) {
  PINT_REQUIRE(dev >= 0 && dev < 256, PINT_ERR_BAD_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Fail{PINT_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
    }
    g_noalloc_ptr[dev] = (double*)p;
  }
  return g_noalloc_ptr[dev];
}
}  // namespace

}  // namespace pint

extern "C" pint_status pint_prolong_noalloc(pint_ctx* ctx, const double* coarse, int count, double* u_out) {
  using namespace pint;
  Ctx* c = (Ctx*)ctx;
  if (!c || !coarse || !u_out || count < 1) {
    set_error("ctx, coarse, u_out and count >= 1 are required");
    return PINT_ERR_BAD_ARG;
  }
  try {
    PINT_REQUIRE(c->have_reduced, PINT_ERR_STATE, "pint_assemble_reduced first");
    int cur = -1;
    PINT_CUDA(cudaGetDevice(&cur));
    PINT_REQUIRE(cur == c->device, PINT_ERR_BAD_ARG,
                 "pint_prolong_noalloc: make the context's device current first");
    PINT_REQUIRE(is_device_ptr(coarse) && is_device_ptr(u_out), PINT_ERR_BAD_ARG,
                 "pint_prolong_noalloc takes device pointers only");
    const int d1 = c->d1, d2 = c->d2, n_raw = c->n_raw;
    const size_t need = (size_t)count * (d1 + d2 + n_raw);
    PINT_REQUIRE(need <= PINT_NOALLOC_SCRATCH_DOUBLES, PINT_ERR_BAD_ARG,
                 "pint_prolong_noalloc: count * (d1 + d2 + n_raw) exceeds the 1048576-double scratch");
    double* s = noalloc_scratch_for_device(c->device);
    double* u = s;
    double* w = u + (size_t)count * d1;
    double* a = w + (size_t)count * d2;
    PINT_CUDA(cudaMemcpy2DAsync(u, (size_t)d1 * 8, coarse, (size_t)(d1 + d2) * 8, (size_t)d1 * 8, count,
                                cudaMemcpyDeviceToDevice, c->stream));
    PINT_CUDA(cudaMemcpy2DAsync(w, (size_t)d2 * 8, coarse + d1, (size_t)(d1 + d2) * 8, (size_t)d2 * 8, count,
                                cudaMemcpyDeviceToDevice, c->stream));
    SplitDev sd = split_dev(c);
    k_from_reduced<<<count, 256, 0, c->stream>>>(u, w, count, n_raw, sd.kind, c->has_bar ? 1.0 / c->L : 0.0,
                                                 c->coef, sd.h1, d1, sd.h2m, (int)c->h2m.size(), c->has_bar, a);
    PINT_LAUNCH_CHECK();
    long long tot = (long long)c->nn * count;
    k_prolong<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(
        (const GWin*)c->d_windesc, c->n_f, c->nc, c->bs, c->ell, c->psi, a, count, u_out);
    PINT_LAUNCH_CHECK();
    return PINT_OK;  // stream-ordered: the result is ready when the context's stream reaches this point
  } catch (const Fail& e) {
    set_error(e.msg);
    return e.code;
  } catch (const std::exception& e) {
    set_error(std::string("host exception: ") + e.what());
    return PINT_ERR_BAD_ARG;
  }
}
