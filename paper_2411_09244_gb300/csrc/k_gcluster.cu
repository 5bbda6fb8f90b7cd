// Coarse sweep of the mixed path on one thread-block cluster.
//
// One sweep of Algorithm 1's sequential correction runs N coarse steps of the
// splitting scheme, eqs. (2.4)-(2.5) with the coarse step Dt, in spectral
// coordinates:
//   u' = (u - Dt CA w + Dt a_n b1) / (1 + Dt Lambda1)
//   w' = (1 - Dt Lambda2) w - Dt CA^T u' + Dt a_n b2
// and applies the update of eq. (2.7), x_{n+1} = G(x_n) + F_n - G_old_n
// (+ c_{n+1} in a correction solve).  The low-precision path only needs G to
// contract the parareal error (its fixed point is that of F, and the FP64
// refinement measures what the low-precision solve leaves), so the whole step
// runs in FP32: products, updates, and the F ends, old G values and jumps it
// reads (FP32 copies).  Only the states X are written back in FP64.
//
// The FP32 coupling CA stays resident in the distributed shared memory of a
// cluster of CL CTAs (rows split evenly).  Per step: each CTA forms u' for its
// rows (warp per row), the partial products CA^T u' over its rows for every
// column, then after a cluster barrier each CTA reduces its slice of columns
// over the CL partials (DSMEM loads in a fixed order, so the sweep is
// deterministic), forms w' for that slice and writes it into every CTA's copy
// of w; a second cluster barrier closes the step.  Both barriers are the
// hardware cluster barrier: no software spin-waits.
#include "common.cuh"

#include <algorithm>

namespace pint {

namespace {

constexpr int GC_THREADS = 1024;
constexpr int GC_MAX_RT = 8;  // rows per warp and CTA (rows per CTA <= 256)
constexpr size_t GC_SMEM = 200 * 1024;  // dynamic shared memory budget per CTA

// nb: coarse steps whose outputs are staged in shared memory before they are
// written out (no global stores inside a chunk, so the release side of the
// cluster barriers has only shared-memory traffic to order)
struct GcLayout {
  int rpc, spc, ng, nb;
  size_t CA, xw, part, gu, acc, gtmp, sbuf, xu, ia, cb, wo, fw, cw, su, sg, sw, sh, n;  // float offsets
  size_t bytes;
};

__host__ __device__ inline GcLayout gc_layout(int d1, int d2, int CL, int nb) {
  GcLayout L{};
  L.nb = nb;
  L.rpc = (d1 + CL - 1) / CL;
  L.spc = (d2 + CL - 1) / CL;
  L.ng = d2 >= GC_THREADS ? 1 : (GC_THREADS / d2 > 8 ? 8 : GC_THREADS / d2);
  size_t o = 0;
  auto take = [&](size_t n) {
    const size_t at = o;
    o += n;
    return at;
  };
  L.CA = take((size_t)L.rpc * d2);
  L.xw = take(d2);       // the whole w (FP32), replicated
  L.part = take(d2);     // this CTA's partial products
  L.gu = take(L.rpc);    // u' rows
  L.acc = take(L.rpc);   // CA w rows
  L.gtmp = take((size_t)L.ng * d2);
  L.sbuf = take(L.spc);  // new w of the own slice, for the broadcast
  L.xu = take(L.rpc);    // own states u
  L.ia = take(L.rpc);    // 1 / (1 + Dt lambda1)
  L.cb = take(L.rpc);    // Dt b1 / (1 + Dt lambda1)
  L.wo = take(L.spc);    // own slice of w
  L.fw = take(L.spc);    // 1 - Dt lambda2
  L.cw = take(L.spc);    // Dt b2
  L.su = take((size_t)nb * L.rpc);  // staged X_u, G_u rows and X_w, G_w slices
  L.sg = take((size_t)nb * L.rpc);
  L.sw = take((size_t)nb * L.spc);
  L.sh = take((size_t)nb * L.spc);
  L.n = o;
  L.bytes = o * 4;
  return L;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t dsmem_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ float ld_dsmem(uint32_t a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_dsmem(uint32_t a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void st_dsmem4(uint32_t a, float4 v) {  // a 16-byte aligned
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}

template <int CL>
__global__ void __launch_bounds__(GC_THREADS, 1) k_g_sweep_cl(GcArgs a, int nb) {
  extern __shared__ __align__(16) unsigned char gsm[];
  const int d1 = a.d1, d2 = a.d2;
  const GcLayout L = gc_layout(d1, d2, CL, nb);
  float* fs = reinterpret_cast<float*>(gsm);
  float *sCA = fs + L.CA, *xw32 = fs + L.xw, *part = fs + L.part, *gu32 = fs + L.gu, *accs = fs + L.acc,
        *gtmp = fs + L.gtmp, *sbuf = fs + L.sbuf, *xu = fs + L.xu, *ia = fs + L.ia, *cb = fs + L.cb,
        *wo = fs + L.wo, *fw = fs + L.fw, *cw = fs + L.cw, *stXu = fs + L.su, *stGu = fs + L.sg, *stXw = fs + L.sw,
        *stGw = fs + L.sh;
  const int rank = (int)cl_rank();
  const int r0 = rank * L.rpc, nr = max(0, min(d1, r0 + L.rpc) - r0);
  const int j0 = rank * L.spc, ns = max(0, min(d2, j0 + L.spc) - j0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float Dt = (float)a.Dt;
  const size_t n0 = (size_t)a.n_lo;
  for (size_t e = tid; e < (size_t)nr * d2; e += GC_THREADS) sCA[e] = a.CA[(size_t)r0 * d2 + e];
  for (int j = tid; j < d2; j += GC_THREADS) xw32[j] = (float)a.Xw[n0 * d2 + j];
  for (int q = tid; q < nr; q += GC_THREADS) {
    const int i = r0 + q;
    xu[q] = (float)a.Xu[n0 * d1 + i];
    ia[q] = (float)(1.0 / (1.0 + a.Dt * a.lam1[i]));
    cb[q] = (float)(a.Dt * a.b1[i] / (1.0 + a.Dt * a.lam1[i]));
  }
  for (int q = tid; q < ns; q += GC_THREADS) {
    const int j = j0 + q;
    wo[q] = (float)a.Xw[n0 * d2 + j];
    fw[q] = (float)(1.0 - a.Dt * a.lam2[j]);
    cw[q] = (float)(a.Dt * a.b2[j]);
  }
  __syncthreads();
  cl_sync();  // every CTA of the cluster is resident before any DSMEM access
  const int rt = nr > warp ? (nr - warp + 31) / 32 : 0;  // matvec rows of this warp: q = warp + 32 t
  // inputs of a step that do not depend on the sweep (F end, old G, jump, for
  // row q = tid and slice entry tid) are fetched one step ahead
  auto fetch = [&](int n, float& pf, float& pg, float& pc, float& wf, float& wg, float& wc, float& am) {
    pf = pg = pc = wf = wg = wc = 0.f;
    am = 0.f;
    if (n >= a.n_hi) return;
    am = (float)a.amp[n];
    if (tid < nr) {
      const int i = r0 + tid;
      if (!a.first) {
        pf = a.Fu[(size_t)n * d1 + i];
        pg = a.Gu[(size_t)n * d1 + i];
      }
      if (a.Cu) pc = a.Cu[(size_t)(n + 1) * d1 + i];
    }
    if (tid < ns) {
      const int j = j0 + tid;
      if (!a.first) {
        wf = a.Fw[(size_t)n * d2 + j];
        wg = a.Gw[(size_t)n * d2 + j];
      }
      if (a.Cw) wc = a.Cw[(size_t)(n + 1) * d2 + j];
    }
  };
  float npf, npg, npc, nwf, nwg, nwc, nam;
  fetch(a.n_lo, npf, npg, npc, nwf, nwg, nwc, nam);
  int nbase = a.n_lo;
  for (int n = a.n_lo; n < a.n_hi; ++n) {
    const int sl = n - nbase;  // staging slot of this step
    const float pf = npf, pg = npg, pc = npc, wf = nwf, wg = nwg, wc = nwc, am = nam;
    // G_old of step n + 1 is read here, before this sweep rewrites it: this
    // step writes G_old of step n only (staged), so the read sees the old value
    fetch(n + 1, npf, npg, npc, nwf, nwg, nwc, nam);
    // u-phase products CA w: one warp per row
#pragma unroll
    for (int t = 0; t < GC_MAX_RT; ++t) {
      if (t < rt) {
        const int q = warp + 32 * t;
        const float* row = sCA + (size_t)q * d2;
        float acc = 0.f;
        for (int j = lane; j < d2; j += 32) acc = fmaf(row[j], xw32[j], acc);
        acc = pintd::warp_sumf(acc);
        if (lane == 0) accs[q] = acc;
      }
    }
    __syncthreads();
    if (tid < nr) {
      const int q = tid;
      const float g = xu[q] * ia[q] - Dt * ia[q] * accs[q] + am * cb[q];
      const float v = (a.first ? g : g + pf - pg) + pc;
      stXu[(size_t)sl * L.rpc + q] = v;
      stGu[(size_t)sl * L.rpc + q] = g;
      xu[q] = v;
      gu32[q] = g;
    }
    __syncthreads();
    // partial products CA^T u' over this CTA's rows, L.ng row groups per column
    {
      const int grp = tid / d2, j = tid - grp * d2;
      if (grp < L.ng) {
        for (int jj = j; jj < d2; jj += GC_THREADS) {  // d2 > GC_THREADS: one group loops over columns
          float acc = 0.f;
          for (int q = grp; q < nr; q += L.ng) acc = fmaf(sCA[(size_t)q * d2 + jj], gu32[q], acc);
          gtmp[(size_t)grp * d2 + jj] = acc;
        }
      }
    }
    __syncthreads();
    for (int j = tid; j < d2; j += GC_THREADS) {
      float s = 0.f;
      for (int g = 0; g < L.ng; ++g) s += gtmp[(size_t)g * d2 + j];
      part[j] = s;
    }
    cl_sync();  // partials of every CTA visible
    if (tid < ns) {
      const int j = j0 + tid;
      float s = 0.f;
#pragma unroll
      for (int r = 0; r < CL; ++r) s += ld_dsmem(dsmem_addr(&part[j], (uint32_t)r));
      const float g = fw[tid] * wo[tid] - Dt * s + am * cw[tid];
      const float v = (a.first ? g : g + wf - wg) + wc;
      stXw[(size_t)sl * L.spc + tid] = v;
      stGw[(size_t)sl * L.spc + tid] = g;
      wo[tid] = v;
      sbuf[tid] = v;
    }
    __syncthreads();
    for (int e = tid; e < ns * CL; e += GC_THREADS) {
      const int q = e % ns, r = e / ns;
      st_dsmem(dsmem_addr(&xw32[j0 + q], (uint32_t)r), sbuf[q]);
    }
    cl_sync();  // new w in every CTA; partial buffers free again
    if (sl + 1 == nb || n + 1 == a.n_hi) {  // write the staged chunk out (states in FP64)
      const int cnt = sl + 1;
      for (int e = tid; e < cnt * nr; e += GC_THREADS) {
        const int st = e / nr, q = e - st * nr;
        a.Xu[(size_t)(nbase + st + 1) * d1 + r0 + q] = (double)stXu[(size_t)st * L.rpc + q];
        a.Gu[(size_t)(nbase + st) * d1 + r0 + q] = stGu[(size_t)st * L.rpc + q];
      }
      for (int e = tid; e < cnt * ns; e += GC_THREADS) {
        const int st = e / ns, q = e - st * ns;
        a.Xw[(size_t)(nbase + st + 1) * d2 + j0 + q] = (double)stXw[(size_t)st * L.spc + q];
        a.Gw[(size_t)(nbase + st) * d2 + j0 + q] = stGw[(size_t)st * L.spc + q];
      }
      __syncthreads();
      nbase = n + 1;
    }
  }
}

// ---------------------------------------------------------------------------
// Register-resident variant for couplings of up to 16 x 6 rows and 9 x 32
// columns per CTA (16 CTAs, 16 warps each).  Profiling the shared-memory
// kernel above showed each step bound by shared-memory bandwidth and issue:
// CA was read from shared memory twice per step (the products CA w and
// CA^T u'), and w once per row.  Here each warp keeps its RT rows of CA in
// registers for the whole sweep (lane l holds columns l + 32 k), w is read
// once per step into registers, and one pass over the rows forms u' and the
// warp's share of CA^T u' together; the warps' shares meet in shared memory,
// the CTAs' in each CTA's receive buffer (as above, one cluster barrier per
// step, every CTA forms the whole w').
// ---------------------------------------------------------------------------
constexpr int GR_WARPS = 16;
constexpr int GR_THREADS = 32 * GR_WARPS;
constexpr int GR_CL = 16;

// one half of the prefetch area: amp (a double, then 2 pad floats), then
// Fu, Gu, Cu (rpc each) and Fw, Gw, Cw (d2p each); a multiple of 4 floats
__host__ __device__ inline size_t gr_half(int rpc, int d2p) {
  return ((size_t)4 + 3 * (size_t)rpc + 3 * (size_t)d2p + 3) / 4 * 4;
}

struct GrLayout {
  int rpc, spc, d2p, nb;
  size_t xw, wsum, recv, ia, cb, fw, cw, pre, su, sg, sw, sh, n;  // float offsets
  size_t bytes;
};

__device__ __forceinline__ void gr_cp4(float* sdst, const float* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void gr_cp8(void* sdst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void gr_cp_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__host__ __device__ inline GrLayout gr_layout(int d1, int d2, int nk, int nb) {
  GrLayout L{};
  L.nb = nb;
  L.rpc = (d1 + GR_CL - 1) / GR_CL;
  L.spc = (d2 + GR_CL - 1) / GR_CL;
  L.d2p = 32 * nk;
  size_t o = 0;
  auto take = [&](size_t n) {
    const size_t at = o;
    o += (n + 3) / 4 * 4;
    return at;
  };
  L.xw = take(L.d2p);                               // the whole w, identical in every CTA
  L.wsum = take((size_t)GR_WARPS * L.d2p);          // the warps' shares of CA^T u'
  L.recv = take((size_t)2 * GR_CL * L.d2p);         // two halves of the CTAs' slots
  L.ia = take(L.rpc);                               // 1 / (1 + Dt lambda1)
  L.cb = take(L.rpc);                               // Dt b1 / (1 + Dt lambda1)
  L.fw = take(L.d2p);                               // 1 - Dt lambda2
  L.cw = take(L.d2p);                               // Dt b2
  L.pre = take((size_t)2 * gr_half(L.rpc, L.d2p));  // next step's inputs, two halves
  L.su = take((size_t)nb * L.rpc);                  // staged X_u, G_u rows and X_w, G_w slices
  L.sg = take((size_t)nb * L.rpc);
  L.sw = take((size_t)nb * L.spc);
  L.sh = take((size_t)nb * L.spc);
  L.n = o;
  L.bytes = o * 4;
  return L;
}

template <int RT, int NK>
__global__ void __launch_bounds__(GR_THREADS, 1) k_g_sweep_clr(GcArgs a, int nb) {
  extern __shared__ __align__(16) unsigned char gsm[];
  const int d1 = a.d1, d2 = a.d2;
  const GrLayout L = gr_layout(d1, d2, NK, nb);
  const int d2p = L.d2p;
  float* fs = reinterpret_cast<float*>(gsm);
  float *xw = fs + L.xw, *wsum = fs + L.wsum, *recv = fs + L.recv, *ia = fs + L.ia, *cb = fs + L.cb,
        *fw = fs + L.fw, *cw = fs + L.cw, *stXu = fs + L.su, *stGu = fs + L.sg, *stXw = fs + L.sw,
        *stGw = fs + L.sh;
  const int rank = (int)cl_rank();
  const int r0 = rank * L.rpc, nr = max(0, min(d1, r0 + L.rpc) - r0);
  const int j0 = rank * L.spc, ns = max(0, min(d2, j0 + L.spc) - j0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float Dt = (float)a.Dt;
  const size_t n0 = (size_t)a.n_lo;
  // this warp's rows q = warp + 16 t of CA, lane l holding columns l + 32 k
  float ca[RT][NK], xu[RT];
#pragma unroll
  for (int t = 0; t < RT; ++t) {
    const int q = warp + GR_WARPS * t;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      const int j = lane + 32 * k;
      ca[t][k] = (q < nr && j < d2) ? a.CA[(size_t)(r0 + q) * d2 + j] : 0.f;
    }
    xu[t] = q < nr ? (float)a.Xu[n0 * d1 + r0 + q] : 0.f;
  }
  for (int j = tid; j < d2p; j += GR_THREADS) {
    xw[j] = j < d2 ? (float)a.Xw[n0 * d2 + j] : 0.f;
    fw[j] = j < d2 ? (float)(1.0 - a.Dt * a.lam2[j]) : 0.f;
    cw[j] = j < d2 ? (float)(a.Dt * a.b2[j]) : 0.f;
  }
  for (int q = tid; q < nr; q += GR_THREADS) {
    const int i = r0 + q;
    ia[q] = (float)(1.0 / (1.0 + a.Dt * a.lam1[i]));
    cb[q] = (float)(a.Dt * a.b1[i] / (1.0 + a.Dt * a.lam1[i]));
  }
  __syncthreads();
  cl_sync();  // every CTA of the cluster is resident before any DSMEM access
  // inputs of a step that do not depend on the sweep (F ends, old G values,
  // jumps, amplitude) are copied one step ahead into the other half of `pre`
  // by asynchronous copies, so no register waits on their global loads:
  // half layout [Fu | Gu | Cu] (rpc each), [Fw | Gw | Cw] (d2p each), amp (2)
  float* pre = fs + L.pre;
  const size_t half = gr_half(L.rpc, d2p);
  auto fetch = [&](int n, int h) {
    float* b = pre + (size_t)h * half;
    double* bam = reinterpret_cast<double*>(b);
    float *bFu = b + 4, *bGu = bFu + L.rpc, *bCu = bGu + L.rpc, *bFw = bCu + L.rpc, *bGw = bFw + d2p,
          *bCw = bGw + d2p;
    if (n >= a.n_hi) return;
    for (int q = tid; q < nr; q += GR_THREADS) {
      const size_t i = (size_t)r0 + q;
      if (!a.first) {
        gr_cp4(bFu + q, a.Fu + (size_t)n * d1 + i);
        gr_cp4(bGu + q, a.Gu + (size_t)n * d1 + i);
      } else {
        bFu[q] = 0.f;
        bGu[q] = 0.f;
      }
      if (a.Cu) gr_cp4(bCu + q, a.Cu + (size_t)(n + 1) * d1 + i);
      else bCu[q] = 0.f;
    }
    if (tid < d2) {
      if (!a.first) {
        gr_cp4(bFw + tid, a.Fw + (size_t)n * d2 + tid);
        gr_cp4(bGw + tid, a.Gw + (size_t)n * d2 + tid);
      } else {
        bFw[tid] = 0.f;
        bGw[tid] = 0.f;
      }
      if (a.Cw) gr_cp4(bCw + tid, a.Cw + (size_t)(n + 1) * d2 + tid);
      else bCw[tid] = 0.f;
    }
    if (tid == 0) gr_cp8(bam, a.amp + n);
  };
  fetch(a.n_lo, 0);
  gr_cp_wait();
  __syncthreads();
  int nbase = a.n_lo;
  for (int n = a.n_lo; n < a.n_hi; ++n) {
    const int sl = n - nbase;  // staging slot of this step
    const int h = (n - a.n_lo) & 1;
    const float* b = pre + (size_t)h * half;
    const float *bFu = b + 4, *bGu = bFu + L.rpc, *bCu = bGu + L.rpc, *bFw = bCu + L.rpc, *bGw = bFw + d2p,
                *bCw = bGw + d2p;
    const float am = (float)*reinterpret_cast<const double*>(b);
    // G_old of step n + 1 is read here, before this sweep rewrites it: this
    // step writes G_old of step n only (staged), so the read sees the old value
    fetch(n + 1, h ^ 1);
    float wl[NK], part[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      wl[k] = xw[lane + 32 * k];
      part[k] = 0.f;
    }
    // one pass over the warp's rows: u' = G's u step, then its CA^T u' share.
    // The RT rows are independent: their products and butterfly reductions
    // are interleaved so that the warp has RT chains in flight, not one.
    float acc[RT], gr[RT];
#pragma unroll
    for (int t = 0; t < RT; ++t) {
      acc[t] = 0.f;
#pragma unroll
      for (int k = 0; k < NK; ++k) acc[t] = fmaf(ca[t][k], wl[k], acc[t]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int t = 0; t < RT; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
#pragma unroll
    for (int t = 0; t < RT; ++t) {
      const int q = warp + GR_WARPS * t;
      gr[t] = 0.f;  // rows past nr: zero coupling rows, no u' and no share
      if (q < nr) {  // warp-uniform
        const float g = xu[t] * ia[q] - Dt * ia[q] * acc[t] + am * cb[q];
        const float v = g + ((bFu[q] - bGu[q]) + bCu[q]);
        if (lane == 0) {
          stXu[(size_t)sl * L.rpc + q] = v;
          stGu[(size_t)sl * L.rpc + q] = g;
        }
        xu[t] = v;
        gr[t] = g;
      }
    }
#pragma unroll
    for (int t = 0; t < RT; ++t)
#pragma unroll
      for (int k = 0; k < NK; ++k) part[k] = fmaf(ca[t][k], gr[t], part[k]);
#pragma unroll
    for (int k = 0; k < NK; ++k) wsum[(size_t)warp * d2p + lane + 32 * k] = part[k];
    __syncthreads();
    // this CTA's CA^T u' into its slot of every CTA's receive half
    float* rh = recv + (size_t)((n - a.n_lo) & 1) * GR_CL * d2p;
    if (4 * tid < d2) {  // four columns per thread, 16-byte stores (rows are 16-byte aligned)
      float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int w = 0; w < GR_WARPS; ++w) {
        const float4 t = reinterpret_cast<const float4*>(wsum + (size_t)w * d2p)[tid];
        sum.x += t.x;
        sum.y += t.y;
        sum.z += t.z;
        sum.w += t.w;
      }
      const float* slot = rh + (size_t)rank * d2p + 4 * tid;
#pragma unroll
      for (int r = 0; r < GR_CL; ++r) st_dsmem4(dsmem_addr(slot, (uint32_t)r), sum);
    }
    cl_sync();  // every CTA's shares delivered to every CTA
    // the whole w' in every CTA, slots summed in rank order (identical copies)
    if (tid < d2) {
      float sum = 0.f;
#pragma unroll
      for (int r = 0; r < GR_CL; ++r) sum += rh[(size_t)r * d2p + tid];
      const float g = fw[tid] * xw[tid] - Dt * sum + am * cw[tid];
      const float v = g + ((bFw[tid] - bGw[tid]) + bCw[tid]);
      xw[tid] = v;
      if (tid >= j0 && tid < j0 + ns) {
        stXw[(size_t)sl * L.spc + (tid - j0)] = v;
        stGw[(size_t)sl * L.spc + (tid - j0)] = g;
      }
    }
    gr_cp_wait();     // this thread's copies of the next step's inputs
    __syncthreads();  // new w and the next inputs before the next step; wsum free again
    if (sl + 1 == nb || n + 1 == a.n_hi) {  // write the staged chunk out (states in FP64)
      const int cnt = sl + 1;
      for (int e = tid; e < cnt * nr; e += GR_THREADS) {
        const int st = e / nr, q = e - st * nr;
        a.Xu[(size_t)(nbase + st + 1) * d1 + r0 + q] = (double)stXu[(size_t)st * L.rpc + q];
        a.Gu[(size_t)(nbase + st) * d1 + r0 + q] = stGu[(size_t)st * L.rpc + q];
      }
      for (int e = tid; e < cnt * ns; e += GR_THREADS) {
        const int st = e / ns, q = e - st * ns;
        a.Xw[(size_t)(nbase + st + 1) * d2 + j0 + q] = (double)stXw[(size_t)st * L.spc + q];
        a.Gw[(size_t)(nbase + st) * d2 + j0 + q] = stGw[(size_t)st * L.spc + q];
      }
      __syncthreads();
      nbase = n + 1;
    }
  }
}

// instantiated shapes: rows per warp RT and column blocks NK (d2 <= 32 NK)
template <int RT, int NK>
bool gr_feasible(size_t bytes) {
  static int ok = -1;
  std::lock_guard<std::mutex> lock(lazy_init_mutex());
  if (ok < 0) {
    ok = 0;
    if (cudaFuncSetAttribute(k_g_sweep_clr<RT, NK>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_g_sweep_clr<RT, NK>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = GR_CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(GR_CL);
    cfg.blockDim = dim3(GR_THREADS);
    cfg.dynamicSmemBytes = GC_SMEM;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_g_sweep_clr<RT, NK>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    ok = nclusters >= 1 ? 1 : 0;
  }
  return ok == 1 && bytes <= GC_SMEM;
}

template <int RT, int NK>
bool gr_launch(Ctx* c, const GcArgs& a) {
  const GrLayout L1 = gr_layout(a.d1, a.d2, NK, 1), L0 = gr_layout(a.d1, a.d2, NK, 0);
  if (!gr_feasible<RT, NK>(L1.bytes)) return false;
  const size_t per = L1.bytes - L0.bytes;
  const int nb = (int)std::min<size_t>((size_t)std::max(a.n_hi - a.n_lo, 1), 1 + (GC_SMEM - L1.bytes) / per);
  const GrLayout L = gr_layout(a.d1, a.d2, NK, nb);
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = GR_CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(GR_CL);
  cfg.blockDim = dim3(GR_THREADS);
  cfg.dynamicSmemBytes = L.bytes;
  cfg.stream = c->stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  PINT_CUDA(cudaLaunchKernelEx(&cfg, k_g_sweep_clr<RT, NK>, a, nb));
  c->launches++;
  return true;
}

// the register variant when an instantiated shape covers the coupling
template <int NK>
bool gr_try_rt(Ctx* c, const GcArgs& a, int rt) {
  if (rt <= 2) return gr_launch<2, NK>(c, a);
  if (rt <= 4) return gr_launch<4, NK>(c, a);
  if (rt <= 6) return gr_launch<6, NK>(c, a);
  return false;
}

bool gr_try(Ctx* c, const GcArgs& a) {
  const int rpc = (a.d1 + GR_CL - 1) / GR_CL, rt = (rpc + GR_WARPS - 1) / GR_WARPS;
  const int nk = (a.d2 + 31) / 32;
  if (a.d2 > GR_THREADS) return false;
  if (nk <= 3) return gr_try_rt<3>(c, a, rt);
  if (nk <= 5) return gr_try_rt<5>(c, a, rt);
  if (nk <= 9) return gr_try_rt<9>(c, a, rt);
  return false;
}

template <int CL>
bool gc_feasible(size_t bytes) {
  static int ok = -1;
  std::lock_guard<std::mutex> lock(lazy_init_mutex());
  if (ok < 0) {
    ok = 0;
    if (cudaFuncSetAttribute(k_g_sweep_cl<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
        cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (CL > 8 && cudaFuncSetAttribute(k_g_sweep_cl<CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(GC_THREADS);
    cfg.dynamicSmemBytes = GC_SMEM;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_g_sweep_cl<CL>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    ok = nclusters >= 1 ? 1 : 0;
  }
  return ok == 1 && bytes <= GC_SMEM;
}

// staging depth: as many coarse steps as fit next to the resident coupling
int gc_chunk(int d1, int d2, int CL, int steps) {
  const GcLayout L1 = gc_layout(d1, d2, CL, 1), L0 = gc_layout(d1, d2, CL, 0);
  const size_t per = L1.bytes - L0.bytes;
  if (L1.bytes > GC_SMEM) return 0;
  return (int)std::min<size_t>((size_t)std::max(steps, 1), 1 + (GC_SMEM - L1.bytes) / per);
}

template <int CL>
void gc_launch(Ctx* c, const GcArgs& a) {
  const int nb = gc_chunk(a.d1, a.d2, CL, a.n_hi - a.n_lo);
  PINT_REQUIRE(nb >= 1, PINT_ERR_BAD_ARG, "coarse sweep does not fit the cluster");
  const GcLayout L = gc_layout(a.d1, a.d2, CL, nb);
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(GC_THREADS);
  cfg.dynamicSmemBytes = L.bytes;
  cfg.stream = c->stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  PINT_CUDA(cudaLaunchKernelEx(&cfg, k_g_sweep_cl<CL>, a, nb));
  c->launches++;
}

}  // namespace

// Cluster size for the FP32 coarse sweep (16 or 8), or 0 when the coupling
// does not fit in the cluster's shared memory (the caller then uses the
// grid-wide FP64 sweep).
int gc_cluster_size(int d1, int d2) {
  for (int CL : {16, 8}) {
    const GcLayout L = gc_layout(d1, d2, CL, 1);
    if (L.rpc > 32 * GC_MAX_RT) continue;
    if (CL == 16 && gc_feasible<16>(L.bytes)) return 16;
    if (CL == 8 && gc_feasible<8>(L.bytes)) return 8;
  }
  return 0;
}

void g_sweep_cluster(Ctx* c, const GcArgs& a, int CL) {
  if (a.n_lo >= a.n_hi) return;
  if (CL == 16 && gr_try(c, a)) return;
  if (CL == 16)
    gc_launch<16>(c, a);
  else if (CL == 8)
    gc_launch<8>(c, a);
  else
    PINT_REQUIRE(false, PINT_ERR_BAD_ARG, "unsupported cluster size");
}

}  // namespace pint
