// Low-precision pieces of the mixed path: the WR iteration of Section 4.2
// (contractions, eq. (4.7) time solve, eq. (4.9) recurrence) in FP32 on FP32
// trajectories, plus the FP64 bookkeeping of the refinement (trajectory
// promotion, fine-scheme residual, continuity jumps).
//
// Per-step sources: the main solve has the constant source amp_n F~ on
// interval n; the correction solve of the refinement has the per-step source
// -e_{n,p} (minus the FP64 residual of the trajectory), passed as
// src_u = -e_u / dt (added to the contraction output, as the constant source
// F1~ is) and src_w = -e_w (added in the recurrence).
#include "common.cuh"

#include <algorithm>

namespace pint {

namespace {

inline unsigned nbl(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// x as a TF32 pair: hi = tf32(x), lo = tf32(x - hi) (round to nearest, ties away)
__device__ __forceinline__ void put_split(float* __restrict__ hi, float* __restrict__ lo, size_t o, float x) {
  uint32_t h, l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  const float hf = __uint_as_float(h);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - hf));
  hi[o] = hf;
  lo[o] = __uint_as_float(l);
}

// Squared WR updates are accumulated in FP32: they only steer the stopping
// test, and FP64 conversions cost time on this part's narrow FP64 pipe.
// Sum v[0..P) over the 32 lanes of a warp and add the P totals to acc[0..P):
// recursive halving leaves each lane the totals of a contiguous slice of
// max(P / 32, 1) entries (P a power of two), so one atomic instruction per
// slice entry covers the warp.
template <int P>
__device__ __forceinline__ void warp_sum_scatter(float* v, float* __restrict__ acc, int stride = 1) {
  const int lane = threadIdx.x & 31;
  int off = 0;
  int mask = 16;
#pragma unroll
  for (int C = P; C > 1 && mask >= 1; C >>= 1, mask >>= 1) {
    const int half = C / 2;
    const bool upper = (lane & mask) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const float send = upper ? v[k] : v[k + half];
      const float keep = upper ? v[k + half] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
    }
    if (upper) off += half;
  }
  // P < 32: lanes differing in the remaining low bits hold the same entries
  for (; mask >= 1; mask >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], mask);
  constexpr int KEEP = (P >= 32) ? P / 32 : 1;
  const int low = (P >= 32) ? 0 : (lane & (32 / P - 1));
  if (low == 0) {
#pragma unroll
    for (int k = 0; k < KEEP; ++k) atomicAdd(&acc[(off + k) * stride], v[k]);
  }
}

// FP32 contraction with the WR column maps in difference form:
// MODE 0: out = AR' [w_p ; w_p - w_{max(p-1,0)}] with AR' = [-CA | -CM/dt]
//         (= AR [w_p ; w_{p-1}] of k_wr_gemm without the CM/dt cancellation),
// MODE 1: out = AS [u_p - u_{max(p-1,0)} ; u_{p+1}]
// Trajectories use padded strides ldu, ldw (multiples of 32, pad entries 0);
// the contraction dimension is K = 2 ld with A zero in the pad columns.
template <int MODE>
__global__ void __launch_bounds__(256) k_wr_gemm32(const float* __restrict__ A, int M, int K,
                                                   const float* __restrict__ Ut, const float* __restrict__ Wt,
                                                   int ldu, int ldw, int P, int ncols, float* __restrict__ out,
                                                   const int* __restrict__ gate) {
  if (gate && *gate) return;
  __shared__ float As[16][129], Bs[16][129];
  const int i0 = blockIdx.y * 128, j0 = blockIdx.x * 128;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 8x8 outputs per thread
  float acc[8][8] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 128; e += 256) {
      int kk = e % 16, r = e / 16;
      int kg = k0 + kk, ig = i0 + r, col = j0 + r;
      float av = (kg < K && ig < M) ? A[(size_t)ig * K + kg] : 0.f;
      float bv = 0.f;
      if (kg < K && col < ncols) {
        int n = col / P, p = col % P;
        if (MODE == 0) {
          const float* Wn = Wt + (size_t)n * (P + 1) * ldw;
          bv = (kg < ldw) ? Wn[(size_t)p * ldw + kg]
                          : Wn[(size_t)p * ldw + (kg - ldw)] - Wn[(size_t)(p >= 1 ? p - 1 : 0) * ldw + (kg - ldw)];
        } else {
          const float* Un = Ut + (size_t)n * (P + 1) * ldu;
          if (kg < ldu) bv = Un[(size_t)p * ldu + kg] - Un[(size_t)(p >= 1 ? p - 1 : 0) * ldu + kg];
          else bv = Un[(size_t)(p + 1) * ldu + (kg - ldu)];
        }
      }
      As[kk][r] = av;
      Bs[kk][r] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[8], b[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        a[q] = As[kk][ty + 16 * q];
        b[q] = Bs[kk][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 8; ++p)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int i = i0 + ty + 16 * p, col = j0 + tx + 16 * q;
      if (i < M && col < ncols) out[(size_t)col * M + i] = acc[p][q];
    }
}

// Any P <= 64 outside {16, 32, 64} (the paper's experiments use P = 30, 40,
// 50): eq. (4.7) with the length-P DFTs written as dense products with the
// P x P DFT matrix, for a tile of 32 modes of one interval per CTA.  The
// scaled right-hand sides X[p][s] (p = step, s = mode) sit in shared memory;
// thread (k, s) forms Y_k = sum_p e^{-2 pi i p k / P} X_p, divides by
// d_k + lambda_s, and the inverse product sum_k e^{+2 pi i p k / P} Q_k gives
// the new states (real part; the imaginary part vanishes for real data).
constexpr int MM_NS = 32;  // modes per CTA
__global__ void __launch_bounds__(256) k_time_solve32_mm(const float* __restrict__ R, int d1, int ldu, int P,
                                                         float* __restrict__ Ut, const float* __restrict__ lam1,
                                                         const float* __restrict__ src,
                                                         const float* __restrict__ b1,
                                                         const double* __restrict__ amp, float alpha, float dt,
                                                         const float2* __restrict__ tw,
                                                         const float2* __restrict__ dsh,
                                                         const float* __restrict__ bpow, float* __restrict__ accU,
                                                         float* __restrict__ B1h, float* __restrict__ B1l,
                                                         const int* __restrict__ gate) {
  if (gate && *gate) return;
  constexpr int LD = MM_NS + 1;
  __shared__ float sX[64 * LD];    // scaled right-hand sides, then the new states
  __shared__ float sQr[64 * LD];   // shifted-solve results (real, imaginary)
  __shared__ float sQi[64 * LD];
  __shared__ float2 stw[64];
  __shared__ float su0[MM_NS], suP[MM_NS];
  const int nloc = blockIdx.y, i0 = blockIdx.x * MM_NS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* Un = Ut + (size_t)nloc * (P + 1) * ldu;
  const float an = (float)amp[nloc];
  for (int k = tid; k < P; k += 256) stw[k] = tw[k];
  if (tid < MM_NS) {
    const int i = i0 + tid;
    su0[tid] = i < d1 ? Un[i] : 0.f;
    suP[tid] = i < d1 ? Un[(size_t)P * ldu + i] : 0.f;  // u_P of the previous iterate
  }
  __syncthreads();
  for (int e = tid; e < P * MM_NS; e += 256) {
    const int p = e / MM_NS, s = e % MM_NS, i = i0 + s;
    float y = 0.f;
    if (i < d1) {
      y = R[((size_t)nloc * P + p) * d1 + i] + (src ? src[((size_t)nloc * P + p) * d1 + i] : b1[i] * an);
      if (p == 0) y += (su0[s] - alpha * suP[s]) / dt;
      y *= bpow[p];
    }
    sX[p * LD + s] = y;
  }
  __syncthreads();
  for (int e = tid; e < P * MM_NS; e += 256) {
    const int k = e / MM_NS, s = e % MM_NS, i = i0 + s;
    float yr = 0.f, yi = 0.f;
    int m = 0;  // (p k) mod P
    for (int p = 0; p < P; ++p) {
      const float2 w = stw[m];
      const float x = sX[p * LD + s];
      yr = fmaf(w.x, x, yr);
      yi = fmaf(w.y, x, yi);
      m += k;
      if (m >= P) m -= P;
    }
    const float2 d = dsh[k];
    const float a = d.x + (i < d1 ? lam1[i] : 0.f), c = d.y, inv = 1.f / (a * a + c * c);
    sQr[k * LD + s] = (yr * a + yi * c) * inv;
    sQi[k * LD + s] = (yi * a - yr * c) * inv;
  }
  __syncthreads();
  for (int e = tid; e < P * MM_NS; e += 256) {
    const int p = e / MM_NS, s = e % MM_NS;
    float y = 0.f;
    int m = 0;  // (p k) mod P; conj(tw) = e^{+2 pi i m / P}
    for (int k = 0; k < P; ++k) {
      const float2 w = stw[m];
      y = fmaf(w.x, sQr[k * LD + s], y);
      y = fmaf(w.y, sQi[k * LD + s], y);
      m += p;
      if (m >= P) m -= P;
    }
    sX[p * LD + s] = y / ((float)P * bpow[p]);
  }
  __syncthreads();
  // new states, column map, squared updates (a warp per step row, lane = mode)
  for (int p = warp; p < P; p += 8) {
    const int i = i0 + lane;
    float dd = 0.f;
    if (i < d1) {
      const float uq = sX[p * LD + lane];
      const float old = Un[(size_t)(p + 1) * ldu + i];
      Un[(size_t)(p + 1) * ldu + i] = uq;
      if (B1h) {  // second-contraction column map [u_p - u_{p-1} ; u_{p+1}]
        const size_t o = ((size_t)nloc * P + p) * 2 * ldu + i;
        const float dp = (p == 0) ? 0.f : sX[(p - 1) * LD + lane] - (p == 1 ? su0[lane] : sX[(p - 2) * LD + lane]);
        put_split(B1h, B1l, o, dp);
        put_split(B1h, B1l, o + ldu, uq);
      }
      dd = (uq - old) * (uq - old);
    }
    dd = pintd::warp_sumf(dd);
    if (lane == 0) atomicAdd(&accU[(size_t)nloc * P + p], dd);
  }
}

// Register-resident variant for P = 16, 32, 64: the P values of a series stay
// in registers.  Forward transform by decimation in frequency (natural order
// in, bit-reversed out), the pointwise divide with the shift table already
// permuted to bit-reversed order, inverse by decimation in time (bit-reversed
// in, natural out); one template instance per stage so every index is a
// compile-time constant.  Squared updates are reduced per warp.
template <int P, int LEN>
__device__ __forceinline__ void dif_stage(float* re, float* im, const float2* __restrict__ tw, float sign) {
#pragma unroll
  for (int i = 0; i < P; i += LEN) {
#pragma unroll
    for (int k = 0; k < LEN / 2; ++k) {
      const float2 t = tw[k * (P / LEN)];
      const float wr = t.x, wi = sign * t.y;
      const int a = i + k, b = i + k + LEN / 2;
      const float dr = re[a] - re[b], di = im[a] - im[b];
      re[a] += re[b];
      im[a] += im[b];
      re[b] = dr * wr - di * wi;
      im[b] = dr * wi + di * wr;
    }
  }
  if constexpr (LEN > 2) dif_stage<P, LEN / 2>(re, im, tw, sign);
}

template <int P, int LEN>
__device__ __forceinline__ void dit_stage(float* re, float* im, const float2* __restrict__ tw, float sign) {
#pragma unroll
  for (int i = 0; i < P; i += LEN) {
#pragma unroll
    for (int k = 0; k < LEN / 2; ++k) {
      const float2 t = tw[k * (P / LEN)];
      const float wr = t.x, wi = sign * t.y;
      const int a = i + k, b = i + k + LEN / 2;
      const float br = re[b] * wr - im[b] * wi, bi = re[b] * wi + im[b] * wr;
      re[b] = re[a] - br;
      im[b] = im[a] - bi;
      re[a] += br;
      im[a] += bi;
    }
  }
  if constexpr (LEN < P) dit_stage<P, LEN * 2>(re, im, tw, sign);
}

template <int P>
__global__ void __launch_bounds__(128) k_time_solve32_t(const float* __restrict__ R, int d1, int ldu,
                                                        float* __restrict__ Ut, const float* __restrict__ lam1,
                                                        const float* __restrict__ src, const float* __restrict__ b1,
                                                        const double* __restrict__ amp, float alpha, float dt,
                                                        const float2* __restrict__ tw,
                                                        const float2* __restrict__ dsh,
                                                        const float* __restrict__ bpow, float* __restrict__ accU,
                                                        float* __restrict__ B1h, float* __restrict__ B1l, const int* __restrict__ gate) {
  if (gate && *gate) return;
  const int nloc = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  float re[P], im[P];
  float* Un = Ut + (size_t)nloc * (P + 1) * ldu;
  const bool act = i < d1;
  float u0 = 0.f;
  if (act) {
    const float cs = src ? 0.f : b1[i] * (float)amp[nloc];
    u0 = Un[i];
    const float first = (u0 - alpha * Un[(size_t)P * ldu + i]) / dt;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      float y = R[((size_t)nloc * P + p) * d1 + i] + (src ? src[((size_t)nloc * P + p) * d1 + i] : cs);
      if (p == 0) y += first;
      re[p] = y * bpow[p];
      im[p] = 0.f;
    }
    dif_stage<P, P>(re, im, tw, 1.f);                  // forward, output in bit-reversed order
    const float li = lam1[i];
#pragma unroll
    for (int q = 0; q < P; ++q) {                      // dsh_br[q] = d_{bitrev(q)}
      const float2 d = dsh[q];
      const float a = d.x + li, b = d.y, den = a * a + b * b;
      const float qr = (re[q] * a + im[q] * b) / den, qi = (im[q] * a - re[q] * b) / den;
      re[q] = qr;
      im[q] = qi;
    }
    dit_stage<P, 2>(re, im, tw, -1.f);                 // inverse from bit-reversed input (without 1/P)
#pragma unroll
    for (int p = 0; p < P; ++p) re[p] = re[p] / ((float)P * bpow[p]);
    // previous iterate: every load issued before any store
#pragma unroll
    for (int p = 0; p < P; ++p) im[p] = Un[(size_t)(p + 1) * ldu + i];
#pragma unroll
    for (int p = 0; p < P; ++p) Un[(size_t)(p + 1) * ldu + i] = re[p];
    if (B1h) {  // second-contraction column map [u_p - u_{p-1} ; u_{p+1}]
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const size_t o = ((size_t)nloc * P + p) * 2 * ldu + i;
        const float dp = (p == 0) ? 0.f : re[p - 1] - (p == 1 ? u0 : re[p - 2]);
        put_split(B1h, B1l, o, dp);
        put_split(B1h, B1l, o + ldu, re[p]);
      }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const float d = re[p] - im[p];
      im[p] = d * d;
    }
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p) im[p] = 0.f;
  }
  (void)lane;
  warp_sum_scatter<P>(im, accU + (size_t)nloc * P);
}

// WR stopping test fused into the W recurrence, the last kernel of a WR
// iteration, in two levels so that no single block walks all entries: the
// blocks of interval n (blockIdx.y) count themselves done on the interval's
// counter; the last of them (all atomics of the interval then visible) takes
// the max of the interval's 2 P squared norms (u and w parts), clears them for
// the next iteration, folds the max into a global max (non-negative floats
// order like their bit patterns) and counts the interval done; the last
// interval writes sqrt(max) and a non-finite flag to out, sets the gate when
// the update is below tol (or non-finite) and resets the global words.  No
// block waits on another.
__device__ void wr_stop_last_block(const WrStop& ws, int P) {
  __shared__ int s_last;
  const int nloc = blockIdx.y, nint = gridDim.y;
  unsigned* cnt_n = ws.counter + 3 + nloc;  // per-interval counters
  unsigned* gmax = ws.counter;              // [0] max bits, [1] non-finite, [2] intervals done
  __threadfence();                          // this block's atomics before its count
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(cnt_n, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  float m = 0.f;
  int bad = 0;
  const int half = ws.cnt / 2;  // u part [0, half), w part [half, cnt); interval n owns P of each
  for (int e = threadIdx.x; e < 2 * P; e += blockDim.x) {
    const int idx = (e < P) ? nloc * P + e : half + nloc * P + (e - P);
    const float v = __ldcg(ws.acc + idx);
    if (!(v <= 3.0e38f)) bad = 1;  // NaN or inf
    m = fmaxf(m, v);
    ws.acc[idx] = 0.f;
  }
  for (int o = 16; o >= 1; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  __shared__ float s_m[32];
  __shared__ int s_b[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) {
    s_m[warp] = m;
    s_b[warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < nw; ++w) {
    m = fmaxf(m, s_m[w]);
    bad |= s_b[w];
  }
  *cnt_n = 0u;
  atomicMax(gmax, __float_as_uint(m));
  if (bad) atomicOr(gmax + 1, 1u);
  __threadfence();
  if (atomicAdd(gmax + 2, 1u) != (unsigned)nint - 1) return;
  __threadfence();
  const float mx = __uint_as_float(__ldcg(gmax));
  const int nf = (int)__ldcg(gmax + 1);
  const double nrm = sqrt((double)mx);
  ws.out[0] = nrm;
  ws.out[1] = nf ? 1.0 : 0.0;
  if (nf || nrm <= ws.tol) *ws.gate = 1;
  gmax[0] = 0u;
  gmax[1] = 0u;
  gmax[2] = 0u;
}

__global__ void __launch_bounds__(128) k_w_sweep32(const float* __restrict__ S, int d2, int ldw, int P,
                                                   float* __restrict__ Wt, const float* __restrict__ lam2,
                                                   const float* __restrict__ src, const float* __restrict__ b2,
                                                   const double* __restrict__ amp, float dt, int nsl,
                                                   size_t slice, float* __restrict__ accW,
                                                   float* __restrict__ B0h, float* __restrict__ B0l, WrStop ws) {
  if (*ws.gate) return;
  const int nloc = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  float* Wn = Wt + (size_t)nloc * (P + 1) * ldw;
  float w = 0.f, fac = 0.f, cs = 0.f;
  if (j < d2) {
    w = Wn[j];
    fac = 1.f - dt * lam2[j];
    cs = src ? 0.f : dt * b2[j] * (float)amp[nloc];
  }
  for (int p = 0; p < P; ++p) {
    double dw = 0.0;
    if (j < d2) {
      float g = src ? src[((size_t)nloc * P + p) * d2 + j] : cs;
      float sv = 0.f;
      for (int z = 0; z < nsl; ++z) sv += S[(size_t)z * slice + ((size_t)nloc * P + p) * d2 + j];
      float wn = fac * w + sv + g;
      float old = Wn[(size_t)(p + 1) * ldw + j];
      dw = (double)(wn - old) * (double)(wn - old);
      Wn[(size_t)(p + 1) * ldw + j] = wn;
      if (B0h && p + 1 < P) {  // first-contraction column map of step p + 1: [w_{p+1} ; w_{p+1} - w_p]
        const size_t o = ((size_t)nloc * P + p + 1) * 2 * ldw + j;
        put_split(B0h, B0l, o, wn);
        put_split(B0h, B0l, o + ldw, wn - w);
      }
      w = wn;
    }
    dw = pintd::warp_sum(dw);
    if ((threadIdx.x & 31) == 0) atomicAdd(&accW[(size_t)nloc * P + p], (float)dw);
  }
  wr_stop_last_block(ws, P);
}

// ---------------------------------------------------------------------------
// Refinement residual contractions in double-float arithmetic.
//
// The residual's terms are O(|x|) and cancel down to the rounding of the FP32
// trajectory, so its products need more than FP32 accumulation but not the
// full FP64 format: ~34 correct bits suffice.  GB300's FP64 pipe is narrow
// (~1.1 TFLOP/s), its FP32 pipe tens of times wider, so the products run as
// double-float arithmetic (a value is the unevaluated pair hi + lo of two
// FP32 numbers, ~48 bits): each product's high part is formed exactly by the
// FMA form of Dekker's product (p = ah bh, e = fma(ah, bh, -p)), the cross
// terms ah bl + al bh join the error term, and the running sum is kept as a
// pair, Knuth's TwoSum on the high parts and the errors summed in FP32.
// Same column maps as k_wr_gemm (FP64 path), operands pre-split into pairs.
// Tiles of TM rows x TN columns, (TM / 16) x (TN / 16) outputs per thread.
// The next 16-wide K tile's operands are loaded into registers while the
// current one is multiplied (its differences formed when they are stored to
// shared memory), so the global loads' latency overlaps the arithmetic.
template <int MODE, int TM, int TN>
__global__ void __launch_bounds__(256) k_wr_gemm_df(const float* __restrict__ Ah, const float* __restrict__ Al,
                                                    int M, int K, const float* __restrict__ Uh,
                                                    const float* __restrict__ Ul, const float* __restrict__ Wh,
                                                    const float* __restrict__ Wl, int d1, int d2, int P, int ncols,
                                                    double* __restrict__ out) {
  constexpr int RM = TM / 16, RN = TN / 16;
  constexpr int NA = 16 * TM / 256, NB = 16 * TN / 256;  // staged elements per thread
  __shared__ float Ash[16][TM + 1], Asl[16][TM + 1], Bsh[16][TN + 1], Bsl[16][TN + 1];
  const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float sh[RM][RN] = {}, sl[RM][RN] = {};
  // element e = tid + 256 q of a stage: K offset e % 16, row / column e / 16.
  // B values: x (the state) and, for a difference, y (the state before it)
  float pah[NA], pal[NA], pxh[NB], pxl[NB], pyh[NB], pyl[NB];
  bool pdf[NB];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int e = tid + 256 * q, kg = k0 + e % 16, ig = i0 + e / 16;
      const bool in = kg < K && ig < M;
      pah[q] = in ? Ah[(size_t)ig * K + kg] : 0.f;
      pal[q] = in ? Al[(size_t)ig * K + kg] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int e = tid + 256 * q, kg = k0 + e % 16, col = j0 + e / 16;
      pxh[q] = pxl[q] = pyh[q] = pyl[q] = 0.f;
      pdf[q] = false;
      if (kg < K && col < ncols) {
        const int n = col / P, p = col % P;
        if (MODE == 0) {  // [w_p ; w_{max(p-1,0)}]
          const size_t base = (size_t)n * (P + 1) * d2;
          const size_t o = (kg < d2) ? base + (size_t)p * d2 + kg
                                     : base + (size_t)(p >= 1 ? p - 1 : 0) * d2 + (kg - d2);
          pxh[q] = Wh[o];
          pxl[q] = Wl[o];
        } else {  // [u_p - u_{max(p-1,0)} ; u_{p+1}]
          const size_t base = (size_t)n * (P + 1) * d1;
          if (kg < d1) {
            const size_t o1 = base + (size_t)p * d1 + kg, o0 = base + (size_t)(p >= 1 ? p - 1 : 0) * d1 + kg;
            pxh[q] = Uh[o1];
            pxl[q] = Ul[o1];
            pyh[q] = Uh[o0];
            pyl[q] = Ul[o0];
            pdf[q] = true;
          } else {
            const size_t o = base + (size_t)(p + 1) * d1 + (kg - d1);
            pxh[q] = Uh[o];
            pxl[q] = Ul[o];
          }
        }
      }
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int e = tid + 256 * q;
      Ash[e % 16][e / 16] = pah[q];
      Asl[e % 16][e / 16] = pal[q];
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int e = tid + 256 * q;
      float bh = pxh[q], bl = pxl[q];
      if (pdf[q]) pintd::df_sub(pxh[q], pxl[q], pyh[q], pyl[q], bh, bl);
      Bsh[e % 16][e / 16] = bh;
      Bsl[e % 16][e / 16] = bl;
    }
  };
  load(0);
  for (int k0 = 0; k0 < K; k0 += 16) {
    store();
    __syncthreads();
    if (k0 + 16 < K) load(k0 + 16);
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a_h[RM], a_l[RM], b_h[RN], b_l[RN];
      // thread (tx, ty) owns rows ty + 16 p and columns tx + 16 q: the 16
      // lanes of a half-warp read 16 consecutive words (no bank conflicts)
#pragma unroll
      for (int q = 0; q < RM; ++q) {
        a_h[q] = Ash[kk][ty + 16 * q];
        a_l[q] = Asl[kk][ty + 16 * q];
      }
#pragma unroll
      for (int q = 0; q < RN; ++q) {
        b_h[q] = Bsh[kk][tx + 16 * q];
        b_l[q] = Bsl[kk][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < RM; ++p)
#pragma unroll
        for (int q = 0; q < RN; ++q) pintd::df_fma(a_h[p], a_l[p], b_h[q], b_l[q], sh[p][q], sl[p][q]);
    }
    __syncthreads();
  }
  for (int p = 0; p < RM; ++p)
    for (int q = 0; q < RN; ++q) {
      const int i = i0 + ty + 16 * p, col = j0 + tx + 16 * q;
      if (i < M && col < ncols) out[(size_t)col * M + i] = (double)sh[p][q] + (double)sl[p][q];
    }
}

// C[i][j] = sum_k A[i][k] B[j][k] (FP64 in and out, row-major) in
// double-float arithmetic on the FP32 pipe: the operands are split into FP32
// pairs as they are staged in shared memory, the products accumulated as in
// k_wr_gemm_df.  For the conversions of coarse states out of the spectral
// coordinates (a few rows against d x d), which the FP64 pipe would take
// ten times longer to do.
template <int T>
__global__ void __launch_bounds__(256) k_gemm_df_nt(const double* __restrict__ A, const double* __restrict__ B,
                                                    int m, int n, int K, double* __restrict__ C) {
  constexpr int R = T / 16;
  __shared__ float Ash[16][T + 1], Asl[16][T + 1], Bsh[16][T + 1], Bsl[16][T + 1];
  const int i0 = blockIdx.y * T, j0 = blockIdx.x * T;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float sh[R][R] = {}, sl[R][R] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * T; e += 256) {
      const int kk = e % 16, r = e / 16, kg = k0 + kk;
      const double a = (kg < K && i0 + r < m) ? A[(size_t)(i0 + r) * K + kg] : 0.0;
      const double b = (kg < K && j0 + r < n) ? B[(size_t)(j0 + r) * K + kg] : 0.0;
      const float ah = (float)a, bh = (float)b;
      Ash[kk][r] = ah;
      Asl[kk][r] = (float)(a - (double)ah);
      Bsh[kk][r] = bh;
      Bsl[kk][r] = (float)(b - (double)bh);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a_h[R], a_l[R], b_h[R], b_l[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        a_h[q] = Ash[kk][ty * R + q];
        a_l[q] = Asl[kk][ty * R + q];
        b_h[q] = Bsh[kk][tx * R + q];
        b_l[q] = Bsl[kk][tx * R + q];
      }
#pragma unroll
      for (int p = 0; p < R; ++p)
#pragma unroll
        for (int q = 0; q < R; ++q) pintd::df_fma(a_h[p], a_l[p], b_h[q], b_l[q], sh[p][q], sl[p][q]);
    }
    __syncthreads();
  }
  for (int p = 0; p < R; ++p)
    for (int q = 0; q < R; ++q) {
      const int i = i0 + ty * R + p, j = j0 + tx * R + q;
      if (i < m && j < n) C[(size_t)i * n + j] = (double)sh[p][q] + (double)sl[p][q];
    }
}

// x -> (h, l) with h = fl32(x), l = fl32(x - h)
__global__ void k_split_df(const double* __restrict__ x, long long n, float* __restrict__ h, float* __restrict__ l) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double v = x[e];
    const float hv = (float)v;
    h[e] = hv;
    l[e] = (float)(v - (double)hv);
  }
}

// ---------------------------------------------------------------------------
// Four-step variant for P = R^2 (R = 4, 8): R lanes share one series.  With
// p = g + R m and k = a + R b (g, a the lane in the group; m, b registers),
//   Y[a + R b] = sum_g w_R^{g b} w_P^{g a} sum_m w_R^{m a} y[g + R m],
// so each lane runs an R-point DFT over its registers, applies its twiddles
// w_P^{g a}, the group transposes its R x R block through shuffles, and a
// second R-point DFT leaves lane a holding Y[a + R b].  The inverse is the
// same procedure with conjugate roots and returns lane g holding y[g + R m].
// The right-hand sides and results pass through a shared-memory tile so that
// every global access is coalesced along the modes.

// cos / sin of 2 pi k / 8
__host__ __device__ constexpr float cos8(int k) {
  return k == 0 ? 1.f : k == 1 ? 0.70710678118654752f : k == 2 ? 0.f : k == 3 ? -0.70710678118654752f
       : k == 4 ? -1.f : k == 5 ? -0.70710678118654752f : k == 6 ? 0.f : 0.70710678118654752f;
}
__host__ __device__ constexpr float sin8(int k) { return cos8((k + 6) & 7); }
__host__ __device__ constexpr int bitrev(int k, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b)
    if (k & (1 << b)) r |= 1 << (bits - 1 - b);
  return r;
}

// radix-2 decimation-in-frequency stages of an R-point DFT with roots
// e^{SGN 2 pi i / R} (R <= 8): natural order in, bit-reversed order out
template <int R, int LEN, int SGN>
__device__ __forceinline__ void small_dif(float* re, float* im) {
#pragma unroll
  for (int i0 = 0; i0 < R; i0 += LEN) {
#pragma unroll
    for (int k = 0; k < LEN / 2; ++k) {
      const int ti = k * (8 / LEN);
      const float wr = cos8(ti), wi = SGN * sin8(ti);
      const int a = i0 + k, b = a + LEN / 2;
      const float dr = re[a] - re[b], di = im[a] - im[b];
      re[a] += re[b];
      im[a] += im[b];
      re[b] = dr * wr - di * wi;
      im[b] = dr * wi + di * wr;
    }
  }
  if constexpr (LEN > 2) small_dif<R, LEN / 2, SGN>(re, im);
}

// out[f] = sum_n x[n] e^{SGN 2 pi i n f / R}, in place, natural order
template <int R, int SGN>
__device__ __forceinline__ void small_dft(float* re, float* im) {
  constexpr int BITS = R == 2 ? 1 : R == 4 ? 2 : 3;
  small_dif<R, R, SGN>(re, im);
  float tr[R], ti[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    tr[k] = re[bitrev(k, BITS)];
    ti[k] = im[bitrev(k, BITS)];
  }
#pragma unroll
  for (int k = 0; k < R; ++k) {
    re[k] = tr[k];
    im[k] = ti[k];
  }
}

// a[t] <- a[(t - g) mod R] for the lane's own g, as log2(R) selected rotations
template <int R>
__device__ __forceinline__ void rotate_right(float* a, int g) {
#pragma unroll
  for (int b = 1; b < R; b <<= 1) {
    const bool on = (g & b) != 0;
    float t2[R];
#pragma unroll
    for (int t = 0; t < R; ++t) t2[t] = a[(t - b + R) % R];
#pragma unroll
    for (int t = 0; t < R; ++t) a[t] = on ? t2[t] : a[t];
  }
}

// lane g of an R-lane group (first lane `base`) holds X_g[0..R); afterwards
// it holds X_0[g] .. X_{R-1}[g].  Round t reads lane (g + t) mod R, which
// sends X_{g+t}[g] once its registers are reversed and rotated by its g.
template <int R>
__device__ __forceinline__ void group_transpose(float* v, int g, int base) {
  float a[R];
#pragma unroll
  for (int t = 0; t < R; ++t) a[t] = v[(R - t) % R];
  rotate_right<R>(a, g);
#pragma unroll
  for (int t = 0; t < R; ++t) a[t] = __shfl_sync(0xffffffffu, a[t], base + ((g + t) & (R - 1)));
  rotate_right<R>(a, g);
#pragma unroll
  for (int t = 0; t < R; ++t) v[t] = a[t];
}

__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Eq. (4.7) for one mode over two intervals at once: every solved series is
// real (the WR system is real), so intervals na (real part) and na + 1
// (imaginary part) share one complex series through the forward DFT, the
// shifted division (a complex scalar per frequency, the same for both) and
// the inverse DFT, and come out as the real and imaginary parts: half the DFT
// work of one series per interval.
template <int R>
__global__ void __launch_bounds__(256, 3) k_time_solve32_sq(const float* __restrict__ Rc, int d1, int ldu,
                                                         float* __restrict__ Ut, const float* __restrict__ lam1,
                                                         const float* __restrict__ src,
                                                         const float* __restrict__ b1,
                                                         const double* __restrict__ amp, float alpha, float dt,
                                                         const float2* __restrict__ tw,
                                                         const float2* __restrict__ dsh,
                                                         const float* __restrict__ bpow, float* __restrict__ accU,
                                                         float* __restrict__ B1h, float* __restrict__ B1l,
                                                         const int* __restrict__ gate, int nact) {
  if (gate && *gate) return;
  constexpr int P = R * R;       // steps per interval
  constexpr int NS = 256 / R;    // series (modes) per block
  constexpr int LD = NS + 1;     // tile row stride
  constexpr int PER = P * NS / 256;
  __shared__ float sT[2][P * LD];  // right-hand sides, then the new states (per interval of the pair)
  __shared__ float sO[2][P * LD];  // previous iterate u_{p+1}
  __shared__ float su0[2][NS];
  const int na = 2 * blockIdx.y, i0 = blockIdx.x * NS;
  const int npair = (na + 1 < nact) ? 2 : 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // every global read of the block is issued at once as asynchronous copies
  // into shared memory (the contraction output and the previous iterate)
  for (int h = 0; h < npair; ++h) {
    const int nloc = na + h;
    const float* Un = Ut + (size_t)nloc * (P + 1) * ldu;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int e = tid + 256 * r, p = e / NS, s = e % NS, i = i0 + s;
      if (i < d1) {
        cp_async4(&sT[h][p * LD + s], Rc + ((size_t)nloc * P + p) * d1 + i);
        cp_async4(&sO[h][p * LD + s], Un + (size_t)(p + 1) * ldu + i);
      } else {
        sT[h][p * LD + s] = 0.f;
        sO[h][p * LD + s] = 0.f;
      }
    }
    if (tid < NS) su0[h][tid] = (i0 + tid < d1) ? Un[i0 + tid] : 0.f;
  }
  cp_async_wait_all();
  __syncthreads();
  // right-hand sides of eq. (4.7) scaled by beta^p, tile [p][mode]
  for (int h = 0; h < npair; ++h) {
    const int nloc = na + h;
    const float an = (float)amp[nloc];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int e = tid + 256 * r, p = e / NS, s = e % NS, i = i0 + s;
      float y = 0.f;
      if (i < d1) {
        y = sT[h][p * LD + s] + (src ? src[((size_t)nloc * P + p) * d1 + i] : b1[i] * an);
        if (p == 0) y += (su0[h][s] - alpha * sO[h][(P - 1) * LD + s]) / dt;  // u_P of the previous iterate
        y *= bpow[p];
      }
      sT[h][p * LD + s] = y;
    }
  }
  __syncthreads();
  // one series per R-lane group; series s = warp + 8 j keeps the tile reads
  // free of bank conflicts for R = 8
  const int g = lane % R, j = lane / R, s = warp + 8 * j, base = lane - g;
  const int i = i0 + s;
  const float li = (i < d1) ? lam1[i] : 0.f;
  float re[R], im[R], twr[R], twi[R];
#pragma unroll
  for (int m = 0; m < R; ++m) {
    re[m] = sT[0][(g + R * m) * LD + s];
    im[m] = npair == 2 ? sT[1][(g + R * m) * LD + s] : 0.f;
  }
#pragma unroll
  for (int a = 0; a < R; ++a) {
    const float2 t = tw[(g * a) % P];  // e^{-2 pi i g a / P}
    twr[a] = t.x;
    twi[a] = t.y;
  }
  small_dft<R, -1>(re, im);
#pragma unroll
  for (int a = 0; a < R; ++a) {
    const float xr = re[a] * twr[a] - im[a] * twi[a], xi = re[a] * twi[a] + im[a] * twr[a];
    re[a] = xr;
    im[a] = xi;
  }
  group_transpose<R>(re, g, base);
  group_transpose<R>(im, g, base);
  small_dft<R, -1>(re, im);  // lane g: Y[g + R b]
#pragma unroll
  for (int b = 0; b < R; ++b) {
    const float2 d = dsh[g + R * b];
    const float a = d.x + li, c = d.y, inv = __frcp_rn(a * a + c * c);
    const float qr = (re[b] * a + im[b] * c) * inv, qi = (im[b] * a - re[b] * c) * inv;
    re[b] = qr;
    im[b] = qi;
  }
  small_dft<R, 1>(re, im);
#pragma unroll
  for (int a = 0; a < R; ++a) {
    const float xr = re[a] * twr[a] + im[a] * twi[a], xi = im[a] * twr[a] - re[a] * twi[a];
    re[a] = xr;
    im[a] = xi;
  }
  group_transpose<R>(re, g, base);
  group_transpose<R>(im, g, base);
  small_dft<R, 1>(re, im);  // lane g: P y[g + R m] (real part: interval na, imaginary part: na + 1)
  __syncthreads();          // every read of the right-hand sides is done
#pragma unroll
  for (int m = 0; m < R; ++m) {
    const float sc = 1.f / ((float)P * bpow[g + R * m]);
    sT[0][(g + R * m) * LD + s] = re[m] * sc;
    sT[1][(g + R * m) * LD + s] = im[m] * sc;
  }
  __syncthreads();
  // new states u_{p+1} (tile row p); the previous iterate is in sO.  Row r
  // of this thread is step p = (tid + 256 r) / NS: the warp's lanes share it
  for (int h = 0; h < npair; ++h) {
    const int nloc = na + h;
    float* Un = Ut + (size_t)nloc * (P + 1) * ldu;
    float dd[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int e = tid + 256 * r, p = e / NS, ss = e % NS, ii = i0 + ss;
      dd[r] = 0.f;
      if (ii < d1) {
        const float uq = sT[h][p * LD + ss];
        Un[(size_t)(p + 1) * ldu + ii] = uq;
        if (B1h) {  // second-contraction column map [u_p - u_{p-1} ; u_{p+1}]
          const size_t o = ((size_t)nloc * P + p) * 2 * ldu + ii;
          const float dp =
              (p == 0) ? 0.f : sT[h][(p - 1) * LD + ss] - (p == 1 ? su0[h][ss] : sT[h][(p - 2) * LD + ss]);
          put_split(B1h, B1l, o, dp);
          put_split(B1h, B1l, o + ldu, uq);
        }
        const float dv = uq - sO[h][p * LD + ss];
        dd[r] = dv * dv;
      }
    }
    // one reduce-scatter over the warp for all PER rows (steps tid / NS + r 256 / NS)
    warp_sum_scatter<PER>(dd, accU + (size_t)nloc * P + (tid - lane) / NS, 256 / NS);
  }
}

// Register variant for P = 16, 32, 64: the contraction inputs and previous
// states of 16 steps at a time are loaded before the recurrence consumes them.
constexpr int MAX_SLICES = 4;
template <int P>
__global__ void __launch_bounds__(32) k_w_sweep32_t(const float* __restrict__ S, int d2, int ldw,
                                                    float* __restrict__ Wt, const float* __restrict__ lam2,
                                                    const float* __restrict__ src, const float* __restrict__ b2,
                                                    const double* __restrict__ amp, float dt, int nsl,
                                                    size_t slice, float* __restrict__ accW,
                                                    float* __restrict__ B0h, float* __restrict__ B0l, WrStop ws) {
  if (*ws.gate) return;
  constexpr int CH = 16;
  const int nloc = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = j < d2;
  float* Wn = Wt + (size_t)nloc * (P + 1) * ldw;
  const float fac = act ? 1.f - dt * lam2[j] : 0.f;
  const float cs = (act && !src) ? dt * b2[j] * (float)amp[nloc] : 0.f;
  float w = act ? Wn[j] : 0.f;
  // chunks of CH steps, kept rolled (a fully unrolled sweep overflows the
  // instruction cache); the squared updates of a chunk are reduced at its end
#pragma unroll 1
  for (int c0 = 0; c0 < P; c0 += CH) {
    float sv[CH], ov[CH], dd[CH];
    if (act) {
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const size_t o = ((size_t)nloc * P + c0 + q) * d2 + j;
        float a = src ? src[o] : cs;
#pragma unroll
        for (int z = 0; z < MAX_SLICES; ++z)
          if (z < nsl) a += S[(size_t)z * slice + o];
        sv[q] = a;
        ov[q] = Wn[(size_t)(c0 + q + 1) * ldw + j];
      }
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int p = c0 + q;
        const float wn = fac * w + sv[q];
        Wn[(size_t)(p + 1) * ldw + j] = wn;
        if (B0h && p + 1 < P) {  // first-contraction column map of step p + 1: [w_{p+1} ; w_{p+1} - w_p]
          const size_t o = ((size_t)nloc * P + p + 1) * 2 * ldw + j;
          put_split(B0h, B0l, o, wn);
          put_split(B0h, B0l, o + ldw, wn - w);
        }
        const float d = wn - ov[q];
        dd[q] = d * d;
        w = wn;
      }
    } else {
#pragma unroll
      for (int q = 0; q < CH; ++q) dd[q] = 0.f;
    }
    warp_sum_scatter<CH>(dd, accW + (size_t)nloc * P + c0);
  }
  wr_stop_last_block(ws, P);
}

// One block per interval for d2 <= 512 (thread j = column j): the squared
// updates of the interval's w steps meet in shared memory instead of global
// atomics, and the block itself takes the interval's max over its 2 P
// squared norms (the u part left in accU by the time solve), so the fused
// stopping test needs one counter per launch, not one per interval.
template <int P>
__global__ void __launch_bounds__(512) k_w_sweep32_b(const float* __restrict__ S, int d2, int ldw,
                                                      float* __restrict__ Wt, const float* __restrict__ lam2,
                                                      const float* __restrict__ src, const float* __restrict__ b2,
                                                      const double* __restrict__ amp, float dt, int nsl,
                                                      size_t slice, float* __restrict__ B0h,
                                                      float* __restrict__ B0l, WrStop ws) {
  if (*ws.gate) return;
  constexpr int CH = 16;
  __shared__ float sW[16][P];  // per-warp sums of the squared w updates
  __shared__ float s_m[32];
  __shared__ int s_b[32];
  const int nloc = blockIdx.x;
  const int j = threadIdx.x, lane = j & 31, warp = j >> 5, nw = (blockDim.x + 31) >> 5;
  const bool act = j < d2;
  float* Wn = Wt + (size_t)nloc * (P + 1) * ldw;
  const float fac = act ? 1.f - dt * lam2[j] : 0.f;
  const float cs = (act && !src) ? dt * b2[j] * (float)amp[nloc] : 0.f;
  float w = act ? Wn[j] : 0.f;
#pragma unroll 1
  for (int c0 = 0; c0 < P; c0 += CH) {
    float sv[CH], ov[CH], dd[CH];
    if (act) {
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const size_t o = ((size_t)nloc * P + c0 + q) * d2 + j;
        float a = src ? src[o] : cs;
#pragma unroll
        for (int z = 0; z < MAX_SLICES; ++z)
          if (z < nsl) a += S[(size_t)z * slice + o];
        sv[q] = a;
        ov[q] = Wn[(size_t)(c0 + q + 1) * ldw + j];
      }
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int p = c0 + q;
        const float wn = fac * w + sv[q];
        Wn[(size_t)(p + 1) * ldw + j] = wn;
        if (B0h && p + 1 < P) {  // first-contraction column map of step p + 1: [w_{p+1} ; w_{p+1} - w_p]
          const size_t o = ((size_t)nloc * P + p + 1) * 2 * ldw + j;
          put_split(B0h, B0l, o, wn);
          put_split(B0h, B0l, o + ldw, wn - w);
        }
        const float d = wn - ov[q];
        dd[q] = d * d;
        w = wn;
      }
    } else {
#pragma unroll
      for (int q = 0; q < CH; ++q) dd[q] = 0.f;
    }
    // butterfly reduce-scatter over the warp: lane pairs (2 l, 2 l + 1) end
    // with the warp's sum for step c0 + off of the chunk
    int off = 0;
    int mask = 16;
#pragma unroll
    for (int C = CH; C > 1; C >>= 1, mask >>= 1) {
      const int half = C / 2;
      const bool upper = (lane & mask) != 0;
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const float send = upper ? dd[k] : dd[k + half];
        const float keep = upper ? dd[k + half] : dd[k];
        dd[k] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
      }
      if (upper) off += half;
    }
    dd[0] += __shfl_xor_sync(0xffffffffu, dd[0], 1);
    if ((lane & 1) == 0) sW[warp][c0 + off] = dd[0];
  }
  __syncthreads();
  // the interval's max over its u and w squared norms; clear the u sums
  float m = 0.f;
  int bad = 0;
  for (int p = j; p < P; p += blockDim.x) {
    float sw = 0.f;
    for (int g = 0; g < nw; ++g) sw += sW[g][p];
    float* au = ws.acc + (size_t)nloc * P + p;
    const float su = __ldcg(au);
    *au = 0.f;
    if (!(sw <= 3.0e38f) || !(su <= 3.0e38f)) bad = 1;  // NaN or inf
    m = fmaxf(m, fmaxf(sw, su));
  }
  for (int o = 16; o >= 1; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if (lane == 0) {
    s_m[warp] = m;
    s_b[warp] = bad;
  }
  __syncthreads();
  if (j != 0) return;
  for (int g = 1; g < nw; ++g) {
    m = fmaxf(m, s_m[g]);
    bad |= s_b[g];
  }
  unsigned* gmax = ws.counter;  // [0] max bits, [1] non-finite, [2] intervals done
  atomicMax(gmax, __float_as_uint(m));
  if (bad) atomicOr(gmax + 1, 1u);
  __threadfence();
  if (atomicAdd(gmax + 2, 1u) != gridDim.x - 1) return;
  __threadfence();
  const float mx = __uint_as_float(__ldcg(gmax));
  const int nf = (int)__ldcg(gmax + 1);
  const double nrm = sqrt((double)mx);
  ws.out[0] = nrm;
  ws.out[1] = nf ? 1.0 : 0.0;
  if (nf || nrm <= ws.tol) *ws.gate = 1;
  gmax[0] = 0u;
  gmax[1] = 0u;
  gmax[2] = 0u;
}

// constant initial trajectories; with B0h, also the first-contraction column
// map [w_p ; w_p - w_{p-1}] = [x_w ; 0] of every step
__global__ void k_init32(const double* __restrict__ Xu, const double* __restrict__ Xw, int d1, int d2, int ldu,
                         int ldw, int P, float* __restrict__ Ut, float* __restrict__ Wt, float* __restrict__ B0h,
                         float* __restrict__ B0l) {
  const int nloc = blockIdx.y;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < (P + 1) * (d1 + d2); e += gridDim.x * blockDim.x) {
    int p = e / (d1 + d2), k = e % (d1 + d2);
    if (k < d1) {
      Ut[((size_t)nloc * (P + 1) + p) * ldu + k] = (float)Xu[(size_t)nloc * d1 + k];
    } else {
      const int j = k - d1;
      const float x = (float)Xw[(size_t)nloc * d2 + j];
      Wt[((size_t)nloc * (P + 1) + p) * ldw + j] = x;
      if (B0h && p < P) {  // constant trajectory: [x_w ; 0]
        const size_t o = ((size_t)nloc * P + p) * 2 * ldw + j;
        put_split(B0h, B0l, o, x);
        put_split(B0h, B0l, o + ldw, 0.f);
      }
    }
  }
}

// interval ends u_P, w_P in FP64 and, when Fu32 is given, in FP32
__global__ void k_ends32(const float* __restrict__ Ut, const float* __restrict__ Wt, int d1, int d2, int ldu,
                         int ldw, int P, double* __restrict__ Fu, double* __restrict__ Fw, float* __restrict__ Fu32,
                         float* __restrict__ Fw32) {
  const int nloc = blockIdx.y;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d1 + d2; e += gridDim.x * blockDim.x) {
    if (e < d1) {
      const float v = Ut[((size_t)nloc * (P + 1) + P) * ldu + e];
      Fu[(size_t)nloc * d1 + e] = (double)v;
      if (Fu32) Fu32[(size_t)nloc * d1 + e] = v;
    } else {
      const float v = Wt[((size_t)nloc * (P + 1) + P) * ldw + (e - d1)];
      Fw[(size_t)nloc * d2 + (e - d1)] = (double)v;
      if (Fw32) Fw32[(size_t)nloc * d2 + (e - d1)] = v;
    }
  }
}

// FP64 trajectory: p = 0 from the FP64 starts, p >= 1 from the FP32 states
__global__ void k_promote(const float* __restrict__ Ut, const float* __restrict__ Wt,
                          const double* __restrict__ Su, const double* __restrict__ Sw, int d1, int d2, int ldu,
                          int ldw, int P, double* __restrict__ Zu, double* __restrict__ Zw) {
  const int n = blockIdx.y;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < (P + 1) * (d1 + d2); e += gridDim.x * blockDim.x) {
    int p = e / (d1 + d2), k = e % (d1 + d2);
    if (k < d1) {
      size_t o = ((size_t)n * (P + 1) + p) * d1 + k;
      Zu[o] = (p == 0) ? Su[(size_t)n * d1 + k] : (double)Ut[((size_t)n * (P + 1) + p) * ldu + k];
    } else {
      size_t o = ((size_t)n * (P + 1) + p) * d2 + (k - d1);
      Zw[o] = (p == 0) ? Sw[(size_t)n * d2 + (k - d1)] : (double)Wt[((size_t)n * (P + 1) + p) * ldw + (k - d1)];
    }
  }
}

// adds a correction trajectory: Z += dZ (p = 0 from the FP64 correction starts)
__global__ void k_add_traj(const float* __restrict__ dUt, const float* __restrict__ dWt,
                           const double* __restrict__ Yu, const double* __restrict__ Yw, int d1, int d2, int ldu,
                           int ldw, int P, double* __restrict__ Zu, double* __restrict__ Zw) {
  const int n = blockIdx.y;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < (P + 1) * (d1 + d2); e += gridDim.x * blockDim.x) {
    int p = e / (d1 + d2), k = e % (d1 + d2);
    if (k < d1) {
      size_t o = ((size_t)n * (P + 1) + p) * d1 + k;
      Zu[o] += (p == 0) ? Yu[(size_t)n * d1 + k] : (double)dUt[((size_t)n * (P + 1) + p) * ldu + k];
    } else {
      size_t o = ((size_t)n * (P + 1) + p) * d2 + (k - d1);
      Zw[o] += (p == 0) ? Yw[(size_t)n * d2 + (k - d1)] : (double)dWt[((size_t)n * (P + 1) + p) * ldw + (k - d1)];
    }
  }
}

// residual of eqs. (2.4)-(2.5) on the FP64 trajectory (see the header):
//   e_u = (1 + dt l1) u_{p+1} - u_p - dt R_p - dt a b1
//   e_w = w_{p+1} - (1 - dt l2) w_p - S_p - dt a b2
// written as the correction sources src_u = -e_u / dt, src_w = -e_w (FP32)
__global__ void k_residual(const double* __restrict__ Zu, const double* __restrict__ Zw,
                           const double* __restrict__ R64, const double* __restrict__ S64,
                           const double* __restrict__ lam1, const double* __restrict__ lam2,
                           const double* __restrict__ b1, const double* __restrict__ b2,
                           const double* __restrict__ amp, double dt, int d1, int d2, int P,
                           float* __restrict__ srcU, float* __restrict__ srcW) {
  const int n = blockIdx.y;
  const double a = amp[n];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P * (d1 + d2); e += gridDim.x * blockDim.x) {
    int p = e / (d1 + d2), k = e % (d1 + d2);
    if (k < d1) {
      const double* Z = Zu + (size_t)n * (P + 1) * d1;
      double r = (1.0 + dt * lam1[k]) * Z[(size_t)(p + 1) * d1 + k] - Z[(size_t)p * d1 + k] -
                 dt * R64[((size_t)n * P + p) * d1 + k] - dt * a * b1[k];
      srcU[((size_t)n * P + p) * d1 + k] = (float)(-r / dt);
    } else {
      int j = k - d1;
      const double* Z = Zw + (size_t)n * (P + 1) * d2;
      double r = Z[(size_t)(p + 1) * d2 + j] - (1.0 - dt * lam2[j]) * Z[(size_t)p * d2 + j] -
                 S64[((size_t)n * P + p) * d2 + j] - dt * a * b2[j];
      srcW[((size_t)n * P + p) * d2 + j] = (float)(-r);
    }
  }
}

// continuity jumps c_n = Z_{n-1,P} - s_n (n = 1..N-1), c_0 = c_N = 0
__global__ void k_continuity(const double* __restrict__ Zu, const double* __restrict__ Zw, int N, int P, int d1,
                             int d2, double* __restrict__ Cu, double* __restrict__ Cw) {
  const int n = blockIdx.y;  // 0..N
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d1 + d2; e += gridDim.x * blockDim.x) {
    bool zero = (n == 0 || n == N);
    if (e < d1) {
      Cu[(size_t)n * d1 + e] = zero ? 0.0
                                    : Zu[((size_t)(n - 1) * (P + 1) + P) * d1 + e] -
                                          Zu[((size_t)n * (P + 1)) * d1 + e];
    } else {
      int j = e - d1;
      Cw[(size_t)n * d2 + j] = zero ? 0.0
                                    : Zw[((size_t)(n - 1) * (P + 1) + P) * d2 + j] -
                                          Zw[((size_t)n * (P + 1)) * d2 + j];
    }
  }
}

// A (rows x 2 dk, FP64) -> A32 (rows x 2 ld, FP32), halves at columns 0 and ld,
// pad columns zero; with hi, also the TF32 pair of every entry
__global__ void k_pad_split(const double* __restrict__ A, int rows, int dk, int ld, float* __restrict__ a32,
                            float* __restrict__ hi, float* __restrict__ lo) {
  long long tot = (long long)rows * 2 * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / (2 * ld)), k = (int)(e % (2 * ld));
    int seg = k / ld, j = k % ld;
    const float v = (j < dk) ? (float)A[(size_t)r * 2 * dk + seg * dk + j] : 0.f;
    a32[e] = v;
    if (hi) put_split(hi, lo, (size_t)e, v);
  }
}

// AR' = [-CA | -CM/dt] (d1 x 2 d2, FP64 couplings) -> FP32 rows of 2 ld with
// both halves padded; with hi, also the TF32 pairs
__global__ void k_ar_diff(const double* __restrict__ CA, const double* __restrict__ CM, double dt, int d1, int d2,
                          int ld, float* __restrict__ a32, float* __restrict__ hi, float* __restrict__ lo) {
  long long tot = (long long)d1 * 2 * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / (2 * ld)), k = (int)(e % (2 * ld));
    const int seg = k / ld, j = k % ld;
    float v = 0.f;
    if (j < d2) v = seg == 0 ? (float)(-CA[(size_t)r * d2 + j]) : (float)(-CM[(size_t)r * d2 + j] / dt);
    a32[e] = v;
    if (hi) put_split(hi, lo, (size_t)e, v);
  }
}

__global__ void k_to_f32(const double* __restrict__ x, long long n, float* __restrict__ y) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) y[e] = (float)x[e];
}

}  // namespace

void mx_contract32(Ctx* c, int mode, const float* A, int M, int K, const float* Ut, const float* Wt, int ldu,
                   int ldw, int P, int ncols, float* out, const int* gate) {
  dim3 grid(nbl(ncols, 128), nbl(M, 128));
  if (mode == 0)
    k_wr_gemm32<0><<<grid, 256, 0, c->stream>>>(A, M, K, Ut, Wt, ldu, ldw, P, ncols, out, gate);
  else
    k_wr_gemm32<1><<<grid, 256, 0, c->stream>>>(A, M, K, Ut, Wt, ldu, ldw, P, ncols, out, gate);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

void mx_time_solve32(Ctx* c, const float* R, int nact, float* Ut, int ldu, const float* lam1, const float* src,
                     const float* b1, const double* amp, const float2* tw, const float2* dsh, const float2* dshbr,
                     const float* bpow, float* accU, float* B1h, float* B1l, const int* gate) {
  const int P = c->P;
  const dim3 grid(nbl(c->d1, 128), nact);
  const float al = (float)c->alpha, dt = (float)c->dt;
  if (P == 64)
    k_time_solve32_sq<8><<<dim3(nbl(c->d1, 32), (nact + 1) / 2), 256, 0, c->stream>>>(
        R, c->d1, ldu, Ut, lam1, src, b1, amp, al, dt, tw, dsh, bpow, accU, B1h, B1l, gate, nact);
  else if (P == 32)
    k_time_solve32_t<32><<<grid, 128, 0, c->stream>>>(R, c->d1, ldu, Ut, lam1, src, b1, amp, al, dt, tw, dshbr, bpow,
                                                       accU, B1h, B1l, gate);
  else if (P == 16)
    k_time_solve32_sq<4><<<dim3(nbl(c->d1, 64), (nact + 1) / 2), 256, 0, c->stream>>>(
        R, c->d1, ldu, Ut, lam1, src, b1, amp, al, dt, tw, dsh, bpow, accU, B1h, B1l, gate, nact);
  else  // other P: the DFTs as products with the DFT matrix
    k_time_solve32_mm<<<dim3(nbl(c->d1, MM_NS), nact), 256, 0, c->stream>>>(R, c->d1, ldu, P, Ut, lam1, src, b1,
                                                                           amp, al, dt, tw, dsh, bpow, accU, B1h,
                                                                           B1l, gate);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

// S holds nsl K-slices of the contraction, slice floats apart (summed here)
void mx_w_sweep32(Ctx* c, const float* S, int nsl, size_t slice, int nact, float* Wt, int ldw, const float* lam2,
                  const float* src, const float* b2, const double* amp, float* accW, float* B0h, float* B0l,
                  const WrStop& ws) {
  PINT_REQUIRE(ws.gate && ws.counter && ws.acc && ws.out, PINT_ERR_BAD_ARG, "WR stopping test arguments");
  PINT_REQUIRE(nsl >= 1 && nsl <= MAX_SLICES, PINT_ERR_BAD_ARG, "too many contraction slices");
  const int P = c->P, d2 = c->d2;
  const float dt = (float)c->dt;
  const dim3 g32(nbl(d2, 32), nact);
  const int tb = (d2 + 31) / 32 * 32;
  if (d2 <= 512 && (P == 64 || P == 32 || P == 16)) {  // one block per interval; accW unused
    if (P == 64)
      k_w_sweep32_b<64><<<nact, tb, 0, c->stream>>>(S, d2, ldw, Wt, lam2, src, b2, amp, dt, nsl, slice, B0h, B0l, ws);
    else if (P == 32)
      k_w_sweep32_b<32><<<nact, tb, 0, c->stream>>>(S, d2, ldw, Wt, lam2, src, b2, amp, dt, nsl, slice, B0h, B0l, ws);
    else
      k_w_sweep32_b<16><<<nact, tb, 0, c->stream>>>(S, d2, ldw, Wt, lam2, src, b2, amp, dt, nsl, slice, B0h, B0l, ws);
  } else if (P == 64)
    k_w_sweep32_t<64><<<g32, 32, 0, c->stream>>>(S, d2, ldw, Wt, lam2, src, b2, amp, dt, nsl, slice, accW, B0h, B0l, ws);
  else if (P == 32)
    k_w_sweep32_t<32><<<g32, 32, 0, c->stream>>>(S, d2, ldw, Wt, lam2, src, b2, amp, dt, nsl, slice, accW, B0h, B0l, ws);
  else if (P == 16)
    k_w_sweep32_t<16><<<g32, 32, 0, c->stream>>>(S, d2, ldw, Wt, lam2, src, b2, amp, dt, nsl, slice, accW, B0h, B0l, ws);
  else
    k_w_sweep32<<<dim3(nbl(d2, 128), nact), 128, 0, c->stream>>>(S, d2, ldw, P, Wt, lam2, src, b2, amp, dt, nsl,
                                                                 slice, accW, B0h, B0l, ws);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

void mx_init32(Ctx* c, const double* Xu, const double* Xw, int nact, float* Ut, float* Wt, int ldu, int ldw,
               float* B0h, float* B0l) {
  k_init32<<<dim3(32, nact), 256, 0, c->stream>>>(Xu, Xw, c->d1, c->d2, ldu, ldw, c->P, Ut, Wt, B0h, B0l);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

void mx_ends32(Ctx* c, const float* Ut, const float* Wt, int ldu, int ldw, int nact, double* Fu, double* Fw,
               float* Fu32, float* Fw32) {
  k_ends32<<<dim3(8, nact), 256, 0, c->stream>>>(Ut, Wt, c->d1, c->d2, ldu, ldw, c->P, Fu, Fw, Fu32, Fw32);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

void mx_promote(Ctx* c, const float* Ut, const float* Wt, int ldu, int ldw, const double* Su, const double* Sw,
                double* Zu, double* Zw) {
  k_promote<<<dim3(64, c->N), 256, 0, c->stream>>>(Ut, Wt, Su, Sw, c->d1, c->d2, ldu, ldw, c->P, Zu, Zw);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

void mx_add_traj(Ctx* c, const float* dUt, const float* dWt, int ldu, int ldw, const double* Yu, const double* Yw,
                 double* Zu, double* Zw) {
  k_add_traj<<<dim3(64, c->N), 256, 0, c->stream>>>(dUt, dWt, Yu, Yw, c->d1, c->d2, ldu, ldw, c->P, Zu, Zw);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

void mx_residual(Ctx* c, const double* Zu, const double* Zw, const double* R64, const double* S64,
                 const double* b1, const double* b2, const double* amp, float* srcU, float* srcW) {
  k_residual<<<dim3(64, c->N), 256, 0, c->stream>>>(Zu, Zw, R64, S64, c->lam1, c->lam2, b1, b2, amp, c->dt,
                                                    c->d1, c->d2, c->P, srcU, srcW);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

void mx_ar_diff(Ctx* c, int ld, float* a32, float* hi, float* lo) {
  k_ar_diff<<<1024, 256, 0, c->stream>>>(c->CA, c->CM, c->dt, c->d1, c->d2, ld, a32, hi, lo);
  PINT_LAUNCH_CHECK();
}

void mx_continuity(Ctx* c, const double* Zu, const double* Zw, double* Cu, double* Cw) {
  k_continuity<<<dim3(8, c->N + 1), 256, 0, c->stream>>>(Zu, Zw, c->N, c->P, c->d1, c->d2, Cu, Cw);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

void mx_pad_split(Ctx* c, const double* A, int rows, int dk, int ld, float* a32, float* hi, float* lo) {
  k_pad_split<<<1024, 256, 0, c->stream>>>(A, rows, dk, ld, a32, hi, lo);
  PINT_LAUNCH_CHECK();
}

void mx_split_df(Ctx* c, const double* x, long long n, float* h, float* l) {
  k_split_df<<<std::min<long long>(nbl(n, 256), 4096), 256, 0, c->stream>>>(x, n, h, l);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

// out = A [column map of the double-float trajectory] (MODE 0: A = AR, rows d1,
// K = 2 d2; MODE 1: A = AS, rows d2, K = 2 d1), all N P columns; T x T tiles
// chosen for an even spread over the SMs
void mx_wr_gemm_df(Ctx* c, int mode, const float* Ah, const float* Al, int M, int K, const float* Uh,
                   const float* Ul, const float* Wh, const float* Wl, int ncols, double* out) {
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  sms = std::max(sms, 1);
  // 16 outputs per thread (64 x 64 or 32 x 128 tiles) keep the FP32 pipe busier
  // than 32 x 32 tiles (4 per thread, bound by shared-memory loads): take the
  // 16-output shape with the larger useful fraction of its tiles, and 32 x 32
  // only when the larger tiles would leave SMs idle
  auto useful = [&](int TM, int TN) {
    const long long t = (long long)nbl(M, TM) * nbl(ncols, TN);
    return (double)M * ncols / ((double)t * TM * TN);
  };
  const long long t64 = (long long)nbl(M, 64) * nbl(ncols, 64), t128 = (long long)nbl(M, 32) * nbl(ncols, 128);
  int choice = useful(32, 128) > useful(64, 64) + 1e-9 ? 1 : 0;
  if ((choice == 0 ? t64 : t128) < sms) choice = 2;
  const int d1 = c->d1, d2 = c->d2, P = c->P;
#define PINT_DF_LAUNCH(MODE, TM, TN)                                                                        \
  k_wr_gemm_df<MODE, TM, TN><<<dim3(nbl(ncols, TN), nbl(M, TM)), 256, 0, c->stream>>>(Ah, Al, M, K, Uh, Ul, Wh, \
                                                                                     Wl, d1, d2, P, ncols, out)
  if (mode == 0) {
    if (choice == 0) PINT_DF_LAUNCH(0, 64, 64);
    else if (choice == 1) PINT_DF_LAUNCH(0, 32, 128);
    else PINT_DF_LAUNCH(0, 32, 32);
  } else {
    if (choice == 0) PINT_DF_LAUNCH(1, 64, 64);
    else if (choice == 1) PINT_DF_LAUNCH(1, 32, 128);
    else PINT_DF_LAUNCH(1, 32, 32);
  }
#undef PINT_DF_LAUNCH
  PINT_LAUNCH_CHECK();
  c->launches++;
}

void mx_gemm_df_nt(Ctx* c, const double* A, const double* B, int m, int n, int K, double* C) {
  if (m <= 0 || n <= 0) return;
  const dim3 grid(nbl(n, 32), nbl(m, 32));
  k_gemm_df_nt<32><<<grid, 256, 0, c->stream>>>(A, B, m, n, K, C);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

void mx_to_f32(Ctx* c, const double* x, long long n, float* y) {
  k_to_f32<<<nbl(n, 256), 256, 0, c->stream>>>(x, n, y);
  PINT_LAUNCH_CHECK();
}

}  // namespace pint
