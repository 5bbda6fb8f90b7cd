// WR contractions on the 5th-generation tensor cores (tcgen05, kind::tf32).
//
// The two contractions of one WR iteration (Section 4.2; a2 and a6 of the
// hot path) are out[col][i] = sum_k T(k, col) C(i, k), where col = (interval,
// step) runs over the N P trajectory columns, i over the modes of the output
// space and C is the coupling operator ([-(CA + CM/dt) | CM/dt] or
// [-CM^T | -dt CA^T], rows padded to K = 2 ld).  T(k, col) is gathered from the
// FP32 trajectories with the step shifts of eqs. (4.8)-(4.9):
//   MODE 0: T = [w_p ; w_{max(p-1,0)}]      MODE 1: T = [u_p - u_{max(p-1,0)} ; u_{p+1}]
//
// One CTA computes a 128-column x BN-mode tile: MMA M = 128 trajectory
// columns (A operand, built in shared memory by all threads), N = BN modes (B
// operand = coupling rows), accumulator in TMEM (128 lanes x BN FP32
// columns), so that each thread's TMEM row is a contiguous run of output
// modes.  FP32 accuracy from TF32 operands: x = hi + lo with hi = tf32(x),
// lo = tf32(x - hi), three MMAs per K step (hi hi + hi lo + lo hi).
// Shared memory holds two K-blocks of 32 in the canonical K-major layout
// without swizzle: 8-row x 16-byte core matrices, the 8 K-chunks of a row
// group contiguous (leading byte offset 128 B), row groups 1024 B apart
// (stride byte offset).  One thread issues the MMAs and commits them to the
// stage's mbarrier; waits are bounded and set an error flag on expiry.
#include "common.cuh"

namespace pint {

namespace {

constexpr int UM = 128;   // MMA M (trajectory columns per CTA)
constexpr int KB = 32;    // K elements per stage
constexpr int THREADS = 256;
constexpr int WAIT_LIMIT = 1 << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version; base offset 0, no swizzle
  return d;
}

// instruction descriptor: D F32, A/B TF32, both K-major, N, M
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (int i = 0; i < WAIT_LIMIT; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return __uint_as_float(h);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of (row, k) in the canonical no-swizzle K-major tile (KB = 32)
__device__ __forceinline__ uint32_t tile_off(int row, int chunk) {
  return (uint32_t)((row >> 3) * 1024 + chunk * 128 + (row & 7) * 16);
}

template <int MODE, int BN>
__global__ void __launch_bounds__(THREADS) k_wr_umma(const float* __restrict__ Chi, const float* __restrict__ Clo,
                                                     int M, int Kp, const float* __restrict__ Ut,
                                                     const float* __restrict__ Wt, int ldu, int ldw, int P,
                                                     int ncols, float* __restrict__ out, int* __restrict__ err) {
  constexpr int A_BYTES = UM * KB * 4;   // 16 KB
  constexpr int B_BYTES = BN * KB * 4;
  constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  constexpr int TCOLS = (BN <= 32) ? 32 : (BN <= 64) ? 64 : (BN <= 128) ? 128 : 256;
  constexpr uint32_t IDESC = idesc_tf32(UM, BN);
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;

  const int col0 = blockIdx.x * UM;
  const int row0 = blockIdx.y * BN;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const int nkb = Kp / KB;
  const int ld = (MODE == 0) ? ldw : ldu;

  int last = -1;  // index of the last committed K-block (uniform)
  for (int kb = 0; kb < nkb; ++kb) {
    const int s = kb & 1;
    uint8_t* base = smem + s * STAGE;
    if (kb >= 2) {
      // the MMAs of K-block kb-2 read this stage: the issuing thread waits for
      // their commit, the barrier publishes the outcome to every thread
      if (tid == 0 && !bar_wait(&bars[s], (uint32_t)(((kb - 2) >> 1) & 1))) s_fail = 1;
      __syncthreads();
      if (s_fail) break;
    }
    const int k0 = kb * KB;
    const int seg = k0 / ld, j0 = k0 - seg * ld;
    // A: trajectory columns, float4 per (column, 4-k chunk)
    for (int idx = tid; idx < UM * 8; idx += THREADS) {
      const int rlow = idx & 7, chunk = (idx >> 3) & 7, rg = idx >> 6;
      const int r = rg * 8 + rlow;
      const int col = col0 + r;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (col < ncols) {
        const int n = col / P, p = col - n * P;
        if (MODE == 0) {
          const int q = (seg == 0) ? p : (p >= 1 ? p - 1 : 0);
          v = *reinterpret_cast<const float4*>(Wt + ((size_t)n * (P + 1) + q) * ldw + j0 + 4 * chunk);
        } else if (seg == 0) {
          float4 a = *reinterpret_cast<const float4*>(Ut + ((size_t)n * (P + 1) + p) * ldu + j0 + 4 * chunk);
          float4 b = *reinterpret_cast<const float4*>(Ut + ((size_t)n * (P + 1) + (p >= 1 ? p - 1 : 0)) * ldu +
                                                      j0 + 4 * chunk);
          v = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
        } else {
          v = *reinterpret_cast<const float4*>(Ut + ((size_t)n * (P + 1) + p + 1) * ldu + j0 + 4 * chunk);
        }
      }
      float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
      float4 l = make_float4(tf32_rna(v.x - h.x), tf32_rna(v.y - h.y), tf32_rna(v.z - h.z), tf32_rna(v.w - h.w));
      const uint32_t o = tile_off(r, chunk);
      *reinterpret_cast<float4*>(base + o) = h;
      *reinterpret_cast<float4*>(base + A_BYTES + o) = l;
    }
    // B: coupling rows (already split), float4 per (row, chunk)
    for (int idx = tid; idx < BN * 8; idx += THREADS) {
      const int rlow = idx & 7, chunk = (idx >> 3) & 7, rg = idx >> 6;
      const int r = rg * 8 + rlow;
      const int row = row0 + r;
      float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
      if (row < M) {
        h = *reinterpret_cast<const float4*>(Chi + (size_t)row * Kp + k0 + 4 * chunk);
        l = *reinterpret_cast<const float4*>(Clo + (size_t)row * Kp + k0 + 4 * chunk);
      }
      const uint32_t o = tile_off(r, chunk);
      *reinterpret_cast<float4*>(base + 2 * A_BYTES + o) = h;
      *reinterpret_cast<float4*>(base + 2 * A_BYTES + B_BYTES + o) = l;
    }
    // make the generic-proxy stores visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = smem_u32(base), a_lo = a_hi + A_BYTES;
      const uint32_t b_hi = a_hi + 2 * A_BYTES, b_lo = b_hi + B_BYTES;
#pragma unroll
      for (int kk = 0; kk < KB / 8; ++kk) {
        const uint32_t ko = kk * 256;  // two 16-byte chunks per K = 8 step
        const uint64_t dah = umma_desc(a_hi + ko, 128, 1024), dal = umma_desc(a_lo + ko, 128, 1024);
        const uint64_t dbh = umma_desc(b_hi + ko, 128, 1024), dbl = umma_desc(b_lo + ko, 128, 1024);
        mma_tf32(tmem, dah, dbh, IDESC, (kb > 0 || kk > 0) ? 1u : 0u);
        mma_tf32(tmem, dah, dbl, IDESC, 1u);
        mma_tf32(tmem, dal, dbh, IDESC, 1u);
      }
      mma_commit(&bars[s]);
    }
    last = kb;
  }
  // the last commit covers every earlier MMA of the issuing thread
  if (tid == 0 && last >= 0 && !bar_wait(&bars[last & 1], (uint32_t)((last >> 1) & 1))) s_fail = 1;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: warp w reads TMEM lanes 32 (w % 4) ..; warps w and w + 4 split the columns
  if (!s_fail) {
    const int lane_base = 32 * (warp & 3);
    const int r = lane_base + (tid & 31);
    const int col = col0 + r;
    const int half = (BN / 16 + 1) / 2;  // 16-column chunks per warp half
    const int c_begin = (warp < 4) ? 0 : half;
    const int c_end = (warp < 4) ? half : BN / 16;
    for (int cc = c_begin; cc < c_end; ++cc) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(cc * 16), v);
      if (col < ncols) {
        float* o = out + (size_t)col * M + row0 + cc * 16;
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (row0 + cc * 16 + q < M) o[q] = v[q];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
  if (tid == 0 && s_fail) atomicExch(err, 1);
}

template <int MODE, int BN>
void launch(Ctx* c, const float* Chi, const float* Clo, int M, int Kp, const float* Ut, const float* Wt, int ldu,
            int ldw, int ncols, float* out, int* err) {
  constexpr int STAGE = 2 * UM * KB * 4 + 2 * BN * KB * 4;
  constexpr int SMEM = 2 * STAGE;
  static bool attr = false;
  if (!attr) {
    PINT_CUDA(cudaFuncSetAttribute(k_wr_umma<MODE, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
    attr = true;
  }
  dim3 grid((ncols + UM - 1) / UM, (M + BN - 1) / BN);
  k_wr_umma<MODE, BN><<<grid, THREADS, SMEM, c->stream>>>(Chi, Clo, M, Kp, Ut, Wt, ldu, ldw, c->P, ncols, out,
                                                          err);
  PINT_LAUNCH_CHECK();
  c->launches++;
}

}  // namespace

// MODE 0: M = d1 modes, Kp = 2 ldw; MODE 1: M = d2, Kp = 2 ldu.  Mode tile
// widths keep the grid near a multiple of the 152 SMs for N P = 4096 columns.
void mx_contract_umma(Ctx* c, int mode, const float* Chi, const float* Clo, int M, int Kp, const float* Ut,
                      const float* Wt, int ldu, int ldw, int ncols, float* out, int* err) {
  if (mode == 0)
    launch<0, 224>(c, Chi, Clo, M, Kp, Ut, Wt, ldu, ldw, ncols, out, err);
  else
    launch<1, 48>(c, Chi, Clo, M, Kp, Ut, Wt, ldu, ldw, ncols, out, err);
}

}  // namespace pint
