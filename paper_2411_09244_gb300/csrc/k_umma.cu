// WR contractions on the 5th-generation tensor cores (tcgen05, kind::tf32).
//
// The two contractions of one WR iteration (Section 4.2, eqs. (4.8)-(4.9))
// are out[col][i] = sum_k C(i, k) B(col, k): i runs over the modes of the
// output space, col = (interval, step) over the trajectory columns, C is the
// coupling operator in difference form ([-CA | -CM/dt] or [-CM^T | -dt CA^T],
// both K halves padded to ld with zeros) and B(col, :) the column map of the
// trajectories (written by the producing kernels of the iteration):
//   first contraction:  B = [w_p ; w_p - w_{max(p-1,0)}]
//   second contraction: B = [u_p - u_{max(p-1,0)} ; u_{p+1}].
// FP32 accuracy from TF32 operands: every operand is stored as a hi/lo pair
// (hi = tf32(x), lo = tf32(x - hi)) and each K step issues three MMAs
// (hi hi + hi lo + lo hi); the dropped lo lo term is below FP32 rounding.
//
// Persistent kernel, one CTA per SM: tiles of 128 modes x tn columns of one
// K slice (MMA M = 128 with A = coupling rows, N = tn in 128..256 with B =
// trajectory columns; tn and the K split chosen per shape by umma_plan) are
// dealt out round-robin.  Warp 0 (one lane) streams 16-wide K stages with TMA
// (64-byte swizzle) into a ring of STAGES buffers across tile
// boundaries; warp 1 allocates TMEM and one lane issues the MMAs into one of
// two accumulators (2 x 256 TMEM columns, lane = mode); warps 2-5 drain the
// other accumulator to global memory meanwhile (stores coalesced along the
// modes).  mbarriers: "full"/"empty" for the ring (TMA transaction count /
// tcgen05.commit), "tfull"/"tempty" for the accumulators (tcgen05.commit /
// 128 epilogue arrivals).  Every wait is bounded: on expiry the kernel records
// an error flag, stops issuing, waits (bounded) for the copies and MMAs it has
// in flight, frees its TMEM and returns.
#include "common.cuh"

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

namespace pint {

namespace {

constexpr int TM = 128;    // modes per tile (MMA M)
constexpr int TNMAX = 256; // trajectory columns per tile (MMA N, chosen per shape: 128..256)
constexpr int KB = 16;     // K elements per stage = one 64-byte swizzle row
constexpr int STAGES = 4;
constexpr int THREADS = 192;     // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int EPI_THREADS = 128;
constexpr int NACC = 2;          // TMEM accumulators
constexpr int WAIT_LIMIT = 1 << 22;
constexpr int OPA = TM * KB * 4;                     // one A operand tile (8 KB)
constexpr int OPBM = TNMAX * KB * 4;                 // room for one B operand tile (16 KB)
constexpr int STAGE_BYTES = 2 * OPA + 2 * OPBM;      // A hi, A lo, B hi, B lo
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;  // + slack for 1024-byte alignment

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: K-major, 64-byte swizzle (rows of 16 TF32),
// 8-row groups 512 bytes apart (stride byte offset), descriptor version 1
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;           // version
  d |= (uint64_t)4 << 61;           // layout: 64-byte swizzle
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
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
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

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// the same box into the same shared-memory offset of every CTA in cta_mask,
// each CTA's mbarrier at bar's offset receiving the bytes it got
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                               uint16_t cta_mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster "
      "[%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "h"(cta_mask)
      : "memory");
}

// arrive once on the mbarrier at bar's offset in every CTA of cta_mask when
// every MMA this thread issued before has completed
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t cta_mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(cta_mask)
      : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// tile tg -> (K slice z, row tile, column tile); column tiles fastest, so CTAs
// working at the same time share the coupling rows in L2
struct Tile {
  int z, row0, col0;
};
__device__ __forceinline__ Tile decode(int tg, int n_ct, int n_rt, int tn) {
  const int per = n_ct * n_rt, rem = tg % per;
  return {tg / per, (rem / n_ct) * TM, (rem % n_ct) * tn};
}

// out + z * ncols * M: the K slice [z kspan, (z + 1) kspan) of the product.
// CL = 2: clusters of two CTAs take row tiles 2 r and 2 r + 1 of the same
// column tile and K slice (a "pair tile"; the second may lie past M and then
// only loads zeros and stores nothing).  Each CTA loads its own A tile and
// half of the B tile, multicast into both CTAs, so a B tile is read from L2
// once per row pair instead of once per row tile; each CTA's MMA commit for
// a stage arrives on both CTAs' "empty" barrier, so neither CTA refills a
// stage (in both) before both have consumed it.
template <int CL>
__global__ void __launch_bounds__(THREADS, 1)
    k_wr_umma(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
              const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, int M, int ncols,
              int kspan, int nsplit, int tn, float* __restrict__ out, int* __restrict__ err,
              const int* __restrict__ gate) {
  const uint32_t IDESC = idesc_tf32(TM, tn);
  if (gate && *gate) return;  // the WR sweep has already converged: no-op launch (every CTA alike)
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], tfull[NACC], tempty[NACC], done;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_fail;
  // the 128-byte swizzle pattern repeats every 1024 bytes: align the ring to it
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);

  const int n_ct = (ncols + tn - 1) / tn, n_rt = (M + TM - 1) / TM;
  const uint32_t stage_tx = 2 * OPA + 2 * tn * KB * 4;  // bytes a stage lands in each CTA
  // CL = 1: tiles; CL = 2: pair tiles (row tiles in pairs), one per cluster
  const int rank = CL == 1 ? 0 : (int)cluster_rank();
  const int n_rg = (n_rt + CL - 1) / CL;  // row groups
  const int n_tiles = n_ct * n_rg * nsplit;
  const int unit = (int)blockIdx.x / CL, nunits = (int)gridDim.x / CL;
  const int my_tiles = unit < n_tiles ? (n_tiles - 1 - unit) / nunits + 1 : 0;
  auto tile_of = [&](int j) {
    Tile T = decode(unit + j * nunits, n_ct, n_rg, tn);
    T.row0 = T.row0 * CL + rank * TM;  // decode gave the row group times TM
    return T;
  };
  const int nkb = kspan / KB;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    s_fail = 0;
    for (int s = 0; s < STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[s])), "r"(CL));
    }
    for (int a = 0; a < NACC; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tfull[a])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tempty[a])), "r"(EPI_THREADS));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(NACC * TNMAX));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (CL > 1) cluster_sync_all();  // the peer's barriers exist before any multicast reaches them
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (continuous ring across tiles) ----------------
      int g = 0;
      bool stop = false;
      for (int j = 0; j < my_tiles && !stop; ++j) {
        const Tile T = tile_of(j);
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % STAGES, use = g / STAGES;
          if (s_fail || (use >= 1 && !bar_wait(&empty[s], (uint32_t)((use - 1) & 1)))) {
            s_fail = 1;
            stop = true;
            break;
          }
          uint8_t* base = smem + s * STAGE_BYTES;
          const int k0 = T.z * kspan + kb * KB;
          bar_expect_tx(&full[s], stage_tx);
          tma_load_2d(base, &mAh, &full[s], k0, T.row0);
          tma_load_2d(base + OPA, &mAl, &full[s], k0, T.row0);
          if (CL == 1) {
            tma_load_2d(base + 2 * OPA, &mBh, &full[s], k0, T.col0);
            tma_load_2d(base + 2 * OPA + OPBM, &mBl, &full[s], k0, T.col0);
          } else {  // this CTA's half of the B rows, into both CTAs
            const int half = tn / 2, off = rank * half * KB * 4;
            tma_load_2d_mc(base + 2 * OPA + off, &mBh, &full[s], k0, T.col0 + rank * half, 0x3);
            tma_load_2d_mc(base + 2 * OPA + OPBM + off, &mBl, &full[s], k0, T.col0 + rank * half, 0x3);
          }
        }
      }
      // copies still in flight must land before the CTA's shared memory goes
      for (int s = 0; s < STAGES && s < g; ++s) {
        const int last_use = (g - 1 - s) / STAGES;
        if (!bar_wait(&full[s], (uint32_t)(last_use & 1))) s_fail = 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int g = 0;
      bool stop = false;
      for (int j = 0; j < my_tiles && !stop; ++j) {
        const int acc = j & 1, u = j >> 1;
        if (s_fail || (u >= 1 && !bar_wait(&tempty[acc], (uint32_t)((u - 1) & 1)))) {
          s_fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(acc * TNMAX);
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % STAGES, use = g / STAGES;
          if (!bar_wait(&full[s], (uint32_t)(use & 1))) {
            s_fail = 1;
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
          for (int kk = 0; kk < KB / 8; ++kk) {
            const uint32_t ko = kk * 32;  // K = 8 TF32 = 32 bytes along the swizzle row
            const uint64_t dah = desc_sw64(base + ko), dal = desc_sw64(base + OPA + ko);
            const uint64_t dbh = desc_sw64(base + 2 * OPA + ko), dbl = desc_sw64(base + 2 * OPA + OPBM + ko);
            mma_tf32(d, dah, dbh, IDESC, (kb > 0 || kk > 0) ? 1u : 0u);
            mma_tf32(d, dah, dbl, IDESC, 1u);
            mma_tf32(d, dal, dbh, IDESC, 1u);
          }
          if (CL == 1) mma_commit(&empty[s]);
          else mma_commit_mc(&empty[s], 0x3);  // the stage is free in both CTAs once both have consumed it
        }
        if (!stop) mma_commit(&tfull[acc]);
      }
      mma_commit(&done);  // arrives once every MMA issued above has completed
    }
  } else {
    // ---------------- epilogue (warps 2-5, TMEM lane quadrant warp % 4) ----------------
    const int qd = warp & 3;
    for (int j = 0; j < my_tiles; ++j) {
      const int acc = j & 1, u = j >> 1;
      // one lane waits and the warp follows its verdict, so the warp stays
      // converged for the .sync.aligned TMEM loads
      int bad = 0;
      if (lane == 0) bad = (s_fail || !bar_wait(&tfull[acc], (uint32_t)(u & 1))) ? 1 : 0;
      bad = __shfl_sync(0xffffffffu, bad, 0);
      if (bad) {
        s_fail = 1;
        break;
      }
      bar_wait(&tfull[acc], (uint32_t)(u & 1));  // completed: returns at once; acquire for every lane
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const Tile T = tile_of(j);
      const int i = T.row0 + 32 * qd + lane;  // output mode of this thread (TMEM lane)
      float* o = out + (size_t)T.z * ncols * M;
      for (int cc = 0; cc < tn; cc += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(acc * TNMAX + cc), v);
        if (i < M) {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int col = T.col0 + cc + q;
            if (col < ncols) o[(size_t)col * M + i] = v[q];
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      bar_arrive(&tempty[acc]);
    }
  }
  __syncwarp();
  // every MMA has completed before the accumulators are freed
  if (!bar_wait(&done, 0u)) s_fail = 1;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // no multicast copy or commit of the peer may target this CTA after it exits
  if (CL > 1) cluster_sync_all();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NACC * TNMAX));
  if (tid == 0 && s_fail) atomicExch(err, 1);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::lock_guard<std::mutex> lock(lazy_init_mutex());
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    PINT_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    PINT_REQUIRE(p && q == cudaDriverEntryPointSuccess, PINT_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// row-major [rows][Kp] FP32 matrix, boxes of box_rows rows x 16 K with the
// 64-byte swizzle; rows past the end read as zero
CUtensorMap make_map(const float* base, int rows, int Kp, int box_rows) {
  CUtensorMap m;
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * 4};
  const cuuint32_t box[2] = {(cuuint32_t)KB, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  PINT_REQUIRE(((uintptr_t)base & 15) == 0 && Kp % KB == 0, PINT_ERR_BAD_ARG, "contraction operand misaligned");
  const CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides,
                                 box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  PINT_REQUIRE(r == CUDA_SUCCESS, PINT_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

}  // namespace

int umma_sms() {
  static int sms = 0;
  std::lock_guard<std::mutex> lock(lazy_init_mutex());
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// clusters of two contraction CTAs that can be resident at once (0: none)
static int umma_pair_clusters();

// Tile width and K split for one contraction shape, picked by a cost model of
// the persistent launch: every CTA runs its tiles back to back, so the time is
// set by the busiest SM, ceil(tiles / CTAs) tiles of (tn / s) column-K work
// each, plus the operand bytes each tile streams through L2 (1 / tn + 1 / 128
// per output; 1 / tn + 1 / 256 when a cluster pair shares its B tile, which
// costs a padded row tile when the row tiles are odd).  The model itself
// never pairs: on the 256x256 workload's shapes paired launches measured
// 48-53 us against 35.7 (d1 rows) and 72 against 38 (d2 rows), so pairing is
// left to the autotuner's measurement.  nsplit = 1 when the consumer cannot
// sum K slices.
static double umma_cost(int M, int ncols, int tn, int s, int pair, int sms) {
  const int n_rt = (M + TM - 1) / TM;
  const int slots = pair ? 2 * umma_pair_clusters() : sms;
  if (slots <= 0) return 1e300;
  const long long units = (long long)((ncols + tn - 1) / tn) * (pair ? (n_rt + 1) / 2 : n_rt) * s;
  const double rounds = (double)((units + slots / (pair ? 2 : 1) - 1) / (slots / (pair ? 2 : 1)));
  return rounds * (double)tn / s * (1.0 + 0.5 * (128.0 / tn + (pair ? 0.5 : 1.0)));
}

void umma_plan(int M, int Kp, int ncols, int maxs, int* tn_out, int* s_out, int* pair_out) {
  const int sms = umma_sms();
  double best = 1e300;
  *tn_out = 128;
  *s_out = 1;
  *pair_out = 0;
  for (int tn = 128; tn <= TNMAX; tn += 32)
    for (int s = 1; s <= maxs; ++s) {
      if (Kp % (KB * s)) continue;
      const double cost = umma_cost(M, ncols, tn, s, 0, sms);
      if (cost < best * 0.999) {
        best = cost;
        *tn_out = tn;
        *s_out = s;
      }
    }
}

// one-time setup of the contraction (kernel attributes, driver entry point,
// cluster occupancy): callers that capture the launches into a CUDA graph run
// it beforehand
static int g_pair_clusters = -1;
void umma_prepare() {
  {
    std::lock_guard<std::mutex> lock(lazy_init_mutex());
    if (g_pair_clusters < 0) {
      PINT_CUDA(cudaFuncSetAttribute(k_wr_umma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
      PINT_CUDA(cudaFuncSetAttribute(k_wr_umma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
      cudaLaunchConfig_t cfg{};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 2;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(2);
      cfg.blockDim = dim3(THREADS);
      cfg.dynamicSmemBytes = SMEM_BYTES;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nc = 0;
      if (cudaOccupancyMaxActiveClusters(&nc, k_wr_umma<2>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        nc = 0;
      }
      g_pair_clusters = nc;  // set last: a failed attempt is retried
    }
  }
  (void)encode_fn();
  (void)umma_sms();
}
static int umma_pair_clusters() {
  umma_prepare();
  return g_pair_clusters;
}

// out[z][col][i] = sum over the z-th K slice of A(i, k) B(col, k); A = Ahi + Alo
// ([M][Kp]), B = Bhi + Blo ([ncols][Kp]), TF32 pairs in FP32 containers, both
// 16-byte aligned with Kp a multiple of 32 nsplit.  pair: clusters of two
// CTAs share B tiles.  gate (device, may be null): the launch does nothing
// when *gate != 0.
void mx_contract_umma(Ctx* c, const float* Ahi, const float* Alo, int M, int Kp, const float* Bhi,
                      const float* Blo, int ncols, int nsplit, int tn, int pair, float* out, int* err,
                      const int* gate) {
  umma_prepare();
  PINT_REQUIRE(nsplit >= 1 && Kp % (KB * nsplit) == 0, PINT_ERR_BAD_ARG,
               "contraction K not divisible by the split");
  PINT_REQUIRE(tn >= 32 && tn <= TNMAX && tn % 32 == 0, PINT_ERR_BAD_ARG, "contraction tile width");
  PINT_REQUIRE(!pair || g_pair_clusters >= 1, PINT_ERR_BAD_ARG, "contraction: no room for clusters of two CTAs");
  if (ncols <= 0 || M <= 0) return;
  const int n_rt = (M + TM - 1) / TM, n_ct = (ncols + tn - 1) / tn;
  const CUtensorMap ah = make_map(Ahi, M, Kp, TM), al = make_map(Alo, M, Kp, TM);
  // a paired CTA loads half of each B tile
  const CUtensorMap bh = make_map(Bhi, ncols, Kp, pair ? tn / 2 : tn), bl = make_map(Blo, ncols, Kp, pair ? tn / 2 : tn);
  const int kspan = Kp / nsplit;
  if (!pair) {
    const int tiles = n_ct * n_rt * nsplit;
    const int grid = std::min(tiles, umma_sms());  // persistent: one CTA per SM at most
    k_wr_umma<1><<<grid, THREADS, SMEM_BYTES, c->stream>>>(ah, al, bh, bl, M, ncols, kspan, nsplit, tn, out, err,
                                                           gate);
  } else {
    const int units = n_ct * ((n_rt + 1) / 2) * nsplit;
    const int clusters = std::min(units, g_pair_clusters);  // persistent: every cluster resident
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = c->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    PINT_CUDA(cudaLaunchKernelEx(&cfg, k_wr_umma<2>, ah, al, bh, bl, M, ncols, kspan, nsplit, tn, out, err, gate));
  }
  PINT_LAUNCH_CHECK();
  c->launches++;
}

// ---------------------------------------------------------------------------
// Autotuner.  The cost model above ranks the (tile width, K split, row
// pairing) choices of a contraction shape; the autotuner times the
// best-ranked few on the live operands with CUDA events on the context's
// stream and keeps the fastest.  Choices live in one process-wide table keyed
// by (M, Kp, ncols, maxs), so a shape is timed once per process (or never,
// when the table was loaded).  Table rows: M, Kp, ncols, maxs, tn, s, pair.
// ---------------------------------------------------------------------------
namespace {
struct TuneVal {
  int tn, s, pair;
  float us;
};
std::mutex& tune_mutex() {
  static std::mutex m;
  return m;
}
std::map<std::array<int, 4>, TuneVal>& tune_table() {
  static std::map<std::array<int, 4>, TuneVal> t;
  return t;
}
constexpr int TUNE_CANDIDATES = 8;
constexpr int TUNE_REPS = 3;
constexpr int TUNE_COLS = 7;
}  // namespace

bool umma_valid_choice(int M, int Kp, int ncols, int maxs, int tn, int s, int pair) {
  return M > 0 && Kp > 0 && ncols > 0 && maxs >= 1 && tn >= 128 && tn <= TNMAX && tn % 32 == 0 && s >= 1 &&
         s <= maxs && Kp % (KB * s) == 0 && (pair == 0 || pair == 1);
}

void umma_choose(Ctx* c, bool tune, const float* Ahi, const float* Alo, int M, int Kp, const float* Bhi,
                 const float* Blo, int ncols, int maxs, float* out, int* err, int* tn_out, int* s_out,
                 int* pair_out) {
  umma_plan(M, Kp, ncols, maxs, tn_out, s_out, pair_out);
  if (ncols <= 0 || M <= 0) return;
  const std::array<int, 4> key{M, Kp, ncols, maxs};
  {
    std::lock_guard<std::mutex> lock(tune_mutex());
    auto it = tune_table().find(key);
    if (it != tune_table().end()) {  // a measured or loaded choice (usable here: pairing needs cluster room)
      if (!it->second.pair || umma_pair_clusters() >= 1) {
        *tn_out = it->second.tn;
        *s_out = it->second.s;
        *pair_out = it->second.pair;
      }
      return;
    }
  }
  if (!tune) return;
  // candidates ranked by the cost model (its own pick first), the best of
  // each pairing kept in the list
  const int sms = umma_sms();
  std::vector<std::pair<double, std::array<int, 3>>> cand[2];
  for (int pair = 0; pair <= (umma_pair_clusters() >= 1 ? 1 : 0); ++pair)
    for (int tn = 128; tn <= TNMAX; tn += 32)
      for (int s = 1; s <= maxs; ++s) {
        if (!umma_valid_choice(M, Kp, ncols, maxs, tn, s, pair)) continue;
        const bool own = tn == *tn_out && s == *s_out && pair == *pair_out;
        cand[pair].push_back({own ? -1.0 : umma_cost(M, ncols, tn, s, pair, sms), {tn, s, pair}});
      }
  std::vector<std::pair<double, std::array<int, 3>>> all;
  for (auto& v : cand) {
    std::sort(v.begin(), v.end());
    if ((int)v.size() > TUNE_CANDIDATES / 2) v.resize(TUNE_CANDIDATES / 2);
    all.insert(all.end(), v.begin(), v.end());
  }
  struct Ev {  // released on every exit, including a thrown failure
    cudaEvent_t e = nullptr;
    ~Ev() {
      if (e) cudaEventDestroy(e);
    }
  } e0, e1;
  PINT_CUDA(cudaEventCreate(&e0.e));
  PINT_CUDA(cudaEventCreate(&e1.e));
  float best = 3.4e38f;
  int btn = *tn_out, bs = *s_out, bp = *pair_out;
  for (auto& cd : all) {
    const int tn = cd.second[0], s = cd.second[1], pair = cd.second[2];
    mx_contract_umma(c, Ahi, Alo, M, Kp, Bhi, Blo, ncols, s, tn, pair, out, err, nullptr);  // warm-up
    PINT_CUDA(cudaEventRecord(e0.e, c->stream));
    for (int r = 0; r < TUNE_REPS; ++r)
      mx_contract_umma(c, Ahi, Alo, M, Kp, Bhi, Blo, ncols, s, tn, pair, out, err, nullptr);
    PINT_CUDA(cudaEventRecord(e1.e, c->stream));
    PINT_CUDA(cudaEventSynchronize(e1.e));
    float ms = 0.f;
    PINT_CUDA(cudaEventElapsedTime(&ms, e0.e, e1.e));
    const float us = 1e3f * ms / TUNE_REPS;
    if (us < best) {
      best = us;
      btn = tn;
      bs = s;
      bp = pair;
    }
  }
  *tn_out = btn;
  *s_out = bs;
  *pair_out = bp;
  std::lock_guard<std::mutex> lock(tune_mutex());
  tune_table()[key] = TuneVal{btn, bs, bp, best};
}

int umma_tuning_count() {
  std::lock_guard<std::mutex> lock(tune_mutex());
  return (int)tune_table().size();
}

int umma_tuning_get(int* rows, float* us, int cap) {
  std::lock_guard<std::mutex> lock(tune_mutex());
  int n = 0;
  for (auto& kv : tune_table()) {
    if (n >= cap) break;
    int* r = rows + TUNE_COLS * n;
    for (int j = 0; j < 4; ++j) r[j] = kv.first[j];
    r[4] = kv.second.tn;
    r[5] = kv.second.s;
    r[6] = kv.second.pair;
    if (us) us[n] = kv.second.us;
    ++n;
  }
  return n;
}

// returns the index of the first invalid row, or -1 when all were merged
int umma_tuning_set(const int* rows, const float* us, int count) {
  for (int i = 0; i < count; ++i) {
    const int* r = rows + TUNE_COLS * i;
    if (!umma_valid_choice(r[0], r[1], r[2], r[3], r[4], r[5], r[6])) return i;
  }
  std::lock_guard<std::mutex> lock(tune_mutex());
  for (int i = 0; i < count; ++i) {
    const int* r = rows + TUNE_COLS * i;
    tune_table()[{r[0], r[1], r[2], r[3]}] = TuneVal{r[4], r[5], r[6], us ? us[i] : 0.f};
  }
  return -1;
}

void umma_tuning_clear() {
  std::lock_guard<std::mutex> lock(tune_mutex());
  tune_table().clear();
}

}  // namespace pint
