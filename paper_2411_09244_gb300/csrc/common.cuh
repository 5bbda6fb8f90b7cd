// Internal definitions shared by the CUDA translation units of libpint.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pint.h"

// Several contexts may be driven from several host threads at once (one
// instance per thread and stream); the process-wide lazy initialisations
// (device attributes, kernel attributes, driver entry points) take this lock.
inline std::mutex& lazy_init_mutex() {
  static std::mutex m;
  return m;
}

namespace pint {

// ---------------------------------------------------------------- errors --
void set_error(const std::string& msg);

struct Fail {
  pint_status code;
  std::string msg;
};

#define PINT_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      throw ::pint::Fail{e_ == cudaErrorMemoryAllocation ? PINT_ERR_OOM : PINT_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_)};        \
    }                                                                                \
  } while (0)

#define PINT_REQUIRE(cond, code, msg)                  \
  do {                                                 \
    if (!(cond)) throw ::pint::Fail{(code), (msg)};    \
  } while (0)

#define PINT_LAUNCH_CHECK() PINT_CUDA(cudaGetLastError())

// ------------------------------------------------------ device buffers --
// Owned device allocation; freed by the context (stream-ordered).
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
};

// per-window description of the oversampled region K_i^+
struct WinDesc {
  int X0, Y0;       // first interior node (x, y) of the window
  int wx, wy;       // interior nodes per side
  int nw;           // wx * wy
  int bx0, bx1, by0, by1;  // coarse blocks inside the window
  int m;            // constraints in the window (sum of aux functions)
  int t0;           // row of the target block's first constraint
  int kt;           // aux functions of the target block (= bases it owns)
  long long psi_off;     // offset of this window's bases in psi (kt * nw doubles)
  long long xpsi_off;    // offset of A/M/S Psi on the closure ((wx+2)(wy+2) per basis)
};

struct Ctx {
  cudaStream_t stream = nullptr;
  int device = 0;             // the device current at pint_setup_fine_grid
  std::vector<void*> allocs;  // everything freed in pint_destroy

  // fine grid (Section 2)
  int n_f = 0;
  int nn = 0;                 // (n_f+1)^2 nodes
  double* kappa = nullptr;    // n_f^2
  double* stA = nullptr;      // 9-point stencils of A_f, M_f and s (kappa_tilde mass)
  double* stM = nullptr;
  double* stS = nullptr;
  bool have_grid = false;

  // multiscale spaces (Section 3)
  int nc = 0, J = 0, ell = 0, bs = 0, nb = 0, n_blocks = 0;
  int kmax = 0;               // capacity of aux functions per block
  double* con_rows = nullptr; // [n_blocks][kmax][nb] constraint functionals
  double* con_gram = nullptr; // [n_blocks][kmax]
  std::vector<int> blk_k, blk_kind_off;  // aux functions per block, offset in raw list
  std::vector<int> kind;      // per raw basis: 0 matrix, 1 fracture, 2 enrichment
  std::vector<int> owner;     // owning block of each raw basis
  int n_raw = 0, L = 0;
  std::vector<WinDesc> win;   // one window per block
  double* psi = nullptr;      // bases on their window interiors
  long long psi_total = 0;
  int* d_windesc = nullptr;   // device copy of WinDesc fields (see k_galerkin)
  int* d_raw_win = nullptr;   // raw basis -> (window, column)
  bool have_spaces = false;

  // Galerkin (eq. (3.8)) on the raw bases and the split
  double* GM = nullptr;       // n_raw x n_raw
  double* GA = nullptr;
  double* GS = nullptr;
  std::vector<int> h1;        // raw index of each V_H1 basis
  std::vector<int> h2m;       // raw index of each matrix basis in V_H2 (after psi_bar)
  int d1 = 0, d2 = 0;
  bool has_bar = false;
  double* d_h1 = nullptr;     // int lists on the device (stored as int*)
  double* coef = nullptr;     // n_raw: s(psi_k, psi_bar)/s(psi_bar, psi_bar) (0 if not in V_H1)
  double* beta = nullptr;     // n_raw: psi_bar = Psi_all beta
  double *M11 = nullptr, *A11 = nullptr, *M22 = nullptr, *A22 = nullptr, *M12 = nullptr,
         *A12 = nullptr;
  bool have_reduced = false;

  // spectral bases and couplings
  double *Q = nullptr, *lam1 = nullptr, *Q2 = nullptr, *lam2 = nullptr;
  double *CM = nullptr, *CA = nullptr;    // Q^T M12 Q2, Q^T A12 Q2 (d1 x d2)
  double *CMt = nullptr, *CAt = nullptr;  // transposes (d2 x d1)
  double* projL = nullptr;                // Cholesky of I - CM^T CM (d2 x d2)
  double* projInv = nullptr;              // (I - CM^T CM)^-1
  double gamma = 0, lam22 = 0, dt_max = 0;

  // time grid
  int N = 0, P = 0, precision = PINT_FP64;
  double T = 0, Dt = 0, dt = 0, alpha = 0;
  bool fine_seq = false;  // PINT_FINE_SEQUENTIAL
  bool autotune = false;  // PINT_AUTOTUNE: measured contraction tiles
  bool coarse64 = false;  // PINT_COARSE_FP64: every coarse sweep of the mixed path in FP64
  bool coarse_grid = false;  // PINT_COARSE_GRID: the first solve's FP32 sweeps grid-wide, not on a cluster
  bool refine64 = false;  // PINT_REFINE_FP64: refinement residual contractions in FP64
  bool carry = false;     // PINT_CARRY_LAGS: lag-carrying variant (FP64, sequential fine steps)
  bool adj_response = false;  // PINT_ADJOINT_RESPONSE: amplitude gradient by <lambda_{n+1}, s>
  bool have_time = false;

  // hot-path operators (FP64): [-G1 | G2] and [-CM^T | -dt CA^T]
  double* AR = nullptr;       // d1 x 2 d2
  double* AS = nullptr;       // d2 x 2 d1
  double2* tw = nullptr;      // twiddles e^{-2 pi i k / P}, k < P
  double2* dshift = nullptr;  // d_k = (1 - beta w^k)/dt
  double* lampow = nullptr;   // beta^p, p = 0..P
  double* GW = nullptr;       // [Dt^2 CA^T D CA | -Dt CA^T D] (d2 x (d2 + d1)), D = (1 + Dt Lambda1)^-1:
                              // the w rows of the folded coarse step
  double* GCD = nullptr;      // CA^T D (d2 x d1)

  // mixed-path state lives in mixed.cu
  void* mixed = nullptr;
  void* adj = nullptr;  // adjoint buffers (k_adjoint.cu)
  // wall time of the setup stages, ms: blocks, windows, Galerkin, reduced,
  // spectral, time-grid operators
  double stage_ms[6] = {0, 0, 0, 0, 0, 0};

  // scratch for solves (grown on demand)
  std::vector<std::pair<void*, size_t>> scratch;
  int launches = 0;
  unsigned graph_epoch = 0;            // bumped whenever hot-path buffers are reallocated
  cudaStream_t cap_stream = nullptr;   // private stream for capturing CUDA graphs
};

void* dalloc(Ctx* c, size_t bytes);
void dfree(Ctx* c, void* p);
// staging of host-or-device input arrays
const double* stage_in(Ctx* c, const double* p, size_t n, std::vector<void*>& tmp);
bool is_device_ptr(const void* p);

// ------------------------------------------------------- stage entry points
void build_fine(Ctx* c, const double* kappa_dev);                  // k_fine.cu
void build_blocks(Ctx* c);                                          // k_blocks.cu
void build_windows(Ctx* c);                                         // k_cem.cu
void build_galerkin(Ctx* c);                                        // k_galerkin.cu
void build_reduced(Ctx* c);                                         // k_galerkin.cu
void build_spectral(Ctx* c);                                        // k_dense.cu
void apply_stencil(Ctx* c, const double* st, const double* x, double* y, int count);  // k_fine.cu
void raw_dot(Ctx* c, const double* vec_nodes, int count, double* out_raw);  // k_galerkin.cu
void to_reduced(Ctx* c, const double* raw, int count, double* v1, double* v2);  // k_galerkin.cu
void prolong_coeffs(Ctx* c, const double* u, const double* w, int count, double* out_nodes);
// the same in double-float arithmetic, with the bases as FP32 pairs (psih, psil)
void prolong_coeffs_df(Ctx* c, const double* u, const double* w, int count, double* out_nodes, const float* psih,
                       const float* psil);
void split_bases(Ctx* c, float* psih, float* psil);

// dense FP64 helpers (k_dense.cu); all matrices row-major on the device
void dense_cholesky(Ctx* c, double* A, int n);              // lower L in place (upper zeroed)
void dense_trsm_lower(Ctx* c, const double* L, double* X, int n, int ncols, bool trans);
void dense_gemm(Ctx* c, const double* A, const double* B, double* C, int m, int n, int k,
                bool ta, bool tb, double alpha, double beta);
void dense_sym_eig(Ctx* c, double* A, double* V, double* lam, int n);  // A destroyed
void dense_gen_eig(Ctx* c, const double* A, const double* B, int n, double* Q, double* lam);
void dense_transpose(Ctx* c, const double* A, int m, int n, double* B);

// hot path (k_hot64.cu)
struct Hot;                                  // solve workspace
void hot_prepare(Ctx* c);                    // operators for the time grid
void hot_release(Ctx* c);
void solve_fp64(Ctx* c, const double* u0_nodes, const double* f_nodes, const double* amp_dev,
                double eps, int k_max, double wr_tol, int wr_max, double* u_out_dev,
                double* coarse_out_dev, pint_stats* st, bool sequential);
void solve_mixed(Ctx* c, const double* u0_nodes, const double* f_nodes, const double* amp_dev, double eps,
                 int k_max, double wr_tol, int wr_max, double* u_out, double* coarse_out, pint_stats* st,
                 int n_refine);
void mixed_release(Ctx* c);
void solve_carry(Ctx* c, const double* u0_nodes, const double* f_nodes, const double* amp_dev, double eps,
                 int k_max, double* u_out, double* coarse_out, pint_stats* st, bool sequential);
void apply_G_dev(Ctx* c, const double* in, int count, const double* f_nodes, const double* amp_dev,
                 double* out);
void apply_F_dev(Ctx* c, const double* in, int count, const double* f_nodes, const double* amp_dev,
                 double wr_tol, int wr_max, double* out, int* iters);

// adjoint of the converged parareal map (k_adjoint.cu); obs and data on the device
void adjoint_solve(Ctx* c, const int* obs, int n_obs, const double* data, const double* u0_nodes,
                   const double* f_nodes, const double* amp_dev, double eps, int k_max, double wr_tol, int wr_max,
                   double* misfit_host, double* grad_u0, double* grad_amp);
void adjoint_release(Ctx* c);
// forward-state access for the adjoint (k_hot64.cu)
void hot_states(Ctx* c, double** Xu, double** Xw);
void unit_response(Ctx* c, double* su, double* sw);
void step_source(Ctx* c, double* cu, double* cw);
// polls of the coarse sweep's grid-barrier waits before they give up (k_hot64.cu)
int wait_limit();
void set_wait_limit(int spins);
int sweep_smem();
void set_sweep_smem(int bytes);

// FP32 coarse sweep on one thread-block cluster (k_gcluster.cu)
// WR stopping test fused into the last kernel of a WR iteration (k_mixed.cu):
// acc holds cnt squared update norms, u parts then w parts, P per interval
// (cleared again by the test); out gets (norm, non-finite flag); gate is set
// when norm <= tol; counter holds 3 + nact words (global max bits, flag,
// intervals done, then one block counter per interval), zero between launches.
struct WrStop {
  float* acc;
  int cnt;
  double tol;
  int* gate;
  double* out;
  unsigned* counter;
};

struct GcArgs {
  const float* CA;  // [d1][d2] FP32 coupling
  const double *lam1, *lam2, *b1, *b2, *amp;
  const float *Fu, *Fw, *Cu, *Cw;  // F ends, jumps (may be null), FP32
  double *Xu, *Xw;                 // states (in/out), FP64
  float *Gu, *Gw;                  // G outputs of the previous sweep (in/out), FP32
  int d1, d2, n_lo, n_hi, first;
  double Dt;
};
int gc_cluster_size(int d1, int d2);
// autotuner table of the tensor-core contractions (k_umma.cu)
int umma_tuning_count();
int umma_tuning_get(int* rows, float* us, int cap);
int umma_tuning_set(const int* rows, const float* us, int count);  // -1, or the first invalid row
void umma_tuning_clear();
void g_sweep_cluster(Ctx* c, const GcArgs& a, int CL);

}  // namespace pint

// ------------------------------------------------------ device helpers --
namespace pintd {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// Double-float arithmetic (a value is the unevaluated pair hi + lo of two
// FP32 numbers, ~48 bits).  df_fma adds (ah + al)(bh + bl) to the running
// pair (sh, sl): the product's high part is exact by the FMA form of Dekker's
// product (p = ah bh, e = fma(ah, bh, -p)), the cross terms join the error
// term, Knuth's TwoSum adds p to sh, and the errors are summed in sl.
__device__ __forceinline__ void df_fma(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float s = sh + p;
  const float bb = s - sh;
  const float err = (sh - (s - bb)) + (p - bb);
  sh = s;
  sl += err + e;
}
// (ah + al) - (bh + bl) as a renormalised pair (TwoSum, then Fast2Sum)
__device__ __forceinline__ void df_sub(float ah, float al, float bh, float bl, float& h, float& l) {
  const float s = ah - bh;
  const float bb = s - ah;
  float e = (ah - (s - bb)) + (-bh - bb);
  e += al - bl;
  h = s + e;
  l = e - (h - s);
}

__device__ __forceinline__ float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// block-wide sum; `sh` holds >= 32 doubles; every thread returns the total
__device__ inline double block_sum(double v, double* sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}
__device__ inline double block_max(double v, double* sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_max(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

// Q1 element matrices from the 1D linear element by tensor products:
// corner a = (ax, ay) in {0,1}^2, counter-clockwise 0:(0,0) 1:(1,0) 2:(1,1) 3:(0,1).
// stiffness = K1 (x) M1 + M1 (x) K1 with K1 = [[1,-1],[-1,1]] (h-free in 2D),
// mass / h^2 = M1 (x) M1 with M1 = [[1/3,1/6],[1/6,1/3]].
__device__ __forceinline__ int corner_x(int a) { return (a == 1 || a == 2) ? 1 : 0; }
__device__ __forceinline__ int corner_y(int a) { return (a >= 2) ? 1 : 0; }
__device__ __forceinline__ double k1d(int i, int j) { return i == j ? 1.0 : -1.0; }
__device__ __forceinline__ double m1d(int i, int j) { return i == j ? (1.0 / 3.0) : (1.0 / 6.0); }
__device__ __forceinline__ double q1_stiff(int a, int b) {
  int ax = corner_x(a), ay = corner_y(a), bx = corner_x(b), by = corner_y(b);
  return k1d(ax, bx) * m1d(ay, by) + m1d(ax, bx) * k1d(ay, by);
}
__device__ __forceinline__ double q1_mass(int a, int b) {
  return m1d(corner_x(a), corner_x(b)) * m1d(corner_y(a), corner_y(b));
}

}  // namespace pintd
