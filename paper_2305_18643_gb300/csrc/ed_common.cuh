// Internal declarations shared by the libed translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "ed.h"

namespace ed {

constexpr int kMaxOrb = 32;      // one 32-bit word per spin
constexpr int kMaxVals = 128;    // distinct off-diagonal h values (7-bit index in a table entry)
constexpr int kMaxHops = 256;    // hops per basis state: N (L - N) <= 16 * 16
constexpr int kMaxPairs = kMaxOrb * (kMaxOrb - 1);

// Packed hopping-table entry: source label << 8 | fermion-sign bit << 7 | value index.
__host__ __device__ inline uint32_t ent_col(uint32_t e) { return e >> 8; }
__host__ __device__ inline uint32_t ent_neg(uint32_t e) { return (e >> 7) & 1u; }
__host__ __device__ inline uint32_t ent_vidx(uint32_t e) { return e & 127u; }
// Entry of the row kernel's slot-major table: (col << 14) | (((vidx << 1) | neg) << 2), so that
// e >> 10 is the byte offset of the column's 16-byte group in shared memory and e & 0x3FC that
// of its signed value in a table of 4-byte values (signed values of one index side by side, so
// the few distinct values of a warp's loads fall in distinct banks).  col < 2^18.
__host__ __device__ inline uint32_t row_ell_pack(uint32_t e) {
  return (ent_col(e) << 14) | (((ent_vidx(e) << 1) | ent_neg(e)) << 2);
}
// Slots of zeros after the last slot of the row kernel's table, so that it may load ahead
// without bounds checks.
constexpr int kEllPad = 8;

struct Error : public std::runtime_error {
  ed_status code;
  Error(ed_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string& msg);
[[noreturn]] void throw_cuda(cudaError_t e, const char* what, const char* file, int line);

#define ED_CUDA(call)                                                  \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) ::ed::throw_cuda(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define ED_CHECK_LAUNCH() ED_CUDA(cudaGetLastError())

// Kernel families timed by the profiler (ed_profile_* in ed.h).
enum KernelId {
  K_TABLES = 0, K_HPSI, K_LANCZOS_STEP, K_LANCZOS_NEXT, K_TRIDIAG, K_VECTOR, K_APPLY_COP, K_GF_EVAL,
  K_BAND, K_BATCH, K_LATTICE, K_COUNT
};
const char* kernel_name(int kid);
void note_launch();  // counts a launch that is timed inside another kernel's scope

// Leading dimension of the library's internal state vectors: rows padded to 128 elements so
// that every vectorized access of the two-pass H.psi stays inside its row.
inline int64_t padded_ld(int64_t d_dn) { return (d_dn + 127) / 128 * 128; }

// Counts every launch of the library; when profiling is on, brackets the launch with CUDA
// events on the launching stream and records the algorithmic bytes it moves.
struct ProfScope {
  int kid;
  cudaStream_t s;
  double bytes;
  cudaEvent_t e0 = nullptr;
  ProfScope(int kid_, cudaStream_t s_, double bytes_);
  ~ProfScope();
};

// Stream on which DevBuf allocates and frees in this thread (stream-ordered: cudaMallocAsync /
// cudaFreeAsync), or nullptr for cudaMalloc / cudaFree.  cudaFree waits for the whole device, so
// code that shares the GPU with other streams of the same process (the server's lanes) sets it to
// the one stream its buffers are used on.
extern thread_local cudaStream_t g_alloc_stream;
struct AllocStreamScope {
  cudaStream_t prev;
  explicit AllocStreamScope(cudaStream_t s) : prev(g_alloc_stream) { g_alloc_stream = s; }
  ~AllocStreamScope() { g_alloc_stream = prev; }
  AllocStreamScope(const AllocStreamScope&) = delete;
  AllocStreamScope& operator=(const AllocStreamScope&) = delete;
};

// Page-locked host scratch of this thread (kPinnedSlots doubles, allocated on first use and kept
// for the thread's life), the landing place of small device-to-host reads.  Slots: [0, 16) ground
// state, 16 continued fractions, 17 band Lanczos.
constexpr int kPinnedSlots = 32;
double* pinned_scratch();

// Allows kernel fn the largest dynamic shared memory of the current device (its opt-in limit less
// the kernel's static shared memory).  Every caller sets the same value, so threads that launch
// the kernel with different sizes at the same time (the server's lanes) cannot undo each other's
// setting between setting it and launching.
template <typename K>
inline void allow_max_dynamic_smem(K* fn) {
  int dev = 0, optin = 0;
  ED_CUDA(cudaGetDevice(&dev));
  ED_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  ED_CUDA(cudaFuncGetAttributes(&fa, (const void*)fn));
  ED_CUDA(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)fa.sharedSizeBytes));
}

// Device buffer with RAII ownership (cudaMalloc / cudaFree, or the stream-ordered pair when
// g_alloc_stream is set at allocation; the buffer is then freed on that stream).
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;  // stream of a stream-ordered allocation
  DevBuf() = default;
  explicit DevBuf(size_t count) { alloc(count); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; o.s = nullptr; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; o.s = nullptr; }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t count) {
    release();
    if (count == 0) return;
    cudaStream_t as = g_alloc_stream;
    cudaError_t e = as ? cudaMallocAsync((void**)&p, count * sizeof(T), as) : cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      throw Error(ED_ERR_OOM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    n = count;
    s = as;
  }
  void release() {
    if (p) {
      if (s)
        cudaFreeAsync(p, s);
      else
        cudaFree(p);
    }
    p = nullptr;
    n = 0;
    s = nullptr;
  }
};

// Host-side model after validation: one-body matrix h over L orbitals and per-orbital U.
struct ModelHost {
  int ns = 0, nb = 0, L = 0;
  std::vector<double> h;        // L x L
  std::vector<double> U;        // L (0 on bath)
  std::vector<double> vals;     // distinct off-diagonal h values
  std::vector<int> pair_a, pair_b, pair_vidx;  // ordered pairs with h[a][b] != 0, a != b
};

// Parameters passed to kernels by value.
struct HopParams {
  double val[kMaxVals];
  float valf[kMaxVals];
  double U[kMaxOrb];
  float Uf[kMaxOrb];
  uint32_t umask;   // orbitals with U != 0
  int nvals;
  int uniform_u;    // 1: every orbital of umask has the same U (u0), so sum_i U_i n_i n_i = u0 popc(...)
  double u0;
  float u0f;
};

// One spin's sector with N particles: basis, two-level rank tables, hopping table, diagonal.
struct SpinTables {
  int L = 0, N = 0, split = 0;
  int64_t dim = 0, nnz = 0;
  DevBuf<uint32_t> basis;      // [dim] bit strings, ascending
  DevBuf<int32_t> rank_lo;     // [2^split]       rank(b) = rank_lo[b & lomask] + rank_hi[b >> split]
  DevBuf<int32_t> rank_hi;     // [2^(L-split)]
  DevBuf<int32_t> ptr;         // [dim + 1]
  DevBuf<uint32_t> ent;        // [nnz]
  int zmax = 0;                // longest row of the table
  DevBuf<uint32_t> ell;        // [zmax][dim] slot-major copy: ell[k * dim + r] = k-th entry of row r
  DevBuf<double> ediag;        // [dim] sum_a h_aa n_a
  DevBuf<float> ediag32;       // [dim]
};

// Read-only device view of a two-spin sector for the H.psi kernels.
struct SectorView {
  int64_t d_up, d_dn, ld;
  const uint32_t* B_up;
  const uint32_t* B_dn;
  const int32_t* ptr_up;
  const uint32_t* ent_up;
  const int32_t* ptr_dn;
  const uint32_t* ent_dn;
  const uint32_t* ell_dn;   // slot-major down-spin table (coalesced across a warp's columns)
  const double* e_up;
  const double* e_dn;
  const float* e_up32;
  const float* e_dn32;
  int64_t two_pass_min_bytes;  // vectors of at least this many bytes take the two-pass H.psi
};

// Preset maximum of a continued fraction of the batched and served forms when the caller gives
// none: high enough that runs stop on convergence on the grid (a 10-orbital sector of ~2.5e4
// states needs about 3,000 levels for 1e-8 on the real axis at eta = 0.05).
constexpr int kCfDefaultMaxLevels = 20000;

// Default of ED_OPT_TWO_PASS_MIN_BYTES: a vector of 32 MiB no longer sits comfortably in L2.
constexpr int64_t kTwoPassMinBytes = int64_t(32) << 20;

struct RankView {
  const int32_t* lo;
  const int32_t* hi;
  int split;
  uint32_t lomask;
};

// Visits every logical element (u, d) of a d_up x d_dn array, f(u, d, u * d_dn + d), without
// 64-bit division: rows over blocks and columns over threads when rows are long, else a flat
// 32-bit index (d_dn < 64 keeps d_up * d_dn < 2^30).
template <typename F>
__device__ __forceinline__ void for_each_element(int64_t du, int64_t dd, F&& f) {
  if (dd >= 64) {
    for (int64_t u = blockIdx.x; u < du; u += gridDim.x)
      for (int64_t d = threadIdx.x; d < dd; d += blockDim.x) f(u, d, u * dd + d);
  } else {
    const uint32_t n = (uint32_t)(du * dd), ddu = (uint32_t)dd;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const uint32_t u = i / ddu;
      f((int64_t)u, (int64_t)(i - u * ddu), (int64_t)i);
    }
  }
}

__device__ __forceinline__ int32_t rank_of(const RankView& r, uint32_t b) {
  return r.lo[b & r.lomask] + r.hi[b >> r.split];
}

// sector.cu
std::unique_ptr<SpinTables> build_spin_tables(const ModelHost& m, int N, cudaStream_t s);
void build_model(const ed_cluster_desc* desc, ModelHost& m, HopParams& hp);  // api.cu
void basis_to_host(int L, int N, uint32_t* out, int64_t dim);
uint64_t binomial(int n, int k);

// hpsi.cu : y = H x (optionally fused Lanczos epilogue), batched over runs via blockIdx.z.
struct LanczosScalars {
  double* alpha;      // [runs][mstride]
  double* beta;       // [runs][mstride + 1], beta[r][n] = b_n (norm); beta[r][0] = 0
  double* beta0;      // [runs] initial norm b_0 (of the unnormalized start vector)
  int* active;        // [runs] 1 while the run continues
  double* partial;    // [runs][nblk][3] block partial sums
  unsigned* counter;  // [runs] blocks finished (reset by the last block)
  int mstride;
  double btol;        // run stops when b_{n+1} < btol * b_0
  int* nsteps;        // [runs] levels completed (alpha_0 .. alpha_{nsteps-1}); may be NULL
};

void launch_hpsi(const SectorView& sv, const HopParams& hp, int dtype, const void* x, void* y,
                 cudaStream_t s);
// y_r = H x_r for `runs` vectors vstride elements apart (one launch pair of the two-pass kernels
// for all of them when they apply, else one product per vector).
void launch_hpsi_block(const SectorView& sv, const HopParams& hp, int dtype, const void* X, void* Y, int64_t vstride,
                       int runs, cudaStream_t s);
// One fused Lanczos step for `runs` vectors stored at X + r * vstride (and XP likewise):
// W = H X - b_n XP written over XP; per-run reductions finish alpha_n, b_{n+1}.
void launch_lanczos_step(const SectorView& sv, const HopParams& hp, int dtype, const void* X,
                         void* XP, int64_t vstride, int runs, int n, const LanczosScalars& ls,
                         int nblk_cap, cudaStream_t s);
int lanczos_blocks(const SectorView& sv);   // partial-sum slots per run of the fused step
int two_pass_blocks(const SectorView& sv, int dtype);

// lanczos.cu
// omega (contiguous) += coef[n + 1] v_{n+1}; its type is omega_dtype (< 0: the vectors' dtype).
void launch_lanczos_next(int dtype, void* W, const void* X, int64_t d_up, int64_t d_dn, int64_t ld,
                         int64_t vstride, int runs, int n, const LanczosScalars& ls,
                         void* omega, const double* coef, cudaStream_t s, int omega_dtype = -1);
void launch_start_vector(int dtype, void* v, int64_t d_up, int64_t d_dn, int64_t ld, uint64_t seed,
                         cudaStream_t s);
// Reductions into a device double: out = <a, b> over d_up x d_dn (two-stage, fixed order).
void launch_dot(int dtype_a, const void* a, int dtype_b, const void* b, int64_t d_up, int64_t d_dn,
                int64_t ld, double* partial, int nblk, double* out, cudaStream_t s);
// y = ca * a + cb * b (elementwise, any dtype combination via conversion); scalars on device
void launch_axpby(int dtype_y, void* y, int dtype_a, const void* a, const double* ca, int dtype_b,
                  const void* b, const double* cb, int64_t d_up, int64_t d_dn, int64_t ld,
                  cudaStream_t s);
// y[u][d] (leading dimension ld_y) = scale * a[u][d] (leading dimension ld_a); scale NULL = 1.
void launch_copy_ld(int dty, void* y, int64_t ld_y, int dta, const void* a, int64_t ld_a, const double* scale,
                    int64_t d_up, int64_t d_dn, cudaStream_t s);
void launch_tridiag_lowest(const double* alpha, const double* beta, int n, double* out_eval,
                           double* out_vec, cudaStream_t s);

struct GroundResult {
  double E0 = 0, residual = 0, gap = 0;
  int iters = 0;
  bool converged = false, degenerate = false;
};

// Several low states of a sector (davidson.cu): energies ascending, relative residuals.
struct LowStatesResult {
  std::vector<double> E, residual;
  int iters = 0;
  bool converged = false;
};

}  // namespace ed

// The opaque cluster handle.
struct ed_cluster {
  ed::ModelHost model;
  ed::HopParams hp;
  ed_cluster_desc desc;  // array pointers inside are cleared
  cudaStream_t stream = nullptr;
  bool owns_stream = true;     // false: the stream belongs to the caller (a server lane)
  int device = 0;
  std::map<int, std::unique_ptr<ed::SpinTables>> spins;  // by particle number
  // ground state (FP64, contiguous d_up x d_dn)
  ed::DevBuf<double> omega;
  bool have_gs = false;
  ed::GroundResult gs;
  int64_t gf_total_steps = 0;
  int band_max_dim = 0;        // Krylov vectors per part of the band Green function (0: default)
  int cf_max_steps = 0;        // steps per continued fraction (0: default)
  double gf_tol = 0.0;         // |Delta G| between convergence checks (0: default)
  bool gf_converged = true;
  size_t gf_mem_budget = 0;    // bytes for Green-function Lanczos vectors (0: default)
  int gf_max_steps = 0;
  int64_t two_pass_min_bytes = ed::kTwoPassMinBytes;  // ED_OPT_TWO_PASS_MIN_BYTES
  int davidson_states = 1;     // ED_OPT_DAVIDSON_STATES: > 1 selects the Davidson method
  bool tensor_gram = true;     // ED_OPT_TENSOR_GRAM: FP32 band Grams on the tensor cores
  double temperature = 0.0;    // ED_OPT_TEMPERATURE of the mixed state
  ed::DevBuf<double> low;      // the low states (FP64, contiguous d_up x d_dn each) of a Davidson run
  std::vector<double> low_E;   // their energies
  ed::SpinTables& tables(int N);
  ed::SectorView view(int n_up, int n_dn, int64_t ld);
};

namespace ed {
std::unique_ptr<ed_cluster> cluster_create_on(const ed_cluster_desc* desc, cudaStream_t stream);
}  // namespace ed
