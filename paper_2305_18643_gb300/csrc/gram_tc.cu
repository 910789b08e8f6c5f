// Gram of FP32 vector blocks on the fifth-generation tensor cores: the projections of the band
// Lanczos orthogonalization (Sec. 4.4), G_b[i][j] = sum_e X_{b,i}[e] Y_j[e] over the vectors'
// elements, a tall-skinny contraction (K = 1.5e8 elements at the 4x4 size, M <= 48, N = 16).
//
// A K-tile is 32 consecutive elements of every vector (one 128-byte row per vector, 128-byte
// swizzle).  Warp 0 loads the rows of the X blocks and of Y with TMA into a stage of shared memory
// (kTcStages stages in flight); warps 4-7 split every value into x = hi + lo with hi = x truncated
// to TF32 (exact in TF32) and lo = x - hi (13 significant bits), hi in place and lo beside it;
// warp 1 issues the MMAs D += A_hi B_hi + A_hi B_lo + A_lo B_hi (kind::tf32, M = 128 rows of which
// the vectors fill the first 16 nx + 16, N = 16 = the Y rows, K = 8 per instruction, 4 per
// K-tile), accumulating in TMEM; every kTcFlush K-tiles warps 4-7 read D (one row per thread) and
// add it to FP64 registers, while the MMAs continue in the second D buffer.  The three products
// carry ~2^-21 relative error each (lo loses <= 2 bits in TF32), FP32 accumulation runs over at
// most kTcFlush tiles, everything beyond is FP64.  CTAs take contiguous element chunks; their FP64
// partials are added in CTA order by the last CTA (a ticket), so results are deterministic.
//
// Every mbarrier wait gives up after kTcSpin polls: the kernel then sets *err, lets the other roles
// leave their loops, waits (bounded) for its TMA loads and MMAs in flight, frees its TMEM and
// returns; the host turns *err into ED_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "ed_common.cuh"

namespace ed {

constexpr int kTcRows = 128;    // MMA M: rows of the A tile (rows past the vectors stay zero)
constexpr int kTcN = 16;        // MMA N: the Y block
constexpr int kTcK = 32;        // elements per K-tile (a 128-byte row)
constexpr int kTcStages = 4;
constexpr int kTcFlush = 16;    // K-tiles accumulated in one TMEM buffer before a flush
constexpr int kTcThreads = 256; // warp 0 TMA, warp 1 MMA + TMEM allocation, warps 4-7 split + flush
constexpr int kTcTmemCols = 64; // two D buffers of 16 columns (the allocation unit is 32 columns)
constexpr long long kTcSpin = 1ll << 27;
constexpr int kTcTile = kTcRows * 128;  // bytes of one operand tile

struct TcShared {
  uint8_t hi[kTcStages][kTcTile];
  uint8_t lo[kTcStages][kTcTile];
  unsigned long long full[kTcStages], conv[kTcStages], empty[kTcStages];
  unsigned long long dfull[2], dempty[2];
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mb_init(unsigned long long* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s32(b)) : "memory");
}
__device__ __forceinline__ void mb_expect(unsigned long long* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mb_try(unsigned long long* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(s32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity; false when it gave up (or another role did).
__device__ __forceinline__ bool mb_wait(unsigned long long* b, uint32_t parity, volatile int* abort) {
  for (long long i = 0; i < kTcSpin; ++i) {
    if (mb_try(b, parity)) return true;
    if ((i & 255) == 255 && *abort) return false;
  }
  return false;
}

__device__ __forceinline__ void tma_rows(void* dst, const CUtensorMap* map, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(s32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(s32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle: rows of 128 bytes,
// 8-row atoms 1024 bytes apart (stride byte offset), leading byte offset unused, version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major, N = 16, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
      ::"r"(d), "l"(a), "l"(b), "r"(kTcIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s32(bar)) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, double (&acc)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] += (double)__uint_as_float(r[i]);
}

// nx X blocks (maps mx0, mx1; rows 16 b of the A tile) and, unless sym, Y (map my; rows 16 nx);
// B = the Y rows (or X block 0 when sym).  Elements [blockIdx.x chunk, +chunk) of n.  P: per-CTA
// partials [gridDim.x][rows][16]; the last CTA writes G[r][j] (rows r of the A tile, FP64).
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap mx0, const __grid_constant__ CUtensorMap mx1,
              const __grid_constant__ CUtensorMap my, int nx, int sym, int64_t n, int64_t chunk,
              double* __restrict__ P, unsigned* __restrict__ ticket, double* __restrict__ G, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  TcShared& S = *reinterpret_cast<TcShared*>(tc_raw + ((1024 - (s32(tc_raw) & 1023)) & 1023));
  __shared__ bool s_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = 16 * nx + (sym ? 0 : 16);       // vector rows of the A tile
  const int boff = sym ? 0 : 16 * nx;              // first B row
  const int nload = nx + (sym ? 0 : 1);            // 16-row TMA boxes per stage
  const int64_t e0 = (int64_t)blockIdx.x * chunk;
  const int64_t e1 = e0 + chunk < n ? e0 + chunk : n;
  const int ntile = e0 < e1 ? (int)((e1 - e0 + kTcK - 1) / kTcK) : 0;
  const int ngroup = (ntile + kTcFlush - 1) / kTcFlush;
  volatile int* abort = &S.abort;

  // zero both tiles of every stage (rows past the vectors must read as zero), barriers, TMEM
  for (int i = threadIdx.x; i < kTcStages * 2 * kTcTile / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(&S.hi[0][0])[i] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mb_init(&S.full[s], 1);
      mb_init(&S.conv[s], 128);
      mb_init(&S.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mb_init(&S.dfull[b], 1);
      mb_init(&S.dempty[b], 128);
    }
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s32(&S.tmem)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeroed tiles, for the tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem;

  if (warp == 0) {
    // ---- producer: TMA rows of every K-tile
    if (lane == 0) {
      int issued = 0;
      for (int t = 0; t < ntile; ++t) {
        const int s = t % kTcStages;
        const uint32_t par = ((t / kTcStages) & 1) ^ 1;
        if (!mb_wait(&S.empty[s], par, abort)) {
          *abort = 1;
          atomicExch(err, 1);
          break;
        }
        mb_expect(&S.full[s], (uint32_t)(nload * 16 * 128));
        const int x = (int)(e0 + (int64_t)t * kTcK);
        tma_rows(&S.hi[s][0], &mx0, x, 0, &S.full[s]);
        if (nx > 1) tma_rows(&S.hi[s][16 * 128], &mx1, x, 0, &S.full[s]);
        if (!sym) tma_rows(&S.hi[s][boff * 128], &my, x, 0, &S.full[s]);
        ++issued;
      }
      // the loads in flight must land before the CTA's shared memory goes away
      for (int t = issued > kTcStages ? issued - kTcStages : 0; t < issued; ++t) {
        const int s = t % kTcStages;
        for (long long i = 0; i < kTcSpin && !mb_try(&S.full[s], (t / kTcStages) & 1); ++i) {
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      int committed_groups = 0;
      for (int t = 0; t < ntile; ++t) {
        const int s = t % kTcStages;
        const int g = t / kTcFlush, db = g & 1;
        if (t % kTcFlush == 0) {  // a new group starts: its D buffer must have been read
          if (!mb_wait(&S.dempty[db], ((g >> 1) & 1) ^ 1, abort)) {
            *abort = 1;
            atomicExch(err, 2);
            break;
          }
        }
        if (!mb_wait(&S.conv[s], (t / kTcStages) & 1, abort)) {
          *abort = 1;
          atomicExch(err, 3);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dcol = tmem + (uint32_t)(db * 32);
        const uint32_t ah = s32(&S.hi[s][0]), al = s32(&S.lo[s][0]);
        const uint32_t bh = ah + (uint32_t)(boff * 128), bl = al + (uint32_t)(boff * 128);
#pragma unroll
        for (int kk = 0; kk < kTcK / 8; ++kk) {
          const int first = (t % kTcFlush == 0 && kk == 0) ? 0 : 1;
          const uint32_t off = (uint32_t)(kk * 32);
          mma_tf32(dcol, sw128_desc(ah + off), sw128_desc(bh + off), first);
          mma_tf32(dcol, sw128_desc(ah + off), sw128_desc(bl + off), 1);
          mma_tf32(dcol, sw128_desc(al + off), sw128_desc(bh + off), 1);
        }
        mma_commit(&S.empty[s]);  // the stage is free once these MMAs have read it
        if (t % kTcFlush == kTcFlush - 1 || t + 1 == ntile) {
          mma_commit(&S.dfull[db]);
          ++committed_groups;
        }
      }
      // MMAs in flight must finish before TMEM and shared memory are released
      if (ntile > 0)
        for (long long i = 0; i < kTcSpin && !mb_try(&S.empty[(ntile - 1) % kTcStages], ((ntile - 1) / kTcStages) & 1); ++i) {
        }
      (void)committed_groups;
    }
  } else if (warp >= 4) {
    // ---- split x = hi + lo, and flush D to FP64 (warp 4 + q reads TMEM lanes 32 q .. 32 q + 31)
    const int tid = threadIdx.x - 128;
    const int q = warp - 4;
    double acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.0;
    bool ok = true;
    // every wait's outcome is made warp-uniform: tcgen05.ld below is a warp-collective instruction
    for (int t = 0; t < ntile && ok; ++t) {
      const int s = t % kTcStages;
      if (!__all_sync(0xffffffffu, mb_wait(&S.full[s], (t / kTcStages) & 1, abort))) {
        *abort = 1;
        atomicExch(err, 4);
        ok = false;
        break;
      }
      float* hi = reinterpret_cast<float*>(&S.hi[s][0]);
      float* lo = reinterpret_cast<float*>(&S.lo[s][0]);
      for (int i = tid; i < rows * kTcK; i += 128) {
        const float x = hi[i];
        const float h = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
        hi[i] = h;
        lo[i] = x - h;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mb_arrive(&S.conv[s]);
      if (t % kTcFlush == kTcFlush - 1 || t + 1 == ntile) {
        const int g = t / kTcFlush, db = g & 1;
        if (!__all_sync(0xffffffffu, mb_wait(&S.dfull[db], (g >> 1) & 1, abort))) {
          *abort = 1;
          atomicExch(err, 5);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(db * 32), acc);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mb_arrive(&S.dempty[db]);
      }
    }
    (void)ngroup;
    const int r = 32 * q + lane;
    if (r < rows) {
      double* Pc = P + ((int64_t)blockIdx.x * rows + r) * 16;
#pragma unroll
      for (int j = 0; j < 16; ++j) Pc[j] = acc[j];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
  }
  // the last CTA adds the partials in CTA order
  __threadfence();
  if (threadIdx.x == 0) {
    const unsigned tk = atomicAdd(ticket, 1u);
    s_last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int q = threadIdx.x; q < rows * 16; q += blockDim.x) {
    double v = 0.0;
    for (unsigned c = 0; c < gridDim.x; ++c) v += __ldcg(P + (int64_t)c * rows * 16 + q);
    G[q] = v;
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// ---------------------------------------------------------------- host side
namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
}  // namespace

static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    else
      cudaGetLastError();
  });
  return g_encode;
}

// rows vectors of n FP32 elements, vstride elements apart, as a 2-D tensor read in boxes of
// 32 elements x 16 rows with 128-byte swizzle (rows past `rows` read as zero).
static CUtensorMap rows_map(const float* base, int rows, int64_t vstride, int64_t n) {
  CUtensorMap m;
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)vstride * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kTcK, 16u};
  const cuuint32_t es[2] = {1u, 1u};
  const CUresult r = encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(ED_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

// The tensor-core Gram applies to FP32 blocks of at most 16 vectors, 16-byte aligned bases and
// strides, on a device of compute capability 10.x with the tensor-map encoder available.
bool gram_tc_usable(const void* X0, const void* X1, const void* Y, int px, int py, int64_t vstride, int64_t n) {
  static int cc = -1;
  if (cc < 0) {
    int dev = 0, major = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) {
      cudaGetLastError();
      major = 0;
    }
    cc = major;
  }
  if (cc != 10 || !encoder()) return false;
  if (px < 1 || px > 16 || py < 1 || py > 16) return false;
  if (n % kTcK != 0 || (vstride * 4) % 16 != 0) return false;
  return (((uintptr_t)X0 | (uintptr_t)X1 | (uintptr_t)Y) & 15) == 0;
}

// G[b][i][j] = sum_e X_b,i[e] Y_j[e] (b < nx, X_0 = X0, X_1 = X1), or X0^T X0 when sym; written
// in the [nx][px][py] layout of the band code's Gram.  err_dev: device int, set on a timeout.
void gram_tc_f32(const float* X0, const float* X1, int nx, int px, const float* Y, int py, bool sym, int64_t vstride,
                 int64_t n, DevBuf<double>& P, DevBuf<unsigned>& tk, DevBuf<double>& Gfull, double* G, int* err_dev,
                 cudaStream_t s);

__global__ void k_gram_tc_pack(const double* __restrict__ Gfull, int nx, int px, int py, double* __restrict__ G) {
  const int total = nx * px * py;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int b = t / (px * py), i = (t / py) % px, j = t % py;
    G[t] = Gfull[(16 * b + i) * 16 + j];
  }
}

void gram_tc_f32(const float* X0, const float* X1, int nx, int px, const float* Y, int py, bool sym, int64_t vstride,
                 int64_t n, DevBuf<double>& P, DevBuf<unsigned>& tk, DevBuf<double>& Gfull, double* G, int* err_dev,
                 cudaStream_t s) {
  const CUtensorMap m0 = rows_map(X0, px, vstride, n);
  const CUtensorMap m1 = rows_map(nx > 1 ? X1 : X0, px, vstride, n);
  const CUtensorMap my = rows_map(sym ? X0 : Y, sym ? px : py, vstride, n);
  int dev = 0, sms = 152;
  ED_CUDA(cudaGetDevice(&dev));
  ED_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t ntile = n / kTcK;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntile / 4, sms));
  const int64_t chunk = (ntile + grid - 1) / grid * kTcK;
  const int rows = 16 * nx + (sym ? 0 : 16);
  if (P.n < (size_t)grid * rows * 16) P.alloc((size_t)grid * rows * 16);
  if (Gfull.n < (size_t)rows * 16) Gfull.alloc((size_t)rows * 16);
  if (tk.n < 1) {
    tk.alloc(1);
    ED_CUDA(cudaMemsetAsync(tk.p, 0, sizeof(unsigned), s));
  }
  const size_t smem = sizeof(TcShared) + 1024;
  static std::once_flag attr_once;
  std::call_once(attr_once, [&] {
    ED_CUDA(cudaFuncSetAttribute((const void*)k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  });
  {
    ProfScope ps_(K_BAND, s, (double)(nx * px + (sym ? 0 : py)) * n * 4.0);
    k_gram_tc<<<grid, kTcThreads, smem, s>>>(m0, m1, my, nx, sym ? 1 : 0, n, chunk, P.p, tk.p, Gfull.p, err_dev);
    ED_CHECK_LAUNCH();
  }
  note_launch();
  k_gram_tc_pack<<<1, 256, 0, s>>>(Gfull.p, sym ? 1 : nx, px, sym ? px : py, G);
  ED_CHECK_LAUNCH();
}

void gram_f32_cuda(const float* X, int nb, int px, const float* Y, int py, int64_t vstride, int64_t n, double* G,
                   cudaStream_t s);

}  // namespace ed

using namespace ed;

extern "C" ed_status ed_gram_f32(const float* X, int nx, const float* Y, int ny, int64_t vstride, int64_t n, int method,
                                 double* G_out) {
  try {
    if (!X || !Y || !G_out) throw Error(ED_ERR_INVALID, "X, Y and G_out must not be NULL");
    if (ny < 1 || ny > 16 || nx < 1 || nx > 32 || (nx > 16 && nx % 2)) throw Error(ED_ERR_INVALID, "need 1 <= ny <= 16 and nx <= 16 or nx = 2 px <= 32");
    if (n < 1 || vstride < n) throw Error(ED_ERR_INVALID, "need n >= 1 and vstride >= n");
    if (method != 0 && method != 1) throw Error(ED_ERR_INVALID, "method must be 0 (CUDA cores) or 1 (tensor cores)");
    const int nb = nx > 16 ? 2 : 1, px = nx > 16 ? nx / 2 : nx;
    const bool sym = X == Y && nx == ny && nb == 1;
    cudaStream_t s = cudaStreamPerThread;
    DevBuf<double> G((size_t)nb * px * ny);
    if (method == 1) {
      const float* X1 = nb > 1 ? X + 16 * vstride : nullptr;
      if (nb > 1 && px != 16) throw Error(ED_ERR_INVALID, "two X blocks must hold 16 vectors each");
      if (!gram_tc_usable(X, nb > 1 ? X1 : X, Y, px, ny, vstride, n))
        throw Error(ED_ERR_INVALID, "the tensor-core Gram cannot take this layout (device, alignment or n % 32)");
      DevBuf<double> P, Gfull;
      DevBuf<unsigned> tk;
      DevBuf<int> err(1);
      ED_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
      gram_tc_f32(X, X1, nb, px, Y, ny, sym, vstride, n, P, tk, Gfull, G.p, err.p, s);
      int e = 0;
      ED_CUDA(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
      ED_CUDA(cudaStreamSynchronize(s));
      if (e) throw Error(ED_ERR_TIMEOUT, "a bounded wait of the tensor-core Gram gave up (role " + std::to_string(e) + ")");
    } else {
      gram_f32_cuda(X, nb, px, Y, ny, vstride, n, G.p, s);
    }
    ED_CUDA(cudaMemcpyAsync(G_out, G.p, G.n * sizeof(double), cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    return ED_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return ED_ERR_INVALID;
  }
}
