// Gram of FP32 vector blocks on the fifth-generation tensor cores: the projections of the band
// Lanczos orthogonalization (Sec. 4.4), G_b[i][j] = sum_e X_{b,i}[e] Y_j[e] over the vectors'
// elements, a tall-skinny contraction (K = 1.5e8 elements at the 4x4 size, at most 32 X rows and
// 16 Y rows).
//
// Layout of one pipeline stage: a 128-row tile of 128-byte rows (32 FP32 elements, 128-byte
// swizzle).  A K-tile is 32 consecutive elements of the R vector rows involved (R = 16 for W^T W,
// 32 for one X block and Y, 48 for two X blocks and Y); KT = 64 / R K-tiles are stacked in rows
// [0, 64) of the stage (one for R = 48), so a stage always carries ~8 KB of vector data.
// TMA loads them; an epilogue warp group splits every value x into a TF32 head h = rn(x) (in
// place) and a TF32 tail l = rn(x - h), written 64 rows further down (two groups of four warps
// take alternate stages, so one splits while the other reads TMEM).  One MMA per 8-element step then multiplies
// the whole tile (all heads and tails: M = 128) by the Y rows of every stacked K-tile, heads and
// tails (N = 128, 112 or 80 rows of the same tile), so a single kind::tf32 MMA yields the four
// products h h, h l, l h and l l of every (i, j) pair, each in its own TMEM cell: no accumulator
// mixes a product with one 2^11 times smaller.  Cross-K-tile cells are computed and ignored.
//
// Accuracy: x = h + l + r with |r| <= 2^-22 |x| (round-to-nearest, unbiased), products of TF32
// values are exact in FP32, and each TMEM cell accumulates the 4 MMAs of one stage only; every
// stage is then read (tcgen05.ld; four D buffers, so the MMAs of a stage never wait for the
// previous stage's read) and added to a Kahan-compensated FP32 sum (the head products)
// or a plain FP32 sum moved to FP64 every 64 stages (the tail products).  CTAs take contiguous
// element chunks; a CTA reduces its lanes in a fixed order, and the last CTA (a ticket) adds the
// per-CTA partials in CTA order, so results are deterministic.
//
// Every mbarrier wait gives up after ~2 s: the kernel then sets *err, lets the other roles leave
// their loops, waits (bounded) for its TMA loads and MMAs in flight, frees its TMEM and returns;
// the host turns *err into ED_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "ed_common.cuh"

namespace ed {

constexpr int kTcK = 32;         // elements per K-tile (a 128-byte row)
constexpr int kTcStages = 8;
constexpr int kTcThreads = 384;  // warp 0 TMA, warp 1 MMA + TMEM, warps 4-7 and 8-11: split + flush
constexpr int kTcDBuf = 4;       // D buffers of up to 128 columns (all of TMEM)
constexpr int kTcTmemCols = 512;
constexpr int kTcX2Every = 64;   // stages between moves of the tail sums to FP64
constexpr long long kTcWaitNs = 2000000000ll;
constexpr int kTcTile = 128 * 128;  // bytes of one stage

struct TcShared {
  uint8_t tile[kTcStages][kTcTile];
  double red[2][128][16];
  unsigned long long full[kTcStages], conv[kTcStages], empty[kTcStages];
  unsigned long long dfull[kTcDBuf], dempty[kTcDBuf];
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
__device__ __forceinline__ long long now_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase of the given parity; false when it gave up (or another role did).
__device__ __forceinline__ bool mb_wait(unsigned long long* b, uint32_t parity, volatile int* abort) {
  if (mb_try(b, parity)) return true;
  const long long t0 = now_ns();
  for (int i = 1;; ++i) {
    if (mb_try(b, parity)) return true;
    if ((i & 63) == 0) {
      if (*abort || now_ns() - t0 > kTcWaitNs) return false;
    }
  }
}
// Bounded wait used while leaving: no abort check (the role's own operations must land).
__device__ __forceinline__ void mb_drain(unsigned long long* b, uint32_t parity) {
  const long long t0 = now_ns();
  while (!mb_try(b, parity) && now_ns() - t0 < kTcWaitNs) {
  }
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
// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major, M = 128, N given.
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s32(bar)) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// R = vector rows of one K-tile: 16 (W^T W: X block 0 is also B), 32 (one X block, then Y),
// 48 (X blocks 0 and 1, then Y).  Elements [blockIdx.x * chunk, +chunk) of n.  P: per-CTA
// partials [gridDim.x][nout], nout = 16 * (X rows); the last CTA writes G[i][j] (FP64).
template <int R>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap mx0, const __grid_constant__ CUtensorMap mx1,
              const __grid_constant__ CUtensorMap my, int64_t n, int64_t chunk, double* __restrict__ P,
              unsigned* __restrict__ ticket, double* __restrict__ G, int* __restrict__ err) {
  constexpr int KT = R == 48 ? 1 : 64 / R;    // K-tiles stacked in one stage
  constexpr int NLOAD = R / 16;               // 16-row TMA boxes per K-tile
  constexpr int XROWS = R == 16 ? 16 : R - 16;  // rows whose Gram is wanted
  constexpr int YOFF = R == 16 ? 0 : R - 16;    // first Y row of a K-tile
  constexpr int N = R == 16 ? 128 : 128 - YOFF; // B rows: [YOFF, 128) of the stage
  constexpr uint32_t IDESC = tc_idesc(N);
  constexpr int NOUT = XROWS * 16;
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  TcShared& S = *reinterpret_cast<TcShared*>(tc_raw + ((1024 - (s32(tc_raw) & 1023)) & 1023));
  __shared__ bool s_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e0 = (int64_t)blockIdx.x * chunk;
  const int64_t e1 = e0 + chunk < n ? e0 + chunk : n;
  const int ntile = e0 < e1 ? (int)((e1 - e0 + kTcK - 1) / kTcK) : 0;
  const int nst = (ntile + KT - 1) / KT;
  volatile int* abort = &S.abort;

  // zero every stage once (rows never loaded must hold finite values), barriers, TMEM
  for (int i = threadIdx.x; i < kTcStages * kTcTile / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(&S.tile[0][0])[i] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mb_init(&S.full[s], 1);
      mb_init(&S.conv[s], 128);
      mb_init(&S.empty[s], 1);
    }
    for (int b = 0; b < kTcDBuf; ++b) {
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
    // ---- producer: TMA rows of every stage (KT K-tiles, NLOAD boxes each)
    if (lane == 0) {
      int issued = 0;
      for (int t = 0; t < nst; ++t) {
        const int s = t % kTcStages;
        if (!mb_wait(&S.empty[s], ((t / kTcStages) & 1) ^ 1, abort)) {
          *abort = 1;
          atomicExch(err, 1);
          break;
        }
        const int kv = ntile - t * KT < KT ? ntile - t * KT : KT;
        mb_expect(&S.full[s], (uint32_t)(kv * NLOAD * 16 * 128));
        for (int kt = 0; kt < kv; ++kt) {
          const int x = (int)(e0 + (int64_t)(t * KT + kt) * kTcK);
          uint8_t* dst = &S.tile[s][kt * R * 128];
          tma_rows(dst, &mx0, x, 0, &S.full[s]);
          if (NLOAD == 3) tma_rows(dst + 16 * 128, &mx1, x, 0, &S.full[s]);
          if (NLOAD >= 2) tma_rows(dst + (NLOAD - 1) * 16 * 128, &my, x, 0, &S.full[s]);
        }
        ++issued;
      }
      // the loads in flight must land before the CTA's shared memory goes away
      for (int t = issued > kTcStages ? issued - kTcStages : 0; t < issued; ++t)
        mb_drain(&S.full[t % kTcStages], (t / kTcStages) & 1);
    }
  } else if (warp == 1) {
    // ---- MMA issuer: D[db] = tile (128 rows) x tile rows [YOFF, 128)^T over the stage's 32 elements
    if (lane == 0) {
      int done = 0;
      for (int t = 0; t < nst; ++t) {
        const int s = t % kTcStages, db = t % kTcDBuf;
        if (!mb_wait(&S.dempty[db], ((t / kTcDBuf) & 1) ^ 1, abort)) {
          *abort = 1;
          atomicExch(err, 2);
          break;
        }
        if (!mb_wait(&S.conv[s], (t / kTcStages) & 1, abort)) {
          *abort = 1;
          atomicExch(err, 3);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a = s32(&S.tile[s][0]);
        const uint32_t b = a + (uint32_t)(YOFF * 128);
#pragma unroll
        for (int kk = 0; kk < kTcK / 8; ++kk)
          mma_tf32(tmem + (uint32_t)(db * 128), sw128_desc(a + 32 * kk), sw128_desc(b + 32 * kk), IDESC, kk);
        mma_commit(&S.empty[s]);  // the stage is free once these MMAs have read it
        mma_commit(&S.dfull[db]);
        ++done;
      }
      // MMAs in flight must finish before TMEM and shared memory are released
      if (done > 0) mb_drain(&S.empty[(done - 1) % kTcStages], ((done - 1) / kTcStages) & 1);
    }
  } else if (warp >= 4) {
    // ---- split x = h + l and read the accumulators.  Two groups of four warps take alternate
    // stages (group grp: stages grp, grp + 2, ...), so one group splits while the other waits on
    // TMEM; warp 4 + 4 grp + q reads TMEM lanes 32 q .. 32 q + 31.
    const int grp = (warp - 4) >> 2;
    const int q = warp & 3;
    const int tid = threadIdx.x - 128 - 128 * grp;
    const int r = 32 * q + lane;          // TMEM lane = tile row of this thread
    const int rl = r & 63;                // row within the head (or tail) half
    const int kt_me = rl / R;             // stacked K-tile of this row (>= KT: unused row)
    const int ra = (32 * q & 63) / R;     // first stacked K-tile this warp's lanes cover
    constexpr int NF4 = KT * R * 128 / 16 / 128;  // float4 groups of data rows per thread and stage
    float s_h[16], c_h[16], x_l[16];
    double x_d[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) s_h[j] = c_h[j] = x_l[j] = 0.f, x_d[j] = 0.0;
    bool ok = true;
    int nflush = 0;

    auto flush = [&](int u) -> bool {
      const int db = u % kTcDBuf;
      // every wait's outcome is made warp-uniform: tcgen05.ld is a warp-collective instruction
      if (!__all_sync(0xffffffffu, mb_wait(&S.dfull[db], (u / kTcDBuf) & 1, abort))) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(db * 128);
      float vh[16], vl[16];
      if constexpr (R == 16) {
        float ah[16], al[16], bh[16], bl[16];
        tmem_ld16(base + (uint32_t)(16 * ra), ah);
        tmem_ld16(base + (uint32_t)(64 + 16 * ra), al);
        tmem_ld16(base + (uint32_t)(16 * ra + 16), bh);
        tmem_ld16(base + (uint32_t)(64 + 16 * ra + 16), bl);
        tmem_wait_ld();
        const bool second = lane >= 16;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          vh[j] = second ? bh[j] : ah[j];
          vl[j] = second ? bl[j] : al[j];
        }
      } else {
        tmem_ld16(base + (uint32_t)(R * ra), vh);
        tmem_ld16(base + (uint32_t)(64 + R * ra), vl);
        tmem_wait_ld();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mb_arrive(&S.dempty[db]);
      if (kt_me < KT && u * KT + kt_me < ntile) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {  // Kahan-compensated head products, plain tail products
          const float y = vh[j] - c_h[j];
          const float t2 = s_h[j] + y;
          c_h[j] = (t2 - s_h[j]) - y;
          s_h[j] = t2;
          x_l[j] += vl[j];
        }
      }
      if (++nflush % kTcX2Every == 0) {
#pragma unroll
        for (int j = 0; j < 16; ++j) x_d[j] += (double)x_l[j], x_l[j] = 0.f;
      }
      return true;
    };

    int last = -1;
    for (int t = grp; t < nst && ok; t += 2) {
      const int s = t % kTcStages;
      if (!__all_sync(0xffffffffu, mb_wait(&S.full[s], (t / kTcStages) & 1, abort))) {
        *abort = 1;
        atomicExch(err, 4);
        ok = false;
        break;
      }
      // data rows [0, KT R): heads in place, tails 64 rows down (loads first, then the stores)
      float4* tl = reinterpret_cast<float4*>(&S.tile[s][0]);
      float4 xv[NF4];
#pragma unroll
      for (int k = 0; k < NF4; ++k) xv[k] = tl[tid + 128 * k];
#pragma unroll
      for (int k = 0; k < NF4; ++k) {
        const float4 x = xv[k];
        float4 h, l;
        h.x = tf32_rn(x.x), h.y = tf32_rn(x.y), h.z = tf32_rn(x.z), h.w = tf32_rn(x.w);
        l.x = tf32_rn(x.x - h.x), l.y = tf32_rn(x.y - h.y), l.z = tf32_rn(x.z - h.z), l.w = tf32_rn(x.w - h.w);
        tl[tid + 128 * k] = h;
        tl[tid + 128 * k + 64 * 128 / 16] = l;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mb_arrive(&S.conv[s]);
      if (last >= 0 && !flush(last)) {
        *abort = 1;
        atomicExch(err, 5);
        ok = false;
      }
      last = t;
    }
    if (ok && last >= 0 && !flush(last)) {
      *abort = 1;
      atomicExch(err, 5);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) S.red[grp][r][j] = ((double)s_h[j] - (double)c_h[j]) + (x_d[j] + (double)x_l[j]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
  }
  // this CTA's partial: G_i,j = sum over the head and tail rows of row i in every stacked K-tile
  for (int o = threadIdx.x; o < NOUT; o += blockDim.x) {
    const int i = o >> 4, j = o & 15;
    double v = 0.0;
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) v += S.red[g][64 * h + kt * R + i][j];
    P[(int64_t)blockIdx.x * NOUT + o] = v;
  }
  // the last CTA adds the partials in CTA order
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned tk = atomicAdd(ticket, 1u);
    s_last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int o = threadIdx.x; o < NOUT; o += blockDim.x) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 0.0;
    const int G8 = (int)gridDim.x & ~7;
    for (int c = 0; c < G8; c += 8) {
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] += __ldcg(P + (int64_t)(c + k) * NOUT + o);
    }
    for (int c = G8; c < (int)gridDim.x; ++c) a[0] += __ldcg(P + (int64_t)c * NOUT + o);
    G[o] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
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

template <int R>
static void launch_gram_tc(const CUtensorMap& m0, const CUtensorMap& m1, const CUtensorMap& my, int64_t n, int grid,
                           int64_t chunk, double* P, unsigned* tk, double* Gfull, int* err_dev, size_t smem,
                           cudaStream_t s) {
  static std::atomic<uint64_t> attr_set{0};  // one bit per device
  int dev = 0;
  ED_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = (uint64_t)1 << (dev & 63);
  if (!(attr_set.load() & bit)) {
    ED_CUDA(cudaFuncSetAttribute((const void*)k_gram_tc<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set.fetch_or(bit);
  }
  k_gram_tc<R><<<grid, kTcThreads, smem, s>>>(m0, m1, my, n, chunk, P, tk, Gfull, err_dev);
  ED_CHECK_LAUNCH();
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
  // one CTA per SM, contiguous chunks of a multiple of 4 K-tiles (full stages but in the last CTA)
  const int64_t ntile = n / kTcK;
  const int64_t per = ((ntile + sms - 1) / sms + 3) / 4 * 4;
  const int grid = (int)((ntile + per - 1) / per);
  const int64_t chunk = per * kTcK;
  const int R = sym ? 16 : 16 * (nx + 1);
  const int nout = 16 * (sym ? 1 : nx) * 16;
  if (P.n < (size_t)grid * nout) P.alloc((size_t)grid * nout);
  if (Gfull.n < (size_t)nout) Gfull.alloc((size_t)nout);
  if (tk.n < 1) {
    tk.alloc(1);
    ED_CUDA(cudaMemsetAsync(tk.p, 0, sizeof(unsigned), s));
  }
  const size_t smem = sizeof(TcShared) + 1024;
  {
    ProfScope ps_(K_BAND, s, (double)(nx * px + (sym ? 0 : py)) * n * 4.0);
    if (R == 16)
      launch_gram_tc<16>(m0, m1, my, n, grid, chunk, P.p, tk.p, Gfull.p, err_dev, smem, s);
    else if (R == 32)
      launch_gram_tc<32>(m0, m1, my, n, grid, chunk, P.p, tk.p, Gfull.p, err_dev, smem, s);
    else
      launch_gram_tc<48>(m0, m1, my, n, grid, chunk, P.p, tk.p, Gfull.p, err_dev, smem, s);
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
