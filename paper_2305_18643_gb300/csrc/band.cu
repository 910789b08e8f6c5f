// K8 + K9: band-Lanczos Green function (Sec. 4.4) on the GPU.
//
// The p = n_sites starting vectors phi_i = c+_i W (electron part) or c_i W (hole part) span the
// first block of the Krylov space {Phi, H Phi, H^2 Phi, ...} of Sec. 4.4.  The space is built a
// block at a time (the band recursion of Sec. 4.4 applied to all p current vectors at once):
//
//   W = H X_j - X_{j-1} B_{j-1}^T,  A_j = X_j^T W,  W -= X_j A_j,
//   W = X_{j+1} B_j  by SVQB: eigen-decomposition G = W^T W = U diag(l) U^T, X_{j+1} = W U l^{-1/2},
//   B_j = l^{1/2} U^T, directions with l below the deflation threshold dropped (kept as zero
//   columns, so the block width stays p and deflated directions decouple).
//
// When the whole basis fits the memory budget, every new block is also orthogonalized against
// all stored blocks (twice); otherwise against the previous two blocks only.  The projection of
// H on the space is the block-tridiagonal matrix T (diagonal blocks A_j, off-diagonal B_j), and
// the Green function of the part is the matrix element of its resolvent between the starting
// vectors, Phi = X_1 R_0:
//
//   G^e(z) = R_0^T [(z + E0) - T]^{-1}_{11} R_0,   G^h(z) = R_0^T [(z - E0) + T]^{-1}_{11} R_0,
//
// which equals the Lehmann sum over the eigenpairs of T (Eq. spectral1 restricted to the
// Krylov space).  It is evaluated bottom-up as a block continued fraction
//   M_k = s - A_k,  M_j = s - A_j - B_j^T M_{j+1}^{-1} B_j,  G = R_0^T M_1^{-1} R_0
// (with A -> -A, s = z - E0 for the hole part).  Every M_j has a positive-definite imaginary
// part for Im z > 0, so Gaussian elimination without pivoting is stable.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "ed_common.cuh"

namespace ed {

bool gram_tc_usable(const void* X0, const void* X1, const void* Y, int px, int py, int64_t vstride, int64_t n);
void gram_tc_f32(const float* X0, const float* X1, int nx, int px, const float* Y, int py, bool sym, int64_t vstride,
                 int64_t n, DevBuf<double>& P, DevBuf<unsigned>& tk, DevBuf<double>& Gfull, double* G, int* err_dev,
                 cudaStream_t s);

// Scratch of the tensor-core Gram (gram_tc.cu) for one band run; err is set by a kernel whose
// bounded waits gave up.
struct GramTc {
  bool enabled = false;
  DevBuf<double> P, Gfull;
  DevBuf<unsigned> tk;
  DevBuf<int> err;
};

constexpr int kBP = 32;     // maximum block width (cluster sites)
constexpr int kGT2 = 256;
constexpr int kTile = 64;   // elements per Gram tile

// ---- Gram of two blocks: G[i][j] = sum_o X_i[o] Y_j[o] over the padded storage (padding is 0)
template <typename T>
struct GAcc;
template <>
struct GAcc<double> {
  double s = 0.0;
  __device__ void add(double v) { s += v; }
  __device__ double get() const { return s; }
};
template <>
struct GAcc<float> {
  float s = 0.f, k = 0.f;
  __device__ void add(float v) {
    const float y = v - k;
    const float t = s + y;
    k = (t - s) - y;
    s = t;
  }
  __device__ double get() const { return (double)s - (double)k; }
};


template <typename T>
struct VE;
template <>
struct VE<float> {
  using v = float4;
  static constexpr int n = 4;
  __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <>
struct VE<double> {
  using v = double2;
  static constexpr int n = 2;
  __device__ static double2 zero() { return make_double2(0.0, 0.0); }
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// 16-byte copy reading src_bytes (0 or 16) from global memory and zero-filling the rest.
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kGramStages = 6;       // tiles staged per CTA (5 in flight while one is used)
constexpr int kGramTilesPerCta = 16; // 4 x 4 pair tiles per CTA (one per warp); more go to blockIdx.z
constexpr int kGramThreads = 32 * kGramTilesPerCta;

// Products of two 16-byte groups added to a pair's partial sum: FP32 as a packed pair of partial
// sums (fma.rn.f32x2 on (x, y) and (z, w)), FP64 as one sum.
struct GPart32 {
  unsigned long long v = 0ull;  // two FP32 partial sums
  __device__ void fma(const float4& a, const float4& b) {
    unsigned long long a0, a1, b0, b1;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a0) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(a1) : "f"(a.z), "f"(a.w));
    asm("mov.b64 %0, {%1, %2};" : "=l"(b0) : "f"(b.x), "f"(b.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(b1) : "f"(b.z), "f"(b.w));
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(v) : "l"(a0), "l"(b0));
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(v) : "l"(a1), "l"(b1));
  }
  __device__ float take() {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    v = 0ull;
    return lo + hi;
  }
};
struct GPart64 {
  double v = 0.0;
  __device__ void fma(const double2& a, const double2& b) {
    v = ::fma(a.x, b.x, v);
    v = ::fma(a.y, b.y, v);
  }
  __device__ double take() {
    const double r = v;
    v = 0.0;
    return r;
  }
};
template <typename T>
struct GPartOf;
template <>
struct GPartOf<float> {
  using t = GPart32;
};
template <>
struct GPartOf<double> {
  using t = GPart64;
};

// Gram G_b[i][j] = sum_e X_b,i[e] Y_j[e] (i < px, j < py <= 32; blockIdx.y = b selects the X
// block: X0 + b xbstride, or X0 / X1 when xbstride == 0; blockIdx.z a group of 16 pair tiles of
// 4 x 4).  Every CTA takes a contiguous chunk of elements (whole tiles of 32 x GR 16-byte groups)
// and copies each tile's rows (X_b, then Y unless sym, where Y is X_b) to shared memory with
// cp.async, kGramStages tiles in flight.  A warp owns one pair tile of its group and multiplies
// it over the tile, GR 16-byte groups per lane (rows padded by 16 bytes: conflict-free 16-byte
// shared loads).  Products are summed per pair over kGramFlush tiles (FP32: packed FMAs), then
// added with compensation; lanes, chunks and blocks are added in a fixed order, the chunks by
// the last CTA of each X block (a ticket), so the result is deterministic.
constexpr int kGramFlush = 4;
template <typename T, int GR>
__global__ void __launch_bounds__(kGramThreads, 1) k_gram(const T* __restrict__ X0, const T* __restrict__ X1,
                                                         int64_t xbstride, int px, const T* __restrict__ Y, int py,
                                                         int sym, int64_t vstride, int64_t n, int64_t chunk,
                                                         double* __restrict__ P, unsigned* __restrict__ ticket,
                                                         double* __restrict__ G) {
  using V = typename VE<T>::v;
  using Part = typename GPartOf<T>::t;
  constexpr int VN = VE<T>::n;    // elements per 16-byte group
  constexpr int E = 32 * GR * VN; // elements per tile
  constexpr int RS = E + VN;      // padded row stride (elements)
  extern __shared__ __align__(16) unsigned char gsm[];
  T* buf = reinterpret_cast<T*>(gsm);
  __shared__ bool s_last;
  const int nrow = px + (sym ? 0 : py);
  const int yoff = sym ? 0 : px;
  const T* X = xbstride ? X0 + blockIdx.y * xbstride : (blockIdx.y == 0 ? X0 : X1);
  const T* Yp = sym ? X : Y;
  const int64_t e_begin = (int64_t)blockIdx.x * chunk;
  const int64_t e_end = e_begin + chunk < n ? e_begin + chunk : n;
  const int ntile = e_begin < e_end ? (int)((e_end - e_begin + E - 1) / E) : 0;  // the last may be partial
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int TI = (px + 3) / 4, TJ = (py + 3) / 4;
  const int q0 = blockIdx.z * kGramTilesPerCta + warp;
  const bool h0 = q0 < TI * TJ;
  const int ti0 = h0 ? q0 / TJ : 0, tj0 = h0 ? q0 % TJ : 0;
  auto stage = [&](int t) {
    if (t < ntile) {
      const int64_t e0 = e_begin + (int64_t)t * E;
      T* dst = buf + (size_t)(t % kGramStages) * nrow * RS;
      for (int q = threadIdx.x; q < nrow * 32 * GR; q += blockDim.x) {
        const int r = q / (32 * GR), g = q - r * (32 * GR);
        const int64_t e = e0 + g * VN;  // groups past n (ragged last tile) are zero-filled
        const T* src = (r < px ? X + (int64_t)r * vstride : Yp + (int64_t)(r - px) * vstride) + (e < n ? e : 0);
        cp_async16_zfill(dst + r * RS + g * VN, src, e < n ? 16 : 0);
      }
    }
    cp_async_commit();  // an empty group past the end keeps the wait count uniform
  };
  GAcc<T> acc0[16];
  Part part0[16];
  // rows of the pair tile (rows past px / py read row 0; those pairs are not written)
  int xr0[4], yr0[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    xr0[a] = (4 * ti0 + a < px ? 4 * ti0 + a : 0) * RS;
    yr0[a] = (4 * tj0 + a < py ? yoff + 4 * tj0 + a : 0) * RS;
  }
#pragma unroll
  for (int t = 0; t < kGramStages - 1; ++t) stage(t);
  for (int t = 0; t < ntile; ++t) {
    stage(t + kGramStages - 1);
    cp_async_wait<kGramStages - 1>();
    __syncthreads();
    const T* b = buf + (size_t)(t % kGramStages) * nrow * RS + lane * VN;
    if (h0) {
#pragma unroll
      for (int g = 0; g < GR; ++g) {
        const T* bg = b + g * 32 * VN;
        V xv[4], yv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          xv[a] = *reinterpret_cast<const V*>(bg + xr0[a]);
          yv[a] = *reinterpret_cast<const V*>(bg + yr0[a]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) part0[a * 4 + c].fma(xv[a], yv[c]);
      }
      if ((t % kGramFlush) == kGramFlush - 1 || t + 1 == ntile) {
#pragma unroll
        for (int k = 0; k < 16; ++k) acc0[k].add(part0[k].take());
      }
    }
    __syncthreads();  // the buffer of tile t is refilled by stage(t + kGramStages) next round
  }
  cp_async_wait<0>();
  const int npair = px * py;
  double* Pc = P + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * npair;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    double v0 = acc0[k].get();
    for (int o = 16; o > 0; o >>= 1) v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    if (lane == 0) {
      const int a = k >> 2, c = k & 3;
      if (h0 && 4 * ti0 + a < px && 4 * tj0 + c < py) Pc[(4 * ti0 + a) * py + 4 * tj0 + c] = v0;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(ticket + blockIdx.y, 1u);
    s_last = (t == gridDim.x * gridDim.z - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double* Pb = P + (int64_t)blockIdx.y * gridDim.x * npair;
  for (int q = threadIdx.x; q < npair; q += blockDim.x) {
    double v = 0.0;
    for (unsigned c = 0; c < gridDim.x; ++c) v += __ldcg(Pb + (int64_t)c * npair + q);
    G[(int64_t)blockIdx.y * npair + q] = v;
  }
  if (threadIdx.x == 0) ticket[blockIdx.y] = 0u;
}

// Y_j[o] (mode 0: =, 1: -=) sum_k X_k[o] C[k][j] for k < K = nb * px, j < py <= PY.  Each thread
// owns one 16-byte group of elements and all PY outputs in registers; the coefficients are
// broadcast from shared memory.  Reads of X at the thread's elements all precede its writes,
// so Y may alias a block of X.  X blocks: X0 + b * xbstride, or X0 / X1 (xbstride == 0).
template <typename T, int PY>
__global__ void __launch_bounds__(kGT2) k_block_axpy(T* __restrict__ Y, int py, const T* X0, const T* X1,
                                                     int64_t xbstride, int nb, int px, const double* __restrict__ C,
                                                     int64_t vstride, int64_t n, int mode) {
  using V = typename VE<T>::v;
  constexpr int NE = VE<T>::n;
  extern __shared__ __align__(16) unsigned char asm_[];
  T* sc = reinterpret_cast<T*>(asm_);  // [K][PY], zero beyond py
  const int K = nb * px;
  for (int t = threadIdx.x; t < K * PY; t += blockDim.x) {
    const int k = t / PY, j = t - k * PY;
    sc[t] = j < py ? (T)C[k * py + j] : T(0);
  }
  __syncthreads();
  const int64_t ng = n / NE;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = g * NE;
    T acc[NE][PY];
#pragma unroll
    for (int e = 0; e < NE; ++e)
#pragma unroll
      for (int j = 0; j < PY; ++j) acc[e][j] = T(0);
    for (int k0 = 0; k0 < K; k0 += 8) {  // 8 independent 16-byte loads in flight per thread
      V xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + u;
        if (k < K) {
          const int b = k / px, i = k - b * px;
          const T* X = xbstride ? X0 + b * xbstride : (b == 0 ? X0 : X1);
          xv[u] = *reinterpret_cast<const V*>(X + i * vstride + o);
        } else {
          xv[u] = V{};
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (k0 + u >= K) break;
        const T* xs = reinterpret_cast<const T*>(&xv[u]);
        const T* c = sc + (k0 + u) * PY;
#pragma unroll
        for (int j = 0; j < PY; ++j) {
          const T cj = c[j];
#pragma unroll
          for (int e = 0; e < NE; ++e) acc[e][j] += xs[e] * cj;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < PY; ++j) {
      if (j >= py) break;
      V* yp = reinterpret_cast<V*>(Y + j * vstride + o);
      V yv = mode ? *yp : V{};
      T* ys = reinterpret_cast<T*>(&yv);
#pragma unroll
      for (int e = 0; e < NE; ++e) ys[e] = mode ? ys[e] - acc[e][j] : acc[e][j];
      *yp = yv;
    }
  }
}

// ---- small dense work of one block step (one thread block) ---------------------------------
// SVQB of a block with Gram G: Cout = U l^{-1/2} (new basis = W Cout), Bout = l^{1/2} U^T
// (W = new basis * Bout); directions with l <= thr are dropped (zero columns / rows).  Writes
// the number of kept directions to *rank.  Parallel two-sided Jacobi on one warp: every round
// applies m/2 disjoint rotations at once (round-robin pairing of the m = p rounded up to even
// indices; an index >= p is a dummy), A <- J^T A J with J block-diagonal, so a sweep is m - 1
// rounds.  Sweeps stop when the off-diagonal norm is below 1e-26 of the total.
__global__ void __launch_bounds__(32) k_svqb(const double* __restrict__ G, int p, double thr,
                                             double* __restrict__ Cout, double* __restrict__ Bout,
                                             int* __restrict__ rank) {
  __shared__ double a[kBP][kBP + 1], v[kBP][kBP + 1];
  __shared__ double cs[kBP / 2], sn[kBP / 2];
  __shared__ int pr[kBP / 2], pq[kBP / 2];
  const int lane = threadIdx.x;
  for (int t = lane; t < p * p; t += 32) {
    const int i = t / p, j = t - i * p;
    a[i][j] = 0.5 * (G[i * p + j] + G[j * p + i]);
    v[i][j] = i == j ? 1.0 : 0.0;
  }
  __syncwarp();
  const int m = p + (p & 1), half = m / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int t = lane; t < p * p; t += 32) {
      const int i = t / p, j = t - i * p;
      tot += a[i][j] * a[i][j];
      if (i != j) off += a[i][j] * a[i][j];
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (!(off > 1e-26 * tot)) break;
    for (int round = 0; round < m - 1; ++round) {
      if (lane < half) {  // pair lane: positions lane and m - 1 - lane of the round-robin circle
        const int pa = lane, pb = m - 1 - lane;
        int r = pa == 0 ? 0 : 1 + (pa - 1 + round) % (m - 1);
        int q = pb == 0 ? 0 : 1 + (pb - 1 + round) % (m - 1);
        if (r > q) {
          const int t = r;
          r = q;
          q = t;
        }
        double c = 1.0, s = 0.0;
        if (q < p) {
          const double arq = a[r][q];
          if (fabs(arq) >= 1e-300) {
            const double theta = (a[q][q] - a[r][r]) / (2.0 * arq);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        pr[lane] = r;
        pq[lane] = q < p ? q : r;  // a dummy pair becomes (r, r) and is skipped below
        cs[lane] = c;
        sn[lane] = s;
      }
      __syncwarp();
      // columns: A <- A J, V <- V J
      for (int t = lane; t < half * p; t += 32) {
        const int i = t / p, k = t - i * p, r = pr[i], q = pq[i];
        if (r == q) continue;
        const double c = cs[i], s = sn[i];
        const double akr = a[k][r], akq = a[k][q];
        a[k][r] = c * akr - s * akq;
        a[k][q] = s * akr + c * akq;
        const double vkr = v[k][r], vkq = v[k][q];
        v[k][r] = c * vkr - s * vkq;
        v[k][q] = s * vkr + c * vkq;
      }
      __syncwarp();
      // rows: A <- J^T A
      for (int t = lane; t < half * p; t += 32) {
        const int i = t / p, k = t - i * p, r = pr[i], q = pq[i];
        if (r == q) continue;
        const double c = cs[i], s = sn[i];
        const double ark = a[r][k], aqk = a[q][k];
        a[r][k] = c * ark - s * aqk;
        a[q][k] = s * ark + c * aqk;
      }
      __syncwarp();
    }
  }
  __syncwarp();
  int r = 0;
  for (int k = 0; k < p; ++k) r += a[k][k] > thr;
  for (int t = lane; t < p * p; t += 32) {
    const int i = t / p, k = t - i * p;
    const double l = a[k][k];
    const bool keep = l > thr;
    Cout[i * p + k] = keep ? v[i][k] / sqrt(l) : 0.0;
    Bout[k * p + i] = keep ? v[i][k] * sqrt(l) : 0.0;
  }
  if (lane == 0) *rank = r;
}

// out = a * b (p x p), optionally transposing b: used to chain the two SVQB factors and to form
// the corrections of the recursion.
__global__ void k_small_gemm(const double* __restrict__ a, const double* __restrict__ b, int p, int tb,
                             double* __restrict__ out, double scale) {
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int i = t / p, j = t - i * p;
    double s = 0.0;
    for (int k = 0; k < p; ++k) s += a[i * p + k] * (tb ? b[j * p + k] : b[k * p + j]);
    out[t] = scale * s;
  }
}

// out = a + beta * out (p x p)
__global__ void k_small_axpy(const double* __restrict__ a, int n, double* __restrict__ out, double beta) {
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) out[t] = a[t] + (beta != 0.0 ? beta * out[t] : 0.0);
}

// out = a, or its symmetric part (sym); each unordered pair is read and written by one thread,
// so out may alias a.
__global__ void k_small_copy(const double* a, int n, double* out, int sym) {
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, j = t - i * n;
    if (!sym) {
      out[t] = a[t];
    } else if (i <= j) {
      const double v = 0.5 * (a[i * n + j] + a[j * n + i]);
      out[i * n + j] = v;
      out[j * n + i] = v;
    }
  }
}

// ---- block continued fraction on the grid --------------------------------------------------
struct BandCoeffs {
  const double* A;   // [k][p][p]
  const double* B;   // [k][p][p]   W_j = X_{j+1} B_j
  const double* R0;  // [p][p]      Phi = X_1 R0
  int k, p;
  double E0, sgn;    // sgn = +1 electron (s = z + E0, M = s - A), -1 hole (s = z - E0, M = s + A)
};

// One thread block per frequency: complex p x p matrices in shared memory.
__global__ void __launch_bounds__(256) k_band_cf(BandCoeffs bc, const double2* __restrict__ z, int nz, int zstride,
                                                 double2* __restrict__ out /* [nz][p][p] */, double2* __restrict__ prev,
                                                 double* __restrict__ maxdiff) {
  __shared__ double2 M[kBP][kBP + 1];
  __shared__ double2 Y[kBP][2 * kBP + 1];
  __shared__ double2 fcol[kBP];
  const int zi = blockIdx.x;
  if (zi * zstride >= nz) return;
  const double2 zz = z[zi * zstride];
  const int p = bc.p;
  const double2 s = make_double2(zz.x + bc.sgn * bc.E0, zz.y);
  const int tid = threadIdx.x, nt = blockDim.x;
  auto init_M = [&](int j) {
    for (int t = tid; t < p * p; t += nt) {
      const int a = t / p, b = t - a * p;
      double v = -bc.sgn * bc.A[((int64_t)j * p + a) * p + b];
      M[a][b] = make_double2((a == b ? s.x : 0.0) + v, a == b ? s.y : 0.0);
    }
  };
  // Solve M Y = rhs (rhs p x m, real) in place: augmented [M | rhs] in Y, no pivoting.
  auto solve = [&](const double* rhs, int m, bool rhs_t) {
    for (int t = tid; t < p * (p + m); t += nt) {
      const int a = t / (p + m), b = t - a * (p + m);
      if (b < p)
        Y[a][b] = M[a][b];
      else {
        const double r = rhs_t ? rhs[(b - p) * p + a] : rhs[a * p + (b - p)];
        Y[a][b] = make_double2(r, 0.0);
      }
    }
    __syncthreads();
    for (int c = 0; c < p; ++c) {
      const double2 piv = Y[c][c];
      const double den = piv.x * piv.x + piv.y * piv.y;
      const double2 ip = make_double2(piv.x / den, -piv.y / den);
      __syncthreads();
      for (int t = tid; t < p + m; t += nt) {  // scale pivot row
        const double2 v = Y[c][t];
        if (t >= c) Y[c][t] = make_double2(v.x * ip.x - v.y * ip.y, v.x * ip.y + v.y * ip.x);
      }
      for (int t = tid; t < p; t += nt) fcol[t] = Y[t][c];
      __syncthreads();
      for (int t = tid; t < p * (p + m); t += nt) {
        const int a = t / (p + m), b = t - a * (p + m);
        if (a == c || b < c) continue;
        const double2 f = fcol[a], v = Y[c][b];
        Y[a][b].x -= f.x * v.x - f.y * v.y;
        Y[a][b].y -= f.x * v.y + f.y * v.x;
      }
      __syncthreads();
    }
  };
  init_M(bc.k - 1);
  __syncthreads();
  for (int j = bc.k - 2; j >= 0; --j) {
    // Y = M_{j+1}^{-1} B_j  (B_j: p x p, row index = new-basis direction)
    solve(bc.B + (int64_t)j * p * p, p, false);
    // M_j = s -/+ A_j - B_j^T Y
    for (int t = tid; t < p * p; t += nt) {
      const int a = t / p, b = t - a * p;
      double2 acc = make_double2(0.0, 0.0);
      for (int k2 = 0; k2 < p; ++k2) {
        const double bk = bc.B[((int64_t)j * p + k2) * p + a];
        acc.x += bk * Y[k2][p + b].x;
        acc.y += bk * Y[k2][p + b].y;
      }
      const double v = -bc.sgn * bc.A[((int64_t)j * p + a) * p + b];
      M[a][b] = make_double2((a == b ? s.x : 0.0) + v - acc.x, (a == b ? s.y : 0.0) - acc.y);
    }
    __syncthreads();
  }
  // G = R0^T M_1^{-1} R0
  solve(bc.R0, p, false);
  double local = 0.0;
  for (int t = tid; t < p * p; t += nt) {
    const int a = t / p, b = t - a * p;
    double2 acc = make_double2(0.0, 0.0);
    for (int k2 = 0; k2 < p; ++k2) {
      const double r = bc.R0[k2 * p + a];
      acc.x += r * Y[k2][p + b].x;
      acc.y += r * Y[k2][p + b].y;
    }
    const int64_t o = (int64_t)zi * p * p + t;
    if (prev) {
      const double2 q = prev[o];
      local = fmax(local, hypot(acc.x - q.x, acc.y - q.y));
      prev[o] = acc;
    } else {
      out[o] = acc;
    }
  }
  if (maxdiff) {
    for (int off = 16; off > 0; off >>= 1) local = fmax(local, __shfl_down_sync(0xffffffffu, local, off));
    if ((tid & 31) == 0) atomicMax((unsigned long long*)maxdiff, __double_as_longlong(local));
  }
}

// ---- driver -----------------------------------------------------------------------------------
static int g_grid(int64_t n, int per) {
  int64_t b = (n + per - 1) / per;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

// G[b][i][j] = <X_b,i, Y_j> for the nb blocks of X (n elements per vector, a multiple of 128).
template <typename T, int GR>
static void gram_launch(const T* X, const T* X1, int64_t xbstride, int nb, int px, const T* Y, int py, bool sym,
                        int64_t vstride, int64_t n, DevBuf<double>& P, DevBuf<unsigned>& tk, double* G, cudaStream_t s) {
  constexpr int E = 32 * GR * VE<T>::n;
  const int ntiles_pair = ((px + 3) / 4) * ((py + 3) / 4);
  const int gz = (ntiles_pair + kGramTilesPerCta - 1) / kGramTilesPerCta;
  int sms = 152, dev = 0;
  ED_CUDA(cudaGetDevice(&dev));
  ED_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t tiles = (n + E - 1) / E;
  const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, std::max(1, sms / (nb * gz))));
  const int64_t chunk = (tiles + nchunk - 1) / nchunk * E;
  const int npair = px * py;
  if (P.n < (size_t)nb * nchunk * npair) P.alloc((size_t)nb * nchunk * npair);
  if (tk.n < (size_t)nb) {
    tk.alloc((size_t)nb);
    ED_CUDA(cudaMemsetAsync(tk.p, 0, (size_t)nb * sizeof(unsigned), s));
  }
  const int nrow = px + (sym ? 0 : py);
  const size_t smem = (size_t)kGramStages * nrow * (E + VE<T>::n) * sizeof(T);
  allow_max_dynamic_smem(k_gram<T, GR>);
  ProfScope ps_(K_BAND, s, 0.0);
  k_gram<T, GR><<<dim3(nchunk, nb, gz), kGramThreads, smem, s>>>(X, X1, xbstride, px, Y, py, sym ? 1 : 0, vstride, n, chunk,
                                                        P.p, tk.p, G);
  ED_CHECK_LAUNCH();
}

template <typename T>
static void gram(const T* X, const T* X1, int64_t xbstride, int nb, int px, const T* Y, int py, int64_t vstride,
                 int64_t n, DevBuf<double>& P, DevBuf<unsigned>& tk, double* G, cudaStream_t s, GramTc* tc = nullptr) {
  const bool sym = nb == 1 && xbstride == 0 && X == Y && px == py;
  if constexpr (std::is_same<T, float>::value) {
    // W^T W of FP32 blocks on the tensor cores, where that kernel is the faster one (measured at
    // the 4x4 band size: 3.3 ms against 3.5 ms on 16 vectors; the projections on one or two X
    // blocks ran 6.6 / 13.1 ms against 5.0 / 9.9 ms on the CUDA cores, so they stay there)
    if (tc && tc->enabled && sym &&
        gram_tc_usable(X, nb > 1 ? X1 : X, Y, px, py, vstride, n)) {
      gram_tc_f32(X, X1, nb, px, Y, py, sym, vstride, n, tc->P, tc->tk, tc->Gfull, G, tc->err.p, s);
      return;
    }
  }
  const int nrow = px + (sym ? 0 : py);
  // 16-byte groups per lane per tile: tiles of at most 32 KB, so kGramStages of them fit shared
  // memory and ~160 KB are in flight per SM
  if (nrow <= 16)
    gram_launch<T, 4>(X, X1, xbstride, nb, px, Y, py, sym, vstride, n, P, tk, G, s);
  else if (nrow <= 32)
    gram_launch<T, 2>(X, X1, xbstride, nb, px, Y, py, sym, vstride, n, P, tk, G, s);
  else
    gram_launch<T, 1>(X, X1, xbstride, nb, px, Y, py, sym, vstride, n, P, tk, G, s);
}

template <typename T, int PY>
static void block_axpy_launch(T* Y, int py, const T* X, const T* X1, int64_t xbstride, int nb, int px, const double* C,
                              int64_t vstride, int64_t n, int mode, cudaStream_t s) {
  const size_t smem = (size_t)nb * px * PY * sizeof(T);
  ProfScope ps_(K_BAND, s, 0.0);
  k_block_axpy<T, PY><<<g_grid(n / VE<T>::n, kGT2), kGT2, smem, s>>>(Y, py, X, X1, xbstride, nb, px, C, vstride, n, mode);
  ED_CHECK_LAUNCH();
}

// Y -= / = X C over nb blocks of X; n is a multiple of the 16-byte element group (padded rows).
template <typename T>
static void block_axpy(T* Y, int py, const T* X, const T* X1, int64_t xbstride, int nb, int px, const double* C,
                       int64_t vstride, int64_t n, int mode, cudaStream_t s) {
  if (py > 16) throw Error(ED_ERR_INVALID, "band Lanczos block width above 16 is not supported");
  const int PYs = py <= 4 ? 4 : py <= 8 ? 8 : 16;
  // at most 64 coefficient rows per launch (one pass over the X blocks they touch)
  const int per = std::max(1, 64 / px);
  for (int b0 = 0; b0 < nb; b0 += per) {
    const int m = std::min(per, nb - b0);
    if (mode == 0 && b0 > 0) throw Error(ED_ERR_INVALID, "block_axpy: assignment over several chunks");
    const T* xa = xbstride ? X + (int64_t)b0 * xbstride : (b0 == 0 ? X : X1);
    const T* xb = xbstride ? nullptr : X1;
    const double* cb = C + (int64_t)b0 * px * py;
    if (PYs == 4)
      block_axpy_launch<T, 4>(Y, py, xa, xb, xbstride, m, px, cb, vstride, n, mode, s);
    else if (PYs == 8)
      block_axpy_launch<T, 8>(Y, py, xa, xb, xbstride, m, px, cb, vstride, n, mode, s);
    else
      block_axpy_launch<T, 16>(Y, py, xa, xb, xbstride, m, px, cb, vstride, n, mode, s);
  }
}

// The CUDA-core FP32 Gram alone (the check of the tensor-core one): nb blocks of px vectors
// (X + b * 16 vstride) against py vectors Y.
void gram_f32_cuda(const float* X, int nb, int px, const float* Y, int py, int64_t vstride, int64_t n, double* G,
                   cudaStream_t s) {
  DevBuf<double> P;
  DevBuf<unsigned> tk;
  gram<float>(X, nb > 1 ? X + 16 * vstride : nullptr, 0, nb, px, Y, py, vstride, n, P, tk, G, s);
  ED_CUDA(cudaStreamSynchronize(s));
}

// FP64 forms of the two block kernels for other drivers (Davidson): G[b][i][j] = sum X_{b,i} Y_j
// over nb blocks of px vectors (X + b xbstride), and Y (mode 0: =, 1: -=) X C.
void gram_f64(const double* X, int64_t xbstride, int nb, int px, const double* Y, int py, int64_t vstride, int64_t n,
              DevBuf<double>& P, DevBuf<unsigned>& tk, double* G, cudaStream_t s) {
  gram<double>(X, nullptr, xbstride, nb, px, Y, py, vstride, n, P, tk, G, s);
}
void block_axpy_f64(double* Y, int py, const double* X, int64_t xbstride, int nb, int px, const double* C,
                    int64_t vstride, int64_t n, int mode, cudaStream_t s) {
  block_axpy<double>(Y, py, X, nullptr, xbstride, nb, px, C, vstride, n, mode, s);
}

struct BandOptions {
  double tol;         // |Delta G| on the grid between checks
  int max_dim;        // Krylov vectors per part
  size_t mem_budget;  // bytes for stored blocks (full reorthogonalization when they fit)
};

void launch_apply_cop_runs(ed_cluster& c, int spin, bool electron, int dtype, const int2* runs_dev, int nruns,
                           void* phi, int64_t vstride, int64_t du, int64_t dd, int64_t ld, cudaStream_t s);

template <typename T>
static bool band_part(ed_cluster& c, int spin, bool electron, const DevBuf<double2>& zd, int nz, double2* Gout,
                      const BandOptions& opt, int64_t* total, int* maxd, bool* converged) {
  cudaStream_t s = c.stream;
  const int dtype = sizeof(T) == 8 ? ED_FP64 : ED_FP32;
  const int nu = c.desc.n_up, nd = c.desc.n_dn, L = c.model.L;
  const int dN = electron ? 1 : -1;
  const int nu_t = nu + (spin == 0 ? dN : 0), nd_t = nd + (spin == 1 ? dN : 0);
  if (nu_t < 0 || nd_t < 0 || nu_t > L || nd_t > L) return false;
  const int p = c.model.ns;
  if (p > kBP) throw Error(ED_ERR_INVALID, "band Lanczos supports at most 32 cluster sites");
  const int64_t ld = padded_ld(c.tables(nd_t).dim);
  SectorView sv = c.view(nu_t, nd_t, ld);
  const int64_t du = sv.d_up, dd = sv.d_dn;
  const int64_t vstride = du * ld;  // one vector (padded storage)
  const int64_t n = vstride;
  const int64_t blk = (int64_t)p * vstride;  // one block of p vectors
  const int64_t reach = du * dd;
  const int kmax = (int)std::max<int64_t>(2, std::min<int64_t>((opt.max_dim + p - 1) / p, (2 * reach) / p + 4));
  const bool full = (size_t)(kmax + 2) * blk * sizeof(T) <= opt.mem_budget;
  // storage: full reorthogonalization keeps every block; otherwise a ring of 3 blocks.
  const int nstore = full ? kmax + 2 : 3;
  DevBuf<T> Vs((size_t)nstore * blk), Wb(blk);
  ED_CUDA(cudaMemsetAsync(Vs.p, 0, (size_t)nstore * blk * sizeof(T), s));
  ED_CUDA(cudaMemsetAsync(Wb.p, 0, blk * sizeof(T), s));
  auto Xb = [&](int j) { return Vs.p + (int64_t)(full ? j : j % 3) * blk; };
  const int pp = p * p;
  double scale2 = 1.0;
  DevBuf<double> A((size_t)kmax * pp), B((size_t)kmax * pp), R0(pp), G((size_t)(kmax + 2) * pp), Cm(pp), Bm(pp),
      C2(pp), B2(pp), tmp(pp), P;
  DevBuf<unsigned> gtk;  // tickets of the Gram kernel (zeroed at allocation, reset by its last CTA)
  DevBuf<int> rank(1);
  GramTc tc;
  tc.enabled = c.tensor_gram && dtype == ED_FP32;
  tc.err.alloc(1);
  ED_CUDA(cudaMemsetAsync(tc.err.p, 0, sizeof(int), s));
  ED_CUDA(cudaMemsetAsync(A.p, 0, (size_t)kmax * pp * sizeof(double), s));
  ED_CUDA(cudaMemsetAsync(B.p, 0, (size_t)kmax * pp * sizeof(double), s));
  // starting block Phi (into W), orthonormalized into X_0 with Phi = X_0 R0
  std::vector<int2> runs_h(p);
  for (int i = 0; i < p; ++i) runs_h[i] = make_int2(i, -1);
  DevBuf<int2> druns(p);
  ED_CUDA(cudaMemcpyAsync(druns.p, runs_h.data(), p * sizeof(int2), cudaMemcpyHostToDevice, s));
  launch_apply_cop_runs(c, spin, electron, dtype, druns.p, p, Wb.p, vstride, du, dd, ld, s);
  // deflation: a direction is dropped when its norm is below eps_rel times the operator scale
  double hscale = 1.0;
  for (double v : c.model.h) hscale = std::max(hscale, std::fabs(v));
  for (double v : c.model.U) hscale = std::max(hscale, std::fabs(v));
  const double eps_rel = dtype == ED_FP64 ? 1e-10 : 1e-4;
  auto orthonormalize = [&](double scale2, double* Bfinal, T* dst) -> int {
    // two SVQB passes: W = X (B2 B1); the second writes the orthonormal block into dst
    int r = 0;
    gram<T>(Wb.p, nullptr, 0, 1, p, Wb.p, p, vstride, n, P, gtk, G.p, s, &tc);
    { ProfScope ps_(K_BAND, s, 0.0); k_svqb<<<1, 32, 0, s>>>(G.p, p, eps_rel * eps_rel * scale2, Cm.p, Bm.p, rank.p); }
    ED_CHECK_LAUNCH();
    block_axpy<T>(Wb.p, p, Wb.p, nullptr, 0, 1, p, Cm.p, vstride, n, 0, s);
    gram<T>(Wb.p, nullptr, 0, 1, p, Wb.p, p, vstride, n, P, gtk, G.p, s, &tc);
    { ProfScope ps_(K_BAND, s, 0.0); k_svqb<<<1, 32, 0, s>>>(G.p, p, 0.25, C2.p, B2.p, rank.p); }
    ED_CHECK_LAUNCH();
    block_axpy<T>(dst, p, Wb.p, nullptr, 0, 1, p, C2.p, vstride, n, 0, s);
    { ProfScope ps_(K_BAND, s, 0.0); k_small_gemm<<<1, 256, 0, s>>>(B2.p, Bm.p, p, 0, Bfinal, 1.0); }
    ED_CHECK_LAUNCH();
    int err = 0;
    ED_CUDA(cudaMemcpyAsync(&r, rank.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaMemcpyAsync(&err, tc.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    if (err) throw Error(ED_ERR_TIMEOUT, "a bounded wait of the tensor-core Gram gave up (role " + std::to_string(err) + ")");
    return r;
  };
  orthonormalize(1.0, R0.p, Xb(0));
  scale2 = hscale * hscale;
  // check grid (every zstride-th frequency)
  const int zstride = std::max(1, nz / 512);
  const int nzc = (nz + zstride - 1) / zstride;
  DevBuf<double2> prev((size_t)nzc * pp);
  ED_CUDA(cudaMemsetAsync(prev.p, 0, (size_t)nzc * pp * sizeof(double2), s));
  DevBuf<double> dmax(1);
  double* hmax = pinned_scratch() + 17;
  const double sgn = electron ? 1.0 : -1.0;
  int k = 0, hits = 0, next_check = 2;
  bool conv = false;
  for (int j = 0; j < kmax; ++j) {
    // W = H X_j
    launch_hpsi_block(sv, c.hp, dtype, Xb(j), Wb.p, vstride, p, s);
    // project W on the previous blocks and remove the projection: on every stored block twice
    // (classical Gram-Schmidt twice), or once on [X_{j-1}, X_j] (the three-term block recurrence,
    // as the band method of Sec. 4.4 orthogonalizes only against the band).  The X_j components
    // give A_j.
    for (int pass = 0; pass < (full ? 2 : 1); ++pass) {
      int nbk;
      if (full) {
        nbk = j + 1;
        gram<T>(Xb(0), nullptr, blk, nbk, p, Wb.p, p, vstride, n, P, gtk, G.p, s);
        block_axpy<T>(Wb.p, p, Xb(0), nullptr, blk, nbk, p, G.p, vstride, n, 1, s);
      } else if (j > 0) {
        nbk = 2;
        gram<T>(Xb(j - 1), Xb(j), 0, 2, p, Wb.p, p, vstride, n, P, gtk, G.p, s, &tc);
        block_axpy<T>(Wb.p, p, Xb(j - 1), Xb(j), 0, 2, p, G.p, vstride, n, 1, s);
      } else {
        nbk = 1;
        gram<T>(Xb(0), nullptr, 0, 1, p, Wb.p, p, vstride, n, P, gtk, G.p, s, &tc);
        block_axpy<T>(Wb.p, p, Xb(0), nullptr, 0, 1, p, G.p, vstride, n, 1, s);
      }
      { ProfScope ps_(K_BAND, s, 0.0); k_small_axpy<<<1, 256, 0, s>>>(G.p + (int64_t)(nbk - 1) * pp, p, A.p + (int64_t)j * pp, pass ? 1.0 : 0.0); }
      ED_CHECK_LAUNCH();
    }
    { ProfScope ps_(K_BAND, s, 0.0); k_small_copy<<<1, 256, 0, s>>>(A.p + (int64_t)j * pp, p, A.p + (int64_t)j * pp, 1); }
    ED_CHECK_LAUNCH();
    // W = X_{j+1} B_j
    const int r = orthonormalize(scale2, B.p + (int64_t)j * pp, j + 1 < kmax ? Xb(j + 1) : Wb.p);
    k = j + 1;
    if (r == 0) {
      conv = true;  // the Krylov space is exhausted: T is exact
      break;
    }
    if (k == next_check || j + 1 == kmax) {
      BandCoeffs bc{A.p, B.p, R0.p, k, p, c.gs.E0, sgn};
      ED_CUDA(cudaMemsetAsync(dmax.p, 0, sizeof(double), s));
      { ProfScope ps_(K_GF_EVAL, s, 0.0); k_band_cf<<<nzc, 256, 0, s>>>(bc, zd.p, nz, zstride, nullptr, prev.p, dmax.p); }
      ED_CHECK_LAUNCH();
      ED_CUDA(cudaMemcpyAsync(hmax, dmax.p, sizeof(double), cudaMemcpyDeviceToHost, s));
      ED_CUDA(cudaStreamSynchronize(s));
      if (*hmax < opt.tol) {
        if (++hits >= 2) {
          conv = true;
          break;
        }
      } else {
        hits = 0;
      }
      next_check = k + std::max(2, k / 8);
    }
  }
  BandCoeffs bc{A.p, B.p, R0.p, k, p, c.gs.E0, sgn};
  { ProfScope ps_(K_GF_EVAL, s, 0.0); k_band_cf<<<nz, 256, 0, s>>>(bc, zd.p, nz, 1, Gout, nullptr, nullptr); }
  ED_CHECK_LAUNCH();
  ED_CUDA(cudaStreamSynchronize(s));
  *total += (int64_t)k * p;
  *maxd = std::max(*maxd, k * p);
  *converged = *converged && conv;
  return true;
}

__global__ void k_gf_add(const double2* __restrict__ a, const double2* __restrict__ b, int64_t n, double2* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (a) {
      v.x += a[t].x;
      v.y += a[t].y;
    }
    if (b) {
      v.x += b[t].x;
      v.y += b[t].y;
    }
    out[t] = v;
  }
}

bool run_green_band(ed_cluster& c, int spin, const double2* z_host, int nz, double2* G_dev) {
  cudaStream_t s = c.stream;
  const int p = c.model.ns;
  const int dtype = c.desc.precision;
  BandOptions opt{c.gf_tol > 0 ? c.gf_tol : (dtype == ED_FP64 ? 1e-10 : 1e-6), c.band_max_dim > 0 ? c.band_max_dim : 20000,
                  c.gf_mem_budget ? c.gf_mem_budget : size_t(32) << 30};
  DevBuf<double2> zd(nz);
  ED_CUDA(cudaMemcpyAsync(zd.p, z_host, nz * sizeof(double2), cudaMemcpyHostToDevice, s));
  DevBuf<double2> Ge((size_t)nz * p * p), Gh((size_t)nz * p * p);
  c.gf_total_steps = 0;
  c.gf_max_steps = 0;
  bool conv = true, he, hh;
  if (dtype == ED_FP64) {
    he = band_part<double>(c, spin, true, zd, nz, Ge.p, opt, &c.gf_total_steps, &c.gf_max_steps, &conv);
    hh = band_part<double>(c, spin, false, zd, nz, Gh.p, opt, &c.gf_total_steps, &c.gf_max_steps, &conv);
  } else {
    he = band_part<float>(c, spin, true, zd, nz, Ge.p, opt, &c.gf_total_steps, &c.gf_max_steps, &conv);
    hh = band_part<float>(c, spin, false, zd, nz, Gh.p, opt, &c.gf_total_steps, &c.gf_max_steps, &conv);
  }
  {
    ProfScope ps_(K_GF_EVAL, s, 0.0);
    const int64_t nn = (int64_t)nz * p * p;
    k_gf_add<<<(unsigned)std::min<int64_t>((nn + 255) / 256, 1024), 256, 0, s>>>(he ? Ge.p : nullptr, hh ? Gh.p : nullptr, nn, G_dev);
    ED_CHECK_LAUNCH();
  }
  ED_CUDA(cudaStreamSynchronize(s));
  return conv;
}

}  // namespace ed
