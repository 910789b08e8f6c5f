// Batched form: many small clusters solved together (ground state, Sec. 4.2, and continued-
// fraction Green function, Sec. 4.3, for each).
//
// 1. Tables of every (cluster, particle number) needed are built by three launches into one
//    arena.  Their sizes follow from closed forms: d = C(L, N) states and at most N (L - N) hops
//    per state, stored slot-major ([zmax][d]) with a per-state count, so no count/scan pass runs.
// 2. A persistent kernel solves the ground states: every block takes the next cluster from an
//    atomic queue (largest sector first) and runs the whole Lanczos ground-state algorithm of
//    the single-cluster path inside the block (block-level fused H.psi with FP64 reductions, the
//    tridiagonal check of tridiag.cuh, the retrace, the FP64 polish and restarts).
// 3. A second persistent kernel runs the continued fractions: every block takes the next
//    (cluster, spin, part, pair) from the queue, applies c+ / c to the ground state and runs the
//    recursion with the convergence check on the frequency grid.
// 4. Two grid-wide kernels evaluate every continued fraction on the grid and assemble G.
// Block width and the element-to-thread mapping of the block-level H.psi are picked by an
// autotuner on the first call for a given batch shape.  No block ever waits on another block.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>

#include "ed_common.cuh"
#include "tridiag.cuh"

namespace ed {

constexpr int kBMaxIter = 600;     // Lanczos levels per ground-state pass
constexpr int kBMaxL = 20;         // orbitals per batched cluster
constexpr int kBCheck = 10;

struct BBinom {
  uint32_t c[kMaxOrb + 1][kMaxOrb + 1];
};

struct BTable {            // one spin sector of one cluster
  int L, N, split, zmax;
  int64_t dim;
  uint32_t* basis;         // [dim]
  int32_t* rank_lo;        // [2^split]
  int32_t* rank_hi;        // [2^(L - split)]
  uint32_t* ell;           // [zmax][dim] packed entries (col << 8 | neg << 7 | vidx)
  uint8_t* cnt;            // [dim] entries of each state
  double* e64;             // [dim] one-body diagonal
  float* e32;
  int cluster;
};

struct BPair {
  uint32_t a, b, vidx, between;
};

struct BCluster {
  HopParams hp;
  int ns, L, n_up, n_dn;
  int t_up, t_dn;            // GS tables
  int t_upp, t_upm, t_dnp, t_dnm;   // N +- 1 tables (-1: none)
  int64_t d;                 // GS sector dimension
  double* omega;             // FP64 ground state [d]
  uint64_t seed;
  double tol;
  int precision;
  // results
  double E0, residual, gap;
  int iters, status;
};

struct BRun {                // one continued fraction
  int cluster, spin, part, i, j;   // part 0 electron, 1 hole; j = -1 for a diagonal run
  int tu, td;                // target sector tables
  int src;                   // table of the changed spin in the GS sector
  int64_t d;                 // target sector dimension
  double* alpha;             // [mmax]
  double* beta;              // [mmax + 1]
  int mmax;                  // levels of this run: min(cap, 2 d + 16), as the single-cluster path
  double b0sq;
  int nsteps;
};

// -------------------------------------------------------------------------------- tables
__global__ void k_bt_basis(BTable* __restrict__ T, BBinom bn) {
  BTable t = T[blockIdx.y];
  const int64_t nlo = int64_t(1) << t.split, nhi = int64_t(1) << (t.L - t.split);
  const int64_t n = max(t.dim, max(nlo, nhi));
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    if (r < t.dim) {
      uint32_t rem = (uint32_t)r, b = 0;
      int p = t.L - 1;
      for (int k = t.N; k >= 1; --k) {
        while (bn.c[p][k] > rem) --p;
        b |= 1u << p;
        rem -= bn.c[p][k];
        --p;
      }
      t.basis[r] = b;
    }
    if (r < nlo) {
      int32_t v = 0;
      int j = 0;
      for (int p = 0; p < t.split; ++p)
        if ((r >> p) & 1) v += (int32_t)bn.c[p][++j];
      t.rank_lo[r] = v;
    }
    if (r < nhi) {
      const int m = t.N - __popc((uint32_t)r);
      int32_t v = -1;
      if (m >= 0 && m <= t.split) {
        v = 0;
        int j = 0;
        for (int q = 0; q < t.L - t.split; ++q)
          if ((r >> q) & 1) v += (int32_t)bn.c[q + t.split][m + (++j)];
      }
      t.rank_hi[r] = v;
    }
  }
}

__global__ void k_bt_fill(BTable* __restrict__ T, const BPair* __restrict__ pairs, const int* __restrict__ pair_off,
                          const double* __restrict__ hdiag /* [cluster][kMaxOrb] */) {
  BTable t = T[blockIdx.y];
  const BPair* pp = pairs + pair_off[t.cluster];
  const int np = pair_off[t.cluster + 1] - pair_off[t.cluster];
  const double* hd = hdiag + (int64_t)t.cluster * kMaxOrb;
  const uint32_t lomask = (1u << t.split) - 1u;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < t.dim; r += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t s = t.basis[r];
    int k = 0;
    for (int q = 0; q < np; ++q) {
      const BPair p = pp[q];
      if (((s >> p.a) & 1u) && !((s >> p.b) & 1u)) {
        const uint32_t c = s ^ (1u << p.a) ^ (1u << p.b);
        const uint32_t neg = __popc(s & p.between) & 1u;
        const uint32_t col = (uint32_t)(t.rank_lo[c & lomask] + t.rank_hi[c >> t.split]);
        if (k < t.zmax) t.ell[(int64_t)k * t.dim + r] = (col << 8) | (neg << 7) | p.vidx;
        ++k;
      }
    }
    t.cnt[r] = (uint8_t)min(k, t.zmax);
    double e = 0.0;
    for (int a = 0; a < t.L; ++a)
      if ((s >> a) & 1u) e += hd[a];
    t.e64[r] = e;
    t.e32[r] = (float)e;
  }
}

// -------------------------------------------------------------------------------- block-level H.psi
template <typename T>
struct BP;
template <>
struct BP<double> {
  __device__ static const double* e(const BTable& t) { return t.e64; }
  __device__ static double val(const HopParams& h, int i) { return h.val[i]; }
  __device__ static double U(const HopParams& h, int i) { return h.U[i]; }
};
template <>
struct BP<float> {
  __device__ static const float* e(const BTable& t) { return t.e32; }
  __device__ static float val(const HopParams& h, int i) { return h.valf[i]; }
  __device__ static float U(const HopParams& h, int i) { return h.Uf[i]; }
};

struct BlockShared {
  double red[3][32];
  double bcast[4];
};

__device__ __forceinline__ void bred3(double& a, double& b, double& c, BlockShared& sh) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) {
    sh.red[0][w] = a;
    sh.red[1][w] = b;
    sh.red[2][w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0, y = 0, z = 0;
    for (int i = 0; i < nw; ++i) {
      x += sh.red[0][i];
      y += sh.red[1][i];
      z += sh.red[2][i];
    }
    sh.bcast[0] = x;
    sh.bcast[1] = y;
    sh.bcast[2] = z;
  }
  __syncthreads();
  a = sh.bcast[0];
  b = sh.bcast[1];
  c = sh.bcast[2];
}

// Per-thread partial sums of <x,w>, <w,w>, <x,x>: FP64 for FP64 vectors; compensated (Kahan) FP32
// for FP32 vectors, so no per-element FP64 arithmetic runs (FP64 is a small fraction of the FP32
// rate on this GPU); the block sums them in FP64.
template <typename T>
struct BPart3;
template <>
struct BPart3<double> {
  double s[3] = {0.0, 0.0, 0.0};
  __device__ void add(double x, double w) {
    s[0] += x * w;
    s[1] += w * w;
    s[2] += x * x;
  }
  __device__ double get(int i) const { return s[i]; }
};
template <>
struct BPart3<float> {
  float s[3] = {0.f, 0.f, 0.f}, k[3] = {0.f, 0.f, 0.f};
  __device__ void add1(int i, float v) {
    const float y = v - k[i];
    const float t = s[i] + y;
    k[i] = (t - s[i]) - y;
    s[i] = t;
  }
  __device__ void add(float x, float w) {
    add1(0, x * w);
    add1(1, w * w);
    add1(2, x * x);
  }
  __device__ double get(int i) const { return (double)s[i] - (double)k[i]; }
};

// W = H X - bcoef * W (in place; W may hold x_prev), with <x,w>, <w,w>, <x,x> returned to every
// thread.  mode 0: element-strided (consecutive threads take consecutive elements); mode 1: one
// warp per row (warp-uniform up-spin entries, lanes over the columns).
template <typename T>
__device__ void block_hx(const BTable& tu, const BTable& td, const T* sval, const T* sU, uint32_t umask, T u0, bool uni,
                         const T* X, T* W, T bcoef, int mode, double& sxw, double& sww, double& sxx, BlockShared& sh) {
  const int64_t du = tu.dim, dd = td.dim;
  const T* eu = BP<T>::e(tu);
  const T* ed = BP<T>::e(td);
  BPart3<T> part;
  auto element = [&](int64_t u, int64_t d) {
    const int64_t o = u * dd + d;
    const uint32_t bu = tu.basis[u], bd = td.basis[d];
    T diag = eu[u] + ed[d];
    uint32_t dbl = bu & bd & umask;
    if (uni) {  // the same U on every interacting orbital: one popcount
      diag += u0 * (T)__popc(dbl);
    } else {
      while (dbl) {
        diag += sU[__ffs(dbl) - 1];
        dbl &= dbl - 1u;
      }
    }
    const T x = X[o];
    T acc = diag * x;
    const T* xr = X + u * dd;
    const int nd = td.cnt[d];
    for (int k = 0; k < nd; ++k) {
      const uint32_t e = td.ell[(int64_t)k * dd + d];
      const T v = sval[ent_vidx(e)];
      acc += (ent_neg(e) ? -v : v) * xr[ent_col(e)];
    }
    const int nu = tu.cnt[u];
    for (int k = 0; k < nu; ++k) {
      const uint32_t e = tu.ell[(int64_t)k * du + u];
      const T v = sval[ent_vidx(e)];
      acc += (ent_neg(e) ? -v : v) * X[(int64_t)ent_col(e) * dd + d];
    }
    const T w = acc - bcoef * W[o];
    W[o] = w;
    part.add(x, w);
  };
  if (mode == 1 && dd >= 16) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t u = warp; u < du; u += nw)
      for (int64_t d = lane; d < dd; d += 32) element(u, d);
  } else {
    // element i = u dd + d, stepped by blockDim.x without a division per element
    const int64_t su = blockDim.x / dd, sd = blockDim.x - su * dd;
    int64_t u = threadIdx.x / dd, d = threadIdx.x - u * dd;
    for (; u < du; u += su, d += sd) {
      if (d >= dd) {
        d -= dd;
        ++u;
        if (u >= du) break;
      }
      element(u, d);
    }
  }
  double a = part.get(0), b = part.get(1), c = part.get(2);
  bred3(a, b, c, sh);
  sxw = a;
  sww = b;
  sxx = c;
}

// Four vectors of one sector interleaved element by element (x[4 o + q] is vector q's element o):
// the continued fractions of one (cluster, spin, part) advance together, so every table entry and
// every gather serves four runs.
template <typename T>
struct alignas(4 * sizeof(T)) Q4 {
  T v[4];
};

// W4 = H X4 - bcoef[q] W4 (in place) for four interleaved vectors, with the per-vector partial sums
// of <x,w>, <w,w>, <x,x> reduced over the block into out[3 q + i].
template <typename T>
__device__ void block_hx4(const BTable& tu, const BTable& td, const T* sval, const T* sU, uint32_t umask, T u0, bool uni,
                          const Q4<T>* X, Q4<T>* W, const T (&bcoef)[4], int mode, double (&out)[12],
                          double (*red)[32], double* bcast) {
  const int64_t du = tu.dim, dd = td.dim;
  const T* eu = BP<T>::e(tu);
  const T* ed = BP<T>::e(td);
  BPart3<T> part[4];
  auto element = [&](int64_t u, int64_t d) {
    const int64_t o = u * dd + d;
    const uint32_t bu = tu.basis[u], bd = td.basis[d];
    T diag = eu[u] + ed[d];
    uint32_t dbl = bu & bd & umask;
    if (uni) {
      diag += u0 * (T)__popc(dbl);
    } else {
      while (dbl) {
        diag += sU[__ffs(dbl) - 1];
        dbl &= dbl - 1u;
      }
    }
    const Q4<T> x = X[o];
    T acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = diag * x.v[q];
    const Q4<T>* xr = X + u * dd;
    const int nd = td.cnt[d];
    for (int k = 0; k < nd; ++k) {
      const uint32_t e = td.ell[(int64_t)k * dd + d];
      const T v = ent_neg(e) ? -sval[ent_vidx(e)] : sval[ent_vidx(e)];
      const Q4<T> g = xr[ent_col(e)];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += v * g.v[q];
    }
    const int nu = tu.cnt[u];
    for (int k = 0; k < nu; ++k) {
      const uint32_t e = tu.ell[(int64_t)k * du + u];
      const T v = ent_neg(e) ? -sval[ent_vidx(e)] : sval[ent_vidx(e)];
      const Q4<T> g = X[(int64_t)ent_col(e) * dd + d];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += v * g.v[q];
    }
    Q4<T> w = W[o];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      w.v[q] = acc[q] - bcoef[q] * w.v[q];
      part[q].add(x.v[q], w.v[q]);
    }
    W[o] = w;
  };
  if (mode == 1 && dd >= 16) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t u = warp; u < du; u += nw)
      for (int64_t d = lane; d < dd; d += 32) element(u, d);
  } else {
    const int64_t su = blockDim.x / dd, sd = blockDim.x - su * dd;
    int64_t u = threadIdx.x / dd, d = threadIdx.x - u * dd;
    for (; u < du; u += su, d += sd) {
      if (d >= dd) {
        d -= dd;
        ++u;
        if (u >= du) break;
      }
      element(u, d);
    }
  }
  // block sums of the twelve partials (fixed order: warps in order, then one thread)
  double v[12];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int i = 0; i < 3; ++i) v[3 * q + i] = part[q].get(i);
#pragma unroll
  for (int i = 0; i < 12; ++i)
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  const int wi = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int i = 0; i < 12; ++i) red[i][wi] = v[i];
  __syncthreads();
  if (threadIdx.x < 12) {
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += red[threadIdx.x][k];
    bcast[threadIdx.x] = s;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 12; ++i) out[i] = bcast[i];
}

__device__ __forceinline__ uint64_t b_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct GSShared {
  BlockShared bs;
  double alpha[kBMaxIter + 2];
  double beta[kBMaxIter + 2];
  double svec[2 * (kBMaxIter + 2)];
  double eval[4];
  float svalf[kMaxVals];
  double svald[kMaxVals];
  float sUf[kMaxOrb];
  double sUd[kMaxOrb];
  int flag;
};

// Hopping values and U of the block's cluster in the precision of the vectors.
template <typename T, typename S>
__device__ __forceinline__ const T* sval_of(const S& g) {
  if constexpr (sizeof(T) == 8)
    return g.svald;
  else
    return g.svalf;
}
template <typename T, typename S>
__device__ __forceinline__ const T* sU_of(const S& g) {
  if constexpr (sizeof(T) == 8)
    return g.sUd;
  else
    return g.sUf;
}

// One Lanczos pass set (first pass + retrace) from the normalized start Vs; the ground state
// accumulates in omega (FP64).  Returns the levels used; eval[0..2] = lowest, second, Ritz.
template <typename T>
__device__ int block_lanczos(const BTable& tu, const BTable& td, uint32_t umask, double u0, bool uni, GSShared& g, T* V0, T* V1,
                             const T* Vs, double* omega, double tol_ritz, int mode, bool* breakdown) {
  const int64_t n = tu.dim * td.dim;
  const T* sval = sval_of<T>(g);
  const T* sU = sU_of<T>(g);
  int m = 0;
  *breakdown = false;
  for (int pass = 0; pass < 2; ++pass) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      V0[i] = Vs[i];
      V1[i] = T(0);
      if (pass == 1) omega[i] = g.svec[0] * (double)Vs[i];
    }
    if (threadIdx.x == 0) g.beta[0] = 0.0;
    __syncthreads();
    T* X = V0;
    T* P = V1;
    const int nmax = pass == 0 ? kBMaxIter : m - 1;
    for (int k = 0; k < nmax; ++k) {
      double sxw, sww, sxx;
      block_hx<T>(tu, td, sval, sU, umask, (T)u0, uni, X, P, (T)g.beta[k], mode, sxw, sww, sxx, g.bs);
      const double alpha = sxx > 0.0 ? sxw / sxx : 0.0;
      const double b2 = sxx > 0.0 ? sww - sxw * sxw / sxx : 0.0;
      const double bn = b2 > 0.0 ? sqrt(b2) : 0.0;
      if (threadIdx.x == 0) {
        g.alpha[k] = alpha;
        g.beta[k + 1] = bn;
      }
      const bool stop_here = !(bn > 1e-13);
      if (!stop_here) {
        const T aT = (T)alpha, ibT = (T)(1.0 / bn);
        const double cf = pass == 1 ? g.svec[k + 1] : 0.0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
          const T v = (P[i] - aT * X[i]) * ibT;
          P[i] = v;
          if (pass == 1) omega[i] += cf * (double)v;
        }
      }
      __syncthreads();
      T* t = X;
      X = P;
      P = t;
      if (pass == 0 && (stop_here || (k + 1) % kBCheck == 0 || k + 1 == kBMaxIter)) {
        const int levels = k + 1;
        tridiag_lowest_block(g.alpha, g.beta, levels, g.eval, g.svec);
        __syncthreads();
        m = levels;
        if (stop_here) {
          *breakdown = true;
          break;
        }
        if (g.eval[2] < tol_ritz * fmax(1.0, fabs(g.eval[0]))) break;
      }
      if (stop_here) break;
    }
  }
  return m;
}

template <typename T>
__device__ void block_ground_state(BCluster& c, const BTable* tabs, GSShared& g, T* V0, T* V1, T* Vs, double* Y64,
                                   double* Vd0, double* Vd1, double* Vds, int mode) {
  const BTable tu = tabs[c.t_up], td = tabs[c.t_dn];
  const int64_t n = c.d;
  double* om = c.omega;
  const uint32_t umask = c.hp.umask;
  int total = 0;
  bool fp64 = sizeof(T) == 8;
  double E = 0.0, res = 0.0, lam0 = 0.0, lam1 = 0.0;
  bool ok = false;
  for (int attempt = 0; attempt < 5 && !ok; ++attempt) {
    double s2 = 0.0, dummy1 = 0.0, dummy2 = 0.0;
    bool brk = false;
    int m;
    if (!fp64) {
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double r = (double)(b_splitmix64(c.seed ^ (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
        Vs[i] = attempt == 0 ? (T)(2.0 * r - 1.0) : (T)om[i];
        s2 += (double)Vs[i] * (double)Vs[i];
      }
      bred3(s2, dummy1, dummy2, g.bs);
      const T f = (T)(1.0 / sqrt(s2));
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) Vs[i] *= f;
      __syncthreads();
      m = block_lanczos<T>(tu, td, umask, c.hp.u0, c.hp.uniform_u != 0, g, V0, V1, Vs, om, 1e-7, mode, &brk);
    } else {
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double r = (double)(b_splitmix64(c.seed ^ (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
        Vds[i] = attempt == 0 && sizeof(T) == 8 ? 2.0 * r - 1.0 : om[i];
        s2 += Vds[i] * Vds[i];
      }
      bred3(s2, dummy1, dummy2, g.bs);
      const double f = 1.0 / sqrt(s2);
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) Vds[i] *= f;
      __syncthreads();
      m = block_lanczos<double>(tu, td, umask, c.hp.u0, c.hp.uniform_u != 0, g, Vd0, Vd1, Vds, om,
                                fmin(1e-2, 0.1 * c.tol), mode, &brk);
    }
    total += m;
    lam0 = g.eval[0];
    lam1 = g.eval[1];
    // FP64 polish: normalize, Rayleigh quotient, explicit residual
    double nn = 0.0, z1 = 0.0, z2 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) nn += om[i] * om[i];
    bred3(nn, z1, z2, g.bs);
    const double f = 1.0 / sqrt(nn);
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      om[i] *= f;
      Y64[i] = 0.0;
    }
    __syncthreads();
    double sxw, sww, sxx;
    block_hx<double>(tu, td, g.svald, g.sUd, umask, c.hp.u0, c.hp.uniform_u != 0, om, Y64, 0.0, mode, sxw, sww, sxx,
                     g.bs);
    E = sxw;
    double r2 = 0.0, q1 = 0.0, q2 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const double rr = Y64[i] - E * om[i];
      r2 += rr * rr;
    }
    bred3(r2, q1, q2, g.bs);
    res = sqrt(fmax(r2, 0.0));
    const double scale = fmax(1.0, fabs(E));
    if (fp64 || c.precision == ED_FP64)
      ok = res / scale <= c.tol || brk;
    else
      ok = (lam1 - E) > 0.0 && res * res / (lam1 - E) <= 1e-11 * scale;
    if (!ok) fp64 = true;  // refine in FP64 from the current state
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    c.E0 = E;
    c.residual = res / fmax(1.0, fabs(E));
    c.iters = total;
    c.gap = lam1 - lam0;
    c.status = !ok ? ED_WARN_NOT_CONVERGED : ((lam1 - lam0) < 1e-8 * fmax(1.0, fabs(lam0)) ? ED_WARN_DEGENERATE : ED_OK);
  }
  __syncthreads();
}

struct BWork {
  char* base;          // per-block workspace
  int64_t stride;      // bytes per block
  int64_t maxd;
  int64_t wmax;        // elements per vector of a warp's slice (warp-level runs)
};

// Runs of at most this many states are done by one warp each (no block barriers per level and
// four to sixteen runs per block at once); larger ones by a whole block.
constexpr int64_t kWarpRunMax = 8192;

template <typename T>
__global__ void k_batch_gs(BCluster* __restrict__ C, const int* __restrict__ order, int n, const BTable* __restrict__ tabs,
                           int* __restrict__ queue, BWork w, int mode) {
  __shared__ GSShared g;
  char* ws = w.base + (int64_t)blockIdx.x * w.stride;
  const int64_t md = w.maxd;
  T* V0 = (T*)ws;
  T* V1 = V0 + md;
  T* Vs = V1 + md;
  double* Y64 = (double*)(ws + ((3 * md * sizeof(T) + 255) / 256) * 256);
  double* Vd0 = Y64 + md;
  double* Vd1 = Vd0 + md;
  double* Vds = Vd1 + md;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) g.flag = atomicAdd(queue, 1);
    __syncthreads();
    const int item = g.flag;
    if (item >= n) return;
    BCluster& c = C[order[item]];
    for (int i = threadIdx.x; i < kMaxVals; i += blockDim.x) {
      g.svalf[i] = c.hp.valf[i];
      g.svald[i] = c.hp.val[i];
    }
    for (int i = threadIdx.x; i < kMaxOrb; i += blockDim.x) {
      g.sUf[i] = c.hp.Uf[i];
      g.sUd[i] = c.hp.U[i];
    }
    __syncthreads();
    block_ground_state<T>(c, tabs, g, V0, V1, Vs, Y64, Vd0, Vd1, Vds, mode);
  }
}

// -------------------------------------------------------------------------------- continued fractions
struct CFShared {
  BlockShared bs;
  double2 prev[4][64];
  double red12[12][32];
  double bcast12[12];
  double maxdiff;
  float svalf[kMaxVals];
  double svald[kMaxVals];
  float sUf[kMaxOrb];
  double sUd[kMaxOrb];
  int flag;
};

__device__ __forceinline__ double2 b_cf_eval(const double* __restrict__ a, const double* __restrict__ b, int m,
                                             double b0sq, double2 z, double E0, double s) {
  if (m <= 0) return make_double2(0.0, 0.0);
  double dr = z.x + s * (a[m - 1] - E0), di = z.y;
  for (int k = m - 2; k >= 0; --k) {
    const double bb = b[k + 1];
    const double q = bb * bb / (dr * dr + di * di);
    dr = z.x + s * (a[k] - E0) - q * dr;
    di = z.y + q * di;
  }
  const double q = b0sq / (dr * dr + di * di);
  return make_double2(q * dr, -q * di);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// W = H X - bcoef W over a sector by one warp (lanes over elements, fixed butterfly sums), with
// <x,w>, <w,w>, <x,x> returned to every lane.  Hopping values and U come from the cluster's
// parameters in global memory (cached).
template <typename T>
__device__ void warp_hx(const BTable& tu, const BTable& td, const HopParams& hp, const T* X, T* W, T bcoef,
                        double& sxw, double& sww, double& sxx) {
  const int lane = threadIdx.x & 31;
  const int64_t du = tu.dim, dd = td.dim;
  const T* eu = BP<T>::e(tu);
  const T* ed = BP<T>::e(td);
  const T u0 = (T)hp.u0;
  const bool uni = hp.uniform_u != 0;
  const uint32_t umask = hp.umask;
  BPart3<T> part;
  const int64_t su = 32 / dd, sd = 32 - su * dd;
  int64_t u = lane / dd, d = lane - u * dd;
  for (; u < du; u += su, d += sd) {
    if (d >= dd) {
      d -= dd;
      ++u;
      if (u >= du) break;
    }
    const int64_t o = u * dd + d;
    const uint32_t bu = tu.basis[u], bd = td.basis[d];
    T diag = eu[u] + ed[d];
    uint32_t dbl = bu & bd & umask;
    if (uni) {
      diag += u0 * (T)__popc(dbl);
    } else {
      while (dbl) {
        diag += BP<T>::U(hp, __ffs(dbl) - 1);
        dbl &= dbl - 1u;
      }
    }
    const T x = X[o];
    T acc = diag * x;
    const T* xr = X + u * dd;
    const int nd = td.cnt[d];
    for (int k = 0; k < nd; ++k) {
      const uint32_t e = td.ell[(int64_t)k * dd + d];
      const T v = BP<T>::val(hp, ent_vidx(e));
      acc += (ent_neg(e) ? -v : v) * xr[ent_col(e)];
    }
    const int nu = tu.cnt[u];
    for (int k = 0; k < nu; ++k) {
      const uint32_t e = tu.ell[(int64_t)k * du + u];
      const T v = BP<T>::val(hp, ent_vidx(e));
      acc += (ent_neg(e) ? -v : v) * X[(int64_t)ent_col(e) * dd + d];
    }
    const T w = acc - bcoef * W[o];
    W[o] = w;
    part.add(x, w);
  }
  sxw = warp_sum(part.get(0));
  sww = warp_sum(part.get(1));
  sxx = warp_sum(part.get(2));
}

// One continued fraction run by one warp: the same steps, check schedule and stopping rule as
// the block-level run of k_batch_cf.
template <typename T>
__device__ void warp_cf_run(BRun& r, const BCluster& c, const BTable* tabs, T* V0, T* V1, const double2* z, int nz,
                            double tol) {
  const int lane = threadIdx.x & 31;
  const int zstride = max(1, (nz + 63) / 64);
  const int nzs = (nz + zstride - 1) / zstride;
  const BTable tu = tabs[r.tu], td = tabs[r.td], src = tabs[r.src];
  const BTable dst = r.spin == 0 ? tu : td;
  const int64_t dd = td.dim, nel = r.d;
  const int64_t dd_s = tabs[c.t_dn].dim;
  const uint32_t lomask = (1u << src.split) - 1u;
  const int create = r.part == 0;
  const int extra = r.spin == 1 ? (c.n_up & 1) : 0;
  double s2 = 0.0;
  for (int64_t idx = lane; idx < nel; idx += 32) {
    const int64_t u = idx / dd, d = idx - u * dd;
    const uint32_t bt = r.spin == 0 ? dst.basis[u] : dst.basis[d];
    double acc = 0.0;
    for (int k = 0; k < 2; ++k) {
      const int site = k == 0 ? r.i : r.j;
      if (site < 0) continue;
      const uint32_t bit = 1u << site;
      if (create ? !(bt & bit) : (bt & bit)) continue;
      const uint32_t sb = bt ^ bit;
      const int64_t rr = src.rank_lo[sb & lomask] + src.rank_hi[sb >> src.split];
      const int neg = (__popc(bt & (bit - 1u)) + extra) & 1;
      const double v = r.spin == 0 ? c.omega[rr * dd_s + d] : c.omega[u * dd_s + rr];
      acc += neg ? -v : v;
    }
    V0[idx] = (T)acc;
    V1[idx] = T(0);
    s2 += acc * acc;
  }
  s2 = warp_sum(s2);
  int steps = 0;
  if (s2 > 1e-28) {
    const T f = (T)(1.0 / sqrt(s2));
    for (int64_t idx = lane; idx < nel; idx += 32) V0[idx] *= f;
    __syncwarp();
    T* X = V0;
    T* P = V1;
    double bprev = 0.0;
    int next_check = 32, hits = 0;
    const double sgn = create ? -1.0 : 1.0;
    double2 prev0 = make_double2(0.0, 0.0), prev1 = make_double2(0.0, 0.0);  // check frequencies lane, lane + 32
    for (int k = 0; k < r.mmax; ++k) {
      double sxw, sww, sxx;
      warp_hx<T>(tu, td, c.hp, X, P, (T)bprev, sxw, sww, sxx);
      const double alpha = sxx > 0.0 ? sxw / sxx : 0.0;
      const double b2 = sxx > 0.0 ? sww - sxw * sxw / sxx : 0.0;
      const double bn = b2 > 0.0 ? sqrt(b2) : 0.0;
      if (lane == 0) {
        r.alpha[k] = alpha;
        r.beta[k + 1] = bn;
      }
      steps = k + 1;
      if (!(bn > 1e-10)) break;
      const T aT = (T)alpha, ibT = (T)(1.0 / bn);
      for (int64_t idx = lane; idx < nel; idx += 32) P[idx] = (P[idx] - aT * X[idx]) * ibT;
      bprev = bn;
      T* t = X;
      X = P;
      P = t;
      __syncwarp();
      if (steps == next_check) {
        double mx = 0.0;
        if (lane < nzs) {
          const double2 gv = b_cf_eval(r.alpha, r.beta, steps, s2, z[lane * zstride], c.E0, sgn);
          mx = fmax(mx, hypot(gv.x - prev0.x, gv.y - prev0.y));
          prev0 = gv;
        }
        if (lane + 32 < nzs) {
          const double2 gv = b_cf_eval(r.alpha, r.beta, steps, s2, z[(lane + 32) * zstride], c.E0, sgn);
          mx = fmax(mx, hypot(gv.x - prev1.x, gv.y - prev1.y));
          prev1 = gv;
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        hits = mx < tol ? hits + 1 : 0;
        if (hits >= 2) break;
        next_check = steps + max(32, steps / 8);
      }
    }
  }
  if (lane == 0) {
    r.b0sq = s2;
    r.nsteps = steps;
  }
  __syncwarp();
}

// Runs order[0, n_block) (the larger ones, largest first) are taken by whole blocks from
// queue[0]; once those are gone, every warp takes runs order[n_block, n) from queue[1] and does
// each alone in its slice of the block's workspace.
template <typename T>
__global__ void __launch_bounds__(512) k_batch_cf(BRun* __restrict__ R, const int* __restrict__ order, int n_block, int n,
                           const int4* __restrict__ groups, int n_groups, const BCluster* __restrict__ C,
                           const BTable* __restrict__ tabs, int* __restrict__ queue, BWork w,
                           const double2* __restrict__ z, int nz, double tol, int mode) {
  __shared__ CFShared g;
  char* ws = w.base + (int64_t)blockIdx.x * w.stride;
  const int zstride = max(1, (nz + 63) / 64);  // at most 64 check frequencies (g.prev)
  const int nzs = (nz + zstride - 1) / zstride;
  // block phase: groups of up to four runs of one (cluster, spin, part), interleaved
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) g.flag = atomicAdd(queue, 1);
    __syncthreads();
    const int item = g.flag;
    if (item >= n_groups) break;
    const int4 gi = groups[item];
    const int rid[4] = {gi.x, gi.y, gi.z, gi.w};
    int m = 0;
    while (m < 4 && rid[m] >= 0) ++m;
    const BRun& r0 = R[rid[0]];
    const BCluster& c = C[r0.cluster];
    for (int i = threadIdx.x; i < kMaxVals; i += blockDim.x) {
      g.svalf[i] = c.hp.valf[i];
      g.svald[i] = c.hp.val[i];
    }
    for (int i = threadIdx.x; i < kMaxOrb; i += blockDim.x) {
      g.sUf[i] = c.hp.Uf[i];
      g.sUd[i] = c.hp.U[i];
    }
    for (int i = threadIdx.x; i < 4 * 64; i += blockDim.x) g.prev[i >> 6][i & 63] = make_double2(0.0, 0.0);
    const BTable tu = tabs[r0.tu], td = tabs[r0.td], src = tabs[r0.src];
    const BTable dst = r0.spin == 0 ? tu : td;
    const int64_t dd = td.dim, nel = r0.d;
    const int64_t dd_s = tabs[c.t_dn].dim;
    const uint32_t lomask = (1u << src.split) - 1u;
    const int create = r0.part == 0;
    const int extra = r0.spin == 1 ? (c.n_up & 1) : 0;
    int si[4], sj[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      si[q] = q < m ? R[rid[q]].i : -1;
      sj[q] = q < m ? R[rid[q]].j : -1;
    }
    Q4<T>* X = reinterpret_cast<Q4<T>*>(ws);
    Q4<T>* P = X + w.maxd;
    double s2[4] = {0.0, 0.0, 0.0, 0.0};
    __syncthreads();
    // phi_q = (c_i [+ c_j])^(+) Omega for every run q in the target sector (pull form, sign of
    // Eq. basis)
    for (int64_t idx = threadIdx.x; idx < nel; idx += blockDim.x) {
      const int64_t u = idx / dd, d = idx - u * dd;
      const uint32_t bt = r0.spin == 0 ? dst.basis[u] : dst.basis[d];
      Q4<T> ph;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double acc = 0.0;
        for (int k = 0; k < 2; ++k) {
          const int site = k == 0 ? si[q] : sj[q];
          if (site < 0) continue;
          const uint32_t bit = 1u << site;
          if (create ? !(bt & bit) : (bt & bit)) continue;
          const uint32_t sb = bt ^ bit;
          const int64_t rr = src.rank_lo[sb & lomask] + src.rank_hi[sb >> src.split];
          const int neg = (__popc(bt & (bit - 1u)) + extra) & 1;
          const double v = r0.spin == 0 ? c.omega[rr * dd_s + d] : c.omega[u * dd_s + rr];
          acc += neg ? -v : v;
        }
        ph.v[q] = (T)acc;
        s2[q] += acc * acc;
      }
      X[idx] = ph;
      P[idx] = Q4<T>{};
    }
    {
      double v4[4] = {s2[0], s2[1], s2[2], s2[3]};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        for (int o = 16; o > 0; o >>= 1) v4[q] += __shfl_down_sync(0xffffffffu, v4[q], o);
      const int wi = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
      __syncthreads();
      if (l == 0)
        for (int q = 0; q < 4; ++q) g.red12[q][wi] = v4[q];
      __syncthreads();
      if (threadIdx.x < 4) {
        double t = 0.0;
        for (int k = 0; k < nw; ++k) t += g.red12[threadIdx.x][k];
        g.bcast12[threadIdx.x] = t;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q) s2[q] = g.bcast12[q];
      __syncthreads();
    }
    bool active[4];
    int steps[4], next_check[4], hits[4];
    double bprev[4];
    T f[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      active[q] = q < m && s2[q] > 1e-28;
      f[q] = active[q] ? (T)(1.0 / sqrt(s2[q])) : T(0);
      steps[q] = 0;
      next_check[q] = 32;
      hits[q] = 0;
      bprev[q] = 0.0;
    }
    for (int64_t idx = threadIdx.x; idx < nel; idx += blockDim.x) {
      Q4<T> x = X[idx];
#pragma unroll
      for (int q = 0; q < 4; ++q) x.v[q] *= f[q];
      X[idx] = x;
    }
    __syncthreads();
    const double sgn = create ? -1.0 : 1.0;
    for (int k = 0; k < r0.mmax && (active[0] || active[1] || active[2] || active[3]); ++k) {
      T bc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) bc[q] = (T)bprev[q];
      double sums[12];
      block_hx4<T>(tu, td, sval_of<T>(g), sU_of<T>(g), c.hp.umask, (T)c.hp.u0, c.hp.uniform_u != 0, X, P, bc, mode,
                   sums, g.red12, g.bcast12);
      T aT[4], ibT[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        aT[q] = T(0);
        ibT[q] = T(0);
        if (!active[q]) continue;
        const double sxw = sums[3 * q], sww = sums[3 * q + 1], sxx = sums[3 * q + 2];
        const double alpha = sxx > 0.0 ? sxw / sxx : 0.0;
        const double b2 = sxx > 0.0 ? sww - sxw * sxw / sxx : 0.0;
        const double bn = b2 > 0.0 ? sqrt(b2) : 0.0;
        if (threadIdx.x == 0) {
          R[rid[q]].alpha[k] = alpha;
          R[rid[q]].beta[k + 1] = bn;
        }
        steps[q] = k + 1;
        if (!(bn > 1e-10)) {
          active[q] = false;
          bprev[q] = 0.0;
          continue;
        }
        aT[q] = (T)alpha;
        ibT[q] = (T)(1.0 / bn);
        bprev[q] = bn;
      }
      for (int64_t idx = threadIdx.x; idx < nel; idx += blockDim.x) {
        const Q4<T> x = X[idx];
        Q4<T> pv = P[idx];
#pragma unroll
        for (int q = 0; q < 4; ++q) pv.v[q] = (pv.v[q] - aT[q] * x.v[q]) * ibT[q];
        P[idx] = pv;
      }
      Q4<T>* t = X;
      X = P;
      P = t;
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (!active[q] || steps[q] != next_check[q]) continue;
        // the continued fraction of run q on every zstride-th frequency, against its last check
        if (threadIdx.x == 0) g.maxdiff = 0.0;
        __syncthreads();
        const BRun& rq = R[rid[q]];
        double mx = 0.0;
        for (int qq = threadIdx.x; qq < nzs; qq += blockDim.x) {
          const double2 gv = b_cf_eval(rq.alpha, rq.beta, steps[q], s2[q], z[qq * zstride], c.E0, sgn);
          mx = fmax(mx, hypot(gv.x - g.prev[q][qq].x, gv.y - g.prev[q][qq].y));
          g.prev[q][qq] = gv;
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long*)&g.maxdiff, __double_as_longlong(mx));
        __syncthreads();
        hits[q] = g.maxdiff < tol ? hits[q] + 1 : 0;
        if (hits[q] >= 2) active[q] = false;
        next_check[q] = steps[q] + max(32, steps[q] / 8);
        __syncthreads();
      }
    }
    if (threadIdx.x == 0)
      for (int q = 0; q < m; ++q) {
        R[rid[q]].b0sq = s2[q];
        R[rid[q]].nsteps = steps[q];
      }
    __syncthreads();
  }
  // warp phase
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* W0 = reinterpret_cast<T*>(ws) + (int64_t)warp * 2 * w.wmax;
  T* W1 = W0 + w.wmax;
  while (true) {
    int t = 0;
    if (lane == 0) t = atomicAdd(queue + 1, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    const int item = n_block + t;
    if (item >= n) return;
    BRun& r = R[order[item]];
    warp_cf_run<T>(r, C[r.cluster], tabs, W0, W1, z, nz, tol);
  }
}

// -------------------------------------------------------------------------------- evaluation on the grid
__global__ void k_bcf_eval(const BRun* __restrict__ R, int nruns, const BCluster* __restrict__ C,
                           const double2* __restrict__ z, int nz, double2* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nz) return;
  for (int q = blockIdx.y; q < nruns; q += gridDim.y) {  // grid.y is capped at 65535
    const BRun& r = R[q];
    out[(int64_t)q * nz + k] =
        b_cf_eval(r.alpha, r.beta, r.nsteps, r.b0sq, z[k], C[r.cluster].E0, r.part == 0 ? -1.0 : 1.0);
  }
}

// G[c][spin][z][i][j] from the runs: base[c][spin][part] = first run of that part (-1: absent).
__global__ void k_bcombine(const BCluster* __restrict__ C, int nclu, const int* __restrict__ base,
                           const int64_t* __restrict__ goff, const double2* __restrict__ Gk, int nz,
                           double2* __restrict__ G) {
  for (int c = blockIdx.y; c < nclu; c += gridDim.y) {  // grid.y is capped at 65535
    const int p = C[c].ns;
    const int64_t per = (int64_t)2 * nz * p * p;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < per; t += (int64_t)gridDim.x * blockDim.x) {
      const int spin = (int)(t / ((int64_t)nz * p * p));
      const int64_t rem = t - (int64_t)spin * nz * p * p;
      const int k = (int)(rem / (p * p));
      const int ij = (int)(rem - (int64_t)k * p * p);
      const int i = ij / p, j = ij - i * p;
      double2 g = make_double2(0.0, 0.0);
      for (int part = 0; part < 2; ++part) {
        const int b0 = base[(c * 2 + spin) * 2 + part];
        if (b0 < 0) continue;
        if (i == j) {
          const double2 v = Gk[(int64_t)(b0 + i) * nz + k];
          g.x += v.x;
          g.y += v.y;
        } else {
          const int lo = min(i, j), hi = max(i, j);
          const int rp = b0 + p + (lo * (2 * p - lo - 1)) / 2 + (hi - lo - 1);
          const double2 vp = Gk[(int64_t)rp * nz + k], vi = Gk[(int64_t)(b0 + lo) * nz + k],
                        vj = Gk[(int64_t)(b0 + hi) * nz + k];
          g.x += 0.5 * (vp.x - vi.x - vj.x);
          g.y += 0.5 * (vp.y - vi.y - vj.y);
        }
      }
      G[goff[c] + t] = g;
    }
  }
}

// -------------------------------------------------------------------------------- host driver
namespace {
struct Arena {
  DevBuf<char> buf;
  size_t used = 0;
  size_t take(size_t bytes) {
    const size_t off = used;
    used += (bytes + 255) / 256 * 256;
    return off;
  }
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune;  // (L_max, d bucket, n bucket, prec) -> (threads, mode)

BBinom make_bbinom() {
  BBinom b;
  std::memset(&b, 0, sizeof(b));
  for (int n = 0; n <= kMaxOrb; ++n) {
    b.c[n][0] = 1;
    for (int k = 1; k <= n; ++k) b.c[n][k] = b.c[n - 1][k - 1] + (k <= n - 1 ? b.c[n - 1][k] : 0);
  }
  return b;
}
}  // namespace

struct BatchResult {
  std::vector<double> E0, residual;
  std::vector<int> status, iters, gf_steps;
};

// Runs the persistent ground-state and continued-fraction kernels with `threads` per block.
// (prof: time each launch with the profiler; off while the launches are captured into a graph)
template <typename T>
static void run_batch_kernels(int threads, int mode, BCluster* C, const int* corder, int nclu, const BTable* tabs,
                              BRun* R, const int* rorder, int nblock_runs, int nruns, const int4* groups, int ngroups,
                              int* queues, const BWork& w, int blocks, const double2* z, int nz, double tol, bool do_gf,
                              cudaStream_t s, bool prof = true) {
  ED_CUDA(cudaMemsetAsync(queues, 0, 3 * sizeof(int), s));
  {
    std::unique_ptr<ProfScope> ps_(prof ? new ProfScope(K_BATCH, s, 0.0) : nullptr);
    k_batch_gs<T><<<blocks, threads, 0, s>>>(C, corder, nclu, tabs, queues, w, mode);
    ED_CHECK_LAUNCH();
  }
  if (do_gf && nruns > 0) {
    std::unique_ptr<ProfScope> ps_(prof ? new ProfScope(K_BATCH, s, 0.0) : nullptr);
    k_batch_cf<T><<<blocks, threads, 0, s>>>(R, rorder, nblock_runs, nruns, groups, ngroups, C, tabs, queues + 1, w, z,
                                             nz, tol, mode);
    ED_CHECK_LAUNCH();
  }
}

// Ends a stream capture left open by an exception (the stream is usable again afterwards).
struct CaptureGuard {
  cudaStream_t s;
  bool open = true;
  ~CaptureGuard() {
    if (!open) return;
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(s, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
  }
};
struct GraphHolder {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  ~GraphHolder() {
    if (x) cudaGraphExecDestroy(x);
    if (g) cudaGraphDestroy(g);
  }
};

// Device bytes batch_solve allocates for these clusters (tables, ground states, continued-fraction
// coefficients, evaluated fractions and the per-block workspace; the caller's G not included).
size_t batch_device_bytes(const ed_cluster_desc* descs, int n, int precision, int nz, int cf_max_steps, int sms) {
  auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
  const int cap = cf_max_steps > 0 ? cf_max_steps : 20000;
  const size_t es = precision == ED_FP64 ? 8 : 4;
  size_t bytes = 0;
  int64_t maxd = 1, nruns = 0;
  for (int c = 0; c < n; ++c) {
    const int L = descs[c].n_sites + descs[c].n_bath, p = descs[c].n_sites;
    const int nu = descs[c].n_up, nd = descs[c].n_dn;
    std::map<int, int64_t> dims;
    auto table = [&](int N) {
      if (N < 0 || N > L || dims.count(N)) return;
      const int64_t d = (int64_t)binomial(L, N);
      dims[N] = d;
      const int split = L / 2, zmax = std::max(1, N * (L - N));
      bytes += r256(d * 4) + r256((size_t(1) << split) * 4) + r256((size_t(1) << (L - split)) * 4) +
               r256((size_t)zmax * d * 4) + r256(d) + r256(d * 8) + r256(d * 4);
    };
    table(nu);
    table(nd);
    const int64_t d = dims[nu] * dims[nd];
    maxd = std::max(maxd, d);
    bytes += r256(d * 8);
    if (nz <= 0) continue;
    for (int dn : {1, -1}) {
      table(nu + dn);
      if (nu != nd) table(nd + dn);
    }
    for (int spin = 0; spin < (nu != nd ? 2 : 1); ++spin)
      for (int dn : {1, -1}) {
        const int nt = (spin == 0 ? nu : nd) + dn;
        if (nt < 0 || nt > L) continue;
        const int64_t dt = (int64_t)binomial(L, nt) * (spin == 0 ? dims[nd] : dims[nu]);
        maxd = std::max(maxd, dt);
        const int64_t mmax = std::max<int64_t>(64, std::min<int64_t>(cap, 2 * dt + 16));
        const int runs = p + p * (p - 1) / 2;
        nruns += runs;
        bytes += (size_t)runs * (r256(mmax * 8) + r256((mmax + 1) * 8));
      }
  }
  bytes += r256((size_t)std::max<int64_t>(nruns, 1) * std::max(nz, 0) * 16);
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(n + nruns, (int64_t)sms * 4));
  const int64_t wmax = std::min<int64_t>(maxd, kWarpRunMax);
  const size_t stride = std::max<size_t>(std::max<size_t>(((3 * maxd * es + 255) / 256) * 256 + 4 * maxd * 8,
                                                          (size_t)16 * 2 * wmax * es),
                                         (size_t)8 * maxd * es) + 256;
  return bytes + (size_t)blocks * stride + (size_t(1) << 20);
}

void batch_solve(const ed_cluster_desc* descs, int n, int precision, const double2* z_host, int nz, bool do_gf,
                 int cf_max_steps, double* E0_out, double* res_out, int* status_out, int* iters_out,
                 int64_t* gf_steps_out, double2* G_dev_out, cudaStream_t s, int fixed_threads, int fixed_mode) {
  static const BBinom bn = make_bbinom();
  if (n <= 0) return;
  // ---- models
  std::vector<ModelHost> models(n);
  std::vector<BCluster> C(n);
  for (int c = 0; c < n; ++c) {
    std::memset(&C[c], 0, sizeof(BCluster));
    build_model(&descs[c], models[c], C[c].hp);
    if (models[c].L > kBMaxL) throw Error(ED_ERR_INVALID, "batched clusters have at most 20 orbitals");
    C[c].ns = models[c].ns;
    C[c].L = models[c].L;
    C[c].n_up = descs[c].n_up;
    C[c].n_dn = descs[c].n_dn;
    C[c].seed = descs[c].seed;
    C[c].tol = descs[c].tol > 0 ? descs[c].tol : 1e-12;
    C[c].precision = precision;
    if (C[c].ns > 32) throw Error(ED_ERR_INVALID, "too many cluster sites");
  }
  // ---- tables: one per (cluster, particle number) needed
  std::vector<BTable> T;
  std::vector<size_t> off_basis, off_lo, off_hi, off_ell, off_cnt, off_e64, off_e32;
  Arena tab;
  std::vector<std::map<int, int>> tindex(n);
  auto need = [&](int c, int N) -> int {
    if (N < 0 || N > C[c].L) return -1;
    auto it = tindex[c].find(N);
    if (it != tindex[c].end()) return it->second;
    BTable t;
    std::memset(&t, 0, sizeof(t));
    t.L = C[c].L;
    t.N = N;
    t.split = t.L / 2;
    t.dim = (int64_t)binomial(t.L, N);
    t.zmax = std::max(1, N * (t.L - N));
    t.cluster = c;
    off_basis.push_back(tab.take(t.dim * 4));
    off_lo.push_back(tab.take((size_t(1) << t.split) * 4));
    off_hi.push_back(tab.take((size_t(1) << (t.L - t.split)) * 4));
    off_ell.push_back(tab.take((size_t)t.zmax * t.dim * 4));
    off_cnt.push_back(tab.take(t.dim));
    off_e64.push_back(tab.take(t.dim * 8));
    off_e32.push_back(tab.take(t.dim * 4));
    T.push_back(t);
    tindex[c][N] = (int)T.size() - 1;
    return (int)T.size() - 1;
  };
  for (int c = 0; c < n; ++c) {
    C[c].t_up = need(c, C[c].n_up);
    C[c].t_dn = need(c, C[c].n_dn);
    C[c].d = T[C[c].t_up].dim * T[C[c].t_dn].dim;
    C[c].t_upp = do_gf ? need(c, C[c].n_up + 1) : -1;
    C[c].t_upm = do_gf ? need(c, C[c].n_up - 1) : -1;
    const bool both = C[c].n_up != C[c].n_dn;
    C[c].t_dnp = do_gf && both ? need(c, C[c].n_dn + 1) : -1;
    C[c].t_dnm = do_gf && both ? need(c, C[c].n_dn - 1) : -1;
  }
  // ---- runs
  const int cap = cf_max_steps > 0 ? cf_max_steps : 20000;
  std::vector<BRun> R;
  std::vector<int> base((size_t)n * 4, -1);
  for (int c = 0; c < n && do_gf; ++c) {
    const int p = C[c].ns;
    const int nspin = C[c].n_up != C[c].n_dn ? 2 : 1;
    for (int spin = 0; spin < nspin; ++spin)
      for (int part = 0; part < 2; ++part) {
        const int tgt = spin == 0 ? (part == 0 ? C[c].t_upp : C[c].t_upm) : (part == 0 ? C[c].t_dnp : C[c].t_dnm);
        if (tgt < 0) continue;
        base[(c * 2 + spin) * 2 + part] = (int)R.size();
        for (int q = 0; q < p + p * (p - 1) / 2; ++q) {
          BRun r;
          std::memset(&r, 0, sizeof(r));
          r.cluster = c;
          r.spin = spin;
          r.part = part;
          if (q < p) {
            r.i = q;
            r.j = -1;
          } else {
            int k = q - p, i = 0;
            while (k >= p - 1 - i) {
              k -= p - 1 - i;
              ++i;
            }
            r.i = i;
            r.j = i + 1 + k;
          }
          r.tu = spin == 0 ? tgt : C[c].t_up;
          r.td = spin == 0 ? C[c].t_dn : tgt;
          r.src = spin == 0 ? C[c].t_up : C[c].t_dn;
          r.d = T[r.tu].dim * T[r.td].dim;
          r.mmax = (int)std::max<int64_t>(64, std::min<int64_t>(cap, 2 * r.d + 16));
          R.push_back(r);
        }
      }
    if (nspin == 1)
      for (int part = 0; part < 2; ++part) base[(c * 2 + 1) * 2 + part] = base[(c * 2 + 0) * 2 + part];
  }
  const int nruns = (int)R.size();
  // ---- arena: tables, ground states, run coefficients, G parts
  std::vector<size_t> off_om(n), off_al(nruns), off_be(nruns);
  for (int c = 0; c < n; ++c) off_om[c] = tab.take(C[c].d * 8);
  for (int r = 0; r < nruns; ++r) {
    off_al[r] = tab.take((size_t)R[r].mmax * 8);
    off_be[r] = tab.take((size_t)(R[r].mmax + 1) * 8);
  }
  const size_t off_gk = tab.take((size_t)std::max(nruns, 1) * nz * sizeof(double2));
  tab.buf.alloc(tab.used);
  char* B = tab.buf.p;
  for (size_t t = 0; t < T.size(); ++t) {
    T[t].basis = (uint32_t*)(B + off_basis[t]);
    T[t].rank_lo = (int32_t*)(B + off_lo[t]);
    T[t].rank_hi = (int32_t*)(B + off_hi[t]);
    T[t].ell = (uint32_t*)(B + off_ell[t]);
    T[t].cnt = (uint8_t*)(B + off_cnt[t]);
    T[t].e64 = (double*)(B + off_e64[t]);
    T[t].e32 = (float*)(B + off_e32[t]);
  }
  for (int c = 0; c < n; ++c) C[c].omega = (double*)(B + off_om[c]);
  for (int r = 0; r < nruns; ++r) {
    R[r].alpha = (double*)(B + off_al[r]);
    R[r].beta = (double*)(B + off_be[r]);
  }
  double2* Gk = (double2*)(B + off_gk);
  // pairs and diagonals
  std::vector<BPair> pairs;
  std::vector<int> pair_off(n + 1, 0);
  std::vector<double> hdiag((size_t)n * kMaxOrb, 0.0);
  for (int c = 0; c < n; ++c) {
    const ModelHost& m = models[c];
    for (size_t k = 0; k < m.pair_a.size(); ++k) {
      const uint32_t a = m.pair_a[k], b = m.pair_b[k];
      const uint32_t lo = std::min(a, b), hi = std::max(a, b);
      const uint32_t between = ((1u << hi) - 1u) ^ ((1u << (lo + 1)) - 1u);
      pairs.push_back(BPair{a, b, (uint32_t)m.pair_vidx[k], between});
    }
    pair_off[c + 1] = (int)pairs.size();
    for (int a = 0; a < m.L; ++a) hdiag[(size_t)c * kMaxOrb + a] = m.h[a * m.L + a];
  }
  // orders: largest first
  std::vector<int> corder(n), rorder(nruns);
  std::iota(corder.begin(), corder.end(), 0);
  std::stable_sort(corder.begin(), corder.end(), [&](int a, int b) { return C[a].d > C[b].d; });
  std::iota(rorder.begin(), rorder.end(), 0);
  std::stable_sort(rorder.begin(), rorder.end(), [&](int a, int b) { return R[a].d > R[b].d; });
  int nblock_runs = 0;  // runs done by whole blocks (the rest by single warps)
  while (nblock_runs < nruns && R[rorder[nblock_runs]].d > kWarpRunMax) ++nblock_runs;
  // block-level runs in groups of up to four of one (cluster, spin, part): one target sector,
  // advanced together (interleaved vectors); the largest-first order keeps each group contiguous
  std::vector<int4> grp;
  for (int i = 0; i < nblock_runs;) {
    int g4[4] = {-1, -1, -1, -1};
    const BRun& a = R[rorder[i]];
    for (int k = 0; k < 4 && i < nblock_runs; ++k) {
      const BRun& b = R[rorder[i]];
      if (k > 0 && (b.cluster != a.cluster || b.spin != a.spin || b.part != a.part)) break;
      g4[k] = rorder[i++];
    }
    grp.push_back(make_int4(g4[0], g4[1], g4[2], g4[3]));
  }
  const int ngroups = (int)grp.size();
  // ---- device descriptors
  DevBuf<BTable> dT(T.size());
  DevBuf<BPair> dP(std::max<size_t>(pairs.size(), 1));
  DevBuf<int> dPoff(n + 1), dCo(n), dRo(std::max(nruns, 1)), dQ(3), dBase((size_t)n * 4);
  DevBuf<double> dHd(hdiag.size());
  DevBuf<BCluster> dC(n);
  DevBuf<BRun> dR(std::max(nruns, 1));
  DevBuf<double2> dz(std::max(nz, 1));
  DevBuf<int4> dG(std::max(ngroups, 1));
  if (ngroups) ED_CUDA(cudaMemcpyAsync(dG.p, grp.data(), ngroups * sizeof(int4), cudaMemcpyHostToDevice, s));
  ED_CUDA(cudaMemcpyAsync(dT.p, T.data(), T.size() * sizeof(BTable), cudaMemcpyHostToDevice, s));
  if (!pairs.empty()) ED_CUDA(cudaMemcpyAsync(dP.p, pairs.data(), pairs.size() * sizeof(BPair), cudaMemcpyHostToDevice, s));
  ED_CUDA(cudaMemcpyAsync(dPoff.p, pair_off.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  ED_CUDA(cudaMemcpyAsync(dHd.p, hdiag.data(), hdiag.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  ED_CUDA(cudaMemcpyAsync(dC.p, C.data(), n * sizeof(BCluster), cudaMemcpyHostToDevice, s));
  ED_CUDA(cudaMemcpyAsync(dCo.p, corder.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  if (nruns) {
    ED_CUDA(cudaMemcpyAsync(dR.p, R.data(), nruns * sizeof(BRun), cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(dRo.p, rorder.data(), nruns * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  ED_CUDA(cudaMemcpyAsync(dBase.p, base.data(), base.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  if (nz) ED_CUDA(cudaMemcpyAsync(dz.p, z_host, nz * sizeof(double2), cudaMemcpyHostToDevice, s));
  // ---- tables
  int64_t maxdim = 0;
  for (const BTable& t : T) maxdim = std::max<int64_t>(maxdim, std::max<int64_t>(t.dim, int64_t(1) << (t.L - t.split)));
  {
    const unsigned gx = (unsigned)std::min<int64_t>((maxdim + 255) / 256, 64);
    ProfScope ps_(K_TABLES, s, 0.0);
    k_bt_basis<<<dim3(gx, (unsigned)T.size()), 256, 0, s>>>(dT.p, bn);
    ED_CHECK_LAUNCH();
  }
  {
    const unsigned gx = (unsigned)std::min<int64_t>((maxdim + 255) / 256, 64);
    ProfScope ps_(K_TABLES, s, 0.0);
    k_bt_fill<<<dim3(gx, (unsigned)T.size()), 256, 0, s>>>(dT.p, dP.p, dPoff.p, dHd.p);
    ED_CHECK_LAUNCH();
  }
  // ---- workspace: per persistent block, 3 + 4 vectors of the largest sector
  int64_t maxd = 1;
  for (int c = 0; c < n; ++c) maxd = std::max(maxd, C[c].d);
  for (int r = 0; r < nruns; ++r) maxd = std::max(maxd, R[r].d);
  const size_t es = precision == ED_FP64 ? 8 : 4;
  // per block: 3 + 4 vectors of the largest sector, or 2 vectors per warp (at most 16) of the
  // largest warp-level run, whichever is more
  const int64_t wmax = std::min<int64_t>(maxd, kWarpRunMax);
  // (or two sets of four interleaved vectors of a group of block-level continued fractions)
  const size_t stride = std::max<size_t>(std::max<size_t>(((3 * maxd * es + 255) / 256) * 256 + 4 * maxd * 8,
                                                          (size_t)16 * 2 * wmax * es),
                                         (size_t)8 * maxd * es) + 256;
  int dev = 0, sms = 0;
  ED_CUDA(cudaGetDevice(&dev));
  ED_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // autotuned block width and mapping (cached per batch shape)
  int Lmax = 0;
  for (int c = 0; c < n; ++c) Lmax = std::max(Lmax, C[c].L);
  int dbucket = 0;
  while ((int64_t(1) << (2 * dbucket)) < maxd) ++dbucket;
  int nbucket = 0;
  while ((1 << nbucket) < n) ++nbucket;
  const auto key = std::make_tuple(Lmax, dbucket, nbucket, precision);
  std::pair<int, int> cfg{256, 0};
  bool tuned = fixed_threads > 0;
  if (tuned) {
    cfg = {fixed_threads, fixed_mode};
  } else {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    tuned = it != g_tune.end();
    if (tuned) cfg = it->second;
  }
  const int per_sm = 4;
  const int blocks = std::max(1, std::min(n + nruns, sms * per_sm));
  DevBuf<char> work((size_t)blocks * stride);
  BWork w{work.p, (int64_t)stride, maxd, wmax};
  if (!tuned) {
    // time the ground-state kernel of the largest clusters with each candidate
    const int sample = std::min(n, std::max(8, blocks));
    const std::pair<int, int> cands[] = {{128, 0}, {256, 0}, {256, 1}, {512, 1}};
    float best = 1e30f;
    cudaEvent_t e0, e1;
    ED_CUDA(cudaEventCreate(&e0));
    ED_CUDA(cudaEventCreate(&e1));
    for (const auto& cd : cands) {
      ED_CUDA(cudaMemcpyAsync(dC.p, C.data(), n * sizeof(BCluster), cudaMemcpyHostToDevice, s));
      ED_CUDA(cudaEventRecord(e0, s));
      if (precision == ED_FP64)
        run_batch_kernels<double>(cd.first, cd.second, dC.p, dCo.p, sample, dT.p, dR.p, dRo.p, 0, 0, nullptr, 0, dQ.p, w, blocks,
                                  dz.p, nz, 0.0, false, s);
      else
        run_batch_kernels<float>(cd.first, cd.second, dC.p, dCo.p, sample, dT.p, dR.p, dRo.p, 0, 0, nullptr, 0, dQ.p, w, blocks,
                                 dz.p, nz, 0.0, false, s);
      ED_CUDA(cudaEventRecord(e1, s));
      ED_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      ED_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        cfg = cd;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ED_CUDA(cudaMemcpyAsync(dC.p, C.data(), n * sizeof(BCluster), cudaMemcpyHostToDevice, s));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = cfg;
  }
  const double gtol = precision == ED_FP64 ? 1e-10 : 1e-6;
  // The solve proper is one CUDA graph: queue reset, the persistent ground-state and
  // continued-fraction kernels, evaluation on the grid and assembly of G.
  std::vector<int64_t> goff(n + 1, 0);
  for (int c = 0; c < n; ++c) goff[c + 1] = goff[c] + (int64_t)2 * nz * C[c].ns * C[c].ns;
  DevBuf<int64_t> dgoff(n + 1);
  ED_CUDA(cudaMemcpyAsync(dgoff.p, goff.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  const bool gf = do_gf && nruns > 0;
  GraphHolder graph;
  {
    CaptureGuard cg{s};
    ED_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    if (precision == ED_FP64)
      run_batch_kernels<double>(cfg.first, cfg.second, dC.p, dCo.p, n, dT.p, dR.p, dRo.p, nblock_runs, nruns, dG.p, ngroups, dQ.p, w, blocks,
                                dz.p, nz, gtol, do_gf, s, false);
    else
      run_batch_kernels<float>(cfg.first, cfg.second, dC.p, dCo.p, n, dT.p, dR.p, dRo.p, nblock_runs, nruns, dG.p, ngroups, dQ.p, w, blocks,
                               dz.p, nz, gtol, do_gf, s, false);
    if (gf) {
      k_bcf_eval<<<dim3((nz + 255) / 256, std::min(nruns, 32768)), 256, 0, s>>>(dR.p, nruns, dC.p, dz.p, nz, Gk);
      ED_CHECK_LAUNCH();
      k_bcombine<<<dim3(64, std::min(n, 32768)), 256, 0, s>>>(dC.p, n, dBase.p, dgoff.p, Gk, nz, G_dev_out);
      ED_CHECK_LAUNCH();
    }
    cg.open = false;
    ED_CUDA(cudaStreamEndCapture(s, &graph.g));
  }
  ED_CUDA(cudaGraphInstantiate(&graph.x, graph.g, 0));
  {
    ProfScope ps_(K_BATCH, s, 0.0);  // counts the graph as one launch of the persistent kernels
    ED_CUDA(cudaGraphLaunch(graph.x, s));
  }
  for (int k = 0; k < (gf ? 3 : 0); ++k) note_launch();  // its other kernels
  ED_CUDA(cudaStreamSynchronize(s));
  // ---- results
  ED_CUDA(cudaMemcpyAsync(C.data(), dC.p, n * sizeof(BCluster), cudaMemcpyDeviceToHost, s));
  std::vector<BRun> Rh(nruns);
  if (nruns) ED_CUDA(cudaMemcpyAsync(Rh.data(), dR.p, nruns * sizeof(BRun), cudaMemcpyDeviceToHost, s));
  ED_CUDA(cudaStreamSynchronize(s));
  if (gf_steps_out) {
    for (int c = 0; c < n; ++c) gf_steps_out[c] = 0;
    for (int r = 0; r < nruns; ++r) gf_steps_out[Rh[r].cluster] += Rh[r].nsteps;
  }
  for (int c = 0; c < n; ++c) {
    if (E0_out) E0_out[c] = C[c].E0;
    if (res_out) res_out[c] = C[c].residual;
    if (status_out) status_out[c] = C[c].status;
    if (iters_out) iters_out[c] = C[c].iters;
  }
}

}  // namespace ed

using namespace ed;

extern "C" ed_status ed_batch_solve(const ed_cluster_desc* descs, int n, int precision, const double* omega, int n_freq,
                                    double eta, int axis, int cf_max_levels, double* E0, double* residual, int* status,
                                    int* iters,
                                    int64_t* gf_steps, double* G_out, int out_is_device) {
  try {
    if (!descs || n < 0) throw Error(ED_ERR_INVALID, "descs is NULL or n < 0");
    if (precision != ED_FP64 && precision != ED_FP32) throw Error(ED_ERR_INVALID, "precision must be ED_FP64 or ED_FP32");
    if (n_freq < 0 || (n_freq > 0 && (!omega || !G_out))) throw Error(ED_ERR_INVALID, "omega and G_out are needed when n_freq > 0");
    if (axis != ED_AXIS_REAL && axis != ED_AXIS_MATSUBARA) throw Error(ED_ERR_INVALID, "bad axis");
    std::vector<double2> z(n_freq);
    for (int k = 0; k < n_freq; ++k) z[k] = axis == ED_AXIS_REAL ? make_double2(omega[k], eta) : make_double2(0.0, omega[k]);
    int64_t total = 0;
    for (int c = 0; c < n; ++c) total += (int64_t)2 * n_freq * descs[c].n_sites * descs[c].n_sites;
    cudaStream_t s = nullptr;
    ED_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct SD {
      cudaStream_t s;
      ~SD() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    } sd{s};
    DevBuf<double2> Gd;
    double2* Gdev = (double2*)G_out;
    if (n_freq > 0 && !out_is_device) {
      Gd.alloc(std::max<int64_t>(total, 1));
      Gdev = Gd.p;
    }
    batch_solve(descs, n, precision, z.data(), n_freq, n_freq > 0, cf_max_levels > 0 ? cf_max_levels : kCfDefaultMaxLevels, E0,
                residual, status, iters, gf_steps, Gdev, s, 0, 0);
    if (n_freq > 0 && !out_is_device) {
      ED_CUDA(cudaMemcpyAsync(G_out, Gd.p, total * sizeof(double2), cudaMemcpyDeviceToHost, s));
      ED_CUDA(cudaStreamSynchronize(s));
    }
    return ED_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return ED_ERR_INVALID;
  }
}
