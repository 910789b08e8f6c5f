// K3: matrix-free factorized H.psi (Eq. factorized, Sec. 4.1) and the fused Lanczos step
// (Eq. LanczosRecursion, Sec. 4.2).
//
//   y[u][d] = D(u, d) x[u][d] + sum_{u'} K_up[u][u'] x[u'][d] + sum_{d'} K_dn[d][d'] x[u][d']
//   D(u, d) = e_up[u] + e_dn[d] + sum_{i in cluster} U_i n_{i up} n_{i dn}
//
// e_s[r] = sum_a h_aa n_a is the one-body diagonal of each spin state; the interaction is a
// popcount-style loop over the set bits of b_up & b_dn & (orbitals with U != 0).  The
// off-diagonal K_s come from the packed tables of sector.cu.  Vectors are psi[u][d] with leading
// dimension ld; the up-spin hop reads whole rows, the down-spin hop gathers inside a row.
//
// The fused step computes w = H x - b_n x_prev, overwrites x_prev with w and reduces
// <x, w>, <w, w>, <x, x> in FP64 with a fixed-order block tree; the last block of each run
// (ticket counter) adds the block partials in a fixed order and finishes
// alpha_n = <x,w>/<x,x> and b_{n+1}^2 = <w,w> - <x,w>^2/<x,x>, so the recursion never leaves
// the device and repeated runs are bitwise identical.
#include "ed_common.cuh"

namespace ed {

constexpr int kThreads = 256;

template <typename T>
struct Prec;
template <>
struct Prec<double> {
  __device__ static const double* e_up(const SectorView& s) { return s.e_up; }
  __device__ static const double* e_dn(const SectorView& s) { return s.e_dn; }
  __device__ static double val(const HopParams& h, int i) { return h.val[i]; }
  __device__ static double U(const HopParams& h, int i) { return h.U[i]; }
};
template <>
struct Prec<float> {
  __device__ static const float* e_up(const SectorView& s) { return s.e_up32; }
  __device__ static const float* e_dn(const SectorView& s) { return s.e_dn32; }
  __device__ static float val(const HopParams& h, int i) { return h.valf[i]; }
  __device__ static float U(const HopParams& h, int i) { return h.Uf[i]; }
};

// Deterministic block reduction of three FP64 sums (fixed shuffle tree, fixed warp order).
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
  __shared__ double sm[3][kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sm[0][w] = a;
    sm[1][w] = b;
    sm[2][w] = c;
  }
  __syncthreads();
  if (w == 0) {
    a = l < kThreads / 32 ? sm[0][l] : 0.0;
    b = l < kThreads / 32 ? sm[1][l] : 0.0;
    c = l < kThreads / 32 ? sm[2][l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
      c += __shfl_down_sync(0xffffffffu, c, o);
    }
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ T hpsi_element(const SectorView& sv, const T* __restrict__ sval, const T* __restrict__ sU,
                                          uint32_t umask, const T* __restrict__ X, int64_t u, int64_t d) {
  const T* xr = X + u * sv.ld;
  uint32_t bu = sv.B_up[u], bd = sv.B_dn[d];
  T diag = Prec<T>::e_up(sv)[u] + Prec<T>::e_dn(sv)[d];
  uint32_t dbl = bu & bd & umask;
  while (dbl) {
    int i = __ffs(dbl) - 1;
    diag += sU[i];
    dbl &= dbl - 1u;
  }
  T acc = diag * xr[d];
  int32_t p0 = sv.ptr_dn[d], p1 = sv.ptr_dn[d + 1];
  for (int32_t k = p0; k < p1; ++k) {
    uint32_t e = __ldg(sv.ent_dn + k);
    T v = sval[ent_vidx(e)];
    T x = __ldg(xr + ent_col(e));
    acc += ent_neg(e) ? -v * x : v * x;
  }
  p0 = sv.ptr_up[u];
  p1 = sv.ptr_up[u + 1];
  for (int32_t k = p0; k < p1; ++k) {
    uint32_t e = __ldg(sv.ent_up + k);
    T v = sval[ent_vidx(e)];
    T x = __ldg(X + (int64_t)ent_col(e) * sv.ld + d);
    acc += ent_neg(e) ? -v * x : v * x;
  }
  return acc;
}

template <typename T>
__device__ __forceinline__ void load_params(const HopParams& hp, T* sval, T* sU) {
  for (int i = threadIdx.x; i < kMaxVals; i += blockDim.x) sval[i] = Prec<T>::val(hp, i);
  for (int i = threadIdx.x; i < kMaxOrb; i += blockDim.x) sU[i] = Prec<T>::U(hp, i);
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_hpsi_flat(SectorView sv, HopParams hp, const T* __restrict__ X,
                                                        T* __restrict__ Y) {
  __shared__ T sval[kMaxVals];
  __shared__ T sU[kMaxOrb];
  load_params<T>(hp, sval, sU);
  const int64_t dim = sv.d_up * sv.d_dn;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < dim; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t u = idx / sv.d_dn, d = idx - u * sv.d_dn;
    Y[u * sv.ld + d] = hpsi_element<T>(sv, sval, sU, hp.umask, X, u, d);
  }
}

// Fused Lanczos step, one run per blockIdx.y.  Grid x is fixed (lanczos_blocks) so that the
// number of partials per run is known.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_lanczos_step(SectorView sv, HopParams hp, const T* __restrict__ X0,
                                                           T* __restrict__ XP0, int64_t vstride, int n,
                                                           LanczosScalars ls) {
  __shared__ T sval[kMaxVals];
  __shared__ T sU[kMaxOrb];
  __shared__ bool s_last;
  const int run = blockIdx.y;
  if (!ls.active[run]) return;
  load_params<T>(hp, sval, sU);
  const T* X = X0 + run * vstride;
  T* XP = XP0 + run * vstride;
  const double bn = ls.beta[(int64_t)run * (ls.mstride + 1) + n];
  const int64_t dim = sv.d_up * sv.d_dn;
  double sxw = 0.0, sww = 0.0, sxx = 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < dim; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t u = idx / sv.d_dn, d = idx - u * sv.d_dn;
    int64_t o = u * sv.ld + d;
    T hx = hpsi_element<T>(sv, sval, sU, hp.umask, X, u, d);
    T w = hx - (T)bn * XP[o];
    XP[o] = w;
    double x = (double)X[o], wd = (double)w;
    sxw += x * wd;
    sww += wd * wd;
    sxx += x * x;
  }
  block_sum3(sxw, sww, sxx);
  double* part = ls.partial + ((int64_t)run * gridDim.x) * 3;
  if (threadIdx.x == 0) {
    part[blockIdx.x * 3 + 0] = sxw;
    part[blockIdx.x * 3 + 1] = sww;
    part[blockIdx.x * 3 + 2] = sxx;
    __threadfence();
    unsigned t = atomicAdd(ls.counter + run, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    a += __ldcg(part + i * 3 + 0);
    b += __ldcg(part + i * 3 + 1);
    c += __ldcg(part + i * 3 + 2);
  }
  block_sum3(a, b, c);
  if (threadIdx.x == 0) {
    double alpha = c > 0.0 ? a / c : 0.0;
    double b2 = c > 0.0 ? b - a * a / c : 0.0;
    double bnext = b2 > 0.0 ? sqrt(b2) : 0.0;
    int64_t base = (int64_t)run * ls.mstride;
    ls.alpha[base + n] = alpha;
    ls.beta[(int64_t)run * (ls.mstride + 1) + n + 1] = bnext;
    if (ls.nsteps) ls.nsteps[run] = n + 1;
    if (!(bnext > ls.btol * ls.beta0[run]) || n + 1 >= ls.mstride) ls.active[run] = 0;
    ls.counter[run] = 0u;
  }
}

static int grid_for(int64_t dim) {
  int64_t b = (dim + kThreads - 1) / kThreads;
  const int64_t cap = 152 * 8;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

int lanczos_blocks(const SectorView& sv) { return grid_for(sv.d_up * sv.d_dn); }

void launch_hpsi(const SectorView& sv, const HopParams& hp, int dtype, const void* x, void* y, cudaStream_t s) {
  int g = grid_for(sv.d_up * sv.d_dn);
  const double es = dtype == ED_FP64 ? 8.0 : 4.0;
  ProfScope ps_(K_HPSI, s, 2.0 * es * (double)(sv.d_up * sv.d_dn));
  if (dtype == ED_FP64)
    k_hpsi_flat<double><<<g, kThreads, 0, s>>>(sv, hp, (const double*)x, (double*)y);
  else
    k_hpsi_flat<float><<<g, kThreads, 0, s>>>(sv, hp, (const float*)x, (float*)y);
  ED_CHECK_LAUNCH();
}

void launch_lanczos_step(const SectorView& sv, const HopParams& hp, int dtype, const void* X, void* XP,
                         int64_t vstride, int runs, int n, const LanczosScalars& ls, int nblk_cap, cudaStream_t s) {
  int g = grid_for(sv.d_up * sv.d_dn);
  if (g > nblk_cap) throw Error(ED_ERR_INVALID, "partial buffer too small");
  dim3 grid(g, runs);
  const double es = dtype == ED_FP64 ? 8.0 : 4.0;
  ProfScope ps_(K_LANCZOS_STEP, s, 3.0 * es * (double)(sv.d_up * sv.d_dn) * runs);
  if (dtype == ED_FP64)
    k_lanczos_step<double><<<grid, kThreads, 0, s>>>(sv, hp, (const double*)X, (double*)XP, vstride, n, ls);
  else
    k_lanczos_step<float><<<grid, kThreads, 0, s>>>(sv, hp, (const float*)X, (float*)XP, vstride, n, ls);
  ED_CHECK_LAUNCH();
}

}  // namespace ed
