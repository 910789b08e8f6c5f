// K4-K6: Lanczos vector updates, reductions, the tridiagonal eigensolver and the ground-state
// driver (Sec. 4.2).
//
// Ground state: v_0 from the seeded splitmix64 stream, normalized; each step is the fused
// kernel of hpsi.cu (w = H v_n - b_n v_{n-1}, FP64 reductions) followed by
// v_{n+1} = (w - a_n v_n) / b_{n+1}.  Every few steps the lowest eigenpair of the tridiagonal
// matrix of Eq. tridiag is found on the device (multisection on the Sturm count, then inverse
// iteration); the run stops when the Ritz estimate b_M |s_M| is below the tolerance.  The ground
// state in the original basis is rebuilt by retracing the recursion (the vectors are not
// stored) and accumulating sum_n s_n v_n; then an explicit FP64 residual ||H W - E W|| and the
// Rayleigh quotient E are taken.  With FP32 vectors the same recursion runs on FP32 storage
// and the result is polished in FP64 (Rayleigh quotient and residual with the FP64 operator,
// and FP64 Lanczos restarted from the FP32 ground state if the energy bound is not met).
#include <algorithm>
#include <cmath>

#include "ed_common.cuh"
#include "tridiag.cuh"

namespace ed {

constexpr int kVT = 256;

__device__ __forceinline__ double ldv(int dt, const void* p, int64_t i) {
  return dt == ED_FP64 ? ((const double*)p)[i] : (double)((const float*)p)[i];
}
__device__ __forceinline__ void stv(int dt, void* p, int64_t i, double v) {
  if (dt == ED_FP64)
    ((double*)p)[i] = v;
  else
    ((float*)p)[i] = (float)v;
}

static int vgrid(int64_t n) {
  int64_t b = (n + kVT - 1) / kVT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
}

// TO: type of the ground-state accumulator omega (the vectors' type, or FP64 for FP32 vectors
// whose sum must keep FP64 precision).
template <typename T, typename TO>
__global__ void __launch_bounds__(kVT) k_lanczos_next(T* __restrict__ W0, const T* __restrict__ X0, int64_t d_up, int64_t d_dn,
                                                      int64_t ld, int64_t vstride, int n, LanczosScalars ls,
                                                      TO* __restrict__ omega, const double* __restrict__ coef) {
  const int run = blockIdx.y;
  if (!ls.active[run]) return;
  T* W = W0 + run * vstride;
  const T* X = X0 + run * vstride;
  const double a = ls.alpha[(int64_t)run * ls.mstride + n];
  const double b = ls.beta[(int64_t)run * (ls.mstride + 1) + n + 1];
  const double ib = 1.0 / b;
  const TO cf = omega ? (TO)coef[n + 1] : TO(0);
  const T aT = (T)a, ibT = (T)ib;
  const int64_t dim = d_up * d_dn;
  for_each_element(d_up, d_dn, [&](int64_t u, int64_t d, int64_t idx) {
    int64_t o = u * ld + d;
    const T vt = (W[o] - aT * X[o]) * ibT;
    W[o] = vt;
    if (omega) omega[idx] += cf * (TO)vt;
    });
}

void launch_lanczos_next(int dtype, void* W, const void* X, int64_t d_up, int64_t d_dn, int64_t ld, int64_t vstride,
                         int runs, int n, const LanczosScalars& ls, void* omega, const double* coef, cudaStream_t s,
                         int omega_dtype) {
  dim3 g(vgrid(d_up * d_dn), runs);
  const double es = dtype == ED_FP64 ? 8.0 : 4.0;
  if (omega_dtype < 0) omega_dtype = dtype;
  const double eo = omega_dtype == ED_FP64 ? 8.0 : 4.0;
  ProfScope ps_(K_LANCZOS_NEXT, s, (3.0 * es + (omega ? 2.0 * eo : 0.0)) * (double)(d_up * d_dn) * runs);
  if (dtype == ED_FP64)
    k_lanczos_next<double, double><<<g, kVT, 0, s>>>((double*)W, (const double*)X, d_up, d_dn, ld, vstride, n, ls,
                                                      (double*)omega, coef);
  else if (omega_dtype == ED_FP64)
    k_lanczos_next<float, double><<<g, kVT, 0, s>>>((float*)W, (const float*)X, d_up, d_dn, ld, vstride, n, ls,
                                                     (double*)omega, coef);
  else
    k_lanczos_next<float, float><<<g, kVT, 0, s>>>((float*)W, (const float*)X, d_up, d_dn, ld, vstride, n, ls,
                                                    (float*)omega, coef);
  ED_CHECK_LAUNCH();
}

// splitmix64 (Steele, Lea & Flood 2014): the counter-based stream of the Lanczos start vector.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_start_vector(int dt, void* v, int64_t d_up, int64_t d_dn, int64_t ld, uint64_t seed) {
  const int64_t dim = d_up * d_dn;
  for_each_element(d_up, d_dn, [&](int64_t u, int64_t d, int64_t idx) {
    double r = (double)(splitmix64(seed ^ (uint64_t)idx) >> 11) * (1.0 / 9007199254740992.0);
    stv(dt, v, u * ld + d, 2.0 * r - 1.0);
    });
}

void launch_start_vector(int dtype, void* v, int64_t d_up, int64_t d_dn, int64_t ld, uint64_t seed, cudaStream_t s) {
  ProfScope ps_(K_VECTOR, s, 0.0);
  k_start_vector<<<vgrid(d_up * d_dn), kVT, 0, s>>>(dtype, v, d_up, d_dn, ld, seed);
  ED_CHECK_LAUNCH();
}

__device__ __forceinline__ double block_sum(double a) {
  __shared__ double sm[kVT / 32];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sm[w] = a;
  __syncthreads();
  if (w == 0) {
    a = l < kVT / 32 ? sm[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  }
  __syncthreads();
  return a;
}

__global__ void k_dot_partial(int dta, const void* a, int dtb, const void* b, int64_t d_up, int64_t d_dn, int64_t ld,
                              double* __restrict__ partial) {
  const int64_t dim = d_up * d_dn;
  double s = 0.0;
  for_each_element(d_up, d_dn, [&](int64_t u, int64_t d, int64_t idx) {
    int64_t o = u * ld + d;
    s += ldv(dta, a, o) * ldv(dtb, b, o);
    });
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_sum_partials(const double* __restrict__ partial, int n, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

void launch_dot(int dta, const void* a, int dtb, const void* b, int64_t d_up, int64_t d_dn, int64_t ld, double* partial,
                int nblk, double* out, cudaStream_t s) {
  int g = std::min(vgrid(d_up * d_dn), nblk);
  {
    ProfScope ps_(K_VECTOR, s, 0.0);
    k_dot_partial<<<g, kVT, 0, s>>>(dta, a, dtb, b, d_up, d_dn, ld, partial);
    ED_CHECK_LAUNCH();
  }
  ProfScope ps_(K_VECTOR, s, 0.0);
  k_sum_partials<<<1, kVT, 0, s>>>(partial, g, out);
  ED_CHECK_LAUNCH();
}

// y = ca * a + cb * b; ca / cb are device scalars (NULL = 0, and the matching vector is unread);
// a scalar pointer with the flag `inv_sqrt` set is used as 1/sqrt(*ca).
__global__ void k_axpby(int dty, void* y, int dta, const void* a, const double* ca, int dtb, const void* b,
                        const double* cb, int64_t d_up, int64_t d_dn, int64_t ld, int inv_sqrt_a, int neg_b) {
  double sa = 0.0, sb = 0.0;
  if (ca) {
    sa = *ca;
    if (inv_sqrt_a) sa = sa > 0.0 ? 1.0 / sqrt(sa) : 0.0;
  }
  if (cb) sb = neg_b ? -*cb : *cb;
  const int64_t dim = d_up * d_dn;
  for_each_element(d_up, d_dn, [&](int64_t u, int64_t d, int64_t idx) {
    int64_t o = u * ld + d;
    double v = 0.0;
    if (ca) v += sa * ldv(dta, a, o);
    if (cb) v += sb * ldv(dtb, b, o);
    stv(dty, y, o, v);
    });
}

static void axpby(int dty, void* y, int dta, const void* a, const double* ca, int dtb, const void* b, const double* cb,
                  int64_t d_up, int64_t d_dn, int64_t ld, cudaStream_t s, int inv_sqrt_a = 0, int neg_b = 0) {
  ProfScope ps_(K_VECTOR, s, 0.0);
  k_axpby<<<vgrid(d_up * d_dn), kVT, 0, s>>>(dty, y, dta, a, ca, dtb, b, cb, d_up, d_dn, ld, inv_sqrt_a, neg_b);
  ED_CHECK_LAUNCH();
}

__global__ void k_copy_ld(int dty, void* y, int64_t ld_y, int dta, const void* a, int64_t ld_a,
                          const double* __restrict__ scale, int64_t d_up, int64_t d_dn) {
  const double f = scale ? *scale : 1.0;
  const int64_t dim = d_up * d_dn;
  for_each_element(d_up, d_dn, [&](int64_t u, int64_t d, int64_t idx) {
    stv(dty, y, u * ld_y + d, f * ldv(dta, a, u * ld_a + d));
    });
}

void launch_copy_ld(int dty, void* y, int64_t ld_y, int dta, const void* a, int64_t ld_a, const double* scale,
                    int64_t d_up, int64_t d_dn, cudaStream_t s) {
  ProfScope ps_(K_VECTOR, s, 0.0);
  k_copy_ld<<<vgrid(d_up * d_dn), kVT, 0, s>>>(dty, y, ld_y, dta, a, ld_a, scale, d_up, d_dn);
  ED_CHECK_LAUNCH();
}

void launch_axpby(int dty, void* y, int dta, const void* a, const double* ca, int dtb, const void* b, const double* cb,
                  int64_t d_up, int64_t d_dn, int64_t ld, cudaStream_t s) {
  axpby(dty, y, dta, a, ca, dtb, b, cb, d_up, d_dn, ld, s);
}

// ---- tridiagonal eigensolver (one block): tridiag.cuh --------------------------------------
__global__ void __launch_bounds__(kVT) k_tridiag_lowest(const double* __restrict__ a, const double* __restrict__ b, int n,
                                                        double* __restrict__ out_eval, double* __restrict__ vec) {
  tridiag_lowest_block(a, b, n, out_eval, vec);
}

void launch_tridiag_lowest(const double* alpha, const double* beta, int n, double* out_eval, double* out_vec,
                           cudaStream_t s) {
  ProfScope ps_(K_TRIDIAG, s, 0.0);
  k_tridiag_lowest<<<1, kVT, 0, s>>>(alpha, beta, n, out_eval, out_vec);
  ED_CHECK_LAUNCH();
}

}  // namespace ed
