// Lowest eigenpair of the Lanczos tridiagonal matrix (Eq. tridiag), computed by one thread block:
// multisection on the Sturm count (every thread evaluates one point per round) for the two
// lowest eigenvalues, then inverse iteration by one thread with a shift just below the lowest
// eigenvalue (T - sigma I is positive definite, so Thomas elimination without pivoting is
// stable).  Used by the single-cluster driver and by the batched per-block solver.
#pragma once

#include <cuda_runtime.h>

namespace ed {

// Matrix of Eq. tridiag with diagonal alpha[0..n-1] and off-diagonal beta[1..n-1].
static __device__ inline int sturm_count(const double* __restrict__ a, const double* __restrict__ b, int n, double x) {
  int cnt = 0;
  double q = a[0] - x;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < n; ++i) {
    if (q == 0.0) q = 1e-300;
    q = a[i] - x - b[i] * b[i] / q;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// out_eval: [0] lowest eigenvalue, [1] second eigenvalue (inf if n < 2), [2] Ritz estimate
// b_n |s_{n-1}|.  out_vec: [0, n) unit eigenvector of the lowest eigenvalue (s_0 >= 0),
// [n, 2n) scratch.
static __device__ void tridiag_lowest_block(const double* __restrict__ a, const double* __restrict__ b, int n,
                                     double* __restrict__ out_eval, double* __restrict__ vec) {
  __shared__ double s_lo, s_hi;
  __shared__ int s_first;
  __shared__ double s_res[2];
  if (threadIdx.x == 0) {
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
      double r = (i > 0 ? fabs(b[i]) : 0.0) + (i + 1 < n ? fabs(b[i + 1]) : 0.0);
      lo = fmin(lo, a[i] - r);
      hi = fmax(hi, a[i] + r);
    }
    double pad = 1e-12 * fmax(1.0, fmax(fabs(lo), fabs(hi))) + 1e-300;
    s_lo = lo - pad;
    s_hi = hi + pad;
  }
  __syncthreads();
  const double glo = s_lo, ghi = s_hi;
  for (int k = 0; k < 2; ++k) {
    if (k == 1 && n < 2) {
      if (threadIdx.x == 0) s_res[1] = INFINITY;
      break;
    }
    double lo = glo, hi = ghi;
    for (int round = 0; round < 16; ++round) {
      if (threadIdx.x == 0) s_first = blockDim.x;
      __syncthreads();
      double x = lo + (hi - lo) * (double)(threadIdx.x + 1) / (double)(blockDim.x + 1);
      if (sturm_count(a, b, n, x) >= k + 1) atomicMin(&s_first, (int)threadIdx.x);
      __syncthreads();
      int j = s_first;
      double nlo = j == 0 ? lo : lo + (hi - lo) * (double)j / (double)(blockDim.x + 1);
      double nhi = j == (int)blockDim.x ? hi : lo + (hi - lo) * (double)(j + 1) / (double)(blockDim.x + 1);
      lo = nlo;
      hi = nhi;
      __syncthreads();
      if (hi - lo <= 4e-16 * fmax(fabs(lo), fabs(hi))) break;
    }
    if (threadIdx.x == 0) s_res[k] = 0.5 * (lo + hi);
    __syncthreads();
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double lam = s_res[0];
  out_eval[0] = lam;
  out_eval[1] = s_res[1];
  // inverse iteration with shift just below lam: T - sigma I is positive definite, so the
  // Thomas elimination without pivoting is stable.
  double scale = fmax(1.0, fmax(fabs(glo), fabs(ghi)));
  double sigma = lam - 1e-10 * scale;
  double* y = vec;
  double* cp = vec + n;
  for (int i = 0; i < n; ++i) y[i] = 1.0 + 0.1 * sin((double)i);
  for (int it = 0; it < 3; ++it) {
    // forward sweep
    double m = a[0] - sigma;
    cp[0] = (n > 1 ? b[1] : 0.0) / m;
    y[0] = y[0] / m;
    for (int i = 1; i < n; ++i) {
      m = (a[i] - sigma) - b[i] * cp[i - 1];
      cp[i] = (i + 1 < n ? b[i + 1] : 0.0) / m;
      y[i] = (y[i] - b[i] * y[i - 1]) / m;
    }
    for (int i = n - 2; i >= 0; --i) y[i] -= cp[i] * y[i + 1];
    double nr = 0.0;
    for (int i = 0; i < n; ++i) nr += y[i] * y[i];
    nr = 1.0 / sqrt(nr);
    for (int i = 0; i < n; ++i) y[i] *= nr;
  }
  if (y[0] < 0.0)
    for (int i = 0; i < n; ++i) y[i] = -y[i];
  out_eval[2] = fabs(b[n]) * fabs(y[n - 1]);
}


}  // namespace ed
