// One element of the factorized product y = H x (Eq. factorized, Sec. 4.1), shared by every
// kernel that computes H.psi element by element (the one-pass kernels of hpsi.cu and the
// allocation-free entry point of noalloc.cu), so that the diagonal and the sign handling exist
// once:
//
//   y[u][d] = D(u, d) x[u][d] + sum_{d'} K_dn[d][d'] x[u][d'] + sum_{u'} K_up[u][u'] x[u'][d]
//   D(u, d) = e_up[u] + e_dn[d] + sum_{i in cluster} U_i n_{i up} n_{i dn}
#pragma once

#include "ed_common.cuh"

namespace ed {

// Per-precision views of the diagonal tables and hopping values.
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

// Deterministic block reduction of three FP64 sums over NT threads (fixed shuffle tree, fixed
// warp order); the totals end in warp 0's lane 0.
template <int NT>
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
  __shared__ double sm[3][NT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sm[0][w] = a;
    sm[1][w] = b;
    sm[2][w] = c;
  }
  __syncthreads();
  if (w == 0) {
    a = l < NT / 32 ? sm[0][l] : 0.0;
    b = l < NT / 32 ? sm[1][l] : 0.0;
    c = l < NT / 32 ? sm[2][l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
      c += __shfl_down_sync(0xffffffffu, c, o);
    }
  }
  __syncthreads();
}

// Hopping values and per-orbital U staged in shared memory (sval[kMaxVals], sU[kMaxOrb]).
template <typename T>
__device__ __forceinline__ void load_params(const HopParams& hp, T* sval, T* sU) {
  for (int i = threadIdx.x; i < kMaxVals; i += blockDim.x) sval[i] = Prec<T>::val(hp, i);
  for (int i = threadIdx.x; i < kMaxOrb; i += blockDim.x) sU[i] = Prec<T>::U(hp, i);
  __syncthreads();
}

// y[u][d] of a vector X with leading dimension sv.ld: the diagonal by masked popcount of the
// doubly occupied interacting orbitals, then the down-spin hops (inside row u) and the up-spin
// hops (down column d), each entry (-1)^{M_ab} h_ab x[source].
template <typename T>
__device__ __forceinline__ T hpsi_element(const SectorView& sv, const T* __restrict__ sval, const T* __restrict__ sU,
                                          uint32_t umask, const T* __restrict__ X, int64_t u, int64_t d) {
  const T* xr = X + u * sv.ld;
  const uint32_t bu = sv.B_up[u], bd = sv.B_dn[d];
  T diag = Prec<T>::e_up(sv)[u] + Prec<T>::e_dn(sv)[d];
  uint32_t dbl = bu & bd & umask;
  while (dbl) {
    diag += sU[__ffs(dbl) - 1];
    dbl &= dbl - 1u;
  }
  T acc = diag * xr[d];
  int32_t p0 = sv.ptr_dn[d], p1 = sv.ptr_dn[d + 1];
  for (int32_t k = p0; k < p1; ++k) {
    const uint32_t e = __ldg(sv.ent_dn + k);
    const T v = sval[ent_vidx(e)];
    const T x = __ldg(xr + ent_col(e));
    acc += ent_neg(e) ? -v * x : v * x;
  }
  p0 = sv.ptr_up[u];
  p1 = sv.ptr_up[u + 1];
  for (int32_t k = p0; k < p1; ++k) {
    const uint32_t e = __ldg(sv.ent_up + k);
    const T v = sval[ent_vidx(e)];
    const T x = __ldg(X + (int64_t)ent_col(e) * sv.ld + d);
    acc += ent_neg(e) ? -v * x : v * x;
  }
  return acc;
}

}  // namespace ed
