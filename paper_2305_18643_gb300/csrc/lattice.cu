// Lattice steps that consume the cluster Green function: cluster perturbation theory (Sec. 3,
// Eqs. CPT1-CPT3) and the CDMFT bath fit (Sec. 6, Eqs. hybridization, CPT_CDMFT, dist_func).
//
// All of it is small dense complex linear algebra repeated over many (k~, z) pairs, so the unit
// of work is one warp per L x L matrix (L <= 32 cluster sites, lane = column): the matrix and its
// inverse live in the warp's slice of shared memory and are reduced by Gauss-Jordan elimination
// with partial pivoting (pivot row found by a warp arg-max).  Sums over k~ (the super-lattice
// average) and over frequencies (the distance and its gradient) run in a fixed order, so repeated
// calls give bitwise identical results.
//
//   V(k~)_{ij}   = sum_bonds t e^{i k~.r~} at (i, j), its conjugate at (j, i)   (Sec. 2.2)
//   G(k~, z)     = [G_c(z)^-1 + Gamma(z) - V(k~)]^-1                             (Eqs. CPT1, CPT_CDMFT)
//   G_per(k, z)  = (1/L) sum_{R R'} e^{-i k.(R - R')} G_{R R'}(k, z)             (Eq. CPT3)
//   G_bar(z)     = mean over k~ of G(k~, z)                                      (CDMFT step 3)
//   A(z)         = Gamma(z) + G_c(z)^-1 - G_bar(z)^-1 = z - h_c - calG_0^-1(z)   (CDMFT step 4)
//   d            = sum_n W_n ||A(z_n) - Gamma'(z_n)||_F^2                         (Eq. dist_func)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ed_common.cuh"

namespace ed {

constexpr int kLatMaxSites = 32;
constexpr int kLatWarps = 4;  // matrices per block of the inversion kernels

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 cinv(double2 a) {
  const double s = 1.0 / cabs2(a);
  return make_double2(a.x * s, -a.y * s);
}

// Inverts the L x L complex matrix a (row-major, leading dimension L) in shared memory into b,
// one warp, lane j owning column j; col is L elements of scratch.  a is destroyed.  Returns false
// (b undefined) if a pivot is exactly zero.
__device__ bool warp_invert(double2* a, double2* b, double2* col, int L) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < L; ++i)
    if (lane < L) b[i * L + lane] = make_double2(i == lane ? 1.0 : 0.0, 0.0);
  __syncwarp();
  bool ok = true;
  for (int k = 0; k < L; ++k) {
    // pivot: the row i >= k with the largest |a[i][k]| (smallest i on ties)
    double best = lane >= k && lane < L ? cabs2(a[lane * L + k]) : -1.0;
    int bi = lane;
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (!(best > 0.0)) ok = false;
    if (bi != k && lane < L) {
      double2 t = a[k * L + lane];
      a[k * L + lane] = a[bi * L + lane];
      a[bi * L + lane] = t;
      t = b[k * L + lane];
      b[k * L + lane] = b[bi * L + lane];
      b[bi * L + lane] = t;
    }
    __syncwarp();
    const double2 inv = ok ? cinv(a[k * L + k]) : make_double2(0.0, 0.0);
    __syncwarp();
    if (lane < L) {
      a[k * L + lane] = cmul(a[k * L + lane], inv);
      b[k * L + lane] = cmul(b[k * L + lane], inv);
      col[lane] = a[lane * L + k];
    }
    __syncwarp();
    if (lane < L) {
      const double2 ak = a[k * L + lane], bk = b[k * L + lane];
      for (int i = 0; i < L; ++i) {
        if (i == k) continue;
        const double2 f = col[i];
        a[i * L + lane] = csub(a[i * L + lane], cmul(f, ak));
        b[i * L + lane] = csub(b[i * L + lane], cmul(f, bk));
      }
    }
    __syncwarp();
  }
  return ok;
}

// Shared memory of one warp: matrix, inverse, pivot column.
__host__ __device__ inline size_t warp_slice(int L) { return (size_t)(2 * L * L + 32) * sizeof(double2); }

// out[m] = (in[m] (+ add[m]))^-1 for count matrices; status[0] counts singular ones.
__global__ void k_invert(const double2* __restrict__ in, const double2* __restrict__ add, double2* __restrict__ out, int L,
                         int64_t count, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char lat_smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double2* a = reinterpret_cast<double2*>(lat_smem + w * warp_slice(L));
  double2* b = a + L * L;
  double2* col = b + L * L;
  for (int64_t m = (int64_t)blockIdx.x * kLatWarps + w; m < count; m += (int64_t)gridDim.x * kLatWarps) {
    const double2* src = in + m * L * L;
    for (int e = lane; e < L * L; e += 32) a[e] = add ? cadd(src[e], add[m * L * L + e]) : src[e];
    __syncwarp();
    const bool ok = warp_invert(a, b, col, L);
    for (int e = lane; e < L * L; e += 32) out[m * L * L + e] = b[e];
    if (!ok && lane == 0) atomicAdd(status, 1);
    __syncwarp();
  }
}

// V[k][i][j] of Sec. 2.2 from the bond list: thread per (k, element), bonds summed in order.
__global__ void k_build_v(const double* __restrict__ kt, int nk, int D, const int* __restrict__ bij,
                          const double* __restrict__ brt, const double* __restrict__ bt, int nb, int L,
                          double2* __restrict__ V) {
  const int64_t n = (int64_t)nk * L * L;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / (L * L)), e = (int)(t % (L * L)), r = e / L, c = e % L;
    double2 v = make_double2(0.0, 0.0);
    for (int q = 0; q < nb; ++q) {
      const int i = bij[2 * q], j = bij[2 * q + 1];
      if (!((i == r && j == c) || (j == r && i == c))) continue;
      double ph = 0.0;
      for (int a = 0; a < D; ++a) ph += kt[k * D + a] * brt[q * D + a];
      double s, co;
      sincos(ph, &s, &co);
      if (i == r && j == c) v = cadd(v, make_double2(bt[q] * co, bt[q] * s));      // t e^{i k.r}
      if (j == r && i == c) v = cadd(v, make_double2(bt[q] * co, -bt[q] * s));     // its conjugate
    }
    V[t] = v;
  }
}

// CPT: warp per (k, z) pair.  mode 0 writes G(k, z); mode 1 the periodized scalar (Eq. CPT3).
__global__ void k_cpt(const double2* __restrict__ Gci, const double2* __restrict__ V, const double* __restrict__ kt,
                      const double* __restrict__ pos, int D, int L, int nz, int nk, int mode, double2* __restrict__ out,
                      int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char lat_smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double2* a = reinterpret_cast<double2*>(lat_smem + w * warp_slice(L));
  double2* b = a + L * L;
  double2* col = b + L * L;
  const int64_t pairs = (int64_t)nk * nz;
  for (int64_t pr = (int64_t)blockIdx.x * kLatWarps + w; pr < pairs; pr += (int64_t)gridDim.x * kLatWarps) {
    const int k = (int)(pr / nz), n = (int)(pr % nz);
    for (int e = lane; e < L * L; e += 32) a[e] = csub(Gci[(int64_t)n * L * L + e], V[(int64_t)k * L * L + e]);
    __syncwarp();
    const bool ok = warp_invert(a, b, col, L);
    if (!ok && lane == 0) atomicAdd(status, 1);
    if (mode == 0) {
      for (int e = lane; e < L * L; e += 32) out[pr * L * L + e] = b[e];
    } else {
      // (1/L) sum_{R R'} e^{-i k.(R - R')} G_{R R'}: lane R' sums its column, then the warp adds
      double2 s = make_double2(0.0, 0.0);
      if (lane < L) {
        for (int r = 0; r < L; ++r) {
          double ph = 0.0;
          for (int d = 0; d < D; ++d) ph += kt[k * D + d] * (pos[r * D + d] - pos[lane * D + d]);
          double sn, cs;
          sincos(-ph, &sn, &cs);
          s = cadd(s, cmul(make_double2(cs, sn), b[r * L + lane]));
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_down_sync(0xffffffffu, s.x, o);
        s.y += __shfl_down_sync(0xffffffffu, s.y, o);
      }
      if (lane == 0) out[pr] = make_double2(s.x / L, s.y / L);
    }
    __syncwarp();
  }
}

// Super-lattice average: block per frequency; warp w inverts k = w, w + kLatWarps, ... and keeps
// its running sum in shared memory; the warps' sums are added in warp order.
__global__ void k_cpt_average(const double2* __restrict__ Gci, const double2* __restrict__ V, int L, int nz, int nk,
                              double2* __restrict__ out, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char lat_smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double2* a = reinterpret_cast<double2*>(lat_smem + w * warp_slice(L));
  double2* b = a + L * L;
  double2* col = b + L * L;
  double2* acc = reinterpret_cast<double2*>(lat_smem + kLatWarps * warp_slice(L)) + w * L * L;
  for (int n = blockIdx.x; n < nz; n += gridDim.x) {
    for (int e = lane; e < L * L; e += 32) acc[e] = make_double2(0.0, 0.0);
    for (int k = w; k < nk; k += kLatWarps) {
      for (int e = lane; e < L * L; e += 32) a[e] = csub(Gci[(int64_t)n * L * L + e], V[(int64_t)k * L * L + e]);
      __syncwarp();
      const bool ok = warp_invert(a, b, col, L);
      if (!ok && lane == 0) atomicAdd(status, 1);
      for (int e = lane; e < L * L; e += 32) acc[e] = cadd(acc[e], b[e]);
      __syncwarp();
    }
    __syncthreads();
    double2* acc0 = reinterpret_cast<double2*>(lat_smem + kLatWarps * warp_slice(L));
    for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
      double2 s = acc0[e];
      for (int q = 1; q < kLatWarps; ++q) s = cadd(s, acc0[q * L * L + e]);
      out[(int64_t)n * L * L + e] = make_double2(s.x / nk, s.y / nk);
    }
    __syncthreads();
  }
}

// Gamma[c][n][mu][nu] = sum_a theta[c][mu][a] theta[c][nu][a] / (z_n - eps[c][a]) (Eq. hybridization).
__global__ void k_hybridization(const double* __restrict__ eps, const double* __restrict__ theta, const double2* __restrict__ z,
                                int L, int nb, int nz, int ncand, double2* __restrict__ out) {
  const int64_t n = (int64_t)ncand * nz * L * L;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / ((int64_t)nz * L * L);
    const int rem = (int)(t % ((int64_t)nz * L * L));
    const int f = rem / (L * L), mu = (rem % (L * L)) / L, nu = rem % L;
    const double* th = theta + c * L * nb;
    const double* ep = eps + c * nb;
    double2 s = make_double2(0.0, 0.0);
    for (int a = 0; a < nb; ++a) {
      const double w = th[mu * nb + a] * th[nu * nb + a];
      s = cadd(s, cmul(make_double2(w, 0.0), cinv(make_double2(z[f].x - ep[a], z[f].y))));
    }
    out[t] = s;
  }
}

// A = Gamma + Gci_raw - Gbar^-1, elementwise (the inverses computed before).
__global__ void k_target(const double2* __restrict__ Gam, const double2* __restrict__ Gci, const double2* __restrict__ Gbi,
                         int64_t n, double2* __restrict__ A) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    double2 v = csub(Gci[t], Gbi[t]);
    if (Gam) v = cadd(v, Gam[t]);
    A[t] = v;
  }
}

// Distance of candidate c: R = A - Gamma_c; d_c = sum_n W_n sum |R|^2, one block per candidate,
// threads over (n, mu, nu) in a fixed order then a fixed tree.
__global__ void k_distance(const double2* __restrict__ A, const double2* __restrict__ Gam, const double* __restrict__ Wn,
                           int L, int nz, double* __restrict__ d) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  const int64_t per = (int64_t)nz * L * L;
  double s = 0.0;
  for (int64_t t = threadIdx.x; t < per; t += blockDim.x) {
    const double2 r = csub(A[t], Gam[c * per + t]);
    s += Wn[t / (L * L)] * cabs2(r);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) d[c] = red[0];
}

// Gradient of d_c with respect to eps_a (p < nb) and theta_{rho a} (p = nb + rho nb + a):
//   d d / d eps_a      = -2 Re sum_n W_n g_a^2 sum_{mu nu} conj(R_{mu nu}) theta_{mu a} theta_{nu a}
//   d d / d theta_{rho a} = -2 Re sum_n W_n g_a [sum_nu conj(R_{rho nu}) theta_{nu a}
//                                               + sum_mu conj(R_{mu rho}) theta_{mu a}]
// with g_a = 1 / (z_n - eps_a) and R = A - Gamma_c; thread per (candidate, parameter).
__global__ void k_distance_grad(const double2* __restrict__ A, const double2* __restrict__ Gam, const double* __restrict__ Wn,
                                const double2* __restrict__ z, const double* __restrict__ eps,
                                const double* __restrict__ theta, int L, int nb, int nz, int ncand,
                                double* __restrict__ grad) {
  const int np = nb + L * nb;
  const int64_t total = (int64_t)ncand * np;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / np), p = (int)(t % np);
    const double* th = theta + (int64_t)c * L * nb;
    const int64_t per = (int64_t)nz * L * L;
    const double2* G = Gam + c * per;
    double acc = 0.0;
    if (p < nb) {
      const int a = p;
      for (int n = 0; n < nz; ++n) {
        const double2 g = cinv(make_double2(z[n].x - eps[c * nb + a], z[n].y));
        double2 s = make_double2(0.0, 0.0);
        for (int mu = 0; mu < L; ++mu)
          for (int nu = 0; nu < L; ++nu) {
            const int64_t e = (int64_t)n * L * L + mu * L + nu;
            const double2 r = csub(A[e], G[e]);
            s = cadd(s, cmul(cconj(r), make_double2(th[mu * nb + a] * th[nu * nb + a], 0.0)));
          }
        acc += Wn[n] * cmul(s, cmul(g, g)).x;
      }
    } else {
      const int rho = (p - nb) / nb, a = (p - nb) % nb;
      for (int n = 0; n < nz; ++n) {
        const double2 g = cinv(make_double2(z[n].x - eps[c * nb + a], z[n].y));
        double2 s = make_double2(0.0, 0.0);
        for (int nu = 0; nu < L; ++nu) {
          const int64_t e1 = (int64_t)n * L * L + rho * L + nu, e2 = (int64_t)n * L * L + nu * L + rho;
          const double2 r1 = csub(A[e1], G[e1]), r2 = csub(A[e2], G[e2]);
          s = cadd(s, cmul(cadd(cconj(r1), cconj(r2)), make_double2(th[nu * nb + a], 0.0)));
        }
        acc += Wn[n] * cmul(s, g).x;
      }
    }
    grad[t] = -2.0 * acc;
  }
}

static unsigned lat_grid(int64_t n, int per_block) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + per_block - 1) / per_block, 152 * 16));
}

// ---------------------------------------------------------------- host side
struct LatticeDev {
  int L, D, nb;
  DevBuf<double> pos, rt, bt;
  DevBuf<int> bij;
};

static void check_lattice(const ed_superlattice* lat) {
  if (!lat) throw Error(ED_ERR_INVALID, "lattice is NULL");
  if (lat->n_sites < 1 || lat->n_sites > kLatMaxSites) throw Error(ED_ERR_INVALID, "need 1 <= n_sites <= 32");
  if (lat->dim < 1 || lat->dim > 3) throw Error(ED_ERR_INVALID, "dim must be 1, 2 or 3");
  if (!lat->pos || !lat->E) throw Error(ED_ERR_INVALID, "pos and E must not be NULL");
  if (lat->n_bonds < 0 || (lat->n_bonds > 0 && (!lat->bonds || !lat->bond_t)))
    throw Error(ED_ERR_INVALID, "bonds and bond_t must not be NULL when n_bonds > 0");
  const int D = lat->dim;
  for (int q = 0; q < lat->n_bonds; ++q) {
    const int i = lat->bonds[q * (2 + D)], j = lat->bonds[q * (2 + D) + 1];
    if (i < 0 || i >= lat->n_sites || j < 0 || j >= lat->n_sites) throw Error(ED_ERR_INVALID, "bond site out of range");
    if (!std::isfinite(lat->bond_t[q])) throw Error(ED_ERR_INVALID, "bond_t has a non-finite entry");
  }
}

static LatticeDev upload_lattice(const ed_superlattice* lat, cudaStream_t s) {
  LatticeDev d;
  d.L = lat->n_sites;
  d.D = lat->dim;
  d.nb = lat->n_bonds;
  const int D = d.D;
  std::vector<double> rt((size_t)std::max(d.nb, 1) * D, 0.0);
  std::vector<int> ij((size_t)std::max(d.nb, 1) * 2, 0);
  for (int q = 0; q < d.nb; ++q) {
    ij[2 * q] = lat->bonds[q * (2 + D)];
    ij[2 * q + 1] = lat->bonds[q * (2 + D) + 1];
    for (int a = 0; a < D; ++a) {
      double v = 0.0;  // r~ = n E
      for (int b = 0; b < D; ++b) v += lat->bonds[q * (2 + D) + 2 + b] * lat->E[b * D + a];
      rt[(size_t)q * D + a] = v;
    }
  }
  d.pos.alloc((size_t)d.L * D);
  d.rt.alloc(rt.size());
  d.bt.alloc(std::max(d.nb, 1));
  d.bij.alloc(ij.size());
  ED_CUDA(cudaMemcpyAsync(d.pos.p, lat->pos, (size_t)d.L * D * sizeof(double), cudaMemcpyHostToDevice, s));
  ED_CUDA(cudaMemcpyAsync(d.rt.p, rt.data(), rt.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  if (d.nb) ED_CUDA(cudaMemcpyAsync(d.bt.p, lat->bond_t, d.nb * sizeof(double), cudaMemcpyHostToDevice, s));
  ED_CUDA(cudaMemcpyAsync(d.bij.p, ij.data(), ij.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  ED_CUDA(cudaStreamSynchronize(s));  // the host vectors above go out of scope
  return d;
}

static void build_v(const LatticeDev& d, const DevBuf<double>& kt, int nk, DevBuf<double2>& V, cudaStream_t s) {
  V.alloc((size_t)nk * d.L * d.L);
  ProfScope ps_(K_LATTICE, s, 0.0);
  k_build_v<<<lat_grid((int64_t)nk * d.L * d.L, 256), 256, 0, s>>>(kt.p, nk, d.D, d.bij.p, d.rt.p, d.bt.p, d.nb, d.L, V.p);
  ED_CHECK_LAUNCH();
}

static void invert_batched(const double2* in, const double2* add, double2* out, int L, int64_t count, int* status,
                           cudaStream_t s) {
  const size_t smem = kLatWarps * warp_slice(L);
  allow_max_dynamic_smem(k_invert);
  ProfScope ps_(K_LATTICE, s, 0.0);
  k_invert<<<lat_grid(count, kLatWarps), 32 * kLatWarps, smem, s>>>(in, add, out, L, count, status);
  ED_CHECK_LAUNCH();
}

// Copies n complex values to the device (or points at them when they already are).
static const double2* dev_in(const double* p, size_t n, bool is_dev, DevBuf<double2>& tmp, cudaStream_t s) {
  if (!p) return nullptr;
  if (is_dev) return reinterpret_cast<const double2*>(p);
  tmp.alloc(n);
  ED_CUDA(cudaMemcpyAsync(tmp.p, p, n * sizeof(double2), cudaMemcpyHostToDevice, s));
  return tmp.p;
}

static void throw_singular(int* st_dev, cudaStream_t s) {
  int st = 0;
  ED_CUDA(cudaMemcpyAsync(&st, st_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  ED_CUDA(cudaStreamSynchronize(s));
  if (st) throw Error(ED_ERR_INVALID, std::to_string(st) + " singular matrices in a batched inversion");
}

__global__ void k_add_sub(const double2* __restrict__ a, const double2* __restrict__ b, double sign, int64_t n,
                          double2* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = make_double2(a[t].x + sign * b[t].x, a[t].y + sign * b[t].y);
}

// Gci = G_c^-1 (+ Gamma) for every frequency, on the device.
static void cluster_inverse(const double2* Gc, const double2* Gam, int L, int nz, DevBuf<double2>& Gci, int* st,
                            cudaStream_t s) {
  const int64_t n = (int64_t)nz * L * L;
  Gci.alloc(n);
  invert_batched(Gc, nullptr, Gci.p, L, nz, st, s);
  if (Gam) {
    ProfScope ps_(K_LATTICE, s, 0.0);
    k_add_sub<<<lat_grid(n, 256), 256, 0, s>>>(Gci.p, Gam, 1.0, n, Gci.p);
    ED_CHECK_LAUNCH();
  }
}

template <typename F>
static ed_status lat_guarded(F&& f) {
  try {
    return f();
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return ED_ERR_OOM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return ED_ERR_INVALID;
  }
}

static void require_lat(bool ok, const char* msg) {
  if (!ok) throw Error(ED_ERR_INVALID, msg);
}

// Distance (and gradient) of n_cand baths against A, all on the device; d and grad to the host.
struct DistanceWork {
  int L, nb, nz;
  DevBuf<double2> z, A, Gam;
  DevBuf<double> W, eps, theta, d, grad;
  void setup(int L_, int nb_, const double* zh, int nz_, const double* Wh, const double* Ah, cudaStream_t s) {
    L = L_;
    nb = nb_;
    nz = nz_;
    z.alloc(nz);
    W.alloc(nz);
    A.alloc((size_t)nz * L * L);
    ED_CUDA(cudaMemcpyAsync(z.p, zh, nz * sizeof(double2), cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(W.p, Wh, nz * sizeof(double), cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(A.p, Ah, (size_t)nz * L * L * sizeof(double2), cudaMemcpyHostToDevice, s));
  }
  void eval(int nc, const double* eps_h, const double* theta_h, double* d_h, double* grad_h, cudaStream_t s) {
    if (eps.n < (size_t)std::max(nc * nb, 1)) eps.alloc(std::max(nc * nb, 1));
    if (theta.n < (size_t)std::max(nc * L * nb, 1)) theta.alloc(std::max(nc * L * nb, 1));
    if (Gam.n < (size_t)nc * nz * L * L) Gam.alloc((size_t)nc * nz * L * L);
    if (d.n < (size_t)nc) d.alloc(nc);
    const int np = nb + L * nb;
    if (grad_h && grad.n < (size_t)std::max(nc * np, 1)) grad.alloc(std::max(nc * np, 1));
    if (nb) {
      ED_CUDA(cudaMemcpyAsync(eps.p, eps_h, (size_t)nc * nb * sizeof(double), cudaMemcpyHostToDevice, s));
      ED_CUDA(cudaMemcpyAsync(theta.p, theta_h, (size_t)nc * L * nb * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    {
      ProfScope ps_(K_LATTICE, s, 0.0);
      k_hybridization<<<lat_grid((int64_t)nc * nz * L * L, 256), 256, 0, s>>>(eps.p, theta.p, z.p, L, nb, nz, nc, Gam.p);
      ED_CHECK_LAUNCH();
    }
    {
      ProfScope ps_(K_LATTICE, s, 0.0);
      k_distance<<<nc, 256, 0, s>>>(A.p, Gam.p, W.p, L, nz, d.p);
      ED_CHECK_LAUNCH();
    }
    if (grad_h && np) {
      ProfScope ps_(K_LATTICE, s, 0.0);
      k_distance_grad<<<lat_grid((int64_t)nc * np, 128), 128, 0, s>>>(A.p, Gam.p, W.p, z.p, eps.p, theta.p, L, nb, nz, nc,
                                                                     grad.p);
      ED_CHECK_LAUNCH();
    }
    ED_CUDA(cudaMemcpyAsync(d_h, d.p, nc * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (grad_h && np)
      ED_CUDA(cudaMemcpyAsync(grad_h, grad.p, (size_t)nc * np * sizeof(double), cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
  }
};

static void check_bath_args(int L, int nb, const double* z, int nz, const double* W, const double* A) {
  require_lat(L >= 1 && L <= kLatMaxSites && nb >= 0, "need 1 <= n_sites <= 32 and n_bath >= 0");
  require_lat(nz >= 1 && z && W && A, "z, weights and A must not be NULL, nz >= 1");
  for (int n = 0; n < nz; ++n) require_lat(std::isfinite(W[n]) && W[n] >= 0.0, "weights must be finite and >= 0");
}

}  // namespace ed

using namespace ed;

extern "C" {

ed_status ed_hybridization(int n_sites, int n_bath, const double* eps, const double* theta, const double* z, int nz,
                           double* Gamma_out, int out_is_device) {
  return lat_guarded([&]() -> ed_status {
    require_lat(n_sites >= 1 && n_sites <= kLatMaxSites && n_bath >= 0, "need 1 <= n_sites <= 32 and n_bath >= 0");
    require_lat(z && Gamma_out && nz >= 1, "z and Gamma_out must not be NULL, nz >= 1");
    require_lat(n_bath == 0 || (eps && theta), "eps and theta must not be NULL when n_bath > 0");
    cudaStream_t s = cudaStreamPerThread;
    const int L = n_sites;
    const size_t n = (size_t)nz * L * L;
    DevBuf<double2> zd(nz), tmp;
    DevBuf<double> ed_(std::max(n_bath, 1)), td((size_t)std::max(L * n_bath, 1));
    ED_CUDA(cudaMemcpyAsync(zd.p, z, nz * sizeof(double2), cudaMemcpyHostToDevice, s));
    if (n_bath) {
      ED_CUDA(cudaMemcpyAsync(ed_.p, eps, n_bath * sizeof(double), cudaMemcpyHostToDevice, s));
      ED_CUDA(cudaMemcpyAsync(td.p, theta, (size_t)L * n_bath * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    double2* out = reinterpret_cast<double2*>(Gamma_out);
    if (!out_is_device) {
      tmp.alloc(n);
      out = tmp.p;
    }
    {
      ProfScope ps_(K_LATTICE, s, 0.0);
      k_hybridization<<<lat_grid((int64_t)n, 256), 256, 0, s>>>(ed_.p, td.p, zd.p, L, n_bath, nz, 1, out);
      ED_CHECK_LAUNCH();
    }
    if (!out_is_device) ED_CUDA(cudaMemcpyAsync(Gamma_out, tmp.p, n * sizeof(double2), cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    return ED_OK;
  });
}

ed_status ed_cpt_green(const ed_superlattice* lat, const double* Gc, const double* Gamma, int nz, const double* kt, int nk,
                       int mode, double* out, int io_is_device) {
  return lat_guarded([&]() -> ed_status {
    check_lattice(lat);
    require_lat(Gc && out && kt && nz >= 1 && nk >= 1, "Gc, kt and out must not be NULL, nz >= 1, nk >= 1");
    require_lat(mode == ED_CPT_MATRIX || mode == ED_CPT_PERIODIZED || mode == ED_CPT_AVERAGE, "unknown mode");
    cudaStream_t s = cudaStreamPerThread;
    const int L = lat->n_sites, D = lat->dim;
    LatticeDev d = upload_lattice(lat, s);
    DevBuf<double> kd((size_t)nk * D);
    ED_CUDA(cudaMemcpyAsync(kd.p, kt, (size_t)nk * D * sizeof(double), cudaMemcpyHostToDevice, s));
    DevBuf<double2> t1, t2, V, Gci, obuf;
    DevBuf<int> st(1);
    ED_CUDA(cudaMemsetAsync(st.p, 0, sizeof(int), s));
    const double2* Gcd = dev_in(Gc, (size_t)nz * L * L, io_is_device, t1, s);
    const double2* Gmd = dev_in(Gamma, (size_t)nz * L * L, io_is_device, t2, s);
    build_v(d, kd, nk, V, s);
    cluster_inverse(Gcd, Gmd, L, nz, Gci, st.p, s);
    const size_t nout = mode == ED_CPT_MATRIX ? (size_t)nk * nz * L * L
                                              : mode == ED_CPT_PERIODIZED ? (size_t)nk * nz : (size_t)nz * L * L;
    double2* o = reinterpret_cast<double2*>(out);
    if (!io_is_device) {
      obuf.alloc(nout);
      o = obuf.p;
    }
    if (mode == ED_CPT_AVERAGE) {
      const size_t smem = kLatWarps * warp_slice(L) + (size_t)kLatWarps * L * L * sizeof(double2);
      allow_max_dynamic_smem(k_cpt_average);
      ProfScope ps_(K_LATTICE, s, 0.0);
      k_cpt_average<<<(unsigned)std::min(nz, 152 * 8), 32 * kLatWarps, smem, s>>>(Gci.p, V.p, L, nz, nk, o, st.p);
      ED_CHECK_LAUNCH();
    } else {
      allow_max_dynamic_smem(k_cpt);
      ProfScope ps_(K_LATTICE, s, 0.0);
      k_cpt<<<lat_grid((int64_t)nk * nz, kLatWarps), 32 * kLatWarps, kLatWarps * warp_slice(L), s>>>(
          Gci.p, V.p, kd.p, d.pos.p, D, L, nz, nk, mode == ED_CPT_MATRIX ? 0 : 1, o, st.p);
      ED_CHECK_LAUNCH();
    }
    if (!io_is_device) ED_CUDA(cudaMemcpyAsync(out, o, nout * sizeof(double2), cudaMemcpyDeviceToHost, s));
    throw_singular(st.p, s);
    return ED_OK;
  });
}

ed_status ed_cdmft_target(const ed_superlattice* lat, const double* Gc, const double* Gamma, int nz, const double* kt,
                          int nk, double* A_out, int io_is_device) {
  return lat_guarded([&]() -> ed_status {
    check_lattice(lat);
    require_lat(Gc && A_out && kt && nz >= 1 && nk >= 1, "Gc, kt and A_out must not be NULL, nz >= 1, nk >= 1");
    cudaStream_t s = cudaStreamPerThread;
    const int L = lat->n_sites, D = lat->dim;
    const int64_t n = (int64_t)nz * L * L;
    LatticeDev d = upload_lattice(lat, s);
    DevBuf<double> kd((size_t)nk * D);
    ED_CUDA(cudaMemcpyAsync(kd.p, kt, (size_t)nk * D * sizeof(double), cudaMemcpyHostToDevice, s));
    DevBuf<double2> t1, t2, V, Gci, Gbar(n), Gbi(n), obuf;
    DevBuf<int> st(1);
    ED_CUDA(cudaMemsetAsync(st.p, 0, sizeof(int), s));
    const double2* Gcd = dev_in(Gc, n, io_is_device, t1, s);
    const double2* Gmd = dev_in(Gamma, n, io_is_device, t2, s);
    build_v(d, kd, nk, V, s);
    cluster_inverse(Gcd, Gmd, L, nz, Gci, st.p, s);  // G_c^-1 + Gamma
    {
      const size_t smem = kLatWarps * warp_slice(L) + (size_t)kLatWarps * L * L * sizeof(double2);
      allow_max_dynamic_smem(k_cpt_average);
      ProfScope ps_(K_LATTICE, s, 0.0);
      k_cpt_average<<<(unsigned)std::min(nz, 152 * 8), 32 * kLatWarps, smem, s>>>(Gci.p, V.p, L, nz, nk, Gbar.p, st.p);
      ED_CHECK_LAUNCH();
    }
    invert_batched(Gbar.p, nullptr, Gbi.p, L, nz, st.p, s);
    double2* o = reinterpret_cast<double2*>(A_out);
    if (!io_is_device) {
      obuf.alloc(n);
      o = obuf.p;
    }
    {
      ProfScope ps_(K_LATTICE, s, 0.0);
      k_add_sub<<<lat_grid(n, 256), 256, 0, s>>>(Gci.p, Gbi.p, -1.0, n, o);  // A = G_c^-1 + Gamma - G_bar^-1
      ED_CHECK_LAUNCH();
    }
    if (!io_is_device) ED_CUDA(cudaMemcpyAsync(A_out, o, n * sizeof(double2), cudaMemcpyDeviceToHost, s));
    throw_singular(st.p, s);
    return ED_OK;
  });
}

ed_status ed_cdmft_distance(int n_sites, int n_bath, int n_cand, const double* eps, const double* theta, const double* z,
                            int nz, const double* weights, const double* A, double* d_out, double* grad_out) {
  return lat_guarded([&]() -> ed_status {
    check_bath_args(n_sites, n_bath, z, nz, weights, A);
    require_lat(n_cand >= 1 && d_out, "n_cand >= 1 and d_out must not be NULL");
    require_lat(n_bath == 0 || (eps && theta), "eps and theta must not be NULL when n_bath > 0");
    cudaStream_t s = cudaStreamPerThread;
    DistanceWork w;
    w.setup(n_sites, n_bath, z, nz, weights, A, s);
    w.eval(n_cand, eps, theta, d_out, grad_out, s);
    return ED_OK;
  });
}

ed_status ed_cdmft_fit(int n_sites, int n_bath, double* eps, double* theta, const unsigned char* theta_free,
                       const double* z, int nz, const double* weights, const double* A, double gtol, int max_iter,
                       double* d_out, int* iters_out) {
  return lat_guarded([&]() -> ed_status {
    check_bath_args(n_sites, n_bath, z, nz, weights, A);
    require_lat(n_bath >= 1 && eps && theta, "a fit needs n_bath >= 1 and eps, theta");
    const int L = n_sites, nb = n_bath, np = nb + L * nb;
    // free parameters: every eps_a, and theta_{mu a} where theta_free says so (NULL: all)
    std::vector<int> idx;
    for (int a = 0; a < nb; ++a) idx.push_back(a);
    for (int q = 0; q < L * nb; ++q)
      if (!theta_free || theta_free[q]) idx.push_back(nb + q);
    const int m = (int)idx.size();
    cudaStream_t s = cudaStreamPerThread;
    DistanceWork w;
    w.setup(L, nb, z, nz, weights, A, s);
    std::vector<double> full(np), g(np);
    std::memcpy(full.data(), eps, nb * sizeof(double));
    std::memcpy(full.data() + nb, theta, (size_t)L * nb * sizeof(double));
    auto f = [&](const std::vector<double>& x, std::vector<double>& gx) {
      std::vector<double> p = full;
      for (int i = 0; i < m; ++i) p[idx[i]] = x[i];
      double d = 0.0;
      w.eval(1, p.data(), p.data() + nb, &d, g.data(), s);
      gx.resize(m);
      for (int i = 0; i < m; ++i) gx[i] = g[idx[i]];
      return d;
    };
    // BFGS with a backtracking (Armijo) line search on the free parameters
    std::vector<double> x(m), gx, xn(m), gn;
    for (int i = 0; i < m; ++i) x[i] = full[idx[i]];
    double fx = f(x, gx);
    std::vector<double> Hinv((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) Hinv[(size_t)i * m + i] = 1.0;
    const int maxit = max_iter > 0 ? max_iter : 500;
    const double gt = gtol > 0.0 ? gtol : 1e-10;
    int it = 0;
    for (; it < maxit; ++it) {
      double gnorm = 0.0;
      for (double v : gx) gnorm = std::max(gnorm, std::fabs(v));
      if (gnorm < gt || fx == 0.0) break;
      std::vector<double> p(m, 0.0);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) p[i] -= Hinv[(size_t)i * m + j] * gx[j];
      double slope = 0.0;
      for (int i = 0; i < m; ++i) slope += p[i] * gx[i];
      if (!(slope < 0.0)) {  // not a descent direction: restart from steepest descent
        std::fill(Hinv.begin(), Hinv.end(), 0.0);
        for (int i = 0; i < m; ++i) Hinv[(size_t)i * m + i] = 1.0, p[i] = -gx[i];
        slope = 0.0;
        for (int i = 0; i < m; ++i) slope += p[i] * gx[i];
      }
      double step = 1.0, fn = 0.0;
      bool accepted = false;
      for (int ls = 0; ls < 60; ++ls) {
        for (int i = 0; i < m; ++i) xn[i] = x[i] + step * p[i];
        fn = f(xn, gn);
        if (std::isfinite(fn) && fn <= fx + 1e-4 * step * slope) {
          accepted = true;
          break;
        }
        step *= 0.5;
      }
      if (!accepted) break;
      std::vector<double> sv(m), yv(m);
      double sy = 0.0;
      for (int i = 0; i < m; ++i) {
        sv[i] = xn[i] - x[i];
        yv[i] = gn[i] - gx[i];
        sy += sv[i] * yv[i];
      }
      const double frel = std::fabs(fx - fn) / std::max(1e-300, std::fabs(fx));
      x = xn;
      gx = gn;
      fx = fn;
      if (sy > 1e-300) {  // H <- (I - r s y^T) H (I - r y s^T) + r s s^T, r = 1 / (y^T s)
        const double r = 1.0 / sy;
        std::vector<double> Hy(m, 0.0);
        for (int i = 0; i < m; ++i)
          for (int j = 0; j < m; ++j) Hy[i] += Hinv[(size_t)i * m + j] * yv[j];
        double yHy = 0.0;
        for (int i = 0; i < m; ++i) yHy += yv[i] * Hy[i];
        for (int i = 0; i < m; ++i)
          for (int j = 0; j < m; ++j)
            Hinv[(size_t)i * m + j] += -r * (Hy[i] * sv[j] + sv[i] * Hy[j]) + (r * r * yHy + r) * sv[i] * sv[j];
      }
      if (frel < 1e-15) break;
    }
    for (int i = 0; i < m; ++i) full[idx[i]] = x[i];
    std::memcpy(eps, full.data(), nb * sizeof(double));
    std::memcpy(theta, full.data() + nb, (size_t)L * nb * sizeof(double));
    if (d_out) *d_out = fx;
    if (iters_out) *iters_out = it;
    return ED_OK;
  });
}

}  // extern "C"
