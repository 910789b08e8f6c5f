// Cluster symmetries (Sec. 4.5): the Hamiltonian restricted to one irreducible representation of
// an Abelian symmetry group, in the basis of symmetrized states, and its ground state.
//
// The group is Abelian, generated by commuting, independent permutations g_j of the orbitals of
// orders n_j (mirrors and two-fold rotations: n_j = 2; four-fold rotations, translations of a
// periodic cluster: n_j = 4, 6, ...), at most 32 elements.  An irrep is named by exponents m_j;
// the element prod_j g_j^{a_j} has the character exp(2 pi i sum_j m_j a_j / n_j).  With only
// +-1 characters the irrep's matrix is real symmetric; otherwise it is complex Hermitian and the
// matrix and every vector hold interleaved (real, imaginary) pairs.
//
// Basis (Sec. 4.5): the binary states (b_up, b_dn) of the sector are grouped into orbits; the
// member with the smallest key b_up 2^L + b_dn represents its orbit, and its symmetrized state
// sum_g chi_g g|r> is kept unless it vanishes (chi_g phi_g(r) = -1 for some g of the stabilizer).
// phi_g(b) is the fermionic sign of moving the creation operators of b to their images: the
// parity of the inversions of the permutation among the occupied orbitals of each spin.  One
// thread tests one binary state; blocks own contiguous ranges of the sector and write their
// representatives in order, so the list comes out sorted by key (the index function of Sec. 4.5
// is then a binary search in it).
//
// Matrix (Eq. matrixElement for normalized states): applying every term of H to a representative
// r gives binary states b_k with amplitudes h_k; with g_k b_k = r_k,
//   <psi(r_k)| H |psi(r)> += h_k phi_{g_k}(b_k) chi_{g_k}^* sqrt(|S_{r_k}| / |S_r|).
// The entries generated from r are stored, conjugated (H is Hermitian), as row r.  A row's
// terms are merged in a thread's local buffer before they are stored, which carries out the
// cancellations that Sec. 4.5 mentions; entries below 1e-13 in magnitude are dropped.  The matrix
// is built twice, counting then filling (the paper stores H once the basis is symmetrized).
//
// Ground state: FP64 Lanczos (Sec. 4.2) on the stored matrix, scalars on the device, checked every
// kSymCheck steps with the block tridiagonal solver; the ground vector is rebuilt by retracing the
// recursion, then restarted from itself until the FP64 residual |H w - E w| reaches
// 1e-12 max(1, |E|).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <vector>

#include "ed_common.cuh"

namespace ed {

constexpr int kSymMaxGen = 5;        // |G| <= 32
constexpr int kSymMaxTerms = 2 * kMaxHops + 1;
constexpr int kSymThreads = 256;
constexpr int kSymChunk = 64 * kSymThreads;  // binary states per block of the basis kernels
constexpr int kSymCheck = 10;
constexpr int kSymRounds = 6;

// Device copy of the group and the model terms that the kernels read.
struct SymDev {
  int L, ng;
  int n_pairs;
  uint8_t perm[1 << kSymMaxGen][kMaxOrb];     // orbital images of every element
  uint32_t inv[1 << kSymMaxGen][kMaxOrb];     // inv[g][i]: orbitals j > i with perm(j) < perm(i)
  double chr[1 << kSymMaxGen], chi[1 << kSymMaxGen];  // character of every element: real, imaginary part
  double hdiag[kMaxOrb];
  double U[kMaxOrb];
  int pa[kMaxPairs], pb[kMaxPairs];           // ordered hopping pairs (a <- b), h_ab != 0
  double pv[kMaxPairs];
};

__device__ __forceinline__ uint32_t sym_move(const uint8_t* p, uint32_t b) {
  uint32_t o = 0;
  while (b) {
    const int i = __ffs(b) - 1;
    b &= b - 1u;
    o |= 1u << p[i];
  }
  return o;
}
__device__ __forceinline__ int sym_parity(const uint32_t* inv, uint32_t b) {
  int par = 0;
  uint32_t x = b;
  while (x) {
    const int i = __ffs(x) - 1;
    x &= x - 1u;
    par ^= __popc(b & inv[i]) & 1;
  }
  return par;
}
__device__ __forceinline__ uint64_t sym_key(uint32_t bu, uint32_t bd, int L) { return ((uint64_t)bu << L) | bd; }

// Is (bu, bd) the representative of a non-vanishing symmetrized state?  Also its stabilizer size.
__device__ bool sym_is_rep(const SymDev& G, uint32_t bu, uint32_t bd, int* stab) {
  const uint64_t k = sym_key(bu, bd, G.L);
  int s = 0;
  for (int g = 0; g < G.ng; ++g) {
    const uint64_t gk = sym_key(sym_move(G.perm[g], bu), sym_move(G.perm[g], bd), G.L);
    if (gk < k) return false;
    if (gk == k) {
      ++s;
      // non-vanishing iff chi_g = phi_g(r) on the stabilizer
      const int ph = sym_parity(G.inv[g], bu) ^ sym_parity(G.inv[g], bd);
      if (fabs(G.chr[g] - (ph ? -1.0 : 1.0)) > 1e-9 || fabs(G.chi[g]) > 1e-9) return false;
    }
  }
  *stab = s;
  return true;
}

// Representative key of the orbit of (bu, bd) and the factor phi_g(b) chi_g^* (real fr, imaginary
// fi) of the first element (in element order) that reaches it (P g = chi_g P for the projector
// P = (1/|G|) sum_g chi_g^* g).
__device__ void sym_rep(const SymDev& G, uint32_t bu, uint32_t bd, uint64_t* rk, double* fr, double* fi) {
  uint64_t best = ~0ull;
  double r = 1.0, i = 0.0;
  for (int g = 0; g < G.ng; ++g) {
    const uint32_t gu = sym_move(G.perm[g], bu), gd = sym_move(G.perm[g], bd);
    const uint64_t gk = sym_key(gu, gd, G.L);
    if (gk < best) {
      best = gk;
      const double ph = (sym_parity(G.inv[g], bu) ^ sym_parity(G.inv[g], bd)) ? -1.0 : 1.0;
      r = ph * G.chr[g];
      i = -ph * G.chi[g];
    }
  }
  *rk = best;
  *fr = r;
  *fi = i;
}

// ---- basis: count, then write, the representatives of every chunk of the sector in order
__global__ void __launch_bounds__(kSymThreads) k_sym_basis(const SymDev* __restrict__ Gp, const uint32_t* __restrict__ Bu,
                                                          const uint32_t* __restrict__ Bd, int64_t du, int64_t dd,
                                                          int64_t* __restrict__ count, const int64_t* __restrict__ offset,
                                                          uint64_t* __restrict__ keys, uint8_t* __restrict__ stab) {
  __shared__ SymDev G;
  __shared__ int s_warp[kSymThreads / 32];
  __shared__ int64_t s_base;
  for (int i = threadIdx.x; i < (int)(sizeof(SymDev) / 4); i += blockDim.x)
    reinterpret_cast<int*>(&G)[i] = reinterpret_cast<const int*>(Gp)[i];
  if (threadIdx.x == 0) s_base = offset ? offset[blockIdx.x] : 0;
  __syncthreads();
  const int64_t n = du * dd;
  const int64_t c0 = (int64_t)blockIdx.x * kSymChunk;
  const int64_t c1 = c0 + kSymChunk < n ? c0 + kSymChunk : n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t total = 0;
  for (int64_t i0 = c0; i0 < c1; i0 += kSymThreads) {
    const int64_t i = i0 + threadIdx.x;
    int st = 0;
    bool rep = false;
    uint32_t bu = 0, bd = 0;
    if (i < c1) {
      const int64_t u = i / dd, d = i - u * dd;
      bu = Bu[u];
      bd = Bd[d];
      rep = sym_is_rep(G, bu, bd, &st);
    }
    // ordered compaction: ranks within the warp, then across warps
    const unsigned m = __ballot_sync(0xffffffffu, rep);
    if (lane == 0) s_warp[warp] = __popc(m);
    __syncthreads();
    int before = 0, tot = 0;
    for (int w = 0; w < kSymThreads / 32; ++w) {
      before += w < warp ? s_warp[w] : 0;
      tot += s_warp[w];
    }
    if (offset && rep) {
      const int64_t o = s_base + total + before + __popc(m & ((1u << lane) - 1u));
      keys[o] = sym_key(bu, bd, G.L);
      stab[o] = (uint8_t)st;
    }
    total += tot;
    __syncthreads();
  }
  if (!offset && threadIdx.x == 0) count[blockIdx.x] = total;
}

__device__ __forceinline__ int64_t sym_find(const uint64_t* __restrict__ keys, int64_t dim, uint64_t k) {
  int64_t lo = 0, hi = dim;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (keys[mid] < k)
      lo = mid + 1;
    else
      hi = mid;
  }
  return (lo < dim && keys[lo] == k) ? lo : -1;
}

// The merged entries of row r (columns ascending); returns their number.  CPLX: val holds
// interleaved (real, imaginary) pairs.
template <bool CPLX>
__device__ int sym_row(const SymDev& G, const uint64_t* __restrict__ keys, const uint8_t* __restrict__ stab, int64_t dim,
                       int64_t r, int32_t* col, double* val) {
  constexpr int W = CPLX ? 2 : 1;
  const uint64_t k = keys[r];
  const uint32_t bu = (uint32_t)(k >> G.L), bd = (uint32_t)(k & ((G.L == 32) ? 0xFFFFFFFFull : ((1ull << G.L) - 1ull)));
  const double sr = (double)stab[r];
  int n = 0;
  double diag = 0.0;
  for (int a = 0; a < G.L; ++a) {
    diag += G.hdiag[a] * (double)(((bu >> a) & 1u) + ((bd >> a) & 1u));
    if ((bu >> a) & (bd >> a) & 1u) diag += G.U[a];
  }
  col[n] = (int32_t)r;
  val[W * n] = diag;
  if (CPLX) val[W * n + 1] = 0.0;
  ++n;
  for (int p = 0; p < G.n_pairs; ++p) {
    const int a = G.pa[p], b = G.pb[p];
    const uint32_t lo = (uint32_t)min(a, b), hi = (uint32_t)max(a, b);
    const uint32_t between = (hi >= 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u)) ^ ((1u << lo) - 1u) ^ (1u << lo);
    for (int spin = 0; spin < 2; ++spin) {
      const uint32_t bs = spin ? bd : bu;
      if (!((bs >> b) & 1u) || ((bs >> a) & 1u)) continue;
      const uint32_t nb = bs ^ (1u << a) ^ (1u << b);
      const int jw = __popc(bs & between) & 1;
      uint64_t rk;
      double fr, fi;
      sym_rep(G, spin ? bu : nb, spin ? nb : bd, &rk, &fr, &fi);
      const int64_t c = sym_find(keys, dim, rk);
      if (c < 0 || n >= kSymMaxTerms) continue;
      const double amp = G.pv[p] * (jw ? -1.0 : 1.0) * sqrt((double)stab[c] / sr);
      // this term is <psi(c)| H |psi(r)>; row r stores its conjugate <psi(r)| H |psi(c)>
      col[n] = (int32_t)c;
      val[W * n] = amp * fr;
      if (CPLX) val[W * n + 1] = -amp * fi;
      ++n;
    }
  }
  // sort by column (insertion: rows hold a few dozen terms), merge, drop cancelled entries
  for (int i = 1; i < n; ++i) {
    const int32_t cc = col[i];
    const double vr = val[W * i], vi = CPLX ? val[W * i + 1] : 0.0;
    int j = i - 1;
    while (j >= 0 && col[j] > cc) {
      col[j + 1] = col[j];
      val[W * (j + 1)] = val[W * j];
      if (CPLX) val[W * (j + 1) + 1] = val[W * j + 1];
      --j;
    }
    col[j + 1] = cc;
    val[W * (j + 1)] = vr;
    if (CPLX) val[W * (j + 1) + 1] = vi;
  }
  int m = 0;
  for (int i = 0; i < n;) {
    const int32_t cc = col[i];
    double sr_ = 0.0, si_ = 0.0;
    while (i < n && col[i] == cc) {
      sr_ += val[W * i];
      if (CPLX) si_ += val[W * i + 1];
      ++i;
    }
    if (hypot(sr_, si_) >= 1e-13) {
      col[m] = cc;
      val[W * m] = sr_;
      if (CPLX) val[W * m + 1] = si_;
      ++m;
    }
  }
  return m;
}

template <bool CPLX>
__global__ void __launch_bounds__(128) k_sym_rows(const SymDev* __restrict__ Gp, const uint64_t* __restrict__ keys,
                                                  const uint8_t* __restrict__ stab, int64_t dim,
                                                  int64_t* __restrict__ rowptr, int32_t* __restrict__ colo,
                                                  double* __restrict__ valo, int fill) {
  constexpr int W = CPLX ? 2 : 1;
  __shared__ SymDev G;
  for (int i = threadIdx.x; i < (int)(sizeof(SymDev) / 4); i += blockDim.x)
    reinterpret_cast<int*>(&G)[i] = reinterpret_cast<const int*>(Gp)[i];
  __syncthreads();
  int32_t col[kSymMaxTerms];
  double val[W * kSymMaxTerms];
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < dim; r += (int64_t)gridDim.x * blockDim.x) {
    const int m = sym_row<CPLX>(G, keys, stab, dim, r, col, val);
    if (!fill) {
      rowptr[r] = m;
    } else {
      const int64_t o = rowptr[r];
      for (int i = 0; i < m; ++i) {
        colo[o + i] = col[i];
        valo[W * (o + i)] = val[W * i];
        if (CPLX) valo[W * (o + i) + 1] = val[W * i + 1];
      }
    }
  }
}

// The last block of a launch to finish (a ticket) sums the per-block partials in a fixed order
// (thread t takes blocks t, t + blockDim.x, ..., then a tree in shared memory) into *out (mode 1:
// its square root) and resets the ticket, so a reduction needs no second launch.
__device__ void sym_finish_last(const double* partial, double* out, int mode, unsigned* ticket) {
  __shared__ bool s_last;
  __shared__ double sm[kSymThreads];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double t = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) t += __ldcg(partial + b);
  sm[threadIdx.x] = t;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *out = mode ? sqrt(fmax(sm[0], 0.0)) : sm[0];
    *ticket = 0u;
  }
}

// ---- y = H x - beta x_prev (x_prev may be NULL); per-block partial <x, y>.  Rows hold ~20
// entries, so a row goes to a group of kSymRowLanes lanes (four rows per warp), each lane taking
// every kSymRowLanes-th entry, summed by a fixed butterfly.
constexpr int kSymRowLanes = 8;
constexpr int kSymRowsPerBlock = kSymThreads / kSymRowLanes;

template <bool CPLX>
__global__ void __launch_bounds__(kSymThreads) k_sym_spmv(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                         const double* __restrict__ val, int64_t dim,
                                                         const double* __restrict__ x, double* __restrict__ y,
                                                         const double* __restrict__ xprev, const double* __restrict__ beta,
                                                         double* __restrict__ partial, unsigned* ticket, double* out) {
  // CPLX: val, x, y, xprev hold interleaved (real, imaginary) pairs; the partial is Re <x, y>
  __shared__ double s_part[kSymRowsPerBlock];
  const int sub = threadIdx.x & (kSymRowLanes - 1), grp = threadIdx.x / kSymRowLanes;
  const double b = (xprev && beta) ? *beta : 0.0;
  double dot = 0.0;
  for (int64_t r0 = (int64_t)blockIdx.x * kSymRowsPerBlock; r0 < dim; r0 += (int64_t)gridDim.x * kSymRowsPerBlock) {
    const int64_t r = r0 + grp;
    double sr = 0.0, si = 0.0;
    if (r < dim) {
      const int64_t e = rowptr[r + 1];
      for (int64_t k = rowptr[r] + sub; k < e; k += kSymRowLanes) {
        if constexpr (CPLX) {
          const double2 v = reinterpret_cast<const double2*>(val)[k];
          const double2 xv = __ldg(reinterpret_cast<const double2*>(x) + col[k]);
          sr += v.x * xv.x - v.y * xv.y;
          si += v.x * xv.y + v.y * xv.x;
        } else {
          sr += val[k] * __ldg(x + col[k]);
        }
      }
    }
#pragma unroll
    for (int o = kSymRowLanes / 2; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      if (CPLX) si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (r < dim && sub == 0) {
      if constexpr (CPLX) {
        if (xprev) {
          sr -= b * xprev[2 * r];
          si -= b * xprev[2 * r + 1];
        }
        y[2 * r] = sr;
        y[2 * r + 1] = si;
        dot += sr * x[2 * r] + si * x[2 * r + 1];
      } else {
        if (xprev) sr -= b * xprev[r];
        y[r] = sr;
        dot += sr * x[r];
      }
    }
  }
  if (sub == 0) s_part[grp] = dot;
  __syncthreads();
  if (threadIdx.x == 0 && partial) {
    double t = 0.0;
    for (int w = 0; w < kSymRowsPerBlock; ++w) t += s_part[w];
    partial[blockIdx.x] = t;
  }
  if (ticket) sym_finish_last(partial, out, 0, ticket);
}

// out = sum of partials in a fixed order (one block); mode 0: out = s, 1: out = sqrt(max(s, 0))
__global__ void k_sym_finish(const double* __restrict__ partial, int n, double* __restrict__ out, int mode) {
  __shared__ double sm[kSymThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = mode ? sqrt(fmax(sm[0], 0.0)) : sm[0];
}

// w -= a x (a = *alpha, or 0 when alpha is NULL); per-block partial |w|^2
__global__ void __launch_bounds__(kSymThreads) k_sym_axpy_norm(double* __restrict__ w, const double* __restrict__ x,
                                                              const double* __restrict__ alpha, int64_t dim,
                                                              double* __restrict__ partial, unsigned* ticket = nullptr,
                                                              double* out = nullptr) {
  __shared__ double sm[kSymThreads];
  const double a = alpha ? *alpha : 0.0;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = alpha ? w[i] - a * x[i] : w[i];
    if (alpha) w[i] = v;
    s += v * v;
  }
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
  if (ticket) sym_finish_last(partial, out, 1, ticket);
}

// v = w / *norm (written over v); omega += coef * v when omega is given
__global__ void k_sym_scale(double* __restrict__ v, const double* __restrict__ w, const double* __restrict__ norm, int64_t dim,
                            double* __restrict__ omega, const double* __restrict__ coef) {
  const double nb = *norm;
  const double f = nb > 0.0 ? 1.0 / nb : 0.0;
  const double cf = omega ? *coef : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = w[i] * f;
    v[i] = x;
    if (omega) omega[i] += cf * x;
  }
}

__device__ __forceinline__ uint64_t sym_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void k_sym_start(double* __restrict__ v, int64_t dim, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = 2.0 * ((double)(sym_splitmix64(seed ^ (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// ---- Green functions with symmetrized operators (Sec. 4.6)
//
// phi = c+_rho Omega (create = 1) or c_rho Omega (create = 0) for c_rho = sum_a m[a] c_{a spin}, in
// pull form over the target irrep's representatives r': the binary state b = c_a r' (create) or
// c+_a r' (annihilate) has the Jordan-Wigner sign (-1)^(occupied modes before mode a), its
// representative r in the source irrep (of Omega) carries phi_g(b) chi_g, and
//   phi[r'] = sum_a m[a] sign_a phi_g(b) chi_g sqrt(|S_r| / |S_r'|) Omega[r]
// (the projector relation c_rho P_alpha' = P_alpha c_rho for +-1 characters, alpha' = alpha beta).
__global__ void __launch_bounds__(128) k_sym_apply(const SymDev* __restrict__ Gsrc, const uint64_t* __restrict__ src_keys,
                                                   const uint8_t* __restrict__ src_stab, int64_t src_dim,
                                                   const double* __restrict__ omega, const uint64_t* __restrict__ tgt_keys,
                                                   const uint8_t* __restrict__ tgt_stab, int64_t tgt_dim,
                                                   const double* __restrict__ m, int create, int spin,
                                                   double* __restrict__ out) {
  __shared__ SymDev G;
  for (int i = threadIdx.x; i < (int)(sizeof(SymDev) / 4); i += blockDim.x)
    reinterpret_cast<int*>(&G)[i] = reinterpret_cast<const int*>(Gsrc)[i];
  __syncthreads();
  const uint64_t lmask = (G.L == 32) ? 0xFFFFFFFFull : ((1ull << G.L) - 1ull);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < tgt_dim; r += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = tgt_keys[r];
    const uint32_t bu = (uint32_t)(k >> G.L), bd = (uint32_t)(k & lmask);
    const double st = (double)tgt_stab[r];
    double acc = 0.0;
    for (int a = 0; a < G.L; ++a) {
      const double w = m[a];
      if (w == 0.0) continue;
      const uint32_t bs = spin ? bd : bu;
      const bool occ = (bs >> a) & 1u;
      if (create ? !occ : occ) continue;
      const uint32_t nb = bs ^ (1u << a);
      const int before = spin ? __popc(bu) + __popc(bd & ((1u << a) - 1u)) : __popc(bu & ((1u << a) - 1u));
      uint64_t rk;
      double f, fi;
      sym_rep(G, spin ? bu : nb, spin ? nb : bd, &rk, &f, &fi);  // +-1 characters here: fi = 0
      const int64_t c = sym_find(src_keys, src_dim, rk);
      if (c < 0) continue;
      acc += w * ((before & 1) ? -1.0 : 1.0) * f * sqrt((double)src_stab[c] / st) * omega[c];
    }
    out[r] = acc;
  }
}

// The same with complex weights and characters (any Abelian group): phi = O Omega for
// O = sum_a w[a] c+_a (create) or sum_a w[a] c_a, w interleaved (real, imaginary) over the L
// orbitals; the target irrep's vector is complex (interleaved), Omega is complex when SRC_CPLX.
// <b| psi_S(r)> = phi_g(b) chi_S(g) (|S_r| / |G|)^(1/2) for g b = r, so every term carries the
// conjugate of the factor phi_g(b) chi_S(g)^* that sym_rep returns:
//   phi[r'] = sum_a w[a] sign_a phi_g(b) chi_S(g) sqrt(|S_r| / |S_r'|) Omega[r].
template <bool SRC_CPLX>
__global__ void __launch_bounds__(128) k_sym_apply_c(const SymDev* __restrict__ Gsrc, const uint64_t* __restrict__ src_keys,
                                                     const uint8_t* __restrict__ src_stab, int64_t src_dim,
                                                     const double* __restrict__ omega, const uint64_t* __restrict__ tgt_keys,
                                                     const uint8_t* __restrict__ tgt_stab, int64_t tgt_dim,
                                                     const double* __restrict__ w, int create, int spin,
                                                     double* __restrict__ out) {
  __shared__ SymDev G;
  for (int i = threadIdx.x; i < (int)(sizeof(SymDev) / 4); i += blockDim.x)
    reinterpret_cast<int*>(&G)[i] = reinterpret_cast<const int*>(Gsrc)[i];
  __syncthreads();
  const uint64_t lmask = (G.L == 32) ? 0xFFFFFFFFull : ((1ull << G.L) - 1ull);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < tgt_dim; r += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = tgt_keys[r];
    const uint32_t bu = (uint32_t)(k >> G.L), bd = (uint32_t)(k & lmask);
    const double st = (double)tgt_stab[r];
    double ar = 0.0, ai = 0.0;
    for (int a = 0; a < G.L; ++a) {
      const double wr = w[2 * a], wi = w[2 * a + 1];
      if (wr == 0.0 && wi == 0.0) continue;
      const uint32_t bs = spin ? bd : bu;
      const bool occ = (bs >> a) & 1u;
      if (create ? !occ : occ) continue;
      const uint32_t nb = bs ^ (1u << a);
      const int before = spin ? __popc(bu) + __popc(bd & ((1u << a) - 1u)) : __popc(bu & ((1u << a) - 1u));
      uint64_t rk;
      double fr, fi;
      sym_rep(G, spin ? bu : nb, spin ? nb : bd, &rk, &fr, &fi);
      const int64_t c = sym_find(src_keys, src_dim, rk);
      if (c < 0) continue;
      const double amp = ((before & 1) ? -1.0 : 1.0) * sqrt((double)src_stab[c] / st);
      // t = w[a] * conj(f) * amp
      const double tr = amp * (wr * fr + wi * fi), ti = amp * (wi * fr - wr * fi);
      const double orr = SRC_CPLX ? omega[2 * c] : omega[c], oi = SRC_CPLX ? omega[2 * c + 1] : 0.0;
      ar += tr * orr - ti * oi;
      ai += tr * oi + ti * orr;
    }
    out[2 * r] = ar;
    out[2 * r + 1] = ai;
  }
}

// out[iz] += coef * b0sq / (z - s (a_0 - E0) - b_1^2 / (z - s (a_1 - E0) - ...)), n levels, s = +1
// for the electron part and -1 for the hole part (Eq. jacobi with the E0 shift); z = zr + i zi.
__global__ void k_sym_cf_eval(const double* __restrict__ alpha, const double* __restrict__ beta, int n, double E0,
                              double b0sq, double s, const double* __restrict__ zr, const double* __restrict__ zi,
                              int nz, double coef, double2* __restrict__ out) {
  for (int iz = blockIdx.x * blockDim.x + threadIdx.x; iz < nz; iz += gridDim.x * blockDim.x) {
    double gr = 0.0, gi = 0.0;  // the tail 1 / (z - ...) built from the last level up
    for (int j = n - 1; j >= 0; --j) {
      const double b2 = j + 1 < n ? beta[j + 1] * beta[j + 1] : 0.0;
      const double dr = zr[iz] - s * (alpha[j] - E0) - b2 * gr;
      const double di = zi[iz] - b2 * gi;
      const double den = dr * dr + di * di;
      gr = dr / den;
      gi = -di / den;
    }
    out[iz].x += coef * b0sq * gr;
    out[iz].y += coef * b0sq * gi;
  }
}

}  // namespace ed

// ---------------------------------------------------------------- the handle
struct ed_sym {
  ed_cluster* c = nullptr;
  int n_gen = 0;
  int n_up = 0, n_dn = 0;     // the sector
  std::vector<int> orders;   // order n_k of every generator
  std::vector<int> irrep;    // exponents m_k: chi(g_a) = exp(2 pi i sum m_k a_k / n_k)
  bool cplx = false;         // some character is complex, or force_cplx: complex matrix and vectors
  bool force_cplx = false;   // complex storage even with real characters (targets of a complex G)
  std::vector<int> perm;     // n_gen x L generator images
  ed::SymDev host;           // host copy of the group (characters of this irrep)
  ed::DevBuf<ed::SymDev> G;
  int64_t dim = 0, nnz = 0;
  ed::DevBuf<uint64_t> keys;
  ed::DevBuf<uint8_t> stab;
  ed::DevBuf<int64_t> rowptr;
  ed::DevBuf<int32_t> col;
  ed::DevBuf<double> val;
  ed::DevBuf<double> omega;  // ground state in the symmetrized basis
  bool have_gs = false;
  double E0 = 0.0, residual = 0.0;
  int iters = 0;             // Lanczos steps of the last ground-state search
};

namespace ed {

static int sym_grid(int64_t n, int per) {
  const int64_t b = (n + per - 1) / per;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

static void sym_build(ed_sym& S, const int* perm, cudaStream_t s) {
  ed_cluster& c = *S.c;
  const ModelHost& m = c.model;
  const int L = m.L, k = S.n_gen;
  SymDev h;
  std::memset(&h, 0, sizeof(h));
  h.L = L;
  h.ng = 1;
  for (int j = 0; j < k; ++j) h.ng *= S.orders[j];
  S.cplx = S.force_cplx;
  for (int g = 0; g < h.ng; ++g) {
    // element g_a = prod_j g_j^{a_j}, a the mixed-radix digits of g (first generator fastest)
    std::vector<int> p(L);
    std::iota(p.begin(), p.end(), 0);
    double phase = 0.0;  // sum_j m_j a_j / n_j
    for (int j = 0, rest = g; j < k; rest /= S.orders[j], ++j) {
      const int aj = rest % S.orders[j];
      for (int t = 0; t < aj; ++t)
        for (int i = 0; i < L; ++i) p[i] = perm[j * L + p[i]];
      phase += (double)S.irrep[j] * aj / S.orders[j];
    }
    for (int i = 0; i < L; ++i) {
      h.perm[g][i] = (uint8_t)p[i];
      uint32_t inv = 0;
      for (int jj = i + 1; jj < L; ++jj)
        if (p[jj] < p[i]) inv |= 1u << jj;
      h.inv[g][i] = inv;
    }
    // exact values on the real axis (the +-1 characters of involutions stay exact)
    const double f = phase - std::floor(phase);
    if (f == 0.0) {
      h.chr[g] = 1.0, h.chi[g] = 0.0;
    } else if (f == 0.5) {
      h.chr[g] = -1.0, h.chi[g] = 0.0;
    } else {
      h.chr[g] = std::cos(2.0 * M_PI * f);
      h.chi[g] = std::sin(2.0 * M_PI * f);
      S.cplx = true;
    }
  }
  for (int a = 0; a < L; ++a) {
    h.hdiag[a] = m.h[(size_t)a * L + a];
    h.U[a] = m.U[a];
  }
  h.n_pairs = (int)m.pair_a.size();
  for (int p = 0; p < h.n_pairs; ++p) {
    h.pa[p] = m.pair_a[p];
    h.pb[p] = m.pair_b[p];
    h.pv[p] = m.h[(size_t)m.pair_a[p] * L + m.pair_b[p]];
  }
  S.host = h;
  S.G.alloc(1);
  ED_CUDA(cudaMemcpyAsync(S.G.p, &S.host, sizeof(SymDev), cudaMemcpyHostToDevice, s));

  SpinTables& tu = c.tables(S.n_up);
  SpinTables& td = c.tables(S.n_dn);
  const int64_t du = tu.dim, dd = td.dim, n = du * dd;
  const int nblk = (int)((n + kSymChunk - 1) / kSymChunk);
  DevBuf<int64_t> cnt(nblk), off(nblk);
  k_sym_basis<<<nblk, kSymThreads, 0, s>>>(S.G.p, tu.basis.p, td.basis.p, du, dd, cnt.p, nullptr, nullptr, nullptr);
  ED_CHECK_LAUNCH();
  std::vector<int64_t> hc(nblk), ho(nblk);
  ED_CUDA(cudaMemcpyAsync(hc.data(), cnt.p, nblk * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  ED_CUDA(cudaStreamSynchronize(s));
  int64_t tot = 0;
  for (int b = 0; b < nblk; ++b) ho[b] = tot, tot += hc[b];
  if (tot >= ((int64_t)1 << 31)) throw Error(ED_ERR_INVALID, "symmetrized sector larger than 2^31 states");
  S.dim = tot;
  S.keys.alloc(std::max<int64_t>(tot, 1));
  S.stab.alloc(std::max<int64_t>(tot, 1));
  ED_CUDA(cudaMemcpyAsync(off.p, ho.data(), nblk * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  k_sym_basis<<<nblk, kSymThreads, 0, s>>>(S.G.p, tu.basis.p, td.basis.p, du, dd, nullptr, off.p, S.keys.p, S.stab.p);
  ED_CHECK_LAUNCH();
  S.rowptr.alloc(tot + 1);
  if (tot == 0) {
    ED_CUDA(cudaMemsetAsync(S.rowptr.p, 0, sizeof(int64_t), s));
    S.nnz = 0;
    return;
  }
  if (S.cplx)
    k_sym_rows<true><<<sym_grid(tot, 128), 128, 0, s>>>(S.G.p, S.keys.p, S.stab.p, tot, S.rowptr.p, nullptr, nullptr, 0);
  else
    k_sym_rows<false><<<sym_grid(tot, 128), 128, 0, s>>>(S.G.p, S.keys.p, S.stab.p, tot, S.rowptr.p, nullptr, nullptr, 0);
  ED_CHECK_LAUNCH();
  std::vector<int64_t> rp(tot + 1);
  ED_CUDA(cudaMemcpyAsync(rp.data(), S.rowptr.p, tot * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  ED_CUDA(cudaStreamSynchronize(s));
  int64_t acc = 0;
  for (int64_t r = 0; r < tot; ++r) {
    const int64_t v = rp[r];
    rp[r] = acc;
    acc += v;
  }
  rp[tot] = acc;
  S.nnz = acc;
  ED_CUDA(cudaMemcpyAsync(S.rowptr.p, rp.data(), (tot + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  S.col.alloc(std::max<int64_t>(acc, 1));
  S.val.alloc(std::max<int64_t>(acc, 1) * (S.cplx ? 2 : 1));
  if (S.cplx)
    k_sym_rows<true><<<sym_grid(tot, 128), 128, 0, s>>>(S.G.p, S.keys.p, S.stab.p, tot, S.rowptr.p, S.col.p, S.val.p, 1);
  else
    k_sym_rows<false><<<sym_grid(tot, 128), 128, 0, s>>>(S.G.p, S.keys.p, S.stab.p, tot, S.rowptr.p, S.col.p, S.val.p, 1);
  ED_CHECK_LAUNCH();
  ED_CUDA(cudaStreamSynchronize(s));
}

// y = H x in the symmetrized basis (device vectors of S.dim values: doubles, or interleaved
// complex pairs when a character is complex)
static void sym_spmv(ed_sym& S, const double* x, double* y, const double* xprev, const double* beta, double* partial,
                     int nblk, cudaStream_t s, unsigned* ticket = nullptr, double* out = nullptr) {
  const double w = S.cplx ? 2.0 : 1.0;
  ProfScope ps_(K_HPSI, s, (double)S.nnz * (4.0 + 8.0 * w) + (double)S.dim * 16.0 * w);
  if (S.cplx)
    k_sym_spmv<true><<<nblk, kSymThreads, 0, s>>>(S.rowptr.p, S.col.p, S.val.p, S.dim, x, y, xprev, beta, partial, ticket,
                                                  out);
  else
    k_sym_spmv<false><<<nblk, kSymThreads, 0, s>>>(S.rowptr.p, S.col.p, S.val.p, S.dim, x, y, xprev, beta, partial, ticket,
                                                   out);
  ED_CHECK_LAUNCH();
}

// FP64 Lanczos ground state of the symmetrized sector (see the header).
static void sym_ground_state(ed_sym& S, double tol, int max_iter, uint64_t seed) {
  cudaStream_t s = S.c->stream;
  const int64_t dim = S.dim, vlen = S.cplx ? 2 * dim : dim;  // vectors: doubles, or interleaved complex
  if (vlen == 0) throw Error(ED_ERR_INVALID, "the irrep has no state in this sector");
  const int M = std::max(2, (int)std::min<int64_t>(max_iter > 0 ? max_iter : 600, dim));
  const int nb = sym_grid(dim, kSymRowsPerBlock), nv = sym_grid(vlen, kSymThreads * 4);
  const int np = std::max(nb, nv);
  DevBuf<double> V0(vlen), V1(vlen), W(vlen), start(vlen), alpha(M + 1), beta(M + 2), evals(3), svec(M + 1), part(np),
      part2(np);
  DevBuf<unsigned> tk(2);
  ED_CUDA(cudaMemsetAsync(tk.p, 0, 2 * sizeof(unsigned), s));
  S.omega.alloc(vlen);
  const double tol_ritz = std::max(tol, 1e-14);
  ED_CUDA(cudaMemsetAsync(beta.p, 0, (M + 2) * sizeof(double), s));
  k_sym_start<<<nv, kSymThreads, 0, s>>>(start.p, vlen, seed);
  ED_CHECK_LAUNCH();
  double host[3] = {0, 0, 0};
  std::vector<double> hb(M + 2);
  S.have_gs = false;
  S.iters = 0;
  for (int round = 0; round < kSymRounds; ++round) {
    // normalize the start vector into V0
    k_sym_axpy_norm<<<nv, kSymThreads, 0, s>>>(start.p, nullptr, nullptr, vlen, part.p);
    k_sym_finish<<<1, kSymThreads, 0, s>>>(part.p, nv, beta.p, 1);
    k_sym_scale<<<nv, kSymThreads, 0, s>>>(V0.p, start.p, beta.p, vlen, nullptr, nullptr);
    ED_CHECK_LAUNCH();
    ED_CUDA(cudaMemsetAsync(beta.p, 0, sizeof(double), s));
    int m = 0;
    for (int pass = 0; pass < 2; ++pass) {
      double* v = V0.p;
      double* vp = V1.p;
      if (pass == 1) {
        k_sym_axpy_norm<<<nv, kSymThreads, 0, s>>>(start.p, nullptr, nullptr, vlen, part.p);
        k_sym_finish<<<1, kSymThreads, 0, s>>>(part.p, nv, W.p, 1);
        ED_CUDA(cudaMemsetAsync(S.omega.p, 0, vlen * sizeof(double), s));
        k_sym_scale<<<nv, kSymThreads, 0, s>>>(V0.p, start.p, W.p, vlen, S.omega.p, svec.p);
        ED_CHECK_LAUNCH();
      }
      ED_CUDA(cudaMemsetAsync(vp, 0, vlen * sizeof(double), s));
      const int nmax = pass == 0 ? M : m - 1;
      for (int n = 0; n < nmax; ++n) {
        // W = H v - b_n v_prev, alpha_n = <v, W>; W -= alpha_n v, b_{n+1} = |W|; v_prev = W / b_{n+1}
        sym_spmv(S, v, W.p, vp, beta.p + n, part.p, nb, s, tk.p, alpha.p + n);
        k_sym_axpy_norm<<<nv, kSymThreads, 0, s>>>(W.p, v, alpha.p + n, vlen, part2.p, tk.p + 1, beta.p + n + 1);
        k_sym_scale<<<nv, kSymThreads, 0, s>>>(vp, W.p, beta.p + n + 1, vlen, pass == 1 ? S.omega.p : nullptr, svec.p + n + 1);
        ED_CHECK_LAUNCH();
        std::swap(v, vp);
        if (pass == 0 && ((n + 1) % kSymCheck == 0 || n + 1 == M)) {
          ED_CUDA(cudaMemcpyAsync(hb.data(), beta.p, (n + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
          ED_CUDA(cudaStreamSynchronize(s));
          int levels = n + 1;
          bool brk = false;
          for (int j = 1; j <= n + 1; ++j)
            if (!(hb[j] > 1e-12)) {
              levels = j;
              brk = true;
              break;
            }
          launch_tridiag_lowest(alpha.p, beta.p, levels, evals.p, svec.p, s);
          ED_CUDA(cudaMemcpyAsync(host, evals.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
          ED_CUDA(cudaStreamSynchronize(s));
          m = levels;
          if (brk || host[2] < tol_ritz * std::max(1.0, std::fabs(host[0]))) break;
        }
      }
    }
    S.iters += m;
    // residual of the rebuilt vector: normalize, E = <w, H w>, r = |H w - E w|
    k_sym_axpy_norm<<<nv, kSymThreads, 0, s>>>(S.omega.p, nullptr, nullptr, vlen, part.p);
    k_sym_finish<<<1, kSymThreads, 0, s>>>(part.p, nv, W.p + 0, 1);
    k_sym_scale<<<nv, kSymThreads, 0, s>>>(start.p, S.omega.p, W.p, vlen, nullptr, nullptr);
    ED_CHECK_LAUNCH();
    ED_CUDA(cudaMemcpyAsync(S.omega.p, start.p, vlen * sizeof(double), cudaMemcpyDeviceToDevice, s));
    sym_spmv(S, S.omega.p, W.p, nullptr, nullptr, part.p, nb, s);
    k_sym_finish<<<1, kSymThreads, 0, s>>>(part.p, nb, evals.p, 0);
    k_sym_axpy_norm<<<nv, kSymThreads, 0, s>>>(W.p, S.omega.p, evals.p, vlen, part.p);
    k_sym_finish<<<1, kSymThreads, 0, s>>>(part.p, nv, evals.p + 1, 1);
    ED_CHECK_LAUNCH();
    ED_CUDA(cudaMemcpyAsync(host, evals.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    S.E0 = host[0];
    S.residual = host[1];
    if (S.residual <= 1e-12 * std::max(1.0, std::fabs(S.E0))) {
      S.have_gs = true;
      return;
    }
    // restart from the rebuilt vector (already normalized in `start`)
    ED_CUDA(cudaMemsetAsync(beta.p, 0, (M + 2) * sizeof(double), s));
  }
}

// The sector of the same group for another particle number and irrep (exponents m_k).
static std::unique_ptr<ed_sym> sym_sibling(const ed_sym& S, int n_up, int n_dn, const std::vector<int>& irrep,
                                           bool force_cplx, cudaStream_t s) {
  auto T = std::make_unique<ed_sym>();
  T->force_cplx = force_cplx;
  T->c = S.c;
  T->n_gen = S.n_gen;
  T->n_up = n_up;
  T->n_dn = n_dn;
  T->orders = S.orders;
  T->irrep = irrep;
  T->perm = S.perm;
  sym_build(*T, T->perm.data(), s);
  return T;
}

constexpr int kSymCfCheck = 40;      // levels between convergence checks on the grid
constexpr int kSymCfMax = 20000;     // preset maximum of a continued fraction

// Lanczos levels a_n, b_n of the sector T from the (unnormalized) vector phi, run until the
// fraction (electron s = +1 or hole s = -1) changes on the grid by less than tol between two
// checks, b_n vanishes, or the preset maximum; then coef * fraction is added to out[nz].
// Returns the number of levels.
static int sym_cf(ed_sym& T, const double* phi, double E0, double s_eh, const DevBuf<double>& zr,
                  const DevBuf<double>& zi, int nz, double tol, double coef, double2* out, cudaStream_t s) {
  const int64_t dim = T.dim, vlen = T.cplx ? 2 * dim : dim;  // vectors: doubles, or interleaved complex
  const int nb = sym_grid(dim, kSymRowsPerBlock), nv = sym_grid(vlen, kSymThreads * 4);
  const int maxn = (int)std::min<int64_t>(kSymCfMax, 2 * dim + 16);
  DevBuf<double> V0(vlen), V1(vlen), W(vlen), alpha(maxn + 1), beta(maxn + 2), part(std::max(nb, nv)),
      part2(std::max(nb, nv)), nrm(1);
  DevBuf<unsigned> tk(2);
  ED_CUDA(cudaMemsetAsync(tk.p, 0, 2 * sizeof(unsigned), s));
  DevBuf<double2> g0(nz), g1(nz);
  ED_CUDA(cudaMemsetAsync(beta.p, 0, (maxn + 2) * sizeof(double), s));
  k_sym_axpy_norm<<<nv, kSymThreads, 0, s>>>(const_cast<double*>(phi), nullptr, nullptr, vlen, part.p);
  k_sym_finish<<<1, kSymThreads, 0, s>>>(part.p, nv, nrm.p, 1);
  k_sym_scale<<<nv, kSymThreads, 0, s>>>(V0.p, phi, nrm.p, vlen, nullptr, nullptr);
  ED_CHECK_LAUNCH();
  double b0 = 0.0;
  ED_CUDA(cudaMemcpyAsync(&b0, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  ED_CUDA(cudaMemsetAsync(V1.p, 0, vlen * sizeof(double), s));
  ED_CUDA(cudaStreamSynchronize(s));
  if (!(b0 > 0.0)) return 0;
  const double b0sq = b0 * b0;
  std::vector<double2> h0(nz), h1(nz);
  std::vector<double> hb(maxn + 2);
  double* v = V0.p;
  double* vp = V1.p;
  int levels = 0, quiet = 0;
  bool have_prev = false;
  for (int n = 0; n < maxn; ++n) {
    sym_spmv(T, v, W.p, vp, beta.p + n, part.p, nb, s, tk.p, alpha.p + n);
    k_sym_axpy_norm<<<nv, kSymThreads, 0, s>>>(W.p, v, alpha.p + n, vlen, part2.p, tk.p + 1, beta.p + n + 1);
    k_sym_scale<<<nv, kSymThreads, 0, s>>>(vp, W.p, beta.p + n + 1, vlen, nullptr, nullptr);
    ED_CHECK_LAUNCH();
    std::swap(v, vp);
    levels = n + 1;
    if ((n + 1) % kSymCfCheck == 0 || n + 1 == maxn) {
      ED_CUDA(cudaMemsetAsync(g1.p, 0, nz * sizeof(double2), s));
      k_sym_cf_eval<<<(nz + 127) / 128, 128, 0, s>>>(alpha.p, beta.p, levels, E0, b0sq, s_eh, zr.p, zi.p, nz, 1.0, g1.p);
      ED_CHECK_LAUNCH();
      ED_CUDA(cudaMemcpyAsync(h1.data(), g1.p, nz * sizeof(double2), cudaMemcpyDeviceToHost, s));
      ED_CUDA(cudaMemcpyAsync(hb.data(), beta.p, (n + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
      ED_CUDA(cudaStreamSynchronize(s));
      // an invariant subspace: stop at the first vanishing b_j
      int brk = -1;
      for (int j = 1; j <= n + 1; ++j)
        if (!(hb[j] > 1e-10 * std::max(1.0, std::fabs(E0)))) {
          brk = j;
          break;
        }
      if (brk > 0) {
        levels = brk;
        break;
      }
      double d = 0.0;
      for (int i = 0; i < nz && have_prev; ++i)
        d = std::max(d, std::hypot(h1[i].x - h0[i].x, h1[i].y - h0[i].y));
      quiet = (have_prev && d < tol) ? quiet + 1 : 0;
      if (quiet >= 2) break;  // two successive checks below the tolerance
      h0.swap(h1);
      have_prev = true;
    }
  }
  k_sym_cf_eval<<<(nz + 127) / 128, 128, 0, s>>>(alpha.p, beta.p, levels, E0, b0sq, s_eh, zr.p, zi.p, nz, coef, out);
  ED_CHECK_LAUNCH();
  ED_CUDA(cudaStreamSynchronize(s));
  return levels;
}

__global__ void k_sym_add(const double* __restrict__ x, const double* __restrict__ y, int64_t n, double* __restrict__ z) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = x[i] + y[i];
}

// z = x + y (mode 0) or x + i y (mode 1) on n interleaved complex values
__global__ void k_sym_combine(const double2* __restrict__ x, const double2* __restrict__ y, int64_t n, int mode,
                              double2* __restrict__ z) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = x[i], b = y[i];
    z[i] = mode ? make_double2(a.x - b.y, a.y + b.x) : make_double2(a.x + b.x, a.y + b.y);
  }
}

// <phi_x| R |phi_y> of one part from its continued fractions: D (diagonal), and for the pair
// rho < sigma (slot k) Pp = <phi_rho + phi_sigma| R |phi_rho + phi_sigma>, Pi the same with
// phi_rho + i phi_sigma.  With X = Pp - D_rho - D_sigma, Y = Pi - D_rho - D_sigma:
// <phi_rho|R|phi_sigma> = (X - i Y) / 2 and <phi_sigma|R|phi_rho> = (X + i Y) / 2.
__device__ __forceinline__ double2 sym_pair_value(int x, int y, int nz, int iz, int nrow, const int* __restrict__ pidx,
                                                  const double2* __restrict__ D, const double2* __restrict__ Pp,
                                                  const double2* __restrict__ Pi) {
  if (x == y) return D[(int64_t)x * nz + iz];
  const int k = pidx[x * nrow + y];
  if (k < 0) return make_double2(0.0, 0.0);
  const double2 dx = D[(int64_t)x * nz + iz], dy = D[(int64_t)y * nz + iz];
  const double2 p = Pp[(int64_t)k * nz + iz], q = Pi[(int64_t)k * nz + iz];
  const double Xr = p.x - dx.x - dy.x, Xi = p.y - dx.y - dy.y;
  const double Yr = q.x - dx.x - dy.x, Yi = q.y - dx.y - dy.y;
  const double sg = x < y ? 1.0 : -1.0;  // x < y: (X - i Y) / 2, else (X + i Y) / 2
  return make_double2(0.5 * (Xr + sg * Yi), 0.5 * (Xi - sg * Yr));
}

// Complex recombination (unitary M, rows c+_rho = sum_a M_rho,a c+_a):
//   G_ab = sum_rho,sigma M_rho,a conj(M_sigma,b) (<phi^e_rho| R_e |phi^e_sigma> + <phi^h_sigma| R_h |phi^h_rho>)
// with phi^e_rho = c+_rho Omega and phi^h_rho = c_rho Omega.  M: [nrow][ns] complex; D, Pp, Pi of
// the electron part first, then of the hole part (offsets nrow nz and npair nz).
__global__ void k_sym_assemble_c(int nz, int ns, int nrow, int npair, const double2* __restrict__ M,
                                 const int* __restrict__ pidx, const double2* __restrict__ D,
                                 const double2* __restrict__ Pp, const double2* __restrict__ Pi,
                                 double2* __restrict__ G) {
  const int64_t total = (int64_t)nz * ns * ns;
  const int64_t dso = (int64_t)nrow * nz, pso = (int64_t)npair * nz;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int iz = (int)(t / (ns * ns)), a = (int)((t / ns) % ns), b = (int)(t % ns);
    double gr = 0.0, gi = 0.0;
    for (int r = 0; r < nrow; ++r) {
      const double2 ma = M[r * ns + a];
      if (ma.x == 0.0 && ma.y == 0.0) continue;
      for (int q = 0; q < nrow; ++q) {
        const double2 mb = M[q * ns + b];
        if (mb.x == 0.0 && mb.y == 0.0) continue;
        if (q != r && pidx[r * nrow + q] < 0) continue;
        // w = M_ra conj(M_qb)
        const double wr = ma.x * mb.x + ma.y * mb.y, wi = ma.y * mb.x - ma.x * mb.y;
        const double2 ke = sym_pair_value(r, q, nz, iz, nrow, pidx, D, Pp, Pi);
        const double2 kh = sym_pair_value(q, r, nz, iz, nrow, pidx, D + dso, Pp + pso, Pi + pso);
        const double kr = ke.x + kh.x, ki = ke.y + kh.y;
        gr += wr * kr - wi * ki;
        gi += wr * ki + wi * kr;
      }
    }
    G[t] = make_double2(gr, gi);
  }
}

// G_ab(z) = sum over rows rho, sigma of the same irrep of M_rho,a M_sigma,b G_rho,sigma(z), with
// G_rho,rho = D_rho and G_rho,sigma = (P_rho,sigma - D_rho - D_sigma) / 2 (the pair combination
// of Sec. 4.3 for a real Hamiltonian).  M: [nrow][ns] (orthonormal rows); pidx[rho][sigma]: the
// pair's slot in P, or -1 when the rows belong to different irreps.  Out: [nz][ns][ns].
__global__ void k_sym_assemble(int nz, int ns, int nrow, const double* __restrict__ M, const int* __restrict__ pidx,
                               const double2* __restrict__ D, const double2* __restrict__ P, double2* __restrict__ G) {
  const int64_t total = (int64_t)nz * ns * ns;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int iz = (int)(t / (ns * ns)), a = (int)((t / ns) % ns), b = (int)(t % ns);
    double gr = 0.0, gi = 0.0;
    for (int r = 0; r < nrow; ++r) {
      const double mra = M[r * ns + a];
      if (mra == 0.0) continue;
      for (int q = 0; q < nrow; ++q) {
        const double w = mra * M[q * ns + b];
        if (w == 0.0) continue;
        double2 g;
        if (q == r) {
          g = D[(int64_t)r * nz + iz];
        } else {
          const int k = pidx[r * nrow + q];
          if (k < 0) continue;
          const double2 p = P[(int64_t)k * nz + iz], d1 = D[(int64_t)r * nz + iz], d2 = D[(int64_t)q * nz + iz];
          g = make_double2(0.5 * (p.x - d1.x - d2.x), 0.5 * (p.y - d1.y - d2.y));
        }
        gr += w * g.x;
        gi += w * g.y;
      }
    }
    G[t] = make_double2(gr, gi);
  }
}

// Green function with symmetrized operators for any Abelian group (complex characters).  Rows:
// for every irrep beta and site orbit, c+_rho = sum_a M_rho,a c+_a with M_rho proportional to sum_g
// chi_beta(g)^* e_{g(a)}, normalized, so that U_h c+_rho U_h^-1 = chi_beta(h) c+_rho; M is unitary.
// c+_rho Omega lies in the irrep alpha + beta of N + 1 and c_rho Omega in alpha - beta of N - 1
// (exponents modulo the orders); every target sector is kept in complex storage.  The diagonal
// <phi_rho|R|phi_rho> and, for two rows of the same beta, the fractions of phi_rho + phi_sigma and
// phi_rho + i phi_sigma give <phi_rho|R|phi_sigma> (R is not symmetric when H is complex).
static void sym_green_general(ed_sym& S, const double* omega, int nz, double eta, int axis, int spin, double* G_out) {
  ed_cluster& c = *S.c;
  cudaStream_t s = c.stream;
  const int L = c.model.L, ns = c.model.ns, ng = S.host.ng, k = S.n_gen;
  auto digits = [&](int g) {
    std::vector<int> a(k);
    for (int j = 0, rest = g; j < k; rest /= S.orders[j], ++j) a[j] = rest % S.orders[j];
    return a;
  };
  std::vector<std::vector<int>> gdig(ng);
  for (int g = 0; g < ng; ++g) gdig[g] = digits(g);
  // rows: the projection of every site orbit onto every irrep beta (element order as in sym_build)
  std::vector<std::vector<int>> row_beta;
  std::vector<std::vector<std::complex<double>>> row_m;
  for (int bm = 0; bm < ng; ++bm) {
    const std::vector<int> beta = digits(bm);
    std::vector<char> seen(ns, 0);
    for (int a = 0; a < ns; ++a) {
      if (seen[a]) continue;
      std::vector<std::complex<double>> v(L, 0.0);
      for (int g = 0; g < ng; ++g) {
        double ph = 0.0;
        for (int j = 0; j < k; ++j) ph += (double)beta[j] * gdig[g][j] / S.orders[j];
        ph -= std::floor(ph);
        v[S.host.perm[g][a]] += std::polar(1.0, -2.0 * M_PI * ph) / (double)ng;
        seen[S.host.perm[g][a]] = 1;
      }
      double nn = 0.0;
      for (auto& x : v) nn += std::norm(x);
      if (nn < 1e-20) continue;
      for (auto& x : v) x /= std::sqrt(nn);
      row_beta.push_back(beta);
      row_m.push_back(v);
    }
  }
  const int nrow = (int)row_m.size();
  if (nrow != ns) throw Error(ED_ERR_INVALID, "symmetrized site operators do not span the sites");
  std::vector<double> zr_h(nz), zi_h(nz);
  for (int i = 0; i < nz; ++i) {
    zr_h[i] = axis == ED_AXIS_MATSUBARA ? 0.0 : omega[i];
    zi_h[i] = axis == ED_AXIS_MATSUBARA ? omega[i] : eta;
  }
  DevBuf<double> zr(nz), zi(nz), Wd(2 * L);
  ED_CUDA(cudaMemcpyAsync(zr.p, zr_h.data(), nz * sizeof(double), cudaMemcpyHostToDevice, s));
  ED_CUDA(cudaMemcpyAsync(zi.p, zi_h.data(), nz * sizeof(double), cudaMemcpyHostToDevice, s));
  std::vector<int> pidx(nrow * nrow, -1);
  int npair = 0;
  for (int r = 0; r < nrow; ++r)
    for (int q = r + 1; q < nrow; ++q)
      if (row_beta[r] == row_beta[q]) pidx[r * nrow + q] = pidx[q * nrow + r] = npair++;
  // electron part first, then hole part
  DevBuf<double2> D((size_t)2 * nrow * nz), Pp((size_t)2 * std::max(1, npair) * nz),
      Pi((size_t)2 * std::max(1, npair) * nz);
  ED_CUDA(cudaMemsetAsync(D.p, 0, D.n * sizeof(double2), s));
  ED_CUDA(cudaMemsetAsync(Pp.p, 0, Pp.n * sizeof(double2), s));
  ED_CUDA(cudaMemsetAsync(Pi.p, 0, Pi.n * sizeof(double2), s));
  const double tol = c.gf_tol > 0.0 ? c.gf_tol : 1e-12;
  const double E0 = S.E0;
  const int nu = S.n_up, nd = S.n_dn;
  for (int part = 0; part < 2; ++part) {  // 0: electron (c+ Omega, N + 1), 1: hole (c Omega, N - 1)
    const int du = spin == 0 ? (part == 0 ? 1 : -1) : 0, dd = spin == 1 ? (part == 0 ? 1 : -1) : 0;
    if (nu + du < 0 || nu + du > L || nd + dd < 0 || nd + dd > L) continue;
    const double s_eh = part == 0 ? 1.0 : -1.0;
    double2* Dp = D.p + (size_t)part * nrow * nz;
    double2* Ppp = Pp.p + (size_t)part * std::max(1, npair) * nz;
    double2* Pip = Pi.p + (size_t)part * std::max(1, npair) * nz;
    std::map<std::vector<int>, std::unique_ptr<ed_sym>> sectors;
    std::vector<DevBuf<double>> phi(nrow);
    std::vector<ed_sym*> tgt(nrow, nullptr);
    for (int r = 0; r < nrow; ++r) {
      std::vector<int> mt(k);  // alpha + beta (electron) or alpha - beta (hole), modulo the orders
      for (int j = 0; j < k; ++j)
        mt[j] = ((S.irrep[j] + (part == 0 ? row_beta[r][j] : -row_beta[r][j])) % S.orders[j] + S.orders[j]) % S.orders[j];
      auto& T = sectors[mt];
      if (!T) T = sym_sibling(S, nu + du, nd + dd, mt, true, s);
      tgt[r] = T.get();
      if (T->dim == 0) continue;
      phi[r].alloc(2 * T->dim);
      // weights of O: M_rho (c+_rho) or conj(M_rho) (c_rho)
      std::vector<double> wh(2 * L);
      for (int a = 0; a < L; ++a) {
        wh[2 * a] = row_m[r][a].real();
        wh[2 * a + 1] = part == 0 ? row_m[r][a].imag() : -row_m[r][a].imag();
      }
      ED_CUDA(cudaMemcpyAsync(Wd.p, wh.data(), 2 * L * sizeof(double), cudaMemcpyHostToDevice, s));
      if (S.cplx)
        k_sym_apply_c<true><<<sym_grid(T->dim, 128), 128, 0, s>>>(S.G.p, S.keys.p, S.stab.p, S.dim, S.omega.p, T->keys.p,
                                                                  T->stab.p, T->dim, Wd.p, part == 0 ? 1 : 0, spin,
                                                                  phi[r].p);
      else
        k_sym_apply_c<false><<<sym_grid(T->dim, 128), 128, 0, s>>>(S.G.p, S.keys.p, S.stab.p, S.dim, S.omega.p, T->keys.p,
                                                                   T->stab.p, T->dim, Wd.p, part == 0 ? 1 : 0, spin,
                                                                   phi[r].p);
      ED_CHECK_LAUNCH();
      ED_CUDA(cudaStreamSynchronize(s));  // Wd is rewritten for the next row
      sym_cf(*T, phi[r].p, E0, s_eh, zr, zi, nz, tol, 1.0, Dp + (size_t)r * nz, s);
    }
    for (int r = 0; r < nrow; ++r)
      for (int q = r + 1; q < nrow; ++q) {
        const int kp = pidx[r * nrow + q];
        if (kp < 0 || tgt[r]->dim == 0) continue;
        const int64_t n = tgt[r]->dim;
        DevBuf<double> sum(2 * n);
        for (int mode = 0; mode < 2; ++mode) {
          k_sym_combine<<<sym_grid(n, kSymThreads * 4), kSymThreads, 0, s>>>(
              reinterpret_cast<const double2*>(phi[r].p), reinterpret_cast<const double2*>(phi[q].p), n, mode,
              reinterpret_cast<double2*>(sum.p));
          ED_CHECK_LAUNCH();
          sym_cf(*tgt[r], sum.p, E0, s_eh, zr, zi, nz, tol, 1.0, (mode ? Pip : Ppp) + (size_t)kp * nz, s);
        }
      }
  }
  std::vector<double2> Mh((size_t)nrow * ns);
  for (int r = 0; r < nrow; ++r)
    for (int a = 0; a < ns; ++a) Mh[(size_t)r * ns + a] = make_double2(row_m[r][a].real(), row_m[r][a].imag());
  DevBuf<double2> Mdev(Mh.size());
  DevBuf<int> Pd(pidx.size());
  DevBuf<double2> G((size_t)nz * ns * ns);
  ED_CUDA(cudaMemcpyAsync(Mdev.p, Mh.data(), Mh.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
  ED_CUDA(cudaMemcpyAsync(Pd.p, pidx.data(), pidx.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  k_sym_assemble_c<<<sym_grid((int64_t)nz * ns * ns, 256), 256, 0, s>>>(nz, ns, nrow, std::max(1, npair), Mdev.p, Pd.p,
                                                                         D.p, Pp.p, Pi.p, G.p);
  ED_CHECK_LAUNCH();
  ED_CUDA(cudaMemcpyAsync(G_out, G.p, (size_t)nz * ns * ns * sizeof(double2), cudaMemcpyDeviceToHost, s));
  ED_CUDA(cudaStreamSynchronize(s));
}

// Green function of the cluster's physical sites for one spin from the irrep ground state of S
// (Sec. 4.6): symmetrized site operators of every irrep beta, continued fractions in the N +- 1
// sectors of the product irrep alpha beta, recombined with the orthogonal matrix M of the
// operators (Q_ar = (M^-1)_a,rho Q_rho,r, here with M^-1 = M^T).
static void sym_green(ed_sym& S, const double* omega, int nz, double eta, int axis, int spin, double* G_out) {
  ed_cluster& c = *S.c;
  cudaStream_t s = c.stream;
  if (!S.have_gs) throw Error(ED_ERR_STATE, "no ground state of this irrep yet (ed_sym_ground_state)");
  for (int g = 0; g < S.host.ng; ++g)
    for (int a = 0; a < c.model.ns; ++a)
      if (S.host.perm[g][a] >= c.model.ns) throw Error(ED_ERR_INVALID, "the group maps a cluster site to a bath orbital");
  for (int o : S.orders)
    if (o != 2) {
      sym_green_general(S, omega, nz, eta, axis, spin, G_out);
      return;
    }
  const int L = c.model.L, ns = c.model.ns, ng = 1 << S.n_gen;
  // rows: the projection of each site orbit onto each irrep beta (generator signs), normalized
  std::vector<std::vector<int>> row_sig;
  std::vector<std::vector<double>> row_m;
  for (int bm = 0; bm < ng; ++bm) {
    std::vector<int> sig(S.n_gen);
    for (int j = 0; j < S.n_gen; ++j) sig[j] = (bm >> j & 1) ? -1 : 1;
    std::vector<char> seen(ns, 0);
    for (int a = 0; a < ns; ++a) {
      if (seen[a]) continue;
      std::vector<double> v(L, 0.0);
      for (int g = 0; g < ng; ++g) {
        int chi = 1;
        for (int j = 0; j < S.n_gen; ++j)
          if (g >> j & 1) chi *= sig[j];
        v[S.host.perm[g][a]] += (double)chi / ng;
        seen[S.host.perm[g][a]] = 1;
      }
      double nn = 0.0;
      for (double x : v) nn += x * x;
      if (nn < 1e-20) continue;
      for (double& x : v) x /= std::sqrt(nn);
      row_sig.push_back(sig);
      row_m.push_back(v);
    }
  }
  const int nrow = (int)row_m.size();
  if (nrow != ns) throw Error(ED_ERR_INVALID, "symmetrized site operators do not span the sites");
  std::vector<double> zr_h(nz), zi_h(nz);
  for (int i = 0; i < nz; ++i) {
    zr_h[i] = axis == ED_AXIS_MATSUBARA ? 0.0 : omega[i];
    zi_h[i] = axis == ED_AXIS_MATSUBARA ? omega[i] : eta;
  }
  DevBuf<double> zr(nz), zi(nz), Md(L);
  ED_CUDA(cudaMemcpyAsync(zr.p, zr_h.data(), nz * sizeof(double), cudaMemcpyHostToDevice, s));
  ED_CUDA(cudaMemcpyAsync(zi.p, zi_h.data(), nz * sizeof(double), cudaMemcpyHostToDevice, s));
  std::vector<int> pidx(nrow * nrow, -1);
  int npair = 0;
  for (int r = 0; r < nrow; ++r)
    for (int q = r + 1; q < nrow; ++q)
      if (row_sig[r] == row_sig[q]) pidx[r * nrow + q] = pidx[q * nrow + r] = npair++;
  DevBuf<double2> D((size_t)std::max(1, nrow) * nz), P((size_t)std::max(1, npair) * nz);
  ED_CUDA(cudaMemsetAsync(D.p, 0, D.n * sizeof(double2), s));
  ED_CUDA(cudaMemsetAsync(P.p, 0, P.n * sizeof(double2), s));
  const double tol = c.gf_tol > 0.0 ? c.gf_tol : 1e-12;
  const double E0 = S.E0;
  const int nu = S.n_up, nd = S.n_dn;
  for (int part = 0; part < 2; ++part) {  // 0: electron (c+ Omega, N + 1), 1: hole (c Omega, N - 1)
    const int du = spin == 0 ? (part == 0 ? 1 : -1) : 0, dd = spin == 1 ? (part == 0 ? 1 : -1) : 0;
    if (nu + du < 0 || nu + du > L || nd + dd < 0 || nd + dd > L) continue;
    const double s_eh = part == 0 ? 1.0 : -1.0;
    std::map<std::vector<int>, std::unique_ptr<ed_sym>> sectors;
    std::vector<DevBuf<double>> phi(nrow);
    std::vector<ed_sym*> tgt(nrow, nullptr);
    for (int r = 0; r < nrow; ++r) {
      std::vector<int> mt(S.n_gen);  // the product irrep alpha beta (exponents modulo 2)
      for (int j = 0; j < S.n_gen; ++j) mt[j] = (S.irrep[j] + (row_sig[r][j] < 0 ? 1 : 0)) & 1;
      auto& T = sectors[mt];
      if (!T) T = sym_sibling(S, nu + du, nd + dd, mt, false, s);
      tgt[r] = T.get();
      if (T->dim == 0) continue;
      phi[r].alloc(T->dim);
      ED_CUDA(cudaMemcpyAsync(Md.p, row_m[r].data(), L * sizeof(double), cudaMemcpyHostToDevice, s));
      k_sym_apply<<<sym_grid(T->dim, 128), 128, 0, s>>>(S.G.p, S.keys.p, S.stab.p, S.dim, S.omega.p, T->keys.p,
                                                        T->stab.p, T->dim, Md.p, part == 0 ? 1 : 0, spin, phi[r].p);
      ED_CHECK_LAUNCH();
      ED_CUDA(cudaStreamSynchronize(s));  // Md is rewritten for the next row
      sym_cf(*T, phi[r].p, E0, s_eh, zr, zi, nz, tol, 1.0, D.p + (size_t)r * nz, s);
    }
    for (int r = 0; r < nrow; ++r)
      for (int q = r + 1; q < nrow; ++q) {
        const int k = pidx[r * nrow + q];
        if (k < 0 || tgt[r]->dim == 0) continue;
        DevBuf<double> sum(tgt[r]->dim);
        k_sym_add<<<sym_grid(tgt[r]->dim, kSymThreads * 4), kSymThreads, 0, s>>>(phi[r].p, phi[q].p, tgt[r]->dim, sum.p);
        ED_CHECK_LAUNCH();
        sym_cf(*tgt[r], sum.p, E0, s_eh, zr, zi, nz, tol, 1.0, P.p + (size_t)k * nz, s);
      }
  }
  std::vector<double> Mh((size_t)nrow * ns);
  for (int r = 0; r < nrow; ++r)
    for (int a = 0; a < ns; ++a) Mh[(size_t)r * ns + a] = row_m[r][a];
  DevBuf<double> Mdev(Mh.size());
  DevBuf<int> Pd(pidx.size());
  DevBuf<double2> G((size_t)nz * ns * ns);
  ED_CUDA(cudaMemcpyAsync(Mdev.p, Mh.data(), Mh.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  ED_CUDA(cudaMemcpyAsync(Pd.p, pidx.data(), pidx.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  k_sym_assemble<<<sym_grid((int64_t)nz * ns * ns, 256), 256, 0, s>>>(nz, ns, nrow, Mdev.p, Pd.p, D.p, P.p, G.p);
  ED_CHECK_LAUNCH();
  ED_CUDA(cudaMemcpyAsync(G_out, G.p, (size_t)nz * ns * ns * sizeof(double2), cudaMemcpyDeviceToHost, s));
  ED_CUDA(cudaStreamSynchronize(s));
}

static void sym_validate(const ed_cluster* c, int n_gen, const int* perm, const int* orders, const int* irrep) {
  if (!c) throw Error(ED_ERR_INVALID, "cluster is NULL");
  if (n_gen < 1 || n_gen > kSymMaxGen) throw Error(ED_ERR_INVALID, "need 1 to 5 generators");
  if (!perm || !orders || !irrep) throw Error(ED_ERR_INVALID, "perm, orders and the irrep must not be NULL");
  const ModelHost& m = c->model;
  const int L = m.L;
  int64_t ng = 1;
  for (int j = 0; j < n_gen; ++j) {
    if (orders[j] < 2) throw Error(ED_ERR_INVALID, "generator orders must be at least 2");
    ng *= orders[j];
    if (ng > (1 << kSymMaxGen)) throw Error(ED_ERR_INVALID, "the group has more than 32 elements");
    if (irrep[j] < 0 || irrep[j] >= orders[j]) throw Error(ED_ERR_INVALID, "irrep exponents must lie in [0, n_k)");
    std::vector<int> seen(L, 0);
    for (int i = 0; i < L; ++i) {
      const int pi = perm[j * L + i];
      if (pi < 0 || pi >= L || seen[pi]++) throw Error(ED_ERR_INVALID, "a generator is not a permutation of the orbitals");
    }
    // g^{n} = identity
    std::vector<int> q(L);
    std::iota(q.begin(), q.end(), 0);
    for (int t = 0; t < orders[j]; ++t)
      for (int i = 0; i < L; ++i) q[i] = perm[j * L + q[i]];
    for (int i = 0; i < L; ++i)
      if (q[i] != i)
        throw Error(ED_ERR_INVALID, orders[j] == 2 ? "a generator is not an involution" : "a generator's order does not divide its n");
  }
  for (int j = 0; j < n_gen; ++j)
    for (int k = j + 1; k < n_gen; ++k)
      for (int i = 0; i < L; ++i)
        if (perm[j * L + perm[k * L + i]] != perm[k * L + perm[j * L + i]])
          throw Error(ED_ERR_INVALID, "generators do not commute");
  // independence: the prod n_k products are distinct
  std::vector<std::vector<int>> els;
  for (int g = 0; g < (int)ng; ++g) {
    std::vector<int> p(L);
    std::iota(p.begin(), p.end(), 0);
    for (int j = 0, rest = g; j < n_gen; rest /= orders[j], ++j)
      for (int t = 0; t < rest % orders[j]; ++t)
        for (int i = 0; i < L; ++i) p[i] = perm[j * L + p[i]];
    for (auto& q : els)
      if (q == p) throw Error(ED_ERR_INVALID, "generators are not independent");
    els.push_back(p);
  }
  double scale = 0.0;
  for (double v : m.h) scale = std::max(scale, std::fabs(v));
  for (int j = 0; j < n_gen; ++j)
    for (int a = 0; a < L; ++a) {
      const int pa = perm[j * L + a];
      if (std::fabs(m.U[pa] - m.U[a]) > 1e-12 * std::max(1.0, std::fabs(m.U[a])))
        throw Error(ED_ERR_INVALID, "the interaction is not invariant under a generator");
      for (int b = 0; b < L; ++b) {
        const int pb = perm[j * L + b];
        if (std::fabs(m.h[(size_t)pa * L + pb] - m.h[(size_t)a * L + b]) > 1e-12 * std::max(1.0, scale))
          throw Error(ED_ERR_INVALID, "the one-body matrix is not invariant under a generator");
      }
    }
}

}  // namespace ed

using namespace ed;

template <typename F>
static ed_status sym_guard(F&& f) {
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

static void sym_require_device(const ed_cluster* c) {
  int dev = -1;
  ED_CUDA(cudaGetDevice(&dev));
  if (dev != c->device) throw Error(ED_ERR_INVALID, "the current device is not the cluster's device");
}

extern "C" {

static ed_status sym_create(ed_cluster* c, int n_gen, const int* perm, const int* orders, const int* irrep, ed_sym** out) {
  if (!out) throw Error(ED_ERR_INVALID, "out is NULL");
  *out = nullptr;
  sym_validate(c, n_gen, perm, orders, irrep);
  sym_require_device(c);
  auto S = std::make_unique<ed_sym>();
  S->c = c;
  S->n_gen = n_gen;
  S->n_up = c->desc.n_up;
  S->n_dn = c->desc.n_dn;
  S->orders.assign(orders, orders + n_gen);
  S->irrep.assign(irrep, irrep + n_gen);
  S->perm.assign(perm, perm + n_gen * c->model.L);
  AllocStreamScope as_(c->stream);
  sym_build(*S, perm, c->stream);
  *out = S.release();
  return ED_OK;
}

ed_status ed_sym_create(ed_cluster* c, int n_gen, const int* perm, const int* signs, ed_sym** out) {
  return sym_guard([&]() -> ed_status {
    if (!signs) throw Error(ED_ERR_INVALID, "signs must not be NULL");
    if (n_gen < 1 || n_gen > kSymMaxGen) throw Error(ED_ERR_INVALID, "need 1 to 5 generators");
    std::vector<int> orders(n_gen, 2), m(n_gen);
    for (int j = 0; j < n_gen; ++j) {
      if (signs[j] != 1 && signs[j] != -1) throw Error(ED_ERR_INVALID, "irrep signs must be +1 or -1");
      m[j] = signs[j] < 0 ? 1 : 0;
    }
    return sym_create(c, n_gen, perm, orders.data(), m.data(), out);
  });
}

ed_status ed_sym_create_abelian(ed_cluster* c, int n_gen, const int* perm, const int* orders, const int* irrep,
                                ed_sym** out) {
  return sym_guard([&]() -> ed_status { return sym_create(c, n_gen, perm, orders, irrep, out); });
}

ed_status ed_sym_is_complex(const ed_sym* S, int* is_complex) {
  return sym_guard([&]() -> ed_status {
    if (!S || !is_complex) throw Error(ED_ERR_INVALID, "handle and is_complex must not be NULL");
    *is_complex = S->cplx ? 1 : 0;
    return ED_OK;
  });
}

ed_status ed_sym_info(const ed_sym* S, int64_t* dim, int64_t* nnz) {
  return sym_guard([&]() -> ed_status {
    if (!S) throw Error(ED_ERR_INVALID, "handle is NULL");
    if (dim) *dim = S->dim;
    if (nnz) *nnz = S->nnz;
    return ED_OK;
  });
}

ed_status ed_sym_basis(const ed_sym* S, uint64_t* keys, uint8_t* stab) {
  return sym_guard([&]() -> ed_status {
    if (!S) throw Error(ED_ERR_INVALID, "handle is NULL");
    sym_require_device(S->c);
    cudaStream_t s = S->c->stream;
    if (keys && S->dim) ED_CUDA(cudaMemcpyAsync(keys, S->keys.p, S->dim * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    if (stab && S->dim) ED_CUDA(cudaMemcpyAsync(stab, S->stab.p, S->dim, cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    return ED_OK;
  });
}

ed_status ed_sym_matrix(const ed_sym* S, int64_t* rowptr, int32_t* col, double* val) {
  return sym_guard([&]() -> ed_status {
    if (!S) throw Error(ED_ERR_INVALID, "handle is NULL");
    sym_require_device(S->c);
    cudaStream_t s = S->c->stream;
    if (rowptr) ED_CUDA(cudaMemcpyAsync(rowptr, S->rowptr.p, (S->dim + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (col && S->nnz) ED_CUDA(cudaMemcpyAsync(col, S->col.p, S->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (val && S->nnz)
      ED_CUDA(cudaMemcpyAsync(val, S->val.p, S->nnz * (S->cplx ? 2 : 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    return ED_OK;
  });
}

ed_status ed_sym_hpsi(ed_sym* S, const double* x, double* y) {
  return sym_guard([&]() -> ed_status {
    if (!S || !x || !y) throw Error(ED_ERR_INVALID, "handle and vectors must not be NULL");
    sym_require_device(S->c);
    if (S->dim == 0) return ED_OK;
    sym_spmv(*S, x, y, nullptr, nullptr, nullptr, sym_grid(S->dim, kSymRowsPerBlock), S->c->stream);
    ED_CUDA(cudaStreamSynchronize(S->c->stream));
    return ED_OK;
  });
}

ed_status ed_sym_ground_state(ed_sym* S, double* E0, double* residual, int* iters) {
  return sym_guard([&]() -> ed_status {
    if (!S) throw Error(ED_ERR_INVALID, "handle is NULL");
    sym_require_device(S->c);
    AllocStreamScope as_(S->c->stream);
    sym_ground_state(*S, S->c->desc.tol, S->c->desc.max_iter, S->c->desc.seed);
    if (E0) *E0 = S->E0;
    if (residual) *residual = S->residual;
    if (iters) *iters = S->iters;
    return S->have_gs ? ED_OK : ED_WARN_NOT_CONVERGED;
  });
}

ed_status ed_sym_ground_vector(const ed_sym* S, double* out) {
  return sym_guard([&]() -> ed_status {
    if (!S || !out) throw Error(ED_ERR_INVALID, "handle and out must not be NULL");
    if (S->omega.n == 0) throw Error(ED_ERR_STATE, "no ground state yet");
    sym_require_device(S->c);
    ED_CUDA(cudaMemcpyAsync(out, S->omega.p, S->dim * (S->cplx ? 2 : 1) * sizeof(double), cudaMemcpyDeviceToHost,
                            S->c->stream));
    ED_CUDA(cudaStreamSynchronize(S->c->stream));
    return ED_OK;
  });
}

ed_status ed_sym_green(ed_sym* S, const double* omega, int n_freq, double eta, int axis, int spin, double* G_out) {
  return sym_guard([&]() -> ed_status {
    if (!S || !omega || !G_out) throw Error(ED_ERR_INVALID, "handle, omega and G_out must not be NULL");
    if (n_freq < 1) throw Error(ED_ERR_INVALID, "n_freq must be positive");
    if (axis != ED_AXIS_REAL && axis != ED_AXIS_MATSUBARA) throw Error(ED_ERR_INVALID, "unknown axis");
    if (spin != 0 && spin != 1) throw Error(ED_ERR_INVALID, "spin must be 0 or 1");
    for (int i = 0; i < n_freq; ++i)
      if (!std::isfinite(omega[i])) throw Error(ED_ERR_INVALID, "non-finite frequency");
    if (!std::isfinite(eta)) throw Error(ED_ERR_INVALID, "non-finite eta");
    sym_require_device(S->c);
    AllocStreamScope as_(S->c->stream);
    sym_green(*S, omega, n_freq, eta, axis, spin, G_out);
    return ED_OK;
  });
}

void ed_sym_destroy(ed_sym* S) {
  if (!S) return;
  try {
    cudaStreamSynchronize(S->c->stream);
    delete S;
  } catch (...) {
  }
}

}  // extern "C"
