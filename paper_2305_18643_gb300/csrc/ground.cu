// Ground-state driver (Sec. 4.2): host orchestration of the device kernels.  The recursion
// coefficients stay on the device; the host only reads the tridiagonal eigen-summary every
// `kCheck` steps to decide convergence.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "ed_common.cuh"

namespace ed {

constexpr int kCheck = 10;
constexpr int kRefineRounds = 4;  // FP64 refinement rounds of an FP32-storage ground state

__global__ void k_scale_inv_sqrt(int dt, void* v, const double* nrm2, int64_t du, int64_t dd, int64_t ld) {
  double f = *nrm2 > 0.0 ? 1.0 / sqrt(*nrm2) : 0.0;
  const int64_t dim = du * dd;
  for_each_element(du, dd, [&](int64_t u, int64_t d, int64_t idx) {
    int64_t o = u * ld + d;
    if (dt == ED_FP64)
      ((double*)v)[o] *= f;
    else
      ((float*)v)[o] = (float)((double)((float*)v)[o] * f);
    });
}

void axpby_inv_sqrt(int dt, void* v, const double* nrm2, int64_t du, int64_t dd, int64_t ld, cudaStream_t s) {
  int64_t b = (du * dd + 255) / 256;
  int g = (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
  ProfScope ps_(K_VECTOR, s, 0.0);
  k_scale_inv_sqrt<<<g, 256, 0, s>>>(dt, v, nrm2, du, dd, ld);
  ED_CHECK_LAUNCH();
}

__global__ void k_axpy_neg(double* y, const double* a, const double* x, int64_t n) {
  double f = *a;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] -= f * x[i];
}

void axpy_neg(double* y, const double* a, const double* x, int64_t n, cudaStream_t s) {
  int64_t b = (n + 255) / 256;
  int g = (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
  ProfScope ps_(K_VECTOR, s, 0.0);
  k_axpy_neg<<<g, 256, 0, s>>>(y, a, x, n);
  ED_CHECK_LAUNCH();
}



// One Lanczos pass set (first pass + retrace) from start vector `v0` (dtype, normalized in
// place).  Writes the normalized-by-construction sum_n s_n v_n into omega (FP64).
struct LanczosRun {
  int M;
  DevBuf<double> alpha, beta, beta0, partial, evals, svec, scal;
  DevBuf<int> active, nsteps;
  DevBuf<unsigned> counter;
  LanczosScalars ls;
  int nblk;
  LanczosRun(int M_, int nblk_) : M(M_), nblk(nblk_) {
    alpha.alloc(M + 1);
    beta.alloc(M + 2);
    beta0.alloc(1);
    partial.alloc(std::max(nblk, 1) * 3 + 8);
    evals.alloc(4);
    svec.alloc(2 * (M + 2));
    scal.alloc(8);
    active.alloc(1);
    nsteps.alloc(1);
    counter.alloc(1);
    ls = LanczosScalars{alpha.p, beta.p, beta0.p, active.p, partial.p, counter.p, M, 1e-13, nsteps.p};
  }
  void reset(cudaStream_t s) {
    const double one = 1.0;
    const int on = 1;
    ED_CUDA(cudaMemsetAsync(beta.p, 0, (M + 2) * sizeof(double), s));
    ED_CUDA(cudaMemcpyAsync(beta0.p, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(active.p, &on, sizeof(int), cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(unsigned), s));
  }
};

static size_t esize(int dtype) { return dtype == ED_FP64 ? sizeof(double) : sizeof(float); }

// Lanczos vectors kept in device memory, so that a Ritz vector is summed in one pass over them
// instead of by retracing the recursion.  The paper retraces because its runs keep three vectors in
// memory (Sec. 4.2); the 280 GB of a GB300 hold a hundred or more vectors of the 4x4 sector, and
// the second pass (as many fused steps as the first) becomes one read of the stored vectors.
// Vectors go into chunks allocated as the run grows, while the device keeps a quarter of its memory
// (at least 8 GiB) free; when a chunk does not fit, or on a server lane (whose memory admission
// counts three vectors per run), storing stops and the run is retraced.
struct VectorStore {
  static constexpr int kChunk = 8;
  size_t vbytes = 0;
  int count = 0;
  bool ok = false;
  std::vector<DevBuf<char>> chunks;
  void start(size_t vb) {
    vbytes = vb;
    count = 0;
    chunks.clear();
    ok = g_alloc_stream == nullptr;
  }
  char* at(int n) { return chunks[n / kChunk].p + (size_t)(n % kChunk) * vbytes; }
  void drop() {
    ok = false;
    chunks.clear();  // cudaFree waits for the copies in flight
    count = 0;
  }
  void push(const void* src, cudaStream_t s) {
    if (!ok) return;
    if (count == (int)chunks.size() * kChunk) {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        drop();
        return;
      }
      const size_t need = (size_t)kChunk * vbytes;
      if (fr < need + std::max<size_t>(tot / 4, size_t(8) << 30)) {
        drop();
        return;
      }
      DevBuf<char> b;
      try {
        b.alloc(need);
      } catch (const Error&) {
        drop();
        return;
      }
      chunks.push_back(std::move(b));
    }
    ED_CUDA(cudaMemcpyAsync(at(count), src, vbytes, cudaMemcpyDeviceToDevice, s));
    ++count;
  }
};

// out[u][d] (FP64, contiguous) = (acc ? out[u][d] : 0) + sum_{n < m} coef[n] v_n[u][d] over m stored
// vectors (leading dimension ld, a multiple of the 16-byte group): rows over blocks, one 16-byte
// group of each vector per thread and load, four vectors in flight; pointers and coefficients
// staged in shared memory.
template <typename T>
__global__ void k_ritz_sum(const T* const* __restrict__ vecs, int m, const double* __restrict__ coef, double* __restrict__ out,
                           int64_t du, int64_t dd, int64_t ld, int acc) {
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int VN = 16 / sizeof(T);
  extern __shared__ __align__(16) unsigned char rs_smem[];
  const T** sp = reinterpret_cast<const T**>(rs_smem);
  double* sc = reinterpret_cast<double*>(rs_smem + (size_t)m * sizeof(T*));
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    sp[i] = vecs[i];
    sc[i] = coef[i];
  }
  __syncthreads();
  for (int64_t u = blockIdx.x; u < du; u += gridDim.x) {
    for (int64_t d0 = (int64_t)threadIdx.x * VN; d0 < dd; d0 += (int64_t)blockDim.x * VN) {
      const int64_t o = u * ld + d0;
      double s[VN];
      if constexpr (sizeof(T) == 4) {
        // FP32 vectors: FP32 products with Kahan-compensated FP32 sums (FP64 runs at a small
        // fraction of the FP32 rate here; the products' rounding, 2^-24 relative, is the order
        // of the vectors' own FP32 storage, and the FP64 refinement that follows removes both)
        float sf[VN], cf[VN];
#pragma unroll
        for (int j = 0; j < VN; ++j) sf[j] = cf[j] = 0.f;
        auto add = [&](float c, const V& a) {
          const float* e = reinterpret_cast<const float*>(&a);
#pragma unroll
          for (int j = 0; j < VN; ++j) {
            const float y = fmaf(c, e[j], -cf[j]);
            const float t = sf[j] + y;
            cf[j] = (t - sf[j]) - y;
            sf[j] = t;
          }
        };
        int n = 0;
        for (; n + 4 <= m; n += 4) {
          V a[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) a[q] = __ldg(reinterpret_cast<const V*>(sp[n + q] + o));
#pragma unroll
          for (int q = 0; q < 4; ++q) add((float)sc[n + q], a[q]);
        }
        for (; n < m; ++n) add((float)sc[n], __ldg(reinterpret_cast<const V*>(sp[n] + o)));
#pragma unroll
        for (int j = 0; j < VN; ++j) s[j] = (double)sf[j] - (double)cf[j];
      } else {
#pragma unroll
        for (int j = 0; j < VN; ++j) s[j] = 0.0;
        int n = 0;
        for (; n + 4 <= m; n += 4) {
          V a[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) a[q] = __ldg(reinterpret_cast<const V*>(sp[n + q] + o));
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const T* e = reinterpret_cast<const T*>(&a[q]);
#pragma unroll
            for (int j = 0; j < VN; ++j) s[j] += sc[n + q] * (double)e[j];
          }
        }
        for (; n < m; ++n) {
          const V a = __ldg(reinterpret_cast<const V*>(sp[n] + o));
          const T* e = reinterpret_cast<const T*>(&a);
#pragma unroll
          for (int j = 0; j < VN; ++j) s[j] += sc[n] * (double)e[j];
        }
      }
#pragma unroll
      for (int j = 0; j < VN; ++j) {
        if (d0 + j >= dd) break;
        const int64_t idx = u * dd + d0 + j;
        out[idx] = acc ? out[idx] + s[j] : s[j];
      }
    }
  }
}

// omega (+)= sum_{n < m} coef[n] store[first + n]
static void ritz_sum(int dtype, VectorStore& st, int first, int m, const double* coef, double* omega, int64_t du,
                     int64_t dd, int64_t ld, int acc, cudaStream_t s) {
  if (m <= 0) return;
  std::vector<const void*> ptr(m);
  for (int n = 0; n < m; ++n) ptr[n] = st.at(first + n);
  DevBuf<const void*> dptr(m);
  ED_CUDA(cudaMemcpyAsync(dptr.p, ptr.data(), m * sizeof(void*), cudaMemcpyHostToDevice, s));
  const size_t smem = (size_t)m * (sizeof(void*) + sizeof(double));
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(du, 152 * 8));
  ProfScope ps_(K_VECTOR, s, (double)m * du * ld * esize(dtype) + 8.0 * du * dd * (acc ? 2 : 1));
  if (dtype == ED_FP64)
    k_ritz_sum<double><<<g, 256, smem, s>>>((const double* const*)dptr.p, m, coef, omega, du, dd, ld, acc);
  else
    k_ritz_sum<float><<<g, 256, smem, s>>>((const float* const*)dptr.p, m, coef, omega, du, dd, ld, acc);
  ED_CHECK_LAUNCH();
  ED_CUDA(cudaStreamSynchronize(s));  // the pointer table goes out of scope
}

// Runs pass 1 (until the Ritz estimate < tol_ritz) and the retrace; returns levels used.
// Pass 0 runs until the Ritz estimate < tol_ritz; the ground state sum_n s_n v_n then comes from
// the stored vectors into omega64 (FP64; *summed64 = true) or, when they could not all be stored,
// from pass 1, a retrace accumulating into omega (the vectors' dtype).  Returns the levels used.
static int lanczos_pass(ed_cluster& c, const SectorView& sv, int dtype, LanczosRun& L, char* V0, char* V1, char* Vstart,
                        void* omega, double* omega64, bool* summed64, double tol_ritz, double* host, bool* breakdown,
                        cudaStream_t s) {
  const int64_t du = sv.d_up, dd = sv.d_dn, ld = sv.ld, dim = du * dd;
  const size_t bytes = (size_t)du * ld * esize(dtype);
  char* V[2] = {V0, V1};
  int m = 0;
  *breakdown = false;
  *summed64 = false;
  VectorStore store;
  for (int pass = 0; pass < 2; ++pass) {
    L.reset(s);
    ED_CUDA(cudaMemcpyAsync(V[0], Vstart, bytes, cudaMemcpyDeviceToDevice, s));
    ED_CUDA(cudaMemsetAsync(V[1], 0, bytes, s));
    if (pass == 0) {
      store.start(bytes);
      store.push(V[0], s);
    }
    if (pass == 1) launch_copy_ld(dtype, omega, dd, dtype, V[0], ld, L.svec.p, du, dd, s);
    int cur = 0;
    const int nmax = pass == 0 ? L.M : m - 1;
    for (int n = 0; n < nmax; ++n) {
      launch_lanczos_step(sv, c.hp, dtype, V[cur], V[cur ^ 1], 0, 1, n, L.ls, L.nblk, s);
      launch_lanczos_next(dtype, V[cur ^ 1], V[cur], du, dd, ld, 0, 1, n, L.ls, pass == 1 ? omega : nullptr, L.svec.p, s);
      if (pass == 0) store.push(V[cur ^ 1], s);
      cur ^= 1;
      if (pass == 0 && ((n + 1) % kCheck == 0 || n + 1 == L.M)) {
        ED_CUDA(cudaMemcpyAsync(host + 8, L.active.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        ED_CUDA(cudaStreamSynchronize(s));
        int act = *(int*)(host + 8);
        int levels = n + 1;
        if (!act) {
          // the run stopped at the first level whose b_{n+1} vanished: find it on the host
          std::vector<double> b(n + 2);
          ED_CUDA(cudaMemcpyAsync(b.data(), L.beta.p, (n + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
          ED_CUDA(cudaStreamSynchronize(s));
          levels = 1;
          while (levels < n + 1 && b[levels] > L.ls.btol) ++levels;
          *breakdown = levels < L.M;
        }
        launch_tridiag_lowest(L.alpha.p, L.beta.p, levels, L.evals.p, L.svec.p, s);
        ED_CUDA(cudaMemcpyAsync(host, L.evals.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        ED_CUDA(cudaStreamSynchronize(s));
        m = levels;
        if (!act || host[2] < tol_ritz * std::max(1.0, std::fabs(host[0]))) break;
      }
    }
    if (pass == 0 && store.ok && store.count >= m) {
      ritz_sum(dtype, store, 0, m, L.svec.p, omega64, du, dd, ld, 0, s);
      *summed64 = true;
      break;
    }
  }
  return m;
}

// One round of FP64 refinement of a ground state found with FP32 vectors.  The Lanczos recursion
// of Sec. 4.2 is restarted from the FP64 vector omega itself: q_0 = omega, a_0 = E (its Rayleigh
// quotient), b_1 q_1 = r = H omega - E omega (computed in FP64 by the caller), and the later
// q_n are stored in FP32.  The lowest Ritz vector s of the tridiagonal matrix gives
// omega <- s_0 omega + s_1 r / |r| + sum_{n >= 2} s_n q_n, summed in FP64 by retracing the recursion.
// The correction sum_{n >= 1} s_n q_n has norm ~|r| / gap, so the FP32 rounding of the q_n
// (relative 6e-8) reaches omega only at ~6e-8 |r| / gap: every round multiplies the residual by
// ~6e-8 |H| / gap, and one or two rounds bring an FP32 ground state (residual ~1e-7 |E|) to the
// 1e-12 of an FP64 one.  V0, V1: FP32 work vectors with leading dimension sv.ld (padding zero);
// r is contiguous FP64 and is read only.  Returns the number of levels.
static int refine_round(ed_cluster& c, const SectorView& sv, LanczosRun& L, float* V0, float* V1, double* omega,
                        const double* r, double E, double rnorm, double tol_ritz, DevBuf<double>& scal, double* host,
                        cudaStream_t s) {
  const int64_t du = sv.d_up, dd = sv.d_dn, ld = sv.ld;
  float* V[2] = {V0, V1};
  int m = 0;
  VectorStore store;  // q_1, q_2, ...: with all of them stored the retrace is skipped
  for (int pass = 0; pass < 2; ++pass) {
    L.reset(s);
    const double a0 = E, b1 = rnorm, inv = 1.0 / rnorm;
    ED_CUDA(cudaMemcpyAsync(L.alpha.p, &a0, sizeof(double), cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(L.beta.p + 1, &b1, sizeof(double), cudaMemcpyHostToDevice, s));
    ED_CUDA(cudaMemcpyAsync(scal.p + 5, &inv, sizeof(double), cudaMemcpyHostToDevice, s));
    launch_copy_ld(ED_FP32, V[0], ld, ED_FP64, omega, dd, nullptr, du, dd, s);       // q_0
    launch_copy_ld(ED_FP32, V[1], ld, ED_FP64, r, dd, scal.p + 5, du, dd, s);        // q_1 = r / |r|
    if (pass == 0) {
      store.start((size_t)du * ld * sizeof(float));
      store.push(V[1], s);
    }
    if (pass == 1) {
      // omega <- s_0 omega + (s_1 / |r|) r, in FP64; the loop adds s_n q_n for n >= 2
      double sv01[2];
      ED_CUDA(cudaMemcpyAsync(sv01, L.svec.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      ED_CUDA(cudaStreamSynchronize(s));
      const double cc[2] = {sv01[0], m > 1 ? sv01[1] * inv : 0.0};
      ED_CUDA(cudaMemcpyAsync(scal.p + 5, cc, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
      launch_axpby(ED_FP64, omega, ED_FP64, omega, scal.p + 5, ED_FP64, r, scal.p + 6, du, dd, dd, s);
    }
    int cur = 1;
    const int nmax = pass == 0 ? L.M : m - 1;
    for (int n = 1; n < nmax; ++n) {
      launch_lanczos_step(sv, c.hp, ED_FP32, V[cur], V[cur ^ 1], 0, 1, n, L.ls, L.nblk, s);
      launch_lanczos_next(ED_FP32, V[cur ^ 1], V[cur], du, dd, ld, 0, 1, n, L.ls, pass == 1 ? omega : nullptr, L.svec.p,
                          s, ED_FP64);
      if (pass == 0) store.push(V[cur ^ 1], s);
      cur ^= 1;
      if (pass == 0 && ((n + 1) % kCheck == 0 || n + 1 == L.M)) {
        ED_CUDA(cudaMemcpyAsync(host + 8, L.active.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        ED_CUDA(cudaStreamSynchronize(s));
        const int act = *(int*)(host + 8);
        int levels = n + 1;
        if (!act) {
          std::vector<double> b(n + 2);
          ED_CUDA(cudaMemcpyAsync(b.data(), L.beta.p, (n + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
          ED_CUDA(cudaStreamSynchronize(s));
          levels = 2;
          while (levels < n + 1 && b[levels] > L.ls.btol) ++levels;
        }
        launch_tridiag_lowest(L.alpha.p, L.beta.p, levels, L.evals.p, L.svec.p, s);
        ED_CUDA(cudaMemcpyAsync(host, L.evals.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        ED_CUDA(cudaStreamSynchronize(s));
        m = levels;
        if (!act || host[2] < tol_ritz) break;
      }
    }
    if (pass == 0 && store.ok && store.count >= m - 1) {
      // omega <- s_0 omega + (s_1 / |r|) r + sum_{n >= 2} s_n q_n, the q_n (n >= 2) from the store
      double sv01[2];
      ED_CUDA(cudaMemcpyAsync(sv01, L.svec.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      ED_CUDA(cudaStreamSynchronize(s));
      const double cc[2] = {sv01[0], m > 1 ? sv01[1] / rnorm : 0.0};
      ED_CUDA(cudaMemcpyAsync(scal.p + 5, cc, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
      launch_axpby(ED_FP64, omega, ED_FP64, omega, scal.p + 5, ED_FP64, r, scal.p + 6, du, dd, dd, s);
      ritz_sum(ED_FP32, store, 1, m - 2, L.svec.p + 2, omega, du, dd, ld, 1, s);
      break;
    }
  }
  return m;
}

GroundResult run_ground_state(ed_cluster& c, int dtype, double tol, int max_iter, uint64_t seed) {
  cudaStream_t s = c.stream;
  const int nu = c.desc.n_up, nd = c.desc.n_dn;
  SpinTables& tu = c.tables(nu);
  SpinTables& td = c.tables(nd);
  (void)tu;
  (void)td;
  const int64_t ld = padded_ld(c.tables(nd).dim);
  SectorView sv = c.view(nu, nd, ld);     // padded internal vectors
  SectorView svc = c.view(nu, nd, 0);     // the contiguous ground state
  const int64_t du = sv.d_up, dd = sv.d_dn, dim = du * dd;
  GroundResult R;
  c.omega.alloc(std::max<int64_t>(dim, 1));
  double* host = pinned_scratch();  // slots 0..15
  if (dim == 0) throw Error(ED_ERR_INVALID, "empty sector");

  const int nblk = lanczos_blocks(sv);
  DevBuf<double> y64(dim);  // FP64 work vector for the polish
  DevBuf<double> scal(8);
  DevBuf<double> part(nblk + 8);
  int dt = dtype;
  int total_iters = 0;
  bool have_start = false;
  for (int attempt = 0; attempt < 6; ++attempt) {
    const size_t bytes = (size_t)du * ld * esize(dt);
    DevBuf<char> V0(bytes), V1(bytes), Vs(bytes);
    ED_CUDA(cudaMemsetAsync(V0.p, 0, bytes, s));
    ED_CUDA(cudaMemsetAsync(V1.p, 0, bytes, s));
    ED_CUDA(cudaMemsetAsync(Vs.p, 0, bytes, s));
    if (!have_start) {
      launch_start_vector(dt, Vs.p, du, dd, ld, seed, s);
    } else {
      launch_copy_ld(dt, Vs.p, ld, ED_FP64, c.omega.p, dd, nullptr, du, dd, s);
    }
    // normalize the start vector
    launch_dot(dt, Vs.p, dt, Vs.p, du, dd, ld, part.p, nblk + 8, scal.p + 0, s);
    axpby_inv_sqrt(dt, Vs.p, scal.p + 0, du, dd, ld, s);  // Vs <- Vs / sqrt(<Vs,Vs>)
    LanczosRun L(std::max(2, max_iter), nblk);
    const double tol_ritz = dt == ED_FP64 ? std::min(1e-2, 0.1 * tol) : 1e-7;
    bool breakdown = false;
    // the retrace accumulates the ground state in the vectors' precision (FP32 form: FP32 sum of
    // the s_n v_n, converted to FP64 once)
    DevBuf<float> om32(dt == ED_FP32 ? dim : 0);
    void* acc = dt == ED_FP32 ? (void*)om32.p : (void*)c.omega.p;
    bool summed64 = false;
    int m = lanczos_pass(c, sv, dt, L, V0.p, V1.p, Vs.p, acc, c.omega.p, &summed64, tol_ritz, host, &breakdown, s);
    if (dt == ED_FP32 && !summed64) launch_copy_ld(ED_FP64, c.omega.p, dd, ED_FP32, om32.p, dd, nullptr, du, dd, s);
    total_iters += m;
    const double lam0 = host[0], lam1 = host[1];
    // FP64 polish: normalize omega, Rayleigh quotient E and explicit residual r = H omega - E omega
    // (left in y64), all with the FP64 operator.
    double E = 0.0, res_abs = 0.0;
    // H omega through rows padded to ld (zero padding), so that large sectors take the two-pass
    // kernels (the contiguous layout would force the one-pass kernel, ~2x slower in FP64)
    DevBuf<double> om_pad, y_pad;
    if (ld != dd) {
      om_pad.alloc((size_t)du * ld);
      y_pad.alloc((size_t)du * ld);
      ED_CUDA(cudaMemsetAsync(om_pad.p, 0, (size_t)du * ld * sizeof(double), s));
      ED_CUDA(cudaMemsetAsync(y_pad.p, 0, (size_t)du * ld * sizeof(double), s));
    }
    auto polish = [&]() {
      launch_dot(ED_FP64, c.omega.p, ED_FP64, c.omega.p, du, dd, dd, part.p, nblk + 8, scal.p + 1, s);
      axpby_inv_sqrt(ED_FP64, c.omega.p, scal.p + 1, du, dd, dd, s);
      if (ld != dd) {
        launch_copy_ld(ED_FP64, om_pad.p, ld, ED_FP64, c.omega.p, dd, nullptr, du, dd, s);
        launch_hpsi(sv, c.hp, ED_FP64, om_pad.p, y_pad.p, s);
        launch_copy_ld(ED_FP64, y64.p, dd, ED_FP64, y_pad.p, ld, nullptr, du, dd, s);
      } else {
        launch_hpsi(svc, c.hp, ED_FP64, c.omega.p, y64.p, s);
      }
      launch_dot(ED_FP64, c.omega.p, ED_FP64, y64.p, du, dd, dd, part.p, nblk + 8, scal.p + 2, s);
      axpy_neg(y64.p, scal.p + 2, c.omega.p, dim, s);  // y <- y - E omega
      launch_dot(ED_FP64, y64.p, ED_FP64, y64.p, du, dd, dd, part.p, nblk + 8, scal.p + 3, s);
      ED_CUDA(cudaMemcpyAsync(host + 4, scal.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
      ED_CUDA(cudaStreamSynchronize(s));
      E = host[6];
      res_abs = std::sqrt(std::max(0.0, host[7]));
    };
    polish();
    double scale = std::max(1.0, std::fabs(E));
    // a breakdown of the recursion (invariant subspace) is exact only with FP64 vectors
    bool ok = res_abs <= tol * scale || (breakdown && dt == ED_FP64);
    if (!ok && dt == ED_FP32) {
      // FP32 storage: FP64 refinement rounds (refine_round) until the FP64 residual meets tol
      for (int round = 0; round < kRefineRounds && !ok; ++round) {
        const double ritz_stop = std::max(0.1 * tol * scale, 1e-6 * res_abs);
        total_iters += refine_round(c, sv, L, (float*)V0.p, (float*)V1.p, c.omega.p, y64.p, E, res_abs, ritz_stop, scal,
                                    host, s);
        polish();
        scale = std::max(1.0, std::fabs(E));
        ok = res_abs <= tol * scale;
      }
    }
    R.E0 = E;
    R.residual = res_abs / scale;
    R.iters = total_iters;
    R.gap = lam1 - lam0;
    R.degenerate = (lam1 - lam0) < 1e-8 * std::max(1.0, std::fabs(lam0));
    if (ok) {
      R.converged = true;
      break;
    }
    // restart from the current ground-state estimate (FP64 refinement for the FP32 form)
    const double one = 1.0;
    ED_CUDA(cudaMemcpyAsync(scal.p + 7, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    have_start = true;
    if (dt == ED_FP32) dt = ED_FP64;
  }
  return R;
}

}  // namespace ed
