// K7 + continued-fraction Green function + K9 (Sec. 4.3, Eqs. green, GreenCF1, jacobi).
//
// Starting vectors: phi = c+_i W (electron part, sector N_s + 1) or c_i W (hole part, N_s - 1)
// for every cluster site i, and (c_i + c_j)+ W / (c_i + c_j) W for every pair i < j.  Each is
// built in pull form: for a target state b' of the changed spin, the source state is b' with
// orbital i removed (creation) or added (annihilation); the fermion sign is the parity of the
// occupied orbitals below i (plus every up electron for a down-spin operator, ordering of
// Eq. basis).
//
// All starting vectors of a sector run the three-term recursion together (one fused launch per
// step, one run per blockIdx.y).  The vectors are not reorthogonalized: run past the dimension
// of the Krylov space the continued fraction converges to the exact resolvent and the ghost
// copies carry no weight.  A run stops when b_n vanishes or when its continued fraction,
// evaluated on the frequency grid every few steps, changes by less than the tolerance twice in
// a row.  G_ii = G^e_ii + G^h_ii and, for a real H, G_ij = (G+_ij - G_ii - G_jj) / 2 for each part.
#include <algorithm>
#include <cmath>

#include "ed_common.cuh"

namespace ed {

constexpr int kGT = 256;

__global__ void k_apply_cop(const double* __restrict__ omega, int64_t dd_s, const uint32_t* __restrict__ B_dst,
                            RankView rv_src, int spin, int create, int extra_parity, const int2* __restrict__ runs,
                            int dtype, void* phi0, int64_t vstride, int64_t du_t, int64_t dd_t, int64_t ld_t) {
  const int run = blockIdx.y;
  const int2 rs = runs[run];
  const int64_t dim = du_t * dd_t;
  for_each_element(du_t, dd_t, [&](int64_t u, int64_t d, int64_t idx) {
    uint32_t bt = spin == 0 ? B_dst[u] : B_dst[d];
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      int site = k == 0 ? rs.x : rs.y;
      if (site < 0) continue;
      uint32_t bit = 1u << site;
      bool ok = create ? (bt & bit) != 0u : (bt & bit) == 0u;
      if (!ok) continue;
      uint32_t src = bt ^ bit;
      int64_t r = rank_of(rv_src, src);
      int neg = (__popc(bt & (bit - 1u)) + extra_parity) & 1;
      double v = spin == 0 ? omega[r * dd_s + d] : omega[u * dd_s + r];
      acc += neg ? -v : v;
    }
    int64_t o = run * vstride + u * ld_t + d;
    if (dtype == ED_FP64)
      ((double*)phi0)[o] = acc;
    else
      ((float*)phi0)[o] = (float)acc;
    });
}

__device__ __forceinline__ double blk_sum(double a) {
  __shared__ double sm[kGT / 32];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sm[w] = a;
  __syncthreads();
  if (w == 0) {
    a = l < kGT / 32 ? sm[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  }
  __syncthreads();
  return a;
}

__device__ __forceinline__ double blk_max(double a) {
  __shared__ double sm[kGT / 32];
  for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sm[w] = a;
  __syncthreads();
  if (w == 0) {
    a = l < kGT / 32 ? sm[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
  }
  __syncthreads();
  return a;
}

// Per-run squared norm: partials over grid x, then one block per run finishes.
__global__ void k_run_norm_partial(int dtype, const void* V0, int64_t vstride, int64_t du, int64_t dd, int64_t ld,
                                   double* __restrict__ partial) {
  const int run = blockIdx.y;
  const int64_t dim = du * dd;
  double s = 0.0;
  for_each_element(du, dd, [&](int64_t u, int64_t d, int64_t idx) {
    int64_t o = run * vstride + u * ld + d;
    double v = dtype == ED_FP64 ? ((const double*)V0)[o] : (double)((const float*)V0)[o];
    s += v * v;
    });
  s = blk_sum(s);
  if (threadIdx.x == 0) partial[(int64_t)run * gridDim.x + blockIdx.x] = s;
}

__global__ void k_run_norm_finish(const double* __restrict__ partial, int nblk, double* __restrict__ b0sq,
                                  double* __restrict__ beta0, int* __restrict__ active) {
  const int run = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += partial[(int64_t)run * nblk + i];
  s = blk_sum(s);
  if (threadIdx.x == 0) {
    b0sq[run] = s;
    beta0[run] = sqrt(s);
    active[run] = s > 1e-28 ? 1 : 0;
  }
}

__global__ void k_run_scale(int dtype, void* V0, int64_t vstride, int64_t du, int64_t dd, int64_t ld,
                            const double* __restrict__ beta0) {
  const int run = blockIdx.y;
  const double b = beta0[run];
  const double f = b > 0.0 ? 1.0 / b : 0.0;
  const int64_t dim = du * dd;
  for_each_element(du, dd, [&](int64_t u, int64_t d, int64_t idx) {
    int64_t o = run * vstride + u * ld + d;
    if (dtype == ED_FP64)
      ((double*)V0)[o] *= f;
    else
      ((float*)V0)[o] = (float)((double)((float*)V0)[o] * f);
    });
}

// Continued fraction of Eq. jacobi shifted by E0 (electron: s = -1, hole: s = +1):
// den_n = z + s (a_n - E0) - b_{n+1}^2 / den_{n+1}, G = b_0^2 / den_0, bottom-up.
__device__ __forceinline__ double2 cf_eval(const double* __restrict__ a, const double* __restrict__ b, int m,
                                           double b0sq, double2 z, double E0, double s) {
  if (m <= 0) return make_double2(0.0, 0.0);
  double dr = z.x + s * (a[m - 1] - E0), di = z.y;
  for (int n = m - 2; n >= 0; --n) {
    double bb = b[n + 1];
    double q = bb * bb / (dr * dr + di * di);
    dr = z.x + s * (a[n] - E0) - q * dr;
    di = z.y + q * di;
  }
  double q = b0sq / (dr * dr + di * di);
  return make_double2(q * dr, -q * di);
}

__global__ void k_cf_check(const double* __restrict__ alpha, const double* __restrict__ beta,
                           const double* __restrict__ b0sq, const int* __restrict__ nsteps, int mstride,
                           int* __restrict__ active, int* __restrict__ hits, double E0, double s,
                           const double2* __restrict__ z, int nz, int zstride, double2* __restrict__ prev, double tol,
                           int* __restrict__ n_active) {
  const int run = blockIdx.x;
  if (!active[run]) return;
  const int m = nsteps[run];
  const double* a = alpha + (int64_t)run * mstride;
  const double* b = beta + (int64_t)run * (mstride + 1);
  double mx = 0.0;
  const int ns = (nz + zstride - 1) / zstride;
  for (int k = threadIdx.x; k < ns; k += blockDim.x) {
    double2 g = cf_eval(a, b, m, b0sq[run], z[k * zstride], E0, s);
    double2 p = prev[(int64_t)run * ns + k];
    mx = fmax(mx, hypot(g.x - p.x, g.y - p.y));
    prev[(int64_t)run * ns + k] = g;
  }
  mx = blk_max(mx);
  if (threadIdx.x == 0) {
    if (mx < tol) {
      if (++hits[run] >= 2) active[run] = 0;
    } else {
      hits[run] = 0;
    }
    if (active[run]) atomicAdd(n_active, 1);
  }
}

__global__ void k_cf_eval_all(const double* __restrict__ alpha, const double* __restrict__ beta,
                              const double* __restrict__ b0sq, const int* __restrict__ nsteps, int mstride, double E0,
                              double s, const double2* __restrict__ z, int nz, double2* __restrict__ out,
                              int64_t out_run_stride) {
  const int run = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nz) return;
  out[(int64_t)run * out_run_stride + k] =
      cf_eval(alpha + (int64_t)run * mstride, beta + (int64_t)run * (mstride + 1), nsteps[run], b0sq[run], z[k], E0, s);
}

// G[z][i][j] = sum over parts of (i == j ? Gk[r_ii] : (Gk[r_ij] - Gk[r_ii] - Gk[r_jj]) / 2).
__global__ void k_gf_combine(const double2* __restrict__ Ge, const double2* __restrict__ Gh, int p, int nz,
                             double2* __restrict__ G) {
  const int64_t total = (int64_t)nz * p * p;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(t / ((int64_t)p * p));
    int ij = (int)(t - (int64_t)k * p * p);
    int i = ij / p, j = ij - i * p;
    double2 g = make_double2(0.0, 0.0);
    const double2* parts[2] = {Ge, Gh};
    for (int q = 0; q < 2; ++q) {
      const double2* Gk = parts[q];
      if (!Gk) continue;
      if (i == j) {
        double2 v = Gk[(int64_t)i * nz + k];
        g.x += v.x;
        g.y += v.y;
      } else {
        int lo = min(i, j), hi = max(i, j);
        int r = p + (lo * (2 * p - lo - 1)) / 2 + (hi - lo - 1);
        double2 vp = Gk[(int64_t)r * nz + k], vi = Gk[(int64_t)lo * nz + k], vj = Gk[(int64_t)hi * nz + k];
        g.x += 0.5 * (vp.x - vi.x - vj.x);
        g.y += 0.5 * (vp.y - vi.y - vj.y);
      }
    }
    G[t] = g;
  }
}

static int ggrid(int64_t n) {
  int64_t b = (n + kGT - 1) / kGT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
}

struct GreenOptions {
  double tol;          // |Delta G| on the grid between checks
  int max_steps;       // per run
  size_t mem_budget;   // bytes for Lanczos vectors of one chunk of runs
};

// Builds the (p + p(p-1)/2) continued fractions of one part (electron or hole) and evaluates
// them on z; Gk[run][nz].  Returns false when the target sector does not exist.
static bool cf_part(ed_cluster& c, int spin, bool electron, int dtype, const DevBuf<double2>& zd, int nz,
                    double2* Gk, const GreenOptions& opt, int64_t* total_steps, int* max_steps) {
  cudaStream_t s = c.stream;
  const int nu = c.desc.n_up, nd = c.desc.n_dn, L = c.model.L;
  const int dN = electron ? 1 : -1;
  const int nu_t = nu + (spin == 0 ? dN : 0), nd_t = nd + (spin == 1 ? dN : 0);
  if (nu_t < 0 || nd_t < 0 || nu_t > L || nd_t > L) return false;
  const int p = c.model.ns;
  const int R = p + p * (p - 1) / 2;
  std::vector<int2> runs_h;
  for (int i = 0; i < p; ++i) runs_h.push_back(make_int2(i, -1));
  for (int i = 0; i < p; ++i)
    for (int j = i + 1; j < p; ++j) runs_h.push_back(make_int2(i, j));

  SpinTables& src = c.tables(spin == 0 ? nu : nd);
  SpinTables& dst = c.tables(spin == 0 ? nu_t : nd_t);
  c.tables(spin == 0 ? nd : nu);
  const int64_t ld = padded_ld(c.tables(nd_t).dim);
  SectorView sv = c.view(nu_t, nd_t, ld);
  const int64_t du = sv.d_up, dd = sv.d_dn, dim = du * dd;
  const int64_t dd_s = c.view(nu, nd, 0).d_dn;
  if (dim == 0) return false;
  const size_t es = dtype == ED_FP64 ? 8 : 4;
  const int64_t vstride = du * ld;
  int Rc = (int)std::max<int64_t>(1, std::min<int64_t>(R, (int64_t)(opt.mem_budget / (2 * vstride * es))));
  const int M = std::max(64, std::min<int>(opt.max_steps, (int)std::min<int64_t>(2 * dim + 16, 1 << 30)));
  const int nblk = lanczos_blocks(sv);
  RankView rv{src.rank_lo.p, src.rank_hi.p, src.split, (uint32_t)((1u << src.split) - 1u)};
  const int extra = spin == 1 ? (nu & 1) : 0;
  const int zstride = std::max(1, nz / 1024);
  const int nzs = (nz + zstride - 1) / zstride;
  DevBuf<int2> druns(R);
  ED_CUDA(cudaMemcpyAsync(druns.p, runs_h.data(), R * sizeof(int2), cudaMemcpyHostToDevice, s));
  int* host_active = (int*)(pinned_scratch() + 16);
  for (int r0 = 0; r0 < R; r0 += Rc) {
    const int rc = std::min(Rc, R - r0);
    DevBuf<char> V0(rc * vstride * es), V1(rc * vstride * es);
    ED_CUDA(cudaMemsetAsync(V0.p, 0, rc * vstride * es, s));
    DevBuf<double> alpha((size_t)rc * M), beta((size_t)rc * (M + 1)), beta0(rc), b0sq(rc), partial((size_t)rc * nblk * 3 + 8);
    DevBuf<int> active(rc), nsteps(rc), hits(rc), nact(1);
    DevBuf<unsigned> counter(rc);
    DevBuf<double2> prev((size_t)rc * nzs);
    ED_CUDA(cudaMemsetAsync(V1.p, 0, rc * vstride * es, s));
    ED_CUDA(cudaMemsetAsync(beta.p, 0, (size_t)rc * (M + 1) * sizeof(double), s));
    ED_CUDA(cudaMemsetAsync(nsteps.p, 0, rc * sizeof(int), s));
    ED_CUDA(cudaMemsetAsync(hits.p, 0, rc * sizeof(int), s));
    ED_CUDA(cudaMemsetAsync(counter.p, 0, rc * sizeof(unsigned), s));
    ED_CUDA(cudaMemsetAsync(prev.p, 0, (size_t)rc * nzs * sizeof(double2), s));
    dim3 g(ggrid(dim), rc);
    { ProfScope ps_(K_APPLY_COP, s, 0.0); k_apply_cop<<<g, kGT, 0, s>>>(c.omega.p, dd_s, dst.basis.p, rv, spin, electron ? 1 : 0, extra, druns.p + r0, dtype,
                                  V0.p, vstride, du, dd, ld); }
    ED_CHECK_LAUNCH();
    { ProfScope ps_(K_VECTOR, s, 0.0); k_run_norm_partial<<<dim3(nblk, rc), kGT, 0, s>>>(dtype, V0.p, vstride, du, dd, ld, partial.p); }
    ED_CHECK_LAUNCH();
    { ProfScope ps_(K_VECTOR, s, 0.0); k_run_norm_finish<<<rc, kGT, 0, s>>>(partial.p, nblk, b0sq.p, beta0.p, active.p); }
    ED_CHECK_LAUNCH();
    { ProfScope ps_(K_VECTOR, s, 0.0); k_run_scale<<<g, kGT, 0, s>>>(dtype, V0.p, vstride, du, dd, ld, beta0.p); }
    ED_CHECK_LAUNCH();
    // relative breakdown test needs b_0 = 1 for the normalized start
    LanczosScalars ls{alpha.p, beta.p, beta0.p, active.p, partial.p, counter.p, M, 0.0, nsteps.p};
    DevBuf<double> one(rc);
    {
      std::vector<double> ones(rc, 1.0);
      ED_CUDA(cudaMemcpyAsync(one.p, ones.data(), rc * sizeof(double), cudaMemcpyHostToDevice, s));
      ED_CUDA(cudaStreamSynchronize(s));
    }
    ls.beta0 = one.p;
    ls.btol = 1e-10;
    char* V[2] = {V0.p, V1.p};
    int cur = 0;
    int next_check = 32;
    for (int n = 0; n < M; ++n) {
      launch_lanczos_step(sv, c.hp, dtype, V[cur], V[cur ^ 1], vstride, rc, n, ls, nblk, s);
      launch_lanczos_next(dtype, V[cur ^ 1], V[cur], du, dd, ld, vstride, rc, n, ls, nullptr, nullptr, s);
      cur ^= 1;
      if (n + 1 == next_check || n + 1 == M) {
        ED_CUDA(cudaMemsetAsync(nact.p, 0, sizeof(int), s));
        { ProfScope ps_(K_GF_EVAL, s, 0.0); k_cf_check<<<rc, kGT, 0, s>>>(alpha.p, beta.p, b0sq.p, nsteps.p, M, active.p, hits.p, c.gs.E0,
                                      electron ? -1.0 : 1.0, zd.p, nz, zstride, prev.p, opt.tol, nact.p); }
        ED_CHECK_LAUNCH();
        ED_CUDA(cudaMemcpyAsync(host_active, nact.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        ED_CUDA(cudaStreamSynchronize(s));
        if (*host_active == 0) break;
        next_check = n + 1 + std::max(32, (n + 1) / 8);
      }
    }
    { ProfScope ps_(K_GF_EVAL, s, 0.0); k_cf_eval_all<<<dim3((nz + kGT - 1) / kGT, rc), kGT, 0, s>>>(alpha.p, beta.p, b0sq.p, nsteps.p, M, c.gs.E0,
                                                                  electron ? -1.0 : 1.0, zd.p, nz, Gk + (int64_t)r0 * nz, nz); }
    ED_CHECK_LAUNCH();
    std::vector<int> st(rc);
    ED_CUDA(cudaMemcpyAsync(st.data(), nsteps.p, rc * sizeof(int), cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    for (int v : st) {
      *total_steps += v;
      *max_steps = std::max(*max_steps, v);
    }
  }
  return true;
}

// phi[r] = (sum over the sites of runs[r]) c+_i W (create) or c_i W, in the target sector of the
// changed spin, rows padded to ld; vectors vstride apart.
void launch_apply_cop_runs(ed_cluster& c, int spin, bool electron, int dtype, const int2* runs_dev, int nruns,
                           void* phi, int64_t vstride, int64_t du, int64_t dd, int64_t ld, cudaStream_t s) {
  const int nu = c.desc.n_up, nd = c.desc.n_dn;
  const int dN = electron ? 1 : -1;
  SpinTables& src = c.tables(spin == 0 ? nu : nd);
  SpinTables& dst = c.tables(spin == 0 ? nu + dN : nd + dN);
  const int64_t dd_s = c.tables(nd).dim;
  RankView rv{src.rank_lo.p, src.rank_hi.p, src.split, (uint32_t)((1u << src.split) - 1u)};
  const int extra = spin == 1 ? (nu & 1) : 0;
  dim3 g(ggrid(du * dd), nruns);
  ProfScope ps_(K_APPLY_COP, s, 0.0);
  k_apply_cop<<<g, kGT, 0, s>>>(c.omega.p, dd_s, dst.basis.p, rv, spin, electron ? 1 : 0, extra, runs_dev, dtype, phi,
                                vstride, du, dd, ld);
  ED_CHECK_LAUNCH();
}

void run_green_cf(ed_cluster& c, int spin, const double2* z_host, int nz, double2* G_dev) {
  cudaStream_t s = c.stream;
  const int p = c.model.ns;
  const int R = p + p * (p - 1) / 2;
  const int dtype = c.desc.precision;
  GreenOptions opt{c.gf_tol > 0 ? c.gf_tol : (dtype == ED_FP64 ? 1e-10 : 1e-6), c.cf_max_steps > 0 ? c.cf_max_steps : 20000,
                   c.gf_mem_budget ? c.gf_mem_budget : size_t(48) << 30};
  DevBuf<double2> zd(nz);
  ED_CUDA(cudaMemcpyAsync(zd.p, z_host, nz * sizeof(double2), cudaMemcpyHostToDevice, s));
  DevBuf<double2> Ge((size_t)R * nz), Gh((size_t)R * nz);
  c.gf_total_steps = 0;
  c.gf_max_steps = 0;
  bool he = cf_part(c, spin, true, dtype, zd, nz, Ge.p, opt, &c.gf_total_steps, &c.gf_max_steps);
  bool hh = cf_part(c, spin, false, dtype, zd, nz, Gh.p, opt, &c.gf_total_steps, &c.gf_max_steps);
  { ProfScope ps_(K_GF_EVAL, s, 0.0); k_gf_combine<<<ggrid((int64_t)nz * p * p), kGT, 0, s>>>(he ? Ge.p : nullptr, hh ? Gh.p : nullptr, p, nz, G_dev); }
  ED_CHECK_LAUNCH();
  ED_CUDA(cudaStreamSynchronize(s));
}

}  // namespace ed
