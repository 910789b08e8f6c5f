// Several low-lying states of a sector by the Davidson method, and the mixed-state Green function
// built on them.  The paper recommends Davidson when the ground state is degenerate, where Lanczos
// converges to an arbitrary vector of the ground manifold (Sec. 4.2), and its library targets
// several low states (Davidson_states) at a low temperature (temperature): Sec. 9, global options.
//
// Block Davidson-Liu in FP64: a basis V (at most kDavMax vectors, thick-restarted to the ~2k
// lowest Ritz vectors) and W = H V; the projection T = V^T W is diagonalized on the host (cyclic Jacobi); the
// residuals r_i = W s_i - lambda_i V s_i of the k lowest Ritz pairs are preconditioned with the
// diagonal of H, t_i = r_i / (lambda_i - D), orthogonalized against V twice and among themselves
// (symmetric orthonormalization, dropping dependent directions), and appended.  Every product with
// H is the library's H.psi kernel; every block operation is the band code's Gram and block-update
// kernels (deterministic reductions).
//
// Mixed state: G(z) = sum_s p_s G_s(z) with G_s the Green function of state s (its own energy in
// the place of E0, Eq. green) and p_s = exp(-(E_s - E_0) / T) / Z over the states found; at T = 0
// equal weights on the states within 1e-9 max(1, |E_0|) of E_0 (the limit T -> 0 of a degenerate
// ground manifold), which makes G independent of the basis chosen inside that manifold.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ed_common.cuh"

namespace ed {

void gram_f64(const double* X, int64_t xbstride, int nb, int px, const double* Y, int py, int64_t vstride, int64_t n,
              DevBuf<double>& P, DevBuf<unsigned>& tk, double* G, cudaStream_t s);
void block_axpy_f64(double* Y, int py, const double* X, int64_t xbstride, int nb, int px, const double* C,
                    int64_t vstride, int64_t n, int mode, cudaStream_t s);
void run_green_cf(ed_cluster& c, int spin, const double2* z_host, int nz, double2* G_dev);
bool run_green_band(ed_cluster& c, int spin, const double2* z_host, int nz, double2* G_dev);

constexpr int kDavBlock = 16;  // vectors per block of the Gram / update kernels
constexpr int kDavMax = 64;    // basis size before a thick restart (64 coefficient rows per update)

// D[u][d] = e_up[u] + e_dn[d] + sum_{i: up and down occupied} U_i, the diagonal of H (Eq. factorized)
__global__ void k_hdiag(SectorView sv, HopParams hp, double* __restrict__ D) {
  for_each_element(sv.d_up, sv.d_dn, [&](int64_t u, int64_t d, int64_t idx) {
    double v = sv.e_up[u] + sv.e_dn[d];
    uint32_t dbl = sv.B_up[u] & sv.B_dn[d] & hp.umask;
    while (dbl) {
      v += hp.U[__ffs(dbl) - 1];
      dbl &= dbl - 1u;
    }
    D[u * sv.ld + d] = v;
  });
}

// T[o] = R[o] / (lam - D[o]), the denominator kept at least `floor` away from zero.
__global__ void k_precond(const double* __restrict__ R, const double* __restrict__ D, double lam, double floor,
                          int64_t du, int64_t dd, int64_t ld, double* __restrict__ T) {
  for_each_element(du, dd, [&](int64_t u, int64_t d, int64_t idx) {
    const int64_t o = u * ld + d;
    double den = lam - D[o];
    if (fabs(den) < floor) den = den < 0.0 ? -floor : floor;
    T[o] = R[o] / den;
  });
}

__global__ void k_cplx_axpy(double2* __restrict__ y, const double2* __restrict__ x, double a, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    y[t] = make_double2(y[t].x + a * x[t].x, y[t].y + a * x[t].y);
}

static unsigned dgrid(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

// Cyclic Jacobi eigen-decomposition of the symmetric m x m matrix A (row-major, destroyed):
// eigenvalues ascending in w, eigenvectors as the columns of V (row-major).
static void jacobi_eig(int m, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        tot += A[(size_t)i * m + j] * A[(size_t)i * m + j];
        if (i != j) off += A[(size_t)i * m + j] * A[(size_t)i * m + j];
      }
    if (!(off > 1e-30 * tot)) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[(size_t)p * m + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double th = (A[(size_t)q * m + q] - A[(size_t)p * m + p]) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {  // columns p, q
          const double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
          A[(size_t)k * m + p] = c * akp - s * akq;
          A[(size_t)k * m + q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q
          const double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
          A[(size_t)p * m + k] = c * apk - s * aqk;
          A[(size_t)q * m + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double vkp = V[(size_t)k * m + p], vkq = V[(size_t)k * m + q];
          V[(size_t)k * m + p] = c * vkp - s * vkq;
          V[(size_t)k * m + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return A[(size_t)a * m + a] < A[(size_t)b * m + b]; });
  w.resize(m);
  std::vector<double> Vs((size_t)m * m);
  for (int j = 0; j < m; ++j) {
    w[j] = A[(size_t)order[j] * m + order[j]];
    for (int i = 0; i < m; ++i) Vs[(size_t)i * m + j] = V[(size_t)i * m + order[j]];
  }
  V.swap(Vs);
}

struct DavWork {
  int64_t du, dd, ld, vstride, n;
  SectorView sv;
  cudaStream_t s;
  DevBuf<double> P, G, C;
  DevBuf<unsigned> tk;
  std::vector<double> hG;
  // G[i][j] = <X_i, Y_j>, i < nx (vectors of X, consecutive), j < ny; to the host as nx x ny
  void gram(const double* X, int nx, const double* Y, int ny, std::vector<double>& out) {
    const int nb = (nx + kDavBlock - 1) / kDavBlock;
    if (G.n < (size_t)nb * kDavBlock * ny) G.alloc((size_t)nb * kDavBlock * ny);
    gram_f64(X, kDavBlock * vstride, nb, kDavBlock, Y, ny, vstride, n, P, tk, G.p, s);
    hG.resize((size_t)nb * kDavBlock * ny);
    ED_CUDA(cudaMemcpyAsync(hG.data(), G.p, hG.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    out.assign((size_t)nx * ny, 0.0);
    for (int i = 0; i < nx; ++i)
      for (int j = 0; j < ny; ++j) out[(size_t)i * ny + j] = hG[(size_t)i * ny + j];
  }
  // Y (ny vectors; mode 0: =, 1: -=) X C with C host nx x ny; X consecutive vectors (nx <= 64)
  void update(double* Y, int ny, const double* X, int nx, const std::vector<double>& Ch, int mode) {
    const int nb = (nx + kDavBlock - 1) / kDavBlock;
    std::vector<double> Cp((size_t)nb * kDavBlock * ny, 0.0);  // rows past nx are zero (zero vectors)
    std::copy(Ch.begin(), Ch.begin() + (size_t)nx * ny, Cp.begin());
    if (C.n < Cp.size()) C.alloc(Cp.size());
    ED_CUDA(cudaMemcpyAsync(C.p, Cp.data(), Cp.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    block_axpy_f64(Y, ny, X, kDavBlock * vstride, nb, kDavBlock, C.p, vstride, n, mode, s);
    ED_CUDA(cudaStreamSynchronize(s));  // Cp goes out of scope
  }
};

// Symmetric orthonormalization of the nt vectors T (in place): G = T^T T = U l U^T, T <- T U l^-1/2
// over the directions with l > rel max(l); returns how many remain (they are moved to the front).
static int orthonormalize_block(DavWork& w, double* T, int nt, double rel) {
  if (nt == 0) return 0;
  std::vector<double> G, l, U;
  w.gram(T, nt, T, nt, G);
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < i; ++j) G[(size_t)i * nt + j] = G[(size_t)j * nt + i] = 0.5 * (G[(size_t)i * nt + j] + G[(size_t)j * nt + i]);
  jacobi_eig(nt, G, l, U);
  const double lmax = l.empty() ? 0.0 : l.back();
  std::vector<int> keep;
  for (int j = nt - 1; j >= 0; --j)
    if (l[j] > rel * lmax && l[j] > 0.0) keep.push_back(j);
  const int nk = (int)keep.size();
  if (nk == 0) return 0;
  std::vector<double> C((size_t)nt * nk);
  for (int i = 0; i < nt; ++i)
    for (int c = 0; c < nk; ++c) C[(size_t)i * nk + c] = U[(size_t)i * nt + keep[c]] / std::sqrt(l[keep[c]]);
  w.update(T, nk, T, nt, C, 0);
  return nk;
}

LowStatesResult run_davidson(ed_cluster& c, int k, double tol, int max_iter, uint64_t seed) {
  cudaStream_t s = c.stream;
  const int nu = c.desc.n_up, nd = c.desc.n_dn;
  const int64_t ld = padded_ld(c.tables(nd).dim);
  DavWork w;
  w.sv = c.view(nu, nd, ld);
  w.s = s;
  w.du = w.sv.d_up;
  w.dd = w.sv.d_dn;
  w.ld = ld;
  w.vstride = w.du * ld;
  w.n = w.vstride;
  const int64_t dim = w.du * w.dd;
  k = (int)std::min<int64_t>(std::max(k, 1), std::min<int64_t>(dim, kDavBlock));
  const int mmax = (int)std::min<int64_t>(kDavMax, std::max<int64_t>(k + 1, std::min<int64_t>(dim, kDavMax)));
  static_assert(kDavMax >= 2 * kDavBlock, "the basis must hold the restart vectors and a block of new ones");
  const size_t vb = (size_t)w.vstride * sizeof(double);
  DevBuf<double> V((size_t)kDavMax * w.vstride), Wv((size_t)kDavMax * w.vstride), Xr((size_t)kDavBlock * w.vstride),
      HX((size_t)kDavBlock * w.vstride), R((size_t)kDavBlock * w.vstride), Tn((size_t)kDavBlock * w.vstride),
      D(w.vstride);
  ED_CUDA(cudaMemsetAsync(V.p, 0, (size_t)kDavMax * vb, s));
  ED_CUDA(cudaMemsetAsync(Wv.p, 0, (size_t)kDavMax * vb, s));
  for (DevBuf<double>* b : {&Xr, &HX, &R, &Tn}) ED_CUDA(cudaMemsetAsync(b->p, 0, (size_t)kDavBlock * vb, s));
  ED_CUDA(cudaMemsetAsync(D.p, 0, vb, s));
  {
    ProfScope ps_(K_VECTOR, s, 0.0);
    k_hdiag<<<dgrid(dim), 256, 0, s>>>(w.sv, c.hp, D.p);
    ED_CHECK_LAUNCH();
  }
  auto vec = [&](DevBuf<double>& b, int i) { return b.p + (int64_t)i * w.vstride; };
  // start: k seeded vectors, orthonormalized
  for (int i = 0; i < k; ++i) launch_start_vector(ED_FP64, vec(V, i), w.du, w.dd, ld, seed + 0x9E3779B97F4A7C15ull * (i + 1), s);
  int m = orthonormalize_block(w, V.p, k, 1e-14);
  m = orthonormalize_block(w, V.p, m, 1e-14);
  for (int i = 0; i < m; ++i) launch_hpsi(w.sv, c.hp, ED_FP64, vec(V, i), vec(Wv, i), s);
  std::vector<double> T((size_t)kDavMax * kDavMax, 0.0), blk;
  auto set_cols = [&](int j0, int nj) {  // T[:, j0 .. j0 + nj) from V^T W
    w.gram(V.p, j0 + nj, vec(Wv, j0), nj, blk);
    for (int i = 0; i < j0 + nj; ++i)
      for (int j = 0; j < nj; ++j) {
        T[(size_t)i * kDavMax + j0 + j] = blk[(size_t)i * nj + j];
        T[(size_t)(j0 + j) * kDavMax + i] = blk[(size_t)i * nj + j];
      }
  };
  set_cols(0, m);
  LowStatesResult out;
  std::vector<double> lam, S, rn(k);
  const int maxit = max_iter > 0 ? max_iter : 600;
  int it = 0;
  bool conv = false;
  for (; it < maxit; ++it) {
    std::vector<double> A((size_t)m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = 0.5 * (T[(size_t)i * kDavMax + j] + T[(size_t)j * kDavMax + i]);
    jacobi_eig(m, A, lam, S);
    const int kk = std::min(k, m);
    // Ritz vectors kept at a thick restart: about twice the states sought (restarting on the k
    // states alone discards the search directions and stalls the method)
    const int kr = std::min(m, std::min(kDavBlock, std::max(2 * k, k + 6)));
    std::vector<double> Sk((size_t)m * kr), SL((size_t)kk * kk, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < kr; ++j) Sk[(size_t)i * kr + j] = S[(size_t)i * m + j];
    for (int j = 0; j < kk; ++j) SL[(size_t)j * kk + j] = lam[j];
    w.update(Xr.p, kr, V.p, m, Sk, 0);   // Ritz vectors
    w.update(HX.p, kr, Wv.p, m, Sk, 0);  // H times them
    ED_CUDA(cudaMemcpyAsync(R.p, HX.p, (size_t)kk * vb, cudaMemcpyDeviceToDevice, s));
    w.update(R.p, kk, Xr.p, kk, SL, 1);  // r_i = H x_i - lambda_i x_i
    std::vector<double> RR;
    w.gram(R.p, kk, R.p, kk, RR);
    int nnew = 0;
    bool all = true;
    for (int i = 0; i < kk; ++i) {
      rn[i] = std::sqrt(std::max(0.0, RR[(size_t)i * kk + i]));
      if (rn[i] > tol * std::max(1.0, std::fabs(lam[i]))) all = false;
    }
    if (all && kk == k) {
      conv = true;
      break;
    }
    if (m == dim) break;  // the basis spans the sector: the Ritz pairs are exact up to rounding
    const double flo = 1e-3 * std::max(1.0, std::fabs(lam[0]));
    for (int i = 0; i < kk; ++i) {
      if (rn[i] <= tol * std::max(1.0, std::fabs(lam[i]))) continue;
      ProfScope ps_(K_VECTOR, s, 0.0);
      k_precond<<<dgrid(dim), 256, 0, s>>>(vec(R, i), D.p, lam[i], flo, w.du, w.dd, ld, vec(Tn, nnew));
      ED_CHECK_LAUNCH();
      ++nnew;
    }
    if (m + nnew > mmax) {  // thick restart on the kr lowest Ritz vectors
      ED_CUDA(cudaMemcpyAsync(V.p, Xr.p, (size_t)kr * vb, cudaMemcpyDeviceToDevice, s));
      ED_CUDA(cudaMemcpyAsync(Wv.p, HX.p, (size_t)kr * vb, cudaMemcpyDeviceToDevice, s));
      ED_CUDA(cudaMemsetAsync(vec(V, kr), 0, (size_t)(kDavMax - kr) * vb, s));
      ED_CUDA(cudaMemsetAsync(vec(Wv, kr), 0, (size_t)(kDavMax - kr) * vb, s));
      m = kr;
      set_cols(0, m);
    }
    for (int pass = 0; pass < 2; ++pass) {  // t <- t - V (V^T t), twice
      std::vector<double> Cm;
      w.gram(V.p, m, Tn.p, nnew, Cm);
      w.update(Tn.p, nnew, V.p, m, Cm, 1);
    }
    const int nk = orthonormalize_block(w, Tn.p, nnew, 1e-20);
    if (nk == 0) break;  // no new direction: stagnation
    ED_CUDA(cudaMemcpyAsync(vec(V, m), Tn.p, (size_t)nk * vb, cudaMemcpyDeviceToDevice, s));
    for (int i = 0; i < nk; ++i) launch_hpsi(w.sv, c.hp, ED_FP64, vec(V, m + i), vec(Wv, m + i), s);
    set_cols(m, nk);
    m += nk;
  }
  // results: energies, residuals and the states, contiguous (d_up x d_dn) for the Green function
  const int kk = std::min(k, m);
  out.E.assign(lam.begin(), lam.begin() + kk);
  out.residual.resize(kk);
  for (int i = 0; i < kk; ++i) out.residual[i] = rn[i] / std::max(1.0, std::fabs(lam[i]));
  out.iters = it;
  out.converged = conv;
  c.low.alloc((size_t)kk * dim);
  for (int i = 0; i < kk; ++i)
    launch_copy_ld(ED_FP64, c.low.p + (int64_t)i * dim, w.dd, ED_FP64, vec(Xr, i), ld, nullptr, w.du, w.dd, s);
  c.omega.alloc(std::max<int64_t>(dim, 1));
  ED_CUDA(cudaMemcpyAsync(c.omega.p, c.low.p, dim * sizeof(double), cudaMemcpyDeviceToDevice, s));
  ED_CUDA(cudaStreamSynchronize(s));
  return out;
}

// Weights of the mixed state (see the file comment).
std::vector<double> mixed_weights(const std::vector<double>& E, double T) {
  std::vector<double> p(E.size(), 0.0);
  if (E.empty()) return p;
  double z = 0.0;
  for (size_t i = 0; i < E.size(); ++i) {
    p[i] = T > 0.0 ? std::exp(-(E[i] - E[0]) / T) : (E[i] - E[0] <= 1e-9 * std::max(1.0, std::fabs(E[0])) ? 1.0 : 0.0);
    z += p[i];
  }
  for (double& v : p) v /= z;
  return p;
}

// G = sum_s p_s G_s over the stored low states: each state in turn becomes the source vector and
// reference energy of the Green-function runs.  Returns false if a band run did not converge.
bool run_green_mixed(ed_cluster& c, int spin, const double2* z_host, int nz, double2* G_dev) {
  cudaStream_t s = c.stream;
  const int p = c.model.ns;
  const int64_t n = (int64_t)nz * p * p;
  const int64_t dim = (int64_t)binomial(c.model.L, c.desc.n_up) * (int64_t)binomial(c.model.L, c.desc.n_dn);
  const std::vector<double> wts = mixed_weights(c.low_E, c.temperature);
  DevBuf<double2> Gs(n);
  ED_CUDA(cudaMemsetAsync(G_dev, 0, n * sizeof(double2), s));
  const double E0 = c.gs.E0;
  bool conv = true;
  for (size_t st = 0; st < wts.size(); ++st) {
    if (wts[st] <= 0.0) continue;
    ED_CUDA(cudaMemcpyAsync(c.omega.p, c.low.p + (int64_t)st * dim, dim * sizeof(double), cudaMemcpyDeviceToDevice, s));
    c.gs.E0 = c.low_E[st];
    if (c.desc.gf_method == ED_GF_CF)
      run_green_cf(c, spin, z_host, nz, Gs.p);
    else
      conv = run_green_band(c, spin, z_host, nz, Gs.p) && conv;
    ProfScope ps_(K_GF_EVAL, s, 0.0);
    k_cplx_axpy<<<dgrid(n), 256, 0, s>>>(G_dev, Gs.p, wts[st], n);
    ED_CHECK_LAUNCH();
  }
  c.gs.E0 = E0;
  ED_CUDA(cudaMemcpyAsync(c.omega.p, c.low.p, dim * sizeof(double), cudaMemcpyDeviceToDevice, s));
  ED_CUDA(cudaStreamSynchronize(s));
  return conv;
}

}  // namespace ed
