// C ABI of libed (declarations and contracts in include/ed.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ed_common.cuh"

namespace ed {

static thread_local std::string g_last_error;
thread_local cudaStream_t g_alloc_stream = nullptr;

namespace {
struct PinnedScratch {
  double* p = nullptr;
  ~PinnedScratch() {
    if (p) cudaFreeHost(p);
  }
};
thread_local PinnedScratch t_pinned;
}  // namespace

double* pinned_scratch() {
  if (!t_pinned.p) ED_CUDA(cudaMallocHost(&t_pinned.p, kPinnedSlots * sizeof(double)));
  return t_pinned.p;
}

void set_last_error(const std::string& msg) { g_last_error = msg; }

void throw_cuda(cudaError_t e, const char* what, const char* file, int line) {
  std::string m = std::string("CUDA error ") + cudaGetErrorString(e) + " in " + what + " (" + file + ":" +
                  std::to_string(line) + ")";
  throw Error(e == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA, m);
}

GroundResult run_ground_state(ed_cluster& c, int dtype, double tol, int max_iter, uint64_t seed);
LowStatesResult run_davidson(ed_cluster& c, int k, double tol, int max_iter, uint64_t seed);
bool run_green_mixed(ed_cluster& c, int spin, const double2* z_host, int nz, double2* G_dev);
std::vector<double> mixed_weights(const std::vector<double>& E, double T);
void run_green_cf(ed_cluster& c, int spin, const double2* z_host, int nz, double2* G_dev);
bool run_green_band(ed_cluster& c, int spin, const double2* z_host, int nz, double2* G_dev);

template <typename F>
static ed_status guarded(F&& f) {
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

static void require(bool ok, const std::string& msg) {
  if (!ok) throw Error(ED_ERR_INVALID, msg);
}

static bool is_finite(double x) { return std::isfinite(x); }

// The cluster's tables and buffers live on the device it was created on; a call that launches
// work must find that device current (caller pointers are addresses on the current device).
static void require_cluster_device(const ed_cluster* c) {
  int dev = -1;
  ED_CUDA(cudaGetDevice(&dev));
  if (dev != c->device)
    throw Error(ED_ERR_INVALID, "the current device (" + std::to_string(dev) + ") is not the cluster's device (" +
                                    std::to_string(c->device) + ")");
}

// Validates a cluster description and builds the one-body matrix h (Eq. Hubbard with the bath
// terms of Eq. cdmft1), the list of hopping pairs and the kernel parameters.
void build_model(const ed_cluster_desc* desc, ModelHost& m, HopParams& hp) {
  require(desc != nullptr, "cluster description is NULL");
  const int ns = desc->n_sites, nb = desc->n_bath, L = ns + nb;
  require(ns >= 1 && nb >= 0 && L <= kMaxOrb, "need n_sites >= 1, n_bath >= 0, n_sites + n_bath <= 32");
  require(desc->t && desc->U, "t and U must not be NULL");
  require(nb == 0 || (desc->eps && desc->theta), "eps and theta must not be NULL when n_bath > 0");
  require(desc->n_up >= 0 && desc->n_up <= L && desc->n_dn >= 0 && desc->n_dn <= L, "sector outside [0, L]");
  require(desc->precision == ED_FP64 || desc->precision == ED_FP32, "precision must be ED_FP64 or ED_FP32");
  require(desc->gf_method == ED_GF_CF || desc->gf_method == ED_GF_BAND, "gf_method must be ED_GF_CF or ED_GF_BAND");
  require(is_finite(desc->mu), "mu is not finite");
  double tmax = 0.0;
  for (int i = 0; i < ns * ns; ++i) {
    require(is_finite(desc->t[i]), "t has a non-finite entry");
    tmax = std::max(tmax, std::fabs(desc->t[i]));
  }
  for (int i = 0; i < ns; ++i)
    for (int j = 0; j < i; ++j)
      require(std::fabs(desc->t[i * ns + j] - desc->t[j * ns + i]) <= 1e-12 * std::max(1.0, tmax), "t is not symmetric");
  for (int i = 0; i < ns; ++i) require(is_finite(desc->U[i]), "U has a non-finite entry");
  for (int a = 0; a < nb; ++a) require(is_finite(desc->eps[a]), "eps has a non-finite entry");
  for (int i = 0; i < ns * nb; ++i) require(is_finite(desc->theta[i]), "theta has a non-finite entry");

  m.ns = ns;
  m.nb = nb;
  m.L = L;
  m.h.assign((size_t)L * L, 0.0);
  m.U.assign(L, 0.0);
  for (int i = 0; i < ns; ++i) {
    for (int j = 0; j < ns; ++j) m.h[i * L + j] = desc->t[i * ns + j];
    m.h[i * L + i] -= desc->mu;
    m.U[i] = desc->U[i];
    for (int a = 0; a < nb; ++a) {
      m.h[i * L + ns + a] = desc->theta[i * nb + a];
      m.h[(ns + a) * L + i] = desc->theta[i * nb + a];
    }
  }
  for (int a = 0; a < nb; ++a) m.h[(ns + a) * L + ns + a] = desc->eps[a];
  for (int a = 0; a < L; ++a)
    for (int b = 0; b < L; ++b) {
      double v = m.h[a * L + b];
      if (a == b || v == 0.0) continue;
      int idx = -1;
      for (size_t k = 0; k < m.vals.size(); ++k)
        if (m.vals[k] == v) idx = (int)k;
      if (idx < 0) {
        require(m.vals.size() < (size_t)kMaxVals, "more than 128 distinct off-diagonal one-body values");
        idx = (int)m.vals.size();
        m.vals.push_back(v);
      }
      m.pair_a.push_back(a);
      m.pair_b.push_back(b);
      m.pair_vidx.push_back(idx);
    }
  std::memset(&hp, 0, sizeof(hp));
  for (size_t k = 0; k < m.vals.size(); ++k) {
    hp.val[k] = m.vals[k];
    hp.valf[k] = (float)m.vals[k];
  }
  hp.nvals = (int)m.vals.size();
  for (int i = 0; i < L; ++i) {
    hp.U[i] = m.U[i];
    hp.Uf[i] = (float)m.U[i];
    if (m.U[i] != 0.0) hp.umask |= 1u << i;
  }
  hp.uniform_u = 1;
  for (int i = 0; i < L; ++i)
    if (((hp.umask >> i) & 1u) && m.U[i] != hp.u0) {
      if (hp.u0 == 0.0)
        hp.u0 = m.U[i];
      else
        hp.uniform_u = 0;
    }
  hp.u0f = (float)hp.u0;
}

// A cluster whose work runs on `stream` (owned by the caller) or, when stream is nullptr, on a
// stream of its own.  Throws ed::Error.
std::unique_ptr<ed_cluster> cluster_create_on(const ed_cluster_desc* desc, cudaStream_t stream) {
  auto c = std::make_unique<ed_cluster>();
  build_model(desc, c->model, c->hp);
  c->desc = *desc;
  c->desc.t = c->desc.U = c->desc.eps = c->desc.theta = nullptr;
  if (!(c->desc.tol > 0.0)) c->desc.tol = 1e-12;
  if (c->desc.max_iter <= 0) c->desc.max_iter = 600;
  ED_CUDA(cudaGetDevice(&c->device));
  if (stream) {
    c->stream = stream;
    c->owns_stream = false;
  } else {
    ED_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  }
  c->tables(desc->n_up);
  c->tables(desc->n_dn);
  return c;
}

}  // namespace ed

using namespace ed;

SpinTables& ed_cluster::tables(int N) {
  auto it = spins.find(N);
  if (it != spins.end()) return *it->second;
  if (N < 0 || N > model.L) throw Error(ED_ERR_INVALID, "particle number outside [0, L]");
  auto t = build_spin_tables(model, N, stream);
  SpinTables& ref = *t;
  spins[N] = std::move(t);
  return ref;
}

SectorView ed_cluster::view(int n_up, int n_dn, int64_t ld) {
  SpinTables& u = tables(n_up);
  SpinTables& d = tables(n_dn);
  SectorView v;
  v.d_up = u.dim;
  v.d_dn = d.dim;
  v.ld = ld > 0 ? ld : d.dim;
  v.B_up = u.basis.p;
  v.B_dn = d.basis.p;
  v.ptr_up = u.ptr.p;
  v.ent_up = u.ent.p;
  v.ptr_dn = d.ptr.p;
  v.ent_dn = d.ent.p;
  v.ell_dn = d.ell.p;
  v.e_up = u.ediag.p;
  v.e_dn = d.ediag.p;
  v.e_up32 = u.ediag32.p;
  v.e_dn32 = d.ediag32.p;
  v.two_pass_min_bytes = two_pass_min_bytes;
  return v;
}

extern "C" {

const char* ed_last_error(void) { return g_last_error.c_str(); }

ed_status ed_cluster_create(const ed_cluster_desc* desc, ed_cluster** out) {
  return guarded([&]() -> ed_status {
    require(desc != nullptr && out != nullptr, "desc and out must not be NULL");
    *out = nullptr;
    *out = ed::cluster_create_on(desc, nullptr).release();
    return ED_OK;
  });
}

void ed_cluster_destroy(ed_cluster* c) {
  if (!c) return;
  try {
    cudaStreamSynchronize(c->stream);
    cudaStream_t s = c->owns_stream ? c->stream : nullptr;
    delete c;
    if (s) cudaStreamDestroy(s);
  } catch (...) {
  }
}

ed_status ed_ground_state(ed_cluster* c, double* E0, double* residual, int* iters) {
  return guarded([&]() -> ed_status {
    require(c != nullptr, "cluster is NULL");
    require_cluster_device(c);
    GroundResult r;
    if (c->davidson_states > 1) {
      LowStatesResult d = run_davidson(*c, c->davidson_states, c->desc.tol, c->desc.max_iter, c->desc.seed);
      c->low_E = d.E;
      r.E0 = d.E[0];
      r.residual = *std::max_element(d.residual.begin(), d.residual.end());
      r.iters = d.iters;
      r.converged = d.converged;
      r.gap = d.E.size() > 1 ? d.E[1] - d.E[0] : 0.0;
      // the mixture covers the degenerate ground manifold only if a state above it was found
      r.degenerate = d.E.size() > 1 && d.E.back() - d.E[0] <= 1e-9 * std::max(1.0, std::fabs(d.E[0]));
    } else {
      r = run_ground_state(*c, c->desc.precision, c->desc.tol, c->desc.max_iter, c->desc.seed);
      c->low_E.clear();
    }
    c->gs = r;
    c->have_gs = true;
    if (E0) *E0 = r.E0;
    if (residual) *residual = r.residual;
    if (iters) *iters = r.iters;
    if (!r.converged) return ED_WARN_NOT_CONVERGED;
    return r.degenerate ? ED_WARN_DEGENERATE : ED_OK;
  });
}

ed_status ed_ground_vector(ed_cluster* c, double* out, int out_is_device) {
  return guarded([&]() -> ed_status {
    require(c != nullptr && out != nullptr, "cluster and out must not be NULL");
    require_cluster_device(c);
    if (!c->have_gs) throw Error(ED_ERR_STATE, "no ground state yet");
    int64_t n = (int64_t)binomial(c->model.L, c->desc.n_up) * (int64_t)binomial(c->model.L, c->desc.n_dn);
    ED_CUDA(cudaMemcpyAsync(out, c->omega.p, n * sizeof(double), out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            c->stream));
    ED_CUDA(cudaStreamSynchronize(c->stream));
    return ED_OK;
  });
}

ed_status ed_green(ed_cluster* c, const double* omega, int n_freq, double eta, int axis, int spin, double* G_out,
                   int out_is_device) {
  return guarded([&]() -> ed_status {
    require(c != nullptr && omega != nullptr && G_out != nullptr, "cluster, omega and G_out must not be NULL");
    require(n_freq > 0, "n_freq must be positive");
    require(axis == ED_AXIS_REAL || axis == ED_AXIS_MATSUBARA, "axis must be ED_AXIS_REAL or ED_AXIS_MATSUBARA");
    require(spin == 0 || spin == 1, "spin must be 0 or 1");
    require(is_finite(eta), "eta is not finite");
    require_cluster_device(c);
    ed_status st = ED_OK;
    if (!c->have_gs) {
      st = ed_ground_state(c, nullptr, nullptr, nullptr);
      if (st < 0) return st;
    }
    std::vector<double2> z(n_freq);
    for (int k = 0; k < n_freq; ++k) {
      require(is_finite(omega[k]), "omega has a non-finite entry");
      z[k] = axis == ED_AXIS_REAL ? make_double2(omega[k], eta) : make_double2(0.0, omega[k]);
    }
    const int p = c->model.ns;
    DevBuf<double2> Gd;
    double2* Gdev = (double2*)G_out;
    if (!out_is_device) {
      Gd.alloc((size_t)n_freq * p * p);
      Gdev = Gd.p;
    }
    if (c->davidson_states > 1) {
      c->gf_converged = run_green_mixed(*c, spin, z.data(), n_freq, Gdev);
      if (!c->gf_converged && st == ED_OK) st = ED_WARN_NOT_CONVERGED;
    } else if (c->desc.gf_method == ED_GF_CF) {
      run_green_cf(*c, spin, z.data(), n_freq, Gdev);
    } else {
      c->gf_converged = run_green_band(*c, spin, z.data(), n_freq, Gdev);
      if (!c->gf_converged && st == ED_OK) st = ED_WARN_NOT_CONVERGED;
    }
    if (!out_is_device) {
      ED_CUDA(cudaMemcpyAsync(G_out, Gd.p, (size_t)n_freq * p * p * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
      ED_CUDA(cudaStreamSynchronize(c->stream));
    }
    return st;
  });
}

ed_status ed_set_option(ed_cluster* c, int option, double value) {
  return guarded([&]() -> ed_status {
    require(c != nullptr, "cluster is NULL");
    require(is_finite(value), "option value is not finite");
    switch (option) {
      case ED_OPT_BAND_MAX_DIM: c->band_max_dim = (int)value; break;
      case ED_OPT_CF_MAX_STEPS: c->cf_max_steps = (int)value; break;
      case ED_OPT_GF_TOL: c->gf_tol = value; break;
      case ED_OPT_DAVIDSON_STATES:
        require(value >= 1.0 && value <= 16.0, "ED_OPT_DAVIDSON_STATES must be in [1, 16]");
        c->davidson_states = (int)value;
        c->have_gs = false;
        break;
      case ED_OPT_TENSOR_GRAM:
        require(value == 0.0 || value == 1.0, "ED_OPT_TENSOR_GRAM must be 0 or 1");
        c->tensor_gram = value != 0.0;
        break;
      case ED_OPT_TEMPERATURE:
        require(value >= 0.0, "ED_OPT_TEMPERATURE must be >= 0");
        c->temperature = value;
        break;
      case ED_OPT_TWO_PASS_MIN_BYTES:
        require(value >= 0.0, "ED_OPT_TWO_PASS_MIN_BYTES must be >= 0");
        c->two_pass_min_bytes = value >= 9.0e18 ? INT64_MAX : (int64_t)value;
        break;
      default: throw Error(ED_ERR_INVALID, "unknown option");
    }
    return ED_OK;
  });
}

ed_status ed_low_states(const ed_cluster* c, int capacity, double* E, double* weights, int* count) {
  return guarded([&]() -> ed_status {
    require(c != nullptr, "cluster is NULL");
    if (!c->have_gs) throw Error(ED_ERR_STATE, "no ground state yet");
    std::vector<double> e = c->low_E.empty() ? std::vector<double>{c->gs.E0} : c->low_E;
    std::vector<double> w = mixed_weights(e, c->low_E.empty() ? 0.0 : c->temperature);
    if (count) *count = (int)e.size();
    const int n = std::min<int>(capacity, (int)e.size());
    for (int i = 0; i < n; ++i) {
      if (E) E[i] = e[i];
      if (weights) weights[i] = w[i];
    }
    return ED_OK;
  });
}

ed_status ed_green_stats(const ed_cluster* c, int64_t* total_steps, int* max_steps) {
  return guarded([&]() -> ed_status {
    require(c != nullptr, "cluster is NULL");
    if (total_steps) *total_steps = c->gf_total_steps;
    if (max_steps) *max_steps = c->gf_max_steps;
    return ED_OK;
  });
}

ed_status ed_sector_dims(const ed_cluster* c, int n_up, int n_dn, int64_t* d_up, int64_t* d_dn) {
  return guarded([&]() -> ed_status {
    require(c != nullptr, "cluster is NULL");
    require(n_up >= 0 && n_up <= c->model.L && n_dn >= 0 && n_dn <= c->model.L, "sector outside [0, L]");
    if (d_up) *d_up = (int64_t)binomial(c->model.L, n_up);
    if (d_dn) *d_dn = (int64_t)binomial(c->model.L, n_dn);
    return ED_OK;
  });
}

ed_status ed_basis(int L, int N, uint32_t* out, int64_t capacity, int64_t* dim) {
  return guarded([&]() -> ed_status {
    require(L >= 1 && L <= kMaxOrb && N >= 0 && N <= L, "need 1 <= L <= 32 and 0 <= N <= L");
    int64_t d = (int64_t)binomial(L, N);
    if (dim) *dim = d;
    require(d < (int64_t(1) << 24), "sector dimension per spin must be < 2^24");
    require(out != nullptr && capacity >= d, "output capacity smaller than C(L, N)");
    basis_to_host(L, N, out, d);
    return ED_OK;
  });
}

ed_status ed_hop_table(ed_cluster* c, int N, int32_t* row_ptr, uint32_t* entries, double* values, int64_t cap_entries,
                       int64_t* n_entries, int* n_values) {
  return guarded([&]() -> ed_status {
    require(c != nullptr, "cluster is NULL");
    require_cluster_device(c);
    SpinTables& t = c->tables(N);
    if (n_entries) *n_entries = t.nnz;
    if (n_values) *n_values = (int)c->model.vals.size();
    require(row_ptr && entries && values, "row_ptr, entries and values must not be NULL");
    require(cap_entries >= t.nnz, "entry capacity too small");
    ED_CUDA(cudaMemcpyAsync(row_ptr, t.ptr.p, (t.dim + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    if (t.nnz) ED_CUDA(cudaMemcpyAsync(entries, t.ent.p, t.nnz * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    ED_CUDA(cudaStreamSynchronize(c->stream));
    for (size_t k = 0; k < c->model.vals.size(); ++k) values[k] = c->model.vals[k];
    return ED_OK;
  });
}

ed_status ed_hpsi(ed_cluster* c, int n_up, int n_dn, int dtype, const void* x, void* y, int64_t ld, void* stream) {
  return guarded([&]() -> ed_status {
    require(c != nullptr && x != nullptr && y != nullptr, "cluster, x and y must not be NULL");
    require(dtype == ED_FP64 || dtype == ED_FP32, "dtype must be ED_FP64 or ED_FP32");
    require_cluster_device(c);
    SectorView sv = c->view(n_up, n_dn, ld);
    require(ld <= 0 || ld >= sv.d_dn, "ld must be >= d_dn (or <= 0 for d_dn)");
    cudaStream_t s = (cudaStream_t)stream;  // NULL is the CUDA default stream
    launch_hpsi(sv, c->hp, dtype, x, y, s);
    return ED_OK;
  });
}

}  // extern "C"
