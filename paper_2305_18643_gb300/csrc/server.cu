// Served form: a request loop that admits cluster solves by device memory and runs them side by
// side on the GPU (continuous batching).
//
// A quantum-cluster method issues one impurity solve per iteration of its outer loop (VCA,
// CDMFT, Sec. 5), and many such loops may share one GPU.  The server takes those solves as they
// come:
//   - max_slots lanes, each a host thread with a non-blocking CUDA stream; every device buffer a
//     lane creates is allocated and freed stream-ordered on that stream, so no lane ever waits
//     for another lane's work;
//   - admission by device memory: a request's footprint follows from closed forms of its sector
//     dimensions (tables, Lanczos vectors, Green-function vectors, G); it is admitted when a lane
//     is free and the footprint fits what is left of the budget.  Order is first come, first
//     served, and a later request that fits may pass a waiting one at most kMaxBypass times;
//   - small requests (every sector at most batch_max_dim elements, <= 20 orbitals, continued
//     fractions) that share precision, grid and level cap are taken together by one lane and
//     solved by the persistent kernels of the batched form with a fixed block configuration;
//     larger requests run the single-cluster path.  The path depends on the request alone, and
//     the arithmetic of neither path depends on the other requests in flight.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ed_common.cuh"

namespace ed {

GroundResult run_ground_state(ed_cluster& c, int dtype, double tol, int max_iter, uint64_t seed);
void run_green_cf(ed_cluster& c, int spin, const double2* z_host, int nz, double2* G_dev);
bool run_green_band(ed_cluster& c, int spin, const double2* z_host, int nz, double2* G_dev);
void batch_solve(const ed_cluster_desc* descs, int n, int precision, const double2* z_host, int nz, bool do_gf,
                 int cf_max_steps, double* E0_out, double* res_out, int* status_out, int* iters_out,
                 int64_t* gf_steps_out, double2* G_dev_out, cudaStream_t s, int fixed_threads, int fixed_mode);
size_t batch_device_bytes(const ed_cluster_desc* descs, int n, int precision, int nz, int cf_max_steps, int sms);

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxBypass = 8;
constexpr int kBatchThreads = 256, kBatchMode = 1;  // fixed block configuration of the batched path
constexpr int kDefaultCfCap = kCfDefaultMaxLevels;
constexpr size_t kMargin = size_t(32) << 20;

// ---------------------------------------------------------------- footprints (closed forms)
size_t spin_table_bytes(int L, int N, int npairs) {
  const int64_t d = (int64_t)binomial(L, N);
  const int split = L / 2;
  const int64_t nnz = (int64_t)npairs * (int64_t)binomial(L - 2, N - 1);
  const int64_t zmax = std::min<int64_t>(npairs, (int64_t)N * (L - N)) + kEllPad;
  return (size_t)d * (4 + 4 + 8 + 4) + 4 + (size_t)std::max<int64_t>(nnz, 1) * 4 + (size_t)zmax * d * 4 +
         ((size_t(1) << split) + (size_t(1) << (L - split))) * 4 + 4096;
}

struct Footprint {
  size_t fixed = 0;      // tables, ground state, G output, largest Green-function part apart from its vectors
  size_t gf_min = 0;     // smallest Green-function vector storage that works
  size_t gf_want = 0;    // storage for the fastest variant (all runs / full reorthogonalization)
  size_t total(size_t gf_budget) const {
    const size_t g = std::max(gf_min, std::min(gf_want, gf_budget));
    return fixed + g + fixed / 20 + kMargin;
  }
};

// Device memory of the single-cluster path for one request.
Footprint single_footprint(const ModelHost& m, const ed_cluster_desc& d, int nz, int cf_cap) {
  Footprint f;
  const int L = m.L, p = m.ns;
  const int npairs = (int)m.pair_a.size();
  const size_t es = d.precision == ED_FP64 ? 8 : 4;
  std::map<int, bool> tabs;
  auto need_table = [&](int N) {
    if (N >= 0 && N <= L && !tabs.count(N)) {
      tabs[N] = true;
      f.fixed += spin_table_bytes(L, N, npairs);
    }
  };
  need_table(d.n_up);
  need_table(d.n_dn);
  const int64_t du = (int64_t)binomial(L, d.n_up), dd = (int64_t)binomial(L, d.n_dn), dim = du * dd;
  // ground state: omega + FP64 polish vector + FP32 retrace sum + 3 Lanczos vectors (FP64 on a restart)
  f.fixed += (size_t)dim * (8 + 8 + 4) + (size_t)3 * du * padded_ld(dd) * 8 + (size_t(1) << 20);
  if (nz <= 0) return f;
  f.fixed += (size_t)2 * nz * p * p * 16;  // G of both spins
  size_t part_fixed = 0, part_min = 0, part_want = 0;
  for (int spin = 0; spin < (d.n_up != d.n_dn ? 2 : 1); ++spin)
    for (int dn : {1, -1}) {
      const int nu_t = d.n_up + (spin == 0 ? dn : 0), nd_t = d.n_dn + (spin == 1 ? dn : 0);
      if (nu_t < 0 || nd_t < 0 || nu_t > L || nd_t > L) continue;
      need_table(spin == 0 ? nu_t : nd_t);
      const int64_t du_t = (int64_t)binomial(L, nu_t), dd_t = (int64_t)binomial(L, nd_t);
      const int64_t vstride = du_t * padded_ld(dd_t), reach = du_t * dd_t;
      size_t fx, mn, wn;
      if (d.gf_method == ED_GF_CF) {
        const int64_t R = p + (int64_t)p * (p - 1) / 2;
        const int64_t M = std::max<int64_t>(64, std::min<int64_t>(cf_cap, 2 * reach + 16));
        fx = (size_t)2 * R * nz * 16 + (size_t)R * (M * 16 + 64 * 16 + 64) + (size_t)nz * 16;
        mn = (size_t)2 * vstride * es;
        wn = (size_t)R * mn;
      } else {
        const int64_t blk = (int64_t)p * vstride;
        const int64_t kmax = std::max<int64_t>(2, std::min<int64_t>((20000 + p - 1) / p, (2 * reach) / p + 4));
        const int64_t nchunk = std::min<int64_t>((vstride + 63) / 64, 152 * 8);
        // stored blocks and the Gram partial sums (against 3 blocks on the ring, every block when full)
        fx = (size_t)2 * nz * p * p * 16 + (size_t)(kmax + 2) * p * p * 8 * 8;
        mn = (size_t)4 * blk * es + (size_t)3 * nchunk * p * p * 8;
        wn = (size_t)(kmax + 3) * blk * es + (size_t)(kmax + 2) * nchunk * p * p * 8;
      }
      part_fixed = std::max(part_fixed, fx);
      part_min = std::max(part_min, mn);
      part_want = std::max(part_want, wn);
    }
  f.fixed += part_fixed;
  f.gf_min = part_min;
  f.gf_want = std::max(part_min, part_want);
  return f;
}

// Green-function vector storage to reserve within `share` bytes: continued fractions use any
// amount between one run's vectors and all runs' (they run in chunks); band Lanczos keeps every
// block only when all of them fit (full reorthogonalization), else a ring of blocks, so it gets
// either the full amount or the ring's.
size_t gf_reservation(const Footprint& f, int gf_method, size_t share) {
  if (gf_method == ED_GF_BAND) return f.gf_want <= share ? f.gf_want : f.gf_min;
  return std::max(f.gf_min, std::min(f.gf_want, share));
}

int64_t largest_sector(const ed_cluster_desc& d, bool gf) {
  const int L = d.n_sites + d.n_bath;
  auto dimN = [&](int N) -> int64_t { return (N < 0 || N > L) ? 0 : (int64_t)binomial(L, N); };
  int64_t mx = dimN(d.n_up) * dimN(d.n_dn);
  if (gf)
    for (int dn : {1, -1}) {
      mx = std::max(mx, dimN(d.n_up + dn) * dimN(d.n_dn));
      mx = std::max(mx, dimN(d.n_up) * dimN(d.n_dn + dn));
    }
  return mx;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

enum State { QUEUED, RUNNING, DONE };

struct Request {
  uint64_t id = 0;
  ed_cluster_desc desc{};
  std::vector<double> t, U, eps, theta, omega;
  int n_freq = 0, axis = ED_AXIS_REAL, cf_cap = kDefaultCfCap;
  double eta = 0.0;
  double* G_out = nullptr;
  int ns = 0, L = 0;
  bool batched = false;
  size_t need = 0, gf_budget = 0;   // reservation on the single path / alone on the batched path
  State state = QUEUED;
  bool cancel = false;
  int inject = 0;
  int bypassed = 0;
  ed_result res{};
  std::string err;
  Clock::time_point t_submit, t_start, t_done;

  ed_cluster_desc bound_desc() const {
    ed_cluster_desc d = desc;
    d.t = const_cast<double*>(t.data());
    d.U = const_cast<double*>(U.data());
    d.eps = eps.empty() ? nullptr : const_cast<double*>(eps.data());
    d.theta = theta.empty() ? nullptr : const_cast<double*>(theta.data());
    return d;
  }
  bool batch_compatible(const Request& o) const {
    return batched && o.batched && desc.precision == o.desc.precision && n_freq == o.n_freq && axis == o.axis &&
           eta == o.eta && cf_cap == o.cf_cap && omega == o.omega;
  }
};

}  // namespace
}  // namespace ed

using namespace ed;

struct ed_server {
  int device = 0, sms = 152;
  size_t budget = 0, reserved = 0, peak_reserved = 0;
  int64_t batch_max_dim = 100000;
  int batch_max_requests = 64;
  double gf_fraction = 0.5;
  bool paused = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<std::thread> lanes;
  std::vector<cudaStream_t> streams;
  bool stop = false;
  uint64_t next_id = 1;
  int running = 0, max_running = 0;
  int64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, batched_solves = 0;

  void finish_locked(Request* r, int status, const std::string& msg) {
    r->state = DONE;
    r->t_done = Clock::now();
    r->res.status = status;
    r->err = msg;
    r->res.queued_ms = r->t_start.time_since_epoch().count() ? ms_between(r->t_submit, r->t_start) : 0.0;
    r->res.run_ms = r->t_start.time_since_epoch().count() ? ms_between(r->t_start, r->t_done) : 0.0;
    r->res.latency_ms = ms_between(r->t_submit, r->t_done);
    if (status == ED_ERR_CANCELLED)
      ++cancelled;
    else if (status < 0)
      ++failed;
    else
      ++completed;
  }

  size_t group_bytes(const std::vector<Request*>& g) const {
    std::vector<ed_cluster_desc> d;
    size_t gout = 0;
    for (Request* r : g) {
      d.push_back(r->bound_desc());
      gout += (size_t)2 * r->n_freq * r->ns * r->ns * 16;
    }
    return batch_device_bytes(d.data(), (int)d.size(), g[0]->desc.precision, g[0]->n_freq, g[0]->cf_cap, sms) + gout +
           kMargin;
  }

  // Picks the next job for a free lane (under mu); reserves its memory.
  bool pick_locked(std::vector<Request*>& job, size_t& bytes) {
    job.clear();
    // requests failed on purpose by the test hook end here, before any device work
    for (auto it = queue.begin(); it != queue.end();) {
      Request* r = reqs[*it].get();
      if (r->inject < 0) {
        r->t_start = Clock::now();
        finish_locked(r, r->inject, "injected failure (host)");
        it = queue.erase(it);
        cv_done.notify_all();
      } else {
        ++it;
      }
    }
    if (queue.empty() || paused) return false;
    const size_t avail = budget - reserved;
    Request* head = reqs[queue.front()].get();
    size_t pos = 0;
    if (head->need > avail) {
      if (head->bypassed >= kMaxBypass) return false;
      for (pos = 1; pos < queue.size(); ++pos)
        if (reqs[queue[pos]]->need <= avail) break;
      if (pos == queue.size()) return false;
      ++head->bypassed;
    }
    Request* r = reqs[queue[pos]].get();
    job.push_back(r);
    bytes = r->need;
    std::vector<size_t> taken{pos};
    if (r->batched) {
      for (size_t q = pos + 1; q < queue.size() && (int)job.size() < batch_max_requests; ++q) {
        Request* o = reqs[queue[q]].get();
        if (!r->batch_compatible(*o)) continue;
        job.push_back(o);
        const size_t b = group_bytes(job);
        if (b > avail) {
          job.pop_back();
          continue;
        }
        bytes = b;
        taken.push_back(q);
      }
      if (job.size() > 1) bytes = group_bytes(job);
    }
    std::sort(taken.rbegin(), taken.rend());
    for (size_t q : taken) queue.erase(queue.begin() + (ptrdiff_t)q);
    reserved += bytes;
    peak_reserved = std::max(peak_reserved, reserved);
    const auto now = Clock::now();
    for (Request* j : job) {
      j->state = RUNNING;
      j->t_start = now;
      j->res.batch_size = (int)job.size();
      j->res.path = j->batched ? 1 : 0;
      j->res.device_bytes = bytes / job.size();
    }
    running += (int)job.size();
    max_running = std::max(max_running, running);
    return true;
  }

  void run_single(Request* r, cudaStream_t st) {
    ed_cluster_desc d = r->bound_desc();
    auto c = cluster_create_on(&d, st);
    c->gf_mem_budget = std::max<size_t>(r->gf_budget, 1);
    c->cf_max_steps = r->cf_cap;
    GroundResult g = run_ground_state(*c, c->desc.precision, c->desc.tol, c->desc.max_iter, c->desc.seed);
    c->gs = g;
    c->have_gs = true;
    r->res.E0 = g.E0;
    r->res.residual = g.residual;
    r->res.iters = g.iters;
    int status = !g.converged ? ED_WARN_NOT_CONVERGED : (g.degenerate ? ED_WARN_DEGENERATE : ED_OK);
    if (r->n_freq > 0) {
      if (cancel_requested(r)) throw Error(ED_ERR_CANCELLED, "cancelled");
      std::vector<double2> z(r->n_freq);
      for (int k = 0; k < r->n_freq; ++k)
        z[k] = r->axis == ED_AXIS_REAL ? make_double2(r->omega[k], r->eta) : make_double2(0.0, r->omega[k]);
      const size_t per = (size_t)r->n_freq * r->ns * r->ns;
      DevBuf<double2> G(2 * per);
      int64_t steps = 0;
      for (int spin = 0; spin < 2; ++spin) {
        if (spin == 1 && d.n_up == d.n_dn) {
          ED_CUDA(cudaMemcpyAsync(G.p + per, G.p, per * sizeof(double2), cudaMemcpyDeviceToDevice, st));
          break;
        }
        if (spin == 1 && cancel_requested(r)) throw Error(ED_ERR_CANCELLED, "cancelled");
        if (c->desc.gf_method == ED_GF_CF) {
          run_green_cf(*c, spin, z.data(), r->n_freq, G.p + spin * per);
        } else if (!run_green_band(*c, spin, z.data(), r->n_freq, G.p + spin * per) && status == ED_OK) {
          status = ED_WARN_NOT_CONVERGED;
        }
        steps += c->gf_total_steps;
      }
      r->res.gf_steps = steps;
      ED_CUDA(cudaMemcpyAsync(r->G_out, G.p, 2 * per * sizeof(double2), cudaMemcpyDeviceToHost, st));
    }
    ED_CUDA(cudaStreamSynchronize(st));
    r->res.status = status;
  }

  void run_batched(const std::vector<Request*>& job, cudaStream_t st) {
    const int n = (int)job.size();
    const Request* r0 = job[0];
    std::vector<ed_cluster_desc> d(n);
    for (int k = 0; k < n; ++k) d[k] = job[k]->bound_desc();
    std::vector<double2> z(r0->n_freq);
    for (int k = 0; k < r0->n_freq; ++k)
      z[k] = r0->axis == ED_AXIS_REAL ? make_double2(r0->omega[k], r0->eta) : make_double2(0.0, r0->omega[k]);
    std::vector<size_t> off(n + 1, 0);
    for (int k = 0; k < n; ++k) off[k + 1] = off[k] + (size_t)2 * r0->n_freq * job[k]->ns * job[k]->ns;
    DevBuf<double2> G(std::max<size_t>(off[n], 1));
    std::vector<double> E0(n), res(n);
    std::vector<int> status(n), iters(n);
    std::vector<int64_t> steps(n);
    batch_solve(d.data(), n, r0->desc.precision, z.data(), r0->n_freq, r0->n_freq > 0, r0->cf_cap, E0.data(),
                res.data(), status.data(), iters.data(), steps.data(), G.p, st, kBatchThreads, kBatchMode);
    for (int k = 0; k < n; ++k)
      if (r0->n_freq > 0)
        ED_CUDA(cudaMemcpyAsync(job[k]->G_out, G.p + off[k], (off[k + 1] - off[k]) * sizeof(double2),
                                cudaMemcpyDeviceToHost, st));
    ED_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < n; ++k) {
      job[k]->res.E0 = E0[k];
      job[k]->res.residual = res[k];
      job[k]->res.iters = iters[k];
      job[k]->res.gf_steps = r0->n_freq > 0 ? steps[k] : 0;
      job[k]->res.status = status[k];
    }
  }

  bool cancel_requested(Request* r) {
    std::lock_guard<std::mutex> lk(mu);
    return r->cancel || stop;
  }

  void lane_main(int lane) {
    cudaSetDevice(device);
    cudaStream_t st = streams[lane];
    AllocStreamScope as(st);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      std::vector<Request*> job;
      size_t bytes = 0;
      cv_work.wait(lk, [&] { return stop || pick_locked(job, bytes); });
      if (job.empty()) break;  // stop
      lk.unlock();
      int code = 0;
      std::string msg;
      try {
        if (job[0]->batched)
          run_batched(job, st);
        else
          run_single(job[0], st);
        // every buffer of the job was freed on st; wait for those frees before returning the memory
        ED_CUDA(cudaStreamSynchronize(st));
      } catch (const Error& e) {
        code = e.code;
        msg = e.what();
      } catch (const std::exception& e) {
        code = ED_ERR_INVALID;
        msg = e.what();
      }
      if (code != 0) {
        cudaStreamSynchronize(st);
        cudaGetLastError();
      }
      lk.lock();
      reserved -= bytes;
      running -= (int)job.size();
      if (job[0]->batched && code == 0) ++batched_solves;
      for (Request* r : job) {
        const bool cancelled_now = r->cancel && code == ED_ERR_CANCELLED;
        if (code != 0)
          finish_locked(r, cancelled_now ? ED_ERR_CANCELLED : code, msg);
        else
          finish_locked(r, r->res.status, "");
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

namespace {

template <typename F>
ed_status srv_guarded(F&& f) {
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

void check_opts(const ed_request_opts* o) {
  if (!o) return;
  if (o->n_freq < 0) throw Error(ED_ERR_INVALID, "n_freq < 0");
  if (o->n_freq > 0 && (!o->omega || !o->G_out)) throw Error(ED_ERR_INVALID, "omega and G_out are needed when n_freq > 0");
  if (o->axis != ED_AXIS_REAL && o->axis != ED_AXIS_MATSUBARA) throw Error(ED_ERR_INVALID, "bad axis");
  if (!std::isfinite(o->eta)) throw Error(ED_ERR_INVALID, "eta is not finite");
  for (int k = 0; k < o->n_freq; ++k)
    if (!std::isfinite(o->omega[k])) throw Error(ED_ERR_INVALID, "omega has a non-finite entry");
}

}  // namespace

extern "C" {

ed_status ed_request_bytes(const ed_cluster_desc* desc, const ed_request_opts* opts, size_t gf_budget_bytes,
                           size_t* bytes) {
  return srv_guarded([&]() -> ed_status {
    if (!desc || !bytes) throw Error(ED_ERR_INVALID, "desc and bytes must not be NULL");
    check_opts(opts);
    ModelHost m;
    HopParams hp;
    build_model(desc, m, hp);
    const int nz = opts ? opts->n_freq : 0;
    const int cap = opts && opts->cf_max_levels > 0 ? opts->cf_max_levels : kDefaultCfCap;
    Footprint f = single_footprint(m, *desc, nz, cap);
    *bytes = f.total(gf_reservation(f, desc->gf_method, gf_budget_bytes > 0 ? gf_budget_bytes : SIZE_MAX / 4));
    return ED_OK;
  });
}

ed_status ed_server_create(size_t mem_budget_bytes, int max_slots, ed_server** out) {
  return srv_guarded([&]() -> ed_status {
    if (!out) throw Error(ED_ERR_INVALID, "out must not be NULL");
    *out = nullptr;
    if (mem_budget_bytes == 0) throw Error(ED_ERR_INVALID, "mem_budget_bytes must be positive");
    if (max_slots < 1 || max_slots > 64) throw Error(ED_ERR_INVALID, "max_slots must be in [1, 64]");
    auto S = std::make_unique<ed_server>();
    ED_CUDA(cudaGetDevice(&S->device));
    ED_CUDA(cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device));
    S->budget = mem_budget_bytes;
    // keep freed stream-ordered memory cached in the device's pool instead of returning it at
    // every synchronization (the lanes allocate and free a request's buffers each time)
    cudaMemPool_t pool;
    ED_CUDA(cudaDeviceGetDefaultMemPool(&pool, S->device));
    uint64_t thr = mem_budget_bytes;
    ED_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    for (int k = 0; k < max_slots; ++k) {
      cudaStream_t s;
      ED_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      S->streams.push_back(s);
    }
    ed_server* raw = S.get();
    for (int k = 0; k < max_slots; ++k) S->lanes.emplace_back([raw, k] { raw->lane_main(k); });
    *out = S.release();
    return ED_OK;
  });
}

void ed_server_destroy(ed_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    for (uint64_t id : srv->queue) srv->finish_locked(srv->reqs[id].get(), ED_ERR_CANCELLED, "server destroyed");
    srv->queue.clear();
    for (auto& kv : srv->reqs)
      if (kv.second->state == RUNNING) kv.second->cancel = true;
  }
  srv->cv_work.notify_all();
  srv->cv_done.notify_all();
  for (auto& t : srv->lanes)
    if (t.joinable()) t.join();
  for (cudaStream_t s : srv->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  delete srv;
}

ed_status ed_server_set_option(ed_server* srv, int option, double value) {
  return srv_guarded([&]() -> ed_status {
    if (!srv) throw Error(ED_ERR_INVALID, "server is NULL");
    if (!std::isfinite(value)) throw Error(ED_ERR_INVALID, "option value is not finite");
    std::lock_guard<std::mutex> lk(srv->mu);
    switch (option) {
      case ED_SRV_BATCH_MAX_DIM:
        if (value < 0) throw Error(ED_ERR_INVALID, "ED_SRV_BATCH_MAX_DIM must be >= 0");
        srv->batch_max_dim = (int64_t)value;
        break;
      case ED_SRV_BATCH_MAX_REQUESTS:
        if (value < 1 || value > 4096) throw Error(ED_ERR_INVALID, "ED_SRV_BATCH_MAX_REQUESTS must be in [1, 4096]");
        srv->batch_max_requests = (int)value;
        break;
      case ED_SRV_GF_BUDGET_FRACTION:
        if (!(value > 0.0 && value <= 1.0)) throw Error(ED_ERR_INVALID, "ED_SRV_GF_BUDGET_FRACTION must be in (0, 1]");
        srv->gf_fraction = value;
        break;
      case ED_SRV_PAUSE:
        if (value != 0.0 && value != 1.0) throw Error(ED_ERR_INVALID, "ED_SRV_PAUSE must be 0 or 1");
        srv->paused = value != 0.0;
        srv->cv_work.notify_all();
        break;
      default:
        throw Error(ED_ERR_INVALID, "unknown server option");
    }
    return ED_OK;
  });
}

ed_status ed_submit(ed_server* srv, const ed_cluster_desc* desc, const ed_request_opts* opts, uint64_t* req_id) {
  return srv_guarded([&]() -> ed_status {
    if (!srv || !desc || !req_id) throw Error(ED_ERR_INVALID, "server, desc and req_id must not be NULL");
    check_opts(opts);
    ModelHost m;
    HopParams hp;
    build_model(desc, m, hp);  // validates the description
    auto r = std::make_unique<Request>();
    r->desc = *desc;
    if (!(r->desc.tol > 0.0)) r->desc.tol = 1e-12;
    if (r->desc.max_iter <= 0) r->desc.max_iter = 600;
    const int ns = desc->n_sites, nb = desc->n_bath;
    r->ns = ns;
    r->L = ns + nb;
    r->t.assign(desc->t, desc->t + (size_t)ns * ns);
    r->U.assign(desc->U, desc->U + ns);
    if (nb) {
      r->eps.assign(desc->eps, desc->eps + nb);
      r->theta.assign(desc->theta, desc->theta + (size_t)ns * nb);
    }
    if (opts) {
      r->n_freq = opts->n_freq;
      r->omega.assign(opts->omega, opts->omega + opts->n_freq);
      r->eta = opts->eta;
      r->axis = opts->axis;
      r->cf_cap = opts->cf_max_levels > 0 ? opts->cf_max_levels : kDefaultCfCap;
      r->G_out = opts->G_out;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) throw Error(ED_ERR_STATE, "server is shutting down");
    const bool gf = r->n_freq > 0;
    r->batched = srv->batch_max_dim > 0 && r->L <= 20 && (!gf || desc->gf_method == ED_GF_CF) &&
                 largest_sector(*desc, gf) <= srv->batch_max_dim;
    if (r->batched) {
      std::vector<Request*> one{r.get()};
      r->need = srv->group_bytes(one);
    } else {
      Footprint f = single_footprint(m, *desc, r->n_freq, r->cf_cap);
      const size_t share = (size_t)(srv->gf_fraction * (double)srv->budget);
      r->gf_budget = gf_reservation(f, desc->gf_method, share);
      r->need = f.total(r->gf_budget);
    }
    if (r->need > srv->budget)
      throw Error(ED_ERR_TOO_LARGE, "request needs " + std::to_string(r->need) + " device bytes, the server's budget is " +
                                        std::to_string(srv->budget));
    r->id = srv->next_id++;
    r->t_submit = Clock::now();
    *req_id = r->id;
    srv->queue.push_back(r->id);
    srv->reqs[r->id] = std::move(r);
    ++srv->submitted;
    srv->cv_work.notify_one();
    return ED_OK;
  });
}

static ed_status collect_locked(ed_server* srv, uint64_t id, ed_result* out) {
  auto it = srv->reqs.find(id);
  if (it == srv->reqs.end()) throw Error(ED_ERR_NOT_FOUND, "unknown or already collected request id");
  Request* r = it->second.get();
  if (r->state != DONE) return ED_PENDING;
  if (out) *out = r->res;
  if (r->res.status < 0) set_last_error(r->err);
  srv->reqs.erase(it);
  return ED_OK;
}

ed_status ed_poll(ed_server* srv, uint64_t req_id, ed_result* out) {
  return srv_guarded([&]() -> ed_status {
    if (!srv) throw Error(ED_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    return collect_locked(srv, req_id, out);
  });
}

ed_status ed_wait(ed_server* srv, uint64_t req_id, double timeout_s, ed_result* out) {
  return srv_guarded([&]() -> ed_status {
    if (!srv) throw Error(ED_ERR_INVALID, "server is NULL");
    if (!(timeout_s >= 0.0) || !std::isfinite(timeout_s)) throw Error(ED_ERR_INVALID, "timeout_s must be finite and >= 0");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) throw Error(ED_ERR_NOT_FOUND, "unknown or already collected request id");
    Request* r = it->second.get();
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    if (!srv->cv_done.wait_until(lk, deadline, [&] { return r->state == DONE; }))
      throw Error(ED_ERR_TIMEOUT, "request still pending after the timeout");
    return collect_locked(srv, req_id, out);
  });
}

ed_status ed_cancel(ed_server* srv, uint64_t req_id) {
  return srv_guarded([&]() -> ed_status {
    if (!srv) throw Error(ED_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end()) throw Error(ED_ERR_NOT_FOUND, "unknown or already collected request id");
    Request* r = it->second.get();
    if (r->state == QUEUED) {
      srv->queue.erase(std::find(srv->queue.begin(), srv->queue.end(), req_id));
      srv->finish_locked(r, ED_ERR_CANCELLED, "cancelled");
      srv->cv_done.notify_all();
      srv->cv_work.notify_all();
    } else if (r->state == RUNNING) {
      r->cancel = true;
    }
    return ED_OK;
  });
}

ed_status ed_server_inject_failure(ed_server* srv, uint64_t req_id, int status) {
  return srv_guarded([&]() -> ed_status {
    if (!srv) throw Error(ED_ERR_INVALID, "server is NULL");
    if (status >= 0) throw Error(ED_ERR_INVALID, "status must be an error code (< 0)");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(req_id);
    if (it == srv->reqs.end() || it->second->state != QUEUED) throw Error(ED_ERR_NOT_FOUND, "request is not queued");
    it->second->inject = status;
    srv->cv_work.notify_all();
    return ED_OK;
  });
}

ed_status ed_server_stats_get(ed_server* srv, ed_server_stats* out) {
  return srv_guarded([&]() -> ed_status {
    if (!srv || !out) throw Error(ED_ERR_INVALID, "server and out must not be NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    out->submitted = srv->submitted;
    out->completed = srv->completed;
    out->failed = srv->failed;
    out->cancelled = srv->cancelled;
    out->queued = (int)srv->queue.size();
    out->running = srv->running;
    out->max_running = srv->max_running;
    out->reserved_bytes = srv->reserved;
    out->peak_reserved_bytes = srv->peak_reserved;
    out->batched_solves = srv->batched_solves;
    return ED_OK;
  });
}

}  // extern "C"
