// Launch counter and per-kernel-family timing (CUDA events on the launching stream).
#include <atomic>
#include <mutex>
#include <vector>

#include "ed_common.cuh"

namespace ed {

namespace {
std::atomic<long long> g_launches{0};
std::atomic<bool> g_enabled{false};
std::mutex g_mu;
struct Pending {
  cudaEvent_t e0, e1;
  int kid;
  double bytes;
};
std::vector<Pending> g_pending;
struct Totals {
  long long launches = 0;
  double ms = 0.0, bytes = 0.0;
};
Totals g_tot[K_COUNT];
const char* kNames[K_COUNT] = {"tables", "hpsi", "lanczos_step", "lanczos_next", "tridiag", "vector",
                               "apply_cop", "gf_eval", "band", "batch", "lattice"};

void drain_locked() {
  for (auto& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      g_tot[p.kid].ms += ms;
    }
    g_tot[p.kid].launches += 1;
    g_tot[p.kid].bytes += p.bytes;
    cudaEventDestroy(p.e0);
    cudaEventDestroy(p.e1);
  }
  g_pending.clear();
  cudaGetLastError();
}
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

const char* kernel_name(int kid) { return (kid >= 0 && kid < K_COUNT) ? kNames[kid] : "?"; }

ProfScope::ProfScope(int kid_, cudaStream_t s_, double bytes_) : kid(kid_), s(s_), bytes(bytes_) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (g_enabled.load(std::memory_order_relaxed)) {
    if (cudaEventCreate(&e0) == cudaSuccess) {
      cudaEventRecord(e0, s);
    } else {
      e0 = nullptr;
      cudaGetLastError();
    }
  }
}

ProfScope::~ProfScope() {
  if (!e0) return;
  cudaEvent_t e1;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaGetLastError();
    return;
  }
  cudaEventRecord(e1, s);
  std::lock_guard<std::mutex> lk(g_mu);
  g_pending.push_back(Pending{e0, e1, kid, bytes});
  if (g_pending.size() > 4096) drain_locked();
}

}  // namespace ed

using namespace ed;

extern "C" {

ed_status ed_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  for (auto& t : g_tot) t = Totals();
  g_enabled.store(on != 0);
  return ED_OK;
}

ed_status ed_profile_read(int kernel, int64_t* launches, double* total_ms, double* alg_bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  if (kernel < 0 || kernel >= K_COUNT) {
    set_last_error("unknown kernel family");
    return ED_ERR_INVALID;
  }
  if (launches) *launches = g_tot[kernel].launches;
  if (total_ms) *total_ms = g_tot[kernel].ms;
  if (alg_bytes) *alg_bytes = g_tot[kernel].bytes;
  return ED_OK;
}

const char* ed_profile_kernel_name(int kernel) { return kernel_name(kernel); }

int64_t ed_launch_count(void) { return (int64_t)g_launches.load(); }

}  // extern "C"
