// ed_hpsi_dots_static: the product y = H x and the reductions <x,y>, <y,y>, <x,x> for callers
// that must not allocate device memory.  An application that hands libed a memory budget it
// manages itself (a caching allocator or a pool reserved at start-up), or that runs its solver
// inside a region where allocating would stall other streams, cannot let the library call
// cudaMalloc.  Here the only scratch, the per-block partial sums of the reductions and the
// ticket that picks the block finishing them, lives in fixed arrays inside libed.
#include <algorithm>
#include <mutex>

#include "ed_common.cuh"
#include "hpsi_element.cuh"

namespace ed {

constexpr int kStaticThreads = 256;
constexpr int kStaticPerThread = 4;
constexpr int kStaticMaxBlocks = 4096;  // 4096 * 3 doubles = 96 KiB of scratch
constexpr int64_t kStaticMaxDim = (int64_t)kStaticMaxBlocks * kStaticThreads * kStaticPerThread;  // 4,194,304

// Shared by every call on a device, and held by every GPU that loads the library until exit.
static __device__ __align__(256) double g_static_partial[kStaticMaxBlocks * 3];
static __device__ __align__(256) unsigned int g_static_ticket[64];

// One thread per element (kStaticPerThread elements per thread, one grid pass); block partial
// sums go to `partial`, the last block (ticket) adds them in block order into out3.
template <typename T>
__global__ void __launch_bounds__(kStaticThreads) k_hpsi_dots_static(SectorView sv, HopParams hp, const T* __restrict__ X,
                                                                     T* __restrict__ Y, double* __restrict__ partial,
                                                                     unsigned int* __restrict__ ticket,
                                                                     double* __restrict__ out3) {
  __shared__ T sval[kMaxVals];
  __shared__ T sU[kMaxOrb];
  __shared__ bool s_last;
  // The host rejects sectors that need more blocks than the fixed scratch has partial slots for;
  // a grid beyond it would write past the array, so such a launch writes nothing at all.
  if (gridDim.x > kStaticMaxBlocks) return;
  load_params<T>(hp, sval, sU);
  const int64_t dim = sv.d_up * sv.d_dn;
  double sxy = 0.0, syy = 0.0, sxx = 0.0;
  for (int k = 0; k < kStaticPerThread; ++k) {
    const int64_t idx = ((int64_t)blockIdx.x * kStaticPerThread + k) * kStaticThreads + threadIdx.x;
    if (idx >= dim) break;
    const int64_t u = idx / sv.d_dn, d = idx - u * sv.d_dn;
    const T acc = hpsi_element<T>(sv, sval, sU, hp.umask, X, u, d);
    Y[u * sv.ld + d] = acc;
    const double xv = (double)X[u * sv.ld + d], yv = (double)acc;
    sxy += xv * yv;
    syy += yv * yv;
    sxx += xv * xv;
  }
  block_sum3<kStaticThreads>(sxy, syy, sxx);
  if (threadIdx.x == 0) {
    partial[blockIdx.x * 3 + 0] = sxy;
    partial[blockIdx.x * 3 + 1] = syy;
    partial[blockIdx.x * 3 + 2] = sxx;
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    a += __ldcg(partial + i * 3 + 0);
    b += __ldcg(partial + i * 3 + 1);
    c += __ldcg(partial + i * 3 + 2);
  }
  block_sum3<kStaticThreads>(a, b, c);
  if (threadIdx.x == 0) {
    out3[0] = a;
    out3[1] = b;
    out3[2] = c;
    *ticket = 0u;
  }
}

namespace {
struct StaticScratch {
  double* partial = nullptr;
  unsigned int* ticket = nullptr;
};
std::mutex g_static_mu;
StaticScratch g_static_dev[64];  // per device ordinal, filled by the first call on that device
}  // namespace

// Device addresses of the fixed scratch on the current device (looked up once per device).
static StaticScratch static_scratch() {
  int dev = 0;
  ED_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error(ED_ERR_INVALID, "device ordinal above 63");
  std::lock_guard<std::mutex> lk(g_static_mu);
  StaticScratch& s = g_static_dev[dev];
  if (!s.partial) {
    void* p = nullptr;
    void* t = nullptr;
    ED_CUDA(cudaGetSymbolAddress(&p, g_static_partial));
    ED_CUDA(cudaGetSymbolAddress(&t, g_static_ticket));
    s.partial = (double*)p;
    s.ticket = (unsigned int*)t;
  }
  return s;
}

}  // namespace ed

using namespace ed;

extern "C" ed_status ed_hpsi_dots_static(ed_cluster* c, int dtype, const void* x, void* y, int64_t ld, double* out3,
                                         void* stream) {
  try {
    if (!c || !x || !y || !out3) throw Error(ED_ERR_INVALID, "cluster, x, y and out3 must not be NULL");
    if (dtype != ED_FP64 && dtype != ED_FP32) throw Error(ED_ERR_INVALID, "dtype must be ED_FP64 or ED_FP32");
    // the cluster's own sector: its tables were built by ed_cluster_create, nothing is allocated
    auto iu = c->spins.find(c->desc.n_up), idn = c->spins.find(c->desc.n_dn);
    if (iu == c->spins.end() || idn == c->spins.end()) throw Error(ED_ERR_STATE, "cluster tables missing");
    const int64_t du = iu->second->dim, dd = idn->second->dim;
    if (du * dd > kStaticMaxDim)
      throw Error(ED_ERR_TOO_LARGE, "sector dimension " + std::to_string(du * dd) +
                                        " exceeds the 4,194,304 elements covered by the fixed scratch of ed_hpsi_dots_static");
    if (ld > 0 && ld < dd) throw Error(ED_ERR_INVALID, "ld must be >= d_dn (or <= 0 for d_dn)");
    // the tables live on the device the cluster was created on; x, y and the scratch are on the
    // current one, so the two must be the same device
    int dev = -1;
    ED_CUDA(cudaGetDevice(&dev));
    if (dev != c->device)
      throw Error(ED_ERR_INVALID, "the current device (" + std::to_string(dev) + ") is not the cluster's device (" +
                                      std::to_string(c->device) + ")");
    SectorView sv = c->view(c->desc.n_up, c->desc.n_dn, ld);
    StaticScratch s = static_scratch();
    cudaStream_t st = (cudaStream_t)stream;
    ED_CUDA(cudaMemsetAsync(s.ticket, 0, sizeof(unsigned int), st));  // the ticket must start at zero
    const int64_t per = (int64_t)kStaticThreads * kStaticPerThread;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, (du * dd + per - 1) / per);
    note_launch();
    if (dtype == ED_FP64)
      k_hpsi_dots_static<double><<<blocks, kStaticThreads, 0, st>>>(sv, c->hp, (const double*)x, (double*)y, s.partial,
                                                                     s.ticket, out3);
    else
      k_hpsi_dots_static<float><<<blocks, kStaticThreads, 0, st>>>(sv, c->hp, (const float*)x, (float*)y, s.partial,
                                                                    s.ticket, out3);
    ED_CHECK_LAUNCH();
    return ED_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return ED_ERR_INVALID;
  }
}
