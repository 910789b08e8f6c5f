// Sector basis and hopping tables of one spin (Sec. 4.1).
//
// K1: the basis of N particles on L orbitals is enumerated by unranking the combinatorial
//     number system: the state of rank r has set bits p_N > ... > p_1 with
//     r = sum_k C(p_k, k), which lists the bit strings in ascending integer order.
// Rank tables: rank(b) = rank_lo[b & lomask] + rank_hi[b >> split], because the sum over the
//     set bits splits into the bits below `split` (whose order index k depends on the low half
//     only) and those above (whose k starts at N - popcount(hi) + 1).
// K2: pull-form hopping table: for the state s of row r and every ordered pair (a, b) with
//     h_ab != 0, a occupied and b empty in s, the source state c = s - 2^a + 2^b contributes
//     K[r, rank(c)] = (-1)^{M_ab} h_ab, M_ab = occupied orbitals strictly between a and b.
#include <algorithm>
#include <cstring>

#include "ed_common.cuh"

namespace ed {

struct Binom {
  uint32_t c[kMaxOrb + 1][kMaxOrb + 1];
};

static Binom make_binom() {
  Binom b;
  std::memset(&b, 0, sizeof(b));
  for (int n = 0; n <= kMaxOrb; ++n) {
    b.c[n][0] = 1;
    for (int k = 1; k <= n; ++k) b.c[n][k] = b.c[n - 1][k - 1] + (k <= n - 1 ? b.c[n - 1][k] : 0);
  }
  return b;
}

uint64_t binomial(int n, int k) {
  if (k < 0 || k > n) return 0;
  uint64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
  return r;
}

__global__ void k_unrank(int L, int N, int64_t dim, Binom bn, uint32_t* __restrict__ out) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= dim) return;
  uint32_t rem = (uint32_t)r, b = 0;
  int p = L - 1;
  for (int k = N; k >= 1; --k) {
    while (bn.c[p][k] > rem) --p;  // C(p, k) = 0 for p < k, so p stops at k - 1 at the latest
    b |= 1u << p;
    rem -= bn.c[p][k];
    --p;
  }
  out[r] = b;
}

__global__ void k_rank_lo(int split, Binom bn, int32_t* __restrict__ out) {
  int64_t lo = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (lo >= (int64_t(1) << split)) return;
  int32_t r = 0;
  int j = 0;
  for (int p = 0; p < split; ++p)
    if ((lo >> p) & 1) r += (int32_t)bn.c[p][++j];
  out[lo] = r;
}

__global__ void k_rank_hi(int L, int N, int split, Binom bn, int32_t* __restrict__ out) {
  int64_t hi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int nh = L - split;
  if (hi >= (int64_t(1) << nh)) return;
  int m = N - __popc((uint32_t)hi);
  if (m < 0 || m > split) {
    out[hi] = -1;
    return;
  }
  int32_t r = 0;
  int j = 0;
  for (int q = 0; q < nh; ++q)
    if ((hi >> q) & 1) r += (int32_t)bn.c[q + split][m + (++j)];
  out[hi] = r;
}

struct PairDev {
  uint32_t a, b, vidx, between;
};

__global__ void k_hop_count(int64_t dim, const uint32_t* __restrict__ basis, const PairDev* __restrict__ pairs,
                            int npairs, int32_t* __restrict__ cnt) {
  __shared__ PairDev sp[kMaxPairs];
  for (int i = threadIdx.x; i < npairs; i += blockDim.x) sp[i] = pairs[i];
  __syncthreads();
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= dim) return;
  uint32_t s = basis[r];
  int c = 0;
  for (int k = 0; k < npairs; ++k) c += ((s >> sp[k].a) & 1u) & (((s >> sp[k].b) & 1u) ^ 1u);
  cnt[r] = c;
}

__global__ void k_hop_fill(int64_t dim, const uint32_t* __restrict__ basis, RankView rv,
                           const PairDev* __restrict__ pairs, int npairs, const int32_t* __restrict__ ptr,
                           uint32_t* __restrict__ ent) {
  __shared__ PairDev sp[kMaxPairs];
  for (int i = threadIdx.x; i < npairs; i += blockDim.x) sp[i] = pairs[i];
  __syncthreads();
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= dim) return;
  uint32_t s = basis[r];
  int32_t o = ptr[r];
  for (int k = 0; k < npairs; ++k) {
    PairDev p = sp[k];
    if (((s >> p.a) & 1u) && !((s >> p.b) & 1u)) {
      uint32_t c = s ^ (1u << p.a) ^ (1u << p.b);
      uint32_t neg = __popc(s & p.between) & 1u;
      ent[o++] = ((uint32_t)rank_of(rv, c) << 8) | (neg << 7) | p.vidx;
    }
  }
}

__global__ void k_max_int(const int32_t* __restrict__ v, int64_t n, int* __restrict__ out) {
  int m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, v[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Slot-major copy of the CSR table for the row kernel: ell[k * dim + r] = k-th entry of row r
// in row_ell_pack form (0 past its end).
__global__ void k_ell_fill(int64_t dim, const int32_t* __restrict__ ptr, const uint32_t* __restrict__ ent, int zmax,
                           uint32_t* __restrict__ ell) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= dim) return;
  const int32_t p0 = ptr[r], n = ptr[r + 1] - p0;
  for (int k = 0; k < zmax; ++k) ell[(int64_t)k * dim + r] = k < n ? row_ell_pack(ent[p0 + k]) : 0u;
}

// Exclusive scan of cnt[0..n) into ptr[0..n] by one block (one-time table construction).
__global__ void k_scan_one_block(const int32_t* __restrict__ cnt, int64_t n, int32_t* __restrict__ ptr) {
  __shared__ int64_t sums[1024];
  int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  int64_t lo = threadIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += cnt[i];
  sums[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      int64_t v = sums[i];
      sums[i] = acc;
      acc += v;
    }
    ptr[n] = (int32_t)acc;
  }
  __syncthreads();
  int64_t acc = sums[threadIdx.x];
  for (int64_t i = lo; i < hi; ++i) {
    ptr[i] = (int32_t)acc;
    acc += cnt[i];
  }
}

struct Diag32 {
  double h[kMaxOrb];
};

__global__ void k_ediag(int64_t dim, int L, const uint32_t* __restrict__ basis, Diag32 hd, double* __restrict__ e,
                        float* __restrict__ e32) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= dim) return;
  uint32_t s = basis[r];
  double acc = 0.0;
  for (int a = 0; a < L; ++a)
    if ((s >> a) & 1u) acc += hd.h[a];
  e[r] = acc;
  e32[r] = (float)acc;
}

static inline unsigned nblocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Slot-major copy of the CSR table (ell[k * dim + r] = an entry of row r, 0 past its end) whose
// order within each row is chosen against shared-memory bank conflicts of the row kernel: there,
// the threads of rows 8m .. 8m+7 gather 16-byte words sx[col] together at every slot, and a
// 16-byte load of 8 threads takes one shared-memory wavefront when their col mod 8 differ.  Per
// group of 8 rows and per slot, a maximum matching of the rows that still have entries to the
// eight residues col mod 8 (augmenting paths; rows with more remaining entries first, each row
// trying its most frequent residues first) picks one entry per matched row; unmatched rows take
// their first remaining entry.  Every row keeps its entry set, so only the order of the
// additions changes.
constexpr int64_t kEllOrderMinDim = 2048;

namespace {
struct BankMatch {
  std::vector<uint32_t>* rem;  // [8] remaining entries of each row
  int owner[8];                // residue -> row (-1 free)
  bool seen[8];
  bool augment(int i) {
    int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t e : rem[i]) ++cnt[ent_col(e) & 7u];
    for (int pass = 0; pass < 8; ++pass) {
      int r = -1;
      for (int k = 0; k < 8; ++k)
        if (cnt[k] > 0 && !seen[k] && (r < 0 || cnt[k] > cnt[r])) r = k;
      if (r < 0) return false;
      seen[r] = true;
      cnt[r] = 0;
      if (owner[r] < 0 || augment(owner[r])) {
        owner[r] = i;
        return true;
      }
    }
    return false;
  }
};
}  // namespace

static void ell_bank_order(const std::vector<int32_t>& ptr, const std::vector<uint32_t>& ent, int64_t dim, int zmax,
                           std::vector<uint32_t>& ell) {
  ell.assign((size_t)zmax * dim, 0u);
  std::vector<uint32_t> rem[8];
  BankMatch bm;
  bm.rem = rem;
  for (int64_t r0 = 0; r0 < dim; r0 += 8) {
    const int nr = (int)std::min<int64_t>(8, dim - r0);
    for (int i = 0; i < 8; ++i) {
      if (i < nr)
        rem[i].assign(ent.begin() + ptr[r0 + i], ent.begin() + ptr[r0 + i + 1]);
      else
        rem[i].clear();
    }
    for (int k = 0;; ++k) {
      int order[8], na = 0;
      for (int i = 0; i < nr; ++i)
        if (!rem[i].empty()) order[na++] = i;
      if (na == 0) break;
      std::sort(order, order + na, [&](int a, int b) { return rem[a].size() > rem[b].size(); });
      for (int r = 0; r < 8; ++r) bm.owner[r] = -1;
      for (int oi = 0; oi < na; ++oi) {
        for (int r = 0; r < 8; ++r) bm.seen[r] = false;
        bm.augment(order[oi]);
      }
      int res_of[8];
      for (int i = 0; i < 8; ++i) res_of[i] = -1;
      for (int r = 0; r < 8; ++r)
        if (bm.owner[r] >= 0) res_of[bm.owner[r]] = r;
      for (int oi = 0; oi < na; ++oi) {
        const int i = order[oi];
        auto& v = rem[i];
        size_t pick = 0;
        if (res_of[i] >= 0)
          for (size_t j = 0; j < v.size(); ++j)
            if ((int)(ent_col(v[j]) & 7u) == res_of[i]) {
              pick = j;
              break;
            }
        ell[(size_t)k * dim + r0 + i] = row_ell_pack(v[pick]);
        v.erase(v.begin() + (ptrdiff_t)pick);
      }
    }
  }
}

std::unique_ptr<SpinTables> build_spin_tables(const ModelHost& m, int N, cudaStream_t s) {
  auto t = std::make_unique<SpinTables>();
  t->L = m.L;
  t->N = N;
  t->dim = (int64_t)binomial(m.L, N);
  if (t->dim >= (int64_t(1) << 24)) throw Error(ED_ERR_INVALID, "sector dimension per spin must be < 2^24");
  t->split = m.L / 2;
  static const Binom bn = make_binom();
  const int bs = 256;
  int64_t dim = t->dim;
  t->basis.alloc(std::max<int64_t>(dim, 1));
  t->rank_lo.alloc(size_t(1) << t->split);
  t->rank_hi.alloc(size_t(1) << (m.L - t->split));
  t->ptr.alloc(dim + 1);
  t->ediag.alloc(std::max<int64_t>(dim, 1));
  t->ediag32.alloc(std::max<int64_t>(dim, 1));
  if (dim > 0) {
    { ProfScope ps_(K_TABLES, s, 0.0); k_unrank<<<nblocks(dim, bs), bs, 0, s>>>(m.L, N, dim, bn, t->basis.p); }
    ED_CHECK_LAUNCH();
  }
  { ProfScope ps_(K_TABLES, s, 0.0); k_rank_lo<<<nblocks(int64_t(1) << t->split, bs), bs, 0, s>>>(t->split, bn, t->rank_lo.p); }
  ED_CHECK_LAUNCH();
  { ProfScope ps_(K_TABLES, s, 0.0); k_rank_hi<<<nblocks(int64_t(1) << (m.L - t->split), bs), bs, 0, s>>>(m.L, N, t->split, bn, t->rank_hi.p); }
  ED_CHECK_LAUNCH();

  std::vector<PairDev> hp(m.pair_a.size());
  for (size_t k = 0; k < hp.size(); ++k) {
    uint32_t a = m.pair_a[k], b = m.pair_b[k];
    uint32_t lo = std::min(a, b), hi = std::max(a, b);
    uint32_t between = (hi >= 1 ? ((1u << hi) - 1u) : 0u) ^ ((lo + 1 >= 32) ? 0xffffffffu : ((1u << (lo + 1)) - 1u));
    hp[k] = PairDev{a, b, (uint32_t)m.pair_vidx[k], between};
  }
  int npairs = (int)hp.size();
  DevBuf<PairDev> dpairs(std::max(npairs, 1));
  if (npairs) ED_CUDA(cudaMemcpyAsync(dpairs.p, hp.data(), npairs * sizeof(PairDev), cudaMemcpyHostToDevice, s));
  DevBuf<int32_t> cnt(std::max<int64_t>(dim, 1));
  if (dim > 0) {
    { ProfScope ps_(K_TABLES, s, 0.0); k_hop_count<<<nblocks(dim, bs), bs, 0, s>>>(dim, t->basis.p, dpairs.p, npairs, cnt.p); }
    ED_CHECK_LAUNCH();
  }
  { ProfScope ps_(K_TABLES, s, 0.0); k_scan_one_block<<<1, 1024, 0, s>>>(cnt.p, dim, t->ptr.p); }
  ED_CHECK_LAUNCH();
  int32_t nnz = 0;
  ED_CUDA(cudaMemcpyAsync(&nnz, t->ptr.p + dim, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  ED_CUDA(cudaStreamSynchronize(s));
  t->nnz = nnz;
  t->ent.alloc(std::max<int64_t>(nnz, 1));
  RankView rv{t->rank_lo.p, t->rank_hi.p, t->split, (uint32_t)((1u << t->split) - 1u)};
  if (dim > 0 && nnz > 0) {
    { ProfScope ps_(K_TABLES, s, 0.0); k_hop_fill<<<nblocks(dim, bs), bs, 0, s>>>(dim, t->basis.p, rv, dpairs.p, npairs, t->ptr.p, t->ent.p); }
    ED_CHECK_LAUNCH();
  }
  {
    DevBuf<int> dz(1);
    ED_CUDA(cudaMemsetAsync(dz.p, 0, sizeof(int), s));
    if (dim > 0) {
      { ProfScope ps_(K_TABLES, s, 0.0); k_max_int<<<std::min<unsigned>(nblocks(dim, bs), 1024), bs, 0, s>>>(cnt.p, dim, dz.p); }
      ED_CHECK_LAUNCH();
    }
    ED_CUDA(cudaMemcpyAsync(&t->zmax, dz.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    ED_CUDA(cudaStreamSynchronize(s));
    t->ell.alloc(std::max<int64_t>((int64_t)(t->zmax + kEllPad) * dim, 1));
    ED_CUDA(cudaMemsetAsync(t->ell.p, 0, (size_t)(t->zmax + kEllPad) * dim * sizeof(uint32_t), s));
    if (dim >= kEllOrderMinDim && t->zmax > 0) {
      // large sectors: slot order chosen on the host against shared-memory bank conflicts
      std::vector<int32_t> hptr(dim + 1);
      std::vector<uint32_t> hent(std::max<int64_t>(nnz, 1));
      ED_CUDA(cudaMemcpyAsync(hptr.data(), t->ptr.p, (dim + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      ED_CUDA(cudaMemcpyAsync(hent.data(), t->ent.p, std::max<int64_t>(nnz, 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
      ED_CUDA(cudaStreamSynchronize(s));
      std::vector<uint32_t> hell;
      ell_bank_order(hptr, hent, dim, t->zmax, hell);
      ED_CUDA(cudaMemcpyAsync(t->ell.p, hell.data(), hell.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
      ED_CUDA(cudaStreamSynchronize(s));
    } else if (dim > 0 && t->zmax > 0) {
      { ProfScope ps_(K_TABLES, s, 0.0); k_ell_fill<<<nblocks(dim, bs), bs, 0, s>>>(dim, t->ptr.p, t->ent.p, t->zmax, t->ell.p); }
      ED_CHECK_LAUNCH();
    }
  }
  Diag32 hd;
  for (int a = 0; a < kMaxOrb; ++a) hd.h[a] = a < m.L ? m.h[a * m.L + a] : 0.0;
  if (dim > 0) {
    { ProfScope ps_(K_TABLES, s, 0.0); k_ediag<<<nblocks(dim, bs), bs, 0, s>>>(dim, m.L, t->basis.p, hd, t->ediag.p, t->ediag32.p); }
    ED_CHECK_LAUNCH();
  }
  ED_CUDA(cudaStreamSynchronize(s));  // dpairs and cnt are released on return
  return t;
}

void basis_to_host(int L, int N, uint32_t* out, int64_t dim) {
  static const Binom bn = make_binom();
  DevBuf<uint32_t> d(std::max<int64_t>(dim, 1));
  if (dim > 0) {
    { ProfScope ps_(K_TABLES, 0, 0.0); k_unrank<<<nblocks(dim, 256), 256>>>(L, N, dim, bn, d.p); }
    ED_CHECK_LAUNCH();
    ED_CUDA(cudaMemcpy(out, d.p, dim * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  }
}

}  // namespace ed
