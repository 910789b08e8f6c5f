/*
 * ed.h -- C ABI of libed, a GB300 (sm_103a) exact-diagonalization impurity solver.
 *
 * The solver follows Sec. 4 of "Pyqcm: An open-source Python library for quantum cluster
 * methods" (arXiv:2305.18643): a Hubbard-like cluster with optional bath orbitals
 * (Eq. Hubbard, Eq. cdmft1) is diagonalized in a fixed (N_up, N_dn) sector with a
 * matrix-free factorized Hamiltonian (Eq. factorized), the Lanczos ground state (Sec. 4.2)
 * and the Lanczos / band-Lanczos Green function (Secs. 4.3, 4.4), evaluated on a frequency
 * grid (Eq. jacobi, Eq. spectral1).
 *
 * Conventions shared by every call:
 *  - Orbitals: cluster sites 0 .. n_sites-1 first, then bath orbitals n_sites .. L-1,
 *    L = n_sites + n_bath <= 32.  Bit a of a spin's bit string is the occupation of orbital a
 *    (Sec. 4.1, Eq. basis); each spin's states are labelled by ascending integer value, which
 *    is the combinatorial-number-system rank.
 *  - Hamiltonian: H = sum_{ab,s} h_ab c+_{as} c_{bs} + sum_{i<n_sites} U_i n_{i up} n_{i dn} with
 *    h_ij = t_ij (sites), h_ii = t_ii - mu (sites), h_{i,ns+a} = theta_ia, h_{ns+a,ns+a} = eps_a.
 *  - State vectors are row-major psi[u][d]: u = up label (slow), d = down label (fast); a
 *    leading dimension ld >= d_dn may pad rows.
 *  - Every call returns an ed_status: 0 = ok, > 0 = pending / warning, < 0 = error.  On error
 *    ed_last_error() returns a message (thread-local, valid until the next call on that thread).
 *  - Host arrays passed in are copied before the call returns; the caller keeps ownership.
 *  - Device pointers are CUDA device addresses on the current device.
 */
#ifndef ED_H
#define ED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int ed_status;

enum {
  ED_OK = 0,
  ED_PENDING = 1,             /* request still running (ed_poll) */
  ED_WARN_DEGENERATE = 2,     /* ground state converged but a second Ritz value lies within
                                 1e-8 max(1,|E0|): G is not unique (Sec. 4.2) */
  ED_WARN_NOT_CONVERGED = 3,  /* max_iter reached; results written are the last iterate */
  ED_ERR_INVALID = -1,        /* bad argument (NaN, non-symmetric t, bad sector, size limits) */
  ED_ERR_OOM = -2,            /* device allocation failed */
  ED_ERR_CUDA = -3,           /* a CUDA call failed */
  ED_ERR_TOO_LARGE = -5,      /* request exceeds the memory budget of a server */
  ED_ERR_TIMEOUT = -6,        /* a bounded device-side wait gave up */
  ED_ERR_STATE = -7,          /* call out of order (e.g. no ground state yet) */
  ED_ERR_NOT_FOUND = -8,      /* unknown request id */
  ED_ERR_CANCELLED = -9
};

enum { ED_FP64 = 0, ED_FP32 = 1 };             /* precision of stored vectors */
enum { ED_GF_CF = 0, ED_GF_BAND = 1 };         /* Green-function method: Sec. 4.3 / Sec. 4.4 */
enum { ED_AXIS_REAL = 0, ED_AXIS_MATSUBARA = 1 };

/* Cluster description (Eq. cdmft1).  All arrays are host arrays, copied at create. */
typedef struct ed_cluster_desc {
  int n_sites;          /* cluster sites, >= 1 */
  int n_bath;           /* bath orbitals, >= 0; n_sites + n_bath <= 32 */
  const double* t;      /* n_sites x n_sites row-major, symmetric; diagonal = on-site energies */
  const double* U;      /* n_sites on-site interactions */
  double mu;            /* chemical potential, acts on cluster sites only */
  const double* eps;    /* n_bath bath energies (absolute); may be NULL if n_bath == 0 */
  const double* theta;  /* n_sites x n_bath row-major hybridizations; may be NULL if n_bath == 0 */
  int n_up, n_dn;       /* sector; 0 <= N_s <= L */
  int precision;        /* ED_FP64 or ED_FP32 (FP32 vectors, FP64 reductions and recurrence,
                           FP64 polish of the ground state) */
  int gf_method;        /* ED_GF_CF or ED_GF_BAND */
  uint64_t seed;        /* Lanczos start vector: v0[u][d] = splitmix64(seed ^ (u * d_dn + d)) */
  double tol;           /* ground-state residual target ||H W - E0 W|| <= tol max(1,|E0|);
                           <= 0 selects 1e-12 */
  int max_iter;         /* Lanczos iterations per ground-state pass; <= 0 selects 600 */
} ed_cluster_desc;

typedef struct ed_cluster ed_cluster;

/* Message of the last error on the calling thread (empty if none).  The string is owned by the
 * library and stays valid until the next libed call on the same thread. */
const char* ed_last_error(void);

/* Validates and copies desc, builds the ground-state sector's basis and hopping tables on the
 * device.  Errors: ED_ERR_INVALID (L > 32, a NaN, t not symmetric, N_s outside [0, L],
 * d_s >= 2^24, more than 128 distinct off-diagonal h values), ED_ERR_OOM, ED_ERR_CUDA.
 * On success *out owns device memory until ed_cluster_destroy. */
ed_status ed_cluster_create(const ed_cluster_desc* desc, ed_cluster** out);

/* Frees every device buffer of the cluster.  NULL is ignored. */
void ed_cluster_destroy(ed_cluster* c);

/* Lanczos ground state (Sec. 4.2): three-term recursion with FP64 reductions, lowest Ritz pair
 * of the tridiagonal matrix, reconstruction of the ground state by retracing the recursion,
 * then an explicit FP64 residual.  Synchronous.  Writes E0 (FP64), the residual
 * ||H W - E0 W|| / max(1,|E0|) with ||W|| = 1, and the number of Lanczos iterations; any output
 * pointer may be NULL.  The ground state stays on the device in the handle.
 * Returns ED_OK, ED_WARN_DEGENERATE or ED_WARN_NOT_CONVERGED (results still written). */
ed_status ed_ground_state(ed_cluster* c, double* E0, double* residual, int* iters);

/* Copies the ground state psi[u][d] (d_up x d_dn, contiguous, FP64) to out (host or device).
 * ED_ERR_STATE if ed_ground_state has not run. */
ed_status ed_ground_vector(ed_cluster* c, double* out, int out_is_device);

/* Cluster Green function G_ij(z), i, j over cluster sites only (Eq. green), for one spin
 * (0 = up, 1 = down), on z_k = omega[k] + i eta (ED_AXIS_REAL) or z_k = i omega[k]
 * (ED_AXIS_MATSUBARA).  Method from desc.gf_method.  Runs ed_ground_state first if needed.
 * G_out: interleaved complex128 [n_freq][n_sites][n_sites] (2 doubles per element), host or
 * device memory as out_is_device says; owned by the caller.  Returns ED_WARN_NOT_CONVERGED when
 * a band run reached its size limit before G converged on the grid (G is still written). */
ed_status ed_green(ed_cluster* c, const double* omega, int n_freq, double eta, int axis, int spin,
                   double* G_out, int out_is_device);

/* Options of a cluster's Green-function runs (defaults in brackets):
 *  ED_OPT_BAND_MAX_DIM  Krylov vectors per part (electron / hole) of the band method [20000];
 *                       the paper's runs stop between 100 and 500 (Sec. 4.4)
 *  ED_OPT_CF_MAX_STEPS  Lanczos steps per continued fraction [20000]
 *  ED_OPT_GF_TOL        a run stops once G on the grid changes by less than this between two
 *                       successive checks, twice [1e-10 for FP64, 1e-6 for FP32 vectors]
 *  ED_OPT_TWO_PASS_MIN_BYTES
 *                       H.psi on the library's own vectors (ground state, continued fractions,
 *                       band Lanczos, ed_hpsi with rows padded to a multiple of 128) takes the
 *                       two-pass kernels (a row pass for the down-spin hops and the diagonal, a
 *                       column pass for the up-spin hops) once a vector holds at least this many
 *                       bytes [33554432: beyond 32 MiB a vector no longer fits L2 comfortably];
 *                       0 selects them at every size.  Both forms compute the same product; the
 *                       option exists so that the two-pass kernels can be checked on sectors
 *                       small enough for a CPU reference.  Must be >= 0.
 *  ED_OPT_DAVIDSON_STATES
 *                       k in [1, 16] [1]: with k > 1 ed_ground_state finds the k lowest states of
 *                       the sector by the Davidson method (FP64 vectors whatever the precision;
 *                       Sec. 4.2 recommends it for degenerate ground states, and the library's
 *                       Davidson_states option of Sec. 9 targets several low states), and ed_green
 *                       returns the mixed-state Green function sum_s p_s G_s(z), G_s that of state s
 *                       (its energy in the place of E0, Eq. green).  Setting it discards the ground
 *                       state found so far.
 *  ED_OPT_TEMPERATURE   T >= 0 [0] of the mixed state: p_s = exp(-(E_s - E_0) / T) / Z over the k
 *                       states; T = 0 gives equal weights to the states within 1e-9 max(1,|E_0|)
 *                       of E_0 (a degenerate ground manifold), so G does not depend on the basis
 *                       chosen inside it.  The paper's temperature option: low, since only a few
 *                       states are kept.
 *  ED_OPT_TENSOR_GRAM   1 [default] or 0: with FP32 vectors, the Gram matrix W^T W of the band
 *                       Lanczos orthogonalization runs on the tensor cores (TMA tile loads,
 *                       tcgen05 MMA on TF32 head/tail splits, compensated sums per stage) where
 *                       the layout allows it; the projections on the previous blocks stay on the
 *                       CUDA cores (faster there); 0 keeps every Gram on the CUDA-core kernel.  A bounded wait of that kernel that gives up makes
 *                       ed_green return ED_ERR_TIMEOUT.
 * ED_ERR_INVALID for an unknown option or a non-finite value. */
enum { ED_OPT_BAND_MAX_DIM = 1, ED_OPT_CF_MAX_STEPS = 2, ED_OPT_GF_TOL = 3, ED_OPT_TWO_PASS_MIN_BYTES = 4,
       ED_OPT_DAVIDSON_STATES = 5, ED_OPT_TEMPERATURE = 6, ED_OPT_TENSOR_GRAM = 7 };
ed_status ed_set_option(ed_cluster* c, int option, double value);

/* The states behind the cluster's Green function after ed_ground_state: their energies (ascending)
 * and mixed-state weights p_s (ED_OPT_TEMPERATURE); one state of weight 1 with the Lanczos method.
 * Writes min(capacity, count) values to each non-NULL array and the number of states to *count.
 * ED_ERR_STATE before ed_ground_state. */
ed_status ed_low_states(const ed_cluster* c, int capacity, double* E, double* weights, int* count);

/* Statistics of the last ed_green: total Lanczos (or band) steps over all starting vectors and
 * the longest run.  Any pointer may be NULL. */
ed_status ed_green_stats(const ed_cluster* c, int64_t* total_steps, int* max_steps);

/* Batched form: n independent clusters solved together.  For each cluster: the Lanczos ground
 * state (as ed_ground_state, at most 600 levels per pass) and, when n_freq > 0, the
 * continued-fraction Green function of Sec. 4.3 for spin up and
 * spin down (spin down equals spin up when n_up == n_dn), on z = omega + i eta (ED_AXIS_REAL)
 * or i omega (ED_AXIS_MATSUBARA); each continued fraction stops when it converges on the grid (as
 * in ed_green) or at the preset maximum of min(cf_max_levels, 2 d + 16) levels (cf_max_levels <= 0
 * selects 20000, so that runs end on convergence: at eta = 0.05 on the real axis a sector of
 * 1e4 - 3e4 states needs 1,500 - 3,000 levels for G to 1e-8; Sec. 4.3 stops at a preset maximum).  All clusters share `precision` (ED_FP64 or ED_FP32); each
 * cluster's seed and tol are taken from its description, its precision and gf_method are
 * ignored.  At most 20 orbitals per cluster.
 *  - E0, residual, status, iters (ground-state levels), gf_steps (continued-fraction levels over
 *    all runs): n values each (host), any may be NULL; status per cluster is ED_OK,
 *    ED_WARN_DEGENERATE or ED_WARN_NOT_CONVERGED.
 *  - G_out: complex128 (2 doubles each), clusters one after the other, cluster c holding
 *    [2 spins][n_freq][n_sites_c][n_sites_c]; host or device memory as out_is_device says.
 * Tables of all clusters are built by three launches; the solve proper is one CUDA graph: a
 * persistent ground-state kernel, in which every thread block takes the next cluster from a
 * queue, largest first; a persistent continued-fraction kernel, in which blocks take the
 * continued fractions of more than 8,192 states and, once those are gone, every warp takes the
 * smaller ones one at a time; then the evaluation on the grid and the assembly of G.  The block width and the mapping of the
 * block-level H.psi are picked by timing candidates on the first call for a batch shape (then
 * cached). */
ed_status ed_batch_solve(const ed_cluster_desc* descs, int n, int precision, const double* omega, int n_freq,
                         double eta, int axis, int cf_max_levels, double* E0, double* residual, int* status, int* iters,
                         int64_t* gf_steps, double* G_out, int out_is_device);

/* ---- served form: continuous batching of cluster solves --------------------------------- */

/* A server solves cluster requests (ground state and, if asked, G of both spins) as they arrive,
 * the way a quantum-cluster code issues one impurity solve per VCA / CDMFT iteration (Sec. 5).
 * It owns max_slots lanes: each lane is a host thread with a CUDA stream of its own.  A request
 * is admitted when a lane is free and its device memory (sector tables, Lanczos vectors,
 * Green-function vectors and G, from closed forms of the sector dimensions) fits what is left
 * of mem_budget_bytes; admission is first-come first-served, and a later request that fits may
 * pass a waiting larger one at most 8 times.  Admitted requests run at the same time on their
 * lanes' streams.  Requests whose sectors (ground-state and N +- 1) hold at most
 * ED_SRV_BATCH_MAX_DIM elements, with at most 20 orbitals, the continued-fraction method and the
 * same precision, frequency grid and level cap, are taken together by one lane and solved by the
 * persistent kernels of ed_batch_solve with a fixed block configuration; larger ones run the
 * single-cluster path (ed_cluster_create, ed_ground_state, ed_green for each spin).  Which path
 * a request takes depends on the request alone, and neither path's arithmetic depends on the
 * other requests, so a request gives the same result alone and among others.
 * Every request and server call is host-side; no device wait is unbounded. */
typedef struct ed_server ed_server;

typedef struct ed_request_opts {
  const double* omega;   /* n_freq frequencies (copied at submit); NULL when n_freq == 0 */
  int n_freq;            /* 0: ground state only */
  double eta;            /* broadening of ED_AXIS_REAL */
  int axis;              /* ED_AXIS_REAL or ED_AXIS_MATSUBARA */
  int cf_max_levels;     /* preset maximum of every continued fraction; <= 0 selects 20000
                            (runs end on convergence on the grid, as in ed_green) */
  double* G_out;         /* host, complex128 [2 spins][n_freq][n_sites][n_sites]; written before
                            ed_poll / ed_wait report completion; the caller keeps it alive until
                            then (NULL allowed when n_freq == 0) */
} ed_request_opts;

typedef struct ed_result {
  int status;            /* the request's final status (ED_OK, a warning or an error code) */
  int path;              /* 0 single-cluster path, 1 batched persistent kernels */
  double E0, residual;   /* as ed_ground_state */
  int iters;             /* ground-state Lanczos levels */
  int batch_size;        /* requests solved together with this one (1 on the single path) */
  int64_t gf_steps;      /* Green-function Lanczos levels */
  double queued_ms;      /* submit -> start on a lane */
  double run_ms;         /* start -> results written */
  double latency_ms;     /* submit -> results written */
  size_t device_bytes;   /* device memory reserved for it at admission */
} ed_result;

/* Creates a server on the current device.  mem_budget_bytes > 0, 1 <= max_slots <= 64.
 * ED_ERR_INVALID, ED_ERR_CUDA. */
ed_status ed_server_create(size_t mem_budget_bytes, int max_slots, ed_server** out);

/* Stops admitting, cancels queued requests, lets running ones reach their next check point
 * (they end with ED_ERR_CANCELLED), joins the lanes and frees everything.  NULL is a no-op. */
void ed_server_destroy(ed_server* srv);

/* Server options: ED_SRV_BATCH_MAX_DIM (largest sector dimension of the batched path; 0 turns it
 * off; default 100000), ED_SRV_BATCH_MAX_REQUESTS (requests per batched solve; default 64),
 * ED_SRV_GF_BUDGET_FRACTION (share of mem_budget_bytes that one request's Green-function
 * vectors may take; default 0.5), ED_SRV_PAUSE (1: lanes take no new request, submitted ones
 * stay queued; 0: admission resumes; default 0).  ED_ERR_INVALID for an unknown option or a
 * bad value. */
enum { ED_SRV_BATCH_MAX_DIM = 1, ED_SRV_BATCH_MAX_REQUESTS = 2, ED_SRV_GF_BUDGET_FRACTION = 3, ED_SRV_PAUSE = 4 };
ed_status ed_server_set_option(ed_server* srv, int option, double value);

/* Device bytes a request would reserve on the single-cluster path with the given Green-function
 * budget (gf_budget_bytes <= 0: unlimited), from closed forms only: no CUDA call, no allocation.
 * Continued fractions reserve up to the budget (their runs go in chunks); band Lanczos reserves
 * all its blocks when they fit the budget, else its ring of blocks.
 * ED_ERR_INVALID for a bad description. */
ed_status ed_request_bytes(const ed_cluster_desc* desc, const ed_request_opts* opts, size_t gf_budget_bytes,
                           size_t* bytes);

/* Queues one request (desc and opts are copied; desc->precision, gf_method, seed, tol and
 * max_iter apply).  *req_id receives its id.  ED_ERR_TOO_LARGE if even its smallest device
 * footprint exceeds the server's budget; ED_ERR_INVALID for a bad description or options;
 * ED_ERR_STATE after ed_server_destroy has begun. */
ed_status ed_submit(ed_server* srv, const ed_cluster_desc* desc, const ed_request_opts* opts, uint64_t* req_id);

/* Non-blocking: ED_PENDING while the request is queued or running; otherwise ED_OK with *out
 * filled (out->status is the request's own status) and the id forgotten; ED_ERR_NOT_FOUND for
 * an unknown or already collected id. */
ed_status ed_poll(ed_server* srv, uint64_t req_id, ed_result* out);

/* As ed_poll, but waits up to timeout_s seconds; ED_ERR_TIMEOUT if the request is still pending
 * then (it keeps running). */
ed_status ed_wait(ed_server* srv, uint64_t req_id, double timeout_s, ed_result* out);

/* Cancels a request: a queued one ends at once, a running one at its next check point (after
 * the ground state, between spins); its final status is ED_ERR_CANCELLED.  ED_ERR_NOT_FOUND for
 * an unknown id. */
ed_status ed_cancel(ed_server* srv, uint64_t req_id);

/* Test hook for failure handling, with the failure made on the host: when a lane picks the
 * request it ends it with `status` (< 0) before any device work, as a failed CUDA call would;
 * the other requests go on.  ED_ERR_NOT_FOUND if the request is not queued. */
ed_status ed_server_inject_failure(ed_server* srv, uint64_t req_id, int status);

typedef struct ed_server_stats {
  int64_t submitted, completed, failed, cancelled;
  int queued, running;            /* now */
  int max_running;                /* most requests on lanes at once so far */
  size_t reserved_bytes;          /* device memory reserved now */
  size_t peak_reserved_bytes;
  int64_t batched_solves;         /* batched-path solves (each of one or more requests) */
} ed_server_stats;
ed_status ed_server_stats_get(ed_server* srv, ed_server_stats* out);

/* ---- lower-level calls (parity tests and benchmarks) ------------------------------------- */

/* Sector dimensions d_up = C(L, n_up), d_dn = C(L, n_dn) of any sector of this cluster. */
ed_status ed_sector_dims(const ed_cluster* c, int n_up, int n_dn, int64_t* d_up, int64_t* d_dn);

/* Basis of one spin with N particles on L orbitals (Sec. 4.1), computed on the device by
 * unranking the combinatorial number system; copied to the host array out[capacity].
 * *dim receives C(L, N).  ED_ERR_INVALID if capacity < C(L, N). */
ed_status ed_basis(int L, int N, uint32_t* out, int64_t capacity, int64_t* dim);

/* Hopping table of one spin with N particles (Sec. 4.1, element (-1)^{M_ab} h_ab), built on
 * the device, copied to host arrays: row_ptr[d + 1] (CSR, pull form: y[r] += K[r, c] x[c]),
 * entries[n] packed as (c << 8) | (sign_bit << 7) | value_index, values[<= 128] the distinct
 * off-diagonal h_ab.  K[r, c] = (sign_bit ? -1 : 1) * values[value_index].  The diagonal
 * h_aa n_a is not in the table.  *n_entries and *n_values receive the counts; ED_ERR_INVALID if
 * cap_entries is too small. */
ed_status ed_hop_table(ed_cluster* c, int N, int32_t* row_ptr, uint32_t* entries, double* values,
                       int64_t cap_entries, int64_t* n_entries, int* n_values);

/* y = H x in sector (n_up, n_dn) on device arrays of d_up rows, leading dimension ld >= d_dn
 * (elements; ld <= 0 means d_dn); dtype ED_FP64 (double) or ED_FP32 (float; products and sums in FP32).  x and y
 * must not overlap.  stream: a cudaStream_t; NULL is the CUDA default stream.  Asynchronous
 * on that stream. */
ed_status ed_hpsi(ed_cluster* c, int n_up, int n_dn, int dtype, const void* x, void* y, int64_t ld,
                  void* stream);

/* y = H x in the cluster's own sector (n_up, n_dn of its description) and, in FP64 device memory,
 * out3[0] = <x, y>, out3[1] = <y, y>, out3[2] = <x, x>, for callers that must not allocate device
 * memory (an application that manages the GPU's memory itself, through its own pool or caching
 * allocator, cannot let the library call cudaMalloc).  The paper has no counterpart: this is an
 * interface of this library.  The call allocates nothing: the reduction scratch is a fixed
 * 96 KiB array inside libed, and the sector's tables are the ones ed_cluster_create built.
 *  - x, y: device arrays of d_up rows with leading dimension ld (ld <= 0 means d_dn), dtype
 *    ED_FP64 or ED_FP32; they must not overlap.  out3: 3 doubles of device memory.
 *  - Sectors larger than 4,194,304 elements (d_up * d_dn) are rejected with ED_ERR_TOO_LARGE.
 *  - The current device must be the one the cluster was created on (its tables live there);
 *    otherwise ED_ERR_INVALID, before any launch.  ed_ground_state, ed_ground_vector, ed_green,
 *    ed_hop_table and ed_hpsi make the same check.
 *  - The first call on a device looks up the scratch array's device address (once per device,
 *    with that device current); make that first call before any stream capture.
 *  - Every call shares the scratch array, and the array keeps the last call's contents; calls
 *    whose kernels overlap on the GPU (different streams or host threads) race on it and must be
 *    ordered by the caller.
 *  - Asynchronous on `stream` (NULL is the CUDA default stream). */
ed_status ed_hpsi_dots_static(ed_cluster* c, int dtype, const void* x, void* y, int64_t ld, double* out3,
                              void* stream);

/* ---- lattice steps on the cluster Green function: CPT (Sec. 3) and the CDMFT bath fit (Sec. 6) -- */

/* A lattice tiled by identical clusters of L sites (Sec. 2): site i of the cluster at super-lattice
 * vector r~ = n E (n an integer vector, E the super-lattice basis) sits at r~ + pos[i].  The
 * one-body terms that join different clusters are listed as bonds: bond q joins site
 * bonds[q (2 + dim)] of the cluster at the origin to site bonds[q (2 + dim) + 1] of the cluster at
 * n = (bonds[q (2 + dim) + 2], ...), with the matrix element bond_t[q] (the Hermitian partner is
 * implied).  Hops inside the cluster belong to the cluster's own t and are not listed.  Host
 * arrays, read during the call only. */
typedef struct ed_superlattice {
  int n_sites;            /* L, 1 <= L <= 32 */
  int dim;                /* D = 1, 2 or 3 */
  const double* pos;      /* L x D site positions */
  const double* E;        /* D x D super-lattice basis, rows e_1 .. e_D */
  int n_bonds;
  const int* bonds;       /* n_bonds x (2 + D) */
  const double* bond_t;   /* n_bonds */
} ed_superlattice;

enum { ED_CPT_MATRIX = 0, ED_CPT_PERIODIZED = 1, ED_CPT_AVERAGE = 2 };

/* Hybridization function Gamma_{mu nu}(z) = sum_a theta_{mu a} theta_{nu a} / (z - eps_a)
 * (Eq. hybridization) on nz complex frequencies z (interleaved re, im; host).  eps: n_bath, theta:
 * n_sites x n_bath row-major (host).  Gamma_out: complex128 [nz][n_sites][n_sites], host or device
 * as out_is_device says.  Synchronous.  ED_ERR_INVALID for bad sizes or NULL arrays. */
ed_status ed_hybridization(int n_sites, int n_bath, const double* eps, const double* theta, const double* z, int nz,
                           double* Gamma_out, int out_is_device);

/* Cluster perturbation theory on nk wave vectors kt (nk x D, host) from the cluster Green function
 * Gc (complex128 [nz][L][L], e.g. the output of ed_green):
 *   ED_CPT_MATRIX      out [nk][nz][L][L] = G(k~, z) = [Gc(z)^-1 + Gamma(z) - V(k~)]^-1
 *                      (Eq. CPT1; with the bath compensation of Eq. CPT_CDMFT when Gamma, complex128
 *                      [nz][L][L], is not NULL)
 *   ED_CPT_PERIODIZED  out [nk][nz] = (1/L) sum_{R R'} e^{-i k.(R - R')} G_{R R'}(k, z) (Eq. CPT3,
 *                      the Green-function periodization, k~ taken equal to k)
 *   ED_CPT_AVERAGE     out [nz][L][L] = the mean of G(k~, z) over the nk given k~, i.e. the
 *                      super-lattice-averaged Green function of the CDMFT loop (Sec. 6, step 3)
 *                      when kt is a grid of the reduced Brillouin zone.
 * V(k~)_{ij} = sum over bonds of t e^{i k~.r~} at (i, j) and its conjugate at (j, i) (the mixed
 * representation of Sec. 2.2).  Gc, Gamma and out are host or device arrays as io_is_device says.
 * Synchronous.  ED_ERR_INVALID for a bad lattice or mode, or when a matrix to invert is singular. */
ed_status ed_cpt_green(const ed_superlattice* lat, const double* Gc, const double* Gamma, int nz, const double* kt, int nk,
                       int mode, double* out, int io_is_device);

/* The fixed part of the CDMFT distance (Sec. 6, steps 3-4): from the cluster Green function Gc of
 * the impurity solved with the current bath, that bath's Gamma (may be NULL: no bath) and the
 * reduced-zone grid kt, A(z) = Gamma(z) + Gc(z)^-1 - G_bar(z)^-1, which equals
 * z - h_c - calG_0(z)^-1 with calG_0^-1 = G_bar^-1 + Sigma_c, so that Eq. dist_func reads
 * d = sum_n W_n ||A(z_n) - Gamma'(z_n)||_F^2 for a trial bath Gamma'.  A_out: complex128
 * [nz][L][L]; Gc, Gamma, A_out host or device as io_is_device says.  Synchronous. */
ed_status ed_cdmft_target(const ed_superlattice* lat, const double* Gc, const double* Gamma, int nz, const double* kt,
                          int nk, double* A_out, int io_is_device);

/* The distance of Eq. dist_func, d_c = sum_n W_n ||A(z_n) - Gamma_c(z_n)||_F^2, for n_cand trial
 * baths at once (eps: n_cand x n_bath, theta: n_cand x n_sites x n_bath), and, when grad_out is
 * not NULL, its gradient: grad_out[c][a] = dd/deps_a, grad_out[c][n_bath + mu n_bath + a] =
 * dd/dtheta_{mu a}.  z: nz complex frequencies, weights: nz values W_n >= 0, A: complex128
 * [nz][n_sites][n_sites] from ed_cdmft_target; all host arrays.  Synchronous. */
ed_status ed_cdmft_distance(int n_sites, int n_bath, int n_cand, const double* eps, const double* theta, const double* z,
                            int nz, const double* weights, const double* A, double* d_out, double* grad_out);

/* Bath fit of the CDMFT loop (Sec. 6, step 4): minimizes the distance over the bath energies and
 * the hybridizations theta_{mu a} with theta_free[mu n_bath + a] != 0 (theta_free NULL: all),
 * starting from eps and theta, which receive the result (host arrays).  BFGS with a backtracking
 * line search on the host; every distance and gradient is computed by ed_cdmft_distance's kernels.
 * Stops when the largest gradient component is below gtol (<= 0: 1e-10), when a step no longer
 * lowers d, or after max_iter iterations (<= 0: 500).  d_out, iters_out may be NULL.  Synchronous. */
ed_status ed_cdmft_fit(int n_sites, int n_bath, double* eps, double* theta, const unsigned char* theta_free,
                       const double* z, int nz, const double* weights, const double* A, double gtol, int max_iter,
                       double* d_out, int* iters_out);

/* Gram matrix of the band Lanczos orthogonalization (Sec. 4.4) on given FP32 vectors, the kernel
 * alone: G[i][j] = sum_{e < n} X_i[e] Y_j[e] in FP64, with nx <= 16 vectors X (or nx = 32: two
 * blocks of 16) and ny <= 16 vectors Y, all device arrays vstride elements apart.  method 1: the
 * tensor-core kernel (tcgen05 MMA, 3xTF32 split, TMA loads); it needs 16-byte-aligned vectors,
 * n % 32 == 0 and vstride % 4 == 0, else ED_ERR_INVALID; ED_ERR_TIMEOUT when its bounded waits gave
 * up.  method 0: the CUDA-core FP32 kernel.  When Y == X and ny == nx <= 16 the symmetric form
 * runs.  G_out: host array of nx x ny doubles.  Synchronous.  For checks of the two kernels. */
ed_status ed_gram_f32(const float* X, int nx, const float* Y, int ny, int64_t vstride, int64_t n, int method,
                      double* G_out);

/* ---- cluster symmetries (Sec. 4.5) ----------------------------------------------------------
 * The Hamiltonian of one irreducible representation of an Abelian symmetry group of the cluster,
 * in the basis of symmetrized states, stored on the device (CSR), and its ground state.
 * The group is generated by n_gen (1..5) commuting, independent involutions of the L orbitals:
 * perm[j * L + i] is the image of orbital i under generator j (host array), applied to both
 * spins; the irrep is named by the characters signs[j] = +1 or -1 of the generators (every
 * irrep of such a group is one-dimensional with characters +-1).  The one-body matrix and U of
 * the cluster must be invariant under every generator (else ED_ERR_INVALID).
 * Basis: one representative per orbit of the binary states (b_up, b_dn) of the cluster's
 * (N_up, N_dn) sector, the one with the smallest key b_up * 2^L + b_dn, kept unless its
 * symmetrized state vanishes; keys ascending.  Matrix elements follow Eq. matrixElement for
 * normalized states (sqrt(|S_r2| / |S_r1|) with S_r the stabilizer), real symmetric; entries of
 * magnitude below 1e-13 after the cancellations of Sec. 4.5 are dropped.
 * The handle borrows the cluster (which must outlive it) and its stream. */
typedef struct ed_sym ed_sym;

/* Builds the basis and the matrix of the irrep.  ED_ERR_INVALID (bad group, non-invariant H,
 * more than 2^31 states), ED_ERR_OOM, ED_ERR_CUDA.  Synchronous. */
ed_status ed_sym_create(ed_cluster* c, int n_gen, const int* perm, const int* signs, ed_sym** out);

/* General Abelian groups (Sec. 4.5): generators of orders orders[j] >= 2 (perm as above, each
 * g_j^{orders[j]} = identity; commuting, independent; at most 32 elements), the irrep named by
 * integers irrep[j] in [0, orders[j]): the element prod_j g_j^{a_j} has the character
 * exp(2 pi i sum_j irrep[j] a_j / orders[j]).  With a complex character (a four-fold rotation, a
 * translation of a ring) the irrep's matrix is complex Hermitian and every vector of the handle
 * (ed_sym_hpsi, ed_sym_ground_vector) and every matrix value (ed_sym_matrix) is an interleaved
 * complex128 pair; ed_sym_is_complex tells.  ed_sym_create is this call with every order 2 and
 * irrep[j] = (signs[j] == -1).  Errors as ed_sym_create. */
ed_status ed_sym_create_abelian(ed_cluster* c, int n_gen, const int* perm, const int* orders, const int* irrep,
                                ed_sym** out);

/* 1 when some character of the irrep is complex (complex matrix and vectors), else 0. */
ed_status ed_sym_is_complex(const ed_sym* s, int* is_complex);

/* Dimension of the symmetrized sector and number of stored matrix entries (either may be NULL). */
ed_status ed_sym_info(const ed_sym* s, int64_t* dim, int64_t* nnz);

/* Host copies of the representatives' keys (dim uint64) and stabilizer sizes (dim bytes); either
 * may be NULL.  Synchronous. */
ed_status ed_sym_basis(const ed_sym* s, uint64_t* keys, uint8_t* stab);

/* Host copies of the CSR matrix: rowptr (dim + 1 int64), col (nnz int32, ascending per row),
 * val (nnz doubles, or nnz interleaved complex128 pairs for a complex irrep); any may be NULL.
 * Synchronous. */
ed_status ed_sym_matrix(const ed_sym* s, int64_t* rowptr, int32_t* col, double* val);

/* y = H x in the symmetrized basis; x, y: device arrays of dim doubles (dim complex128 pairs for
 * a complex irrep) on the cluster's device (y must not alias x).  Synchronous. */
ed_status ed_sym_hpsi(ed_sym* s, const double* x, double* y);

/* Lowest eigenvalue of the irrep's H by FP64 Lanczos (Sec. 4.2) with the cluster's tol, max_iter
 * and seed; the ground vector is kept in the handle.  residual = |H w - E0 w| of the normalized
 * vector; ED_WARN_NOT_CONVERGED when it stays above 1e-12 max(1, |E0|) (results still written).
 * ED_ERR_INVALID for an empty irrep.  Any output pointer may be NULL.  Synchronous. */
ed_status ed_sym_ground_state(ed_sym* s, double* E0, double* residual, int* iters);

/* Host copy of the ground vector (dim doubles, or dim complex128 pairs for a complex irrep;
 * normalized).  ED_ERR_STATE before ed_sym_ground_state. */
ed_status ed_sym_ground_vector(const ed_sym* s, double* out);

/* Green function of the cluster's physical sites for one spin (0 = up, 1 = down) from the irrep's
 * ground state (Sec. 4.6): the site operators are symmetrized (c+_rho = sum_a M_rho,a c+_a, the
 * projections of every site orbit onto every irrep beta; M orthogonal, or unitary for complex
 * characters), c+_rho Omega lands in the N + 1 sector of the irrep alpha + beta and c_rho Omega in
 * the N - 1 sector of alpha - beta (exponents modulo the orders; the same irrep for involutions),
 * where continued fractions (Eq. jacobi; off-diagonal pairs as in Sec. 4.3, with the pair
 * phi_rho + i phi_sigma added when characters are complex) run on the stored matrices until they
 * change by less than the cluster's ED_OPT_GF_TOL (0: 1e-12) at two successive checks, and
 * G_ab = sum M_rho,a conj(M_sigma,b) G_rho,sigma.  z_k = omega[k] + i eta (ED_AXIS_REAL) or
 * i omega[k] (ED_AXIS_MATSUBARA).  G_out: host, interleaved complex128 [n_freq][n_sites][n_sites].
 * The group must map cluster sites to cluster sites (else ED_ERR_INVALID).  ED_ERR_STATE before
 * ed_sym_ground_state.  G is the
 * ground-state G when the irrep holds the sector's (non-degenerate) ground state.  Synchronous. */
ed_status ed_sym_green(ed_sym* s, const double* omega, int n_freq, double eta, int axis, int spin, double* G_out);

void ed_sym_destroy(ed_sym* s);

/* ---- measurement of the library's own kernels (no counterpart in the paper) --------------- */

/* Kernel families. */
enum {
  ED_K_TABLES = 0,        /* basis, rank and hopping-table construction */
  ED_K_HPSI = 1,          /* standalone H.psi (ed_hpsi, ground-state polish) */
  ED_K_LANCZOS_STEP = 2,  /* fused H.psi + Lanczos epilogue: algorithmic bytes 3 x d x elem */
  ED_K_LANCZOS_NEXT = 3,  /* v_{n+1} = (w - a v_n) / b */
  ED_K_TRIDIAG = 4,
  ED_K_VECTOR = 5,        /* reductions, scaling, start vectors */
  ED_K_APPLY_COP = 6,     /* c+ / c applied to the ground state */
  ED_K_GF_EVAL = 7,       /* Green-function evaluation and assembly on the grid */
  ED_K_BAND = 8,          /* band-Lanczos orthogonalization */
  ED_K_BATCH = 9,         /* persistent kernels of the batched form */
  ED_K_LATTICE = 10,      /* CPT and CDMFT kernels (batched small-matrix inversions, distance) */
  ED_K_COUNT = 11
};

/* Turns per-family timing on (1) or off (0) and clears the totals.  While on, each launch of a
 * family is bracketed by CUDA events on the stream it is launched on. */
ed_status ed_profile_enable(int on);

/* Totals since the last ed_profile_enable: launches, summed event time (ms) and summed
 * algorithmic bytes (the bytes the method must move; 0 for families without a byte model).
 * Synchronizes with the recorded events.  Any output may be NULL. */
ed_status ed_profile_read(int kernel, int64_t* launches, double* total_ms, double* alg_bytes);

/* Name of a kernel family ("lanczos_step", ...). */
const char* ed_profile_kernel_name(int kernel);

/* Number of kernels this library has launched in the process so far (always counted). */
int64_t ed_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* ED_H */
