"""Thin ctypes binding of libed (include/ed.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  All computation happens in
libed.so's CUDA kernels; there is no CPU path.  If the library has not been built the first
call raises ``RuntimeError`` (build it with ``python -m paper_2305_18643_gb300.build``).
Device arrays are passed as integer device pointers (e.g. ``torch.Tensor.data_ptr()``).
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

ED_OK, ED_PENDING, ED_WARN_DEGENERATE, ED_WARN_NOT_CONVERGED = 0, 1, 2, 3
ED_ERR_INVALID, ED_ERR_OOM, ED_ERR_CUDA, ED_ERR_TOO_LARGE = -1, -2, -3, -5
ED_ERR_TIMEOUT, ED_ERR_STATE, ED_ERR_NOT_FOUND, ED_ERR_CANCELLED = -6, -7, -8, -9
ED_FP64, ED_FP32 = 0, 1
ED_GF_CF, ED_GF_BAND = 0, 1
ED_AXIS_REAL, ED_AXIS_MATSUBARA = 0, 1

_dp = C.POINTER(C.c_double)


class ed_cluster_desc(C.Structure):
    _fields_ = [("n_sites", C.c_int), ("n_bath", C.c_int), ("t", _dp), ("U", _dp), ("mu", C.c_double),
                ("eps", _dp), ("theta", _dp), ("n_up", C.c_int), ("n_dn", C.c_int), ("precision", C.c_int),
                ("gf_method", C.c_int), ("seed", C.c_uint64), ("tol", C.c_double), ("max_iter", C.c_int)]


class EDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libed status %d: %s" % (status, msg))
        self.status = status


_lib = None


def library_path():
    return _build.LIB


def lib():
    """The loaded libed.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libed.so not found at %s; build it with `python -m paper_2305_18643_gb300.build`" % path)
        L = C.CDLL(path)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
        sig = {
            "ed_cluster_create": (i32, [C.POINTER(ed_cluster_desc), C.POINTER(vp)]),
            "ed_cluster_destroy": (None, [vp]),
            "ed_ground_state": (i32, [vp, _dp, _dp, C.POINTER(i32)]),
            "ed_ground_vector": (i32, [vp, vp, i32]),
            "ed_green": (i32, [vp, _dp, i32, C.c_double, i32, i32, vp, i32]),
            "ed_green_stats": (i32, [vp, C.POINTER(i64), C.POINTER(i32)]),
            "ed_low_states": (i32, [vp, i32, _dp, _dp, C.POINTER(i32)]),
            "ed_gram_f32": (i32, [vp, i32, vp, i32, i64, i64, i32, _dp]),
            "ed_sector_dims": (i32, [vp, i32, i32, C.POINTER(i64), C.POINTER(i64)]),
            "ed_basis": (i32, [i32, i32, vp, i64, C.POINTER(i64)]),
            "ed_hop_table": (i32, [vp, i32, vp, vp, vp, i64, C.POINTER(i64), C.POINTER(i32)]),
            "ed_hpsi": (i32, [vp, i32, i32, i32, vp, vp, i64, vp]),
            "ed_last_error": (C.c_char_p, []),
            "ed_profile_enable": (i32, [i32]),
            "ed_profile_read": (i32, [i32, C.POINTER(i64), _dp, _dp]),
            "ed_profile_kernel_name": (C.c_char_p, [i32]),
            "ed_launch_count": (i64, []),
            "ed_set_option": (i32, [vp, i32, C.c_double]),
            "ed_hpsi_dots_static": (i32, [vp, i32, vp, vp, i64, vp, vp]),
            "ed_batch_solve": (i32, [C.POINTER(ed_cluster_desc), i32, i32, _dp, i32, C.c_double, i32, i32, _dp, _dp,
                                     C.POINTER(i32), C.POINTER(i32), C.POINTER(i64), vp, i32]),
        }
        sig.update(_server_sigs)
        sig.update(_lattice_sigs)
        sig.update(_sym_sigs)
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def ed_last_error():
    return lib().ed_last_error().decode()


def _check(st):
    if st < 0:
        raise EDError(st, ed_last_error())
    return st


def _arr(a, n):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())
    if a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def ed_cluster_create(cluster, precision=ED_FP64, gf_method=ED_GF_CF, seed=0, tol=0.0, max_iter=0):
    """Create a cluster handle from a dict with t, U, mu, eps, theta, n_up, n_dn."""
    ns = int(np.asarray(cluster["t"]).shape[0])
    eps = np.asarray(cluster.get("eps", np.zeros(0)), dtype=np.float64).ravel()
    nb = int(eps.size)
    keep = [_arr(cluster["t"], ns * ns), _arr(np.broadcast_to(np.asarray(cluster["U"], float), (ns,)), ns),
            _arr(eps, nb) if nb else None,
            _arr(cluster.get("theta", np.zeros((ns, 0))), ns * nb) if nb else None]
    ptr = [k.ctypes.data_as(_dp) if k is not None else None for k in keep]
    d = ed_cluster_desc(ns, nb, ptr[0], ptr[1], float(cluster["mu"]), ptr[2], ptr[3], int(cluster["n_up"]),
                        int(cluster["n_dn"]), int(precision), int(gf_method), int(seed) & (2 ** 64 - 1),
                        float(tol), int(max_iter))
    h = C.c_void_p()
    _check(lib().ed_cluster_create(C.byref(d), C.byref(h)))
    return h


def ed_cluster_destroy(h):
    if h:
        lib().ed_cluster_destroy(h)


def ed_ground_state(h):
    """Returns (status, E0, residual, iters)."""
    E0, res, it = C.c_double(), C.c_double(), C.c_int()
    st = _check(lib().ed_ground_state(h, C.byref(E0), C.byref(res), C.byref(it)))
    return st, E0.value, res.value, it.value


def ed_sector_dims(h, n_up, n_dn):
    du, dd = C.c_int64(), C.c_int64()
    _check(lib().ed_sector_dims(h, int(n_up), int(n_dn), C.byref(du), C.byref(dd)))
    return du.value, dd.value


def ed_ground_vector(h, n_up, n_dn, out_ptr=None):
    """Ground state psi[u, d] (FP64).  With out_ptr (device pointer) it is copied there."""
    if out_ptr is not None:
        _check(lib().ed_ground_vector(h, C.c_void_p(out_ptr), 1))
        return None
    du, dd = ed_sector_dims(h, n_up, n_dn)
    out = np.empty((du, dd))
    _check(lib().ed_ground_vector(h, out.ctypes.data_as(C.c_void_p), 0))
    return out


def ed_green(h, omega, eta, n_sites, axis=ED_AXIS_REAL, spin=0, out_ptr=None):
    """G[nz, n_sites, n_sites] complex128 (host), or written to device pointer out_ptr.
    Returns (status, G or None)."""
    om = _arr(omega, np.asarray(omega).size)
    if out_ptr is not None:
        st = _check(lib().ed_green(h, om.ctypes.data_as(_dp), om.size, float(eta), int(axis), int(spin),
                                   C.c_void_p(out_ptr), 1))
        return st, None
    G = np.empty((om.size, n_sites, n_sites), dtype=np.complex128)
    st = _check(lib().ed_green(h, om.ctypes.data_as(_dp), om.size, float(eta), int(axis), int(spin),
                               G.ctypes.data_as(C.c_void_p), 0))
    return st, G


ED_OPT_BAND_MAX_DIM, ED_OPT_CF_MAX_STEPS, ED_OPT_GF_TOL, ED_OPT_TWO_PASS_MIN_BYTES = 1, 2, 3, 4
ED_OPT_DAVIDSON_STATES, ED_OPT_TEMPERATURE, ED_OPT_TENSOR_GRAM = 5, 6, 7


def ed_gram_f32(x_ptr, nx, y_ptr, ny, vstride, n, method):
    """G[nx, ny] (FP64, host) = X Y^T over n elements of FP32 device vectors vstride apart;
    method 1 = tensor cores, 0 = CUDA cores."""
    G = np.empty((nx, ny))
    _check(lib().ed_gram_f32(C.c_void_p(x_ptr), int(nx), C.c_void_p(y_ptr), int(ny), int(vstride), int(n),
                             int(method), G.ctypes.data_as(_dp)))
    return G


def ed_low_states(h, capacity=16):
    """(energies, mixed-state weights) of the states behind the cluster's Green function."""
    E, wt, n = np.zeros(capacity), np.zeros(capacity), C.c_int()
    _check(lib().ed_low_states(h, int(capacity), E.ctypes.data_as(_dp), wt.ctypes.data_as(_dp), C.byref(n)))
    k = min(n.value, capacity)
    return E[:k], wt[:k]


def ed_set_option(h, option, value):
    _check(lib().ed_set_option(h, int(option), float(value)))


def ed_green_stats(h):
    tot, mx = C.c_int64(), C.c_int()
    _check(lib().ed_green_stats(h, C.byref(tot), C.byref(mx)))
    return tot.value, mx.value


def ed_basis(L, N):
    dim = C.c_int64()
    lib().ed_basis(int(L), int(N), None, 0, C.byref(dim))
    out = np.empty(max(dim.value, 1), dtype=np.uint32)
    _check(lib().ed_basis(int(L), int(N), out.ctypes.data_as(C.c_void_p), out.size, C.byref(dim)))
    return out[: dim.value]


def ed_hop_table(h, N, L):
    """(row_ptr int32[d+1], entries uint32[nnz], values float64[nvals]) of one spin with N particles."""
    nnz, nv = C.c_int64(), C.c_int()
    lib().ed_hop_table(h, int(N), None, None, None, 0, C.byref(nnz), C.byref(nv))
    import math
    d = math.comb(L, N)
    ptr = np.empty(d + 1, dtype=np.int32)
    ent = np.empty(max(nnz.value, 1), dtype=np.uint32)
    vals = np.empty(128, dtype=np.float64)
    _check(lib().ed_hop_table(h, int(N), ptr.ctypes.data_as(C.c_void_p), ent.ctypes.data_as(C.c_void_p),
                              vals.ctypes.data_as(C.c_void_p), ent.size, C.byref(nnz), C.byref(nv)))
    return ptr, ent[: nnz.value], vals[: nv.value]


def ed_hpsi(h, n_up, n_dn, dtype, x_ptr, y_ptr, ld=0, stream=0):
    """y = H x on device pointers (FP64 or FP32), asynchronous on `stream` (0 = the CUDA default stream)."""
    _check(lib().ed_hpsi(h, int(n_up), int(n_dn), int(dtype), C.c_void_p(x_ptr), C.c_void_p(y_ptr), int(ld),
                         C.c_void_p(stream) if stream else None))


ED_K_TABLES, ED_K_HPSI, ED_K_LANCZOS_STEP, ED_K_LANCZOS_NEXT, ED_K_TRIDIAG = 0, 1, 2, 3, 4
ED_K_VECTOR, ED_K_APPLY_COP, ED_K_GF_EVAL, ED_K_BAND, ED_K_BATCH, ED_K_LATTICE, ED_K_COUNT = 5, 6, 7, 8, 9, 10, 11


def ed_profile_enable(on):
    _check(lib().ed_profile_enable(1 if on else 0))


def ed_profile_read(kernel):
    """(launches, total_ms, algorithmic_bytes) of one kernel family since ed_profile_enable."""
    n, ms, by = C.c_int64(), C.c_double(), C.c_double()
    _check(lib().ed_profile_read(int(kernel), C.byref(n), C.byref(ms), C.byref(by)))
    return n.value, ms.value, by.value


def ed_profile_kernel_name(kernel):
    return lib().ed_profile_kernel_name(int(kernel)).decode()


def ed_launch_count():
    return int(lib().ed_launch_count())


def ed_hpsi_dots_static(h, dtype, x_ptr, y_ptr, out3_ptr, ld=0, stream=0):
    """y = H x in the cluster's own sector and <x,y>, <y,y>, <x,x> into out3 (device FP64), using
    the library's fixed scratch instead of device allocations; asynchronous on `stream`."""
    _check(lib().ed_hpsi_dots_static(h, int(dtype), C.c_void_p(x_ptr), C.c_void_p(y_ptr), int(ld),
                                     C.c_void_p(out3_ptr), C.c_void_p(stream) if stream else None))


def _desc_array(clusters, seed=0, tol=0.0):
    keep, descs = [], (ed_cluster_desc * max(len(clusters), 1))()
    for k, cl in enumerate(clusters):
        ns = int(np.asarray(cl["t"]).shape[0])
        eps = np.asarray(cl.get("eps", np.zeros(0)), dtype=np.float64).ravel()
        nb = int(eps.size)
        arrs = [_arr(cl["t"], ns * ns), _arr(np.broadcast_to(np.asarray(cl["U"], float), (ns,)), ns),
                _arr(eps, nb) if nb else None, _arr(cl.get("theta", np.zeros((ns, 0))), ns * nb) if nb else None]
        keep.append(arrs)
        ptr = [a.ctypes.data_as(_dp) if a is not None else None for a in arrs]
        descs[k] = ed_cluster_desc(ns, nb, ptr[0], ptr[1], float(cl["mu"]), ptr[2], ptr[3], int(cl["n_up"]),
                                   int(cl["n_dn"]), 0, 0, (int(seed) + k) & (2 ** 64 - 1), float(tol), 0)
    return descs, keep


def ed_batch_solve(clusters, precision=ED_FP64, omega=None, eta=0.05, axis=ED_AXIS_REAL, seed=0, tol=0.0,
                   out_ptr=None, cf_max_levels=0):
    """Solve many clusters together.  Returns (E0, residual, status, iters, G) where G is a list of
    complex128 arrays [2, n_freq, n_sites, n_sites] (None when omega is None or out_ptr is given).
    cf_max_levels caps every continued fraction (<= 0: the library's preset of 20000 levels, so
    that runs end on convergence on the grid); the
    continued-fraction levels of each cluster are left in ed_batch_solve.gf_steps."""
    n = len(clusters)
    descs, keep = _desc_array(clusters, seed, tol)
    om = _arr(omega, np.asarray(omega).size) if omega is not None else np.zeros(0)
    nf = om.size
    E0, res = np.zeros(max(n, 1)), np.zeros(max(n, 1))
    st, it = np.zeros(max(n, 1), dtype=np.int32), np.zeros(max(n, 1), dtype=np.int32)
    gs = np.zeros(max(n, 1), dtype=np.int64)
    sizes = [2 * nf * int(np.asarray(cl["t"]).shape[0]) ** 2 for cl in clusters]
    G = None
    if out_ptr is not None:
        gptr, dev = C.c_void_p(out_ptr), 1
    else:
        G = np.zeros(max(sum(sizes), 1), dtype=np.complex128)
        gptr, dev = G.ctypes.data_as(C.c_void_p), 0
    _check(lib().ed_batch_solve(descs, n, int(precision), om.ctypes.data_as(_dp), nf, float(eta), int(axis),
                                int(cf_max_levels), E0.ctypes.data_as(_dp), res.ctypes.data_as(_dp),
                                st.ctypes.data_as(C.POINTER(C.c_int)), it.ctypes.data_as(C.POINTER(C.c_int)),
                                gs.ctypes.data_as(C.POINTER(C.c_int64)), gptr if nf else None, dev))
    Gs = None
    if G is not None and nf:
        Gs, o = [], 0
        for cl, sz in zip(clusters, sizes):
            ns = int(np.asarray(cl["t"]).shape[0])
            Gs.append(G[o:o + sz].reshape(2, nf, ns, ns))
            o += sz
    ed_batch_solve.gf_steps = gs[:n]
    return E0[:n], res[:n], st[:n], it[:n], Gs


class Cluster:
    """Owning wrapper of a cluster handle (context manager)."""

    def __init__(self, cluster, **kw):
        self.desc = cluster
        self.h = ed_cluster_create(cluster, **kw)
        self.ns = int(np.asarray(cluster["t"]).shape[0])
        self.n_up, self.n_dn = int(cluster["n_up"]), int(cluster["n_dn"])

    def close(self):
        if self.h:
            ed_cluster_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ground_state(self):
        return ed_ground_state(self.h)

    def ground_vector(self):
        return ed_ground_vector(self.h, self.n_up, self.n_dn)

    def green(self, omega, eta, axis=ED_AXIS_REAL, spin=0):
        return ed_green(self.h, omega, eta, self.ns, axis, spin)[1]


# ----------------------------------------------------------------------------- served form
class ed_request_opts(C.Structure):
    _fields_ = [("omega", _dp), ("n_freq", C.c_int), ("eta", C.c_double), ("axis", C.c_int),
                ("cf_max_levels", C.c_int), ("G_out", _dp)]


class ed_result(C.Structure):
    _fields_ = [("status", C.c_int), ("path", C.c_int), ("E0", C.c_double), ("residual", C.c_double),
                ("iters", C.c_int), ("batch_size", C.c_int), ("gf_steps", C.c_int64), ("queued_ms", C.c_double),
                ("run_ms", C.c_double), ("latency_ms", C.c_double), ("device_bytes", C.c_size_t)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ed_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("cancelled", C.c_int64), ("queued", C.c_int), ("running", C.c_int), ("max_running", C.c_int),
                ("reserved_bytes", C.c_size_t), ("peak_reserved_bytes", C.c_size_t),
                ("batched_solves", C.c_int64)]


ED_SRV_BATCH_MAX_DIM, ED_SRV_BATCH_MAX_REQUESTS, ED_SRV_GF_BUDGET_FRACTION, ED_SRV_PAUSE = 1, 2, 3, 4

_server_sigs = {
    "ed_server_create": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(C.c_void_p)]),
    "ed_server_destroy": (None, [C.c_void_p]),
    "ed_server_set_option": (C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    "ed_request_bytes": (C.c_int, [C.POINTER(ed_cluster_desc), C.POINTER(ed_request_opts), C.c_size_t,
                                   C.POINTER(C.c_size_t)]),
    "ed_submit": (C.c_int, [C.c_void_p, C.POINTER(ed_cluster_desc), C.POINTER(ed_request_opts),
                            C.POINTER(C.c_uint64)]),
    "ed_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(ed_result)]),
    "ed_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_double, C.POINTER(ed_result)]),
    "ed_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "ed_server_inject_failure": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int]),
    "ed_server_stats_get": (C.c_int, [C.c_void_p, C.POINTER(ed_server_stats)]),
}


def _slib():
    return lib()


def _one_desc(cluster, precision, gf_method, seed, tol, max_iter=0):
    descs, keep = _desc_array([cluster], seed, tol)
    d = descs[0]
    d.precision, d.gf_method, d.max_iter = int(precision), int(gf_method), int(max_iter)
    return d, keep


def ed_request_bytes(cluster, n_freq=0, precision=ED_FP64, gf_method=ED_GF_CF, cf_max_levels=0, gf_budget=0):
    """Device bytes of one request on the single-cluster path (host-side closed forms only)."""
    d, keep = _one_desc(cluster, precision, gf_method, 0, 0.0)
    om = np.zeros(max(n_freq, 1))
    G = np.zeros(1, dtype=np.complex128)
    o = ed_request_opts(om.ctypes.data_as(_dp), int(n_freq), 0.05, ED_AXIS_REAL, int(cf_max_levels),
                        G.ctypes.data_as(_dp))
    out = C.c_size_t()
    _check(_slib().ed_request_bytes(C.byref(d), C.byref(o), int(gf_budget), C.byref(out)))
    return out.value


class Server:
    """ed_server_* with Python-owned request buffers.  submit() returns the request id; poll() /
    wait() return (ed_result dict, G [2, n_freq, n_sites, n_sites] or None) once it is done."""

    def __init__(self, mem_budget_bytes, max_slots=4, **options):
        h = C.c_void_p()
        _check(_slib().ed_server_create(int(mem_budget_bytes), int(max_slots), C.byref(h)))
        self.h = h
        self._live = {}
        names = {"batch_max_dim": ED_SRV_BATCH_MAX_DIM, "batch_max_requests": ED_SRV_BATCH_MAX_REQUESTS,
                 "gf_budget_fraction": ED_SRV_GF_BUDGET_FRACTION, "paused": ED_SRV_PAUSE}
        for k, v in options.items():
            _check(_slib().ed_server_set_option(self.h, names[k], float(v)))

    def submit(self, cluster, omega=None, eta=0.05, axis=ED_AXIS_REAL, precision=ED_FP64, gf_method=ED_GF_CF,
               seed=0, tol=0.0, cf_max_levels=0, max_iter=0):
        d, keep = _one_desc(cluster, precision, gf_method, seed, tol, max_iter)
        ns = int(np.asarray(cluster["t"]).shape[0])
        om = _arr(omega, np.asarray(omega).size) if omega is not None else np.zeros(0)
        nf = om.size
        G = np.zeros((2, nf, ns, ns), dtype=np.complex128) if nf else None
        o = ed_request_opts(om.ctypes.data_as(_dp) if nf else None, nf, float(eta), int(axis), int(cf_max_levels),
                            G.ctypes.data_as(_dp) if nf else None)
        rid = C.c_uint64()
        _check(_slib().ed_submit(self.h, C.byref(d), C.byref(o), C.byref(rid)))
        self._live[rid.value] = (G, om, keep)
        return rid.value

    def _done(self, rid, st, res):
        if st == ED_PENDING:
            return None
        G = self._live.pop(rid)[0]
        out = res.as_dict()
        if out["status"] < 0:
            out["error"] = ed_last_error()  # the request's own message (set by the collecting call)
        return out, G

    def poll(self, rid):
        res = ed_result()
        st = _check(_slib().ed_poll(self.h, int(rid), C.byref(res)))
        return self._done(rid, st, res)

    def wait(self, rid, timeout_s=600.0):
        res = ed_result()
        st = _check(_slib().ed_wait(self.h, int(rid), float(timeout_s), C.byref(res)))
        return self._done(rid, st, res)

    def pause(self, on=True):
        """Stop (on) or resume (off) admission; submitted requests stay queued while paused."""
        _check(_slib().ed_server_set_option(self.h, ED_SRV_PAUSE, 1.0 if on else 0.0))

    def cancel(self, rid):
        _check(_slib().ed_cancel(self.h, int(rid)))

    def inject_failure(self, rid, status=ED_ERR_CUDA):
        _check(_slib().ed_server_inject_failure(self.h, int(rid), int(status)))

    def stats(self):
        s = ed_server_stats()
        _check(_slib().ed_server_stats_get(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if self.h:
            _slib().ed_server_destroy(self.h)
            self.h = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- lattice steps (CPT, CDMFT)
class ed_superlattice(C.Structure):
    _fields_ = [("n_sites", C.c_int), ("dim", C.c_int), ("pos", _dp), ("E", _dp), ("n_bonds", C.c_int),
                ("bonds", C.POINTER(C.c_int)), ("bond_t", _dp)]


ED_CPT_MATRIX, ED_CPT_PERIODIZED, ED_CPT_AVERAGE = 0, 1, 2

_lattice_sigs = {
    "ed_hybridization": (C.c_int, [C.c_int, C.c_int, _dp, _dp, _dp, C.c_int, C.c_void_p, C.c_int]),
    "ed_cpt_green": (C.c_int, [C.POINTER(ed_superlattice), C.c_void_p, C.c_void_p, C.c_int, _dp, C.c_int, C.c_int,
                               C.c_void_p, C.c_int]),
    "ed_cdmft_target": (C.c_int, [C.POINTER(ed_superlattice), C.c_void_p, C.c_void_p, C.c_int, _dp, C.c_int,
                                  C.c_void_p, C.c_int]),
    "ed_cdmft_distance": (C.c_int, [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, C.c_int, _dp, _dp, _dp, _dp]),
    "ed_cdmft_fit": (C.c_int, [C.c_int, C.c_int, _dp, _dp, C.POINTER(C.c_ubyte), _dp, C.c_int, _dp, _dp,
                               C.c_double, C.c_int, _dp, C.POINTER(C.c_int)]),
}


def _c128(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if shape is not None and a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


def _superlattice(lat):
    """ed_superlattice from a dict {"t_c", "pos", "E", "bonds": [(i, j, n, t)]}; returns
    (struct, arrays kept alive)."""
    pos = np.ascontiguousarray(np.asarray(lat["pos"], dtype=np.float64))
    L, D = pos.shape
    E = np.ascontiguousarray(np.asarray(lat["E"], dtype=np.float64).reshape(D, D))
    nb = len(lat["bonds"])
    bonds = np.zeros((max(nb, 1), 2 + D), dtype=np.int32)
    bt = np.zeros(max(nb, 1))
    for q, (i, j, n, t) in enumerate(lat["bonds"]):
        bonds[q, 0], bonds[q, 1] = i, j
        bonds[q, 2:] = np.atleast_1d(n)
        bt[q] = t
    s = ed_superlattice(L, D, pos.ctypes.data_as(_dp), E.ctypes.data_as(_dp), nb,
                        bonds.ctypes.data_as(C.POINTER(C.c_int)), bt.ctypes.data_as(_dp))
    return s, (pos, E, bonds, bt)


def ed_hybridization(theta, eps, z):
    """Gamma[nz, L, L] (Eq. hybridization) for theta (L, nb), eps (nb,), complex z (nz,)."""
    theta = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    L, nb = theta.shape
    eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).ravel())
    z = _c128(z).ravel()
    out = np.empty((z.size, L, L), dtype=np.complex128)
    _check(lib().ed_hybridization(L, nb, eps.ctypes.data_as(_dp), theta.ctypes.data_as(_dp),
                                  z.view(np.float64).ctypes.data_as(_dp), z.size, out.ctypes.data_as(C.c_void_p), 0))
    return out


def ed_cpt_green(lat, Gc, kt, mode=ED_CPT_MATRIX, Gamma=None):
    """CPT from the cluster Green function Gc[nz, L, L] on wave vectors kt[nk, D] (host arrays).
    Returns G[nk, nz, L, L] (ED_CPT_MATRIX), G_per[nk, nz] (ED_CPT_PERIODIZED) or G_bar[nz, L, L]
    (ED_CPT_AVERAGE)."""
    s, keep = _superlattice(lat)
    Gc = _c128(Gc)
    nz, L = Gc.shape[0], Gc.shape[1]
    kt = np.ascontiguousarray(np.asarray(kt, dtype=np.float64).reshape(-1, s.dim))
    nk = kt.shape[0]
    Gm = _c128(Gamma) if Gamma is not None else None
    shape = {ED_CPT_MATRIX: (nk, nz, L, L), ED_CPT_PERIODIZED: (nk, nz), ED_CPT_AVERAGE: (nz, L, L)}[mode]
    out = np.empty(shape, dtype=np.complex128)
    _check(lib().ed_cpt_green(C.byref(s), Gc.ctypes.data_as(C.c_void_p),
                              Gm.ctypes.data_as(C.c_void_p) if Gm is not None else None, nz,
                              kt.ctypes.data_as(_dp), nk, int(mode), out.ctypes.data_as(C.c_void_p), 0))
    return out


def ed_cdmft_target(lat, Gc, kt, Gamma=None):
    """A[nz, L, L] = Gamma + Gc^-1 - G_bar^-1 (CDMFT steps 3-4) on the reduced-zone grid kt."""
    s, keep = _superlattice(lat)
    Gc = _c128(Gc)
    nz, L = Gc.shape[0], Gc.shape[1]
    kt = np.ascontiguousarray(np.asarray(kt, dtype=np.float64).reshape(-1, s.dim))
    Gm = _c128(Gamma) if Gamma is not None else None
    out = np.empty((nz, L, L), dtype=np.complex128)
    _check(lib().ed_cdmft_target(C.byref(s), Gc.ctypes.data_as(C.c_void_p),
                                 Gm.ctypes.data_as(C.c_void_p) if Gm is not None else None, nz,
                                 kt.ctypes.data_as(_dp), kt.shape[0], out.ctypes.data_as(C.c_void_p), 0))
    return out


def ed_cdmft_distance(theta, eps, z, weights, A, grad=False):
    """Distances (and gradients) of n_cand trial baths: theta (n_cand, L, nb), eps (n_cand, nb).
    Returns d[n_cand] (and grad[n_cand, nb + L nb])."""
    theta = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    if theta.ndim == 2:
        theta = theta[None]
    nc, L, nb = theta.shape
    eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(nc, nb))
    z = _c128(z).ravel()
    W = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).ravel())
    A = _c128(A)
    d = np.empty(nc)
    g = np.empty((nc, nb + L * nb)) if grad else None
    _check(lib().ed_cdmft_distance(L, nb, nc, eps.ctypes.data_as(_dp), theta.ctypes.data_as(_dp),
                                   z.view(np.float64).ctypes.data_as(_dp), z.size, W.ctypes.data_as(_dp),
                                   A.view(np.float64).ctypes.data_as(_dp), d.ctypes.data_as(_dp),
                                   g.ctypes.data_as(_dp) if grad else None))
    return (d, g) if grad else d


def ed_cdmft_fit(theta, eps, z, weights, A, theta_free=None, gtol=0.0, max_iter=0):
    """Bath fit (CDMFT step 4) from the starting bath (theta (L, nb), eps (nb,)); returns
    (theta, eps, d, iterations)."""
    theta = np.array(theta, dtype=np.float64, order="C")
    L, nb = theta.shape
    eps = np.array(eps, dtype=np.float64).ravel().copy()
    z = _c128(z).ravel()
    W = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).ravel())
    A = _c128(A)
    free = None
    if theta_free is not None:
        free = np.ascontiguousarray(np.asarray(theta_free, dtype=np.uint8).reshape(L, nb))
    d, it = C.c_double(), C.c_int()
    _check(lib().ed_cdmft_fit(L, nb, eps.ctypes.data_as(_dp), theta.ctypes.data_as(_dp),
                              free.ctypes.data_as(C.POINTER(C.c_ubyte)) if free is not None else None,
                              z.view(np.float64).ctypes.data_as(_dp), z.size, W.ctypes.data_as(_dp),
                              A.view(np.float64).ctypes.data_as(_dp), float(gtol), int(max_iter), C.byref(d),
                              C.byref(it)))
    return theta, eps, d.value, it.value

# ---- cluster symmetries (Sec. 4.5) -------------------------------------------------------------
_ip = C.POINTER(C.c_int)
_sym_sigs = {
    "ed_sym_create": (C.c_int, [C.c_void_p, C.c_int, _ip, _ip, C.POINTER(C.c_void_p)]),
    "ed_sym_create_abelian": (C.c_int, [C.c_void_p, C.c_int, _ip, _ip, _ip, C.POINTER(C.c_void_p)]),
    "ed_sym_is_complex": (C.c_int, [C.c_void_p, _ip]),
    "ed_sym_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "ed_sym_basis": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "ed_sym_matrix": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ed_sym_hpsi": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "ed_sym_ground_state": (C.c_int, [C.c_void_p, _dp, _dp, C.POINTER(C.c_int)]),
    "ed_sym_ground_vector": (C.c_int, [C.c_void_p, _dp]),
    "ed_sym_green": (C.c_int, [C.c_void_p, _dp, C.c_int, C.c_double, C.c_int, C.c_int, _dp]),
    "ed_sym_destroy": (None, [C.c_void_p]),
}


def ed_sym_create(h, perms, signs):
    """Handle of one irrep (generator signs `signs`, +-1) of the group generated by the orbital
    involutions `perms` (n_gen x L images), for the cluster h's sector."""
    P = np.ascontiguousarray(np.asarray(perms, dtype=np.int32).reshape(len(signs), -1))
    sg = np.ascontiguousarray(np.asarray(signs, dtype=np.int32))
    out = C.c_void_p()
    _check(lib().ed_sym_create(h, int(len(sg)), P.ctypes.data_as(_ip), sg.ctypes.data_as(_ip), C.byref(out)))
    return out


def ed_sym_create_abelian(h, perms, orders, irrep):
    """Handle of the irrep with exponents `irrep` (0 <= m_k < orders[k]) of the Abelian group
    generated by the orbital permutations `perms` of the given orders."""
    P = np.ascontiguousarray(np.asarray(perms, dtype=np.int32).reshape(len(orders), -1))
    od = np.ascontiguousarray(np.asarray(orders, dtype=np.int32))
    ir = np.ascontiguousarray(np.asarray(irrep, dtype=np.int32))
    out = C.c_void_p()
    _check(lib().ed_sym_create_abelian(h, int(len(od)), P.ctypes.data_as(_ip), od.ctypes.data_as(_ip),
                                       ir.ctypes.data_as(_ip), C.byref(out)))
    return out


def ed_sym_is_complex(s):
    v = C.c_int()
    _check(lib().ed_sym_is_complex(s, C.byref(v)))
    return bool(v.value)


def ed_sym_info(s):
    """(dimension, stored entries) of the symmetrized sector."""
    d, z = C.c_int64(), C.c_int64()
    _check(lib().ed_sym_info(s, C.byref(d), C.byref(z)))
    return d.value, z.value


def ed_sym_basis(s):
    """(keys b_up 2^L + b_dn, stabilizer sizes) of the representatives, ascending keys."""
    d, _ = ed_sym_info(s)
    keys = np.zeros(d, dtype=np.uint64)
    st = np.zeros(d, dtype=np.uint8)
    _check(lib().ed_sym_basis(s, keys.ctypes.data, st.ctypes.data))
    return keys, st


def ed_sym_matrix(s):
    """(rowptr, col, val) of the stored matrix (host copies)."""
    d, z = ed_sym_info(s)
    rp = np.zeros(d + 1, dtype=np.int64)
    col = np.zeros(z, dtype=np.int32)
    val = np.zeros(z, dtype=np.complex128 if ed_sym_is_complex(s) else np.float64)
    _check(lib().ed_sym_matrix(s, rp.ctypes.data, col.ctypes.data, val.ctypes.data))
    return rp, col, val


def ed_sym_hpsi(s, x_ptr, y_ptr):
    """y = H x in the symmetrized basis (device pointers)."""
    _check(lib().ed_sym_hpsi(s, C.c_void_p(x_ptr), C.c_void_p(y_ptr)))


def ed_sym_ground_state(s):
    """(E0, residual, iterations, status)."""
    E, r, it = C.c_double(), C.c_double(), C.c_int()
    st = _check(lib().ed_sym_ground_state(s, C.byref(E), C.byref(r), C.byref(it)))
    return E.value, r.value, it.value, st


def ed_sym_ground_vector(s):
    d, _ = ed_sym_info(s)
    v = np.zeros(d, dtype=np.complex128 if ed_sym_is_complex(s) else np.float64)
    _check(lib().ed_sym_ground_vector(s, v.ctypes.data_as(_dp)))
    return v


def ed_sym_green(s, omega, n_sites, eta=0.05, axis=ED_AXIS_REAL, spin=0):
    """G[n_freq, n_sites, n_sites] (complex, host) from the irrep's ground state (symmetrized operators)."""
    om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
    G = np.zeros((len(om), n_sites, n_sites), dtype=np.complex128)
    _check(lib().ed_sym_green(s, om.ctypes.data_as(_dp), len(om), float(eta), int(axis), int(spin),
                              G.ctypes.data_as(_dp)))
    return G


def ed_sym_destroy(s):
    lib().ed_sym_destroy(s)
