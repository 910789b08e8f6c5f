"""Memoized oracle calls for the GPU tests (test infrastructure, not part of the oracle).

Many GPU tests compare with the oracle's exact Green function of the same cluster, sector and
spin, each time on a different frequency grid, and with the ground state of the same large
sector.  The exact Green function diagonalizes the N +- 1 sectors in full, so repeating it is
the main cost of the GPU suite.  These wrappers keep, for the session, the poles and residues
(Q, w) that the oracle's green_exact returns, and evaluate the oracle's own Lehmann sum
(lehmann_green) at the frequencies asked; ground states are kept the same way.  Nothing of the
oracle's arithmetic changes: a cached call returns what the uncached one would, up to the
rounding order of the dense diagonalizations, which run on every host core here.  The CPU pin and
planted-mistake tests call the oracle directly, never these wrappers.
"""

import contextlib
import ctypes
import glob
import hashlib
import os

import numpy as np

import oracle as O

_green = {}
_ground = {}
_ops = {}


def _openblas_threads_api():
    """(set, get) of numpy's bundled OpenBLAS thread count, or None where it cannot be found."""
    libdir = os.path.join(os.path.dirname(os.path.dirname(np.__file__)), "numpy.libs")
    for path in glob.glob(os.path.join(libdir, "*openblas*")):
        try:
            lib = ctypes.CDLL(path)
        except OSError:
            continue
        for s, g in (("scipy_openblas_set_num_threads64_", "scipy_openblas_get_num_threads64_"),
                     ("scipy_openblas_set_num_threads", "scipy_openblas_get_num_threads"),
                     ("openblas_set_num_threads64_", "openblas_get_num_threads64_"),
                     ("openblas_set_num_threads", "openblas_get_num_threads")):
            if hasattr(lib, s) and hasattr(lib, g):
                fs, fg = getattr(lib, s), getattr(lib, g)
                fs.argtypes, fs.restype, fg.restype = [ctypes.c_int], None, ctypes.c_int
                return fs, fg
    return None


_BLAS = _openblas_threads_api()


@contextlib.contextmanager
def dense_blas_threads():
    """The suite runs BLAS on one thread (the oracle's Lanczos recursions on small vectors are
    fastest there); the full diagonalizations of the exact Green function take every host core
    for their duration."""
    if _BLAS is None:
        yield
        return
    fs, fg = _BLAS
    old = fg()
    n = int(os.environ.get("ED_DENSE_BLAS_THREADS", "0")) or min(16, os.cpu_count() or 1)
    fs(max(1, n))
    try:
        yield
    finally:
        fs(old)


def _key(m, *rest):
    h = hashlib.sha256()
    for a in (m.h, m.U):
        h.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    h.update(repr((int(m.ns), int(m.L)) + tuple(rest)).encode())
    return h.hexdigest()


def green_exact(m, n_up, n_dn, z, spin=0, **kw):
    """O.green_exact(m, n_up, n_dn, z, spin) with the poles and residues of each (cluster,
    sector, spin) computed once.  Calls with other keywords go to the oracle unchanged."""
    if kw:
        with dense_blas_threads():
            return O.green_exact(m, n_up, n_dn, z, spin=spin, **kw)
    k = _key(m, n_up, n_dn, spin)
    if k not in _green:
        with dense_blas_threads():
            _, Q, w, E0, gap = O.green_exact(m, n_up, n_dn, np.zeros(0, dtype=np.complex128), spin=spin)
        _green[k] = (Q, w, E0, gap)
    Q, w, E0, gap = _green[k]
    return O.lehmann_green(Q, w, z), Q.copy(), w.copy(), E0, gap


def ground_state(m, n_up, n_dn):
    """O.ground_state(O.sector_hamiltonian(m, n_up, n_dn)), computed once per cluster and sector."""
    k = _key(m, n_up, n_dn)
    if k not in _ground:
        with dense_blas_threads():
            _ground[k] = O.ground_state(O.sector_hamiltonian(m, n_up, n_dn))
    E0, Om, gap = _ground[k]
    return E0, Om.copy(), gap


def sector_hamiltonian(m, n_up, n_dn):
    """O.sector_hamiltonian(m, n_up, n_dn), built once per cluster and sector (the 4x4 sector's
    diagonal alone has 1.66e8 elements)."""
    k = _key(m, n_up, n_dn, "op")
    if k not in _ops:
        _ops[k] = O.sector_hamiltonian(m, n_up, n_dn)
    return _ops[k]


def irrep_ground_energy(H, m, n_up, n_dn, gens, irrep, orders=None):
    """The symmetry oracle's irrep_ground_energy, given the irrep matrix H that the caller has
    already built with symmetric_hamiltonian for the same arguments: the oracle's own function
    and eigensolver run, without building H a second time."""
    import oracle.symmetry_oracle as S

    build = S.symmetric_hamiltonian
    S.symmetric_hamiltonian = lambda *a, **k: (H, None)
    try:
        with dense_blas_threads():
            return S.irrep_ground_energy(m, n_up, n_dn, gens, irrep, orders=orders)
    finally:
        S.symmetric_hamiltonian = build
