"""Writes tests/golden/ladder14_band.npz: the oracle's reference for the 2x7 ladder, the
14-orbital served-workload cluster whose 94 MB FP64 vectors make the library take its two-pass
H.psi kernels by itself.

Stored: the ground energy E0 (Sec. 4.2, ARPACK on the factorized H of Eq. factorized) and the
band-Lanczos Green function of Sec. 4.4 on two blocks (28 Krylov vectors per part) at 64
Matsubara frequencies (beta = 50), built from the oracle's own ground state.  Every value comes
from oracle/ and the seeded generator in paper_2305_18643_gb300.workloads; nothing from the CUDA
path.  A run takes several minutes of one CPU core (ARPACK on 11,778,624 states):

    python tests/golden/make_ladder14.py
"""

import os
import sys
import time

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2305_18643_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "ladder14_band.npz")
SEED = 4        # np.random.default_rng(SEED) draws the t' signs of the 2x7 ladder
R = 28          # Krylov vectors per part: two blocks of the 14 sites' starting vectors (the library's minimum)
N_FREQ = 64
BETA = 50.0


def main():
    c = W.served_request(np.random.default_rng(SEED), sizes=(14,))
    m = O.Model(c["t"], c["U"], c["mu"], c["eps"], c["theta"])
    t0 = time.time()
    op = O.sector_hamiltonian(m, c["n_up"], c["n_dn"])
    E0, Om, gap = O.ground_state(op, k=2, tol=1e-12)
    t1 = time.time()
    om = W.matsubara_grid(N_FREQ, BETA)
    G = O.green_band(m, c["n_up"], c["n_dn"], 1j * om, max_dim=R, ground=(E0, Om))[0]
    t2 = time.time()
    np.savez_compressed(OUT, E0=E0, gap=gap, omega=om, G=G, R=R, seed=SEED)
    print("E0 %.15f gap %.3e (ground state %.0f s, band G %.0f s) -> %s" % (E0, gap, t1 - t0, t2 - t1, OUT))


if __name__ == "__main__":
    main()
