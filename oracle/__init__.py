"""Plain FP64 CPU oracle for the exact-diagonalization hot path.

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may
import it. The product path (``paper_2305_18643_gb300``) never imports it, and
it never imports the product path: the two share no code. Inputs come from the
seeded generators in ``paper_2305_18643_gb300.workloads`` and are passed in as
plain arrays.

Every function cites the section / equation of the paper (arXiv:2305.18643,
"Pyqcm: An open-source Python library for quantum cluster methods") that it
restates. Parity status of each function is listed in ``ed_oracle``'s header.
"""

from .ed_oracle import *  # noqa: F401,F403
