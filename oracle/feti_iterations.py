"""PCG iteration counts of the oracle's FETI (Algorithm 1, FP64, tolerance 1e-10) on a named
workload of ``workloads``, and the solution's relative nodal error against the oracle's
single-domain solve (test infrastructure; calls only the oracle and the input generators).

    python -m oracle.feti_iterations peridynamic_2d

The benchmark's timing of the oracle on the host cores scales a sampled per-iteration time
by these counts.
"""
from __future__ import annotations

import sys
import time

import numpy as np

import workloads as W

from . import problem as oprob
from .feti import Feti


def main(name: str) -> None:
    w = getattr(W, name)()
    t0 = time.perf_counter()
    fo = Feti(w.mesh, w.kernel, w.labels, w.K)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    u, info = fo.solve(w.rhs, w.rhs_kind)
    t_solve = time.perf_counter() - t0
    its = info["iterations"]
    ref = oprob.Monolithic(w.mesh, w.kernel).solve(w.rhs, w.rhs_kind)
    err = oprob.rel_nodal_error(u, ref, w.mesh, w.kernel.ncomp).max()
    print(f"{name}: PCG iterations per right-hand side min {its.min()} max {its.max()}; "
          f"FETI vs single-domain {err:.3e}; setup {t_setup:.1f} s, solve {t_solve:.1f} s")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "peridynamic_2d")
