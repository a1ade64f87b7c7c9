"""Reference eigenvalues of the full 4x4 graphene workload (a = 4.65 bohr,
32 atoms, Ecut 30 Ha -> 1417 G, 64x64 grid, 80 B-splines on [-12, 12], KB
s+p projectors, Gamma, 80 roots) from the FP64 oracle alone: the generalized
Lanczos-Krylov iteration of §II.C on the oracle's matrix-free apply,
converged to a residual ||H x - eps S x||_{S^-1} < 1e-9.

The basis (113,360 functions) is beyond a dense solve; this is the oracle's
iterative route.  The oracle rebuilds its local-potential and projector
factors on every apply; this script computes them once and hands the same
arrays to every apply (identical arithmetic, minutes instead of hours).

Writes graphene_eigs.txt (one line, 80 values in Ha).  Calls only oracle/
and the seeded workload description."""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, HERE)

from make_slab_eigs import free_electron_start   # noqa: E402
from oracle import eigen as E                      # noqa: E402
from oracle import hamiltonian as Hm               # noqa: E402
from paper_1406_4960_gb300 import workloads as W   # noqa: E402


def main():
    w = W.graphene()
    t0 = time.time()
    m = Hm.model_from_workload(w)
    terms = m.local_terms()
    kb = m.kb_projectors()
    m.local_terms = lambda: terms
    m.kb_projectors = lambda: kb
    ops = E.BlockOps(m)
    X0 = free_electron_start(m, w.nbands + E.default_guard(w.nbands))
    hist = []
    eps, X, info = E.lanczos_krylov(ops, X0, w.nbands, block=4, tol=1e-9, max_cycles=400, history=hist)
    print("graphene: %d cycles, max residual %.2e, %.0f s" % (
        info["cycles"], info["residuals"].max(), time.time() - t0), flush=True)
    with open(os.path.join(HERE, "graphene_eigs.txt"), "w") as f:
        f.write("# graphene 4x4 workload (1417 G x 80 B-splines, 128 projectors, Gamma), 80 roots (Ha)\n")
        f.write("# written by make_graphene_eigs.py: oracle Lanczos-Krylov (Sec. II.C), residual < 1e-9\n")
        f.write(" ".join("%.15e" % e for e in eps) + "\n")


if __name__ == "__main__":
    main()
