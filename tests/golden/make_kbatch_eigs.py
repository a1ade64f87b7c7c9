"""Reference eigenvalues of four k-points of the batched-k workload (2x2
graphene cell, Ecut 30 Ha, 32x32 grid, 100 B-splines on [-12, 12], 24 roots
per k-point) from the FP64 oracle alone.

The four k-points are picked from the 64 seeded wedge points to span the
spread of cutoff-disc sizes: index 23 (smallest disc, 352 G), index 3
(largest, 361 G), and indices 0 and 40.  Each is solved by the generalized
Lanczos-Krylov iteration of §II.C on the oracle's matrix-free apply,
converged to a residual ||H x - eps S x||_{S^-1} < 1e-9.

Writes kbatch_eigs.txt: one line per k-point, the k index first, then the
24 eigenvalues in Ha.  Calls only oracle/ and the seeded workload
description."""
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

KPOINTS = (0, 3, 23, 40)


def main():
    w = W.kbatch()
    lines = []
    for ik in KPOINTS:
        t0 = time.time()
        m = Hm.model_from_workload(w, ik)
        ops = E.BlockOps(m)
        X0 = free_electron_start(m, w.nbands + E.default_guard(w.nbands))
        eps, X, info = E.lanczos_krylov(ops, X0, w.nbands, block=4, tol=1e-9, max_cycles=400)
        print("k %d (%d G): %d cycles, max residual %.2e, %.0f s" % (
            ik, m.ng, info["cycles"], info["residuals"].max(), time.time() - t0), flush=True)
        lines.append("%d " % ik + " ".join("%.15e" % e for e in eps))
    with open(os.path.join(HERE, "kbatch_eigs.txt"), "w") as f:
        f.write("# batched-k workload (2x2 graphene, Ecut 30 Ha, 100 B-splines), 4 of its 64 k-points x 24 roots (Ha)\n")
        f.write("# written by make_kbatch_eigs.py: oracle Lanczos-Krylov (Sec. II.C), residual < 1e-9; first column = k index\n")
        for l in lines:
            f.write(l + "\n")


if __name__ == "__main__":
    main()
