"""Second, independent route to the slab workload's reference eigenvalues:
the definition itself -- the dense generalized eigenproblem H c = eps S c
reduced by the Cholesky factor of S and solved by LAPACK -- instead of the
Lanczos-Krylov iteration that wrote slab_eigs.txt.

The basis index is j*N_G + g and S = S_z (x) I_G (§II.B.1, Eqs. (7)-(8): S is
diagonal in G), so S = L L^H with L = L_z (x) I_G and the reduced matrix
H~ = (L_z^-1 (x) I) H (L_z^-1 (x) I)^H is formed by contracting L_z^-1 on the
two spline indices of H -- the same matrix that a dense Cholesky of S would
give, at a cost the 21480-dimensional slab basis allows.  The script first
checks that this structured reduction reproduces the oracle's plain
`generalized_lowest` on the tiny cell.

The slab's 2x2 Monkhorst-Pack k-points come in time-reversal pairs (k0, k3)
and (k1, k2) with identical spectra, so k-points 0 and 1 cover all four.

Writes slab_eigs_dense.txt: one line per k-point, the k index first, then the
32 lowest eigenvalues in Ha.  Calls only oracle/, numpy/scipy and the seeded
workload description.  Needs about 30 GB of host memory and some minutes per
k-point."""
import os
import sys
import time

import numpy as np
import scipy.linalg as sl

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import eigen as E                      # noqa: E402
from oracle import hamiltonian as Hm               # noqa: E402
from paper_1406_4960_gb300 import workloads as W   # noqa: E402

KPOINTS = (0, 1)


def reduced_lowest(m, nroots):
    """Lowest eigenvalues of H c = eps S c for one oracle model, through the
    G-diagonal Cholesky factor of S."""
    nb, ng = m.nb, m.ng
    H = m.dense_H()
    Li = np.linalg.inv(np.linalg.cholesky(m.S)).astype(np.complex128)
    # left factor: rows (i, g) <- sum_j Li[i, j] H[(j, g), :]
    H = (Li @ H.reshape(nb, ng * nb * ng)).reshape(nb * ng, nb, ng)
    # right factor: columns (l, h) <- sum_j H[:, (j, h)] conj(Li[l, j])
    H = np.ascontiguousarray(np.einsum("rjh,lj->rlh", H, Li.conj(), optimize=True)).reshape(nb * ng, nb * ng)
    return sl.eigh(H, eigvals_only=True, subset_by_index=[0, nroots - 1], driver="evr",
                   overwrite_a=True, check_finite=False)


def check_on_tiny():
    w = W.tiny()
    m = Hm.model_from_workload(w)
    a = reduced_lowest(m, w.nbands)
    b = E.generalized_lowest(m.dense_H(), m.dense_S(), w.nbands)
    err = float(np.abs(a - b).max())
    assert err < 1e-10, "structured reduction disagrees with the plain definition: %.3e" % err
    print("tiny cell: structured reduction vs generalized_lowest %.2e Ha" % err, flush=True)


def main():
    check_on_tiny()
    w = W.slab()
    lines = []
    for ik in KPOINTS:
        t0 = time.time()
        m = Hm.model_from_workload(w, ik)
        ev = reduced_lowest(m, w.nbands)
        print("k %d: basis %d, %.0f s" % (ik, m.nbasis, time.time() - t0), flush=True)
        lines.append("%d " % ik + " ".join("%.15e" % e for e in ev))
    with open(os.path.join(HERE, "slab_eigs_dense.txt"), "w") as f:
        f.write("# slab workload, k-points 0 and 1 (k3 = -k0 and k2 = -k1 share their spectra), 32 roots (Ha)\n")
        f.write("# written by make_slab_dense.py: dense Cholesky-reduced generalized problem, LAPACK; first column = k index\n")
        for l in lines:
            f.write(l + "\n")


if __name__ == "__main__":
    main()
