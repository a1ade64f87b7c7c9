"""Helpers shared by the GPU parity tests: library <-> oracle layout mapping."""
import numpy as np

from paper_1406_4960_gb300 import workloads as W


def gmap(handle, model, ik=0):
    """perm[g_lib] = g_oracle for the same integer G vectors (bit-exact set check)."""
    lib = handle.gvectors(ik)
    ora = {tuple(v): i for i, v in enumerate(model.gidx.tolist())}
    assert len(lib) == len(ora), "disc sizes differ: %d vs %d" % (len(lib), len(ora))
    return np.array([ora[tuple(v)] for v in lib.tolist()])


def lib_block(x_oracle, perm, ldg, dtype):
    """Oracle-ordered X[b][j][g] -> library layout with padding (numpy)."""
    nbands, nb, ng = x_oracle.shape
    out = np.zeros((nbands, nb, ldg), dtype=dtype)
    out[:, :, :ng] = x_oracle[:, :, perm]
    return out


def oracle_block(y_lib, perm):
    ng = len(perm)
    out = np.zeros(y_lib.shape[:2] + (ng,), dtype=np.complex128)
    out[:, :, perm] = y_lib[:, :, :ng]
    return out


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(1e-300, np.abs(b).max()))
