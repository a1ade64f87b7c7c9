"""Thin Python binding of the C ABI in include/mb.h (argument marshalling only).

Every step of the H/S apply and of the eigensolver runs in libmbgb300.so;
PyTorch only provides device memory and streams.  Loading fails loudly when
the library has not been built: there is no fallback."""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

MB_FP64, MB_FP32, MB_BF16 = 0, 1, 2
PREC = {"fp64": MB_FP64, "fp32": MB_FP32, "bf16": MB_BF16}
ERRORS = {0: "MB_OK", 1: "MB_EINVAL", 2: "MB_ENOMEM", 3: "MB_ENOTCONV", 4: "MB_ETIMEOUT",
          5: "MB_ECUDA", 6: "MB_EUNSUPPORTED"}

EXPORTS = ("mb_setup", "mb_destroy", "mb_sizes", "mb_gvectors", "mb_zplanes",
           "mb_set_local_potential", "mb_apply_H", "mb_apply_H_batch", "mb_apply_S",
           "mb_apply_Sinv", "mb_eigsolve", "mb_strerror", "mb_last_cuda_error",
           "mb_set_profiling", "mb_profile_read", "mb_profile_reset", "mb_launch_count",
           "mb_kernel_name", "mb_apply_H_noalloc", "mb_server_create", "mb_server_submit",
           "mb_server_wait", "mb_server_stats", "mb_server_destroy", "mb_autotune",
           "mb_plane_kernel_name", "mb_autotune_report", "mb_plane_kernel_candidates",
           "mb_plane_kernel_select", "mb_apply_S_batch", "mb_apply_Sinv_batch", "mb_status",
           "mb_local_potential", "mb_density", "mb_hartree", "mb_xc_lda", "mb_scf")


class MBError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__("%s (%d)%s" % (ERRORS.get(code, "?"), code, (": " + msg) if msg else ""))


class _Cell(ctypes.Structure):
    _fields_ = [("a1", ctypes.c_double * 2), ("a2", ctypes.c_double * 2)]


class _Atom(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_double * 3), ("A", ctypes.c_double), ("w", ctypes.c_double),
                ("nproj", ctypes.c_int), ("E", ctypes.c_double * 4), ("rc", ctypes.c_double),
                ("E2s", ctypes.c_double), ("E12", ctypes.c_double), ("Z", ctypes.c_double),
                ("Rcore", ctypes.c_double), ("q", ctypes.c_double * 4), ("q2s", ctypes.c_double),
                ("q12", ctypes.c_double), ("rQ", ctypes.c_double)]


class _Opts(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("nquad", ctypes.c_int),
                ("device", ctypes.c_int), ("max_bands", ctypes.c_int),
                ("precond_shift", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("applies", ctypes.c_int),
                ("max_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("finish_cycles", ctypes.c_int)]


class _Request(ctypes.Structure):
    _fields_ = [("cell", _Cell), ("kpts", ctypes.POINTER(ctypes.c_double)), ("nk", ctypes.c_int),
                ("ecut", ctypes.c_double), ("breaks", ctypes.POINTER(ctypes.c_double)),
                ("nbreaks", ctypes.c_int), ("order", ctypes.c_int), ("atoms", ctypes.POINTER(_Atom)),
                ("natoms", ctypes.c_int), ("opts", _Opts), ("nbands", ctypes.c_int),
                ("tol", ctypes.c_double), ("prec", ctypes.c_int)]


class ScfOpts(ctypes.Structure):
    _fields_ = [("nbands", ctypes.c_int), ("nelec", ctypes.c_double), ("sigma", ctypes.c_double),
                ("mix_weight", ctypes.c_double), ("g_max", ctypes.c_double), ("pulay_depth", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("eig_tol", ctypes.c_double),
                ("prec", ctypes.c_int), ("kweights", ctypes.POINTER(ctypes.c_double))]


class ScfInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("dv", ctypes.c_double), ("mu", ctypes.c_double),
                ("nelec", ctypes.c_double), ("eig_cycles", ctypes.c_int), ("seconds", ctypes.c_double),
                ("seconds_eig", ctypes.c_double), ("seconds_density", ctypes.c_double),
                ("seconds_potential", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("krylov_depth", ctypes.c_int), ("block", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("polish", ctypes.c_int), ("guard", ctypes.c_int),
                ("warm_start", ctypes.c_int)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """The ctypes handle of libmbgb300.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libmbgb300.so is not built (run __graft_entry__.build())")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    lib.mb_setup.argtypes = [ctypes.POINTER(_Cell), dp, ctypes.c_int, ctypes.c_double, dp,
                             ctypes.c_int, ctypes.c_int, ctypes.POINTER(_Atom), ctypes.c_int,
                             ctypes.POINTER(_Opts), ctypes.POINTER(vp)]
    lib.mb_destroy.argtypes = [vp]
    lib.mb_destroy.restype = None
    lib.mb_sizes.argtypes = [vp, ctypes.c_int, ip, ip, ip]
    lib.mb_gvectors.argtypes = [vp, ctypes.c_int, ip]
    lib.mb_zplanes.argtypes = [vp, ip, dp, dp]
    lib.mb_set_local_potential.argtypes = [vp, dp]
    lib.mb_local_potential.argtypes = [vp, dp]
    lib.mb_density.argtypes = [vp, vp, ctypes.c_int, dp, vp, vp]
    lib.mb_hartree.argtypes = [vp, vp, vp, vp]
    lib.mb_xc_lda.argtypes = [vp, vp, vp, vp, vp]
    lib.mb_scf.argtypes = [vp, ctypes.POINTER(ScfOpts), dp, vp, ctypes.POINTER(ScfInfo)]
    lib.mb_apply_H.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    lib.mb_apply_H_batch.argtypes = [vp, ctypes.c_int, ip, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.c_int, ctypes.c_int, vp]
    lib.mb_apply_S.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    lib.mb_apply_Sinv.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    for fn in (lib.mb_apply_S_batch, lib.mb_apply_Sinv_batch):
        fn.argtypes = [vp, ctypes.c_int, ip, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, vp]
    lib.mb_status.argtypes = [vp]
    lib.mb_eigsolve.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, vp,
                                ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]
    lib.mb_strerror.argtypes = [ctypes.c_int]
    lib.mb_strerror.restype = ctypes.c_char_p
    lib.mb_last_cuda_error.argtypes = [vp]
    lib.mb_last_cuda_error.restype = ctypes.c_char_p
    lib.mb_set_profiling.argtypes = [vp, ctypes.c_int]
    lib.mb_profile_read.argtypes = [vp, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_longlong)]
    lib.mb_profile_reset.argtypes = [vp]
    lib.mb_launch_count.argtypes = [vp]
    lib.mb_launch_count.restype = ctypes.c_longlong
    lib.mb_apply_H_noalloc.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    lib.mb_server_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(vp)]
    lib.mb_server_submit.argtypes = [vp, ctypes.POINTER(_Request), ctypes.POINTER(ctypes.c_longlong)]
    lib.mb_server_wait.argtypes = [vp, ctypes.c_longlong, dp, ctypes.POINTER(SolveInfo), dp, dp, ctypes.c_double]
    lib.mb_server_stats.argtypes = [vp, ip, ip, ip, dp, dp]
    lib.mb_server_destroy.argtypes = [vp]
    lib.mb_server_destroy.restype = None
    lib.mb_autotune.argtypes = [vp, ctypes.c_int, ctypes.c_int, ip, ip, dp]
    lib.mb_plane_kernel_name.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]
    lib.mb_autotune_report.argtypes = [vp, ctypes.c_char_p, ctypes.c_int]
    lib.mb_plane_kernel_candidates.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int]
    lib.mb_plane_kernel_select.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int]
    lib.mb_kernel_name.argtypes = [ctypes.c_int]
    lib.mb_kernel_name.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _dptr(a) -> ctypes.POINTER(ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(int(stream.cuda_stream))


def _atoms_array(atoms):
    arr = (_Atom * max(1, len(atoms)))()
    for i, at in enumerate(atoms):
        arr[i].pos = (ctypes.c_double * 3)(*at.pos)
        arr[i].A = at.A
        arr[i].w = at.w
        arr[i].nproj = at.nproj
        arr[i].E = (ctypes.c_double * 4)(*at.E)
        arr[i].rc = at.rc
        arr[i].E2s = getattr(at, "e2s", 0.0)
        arr[i].E12 = getattr(at, "e12", 0.0)
        arr[i].Z = getattr(at, "Z", 0.0)
        arr[i].Rcore = getattr(at, "Rcore", 0.0)
        arr[i].q = (ctypes.c_double * 4)(*getattr(at, "q", (0.0, 0.0, 0.0, 0.0)))
        arr[i].q2s = getattr(at, "q2s", 0.0)
        arr[i].q12 = getattr(at, "q12", 0.0)
        arr[i].rQ = getattr(at, "rQ", 0.0)
    return arr


class Server:
    """The continuous-batching solve server (mb_server_*)."""

    def __init__(self, device=0, slots=4, hbm_budget_bytes=64e9):
        self._lib = load()
        s = ctypes.c_void_p()
        rc = self._lib.mb_server_create(int(device), int(slots), float(hbm_budget_bytes), ctypes.byref(s))
        if rc:
            raise MBError(rc, "mb_server_create")
        self._s = s
        self._meta = {}

    def submit(self, w, nbands, tol=1e-6, prec="fp32", max_bands=128):
        kp = np.ascontiguousarray(np.asarray(w.kpts, dtype=np.float64).reshape(-1, 2))
        br = np.ascontiguousarray(np.asarray(w.breaks, dtype=np.float64))
        atoms = _atoms_array(w.atoms)
        req = _Request(_Cell((ctypes.c_double * 2)(*w.a1), (ctypes.c_double * 2)(*w.a2)),
                       _dptr(kp), kp.shape[0], float(w.ecut), _dptr(br), len(br), int(w.order),
                       atoms, len(w.atoms),
                       _Opts(int(w.grid[0]), int(w.grid[1]), int(w.nquad), 0, int(max_bands), 0.0),
                       int(nbands), float(tol), PREC[prec] if isinstance(prec, str) else int(prec))
        t = ctypes.c_longlong()
        rc = self._lib.mb_server_submit(self._s, ctypes.byref(req), ctypes.byref(t))
        if rc:
            raise MBError(rc, "mb_server_submit")
        self._meta[t.value] = (kp.shape[0], int(nbands))
        return t.value

    def wait(self, ticket, timeout_s=0.0, phases=False):
        """(rc, eigenvalues (nk, nbands), SolveInfo, latency s[, (queue, setup, solve) s])."""
        nk, nb = self._meta.pop(ticket)
        ev = np.zeros(nk * nb)
        info = SolveInfo()
        lat = ctypes.c_double()
        ph = np.zeros(3)
        rc = self._lib.mb_server_wait(self._s, ticket, _dptr(ev), ctypes.byref(info), ctypes.byref(lat),
                                      _dptr(ph), float(timeout_s))
        if phases:
            return rc, ev.reshape(nk, nb), info, lat.value, tuple(ph)
        return rc, ev.reshape(nk, nb), info, lat.value

    def stats(self):
        q, r, pr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        b, pb = ctypes.c_double(), ctypes.c_double()
        self._lib.mb_server_stats(self._s, ctypes.byref(q), ctypes.byref(r), ctypes.byref(pr),
                                  ctypes.byref(b), ctypes.byref(pb))
        return {"queued": q.value, "running": r.value, "peak_running": pr.value,
                "bytes_in_use": b.value, "peak_bytes": pb.value}

    def close(self):
        if getattr(self, "_s", None):
            self._lib.mb_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Handle:
    """One mb_handle: basis tables of a workload resident on a CUDA device."""

    def __init__(self, a1, a2, kpts, ecut, breaks, order, atoms, grid, nquad=0, device=0,
                 max_bands=128, precond_shift=0.0):
        self._lib = load()
        kp = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 2))
        br = np.ascontiguousarray(np.asarray(breaks, dtype=np.float64))
        cell = _Cell((ctypes.c_double * 2)(*a1), (ctypes.c_double * 2)(*a2))
        arr = _atoms_array(atoms)
        opts = _Opts(int(grid[0]), int(grid[1]), int(nquad), int(device), int(max_bands),
                     float(precond_shift))
        h = ctypes.c_void_p()
        rc = self._lib.mb_setup(ctypes.byref(cell), _dptr(kp), kp.shape[0], float(ecut), _dptr(br),
                                len(br), int(order), arr, len(atoms), ctypes.byref(opts),
                                ctypes.byref(h))
        if rc:
            raise MBError(rc, "mb_setup")
        self._h = h
        self.nk = kp.shape[0]
        self.device = device
        self.grid = (int(grid[0]), int(grid[1]))

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(w.a1, w.a2, w.kpts, w.ecut, w.breaks, w.order, w.atoms, w.grid, w.nquad, **kw)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc:
            msg = self._lib.mb_last_cuda_error(self._h).decode() if rc == 5 else ""
            raise MBError(rc, what + (" " + msg if msg else ""))

    def sizes(self, ik=0):
        ng, nb, ldg = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.mb_sizes(self._h, ik, ctypes.byref(ng), ctypes.byref(nb),
                                       ctypes.byref(ldg)), "mb_sizes")
        return ng.value, nb.value, ldg.value

    def gvectors(self, ik=0):
        ng, _, _ = self.sizes(ik)
        out = np.zeros(2 * ng, dtype=np.int32)
        self._check(self._lib.mb_gvectors(self._h, ik, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
                    "mb_gvectors")
        return out.reshape(ng, 2)

    def zplanes(self):
        nq = ctypes.c_int()
        self._check(self._lib.mb_zplanes(self._h, ctypes.byref(nq), None, None), "mb_zplanes")
        zq = np.zeros(nq.value)
        wq = np.zeros(nq.value)
        self._check(self._lib.mb_zplanes(self._h, None, _dptr(zq), _dptr(wq)), "mb_zplanes")
        return zq, wq

    def set_local_potential(self, V):
        V = np.ascontiguousarray(np.asarray(V, dtype=np.float64))
        zq, _ = self.zplanes()
        if V.size != len(zq) * self.grid[0] * self.grid[1]:
            raise MBError(1, "local potential must hold nq * n1 * n2 values")
        self._check(self._lib.mb_set_local_potential(self._h, _dptr(V)), "mb_set_local_potential")

    # ---- the self-consistent loop (fields: CUDA float64 tensors nq x n1 x n2)
    def _field_ok(self, t, name):
        zq, _ = self.zplanes()
        n = len(zq) * self.grid[0] * self.grid[1]
        if t.dtype.itemsize != 8 or t.is_complex() or t.numel() != n or not t.is_cuda or not t.is_contiguous():
            raise MBError(1, "%s must be a contiguous CUDA float64 tensor of %d elements" % (name, n))

    def density(self, evecs, nbands, occ, rho, stream=None):
        """rho <- sum_{k,n} f_nk |phi_nk|^2 of the eigenvector blocks evecs."""
        need = sum(nbands * self.sizes(ik)[1] * self.sizes(ik)[2] for ik in range(self.nk))
        if evecs.dtype.itemsize != 16 or evecs.numel() < need or not evecs.is_cuda or not evecs.is_contiguous():
            raise MBError(1, "evecs must be a contiguous CUDA complex128 buffer of %d elements" % need)
        self._field_ok(rho, "rho")
        occ = np.ascontiguousarray(np.asarray(occ, dtype=np.float64).reshape(self.nk * nbands))
        self._check(self._lib.mb_density(self._h, ctypes.c_void_p(evecs.data_ptr()), nbands, _dptr(occ),
                                         ctypes.c_void_p(rho.data_ptr()), _stream_ptr(stream)), "mb_density")

    def hartree(self, rho, vh, stream=None):
        self._field_ok(rho, "rho")
        self._field_ok(vh, "vh")
        self._check(self._lib.mb_hartree(self._h, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(vh.data_ptr()),
                                         _stream_ptr(stream)), "mb_hartree")

    def xc_lda(self, rho, vxc, exc=None, stream=None):
        self._field_ok(rho, "rho")
        self._field_ok(vxc, "vxc")
        if exc is not None:
            self._field_ok(exc, "exc")
        self._check(self._lib.mb_xc_lda(self._h, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(vxc.data_ptr()),
                                        ctypes.c_void_p(exc.data_ptr()) if exc is not None else None,
                                        _stream_ptr(stream)), "mb_xc_lda")

    def scf(self, nbands, tol, sigma, nelec=0.0, mix_weight=0.0, g_max=0.0, pulay_depth=0, max_iter=0,
            eig_tol=0.0, prec="fp64", kweights=None, rho_out=None, allow_notconv=False):
        """Self-consistent loop; returns (evals (nk, nbands), ScfInfo)."""
        kw = None
        if kweights is not None:
            kw = np.ascontiguousarray(np.asarray(kweights, dtype=np.float64).reshape(self.nk))
        o = ScfOpts(int(nbands), float(nelec), float(sigma), float(mix_weight), float(g_max), int(pulay_depth),
                    float(tol), int(max_iter), float(eig_tol), self._prec(prec),
                    kw.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if kw is not None else None)
        if rho_out is not None:
            self._field_ok(rho_out, "rho_out")
        ev = np.zeros(self.nk * nbands)
        info = ScfInfo()
        rc = self._lib.mb_scf(self._h, ctypes.byref(o), _dptr(ev),
                              ctypes.c_void_p(rho_out.data_ptr()) if rho_out is not None else None,
                              ctypes.byref(info))
        if rc and not (rc == 3 and allow_notconv):
            self._check(rc, "mb_scf")
        return ev.reshape(self.nk, nbands), info

    def local_potential(self):
        """The local potential table V[q][i1][i2] (Ha) the applies use."""
        zq, _ = self.zplanes()
        V = np.zeros((len(zq), self.grid[0], self.grid[1]))
        self._check(self._lib.mb_local_potential(self._h, _dptr(V)), "mb_local_potential")
        return V

    # ---- applies on torch device tensors --------------------------------
    @staticmethod
    def _prec(prec):
        return PREC[prec] if isinstance(prec, str) else int(prec)

    def _check_block(self, ik, T, prec):
        """Reject tensors whose size, dtype or placement would make the kernels
        read or write outside them."""
        import torch
        ng, nb, ldg = self.sizes(ik)
        want = torch.complex128 if self._prec(prec) == MB_FP64 else torch.complex64
        if T.dtype != want or not T.is_cuda or not T.is_contiguous():
            raise MBError(1, "block must be a contiguous CUDA %s tensor" % want)
        if T.dim() != 3 or T.shape[1] != nb or T.shape[2] != ldg:
            raise MBError(1, "block shape must be (nbands, %d, %d), got %s" % (nb, ldg, tuple(T.shape)))
        if T.device.index != self.device:
            raise MBError(1, "block is on cuda:%s, handle on cuda:%d" % (T.device.index, self.device))
        return T.shape[0]

    def apply_H(self, ik, X, Y, prec="fp64", stream=None):
        nb = self._check_block(ik, X, prec)
        if self._check_block(ik, Y, prec) != nb:
            raise MBError(1, "X and Y band counts differ")
        self._check(self._lib.mb_apply_H(self._h, ik, ctypes.c_void_p(X.data_ptr()),
                                         ctypes.c_void_p(Y.data_ptr()), nb, self._prec(prec),
                                         _stream_ptr(stream)), "mb_apply_H")

    def apply_H_batch(self, iks: Sequence[int], Xs, Ys, prec="fp64", stream=None):
        n = len(iks)
        if len(Xs) != n or len(Ys) != n:
            raise MBError(1, "one X and one Y per k-point")
        for ik, X, Y in zip(iks, Xs, Ys):
            if self._check_block(ik, X, prec) != Xs[0].shape[0] or self._check_block(ik, Y, prec) != Xs[0].shape[0]:
                raise MBError(1, "all blocks need the same band count")
        ik_arr = (ctypes.c_int * n)(*iks)
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in Xs])
        yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in Ys])
        self._check(self._lib.mb_apply_H_batch(self._h, n, ik_arr, xp, yp, Xs[0].shape[0],
                                               self._prec(prec), _stream_ptr(stream)), "mb_apply_H_batch")

    def apply_S(self, ik, X, Y, prec="fp64", stream=None):
        if self._check_block(ik, X, prec) != self._check_block(ik, Y, prec):
            raise MBError(1, "X and Y band counts differ")
        self._check(self._lib.mb_apply_S(self._h, ik, ctypes.c_void_p(X.data_ptr()),
                                         ctypes.c_void_p(Y.data_ptr()), X.shape[0],
                                         self._prec(prec), _stream_ptr(stream)), "mb_apply_S")

    def apply_Sinv(self, ik, X, Y, prec="fp64", stream=None):
        if self._check_block(ik, X, prec) != self._check_block(ik, Y, prec):
            raise MBError(1, "X and Y band counts differ")
        self._check(self._lib.mb_apply_Sinv(self._h, ik, ctypes.c_void_p(X.data_ptr()),
                                            ctypes.c_void_p(Y.data_ptr()), X.shape[0],
                                            self._prec(prec), _stream_ptr(stream)), "mb_apply_Sinv")

    def _banded_batch(self, fn, name, iks, Xs, Ys, prec, stream):
        n = len(iks)
        if len(Xs) != n or len(Ys) != n:
            raise MBError(1, "one X and one Y per k-point")
        for ik, X, Y in zip(iks, Xs, Ys):
            if self._check_block(ik, X, prec) != Xs[0].shape[0] or self._check_block(ik, Y, prec) != Xs[0].shape[0]:
                raise MBError(1, "all blocks need the same band count")
        ik_arr = (ctypes.c_int * n)(*iks)
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in Xs])
        yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in Ys])
        self._check(fn(self._h, n, ik_arr, xp, yp, Xs[0].shape[0], self._prec(prec), _stream_ptr(stream)), name)

    def apply_S_batch(self, iks, Xs, Ys, prec="fp64", stream=None):
        self._banded_batch(self._lib.mb_apply_S_batch, "mb_apply_S_batch", iks, Xs, Ys, prec, stream)

    def apply_Sinv_batch(self, iks, Xs, Ys, prec="fp64", stream=None):
        self._banded_batch(self._lib.mb_apply_Sinv_batch, "mb_apply_Sinv_batch", iks, Xs, Ys, prec, stream)

    def status(self):
        """MB_OK, or raises MBError(MB_ETIMEOUT) when a bounded device wait ran out."""
        self._check(self._lib.mb_status(self._h), "mb_status")

    def autotune(self, nbands, prec="fp32"):
        bt, waves, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(self._lib.mb_autotune(self._h, int(nbands), self._prec(prec), ctypes.byref(bt),
                                          ctypes.byref(waves), ctypes.byref(ms)), "mb_autotune")
        return {"bands_per_cta": bt.value if bt.value > 0 else None, "waves": waves.value, "ms": ms.value,
                "kernel": self.plane_kernel_name(self.nk, nbands, prec)}

    def plane_kernel_candidates(self, nk, nbands, prec="fp32"):
        ids = (ctypes.c_int * 16)()
        n = self._lib.mb_plane_kernel_candidates(self._h, int(nk), int(nbands), self._prec(prec), ids, 16)
        if n < 0:
            raise MBError(-n, "mb_plane_kernel_candidates")
        return list(ids[:n])

    def plane_kernel_select(self, nk, nbands, prec, kernel_id, waves=0, persistent=False):
        self._check(self._lib.mb_plane_kernel_select(self._h, int(nk), int(nbands), self._prec(prec), int(kernel_id),
                                                     int(waves), 1 if persistent else 0), "mb_plane_kernel_select")

    def autotune_report(self):
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(self._lib.mb_autotune_report(self._h, buf, 1 << 16), "mb_autotune_report")
        return buf.value.decode()

    def plane_kernel_name(self, nk, nbands, prec="fp32"):
        buf = ctypes.create_string_buffer(128)
        self._check(self._lib.mb_plane_kernel_name(self._h, int(nk), int(nbands), self._prec(prec), buf, 128),
                    "mb_plane_kernel_name")
        return buf.value.decode()

    def eigsolve(self, nbands, tol, prec="fp64", evecs=None, krylov_depth=0, block=0,
                 max_cycles=0, polish=0, stream=None, allow_notconv=False, guard=0, warm_start=False):
        ev = np.zeros(self.nk * nbands)
        info = SolveInfo()
        if warm_start and evecs is None:
            raise MBError(1, "warm_start needs the start vectors in evecs")
        so = SolveOpts(krylov_depth, block, max_cycles, polish, guard, int(bool(warm_start)))
        if evecs is not None:
            need = sum(nbands * self.sizes(ik)[1] * self.sizes(ik)[2] for ik in range(self.nk))
            if evecs.dtype.itemsize != 16 or evecs.numel() < need or not evecs.is_cuda or not evecs.is_contiguous():
                raise MBError(1, "evecs must be a contiguous CUDA complex128 buffer of %d elements" % need)
        rc = self._lib.mb_eigsolve(self._h, nbands, float(tol), self._prec(prec), _dptr(ev),
                                   ctypes.c_void_p(evecs.data_ptr()) if evecs is not None else None,
                                   ctypes.byref(so), ctypes.byref(info), _stream_ptr(stream))
        if rc and not (rc == 3 and allow_notconv):
            self._check(rc, "mb_eigsolve")
        return ev.reshape(self.nk, nbands), info
