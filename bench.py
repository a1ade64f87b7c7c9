"""Benchmark of the mixed-basis hot path on GB300.

Workload (N=1): the C(001)-(2x1)-like slab -- rectangular 9.5 x 4.75 bohr
cell, 12 pseudo-atoms, Ecut 25 Ha (179-ish G per k), 32x16 grid, 120 order-6
B-splines on slab-dense/geometric knots, KB s+p projectors, 2x2 k-points,
32 bands.  Synthetic, seeded inputs.

A step is one H application to the 32-band block at all 4 k-points in one
batched call (B-spline evaluation, inverse FFTs, potential product, forward
FFTs, adjoint, banded kinetic term, projector contractions).  `value` is
Hpsi GB/s = algorithmic bytes / device time; the same apply in FP64 and the
mixed-precision and plain-FP64 eigensolves are reported beside it.

--impl reference times the CPU oracle (plain FP64 numpy/C) on a bounded
sample of the same workload.

Multi-GPU (torchrun): every rank runs an independent replica of the workload
(k-point sets are independent problems; no collective on the data path), the
step time is the max over ranks and `value` sums all ranks' bytes.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The serving section runs up to 8 requests at once, each with a solve
# stream, a projector stream and a set-up stream: give the process enough
# hardware work queues that a request's set-up copies do not wait behind
# another request's kernels (read when the CUDA context is created).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "Hψ GB/s & eigensolves/s at 1e-6 Ha vs plain FP64 GPU; p50/p99 solve latency"
# The plane kernel's sources: its DRAM traffic (from an ncu capture, recorded
# in the profile summary below with the kernel instance) is reported only
# while these are unchanged and the same instance runs.
PLANE_SOURCES = ("plane_reg.cu", "apply_common.cuh", "cplx.cuh")
PLANE_PROFILES = {
    "slab": "profiles/plane32_kernel_slab_fp32.md",
    "graphene": "profiles/plane32_kernel_graphene_fp32.md",
    "kbatch": "profiles/plane32_kernel_kbatch_fp32.md",
}


def plane_sources_hash():
    """sha256 (first 16 hex digits) of the plane kernel's source files."""
    import hashlib
    d = hashlib.sha256()
    for f in PLANE_SOURCES:
        with open(os.path.join(ROOT, "paper_1406_4960_gb300", "csrc", f), "rb") as fh:
            d.update(fh.read())
    return d.hexdigest()[:16]


def plane_traffic(workload, kernel):
    """(bytes per launch, note): dram__bytes_read.sum + dram__bytes_write.sum of
    one plane-kernel launch from the committed ncu summary, or None when the
    summary is missing, was taken on other kernel sources or of another
    kernel instance."""
    import re
    path = os.path.join(ROOT, PLANE_PROFILES.get(workload, ""))
    if not os.path.isfile(path):
        return None, "no ncu summary for this workload"
    lines = re.findall(r"traffic per launch: (\d+) bytes; kernel = (.+?); kernel sources sha256 = ([0-9a-f]{16})",
                       open(path).read())
    if not lines:
        return None, "ncu summary has no traffic line"
    want = kernel.replace(" persistent", "").strip()
    for nbytes, name, sha in lines:
        if name.strip() == want:
            if sha != plane_sources_hash():
                return None, "kernel sources changed since the ncu capture"
            return float(nbytes), "ncu capture of this instance (%s)" % PLANE_PROFILES[workload]
    return None, "no ncu capture of this instance"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def workload_sizes(h, w, prec):
    """Algorithmic bytes and plane-kernel flops of one batched apply."""
    cb = 16 if prec == "fp64" else 8
    rb = cb // 2
    zq, _ = h.zplanes()
    nq = len(zq)
    n1, n2 = w.grid
    N = n1 * n2
    nproj = sum(a.nproj for a in w.atoms)
    byts = nq * N * rb
    flops = 0.0
    for ik in range(w.nk):
        ng, nb, ldg = h.sizes(ik)
        byts += 2 * ng * nb * w.nbands * cb + nproj * (ng + nb) * cb
        flops += w.nbands * nq * (8 * w.order * ng + 10 * N * math.log2(N) + 2 * N)
    return byts, flops


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w, budget_s=12.0, impl_steps=None):
    """The FP64 oracle applying H to the 32-band block, one k-point at a time,
    until the budget is spent; returns (GB/s, cores, sample, seconds)."""
    from oracle import hamiltonian as Hm
    from paper_1406_4960_gb300 import workloads as W
    t_setup = time.perf_counter()
    models = [Hm.model_from_workload(w, ik) for ik in range(w.nk)]
    del t_setup
    nproj = sum(a.nproj for a in w.atoms)
    n1, n2 = w.grid
    nq = models[0].zb.zq.size
    done_bytes, t_used, n_apply = 0.0, 0.0, 0
    ik = 0
    while (n_apply < impl_steps) if impl_steps is not None else (t_used < budget_s):
        m = models[ik % w.nk]
        X = W.random_block(w.nbands, m.nb, m.ng, seed=500 + ik)
        t0 = time.perf_counter()
        m.apply_H(X)
        t_used += time.perf_counter() - t0
        done_bytes += 2 * m.ng * m.nb * w.nbands * 8 + nproj * (m.ng + m.nb) * 8 + nq * n1 * n2 * 4 / w.nk
        n_apply += 1
        ik += 1
    cores = _blas_threads()
    sample = "%d single-k-point H applies of the %d-band block (FP64 oracle, bytes counted at FP32 widths)" % (
        n_apply, w.nbands)
    return done_bytes / t_used / 1e9, cores, sample, t_used, n_apply


def cpu_solve_tiny():
    """The FP64 oracle's dense generalized solve of the tiny cell (45 G x 40
    B-splines, 1800 basis functions, 8 roots): assembly and solve seconds."""
    from oracle import eigen as E
    from oracle import hamiltonian as Hm
    from paper_1406_4960_gb300 import workloads as W
    w = W.tiny()
    t0 = time.perf_counter()
    m = Hm.model_from_workload(w)
    H, S = m.dense_H(), m.dense_S()
    t1 = time.perf_counter()
    E.generalized_lowest(H, S, w.nbands)
    t2 = time.perf_counter()
    return {"workload": "tiny: 45 G x 40 B-splines (1800 basis functions), 8 roots, dense FP64",
            "assembly_seconds": t1 - t0, "solve_seconds": t2 - t1}


def golden_slab():
    """Oracle eigenvalues of the slab workload (tests/golden/slab_eigs.txt,
    written by tests/golden/make_slab_eigs.py from the oracle alone)."""
    path = os.path.join(ROOT, "tests", "golden", "slab_eigs.txt")
    if not os.path.exists(path):
        return None
    rows = [l for l in open(path) if l.strip() and not l.startswith("#")]
    return np.array([[float(x) for x in r.split()] for r in rows])


def eig_bench(h, w, args):
    """Mixed-precision and plain-FP64 eigensolves of the whole workload
    (4 k-points x 32 roots, residual tolerance 1e-6 Ha, which bounds every
    eigenvalue error by 1e-6 Ha); wall time per solve = solve latency."""
    ref = golden_slab()
    out = {"tol_ha": 1e-6, "roots": w.nbands, "kpoints": w.nk}
    for prec, reps in (("fp32", args.eig_reps), ("fp64", max(1, args.eig_reps // 2))):
        h.eigsolve(w.nbands, 1e-6, prec)          # warm-up (module load, set-up of factors)
        times, infos, ev = [], [], None
        for _ in range(reps):
            t0 = time.perf_counter()
            ev, info = h.eigsolve(w.nbands, 1e-6, prec)
            times.append(time.perf_counter() - t0)
            infos.append(info)
        ts = np.array(times) * 1e3
        # one more solve with per-kernel event timing (not part of the timed reps)
        import ctypes
        lib = h._lib
        lib.mb_profile_reset(h._h)
        lib.mb_set_profiling(h._h, 1)
        n0 = lib.mb_launch_count(h._h)
        h.eigsolve(w.nbands, 1e-6, prec)
        nl = lib.mb_launch_count(h._h) - n0
        lib.mb_set_profiling(h._h, 0)
        kms = {}
        for kid in range(13):
            t_, c_ = ctypes.c_double(), ctypes.c_longlong()
            lib.mb_profile_read(h._h, kid, ctypes.byref(t_), ctypes.byref(c_))
            if c_.value:
                kms[lib.mb_kernel_name(kid).decode()] = [round(t_.value, 3), int(c_.value)]
        rec = {"kernels_ms_launches": kms, "launches": int(nl),"solves_per_s": 1e3 / float(np.mean(ts)), "ms_p50": float(np.percentile(ts, 50)),
               "ms_p99": float(np.percentile(ts, 99)), "reps": reps, "cycles": infos[-1].cycles,
               "applies": infos[-1].applies, "max_residual": infos[-1].max_residual,
               "max_abs_err_vs_oracle_ha": None if ref is None else float(np.abs(ev - ref).max())}
        out["mixed" if prec == "fp32" else "fp64"] = rec
    out["mixed_speedup_vs_fp64"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    return out


def golden(name):
    """Oracle eigenvalues written by a tests/golden/make_*.py script (which
    calls only oracle/): {k index: values}, or None if the file is absent."""
    path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(path):
        return None
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    if name == "graphene_eigs.txt":
        return {0: np.array(rows[0], dtype=float)}
    return {int(r[0]): np.array(r[1:], dtype=float) for r in rows}


def solve_record(h, nbands, prec, ref, reps=1):
    """Wall time, cycles, residual and error vs oracle eigenvalues of `reps`
    eigensolves of every k-point of a handle."""
    times, ev, info = [], None, None
    for _ in range(reps):
        t0 = time.perf_counter()
        ev, info = h.eigsolve(nbands, 1e-6, prec)
        times.append(time.perf_counter() - t0)
    err = None
    if ref:
        err = float(max(np.abs(ev[k] - v).max() for k, v in ref.items()))
    return {"seconds": float(np.median(times)), "solves_per_s": 1.0 / float(np.median(times)),
            "cycles": info.cycles, "finish_cycles": info.finish_cycles, "max_residual": info.max_residual,
            "max_abs_err_vs_oracle_ha": err,
            "oracle_kpoints": None if not ref else sorted(ref)}, ev


def graphene_bench(mb, W, local, args, timed, peak32):
    """Config 2: the 4x4 graphene cell (1417 G, 80 splines, 64x64 grid, 128
    projectors, 80 bands).  FP32, FP64 and BF16-projector applies of the
    80-band block (the plane kernel's roofline from the FP32 steps), then a
    mixed-precision and a plain-FP64 eigensolve of 80 roots against the
    oracle's eigenvalues (tests/golden/graphene_eigs.txt)."""
    w = W.graphene()
    h = mb.Handle.from_workload(w, device=local)
    tune = h.autotune(w.nbands, "fp32")
    steps = 10
    ms32, launches, prof_plane = timed(h, w, "fp32", steps, 3, profile=2, sync_ranks=False)
    ms64, _, _ = timed(h, w, "fp64", 3, 2, sync_ranks=False)
    msbf, _, _ = timed(h, w, "bf16", 5, 2, sync_ranks=False)
    _, _, prof = timed(h, w, "fp32", 5, 1, profile=1, sync_ranks=False)
    b32, f32 = workload_sizes(h, w, "fp32")
    b64, _ = workload_sizes(h, w, "fp64")
    out = {"workload": "graphene: 4x4 cell, 32 atoms, Ecut 30 Ha, 64x64 grid, 80 B-splines, Gamma, 80 bands",
           "fp32": {"value": b32 / (ms32 * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": ms32,
                    "kernels_ms_per_step": {k: v[0] / 5 for k, v in prof.items()},
                    "gpu_launches_per_step": int(launches) // steps},
           "fp64": {"value": b64 / (ms64 * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": ms64},
           "bf16": {"value": b32 / (msbf * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": msbf},
           "autotune": tune,
           "roofline": plane_roofline(prof_plane, f32, steps, ms32, h.plane_kernel_name(w.nk, w.nbands, "fp32"),
                                      "graphene", peak32)}
    if not args.no_eig:
        ref = golden("graphene_eigs.txt")
        mixed, e32 = solve_record(h, w.nbands, "fp32", ref)
        plain, e64 = solve_record(h, w.nbands, "fp64", ref)
        out["eigsolve"] = {"tol_ha": 1e-6, "roots": w.nbands, "mixed": mixed, "fp64": plain,
                           "mixed_speedup_vs_fp64": plain["seconds"] / mixed["seconds"],
                           "mixed_vs_fp64_max_diff_ha": float(np.abs(e32 - e64).max())}
    h.close()
    return out


def kbatch_bench(mb, W, local, args, timed, peak32):
    """Config 3: the 2x2 graphene cell with 64 wedge k-points x 24 bands.  The
    plane-kernel launch shape is autotuned for the batch, then one FP32 H
    apply of all 64 k-points (one launch sequence) is timed; then one
    mixed-precision and one plain-FP64 eigensolve of all 64 k-points (grand
    cycles replayed as CUDA graphs), checked against the oracle's eigenvalues
    at four of the k-points (tests/golden/kbatch_eigs.txt)."""
    w = W.kbatch()
    h = mb.Handle.from_workload(w, device=local)
    tune = h.autotune(w.nbands, "fp32")
    steps = 10
    ms, launches, prof_plane = timed(h, w, "fp32", steps, 3, profile=2, sync_ranks=False)
    byts, flops = workload_sizes(h, w, "fp32")
    out = {"workload": "kbatch: 2x2 graphene, Ecut 30 Ha, 32x32 grid, 100 B-splines, 64 k x 24 bands",
           "autotune": tune, "apply_ms": ms, "apply_gbs": byts / (ms * 1e-3) / 1e9,
           "gpu_launches_per_apply": int(launches) // steps,
           "roofline": plane_roofline(prof_plane, flops, steps, ms, h.plane_kernel_name(w.nk, w.nbands, "fp32"),
                                      "kbatch", peak32)}
    if not args.no_kbatch_solve:
        ref = golden("kbatch_eigs.txt")
        mixed, _ = solve_record(h, w.nbands, "fp32", ref)
        plain, _ = solve_record(h, w.nbands, "fp64", ref)
        out["eigsolve"] = {"tol_ha": 1e-6, "roots": w.nbands, "kpoints": w.nk, "mixed": mixed, "fp64": plain,
                           "mixed_speedup_vs_fp64": plain["seconds"] / mixed["seconds"]}
    h.close()
    return out


def probe_fp64_peak(lib, device):
    """Measured FP64 FMA rate (TFLOP/s) of this GPU, or None."""
    import ctypes
    fn = lib.mb_probe_fp64_fma
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    tf, ms = ctypes.c_double(), ctypes.c_double()
    return tf.value if fn(device, 5, ctypes.byref(tf), ctypes.byref(ms)) == 0 else None


SCF_Z, SCF_RCORE = 4.0, 0.6          # carbon-like core charges on the slab's 12 atoms: 48 electrons
SCF_SIGMA, SCF_W, SCF_GMAX = 0.01, 0.5, 1.0
SCF_TOL = 0.5e-6                     # the paper's criterion: V_scf changes by less than 1e-6 Ry
SCF_USPP_Q, SCF_USPP_RQ = (0.5, 0.2, 0.2, 0.2), 0.8   # synthetic ultrasoft q (1s, p) and charge radius


def scf_workload(W):
    return W.with_core(W.slab(), SCF_Z, SCF_RCORE, name="slab-scf")


def density_flops(h, w, nbands):
    """Algorithmic flops of one density: per (k, band, plane) the B-spline
    evaluation (4 kappa ng), one inverse FFT (5 N log2 N) and f |psi|^2 (4 N)."""
    N = w.grid[0] * w.grid[1]
    zq, _ = h.zplanes()
    tot = 0.0
    for ik in range(w.nk):
        ng = h.sizes(ik)[0]
        tot += nbands * len(zq) * (4 * w.order * ng + 5 * N * math.log2(N) + 4 * N)
    return tot


def scf_steps(mb, h, w, local):
    """The self-consistent loop's device steps alone on a handle's current
    potential: the density of its lowest w.nbands roots (the first 24 per
    k-point filled), its Coulomb and LDA potentials, each timed with CUDA
    events on its stream; the density kernel's roofline against the measured
    FP64 FMA rate."""
    import torch
    need = sum(w.nbands * h.sizes(ik)[1] * h.sizes(ik)[2] for ik in range(w.nk))
    evecs = torch.zeros(need, dtype=torch.complex128, device="cuda:%d" % local)
    h.eigsolve(w.nbands, SCF_TOL, "fp32", evecs=evecs)
    zq, _ = h.zplanes()
    shape = (len(zq), w.grid[0], w.grid[1])
    rho = torch.zeros(shape, dtype=torch.float64, device="cuda:%d" % local)
    vh, vx = torch.zeros_like(rho), torch.zeros_like(rho)
    occ = np.zeros((w.nk, w.nbands))
    occ[:, :24] = 2.0 / w.nk
    st = torch.cuda.Stream(device=local)
    ms = {}
    for name, fn in (("density", lambda: h.density(evecs, w.nbands, occ, rho, stream=st)),
                     ("hartree", lambda: h.hartree(rho, vh, stream=st)),
                     ("xc", lambda: h.xc_lda(rho, vx, stream=st))):
        for _ in range(2):
            fn()
        reps = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(local)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize(local)
        ms[name] = e0.elapsed_time(e1) / reps
    fl = density_flops(h, w, w.nbands)
    peak64 = probe_fp64_peak(mb.load(), local)
    ach = fl / (ms["density"] * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": ach, "peak": peak64, "unit": "TFLOP/s",
            "frac": ach / peak64 if peak64 else None, "gflop": fl / 1e9,
            "peak_source": "measured: FP64 DFMA loop on this GPU (mb_probe_fp64_fma)",
            "note": "mb_density as called: occupation upload, partial planes, fixed-order reduction included"}
    return ms, roof


def scf_bench(mb, W, local, args):
    """Section (f)3: the self-consistent loop on the slab with carbon-like core
    charges (48 electrons in 32 bands per k-point), to the paper's criterion,
    with mixed-precision and with plain FP64 eigensolves; then the density,
    Coulomb and LDA steps alone, timed with CUDA events on their stream (the
    density kernel's roofline against the measured FP64 FMA rate)."""
    import torch
    w = scf_workload(W)
    out = {"workload": "slab with core charges Z = %g, R_c = %g bohr on its 12 atoms (48 electrons), 4 k x 32 "
                       "bands, Fermi-Dirac %g Ha, Kerker W %g g_max %g, Pulay 4" % (SCF_Z, SCF_RCORE, SCF_SIGMA,
                                                                                     SCF_W, SCF_GMAX),
           "tol_ha": SCF_TOL}
    evs = {}
    for prec in ("fp32", "fp64"):
        h = mb.Handle.from_workload(w, device=local)
        ev, info = h.scf(w.nbands, SCF_TOL, SCF_SIGMA, mix_weight=SCF_W, g_max=SCF_GMAX, prec=prec,
                         eig_tol=SCF_TOL / 5, max_iter=80, allow_notconv=True)
        evs[prec] = ev
        out["mixed" if prec == "fp32" else "fp64"] = {
            "converged": bool(info.dv < SCF_TOL), "iterations": info.iterations, "seconds": info.seconds,
            "seconds_eig": info.seconds_eig, "seconds_density": info.seconds_density,
            "seconds_potential": info.seconds_potential, "eig_cycles": info.eig_cycles, "dv_ha": info.dv,
            "fermi_ha": info.mu, "nelec": info.nelec}
        if prec == "fp32":
            # the device steps alone, on the converged potential
            out["steps_ms"], out["density_roofline"] = scf_steps(mb, h, w, local)
        h.close()
    out["mixed_speedup_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    out["mixed_vs_fp64_max_eig_diff_ha"] = float(np.abs(evs["fp32"] - evs["fp64"]).max())
    # the same slab with ultrasoft augmentation on every projector (section (f)4)
    wu = W.with_uspp(w, SCF_USPP_Q, SCF_USPP_RQ)
    h = mb.Handle.from_workload(wu, device=local)
    ev, info = h.scf(wu.nbands, SCF_TOL, SCF_SIGMA, mix_weight=SCF_W, g_max=SCF_GMAX, prec="fp32",
                     eig_tol=SCF_TOL / 5, max_iter=80, allow_notconv=True)
    out["uspp_mixed"] = {"q": list(SCF_USPP_Q), "rQ": SCF_USPP_RQ, "converged": bool(info.dv < SCF_TOL),
                         "iterations": info.iterations, "seconds": info.seconds, "seconds_eig": info.seconds_eig,
                         "eig_cycles": info.eig_cycles, "dv_ha": info.dv, "fermi_ha": info.mu,
                         "nelec": info.nelec, "lowest_ha": float(ev.min())}
    h.close()
    # the 4x4 graphene cell with the same core charges (128 electrons in 80 bands)
    wg = W.with_core(W.graphene(), SCF_Z, SCF_RCORE, name="graphene-scf")
    h = mb.Handle.from_workload(wg, device=local)
    evg, infog = h.scf(wg.nbands, SCF_TOL, SCF_SIGMA, mix_weight=SCF_W, g_max=SCF_GMAX, prec="fp32",
                       eig_tol=SCF_TOL / 5, max_iter=80, allow_notconv=True)
    out["graphene_mixed"] = {"workload": "graphene 4x4 (1417 G, 64x64 grid, 80 B-splines) with Z = %g core "
                                         "charges on its 32 atoms: 128 electrons in 80 bands" % SCF_Z,
                             "converged": bool(infog.dv < SCF_TOL), "iterations": infog.iterations,
                             "seconds": infog.seconds, "seconds_eig": infog.seconds_eig,
                             "seconds_density": infog.seconds_density, "eig_cycles": infog.eig_cycles,
                             "dv_ha": infog.dv, "fermi_ha": infog.mu, "nelec": infog.nelec}
    h.close()
    return out


def serve_run(mb, W, local, args, reqs, prec):
    """Replay `reqs` in real time (Poisson arrival times) into a fresh
    continuous-batching server; returns its record."""
    import torch
    free, total = torch.cuda.mem_get_info(local)
    budget = 0.7 * free
    srv = mb.Server(device=local, slots=args.serve_slots, hbm_budget_bytes=budget)
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        dt = r.arrival_s - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        tickets.append(srv.submit(W.request_workload(r), r.nbands, 1e-6, prec))
    lats, phases, bad, cycles = [], [], 0, []
    for t in tickets:
        rc, ev, info, lat, ph = srv.wait(t, phases=True)
        bad += rc != 0
        lats.append(lat)
        phases.append(ph)
        cycles.append(info.cycles)
    elapsed = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    la = np.array(lats) * 1e3
    ph = np.array(phases)
    return {"requests": len(reqs), "slots": args.serve_slots, "hbm_budget_gb": budget / 1e9,
            "seconds": elapsed, "solves_per_s": len(reqs) / elapsed,
            "p50_ms": float(np.percentile(la, 50)), "p99_ms": float(np.percentile(la, 99)),
            "mean_queue_ms": 1e3 * float(ph[:, 0].mean()), "mean_setup_ms": 1e3 * float(ph[:, 1].mean()),
            "mean_solve_ms": 1e3 * float(ph[:, 2].mean()),
            "setup_share_of_busy": float(ph[:, 1].sum() / max(1e-12, ph[:, 1:].sum())),
            "failed": int(bad), "peak_running": st["peak_running"], "peak_gb": st["peak_bytes"] / 1e9}


def serve_bench(mb, W, local, args):
    """Config 4, the serving stream: 256 Poisson arrivals (50/s) of slab
    solves drawn from the tiny/slab/graphene workloads (Nz 40-160, 8-80
    bands, 1-8 k-points), replayed in real time into the continuous-batching
    server.  The whole stream in mixed precision, and -- the comparison the
    stream's FP64 cost allows -- its first --serve-cmp-n requests through a
    mixed and a plain-FP64 server each."""
    reqs = W.serve_stream()
    out = {"mixed": serve_run(mb, W, local, args, reqs[:args.serve_n], "fp32")}
    if args.serve_cmp_n > 0:
        pre = reqs[:args.serve_cmp_n]
        cmp_m = serve_run(mb, W, local, args, pre, "fp32")
        cmp_p = serve_run(mb, W, local, args, pre, "fp64")
        out["prefix"] = {"requests": len(pre), "mixed": cmp_m, "fp64": cmp_p,
                         "mixed_speedup_vs_fp64": cmp_m["solves_per_s"] / cmp_p["solves_per_s"]}
    return out


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 1) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def run_reference(args):
    from paper_1406_4960_gb300 import workloads as W
    w = W.slab()
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline(w, budget_s=0.0, impl_steps=1)
    t0 = time.perf_counter()
    per_step = []
    gbs_all = []
    for _ in range(args.steps):
        gbs, cores, sample, secs, n = cpu_baseline(w, budget_s=0.0, impl_steps=1)
        per_step.append(secs)
        gbs_all.append(gbs)
    wall = time.perf_counter() - t0
    value = float(np.mean(gbs_all))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(per_step)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(1),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": "per step: 1 single-k-point H apply of the 32-band block in FP64 "
                                   "(the oracle; a bounded sample of the 4-k batched apply)"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line))


def config_of(world):
    """The benchmark configuration (both arms report the same one)."""
    return {"workload": "slab: C(001)-like, 12 atoms, Ecut 25 Ha, 32x16 grid, 120 B-splines, 4 k, 32 bands",
            "step": "one batched H apply, 4 k x 32 bands (precision: the line's dtype)",
            "l2": "flushed between timed steps, outside the events: a 256 MB buffer written, then another 256 MB read",
            "parallelism": "replica per GPU" if world > 1 else "1 GPU"}


def rank_env():
    """(world, rank, local rank) of a torchrun launch; (1, 0, 0) otherwise."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, world, device="cuda"):
    """The largest of every rank's x (the step time the job is charged)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(base, rank):
    """Each rank applies H to its own seeded block (independent replicas)."""
    return base + 7919 * rank


def job_gbs(bytes_per_rank, ms_max, world):
    """Whole-job throughput: the bytes all ranks processed over the slowest
    rank's time."""
    return world * bytes_per_rank / (ms_max * 1e-3) / 1e9


def probe_fp32_peak(lib, device):
    """Measured FP32 FMA throughput of this GPU (TFLOP/s), or None."""
    import ctypes
    fn = lib.mb_probe_fp32_fma
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    t, ms = ctypes.c_double(), ctypes.c_double()
    if fn(int(device), 5, ctypes.byref(t), ctypes.byref(ms)) != 0:
        return None
    return t.value


def plane_roofline(prof_plane, flops_per_step, steps, step_ms, kernel, workload, peak):
    """Roofline object of the plane kernel from its CUDA-event totals inside
    the timed steps (profiling mode 2)."""
    if "plane" not in prof_plane:
        return None
    t, c = prof_plane["plane"]
    per_launch_ms = t / c
    launches_per_step = max(1, c // steps)
    ach = flops_per_step / launches_per_step / (per_launch_ms * 1e-3) / 1e12
    traffic, note = plane_traffic(workload, kernel)
    derived = 152 * 128 * 2 * 2.070e-3
    p = peak if peak else derived
    return {"bound": "alu", "achieved": ach, "peak": p, "unit": "TFLOP/s", "frac": ach / p,
            "traffic": traffic, "traffic_source": note, "kernel": kernel,
            "peak_source": ("measured: FP32 FFMA loop on this GPU (mb_probe_fp32_fma), of measured"
                            if peak else "derived: 152 SM x 128 FP32 lanes x 2 x 2.07 GHz (probe failed)"),
            "kernel_ms": per_launch_ms, "share_of_step": t / steps / step_ms}


def run_ours(args):
    import ctypes
    import torch
    import torch.distributed as dist
    from paper_1406_4960_gb300 import mb, workloads as W

    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    def allmax(x):
        return max_over_ranks(x, world, "cuda")

    w = W.slab()
    lib = mb.load(build_if_missing=True)
    h = mb.Handle.from_workload(w, device=local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_rd = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_sink = torch.empty((), dtype=torch.float32, device="cuda")

    def flush_l2():
        # outside the timed events: write a buffer twice the L2, then read
        # another one, so every timed region starts from an L2 holding none
        # of its inputs and no dirty lines of the flush itself
        flush.zero_()
        torch.sum(flush_rd, dim=0, out=flush_sink)

    def blocks(hd, wd, prec, seed):
        dt = torch.complex128 if prec == "fp64" else torch.complex64
        Xs, Ys = [], []
        for ik in range(wd.nk):
            ng, nb, ldg = hd.sizes(ik)
            x = W.random_block(wd.nbands, nb, ng, seed=seed + ik, ld=ldg)
            Xs.append(torch.from_numpy(x).to(dt).cuda())
            Ys.append(torch.zeros_like(Xs[-1]))
        return Xs, Ys

    def read_profile(hd):
        prof = {}
        lib.mb_set_profiling(hd._h, 0)
        for kid in range(13):
            t, c = ctypes.c_double(), ctypes.c_longlong()
            lib.mb_profile_read(hd._h, kid, ctypes.byref(t), ctypes.byref(c))
            if c.value:
                prof[lib.mb_kernel_name(kid).decode()] = (t.value, c.value)
        return prof

    def timed(hd, wd, prec, steps, warmup, profile=0, sync_ranks=True):
        # profile: 0 none, 1 events around every kernel (a breakdown run),
        # 2 events around the plane kernel only (inside the timed steps)
        iks = list(range(wd.nk))
        Xs, Ys = blocks(hd, wd, prec, replica_seed(1000, rank))
        for _ in range(warmup):
            hd.apply_H_batch(iks, Xs, Ys, prec, stream)
        torch.cuda.synchronize()
        if profile:
            lib.mb_profile_reset(hd._h)
            lib.mb_set_profiling(hd._h, profile)
        n0 = lib.mb_launch_count(hd._h)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if sync_ranks:
            barrier()
        torch.cuda.synchronize()
        for i in range(steps):
            flush_l2()                         # L2 flush outside the timed events
            ev[i][0].record(stream)
            hd.apply_H_batch(iks, Xs, Ys, prec, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if sync_ranks:
            barrier()
        launches = lib.mb_launch_count(hd._h) - n0
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        prof = read_profile(hd) if profile else {}
        return (allmax(ms) if sync_ranks else ms), launches, prof

    if args.scf_only:
        h.close()
        print(json.dumps({"scf": scf_bench(mb, W, local, args)}))
        return
    if args.scf_steps_only:
        h.close()
        ws = scf_workload(W)
        hs = mb.Handle.from_workload(ws, device=local)
        ms, roof = scf_steps(mb, hs, ws, local)
        hs.close()
        print(json.dumps({"scf_steps_ms": ms, "density_roofline": roof}))
        return
    if args.serve_only:
        h.close()
        print(json.dumps({"serve": serve_bench(mb, W, local, args)}))
        return
    if args.eig_only:
        # one mixed and/or one plain-FP64 solve (for launch lists under ncu)
        if args.eig_workload != "slab":
            h.close()
            w = W.BY_NAME[args.eig_workload]()
            h = mb.Handle.from_workload(w, device=local)
        for prec in args.eig_prec.split(","):
            t0 = time.perf_counter()
            ev, info = h.eigsolve(w.nbands, 1e-6, prec)
            print(json.dumps({"eig_only": prec, "seconds": time.perf_counter() - t0, "cycles": info.cycles}))
        h.close()
        return
    if args.apply_only:
        # the FP32 batched apply of one workload only (for ncu captures)
        if args.apply_workload != "slab":
            h.close()
            w = W.BY_NAME[args.apply_workload]()
            h = mb.Handle.from_workload(w, device=local)
        tune = h.autotune(w.nbands, args.apply_prec) if args.apply_tune else None
        if args.apply_kernel is not None:
            h.plane_kernel_select(w.nk, w.nbands, args.apply_prec, args.apply_kernel, 0, args.apply_persistent)
        ms, _, _ = timed(h, w, args.apply_prec, args.steps, args.warmup)
        _, _, prof = timed(h, w, args.apply_prec, args.steps, 2, profile=2)
        if tune:
            print(h.autotune_report())
        print(json.dumps({"apply_only": args.apply_workload, "prec": args.apply_prec, "ms": ms, "autotune": tune,
                          "kernel": h.plane_kernel_name(w.nk, w.nbands, args.apply_prec),
                          "plane_ms": prof["plane"][0] / prof["plane"][1] if "plane" in prof else None}))
        h.close()
        return

    # launch shapes of the timed apply picked by the library's autotuner
    tune = h.autotune(w.nbands, "fp32")
    # the denominator of the plane kernel's roofline, measured just before
    # the timed region at the clocks the GPU is running
    peak32 = probe_fp32_peak(lib, local)
    # the timed FP32 steps bracket only the plane kernel with events (its
    # duration for the roofline, measured over the timed region)
    clocks = Clocks(local)
    clocks.start()
    ms32, launches, prof_plane = timed(h, w, "fp32", args.steps, args.warmup, profile=2)
    clk = clocks.stop()
    n32p, n64p, nbfp = min(args.steps, 20), 3, 3           # steps of the breakdown runs
    _, _, prof = timed(h, w, "fp32", n32p, 3, profile=1)
    ms64, _, _ = timed(h, w, "fp64", max(3, args.steps // 5), 3)
    _, _, prof64 = timed(h, w, "fp64", n64p, 1, profile=1)
    msbf, _, _ = timed(h, w, "bf16", max(3, args.steps // 5), 3)
    _, _, profbf = timed(h, w, "bf16", nbfp, 1, profile=1)

    # S and S^-1 (row a7) on the same blocks, all k-points in one batched
    # launch, FP32 and FP64; L2 flushed before each timed launch
    def timed_banded(which, prec, reps=10):
        Xs, Ys = blocks(h, w, prec, replica_seed(3000, rank))
        iks = list(range(w.nk))
        fn = h.apply_S_batch if which == "S" else h.apply_Sinv_batch
        for _ in range(3):
            fn(iks, Xs, Ys, prec, stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for i in range(reps):
            flush_l2()
            ev[i][0].record(stream)
            fn(iks, Xs, Ys, prec, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        h.status()
        ms = sum(a.elapsed_time(b) for a, b in ev) / reps
        byts = sum(2 * x.numel() * x.element_size() for x in Xs)     # read X, write Y
        return {"ms": ms, "GB/s": byts / (ms * 1e-3) / 1e9,
                "of_hbm_peak": byts / (ms * 1e-3) / 1e9 / _peaks().get("hbm_gbs", 6797.2),
                "launches": 1}

    banded = {"%s_%s" % (w_, p_): timed_banded(w_, p_) for w_ in ("S", "Sinv") for p_ in ("fp32", "fp64")}

    bytes32, flops32 = workload_sizes(h, w, "fp32")
    bytes64, _ = workload_sizes(h, w, "fp64")
    value = job_gbs(bytes32, ms32, world)

    # e2e: every step copies its X from pinned host memory, applies H and
    # copies Y back.  Steps are pipelined over two device buffer sets and three
    # streams (host->device copy, apply, device->host copy), so the copy
    # engines overlap the previous/next step's apply.
    iks = list(range(w.nk))
    sets = [blocks(h, w, "fp32", replica_seed(2000 + 10 * i, rank)) for i in range(2)]
    hX = [x.cpu().pin_memory() for x in sets[0][0]]
    hY = [[torch.empty_like(y, device="cpu").pin_memory() for y in sets[i][1]] for i in range(2)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    s_cmp = stream

    def e2e_run(nsteps):
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_cmp = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        used = [False, False]
        for i in range(nsteps):
            u = i % 2
            Xd, Yd = sets[u]
            if used[u]:
                s_in.wait_event(ev_cmp[u])          # the apply of step i-2 has read Xd
            with torch.cuda.stream(s_in):
                for a, b in zip(hX, Xd):
                    b.copy_(a, non_blocking=True)
            ev_in[u].record(s_in)
            s_cmp.wait_event(ev_in[u])
            if used[u]:
                s_cmp.wait_event(ev_out[u])         # the copy-out of step i-2 has read Yd
            h.apply_H_batch(iks, Xd, Yd, "fp32", s_cmp)
            ev_cmp[u].record(s_cmp)
            s_out.wait_event(ev_cmp[u])
            with torch.cuda.stream(s_out):
                for a, b in zip(Yd, hY[u]):
                    b.copy_(a, non_blocking=True)
            ev_out[u].record(s_out)
            used[u] = True
        return ev_out

    e2e_run(3)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    s_cmp.wait_event(e0)
    s_out.wait_event(e0)
    last = e2e_run(args.steps)
    for ev in last:
        s_in.wait_event(ev)
    e1.record(s_in)
    torch.cuda.synchronize()
    e2e_ms = allmax(e0.elapsed_time(e1) / args.steps)
    h2d = sum(x.numel() * x.element_size() for x in hX)
    d2h = sum(y.numel() * y.element_size() for y in hY[0])

    roof = plane_roofline(prof_plane, flops32, args.steps, ms32, h.plane_kernel_name(w.nk, w.nbands, "fp32"), "slab",
                          peak32)

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms32,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": config_of(world),
        "fp64_apply": {"value": job_gbs(bytes64, ms64, world), "unit": "GB/s", "ms_per_step": ms64},
        "kernels_ms_per_step": {k: v[0] / n32p for k, v in prof.items()},
        "kernels_ms_per_step_fp64": {k: v[0] / n64p for k, v in prof64.items()},
        "banded_S_Sinv": banded,
        "bf16_apply": {"value": job_gbs(bytes32, msbf, world), "unit": "GB/s", "ms_per_step": msbf,
                       "note": "FP32 planes, projector contractions in BF16 on tcgen05 tensor cores",
                       "kernels_ms_per_step": {k: v[0] / nbfp for k, v in profbf.items()}},
        "gpu_launches": int(launches),
        "e2e": {"value": job_gbs(bytes32, e2e_ms, world), "unit": "GB/s", "ms_per_step": e2e_ms,
                "pipeline": "2 buffer sets; H2D, apply and D2H on separate streams",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "roofline": roof,
        "autotune": tune,
        "fp32_peak_tflops_measured": peak32,
        "clocks": clk,
    }
    if not args.no_eig:
        line["eigsolve"] = eig_bench(h, w, args)
    h.close()
    if not args.no_graphene:
        line["graphene"] = graphene_bench(mb, W, local, args, timed, peak32)
    if not args.no_kbatch:
        line["kbatch"] = kbatch_bench(mb, W, local, args, timed, peak32)
    if not args.no_scf:
        line["scf"] = scf_bench(mb, W, local, args)
    if not args.no_serve:
        line["serve"] = serve_bench(mb, W, local, args)
    if rank == 0 and world == 1 and not args.no_cpu:
        gbs, cores, sample, secs, n = cpu_baseline(w, budget_s=args.cpu_budget)
        line["cpu_baseline"] = {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
                                "sample": sample, "seconds": secs, "solve": cpu_solve_tiny()}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-eig", action="store_true")
    ap.add_argument("--eig-only", action="store_true")
    ap.add_argument("--no-kbatch", action="store_true")
    ap.add_argument("--no-kbatch-solve", action="store_true")
    ap.add_argument("--no-graphene", action="store_true")
    ap.add_argument("--apply-only", action="store_true", help="time one FP32 batched apply only")
    ap.add_argument("--apply-workload", default="slab", help="workload of --apply-only")
    ap.add_argument("--apply-prec", default="fp32", help="precision of --apply-only")
    ap.add_argument("--apply-tune", action="store_true", help="autotune the launch shape of --apply-only")
    ap.add_argument("--apply-kernel", type=int, default=None, help="compact-plane instance id for --apply-only")
    ap.add_argument("--apply-persistent", action="store_true", help="persistent launch for --apply-kernel")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-scf", action="store_true")
    ap.add_argument("--scf-only", action="store_true", help="run the self-consistent loop section only")
    ap.add_argument("--scf-steps-only", action="store_true",
                    help="time the density, Coulomb and LDA steps of the loop's slab once (no loop)")
    ap.add_argument("--serve-n", type=int, default=256)
    ap.add_argument("--serve-cmp-n", type=int, default=12, help="requests of the mixed vs plain-FP64 server comparison")
    ap.add_argument("--serve-only", action="store_true", help="run the serving section only")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--eig-reps", type=int, default=6)
    ap.add_argument("--eig-prec", default="fp32,fp64", help="precisions of --eig-only (comma-separated)")
    ap.add_argument("--eig-workload", default="slab", help="workload of --eig-only (slab, graphene, kbatch, tiny)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
