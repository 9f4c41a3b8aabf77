"""Throughput benchmark of the spinor real-time propagation step.

Default workload (the headline): the large supercell -- 128 synthetic Z=8 atoms on a jittered
4x4x4 bcc lattice (a = 5.425 bohr, 21.7 bohr cube), 96^3 grid, Gamma point, 1024 occupied
spinors, L.S 0.02 Ha, Gaussian x-polarised laser in velocity gauge, dt = 0.04, ETRS with
Chebyshev exponentials and one corrector pass, FP32-mixed precision.  A step is one full ETRS
step over all spinors; the metric is spinor-grid-point updates per second, N_k N_occ N_g steps / s.
Extra blocks: the magnetic cluster (64^3, 104 spinors) with its FP64 comparison and propagator
variants, the bcc supercell (48^3, 8 k-points x 128 spinors), and the differentiation workload
(48^3 cluster, 500 steps, checkpoints every 50) timed forward + backward.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 (torchrun), every rank runs an independent replica (the path does not shard:
one GPU, no collectives); value = all ranks' updates / max-over-ranks time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spinor·gridpt updates/s; mixed vs FP64 path at |Δm(T)|≤1e-5; adjoint grad/s"
UNIT = "spinor*gridpt updates/s"
LASER = "laser E0=0.01 w=0.057 FWHM 10 fs x-pol velocity gauge, dt=0.04, ETRS + Chebyshev, n_sc=1"
WORKLOADS = {
    "large": ("large supercell: 128 synthetic Z=8 atoms, 4x4x4 bcc-like a=5.425 bohr jittered 0.1 bohr, "
              "21.7 bohr cube, 96^3 grid, Gamma, 1024 occupied spinors (of 1088), L.S 0.02 Ha, l<=2 KB "
              "projectors, " + LASER),
    "cluster": ("magnetic cluster: 13 synthetic Z=8 atoms, icosahedron 4.7 bohr, 24 bohr cube, 64^3 grid, "
                "104 occupied spinors (of 112), L.S 0.02 Ha, l<=2 KB projectors, " + LASER),
    "bcc": ("bcc supercell: 2x2x2 bcc a=5.42 bohr, 16 synthetic Z=8 atoms, L.S 0.02 Ha, 48^3 grid, "
            "8 Monkhorst-Pack k-points x 128 occupied spinors (of 144), static B_x=0.001 + " + LASER),
}


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- workload
def make_workload(name, nsteps, states=0, c64=True):
    """(workload, spinors) of one benchmark configuration; `states` > 0 keeps only the first
    spinors of each k-point (a small profiling case, not a benchmark line)."""
    from paper_2506_21908_gb300 import synthetic as S
    dt = np.complex64 if c64 else np.complex128
    if name == "large":
        wl = S.large(nsteps=nsteps)
        psi = S.large_states(wl, select=np.arange(states) if states else None, dtype=dt)
    elif name == "cluster":
        wl = S.cluster(n=64, nsteps=nsteps)
        psi = S.cluster_states(wl)
    elif name == "bcc":
        wl = S.bcc(nsteps=nsteps)
        psi = S.bcc_states(wl)
    else:
        raise ValueError(name)
    if states and psi.shape[1] > states:
        psi = psi[:, :states]
    psi = np.ascontiguousarray(psi, dtype=dt)
    wl.occ = np.ascontiguousarray(wl.occ[:, :psi.shape[1]])
    return wl, psi


# --------------------------------------------------------------------------- oracle timing
# One oracle process: builds the oracle for the workload with one spinor, then times a bounded
# sample of its step -- a Chebyshev series of order 2 (two Hamiltonian applications with the
# recurrence and accumulation) and one density + potential evaluation -- and scales it to the
# step's (K_full + 2 K_half) Hamiltonian applications and three density + potential evaluations.
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
from paper_2506_21908_gb300 import synthetic as S
from oracle import System, Oracle
from oracle.tddft import FieldTable, exp_chebyshev
name, idx, nrep = %(name)r, %(idx)d, %(nrep)d
if name == "large":
    wl = S.large(nsteps=16)
    psi = S.large_states(wl, select=[idx], dtype=np.complex128)
elif name == "cluster":
    wl = S.cluster(n=64, nsteps=16)
    psi = S.cluster_states(wl)[:, idx:idx + 1]
else:
    wl = S.bcc(nsteps=16)
    psi = S.bcc_states(wl)[:1, idx:idx + 1]
    wl.kpts, wl.kw = wl.kpts[:1], np.ones(1)
wl.occ = np.ones((1, 1))
s = System.from_workload(wl)
o = Oracle(s, FieldTable(wl.times, wl.A, wl.B), wl.dt, psi, n_sc=1, cheb_tol=1e-9)
A, B = o.f.at(0.0)
h = lambda x: s.apply_h(x, o.V, A)
out = []
for r in range(nrep):
    t0 = time.perf_counter()
    exp_chebyshev(h, o.psi, wl.dt, o.emin, o.emax, 2)
    t1 = time.perf_counter()
    s.potential(s.rho_v(o.psi), B)
    t2 = time.perf_counter()
    step = 0.5 * (t1 - t0) * (o.K_full + 2 * o.K_half) + 3 * (t2 - t1)
    out.append(step)
json.dump(dict(step_s=out, ng=wl.ng, K=[o.K_full, o.K_half]), sys.stdout)
"""


def time_oracle(name, procs, nrep=1):
    """Run `procs` single-threaded oracle processes at once (one spinor each, different spinors);
    returns the per-process results."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    ps = []
    for i in range(procs):
        code = ORACLE_SNIPPET % dict(root=ROOT, name=name, idx=(37 * i) % 100, nrep=nrep)
        ps.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                   text=True, env=env))
    res = []
    for p in ps:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("oracle timing failed: " + err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    return res


def cpu_baseline(name):
    """The oracle on one host core and on all host cores (one process per core, each with its own
    spinor): spinor-grid-point updates per second of a full ETRS step, from the bounded sample."""
    ncores = os.cpu_count() or 1
    one = time_oracle(name, 1)[0]
    allc = time_oracle(name, ncores) if ncores > 1 else [one]
    v1 = one["ng"] / one["step_s"][0]
    vall = len(allc) * allc[0]["ng"] / max(r["step_s"][0] for r in allc)
    sample = ("per process: one spinor of the %s workload, FP64 numpy oracle, single-threaded; timed: a "
              "Chebyshev series of order 2 (2 Hamiltonian applications) and one density + potential "
              "evaluation, scaled to the step's K_full + 2 K_half = %d applications and 3 evaluations; "
              "%d processes at once" % (name, sum(one["K"]) + one["K"][1], ncores))
    return {"value": vall, "unit": UNIT, "cores": len(allc), "kind": "oracle", "sample": sample,
            "cores_1": {"value": v1, "cores": 1, "step_s_per_spinor": one["step_s"][0]},
            "step_s_per_spinor_all_cores": max(r["step_s"][0] for r in allc)}


# --------------------------------------------------------------------------- ours
# CUDA sources that define each kernel class (its kernels, the device helpers they inline and
# the parameter structs they take).
KERNEL_SOURCES = {
    "epilogue": ("epilogue.cu", "proj_tile.cu", "bulk.cuh", "kepi.cuh", "fft.cuh", "impl.cuh", "kcommon.cuh"),
    "fft_xy": ("kernels.cu", "fft_tma.cu", "bulk.cuh", "fft.cuh", "impl.cuh", "kcommon.cuh"),
    "fft_z_kinetic": ("kernels.cu", "fft.cuh", "impl.cuh", "kcommon.cuh"),
    "proj_gather": ("kernels.cu", "proj_tile.cu", "bulk.cuh", "kepi.cuh", "fft.cuh", "impl.cuh", "kcommon.cuh"),
    "proj_scatter": ("proj_tile.cu", "bulk.cuh", "fft.cuh", "impl.cuh", "kcommon.cuh"),
}


def kernel_source_hash(kernel_class):
    """SHA-256 over the CUDA sources of one kernel class (all of them for a class not listed),
    to tie a stored ncu traffic figure to the kernels it measured."""
    import hashlib
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2506_21908_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel_class) or [f for f in os.listdir(src) if f.endswith((".cu", ".cuh"))]
    for f in sorted(files):
        path = os.path.join(src, f)
        if os.path.exists(path):
            h.update(f.encode())
            h.update(open(path, "rb").read())
    return h.hexdigest()


def measured_traffic(kernel_class, workload, units_per_launch):
    """DRAM bytes (read + write) per launch of `kernel_class` from the committed ncu summary
    profiles/traffic_<class>_<workload>.txt (bytes per spinor-gridpoint unit, averaged over the
    captured launches, plus an optional per-launch constant such as a table read once per launch),
    scaled to this launch size; None when there is no summary or the kernels changed since it was
    taken."""
    path = os.path.join(ROOT, "profiles", "traffic_%s_%s.txt" % (kernel_class, workload))
    if not os.path.exists(path):
        return None, "no ncu summary for this kernel and workload"
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith((" ", "#")):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256") != kernel_source_hash(kernel_class):
        return None, "kernels changed since the ncu capture (%s)" % os.path.basename(path)
    const = float(kv.get("dram_bytes_per_launch_const", "0"))
    return float(kv["dram_bytes_per_unit"]) * units_per_launch + const, os.path.basename(path)


def hbm_peak():
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(peaks["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy)"
    except Exception:
        return 6800.0, "fallback"


class Ctx:
    def __init__(self, torch, dist, stream):
        self.torch, self.dist, self.stream = torch, dist, stream

    def barrier(self):
        self.torch.cuda.synchronize()
        if self.dist is not None:
            self.dist.barrier()


def timed_steps(ctx, h, steps):
    """Time `steps` steps of handle h on the device (CUDA events on the handle's stream, barrier
    and synchronise on both sides) with the library's per-kernel-class profile."""
    torch = ctx.torch
    ctx.barrier()
    l0 = h.info()["launches"]
    h.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.barrier()
    e0.record()
    h.step(steps)
    e1.record()
    ctx.barrier()
    ms = e0.elapsed_time(e1)
    prof = h.profile_read()
    h.profile(False)
    return ms, prof, h.info()["launches"] - l0


def roofline_of(prof, units_per_launch, workload):
    dom = max(prof, key=lambda k: prof[k]["ms"])
    pk = prof[dom]
    hbm, src = hbm_peak()
    avg_ms = pk["ms"] / max(pk["launches"], 1)
    bytes_per_launch = pk["bytes"] / max(pk["launches"], 1)
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    traffic, tsrc = measured_traffic(dom, workload, units_per_launch)
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "peak_source": src, "traffic": traffic, "traffic_source": tsrc,
            "bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms,
            "share": pk["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-9)}


def kernel_table(prof):
    return {k: {"ms_total": v["ms"], "launches": v["launches"],
                "gbs": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 and v["bytes"] > 0 else None}
            for k, v in prof.items() if v["launches"]}


def run_ours(args):
    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2506_21908_gb300 import _lib
    from paper_2506_21908_gb300.replicas import aggregate

    # CPU oracle baseline first (separate processes, before any GPU work on this rank)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)

    stream = torch.cuda.current_stream().cuda_stream
    ctx = Ctx(torch, dist, stream)
    peaks = _lib.measure_peaks() if not args.no_peaks else None

    def max_over_ranks(x):
        return aggregate(0.0, x)[1]

    # ---------------- headline: FP32-mixed steps of the workload
    wl, psi0 = make_workload(args.workload, args.warmup + args.steps + 64, args.states)
    ups = wl.updates_per_step
    h = _lib.TDDFT.from_workload(wl, precision=_lib.FP32_MIXED, proj_mode=args.proj, stream=stream)
    h.set_fields(wl.times, wl.A, wl.B)
    psi_dev = torch.from_numpy(psi0).to("cuda")
    h.set_states(psi_dev, 0.0)
    del psi_dev
    torch.cuda.empty_cache()
    info = h.info()
    h.step(args.warmup)
    ctx.barrier()
    clk = ClockSampler(local)
    clk.start()
    ms, prof, launches = timed_steps(ctx, h, args.steps)
    clocks = clk.stop()
    total_units, sec = aggregate(ups * args.steps, ms / 1e3)  # replicas: sum of units, max of time
    ms_step = sec * 1e3 / args.steps
    value = total_units / sec
    units_per_launch = wl.nk * psi0.shape[1] * wl.ng
    roofline = roofline_of(prof, units_per_launch, args.workload)
    kernels = kernel_table(prof)
    _, _, E_mixed, norms = h.observables(fields=False, check=False)

    # ---------------- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        # the FP32-mixed handle takes its spinors as complex64 (tddft_set_states_c64)
        pinned = torch.from_numpy(np.ascontiguousarray(psi0, dtype=np.complex64)).pin_memory()
        n_out = np.empty((wl.n,) * 3)
        m_out = np.empty((3,) + (wl.n,) * 3)
        K2 = 2

        def e2e_iteration():
            h.set_states(pinned, 0.0)
            h.step(1)
            st = h.lib.tddft_observables(h.h, _lib._ptr(n_out), _lib._ptr(m_out), None, None, None)
            assert st in (0, -6), st

        e2e_iteration()  # untimed warm-up: first transfer from the freshly page-locked buffer
        ctx.barrier()
        t0 = time.perf_counter()
        for _ in range(K2):
            e2e_iteration()
        ctx.barrier()
        dt_e2e = max_over_ranks(time.perf_counter() - t0) / K2
        e2e = {"value": ups * world / dt_e2e, "unit": UNIT, "h2d_bytes_per_step": int(pinned.numel() * 8),
               "d2h_bytes_per_step": int(4 * wl.ng * 8), "ms_per_step": dt_e2e * 1e3,
               "what": "set_states_c64(pinned host complex64) + 1 step + observables(n, m to host), per iteration"}
        del pinned
    h.close()
    del psi0
    torch.cuda.empty_cache()

    # ---------------- the magnetic cluster: throughput, FP64 path and propagator variants
    cluster = None
    if not args.no_cluster and args.workload != "cluster":
        cluster = cluster_block(args, ctx, _lib, aggregate)

    # ---------------- the bcc supercell (k-points with Bloch phases)
    bcc = None
    if not args.no_bcc and args.workload != "bcc":
        bcc = throughput_block(args, ctx, _lib, aggregate, "bcc", steps=3)[0]

    # ---------------- adjoint gradient (differentiation workload)
    adjoint = None
    if not args.no_adjoint:
        adjoint = adjoint_block(args, ctx, _lib, max_over_ranks)

    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload] if not args.states else
                   WORKLOADS[args.workload] + " [profiling case: %d spinors per k]" % psi0_states(wl),
                   "precision": "FP32-mixed (c64 spinors/FFT/potential/projectors; f64 density, XC, Hartree, "
                                "energies)", "grid": wl.n, "spinors_per_k": psi0_states(wl), "kpoints": wl.nk,
                   "atoms": len(wl.pos), "K_full": info["K_full"], "K_half": info["K_half"],
                   "l2": "inputs larger than L2: %.0f MB spinor array per pass" % (units_per_launch * 16 / 1e6),
                   "projector_contraction": PROJ_NAMES[args.proj],
                   "parallelism": "replicas only" if world > 1 else "single GPU"},
        "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "measured_peaks_tflops": peaks, "M_final": E_mixed["M"].tolist(), "max_norm_error": float(np.abs(norms - 1.0).max()),
        "cluster": cluster, "bcc": bcc, "adjoint": adjoint,
    }
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


PROJ_NAMES = {1: "FP32 CUDA cores", 2: "TF32 tensor cores (tcgen05, brick by brick)",
              3: "split TF32 x3 tensor cores (tcgen05, brick by brick)",
              4: "split BF16 x3 tensor cores (tcgen05, brick by brick)",
              5: "split FP16 x3 tensor cores (tcgen05, brick by brick)"}


def psi0_states(wl):
    return int(wl.occ.shape[1])


def throughput_block(args, ctx, _lib, aggregate, name, steps, warm=2):
    """FP32-mixed throughput of another configuration (not the headline)."""
    wl, psi0 = make_workload(name, warm + steps + 8)
    h = _lib.TDDFT.from_workload(wl, precision=_lib.FP32_MIXED, proj_mode=args.proj, stream=ctx.stream)
    h.set_fields(wl.times, wl.A, wl.B)
    h.set_states(psi0, 0.0)
    info = h.info()
    h.step(warm)
    ms, prof, launches = timed_steps(ctx, h, steps)
    units, sec = aggregate(wl.updates_per_step * steps, ms / 1e3)
    rec = {"workload": WORKLOADS[name], "value": units / sec, "unit": UNIT, "ms_per_step": sec * 1e3 / steps,
           "steps": steps, "K_full": info["K_full"], "K_half": info["K_half"], "gpu_launches": launches,
           "roofline": roofline_of(prof, wl.nk * psi0.shape[1] * wl.ng, name), "kernels": kernel_table(prof)}
    h.close()
    return rec, wl, psi0


def cluster_block(args, ctx, _lib, aggregate):
    torch = ctx.torch
    rec, wl, psi0 = throughput_block(args, ctx, _lib, aggregate, "cluster", steps=10, warm=3)
    ups = wl.updates_per_step
    nst = 3 + 10
    # mixed-vs-FP64 on the same start (the mixed run again from t = 0 for nst steps)
    g = _lib.TDDFT.from_workload(wl, precision=_lib.FP32_MIXED, proj_mode=args.proj, stream=ctx.stream)
    g.set_fields(wl.times, wl.A, wl.B)
    g.set_states(psi0, 0.0)
    g.step(args.fp64_steps)
    n32, m32, E32, _ = g.observables(fields=True, check=False)
    g.close()
    if not args.no_fp64:
        g = _lib.TDDFT.from_workload(wl, precision=_lib.FP64, stream=ctx.stream)
        g.set_fields(wl.times, wl.A, wl.B)
        g.set_states(psi0.astype(np.complex128), 0.0)
        _, _, E0, _ = g.observables(fields=False, check=False)
        g.step(1)
        ctx.barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        g.step(2)
        f1.record()
        ctx.barrier()
        ms64 = f0.elapsed_time(f1) / 2
        g.step(args.fp64_steps - 3)
        n64, m64, E64, _ = g.observables(fields=True, check=False)
        g.close()
        rec["fp64"] = {"value": ups / (ms64 / 1e3), "ms_per_step": ms64,
                       "speedup_mixed_vs_fp64": ms64 / rec["ms_per_step"],
                       "steps_compared": args.fp64_steps,
                       "dM_per_atom_muB": float(np.linalg.norm(E32["M"] - E64["M"]) / len(wl.pos)),
                       "max_dn_rel": float(np.abs(n32 - n64).max() / np.abs(n64).max()),
                       "max_dm_rel": float(np.abs(m32 - m64).max() / np.abs(m64).max()),
                       "dE_Ha": float(abs(E32["total"] - E64["total"])),
                       "E_drift_fp64_Ha": float(E64["total"] - E0["total"])}
    if not args.no_propagators:
        props = {"steps": nst, "reference": "Chebyshev ETRS, same start"}
        for name, kind in (("taylor4", _lib.EXP_TAYLOR), ("crank_nicolson", _lib.EXP_CRANK_NICOLSON)):
            g = _lib.TDDFT.from_workload(wl, precision=_lib.FP32_MIXED, exp_kind=kind, stream=ctx.stream)
            g.set_fields(wl.times, wl.A, wl.B)
            g.set_states(psi0, 0.0)
            gi = g.info()
            terms = (gi["K_full"] + 2 * gi["K_half"]) if kind == _lib.EXP_CRANK_NICOLSON else 12
            p = {"K_full": gi["K_full"], "K_half": gi["K_half"], "h_applies_per_step": terms}
            try:
                g.step(1)
                ctx.barrier()
                p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                p0.record()
                g.step(2)
                p1.record()
                ctx.barrier()
                msp = p0.elapsed_time(p1) / 2
                p.update(ms_per_step=msp, value=ups / (msp / 1e3))
                g.step(args.fp64_steps - 3)
                _, _, Ep, nrm = g.observables(fields=False, check=False)
                p.update(dM_per_atom_muB_vs_chebyshev=float(np.linalg.norm(Ep["M"] - E32["M"]) / len(wl.pos)),
                         max_norm_error=float(np.abs(nrm - 1.0).max()), status=int(Ep["status"]))
            except _lib.TddftError as err:  # e.g. Taylor-4 leaving the spectral window (unstable)
                ctx.barrier()
                p.update(status=err.status, error=str(err)[:160])
            g.close()
            props[name] = p
        rec["propagators"] = props
    return rec


def adjoint_block(args, ctx, _lib, max_over_ranks):
    """The differentiation workload: 13-atom cluster at 48^3, 104 spinors, 64-sample laser
    envelope, L = M_z(T) after `adj_steps` steps with checkpoints every `adj_ckpt`; one gradient =
    the forward run and the discrete-adjoint backward run through the autograd wrapper."""
    torch = ctx.torch
    from paper_2506_21908_gb300 import synthetic as S
    from paper_2506_21908_gb300.autograd import MagnetizationFromPulse, PulseBasis, mz_seed
    nst = args.adj_steps
    dwl = S.cluster(n=48, nsteps=nst, laser=False)
    dpsi = S.cluster_states(dwl)
    basis = PulseBasis(dwl.times, 64, mode="laser", omega=0.057)
    a0 = np.random.default_rng(20250624).uniform(0.0, 0.01, 64)
    res = {}
    precs = [(_lib.FP32_MIXED, "fp32_mixed")] + ([(_lib.FP64, "fp64")] if args.adj_fp64 else [])
    for prec, name in precs:
        hd = _lib.TDDFT.from_workload(dwl, precision=prec, stream=ctx.stream)
        a = torch.tensor(a0, requires_grad=True)
        ctx.barrier()
        t0 = time.perf_counter()
        L = MagnetizationFromPulse.apply(a, hd, dpsi, basis, nst, mz_seed(48, dwl.L), args.adj_ckpt)
        L.backward()
        ctx.barrier()
        dt_g = max_over_ranks(time.perf_counter() - t0)
        res[name] = {"seconds": dt_g, "grad_per_s": 1.0 / dt_g, "loss": float(L.detach()),
                     "grad_norm": float(a.grad.norm())}
        hd.close()
    return {"workload": "13-atom cluster, 48^3, 104 spinors, 64-sample laser envelope, L = M_z(T)",
            "steps": nst, "ckpt_every": args.adj_ckpt, "per_precision": res,
            "what": "forward + discrete-adjoint backward of the whole horizon, one 64-parameter gradient (measured)"}


# --------------------------------------------------------------------------- accuracy over a horizon
def run_horizon(args):
    """Mixed (FP32, the bench's projector mode) against the FP64 path on the same start over a long
    horizon: |dM| per atom (mu_B), max |dn| and |dm| relative to the FP64 fields, the total
    energies and the FP64 path's own energy drift, every `--horizon-every` steps.  One JSON line
    per configuration (not a throughput line)."""
    import torch
    from paper_2506_21908_gb300 import _lib
    stream = torch.cuda.current_stream().cuda_stream
    plan = [("cluster", args.horizon), ("bcc", args.horizon_bcc), ("large", args.horizon_large)]
    for name, nst in plan:
        if nst <= 0:
            continue
        wl, psi0 = make_workload(name, nst + 8)
        every = max(1, min(args.horizon_every, nst))
        hs = []
        for prec, proj in ((_lib.FP32_MIXED, args.proj), (_lib.FP64, None)):
            h = _lib.TDDFT.from_workload(wl, precision=prec, proj_mode=proj, stream=stream)
            h.set_fields(wl.times, wl.A, wl.B)
            h.set_states(psi0, 0.0)
            hs.append(h)
        info32, info64 = hs[0].info(), hs[1].info()
        rows = []
        t_wall = time.time()
        E0 = None
        for done in range(0, nst + 1, every):
            if done:
                for h in hs:
                    h.step(every)
            torch.cuda.synchronize()
            obs = [h.observables(fields=True, check=False) for h in hs]
            (n32, m32, E32, _), (n64, m64, E64, _) = obs
            if E0 is None:
                E0 = E64["total"]
            rows.append({"step": done, "t": E64["t"],
                         "dM_per_atom_muB": float(np.linalg.norm(E32["M"] - E64["M"]) / len(wl.pos)),
                         "max_dn_rel": float(np.abs(n32 - n64).max() / np.abs(n64).max()),
                         "max_dm_rel": float(np.abs(m32 - m64).max() / np.abs(m64).max()),
                         "E_fp32": E32["total"], "E_fp64": E64["total"], "E_fp64_drift": E64["total"] - E0,
                         "M_fp64": E64["M"].tolist()})
        for h in hs:
            h.close()
        print(json.dumps({"horizon": name, "workload": WORKLOADS[name], "steps": nst, "every": every,
                          "projector_contraction": PROJ_NAMES[args.proj], "K_fp32": [info32["K_full"], info32["K_half"]],
                          "K_fp64": [info64["K_full"], info64["K_half"]], "wall_s": time.time() - t_wall,
                          "max_dM_per_atom_muB": max(r["dM_per_atom_muB"] for r in rows), "rows": rows}), flush=True)


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 CPU oracle on the host cores (one single-threaded process per core, one spinor
    each), each step the bounded sample of time_oracle, on the headline workload."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    ncores = os.cpu_count() or 1
    res = time_oracle(args.workload, ncores, nrep=args.warmup + args.steps)
    per_step = [max(r["step_s"][i] for r in res) for i in range(args.warmup, args.warmup + args.steps)]
    t = statistics.mean(per_step)
    value = ncores * res[0]["ng"] / t
    sample = ("each step: %d single-threaded FP64 numpy oracle processes at once, one spinor of the %s "
              "workload each; timed: a Chebyshev series of order 2 and one density + potential evaluation, "
              "scaled to a full ETRS step (K = %s)" % (ncores, args.workload, res[0]["K"]))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOADS[args.workload], "precision": "FP64 CPU oracle", "sample": sample},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=25, help="steps of the cluster's mixed-vs-FP64 comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-cluster", action="store_true")
    ap.add_argument("--no-bcc", action="store_true")
    ap.add_argument("--no-peaks", action="store_true", help="skip the FMA / tensor-core peak microbenchmarks")
    ap.add_argument("--proj", type=int, default=5, help="projector contraction: " + str(PROJ_NAMES))
    ap.add_argument("--no-propagators", action="store_true", help="skip the Taylor-4 / Crank-Nicolson comparison")
    ap.add_argument("--adj-steps", type=int, default=500)
    ap.add_argument("--adj-ckpt", type=int, default=50)
    ap.add_argument("--adj-fp64", action="store_true", help="also time the FP64 adjoint (slow)")
    ap.add_argument("--states", type=int, default=0,
                    help="propagate only the first N spinors (small profiling case; not the headline)")
    ap.add_argument("--horizon", type=int, default=0,
                    help="accuracy run instead of the benchmark: cluster steps of mixed against FP64")
    ap.add_argument("--horizon-bcc", type=int, default=0)
    ap.add_argument("--horizon-large", type=int, default=0)
    ap.add_argument("--horizon-every", type=int, default=50)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.horizon or args.horizon_bcc or args.horizon_large:
        run_horizon(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
