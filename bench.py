"""Throughput benchmark of the spinor real-time propagation step.

Default workload: the magnetic-cluster case -- 13 synthetic Z=8 atoms on an icosahedron
(centre-vertex 4.7 bohr) in a 24 bohr cube, 64^3 grid, 104 occupied spinors, L.S 0.02 Ha,
Gaussian x-polarised laser in velocity gauge, dt = 0.04, ETRS with Chebyshev exponentials
and one corrector pass, FP32-mixed precision.  A step is one full ETRS step over all
spinors; the metric is spinor-grid-point updates per second, N_k N_occ N_g steps / s.

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
WORKLOAD = ("magnetic cluster: 13 synthetic Z=8 atoms, icosahedron 4.7 bohr, 24 bohr cube, 64^3 grid, "
            "104 occupied spinors (of 112), L.S 0.02 Ha, l<=2 KB projectors, laser E0=0.01 w=0.057 "
            "FWHM 10 fs x-pol velocity gauge, dt=0.04, ETRS + Chebyshev, n_sc=1")


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
def cluster_workload(nsteps):
    from paper_2506_21908_gb300 import synthetic as S
    wl = S.cluster(n=64, nsteps=nsteps)
    return wl


def make_states(wl):
    from paper_2506_21908_gb300 import synthetic as S
    return S.cluster_states(wl)


# --------------------------------------------------------------------------- oracle timing
ORACLE_SNIPPET = r"""
import json, sys, time, os
sys.path.insert(0, %(root)r)
import numpy as np
from paper_2506_21908_gb300 import synthetic as S
from oracle import System, Oracle
from oracle.tddft import FieldTable
wl = S.cluster(n=64, nsteps=%(nsteps)d)
nb = %(nbands)d
psi = S.atomic_orbital_states(wl.L, wl.n, wl.pos, wl.kpts, S.cluster_axes(len(wl.pos)), seed=wl.seed)[:, :nb]
wl.occ = wl.occ[:, :nb]
s = System.from_workload(wl)
o = Oracle(s, FieldTable(wl.times, wl.A, wl.B), wl.dt, psi, n_sc=1)
times = []
for i in range(%(warm)d + %(steps)d):
    t0 = time.perf_counter(); o.step(); times.append(time.perf_counter() - t0)
json.dump(dict(times=times[%(warm)d:], nbands=nb, ng=wl.ng, K=[o.K_full, o.K_half]), sys.stdout)
"""


def time_oracle(nbands, steps, warm=0):
    """Run the oracle single-threaded in a separate process on a sample of bands."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET % dict(root=ROOT, nsteps=max(16, warm + steps + 2), nbands=nbands, warm=warm, steps=steps)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d


# --------------------------------------------------------------------------- ours
# CUDA sources that define each kernel class (its kernels, the device helpers they inline and
# the parameter structs they take).
KERNEL_SOURCES = {
    "epilogue": ("epilogue.cu", "kepi.cuh", "fft.cuh", "impl.cuh", "kcommon.cuh"),
    "fft_xy": ("kernels.cu", "fft_tma.cu", "bulk.cuh", "fft.cuh", "impl.cuh", "kcommon.cuh"),
    "fft_z_kinetic": ("kernels.cu", "kin_cluster.cu", "fft.cuh", "impl.cuh", "kcommon.cuh"),
    "proj_gather": ("kernels.cu", "proj_tc.cu", "kepi.cuh", "fft.cuh", "impl.cuh", "kcommon.cuh"),
}


def kernel_source_hash(kernel_class):
    """SHA-256 over the CUDA sources of one kernel class (all of them for a class not listed),
    to tie a stored ncu traffic figure to the kernels it measured."""
    import hashlib
    h = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2506_21908_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel_class) or [f for f in os.listdir(src) if f.endswith((".cu", ".cuh"))]
    for f in sorted(files):
        h.update(f.encode())
        h.update(open(os.path.join(src, f), "rb").read())
    return h.hexdigest()


def measured_traffic(kernel_class, units_per_launch):
    """DRAM bytes (read + write) per launch of `kernel_class` from the committed ncu summary
    profiles/traffic_<class>_cluster64_fp32mixed.txt (bytes per spinor-gridpoint unit, averaged over
    the launches of one step), scaled to this launch size; None when there is no summary or the
    kernels changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic_%s_cluster64_fp32mixed.txt" % kernel_class)
    if not os.path.exists(path):
        return None, "no ncu summary for this kernel"
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith((" ", "#")):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256") != kernel_source_hash(kernel_class):
        return None, "kernels changed since the ncu capture (%s)" % os.path.basename(path)
    return float(kv["dram_bytes_per_unit"]) * units_per_launch, os.path.basename(path)


def run_ours(args):
    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2506_21908_gb300 import _lib

    # CPU oracle baseline first (separate process, before heavy GPU work on this rank)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        d = time_oracle(nbands=args.oracle_bands, steps=1)
        t = statistics.mean(d["times"])
        cpu = {"value": d["nbands"] * d["ng"] / t, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "one ETRS step of the cluster workload restricted to %d of 104 spinors (FP64 numpy, "
                         "K=%s, %.1f s)" % (d["nbands"], d["K"], t)}

    wl = cluster_workload(args.warmup + args.steps + 64)
    psi0 = make_states(wl)
    if args.states:
        psi0 = np.ascontiguousarray(psi0[:, :args.states])
        wl.occ = wl.occ[:, :args.states]
    ups = wl.updates_per_step
    stream = torch.cuda.current_stream().cuda_stream

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    from paper_2506_21908_gb300.replicas import aggregate

    def max_over_ranks(x):
        return aggregate(0.0, x)[1]

    # ---------------- mixed precision (the headline)
    h = _lib.TDDFT.from_workload(wl, precision=_lib.FP32_MIXED, proj_mode=args.proj, stream=stream)
    h.set_fields(wl.times, wl.A, wl.B)
    psi_dev = torch.from_numpy(psi0).to("cuda")
    h.set_states(psi_dev, 0.0)
    info = h.info()
    h.step(args.warmup)
    barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = h.info()["launches"]
    h.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record()
    h.step(args.steps)
    e1.record()
    barrier()
    ms = e0.elapsed_time(e1)
    prof = h.profile_read()
    h.profile(False)
    launches = h.info()["launches"] - l0
    clocks = clk.stop()
    total_units, sec = aggregate(ups * args.steps, ms / 1e3)  # replicas: sum of units, max of time
    ms_step = sec * 1e3 / args.steps
    value = total_units / sec
    _, _, E_mixed, _ = h.observables(fields=False, check=False)
    M_mixed = E_mixed["M"]

    # roofline of the dominant kernel class
    dom = max(prof, key=lambda k: prof[k]["ms"])
    pk = prof[dom]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm = float(peaks["hbm_gbs"])
        peak_src = "measured"
    except Exception:
        hbm = 6800.0
        peak_src = "fallback"
    avg_ms = pk["ms"] / max(pk["launches"], 1)
    bytes_per_launch = pk["bytes"] / max(pk["launches"], 1)
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    traffic, traffic_src = measured_traffic(dom, wl.nk * psi0.shape[1] * wl.ng)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": peak_src, "traffic": traffic, "traffic_source": traffic_src,
                "bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms,
                "share": pk["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-9)}
    kernels = {k: {"ms_total": v["ms"], "launches": v["launches"],
                   "gbs": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 and v["bytes"] > 0 else None}
               for k, v in prof.items() if v["launches"]}

    # ---------------- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        # the FP32-mixed handle takes its spinors as complex64 (tddft_set_states_c64)
        pinned = torch.from_numpy(psi0.astype(np.complex64)).pin_memory()
        n_out = np.empty((wl.n,) * 3)
        m_out = np.empty((3,) + (wl.n,) * 3)
        K2 = max(2, min(args.steps, 5))

        def e2e_iteration():
            h.set_states(pinned, 0.0)
            h.step(1)
            st = h.lib.tddft_observables(h.h, _lib._ptr(n_out), _lib._ptr(m_out), None, None, None)
            assert st in (0, -6), st

        e2e_iteration()  # untimed warm-up: first transfer from the freshly page-locked buffer
        barrier()
        t0 = time.perf_counter()
        for _ in range(K2):
            e2e_iteration()
        barrier()
        dt_e2e = max_over_ranks(time.perf_counter() - t0) / K2
        e2e = {"value": ups * world / dt_e2e, "unit": UNIT, "h2d_bytes_per_step": int(pinned.numel() * 8),
               "d2h_bytes_per_step": int(4 * wl.ng * 8), "ms_per_step": dt_e2e * 1e3,
               "what": "set_states_c64(pinned host complex64) + 1 step + observables(n, m to host), per iteration"}
    h.close()
    del psi_dev

    # ---------------- FP64 GPU path (same start, fewer steps) and mixed-vs-FP64 magnetisation
    fp64 = None
    if not args.no_fp64:
        nst = args.warmup + args.steps
        g = _lib.TDDFT.from_workload(wl, precision=_lib.FP64, stream=stream)
        g.set_fields(wl.times, wl.A, wl.B)
        g.set_states(psi0, 0.0)
        g.step(1)
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        g.step(2)
        f1.record()
        barrier()
        ms64 = f0.elapsed_time(f1) / 2
        g.step(nst - 3)
        _, _, E64, _ = g.observables(fields=False, check=False)
        g.close()
        dm = float(np.linalg.norm(M_mixed - E64["M"]) / len(wl.pos))
        fp64 = {"value": ups / (ms64 / 1e3), "ms_per_step": ms64, "speedup_mixed_vs_fp64": (ups / (ms_step / 1e3)) / (ups / (ms64 / 1e3)),
                "dm_per_atom_muB": dm, "steps_compared": nst, "K_fp64": None}

    # ---------------- propagator comparison: Taylor-4 and Crank-Nicolson against Chebyshev
    propagators = None
    if not args.no_propagators:
        nst = args.warmup + args.steps
        propagators = {"steps": nst, "reference": "Chebyshev ETRS (the headline path), same start"}
        for name, kind in (("taylor4", _lib.EXP_TAYLOR), ("crank_nicolson", _lib.EXP_CRANK_NICOLSON)):
            g = _lib.TDDFT.from_workload(wl, precision=_lib.FP32_MIXED, exp_kind=kind, stream=stream)
            g.set_fields(wl.times, wl.A, wl.B)
            g.set_states(psi0, 0.0)
            gi = g.info()
            terms = (gi["K_full"] + 2 * gi["K_half"]) if kind == _lib.EXP_CRANK_NICOLSON else 12
            rec = {"K_full": gi["K_full"], "K_half": gi["K_half"], "h_applies_per_step": terms}
            try:
                g.step(1)
                barrier()
                p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                p0.record()
                g.step(2)
                p1.record()
                barrier()
                msp = p0.elapsed_time(p1) / 2
                rec.update(ms_per_step=msp, value=ups / (msp / 1e3))
                g.step(nst - 3)
                _, _, Ep, nrm = g.observables(fields=False, check=False)
                rec.update(dm_per_atom_muB_vs_chebyshev=float(np.linalg.norm(Ep["M"] - M_mixed) / len(wl.pos)),
                           max_norm_error=float(np.abs(nrm - 1.0).max()), status=int(Ep["status"]))
            except _lib.TddftError as err:  # e.g. Taylor-4 leaving the spectral window (unstable)
                barrier()
                rec.update(status=err.status, error=str(err)[:160])
            g.close()
            propagators[name] = rec
        propagators["chebyshev"] = {"ms_per_step": ms_step, "K_full": info["K_full"], "K_half": info["K_half"],
                                    "h_applies_per_step": info["K_full"] + 2 * info["K_half"]}

    # ---------------- adjoint gradient (differentiation workload, bounded horizon)
    adjoint = None
    if not args.no_adjoint:
        from paper_2506_21908_gb300 import synthetic as S
        from paper_2506_21908_gb300.autograd import MagnetizationFromPulse, PulseBasis, mz_seed
        nst = args.adj_steps
        dwl = S.cluster(n=48, nsteps=nst, laser=False)
        dpsi = S.cluster_states(dwl)
        basis = PulseBasis(dwl.times, 64, mode="laser", omega=0.057)
        a0 = np.random.default_rng(20250624).uniform(0.0, 0.01, 64)
        res = {}
        for prec, name in ((_lib.FP32_MIXED, "fp32_mixed"), (_lib.FP64, "fp64")):
            hd = _lib.TDDFT.from_workload(dwl, precision=prec, stream=stream)
            a = torch.tensor(a0, requires_grad=True)
            barrier()
            t0 = time.perf_counter()
            L = MagnetizationFromPulse.apply(a, hd, dpsi, basis, nst, mz_seed(48, dwl.L), args.adj_ckpt)
            L.backward()
            barrier()
            dt_g = max_over_ranks(time.perf_counter() - t0)
            res[name] = {"seconds": dt_g, "grad_per_s": 1.0 / dt_g, "loss": float(L.detach()),
                         "grad_norm": float(a.grad.norm())}
            hd.close()
        g32 = None
        adjoint = {"workload": "13-atom cluster, 48^3, 104 spinors, 64-sample laser envelope, L = M_z(T)",
                   "steps": nst, "ckpt_every": args.adj_ckpt, "per_precision": res,
                   "grad_per_s_500_steps_est": {k: 1.0 / (v["seconds"] * 500.0 / nst) for k, v in res.items()},
                   "what": "forward + discrete-adjoint backward of the whole horizon, one 64-parameter gradient"}

    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "FP32-mixed (c64 spinors/FFT/potential/projectors; "
                   "f64 density, XC, Hartree, energies)", "grid": 64, "spinors": 104, "K_full": info["K_full"],
                   "K_half": info["K_half"], "l2": "inputs larger than L2: 436 MB spinor array per pass",
                   "projector_contraction": {1: "FP32 CUDA cores", 2: "TF32 tensor cores (tcgen05)",
                                             3: "3xTF32 tensor cores (tcgen05)"}[args.proj],
                   "parallelism": "replicas only" if world > 1 else "single GPU"},
        "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "fp64": fp64, "propagators": propagators, "adjoint": adjoint,
    }
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    d = time_oracle(nbands=1, steps=args.steps, warm=args.warmup)
    ts = d["times"]
    t = statistics.mean(ts)
    value = d["nbands"] * d["ng"] / t
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "precision": "FP64 CPU oracle",
                                "sample": "%d of 104 spinors per step" % d["nbands"]},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": "each step: one ETRS step of the cluster workload on %d of 104 spinors "
                                      "(numpy FP64, single thread)" % d["nbands"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--oracle-bands", type=int, default=2)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--proj", type=int, default=1,
                    help="projector contraction: 1 FP32 CUDA cores, 2 TF32 tensor cores, 3 TF32x3 tensor cores")
    ap.add_argument("--no-propagators", action="store_true", help="skip the Taylor-4 / Crank-Nicolson comparison")
    ap.add_argument("--adj-steps", type=int, default=20)
    ap.add_argument("--adj-ckpt", type=int, default=10)
    ap.add_argument("--states", type=int, default=0,
                    help="propagate only the first N spinors (small profiling case; not the headline)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
