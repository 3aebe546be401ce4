"""Benchmark of the lattice Boltzmann hot path on GB300.

Workload (the pipe-flow configuration of Sec. 2.1 on a reduced grid): a
periodic pipe of diameter 146 lu and length 438 lu in a 148x148x438 D3Q19
grid, FP32 populations, SRT collision, nu = 0.0032 (Table 1), body force from
Re_tau = 180, initial laminar profile plus 5 % seeded divergence-free
perturbations (synthetic stand-in for the developed turbulent pipe flow).
One step = one lbm_step: the fused pull-stream-collide sweep with the linear
interpolated bounce-back wall. The populations (2 x 1.46 GB) are far larger
than L2, so no flush is needed between steps.

Also reported in the same line: the IBM-B wall, FP16/BF16 population storage,
and the particle-laden 256^3 box with 2000 moving spheres (IBB and IBM-B), the
oracle (CPU, FP64) on a bounded sample of the pipe, and the end-to-end rate
through the C ABI with the initial field uploaded from pinned host memory and
the final velocity field read back.

--impl reference times the oracle (the plain CPU implementation) on a
148x148x32 slab of the same pipe per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

PIPE = workloads.PIPE_148
PP = workloads.pipe_parameters(PIPE["radius"], PIPE["nu"], PIPE["re_tau"])
NZ = PIPE["nz"]  # pipe length; --nz shortens it for profiler captures
HBM_FALLBACK = 6800.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


def pipe_field(nz=None):
    nz = nz or NZ
    return workloads.pipe_velocity(PIPE["nx"], PIPE["ny"], nz, PIPE["radius"], PP["u_bulk"],
                                   PIPE["perturbation"], seed=0)


# ------------------------------------------------------------------ clocks --
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.p = None
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="lbm_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower() == "active":
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------ replica timing ----
def max_over_ranks(torch, dist, ms, device):
    """Slowest rank's time: every replica waits for it."""
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(fluid_cells, steps, world, ms_max):
    """Whole-job rate: the cells of all replicas over the slowest time."""
    return fluid_cells * steps * world / (ms_max * 1e-3) / 1e6


# ------------------------------------------------------------- GPU runs ----
def run_case(lbm, torch, name, nx, ny, nz, tau, force, storage, rates, bc, steps, warmup, setup, fluid_cells=None,
             profile=True):
    """Build one context, warm up, time `steps` steps with CUDA events on the
    library's stream; returns MLUPS and the per-group kernel profile."""
    L = lbm.Lattice(nx, ny, nz, tau, force=force, storage=storage, rates=rates,
                    max_particles=setup.get("max_particles", 0))
    setup["init"](L)
    L.step(warmup, bc)
    torch.cuda.synchronize()
    if fluid_cells is None:
        fluid_cells = int(np.count_nonzero((L.flags() & 1) == 0)) if bc == lbm.BC_IBB else nx * ny * nz
    s = L.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if profile:
        L.profile_enable(True)
    torch.cuda.synchronize()
    e0.record(s)
    L.step(steps, bc)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = L.profile(0) if profile else None
    st = L.stats(0)
    ok = bool(np.isfinite(st["kinetic_energy"]))
    # algorithmic bytes of one sweep launch: every visited cell reads and
    # writes 19 populations; the flag byte is read where the sweep needs it
    # (the pipe's IBB sweep walks fluid-run segments and reads no flags)
    sb = {lbm.F64: 8, lbm.F32: 4}.get(storage, 2)
    N = nx * ny * nz
    if bc == lbm.BC_IBB:
        fluid = int(np.count_nonzero((L.flags() & 1) == 0))
        bulk_bytes = 2 * 19 * sb * fluid + (0 if setup.get("segments") else N)
    elif bc in (lbm.BC_IBM_U, lbm.BC_IBM_B):
        bulk_bytes = 2 * 19 * sb * N + N
    else:
        bulk_bytes = 2 * 19 * sb * N
    L.close()
    del L
    torch.cuda.empty_cache()
    return dict(name=name, ms=ms, steps=steps, mlups=fluid_cells * steps / (ms * 1e-3) / 1e6, fluid_cells=fluid_cells,
                bulk_bytes=bulk_bytes, ncells=N, prof=prof, finite=ok)


def pipe_setup(lbm, storage=None):
    u = pipe_field()

    def init(L):
        L.init_velocity(u)
        L.set_pipe(PIPE["radius"])
    return dict(init=init, segments=True)


def hit_setup(n, n_particles, seed=0):
    u = workloads.hit_velocity(n, seed=seed, k_peak=8.0, u_rms=0.03, dtype=np.float64)
    X = workloads.place_spheres((n, n, n), n_particles, 4.0, 1.0, seed=seed)

    def init(L):
        L.init_velocity(u)
        L.add_spheres(X, 4.0, density_ratio=5.0)
    return dict(init=init, max_particles=n_particles)


def config4_report(lbm, torch, n=512, n_particles=16000, steps=10, warmup=3):
    """512^3 particle-laden box with 16000 moving spheres of radius 4 (the
    3.2 % volume fraction of the 256^3 / 2000-sphere case), IBB, d'Humieres
    rates, tau = 0.51, under FP32, FP16 and BF16 population storage on the
    same GPU: MLUPS, step time, the bulk sweep's algorithmic GB/s. The
    initial field is the 256^3 synthetic HIT field tiled 2 x 2 x 2 (periodic
    and divergence-free; it sets the flow, not the throughput)."""
    u = np.tile(workloads.hit_velocity(n // 2, seed=0, k_peak=8.0, u_rms=0.03), (1, 2, 2, 2))
    X = workloads.place_spheres((n, n, n), n_particles, 4.0, 1.0, seed=0)
    setup = dict(init=lambda L: (L.init_velocity(u), L.add_spheres(X, 4.0, density_ratio=5.0)),
                 max_particles=n_particles)
    out = {"workload": f"{n}^3 D3Q19, {n_particles} moving spheres R=4, IBB, MRT, tau=0.51, {steps} steps"}
    for name, st in (("f32", lbm.F32), ("f16s", lbm.F16S), ("bf16s", lbm.BF16S)):
        r = run_case(lbm, torch, "config4_" + name, n, n, n, 0.51, (0, 0, 0), st, lbm.RATES_DHUMIERES, lbm.BC_IBB,
                     steps, warmup, setup)
        p = r["prof"]
        bms = p["ms"]["bulk"] / max(1, p["spans"]["bulk"])
        out[name] = {"mlups": round(r["mlups"], 1), "ms_per_step": round(r["ms"] / r["steps"], 4),
                     "bulk_kernel_gbs": round(r["bulk_bytes"] / (bms * 1e-3) / 1e9, 1),
                     "group_ms_per_step": {k: round(v / r["steps"], 4) for k, v in p["ms"].items() if v > 0},
                     "finite": r["finite"]}
    return out


def precision_report(lbm, torch, n=64, n_particles=31, steps=200):
    """Population storage precision against FP64 storage (which matches the
    FP64 oracle to 1e-12) on the 64^3 particle-laden box: 31 spheres of
    radius 4 (the 3.2 % volume fraction of the 512^3 / 16000-sphere case),
    IBB, d'Humieres rates, tau = 0.51, 200 steps. Field errors are
    max|x - x_ref| / max|x_ref|; statistics relative errors."""
    u = workloads.hit_velocity(n, seed=0)
    X = workloads.place_spheres((n, n, n), n_particles, 4.0, 1.0, seed=0)
    res = {}
    ref = None
    for name, st in (("f64", lbm.F64), ("f32", lbm.F32), ("f16s", lbm.F16S), ("bf16s", lbm.BF16S)):
        L = lbm.Lattice(n, n, n, 0.51, storage=st, rates=lbm.RATES_DHUMIERES, max_particles=n_particles)
        L.init_velocity(u)
        L.add_spheres(X, 4.0, density_ratio=5.0)
        L.step(steps, lbm.BC_IBB)
        rho, uu = L.macro()
        stt = L.stats(lbm.STATS_BINS)
        P = L.particles()
        fl = L.flags()
        L.close()
        cur = dict(rho=rho, u=uu, st=stt, P=P, fluid=(fl & 1) == 0)
        if ref is None:
            ref = cur
            continue
        m = cur["fluid"] & ref["fluid"]

        def fe(a, b):
            return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
        res[name] = {
            "e_rho": fe(cur["rho"][m] - 1.0, ref["rho"][m] - 1.0),
            "e_u": fe(cur["u"][:, m], ref["u"][:, m]),
            "ke_rel": abs(cur["st"]["kinetic_energy"] / ref["st"]["kinetic_energy"] - 1.0),
            "eps_rel": abs(cur["st"]["dissipation"] / ref["st"]["dissipation"] - 1.0),
            "particle_ke_rel": abs(cur["st"]["particle_ke"] / ref["st"]["particle_ke"] - 1.0),
            "particle_ake_rel": abs(cur["st"]["particle_ake"] / max(ref["st"]["particle_ake"], 1e-300) - 1.0),
        }
        res[name] = {k: float("%.3g" % v) for k, v in res[name].items()}
    res["config"] = f"{n}^3, {n_particles} spheres R=4, IBB, tau=0.51, {steps} steps; e_rho on rho-1"
    return res


def spectrum_report(lbm, torch, n=256, nbins=222, reps=3):
    """Time of the 3D energy and dissipation spectra (masked statistics
    velocity, three FP32 FFTs of 256^3 and shell sums) on the HIT field."""
    u = workloads.hit_velocity(n, seed=0, k_peak=8.0, u_rms=0.03, dtype=np.float64)
    L = lbm.Lattice(n, n, n, 0.51, storage=lbm.F32, rates=lbm.RATES_DHUMIERES)
    L.init_velocity(u)
    L.step(5)
    L.spectrum(nbins)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        E, D = L.spectrum(nbins)
    ms = (time.perf_counter() - t0) * 1e3 / reps
    L.close()
    k_peak = int(np.argmax(E[1:]) + 1)
    return {"grid": f"{n}^3", "ms_per_spectrum": round(ms, 3), "nbins": nbins, "energy_peak_shell": k_peak,
            "kinetic_energy": float(E.sum()), "spectral_dissipation": float(D.sum())}


def budget_report(lbm, torch, nbins=64, steps=20, reps=5):
    """Time of the pipe's component-wise TKE budget (Eq. 1a-c: two binned
    passes over the 148x148x438 pipe, FP64 sums) on the benchmark pipe,
    FP32, IBB, after a few steps; the near-wall dissipation and production
    show that the terms are populated."""
    L = lbm.Lattice(PIPE["nx"], PIPE["ny"], PIPE["nz"], PP["tau"], force=(0, 0, PP["g"]), storage=lbm.F32)
    L.init_velocity(pipe_field(PIPE["nz"]))
    L.set_pipe(PIPE["radius"])
    L.step(steps, lbm.BC_IBB)
    L.tke_budget(nbins)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        B = L.tke_budget(nbins)
    ms = (time.perf_counter() - t0) * 1e3 / reps
    L.close()
    return {"grid": f"{PIPE['nx']}x{PIPE['ny']}x{PIPE['nz']}", "nbins": nbins, "ms_per_budget": round(ms, 3),
            "cells": int(B[:, 0].sum()), "min_E_Dz": float(B[:, 5].min()), "max_abs_E_Oz": float(np.abs(B[:, 1]).max()),
            "finite": bool(np.all(np.isfinite(B)))}


def q27_report(lbm, torch, steps=200, warmup=10):
    """D3Q27 (the velocity set of the paper's pipe solver), FP32, BGK, on the
    benchmark pipe 148x148x438 with its linear IBB wall inside the sweep and
    the Re_tau = 180 body force: time per step from CUDA events on the
    library's stream, MLUPS over the fluid cells, and the sweep's
    algorithmic bandwidth (27 x 4 B read and 27 x 4 B written per fluid
    cell)."""
    nx, ny, nz = PIPE["nx"], PIPE["ny"], NZ
    L = lbm.Lattice(nx, ny, nz, PP["tau"], force=(0, 0, PP["g"]), storage=lbm.F32, lattice=27)
    L.init_velocity(pipe_field())
    L.set_pipe(PIPE["radius"])
    fluid = int(np.count_nonzero((L.flags() & 1) == 0))
    L.step(warmup, lbm.BC_IBB)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(L.stream)
    L.step(steps, lbm.BC_IBB)
    e1.record(L.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    _, v = L.macro()
    finite = bool(np.all(np.isfinite(v)))
    L.close()
    return {"workload": f"pipe D=146 in {nx}x{ny}x{nz} D3Q27, linear IBB wall", "storage": "f32", "steps": steps,
            "ms_per_step": round(ms, 4), "mlups": round(fluid / (ms * 1e-3) / 1e6, 1),
            "algorithmic_gbs": round(2 * 27 * 4 * fluid / (ms * 1e-3) / 1e9, 1), "finite": finite}


def closure_report(lbm, torch, n=256, n_particles=2000, steps=100):
    """Learned closure on the particle-laden 256^3 box (IBM-B): paired
    IBB/IBM-B runs of seeds 0-7 give up to 1e6 training samples, seeds 8-9
    are held out. Reports the near-surface (r/r_p in (1, 1.5]) dissipation
    profile error against IBB for plain IBM-B and with the closure, and the
    cost of one closure inference pass in the diagnostic."""
    from paper_1906_05448_gb300 import closure
    us, gs = 0.03, 4.0 / 0.03
    t0 = time.perf_counter()
    X, T = closure.paired_samples(n, n_particles, range(8), steps, us, gs)
    t1 = time.perf_counter()
    X, T = closure.shuffle(X, T, 0, limit=1000000)
    mlp = lbm.MLP()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    w, last = mlp.train(X, T, closure.init_weights(0), epochs=20, batch=4096, lr=1e-3)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    e_plain, e_closure = closure.evaluate(n, n_particles, [8, 9], steps, w.cpu().numpy(), us, gs)
    # inference cost per diagnostic: (1) fused, the tensor-core kernel inside
    # lbm_stats(LBM_STATS_CLOSURE) (the library's "closure" event span), and
    # the whole closure share of the diagnostic (stats with minus without);
    # (2) the same network over a feature array in HBM (lbm_mlp_forward,
    # including its weight packing and synchronisation)
    (ibb, bcb), (ibm, bcm) = closure.hit_pair(n, n_particles, 8)
    ibb.close()
    ibm.step(steps, bcm)
    Xs, _ = ibm.closure_samples(us, 1500 * n_particles)
    ibm.closure_set_weights(w.cpu().numpy(), us, gs)
    reps = 5

    def stats_ms(flags):
        ibm.stats(flags)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        for _ in range(reps):
            ibm.stats(flags)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    plain_ms = min(stats_ms(0), stats_ms(0))
    with_ms = min(stats_ms(lbm.STATS_CLOSURE), stats_ms(lbm.STATS_CLOSURE))
    ibm.profile_enable(True)
    for _ in range(reps):
        ibm.stats(lbm.STATS_CLOSURE)
    pr = ibm.profile(0)
    fused_ms = pr["ms"]["closure"] / max(1, pr["spans"]["closure"])
    ibm.close()
    wt = w.to(Xs.device)
    mlp.forward(Xs, wt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    e0.record()
    for _ in range(10):
        mlp.forward(Xs, wt)
    e1.record()
    torch.cuda.synchronize()
    inf_ms = e0.elapsed_time(e1) / 10
    flops = 2.0 * (85 * 64 + 64 * 64 * 2 + 64 * 9) * Xs.shape[0]
    return {"workload": f"{n}^3, {n_particles} spheres R=4, IBM-B vs IBB, {steps} steps, seeds 0-7 train / 8-9 eval",
            "train_samples": int(X.shape[0]), "data_gen_s": round(t1 - t0, 1), "train_s": round(t3 - t2, 2),
            "train_loss": round(last, 4), "zero_predictor_loss": round(float((T ** 2).mean()), 4),
            "near_surface_eps_error_plain_ibm": round(e_plain, 4),
            "near_surface_eps_error_closure": round(e_closure, 4),
            "inference_samples": int(Xs.shape[0]),
            "fused_kernel_ms_per_diagnostic": round(fused_ms, 4),
            "fused_kernel_tflops": round(flops / (fused_ms * 1e-3) / 1e12, 2),
            "closure_share_of_stats_ms": round(with_ms - plain_ms, 4), "stats_ms": round(plain_ms, 4),
            "forward_from_hbm_ms": round(inf_ms, 4),
            "forward_from_hbm_tflops": round(flops / (inf_ms * 1e-3) / 1e12, 2)}


def e2e_pipe(lbm, torch, steps):
    """Same workload through the C ABI from host buffers: the initial field is
    uploaded from pinned host memory and the final velocity field read back,
    both inside the timed region."""
    nx, ny, nz = PIPE["nx"], PIPE["ny"], NZ
    N = nx * ny * nz
    u = pipe_field()
    host_in = torch.empty(3 * N, dtype=torch.float64, pin_memory=True)
    host_in.numpy()[:] = u.reshape(-1)
    host_out = torch.empty(3 * N, dtype=torch.float64, pin_memory=True)
    L = lbm.Lattice(nx, ny, nz, PP["tau"], force=(0, 0, PP["g"]), storage=lbm.F32, rates=lbm.RATES_SRT)
    L.set_pipe(PIPE["radius"])
    fluid = int(np.count_nonzero((L.flags() & 1) == 0))
    import ctypes
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = L.L.lbm_init_velocity(L.h, ctypes.cast(host_in.data_ptr(), ctypes.POINTER(ctypes.c_double)), 1.0)
    L._check(rc)
    L.step(steps, lbm.BC_IBB)
    rc = L.L.lbm_get_field(L.h, lbm.FIELD_U, ctypes.c_void_p(host_out.data_ptr()), 3 * N * 8)
    L._check(rc)
    t1 = time.perf_counter()
    L.close()
    sec = t1 - t0
    return dict(value=fluid * steps / sec / 1e6, unit="MLUPS", h2d_bytes_per_step=3 * N * 8 // steps,
                d2h_bytes_per_step=3 * N * 8 // steps, steps=steps, seconds=sec)


# ------------------------------------------------------------ CPU oracle ---
def oracle_pipe_slab(nz_slab, steps, threads=None):
    import oracle
    if threads:
        oracle.set_threads(threads)
    nx, ny = PIPE["nx"], PIPE["ny"]
    S = oracle.Sim(nx, ny, nz_slab, PP["tau"], force=(0, 0, PP["g"]))
    S.init_velocity(pipe_field(nz_slab))
    S.set_pipe(PIPE["radius"])
    fluid = int(np.count_nonzero(S.solid()[0] == 0))
    S.step(1, oracle.BC_IBB)
    t0 = time.perf_counter()
    S.step(steps, oracle.BC_IBB)
    sec = time.perf_counter() - t0
    S.close()
    return fluid * steps / sec / 1e6, sec, oracle.get_threads(), fluid


def cpu_baseline(target_seconds=12.0):
    # calibrate on one step, then run ~target_seconds of oracle work
    _, sec1, cores, _ = oracle_pipe_slab(16, 1)
    steps = max(1, int(target_seconds / max(sec1, 1e-3)))
    mlups, sec, cores, fluid = oracle_pipe_slab(16, steps)
    return {"value": round(mlups, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, IBB pipe slab 148x148x16 ({fluid} fluid cells), {steps} steps, {sec:.1f} s"}


SWEEP_SOURCES = {"stream_collide_pipe_pipe148_f32": ("sweep_pipe.cu", "lbm_device.cuh", "segments.h"),
                 "stream_collide_bulk_pipe148_ibm_f32": ("sweep.cu", "lbm_device.cuh")}


def source_hash(kernel_key):
    """Hash of a sweep kernel's sources (kernel, device header, segment
    list): a recorded DRAM traffic figure is used only while it matches."""
    h = hashlib.sha256()
    for f in SWEEP_SOURCES[kernel_key]:
        with open(os.path.join(ROOT, "paper_1906_05448_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))
        e = d[kernel_key]
        if e.get("source_hash") != source_hash(kernel_key):
            return None
        return e["dram_bytes_per_launch"]
    except Exception:
        return None


def profile_case(case, steps, warmup):
    """One workload alone, for a profiler's launch list or a kernel capture
    (the bench line itself is not printed): the particle-laden 256^3 box
    (IBB or IBM-B), the closure diagnostic on the 256^3 (or 128^3, 250
    spheres) IBM-B box after `warmup` steps, repeated `steps` times, or the
    D3Q27 pipe (FP32, its length from --nz) for `steps` steps."""
    import torch
    from paper_1906_05448_gb300 import build as B
    from paper_1906_05448_gb300 import lbm
    B.build()
    lbm.load()
    if case == "q27_pipe":
        print(json.dumps({"case": case, **q27_report(lbm, torch, steps=steps, warmup=warmup)}))
        return
    if case.startswith("hit256"):
        bc = lbm.BC_IBB if case == "hit256_ibb" else lbm.BC_IBM_B
        r = run_case(lbm, torch, case, 256, 256, 256, 0.51, (0, 0, 0), lbm.F32, lbm.RATES_DHUMIERES, bc, steps,
                     warmup, hit_setup(256, 2000))
        p = r["prof"]
        print(json.dumps({"case": case, "ms_per_step": round(r["ms"] / steps, 4),
                          "group_ms_per_step": {k: round(v / steps, 4) for k, v in p["ms"].items() if v > 0}}))
        return
    from paper_1906_05448_gb300 import closure
    n, npart = (256, 2000) if case == "closure256" else (128, 250)
    (ibb, _), (ibm, bcm) = closure.hit_pair(n, npart, 8)
    ibb.close()
    ibm.step(warmup, bcm)
    ibm.closure_set_weights(closure.init_weights(1), 0.03, 4.0 / 0.03)
    ibm.profile_enable(True)
    for _ in range(steps):
        ibm.stats(lbm.STATS_CLOSURE)
    p = ibm.profile(0)
    ibm.close()
    print(json.dumps({"case": case, "closure_kernel_ms": round(p["ms"]["closure"] / max(1, p["spans"]["closure"]), 4)}))


# ------------------------------------------------------------------ main ---
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--nz", type=int, default=PIPE["nz"],
                    help="pipe length in cells (default 438; shorter only for profiler captures)")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16s", "bf16s"],
                    help="population storage of the main line (default f32; 16-bit only for profiler captures, "
                         "whose line is then not the benchmark's)")
    ap.add_argument("--wall", default="ibb", choices=["ibb", "ibm_b"],
                    help="wall treatment of the main line (default ibb; ibm_b only for profiler captures "
                         "of the IBM step, whose line is then not the benchmark's)")
    ap.add_argument("--case", default=None,
                    choices=["hit256_ibb", "hit256_ibm_b", "closure256", "closure128", "q27_pipe"],
                    help="profiler captures only: run this one workload (--steps steps after --warmup) "
                         "and print its timings instead of the bench line")
    args = ap.parse_args()
    global NZ
    NZ = args.nz
    if args.case:
        return profile_case(args.case, args.steps, args.warmup)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        oracle.build()
        nz = 32
        # warm-up steps of the sample, then the timed steps
        oracle_pipe_slab(nz, max(1, min(args.warmup, 3)))
        mlups, sec, cores, fluid = oracle_pipe_slab(nz, args.steps)
        line = {"metric": "MLUPS (pipe 148x148x438, IBB wall)", "value": round(mlups, 4), "unit": "MLUPS",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(1e3 * sec / args.steps, 3), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "impl": "reference",
                "config": {"workload": "pipe D=146 L=438 in 148x148x438 D3Q19, IBB; oracle sample: 148x148x32 slab",
                           "l2": "oracle on host cores"},
                "cpu_baseline": {"value": round(mlups, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                                 "sample": f"148x148x32 slab of the pipe ({fluid} fluid cells) per step"},
                "e2e": {"value": round(mlups, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_1906_05448_gb300 import build as B
    from paper_1906_05448_gb300 import lbm
    B.build()
    lbm.load()
    dev = torch.cuda.current_device()
    hbm_peak, peak_kind = peaks()

    # main line: pipe, IBB, FP32 (replicas on every rank)
    setup = pipe_setup(lbm)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    main_bc = lbm.BC_IBB if args.wall == "ibb" else lbm.BC_IBM_B
    main_res = run_case(lbm, torch, "pipe_" + args.wall + "_" + args.storage, PIPE["nx"], PIPE["ny"], NZ, PP["tau"],
                        (0, 0, PP["g"]), lbm.STORAGE[args.storage], lbm.RATES_SRT, main_bc, args.steps, args.warmup,
                        setup)
    clk = clocks.stop()
    ms_total = main_res["ms"]
    if dist:
        ms_total = max_over_ranks(torch, dist, ms_total, "cuda")
        dist.barrier()
    value = job_mlups(main_res["fluid_cells"], args.steps, world, ms_total)
    prof = main_res["prof"]
    bulk_ms = prof["ms"]["bulk"] / max(1, prof["spans"]["bulk"])
    bulk_bytes = main_res["bulk_bytes"]  # 2 x 19 x 4 B per fluid cell
    achieved = bulk_bytes / (bulk_ms * 1e-3) / 1e9
    launches = sum(prof["launches"].values())

    variants = {}
    if not args.no_variants and rank == 0:
        for name, storage, bc in (("pipe_ibm_u_f32", lbm.F32, lbm.BC_IBM_U), ("pipe_ibm_b_f32", lbm.F32, lbm.BC_IBM_B),
                                  ("pipe_ibb_f16s", lbm.F16S, lbm.BC_IBB), ("pipe_ibb_bf16s", lbm.BF16S, lbm.BC_IBB)):
            r = run_case(lbm, torch, name, PIPE["nx"], PIPE["ny"], NZ, PP["tau"], (0, 0, PP["g"]),
                         storage, lbm.RATES_SRT, bc, args.steps, min(args.warmup, 10), pipe_setup(lbm))
            p = r["prof"]
            bms = p["ms"]["bulk"] / max(1, p["spans"]["bulk"])
            variants[name] = {"mlups": round(r["mlups"], 1), "ms_per_step": round(r["ms"] / r["steps"], 4),
                              "bulk_kernel_gbs": round(r["bulk_bytes"] / (bms * 1e-3) / 1e9, 1),
                              "group_ms_per_step": {k: round(v / r["steps"], 4) for k, v in p["ms"].items() if v > 0},
                              "finite": r["finite"]}
        hs = hit_setup(256, 2000)
        for name, bc in (("hit256_2000p_ibb_f32", lbm.BC_IBB), ("hit256_2000p_ibm_b_f32", lbm.BC_IBM_B)):
            r = run_case(lbm, torch, name, 256, 256, 256, 0.51, (0, 0, 0), lbm.F32, lbm.RATES_DHUMIERES, bc,
                         max(20, args.steps // 4), 5, hs)
            p = r["prof"]
            variants[name] = {"mlups": round(r["mlups"], 1), "ms_per_step": round(r["ms"] / r["steps"], 4),
                              "group_ms_per_step": {k: round(v / r["steps"], 4) for k, v in p["ms"].items() if v > 0},
                              "launches_per_step": round(sum(p["launches"].values()) / r["steps"], 1),
                              "finite": r["finite"]}

    precision = None
    config4 = None
    closure_res = None
    spectrum_res = None
    budget_res = None
    q27_res = None
    if not args.no_variants and rank == 0:
        precision = precision_report(lbm, torch)
        try:
            config4 = config4_report(lbm, torch)
        except Exception as ex:  # a variant's failure must not lose the line
            config4 = {"error": str(ex)[:200]}
        closure_res = closure_report(lbm, torch)
        spectrum_res = spectrum_report(lbm, torch)
        try:
            budget_res = budget_report(lbm, torch)
        except Exception as ex:  # a diagnostic's failure must not lose the line
            budget_res = {"error": str(ex)[:200]}
        try:
            q27_res = q27_report(lbm, torch)
        except Exception as ex:
            q27_res = {"error": str(ex)[:200]}

    e2e = None
    if rank == 0 and not args.no_e2e:
        e2e = e2e_pipe(lbm, torch, args.steps)
        e2e = {k: (round(v, 3) if isinstance(v, float) else v) for k, v in e2e.items()}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        cpu = cpu_baseline()

    if rank == 0:
        line = {
            "metric": "MLUPS (pipe 148x148x438, IBB wall)" if args.wall == "ibb" else "MLUPS (pipe, IBM-B wall)",
            "value": round(value, 1),
            "unit": "MLUPS",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(ms_total / args.steps, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",  # the collision arithmetic; the storage is in config
            "data": "synthetic",
            "config": {"workload": f"pipe D=146 L={NZ} in 148x148x{NZ} D3Q19, {args.storage.upper()} populations, SRT, nu=0.0032, "
                                   "Re_tau=180 body force, " + ("linear IBB wall" if args.wall == "ibb" else "IBM-B wall"),
                       "fluid_cells": main_res["fluid_cells"], "parallelism": f"replicas x{world}",
                       "l2": "no flush: populations 2x1.46 GB >> 129 MB L2"},
            "roofline": {"bound": "hbm",
                         "kernel": ("stream_collide_pipe<" if args.wall == "ibb" else "stream_collide_bulk<") +
                                   args.storage + ",srt," + args.wall[:3] + ">",
                         "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(achieved / hbm_peak, 4), "peak_source": peak_kind,
                         "traffic": traffic_for("stream_collide_pipe_pipe148_f32")
                         if (args.wall == "ibb" and args.storage == "f32" and NZ == PIPE["nz"]) else None,
                         "algorithmic_bytes_per_launch": bulk_bytes,
                         "avg_launch_ms": round(bulk_ms, 5),
                         "step_achieved": round(bulk_bytes / (ms_total / args.steps * 1e-3) / 1e9, 1),
                         "step_frac": round(bulk_bytes / (ms_total / args.steps * 1e-3) / 1e9 / hbm_peak, 4)},
            "group_ms_per_step": {k: round(v / args.steps, 4) for k, v in prof["ms"].items() if v > 0},
            "gpu_launches": int(launches),
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "variants": variants,
            "precision_vs_f64": precision,
            "config4": config4,
            "closure": closure_res,
            "spectrum": spectrum_res,
            "tke_budget": budget_res,
            "d3q27": q27_res,
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
