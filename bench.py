"""Benchmark of the plane-wave H|psi> + block Davidson hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one full eigensolve of the medium workload (cubic cell a = 20 bohr,
64 atoms, 40 Ry: 34,265 plane waves, FFT box 90^3, 576 projectors; lowest 128
bands from seeded random starting bands to max ||H x - theta x|| <= 1e-8 Ha) in
mixed precision (a reduced-precision phase of FP32 FFTs, BF16 tensor-core
projector GEMMs, FP32-equivalent tensor-core subspace GEMMs, FP32 Jacobi and
Cholesky; then FP64 Rayleigh-Ritz, Cholesky and residuals, with
Jacobi-Davidson corrections from the reduced-precision operator).  Every
row of the hot path runs
inside a step: H|psi> (scatter, FFTs, V, kinetic, becp, D, back-projection),
subspace overlaps, Cholesky-QR, Jacobi, residuals, preconditioner.

value = band-applies of H per second through the whole solver (all bands to
which H was applied, in any precision, divided by the solve time); ms_per_step
is the time-to-1e-8-residual.  The same line carries the plain FP64 GPU solve
of the same system (mixed vs FP64), H|psi>-only throughputs, the roofline of
the dominant kernel, the end-to-end number through host buffers, the oracle's
CPU throughput and the SM clocks seen during the timed region.

Multi-GPU (torchrun): independent replicas, one per GPU (different seeds), no
data-path collective; value sums all ranks' band-applies over the slowest
rank's time (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hpsi band-applies/s and Davidson time-to-1e-8 residual, mixed vs FP64, 1 GB300"
WORKLOAD = "medium"
TOL = 1e-8
SWITCH_TOL = 1e-3
JD_INNER = 20
MULT = 3
# Fallback peaks (no measured-peaks file on this machine): HBM copy bandwidth
# and the derived CUDA-core arithmetic peaks (lanes x FMA x clock).
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
FP64_ALU_TFLOPS = 1.25     # nominal FP64 rate of the part
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x FMA x max clock


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--skip-fp64", action="store_true", help="omit the FP64 comparison solve")
    p.add_argument("--skip-batched", action="store_true", help="omit the batched cells x k-points solve")
    p.add_argument("--profile", action="store_true",
                   help="for a profiler's launch list: only the warm-up and timed solves, a short "
                        "JSON line (no FP64 solve, H-only, e2e, batched or CPU legs)")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return d, "measured"
        except Exception:
            pass
    return dict(FALLBACK), "fallback"


def setup_inputs(seed):
    from paper_1709_10010_gb300 import synthetic as syn
    cfg = syn.CONFIGS[WORKLOAD]
    cell = syn.config_cell(WORKLOAD, seed)
    return cfg, cell


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"pwh_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def reduce_over_ranks(dist, elapsed, units, device):
    """Replicas: the slowest rank's time and the units of all ranks (max and
    sum over the process group; unchanged without one)."""
    if dist is None:
        return elapsed, units
    import torch
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return float(t.item()), float(c.item())


# ------------------------------------------------------------------ ours ----
def run_ours(a):
    import torch
    import paper_1709_10010_gb300 as pwh
    from paper_1709_10010_gb300 import synthetic as syn

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1709_10010_gb300 import build
    build.build()
    cfg, cell = setup_inputs(seed=rank)
    nb = cfg["nb"]
    s = pwh.System.from_cell(cell, precision="mixed")
    miller = s.miller()
    v = syn.potential_grid(cell, s.fft)
    beta = syn.projectors(cell, miller)
    D = syn.d_diagonal(cell)
    s.set_potential(v)
    s.set_projectors(beta, D)
    psi0_h = syn.initial_bands(rank, s.npw, nb)
    psi0 = torch.from_numpy(psi0_h).cuda()
    psi = torch.empty_like(psi0)
    stream = torch.cuda.current_stream()

    def solve(mixed=True):
        psi.copy_(psi0)
        return s.davidson(psi, tol=TOL, mult=MULT, mixed=mixed, switch_tol=SWITCH_TOL,
                          jd_inner=JD_INNER if mixed else 0)

    for _ in range(a.warmup):
        solve()
    torch.cuda.synchronize()

    # ---- timed region: K full mixed-precision solves
    clocks = ClockSampler(dev) if rank == 0 else None
    if clocks:
        clocks.start()
    s.set_kernel_timing(True)
    launches0 = pwh.launch_count()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("bench_timed")
    e0.record(stream)
    n_apply, stats = 0, []
    eig = None
    for _ in range(a.steps):
        eig, st, status = solve()
        assert status == 0, status
        n_apply += st["n_apply"]
        stats.append(st)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    elapsed = e0.elapsed_time(e1) / 1e3
    launches = pwh.launch_count() - launches0
    ktimes = s.kernel_times()
    s.set_kernel_timing(False)
    clk = clocks.stop() if clocks else None
    t_max, tot_apply = reduce_over_ranks(dist, elapsed, n_apply, "cuda")
    if rank != 0:
        dist.destroy_process_group() if dist is not None else None
        return
    ms_per_step = 1e3 * elapsed / a.steps
    if a.profile:
        print(json.dumps({"metric": METRIC, "value": tot_apply / t_max, "unit": "band-applies/s",
                          "ms_per_step": ms_per_step, "steps": a.steps, "warmup": a.warmup,
                          "profile_run": True, "gpu_launches": int(launches)}))
        return

    # ---- mixed vs FP64: one plain FP64 solve of the same system
    fp64 = None
    if not a.skip_fp64:
        psi.copy_(psi0)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        eig64, st64, status64 = s.davidson(psi, tol=TOL, mult=MULT, mixed=False)
        f1.record(stream)
        torch.cuda.synchronize()
        fp64 = {"time_s": f0.elapsed_time(f1) / 1e3, "iters": st64["iters"],
                "n_apply": st64["n_apply"], "status": status64,
                "max_abs_dlambda_mixed_vs_fp64_ha": float(np.abs(eig - eig64).max())}

    # ---- H|psi> alone (128 bands), FP64 and mixed
    hpsi_only = {}
    out = torch.empty_like(psi0)
    for prec in ("fp64", "mixed"):
        s.set_precision(prec)
        for _ in range(3):
            s.apply_h(psi0, out)
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10 if prec == "mixed" else 3
        h0.record(stream)
        for _ in range(reps):
            s.apply_h(psi0, out)
        h1.record(stream)
        torch.cuda.synchronize()
        hpsi_only[prec] = nb * reps / (h0.elapsed_time(h1) / 1e3)
    s.set_precision("mixed")

    # ---- end to end through host buffers (pinned), copies inside the timed region
    pin_in = torch.from_numpy(psi0_h).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    dbuf = torch.empty_like(psi0)
    ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_apply = 0
    torch.cuda.synchronize()
    ee0.record(stream)
    for _ in range(a.steps):
        dbuf.copy_(pin_in, non_blocking=True)
        eig_e, st_e, status_e = s.davidson(dbuf, tol=TOL, mult=MULT, mixed=True,
                                           switch_tol=SWITCH_TOL, jd_inner=JD_INNER)
        pin_out.copy_(dbuf, non_blocking=True)
        e2e_apply += st_e["n_apply"]
    ee1.record(stream)
    torch.cuda.synchronize()
    e2e_time = ee0.elapsed_time(ee1) / 1e3
    bi = psi0_h.nbytes
    bo = psi0_h.nbytes + nb * 8

    # ---- batched workload: 32 cells x 8 k-points solved concurrently
    batched = None if a.skip_batched else run_batched(pwh, syn, torch)

    # ---- roofline of the dominant kernel family of the timed region
    roof = roofline(ktimes)

    # ---- CPU baseline: the oracle on a bounded sample of the same workload
    cpu = cpu_baseline(cell, s, v, beta, D, psi0_h)

    med = stats[len(stats) // 2]
    line = {
        "metric": METRIC, "value": tot_apply / t_max, "unit": "band-applies/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32+bf16",
        "data": "synthetic (seeded cell, Gaussian potential and projectors, random start)",
        "config": {"workload": f"{WORKLOAD}: a=20 bohr cubic, 64 atoms, 40 Ry, npw={s.npw}, "
                               f"FFT {s.fft[0]}^3, {beta.shape[0]} projectors, lowest {nb} bands "
                               f"to 1e-8, mixed precision",
                   "npw": s.npw, "fft": list(s.fft), "nproj": int(beta.shape[0]), "nb": nb,
                   "tol": TOL, "switch_tol": SWITCH_TOL, "jd_inner": JD_INNER, "m_max": MULT * nb,
                   "l2": "working set (V, HV: 2 x npw x m_max x 16 B = 421 MB) larger than L2",
                   "parallelism": f"replicas x{world}"},
        "time_to_1e-8_s": {"mixed": ms_per_step / 1e3, "fp64": fp64["time_s"] if fp64 else None},
        "davidson": {"mixed": {k: med[k] for k in ("iters", "n_apply", "n_apply_fp64",
                                                   "switch_iter", "t_mixed_s", "t_fp64_s",
                                                   "max_resid")},
                     "fp64": fp64},
        "hpsi_only_band_applies_s": hpsi_only,
        "batched": batched,
        "kernels": {k: {"launches": d["launches"], "ms": round(d["ms"], 3),
                        "share": round(d["ms"] / max(1e-9, sum(x["ms"] for x in ktimes.values())), 4),
                        "frac": (lambda r: None if r is None or r["frac"] is None else round(r["frac"], 4))(
                            family_roofline(k, d))}
                    for k, d in ktimes.items() if d["launches"]},
        "roofline": roof,
        "e2e": {"value": e2e_apply / e2e_time, "unit": "band-applies/s",
                "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                "time_to_1e-8_s": e2e_time / a.steps},
        "gpu_launches": int(launches),
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def run_batched(pwh, syn, torch, ncells=32, nthreads=16):
    """32 cubic cells (a ~ U(8,14) bohr, 4-16 atoms, 30 Ry) x the eight k-points of
    a 2x2x2 Monkhorst-Pack grid = 256 independent systems with 24-48 bands each,
    all solved to 1e-8 (mixed + Jacobi-Davidson) by pwh_batch_davidson_solve,
    one stream per system.  One warm-up pass, then one timed pass."""
    work = syn.batched_workload(ncells=ncells, seed=0)
    systems, starts, streams = [], [], []
    vcache = {}
    for i, (cell, nb) in enumerate(work):
        st = torch.cuda.Stream()
        s = pwh.System.from_cell(cell, precision="mixed", stream=st.cuda_stream)
        key = i // 8
        if key not in vcache:
            vcache[key] = syn.potential_grid(cell, s.fft)
        s.set_potential(vcache[key])
        s.set_projectors(syn.projectors(cell, s.miller()), syn.d_diagonal(cell))
        systems.append(s)
        streams.append(st)
        starts.append(syn.initial_bands(i, s.npw, nb))
    res = {}
    for tag in ("warmup", "timed"):
        psis = [torch.from_numpy(p0).cuda() for p0 in starts]
        torch.cuda.synchronize()
        t0 = time.time()
        eigs, stats, status, st_all = pwh.batch_davidson(systems, psis, tol=TOL, mult=MULT,
                                                          switch_tol=SWITCH_TOL, jd_inner=JD_INNER,
                                                          nthreads=nthreads)
        torch.cuda.synchronize()
        res[tag] = (time.time() - t0, eigs, stats, status)
    dt, eigs, stats, status = res["timed"]
    n_apply = sum(x["n_apply"] for x in stats)
    # the same spectrum at k and -k (time reversal): a built-in consistency check
    tr = max(float(np.abs(eigs[8 * c] - eigs[8 * c + 7]).max()) for c in range(ncells))
    return {"workload": f"{ncells} cells a~U(8,14) bohr, 4-16 atoms, 30 Ry, x 8 k-points "
                        f"(2x2x2 Monkhorst-Pack): {len(systems)} systems, npw "
                        f"{min(s.npw for s in systems)}-{max(s.npw for s in systems)}, "
                        f"{sum(int(p.shape[0]) for p in starts)} bands in total",
            "threads": nthreads, "time_to_1e-8_s": dt, "band_applies_s": n_apply / dt,
            "all_converged": all(x == 0 for x in status),
            "max_dlambda_k_vs_minus_k_ha": tr}


FAMILY_BOUND = {
    # family: (bound, counter, peak key)
    "fft_plane_fp32": ("alu", "flops", "fp32"), "fft_plane_fp64": ("alu", "flops", "fp64"),
    "fft_z_inverse_fp32": ("hbm", "bytes", "hbm"), "fft_z_forward_fp32": ("hbm", "bytes", "hbm"),
    "fft_z_inverse_fp64": ("alu", "flops", "fp64"), "fft_z_forward_fp64": ("alu", "flops", "fp64"),
    "tc_gemm_becp": ("tensor", "flops", "bf16"), "tc_gemm_backproj": ("tensor", "flops", "bf16"),
    "cgemm_fp64": ("alu", "flops", "fp64"), "cgemm_fp32": ("alu", "flops", "fp32"),
    "jacobi_fp64": ("alu", "flops", "fp64"), "cholqr_fp64": ("alu", "flops", "fp64"),
    "jacobi_fp32": ("alu", "flops", "fp32"), "zgemm_fp64_tc": ("tensor", "flops", "bf16"),
    "zgemm_fp32_tc": ("tensor", "flops", "bf16"),
}


def family_roofline(fam, d):
    pk, src = peaks()
    bound, counter, key = FAMILY_BOUND[fam]
    if d["launches"] == 0:
        return None
    sec = d["ms"] / 1e3 / d["launches"]
    work = d[counter] / d["launches"]
    if key == "hbm":
        peak, unit, psrc = pk.get("hbm_gbs"), "GB/s", f"{src} HBM copy bandwidth"
        achieved = work / sec / 1e9
    elif key == "bf16":
        peak, unit, psrc = pk.get("bf16_tflops"), "TFLOP/s", f"{src} dense BF16"
        achieved = work / sec / 1e12
    elif key == "fp32":
        peak, unit, psrc = FP32_ALU_TFLOPS, "TFLOP/s", "derived FP32 CUDA-core rate"
        achieved = work / sec / 1e12
    else:
        peak, unit, psrc = FP64_ALU_TFLOPS, "TFLOP/s", "nominal FP64 rate"
        achieved = work / sec / 1e12
    return {"kernel": fam, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": (achieved / peak) if (peak and work) else None, "traffic": None,
            "avg_launch_ms": d["ms"] / d["launches"], "peak_source": psrc}


def roofline(kt):
    """Roofline of the kernel family with the largest device time in the timed
    region (CUDA events on the solver's stream), its algorithmic work per launch
    divided by its average launch duration."""
    fams = {k: v for k, v in kt.items() if v["launches"]}
    fam = max(fams, key=lambda k: fams[k]["ms"])
    tot = sum(v["ms"] for v in fams.values())
    r = family_roofline(fam, fams[fam])
    r["share_of_timed_kernels"] = fams[fam]["ms"] / tot
    return r


def cpu_baseline(cell, s, v, beta, D, psi0_h, iters=1):
    """The oracle (numpy FP64) on a bounded sample: the first Davidson iteration
    of the same workload (H applied to the 128 starting bands, Rayleigh-Ritz,
    residuals)."""
    from oracle import basis as ob
    from oracle import davidson as od
    from oracle import hamiltonian as oh
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    t = time.time()
    res = od.davidson(lambda X: oh.apply_h(b, v, beta, D, X.T).T, b.kinetic, psi0_h.T,
                      psi0_h.shape[0], tol=TOL, max_iter=iters, m_max=MULT * psi0_h.shape[0])
    dt = time.time() - t
    return {"value": res.n_apply / dt, "unit": "band-applies/s", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle", "sample": f"{iters} Davidson iteration(s) of the same workload "
                                         f"({res.n_apply} band-applies, {dt:.1f} s)"}


# ------------------------------------------------------------- reference ----
def run_reference(a):
    """The oracle as the reference arm: each step a bounded sample (one Davidson
    iteration, 128 band-applies) of the same workload on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1709_10010_gb300 import synthetic as syn
    from oracle import basis as ob
    cfg, cell = setup_inputs(seed=0)
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    v = syn.potential_grid(cell, b.fft)
    beta = syn.projectors(cell, b.miller)
    D = syn.d_diagonal(cell)
    psi0 = syn.initial_bands(0, b.npw, cfg["nb"])

    class S:
        npw = b.npw
    for _ in range(a.warmup):
        cpu_baseline(cell, S, v, beta, D, psi0[:8])
    vals, t_all, n_all = [], 0.0, 0
    for _ in range(a.steps):
        r = cpu_baseline(cell, S, v, beta, D, psi0)
        vals.append(r["value"])
        n_all += cfg["nb"]
        t_all += cfg["nb"] / r["value"]
    value = n_all / t_all
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "band-applies/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * t_all / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: a=20 bohr cubic, 64 atoms, 40 Ry, npw={b.npw}, "
                                   f"{beta.shape[0]} projectors, 128 bands; bounded sample: "
                                   f"one Davidson iteration per step"},
            "cpu_baseline": {"value": value, "unit": "band-applies/s",
                             "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                             "sample": "one Davidson iteration (128 band-applies) per step"},
            "e2e": {"value": value, "unit": "band-applies/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
