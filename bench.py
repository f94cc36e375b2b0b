"""Benchmark of the plane-wave H|psi> + block Davidson hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one full eigensolve of the large workload (cubic cell a = 30 bohr,
216 atoms, 50 Ry: 161,235 plane waves, FFT box 144^3, 1,944 s,p,d projectors;
lowest 512 bands from seeded random starting bands to max ||H x - theta x|| <=
1e-8 Ha) in mixed precision: a reduced-precision phase (FP32 FFTs, BF16
tensor-core projector GEMMs, FP32-equivalent tensor-core subspace GEMMs, FP32
Jacobi and Cholesky), then Jacobi-Davidson steps whose Rayleigh-Ritz,
Cholesky and residuals run in FP64.  Every row of the hot path runs inside a
step: H|psi> (scatter, FFTs, V, kinetic, becp, D, back-projection), subspace
overlaps, Cholesky-QR, Jacobi, residuals, preconditioner.

value = band-applies of H per second through the solver (all bands to which H
was applied, in any precision, divided by the solve time); ms_per_step is the
time-to-1e-8-residual.  The same line carries:
  * the plain FP64 GPU solve of the same system (mixed vs FP64);
  * steady-state H|psi>-only throughput on the 512 resident bands (median of
    20 CUDA-event-timed applications, FP64 and mixed);
  * the roofline of the dominant kernel family, from a separate solve with the
    library's per-family event timer on (not inside the timed region);
  * the end-to-end solve through the C ABI with host buffers;
  * the medium cell (34,265 plane waves, 128 bands) and the batched workload as
    secondary lines;
  * the oracle's CPU throughput and the SM clocks seen during the timed region.

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
WORKLOAD = "large"
TOL = 1e-8
SWITCH_TOL = 1e-3
JD_INNER = 16         # inner CG steps of a Jacobi-Davidson correction (sweep: 12, 14, 16, 20, 24)
MULT = 3
HPSI_REPS = 20      # H|psi>-only repeats (median reported)
ACE_NOCC = 32       # occupied bands of the exact-exchange (ACE) leg
E2E_STEPS = 3       # end-to-end solves through host buffers
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
    p.add_argument("--skip-medium", action="store_true", help="omit the medium-cell secondary line")
    p.add_argument("--skip-ace", action="store_true",
                   help="omit the exact-exchange / ACE leg on the medium cell")
    p.add_argument("--skip-gamma", action="store_true",
                   help="omit the real-band (k = 0 half-sphere) solve of the same workload")
    p.add_argument("--workload", default=WORKLOAD, choices=["large", "medium", "small"],
                   help="system of the timed solves (default: the large cell)")
    p.add_argument("--mult", type=int, default=MULT, help="m_max = mult x nb")
    p.add_argument("--hpsi-only", choices=["mixed", "fp64"], default=None,
                   help="for profilers: W + K applications of H (this precision) to the "
                        "workload's bands, a short JSON line, nothing else")
    p.add_argument("--eigh", type=int, default=0, metavar="N",
                   help="for profilers: W + K reduced-precision Rayleigh-Ritz eigensolves "
                        "(pwh_subspace_eigh, the FP32 Jacobi stage) of a seeded random Hermitian "
                        "N x N matrix, a short JSON line, nothing else")
    p.add_argument("--gemm", default=None, metavar="M,N,K,PREC,CONJ",
                   help="for profilers: W + K subspace GEMMs (pwh_subspace_gemm) of this shape, "
                        "precision fp64|mixed and op(A) = A^H when CONJ is 1, on seeded random "
                        "operands, a short JSON line, nothing else")
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
def make_system(pwh, syn, cell, precision="mixed", stream=None):
    s = pwh.System.from_cell(cell, precision=precision, stream=stream)
    v = syn.potential_grid(cell, s.fft)
    beta = syn.projectors(cell, s.miller())
    D = syn.d_diagonal(cell)
    s.set_potential(v)
    s.set_projectors(beta, D)
    return s, v, beta, D


def timed(torch, stream, fn):
    """fn() bracketed by CUDA events on the stream; returns (seconds, result)."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    r = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3, r


def hpsi_only(torch, s, psi0, reps=HPSI_REPS):
    """Steady-state H|psi> throughput on the resident bands: median over reps
    CUDA-event-timed applications, per precision."""
    out = torch.empty_like(psi0)
    stream = torch.cuda.current_stream()
    res = {}
    for prec in ("fp64", "mixed"):
        s.set_precision(prec)
        for _ in range(3):
            s.apply_h(psi0, out)
        ts = [timed(torch, stream, lambda: s.apply_h(psi0, out))[0] for _ in range(reps)]
        med = statistics.median(ts)
        res[prec] = {"band_applies_s": psi0.shape[0] / med, "median_ms": 1e3 * med,
                     "repeats": reps}
    # the same number of real bands at k = 0 on the half sphere (two real bands
    # per complex FFT; the imaginary part stored at G = 0 is ignored)
    nh = len(s.gamma_half())
    psig = psi0[:, :nh].contiguous()
    outg = torch.empty_like(psig)
    for prec in ("fp64", "mixed"):
        s.set_precision(prec)
        for _ in range(3):
            s.apply_h_gamma(psig, outg)
        ts = [timed(torch, stream, lambda: s.apply_h_gamma(psig, outg))[0] for _ in range(reps)]
        med = statistics.median(ts)
        res["gamma_real_" + prec] = {"band_applies_s": psig.shape[0] / med, "median_ms": 1e3 * med,
                                     "repeats": reps, "npw_half": nh}
    del psig, outg
    s.set_precision("mixed")
    return res


def gamma_solve(torch, s, nb, steps, seed=0):
    """The same eigenproblem as real bands at k = 0: nb half-sphere bands from
    the seeded generator, mixed + Jacobi-Davidson to 1e-8 (pwh_davidson_solve_gamma),
    one warm-up solve, then the median of `steps` CUDA-event-timed solves."""
    from paper_1709_10010_gb300 import synthetic as syn
    nh = len(s.gamma_half())
    psi0 = torch.from_numpy(syn.initial_bands(seed, nh, nb)).cuda()
    psi = torch.empty_like(psi0)
    stream = torch.cuda.current_stream()

    def solve():
        psi.copy_(psi0)
        return s.davidson_gamma(psi, tol=TOL, mult=MULT, mixed=True, switch_tol=SWITCH_TOL,
                                jd_inner=JD_INNER)
    solve()
    runs = [timed(torch, stream, solve) for _ in range(max(1, steps))]
    t = statistics.median(r[0] for r in runs)
    eig, st, status = runs[-1][1]
    assert status == 0, status
    return {"time_to_1e-8_s": t, "band_applies_s": st["n_apply"] / t, "iters": st["iters"],
            "n_apply": st["n_apply"], "n_apply_fp64": st["n_apply_fp64"], "npw_half": nh,
            "steps": len(runs), "eig": eig}


def run_eigh(torch, pwh, syn, a):
    """Profiling entry for the subspace eigensolver alone: the lowest N/3
    eigenpairs of a seeded random Hermitian N x N matrix in reduced precision
    (the FP32 Jacobi stage of the reduced phase), W untimed and K timed calls."""
    n = a.eigh
    s = pwh.System.from_cell(syn.config_cell("small", 0), precision="mixed")
    H = torch.from_numpy(syn.random_hermitian(0, n).T.copy()).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        s.subspace_eigh(H, n // 3, precision="mixed")
    t, _ = timed(torch, stream, lambda: [s.subspace_eigh(H, n // 3, precision="mixed")
                                         for _ in range(a.steps)])
    s.sync()
    print(json.dumps({"metric": "reduced-precision subspace eigensolves/s", "value": a.steps / t,
                      "ms_per_call": 1e3 * t / a.steps, "n": n, "steps": a.steps,
                      "warmup": a.warmup}))


def run_gemm(torch, pwh, syn, a):
    """Profiling entry for one subspace-GEMM shape: C = op(A) B with seeded
    N(0,1) complex operands, W untimed and K timed calls."""
    M, N, K, prec, conj = a.gemm.split(",")
    M, N, K, conj = int(M), int(N), int(K), conj == "1"
    s = pwh.System.from_cell(syn.config_cell("small", 0), precision="mixed")
    g = torch.Generator(device="cuda").manual_seed(0)
    ra, ka = (K, M) if conj else (M, K)             # stored A: ra rows x ka columns
    A = torch.randn((ka, ra), dtype=torch.complex128, device="cuda", generator=g)
    B = torch.randn((N, K), dtype=torch.complex128, device="cuda", generator=g)
    C = torch.zeros((N, M), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        s.gemm(A, B, C, conj_a=conj, precision=prec)
    t, _ = timed(torch, stream, lambda: [s.gemm(A, B, C, conj_a=conj, precision=prec)
                                         for _ in range(a.steps)])
    print(json.dumps({"metric": "subspace GEMM TFLOP/s (8 M N K complex flops)",
                      "value": 8.0 * M * N * K * a.steps / t / 1e12, "ms_per_call": 1e3 * t / a.steps,
                      "shape": [M, N, K], "precision": prec, "conj_a": conj, "steps": a.steps,
                      "warmup": a.warmup}))


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
    if a.eigh:
        run_eigh(torch, pwh, syn, a)
        return
    if a.gemm:
        run_gemm(torch, pwh, syn, a)
        return
    cfg = syn.CONFIGS[a.workload]
    cell = syn.config_cell(a.workload, seed=rank)
    nb = cfg["nb"]
    s, v, beta, D = make_system(pwh, syn, cell)
    psi0_h = syn.initial_bands(rank, s.npw, nb)
    psi0 = torch.from_numpy(psi0_h).cuda()
    psi = torch.empty_like(psi0)
    stream = torch.cuda.current_stream()

    def solve(mixed=True):
        psi.copy_(psi0)
        return s.davidson(psi, tol=TOL, mult=a.mult, mixed=mixed, switch_tol=SWITCH_TOL,
                          jd_inner=JD_INNER if mixed else 0)

    if a.hpsi_only:
        s.set_precision(a.hpsi_only)
        out = torch.empty_like(psi0)
        for _ in range(a.warmup):
            s.apply_h(psi0, out)
        t, _ = timed(torch, stream, lambda: [s.apply_h(psi0, out) for _ in range(a.steps)])
        s.sync()
        print(json.dumps({"metric": "H band-applies/s", "value": nb * a.steps / t,
                          "ms_per_apply": 1e3 * t / a.steps, "precision": a.hpsi_only,
                          "workload": a.workload, "nb": nb, "steps": a.steps,
                          "warmup": a.warmup}))
        return

    for _ in range(a.warmup):
        solve()
    torch.cuda.synchronize()

    # ---- timed region: K full mixed-precision solves to 1e-8 (no kernel timer)
    clocks = ClockSampler(dev) if rank == 0 else None
    if clocks:
        clocks.start()
    launches0 = pwh.launch_count()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n_apply, stats = 0, []
    eig = None
    for _ in range(a.steps):
        eig, st, status = solve()
        assert status == 0, status
        n_apply += st["n_apply"]
        stats.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    elapsed = e0.elapsed_time(e1) / 1e3
    launches = pwh.launch_count() - launches0
    clk = clocks.stop() if clocks else None
    t_max, tot_apply = reduce_over_ranks(dist, elapsed, n_apply, "cuda")
    if rank != 0:
        dist.destroy_process_group() if dist is not None else None
        return
    ms_per_step = 1e3 * elapsed / a.steps
    if a.profile:
        print(json.dumps({"metric": METRIC, "value": tot_apply / t_max, "unit": "band-applies/s",
                          "ms_per_step": ms_per_step, "steps": a.steps, "warmup": a.warmup,
                          "profile_run": True, "gpu_launches": int(launches),
                          "workload": a.workload}))
        return

    # ---- per-family kernel times: one more solve with the library's event
    # timer on (a separate pass, outside the timed region)
    s.set_kernel_timing(True)
    solve()
    torch.cuda.synchronize()
    ktimes = s.kernel_times()
    s.set_kernel_timing(False)

    # ---- mixed vs FP64: one plain FP64 solve of the same system
    fp64 = None
    if not a.skip_fp64:
        t64, (eig64, st64, status64) = timed(torch, stream, lambda: solve(mixed=False))
        fp64 = {"time_s": t64, "iters": st64["iters"], "n_apply": st64["n_apply"],
                "status": status64,
                "max_abs_dlambda_mixed_vs_fp64_ha": float(np.abs(eig - eig64).max())}

    # ---- H|psi> alone on the 512 resident bands, FP64 and mixed
    hp = hpsi_only(torch, s, psi0)

    # ---- the same eigenproblem as real bands at k = 0 (half sphere)
    gam = None
    if not a.skip_gamma:
        gam = gamma_solve(torch, s, nb, a.steps)
        gam["max_abs_dlambda_vs_complex_ha"] = float(np.abs(gam.pop("eig") - eig).max())

    # ---- end to end through the C ABI with host buffers: pwh_davidson_solve_host
    # copies the pinned starting bands in and the eigenvectors out inside the call
    pin = torch.from_numpy(psi0_h).pin_memory()
    pin_np = pin.numpy()
    e2e_steps = min(a.steps, E2E_STEPS)
    e2e_apply, e2e_time = 0, 0.0
    for _ in range(e2e_steps):
        pin_np[...] = psi0_h
        t0 = time.perf_counter()
        _, st_e, status_e = s.davidson_host(pin_np, tol=TOL, mult=a.mult, mixed=True,
                                            switch_tol=SWITCH_TOL, jd_inner=JD_INNER)
        e2e_time += time.perf_counter() - t0
        assert status_e == 0, status_e
        e2e_apply += st_e["n_apply"]
    bi = psi0_h.nbytes
    bo = psi0_h.nbytes + nb * 8

    # ---- the medium cell (34,265 plane waves, 128 bands) as a secondary line
    medium = None if (a.skip_medium or a.workload == "medium") else run_medium(pwh, syn, torch)
    # ---- exact exchange: ACE built and applied on the medium cell
    ace = None if a.skip_ace else run_ace(pwh, syn, torch)
    # ---- batched workload: 32 cells x 8 k-points solved concurrently
    batched = None if a.skip_batched else run_batched(pwh, syn, torch)

    # ---- roofline of the dominant kernel family of a solve
    roof = roofline(ktimes, s)

    # ---- CPU baseline: the oracle on a bounded sample of the same workload
    cpu = cpu_baseline(cell, s.npw, s.fft, v, beta, D, psi0_h)

    med = stats[len(stats) // 2]
    ktot = sum(x["ms"] for x in ktimes.values())
    line = {
        "metric": METRIC, "value": tot_apply / t_max, "unit": "band-applies/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32+bf16",
        "data": "synthetic (seeded cell, Gaussian potential and projectors, random start)",
        "config": {"workload": f"{a.workload}: a={cfg['a']:g} bohr cubic, {cfg['natoms']} atoms, "
                               f"{cfg['ecut_ry']:g} Ry, npw={s.npw}, FFT {s.fft[0]}^3, "
                               f"{beta.shape[0]} projectors, lowest {nb} bands to max||r|| <= 1e-8, "
                               f"mixed precision + Jacobi-Davidson",
                   "npw": s.npw, "fft": list(s.fft), "nproj": int(beta.shape[0]), "nb": nb,
                   "tol": TOL, "switch_tol": SWITCH_TOL, "jd_inner": JD_INNER, "m_max": a.mult * nb,
                   "step": "one full eigensolve from the seeded random start to 1e-8",
                   "l2": f"inputs larger than L2 (V, HV: 2 x npw x m_max x 16 B = "
                         f"{2 * s.npw * a.mult * nb * 16 / 1e9:.1f} GB; FP64 beta {beta.nbytes / 1e9:.1f} GB)",
                   "parallelism": f"replicas x{world}"},
        "time_to_1e-8_s": {"mixed": ms_per_step / 1e3, "fp64": fp64["time_s"] if fp64 else None,
                           "fp64_over_mixed": (fp64["time_s"] / (ms_per_step / 1e3)) if fp64 else None},
        "davidson": {"mixed": {k: med[k] for k in ("iters", "n_apply", "n_apply_fp64",
                                                   "switch_iter", "t_mixed_s", "t_fp64_s",
                                                   "max_resid")},
                     "fp64": fp64},
        "hpsi_only": hp,
        "gamma_real_bands": gam,
        "medium": medium,
        "ace": ace,
        "batched": batched,
        "kernels": {k: {"launches": d["launches"], "ms": round(d["ms"], 3),
                        "share": round(d["ms"] / max(1e-9, ktot), 4),
                        "frac": (lambda r: None if r is None or r["frac"] is None else round(r["frac"], 4))(
                            family_roofline(k, d, s))}
                    for k, d in ktimes.items() if d["launches"]},
        "roofline": roof,
        "e2e": {"value": e2e_apply / e2e_time, "unit": "band-applies/s",
                "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                "time_to_1e-8_s": e2e_time / e2e_steps, "steps": e2e_steps,
                "entry_point": "pwh_davidson_solve_host (pinned host bands in and out)"},
        "gpu_launches": int(launches),
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def run_medium(pwh, syn, torch):
    """The medium cell (a = 20 bohr, 64 atoms, 40 Ry: 34,265 plane waves, 90^3,
    576 projectors), lowest 128 bands: mixed + Jacobi-Davidson (median of three
    solves after one warm-up) and one plain FP64 solve, CUDA-event timed."""
    cell = syn.config_cell("medium", 0)
    nb = syn.CONFIGS["medium"]["nb"]
    s, v, beta, D = make_system(pwh, syn, cell)
    psi0 = torch.from_numpy(syn.initial_bands(0, s.npw, nb)).cuda()
    psi = torch.empty_like(psi0)
    stream = torch.cuda.current_stream()

    def solve(mixed):
        psi.copy_(psi0)
        return s.davidson(psi, tol=TOL, mult=MULT, mixed=mixed, switch_tol=SWITCH_TOL,
                          jd_inner=JD_INNER if mixed else 0)
    solve(True)
    ts = [timed(torch, stream, lambda: solve(True)) for _ in range(3)]
    tmix = statistics.median(t for t, _ in ts)
    eig = ts[-1][1][0]
    t64, (eig64, st64, _) = timed(torch, stream, lambda: solve(False))
    hp = hpsi_only(torch, s, psi0)
    # the generalised problem H x = e S x of ultrasoft / PAW projectors:
    # S = 1 + sum_i |beta_i> q_i <beta_i|, q_i ~ U(0.1, 0.8) (seeded)
    q = np.random.default_rng(8).uniform(0.1, 0.8, beta.shape[0])
    t_set, _ = timed(torch, stream, lambda: s.set_overlap(q))
    solve(True)
    t_gen, (eig_g, st_g, status_g) = timed(torch, stream, lambda: solve(True))
    assert status_g == 0
    s.set_overlap(None)
    s.close()
    return {"workload": f"medium: a=20 bohr, 64 atoms, 40 Ry, npw={s.npw}, 90^3, 576 projectors, "
                        f"{nb} bands", "time_to_1e-8_s": {"mixed": tmix, "fp64": t64},
            "fp64_over_mixed": t64 / tmix, "iters": {"mixed": ts[-1][1][1]["iters"],
                                                     "fp64": st64["iters"]},
            "max_abs_dlambda_mixed_vs_fp64_ha": float(np.abs(eig - eig64).max()),
            "hpsi_only": hp,
            "generalised": {"problem": "H x = e S x, S = 1 + sum_i |beta_i> q_i <beta_i|, "
                                       "q_i ~ U(0.1, 0.8), mixed + Jacobi-Davidson",
                            "set_overlap_s": t_set, "time_to_1e-8_s": t_gen,
                            "iters": st_g["iters"],
                            "lowest_eig_shift_ha": float(eig_g[0] - eig[0])}}


def run_ace(pwh, syn, torch, nocc=ACE_NOCC):
    """Exact exchange on the medium cell: the ACE operator built from the
    lowest `nocc` bands (one FP64 solve supplies them; pair densities and
    Poisson solves on the 90^3 box), H|psi> on the 128 resident bands with and
    without the ACE term (median of 20), and one mixed + Jacobi-Davidson solve
    of H + V_ACE to 1e-8 (alpha = 0.25, the PBE0 fraction), CUDA-event timed."""
    cell = syn.config_cell("medium", 0)
    nb = syn.CONFIGS["medium"]["nb"]
    s, v, beta, D = make_system(pwh, syn, cell)
    stream = torch.cuda.current_stream()
    psi0 = torch.from_numpy(syn.initial_bands(0, s.npw, nb)).cuda()
    psi = psi0.clone()
    eig0, _, status = s.davidson(psi, tol=TOL, mult=MULT, mixed=True, switch_tol=SWITCH_TOL,
                                 jd_inner=JD_INNER)
    assert status == 0
    occ_bands = psi[:nocc].contiguous()
    occ = np.full(nocc, 2.0)
    t_build, rank = timed(torch, stream, lambda: s.set_ace(occ_bands, occ, 0.25))
    out = torch.empty_like(psi0)
    res = {}
    for label, on in (("without_ace", False), ("with_ace", True)):
        if not on:
            s.set_ace(None)
        else:
            s.set_ace(occ_bands, occ, 0.25)
        for _ in range(3):
            s.apply_h(psi0, out)
        ts = [timed(torch, stream, lambda: s.apply_h(psi0, out))[0] for _ in range(HPSI_REPS)]
        res[label] = {"band_applies_s": nb / statistics.median(ts),
                      "median_ms": 1e3 * statistics.median(ts)}

    def solve():
        psi.copy_(psi0)
        return s.davidson(psi, tol=TOL, mult=MULT, mixed=True, switch_tol=SWITCH_TOL,
                          jd_inner=JD_INNER)
    solve()
    t_solve, (eig, st, status) = timed(torch, stream, solve)
    assert status == 0
    s.close()
    return {"workload": f"medium cell, ACE from the lowest {nocc} bands (weights 2, alpha 0.25), "
                        f"{nb} bands to 1e-8", "nocc": nocc, "rank": int(rank),
            "ace_build_s": t_build, "pair_densities": nocc * nocc, "hpsi_only_mixed": res,
            "solve_with_ace_s": t_solve, "iters": st["iters"],
            "lowest_eig_shift_ha": float(eig[0] - eig0[0])}


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


# The FP64-accurate FFT passes of the compiled box sizes run in double-float
# arithmetic (pairs of FP32 numbers) on the FP32 pipes: a double-float add is
# 20 FP32 instructions, a multiply 7, and the nominal 5 N log2 N flops of a
# transform are 6 adds and 4 multiplies in 10, so one FP64-equivalent flop
# costs 14.8 FP32 instructions; the pipes issue 152 x 128 x 2.07e9 of those a
# second (half the FP32 flop rate, which counts an FMA as two).
DF_FP32_OPS_PER_FLOP = (6 * 20 + 4 * 7) / 10
DF_ALU_TFLOPS = FP32_ALU_TFLOPS / 2 / DF_FP32_OPS_PER_FLOP

FAMILY_BOUND = {
    # family: (bound, counter, peak key)
    "fft_plane_fp32": ("alu", "flops", "fp32"), "fft_plane_fp64": ("alu", "flops", "df"),
    "fft_z_inverse_fp32": ("hbm", "bytes", "hbm"), "fft_z_forward_fp32": ("hbm", "bytes", "hbm"),
    "fft_z_inverse_fp64": ("alu", "flops", "df"), "fft_z_forward_fp64": ("alu", "flops", "df"),
    "tc_gemm_becp": ("tensor", "flops", "bf16"), "tc_gemm_backproj": ("tensor", "flops", "bf16"),
    "cgemm_fp64": ("alu", "flops", "fp64"), "cgemm_fp32": ("alu", "flops", "fp32"),
    "jacobi_fp64": ("alu", "flops", "fp64"), "cholqr_fp64": ("alu", "flops", "fp64"),
    "jacobi_fp32": ("alu", "flops", "fp32"), "zgemm_fp64_tc": ("tensor", "flops", "bf16"),
    "zgemm_fp32_tc": ("tensor", "flops", "bf16"),
}


# DRAM traffic per unit of work of a kernel family, from ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum per launch divided by the
# units that launch processed; summaries and commands under profiles/).
# Families missing here report traffic null.
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) behind the
# roofline, from ncu captures summarised under profiles/: per launch of a
# family as it runs in the large solve (the capture made inside the same
# command), or per counted flop of one representative product, scaled by the
# launch's flops.  A family whose kernels changed after the capture is absent
# (traffic null).
TRAFFIC_PER_LAUNCH = {    # family -> bytes per launch
    # (the FP32 Jacobi's capture, profiles/jacobi_fp32_large_solve_dram.md,
    # predates the kernel's current phase-1 schedule and double buffering)
}
TRAFFIC_PER_FLOP = {      # family -> bytes per counted flop
    # one 1088 x 544 x 16,384 FP64-equivalent product on the persistent
    # tensor-core kernel (bench.py --gemm 1088,544,16384,fp64,1): 6.12 GB of
    # DRAM traffic over its six kernels for 2.79e12 counted tensor flops
    # (profiles/oz_gemm_fp64_conj_1088x544x16384.md)
    "zgemm_fp64_tc": 6.118e9 / 2.7928e12,
}


def family_roofline(fam, d, s=None):
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
    elif key == "df":
        peak, unit = DF_ALU_TFLOPS, "TFLOP/s"
        psrc = "derived double-float rate (FP32 instruction rate / 14.8)"
        achieved = work / sec / 1e12
    else:
        peak, unit, psrc = FP64_ALU_TFLOPS, "TFLOP/s", "nominal FP64 rate"
        achieved = work / sec / 1e12
    traffic = None
    if fam in TRAFFIC_PER_LAUNCH:
        traffic = TRAFFIC_PER_LAUNCH[fam]
    elif fam in TRAFFIC_PER_FLOP and work:
        traffic = TRAFFIC_PER_FLOP[fam] * work
    return {"kernel": fam, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": (achieved / peak) if (peak and work) else None, "traffic": traffic,
            "avg_launch_ms": d["ms"] / d["launches"], "peak_source": psrc}


def roofline(kt, s=None):
    """Roofline of the kernel family with the largest device time in a solve
    (CUDA events on the solver's stream), its algorithmic work per launch
    divided by its average launch duration."""
    fams = {k: v for k, v in kt.items() if v["launches"]}
    fam = max(fams, key=lambda k: fams[k]["ms"])
    tot = sum(v["ms"] for v in fams.values())
    r = family_roofline(fam, fams[fam], s)
    r["share_of_timed_kernels"] = fams[fam]["ms"] / tot
    return r


CPU_SAMPLE_BANDS = 64   # bands per oracle H application in the CPU baseline (about 10 s)
REF_SAMPLE_BANDS = 4    # bands per step of the reference arm


def oracle_apply(cell, v, beta, D, psi_h):
    """The oracle's FP64 H (FFT route) on the host cores; returns seconds."""
    from oracle import basis as ob
    from oracle import hamiltonian as oh
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    t = time.perf_counter()
    oh.apply_h(b, v, beta, D, psi_h)
    return time.perf_counter() - t


def cpu_baseline(cell, npw, fft, v, beta, D, psi0_h, nbands=CPU_SAMPLE_BANDS):
    """The oracle (numpy FP64) on a bounded sample of the same workload: one
    application of H to the first `nbands` starting bands (scatter, 3D FFTs,
    potential, gather, kinetic, projector products), band-applies/s."""
    dt = oracle_apply(cell, v, beta, D, psi0_h[:nbands])
    return {"value": nbands / dt, "unit": "band-applies/s", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle", "sample": f"H applied to {nbands} of the {psi0_h.shape[0]} starting "
                                         f"bands of the same workload ({dt:.1f} s)"}


# ------------------------------------------------------------- reference ----
def run_reference(a):
    """The oracle as the reference arm: each step a bounded sample of the same
    workload on the host cores (H applied to REF_SAMPLE_BANDS bands)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1709_10010_gb300 import synthetic as syn
    from oracle import basis as ob
    cfg = syn.CONFIGS[WORKLOAD]
    cell = syn.config_cell(WORKLOAD, 0)
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    v = syn.potential_grid(cell, b.fft)
    beta = syn.projectors(cell, b.miller)
    D = syn.d_diagonal(cell)
    psi0 = syn.initial_bands(0, b.npw, cfg["nb"])
    nb = REF_SAMPLE_BANDS
    for i in range(a.warmup):
        oracle_apply(cell, v, beta, D, psi0[:1])
    t_all = 0.0
    for i in range(a.steps):
        j = (i * nb) % cfg["nb"]
        t_all += oracle_apply(cell, v, beta, D, psi0[j:j + nb])
    value = nb * a.steps / t_all
    sample = f"H applied to {nb} of the {cfg['nb']} starting bands per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "band-applies/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * t_all / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"large: a=30 bohr cubic, 216 atoms, 50 Ry, npw={b.npw}, "
                                   f"{beta.shape[0]} projectors, {cfg['nb']} bands; bounded "
                                   f"sample: {sample}"},
            "cpu_baseline": {"value": value, "unit": "band-applies/s",
                             "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                             "sample": sample},
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
