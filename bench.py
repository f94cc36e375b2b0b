"""Benchmark of the plane-wave H|psi> + Davidson hot path on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload medium] [--mode fp64|mixed]

Prints ONE JSON line (rank 0).  See the design doc for the workload, the metric and
the roofline accounting.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hpsi band-applies/s and Davidson time-to-1e-8 residual, mixed vs FP64, 1 GB300"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="medium")
    p.add_argument("--mode", default="fp64", choices=["fp64", "mixed"])
    return p.parse_args()


def build_inputs(name, seed=0):
    from paper_1709_10010_gb300 import synthetic as syn
    cfg = syn.CONFIGS[name]
    cell = syn.config_cell(name, seed)
    return cfg, cell


def main():
    a = parse()
    import torch
    import paper_1709_10010_gb300 as pwh
    from paper_1709_10010_gb300 import synthetic as syn
    torch.cuda.set_device(0)
    cfg, cell = build_inputs(a.workload)
    s = pwh.System.from_cell(cell, precision=a.mode)
    miller = s.miller()
    v = syn.potential_grid(cell, s.fft)
    beta = syn.projectors(cell, miller)
    s.set_potential(v)
    s.set_projectors(beta, syn.d_diagonal(cell))
    nb = cfg["nb"]
    psi = torch.from_numpy(syn.initial_bands(0, s.npw, nb)).cuda()
    hpsi = torch.empty_like(psi)
    for _ in range(a.warmup):
        s.apply_h(psi, hpsi)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.steps):
        s.apply_h(psi, hpsi)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    out = {"metric": METRIC, "value": nb / (ms * 1e-3), "unit": "band-applies/s", "n_gpus": 1,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
           "mode": a.mode, "config": {"workload": a.workload, "npw": s.npw, "fft": s.fft, "nb": nb,
                                      "nproj": int(beta.shape[0])}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
