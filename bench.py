#!/usr/bin/env python3
"""Throughput of the batched phaseless-AFQMC walker step on GB300.

Default workload (the throughput case): solid-like synthetic Hamiltonian with M=512
orbitals, N_up=N_dn=128, Nchol=2560 Cholesky vectors (h banded, bandwidth 64,
N(0, 0.2); L_n symmetric N(0,1) x 0.5 exp(-n/200) / sqrt(M)), 1024 walkers per GPU,
tau=0.005, QR every 5 steps, mixed-estimator energy measured every step, BF16X3
tensor-core contractions with FP64 LU / QR / reductions.  One timed "step" is one
full walker step for every walker (overlap, Green's function, energy + force bias,
fields, HS potential, Taylor propagator, new overlap, weights, QR amortised).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

For N > 1 launch with torch.distributed.run; each rank owns an independent walker set
(walkers are independent: weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walker-steps/sec at M=512,N=128,Nchol=2560; mixed vs FP64 at ≤1 mHa"
UNIT = "walker-steps/s"
WORKLOAD = ("solid-like synthetic Hamiltonian: M=512, N_up=N_dn=128, Nchol=2560, h banded (bw 64), "
            "L_n decay exp(-n/200), W=1024 walkers/GPU, tau=0.005, QR/5, energy measured every step")


def workload_desc(wl):
    """The config description of a single-system workload (the throughput system's fixed text)."""
    if wl.name == "m512":
        return WORKLOAD.replace("W=1024", f"W={wl.W}")
    kind = "solid-like" if wl.band else "molecule-like"
    return (f"{kind} synthetic Hamiltonian: M={wl.M}, N_up={wl.Nup}, N_dn={wl.Ndn}, Nchol={wl.Nchol}, "
            f"L_n decay exp(-n/{wl.decay:g}), W={wl.W} walkers/GPU, tau={wl.tau}, QR/{wl.k_qr}, "
            "energy measured every step")


def workload_metric(wl):
    return METRIC if wl.name == "m512" else f"walker-steps/sec at M={wl.M},N={wl.Nup},Nchol={wl.Nchol}"


def l2_note(wl):
    """Whether the step's streamed inputs (Ltilde planes, Theta pair) exceed the 129 MB L2."""
    lt = 3 * 2 * wl.Nchol * wl.Nup * wl.M
    th = 2 * 2 * 2 * 2 * wl.W * wl.Nup * wl.M
    big = lt > 129e6 or th > 129e6
    return (f"inputs larger than L2 (Ltilde planes {lt / 1e9:.2f} GB, Theta pair {th / 1e9:.2f} GB per step)" if big
            else f"inputs fit in L2 (Ltilde planes {lt / 1e6:.0f} MB, Theta pair {th / 1e6:.0f} MB); no flush")


# DRAM bytes of one launch of the energy kernel at this workload (dram__bytes_read.sum +
# dram__bytes_write.sum, one ncu capture of this script; the summary and its command are in
# profiles/).  The figure holds for the kernel source it was taken on: a digest of that source
# (the energy-kernel section of kernels_tc.cu and the PTX wrappers) gates it.
# DRAM bytes per launch of the energy kernel at the bench workload: one-pass ncu counters on a
# W = 16 launch of the same kernel (2,465,579,264 read + 5,491,968 written), scaled by 64 to
# W = 1024 -- the kernel streams L~ once per window of 8 walker-spin groups, so its traffic grows
# in proportion to W (profiles/energy_pair_kernel_traffic_m512.md).  Reported only while the
# kernel's source matches the digest it was measured on.
ENERGY_TRAFFIC = {"bytes": 64 * (2465579264 + 5491968), "src_digest": "ea121992e632cfdb"}


def energy_src_digest() -> str:
    import hashlib
    csrc = os.path.join(ROOT, "paper_2003_01831_gb300", "csrc")
    src = open(os.path.join(csrc, "kernels_tc.cu")).read()
    a = src.index("// --------------------------------------------------------------------------- energy kernel")
    b = src.index("// --------------------------------------------------------------------------- row split")
    h = hashlib.sha1(src[a:b].encode())
    h.update(open(os.path.join(csrc, "tc_ptx.cuh")).read().encode())
    return h.hexdigest()[:16]


def energy_traffic():
    if ENERGY_TRAFFIC["bytes"] is None or ENERGY_TRAFFIC["src_digest"] != energy_src_digest():
        return None
    return ENERGY_TRAFFIC["bytes"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), d.get("hbm_gbs", 6800.0), "measured"
    return 1900.0, 1700.0, 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def build_system(wl):
    from paper_2003_01831_gb300 import synthetic as syn
    rng = wl.rng()
    h, L, E0 = syn.make_hamiltonian(wl.M, wl.Nchol, rng, decay=wl.decay, band=wl.band, reading=wl.reading)
    Psi = syn.make_trial(h, wl.Nup, wl.Ndn)
    return h, L, E0, Psi


CHECK_W = 4              # walkers of the full-size oracle check (walker 0 is compared)


def oracle_config1():
    """The oracle on the small molecule-like workload in full: M=24, N=5+5, Nchol=120, 16
    walkers, 50 steps, QR every 5 steps, energy measured every step (caller fields)."""
    from oracle import afqmc as O
    from paper_2003_01831_gb300 import synthetic as syn
    wl = syn.workload("m24")
    h, L, E0 = syn.make_hamiltonian(wl.M, wl.Nchol, wl.rng(), decay=wl.decay, band=wl.band, reading=wl.reading)
    Psi = syn.make_trial(h, wl.Nup, wl.Ndn)
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    p = O.Params(tau=wl.tau, k_taylor=6, k_qr=wl.k_qr)
    B = O.half_one_body_propagator(ham, wl.tau)
    wk = O.init_walkers(ham, Psi, wl.W)
    x = syn.make_fields(wl.nsteps, wl.W, wl.Nchol, seed=0)
    t0 = time.perf_counter()
    for s in range(wl.nsteps):
        O.step(ham, Psi, B, wk, x[s], p)
    t = time.perf_counter() - t0
    return {"value": wl.W * wl.nsteps / t, "unit": UNIT, "walkers": wl.W, "steps": wl.nsteps, "seconds": t,
            "extrapolated": False,
            "workload": "molecule-like M=24, N=5+5, Nchol=120, tau=0.005, QR/5, energy every step, measured in full"}


def cpu_baseline(wl, h, L, E0, Psi):
    """The oracle as it stands, on the host cores: one walker-step of the full-size throughput
    system (M=512, N=128+128, Nchol=2560), timed directly, beside the small workload run in
    full.  The same oracle step doubles as a full-size check of the mixed-precision GPU path:
    a BF16X3 walker set takes one step with the same caller fields, and walker 0's local
    energy, weight and log-overlap after the step are compared with the oracle's."""
    import torch
    from oracle import afqmc as O
    from paper_2003_01831_gb300 import api, synthetic as syn
    from paper_2003_01831_gb300.walkers import AFQMC
    cores = len(os.sched_getaffinity(0))
    x = syn.make_fields(1, CHECK_W, wl.Nchol, seed=99)
    stream = torch.cuda.current_stream().cuda_stream
    with AFQMC(h, L, E0, Psi[0], Psi[1], CHECK_W, wl.tau, k_qr=wl.k_qr, precision=api.PREC_BF16X3,
               stream=stream) as g:
        g.step(1, x, measure_every=1)
        E_gpu, w_gpu, l_gpu, _ = g.energy()
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    p = O.Params(tau=wl.tau, k_taylor=6, k_qr=wl.k_qr)
    B = O.half_one_body_propagator(ham, wl.tau)
    wk = O.init_walkers(ham, Psi, 1)
    t0 = time.perf_counter()
    O.step(ham, Psi, B, wk, x[0, :1], p)
    t = time.perf_counter() - t0
    E_o = O.local_energy(ham, Psi, wk.Phi)[0][0]
    check = {"walker": 0, "after_steps": 1, "E_L_gpu_mixed": [E_gpu[0].real, E_gpu[0].imag],
             "E_L_oracle": [E_o.real, E_o.imag], "abs_dE_L_Ha": float(abs(E_gpu[0] - E_o)),
             "rel_dw": float(abs(w_gpu[0] - wk.w[0]) / abs(wk.w[0])),
             "abs_dlogS": float(abs(l_gpu[0] - wk.logS[0])), "bar_Ha": 1e-3}
    return {"value": 1.0 / t, "unit": UNIT, "cores": cores, "kind": "oracle", "extrapolated": False,
            "sample": f"one walker-step of the throughput system itself (M={wl.M}, N={wl.Nup}+{wl.Ndn}, "
                      f"Nchol={wl.Nchol}, energy measured), timed directly: {t:.1f} s; set-up excluded",
            "config1": oracle_config1(), "full_size_check": check}


def run_reference(args, wl, rank, world):
    """The oracle as it stands on the host cores, timed directly on the throughput system
    itself (M=512, N=128+128, Nchol=2560): every timed step is one oracle walker-step (energy
    measured, caller fields), about 9 s on 16 cores.  Walkers are independent, so one walker of
    the workload is the bounded sample of each step; value = walker-steps per second."""
    if rank != 0:
        return 0
    from oracle import afqmc as O
    from paper_2003_01831_gb300 import synthetic as syn
    cores = len(os.sched_getaffinity(0))
    h, L, E0, Psi = build_system(wl)
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    p = O.Params(tau=wl.tau, k_taylor=6, k_qr=wl.k_qr)
    B = O.half_one_body_propagator(ham, wl.tau)
    wk = O.init_walkers(ham, Psi, 1)
    x = syn.make_fields(args.warmup + args.steps, 1, wl.Nchol, seed=0)
    for s in range(args.warmup):
        O.step(ham, Psi, B, wk, x[s], p)
    t0 = time.perf_counter()
    for s in range(args.warmup, args.warmup + args.steps):
        O.step(ham, Psi, B, wk, x[s], p)
    t = (time.perf_counter() - t0) / max(args.steps, 1)
    v = 1.0 / t
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD + "; each timed step is one walker of it", "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "extrapolated": False,
                             "sample": f"each step: one oracle walker-step of the throughput system itself "
                                       f"(M={wl.M}, N={wl.Nup}+{wl.Ndn}, Nchol={wl.Nchol}, energy measured), "
                                       f"timed directly; set-up excluded"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def step_floor(wl, bf16_sust, hbm_gbs, sm_max_mhz):
    """Roofline time of one whole step (every phase at its own bound, summed): the dense
    contractions -- energy T = Ltilde Theta (8 W Nchol N^2 M), HS potential (4 W M^2 Nchol),
    Taylor terms (2 spins x K x 8 W M^2 N), the two one-body factors (2 spins x 2 x 4 W M^2 N),
    overlaps and Green's function (2 spins x (2 x 4 + 8) W M N^2) -- at the sustained tensor
    peak; the overlap inverse (2W complex N^3 Gauss-Jordan, 8 N^3 flops each) and the QR
    (2W x (16 M N^2 + 8 N^3) per QR, every k_qr steps) at the FP64 DFMA peak; the bytes
    that must move (Ltilde pair, L^T slices, walkers in and out) at the copy bandwidth."""
    W, M, N, nch, K = wl.W, wl.M, wl.Nup, wl.Nchol, 6
    tensor = (8.0 * W * nch * N * N * M + 4.0 * W * M * M * nch + 2 * K * 8.0 * W * M * M * N
              + 2 * 2 * 4.0 * W * M * M * N + 2 * 16.0 * W * M * N * N)
    fp64 = 2 * W * 8.0 * N ** 3 + 2 * W * (16.0 * M * N * N + 8.0 * N ** 3) / max(wl.k_qr, 1)
    fp64_peak = 304 * 2 * sm_max_mhz * 1e6
    nbytes = nch * N * M * 4 + 3 * M * M * nch * 2 + 2 * 2 * W * 2 * N * M * 8
    t = tensor / (bf16_sust * 1e12) + fp64 / fp64_peak + nbytes / (hbm_gbs * 1e9)
    return 1e3 * t, {"tensor_flops": tensor, "fp64_flops": fp64, "bytes": nbytes}


FP64_CMP = (64, 10)     # walkers and steps of the FP64-versus-mixed comparison


def fp64_compare(wl, h, L, E0, Psi, seed):
    """The plain FP64 GPU step against the mixed-precision (BF16X3) step on the same system,
    walkers and fields: both walker sets start at the trial and draw the same Philox fields
    (same seed and walker offset), with the energy measured every step and QR every k_qr
    steps.  Each is timed with CUDA events over the whole run (E_mix written to device
    memory, so nothing synchronises inside)."""
    import torch
    from paper_2003_01831_gb300 import api
    from paper_2003_01831_gb300.walkers import AFQMC
    W, steps = FP64_CMP
    stream = torch.cuda.current_stream().cuda_stream
    out, traces = {}, {}
    for name, prec in (("fp64", api.PREC_FP64), ("mixed", api.PREC_BF16X3)):
        with AFQMC(h, L, E0, Psi[0], Psi[1], W, wl.tau, k_qr=wl.k_qr, precision=prec, stream=stream) as g:
            tr = torch.zeros(steps, dtype=torch.complex128, device="cuda")
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            api.afqmc_step(g.wk, steps, None, seed, 1, tr, stream)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            traces[name] = tr.cpu().numpy()
            out[name] = {"value": W * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps}
    d = np.abs(traces["fp64"] - traces["mixed"])
    out.update({"walkers": W, "steps": steps, "fields": f"device Philox, seed {seed}, identical for both",
                "E_mix_fp64": [float(v) for v in traces["fp64"].real],
                "max_abs_dE_mix_Ha": float(d.max()), "bar_Ha": 1e-3,
                "mixed_over_fp64_same_walkers": out["mixed"]["value"] / out["fp64"]["value"]})
    return out


def batch_line(args, rank, world):
    """Uneven multi-system batch: 64 systems, M ~ U{32..256}, N = floor(M/4), Nchol = 5M,
    W ~ U{32..256}, tau = 0.01, QR every 10 steps, BF16X3 (padded to tensor-core shapes),
    energy measured every step, one CUDA-graph launch per step, autotuned launch shapes."""
    import torch
    from paper_2003_01831_gb300 import api, synthetic as syn
    from paper_2003_01831_gb300.walkers import Batch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dims = syn.uneven_batch(64)
    systems = []
    for i, d in enumerate(dims):
        h, L, E0, Psi = syn.make_uneven_system(d, i)
        systems.append((h, L, E0, Psi[0], Psi[1], d.W))
    prec = api.PREC_BF16X3 if args.precision == "bf16x3" else api.PREC_FP64
    lib = api.lib()
    lib.afqmc_debug_set_batch_padding.argtypes = [ctypes.c_int]
    api._check(lib.afqmc_debug_set_batch_padding(args.batch_pad_granule))
    b = Batch(systems, 0.01, precision=prec, k_qr=10)
    del systems
    tuned_ms = b.autotune(reps=2)
    shape, _ = b.info(0)
    seed = 4321 + rank
    b.step(args.warmup, seed=seed, measure_every=1)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        torch.cuda.nvtx.range_push("afqmc_timed")
        ev0.record()
        b.step(args.steps, seed=seed, measure_every=1)
        ev1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms = ev0.elapsed_time(ev1)
    Wtot = sum(d.W for d in dims)
    value = world * Wtot * args.steps / (ms / 1e3)
    _, nk = b.info(0)
    # algorithmic flops of the energy contraction (the dominant term): 8 W Nchol N^2 M per system,
    # and the flops the padded shapes (M', N', Nchol') run
    alg = sum(8.0 * d.W * d.Nchol * d.N * d.N * d.M for d in dims)
    padded, tiles = 0.0, 0.0
    for i, d in enumerate(dims):
        sh_i, _ = b.info(i)
        Mp, Np, Ncp = int(sh_i[0]), int(sh_i[1]), int(sh_i[2])
        padded += 8.0 * d.W * Ncp * Np ** 2 * Mp
        # what the tensor cores issue (per product): pair tiles of 2 x 128 rows (floor(128/N')
        # Cholesky vectors each) by 256 columns (floor(128/N') walker-spins), K = M'
        G = 128 // Np
        n_pairs = -(-(-(-Ncp // G)) // 2)
        ws_groups = -(-(2 * d.W) // G)
        tiles += 2.0 * n_pairs * ws_groups * 128 * 256 * 2.0 * Mp
    _, bf16_sust, _, src = peaks()
    ach = alg / (ms / args.steps / 1e3) / 1e12
    line = {"metric": "walker-steps/sec, 64 uneven systems (M~U{32..256}, N=M/4, Nchol=5M, W~U{32..256})",
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16 row-scaled splits (1-3 slices, f32 accumulate) + f64" if prec == api.PREC_BF16X3 else "f64",
            "data": "synthetic",
            "config": {"workload": f"64 uneven molecule-like systems, {Wtot} walkers in total, tau=0.01, QR/10, "
                                   "energy every step, padded to tensor-core shapes, one graph launch per step",
                       "l2": "inputs larger than L2", "parallelism": f"walker replicas x{world}",
                       "autotuned": {"graph_branches": int(shape[3]), "gemm_bn_max": int(shape[4]),
                                     "grid_cap": int(shape[5]),
                                     "energy_launch": "one persistent launch over every system" if int(shape[6])
                                     else "one launch per system", "energy_k_chunk": int(shape[7]),
                                     "tuned_ms_per_step": tuned_ms},
                       "n_padding": f"N' = N rounded up to a multiple of {args.batch_pad_granule}"
                                    if args.batch_pad_granule == 8 else "N' in {32, 64, 128}",
                       "padded_energy_flops_over_algorithmic": padded / alg,
                       "energy_tile_flops_over_algorithmic": tiles / alg},
            "clocks": clk.summary(), "gpu_launches": int(nk) * args.steps if nk > 0 else None,
            "roofline": {"bound": "tensor", "achieved": ach, "peak": bf16_sust, "unit": "TFLOP/s",
                         "frac": ach / bf16_sust, "traffic": None,
                         "kernel": "whole step (energy-contraction flops of every system / step time)",
                         "peak_source": f"bf16_tflops_sustained of {src} peaks"}}
    b.close()
    return line


def run_batch(args, rank, world):
    line = batch_line(args, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def config2_compare(seed, steps=5):
    """The molecule-like workload at its stated size (M=128, N=32+32, Nchol=640, W=512, QR/10):
    the mixed-precision and the plain FP64 GPU step on the same walkers and Philox fields, one
    untimed step then `steps` timed ones (energy every step), E_mix compared over all of them."""
    import torch
    from paper_2003_01831_gb300 import api, synthetic as syn
    from paper_2003_01831_gb300.walkers import AFQMC
    wl = syn.workload("m128")
    h, L, E0, Psi = build_system(wl)
    stream = torch.cuda.current_stream().cuda_stream
    out, traces = {}, {}
    for name, prec in (("fp64", api.PREC_FP64), ("mixed", api.PREC_BF16X3)):
        with AFQMC(h, L, E0, Psi[0], Psi[1], wl.W, wl.tau, k_qr=wl.k_qr, precision=prec, stream=stream) as g:
            tr = torch.zeros(steps + 1, dtype=torch.complex128, device="cuda")
            api.afqmc_step(g.wk, 1, None, seed, 1, tr[:1], stream)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            api.afqmc_step(g.wk, steps, None, seed, 1, tr[1:], stream)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            traces[name] = tr.cpu().numpy()
            out[name] = {"value": wl.W / (ms / 1e3), "unit": UNIT, "ms_per_step": ms}
    d = np.abs(traces["fp64"] - traces["mixed"])
    out.update({"workload": workload_desc(wl), "steps": steps + 1, "fields": f"device Philox, seed {seed}",
                "max_abs_dE_mix_Ha": float(d.max()), "bar_Ha": 1e-3,
                "mixed_over_fp64": out["mixed"]["value"] / out["fp64"]["value"]})
    return out


def run_bp(args, rank, world):
    """Back-propagated one-body density matrix at the throughput system: W walkers (BF16X3 by
    default) take --warmup steps, open a window of nbp = --steps steps and step through it;
    afqmc_bp_rdm1 then carries the trial back through the window's adjoint propagators and
    forms the weighted density matrices (FP64 zgemm and the batched inverse).  value =
    back-propagated walker-steps per second of that call, timed with CUDA events on the
    launching stream."""
    import torch
    from paper_2003_01831_gb300 import api, synthetic as syn
    from paper_2003_01831_gb300.walkers import AFQMC
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    wl = syn.workload("m512", W=args.walkers or 1024)
    h, L, E0, Psi = build_system(wl)
    prec = api.PREC_BF16X3 if args.precision == "bf16x3" else api.PREC_FP64
    stream = torch.cuda.current_stream().cuda_stream
    g = AFQMC(h, L, E0, Psi[0], Psi[1], wl.W, wl.tau, k_qr=wl.k_qr, precision=prec, stream=stream,
              walker_offset=rank * wl.W)
    del L
    seed, nbp, M, K = 1234, args.steps, wl.M, 6
    for _ in range(args.warmup):
        g.step(1, None, seed=seed, measure_every=1)
    g.bp_begin(nbp)
    g.step(nbp, None, seed=seed, measure_every=1)
    torch.cuda.synchronize()
    G = [torch.empty((M, M), dtype=torch.complex128, device="cuda") for _ in range(2)]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record()
        api.afqmc_bp_rdm1(g.wk, G[0], G[1], stream)
        ev1.record()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    trace = [float(torch.trace(G[s]).real) for s in range(2)]
    # end to end through the public API: the same call with host outputs
    Gh = [np.zeros((M, M), dtype=np.complex128) for _ in range(2)]
    t0 = time.perf_counter()
    api.afqmc_bp_rdm1(g.wk, Gh[0], Gh[1], stream)
    e2e_s = time.perf_counter() - t0
    # the final estimate alone: a window of no steps (the same overlap, inverse and walker sum)
    g.bp_begin(0)
    torch.cuda.synchronize()
    ev0.record()
    api.afqmc_bp_rdm1(g.wk, G[0], G[1], stream)
    ev1.record()
    torch.cuda.synchronize()
    est_ms = ev0.elapsed_time(ev1)
    g.close()
    W, nch, Ns = wl.W, wl.Nchol, (wl.Nup, wl.Ndn)
    # algorithmic FP64 flops: per back step the HS potential (complex x real, 4 W M^2 Nchol), K
    # Taylor terms (complex, 8 W M^2 N each) and B twice (complex x real) per spin; then per spin
    # the overlap, Theta (8 W M N^2 each), the inverse (~8 W N^3) and the walker sum (8 M^2 W N)
    back = nbp * (4.0 * W * M * M * nch + sum((8.0 * K + 8.0) * W * M * M * n for n in Ns))
    # final estimate: overlap, inverse, Theta and the walker sum M x M x (W N): in FP64 on an FP64
    # walker set; on a BF16X3 one the three GEMMs run on the tensor cores and the inverse in
    # float pairs on the fp32 pipe
    est_fp64 = sum(16.0 * W * M * n * n + 8.0 * W * n ** 3 for n in Ns)
    est_sum = sum(8.0 * M * M * W * n for n in Ns)
    est = est_fp64 + est_sum
    clocks = clk.summary()
    fp64_peak = 304 * 2 * (clocks.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
    _, bf16_sust, _, src = peaks()
    tc_back = prec == api.PREC_BF16X3
    back_ms = max(ms - est_ms, 1e-6)
    back_peak = bf16_sust if tc_back else fp64_peak
    phases = {"back_steps": {"ms": back_ms, "algorithmic_flops": back,
                             "achieved_tflops": back / (back_ms / 1e3) / 1e12,
                             "peak": back_peak, "bound": "tensor" if tc_back else "alu (FP64 DFMA)",
                             "frac": back / (back_ms / 1e3) / 1e12 / back_peak},
              "final_estimate": ({"ms": est_ms, "algorithmic_flops": est,
                                  "achieved_tflops": est / (est_ms / 1e3) / 1e12, "peak": bf16_sust,
                                  "bound": "tensor (overlap, Theta and walker-sum GEMMs; the inverse in float "
                                           "pairs on the fp32 pipe)",
                                  "frac": est / (est_ms / 1e3) / 1e12 / bf16_sust} if tc_back else
                                 {"ms": est_ms, "algorithmic_flops": est,
                                  "achieved_tflops": est / (est_ms / 1e3) / 1e12, "peak": fp64_peak,
                                  "bound": "alu (FP64 DFMA)",
                                  "frac": est / (est_ms / 1e3) / 1e12 / fp64_peak})}
    dom = "back_steps" if back_ms >= est_ms else "final_estimate"
    # launches: per back step conj + HS GEMM + per spin (B, K Taylor terms, B, QR every k_qr);
    # then per spin overlap, inverse, Theta, two layout passes, walker-sum GEMM, transpose, check
    qr = sum(1 for k in range(nbp) if wl.k_qr > 0 and (k + 1) % wl.k_qr == 0 and k + 1 < nbp)
    if prec == api.PREC_BF16X3:   # layout passes, per back step the three-slice propagation's kernels
        launches = 1 + 2 + 2 + nbp * (8 + 2 * K) + qr * 6 + 2 + 14 + 2 * 6   # estimate: Green's functions, walker sums
    else:
        launches = 1 + 2 + nbp * (2 + 2 * (K + 2)) + 2 * qr + 2 * 8
    line = {"metric": "back-propagated walker-steps/sec (one-body density matrix of a window at M=512, N=128, "
                      "Nchol=2560)",
            "value": world * W * nbp / (ms / 1e3), "unit": "walker-steps/s", "n_gpus": world, "steps": nbp,
            "warmup": args.warmup, "ms_per_step": ms / nbp, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f16 row-scaled splits (3 slices) + f64" if prec == api.PREC_BF16X3 else "f64",
            "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}; back-propagation window of {nbp} steps, walkers "
                                   f"{'BF16X3' if prec == api.PREC_BF16X3 else 'FP64'}",
                       "l2": "inputs larger than L2 (L 5.4 GB, walkers 1.1 GB per spin)",
                       "parallelism": f"walker replicas x{world}"},
            "clocks": clocks, "gpu_launches": launches,
            "e2e": {"value": world * W * nbp / e2e_s, "unit": "walker-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 2 * 16 * M * M, "per": "one afqmc_bp_rdm1 call, host outputs"},
            "traces": trace, "phases": phases,
            # the phase that takes most of the call: back steps (three-slice tcgen05 propagation on
            # a BF16X3 walker set, zgemm on an FP64 one) or the FP64 final estimate
            "roofline": {"bound": "tensor" if tc_back else "alu",
                         "achieved": phases[dom]["achieved_tflops"], "peak": phases[dom]["peak"],
                         "unit": "TFLOP/s", "frac": phases[dom]["frac"], "traffic": None,
                         "kernel": ("afqmc_bp_rdm1 back steps (tcgen05 three-slice propagation, adjoint)"
                                    if tc_back else "afqmc_bp_rdm1 back steps (FP64 zgemm)")
                         if dom == "back_steps" else
                         ("afqmc_bp_rdm1 final estimate (overlap, Theta and walker sum on tcgen05, float-pair "
                          "inverse)" if tc_back else
                          "afqmc_bp_rdm1 final estimate (FP64 zgemm, batched inverse, split walker sum)"),
                         "phase": dom,
                         "peak_source": (f"bf16_tflops_sustained of {src} peaks (algorithmic complex flops)"
                                         if tc_back else
                                         "FP64 DFMA pipe: 304 DFMA per clock x 2 flops x max SM clock")}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_grad(args, rank, world):
    """Differentiation workload (M=256, N=64+64, Nchol=1280, W=256 walkers near the trial): each
    timed step is one forward local energy and log-overlap plus the backward pass with respect to
    the trial orbitals and the Cholesky tensor, through autograd.LocalEnergy on device tensors
    (FP64 adjoint, Theta recomputed).  value = walker gradients per second."""
    import torch
    from paper_2003_01831_gb300 import synthetic as syn
    from paper_2003_01831_gb300.autograd import local_energy
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = syn.workload("m256", W=args.walkers or 256)
    rng = wl.rng()
    h, L, E0 = syn.make_hamiltonian(wl.M, wl.Nchol, rng)
    Psi = syn.make_trial(h, wl.Nup, wl.Ndn)
    W, M = wl.W, wl.M
    Phi = []
    for s in range(2):
        z = Psi[s][None] + 0.1 * (rng.standard_normal((W, M, wl.Nup)) + 1j * rng.standard_normal((W, M, wl.Nup)))
        Phi.append(torch.tensor(np.linalg.qr(z)[0], device=dev))
    Lt = torch.tensor(L, device=dev, requires_grad=True)
    del L
    ht = torch.tensor(h, device=dev)
    Pu = torch.tensor(Psi[0], device=dev, requires_grad=True)
    Pd = torch.tensor(Psi[1], device=dev, requires_grad=True)
    gE = torch.ones(W, dtype=torch.complex128, device=dev)

    def one():
        E, lS = local_energy(Pu, Pd, Lt, ht, E0, Phi[0], Phi[1])
        loss = torch.sum(torch.real(torch.conj(gE) * E + lS))
        Pu.grad = Pd.grad = Lt.grad = None
        loss.backward()

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            one()
        ev1.record()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    N, nch = wl.Nup, wl.Nchol
    # algorithmic FP64 flops per evaluation, per (Cholesky vector, walker, spin): T = Ltilde Theta in
    # the forward and again in the backward (4 N^2 M each, real x complex), U = Theta T (8 M N^2),
    # sum_n L_n U_n (4 M^2 N); plus the dL products F = V Psi^+ (8 M^2 N per vector and spin)
    flops = 2.0 * W * nch * (16.0 * N * N * M + 4.0 * M * M * N) + 2.0 * nch * 8.0 * M * M * N
    clocks = clk.summary()
    fp64_peak = 304 * 2 * (clocks.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
    ach = flops / (ms / 1e3) / 1e12
    line = {"metric": "walker gradients/sec (local energy and log-overlap w.r.t. trial and Cholesky tensor) "
                      "at M=256, N=64, Nchol=1280",
            "value": world * W / (ms / 1e3), "unit": "walker-gradients/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"differentiation system M=256, N=64+64, Nchol=1280, W={W} walkers near the "
                                   "trial; one step = forward + backward through autograd.LocalEnergy on device "
                                   "tensors", "l2": "inputs larger than L2 (L 0.67 GB)",
                       "parallelism": f"walker replicas x{world}"},
            "clocks": clocks,
            "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": ach / fp64_peak, "traffic": None,
                         "kernel": "whole forward + backward (FP64 adjoint GEMMs)",
                         "peak_source": "FP64 DFMA pipe: 304 DFMA per clock x 2 flops x max SM clock"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_fp64_variant(args, rank, world):
    """The wider rows on the FP64 path, at the m128 system (M=128, N=32+32, Nchol=640,
    W=512, tau=0.005, QR/10, energy every step, Philox fields):
      cplx128 -- general complex Cholesky vectors (complex N(0,1) x 0.5 e^{-n/20} / sqrt(M)),
                 run as their 1280 Hermitian-split vectors;
      msd128  -- a 4-determinant non-orthogonal trial (the lowest orbitals of h plus 0.3 x
                 complex N(0,1) per determinant, complex N(0,1) coefficients).
    value = walker-steps/s (CUDA events); roofline: the step's algorithmic FP64 flops of the
    energy contraction (per determinant) over the DFMA pipe's peak at the maximum SM clock."""
    import torch
    from paper_2003_01831_gb300 import api, synthetic as syn
    from paper_2003_01831_gb300.walkers import AFQMC
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    wl = syn.workload("m128", W=args.walkers or 512)
    rng = wl.rng()
    h, L, E0 = syn.make_hamiltonian(wl.M, wl.Nchol, rng, decay=wl.decay, band=wl.band, reading=wl.reading)
    P = syn.make_trial(h, wl.Nup, wl.Ndn)
    kw, Psi, ND, nv, lt_complex = {}, P, 1, wl.Nchol, False
    if args.workload == "cplx128":
        scale = 0.5 * np.exp(-np.arange(wl.Nchol) / wl.decay)[:, None, None] / np.sqrt(wl.M)
        L = scale * (rng.standard_normal(L.shape) + 1j * rng.standard_normal(L.shape))
        nv, lt_complex = 2 * wl.Nchol, True
        desc = f"complex Cholesky vectors (Hermitian split: {nv} vectors)"
    else:
        ND = 4
        crn = lambda *sh: rng.standard_normal(sh) + 1j * rng.standard_normal(sh)
        Psi = [np.stack([P[s] + 0.3 * crn(wl.M, P[s].shape[1]) for _ in range(ND)]) for s in range(2)]
        kw["coeffs"] = crn(ND)
        lt_complex = True
        desc = f"{ND}-determinant non-orthogonal trial"
    stream = torch.cuda.current_stream().cuda_stream
    g = AFQMC(h, L, E0, Psi[0], Psi[1], wl.W, wl.tau, k_qr=wl.k_qr, precision=api.PREC_FP64, stream=stream,
              walker_offset=rank * wl.W, **kw)
    seed = 1234
    for _ in range(args.warmup):
        g.step(1, None, seed=seed, measure_every=1)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            g.step(1, None, seed=seed, measure_every=1)
        ev1.record()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    _, kernels_per_step = api.afqmc_last_step_stats(g.wk)
    g.close()
    W, M, N = wl.W, wl.M, wl.Nup
    # T = Ltilde Theta per determinant, spin and vector: N x M x N complex MACs (8 flops), or
    # real x complex (4 flops) for a real trial and real L
    alg = ND * 2 * W * nv * N * N * M * (8.0 if lt_complex else 4.0)
    clocks = clk.summary()
    peak = 304 * 2 * clocks["sm_max_mhz"] * 1e6 / 1e12 if clocks.get("sm_max_mhz") else None
    ach = alg / (ms / 1e3) / 1e12
    line = {"metric": f"walker-steps/sec at M=128, N=32, Nchol=640 with {desc} (FP64 path)",
            "value": world * W / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"m128 molecule-like system, W={W} walkers/GPU, tau=0.005, QR/10, energy every "
                                   f"step, {desc}", "l2": "inputs larger than L2",
                       "parallelism": f"walker replicas x{world}"},
            "clocks": clocks, "gpu_launches": int(kernels_per_step * args.steps) if kernels_per_step > 0 else None,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak if peak else None, "traffic": None,
                         "kernel": "whole FP64 step (energy-contraction flops / step time)",
                         "peak_source": "FP64 DFMA pipe: 304 DFMA per clock x 2 flops x max SM clock"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_thc(args, rank, world):
    """Tensor-hypercontraction Hamiltonian (Sec. V, Eqs. (4)-(6)) on the FP64 path, shaped like the
    molecule-like throughput system: M=128, N=32+32, N_mu = 8 M = 1024 interpolating points
    (X ~ N(0, 1/M), kernel B B^T with B ~ N(0, 0.5/sqrt(N_mu))), h molecule-like, W=512,
    tau=0.005, QR/10, energy measured every step, Philox fields.  value = walker-steps/s (CUDA
    events); roofline: the step's algorithmic FP64 flops of the contractions through the points
    (Z = Theta^T X, T = (Psi^+ X)^T Z, X diag(U c) X^T) over the DFMA pipe's peak."""
    import torch
    from paper_2003_01831_gb300 import api, synthetic as syn
    from paper_2003_01831_gb300.walkers import AFQMC
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    M, N, Nmu, W, tau, kqr = 128, 32, 1024, args.walkers or 512, 0.005, 10
    rng = np.random.default_rng(1006)
    h, _, E0 = syn.make_hamiltonian(M, 1, rng)
    X, Mk = syn.make_thc(M, Nmu, rng)
    Psi = syn.make_trial(h, N, N)
    stream = torch.cuda.current_stream().cuda_stream
    g = AFQMC(h, None, E0, Psi[0], Psi[1], W, tau, k_qr=kqr, precision=api.PREC_FP64, stream=stream,
              walker_offset=rank * W, thc=(X, Mk))
    nch = g.Nchol
    seed = 1234
    for _ in range(args.warmup):
        g.step(1, None, seed=seed, measure_every=1)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            g.step(1, None, seed=seed, measure_every=1)
        ev1.record()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    _, kernels_per_step = api.afqmc_last_step_stats(g.wk)
    g.close()
    # per walker and spin: Z (complex x real, 4 N M Nmu), T (4 N Nmu^2); per walker: the HS
    # potential X diag(d) X^T (complex x real, 4 M^2 Nmu) -- the contractions through the points
    alg = W * (2 * (4.0 * N * M * Nmu + 4.0 * N * Nmu * Nmu) + 4.0 * M * M * Nmu)
    clocks = clk.summary()
    peak = 304 * 2 * clocks["sm_max_mhz"] * 1e6 / 1e12 if clocks.get("sm_max_mhz") else None
    ach = alg / (ms / 1e3) / 1e12
    line = {"metric": "walker-steps/sec at M=128, N=32, N_mu=1024 with a THC Hamiltonian (FP64 path)",
            "value": world * W / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"THC molecule-like system: M={M}, N={N}+{N}, N_mu={Nmu} (rank {nch} "
                                   f"fields), W={W} walkers/GPU, tau={tau}, QR/{kqr}, energy every step",
                       "l2": "inputs larger than L2", "parallelism": f"walker replicas x{world}"},
            "clocks": clocks, "gpu_launches": int(kernels_per_step * args.steps) if kernels_per_step > 0 else None,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak if peak else None, "traffic": None,
                         "kernel": "whole FP64 step (THC contraction flops / step time)",
                         "peak_source": "FP64 DFMA pipe: 304 DFMA per clock x 2 flops x max SM clock"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="m512")
    ap.add_argument("--walkers", type=int, default=0)
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp64"])
    ap.add_argument("--energy-terms", type=int, default=0, choices=[0, 1, 2, 3, 4])
    ap.add_argument("--energy-pair", type=int, default=-1, choices=[-1, 0, 1],
                    help="energy kernel form: 0 one CTA per tile, 1 CTA pairs, -1 the library default")
    ap.add_argument("--batch-pad-granule", type=int, default=8, choices=[8, 32],
                    help="batch64: pad each system's N to a multiple of 8 (default) or to 32/64/128")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-config2", action="store_true", help="skip the m128 mixed-vs-FP64 key of the default line")
    ap.add_argument("--no-batch-line", action="store_true", help="skip the batch64 key of the default line")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_2003_01831_gb300 import synthetic as syn
    if args.workload in ("cplx128", "msd128"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle baseline is defined for the "
                              "single-system throughput workload only"}), flush=True)
            return 0
        return run_fp64_variant(args, rank, world)
    if args.workload == "thc128":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle baseline is defined for the "
                              "single-system throughput workload only"}), flush=True)
            return 0
        return run_thc(args, rank, world)
    if args.workload == "grad256":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle baseline is defined for the "
                              "single-system throughput workload only"}), flush=True)
            return 0
        return run_grad(args, rank, world)
    if args.workload == "bp512":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle baseline is defined for the "
                              "single-system throughput workload only"}), flush=True)
            return 0
        return run_bp(args, rank, world)
    wl = syn.workload(args.workload if args.workload != "batch64" else "m512")
    if args.walkers:
        wl = syn.workload(wl.name, W=args.walkers)
    if args.workload == "batch64":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle baseline is defined for the "
                              "single-system throughput workload only"}), flush=True)
            return 0
        return run_batch(args, rank, world)
    if args.impl == "reference":
        return run_reference(args, wl, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2003_01831_gb300 import api, distributed
    from paper_2003_01831_gb300.walkers import AFQMC

    h, L, E0, Psi = build_system(wl)
    prec = api.PREC_BF16X3 if args.precision == "bf16x3" else api.PREC_FP64
    stream = torch.cuda.current_stream().cuda_stream
    if args.energy_pair >= 0:
        api.lib().afqmc_debug_set_energy_variant.argtypes = [ctypes.c_int]
        api._check(api.lib().afqmc_debug_set_energy_variant(args.energy_pair))
    # rank r holds walkers [r W, (r + 1) W) of one population: same seed, offset Philox counter
    g = AFQMC(h, L, E0, Psi[0], Psi[1], wl.W, wl.tau, k_qr=wl.k_qr, precision=prec, stream=stream,
              walker_offset=rank * wl.W, energy_terms=args.energy_terms)
    seed = 1234

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up
    for _ in range(args.warmup):
        g.step(1, None, seed=seed, measure_every=1)
    barrier()
    # timed region: device-resident inputs (fields drawn on the device)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # with several ranks every measured step also combines the population's E_mix: the library
    # writes this rank's partial sums (sum w E_L, sum w) to device memory and NCCL all-reduces
    # them on the device
    sums = torch.zeros((args.steps, 4), dtype=torch.float64, device="cuda") if dist is not None else None
    with Clocks(local) as clk:
        torch.cuda.nvtx.range_push("afqmc_timed")
        ev0.record()
        for i in range(args.steps):
            g.step(1, None, seed=seed, measure_every=1)
            if dist is not None:
                api.afqmc_mixed_sums(g.wk, 1, sums[i], stream)
                distributed.allreduce_sums(sums[i])
        ev1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms_total = ev0.elapsed_time(ev1)
    emix_population = distributed.emix_from_sums(sums) if dist is not None else None
    # secondary number: energy measured every 10th step (the other steps contract only the force
    # bias, t_n = Tr(Ltilde_n Theta))
    barrier()
    es0 = torch.cuda.Event(enable_timing=True)
    es1 = torch.cuda.Event(enable_timing=True)
    es0.record()
    g.step(10, None, seed=seed, measure_every=10)
    es1.record()
    torch.cuda.synchronize()
    sec_ms = es0.elapsed_time(es1) / 10
    secondary = {"metric": "walker-steps/sec with the energy measured every 10th step", "unit": UNIT,
                 "value": world * wl.W / (sec_ms / 1e3), "ms_per_step": sec_ms, "steps": 10}
    # duration of the dominant kernel (events recorded around it by the library on the launching
    # stream); read after each step, which synchronises, so it is kept out of the timed loop
    e_ms = []
    for _ in range(min(args.steps, 3)):
        g.step(1, None, seed=seed, measure_every=1)
        e_ms.append(api.afqmc_last_step_stats(g.wk)[0])
    t = torch.tensor([ms_total], device="cuda")
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_total = float(t.item())
    value = world * wl.W * args.steps / (ms_total / 1e3)
    clocks = clk.summary()

    # end to end through the public API with host buffers: fields from pinned host memory,
    # the step's energy read back to the host
    x_host = torch.empty((1, wl.W, wl.Nchol), dtype=torch.float64).pin_memory()
    x_host.copy_(torch.from_numpy(syn.make_fields(1, wl.W, wl.Nchol, seed=7)))
    xn = x_host.numpy()
    e2e_steps = max(2, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        trace = g.step(1, xn, measure_every=1)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * wl.W * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(xn.nbytes), "d2h_bytes_per_step": int(trace.nbytes)}
    _, kernels_per_step = api.afqmc_last_step_stats(g.wk)

    # roofline of the dominant kernel: the fused energy contraction; issued tensor flops are the
    # mean number of split products per tile times the algorithmic ones
    lib = api.lib()
    lib.afqmc_debug_energy_products.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    mean_products = ctypes.c_double(0.0)
    issued = None
    if prec == api.PREC_BF16X3 and lib.afqmc_debug_energy_products(g.wk, ctypes.addressof(mean_products)) == 0:
        issued = mean_products.value
    bf16_burst, bf16_sust, hbm, src = peaks()
    N, M, nch, W = wl.Nup, wl.M, wl.Nchol, wl.W
    alg_flops = 8.0 * W * nch * N * N * M          # 2 spins x real-complex T = Ltilde Theta
    e_avg = float(np.mean([m for m in e_ms if m > 0])) if any(m > 0 for m in e_ms) else None
    roof = None
    if e_avg:
        ach = alg_flops / (e_avg / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": bf16_sust, "unit": "TFLOP/s",
                "frac": ach / bf16_sust, "traffic": energy_traffic() if args.walkers == 0 else None,
                "kernel": "tc_energy_kernel<128> (one CTA per tile)" if args.energy_pair == 0
                else "tc_energy_pair_kernel<128> (CTA pairs, cta_group::2)",
                "avg_launch_ms": e_avg, "issued_over_algorithmic": issued,
                "peak_source": f"bf16_tflops_sustained of {src} peaks (kernel timed inside a long step)"}
    if roof is not None:
        floor_ms, floor_parts = step_floor(wl, bf16_sust, hbm, clocks.get("sm_max_mhz") or 2070.0)
        roof["step_frac"] = floor_ms / (ms_total / args.steps)
        roof["step_floor_ms"] = floor_ms
        roof["step_floor_parts"] = floor_parts
        if issued:
            roof["issued_ceiling_frac"] = 1.0 / issued
    line = {"metric": workload_metric(wl), "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f16 row-scaled splits (1-3 slices, f32 accumulate) + f64" if prec == api.PREC_BF16X3 else "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(wl), "l2": l2_note(wl),
                       "parallelism": f"walker replicas x{world}"},
            "clocks": clocks, "e2e": e2e, "secondary": secondary,
            "gpu_launches": int(kernels_per_step * args.steps) if kernels_per_step > 0 else None,
            "roofline": roof}
    if emix_population is not None:
        line["population_E_mix"] = [float(v) for v in emix_population.real]
    g.close()
    if world == 1 and not args.no_fp64_compare:
        cmp = fp64_compare(wl, h, L, E0, Psi, seed)
        cmp["mixed_over_fp64_at_bench_walkers"] = value / cmp["fp64"]["value"]
        line["fp64_compare"] = cmp
    if world == 1 and not args.no_config2:
        line["config2_compare"] = config2_compare(seed)
    if world == 1 and not args.no_batch_line:
        bargs = argparse.Namespace(**vars(args))
        bargs.steps, bargs.warmup = 5, 2
        bl = batch_line(bargs, rank, world)
        line["batch64"] = {k: bl[k] for k in ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "clocks",
                                              "roofline")}
        line["batch64"]["config"] = bl["config"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, h, L, E0, Psi)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
