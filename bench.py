"""Benchmark: 21-cm likelihood evaluations per second on 128^3 x 3-redshift boxes.

One step = one batched likelihood call (eor_likelihood) for W walkers: per walker and
redshift the whole excursion-set path (tables, filter + inverse FFT per radius, flag,
partial ionization, delta T_b, power spectrum) and the chi^2, summed over redshifts. One
evaluation = one walker's three-redshift chi^2. Inputs are seeded synthetic boxes (a BBKS
Gaussian random field grown to z and clipped at delta > -1) and walker parameters drawn
uniformly from zeta in [5, 100], R_mfp in [5, 20] Mpc, log10 T_vir in [4, 6].

    python bench.py [--gpus N] [--steps K] [--warmup W] [--walkers 128] [--impl reference]

Under torchrun (N > 1) each rank evaluates its own walkers on its own GPU (weak scaling);
ranks share no data, only a barrier and the max of the timings. Rank 0 prints one JSON
line. `--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload instead.
"""
from __future__ import annotations

import argparse
import math
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "21cm likelihood evals/s at 128³×3z, batched vs plain; HBM roofline %"
N, BOX, ZS = 128, 250.0, (8.0, 9.0, 10.0)
FIDUCIAL = (30.0, 15.0, 4.7)
WORKLOAD = "128^3 boxes, L=250 Mpc, z=8,9,10; batched walkers (zeta, R_mfp, log10 T_vir) uniform in [5,100]x[5,20]x[4,6]"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--walkers", type=int, default=128)
    ap.add_argument("--nz", type=int, default=3, choices=[1, 2, 3],
                    help="redshifts of the workload used (the first of z = 8, 9, 10); fewer only for small profiling cases")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-walkers", type=int, default=16, help="walkers timed one call each (plain path)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-trace", action="store_true", help="time without the per-kernel event brackets")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--no-direct", action="store_true", help="skip timing the per-radius FFT method")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparison")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch schedule (profiling runs)")
    ap.add_argument("--ps-split", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="force the power spectrum's tiling after the autotuner (0 slab passes, 1 planes, "
                         "2 plane clusters; -1: keep its choice)")
    ap.add_argument("--no-emulator", action="store_true", help="skip the surrogate leg")
    ap.add_argument("--no-mcmc", action="store_true", help="skip the device-side sampler leg")
    ap.add_argument("--mcmc-steps", type=int, default=10)
    ap.add_argument("--no-two-pop", action="store_true", help="skip the 256^3 two-population leg")
    ap.add_argument("--two-pop-walkers", type=int, default=64)
    ap.add_argument("--two-pop-only", action="store_true",
                    help="time only the 256^3 two-population workload (its own JSON object)")
    ap.add_argument("--two-pop-efficiency", type=int, default=1, choices=[0, 1],
                    help="efficiency model of the 256^3 leg (0: the step function, for comparison)")
    ap.add_argument("--emu-train", type=int, default=20000, help="simulated walkers the surrogate trains on")
    ap.add_argument("--emu-steps", type=int, default=32000, help="Adam steps of the surrogate")
    ap.add_argument("--emu-walkers", type=int, default=4096, help="walkers per surrogate likelihood call")
    return ap.parse_args()


def dist_env():
    """(rank, world size, local rank) under torchrun; a single process otherwise."""
    world = int(os.environ.get("WORLD_SIZE", 1))
    if world <= 1:
        return 0, 1, 0
    return int(os.environ.get("RANK", 0)), world, int(os.environ.get("LOCAL_RANK", 0))


# ------------------------------------------------------------------ CPU oracle (baseline / reference arm)

def oracle_sample(seconds: float, walkers_params, delta, mock, sigma, gpu=None):
    """Time the FP64 oracle on (walker, redshift) realizations of the workload until the
    budget is spent (at least one). Returns (evals/s, realizations, seconds, threads, parity):
    with gpu = (x_HI boxes [walker][z] (torch, device), Delta^2 [walker][z][bin]) of the
    batched GPU path on the same walkers, parity holds the errors of those realizations
    against the oracle's (outside the timed sum)."""
    import oracle
    orc = oracle.Oracle()
    t0 = time.perf_counter()
    done, el, errs = 0, 0.0, []
    while True:
        w, j = divmod(done, len(ZS))
        w %= len(walkers_params)
        t1 = time.perf_counter()
        ion = orc.ionize(delta[j], BOX, ZS[j], *walkers_params[w])
        d2, _, cnt = oracle.power_spectrum(ion["dtb"], BOX, 14, 0.1, 1.5)
        c_ref = oracle.chi2(d2, cnt, mock[j], sigma[j])
        el += time.perf_counter() - t1
        done += 1
        if gpu is not None:
            xg = gpu[0][w, j].double().cpu().numpy()
            diff = np.abs(xg - ion["xhi"])
            flipped = diff > 1e-3
            ok = cnt > 0
            dg = gpu[1][w, j]
            if ion["xhi_mean"] > 0.01:
                pe = float(np.max(np.abs(dg[ok] - d2[ok]) / np.abs(d2[ok])))
            else:
                pe = float(np.max(np.abs(dg[ok] - d2[ok])) / max(np.max(np.abs(d2[ok])), 1e-6))
            c_gpu = oracle.chi2(dg, cnt, mock[j], sigma[j])
            errs.append((float(flipped.mean()), float(diff[~flipped].max()) if (~flipped).any() else 0.0, pe,
                         abs(c_gpu - c_ref) / max(abs(c_ref), 1e-12)))
        if time.perf_counter() - t0 >= seconds:
            break
    per_eval = el / done * len(ZS)
    parity = None
    if errs:
        e = np.array(errs)
        parity = {"realizations": len(errs), "flipped_frac_max": float(e[:, 0].max()),
                  "xhi_abs_err_max": float(e[:, 1].max()), "xhi_abs_err_median": float(np.median(e[:, 1])),
                  "d2_rel_err_max": float(e[:, 2].max()), "d2_rel_err_median": float(np.median(e[:, 2])),
                  "chi2_rel_err_max": float(e[:, 3].max()),
                  "tolerances": {"flipped": 1e-4, "xhi": 1e-4, "d2": 1e-3},
                  "def": "batched GPU x_HI and Delta^2 of the sampled (walker, z) against the FP64 oracle; "
                         "chi^2 per redshift on a flat mock (10 mK^2, sigma 20 %)"}
    return 1.0 / per_eval, done, el, orc.threads, parity


def oracle_one_thread():
    """Seconds of one 128^3 realization (fiducial walker, z = 9) by the oracle on one host
    thread, the setting of the paper's single-core timing (Sec. 2.3), and the CPU model."""
    import oracle
    from paper_1501_06576_gb300 import synth
    orc = oracle.Oracle()
    before = orc.threads
    orc.lib.or_set_threads(1)
    try:
        box = synth.density_boxes(N, BOX, (9.0,), seed=1)[0]
        t0 = time.perf_counter()
        ion = orc.ionize(box, BOX, 9.0, *FIDUCIAL)
        oracle.power_spectrum(ion["dtb"], BOX, 14, 0.1, 1.5)
        secs = time.perf_counter() - t0
    finally:
        orc.lib.or_set_threads(before)
    return secs


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    from paper_1501_06576_gb300 import synth
    import oracle
    delta = synth.density_boxes(N, BOX, ZS, seed=1)
    params = synth.walker_params(max(args.walkers, 1), seed=3)
    mock = np.full((len(ZS), 14), 10.0)
    sigma = 0.2 * mock
    per_step = []
    orc = oracle.Oracle()
    for s in range(args.warmup + args.steps):
        w = s % len(params)
        j = s % len(ZS)
        t0 = time.perf_counter()
        ion = orc.ionize(delta[j], BOX, ZS[j], *params[w])
        d2, _, cnt = oracle.power_spectrum(ion["dtb"], BOX, 14, 0.1, 1.5)
        oracle.chi2(d2, cnt, mock[j], sigma[j])
        if s >= args.warmup:
            per_step.append(time.perf_counter() - t0)
    mean = statistics.mean(per_step)
    value = 1.0 / (mean * len(ZS))
    sample = "each step: one walker at one redshift of the workload (128^3 ionization over its radius ladder, delta T_b, Delta^2, chi^2), FP64; evals/s = 1 / (3 x seconds per realization)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "box_mpc": BOX, "z": list(ZS), "walkers": args.walkers},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": orc.threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm helpers

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources of each traced kernel class: a traffic record taken before a change to them is
# not used
CLASS_SOURCES = {
    "basis_ionize": ("basis.cu", "tcgen05.cu", "tc.cuh"),
    "forward_fft": ("kernels.cu", "fft_core.cuh", "eor_internal.cuh"),
    "ps_plane": ("kernels.cu", "fft_core.cuh", "eor_internal.cuh"),
}


def class_source_hash(kernel_class: str) -> str:
    """Hash of the sources of a kernel class's kernels."""
    h = hashlib.sha256()
    for name in CLASS_SOURCES[kernel_class]:
        with open(os.path.join(ROOT, "paper_1501_06576_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_launch_traffic(kernel_class: str, units: float, ps_split=None):
    """DRAM bytes (read + write) of one launch that processes `units` units of its class, from
    the committed ncu capture (bytes per unit, as measured on a launch of the same grid size
    n and spectrum tiling), or None if the class's sources, the grid or the tiling (the
    spectrum's classes run different kernels per tiling) differ from the capture's."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d["per_class"][kernel_class]
        if e["source_hash"] != class_source_hash(kernel_class) or e["n"] != N:
            return None
        if "ps_split" in e and e["ps_split"] != ps_split:
            return None
        return e["bytes_per_unit"] * units
    except Exception:
        return None


SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0


def fp32_peak_tflops() -> float:
    """FP32 FMA peak from unit counts and the maximum SM clock: 152 SMs x 128 lanes x 2 flop."""
    return SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12


def tf32_peak_tflops():
    """Dense TF32 tensor peak: the measured BF16 GEMM peak (sustained: the contraction runs
    inside a long step) times the nominal TF32/BF16 ratio 1.1/2.25."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            bf16 = float(json.load(f)["bf16_tflops_sustained"])
        kind = "measured bf16 sustained x 1.1/2.25"
    except Exception:
        bf16, kind = 1700.0, "fallback bf16 sustained x 1.1/2.25"
    return bf16 * 1.1 / 2.25, kind


def fp16_peak_tflops():
    """Dense FP16 tensor peak: the measured BF16 GEMM peak (FP16 and BF16 run at the same
    rate), sustained (the contraction runs inside a long step)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "measured bf16 sustained (FP16 runs at the BF16 rate)"
    except Exception:
        return 1700.0, "fallback bf16 sustained"


def f16_column_chunks(ladders) -> int:
    """256-column chunks of the FP16 contraction for walkers with these radius counts: each
    walker's radii above R_cell in groups of 32 (at least one group; a two-group walker starts
    on an even group)."""
    g = 0
    for nr in ladders:
        ng = max(1, -(-(nr - 1) // 32))
        if ng == 2 and g % 2:
            g += 1
        g += ng
    return -(-g * 32 // 256)


def time_direct(ctx, eor21, torch, stream, flush, d_params, d_mock, d_sigma, W, steps, method=None, note=None):
    """Batched evals/s of another method on the same walkers (comparison only): by default
    the per-radius FFT method."""
    ctx.set_method(eor21.EOR_METHOD_DIRECT if method is None else method)
    for _ in range(2):
        ctx.likelihood(d_params, d_mock, d_sigma)
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dsteps = max(2, steps // 3)
    flush.zero_()
    d0.record(stream)
    for _ in range(dsteps):
        ctx.likelihood(d_params, d_mock, d_sigma)
    d1.record(stream)
    torch.cuda.synchronize()
    ctx.set_method(eor21.EOR_METHOD_BASIS)
    return {"value": W * dsteps / (d0.elapsed_time(d1) / 1e3), "unit": "evals/s",
            "note": note or "filter + inverse FFT per radius (EOR_METHOD_DIRECT), same walkers"}


def time_cufft(ctx, eor21, torch, stream, d_delta, d_params, d_mock, d_sigma, W, tasks, step_share):
    """cuFFT (through torch.fft), timed only as a comparison for the hand-written FFT passes,
    on the same transforms: (1) the forward R2C of the density boxes, once per box; (2) the
    filter W(kR) times the density spectrum and the C2R back to the cells, per (walker, z,
    radius), the work of the per-radius method; (3) the R2C of a delta T_b box, per (walker, z).
    Each against the library's own kernels on the same workload (CUDA-event traces). Nothing
    here feeds a result of the library."""
    n, nz = N, len(ZS)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    out = {}
    with torch.cuda.stream(stream):
        # (1) forward R2C of the n_z density boxes
        ms = timed(lambda: torch.fft.rfftn(d_delta, dim=(1, 2, 3)))
        ctx.trace(True)
        ctx.init_boxes(d_delta)
        ours = ctx.trace_read().get("forward_fft", (0.0, 0))[0]
        out["density_r2c_per_box_ms"] = {"cufft": ms / nz, "ours": ours / nz}
        # (2) filter + C2R per radius task, batches of 16 radii on one box
        kf = 2.0 * math.pi / BOX
        f = torch.fft.fftfreq(n, d=1.0 / n, device="cuda") * kf
        fz = torch.fft.rfftfreq(n, d=1.0 / n, device="cuda") * kf
        kk = torch.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + fz[None, None, :] ** 2)
        spec = torch.fft.rfftn(d_delta[0], dim=(0, 1, 2))
        radii = torch.exp(torch.linspace(math.log(1.3), math.log(20.0), 16, device="cuda")).view(16, 1, 1, 1)
        x = kk[None] * radii
        xs = torch.where(x > 1e-3, x, torch.ones_like(x))
        win = torch.where(x > 1e-3, 3.0 * (torch.sin(xs) - xs * torch.cos(xs)) / xs ** 3, torch.ones_like(x))
        ms = timed(lambda: torch.fft.irfftn(spec[None] * win, s=(n, n, n), dim=(1, 2, 3)))
        ctx.set_method(eor21.EOR_METHOD_DIRECT)
        ctx.likelihood(d_params, d_mock, d_sigma)
        t = ctx.trace_read()
        ctx.set_method(eor21.EOR_METHOD_BASIS)
        ctx.trace(False)
        ours = t.get("filter_plane", (0.0, 0))[0] + t.get("pencil_ionize", (0.0, 0))[0]
        out["filter_c2r_per_radius_ms"] = {"cufft": ms / 16, "ours_direct_method": ours / max(tasks, 1),
                                           "note": "ours also tests Eq. 1 per cell and, at R_cell, forms x_HI, "
                                                   "delta T_b and its R2C along z"}
        del x, xs, win
        # (3) R2C of delta T_b boxes, batches of 32
        boxes = torch.randn((32, n, n, n), dtype=torch.float32, device="cuda")
        ms = timed(lambda: torch.fft.rfftn(boxes, dim=(1, 2, 3)))
        ours = (step_share.get("forward_fft", 0.0) + step_share.get("ps_plane", 0.0)) / (W * nz)
        out["dtb_r2c_per_pair_ms"] = {"cufft": ms / 32, "ours": ours,
                                      "note": "ours also bins k^3 |X|^2 into the 14 shells (FP64 sums)"}
        del boxes
    for v in out.values():
        v["ours_over_cufft"] = (v.get("ours") or v.get("ours_direct_method")) / v["cufft"]
    return out


def time_emulator(ctx, eor21, synth, torch, stream, flush, d_mock, d_sigma, args):
    """The learned surrogate on the same boxes: train on simulated spectra of args.emu_train
    walkers (x 3 redshifts), calibrate the fallback threshold on 2048 more, then time
    likelihood calls of args.emu_walkers walkers (emulated where trusted, simulated
    otherwise) and measure the emulated spectra against the simulation on those walkers."""
    cap = ctx.cfg.max_walkers

    def simulate(p):
        chis, d2s = [], []
        for i in range(0, len(p), cap):
            c, d = ctx.likelihood(torch.from_numpy(p[i:i + cap]).cuda(), d_mock, d_sigma, want_d2=True)
            chis.append(c)
            d2s.append(d)
        return torch.cat(chis), torch.cat(d2s)

    train_p = synth.walker_params(args.emu_train, seed=100)
    val_p = synth.walker_params(2048, seed=101)
    test_p = synth.walker_params(args.emu_walkers, seed=102)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, train_d2 = simulate(train_p)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    _, val_d2 = simulate(val_p)
    test_chi, test_d2 = simulate(test_p)
    emu = eor21.Emulator(z=ZS, members=4, max_rows=max(16384, len(ZS) * args.emu_walkers),
                         max_samples=len(ZS) * args.emu_train, seed=3, stream=stream.cuda_stream)
    emu.set_data(torch.from_numpy(train_p).cuda(), train_d2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = emu.train(args.emu_steps, 1024, 2e-3, seed=11)
    train_s = time.perf_counter() - t0
    tau, val_frac = emu.calibrate(torch.from_numpy(val_p).cuda(), val_d2, recall=0.99)
    d_test = torch.from_numpy(test_p).cuda()
    # accuracy on the timed walkers, against their simulated spectra
    pred, _, fb = emu.predict(test_p)
    truth = test_d2.cpu().numpy()
    ok = np.isfinite(truth) & (truth > emu.cfg.d2_floor)
    err = np.where(ok, np.abs(10.0 ** pred / np.where(ok, truth, 1.0) - 1.0), 0.0).max(axis=(1, 2))
    acc = fb == 0
    # device time of the prediction alone (features, 4 layers x 4 members, combination)
    for _ in range(3):
        emu.predict(d_test)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        emu.predict(d_test)
    e1.record(stream)
    torch.cuda.synchronize()
    predict_ms = e0.elapsed_time(e1) / 10
    for _ in range(2):
        emu.likelihood(ctx, d_test, d_mock, d_sigma)
    steps = max(3, args.steps // 2)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        chi, _, fb2 = emu.likelihood(ctx, d_test, d_mock, d_sigma)
        b.record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    same = bool(torch.equal(chi[fb2 == 1], test_chi[fb2 == 1]))
    emu.close()
    return {"value": args.emu_walkers * steps / (ms / 1e3), "unit": "evals/s", "walkers_per_call": args.emu_walkers,
            "fallback_frac": float(1 - acc.mean()), "miss_frac_over_5pct": float(np.mean(err[acc] > 0.05)) if acc.any() else 0.0,
            "median_rel_err_emulated": float(np.median(err[acc])) if acc.any() else None,
            "p99_rel_err_emulated": float(np.quantile(err[acc], 0.99)) if acc.any() else None,
            "tau_dex": tau, "val_fallback_frac": val_frac, "fallback_chi2_equals_simulation": same,
            "predict_ms": predict_ms, "train": {"walkers": args.emu_train, "samples": args.emu_train * len(ZS),
                                                "steps": args.emu_steps, "batch": 1024, "members": 4,
                                                "seconds": train_s, "final_loss": [float(x) for x in loss]},
            "datagen_s": gen_s,
            "note": "surrogate (4 MLPs 4-256-256-256-14, bf16 weights) with simulation fallback; evals/s over "
                    "likelihood calls of walkers_per_call walkers, device-resident inputs"}


def time_mcmc(ctx, eor21, synth, torch, stream, mock, sigma, args):
    """The device-side stretch-move sampler on the same boxes: an ensemble of twice the
    context's walkers (each half is one batched likelihood call per step), timed with CUDA
    events over args.mcmc_steps steps after two warm-up steps."""
    w = 2 * ctx.cfg.max_walkers
    smp = eor21.Sampler(ctx, n_walkers=w, seed=17)
    x0 = synth.walker_params(w, seed=200, zeta=(20.0, 40.0), r_mfp=(10.0, 20.0), log10_tvir=(4.4, 5.0))
    smp.start(x0, mock, sigma)
    smp.run(2, want_chain=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    smp.run(args.mcmc_steps, want_chain=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    _, lnp, acc = smp.run(2)
    smp.close()
    return {"value": w * args.mcmc_steps / (ms / 1e3), "unit": "evals/s", "walkers": w,
            "steps_per_s": args.mcmc_steps / (ms / 1e3), "ms_per_step": ms / args.mcmc_steps,
            "acceptance_last_steps": float(acc.mean()),
            "note": "stretch-move ensemble sampler on the device: per step two half-ensemble proposals, each "
                    "evaluated by one batched likelihood graph replay, Metropolis decisions on the device; no host "
                    "round trip between steps"}


def time_two_pop(eor21, synth, torch, stream, flush, args):
    """The two-population workload: 256^3 boxes, L = 500 Mpc, z = 8, 9, 10, 64 walkers whose
    efficiency is two power laws zeta_i0 (M / 1e10 Msun)^alpha_i above their own M_min(T_vir,i)
    (efficiency_model 1), batched in one graph replay per step; mock from the seed + 1 boxes at
    (30, 15 Mpc, 4.7) with (alpha_1, zeta_20, alpha_2, log10 T_2) = (0.3, 10, -0.3, 5.3), sigma =
    20 % of it. Timed with CUDA events over args.steps replays after two warm-up replays, L2
    flushed before the timed region."""
    n, box, zs, w = 256, 500.0, (8.0, 9.0, 10.0), args.two_pop_walkers
    model = args.two_pop_efficiency
    rng = np.random.default_rng(31)
    base = np.column_stack([rng.uniform(5, 100, w), rng.uniform(5, 20, w), rng.uniform(4, 6, w)])
    extra = np.column_stack([rng.uniform(-0.5, 0.5, w), rng.uniform(5, 100, w), rng.uniform(-0.5, 0.5, w),
                             rng.uniform(4, 6, w)])
    with torch.cuda.stream(stream):
        ctx = eor21.Context(n=n, box_mpc=box, z=zs, max_walkers=w, efficiency_model=model, stream=stream.cuda_stream)
        ctx.init_boxes(torch.from_numpy(synth.density_boxes(n, box, zs, seed=11)).cuda())
        if model:
            ctx.set_efficiency(np.array([[0.3, 10.0, -0.3, 5.3]] * w))
        ctx.set_params(np.array([[30.0, 15.0, 4.7]]))
        ctx.run_ionization()
        mock = np.ascontiguousarray(ctx.power_spectrum()[0][0])
        ctx.init_boxes(torch.from_numpy(synth.density_boxes(n, box, zs, seed=10)).cuda())
        if model:
            ctx.set_efficiency(extra)
        d_params = torch.from_numpy(base).cuda()
        d_mock = torch.from_numpy(mock).cuda()
        d_sigma = torch.from_numpy(0.2 * mock).cuda()
        ctx.autotune(d_params, d_mock, d_sigma, reps=1)   # launch schedule for this workload (untimed)
        schedule = ctx.get_tuning()
        for _ in range(2):
            ctx.likelihood(d_params, d_mock, d_sigma)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        for _ in range(args.steps):
            ctx.likelihood(d_params, d_mock, d_sigma)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        # one more replay with per-launch events: the share of each kernel class (not timed above)
        ctx.trace(True)
        ctx.likelihood(d_params, d_mock, d_sigma)
        torch.cuda.synchronize()
        cls = ctx.trace_read()
        ctx.trace(False)
        total = sum(v[0] for v in cls.values()) or 1.0
        share = {k: {"ms": v[0], "launches": v[1], "share": v[0] / total} for k, v in cls.items() if v[1] > 0}
        rank, _ = ctx.basis_info()[:2]
        kind, kslots = ctx.contraction_info()
        radii = sum(len(ctx.walker_ladder(k)) for k in range(w)) * len(zs)
        launches = ctx.launch_count()
        ctx.close()
    rates = two_pop_rates(share, rank, radii, n, box, w * len(zs), fp16=kind == eor21.EOR_CONTRACT_FP16)
    return {"value": w / (ms / 1e3), "unit": "evals/s", "ms_per_step": ms, "walkers": w,
            "workload": ("256^3, L = 500 Mpc, z = 8, 9, 10, two populations (efficiency_model 1), alpha in "
                         "[-0.5, 0.5], zeta_i0 in [5, 100], log10 T_vir,i in [4, 6], R_mfp in [5, 20] Mpc") if model else
                        "256^3, L = 500 Mpc, z = 8, 9, 10, step-function efficiency (comparison), zeta in [5, 100], "
                        "log10 T_vir in [4, 6], R_mfp in [5, 20] Mpc",
            "radius_tasks_per_step": radii, "basis_rank": rank, "gpu_launches_per_step": launches,
            "schedule": schedule,
            "classes_traced_step": share, "rates": rates, "dtype": "f32 (FP64 tables)"}


def two_pop_rates(share, rank: int, radii: int, n: int, box: float, pairs: int, fp16: bool = False) -> dict:
    """Achieved rates of the traced replay: the contraction's useful TFLOP/s (2 x rank flop per
    cell and radius task) and the power spectrum's algorithmic GB/s (per (walker, z): the R2C
    pencil pass reads the n^3 delta T_b box and writes the nh n^2 half spectrum; the row pass
    reads and writes, the column pass reads, the planes holding a binned mode)."""
    out = {}
    try:
        hbm_peak, hbm_kind = measured_peak()
        c_ms = share.get("basis_ionize", {}).get("ms", 0.0)
        if c_ms > 0:
            tflops = 2.0 * rank * n ** 3 * radii / (c_ms / 1e3) / 1e12
            peak, kind = fp16_peak_tflops() if fp16 else tf32_peak_tflops()
            out["contraction"] = {"achieved": tflops, "unit": "TFLOP/s", "peak": peak, "frac": tflops / peak,
                                  "peak_kind": kind}
        kf = 2.0 * math.pi / box
        planes = 0
        while planes < n // 2 + 1 and kf * planes < 1.5:
            planes += 1
        plane_bytes = n * n * 8
        fwd_ms = share.get("forward_fft", {}).get("ms", 0.0)
        ps_ms = share.get("ps_plane", {}).get("ms", 0.0)
        if fwd_ms > 0:
            b = pairs * (n ** 3 * 4 + (n // 2 + 1) * plane_bytes)
            out["pencil_r2c"] = {"achieved": b / (fwd_ms / 1e3) / 1e9, "unit": "GB/s", "peak": hbm_peak,
                                 "frac": b / (fwd_ms / 1e3) / 1e9 / hbm_peak, "peak_kind": hbm_kind}
        if ps_ms > 0:
            b = pairs * 3 * planes * plane_bytes
            out["ps_line_passes"] = {"achieved": b / (ps_ms / 1e3) / 1e9, "unit": "GB/s", "peak": hbm_peak,
                                     "frac": b / (ps_ms / 1e3) / 1e9 / hbm_peak, "peak_kind": hbm_kind}
    except Exception as err:   # rates are a report; the timing above stands without them
        out["error"] = str(err)
    return out


def main():
    global ZS
    args = parse()
    ZS = ZS[:args.nz]
    rank, world, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    from paper_1501_06576_gb300 import eor21, shard, synth

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    W = args.walkers
    if args.two_pop_only:
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        print(json.dumps({"two_population": time_two_pop(eor21, synth, torch, stream, flush, args)}))
        return 0

    delta = synth.density_boxes(N, BOX, ZS, seed=1)
    mock_delta = synth.density_boxes(N, BOX, ZS, seed=2)
    params = synth.walker_params(W, seed=3 + rank)

    with torch.cuda.stream(stream):
        ctx = eor21.Context(n=N, box_mpc=BOX, z=ZS, max_walkers=W, stream=stream.cuda_stream)
        # the mock: the fiducial model on the independent seed + 1 boxes (set-up, untimed)
        ctx.init_boxes(torch.from_numpy(mock_delta).cuda())
        ctx.set_params(np.array([FIDUCIAL]))
        ctx.run_ionization()
        mock = ctx.power_spectrum()[0][0]
        sigma = 0.2 * mock
        ctx.init_boxes(torch.from_numpy(delta).cuda())
        d_params = torch.from_numpy(params).cuda()
        d_mock = torch.from_numpy(np.ascontiguousarray(mock)).cuda()
        d_sigma = torch.from_numpy(np.ascontiguousarray(sigma)).cuda()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        # launch schedule picked by the library's autotuner on these walkers (untimed set-up)
        if not args.no_autotune:
            ctx.autotune(d_params, d_mock, d_sigma, reps=3)
        if args.ps_split >= 0:
            ctx.set_ps_split(args.ps_split)
        schedule = ctx.get_tuning()
        if args.ps_split >= 0:
            schedule["forced"] = "ps_split"
        ctx.trace(not args.no_trace)
        for _ in range(args.warmup):
            ctx.likelihood(d_params, d_mock, d_sigma)
        stream.synchronize()

        # ---------------- timed region: device-resident inputs
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        time.sleep(0.3)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        class_ms, class_launches = {}, {}
        launches = 0
        for s in range(args.steps):
            flush.zero_()
            starts[s].record(stream)
            ctx.likelihood(d_params, d_mock, d_sigma)
            ends[s].record(stream)
            launches += ctx.launch_count()
            if not args.no_trace:
                for k, (ms, cnt) in ctx.trace_read().items():
                    class_ms[k] = class_ms.get(k, 0.0) + ms
                    class_launches[k] = class_launches.get(k, 0) + cnt
        torch.cuda.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        clk = clocks.stop()
        total_ms = sum(step_ms)
        if world > 1:
            total_ms = shard.max_over_ranks(total_ms)      # timing only: no data-path collective
            torch.distributed.barrier()
        value = W * world * args.steps / (total_ms / 1e3)

        # units: one per (walker, z, radius)
        ctx.set_params(params)
        ladders = [len(ctx.walker_ladder(w)) for w in range(W)]
        tasks_per_step = sum(ladders) * len(ZS)
        basis_rank, basis_resid = ctx.basis_info()
        contract_kind, k_slots = ctx.contraction_info()

        # ---------------- the per-radius FFT method on the same workload (for comparison)
        ctx.trace(False)
        direct = simt = tf32 = None
        for _ in range(0 if args.no_direct else 1):
            direct = time_direct(ctx, eor21, torch, stream, flush, d_params, d_mock, d_sigma, W, args.steps)
            simt = time_direct(ctx, eor21, torch, stream, flush, d_params, d_mock, d_sigma, W, args.steps,
                               method=eor21.EOR_METHOD_BASIS_SIMT,
                               note="basis contraction on the FP32 units (EOR_METHOD_BASIS_SIMT), same walkers")
            tf32 = time_direct(ctx, eor21, torch, stream, flush, d_params, d_mock, d_sigma, W, args.steps,
                               method=eor21.EOR_METHOD_BASIS_TF32,
                               note="basis contraction on 3xTF32 tensor-core operands with x_HI and delta T_b in "
                                    "its epilogue (EOR_METHOD_BASIS_TF32), same walkers")

        # ---------------- end to end through host buffers (pinned), D2H of chi^2 every step
        h_params = torch.from_numpy(params).pin_memory().numpy()
        h_mock = torch.from_numpy(np.ascontiguousarray(mock)).pin_memory().numpy()
        h_sigma = torch.from_numpy(np.ascontiguousarray(sigma)).pin_memory().numpy()
        ctx.trace(False)
        ctx.likelihood(h_params, h_mock, h_sigma)        # capture outside the timed loop
        e2e_s = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            chi2 = ctx.likelihood(h_params, h_mock, h_sigma)
            e2e_s += time.perf_counter() - t0
        assert np.all(np.isfinite(chi2))
        e2e = W * world * args.steps / e2e_s
        h2d = h_params.nbytes + h_mock.nbytes + h_sigma.nbytes
        d2h = chi2.nbytes

        # ---------------- plain path: one walker per call
        pw = min(args.plain_walkers, W)
        for w in range(2):
            ctx.likelihood(d_params[w:w + 1], d_mock, d_sigma)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for w in range(pw):
            ctx.likelihood(d_params[w:w + 1], d_mock, d_sigma)
        p1.record(stream)
        torch.cuda.synchronize()
        plain = pw / (p0.elapsed_time(p1) / 1e3)

        # ---------------- x_HI and Delta^2 of the batch, for the oracle parity sample (untimed)
        gpu_parity = None
        if not args.no_cpu_baseline and world == 1:
            ctx.set_params(params)
            xg, _ = ctx.run_ionization(want_xhi=True, device=True)
            gpu_parity = (xg, ctx.power_spectrum()[0])

        # ---------------- cuFFT on the same transforms (comparison only)
        cufft = None
        if not args.no_cufft and rank == 0:
            per_step = {k: v / args.steps for k, v in class_ms.items()}
            cufft = time_cufft(ctx, eor21, torch, stream, torch.from_numpy(delta).cuda(), d_params, d_mock,
                               d_sigma, W, tasks_per_step, per_step)

        # ---------------- the device-side ensemble sampler on the same likelihood
        mcmc = None
        if not args.no_mcmc and rank == 0:
            ctx.trace(False)
            mcmc = time_mcmc(ctx, eor21, synth, torch, stream, np.ascontiguousarray(mock),
                             np.ascontiguousarray(sigma), args)

        # ---------------- the learned surrogate with simulation fallback (same boxes)
        emulator = None
        if not args.no_emulator and rank == 0:
            emulator = time_emulator(ctx, eor21, synth, torch, stream, flush, d_mock, d_sigma, args)

    # ---------------- the 256^3 two-population workload (its own context)
    two_pop = None
    if not args.no_two_pop and rank == 0:
        ctx.close()
        try:
            two_pop = time_two_pop(eor21, synth, torch, stream, flush, args)
        except eor21.EorError as err:
            two_pop = {"error": str(err)}

    if rank != 0:
        return 0

    # ---------------- roofline of each kernel class of the step, and of the dominant one
    roof, kernel_rates = None, {}
    if class_ms:
        share = {k: class_ms[k] / sum(class_ms.values()) for k in class_ms if class_ms[k] > 0}
        pairs_per_step = W * len(ZS)
        hbm_peak_v, hbm_kind_v = measured_peak()
        nspec_b = (N // 2 + 1) * N * N * 8
        kf = 2.0 * math.pi / BOX
        planes = sum(1 for kz in range(N // 2 + 1) if kf * kz < 1.5)
        for cls, ms_total in class_ms.items():
            launches_c = max(class_launches.get(cls, 0), 1)
            avg_ms = ms_total / launches_c
            if cls == "basis_ionize":
                # useful flops = 2 x rank per (cell, walker, redshift, radius)
                flops_per_unit = 2.0 * basis_rank * N ** 3
                units = tasks_per_step * args.steps / launches_c
                achieved = flops_per_unit * units / (avg_ms / 1e3) / 1e12
                if contract_kind == eor21.EOR_CONTRACT_FP16:
                    peak, peak_kind = fp16_peak_tflops()
                    executed = 2 * k_slots * N ** 3 * f16_column_chunks(ladders) * 256 * len(ZS)
                    tf32_peak, _ = tf32_peak_tflops()
                    extra = {"executed_fp16_tflops": executed * args.steps / launches_c / (avg_ms / 1e3) / 1e12,
                             "frac_of_tf32_peak": achieved / tf32_peak, "k_slots": k_slots}
                    bound = "tensor"
                elif contract_kind == eor21.EOR_CONTRACT_TF32:
                    peak, peak_kind = tf32_peak_tflops()
                    extra, bound = {}, "tensor"
                else:
                    peak, peak_kind = fp32_peak_tflops(), "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"
                    extra, bound = {}, "alu"
                kernel_rates[cls] = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                     "frac": achieved / peak, "traffic": ncu_launch_traffic(cls, units), "kernel": cls,
                                     "peak_kind": peak_kind, "flops_per_unit": flops_per_unit,
                                     "unit_def": "one (walker, redshift, radius) over all cells",
                                     "units_per_launch": units, "avg_launch_ms": avg_ms, **extra}
            elif cls in ("forward_fft", "ps_plane"):
                # per (walker, redshift): the first pass (slab or pencil) reads the flag words and its
                # share of delta and delta at R_cell and writes the kz planes (the slab pass only those
                # with a binned mode, the pencil pass all n/2 + 1); the second pass (x lines or planes)
                # reads the planes that hold a binned mode
                slab = schedule.get("ps_split") == 0
                if cls == "forward_fft":
                    per_unit = (planes * N * N * 8 if slab else nspec_b) + N ** 3 // 8 + 2 * N ** 3 * 4 // W
                    udef = ("one (walker, redshift): " + (f"write of the {planes} binned kz planes" if slab else
                                                          "half spectrum write") +
                            " + flag words + delta, delta_Rcell share")
                else:
                    per_unit = planes * N * N * 8
                    udef = f"one (walker, redshift): read of the {planes} kz planes with a binned mode"
                units = pairs_per_step * args.steps / launches_c
                achieved = per_unit * units / (avg_ms / 1e3) / 1e9
                kernel_rates[cls] = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak_v, "unit": "GB/s",
                                     "frac": achieved / hbm_peak_v,
                                     "traffic": ncu_launch_traffic(cls, units, schedule.get("ps_split")), "kernel": cls,
                                     "peak_kind": hbm_kind_v, "bytes_per_unit": per_unit, "unit_def": udef,
                                     "units_per_launch": units, "avg_launch_ms": avg_ms}
        dom = max((k for k in class_ms if k in kernel_rates), key=lambda k: class_ms[k])
        roof = dict(kernel_rates[dom], share=share)
    hbm_peak, hbm_kind = measured_peak()
    # the excursion-set path's algorithmic HBM bytes per (walker, z, radius) of a per-radius FFT
    # design: read the density spectrum (nh n^2 complex64) and read + write the cell's flag byte
    task_bytes = (N // 2 + 1) * N * N * 8 + 2 * N ** 3
    per_radius_rate = task_bytes * tasks_per_step * args.steps / (total_ms / 1e3) / 1e9

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        flat = np.full((len(ZS), 14), 10.0)     # the oracle takes no input from the GPU path
        cv, nrel, secs, cores, parity = oracle_sample(args.cpu_seconds, params, delta, flat, 0.2 * flat,
                                                      gpu=(gpu_parity[0], gpu_parity[1]) if gpu_parity else None)
        one = oracle_one_thread()
        cpu = {"value": cv, "unit": "evals/s", "cores": cores, "kind": "oracle",
               "sample": f"{nrel} (walker, redshift) realizations of the workload in {secs:.1f} s (FP64, "
                         f"128^3, full radius ladder, delta T_b, Delta^2, chi^2); evals/s = 1/(3 x s per realization)",
               "one_thread_s_per_realization": one,
               "one_thread_evals_per_s": 1.0 / (3.0 * one),
               "one_thread_sample": "fiducial walker (30, 15 Mpc, 4.7) at z = 9, 31 radii, FP64, one host thread "
                                    "(the paper quotes about 3 s per 128^3 realization on one core, Sec. 2.3)",
               "cpu_model": cpu_model(), "host_threads": os.cpu_count()}
    else:
        parity = None

    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "box_mpc": BOX, "z": list(ZS), "walkers_per_gpu": W,
                       "radius_tasks_per_step": tasks_per_step, "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "parallelism": f"walkers sharded over {world} GPU(s)", "traced": not args.no_trace,
                       "schedule": {**schedule,
                                    "picked_by": "library default (--no-autotune)" if args.no_autotune else "eor_autotune"}},
            "e2e": {"value": e2e, "unit": "evals/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "roofline": roof, "kernel_rates": kernel_rates,
            "method": {"name": "basis", "rank": basis_rank, "max_residual": basis_resid,
                       "contraction": {eor21.EOR_CONTRACT_FP16: "tcgen05 FP16 hi/lo, 3 products along K",
                                       eor21.EOR_CONTRACT_TF32: "tcgen05 3xTF32",
                                       eor21.EOR_CONTRACT_FP32: "FP32 FMA"}.get(contract_kind, "none"),
                       "k_slots": k_slots},
            "emulator": emulator, "mcmc": mcmc, "two_population": two_pop,
            "basis_fp32_units": simt, "basis_tf32": tf32, "direct_method": direct,
            "per_radius_fft_bytes_over_step": {
                "value": per_radius_rate, "unit": "GB/s", "frac_of_hbm": per_radius_rate / hbm_peak,
                "peak_kind": hbm_kind,
                "def": "bytes a per-radius FFT design must move (per (walker, z, radius): density half spectrum + "
                       "flag read/write) over the step time; the basis method does not move them, so this is "
                       "not a measured roofline"},
            "cufft": cufft,
            "parity_vs_oracle": parity,
            "plain": {"value": plain, "unit": "evals/s", "walkers_timed": pw,
                      "note": "same kernels, one walker per eor_likelihood call"},
            "batched_over_plain": value / (plain * world),
            "cpu_baseline": cpu, "clocks": clk}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
