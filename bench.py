#!/usr/bin/env python
"""Throughput of the NeRF-CBCT training step on GB300 (ray-samples/s, fwd+bwd+Adam).

A step is one pass of the whole hot path over one batch: ray setup and sampling,
hash gather, Normalized Hash Encoder, MLP, Beer-Lambert ray sum, loss, the
backward (MLP, LN, hash scatter) and Adam over every parameter a step can reach
(a dense level's entries past its (N_l + 1)^3 grid vertices are never reached and
Adam leaves them as they are). The default
workload is the paper-scale FP32 configuration: a 128^3 textured ellipsoid
phantom, 50 views of a 256x256 detector, L=16 F=2 T=2^19 levels 16..2048,
LayerNorm, 4x32 MLP, 2048 rays x 192 samples per step. Inputs are synthetic
(seeded phantom projected by the library, Poisson noise at I0 = 1e5); every
batch uses pixels whose ray meets the volume, in ascending pixel id. The e2e
number copies each step's pixels and measurements from pinned host memory and
its loss back, and reads every loss on the host one step behind.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun), every rank trains its own replica on its own batches
(weak scaling, no collective on the data path); value = all ranks' samples / the
slowest rank's time. ``--impl reference`` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import signal
import subprocess
import sys
import tempfile
import time

if "--cpu-worker" in sys.argv or "reference" in sys.argv:
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"          # the CPU oracle runs on one core

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402

METRIC = "ray-samples/s fwd+bwd; seconds to 30 dB PSNR, mixed vs FP32, same GB300"
UNIT = "ray-samples/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="paper_fp32", choices=sorted(S.WORKLOADS))
    p.add_argument("--mixed", default="paper_bf16", help="mixed-precision workload measured beside ('' = skip)")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-psnr", action="store_true", help="skip the time-to-PSNR runs")
    p.add_argument("--no-l2", action="store_true", help="skip the gather / scatter L2 roofline probes")
    p.add_argument("--large", default="large_bf16", help="large workload measured beside ('' = skip)")
    p.add_argument("--no-mci", action="store_true", help="skip the compact MCI block of the default run")
    p.add_argument("--psnr-steps", type=int, default=3000, help="step cap of the time-to-PSNR runs")
    p.add_argument("--experiment", default="", choices=["", "mci", "fftmask", "variants", "ablation", "variation",
                                                          "views", "precision"])
    p.add_argument("--precision-seeds", type=int, default=5, help="precision: scans (seeds) to train")
    p.add_argument("--views", default="10,25,50,100", help="views: comma-separated view counts")
    p.add_argument("--variation-steps", type=int, default=1500, help="variation: training steps per arm")
    p.add_argument("--mask-step", type=int, default=500, help="fftmask: step at which the mask is chosen")
    p.add_argument("--mask-grid", type=int, default=64, help="fftmask: voxel grid of the feature spectra")
    p.add_argument("--mci-cases", type=int, default=8)
    p.add_argument("--mci-heldout", type=int, default=8)
    p.add_argument("--mci-recon-steps", type=int, default=1500)
    p.add_argument("--mci-pretrain-steps", type=int, default=2000)
    p.add_argument("--cpu-worker", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--seed", type=int, default=0)
    return p.parse_args()


# ------------------------------------------------------------------------------ CPU oracle
ORACLE_RAYS = 16          # rays per bounded oracle batch


def _oracle_worker(args):
    """One CPU worker: oracle forward + loss + backward (Sec. 2.5) on bounded batches of
    ORACLE_RAYS rays for about `seconds`, then one dense Adam update of its 1/n_share
    of the parameters. Returns (rays, seconds of ray work, seconds of Adam)."""
    name, seconds, seed, share, n_share = args
    import oracle
    w = S.WORKLOADS[name]
    g, f = w.geometry, w.field
    tab, du, dv = oracle.view_table(g.n_views, g.angle0_rad, g.span_rad, g.dso_mm, g.dsd_mm,
                                    g.det_du_mm, g.det_dv_mm, g.vol_side_mm)
    og = (tab, du, dv, g.det_nu, g.det_nv)
    rng = np.random.default_rng(seed)
    flat = S.init_params(f, 0).astype(np.float64)
    rays, t_rays = 0, 0.0
    grad = None
    while t_rays < seconds:
        view = int(rng.integers(0, g.n_views))
        _, _, _, _, hit = oracle.ray_setup(tab, du, dv, g.det_nu, g.det_nv, view, np.arange(g.det_nu * g.det_nv))
        pix = rng.choice(np.nonzero(hit)[0], size=ORACLE_RAYS, replace=False).astype(np.int32)
        a_meas = rng.uniform(0, 1, size=ORACLE_RAYS).astype(np.float32)
        t0 = time.perf_counter()
        A, cache = oracle.render_forward(flat, f, og, view, pix, w.n_samples)
        _, dLdA = oracle.loss_and_grad(A, a_meas, f.loss)
        grad = oracle.render_backward(cache, dLdA, f)
        t_rays += time.perf_counter() - t0
        rays += ORACLE_RAYS
    lo, hi = flat.size * share // n_share, flat.size * (share + 1) // n_share
    st = oracle.AdamState(np.zeros(hi - lo), np.zeros(hi - lo), 0)
    t0 = time.perf_counter()
    oracle.adam_step(flat[lo:hi], grad[lo:hi], st, f)
    return rays, t_rays, time.perf_counter() - t0


class OraclePool:
    """The CPU oracle on `workers` host cores (spawned processes, one BLAS thread each).
    A measurement scales the bounded sample to a full step of the workload: the ray
    work's rate summed over the cores gives R rays' time, plus the slowest core's
    share of the dense Adam update."""

    def __init__(self, workers: int):
        import multiprocessing as mp
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        self.workers = workers
        self.pool = mp.get_context("spawn").Pool(workers)

    def measure(self, w: S.Workload, seconds: float, seed: int):
        res = self.pool.map(_oracle_worker, [(w.name, seconds, seed * 1000 + k, k, self.workers)
                                             for k in range(self.workers)])
        ray_rate = sum(r[0] / r[1] for r in res)
        t_adam = max(r[2] for r in res)
        step_s = w.n_rays / ray_rate + t_adam
        rays = sum(r[0] for r in res)
        f = w.field
        desc = (f"{rays} rays x {w.n_samples} samples of oracle forward+loss+backward in batches of "
                f"{ORACLE_RAYS} on the {w.name} field (L={f.n_levels}, T=2^{f.log2_T}) over {self.workers} "
                f"cores, plus a dense Adam over all {S.param_layout(f)['_total'][1]} parameters split "
                f"across the cores, scaled to one {w.n_rays}-ray step ({step_s:.3f} s), float64 numpy")
        return w.n_rays * w.n_samples / step_s, step_s, desc

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(w: S.Workload, seconds: float, seed: int):
    """Runs the oracle on every host core in a fresh interpreter that never touches
    the GPU (CUDA_VISIBLE_DEVICES empty)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", "--workload", w.name,
           "--cpu-seconds", str(seconds), "--seed", str(seed)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=seconds * 20 + 300)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "error": r.stderr[-300:]}
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": out["value"], "unit": UNIT, "cores": out["cores"], "kind": "oracle", "sample": out["sample"]}


# ------------------------------------------------------------------------------ GPU helpers
def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return FALLBACK_PEAKS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def source_sha():
    """sha256 (16 hex digits) of every file of the CUDA sources."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2506_19742_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


TRAIN_KERNEL_UNITS = ("nh_train_f32.cu", "nh_train_bf16.cu", "nh_train_f16.cu")


def kernel_sha():
    """sha256 (16 hex digits) of the training kernel's own sources: the translation
    units that compile k_ray_train and every CUDA-source header they include,
    followed transitively (names and contents, in name order). Kernels in other
    translation units do not change it."""
    csrc = os.path.join(ROOT, "paper_2506_19742_gb300", "csrc")
    seen, todo = set(), list(TRAIN_KERNEL_UNITS)
    while todo:
        f = todo.pop()
        if f in seen:
            continue
        seen.add(f)
        with open(os.path.join(csrc, f)) as fh:
            todo.extend(re.findall(r'#include "([^"/]+)"', fh.read()))
    h = hashlib.sha256()
    for f in sorted(seen):
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if the training
    kernel's sources are still those it profiled."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m1 = re.search(r"kernel_sha:\s*([0-9a-f]+)", txt)
    m2 = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m1 or not m2 or m1.group(1) != kernel_sha():
        return None
    return float(m2.group(1))


def make_scan(nh, torch, w: S.Workload, seed: int, device):
    """Phantom, measured projections (library projector + Poisson noise) and the
    per-view pixels whose rays meet the volume."""
    geom = nh.Geometry.from_config(w.geometry)
    vol, _ = S.phantom(w, seed)
    D = vol.shape[0]
    g = w.geometry
    proj = torch.empty(g.n_views * g.det_nv * g.det_nu, device=device)
    nh.project(geom, torch.from_numpy(vol.astype(np.float32)).to(device), 2, proj)
    ones = torch.ones(D ** 3, device=device)
    hitp = torch.empty_like(proj)
    nh.project(geom, ones, 1, hitp)
    torch.cuda.synchronize()
    clean = proj.view(g.n_views, -1).cpu().numpy()
    hit = hitp.view(g.n_views, -1).cpu().numpy() > 0
    a_meas = S.poisson_measure(clean, w.I0, seed + 1)
    cands = [np.nonzero(hit[v])[0] for v in range(g.n_views)]
    return geom, vol, a_meas, cands


def device_batches(torch, w: S.Workload, cands, a_meas_all, n, seed, dev):
    """n seeded batches (view, pix, a_meas) uploaded to the device, cycled forever."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        view, pix = S.pick_rays(rng, w.geometry.n_views, cands, w.n_rays)
        out.append((view, torch.from_numpy(pix).to(dev),
                    torch.from_numpy(a_meas_all[view][pix].astype(np.float32)).to(dev)))

    def gen():
        while True:
            yield from out
    return gen()


def time_to_psnr(nh, torch, recon, w: S.Workload, seed, dev, targets=(25.0, 30.0, 35.0), max_steps=3000,
                 eval_every=50, params=None, scan=None, ln_mlp=None):
    """Trains workload w from its seeded phantom until the PSNR targets (or max_steps);
    seconds are GPU time of the training steps only. ln_mlp: LN + MLP weights loaded
    before training (Mapping Consistency Initialization)."""
    geom, vol, a_meas_all, cands = scan if scan is not None else make_scan(nh, torch, w, seed, dev)
    vol_gt = torch.from_numpy(vol.astype(np.float32).ravel()).to(dev)
    rec = recon.Reconstruction(w.field, geom, params=params if params is not None else S.init_params(w.field, seed))
    if ln_mlp is not None:
        recon.transfer(ln_mlp, rec.field)
    res = recon.train_to_psnr(rec, device_batches(torch, w, cands, a_meas_all, 500, seed + 5, dev),
                              w.n_samples, vol_gt, targets=targets, eval_every=eval_every, max_steps=max_steps)
    return res, rec


def mci_experiment(nh, torch, recon, w: S.Workload, dev, cases, recon_steps, pretrain_steps, heldout, max_steps,
                   seed):
    """Mapping Consistency Initialization (Sec. 2.1, 2.4): reconstruct `cases`
    pre-training phantoms (seeds 100..) with the plain FP32 method for recon_steps
    steps, fit one LN + MLP to those reconstructions with the voxel loss (Eq. 2) for
    pretrain_steps steps, then train `heldout` held-out phantoms (seeds 200..) from
    that LN + MLP or from random initialisation (the same hash tables) and record
    steps / seconds to 25, 30 and 35 dB; also the 256^3 full-volume query rate."""
    cfg = w.field
    t0 = time.perf_counter()
    vols, rec_psnr = [], []
    for s in range(100, 100 + cases):
        res, rec = time_to_psnr(nh, torch, recon, w, s, dev, targets=(99.0,), max_steps=recon_steps,
                                eval_every=recon_steps)
        vols.append(rec.volume(w.vol_D))
        rec_psnr.append(res["final_psnr"])
        del rec
    shared, pre_curve = recon.pretrain_mci(cfg, vols, steps=pretrain_steps, points_per_step=65536, seed=seed)
    del vols
    rows = []
    for s in range(200, 200 + heldout):
        scan = make_scan(nh, torch, w, s, dev)
        p0 = S.init_params(cfg, s)
        rr, _ = time_to_psnr(nh, torch, recon, w, s, dev, targets=(25.0, 30.0, 35.0), max_steps=max_steps,
                             params=p0, scan=scan)
        rm, rec = time_to_psnr(nh, torch, recon, w, s, dev, targets=(25.0, 30.0, 35.0),
                               max_steps=max_steps, params=p0, scan=scan, ln_mlp=shared)
        rows.append({"seed": s, "random": {k: rr[k] for k in ("steps_to", "seconds_to", "final_psnr")},
                     "mci": {k: rm[k] for k in ("steps_to", "seconds_to", "final_psnr")},
                     "psnr_at": {"random": rr["curve"][:6], "mci": rm["curve"][:6]}})
    # full-volume query throughput at 256^3 (M(x, y, z) of Eq. 2 on every voxel centre)
    out = torch.empty(256 ** 3, device=dev)
    for _ in range(3):
        nh.query_volume(rec.field, 256, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        nh.query_volume(rec.field, 256, out)
    e1.record()
    torch.cuda.synchronize()
    q_ms = e0.elapsed_time(e1) / 10

    def mean_steps(key, t):
        v = [r[key]["steps_to"][t] for r in rows]
        return None if any(x is None for x in v) else float(np.mean(v))

    def mean_psnr_at(key, step):
        v = [next((c[2] for c in r["psnr_at"][key] if c[0] == step), None) for r in rows]
        return None if any(x is None for x in v) else round(float(np.mean(v)), 3)

    return {"experiment": "mci", "workload": w.name, "precision": cfg.precision,
            "pretrain_cases": cases, "recon_steps": recon_steps,
            "pretrain_recon_psnr": rec_psnr, "pretrain_steps": pretrain_steps,
            "pretrain_points_per_step": 65536, "pretrain_loss": pre_curve,
            "heldout": rows, "max_steps": max_steps,
            "mean_steps_to": {t: {"random": mean_steps("random", t), "mci": mean_steps("mci", t)}
                              for t in ("25.0", "30.0", "35.0")},
            "mean_psnr_at_step_50": {"random": mean_psnr_at("random", 50), "mci": mean_psnr_at("mci", 50)},
            "query_256_ms": q_ms, "query_points_per_s": 256 ** 3 / (q_ms / 1e3),
            "wall_seconds": time.perf_counter() - t0}


def run_mci(args):
    """The MCI experiment at the sizes given on the command line (see mci_experiment)."""
    import torch
    from paper_2506_19742_gb300 import build as nhbuild
    from paper_2506_19742_gb300 import nhcbct as nh
    from paper_2506_19742_gb300 import recon
    nhbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    line = mci_experiment(nh, torch, recon, S.WORKLOADS[args.workload], dev, args.mci_cases, args.mci_recon_steps,
                          args.mci_pretrain_steps, args.mci_heldout, args.psnr_steps, args.seed)
    print(json.dumps(line))


class Ranks:
    """Barrier and max over the job's ranks (one process per GPU); with no process
    group both are no-ops."""

    def __init__(self, dist, device):
        self.dist, self.device = dist, device

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def allmax(self, x: float) -> float:
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([x], device=self.device, dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def job_value(samples_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank's samples over the slowest rank's time."""
    return float(samples_per_rank) * world / (ms_max / 1e3)


def event_ms(torch, fn, n=5, warm=1):
    """Mean device time of fn() over n runs (CUDA events on the current stream)."""
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in evs]))


def l2_roofline(nh, torch, geom, fields, batch, N, dev):
    """The gather and scatter stages alone (encode_points / scatter_points at one
    batch's sample positions) against the chip's measured L2 capacity: streaming L2
    read bandwidth, and the rates of uniformly random corner-sized loads and float2
    atomics on tables of the stages' own sizes (the probe kernels). Fractions:
    algorithmic bytes (L 8 F x element size per point) and 32-byte sectors per corner
    over the L2 bandwidth, corner loads / atomics over the random-access probe rate."""
    sink = torch.zeros(1, device=dev)
    buf = torch.zeros(48 << 20 >> 2, device=dev)            # 48 MB: resident in the 126 MB L2
    reps = 10
    t = event_ms(torch, lambda: nh.probe_l2_read(buf, reps, sink))
    l2_gbs = buf.numel() * 4 * reps / (t / 1e3) / 1e9
    del buf
    view, pix, _ = batch
    R = pix.numel()
    xyz = torch.empty(R * N * 3, device=dev)
    delta = torch.empty(R, device=dev)
    nh.sample_rays(geom, view, pix, N, xyz, delta)
    n = R * N
    out = {"l2_read_gbs": round(l2_gbs, 1), "points": n,
           "method": "probe_l2_read of a 48 MB buffer x10 sweeps; probe_random_gather / probe_random_red "
                     "(float2) / probe_random_red16 (bf16x2) on tables of the stage's size; encode_points / "
                     "scatter_points at one batch's samples"}
    for name, fld in fields.items():
        cfg = fld.cfg
        L, F = cfg.n_levels, cfg.n_feat
        tb = 4 if cfg.precision == S.PREC_F32 else 2
        corners = n * L * 8
        h = torch.empty(n * L * F, device=dev)
        t_g = event_ms(torch, lambda: nh.encode_points(fld, xyz, h))
        table = fld.params if cfg.precision == S.PREC_F32 else fld.tables_lp
        tbytes = L * cfg.T * F * tb
        n_ent = 1 << ((L * cfg.T).bit_length() - 1)          # a power of two for the probe
        tab = table.view(torch.uint8)[: n_ent * F * tb]
        done = [0]

        def gprobe():
            done[0] = nh.probe_random_gather(tab, F * tb, corners, sink)
        t_pg = event_ms(torch, gprobe)
        gather = {"ms": round(t_g, 4), "corner_loads": corners,
                  "algorithmic_gbs": round(corners * F * tb / (t_g / 1e3) / 1e9, 1),
                  "sector_gbs": round(corners * 32 / (t_g / 1e3) / 1e9, 1),
                  "probe_random_loads_per_s": done[0] / (t_pg / 1e3)}
        gather["frac_l2_algorithmic"] = round(gather["algorithmic_gbs"] / l2_gbs, 4)
        gather["frac_l2_sectors"] = round(gather["sector_gbs"] / l2_gbs, 4)
        gather["frac_random_probe"] = round((corners / (t_g / 1e3)) / gather["probe_random_loads_per_s"], 4)
        dh = torch.randn(n * L * F, device=dev) * 1e-3
        t_s = event_ms(torch, lambda: nh.scatter_points(fld, xyz, dh))
        gtab = fld.grads[: n_ent * F]

        def rprobe():
            done[0] = nh.probe_random_red(gtab, corners)
        t_pr = event_ms(torch, rprobe)
        n16 = [0]
        gtab16 = fld.grads[: n_ent]                          # n_ent 4-byte entries

        def rprobe16():
            n16[0] = nh.probe_random_red16(gtab16, S.PREC_BF16, corners)
        t_pr16 = event_ms(torch, rprobe16)
        fld.grads.zero_()
        scatter = {"ms": round(t_s, 4), "corner_atomics": corners,
                   "algorithmic_gbs": round(corners * F * 4 / (t_s / 1e3) / 1e9, 1),
                   "probe_random_atomics_per_s": done[0] / (t_pr / 1e3),
                   "probe_random_bf16x2_atomics_per_s": n16[0] / (t_pr16 / 1e3)}
        scatter["frac_l2_algorithmic"] = round(scatter["algorithmic_gbs"] / l2_gbs, 4)
        scatter["frac_random_probe"] = round((corners / (t_s / 1e3)) / scatter["probe_random_atomics_per_s"], 4)
        out[name] = {"table_mb": round(tbytes / 1e6, 1), "gather": gather, "scatter": scatter}
    return out


def train_arm(nh, torch, recon, cm, w, scan, seed, steps, jitter=False, mask_step=0, mask_grid=64, ln_mlp=None,
              ssim_at=()):
    """Trains workload w on a scan from seed's initialisation for `steps` steps; PSNR
    every 50 steps (not timed). jitter: a new stratified-jitter seed every step;
    mask_step > 0: FFT channel mask chosen at the end of the 50-step block holding
    that step (between steps, outside the timed region); ssim_at: steps (multiples
    of 50) at which the 3-D SSIM is also recorded."""
    geom, vol, a_meas_all, cands = scan
    dev = torch.device("cuda", 0)
    vol_gt = torch.from_numpy(vol.astype(np.float32).ravel()).to(dev)
    rec = recon.Reconstruction(w.field, geom, params=S.init_params(w.field, seed))
    if ln_mlp is not None:
        recon.transfer(ln_mlp, rec.field)
    it = device_batches(torch, w, cands, a_meas_all, 500, seed + 5, dev)
    stream = torch.cuda.current_stream()
    curve, reached, train_ms, out = [], {}, 0.0, {}
    for s0 in range(0, steps, 50):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(s0 + 1, min(steps, s0 + 50) + 1):
            view, pix, a = next(it)
            rec.step(view, pix, a, w.n_samples, jitter_seed=(0x9E3779B9 * s + 1) if jitter else 0)
        e1.record(stream)
        e1.synchronize()
        train_ms += e0.elapsed_time(e1)
        if mask_step and s0 < mask_step <= s0 + 50:     # chosen between steps, not timed
            mask, frac = cm.select_channel_mask(rec.field, G=mask_grid)
            out["mask"] = mask.astype(int).tolist()
            out["high_frequency_fraction"] = [round(float(x), 3) for x in frac]
        p = rec.psnr(vol_gt)
        curve.append((min(steps, s0 + 50), round(train_ms / 1e3, 4), round(p, 3)))
        if curve[-1][0] in ssim_at:
            out.setdefault("ssim_at_step", {})[curve[-1][0]] = round(rec.ssim(vol_gt), 4)
        for t in (25.0, 30.0, 35.0):
            if t not in reached and p >= t:
                reached[t] = (curve[-1][0], curve[-1][1])
    out.update({"final_psnr": curve[-1][2], "best_psnr": max(c[2] for c in curve),
                "final_ssim": round(rec.ssim(vol_gt), 4),
                "steps_to": {str(t): reached[t][0] if t in reached else None for t in (25.0, 30.0, 35.0)},
                "seconds_to": {str(t): reached[t][1] if t in reached else None for t in (25.0, 30.0, 35.0)},
                "ms_per_step": round(train_ms / steps, 4), "psnr_at": [c[::2] for c in curve[:: max(1, len(curve) // 12)]],
                "curve": [c[::2] for c in curve]})
    return out


def run_variants(args):
    """The paper's own step shape and sampling (Sec. 3.1: one view, 1024 rays x 320
    samples, the L1 loss of Eq. 3) against the benchmark's (2048 x 192, squared error,
    midpoint samples), with stratified jitter and with FFT channel masking, on the same
    scan and initialisation."""
    import torch
    from paper_2506_19742_gb300 import build as nhbuild
    from paper_2506_19742_gb300 import channel_mask as cm
    from paper_2506_19742_gb300 import nhcbct as nh
    from paper_2506_19742_gb300 import recon
    nhbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = S.WORKLOADS[args.workload]
    faithful = S.WORKLOADS["paper320_fp32" if base.field.precision == S.PREC_F32 else "paper320_bf16"]
    scan = make_scan(nh, torch, base, args.seed, dev)
    arms = [("bench shape: 2048 x 192, MSE, midpoint", base, {}),
            ("paper shape: 1024 x 320, L1, midpoint", faithful, {}),
            ("paper shape, stratified jitter", faithful, {"jitter": True}),
            ("paper shape, jitter + FFT mask at step 500", faithful, {"jitter": True, "mask_step": 500})]
    out = {"experiment": "variants", "steps": args.psnr_steps, "arms": {}}
    for name, w, kw in arms:
        r = train_arm(nh, torch, recon, cm, w, scan, args.seed, args.psnr_steps, **kw)
        r.pop("curve")
        out["arms"][name] = {"workload": w.name, **r}
    print(json.dumps(out))


def run_ablation(args):
    """The paper's ablation grid (Sec. 3.4) on one held-out scan: hash-feature
    normalization (LayerNorm or none, Sec. 2.3) x initialisation (random, or MCI
    pre-trained with the same normalization, Sec. 2.4) x FFT channel mask (none, or
    chosen at step --mask-step). MCI here pre-trains on --mci-cases reconstructions."""
    import dataclasses
    import torch
    from paper_2506_19742_gb300 import build as nhbuild
    from paper_2506_19742_gb300 import channel_mask as cm
    from paper_2506_19742_gb300 import nhcbct as nh
    from paper_2506_19742_gb300 import recon
    nhbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = S.WORKLOADS[args.workload]
    out = {"experiment": "ablation", "workload": base.name, "steps": args.psnr_steps, "mci_cases": args.mci_cases,
           "mci_recon_steps": args.mci_recon_steps, "mci_pretrain_steps": args.mci_pretrain_steps,
           "mask_step": args.mask_step, "arms": {}}
    scan = make_scan(nh, torch, base, 200 + args.seed, dev)
    for norm_name, norm in (("LN", S.NORM_LN), ("none", S.NORM_NONE)):
        w = dataclasses.replace(base, field=dataclasses.replace(base.field, norm=norm))
        vols = []
        for c in range(100, 100 + args.mci_cases):
            _, rec = time_to_psnr(nh, torch, recon, w, c, dev, targets=(99.0,), max_steps=args.mci_recon_steps,
                                  eval_every=args.mci_recon_steps)
            vols.append(rec.volume(w.vol_D))
            del rec
        shared, _ = recon.pretrain_mci(w.field, vols, steps=args.mci_pretrain_steps, points_per_step=65536,
                                       seed=args.seed)
        del vols
        for init in ("random", "MCI"):
            for mask in (0, args.mask_step):
                name = f"norm={norm_name} init={init} mask={'step %d' % mask if mask else 'none'}"
                r = train_arm(nh, torch, recon, cm, w, scan, 200 + args.seed, args.psnr_steps, mask_step=mask,
                              ln_mlp=shared if init == "MCI" else None, ssim_at=(200, 500, 1000))
                out["arms"][name] = {k: r.get(k) for k in ("final_psnr", "best_psnr", "final_ssim", "ssim_at_step",
                                                           "steps_to", "seconds_to")}
                at = dict((c[0], c[1]) for c in r["curve"])
                out["arms"][name]["psnr_at_step"] = {t: at.get(t) for t in (50, 100, 200, 500, 1000)}
    print(json.dumps(out))


def run_views(args):
    """Reconstruction quality against the number of projection views (Fig. 7 of
    the paper, which scores it in SSIM on three cases). For each view count the
    geometry keeps its detector and spreads the views evenly over 360 degrees; on
    each of three held-out phantoms two arms train for --psnr-steps steps: the
    plain hash encoder from random initialisation (the NAF-style baseline), the
    Normalized Hash Encoder from random initialisation, and the whole method (NHE
    with LN + MLP from MCI pre-training on --mci-cases reconstructions at the
    default 50 views). Reports 3-D SSIM at steps 200 / 500 / 1000 and at the end,
    and the final PSNR."""
    import dataclasses
    import torch
    from paper_2506_19742_gb300 import build as nhbuild
    from paper_2506_19742_gb300 import channel_mask as cm
    from paper_2506_19742_gb300 import nhcbct as nh
    from paper_2506_19742_gb300 import recon
    nhbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = S.WORKLOADS[args.workload]
    views = [int(v) for v in args.views.split(",")]
    cases = [200 + args.seed + c for c in range(3)]
    w_ln = dataclasses.replace(base, field=dataclasses.replace(base.field, norm=S.NORM_LN))
    w_plain = dataclasses.replace(base, field=dataclasses.replace(base.field, norm=S.NORM_NONE))
    vols = []
    for c in range(100, 100 + args.mci_cases):
        _, rec = time_to_psnr(nh, torch, recon, w_ln, c, dev, targets=(99.0,), max_steps=args.mci_recon_steps,
                              eval_every=args.mci_recon_steps)
        vols.append(rec.volume(w_ln.vol_D))
        del rec
    shared, _ = recon.pretrain_mci(w_ln.field, vols, steps=args.mci_pretrain_steps, points_per_step=65536,
                                   seed=args.seed)
    del vols
    out = {"experiment": "views", "workload": base.name, "steps": args.psnr_steps, "cases": cases,
           "mci_cases": args.mci_cases, "ssim": "3-D, Gaussian 11^3 window, sigma 1.5, data range 1",
           "views": {}}
    arms = (("hash encoder, random init", w_plain, None), ("NHE, random init", w_ln, None),
            ("NHE + MCI", w_ln, shared))
    checkpoints = tuple(t for t in (200, 500, 1000) if t < args.psnr_steps)
    for V in views:
        row = {name: {"ssim": [], "psnr": [], "ssim_at_step": []} for name, _, _ in arms}
        for seed in cases:
            geo = dataclasses.replace(base.geometry, n_views=V)
            scan = make_scan(nh, torch, dataclasses.replace(base, geometry=geo), seed, dev)
            for name, w, ln_mlp in arms:
                wv = dataclasses.replace(w, geometry=geo)
                r = train_arm(nh, torch, recon, cm, wv, scan, seed, args.psnr_steps, ln_mlp=ln_mlp,
                              ssim_at=checkpoints)
                row[name]["ssim"].append(r["final_ssim"])
                row[name]["psnr"].append(r["final_psnr"])
                row[name]["ssim_at_step"].append(r.get("ssim_at_step", {}))
            del scan
        for name in row:
            row[name]["mean_ssim"] = round(float(np.mean(row[name]["ssim"])), 4)
            row[name]["mean_psnr"] = round(float(np.mean(row[name]["psnr"])), 3)
            row[name]["mean_ssim_at_step"] = {
                t: round(float(np.mean([d[t] for d in row[name]["ssim_at_step"]])), 4) for t in checkpoints
                if all(t in d for d in row[name]["ssim_at_step"])}
        out["views"][V] = row
    print(json.dumps(out))


def run_variation(args):
    """The MLP-variation probe behind the paper's motivation for the Normalized Hash
    Encoder (Sec. 1 and 2.3, Fig. 3): hash features come from a different subset of
    table entries every step while every MLP weight moves, so the network's mapping
    drifts. Every 100 steps the hash tables and mu at P fixed points are recorded;
    100 steps later the recorded tables are evaluated with the current LN + MLP
    (field_export / field_import of NH_PART_HASH and NH_PART_LN | NH_PART_MLP), and
    the mean |mu_later(features_then) - mu_then| is the variation. Run with and
    without the normalization on the same scan and initialisation."""
    import dataclasses
    import torch
    from paper_2506_19742_gb300 import build as nhbuild
    from paper_2506_19742_gb300 import nhcbct as nh
    from paper_2506_19742_gb300 import recon
    nhbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = S.WORKLOADS[args.workload]
    geom, vol, a_meas_all, cands = make_scan(nh, torch, base, args.seed, dev)
    vol_gt = torch.from_numpy(vol.astype(np.float32).ravel()).to(dev)
    xyz = torch.from_numpy(np.random.default_rng(args.seed + 9).random((65536, 3)).astype(np.float32)).to(dev)
    out = {"experiment": "variation", "workload": base.name, "points": 65536, "interval": 100, "arms": {}}
    for norm_name, norm in (("LN", S.NORM_LN), ("none", S.NORM_NONE)):
        cfg = dataclasses.replace(base.field, norm=norm)
        w = dataclasses.replace(base, field=cfg)
        rec = recon.Reconstruction(cfg, geom, params=S.init_params(cfg, args.seed))
        probe = nh.Field(cfg, params=S.init_params(cfg, args.seed))
        it = device_batches(torch, w, cands, a_meas_all, 500, args.seed + 5, dev)
        mu_then = torch.empty(65536, device=dev)
        mu_now = torch.empty(65536, device=dev)
        tables_then, series = None, []
        for s in range(1, args.variation_steps + 1):
            view, pix, a = next(it)
            rec.step(view, pix, a, w.n_samples)
            if s % 100 == 0:
                if tables_then is not None:
                    probe.import_(nh.PART_HASH, tables_then)
                    probe.import_(nh.PART_LN | nh.PART_MLP, rec.field.export(nh.PART_LN | nh.PART_MLP))
                    nh.query_points(probe, xyz, mu_now)
                    series.append((s, round(float((mu_now - mu_then).abs().mean()), 6),
                                   round(rec.psnr(vol_gt), 3)))
                tables_then = rec.field.export(nh.PART_HASH)
                nh.query_points(rec.field, xyz, mu_then)
        out["arms"][norm_name] = {"series": series,
                                  "mean_variation": round(float(np.mean([v for _, v, _ in series])), 6)}
    print(json.dumps(out))


def run_precision(args):
    """The mixed-precision target on several scans: for each of --precision-seeds
    seeds, the paper-scale scan trained from the same initialisation and batches in
    FP32 (twice), in BF16 and in FP16 (with its dynamic loss scale) for --psnr-steps
    steps; final PSNR and 3-D SSIM, steps and seconds to 30 dB, and the per-seed and
    mean final-PSNR differences to the first FP32 run. Hash-gradient atomics add in
    no fixed order, so one run per seed is one draw; the second FP32 run measures
    that run-to-run spread against which the precisions are compared."""
    import dataclasses
    import torch
    from paper_2506_19742_gb300 import build as nhbuild
    from paper_2506_19742_gb300 import channel_mask as cm
    from paper_2506_19742_gb300 import nhcbct as nh
    from paper_2506_19742_gb300 import recon
    nhbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = S.WORKLOADS[args.workload]
    arms = {"fp32": base,
            "fp32_repeat": base,
            "bf16": dataclasses.replace(base, field=dataclasses.replace(base.field, precision=S.PREC_BF16)),
            "f16": dataclasses.replace(base, field=dataclasses.replace(base.field, precision=S.PREC_F16,
                                                                        loss_scale_init=1024.0,
                                                                        growth_interval=200))}
    out = {"experiment": "precision", "workload": base.name, "steps": args.psnr_steps, "seeds": []}
    for k in range(args.precision_seeds):
        seed = 300 + k
        scan = make_scan(nh, torch, base, seed, dev)
        row = {"seed": seed}
        for name, w in arms.items():
            r = train_arm(nh, torch, recon, cm, w, scan, seed, args.psnr_steps)
            row[name] = {kk: r[kk] for kk in ("final_psnr", "best_psnr", "final_ssim", "steps_to", "seconds_to",
                                              "ms_per_step")}
        for name in ("fp32_repeat", "bf16", "f16"):
            row[name]["final_psnr_delta_db"] = round(row[name]["final_psnr"] - row["fp32"]["final_psnr"], 3)
        out["seeds"].append(row)
        del scan
    for name in ("fp32_repeat", "bf16", "f16"):
        d = np.array([r[name]["final_psnr_delta_db"] for r in out["seeds"]])
        out[name + "_final_psnr_delta_db"] = {"mean": round(float(d.mean()), 3), "std": round(float(d.std()), 3),
                                               "min": round(float(d.min()), 3), "max": round(float(d.max()), 3),
                                               "within_0.1": int(np.sum(np.abs(d) <= 0.1))}
    print(json.dumps(out))


def run_fftmask(args):
    """FFT channel masking (Sec. 2.3) on the benchmark scan: the same initialisation
    and batches trained with no mask, and with the mask chosen from the hash
    features' spectra after --mask-step steps (channel_mask.select_channel_mask),
    to --psnr-steps steps; PSNR every 50 steps (evaluation not timed)."""
    import torch
    from paper_2506_19742_gb300 import build as nhbuild
    from paper_2506_19742_gb300 import channel_mask as cm
    from paper_2506_19742_gb300 import nhcbct as nh
    from paper_2506_19742_gb300 import recon
    nhbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = S.WORKLOADS[args.workload]
    geom, vol, a_meas_all, cands = make_scan(nh, torch, w, args.seed, dev)
    vol_gt = torch.from_numpy(vol.astype(np.float32).ravel()).to(dev)
    out = {"experiment": "fftmask", "workload": w.name, "mask_step": args.mask_step, "steps": args.psnr_steps,
           "grid": args.mask_grid, "cutoff": 0.25, "threshold": 0.85}
    for arm in ("none", "fft"):
        rec = recon.Reconstruction(w.field, geom, params=S.init_params(w.field, args.seed))
        it = device_batches(torch, w, cands, a_meas_all, 500, args.seed + 5, dev)
        curve, reached = [], {}
        for s in range(1, args.psnr_steps + 1):
            view, pix, a = next(it)
            rec.step(view, pix, a, w.n_samples)
            if arm == "fft" and s == args.mask_step:
                mask, frac = cm.select_channel_mask(rec.field, G=args.mask_grid)
                out["mask"] = mask.astype(int).tolist()
                out["high_frequency_fraction"] = [round(float(x), 3) for x in frac]
            if s % 50 == 0:
                p = rec.psnr(vol_gt)
                curve.append((s, round(p, 3)))
                for t in (25.0, 30.0, 35.0):
                    if t not in reached and p >= t:
                        reached[t] = s
        out[arm] = {"final_psnr": curve[-1][1], "best_psnr": max(c[1] for c in curve),
                    "steps_to": {str(t): reached.get(t) for t in (25.0, 30.0, 35.0)},
                    "psnr_at": curve[:: max(1, len(curve) // 12)]}
    print(json.dumps(out))


def optimizer_params(f: S.FieldConfig) -> int:
    """Parameters the optimizer visits: every entry of a hashed level, the first
    (N_l + 1)^3 entries of a dense level (rounded up to whole groups of four floats;
    no corner index reaches the rest) and the LN / MLP block."""
    T, F, L = 2 ** f.log2_T, f.n_feat, f.n_levels
    step = (math.log(f.max_res) - math.log(f.base_res)) / (L - 1) if L > 1 else 0.0
    n = S.param_layout(f)["_total"][1] - L * T * F
    for l in range(L):
        res = int(math.floor(f.base_res * math.exp(l * step) + 1e-9)) if L > 1 else f.base_res
        live = (res + 1) ** 3 if (res + 1) ** 3 <= T else T
        n += min(T * F, -(-live * F // 4) * 4)
    return n


def measure_large(nh, torch, wl: S.Workload, seed: int, K: int, W: int, dev, peaks, peak_kind):
    """The large configuration (256^3 shell phantom, 100 views of 512^2, T = 2^21 BF16
    tables, 8192 rays x 256 samples): its own scan and batches, K timed train_steps
    after W warm-up steps, then the fused kernel and Adam timed alone. Here the
    tables (128 MiB BF16 + 256 MiB FP32 master), gradient tables and Adam state
    (1 GiB together) exceed the L2, so HBM is the bound for both kernels."""
    geom, _, a_meas_all, cands = make_scan(nh, torch, wl, seed, dev)
    R, N = wl.n_rays, wl.n_samples
    rng = np.random.default_rng(seed + 3)
    batches = []
    for _ in range(W + K):
        view, pix = S.pick_rays(rng, wl.geometry.n_views, cands, R)
        batches.append((view, torch.from_numpy(pix).to(dev),
                        torch.from_numpy(a_meas_all[view][pix].astype(np.float32)).to(dev)))
    field = nh.Field(wl.field, params=S.init_params(wl.field, seed))
    ws = nh.workspace(nh.step_workspace_bytes(field, R, N), dev)
    loss = torch.zeros(1, device=dev)
    stream = torch.cuda.current_stream()
    for v, p, a in batches[:W]:
        nh.train_step(field, geom, v, p, a, N, loss, ws)
    torch.cuda.synchronize()
    phys = torch.cuda.current_device()
    with ClockSampler(phys) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for v, p, a in batches[W:]:
            nh.train_step(field, geom, v, p, a, N, loss, ws)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    nk = min(K, 20)

    def timed(fn):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nk)]
        for i in range(nk):
            evs[i][0].record(stream)
            fn(i)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([x.elapsed_time(y) for x, y in evs]))

    t_acc = timed(lambda i: nh.accumulate_step(field, geom, batches[W + i][0], batches[W + i][1],
                                               batches[W + i][2], N, loss, ws))
    launch = nh.launch_info()
    t_adam = timed(lambda i: nh.optimizer_step(field))
    f = wl.field
    L, F = f.n_levels, f.n_feat
    bytes_per_sample = L * 8 * F * 2 + L * 8 * F * 4      # one BF16 gather + one FP32 scatter payload
    n_params = S.param_layout(f)["_total"][1]
    n_visit = optimizer_params(f)
    adam_bytes = 34 * n_visit                              # p, m, v, g read; p, m, v, g written; 16-bit copy
    peak = peaks["hbm_gbs"]
    ach = bytes_per_sample * R * N / (t_acc / 1e3) / 1e9
    ach_adam = adam_bytes / (t_adam / 1e3) / 1e9
    return {"workload": wl.name, "value": R * N * K / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / K,
            "steps": K, "warmup": W, "dtype": "bf16", "clocks": clk.summary(),
            "config": {"rays_per_step": R, "samples_per_ray": N, "levels": L, "features": F, "log2_T": f.log2_T,
                       "resolutions": [f.base_res, f.max_res], "mlp": f"{f.hidden_layers}x{f.width}",
                       "volume": wl.vol_D, "views": wl.geometry.n_views,
                       "detector": [wl.geometry.det_nu, wl.geometry.det_nv]},
            "launch_ms": {"forward+loss+backward": round(t_acc, 4), "adam": round(t_adam, 4)},
            "launch": launch,
            "roofline": {"kernel": "k_ray_train", "bound": "hbm", "achieved": round(ach, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(ach / peak, 4), "peak_source": f"{peak_kind} hbm_gbs",
                         "bytes_per_sample": bytes_per_sample, "units_per_launch": R * N,
                         "traffic": profiled_traffic("ray_train", wl.name)},
            "adam_roofline": {"kernel": "k_adam", "bound": "hbm", "achieved": round(ach_adam, 1), "peak": peak,
                              "unit": "GB/s", "frac": round(ach_adam / peak, 4), "bytes_per_param": 34,
                              "params": n_visit, "params_total": n_params}}


def run_ours(args, rank: int, world: int, local_rank: int):
    import torch
    from paper_2506_19742_gb300 import build as nhbuild
    from paper_2506_19742_gb300 import nhcbct as nh

    nhbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    ranks = Ranks(dist, dev)
    barrier, allmax = ranks.barrier, ranks.allmax

    w = S.WORKLOADS[args.workload]
    seed = args.seed + 1000 * rank
    geom, vol, a_meas_all, cands = make_scan(nh, torch, w, seed, dev)
    R, N = w.n_rays, w.n_samples
    K, W = args.steps, args.warmup
    rng = np.random.default_rng(seed + 2)

    def make_batches(n):
        out = []
        for _ in range(n):
            view, pix = S.pick_rays(rng, w.geometry.n_views, cands, R)
            out.append((view, pix, a_meas_all[view][pix].astype(np.float32)))
        return out

    host_batches = make_batches(W + K)
    dev_batches = [(v, torch.from_numpy(p).to(dev), torch.from_numpy(a).to(dev)) for v, p, a in host_batches]

    def measure(wl: S.Workload):
        field = nh.Field(wl.field, params=S.init_params(wl.field, seed))
        ws = nh.workspace(nh.step_workspace_bytes(field, R, N), dev)
        loss = torch.zeros(1, device=dev)
        stream = torch.cuda.current_stream()
        for v, p, a in dev_batches[:W]:
            nh.train_step(field, geom, v, p, a, N, loss, ws)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for v, p, a in dev_batches[W:]:
            nh.train_step(field, geom, v, p, a, N, loss, ws)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return field, ws, e0.elapsed_time(e1)

    phys = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[local_rank]
               if os.environ.get("CUDA_VISIBLE_DEVICES") else local_rank)
    with ClockSampler(phys) as clk:
        field, ws, ms = measure(w)
    clocks = clk.summary()
    ms = allmax(ms)
    samples_all = float(R * N * K * world)
    value = job_value(R * N * K, world, ms)

    # per-kernel durations (CUDA events on the launching stream) for the roofline
    stream = torch.cuda.current_stream()
    nk = min(K, 20)

    def timed(fn):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nk)]
        for i in range(nk):
            evs[i][0].record(stream)
            fn(i)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in evs]))



    fused = (N + 31) // 32 <= 16          # the library fuses rays of up to 16 chunks
    loss_k = torch.zeros(1, device=dev)

    def kernel_ms(fld, wsp):
        """Device time of the step's parts: forward + loss + backward (one fused kernel
        when rays fit a CTA, else three), then Adam; each timed alone with CUDA events."""
        t_acc = timed(lambda i: nh.accumulate_step(fld, geom, dev_batches[W + i][0], dev_batches[W + i][1],
                                                   dev_batches[W + i][2], N, loss_k, wsp))
        info = nh.launch_info()
        t_a = timed(lambda i: nh.optimizer_step(fld))
        return t_acc, t_a, info

    t_acc, t_adam, launch = kernel_ms(field, ws)
    peaks, peak_kind = read_peaks()
    tb = 4 if w.field.precision == S.PREC_F32 else 2
    L, F = w.field.n_levels, w.field.n_feat
    # algorithmic bytes per ray-sample: one trilinear gather (8 corners x F features per
    # level) and one scatter of the same payload as float32 into the gradient tables;
    # the split path re-gathers in its backward
    bytes_per_sample = L * 8 * F * tb * (1 if fused else 2) + L * 8 * F * 4
    achieved = bytes_per_sample * R * N / (t_acc / 1e3) / 1e9
    peak = peaks["hbm_gbs"]
    kname = "ray_train" if fused else "ray_backward"
    roofline = {"kernel": "k_" + kname, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": profiled_traffic(kname, w.name),
                "peak_source": f"{peak_kind} hbm_gbs",
                "bytes_per_sample": bytes_per_sample, "units_per_launch": R * N,
                "launch_ms": {"forward+loss+backward": round(t_acc, 4), "adam": round(t_adam, 4)},
                "launch": launch}

    # end to end through the host-buffer entry point (pinned host in, loss out). Every
    # step copies its pixels and measurements from pinned host memory and its loss
    # back to the host, and the host reads every step's loss, one step behind: step
    # k's loss is read once step k + 1 is enqueued, as a training loop that logs its
    # loss does, so the GPU does not wait for the host between steps.
    pins = [(v, torch.from_numpy(p).pin_memory(), torch.from_numpy(a).pin_memory()) for v, p, a in host_batches]
    loss_h = [torch.zeros(1).pin_memory() for _ in range(2)]
    for v, p, a in pins[:W]:
        nh.train_step_host(field, geom, v, p, a, N, loss_h[0], ws)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    losses, done = [], []
    for k, (v, p, a) in enumerate(pins[W:]):
        nh.train_step_host(field, geom, v, p, a, N, loss_h[k % 2], ws)
        done.append(torch.cuda.Event())
        done[k].record(stream)
        if k >= 1:
            done[k - 1].synchronize()
            losses.append(float(loss_h[(k - 1) % 2][0]))
    done[-1].synchronize()
    losses.append(float(loss_h[(len(done) - 1) % 2][0]))
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = allmax(max(e0.elapsed_time(e1), (time.perf_counter() - t0) * 1e3))
    e2e = {"value": samples_all / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": R * 4 + R * 4,
           "d2h_bytes_per_step": 4}

    mixed = None
    if args.mixed and args.mixed != args.workload:
        wm = S.WORKLOADS[args.mixed]
        if wm.n_rays == R and wm.n_samples == N and wm.geometry == w.geometry:
            field_m, ws_m, ms_m = measure(wm)
            ms_m = allmax(ms_m)
            tacc, ta, _ = kernel_ms(field_m, ws_m)
            mixed = {"workload": wm.name, "value": samples_all / (ms_m / 1e3), "unit": UNIT,
                     "ms_per_step": ms_m / K, "speedup_vs_fp32": (samples_all / (ms_m / 1e3)) / value,
                     "launch_ms": {"forward+loss+backward": round(tacc, 4), "adam": round(ta, 4)}}

    l2 = None
    if rank == 0 and not args.no_l2:
        flds = {w.name: field}
        if mixed is not None:
            flds[mixed["workload"]] = field_m
        l2 = l2_roofline(nh, torch, geom, flds, dev_batches[W], N, dev)
        # the fused kernel against the time its gather and scatter take on their own
        # (each at the L2's random-access limit): the share of the kernel that the
        # table traffic alone would need
        st = l2[w.name]
        floor = st["gather"]["ms"] + st["scatter"]["ms"]
        roofline["random_access_floor_ms"] = round(floor, 4)
        roofline["frac_random_access_floor"] = round(floor / t_acc, 4)
        if mixed is not None:
            stm = l2[mixed["workload"]]
            fm = stm["gather"]["ms"] + stm["scatter"]["ms"]
            mixed["random_access_floor_ms"] = round(fm, 4)
            mixed["frac_random_access_floor"] = round(fm / mixed["launch_ms"]["forward+loss+backward"], 4)

    # time to PSNR: FP32 and the mixed-precision workload on the same scan
    psnr = None
    if not args.no_psnr and rank == 0:
        from paper_2506_19742_gb300 import recon
        scan = (geom, vol, a_meas_all, cands)
        vol_gt = torch.from_numpy(vol.astype(np.float32).ravel()).to(dev)
        r32, rec = time_to_psnr(nh, torch, recon, w, seed, dev, scan=scan, max_steps=args.psnr_steps)
        psnr = {"fp32": {k: r32[k] for k in ("steps_to", "seconds_to", "final_psnr", "best_psnr", "steps")}}
        psnr["fp32"]["final_ssim"] = round(rec.ssim(vol_gt), 4)
        del rec
        if args.mixed and S.WORKLOADS[args.mixed].geometry == w.geometry:
            rmx, rec = time_to_psnr(nh, torch, recon, S.WORKLOADS[args.mixed], seed, dev, scan=scan,
                                    max_steps=args.psnr_steps)
            psnr["mixed"] = {k: rmx[k] for k in ("steps_to", "seconds_to", "final_psnr", "best_psnr", "steps")}
            psnr["mixed"]["final_ssim"] = round(rec.ssim(vol_gt), 4)
            del rec
            s32, smx = r32["seconds_to"].get("30.0"), rmx["seconds_to"].get("30.0")
            psnr["seconds_to_30dB_fp32_over_mixed"] = (s32 / smx) if (s32 and smx) else None
            psnr["final_psnr_delta_db"] = round(rmx["final_psnr"] - r32["final_psnr"], 3)

    large = None
    if rank == 0 and args.large and args.large != args.workload:
        del field, ws
        if mixed is not None:
            del field_m, ws_m
        torch.cuda.empty_cache()
        large = measure_large(nh, torch, S.WORKLOADS[args.large], seed, K, W, dev, peaks, peak_kind)

    mci = None
    if rank == 0 and not args.no_mci:
        from paper_2506_19742_gb300 import recon
        # compact form of the MCI experiment (bench.py --experiment mci runs it at
        # 8 + 8 cases): 4 pre-training reconstructions, 2 held-out phantoms
        m = mci_experiment(nh, torch, recon, w, dev, cases=4, recon_steps=1000, pretrain_steps=1500, heldout=2,
                           max_steps=1500, seed=args.seed)
        mci = {k: m[k] for k in ("workload", "pretrain_cases", "recon_steps", "pretrain_recon_psnr",
                                 "pretrain_steps", "max_steps", "mean_steps_to", "mean_psnr_at_step_50",
                                 "query_points_per_s", "wall_seconds")}
        mci["heldout"] = [{"seed": r["seed"], "random": r["random"], "mci": r["mci"]} for r in m["heldout"]]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_seconds, args.seed)

    if dist is not None:
        barrier()                      # rank 0's extra measurements are done before teardown
        dist.destroy_process_group()
    if rank != 0:
        return
    f = w.field
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if f.precision == S.PREC_F32 else ("bf16" if f.precision == S.PREC_BF16 else "f16"),
        "data": "synthetic",
        "config": {"workload": w.name, "rays_per_step": R, "samples_per_ray": N,
                   "levels": f.n_levels, "features": f.n_feat, "log2_T": f.log2_T,
                   "resolutions": [f.base_res, f.max_res], "norm": f.norm, "mlp": f"{f.hidden_layers}x{f.width}",
                   "volume": w.vol_D, "views": w.geometry.n_views,
                   "detector": [w.geometry.det_nu, w.geometry.det_nv],
                   "l2": "working set larger than L2: each step's Adam streams "
                         f"{4 * 4 * optimizer_params(f) / 1e6:.0f} MB of parameter state",
                   "optimizer": f"Adam (torch semantics), dense over the {optimizer_params(f)} parameters a step "
                                f"can reach of {S.param_layout(f)['_total'][1]}; the others (dense levels' entries "
                                "past their (N+1)^3 vertices) never get a gradient, and their update is exactly zero",
                   "parallelism": f"replicas x{world}"},
        "clocks": clocks, "e2e": e2e, "gpu_launches": (3 if fused else 5) * K, "roofline": roofline, "cpu_baseline": cpu,
        "mixed": mixed, "l2_roofline": l2, "psnr": psnr, "large": large, "mci": mci,
        "final_loss": losses[-1] if losses else None,
    }
    print(json.dumps(line))


def run_reference(args, rank: int, world: int):
    """The CPU oracle as the reference arm: each step is one bounded sample of the
    workload on every host core, scaled to a full step (OraclePool)."""
    if rank != 0:
        return
    w = S.WORKLOADS[args.workload]
    pool = OraclePool(cpu_cores())
    per_step = 2.0
    for k in range(args.warmup):
        pool.measure(w, 0.2, args.seed + 100 + k)
    total_s, desc = 0.0, ""
    for k in range(args.steps):
        _, step_s, desc = pool.measure(w, per_step, args.seed + k)
        total_s += step_s
    pool.close()
    value = w.n_rays * w.n_samples * args.steps / total_s
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "rays_per_step": w.n_rays, "samples_per_ray": w.n_samples},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.workers, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse_args()
    if args.cpu_worker:
        pool = OraclePool(cpu_cores())
        value, _, desc = pool.measure(S.WORKLOADS[args.workload], args.cpu_seconds, args.seed)
        pool.close()
        print(json.dumps({"value": value, "sample": desc, "cores": pool.workers}))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.experiment == "mci":
        if rank == 0:
            run_mci(args)
    elif args.experiment == "fftmask":
        if rank == 0:
            run_fftmask(args)
    elif args.experiment == "variants":
        if rank == 0:
            run_variants(args)
    elif args.experiment == "ablation":
        if rank == 0:
            run_ablation(args)
    elif args.experiment == "variation":
        if rank == 0:
            run_variation(args)
    elif args.experiment == "views":
        if rank == 0:
            run_views(args)
    elif args.experiment == "precision":
        if rank == 0:
            run_precision(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
