"""Benchmark: Mpaths/s of the proxy-tracing BDPT render with the learned
light-subspace proposal against the plain subspace table, at equal time.

Default workload (the configuration the metric is quoted on): the glossy
procedural scene at 1024x1024 -- about 1.05M triangles in 2,000 seeded
instances, GGX conductors of roughness log-uniform in [0.005, 0.1] on half
of them, 3 quad lights, max depth 10, M = 10,000 light sub-paths and about
400 incomplete light sub-paths estimated per iteration (5 repeats) -- with
K_S = 64 light subspaces and the proposal network trained on the
renderer's own 2^22 connection samples before timing.

One step = one full render of the workload's iterations (light pass, pool
build, reciprocal estimation, the proposal network, eye pass with
connections, proxy retrace and MIS, film accumulation) on inputs resident on
the device; the tables are learned and the network trained once before
timing (the paper's preprocessing). Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload glossy|glossy512|projector|projector_r001|small|glossy_small|batch|subspace|rr]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm of this build: there is no runnable upstream).
"""

from __future__ import annotations

import argparse
import hashlib
import math
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpaths/s and equal-time MAPE vs CPU oracle; learned vs plain proposal, 1 GB300"
ENTRY_TARGET = 400          # incomplete light sub-paths estimated per iteration (paper: up to 400)
BOOTH = 0.0                 # --booth: Booth's Russian roulette scale in the estimator (0: the paper's RRS)
TRACE = 1                   # --trace: 1 = estimator traces and occlusion answers on persistent warps, 0 = one ray per thread
TRIAL_CAP = 1 << 20         # node cap per reciprocal estimate


def _glossy(W, n_inst=2000):
    def make():
        from paper_2503_23412_gb300 import scenes
        return scenes.glossy(W, W, n_inst=n_inst)
    return make


def _projector(W, rough=0.1):
    def make():
        from paper_2503_23412_gb300 import scenes
        return scenes.projector(W, W, lens_rough=rough)
    return make


GLOSSY_DESC = ("glossy %dx%d, %d spp per step, max depth 10: ~1.05M triangles in 2,000 seeded instances (icospheres "
               "of 80/1280 triangles and boxes) in a 20^3 volume, GGX conductors with roughness log-uniform in "
               "[0.005, 0.1] on half of them, Lambert elsewhere, 3 quad lights of radiance log-uniform in [1, 50]; "
               "M=10000 light sub-paths/iteration, 5 reciprocal repeats, 300 eye / %d light / 100 specular / 10 "
               "control subspaces")
PROJ_DESC = ("projector %dx%d, %d spp, max depth 8: textured 0.1x0.1 emitter in an absorbing box, biconvex GGX "
             "dielectric lens (IOR 1.5, roughness %g, ~19.5k triangles), diffuse room; M=%d light sub-paths/iteration, "
             "5 reciprocal repeats, 300 eye / 300 light / 100 specular / 10 control subspaces")
WORKLOADS = {
    # the learned-proposal comparison at 1024^2 on the ~1M-triangle glossy scene, K = 64
    # the estimator's B: the learned cell bound (pilot off) from 1,024 draws per entry over 8 learning
    # iterations; per-entry pilots miss the brighter of several lights and make the chains split without end
    "glossy": dict(make=_glossy(1024), W=1024, spp=8, depth=10, M=10000, KS=64, proposal="learned",
                   train_samples=1 << 22, ref_mult=64, pilot_max=-1, learn_nb=1024, learn_iters=8,
                   oracle_px=1024, oracle_est=48, desc=GLOSSY_DESC % (1024, 1024, 8, 64)),
    # the same generator at 512^2, 128 spp, with the table proposal and 300 light subspaces
    "glossy512": dict(make=_glossy(512), W=512, spp=128, depth=10, M=10000, KS=300, proposal="table",
                      train_samples=1 << 22, ref_mult=0, pilot_max=-1, learn_nb=1024, learn_iters=8,
                      oracle_px=1024, oracle_est=48, desc=GLOSSY_DESC % (512, 512, 128, 300)),
    "projector": dict(make=_projector(256), W=256, spp=64, depth=8, M=10000, KS=300, proposal="table",
                      train_samples=3 << 20, ref_mult=16, desc=PROJ_DESC % (256, 256, 64, 0.1, 10000)),
    # the projector with the lens at the paper's specular roughness (0.01, alpha = 1e-4)
    "projector_r001": dict(make=_projector(256, 0.01), W=256, spp=64, depth=8, M=10000, KS=300, proposal="table",
                           train_samples=3 << 20, ref_mult=16, desc=PROJ_DESC % (256, 256, 64, 0.01, 10000)),
    # small cases for profiler captures (same kernels; the glossy one keeps the 1M-triangle BVH)
    "small": dict(make=_projector(64), W=64, spp=4, depth=8, M=2000, KS=300, proposal="table",
                  train_samples=1 << 20, ref_mult=0, desc=PROJ_DESC % (64, 64, 4, 0.1, 2000)),
    "glossy_small": dict(make=_glossy(256), W=256, spp=2, depth=10, M=10000, KS=64, proposal="learned",
                         train_samples=1 << 20, ref_mult=0, pilot_max=-1, learn_nb=1024, learn_iters=8,
                         oracle_px=256, oracle_est=16, desc=GLOSSY_DESC % (256, 256, 2, 64)),
}
WL = WORKLOADS["glossy"]
W = H = WL["W"]
SPP, DEPTH, M = WL["spp"], WL["depth"], WL["M"]
WORKLOAD = WL["desc"]
FALLBACK_HBM = 6800.0


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_iter_base(rank):
    """First iteration number of a rank. Ranks are replicas: each renders its
    own iterations (disjoint ranges), with no collective on the data path."""
    return rank * (1 << 24)


def job_ms(local_ms, dist=None, device="cpu"):
    """Whole-job time of the timed region: the slowest rank's (MAX over ranks)."""
    if dist is None:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(paths_per_rank, ws, total_ms):
    """Whole-job throughput in Mpaths/s: the paths of all ranks over the slowest rank's time."""
    return paths_per_rank * ws / (total_ms * 1e-3) / 1e6


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def src_sha(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


EYE_SRC = ["paper_2503_23412_gb300/csrc/pb_eye.cu", "paper_2503_23412_gb300/csrc/pb_device.cuh",
           "paper_2503_23412_gb300/csrc/pb_kernels.h"]
REC_SRC = ["paper_2503_23412_gb300/csrc/pb_light.cu", "paper_2503_23412_gb300/csrc/pb_recip.cu",
           "paper_2503_23412_gb300/csrc/pb_recip_long.cuh", "paper_2503_23412_gb300/csrc/pb_wavefront.cu",
           "paper_2503_23412_gb300/csrc/pb_entry.cuh", "paper_2503_23412_gb300/csrc/pb_estimator.cuh",
           "paper_2503_23412_gb300/csrc/pb_device.cuh", "paper_2503_23412_gb300/csrc/pb_kernels.h"]


def traffic_for(kernel, sha):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of that kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d or d.get("src_sha") != sha:
        return None
    return d.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
def oracle_tables(scene, tables=None):
    """Tables for the oracle's timing runs: the given ones (the device's, read
    back, so that the oracle estimates the same incomplete sub-paths), else
    learned by the oracle itself from random centroids in one small learning
    pass. That pass caps each estimate at 8,192 nodes, so the learned cost
    bound leaves every cell with a longer chain to the other strategies,
    which can only shorten the oracle's work."""
    import oracle as O
    from paper_2503_23412_gb300 import scenes
    o = O.Oracle(scene)
    if tables is None:
        # learning renders every pixel once: do it at most 128 x 128 through
        # the same camera, then spread the tile grid to the full image
        lw = min(W, 128)
        small = dict(scene, cam=np.array(scene["cam"], np.float32))
        small["cam"][10] = small["cam"][11] = lw
        ol = O.Oracle(small) if lw < W else o
        tab = scenes.random_tables(small, KT=300, KS=WL["KS"], KSp=100, KC=10)
        tables = ol.learn(O.params(M=1000, M_p=1000, max_depth=DEPTH, trial_cap=8192), tab, 1 << 21, 1,
                          n_bsamples=16)
        if lw < W:
            tile = int(tables["tile"])
            gw = (W + tile - 1) // tile
            pos = np.minimum((np.arange(gw) * tile * lw) // (W * tile), tables["pi_grid"].shape[0] - 1)
            tables["pi_grid"] = np.ascontiguousarray(tables["pi_grid"][np.ix_(pos, pos)])
    return o, o.tables(tables)


def oracle_iteration_rate(o, td, M_p, it, npx, keep=False, threads=1, n_est=None):
    """CPU oracle, one iteration of the workload measured in two parts: the
    light side (light pass, pool, reciprocal estimates) and the eye paths of
    the first `npx` pixels. With n_est, only that many entries (evenly
    spread over the iteration's pool) are estimated and their time is scaled
    to the whole pool; the eye paths then use those estimates and the mean of
    them elsewhere (their time does not depend on the values). With
    threads > 1 the estimates (in small entry ranges) and the eye paths
    (split by pixel) run on that many threads; the oracle only reads its
    scene, and its C calls release the GIL. Returns the extrapolated
    full-iteration rate W*H / (t_light + W*H * t_pixel) in Mpaths/s, the wall
    seconds spent, and the number of entries estimated of the pool's."""
    import oracle as O
    from concurrent.futures import ThreadPoolExecutor
    p = O.params(M=M, M_p=M_p, max_depth=DEPTH, booth=BOOTH, trial_cap=TRIAL_CAP,
                 pilot_max=1024 if WL.get("pilot_max", 0) >= 0 else 0)
    t0 = time.perf_counter()
    tri, bary = o.light_pass(p, it)
    _, n = o.iteration_estimates(p, td, it, tri, bary, 0, 0)
    t_lp = time.perf_counter() - t0
    ns = n if n_est is None else max(1, min(n, n_est))
    # ranges of entries: all of them, or ns entries in blocks spread over the pool
    parts = max(1, min(ns, 4 * threads))
    if ns == n:
        ranges = [(n * i // parts, n * (i + 1) // parts) for i in range(parts)]
    else:
        blk = max(1, ns // parts)
        ranges = [(k, min(n, k + blk)) for k in (n * i // parts for i in range(parts))]
    t0 = time.perf_counter()
    if threads > 1:
        with ThreadPoolExecutor(threads) as ex:
            got = list(ex.map(lambda kr: o.iteration_estimates(p, td, it, tri, bary, kr[0], kr[1])[0], ranges))
    else:
        got = [o.iteration_estimates(p, td, it, tri, bary, kr[0], kr[1])[0] for kr in ranges]
    t_est = time.perf_counter() - t0
    done = sum(len(g) for g in got)
    rhat = np.full(n, float(np.mean(np.concatenate(got))) if done else 1.0)
    for (k0, _), g in zip(ranges, got):
        rhat[k0:k0 + len(g)] = g
    t_light = t_lp + t_est * n / max(done, 1)
    t0 = time.perf_counter()
    o.iteration(p, td, it, tri, bary, pix_lo=0, pix_hi=0, rhat=rhat)
    t_pool = time.perf_counter() - t0
    t0 = time.perf_counter()
    if threads > 1:
        pr = [(npx * i // threads, npx * (i + 1) // threads) for i in range(threads)]
        with ThreadPoolExecutor(threads) as ex:
            parts_rgb = list(ex.map(lambda q: o.iteration(p, td, it, tri, bary, pix_lo=q[0], pix_hi=q[1],
                                                          rhat=rhat)["rgb"], pr))
        rgb = np.concatenate(parts_rgb)
    else:
        rgb = o.iteration(p, td, it, tri, bary, pix_lo=0, pix_hi=npx, rhat=rhat)["rgb"]
    t_eye = max(time.perf_counter() - t0 - t_pool, 1e-9)
    rate = W * H / (t_light + W * H * t_eye / npx) / 1e6
    secs = t_lp + t_est + t_pool + t_eye
    if keep:
        return rate, secs, (done, n), np.asarray(rgb, np.float64)
    return rate, secs, (done, n)


def oracle_threads():
    """Host cores this process may run on (its CPU affinity), at most 64."""
    try:
        n = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        n = os.cpu_count() or 1
    return max(1, min(64, n))


def oracle_sample(scene, M_p, npx=2048, tables=None, n_est=None):
    """Returns the extrapolated rate on all host cores, its description, the
    thread count and the sampled pixels' 1-spp radiance (first `npx`
    pixels)."""
    o, td = oracle_tables(scene, tables)
    nt = oracle_threads()
    note = ""
    try:
        rate, secs, (done, n), rgb = oracle_iteration_rate(o, td, M_p, 0, npx, keep=True, threads=nt, n_est=n_est)
    except Exception as e:   # keep the bench line: time on one thread and say why
        note = " (threaded timing failed: %s; timed on 1 thread)" % str(e).splitlines()[0][:120]
        nt = 1
        rate, secs, (done, n), rgb = oracle_iteration_rate(o, td, M_p, 0, npx, keep=True, threads=1, n_est=n_est)
    desc = ("1 iteration on %d threads: light pass (M=%d), reciprocal estimates of %d of the pool's %d incomplete "
            "sub-paths (M_p=%d, split by entry, time scaled to the pool) and eye paths of %d of %d pixels (split by "
            "pixel; %.1f s); extrapolated to the full %dx%d iteration"
            % (nt, M, done, n, M_p, npx, W * H, secs, W, H)) + note
    return rate, desc, nt, rgb


def roulette_name():
    return "paper's RRS function" if BOOTH <= 0 else "Booth's roulette, c = %g" % BOOTH


def mape(x, ref):
    """mean over pixels and channels of |x - r| / (r + eps), eps = 1e-2 mean(r)"""
    x, ref = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    eps = 1e-2 * float(ref.mean())
    return float(np.mean(np.abs(x - ref) / (ref + eps)))


def oracle_M_p(o, td):
    """Light sub-paths the oracle scans for about ENTRY_TARGET incomplete
    sub-paths per iteration (counted after the learned cost bound)."""
    import oracle as O
    p = O.params(M=M, M_p=M, max_depth=DEPTH, trial_cap=TRIAL_CAP,
                 pilot_max=1024 if WL.get("pilot_max", 0) >= 0 else 0)
    tri, bary = o.light_pass(p, 1 << 20)
    _, n = o.iteration_estimates(p, td, 1 << 20, tri, bary, 0, 0)
    return int(min(M, max(1, round(ENTRY_TARGET * M / max(n, 1)))))


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    t0 = time.perf_counter()
    sc = WL["make"]()
    o, td = oracle_tables(sc)
    M_p = oracle_M_p(o, td)
    setup_s = time.perf_counter() - t0
    npx = WL.get("oracle_px", 1024)
    n_est = WL.get("oracle_est")
    nt = oracle_threads()
    vals, secs, cnt = [], [], []
    for k in range(args.warmup + args.steps):
        v, sec, dn = oracle_iteration_rate(o, td, M_p, k, npx, threads=nt, n_est=n_est)
        if k >= args.warmup:
            vals.append(v)
            secs.append(sec)
            cnt.append(dn)
    v = float(np.mean(vals))
    desc = ("per step 1 iteration on %d threads: light pass (M=%d), reciprocal estimates of %d of about %d "
            "incomplete sub-paths per iteration (M_p=%d, split by entry, time scaled to the pool), eye paths of %d of "
            "%d pixels (split by pixel); extrapolated to the full iteration; tables learned by the oracle (%.0f s)"
            % (nt, M, int(np.mean([c[0] for c in cnt])), int(np.mean([c[1] for c in cnt])), M_p, npx, W * H,
               setup_s))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpaths/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": desc, "M_p": M_p, "roulette": roulette_name(),
                      "proposal": "table (the oracle's learned proposal needs the device-trained network)"},
           "cpu_baseline": {"value": v, "unit": "Mpaths/s", "cores": nt, "kind": "oracle", "sample": desc},
           "e2e": {"value": v, "unit": "Mpaths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def train_network(N, r, M_p, base_iter):
    """Online training of the proposal network on 2^22 (or the workload's
    count of) connection samples the renderer generates, in rounds of 2^20."""
    rounds = max(1, WL["train_samples"] >> 20)
    t0 = time.perf_counter()
    tr = r.train_proposal(N.config(M=M, M_p=M_p, max_depth=DEPTH, seed=7, trial_cap=TRIAL_CAP,
                                   pilot_max=WL.get("pilot_max", 0)),
                          N.train_desc(samples=1 << 20, rounds=rounds, steps=500, batch=8192, lr=3e-3, seed=5,
                                       iter0=(1 << 23) + base_iter, proxy=1))
    tr["train_s"] = time.perf_counter() - t0
    return tr


def equal_time_study(N, r, M_p, base_iter, ms, tables_used):
    """Learned vs plain proposal on the bench workload at equal wall time:
    `ms` holds one step's device time under each proposal. A reference of
    ref_mult x SPP iterations (table proposal, disjoint iterations) is
    rendered; the table image of one step (SPP iterations) and the learned
    image of as many iterations as fit the same time are compared with it by
    MAPE. Also the connection estimate's second moment under both proposals
    (both are unbiased, so the smaller one is the better proposal). Untimed
    with respect to the headline number."""
    base = dict(M=M, M_p=M_p, max_depth=DEPTH, seed=7, trial_cap=TRIAL_CAP, pilot_max=WL.get("pilot_max", 0))
    ref_spp = WL["ref_mult"] * SPP
    mt = r.connection_moments(N.config(spp=4, iter0=base_iter + (5 << 20), **base))
    ml = r.connection_moments(N.config(spp=4, iter0=base_iter + (5 << 20), proposal=2, **base))
    t0 = time.perf_counter()
    r.clear()
    st_ref = r.render(N.config(spp=ref_spp, iter0=base_iter + (2 << 20), **base), allow_truncated=True)
    ref = r.film().astype(np.float64)
    ref_s = time.perf_counter() - t0
    spp_l = max(1, int(round(SPP * ms["table"] / ms["learned"])))
    r.clear()
    r.render(N.config(spp=SPP, iter0=base_iter + (3 << 20), **base), allow_truncated=True)
    img_t = r.film().astype(np.float64)
    r.clear()
    r.render(N.config(spp=spp_l, iter0=base_iter + (4 << 20), proposal=2, **base), allow_truncated=True)
    img_l = r.film().astype(np.float64)
    r.clear()
    return {
        "seconds": ms["table"] * 1e-3,
        "reference": "%d iterations (%dx a step), table proposal, disjoint iterations; %d truncated estimates; "
                     "%.0f s" % (ref_spp, WL["ref_mult"], st_ref["n_truncated"], ref_s),
        "mape": {"table": mape(img_t, ref), "learned": mape(img_l, ref)},
        "spp": {"table": SPP, "learned": spp_l},
        "connection_second_moment": {"table": mt["m2"], "learned": ml["m2"], "gain": mt["m2"] / max(ml["m2"], 1e-300),
                                     "mean_table": mt["mean"], "mean_learned": ml["mean"]},
        "_ref": ref, "_ref_spp": ref_spp,
    }


def workload_parity(N, r, o, td, M_p, n_iter=2, rows=2, n_est=32):
    """Parity with the oracle on the bench workload itself, path by path: for
    n_iter iterations the device runs one iteration (pb_iteration: light
    pass, pool, estimates, eye pass) and the oracle recomputes the eye paths
    of `rows` image rows through the middle from the same light geometry and
    the device's estimates, and n_est of the estimates from scratch. Reports
    the share of paths and estimates whose topology signatures agree and the
    relative errors where they do (path error relative to its largest
    channel)."""
    import oracle as O
    from concurrent.futures import ThreadPoolExecutor
    pm = 1024 if WL.get("pilot_max", 0) >= 0 else 0
    p = O.params(M=M, M_p=M_p, max_depth=DEPTH, trial_cap=TRIAL_CAP, pilot_max=pm)
    cfg = N.config(M=M, M_p=M_p, max_depth=DEPTH, seed=7, trial_cap=TRIAL_CAP, pilot_max=WL.get("pilot_max", 0))
    lo, hi = (H // 2 - rows // 2) * W, (H // 2 - rows // 2 + rows) * W
    nt = oracle_threads()
    t0 = time.perf_counter()
    errs, same_n, tot_n, e_errs, e_same, e_tot = [], 0, 0, [], 0, 0
    for it in range(n_iter):
        itn = (7 << 20) + it
        tri, bary = r.light_pass(cfg, itn)
        got = r.iteration(cfg, itn, tri, bary, cap=1 << 20)
        if o.iteration_estimates(p, td, itn, tri, bary, 0, 0)[1] != len(got["rhat"]):
            continue   # the two pools differ (a label decided differently): the estimates do not line up
        pr = [(lo + (hi - lo) * i // nt, lo + (hi - lo) * (i + 1) // nt) for i in range(nt)]
        with ThreadPoolExecutor(nt) as ex:
            parts = list(ex.map(lambda q: o.iteration(p, td, itn, tri, bary, pix_lo=q[0], pix_hi=q[1],
                                                      rhat=got["rhat"].astype(np.float64)), pr))
        ref_rgb = np.concatenate([x["rgb"] for x in parts])
        ref_sig = np.concatenate([x["sig"] for x in parts])
        same = ref_sig == got["sig"][lo:hi]
        same_n += int(same.sum())
        tot_n += len(same)
        a, b = ref_rgb[same], got["rgb"][lo:hi][same].astype(np.float64)
        mag = np.abs(a).max(1)
        d = np.abs(a - b).max(1)
        errs.append(np.where(mag > 0, d / np.where(mag > 0, mag, 1.0), np.where(d > 0, 1.0, 0.0)))
        # a spread subset of the estimates, from scratch on the oracle
        n = len(got["rhat"])
        ks = sorted(set(int(k) for k in np.linspace(0, n - 1, min(n, n_est))))
        with ThreadPoolExecutor(nt) as ex:
            est = list(ex.map(lambda k: o.iteration_estimates(p, td, itn, tri, bary, k, k + 1)[0], ks))
        for k, e in zip(ks, est):
            if len(e) == 0:
                continue
            e_tot += 1
            rel = abs(e[0] - got["rhat"][k]) / max(abs(e[0]), 1e-30)
            e_errs.append(rel)
            e_same += int(rel <= 1e-3)
    errs = np.concatenate(errs) if errs else np.zeros(0)
    q = lambda x, v: float(np.quantile(x, v)) if len(x) else None
    return {"iterations": n_iter, "pixels_per_iteration": int(hi - lo), "topology_agreement": same_n / max(tot_n, 1),
            "path_rel_err": {"median": q(errs, 0.5), "p99": q(errs, 0.99), "p999": q(errs, 0.999),
                             "max": q(errs, 1.0)},
            "paths_within_1e-4": float((errs <= 1e-4).mean()) if len(errs) else None,
            "estimates_checked": e_tot, "estimates_within_1e-3": e_same / max(e_tot, 1),
            "estimate_rel_err_max": max(e_errs) if e_errs else None,
            "seconds": time.perf_counter() - t0, "threads": nt}


def run_subspace_ablation(args):
    """The paper's subspace-selection comparison on the water-pool scene:
    only the proxy strategy's paths are rendered (film mode 1), at equal
    iterations, with the learned selection rows Gamma' and with uniform rows,
    against a reference rendered with the learned rows on disjoint
    iterations. Prints one JSON line with both MAPEs. 1 GPU, rank 0 only."""
    import torch
    ws, rank, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_2503_23412_gb300 import native as N
    from paper_2503_23412_gb300 import scenes
    Wa = Ha = 128
    spp, ref_spp, depth, Ma = 128, 2048, 8, 10000
    sc = scenes.water(Wa, Ha)
    r = N.Renderer(sc, None, device=local)
    st = r.prepare(N.config(M=Ma, M_p=Ma, max_depth=depth), n_iter=4, iter0=1 << 22, n_bsamples=32, lloyd_iters=8,
                   KT=64, KS=64, KSp=32, KC=4)
    learned = r.tables_readback()
    uniform = dict(learned, gamma_proxy=np.full_like(learned["gamma_proxy"], 1.0 / learned["gamma_proxy"].shape[1]))
    # about ENTRY_TARGET incomplete sub-paths per iteration (the paper's practical limit), as the
    # other workloads; with all M light paths the water scene's pool outgrows the chain slots
    frac = st["n_entries"] / float(4 * Ma)
    M_p = int(min(Ma, max(1, round(ENTRY_TARGET / max(frac, 1e-9)))))
    base = dict(M=Ma, M_p=M_p, max_depth=depth, seed=7, film=1)

    def render(tables, n, iter0):
        r.upload_tables(tables)
        r.clear()
        st = r.render(N.config(spp=n, iter0=iter0, **base), allow_truncated=True)
        return r.film().astype(np.float64), st

    ref, _ = render(learned, ref_spp, 1 << 24)
    img_l, st_l = render(learned, spp, 0)
    img_u, st_u = render(uniform, spp, 0)
    out = {"metric": "proxy-only MAPE at equal iterations, importance vs uniform subspace selection",
           "unit": "MAPE", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "water pool %dx%d, depth %d, M=%d, M_p=%d, %d iterations each, reference %d "
                                  "iterations" % (Wa, Ha, depth, Ma, M_p, spp, ref_spp), "film": "proxy strategy only"},
           "mape": {"importance": mape(img_l, ref), "uniform": mape(img_u, ref)},
           "proxy_ok": {"importance": st_l["n_proxy_ok"], "uniform": st_u["n_proxy_ok"]},
           "ms": {"importance": st_l["ms"], "uniform": st_u["ms"]}}
    print(json.dumps(out))


def run_rr_ablation(args):
    """The paper's RR ablation on the projector workload: MAPE at equal time
    of the paper's RRS function and of Booth's roulette at scales 10 ... 10^4,
    against a reference rendered with the paper's function on disjoint
    iterations. The time budget is one 64-iteration render with the paper's
    function. Prints one JSON line. 1 GPU, rank 0 only."""
    import torch
    ws, rank, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_2503_23412_gb300 import native as N
    from paper_2503_23412_gb300 import scenes
    sc = scenes.projector(W, H)
    r = N.Renderer(sc, None, device=local)
    st = r.prepare(N.config(M=M, M_p=M, max_depth=DEPTH, spp=1, seed=7), n_iter=4, iter0=1 << 22, n_bsamples=32,
                   lloyd_iters=8, KT=300, KS=300, KSp=100, KC=10, tile=10)
    frac = st["n_entries"] / float(4 * M)
    M_p = int(min(M, max(1, round(ENTRY_TARGET / max(frac, 1e-9)))))
    base = dict(M=M, M_p=M_p, max_depth=DEPTH, seed=7, trial_cap=TRIAL_CAP)

    def render(n, iter0, booth):
        r.clear()
        s_ = r.render(N.config(spp=n, iter0=iter0, booth=booth, **base), allow_truncated=True)
        return r.film().astype(np.float64), s_

    ref, _ = render(16 * SPP, 1 << 24, 0.0)
    img, st0 = render(SPP, 0, 0.0)
    budget = st0["ms"]
    rows = {"paper_rrs": {"spp": SPP, "ms": budget, "mape": mape(img, ref), "nodes": st0["n_nodes"]}}
    for c in (10.0, 100.0, 1000.0, 10000.0):
        _, probe = render(8, 1 << 23, c)                       # time per iteration with this scale
        n = max(1, int(round(8 * budget / max(probe["ms"], 1e-6))))
        img_c, st_c = render(n, 0, c)
        rows["booth_%g" % c] = {"spp": n, "ms": st_c["ms"], "mape": mape(img_c, ref), "nodes": st_c["n_nodes"],
                                "truncated": st_c["n_truncated"]}
    out = {"metric": "equal-time MAPE of the reciprocal estimator's Russian roulette: paper's RRS vs Booth",
           "unit": "MAPE", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
           "config": {"workload": WORKLOAD, "M_p": M_p, "reference": "%d iterations, paper's RRS" % (16 * SPP),
                      "budget_ms": budget},
           "rows": rows}
    print(json.dumps(out))


def run_batch(args):
    """Batched workload: procedural glass / GGX / diffuse scenes of uneven
    size rendered by one graph launch (pb_render_batch), each with its
    autotuned configuration, against the same scenes rendered one after
    another. 1 GPU, rank 0 only."""
    import torch
    ws, rank, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_2503_23412_gb300 import native as N
    from paper_2503_23412_gb300 import scenes
    specs = scenes.batch_specs(args.scenes, seed=1)
    depth, Mb = 10, 10000
    rs, cfgs, tuned = [], [], 0
    t0 = time.perf_counter()
    for (w_, h_, spp, nt, sd) in specs:
        sc = scenes.glossy_mix(w_, h_, nt, seed=sd)
        r = N.Renderer(sc)
        st = r.prepare(N.config(M=Mb, M_p=Mb, max_depth=depth), n_iter=2, iter0=1 << 22, n_bsamples=16,
                       lloyd_iters=6, KT=64, KS=64, KSp=32, KC=4)
        frac = st["n_entries"] / float(2 * Mb)
        mp = int(min(Mb, max(1, round(ENTRY_TARGET / max(frac, 1e-9)))))
        cfg = N.config(M=Mb, M_p=mp, max_depth=depth, spp=spp, seed=7)
        best, cached = r.autotune(cfg, trial_iters=16)
        tuned += 0 if cached else 1
        rs.append(r)
        cfgs.append(best)
    setup_s = time.perf_counter() - t0
    paths = sum(w_ * h_ * spp for (w_, h_, spp, _, _) in specs)
    # one after another, eager
    seq_ms = 0.0
    for r, c in zip(rs, cfgs):
        r.clear()
        seq_ms += r.render(c, allow_truncated=True)["ms"]
    # one graph launch per batch: the first captures every scene's graph
    for k in range(args.warmup + args.steps):
        for r in rs:
            r.clear()
        for c in cfgs:
            c.iter0 = (k + 1) * 4096
        st = N.render_batch(rs, cfgs, allow_truncated=True)
        if k == args.warmup:
            times = []
        if k >= args.warmup:
            times.append(st[0]["batch_ms"])
    batch_ms = float(np.mean(times))
    out = {"metric": "Mpaths/s, batched render of procedural scenes in one graph launch", "value": paths / (batch_ms * 1e-3) / 1e6,
           "unit": "Mpaths/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": batch_ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batch of %d glass/GGX/diffuse scenes (20/40/40), 1k-500k triangles log-uniform, "
                                  "{128,256,512}^2, spp 16-256 log-uniform, depth %d, M=%d" % (len(specs), depth, Mb),
                      "scenes": [{"W": w_, "spp": s_, "tris": t_} for (w_, _, s_, t_, _) in specs],
                      "paths_per_step": paths, "sequential_eager_ms": seq_ms,
                      "sequential_eager_mpaths": paths / (seq_ms * 1e-3) / 1e6,
                      "speedup_vs_sequential": seq_ms / batch_ms, "setup_s": setup_s, "autotuned_buckets": tuned,
                      "tuned": [{"batch": c.batch, "estimator": c.estimator} for c in cfgs]}}
    print(json.dumps(out))
    for r in rs:
        r.close()


# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_2503_23412_gb300 import native as N

    proposal = args.proposal or WL["proposal"]
    sc = WL["make"]()
    stream = torch.cuda.current_stream()
    n_learn = WL.get("learn_iters", 4 if M >= 10000 else 2)
    pilot = WL.get("pilot_max", 0)
    t0 = time.perf_counter()
    r = N.Renderer(sc, None, device=local, stream=stream.cuda_stream)
    upload_s = time.perf_counter() - t0
    # learn the tables on the device (the paper's preprocessing)
    learn_cfg = N.config(M=M, M_p=M, max_depth=DEPTH, spp=1, seed=7, trial_cap=TRIAL_CAP, pilot_max=pilot)
    t0 = time.perf_counter()
    st = r.prepare(learn_cfg, n_iter=n_learn, iter0=1 << 22, n_bsamples=WL.get("learn_nb", 32), lloyd_iters=8,
                   KT=300, KS=WL["KS"], KSp=100, KC=10, tile=10)
    learn_s = time.perf_counter() - t0
    tables = r.tables_readback()
    gated = int((tables["mis_tab"] == 0).sum())
    # M_p for about ENTRY_TARGET incomplete sub-paths per iteration, counted after the learned cost bound
    cal = r.render(N.config(M=M, M_p=M, max_depth=DEPTH, spp=2, seed=7, iter0=3 << 21, trial_cap=TRIAL_CAP,
                            pilot_max=pilot), allow_truncated=True)
    r.clear()
    frac = cal["n_entries"] / float(2 * M)
    M_p = int(min(M, max(1, round(ENTRY_TARGET / max(frac, 1e-9)))))
    base_iter = rank_iter_base(rank)
    study_on = rank == 0 and WL["ref_mult"] > 0 and BOOTH <= 0 and not args.no_study
    trained = None
    if proposal == "learned" or study_on:
        trained = train_network(N, r, M_p, base_iter)   # before timing, like the tables
    cfg = N.config(M=M, M_p=M_p, max_depth=DEPTH, spp=SPP, seed=7, booth=BOOTH, trace=TRACE, trial_cap=TRIAL_CAP,
                   proposal=2 if proposal == "learned" else 0, pilot_max=pilot)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(i, count=False, prop=None):
        cfg.iter0 = base_iter + i * SPP
        cfg.count_traversal = 1 if count else 0
        old = cfg.proposal
        if prop is not None:
            cfg.proposal = prop
        r.clear()
        out = r.render(cfg, allow_truncated=True)
        cfg.proposal = old
        return out

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    times, stats = [], []
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.nvtx.range_push("timed_step")   # profilers select the timed launches by this range
            e0.record(stream)
            stats.append(step(args.warmup + i))
            e1.record(stream)
            torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    if dist:
        dist.barrier()
    total_ms = job_ms(float(np.sum(times)), dist, "cuda")
    value = job_value(W * H * SPP * args.steps, ws, total_ms)
    nxt = args.warmup + args.steps
    # the other proposal, for the equal-time comparison (untimed with respect to the headline)
    other_ms = None
    if study_on:
        other = 0 if cfg.proposal == 2 else 2
        step(nxt, prop=other)
        ot = []
        for i in range(2):
            flush.zero_()
            torch.cuda.synchronize()
            ot.append(step(nxt + 1 + i, prop=other)["ms"])
        other_ms = float(np.mean(ot))
        nxt += 3
    # traversal work of one step (untimed counting run) -> algorithmic bytes
    cst = step(nxt, count=True)
    nxt += 1
    mean = {k: float(np.mean([s[k] for s in stats]))
            for k in ("ms_light", "ms_pool", "ms_recip", "ms_mlp", "ms_eye", "ms_eye_feat", "ms_eye_occ")}
    waves = stats[-1]["n_waves"]
    # the three traversal stages: the estimator's wavefront, the camera sub-paths (feature pass) and the
    # eye side's occlusion answers; algorithmic bytes = 64 per node visit + 48 per triangle test
    stages = {
        "k_recip": ((64.0 * cst["rec_nodes"] + 48.0 * cst["rec_tris"]) / waves, mean["ms_recip"] / waves),
        "k_eye_feat": ((64.0 * cst["cam_nodes"] + 48.0 * cst["cam_tris"]) / waves, mean["ms_eye_feat"] / waves),
        "k_eye_occ": ((64.0 * cst["shd_nodes"] + 48.0 * cst["shd_tris"]) / waves, mean["ms_eye_occ"] / waves),
    }
    dom = max(stages, key=lambda k: stages[k][1])
    b, ms = stages[dom]
    peak, peak_kind = peaks()
    achieved = b / (ms * 1e-3) / 1e9
    sha = src_sha(REC_SRC if dom == "k_recip" else EYE_SRC)
    # end to end through the C ABI with host buffers, every step: scene upload (host BVH build included),
    # tables and network upload, render, film readback
    w_net = r.mlp_readback() if cfg.proposal == 2 else None
    w_prx = r.mlp_proxy_readback() if cfg.proposal == 2 else None
    h2d = sum(v.nbytes for v in sc.values()) + sum(v.nbytes for v in tables.values() if isinstance(v, np.ndarray))
    h2d += 0 if w_net is None else w_net.nbytes + w_prx.nbytes
    d2h = W * H * 3 * 4
    e2e_t = []
    for i in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r.upload_scene(sc)
        r.upload_tables(tables)
        if w_net is not None:
            r.mlp_upload(w_net)
            r.mlp_proxy_upload(w_prx)
        cfg.iter0 = base_iter + (nxt + i) * SPP
        cfg.count_traversal = 0
        r.clear()
        r.render(cfg, allow_truncated=True)
        r.film()
        e2e_t.append(time.perf_counter() - t0)
    nxt += 3
    e2e = W * H * SPP * ws / float(np.mean(e2e_t)) / 1e6
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    study = None
    if study_on:
        ms_pair = {"learned": total_ms / args.steps, "table": other_ms} if cfg.proposal == 2 else \
            {"table": total_ms / args.steps, "learned": other_ms}
        study = equal_time_study(N, r, M_p, base_iter, ms_pair, tables)
        study["learned_value"] = W * H * SPP / (ms_pair["learned"] * 1e-3) / 1e6
        study["table_value"] = W * H * SPP / (ms_pair["table"] * 1e-3) / 1e6
    # the oracle on all host cores, with the device's tables (the same incomplete sub-paths are estimated)
    cpu_v, cpu_desc, cpu_nt, cpu_px = oracle_sample(sc, M_p, npx=WL.get("oracle_px", 2048), tables=tables,
                                                    n_est=WL.get("oracle_est"))
    if study is not None:
        ref = study.pop("_ref")
        ref_spp = study.pop("_ref_spp")
        o, td = oracle_tables(sc, tables)
        study["workload_parity"] = workload_parity(N, r, o, td, M_p)
        npx = len(cpu_px)
        study["mape"]["cpu_oracle_1spp"] = mape(cpu_px, ref[:npx])
        study["cpu_oracle"] = {"spp": 1, "pixels": npx, "threads": cpu_nt,
                               "seconds_per_spp_full_image": W * H / (cpu_v * 1e6),
                               "note": "device tables; MAPE over the first %d pixels" % npx}
    out = {
        "metric": METRIC, "value": value, "unit": "Mpaths/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "proposal": ("learned: networks for the connection's light subspace S and the proxy's specular "
                                "subspace S', each mixed 0.9 / 0.1 with its table row" if proposal == "learned"
                                else "table rows Gamma and Gamma'"),
                   "M": M, "M_p": M_p, "spp": SPP, "max_depth": DEPTH,
                   "triangles": int(len(sc["tris"])), "trial_cap": TRIAL_CAP,
                   "l2": "256 MiB buffer written before every timed step",
                   "tables": "learned on the device before timing (%.1f s, %d learning iterations); %d of %d "
                             "(u, S', C) cells left to the other strategies by the learned cost bound"
                             % (learn_s, n_learn, gated, tables["mis_tab"].size),
                   "scene_upload_s": upload_s,
                   "stage_ms_per_step": mean, "entries_per_iteration": stats[-1]["n_entries"] / SPP,
                   "truncated_estimates_per_step": int(max(s["n_truncated"] for s in stats)),
                   "estimator_nodes_per_step": stats[-1]["n_nodes"], "parallelism": "replicas" if ws > 1 else "1 GPU",
                   "roulette": roulette_name(),
                   "estimator_bound": ("per-entry pilot maximum of f/q (learned cell value when the pilot saw no f > 0)"
                                       if pilot >= 0 else "learned (u, S', C) cell maximum of f/q, %d draws per entry "
                                       "over %d learning iterations" % (WL.get("learn_nb", 32), n_learn)),
                   "traversal": "persistent warps, lane refill (estimator trace stages, occlusion answers)" if TRACE else "one ray per thread"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic_for(dom, sha),
                     "algorithmic_bytes_per_launch": b, "launch_ms": ms, "src_sha": sha},
        # both traversal-bound stages against the same denominator (the dominant one is "roofline")
        "roofline_stages": {
            name: {"achieved": bb / (mm * 1e-3) / 1e9, "frac": bb / (mm * 1e-3) / 1e9 / peak, "unit": "GB/s",
                   "algorithmic_bytes_per_wave": bb, "ms_per_wave": mm}
            for name, (bb, mm) in stages.items() if mm > 0},
        "cpu_baseline": {"value": cpu_v, "unit": "Mpaths/s", "cores": cpu_nt, "kind": "oracle", "sample": cpu_desc},
        "e2e": {"value": e2e, "unit": "Mpaths/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h},
        "clocks": clk.summary(),
        "gpu_launches": int(sum(s["n_launches"] for s in stats)),
    }
    if study is not None:
        out["equal_time"] = study
    if trained is not None:
        out["config"]["proposal_training"] = trained
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def main():
    global W, H, SPP, M, DEPTH, WORKLOAD, WL, BOOTH, TRACE
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--proposal", default=None, choices=["table", "learned"],
                    help="light-subspace proposal of the timed steps (default: the workload's; learned: trained "
                         "before timing)")
    ap.add_argument("--workload", default="glossy", choices=sorted(WORKLOADS) + ["batch", "subspace", "rr"],
                    help="glossy: the learned-proposal comparison at 1024^2 on the ~1M-triangle glossy scene; "
                         "glossy512: the same scene at 512^2, 128 spp, table proposal; projector: the caustic "
                         "scene at 256^2, 64 spp; projector_r001: its lens at roughness 0.01; small / glossy_small: "
                         "profiler cases; batch: procedural scenes of uneven size in one graph launch; "
                         "subspace: the proxy-only selection comparison on the water scene; "
                         "rr: equal-time MAPE of the paper's RRS against Booth's roulette")
    ap.add_argument("--scenes", type=int, default=16, help="scenes of the batch workload")
    ap.add_argument("--booth", type=float, default=0.0,
                    help="Booth's Russian roulette of this scale in the reciprocal estimator (the RR ablation's "
                         "baseline; 0: the paper's RRS function)")
    ap.add_argument("--trace", type=int, default=1, choices=[0, 1],
                    help="1 (default): the estimator's trace stages and the eye pass's occlusion answers on "
                         "persistent warps that refill idle lanes; 0: one ray per thread")
    ap.add_argument("--no-study", action="store_true", help="skip the equal-time study and the oracle validation")
    args = ap.parse_args()
    BOOTH = max(0.0, args.booth)
    TRACE = args.trace
    if args.workload in WORKLOADS:
        WL = WORKLOADS[args.workload]
        W = H = WL["W"]
        SPP, DEPTH, M, WORKLOAD = WL["spp"], WL["depth"], WL["M"], WL["desc"]
    elif args.workload == "rr":
        WL = WORKLOADS["projector"]
        W = H = WL["W"]
        SPP, DEPTH, M, WORKLOAD = WL["spp"], WL["depth"], WL["M"], WL["desc"]
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "subspace":
        run_subspace_ablation(args)
    elif args.workload == "rr":
        run_rr_ablation(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
