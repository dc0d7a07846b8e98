"""Benchmark: Mpaths/s of the proxy-tracing BDPT render on the projector
workload (256x256, 64 spp, max depth 8, M = 10,000 light sub-paths,
reciprocal estimates on ~400 incomplete light sub-paths per iteration).

One step = one full render of the workload (64 iterations: light pass, pool
build, reciprocal estimation, eye pass with connections, proxy retrace and
MIS, film accumulation) on inputs resident on the device. The subspace
tables are learned on the device once before timing (the paper's
preprocessing). Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm of this build: there is no runnable upstream).
"""

from __future__ import annotations

import argparse
import hashlib
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
W, H, SPP, DEPTH, M = 256, 256, 64, 8, 10000   # projector workload; --workload small shrinks it
ENTRY_TARGET = 400          # incomplete light sub-paths estimated per iteration (paper: up to 400)
BOOTH = 0.0                 # --booth: Booth's Russian roulette scale in the estimator (0: the paper's RRS)
TRACE = 0                   # --trace: 1 = the estimator's trace stages on persistent warps with lane refill
WORKLOAD = ("projector 256x256, 64 spp, max depth 8: textured 0.1x0.1 emitter in an absorbing box, "
            "biconvex GGX dielectric lens (IOR 1.5, ~19.5k triangles), diffuse room; M=10000 light "
            "sub-paths/iteration, 5 reciprocal repeats, 300 eye / 300 light / 100 specular / 10 control subspaces")
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
def oracle_tables(scene):
    """Tables for the oracle's timing runs, learned by the oracle itself
    (random centroids, B / MIS / Gamma / grid from one small learning pass)."""
    import oracle as O
    from paper_2503_23412_gb300 import scenes
    o = O.Oracle(scene)
    tab = scenes.random_tables(scene, KT=300, KS=300, KSp=100, KC=10)
    tab = o.learn(O.params(M=1000, M_p=1000, max_depth=DEPTH), tab, 1 << 21, 1, n_bsamples=16)
    return o, o.tables(tab)


def oracle_iteration_rate(o, td, M_p, it, npx, keep=False, threads=1):
    """CPU oracle, one iteration of the workload measured in two parts: the
    light side (light pass, pool, all reciprocal estimates) and the eye paths
    of the first `npx` pixels (reusing those estimates). With threads > 1 the
    estimates (in small entry ranges) and the eye paths (split by pixel) run
    on that many threads; the oracle only reads its scene, and its C calls
    release the GIL. Returns the extrapolated full-iteration rate
    W*H / (t_light + W*H * t_pixel) in Mpaths/s and the wall seconds spent."""
    import oracle as O
    from concurrent.futures import ThreadPoolExecutor
    p = O.params(M=M, M_p=M_p, max_depth=DEPTH, booth=BOOTH)
    t0 = time.perf_counter()
    tri, bary = o.light_pass(p, it)
    if threads > 1:
        _, n = o.iteration_estimates(p, td, it, tri, bary, 0, 0)
        parts = 4 * threads   # chain lengths vary widely: small ranges, taken as threads free up
        ranges = [(n * i // parts, n * (i + 1) // parts) for i in range(parts)]
        with ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(lambda kr: o.iteration_estimates(p, td, it, tri, bary, kr[0], kr[1])[0], ranges))
        rhat = np.concatenate(parts)
    else:
        rhat = o.iteration(p, td, it, tri, bary, pix_lo=0, pix_hi=0)["rhat"]
    t_light = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.iteration(p, td, it, tri, bary, pix_lo=0, pix_hi=0, rhat=rhat)
    t_pool = time.perf_counter() - t0
    t0 = time.perf_counter()
    if threads > 1:
        ranges = [(npx * i // threads, npx * (i + 1) // threads) for i in range(threads)]
        with ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(lambda pr: o.iteration(p, td, it, tri, bary, pix_lo=pr[0], pix_hi=pr[1],
                                                       rhat=rhat)["rgb"], ranges))
        rgb = np.concatenate(parts)
    else:
        rgb = o.iteration(p, td, it, tri, bary, pix_lo=0, pix_hi=npx, rhat=rhat)["rgb"]
    t_eye = max(time.perf_counter() - t0 - t_pool, 1e-9)
    rate = W * H / (t_light + W * H * t_eye / npx) / 1e6
    if keep:
        return rate, t_light + t_pool + t_eye, np.asarray(rgb, np.float64)
    return rate, t_light + t_pool + t_eye


def oracle_threads():
    """Host cores this process may run on (its CPU affinity), at most 64."""
    try:
        n = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        n = os.cpu_count() or 1
    return max(1, min(64, n))


def oracle_sample(scene, M_p, npx=2048):
    """Returns the extrapolated rate on all host cores, its description, the
    thread count and the sampled pixels' 1-spp radiance (first `npx`
    pixels)."""
    o, td = oracle_tables(scene)
    nt = oracle_threads()
    note = ""
    try:
        rate, secs, rgb = oracle_iteration_rate(o, td, M_p, 0, npx, keep=True, threads=nt)
    except Exception as e:   # keep the bench line: time on one thread and say why
        note = " (threaded timing failed: %s; timed on 1 thread)" % str(e).splitlines()[0][:120]
        nt = 1
        rate, secs, rgb = oracle_iteration_rate(o, td, M_p, 0, npx, keep=True, threads=1)
    desc = ("1 iteration on %d threads: light pass (M=%d), reciprocal estimates (M_p=%d, split by entry) and eye "
            "paths of %d of %d pixels (split by pixel; %.1f s); extrapolated to the full %dx%d iteration"
            % (nt, M, M_p, npx, W * H, secs, W, H)) + note
    return rate, desc, nt, rgb


def roulette_name():
    return "paper's RRS function" if BOOTH <= 0 else "Booth's roulette, c = %g" % BOOTH


def mape(x, ref):
    """mean over pixels and channels of |x - r| / (r + eps), eps = 1e-2 mean(r)"""
    x, ref = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    eps = 1e-2 * float(ref.mean())
    return float(np.mean(np.abs(x - ref) / (ref + eps)))


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2503_23412_gb300 import scenes
    sc = scenes.projector(W, H)
    o, td = oracle_tables(sc)
    M_p = int(os.environ.get("PB_BENCH_MP", "1400"))
    npx = 1024
    nt = oracle_threads()
    vals, secs = [], []
    for k in range(args.warmup + args.steps):
        v, sec = oracle_iteration_rate(o, td, M_p, k, npx, threads=nt)
        if k >= args.warmup:
            vals.append(v)
            secs.append(sec)
    v = float(np.mean(vals))
    desc = ("per step 1 iteration on %d threads: light pass (M=%d), reciprocal estimates (M_p=%d, split by "
            "entry), eye paths of %d of %d pixels (split by pixel); extrapolated to the full iteration"
            % (nt, M, M_p, npx, W * H))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpaths/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": desc, "M_p": M_p, "roulette": roulette_name()},
           "cpu_baseline": {"value": v, "unit": "Mpaths/s", "cores": nt, "kind": "oracle", "sample": desc},
           "e2e": {"value": v, "unit": "Mpaths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


REF_SPP = 1024


def equal_time_study(N, r, M_p, base_iter, table_ms):
    """Learned vs plain proposal on the bench workload: trains the network on
    the renderer's connections, times a learned-proposal step, renders a
    REF_SPP reference (table proposal, disjoint iterations) and compares image
    MAPE at equal wall time (one table step). Untimed with respect to the
    headline number."""
    base = dict(M=M, M_p=M_p, max_depth=DEPTH, seed=7)
    t0 = time.perf_counter()
    tr = r.train_proposal(N.config(**base), N.train_desc(samples=1 << 20, rounds=3, steps=500, batch=8192, lr=3e-3,
                                                         seed=5, iter0=(1 << 23) + base_iter))
    train_s = time.perf_counter() - t0
    # learned-proposal step (same workload)
    r.clear()
    r.render(N.config(spp=SPP, iter0=base_iter + (1 << 20), proposal=1, **base), allow_truncated=True)
    r.clear()
    sl = r.render(N.config(spp=SPP, iter0=base_iter + (1 << 20) + SPP, proposal=1, **base), allow_truncated=True)
    learned_ms = sl["ms"]
    # connection-estimate moments under both proposals (8 iterations each)
    mt = r.connection_moments(N.config(spp=8, iter0=base_iter + (5 << 20), **base))
    ml = r.connection_moments(N.config(spp=8, iter0=base_iter + (5 << 20), proposal=1, **base))
    # reference
    r.clear()
    r.render(N.config(spp=REF_SPP, iter0=base_iter + (2 << 20), **base), allow_truncated=True)
    ref = r.film().astype(np.float64)
    # equal wall time: one table step (SPP iterations) vs as many learned iterations as fit
    spp_l = max(1, int(round(SPP * table_ms / learned_ms)))
    r.clear()
    r.render(N.config(spp=SPP, iter0=base_iter + (3 << 20), **base), allow_truncated=True)
    img_t = r.film().astype(np.float64)
    r.clear()
    r.render(N.config(spp=spp_l, iter0=base_iter + (4 << 20), proposal=1, **base), allow_truncated=True)
    img_l = r.film().astype(np.float64)
    r.clear()
    return {
        "seconds": table_ms * 1e-3,
        "reference": "%d spp, table proposal, disjoint iterations" % REF_SPP,
        "mape": {"table": mape(img_t, ref), "learned": mape(img_l, ref)},
        "spp": {"table": SPP, "learned": spp_l},
        "learned": {"value": W * H * SPP / (learned_ms * 1e-3) / 1e6, "unit": "Mpaths/s", "ms_per_step": learned_ms,
                    "ms_mlp_per_step": sl["ms_mlp"], "train_s": train_s, "train": tr},
        "connection_second_moment": {"table": mt["m2"], "learned": ml["m2"], "gain": mt["m2"] / ml["m2"],
                                     "mean_table": mt["mean"], "mean_learned": ml["mean"]},
        "_ref": ref,
    }


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
    r.prepare(N.config(M=Ma, M_p=Ma, max_depth=depth), n_iter=4, iter0=1 << 22, n_bsamples=32, lloyd_iters=8,
              KT=64, KS=64, KSp=32, KC=4)
    learned = r.tables_readback()
    uniform = dict(learned, gamma_proxy=np.full_like(learned["gamma_proxy"], 1.0 / learned["gamma_proxy"].shape[1]))
    base = dict(M=Ma, M_p=Ma, max_depth=depth, seed=7, film=1)

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
           "config": {"workload": "water pool %dx%d, depth %d, M=%d, %d iterations each, reference %d iterations"
                      % (Wa, Ha, depth, Ma, spp, ref_spp), "film": "proxy strategy only"},
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
    base = dict(M=M, M_p=M_p, max_depth=DEPTH, seed=7)

    def render(n, iter0, booth):
        r.clear()
        s_ = r.render(N.config(spp=n, iter0=iter0, booth=booth, **base), allow_truncated=True)
        return r.film().astype(np.float64), s_

    ref, _ = render(REF_SPP, 1 << 24, 0.0)
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
           "config": {"workload": WORKLOAD, "M_p": M_p, "reference": "%d iterations, paper's RRS" % REF_SPP,
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
    from paper_2503_23412_gb300 import scenes

    sc = scenes.projector(W, H)
    stream = torch.cuda.current_stream()
    n_learn = 4 if M >= 10000 else 2
    r = N.Renderer(sc, None, device=local, stream=stream.cuda_stream)
    # learn the tables on the device (paper's preprocessing), calibrate M_p for ~400 entries/iteration
    learn_cfg = N.config(M=M, M_p=M, max_depth=DEPTH, spp=1, seed=7)
    t0 = time.perf_counter()
    st = r.prepare(learn_cfg, n_iter=n_learn, iter0=1 << 22, n_bsamples=32, lloyd_iters=8,
                   KT=300, KS=300, KSp=100, KC=10, tile=10)
    learn_s = time.perf_counter() - t0
    frac = st["n_entries"] / float(n_learn * M)
    M_p = int(min(M, max(1, round(ENTRY_TARGET / max(frac, 1e-9)))))
    tables = r.tables_readback()
    base_iter = rank_iter_base(rank)
    cfg = N.config(M=M, M_p=M_p, max_depth=DEPTH, spp=SPP, seed=7, booth=BOOTH, trace=TRACE)
    trained = None
    if args.proposal == "learned":
        # the network is trained before timing, like the tables
        trained = r.train_proposal(N.config(M=M, M_p=M_p, max_depth=DEPTH, seed=7),
                                   N.train_desc(samples=1 << 20, rounds=3, steps=500, batch=8192, lr=3e-3, seed=5,
                                                iter0=(1 << 23) + base_iter))
        cfg.proposal = 1
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(i, count=False):
        cfg.iter0 = base_iter + i * SPP
        cfg.count_traversal = 1 if count else 0
        r.clear()
        return r.render(cfg, allow_truncated=True)

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
            e0.record(stream)
            stats.append(step(args.warmup + i))
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    if dist:
        dist.barrier()
    total_ms = job_ms(float(np.sum(times)), dist, "cuda")
    paths = W * H * SPP * args.steps * ws
    value = job_value(W * H * SPP * args.steps, ws, total_ms)
    # traversal work of one step (untimed counting run) -> algorithmic bytes
    cst = step(args.warmup + args.steps, count=True)
    mean = {k: float(np.mean([s[k] for s in stats])) for k in ("ms_light", "ms_pool", "ms_recip", "ms_mlp", "ms_eye")}
    waves = stats[-1]["n_waves"]
    eye_ms, rec_ms = mean["ms_eye"] / waves, mean["ms_recip"] / waves
    eye_bytes = (64.0 * cst["eye_nodes"] + 48.0 * cst["eye_tris"]) / waves
    rec_bytes = (64.0 * cst["rec_nodes"] + 48.0 * cst["rec_tris"]) / waves
    dom = "k_eye" if eye_ms >= rec_ms else "k_recip"
    b, ms = (eye_bytes, eye_ms) if dom == "k_eye" else (rec_bytes, rec_ms)
    peak, peak_kind = peaks()
    achieved = b / (ms * 1e-3) / 1e9
    sha = src_sha(EYE_SRC if dom == "k_eye" else REC_SRC)
    # end to end through the C ABI with host buffers: scene + tables upload, render, film readback
    h2d = sum(v.nbytes for v in sc.values()) + sum(v.nbytes for v in tables.values() if isinstance(v, np.ndarray))
    d2h = W * H * 3 * 4
    e2e_t = []
    for i in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r.upload_scene(sc)
        r.upload_tables(tables)
        cfg.iter0 = base_iter + (args.warmup + args.steps + 1 + i) * SPP
        cfg.count_traversal = 0
        r.render(cfg, allow_truncated=True)
        img = r.film()
        e2e_t.append(time.perf_counter() - t0)
    e2e = W * H * SPP * ws / float(np.mean(e2e_t)) / 1e6
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    study = None
    if args.workload != "small" and args.proposal == "table" and BOOTH <= 0:
        study = equal_time_study(N, r, M_p, base_iter, total_ms / args.steps)
    cpu_v, cpu_desc, cpu_nt, cpu_px = oracle_sample(sc, M_p)
    if study is not None:
        ref = study.pop("_ref")
        npx = len(cpu_px)
        study["mape"]["cpu_oracle_1spp"] = mape(cpu_px, ref[:npx])
        study["cpu_oracle"] = {"spp": 1, "pixels": npx, "threads": cpu_nt,
                               "seconds_per_spp_full_image": W * H / (cpu_v * 1e6),
                               "note": "oracle's own learned tables; MAPE over its first %d pixels" % npx}
    out = {
        "metric": METRIC, "value": value, "unit": "Mpaths/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "M": M, "M_p": M_p, "spp": SPP, "max_depth": DEPTH,
                   "l2": "256 MiB buffer written before every timed step",
                   "tables": "learned on the device before timing (%.1f s, %d learning iterations)" % (learn_s, n_learn),
                   "stage_ms_per_step": mean, "entries_per_iteration": stats[-1]["n_entries"] / SPP,
                   "truncated_estimates_per_step": stats[-1]["n_truncated"],
                   "estimator_nodes_per_step": stats[-1]["n_nodes"], "parallelism": "replicas" if ws > 1 else "1 GPU",
                   "proposal": args.proposal, "roulette": roulette_name(),
                   "trace_stages": "persistent warps, lane refill" if TRACE else "one query per thread"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic_for(dom, sha),
                     "algorithmic_bytes_per_launch": b, "launch_ms": ms, "src_sha": sha},
        # both traversal-bound stages against the same denominator (the dominant one is "roofline")
        "roofline_stages": {
            name: {"achieved": bb / (mm * 1e-3) / 1e9, "frac": bb / (mm * 1e-3) / 1e9 / peak, "unit": "GB/s",
                   "algorithmic_bytes_per_wave": bb, "ms_per_wave": mm}
            for name, bb, mm in (("k_recip", rec_bytes, rec_ms), ("k_eye", eye_bytes, eye_ms)) if mm > 0},
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
    global W, H, SPP, M, WORKLOAD, BOOTH, TRACE
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--proposal", default="table", choices=["table", "learned"],
                    help="light-subspace proposal of the timed steps (learned: trained before timing)")
    ap.add_argument("--workload", default="projector", choices=["projector", "small", "batch", "subspace", "rr"],
                    help="small: the same scene and pipeline at 64x64, 4 spp, M=2000 (profiling captures); "
                         "batch: procedural scenes of uneven size in one graph launch; "
                         "subspace: the proxy-only selection comparison on the water scene; "
                         "rr: equal-time MAPE of the paper's RRS against Booth's roulette")
    ap.add_argument("--scenes", type=int, default=16, help="scenes of the batch workload")
    ap.add_argument("--booth", type=float, default=0.0,
                    help="Booth's Russian roulette of this scale in the reciprocal estimator (the RR ablation's "
                         "baseline; 0: the paper's RRS function)")
    ap.add_argument("--trace", type=int, default=0, choices=[0, 1],
                    help="1: the estimator's trace stages on persistent warps that refill idle lanes")
    args = ap.parse_args()
    BOOTH = max(0.0, args.booth)
    TRACE = args.trace
    if args.workload == "small":
        W, H, SPP, M = 64, 64, 4, 2000
        WORKLOAD = WORKLOAD.replace("256x256, 64 spp", "64x64, 4 spp").replace("M=10000", "M=2000")
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
