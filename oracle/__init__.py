"""CPU oracle for proxy-tracing BDPT -- TEST INFRASTRUCTURE ONLY.

A plain FP64 C restatement of arXiv 2503.23412 (see oracle.h for the
sections it follows), loaded through ctypes. Only tests/,
__graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may use
it; the renderer in paper_2503_23412_gb300 never imports it.
"""

from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SOURCES = ["or_philox.c", "or_scene.c", "or_bsdf.c", "or_recip.c", "or_render.c", "or_mlp.c"]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (host code only; builds on x86 and Arm)."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "oracle.h"), os.path.join(HERE, "or_internal.h")]
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in deps):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


# default bound on a cell's mean estimator nodes per estimate in learning
MAX_CHAIN = 4096.0


class SceneDesc(C.Structure):
    _fields_ = [("nv", C.c_int), ("nt", C.c_int), ("nm", C.c_int),
                ("verts", C.c_void_p), ("uvs", C.c_void_p), ("tris", C.c_void_p),
                ("tri_mat", C.c_void_p), ("mats", C.c_void_p),
                ("tex_w", C.c_int), ("tex_h", C.c_int), ("tex", C.c_void_p), ("cam", C.c_void_p)]


class TablesDesc(C.Structure):
    _fields_ = [("KT", C.c_int), ("KS", C.c_int), ("KSp", C.c_int), ("KC", C.c_int),
                ("bbox_lo", C.c_void_p), ("bbox_hi", C.c_void_p),
                ("cent_T", C.c_void_p), ("cent_S", C.c_void_p), ("cent_Sp", C.c_void_p),
                ("cent_C", C.c_void_p), ("gamma_conn", C.c_void_p), ("gamma_proxy", C.c_void_p),
                ("B_tab", C.c_void_p), ("mis_tab", C.c_void_p),
                ("tile", C.c_int), ("grid_w", C.c_int), ("grid_h", C.c_int), ("pi_grid", C.c_void_p),
                ("mlp_w", C.c_void_p), ("mlp_wp", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("seed", C.c_uint32), ("max_depth", C.c_int), ("M", C.c_int), ("M_p", C.c_int),
                ("repeats", C.c_int), ("proxy", C.c_int), ("trial_cap", C.c_int), ("conn", C.c_int),
                ("pilot_min", C.c_int), ("pilot_max", C.c_int), ("side_in", C.c_double), ("booth", C.c_double),
                ("film", C.c_int), ("split_cap", C.c_int), ("fixed_bound", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n_entries", C.c_int64), ("n_truncated", C.c_int64), ("n_nodes", C.c_int64),
                ("n_conn", C.c_int64), ("n_proxy", C.c_int64), ("n_proxy_ok", C.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Entry(C.Structure):
    _fields_ = [("y_tri", C.c_int), ("y_b1", C.c_double), ("y_b2", C.c_double), ("u", C.c_int),
                ("type", C.c_int), ("h_tri", C.c_int), ("h_b1", C.c_double), ("h_b2", C.c_double),
                ("back", C.c_int), ("side_in", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        vp = C.c_void_p
        L.or_create.restype = vp
        L.or_create.argtypes = [C.POINTER(SceneDesc)]
        L.or_free.argtypes = [vp]
        L.or_uniform.restype = C.c_double
        L.or_uniform.argtypes = [C.c_uint32] * 6
        L.or_philox_block.argtypes = [vp, vp, vp]
        L.or_closest_batch.argtypes = [vp, C.c_int, vp, vp]
        L.or_occluded_batch.argtypes = [vp, C.c_int, vp, vp]
        L.or_bsdf_eval_x.argtypes = [vp, vp, vp, vp, vp]
        L.or_bsdf_pdf_x.restype = C.c_double
        L.or_bsdf_pdf_x.argtypes = [vp, vp, vp, vp]
        L.or_bsdf_sample_x.restype = C.c_int
        L.or_bsdf_sample_x.argtypes = [vp, vp, vp, C.c_double, C.c_double, C.c_double, vp]
        L.or_recip_1d.restype = C.c_int
        L.or_recip_1d.argtypes = [C.c_int, C.c_double, C.c_int, C.c_uint32, C.c_int, vp, vp, vp]
        L.or_recip_1d_booth.restype = C.c_int
        L.or_recip_1d_booth.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, C.c_uint32, C.c_int, vp, vp, vp]
        L.or_entry_fq.argtypes = [vp, C.POINTER(Entry), C.c_int, C.c_uint32, C.c_uint32, C.c_uint32, vp, vp]
        L.or_bf16.restype = C.c_double
        L.or_bf16.argtypes = [C.c_double]
        L.or_mlp_logits.restype = None
        L.or_mlp_logits.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, vp, C.c_int, vp]
        L.or_mlp_select.restype = C.c_int
        L.or_mlp_select.argtypes = [vp, C.c_int, vp, C.c_int, vp, vp, C.c_double, C.POINTER(C.c_double)]
        L.or_mlp_loss_grad.restype = C.c_double
        L.or_mlp_loss_grad.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, vp]
        L.or_mlp_adam.restype = None
        L.or_mlp_adam.argtypes = [C.c_int, vp, vp, vp, vp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_entry_pilot.restype = C.c_double
        L.or_entry_pilot.argtypes = [vp, C.POINTER(Entry), C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, C.c_int]
        L.or_entry_recip.restype = C.c_int
        L.or_entry_recip.argtypes = [vp, C.POINTER(Entry), C.c_double, C.c_int, C.c_uint32, C.c_int, vp, vp, vp]
        L.or_entry_recip_booth.restype = C.c_int
        L.or_entry_recip_booth.argtypes = [vp, C.POINTER(Entry), C.c_double, C.c_double, C.c_int, C.c_uint32,
                                           C.c_int, vp, vp, vp]
        L.or_light_pass.argtypes = [vp, C.POINTER(Params), C.c_int, vp, vp]
        L.or_iteration_estimates.restype = C.c_int
        L.or_iteration_estimates.argtypes = [vp, C.POINTER(Params), C.POINTER(TablesDesc), C.c_int, vp, vp, C.c_int,
                                             C.c_int, vp]
        L.or_iteration.argtypes = [vp, C.POINTER(Params), C.POINTER(TablesDesc), C.c_int, vp, vp, C.c_int,
                                   C.c_int, vp, vp, vp, C.c_int, vp, vp, vp, vp, C.POINTER(Stats)]
        L.or_entries.restype = C.c_int
        L.or_entries.argtypes = [vp, C.POINTER(Params), vp, vp, C.c_int, vp, vp]
        L.or_render.argtypes = [vp, C.POINTER(Params), C.POINTER(TablesDesc), C.c_int, C.c_int, C.c_int,
                                C.c_int, vp, C.POINTER(Stats)]
        L.or_set_split_default.argtypes = [C.c_int]
        L.or_set_split_default.restype = None
        L.or_set_fixed_bound_default.argtypes = [C.c_int]
        L.or_set_fixed_bound_default.restype = None
        L.or_learn.argtypes = [vp, C.POINTER(Params), C.POINTER(TablesDesc), C.c_int, C.c_int, C.c_int,
                               C.c_double, vp, vp, vp, vp, vp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Oracle:
    """Handle on one scene. Keeps the numpy inputs alive while in use."""

    def __init__(self, scene):
        self.L = lib()
        self.sc = {k: np.ascontiguousarray(v) for k, v in scene.items()}
        sc = self.sc
        tex = sc["tex"]
        self.desc = SceneDesc(len(sc["verts"]), len(sc["tris"]), len(sc["mats"]),
                              _p(sc["verts"]), _p(sc["uvs"]), _p(sc["tris"]), _p(sc["tri_mat"]),
                              _p(sc["mats"]), tex.shape[1], tex.shape[0], _p(tex), _p(sc["cam"]))
        self.h = self.L.or_create(C.byref(self.desc))
        self.W, self.H = int(sc["cam"][10]), int(sc["cam"][11])

    def close(self):
        if self.h:
            self.L.or_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- tables ---------------------------------------------------------------
    def tables(self, t):
        keep = {k: np.ascontiguousarray(v) for k, v in t.items() if isinstance(v, np.ndarray)}
        gh, gw = keep["pi_grid"].shape
        KSp, KC = keep["cent_Sp"].shape[0], keep["cent_C"].shape[0]
        d = TablesDesc(keep["cent_T"].shape[0], keep["cent_S"].shape[0], KSp, KC,
                       _p(keep["bbox_lo"]), _p(keep["bbox_hi"]), _p(keep["cent_T"]), _p(keep["cent_S"]),
                       _p(keep["cent_Sp"]), _p(keep["cent_C"]), _p(keep["gamma_conn"]),
                       _p(keep["gamma_proxy"]), _p(keep["B_tab"]), _p(keep["mis_tab"]),
                       int(t["tile"]), gw, gh, _p(keep["pi_grid"]), None, None)
        if t.get("mlp_w") is not None:
            keep["mlp_w"] = np.ascontiguousarray(t["mlp_w"], np.float64)
            d.mlp_w = _p(keep["mlp_w"])
        if t.get("mlp_wp") is not None:   # the proxy strategy's network (K = KSp)
            keep["mlp_wp"] = np.ascontiguousarray(t["mlp_wp"], np.float64)
            d.mlp_wp = _p(keep["mlp_wp"])
        d._keep = keep
        return d

    # -- queries ------------------------------------------------------------
    def closest(self, o, d, skip=None):
        n = len(o)
        rays = np.zeros((n, 7), np.float64)
        rays[:, :3], rays[:, 3:6] = o, d
        rays[:, 6] = -1 if skip is None else skip
        out = np.zeros((n, 4), np.float64)
        self.L.or_closest_batch(self.h, n, _p(rays), _p(out))
        return out

    def occluded(self, a, b, skip_a, skip_b):
        n = len(a)
        seg = np.zeros((n, 8), np.float64)
        seg[:, :3], seg[:, 3:6], seg[:, 6], seg[:, 7] = a, b, skip_a, skip_b
        out = np.zeros(n, np.int32)
        self.L.or_occluded_batch(self.h, n, _p(seg), _p(out))
        return out

    def light_pass(self, params, iteration):
        L = params.max_depth - 1
        tri = np.zeros((params.M, L), np.int32)
        bary = np.zeros((params.M, L, 2), np.float32)
        self.L.or_light_pass(self.h, C.byref(params), iteration, _p(tri), _p(bary))
        return tri, bary

    def entries(self, params, tri, bary, cap=100000):
        out = (Entry * cap)()
        li = np.zeros(cap, np.int32)
        n = self.L.or_entries(self.h, C.byref(params), _p(tri), _p(bary), cap, out, _p(li))
        return [out[i] for i in range(min(n, cap))], li[:min(n, cap)]

    def iteration(self, params, tables, iteration, tri, bary, pix_lo=0, pix_hi=None, rhat=None, cap=100000):
        pix_hi = self.W * self.H if pix_hi is None else pix_hi
        n = pix_hi - pix_lo
        rgb = np.zeros((n, 3), np.float64)
        sig = np.zeros(n, np.uint32)
        ne = C.c_int(0)
        er = np.zeros(cap, np.float64)
        es = np.zeros(cap, np.uint32)
        en = np.zeros(cap, np.float64)
        st = Stats()
        rh = None if rhat is None else np.ascontiguousarray(rhat, np.float64)
        self.L.or_iteration(self.h, C.byref(params), C.byref(tables), iteration, _p(tri), _p(bary),
                            pix_lo, pix_hi, _p(rh), _p(rgb), _p(sig), cap, C.byref(ne), _p(er), _p(es),
                            _p(en), C.byref(st))
        k = min(ne.value, cap)
        return dict(rgb=rgb, sig=sig, rhat=er[:k], entry_sig=es[:k], entry_nodes=en[:k], stats=st.as_dict())

    def iteration_estimates(self, params, tables, iteration, tri, bary, k_lo, k_hi):
        """Estimates of entries [k_lo, k_hi) of an iteration (as iteration()
        computes them) and the iteration's entry count. The C call releases
        the GIL and only reads the handle, so threads can share it."""
        out = np.zeros(max(k_hi - k_lo, 1), np.float64)
        tri = np.ascontiguousarray(tri, np.int32)
        bary = np.ascontiguousarray(bary, np.float32)
        n = self.L.or_iteration_estimates(self.h, C.byref(params), C.byref(tables), iteration, _p(tri), _p(bary),
                                          k_lo, k_hi, _p(out))
        return out[:max(0, min(k_hi, n) - k_lo)], n

    def render(self, params, tables, iter0, n_iter, pix_lo=0, pix_hi=None):
        pix_hi = self.W * self.H if pix_hi is None else pix_hi
        film = np.zeros((self.W * self.H, 3), np.float64)
        st = Stats()
        self.L.or_render(self.h, C.byref(params), C.byref(tables), iter0, n_iter, pix_lo, pix_hi,
                         _p(film), C.byref(st))
        return film, st.as_dict()

    def learn(self, params, tables_np, iter0, n_iter, n_bsamples=16, max_chain=MAX_CHAIN):
        """Learned tables (see or_learn). max_chain: cells whose learning
        estimates average more estimator nodes than this (or truncated) get
        MIS scale 0 and leave the proxy pool; 0 turns the rule off."""
        t = dict(tables_np)
        KT, KS = t["cent_T"].shape[0], t["cent_S"].shape[0]
        KSp, KC = t["cent_Sp"].shape[0], t["cent_C"].shape[0]
        B = np.zeros((4, KSp, KC + 1), np.float32)
        mis = np.zeros((4, KSp, KC + 1), np.float32)
        gc = np.zeros((KT, KS), np.float32)
        gp = np.zeros((KT, KSp), np.float32)
        pi = np.zeros_like(t["pi_grid"], np.float32)
        td = self.tables(t)
        self.L.or_learn(self.h, C.byref(params), C.byref(td), iter0, n_iter, n_bsamples, float(max_chain),
                        _p(B), _p(mis), _p(gc), _p(gp), _p(pi))
        t.update(B_tab=B, mis_tab=mis, gamma_conn=gc, gamma_proxy=gp, pi_grid=pi)
        return t

    def entry_fq(self, entry, n, seed=1, a=0, b=0):
        f = np.zeros(n, np.float64)
        q = np.zeros(n, np.float64)
        self.L.or_entry_fq(self.h, C.byref(entry), n, seed, a, b, _p(f), _p(q))
        return f, q

    def entry_pilot(self, entry, seed=1, a=0, b=0, min_draws=64, max_draws=1024):
        return self.L.or_entry_pilot(self.h, C.byref(entry), seed, a, b, min_draws, max_draws)

    def entry_recip(self, entry, B, n, seed=1, cap=1 << 16, booth=0.0):
        t = np.zeros(n, np.float64)
        i = np.zeros(n, np.float64)
        nn = np.zeros(n, np.float64)
        tr = self.L.or_entry_recip_booth(self.h, C.byref(entry), B, float(booth), n, seed, cap, _p(t), _p(i),
                                         _p(nn))
        return t, i, nn, tr


SPLIT_CAP = 1 << 16   # default node index from which the estimator stops splitting


def params(seed=7, max_depth=6, M=10000, M_p=10000, repeats=5, proxy=1, trial_cap=1 << 16, conn=1, pilot_min=64,
           pilot_max=1024, side_in=0.0, booth=0.0, film=0, split_cap=SPLIT_CAP, fixed_bound=0):
    """pilot_max = 0 turns the per-entry pilot off (B from the learned table);
    side_in = 0 is an even split of the cosine draws at dielectric vertices;
    booth > 0 estimates with Booth's Russian roulette of that scale;
    film = 1 keeps only the proxy strategy's weighted contributions in the
    pixel values, 2 all but those (the strategies and weights are unchanged);
    split_cap: from this pre-order node on, a node with |g| > 1 continues
    with one child of weight g instead of splitting (<= 0: never);
    fixed_bound = 1 keeps one B per estimate (the paper's walk), 0 lets a
    node with f/q > 2B hand its children the bound f/q (the raise rule)."""
    return Params(seed, max_depth, M, M_p, repeats, proxy, trial_cap, conn, pilot_min, pilot_max, side_in, booth,
                  film, split_cap, fixed_bound)


def philox(ctr, key):
    ctr = np.asarray(ctr, np.uint32)
    key = np.asarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox_block(_p(ctr), _p(key), _p(out))
    return out


def uniform(seed, kind, a, b, c, d):
    return lib().or_uniform(seed, kind, a, b, c, d)


# -- learned proposal (or_mlp.c) ------------------------------------------------
def mlp_nparams(K, KT):
    return 64 * 16 + 64 * 64 + 64 + 65 * K + 4 * KT


def mlp_init(K, KT, seed=0):
    """Flat weights: He-uniform hidden layers, small output layer, N(0, 0.5) embedding."""
    rng = np.random.default_rng(seed)
    w = np.zeros(mlp_nparams(K, KT))
    o = 0
    w[o:o + 1024] = rng.uniform(-1, 1, 1024) * math.sqrt(6 / 16); o += 1024
    w[o:o + 4096] = rng.uniform(-1, 1, 4096) * math.sqrt(6 / 64); o += 4096
    o += 64
    w[o:o + 64 * K] = rng.uniform(-1, 1, 64 * K) * 0.05; o += 64 * K
    o += K
    w[o:o + 4 * KT] = rng.normal(0, 0.5, 4 * KT)
    return w


def bf16(x):
    x = np.asarray(x, np.float64)
    return np.vectorize(lib().or_bf16)(x) if x.ndim else lib().or_bf16(float(x))


def mlp_logits(w, K, KT, raw, T, bf16_ops=False):
    raw = np.ascontiguousarray(raw, np.float64)
    T = np.ascontiguousarray(T, np.int32)
    n = len(T)
    z = np.zeros((n, K))
    lib().or_mlp_logits(_p(np.ascontiguousarray(w, np.float64)), K, KT, n, _p(raw), _p(T), int(bf16_ops), _p(z))
    return z


def mlp_select(w, K, raw, T, g, start, u):
    Q = C.c_double(0.0)
    S = lib().or_mlp_select(_p(np.ascontiguousarray(w, np.float64)), K, _p(np.ascontiguousarray(raw, np.float64)),
                            int(T), _p(np.ascontiguousarray(g, np.float32)), _p(np.ascontiguousarray(start, np.int32)),
                            float(u), C.byref(Q))
    return S, Q.value


def mlp_loss_grad(w, K, KT, raw, T, S, wt):
    w = np.ascontiguousarray(w, np.float64)
    g = np.zeros_like(w)
    n = len(T)
    loss = lib().or_mlp_loss_grad(_p(w), K, KT, n, _p(np.ascontiguousarray(raw, np.float64)),
                                  _p(np.ascontiguousarray(T, np.int32)), _p(np.ascontiguousarray(S, np.int32)),
                                  _p(np.ascontiguousarray(wt, np.float64)), _p(g))
    return loss, g


def mlp_adam(w, g, m1, m2, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    w, m1, m2 = (np.array(a, np.float64) for a in (w, m1, m2))
    lib().or_mlp_adam(len(w), _p(w), _p(np.ascontiguousarray(g, np.float64)), _p(m1), _p(m2), int(t), lr, beta1,
                      beta2, eps)
    return w, m1, m2


def set_split_default(split):
    """split limit of recip_1d and Oracle.entry_recip (default 2^16; <= 0: never split-limited)"""
    lib().or_set_split_default(int(split))


def set_fixed_bound_default(fixed):
    """bound rule of recip_1d and Oracle.entry_recip (default 0: the raise rule; 1: one B per estimate)"""
    lib().or_set_fixed_bound_default(int(fixed))


def recip_1d(fn, B, n, seed=1, cap=1 << 20, booth=0.0):
    """booth > 0: Booth's Russian roulette with that scale instead of the
    paper's RRS function."""
    t = np.zeros(n, np.float64)
    i = np.zeros(n, np.float64)
    nn = np.zeros(n, np.float64)
    tr = lib().or_recip_1d_booth(fn, B, float(booth), n, seed, cap, _p(t), _p(i), _p(nn))
    return t, i, nn, tr


def bsdf_eval(mat, n, wl, we):
    out = np.zeros(3, np.float64)
    m = np.ascontiguousarray(mat, np.float32)
    a = [np.ascontiguousarray(x, np.float64) for x in (n, wl, we)]
    lib().or_bsdf_eval_x(_p(m), _p(a[0]), _p(a[1]), _p(a[2]), _p(out))
    return out


def bsdf_pdf(mat, n, wg, ws):
    m = np.ascontiguousarray(mat, np.float32)
    a = [np.ascontiguousarray(x, np.float64) for x in (n, wg, ws)]
    return lib().or_bsdf_pdf_x(_p(m), _p(a[0]), _p(a[1]), _p(a[2]))


def bsdf_sample(mat, n, wg, u0, u1, u2):
    m = np.ascontiguousarray(mat, np.float32)
    a = [np.ascontiguousarray(x, np.float64) for x in (n, wg)]
    ws = np.zeros(3, np.float64)
    ok = lib().or_bsdf_sample_x(_p(m), _p(a[0]), _p(a[1]), u0, u1, u2, _p(ws))
    return ok, ws
