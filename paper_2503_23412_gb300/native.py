"""ctypes binding of libproxybdpt.so (include/proxybdpt.h).

Argument marshalling only: every step of the render runs in the library's
CUDA kernels. Functions keep the C names (pb_create, pb_scene_upload, ...);
`Renderer` bundles a context with the numpy arrays it was fed. Loading fails
loudly when the compiled library is missing -- there is no fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "_build", "libproxybdpt.so")

PB_OK, PB_ERR_ARG, PB_ERR_OOM, PB_ERR_CUDA, PB_ERR_TIMEOUT, PB_ERR_TRUNCATED, PB_ERR_STATE = range(7)


class pb_scene_desc(C.Structure):
    _fields_ = [("nv", C.c_int), ("nt", C.c_int), ("nm", C.c_int),
                ("verts", C.c_void_p), ("uvs", C.c_void_p), ("tris", C.c_void_p),
                ("tri_mat", C.c_void_p), ("mats", C.c_void_p),
                ("tex_w", C.c_int), ("tex_h", C.c_int), ("tex", C.c_void_p), ("cam", C.c_void_p)]


class pb_tables_desc(C.Structure):
    _fields_ = [("KT", C.c_int), ("KS", C.c_int), ("KSp", C.c_int), ("KC", C.c_int),
                ("bbox_lo", C.c_void_p), ("bbox_hi", C.c_void_p),
                ("cent_T", C.c_void_p), ("cent_S", C.c_void_p), ("cent_Sp", C.c_void_p),
                ("cent_C", C.c_void_p), ("gamma_conn", C.c_void_p), ("gamma_proxy", C.c_void_p),
                ("B_tab", C.c_void_p), ("mis_tab", C.c_void_p),
                ("tile", C.c_int), ("grid_w", C.c_int), ("grid_h", C.c_int), ("pi_grid", C.c_void_p)]


class pb_config(C.Structure):
    _fields_ = [("seed", C.c_uint32), ("spp", C.c_int), ("max_depth", C.c_int), ("M", C.c_int),
                ("M_p", C.c_int), ("repeats", C.c_int), ("proxy", C.c_int), ("conn", C.c_int),
                ("trial_cap", C.c_int), ("iter0", C.c_int), ("batch", C.c_int), ("count_traversal", C.c_int),
                ("chain_handoff", C.c_int), ("pilot_min", C.c_int), ("pilot_max", C.c_int), ("proposal", C.c_int),
                ("graph", C.c_int), ("side_in", C.c_float), ("estimator", C.c_int), ("booth", C.c_float),
                ("trace", C.c_int), ("film", C.c_int), ("split_cap", C.c_int),
                ("fixed_bound", C.c_int)]


class pb_stats(C.Structure):
    _fields_ = [("ms", C.c_double), ("mpaths_per_s", C.c_double), ("n_entries", C.c_int64),
                ("n_truncated", C.c_int64), ("n_nodes", C.c_int64), ("n_conn", C.c_int64),
                ("n_proxy", C.c_int64), ("n_proxy_ok", C.c_int64), ("ms_light", C.c_double),
                ("ms_pool", C.c_double), ("ms_recip", C.c_double), ("ms_eye", C.c_double),
                ("n_launches", C.c_int64), ("n_waves", C.c_int64), ("eye_nodes", C.c_int64),
                ("eye_tris", C.c_int64), ("eye_rays", C.c_int64), ("rec_nodes", C.c_int64),
                ("rec_tris", C.c_int64), ("rec_rays", C.c_int64), ("ms_mlp", C.c_double), ("batch_ms", C.c_double),
                ("ms_eye_feat", C.c_double), ("ms_eye_occ", C.c_double), ("cam_nodes", C.c_int64),
                ("cam_tris", C.c_int64), ("cam_rays", C.c_int64), ("shd_nodes", C.c_int64), ("shd_tris", C.c_int64),
                ("shd_rays", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pb_train_desc(C.Structure):
    _fields_ = [("samples", C.c_int), ("rounds", C.c_int), ("steps", C.c_int), ("batch", C.c_int), ("lr", C.c_float),
                ("seed", C.c_uint32), ("iter0", C.c_int), ("max_iters_per_round", C.c_int),
                ("iters_per_wave", C.c_int), ("reinit", C.c_int), ("learned_first", C.c_int), ("proxy", C.c_int)]


class pb_train_stats(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("samples", C.c_int64), ("steps", C.c_int64), ("loss_first", C.c_double),
                ("loss_last", C.c_double), ("samples_proxy", C.c_int64), ("loss_proxy_first", C.c_double),
                ("loss_proxy_last", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pb_learn_desc(C.Structure):
    _fields_ = [("KT", C.c_int), ("KS", C.c_int), ("KSp", C.c_int), ("KC", C.c_int), ("tile", C.c_int),
                ("n_iter", C.c_int), ("iter0", C.c_uint32), ("n_bsamples", C.c_int), ("lloyd_iters", C.c_int),
                ("keep_centroids", C.c_int), ("b_safety", C.c_float), ("max_chain", C.c_float)]


class pb_tables_host(C.Structure):
    _fields_ = [("KT", C.c_int), ("KS", C.c_int), ("KSp", C.c_int), ("KC", C.c_int), ("tile", C.c_int),
                ("grid_w", C.c_int), ("grid_h", C.c_int)] + [
        (n, C.c_void_p) for n in ("bbox_lo", "bbox_hi", "cent_T", "cent_S", "cent_Sp", "cent_C", "gamma_conn",
                                  "gamma_proxy", "B_tab", "mis_tab", "pi_grid")]


_lib = None

EXPORTS = ["pb_create", "pb_destroy", "pb_last_error", "pb_scene_upload", "pb_tables_upload", "pb_render",
           "pb_film_clear", "pb_film_readback", "pb_film_device", "pb_trace", "pb_occluded", "pb_light_pass",
           "pb_iteration", "pb_prepare", "pb_tables_readback", "pb_recip_estimates_noalloc", "pb_mlp_nparams",
           "pb_mlp_upload", "pb_mlp_readback", "pb_mlp_logits", "pb_mlp_grad", "pb_mlp_train_batch",
           "pb_train_proposal", "pb_connection_moments", "pb_render_batch", "pb_autotune", "pb_autotune_cache_save",
           "pb_autotune_cache_load", "pb_autotune_cache_clear", "pb_read_bandwidth", "pb_mlp_proxy_upload",
           "pb_mlp_proxy_readback"]


def lib(path=LIB):
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libproxybdpt.so is not built (%s); run paper_2503_23412_gb300.build.build()" % path)
    L = C.CDLL(path)
    vp, i32 = C.c_void_p, C.c_int
    L.pb_create.argtypes = [C.POINTER(vp), i32, vp]
    L.pb_destroy.argtypes = [vp]
    L.pb_destroy.restype = None
    L.pb_last_error.argtypes = [vp]
    L.pb_last_error.restype = C.c_char_p
    L.pb_scene_upload.argtypes = [vp, C.POINTER(pb_scene_desc)]
    L.pb_tables_upload.argtypes = [vp, C.POINTER(pb_tables_desc)]
    L.pb_render.argtypes = [vp, C.POINTER(pb_config), C.POINTER(pb_stats)]
    L.pb_film_clear.argtypes = [vp]
    L.pb_film_readback.argtypes = [vp, vp, C.c_size_t]
    L.pb_film_device.argtypes = [vp, C.POINTER(vp), C.POINTER(C.c_int64)]
    L.pb_trace.argtypes = [vp, vp, i32, vp]
    L.pb_occluded.argtypes = [vp, vp, i32, vp]
    L.pb_light_pass.argtypes = [vp, C.POINTER(pb_config), i32, vp, vp]
    L.pb_iteration.argtypes = [vp, C.POINTER(pb_config), i32, vp, vp, vp, vp, vp, i32, C.POINTER(i32), vp, vp, vp,
                               C.POINTER(pb_stats)]
    L.pb_prepare.argtypes = [vp, C.POINTER(pb_config), C.POINTER(pb_learn_desc), C.POINTER(pb_stats)]
    L.pb_tables_readback.argtypes = [vp, C.POINTER(pb_tables_host)]
    L.pb_recip_estimates_noalloc.argtypes = [vp, C.POINTER(pb_config), i32, i32, vp, vp, vp, vp, vp, vp,
                                             C.POINTER(i32)]
    L.pb_mlp_upload.argtypes = [vp, vp, C.c_size_t]
    L.pb_mlp_readback.argtypes = [vp, vp, C.c_size_t]
    L.pb_mlp_proxy_upload.argtypes = [vp, vp, C.c_size_t]
    L.pb_mlp_proxy_readback.argtypes = [vp, vp, C.c_size_t]
    L.pb_mlp_logits.argtypes = [vp, i32, vp, vp, vp]
    L.pb_mlp_grad.argtypes = [vp, i32, vp, vp, vp, vp, vp, C.POINTER(C.c_float)]
    L.pb_mlp_train_batch.argtypes = [vp, i32, vp, vp, vp, vp, C.c_float, C.POINTER(C.c_float)]
    L.pb_train_proposal.argtypes = [vp, C.POINTER(pb_config), C.POINTER(pb_train_desc), C.POINTER(pb_train_stats)]
    L.pb_connection_moments.argtypes = [vp, C.POINTER(pb_config), vp]
    L.pb_render_batch.argtypes = [vp, vp, i32, vp]
    L.pb_autotune.argtypes = [vp, C.POINTER(pb_config), i32, C.POINTER(pb_config), C.POINTER(i32)]
    L.pb_autotune_cache_save.argtypes = [C.c_char_p]
    L.pb_autotune_cache_load.argtypes = [C.c_char_p]
    L.pb_autotune_cache_clear.argtypes = []
    L.pb_read_bandwidth.argtypes = [i32, C.c_size_t, i32, C.POINTER(C.c_double)]
    for n in EXPORTS:
        if n not in ("pb_destroy", "pb_last_error", "pb_autotune_cache_clear"):
            getattr(L, n).restype = i32
    L.pb_autotune_cache_clear.restype = None
    L.pb_mlp_nparams.argtypes = [i32, i32]
    L.pb_mlp_nparams.restype = C.c_size_t
    _lib = L
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class PBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("proxybdpt status %d: %s" % (status, msg))
        self.status = status


def config(seed=7, spp=1, max_depth=6, M=10000, M_p=10000, repeats=5, proxy=1, conn=1, trial_cap=1 << 16, iter0=0,
           batch=0, count_traversal=0, chain_handoff=0, pilot_min=0, pilot_max=0, proposal=0, graph=0, side_in=0.0,
           estimator=0, booth=0.0, trace=0, film=0, split_cap=0, fixed_bound=0):
    """booth > 0: Booth's Russian roulette of that scale in the reciprocal
    estimator (wavefront schedule only); 0: the paper's RRS function.
    trace = 1: the wavefront's trace stages run on persistent warps that
    refill idle lanes (same answers). film = 1 keeps only the proxy
    strategy's weighted contributions in the film, 2 all but those.
    split_cap: the estimator's split limit (0: node 65536; negative: never).
    fixed_bound = 1: one B per estimate (the paper's walk); 0: a node with
    f/q > 2B hands its children the bound f/q (the raise rule)."""
    return pb_config(seed, spp, max_depth, M, M_p, repeats, proxy, conn, trial_cap, iter0, batch, count_traversal,
                     chain_handoff, pilot_min, pilot_max, proposal, graph, side_in, estimator, booth, trace, film,
                     split_cap, fixed_bound)


def render_batch(renderers, cfgs, allow_truncated=False):
    """One graph launch rendering every scene (see pb_render_batch); returns per-scene stats."""
    L = lib()
    n = len(renderers)
    hs = (C.c_void_p * n)(*[r.h for r in renderers])
    cs = (pb_config * n)(*cfgs)
    st = (pb_stats * n)()
    rc = L.pb_render_batch(hs, cs, n, st)
    ok = (PB_OK, PB_ERR_TRUNCATED) if allow_truncated else (PB_OK,)
    if rc not in ok:
        raise PBError(rc, L.pb_last_error(renderers[0].h).decode())
    return [s.as_dict() for s in st]


def autotune_cache_save(path):
    if lib().pb_autotune_cache_save(path.encode()) != PB_OK:
        raise PBError(PB_ERR_ARG, "cannot write " + path)


def autotune_cache_load(path):
    if lib().pb_autotune_cache_load(path.encode()) != PB_OK:
        raise PBError(PB_ERR_ARG, "cannot read " + path)


def autotune_cache_clear():
    lib().pb_autotune_cache_clear()


def read_bandwidth(device, nbytes, reps):
    """Read rate in GB/s of a buffer of nbytes read reps times (see pb_read_bandwidth)."""
    g = C.c_double(0.0)
    rc = lib().pb_read_bandwidth(device, nbytes, reps, C.byref(g))
    if rc != PB_OK:
        raise PBError(rc, "pb_read_bandwidth failed")
    return g.value


def train_desc(samples=1 << 20, rounds=2, steps=400, batch=4096, lr=1e-3, seed=1, iter0=1 << 23, max_iters_per_round=0,
               iters_per_wave=0, reinit=0, learned_first=0, proxy=0):
    """proxy = 1 also trains the proxy strategy's network (render with proposal = 2)."""
    return pb_train_desc(samples, rounds, steps, batch, lr, seed, iter0, max_iters_per_round, iters_per_wave, reinit,
                         learned_first, proxy)


def tables_desc(t, W, H):
    keep = {k: np.ascontiguousarray(v, np.float32) for k, v in t.items() if isinstance(v, np.ndarray)}
    tile = int(t["tile"])
    gh, gw = keep["pi_grid"].shape
    d = pb_tables_desc(keep["cent_T"].shape[0], keep["cent_S"].shape[0], keep["cent_Sp"].shape[0],
                       keep["cent_C"].shape[0], _p(keep["bbox_lo"]), _p(keep["bbox_hi"]), _p(keep["cent_T"]),
                       _p(keep["cent_S"]), _p(keep["cent_Sp"]), _p(keep["cent_C"]), _p(keep["gamma_conn"]),
                       _p(keep["gamma_proxy"]), _p(keep["B_tab"]), _p(keep["mis_tab"]), tile, gw, gh,
                       _p(keep["pi_grid"]))
    d._keep = keep
    return d


class Renderer:
    """One renderer context on one device with a scene and tables."""

    def __init__(self, scene, tables=None, device=0, stream=None):
        self.L = lib()
        self.h = C.c_void_p()
        st = self.L.pb_create(C.byref(self.h), device, stream)
        if st != PB_OK:
            raise PBError(st, "pb_create failed")
        self.W, self.H = int(scene["cam"][10]), int(scene["cam"][11])
        self.upload_scene(scene)
        if tables is not None:
            self.upload_tables(tables)

    def _check(self, st, ok=(PB_OK,)):
        if st not in ok:
            raise PBError(st, self.L.pb_last_error(self.h).decode())
        return st

    def upload_scene(self, scene):
        sc = {k: np.ascontiguousarray(v) for k, v in scene.items()}
        tex = sc["tex"]
        d = pb_scene_desc(len(sc["verts"]), len(sc["tris"]), len(sc["mats"]), _p(sc["verts"]), _p(sc["uvs"]),
                          _p(sc["tris"]), _p(sc["tri_mat"]), _p(sc["mats"]), tex.shape[1], tex.shape[0], _p(tex),
                          _p(sc["cam"]))
        self._check(self.L.pb_scene_upload(self.h, C.byref(d)))
        self.scene = sc

    def upload_tables(self, t):
        d = tables_desc(t, self.W, self.H)
        self._check(self.L.pb_tables_upload(self.h, C.byref(d)))
        self.tables = t

    def prepare(self, cfg, n_iter=8, iter0=1 << 20, n_bsamples=32, lloyd_iters=8, keep_centroids=False,
                KT=300, KS=300, KSp=100, KC=10, tile=10, b_safety=0.0, max_chain=0.0):
        """Learns the subspace tables on the device (see pb_prepare)."""
        d = pb_learn_desc(KT, KS, KSp, KC, tile, n_iter, iter0, n_bsamples, lloyd_iters, 1 if keep_centroids else 0,
                          b_safety, max_chain)
        st = pb_stats()
        self._check(self.L.pb_prepare(self.h, C.byref(cfg), C.byref(d), C.byref(st)))
        return st.as_dict()

    def tables_readback(self):
        t = pb_tables_host()
        self._check(self.L.pb_tables_readback(self.h, C.byref(t)))
        out = dict(bbox_lo=np.zeros(3, np.float32), bbox_hi=np.zeros(3, np.float32),
                   cent_T=np.zeros((t.KT, 9), np.float32), cent_S=np.zeros((t.KS, 9), np.float32),
                   cent_Sp=np.zeros((t.KSp, 6), np.float32), cent_C=np.zeros((t.KC, 3), np.float32),
                   gamma_conn=np.zeros((t.KT, t.KS), np.float32), gamma_proxy=np.zeros((t.KT, t.KSp), np.float32),
                   B_tab=np.zeros((4, t.KSp, t.KC + 1), np.float32), mis_tab=np.zeros((4, t.KSp, t.KC + 1), np.float32),
                   pi_grid=np.zeros((t.grid_h, t.grid_w), np.float32))
        for k, v in out.items():
            setattr(t, k, v.ctypes.data)
        self._check(self.L.pb_tables_readback(self.h, C.byref(t)))
        out["tile"] = np.int32(t.tile)
        return out

    def render(self, cfg, allow_truncated=False):
        st = pb_stats()
        ok = (PB_OK, PB_ERR_TRUNCATED) if allow_truncated else (PB_OK,)
        self._check(self.L.pb_render(self.h, C.byref(cfg), C.byref(st)), ok)
        return st.as_dict()

    def clear(self):
        self._check(self.L.pb_film_clear(self.h))

    def film(self):
        out = np.zeros((self.H * self.W, 3), np.float32)
        self._check(self.L.pb_film_readback(self.h, _p(out), out.size))
        return out

    def film_device(self):
        p = C.c_void_p()
        n = C.c_int64()
        self._check(self.L.pb_film_device(self.h, C.byref(p), C.byref(n)))
        return p.value, n.value

    def trace(self, o, d, skip=None):
        n = len(o)
        rays = np.zeros((n, 7), np.float32)
        rays[:, :3], rays[:, 3:6] = o, d
        rays[:, 6] = -1 if skip is None else skip
        hits = np.zeros((n, 4), np.float32)
        self._check(self.L.pb_trace(self.h, _p(rays), n, _p(hits)))
        return hits

    def occluded(self, a, b, skip_a, skip_b):
        n = len(a)
        seg = np.zeros((n, 8), np.float32)
        seg[:, :3], seg[:, 3:6], seg[:, 6], seg[:, 7] = a, b, skip_a, skip_b
        out = np.zeros(n, np.int32)
        self._check(self.L.pb_occluded(self.h, _p(seg), n, _p(out)))
        return out

    def light_pass(self, cfg, iteration):
        Lv = cfg.max_depth - 1
        tri = np.zeros((cfg.M, Lv), np.int32)
        bary = np.zeros((cfg.M, Lv, 2), np.float32)
        self._check(self.L.pb_light_pass(self.h, C.byref(cfg), iteration, _p(tri), _p(bary)))
        return tri, bary

    def iteration(self, cfg, iteration, tri, bary, rhat=None, cap=100000):
        tri = np.ascontiguousarray(tri, np.int32)
        bary = np.ascontiguousarray(bary, np.float32)
        rgb = np.zeros((self.W * self.H, 3), np.float32)
        sig = np.zeros(self.W * self.H, np.uint32)
        ne = C.c_int(0)
        er = np.zeros(cap, np.float32)
        es = np.zeros(cap, np.uint32)
        en = np.zeros(cap, np.float32)
        st = pb_stats()
        rh = None
        if rhat is not None:
            rh = np.zeros(cfg.M * (cfg.max_depth - 1), np.float64)
            rh[:len(rhat)] = rhat
        self._check(self.L.pb_iteration(self.h, C.byref(cfg), iteration, _p(tri), _p(bary), _p(rh), _p(rgb),
                                        _p(sig), cap, C.byref(ne), _p(er), _p(es), _p(en), C.byref(st)))
        k = min(ne.value, cap)
        return dict(rgb=rgb, sig=sig, rhat=er[:k], entry_sig=es[:k], entry_nodes=en[:k], stats=st.as_dict())

    def recip_estimates_noalloc(self, cfg, iteration, n, d_tri, d_bary, d_info, d_B, d_rhat, d_nodes=None):
        """Allocation-free reciprocal estimates on caller device buffers (raw
        device addresses); returns the number of truncated entries."""
        ntr = C.c_int(0)
        self._check(self.L.pb_recip_estimates_noalloc(self.h, C.byref(cfg), iteration, n, d_tri, d_bary, d_info, d_B,
                                                      d_rhat, d_nodes, C.byref(ntr)))
        return ntr.value

    # -- learned proposal ---------------------------------------------------------
    def _table_dims(self):
        t = pb_tables_host()
        self._check(self.L.pb_tables_readback(self.h, C.byref(t)))   # null arrays: sizes only
        return t.KS, t.KT

    @property
    def KS(self):
        return self._table_dims()[0]

    @property
    def KT(self):
        return self._table_dims()[1]

    def mlp_nparams(self):
        return int(self.L.pb_mlp_nparams(self.KS, self.KT))

    def mlp_upload(self, w):
        w = np.ascontiguousarray(w, np.float32)
        self._check(self.L.pb_mlp_upload(self.h, _p(w), w.size))

    def mlp_proxy_nparams(self):
        t = pb_tables_host()
        self._check(self.L.pb_tables_readback(self.h, C.byref(t)))
        return int(self.L.pb_mlp_nparams(t.KSp, t.KT))

    def mlp_proxy_upload(self, w):
        w = np.ascontiguousarray(w, np.float32)
        self._check(self.L.pb_mlp_proxy_upload(self.h, _p(w), w.size))

    def mlp_proxy_readback(self):
        w = np.zeros(self.mlp_proxy_nparams(), np.float32)
        self._check(self.L.pb_mlp_proxy_readback(self.h, _p(w), w.size))
        return w

    def mlp_readback(self):
        w = np.zeros(self.mlp_nparams(), np.float32)
        self._check(self.L.pb_mlp_readback(self.h, _p(w), w.size))
        return w

    def mlp_logits(self, raw, T):
        raw = np.ascontiguousarray(raw, np.float32)
        T = np.ascontiguousarray(T, np.int32)
        z = np.zeros((len(T), self.KS), np.float32)
        self._check(self.L.pb_mlp_logits(self.h, len(T), _p(raw), _p(T), _p(z)))
        return z

    def mlp_grad(self, raw, T, S, w):
        raw, w = (np.ascontiguousarray(a, np.float32) for a in (raw, w))
        T, S = (np.ascontiguousarray(a, np.int32) for a in (T, S))
        g = np.zeros(self.mlp_nparams(), np.float32)
        loss = C.c_float(0.0)
        self._check(self.L.pb_mlp_grad(self.h, len(T), _p(raw), _p(T), _p(S), _p(w), _p(g), C.byref(loss)))
        return loss.value, g

    def mlp_train_batch(self, raw, T, S, w, lr):
        raw, w = (np.ascontiguousarray(a, np.float32) for a in (raw, w))
        T, S = (np.ascontiguousarray(a, np.int32) for a in (T, S))
        loss = C.c_float(0.0)
        self._check(self.L.pb_mlp_train_batch(self.h, len(T), _p(raw), _p(T), _p(S), _p(w), lr, C.byref(loss)))
        return loss.value

    def autotune(self, cfg, trial_iters=32):
        best = pb_config()
        fc = C.c_int(0)
        self._check(self.L.pb_autotune(self.h, C.byref(cfg), trial_iters, C.byref(best), C.byref(fc)))
        return best, bool(fc.value)

    def connection_moments(self, cfg):
        out = np.zeros(3)
        self._check(self.L.pb_connection_moments(self.h, C.byref(cfg), _p(out)))
        n, s1, s2 = out
        return dict(n=n, mean=s1 / max(n, 1), m2=s2 / max(n, 1), relvar=(s2 / max(n, 1)) / max((s1 / max(n, 1)) ** 2, 1e-300) - 1)

    def train_proposal(self, cfg, td):
        st = pb_train_stats()
        self._check(self.L.pb_train_proposal(self.h, C.byref(cfg), C.byref(td), C.byref(st)))
        return st.as_dict()

    def close(self):
        if self.h:
            self.L.pb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
