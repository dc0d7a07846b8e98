"""The oracle's ranged estimate entry point (used to time the oracle on all
host cores) returns exactly the estimates of a whole iteration, also when
threads share the handle."""

from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle as O
from paper_2503_23412_gb300 import scenes


def test_ranged_estimates_equal_the_iteration_on_threads():
    sc = scenes.projector(16, 16, lens_tris_per_cap=400, flat=True)
    o = O.Oracle(sc)
    tab = scenes.random_tables(sc, KT=8, KS=8, KSp=4, KC=2)
    tab = o.learn(O.params(M=600, M_p=600, max_depth=6), tab, 1000, 1, n_bsamples=16)
    td = o.tables(tab)
    for booth in (0.0, 30.0):
        p = O.params(M=600, M_p=600, max_depth=6, booth=booth)
        tri, bary = o.light_pass(p, 3)
        whole = o.iteration(p, td, 3, tri, bary, pix_lo=0, pix_hi=0)["rhat"]
        n = len(whole)
        assert n > 20
        ranges = [(n * i // 7, n * (i + 1) // 7) for i in range(7)]
        with ThreadPoolExecutor(4) as ex:
            parts = list(ex.map(lambda kr: o.iteration_estimates(p, td, 3, tri, bary, kr[0], kr[1]), ranges))
        assert all(cnt == n for _, cnt in parts)
        np.testing.assert_array_equal(np.concatenate([v for v, _ in parts]), whole)
        # a range past the end is clipped
        v, cnt = o.iteration_estimates(p, td, 3, tri, bary, n - 2, n + 5)
        np.testing.assert_array_equal(v, whole[n - 2:])


def test_water_scene_has_diffuse_next_to_specular():
    """The subspace-selection ablation's scene: the water surface faces up,
    lies between the pool floor and the light, and the light's paths leave
    incomplete sub-paths ending on it (mostly L S, u = 1)."""
    sc = scenes.water(16, 16)
    V, T, mats = sc["verts"].astype(np.float64), sc["tris"], sc["mats"]
    water = np.where(mats[sc["tri_mat"], 0] == 2)[0]
    assert len(water) == 2 * 48 * 48
    v = V[T[water]]
    n = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    assert np.all(n[:, 1] > 0)
    assert 0.3 < v[..., 1].min() and v[..., 1].max() < 0.4
    o = O.Oracle(sc)
    p = O.params(M=2000, M_p=2000, max_depth=6)
    tri, bary = o.light_pass(p, 1)
    ents, _ = o.entries(p, tri, bary)
    u = np.array([e.u for e in ents])
    assert len(ents) > 100 and (u == 1).mean() > 0.9 and u.min() >= 1
    assert all(mats[sc["tri_mat"][e.y_tri], 0] == 2 for e in ents)
