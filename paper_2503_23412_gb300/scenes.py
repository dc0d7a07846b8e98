"""Seeded synthetic inputs: procedural scenes and random subspace tables.

This module holds no rendering arithmetic. It only lays out triangles,
materials, emitter textures and cameras as flat numpy arrays, and draws
random (but valid) table inputs. Both the CUDA renderer and the CPU oracle
consume exactly these arrays, so the two see bit-identical inputs.

Scene arrays (all little-endian, C-contiguous):

  verts   float32 [nv, 3]   vertex positions
  uvs     float32 [nv, 2]   per-vertex texture coordinates (emitter texturing)
  tris    int32   [nt, 3]   vertex indices; geometric normal = (v1-v0) x (v2-v0)
  tri_mat int32   [nt]      material index per triangle
  mats    float32 [nm, 12]  material records, see MAT_* below
  tex     float32 [th, tw, 3] emission texture (row 0 is v=0)
  cam     float32 [12]      pos(3) look_at(3) up(3) vfov_deg W H

Material record layout (MAT_STRIDE floats):
  [0] kind (0 Lambert, 1 GGX conductor, 2 GGX rough dielectric)
  [1:4] colour: Lambert albedo / conductor F0 / dielectric tint (unused, 1)
  [4] roughness r (GGX alpha = r^2); a conductor or dielectric with r < 0.2
      is a specular ("S") vertex in the paper's notation (Sec. 1 footnote,
      Sec. 6.1.1 "Renderer Setting")
  [5] index of refraction (dielectric, inside medium; outside is 1)
  [6:9] emitted radiance Le (front side only; 0 = not an emitter)
  [9] 1 if Le is multiplied by the texture looked up at the surface uv
"""

from __future__ import annotations

import math

import numpy as np

MAT_STRIDE = 12
LAMBERT, CONDUCTOR, DIELECTRIC = 0, 1, 2


def material(kind, color=(0.0, 0.0, 0.0), rough=1.0, ior=1.5, Le=(0.0, 0.0, 0.0), textured=False):
    m = np.zeros(MAT_STRIDE, np.float32)
    m[0] = kind
    m[1:4] = color
    m[4] = rough
    m[5] = ior
    m[6:9] = Le
    m[9] = 1.0 if textured else 0.0
    return m


class _Builder:
    def __init__(self):
        self.verts, self.uvs, self.tris, self.tmat, self.mats = [], [], [], [], []
        self.nv = 0

    def add_material(self, m):
        self.mats.append(m)
        return len(self.mats) - 1

    def add_mesh(self, verts, tris, mat, uvs=None):
        verts = np.asarray(verts, np.float64)
        tris = np.asarray(tris, np.int64)
        if uvs is None:
            uvs = np.zeros((len(verts), 2))
        self.verts.append(verts)
        self.uvs.append(np.asarray(uvs, np.float64))
        self.tris.append(tris + self.nv)
        self.tmat.append(np.full(len(tris), mat, np.int64))
        self.nv += len(verts)

    def add_quad(self, center, eu, ev, normal, mat, uv=False):
        """Quad center +- eu +- ev, wound so its geometric normal points along `normal`."""
        c, eu, ev = (np.asarray(a, np.float64) for a in (center, eu, ev))
        p = np.array([c - eu - ev, c + eu - ev, c + eu + ev, c - eu + ev])
        uvs = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float64)
        t = np.array([[0, 1, 2], [0, 2, 3]])
        n = np.cross(p[1] - p[0], p[2] - p[0])
        if np.dot(n, normal) < 0:
            t = t[:, ::-1]
        self.add_mesh(p, t, mat, uvs if uv else None)

    def add_box(self, lo, hi, mat, inward):
        lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
        c, h = (lo + hi) / 2, (hi - lo) / 2
        s = -1.0 if inward else 1.0
        for ax in range(3):
            a1, a2 = [a for a in range(3) if a != ax]
            for sgn in (-1.0, 1.0):
                cc = c.copy()
                cc[ax] += sgn * h[ax]
                eu = np.zeros(3)
                ev = np.zeros(3)
                eu[a1] = h[a1]
                ev[a2] = h[a2]
                n = np.zeros(3)
                n[ax] = sgn * s
                self.add_quad(cc, eu, ev, n, mat)

    def build(self, tex, cam):
        return dict(
            verts=np.ascontiguousarray(np.concatenate(self.verts), np.float32),
            uvs=np.ascontiguousarray(np.concatenate(self.uvs), np.float32),
            tris=np.ascontiguousarray(np.concatenate(self.tris), np.int32),
            tri_mat=np.ascontiguousarray(np.concatenate(self.tmat), np.int32),
            mats=np.ascontiguousarray(np.stack(self.mats), np.float32),
            tex=np.ascontiguousarray(tex, np.float32),
            cam=np.asarray(cam, np.float32),
        )


def icosphere(subdiv):
    """Unit icosphere with outward winding; 20 * 4**subdiv triangles."""
    t = (1.0 + 5 ** 0.5) / 2
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    v = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            k = (min(a, b), max(a, b))
            if k not in cache:
                p = v[a] + v[b]
                v.append(p / np.linalg.norm(p))
                cache[k] = len(v) - 1
            return cache[k]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    verts = np.array(v)
    tris = np.array(f, np.int64)
    # make every triangle's winding point away from the centre
    p0, p1, p2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    flip = np.einsum("ij,ij->i", n, p0 + p1 + p2) < 0
    tris[flip] = tris[flip][:, ::-1]
    return verts, tris


def cornell(W=64, H=64, mirror_rough=0.1, glass_rough=0.1):
    """Procedural Cornell box in the unit cube, open at z=0 toward the camera.

    Five diffuse walls (albedo 0.7; left red, right green), a 0.2 x 0.2 area
    light of radiance 15 under the ceiling, a 320-triangle GGX dielectric
    sphere (IOR 1.5) and a 320-triangle GGX mirror sphere (F0 0.95), both
    radius 0.15 and roughness below the specular threshold.
    """
    b = _Builder()
    white = b.add_material(material(LAMBERT, (0.7, 0.7, 0.7)))
    red = b.add_material(material(LAMBERT, (0.7, 0.1, 0.1)))
    green = b.add_material(material(LAMBERT, (0.1, 0.7, 0.1)))
    light = b.add_material(material(LAMBERT, (0.0, 0.0, 0.0), Le=(15.0, 15.0, 15.0)))
    glass = b.add_material(material(DIELECTRIC, (1, 1, 1), rough=glass_rough, ior=1.5))
    mirror = b.add_material(material(CONDUCTOR, (0.95, 0.95, 0.95), rough=mirror_rough))
    b.add_quad((0.5, 0.0, 0.5), (0.5, 0, 0), (0, 0, 0.5), (0, 1, 0), white)   # floor
    b.add_quad((0.5, 1.0, 0.5), (0.5, 0, 0), (0, 0, 0.5), (0, -1, 0), white)  # ceiling
    b.add_quad((0.5, 0.5, 1.0), (0.5, 0, 0), (0, 0.5, 0), (0, 0, -1), white)  # back
    b.add_quad((0.0, 0.5, 0.5), (0, 0.5, 0), (0, 0, 0.5), (1, 0, 0), red)     # x=0 wall
    b.add_quad((1.0, 0.5, 0.5), (0, 0.5, 0), (0, 0, 0.5), (-1, 0, 0), green)  # x=1 wall
    b.add_quad((0.5, 0.999, 0.5), (0.1, 0, 0), (0, 0, 0.1), (0, -1, 0), light)
    sv, st = icosphere(2)
    b.add_mesh(sv * 0.15 + np.array([0.3, 0.1505, 0.35]), st, glass)
    b.add_mesh(sv * 0.15 + np.array([0.7, 0.1505, 0.65]), st, mirror)
    cam = [0.5, 0.5, -1.4, 0.5, 0.5, 0.5, 0, 1, 0, 40.0, W, H]
    return b.build(np.zeros((1, 1, 3)), cam)


def spherical_cap_lens(radius_aperture, R, z_center, rings, segs, center_xy):
    """Closed biconvex lens: two spherical caps of curvature radius R meeting at a
    rim of radius `radius_aperture` in the plane z = z_center. Outward winding."""
    h = R - math.sqrt(R * R - radius_aperture ** 2)
    verts, tris = [], []
    theta_max = math.asin(radius_aperture / R)

    def cap(sign):
        base = len(verts)
        cz = z_center - sign * (R - h)     # sphere centre on the far side
        verts.append((center_xy[0], center_xy[1], cz + sign * R))   # pole
        for i in range(1, rings + 1):
            th = theta_max * i / rings
            for j in range(segs):
                ph = 2 * math.pi * j / segs
                r = R * math.sin(th)
                verts.append((center_xy[0] + r * math.cos(ph), center_xy[1] + r * math.sin(ph),
                              cz + sign * R * math.cos(th)))
        for j in range(segs):
            tris.append((base, base + 1 + j, base + 1 + (j + 1) % segs))
        for i in range(1, rings):
            r0 = base + 1 + (i - 1) * segs
            r1 = base + 1 + i * segs
            for j in range(segs):
                a, bb = r0 + j, r0 + (j + 1) % segs
                c, d = r1 + j, r1 + (j + 1) % segs
                tris.append((a, c, d))
                tris.append((a, d, bb))
        return base

    cap(+1.0)
    cap(-1.0)
    verts = np.array(verts, np.float64)
    tris = np.array(tris, np.int64)
    # the two rims coincide geometrically (same ring of points); orient outward
    p0, p1, p2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    c = np.array([center_xy[0], center_xy[1], z_center])
    flip = np.einsum("ij,ij->i", n, (p0 + p1 + p2) / 3 - c) < 0
    tris[flip] = tris[flip][:, ::-1]
    return verts, tris


def projector(W=256, H=256, lens_tris_per_cap=10000, lens_rough=0.1, seed=2, flat=False):
    """Projector-like caustic scene.

    A 0.1 x 0.1 emitter textured with seeded 256x256 RGB noise (scale 50)
    sits in an absorbing box whose opening faces a biconvex GGX dielectric
    lens (IOR 1.5, about 2 x `lens_tris_per_cap` triangles). The lens images
    the texture onto a diffuse wall; floor and the other room surfaces are
    diffuse with albedo drawn uniformly in [0.5, 0.8]. Light paths of the
    form L S S D dominate the projected image.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    b = _Builder()
    alb = rng.uniform(0.5, 0.8, size=6)
    walls = [b.add_material(material(LAMBERT, (a, a, a))) for a in alb]
    black = b.add_material(material(LAMBERT, (0, 0, 0)))
    light = b.add_material(material(LAMBERT, (0, 0, 0), Le=(50.0, 50.0, 50.0), textured=True))
    glass = b.add_material(material(DIELECTRIC, (1, 1, 1), rough=lens_rough, ior=1.5))
    # room x in [-2,2], y in [0,3], z in [-1,5]; the projection wall is z=5
    lo, hi = np.array([-2.0, 0.0, -1.0]), np.array([2.0, 3.0, 5.0])
    c, h = (lo + hi) / 2, (hi - lo) / 2
    k = 0
    for ax in range(3):
        a1, a2 = [a for a in range(3) if a != ax]
        for sgn in (-1.0, 1.0):
            cc = c.copy()
            cc[ax] += sgn * h[ax]
            eu, ev, n = np.zeros(3), np.zeros(3), np.zeros(3)
            eu[a1], ev[a2], n[ax] = h[a1], h[a2], -sgn
            b.add_quad(cc, eu, ev, n, walls[k])
            k += 1
    # emitter at z=2.5 facing +z, centre (0, 1.2)
    ez = 2.5
    b.add_quad((0.0, 1.2, ez), (0.05, 0, 0), (0, 0.05, 0), (0, 0, 1), light, uv=True)
    # absorbing housing: back plate and four side walls, open toward +z
    hw, depth = 0.1, 0.12
    b.add_quad((0.0, 1.2, ez - 0.01), (hw, 0, 0), (0, hw, 0), (0, 0, 1), black)
    for ax, sgn in ((0, -1), (0, 1), (1, -1), (1, 1)):
        cc = np.array([0.0, 1.2, ez - 0.01 + depth / 2])
        cc[ax] += sgn * hw
        eu = np.zeros(3)
        eu[1 - ax] = hw
        ev = np.array([0.0, 0.0, depth / 2])
        n = np.zeros(3)
        n[ax] = -sgn
        b.add_quad(cc, eu, ev, n, black)
    # lens: object distance 0.5, image distance 2.0 -> f = 0.4, R = 0.4 (thin lens)
    segs = max(8, int(round(math.sqrt(lens_tris_per_cap / 2.0) * 2)))
    rings = max(2, int(round(lens_tris_per_cap / (2.0 * segs))))
    lv, lt = spherical_cap_lens(0.2, 0.4, 3.0, rings, segs, (0.0, 1.2))
    b.add_mesh(lv, lt, glass)
    tex = rng.uniform(0.0, 1.0, size=(256, 256, 3))
    if flat:   # same scene with a constant texture (isolates geometry from texture gradients)
        tex = np.full((256, 256, 3), 0.5)
    cam = [1.3, 1.5, 0.2, 0.0, 1.2, 5.0, 0, 1, 0, 45.0, W, H]
    return b.build(tex, cam)


def furnace(rho=0.5, Le=1.0, W=8, H=8, spheres=False, rough=0.1):
    """Closed unit box whose six inward-facing walls all emit Le and reflect
    with Lambert albedo rho; the camera sits inside. With no spheres every
    pixel's radiance is Le * sum_{j<K} rho^j for paths of at most K segments."""
    b = _Builder()
    wall = b.add_material(material(LAMBERT, (rho, rho, rho), Le=(Le, Le, Le)))
    b.add_box((0, 0, 0), (1, 1, 1), wall, inward=True)
    if spheres:
        glass = b.add_material(material(DIELECTRIC, (1, 1, 1), rough=rough, ior=1.5))
        sv, st = icosphere(2)
        b.add_mesh(sv * 0.12 + np.array([0.3, 0.3, 0.6]), st, glass)
    cam = [0.5, 0.5, 0.1, 0.5, 0.5, 1.0, 0, 1, 0, 60.0, W, H]
    return b.build(np.zeros((1, 1, 3)), cam)


def glossy(W=512, H=512, n_inst=2000, seed=1, n_lights=3):
    """Glossy-heavy procedural scene: `n_inst` seeded instances (half
    icospheres of 80 or 1280 triangles, four in five of them 1280, half
    boxes; about 1.05M triangles at 2,000 instances) uniformly in a 20^3 volume,
    GGX conductors with roughness log-uniform in [0.005, 0.1] on half of them
    and Lambert (albedo U[0.3, 0.8]) on the rest, `n_lights` quad lights of
    radiance log-uniform in [1, 50], inside a diffuse enclosure."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = _Builder()
    encl = b.add_material(material(LAMBERT, (0.5, 0.5, 0.5)))
    b.add_box((-1, -1, -1), (21, 21, 21), encl, inward=True)
    spheres = {s: icosphere(s) for s in (1, 2, 3)}
    for i in range(n_inst):
        if rng.uniform() < 0.5:
            m = material(CONDUCTOR, tuple(rng.uniform(0.6, 0.95, 3)),
                         rough=float(math.exp(rng.uniform(math.log(0.005), math.log(0.1)))))
        else:
            m = material(LAMBERT, tuple(rng.uniform(0.3, 0.8, 3)))
        mi = b.add_material(m)
        c = rng.uniform(0, 20, 3)
        size = rng.uniform(0.2, 0.8)
        if i % 2 == 0:
            sub = int(rng.choice([1, 3, 3, 3, 3]))
            sv, st = spheres[sub]
            b.add_mesh(sv * size + c, st, mi)
        else:
            b.add_box(c - size, c + size, mi, inward=False)
    for _ in range(n_lights):
        L = float(math.exp(rng.uniform(0.0, math.log(50.0))))
        li = b.add_material(material(LAMBERT, (0, 0, 0), Le=(L, L, L)))
        c = rng.uniform(2, 18, 3)
        c[1] = 20.9
        b.add_quad(c, (0.8, 0, 0), (0, 0, 0.8), (0, -1, 0), li)
    cam = [10.0, 10.0, -0.9, 10.0, 10.0, 10.0, 0, 1, 0, 70.0, W, H]
    return b.build(np.zeros((1, 1, 3)), cam)


def water(W=128, H=128, grid=48, depth=0.35, amp=0.015, rough=0.1, seed=3):
    """Diffuse surfaces next to a specular one, for the subspace-selection
    ablation: a 2 x 2 pool (diffuse floor albedo 0.6 at y = 0, diffuse walls
    up to y = 0.5) filled to `depth` with water, a GGX dielectric (IOR 1.33)
    heightfield of grid x grid cells whose height carries three seeded
    sinusoidal waves of amplitude `amp`. A 0.3 x 0.3 light (Le = 10) hangs at
    y = 2 off the centre, and the camera looks down into the pool at 45
    degrees. Light reaches the floor through the surface (L S D), and the
    camera sees the floor through it (D S E)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = _Builder()
    floor_m = b.add_material(material(LAMBERT, (0.6, 0.6, 0.6)))
    wall_m = b.add_material(material(LAMBERT, (0.5, 0.55, 0.6)))
    water_m = b.add_material(material(DIELECTRIC, (1, 1, 1), rough=rough, ior=1.33))
    light = b.add_material(material(LAMBERT, (0, 0, 0), Le=(10.0, 10.0, 10.0)))
    b.add_quad((0.0, 0.0, 0.0), (1.0, 0, 0), (0, 0, 1.0), (0, 1, 0), floor_m)
    for ax, sgn in ((0, -1.0), (0, 1.0), (2, -1.0), (2, 1.0)):
        c = np.array([0.0, 0.25, 0.0])
        c[ax] = sgn
        eu = np.zeros(3)
        eu[2 - ax] = 1.0
        n = np.zeros(3)
        n[ax] = -sgn
        b.add_quad(c, eu, (0, 0.25, 0), n, wall_m)
    k = rng.uniform(4.0, 9.0, (3, 2)) * rng.choice([-1.0, 1.0], (3, 2))
    ph = rng.uniform(0, 2 * np.pi, 3)
    g = np.linspace(-1.0, 1.0, grid + 1)
    X, Z = np.meshgrid(g, g, indexing="ij")
    Y = depth + amp / 3 * sum(np.sin(k[i, 0] * X + k[i, 1] * Z + ph[i]) for i in range(3))
    verts = np.stack([X, Y, Z], -1).reshape(-1, 3)
    idx = np.arange((grid + 1) ** 2).reshape(grid + 1, grid + 1)
    a0, a1 = idx[:-1, :-1].ravel(), idx[1:, :-1].ravel()
    b0, b1 = idx[:-1, 1:].ravel(), idx[1:, 1:].ravel()
    tris = np.concatenate([np.stack([a0, b0, b1], 1), np.stack([a0, b1, a1], 1)])
    v = verts[tris]
    up = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])[:, 1] > 0
    tris[~up] = tris[~up][:, ::-1]   # every surface triangle faces up (out of the water)
    b.add_mesh(verts, tris, water_m)
    b.add_quad((0.3, 2.0, 0.2), (0.15, 0, 0), (0, 0, 0.15), (0, -1, 0), light)
    cam = [0.0, 1.8, -2.4, 0.0, 0.1, 0.0, 0, 1, 0, 45.0, W, H]
    return b.build(np.zeros((1, 1, 3)), cam)


def glossy_mix(W=256, H=256, n_tris=20000, seed=1, n_lights=3, glass=0.2, ggx=0.4):
    """A scene of the batched workload: seeded instances (icospheres of
    80..1280 triangles and boxes) in a 20^3 volume until about `n_tris`
    triangles, materials glass / GGX conductor / Lambert in the ratio
    glass : ggx : rest (roughness log-uniform in [0.005, 0.1], IOR 1.5),
    `n_lights` quad lights of radiance log-uniform in [1, 50], inside a
    diffuse enclosure."""
    rng = np.random.Generator(np.random.PCG64(seed))
    b = _Builder()
    encl = b.add_material(material(LAMBERT, (0.5, 0.5, 0.5)))
    b.add_box((-1, -1, -1), (21, 21, 21), encl, inward=True)
    spheres = {s: icosphere(s) for s in (1, 2, 3)}
    tris, i = 12, 0
    while tris < n_tris:
        x = rng.uniform()
        rough = float(math.exp(rng.uniform(math.log(0.005), math.log(0.1))))
        if x < glass:
            m = material(DIELECTRIC, (1, 1, 1), rough=rough, ior=1.5)
        elif x < glass + ggx:
            m = material(CONDUCTOR, tuple(rng.uniform(0.6, 0.95, 3)), rough=rough)
        else:
            m = material(LAMBERT, tuple(rng.uniform(0.3, 0.8, 3)))
        mi = b.add_material(m)
        c = rng.uniform(0, 20, 3)
        size = rng.uniform(0.2, 0.8)
        if i % 2 == 0:
            sub = int(rng.choice([1, 2, 3, 3, 3]))
            sv, st = spheres[sub]
            b.add_mesh(sv * size + c, st, mi)
            tris += len(st)
        else:
            b.add_box(c - size, c + size, mi, inward=False)
            tris += 12
        i += 1
    for _ in range(n_lights):
        L = float(math.exp(rng.uniform(0.0, math.log(50.0))))
        li = b.add_material(material(LAMBERT, (0, 0, 0), Le=(L, L, L)))
        c = rng.uniform(2, 18, 3)
        c[1] = 20.9
        b.add_quad(c, (0.8, 0, 0), (0, 0, 0.8), (0, -1, 0), li)
    cam = [10.0, 10.0, -0.9, 10.0, 10.0, 10.0, 0, 1, 0, 70.0, W, H]
    return b.build(np.zeros((1, 1, 3)), cam)


def batch_specs(n=64, seed=1, tris=(1000, 500000), res=(128, 256, 512), spp=(16, 256)):
    """Per-scene (W, H, spp, triangles, seed) of the batched workload:
    triangle counts and spp log-uniform in the given ranges, square
    resolutions uniform over `res`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n):
        t = int(math.exp(rng.uniform(math.log(tris[0]), math.log(tris[1]))))
        r = int(rng.choice(res))
        s = int(round(math.exp(rng.uniform(math.log(spp[0]), math.log(spp[1])))))
        out.append((r, r, s, t, 1000 + k))
    return out


SCENES = {"cornell": cornell, "projector": projector, "furnace": furnace, "glossy": glossy}


# ---------------------------------------------------------------------------
# Random table inputs (valid by construction; used to drive parity tests with
# tables that neither implementation computed).

def scene_bbox(scene):
    v = scene["verts"].astype(np.float32)
    return v.min(0), v.max(0)


def _unit(rng, n):
    x = rng.normal(size=(n, 3))
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def random_tables(scene, seed=5, KT=32, KS=32, KSp=16, KC=4, tile=10, B=1.0, mis=1.0):
    """Random subspace tables: centroids (eye T, light S: pos/normal/dir 9-d;
    specular S': pos/normal 6-d; control C: pos 3-d, all in bbox-normalised
    coordinates), selection matrices with every entry >= 0.1/K, a per-tile
    proxy probability in {1.0, 0.2}, and constant B / MIS-scale tables."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W, H = int(scene["cam"][10]), int(scene["cam"][11])
    lo, hi = scene_bbox(scene)

    def cent9(K):
        return np.concatenate([rng.uniform(0, 1, (K, 3)), _unit(rng, K), _unit(rng, K)], 1)

    def gamma(K1, K2):
        g = rng.uniform(0.2, 1.0, (K1, K2))
        return g / g.sum(1, keepdims=True)

    gw, gh = (W + tile - 1) // tile, (H + tile - 1) // tile
    return dict(
        bbox_lo=lo.astype(np.float32), bbox_hi=hi.astype(np.float32),
        cent_T=cent9(KT).astype(np.float32), cent_S=cent9(KS).astype(np.float32),
        cent_Sp=np.concatenate([rng.uniform(0, 1, (KSp, 3)), _unit(rng, KSp)], 1).astype(np.float32),
        cent_C=rng.uniform(0, 1, (KC, 3)).astype(np.float32),
        gamma_conn=gamma(KT, KS).astype(np.float32),
        gamma_proxy=gamma(KT, KSp).astype(np.float32),
        B_tab=np.full((4, KSp, KC + 1), B, np.float32),
        mis_tab=np.full((4, KSp, KC + 1), mis, np.float32),
        tile=np.int32(tile),
        pi_grid=rng.choice(np.array([1.0, 0.2], np.float32), size=(gh, gw)).astype(np.float32),
    )


def pin_square_light(a=0.1, h=0.5, spec_size=1e-3, rough=0.1, dielectric=False, flip=False):
    """A square emitter (half-size a, Le=1) at height h facing down over a tiny
    GGX triangle at the origin (conductor, or dielectric of IOR 1.5) facing up
    (down with `flip`); nothing else."""
    b = _Builder()
    light = b.add_material(material(LAMBERT, (0, 0, 0), Le=(1.0, 1.0, 1.0)))
    if dielectric:
        spec = b.add_material(material(DIELECTRIC, (1, 1, 1), rough=rough, ior=1.5))
    else:
        spec = b.add_material(material(CONDUCTOR, (0.9, 0.9, 0.9), rough=rough))
    b.add_quad((0.0, h, 0.0), (a, 0, 0), (0, 0, a), (0, -1, 0), light)
    s = spec_size
    tri = np.array([[-s, 0, -s], [s, 0, -s], [0, 0, s]], np.float64)
    t = np.array([[0, 1, 2]])
    n = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    if (n[1] < 0) != flip:
        t = t[:, ::-1]
    b.add_mesh(tri, t, spec)
    cam = [0, 2, -2, 0, 0, 0, 0, 1, 0, 40.0, 4, 4]
    return b.build(np.zeros((1, 1, 3)), cam)


def pin_floor_light(a=0.1, h=1.0, floor=1.0, albedo=0.5, ypos=(0.5, 0.3, 0.0), spec_size=1e-3):
    """Square emitter (half-size a, Le=1) at height h facing down, a diffuse
    floor quad (half-size `floor`) at y=0, and a tiny GGX conductor triangle
    at `ypos` facing down toward the floor."""
    b = _Builder()
    light = b.add_material(material(LAMBERT, (0, 0, 0), Le=(1.0, 1.0, 1.0)))
    fl = b.add_material(material(LAMBERT, (albedo, albedo, albedo)))
    spec = b.add_material(material(CONDUCTOR, (0.9, 0.9, 0.9), rough=0.1))
    b.add_quad((0.0, h, 0.0), (a, 0, 0), (0, 0, a), (0, -1, 0), light)
    b.add_quad((0.0, 0.0, 0.0), (floor, 0, 0), (0, 0, floor), (0, 1, 0), fl)
    s = spec_size
    c = np.array(ypos, np.float64)
    tri = np.array([c + [-s, 0, -s], c + [s, 0, -s], c + [0, 0, s]])
    t = np.array([[0, 1, 2]])
    n = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    if n[1] > 0:
        t = t[:, ::-1]
    b.add_mesh(tri, t, spec)
    cam = [0, 2, -2, 0, 0, 0, 0, 1, 0, 40.0, 4, 4]
    return b.build(np.zeros((1, 1, 3)), cam)


def pin_mirror_light(a=0.2, h=0.5, floor=1.0, ypos=(0.35, 0.3, 0.0), rough=0.03, spec_size=1e-3):
    """Square emitter (half-size a, Le=1) at height h facing down, a GGX
    conductor floor (half-size `floor`, roughness `rough`) at y=0 facing up,
    and a tiny GGX conductor triangle at `ypos` facing down toward the floor:
    light reaches the triangle through one near-mirror bounce (L S S)."""
    b = _Builder()
    light = b.add_material(material(LAMBERT, (0, 0, 0), Le=(1.0, 1.0, 1.0)))
    mir = b.add_material(material(CONDUCTOR, (0.9, 0.9, 0.9), rough=rough))
    spec = b.add_material(material(CONDUCTOR, (0.9, 0.9, 0.9), rough=0.1))
    b.add_quad((0.0, h, 0.0), (a, 0, 0), (0, 0, a), (0, -1, 0), light)
    b.add_quad((0.0, 0.0, 0.0), (floor, 0, 0), (0, 0, floor), (0, 1, 0), mir)
    s = spec_size
    c = np.array(ypos, np.float64)
    tri = np.array([c + [-s, 0, -s], c + [s, 0, -s], c + [0, 0, s]])
    t = np.array([[0, 1, 2]])
    n = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    if n[1] > 0:
        t = t[:, ::-1]
    b.add_mesh(tri, t, spec)
    cam = [0, 2, -2, 0, 0, 0, 0, 1, 0, 40.0, 4, 4]
    return b.build(np.zeros((1, 1, 3)), cam)


def pin_lit_floor(W=12, H=12, a=0.1, h=1.0, floor=1.0, albedo=0.5, cam_pos=(0.0, 2.0, -2.0)):
    """Square emitter (half-size a, Le=1) at height h facing down over a
    diffuse floor quad (half-size `floor`, albedo) at y=0; a W x H pinhole
    camera at cam_pos looking at the origin (up +y, 40 degrees)."""
    b = _Builder()
    light = b.add_material(material(LAMBERT, (0, 0, 0), Le=(1.0, 1.0, 1.0)))
    fl = b.add_material(material(LAMBERT, (albedo, albedo, albedo)))
    b.add_quad((0.0, h, 0.0), (a, 0, 0), (0, 0, a), (0, -1, 0), light)
    b.add_quad((0.0, 0.0, 0.0), (floor, 0, 0), (0, 0, floor), (0, 1, 0), fl)
    cam = [cam_pos[0], cam_pos[1], cam_pos[2], 0, 0, 0, 0, 1, 0, 40.0, W, H]
    return b.build(np.zeros((1, 1, 3)), cam)


def pin_visible_light(W=32, H=24, vfov=40.0, x=(0.1, 0.5), y=(0.05, 0.3), z=2.0, tex=None):
    """Pinhole camera at the origin looking along +z (up +y) and one
    emitter rectangle x0..x1 by y0..y1 in the plane at depth z, facing the
    camera (Le = 1, or the texture `tex` [th][tw][3] with u along +x from x0
    and v along +y from y0); nothing else."""
    b = _Builder()
    light = b.add_material(material(LAMBERT, (0, 0, 0), Le=(1.0, 1.0, 1.0), textured=tex is not None))
    cx, cy = 0.5 * (x[0] + x[1]), 0.5 * (y[0] + y[1])
    b.add_quad((cx, cy, z), (0.5 * (x[1] - x[0]), 0, 0), (0, 0.5 * (y[1] - y[0]), 0), (0, 0, -1), light,
               uv=tex is not None)
    cam = [0, 0, 0, 0, 0, 1, 0, 1, 0, vfov, W, H]
    return b.build(np.zeros((1, 1, 3)) if tex is None else tex, cam)


def pin_two_targets(a=0.2, light_y=1.0, targets=((-0.1, 0.5), (0.1, 0.2)), half=0.03, rough=0.1):
    """A square emitter (half-size a, Le=1) at height light_y facing down,
    and two small square GGX conductors (half-size `half`) facing up at
    (x, y) = targets[i], z = 0, each wholly inside the emitter's footprint;
    nothing else. Light reaches each target directly (L S entries)."""
    b = _Builder()
    light = b.add_material(material(LAMBERT, (0, 0, 0), Le=(1.0, 1.0, 1.0)))
    spec = b.add_material(material(CONDUCTOR, (0.9, 0.9, 0.9), rough=rough))
    b.add_quad((0.0, light_y, 0.0), (a, 0, 0), (0, 0, a), (0, -1, 0), light)
    for (x, y) in targets:
        b.add_quad((x, y, 0.0), (half, 0, 0), (0, 0, half), (0, 1, 0), spec)
    cam = [0, 2, -2, 0, 0, 0, 0, 1, 0, 40.0, 4, 4]
    return b.build(np.zeros((1, 1, 3)), cam)


def pin_albedo_walls(W=24, H=24, left=0.8, right=0.2, floor=0.5, a=0.2):
    """Mirror-symmetric open box about x = 0: a diffuse floor (albedo
    `floor`) at y = 0 over [-1, 1]^2 in x, z, a left wall at x = -1 (albedo
    `left`) and a right wall at x = +1 (albedo `right`), both up to y = 1
    and facing inward, and a square emitter (half-size a, Le = 5) facing
    down at (0, 1, 0.7). The pinhole camera sits on the symmetry plane at
    (0, 3, -0.5) looking at (0, 0, -0.2) with a 24 degree field, so it sees
    only the floor."""
    b = _Builder()
    fl = b.add_material(material(LAMBERT, (floor, floor, floor)))
    lw = b.add_material(material(LAMBERT, (left, left, left)))
    rw = b.add_material(material(LAMBERT, (right, right, right)))
    light = b.add_material(material(LAMBERT, (0, 0, 0), Le=(5.0, 5.0, 5.0)))
    b.add_quad((0.0, 0.0, 0.0), (1.0, 0, 0), (0, 0, 1.0), (0, 1, 0), fl)
    b.add_quad((-1.0, 0.5, 0.0), (0, 0.5, 0), (0, 0, 1.0), (1, 0, 0), lw)
    b.add_quad((1.0, 0.5, 0.0), (0, 0.5, 0), (0, 0, 1.0), (-1, 0, 0), rw)
    b.add_quad((0.0, 1.0, 0.7), (a, 0, 0), (0, 0, a), (0, -1, 0), light)
    cam = [0.0, 3.0, -0.5, 0.0, 0.0, -0.2, 0, 0, 1, 24.0, W, H]
    return b.build(np.zeros((1, 1, 3)), cam)


def caustic_mini(W=16, H=16, rough=0.1):
    """Small open caustic scene: a 0.1 x 0.1 light above a diffuse floor and a
    tilted GGX mirror that focuses part of its light onto the floor (L S D E
    and L D S D E paths); the camera looks down at the lit floor."""
    b = _Builder()
    fl = b.add_material(material(LAMBERT, (0.7, 0.7, 0.7)))
    light = b.add_material(material(LAMBERT, (0, 0, 0), Le=(30.0, 30.0, 30.0)))
    mirror = b.add_material(material(CONDUCTOR, (0.9, 0.9, 0.9), rough=rough))
    b.add_quad((0.0, 0.0, 0.0), (1.0, 0, 0), (0, 0, 1.0), (0, 1, 0), fl)
    b.add_quad((-0.5, 1.0, 0.0), (0.05, 0, 0), (0, 0, 0.05), (0, -1, 0), light)
    n = np.array([-1.0, -1.0, 0.0]) / np.sqrt(2.0)
    eu = np.array([1.0, -1.0, 0.0]) / np.sqrt(2.0) * 0.15
    b.add_quad((0.3, 0.6, 0.0), eu, (0, 0, 0.15), n, mirror)
    cam = [0.45, 2.2, 0.01, 0.45, 0.0, 0.0, 0, 1, 0, 30.0, W, H]
    return b.build(np.zeros((1, 1, 3)), cam)
