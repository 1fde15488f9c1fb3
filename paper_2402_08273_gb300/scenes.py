"""Seeded procedural scene generators (inputs only).

Every scene is a plain dict of numpy arrays describing an indexed triangle mesh,
its materials and a pinhole camera.  Nothing here evaluates the light-transport
method: these are the synthetic inputs that the CUDA library and the CPU oracle
both consume.  The paper's own scenes (Fireplace Room, Necklace, Living Room,
Ajar Door; Sec. 7.1) are not available, so these generators stand in for their
character: a Cornell box, two rooms joined by a narrow door gap (hard indirect
lighting through a narrow opening, like Ajar Door), a white furnace with an
analytic answer, and a glossy corridor lit through a slit.

Scene dict keys
    verts      float32 [nv, 3]   vertex positions
    tris       uint32  [nt, 3]   vertex indices per triangle
    mat_id     uint32  [nt]      material index per triangle
    mat_type   int32   [nm]      0 = Lambertian, 1 = GGX microfacet reflector
    albedo     float32 [nm, 3]   Lambert albedo, or GGX Fresnel F0
    emission   float32 [nm, 3]   radiance emitted from the front face (winding)
    roughness  float32 [nm]      GGX alpha (ignored for Lambert)
    camera     float32 [10]      pos xyz, look-at xyz, up xyz, vertical fov (deg)
"""
from __future__ import annotations

import math

import numpy as np

LAMBERT = 0
GGX = 1


class _Builder:
    def __init__(self):
        self.verts: list[np.ndarray] = []
        self.tris: list[np.ndarray] = []
        self.mat: list[np.ndarray] = []
        self.nv = 0
        self.mat_type: list[int] = []
        self.albedo: list[tuple] = []
        self.emission: list[tuple] = []
        self.rough: list[float] = []

    def material(self, mtype=LAMBERT, albedo=(0.7, 0.7, 0.7), emission=(0.0, 0.0, 0.0),
                 roughness=0.0) -> int:
        self.mat_type.append(int(mtype))
        self.albedo.append(tuple(float(a) for a in albedo))
        self.emission.append(tuple(float(e) for e in emission))
        self.rough.append(float(roughness))
        return len(self.mat_type) - 1

    def mesh(self, v: np.ndarray, t: np.ndarray, mat: int):
        v = np.asarray(v, np.float64).reshape(-1, 3)
        t = np.asarray(t, np.int64).reshape(-1, 3)
        self.verts.append(v)
        self.tris.append(t + self.nv)
        self.mat.append(np.full(len(t), mat, np.int64))
        self.nv += len(v)

    def quad(self, p0, p1, p2, p3, mat: int):
        """Quad p0 p1 p2 p3 (counter-clockwise seen from the front side)."""
        self.mesh(np.array([p0, p1, p2, p3]), np.array([[0, 1, 2], [0, 2, 3]]), mat)

    def box(self, lo, hi, mat: int, inward=False, open_faces=()):
        """Axis-aligned box; `open_faces` names faces left out ("x0", "y1", ...)."""
        x0, y0, z0 = lo
        x1, y1, z1 = hi
        c = [(x0, y0, z0), (x1, y0, z0), (x1, y1, z0), (x0, y1, z0),
             (x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)]
        # outward-facing quads (counter-clockwise seen from outside)
        faces = [("z0", (0, 3, 2, 1)),
                 ("z1", (4, 5, 6, 7)),
                 ("x0", (0, 4, 7, 3)),
                 ("x1", (1, 2, 6, 5)),
                 ("y0", (0, 1, 5, 4)),
                 ("y1", (3, 7, 6, 2))]
        for name, f in faces:
            if name in open_faces:
                continue
            q = [c[i] for i in f]
            if inward:
                q = q[::-1]
            self.quad(*q, mat)

    def build(self, camera, n_tris: int | None = None) -> dict:
        verts = np.concatenate(self.verts).astype(np.float32)
        tris = np.concatenate(self.tris)
        mat = np.concatenate(self.mat)
        if n_tris is not None:
            if len(tris) < n_tris:
                raise ValueError(f"generator produced {len(tris)} < {n_tris} triangles")
            tris = tris[:n_tris]
            mat = mat[:n_tris]
        return {
            "verts": verts,
            "tris": tris.astype(np.uint32),
            "mat_id": mat.astype(np.uint32),
            "mat_type": np.array(self.mat_type, np.int32),
            "albedo": np.array(self.albedo, np.float32).reshape(-1, 3),
            "emission": np.array(self.emission, np.float32).reshape(-1, 3),
            "roughness": np.array(self.rough, np.float32),
            "camera": np.array(camera, np.float32),
        }


def cornell_box() -> dict:
    """Cornell box in [0,1]^3, open toward the camera (z = 0 face missing).

    5 walls (10 triangles), two axis-aligned boxes (24 triangles), and a
    0.2 x 0.2 emitting quad just under the ceiling facing down (2 triangles,
    emission 17).  White albedo 0.7, red wall (0.7, 0.1, 0.1) at x = 0, green
    wall (0.1, 0.7, 0.1) at x = 1.  Camera at (0.5, 0.5, -1.2), vfov 45 deg.
    """
    b = _Builder()
    white = b.material(LAMBERT, (0.7, 0.7, 0.7))
    red = b.material(LAMBERT, (0.7, 0.1, 0.1))
    green = b.material(LAMBERT, (0.1, 0.7, 0.1))
    light = b.material(LAMBERT, (0.0, 0.0, 0.0), (17.0, 17.0, 17.0))
    b.quad((0, 0, 0), (0, 0, 1), (1, 0, 1), (1, 0, 0), white)      # floor, up
    b.quad((0, 1, 0), (1, 1, 0), (1, 1, 1), (0, 1, 1), white)      # ceiling, down
    b.quad((0, 0, 1), (0, 1, 1), (1, 1, 1), (1, 0, 1), white)      # back, -z
    b.quad((0, 0, 0), (0, 1, 0), (0, 1, 1), (0, 0, 1), red)        # left x=0, +x
    b.quad((1, 0, 0), (1, 0, 1), (1, 1, 1), (1, 1, 0), green)      # right x=1, -x
    b.box((0.53, 0.0, 0.55), (0.83, 0.6, 0.85), white)             # tall box
    b.box((0.17, 0.0, 0.15), (0.47, 0.3, 0.45), white)             # short box
    y = 0.999
    b.quad((0.4, y, 0.4), (0.6, y, 0.4), (0.6, y, 0.6), (0.4, y, 0.6), light)  # faces -y
    return b.build(camera=(0.5, 0.5, -1.2, 0.5, 0.5, 0.0, 0.0, 1.0, 0.0, 45.0))


def furnace(rho: float = 0.5, le: float = 1.0) -> dict:
    """Closed unit cube, every inner face Lambertian rho and emitting le.

    With d surface interactions and next-event estimation at each, every
    pixel's expected radiance is le * sum_{i=0..d} rho^i.  With rho = 0 every
    path contributes exactly le, so the target is constant.
    """
    b = _Builder()
    m = b.material(LAMBERT, (rho, rho, rho), (le, le, le))
    b.box((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), m, inward=True)
    return b.build(camera=(0.5, 0.5, 0.5, 0.5, 0.5, 1.0, 0.0, 1.0, 0.0, 60.0))


def furnace_uneven(rho: float = 0.5, le: float = 1.0, hub=(0.93, 0.9)) -> dict:
    """The furnace cube of furnace() with every face split into four
    triangles of very different areas: a fan from an off-centre point `hub`
    (in the face's own coordinates) to its corners.  The closed form is the
    same (le * sum_{i<=d} rho^i at every pixel), but next-event estimation
    is unbiased only if it picks a light triangle in proportion to its area.
    """
    b = _Builder()
    m = b.material(LAMBERT, (rho, rho, rho), (le, le, le))
    h0, h1 = hub
    # each face: origin o, in-face axes a1, a2, oriented so that a1 x a2 points into the cube
    faces = [((0, 0, 0), (0, 0, 1), (1, 0, 0)),   # y = 0, normal +y
             ((0, 1, 0), (1, 0, 0), (0, 0, 1)),   # y = 1, normal -y
             ((0, 0, 0), (1, 0, 0), (0, 1, 0)),   # z = 0, normal +z
             ((0, 0, 1), (0, 1, 0), (1, 0, 0)),   # z = 1, normal -z
             ((0, 0, 0), (0, 1, 0), (0, 0, 1)),   # x = 0, normal +x
             ((1, 0, 0), (0, 0, 1), (0, 1, 0))]   # x = 1, normal -x
    for o, a1, a2 in faces:
        o, a1, a2 = np.array(o, float), np.array(a1, float), np.array(a2, float)
        corners = [o, o + a1, o + a1 + a2, o + a2]
        hubp = o + h0 * a1 + h1 * a2
        v = np.array([hubp] + corners)
        t = np.array([[0, 1 + i, 1 + (i + 1) % 4] for i in range(4)])
        b.mesh(v, t, m)
    return b.build(camera=(0.5, 0.5, 0.5, 0.5, 0.5, 1.0, 0.0, 1.0, 0.0, 60.0))


def _sphere(rng, center, radius, n_seg, n_ring, jitter):
    th = np.linspace(0.0, math.pi, n_ring + 1)
    ph = np.linspace(0.0, 2.0 * math.pi, n_seg, endpoint=False)
    T, P = np.meshgrid(th[1:-1], ph, indexing="ij")
    v = np.stack([np.sin(T) * np.cos(P), np.cos(T), np.sin(T) * np.sin(P)], -1).reshape(-1, 3)
    v = np.concatenate([[[0.0, 1.0, 0.0]], v, [[0.0, -1.0, 0.0]]])
    edge = radius * 2.0 * math.pi / n_seg
    v = center + radius * v + rng.uniform(-jitter * edge, jitter * edge, v.shape)
    tris = []
    nr = n_ring - 1
    for s in range(n_seg):
        s1 = (s + 1) % n_seg
        tris.append((0, 1 + s1, 1 + s))
        for r in range(nr - 1):
            a, b_ = 1 + r * n_seg + s, 1 + r * n_seg + s1
            c, d = 1 + (r + 1) * n_seg + s, 1 + (r + 1) * n_seg + s1
            tris.append((a, b_, d))
            tris.append((a, d, c))
        last = 1 + nr * n_seg
        tris.append((1 + (nr - 1) * n_seg + s, 1 + (nr - 1) * n_seg + s1, last))
    return v, np.array(tris)


def _torus(rng, center, R, r, n_u, n_v, jitter):
    u = np.linspace(0.0, 2.0 * math.pi, n_u, endpoint=False)
    w = np.linspace(0.0, 2.0 * math.pi, n_v, endpoint=False)
    U, W = np.meshgrid(u, w, indexing="ij")
    v = np.stack([(R + r * np.cos(W)) * np.cos(U), r * np.sin(W),
                  (R + r * np.cos(W)) * np.sin(U)], -1).reshape(-1, 3)
    edge = r * 2.0 * math.pi / n_v
    v = center + v + rng.uniform(-jitter * edge, jitter * edge, v.shape)
    i, j = np.meshgrid(np.arange(n_u), np.arange(n_v), indexing="ij")
    a = i * n_v + j
    b_ = ((i + 1) % n_u) * n_v + j
    c = ((i + 1) % n_u) * n_v + (j + 1) % n_v
    d = i * n_v + (j + 1) % n_v
    t = np.concatenate([np.stack([a, b_, c], -1).reshape(-1, 3),
                        np.stack([a, c, d], -1).reshape(-1, 3)])
    return v, t


def _random_material(b: _Builder, rng) -> int:
    if rng.uniform() < 0.5:
        return b.material(LAMBERT, rng.uniform(0.2, 0.8, 3))
    return b.material(GGX, rng.uniform(0.2, 0.9, 3), roughness=rng.uniform(0.05, 0.5))


def _fill(b: _Builder, rng, n_tris_target, region_fn, size_range=(0.06, 0.3), jitter=0.2):
    """Add seeded jittered spheres and tori until n_tris_target is reached."""
    count = sum(len(t) for t in b.tris)
    while count < n_tris_target:
        center = region_fn(rng)
        mat = _random_material(b, rng)
        if rng.uniform() < 0.5:
            rad = rng.uniform(*size_range)
            n_seg = int(rng.integers(24, 72))
            n_ring = int(rng.integers(12, 36))
            v, t = _sphere(rng, center, rad, n_seg, n_ring, jitter)
        else:
            R = rng.uniform(*size_range)
            r = R * rng.uniform(0.15, 0.45)
            n_u = int(rng.integers(24, 72))
            n_v = int(rng.integers(8, 24))
            v, t = _torus(rng, center, R, r, n_u, n_v, jitter)
        b.mesh(v, t, mat)
        count += len(t)


def two_rooms(n_tris: int = 200_000, seed: int = 0) -> dict:
    """Two 4 x 2.5 x 4 m rooms joined by a 5 cm x 2 m door gap.

    The rooms share a 10 cm wall at x in [4, 4.1]; the only opening is the gap
    z in [1.975, 2.025], y in [0, 2].  A 1 x 1 m quad light (emission 60)
    hangs under the far room's ceiling, so the camera room is lit only through
    the gap.  Seeded jittered spheres and tori (50 % Lambert albedo U[0.2,0.8],
    50 % GGX roughness U[0.05,0.5]) fill both rooms up to exactly n_tris
    triangles.
    """
    rng = np.random.default_rng(seed)
    b = _Builder()
    white = b.material(LAMBERT, (0.7, 0.7, 0.7))
    wallm = b.material(LAMBERT, (0.6, 0.55, 0.5))
    light = b.material(LAMBERT, (0.0, 0.0, 0.0), (60.0, 60.0, 60.0))
    b.box((0.0, 0.0, 0.0), (8.1, 2.5, 4.0), white, inward=True)
    gz0, gz1 = 1.975, 2.025
    b.box((4.0, 0.0, 0.0), (4.1, 2.5, gz0), wallm)
    b.box((4.0, 0.0, gz1), (4.1, 2.5, 4.0), wallm)
    b.box((4.0, 2.0, gz0), (4.1, 2.5, gz1), wallm)
    y = 2.49
    b.quad((6.0, y, 1.5), (7.0, y, 1.5), (7.0, y, 2.5), (6.0, y, 2.5), light)  # faces -y
    cam = np.array([0.8, 1.4, 0.6])

    def region(rng_):
        while True:
            p = np.array([rng_.uniform(0.3, 7.8), rng_.uniform(0.2, 2.2), rng_.uniform(0.3, 3.7)])
            if 3.6 < p[0] < 4.5:
                continue
            if np.linalg.norm(p - cam) < 1.0:
                continue
            if p[0] > 5.5 and p[1] > 1.6 and 1.0 < p[2] < 3.0:
                continue  # keep the light unobstructed
            return p

    _fill(b, rng, n_tris, region)
    return b.build(camera=(0.8, 1.4, 0.6, 4.0, 1.0, 2.4, 0.0, 1.0, 0.0, 60.0), n_tris=n_tris)


def glossy_corridor(n_tris: int = 2_000_000, seed: int = 0) -> dict:
    """A 20 m glossy corridor lit through a 5 cm ceiling slit, plus a sphere.

    Corridor x in [0, 20], y in [0, 3], z in [0, 3] with GGX walls
    (roughness 0.1-0.3).  The ceiling has a slit z in [1.475, 1.525] along
    x in [2, 18]; a strong emitter above it lights the corridor only through
    the slit.  A near-specular sphere (GGX alpha 0.02) sits mid-corridor.
    Seeded jittered spheres and tori fill the corridor up to n_tris.
    """
    rng = np.random.default_rng(seed)
    b = _Builder()
    floor = b.material(GGX, (0.6, 0.6, 0.6), roughness=0.3)
    walls = b.material(GGX, (0.7, 0.65, 0.6), roughness=0.15)
    ceil = b.material(LAMBERT, (0.5, 0.5, 0.5))
    light = b.material(LAMBERT, (0.0, 0.0, 0.0), (400.0, 380.0, 340.0))
    mirror = b.material(GGX, (0.95, 0.95, 0.95), roughness=0.02)
    b.quad((0, 0, 0), (0, 0, 3), (20, 0, 3), (20, 0, 0), floor)
    b.quad((0, 0, 0), (20, 0, 0), (20, 3, 0), (0, 3, 0), walls)
    b.quad((0, 0, 3), (0, 3, 3), (20, 3, 3), (20, 0, 3), walls)
    b.quad((0, 0, 0), (0, 3, 0), (0, 3, 3), (0, 0, 3), walls)
    b.quad((20, 0, 0), (20, 0, 3), (20, 3, 3), (20, 3, 0), walls)
    s0, s1 = 1.475, 1.525
    b.box((0.0, 3.0, 0.0), (20.0, 3.1, s0), ceil)
    b.box((0.0, 3.0, s1), (20.0, 3.1, 3.0), ceil)
    b.box((0.0, 3.0, s0), (2.0, 3.1, s1), ceil)
    b.box((18.0, 3.0, s0), (20.0, 3.1, s1), ceil)
    y = 3.4
    b.quad((2.0, y, 0.5), (18.0, y, 0.5), (18.0, y, 2.5), (2.0, y, 2.5), light)  # faces -y
    # light box above the slit, open at the bottom: its light reaches the
    # corridor only through the slit in the ceiling slab below it
    b.box((0.0, 3.1, 0.0), (20.0, 3.5, 3.0), ceil, inward=True, open_faces=("y0",))
    v, t = _sphere(rng, np.array([10.0, 0.8, 1.5]), 0.8, 96, 48, 0.0)
    b.mesh(v, t, mirror)
    cam = np.array([0.6, 1.6, 1.5])

    def region(rng_):
        while True:
            p = np.array([rng_.uniform(0.5, 19.5), rng_.uniform(0.2, 2.6), rng_.uniform(0.3, 2.7)])
            if np.linalg.norm(p - cam) < 1.5:
                continue
            if np.linalg.norm(p - np.array([10.0, 0.8, 1.5])) < 1.2:
                continue
            return p

    _fill(b, rng, n_tris, region, size_range=(0.05, 0.25))
    return b.build(camera=(0.6, 1.6, 1.5, 10.0, 1.2, 1.5, 0.0, 1.0, 0.0, 55.0), n_tris=n_tris)


# A 2-D toy integrand on [0,1]^2 with known integral and region masses:
#   f(u) = base + box_height * 1[u in box] + amp * exp(-|u - mu|^2 / (2 s^2)).
# Box corners are multiples of 1/16, so the indicator is decided identically in
# binary32 and binary64.  Parameter vector layout (float64[10]):
#   base, box_height, bx0, bx1, by0, by1, amp, mu_x, mu_y, s    (10 values)
TOY_DEFAULT = np.array([1.0, 99.0, 0.625, 0.8125, 0.125, 0.3125, 50.0, 0.3, 0.7, 0.05],
                       np.float64)


def toy_region_masses(params, width, height, region_px):
    """Closed-form integral of the toy integrand over every screen region.

    Region k covers pixels [i r, min((i+1) r, W)) x [j r, min((j+1) r, H)),
    i.e. u0 in [i r / W, ...), u1 in [j r / H, ...).  Returns float64 [m].
    """
    base, bh, bx0, bx1, by0, by1, amp, mx, my, s = [float(p) for p in params]
    nx = (width + region_px - 1) // region_px
    ny = (height + region_px - 1) // region_px
    out = np.zeros(nx * ny)
    rt2s = math.sqrt(2.0) * s

    def gauss_1d(a, c, mu):
        return 0.5 * (math.erf((c - mu) / rt2s) - math.erf((a - mu) / rt2s)) * math.sqrt(2 * math.pi) * s

    for j in range(ny):
        y0 = j * region_px / height
        y1 = min((j + 1) * region_px, height) / height
        for i in range(nx):
            x0 = i * region_px / width
            x1 = min((i + 1) * region_px, width) / width
            area = (x1 - x0) * (y1 - y0)
            ox = max(0.0, min(x1, bx1) - max(x0, bx0))
            oy = max(0.0, min(y1, by1) - max(y0, by0))
            out[j * nx + i] = base * area + bh * ox * oy + amp * gauss_1d(x0, x1, mx) * gauss_1d(y0, y1, my)
    return out


def toy_rect_mass(params, x0, x1, y0, y1) -> float:
    """Closed-form integral of the toy integrand over [x0,x1) x [y0,y1)."""
    base, bh, bx0, bx1, by0, by1, amp, mx, my, s = [float(p) for p in params]
    rt2s = math.sqrt(2.0) * s

    def g1(a, c, mu):
        return 0.5 * (math.erf((c - mu) / rt2s) - math.erf((a - mu) / rt2s)) * math.sqrt(2 * math.pi) * s

    ox = max(0.0, min(x1, bx1) - max(x0, bx0))
    oy = max(0.0, min(y1, by1) - max(y0, by0))
    return base * (x1 - x0) * (y1 - y0) + bh * ox * oy + amp * g1(x0, x1, mx) * g1(y0, y1, my)


def scene_stats(scene: dict) -> dict:
    return {"n_tris": int(len(scene["tris"])), "n_verts": int(len(scene["verts"])),
            "n_mats": int(len(scene["mat_type"]))}


def batch_workload(n_scenes: int = 32, seed: int = 0, tri_range=(1_000, 500_000), chain_range=(1 << 10, 1 << 17)):
    """Seeded population of uneven problems for batched stepping: per member a
    procedural scene (two rooms or glossy corridor, alternately) with a
    triangle count log-uniform in tri_range, a square image of side 128, 256,
    512 or 1024, regions of 4, 8, 16 or 32 px, a chain count log-uniform in
    chain_range and a depth in 5..12.  Returns [(scene, chain params)]; every
    member shares epoch_len 16."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_scenes):
        n_tris = int(round(math.exp(rng.uniform(math.log(tri_range[0]), math.log(tri_range[1])))))
        side = int(rng.choice([128, 256, 512, 1024]))
        r = int(rng.choice([4, 8, 16, 32]))
        C = int(round(math.exp(rng.uniform(math.log(chain_range[0]), math.log(chain_range[1])))))
        d = int(rng.integers(5, 13))
        gen = two_rooms if i % 2 == 0 else glossy_corridor
        scene = gen(n_tris=n_tris, seed=seed * 1000 + i)
        params = dict(n_chains=C, width=side, height=side, region_px=r, max_depth=d, epoch_len=16,
                      n_bootstrap=max(1 << 16, 8 * C), p_large=0.3, seed=seed * 1000 + i + 1)
        out.append((scene, params))
    return out
