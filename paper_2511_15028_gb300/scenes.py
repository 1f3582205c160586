"""Seeded synthetic scenes and ray batches.

This module is the only code shared by the CUDA path, its tests and the CPU
oracle. It holds input synthesis only (geometry, cameras, random rays); none of
the traversal, intersection or layout arithmetic lives here.

The paper's evaluation scenes (Section 9.1: lucy, power-plant, san-miguel,
sheep, hairball, sponza, white-oak; 36.8K to 28M triangles) are not available,
so these generators stand in for them with the same triangle-count range and
the paper's primary (coherent camera) versus secondary (incoherent) ray split
(Section 9.2.1).

Conventions
-----------
* vertices: float32 ``[n_verts, 3]``; indices: uint32 ``[n_tris, 3]`` or None
  for a triangle soup (triangle ``i`` = vertices ``3i, 3i+1, 3i+2``).
* rays: float32 ``[n, 8]`` = ``(ox, oy, oz, tmin, dx, dy, dz, tmax)``.
* hits (where a generator consumes them): float32 ``t, u, v`` and uint32
  ``prim``; ``u`` weights ``p1`` and ``v`` weights ``p2``.
* every generator takes an explicit seed and draws from numpy's PCG64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MISS = 0xFFFFFFFF
TMIN = 1e-4


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Scene:
    verts: np.ndarray                 # float32 [n_verts, 3]
    indices: np.ndarray | None        # uint32 [n_tris, 3] or None (soup)
    name: str = ""

    @property
    def n_tris(self) -> int:
        if self.indices is not None:
            return int(self.indices.shape[0])
        return int(self.verts.shape[0] // 3)

    def triangles(self) -> np.ndarray:
        """float32 [n_tris, 9]: p0, p1, p2 of every triangle in id order."""
        if self.indices is None:
            return np.ascontiguousarray(self.verts.reshape(-1, 9))
        return np.ascontiguousarray(self.verts[self.indices].reshape(-1, 9))


def make_rays(o: np.ndarray, d: np.ndarray, tmin, tmax) -> np.ndarray:
    n = o.shape[0]
    r = np.empty((n, 8), dtype=np.float32)
    r[:, 0:3] = o
    r[:, 3] = tmin
    r[:, 4:7] = d
    r[:, 7] = tmax
    return r


# ---------------------------------------------------------------- cameras


def _normalize(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def pinhole_rays(eye, target, up, vfov_deg: float, width: int, height: int,
                 tmin: float = TMIN, tmax: float = np.inf) -> np.ndarray:
    """Pinhole camera through pixel centres, row-major (row 0 at the top).

    Directions are built and normalised in float64, then rounded to float32.
    """
    eye = np.asarray(eye, np.float64)
    f = _normalize(np.asarray(target, np.float64) - eye)
    r = _normalize(np.cross(f, np.asarray(up, np.float64)))
    u = np.cross(r, f)
    th = math.tan(math.radians(vfov_deg) / 2)
    aspect = width / height
    sx = ((np.arange(width) + 0.5) / width * 2 - 1) * th * aspect
    sy = (1 - (np.arange(height) + 0.5) / height * 2) * th
    SX, SY = np.meshgrid(sx, sy)
    d = f[None, :] + SX.reshape(-1, 1) * r[None, :] + SY.reshape(-1, 1) * u[None, :]
    d = _normalize(d)
    o = np.broadcast_to(eye, d.shape)
    return make_rays(o.astype(np.float32), d.astype(np.float32), tmin, tmax)


# ---------------------------------------------------------------- meshes


def grid_mesh(zfun, nqx: int, nqy: int, x0=-1.0, x1=1.0, y0=-1.0, y1=1.0):
    """Height field over a (nqx+1) x (nqy+1) vertex grid.

    Quad (i, j) gives triangles (v00, v10, v11) and (v00, v11, v01) with ids
    2*(j*nqx + i) + k.
    """
    nvx, nvy = nqx + 1, nqy + 1
    xs = np.linspace(x0, x1, nvx)
    ys = np.linspace(y0, y1, nvy)
    X, Y = np.meshgrid(xs, ys)
    Z = zfun(X, Y)
    verts = np.stack([X, Y, Z], -1).reshape(-1, 3).astype(np.float32)
    ii, jj = np.meshgrid(np.arange(nqx, dtype=np.int64), np.arange(nqy, dtype=np.int64))
    v00 = jj * nvx + ii
    v10 = v00 + 1
    v01 = v00 + nvx
    v11 = v01 + 1
    t0 = np.stack([v00, v10, v11], -1)
    t1 = np.stack([v00, v11, v01], -1)
    idx = np.stack([t0, t1], axis=2).reshape(-1, 3).astype(np.uint32)
    return verts, idx


def value_noise_fbm(X, Y, rng, octaves=6, lacunarity=2, gain=0.5,
                    amplitude=0.25, base_res=4):
    """Fractal sum of value-noise octaves over [-1, 1]^2 (smoothstep-bilinear
    interpolation of a seeded lattice per octave)."""
    z = np.zeros_like(X)
    amp = 1.0
    res = base_res
    for _ in range(octaves):
        table = rng.uniform(-1.0, 1.0, size=(res + 1, res + 1))
        gx = (X + 1) * 0.5 * res
        gy = (Y + 1) * 0.5 * res
        i0 = np.clip(np.floor(gx).astype(np.int64), 0, res - 1)
        j0 = np.clip(np.floor(gy).astype(np.int64), 0, res - 1)
        fx = gx - i0
        fy = gy - j0
        sx = fx * fx * (3 - 2 * fx)
        sy = fy * fy * (3 - 2 * fy)
        a = table[j0, i0]
        b = table[j0, i0 + 1]
        c = table[j0 + 1, i0]
        d = table[j0 + 1, i0 + 1]
        z += amp * ((a * (1 - sx) + b * sx) * (1 - sy) + (c * (1 - sx) + d * sx) * sy)
        amp *= gain
        res *= lacunarity
    return amplitude * z


def icosphere(subdiv: int):
    """Unit icosphere: 20 * 4**subdiv triangles, vertices on the unit sphere."""
    p = (1 + 5 ** 0.5) / 2
    v = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
         (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
         (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    verts = [np.array(x, np.float64) / np.linalg.norm(x) for x in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts, np.float64), np.array(faces, np.int64)


def random_rotations(rng, n):
    """n uniformly random rotation matrices (from normalised Gaussian quaternions)."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def random_soup(rng, n: int, mu=math.log(0.002), sigma=0.5, lo=0.0, hi=1.0,
                chunk=1 << 20) -> np.ndarray:
    """n equilateral triangles: centroids uniform in [lo, hi]^3, edge length
    log-normal(mu, sigma), uniformly random orientation. float32 [3n, 3]."""
    out = np.empty((n, 3, 3), np.float32)
    ang = np.array([0.0, 2 * math.pi / 3, 4 * math.pi / 3])
    unit = np.stack([np.cos(ang), np.sin(ang), np.zeros(3)], -1)  # circumradius 1
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        c = rng.uniform(lo, hi, size=(m, 3))
        edge = rng.lognormal(mu, sigma, size=m)
        R = random_rotations(rng, m)
        local = unit[None, :, :] * (edge / math.sqrt(3))[:, None, None]
        out[s:s + m] = (c[:, None, :] + np.einsum('nij,nkj->nki', R, local)).astype(np.float32)
    return out.reshape(-1, 3)


def random_rays(rng, n: int, lo, hi, tmin=TMIN, tmax=np.inf) -> np.ndarray:
    """Origins uniform in the box [lo, hi], directions uniform on the sphere."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    o = lo + (hi - lo) * rng.uniform(size=(n, 3))
    d = _normalize(rng.normal(size=(n, 3)))
    return make_rays(o.astype(np.float32), d.astype(np.float32), tmin, tmax)


# ---------------------------------------------------------------- workloads


def config1_scene(seed: int = 1001) -> Scene:
    """64 x 32 quad grid over [-1,1]^2, z = 0.2 sin(3x) cos(2y) + U(+-0.01):
    4,096 triangles (indexed)."""
    rng = rng_for(seed)
    verts, idx = grid_mesh(
        lambda X, Y: 0.2 * np.sin(3 * X) * np.cos(2 * Y) + rng.uniform(-0.01, 0.01, X.shape),
        64, 32)
    return Scene(verts, idx, "grid64x32")


def config1_rays() -> np.ndarray:
    """128 x 128 pinhole rays, eye (0,0,3) looking at the origin, 60 deg FOV."""
    return pinhole_rays((0, 0, 3), (0, 0, 0), (0, 1, 0), 60.0, 128, 128)


def config2_scene(seed: int = 1002, side: int = 724, n_spheres: int = 256) -> Scene:
    """fBm value-noise height field with side x side vertices over [-1,1]^2
    plus n_spheres subdivision-3 icospheres (1,280 triangles each); indexed."""
    rng = rng_for(seed)
    hv, hi = grid_mesh(lambda X, Y: value_noise_fbm(X, Y, rng), side - 1, side - 1)
    sv, sf = icosphere(3)
    cx = rng.uniform(-1, 1, n_spheres)
    cy = rng.uniform(-1, 1, n_spheres)
    cz = rng.uniform(0, 0.5, n_spheres)
    rad = np.exp(rng.uniform(math.log(0.005), math.log(0.05), n_spheres))
    vs = [hv]
    fs = [hi.astype(np.int64)]
    base = hv.shape[0]
    for k in range(n_spheres):
        vs.append((sv * rad[k] + np.array([cx[k], cy[k], cz[k]])).astype(np.float32))
        fs.append(sf + base)
        base += sv.shape[0]
    return Scene(np.concatenate(vs).astype(np.float32),
                 np.concatenate(fs).astype(np.uint32), "fbm724+256spheres")


CONFIG2_EYE = (0.0, -2.2, 1.4)
CONFIG2_LIGHT = (2.0, 2.0, 3.0)


def config2_primary(width: int = 1920, height: int = 1080) -> np.ndarray:
    return pinhole_rays(CONFIG2_EYE, (0, 0, 0), (0, 0, 1), 45.0, width, height)


def _hit_frame(scene: Scene, rays: np.ndarray, hits_t, hits_u, hits_v, hits_prim):
    """Hit points (barycentric, float64) and unit normals facing the incoming ray."""
    ok = hits_prim != MISS
    prim = hits_prim[ok].astype(np.int64)
    tri = scene.triangles()[prim].astype(np.float64).reshape(-1, 3, 3)
    u = hits_u[ok].astype(np.float64)[:, None]
    v = hits_v[ok].astype(np.float64)[:, None]
    p = (1 - u - v) * tri[:, 0] + u * tri[:, 1] + v * tri[:, 2]
    n = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    nn = np.linalg.norm(n, axis=1, keepdims=True)
    n = n / np.where(nn == 0, 1, nn)
    d = rays[ok, 4:7].astype(np.float64)
    flip = np.sum(n * d, axis=1) > 0
    n[flip] = -n[flip]
    return ok, p, n


def bounce_rays(scene: Scene, rays, t, u, v, prim, seed: int) -> np.ndarray:
    """One cosine-weighted diffuse bounce per hit: origin = hit point, about the
    normal faced toward the incoming ray. Rays of missed pixels are dropped."""
    rng = rng_for(seed)
    ok, p, n = _hit_frame(scene, rays, t, u, v, prim)
    m = p.shape[0]
    r1 = rng.uniform(size=m)
    r2 = rng.uniform(size=m)
    phi = 2 * math.pi * r1
    sr = np.sqrt(r2)
    local = np.stack([sr * np.cos(phi), sr * np.sin(phi), np.sqrt(1 - r2)], -1)
    a = np.where(np.abs(n[:, :1]) > 0.9, np.array([[0, 1, 0]]), np.array([[1, 0, 0]]))
    t1 = _normalize(np.cross(a, n))
    t2 = np.cross(n, t1)
    d = _normalize(local[:, :1] * t1 + local[:, 1:2] * t2 + local[:, 2:3] * n)
    return make_rays(p.astype(np.float32), d.astype(np.float32), TMIN, np.inf)


def shadow_rays(scene: Scene, rays, t, u, v, prim, light=CONFIG2_LIGHT) -> np.ndarray:
    """One any-hit ray per hit toward a point light, tmax = (1 - 1e-4) * dist."""
    ok, p, _ = _hit_frame(scene, rays, t, u, v, prim)
    L = np.asarray(light, np.float64)[None, :] - p
    dist = np.linalg.norm(L, axis=1)
    d = L / dist[:, None]
    return make_rays(p.astype(np.float32), d.astype(np.float32), TMIN,
                     ((1 - 1e-4) * dist).astype(np.float32))


def config3_scene(seed: int = 1003, n: int = 1 << 23) -> Scene:
    """Random equilateral soup in the unit cube (2^23 triangles by default)."""
    rng = rng_for(seed)
    return Scene(random_soup(rng, n), None, f"soup{n}")


def config3_rays(seed: int = 2003, n: int = 1 << 23, tmax=np.inf) -> np.ndarray:
    rng = rng_for(seed)
    return random_rays(rng, n, (0, 0, 0), (1, 1, 1), TMIN, tmax)


def config5_weights(n: int, seed: int = 1005):
    """Loss weights w, a, b ~ N(0, 1) for L = sum w t + a u + b v."""
    rng = rng_for(seed)
    return (rng.normal(size=n).astype(np.float32),
            rng.normal(size=n).astype(np.float32),
            rng.normal(size=n).astype(np.float32))


def config4_workload(seed: int = 1004, n_scenes: int = 64,
                     tri_range=(1e3, 2e6), ray_range=(1e3, 1e6), scale: float = 1.0):
    """Uneven multi-scene batch: per scene a soup or fBm height field (type by
    seed) with a log-uniform triangle count, and its own ray batch of
    log-uniform size, half camera rays and half random rays in the scene box.

    ``scale`` multiplies both ranges (small cases for tests)."""
    rng = rng_for(seed)
    out = []
    for s in range(n_scenes):
        n = int(math.exp(rng.uniform(math.log(tri_range[0] * scale), math.log(tri_range[1] * scale))))
        m = int(math.exp(rng.uniform(math.log(ray_range[0] * scale), math.log(ray_range[1] * scale))))
        n = max(n, 2)
        m = max(m, 2)
        kind = int(rng.integers(0, 2))
        srng = rng_for(seed * 1000 + s + 1)
        if kind == 0:
            mu = math.log(0.002 * math.sqrt((1 << 23) / n))
            sc = Scene(random_soup(srng, n, mu=mu), None, f"soup{n}")
        else:
            side = int(math.ceil(math.sqrt(n / 2))) + 1
            v, i = grid_mesh(lambda X, Y: value_noise_fbm(X, Y, srng), side - 1, side - 1)
            sc = Scene(v, i, f"fbm{side}")
        lo = sc.verts.min(axis=0).astype(np.float64)
        hi = sc.verts.max(axis=0).astype(np.float64)
        ctr = (lo + hi) / 2
        rad = float(np.linalg.norm(hi - lo)) / 2 + 1e-3
        th = srng.uniform(0, 2 * math.pi)
        ph = srng.uniform(0.2, 1.2)
        eye = ctr + 2.5 * rad * np.array([math.cos(th) * math.cos(ph),
                                           math.sin(th) * math.cos(ph), math.sin(ph)])
        mc = m // 2
        w = max(1, int(math.sqrt(mc)))
        h = max(1, mc // w)
        cam = pinhole_rays(eye, ctr, (0, 0, 1), 45.0, w, h)
        rnd = random_rays(srng, m - w * h, lo, hi)
        out.append((sc, np.concatenate([cam, rnd])))
    return out
