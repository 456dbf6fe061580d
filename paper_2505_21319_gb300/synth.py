"""Seeded synthetic inputs: analytic SDF shapes, query samplers, parameter init.

This module holds input generation only (none of the representation's
arithmetic), so both the CUDA path and the FP64 oracle's tests may use it.

The paper fits real meshes (Thingi10k and others, Sec. 4.2), which are not
available; analytic shapes stand in for them, sampled with the paper's
per-iteration structure: half the points uniform in the bounding volume, half
near the surface (Sec. 4.2).

Shapes: unions (min) of spheres, axis-aligned boxes and z-axis tori.
  sphere  centre c, radius s                      |q - c| - s
  box     centre c, half-extents e (3 values)     exact box distance
  torus   centre c, major radius s, minor s/3     exact torus distance
Surface samples: a primitive is chosen with probability proportional to its
area, a point is drawn uniformly on its surface, kept only if it lies on the
union's boundary (union SDF >= -1e-6), then displaced by N(0, sigma^2 I).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SPHERE, BOX, TORUS = 0, 1, 2


def rng(seed: int) -> np.random.Generator:
    """Counter-based Philox generator for a seed (same stream on every host)."""
    return np.random.Generator(np.random.Philox(int(seed)))


@dataclass
class Shape:
    kind: np.ndarray                       # (P,) int
    centre: np.ndarray                     # (P, 3)
    size: np.ndarray                       # (P, 3): sphere radius / box half-extents / torus (major, minor, 0)
    meta: dict = field(default_factory=dict)

    def sdf(self, q: np.ndarray) -> np.ndarray:
        """Union SDF (FP64) at points q (N, 3)."""
        q = np.asarray(q, dtype=np.float64)
        out = np.full(q.shape[0], np.inf)
        for k, c, s in zip(self.kind, self.centre, self.size):
            out = np.minimum(out, _prim_sdf(k, c, s, q))
        return out


def _prim_sdf(kind, c, s, q):
    p = q - c
    if kind == SPHERE:
        return np.linalg.norm(p, axis=1) - s[0]
    if kind == BOX:
        d = np.abs(p) - s
        outside = np.linalg.norm(np.maximum(d, 0.0), axis=1)
        inside = np.minimum(np.max(d, axis=1), 0.0)
        return outside + inside
    if kind == TORUS:
        ring = np.sqrt(p[:, 0] ** 2 + p[:, 1] ** 2) - s[0]
        return np.sqrt(ring ** 2 + p[:, 2] ** 2) - s[1]
    raise ValueError(kind)


def _prim_area(kind, s):
    if kind == SPHERE:
        return 4.0 * np.pi * s[0] ** 2
    if kind == BOX:
        return 8.0 * (s[0] * s[1] + s[1] * s[2] + s[0] * s[2])
    if kind == TORUS:
        return 4.0 * np.pi ** 2 * s[0] * s[1]
    raise ValueError(kind)


def _prim_surface(kind, c, s, n, g: np.random.Generator):
    if kind == SPHERE:
        v = g.standard_normal((n, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        return c + s[0] * v
    if kind == BOX:
        areas = np.array([s[1] * s[2], s[1] * s[2], s[0] * s[2], s[0] * s[2], s[0] * s[1], s[0] * s[1]])
        face = g.choice(6, size=n, p=areas / areas.sum())
        u = g.uniform(-1.0, 1.0, size=(n, 3)) * s
        axis = face // 2
        sign = np.where(face % 2 == 0, -1.0, 1.0)
        u[np.arange(n), axis] = sign * s[axis]
        return c + u
    if kind == TORUS:
        R, r = s[0], s[1]
        out = np.empty((0, 3))
        while out.shape[0] < n:   # rejection on the area element (R + r cos v)
            m = 2 * (n - out.shape[0]) + 16
            uu = g.uniform(0, 2 * np.pi, m)
            vv = g.uniform(0, 2 * np.pi, m)
            keep = g.uniform(0, 1, m) * (R + r) <= R + r * np.cos(vv)
            uu, vv = uu[keep], vv[keep]
            pts = np.stack([(R + r * np.cos(vv)) * np.cos(uu), (R + r * np.cos(vv)) * np.sin(uu), r * np.sin(vv)], 1)
            out = np.concatenate([out, pts])
        return c + out[:n]
    raise ValueError(kind)


def sphere(radius: float = 0.5, centre=(0.0, 0.0, 0.0)) -> Shape:
    return Shape(np.array([SPHERE]), np.array([centre], dtype=np.float64),
                 np.array([[radius, 0.0, 0.0]]), {"name": f"sphere r={radius}"})


def random_union(seed: int, n_prims: int = 8, centre_range: float = 0.6, size_range=(0.1, 0.3)) -> Shape:
    """Union of ``n_prims`` primitives, kind uniform over {sphere, box, torus},
    centres U[-centre_range, centre_range]^3, size U[size_range]: sphere radius,
    box half-extent per axis, torus major radius (minor = major / 3)."""
    g = rng(seed)
    kind = g.integers(0, 3, size=n_prims)
    centre = g.uniform(-centre_range, centre_range, size=(n_prims, 3))
    size = np.zeros((n_prims, 3))
    for i, k in enumerate(kind):
        if k == SPHERE:
            size[i, 0] = g.uniform(*size_range)
        elif k == BOX:
            size[i] = g.uniform(*size_range, size=3)
        else:
            size[i, 0] = g.uniform(*size_range)
            size[i, 1] = size[i, 0] / 3.0
    return Shape(kind, centre, size, {"name": f"union{n_prims} seed={seed}"})


def surface_points(shape: Shape, n: int, g: np.random.Generator) -> np.ndarray:
    """n points uniformly distributed (by area) on the union's boundary."""
    areas = np.array([_prim_area(k, s) for k, s in zip(shape.kind, shape.size)])
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 64
        which = g.choice(len(areas), size=m, p=areas / areas.sum())
        pts = np.empty((m, 3))
        for i in range(len(areas)):
            sel = which == i
            if sel.any():
                pts[sel] = _prim_surface(shape.kind[i], shape.centre[i], shape.size[i], int(sel.sum()), g)
        pts = pts[shape.sdf(pts) >= -1e-6]
        out = np.concatenate([out, pts])
    return out[:n]


def sample_batch(shape: Shape, J: int, seed: int, sigma: float = 0.01, near_frac: float = 0.5) -> np.ndarray:
    """(J, 4) float32 rows (x, y, z, target SDF): ``J - n_near`` uniform points
    in [-1,1]^3 and ``n_near = round(near_frac*J)`` surface points displaced by
    N(0, sigma^2 I).  The target is the FP64 SDF at the FP32-rounded point."""
    g = rng(seed)
    n_near = int(round(near_frac * J))
    n_vol = J - n_near
    vol = g.uniform(-1.0, 1.0, size=(n_vol, 3))
    near = surface_points(shape, n_near, g) + sigma * g.standard_normal((n_near, 3)) if n_near else np.empty((0, 3))
    q = np.concatenate([vol, near]).astype(np.float32)
    perm = g.permutation(J)
    q = q[perm]
    out = np.empty((J, 4), dtype=np.float32)
    out[:, :3] = q
    out[:, 3] = shape.sdf(q.astype(np.float64)).astype(np.float32)
    return out


def init_params(R: int, seed: int, std: float = 1e-3) -> np.ndarray:
    """(R^3, 13) float32 parameters, every slot N(0, std^2)."""
    return (rng(seed).standard_normal((R ** 3, 13)) * std).astype(np.float32)


def random_params(R: int, seed: int, delta_scale: float = 0.3, b_scale: float = 0.3, value_scale: float = 0.5) -> np.ndarray:
    """(R^3, 13) float32 parameters with every slot far from zero, for parity
    tests: offsets up to ``delta_scale`` grid spacings, log-scales N(0, b_scale^2),
    values N(0, value_scale^2)."""
    g = rng(seed)
    h = 2.0 / R
    p = np.empty((R ** 3, 13))
    p[:, 0:3] = g.uniform(-delta_scale, delta_scale, size=(R ** 3, 3)) * h
    p[:, 3:5] = g.standard_normal((R ** 3, 2)) * b_scale
    p[:, 5:13] = g.standard_normal((R ** 3, 8)) * value_scale
    return p.astype(np.float32)



def _grid_positions(R: int) -> np.ndarray:
    c = -1.0 + (np.arange(R) + 0.5) * (2.0 / R)
    a, b, d = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([a.ravel(), b.ravel(), d.ravel()], 1)


def _sdf_grad(shape: Shape, x: np.ndarray, eps: float = 1e-5) -> np.ndarray:
    g = np.empty_like(x)
    for a in range(3):
        dx = np.zeros(3)
        dx[a] = eps
        g[:, a] = (shape.sdf(x + dx) - shape.sdf(x - dx)) / (2 * eps)
    return g


def sdf_params(shape: Shape, R: int, seed: int, noise: float = 0.02, delta_scale: float = 0.3,
               b_scale: float = 0.3) -> np.ndarray:
    """(R^3, 13) float32 parameters shaped like a fitted grid: every key's
    value is the first-order Taylor expansion of the shape's SDF about the
    key (constant = SDF there, linear term = its gradient) plus N(0, noise^2)
    perturbations; offsets U(-delta_scale, delta_scale) grid spacings;
    log-scales N(0, b_scale^2)."""
    g = rng(seed)
    h = 2.0 / R
    k = _grid_positions(R)
    delta = g.uniform(-delta_scale, delta_scale, size=(R ** 3, 3)) * h
    p = np.empty((R ** 3, 13))
    p[:, 0:3] = delta
    p[:, 3:5] = g.standard_normal((R ** 3, 2)) * b_scale
    p[:, 5] = shape.sdf(k) + noise * g.standard_normal(R ** 3)
    p[:, 6:9] = _sdf_grad(shape, k) + noise * g.standard_normal((R ** 3, 3))
    ko = k + delta
    p[:, 9] = shape.sdf(ko) + noise * g.standard_normal(R ** 3)
    p[:, 10:13] = _sdf_grad(shape, ko) + noise * g.standard_normal((R ** 3, 3))
    return p.astype(np.float32)


def variant_params(shape: Shape | None, R: int, sets: int, deg: int, learn: int, seed: int, noise: float = 0.02,
                   delta_scale: float = 0.3, b_scale: float = 0.3, high_scale: float = 1.0) -> np.ndarray:
    """(R^3, channels) float32 parameters of an ablation variant in the layout
    [Delta (3) if offset keys] [b per key set if learnable] [phi per key set]
    (grid set first), phi = (o, d, S (6), T (10)) truncated to the degree.
    With a shape: o and d are the SDF and its gradient at the key plus
    N(0, noise^2), second and third order entries N(0, high_scale^2); without
    one every value entry is N(0, 0.5^2).  Offsets U(+-delta_scale) grid
    spacings, log-scales N(0, b_scale^2)."""
    g = rng(seed)
    nv = [1, 4, 10, 20][deg]
    nsets = (sets & 1) + ((sets >> 1) & 1)
    base = 3 if sets & 2 else 0
    ch = base + learn * nsets + nv * nsets
    p = np.zeros((R ** 3, ch))
    k = _grid_positions(R)
    delta = g.uniform(-delta_scale, delta_scale, size=(R ** 3, 3)) * (2.0 / R)
    if sets & 2:
        p[:, 0:3] = delta
    if learn:
        p[:, base:base + nsets] = g.standard_normal((R ** 3, nsets)) * b_scale
    off = base + learn * nsets
    for si, s in enumerate([s for s in (0, 1) if sets & (1 << s)]):
        pos = k + (delta if s == 1 else 0.0)
        phi = np.zeros((R ** 3, 20))
        if shape is None:
            phi[:] = g.standard_normal((R ** 3, 20)) * 0.5
        else:
            phi[:, 0] = shape.sdf(pos) + noise * g.standard_normal(R ** 3)
            phi[:, 1:4] = _sdf_grad(shape, pos) + noise * g.standard_normal((R ** 3, 3))
            phi[:, 4:20] = g.standard_normal((R ** 3, 16)) * high_scale
        p[:, off + si * nv: off + (si + 1) * nv] = phi[:, :nv]
    return p.astype(np.float32)


# ------------------------------------------------- device-side sampling
#
# The same distributions drawn with torch on a device (FP64 arithmetic, a
# torch Philox generator seeded per call: a different random stream from the
# numpy sampler above).  For query pools too large to draw on the host in
# reasonable time (many shapes, millions of rows each).

def _torch_sdf(shape: Shape, q):
    import torch
    out = torch.full((q.shape[0],), float("inf"), dtype=torch.float64, device=q.device)
    for k, c, s in zip(shape.kind, shape.centre, shape.size):
        p = q - torch.tensor(c, dtype=torch.float64, device=q.device)
        if k == SPHERE:
            d = torch.linalg.norm(p, dim=1) - s[0]
        elif k == BOX:
            e = torch.abs(p) - torch.tensor(s, dtype=torch.float64, device=q.device)
            d = torch.linalg.norm(torch.clamp(e, min=0.0), dim=1) + torch.clamp(e.max(dim=1).values, max=0.0)
        else:
            ring = torch.sqrt(p[:, 0] ** 2 + p[:, 1] ** 2) - s[0]
            d = torch.sqrt(ring ** 2 + p[:, 2] ** 2) - s[1]
        out = torch.minimum(out, d)
    return out


def _torch_prim_surface(kind, c, s, n, gen, device):
    import torch
    f64 = dict(dtype=torch.float64, device=device)
    if kind == SPHERE:
        v = torch.randn((n, 3), generator=gen, **f64)
        v = v / torch.linalg.norm(v, dim=1, keepdim=True)
        return torch.tensor(c, **f64) + s[0] * v
    if kind == BOX:
        areas = torch.tensor([s[1] * s[2], s[1] * s[2], s[0] * s[2], s[0] * s[2], s[0] * s[1], s[0] * s[1]], **f64)
        face = torch.multinomial(areas / areas.sum(), n, replacement=True, generator=gen)
        ext = torch.tensor(s, **f64)
        u = (torch.rand((n, 3), generator=gen, **f64) * 2.0 - 1.0) * ext
        axis = face // 2
        sign = torch.where(face % 2 == 0, -1.0, 1.0).to(torch.float64)
        u[torch.arange(n, device=device), axis] = sign * ext[axis]
        return torch.tensor(c, **f64) + u
    R, r = s[0], s[1]
    parts, have = [], 0
    while have < n:   # rejection on the area element (R + r cos v)
        m = 2 * (n - have) + 16
        uu = torch.rand(m, generator=gen, **f64) * 2 * np.pi
        vv = torch.rand(m, generator=gen, **f64) * 2 * np.pi
        keep = torch.rand(m, generator=gen, **f64) * (R + r) <= R + r * torch.cos(vv)
        uu, vv = uu[keep], vv[keep]
        parts.append(torch.stack([(R + r * torch.cos(vv)) * torch.cos(uu), (R + r * torch.cos(vv)) * torch.sin(uu),
                                  r * torch.sin(vv)], 1))
        have += parts[-1].shape[0]
    return torch.tensor(c, **f64) + torch.cat(parts)[:n]


def surface_points_torch(shape: Shape, n: int, gen, device):
    """n points uniformly (by area) on the union's boundary, on a device."""
    import torch
    areas = torch.tensor([_prim_area(k, s) for k, s in zip(shape.kind, shape.size)], dtype=torch.float64)
    parts, have = [], 0
    while have < n:
        m = 2 * (n - have) + 64
        which = torch.multinomial(areas / areas.sum(), m, replacement=True, generator=torch.Generator().manual_seed(
            int(torch.randint(0, 2 ** 62, (1,), generator=gen, device=device).item())))
        counts = torch.bincount(which, minlength=len(areas)).tolist()
        pts = torch.cat([_torch_prim_surface(shape.kind[i], shape.centre[i], shape.size[i], counts[i], gen, device)
                         for i in range(len(areas)) if counts[i] > 0])
        pts = pts[_torch_sdf(shape, pts) >= -1e-6]
        parts.append(pts)
        have += pts.shape[0]
    out = torch.cat(parts)
    return out[torch.randperm(out.shape[0], generator=gen, device=device)[:n]]


def sample_batch_torch(shape: Shape, J: int, seed: int, device, sigma: float = 0.01, near_frac: float = 0.5):
    """sample_batch's distribution drawn on ``device``: a (J, 4) float32 tensor
    of rows (x, y, z, target SDF), the target the FP64 SDF at the
    FP32-rounded point."""
    import torch
    gen = torch.Generator(device=device).manual_seed(int(seed))
    n_near = int(round(near_frac * J))
    n_vol = J - n_near
    vol = torch.rand((n_vol, 3), generator=gen, dtype=torch.float64, device=device) * 2.0 - 1.0
    parts = [vol]
    if n_near:
        parts.append(surface_points_torch(shape, n_near, gen, device)
                     + sigma * torch.randn((n_near, 3), generator=gen, dtype=torch.float64, device=device))
    q = torch.cat(parts).to(torch.float32)
    q = q[torch.randperm(J, generator=gen, device=device)]
    out = torch.empty((J, 4), dtype=torch.float32, device=device)
    out[:, :3] = q
    out[:, 3] = _torch_sdf(shape, q.to(torch.float64)).to(torch.float32)
    return out


def sdf_grid_torch(shape: Shape, R: int, device):
    """The shape's SDF at the R^3 cell centres -1 + (i + 0.5) 2/R, (R, R, R)
    float32 (x slowest), on ``device``."""
    import torch
    c = -1.0 + (torch.arange(R, dtype=torch.float64, device=device) + 0.5) * (2.0 / R)
    X, Y, Z = torch.meshgrid(c, c, c, indexing="ij")
    return _torch_sdf(shape, torch.stack([X, Y, Z], -1).reshape(-1, 3)).reshape(R, R, R).to(torch.float32)
