"""Seeded synthetic voxel geometries shared by the FP64 oracle and the CUDA path.

This module only draws random numbers and voxelises shapes.  It holds none of
the lattice Boltzmann arithmetic (no stencils, no collision, no streaming), so
both sides of every parity test can consume the same input without sharing
method code.

Flag convention (one uint8 per voxel, array shape ``(nz, ny, nx)`` so that the
linear voxel id is ``x + nx*(y + ny*z)``, x fastest):

    0  fluid
    1  solid / no-slip wall
    2  velocity inlet (moving wall, per-voxel velocity given separately)
    3  pressure outlet

The workloads imitate the paper's applications (porous media from a particle
packing, a free flow over a particle bed, a coronary artery tree; Sec. 6) with
synthetic stand-ins, since neither the MESA-PD packing nor the patient geometry
is available.  Random draws use numpy's PCG64 ``default_rng(seed)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FLUID, WALL, INLET, OUTLET = 0, 1, 2, 3


@dataclass
class Geometry:
    """A voxel box plus the boundary data that goes with it."""

    flags: np.ndarray                      # uint8 (nz, ny, nx)
    periodic: int = 7                      # bit0 x, bit1 y, bit2 z
    inlet_u: np.ndarray | None = None      # float (n_inlet, 3), ascending voxel order
    rho_out: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        nz, ny, nx = self.flags.shape
        return nx, ny, nz

    @property
    def porosity(self) -> float:
        return float(np.count_nonzero(self.flags == FLUID)) / self.flags.size


# ----------------------------------------------------------------------------
# sphere voxelisation helpers
# ----------------------------------------------------------------------------

def _stamp_sphere(flags: np.ndarray, centre, radius: float, value: int,
                  periodic: int) -> int:
    """Set voxels whose centre lies within ``radius`` of ``centre``.

    Distances use the minimum image on periodic axes; on other axes the sphere
    is clipped to the box.  Returns how many voxels changed from FLUID.
    """
    nz, ny, nx = flags.shape
    dims = (nx, ny, nz)
    axes = []
    for a in range(3):
        lo = int(math.floor(centre[a] - radius))
        hi = int(math.ceil(centre[a] + radius))
        idx = np.arange(lo, hi + 1)
        off = idx - centre[a]
        if periodic >> a & 1:
            idx = np.mod(idx, dims[a])
        else:
            keep = (idx >= 0) & (idx < dims[a])
            idx, off = idx[keep], off[keep]
        axes.append((idx, off))
    (ix, ox), (iy, oy), (iz, oz) = axes
    if ix.size == 0 or iy.size == 0 or iz.size == 0:
        return 0
    d2 = oz[:, None, None] ** 2 + oy[None, :, None] ** 2 + ox[None, None, :] ** 2
    inside = d2 <= radius * radius
    sub = flags[np.ix_(iz, iy, ix)]
    target = inside & (sub == FLUID)
    changed = int(np.count_nonzero(target))
    sub[target] = value
    flags[np.ix_(iz, iy, ix)] = sub
    return changed


def boolean_spheres(n: int | tuple, porosity: float, seed: int,
                    rmin: float = 6.0, rmax: float = 12.0) -> Geometry:
    """Periodic Boolean model: overlapping spheres, r ~ U(rmin, rmax), centres
    uniform, added one at a time until the voxel porosity is <= ``porosity``.

    Stand-in for the porous-media packings of Sec. 6.1 at a chosen porosity
    (the Boolean model reaches any porosity, including 0.3, which a
    non-overlapping packing cannot)."""
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    rng = np.random.default_rng(seed)
    flags = np.zeros((nz, ny, nx), np.uint8)
    total = flags.size
    fluid = total
    spheres = 0
    while fluid / total > porosity:
        c = rng.uniform(0.0, 1.0, 3) * (nx, ny, nz)
        r = rng.uniform(rmin, rmax)
        fluid -= _stamp_sphere(flags, c, r, WALL, 7)
        spheres += 1
    return Geometry(flags, 7, meta=dict(kind="boolean_spheres", seed=seed,
                                        target_porosity=porosity, spheres=spheres,
                                        rmin=rmin, rmax=rmax))


def _relax_nonoverlapping(centres: np.ndarray, radius: float, box: np.ndarray,
                          iters: int = 20000) -> np.ndarray:
    """Push overlapping equal spheres apart (minimum image) until none overlap."""
    d_min = 2.0 * radius
    c = centres.copy()
    for _ in range(iters):
        diff = c[:, None, :] - c[None, :, :]
        diff -= box * np.round(diff / box)
        dist = np.sqrt((diff ** 2).sum(-1))
        np.fill_diagonal(dist, np.inf)
        overlap = np.clip(d_min - dist, 0.0, None)
        if overlap.max() <= 1e-9:
            return np.mod(c, box)
        with np.errstate(invalid="ignore", divide="ignore"):
            push = np.where(overlap[..., None] > 0,
                            diff / dist[..., None] * (0.5 * overlap[..., None] + 1e-3), 0.0)
        c = np.mod(c + push.sum(1), box)
    raise RuntimeError("sphere relaxation did not converge")


def relaxed_spheres(n: int = 32, radius: float = 4.0, porosity: float = 0.5,
                    seed: int = 1) -> Geometry:
    """Periodic packing of non-overlapping equal spheres whose voxel porosity
    is closest to ``porosity`` (uniform placement, then relaxation).

    The 32^3, r = 4, porosity 0.5 small case."""
    box = np.array([n, n, n], float)
    v_sphere = 4.0 / 3.0 * math.pi * radius ** 3
    n_guess = int(round((1.0 - porosity) * n ** 3 / v_sphere))
    best = None
    for count in range(max(1, n_guess - 4), n_guess + 5):
        rng = np.random.default_rng(seed * 1000 + count)
        cs = _relax_nonoverlapping(rng.uniform(0.0, 1.0, (count, 3)) * box, radius, box)
        flags = np.zeros((n, n, n), np.uint8)
        for c in cs:
            _stamp_sphere(flags, c, radius, WALL, 7)
        phi = float(np.count_nonzero(flags == FLUID)) / flags.size
        if best is None or abs(phi - porosity) < abs(best[0] - porosity):
            best = (phi, flags, count)
    phi, flags, count = best
    return Geometry(flags, 7, meta=dict(kind="relaxed_spheres", seed=seed, radius=radius,
                                        spheres=count, target_porosity=porosity))


def random_solids(n: int | tuple, solid_fraction: float, seed: int,
                  periodic: int = 7, walls_z: bool = False) -> Geometry:
    """Independent random solid voxels (tiny brute-force cases)."""
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    rng = np.random.default_rng(seed)
    flags = (rng.uniform(0.0, 1.0, (nz, ny, nx)) < solid_fraction).astype(np.uint8)
    if walls_z:
        flags[0] = WALL
        flags[-1] = WALL
    return Geometry(flags, periodic, meta=dict(kind="random_solids", seed=seed))


def channel(nx: int, ny: int, h: int, top: int = WALL, top_u=(0.0, 0.0, 0.0)) -> Geometry:
    """Plane channel periodic in x and y: wall plane at z = 0, ``top`` plane at
    z = h + 1, fluid at z = 1..h.  With ``top = INLET`` the top plane is a
    moving wall with velocity ``top_u`` (Couette flow)."""
    flags = np.zeros((h + 2, ny, nx), np.uint8)
    flags[0] = WALL
    flags[-1] = top
    inlet_u = None
    if top == INLET:
        inlet_u = np.tile(np.asarray(top_u, float), (nx * ny, 1))
    return Geometry(flags, 3, inlet_u=inlet_u, meta=dict(kind="channel", h=h))


def plug_duct(nx: int, ny: int, nz: int, u_in: float, rho_out: float = 1.0) -> Geometry:
    """Inlet plane at x = 0 (velocity (u_in,0,0)), outlet plane at x = nx-1,
    periodic in y and z, no walls: a uniform plug flow."""
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[:, :, 0] = INLET
    flags[:, :, -1] = OUTLET
    inlet_u = np.tile(np.array([u_in, 0.0, 0.0]), (ny * nz, 1))
    return Geometry(flags, 6, inlet_u=inlet_u, rho_out=rho_out,
                    meta=dict(kind="plug_duct", u_in=u_in))


def particle_bed(nx: int = 512, ny: int = 256, nz: int = 256, bed_top: int = 128,
                 radius: float = 8.0, bed_porosity: float = 0.4, u_in: float = 0.05,
                 rho_out: float = 1.0, seed: int = 21) -> Geometry:
    """Free flow over a particle bed (stand-in for Sec. 6.2).

    Velocity inlet plane x = 0 (u = (u_in,0,0)), pressure outlet plane
    x = nx-1, no-slip planes z = 0 and z = nz-1, periodic in y.  The bed is
    the slab z in [1, bed_top]: Boolean spheres of fixed radius, clipped to the
    slab, added until the slab porosity is <= ``bed_porosity``."""
    rng = np.random.default_rng(seed)
    flags = np.zeros((nz, ny, nx), np.uint8)
    slab = np.zeros((bed_top, ny, nx), np.uint8)
    total = slab.size
    fluid = total
    spheres = 0
    while fluid / total > bed_porosity:
        c = rng.uniform(0.0, 1.0, 3) * (nx, ny, bed_top)
        fluid -= _stamp_sphere(slab, c, radius, WALL, 2)   # periodic in y only
        spheres += 1
    flags[1:bed_top + 1] = slab
    flags[0] = WALL
    flags[-1] = WALL
    flags[1:-1, :, 0] = np.where(flags[1:-1, :, 0] == FLUID, INLET, flags[1:-1, :, 0])
    flags[1:-1, :, -1] = np.where(flags[1:-1, :, -1] == FLUID, OUTLET, flags[1:-1, :, -1])
    n_in = int(np.count_nonzero(flags == INLET))
    inlet_u = np.tile(np.array([u_in, 0.0, 0.0]), (n_in, 1))
    return Geometry(flags, 2, inlet_u=inlet_u, rho_out=rho_out,
                    meta=dict(kind="particle_bed", seed=seed, spheres=spheres,
                              bed_top=bed_top, radius=radius, u_in=u_in))


def _rotate_about(v: np.ndarray, axis: np.ndarray, ang: float) -> np.ndarray:
    axis = axis / np.linalg.norm(axis)
    return (v * math.cos(ang) + np.cross(axis, v) * math.sin(ang)
            + axis * np.dot(axis, v) * (1.0 - math.cos(ang)))


def _tree_segments(seed: int, depth: int, r0: float, r_leaf: float, lam: float, start):
    rng = np.random.default_rng(seed)
    segs = []  # (p0, p1, r, is_leaf)

    def grow(p0, d, level):
        r = r0 * (r_leaf / r0) ** (level / depth)
        p1 = p0 + d * lam * r
        leaf = level == depth
        segs.append((p0, p1, r, leaf))
        if leaf:
            return
        perp = np.cross(d, [0.0, 0.0, 1.0] if abs(d[2]) < 0.9 else [0.0, 1.0, 0.0])
        perp /= np.linalg.norm(perp)
        az = rng.uniform(0.0, 2.0 * math.pi)
        perp = _rotate_about(perp, d, az)
        for sgn in (1.0, -1.0):
            ang = math.radians(rng.uniform(20.0, 60.0))
            dc = _rotate_about(d, perp, sgn * ang)
            grow(p1, dc / np.linalg.norm(dc), level + 1)

    grow(np.asarray(start, float), np.array([1.0, 0.0, 0.0]), 0)
    return segs


def _stamp_segments(shape, segs, coarse=1):
    """Voxels whose centre lies within r of a segment (capsules).  With
    coarse = c > 1 the box is sampled at every c-th voxel centre."""
    nx, ny, nz = (-(-n // coarse) for n in shape)
    inside = np.zeros((nz, ny, nx), bool)
    for p0, p1, r, _ in segs:
        if coarse > 1:
            p0, p1, r = (p0 - (coarse - 1) / 2.0) / coarse, (p1 - (coarse - 1) / 2.0) / coarse, r / coarse
        lo = np.maximum(np.floor(np.minimum(p0, p1) - r).astype(int), 0)
        hi = np.minimum(np.ceil(np.maximum(p0, p1) + r).astype(int), [nx - 1, ny - 1, nz - 1])
        if np.any(hi < lo):
            continue
        zs, ys, xs = (np.arange(lo[2], hi[2] + 1), np.arange(lo[1], hi[1] + 1),
                      np.arange(lo[0], hi[0] + 1))
        P = np.stack(np.meshgrid(xs, ys, zs, indexing="xy"), -1).astype(float)
        # meshgrid(xs, ys, zs, indexing='xy') gives shape (ny, nx, nz); reorder to (nz, ny, nx)
        P = P.transpose(2, 0, 1, 3)
        d = p1 - p0
        L2 = float(d @ d)
        t = np.clip(((P - p0) @ d) / L2, 0.0, 1.0)
        dist2 = ((P - p0 - t[..., None] * d) ** 2).sum(-1)
        inside[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] |= dist2 <= r * r
    return inside


def artery_tree(nx: int = 1024, ny: int = 512, nz: int = 512, depth: int = 6,
                r0: float = 20.0, r_leaf: float = 4.0, u_max: float = 0.01,
                target_fluid: float = 0.03, seed: int = 31, lam: float | None = None) -> Geometry:
    """Synthetic coronary-like tree (stand-in for Sec. 6.3).

    A seeded random binary tree of capsules (depth ``depth``, radius shrinking
    geometrically from ``r0`` to ``r_leaf``, branch angles U(20, 60) degrees at
    uniform azimuth) rooted at the centre of the x = 0 face, along +x.  Segment
    length is ``lam * r``; without ``lam`` it is chosen by bisection so the
    fluid fraction comes close to ``target_fluid`` (the tree may not reach it;
    the achieved fraction is reported in ``meta``).  Inlet: the root disc on
    the x = 0 face with a parabolic profile of peak ``u_max``.  Outlets: leaf
    end caps and wherever the tree crosses another box face.  Everything else
    is wall."""
    start = (0.0, ny / 2.0, nz / 2.0)

    def build(l, coarse=1):
        segs = _tree_segments(seed, depth, r0, r_leaf, l, start)
        return segs, _stamp_segments((nx, ny, nz), segs, coarse)

    if lam is None:     # bisection on a 4x coarser sampling of the box
        lo, hi = 1.0, 40.0
        for _ in range(12):
            mid = 0.5 * (lo + hi)
            _, ins = build(mid, 4)
            if ins.mean() < target_fluid:
                lo = mid
            else:
                hi = mid
        lam = 0.5 * (lo + hi)
    segs, inside = build(lam)
    flags = np.where(inside, FLUID, WALL).astype(np.uint8)
    # outlets: leaf end caps (the last voxel layer of each leaf capsule's tip)
    for p0, p1, r, leaf in segs:
        if not leaf:
            continue
        d = (p1 - p0) / np.linalg.norm(p1 - p0)
        tip = p1 + d * r
        cap = _stamp_segments((nx, ny, nz), [(tip - d * 1.5, tip, r, True)])
        flags[cap & inside] = OUTLET
    # any fluid on a box face other than the inlet face becomes an outlet
    for sl in [(slice(None), slice(None), -1), (slice(None), 0, slice(None)),
               (slice(None), -1, slice(None)), (0, slice(None), slice(None)),
               (-1, slice(None), slice(None))]:
        face = flags[sl]
        face[face == FLUID] = OUTLET
    # inlet: root disc at x = 0
    face = flags[:, :, 0]
    zz, yy = np.meshgrid(np.arange(nz), np.arange(ny), indexing="ij")
    rr2 = (yy - start[1]) ** 2 + (zz - start[2]) ** 2
    disc = (face != WALL) & (rr2 <= r0 * r0)
    face[disc] = INLET
    # inlet velocities in ascending voxel order (x = 0 face: order by z then y)
    sel = np.argwhere(flags == INLET)           # rows (z, y, x) already ascending
    r2 = (sel[:, 1] - start[1]) ** 2 + (sel[:, 0] - start[2]) ** 2
    ux = u_max * np.clip(1.0 - r2 / (r0 * r0), 0.0, None)
    inlet_u = np.stack([ux, np.zeros_like(ux), np.zeros_like(ux)], 1)
    fluid = float(np.count_nonzero(flags == FLUID)) / flags.size
    return Geometry(flags, 0, inlet_u=inlet_u, rho_out=1.0,
                    meta=dict(kind="artery_tree", seed=seed, lam=lam, depth=depth,
                              fluid_fraction=fluid, segments=len(segs)))


def taylor_green_fields(L: int, nz: int, U: float):
    """Initial density and velocity of a 2-D Taylor-Green vortex on an
    L x L x nz periodic box: u = U(-cos kx sin ky, sin kx cos ky, 0),
    rho = 1 - (3U^2/4)(cos 2kx + cos 2ky), k = 2 pi / L.  Returns
    (rho[N], u[N,3]) in voxel order.  (Closed-form initial data; the
    decay rate it should show is checked in the oracle tests.)"""
    k = 2.0 * math.pi / L
    z, y, x = np.meshgrid(np.arange(nz), np.arange(L), np.arange(L), indexing="ij")
    ux = -U * np.cos(k * x) * np.sin(k * y)
    uy = U * np.sin(k * x) * np.cos(k * y)
    rho = 1.0 - 0.75 * U * U * (np.cos(2 * k * x) + np.cos(2 * k * y))
    u = np.stack([ux, uy, np.zeros_like(ux)], -1).reshape(-1, 3)
    return rho.reshape(-1), u


def serving_request(i: int):
    """The i-th permeability request of the serving stream: a periodic Boolean
    sphere packing of edge drawn from {64, 96, 128, 192}, porosity U(0.3, 0.8),
    radii U(6, 12), seed 41000 + i."""
    rng = np.random.default_rng(41000 + i)
    n = int(rng.choice([64, 96, 128, 192]))
    phi = float(rng.uniform(0.3, 0.8))
    g = boolean_spheres(n, phi, seed=41000 + i)
    g.meta.update(request=i, edge=n)
    return g
