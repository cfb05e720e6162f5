"""Seeded synthetic inputs for the DG-SWEM hot path.

This module produces meshes, nodal bathymetry, nodal initial states and the
physical parameters of each workload.  It holds none of the method's
arithmetic (no basis, quadrature, flux or time stepping): every number it
emits is a plain function of a seed and a coordinate, so both the CUDA path
and the CPU oracle can be fed from it.

The paper's own workload (Hurricane Harvey on the 6.7M-element TX2008 mesh
with HURDAT2 best-track forcing, Sec. 6.1) is not available here; the
generators below stand in for it with unstructured-triangle meshes of
O(1e5..1e6) elements, deep-basin-to-shelf-to-land bathymetry, a tidal open
boundary and a parametric hurricane.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: draw i of
stream s is splitmix64_mix(s * 2**32 + i).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# boundary edge type codes shared by both sides (an interface value, not arithmetic)
BC_LAND = 0
BC_OPEN = 1
BC_RIVER = 2

FRICTION_NONE = 0
FRICTION_MANNING = 1
FRICTION_QUADRATIC = 2

FP64 = 0
FP32_MIXED = 1

# SSP Runge-Kutta schemes (interface codes shared by both sides)
RK_SSP22, RK_SSP33, RK_SSP32, RK_SSP42, RK_SSP52, RK_SSP43, RK_CUSTOM = range(7)

# numerical fluxes
FLUX_LLF, FLUX_ROE = 0, 1


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each 64-bit counter value (vectorised)."""
    with np.errstate(over="ignore"):
        z = counter.astype(np.uint64) * _GOLDEN + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n uniforms in [0, 1) from stream `stream` of seed `seed` (53-bit mantissa)."""
    base = (np.uint64(seed) << np.uint64(40)) ^ (np.uint64(stream) << np.uint64(32))
    bits = splitmix64(base + np.arange(n, dtype=np.uint64))
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class Mesh:
    xy: np.ndarray          # [n_nodes, 2] float64, metres
    tri: np.ndarray         # [n_elems, 3] int32, counter-clockwise, 0-based
    bedge: np.ndarray       # [n_bedges, 2] int32 node pairs
    bedge_type: np.ndarray  # [n_bedges] int32, BC_LAND / BC_OPEN

    @property
    def n_nodes(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.tri.shape[0])


def grid_mesh(nx: int, ny: int, lx: float, ly: float, seed: int, jitter: float = 0.0,
              open_sides=(), flip=None, river_sides=()) -> Mesh:
    """nx-by-ny squares on [0,lx]x[0,ly], each split along a seeded-random diagonal.

    Interior vertices are moved by up to `jitter` times the cell size in each
    coordinate (uniform in a square).  Boundary edges on the sides listed in
    `open_sides` (any of 'left', 'right', 'bottom', 'top') are open, those on `river_sides` river
    inflow edges, the rest land.
    Node (i, j) has index j*(nx+1)+i; triangles are counter-clockwise.  `flip`
    (optional, [ny, nx] bool) fixes the diagonal of each cell instead of the seed.
    """
    hx, hy = lx / nx, ly / ny
    i, j = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    x = (i * hx).astype(np.float64).ravel()
    y = (j * hy).astype(np.float64).ravel()
    x[i.ravel() == nx] = lx
    y[j.ravel() == ny] = ly
    if jitter > 0.0:
        interior = ((i > 0) & (i < nx) & (j > 0) & (j < ny)).ravel()
        n = x.size
        ux = uniform(seed, 1, n)
        uy = uniform(seed, 2, n)
        x = np.where(interior, x + (2.0 * ux - 1.0) * jitter * hx, x)
        y = np.where(interior, y + (2.0 * uy - 1.0) * jitter * hy, y)
    xy = np.stack([x, y], axis=1)

    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ci, cj = ci.ravel(), cj.ravel()
    n00 = cj * (nx + 1) + ci
    n10 = n00 + 1
    n01 = n00 + (nx + 1)
    n11 = n01 + 1
    if flip is None:
        flip = uniform(seed, 3, ci.size) < 0.5
    else:
        flip = np.asarray(flip, bool).reshape(-1)
    # diagonal n00-n11 (flip False) or n10-n01 (flip True)
    t1 = np.where(flip[:, None], np.stack([n00, n10, n01], 1), np.stack([n00, n10, n11], 1))
    t2 = np.where(flip[:, None], np.stack([n10, n11, n01], 1), np.stack([n00, n11, n01], 1))
    tri = np.empty((2 * ci.size, 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2

    edges, types = [], []

    def side(name, pairs):
        edges.append(pairs)
        code = BC_OPEN if name in open_sides else (BC_RIVER if name in river_sides else BC_LAND)
        types.append(np.full(len(pairs), code, np.int32))

    ib = np.arange(nx)
    side("bottom", np.stack([ib, ib + 1], 1))
    top = ny * (nx + 1)
    side("top", np.stack([top + ib + 1, top + ib], 1))
    jb = np.arange(ny)
    side("left", np.stack([(jb + 1) * (nx + 1), jb * (nx + 1)], 1))
    side("right", np.stack([jb * (nx + 1) + nx, (jb + 1) * (nx + 1) + nx], 1))
    bedge = np.concatenate(edges).astype(np.int32)
    btype = np.concatenate(types).astype(np.int32)
    return Mesh(xy=np.ascontiguousarray(xy), tri=tri, bedge=bedge, bedge_type=btype)


def perlin2d(x: np.ndarray, y: np.ndarray, seed: int) -> np.ndarray:
    """Classic 2D gradient (Perlin) noise with a seeded 256-entry gradient table, range ~[-1, 1]."""
    ang = 2.0 * math.pi * uniform(seed, 7, 256)
    gx, gy = np.cos(ang), np.sin(ang)
    perm = np.argsort(uniform(seed, 8, 256)).astype(np.int64)
    xi = np.floor(x).astype(np.int64)
    yi = np.floor(y).astype(np.int64)
    fx, fy = x - xi, y - yi

    def grad(ix, iy, dx, dy):
        h = perm[(perm[ix & 255] + iy) & 255]
        return gx[h] * dx + gy[h] * dy

    def fade(t):
        return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)

    n00 = grad(xi, yi, fx, fy)
    n10 = grad(xi + 1, yi, fx - 1.0, fy)
    n01 = grad(xi, yi + 1, fx, fy - 1.0)
    n11 = grad(xi + 1, yi + 1, fx - 1.0, fy - 1.0)
    u, v = fade(fx), fade(fy)
    nx0 = n00 + u * (n10 - n00)
    nx1 = n01 + u * (n11 - n01)
    return (nx0 + v * (nx1 - nx0)) * math.sqrt(2.0)


def default_params(**kw) -> dict:
    """Physical and numerical parameters; field names follow the C-ABI parameter block."""
    p = dict(p=1, precision=FP64, g=9.81, cfl=0.3, dt=0.0, h0=0.0,
             friction=FRICTION_NONE, manning_n=0.0, cf=0.0, limiter=0,
             coriolis=0, coriolis_lat_deg=0.0,
             tide_amp=0.0, tide_period=44714.0, tide_phase=0.0,
             hurricane=0, pc_hpa=950.0, pn_hpa=1013.0, rmax_m=40000.0, holland_b=1.5,
             vt_ms=5.0, track_x0=0.0, track_y0=0.0, track_heading=0.0,
             rho_air=1.15, rho_water=1000.0, rk_scheme=0, rk_stages=0, rk_coeffs=None, flux=0,
             rain_rate=0.0, river_q=0.0)
    for k, v in kw.items():
        if k not in p:
            raise KeyError(k)
        p[k] = v
    return p


@dataclasses.dataclass
class Case:
    name: str
    mesh: Mesh
    bathy: np.ndarray        # [n_nodes] h_b, positive downward (m)
    init_nodal: np.ndarray   # [3, n_nodes]: zeta, qx, qy at nodes
    params: dict
    steps: int


def config1(n: int = 20, lake: bool = False, seed: int = 1) -> Case:
    """1 km square, n x n cells, land all round, Manning n=0.02, Gaussian hump (or lake at rest)."""
    L = 1000.0
    mesh = grid_mesh(n, n, L, L, seed)
    x, y = mesh.xy[:, 0], mesh.xy[:, 1]
    hb = 10.0 + 2.0 * np.sin(np.pi * x / L)
    init = np.zeros((3, mesh.n_nodes))
    if not lake:
        r2 = (x - 0.5 * L) ** 2 + (y - 0.5 * L) ** 2
        init[0] = 0.1 * np.exp(-r2 / 100.0 ** 2)
    prm = default_params(friction=FRICTION_MANNING, manning_n=0.02, limiter=0, h0=0.0)
    return Case("config1" + ("-lake" if lake else ""), mesh, hb, init, prm, 200)


def config2(n: int = 316, seed: int = 2, p: int = 1, precision: int = FP64) -> Case:
    """100 km x 50 km shelf with dry land, M2 tide on x=0, wet/dry, quadratic friction."""
    lx, ly, h0 = 100e3, 50e3, 0.01
    mesh = grid_mesh(n, n, lx, ly, seed, jitter=0.2, open_sides=("left",))
    x = mesh.xy[:, 0]
    hb = 50.0 - 52.0 * x / lx
    init = np.zeros((3, mesh.n_nodes))
    init[0] = np.maximum(0.0, h0 - hb)
    prm = default_params(p=p, precision=precision, friction=FRICTION_QUADRATIC, cf=0.0025,
                         limiter=1, h0=h0, tide_amp=0.5, tide_period=44714.0)
    return Case("config2", mesh, hb, init, prm, 2000)


def basin_bathymetry(xy: np.ndarray, seed: int) -> np.ndarray:
    """4000 m basin, tanh shelf ramp to 20 m near x = 250 km, 5% Perlin noise (20 km scale)."""
    x, y = xy[:, 0], xy[:, 1]
    ramp = 20.0 + (4000.0 - 20.0) * 0.5 * (1.0 - np.tanh((x - 250e3) / 30e3))
    return ramp * (1.0 + 0.05 * perlin2d(x / 20e3, y / 20e3, seed))


def storm_track(seed: int) -> dict:
    """Seeded storm start position (m), heading (rad) and central pressure (hPa)."""
    u = uniform(seed, 11, 4)
    return dict(track_x0=100e3 + 50e3 * u[0], track_y0=75e3 + 150e3 * u[1],
                track_heading=math.radians(-20.0 + 40.0 * u[2]),
                pc_hpa=930.0 + 50.0 * u[3])


def config3(n: int = 1265, seed: int = 3, precision: int = FP64) -> Case:
    """400 km x 300 km basin-to-shelf domain, moving hurricane, Coriolis at 28N, wet/dry on."""
    mesh = grid_mesh(n, n, 400e3, 300e3, seed)
    hb = basin_bathymetry(mesh.xy, seed)
    init = np.zeros((3, mesh.n_nodes))
    trk = storm_track(seed)
    trk["pc_hpa"] = 950.0
    prm = default_params(precision=precision, friction=FRICTION_QUADRATIC, cf=0.0025, limiter=1,
                         h0=0.01, coriolis=1, coriolis_lat_deg=28.0, hurricane=1,
                         rmax_m=40e3, vt_ms=5.0, **trk)
    return Case("config3", mesh, hb, init, prm, 500)


ENSEMBLE_MESH_N = (158, 316, 447, 632)
ENSEMBLE_MESH_SEEDS = (50, 200, 400, 800)


def ensemble(members_per_mesh: int = 16, mesh_n=ENSEMBLE_MESH_N, precision: int = FP32_MIXED):
    """Storm ensemble: each mesh (config-3 bathymetry) carries `members_per_mesh` scenarios.

    Returns (meshes, bathys, member_list) where member_list holds
    (mesh_index, params, init_nodal) per scenario; scenario seeds are 1000+i.
    """
    meshes, bathys, members = [], [], []
    sid = 0
    for mi, (n, s) in enumerate(zip(mesh_n, ENSEMBLE_MESH_SEEDS)):
        m = grid_mesh(n, n, 400e3, 300e3, s)
        meshes.append(m)
        bathys.append(basin_bathymetry(m.xy, s))
        for _ in range(members_per_mesh):
            trk = storm_track(1000 + sid)
            prm = default_params(precision=precision, friction=FRICTION_QUADRATIC, cf=0.0025,
                                 limiter=1, h0=0.01, coriolis=1, coriolis_lat_deg=28.0,
                                 hurricane=1, rmax_m=40e3, vt_ms=5.0, **trk)
            members.append((mi, prm, None))  # the storms start from rest (zeta = q = 0)
            sid += 1
    return meshes, bathys, members
