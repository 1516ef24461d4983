"""Seeded synthetic inputs shaped like the paper's porous-cylinder cases.

This module is shared by the FP64 oracle (``oracle/``) and the CUDA path
(``paper_2606_31707_b300``).  It holds geometry, seeds and physical
parameters only: no lattice Boltzmann arithmetic (no relaxation time, no
equilibrium, no streaming).  Everything it returns is a plain numpy array or
a plain Python value.

Geometry follows the paper's cylinder cases (Sec. 5.2-5.4, Tables 1-3):
a cylinder of lattice porosity d = 0 inside and d = 1 in the bulk (Sec. 5.1),
placed in a channel with an inflow at x = 0 and an outflow at x = Nx-1 and
periodic lateral walls.  The paper gives the cylinder a sharp d; the
synthetic inputs blend it with a tanh profile and seed a jitter or a porous
ring so that the porosity field, the control of the sensitivity analysis
(Sec. 3.1), is non-trivial.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

__all__ = [
    "Regions",
    "Workload",
    "cylinder_porosity",
    "ring_porosity",
    "grf_porosity",
    "velocity_perturbation",
    "make_workload",
    "WORKLOADS",
]


@dataclasses.dataclass(frozen=True)
class Regions:
    """Index boxes (half-open) of the objective and design regions.

    ``ffa_x`` is the x index of the far-field plane Gamma_J of the drag
    functional (Sec. 4.2); ``ffa_y``/``ffa_z`` its extent.  ``diss_box`` is
    the objective domain Omega_J of the dissipation functional (Sec. 4.3) as
    (x0, x1, y0, y1, z0, z1).  ``design_box`` is the control domain
    Omega_alpha (Sec. 3.1) on which the gradient is reported.
    """

    ffa_x: int
    ffa_y: Tuple[int, int]
    ffa_z: Tuple[int, int]
    diss_box: Tuple[int, int, int, int, int, int]
    design_box: Tuple[int, int, int, int, int, int]


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic case: grid, flow parameters, porosity and regions.

    ``q`` is 9 (D2Q9) or 19 (D3Q19); ``dims`` is (nx, ny, nz) with nz = 1 in
    2D.  ``u0`` is the inflow velocity, ``Re`` the Reynolds number based on
    the length ``L`` (the cylinder diameter unless stated), ``Cs`` the
    Smagorinsky constant (0 = plain BGK).  ``steps``/``avg_window`` are the
    primal step count and the number of final steps that are averaged.
    ``collision`` is the collision the case is run with by default: BGK
    (with the Smagorinsky relaxation time when ``Cs`` > 0) for every case;
    the recursive regularised collision of the paper's turbulent model is the
    alternative for the LES cases.
    """

    name: str
    q: int
    dims: Tuple[int, int, int]
    u0: float
    Re: float
    L: float
    Cs: float
    steps: int
    avg_window: int
    regions: Regions
    porosity: np.ndarray          # (nz, ny, nx) float64 in [0, 1]
    u_perturb: Optional[np.ndarray]  # (3, nz, ny, nx) float64 or None
    storage: str = "fp32"
    collision: str = "bgk"        # "bgk" or "rr" (the turbulent model's regularised collision)

    @property
    def cells(self) -> int:
        nx, ny, nz = self.dims
        return nx * ny * nz


# --------------------------------------------------------------------------
# porosity generators
# --------------------------------------------------------------------------

def _radius_grid(dims, xc, yc):
    nx, ny, nz = dims
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    return np.broadcast_to(r, (nz, ny, nx)).copy()


def cylinder_porosity(dims, xc, yc, R, width=2.0, jitter=0.0, seed=0):
    """Cylinder (axis along z) blended by 0.5*(1 + tanh((r - R)/width)).

    r is the distance of cell centre (x, y) from (xc, yc).  With ``jitter``
    > 0, cells of the interface band (0.01 < d < 0.99) get a seeded
    U(-jitter, jitter) offset, then d is clipped to [0, 1].
    """
    r = _radius_grid(dims, xc, yc)
    d = 0.5 * (1.0 + np.tanh((r - R) / width))
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        band = (d > 0.01) & (d < 0.99)
        noise = rng.uniform(-jitter, jitter, size=d.shape)
        d = np.where(band, d + noise, d)
    return np.clip(d, 0.0, 1.0)


def ring_porosity(d_cyl, dims, xc, yc, R, ring=10, block=10, lo=0.2, hi=0.8, seed=0):
    """Porous ring R <= r < R + ring around a cylinder field ``d_cyl``.

    The plane is tiled in ``block`` x ``block`` cells; every tile draws one
    seeded U(lo, hi) value, applied (as a minimum with the cylinder field)
    to the ring cells it covers.
    """
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    tiles = rng.uniform(lo, hi, size=((ny + block - 1) // block, (nx + block - 1) // block))
    tile_field = np.repeat(np.repeat(tiles, block, axis=0), block, axis=1)[:ny, :nx]
    r = _radius_grid(dims, xc, yc)
    in_ring = (r >= R) & (r < R + ring)
    d = np.where(in_ring, np.minimum(d_cyl, tile_field[None, :, :]), d_cyl)
    return np.clip(d, 0.0, 1.0)


def grf_porosity(dims, box, corr=8.0, seed=0):
    """Gaussian random field inside ``box`` = (x0, x1, y0, y1); d = 1 outside.

    White N(0, 1) noise over the box is smoothed by a Gaussian of standard
    deviation ``corr`` cells, standardised, and mapped to
    clip(0.5 + 0.25 z, 0, 1).
    """
    from scipy.ndimage import gaussian_filter

    nx, ny, nz = dims
    x0, x1, y0, y1 = box
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(size=(y1 - y0, x1 - x0))
    z = gaussian_filter(z, sigma=corr)
    z = (z - z.mean()) / z.std()
    d = np.ones((nz, ny, nx))
    d[:, y0:y1, x0:x1] = np.clip(0.5 + 0.25 * z, 0.0, 1.0)[None]
    return d


def velocity_perturbation(dims, amplitude, seed=0):
    """Seeded U(-amplitude, amplitude) perturbation of u_y, shape (3, nz, ny, nx)."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed + 7919)
    up = np.zeros((3, nz, ny, nx))
    up[1] = rng.uniform(-amplitude, amplitude, size=(nz, ny, nx))
    return up


# --------------------------------------------------------------------------
# the cases
# --------------------------------------------------------------------------

def _regions_cyl(dims, xc, D, ffa_offset=5.0, diss_half=11.0):
    nx, ny, nz = dims
    fx = int(round(xc + ffa_offset * D))
    fx = min(max(fx, 1), nx - 2)
    x0 = max(0, int(round(xc - diss_half * D)))
    x1 = min(nx, int(round(xc + diss_half * D)))
    return Regions(ffa_x=fx, ffa_y=(0, ny), ffa_z=(0, nz),
                   diss_box=(x0, x1, 0, ny, 0, nz),
                   design_box=(0, nx, 0, ny, 0, nz))


def make_workload(name: str, seed: int = 0, **over) -> Workload:
    """Build one of the named synthetic cases (see ``WORKLOADS``)."""
    if name == "cyl2d_re20":
        # steady laminar D2Q9, 200x80, D = 20 at (50, 40), Re = 20, FP64
        dims = (200, 80, 1)
        xc, yc, D = 50.0, 40.0, 20.0
        d = cylinder_porosity(dims, xc, yc, D / 2, 2.0, jitter=0.01, seed=seed)
        wl = Workload(name, 9, dims, 0.05, 20.0, D, 0.0, 6000, 1,
                      _regions_cyl(dims, xc, D), d, None, "fp64")
    elif name == "karman2d_re100":
        # unsteady D2Q9, 1100x410, D = 50 at (125, 205), Re = 100, FP32
        dims = (1100, 410, 1)
        xc, yc, D = 125.0, 205.0, 50.0
        d = cylinder_porosity(dims, xc, yc, D / 2, 2.0, jitter=0.01, seed=seed)
        d = ring_porosity(d, dims, xc, yc, D / 2, 10, 10, 0.2, 0.8, seed=seed + 1)
        up = velocity_perturbation(dims, 1e-3 * 0.04, seed)
        wl = Workload(name, 9, dims, 0.04, 100.0, D, 0.0, 225_000, 150_000,
                      _regions_cyl(dims, xc, D), d, up, "fp32")
    elif name in ("les3d_re3900", "les3d_re3900_quarter", "les3d_re3900_slab"):
        # the LES case (640x320x100, D = 32); its quarter-scale copy (D = 8);
        # and a 24-cell-deep slab of the full-resolution case (4.9 M cells, a
        # few GB on the device: the size for kernel profiles)
        quarter = name.endswith("quarter")
        D = 8.0 if quarter else 32.0
        dims = (160, 80, 25) if quarter else ((640, 320, 24) if name.endswith("slab") else (640, 320, 100))
        xc, yc = 5 * D, 5 * D
        d = cylinder_porosity(dims, xc, yc, D / 2, 2.0, jitter=0.01, seed=seed)
        cu = int(D / 0.05)  # steps per convective unit D/u0
        up = velocity_perturbation(dims, 1e-3 * 0.05, seed)
        wl = Workload(name, 19, dims, 0.05, 3900.0, D, 0.1, 100 * cu, 50 * cu,
                      _regions_cyl(dims, xc, D), d, up, "fp32", "bgk")
    elif name == "grf2d_re40":
        # differentiation case: D2Q9 400x160, GRF in a 60x60 box at (100, 80)
        dims = (400, 160, 1)
        box = (70, 130, 50, 110)
        d = grf_porosity(dims, box, 8.0, seed)
        regions = Regions(ffa_x=300, ffa_y=(0, 160), ffa_z=(0, 1),
                          diss_box=(0, 400, 0, 160, 0, 1),
                          design_box=(70, 130, 50, 110, 0, 1))
        wl = Workload(name, 9, dims, 0.05, 40.0, 60.0, 0.0, 20000, 1, regions, d, None, "fp32")
    elif name == "karman2d_4096":
        # the Karman geometry scaled to a 4096 x 4096 D2Q9 grid (D = 500): a working set
        # (0.6 GB of FP32 populations) far beyond L2, for the HBM-bound D2Q9 rates
        dims = (4096, 4096, 1)
        xc, yc, D = 1250.0, 2048.0, 500.0
        d = cylinder_porosity(dims, xc, yc, D / 2, 2.0, jitter=0.01, seed=seed)
        d = ring_porosity(d, dims, xc, yc, D / 2, 10, 10, 0.2, 0.8, seed=seed + 1)
        up = velocity_perturbation(dims, 1e-3 * 0.04, seed)
        wl = Workload(name, 9, dims, 0.04, 100.0, D, 0.0, 3000, 1000,
                      _regions_cyl(dims, xc, D, diss_half=2.0), d, up, "fp32")
    elif name.startswith("tiny"):
        # small cases for tests: tiny2d / tiny3d
        if name == "tiny3d":
            dims = (24, 12, 6)
            q = 19
        else:
            dims = (32, 16, 1)
            q = 9
        xc, yc, D = 10.0, dims[1] / 2.0, 6.0
        d = cylinder_porosity(dims, xc, yc, D / 2, 1.5, jitter=0.01, seed=seed)
        regions = _regions_cyl(dims, xc, D, ffa_offset=2.0, diss_half=1.5)
        wl = Workload(name, q, dims, 0.05, 5.0, D, 0.0, 400, 1, regions, d, None, "fp64")
    else:
        raise KeyError(name)
    if over:
        wl = dataclasses.replace(wl, **over)
    return wl


WORKLOADS = ("cyl2d_re20", "karman2d_re100", "karman2d_4096", "les3d_re3900", "les3d_re3900_quarter",
             "les3d_re3900_slab",
             "grf2d_re40", "tiny2d", "tiny3d")


def serving_request_stream(n_requests: int, rate_per_s: float = 200.0, seed: int = 0):
    """Poisson arrivals of mixed-size sensitivity requests.

    Returns a list of dicts (arrival time s, name, dims, q, Re, seed).  Sizes
    are drawn uniformly from the D2Q9 grids {200x80, 800x320, 2000x800} and
    the D3Q19 grids {128^3, 256x128x64}; Re ~ U[20, 200].
    """
    rng = np.random.default_rng(seed)
    sizes = [((200, 80, 1), 9), ((800, 320, 1), 9), ((2000, 800, 1), 9),
             ((128, 128, 128), 19), ((256, 128, 64), 19)]
    t = 0.0
    out = []
    for k in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        dims, q = sizes[rng.integers(len(sizes))]
        out.append(dict(t=t, dims=dims, q=q, Re=float(rng.uniform(20, 200)),
                        seed=int(rng.integers(1 << 30))))
    return out


def serving_porosity(dims, seed):
    """Cylinder of diameter ny/4 at (ny/2, ny/2) plus a seeded porous ring."""
    nx, ny, nz = dims
    D = ny / 4.0
    xc, yc = ny / 2.0, ny / 2.0
    d = cylinder_porosity(dims, xc, yc, D / 2, 2.0, jitter=0.01, seed=seed)
    ring = max(2, int(math.ceil(D / 5)))
    return ring_porosity(d, dims, xc, yc, D / 2, ring, ring, 0.2, 0.8, seed=seed + 1)
