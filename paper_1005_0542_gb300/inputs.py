"""Seeded synthetic workloads (media, sources, receivers, request traces).

This module draws random numbers and lays out positions; it holds none of the method's
arithmetic (no operator, transform or solver).  Both the CUDA library's tests/benches and the
CPU oracle take the arrays it returns.  Everything is float64 numpy on the host, row-major
[z][x] with x fastest, interior nodes only (the Dirichlet frame is implicit).

Stand-ins for the paper's media (its Marmousi and thin-layer models are not available):
layered and random media with the paper-like parameter ranges below.

* ``two_layer``        128 x 128, 10 m, c = 2000/3000 m/s, rho = 1000/2000 kg/m^3, interface at
                       row 64, Ricker 30 Hz at (64, 16), h = 200, alpha = 9, 64 harmonics.
* ``random_layered``   20 equal layers in z, c ~ U(1500, 4500) per layer times (1 + eps),
                       eps ~ N(0, 0.025^2) clipped to +-0.05 i.i.d. per node; Gardner-type
                       rho = 310 c^0.25 kg/m^3.
* ``elastic_layered``  20 layers, Vp ~ U(2000, 5000), Vs = Vp / 1.73, rho ~ U(1800, 2600), plus a
                       dipping interface from z = 0.4 nz at x = 0 to z = 0.6 nz at x = nx-1
                       below which an independent set of layer draws replaces the first.

Every wavelet is a Ricker with delay t0 = 2.5 / f0, so |f(0)| ~ 2e-25: with alpha = 9 the
Laguerre series needs u = O(t^{alpha/2}) at t = 0 (initial data, Eq. 4), and a wavelet that
starts at 1e-8 (t0 = 1.5 / f0) feeds harmonics that grow like m^{alpha/2 - 1}.
"""
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

SEED_BASE = 1005


@dataclass
class Shot:
    """One synthetic problem (acoustic if ``vs`` is None)."""
    name: str
    nx: int
    nz: int
    hx: float
    hz: float
    c: np.ndarray                 # acoustic velocity, or Vp for elastic  [nz, nx]
    rho: np.ndarray               # density                                [nz, nx]
    vs: Optional[np.ndarray]      # shear velocity (elastic only)
    h: float                      # Laguerre parameter (1/s)
    alpha: int                    # Laguerre order
    n_harm: int
    f0: float                     # wavelet peak frequency (Hz)
    t0: float                     # wavelet delay (s)
    sources: List[Tuple[int, int]] = field(default_factory=list)   # (ix, iz)
    receivers: List[Tuple[int, int]] = field(default_factory=list)
    t_out: np.ndarray = None
    tol: float = 1e-10
    restart: int = 20


def _receivers_line(nx, iz, count):
    step = max(1, nx // count)
    return [(ix, iz) for ix in range(step // 2, nx, step)][:count]


def two_layer(n_harm=64, nx=128, nz=128):
    """Two-layer acoustic model with the interface at row nz/2 (row 64 at 128 x 128)."""
    c = np.full((nz, nx), 2000.0)
    rho = np.full((nz, nx), 1000.0)
    c[nz // 2:, :] = 3000.0
    rho[nz // 2:, :] = 2000.0
    f0 = 30.0
    return Shot("two_layer_128", nx, nz, 10.0, 10.0, c, rho, None, 200.0, 9, n_harm, f0,
                2.5 / f0, sources=[(nx // 2, 16)], receivers=_receivers_line(nx, 16, 16),
                t_out=np.linspace(0.002, 0.6, 300))


def random_layered_velocity(nx, nz, rng, layers=20, lo=1500.0, hi=4500.0, pert=0.05):
    """c per layer ~ U(lo, hi), multiplied by (1 + eps) per node, eps ~ N(0, (pert/2)^2)
    clipped to +-pert."""
    lay = rng.uniform(lo, hi, size=layers)
    rows = (np.arange(nz) * layers) // nz
    c = np.repeat(lay[rows][:, None], nx, axis=1)
    eps = np.clip(rng.normal(0.0, pert / 2.0, size=(nz, nx)), -pert, pert)
    return c * (1.0 + eps)


def gardner_density(c):
    """rho = 310 c^0.25 (kg/m^3, c in m/s): the Gardner-type relation of the workload."""
    return 310.0 * np.asarray(c, dtype=np.float64) ** 0.25


def random_layered(nx=2048, nz=1024, hx=5.0, n_harm=512, seed=SEED_BASE + 2, f0=25.0,
                   sources=None, name="random_layered"):
    """Acoustic random layered model (default 2048 x 1024, 5 m, 512 harmonics, one source)."""
    rng = np.random.default_rng(seed)
    c = random_layered_velocity(nx, nz, rng)
    rho = gardner_density(c)
    if sources is None:
        sources = [(nx // 2, min(16, nz - 1))]
    return Shot(f"{name}_{nx}x{nz}", nx, nz, hx, hx, c, rho, None, 200.0, 9, n_harm, f0,
                2.5 / f0, sources=sources, receivers=_receivers_line(nx, min(2, nz - 1), 64),
                t_out=np.linspace(0.002, 1.0, 500))


def cylindrical(nr=2048, nz=2048, h=None, n_harm=3000, layered=False, seed=SEED_BASE + 5, f0=30.0,
                elastic=False):
    """The paper's axisymmetric acoustic experiment (Sec. 3.2): a point source on the axis at the
    free surface, the Gaussian-modulated sine of Eq. 23 (f0 = 30 Hz, t0 = 0.2 s, gamma = 4),
    alpha = 9, Laguerre h = 400, mesh step lambda/40, receivers on the surface row.  Homogeneous
    (c = 2000 m/s, rho = 1000 kg/m^3) as in the paper, or a random layered medium (the layers
    along z, the generator of the Cartesian workload) for the iterative behaviour.  Fields are
    [nr][nz] (depth fastest); sources / receivers are (radius index, depth index).
    elastic=True: the same model read as Vp with Vs = Vp / 1.73 (Sec. 2.2's axisymmetric elastic
    problem; the source becomes a vertical force on the axis)."""
    c0 = 2000.0
    if h is None:
        h = c0 / f0 / 40.0
    if layered:
        rng = np.random.default_rng(seed)
        c = np.ascontiguousarray(random_layered_velocity(nr, nz, rng).T)   # layers along z, [nr][nz]
    else:
        c = np.full((nr, nz), c0)
    rho = gardner_density(c) if layered else np.full((nr, nz), 1000.0)
    rcv = [(i, 0) for i in range(0, nr, max(1, nr // 64))][:64]
    vs = c / 1.73 if elastic else None
    kind = ("elastic_" if elastic else "") + ("layered" if layered else "homogeneous")
    return Shot(f"cylindrical_{kind}_{nr}x{nz}", nr, nz, h, h, c, rho, vs,
                400.0, 9, n_harm, f0, 0.2, sources=[(0, 0)], receivers=rcv,
                t_out=np.linspace(0.002, 1.0, 500))


def surface_line_sources(nx, count, iz=2):
    """count sources at ix = round((s + 1/2) nx / count), depth row iz."""
    return [(int(round((s + 0.5) * nx / count)), iz) for s in range(count)]


def elastic_layered(nx=4096, nz=2048, hx=2.5, n_harm=1024, seed=SEED_BASE + 4, nsrc=16,
                    f0=20.0):
    """Elastic random layered model with a dipping interface."""
    rng = np.random.default_rng(seed)
    layers = 20
    rows = (np.arange(nz) * layers) // nz
    vp1, rho1 = rng.uniform(2000.0, 5000.0, layers), rng.uniform(1800.0, 2600.0, layers)
    vp2, rho2 = rng.uniform(2000.0, 5000.0, layers), rng.uniform(1800.0, 2600.0, layers)
    vp = np.repeat(vp1[rows][:, None], nx, axis=1)
    rho = np.repeat(rho1[rows][:, None], nx, axis=1)
    zi = np.arange(nz)[:, None].astype(np.float64)
    xi = np.arange(nx)[None, :].astype(np.float64)
    z_int = 0.4 * nz + 0.2 * nz * xi / max(1, nx - 1)
    below = zi >= z_int
    vp = np.where(below, vp2[rows][:, None], vp)
    rho = np.where(below, rho2[rows][:, None], rho)
    vs = vp / 1.73
    srcs = surface_line_sources(nx, nsrc, iz=min(2, nz - 1))
    return Shot(f"elastic_layered_{nx}x{nz}", nx, nz, hx, hx, vp, rho, vs, 300.0, 8, n_harm, f0,
                2.5 / f0, sources=srcs, receivers=_receivers_line(nx, min(2, nz - 1), 64),
                t_out=np.linspace(0.002, 1.0, 500))


def random_rhs(nrhs, nz, nx, seed=SEED_BASE + 2):
    """Standalone preconditioner input: i.i.d. N(0, 1) right-hand sides [nrhs, nz, nx]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nrhs, nz, nx))


SERVE_MESHES = [(256, 256), (512, 1024), (1024, 2048), (2048, 1024), (4096, 2048)]


def request_trace(count=256, rate=50.0, seed=SEED_BASE + 5, meshes=None, n_lo=128, n_hi=1024,
                  kinds=("acoustic", "elastic")):
    """Poisson arrivals of shots: list of dicts (arrival time, kind, mesh (nx, nz), n_harm, seed).

    The media themselves are generated per request from ``seed`` with ``random_layered`` /
    ``elastic_layered`` at the drawn mesh."""
    rng = np.random.default_rng(seed)
    meshes = SERVE_MESHES if meshes is None else meshes
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    for i in range(count):
        nx, nz = meshes[rng.integers(len(meshes))]
        out.append(dict(arrival=float(t[i]), kind=kinds[rng.integers(len(kinds))], nx=nx, nz=nz,
                        n_harm=int(rng.integers(n_lo, n_hi + 1)), seed=int(rng.integers(1 << 30))))
    return out
