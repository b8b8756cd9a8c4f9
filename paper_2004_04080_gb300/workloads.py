"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the lattice-Boltzmann method: it only draws
initial densities and particle placements from seeds and names the workload
configurations.  Both the CUDA path and the CPU oracle are fed from here, so
neither needs to reproduce the other's random numbers.

* Per-site noise: eta = 2 U - 1 with U the top 53 bits of SplitMix64(seed ^ s)
  (s = x + nx (y + ny z)), i.e. eta ~ U(-1, 1), as in the random-fill boxes of
  the paper's benchmarks (Sec. 5.1), with the mixture written as
  rho_A = m (1 + a eta), rho_B = m (1 - a eta).
* Particles: random sequential addition of centres uniformly in the box with a
  minimum centre distance (Sec. 5.1 places equal spheres at random), drawn from
  numpy's PCG64 with the given seed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

_M64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on a uint64 array."""
    z = (x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(_M64)
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & np.uint64(_M64)
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & np.uint64(_M64)
    return z ^ (z >> np.uint64(31))


def site_noise(n_sites: int, seed: int) -> np.ndarray:
    """eta_s ~ U(-1, 1) per site s, from SplitMix64(seed ^ s)."""
    s = np.arange(n_sites, dtype=np.uint64) ^ np.uint64(seed & _M64)
    with np.errstate(over="ignore"):
        z = splitmix64(s)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


def mixture_densities(shape, seed: int, mean: float = 0.5, amp: float = 0.01):
    """rho_A = mean (1 + amp eta), rho_B = mean (1 - amp eta), flat site order."""
    nx, ny, nz = shape
    eta = site_noise(nx * ny * nz, seed)
    return mean * (1.0 + amp * eta), mean * (1.0 - amp * eta)


def place_colloids(shape, n: int, radius: float, seed: int, min_dist: float,
                   wall_gap: Optional[float] = None, max_tries: int = 200000):
    """Random sequential addition of n centres with pairwise minimum-image
    distance >= min_dist.  With ``wall_gap`` the z coordinate is kept within
    [wall_gap - 1/2, nz - 1/2 - wall_gap] (walls normal to z)."""
    L = np.asarray(shape, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = np.empty((n, 3))
    k = 0
    tries = 0
    # coarse cell grid to keep placement O(n)
    cell = max(min_dist, 1.0)
    ncell = np.maximum((L // cell).astype(int), 1)
    grid: dict = {}
    while k < n:
        tries += 1
        if tries > max_tries + 50 * n:
            raise RuntimeError("could not place %d particles (placed %d)" % (n, k))
        c = rng.random(3) * L
        if wall_gap is not None:
            lo, hi = wall_gap - 0.5, L[2] - 0.5 - wall_gap
            c[2] = lo + (hi - lo) * rng.random()
        ci = (c // (L / ncell)).astype(int) % ncell
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    key = tuple((ci + (dx, dy, dz)) % ncell)
                    for j in grid.get(key, ()):
                        d = c - pos[j]
                        d[:2] -= L[:2] * np.round(d[:2] / L[:2])
                        if wall_gap is None:
                            d[2] -= L[2] * np.round(d[2] / L[2])
                        if d @ d < min_dist * min_dist:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            pos[k] = c
            grid.setdefault(tuple(ci), []).append(k)
            k += 1
    return pos


def droplet_densities(shape, centres, radius: float, rich: float, poor: float, width: float = 2.0):
    """Spheres of B-rich fluid in an A-rich matrix, flat site order: with s
    the largest over the droplets of 1/2 (1 - tanh((r - R) / width)), r the
    minimum-image distance to a centre, rho_B = poor + (rich - poor) s and
    rho_A = rich + poor - rho_B."""
    nx, ny, nz = shape
    s = np.zeros((nz, ny, nx))
    m = int(math.ceil(radius + 4.0 * width))
    off = np.arange(-m, m + 1)
    for c in np.asarray(centres, dtype=np.float64):
        ic = np.floor(c).astype(int)
        X, Y, Z = ic[0] + off, ic[1] + off, ic[2] + off
        dx, dy, dz = X - c[0], Y - c[1], Z - c[2]
        r = np.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2)
        v = 0.5 * (1.0 - np.tanh((r - radius) / width))
        ix, iy, iz = np.mod(X, nx), np.mod(Y, ny), np.mod(Z, nz)
        sub = s[np.ix_(iz, iy, ix)]
        s[np.ix_(iz, iy, ix)] = np.maximum(sub, v)
    rb = poor + (rich - poor) * s.ravel()
    return rich + poor - rb, rb


def default_params() -> dict:
    """Parameter defaults (names follow the C-ABI's lb_params)."""
    return dict(
        tau=(1.0, 1.0), G=0.0, zeta=(0.0, 0.0), rho0=(0.5, 0.5), bc=(1, 1, 1),
        wall_u_lo=(0.0, 0.0, 0.0), wall_u_hi=(0.0, 0.0, 0.0), body_force=(0.0, 0.0, 0.0),
        hertz_K=0.0, hertz_sigma=0.0, hertz_rcap=0.0,
        lub_on=0, lub_hn=0.67, lub_hmin=0.5, lub_scale=0.1,
        side_wall_k=0.0, side_wall_d=0.0, rotate=1,
        janus=0, janus_theta0=108.0, janus_width=10.0,
        rcut=0.0, delr=0.0,
        open=(0, 0), open_rho=(1.0, 1.0, 1.0, 1.0), open_extrap=0,
    )


@dataclasses.dataclass
class Workload:
    """A named synthetic workload: box, physics parameters and particles."""

    name: str
    shape: tuple
    steps: int
    params: dict
    radius: float = 0.0
    n_colloids: int = 0
    particle_density: float = 1.0
    seed: int = 1
    mean: float = 0.5
    amp: float = 0.01
    wall_gap: Optional[float] = None
    # B-rich droplets in an A-rich matrix instead of the noisy 50/50 mixture:
    # dict(n, radius, rich, poor, width, min_dist)
    droplets: Optional[dict] = None

    @property
    def n_sites(self) -> int:
        return int(np.prod(self.shape))

    def droplet_centres(self):
        d = self.droplets
        return place_colloids(self.shape, d["n"], d["radius"], self.seed + 2, d["min_dist"])

    def densities(self):
        if self.droplets is not None:
            d = self.droplets
            return droplet_densities(self.shape, self.droplet_centres(), d["radius"], d["rich"], d["poor"],
                                     d["width"])
        return mixture_densities(self.shape, self.seed, self.mean, self.amp)

    def colloids(self):
        if self.n_colloids == 0:
            return None
        R = self.radius
        sigma = self.params.get("hertz_sigma", 2 * R + 1) or (2 * R + 1)
        pos = place_colloids(self.shape, self.n_colloids, R, self.seed + 1, sigma,
                             wall_gap=self.wall_gap)
        mass = self.particle_density * 4.0 / 3.0 * math.pi * R ** 3
        out = dict(pos=pos, radius=np.full(self.n_colloids, R), mass=np.full(self.n_colloids, mass))
        if self.params.get("janus"):
            out["quat"] = random_orientations(self.n_colloids, self.seed + 3)
        return out


def random_orientations(n: int, seed: int) -> np.ndarray:
    """n unit quaternions (w, x, y, z) uniform over the rotations: normalised
    4-D standard normal draws (PCG64 with the given seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1)[:, None]


def n_for_fraction(shape, radius: float, phi: float) -> int:
    """Number of spheres of the given radius filling volume fraction phi."""
    return int(round(phi * float(np.prod(shape)) / (4.0 / 3.0 * math.pi * radius ** 3)))


def _hertz(R):
    return dict(hertz_K=20.0, hertz_sigma=2 * R + 1.0, hertz_rcap=2 * R)


def workload(name: str, scale: Optional[tuple] = None, calib: Optional[dict] = None) -> Workload:
    """The paper-shaped workloads.  ``scale`` overrides the box (same physics,
    particle and droplet counts rescaled to keep the volume fractions).
    ``calib`` (the Pickering emulsion only): the coexistence densities
    ``rho_rich``, ``rho_poor`` and the wetting parameter ``delta_77`` of the
    demixing mixture, measured with the oracle (tests/golden)."""
    base = default_params()
    if name == "small_fp64":
        # 32^3 periodic, tau=1, G=0.65, 50/50 +-1 %, 4 neutral R=4.5 spheres, 100 steps
        p = dict(base, G=0.65, **_hertz(4.5))
        w = Workload(name, (32, 32, 32), 100, p, radius=4.5, n_colloids=4)
    elif name == "bijel128":
        # 128^3 periodic, R=5, phi=0.20, neutral wetting, Hertz contact, 1000 steps
        p = dict(base, G=0.65, **_hertz(5.0))
        shape = (128, 128, 128)
        w = Workload(name, shape, 1000, p, radius=5.0, n_colloids=n_for_fraction(shape, 5.0, 0.20))
    elif name == "bijel_demix":
        # the bijel with a demixing mixture: rho0 = 1 per component, so that
        # G rho_tot = 1.3 exceeds the critical 2 - 1/tau = 1 by the paper's own
        # ratio (its benchmark uses 1.0 / 1.0 at G = 0.65); 128^3, R = 5,
        # phi = 0.20, neutral wetting
        p = dict(base, G=0.65, rho0=(1.0, 1.0), **_hertz(5.0))
        shape = (128, 128, 128)
        w = Workload(name, shape, 5000, p, radius=5.0, n_colloids=n_for_fraction(shape, 5.0, 0.20), mean=1.0)
    elif name == "adjoint64":
        p = dict(base, G=0.65, **_hertz(4.5))
        w = Workload(name, (64, 64, 64), 500, p, radius=4.5, n_colloids=8)
    elif name == "shear512":
        # 512x512x256, walls normal to z moving at +-0.05 x, R=5.5, phi=0.15
        R = 5.5
        p = dict(base, G=0.65, bc=(1, 1, 0), wall_u_lo=(-0.05, 0.0, 0.0),
                 wall_u_hi=(0.05, 0.0, 0.0), side_wall_k=1.0, side_wall_d=R + 1.0, **_hertz(R))
        shape = (512, 512, 256)
        w = Workload(name, shape, 20000, p, radius=R, n_colloids=n_for_fraction(shape, R, 0.15),
                     wall_gap=R + 1.0)
    elif name == "pickering256":
        # 256^3 periodic, 64 B-rich droplets of R = 16 (6.5 % of the volume)
        # in an A-rich matrix (tanh profile of width 2 between the coexistence
        # densities of the demixing mixture, rho0 = 1 per component), R = 5
        # particles at phi = 0.10 with a contact angle of 77 degrees through
        # the matrix (zeta_A = +Delta, zeta_B = -Delta), 5000 steps
        if calib is None:
            raise ValueError("pickering256 needs the calibration (rho_rich, rho_poor, delta_77)")
        dl = float(calib["delta_77"])
        p = dict(base, G=0.65, rho0=(1.0, 1.0), zeta=(dl, -dl), **_hertz(5.0))
        shape = (256, 256, 256)
        w = Workload(name, shape, 5000, p, radius=5.0, n_colloids=n_for_fraction(shape, 5.0, 0.10), mean=1.0,
                     droplets=dict(n=64, radius=16.0, rich=float(calib["rho_rich"]),
                                   poor=float(calib["rho_poor"]), width=2.0, min_dist=2 * 16.0 + 6.0))
    elif name == "janus_lub256":
        # the colloid benchmark of Sec. 5.1 with the MD-room input of App. D:
        # demixing mixture (density 1.0 per component with standard deviation
        # 0.004: amp = 0.004 sqrt 3 for the uniform noise), G = 0.65; R = 5.5
        # Janus particles (wettability angle 108 degrees, switch width 10,
        # wetting constants 0.1 / 0.1) of mass 472 at random orientations,
        # lubrication (0.1, 0.67, 0.5), Hertz (20, 12, 11), pair list with
        # rcut 12 and skin delr 1; phi = 0.10 in a 256^3 periodic box
        R = 5.5
        p = dict(base, G=0.65, rho0=(1.0, 1.0), zeta=(0.1, 0.1), janus=1, janus_theta0=108.0,
                 janus_width=10.0, lub_on=1, lub_scale=0.1, lub_hn=0.67, lub_hmin=0.5, hertz_K=20.0,
                 hertz_sigma=12.0, hertz_rcap=11.0, rcut=12.0, delr=1.0)
        shape = (256, 256, 256)
        w = Workload(name, shape, 1000, p, radius=R, n_colloids=n_for_fraction(shape, R, 0.10), mean=1.0,
                     amp=0.004 * math.sqrt(3.0), particle_density=472.0 / (4.0 / 3.0 * math.pi * R ** 3))
    else:
        raise KeyError(name)
    if scale is not None:
        frac = float(np.prod(scale)) / float(np.prod(w.shape))
        w.n_colloids = int(round(w.n_colloids * frac))
        if w.droplets is not None:
            w.droplets = dict(w.droplets, n=max(1, int(round(w.droplets["n"] * frac))))
        w.shape = tuple(scale)
    return w
