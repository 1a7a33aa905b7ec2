"""Seeded synthetic drop configurations shared by the CUDA path, the tests and the bench.

This module draws random numbers and lays them out; it performs none of the boundary
integral method's arithmetic (no quadrature, no transforms, no kernels).  Every drop
surface is written directly as spherical-harmonic (SH) coefficients of x(theta, phi),
so no SH synthesis or analysis is needed to build an input.

Coefficient layout (real-packed, per scalar, degree p): (p+1)**2 doubles, index
n*(n+1)+m holds Re f_n^m for m >= 0 and Im f_n^{|m|} for m < 0.  For a real function
f_n^{-m} = (-1)^m conj(f_n^m) (Section 1.2), so this packing is lossless.

Shapes follow the workloads of the paper: a sphere of radius a centred at c has
x_0^0 = sqrt(4 pi) c and the degree-1 coefficients of a * (unit sphere) below;
ellipsoids are a linear map of the unit sphere (degree 1 only); perturbations add
random degree 1..nmax coefficients scaled so that the sup-norm of each component of
the perturbation is bounded by the stated amplitude (|Y_n^m| <= sqrt((2n+1)/(4 pi))).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 1707021560


def ncoef(p: int) -> int:
    return (p + 1) * (p + 1)


def cidx(n: int, m: int) -> int:
    return n * (n + 1) + m


# Unit-sphere coordinates x = sin(t)cos(f), y = sin(t)sin(f), z = cos(t) in the
# orthonormal, Condon-Shortley-phased basis of Section 1.2:
#   z = sqrt(4pi/3) Y_1^0,  x = sqrt(2pi/3)(Y_1^-1 - Y_1^1),  y = i sqrt(2pi/3)(Y_1^-1 + Y_1^1).
_S = math.sqrt(2.0 * math.pi / 3.0)
UNIT_SPHERE_DEG1 = {
    # component -> {(n, m) packed index: value}
    0: {cidx(1, 1): -_S},           # Re x_1^1
    1: {cidx(1, -1): _S},           # Im y_1^1
    2: {cidx(1, 0): math.sqrt(4.0 * math.pi / 3.0)},  # z_1^0
}


def sphere_coef(p: int, radius: float = 1.0, centre=(0.0, 0.0, 0.0), axes=None, rot=None) -> np.ndarray:
    """x coefficients [3][(p+1)^2] of the ellipsoid  c + Q diag(axes) s,  s on the unit sphere."""
    assert p >= 1
    if axes is None:
        axes = (radius, radius, radius)
    A = np.diag(np.asarray(axes, dtype=np.float64))
    if rot is not None:
        A = np.asarray(rot, dtype=np.float64) @ A
    unit = np.zeros((3, ncoef(p)))
    for c, ent in UNIT_SPHERE_DEG1.items():
        for k, v in ent.items():
            unit[c, k] = v
    x = A @ unit
    x[:, 0] += math.sqrt(4.0 * math.pi) * np.asarray(centre, dtype=np.float64)
    return x


def random_bandlimited(rng: np.random.Generator, p: int, ncomp: int, decay_pow: float = 2.0) -> np.ndarray:
    """Random real band-limited scalars: Re, Im ~ N(0,1)/(n+1)^decay_pow, Im = 0 at m = 0."""
    out = np.zeros((ncomp, ncoef(p)))
    for c in range(ncomp):
        for n in range(p + 1):
            s = 1.0 / (n + 1.0) ** decay_pow
            out[c, cidx(n, 0)] = rng.standard_normal() * s
            for m in range(1, n + 1):
                out[c, cidx(n, m)] = rng.standard_normal() * s
                out[c, cidx(n, -m)] = rng.standard_normal() * s
    return out


def supnorm_bound(coef: np.ndarray, p: int) -> float:
    """Upper bound of max |f| over the sphere for one real-packed scalar."""
    tot = 0.0
    for n in range(p + 1):
        ymax = math.sqrt((2 * n + 1) / (4 * math.pi))
        tot += abs(coef[cidx(n, 0)]) * ymax
        for m in range(1, n + 1):
            tot += 2.0 * math.hypot(coef[cidx(n, m)], coef[cidx(n, -m)]) * ymax
    return tot


def perturbation(rng: np.random.Generator, p: int, nmin: int, nmax: int, amplitude: float) -> np.ndarray:
    """Vector perturbation [3][(p+1)^2], degrees nmin..nmax, each component bounded by amplitude."""
    d = np.zeros((3, ncoef(p)))
    for c in range(3):
        for n in range(nmin, min(nmax, p) + 1):
            d[c, cidx(n, 0)] = rng.standard_normal()
            for m in range(1, n + 1):
                d[c, cidx(n, m)] = rng.standard_normal()
                d[c, cidx(n, -m)] = rng.standard_normal()
    s = max(supnorm_bound(d[c], p) for c in range(3))
    return d * (amplitude / s) if s > 0 else d


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform proper rotation from a normalised Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def pack_drops(coefs: list[np.ndarray]) -> np.ndarray:
    """Concatenate per-drop [ncomp][(p_i+1)^2] blocks into one flat array [drop][comp][coef]."""
    return np.concatenate([c.reshape(-1) for c in coefs]).astype(np.float64)


@dataclass
class Workload:
    """One seeded configuration.  All per-drop arrays are flat, drop-major."""
    name: str
    p: list            # SH degree of each drop
    pq: list           # degree of the self (singular) quadrature grid of each drop
    up: int            # upsampling factor U for the intermediate region
    xcoef: np.ndarray  # [drop][3][(p+1)^2]
    lam: np.ndarray    # viscosity ratio of each drop
    density: np.ndarray            # [drop][3][(p+1)^2] random test density
    gamma: np.ndarray | None = None  # [drop][1][(p+1)^2] surfactant coefficients
    elasticity: float = 0.0          # linear equation of state sigma = 1 - E * Gamma
    shear: float = 0.0               # u_inf = (shear * z, 0, 0)
    bounding: np.ndarray | None = None  # bounding radius per drop (for sampling)
    extra: dict = field(default_factory=dict)

    @property
    def ndrop(self) -> int:
        return len(self.p)


def _rng(stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(MASTER_SEED, spawn_key=(stream,))))


def _gamma_const(p: int, value: float) -> np.ndarray:
    g = np.zeros((1, ncoef(p)))
    g[0, 0] = value * math.sqrt(4.0 * math.pi)
    return g


def single_sphere(p: int = 16, pq: int | None = None, seed_stream: int = 0) -> Workload:
    """Unit sphere at the origin, lambda = 1, random band-limited vector density."""
    rng = _rng(seed_stream)
    x = sphere_coef(p)
    f = random_bandlimited(rng, p, 3)
    return Workload("sphere", [p], [pq if pq is not None else p], 1, pack_drops([x]),
                    np.array([1.0]), pack_drops([f]), gamma=pack_drops([_gamma_const(p, 1.0)]),
                    bounding=np.array([1.0]))


def perturbed_drop(p: int = 32, pq: int | None = None, amplitude: float = 0.05, nmax: int = 6,
                   lam: float = 5.0, seed_stream: int = 1) -> Workload:
    """Sphere plus a seeded SH perturbation of degrees 1..nmax, in shear (z, 0, 0)."""
    rng = _rng(seed_stream)
    x = sphere_coef(p) + perturbation(rng, p, 1, nmax, amplitude)
    f = random_bandlimited(rng, p, 3)
    if pq is None:
        pq = 2 * (p + 1) - 1
    return Workload("perturbed", [p], [pq], 1, pack_drops([x]), np.array([lam]), pack_drops([f]),
                    gamma=pack_drops([_gamma_const(p, 1.0)]), elasticity=0.0, shear=1.0,
                    bounding=np.array([1.0 + amplitude]))


def two_drops(p: int = 32, gap: float = 0.05, up: int = 4, lam: float = 0.5, seed_stream: int = 2) -> Workload:
    """Two unit spheres on the z axis at surface gap `gap`, Gamma = 1 + 0.3 Y_2^0, sigma = 1 - 0.2 Gamma."""
    rng = _rng(seed_stream)
    zc = 1.0 + gap / 2.0
    xs = [sphere_coef(p, centre=(0, 0, zc)), sphere_coef(p, centre=(0, 0, -zc))]
    fs = [random_bandlimited(rng, p, 3) for _ in range(2)]
    gs = []
    for _ in range(2):
        g = _gamma_const(p, 1.0)
        g[0, cidx(2, 0)] = 0.3
        gs.append(g)
    return Workload("two_drops", [p, p], [p, p], up, pack_drops(xs), np.array([lam, lam]), pack_drops(fs),
                    gamma=pack_drops(gs), elasticity=0.2, shear=1.0, bounding=np.array([1.0, 1.0]),
                    extra={"gap": gap})


def _rsa(rng, radii, box, gap, max_tries=200000):
    n = len(radii)
    centres = np.zeros((n, 3))
    placed = 0
    tries = 0
    order = np.argsort(-radii)  # place large drops first
    out = np.zeros((n, 3))
    for idx in order:
        r = radii[idx]
        while True:
            tries += 1
            if tries > max_tries:
                raise RuntimeError("random sequential addition did not converge")
            c = rng.uniform(r, box - r, size=3)
            if placed == 0:
                break
            d = np.linalg.norm(centres[:placed] - c, axis=1)
            if np.all(d >= radii[order[:placed]] + r + gap):
                break
        centres[placed] = c
        out[idx] = c
        placed += 1
    return out


def batch_spheres(ndrop: int = 64, degrees=(16, 24, 32, 48), box: float = 14.07, gap: float = 0.5,
                  up: int = 2, seed_stream: int = 3) -> Workload:
    """Non-overlapping spheres of uneven degree, radii U[0.8,1.2], lambda U[0.2,5]."""
    rng = _rng(seed_stream)
    ps = [int(v) for v in rng.choice(np.asarray(degrees), size=ndrop)]
    radii = rng.uniform(0.8, 1.2, size=ndrop)
    lam = rng.uniform(0.2, 5.0, size=ndrop)
    centres = _rsa(rng, radii, box, gap)
    xs = [sphere_coef(p, radius=r, centre=c) for p, r, c in zip(ps, radii, centres)]
    fs = [random_bandlimited(rng, p, 3) for p in ps]
    gs = [_gamma_const(p, 1.0) for p in ps]
    return Workload("batch_spheres", ps, list(ps), up, pack_drops(xs), lam, pack_drops(fs),
                    gamma=pack_drops(gs), bounding=radii.copy(), extra={"box": box, "centres": centres})


def deformed_drops(ndrop: int = 512, p: int = 24, box: float = 27.8, gap: float = 0.5, noise: float = 0.1,
                   nmax: int = 8, up: int = 2, seed_stream: int = 4) -> Workload:
    """Randomly oriented ellipsoids (axes U[0.7,1.3]) plus SH noise, random decaying Gamma."""
    rng = _rng(seed_stream)
    axes = rng.uniform(0.7, 1.3, size=(ndrop, 3))
    bound = axes.max(axis=1) + noise
    lam = rng.uniform(0.2, 5.0, size=ndrop)
    centres = _rsa(rng, bound, box, gap)
    xs, fs, gs = [], [], []
    for i in range(ndrop):
        Q = random_rotation(rng)
        x = sphere_coef(p, centre=centres[i], axes=axes[i], rot=Q) + perturbation(rng, p, 2, nmax, noise)
        xs.append(x)
        fs.append(random_bandlimited(rng, p, 3))
        g = random_bandlimited(rng, p, 1) * 0.1
        g[0, 0] = math.sqrt(4.0 * math.pi)
        gs.append(g)
    return Workload("deformed_drops", [p] * ndrop, [p] * ndrop, up, pack_drops(xs), lam, pack_drops(fs),
                    gamma=pack_drops(gs), elasticity=0.2, shear=1.0, bounding=bound,
                    extra={"box": box, "centres": centres})


def config(name: str) -> Workload:
    """The seeded workloads, by name: c1 .. c5, and c4s, a 16-drop version of c4 with degrees
    {16, 24} at the same volume fraction (a size small enough for kernel profiling)."""
    return {
        "c1": lambda: single_sphere(16),
        "c2": lambda: perturbed_drop(32),
        "c3": lambda: two_drops(32),
        "c4": lambda: batch_spheres(),
        "c4s": lambda: batch_spheres(ndrop=16, degrees=(16, 24), box=8.86, seed_stream=5),
        "c5": lambda: deformed_drops(),
    }[name]()
