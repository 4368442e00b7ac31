"""Seeded synthetic inputs shared by the CUDA path, its tests, the bench and the oracle.

This module holds no arithmetic of the method: it only draws random numbers,
places Lagrangian markers on the curves the experiments use, and fills the
plain parameter records (grid size, density, viscosity, time step, force-law
stiffnesses) that describe one linear system K_E x = b of Eq. (Eul_schur).

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), a public counter-style
generator, so any other implementation of it reproduces the same vectors.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

BASE_SEED = 20261202


def splitmix64(seed: int, n: int) -> np.ndarray:
    """The first n outputs of splitmix64 started from state `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GOLDEN * np.arange(1, n + 1, dtype=np.uint64)
        z = state
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, n: int) -> np.ndarray:
    """n doubles uniform on [-1, 1): 2 * (x >> 11) * 2^-53 - 1 for splitmix64 outputs x."""
    x = splitmix64(seed, n) >> np.uint64(11)
    return 2.0 * x.astype(np.float64) * (2.0 ** -53) - 1.0


def rhs(N: int, seed: int) -> np.ndarray:
    """Right-hand side of length 3N^2 (u | v | p blocks, index j*N + i) drawn uniform on
    [-1, 1); the pressure block is shifted to zero mean so the periodic system is consistent."""
    b = uniform_pm1(seed, 3 * N * N)
    p = b[2 * N * N:]
    p -= p.mean()
    return b


# --------------------------------------------------------------------------- markers

def ellipse_points(M: int, cx: float, cy: float, a: float, b: float) -> np.ndarray:
    th = 2.0 * np.pi * np.arange(M) / M
    return np.stack([cx + a * np.cos(th), cy + b * np.sin(th)], axis=1)


def polar_curve_points(M: int, cx: float, cy: float, r0: float, r1: float, k: int) -> np.ndarray:
    """Markers at equal parameter angle on r(theta) = r0 + r1 cos(k theta)."""
    th = 2.0 * np.pi * np.arange(M) / M
    r = r0 + r1 * np.cos(k * th)
    return np.stack([cx + r * np.cos(th), cy + r * np.sin(th)], axis=1)


def polygon_length(X: np.ndarray, closed: bool) -> float:
    d = np.diff(X, axis=0)
    length = float(np.sum(np.hypot(d[:, 0], d[:, 1])))
    if closed:
        length += float(np.hypot(*(X[0] - X[-1])))
    return length


def _curve_perimeter(fn, samples: int = 1 << 16) -> float:
    return polygon_length(fn(samples), True)


# --------------------------------------------------------------------------- systems

LAW_TARGET = 0
LAW_MEMBRANE = 1
LAW_BEAM = 2
LAW_FIBER = 3
LAW_NAMES = {LAW_TARGET: "target", LAW_MEMBRANE: "membrane", LAW_BEAM: "beam", LAW_FIBER: "fiber"}


@dataclass
class System:
    """One linear system K_E x = b on the periodic square [0, L)^2 with an N x N MAC grid."""
    name: str
    N: int
    L: float
    rho: float
    mu: float
    dt: float
    law: int
    closed: bool
    X: np.ndarray            # (M, 2) marker positions (configuration X^n)
    ds: float                # uniform Lagrangian spacing used by the force stencils
    omega: np.ndarray        # (M,) quadrature weights
    k_target: float = 0.0
    k_stretch: float = 0.0
    k_bend: float = 0.0
    seed: int = BASE_SEED
    X_target: np.ndarray | None = None  # (M, 2) target positions at step n+1 (target law)
    meta: dict = field(default_factory=dict)
    bc: str = "periodic"     # "periodic", or "channel" (Sec. 5.3: inflow on top, traction outflow below)

    @property
    def M(self) -> int:
        return int(self.X.shape[0])

    @property
    def h(self) -> float:
        return self.L / self.N

    def rhs(self) -> np.ndarray:
        return rhs(self.N, self.seed)


def _closed_system(name, N, X, law, rho, mu, dt, seed, **k) -> System:
    M = X.shape[0]
    ds = polygon_length(X, True) / M
    return System(name=name, N=N, L=1.0, rho=rho, mu=mu, dt=dt, law=law, closed=True,
                  X=np.ascontiguousarray(X, dtype=np.float64), ds=ds,
                  omega=np.full(M, ds), seed=seed, **k)


def target_circle(N: int = 32, M: int = 128, kappa: float = 1e4, dt: float = 1e-3,
                  mu: float = 0.01, seed: int | None = None) -> System:
    """Tethered points on the circle of radius 0.25 about (0.5, 0.5): E = -kappa I."""
    X = ellipse_points(M, 0.5, 0.5, 0.25, 0.25)
    return _closed_system(f"target-circle-N{N}", N, X, LAW_TARGET, 1.0, mu, dt,
                          BASE_SEED + 1000 if seed is None else seed, k_target=kappa)


def membrane_ellipse(N: int, kappa: float, a: float = 0.3, b: float = 0.2, M: int | None = None,
                     dt: float | None = None, mu: float = 1e-2, seed: int | None = None) -> System:
    """Spring-tension membrane on an ellipse about (0.5, 0.5), 4N markers unless M is given."""
    M = 4 * N if M is None else M
    X = ellipse_points(M, 0.5, 0.5, a, b)
    dt = 0.5 / N if dt is None else dt
    return _closed_system(f"membrane-ellipse-N{N}-k{kappa:g}", N, X, LAW_MEMBRANE, 1.0, mu, dt,
                          BASE_SEED + 2000 + N if seed is None else seed, k_stretch=kappa)


def beam_curve(N: int = 512, M: int = 2048, k_bend: float = 1e3, k_stretch: float = 1e5,
               dt: float | None = None, mu: float = 1e-2, seed: int | None = None) -> System:
    """Closed beam on r(theta) = 0.23 + 0.035 cos(3 theta) about (0.5, 0.5)."""
    X = polar_curve_points(M, 0.5, 0.5, 0.23, 0.035, 3)
    dt = 0.5 / N if dt is None else dt
    return _closed_system(f"beam-curve-N{N}", N, X, LAW_BEAM, 1.0, mu, dt,
                          BASE_SEED + 3000 + N if seed is None else seed,
                          k_bend=k_bend, k_stretch=k_stretch)


# The paper's own experiment set-ups (Sec. 5.1 and 5.2), with the spacings the text gives.

def paper_membrane(N: int, kappa: float = 1e4, mu: float = 1e-2) -> System:
    """Ellipse with semi-axes 0.23 (x) and 0.27 (y), marker spacing about h/2, dt = h/2."""
    per = _curve_perimeter(lambda m: ellipse_points(m, 0.5, 0.5, 0.23, 0.27))
    M = int(math.ceil(per / (0.5 / N)))
    return membrane_ellipse(N, kappa, a=0.23, b=0.27, M=M, dt=0.5 / N, mu=mu,
                            seed=BASE_SEED + 100 + N)


def paper_beam(N: int, k_bend: float = 1.0, mu: float = 1e-2) -> System:
    """Closed beam r = 0.23 + 0.035 cos 3theta, spacing about h, bending only, dt = h/2."""
    per = _curve_perimeter(lambda m: polar_curve_points(m, 0.5, 0.5, 0.23, 0.035, 3))
    M = int(math.ceil(per / (1.0 / N)))
    return beam_curve(N, M=M, k_bend=k_bend, k_stretch=0.0, dt=0.5 / N, mu=mu,
                      seed=BASE_SEED + 200 + N)


def paper_target_rows(N: int, kappa: float = 1e6, mu: float = 1.0) -> System:
    """Two rows of tethered points at y = 0.25 and y = 0.75 spanning the periodic width,
    spacing h/2 per row, dt = h/2.  Each row is an open curve; E = -kappa I has no
    inter-marker coupling, so the rows can share one marker list."""
    per_row = 2 * N
    x = (np.arange(per_row) + 0.25) * (0.5 / N)
    X = np.concatenate([np.stack([x, np.full(per_row, 0.25)], 1),
                        np.stack([x, np.full(per_row, 0.75)], 1)])
    ds = 0.5 / N
    dt = 0.5 / N
    # the lower row's targets move with velocity -U, the upper row's with +U (U = 0.05)
    Xt = X.copy()
    Xt[:per_row, 0] -= 0.05 * dt
    Xt[per_row:, 0] += 0.05 * dt
    return System(name=f"target-rows-N{N}", N=N, L=1.0, rho=1.0, mu=mu, dt=dt,
                  law=LAW_TARGET, closed=False, X=X, ds=ds, omega=np.full(X.shape[0], ds),
                  k_target=kappa, seed=BASE_SEED + 300 + N, X_target=Xt)


def config1() -> System:
    """Plain FP64 case: 32x32 grid, 128 tethered points on a circle, kappa 1e4, dt 1e-3."""
    return target_circle(32, 128, 1e4, 1e-3, 0.01, seed=BASE_SEED + 1000)


def config2(N: int = 256, kappa: float = 1e4) -> System:
    """Elliptic membrane (semi-axes 0.3, 0.2), 4N markers, spring stiffness kappa."""
    assert N in (128, 256)
    return membrane_ellipse(N, kappa, seed=BASE_SEED + 2000 + N + int(round(math.log10(kappa))))


def config3() -> System:
    """Beam with stretching on a 512x512 grid, 2048 markers, bending 1e3, stretching 1e5."""
    return beam_curve(512, 2048, 1e3, 1e5, seed=BASE_SEED + 3000)


def config4(count: int = 64) -> list[System]:
    """Uneven batch: N from {64, 96, 128, 192, 256}, law from {target, membrane, beam},
    stiffness log-uniform on [1e2, 1e6], each with its own seeded right-hand side."""
    out = []
    draws = splitmix64(BASE_SEED + 4000, 3 * count)
    grids = (64, 96, 128, 192, 256)
    for s in range(count):
        N = grids[int(draws[3 * s] % np.uint64(5))]
        law = int(draws[3 * s + 1] % np.uint64(3))
        u = float(draws[3 * s + 2] >> np.uint64(11)) * 2.0 ** -53
        kappa = 10.0 ** (2.0 + 4.0 * u)
        seed = BASE_SEED + 4000 + s
        if law == LAW_TARGET:
            sysm = target_circle(N, 4 * N, kappa, dt=0.5 / N, mu=1e-2, seed=seed)
        elif law == LAW_MEMBRANE:
            sysm = membrane_ellipse(N, kappa, seed=seed)
        else:
            sysm = beam_curve(N, 4 * N, k_bend=kappa, k_stretch=100.0 * kappa, seed=seed)
        out.append(replace(sysm, name=f"batch{s}-{sysm.name}"))
    return out


# --------------------------------------------------------------------------- time series

def tethered_ring(N: int, kappa_s: float = 1.0, kappa_t: float = 10.0, radius: float = 0.2,
                  mu: float = 4e-3, dt_factor: float = 0.05) -> System:
    """Closed elastic ring (spring-tension law) of the given radius about (0.5, 0.5), marker
    spacing about h/2, tethered to its initial positions with stiffness kappa_t; dt = 0.05 h.
    The periodic stand-in for a flexible structure held in a forced flow (mu = 4e-3 gives
    Re ~ 100 for unit velocity and length 0.4); dt = dt_factor * h."""
    per = 2.0 * np.pi * radius
    M = int(math.ceil(per / (0.5 / N)))
    X = ellipse_points(M, 0.5, 0.5, radius, radius)
    sysm = _closed_system(f"tethered-ring-N{N}", N, X, LAW_MEMBRANE, 1.0, mu, dt_factor / N,
                          BASE_SEED + 5000 + N, k_stretch=kappa_s, k_target=kappa_t)
    sysm.X_target = X.copy()
    return sysm


def shear_forcing(N: int, t: float, amplitude: float = 1.0, period: float = 0.5) -> np.ndarray:
    """Time-periodic body force on the velocity faces (u block then v block):
    f_u = A sin(2 pi y) sin(2 pi t / T),  f_v = (A/2) sin(2 pi x) cos(2 pi t / T)."""
    h = 1.0 / N
    j, i = np.divmod(np.arange(N * N), N)
    yu = (j + 0.5) * h
    xv = (i + 0.5) * h
    w = 2.0 * np.pi * t / period
    fu = amplitude * np.sin(2.0 * np.pi * yu) * np.sin(w)
    fv = 0.5 * amplitude * np.sin(2.0 * np.pi * xv) * np.cos(w)
    return np.concatenate([fu, fv])


# --------------------------------------------------------------------------- fiber (Sec. 5.3)


def fiber_channel(N: int = 16, bend: float = 1.5, jitter: float = 0.05) -> System:
    """The same fiber and parameters in the benchmark's channel (bc = "channel"): periodic in x,
    inflow on the top wall y = 2, traction outflow on y = 0 (Sec. 5.3)."""
    from dataclasses import replace
    rec = fiber_periodic(N, bend, jitter)
    return replace(rec, name=f"fiber-channel-N{N}", bc="channel")


def fiber_periodic(N: int = 16, bend: float = 1.5, jitter: float = 0.05) -> System:
    """The clamped fiber of Sec. 5.3 on a periodic stand-in of its domain: the square (0, 2)^2
    with 2N x 2N cells (h = 1/N), rho = 1, mu = 1.875e-3, dt = 0.05 h.  M = 0.75 N + 1
    markers at spacing ds = h/2 (13, 25, 49, 97 at N = 16 ... 128), midpoint marker at the
    clamp (1, 1.5).  The configuration is the straight fiber with its free ends bent
    downstream, y = 1.5 - bend (x - 1)^2, plus a seeded jitter of `jitter` ds per coordinate
    (a Newton iterate's shape); the force and tangent are taken there.  Stiffnesses: EI =
    2.63672e-2; K_s, K_p, K_t = 375, 1200, 7.03125 at N = 64, proportional to N."""
    h = 1.0 / N
    ds = h / 2.0
    M = int(round(0.375 / ds)) + 1
    m = M // 2
    x = 1.0 + (np.arange(M) - m) * ds
    X = np.stack([x, 1.5 - bend * (x - 1.0) ** 2], 1)
    X = X + jitter * ds * uniform_pm1(BASE_SEED + 7000 + N, 2 * M).reshape(M, 2)
    X[m] = (1.0, 1.5)
    f = N / 64.0
    return System(name=f"fiber-N{N}", N=2 * N, L=2.0, rho=1.0, mu=1.875e-3, dt=0.05 * h, law=LAW_FIBER,
                  closed=False, X=np.ascontiguousarray(X), ds=ds, omega=np.full(M, ds),
                  k_stretch=375.0 * f, k_bend=2.63672e-2, seed=BASE_SEED + 7100 + N,
                  meta={"k_pos": 1200.0 * f, "k_tan": 7.03125 * f, "X_c": (1.0, 1.5)})
