"""Seeded synthetic inputs: source/target geometries and signal parameters.

This module holds none of the method's arithmetic.  It draws geometries and signal
parameters with numpy's PCG64 generator and evaluates the signal formula at grid
times; both the CUDA path (which receives sigma_j(t_n) samples) and the oracle
(which evaluates the same formula at arbitrary times in its own C code) take
their inputs from here.

Workload shapes follow the paper's examples (Sec. 7): point sources on closed
curves (Sec. 7.3-7.4, "sources on a circle" / "complicated closed curve", which
model discretised layer potentials) or uniformly random in a square (Sec. 7.2),
each with a band-limited time signature.  The paper's erf-switched sinusoid
(Eq. exampleDensities) is available as the ``erf`` family; the default
``gauss3`` family is a sum of three Gaussian-enveloped sinusoids with carrier
2*pi rad per unit time (one wavelength per unit length).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NPAR = 8
SEED0 = 20260703


@dataclass
class Workload:
    name: str
    src_xy: np.ndarray          # (M, 2) float64
    params: np.ndarray          # (M, 8) float64 signal parameters
    family: str                 # "gauss3" | "erf"
    dt: float
    n_steps: int
    band_limit: float           # K_0, rad per unit time
    tol: float = 1e-6
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return self.src_xy.shape[0]

    def times(self, n0: int, n1: int) -> np.ndarray:
        """Grid times t_n = n dt for n in [n0, n1)."""
        return np.arange(n0, n1, dtype=np.float64) * self.dt

    def sigma(self, n0: int, n1: int) -> np.ndarray:
        """Samples sigma_j(t_n) for n in [n0, n1): array (n1 - n0, M)."""
        return sample_sigma(self.params, self.times(n0, n1), self.family)


# ------------------------------------------------------------------ geometry
def uniform_square(M: int, side: float, rng: np.random.Generator) -> np.ndarray:
    return rng.uniform(0.0, side, size=(M, 2))


def _ellipse_points(a: float, b: float, theta: float, cx: float, cy: float, n: int, phase: float) -> np.ndarray:
    """n points equispaced in arclength on an ellipse (semi-axes a, b, rotated by theta)."""
    fine = max(4096, 64 * n)
    s = np.linspace(0.0, 2 * math.pi, fine + 1)
    dx = -a * np.sin(s)
    dy = b * np.cos(s)
    seg = np.sqrt(dx * dx + dy * dy)
    arc = np.concatenate([[0.0], np.cumsum(0.5 * (seg[1:] + seg[:-1]) * (s[1] - s[0]))])
    target = (np.arange(n) + phase) / n * arc[-1]
    par = np.interp(target, arc, s)
    x = a * np.cos(par)
    y = b * np.sin(par)
    c, sn = math.cos(theta), math.sin(theta)
    return np.stack([cx + c * x - sn * y, cy + sn * x + c * y], axis=1)


def ellipses(M: int, n_ell: int, axis_lo: float, axis_hi: float, box: float, rng: np.random.Generator) -> np.ndarray:
    """M points on n_ell random ellipses inside [0, box]^2, split by perimeter, equispaced in arclength."""
    a = rng.uniform(axis_lo, axis_hi, n_ell)
    b = rng.uniform(axis_lo, axis_hi, n_ell)
    th = rng.uniform(0.0, math.pi, n_ell)
    hx = np.sqrt((a * np.cos(th)) ** 2 + (b * np.sin(th)) ** 2)
    hy = np.sqrt((a * np.sin(th)) ** 2 + (b * np.cos(th)) ** 2)
    if np.any(2 * hx >= box) or np.any(2 * hy >= box):
        raise ValueError("ellipse larger than the box")
    cx = rng.uniform(hx, box - hx)
    cy = rng.uniform(hy, box - hy)
    h = ((a - b) / (a + b)) ** 2
    per = math.pi * (a + b) * (1 + 3 * h / (10 + np.sqrt(4 - 3 * h)))  # Ramanujan
    counts = np.floor(M * per / per.sum()).astype(int)
    counts[np.argsort(-per)[: M - counts.sum()]] += 1
    phase = rng.uniform(0.0, 1.0, n_ell)
    pts = [_ellipse_points(a[k], b[k], th[k], cx[k], cy[k], counts[k], phase[k]) for k in range(n_ell)]
    return np.concatenate(pts, axis=0)


# ------------------------------------------------------------------- signals
def gauss3_params(M: int, T: float, rng: np.random.Generator, s_env: float = 1.0,
                  omega: float = 2 * math.pi, lead: float = 8.0) -> np.ndarray:
    """sigma_j(t) = sum_{q=1..3} a_q exp(-(t - c_q)^2 / (2 s^2)) sin(omega (t - c_q)),
    a_q ~ U[-1, 1], c_q = lead*s + d_q with delays d_q ~ U[0, T/2]."""
    p = np.zeros((M, NPAR))
    p[:, 0:3] = rng.uniform(-1.0, 1.0, size=(M, 3))
    p[:, 3:6] = lead * s_env + rng.uniform(0.0, 0.5 * T, size=(M, 3))
    p[:, 6] = s_env
    p[:, 7] = omega
    return p


def erf_params(M: int, rng: np.random.Generator, omega_max: float, t0_lo: float, t0_hi: float,
               cube_root: bool = True) -> np.ndarray:
    """Paper's Eq. exampleDensities: 0.5 (erf(5 (t - t0)) + 1) sin(omega (t - t0))."""
    p = np.zeros((M, NPAR))
    p[:, 0] = rng.uniform(t0_lo, t0_hi, M)
    z = rng.uniform(0.0, 1.0, M)
    p[:, 1] = omega_max * (np.cbrt(z) if cube_root else z)
    return p


def sample_sigma(params: np.ndarray, t: np.ndarray, family: str) -> np.ndarray:
    """sigma_j(t_n), array (len(t), M); zero for t <= 0."""
    t = np.asarray(t, dtype=np.float64)[:, None]
    p = params
    if family == "gauss3":
        s = p[None, :, 6]
        w = p[None, :, 7]
        out = np.zeros((t.shape[0], p.shape[0]))
        for q in range(3):
            z = t - p[None, :, 3 + q]
            out += p[None, :, q] * np.exp(-z * z / (2 * s * s)) * np.sin(w * z)
    elif family == "erf":
        from scipy.special import erf
        z = t - p[None, :, 0]
        out = 0.5 * (erf(5.0 * z) + 1.0) * np.sin(p[None, :, 1] * z)
    elif family == "poly":
        out = p[None, :, 0] + t * (p[None, :, 1] + t * p[None, :, 2])
    else:
        raise ValueError(family)
    return np.where(t > 0, out, 0.0)


def band_limit(params: np.ndarray, family: str, eps: float) -> float:
    """epsilon-bandwidth K_0 of the signal family (rad per unit time)."""
    if family == "gauss3":
        return float(np.max(np.abs(params[:, 7])) + math.sqrt(2 * math.log(1 / eps)) / np.min(params[:, 6]))
    if family == "erf":
        return float(np.max(np.abs(params[:, 1])) + 10 * math.sqrt(math.log(1 / eps)))  # Sec. 7
    raise ValueError(family)


# ------------------------------------------------------------- named configs
def make(name: str, seed_offset: int = 0, tol: float = 1e-6) -> Workload:
    """Named workloads (config units: unit wave speed, carrier 2 pi, dt = 0.1 ~ 10 steps/period)."""
    eps = tol / 1000.0
    dt = 0.1
    idx = {"cfg1": 0, "cfg2": 1, "cfg3": 2, "cfg4": 3}.get(name, 9)
    rng = np.random.Generator(np.random.PCG64(SEED0 + idx + 1000 * seed_offset))
    if name == "cfg1":  # M=200 coincident sources/targets uniform in a 5x5-wavelength square
        M, Nt, box = 200, 100, 5.0
        xy = uniform_square(M, box, rng)
    elif name == "cfg2":  # M=1e4 on 6 ellipses (semi-axes 2-8) in a 30x30 box
        M, Nt, box = 10_000, 2000, 30.0
        xy = ellipses(M, 6, 2.0, 8.0, box, rng)
    elif name == "cfg3":  # M=1e5 on 40 ellipses in a 100x100 box
        M, Nt, box = 100_000, 4000, 100.0
        xy = ellipses(M, 40, 2.0, 8.0, box, rng)
    elif name == "cfg4":  # M=1e6 on 100 ellipses (semi-axes 10-40) in a 300x300 box
        M, Nt, box = 1_000_000, 3000, 300.0
        xy = ellipses(M, 100, 10.0, 40.0, box, rng)
    else:
        raise ValueError(name)
    T = Nt * dt
    par = gauss3_params(M, T, rng)
    return Workload(name, xy, par, "gauss3", dt, Nt, band_limit(par, "gauss3", eps), tol,
                    {"box": box, "seed": SEED0 + idx + 1000 * seed_offset})


def small(M: int, box: float, n_steps: int, seed: int, curve: bool = False, dt: float = 0.1,
          tol: float = 1e-6, lead: float = 8.0, spread: float | None = None) -> Workload:
    """Small seeded workload for parity tests (uniform square, or ellipses when ``curve``)."""
    rng = np.random.Generator(np.random.PCG64(SEED0 + 7919 * seed))
    if curve:
        lo, hi = 0.1 * box, 0.3 * box
        xy = ellipses(M, max(1, M // 40), lo, hi, box, rng)
    else:
        xy = uniform_square(M, box, rng)
    T = n_steps * dt
    par = gauss3_params(M, T if spread is None else spread, rng, lead=lead)
    return Workload(f"small{M}", xy, par, "gauss3", dt, n_steps, band_limit(par, "gauss3", tol / 1000), tol,
                    {"box": box, "seed": seed})


# ---------------------------------------------------------------- serving mix
def serve_requests(n: int, seed: int = 0, tol: float = 1e-6, dt: float = 0.1) -> list[Workload]:
    """A mix of independent requests for the request server: M log-uniform in [1e3, 1e5], N_t uniform
    in [500, 4000], points on max(1, M/1700) random ellipses (semi-axes 1/15..4/15 of the box).  The
    box side is 0.3 sqrt(M) x U[0.8, 1.25], clipped to [10, 100] wavelengths, which keeps the point
    density along the curves near that of the 10^4- and 10^5-point ellipse workloads."""
    rng = np.random.Generator(np.random.PCG64(SEED0 + 104729 * (seed + 1)))
    eps = tol / 1000.0
    out = []
    for i in range(n):
        M = int(round(math.exp(rng.uniform(math.log(1e3), math.log(1e5)))))
        Nt = int(rng.integers(500, 4001))
        box = float(np.clip(0.3 * math.sqrt(M) * rng.uniform(0.8, 1.25), 10.0, 100.0))
        xy = ellipses(M, max(1, M // 1700), box / 15, 4 * box / 15, box, rng)
        par = gauss3_params(M, Nt * dt, rng)
        out.append(Workload(f"req{i}", xy, par, "gauss3", dt, Nt, band_limit(par, "gauss3", eps), tol,
                            {"box": box, "seed": seed, "index": i}))
    return out


# -------------------------------------------------- the paper's grid-target examples
def paper_grid_workload(kind: str, M: int, n_grid: int, omega_max: float, seed: int = 0, T: float = 8.0,
                        tol: float = 1e-6, k0dt: float = 1.1) -> tuple[Workload, np.ndarray]:
    """The large examples of Sec. 7 at a chosen size, in the paper's own units (the domain B = [-1,1]^2,
    unit wave speed, final time T = 8), with erf-switched sines (Eq. exampleDensities) and an
    n_grid x n_grid regular target grid covering B:
      random : sources uniform in B, t0 ~ U[1.5, 7], w = omega_max z^(1/3) (Sec. "Random space-filling
               sources");
      circle : M equispaced sources on x(s) = (0.8 cos s + 0.2, 0.8 sin s + 0.2), t0 and w rising linearly
               in s from 1.5 to 7 and from 0 to omega_max (Sec. "Sources on a circle");
      wiggly : M sources equispaced in s on x(s) = r(s) (cos s, sin s), r(s) = 0.61 + 0.2 cos 60s
               - 0.1 sin 20s + 0.05 cos 30s - 0.1 cos 40s, t0 rising in s from 1.5 to 7, w = omega_max
               z^(1/3) (Sec. "Sources on a complicated closed curve").
    The paper runs them with omega_max = 300 pi at M = 10^5 (circle) and 10^6; at a smaller M a smaller
    omega_max keeps the number of sources near a target comparable.  dt is set so that K0 dt = k0dt
    (1.10 in the paper's runs), with K0 = omega_max + 10 sqrt(ln(1/eps)), eps = tol / 1000."""
    rng = np.random.Generator(np.random.PCG64(SEED0 + 31337 + 7919 * seed))
    s = 2.0 * math.pi * np.arange(M) / M
    par = np.zeros((M, NPAR))
    if kind == "random":
        xy = rng.uniform(-1.0, 1.0, size=(M, 2))
        par[:, 0] = rng.uniform(1.5, 7.0, M)
        par[:, 1] = omega_max * np.cbrt(rng.uniform(0.0, 1.0, M))
    elif kind == "circle":
        xy = np.stack([0.8 * np.cos(s) + 0.2, 0.8 * np.sin(s) + 0.2], axis=1)
        par[:, 0] = 1.5 + 5.5 * s / (2 * math.pi)
        par[:, 1] = omega_max * s / (2 * math.pi)
    elif kind == "wiggly":
        r = 0.61 + 0.2 * np.cos(60 * s) - 0.1 * np.sin(20 * s) + 0.05 * np.cos(30 * s) - 0.1 * np.cos(40 * s)
        xy = np.stack([r * np.cos(s), r * np.sin(s)], axis=1)
        par[:, 0] = 1.5 + 5.5 * s / (2 * math.pi)
        par[:, 1] = omega_max * np.cbrt(rng.uniform(0.0, 1.0, M))
    else:
        raise ValueError(kind)
    K0 = band_limit(par, "erf", tol / 1000.0)
    n_steps = int(math.ceil(T * K0 / k0dt))
    g = np.linspace(-1.0, 1.0, n_grid)
    tgt = np.stack(np.meshgrid(g, g, indexing="ij"), axis=-1).reshape(-1, 2)
    wl = Workload(f"paper-{kind}{M}", xy, par, "erf", T / n_steps, n_steps, K0, tol,
                  {"box": 2.0, "seed": seed, "omega_max": omega_max})
    return wl, tgt
