"""Seeded synthetic inputs for the Legendre-Galerkin solve (shared by tests, bench, smoke).

This module holds no arithmetic of the method itself: it only defines the
coefficient functions a(x), b(x) and right-hand sides f(x) of the model
problem -div(a grad u) + b u = f on [-1,1]^d and samples them on a tensor
Legendre-Gauss grid (nodes from ``numpy.polynomial.legendre.leggauss``,
ascending, x fastest).  Both the CUDA path and the CPU oracle receive the same
sample arrays.

Random draws use SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) for uniforms and
the Box-Muller transform for normals, so that every workload is reproducible
from its seed on any machine.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """``count`` successive SplitMix64 outputs of the stream started at ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, count: int) -> np.ndarray:
    """Uniforms in (0, 1) from the top 53 bits of SplitMix64."""
    z = splitmix64(seed, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normals(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniforms(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(2.0 * math.pi * u2)
    out[1::2] = r * np.sin(2.0 * math.pi * u2)
    return out[:count]


class Stream:
    """Sequential normal draws from one seed (each call continues the stream)."""

    def __init__(self, seed: int):
        self.seed = seed
        self.pos = 0

    def normals(self, count: int) -> np.ndarray:
        # regenerate the prefix; streams here are short enough for this
        allv = normals(self.seed, self.pos + count)
        out = allv[self.pos:self.pos + count]
        self.pos += count
        return out


def nodes(Q: int) -> np.ndarray:
    x, _ = npleg.leggauss(Q)
    return x


def _grid_eval(d: int, Q: int, coef: np.ndarray) -> np.ndarray:
    """Values of sum c[p0,p1,p2] L_p0(x) L_p1(y) L_p2(z) on the Q^d grid, x fastest.
    ``coef`` is indexed [p0] / [p0, p1] / [p0, p1, p2] (x degree first)."""
    x = nodes(Q)
    if d == 1:
        return npleg.legval(x, coef)
    if d == 2:
        return npleg.leggrid2d(x, x, coef).T.copy()          # [y][x]
    return npleg.leggrid3d(x, x, x, coef).transpose(2, 1, 0).copy()  # [z][y][x]


def legendre_series_coeffs(d: int, deg: int, sigma: float, stream: Stream,
                           power: float = 2.0) -> np.ndarray:
    """c_idx ~ N(0, sigma^2 / (1 + |idx|_1)^power), tensor degree <= deg, x index first."""
    shape = (deg + 1,) * d
    idx = np.indices(shape).sum(axis=0)
    z = stream.normals(int(np.prod(shape))).reshape(shape)
    return sigma * z / (1.0 + idx) ** (power / 2.0)


def exp_series_samples(d: int, Q: int, deg: int, sigma: float, stream: Stream) -> np.ndarray:
    """exp(g) with g a random Legendre series of tensor degree <= deg (positive coefficient)."""
    c = legendre_series_coeffs(d, deg, sigma, stream)
    return np.exp(_grid_eval(d, Q, c)).ravel()


def rhs_coeffs(d: int, N: int, stream: Stream) -> np.ndarray:
    """f coefficients f_idx ~ N(0, 1/(1+|idx|_1)^4) for every index <= N (x index first)."""
    return legendre_series_coeffs(d, N, 1.0, stream, power=4.0)


def rhs_samples_from_coeffs(d: int, Q: int, fc: np.ndarray) -> np.ndarray:
    return _grid_eval(d, Q, fc).ravel()


def coeffs_fastest_first(fc: np.ndarray) -> np.ndarray:
    """Reorder an [p0, p1(, p2)] coefficient array to memory order with p0 fastest."""
    return np.ascontiguousarray(fc.T).ravel()


# --------------------------------------------------------------------------
# Named workloads (problem sizes of the configurations measured)

def manufactured_2d(N: int = 64, T: int = 8, Q: int | None = None) -> dict:
    """2D, a = 1 + 0.5 exp(-(x^2+y^2)), b = 1 + 0.5 x y, u = sin(pi x) sin(pi y) exp(x+y),
    f = -div(a grad u) + b u evaluated analytically at the grid.  Deterministic."""
    Q = N + 2 if Q is None else Q
    x = nodes(Q)
    X, Y = np.meshgrid(x, x, indexing="xy")  # X[j, i] = x_i (x fastest)
    E = np.exp(-(X ** 2 + Y ** 2))
    a = 1.0 + 0.5 * E
    ax = -X * E
    ay = -Y * E
    b = 1.0 + 0.5 * X * Y
    pi = math.pi
    sx, sy = np.sin(pi * X), np.sin(pi * Y)
    cx, cy = np.cos(pi * X), np.cos(pi * Y)
    ex = np.exp(X + Y)
    u = sx * sy * ex
    ux = ex * sy * (pi * cx + sx)
    uy = ex * sx * (pi * cy + sy)
    uxx = ex * sy * (2 * pi * cx + (1 - pi * pi) * sx)
    uyy = ex * sx * (2 * pi * cy + (1 - pi * pi) * sy)
    f = -(a * (uxx + uyy) + ax * ux + ay * uy) + b * u
    return dict(name=f"manufactured-2d-N{N}-T{T}", d=2, N=N, Q=Q, T=T,
                a=a.ravel(), b=b.ravel(), f=f.ravel(), u_exact=u.ravel())


def random_exp_problem(d: int, N: int, T: int, seed_a: int, seed_b: int, seed_f: int,
                       sigma: float = 0.5, coef_deg: int | None = None, Q: int | None = None,
                       f_deg: int | None = None) -> dict:
    """a = exp(g_a), b = exp(g_b), g a random Legendre series (degree coef_deg, default T,
    variance sigma^2/(1+|idx|)^2); f with random Legendre coefficients
    ~ N(0, 1/(1+|idx|)^4) up to degree f_deg (default N)."""
    Q = N + 2 if Q is None else Q
    cd = T if coef_deg is None else coef_deg
    fd = N if f_deg is None else f_deg
    a = exp_series_samples(d, Q, cd, sigma, Stream(seed_a))
    b = exp_series_samples(d, Q, cd, sigma, Stream(seed_b))
    fc = rhs_coeffs(d, fd, Stream(seed_f))
    f = rhs_samples_from_coeffs(d, Q, fc)
    return dict(name=f"exp-series-{d}d-N{N}-T{T}", d=d, N=N, Q=Q, T=T, a=a, b=b, f=f,
                fcoef=coeffs_fastest_first(fc), f_deg=fd, sigma=sigma)


def exp_2d_n512(N: int = 512, T: int = 8) -> dict:
    """2D FP64, N=512 (261,121 unknowns), T=8, seeds 1 (a), 2 (b), 3 (f)."""
    p = random_exp_problem(2, N, T, 1, 2, 3)
    p["name"] = f"2d-exp-series-N{N}-T{T}"
    return p


def exp_3d(N: int = 128, T: int = 6) -> dict:
    """3D, N=128 (~2.05M unknowns), T=6, coefficient degree <= 6, seeds 11-13."""
    p = random_exp_problem(3, N, T, 11, 12, 13, coef_deg=6)
    p["name"] = f"3d-exp-series-N{N}-T{T}"
    return p


def batch_problems(count: int = 256, T: int = 8, seed: int = 21,
                   sizes=tuple(range(32, 257, 16))) -> list:
    """``count`` independent 2D problems, N uniform on ``sizes`` (seed 21); problem i draws
    its a, b and f from the SplitMix64 streams 4*(1000+i) + {0, 1, 2}."""
    u = uniforms(seed, count)
    Ns = [sizes[min(int(v * len(sizes)), len(sizes) - 1)] for v in u]
    out = []
    for i, N in enumerate(Ns):
        s = 4 * (1000 + i)
        out.append(random_exp_problem(2, N, T, s, s + 1, s + 2))
    return out


def serving_stream(count: int, seed: int = 31, rate_hz: float = 100.0,
                   n2d=(64, 1024), n3d=(32, 160), sigma=(0.5, 2.3), frac_2d: float = 0.7,
                   Ts=(4, 8)) -> list:
    """Poisson-arrival request stream: 70% 2D solves with N log-uniform in n2d, 30% 3D
    with N uniform in n3d; T from Ts with equal probability; sigma uniform in the range.
    Each request is (arrival_s, d, N, T, sigma, seed)."""
    u = uniforms(seed, 6 * count).reshape(count, 6)
    t = 0.0
    reqs = []
    for i in range(count):
        t += -math.log(u[i, 0]) / rate_hz
        is2d = u[i, 1] < frac_2d
        if is2d:
            N = int(round(math.exp(math.log(n2d[0]) + u[i, 2] * (math.log(n2d[1]) - math.log(n2d[0])))))
            d = 2
        else:
            N = int(n3d[0] + min(int(u[i, 2] * (n3d[1] - n3d[0] + 1)), n3d[1] - n3d[0]))
            d = 3
        T = Ts[min(int(u[i, 3] * len(Ts)), len(Ts) - 1)]
        sg = sigma[0] + u[i, 4] * (sigma[1] - sigma[0])
        reqs.append(dict(arrival_s=t, d=d, N=N, T=T, sigma=sg, seed=100000 + 4 * i))
    return reqs


def polynomial_coefficient_problem(d: int, N: int, T: int, deg_a: int, deg_b: int,
                                   seed: int, Q: int | None = None) -> dict:
    """a, b positive tensor polynomials of small degree (for exactness checks):
    a = 2 + 0.3 * (random series of degree deg_a), b = 1 + 0.2 * (series of degree deg_b)."""
    Q = N + 2 if Q is None else Q
    st = Stream(seed)
    ca = legendre_series_coeffs(d, deg_a, 1.0, st)
    cb = legendre_series_coeffs(d, deg_b, 1.0, st)
    ca.flat[0] = 0.0
    cb.flat[0] = 0.0
    a = 2.0 + 0.3 * _grid_eval(d, Q, ca).ravel() / max(1.0, np.abs(ca).sum())
    b = 1.0 + 0.2 * _grid_eval(d, Q, cb).ravel() / max(1.0, np.abs(cb).sum())
    fc = rhs_coeffs(d, min(N, 12), st)
    f = rhs_samples_from_coeffs(d, Q, fc)
    return dict(name=f"poly-{d}d-N{N}", d=d, N=N, Q=Q, T=T, a=a, b=b, f=f,
                fcoef=coeffs_fastest_first(fc), f_deg=min(N, 12))


def grid_coords(d: int, Q: int) -> list:
    """Coordinates of the Q^d tensor Gauss grid (x fastest): [x, y, z][:d], each Q^d long."""
    x = nodes(Q)
    mesh = np.meshgrid(*([x] * d), indexing="ij")  # mesh[k] varies along array axis k (axis 0 slowest)
    return [mesh[d - 1 - i].ravel() for i in range(d)]


def paper_example(example: str, d: int, N: int) -> dict:
    """The coefficients of the paper's iteration experiments (Sec. 5, Examples 1-4) on the
    N+1-point Gauss grid the paper uses.  Example "a": beta = (2|x|^2 + 1)^4, alpha =
    cos(x + y + z) (d = 1, 2, 3 as Examples 1-3); "b": beta = exp(2(x + y + z)), alpha = 0;
    "4": Example 4, one coefficient per direction, beta_1 = exp(2x), beta_2 = cos(y),
    beta_3 = cos(z), alpha = 0.  The paper states neither f nor x0: f = 1, x0 = 0 here.
    Returns a (list of d per-direction samples), b, f and Q."""
    Q = N + 1
    g = grid_coords(d, Q)
    s = sum(g)
    if example == "a":
        beta = (2.0 * sum(v * v for v in g) + 1.0) ** 4
        a = [beta] * d
        b = np.cos(s)
    elif example == "b":
        a = [np.exp(2.0 * s)] * d
        b = np.zeros(Q ** d)
    elif example == "4":
        a = [np.exp(2.0 * g[0])] + [np.cos(g[i]) for i in range(1, d)]
        b = np.zeros(Q ** d)
    else:
        raise ValueError(example)
    return dict(name=f"example-{example}-{d}d-N{N}", d=d, N=N, Q=Q, a=a, b=b, f=np.ones(Q ** d))
