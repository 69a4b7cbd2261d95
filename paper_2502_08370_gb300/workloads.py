"""Seeded synthetic inputs for the parareal + splitting solver.

This module generates the input arrays (initial states, diffusion fields,
sources, targets) of the five workloads the library is tested and measured on.
It holds none of the method's arithmetic: it never discretises, splits, solves
or iterates.  It is the one module that both the CUDA path's tests/benchmark
and the FP64 CPU oracle are fed from.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the finaliser constants are the
published ones), mapped to doubles in [0,1) with the top 53 bits, and to
normals by the Box-Muller transform.

Workloads (the paper's experiments use closed-form manufactured solutions,
Sec. 5; these follow the same shapes and value ranges):

* ``heat2d_63``      2-D heat, 63x63 interior, a = 1, f = 0, N = 16, s = 64, T = 1.
                     u0 = sin(pi x) sin(pi y) + 8 random sine modes, A ~ U(-1,1),
                     p, q ~ U{1..63}; tol 1e-10.
* ``heat3d_255``     3-D, 255^3, a = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z) (nodal,
                     boundary included), f = g1(x) g2(y) g3(z) with
                     g_i = sum_{m=1..4} c_{i,m} sin(m pi .), c ~ U(-1,1), constant in time;
                     u0 = sin(pi x) sin(pi y) sin(pi z); N = 64, s = 32, T = 1; tol 1e-8.
* ``dd2d_1023``      2-D, 1023^2, DD splitting 8x8 boxes, overlap 8 cells, a = 1, f = 0,
                     u0 = 16 random sine modes with p, q ~ U{1..32}; N = 32, s = 64,
                     T = 0.5; tol 1e-10.
* ``batch256``       256 2-D problems: nx, ny ~ {63,127,255,511}, N ~ {8,16,32,64},
                     s ~ U{16..128}, T = 1, a = exp(g) with g ~ N(0, 0.25) i.i.d. on the
                     (n+2)^2 nodes smoothed by 4 passes of [1,2,1]/4 per axis
                     (replicated edges); u0 as heat2d with p, q <= min(nx, ny); tol 1e-8.
* ``adjoint2d_511``  2-D, 511^2, a as batch256, u0 as heat2d, N = 32, s = 64, T = 0.05 (so that
                     u(T) stays O(1e-1) and J is resolvable by finite differences).

Every function takes the grid sizes as arguments, so the same recipe also
yields the small cases of the tests.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """SplitMix64 stream: state += golden gamma; output = finaliser(state)."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            idx = np.arange(1, n + 1, dtype=np.uint64)
            z = self.state + idx * _GOLDEN
            self.state = self.state + np.uint64(n) * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Uniform integers in [lo, hi] (inclusive)."""
        u = self.uniform(n)
        return lo + np.minimum((u * (hi - lo + 1)).astype(np.int64), hi - lo)

    def normal(self, n: int) -> np.ndarray:
        u1 = 1.0 - self.uniform(n)  # (0, 1]
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _axis(n: int) -> np.ndarray:
    return np.arange(1, n + 1) / (n + 1.0)


def _axis_with_boundary(n: int) -> np.ndarray:
    return np.arange(0, n + 2) / (n + 1.0)


def sine_sum_2d(nx, ny, amps, ps, qs, base=True):
    """u(x, y) = [sin(pi x) sin(pi y)] + sum_m A_m sin(p_m pi x) sin(q_m pi y), shape (ny, nx)."""
    x, y = _axis(nx), _axis(ny)
    u = np.zeros((ny, nx))
    if base:
        u += np.outer(np.sin(np.pi * y), np.sin(np.pi * x))
    for A, p, q in zip(amps, ps, qs):
        u += A * np.outer(np.sin(q * np.pi * y), np.sin(p * np.pi * x))
    return u


def heat2d_u0(nx, ny, seed=1, modes=8, pmax=None):
    """u0 of the 2-D heat workloads: the base mode plus `modes` random sine modes."""
    r = SplitMix64(seed)
    pmax = pmax if pmax is not None else min(nx, ny)
    amps = r.uniform(modes, -1.0, 1.0)
    ps = r.integers(1, pmax, modes)
    qs = r.integers(1, pmax, modes)
    return sine_sum_2d(nx, ny, amps, ps, qs, base=True), (amps, ps, qs)


def heat2d_63(n=63, N=16, s=64, seed=1):
    u0, modes = heat2d_u0(n, n, seed)
    return dict(n=(n, n), a=None, c=0.0, src=None, src_t=None, u0=u0, T=1.0, N=N, g=1, s=s,
                tol=1e-10, split="dim", modes=modes)


def heat3d_a(nx, ny, nz):
    """a = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z) on the (n+2)^3 nodal grid, shape (nz+2, ny+2, nx+2)."""
    x, y, z = _axis_with_boundary(nx), _axis_with_boundary(ny), _axis_with_boundary(nz)
    return 1.0 + 0.5 * np.einsum("k,j,i->kji", np.sin(2 * np.pi * z), np.sin(2 * np.pi * y), np.sin(2 * np.pi * x))


def heat3d_src(nx, ny, nz, seed=2):
    r = SplitMix64(seed)
    c = r.uniform(12, -1.0, 1.0).reshape(3, 4)
    gs = []
    for d, n in enumerate((nx, ny, nz)):
        x = _axis(n)
        gs.append(sum(c[d, m - 1] * np.sin(m * np.pi * x) for m in range(1, 5)))
    return np.einsum("k,j,i->kji", gs[2], gs[1], gs[0])


def heat3d_u0(nx, ny, nz):
    x, y, z = _axis(nx), _axis(ny), _axis(nz)
    return np.einsum("k,j,i->kji", np.sin(np.pi * z), np.sin(np.pi * y), np.sin(np.pi * x))


def heat3d_255(n=255, N=64, s=32, seed=2):
    nx = ny = nz = n
    return dict(n=(nx, ny, nz), a=heat3d_a(nx, ny, nz), c=0.0, src=heat3d_src(nx, ny, nz, seed), src_t=None,
                u0=heat3d_u0(nx, ny, nz), T=1.0, N=N, g=1, s=s, tol=1e-8, split="dim")


def dd2d_1023(n=1023, boxes=8, overlap_cells=8, N=32, s=64, seed=3, T=0.5):
    r = SplitMix64(seed)
    amps = r.uniform(16, -1.0, 1.0)
    ps = r.integers(1, 32, 16)
    qs = r.integers(1, 32, 16)
    u0 = sine_sum_2d(n, n, amps, ps, qs, base=False)
    return dict(n=(n, n), a=None, c=0.0, src=None, src_t=None, u0=u0, T=T, N=N, g=1, s=s, tol=1e-10,
                split="dd", boxes=(boxes, boxes), overlap=overlap_cells / (n + 1.0))


def smooth_lognormal_a(nx, ny, seed, var=0.25, passes=4):
    """a = exp(g~) on the (ny+2, nx+2) nodal grid; g ~ N(0, var) i.i.d., smoothed by
    `passes` passes of the separable [1,2,1]/4 filter with replicated edges."""
    r = SplitMix64(seed)
    g = np.sqrt(var) * r.normal((nx + 2) * (ny + 2)).reshape(ny + 2, nx + 2)
    for _ in range(passes):
        gp = np.pad(g, ((0, 0), (1, 1)), mode="edge")
        g = 0.25 * gp[:, :-2] + 0.5 * gp[:, 1:-1] + 0.25 * gp[:, 2:]
        gp = np.pad(g, ((1, 1), (0, 0)), mode="edge")
        g = 0.25 * gp[:-2, :] + 0.5 * gp[1:-1, :] + 0.25 * gp[2:, :]
    return np.exp(g)


def batch256(count=256, seed=4, sizes=(63, 127, 255, 511), slices=(8, 16, 32, 64), s_range=(16, 128)):
    """The heterogeneous batch: a list of `count` problem dicts (2-D, dimensional splitting)."""
    r = SplitMix64(seed)
    size_idx = r.integers(0, len(sizes) - 1, 2 * count).reshape(count, 2)
    n_idx = r.integers(0, len(slices) - 1, count)
    s_val = r.integers(s_range[0], s_range[1], count)
    sub_seeds = r.next_u64(count)
    probs = []
    for b in range(count):
        nx, ny = sizes[size_idx[b, 0]], sizes[size_idx[b, 1]]
        ss = int(sub_seeds[b] & np.uint64(0x7FFFFFFF))
        a = smooth_lognormal_a(nx, ny, ss)
        u0, _ = heat2d_u0(nx, ny, ss + 1, pmax=min(nx, ny))
        probs.append(dict(n=(nx, ny), a=a, c=0.0, src=None, src_t=None, u0=u0, T=1.0,
                          N=int(slices[n_idx[b]]), g=1, s=int(s_val[b]), tol=1e-8, split="dim"))
    return probs


def adjoint2d_511(n=511, N=32, s=64, seed=5, T=0.05):
    a = smooth_lognormal_a(n, n, seed)
    u0, _ = heat2d_u0(n, n, seed + 1)
    r = SplitMix64(seed + 2)
    pert = smooth_lognormal_a(n, n, seed + 3, var=1.0)
    a_target = a * (1.0 + 0.1 * (np.log(pert)))
    dirs_seed = int(r.next_u64(1)[0] & np.uint64(0x7FFFFFFF))
    return dict(n=(n, n), a=a, c=0.0, src=None, src_t=None, u0=u0, T=T, N=N, g=1, s=s, tol=1e-10,
                split="dim", a_target=a_target, dirs_seed=dirs_seed)


def random_directions(shape, count, seed):
    """`count` seeded unit directions (Frobenius norm 1) of the given shape."""
    r = SplitMix64(seed)
    out = []
    for _ in range(count):
        v = r.normal(int(np.prod(shape))).reshape(shape)
        out.append(v / np.linalg.norm(v))
    return out


def manufactured(n, T, N, s):
    """Manufactured solution of Sec. 5: u = sin(2 pi t) sin(2 pi x) sin(2 pi y), D = I.
    f = sin(2 pi x) sin(2 pi y) [2 pi cos(2 pi t) + 8 pi^2 sin(2 pi t)] is separable:
    returns (src on the interior grid, src_t at the fine times j T/(N s), exact(t))."""
    nx, ny = n
    x, y = _axis(nx), _axis(ny)
    S = np.outer(np.sin(2 * np.pi * y), np.sin(2 * np.pi * x))
    t = np.arange(N * s + 1) * (T / (N * s))
    st = 2 * np.pi * np.cos(2 * np.pi * t) + 8 * np.pi ** 2 * np.sin(2 * np.pi * t)

    def exact(tt):
        return np.sin(2 * np.pi * tt) * S

    return S, st, exact


def full_tensor_coefficients(nx, ny):
    """Diffusion tensor of Sec. 5.2 on the (ny+2, nx+2) nodal grid (boundary included):
    d11 = d22 = 1 / (2 + cos(3 pi x) cos(2 pi y)), d12 = 1/4.  Returns (d11, d12)."""
    x, y = _axis_with_boundary(nx), _axis_with_boundary(ny)
    d = 1.0 / (2.0 + np.outer(np.cos(2 * np.pi * y), np.cos(3 * np.pi * x)))
    return d, np.full_like(d, 0.25)


def full_tensor_div_grad_S(x, y):
    """div(D grad S) for S = sin(2 pi x) sin(2 pi y) and the tensor of Sec. 5.2, in closed form:
    d (S_xx + S_yy) + d_x S_x + d_y S_y + 2 d12 S_xy, d = 1/g, g = 2 + cos(3 pi x) cos(2 pi y)."""
    X, Y = np.meshgrid(x, y)
    tp = 2 * np.pi
    g = 2.0 + np.cos(3 * np.pi * X) * np.cos(tp * Y)
    d = 1.0 / g
    gx = -3 * np.pi * np.sin(3 * np.pi * X) * np.cos(tp * Y)
    gy = -tp * np.cos(3 * np.pi * X) * np.sin(tp * Y)
    S = np.sin(tp * X) * np.sin(tp * Y)
    Sx = tp * np.cos(tp * X) * np.sin(tp * Y)
    Sy = tp * np.sin(tp * X) * np.cos(tp * Y)
    Sxy = tp * tp * np.cos(tp * X) * np.cos(tp * Y)
    return d * (-2 * tp * tp * S) - gx / g ** 2 * Sx - gy / g ** 2 * Sy + 2 * 0.25 * Sxy


def manufactured_full_tensor(n, T, N, s):
    """Manufactured problem of Sec. 5.2: u = sin(2 pi t) sin(2 pi x) sin(2 pi y) with the full
    tensor above, f = u_t - div(D grad u) = S 2 pi cos(2 pi t) - div(D grad S) sin(2 pi t): two
    separable terms.  Returns dict(a, d12, src, src_t, src2, src2_t, exact)."""
    nx, ny = n
    x, y = _axis(nx), _axis(ny)
    S = np.outer(np.sin(2 * np.pi * y), np.sin(2 * np.pi * x))
    t = np.arange(N * s + 1) * (T / (N * s))
    a, d12 = full_tensor_coefficients(nx, ny)

    def exact(tt):
        return np.sin(2 * np.pi * tt) * S

    return dict(a=a, d12=d12, src=S, src_t=2 * np.pi * np.cos(2 * np.pi * t), src2=-full_tensor_div_grad_S(x, y),
                src2_t=np.sin(2 * np.pi * t), exact=exact)
