"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the FastVPINNs method itself: it makes
meshes (vertex coordinates + 4-vertex cells), boundary and sensor points,
MLP parameter vectors and the closed-form exact solutions / source terms of
the model problems.  Quadrature, test functions, the bilinear map, the MLP,
the residual and the loss live elsewhere (the oracle and the CUDA library
each have their own).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here from its
published definition.  A generator is addressed by (seed, stream); the
stream numbers are fixed by convention:

    0 = mesh jitter, 1 = MLP init, 2 = sensors, 3 = batch draws,
    100 + i = MLP of batch instance i.

Problem family (paper Sec. 2.1, Eq. CD2D_strong):  -eps*Lap(u) + b.grad(u) = f
in Omega, u = g on the boundary.  Poisson is eps = 1, b = 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    """SplitMix64: state += golden gamma; output = mix64(state).

    (seed, stream) -> initial state mix64(seed + golden*(stream+1)) mod 2^64,
    so that distinct streams of one seed start far apart.
    """

    def __init__(self, seed: int, stream: int = 0):
        self.state = _mix64((seed + GOLDEN * (stream + 1)) & MASK64)

    def next_u64(self) -> int:
        self.state = (self.state + GOLDEN) & MASK64
        return _mix64(self.state)

    def uniform(self) -> float:
        """Double in [0, 1): top 53 bits times 2^-53."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniforms(self, n: int) -> np.ndarray:
        return np.array([self.uniform() for _ in range(n)], dtype=np.float64)


# ----------------------------------------------------------------------------
# MLP parameters.  Flat layout, layer by layer: W (row-major [out][in]) then b.
# ----------------------------------------------------------------------------

def mlp_param_count(widths: List[int]) -> int:
    return sum(widths[i + 1] * widths[i] + widths[i + 1] for i in range(len(widths) - 1))


def glorot_params(widths: List[int], seed: int, stream: int = 1, gain: float = 1.0) -> np.ndarray:
    """Glorot-uniform weights U(+-gain*sqrt(6/(n_in+n_out))), biases 0.

    Draw order: layer by layer, W row-major [out][in].
    """
    rng = SplitMix64(seed, stream)
    out = []
    for i in range(len(widths) - 1):
        n_in, n_out = widths[i], widths[i + 1]
        a = gain * math.sqrt(6.0 / (n_in + n_out))
        w = (2.0 * rng.uniforms(n_out * n_in) - 1.0) * a
        out.append(w)
        out.append(np.zeros(n_out))
    return np.concatenate(out)


def random_bias_params(widths: List[int], seed: int, stream: int = 1, gain: float = 1.0,
                       bias_scale: float = 0.3) -> np.ndarray:
    """Glorot weights plus non-zero uniform biases U(+-bias_scale) (used so
    that bias gradients are exercised at non-trivial values)."""
    rng = SplitMix64(seed, stream)
    out = []
    for i in range(len(widths) - 1):
        n_in, n_out = widths[i], widths[i + 1]
        a = gain * math.sqrt(6.0 / (n_in + n_out))
        out.append((2.0 * rng.uniforms(n_out * n_in) - 1.0) * a)
        out.append((2.0 * rng.uniforms(n_out) - 1.0) * bias_scale)
    return np.concatenate(out)


# ----------------------------------------------------------------------------
# Meshes.  vertices: (n_v, 2) float64; cells: (n_e, 4) int32, counter-clockwise
# b0, b1, b2, b3 (reference corners (-1,-1), (1,-1), (1,1), (-1,1)).
# ----------------------------------------------------------------------------

@dataclass
class Mesh:
    vertices: np.ndarray
    cells: np.ndarray

    @property
    def n_elements(self) -> int:
        return int(self.cells.shape[0])

    def subset(self, lo: int, hi: int) -> "Mesh":
        return Mesh(self.vertices, np.ascontiguousarray(self.cells[lo:hi]))


def rect_grid(nx: int, ny: int, x0=0.0, x1=1.0, y0=0.0, y1=1.0) -> Mesh:
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(xs, ys)  # [j][i]
    verts = np.stack([X.ravel(), Y.ravel()], axis=1)
    cells = []
    for j in range(ny):
        for i in range(nx):
            n0 = j * (nx + 1) + i
            cells.append([n0, n0 + 1, n0 + nx + 2, n0 + nx + 1])
    return Mesh(np.ascontiguousarray(verts, dtype=np.float64), np.array(cells, dtype=np.int32))


def _incident_min_edge(verts: np.ndarray, cells: np.ndarray) -> np.ndarray:
    h = np.full(verts.shape[0], np.inf)
    for c in cells:
        for k in range(4):
            a, b = c[k], c[(k + 1) % 4]
            d = float(np.hypot(*(verts[a] - verts[b])))
            h[a] = min(h[a], d)
            h[b] = min(h[b], d)
    return h


def jitter_nodes(mesh: Mesh, movable: np.ndarray, frac: float, seed: int,
                 h_fixed: Optional[float] = None) -> Mesh:
    """Move each movable node by U(-frac, frac)*h in x and y independently
    (node order, x then y; stream 0).  h = h_fixed, else the shortest edge
    incident to the node (measured before any node moves)."""
    rng = SplitMix64(seed, 0)
    v = mesh.vertices.copy()
    h = np.full(v.shape[0], h_fixed) if h_fixed is not None else _incident_min_edge(mesh.vertices, mesh.cells)
    for n in range(v.shape[0]):
        if not movable[n]:
            continue
        dx = (2.0 * rng.uniform() - 1.0) * frac * h[n]
        dy = (2.0 * rng.uniform() - 1.0) * frac * h[n]
        v[n, 0] += dx
        v[n, 1] += dy
    return Mesh(v, mesh.cells)


def disc_butterfly(n_core: int = 16, n_rad: int = 12, core_half: float = 0.5) -> Mesh:
    """Unit-disc O-grid: an n_core x n_core core square [-h, h]^2 plus four
    outer blocks (n_core tangential x n_rad radial) blending each core edge
    linearly to its quarter arc of the unit circle.  Core corners map to the
    angles 45 + 90k degrees.  n_core=16, n_rad=12 gives 1024 quads."""
    nc = n_core
    verts = []
    for j in range(nc + 1):
        for i in range(nc + 1):
            verts.append((-core_half + 2 * core_half * i / nc, -core_half + 2 * core_half * j / nc))

    def core_id(i, j):
        return j * (nc + 1) + i

    def edge_core(k, i):
        # core node at position i (CCW) along edge k: 0 right, 1 top, 2 left, 3 bottom
        if k == 0:
            return core_id(nc, i)
        if k == 1:
            return core_id(nc - i, nc)
        if k == 2:
            return core_id(0, nc - i)
        return core_id(i, 0)

    outer = {}  # (k, i, r) -> node id for r >= 1, i in [0, nc)
    for k in range(4):
        for r in range(1, n_rad + 1):
            for i in range(nc):
                p = np.array(verts[edge_core(k, i)])
                th = math.radians(-45.0 + 90.0 * k) + (math.pi / 2) * i / nc
                a = np.array([math.cos(th), math.sin(th)])
                s = r / n_rad
                q = (1 - s) * p + s * a
                outer[(k, i, r)] = len(verts)
                verts.append((float(q[0]), float(q[1])))

    def node(k, i, r):
        if i == nc:
            k, i = (k + 1) % 4, 0
        if r == 0:
            return edge_core(k, i)
        return outer[(k, i, r)]

    cells = []
    for j in range(nc):
        for i in range(nc):
            cells.append([core_id(i, j), core_id(i + 1, j), core_id(i + 1, j + 1), core_id(i, j + 1)])
    for k in range(4):
        for r in range(n_rad):
            for i in range(nc):
                # xi radial (outwards), eta tangential (counter-clockwise)
                cells.append([node(k, i, r), node(k, i, r + 1), node(k, i + 1, r + 1), node(k, i + 1, r)])
    return Mesh(np.array(verts, dtype=np.float64), np.array(cells, dtype=np.int32))


def annulus_ogrid(n_theta: int = 128, n_r: int = 64, r_in: float = 0.5,
                  R: Callable[[np.ndarray], np.ndarray] = lambda th: 1.0 + 0.1 * np.cos(12 * th)) -> Mesh:
    """Annulus r_in <= r <= R(theta): node (j, i) at r = r_in + (R(theta_i)-r_in) j/n_r,
    theta_i = 2 pi i / n_theta.  Cells have xi radial and eta angular."""
    verts = np.zeros(((n_r + 1) * n_theta, 2))
    for j in range(n_r + 1):
        for i in range(n_theta):
            th = 2 * math.pi * i / n_theta
            r = r_in + (float(R(np.array(th))) - r_in) * j / n_r
            verts[j * n_theta + i] = (r * math.cos(th), r * math.sin(th))
    cells = []
    for j in range(n_r):
        for i in range(n_theta):
            i1 = (i + 1) % n_theta
            cells.append([j * n_theta + i, (j + 1) * n_theta + i, (j + 1) * n_theta + i1, j * n_theta + i1])
    return Mesh(verts, np.array(cells, dtype=np.int32))


def boundary_nodes_of(mesh: Mesh) -> np.ndarray:
    """Mask of nodes on the mesh boundary (edges used by exactly one cell)."""
    count = {}
    for c in mesh.cells:
        for k in range(4):
            a, b = int(c[k]), int(c[(k + 1) % 4])
            key = (min(a, b), max(a, b))
            count[key] = count.get(key, 0) + 1
    mask = np.zeros(mesh.vertices.shape[0], dtype=bool)
    for (a, b), n in count.items():
        if n == 1:
            mask[a] = mask[b] = True
    return mask


# ----------------------------------------------------------------------------
# Exact solutions and source terms (closed forms of the model problems).
# ----------------------------------------------------------------------------

def sinsin(omega: float):
    """u = sin(w x) sin(w y); -Lap u = 2 w^2 u."""
    u = lambda x, y: np.sin(omega * x) * np.sin(omega * y)
    f = lambda x, y: 2.0 * omega * omega * np.sin(omega * x) * np.sin(omega * y)
    return u, f


def sincos(omega: float):
    """u = sin(w x) cos(w y); -Lap u = 2 w^2 u."""
    u = lambda x, y: np.sin(omega * x) * np.cos(omega * y)
    f = lambda x, y: 2.0 * omega * omega * np.sin(omega * x) * np.cos(omega * y)
    return u, f


def inverse_exact(eps_true: float = 0.3, a: float = 0.3, bx: float = 0.1):
    """u = 10 sin(x) tanh(x) exp(-a x^2) (depends on x only; paper Sec. 4.7.1)
    and f = -eps u'' + bx u' with hand-derived u', u''."""
    def parts(x):
        s, c, t = np.sin(x), np.cos(x), np.tanh(x)
        sech2 = 1.0 - t * t
        E = np.exp(-a * x * x)
        g = c * t + s * sech2 - 2.0 * a * x * s * t
        gp = (-s * t + 2.0 * c * sech2 - 2.0 * s * t * sech2
              - 2.0 * a * (s * t + x * c * t + x * s * sech2))
        u = 10.0 * s * t * E
        up = 10.0 * E * g
        upp = 10.0 * E * (-2.0 * a * x * g + gp)
        return u, up, upp

    u = lambda x, y: parts(np.asarray(x, dtype=np.float64))[0] + 0.0 * np.asarray(y)
    up = lambda x, y: parts(np.asarray(x, dtype=np.float64))[1] + 0.0 * np.asarray(y)
    upp = lambda x, y: parts(np.asarray(x, dtype=np.float64))[2] + 0.0 * np.asarray(y)
    f = lambda x, y: -eps_true * upp(x, y) + bx * up(x, y)
    return u, f, up, upp


# ----------------------------------------------------------------------------
# Boundary / sensor point sets.
# ----------------------------------------------------------------------------

def square_boundary_points(n_per_side: int, x0=0.0, x1=1.0, y0=0.0, y1=1.0) -> np.ndarray:
    """n_per_side points per side at t = k/n_per_side, counter-clockwise from
    (x0, y0); each corner appears once."""
    t = np.arange(n_per_side) / n_per_side
    pts = [np.stack([x0 + (x1 - x0) * t, np.full_like(t, y0)], 1),
           np.stack([np.full_like(t, x1), y0 + (y1 - y0) * t], 1),
           np.stack([x1 - (x1 - x0) * t, np.full_like(t, y1)], 1),
           np.stack([np.full_like(t, x0), y1 - (y1 - y0) * t], 1)]
    return np.ascontiguousarray(np.concatenate(pts), dtype=np.float64)


def circle_points(n: int, r=1.0) -> np.ndarray:
    th = 2 * np.pi * np.arange(n) / n
    return np.ascontiguousarray(np.stack([r * np.cos(th), r * np.sin(th)], 1))


def annulus_boundary_points(n_per_curve: int, r_in=0.5) -> np.ndarray:
    th = 2 * np.pi * np.arange(n_per_curve) / n_per_curve
    R = 1.0 + 0.1 * np.cos(12 * th)
    inner = np.stack([r_in * np.cos(th), r_in * np.sin(th)], 1)
    outer = np.stack([R * np.cos(th), R * np.sin(th)], 1)
    return np.ascontiguousarray(np.concatenate([inner, outer]))


def uniform_points(n: int, seed: int, stream: int, lo=-1.0, hi=1.0) -> np.ndarray:
    rng = SplitMix64(seed, stream)
    u = rng.uniforms(2 * n).reshape(n, 2)
    return np.ascontiguousarray(lo + (hi - lo) * u)


# ----------------------------------------------------------------------------
# The five workload configurations.
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    name: str
    mesh: Mesh
    quad_order: int          # Q: GLL points per direction
    test_order: int          # T: test functions per direction
    widths: List[int]        # [2, h1, ..., hH, 1]
    params: np.ndarray       # flat float64
    u_exact: Callable
    f: Callable
    bd_xy: np.ndarray
    bd_g: np.ndarray
    eps: float = 1.0
    b: tuple = (0.0, 0.0)
    tau: float = 10.0
    sensor_xy: np.ndarray = field(default_factory=lambda: np.zeros((0, 2)))
    sensor_u: np.ndarray = field(default_factory=lambda: np.zeros(0))
    gamma: float = 10.0
    precision: str = "fp64"

    @property
    def n_points(self) -> int:
        return self.mesh.n_elements * self.quad_order ** 2


def tiny_square() -> Problem:
    """Poisson on [0,1]^2, 4x4 uniform quads, Q=5, T=5, MLP 2-30-30-30-1
    (Glorot, seed 0), 400 boundary points, FP64."""
    mesh = rect_grid(4, 4)
    u, f = sinsin(2 * math.pi)
    widths = [2, 30, 30, 30, 1]
    bd = square_boundary_points(100)
    return Problem("tiny-poisson-4x4", mesh, 5, 5, widths, glorot_params(widths, 0, 1), u, f,
                   bd, u(bd[:, 0], bd[:, 1]), precision="fp64")


def skewed_disc() -> Problem:
    """Poisson on the unit disc, 1024-quad butterfly O-grid, interior nodes
    jittered +-0.2 h (seed 1), Q=8, T=6, u = sin(4 pi x) cos(4 pi y),
    MLP 2-30x3-1 (seed 1), 1000 boundary points on the circle, FP32."""
    base = disc_butterfly(16, 12)
    movable = ~boundary_nodes_of(base)
    mesh = jitter_nodes(base, movable, 0.2, seed=1)
    u, f = sincos(4 * math.pi)
    widths = [2, 30, 30, 30, 1]
    bd = circle_points(1000)
    return Problem("skewed-disc-1024", mesh, 8, 6, widths, glorot_params(widths, 1, 1), u, f,
                   bd, u(bd[:, 0], bd[:, 1]), precision="fp32")


def gear_annulus() -> Problem:
    """Poisson on the gear-like annulus 0.5 <= r <= 1 + 0.1 cos(12 theta),
    128 x 64 O-grid (8192 quads), Q=10, T=8, u = sin(8 pi x) sin(8 pi y),
    MLP 2-50x4-1 (seed 0), 1000 boundary points (500 per curve)."""
    mesh = annulus_ogrid(128, 64)
    u, f = sinsin(8 * math.pi)
    widths = [2, 50, 50, 50, 50, 1]
    bd = annulus_boundary_points(500)
    return Problem("gear-annulus-8192", mesh, 10, 8, widths, glorot_params(widths, 0, 1), u, f,
                   bd, u(bd[:, 0], bd[:, 1]), precision="fp32")


def inverse_cd2d(n: int = 256) -> Problem:
    """Inverse CD2D: -eps Lap u + b.grad u = f on [-1,1]^2, n x n quads with
    interior nodes jittered +-0.15 h (h = 2/n, seed 3), Q=5, T=5, b=(0.1,0),
    eps trainable (true 0.3, start 2.0), u = 10 sin x tanh x exp(-0.3 x^2),
    1000 boundary points, 500 sensors (seed 3, stream 2), MLP 2-30x3-1."""
    base = rect_grid(n, n, -1.0, 1.0, -1.0, 1.0)
    movable = ~boundary_nodes_of(base)
    mesh = jitter_nodes(base, movable, 0.15, seed=3, h_fixed=2.0 / n)
    u, f, _, _ = inverse_exact(0.3, 0.3, 0.1)
    widths = [2, 30, 30, 30, 1]
    bd = square_boundary_points(250, -1, 1, -1, 1)
    sens = uniform_points(500, 3, 2)
    return Problem("inverse-cd2d-%dx%d" % (n, n), mesh, 5, 5, widths, glorot_params(widths, 3, 1), u, f,
                   bd, u(bd[:, 0], bd[:, 1]), eps=2.0, b=(0.1, 0.0), tau=10.0,
                   sensor_xy=sens, sensor_u=u(sens[:, 0], sens[:, 1]), gamma=10.0, precision="fp32")


def poisson_batch(n_instances: int = 64, seed: int = 4) -> List[Problem]:
    """64 Poisson instances on uniform grids of [0,1]^2; per instance draw
    (stream 3, in order) N_e log-uniform in [100, 16384], Q = 5 + floor(6U),
    T = 4 + floor(5U); separate MLP 2-30x3-1 per instance (stream 100+i)."""
    rng = SplitMix64(seed, 3)
    u, f = sinsin(2 * math.pi)
    widths = [2, 30, 30, 30, 1]
    bd = square_boundary_points(100)
    out = []
    for i in range(n_instances):
        ue = rng.uniform()
        ne = int(round(math.exp(math.log(100.0) + ue * math.log(163.84))))
        Q = 5 + int(math.floor(6 * rng.uniform()))
        T = 4 + int(math.floor(5 * rng.uniform()))
        nx = max(1, int(round(math.sqrt(ne))))
        ny = max(1, int(round(ne / nx)))
        mesh = rect_grid(nx, ny)
        out.append(Problem("batch-%02d" % i, mesh, Q, T, widths, glorot_params(widths, seed, 100 + i), u, f,
                           bd, u(bd[:, 0], bd[:, 1]), precision="fp32"))
    return out


def eps_field_disc() -> Problem:
    """Space-dependent diffusion (Sec. 4.7.2): -div(eps(x, y) grad u) + b . grad u = f
    on the skewed 1024-element disc (Q=8, T=6), f = 10, b = (1, 0); one
    network 2-30x3-2 with outputs (u, eps) (seed 5); 1000 boundary points with
    g = 0 and 500 sensors (seed 5, stream 2) in the disc.  The paper's sensor
    data come from a finite-element reference that is not available; the
    synthetic observations are u_obs = 5 (1 - x^2 - y^2), the solution of
    -0.5 Lap u = 10 with u = 0 on the circle."""
    base = disc_butterfly(16, 12)
    mesh = jitter_nodes(base, ~boundary_nodes_of(base), 0.2, seed=1)
    widths = [2, 30, 30, 30, 2]
    u_obs = lambda x, y: 5.0 * (1.0 - x * x - y * y)
    f = lambda x, y: 10.0 + 0.0 * x
    bd = circle_points(1000)
    r = np.sqrt(SplitMix64(5, 2).uniforms(500))
    th = 2 * math.pi * SplitMix64(5, 3).uniforms(500)
    sens = np.stack([0.95 * r * np.cos(th), 0.95 * r * np.sin(th)], axis=1)
    return Problem("eps-field-disc-1024", mesh, 8, 6, widths, glorot_params(widths, 5, 1), u_obs, f,
                   bd, np.zeros(len(bd)), eps=1.0, b=(1.0, 0.0), tau=10.0,
                   sensor_xy=sens, sensor_u=u_obs(sens[:, 0], sens[:, 1]), gamma=10.0, precision="fp32")


WORKLOADS = {"tiny": tiny_square, "disc": skewed_disc, "annulus": gear_annulus, "inverse": inverse_cd2d}
