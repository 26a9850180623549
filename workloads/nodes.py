"""Seeded node sets shaped like the cube, sphere and casing workloads.

Every generator returns a :class:`NodeSet` whose rows are ordered interior
nodes first, then boundary (Dirichlet) nodes, matching the block order of the
collocation system [H; R] (Sec. 2.1, eq. augmented_system).  Centres and
collocation points coincide (Sec. 2.1, collocation framework).

Seeds: a workload preset numbered ``i`` draws from
``numpy.random.Generator(PCG64(9798 + i))``; its evaluation points from
``PCG64(9798 + i + 1000)``; batch instance ``b`` from ``PCG64(9798 + 400 + b)``.
The paper's own node sets came from Gmsh meshes that are not available, so
these synthetic sets stand in for them (Sec. 5, experimental setup).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 9798


@dataclass
class NodeSet:
    """Collocation nodes X (N x 3, float64, interior rows first)."""

    X: np.ndarray
    n_interior: int
    domain: str
    name: str = ""
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_boundary(self) -> int:
        return self.n - self.n_interior

    def soa(self) -> np.ndarray:
        """Structure-of-arrays copy [3][N] (x row, y row, z row), float64."""
        return np.ascontiguousarray(self.X.T)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------
# low-level point sets
# ----------------------------------------------------------------------------

def _grid_axis(n: int) -> np.ndarray:
    return np.linspace(0.0, 1.0, n)


def _lex(P: np.ndarray) -> np.ndarray:
    order = np.lexsort((P[:, 2], P[:, 1], P[:, 0]))
    return P[order]


def cube_face_grid(n_f: int) -> np.ndarray:
    """Unique points of an n_f x n_f grid on each of the 6 faces of [0,1]^3.

    Edge and corner points shared by two or three faces appear once, so the
    count is n_f^3 - (n_f - 2)^3.
    """
    g = _grid_axis(n_f)
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    on_b = np.any((P == 0.0) | (P == 1.0), axis=1)
    return _lex(P[on_b])


def scrambled_halton(n: int, rng: np.random.Generator, bases=(2, 3, 5),
                     skip: int = 1) -> np.ndarray:
    """Halton points with a random digit permutation per base and per digit.

    Point ``i`` (``i = skip .. skip+n-1``) has coordinate
    ``sum_d pi_{b,d}(a_d(i)) b^{-(d+1)}`` over enough digits d to resolve
    double precision, where ``a_d(i)`` are the base-b digits of i.
    """
    out = np.empty((n, len(bases)))
    idx = np.arange(skip, skip + n, dtype=np.int64)
    for col, b in enumerate(bases):
        ndig = int(math.ceil(53 * math.log(2) / math.log(b)))
        perms = [rng.permutation(b) for _ in range(ndig)]
        x = np.zeros(n)
        rem = idx.copy()
        scale = 1.0 / b
        for d in range(ndig):
            digit = rem % b
            rem //= b
            x += perms[d][digit] * scale
            scale /= b
        out[:, col] = x
    return out


def fibonacci_sphere(n: int) -> np.ndarray:
    """Fibonacci lattice on the unit sphere: z_i = 1-(2i+1)/n, phi_i = i*pi*(3-sqrt5)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def uniform_ball(n: int, rng: np.random.Generator, radius: float = 1.0) -> np.ndarray:
    """n points uniform in the open ball, by rejection from the cube [-r, r]^3."""
    pts = []
    have = 0
    while have < n:
        P = rng.uniform(-radius, radius, size=(max(2 * (n - have), 64), 3))
        P = P[np.sum(P * P, axis=1) < radius * radius]
        pts.append(P)
        have += P.shape[0]
    return np.concatenate(pts)[:n]


def uniform_cube(n: int, rng: np.random.Generator) -> np.ndarray:
    """n points uniform in the open unit cube (0,1)^3."""
    P = rng.uniform(0.0, 1.0, size=(n, 3))
    # uniform() samples [0,1); a coordinate of exactly 0 would sit on a face
    P[P == 0.0] = 0.5
    return P


# ----------------------------------------------------------------------------
# workload node sets
# ----------------------------------------------------------------------------

def cube_grid(n_side: int = 10) -> NodeSet:
    """n_side^3 uniform grid on [0,1]^3; faces are Dirichlet nodes."""
    g = _grid_axis(n_side)
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    on_b = np.any((P == 0.0) | (P == 1.0), axis=1)
    X = np.concatenate([_lex(P[~on_b]), _lex(P[on_b])])
    return NodeSet(np.ascontiguousarray(X), int((~on_b).sum()), "cube",
                   f"cube_grid{n_side ** 3}")


def cube_faces_halton(n: int = 8000, n_f: int = 21, seed: int = BASE_SEED + 2) -> NodeSet:
    """Face-grid boundary (n_f per edge) + scrambled 3D Halton interior filling to n."""
    B = cube_face_grid(n_f)
    n_int = n - B.shape[0]
    if n_int < 0:
        raise ValueError("boundary grid larger than n")
    rng = _rng(seed)
    I = scrambled_halton(n_int, rng)
    X = np.concatenate([I, B])
    return NodeSet(np.ascontiguousarray(X), n_int, "cube", f"cube_halton{n}")


def cube_faces_random(n: int, boundary_share: float, rng: np.random.Generator) -> NodeSet:
    """Face grid with n_f = round(sqrt(share*n/6)) + 1 per edge, uniform interior."""
    n_f = int(round(math.sqrt(boundary_share * n / 6.0))) + 1
    B = cube_face_grid(n_f)
    n_int = n - B.shape[0]
    I = uniform_cube(n_int, rng)
    return NodeSet(np.ascontiguousarray(np.concatenate([I, B])), n_int, "cube",
                   f"cube_random{n}")


def sphere_fibonacci_ball(n_boundary: int = 4000, n_interior: int = 16000,
                          seed: int = BASE_SEED + 3) -> NodeSet:
    """Fibonacci lattice on r=1 + uniform interior of the open unit ball."""
    rng = _rng(seed)
    I = uniform_ball(n_interior, rng)
    B = fibonacci_sphere(n_boundary)
    return NodeSet(np.ascontiguousarray(np.concatenate([I, B])), n_interior,
                   "sphere", f"sphere{n_boundary + n_interior}")


# --- pump-casing-like union: cylinder + log-spiral volute tube + outlet pipe ----

_CYL_R, _CYL_H = 0.5, 0.4
_SP_A, _SP_B = 0.5, 0.15
_TUBE_R0, _TUBE_R1 = 0.1, 0.3
_PIPE_R, _PIPE_L = 0.25, 0.6


def _spiral(theta):
    R = _SP_A * np.exp(_SP_B * theta)
    return np.stack([R * np.cos(theta), R * np.sin(theta), np.zeros_like(theta)], axis=-1)


def _spiral_d(theta):
    R = _SP_A * np.exp(_SP_B * theta)
    dR = _SP_B * R
    return np.stack([dR * np.cos(theta) - R * np.sin(theta),
                     dR * np.sin(theta) + R * np.cos(theta), np.zeros_like(theta)], axis=-1)


def _tube_radius(theta):
    return _TUBE_R0 + (_TUBE_R1 - _TUBE_R0) * theta / (2.0 * math.pi)


_TH_S = np.linspace(0.0, 2.0 * math.pi, 1201)
_C_S = _spiral(_TH_S)
_R_S = _tube_radius(_TH_S)
_P0 = _spiral(np.array([2.0 * math.pi]))[0]
_T0 = _spiral_d(np.array([2.0 * math.pi]))[0]
_T0 = _T0 / np.linalg.norm(_T0)


def _in_cyl(P):
    return (P[:, 0] ** 2 + P[:, 1] ** 2 < _CYL_R ** 2) & (np.abs(P[:, 2]) < _CYL_H / 2)


def _in_tube(P):
    out = np.zeros(P.shape[0], dtype=bool)
    for s in range(0, P.shape[0], 4096):
        Q = P[s:s + 4096]
        d = np.sqrt(((Q[:, None, :] - _C_S[None, :, :]) ** 2).sum(-1)) - _R_S[None, :]
        out[s:s + 4096] = d.min(axis=1) < 0.0
    return out


def _in_pipe(P):
    v = P - _P0
    t = v @ _T0
    perp = v - t[:, None] * _T0[None, :]
    return (t > 0.0) & (t < _PIPE_L) & (np.sum(perp * perp, axis=1) < _PIPE_R ** 2)


def _in_pump(P):
    return _in_cyl(P) | _in_tube(P) | _in_pipe(P)


def _sample_cyl_surface(m, rng):
    lat, cap = 2 * math.pi * _CYL_R * _CYL_H, math.pi * _CYL_R ** 2
    w = np.array([lat, cap, cap])
    part = rng.choice(3, size=m, p=w / w.sum())
    P = np.empty((m, 3))
    th = rng.uniform(0, 2 * math.pi, m)
    z = rng.uniform(-_CYL_H / 2, _CYL_H / 2, m)
    rr = _CYL_R * np.sqrt(rng.uniform(0, 1, m))
    lat_m = part == 0
    P[lat_m] = np.stack([_CYL_R * np.cos(th), _CYL_R * np.sin(th), z], 1)[lat_m]
    for k, zc in ((1, -_CYL_H / 2), (2, _CYL_H / 2)):
        msk = part == k
        P[msk] = np.stack([rr * np.cos(th), rr * np.sin(th), np.full(m, zc)], 1)[msk]
    return P


def _sample_tube_surface(m, rng):
    # area density along theta ~ 2*pi*rho(theta)*|c'(theta)|
    dens = 2 * math.pi * _R_S * np.linalg.norm(_spiral_d(_TH_S), axis=1)
    cdf = np.cumsum(dens)
    cdf /= cdf[-1]
    th = np.interp(rng.uniform(0, 1, m), cdf, _TH_S)
    c = _spiral(th)
    t = _spiral_d(th)
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    nrm = np.stack([t[:, 1], -t[:, 0], np.zeros(m)], 1)
    b = np.tile(np.array([0.0, 0.0, 1.0]), (m, 1))
    psi = rng.uniform(0, 2 * math.pi, m)
    rho = _tube_radius(th)
    return c + rho[:, None] * (np.cos(psi)[:, None] * nrm + np.sin(psi)[:, None] * b)


def _sample_pipe_surface(m, rng):
    lat, cap = 2 * math.pi * _PIPE_R * _PIPE_L, math.pi * _PIPE_R ** 2
    u = np.cross(_T0, np.array([0.0, 0.0, 1.0]))
    u /= np.linalg.norm(u)
    v = np.cross(_T0, u)
    is_cap = rng.uniform(0, 1, m) < cap / (lat + cap)
    psi = rng.uniform(0, 2 * math.pi, m)
    t = np.where(is_cap, _PIPE_L, rng.uniform(0, _PIPE_L, m))
    r = np.where(is_cap, _PIPE_R * np.sqrt(rng.uniform(0, 1, m)), _PIPE_R)
    return (_P0[None, :] + t[:, None] * _T0[None, :]
            + r[:, None] * (np.cos(psi)[:, None] * u + np.sin(psi)[:, None] * v))


def pump_like(n_boundary: int = 8000, n_interior: int = 32000,
              seed: int = BASE_SEED + 5) -> NodeSet:
    """Casing-like union: cylinder (r=0.5, h=0.4), volute tube on the log spiral
    R = 0.5 e^{0.15 theta} (tube radius 0.1 -> 0.3), outlet pipe (r=0.25, L=0.6).

    Boundary nodes: area-proportional samples of each part's surface, keeping
    only those not inside another part.  Interior nodes: rejection sampling of
    the union from its bounding box.
    """
    rng = _rng(seed)
    areas = np.array([2 * math.pi * _CYL_R * _CYL_H + 2 * math.pi * _CYL_R ** 2,
                      float(np.trapezoid(2 * math.pi * _R_S * np.linalg.norm(_spiral_d(_TH_S), axis=1), _TH_S)),
                      2 * math.pi * _PIPE_R * _PIPE_L + math.pi * _PIPE_R ** 2])
    share = areas / areas.sum()
    bpts = []
    have = 0
    while have < n_boundary:
        m = 2 * (n_boundary - have) + 256
        counts = rng.multinomial(m, share)
        parts = [(_sample_cyl_surface(counts[0], rng), 0),
                 (_sample_tube_surface(counts[1], rng), 1),
                 (_sample_pipe_surface(counts[2], rng), 2)]
        for P, pid in parts:
            keep = np.ones(P.shape[0], dtype=bool)
            if pid != 0:
                keep &= ~_in_cyl(P)
            if pid != 1:
                keep &= ~_in_tube(P)
            if pid != 2:
                keep &= ~_in_pipe(P)
            bpts.append(P[keep])
            have += int(keep.sum())
    B = np.concatenate(bpts)
    B = B[rng.permutation(B.shape[0])[:n_boundary]]
    lo = B.min(axis=0)
    hi = B.max(axis=0)
    ipts = []
    have = 0
    while have < n_interior:
        P = rng.uniform(lo, hi, size=(max(4 * (n_interior - have), 1024), 3))
        P = P[_in_pump(P)]
        ipts.append(P)
        have += P.shape[0]
    I = np.concatenate(ipts)[:n_interior]
    return NodeSet(np.ascontiguousarray(np.concatenate([I, B])), n_interior, "pump",
                   f"pump{n_boundary + n_interior}")


def inside(domain: str, P: np.ndarray) -> np.ndarray:
    if domain == "cube":
        return np.all((P > 0.0) & (P < 1.0), axis=1)
    if domain == "sphere":
        return np.sum(P * P, axis=1) < 1.0
    if domain == "pump":
        return _in_pump(P)
    raise ValueError(domain)


def test_points(nodes: NodeSet, m: int = 2000, seed: int | None = None) -> np.ndarray:
    """m seeded points uniform in the open domain (evaluation points for u)."""
    rng = _rng(BASE_SEED + 1000 if seed is None else seed)
    if nodes.domain == "cube":
        return uniform_cube(m, rng)
    if nodes.domain == "sphere":
        return uniform_ball(m, rng)
    lo, hi = nodes.X.min(axis=0), nodes.X.max(axis=0)
    out, have = [], 0
    while have < m:
        P = rng.uniform(lo, hi, size=(4 * (m - have) + 256, 3))
        P = P[inside(nodes.domain, P)]
        out.append(P)
        have += P.shape[0]
    return np.concatenate(out)[:m]


def batch_instances(count: int = 96, n_lo: int = 2000, n_hi: int = 16000,
                    seed0: int = BASE_SEED + 400):
    """Uneven batch: per instance (NodeSet, c, k, d).

    geometry ~ Bernoulli(1/2) cube/sphere; N ~ U{n_lo..n_hi}; c log-uniform in
    [0.05, 1]; k ~ U[1, 20]; plane-wave direction d uniform on S^2.
    Cube boundary: face grid (30% share); sphere boundary: Fibonacci (20%).
    """
    out = []
    for b in range(count):
        rng = _rng(seed0 + b)
        is_cube = rng.uniform() < 0.5
        n = int(rng.integers(n_lo, n_hi + 1))
        c = float(math.exp(rng.uniform(math.log(0.05), math.log(1.0))))
        k = float(rng.uniform(1.0, 20.0))
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if is_cube:
            ns = cube_faces_random(n, 0.30, rng)
        else:
            nb = int(round(0.20 * n))
            I = uniform_ball(n - nb, rng)
            ns = NodeSet(np.ascontiguousarray(np.concatenate([I, fibonacci_sphere(nb)])),
                         n - nb, "sphere", f"sphere{n}")
        ns.params = dict(c=c, k=k, d=d, seed=seed0 + b)
        out.append(ns)
    return out


_PUMP_POOL = None


def _pump_pool():
    """One large casing-like sample (16 000 boundary, 64 000 interior nodes),
    drawn once per process; pump_subsample takes instances from it."""
    global _PUMP_POOL
    if _PUMP_POOL is None:
        ns = pump_like(16000, 64000, seed=BASE_SEED + 650)
        _PUMP_POOL = (ns.X[ns.n_interior:].copy(), ns.X[:ns.n_interior].copy())
    return _PUMP_POOL


def pump_subsample(n: int, boundary_share: float, rng: np.random.Generator) -> NodeSet:
    """Casing-like node set of n nodes: a uniform subsample (without
    replacement) of the pool's boundary and interior nodes, which is again a
    uniform sample of the surface and of the volume (pump_like itself takes
    seconds per call at these sizes)."""
    B, I = _pump_pool()
    nb = int(round(boundary_share * n))
    ni = n - nb
    if nb > B.shape[0] or ni > I.shape[0]:
        raise ValueError(f"pump_subsample: n = {n} exceeds the pool")
    bsel = np.sort(rng.choice(B.shape[0], nb, replace=False))
    isel = np.sort(rng.choice(I.shape[0], ni, replace=False))
    return NodeSet(np.ascontiguousarray(np.concatenate([I[isel], B[bsel]])), ni, "pump", f"pump{n}")


def stop_instances(count: int, n_lo: int, n_hi: int, seed0: int = BASE_SEED + 600,
                   gauss_share: float = 0.5, pump_share: float = 0.0):
    """Training / evaluation runs for the learned stopping index.

    Node sets and (c, k) are drawn like the batched sweep (cube or sphere,
    N ~ U{n_lo..n_hi}, c log-uniform in [0.05, 1], k ~ U[1, 20]); with
    probability pump_share the node set is casing-like instead (pump_subsample,
    boundary share 0.2).  The exact solution is a plane wave sin(k d.X) with d
    uniform on S^2, or, with probability gauss_share, the Gaussian
    exp(-|X - X0|^2 / sigma) of the paper's examples with sigma log-uniform in
    [0.05, 10] (the casing example uses sigma = 10) and X0 uniform in the
    middle half of the domain (a random interior node for the casing).
    params: c, k, seed, rhs ('plane' | 'gauss'), d or (sigma, center).
    With pump_share = 0 the draws are those of the cube/sphere-only sampler.
    """
    out = []
    for b in range(count):
        rng = _rng(seed0 + b)
        u = rng.uniform()
        is_pump = u < pump_share
        is_cube = (not is_pump) and (u - pump_share) / (1.0 - pump_share) < 0.5
        n = int(rng.integers(n_lo, n_hi + 1))
        c = float(math.exp(rng.uniform(math.log(0.05), math.log(1.0))))
        k = float(rng.uniform(1.0, 20.0))
        if is_pump:
            ns = pump_subsample(n, 0.20, rng)
            center = ns.X[int(rng.integers(ns.n_interior))].copy()
        elif is_cube:
            ns = cube_faces_random(n, 0.30, rng)
            center = rng.uniform(0.25, 0.75, 3)
        else:
            nb = int(round(0.20 * n))
            I = uniform_ball(n - nb, rng)
            ns = NodeSet(np.ascontiguousarray(np.concatenate([I, fibonacci_sphere(nb)])),
                         n - nb, "sphere", f"sphere{n}")
            center = uniform_ball(1, rng, 0.5)[0]
        if rng.uniform() < gauss_share:
            sigma = float(math.exp(rng.uniform(math.log(0.05), math.log(10.0))))
            ns.params = dict(c=c, k=k, seed=seed0 + b, rhs="gauss", sigma=sigma, center=center)
        else:
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            ns.params = dict(c=c, k=k, seed=seed0 + b, rhs="plane", d=d)
        out.append(ns)
    return out


def _lattice_boundary_share(n: int) -> float:
    """Boundary share of an m^3 lattice with m^3 close to n: 1 - ((m-2)/m)^3."""
    m = max(3, int(round(n ** (1.0 / 3.0))))
    return 1.0 - ((m - 2) / m) ** 3


def _cube_faces_points(nb: int, pts2d: np.ndarray) -> np.ndarray:
    """nb points on the 6 faces of [0,1]^3 from 2D points in [0,1)^2, dealt to
    the faces in turn (face f: coordinate f//2 fixed at f%2)."""
    out = np.empty((nb, 3))
    for i in range(nb):
        f = i % 6
        u, v = pts2d[i]
        ax = f // 2
        rest = [a for a in range(3) if a != ax]
        out[i, ax] = float(f % 2)
        out[i, rest[0]] = u
        out[i, rest[1]] = v
    return out


def paper_nodes(domain: str, dist: str, n: int, seed: int) -> NodeSet:
    """Node sets shaped like the cube and sphere examples (Sec. 5, Examples 1
    and 2), whose Gmsh meshes are not available: 'random' (i.i.d. uniform),
    'uniform' (a cubic lattice, clipped to the ball for the sphere, of about
    n points) and 'halton' (scrambled Halton), with the boundary share of an
    m^3 lattice (cube: nodes on the faces; sphere: a Fibonacci lattice on the
    unit sphere).  Interior nodes first."""
    rng = _rng(seed)
    share = _lattice_boundary_share(n)
    if domain == "cube":
        if dist == "uniform":
            m = max(3, int(round(n ** (1.0 / 3.0))))
            g = np.linspace(0.0, 1.0, m)
            P = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
            on_b = np.any((P == 0.0) | (P == 1.0), axis=1)
            return NodeSet(np.ascontiguousarray(np.concatenate([P[~on_b], P[on_b]])), int((~on_b).sum()),
                           "cube", f"cube_uniform{P.shape[0]}")
        nb = int(round(share * n))
        ni = n - nb
        if dist == "random":
            I = uniform_cube(ni, rng)
            B = _cube_faces_points(nb, rng.uniform(0.0, 1.0, size=(nb, 2)))
        elif dist == "halton":
            I = scrambled_halton(ni, rng)
            B = _cube_faces_points(nb, scrambled_halton(nb, rng, bases=(2, 3)))
            I[(I == 0.0)] = 0.5
        else:
            raise ValueError(dist)
        return NodeSet(np.ascontiguousarray(np.concatenate([I, B])), ni, "cube", f"cube_{dist}{n}")
    if domain == "sphere":
        nb = int(round(share * n))
        ni = n - nb
        if dist == "uniform":
            h = (4.0 / 3.0 * math.pi / ni) ** (1.0 / 3.0)
            for _ in range(8):  # lattice spacing giving about ni points inside r < 1 - h/2
                g = np.arange(-1.0 + h / 2, 1.0, h)
                P = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
                I = P[np.sum(P * P, axis=1) < (1.0 - 0.5 * h) ** 2]
                h *= (I.shape[0] / ni) ** (1.0 / 3.0)
        elif dist == "random":
            I = uniform_ball(ni, rng)
        elif dist == "halton":
            out, have, skip = [], 0, 1
            while have < ni:
                H = 2.0 * scrambled_halton(2 * ni, _rng(seed + 1), skip=skip) - 1.0
                skip += 2 * ni
                H = H[np.sum(H * H, axis=1) < 1.0]
                out.append(H)
                have += H.shape[0]
            I = np.concatenate(out)[:ni]
        else:
            raise ValueError(dist)
        B = fibonacci_sphere(nb)
        return NodeSet(np.ascontiguousarray(np.concatenate([I, B])), I.shape[0], "sphere",
                       f"sphere_{dist}{I.shape[0] + nb}")
    raise ValueError(domain)


# ----------------------------------------------------------------------------
# named workload presets
# ----------------------------------------------------------------------------

def _preset_cube1000():
    ns = cube_grid(10)
    ns.params = dict(c=0.3, k=2.0, steps=40)
    return ns


def _preset_cube8000():
    ns = cube_faces_halton(8000, 21)
    ns.params = dict(c=0.2, k=5.0, steps=100, c_values=(0.1, 0.2, 0.5), k_values=(2.0, 5.0))
    return ns


def _preset_sphere20000():
    ns = sphere_fibonacci_ball(4000, 16000)
    ns.params = dict(c=0.15, k=10.0, steps=150)
    return ns


def _preset_pump40000():
    ns = pump_like(8000, 32000)
    ns.params = dict(c=0.1, k=8.0, steps=150)
    return ns


PRESETS = {
    "cube1000": _preset_cube1000,
    "cube8000": _preset_cube8000,
    "sphere20000": _preset_sphere20000,
    "pump40000": _preset_pump40000,
}


def preset(name: str) -> NodeSet:
    return PRESETS[name]()
