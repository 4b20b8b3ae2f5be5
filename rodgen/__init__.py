"""Seeded synthetic rod workloads.

This module only builds inputs: rod counts and lengths, materials, loads, and an initial
state (straight rods, orthonormal director frames, optional random rigid motion).  It
holds none of the time-stepping method's arithmetic; both the CPU oracle tests and the
CUDA path consume what it produces.

Workloads (sizes as in the paper's case studies, synthetic stand-ins for their data):
  * ``cantilever``     -- one clamped rod with a transverse tip force and linear damping;
  * ``cilia_carpet``   -- a square carpet of clamped upright rods driven by a sinusoidal
                          base couple with seeded phases and Stokes drag (the magnetic
                          cilia carpets of the results section are the model for it);
  * ``random_packing`` -- free rods with seeded lengths, positions and orientations in a
                          box, with gravity and rod-rod contact (the fibrous packings of
                          the results section are the model for it);
  * ``adjoint_batch``  -- clamped rods with seeded rest curvatures, element couples and
                          tip targets (parameters of the gradient workload).
State layout: component-major arrays, x/v of shape (3, nodes), Q of shape (9, elements)
with Q[3a+b, i] the b-th lab component of director a+1, w of shape (3, elements).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "RodProblem",
    "cantilever",
    "cilia_carpet",
    "random_packing",
    "adjoint_batch",
    "perturbed",
    "quat_to_matrix",
]


@dataclass
class RodProblem:
    name: str
    n_elem: np.ndarray                 # (R,) int32
    rest_len: np.ndarray               # (E,)
    radius: np.ndarray                 # (R,)
    youngs: np.ndarray                 # (R,)
    shear_mod: np.ndarray              # (R,)
    density: np.ndarray                # (R,)
    x: np.ndarray                      # (3, N)
    v: np.ndarray                      # (3, N)
    Q: np.ndarray                      # (9, E)
    w: np.ndarray                      # (3, E)
    alpha_c: float = 4.0 / 3.0
    clamp_base: Optional[np.ndarray] = None   # (R,) int8
    rest_kappa: Optional[np.ndarray] = None   # (3, V)
    rest_sigma: Optional[np.ndarray] = None   # (3, E)
    gravity: np.ndarray = field(default_factory=lambda: np.zeros(3))
    nu_damp: float = 0.0
    stokes_gamma: float = 0.0
    tip_force: Optional[np.ndarray] = None    # (3, R)
    act_amp: Optional[np.ndarray] = None      # (R,)
    act_period: Optional[np.ndarray] = None   # (R,)
    act_phase: Optional[np.ndarray] = None    # (R,)
    elem_couple: Optional[np.ndarray] = None  # (3, E)
    contact: bool = False
    contact_k: float = 0.0
    contact_c: float = 0.0
    cell_size: float = 0.0
    contact_mu: float = 0.0                   # rod-rod friction coefficient
    contact_vslip: float = 0.0                # slip velocity of the regularised Coulomb law
    magnetization: Optional[np.ndarray] = None  # (3, E) per unit reference length, local frame
    field_b0: np.ndarray = field(default_factory=lambda: np.zeros(3))
    field_bc: np.ndarray = field(default_factory=lambda: np.zeros(3))
    field_bs: np.ndarray = field(default_factory=lambda: np.zeros(3))
    field_omega: float = 0.0
    muscle_amp: Optional[np.ndarray] = None        # (R,)
    muscle_period: Optional[np.ndarray] = None     # (R,)
    muscle_wavelength: Optional[np.ndarray] = None # (R,)
    muscle_phase: Optional[np.ndarray] = None      # (R,)
    wall_point: Optional[np.ndarray] = None        # (n_walls, 3)
    wall_normal: Optional[np.ndarray] = None       # (n_walls, 3), unit
    wall_velocity: Optional[np.ndarray] = None     # (n_walls, 3)
    wall_k: float = 0.0
    wall_c: float = 0.0
    wall_mu: float = 0.0
    wall_vslip: float = 0.0
    dt: float = 1e-5
    n_steps: int = 1
    t0: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def n_rods(self) -> int:
        return int(self.n_elem.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.n_elem.sum())

    @property
    def n_nodes(self) -> int:
        return self.n_elems + self.n_rods

    @property
    def n_voronoi(self) -> int:
        return self.n_elems - self.n_rods

    def node_offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.n_elem + 1)]).astype(np.int64)

    def elem_offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.n_elem)]).astype(np.int64)

    def state(self):
        return self.x.copy(), self.v.copy(), self.Q.copy(), self.w.copy()

    def replace(self, **kw) -> "RodProblem":
        return dataclasses.replace(self, **kw)

    def take_rods(self, r0: int, r1: int) -> "RodProblem":
        """The sub-ensemble of rods r0 .. r1 - 1 with their state, constants and loads (global
        settings unchanged)."""
        R = self.n_rods
        if not (0 <= r0 < r1 <= R):
            raise ValueError("need 0 <= r0 < r1 <= n_rods")
        eo, no = self.elem_offsets(), self.node_offsets()
        e0, e1, n0, n1 = int(eo[r0]), int(eo[r1]), int(no[r0]), int(no[r1])
        v0, v1 = e0 - r0, e1 - r1
        per_rod, per_elem, per_node, per_vor = {}, {}, {}, {}
        for f in dataclasses.fields(self):
            a = getattr(self, f.name)
            if not isinstance(a, np.ndarray) or f.name in ("gravity", "field_b0", "field_bc", "field_bs") \
                    or f.name.startswith("wall_"):
                continue
            last = a.shape[-1]
            if f.name == "n_elem" or (a.ndim == 1 and last == R and f.name != "rest_len"):
                per_rod[f.name] = a[r0:r1].copy()
            elif a.ndim == 2 and last == R and f.name in ("tip_force",):
                per_rod[f.name] = a[:, r0:r1].copy()
            elif f.name in ("x", "v"):
                per_node[f.name] = a[:, n0:n1].copy()
            elif f.name == "rest_kappa":
                per_vor[f.name] = a[:, v0:v1].copy()
            elif f.name == "rest_len":
                per_elem[f.name] = a[e0:e1].copy()
            elif a.shape[-1] == self.n_elems:
                per_elem[f.name] = a[..., e0:e1].copy()
        return dataclasses.replace(self, name=f"{self.name}_rods{r0}-{r1}", **per_rod, **per_elem, **per_node,
                                   **per_vor)


# ----------------------------------------------------------------------------- helpers

def quat_to_matrix(q: np.ndarray) -> np.ndarray:
    """Rotation matrices (..., 3, 3) from unit quaternions (..., 4) = (w, x, y, z)."""
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _frames(d3: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Director rows (d1, d2, d3) for unit tangents d3 (R, 3); d1 is ref projected off d3."""
    d1 = ref - (ref * d3).sum(-1, keepdims=True) * d3
    d1 /= np.linalg.norm(d1, axis=-1, keepdims=True)
    d2 = np.cross(d3, d1)
    return np.stack([d1, d2, d3], axis=1)  # (R, 3 rows, 3 comps)


def _straight_rods(n_elem, rest_len, base, d3, ref):
    """Nodes along straight lines from ``base`` in direction ``d3``; one frame per rod."""
    R = n_elem.shape[0]
    E = int(n_elem.sum())
    N = E + R
    x = np.empty((3, N))
    Q = np.empty((9, E))
    frames = _frames(d3, ref)
    node0 = 0
    elem0 = 0
    for r in range(R):
        n = int(n_elem[r])
        s = np.concatenate([[0.0], np.cumsum(rest_len[elem0:elem0 + n])])
        x[:, node0:node0 + n + 1] = base[r][:, None] + d3[r][:, None] * s[None, :]
        Q[:, elem0:elem0 + n] = frames[r].reshape(9)[:, None]
        node0 += n + 1
        elem0 += n
    return x, Q


def _uniform(R, val):
    return np.full(R, float(val))


# ----------------------------------------------------------------------------- workloads

def cantilever(n: int = 100, length: float = 1.0, radius: float = 0.01, youngs: float = 1e6,
               tip_force: float = 1e-2, nu: float = 0.1, dt: float = 1e-5, n_steps: int = 10_000,
               shear_ratio: float = 1.5, density: float = 1000.0) -> RodProblem:
    """One rod along lab z, clamped at node 0, tip force along lab y."""
    n_elem = np.array([n], dtype=np.int32)
    rest_len = np.full(n, length / n)
    d3 = np.array([[0.0, 0.0, 1.0]])
    x, Q = _straight_rods(n_elem, rest_len, np.zeros((1, 3)), d3, np.array([[1.0, 0.0, 0.0]]))
    E = n
    return RodProblem(
        name=f"cantilever_n{n}", n_elem=n_elem, rest_len=rest_len,
        radius=_uniform(1, radius), youngs=_uniform(1, youngs), shear_mod=_uniform(1, youngs / shear_ratio),
        density=_uniform(1, density), x=x, v=np.zeros_like(x), Q=Q, w=np.zeros((3, E)),
        clamp_base=np.ones(1, dtype=np.int8), nu_damp=nu,
        tip_force=np.array([[0.0], [tip_force], [0.0]]), dt=dt, n_steps=n_steps)


def cilia_carpet(side: int = 64, n: int = 50, spacing: float = 0.05, length: float = 0.2,
                 radius: float = 0.005, youngs: float = 1e6, density: float = 1000.0,
                 period: float = 1.0, amp_factor: float = 0.5, gamma: float = 1.0,
                 dt: float = 1e-5, n_steps: int = 10_000, seed: int = 1234,
                 amp_range=None, period_range=None, random_azimuth: bool = False) -> RodProblem:
    """side x side upright clamped rods on a square grid, sinusoidal base couple about d1.

    Amplitude A0 = amp_factor * E I / L, phases uniform in [0, 2 pi) from ``seed``; with
    ``amp_range`` / ``period_range`` every rod draws its own amp_factor / period uniformly.
    d1 is the lab x axis, or with ``random_azimuth`` a horizontal direction drawn per rod (so
    that each rod beats in a plane of its own)."""
    rng = np.random.default_rng(seed)
    R = side * side
    n_elem = np.full(R, n, dtype=np.int32)
    rest_len = np.full(R * n, length / n)
    gx, gy = np.meshgrid(np.arange(side) * spacing, np.arange(side) * spacing, indexing="ij")
    base = np.stack([gx.ravel(), gy.ravel(), np.zeros(R)], axis=1)
    d3 = np.tile([0.0, 0.0, 1.0], (R, 1))
    d1 = np.tile([1.0, 0.0, 0.0], (R, 1))
    if random_azimuth:
        psi = np.random.default_rng([seed, 7]).uniform(0.0, 2 * np.pi, R)
        d1 = np.stack([np.cos(psi), np.sin(psi), np.zeros(R)], axis=1)
    x, Q = _straight_rods(n_elem, rest_len, base, d3, d1)
    I = np.pi * radius ** 4 / 4
    phase = rng.uniform(0.0, 2 * np.pi, R)
    amp = _uniform(R, amp_factor * youngs * I / length)
    per = _uniform(R, period)
    if amp_range is not None:
        amp = rng.uniform(amp_range[0], amp_range[1], R) * youngs * I / length
    if period_range is not None:
        per = rng.uniform(period_range[0], period_range[1], R)
    return RodProblem(
        name=f"cilia_carpet_{side}x{side}_n{n}", n_elem=n_elem, rest_len=rest_len,
        radius=_uniform(R, radius), youngs=_uniform(R, youngs), shear_mod=_uniform(R, youngs / 1.5),
        density=_uniform(R, density), x=x, v=np.zeros_like(x), Q=Q, w=np.zeros((3, R * n)),
        clamp_base=np.ones(R, dtype=np.int8), stokes_gamma=gamma,
        act_amp=amp, act_period=per, act_phase=phase, dt=dt, n_steps=n_steps)


def random_packing(n_rods: int = 10_000, nmin: int = 16, nmax: int = 256, box: float = 1.0,
                   rest_len: float = 1e-3, radius: float = 0.005, youngs: float = 1e6,
                   density: float = 1000.0, speed: float = 0.25, spin: float = 0.0,
                   contact_k: float = 1e4, contact_c: float = 10.0, gravity: float = 9.81,
                   dt: float = 5e-6, n_steps: int = 5000, seed: int = 1234,
                   allow_overlap: bool = False, margin: float = 5e-4) -> RodProblem:
    """Free straight rods, lengths n ~ U{nmin..nmax} elements of ``rest_len``, centres uniform in
    the box, axes uniform on the sphere, a rigid velocity uniform in [-speed, speed]^3 per rod.

    Unless ``allow_overlap``, rods are placed one by one (longest first) and a candidate is
    redrawn while any of its sample points lies closer than 2 r + sample spacing + margin to
    a sample point of an already placed rod, so the initial packing has no overlap."""
    rng = np.random.default_rng(seed)
    n_elem = rng.integers(nmin, nmax + 1, n_rods).astype(np.int32)
    lengths = n_elem * rest_len
    centers = np.empty((n_rods, 3))
    axes = np.empty((n_rods, 3))

    def draw_axis():
        a = rng.normal(size=3)
        return a / np.linalg.norm(a)

    if allow_overlap:
        for r in range(n_rods):
            centers[r] = rng.uniform(0.0, box, 3)
            axes[r] = draw_axis()
    else:
        _place_without_overlap(rng, lengths, box, radius, margin, centers, axes)
    base = centers - 0.5 * lengths[:, None] * axes
    # reference direction for d1: a seeded random vector, re-drawn when nearly parallel
    ref = rng.normal(size=(n_rods, 3))
    par = np.abs((ref / np.linalg.norm(ref, axis=1, keepdims=True) * axes).sum(1)) > 0.99
    ref[par] = np.cross(axes[par], [1.0, 0.0, 0.0]) + np.cross(axes[par], [0.0, 1.0, 0.0])
    rl = np.full(int(n_elem.sum()), rest_len)
    x, Q = _straight_rods(n_elem, rl, base, axes, ref)
    vel = rng.uniform(-speed, speed, (n_rods, 3))
    node_counts = n_elem + 1
    v = np.repeat(vel, node_counts, axis=0).T.copy()
    w = np.zeros((3, int(n_elem.sum())))
    if spin > 0:
        w[:] = np.repeat(rng.uniform(-spin, spin, (n_rods, 3)), n_elem, axis=0).T
    R = n_rods
    return RodProblem(
        name=f"random_packing_{n_rods}", n_elem=n_elem, rest_len=rl,
        radius=_uniform(R, radius), youngs=_uniform(R, youngs), shear_mod=_uniform(R, youngs / 1.5),
        density=_uniform(R, density), x=x, v=np.ascontiguousarray(v), Q=Q, w=w,
        gravity=np.array([0.0, 0.0, -gravity]), contact=True, contact_k=contact_k,
        contact_c=contact_c, cell_size=2 * radius, dt=dt, n_steps=n_steps)


def random_packing_cached(seed: int = 1234, cache_dir: Optional[str] = None) -> RodProblem:
    """The default 10^4-rod packing of ``random_packing(seed=seed)``, kept as an .npz file in
    ``cache_dir`` (default: the system's temporary directory) because the placement without
    overlap takes tens of seconds; a missing or unreadable file is regenerated."""
    import hashlib
    import os
    import tempfile
    cache_dir = cache_dir or os.path.join(tempfile.gettempdir(), "rodbench_cache")
    os.makedirs(cache_dir, exist_ok=True)
    key = hashlib.sha1(f"random_packing-default-{seed}-v3".encode()).hexdigest()[:12]
    path = os.path.join(cache_dir, f"packing_{key}.npz")
    if os.path.exists(path):
        try:
            z = np.load(path)
            base = random_packing(n_rods=10, seed=seed)  # cheap template for the other fields
            return base.replace(n_elem=z["n_elem"], rest_len=z["rest_len"], radius=z["radius"], youngs=z["youngs"],
                                shear_mod=z["shear_mod"], density=z["density"], x=z["x"], v=z["v"], Q=z["Q"],
                                w=z["w"], name=f"random_packing_{int(z['n_elem'].size)}")
        except Exception:
            pass
    p = random_packing(seed=seed)
    tmp = path + f".{os.getpid()}.npz"
    np.savez(tmp, n_elem=p.n_elem, rest_len=p.rest_len, radius=p.radius, youngs=p.youngs,
             shear_mod=p.shear_mod, density=p.density, x=p.x, v=p.v, Q=p.Q, w=p.w)
    os.replace(tmp, path)
    return p


def _axis_distance(c1, a1, h1, c2, a2, h2):
    """Exact distance between the axis segments c + t a, |t| <= h (vectorised over pairs): the
    minimum of the convex quadratic over the rectangle is either its free stationary point (if
    inside) or the minimum over one of the four edges, so all five candidates are evaluated."""
    r = c1 - c2
    b = (a1 * a2).sum(1)
    d = (a1 * r).sum(1)
    e = (a2 * r).sum(1)

    def dist(t, u):
        return np.linalg.norm(r + t[:, None] * a1 - u[:, None] * a2, axis=1)

    best = np.full(len(r), np.inf)
    den = 1.0 - b * b
    ok = den > 1e-12
    t0 = np.where(ok, (b * e - d) / np.where(ok, den, 1.0), 0.0)
    u0 = np.where(ok, (e - b * d) / np.where(ok, den, 1.0), 0.0)
    inside = ok & (np.abs(t0) <= h1) & (np.abs(u0) <= h2)
    best = np.where(inside, dist(t0, u0), best)
    for side in (-1.0, 1.0):
        t = side * h1                                    # edge t = +-h1: best u
        u = np.clip(b * t + e, -h2, h2)
        best = np.minimum(best, dist(t, u))
        u = side * h2                                    # edge u = +-h2: best t
        t = np.clip(b * u - d, -h1, h1)
        best = np.minimum(best, dist(t, u))
    return best


def _neighbour_pairs(cq, cp, cell):
    """Index pairs (i in cq, j in cp) whose points share or neighbour a cubic cell of edge ``cell``."""
    lo = np.minimum(cq.min(0), cp.min(0)) - cell
    kq = np.floor((cq - lo) / cell).astype(np.int64)
    kp = np.floor((cp - lo) / cell).astype(np.int64)
    dim = np.maximum(kq.max(0), kp.max(0)) + 3
    key = (kp[:, 2] * dim[1] + kp[:, 1]) * dim[0] + kp[:, 0]
    order = np.argsort(key, kind="stable")
    sk = key[order]
    ii, jj = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                kk = ((kq[:, 2] + dz) * dim[1] + (kq[:, 1] + dy)) * dim[0] + (kq[:, 0] + dx)
                s = np.searchsorted(sk, kk, side="left")
                e = np.searchsorted(sk, kk, side="right")
                cnt = e - s
                tot = int(cnt.sum())
                if tot == 0:
                    continue
                qi = np.repeat(np.arange(len(cq)), cnt)
                off = np.arange(tot) - np.repeat(np.cumsum(cnt) - cnt, cnt)
                ii.append(qi)
                jj.append(order[np.repeat(s, cnt) + off])
    if not ii:
        return np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64)
    return np.concatenate(ii), np.concatenate(jj)


def _conflicts(cq, aq, hq, cp, ap, hp, gap):
    """Pairs (i, j) of capsules (axis segments + radius gap/2 each) closer than ``gap``."""
    if len(cq) == 0 or len(cp) == 0:
        return np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64)
    cell = 2.0 * max(hq.max(), hp.max()) + gap
    i, j = _neighbour_pairs(cq, cp, cell)
    near = np.linalg.norm(cq[i] - cp[j], axis=1) < hq[i] + hp[j] + gap
    i, j = i[near], j[near]
    d = _axis_distance(cq[i], aq[i], hq[i], cp[j], ap[j], hp[j])
    hit = d < gap
    return i[hit], j[hit]


def _place_without_overlap(rng, lengths, box, radius, margin, centers, axes):
    """Random sequential addition, longest rods first, in batches: a candidate (centre, axis) is
    drawn for each of the next ``window`` unplaced rods, candidates closer than 2 r + margin to a
    placed rod are rejected, the rest are accepted greedily in length order unless they conflict
    with an earlier accepted candidate of the same batch; rejected rods are redrawn."""
    gap = 2.0 * radius + margin
    half = 0.5 * lengths
    queue = np.argsort(-lengths, kind="stable")
    placed = np.zeros(0, dtype=np.int64)
    window = 512
    for _ in range(20000):
        if len(queue) == 0:
            return
        todo = queue[:window]
        m = len(todo)
        c = rng.uniform(0.0, box, (m, 3))
        a = rng.normal(size=(m, 3))
        a /= np.linalg.norm(a, axis=1, keepdims=True)
        h = half[todo]
        bad = np.zeros(m, dtype=bool)
        if len(placed):
            i, _ = _conflicts(c, a, h, centers[placed], axes[placed], half[placed], gap)
            bad[i] = True
        i, j = _conflicts(c, a, h, c, a, h, gap)
        keep = i > j
        i, j = i[keep], j[keep]
        order = np.argsort(i, kind="stable")
        i, j = i[order], j[order]
        starts = np.searchsorted(i, np.arange(m), side="left")
        ends = np.searchsorted(i, np.arange(m), side="right")
        take = np.zeros(m, dtype=bool)
        for q in range(m):
            if bad[q]:
                continue
            if ends[q] > starts[q] and take[j[starts[q]:ends[q]]].any():
                continue
            take[q] = True
        rods = todo[take]
        centers[rods] = c[take]
        axes[rods] = a[take]
        placed = np.concatenate([placed, rods])
        queue = np.concatenate([todo[~take], queue[window:]])
    raise RuntimeError("random_packing: could not place every rod; lower the density")


def adjoint_batch(n_rods: int = 1024, n: int = 64, length: float = 0.2, radius: float = 0.005,
                  youngs: float = 1e6, density: float = 1000.0, kappa_scale: float = 0.5,
                  couple_scale: float = 1e-6, target_scale: float = 0.01, spacing: float = 0.05,
                  dt: float = 1e-5, n_steps: int = 2000, seed: int = 1234) -> RodProblem:
    """Clamped upright rods with seeded rest curvature (N(0, kappa_scale) 1/m), constant element
    couples (N(0, couple_scale) N m) and tip targets (undeformed tip + N(0, target_scale) m)."""
    rng = np.random.default_rng(seed)
    side = int(np.ceil(np.sqrt(n_rods)))
    n_elem = np.full(n_rods, n, dtype=np.int32)
    rest_len = np.full(n_rods * n, length / n)
    gx, gy = np.meshgrid(np.arange(side) * spacing, np.arange(side) * spacing, indexing="ij")
    base = np.stack([gx.ravel(), gy.ravel(), np.zeros(side * side)], axis=1)[:n_rods]
    d3 = np.tile([0.0, 0.0, 1.0], (n_rods, 1))
    x, Q = _straight_rods(n_elem, rest_len, base, d3, np.tile([1.0, 0.0, 0.0], (n_rods, 1)))
    E = n_rods * n
    V = E - n_rods
    R = n_rods
    kappa0 = rng.normal(0.0, kappa_scale, (3, V))
    couples = rng.normal(0.0, couple_scale, (3, E))
    tips = x[:, np.cumsum(n_elem + 1) - 1]
    targets = tips + rng.normal(0.0, target_scale, (3, R))
    return RodProblem(
        name=f"adjoint_{n_rods}x{n}", n_elem=n_elem, rest_len=rest_len,
        radius=_uniform(R, radius), youngs=_uniform(R, youngs), shear_mod=_uniform(R, youngs / 1.5),
        density=_uniform(R, density), x=x, v=np.zeros_like(x), Q=Q, w=np.zeros((3, E)),
        clamp_base=np.ones(R, dtype=np.int8), rest_kappa=kappa0, elem_couple=couples,
        dt=dt, n_steps=n_steps, extra={"targets": targets})


def perturbed(p: RodProblem, seed: int = 7, pos: float = 1e-3, vel: float = 0.1, rot: float = 0.05,
              omega: float = 5.0) -> RodProblem:
    """Copy of ``p`` with seeded random perturbations of every state array (positions by
    ``pos`` times the element rest length, velocities, director rotations by angles of about
    ``rot`` rad built from random unit quaternions, angular velocities)."""
    rng = np.random.default_rng(seed)
    x, v, Q, w = p.state()
    N, E = x.shape[1], Q.shape[1]
    scale = np.median(p.rest_len)
    x = x + rng.normal(0.0, pos * scale, x.shape)
    v = v + rng.normal(0.0, vel, v.shape)
    q = np.concatenate([np.ones((E, 1)), rng.normal(0.0, 0.5 * rot, (E, 3))], axis=1)
    Rm = quat_to_matrix(q)                                    # (E, 3, 3)
    Qm = Q.T.reshape(E, 3, 3)
    Qn = np.einsum("eab,ebc->eac", Qm, Rm.transpose(0, 2, 1))  # rows rotated: d_a <- R d_a
    Q = Qn.reshape(E, 9).T.copy()
    w = w + rng.normal(0.0, omega, w.shape)
    return p.replace(x=x, v=v, Q=Q, w=w)
