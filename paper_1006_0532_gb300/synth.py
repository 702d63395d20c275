"""Seeded synthetic inputs: unstructured triangle grids and prescribed nodal fields.

This module produces *input data only* (node coordinates, triangles, edge tags,
nodal Eulerian fields, model parameters).  It contains none of the particle
method's arithmetic: no shapefunctions, no stochastic updates, no tracking, no
statistics.  Both the CUDA library and the CPU oracle consume what it returns.

Workloads (the paper's test cases, Sect. 4.1 and 4.2, rebuilt synthetically
because its DNS and wind-tunnel data are not part of the method):

* ``channel_grid`` -- the 2-D channel cross-section [0, Lx] x [0, 1], walls at
  y = 0 and y = 1 (no-slip), periodic in x.  A jittered lattice whose quads are
  split along the diagonal that passes the local empty-circumcircle test, so the
  node valence varies like an unstructured Delaunay mesh.  Rows are uniform or
  geometrically graded toward both walls (first cell at y+ ~ 1).
* ``channel_fields`` -- prescribed nodal fields for fully developed channel flow
  at friction Reynolds number Re_tau: Reichardt mean velocity, a smooth
  turbulent kinetic energy and frequency profile, a realisable Reynolds stress,
  the mean-pressure gradient of Eq. 63, a local algebraic form for the
  elliptic-relaxation tensor and the Eq. 58 wall frequency.

Nodal field layout (32 doubles per node):
  0-2   <U_i>                      3-4   d<P>/dx_j (rho = 1)
  5-10  d<U_i>/dx_j (i-major, j = x, y)
  11-13 laplacian <U_i>            14-22 wp_ij (3 x 3 row-major)
  23-28 <u_i u_j> (xx, yy, zz, xy, xz, yz)
  29    <omega>                    30    omega_w (Eq. 58 mean at walls)
  31    reserved (0)
Edge tags (int8 per element edge k, the edge opposite local vertex k):
  0 interior, 1 no-slip wall, 2 free-slip boundary.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

NF = 32           # nodal field slots
NSTAT = 13        # statistics per element / node

# Table 4 of the paper (model constants for velocity and frequency).
TABLE4 = dict(C1=1.85, C2=0.63, C3=5.0, C4=0.25, CT=6.0, CL=0.134, Ceta=72.0,
              Cv=1.4, gamma5=0.1, Cw1=0.5, Cw2=0.73)


@dataclass
class Grid:
    node_xy: np.ndarray      # float64 [nn, 2]
    tri: np.ndarray          # int32 [ne, 3], counter-clockwise (minimum image in x)
    edge_tag: np.ndarray     # int8 [ne, 3]
    period_x: float          # 0.0 = not periodic

    @property
    def nn(self) -> int:
        return int(self.node_xy.shape[0])

    @property
    def ne(self) -> int:
        return int(self.tri.shape[0])


def _geometric_rows(ny: int, y1: float) -> np.ndarray:
    """Node rows on [0, 1] with cell widths y1 * r**min(k, ncell-1-k), symmetric about 0.5."""
    ncell = ny - 1
    k = np.arange(ncell)
    m = np.minimum(k, ncell - 1 - k)

    def total(r: float) -> float:
        return float(np.sum(y1 * r ** m))

    lo, hi = 1.0, 2.0
    while total(hi) < 1.0:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < 1.0:
            lo = mid
        else:
            hi = mid
    h = y1 * (0.5 * (lo + hi)) ** m
    y = np.concatenate([[0.0], np.cumsum(h)])
    y[-1] = 1.0
    return y


def _incircle(ax, ay, bx, by, cx, cy, dx, dy) -> np.ndarray:
    """> 0 where d lies inside the circumcircle of the counter-clockwise triangle abc."""
    adx, ady = ax - dx, ay - dy
    bdx, bdy = bx - dx, by - dy
    cdx, cdy = cx - dx, cy - dy
    ad = adx * adx + ady * ady
    bd = bdx * bdx + bdy * bdy
    cd = cdx * cdx + cdy * cdy
    return (adx * (bdy * cd - bd * cdy) - ady * (bdx * cd - bd * cdx)
            + ad * (bdx * cdy - bdy * cdx))


def channel_grid(nx: int, ny: int, lx: float = 2.0, graded_y1: float | None = None,
                 jitter_x: float = 0.2, jitter_y: float = 0.1, seed: int = 1) -> Grid:
    """Periodic-in-x channel grid with nx columns and ny node rows (2 nx (ny-1) triangles).

    Wall rows (y = 0, 1) are jittered in x only, so wall edges lie exactly on the walls.
    Interior nodes move by up to +-jitter_x * dx in x and +-jitter_y * (smaller adjacent
    row spacing) in y.  Each quad takes the diagonal that satisfies the empty-circle test.
    """
    rng = np.random.default_rng(seed)
    dx = lx / nx
    if graded_y1 is None:
        ys = np.linspace(0.0, 1.0, ny)
    else:
        ys = _geometric_rows(ny, graded_y1)
    xs = np.arange(nx) * dx
    X = np.repeat(xs[None, :], ny, axis=0).copy()
    Y = np.repeat(ys[:, None], nx, axis=1).copy()
    X += rng.uniform(-jitter_x, jitter_x, size=X.shape) * dx
    dy_loc = np.empty(ny)
    dy_loc[0] = ys[1] - ys[0]
    dy_loc[-1] = ys[-1] - ys[-2]
    dy_loc[1:-1] = np.minimum(ys[1:-1] - ys[:-2], ys[2:] - ys[1:-1])
    jy = rng.uniform(-jitter_y, jitter_y, size=Y.shape) * dy_loc[:, None]
    jy[0, :] = 0.0
    jy[-1, :] = 0.0
    Y += jy
    X = np.mod(X, lx)
    node_xy = np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64)

    def nid(j, i):
        return j * nx + (i % nx)

    # quad (i, j): corners p00=(i,j), p10=(i+1,j), p11=(i+1,j+1), p01=(i,j+1)
    J, I = np.meshgrid(np.arange(ny - 1), np.arange(nx), indexing="ij")
    J = J.ravel()
    I = I.ravel()
    n00, n10, n11, n01 = nid(J, I), nid(J, I + 1), nid(J + 1, I + 1), nid(J + 1, I)

    def unwrapped(n, ref):
        x = node_xy[n, 0].copy()
        d = x - node_xy[ref, 0]
        x = np.where(d > 0.5 * lx, x - lx, np.where(d < -0.5 * lx, x + lx, x))
        return x, node_xy[n, 1]

    x00, y00 = unwrapped(n00, n00)
    x10, y10 = unwrapped(n10, n00)
    x11, y11 = unwrapped(n11, n00)
    x01, y01 = unwrapped(n01, n00)
    # Diagonal p00-p11 gives (p00,p10,p11),(p00,p11,p01); it is Delaunay in the quad iff
    # p01 is not inside the circumcircle of (p00,p10,p11).
    use_a = _incircle(x00, y00, x10, y10, x11, y11, x01, y01) <= 0.0

    def area2(ax, ay, bx, by, cx, cy):
        return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)

    a_ok = (area2(x00, y00, x10, y10, x11, y11) > 0) & (area2(x00, y00, x11, y11, x01, y01) > 0)
    b_ok = (area2(x00, y00, x10, y10, x01, y01) > 0) & (area2(x10, y10, x11, y11, x01, y01) > 0)
    use_a = np.where(a_ok & b_ok, use_a, a_ok)
    if not np.all(np.where(use_a, a_ok, b_ok)):
        raise ValueError("jitter too large: a quad admits no valid split")

    t1 = np.where(use_a[:, None], np.stack([n00, n10, n11], 1), np.stack([n00, n10, n01], 1))
    t2 = np.where(use_a[:, None], np.stack([n00, n11, n01], 1), np.stack([n10, n11, n01], 1))
    tri = np.empty((2 * t1.shape[0], 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2

    # Edge tags: an edge with both ends on the same wall row is a no-slip wall edge.
    on_bottom = np.zeros(node_xy.shape[0], bool)
    on_top = np.zeros(node_xy.shape[0], bool)
    on_bottom[:nx] = True
    on_top[(ny - 1) * nx:] = True
    edge_tag = np.zeros(tri.shape, dtype=np.int8)
    for k in range(3):
        a = tri[:, (k + 1) % 3]
        b = tri[:, (k + 2) % 3]
        wall = (on_bottom[a] & on_bottom[b]) | (on_top[a] & on_top[b])
        edge_tag[:, k] = np.where(wall, 1, 0)
    return Grid(node_xy=node_xy, tri=tri, edge_tag=edge_tag, period_x=float(lx))


# ----------------------------------------------------------------------------------------
# Prescribed channel fields.
# ----------------------------------------------------------------------------------------

def _reichardt(yp):
    """Reichardt's mean-velocity profile U+(y+) and its first two y+-derivatives."""
    kap = 0.41
    a = np.log1p(kap * yp) / kap
    da = 1.0 / (1.0 + kap * yp)
    dda = -kap / (1.0 + kap * yp) ** 2
    e1 = np.exp(-yp / 11.0)
    e3 = np.exp(-yp / 3.0)
    b = 7.8 * (1.0 - e1 - (yp / 11.0) * e3)
    db = 7.8 * (e1 / 11.0 - e3 / 11.0 + (yp / 33.0) * e3)
    ddb = 7.8 * (-e1 / 121.0 + e3 / 33.0 + e3 / 33.0 - (yp / 99.0) * e3)
    return a + b, da + db, dda + ddb


def channel_fields(grid: Grid, re_tau: float, u_tau: float = 0.05, h: float = 0.5,
                   params: dict | None = None) -> np.ndarray:
    """Nodal fields [nn, 32] for statistically stationary channel flow at Re_tau."""
    c = dict(TABLE4)
    if params:
        c.update({k: v for k, v in params.items() if k in c})
    nu = u_tau * h / re_tau
    y = grid.node_xy[:, 1]
    yw = np.minimum(y, 1.0 - y)
    s = np.where(y < 0.5, 1.0, -1.0)               # d(yw)/dy
    yp = u_tau * yw / nu
    iscale = u_tau / nu                            # d(y+)/d(yw)

    up, dup, ddup = _reichardt(yp)
    U = u_tau * up
    dUdy = s * u_tau * iscale * dup
    d2Udy2 = u_tau * iscale ** 2 * ddup

    ek = np.exp(-yp / 10.0)
    kp = 3.33 * (1.0 - ek) ** 2
    dkp = 3.33 * 2.0 * (1.0 - ek) * ek / 10.0
    k = u_tau ** 2 * kp
    dkdy = s * u_tau ** 2 * iscale * dkp
    fv = (1.0 - np.exp(-yp / 26.0)) ** 2
    uv = -s * u_tau ** 2 * (1.0 - yw / h) * fv
    wp = 0.73 / (yp + 8.1)
    om = (u_tau ** 2 / nu) * wp

    F = np.zeros((grid.nn, NF), dtype=np.float64)
    F[:, 0] = U
    F[:, 3] = -u_tau ** 2 / h                      # driving streamwise pressure gradient
    F[:, 4] = -(2.0 / 3.0) * dkdy                  # Eq. 63 with <v^2> = 2k/3
    F[:, 6] = dUdy                                 # dU/dy
    F[:, 11] = d2Udy2
    # Elliptic-relaxation tensor: local algebraic (L -> 0) form, isotropic part plus a
    # production-like part proportional to the mean velocity gradient.
    grad = np.zeros((grid.nn, 3, 3))
    grad[:, 0, 1] = dUdy
    wpij = np.zeros((grid.nn, 3, 3))
    for i in range(3):
        wpij[:, i, i] += 0.5 * (1.0 - c["C1"]) * k * om
    wpij += c["C2"] * k[:, None, None] * grad
    F[:, 14:23] = wpij.reshape(grid.nn, 9)
    F[:, 23] = 2.0 * k / 3.0
    F[:, 24] = 2.0 * k / 3.0
    F[:, 25] = 2.0 * k / 3.0
    F[:, 26] = uv
    F[:, 29] = om
    # Eq. 58 mean frequency at the wall, (1/C_T) d sqrt(2k)/dy at y = 0 for this k profile.
    F[:, 30] = (1.0 / c["CT"]) * u_tau * iscale * math.sqrt(2.0 * 3.33) / 10.0
    return F


def channel_nu(re_tau: float, u_tau: float = 0.05, h: float = 0.5) -> float:
    return u_tau * h / re_tau


def uniform_fields(nn: int, U=(0.0, 0.0, 0.0), dP=(0.0, 0.0), grad=None, lap=(0.0, 0.0, 0.0),
                   wp=None, uu=None, omega=1.0, omega_w=1.0) -> np.ndarray:
    """Spatially constant nodal fields (homogeneous test flows)."""
    F = np.zeros((nn, NF), dtype=np.float64)
    F[:, 0:3] = U
    F[:, 3:5] = dP
    if grad is not None:
        F[:, 5:11] = np.asarray(grad, dtype=np.float64).reshape(6)
    F[:, 11:14] = lap
    if wp is not None:
        F[:, 14:23] = np.asarray(wp, dtype=np.float64).reshape(9)
    if uu is None:
        uu = (2.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 0.0, 0.0, 0.0)
    F[:, 23:29] = uu
    F[:, 29] = omega
    F[:, 30] = omega_w
    return F


# ----------------------------------------------------------------------------------------
# Named workloads.
# ----------------------------------------------------------------------------------------

def workload(name: str, ppe: int | None = None) -> dict:
    """Grid, fields and parameters of a named synthetic workload (``ppe`` overrides the
    particles per element, and with it the particle-number floor of one tenth of it).

    ``channel_2k``  : 46 x 24 nodes, 2116 triangles, Re_tau 392, 100 particles per element,
                      dt 1e-4, constant C0 = 3.5 and C_phi = 2 mixing, Philox seed 1.
    ``channel_50k`` : 200 x 126 nodes graded to y+ = 1 at both walls, 50,000 triangles,
                      Re_tau 1080, 500 particles per element (25M), Eq. 11 C0 and Eq. 25 t_m.
    ``channel_tiny``: 8 x 5 nodes, 64 triangles (parity at sizes the oracle finishes fast).
    """
    if name == "channel_2k":
        g = channel_grid(46, 24, jitter_x=0.2, jitter_y=0.1, seed=1)
        re = 392.0
        p = dict(c0_mode=1, C0=3.5, tm_mode=1, Cphi=2.0, seed=1, ppe=100, dt=1e-4, steps=10)
    elif name == "channel_50k":
        re = 1080.0
        nu = channel_nu(re)
        g = channel_grid(200, 126, graded_y1=nu / 0.05, jitter_x=0.2, jitter_y=0.1, seed=2)
        p = dict(c0_mode=0, C0=0.0, tm_mode=0, Cphi=2.0, seed=2, ppe=500, dt=1e-4, steps=200)
    elif name == "channel_tiny":
        g = channel_grid(8, 5, jitter_x=0.2, jitter_y=0.1, seed=3)
        re = 392.0
        p = dict(c0_mode=1, C0=3.5, tm_mode=1, Cphi=2.0, seed=3, ppe=40, dt=1e-4, steps=3)
    else:
        raise KeyError(name)
    if ppe is not None:
        p["ppe"] = int(ppe)
    nu = channel_nu(re)
    fields = channel_fields(g, re)
    params = dict(TABLE4)
    params.update(nu=nu, Cs=0.02, Ct=0.7, src_x=0.5, src_y=0.5, src_r=0.02,
                  bins=(4, 4, 4), min_per_bin=2, minnpel=max(1, p["ppe"] // 10),
                  interp_mode=0, period_x=g.period_x)
    params.update({k: v for k, v in p.items() if k not in ("ppe", "dt", "steps")})
    return dict(name=name, grid=g, fields=fields, params=params, ppe=p["ppe"], dt=p["dt"],
                steps=p["steps"], re_tau=re)


def redistribution_workload(name: str, ppe: int | None = None, ratio: int = 10) -> dict:
    """The particle-redistribution test of Sect. 3.7 (Fig. 3): the simplified model of
    Eqs. 46-47 (``model = 1``, alpha = 0.5) on a rectangle [0, 1] x [0, 1], periodic in x,
    with free-slip boundaries at y = 0 and y = 1 and rows graded geometrically toward both
    (the stretching that empties the thin cells unless particle-number control refills
    them).  Equal particles per element at the start; velocities N(0, 1) per component
    (Eq. 48: zero mean field, <u_i u_j> = delta_ij); MINNPEL = ppe / ratio (Eq. 51: the
    ratio is held fixed across particle numbers); no scalar source.

    ``redist_1k``  : 24 columns x 33 node rows, first row 2e-3 high, 1536 triangles,
                     200 particles per element (Fig. 4 uses 50 to 800), dt 0.01.
    ``redist_tiny``: 8 columns x 7 node rows, first row 0.02 high, 96 triangles, 40 per
                     element (parity at sizes the oracle finishes fast).
    """
    if name == "redist_1k":
        g = channel_grid(24, 33, lx=1.0, graded_y1=2e-3, jitter_x=0.2, jitter_y=0.1, seed=7)
        p = dict(seed=7, ppe=200, dt=0.01, steps=400)
    elif name == "redist_tiny":
        g = channel_grid(8, 7, lx=1.0, graded_y1=0.02, jitter_x=0.2, jitter_y=0.1, seed=8)
        p = dict(seed=8, ppe=40, dt=0.01, steps=20)
    else:
        raise KeyError(name)
    if ppe is not None:
        p["ppe"] = int(ppe)
    # the channel walls become free-slip boundaries
    tag = np.where(g.edge_tag == 1, 2, g.edge_tag).astype(np.int8)
    g = Grid(node_xy=g.node_xy, tri=g.tri, edge_tag=tag, period_x=g.period_x)
    fields = uniform_fields(g.nn, U=(0.0, 0.0, 0.0), uu=(1.0, 1.0, 1.0, 0.0, 0.0, 0.0),
                            omega=1.0, omega_w=1.0)
    params = dict(TABLE4)
    params.update(model=1, alpha=0.5, nu=0.0, source_on=0, bins=(4, 4, 4), min_per_bin=2,
                  minnpel=max(1, p["ppe"] // ratio), interp_mode=0, period_x=g.period_x,
                  seed=p["seed"])
    return dict(name=name, grid=g, fields=fields, params=params, ppe=p["ppe"], dt=p["dt"],
                steps=p["steps"])


# ----------------------------------------------------------------------------------------
# Batches of independent instances (inputs of one batched context).
# ----------------------------------------------------------------------------------------

def channel_instance(n_tri: int, re_tau: float, seed: int, ppe: int, src=(0.5, 0.5),
                     philox_seed: int = 1, instance: int = 0) -> dict:
    """A jittered channel grid of about n_tri triangles (cells about square on [0, 2] x
    [0, 1]), its fields, and the parameters of one instance (C0 from Eq. 11, t_m from
    Eq. 25, MINNPEL = ppe / 10)."""
    rows = max(2, int(round(math.sqrt(n_tri / 4.0))))
    g = channel_grid(2 * rows, rows + 1, jitter_x=0.2, jitter_y=0.1, seed=seed)
    nu = channel_nu(re_tau)
    params = dict(TABLE4)
    params.update(nu=nu, Cs=0.02, Ct=0.7, src_x=float(src[0]), src_y=float(src[1]), src_r=0.02,
                  bins=(4, 4, 4), min_per_bin=2, minnpel=max(1, ppe // 10), interp_mode=0,
                  period_x=g.period_x, c0_mode=0, C0=0.0, tm_mode=0, Cphi=2.0,
                  seed=int(philox_seed), instance=int(instance), source_on=1)
    return dict(grid=g, fields=channel_fields(g, re_tau), params=params, ppe=int(ppe))


def union(instances: list[dict]):
    """Disjoint union of the instances' grids and fields: (grid, fields, elem_first,
    node_first); element and node ids of instance k are offset by elem_first[k] and
    node_first[k]."""
    xy, tri, tag, fl = [], [], [], []
    ef, nf = [0], [0]
    for it in instances:
        g = it["grid"]
        xy.append(g.node_xy)
        tri.append(g.tri + nf[-1])
        tag.append(g.edge_tag)
        fl.append(it["fields"])
        ef.append(ef[-1] + g.ne)
        nf.append(nf[-1] + g.nn)
    grid = Grid(np.concatenate(xy), np.concatenate(tri).astype(np.int32),
                np.concatenate(tag).astype(np.int8), instances[0]["grid"].period_x)
    return grid, np.concatenate(fl), np.array(ef, dtype=np.int32), np.array(nf, dtype=np.int64)


def canyon_scale(n_tri: int) -> int:
    """Scale k of a street-canyon grid of about n_tri triangles (canyon_instance: 120 k^2)."""
    return max(3, int(round(math.sqrt(n_tri / 120.0))))


def canyon_instance(n_tri: int, seed: int, ppe: int, src=(2.0, 0.5), philox_seed: int = 1,
                    instance: int = 0) -> dict:
    """A street-canyon grid of 120 k^2 triangles (k = canyon_scale(n_tri): 4k cavity columns,
    12k channel columns, 3k rows in the channel and in the cavity, first rows 0.08/k high),
    its fields at Re_0 = 12,000, and the parameters of one instance (C0 from Eq. 11, t_m from
    Eq. 25, MINNPEL = ppe / 10, source disc of radius 0.02)."""
    k = canyon_scale(n_tri)
    g = canyon_grid(4 * k, 12 * k, 3 * k, 3 * k, h0=0.08 / k, seed=seed)
    nu = 1.0 / 12000.0
    params = dict(TABLE4)
    params.update(nu=nu, Cs=0.02, Ct=0.7, src_x=float(src[0]), src_y=float(src[1]), src_r=0.02,
                  bins=(4, 4, 4), min_per_bin=2, minnpel=max(1, ppe // 10), interp_mode=0,
                  period_x=g.period_x, c0_mode=0, C0=0.0, tm_mode=0, Cphi=2.0,
                  seed=int(philox_seed), instance=int(instance), source_on=1)
    return dict(grid=g, fields=canyon_fields(g, nu), params=params, ppe=int(ppe))


def ensemble(n_inst: int = 64, tri_lo: float = 1000.0, tri_hi: float = 60000.0,
             ppe_lo: int = 50, ppe_hi: int = 500, total_lo: float = 2.7e8,
             total_hi: float = 3.3e8, key: int = 5) -> list[dict]:
    """The ensemble of independent instances, channel grids at even k and street-canyon
    grids at odd k: triangle counts log-uniform in [tri_lo, tri_hi], particles per element
    uniform in [ppe_lo, ppe_hi], redrawn with the next key until the particle total lies in
    [total_lo, total_hi]; source position (channel: x 0.25..1.75, y 0.2..0.8; cavity:
    x 1.6..2.4, y 0.1..0.9) and Philox seed (1000 + k) per instance."""
    while True:
        rng = np.random.default_rng(key)
        u = rng.random(n_inst)
        v = rng.random(n_inst)
        w = rng.random(n_inst)
        tris = np.round(np.exp(np.log(tri_lo) + u * np.log(tri_hi / tri_lo))).astype(int)
        ppes = (ppe_lo + np.floor(w * (ppe_hi - ppe_lo + 1))).astype(int)
        rows = np.maximum(2, np.round(np.sqrt(tris / 4.0))).astype(int)
        ks = np.array([canyon_scale(int(t)) for t in tris])
        ne = np.where(np.arange(n_inst) % 2 == 0, 4 * rows * rows, 120 * ks * ks)
        total = float(np.sum(ne * ppes))
        if total_lo <= total <= total_hi:
            break
        key += 1
    out = []
    for k in range(n_inst):
        if k % 2 == 0:
            src = (0.25 + 1.5 * u[k], 0.2 + 0.6 * v[k])
            out.append(channel_instance(int(tris[k]), 392.0, seed=100 + k, ppe=int(ppes[k]),
                                        src=src, philox_seed=1000 + k, instance=k))
        else:
            src = (1.6 + 0.8 * u[k], 0.1 + 0.8 * v[k])
            out.append(canyon_instance(int(tris[k]), seed=100 + k, ppe=int(ppes[k]), src=src,
                                       philox_seed=1000 + k, instance=k))
    return out


# ----------------------------------------------------------------------------------------
# Street canyon: a periodic channel [0, 4] x [1, 2] over a cavity [1.5, 2.5] x [0, 1].
# ----------------------------------------------------------------------------------------

def _graded(n: int, length: float, h0: float, both: bool) -> np.ndarray:
    """n cells on [0, length]: geometric widths from h0 at the start (and, with both, at the
    end too), growth ratio solved so the widths sum to length."""
    k = np.arange(n)
    m = np.minimum(k, n - 1 - k) if both else k

    def total(r: float) -> float:
        return float(np.sum(h0 * r ** m))

    if total(1.0) >= length:                        # uniform cells already fit
        return np.linspace(0.0, length, n + 1)
    lo, hi = 1.0, 2.0
    while total(hi) < length:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < length:
            lo = mid
        else:
            hi = mid
    w = h0 * (0.5 * (lo + hi)) ** m
    x = np.concatenate([[0.0], np.cumsum(w)])
    x *= length / x[-1]
    return x


def canyon_grid(nc: int, no: int, ny: int, mc: int, h0: float, jitter_x: float = 0.2,
                jitter_y: float = 0.1, seed: int = 1) -> Grid:
    """Street-canyon grid.  The upper block has nc + no node columns (periodic in x with
    period 4): nc cells across the cavity opening [1.5, 2.5] and no cells over [2.5, 5.5]
    (wrapping to 1.5), both graded toward x = 1.5 and 2.5; ny cells in y over [1, 2]
    graded toward the floor y = 1.  The cavity has the opening's nc cells in x and mc cells
    in y over [0, 1], graded toward all its walls; its top node row is the upper block's
    floor row.  Edge tags: free-slip (2) at y = 2; no-slip (1) on the floor outside the
    opening, on the cavity's side walls and on its bottom.  Nodes on boundaries and on the
    floor row move only along their line; corners stay put."""
    rng = np.random.default_rng(seed)
    L = 4.0
    xc = 1.5 + _graded(nc, 1.0, h0, True)                  # opening, both ends refined
    xo = 2.5 + _graded(no, 3.0, h0, True)[1:-1]            # outer part, wraps to 1.5
    xs = np.concatenate([xc, xo])                          # nx = nc + no columns
    nx = xs.shape[0]
    yu = 1.0 + _graded(ny, 1.0, h0, False)                  # upper rows, refined at the floor
    yc = _graded(mc, 1.0, h0, True)[:-1]                    # cavity rows below y = 1
    # upper block nodes
    XU = np.repeat(xs[None, :], ny + 1, axis=0)
    YU = np.repeat(yu[:, None], nx, axis=1)
    # cavity nodes (rows below the floor row), columns of the opening
    XC = np.repeat(xc[None, :], mc, axis=0)
    YC = np.repeat(yc[:, None], nc + 1, axis=1)

    def local(v):
        d = np.empty_like(v)
        d[0] = v[1] - v[0]
        d[-1] = v[-1] - v[-2]
        d[1:-1] = np.minimum(v[1:-1] - v[:-2], v[2:] - v[1:-1])
        return d

    dxu = np.minimum(np.abs(np.diff(np.concatenate([xs, [xs[0] + L]]))),
                     np.abs(np.diff(np.concatenate([[xs[-1] - L], xs]))))
    dyu, dxc, dyc = local(yu), local(xc), local(np.concatenate([yc, [1.0]]))[:-1]
    jxu = rng.uniform(-jitter_x, jitter_x, XU.shape) * dxu[None, :]
    jyu = rng.uniform(-jitter_y, jitter_y, YU.shape) * dyu[:, None]
    jxc = rng.uniform(-jitter_x, jitter_x, XC.shape) * dxc[None, :]
    jyc = rng.uniform(-jitter_y, jitter_y, YC.shape) * dyc[:, None]
    jyu[0, :] = 0.0                 # floor row
    jyu[-1, :] = 0.0                # top
    jxu[:, 0] = 0.0                 # x = 1.5 and 2.5 lines stay straight in the upper block's
    jxu[:, nc] = 0.0                # floor row (corners) ...
    jxu[1:, 0] = rng.uniform(-jitter_x, jitter_x, ny) * dxu[0]     # ... but move above it
    jxu[1:, nc] = rng.uniform(-jitter_x, jitter_x, ny) * dxu[nc]
    jxc[:, 0] = 0.0                 # cavity side walls
    jxc[:, -1] = 0.0
    jyc[0, :] = 0.0                 # cavity bottom
    XU = np.mod(XU + jxu, L)
    YU = YU + jyu
    XC = XC + jxc
    YC = YC + jyc
    nu_nodes = (ny + 1) * nx
    node_xy = np.concatenate([np.stack([XU.ravel(), YU.ravel()], 1),
                              np.stack([XC.ravel(), YC.ravel()], 1)]).astype(np.float64)

    def uid(j, i):
        return j * nx + (i % nx)

    def cid(j, i):   # cavity row j (mc = the floor row of the upper block)
        return np.where(j >= mc, uid(0, i), nu_nodes + np.minimum(j, mc - 1) * (nc + 1) + i)

    quads = []
    J, I = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    J, I = J.ravel(), I.ravel()
    quads.append(np.stack([uid(J, I), uid(J, I + 1), uid(J + 1, I + 1), uid(J + 1, I)], 1))
    J, I = np.meshgrid(np.arange(mc), np.arange(nc), indexing="ij")
    J, I = J.ravel(), I.ravel()
    quads.append(np.stack([cid(J, I), cid(J, I + 1), cid(J + 1, I + 1), cid(J + 1, I)], 1))
    q = np.concatenate(quads)
    n00, n10, n11, n01 = q[:, 0], q[:, 1], q[:, 2], q[:, 3]

    def unwrapped(n, ref):
        x = node_xy[n, 0].copy()
        d = x - node_xy[ref, 0]
        x = np.where(d > 0.5 * L, x - L, np.where(d < -0.5 * L, x + L, x))
        return x, node_xy[n, 1]

    x00, y00 = unwrapped(n00, n00)
    x10, y10 = unwrapped(n10, n00)
    x11, y11 = unwrapped(n11, n00)
    x01, y01 = unwrapped(n01, n00)
    use_a = _incircle(x00, y00, x10, y10, x11, y11, x01, y01) <= 0.0

    def area2(ax, ay, bx, by, cx, cy):
        return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)

    # nodes on the solid boundary (walls and the free-slip top): no triangle may have all
    # three there (near a corner that would make a triangle with no interior node)
    nn = node_xy.shape[0]
    bnd = np.zeros(nn, bool)
    bnd[:nx] = True                                  # floor row (walls, corners, opening)
    bnd[ny * nx:(ny + 1) * nx] = True                # top
    cav_ids = np.arange(nu_nodes, nn)
    cc = (cav_ids - nu_nodes) % (nc + 1)
    cr = (cav_ids - nu_nodes) // (nc + 1)
    bnd[cav_ids[(cc == 0) | (cc == nc) | (cr == 0)]] = True
    a_allb = (bnd[n00] & bnd[n10] & bnd[n11]) | (bnd[n00] & bnd[n11] & bnd[n01])
    b_allb = (bnd[n00] & bnd[n10] & bnd[n01]) | (bnd[n10] & bnd[n11] & bnd[n01])
    a_ok = (area2(x00, y00, x10, y10, x11, y11) > 0) & (area2(x00, y00, x11, y11, x01, y01) > 0)
    b_ok = (area2(x00, y00, x10, y10, x01, y01) > 0) & (area2(x10, y10, x11, y11, x01, y01) > 0)
    a_good, b_good = a_ok & ~a_allb, b_ok & ~b_allb
    use_a = np.where(a_good & b_good, use_a, np.where(a_good, True, np.where(b_good, False, a_ok)))
    if not np.all(np.where(use_a, a_ok, b_ok)):
        raise ValueError("jitter too large: a quad admits no valid split")
    t1 = np.where(use_a[:, None], np.stack([n00, n10, n11], 1), np.stack([n00, n10, n01], 1))
    t2 = np.where(use_a[:, None], np.stack([n00, n11, n01], 1), np.stack([n10, n11, n01], 1))
    tri = np.empty((2 * t1.shape[0], 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2

    # boundary classes of the nodes
    ids = np.arange(nn)
    col = np.full(nn, -1)
    col[:nu_nodes] = ids[:nu_nodes] % nx
    row_u = np.full(nn, -1)
    row_u[:nu_nodes] = ids[:nu_nodes] // nx
    ccol = np.full(nn, -1)
    crow = np.full(nn, -1)
    ccol[nu_nodes:] = (ids[nu_nodes:] - nu_nodes) % (nc + 1)
    crow[nu_nodes:] = (ids[nu_nodes:] - nu_nodes) // (nc + 1)
    top = row_u == ny
    floor = row_u == 0
    in_open = floor & (col >= 0) & (col <= nc)             # floor nodes over the opening
    left = (ccol == 0) | (floor & (col == 0))
    right = (ccol == nc) | (floor & (col == nc))
    bottom = crow == 0
    edge_tag = np.zeros(tri.shape, dtype=np.int8)
    for k in range(3):
        a = tri[:, (k + 1) % 3]
        b = tri[:, (k + 2) % 3]
        fs = top[a] & top[b]
        floor_wall = floor[a] & floor[b] & ~(in_open[a] & in_open[b])
        cav_wall = ((left[a] & left[b]) | (right[a] & right[b]) | (bottom[a] & bottom[b])) & \
            ((a >= nu_nodes) | (b >= nu_nodes))
        edge_tag[:, k] = np.where(fs, 2, np.where(floor_wall | cav_wall, 1, 0))
    return Grid(node_xy=node_xy, tri=tri, edge_tag=edge_tag, period_x=L)


def canyon_fields(grid: Grid, nu: float, u_tau: float = 0.05, umax_cav: float = 0.3,
                  params: dict | None = None) -> np.ndarray:
    """Nodal fields [nn, 32] of the street canyon.  Above the floor (y >= 1): the
    half-channel profiles of channel_fields with wall distance y - 1 and height 1 (total
    shear stress falling linearly to zero at the free-slip top).  In the cavity: the vortex
    of streamfunction A sin^2(pi (x - 1.5)) sin^2(pi y) with max |U| = umax_cav, k and omega
    of the near-wall forms (half the channel's) in the distance to the nearest cavity wall,
    isotropic stresses, no mean-pressure gradient.  k and omega use the distance to the
    nearest solid wall everywhere (over the opening: to its corners), so they vanish on
    walls only.  Derivatives are analytic."""
    c = dict(TABLE4)
    if params:
        c.update({k: v for k, v in params.items() if k in c})
    x = grid.node_xy[:, 0]
    y = grid.node_xy[:, 1]
    F = np.zeros((grid.nn, NF), dtype=np.float64)
    iscale = u_tau / nu
    up_m = y >= 1.0
    cav = ~up_m
    # distance to the nearest solid wall (the floor outside the opening, the cavity walls;
    # over the opening the nearest of its two corners) and its y-derivative
    xm = np.mod(x, 4.0)
    over = (xm > 1.5) & (xm < 2.5)
    dcorner = np.sqrt(np.minimum((xm - 1.5) ** 2, (xm - 2.5) ** 2) + (y - 1.0) ** 2)
    dw_up = np.where(over, dcorner, np.maximum(y - 1.0, 0.0))
    ddw_dy = np.where(over, (y - 1.0) / np.maximum(dcorner, 1e-300), 1.0)
    xi = x - 1.5
    dw_cav = np.maximum(np.minimum(np.minimum(xi, 1.0 - xi), y), 0.0)
    dw = np.where(up_m, dw_up, dw_cav)
    dp_ = iscale * dw
    ek = np.exp(-dp_ / 10.0)
    kp = 3.33 * (1.0 - ek) ** 2
    dkp = 3.33 * 2.0 * (1.0 - ek) * ek / 10.0
    k_w = u_tau ** 2 * kp
    om_w = (u_tau ** 2 / nu) * 0.73 / (dp_ + 8.1)
    # upper part: half-channel mean velocity in y - 1
    yw = np.maximum(y - 1.0, 0.0)
    yp = iscale * yw
    upv, dup, ddup = _reichardt(yp)
    fv = (1.0 - np.exp(-dp_ / 26.0)) ** 2
    F[up_m, 0] = (u_tau * upv)[up_m]
    F[up_m, 3] = -u_tau ** 2 / 1.0
    F[up_m, 4] = (-(2.0 / 3.0) * u_tau ** 2 * iscale * dkp * ddw_dy)[up_m]
    F[up_m, 6] = (u_tau * iscale * dup)[up_m]
    F[up_m, 11] = (u_tau * iscale ** 2 * ddup)[up_m]
    F[up_m, 23] = F[up_m, 24] = F[up_m, 25] = (2.0 * k_w / 3.0)[up_m]
    F[up_m, 26] = (-u_tau ** 2 * (1.0 - yw) * fv)[up_m]
    F[up_m, 29] = om_w[up_m]
    # cavity vortex
    A = umax_cav / math.pi
    xi = x - 1.5
    s2x, s2y = np.sin(2 * math.pi * xi), np.sin(2 * math.pi * y)
    c2x, c2y = np.cos(2 * math.pi * xi), np.cos(2 * math.pi * y)
    sx2, sy2 = np.sin(math.pi * xi) ** 2, np.sin(math.pi * y) ** 2
    pi = math.pi
    U = A * pi * sx2 * s2y
    V = -A * pi * s2x * sy2
    dUdx = A * pi ** 2 * s2x * s2y
    dUdy = 2 * A * pi ** 2 * sx2 * c2y
    dVdx = -2 * A * pi ** 2 * c2x * sy2
    dVdy = -dUdx
    lapU = 2 * A * pi ** 3 * c2x * s2y - 4 * pi ** 2 * U
    lapV = -4 * pi ** 2 * V - 2 * A * pi ** 3 * s2x * c2y
    k_ref = 0.5 * 3.33 * u_tau ** 2                 # cavity: half the channel's outer k
    k_c = 0.5 * k_w
    om_c = 0.5 * om_w
    F[cav, 0], F[cav, 1] = U[cav], V[cav]
    F[cav, 5], F[cav, 6], F[cav, 7], F[cav, 8] = dUdx[cav], dUdy[cav], dVdx[cav], dVdy[cav]
    F[cav, 11], F[cav, 12] = lapU[cav], lapV[cav]
    F[cav, 23] = F[cav, 24] = F[cav, 25] = (2.0 * k_c / 3.0)[cav]
    F[cav, 29] = om_c[cav]
    # elliptic-relaxation tensor (local algebraic form) from the fields above
    k_all = 0.5 * (F[:, 23] + F[:, 24] + F[:, 25])
    grad = np.zeros((grid.nn, 3, 3))
    grad[:, 0, 0], grad[:, 0, 1] = F[:, 5], F[:, 6]
    grad[:, 1, 0], grad[:, 1, 1] = F[:, 7], F[:, 8]
    wpij = np.zeros((grid.nn, 3, 3))
    for i in range(3):
        wpij[:, i, i] += 0.5 * (1.0 - c["C1"]) * k_all * F[:, 29]
    wpij += c["C2"] * k_all[:, None, None] * grad
    F[:, 14:23] = wpij.reshape(grid.nn, 9)
    # Eq. 58 wall frequency: (1/C_T) d sqrt(2k)/dn at the wall for these k profiles
    F[:, 30] = np.where(up_m, (1.0 / c["CT"]) * u_tau * iscale * math.sqrt(2.0 * 3.33) / 10.0,
                        (1.0 / c["CT"]) * math.sqrt(2.0 * k_ref) * iscale / 10.0)
    return F


def canyon_workload(name: str, ppe: int | None = None) -> dict:
    """``canyon_2k``: about 2,000 triangles, 20 particles per element, FP64 parity size.
    ``canyon_200k``: about 200,000 triangles graded to y+ = 1 at the floor and the cavity
    walls and corners, 100 particles per element (about 20M).  Re_0 = 12,000 (U_max = 1,
    H = 1, nu = 1/12,000); source disc of radius 0.01 at (2.0, 0.5); Eq. 11 C0, Eq. 25 t_m;
    MINNPEL = ppe / 10; dt = 1e-4."""
    nu = 1.0 / 12000.0
    if name == "canyon_2k":
        g = canyon_grid(16, 48, 12, 12, h0=0.02, seed=4)
        p = dict(ppe=20, seed=4, src_r=0.05)
    elif name == "canyon_200k":
        g = canyon_grid(160, 480, 125, 125, h0=nu / 0.05, seed=5)
        p = dict(ppe=100, seed=5, src_r=0.01)
    else:
        raise KeyError(name)
    if ppe is not None:
        p["ppe"] = int(ppe)
    params = dict(TABLE4)
    params.update(nu=nu, Cs=0.02, Ct=0.7, src_x=2.0, src_y=0.5, src_r=p["src_r"],
                  bins=(4, 4, 4), min_per_bin=2, minnpel=max(1, p["ppe"] // 10),
                  interp_mode=0, period_x=g.period_x, c0_mode=0, C0=0.0, tm_mode=0, Cphi=2.0,
                  seed=p["seed"], source_on=1)
    return dict(name=name, grid=g, fields=canyon_fields(g, nu), params=params, ppe=p["ppe"],
                dt=1e-4, steps=3)
