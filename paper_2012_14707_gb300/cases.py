"""Seeded synthetic inputs for the slip-wall D2Q9 solver.

This module builds geometry only: solid masks, the boundary links
(fluid node, unknown incoming direction, distance ratio gamma, wall velocity
at the wall point) and the scalar case data (Kn, characteristic length H,
body acceleration).  It holds none of the method's arithmetic: no relaxation
times, no slip coefficients, no collision or boundary formulas.  Both the
FP64 oracle and the CUDA library consume exactly these arrays, so the two
sides see identical distance ratios.

Conventions (Sec. 2, Eq. 3 and Fig. 1 of the paper):
  * D2Q9 velocities c_0..c_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),
    (-1,-1),(1,-1).
  * Node (x, y) sits at the point (x, y); the mask is row-major, index
    y*nx + x, 1 = solid.
  * A link (x, y, i, q) exists when (x, y) is fluid and the node x_r = x - c_i
    is solid: f_i at (x, y) is unknown after streaming.  q is the paper's
    gamma = |x_b - x_f| / |x_r - x_f|, in (0, 1], with x_b the wall point on
    the segment x_f -> x_r.
  * Non-periodic axes always have solid first and last rows/columns.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.int64)
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.int64)


@dataclasses.dataclass
class Case:
    """One solver input.  Arrays are host numpy arrays."""

    name: str
    nx: int
    ny: int
    periodic_x: bool
    periodic_y: bool
    solid: np.ndarray  # uint8 [ny, nx]
    link_x: np.ndarray  # int32 [n_links]
    link_y: np.ndarray  # int32
    link_dir: np.ndarray  # int32, 1..8
    link_q: np.ndarray  # float64, gamma in (0, 1]
    link_ubx: np.ndarray  # float64, wall velocity at x_b
    link_uby: np.ndarray  # float64
    Kn: float
    H: float  # characteristic length in lattice units (Kn = lambda / H)
    ax: float = 0.0
    ay: float = 0.0
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_links(self) -> int:
        return int(self.link_x.shape[0])

    @property
    def n_fluid(self) -> int:
        return int((self.solid == 0).sum())

    def links_sorted(self) -> "Case":
        """Same case with links ordered by (y, x, dir)."""
        order = np.lexsort((self.link_dir, self.link_x, self.link_y))
        return dataclasses.replace(
            self,
            link_x=self.link_x[order], link_y=self.link_y[order],
            link_dir=self.link_dir[order], link_q=self.link_q[order],
            link_ubx=self.link_ubx[order], link_uby=self.link_uby[order])


# --------------------------------------------------------------------------
# generic helpers
# --------------------------------------------------------------------------

def _wall_candidates(solid: np.ndarray, periodic_x: bool, periodic_y: bool):
    """All (x, y, i) with (x, y) fluid and (x, y) - c_i solid.

    Out-of-domain neighbours on a non-periodic axis count as solid; the
    generators below never put fluid on such an edge, so that case does not
    arise for the cases built here.
    """
    ny, nx = solid.shape
    ys, xs = np.nonzero(solid == 0)
    out_x, out_y, out_i, out_rx, out_ry = [], [], [], [], []
    for i in range(1, 9):
        rx = xs - CX[i]
        ry = ys - CY[i]
        if periodic_x:
            rx = rx % nx
        if periodic_y:
            ry = ry % ny
        inside = (rx >= 0) & (rx < nx) & (ry >= 0) & (ry < ny)
        hit = np.ones_like(inside)
        hit[inside] = solid[ry[inside], rx[inside]] != 0
        out_x.append(xs[hit]); out_y.append(ys[hit])
        out_i.append(np.full(int(hit.sum()), i, dtype=np.int64))
        out_rx.append(rx[hit]); out_ry.append(ry[hit])
    return (np.concatenate(out_x), np.concatenate(out_y), np.concatenate(out_i),
            np.concatenate(out_rx), np.concatenate(out_ry))


def _segment_circle_t(px, py, dx, dy, cx, cy, R, inner):
    """Parameter t in (0, 1] where p + t*d first meets the circle |. - c| = R.

    `inner=True`: p is outside the circle and p + d inside or on it (the
    smaller root).  `inner=False`: p inside, p + d outside or on it (the
    larger root).  Plain quadratic formula in FP64.
    """
    ox = px - cx
    oy = py - cy
    a = dx * dx + dy * dy
    b = 2.0 * (ox * dx + oy * dy)
    c = ox * ox + oy * oy - R * R
    disc = np.maximum(b * b - 4.0 * a * c, 0.0)
    sq = np.sqrt(disc)
    t = np.where(inner, (-b - sq) / (2.0 * a), (-b + sq) / (2.0 * a))
    return np.clip(t, np.finfo(np.float64).tiny, 1.0)


def _make_case(name, solid, periodic_x, periodic_y, lx, ly, li, q, ubx, uby,
               Kn, H, ax=0.0, ay=0.0, meta=None) -> Case:
    ny, nx = solid.shape
    return Case(
        name=name, nx=nx, ny=ny, periodic_x=periodic_x, periodic_y=periodic_y,
        solid=np.ascontiguousarray(solid, dtype=np.uint8),
        link_x=np.asarray(lx, np.int32), link_y=np.asarray(ly, np.int32),
        link_dir=np.asarray(li, np.int32), link_q=np.asarray(q, np.float64),
        link_ubx=np.asarray(ubx, np.float64), link_uby=np.asarray(uby, np.float64),
        Kn=float(Kn), H=float(H), ax=float(ax), ay=float(ay),
        meta=dict(meta or {})).links_sorted()


# --------------------------------------------------------------------------
# flat channel, periodic in x (Sec. 4.A.1, Fig. 3)
# --------------------------------------------------------------------------

def channel(nx: int, m: int, q_bottom: float, q_top: float, Kn: float,
            ax: float = 1e-6, H: float | None = None,
            u_bottom: float = 0.0, u_top: float = 0.0,
            name: str = "slip_channel") -> Case:
    """Channel with m fluid rows between two flat walls.

    Rows 0 and m+1 are solid.  The lower wall lies q_bottom below the first
    fluid row, the upper wall q_top above the last, so every link of a wall
    row has gamma = q of that wall (a diagonal link crosses the wall at the
    same fraction of its length as a vertical one).  The default H is the
    wall-to-wall distance m - 1 + q_bottom + q_top; y of fluid row j
    (1-based) measured from the lower wall is j - 1 + q_bottom.
    """
    ny = m + 2
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    lx, ly, li, rx, ry = _wall_candidates(solid, True, False)
    bottom = ry == 0
    q = np.where(bottom, q_bottom, q_top)
    ubx = np.where(bottom, u_bottom, u_top)
    uby = np.zeros_like(ubx)
    if H is None:
        H = m - 1 + q_bottom + q_top
    return _make_case(name, solid, True, False, lx, ly, li, q, ubx, uby, Kn, H,
                      ax=ax, meta=dict(m=m, q_bottom=q_bottom, q_top=q_top))


# --------------------------------------------------------------------------
# cylindrical Couette flow (Sec. 4.B, Fig. 9)
# --------------------------------------------------------------------------

def annulus(n: int, R1: float, R2: float, Kn: float, omega1: float,
            omega2: float = 0.0, center: float | None = None,
            name: str = "couette", ny: int | None = None) -> Case:
    """n x n lattice (n x ny if ny is given), concentric circles about
    `center` (default the lattice centre).

    A node is solid when its distance r from the centre has r <= R1 or
    r >= R2.  Each link's gamma comes from the exact segment-circle
    intersection; the wall velocity at x_b is omega x (x_b - centre) of the
    wall that was hit.  H = R2 - R1 (Kn = lambda / (R2 - R1)).
    """
    nyy = n if ny is None else int(ny)
    c = (n - 1) / 2.0 if center is None else float(center)
    cy = (nyy - 1) / 2.0 if center is None else float(center)
    yy, xx = np.mgrid[0:nyy, 0:n].astype(np.float64)
    rr = np.hypot(xx - c, yy - cy)
    solid = ((rr <= R1) | (rr >= R2)).astype(np.uint8)
    if R2 > min(c, cy):
        raise ValueError("outer circle must leave a solid edge row")
    lx, ly, li, rx, ry = _wall_candidates(solid, False, False)
    r_ref = np.hypot(rx - c, ry - cy)
    inner = r_ref <= R1
    px = lx.astype(np.float64)
    py = ly.astype(np.float64)
    dx = -CX[li].astype(np.float64)
    dy = -CY[li].astype(np.float64)
    t = _segment_circle_t(px, py, dx, dy, c, cy, np.where(inner, R1, R2), inner)
    bx = px + t * dx - c
    by = py + t * dy - cy
    om = np.where(inner, omega1, omega2)
    ubx = -om * by
    uby = om * bx
    return _make_case(name, solid, False, False, lx, ly, li, t, ubx, uby, Kn,
                      R2 - R1, meta=dict(R1=R1, R2=R2, center=c, center_y=cy,
                                         omega1=omega1, omega2=omega2))


# --------------------------------------------------------------------------
# x-periodic channel packed with random cylinders
# --------------------------------------------------------------------------

def cylinder_array(nx: int, ny: int, seed: int, porosity: float = 0.7,
                   r_min: float = 8.0, r_max: float = 32.0,
                   clearance: float = 2.0, Kn: float = 0.02, ax: float = 1e-5,
                   max_trials: int | None = None,
                   name: str = "cylinder_array") -> Case:
    """Random sequential addition of non-overlapping cylinders.

    Rows 0 and ny-1 are solid, with flat walls halfway (gamma = 1/2) between
    them and the adjacent fluid rows.  Radii are uniform in [r_min, r_max];
    every cylinder keeps `clearance` nodes from the walls, from the x ends
    (no wrap across the periodic seam) and from every other cylinder.
    Cylinders are added until the node porosity drops to `porosity` or
    `max_trials` candidates were rejected in a row.  H is the mean cylinder
    diameter actually placed.
    """
    rng = np.random.default_rng(seed)
    cell = 2.0 * r_max + clearance
    grid: dict[tuple[int, int], list[int]] = {}
    cxs: list[float] = []
    cys: list[float] = []
    rs: list[float] = []
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    label = np.full((ny, nx), -1, np.int32)
    n_total = nx * ny
    n_solid = int(solid.sum())
    max_trials = max_trials or 20000
    misses = 0
    batch = 4096
    while n_solid / n_total < 1.0 - porosity and misses < max_trials:
        rad = rng.uniform(r_min, r_max, batch)
        ccx = rng.uniform(0.0, nx - 1.0, batch)
        ccy = rng.uniform(0.0, ny - 1.0, batch)
        for k in range(batch):
            R, X, Y = float(rad[k]), float(ccx[k]), float(ccy[k])
            if (X - R < clearance or X + R > nx - 1 - clearance
                    or Y - R < 1.0 + clearance or Y + R > ny - 2 - clearance):
                misses += 1
                continue
            ix, iy = int(X / cell), int(Y / cell)
            ok = True
            for jx in (ix - 1, ix, ix + 1):
                for jy in (iy - 1, iy, iy + 1):
                    for idx in grid.get((jx, jy), ()):
                        if math.hypot(X - cxs[idx], Y - cys[idx]) < R + rs[idx] + clearance:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                misses += 1
                if misses >= max_trials:
                    break
                continue
            misses = 0
            idx = len(rs)
            cxs.append(X); cys.append(Y); rs.append(R)
            grid.setdefault((ix, iy), []).append(idx)
            x0, x1 = int(math.ceil(X - R)), int(math.floor(X + R))
            y0, y1 = int(math.ceil(Y - R)), int(math.floor(Y + R))
            sy, sx = np.mgrid[y0:y1 + 1, x0:x1 + 1]
            inside = (sx - X) ** 2 + (sy - Y) ** 2 <= R * R
            sub = solid[y0:y1 + 1, x0:x1 + 1]
            n_solid += int((inside & (sub == 0)).sum())
            sub[inside] = 1
            label[y0:y1 + 1, x0:x1 + 1][inside] = idx
            if n_solid / n_total >= 1.0 - porosity:
                break
    cxa = np.asarray(cxs)
    cya = np.asarray(cys)
    ra = np.asarray(rs)
    lx, ly, li, rx, ry = _wall_candidates(solid, True, False)
    lab = label[ry, rx]
    wall = lab < 0
    q = np.full(lx.shape, 0.5)
    if (~wall).any():
        sel = ~wall
        k = lab[sel]
        px = lx[sel].astype(np.float64)
        py = ly[sel].astype(np.float64)
        dx = -CX[li[sel]].astype(np.float64)
        dy = -CY[li[sel]].astype(np.float64)
        q[sel] = _segment_circle_t(px, py, dx, dy, cxa[k], cya[k], ra[k],
                                   np.ones(px.shape, bool))
    zeros = np.zeros(lx.shape)
    H = float(2.0 * ra.mean()) if len(ra) else float(ny - 2)
    return _make_case(name, solid, True, False, lx, ly, li, q, zeros, zeros, Kn,
                      H, ax=ax, meta=dict(seed=seed, n_cylinders=len(rs),
                                          porosity=1.0 - n_solid / n_total,
                                          centers_x=cxa, centers_y=cya, radii=ra))


def periodic_box(nx: int, ny: int, name: str = "periodic_box",
                 Kn: float = 0.05, H: float = 10.0, ax: float = 0.0,
                 ay: float = 0.0) -> Case:
    """Fully periodic box with no solid node and no link."""
    solid = np.zeros((ny, nx), np.uint8)
    e = np.zeros(0)
    return _make_case(name, solid, True, True, e, e, e, e, e, e, Kn, H,
                      ax=ax, ay=ay)


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------

def config_poiseuille() -> Case:
    """4 x 32 fluid nodes, x-periodic, gamma 0.5 below and 0.3 above,
    Kn = 0.05, a = 1e-6 (FP64 closed-form workload)."""
    return channel(4, 32, 0.5, 0.3, Kn=0.05, ax=1e-6, name="poiseuille_4x32")


def config_couette(Kn: float = 0.05, n: int = 256, R1: float = 60.0,
                   R2: float = 120.0, mach: float = 0.05) -> Case:
    """256^2 annulus, R1 = 60, R2 = 120, inner wall at Ma ~ 0.05, outer at rest."""
    omega1 = mach * math.sqrt(1.0 / 3.0) / R1
    return annulus(n, R1, R2, Kn, omega1, 0.0, name=f"couette_{n}_Kn{Kn:g}")


def config_throughput(seed: int = 0, nx: int = 8192, ny: int = 4096,
                      ax: float = 1e-5) -> Case:
    """8192 x 4096 x-periodic channel of random cylinders (radius 8-32,
    porosity 0.7), Kn = 0.02."""
    return cylinder_array(nx, ny, seed, porosity=0.7, Kn=0.02, ax=ax,
                          name=f"cylinders_{nx}x{ny}_s{seed}")


def random_populations(nx: int, ny: int, seed: int, amp: float = 1e-3) -> np.ndarray:
    """Seeded population field f[9][ny][nx] = w_i (1 + amp * N(0, 1)): a
    perturbed rest state to start parity runs from (an input, not a
    solution of anything)."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    rng = np.random.default_rng(seed)
    return w[:, None, None] * (1.0 + amp * rng.standard_normal((9, ny, nx)))


# --------------------------------------------------------------------------
# inclined channel (Sec. 4.A.2, Fig. 6)
# --------------------------------------------------------------------------

def inclined_channel(nx: int, tan_theta: float, n_ab: float, Kn: float, a: float = 1e-6,
                     offset: float = 0.37, name: str | None = None) -> Case:
    """Channel whose flat walls are inclined at angle theta to the x axis.

    The lattice is nx wide and ny = nx tan(theta) high (an integer), periodic
    in both directions, so that the band wraps onto itself: that is the
    channel periodic along its own direction, one period per lattice.  The
    fluid band lies between the lines y = x tan(theta) + offset and
    y = x tan(theta) + offset + n_ab (vertical extent n_ab, perpendicular
    width H = n_ab cos(theta)), taken modulo ny; the rest is solid.  Each
    link's gamma is the exact crossing of its segment with the wall line it
    cuts.  The body force a acts along the channel, (cos, sin)(theta) a.
    meta holds the line data to evaluate the analytic profile: the signed
    perpendicular distance y' of a node from the lower wall.
    """
    ny_f = nx * tan_theta
    ny = int(round(ny_f))
    if abs(ny - ny_f) > 1e-9 or ny < 2:
        raise ValueError("nx * tan(theta) must be an integer >= 2")
    if n_ab > ny - 2:
        raise ValueError("the band must leave at least two solid rows")
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    # vertical coordinate above the lower wall, folded into [0, ny)
    s = np.mod(yy - xx * tan_theta - offset, ny)
    solid = (~((s > 0.0) & (s < n_ab))).astype(np.uint8)
    lx, ly, li, rx, ry = _wall_candidates(solid, True, True)
    px = lx.astype(np.float64)
    py = ly.astype(np.float64)
    dx = -CX[li].astype(np.float64)
    dy = -CY[li].astype(np.float64)
    # s along the segment p + t d: s(t) = s0 + t (dy - dx tan);  the wall hit
    # is s = 0 (lower) when s decreases, s = n_ab (upper) when it increases.
    s0 = np.mod(py - px * tan_theta - offset, ny)
    ds = dy - dx * tan_theta
    target = np.where(ds < 0, 0.0, n_ab)
    t = (target - s0) / ds
    if np.any(~np.isfinite(t)) or np.any(t <= 0) or np.any(t > 1 + 1e-12):
        raise ValueError("link without a wall crossing in (0, 1]")
    t = np.minimum(t, 1.0)
    zeros = np.zeros(lx.shape)
    cos_t = 1.0 / math.sqrt(1.0 + tan_theta ** 2)
    sin_t = tan_theta * cos_t
    H = n_ab * cos_t
    nm = name or f"inclined_{nx}_tan{tan_theta:g}_nab{n_ab:g}"
    return _make_case(nm, solid, True, True, lx, ly, li, t, zeros, zeros, Kn, H,
                      ax=a * cos_t, ay=a * sin_t,
                      meta=dict(tan_theta=tan_theta, offset=offset, n_ab=n_ab, cos=cos_t,
                                sin=sin_t, a=a))


def inclined_coordinates(case: Case) -> tuple[np.ndarray, np.ndarray]:
    """(y', unit vector along the channel) for an inclined_channel case:
    y' = perpendicular distance of each node from the lower wall."""
    m = case.meta
    yy, xx = np.mgrid[0:case.ny, 0:case.nx].astype(np.float64)
    s = np.mod(yy - xx * m["tan_theta"] - m["offset"], case.ny)
    return s * m["cos"], np.array([m["cos"], m["sin"]])


# --------------------------------------------------------------------------
# batch of uneven cases
# --------------------------------------------------------------------------

def batch_cases(n_cases: int = 512, seed: int = 0, nx_range=(64, 1024), ny_range=(64, 512),
                kn_range=(0.001, 0.1)) -> list[Case]:
    """Seeded batch: sizes uniform over nx_range x ny_range, geometry uniform
    over {slip channel, annulus, random cylinder array}, Kn log-uniform over
    kn_range, driving at Ma ~ 0.02-0.05 (wall speed) or a fixed small body
    force.

    * channel: gamma of each wall ~ U(0.05, 1], force 2e-6 along x;
    * annulus: R2 = 0.45 min(nx, ny), R1 = beta R2 with beta ~ U[0.2, 0.6],
      inner wall at Ma ~ U[0.02, 0.05], outer at rest;
    * cylinder array: radii U[8, min(32, min(nx, ny) / 8)], porosity 0.7,
      force 5e-6 along x.
    """
    rng = np.random.default_rng(seed)
    out = []
    cs = math.sqrt(1.0 / 3.0)
    for k in range(n_cases):
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        kind = int(rng.integers(0, 3))
        Kn = float(math.exp(rng.uniform(math.log(kn_range[0]), math.log(kn_range[1]))))
        if kind == 0:
            gb, gt = float(rng.uniform(0.05, 1.0)), float(rng.uniform(0.05, 1.0))
            c = channel(nx, ny - 2, gb, gt, Kn=Kn, ax=2e-6, name=f"b{k}_channel")
        elif kind == 1:
            R2 = 0.45 * min(nx, ny)
            R1 = float(rng.uniform(0.2, 0.6)) * R2
            ma = float(rng.uniform(0.02, 0.05))
            c = annulus(nx, R1, R2, Kn, ma * cs / R1, 0.0, name=f"b{k}_annulus", ny=ny)
        else:
            rmax = max(8.0, min(32.0, min(nx, ny) / 8.0))
            c = cylinder_array(nx, ny, int(rng.integers(0, 2**31)), porosity=0.7, r_min=8.0,
                               r_max=rmax, Kn=Kn, ax=5e-6, name=f"b{k}_cylinders")
        c.meta["batch_kind"] = ("channel", "annulus", "cylinders")[kind]
        out.append(c)
    return out


def signed_distance(case: Case, clip: float = 32.0) -> np.ndarray:
    """Signed distance (lattice units, clipped to +-clip) of every node to
    the nearest wall of a cylinder_array or channel case: positive in the
    fluid, negative inside solids.  Flat walls sit half a spacing inside
    the solid edge rows (gamma = 1/2 for the cylinder arrays)."""
    ny, nx = case.solid.shape
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    if "q_bottom" in case.meta:
        lo = 1.0 - case.meta["q_bottom"]
        hi = ny - 2 + case.meta["q_top"]
    else:
        lo, hi = 0.5, ny - 1.5
    d = np.minimum(yy - lo, hi - yy)
    d = np.minimum(d, clip)
    cxs = case.meta.get("centers_x", np.zeros(0))
    cys = case.meta.get("centers_y", np.zeros(0))
    rs = case.meta.get("radii", np.zeros(0))
    for X, Y, R in zip(cxs, cys, rs):
        x0, x1 = max(0, int(X - R - clip)), min(nx, int(X + R + clip) + 2)
        y0, y1 = max(0, int(Y - R - clip)), min(ny, int(Y + R + clip) + 2)
        sub = np.hypot(xx[y0:y1, x0:x1] - X, yy[y0:y1, x0:x1] - Y) - R
        d[y0:y1, x0:x1] = np.minimum(d[y0:y1, x0:x1], sub)
    return np.clip(d, -clip, clip)


# --------------------------------------------------------------------------
# three dimensions (D3Q19): the extension the paper names as future work
# --------------------------------------------------------------------------
#
# D3Q19 velocities, in the order both the oracle and the library use: the
# rest velocity, the six axes (+x, -x, +y, -y, +z, -z), then the diagonals of
# the xy, xz and yz planes, each as (+, +), (+, -), (-, +), (-, -).  Node
# (x, y, z) has index (z * ny + y) * nx + x; masks are [nz, ny, nx].

def _d3q19_velocities():
    c = [(0, 0, 0)]
    for a in range(3):
        for s in (1, -1):
            v = [0, 0, 0]
            v[a] = s
            c.append(tuple(v))
    for a, b in ((0, 1), (0, 2), (1, 2)):
        for s1 in (1, -1):
            for s2 in (1, -1):
                v = [0, 0, 0]
                v[a], v[b] = s1, s2
                c.append(tuple(v))
    return np.array(c, dtype=np.int64)


C3 = _d3q19_velocities()


@dataclasses.dataclass
class Case3D:
    """One three-dimensional solver input (D3Q19).  Arrays are host numpy arrays."""

    name: str
    nx: int
    ny: int
    nz: int
    periodic: tuple  # (x, y, z) booleans
    solid: np.ndarray  # uint8 [nz, ny, nx]
    link_x: np.ndarray  # int32 [n_links]
    link_y: np.ndarray
    link_z: np.ndarray
    link_dir: np.ndarray  # int32, 1..18
    link_q: np.ndarray  # float64, gamma in (0, 1]
    link_ub: np.ndarray  # float64 [n_links, 3], wall velocity at x_b
    Kn: float
    H: float
    a: tuple = (0.0, 0.0, 0.0)  # body acceleration
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_links(self) -> int:
        return int(self.link_x.shape[0])

    @property
    def n_fluid(self) -> int:
        return int((self.solid == 0).sum())


def _wall_candidates_3d(solid: np.ndarray, periodic):
    """All (x, y, z, i) with (x, y, z) fluid and (x, y, z) - c_i solid."""
    nz, ny, nx = solid.shape
    zs, ys, xs = np.nonzero(solid == 0)
    out = [[], [], [], [], [], [], []]
    dims = (nx, ny, nz)
    for i in range(1, 19):
        r = [xs - C3[i, 0], ys - C3[i, 1], zs - C3[i, 2]]
        inside = np.ones(xs.shape, bool)
        for a in range(3):
            if periodic[a]:
                r[a] = r[a] % dims[a]
            else:
                inside &= (r[a] >= 0) & (r[a] < dims[a])
        hit = np.ones(xs.shape, bool)
        hit[inside] = solid[r[2][inside], r[1][inside], r[0][inside]] != 0
        for lst, v in zip(out, (xs, ys, zs, np.full(xs.shape, i), r[0], r[1], r[2])):
            lst.append(v[hit])
    return tuple(np.concatenate(v) for v in out)


def _make_case3d(name, solid, periodic, lx, ly, lz, li, q, ub, Kn, H, a, meta=None) -> Case3D:
    order = np.lexsort((li, lx, ly, lz))
    nz, ny, nx = solid.shape
    return Case3D(name=name, nx=nx, ny=ny, nz=nz, periodic=tuple(bool(p) for p in periodic),
                  solid=np.ascontiguousarray(solid, np.uint8),
                  link_x=np.asarray(lx, np.int32)[order], link_y=np.asarray(ly, np.int32)[order],
                  link_z=np.asarray(lz, np.int32)[order], link_dir=np.asarray(li, np.int32)[order],
                  link_q=np.asarray(q, np.float64)[order],
                  link_ub=np.ascontiguousarray(np.asarray(ub, np.float64).reshape(-1, 3)[order]),
                  Kn=float(Kn), H=float(H), a=tuple(float(v) for v in a), meta=dict(meta or {}))


def channel3d(nx: int, ny: int, m: int, q_bottom: float, q_top: float, Kn: float,
              ax: float = 1e-6, u_top: float = 0.0, name: str = "slip_channel_3d") -> Case3D:
    """Channel with m fluid layers between two flat walls normal to z,
    periodic in x and y: layers z = 0 and m + 1 are solid, the lower wall
    lies q_bottom below the first fluid layer and the upper one q_top above
    the last (every link of a wall layer has gamma = q of that wall), the
    upper wall moves along x at u_top.  H = m - 1 + q_bottom + q_top."""
    nz = m + 2
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[0] = 1
    solid[nz - 1] = 1
    lx, ly, lz, li, rx, ry, rz = _wall_candidates_3d(solid, (True, True, False))
    bottom = rz == 0
    q = np.where(bottom, q_bottom, q_top)
    ub = np.zeros((lx.shape[0], 3))
    ub[~bottom, 0] = u_top
    return _make_case3d(name, solid, (True, True, False), lx, ly, lz, li, q, ub, Kn,
                        m - 1 + q_bottom + q_top, (ax, 0.0, 0.0),
                        meta=dict(m=m, q_bottom=q_bottom, q_top=q_top))


def periodic_box3d(nx: int, ny: int, nz: int, a=(1e-5, 0.0, 0.0), Kn: float = 0.05,
                   name: str = "box_3d") -> Case3D:
    """Fully periodic box without walls (no links)."""
    solid = np.zeros((nz, ny, nx), np.uint8)
    e = np.zeros(0, np.int32)
    return _make_case3d(name, solid, (True, True, True), e, e, e, e, np.zeros(0), np.zeros((0, 3)),
                        Kn, float(min(nx, ny, nz)), a)


def sphere_array3d(n: int, n_spheres: int, r_range=(3.0, 6.0), seed: int = 0, Kn: float = 0.02,
                   a=(1e-5, 0.0, 0.0), name: str = "spheres_3d") -> Case3D:
    """Periodic n^3 box with non-overlapping spheres (seeded random
    sequential addition, radii uniform in r_range, 2-node clearance, wrapped
    distances); gamma from the exact segment-sphere intersection (the nearest
    periodic image of the sphere), walls at rest.  H = mean diameter."""
    rng = np.random.default_rng(seed)
    centres, radii = [], []
    tries = 0
    while len(centres) < n_spheres and tries < 20000:
        tries += 1
        r = rng.uniform(*r_range)
        c = rng.uniform(0, n, size=3)
        ok = True
        for c2, r2 in zip(centres, radii):
            d = np.abs(c - c2)
            d = np.minimum(d, n - d)
            if np.sqrt((d * d).sum()) < r + r2 + 2.0:
                ok = False
                break
        if ok:
            centres.append(c)
            radii.append(r)
    zz, yy, xx = np.mgrid[0:n, 0:n, 0:n].astype(np.float64)
    solid = np.zeros((n, n, n), np.uint8)
    owner = np.full((n, n, n), -1, np.int64)
    for k, (c, r) in enumerate(zip(centres, radii)):
        dx = (xx - c[0] + n / 2) % n - n / 2
        dy = (yy - c[1] + n / 2) % n - n / 2
        dz = (zz - c[2] + n / 2) % n - n / 2
        inside = dx * dx + dy * dy + dz * dz <= r * r
        solid[inside] = 1
        owner[inside] = k
    lx, ly, lz, li, rx, ry, rz = _wall_candidates_3d(solid, (True, True, True))
    q = np.empty(lx.shape[0])
    for t in range(lx.shape[0]):
        k = owner[rz[t], ry[t], rx[t]]
        c, r = centres[k], radii[k]
        p = np.array([lx[t], ly[t], lz[t]], np.float64)
        p = c + ((p - c + n / 2) % n - n / 2)  # the fluid node next to the nearest image
        d = -C3[li[t]].astype(np.float64)
        o = p - c
        aa, bb, cc = d @ d, 2 * (o @ d), o @ o - r * r
        q[t] = min(1.0, max(np.finfo(np.float64).tiny,
                            (-bb - math.sqrt(max(bb * bb - 4 * aa * cc, 0.0))) / (2 * aa)))
    H = 2.0 * float(np.mean(radii)) if radii else float(n)
    return _make_case3d(name, solid, (True, True, True), lx, ly, lz, li, q,
                        np.zeros((lx.shape[0], 3)), Kn, H, a,
                        meta=dict(n_spheres=len(centres)))


def sphere_pack3d(nx: int, ny: int, nz: int, seed: int = 0, porosity: float = 0.8,
                  r_range=(6.0, 12.0), Kn: float = 0.02, a=(1e-6, 0.0, 0.0),
                  clearance: float = 1.0, name: str = "sphere_pack_3d") -> Case3D:
    """Periodic nx x ny x nz box filled with non-overlapping spheres (seeded
    random sequential addition, radii uniform in r_range, `clearance` nodes
    between surfaces, wrapped distances) until their volume reaches
    (1 - porosity) of the box; gamma from the exact segment-sphere
    intersection with the nearest periodic image; walls at rest; H = mean
    diameter.  Vectorised for lattices of tens of millions of nodes."""
    rng = np.random.default_rng(seed)
    dims = np.array([nx, ny, nz], np.float64)
    target = (1.0 - porosity) * nx * ny * nz
    centres = np.zeros((0, 3))
    radii = np.zeros(0)
    vol, tries = 0.0, 0
    while vol < target and tries < 200000:
        tries += 1
        r = rng.uniform(*r_range)
        c = rng.uniform(0.0, 1.0, size=3) * dims
        if centres.shape[0]:
            d = np.abs(centres - c)
            d = np.minimum(d, dims - d)
            if (np.sqrt((d * d).sum(axis=1)) < radii + r + clearance).any():
                continue
        centres = np.vstack([centres, c])
        radii = np.append(radii, r)
        vol += 4.0 / 3.0 * math.pi * r ** 3
    solid = np.zeros((nz, ny, nx), np.uint8)
    owner = np.full((nz, ny, nx), -1, np.int32)
    for k in range(radii.shape[0]):
        c, r = centres[k], radii[k]
        lo = np.floor(c - r).astype(np.int64)
        hi = np.ceil(c + r).astype(np.int64)
        ax = [np.arange(lo[e], hi[e] + 1) for e in range(3)]
        gz, gy, gx = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        inside = (gx - c[0]) ** 2 + (gy - c[1]) ** 2 + (gz - c[2]) ** 2 <= r * r
        ix, iy, iz = gx[inside] % nx, gy[inside] % ny, gz[inside] % nz
        solid[iz, iy, ix] = 1
        owner[iz, iy, ix] = k
    lx, ly, lz, li, rx, ry, rz = _wall_candidates_3d(solid, (True, True, True))
    k = owner[rz, ry, rx]
    cc, rr = centres[k], radii[k]
    p = np.stack([lx, ly, lz], axis=1).astype(np.float64)
    p = cc + ((p - cc + dims / 2) % dims - dims / 2)  # the fluid node next to the nearest image
    d = -C3[li].astype(np.float64)
    o = p - cc
    aa = (d * d).sum(axis=1)
    bb = 2.0 * (o * d).sum(axis=1)
    ee = (o * o).sum(axis=1) - rr * rr
    t = (-bb - np.sqrt(np.maximum(bb * bb - 4.0 * aa * ee, 0.0))) / (2.0 * aa)
    q = np.clip(t, np.finfo(np.float64).tiny, 1.0)
    H = 2.0 * float(radii.mean()) if radii.shape[0] else float(min(nx, ny, nz))
    return _make_case3d(name, solid, (True, True, True), lx, ly, lz, li, q,
                        np.zeros((lx.shape[0], 3)), Kn, H, a,
                        meta=dict(n_spheres=int(radii.shape[0]), porosity=porosity,
                                  centres=centres, radii=radii))
