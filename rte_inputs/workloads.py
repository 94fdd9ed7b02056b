"""Seeded synthetic workloads (inputs only; no arithmetic of the method).

Units: cm and ps.  Every medium is a pair of FP64 arrays (mua, mus) of shape
(ny, nx), indexed [j, i] = value at (x_i, y_j) with x_i = xmin + i dx and
y_j = ymin + j dy, so nx and ny count grid points (N_x + 1 in the paper's
notation, Sec. 4.3).  Beams follow eqs. (RTEsources2)/(sourcelab); detectors
follow eq. (OpMed).  The speed of light in the medium is carried as an input
(c = c0 / n_in with c0 = 0.0299792458 cm/ps) so that no side derives it.

The paper's media (an MRI neck section, a layered head) and its lab data are
not available; these seeded media stand in for them, with the sizes, optical
ranges and source/detector layouts of the workloads the method is run on.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

C0_CM_PER_PS = 0.0299792458
BASE_SEED = 2202_09421


@dataclass
class Grid:
    nx: int
    ny: int
    xmin: float
    xmax: float
    ymin: float
    ymax: float
    M: int

    @property
    def dx(self) -> float:
        return (self.xmax - self.xmin) / (self.nx - 1)

    @property
    def dy(self) -> float:
        return (self.ymax - self.ymin) / (self.ny - 1)


@dataclass
class Optics:
    g: float = 0.9            # Henyey-Greenstein anisotropy
    n_in: float = 1.4         # refractive index inside the domain
    n_out: float = 1.0        # refractive index outside
    hg_exponent: float = 1.5  # exponent of the HG denominator as printed


@dataclass
class Beam:
    """One laser beam s_k: position on the boundary, direction theta (rad),
    spatial spread sigma_x (cm), angular spread sigma_theta (rad), temporal
    centre t_s and spread sigma_t (ps), delay tau (ps).  profile 0: Gaussian
    exp(-(t - t_s)^2 / (2 sigma_t^2)); profile 1: window w(|t - t_s| / sigma_t)."""
    x: float
    y: float
    theta: float
    sigma_x: float = 0.3
    sigma_theta: float = np.pi / 4
    t_s: float = 30.0
    sigma_t: float = 10.0
    tau: float = 0.0
    profile: int = 0
    amplitude: float = 1.0


@dataclass
class Detector:
    x: float
    y: float
    sigma_d: float = 0.2


@dataclass
class Workload:
    name: str
    grid: Grid
    optics: Optics
    mua: np.ndarray
    mus: np.ndarray
    c: float                       # cm/ps
    dt: float                      # ps
    n_steps: int
    groups: List[List[Beam]]       # one list of beams per generalized source q_i
    detectors: List[Detector]
    snap_steps: List[int] = field(default_factory=list)

    @property
    def updates(self) -> int:
        """cell-ordinate-step updates of one forward solve over all groups."""
        g = self.grid
        return g.nx * g.ny * g.M * self.n_steps * len(self.groups)


def face_point(face: str, s: float, L: float):
    """Point at fraction s along a face of the square [0, L]^2 and the inward
    normal direction angle: bottom (y=0) -> pi/2, right (x=L) -> pi,
    top (y=L) -> 3pi/2, left (x=0) -> 0."""
    if face == "bottom":
        return s * L, 0.0, np.pi / 2
    if face == "right":
        return L, s * L, np.pi
    if face == "top":
        return (1 - s) * L, L, 3 * np.pi / 2
    if face == "left":
        return 0.0, (1 - s) * L, 0.0
    raise ValueError(face)


FACES = ("bottom", "right", "top", "left")


def perimeter_detectors(L: float, per_face: int, sigma_d: float = 0.2):
    """per_face detectors on each face at fractions (k + 1/2) / per_face."""
    dets = []
    for face in FACES:
        for k in range(per_face):
            x, y, _ = face_point(face, (k + 0.5) / per_face, L)
            dets.append(Detector(x, y, sigma_d))
    return dets


def perimeter_beams(L: float, per_face: int, **kw):
    beams = []
    for face in FACES:
        for k in range(per_face):
            x, y, th = face_point(face, (k + 0.5) / per_face, L)
            beams.append(Beam(x, y, th, **kw))
    return beams


def _coords(grid: Grid):
    x = grid.xmin + grid.dx * np.arange(grid.nx)
    y = grid.ymin + grid.dy * np.arange(grid.ny)
    return np.meshgrid(x, y)          # arrays [j, i]


def _disks(grid: Grid, rng, n, r_rng, a_rng, b_rng, margin, a, b):
    X, Y = _coords(grid)
    a, b = a.copy(), b.copy()
    L = grid.xmax - grid.xmin
    for _ in range(n):
        r = rng.uniform(*r_rng)
        cx = rng.uniform(grid.xmin + margin + r, grid.xmin + L - margin - r)
        cy = rng.uniform(grid.ymin + margin + r, grid.ymin + L - margin - r)
        inside = (X - cx) ** 2 + (Y - cy) ** 2 <= r * r
        a[inside] = rng.uniform(*a_rng)
        b[inside] = rng.uniform(*b_rng)
    return a, b


def workload_small(n_steps: int = 200, dt: float = 0.05) -> Workload:
    """64 x 64 points on [0,2]^2, M = 16, homogeneous mua = 0.1, mus = 100,
    g = 0.9, n = 1.4; one beam at the bottom-face centre (Gaussian in time,
    sigma_t = 10 ps, t_s = 30 ps); 8 detectors (2 per face)."""
    grid = Grid(64, 64, 0.0, 2.0, 0.0, 2.0, 16)
    opt = Optics(g=0.9)
    a = np.full((64, 64), 0.1)
    b = np.full((64, 64), 100.0)
    beam = Beam(1.0, 0.0, np.pi / 2)
    return Workload("small64_M16", grid, opt, a, b, C0_CM_PER_PS / opt.n_in, dt,
                    n_steps, [[beam]], perimeter_detectors(2.0, 2),
                    snap_steps=[n_steps - 1])


def workload_tomo256(n_steps: int = 2000, dt: float = 0.04, n_sources: int = 16,
                     seed: int = BASE_SEED + 2) -> Workload:
    """256 x 256 points on [0,4]^2, M = 32; background mua = 0.1, mus = 100,
    g = 0.9, n = 1.4, plus 3 seeded disks (r 0.2-0.5 cm, mua 0.2-0.5,
    mus 50-150) at least 0.5 cm from the boundary; 16 beams (4 per face) fired
    one at a time (16 groups); 32 detectors (8 per face)."""
    rng = np.random.default_rng(seed)
    grid = Grid(256, 256, 0.0, 4.0, 0.0, 4.0, 32)
    opt = Optics(g=0.9)
    a = np.full((256, 256), 0.1)
    b = np.full((256, 256), 100.0)
    a, b = _disks(grid, rng, 3, (0.2, 0.5), (0.2, 0.5), (50, 150), 0.5, a, b)
    beams = perimeter_beams(4.0, 4)[:n_sources]
    return Workload("tomo256_M32", grid, opt, a, b, C0_CM_PER_PS / opt.n_in, dt,
                    n_steps, [[bm] for bm in beams], perimeter_detectors(4.0, 8),
                    snap_steps=[n_steps - 1])


def smooth_field(grid: Grid, rng, sigma_cm: float, lo: float, hi: float):
    """Seeded white noise, Gaussian-filtered (sigma in cm, periodic FFT
    filter), affinely rescaled to [lo, hi]."""
    noise = rng.standard_normal((grid.ny, grid.nx))
    ky = np.fft.fftfreq(grid.ny, d=grid.dy)
    kx = np.fft.fftfreq(grid.nx, d=grid.dx)
    K2 = ky[:, None] ** 2 + kx[None, :] ** 2
    sm = np.real(np.fft.ifft2(np.fft.fft2(noise) * np.exp(-2 * np.pi ** 2 * sigma_cm ** 2 * K2)))
    sm = (sm - sm.min()) / (sm.max() - sm.min())
    return lo + (hi - lo) * sm


def workload_precision512(n_steps: int = 3000, dt: float = 0.02,
                          seed: int = BASE_SEED + 3) -> Workload:
    """512 x 512 points on [0,4]^2, M = 64, g = 0.8; smooth random
    mua in [0.05, 0.3] and mus in [50, 150]; one beam; 32 detectors."""
    rng = np.random.default_rng(seed)
    grid = Grid(512, 512, 0.0, 4.0, 0.0, 4.0, 64)
    opt = Optics(g=0.8)
    a = smooth_field(grid, rng, 0.3, 0.05, 0.3)
    b = smooth_field(grid, rng, 0.3, 50.0, 150.0)
    beam = Beam(2.0, 0.0, np.pi / 2)
    return Workload("precision512_M64", grid, opt, a, b, C0_CM_PER_PS / opt.n_in,
                    dt, n_steps, [[beam]], perimeter_detectors(4.0, 8),
                    snap_steps=[n_steps - 1])


def workload_mss256(n_steps: int = 3000, dt: float = 0.04, target: bool = False,
                    seed: int = BASE_SEED + 4) -> Workload:
    """Config-2 grid with 16 beams in 4 Multiple-Staggered-Source groups (one
    beam per face per group) with seeded delays in [0, T/2].  target=False:
    homogeneous background (where the gradient is taken); target=True: the
    seeded inclusion medium that generates the data."""
    rng = np.random.default_rng(seed)
    grid = Grid(256, 256, 0.0, 4.0, 0.0, 4.0, 32)
    opt = Optics(g=0.9)
    a = np.full((256, 256), 0.1)
    b = np.full((256, 256), 100.0)
    inc = _disks(grid, rng, 3, (0.2, 0.5), (0.2, 0.5), (50, 150), 0.5, a, b)
    if target:
        a, b = inc[0], b
    T = n_steps * dt
    groups = []
    for gi in range(4):
        grp = []
        for face in FACES:
            x, y, th = face_point(face, (gi + 0.5) / 4, 4.0)
            grp.append(Beam(x, y, th, tau=float(rng.uniform(0, T / 2))))
        groups.append(grp)
    return Workload("mss256_M32", grid, opt, a, b, C0_CM_PER_PS / opt.n_in, dt,
                    n_steps, groups, perimeter_detectors(4.0, 8))


def neck_medium(grid: Grid, rng):
    """Elliptical neck-like cross-section: layered annuli (skin/fat/muscle-
    like), an airway disk (low absorption) and 1-2 vessel disks (high
    absorption); a low-scattering coupling layer outside the ellipse."""
    X, Y = _coords(grid)
    L = grid.xmax - grid.xmin
    cx, cy = grid.xmin + L / 2, grid.ymin + L / 2
    ax, ay = 0.42 * L, 0.35 * L
    rho = np.sqrt(((X - cx) / ax) ** 2 + ((Y - cy) / ay) ** 2)
    a = np.full(X.shape, 0.02)
    b = np.full(X.shape, 10.0)
    layers = [(1.0, rng.uniform(0.1, 0.3), rng.uniform(80, 120)),
              (0.93, rng.uniform(0.02, 0.08), rng.uniform(60, 100)),
              (0.8, rng.uniform(0.1, 0.3), rng.uniform(40, 90))]
    for r, av, bv in layers:
        a[rho <= r] = av
        b[rho <= r] = bv
    aw = (X - cx) ** 2 + (Y - (cy + 0.1 * ay)) ** 2 <= (0.12 * ay) ** 2
    a[aw], b[aw] = 0.02, 10.0
    for _ in range(int(rng.integers(1, 3))):
        vr = rng.uniform(0.04, 0.07) * L
        vx = cx + rng.uniform(-0.5, 0.5) * ax
        vy = cy + rng.uniform(-0.6, -0.2) * ay
        v = (X - vx) ** 2 + (Y - vy) ** 2 <= vr * vr
        a[v], b[v] = 1.0, 100.0
    return a, b


def workload_batched(n_solves: int = 48, n_steps: int = 1500, dt: float = 0.04,
                     seed: int = BASE_SEED + 5):
    """48 independent solves on grids drawn from {128, 192, 256, 384}^2 with
    dx = 4/255 cm, M = 32, each a neck-like medium with its own beam."""
    rng = np.random.default_rng(seed)
    h = 4.0 / 255
    out = []
    for s in range(n_solves):
        n = int(rng.choice([128, 192, 256, 384]))
        L = h * (n - 1)
        grid = Grid(n, n, 0.0, L, 0.0, L, 32)
        a, b = neck_medium(grid, rng)
        face = ("bottom", "right", "top", "left")[s % 4]
        x, y, th = face_point(face, float(rng.uniform(0.3, 0.7)), L)
        out.append(Workload(f"neck{n}_M32_{s}", grid, Optics(g=0.9), a, b,
                            C0_CM_PER_PS / 1.4, dt, n_steps, [[Beam(x, y, th)]],
                            perimeter_detectors(L, 8)))
    return out


def workload_custom(nx: int, ny: int, M: int, n_steps: int, dt: float,
                    L: float = 1.0, g: float = 0.9, mua: float = 0.1,
                    mus: float = 100.0, n_groups: int = 1, seed: int = BASE_SEED,
                    heterogeneous: bool = True, n_det_per_face: int = 2,
                    t_s: float = 3.0, sigma_t: float = 1.0) -> Workload:
    """Small seeded case for tests: [0, L] x [0, L*(ny-1)/(nx-1)] (equal
    spacing), optional seeded disk inclusions, n_groups single-beam groups."""
    rng = np.random.default_rng(seed)
    h = L / (nx - 1)
    grid = Grid(nx, ny, 0.0, L, 0.0, h * (ny - 1), M)
    a = np.full((ny, nx), float(mua))
    b = np.full((ny, nx), float(mus))
    if heterogeneous:
        X, Y = _coords(grid)
        for _ in range(2):
            r = rng.uniform(0.1, 0.2) * L
            cx, cy = rng.uniform(0.3, 0.7) * L, rng.uniform(0.3, 0.7) * grid.ymax
            m = (X - cx) ** 2 + (Y - cy) ** 2 <= r * r
            a[m] = mua * rng.uniform(2, 5)
            b[m] = mus * rng.uniform(0.5, 1.5)
    Ly = grid.ymax
    groups = []
    for k in range(n_groups):
        face = FACES[k % 4]
        s = rng.uniform(0.3, 0.7)
        if face == "bottom":
            bm = Beam(s * L, 0.0, np.pi / 2)
        elif face == "right":
            bm = Beam(L, s * Ly, np.pi)
        elif face == "top":
            bm = Beam(s * L, Ly, 3 * np.pi / 2)
        else:
            bm = Beam(0.0, s * Ly, 0.0)
        bm.sigma_x = 0.15 * L
        bm.t_s, bm.sigma_t = t_s, sigma_t
        groups.append([bm])
    dets = []
    for face in FACES:
        for k in range(n_det_per_face):
            s = (k + 0.5) / n_det_per_face
            if face == "bottom":
                dets.append(Detector(s * L, 0.0, 0.2 * L))
            elif face == "right":
                dets.append(Detector(L, s * Ly, 0.2 * L))
            elif face == "top":
                dets.append(Detector(s * L, Ly, 0.2 * L))
            else:
                dets.append(Detector(0.0, s * Ly, 0.2 * L))
    return Workload(f"custom{nx}x{ny}_M{M}", grid, Optics(g=g), a, b,
                    C0_CM_PER_PS / 1.4, dt, n_steps, groups, dets,
                    snap_steps=[n_steps - 1])


def add_relative_noise(curves: np.ndarray, level: float = 0.10, seed: int = BASE_SEED + 7) -> np.ndarray:
    """Synthetic measurement noise: every detector reading G becomes
    G (1 + level xi) with xi ~ N(0, 1) drawn from a seeded generator (the
    reading taken of the paper's "10% random noise")."""
    rng = np.random.default_rng(seed)
    return curves * (1.0 + level * rng.standard_normal(curves.shape))


def workload_inverse(mode: str = "mss", n: int = 64, n_steps: int = 2000, dt: float = 0.04,
                     target: bool = False, seed: int = BASE_SEED + 8) -> Workload:
    """Inverse-problem medium: n x n points at dx = 2/127 cm (n = 64: a 1 cm
    square, which the diffusing light crosses within the 80 ps window),
    M = 32, background mua = 0.1 (the lower bound of the reconstruction),
    mus = 100, g = 0.9; the target adds two seeded absorbing disks (mua
    0.3-0.6, r 0.15-0.3 * L/2 cm).  mode "ts": 16 single-beam sources, 4 per
    face; "mss": the same 16 beams as 4 staggered groups (one per face,
    delays in [0, T/2]); 32 detectors, 8 per face."""
    rng = np.random.default_rng(seed)
    h = 2.0 / 127
    L = h * (n - 1)
    grid = Grid(n, n, 0.0, L, 0.0, L, 32)
    a = np.full((n, n), 0.1)
    b = np.full((n, n), 100.0)
    X, Y = _coords(grid)
    disks = []
    for _ in range(2):
        r = rng.uniform(0.15, 0.3) * L / 2
        cx, cy = rng.uniform(0.3 * L, 0.7 * L), rng.uniform(0.3 * L, 0.7 * L)
        disks.append((cx, cy, r, rng.uniform(0.3, 0.6)))
    if target:
        for cx, cy, r, av in disks:
            a[(X - cx) ** 2 + (Y - cy) ** 2 <= r * r] = av
    T = n_steps * dt
    beams = []
    for gi in range(4):
        grp = []
        for face in FACES:
            x, y, th = face_point(face, (gi + 0.5) / 4, L)
            grp.append(Beam(x, y, th, tau=float(rng.uniform(0, T / 2)) if mode == "mss" else 0.0))
        beams.append(grp)
    groups = beams if mode == "mss" else [[bm] for grp in beams for bm in grp]
    return Workload(f"inverse{n}_{mode}", grid, Optics(g=0.9), a, b, C0_CM_PER_PS / 1.4, dt, n_steps,
                    groups, perimeter_detectors(L, 8))
