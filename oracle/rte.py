"""FP64 FC-DOM forward march, detectors, objective, continuous adjoint and
gradient for the 2D time-domain RTE (Gaggioli & Bruno).  Test infrastructure
only (see oracle/__init__.py).

State layout here is the paper's: u[m, j, i] = u_m(x_i, y_j) (Sec. 4.1, 4.3).

Readings of points where the paper is silent or garbled (each is also listed
with the design notes):
  * AB4 coefficients: the printed chi_0 = 55/44 and the missing chi_3 are
    typos; the standard 55/24, -59/24, 37/24, -9/24 are used (Sec. 4.2).
  * Start-up: the first four time levels t^1..t^4 (t^k = (k-1) dt) are zero,
    with zero history; step s (0-based) produces level k = s + 5 at time
    t = (s + 4) dt, and the boundary condition is imposed at that time.
  * FC period b = N_p dx (the period of N_p samples), not (N_p - 1) dx; the
    Nyquist mode's derivative is zero (eq. RTEFCSum).
  * Henyey-Greenstein exponent as printed (3/2) by default, 1 selectable;
    the numerical normalisation of Sec. 4.1 is applied in both cases.
  * Fresnel coefficient: unpolarised reflectance (r_s^2 + r_p^2)/2 from n_in
    to n_out, 1 beyond the critical angle, a function of |theta . nu|.
  * Reflection on the square: theta_r = 2 theta_nu - theta + pi gives
    m -> M/2 - m on the x-faces and m -> -m on the y-faces (M even).
  * Corners: boundary values are read from the pre-BC field; an ordinate that
    enters through both faces of a corner follows the face with the larger
    |theta . nu| (the y-face on a tie); ordinates with theta . nu = 0 get no
    boundary condition.
  * Sources: q(x, theta, t) = sum over the group's beams of eq. (RTEsources2),
    evaluated at every boundary node for every incoming ordinate; the angular
    departure is the periodic distance |theta - theta_k| in [0, pi].
  * Detectors: trapezoid rule along each face (half weight at the two face
    ends, each corner counted once per face), ordinates with theta . nu > 0.
  * Objective: rectangle rule in time over the recorded levels.
  * Adjoint: lambda vanishes at t^K .. t^{K+3}; the backward AB4 march
    produces t^{K-1} down to t^5; with mu_m = lambda_{m + M/2} it is the
    forward march with the residual injected on the incoming ordinates of mu.
  * Gradient cell weight: trapezoid area of the grid node (the integral of the
    pyramid perturbation of Sec. 3.6), times dtheta dt per level.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fcgram

AB4 = (55.0 / 24.0, -59.0 / 24.0, 37.0 / 24.0, -9.0 / 24.0)
TIE_TOL = 1e-12


# --------------------------------------------------------------------------
# Sec. 2 and Sec. 4.1: ordinates, window, phase function, Fresnel coefficient
# --------------------------------------------------------------------------

def ordinates(M: int):
    """eq. (RTETrapz): theta_m = 2 pi (m-1)/M (here 0-based m), w_m = 2 pi/M,
    xi_m = cos theta_m, eta_m = sin theta_m."""
    theta = 2.0 * np.pi * np.arange(M) / M
    return theta, 2.0 * np.pi / M, np.cos(theta), np.sin(theta)


def window(v):
    """eq. (sourcelabwind): 1 at 0, exp(2 e^{-1/|v|} / (|v| - 1)) on 0<|v|<1,
    0 for |v| >= 1."""
    v = np.abs(np.asarray(v, dtype=np.float64))
    out = np.zeros_like(v)
    out[v == 0] = 1.0
    inner = (v > 0) & (v < 1)
    vi = v[inner]
    out[inner] = np.exp(2.0 * np.exp(-1.0 / vi) / (vi - 1.0))
    return out


def henyey_greenstein(cos_angle, g: float, exponent: float = 1.5):
    """eq. (Henyey-Greenstein): (1/2pi)(1-g^2)/(1+g^2-2g cos)^exponent."""
    return (1.0 / (2.0 * np.pi)) * (1.0 - g * g) / (1.0 + g * g - 2.0 * g * cos_angle) ** exponent


def phase_matrix(M: int, g: float, exponent: float = 1.5) -> np.ndarray:
    """P~[m, m'] = w_{m'} p_{m,m'}, with p normalised so that its trapezoid
    integral over theta' is one for every m (Sec. 4.1)."""
    theta, w, _, _ = ordinates(M)
    p = henyey_greenstein(np.cos(theta[:, None] - theta[None, :]), g, exponent)
    p = p / (w * p.sum(axis=1, keepdims=True))
    return w * p


def fresnel(cos_i, n_in: float = 1.4, n_out: float = 1.0):
    """Unpolarised Fresnel reflectance for light inside (n_in) hitting the
    boundary at incidence cosine cos_i; total reflection beyond the critical
    angle (reading of Sec. 2's unspecified f)."""
    cos_i = np.abs(np.asarray(cos_i, dtype=np.float64))
    sin_i = np.sqrt(np.maximum(0.0, 1.0 - cos_i ** 2))
    sin_t = n_in / n_out * sin_i
    out = np.ones_like(cos_i)
    ok = sin_t < 1.0
    cos_t = np.sqrt(1.0 - sin_t[ok] ** 2)
    ci = cos_i[ok]
    rs = (n_in * ci - n_out * cos_t) / (n_in * ci + n_out * cos_t)
    rp = (n_out * ci - n_in * cos_t) / (n_out * ci + n_in * cos_t)
    out[ok] = 0.5 * (rs ** 2 + rp ** 2)
    return out


def temporal_profile(t, beam):
    """T(t - tau): profile 0 Gaussian exp(-(t-tau-t_s)^2/(2 sigma_t^2)),
    profile 1 the window w(|t - tau - t_s| / sigma_t) of eq. (sourcelab)."""
    tt = t - beam.tau - beam.t_s
    if beam.profile == 0:
        return np.exp(-tt * tt / (2.0 * beam.sigma_t ** 2))
    return float(window(np.abs(tt) / beam.sigma_t))


def angular_distance(a, b):
    d = np.mod(np.abs(a - b), 2.0 * np.pi)
    return np.minimum(d, 2.0 * np.pi - d)


# --------------------------------------------------------------------------
# Boundary geometry on the square (eq. RTE third line; eq. OpMed)
# --------------------------------------------------------------------------

# faces: (name, outward normal nu, angle theta_nu)
FACES = (("left", (-1.0, 0.0)), ("right", (1.0, 0.0)),
         ("bottom", (0.0, -1.0)), ("top", (0.0, 1.0)))


@dataclass
class BoundaryTables:
    nodes_j: np.ndarray      # boundary node rows
    nodes_i: np.ndarray      # boundary node columns
    active: np.ndarray       # [node, m] True where a BC is imposed
    refl: np.ndarray         # [node, m] reflected ordinate m_r
    fcoef: np.ndarray        # [node, m] Fresnel f(|theta.nu|) of the governing face
    face_nodes: list         # per face: (j array, i array, trapezoid weights)
    face_cos: np.ndarray     # [face, m] theta_m . nu_face


def boundary_tables(grid, optics) -> BoundaryTables:
    M = grid.M
    if M % 2:
        raise ValueError("M must be even for the reflection maps")
    _, _, xi, eta = ordinates(M)
    nx, ny = grid.nx, grid.ny
    face_cos = np.array([nu[0] * xi + nu[1] * eta for _, nu in FACES])
    m = np.arange(M)
    refl_face = np.array([(M // 2 - m) % M, (M // 2 - m) % M, (-m) % M, (-m) % M])
    fres_face = fresnel(face_cos, optics.n_in, optics.n_out)

    def on_faces(j, i):
        f = []
        if i == 0:
            f.append(0)
        if i == nx - 1:
            f.append(1)
        if j == 0:
            f.append(2)
        if j == ny - 1:
            f.append(3)
        return f

    nodes = [(j, i) for j in range(ny) for i in range(nx)
             if i in (0, nx - 1) or j in (0, ny - 1)]
    nj = np.array([p[0] for p in nodes])
    ni = np.array([p[1] for p in nodes])
    active = np.zeros((len(nodes), M), dtype=bool)
    refl = np.zeros((len(nodes), M), dtype=np.int64)
    fco = np.zeros((len(nodes), M))
    for n, (j, i) in enumerate(nodes):
        faces = on_faces(j, i)
        for mm in range(M):
            incoming = [F for F in faces if face_cos[F, mm] < -TIE_TOL]
            if not incoming:
                continue
            if len(incoming) == 1:
                F = incoming[0]
            else:
                Fx, Fy = incoming  # x-face first (0/1), then y-face (2/3)
                cx, cy = abs(face_cos[Fx, mm]), abs(face_cos[Fy, mm])
                F = Fx if cx > cy + TIE_TOL else Fy
            active[n, mm] = True
            refl[n, mm] = refl_face[F, mm]
            fco[n, mm] = fres_face[F, mm]
    # Trapezoid nodes per face, ordered along the face.
    face_nodes = []
    for F in range(4):
        if F in (0, 1):
            jj = np.arange(ny)
            ii = np.full(ny, 0 if F == 0 else nx - 1)
            wgt = np.full(ny, grid.dy)
        else:
            ii = np.arange(nx)
            jj = np.full(nx, 0 if F == 2 else ny - 1)
            wgt = np.full(nx, grid.dx)
        wgt[0] *= 0.5
        wgt[-1] *= 0.5
        face_nodes.append((jj, ii, wgt))
    return BoundaryTables(nj, ni, active, refl, fco, face_nodes, face_cos)


# --------------------------------------------------------------------------
# The solver: Algorithm 1, on one domain or decomposed (fc_parts)
# --------------------------------------------------------------------------

class Solver:
    """fc_parts = (parts along x, parts along y): the subdomain decomposition
    of Sec. 4.4 / Algorithm 1 (FC on each part's segment with two fringe
    points, fringes exchanged every step); (1, 1) is one domain."""

    def __init__(self, wl, tables=None, fresnel_override=None, fc_parts=(1, 1)):
        self.wl = wl
        self.fc_parts = tuple(fc_parts)
        g = wl.grid
        self.grid = g
        self.M = g.M
        self.theta, self.w, self.xi, self.eta = ordinates(g.M)
        self.P = phase_matrix(g.M, wl.optics.g, wl.optics.hg_exponent)
        self.a = np.asarray(wl.mua, dtype=np.float64)
        self.b = np.asarray(wl.mus, dtype=np.float64)
        self.c = wl.c
        self.dt = wl.dt
        self.tables = tables if tables is not None else fcgram.load_tables()
        self.bt = boundary_tables(g, wl.optics)
        if fresnel_override is not None:
            self.bt.fcoef[:] = fresnel_override
        X = g.xmin + g.dx * np.arange(g.nx)
        Y = g.ymin + g.dy * np.arange(g.ny)
        self.X, self.Y = X, Y
        self.bx = X[self.bt.nodes_i]
        self.by = Y[self.bt.nodes_j]

    # --- spatial operator ------------------------------------------------
    def dx(self, u):
        """Algorithm 1, x-lines: FC derivative along i for every (m, j)."""
        return fcgram.fc_derivative_parts(u, self.grid.dx, axis=2, parts=self.fc_parts[0], tables=self.tables)

    def dy(self, u):
        """Algorithm 1, y-lines: FC derivative along j for every (m, i)."""
        return fcgram.fc_derivative_parts(u, self.grid.dy, axis=1, parts=self.fc_parts[1], tables=self.tables)

    def scatter(self, u):
        """sum_{m'} w_{m'} p_{m,m'} u_{m'} at every node."""
        return np.tensordot(self.P, u, axes=(1, 0))

    def L(self, u):
        """eq. (RTEAB4L): b sum w p u - (b + a) u - theta_m . grad u."""
        return (self.b * self.scatter(u) - (self.a + self.b) * u
                - self.xi[:, None, None] * self.dx(u)
                - self.eta[:, None, None] * self.dy(u))

    # --- boundary data ---------------------------------------------------
    def beam_inflow(self, beams, t):
        """q(x, theta_m, t) at every boundary node: sum of eq. (RTEsources2)."""
        q = np.zeros((len(self.bx), self.M))
        for bm in beams:
            sp = np.exp(-((self.bx - bm.x) ** 2 + (self.by - bm.y) ** 2) / (2 * bm.sigma_x ** 2))
            ang = window(angular_distance(self.theta, bm.theta) / bm.sigma_theta)
            q += bm.amplitude * temporal_profile(t, bm) * sp[:, None] * ang[None, :]
        return q

    def apply_bc(self, u_new, q):
        """Third line of eq. (RTE) on Gamma_-: u = f u(theta_r) + q, with the
        reflected values read from the field before any node is updated."""
        bt = self.bt
        pre = u_new[:, bt.nodes_j, bt.nodes_i].T          # [node, m]
        reflected = np.take_along_axis(pre, bt.refl, axis=1)
        val = np.where(bt.active, bt.fcoef * reflected + q, pre)
        u_new[:, bt.nodes_j, bt.nodes_i] = val.T

    def exitance(self, u):
        """Per face node: sum over theta.nu > 0 of w (1 - f) (theta.nu) u_m,
        the integrand of eq. (OpMed) before the detector window."""
        out = []
        wl = self.wl
        for F, (jj, ii, _) in enumerate(self.bt.face_nodes):
            cosv = self.bt.face_cos[F]
            wt = np.where(cosv > TIE_TOL,
                          self.w * (1 - fresnel(cosv, wl.optics.n_in, wl.optics.n_out)) * cosv, 0.0)
            out.append(wt @ u[:, jj, ii])
        return out

    def detector_weights(self, detectors):
        """[det] -> per face: trapezoid weight times w(|x - x_j| / sigma_d)."""
        W = []
        for F, (jj, ii, wgt) in enumerate(self.bt.face_nodes):
            xs, ys = self.X[ii], self.Y[jj]
            Wf = np.array([wgt * window(np.hypot(xs - d.x, ys - d.y) / d.sigma_d)
                           for d in detectors])
            W.append(Wf)
        return W

    def fluence(self, u):
        """eq. (photondensity) with the trapezoid rule: sum_m w u_m."""
        return self.w * u.sum(axis=0)

    def photon_balance(self, u):
        """Terms of the photon balance that integrating eq. (RTE) over theta
        and Omega gives (the scattering term integrates to zero by the
        normalisation of Sec. 4.1): photons in the domain int Phi / c, the
        absorption rate int a Phi, and the net outward flux through the
        boundary int_{dOmega} int (theta . nu) u dtheta, with the trapezoid
        rule in angle, over the nodes (node areas) and along each face.  The
        time derivative of the first equals minus the sum of the other two;
        the inflow of the sources enters the net flux with a negative sign."""
        area = self.node_area()
        phi = self.fluence(u)
        photons = float(np.sum(area * phi)) / self.c
        absorption = float(np.sum(area * self.a * phi))
        flux = 0.0
        for F, (jj, ii, wg) in enumerate(self.bt.face_nodes):
            flux += float(np.sum(wg * ((self.w * self.bt.face_cos[F]) @ u[:, jj, ii])))
        return photons, absorption, flux

    # --- forward march ---------------------------------------------------
    def forward(self, beams, n_steps, detectors=None, snap_steps=(),
                keep_states=False, inflow=None, volume_source=None, init=None,
                t_first=None):
        """Algorithm 1 with AB4 (eq. RTEAB4).  Returns a dict with the
        detector curves [det, step] (if detectors), exitance rings, fluence
        snapshots and optionally every post-BC state (for the adjoint).

        inflow(t) / volume_source(t) / init replace the beam data, add a
        volumetric source to L, or start from given levels (test hooks)."""
        M, g = self.M, self.grid
        if init is None:
            u = np.zeros((M, g.ny, g.nx))
            hist = [np.zeros_like(u) for _ in range(3)]       # L^{k-1}, L^{k-2}, L^{k-3}
            t0 = 3.0 * self.dt
        else:
            u, hist, t0 = init
            u = u.copy()
            hist = [h.copy() for h in hist]
        ex_hist = [[] for _ in range(4)]
        snaps = {}
        states = []
        for s in range(n_steps):
            t_cur = t0 + s * self.dt
            Lk = self.L(u)
            if volume_source is not None:
                Lk = Lk + volume_source(t_cur)
            incr = AB4[0] * Lk + AB4[1] * hist[0] + AB4[2] * hist[1] + AB4[3] * hist[2]
            u_new = u + self.c * self.dt * incr
            t_new = t_cur + self.dt
            q = inflow(t_new) if inflow is not None else self.beam_inflow(beams, t_new)
            self.apply_bc(u_new, q)
            hist = [Lk, hist[0], hist[1]]
            u = u_new
            for F, e in enumerate(self.exitance(u)):
                ex_hist[F].append(e)
            if s in snap_steps:
                snaps[s] = self.fluence(u)
            if keep_states:
                states.append(u.copy())
        out = {"u": u, "hist": hist, "t_end": t0 + n_steps * self.dt,
               "exitance": [np.array(e).T for e in ex_hist],    # [face][node, step]
               "fluence": snaps}
        if detectors is not None:
            out["curves"] = self.readout(out["exitance"], detectors)
        if keep_states:
            out["states"] = states
        return out

    def readout(self, exitance, detectors):
        """eq. (OpMed): G_j(t) = sum_faces sum_nodes weight * w_j * exitance."""
        W = self.detector_weights(detectors)
        return sum(W[F] @ exitance[F] for F in range(4))       # [det, step]

    # --- objective and adjoint --------------------------------------------
    def objective(self, curves, measured):
        """eq. (FObj) for one generalized source: 1/2 sum_j int (G_j - G~_j)^2 dt."""
        r = curves - measured
        return 0.5 * float(np.sum(r * r)) * self.dt

    def node_area(self):
        g = self.grid
        wx = np.full(g.nx, g.dx)
        wy = np.full(g.ny, g.dy)
        wx[[0, -1]] *= 0.5
        wy[[0, -1]] *= 0.5
        return wy[:, None] * wx[None, :]

    # --- exact discrete adjoint (the transpose of the discrete march) --------
    def _dense_derivatives(self):
        """Dense x and y FC operators (D g = derivative of g) of this solver's
        (possibly decomposed) derivative, built by applying it to the identity."""
        if not hasattr(self, "_Dx"):
            g = self.grid
            self._Dx = fcgram.fc_derivative_parts(np.eye(g.nx), g.dx, axis=-1, parts=self.fc_parts[0],
                                                  tables=self.tables).T
            self._Dy = fcgram.fc_derivative_parts(np.eye(g.ny), g.dy, axis=-1, parts=self.fc_parts[1],
                                                  tables=self.tables).T
        return self._Dx, self._Dy

    def L_transpose(self, v):
        """Transpose of the linear map u -> L(u) of eq. (RTEAB4L) on v[m, j, i]:
        b P^T v - (a + b) v - xi_m D_x^T v - eta_m D_y^T v."""
        Dx, Dy = self._dense_derivatives()
        dxT = np.tensordot(v, Dx, axes=([2], [0]))                  # sum_k v[m, j, k] D_x[k, i]
        dyT = np.einsum("kj,mki->mji", Dy, v)                       # sum_k D_y[k, j] v[m, k, i]
        return (self.b * np.tensordot(self.P.T, v, axes=(1, 0)) - (self.a + self.b) * v
                - self.xi[:, None, None] * dxT - self.eta[:, None, None] * dyT)

    def bc_transpose(self, ubar):
        """Transpose of the linear part of apply_bc (the source term does not
        depend on the field): an active (node, m) takes f times the pre-BC
        value of ordinate refl(m), every other entry keeps its own value."""
        bt = self.bt
        out = ubar.copy()
        ob = ubar[:, bt.nodes_j, bt.nodes_i].T                      # [node, m]
        pre_bar = np.where(bt.active, 0.0, ob)
        contrib = np.where(bt.active, bt.fcoef * ob, 0.0)
        np.add.at(pre_bar, (np.arange(ob.shape[0])[:, None], bt.refl), contrib)
        out[:, bt.nodes_j, bt.nodes_i] = pre_bar.T
        return out

    def _exit_weights(self):
        wl = self.wl
        return [np.where(cosv > TIE_TOL, self.w * (1 - fresnel(cosv, wl.optics.n_in, wl.optics.n_out)) * cosv, 0.0)
                for cosv in self.bt.face_cos]

    def readout_transpose(self, rs, W, wts):
        """Transpose of u -> dt-weighted curves of one recorded level
        (exitance of eq. OpMed, then the detector sums) applied to the
        residuals rs[det]."""
        ub = np.zeros((self.M, self.grid.ny, self.grid.nx))
        for F, (jj, ii, _) in enumerate(self.bt.face_nodes):
            e_bar = (W[F].T @ rs) * self.dt                          # [node]
            np.add.at(ub, (slice(None), jj, ii), wts[F][:, None] * e_bar[None, :])
        return ub

    def discrete_adjoint_gradient(self, beams, n_steps, detectors, measured):
        """Exact gradient of the discrete objective (eq. FObj with the
        rectangle rule over the recorded levels) with respect to the nodal
        values of a and b: the reverse sweep of the discrete march (AB4,
        boundary condition, exitance, readout), with the transposed FC
        operators.  Returns (J, dJ/da [ny, nx], dJ/db [ny, nx])."""
        fwd = self.forward(beams, n_steps, detectors, keep_states=True)
        r = fwd["curves"] - measured                                 # [det, step]
        J = self.objective(fwd["curves"], measured)
        states = [np.zeros_like(fwd["states"][0])] + fwd["states"]  # u^0 .. u^N
        W = self.detector_weights(detectors)
        wts = self._exit_weights()
        cdt = self.c * self.dt
        ubar = self.readout_transpose(r[:, n_steps - 1], W, wts)     # adjoint of u^N
        Lbar = {}
        ga = np.zeros((self.grid.ny, self.grid.nx))
        gb = np.zeros_like(ga)
        for s in range(n_steps - 1, -1, -1):
            # step s: u^{s+1} = BC(u^s + c dt sum_i chi_i L^{s-i})
            utb = self.bc_transpose(ubar)
            for i in range(4):
                if s - i >= 0:
                    Lbar[s - i] = Lbar.get(s - i, 0.0) + cdt * AB4[i] * utb
            Lb = Lbar.pop(s)                                         # complete: steps s..s+3 are done
            u_s = states[s]
            ubar = utb + self.L_transpose(Lb)
            if s >= 1:
                ubar = ubar + self.readout_transpose(r[:, s - 1], W, wts)
            ga -= (Lb * u_s).sum(axis=0)
            gb += (Lb * (self.scatter(u_s) - u_s)).sum(axis=0)
        return J, ga, gb

    def tangent_linear_objective(self, beams, n_steps, detectors, measured, da, db):
        """Forward-mode derivative of the discrete objective in the direction
        (da, db) of nodal perturbations of a and b (the tangent-linear march;
        an independent check of the discrete adjoint)."""
        fwd = self.forward(beams, n_steps, detectors, keep_states=True)
        r = fwd["curves"] - measured
        states = [np.zeros_like(fwd["states"][0])] + fwd["states"]
        cdt = self.c * self.dt
        du = np.zeros_like(states[0])
        dh = [np.zeros_like(du) for _ in range(3)]
        zero_q = np.zeros((len(self.bx), self.M))
        dJ = 0.0
        for s in range(n_steps):
            u_s = states[s]
            dL = self.L(du) - da * u_s + db * (self.scatter(u_s) - u_s)
            du = du + cdt * (AB4[0] * dL + AB4[1] * dh[0] + AB4[2] * dh[1] + AB4[3] * dh[2])
            self.apply_bc(du, zero_q)
            dh = [dL, dh[0], dh[1]]
            dG = self.readout([e[:, None] for e in self.exitance(du)], detectors)[:, 0]
            dJ += float(np.sum(r[:, s] * dG)) * self.dt
        return dJ

    def adjoint_gradient(self, beams, n_steps, detectors, measured):
        """Forward solve, residual, backward adjoint march of eq.
        (AdjointProblem) and the gradient of eq. (FDwin22) per grid node.
        Returns (J, dJ/dmua [ny, nx], dJ/dmus [ny, nx], curves)."""
        M = self.M
        fwd = self.forward(beams, n_steps, detectors, keep_states=True)
        curves = fwd["curves"]
        resid = curves - measured                          # [det, step]
        J = self.objective(curves, measured)
        # rho(x, t) = sum_j r_j(t) w(|x - x_j| / sigma_d) at every boundary
        # node: the pointwise detector term of eq. (AdjointProblem).
        Wnode = np.array([window(np.hypot(self.bx - d.x, self.by - d.y) / d.sigma_d)
                          for d in detectors])             # [det, node]
        flip = (np.arange(M) + M // 2) % M                 # mu_m = lambda_{m + M/2}
        grad_a = np.zeros((self.grid.ny, self.grid.nx))
        grad_b = np.zeros_like(grad_a)
        one_minus_f = 1.0 - self.bt.fcoef                  # f of the governing face

        mu = np.zeros((M, self.grid.ny, self.grid.nx))
        hist = [np.zeros_like(mu) for _ in range(3)]
        area = self.node_area() * (2 * np.pi / M) * self.dt
        for sp in range(n_steps - 1):
            Lk = self.L(mu)
            incr = AB4[0] * Lk + AB4[1] * hist[0] + AB4[2] * hist[1] + AB4[3] * hist[2]
            mu_new = mu + self.c * self.dt * incr
            lvl = n_steps - 2 - sp                         # forward step index of this level
            rho = Wnode.T @ resid[:, lvl]
            self.apply_bc(mu_new, one_minus_f * rho[:, None])
            hist = [Lk, hist[0], hist[1]]
            mu = mu_new
            lam = mu[flip]                                 # lambda_m = mu_{m + M/2}
            u = fwd["states"][lvl]
            grad_a -= area * np.sum(lam * u, axis=0)
            grad_b -= area * np.sum(lam * (u - self.scatter(u)), axis=0)
        return J, grad_a, grad_b, curves
