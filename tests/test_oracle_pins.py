"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  None of them re-types the oracle's
formula: they compare it with closed forms, textbook identities, values the
paper prints, invariants, or convergence rates."""
import numpy as np
import pytest
from scipy import integrate
from scipy.special import i0

from conftest import golden
from oracle import fcgram
from oracle import rte
from rte_inputs import Beam, Grid, Optics, Workload, workload_custom, workload_small


# ---------------------------------------------------------------- quadrature
def test_kphi_closed_form_and_paper_value():
    """Sec. 5: k_Phi = int exp(-cos^2) = 2 pi e^{-1/2} I_0(1/2) (Bessel
    generating function); the paper prints 4.052876133898710."""
    closed = 2 * np.pi * np.exp(-0.5) * i0(0.5)
    assert abs(closed - golden("k_phi")) < 1e-14


def test_trapezoid_ordinates_spectral_convergence():
    """Sec. 4.1, eq. (RTETrapz): trapezoid rule on theta_m = 2 pi m / M is
    spectrally accurate for the periodic integrand of Sec. 5."""
    exact = golden("k_phi")
    errs = []
    for M in (4, 8, 12, 16, 24):
        theta, w, xi, eta = rte.ordinates(M)
        assert np.allclose(xi ** 2 + eta ** 2, 1)
        errs.append(abs(w * np.exp(-np.cos(theta) ** 2).sum() - exact))
    # aliasing error ~ 4 pi e^{-1/2} I_{M/2}(1/2): 2.6e-6, 2.9e-9, ~1e-15
    assert errs[2] < 1e-5 and errs[3] < 1e-8 and errs[4] < 1e-13
    assert all(errs[k + 1] < errs[k] * 1e-2 for k in range(3))


# ---------------------------------------------------------------- window
def test_window_function_values():
    """eq. (sourcelabwind): w(0) = 1, w = 0 for |v| >= 1, even, in (0, 1)
    inside; w(1/2) = exp(2 e^{-2} / (-1/2)) = exp(-4 e^{-2})."""
    v = np.array([0.0, 0.5, -0.5, 1.0, -1.0, 1.5])
    w = rte.window(v)
    assert w[0] == 1.0 and w[3] == 0 and w[4] == 0 and w[5] == 0
    assert abs(w[1] - np.exp(-4 * np.exp(-2))) < 1e-15 and w[1] == w[2]
    x = np.linspace(-0.999, 0.999, 2001)
    wx = rte.window(x)
    assert np.all(wx > 0) and np.all(wx <= 1)
    # C-infinity at the support edge: w(0.99) = exp(-200 e^{-1/0.99}) ~ 1e-32
    assert rte.window(np.array([0.99]))[0] < 1e-30


# ---------------------------------------------------------------- phase
@pytest.mark.parametrize("g", [0.0, 0.5, 0.8, 0.9])
@pytest.mark.parametrize("exponent", [1.5, 1.0])
def test_phase_normalisation_symmetry(g, exponent):
    """Sec. 4.1: the numerical integral of the phase function is one, so every
    row of P~ (and, P~ being symmetric circulant, every column) sums to 1."""
    for M in (8, 16, 32):
        P = rte.phase_matrix(M, g, exponent)
        assert np.allclose(P.sum(axis=1), 1, atol=1e-14)
        assert np.allclose(P, P.T, atol=1e-15)
        assert np.allclose(P, np.roll(np.roll(P, 1, 0), 1, 1), atol=1e-15)
        if g == 0:
            assert np.allclose(P, 1.0 / M)


def test_phase_2d_hg_is_poisson_kernel():
    """With the 2D exponent 1 the HG function is the Poisson kernel: its
    integral is exactly 1 and its k-th Fourier cosine coefficient is g^k, so
    the eigenvalues of P~ are g^|k| (up to aliasing ~ g^M)."""
    g = 0.8
    val, _ = integrate.quad(lambda t: rte.henyey_greenstein(np.cos(t), g, 1.0), 0, 2 * np.pi,
                            epsabs=1e-13, limit=200)
    assert abs(val - 1) < 1e-11
    M = 64
    ev = np.sort(np.linalg.eigvalsh(rte.phase_matrix(M, g, 1.0)))[::-1]
    # trapezoid sampling aliases mode k onto k + jM: eigenvalue
    # sum_j g^|k + jM| / sum_j g^|jM|
    alias = lambda k: sum(g ** abs(k + j * M) for j in range(-6, 7))
    lam = np.array([alias(k) / alias(0) for k in range(M)])
    assert np.allclose(ev, np.sort(lam)[::-1], atol=1e-13)
    assert abs(lam[1] - g) < 1e-5


def test_phase_mean_cosine_sign():
    """Forward scattering for g > 0: the mean cosine sum_m' P~ cos(theta_m -
    theta_m') is positive and increases with g (a sign or index slip in the
    angle difference flips it)."""
    M = 32
    th, _, _, _ = rte.ordinates(M)
    cosd = np.cos(th[:, None] - th[None, :])
    mc = [(rte.phase_matrix(M, g) * cosd).sum(axis=1)[0] for g in (0.0, 0.3, 0.6, 0.9)]
    assert abs(mc[0]) < 1e-14 and 0 < mc[1] < mc[2] < mc[3] < 1


# ---------------------------------------------------------------- Fresnel
def test_fresnel_textbook_forms():
    """Fresnel reflectance in the independent sine/tangent forms:
    r_s = -sin(i - t)/sin(i + t), r_p = tan(i - t)/tan(i + t); normal
    incidence ((n1 - n2)/(n1 + n2))^2; total reflection past asin(1/1.4)."""
    n1, n2 = golden("n_tissue"), 1.0
    assert abs(rte.fresnel(1.0, n1, n2) - ((n1 - n2) / (n1 + n2)) ** 2) < 1e-15
    crit = np.arcsin(n2 / n1)
    for ang in np.linspace(0.05, crit - 0.02, 12):
        t = np.arcsin(n1 / n2 * np.sin(ang))
        rs = -np.sin(ang - t) / np.sin(ang + t)
        rp = np.tan(ang - t) / np.tan(ang + t)
        assert abs(rte.fresnel(np.cos(ang), n1, n2) - 0.5 * (rs ** 2 + rp ** 2)) < 1e-13
    for ang in np.linspace(crit + 1e-6, np.pi / 2, 5):
        assert rte.fresnel(np.cos(ang), n1, n2) == 1.0
    brewster = np.arctan(n2 / n1)
    t = np.arcsin(n1 / n2 * np.sin(brewster))
    rs = -np.sin(brewster - t) / np.sin(brewster + t)
    assert abs(rte.fresnel(np.cos(brewster), n1, n2) - 0.5 * rs ** 2) < 1e-14


# ---------------------------------------------------------------- reflection maps
def test_reflection_maps_are_specular():
    """eq. (RTE): theta_r = 2 theta_nu - theta + pi keeps the tangential and
    flips the normal component of the direction, on every face."""
    M = 16
    grid = Grid(9, 7, 0.0, 1.0, 0.0, 0.75, M)
    bt = rte.boundary_tables(grid, Optics())
    th, _, xi, eta = rte.ordinates(M)
    normals = {0: (-1, 0), 1: (1, 0), 2: (0, -1), 3: (0, 1)}
    for n in range(len(bt.nodes_j)):
        j, i = bt.nodes_j[n], bt.nodes_i[n]
        for m in np.nonzero(bt.active[n])[0]:
            r = bt.refl[n, m]
            faces = [F for F, ok in ((0, i == 0), (1, i == grid.nx - 1),
                                     (2, j == 0), (3, j == grid.ny - 1)) if ok]
            # the governing face: m incoming, r its specular image
            good = []
            for F in faces:
                nu = normals[F]
                dn_m = xi[m] * nu[0] + eta[m] * nu[1]
                dn_r = xi[r] * nu[0] + eta[r] * nu[1]
                dt_m = -xi[m] * nu[1] + eta[m] * nu[0]
                dt_r = -xi[r] * nu[1] + eta[r] * nu[0]
                good.append(dn_m < 0 and abs(dn_m + dn_r) < 1e-12 and abs(dt_m - dt_r) < 1e-12)
            assert any(good)
    # every incoming ordinate at a non-corner node is active, outgoing never
    for n in range(len(bt.nodes_j)):
        j, i = bt.nodes_j[n], bt.nodes_i[n]
        if i == 0 and 0 < j < grid.ny - 1:
            assert np.array_equal(bt.active[n], xi > 1e-12)


# ---------------------------------------------------------------- FC derivative
def test_fc_paper_example_sizes_and_accuracy():
    """Sec. 4.3 worked example: g = 12 + x^2 - e^{x/3} on [0, 6] with 61 points,
    d = 5, C = 25, E = 4, N_p = 90 = 2 x 3 x 3 x 5; its FC derivative matches
    2x - e^{x/3}/3."""
    n = golden("fc_example_points")
    Q, A = fcgram.load_tables()
    assert Q.shape[0] == golden("fc_d") and A.shape[0] == golden("fc_example_C")
    Np = fcgram.continued_length(n)
    assert Np == golden("fc_example_Np") and Np - n - A.shape[0] == golden("fc_example_E")
    x = np.linspace(0, 6, n)
    g = 12 + x ** 2 - np.exp(x / 3)
    dg = fcgram.fc_derivative(g, x[1] - x[0])
    assert np.abs(dg - (2 * x - np.exp(x / 3) / 3)).max() < 1e-6


def test_fc_high_order_convergence():
    """Sec. 4.3: high-order accuracy under refinement (observed order > 3.5)
    for non-periodic smooth functions."""
    for f, df in ((lambda x: 12 + x ** 2 - np.exp(x / 3), lambda x: 2 * x - np.exp(x / 3) / 3),
                  (lambda x: np.sin(1.3 * x + 0.4), lambda x: 1.3 * np.cos(1.3 * x + 0.4))):
        errs = []
        for n in (41, 81, 161):
            x = np.linspace(0, 6, n)
            errs.append(np.abs(fcgram.fc_derivative(f(x), x[1] - x[0]) - df(x)).max())
        orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        assert np.all(orders > 3.5), orders


def test_fc_reproduces_low_degree_polynomials():
    """The continuation is built from the Gram basis of degree < d = 5, so
    polynomials of degree <= 4 are differentiated to table accuracy."""
    for n in (64, 128):
        x = np.linspace(0, 1, n)
        for p in range(5):
            d = fcgram.fc_derivative(x ** p, x[1] - x[0])
            exact = p * x ** (p - 1) if p else 0 * x
            assert np.abs(d - exact).max() < 1e-9 * max(1, np.abs(exact).max())


def test_fc_tables_structure():
    """Gram basis: orthonormal columns, column j a polynomial of degree j
    (orthogonal to lower monomials); continuations decay to ~0 at the end of
    the C continuation points; the continued vector of smooth data is smooth
    (fast decay of its Fourier coefficients)."""
    Q, A = fcgram.load_tables()
    d = Q.shape[0]
    assert np.allclose(Q.T @ Q, np.eye(d), atol=1e-14)
    z = np.arange(d, dtype=float)
    V = np.vander(z, d, increasing=True)
    assert np.allclose(np.tril(Q.T @ V, -1), 0, atol=1e-9)   # P_j _|_ z^k, k < j
    assert np.abs(A[-3:]).max() < 1e-6 * max(1, np.abs(A).max())
    x = np.linspace(0, 1, 100)
    gc = fcgram.fc_extend(np.exp(x) * np.cos(2 * x))
    spec = np.abs(np.fft.rfft(gc))
    freq = np.arange(len(spec)) / len(gc)          # cycles per grid spacing
    # the continuation is band-limited to K / period = 18 / 60 = 0.3 cycles
    assert spec[freq > 0.35].max() < 1e-9 * spec.max()


def test_fc_dense_operator_equals_fft_path():
    """The dense operator D (column j = derivative of e_j) reproduces the FFT
    path on arbitrary data (linearity of eqs. RTEFCSum-RTEFCSumder)."""
    rng = np.random.default_rng(1)
    for n in (20, 64, 131):
        h = 0.1
        D = fcgram.derivative_matrix(n, h)
        g = rng.standard_normal((3, n))
        scale = (np.abs(g) @ np.abs(D).T).max()     # rounding scale of the sum
        assert np.abs(g @ D.T - fcgram.fc_derivative(g, h)).max() < 1e-12 * scale


def test_fc_filter_only_touches_top_modes():
    """eq. (FFilter) with alpha = 2, beta = 55: sigma(k) = exp(-2 |2k/N_p|^110)
    is 1 to 1e-5 below 90% of Nyquist and e^{-2} at Nyquist."""
    Np, h = 90, 1.0
    mult = fcgram.spectral_multiplier(Np, h)
    k = np.fft.fftfreq(Np, 1 / Np)
    ideal = 2j * np.pi * k / (Np * h)
    low = np.abs(2 * k / Np) < 0.9
    assert np.allclose(mult[low], ideal[low], rtol=1e-5, atol=0)
    assert mult[Np // 2] == 0                       # Nyquist mode dropped (even N_p)
    top = Np // 2 - 1
    assert abs(abs(mult[top]) / abs(ideal[top]) - np.exp(-2 * (2 * top / Np) ** 110)) < 1e-12


# ---------------------------------------------------------------- AB4 + mirror box
def test_ab4_uniform_isotropic_mirror_box_decays_by_principal_root():
    """Perfect mirror (f = 1), no source, uniform isotropic field: streaming
    and scattering vanish, L(u) = -a u, and AB4 (eq. RTEAB4) started on its
    own principal root rho reproduces u^k = rho^k u^0; rho ~ exp(-c a dt)
    to fifth order in z = -c a dt."""
    wl = workload_custom(20, 16, 8, 0, 0.05, mua=0.7, mus=30.0, heterogeneous=False)
    wl.mua = np.full_like(wl.mua, 0.7)
    S = rte.Solver(wl, fresnel_override=1.0)
    z = -wl.c * 0.7 * wl.dt
    chi = [golden("ab4_chi1"), golden("ab4_chi2"), golden("ab4_chi3")]
    chi0 = 1 - sum(chi)       # consistency of AB4: the coefficients sum to 1
    assert abs(chi0 - 55 / 24) < 1e-15
    # rho^4 = rho^3 + z (chi0 rho^3 + chi1 rho^2 + chi2 rho + chi3)
    roots = np.roots([1, -(1 + z * chi0), -z * chi[0], -z * chi[1], -z * chi[2]])
    rho = roots[np.argmin(np.abs(roots - 1))].real
    assert abs(rho - np.exp(z)) < 2 * abs(z) ** 5
    u0 = np.ones((8, wl.grid.ny, wl.grid.nx))
    hist = [-0.7 * u0 * rho ** (-k) for k in (1, 2, 3)]
    out = S.forward([], 40, inflow=lambda t: 0.0, init=(u0, hist, 0.0))
    assert np.allclose(out["u"], rho ** 40, rtol=1e-9, atol=0)


# ---------------------------------------------------------------- manufactured solution
def _mms(n, M, dt, T, a=0.35, b=20.0):
    """Sec. 5, eqs. (RTEdisp)/(RTEmansol): u = exp(-(x-t)^2-(y-t)^2-cos^2 theta)
    on [0,3]^2, g = 0, c = 1, with its volumetric source and Dirichlet inflow."""
    kphi = golden("k_phi")
    g = Grid(n, n, 0.0, 3.0, 0.0, 3.0, M)
    wl = Workload("mms", g, Optics(g=0.0), np.full((n, n), a), np.full((n, n), b), 1.0, dt, 0, [[]], [])
    S = rte.Solver(wl, fresnel_override=0.0)
    th = S.theta[:, None, None]
    X, Y = S.X[None, None, :], S.Y[None, :, None]

    def uex(t):
        return np.exp(-(X - t) ** 2 - (Y - t) ** 2 - np.cos(th) ** 2)

    def q(t):
        Xs, Ys = X - t, Y - t
        return (uex(t) * (2 * Xs + 2 * Ys - 2 * np.cos(th) * Xs - 2 * np.sin(th) * Ys + a + b)
                - b * kphi / (2 * np.pi) * np.exp(-Xs ** 2 - Ys ** 2))

    hist = [S.L(uex(-k * dt)) + q(-k * dt) for k in (1, 2, 3)]
    out = S.forward([], int(round(T / dt)), volume_source=q, init=(uex(0.0), hist, 0.0),
                    inflow=lambda t: uex(t)[:, S.bt.nodes_j, S.bt.nodes_i].T)
    t = out["t_end"]
    exact = kphi * np.exp(-(S.X[None, :] - t) ** 2 - (S.Y[:, None] - t) ** 2)
    return S.fluence(out["u"]), exact


def test_mms_spatial_high_order():
    """Sec. 5: high-order convergence in dx (observed order > 4)."""
    errs = [np.abs(np.subtract(*_mms(n, 16, 0.001, 0.1))).max() for n in (25, 37, 49)]
    ratio = np.array([1.5, 49 / 37 * 36 / 48 * 48 / 36])
    orders = np.log(np.array(errs[:-1]) / np.array(errs[1:])) / np.log([36 / 24, 48 / 36])
    assert errs[-1] < 2e-6 and np.all(orders > 4), (errs, orders, ratio)


def test_mms_angular_spectral():
    """Sec. 5: spectral convergence in theta (error drops > 10x per +2
    ordinates)."""
    errs = [np.abs(np.subtract(*_mms(40, M, 0.002, 0.1))).max() for M in (6, 8, 10)]
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10


def test_mms_time_fourth_order():
    """Sec. 4.2/5: AB4 is fourth order in dt (self-convergence on a fixed
    grid against a fine-dt run)."""
    ref, _ = _mms(33, 12, 0.0005, 0.32)
    errs = [np.abs(_mms(33, 12, dt, 0.32)[0] - ref).max() for dt in (0.008, 0.004)]
    order = np.log2(errs[0] / errs[1])
    assert 3.7 < order < 4.3, (errs, order)


# ---------------------------------------------------------------- symmetry, linearity
def test_mirror_symmetric_setup_gives_symmetric_fluence():
    """A homogeneous square with one beam at the bottom-face centre pointing
    along +y is symmetric under x -> L - x: so is Phi (to rounding)."""
    wl = workload_small(n_steps=60, dt=0.05)
    S = rte.Solver(wl)
    out = S.forward(wl.groups[0], wl.n_steps, wl.detectors, snap_steps=[59])
    phi = out["fluence"][59]
    assert phi.max() > 1e-3
    assert np.abs(phi - phi[:, ::-1]).max() < 1e-12 * phi.max()
    c = out["curves"]
    assert np.allclose(c[0], c[1], rtol=1e-10, atol=1e-300)   # the two bottom detectors


def test_mss_curves_superpose_delayed_single_beams():
    """eqs. (RTEsources)/(RTE) are linear in q: the detector curves of a
    two-beam staggered group equal the sum of the single-beam curves."""
    wl = workload_custom(24, 20, 8, 120, 0.04, n_groups=2, t_s=1.0, sigma_t=0.4)
    b1, b2 = wl.groups[0][0], wl.groups[1][0]
    b2.tau = 0.8
    S = rte.Solver(wl)
    c1 = S.forward([b1], 120, wl.detectors)["curves"]
    c2 = S.forward([b2], 120, wl.detectors)["curves"]
    c12 = S.forward([b1, b2], 120, wl.detectors)["curves"]
    assert np.abs(c12).max() > 0
    assert np.abs(c12 - (c1 + c2)).max() < 1e-9 * np.abs(c12).max()


# ---------------------------------------------------------------- detectors
def test_detector_operator_on_uniform_field():
    """eq. (OpMed) on u = 1: G_j = [int w(|s|/sigma_d) ds] x
    [int_{-pi/2}^{pi/2} (1 - f(cos p)) cos p dp] for a detector in the middle
    of a face (scipy quad for both factors).  The angular integrand has a
    square-root kink at the critical angle, so the trapezoid error falls like
    M^{-3/2}: 1.5% at M = 64, 0.2% at M = 256."""
    from rte_inputs import Detector
    ang, _ = integrate.quad(lambda p: (1 - rte.fresnel(np.cos(p))) * np.cos(p), -np.pi / 2, np.pi / 2,
                            points=[-np.arcsin(1 / 1.4), np.arcsin(1 / 1.4)], epsabs=1e-13)
    sp, _ = integrate.quad(lambda v: rte.window(np.array([v]))[0], -1, 1, epsabs=1e-13)
    det = [Detector(1.0, 0.0, 0.3), Detector(2.0, 0.9, 0.25)]
    rel = []
    for M in (64, 256):
        n = 161
        grid = Grid(n, n, 0.0, 2.0, 0.0, 2.0, M)
        wl = Workload("u1", grid, Optics(), np.zeros((n, n)), np.zeros((n, n)), 0.02, 0.01, 0, [[]], [])
        S = rte.Solver(wl)
        ex = S.exitance(np.ones((M, n, n)))
        G = S.readout([e[:, None] for e in ex], det)[:, 0]
        rel.append([abs(G[k] / (d.sigma_d * sp * ang) - 1) for k, d in enumerate(det)])
    rel = np.array(rel)
    assert np.all(rel[0] < 0.025) and np.all(rel[1] < 0.003)
    assert np.all(np.log(rel[0] / rel[1]) / np.log(4) > 1.3)


# ---------------------------------------------------------------- photon balance
def test_photon_balance_with_fresnel_boundary():
    """Integrating eq. (RTE) over theta and Omega (scattering conserves):
    d/dt int Phi / c = -(net boundary flux) - int a Phi.  Checked over a run
    with a beam and Fresnel reflection, to discretisation accuracy."""
    errs = []
    for n, dt, steps in ((32, 0.04, 500), (48, 0.03, 667)):
        wl = workload_custom(n, n, 8, steps, dt, L=1.0, mua=0.5, mus=10.0, heterogeneous=False,
                             t_s=6.0, sigma_t=2.0)
        S = rte.Solver(wl)
        out = S.forward(wl.groups[0], steps, keep_states=True)
        N, absn, flux = (np.array(v) for v in zip(*(S.photon_balance(u) for u in out["states"])))
        rate = -flux - absn
        lhs = N[-1] - N[0]
        rhs = np.trapezoid(rate, dx=dt)
        errs.append(abs(lhs - rhs) / np.abs(N).max())
    assert max(errs) < 2e-3, errs


def test_photon_balance_terms_closed_forms():
    """The balance terms on fields with closed-form integrals: a uniform
    isotropic u = 1 holds int Phi / c = 2 pi |Omega| / c and absorbs
    2 pi int a; its net boundary flux is zero (every face sees as much
    outflow as inflow).  The field u_m(x, y) = max(0, cos theta_m) x / L
    (photons moving in +x, growing along x) has no flux through the left
    face (x = 0) and none through the bottom and top faces (the angular sum
    of sin theta over the forward half-circle vanishes); through the right
    face it carries L int_{-pi/2}^{pi/2} cos^2 = L pi / 2, which the
    trapezoid rule on 64 ordinates gives exactly (cos^2 sums to M/2 over
    the circle, half of it on the forward side)."""
    n, M, L = 33, 64, 2.0
    wl = workload_custom(n, n, M, 1, 0.01, L=L, mua=0.3, mus=10.0, heterogeneous=False)
    S = rte.Solver(wl)
    N, absn, flux = S.photon_balance(np.ones((M, n, n)))
    assert abs(N - 2 * np.pi * L * L / wl.c) < 1e-12 * N
    assert abs(absn - 2 * np.pi * 0.3 * L * L) < 1e-12 * absn
    assert abs(flux) < 1e-12
    theta, _, _, _ = rte.ordinates(M)
    u = np.maximum(0.0, np.cos(theta))[:, None, None] * (S.X / L)[None, None, :] * np.ones((1, n, 1))
    _, _, flux = S.photon_balance(u)
    assert abs(flux - L * np.pi / 2) < 1e-12


# ---------------------------------------------------------------- subdomains
def test_subdomain_segments_layout():
    """Sec. 4.4: owned ranges tile the line, two fringe points on interior
    sides only, neighbouring segments overlap by four points."""
    from oracle.fcgram import subdomain_segments
    segs = subdomain_segments(101, 4)
    assert segs[0][0] == 0 and segs[-1][1] == 101
    for (lo, hi, slo, shi), (lo2, hi2, slo2, shi2) in zip(segs, segs[1:]):
        assert hi == lo2 and shi - slo2 == 4
    assert segs[0][2] == 0 and segs[-1][3] == 101
    assert all(slo == lo - 2 for lo, hi, slo, shi in segs[1:]) and all(shi == hi + 2 for lo, hi, slo, shi in segs[:-1])


def test_subdomain_derivative_one_part_is_global():
    from oracle.fcgram import fc_derivative, fc_derivative_parts
    x = np.linspace(0.0, 2.0, 70)
    g = np.stack([np.sin(3 * x), np.exp(-x) * x ** 2])
    assert np.array_equal(fc_derivative_parts(g, x[1] - x[0], parts=1), fc_derivative(g, x[1] - x[0]))


def test_subdomain_derivative_reproduces_low_degree_polynomials():
    """Each segment's FC reproduces polynomials of degree < d = 5 (their
    continuation is exact to table accuracy), so the decomposed derivative of
    a global quartic is exact at every point, fringes or not."""
    from oracle.fcgram import fc_derivative_parts
    x = np.linspace(-1.0, 1.5, 97)
    h = x[1] - x[0]
    p = 0.3 - 1.2 * x + 0.7 * x ** 2 + 0.25 * x ** 3 - 0.4 * x ** 4
    dp = -1.2 + 1.4 * x + 0.75 * x ** 2 - 1.6 * x ** 3
    for parts in (2, 3, 5):
        d = fc_derivative_parts(p, h, parts=parts)
        assert np.abs(d - dp).max() < 1e-8 * np.abs(dp).max(), parts


def test_subdomain_derivative_converges():
    """Smooth function, 4 parts: the error falls at high order under
    refinement (each segment keeps the FC accuracy of Sec. 4.3)."""
    from oracle.fcgram import fc_derivative_parts
    errs = []
    ns = (81, 161, 321)
    for n in ns:
        x = np.linspace(0.0, 3.0, n)
        f = np.exp(np.sin(2 * x)) + np.cos(5 * x)
        df = 2 * np.cos(2 * x) * np.exp(np.sin(2 * x)) - 5 * np.sin(5 * x)
        d = fc_derivative_parts(f, x[1] - x[0], parts=4)
        errs.append(np.abs(d - df).max())
    orders = [np.log(errs[k] / errs[k + 1]) / np.log((ns[k + 1] - 1) / (ns[k] - 1)) for k in range(2)]
    assert min(orders) > 3.5, (errs, orders)


# ------------------------------------------------------------ brute force
def _dense_scheme(wl):
    """The step of the scheme on a small grid as dense matrices of the
    (nx ny M)-vector u[m, j, i], assembled from the definitions: L of eq.
    (RTEAB4L) as Kronecker products (scattering P~ over ordinates at each
    node, D_x along i, D_y along j, the local a, b), and the boundary
    condition of eq. (RTE) as a matrix found by geometry (incoming where
    theta.nu < 0, the governing face at a corner the larger |theta.nu|, the
    y-face on a tie, the reflected ordinate the one whose direction is the
    mirror image), with the rows it imposes (Gamma_-, where the source
    enters)."""
    from oracle.fcgram import fc_derivative
    g, M = wl.grid, wl.grid.M
    nn = g.nx * g.ny
    th = 2 * np.pi * np.arange(M) / M
    cx, sy = np.cos(th), np.sin(th)
    Dx = fc_derivative(np.eye(g.nx), g.dx, axis=0)          # column k: derivative of e_k
    Dy = fc_derivative(np.eye(g.ny), g.dy, axis=0)
    P = rte.phase_matrix(M, wl.optics.g, wl.optics.hg_exponent)
    a_rep = np.tile(np.asarray(wl.mua, dtype=float).ravel(), M)
    b_rep = np.tile(np.asarray(wl.mus, dtype=float).ravel(), M)
    Lmat = (b_rep[:, None] * np.kron(P, np.eye(nn)) - np.diag(a_rep + b_rep)
            - np.kron(np.diag(cx), np.kron(np.eye(g.ny), Dx))
            - np.kron(np.diag(sy), np.kron(Dy, np.eye(g.nx))))
    normals = {0: (-1.0, 0.0), 1: (1.0, 0.0), 2: (0.0, -1.0), 3: (0.0, 1.0)}
    Bmat = np.eye(M * nn)
    imposed = np.zeros(M * nn, dtype=bool)
    for j in range(g.ny):
        for i in range(g.nx):
            faces = [F for F, on in ((0, i == 0), (1, i == g.nx - 1), (2, j == 0), (3, j == g.ny - 1)) if on]
            for m in range(M):
                dots = {F: normals[F][0] * cx[m] + normals[F][1] * sy[m] for F in faces}
                inc = [F for F in faces if dots[F] < -1e-12]
                if not inc:
                    continue
                F = inc[0] if len(inc) == 1 else max(inc, key=lambda f: (abs(dots[f]) - (1e-12 if f < 2 else 0.0)))
                # mirror the normal component of theta_m across face F
                nu = normals[F]
                rx, ry = cx[m] - 2 * dots[F] * nu[0], sy[m] - 2 * dots[F] * nu[1]
                mr = int(np.argmin(np.hypot(cx - rx, sy - ry)))
                row = m * nn + j * g.nx + i
                imposed[row] = True
                Bmat[row, :] = 0.0
                Bmat[row, mr * nn + j * g.nx + i] = rte.fresnel(abs(dots[F]), wl.optics.n_in, wl.optics.n_out)
    return Lmat, Bmat, imposed


def _dense_readout(wl):
    """eq. (OpMed) as a [detector x state] matrix: per face, trapezoid weight
    along the face x detector window x sum over outgoing ordinates of
    w (1 - f) theta.nu."""
    g, M = wl.grid, wl.grid.M
    nn = g.nx * g.ny
    th = 2 * np.pi * np.arange(M) / M
    X = g.xmin + g.dx * np.arange(g.nx)
    Y = g.ymin + g.dy * np.arange(g.ny)
    R = np.zeros((len(wl.detectors), M * nn))
    faces = (((-1.0, 0.0), [(j, 0) for j in range(g.ny)], g.dy), ((1.0, 0.0), [(j, g.nx - 1) for j in range(g.ny)], g.dy),
             ((0.0, -1.0), [(0, i) for i in range(g.nx)], g.dx), ((0.0, 1.0), [(g.ny - 1, i) for i in range(g.nx)], g.dx))
    for nu, nodes, h in faces:
        cosv = nu[0] * np.cos(th) + nu[1] * np.sin(th)
        out = cosv > 1e-12
        wm = np.where(out, (2 * np.pi / M) * (1 - rte.fresnel(np.abs(cosv), wl.optics.n_in, wl.optics.n_out)) * cosv, 0)
        for k, (j, i) in enumerate(nodes):
            trap = h * (0.5 if k in (0, len(nodes) - 1) else 1.0)
            for d, det in enumerate(wl.detectors):
                wd = trap * rte.window(np.hypot(X[i] - det.x, Y[j] - det.y) / det.sigma_d)
                R[d, np.arange(M) * nn + j * g.nx + i] += wd * wm
    return R


def _dense_march(wl, S, Lmat, Bmat, imposed):
    g, M = wl.grid, wl.grid.M
    ab4 = np.array([55.0, -59.0, 37.0, -9.0]) / 24.0
    bj, bi = S.bt.nodes_j, S.bt.nodes_i
    u = np.zeros(M * g.nx * g.ny)
    hist = [np.zeros_like(u) for _ in range(3)]
    cdt = wl.c * wl.dt
    states = [u]
    for s in range(wl.n_steps):
        Lk = Lmat @ u
        pre = u + cdt * (ab4[0] * Lk + ab4[1] * hist[0] + ab4[2] * hist[1] + ab4[3] * hist[2])
        q = np.zeros((M, g.ny, g.nx))
        q[:, bj, bi] = S.beam_inflow(wl.groups[0], (4 + s) * wl.dt).T
        u = Bmat @ pre + np.where(imposed, q.ravel(), 0.0)
        hist = [Lk, hist[0], hist[1]]
        states.append(u)
    return states


def test_brute_force_dense_march_on_tiny_grid():
    """The whole scheme on a 12 x 10 grid with M = 8 as one dense linear map
    of the state (`_dense_scheme`), marched with AB4 (eq. RTEAB4) from zero
    start levels: the oracle's per-line march must agree to rounding at every
    step, and its detector curves with the dense readout of eq. (OpMed)."""
    wl = workload_custom(12, 10, 8, 30, 0.04, L=11 / 66, mus=20.0, n_groups=1, t_s=0.5, sigma_t=0.3)
    S = rte.Solver(wl)
    out = S.forward(wl.groups[0], wl.n_steps, wl.detectors, keep_states=True)
    states = _dense_march(wl, S, *_dense_scheme(wl))
    worst = max(np.abs(states[s + 1] - out["states"][s].ravel()).max() / np.abs(out["states"][s]).max()
                for s in range(wl.n_steps))
    R = _dense_readout(wl)
    curves = np.stack([R @ u for u in states[1:]], axis=1)
    ec = np.abs(curves - out["curves"]).max() / np.abs(out["curves"]).max()
    print(f"dense march vs oracle: state {worst:.1e}, curves {ec:.1e}")
    assert np.abs(out["states"][-1]).max() > 0
    assert worst < 1e-11 and ec < 1e-9, (worst, ec)


def test_brute_force_discrete_gradient_on_tiny_grid():
    """The exact gradient of the discrete objective by forward-mode
    sensitivities of the dense march: for every node n, the perturbation of
    a at n changes L by -u at that node, and dJ/da_n = sum_s dt r^s . R du^s.
    The oracle's reverse sweep (discrete_adjoint_gradient) must give the same
    gradient to rounding."""
    wl = workload_custom(12, 10, 8, 24, 0.04, L=11 / 66, mus=20.0, n_groups=1, t_s=0.5, sigma_t=0.3)
    tgt = workload_custom(12, 10, 8, 24, 0.04, L=11 / 66, mus=20.0, n_groups=1, t_s=0.5, sigma_t=0.3, seed=5)
    meas = rte.Solver(tgt).forward(tgt.groups[0], 24, tgt.detectors)["curves"] * 0.8
    S = rte.Solver(wl)
    Lmat, Bmat, imposed = _dense_scheme(wl)
    states = _dense_march(wl, S, Lmat, Bmat, imposed)
    R = _dense_readout(wl)
    resid = np.stack([R @ u for u in states[1:]], axis=1) - meas
    g, M = wl.grid, wl.grid.M
    nn = g.nx * g.ny
    sel = np.tile(np.eye(nn), (M, 1))                       # row (m, node) -> column node
    ab4 = np.array([55.0, -59.0, 37.0, -9.0]) / 24.0
    cdt = wl.c * wl.dt
    dU = np.zeros((M * nn, nn))                             # column n: du for a perturbation at node n
    dH = [np.zeros_like(dU) for _ in range(3)]
    grad = np.zeros(nn)
    for s in range(wl.n_steps):
        dL = Lmat @ dU - states[s][:, None] * sel
        dU = Bmat @ (dU + cdt * (ab4[0] * dL + ab4[1] * dH[0] + ab4[2] * dH[1] + ab4[3] * dH[2]))
        dH = [dL, dH[0], dH[1]]
        grad += wl.dt * (resid[:, s] @ (R @ dU))
    _, ga, _ = S.discrete_adjoint_gradient(wl.groups[0], wl.n_steps, wl.detectors, meas)
    err = np.linalg.norm(ga.ravel() - grad) / np.linalg.norm(grad)
    print(f"reverse sweep vs dense forward-mode gradient: {err:.1e}")
    assert np.linalg.norm(grad) > 0
    assert err < 1e-9, err


# ---------------------------------------------------------------- beam sources
def _source_solver(n=129, M=16, L=4.0):
    """An oracle solver on [0, L]^2 whose only role is to evaluate the beam
    sources of eq. (RTEsources2) at its boundary nodes."""
    grid = Grid(n, n, 0.0, L, 0.0, L, M)
    wl = Workload("src", grid, Optics(), np.full((n, n), 0.1), np.full((n, n), 10.0), 0.02, 0.01, 0,
                  [[]], [])
    return rte.Solver(wl)


def _face_values(S, q, face, m):
    """q[node, m] along one face (nodes in the face's order) with the face's
    trapezoid weights and node coordinates."""
    jj, ii, wgt = S.bt.face_nodes[face]
    index = {(j, i): k for k, (j, i) in enumerate(zip(S.bt.nodes_j, S.bt.nodes_i))}
    rows = np.array([index[(j, i)] for j, i in zip(jj, ii)])
    return q[rows, m], wgt, S.X[ii], S.Y[jj]


def test_beam_spatial_footprint_is_gaussian_of_spread_sigma_x():
    """eq. (RTEsources2), spatial factor exp(-|x - x_k|^2 / (2 sigma_x^2)):
    along the face through a mid-face beam (direction on an ordinate, time at
    the temporal centre, so the other factors are 1) its integral is
    sigma_x sqrt(2 pi), its mean the beam position and its variance
    sigma_x^2 (the trapezoid rule is exact to rounding for a Gaussian this
    well resolved, and the tails beyond the face ends are below 1e-10)."""
    S = _source_solver()
    sig = 0.3
    bm = Beam(2.0, 0.0, np.pi / 2, sigma_x=sig, t_s=30.0, sigma_t=10.0, tau=5.0)
    q = S.beam_inflow([bm], 35.0)
    m_k = S.M // 4                                                  # theta_m = pi / 2
    v, wgt, xs, _ = _face_values(S, q, 2, m_k)
    mass = np.sum(wgt * v)
    assert abs(mass / (sig * np.sqrt(2 * np.pi)) - 1) < 1e-9
    mean = np.sum(wgt * xs * v) / mass
    var = np.sum(wgt * (xs - mean) ** 2 * v) / mass
    assert abs(mean - 2.0) < 1e-12
    assert abs(var / sig ** 2 - 1) < 1e-8
    # the other faces are at least 2 cm (6.7 sigma_x) away
    for F in (0, 1, 3):
        vf, _, _, _ = _face_values(S, q, F, m_k)
        assert np.max(np.abs(vf)) < 3e-10


@pytest.mark.parametrize("theta_k", [np.pi / 2, 0.0, 0.1, 2 * np.pi - 0.05])
def test_beam_angular_factor_integral_and_direction(theta_k):
    """eq. (RTEsources2), angular factor w(|theta - theta_k| / sigma_theta)
    with the departure taken on the circle: at the beam's own node, at its
    temporal centre, the trapezoid sum over the ordinates (Sec. 4.1) equals
    sigma_theta int_{-1}^{1} w(v) dv, and the circular mean of the factor
    points along theta_k.  Beams near theta = 0 have half their support on
    the far side of 2 pi; a distance that does not wrap loses it."""
    S = _source_solver(n=33, M=512)
    st = np.pi / 4
    bm = Beam(2.0, 0.0, theta_k, sigma_theta=st, t_s=30.0, sigma_t=10.0)
    q = S.beam_inflow([bm], 30.0)
    node = int(np.flatnonzero((S.bt.nodes_j == 0) & (S.bt.nodes_i == 16))[0])   # x = 2, y = 0
    ang = q[node]
    theta, w, _, _ = rte.ordinates(S.M)
    ref, _ = integrate.quad(lambda v: rte.window(np.array([v]))[0], -1.0, 1.0, epsabs=1e-14, limit=200)
    assert abs(w * ang.sum() / (st * ref) - 1) < 1e-9
    z = np.sum(w * ang * np.exp(1j * theta))
    assert abs(np.angle(z * np.exp(-1j * theta_k))) < 1e-9


def test_beam_temporal_profiles_centre_spread_and_delay():
    """T(t - tau) of eq. (RTEsources2): the Gaussian reaches 1 at
    t = tau + t_s and exp(-1/2) at tau + t_s +- sigma_t, with integral
    sigma_t sqrt(2 pi); the window profile of eq. (sourcelab) is 1 at the
    centre, w(1/2) = exp(-4 e^{-2}) at +- sigma_t / 2 and 0 from +- sigma_t
    on.  Evaluated through the source term at the beam's own node and
    direction, where q = amplitude T."""
    S = _source_solver(n=33, M=16)
    node = int(np.flatnonzero((S.bt.nodes_j == 0) & (S.bt.nodes_i == 16))[0])
    m_k = S.M // 4
    amp, ts, sg, tau = 2.5, 30.0, 10.0, 7.0
    gauss = Beam(2.0, 0.0, np.pi / 2, t_s=ts, sigma_t=sg, tau=tau, amplitude=amp)
    win = Beam(2.0, 0.0, np.pi / 2, t_s=ts, sigma_t=sg, tau=tau, profile=1, amplitude=amp)

    def T(bm, t):
        return S.beam_inflow([bm], t)[node, m_k] / amp

    c = tau + ts
    assert abs(T(gauss, c) - 1) < 1e-15
    for t in (c - sg, c + sg):
        assert abs(T(gauss, t) - np.exp(-0.5)) < 1e-15
    assert abs(T(gauss, ts) - 1) > 0.1                                # the delay matters
    tt = np.linspace(c - 12 * sg, c + 12 * sg, 4801)
    vals = np.array([T(gauss, t) for t in tt])
    assert abs(np.trapezoid(vals, tt) / (sg * np.sqrt(2 * np.pi)) - 1) < 1e-12
    assert T(win, c) == 1.0
    for t in (c - sg / 2, c + sg / 2):
        assert abs(T(win, t) - np.exp(-4 * np.exp(-2))) < 1e-15
    for t in (c - sg, c + sg, c + 1.5 * sg):
        assert T(win, t) == 0.0


def test_two_beams_on_one_face_superpose():
    """eq. (RTEsources): a generalized source is the sum of its beams.  Two
    beams on the bottom face with amplitudes A1, A2 and staggered delays
    give, along that face, the integral sigma_x sqrt(2 pi) (A1 T1 + A2 T2)
    and the first moment (A1 T1 x1 + A2 T2 x2) / (A1 T1 + A2 T2), with
    T1 = 1 at the first beam's centre and T2 = exp(-(tau1 - tau2)^2 /
    (2 sigma_t^2)) there."""
    S = _source_solver()
    sig, ts, sg = 0.2, 30.0, 10.0
    b1 = Beam(1.4, 0.0, np.pi / 2, sigma_x=sig, t_s=ts, sigma_t=sg, tau=0.0, amplitude=1.0)
    b2 = Beam(2.6, 0.0, np.pi / 2, sigma_x=sig, t_s=ts, sigma_t=sg, tau=6.0, amplitude=0.6)
    q = S.beam_inflow([b1, b2], ts)
    v, wgt, xs, _ = _face_values(S, q, 2, S.M // 4)
    w1, w2 = 1.0, 0.6 * np.exp(-36.0 / (2 * sg ** 2))
    mass = np.sum(wgt * v)
    assert abs(mass / (sig * np.sqrt(2 * np.pi) * (w1 + w2)) - 1) < 1e-9
    assert abs(np.sum(wgt * xs * v) / mass - (w1 * 1.4 + w2 * 2.6) / (w1 + w2)) < 1e-9
