"""FC-Gram continuation and the filtered Fourier-continuation derivative
(Sec. 4.3, eqs. RTEFCSum, FFilter, RTEFCSumder; the four-step continuation
procedure listed there).  Oracle side: test infrastructure only.

The paper cites its continuation tables (Albin & Bruno 2011, Amlani & Bruno
2016) without printing them.  The tables used here follow this recipe, stated
in full so that it can be checked:

* unit grid spacing; the d matching points sit at z = 0, 1, ..., d-1, with
  z = d-1 the boundary point of the line;
* Gram basis: the polynomials of degree < d orthonormal for the discrete inner
  product on the d matching points (Gram-Schmidt on monomials, in mpmath);
* each Gram polynomial P_j is continued to zero by the trigonometric
  polynomial of period PERIOD = 2(d + C) with modes |k| <= K that best matches,
  in least squares on n_os points per unit spacing, P_j on [0, d-1] and 0 on
  the interval [d + C, 2d + C - 1]; the continuation values are its samples at
  z = d, ..., d + C - 1.  The least-squares problem is solved by a QR
  factorisation in 50-digit arithmetic and rounded to FP64 at the end.

``python -m oracle.fcgram`` regenerates ``oracle/tables/fcgram_d5_C25.txt``
(needs mpmath, which only the development machine has); the runtime reads the
committed text file.
"""
from __future__ import annotations

import os

import numpy as np

TABLE_DIR = os.path.join(os.path.dirname(__file__), "tables")

# Recipe constants (see module docstring).
FC_D = 5          # matching points d_l = d_r = 5 (Sec. 4.3)
FC_C = 25         # continuation points, as in the paper's worked example
FC_NOS = 20       # oversampling per unit spacing in the least-squares fit
FC_K = 18         # trigonometric modes |k| <= K
FILTER_ALPHA = 2.0    # eq. (FFilter): alpha = 2
FILTER_BETA = 55.0    # eq. (FFilter): beta = 55


def _table_path(d: int, C: int) -> str:
    return os.path.join(TABLE_DIR, f"fcgram_d{d}_C{C}.txt")


def generate_tables(d: int = FC_D, C: int = FC_C, n_os: int = FC_NOS,
                    K: int = FC_K, dps: int = 50):
    """Build (Q, A): Q[i, j] = P_j(z_i) (d x d, orthonormal columns) and
    A[r, j] = continuation of P_j at z = d + r (C x d).  mpmath only."""
    import mpmath as mp

    mp.mp.dps = dps
    z = [mp.mpf(i) for i in range(d)]
    # Step 1 of the paper's procedure needs the Gram basis on the matching
    # points: Gram-Schmidt (twice, for orthogonality) on 1, z, z^2, ...
    cols = []
    for j in range(d):
        v = [zi ** j for zi in z]
        for _ in range(2):
            for c in cols:
                s = mp.fsum(v[i] * c[i] for i in range(d))
                v = [v[i] - s * c[i] for i in range(d)]
        nrm = mp.sqrt(mp.fsum(x * x for x in v))
        cols.append([x / nrm for x in v])

    def gram_poly(j, x):
        # The degree < d polynomial through (z_i, P_j(z_i)), Lagrange form.
        total = mp.mpf(0)
        for i in range(d):
            li = mp.mpf(1)
            for k in range(d):
                if k != i:
                    li *= (x - z[k]) / (z[i] - z[k])
            total += cols[j][i] * li
        return total

    period = 2 * (d + C)
    match_pts = [mp.mpf(i) / n_os for i in range((d - 1) * n_os + 1)]
    zero_pts = [d + C + mp.mpf(i) / n_os for i in range((d - 1) * n_os + 1)]
    pts = match_pts + zero_pts
    nb = 2 * K + 1

    def basis_row(x):
        row = [mp.mpf(1)]
        for k in range(1, K + 1):
            ang = 2 * mp.pi * k * x / period
            row += [mp.cos(ang), mp.sin(ang)]
        return row

    Amat = mp.matrix([basis_row(x) for x in pts])
    Qf, Rf = mp.qr(Amat)
    Acont = np.zeros((C, d))
    for j in range(d):
        rhs = mp.matrix([gram_poly(j, x) for x in match_pts] + [0] * len(zero_pts))
        y = Qf.T * rhs
        coef = [mp.mpf(0)] * nb
        for i in reversed(range(nb)):
            s = y[i] - mp.fsum(Rf[i, k] * coef[k] for k in range(i + 1, nb))
            coef[i] = s / Rf[i, i]
        for r in range(C):
            Acont[r, j] = float(mp.fdot(coef, basis_row(mp.mpf(d + r))))
    Q = np.array([[float(cols[j][i]) for j in range(d)] for i in range(d)])
    return Q, Acont


def write_tables(d: int = FC_D, C: int = FC_C) -> str:
    Q, A = generate_tables(d, C)
    path = _table_path(d, C)
    os.makedirs(TABLE_DIR, exist_ok=True)
    with open(path, "w") as fh:
        fh.write(f"# FC-Gram tables d={d} C={C} n_os={FC_NOS} K={FC_K} "
                 f"period=2(d+C); written by python -m oracle.fcgram\n")
        fh.write("# Q (d rows x d cols): Gram polynomials at z=0..d-1\n")
        for row in Q:
            fh.write(" ".join(repr(float(v)) for v in row) + "\n")
        fh.write("# A (C rows x d cols): continuation of P_j at z=d..d+C-1\n")
        for row in A:
            fh.write(" ".join(repr(float(v)) for v in row) + "\n")
    return path


def load_tables(d: int = FC_D, C: int = FC_C):
    """Read the committed (Q, A) tables."""
    rows = []
    with open(_table_path(d, C)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([float(v) for v in line.split()])
    arr = np.array(rows)
    return arr[:d], arr[d:d + C]


def smooth5(n: int) -> int:
    """Smallest integer >= n whose prime factors are all <= 5 (Sec. 4.3:
    E extra zeros make N_p a product of small primes)."""
    m = n
    while True:
        r = m
        for p in (2, 3, 5):
            while r % p == 0:
                r //= p
        if r == 1:
            return m
        m += 1


def continued_length(n: int, C: int = FC_C) -> int:
    """N_p = N_x + 1 + C + E for a line of n = N_x + 1 points."""
    return smooth5(n + C)


def fc_extend(g: np.ndarray, tables=None) -> np.ndarray:
    """Steps 1-4 of the continuation procedure along the LAST axis.

    g has shape (..., n).  Returns g_c with shape (..., N_p):
    g_c = [g ; g_l + g_r], where g_r continues the last d values to zero
    towards the right and g_l continues the first d values to zero towards the
    left (mirror image), each padded with E zeros to length C + E."""
    Q, A = tables if tables is not None else load_tables()
    d, C = Q.shape[0], A.shape[0]
    n = g.shape[-1]
    if n < 2 * d:
        raise ValueError("line shorter than 2d points")
    Np = continued_length(n, C)
    E = Np - n - C
    # Step 1: project the matching values onto the Gram basis.
    right_match = g[..., n - d:]                 # z = 0..d-1, boundary at z=d-1
    left_match = g[..., :d][..., ::-1]           # mirrored: g_1 sits at z = d-1
    coef_r = right_match @ Q                     # (Q^T g) for every line
    coef_l = left_match @ Q
    # Step 2: continuations to zero of each Gram polynomial.
    gt_r = coef_r @ A.T                          # values at distance 1..C past g_{N+1}
    gt_l = coef_l @ A.T                          # values at distance 1..C before g_1
    # Step 3: pad to length C + E.  g_r decays from the right end of g; g_l is
    # stored reversed so that it rises into g_1 across the periodic seam.
    shape = g.shape[:-1]
    g_r = np.concatenate([gt_r, np.zeros(shape + (E,))], axis=-1)
    g_l = np.concatenate([np.zeros(shape + (E,)), gt_l[..., ::-1]], axis=-1)
    # Step 4: the continued vector.
    return np.concatenate([g, g_l + g_r], axis=-1)


def spectral_multiplier(Np: int, h: float, alpha: float = FILTER_ALPHA,
                        beta: float = FILTER_BETA) -> np.ndarray:
    """(2 pi i k / b) exp(-alpha |2k/N_p|^(2 beta)) in numpy's FFT ordering,
    with period b = N_p h and the Nyquist mode (even N_p) set to zero."""
    k = np.fft.fftfreq(Np, d=1.0 / Np)
    period = Np * h
    filt = np.exp(-alpha * np.abs(2.0 * k / Np) ** (2.0 * beta))
    mult = 2j * np.pi * k / period * filt
    if Np % 2 == 0:
        mult[Np // 2] = 0.0
    return mult


def fc_derivative(g: np.ndarray, h: float, axis: int = -1, tables=None,
                  alpha: float = FILTER_ALPHA, beta: float = FILTER_BETA) -> np.ndarray:
    """d g / d x along ``axis`` by eq. (RTEFCSumder): continue, FFT, filter and
    multiply by 2 pi i k / b, inverse FFT, keep the first n values."""
    g = np.moveaxis(np.asarray(g, dtype=np.float64), axis, -1)
    n = g.shape[-1]
    gc = fc_extend(g, tables)
    Np = gc.shape[-1]
    a_k = np.fft.fft(gc, axis=-1)
    dg = np.fft.ifft(a_k * spectral_multiplier(Np, h, alpha, beta), axis=-1)
    return np.moveaxis(dg.real[..., :n], -1, axis)


FRINGE = 2   # fringe points added on each interior side of a subdomain (Sec. 4.4)


def subdomain_segments(n: int, parts: int):
    """The decomposition of Sec. 4.4 along one axis: the n points are split
    into `parts` contiguous owned ranges [k n / parts, (k + 1) n / parts)
    (the interior regions), and each owned range is extended by FRINGE
    points on every side that is not a physical end of the line (the
    overlapping subdomain).  Returns (lo, hi, seg_lo, seg_hi) per part."""
    out = []
    for k in range(parts):
        lo, hi = k * n // parts, (k + 1) * n // parts
        seg_lo = lo - FRINGE if k > 0 else lo
        seg_hi = hi + FRINGE if k < parts - 1 else hi
        out.append((lo, hi, seg_lo, seg_hi))
    return out


def fc_derivative_parts(g: np.ndarray, h: float, axis: int = -1, parts: int = 1, tables=None,
                        alpha: float = FILTER_ALPHA, beta: float = FILTER_BETA) -> np.ndarray:
    """The x- or y-derivative of the decomposed scheme of Algorithm 1: every
    subdomain continues and differentiates its own segment (eq. RTEFCSumder
    on that segment alone), and after the fringe exchange each point holds
    the value its own subdomain computed, so a point's derivative is the
    segment derivative of the part that owns it.  parts = 1 is the global
    derivative."""
    if parts <= 1:
        return fc_derivative(g, h, axis=axis, tables=tables, alpha=alpha, beta=beta)
    g = np.moveaxis(np.asarray(g, dtype=np.float64), axis, -1)
    out = np.empty_like(g)
    for lo, hi, slo, shi in subdomain_segments(g.shape[-1], parts):
        d = fc_derivative(g[..., slo:shi], h, axis=-1, tables=tables, alpha=alpha, beta=beta)
        out[..., lo:hi] = d[..., lo - slo:hi - slo]
    return np.moveaxis(out, -1, axis)


def derivative_matrix(n: int, h: float, tables=None) -> np.ndarray:
    """The dense n x n operator D with D @ g == fc_derivative(g, h): column j
    is the FC derivative of the j-th unit vector."""
    return fc_derivative(np.eye(n), h, axis=-1, tables=tables).T


if __name__ == "__main__":
    print(write_tables())
