"""Generates the constant tables of the CUDA path (run once; output is committed).

    python -m paper_2303_13632_gb300.gen.gen_tables

Writes ``csrc/eri_tables.inc`` with
  * Rys roots x_mu = t_mu^2 and weights w_mu of the weight exp(-T t^2) on t in [0, 1]
    (Sec. II-C, Eq. 5 inputs R_Rys), for n_Rys = 1..RYS_NMAX, as piecewise polynomials of
    degree RYS_DEG in u = 2(T - k) - 1 on unit intervals [k, k+1) of T in [0, T_asym(n)):
    fitted as Chebyshev series (interpolation at Chebyshev points) and converted exactly, at
    40 digits, to monomial coefficients so the device evaluates them by Horner's rule (one
    FMA per term); and the 2n-point Gauss-Hermite nodes/weights for the large-T limit
        x_mu = u_mu^2 / T,  w_mu = H_mu / sqrt(T)      (T >= T_asym(n));
  * FP32 copies of the monomial coefficients j >= RYS_TAIL: the device runs that part of
    Horner's rule in FP32 (with u rounded to FP32) and the rest in FP64.  The tail is below
    1e-9 of the value over every piece, and the whole evaluation, emulated here with numpy
    float32, is verified against fresh high-precision values before the file is written;
  * the Boys function F_m(T_k) on the grid T_k = k * BOYS_STEP (k < BOYS_NGRID) for
    m = 0..BOYS_MCOLS-1, used by a Taylor expansion plus downward recursion.

Everything is computed with mpmath at 40 significant digits, independently of the
CPU oracle.  The roots and weights come from the discretised Stieltjes procedure on a
160-point Gauss-Legendre rule in t (well conditioned, unlike the moment route) and the
eigen-decomposition of the Jacobi matrix.  Each Chebyshev piece is verified at random
points against fresh high-precision values before the file is written.
"""
from __future__ import annotations

import os
import sys
import time

import mpmath as mp
import numpy as np

mp.mp.dps = 40

RYS_NMAX = 9          # orders needed: forward L <= 12 -> 7; derivative classes need up to 9
RYS_DEG = 12          # polynomial degree per unit interval
RYS_TAIL = 10         # coefficients j >= RYS_TAIL are also stored as FP32 (evaluated in FP32)
GL_N = 160            # Gauss-Legendre points discretising the Rys measure
BOYS_STEP = 0.1
BOYS_TMAX = 50.0      # F_m(T) for T >= BOYS_TMAX comes from the asymptotic form
BOYS_MMAX = 16        # highest order served by the device Boys function
BOYS_TAYLOR = 10      # Taylor terms
BOYS_MCOLS = BOYS_MMAX + BOYS_TAYLOR + 1
BOYS_NGRID = int(round(BOYS_TMAX / BOYS_STEP)) + 2

_HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(_HERE), "csrc", "eri_tables.inc")


def _legendre_pn(x, N):
    p0, p1 = mp.mpf(1), x
    for k in range(2, N + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    return p0, p1


def gauss_legendre_01(N):
    xs, _ = np.polynomial.legendre.leggauss(N)
    nodes, weights = [], []
    for x0 in xs:
        x = mp.mpf(x0)
        for _ in range(8):
            p0, p1 = _legendre_pn(x, N)
            dp = N * (x * p1 - p0) / (x * x - 1)
            x = x - p1 / dp
        p0, p1 = _legendre_pn(x, N)
        dp = N * (x * p1 - p0) / (x * x - 1)
        nodes.append((x + 1) / 2)
        weights.append(1 / ((1 - x * x) * dp * dp))
    return nodes, weights


GL_T, GL_W = gauss_legendre_01(GL_N)
GL_X = [t * t for t in GL_T]


def rys_roots_weights(n, T):
    """Gauss rule of order n for the measure exp(-T t^2) dt on [0,1] in the variable x = t^2."""
    T = mp.mpf(T)
    mass = [w * mp.exp(-T * x) for w, x in zip(GL_W, GL_X)]
    alpha, beta = [], []
    p_prev = [mp.mpf(0)] * GL_N
    p = [mp.mpf(1)] * GL_N
    nrm_prev = None
    for k in range(n):
        nrm = mp.fsum(m * v * v for m, v in zip(mass, p))
        a = mp.fsum(m * x * v * v for m, x, v in zip(mass, GL_X, p)) / nrm
        b = nrm if k == 0 else nrm / nrm_prev
        alpha.append(a)
        beta.append(b)
        p_new = [(x - a) * v - (b if k > 0 else 0) * u for x, v, u in zip(GL_X, p, p_prev)]
        p_prev, p, nrm_prev = p, p_new, nrm
    J = mp.matrix(n, n)
    for i in range(n):
        J[i, i] = alpha[i]
        if i + 1 < n:
            J[i, i + 1] = J[i + 1, i] = mp.sqrt(beta[i + 1])
    E, Q = mp.eigsy(J)
    pairs = sorted((E[i], beta[0] * Q[0, i] ** 2) for i in range(n))
    return [x for x, _ in pairs], [w for _, w in pairs]


def hermite_positive(n):
    """Positive nodes u and weights H of the 2n-point Gauss-Hermite rule (weight exp(-u^2))."""
    N = 2 * n
    xs, _ = np.polynomial.hermite.hermgauss(N)
    out = []
    for x0 in xs:
        if x0 <= 0:
            continue
        x = mp.mpf(x0)
        for _ in range(10):
            h0, h1 = mp.mpf(1), 2 * x
            for k in range(1, N):
                h0, h1 = h1, 2 * x * h1 - 2 * k * h0
            x = x - h1 / (2 * N * h0)
        h0, h1 = mp.mpf(1), 2 * x
        for k in range(1, N):
            h0, h1 = h1, 2 * x * h1 - 2 * k * h0
        w = mp.mpf(2) ** (N - 1) * mp.factorial(N) * mp.sqrt(mp.pi) / (N * N * h0 * h0)
        out.append((x, w))
    out.sort()
    return out


def asym_error(n, T, herm):
    x, w = rys_roots_weights(n, T)
    e = 0.0
    for i in range(n):
        e = max(e, float(abs((x[i] - herm[i][0] ** 2 / T) / x[i])),
                float(abs((w[i] - herm[i][1] / mp.sqrt(T)) / w[i])))
    return e


def chebyshev_piece(n, a, b, deg):
    nodes = [(a + b) / 2 + (b - a) / 2 * mp.cos(mp.pi * (k + mp.mpf(1) / 2) / (deg + 1))
             for k in range(deg + 1)]
    vals = [rys_roots_weights(n, t) for t in nodes]
    coefs = []
    for mu in range(n):
        for kind in (0, 1):
            fv = [v[kind][mu] for v in vals]
            c = []
            for j in range(deg + 1):
                s = mp.fsum(fv[k] * mp.cos(mp.pi * j * (k + mp.mpf(1) / 2) / (deg + 1))
                            for k in range(deg + 1)) * 2 / (deg + 1)
                c.append(s)
            c[0] /= 2
            coefs.append(c)
    return coefs


def cheb_to_monomial(c):
    """Monomial coefficients a_i of sum_j c_j T_j(u) (exact integer recurrence, mp arithmetic)."""
    deg = len(c) - 1
    Tm = [[0] * (deg + 1) for _ in range(deg + 1)]
    Tm[0][0] = 1
    if deg >= 1:
        Tm[1][1] = 1
    for j in range(2, deg + 1):
        for i in range(deg + 1):
            Tm[j][i] = (2 * Tm[j - 1][i - 1] if i > 0 else 0) - Tm[j - 2][i]
    return [mp.fsum(c[j] * Tm[j][i] for j in range(deg + 1)) for i in range(deg + 1)]


def horner_split(a, u):
    """The device evaluation: terms j >= RYS_TAIL by Horner in FP32 on float32(u), the rest in
    FP64."""
    uf = np.float32(u)
    sf = np.float32(a[-1])
    for j in range(len(a) - 2, RYS_TAIL - 1, -1):
        sf = np.float32(np.float32(sf * uf) + np.float32(a[j]))
    s = float(sf)
    for j in range(RYS_TAIL - 1, -1, -1):
        s = s * u + a[j]
    return s


def boys_mp(m, T):
    """F_m(T) = 1F1(m + 1/2; m + 3/2; -T) / (2m + 1)."""
    return mp.hyp1f1(m + mp.mpf(1) / 2, m + mp.mpf(3) / 2, -mp.mpf(T)) / (2 * m + 1)


def fmt(v: float) -> str:
    return float(v).hex()


def main():
    t0 = time.time()
    rng = np.random.default_rng(2303)
    lines = []
    lines.append("/* Generated by paper_2303_13632_gb300/gen/gen_tables.py -- do not edit. */")
    lines.append(f"#define RYS_NMAX {RYS_NMAX}")
    lines.append(f"#define RYS_DEG {RYS_DEG}")
    lines.append(f"#define BOYS_STEP {BOYS_STEP!r}")
    lines.append(f"#define BOYS_TMAX {BOYS_TMAX!r}")
    lines.append(f"#define BOYS_MMAX {BOYS_MMAX}")
    lines.append(f"#define BOYS_TAYLOR {BOYS_TAYLOR}")
    lines.append(f"#define BOYS_MCOLS {BOYS_MCOLS}")
    lines.append(f"#define BOYS_NGRID {BOYS_NGRID}")
    tasym, offsets, cheb, hx, hw = [0], [0], [], [0.0], [0.0]
    hoff = [0, 1]
    worst = 0.0
    tail_worst = 0.0
    for n in range(1, RYS_NMAX + 1):
        herm = hermite_positive(n)
        T = 30
        while True:
            if asym_error(n, T, herm) < 1e-16 and asym_error(n, T + 0.5, herm) < 1e-16:
                break
            T += 1
        tasym.append(T)
        offsets.append(len(cheb))
        for k in range(T):
            piece = [cheb_to_monomial(c) for c in chebyshev_piece(n, k, k + 1, RYS_DEG)]
            piece_d = [[float(v) for v in a] for a in piece]
            for _ in range(8):
                Tt = k + rng.random()
                x, w = rys_roots_weights(n, Tt)
                u = 2 * (Tt - k) - 1
                for mu in range(n):
                    worst = max(worst,
                                abs(horner_split(piece_d[2 * mu], u) - float(x[mu])) / float(x[mu]),
                                abs(horner_split(piece_d[2 * mu + 1], u) - float(w[mu])) / float(w[mu]))
            # tail bound: |sum_{j >= RYS_TAIL} a_j u^j| / |p(u)| on a grid of the piece
            uu = np.linspace(-1.0, 1.0, 41)
            for a, ad in zip(piece, piece_d):
                pv = np.array([float(mp.polyval(a[::-1], mp.mpf(v))) for v in uu])
                tv = np.abs(sum(ad[j] * uu ** j for j in range(RYS_TAIL, RYS_DEG + 1)))
                tail_worst = max(tail_worst, float(np.max(tv / np.abs(pv))))
            for f in piece_d:
                cheb.extend(f)
        for u, h in herm:
            hx.append(float(u * u))
            hw.append(float(h))
        hoff.append(len(hx))
        print(f"n={n}: T_asym={T}, pieces={T}, worst so far {worst:.3e}, tail {tail_worst:.2e}, "
              f"{time.time() - t0:.0f}s", flush=True)
    if worst > 6e-16:
        sys.exit(f"polynomial fit check failed: {worst}")
    if tail_worst > 1e-9:
        sys.exit(f"polynomial tail too large for FP32 evaluation: {tail_worst}")
    nfun = len(cheb) // (RYS_DEG + 1)
    tail = [float(np.float32(v)) for f in range(nfun)
            for v in cheb[f * (RYS_DEG + 1) + RYS_TAIL:(f + 1) * (RYS_DEG + 1)]]
    lines.append("/* first T of the Gauss-Hermite regime for n = index */")
    lines.append("static const int rys_tasym_h[RYS_NMAX + 1] = {" + ", ".join(map(str, tasym)) + "};")
    lines.append("/* offset (doubles) of the pieces of order n; piece k of order n holds 2n polynomials of")
    lines.append("   RYS_DEG+1 monomial coefficients in u = 2(T - k) - 1: x_1, w_1, x_2, w_2, ... */")
    lines.append("static const long rys_offset_h[RYS_NMAX + 1] = {" + ", ".join(map(str, offsets)) + "};")
    lines.append(f"#define RYS_POLY_LEN {len(cheb)}")
    lines.append("static const double rys_poly_h[RYS_POLY_LEN] = {")
    for i in range(0, len(cheb), 4):
        lines.append("  " + ", ".join(fmt(v) for v in cheb[i:i + 4]) + ",")
    lines.append("};")
    lines.append(f"#define RYS_TAIL {RYS_TAIL}")
    lines.append(f"/* FP32 copies of coefficients RYS_TAIL..RYS_DEG of each polynomial (worst tail/|p| = {tail_worst:.2e}) */")
    lines.append(f"#define RYS_TAIL_LEN {len(tail)}")
    lines.append("static const float rys_tail_f_h[RYS_TAIL_LEN] = {")
    for i in range(0, len(tail), 5):
        lines.append("  " + ", ".join(float(v).hex() + "f" for v in tail[i:i + 5]) + ",")
    lines.append("};")
    lines.append("/* Gauss-Hermite: index hermite_offset[n] + mu - 1 holds u_mu^2 and H_mu of order n */")
    lines.append("static const int rys_herm_offset_h[RYS_NMAX + 2] = {" + ", ".join(map(str, hoff)) + "};")
    lines.append(f"#define RYS_HERM_LEN {len(hx)}")
    lines.append("static const double rys_herm_x2_h[RYS_HERM_LEN] = {" + ", ".join(fmt(v) for v in hx) + "};")
    lines.append("static const double rys_herm_w_h[RYS_HERM_LEN] = {" + ", ".join(fmt(v) for v in hw) + "};")
    # Boys grid
    grid = []
    for k in range(BOYS_NGRID):
        T = mp.mpf(k) * mp.mpf(BOYS_STEP)
        for m in range(BOYS_MCOLS):
            grid.append(float(boys_mp(m, T)))
    lines.append(f"#define BOYS_GRID_LEN {len(grid)}")
    lines.append("/* F_m(k * BOYS_STEP) at index k * BOYS_MCOLS + m */")
    lines.append("static const double boys_grid_h[BOYS_GRID_LEN] = {")
    for i in range(0, len(grid), 4):
        lines.append("  " + ", ".join(fmt(v) for v in grid[i:i + 4]) + ",")
    lines.append("};")
    # Taylor coefficients of F_0 and F_1 about each grid point, already divided by j!, so that
    # F_0(T_k - d) = sum_j t[j] d^j and F_1(T_k - d) = sum_j t[BOYS_TAYLOR + j] d^j
    t01 = []
    for k in range(BOYS_NGRID):
        T = mp.mpf(k) * mp.mpf(BOYS_STEP)
        F = [boys_mp(m, T) for m in range(BOYS_TAYLOR + 1)]
        t01 += [float(F[j] / mp.factorial(j)) for j in range(BOYS_TAYLOR)]
        t01 += [float(F[j + 1] / mp.factorial(j)) for j in range(BOYS_TAYLOR)]
    lines.append(f"#define BOYS_T01_LEN {len(t01)}")
    lines.append("/* F_0 and F_1 Taylor coefficients F_{m+j}(k * BOYS_STEP) / j! at index")
    lines.append("   k * 2 * BOYS_TAYLOR + m * BOYS_TAYLOR + j */")
    lines.append("static const double boys_t01_h[BOYS_T01_LEN] = {")
    for i in range(0, len(t01), 4):
        lines.append("  " + ", ".join(fmt(v) for v in t01[i:i + 4]) + ",")
    lines.append("};")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"wrote {OUT}: {len(cheb)} polynomial coefficients, {len(grid)} Boys values, "
          f"fit check {worst:.3e}, {time.time() - t0:.0f}s")


if __name__ == "__main__":
    main()
