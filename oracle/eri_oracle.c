/*
 * eri_oracle.c -- plain, slow FP64 CPU oracle for electron repulsion integrals.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or generator with the CUDA path.
 *
 * What it computes (arXiv 2303.13632):
 *   - normalised primitive Cartesian GTOs (Sec. II-A, Eq. for g_{a,R_A}), with the
 *     axis-aligned normalisation of Kenny et al. applied to every component of a shell;
 *   - the ERI [ab|cd] of Eq. 1 for whole shell quartets, contracted over primitives
 *     (contracted function = sum_k c_k N(alpha_k, L) g_k, no renormalisation);
 *   - the Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt;
 *   - the lossy compression of Sec. II-D: eps = b_max / (2^{n-1}-1) (Eq. 9),
 *     q = ANINT(x / eps) (Eq. 10), x~ = q * eps (Eq. 11);
 *   - nuclear-centre and exponent gradients of E = sum G_abcd (ab|cd);
 *   - the Coulomb and exchange matrices J and K of a density matrix (orc_digest_jk).
 *
 * The reference ERIs are NOT evaluated with the paper's Rys scheme.  Two independent
 * exact-in-principle schemes named in Sec. II-C are used instead:
 *   (1) Obara-Saika vertical recursion to [e0|f0] followed by the Head-Gordon-Pople
 *       horizontal transfer (orc_eri_quartet), and
 *   (2) McMurchie-Davidson Hermite expansion (orc_eri_quartet_md).
 * They share only the Boys function, which is pinned on its own by the tests.
 * A third route, (3) the paper's own Rys scheme written out step by step (orc_eri_quartet_rys,
 * with roots and weights from orc_rys_roots), checks the readings of Sec. II-C (the B and C
 * coefficients of Eq. 6, the single weight factor, n_Rys) against (1) and (2).
 *
 * Cartesian component order within a shell of angular momentum L: a_x runs from
 * L down to 0, then a_y from L-a_x down to 0 (xx, xy, xz, yy, yz, zz for L=2).
 * Output order within a shell quartet: a slowest, d fastest (row major).
 *
 * All arithmetic is IEEE double; no platform-specific code.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------- */
/* Cartesian bookkeeping                                                      */
/* ------------------------------------------------------------------------- */

static int ncart(int L) { return (L + 1) * (L + 2) / 2; }

/* number of Cartesian triples with total degree <= L */
static int ntrip(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }

/* index of component (ax, ay, az) within its shell, order as documented above */
static int cart_index(int ax, int ay, int az)
{
    int L = ax + ay + az;
    (void)ay;
    return (L - ax) * (L - ax + 1) / 2 + az;
}

/* compact index of a triple over all degrees: all triples of degree < L come first */
static int trip_index(const int e[3])
{
    int L = e[0] + e[1] + e[2];
    return L * (L + 1) * (L + 2) / 6 + cart_index(e[0], e[1], e[2]);
}

static void cart_comp(int L, int idx, int c[3])
{
    int k = 0;
    for (int ax = L; ax >= 0; --ax)
        for (int ay = L - ax; ay >= 0; --ay) {
            if (k == idx) {
                c[0] = ax;
                c[1] = ay;
                c[2] = L - ax - ay;
                return;
            }
            ++k;
        }
    c[0] = c[1] = c[2] = -1;
}

int orc_ncart(int L) { return ncart(L); }

void orc_cart_comp(int L, int idx, int *c) { cart_comp(L, idx, c); }

/* (2L-1)!! with (-1)!! = 1 */
static double double_factorial_odd(int L)
{
    double r = 1.0;
    for (int k = 2 * L - 1; k > 1; k -= 2)
        r *= (double)k;
    return r;
}

/* Normalisation of Sec. II-A: the axis-aligned component x^L exp(-alpha r^2) has unit norm.
 * N = (2 alpha / pi)^{3/4} (4 alpha)^{L/2} / sqrt((2L-1)!!). */
double orc_norm(double alpha, int L)
{
    return pow(2.0 * alpha / ORC_PI, 0.75) * pow(4.0 * alpha, 0.5 * L) /
           sqrt(double_factorial_odd(L));
}

/* ------------------------------------------------------------------------- */
/* Boys function  F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt                      */
/* ------------------------------------------------------------------------- */

#define ORC_BOYS_SERIES_TMAX 40.0

/* Fills F[0..mmax].  For T <= 40 the top order comes from the positive series
 * F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)), followed by the
 * stable downward recursion F_m = (2T F_{m+1} + exp(-T)) / (2m+1).  For T > 40,
 * F_0 = sqrt(pi/T) erf(sqrt(T)) / 2 and the upward recursion
 * F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T), which is stable there for m < 40. */
void orc_boys(int mmax, double T, double *F)
{
    double eT = exp(-T);
    if (T <= ORC_BOYS_SERIES_TMAX) {
        double term = 1.0 / (2 * mmax + 1);
        double sum = term;
        for (int k = 1; k < 2000; ++k) {
            term *= 2.0 * T / (double)(2 * mmax + 2 * k + 1);
            sum += term;
            if (term < 1e-18 * sum && 2.0 * T < (double)(2 * mmax + 2 * k + 1))
                break;
        }
        F[mmax] = eT * sum;
        for (int m = mmax - 1; m >= 0; --m)
            F[m] = (2.0 * T * F[m + 1] + eT) / (double)(2 * m + 1);
    } else {
        F[0] = 0.5 * sqrt(ORC_PI / T) * erf(sqrt(T));
        for (int m = 0; m < mmax; ++m)
            F[m + 1] = ((double)(2 * m + 1) * F[m] - eT) / (2.0 * T);
    }
}

/* ------------------------------------------------------------------------- */
/* Obara-Saika vertical recursion for [e0|f0]^(m) of one primitive quartet    */
/* ------------------------------------------------------------------------- */

typedef struct {
    double PA[3], WP[3], QC[3], WQ[3];
    double p, q, rho;
    double oo2p, oo2q, oo2pq; /* 1/(2p), 1/(2q), 1/(2(p+q)) */
    double pref;              /* 2 pi^{5/2} / (p q sqrt(p+q)) K_AB K_CD */
    double F[64];             /* Boys values */
    int e_hi, f_hi, m_hi;
    int ne, nf, nm;
    double *val;
    unsigned char *done;
} vrr_ctx;

static double vrr(vrr_ctx *c, const int e[3], const int f[3], int m);

static double vrr_at(vrr_ctx *c, int e0, int e1, int e2, int f0, int f1, int f2, int m)
{
    if (e0 < 0 || e1 < 0 || e2 < 0 || f0 < 0 || f1 < 0 || f2 < 0)
        return 0.0;
    int e[3] = {e0, e1, e2}, f[3] = {f0, f1, f2};
    return vrr(c, e, f, m);
}

static double vrr(vrr_ctx *c, const int e[3], const int f[3], int m)
{
    size_t key = ((size_t)trip_index(e) * c->nf + trip_index(f)) * c->nm + m;
    if (c->done[key])
        return c->val[key];
    double v;
    int le = e[0] + e[1] + e[2], lf = f[0] + f[1] + f[2];
    if (le == 0 && lf == 0) {
        v = c->pref * c->F[m];
    } else if (lf > 0) {
        /* build on the ket: [e0|(f'+1_i)0] */
        int i = (f[0] > 0) ? 0 : ((f[1] > 0) ? 1 : 2);
        int fp[3] = {f[0], f[1], f[2]};
        fp[i] -= 1;
        int fm[3] = {fp[0], fp[1], fp[2]};
        fm[i] -= 1;
        int em[3] = {e[0], e[1], e[2]};
        em[i] -= 1;
        v = c->QC[i] * vrr(c, e, fp, m) + c->WQ[i] * vrr(c, e, fp, m + 1);
        if (fp[i] > 0)
            v += fp[i] * c->oo2q *
                 (vrr_at(c, e[0], e[1], e[2], fm[0], fm[1], fm[2], m) -
                  c->rho / c->q * vrr_at(c, e[0], e[1], e[2], fm[0], fm[1], fm[2], m + 1));
        if (e[i] > 0)
            v += e[i] * c->oo2pq * vrr_at(c, em[0], em[1], em[2], fp[0], fp[1], fp[2], m + 1);
    } else {
        /* build on the bra: [(e'+1_i)0|00] */
        int i = (e[0] > 0) ? 0 : ((e[1] > 0) ? 1 : 2);
        int ep[3] = {e[0], e[1], e[2]};
        ep[i] -= 1;
        int zero[3] = {0, 0, 0};
        v = c->PA[i] * vrr(c, ep, zero, m) + c->WP[i] * vrr(c, ep, zero, m + 1);
        if (ep[i] > 0) {
            int em[3] = {ep[0], ep[1], ep[2]};
            em[i] -= 1;
            v += ep[i] * c->oo2p * (vrr(c, em, zero, m) - c->rho / c->p * vrr(c, em, zero, m + 1));
        }
    }
    c->done[key] = 1;
    c->val[key] = v;
    return v;
}

/* Accumulates w * [e0|f0]^(0) into tab[trip(e)][trip(f)] for every |e| <= e_hi, |f| <= f_hi,
 * for unnormalised primitives (x-A)^a exp(-a |r-A|^2) etc. */
static void vrr_prim_accumulate(const double A[3], double ea, const double B[3], double eb,
                                const double C[3], double ec, const double D[3], double ed,
                                int e_hi, int f_hi, double w, double *tab)
{
    vrr_ctx c;
    double p = ea + eb, q = ec + ed;
    double P[3], Q[3], W[3], ab2 = 0.0, cd2 = 0.0, pq2 = 0.0;
    for (int i = 0; i < 3; ++i) {
        P[i] = (ea * A[i] + eb * B[i]) / p;
        Q[i] = (ec * C[i] + ed * D[i]) / q;
        W[i] = (p * P[i] + q * Q[i]) / (p + q);
        ab2 += (A[i] - B[i]) * (A[i] - B[i]);
        cd2 += (C[i] - D[i]) * (C[i] - D[i]);
        pq2 += (P[i] - Q[i]) * (P[i] - Q[i]);
        c.PA[i] = P[i] - A[i];
        c.WP[i] = W[i] - P[i];
        c.QC[i] = Q[i] - C[i];
        c.WQ[i] = W[i] - Q[i];
    }
    c.p = p;
    c.q = q;
    c.rho = p * q / (p + q);
    c.oo2p = 0.5 / p;
    c.oo2q = 0.5 / q;
    c.oo2pq = 0.5 / (p + q);
    double Kab = exp(-ea * eb / p * ab2), Kcd = exp(-ec * ed / q * cd2);
    c.pref = 2.0 * pow(ORC_PI, 2.5) / (p * q * sqrt(p + q)) * Kab * Kcd;
    c.e_hi = e_hi;
    c.f_hi = f_hi;
    c.m_hi = e_hi + f_hi;
    orc_boys(c.m_hi, c.rho * pq2, c.F);
    c.ne = ntrip(e_hi);
    c.nf = ntrip(f_hi);
    c.nm = c.m_hi + 1;
    size_t n = (size_t)c.ne * c.nf * c.nm;
    c.val = (double *)malloc(n * sizeof(double));
    c.done = (unsigned char *)calloc(n, 1);
    for (int le = 0; le <= e_hi; ++le)
        for (int ie = 0; ie < ncart(le); ++ie) {
            int e[3];
            cart_comp(le, ie, e);
            for (int lf = 0; lf <= f_hi; ++lf)
                for (int jf = 0; jf < ncart(lf); ++jf) {
                    int f[3];
                    cart_comp(lf, jf, f);
                    tab[(size_t)trip_index(e) * c.nf + trip_index(f)] += w * vrr(&c, e, f, 0);
                }
        }
    free(c.val);
    free(c.done);
}

/* ------------------------------------------------------------------------- */
/* Head-Gordon-Pople horizontal transfer                                      */
/* ------------------------------------------------------------------------- */

typedef struct {
    const double *tab; /* [ntrip(e_hi)][ntrip(f_hi)] */
    int nf;
    double AB[3], CD[3];
} hrr_ctx;

/* (a b | f 0): (a, b+1_i| = (a+1_i, b| + AB_i (a, b| */
static double hrr_bra(const hrr_ctx *h, int a0, int a1, int a2, int b0, int b1, int b2, int fi)
{
    if (b0 + b1 + b2 == 0) {
        int a[3] = {a0, a1, a2};
        return h->tab[(size_t)trip_index(a) * h->nf + fi];
    }
    int i = (b0 > 0) ? 0 : ((b1 > 0) ? 1 : 2);
    int b[3] = {b0, b1, b2};
    b[i] -= 1;
    int ap[3] = {a0, a1, a2};
    ap[i] += 1;
    return hrr_bra(h, ap[0], ap[1], ap[2], b[0], b[1], b[2], fi) +
           h->AB[i] * hrr_bra(h, a0, a1, a2, b[0], b[1], b[2], fi);
}

/* (ab | c d) from X[f] = (ab|f0): (ab|c, d+1_i) = (ab|c+1_i, d) + CD_i (ab|c, d) */
static double hrr_ket(const double *X, const hrr_ctx *h, int c0, int c1, int c2, int d0, int d1,
                      int d2)
{
    if (d0 + d1 + d2 == 0) {
        int c[3] = {c0, c1, c2};
        return X[trip_index(c)];
    }
    int i = (d0 > 0) ? 0 : ((d1 > 0) ? 1 : 2);
    int d[3] = {d0, d1, d2};
    d[i] -= 1;
    int cp[3] = {c0, c1, c2};
    cp[i] += 1;
    return hrr_ket(X, h, cp[0], cp[1], cp[2], d[0], d[1], d[2]) +
           h->CD[i] * hrr_ket(X, h, c0, c1, c2, d[0], d[1], d[2]);
}

/* Transfers the table of [e0|f0] (|e| <= e_hi, |f| <= f_hi) to (ab|cd) for shells
 * La, Lb, Lc, Ld (requires La+Lb <= e_hi, Lc+Ld <= f_hi); out is row major. */
static void hrr_shells(const double *tab, int e_hi, int f_hi, const double A[3], const double B[3],
                       const double C[3], const double D[3], int La, int Lb, int Lc, int Ld,
                       double *out)
{
    hrr_ctx h;
    h.tab = tab;
    h.nf = ntrip(f_hi);
    for (int i = 0; i < 3; ++i) {
        h.AB[i] = A[i] - B[i];
        h.CD[i] = C[i] - D[i];
    }
    int na = ncart(La), nb = ncart(Lb), nc = ncart(Lc), nd = ncart(Ld);
    double *X = (double *)calloc((size_t)h.nf, sizeof(double));
    for (int ia = 0; ia < na; ++ia)
        for (int ib = 0; ib < nb; ++ib) {
            int a[3], b[3];
            cart_comp(La, ia, a);
            cart_comp(Lb, ib, b);
            memset(X, 0, sizeof(double) * h.nf);
            for (int lf = Lc; lf <= Lc + Ld; ++lf)
                for (int jf = 0; jf < ncart(lf); ++jf) {
                    int f[3];
                    cart_comp(lf, jf, f);
                    int fi = trip_index(f);
                    X[fi] = hrr_bra(&h, a[0], a[1], a[2], b[0], b[1], b[2], fi);
                }
            for (int ic = 0; ic < nc; ++ic)
                for (int id = 0; id < nd; ++id) {
                    int c[3], d[3];
                    cart_comp(Lc, ic, c);
                    cart_comp(Ld, id, d);
                    out[((size_t)(ia * nb + ib) * nc + ic) * nd + id] =
                        hrr_ket(X, &h, c[0], c[1], c[2], d[0], d[1], d[2]);
                }
        }
    free(X);
}

/* ------------------------------------------------------------------------- */
/* Shell-quartet ERIs (Obara-Saika + Head-Gordon-Pople)                       */
/* ------------------------------------------------------------------------- */

typedef struct {
    double center[3];
    int32_t L;
    int32_t nprim;
    const double *exps;
    const double *coefs;
} orc_shell;

/* (ab|cd) for contracted, normalised shells; out has ncart(La)*ncart(Lb)*ncart(Lc)*ncart(Ld)
 * entries, row major (a slowest). */
int orc_eri_quartet(const orc_shell *sa, const orc_shell *sb, const orc_shell *sc,
                    const orc_shell *sd, double *out)
{
    int La = sa->L, Lb = sb->L, Lc = sc->L, Ld = sd->L;
    if (La < 0 || Lb < 0 || Lc < 0 || Ld < 0 || La + Lb + Lc + Ld > 40)
        return -1;
    int e_hi = La + Lb, f_hi = Lc + Ld;
    size_t ntab = (size_t)ntrip(e_hi) * ntrip(f_hi);
    double *tab = (double *)calloc(ntab, sizeof(double));
    for (int i = 0; i < sa->nprim; ++i)
        for (int j = 0; j < sb->nprim; ++j)
            for (int k = 0; k < sc->nprim; ++k)
                for (int l = 0; l < sd->nprim; ++l) {
                    double w = sa->coefs[i] * orc_norm(sa->exps[i], La) * sb->coefs[j] *
                               orc_norm(sb->exps[j], Lb) * sc->coefs[k] *
                               orc_norm(sc->exps[k], Lc) * sd->coefs[l] *
                               orc_norm(sd->exps[l], Ld);
                    vrr_prim_accumulate(sa->center, sa->exps[i], sb->center, sb->exps[j],
                                        sc->center, sc->exps[k], sd->center, sd->exps[l], e_hi,
                                        f_hi, w, tab);
                }
    hrr_shells(tab, e_hi, f_hi, sa->center, sb->center, sc->center, sd->center, La, Lb, Lc, Ld,
               out);
    free(tab);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* McMurchie-Davidson evaluator (independent second route)                    */
/* ------------------------------------------------------------------------- */

/* Hermite expansion coefficients E^{ij}_t of a 1-D Gaussian product (exponents a, b,
 * separation XAB = A - B).  E[i][j][t], i <= imax, j <= jmax, t <= i + j. */
#define MD_LMAX 12
typedef struct {
    double E[MD_LMAX + 1][MD_LMAX + 1][2 * MD_LMAX + 2];
} md_e;

static void md_hermite_e(double a, double b, double XAB, int imax, int jmax, md_e *out)
{
    double p = a + b, mu = a * b / p;
    double XPA = -b / p * XAB, XPB = a / p * XAB;
    memset(out, 0, sizeof(*out));
    out->E[0][0][0] = exp(-mu * XAB * XAB);
    for (int i = 0; i <= imax; ++i)
        for (int j = 0; j <= jmax; ++j) {
            if (i == 0 && j == 0)
                continue;
            for (int t = 0; t <= i + j; ++t) {
                double v = 0.0;
                if (i > 0) {
                    /* E^{i,j}_t = E^{i-1,j}_{t-1}/(2p) + XPA E^{i-1,j}_t + (t+1) E^{i-1,j}_{t+1} */
                    if (t > 0)
                        v += out->E[i - 1][j][t - 1] / (2.0 * p);
                    v += XPA * out->E[i - 1][j][t];
                    v += (t + 1) * out->E[i - 1][j][t + 1];
                } else {
                    if (t > 0)
                        v += out->E[i][j - 1][t - 1] / (2.0 * p);
                    v += XPB * out->E[i][j - 1][t];
                    v += (t + 1) * out->E[i][j - 1][t + 1];
                }
                out->E[i][j][t] = v;
            }
        }
}

/* Hermite Coulomb integrals R^n_{tuv}(rho, PQ) for t+u+v+n <= L. */
typedef struct {
    int L;
    double rho, X, Y, Z;
    double F[64];
    double *val;
    unsigned char *done;
} md_r;

static size_t md_r_key(const md_r *r, int n, int t, int u, int v)
{
    int d = r->L + 1;
    return (((size_t)n * d + t) * d + u) * d + v;
}

static double md_rtuv(md_r *r, int n, int t, int u, int v)
{
    if (t < 0 || u < 0 || v < 0)
        return 0.0;
    size_t key = md_r_key(r, n, t, u, v);
    if (r->done[key])
        return r->val[key];
    double val;
    if (t == 0 && u == 0 && v == 0) {
        val = pow(-2.0 * r->rho, n) * r->F[n];
    } else if (t > 0) {
        val = (t - 1) * md_rtuv(r, n + 1, t - 2, u, v) + r->X * md_rtuv(r, n + 1, t - 1, u, v);
    } else if (u > 0) {
        val = (u - 1) * md_rtuv(r, n + 1, t, u - 2, v) + r->Y * md_rtuv(r, n + 1, t, u - 1, v);
    } else {
        val = (v - 1) * md_rtuv(r, n + 1, t, u, v - 2) + r->Z * md_rtuv(r, n + 1, t, u, v - 1);
    }
    r->done[key] = 1;
    r->val[key] = val;
    return val;
}

int orc_eri_quartet_md(const orc_shell *sa, const orc_shell *sb, const orc_shell *sc,
                       const orc_shell *sd, double *out)
{
    int La = sa->L, Lb = sb->L, Lc = sc->L, Ld = sd->L;
    if (La < 0 || Lb < 0 || Lc < 0 || Ld < 0 || La + Lb > MD_LMAX || Lc + Ld > MD_LMAX)
        return -1;
    int na = ncart(La), nb = ncart(Lb), nc = ncart(Lc), nd = ncart(Ld);
    size_t nout = (size_t)na * nb * nc * nd;
    memset(out, 0, nout * sizeof(double));
    int L = La + Lb + Lc + Ld;
    md_e *Eab = (md_e *)malloc(3 * sizeof(md_e));
    md_e *Ecd = (md_e *)malloc(3 * sizeof(md_e));
    md_r r;
    r.L = L;
    size_t nr = (size_t)(L + 1) * (L + 1) * (L + 1) * (L + 1);
    r.val = (double *)malloc(nr * sizeof(double));
    r.done = (unsigned char *)malloc(nr);
    for (int i = 0; i < sa->nprim; ++i)
        for (int j = 0; j < sb->nprim; ++j)
            for (int k = 0; k < sc->nprim; ++k)
                for (int l = 0; l < sd->nprim; ++l) {
                    double a = sa->exps[i], b = sb->exps[j], c = sc->exps[k], d = sd->exps[l];
                    double p = a + b, q = c + d;
                    double w = sa->coefs[i] * orc_norm(a, La) * sb->coefs[j] * orc_norm(b, Lb) *
                               sc->coefs[k] * orc_norm(c, Lc) * sd->coefs[l] * orc_norm(d, Ld);
                    double P[3], Q[3];
                    for (int x = 0; x < 3; ++x) {
                        P[x] = (a * sa->center[x] + b * sb->center[x]) / p;
                        Q[x] = (c * sc->center[x] + d * sd->center[x]) / q;
                        md_hermite_e(a, b, sa->center[x] - sb->center[x], La, Lb, &Eab[x]);
                        md_hermite_e(c, d, sc->center[x] - sd->center[x], Lc, Ld, &Ecd[x]);
                    }
                    r.rho = p * q / (p + q);
                    r.X = P[0] - Q[0];
                    r.Y = P[1] - Q[1];
                    r.Z = P[2] - Q[2];
                    orc_boys(L, r.rho * (r.X * r.X + r.Y * r.Y + r.Z * r.Z), r.F);
                    memset(r.done, 0, nr);
                    double pref = w * 2.0 * pow(ORC_PI, 2.5) / (p * q * sqrt(p + q));
                    for (int ia = 0; ia < na; ++ia)
                        for (int ib = 0; ib < nb; ++ib)
                            for (int ic = 0; ic < nc; ++ic)
                                for (int id = 0; id < nd; ++id) {
                                    int ca[3], cb[3], cc[3], cd[3];
                                    cart_comp(La, ia, ca);
                                    cart_comp(Lb, ib, cb);
                                    cart_comp(Lc, ic, cc);
                                    cart_comp(Ld, id, cd);
                                    double sum = 0.0;
                                    for (int t = 0; t <= ca[0] + cb[0]; ++t)
                                        for (int u = 0; u <= ca[1] + cb[1]; ++u)
                                            for (int v = 0; v <= ca[2] + cb[2]; ++v) {
                                                double eab = Eab[0].E[ca[0]][cb[0]][t] *
                                                             Eab[1].E[ca[1]][cb[1]][u] *
                                                             Eab[2].E[ca[2]][cb[2]][v];
                                                for (int tt = 0; tt <= cc[0] + cd[0]; ++tt)
                                                    for (int uu = 0; uu <= cc[1] + cd[1]; ++uu)
                                                        for (int vv = 0; vv <= cc[2] + cd[2]; ++vv) {
                                                            double ecd =
                                                                Ecd[0].E[cc[0]][cd[0]][tt] *
                                                                Ecd[1].E[cc[1]][cd[1]][uu] *
                                                                Ecd[2].E[cc[2]][cd[2]][vv];
                                                            double sgn =
                                                                ((tt + uu + vv) & 1) ? -1.0 : 1.0;
                                                            sum += eab * sgn * ecd *
                                                                   md_rtuv(&r, 0, t + tt, u + uu,
                                                                           v + vv);
                                                        }
                                            }
                                    out[((size_t)(ia * nb + ib) * nc + ic) * nd + id] +=
                                        pref * sum;
                                }
                }
    free(Eab);
    free(Ecd);
    free(r.val);
    free(r.done);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The paper's Rys route (Sec. II-C), a third cross-check of the readings     */
/* ------------------------------------------------------------------------- */

/* Gauss-Legendre rule on [-1, 1] with n points: Newton iteration on the Legendre polynomial
 * P_n from the three-term recurrence, weights 2 / ((1 - x^2) P_n'(x)^2). */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int k = 1; k <= n; ++k) {
                double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            double dz = p0 / dp;
            z -= dz;
            if (fabs(dz) < 1e-17)
                break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Eigenvalues of a symmetric n x n matrix (row major, destroyed) by cyclic Jacobi rotations. */
static void jacobi_eigenvalues(int n, double *a, double *ev)
{
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i) {
            diag += a[i * n + i] * a[i * n + i];
            for (int j = i + 1; j < n; ++j)
                off += a[i * n + j] * a[i * n + j];
        }
        if (off <= 1e-36 * diag)
            break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = a[p * n + q];
                if (apq == 0.0)
                    continue;
                double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) { /* columns p, q */
                    double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - sn * akq;
                    a[k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { /* rows p, q */
                    double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - sn * aqk;
                    a[q * n + k] = sn * apk + c * aqk;
                }
            }
    }
    for (int i = 0; i < n; ++i)
        ev[i] = a[i * n + i];
}

#define RYS_PANELS 8
#define RYS_GAUSS 32
#define RYS_NMAX 16

/* Rys roots x_mu = t_mu^2 in (0, 1) and weights w_mu > 0, mu = 1..n, at argument T: the n-point
 * Gauss rule of the measure on (0, 1) whose moments are the Boys values,
 * sum_mu w_mu x_mu^k = F_k(T) = int_0^1 t^{2k} exp(-T t^2) dt for k < 2n (Sec. II-C).
 * Here the measure is discretised by composite Gauss-Legendre in t on [0, b] (b = 1, or
 * 13 / sqrt(T) when smaller: beyond it exp(-T t^2) < 1e-73), its orthonormal polynomials are
 * generated by the Stieltjes procedure, the roots are the eigenvalues of their Jacobi matrix
 * and the weights the Christoffel numbers 1 / sum_k q_k(x_mu)^2.  Returns -1 if n is out of
 * range. */
int orc_rys_roots(int n, double T, double *x, double *w)
{
    if (n < 1 || n > RYS_NMAX || !(T >= 0.0))
        return -1;
    enum { M = RYS_PANELS * RYS_GAUSS };
    double gx[RYS_GAUSS], gw[RYS_GAUSS], nx[M], nw[M];
    gauss_legendre(RYS_GAUSS, gx, gw);
    double b = 1.0;
    if (T > 169.0)
        b = 13.0 / sqrt(T);
    double h = b / RYS_PANELS;
    for (int pnl = 0; pnl < RYS_PANELS; ++pnl)
        for (int g = 0; g < RYS_GAUSS; ++g) {
            double t = h * (pnl + 0.5 * (gx[g] + 1.0));
            nx[pnl * RYS_GAUSS + g] = t * t;
            nw[pnl * RYS_GAUSS + g] = 0.5 * h * gw[g] * exp(-T * t * t);
        }
    /* Stieltjes procedure with orthonormal polynomials q_k evaluated on the nodes */
    double q_prev[M], q_cur[M], alpha[RYS_NMAX], beta[RYS_NMAX + 1];
    double mass = 0.0;
    for (int j = 0; j < M; ++j)
        mass += nw[j];
    for (int j = 0; j < M; ++j) {
        q_prev[j] = 0.0;
        q_cur[j] = 1.0 / sqrt(mass);
    }
    beta[0] = 0.0;
    for (int k = 0; k < n; ++k) {
        double a = 0.0;
        for (int j = 0; j < M; ++j)
            a += nw[j] * nx[j] * q_cur[j] * q_cur[j];
        alpha[k] = a;
        double r[M], nrm = 0.0;
        for (int j = 0; j < M; ++j) {
            r[j] = (nx[j] - a) * q_cur[j] - beta[k] * q_prev[j];
            nrm += nw[j] * r[j] * r[j];
        }
        beta[k + 1] = sqrt(nrm);
        for (int j = 0; j < M; ++j) {
            q_prev[j] = q_cur[j];
            q_cur[j] = r[j] / beta[k + 1];
        }
    }
    /* Jacobi matrix: alpha on the diagonal, beta[1..n-1] beside it */
    double J[RYS_NMAX * RYS_NMAX];
    memset(J, 0, sizeof(J));
    for (int k = 0; k < n; ++k) {
        J[k * n + k] = alpha[k];
        if (k + 1 < n)
            J[k * n + k + 1] = J[(k + 1) * n + k] = beta[k + 1];
    }
    jacobi_eigenvalues(n, J, x);
    for (int mu = 0; mu < n; ++mu) { /* Christoffel numbers from the same recurrence */
        double qp = 0.0, qc = 1.0 / sqrt(mass), s = qc * qc;
        for (int k = 0; k + 1 < n; ++k) {
            double qn = ((x[mu] - alpha[k]) * qc - beta[k] * qp) / beta[k + 1];
            qp = qc;
            qc = qn;
            s += qc * qc;
        }
        w[mu] = 1.0 / s;
    }
    /* ascending roots */
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && x[j] < x[j - 1]; --j) {
            double tx = x[j]; x[j] = x[j - 1]; x[j - 1] = tx;
            double tw = w[j]; w[j] = w[j - 1]; w[j - 1] = tw;
        }
    return 0;
}

/* (ab|cd) of contracted shells by Rys quadrature, following Sec. II-C step by step:
 * per primitive quartet p = a + b, q = c + d, P, Q, rho = p q / (p + q), T = rho |P - Q|^2;
 * n_Rys = floor(L / 2) + 1 roots; per root the B and C coefficients of the standard Rys
 * definitions, B00 = x / (2(p+q)), B10 = (1 - q x / (p+q)) / (2p), B01 = (1 - p x / (p+q)) / (2q),
 * C00 = (P - A) - (q x / (p+q)) (P - Q), C00' = (Q - C) + (p x / (p+q)) (P - Q);
 * the 2-D integrals I(i, k) per Cartesian direction by the vertical recursion of Eq. 6 from
 * I(0, 0) = 1 (x and y) and I(0, 0) = 2 pi^{5/2} / (p q sqrt(p+q)) K_AB K_CD w_mu (z), the weight
 * counted once; the horizontal transfer of Eq. 7 to I(i, j, k, l) with A - B and C - D; the
 * quadrature of Eq. 8, sum over roots of Ix Iy Iz; and the sum over primitives with
 * c N(alpha, L) per shell. */
#define RYS_L 12
int orc_eri_quartet_rys(const orc_shell *sa, const orc_shell *sb, const orc_shell *sc,
                        const orc_shell *sd, double *out)
{
    int La = sa->L, Lb = sb->L, Lc = sc->L, Ld = sd->L;
    if (La < 0 || Lb < 0 || Lc < 0 || Ld < 0 || La + Lb > RYS_L || Lc + Ld > RYS_L)
        return -1;
    int na = ncart(La), nb = ncart(Lb), nc = ncart(Lc), nd = ncart(Ld);
    memset(out, 0, (size_t)na * nb * nc * nd * sizeof(double));
    int eh = La + Lb, fh = Lc + Ld, nrys = (La + Lb + Lc + Ld) / 2 + 1;
    const double *A = sa->center, *B = sb->center, *C = sc->center, *D = sd->center;
    /* 2-D integrals G[i][k] and the transferred H[i][j][k][l] of one direction */
    double G[RYS_L + 1][RYS_L + 1];
    double X[RYS_L + 1][RYS_L + 1][RYS_L + 1]; /* X[i][j][k]: bra transferred, k <= fh */
    double *H = (double *)malloc(sizeof(double) * 3 * (La + 1) * (Lb + 1) * (Lc + 1) * (Ld + 1));
    for (int i = 0; i < sa->nprim; ++i)
        for (int j = 0; j < sb->nprim; ++j)
            for (int k = 0; k < sc->nprim; ++k)
                for (int l = 0; l < sd->nprim; ++l) {
                    double ea = sa->exps[i], eb = sb->exps[j], ec = sc->exps[k], ed = sd->exps[l];
                    double cw = sa->coefs[i] * orc_norm(ea, La) * sb->coefs[j] * orc_norm(eb, Lb) *
                                sc->coefs[k] * orc_norm(ec, Lc) * sd->coefs[l] * orc_norm(ed, Ld);
                    double p = ea + eb, q = ec + ed, P[3], Q[3], AB2 = 0.0, CD2 = 0.0, PQ2 = 0.0;
                    for (int x = 0; x < 3; ++x) {
                        P[x] = (ea * A[x] + eb * B[x]) / p;
                        Q[x] = (ec * C[x] + ed * D[x]) / q;
                        AB2 += (A[x] - B[x]) * (A[x] - B[x]);
                        CD2 += (C[x] - D[x]) * (C[x] - D[x]);
                        PQ2 += (P[x] - Q[x]) * (P[x] - Q[x]);
                    }
                    double rho = p * q / (p + q), T = rho * PQ2;
                    double pref = 2.0 * pow(ORC_PI, 2.5) / (p * q * sqrt(p + q)) *
                                  exp(-ea * eb / p * AB2) * exp(-ec * ed / q * CD2);
                    double rt[RYS_NMAX], wt[RYS_NMAX];
                    orc_rys_roots(nrys, T, rt, wt);
                    for (int mu = 0; mu < nrys; ++mu) {
                        double x = rt[mu];
                        double B00 = x / (2.0 * (p + q));
                        double B10 = (1.0 - q * x / (p + q)) / (2.0 * p);
                        double B01 = (1.0 - p * x / (p + q)) / (2.0 * q);
                        for (int dir = 0; dir < 3; ++dir) {
                            double C00 = (P[dir] - A[dir]) - q * x / (p + q) * (P[dir] - Q[dir]);
                            double C00p = (Q[dir] - C[dir]) + p * x / (p + q) * (P[dir] - Q[dir]);
                            /* Eq. 6: first along k with i = 0, then along i for every k */
                            G[0][0] = dir == 2 ? pref * wt[mu] : 1.0;
                            for (int kk = 0; kk < fh; ++kk)
                                G[0][kk + 1] = kk * B01 * (kk > 0 ? G[0][kk - 1] : 0.0) +
                                               C00p * G[0][kk];
                            for (int ii = 0; ii < eh; ++ii)
                                for (int kk = 0; kk <= fh; ++kk)
                                    G[ii + 1][kk] = ii * B10 * (ii > 0 ? G[ii - 1][kk] : 0.0) +
                                                    kk * B00 * (kk > 0 ? G[ii][kk - 1] : 0.0) +
                                                    C00 * G[ii][kk];
                            /* Eq. 7 on the bra: X(i, j) = X(i+1, j-1) + (A - B) X(i, j-1) */
                            double ABd = A[dir] - B[dir], CDd = C[dir] - D[dir];
                            for (int kk = 0; kk <= fh; ++kk) {
                                for (int ii = 0; ii <= eh; ++ii)
                                    X[ii][0][kk] = G[ii][kk];
                                for (int jj = 1; jj <= Lb; ++jj)
                                    for (int ii = 0; ii <= eh - jj; ++ii)
                                        X[ii][jj][kk] = X[ii + 1][jj - 1][kk] + ABd * X[ii][jj - 1][kk];
                            }
                            /* Eq. 7 on the ket, per (i <= La, j <= Lb) */
                            for (int ii = 0; ii <= La; ++ii)
                                for (int jj = 0; jj <= Lb; ++jj) {
                                    double Y[RYS_L + 1][RYS_L + 1];
                                    for (int kk = 0; kk <= fh; ++kk)
                                        Y[kk][0] = X[ii][jj][kk];
                                    for (int ll = 1; ll <= Ld; ++ll)
                                        for (int kk = 0; kk <= fh - ll; ++kk)
                                            Y[kk][ll] = Y[kk + 1][ll - 1] + CDd * Y[kk][ll - 1];
                                    for (int kk = 0; kk <= Lc; ++kk)
                                        for (int ll = 0; ll <= Ld; ++ll)
                                            H[(((dir * (La + 1) + ii) * (Lb + 1) + jj) * (Lc + 1) + kk) *
                                                  (Ld + 1) + ll] = Y[kk][ll];
                                }
                        }
                        /* Eq. 8: one term of the quadrature per root */
#define HIDX(dir, a, b, c, d) \
    H[((((dir) * (La + 1) + (a)) * (Lb + 1) + (b)) * (Lc + 1) + (c)) * (Ld + 1) + (d)]
                        for (int ia = 0; ia < na; ++ia)
                            for (int ib = 0; ib < nb; ++ib)
                                for (int ic = 0; ic < nc; ++ic)
                                    for (int id = 0; id < nd; ++id) {
                                        int ca[3], cb[3], cc[3], cd[3];
                                        cart_comp(La, ia, ca);
                                        cart_comp(Lb, ib, cb);
                                        cart_comp(Lc, ic, cc);
                                        cart_comp(Ld, id, cd);
                                        double v = HIDX(0, ca[0], cb[0], cc[0], cd[0]) *
                                                   HIDX(1, ca[1], cb[1], cc[1], cd[1]) *
                                                   HIDX(2, ca[2], cb[2], cc[2], cd[2]);
                                        out[((size_t)(ia * nb + ib) * nc + ic) * nd + id] += cw * v;
                                    }
#undef HIDX
                    }
                }
    free(H);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Gradients of E = sum_abcd G_abcd (ab|cd)                                   */
/* ------------------------------------------------------------------------- */

/* d g_a / d A_xi = 2 alpha g~_{a+1_xi} - a_xi g~_{a-1_xi}   (same normalisation N(alpha, L_a))
 * d g_a / d alpha = (2 L_a + 3)/(4 alpha) g_a - sum_xi g~_{a+2_xi}
 * where g~ carries the coefficient and normalisation of the unshifted function.
 *
 * For one shell quartet and upstream G (row-major like the ERIs), adds
 *   dR[4][3] : dE/d(centre) of shells a, b, c, d,
 *   dalpha_x[k] : dE/d(alpha_k) for primitive k of shell x (x = a, b, c, d).
 * The caller zeroes the outputs. */
typedef struct {
    int La, Lb, Lc, Ld;
    const double *A, *B, *C, *D;
} grad_geom;

/* Contracted table accumulation with a per-primitive weight callback:
 * tab += sum_prims w(prims) [e0|f0]. */
static void shifted_eri(const orc_shell *s[4], int shift_shell, int shift_dL, int only_prim,
                        int weight_kind, double *out)
{
    /* weight_kind: 0 -> c N products;  1 -> c N products * 2 alpha(shift shell prim) */
    int L[4] = {s[0]->L, s[1]->L, s[2]->L, s[3]->L};
    int Ls[4] = {L[0], L[1], L[2], L[3]};
    Ls[shift_shell] += shift_dL;
    int e_hi = Ls[0] + Ls[1], f_hi = Ls[2] + Ls[3];
    size_t ntab = (size_t)ntrip(e_hi) * ntrip(f_hi);
    double *tab = (double *)calloc(ntab, sizeof(double));
    for (int i = 0; i < s[0]->nprim; ++i)
        for (int j = 0; j < s[1]->nprim; ++j)
            for (int k = 0; k < s[2]->nprim; ++k)
                for (int l = 0; l < s[3]->nprim; ++l) {
                    int idx[4] = {i, j, k, l};
                    if (only_prim >= 0 && idx[shift_shell] != only_prim)
                        continue;
                    double w = 1.0;
                    for (int x = 0; x < 4; ++x)
                        w *= s[x]->coefs[idx[x]] * orc_norm(s[x]->exps[idx[x]], L[x]);
                    if (weight_kind == 1)
                        w *= 2.0 * s[shift_shell]->exps[idx[shift_shell]];
                    vrr_prim_accumulate(s[0]->center, s[0]->exps[i], s[1]->center,
                                        s[1]->exps[j], s[2]->center, s[2]->exps[k], s[3]->center,
                                        s[3]->exps[l], e_hi, f_hi, w, tab);
                }
    hrr_shells(tab, e_hi, f_hi, s[0]->center, s[1]->center, s[2]->center, s[3]->center, Ls[0],
               Ls[1], Ls[2], Ls[3], out);
    free(tab);
}

/* index of component tuple in a shell-quartet array with shell angular momenta Ls */
static size_t quartet_index(const int Ls[4], int comp[4][3])
{
    size_t idx = 0;
    for (int x = 0; x < 4; ++x)
        idx = idx * ncart(Ls[x]) + cart_index(comp[x][0], comp[x][1], comp[x][2]);
    return idx;
}

int orc_eri_grad_quartet(const orc_shell *sa, const orc_shell *sb, const orc_shell *sc,
                         const orc_shell *sd, const double *G, double *dR /* [4][3] */,
                         double *da, double *db, double *dc, double *dd)
{
    const orc_shell *s[4] = {sa, sb, sc, sd};
    double *dalpha[4] = {da, db, dc, dd};
    int L[4] = {sa->L, sb->L, sc->L, sd->L};
    int n[4] = {ncart(L[0]), ncart(L[1]), ncart(L[2]), ncart(L[3])};
    size_t nout = (size_t)n[0] * n[1] * n[2] * n[3];
    for (int x = 0; x < 4; ++x) {
        int Lp[4] = {L[0], L[1], L[2], L[3]};
        Lp[x] += 1;
        size_t np = (size_t)ncart(Lp[0]) * ncart(Lp[1]) * ncart(Lp[2]) * ncart(Lp[3]);
        double *plus = (double *)malloc(np * sizeof(double));
        shifted_eri(s, x, +1, -1, 1, plus);
        double *minus = NULL;
        int Lm[4] = {L[0], L[1], L[2], L[3]};
        Lm[x] -= 1;
        if (L[x] > 0) {
            size_t nm = (size_t)ncart(Lm[0]) * ncart(Lm[1]) * ncart(Lm[2]) * ncart(Lm[3]);
            minus = (double *)malloc(nm * sizeof(double));
            shifted_eri(s, x, -1, -1, 0, minus);
        }
        for (size_t o = 0; o < nout; ++o) {
            if (G[o] == 0.0)
                continue;
            int comp[4][3];
            size_t r = o;
            for (int y = 3; y >= 0; --y) {
                cart_comp(L[y], (int)(r % n[y]), comp[y]);
                r /= n[y];
            }
            for (int xi = 0; xi < 3; ++xi) {
                int cp[4][3];
                memcpy(cp, comp, sizeof(cp));
                cp[x][xi] += 1;
                double g = plus[quartet_index(Lp, cp)];
                if (comp[x][xi] > 0) {
                    int cm[4][3];
                    memcpy(cm, comp, sizeof(cm));
                    cm[x][xi] -= 1;
                    g -= comp[x][xi] * minus[quartet_index(Lm, cm)];
                }
                dR[x * 3 + xi] += G[o] * g;
            }
        }
        free(plus);
        free(minus);
        /* exponent derivatives, one primitive at a time */
        int L2[4] = {L[0], L[1], L[2], L[3]};
        L2[x] += 2;
        size_t n2 = (size_t)ncart(L2[0]) * ncart(L2[1]) * ncart(L2[2]) * ncart(L2[3]);
        double *p2 = (double *)malloc(n2 * sizeof(double));
        double *base = (double *)malloc(nout * sizeof(double));
        for (int k = 0; k < s[x]->nprim; ++k) {
            shifted_eri(s, x, +2, k, 0, p2);
            shifted_eri(s, x, 0, k, 0, base);
            double alpha = s[x]->exps[k];
            double acc = 0.0;
            for (size_t o = 0; o < nout; ++o) {
                if (G[o] == 0.0)
                    continue;
                int comp[4][3];
                size_t r = o;
                for (int y = 3; y >= 0; --y) {
                    cart_comp(L[y], (int)(r % n[y]), comp[y]);
                    r /= n[y];
                }
                double g = (2.0 * L[x] + 3.0) / (4.0 * alpha) * base[o];
                for (int xi = 0; xi < 3; ++xi) {
                    int cp[4][3];
                    memcpy(cp, comp, sizeof(cp));
                    cp[x][xi] += 2;
                    g -= p2[quartet_index(L2, cp)];
                }
                acc += G[o] * g;
            }
            dalpha[x][k] += acc;
        }
        free(p2);
        free(base);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Batched drivers over a shell table (structure of arrays)                  */
/* ------------------------------------------------------------------------- */

typedef struct {
    const double *centers; /* [n_shells][3] */
    const int32_t *L;      /* [n_shells] */
    const int32_t *nprim;  /* [n_shells] */
    const int64_t *pofs;   /* [n_shells] offset into exps/coefs */
    const double *exps;
    const double *coefs;
} orc_table;

static void table_shell(const orc_table *t, int32_t i, orc_shell *s)
{
    s->center[0] = t->centers[3 * (size_t)i];
    s->center[1] = t->centers[3 * (size_t)i + 1];
    s->center[2] = t->centers[3 * (size_t)i + 2];
    s->L = t->L[i];
    s->nprim = t->nprim[i];
    s->exps = t->exps + t->pofs[i];
    s->coefs = t->coefs + t->pofs[i];
}

/* ERIs of n_quartets shell quartets; quartet q writes at out + offsets[q].  method 0 = OS/HGP,
 * 1 = McMurchie-Davidson, 2 = the paper's Rys route (cross-check).  nthreads <= 0 uses the OpenMP default.  Returns 0 on success. */
int orc_eri_batch(const double *centers, const int32_t *L, const int32_t *nprim,
                  const int64_t *pofs, const double *exps, const double *coefs,
                  const int32_t *quartets, int64_t n_quartets, const int64_t *offsets,
                  double *out, int method, int nthreads)
{
    orc_table t = {centers, L, nprim, pofs, exps, coefs};
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) reduction(| : err)
#endif
    for (int64_t q = 0; q < n_quartets; ++q) {
        orc_shell s[4];
        for (int x = 0; x < 4; ++x)
            table_shell(&t, quartets[4 * q + x], &s[x]);
        int rc = method == 0   ? orc_eri_quartet(&s[0], &s[1], &s[2], &s[3], out + offsets[q])
                 : method == 1 ? orc_eri_quartet_md(&s[0], &s[1], &s[2], &s[3], out + offsets[q])
                               : orc_eri_quartet_rys(&s[0], &s[1], &s[2], &s[3], out + offsets[q]);
        err |= (rc != 0);
    }
    return err ? -1 : 0;
}

/* Gradient of E = sum_q sum_abcd G[q]_abcd (ab|cd)_q.  G of quartet q starts at G + offsets[q].
 * dR: [n_shells][3], dalpha: [total primitives] (indexed like exps).  Outputs are accumulated;
 * runs single threaded so that the accumulation order is fixed. */
int orc_eri_grad_batch(const double *centers, const int32_t *L, const int32_t *nprim,
                       const int64_t *pofs, const double *exps, const double *coefs,
                       const int32_t *quartets, int64_t n_quartets, const int64_t *offsets,
                       const double *G, double *dR, double *dalpha)
{
    orc_table t = {centers, L, nprim, pofs, exps, coefs};
    for (int64_t q = 0; q < n_quartets; ++q) {
        orc_shell s[4];
        int32_t id[4];
        for (int x = 0; x < 4; ++x) {
            id[x] = quartets[4 * q + x];
            table_shell(&t, id[x], &s[x]);
        }
        double r[12] = {0};
        double *da[4];
        for (int x = 0; x < 4; ++x)
            da[x] = (double *)calloc((size_t)s[x].nprim, sizeof(double));
        orc_eri_grad_quartet(&s[0], &s[1], &s[2], &s[3], G + offsets[q], r, da[0], da[1], da[2],
                             da[3]);
        for (int x = 0; x < 4; ++x) {
            for (int xi = 0; xi < 3; ++xi)
                dR[3 * (size_t)id[x] + xi] += r[3 * x + xi];
            for (int k = 0; k < s[x].nprim; ++k)
                dalpha[pofs[id[x]] + k] += da[x][k];
            free(da[x]);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Coulomb and exchange digestion of ERI blocks                               */
/* ------------------------------------------------------------------------- */

/* What the ERIs, and their compressed copies, are computed for (Sec. I: the Hartree-Fock
 * exchange of hybrid DFT in AIMD; Sec. II-D: ERIs kept compressed in memory between uses) is
 * their contraction with a density matrix D.  For every listed shell quartet (a b | c d), with
 * its ERI block x laid out as eri_batch writes it, and basis functions mu of a, nu of b, lam of
 * c, sig of d:
 *   J[mu][nu]  += sum_{lam, sig} (mu nu | lam sig) D[lam][sig]   (Coulomb)
 *   K[mu][lam] += sum_{nu, sig}  (mu nu | lam sig) D[nu][sig]    (exchange)
 * Every listed quartet counts once, as listed: no permutation of it is implied.  bf_off[s] is the
 * first basis function of shell s; D, J and K are n_bf x n_bf, row major; J and K accumulate. */
void orc_digest_jk(const double *x, const int64_t *offsets, const int32_t *quartets,
                   int64_t n_quartets, const int32_t *L, const int64_t *bf_off, int64_t n_bf,
                   const double *D, double *J, double *K)
{
    for (int64_t q = 0; q < n_quartets; ++q) {
        const int32_t *s = quartets + 4 * q;
        int n[4];
        int64_t o[4];
        for (int i = 0; i < 4; ++i) {
            n[i] = ncart(L[s[i]]);
            o[i] = bf_off[s[i]];
        }
        const double *v = x + offsets[q];
        for (int a = 0; a < n[0]; ++a)
            for (int b = 0; b < n[1]; ++b)
                for (int c = 0; c < n[2]; ++c)
                    for (int d = 0; d < n[3]; ++d) {
                        double e = v[((a * n[1] + b) * n[2] + c) * n[3] + d];
                        int64_t mu = o[0] + a, nu = o[1] + b, lam = o[2] + c, sig = o[3] + d;
                        J[mu * n_bf + nu] += e * D[lam * n_bf + sig];
                        K[mu * n_bf + lam] += e * D[nu * n_bf + sig];
                    }
    }
}

/* ------------------------------------------------------------------------- */
/* Compression (Sec. II-D, Eqs. 9-11)                                        */
/* ------------------------------------------------------------------------- */

/* ANINT: nearest integer, halves away from zero */
static double anint(double x) { return x >= 0.0 ? floor(x + 0.5) : -floor(-x + 0.5); }

/* One quartet of n values -> n-bit integers q and scale eps.
 *   b_max = max |x|, M = 2^{bits-1} - 1, eps = b_max / M (Eq. 9) rounded to FP32 for storage,
 *   q = ANINT(x / eps) (Eq. 10) with the stored eps, clamped to [-M, M].
 * b_max = 0 gives eps = 0 and q = 0.  Supported widths are 2..24: eps has a 24-bit
 * significand, so for wider codes its rounding alone can move b_max / eps past M + 1/2. */
void orc_compress_quartet(const double *x, int64_t n, int bits, int32_t *q, float *eps)
{
    double bmax = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (fabs(x[i]) > bmax)
            bmax = fabs(x[i]);
    double M = ldexp(1.0, bits - 1) - 1.0;
    float e = (float)(bmax / M);
    *eps = e;
    for (int64_t i = 0; i < n; ++i) {
        if (e == 0.0f) {
            q[i] = 0;
            continue;
        }
        double v = anint(x[i] / (double)e);
        if (v > M)
            v = M;
        if (v < -M)
            v = -M;
        q[i] = (int32_t)v;
    }
}

/* Eq. 11 */
void orc_decompress_quartet(const int32_t *q, int64_t n, float eps, double *x)
{
    for (int64_t i = 0; i < n; ++i)
        x[i] = (double)q[i] * (double)eps;
}

/* Little-endian, least-significant-bit-first bitstream of count n-bit two's complement fields:
 * field v occupies stream bits [v*bits, v*bits + bits); stream bit s is bit (s % 32) of 32-bit
 * word s / 32.  words must hold ceil(count*bits/32) entries and is overwritten. */
void orc_pack_bits(const int32_t *q, int64_t count, int bits, uint32_t *words)
{
    int64_t nw = (count * bits + 31) / 32;
    memset(words, 0, (size_t)nw * sizeof(uint32_t));
    uint64_t mask = (bits == 32) ? 0xffffffffull : ((1ull << bits) - 1ull);
    for (int64_t v = 0; v < count; ++v) {
        uint64_t code = (uint64_t)(uint32_t)q[v] & mask;
        for (int b = 0; b < bits; ++b) {
            int64_t s = v * bits + b;
            if ((code >> b) & 1ull)
                words[s / 32] |= (uint32_t)1u << (s % 32);
        }
    }
}

void orc_unpack_bits(const uint32_t *words, int64_t count, int bits, int32_t *q)
{
    for (int64_t v = 0; v < count; ++v) {
        uint32_t code = 0;
        for (int b = 0; b < bits; ++b) {
            int64_t s = v * bits + b;
            if ((words[s / 32] >> (s % 32)) & 1u)
                code |= (uint32_t)1u << b;
        }
        /* sign extension of an n-bit field */
        if (bits < 32 && (code >> (bits - 1)) & 1u)
            code |= ~((1u << bits) - 1u);
        q[v] = (int32_t)code;
    }
}

/* The paper's output chunks (Sec. III-C, compress-store loops): the ERIs of each quartet are
 * written as 512-bit words, each holding F = floor(512/bits) n-bit fields; ERIs that do not fit
 * into the current chunk are carried over and written first into the next one, and the last
 * chunk of a quartet is padded, so a quartet takes n_CS = ceil(n_eri / F) chunks and no chunk
 * holds ERIs of two quartets.  Field j of a chunk occupies chunk bits [j*bits, j*bits + bits),
 * chunk bit s being bit (s % 32) of 32-bit word s / 32 of the chunk (the paper does not fix the
 * bit order inside a chunk; this one matches the dense stream).  Unused bits are zero.
 * q holds n_quartets * n_eri codes, quartet after quartet; words must hold
 * n_quartets * n_CS * 16 entries and is overwritten. */
void orc_pack_paper512(const int32_t *q, int64_t n_quartets, int64_t n_eri, int bits,
                       uint32_t *words)
{
    int64_t F = 512 / bits;
    int64_t n_cs = (n_eri + F - 1) / F;
    memset(words, 0, (size_t)(n_quartets * n_cs * 16) * sizeof(uint32_t));
    uint64_t mask = (bits == 32) ? 0xffffffffull : ((1ull << bits) - 1ull);
    for (int64_t i = 0; i < n_quartets; ++i) {
        int64_t chunk = 0, field = 0; /* position of the next field within the quartet */
        for (int64_t e = 0; e < n_eri; ++e) {
            if (field == F) { /* chunk full: the remaining ERIs go to the next chunk */
                ++chunk;
                field = 0;
            }
            uint32_t *z = words + (i * n_cs + chunk) * 16;
            uint64_t code = (uint64_t)(uint32_t)q[i * n_eri + e] & mask;
            for (int b = 0; b < bits; ++b) {
                int64_t s = field * bits + b;
                if ((code >> b) & 1ull)
                    z[s / 32] |= (uint32_t)1u << (s % 32);
            }
            ++field;
        }
    }
}

void orc_unpack_paper512(const uint32_t *words, int64_t n_quartets, int64_t n_eri, int bits,
                         int32_t *q)
{
    int64_t F = 512 / bits;
    int64_t n_cs = (n_eri + F - 1) / F;
    for (int64_t i = 0; i < n_quartets; ++i)
        for (int64_t e = 0; e < n_eri; ++e) {
            const uint32_t *z = words + (i * n_cs + e / F) * 16;
            int64_t field = e % F;
            uint32_t code = 0;
            for (int b = 0; b < bits; ++b) {
                int64_t s = field * bits + b;
                if ((z[s / 32] >> (s % 32)) & 1u)
                    code |= (uint32_t)1u << b;
            }
            if (bits < 32 && (code >> (bits - 1)) & 1u)
                code |= ~((1u << bits) - 1u);
            q[i * n_eri + e] = (int32_t)code;
        }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
