/*
 * fmm_oracle.c -- plain, slow, FP64 CPU reference for the periodic fast
 * multipole method with a uniform neutralising background charge
 * (Urano, Shinoda, Yoshii & Okazaki, arXiv:2003.13218).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library.  The CUDA library shares
 * no code, header, table or constant with it.
 *
 * Two parts:
 *   O1  oracle_ewald  -- the definition: Ewald sum of point charges plus the
 *       background charge under the conducting boundary (Appendix A: real
 *       term, reciprocal term over k != 0, self term, charged-system term).
 *   O2  oracle_fmm*   -- the algorithm, step by step in the paper's order and
 *       notation (Appendix B): leaf assignment, P2M (Eq. P2M), M2M, the
 *       lattice sum at level 0 (Eq. 12 with its self term), M2L over each
 *       level's interaction list (Eq. Lcoeffdef), L2L and merge, L2P and the
 *       far-field energy (Eq. EqFF), the near-field pair sum (Eq. EqNF) and
 *       the background-charge terms of Eq. Velecfull; forces are the exact
 *       gradient of that energy; the solute-solvent energy follows
 *       Eq. FMMcalc.
 *
 * Conventions (the paper leaves the normalisation to the cited solid-harmonic
 * literature; this one makes Eq. P2M, Eq. Lcoeffdef and Eq. EqFF hold exactly
 * as printed, with no conjugates):
 *   R_n^m(r) = r^n P_n^m(cos t) e^{i m phi} / (n+m)!
 *   I_n^m(r) = (-1)^(n+m) (n-m)! P_n^m(cos t) e^{i m phi} / r^(n+1)
 * with P_n^m the associated Legendre function including the Condon-Shortley
 * phase, P_n^{-m} = (-1)^m (n-m)!/(n+m)! P_n^m.  Then
 *   1/|D + y| = sum_{N,M} R_N^M(y) I_N^{-M}(D)   (|y| < |D|),
 *   R_N^M(a + b) = sum_{n,m} R_n^m(a) R_{N-n}^{M-m}(b).
 * Coefficients are stored as full complex arrays, index n*n + n + m.
 *
 * Readings of the paper used here (see the design notes):
 *  - the reciprocal sum of Eq. 12 runs over k != 0 (the k = 0 part is the
 *    background-charge analysis that yields Eq. 6 and Eq. surfchargedend);
 *  - the level-0 lattice operator covers the images outside the
 *    (2 ws + 1)^3 block of image cells around the unit cell; the block itself
 *    is covered by the M2L of levels 1..l_max and the near field, whose
 *    stencils wrap periodically;
 *  - the interaction list of a cell at level l: children of the parent's
 *    (2 ws + 1)^3 neighbours that are not its own neighbours;
 *  - the signs of the background-charge block follow Eq. Velecfull.
 *
 * Compile: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define HIDX(n, m) ((n) * (n) + (n) + (m))
#define NCOEF(p) (((p) + 1) * ((p) + 1))

static const double PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* factorials                                                                */
/* ------------------------------------------------------------------------ */
static double factorial(int n)
{
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= (double)k;
    return f;
}

/* ------------------------------------------------------------------------ */
/* associated Legendre functions P_n^m(x), 0 <= m <= n <= pmax, with the     */
/* Condon-Shortley phase; s = sqrt(1 - x^2) >= 0.  Textbook recurrences:     */
/*   P_m^m = -(2m-1) s P_{m-1}^{m-1},  P_{m+1}^m = (2m+1) x P_m^m,           */
/*   (n-m) P_n^m = (2n-1) x P_{n-1}^m - (n+m-1) P_{n-2}^m.                   */
/* ------------------------------------------------------------------------ */
static void legendre(int pmax, double x, double s, double *P /* [(pmax+1)^2] */)
{
    int W = pmax + 1;
    for (int i = 0; i < W * W; ++i) P[i] = 0.0;
    P[0] = 1.0;
    for (int m = 1; m <= pmax; ++m) P[m * W + m] = -(2.0 * m - 1.0) * s * P[(m - 1) * W + (m - 1)];
    for (int m = 0; m < pmax; ++m) P[(m + 1) * W + m] = (2.0 * m + 1.0) * x * P[m * W + m];
    for (int m = 0; m <= pmax; ++m)
        for (int n = m + 2; n <= pmax; ++n)
            P[n * W + m] = ((2.0 * n - 1.0) * x * P[(n - 1) * W + m] - (n + m - 1.0) * P[(n - 2) * W + m]) / (double)(n - m);
}

static void spherical(const double v[3], double *r, double *c, double *s, cplx *eiphi)
{
    double rho = sqrt(v[0] * v[0] + v[1] * v[1]);
    *r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (*r > 0.0) {
        *c = v[2] / *r;
        *s = rho / *r;
    } else {
        *c = 1.0;
        *s = 0.0;
    }
    *eiphi = rho > 0.0 ? (v[0] + I * v[1]) / rho : 1.0;
}

/* regular solid harmonics R_n^m(v), n <= p, all m */
void oracle_regular(int p, const double v[3], cplx *R)
{
    double r, c, s;
    cplx e;
    spherical(v, &r, &c, &s, &e);
    double *P = malloc(sizeof(double) * NCOEF(p));
    legendre(p, c, s, P);
    for (int n = 0; n <= p; ++n) {
        double rn = pow(r, n);
        for (int m = 0; m <= n; ++m) {
            cplx val = rn * P[n * (p + 1) + m] * cpow(e, m) / factorial(n + m);
            R[HIDX(n, m)] = val;
            if (m > 0) R[HIDX(n, -m)] = ((m & 1) ? -1.0 : 1.0) * conj(val);
        }
    }
    free(P);
}

/* irregular solid harmonics I_n^m(v), n <= pmax, all m (v != 0) */
void oracle_irregular(int pmax, const double v[3], cplx *Iv)
{
    double r, c, s;
    cplx e;
    spherical(v, &r, &c, &s, &e);
    double *P = malloc(sizeof(double) * NCOEF(pmax));
    legendre(pmax, c, s, P);
    for (int n = 0; n <= pmax; ++n) {
        double rinv = 1.0 / pow(r, n + 1);
        for (int m = 0; m <= n; ++m) {
            double sign = ((n + m) & 1) ? -1.0 : 1.0;
            cplx val = sign * factorial(n - m) * P[n * (pmax + 1) + m] * cpow(e, m) * rinv;
            Iv[HIDX(n, m)] = val;
            if (m > 0) Iv[HIDX(n, -m)] = ((m & 1) ? -1.0 : 1.0) * conj(val);
        }
    }
    free(P);
}

/* ------------------------------------------------------------------------ */
/* the five FMM operators of Appendix B                                      */
/* ------------------------------------------------------------------------ */

/* Eq. P2M: M_n^m += sum_j q_j R_n^m(r_M - r_j) */
void oracle_p2m(int p, int n_src, const double *src, const double *q, const double centre[3], cplx *M)
{
    cplx *R = malloc(sizeof(cplx) * NCOEF(p));
    for (int j = 0; j < n_src; ++j) {
        double v[3] = {centre[0] - src[3 * j], centre[1] - src[3 * j + 1], centre[2] - src[3 * j + 2]};
        oracle_regular(p, v, R);
        for (int i = 0; i < NCOEF(p); ++i) M[i] += q[j] * R[i];
    }
    free(R);
}

/* M2M (Appendix B, "translational shift" of child moments to the parent
 * centre): M_n^m(P) += sum_{k,l} R_{n-k}^{m-l}(r_P - r_C) M_k^l(C) */
void oracle_m2m(int p, const cplx *Mc, const double child[3], const double parent[3], cplx *Mp)
{
    cplx *R = malloc(sizeof(cplx) * NCOEF(p));
    double v[3] = {parent[0] - child[0], parent[1] - child[1], parent[2] - child[2]};
    oracle_regular(p, v, R);
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx acc = 0.0;
            for (int k = 0; k <= n; ++k)
                for (int l = -k; l <= k; ++l) {
                    int dm = m - l, dn = n - k;
                    if (dm < -dn || dm > dn) continue;
                    acc += R[HIDX(dn, dm)] * Mc[HIDX(k, l)];
                }
            Mp[HIDX(n, m)] += acc;
        }
    free(R);
}

/* Eq. Lcoeffdef: Lbar_n^m += sum_{lambda<=p, eta} M_lambda^eta I_{n+lambda}^{-(m+eta)}(r_L - r_M)
 * with the irregular harmonics I given for degrees 0..2p */
static void m2l_with(int p, const cplx *M, const cplx *Iv, cplx *L)
{
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx acc = 0.0;
            for (int lam = 0; lam <= p; ++lam)
                for (int eta = -lam; eta <= lam; ++eta)
                    acc += M[HIDX(lam, eta)] * Iv[HIDX(n + lam, -(m + eta))];
            L[HIDX(n, m)] += acc;
        }
}

void oracle_m2l(int p, const cplx *M, const double src_centre[3], const double tgt_centre[3], cplx *L)
{
    cplx *Iv = malloc(sizeof(cplx) * NCOEF(2 * p));
    double v[3] = {tgt_centre[0] - src_centre[0], tgt_centre[1] - src_centre[1], tgt_centre[2] - src_centre[2]};
    oracle_irregular(2 * p, v, Iv);
    m2l_with(p, M, Iv, L);
    free(Iv);
}

/* L2L (Appendix B): Lunder_k^l(C) += sum_{n>=k, m} L_n^m(P) R_{n-k}^{m-l}(r_C - r_P) */
void oracle_l2l(int p, const cplx *Lp, const double parent[3], const double child[3], cplx *Lc)
{
    cplx *R = malloc(sizeof(cplx) * NCOEF(p));
    double v[3] = {child[0] - parent[0], child[1] - parent[1], child[2] - parent[2]};
    oracle_regular(p, v, R);
    for (int k = 0; k <= p; ++k)
        for (int l = -k; l <= k; ++l) {
            cplx acc = 0.0;
            for (int n = k; n <= p; ++n)
                for (int m = -n; m <= n; ++m) {
                    int dn = n - k, dm = m - l;
                    if (dm < -dn || dm > dn) continue;
                    acc += Lp[HIDX(n, m)] * R[HIDX(dn, dm)];
                }
            Lc[HIDX(k, l)] += acc;
        }
    free(R);
}

/* L2P (Eq. EqFF): Phi(r) = sum_{n,m} L_n^m R_n^m(r - r_L'), and its gradient
 * from  d/dz R_n^m = R_{n-1}^m,
 *       d/dx R_n^m = (R_{n-1}^{m+1} - R_{n-1}^{m-1}) / 2,
 *       d/dy R_n^m = -i (R_{n-1}^{m+1} + R_{n-1}^{m-1}) / 2,
 * which follow from the addition theorem with a first-order shift. */
void oracle_l2p(int p, const cplx *L, const double centre[3], const double r[3], double *phi, double grad[3])
{
    cplx *R = malloc(sizeof(cplx) * NCOEF(p));
    double v[3] = {r[0] - centre[0], r[1] - centre[1], r[2] - centre[2]};
    oracle_regular(p, v, R);
    cplx f = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            f += L[HIDX(n, m)] * R[HIDX(n, m)];
            if (n == 0) continue;
            cplx up = (m + 1 <= n - 1) ? R[HIDX(n - 1, m + 1)] : 0.0;
            cplx dn = (m - 1 >= -(n - 1)) ? R[HIDX(n - 1, m - 1)] : 0.0;
            cplx mid = (m <= n - 1 && m >= -(n - 1)) ? R[HIDX(n - 1, m)] : 0.0;
            gx += L[HIDX(n, m)] * 0.5 * (up - dn);
            gy += L[HIDX(n, m)] * (-0.5 * I) * (up + dn);
            gz += L[HIDX(n, m)] * mid;
        }
    *phi = creal(f);
    if (grad) {
        grad[0] = creal(gx);
        grad[1] = creal(gy);
        grad[2] = creal(gz);
    }
    free(R);
}

/* ------------------------------------------------------------------------ */
/* Eq. 12: lattice sum of I_j^k over image cells nu != 0, Ewald split into   */
/* real (12a), reciprocal over k != 0 (12b) and self (12c) terms; then the   */
/* (2ws+1)^3 block of near images is taken out (it is covered by the M2L of  */
/* levels 1..l_max and the near field).                                      */
/* Regularised upper incomplete gamma Q(a, x) = Gamma(a, x)/Gamma(a) for     */
/* a = j + 1/2 from Q(1/2, x) = erfc(sqrt x) and the textbook recurrence     */
/* Gamma(a+1, x) = a Gamma(a, x) + x^a e^{-x}.                               */
/* ------------------------------------------------------------------------ */
static double gamma_half(int j) /* Gamma(j + 1/2) */
{
    double g = sqrt(PI);
    for (int i = 0; i < j; ++i) g *= (i + 0.5);
    return g;
}

static void q_half_all(int jmax, double x, double *Q)
{
    Q[0] = erfc(sqrt(x));
    for (int j = 0; j < jmax; ++j) {
        double a = j + 0.5;
        Q[j + 1] = Q[j] + pow(x, a) * exp(-x) / gamma_half(j + 1);
    }
}

/* S[HIDX(j,k)] for j <= jmax; b = box side, kappa = splitting parameter */
void oracle_lattice(int jmax, double b, double kappa, int ws, int nu_max, int n_kmax, cplx *S)
{
    int NC = NCOEF(jmax);
    double V = b * b * b;
    cplx *real = calloc(NC, sizeof(cplx));
    cplx *recip = calloc(NC, sizeof(cplx));
    cplx *block = calloc(NC, sizeof(cplx));
    cplx *Iv = malloc(sizeof(cplx) * NC);
    double *Q = malloc(sizeof(double) * (jmax + 1));
    /* (12a) real-space term over nu != 0 */
    for (int nx = -nu_max; nx <= nu_max; ++nx)
        for (int ny = -nu_max; ny <= nu_max; ++ny)
            for (int nz = -nu_max; nz <= nu_max; ++nz) {
                if (nx == 0 && ny == 0 && nz == 0) continue;
                double v[3] = {nx * b, ny * b, nz * b};
                double r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                oracle_irregular(jmax, v, Iv);
                q_half_all(jmax, kappa * kappa * r2, Q);
                for (int j = 0; j <= jmax; ++j)
                    for (int k = -j; k <= j; ++k) real[HIDX(j, k)] += Iv[HIDX(j, k)] * Q[j];
                if (abs(nx) <= ws && abs(ny) <= ws && abs(nz) <= ws)
                    for (int i = 0; i < NC; ++i) block[i] += Iv[i];
            }
    /* (12b) reciprocal term over k != 0, k = 2 pi n / b */
    for (int nx = -n_kmax; nx <= n_kmax; ++nx)
        for (int ny = -n_kmax; ny <= n_kmax; ++ny)
            for (int nz = -n_kmax; nz <= n_kmax; ++nz) {
                if (nx == 0 && ny == 0 && nz == 0) continue;
                double kv[3] = {2 * PI * nx / b, 2 * PI * ny / b, 2 * PI * nz / b};
                double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
                double kk = sqrt(k2);
                oracle_irregular(jmax, kv, Iv);
                double g = exp(-k2 / (4 * kappa * kappa));
                for (int j = 0; j <= jmax; ++j)
                    for (int k = -j; k <= j; ++k) recip[HIDX(j, k)] += Iv[HIDX(j, k)] * pow(kk, 2 * j - 1) * g;
            }
    for (int j = 0; j <= jmax; ++j) {
        cplx ij = cpow(I, j);
        double pref = pow(PI, 1.5) / (pow(2.0, j - 2) * gamma_half(j) * V);
        for (int k = -j; k <= j; ++k) {
            cplx val = real[HIDX(j, k)] + pref * ij * recip[HIDX(j, k)];
            if (j == 0 && k == 0) val -= 2.0 * kappa / sqrt(PI); /* (12c) self term */
            S[HIDX(j, k)] = val - block[HIDX(j, k)];
        }
    }
    free(real);
    free(recip);
    free(block);
    free(Iv);
    free(Q);
}

/* ------------------------------------------------------------------------ */
/* O2: the plain FMM                                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int N, d, p, ws;
    double L, kappa;
    const double *pos, *q;
    double *w;           /* wrapped positions [N*3] */
    int nleaf;           /* 2^d per side */
    int *leaf_of;        /* [N] linear leaf index */
    int *start, *list;   /* CSR particle lists per leaf */
    cplx **M, **Lc;      /* per level: [8^l * NCOEF] */
} fmm_t;

static int lin(int ix, int iy, int iz, int n) { return ix + n * (iy + n * iz); }
static int wrapi(int i, int n) { return ((i % n) + n) % n; }

static void cell_centre(int l, int ix, int iy, int iz, double L, double c[3])
{
    double h = L / (double)(1 << l);
    c[0] = (ix + 0.5) * h;
    c[1] = (iy + 0.5) * h;
    c[2] = (iz + 0.5) * h;
}

/* wrap into [0, L) and assign the leaf: leaf = floor(x * 2^d / L), clamped */
static void assign(fmm_t *F)
{
    double scale = (double)F->nleaf / F->L;
    for (int i = 0; i < F->N; ++i) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            double x = F->pos[3 * i + a];
            double w = x - F->L * floor(x / F->L);
            if (w >= F->L) w -= F->L;
            if (w < 0.0) w = 0.0;
            F->w[3 * i + a] = w;
            int k = (int)floor(w * scale);
            if (k < 0) k = 0;
            if (k > F->nleaf - 1) k = F->nleaf - 1;
            c[a] = k;
        }
        F->leaf_of[i] = lin(c[0], c[1], c[2], F->nleaf);
    }
    int nl = F->nleaf * F->nleaf * F->nleaf;
    for (int c = 0; c <= nl; ++c) F->start[c] = 0;
    for (int i = 0; i < F->N; ++i) F->start[F->leaf_of[i] + 1]++;
    for (int c = 0; c < nl; ++c) F->start[c + 1] += F->start[c];
    int *fill = calloc(nl, sizeof(int));
    for (int i = 0; i < F->N; ++i) {
        int c = F->leaf_of[i];
        F->list[F->start[c] + fill[c]++] = i;
    }
    free(fill);
}

static void fmm_alloc(fmm_t *F)
{
    F->nleaf = 1 << F->d;
    int nl = F->nleaf * F->nleaf * F->nleaf;
    F->w = malloc(sizeof(double) * 3 * F->N);
    F->leaf_of = malloc(sizeof(int) * F->N);
    F->start = malloc(sizeof(int) * (nl + 1));
    F->list = malloc(sizeof(int) * F->N);
    F->M = malloc(sizeof(cplx *) * (F->d + 1));
    F->Lc = malloc(sizeof(cplx *) * (F->d + 1));
    for (int l = 0; l <= F->d; ++l) {
        size_t n = (size_t)1 << (3 * l);
        F->M[l] = calloc(n * NCOEF(F->p), sizeof(cplx));
        F->Lc[l] = calloc(n * NCOEF(F->p), sizeof(cplx));
    }
}

static void fmm_free(fmm_t *F)
{
    free(F->w);
    free(F->leaf_of);
    free(F->start);
    free(F->list);
    for (int l = 0; l <= F->d; ++l) {
        free(F->M[l]);
        free(F->Lc[l]);
    }
    free(F->M);
    free(F->Lc);
}

/* P2M at every leaf, then M2M up to level 0.  qmask (nullable) selects which
 * charges take part (the solute-only pass of Eq. FMMcalc). */
static void upward(fmm_t *F, const unsigned char *qmask)
{
    int p = F->p, NC = NCOEF(p);
    int n = F->nleaf;
    double *qq = malloc(sizeof(double) * F->N);
    for (int i = 0; i < F->N; ++i) qq[i] = (qmask && !qmask[i]) ? 0.0 : F->q[i];
#pragma omp parallel for schedule(dynamic, 16)
    for (int c = 0; c < n * n * n; ++c) {
        int ix = c % n, iy = (c / n) % n, iz = c / (n * n);
        double ctr[3];
        cell_centre(F->d, ix, iy, iz, F->L, ctr);
        cplx *M = F->M[F->d] + (size_t)c * NC;
        for (int i = 0; i < NC; ++i) M[i] = 0.0;
        for (int t = F->start[c]; t < F->start[c + 1]; ++t) {
            int j = F->list[t];
            oracle_p2m(p, 1, F->w + 3 * j, qq + j, ctr, M);
        }
    }
    for (int l = F->d - 1; l >= 0; --l) {
        int np = 1 << l;
#pragma omp parallel for schedule(dynamic, 4)
        for (int c = 0; c < np * np * np; ++c) {
            int px = c % np, py = (c / np) % np, pz = c / (np * np);
            double pc[3];
            cell_centre(l, px, py, pz, F->L, pc);
            cplx *Mp = F->M[l] + (size_t)c * NC;
            for (int i = 0; i < NC; ++i) Mp[i] = 0.0;
            for (int ch = 0; ch < 8; ++ch) {
                int cx = 2 * px + (ch & 1), cy = 2 * py + ((ch >> 1) & 1), cz = 2 * pz + ((ch >> 2) & 1);
                double cc[3];
                cell_centre(l + 1, cx, cy, cz, F->L, cc);
                oracle_m2m(p, F->M[l + 1] + (size_t)lin(cx, cy, cz, 2 * np) * NC, cc, pc, Mp);
            }
        }
    }
    free(qq);
}

/* Downward pass: lattice at level 0, then for l = 1..d: L2L from the parent
 * plus M2L over the interaction list, restricted to cells with need[l][c]
 * (need == NULL: all cells). */
static void downward(fmm_t *F, unsigned char **need)
{
    int p = F->p, NC = NCOEF(p), ws = F->ws;
    /* level 0: Lbar(0) = sum M(0) S  (Eq. 12 replacing I in Eq. Lcoeffdef) */
    cplx *S = malloc(sizeof(cplx) * NCOEF(2 * p));
    double kb = F->kappa * F->L;
    int nu_max = (int)ceil(7.0 / kb) + ws + 2;
    int n_kmax = (int)ceil(2.0 * kb * 6.5 / (2 * PI)) + 2;
    oracle_lattice(2 * p, F->L, F->kappa, ws, nu_max, n_kmax, S);
    for (int i = 0; i < NC; ++i) F->Lc[0][i] = 0.0;
    m2l_with(p, F->M[0], S, F->Lc[0]);
    free(S);
    for (int l = 1; l <= F->d; ++l) {
        int n = 1 << l;
        double h = F->L / n;
#pragma omp parallel for schedule(dynamic, 1)
        for (int c = 0; c < n * n * n; ++c) {
            if (need && !need[l][c]) continue;
            int tx = c % n, ty = (c / n) % n, tz = c / (n * n);
            double tc[3];
            cell_centre(l, tx, ty, tz, F->L, tc);
            cplx *Lt = F->Lc[l] + (size_t)c * NC;
            for (int i = 0; i < NC; ++i) Lt[i] = 0.0;
            /* L2L from the parent (the merge Lbar + Lunder of Appendix B) */
            int px = tx >> 1, py = ty >> 1, pz = tz >> 1;
            double pc[3];
            cell_centre(l - 1, px, py, pz, F->L, pc);
            oracle_l2l(p, F->Lc[l - 1] + (size_t)lin(px, py, pz, n / 2) * NC, pc, tc, Lt);
            /* M2L over the interaction list (sources may be periodic images) */
            for (int dz = -ws; dz <= ws; ++dz)
                for (int dy = -ws; dy <= ws; ++dy)
                    for (int dx = -ws; dx <= ws; ++dx)
                        for (int ch = 0; ch < 8; ++ch) {
                            int sx = 2 * (px + dx) + (ch & 1);
                            int sy = 2 * (py + dy) + ((ch >> 1) & 1);
                            int sz = 2 * (pz + dz) + ((ch >> 2) & 1);
                            if (abs(sx - tx) <= ws && abs(sy - ty) <= ws && abs(sz - tz) <= ws) continue;
                            double sc[3] = {(sx + 0.5) * h, (sy + 0.5) * h, (sz + 0.5) * h};
                            int s = lin(wrapi(sx, n), wrapi(sy, n), wrapi(sz, n), n);
                            oracle_m2l(p, F->M[l] + (size_t)s * NC, sc, tc, Lt);
                        }
        }
    }
}

/* near field (Eq. EqNF): phi_i = sum_{j in NF, j != i} q_j / r_ij over the
 * (2ws+1)^3 leaves around i's leaf, periodic; optional pair forces */
static void near_field(fmm_t *F, int i, const unsigned char *jmask, int jmask_val, double *phi, double f[3])
{
    int n = F->nleaf, ws = F->ws;
    int c = F->leaf_of[i];
    int cx = c % n, cy = (c / n) % n, cz = c / (n * n);
    double acc = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
    for (int dz = -ws; dz <= ws; ++dz)
        for (int dy = -ws; dy <= ws; ++dy)
            for (int dx = -ws; dx <= ws; ++dx) {
                int sx = cx + dx, sy = cy + dy, sz = cz + dz;
                double shift[3] = {F->L * floor((double)sx / n), F->L * floor((double)sy / n), F->L * floor((double)sz / n)};
                int s = lin(wrapi(sx, n), wrapi(sy, n), wrapi(sz, n), n);
                for (int t = F->start[s]; t < F->start[s + 1]; ++t) {
                    int j = F->list[t];
                    if (j == i) continue;
                    if (jmask && jmask[j] != jmask_val) continue;
                    double v[3] = {F->w[3 * i] - (F->w[3 * j] + shift[0]),
                                   F->w[3 * i + 1] - (F->w[3 * j + 1] + shift[1]),
                                   F->w[3 * i + 2] - (F->w[3 * j + 2] + shift[2])};
                    double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                    acc += F->q[j] / r;
                    double r3 = r * r * r;
                    fx += F->q[j] * v[0] / r3;
                    fy += F->q[j] * v[1] / r3;
                    fz += F->q[j] * v[2] / r3;
                }
            }
    *phi = acc;
    if (f) {
        f[0] = fx;
        f[1] = fy;
        f[2] = fz;
    }
}

static void far_field(fmm_t *F, int i, double *phi, double grad[3])
{
    int n = F->nleaf;
    int c = F->leaf_of[i];
    double ctr[3];
    cell_centre(F->d, c % n, (c / n) % n, c / (n * n), F->L, ctr);
    oracle_l2p(F->p, F->Lc[F->d] + (size_t)c * NCOEF(F->p), ctr, F->w + 3 * i, phi, grad);
}

/* Neumaier (compensated) summation */
typedef struct { double s, c; } ksum;
static void kadd(ksum *k, double x)
{
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else k->c += (x - t) + k->s;
    k->s = t;
}
static double kval(const ksum *k) { return k->s + k->c; }

/* background-charge block moments over a charge subset (mask == NULL: all):
 * Q = sum q, mu = sum q r, S2 = sum q r^2 with the wrapped coordinates. */
static void bc_moments(fmm_t *F, const unsigned char *mask, int val, double *Q, double mu[3], double *S2)
{
    ksum kq = {0, 0}, kx = {0, 0}, ky = {0, 0}, kz = {0, 0}, ks = {0, 0};
    for (int i = 0; i < F->N; ++i) {
        if (mask && mask[i] != val) continue;
        double *r = F->w + 3 * i;
        kadd(&kq, F->q[i]);
        kadd(&kx, F->q[i] * r[0]);
        kadd(&ky, F->q[i] * r[1]);
        kadd(&kz, F->q[i] * r[2]);
        kadd(&ks, F->q[i] * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]));
    }
    *Q = kval(&kq);
    mu[0] = kval(&kx);
    mu[1] = kval(&ky);
    mu[2] = kval(&kz);
    *S2 = kval(&ks);
}

static int fmm_setup(fmm_t *F, int N, const double *pos, const double *q, double L, int d, int p, int ws, double kappa)
{
    if (N < 1 || d < 1 || p < 0 || ws < 1 || !(L > 0.0) || (1 << d) <= 2 * ws + 1) return 1;
    memset(F, 0, sizeof(*F));
    F->N = N;
    F->d = d;
    F->p = p;
    F->ws = ws;
    F->L = L;
    F->kappa = kappa;
    F->pos = pos;
    F->q = q;
    fmm_alloc(F);
    assign(F);
    return 0;
}

/*
 * Full evaluation.  Outputs (each nullable):
 *   phi_nf[N], phi_ff[N]  per-particle near/far potentials
 *   forces[3N]            F_i = -dE/dr_i
 *   terms[6]              near, far, charged, quad_surface, dipole_surface, total
 */
int oracle_fmm(int N, const double *pos, const double *q, double L, int d, int p, int ws, double kappa,
               double *phi_nf, double *phi_ff, double *forces, double *terms)
{
    fmm_t F;
    if (fmm_setup(&F, N, pos, q, L, d, p, ws, kappa)) return 1;
    upward(&F, NULL);
    downward(&F, NULL);
    double *pn = malloc(sizeof(double) * N), *pf = malloc(sizeof(double) * N);
    double *fn = malloc(sizeof(double) * 3 * N), *gf = malloc(sizeof(double) * 3 * N);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < N; ++i) {
        near_field(&F, i, NULL, 0, pn + i, fn + 3 * i);
        far_field(&F, i, pf + i, gf + 3 * i);
    }
    double Q, mu[3], S2, V = L * L * L;
    bc_moments(&F, NULL, 0, &Q, mu, &S2);
    ksum kn = {0, 0}, kf = {0, 0};
    for (int i = 0; i < N; ++i) {
        kadd(&kn, 0.5 * q[i] * pn[i]);
        kadd(&kf, 0.5 * q[i] * pf[i]);
    }
    double e_near = kval(&kn), e_far = kval(&kf);
    double e_cha = -PI / (2.0 * V * kappa * kappa) * Q * Q;                /* Eq. 6 */
    double e_quad = 2.0 * PI / (3.0 * V) * Q * S2;                         /* Eq. surfchargedend */
    double e_dip = -2.0 * PI / (3.0 * V) * (mu[0] * mu[0] + mu[1] * mu[1] + mu[2] * mu[2]); /* App. D */
    if (terms) {
        terms[0] = e_near;
        terms[1] = e_far;
        terms[2] = e_cha;
        terms[3] = e_quad;
        terms[4] = e_dip;
        ksum kt = {0, 0};
        kadd(&kt, e_near);
        kadd(&kt, e_far);
        kadd(&kt, e_cha);
        kadd(&kt, e_quad);
        kadd(&kt, e_dip);
        terms[5] = kval(&kt);
    }
    if (phi_nf) memcpy(phi_nf, pn, sizeof(double) * N);
    if (phi_ff) memcpy(phi_ff, pf, sizeof(double) * N);
    if (forces) {
        double c = 4.0 * PI / (3.0 * V);
        for (int i = 0; i < N; ++i)
            for (int a = 0; a < 3; ++a)
                forces[3 * i + a] = q[i] * fn[3 * i + a] - q[i] * gf[3 * i + a] - c * q[i] * (Q * F.w[3 * i + a] - mu[a]);
    }
    free(pn);
    free(pf);
    free(fn);
    free(gf);
    fmm_free(&F);
    return 0;
}

/*
 * Per-particle near/far potentials and forces for a sample of particles.
 * The upward pass runs over all charges; the downward pass only over the
 * ancestors of the sampled leaves (the same operators, fewer target cells).
 * The background-charge force -(4 pi / 3V) q_i (Q r_i - mu) is included.
 */
int oracle_fmm_sampled(int N, const double *pos, const double *q, double L, int d, int p, int ws, double kappa,
                       int ns, const int64_t *idx, double *phi_nf, double *phi_ff, double *forces)
{
    fmm_t F;
    if (fmm_setup(&F, N, pos, q, L, d, p, ws, kappa)) return 1;
    for (int s = 0; s < ns; ++s)
        if (idx[s] < 0 || idx[s] >= N) {
            fmm_free(&F);
            return 1;
        }
    unsigned char **need = malloc(sizeof(unsigned char *) * (d + 1));
    for (int l = 0; l <= d; ++l) need[l] = calloc((size_t)1 << (3 * l), 1);
    for (int s = 0; s < ns; ++s) {
        int c = F.leaf_of[idx[s]];
        int n = F.nleaf;
        int x = c % n, y = (c / n) % n, z = c / (n * n);
        for (int l = d; l >= 0; --l) {
            int nl = 1 << l;
            need[l][lin(x, y, z, nl)] = 1;
            x >>= 1;
            y >>= 1;
            z >>= 1;
        }
    }
    upward(&F, NULL);
    downward(&F, need);
    double Q, mu[3], S2, V = L * L * L;
    bc_moments(&F, NULL, 0, &Q, mu, &S2);
    double c = 4.0 * PI / (3.0 * V);
    for (int s = 0; s < ns; ++s) {
        int i = (int)idx[s];
        double pn, pf, fn[3], gf[3];
        near_field(&F, i, NULL, 0, &pn, fn);
        far_field(&F, i, &pf, gf);
        if (phi_nf) phi_nf[s] = pn;
        if (phi_ff) phi_ff[s] = pf;
        if (forces)
            for (int a = 0; a < 3; ++a)
                forces[3 * s + a] = q[i] * fn[a] - q[i] * gf[a] - c * q[i] * (Q * F.w[3 * i + a] - mu[a]);
    }
    for (int l = 0; l <= d; ++l) free(need[l]);
    free(need);
    fmm_free(&F);
    return 0;
}

/*
 * Solute-solvent interaction energy with the reduced far field (Eq. FMMcalc).
 *   A = sum_{i in u} q_i Phi_{u,v}(r_i)   far field of all charges, at solute
 *   B = sum_{i in u} q_i Phi_u(r_i)       far field of solute charges only
 *   C = sum_{j in v} q_j Phi_u(r_j)
 * The paper's V_uv^FF is A - B + C, a sum of q Phi without the factor 1/2, so
 * it counts the solute-solvent far-field interaction W twice: W = (A - B + C)/2.
 * E_uv = NF_uv + W + (background cross terms: Eq. 6, Eq. surfchargedend and
 * the dipole term of Eq. Velecfull split between the solute set with its own
 * neutralising charge and the solvent set with its own):
 *   -pi Qu Qv / (V kappa^2) + (2 pi / 3V)(Qu S2v + Qv S2u) - (4 pi / 3V) mu_u . mu_v
 * out[8] = {E_uv, W, A, B, C, NF_uv, bc_cross, 0}
 */
int oracle_fmm_solute_solvent(int N, const double *pos, const double *q, const unsigned char *is_solute,
                              double L, int d, int p, int ws, double kappa, double *out)
{
    fmm_t F;
    if (fmm_setup(&F, N, pos, q, L, d, p, ws, kappa)) return 1;
    double *phi_all = malloc(sizeof(double) * N), *phi_u = malloc(sizeof(double) * N);
    upward(&F, NULL);
    downward(&F, NULL);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < N; ++i) far_field(&F, i, phi_all + i, NULL);
    upward(&F, is_solute);
    downward(&F, NULL);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < N; ++i) far_field(&F, i, phi_u + i, NULL);
    ksum ka = {0, 0}, kb = {0, 0}, kc = {0, 0}, knf = {0, 0};
    for (int i = 0; i < N; ++i) {
        if (is_solute[i]) {
            kadd(&ka, q[i] * phi_all[i]);
            kadd(&kb, q[i] * phi_u[i]);
            double pn;
            near_field(&F, i, is_solute, 0, &pn, NULL); /* solvent partners only */
            kadd(&knf, q[i] * pn);
        } else {
            kadd(&kc, q[i] * phi_u[i]);
        }
    }
    double A = kval(&ka), B = kval(&kb), C = kval(&kc), NF = kval(&knf);
    double Qu, Qv, muu[3], muv[3], S2u, S2v, V = L * L * L;
    bc_moments(&F, is_solute, 1, &Qu, muu, &S2u);
    bc_moments(&F, is_solute, 0, &Qv, muv, &S2v);
    double bc = -PI * Qu * Qv / (V * kappa * kappa) + 2.0 * PI / (3.0 * V) * (Qu * S2v + Qv * S2u) -
                4.0 * PI / (3.0 * V) * (muu[0] * muv[0] + muu[1] * muv[1] + muu[2] * muv[2]);
    double W = 0.5 * (A - B + C);
    out[0] = NF + W + bc;
    out[1] = W;
    out[2] = A;
    out[3] = B;
    out[4] = C;
    out[5] = NF;
    out[6] = bc;
    out[7] = 0.0;
    free(phi_all);
    free(phi_u);
    fmm_free(&F);
    return 0;
}

/*
 * Soft-core solute-solvent near field.  The paper's soft-core form for the
 * solute-solvent LJ interaction (Calculation detail) replaces r_ij by
 * (alpha lambda A^c + r_ij^c)^(1/c), alpha = 0.2, c = 6, and remarks that
 * the same approach applies to the electrostatic NF term.  Reading: on the
 * solute-solvent pairs of the near field (Eq. EqNF's stencil of (2 ws + 1)^3
 * leaves), with one length A for every pair,
 *   E_sc(lambda) = sum_{i in u} sum_{j in v, j in NF(i)} q_i q_j
 *                                    / (alpha lambda A^c + r_ij^c)^(1/c),
 *   dE_sc/dlambda = -(alpha A^c / c) sum q_i q_j
 *                                    (alpha lambda A^c + r_ij^c)^(-1/c - 1).
 * At lambda = 0 E_sc is the plain NF_uv of Eq. FMMcalc's near-field part.
 * out[2] = {E_sc, dE_sc/dlambda}.
 */
int oracle_softcore_nf_uv(int N, const double *pos, const double *q, const unsigned char *is_solute, double L, int d,
                          int ws, double lambda, double alpha, double A, int c, double *out)
{
    fmm_t F;
    if (c < 1 || !(A >= 0.0) || fmm_setup(&F, N, pos, q, L, d, 0, ws, 1.0)) return 1;
    int n = F.nleaf;
    double Ac = pow(A, (double)c);
    ksum ke = {0, 0}, kd = {0, 0};
    for (int i = 0; i < N; ++i) {
        if (!is_solute[i]) continue;
        int cl = F.leaf_of[i];
        int cx = cl % n, cy = (cl / n) % n, cz = cl / (n * n);
        for (int dz = -ws; dz <= ws; ++dz)
            for (int dy = -ws; dy <= ws; ++dy)
                for (int dx = -ws; dx <= ws; ++dx) {
                    int sx = cx + dx, sy = cy + dy, sz = cz + dz;
                    double shift[3] = {L * floor((double)sx / n), L * floor((double)sy / n), L * floor((double)sz / n)};
                    int sl = lin(wrapi(sx, n), wrapi(sy, n), wrapi(sz, n), n);
                    for (int t = F.start[sl]; t < F.start[sl + 1]; ++t) {
                        int j = F.list[t];
                        if (is_solute[j]) continue;
                        double v[3] = {F.w[3 * i] - (F.w[3 * j] + shift[0]), F.w[3 * i + 1] - (F.w[3 * j + 1] + shift[1]),
                                       F.w[3 * i + 2] - (F.w[3 * j + 2] + shift[2])};
                        double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                        double base = alpha * lambda * Ac + pow(r, (double)c);
                        double reff = pow(base, 1.0 / c);
                        kadd(&ke, q[i] * q[j] / reff);
                        kadd(&kd, -(alpha * Ac / c) * q[i] * q[j] / (reff * base));
                    }
                }
    }
    out[0] = kval(&ke);
    out[1] = kval(&kd);
    fmm_free(&F);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* O1: Ewald sum with point charges and background charge, conducting       */
/* boundary (Appendix A).                                                     */
/*   E = 1/2 sum'_nu sum_ij q_i q_j erfc(kappa r)/r                            */
/*     + (2 pi / V) sum_{k != 0} e^{-k^2/4kappa^2}/k^2 |S(k)|^2                */
/*     - kappa/sqrt(pi) sum q_i^2 - pi Q^2 / (2 V kappa^2)                     */
/* rcut: real-space cutoff; nk: |n_x|,|n_y|,|n_z| <= nk with k = 2 pi n / b,   */
/* k <= kmax.  parts[4] = {real, reciprocal, self, charged}.                   */
/* ------------------------------------------------------------------------ */
int oracle_ewald(int N, const double *pos, const double *q, double b, double kappa, double rcut, double kmax,
                 double *energy, double *forces, double *parts)
{
    if (N < 1 || !(b > 0.0) || !(kappa > 0.0)) return 1;
    double V = b * b * b;
    int nimg = (int)floor(rcut / b) + 1; /* |dx + n b| > rcut for |n| > nimg since |dx| < b */
    double *er = calloc(N, sizeof(double));
    double *fr = calloc(3 * (size_t)N, sizeof(double));
#pragma omp parallel for schedule(dynamic, 8)
    for (int i = 0; i < N; ++i) {
        ksum acc = {0, 0};
        double f[3] = {0, 0, 0};
        for (int j = 0; j < N; ++j)
            for (int nx = -nimg; nx <= nimg; ++nx)
                for (int ny = -nimg; ny <= nimg; ++ny)
                    for (int nz = -nimg; nz <= nimg; ++nz) {
                        if (i == j && nx == 0 && ny == 0 && nz == 0) continue;
                        double v[3] = {pos[3 * i] - pos[3 * j] + nx * b, pos[3 * i + 1] - pos[3 * j + 1] + ny * b,
                                       pos[3 * i + 2] - pos[3 * j + 2] + nz * b};
                        double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                        if (r > rcut) continue;
                        double e = erfc(kappa * r) / r;
                        kadd(&acc, 0.5 * q[i] * q[j] * e);
                        double g = q[i] * q[j] * (e + 2.0 * kappa / sqrt(PI) * exp(-kappa * kappa * r * r)) / (r * r);
                        f[0] += g * v[0];
                        f[1] += g * v[1];
                        f[2] += g * v[2];
                    }
        er[i] = kval(&acc);
        fr[3 * i] = f[0];
        fr[3 * i + 1] = f[1];
        fr[3 * i + 2] = f[2];
    }
    ksum ereal = {0, 0};
    for (int i = 0; i < N; ++i) kadd(&ereal, er[i]);
    /* reciprocal */
    int nk = (int)ceil(kmax * b / (2 * PI));
    int side = 2 * nk + 1;
    int nvec = side * side * side;
    double *erk = calloc(nvec, sizeof(double));
    double *fk = calloc(3 * (size_t)N, sizeof(double));
#pragma omp parallel
    {
        double *fk_local = calloc(3 * (size_t)N, sizeof(double));
#pragma omp for schedule(dynamic, 4)
        for (int t = 0; t < nvec; ++t) {
            int nx = t % side - nk, ny = (t / side) % side - nk, nz = t / (side * side) - nk;
            if (nx == 0 && ny == 0 && nz == 0) continue;
            double kv[3] = {2 * PI * nx / b, 2 * PI * ny / b, 2 * PI * nz / b};
            double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
            if (k2 > kmax * kmax) continue;
            ksum sr = {0, 0}, si = {0, 0};
            for (int j = 0; j < N; ++j) {
                double ph = kv[0] * pos[3 * j] + kv[1] * pos[3 * j + 1] + kv[2] * pos[3 * j + 2];
                kadd(&sr, q[j] * cos(ph));
                kadd(&si, q[j] * sin(ph));
            }
            double Sr = kval(&sr), Si = kval(&si);
            double fac = exp(-k2 / (4 * kappa * kappa)) / k2;
            erk[t] = 2.0 * PI / V * fac * (Sr * Sr + Si * Si);
            /* F_i = (4 pi q_i / V) sum_k fac k Im(e^{i k r_i} conj S) */
            for (int i = 0; i < N; ++i) {
                double ph = kv[0] * pos[3 * i] + kv[1] * pos[3 * i + 1] + kv[2] * pos[3 * i + 2];
                double im = sin(ph) * Sr - cos(ph) * Si;
                double g = 4.0 * PI * q[i] / V * fac * im;
                fk_local[3 * i] += g * kv[0];
                fk_local[3 * i + 1] += g * kv[1];
                fk_local[3 * i + 2] += g * kv[2];
            }
        }
#pragma omp critical
        for (int i = 0; i < 3 * N; ++i) fk[i] += fk_local[i];
        free(fk_local);
    }
    ksum erec = {0, 0};
    for (int t = 0; t < nvec; ++t) kadd(&erec, erk[t]);
    ksum q2 = {0, 0}, qs = {0, 0};
    for (int i = 0; i < N; ++i) {
        kadd(&q2, q[i] * q[i]);
        kadd(&qs, q[i]);
    }
    double Q = kval(&qs);
    double e_self = -kappa / sqrt(PI) * kval(&q2);
    double e_cha = -PI / (2.0 * V * kappa * kappa) * Q * Q;
    double e_real = kval(&ereal), e_rec = kval(&erec);
    ksum tot = {0, 0};
    kadd(&tot, e_real);
    kadd(&tot, e_rec);
    kadd(&tot, e_self);
    kadd(&tot, e_cha);
    *energy = kval(&tot);
    if (parts) {
        parts[0] = e_real;
        parts[1] = e_rec;
        parts[2] = e_self;
        parts[3] = e_cha;
    }
    if (forces)
        for (int i = 0; i < 3 * N; ++i) forces[i] = fr[i] + fk[i];
    free(er);
    free(fr);
    free(erk);
    free(fk);
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
