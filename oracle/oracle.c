/*
 * oracle.c -- plain, slow, FP64 CPU reference for the FMM force solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header, table
 * or generator with the CUDA path.
 *
 * What it computes, and where the definition comes from:
 *   - orc_direct: softened O(N^2) direct sum, the exact target of the method
 *     (Sec. 2 names direct PP summation as the accurate reference; softening
 *     scale Sec. 3.1).  Plummer kernel G(r) = (r^2 + eps^2)^(-1/2), G = 1:
 *         a_i   =  sum_{j!=i} m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2)
 *         phi_i = -sum_{j!=i} m_j / (|x_j - x_i|^2 + eps^2)^(1/2)
 *     Kahan-compensated sums.
 *   - Expansion operators (Sec. 3.1: moments to 4th order about the centre of
 *     mass, local expansion to 5th order).  All are Taylor's theorem in
 *     multi-index form, written out directly:
 *         D^n G(r)        Cartesian derivatives of G, through the Hermite form
 *                         of derivatives of a function of r.r
 *         P2M   M_n  = sum_j m_j y_j^n                       (|n| <= 4)
 *         M2P   a_i  = sum_n (-1)^|n| / n! M_n D^(n+e_i) G(x - z)
 *         M2L   L_k  = sum_{|n|+|k|<=5} (-1)^|n| / n! M_n D^(n+k) G(c - z)
 *         P2L   L_k  = m D^k G(c - x_j)                       (|k| <= 5)
 *         L2L   L'_k = sum_{|j|<=5-|k|} t^j / j! L_(k+j)
 *         L2P   a_i  = sum_{|k|<=4} u^k / k! L_(k+e_i)
 *   - Periodic boundaries (Sec. 3.1): orc_direct_periodic, the periodic direct sum in the unit
 *     box (Ewald summation with a uniform background; the copies inside the replica shell
 *     softened, as the walk over them is); orc_ewald_derivs, the derivatives to 5th order of the
 *     correction kernel F = periodic potential less the shell's Newtonian copies; orc_ewald_m2p,
 *     the correction from a cell's moments.
 *   - orc_fmm_*: a plain recursive FMM (Sec. 3.1): Morton-ordered binary tree
 *     with buckets of <= b particles, exact b_max about the centre of mass,
 *     opening radius R_O = b_max / theta, checklist walk with outcomes
 *     accept (CC/CP) / defer / PC / PP / open, groups of <= g particles.
 *     Opening decisions are integer outcomes decided by floating point; they
 *     are taken in single precision (the precision the paper uses for the
 *     interaction work, Sec. 3.1), with a fixed operation order and no fused
 *     multiply-add, so that any implementation following the same order takes
 *     identical decisions.  All force arithmetic is FP64.  orc_fmm_create_periodic starts the
 *     walk from the root and its 26 (or 124) copies and adds the Ewald correction of the root's
 *     moments for the copies beyond.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (oracle/build.py).
 * -ffp-contract=off is required for the single-precision decisions.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* multi-index tables: all n = (a,b,c) with a+b+c <= 5, ordered by     */
/* total order, then a descending, then b descending                    */
/* ------------------------------------------------------------------ */
#define ORD 5
#define NMI 56 /* |n| <= 5 */
#define NM4 35 /* |n| <= 4 */

static int MI[NMI][3];
static int MIDX[ORD + 1][ORD + 1][ORD + 1];
static double FACT[16];
static int tables_ready = 0;

static void make_tables(void)
{
    int i = 0;
    for (int o = 0; o <= ORD; o++)
        for (int a = o; a >= 0; a--)
            for (int b = o - a; b >= 0; b--) {
                int c = o - a - b;
                MI[i][0] = a;
                MI[i][1] = b;
                MI[i][2] = c;
                MIDX[a][b][c] = i;
                i++;
            }
    FACT[0] = 1.0;
    for (int k = 1; k < 16; k++) FACT[k] = FACT[k - 1] * k;
    tables_ready = 1;
}

__attribute__((constructor)) static void orc_init(void) { make_tables(); }

static inline int order_of(int i) { return MI[i][0] + MI[i][1] + MI[i][2]; }
static inline double mfact(int i) { return FACT[MI[i][0]] * FACT[MI[i][1]] * FACT[MI[i][2]]; }
static inline int idx_add(int i, int j)
{
    int a = MI[i][0] + MI[j][0], b = MI[i][1] + MI[j][1], c = MI[i][2] + MI[j][2];
    if (a + b + c > ORD) return -1;
    return MIDX[a][b][c];
}

void orc_multi_index(int *out)
{
    for (int i = 0; i < NMI; i++) {
        out[3 * i] = MI[i][0];
        out[3 * i + 1] = MI[i][1];
        out[3 * i + 2] = MI[i][2];
    }
}

/* u^n for all |n| <= 5 */
static void monomials(const double u[3], double P[NMI])
{
    double px[ORD + 1], py[ORD + 1], pz[ORD + 1];
    px[0] = py[0] = pz[0] = 1.0;
    for (int k = 1; k <= ORD; k++) {
        px[k] = px[k - 1] * u[0];
        py[k] = py[k - 1] * u[1];
        pz[k] = pz[k - 1] * u[2];
    }
    for (int i = 0; i < NMI; i++) P[i] = px[MI[i][0]] * py[MI[i][1]] * pz[MI[i][2]];
}

/* Hermite coefficient: number of ways to pick k disjoint pairs out of n indices */
static double herm(int n, int k) { return FACT[n] / (ldexp(1.0, k) * FACT[k] * FACT[n - 2 * k]); }

/*
 * Derivatives of a function of s = r.r.  With h(s) and d_m = 2^m h^(m)(s), the Hermite form
 *   D^(a,b,c) h = sum_{i<=a/2, j<=b/2, k<=c/2} H(a,i) H(b,j) H(c,k)
 *                 x^(a-2i) y^(b-2j) z^(c-2k) d_(a+b+c-i-j-k)
 * gives every |n| <= 5.  radial_tensor_acc adds w * D^n h(r) to D.
 */
static void radial_tensor_acc(const double r[3], const double d[ORD + 1], double w, double D[NMI])
{
    double px[ORD + 1], py[ORD + 1], pz[ORD + 1];
    px[0] = py[0] = pz[0] = 1.0;
    for (int k = 1; k <= ORD; k++) {
        px[k] = px[k - 1] * r[0];
        py[k] = py[k - 1] * r[1];
        pz[k] = pz[k - 1] * r[2];
    }
    for (int n = 0; n < NMI; n++) {
        int a = MI[n][0], b = MI[n][1], c = MI[n][2];
        double s = 0.0;
        for (int i = 0; 2 * i <= a; i++)
            for (int j = 0; 2 * j <= b; j++)
                for (int k = 0; 2 * k <= c; k++)
                    s += herm(a, i) * herm(b, j) * herm(c, k) * px[a - 2 * i] * py[b - 2 * j] *
                         pz[c - 2 * k] * d[a + b + c - i - j - k];
        D[n] += w * s;
    }
}

/* G = (s + eps2)^(-1/2): d_m = (-1)^m (2m-1)!! R^-(2m+1), R^2 = s + eps2 (m = 0..mmax) */
static void plummer_scalars(double R2, int mmax, double *d)
{
    double iR = 1.0 / sqrt(R2), iR2 = iR * iR;
    double dfact = 1.0; /* (2m-1)!! */
    double p = iR;
    for (int m = 0; m <= mmax; m++) {
        if (m > 0) dfact *= (2.0 * m - 1.0);
        d[m] = ((m & 1) ? -1.0 : 1.0) * dfact * p;
        p *= iR2;
    }
}

/* D^n G(r) for |n| <= 5 with G = (r.r + eps2)^(-1/2) */
void orc_green_derivs(const double r[3], double eps2, double D[NMI])
{
    double d[ORD + 1];
    plummer_scalars(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + eps2, ORD, d);
    for (int n = 0; n < NMI; n++) D[n] = 0.0;
    radial_tensor_acc(r, d, 1.0, D);
}

/* P2M: M_n = sum_j m_j (x_j - c)^n for |n| <= 4 */
static void p2m_acc(double m, const double y[3], double M[NM4])
{
    double P[NMI];
    monomials(y, P);
    for (int i = 0; i < NM4; i++) M[i] += m * P[i];
}

void orc_p2m(long n, const double *pos /* 3n SoA */, const double *mass, const double c[3], double *M)
{
    for (int i = 0; i < NM4; i++) M[i] = 0.0;
    for (long j = 0; j < n; j++) {
        double y[3] = {pos[j] - c[0], pos[n + j] - c[1], pos[2 * n + j] - c[2]};
        p2m_acc(mass[j], y, M);
    }
}

/* the field of moments M given the derivatives D of the kernel at r = x - z:
 *   Phi = sum_n (-1)^|n| / n! M_n D_n,  a_i = sum_n (-1)^|n| / n! M_n D_(n+e_i);  acc += a, *pot -= Phi */
static void contract_m2p(const double M[NM4], const double D[NMI], double acc[3], double *pot)
{
    double Phi = 0.0, a[3] = {0.0, 0.0, 0.0};
    for (int n = 0; n < NM4; n++) {
        double w = ((order_of(n) & 1) ? -1.0 : 1.0) / mfact(n) * M[n];
        Phi += w * D[n];
        for (int q = 0; q < 3; q++) a[q] += w * D[idx_add(n, 1 + q)];
    }
    for (int q = 0; q < 3; q++) acc[q] += a[q];
    *pot -= Phi;
}

/* M2P: field at x of the moments M about z */
static void m2p_acc(const double M[NM4], const double z[3], const double x[3], double eps2, double acc[3],
                    double *pot)
{
    double r[3] = {x[0] - z[0], x[1] - z[1], x[2] - z[2]};
    double D[NMI];
    orc_green_derivs(r, eps2, D);
    contract_m2p(M, D, acc, pot);
}

void orc_m2p(const double *M, const double z[3], const double x[3], double eps2, double acc[3], double *pot)
{
    acc[0] = acc[1] = acc[2] = 0.0;
    *pot = 0.0;
    m2p_acc(M, z, x, eps2, acc, pot);
}

/* M2L: L_k += sum_{|n|+|k|<=5} (-1)^|n|/n! M_n D^(n+k) G(c - z) */
static void m2l_acc(const double M[NM4], const double z[3], const double c[3], double eps2, double L[NMI])
{
    double r[3] = {c[0] - z[0], c[1] - z[1], c[2] - z[2]};
    double D[NMI];
    orc_green_derivs(r, eps2, D);
    for (int k = 0; k < NMI; k++) {
        double s = 0.0;
        for (int n = 0; n < NM4; n++) {
            int nk = idx_add(n, k);
            if (nk < 0) continue;
            s += ((order_of(n) & 1) ? -1.0 : 1.0) / mfact(n) * M[n] * D[nk];
        }
        L[k] += s;
    }
}

void orc_m2l(const double *M, const double z[3], const double c[3], double eps2, double *L)
{
    for (int k = 0; k < NMI; k++) L[k] = 0.0;
    m2l_acc(M, z, c, eps2, L);
}

/* P2L: L_k += m D^k G(c - x) */
static void p2l_acc(double m, const double x[3], const double c[3], double eps2, double L[NMI])
{
    double r[3] = {c[0] - x[0], c[1] - x[1], c[2] - x[2]};
    double D[NMI];
    orc_green_derivs(r, eps2, D);
    for (int k = 0; k < NMI; k++) L[k] += m * D[k];
}

void orc_p2l(double m, const double x[3], const double c[3], double eps2, double *L)
{
    for (int k = 0; k < NMI; k++) L[k] = 0.0;
    p2l_acc(m, x, c, eps2, L);
}

/* L2L: re-expand L about c at c + t */
void orc_l2l(const double *L, const double t[3], double *Lo)
{
    double T[NMI];
    monomials(t, T);
    for (int k = 0; k < NMI; k++) {
        double s = 0.0;
        for (int j = 0; j < NMI; j++) {
            int kj = idx_add(k, j);
            if (kj < 0) continue;
            s += T[j] / mfact(j) * L[kj];
        }
        Lo[k] = s;
    }
}

/* L2P: acc += grad Phi at c + u, *pot -= Phi */
static void l2p_acc(const double L[NMI], const double u[3], double acc[3], double *pot)
{
    double U[NMI];
    monomials(u, U);
    double Phi = 0.0, a[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < NMI; k++) {
        double w = U[k] / mfact(k);
        Phi += w * L[k];
        if (order_of(k) <= ORD - 1)
            for (int q = 0; q < 3; q++) a[q] += w * L[idx_add(k, 1 + q)];
    }
    for (int q = 0; q < 3; q++) acc[q] += a[q];
    *pot -= Phi;
}

void orc_l2p(const double *L, const double u[3], double acc[3], double *pot)
{
    acc[0] = acc[1] = acc[2] = 0.0;
    *pot = 0.0;
    l2p_acc(L, u, acc, pot);
}

/* ------------------------------------------------------------------ */
/* direct sum (the ground truth)                                       */
/* ------------------------------------------------------------------ */
void orc_direct(long n, const double *pos, const double *mass, double eps, long ns, const long *sinks,
                double *acc /* 3 ns SoA */, double *pot /* ns */)
{
    const double *X = pos, *Y = pos + n, *Z = pos + 2 * n;
    double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 8)
    for (long q = 0; q < ns; q++) {
        long i = sinks ? sinks[q] : q;
        double s[4] = {0, 0, 0, 0}, cmp[4] = {0, 0, 0, 0};
        for (long j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = X[j] - X[i], dy = Y[j] - Y[i], dz = Z[j] - Z[i];
            double R2 = dx * dx + dy * dy + dz * dz + eps2;
            double iR = 1.0 / sqrt(R2);
            double miR = mass[j] * iR;
            double miR3 = miR * iR * iR;
            double t[4] = {miR3 * dx, miR3 * dy, miR3 * dz, -miR};
            for (int c = 0; c < 4; c++) { /* Kahan */
                double yk = t[c] - cmp[c];
                double tk = s[c] + yk;
                cmp[c] = (tk - s[c]) - yk;
                s[c] = tk;
            }
        }
        acc[q] = s[0];
        acc[ns + q] = s[1];
        acc[2 * ns + q] = s[2];
        pot[q] = s[3];
    }
}

/* ------------------------------------------------------------------ */
/* periodic boundaries (Sec. 3.1): the unit box and its replicas       */
/* ------------------------------------------------------------------ */
/*
 * psi(r): the potential of a unit mass at the origin and at every periodic copy r + n (n integer),
 * less a uniform background of unit density, with zero mean over the box.  Ewald's split with any
 * alpha > 0 writes it as
 *   psi(r) = sum_n erfc(alpha |r+n|) / |r+n|
 *          + sum_{h != 0} exp(-pi^2 h^2 / alpha^2) / (pi h^2) cos(2 pi h.r)  -  pi / alpha^2.
 *
 * The paper gives the method (the root and its 26 or 124 replicas on the checklist, the rest
 * from a 5th-order multipole approximation of the Ewald sum), not the sum it approximates.
 * Reading: the copies inside the replica shell N = { n : |n|_inf <= nrep } use the softened
 * kernel G, as the walk over those replicas does; beyond N the Newtonian Ewald sum applies.
 * Between a sink and a source at offset r = x_i - x_j the kernel is
 *   K(r) = sum_{n in N} G(r + n) + F(r),   F(r) = psi(r) - sum_{n in N} 1 / |r + n|
 * (the n = 0 term of G dropped for the particle itself), and
 *   phi_i = -sum_j m_j K(x_i - x_j),   a_i = sum_j m_j grad K(x_i - x_j).
 * F has no singularity for r in (-nrep-1, nrep+1)^3, which holds every offset between two
 * points of the box.  Functions here take offsets with |r_a| < 1.
 */
#define EWALD_CUT 8.0 /* drop real-space copies with alpha |r+n| >= 8 and reciprocal terms with pi |h| / alpha >= 8 */

/* erfc(alpha sqrt(s)) / sqrt(s): d_m = (-1)^m B_m,
 *   B_0 = erfc(alpha r) / r,  B_m = ((2m-1) B_(m-1) + (2 alpha^2)^m exp(-alpha^2 r^2) / (alpha sqrt(pi))) / r^2
 * (B_m = (-(1/r) d/dr)^m B_0) */
static void erfc_scalars(double s, double alpha, int mmax, double *d)
{
    double r = sqrt(s);
    double g = exp(-alpha * alpha * s) / (alpha * sqrt(M_PI));
    double B = erfc(alpha * r) / r, p = 1.0;
    d[0] = B;
    for (int m = 1; m <= mmax; m++) {
        p *= 2.0 * alpha * alpha;
        B = ((2.0 * m - 1.0) * B + p * g) / s;
        d[m] = (m & 1) ? -B : B;
    }
}

/* erf(alpha sqrt(s)) / sqrt(s), finite at s = 0.  While alpha^2 s < 2.25 from its power series,
 *   h(s) = 2 alpha / sqrt(pi) sum_k (-alpha^2 s)^k / (k! (2k+1)),
 *   h^(m)(s) = 2 alpha / sqrt(pi) sum_{k>=m} (-alpha^2)^k s^(k-m) / ((k-m)! (2k+1)),
 * else as 1/r less the erfc part. */
static void erf_scalars(double s, double alpha, int mmax, double *d)
{
    double a2 = alpha * alpha;
    if (a2 * s < 2.25) {
        double c = 2.0 * alpha / sqrt(M_PI);
        for (int m = 0; m <= mmax; m++) {
            double sum = 0.0, t = 1.0; /* t = (-a2 s)^j / j! with j = k - m */
            for (int j = 0; j < 60; j++) {
                sum += t / (2.0 * (m + j) + 1.0);
                t *= -a2 * s / (j + 1.0);
            }
            d[m] = c * sum; /* times 2^m (-a2)^m below */
            for (int q = 0; q < m; q++) d[m] *= -2.0 * a2;
        }
        return;
    }
    double N[ORD + 1], B[ORD + 1];
    plummer_scalars(s, mmax, N);
    erfc_scalars(s, alpha, mmax, B);
    for (int m = 0; m <= mmax; m++) d[m] = N[m] - B[m];
}

/* reciprocal vectors of the half space (h and -h together): count, or fill h[3k] and coef[k] =
 * 2 exp(-pi^2 h^2 / alpha^2) / (pi h^2) */
static long recip_vectors(double alpha, double *hv, double *coef)
{
    int H = (int)ceil(EWALD_CUT * alpha / M_PI);
    long k = 0;
    for (int hx = 0; hx <= H; hx++)
        for (int hy = -H; hy <= H; hy++)
            for (int hz = -H; hz <= H; hz++) {
                if (hx == 0 && (hy < 0 || (hy == 0 && hz <= 0))) continue;
                double h2 = (double)hx * hx + (double)hy * hy + (double)hz * hz;
                if (M_PI * sqrt(h2) / alpha >= EWALD_CUT) continue;
                if (hv) {
                    hv[3 * k] = hx;
                    hv[3 * k + 1] = hy;
                    hv[3 * k + 2] = hz;
                    coef[k] = 2.0 * exp(-M_PI * M_PI * h2 / (alpha * alpha)) / (M_PI * h2);
                }
                k++;
            }
    return k;
}

/* range of copies n_a along one axis: the replica shell, and every copy with |r_a + n_a| < cut */
static void copy_range(double ra, int nrep, double cut, int *lo, int *hi)
{
    int a = (int)ceil(-ra - cut), b = (int)floor(-ra + cut);
    *lo = a < -nrep ? a : -nrep;
    *hi = b > nrep ? b : nrep;
}

/* D^n F(r) for |n| <= 5 (F = psi less the Newtonian copies inside the replica shell) */
void orc_ewald_derivs(const double r[3], int nrep, double alpha, double D[NMI])
{
    for (int n = 0; n < NMI; n++) D[n] = 0.0;
    double d[ORD + 1], cut = EWALD_CUT / alpha;
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) copy_range(r[a], nrep, cut, &lo[a], &hi[a]);
    for (int nx = lo[0]; nx <= hi[0]; nx++)
        for (int ny = lo[1]; ny <= hi[1]; ny++)
            for (int nz = lo[2]; nz <= hi[2]; nz++) {
                double u[3] = {r[0] + nx, r[1] + ny, r[2] + nz};
                double s = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                int in_shell = abs(nx) <= nrep && abs(ny) <= nrep && abs(nz) <= nrep;
                if (in_shell) {
                    erf_scalars(s, alpha, ORD, d);
                    radial_tensor_acc(u, d, -1.0, D);
                } else if (alpha * sqrt(s) < EWALD_CUT) {
                    erfc_scalars(s, alpha, ORD, d);
                    radial_tensor_acc(u, d, 1.0, D);
                }
            }
    long nh = recip_vectors(alpha, NULL, NULL);
    double *hv = malloc(3 * nh * sizeof(double)), *coef = malloc(nh * sizeof(double));
    recip_vectors(alpha, hv, coef);
    for (long k = 0; k < nh; k++) {
        /* D^n cos(2 pi h.r) = (2 pi h)^n cos(2 pi h.r + |n| pi / 2) */
        double th = 2.0 * M_PI * (hv[3 * k] * r[0] + hv[3 * k + 1] * r[1] + hv[3 * k + 2] * r[2]);
        double cs = cos(th), sn = sin(th);
        double ph[4] = {cs, -sn, -cs, sn};
        double kx[ORD + 1], ky[ORD + 1], kz[ORD + 1];
        kx[0] = ky[0] = kz[0] = 1.0;
        for (int q = 1; q <= ORD; q++) {
            kx[q] = kx[q - 1] * 2.0 * M_PI * hv[3 * k];
            ky[q] = ky[q - 1] * 2.0 * M_PI * hv[3 * k + 1];
            kz[q] = kz[q - 1] * 2.0 * M_PI * hv[3 * k + 2];
        }
        for (int n = 0; n < NMI; n++)
            D[n] += coef[k] * kx[MI[n][0]] * ky[MI[n][1]] * kz[MI[n][2]] * ph[order_of(n) & 3];
    }
    free(hv);
    free(coef);
    D[0] -= M_PI / (alpha * alpha);
}

/* the correction for the copies beyond the replica shell, from moments M (|n| <= 4) about z:
 * the M2P contraction with D^n F(x - z) */
void orc_ewald_m2p(const double *M, const double z[3], const double x[3], int nrep, double alpha, double acc[3],
                   double *pot)
{
    double r[3] = {x[0] - z[0], x[1] - z[1], x[2] - z[2]}, D[NMI];
    orc_ewald_derivs(r, nrep, alpha, D);
    acc[0] = acc[1] = acc[2] = 0.0;
    *pot = 0.0;
    contract_m2p(M, D, acc, pot);
}

/* the periodic direct sum (the reading above): every source, every copy, for each sink.
 * Reciprocal space through the structure factors C(h) + i S(h) = sum_j m_j exp(2 pi i h.x_j). */
void orc_direct_periodic(long n, const double *pos, const double *mass, double eps, int nrep, double alpha,
                         long ns, const long *sinks, double *acc /* 3 ns SoA */, double *pot /* ns */)
{
    const double *X = pos, *Y = pos + n, *Z = pos + 2 * n;
    double eps2 = eps * eps, cut = EWALD_CUT / alpha, mtot = 0.0;
    for (long j = 0; j < n; j++) mtot += mass[j];
    long nh = recip_vectors(alpha, NULL, NULL);
    double *hv = malloc(3 * nh * sizeof(double)), *coef = malloc(nh * sizeof(double));
    double *Cs = malloc(nh * sizeof(double)), *Sn = malloc(nh * sizeof(double));
    recip_vectors(alpha, hv, coef);
#pragma omp parallel for schedule(dynamic, 16)
    for (long k = 0; k < nh; k++) {
        double c = 0.0, sn = 0.0;
        for (long j = 0; j < n; j++) {
            double th = 2.0 * M_PI * (hv[3 * k] * X[j] + hv[3 * k + 1] * Y[j] + hv[3 * k + 2] * Z[j]);
            c += mass[j] * cos(th);
            sn += mass[j] * sin(th);
        }
        Cs[k] = c;
        Sn[k] = sn;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (long q = 0; q < ns; q++) {
        long i = sinks ? sinks[q] : q;
        double a[3] = {0, 0, 0}, ph = 0.0, d[2];
        for (long j = 0; j < n; j++) {
            double r[3] = {X[i] - X[j], Y[i] - Y[j], Z[i] - Z[j]};
            int lo[3], hi[3];
            for (int ax = 0; ax < 3; ax++) copy_range(r[ax], nrep, cut, &lo[ax], &hi[ax]);
            double kp = 0.0, kg[3] = {0, 0, 0};
            for (int nx = lo[0]; nx <= hi[0]; nx++)
                for (int ny = lo[1]; ny <= hi[1]; ny++)
                    for (int nz = lo[2]; nz <= hi[2]; nz++) {
                        double u[3] = {r[0] + nx, r[1] + ny, r[2] + nz};
                        double s = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                        int in_shell = abs(nx) <= nrep && abs(ny) <= nrep && abs(nz) <= nrep;
                        double w0 = 0.0, w1 = 0.0; /* kernel value and 2 dK/ds */
                        if (in_shell) {
                            if (!(j == i && nx == 0 && ny == 0 && nz == 0)) {
                                plummer_scalars(s + eps2, 1, d);
                                w0 += d[0];
                                w1 += d[1];
                            }
                            erf_scalars(s, alpha, 1, d);
                            w0 -= d[0];
                            w1 -= d[1];
                        } else if (alpha * sqrt(s) < EWALD_CUT) {
                            erfc_scalars(s, alpha, 1, d);
                            w0 += d[0];
                            w1 += d[1];
                        }
                        kp += w0;
                        for (int ax = 0; ax < 3; ax++) kg[ax] += w1 * u[ax];
                    }
            ph -= mass[j] * kp;
            for (int ax = 0; ax < 3; ax++) a[ax] += mass[j] * kg[ax];
        }
        for (long k = 0; k < nh; k++) {
            double th = 2.0 * M_PI * (hv[3 * k] * X[i] + hv[3 * k + 1] * Y[i] + hv[3 * k + 2] * Z[i]);
            double cs = cos(th), sn = sin(th);
            /* sum_j m_j cos(th_i - th_j) and sum_j m_j sin(th_i - th_j) */
            double cd = cs * Cs[k] + sn * Sn[k], sd = sn * Cs[k] - cs * Sn[k];
            ph -= coef[k] * cd;
            for (int ax = 0; ax < 3; ax++) a[ax] -= coef[k] * 2.0 * M_PI * hv[3 * k + ax] * sd;
        }
        ph += mtot * M_PI / (alpha * alpha);
        acc[q] = a[0];
        acc[ns + q] = a[1];
        acc[2 * ns + q] = a[2];
        pot[q] = ph;
    }
    free(hv);
    free(coef);
    free(Cs);
    free(Sn);
}

/* ------------------------------------------------------------------ */
/* plain FMM                                                           */
/* ------------------------------------------------------------------ */
enum { K_PP = 0, K_PC = 1, K_CC = 2, K_CP = 3 };
enum { O_ACCEPT = 1, O_DEFER = 2, O_PC = 3, O_PP = 4, O_OPEN = 5 };

/* a checklist entry: a cell or a particle, in the box (sh = 0) or in the periodic copy shifted by sh */
typedef struct {
    long id;
    int particle;
    int sh[3];
} entry;

typedef struct {
    long *sink, *first, *count, *cell; /* cell = source cell id, -1 for a particle entry */
    int *shift;                        /* the copy: (sx + 2) * 25 + (sy + 2) * 5 + (sz + 2), |s| <= 2 */
    long n, cap;
} elist;

static int shift_code(const int sh[3]) { return (sh[0] + 2) * 25 + (sh[1] + 2) * 5 + (sh[2] + 2); }
static void shift_of(int code, double v[3])
{
    v[0] = code / 25 - 2;
    v[1] = (code / 5) % 5 - 2;
    v[2] = code % 5 - 2;
}

typedef struct {
    long n;
    int b, g;
    double eps, theta;
    int nrep; /* periodic: the root's copies |n|_inf <= nrep start the walk; -1 for an isolated box */
    long *perm;
    uint64_t *key;
    double *X, *Y, *Z, *m;
    unsigned char *act;
    /* cells */
    long nc, depth;
    long *first, *count, *child, *parent, *nact, *level;
    double *mass, *com, *lo, *hi, *bmax, *mom;
    float *comf, *lof, *hif, *bmaxf, *rof;
    /* walk output */
    elist lists[4];
    long ng;
    long *gcell, *gseg; /* per group: cell, [pp_begin, pp_end, pc_begin, pc_end] */
    double *gL;         /* 56 per group */
    long gcap;
    int status;
} orc_fmm;

static void elist_push(elist *l, long sink, long first, long count, long cell, const int sh[3])
{
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 1024;
        l->sink = realloc(l->sink, l->cap * sizeof(long));
        l->first = realloc(l->first, l->cap * sizeof(long));
        l->count = realloc(l->count, l->cap * sizeof(long));
        l->cell = realloc(l->cell, l->cap * sizeof(long));
        l->shift = realloc(l->shift, l->cap * sizeof(int));
    }
    l->sink[l->n] = sink;
    l->first[l->n] = first;
    l->count[l->n] = count;
    l->cell[l->n] = cell;
    l->shift[l->n] = shift_code(sh);
    l->n++;
}

static uint64_t morton_key(double x, double y, double z)
{
    uint64_t q[3];
    double v[3] = {x, y, z};
    for (int a = 0; a < 3; a++) {
        double s = v[a] * 2097152.0; /* 2^21, exact */
        if (s < 0.0) s = 0.0;
        uint64_t u = (uint64_t)s;
        if (u > 2097151u) u = 2097151u;
        q[a] = u;
    }
    uint64_t k = 0;
    for (int l = 0; l < 63; l++) {
        int axis = l % 3, bit = 20 - l / 3;
        k |= ((q[axis] >> bit) & 1u) << (62 - l);
    }
    return k;
}

static int cmp_key(const void *pa, const void *pb, void *ctx)
{
    long a = *(const long *)pa, b = *(const long *)pb;
    const uint64_t *key = (const uint64_t *)ctx;
    uint64_t ka = key[a], kb = key[b];
    if (ka < kb) return -1;
    if (ka > kb) return 1;
    return (a < b) ? -1 : (a > b);
}

static int clz64(uint64_t v) { return v ? __builtin_clzll(v) : 64; }

/* split point of the sorted range [f, l] (inclusive): first index of the right child */
static long split_range(const uint64_t *key, long f, long l)
{
    if (key[f] != key[l]) {
        int L = clz64(key[f] ^ key[l]);
        uint64_t bit = 1ull << (63 - L);
        long lo = f, hi = l; /* key[lo] has bit clear, key[hi] has it set */
        while (hi - lo > 1) {
            long mid = lo + (hi - lo) / 2;
            if (key[mid] & bit) hi = mid;
            else lo = mid;
        }
        return hi;
    }
    /* identical keys: split on the highest differing bit of the positions */
    uint64_t x = (uint64_t)f ^ (uint64_t)l;
    int hb = 63 - clz64(x);
    return (long)(((uint64_t)l >> hb) << hb);
}

static long build_rec(orc_fmm *t, long f, long cnt, long parent, long lev)
{
    long c = t->nc++;
    t->first[c] = f;
    t->count[c] = cnt;
    t->parent[c] = parent;
    t->level[c] = lev;
    if (lev > t->depth) t->depth = lev;
    t->child[2 * c] = t->child[2 * c + 1] = -1;
    if (cnt > t->b) {
        long m = split_range(t->key, f, f + cnt - 1);
        long c0 = build_rec(t, f, m - f, c, lev + 1);
        long c1 = build_rec(t, m, f + cnt - m, c, lev + 1);
        t->child[2 * c] = c0;
        t->child[2 * c + 1] = c1;
    }
    return c;
}

static void cell_props(orc_fmm *t, long c)
{
    long f = t->first[c], cnt = t->count[c];
    double M = 0, sx = 0, sy = 0, sz = 0;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    long na = 0;
    for (long j = f; j < f + cnt; j++) {
        M += t->m[j];
        sx += t->m[j] * t->X[j];
        sy += t->m[j] * t->Y[j];
        sz += t->m[j] * t->Z[j];
        double p[3] = {t->X[j], t->Y[j], t->Z[j]};
        for (int a = 0; a < 3; a++) {
            if (p[a] < lo[a]) lo[a] = p[a];
            if (p[a] > hi[a]) hi[a] = p[a];
        }
        na += t->act[j] ? 1 : 0;
    }
    double com[3] = {sx / M, sy / M, sz / M};
    double b2 = 0.0;
    double *mom = t->mom + NM4 * c;
    for (int i = 0; i < NM4; i++) mom[i] = 0.0;
    for (long j = f; j < f + cnt; j++) {
        double dx = t->X[j] - com[0], dy = t->Y[j] - com[1], dz = t->Z[j] - com[2];
        double d2 = dx * dx + dy * dy;
        d2 = d2 + dz * dz;
        if (d2 > b2) b2 = d2;
        double y[3] = {dx, dy, dz};
        p2m_acc(t->m[j], y, mom);
    }
    t->mass[c] = M;
    t->nact[c] = na;
    for (int a = 0; a < 3; a++) {
        t->com[3 * c + a] = com[a];
        t->lo[3 * c + a] = lo[a];
        t->hi[3 * c + a] = hi[a];
        t->comf[3 * c + a] = (float)com[a];
        t->lof[3 * c + a] = (float)lo[a];
        t->hif[3 * c + a] = (float)hi[a];
    }
    t->bmax[c] = sqrt(b2);
    t->bmaxf[c] = (float)t->bmax[c];
    t->rof[c] = (cnt == 1) ? 0.0f : t->bmaxf[c] / (float)t->theta;
}

/* geometry of a checklist entry, single precision; a copy's coordinates are shifted in double
 * precision and then rounded */
typedef struct {
    float c[3], lo[3], hi[3], ro;
    int pointlike, leaf;
} sgeom;

static void entry_geom(const orc_fmm *t, entry e, sgeom *s)
{
    if (e.particle) {
        float p[3] = {(float)(t->X[e.id] + e.sh[0]), (float)(t->Y[e.id] + e.sh[1]), (float)(t->Z[e.id] + e.sh[2])};
        for (int a = 0; a < 3; a++) s->c[a] = s->lo[a] = s->hi[a] = p[a];
        s->ro = 0.0f;
        s->pointlike = 1;
        s->leaf = 1;
    } else {
        long c = e.id;
        for (int a = 0; a < 3; a++) {
            if (e.sh[a] == 0) {
                s->c[a] = t->comf[3 * c + a];
                s->lo[a] = t->lof[3 * c + a];
                s->hi[a] = t->hif[3 * c + a];
            } else {
                s->c[a] = (float)(t->com[3 * c + a] + e.sh[a]);
                s->lo[a] = (float)(t->lo[3 * c + a] + e.sh[a]);
                s->hi[a] = (float)(t->hi[3 * c + a] + e.sh[a]);
            }
        }
        s->ro = t->rof[c];
        s->pointlike = (t->count[c] == 1);
        s->leaf = (t->count[c] <= t->b);
    }
}

/*
 * Opening decision for sink cell k and source s (Sec. 3.1), single precision,
 * fixed operation order, no fused multiply-add.
 *   accept (CC/CP) : d > 1.5 R_O(k) + R_O(s)  and  bbox gap >= 2 eps
 *   k not a group  : defer if s is point-like or R_O(s) <= R_O(k), else open
 *   k a group      : PP if s is point-like; PC if d > R_O(s) + b_max(k);
 *                    PP if s is a bucket; else open
 */
static int decide(const orc_fmm *t, long k, const sgeom *s, int k_group, float four_eps2)
{
    float dx = t->comf[3 * k] - s->c[0];
    float dy = t->comf[3 * k + 1] - s->c[1];
    float dz = t->comf[3 * k + 2] - s->c[2];
    float d2 = dx * dx;
    d2 = d2 + dy * dy;
    d2 = d2 + dz * dz;
    float rk = t->rof[k];
    float thr = 1.5f * rk;
    thr = thr + s->ro;
    float gap[3];
    for (int a = 0; a < 3; a++) {
        float g1 = s->lo[a] - t->hif[3 * k + a];
        float g2 = t->lof[3 * k + a] - s->hi[a];
        float g = g1 > g2 ? g1 : g2;
        gap[a] = g > 0.0f ? g : 0.0f;
    }
    float gap2 = gap[0] * gap[0];
    gap2 = gap2 + gap[1] * gap[1];
    gap2 = gap2 + gap[2] * gap[2];
    if (d2 > thr * thr && gap2 >= four_eps2) return O_ACCEPT;
    if (!k_group) {
        if (s->pointlike || s->ro <= rk) return O_DEFER;
        return O_OPEN;
    }
    if (s->pointlike) return O_PP;
    float u = s->ro + t->bmaxf[k];
    if (d2 > u * u) return O_PC;
    if (s->leaf) return O_PP;
    return O_OPEN;
}

static void group_push(orc_fmm *t, long k, long s0, long s1, long s2, long s3, const double *L)
{
    if (t->ng == t->gcap) {
        t->gcap = t->gcap ? 2 * t->gcap : 1024;
        t->gcell = realloc(t->gcell, t->gcap * sizeof(long));
        t->gseg = realloc(t->gseg, 4 * t->gcap * sizeof(long));
        t->gL = realloc(t->gL, NMI * t->gcap * sizeof(double));
    }
    t->gcell[t->ng] = k;
    t->gseg[4 * t->ng] = s0;
    t->gseg[4 * t->ng + 1] = s1;
    t->gseg[4 * t->ng + 2] = s2;
    t->gseg[4 * t->ng + 3] = s3;
    memcpy(t->gL + NMI * t->ng, L, NMI * sizeof(double));
    t->ng++;
}

static void walk(orc_fmm *t, long k, const entry *cl, long ncl, const double *Lpar, long par)
{
    double L[NMI];
    if (par < 0) {
        for (int i = 0; i < NMI; i++) L[i] = 0.0;
    } else {
        double tv[3] = {t->com[3 * k] - t->com[3 * par], t->com[3 * k + 1] - t->com[3 * par + 1],
                        t->com[3 * k + 2] - t->com[3 * par + 2]};
        orc_l2l(Lpar, tv, L);
    }
    int kg = t->count[k] <= t->g;
    float e2 = (float)(2.0 * t->eps);
    float four_eps2 = e2 * e2;
    double eps2 = t->eps * t->eps;
    long cap = ncl + 64, nq = ncl, nd = 0, capd = ncl + 64;
    entry *q = malloc(cap * sizeof(entry));
    entry *def = malloc(capd * sizeof(entry));
    memcpy(q, cl, ncl * sizeof(entry));
    long pp0 = t->lists[K_PP].n, pc0 = t->lists[K_PC].n;
    const double *ck = t->com + 3 * k;
    for (long i = 0; i < nq; i++) {
        entry e = q[i];
        sgeom s;
        entry_geom(t, e, &s);
        int o = decide(t, k, &s, kg, four_eps2);
        long sf = e.particle ? e.id : t->first[e.id];
        long sn = e.particle ? 1 : t->count[e.id];
        switch (o) {
        case O_ACCEPT:
            if (s.pointlike) {
                double xs[3] = {t->X[sf] + e.sh[0], t->Y[sf] + e.sh[1], t->Z[sf] + e.sh[2]};
                p2l_acc(t->m[sf], xs, ck, eps2, L);
                elist_push(&t->lists[K_CP], k, sf, 1, e.particle ? -1 : e.id, e.sh);
            } else {
                const double *cs = t->com + 3 * e.id;
                double zs[3] = {cs[0] + e.sh[0], cs[1] + e.sh[1], cs[2] + e.sh[2]};
                m2l_acc(t->mom + NM4 * e.id, zs, ck, eps2, L);
                elist_push(&t->lists[K_CC], k, sf, sn, e.id, e.sh);
            }
            break;
        case O_DEFER:
            if (nd == capd) {
                capd *= 2;
                def = realloc(def, capd * sizeof(entry));
            }
            def[nd++] = e;
            break;
        case O_PC:
            elist_push(&t->lists[K_PC], k, sf, sn, e.id, e.sh);
            break;
        case O_PP:
            elist_push(&t->lists[K_PP], k, sf, sn, e.particle ? -1 : e.id, e.sh);
            break;
        case O_OPEN: {
            long c = e.id;
            long add = (t->count[c] <= t->b) ? t->count[c] : 2;
            if (nq + add > cap) {
                while (nq + add > cap) cap *= 2;
                q = realloc(q, cap * sizeof(entry));
            }
            /* the children (or a leaf's particles) stay in the same copy */
            if (t->count[c] <= t->b) {
                for (long j = 0; j < t->count[c]; j++) {
                    q[nq] = e;
                    q[nq].id = t->first[c] + j;
                    q[nq].particle = 1;
                    nq++;
                }
            } else {
                q[nq] = e;
                q[nq].id = t->child[2 * c];
                nq++;
                q[nq] = e;
                q[nq].id = t->child[2 * c + 1];
                nq++;
            }
        } break;
        }
    }
    free(q);
    if (kg) {
        group_push(t, k, pp0, t->lists[K_PP].n, pc0, t->lists[K_PC].n, L);
    } else {
        for (int h = 0; h < 2; h++) {
            long c = t->child[2 * k + h];
            if (t->nact[c] > 0) walk(t, c, def, nd, L, k);
        }
    }
    free(def);
}

void orc_fmm_free(orc_fmm *t);

static orc_fmm *fmm_create(long n, const double *pos, const double *mass, const unsigned char *active, double eps,
                          double theta, int b, int g, int nrep)
{
    if (!tables_ready) make_tables();
    orc_fmm *t = calloc(1, sizeof(orc_fmm));
    t->n = n;
    t->b = b;
    t->g = g;
    t->eps = eps;
    t->theta = theta;
    t->nrep = nrep;
    if (n <= 0) return t;
    t->key = malloc(n * sizeof(uint64_t));
    t->perm = malloc(n * sizeof(long));
    for (long i = 0; i < n; i++) {
        t->key[i] = morton_key(pos[i], pos[n + i], pos[2 * n + i]);
        t->perm[i] = i;
    }
    qsort_r(t->perm, n, sizeof(long), cmp_key, t->key);
    uint64_t *ks = malloc(n * sizeof(uint64_t));
    t->X = malloc(n * sizeof(double));
    t->Y = malloc(n * sizeof(double));
    t->Z = malloc(n * sizeof(double));
    t->m = malloc(n * sizeof(double));
    t->act = malloc(n);
    for (long i = 0; i < n; i++) {
        long p = t->perm[i];
        ks[i] = t->key[p];
        t->X[i] = pos[p];
        t->Y[i] = pos[n + p];
        t->Z[i] = pos[2 * n + p];
        t->m[i] = mass[p];
        t->act[i] = active ? (active[p] != 0) : 1;
    }
    free(t->key);
    t->key = ks;
    long cap = 2 * n + 1;
    t->first = malloc(cap * sizeof(long));
    t->count = malloc(cap * sizeof(long));
    t->child = malloc(2 * cap * sizeof(long));
    t->parent = malloc(cap * sizeof(long));
    t->level = malloc(cap * sizeof(long));
    t->nact = malloc(cap * sizeof(long));
    build_rec(t, 0, n, -1, 0);
    long nc = t->nc;
    t->mass = malloc(nc * sizeof(double));
    t->com = malloc(3 * nc * sizeof(double));
    t->lo = malloc(3 * nc * sizeof(double));
    t->hi = malloc(3 * nc * sizeof(double));
    t->bmax = malloc(nc * sizeof(double));
    t->mom = malloc(NM4 * nc * sizeof(double));
    t->comf = malloc(3 * nc * sizeof(float));
    t->lof = malloc(3 * nc * sizeof(float));
    t->hif = malloc(3 * nc * sizeof(float));
    t->bmaxf = malloc(nc * sizeof(float));
    t->rof = malloc(nc * sizeof(float));
#pragma omp parallel for schedule(dynamic, 64)
    for (long c = 0; c < nc; c++) cell_props(t, c);
    if (t->nact[0] > 0) {
        /* the checklist starts with the root, and in a periodic box with its copies of the shell */
        int R = nrep > 0 ? nrep : 0;
        long ne = 0;
        entry *cl = malloc((2 * R + 1) * (2 * R + 1) * (2 * R + 1) * sizeof(entry));
        for (int sx = -R; sx <= R; sx++)
            for (int sy = -R; sy <= R; sy++)
                for (int sz = -R; sz <= R; sz++) {
                    entry e = {0, 0, {sx, sy, sz}};
                    cl[ne++] = e;
                }
        walk(t, 0, cl, ne, NULL, -1);
        free(cl);
    }
    return t;
}

orc_fmm *orc_fmm_create(long n, const double *pos, const double *mass, const unsigned char *active, double eps,
                        double theta, int b, int g)
{
    return fmm_create(n, pos, mass, active, eps, theta, b, g, -1);
}

/* periodic unit box (Sec. 3.1): the walk starts from the root and its copies |n|_inf <= nrep
 * (26 copies for nrep = 1, 124 for nrep = 2); the copies beyond come from the Ewald correction */
orc_fmm *orc_fmm_create_periodic(long n, const double *pos, const double *mass, const unsigned char *active,
                                 double eps, double theta, int b, int g, int nrep)
{
    if (nrep < 0 || nrep > 2) return NULL;
    return fmm_create(n, pos, mass, active, eps, theta, b, g, nrep);
}

/* evaluate the lists: terms bit 1 = PP, 2 = PC, 4 = local expansion (CC+CP), 8 = the Ewald correction
 * of a periodic box (the root's moments, 5th order).
 * acc (3n SoA) and pot (n) in the caller's original order; inactive particles untouched. */
int orc_fmm_eval(orc_fmm *t, int terms, double *acc, double *pot)
{
    long n = t->n;
    double eps2 = t->eps * t->eps;
#pragma omp parallel for schedule(dynamic, 4)
    for (long gi = 0; gi < t->ng; gi++) {
        long k = t->gcell[gi];
        const long *seg = t->gseg + 4 * gi;
        const double *L = t->gL + NMI * gi;
        for (long i = t->first[k]; i < t->first[k] + t->count[k]; i++) {
            if (!t->act[i]) continue;
            double a[3] = {0, 0, 0}, ph = 0.0;
            double xi[3] = {t->X[i], t->Y[i], t->Z[i]};
            if (terms & 1) {
                for (long e = seg[0]; e < seg[1]; e++) {
                    long f = t->lists[K_PP].first[e], c = t->lists[K_PP].count[e];
                    double sv[3];
                    shift_of(t->lists[K_PP].shift[e], sv);
                    int same = sv[0] == 0.0 && sv[1] == 0.0 && sv[2] == 0.0;
                    for (long j = f; j < f + c; j++) {
                        if (j == i && same) continue;
                        double dx = (t->X[j] + sv[0]) - xi[0], dy = (t->Y[j] + sv[1]) - xi[1],
                               dz = (t->Z[j] + sv[2]) - xi[2];
                        double R2 = dx * dx + dy * dy + dz * dz + eps2;
                        double iR = 1.0 / sqrt(R2);
                        double miR = t->m[j] * iR, miR3 = miR * iR * iR;
                        a[0] += miR3 * dx;
                        a[1] += miR3 * dy;
                        a[2] += miR3 * dz;
                        ph -= miR;
                    }
                }
            }
            if (terms & 2) {
                for (long e = seg[2]; e < seg[3]; e++) {
                    long s = t->lists[K_PC].cell[e];
                    double sv[3];
                    shift_of(t->lists[K_PC].shift[e], sv);
                    const double *cs = t->com + 3 * s;
                    double zs[3] = {cs[0] + sv[0], cs[1] + sv[1], cs[2] + sv[2]};
                    m2p_acc(t->mom + NM4 * s, zs, xi, eps2, a, &ph);
                }
            }
            if (terms & 4) {
                double u[3] = {xi[0] - t->com[3 * k], xi[1] - t->com[3 * k + 1], xi[2] - t->com[3 * k + 2]};
                l2p_acc(L, u, a, &ph);
            }
            if ((terms & 8) && t->nrep >= 0) {
                double ea[3], ep;
                orc_ewald_m2p(t->mom, t->com, xi, t->nrep, 3.0, ea, &ep);
                for (int q = 0; q < 3; q++) a[q] += ea[q];
                ph += ep;
            }
            long p = t->perm[i];
            acc[p] = a[0];
            acc[n + p] = a[1];
            acc[2 * n + p] = a[2];
            pot[p] = ph;
        }
    }
    return 0;
}

long orc_fmm_ncell(const orc_fmm *t) { return t->nc; }
long orc_fmm_ngroup(const orc_fmm *t) { return t->ng; }
long orc_fmm_nentries(const orc_fmm *t, int kind) { return t->lists[kind].n; }

void orc_fmm_perm(const orc_fmm *t, long *perm) { memcpy(perm, t->perm, t->n * sizeof(long)); }
void orc_fmm_keys(const orc_fmm *t, uint64_t *k) { memcpy(k, t->key, t->n * sizeof(uint64_t)); }

void orc_fmm_cells(const orc_fmm *t, long *first, long *count, long *parent, long *child, long *nact, double *mass,
                   double *com, double *lo, double *hi, double *bmax, double *mom)
{
    long nc = t->nc;
    memcpy(first, t->first, nc * sizeof(long));
    memcpy(count, t->count, nc * sizeof(long));
    memcpy(parent, t->parent, nc * sizeof(long));
    memcpy(child, t->child, 2 * nc * sizeof(long));
    memcpy(nact, t->nact, nc * sizeof(long));
    memcpy(mass, t->mass, nc * sizeof(double));
    memcpy(com, t->com, 3 * nc * sizeof(double));
    memcpy(lo, t->lo, 3 * nc * sizeof(double));
    memcpy(hi, t->hi, 3 * nc * sizeof(double));
    memcpy(bmax, t->bmax, nc * sizeof(double));
    memcpy(mom, t->mom, NM4 * nc * sizeof(double));
}

void orc_fmm_entries(const orc_fmm *t, int kind, long *sink, long *first, long *count)
{
    const elist *l = &t->lists[kind];
    memcpy(sink, l->sink, l->n * sizeof(long));
    memcpy(first, l->first, l->n * sizeof(long));
    memcpy(count, l->count, l->n * sizeof(long));
}

/* the copy of each entry's source, as (sx, sy, sz) triples */
void orc_fmm_entry_shifts(const orc_fmm *t, int kind, int *out)
{
    const elist *l = &t->lists[kind];
    for (long e = 0; e < l->n; e++) {
        double v[3];
        shift_of(l->shift[e], v);
        for (int a = 0; a < 3; a++) out[3 * e + a] = (int)v[a];
    }
}

void orc_fmm_groups(const orc_fmm *t, long *cell, double *L)
{
    memcpy(cell, t->gcell, t->ng * sizeof(long));
    memcpy(L, t->gL, NMI * t->ng * sizeof(double));
}

/* out: [pp pairs, pc pairs, cc entries, cp entries, groups, cells, buckets, depth] */
void orc_fmm_counts(const orc_fmm *t, long *out)
{
    long npp = 0, npc = 0;
    for (long gi = 0; gi < t->ng; gi++) {
        long k = t->gcell[gi];
        long na = t->nact[k];
        const long *seg = t->gseg + 4 * gi;
        long src = 0;
        for (long e = seg[0]; e < seg[1]; e++) src += t->lists[K_PP].count[e];
        npp += na * src;
        npc += na * (seg[3] - seg[2]);
    }
    long nb = 0;
    for (long c = 0; c < t->nc; c++) nb += (t->count[c] <= t->b);
    out[0] = npp;
    out[1] = npc;
    out[2] = t->lists[K_CC].n;
    out[3] = t->lists[K_CP].n;
    out[4] = t->ng;
    out[5] = t->nc;
    out[6] = nb;
    out[7] = t->depth;
}

void orc_fmm_free(orc_fmm *t)
{
    if (!t) return;
    void *ps[] = {t->perm, t->key, t->X, t->Y, t->Z, t->m, t->act, t->first, t->count, t->child, t->parent,
                  t->nact, t->level, t->mass, t->com, t->lo, t->hi, t->bmax, t->mom, t->comf, t->lof, t->hif,
                  t->bmaxf, t->rof, t->gcell, t->gseg, t->gL};
    for (size_t i = 0; i < sizeof(ps) / sizeof(ps[0]); i++) free(ps[i]);
    for (int k = 0; k < 4; k++) {
        free(t->lists[k].sink);
        free(t->lists[k].first);
        free(t->lists[k].count);
        free(t->lists[k].cell);
        free(t->lists[k].shift);
    }
    free(t);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
