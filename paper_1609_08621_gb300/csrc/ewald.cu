// Ewald correction of the periodic unit box (Sec. 3.1, periodic boundaries; Sec. 3.3, the
// Ewald evaluation on the GPU).
//
// In a periodic box the walk starts from the root and its copies n, |n|_inf <= R (26 or 124), and
// the copies beyond that shell enter through a 5th-order multipole approximation of the Ewald sum.
// The sum approximated, for a sink at x and the box's mass distribution:
//     K(r) = sum_{|n|_inf <= R} G(r + n) + F(r),   F(r) = psi(r) - sum_{|n|_inf <= R} 1 / |r + n|,
// where G is the softened kernel of the walk and psi the periodic Newtonian potential of a unit mass
// with a uniform background of the mean density and zero mean over the box:
//     psi(r) = sum_n erfc(alpha |r + n|) / |r + n|
//            + sum_{h != 0} exp(-pi^2 h^2 / alpha^2) / (pi h^2) cos(2 pi h.r) - pi / alpha^2
// (Ewald's split; psi does not depend on alpha > 0).  F is smooth for every offset between two
// points of the box.  With the root's moments M_n (|n| <= 4, about its centre of mass z) the
// correction field is
//     Phi_E(x) = sum_n (-1)^|n| / n! M_n D^n F(x - z),   acceleration += grad Phi_E, potential -= Phi_E.
//
// On this GPU FP64 runs at 1/64 of the FP32 rate, so the correction is not evaluated per particle
// as the paper does.  Phi_E is smooth over the whole box (its nearest singularity lies beyond the
// replica shell, >= 1.1 away), so once per solve, in FP64, its Taylor expansion to order EW_P is
// formed about the centre y_c of each of EW_G^3 sub-cubes of the box:
//     E_k(y_c) = D^k Phi_E(y_c) = sum_n (-1)^|n| / n! M_n D^(n+k) F(y_c - z),   |k| <= EW_P,
// which needs the derivatives of F to order EW_P + 4 at EW_G^3 points.  Each group re-expands its
// sub-cube's polynomial at its own centre of mass, keeping order 5 there,
//     L_k(c_g) = sum_j E_(k+j)(y_c) t^j / j!,   t = c_g - y_c,  |k| <= 5,  |k + j| <= EW_P,
// adds it to the local expansion of its walk, and L2P evaluates both.  The Taylor remainder on a
// sub-cube of side 1/4 (|t| <= sqrt(3)/8) falls about as (|t| / 1.1)^(EW_P + 1).  Measured against
// the oracle's per-particle correction on a clustered box with a tenth of its particles at the
// faces, relative to each particle's total acceleration: rms 4.0e-5 (maximum 1.1e-3) for a grid of
// order-5 expansions, rms 8.8e-6 (maximum 1.6e-4) for order 7 and the same for order 9, where the
// FP32 coefficients and their re-expansion set the floor; order 7 is the default.
//
// Derivatives of a radial function f(s), s = u.u, follow the recursion of Hermite-type tensors
// (as in McMurchie and Davidson's integral scheme): with R^(n)_0 = 2^n f^(n)(s) and
//     R^(n)_(m + e_a) = u_a R^(n+1)_m + m_a R^(n+1)_(m - e_a)     (Leibniz on 2 u_a f'(s)),
// R^(0)_m = D^m f(u).  Multi-indices m = (a, b, c) are ordered by total order, then a descending,
// then b descending (the order of the local coefficients).
#include <math.h>

#include "expansions.cuh"
#include "fmm_internal.cuh"

#ifndef EW_P
#define EW_P 7  // order of the sub-cube expansions
#endif
#define EW_G 4                                      // sub-cubes per axis
#define EW_NG (EW_G * EW_G * EW_G)                  // expansion centres
#define EW_D (EW_P + 4)                             // derivative order: moments (4) + expansion
#define EW_NI(o) (((o) + 1) * ((o) + 2) * ((o) + 3) / 6)  // multi-indices of order <= o
#define EW_ND EW_NI(EW_D)
#define EW_NP EW_NI(EW_P)
#define EW_ALPHA 2.5  // Ewald split parameter
#define EW_CUT 8.0    // real-space copies with alpha |r+n| >= 8 and reciprocal vectors with
                      // pi |h| / alpha >= 8 lie far below FP64 rounding
#define EW_HMAX 7     // ceil(EW_CUT * EW_ALPHA / pi)
#define EW_THREADS 256
#define EW_WARPS (EW_THREADS / 32)
#define EW_HCHUNK 64  // reciprocal vectors staged per round

static_assert(FMM_NL == EW_NI(5), "the group expansions are of order 5");

// position of multi-index (a, b, c) in the ordering above
__device__ __forceinline__ int ew_index(int a, int b, int c)
{
    const int o = a + b + c;
    return o * (o + 1) * (o + 2) / 6 + (o - a) * (o - a + 1) / 2 + (o - a - b);
}

// multi-index at position i
__device__ __forceinline__ void ew_multi(int i, int& a, int& b, int& c)
{
    int o = 0;
    while (EW_NI(o) <= i) o++;
    int r = i - (o > 0 ? EW_NI(o - 1) : 0);
    a = o;
    while (r > o - a) {
        r -= o - a + 1;
        a--;
    }
    b = o - a - r;
    c = o - a - b;
}

// s-derivatives d[l] = (d/ds)^l g(s), l <= EW_D, of g(s) = erfc(alpha sqrt s) / sqrt s (outside
// the replica shell) or g(s) = -erf(alpha sqrt s) / sqrt s (inside it: the Newtonian copy the walk
// covers with G is taken out of psi).  With B_0 = erfc(alpha r) / r and
//     B_l = (-(1/r) d/dr)^l B_0 = ((2l - 1) B_(l-1) + (2 alpha^2)^l exp(-alpha^2 r^2) / (alpha sqrt pi)) / r^2,
// (d/ds)^l = (1/(2r) d/dr)^l gives d[l] = (-1/2)^l B_l.  -erf/r = erfc/r - 1/r, and
// (d/ds)^l s^(-1/2) = (-1/2)^l (2l - 1)!! s^(-l-1/2).  Near r = 0, where that difference cancels,
// -erf(alpha r)/r comes from its power series instead:
//     -erf(alpha sqrt s)/sqrt s = -(2 alpha / sqrt pi) sum_k (-alpha^2 s)^k / (k! (2k + 1)),
//     d[l] = -(2 alpha / sqrt pi) (-alpha^2)^l sum_j (-alpha^2 s)^j / (j! (2l + 2j + 1)).
__device__ void ew_scalars(double s, bool shell, double* d)
{
    const double al = EW_ALPHA, a2 = al * al;
    const double rpi = 1.7724538509055160273;  // sqrt(pi)
    if (shell && a2 * s < 2.25) {
        const double c = -2.0 * al / rpi;
        double pl = 1.0;  // (-alpha^2)^l
        for (int l = 0; l <= EW_D; l++) {
            double sum = 0.0, t = 1.0;  // t = (-a2 s)^j / j!
            for (int j = 0; j < 40; j++) {
                sum += t / (2.0 * (l + j) + 1.0);
                t *= -a2 * s / (j + 1.0);
            }
            d[l] = c * pl * sum;
            pl *= -a2;
        }
        return;
    }
    const double r = sqrt(s);
    const double g = exp(-a2 * s) / (al * rpi);
    double B = erfc(al * r) / r, p = 1.0, h = 1.0, dfac = 1.0, sl = 1.0;  // h = (-1/2)^l, sl = s^l
    d[0] = shell ? B - 1.0 / r : B;
    for (int l = 1; l <= EW_D; l++) {
        p *= 2.0 * a2;
        B = ((2.0 * l - 1.0) * B + p * g) / s;
        h *= -0.5;
        dfac *= 2.0 * l - 1.0;
        sl *= s;
        d[l] = h * B;
        if (shell) d[l] -= h * dfac / (r * sl);
    }
}

// Deterministic compaction over the block: the position of this thread's kept item among the
// kept items of the round, in thread order, and their number.  Every thread of the block calls it.
__device__ __forceinline__ int ew_compact(bool keep, int* wsum, int& total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned int m = __ballot_sync(FMM_FULL_MASK, keep);
    if (lane == 0) wsum[w] = __popc(m);
    __syncthreads();
    int off = 0, tot = 0;
    for (int i = 0; i < EW_WARPS; i++) {
        if (i < w) off += wsum[i];
        tot += wsum[i];
    }
    __syncthreads();
    total = tot;
    return off + __popc(m & fmm_lanemask_lt());
}

struct EwaldSmem {
    double su[EW_THREADS][3];             // kept copies of one round: u = r + n
    double sd[EW_THREADS][EW_D + 1];      // and their s-derivative scalars
    double R[EW_WARPS][2][EW_ND];         // per warp: two levels of the recursion
    double acc[EW_WARPS][EW_ND];          // per warp: sum of its copies' D^m
    double hp[EW_HCHUNK][3][EW_D + 1];    // reciprocal vectors: powers (2 pi h_a)^p
    double hc[EW_HCHUNK][2];              // coef * (cos, sin) of 2 pi h.r
    double D[EW_ND];                      // D^m F(r)
    // recursion table per entry m (|m| >= 1): the axis a it recurses along, m_a, and the
    // positions of m - e_a and m - 2 e_a (-1 when m_a < 2)
    short i1[EW_ND], i2[EW_ND];
    unsigned char ax[EW_ND], ma[EW_ND];
    int wsum[EW_WARPS];
};

size_t fmm_ewald_smem() { return sizeof(EwaldSmem); }

// One block per sub-cube centre y_c: D^m F(y_c - z) for |m| <= EW_D, then the expansion of the
// correction field from the root's moments.  rec: the root's moment record (FP32: M, M2 (6),
// M3 (10), M4 (15)); E: EW_NP FP32 coefficients per centre.
__global__ void __launch_bounds__(EW_THREADS) k_ewald_grid(const Com4* __restrict__ com, const float* __restrict__ rec,
                                                           int root, int R, float* __restrict__ E)
{
    extern __shared__ __align__(16) unsigned char ew_raw[];
    EwaldSmem& S = *reinterpret_cast<EwaldSmem*>(ew_raw);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int cx = blockIdx.x % EW_G, cy = (blockIdx.x / EW_G) % EW_G, cz = blockIdx.x / (EW_G * EW_G);
    const Com4 z = com[root];
    const double r[3] = {(cx + 0.5) / EW_G - z.x, (cy + 0.5) / EW_G - z.y, (cz + 0.5) / EW_G - z.z};
    for (int i = lane; i < EW_ND; i += 32) S.acc[w][i] = 0.0;
    for (int i = tid; i < EW_ND; i += EW_THREADS) {
        int a = 0, b = 0, c = 0;
        ew_multi(i, a, b, c);
        const int x = a > 0 ? 0 : (b > 0 ? 1 : 2);  // the first axis with a non-zero index
        const int m = x == 0 ? a : (x == 1 ? b : c);
        S.ax[i] = (unsigned char)x;
        S.ma[i] = (unsigned char)m;
        S.i1[i] = i == 0 ? -1 : (short)ew_index(a - (x == 0), b - (x == 1), c - (x == 2));
        S.i2[i] = m < 2 ? -1 : (short)ew_index(a - 2 * (x == 0), b - 2 * (x == 1), c - 2 * (x == 2));
    }
    __syncthreads();
    // real space: the shell's copies (-erf) and every copy beyond it within the cut (erfc), in
    // rounds of EW_THREADS candidates n; each warp runs the recursion for every EW_WARPS-th copy
    const double cut = EW_CUT / EW_ALPHA;
    const int nmax = R + (int)ceil(cut) + 1, wd = 2 * nmax + 1, ncand = wd * wd * wd;
    for (int c0 = 0; c0 < ncand; c0 += EW_THREADS) {
        const int ci = c0 + tid;
        bool keep = false, shell = false;
        double u0 = 0.0, u1 = 0.0, u2 = 0.0, s = 0.0;
        if (ci < ncand) {
            const int nx = ci % wd - nmax, ny = (ci / wd) % wd - nmax, nz = ci / (wd * wd) - nmax;
            u0 = r[0] + nx;
            u1 = r[1] + ny;
            u2 = r[2] + nz;
            s = u0 * u0 + u1 * u1 + u2 * u2;
            shell = abs(nx) <= R && abs(ny) <= R && abs(nz) <= R;
            keep = shell || s < cut * cut;
        }
        int nk = 0;
        const int slot = ew_compact(keep, S.wsum, nk);
        if (keep) {
            double d[EW_D + 1];
            ew_scalars(s, shell, d);
            S.su[slot][0] = u0;
            S.su[slot][1] = u1;
            S.su[slot][2] = u2;
            for (int l = 0; l <= EW_D; l++) S.sd[slot][l] = d[l];
        }
        __syncthreads();
        for (int q = w; q < nk; q += EW_WARPS) {
            const double ux[3] = {S.su[q][0], S.su[q][1], S.su[q][2]};
            // level n = EW_D holds R^(EW_D)_0 only; each level below adds one order
            double* prev = S.R[w][0];
            double* cur = S.R[w][1];
            if (lane == 0) prev[0] = ldexp(S.sd[q][EW_D], EW_D);
            __syncwarp();
            for (int n = EW_D - 1; n >= 0; n--) {
                const int cnt = EW_NI(EW_D - n);
                for (int i = lane; i < cnt; i += 32) {
                    double v;
                    if (i == 0) {
                        v = ldexp(S.sd[q][n], n);
                    } else {
                        v = ux[S.ax[i]] * prev[S.i1[i]];
                        if (S.i2[i] >= 0) v += (double)(S.ma[i] - 1) * prev[S.i2[i]];
                    }
                    cur[i] = v;
                }
                __syncwarp();
                double* t = prev;
                prev = cur;
                cur = t;
            }
            for (int i = lane; i < EW_ND; i += 32) S.acc[w][i] += prev[i];
            __syncwarp();
        }
        __syncthreads();
    }
    // reciprocal space over the half space of h (h and -h together): coef = 2 exp(-pi^2 h^2 /
    // alpha^2) / (pi h^2), D^m cos(2 pi h.r) = (2 pi h)^m cos(2 pi h.r + |m| pi / 2); the vectors
    // are compacted in candidate order and staged with their powers
    const double PI = 3.14159265358979323846;
    const int hw = 2 * EW_HMAX + 1, nh = (EW_HMAX + 1) * hw * hw;
    double dm[(EW_ND + EW_THREADS - 1) / EW_THREADS];  // this thread's components m = tid + k * EW_THREADS
    int ma[(EW_ND + EW_THREADS - 1) / EW_THREADS], mb[(EW_ND + EW_THREADS - 1) / EW_THREADS],
        mc[(EW_ND + EW_THREADS - 1) / EW_THREADS];
#pragma unroll
    for (int k = 0; k < (EW_ND + EW_THREADS - 1) / EW_THREADS; k++) {
        dm[k] = 0.0;
        ma[k] = mb[k] = mc[k] = 0;
        if (tid + k * EW_THREADS < EW_ND) ew_multi(tid + k * EW_THREADS, ma[k], mb[k], mc[k]);
    }
    for (int c0 = 0; c0 < nh; c0 += EW_THREADS) {
        const int hi = c0 + tid;
        bool keep = false;
        int hx = 0, hy = 0, hz = 0;
        double h2 = 0.0;
        if (hi < nh) {
            hx = hi / (hw * hw);
            hy = (hi / hw) % hw - EW_HMAX;
            hz = hi % hw - EW_HMAX;
            const bool half = hx > 0 || (hx == 0 && (hy > 0 || (hy == 0 && hz > 0)));
            h2 = (double)hx * hx + (double)hy * hy + (double)hz * hz;
            keep = half && PI * sqrt(h2) / EW_ALPHA < EW_CUT;
        }
        int nk = 0;
        const int slot = ew_compact(keep, S.wsum, nk);
        // stage the kept vectors EW_HCHUNK at a time (slot order)
        for (int b0 = 0; b0 < nk; b0 += EW_HCHUNK) {
            if (keep && slot >= b0 && slot < b0 + EW_HCHUNK) {
                const int j = slot - b0;
                const double coef = 2.0 * exp(-PI * PI * h2 / (EW_ALPHA * EW_ALPHA)) / (PI * h2);
                const double th = 2.0 * PI * (hx * r[0] + hy * r[1] + hz * r[2]);
                S.hc[j][0] = coef * cos(th);
                S.hc[j][1] = coef * sin(th);
                const double k3[3] = {2.0 * PI * hx, 2.0 * PI * hy, 2.0 * PI * hz};
                for (int ax = 0; ax < 3; ax++) {
                    double p = 1.0;
                    for (int e = 0; e <= EW_D; e++) {
                        S.hp[j][ax][e] = p;
                        p *= k3[ax];
                    }
                }
            }
            __syncthreads();
            const int nb = min(EW_HCHUNK, nk - b0);
#pragma unroll
            for (int k = 0; k < (EW_ND + EW_THREADS - 1) / EW_THREADS; k++) {
                if (tid + k * EW_THREADS >= EW_ND) continue;
                const int ph = (ma[k] + mb[k] + mc[k]) & 3;  // cos, -sin, -cos, sin
                const int cs = (ph & 1) ? 1 : 0;
                const double sg = (ph == 1 || ph == 2) ? -1.0 : 1.0;
                double sum = 0.0;
                for (int j = 0; j < nb; j++)
                    sum += S.hp[j][0][ma[k]] * S.hp[j][1][mb[k]] * S.hp[j][2][mc[k]] * S.hc[j][cs];
                dm[k] += sg * sum;
            }
            __syncthreads();
        }
    }
    // D^m F = the warps' real-space sums (in warp order) + the reciprocal sum; the constant
    // -pi / alpha^2 enters D^0
#pragma unroll
    for (int k = 0; k < (EW_ND + EW_THREADS - 1) / EW_THREADS; k++) {
        const int i = tid + k * EW_THREADS;
        if (i >= EW_ND) continue;
        double v = 0.0;
        for (int q = 0; q < EW_WARPS; q++) v += S.acc[q][i];
        v += dm[k];
        if (i == 0) v -= PI / (EW_ALPHA * EW_ALPHA);
        S.D[i] = v;
    }
    __syncthreads();
    // E_k = sum_n (-1)^|n| / n! M_n D^(n+k), moments of order 0, 2, 3, 4 (slot s >= 1 is
    // multi-index s + 3 of the ordering)
    for (int i = tid; i < EW_NP; i += EW_THREADS) {
        int ka, kb, kc;
        ew_multi(i, ka, kb, kc);
        double L = 0.0;
        for (int sl = 0; sl < FMM_NMOM; sl++) {
            int na = 0, nb = 0, nc = 0;
            if (sl > 0) ew_multi(sl + 3, na, nb, nc);
            double fact = 1.0;
            for (int q = 2; q <= na; q++) fact *= q;
            for (int q = 2; q <= nb; q++) fact *= q;
            for (int q = 2; q <= nc; q++) fact *= q;
            const double sign = ((na + nb + nc) & 1) ? -1.0 : 1.0;
            L += sign / fact * (double)rec[sl] * S.D[ew_index(na + ka, nb + kb, nc + kc)];
        }
        E[blockIdx.x * EW_NP + i] = (float)L;
    }
}

// One warp per group: the sub-cube's order-EW_P polynomial re-expanded at the group's centre of
// mass to order 5 (L_k = sum_j E_(k+j) t^j / j!), added to the walk's local expansion (keep_walk)
// or replacing it (the correction alone).  The (k, j) pairs, |k| <= 5, |k + j| <= EW_P, are listed
// once per block: pair p of output k holds the positions of k + j and of j.
#define EWG_WARPS 4
// the number of (k, j) pairs: sum over the orders o <= 5 of k of (o + 1)(o + 2)/2 EW_NI(EW_P - o)
__host__ __device__ constexpr int ew_pair_count()
{
    int t = 0;
    for (int o = 0; o <= 5; o++) t += (o + 1) * (o + 2) / 2 * EW_NI(EW_P - o);
    return t;
}
#define EWG_PAIRS ew_pair_count()
__global__ void __launch_bounds__(EWG_WARPS * 32) k_ewald_groups(const Group* __restrict__ groups,
                                                                 const unsigned long long* __restrict__ ngroups_dev,
                                                                 long long cap_groups, const Com4* __restrict__ com,
                                                                 const float* __restrict__ E, float* __restrict__ Lg,
                                                                 int keep_walk, const DevCounters* __restrict__ ctr)
{
    if (fmm_overflowed(ctr)) return;
    __shared__ float mono[EWG_WARPS][EW_NP], coef[EWG_WARPS][EW_NP];
    __shared__ short pk[EWG_PAIRS], pj[EWG_PAIRS];
    __shared__ int poff[FMM_NL + 1];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        int o = 0;
        for (int k = 0; k < FMM_NL; k++) {
            int a, b, c;
            ew_multi(k, a, b, c);
            poff[k] = o;
            o += EW_NI(EW_P - (a + b + c));
        }
        poff[FMM_NL] = o;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < FMM_NL; k += blockDim.x) {
        int ka, kb, kc;
        ew_multi(k, ka, kb, kc);
        for (int j = 0, p = poff[k]; p < poff[k + 1]; j++, p++) {
            int ja, jb, jc;
            ew_multi(j, ja, jb, jc);
            pk[p] = (short)ew_index(ka + ja, kb + jb, kc + jc);
            pj[p] = (short)j;
        }
    }
    __syncthreads();
    const long long ng = (long long)min(*ngroups_dev, (unsigned long long)cap_groups);
    const long long nw = (long long)gridDim.x * EWG_WARPS;
    for (long long gi = (long long)blockIdx.x * EWG_WARPS + wl; gi < ng; gi += nw) {
        const Com4 c = com[groups[gi].cell];
        const int ix = min(max((int)floor(c.x * EW_G), 0), EW_G - 1);
        const int iy = min(max((int)floor(c.y * EW_G), 0), EW_G - 1);
        const int iz = min(max((int)floor(c.z * EW_G), 0), EW_G - 1);
        const int cell = ix + EW_G * (iy + EW_G * iz);
        const float t[3] = {__double2float_rn(c.x - (ix + 0.5) / EW_G), __double2float_rn(c.y - (iy + 0.5) / EW_G),
                            __double2float_rn(c.z - (iz + 0.5) / EW_G)};
        for (int i = lane; i < EW_NP; i += 32) {
            int a, b, cc;
            ew_multi(i, a, b, cc);
            float m = 1.0f;
            for (int q = 1; q <= a; q++) m *= t[0] / q;
            for (int q = 1; q <= b; q++) m *= t[1] / q;
            for (int q = 1; q <= cc; q++) m *= t[2] / q;
            mono[wl][i] = m;
            coef[wl][i] = E[cell * EW_NP + i];
        }
        __syncwarp();
        float* out = Lg + gi * FMM_NL;
        for (int k = lane; k < FMM_NL; k += 32) {
            float sum = 0.0f;
            for (int p = poff[k]; p < poff[k + 1]; p++) sum = fmaf(coef[wl][pk[p]], mono[wl][pj[p]], sum);
            out[k] = keep_walk ? out[k] + sum : sum;
        }
        __syncwarp();
    }
}

long long fmm_ewald_floats() { return (long long)EW_NG * EW_NP; }

static std::atomic<unsigned long long> g_ewald_attr{0};

// The sub-cube expansions need only the root's moments and centre of mass: they can run on a side
// stream beside the walk.
cudaError_t fmm_launch_ewald_grid(DevTree& t, int terms, cudaStream_t s)
{
    if (t.per_R <= 0 || !(terms & 8)) return cudaSuccess;
    if (!t.ewald_L) return cudaErrorInvalidValue;
    cudaError_t e = fmm_smem_attr_once(k_ewald_grid, (int)sizeof(EwaldSmem), g_ewald_attr);
    if (e != cudaSuccess) return e;
    k_ewald_grid<<<EW_NG, EW_THREADS, sizeof(EwaldSmem), s>>>(t.com, t.rec, 0, t.per_R, t.ewald_L);
    return cudaGetLastError();
}

// After the walk's local expansions of the groups (and the sub-cube expansions).
cudaError_t fmm_launch_ewald_groups(DevTree& t, DevWalk& w, DevCounters* ctr, int terms, cudaStream_t s)
{
    if (t.per_R <= 0 || !(terms & 8)) return cudaSuccess;
    const long long blocks = std::min<long long>(std::max<long long>(fmm_ceil_div(w.cap_groups, EWG_WARPS), 1), 152 * 16);
    k_ewald_groups<<<(unsigned)blocks, EWG_WARPS * 32, 0, s>>>(w.groups, &ctr->n_groups, w.cap_groups, t.com,
                                                                t.ewald_L, w.Lg, (terms & 4) ? 1 : 0, ctr);
    return cudaGetLastError();
}
