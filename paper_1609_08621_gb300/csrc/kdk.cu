// Individual time steps on rungs with the hierarchical kick-drift-kick leapfrog (Sec. 3.2).
//
// Particle i sits on rung r_i with step dt0 / 2^r_i (Sec. 3.2: time steps restricted to
// 2^-l of the base step).  The base step is cut into 2^R substeps of h = dt0 / 2^R; a
// particle is active at substep s when s is a multiple of 2^(R - r_i), i.e. where its
// kicks line up with those of the coarser rungs (Fig. KDK).  At substep s, for active
// particles: closing half kick with the force just computed, rung reassignment from
// Delta T_i = 0.2 sqrt(eps / |a_i|) (Sec. 3.2), opening half kick of the new step; then
// every particle drifts by h.  All of it in FP64.
//
// Rung choice is an integer decided by floating point, made reproducible by avoiding
// log2: r = the smallest r in [0, R] with dt0 <= Delta T * 2^r (scaling by 2^r is exact),
// with |a| = sqrt((ax^2 + ay^2) + az^2) and Delta T computed step by step without fused
// operations.  A particle may move to a coarser rung only at a substep where that rung
// is synchronised.
#include <math.h>

#include "f64bits.cuh"
#include "fmm_internal.cuh"

__device__ __forceinline__ int target_rung(float ax, float ay, float az, double eps, double dt0, int R)
{
    if (R == 0) return 0;  // a single rung: nothing to decide (and FP64 sqrt and division are slow here)
    double x = ax, y = ay, z = az;
    double a2 = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
    double am = __dsqrt_rn(a2);
    if (!(am > 0.0)) return 0;
    double dt = __dmul_rn(0.2, __dsqrt_rn(__ddiv_rn(eps, am)));
    int r = 0;
    while (r < R && dt0 > ldexp(dt, r)) r++;
    return r;
}

__global__ void k_assign_rungs(const float* __restrict__ acc, unsigned char* __restrict__ rung, long long n,
                               double eps, double dt0, int R)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    rung[i] = (unsigned char)target_rung(acc[i], acc[n + i], acc[2 * n + i], eps, dt0, R);
}

// dt0 2^-k as ldexp gives it, by one exact multiplication with the power of two built from its bits
__device__ __forceinline__ double pow2_scale(double dt0, int k)
{
    return __dmul_rn(dt0, fmm_dfrom((unsigned long long)(1023 - k) << 52));
}

// FP64 issues at 1/64 of the FP32 rate on this GPU: the kicks and the drift are FP64 arithmetic, while
// the widening of the FP32 accelerations and the box check of the new position use the encodings
// (f64bits.cuh) and give the same values.
__global__ void k_kick_drift(double* __restrict__ pos, double* __restrict__ vel, const float* __restrict__ acc,
                             unsigned char* __restrict__ rung, unsigned char* __restrict__ active_next, long long n,
                             double eps, double dt0, int R, long long s, int closing, unsigned int* __restrict__ status)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = rung[i];
    double vx = vel[i], vy = vel[n + i], vz = vel[2 * n + i];
    if ((s & ((1LL << (R - r)) - 1)) == 0) {
        float fx = acc[i], fy = acc[n + i], fz = acc[2 * n + i];
        double ax = fmm_f2d(fx), ay = fmm_f2d(fy), az = fmm_f2d(fz);
        if (closing) {
            double hk = pow2_scale(dt0, r + 1);
            vx += ax * hk;
            vy += ay * hk;
            vz += az * hk;
        }
        int rt = target_rung(fx, fy, fz, eps, dt0, R);
        int rn = rt;
        if (rt < r) {
            rn = rt;
            while (rn < r && (s & ((1LL << (R - rn)) - 1)) != 0) rn++;
        }
        r = rn;
        rung[i] = (unsigned char)r;
        double hk = pow2_scale(dt0, r + 1);
        vx += ax * hk;
        vy += ay * hk;
        vz += az * hk;
        vel[i] = vx;
        vel[n + i] = vy;
        vel[2 * n + i] = vz;
    }
    double h = pow2_scale(dt0, R);
    double x = pos[i] + vx * h, y = pos[n + i] + vy * h, z = pos[2 * n + i] + vz * h;
    if (!(fmm_in_unit(x) && fmm_in_unit(y) && fmm_in_unit(z))) atomicOr(status, FMM_DEV_ERR_ARG);
    pos[i] = x;
    pos[n + i] = y;
    pos[2 * n + i] = z;
    long long s1 = s + 1;
    active_next[i] = ((s1 & ((1LL << (R - r)) - 1)) == 0) ? 1 : 0;
}

cudaError_t fmm_launch_kick_drift(double* pos, double* vel, const float* acc, unsigned char* rung,
                                  unsigned char* active_next, long long n, double eps, double dt0, int max_rung,
                                  int substep, int closing, DevCounters* ctr, cudaStream_t s)
{
    k_kick_drift<<<(unsigned)fmm_ceil_div(n, 256), 256, 0, s>>>(pos, vel, acc, rung, active_next, n, eps, dt0,
                                                                max_rung, substep, closing, &ctr->status);
    return cudaGetLastError();
}

// The same schedule on compressed storage (Sec. 3.4, memory): positions as 32-bit fixed-point
// coordinates x = u 2^-32 of the unit box, velocities as FP32.  Within a substep the kicks are FP64
// (v = fl64(v32), v += a hk for each half kick, each product and sum rounded once: no fused
// operations), and the velocity is stored rounded to FP32.  The drift moves u by the nearest integer
// of v32 h 2^32, computed in FP64 (x 2^32 is exact), ties to even.  In the periodic box (periodic != 0)
// u wraps modulo 2^32, which is the box's periodicity; in the isolated box a particle leaving
// [0, 1) sets the argument error bit and keeps its old position.
__global__ void k_kick_drift_i32(unsigned int* __restrict__ ipos, float* __restrict__ vel,
                                 const float* __restrict__ acc, unsigned char* __restrict__ rung,
                                 unsigned char* __restrict__ active_next, long long n, double eps, double dt0, int R,
                                 long long s, int closing, int periodic, unsigned int* __restrict__ status)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = rung[i];
    float v32[3] = {vel[i], vel[n + i], vel[2 * n + i]};
    if ((s & ((1LL << (R - r)) - 1)) == 0) {
        const float f[3] = {acc[i], acc[n + i], acc[2 * n + i]};
        double v[3] = {v32[0], v32[1], v32[2]};
        if (closing) {
            const double hk = ldexp(dt0, -r - 1);
            for (int a = 0; a < 3; a++) v[a] = __dadd_rn(v[a], __dmul_rn((double)f[a], hk));
        }
        int rt = target_rung(f[0], f[1], f[2], eps, dt0, R);
        int rn = rt;
        if (rt < r) {
            rn = rt;
            while (rn < r && (s & ((1LL << (R - rn)) - 1)) != 0) rn++;
        }
        r = rn;
        rung[i] = (unsigned char)r;
        const double hk = ldexp(dt0, -r - 1);
        for (int a = 0; a < 3; a++) {
            v[a] = __dadd_rn(v[a], __dmul_rn((double)f[a], hk));
            v32[a] = __double2float_rn(v[a]);
            vel[a * n + i] = v32[a];
        }
    }
    const double h = ldexp(dt0, -R);
    long long u[3];
    bool out = false;
    for (int a = 0; a < 3; a++) {
        const long long d = __double2ll_rn(__dmul_rn(__dmul_rn((double)v32[a], h), 4294967296.0));
        u[a] = (long long)ipos[a * n + i] + d;
        if (periodic) u[a] &= 0xffffffffLL;
        else if (u[a] < 0 || u[a] > 0xffffffffLL) out = true;
    }
    if (out) {
        atomicOr(status, FMM_DEV_ERR_ARG);
    } else {
        for (int a = 0; a < 3; a++) ipos[a * n + i] = (unsigned int)u[a];
    }
    long long s1 = s + 1;
    active_next[i] = ((s1 & ((1LL << (R - r)) - 1)) == 0) ? 1 : 0;
}

cudaError_t fmm_launch_kick_drift_i32(unsigned int* ipos, float* vel, const float* acc, unsigned char* rung,
                                      unsigned char* active_next, long long n, double eps, double dt0, int max_rung,
                                      int substep, int closing, int periodic, DevCounters* ctr, cudaStream_t s)
{
    k_kick_drift_i32<<<(unsigned)fmm_ceil_div(n, 256), 256, 0, s>>>(ipos, vel, acc, rung, active_next, n, eps, dt0,
                                                                    max_rung, substep, closing, periodic,
                                                                    &ctr->kdk_status);
    return cudaGetLastError();
}

cudaError_t fmm_launch_assign_rungs(const float* acc, unsigned char* rung, long long n, double eps, double dt0,
                                    int max_rung, cudaStream_t s)
{
    k_assign_rungs<<<(unsigned)fmm_ceil_div(n, 256), 256, 0, s>>>(acc, rung, n, eps, dt0, max_rung);
    return cudaGetLastError();
}
