// GENERATED by gen_expansions.py -- do not edit by hand.
// Straight-line FP32 expansion operators for the Plummer-softened Green's function,
// multipoles of order 4 about the centre of mass and local expansions of order 5 (Sec. 3.1).
#pragma once

#define FMM_NL 56      /* local coefficients, |k| <= 5 */
#define FMM_NMOM 32    /* moment slots: M, M2, M3, M4 */
#define FMM_NREC 44    /* moment record incl. traces */

/* 1/sqrt(x) for x >= eps^2 > 0, which is never subnormal: the approximate reciprocal square
   root instruction in its subnormal-flushing form, which needs no scaling of subnormal inputs
   around the special-function unit (PTX ISA, rsqrt.approx.ftz.f32) */
__device__ __forceinline__ float fmm_rsqrt(float x)
{
#ifdef __CUDA_ARCH__
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
#else  /* host builds of these operators (tests): 1 / sqrt(x) in single precision */
    return 1.0f / sqrtf(x);
#endif
}

/* multi-index table (a, b, c) of the local coefficients, in storage order */
static const int fmm_multi_index_table[FMM_NL * 3] = {
    0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1, 2, 0, 0, 1, 1, 0, 1, 0, 1, 0, 2, 0, 0, 1, 1, 0, 0, 2, 3, 0, 0, 2, 1, 0, 2, 0, 1, 1, 2, 0, 1, 1, 1, 1, 0, 2, 0, 3, 0, 0, 2, 1, 0, 1, 2, 0, 0, 3, 4, 0, 0, 3, 1, 0, 3, 0, 1, 2, 2, 0, 2, 1, 1, 2, 0, 2, 1, 3, 0, 1, 2, 1, 1, 1, 2, 1, 0, 3, 0, 4, 0, 0, 3, 1, 0, 2, 2, 0, 1, 3, 0, 0, 4, 5, 0, 0, 4, 1, 0, 4, 0, 1, 3, 2, 0, 3, 1, 1, 3, 0, 2, 2, 3, 0, 2, 2, 1, 2, 1, 2, 2, 0, 3, 1, 4, 0, 1, 3, 1, 1, 2, 2, 1, 1, 3, 1, 0, 4, 0, 5, 0, 0, 4, 1, 0, 3, 2, 0, 2, 3, 0, 1, 4, 0, 0, 5
};
/* moment slot -> multi-index */
static const int fmm_moment_index_table[FMM_NMOM * 3] = {
    0, 0, 0, 2, 0, 0, 1, 1, 0, 1, 0, 1, 0, 2, 0, 0, 1, 1, 0, 0, 2, 3, 0, 0, 2, 1, 0, 2, 0, 1, 1, 2, 0, 1, 1, 1, 1, 0, 2, 0, 3, 0, 0, 2, 1, 0, 1, 2, 0, 0, 3, 4, 0, 0, 3, 1, 0, 3, 0, 1, 2, 2, 0, 2, 1, 1, 2, 0, 2, 1, 3, 0, 1, 2, 1, 1, 1, 2, 1, 0, 3, 0, 4, 0, 0, 3, 1, 0, 2, 2, 0, 1, 3, 0, 0, 4
};

__device__ __forceinline__ void fmm_green_scaled(float qx, float qy, float qz, float* __restrict__ D)
{
    const float q100 = qx;
    const float q010 = qy;
    const float q001 = qz;
    const float q200 = q100 * qx;
    const float q110 = q010 * qx;
    const float q101 = q001 * qx;
    const float q020 = q010 * qy;
    const float q011 = q001 * qy;
    const float q002 = q001 * qz;
    const float q300 = q200 * qx;
    const float q210 = q110 * qx;
    const float q201 = q101 * qx;
    const float q120 = q020 * qx;
    const float q111 = q011 * qx;
    const float q102 = q002 * qx;
    const float q030 = q020 * qy;
    const float q021 = q011 * qy;
    const float q012 = q002 * qy;
    const float q003 = q002 * qz;
    const float q400 = q300 * qx;
    const float q310 = q210 * qx;
    const float q301 = q201 * qx;
    const float q220 = q120 * qx;
    const float q211 = q111 * qx;
    const float q202 = q102 * qx;
    const float q130 = q030 * qx;
    const float q121 = q021 * qx;
    const float q112 = q012 * qx;
    const float q103 = q003 * qx;
    const float q040 = q030 * qy;
    const float q031 = q021 * qy;
    const float q022 = q012 * qy;
    const float q013 = q003 * qy;
    const float q004 = q003 * qz;
    const float q500 = q400 * qx;
    const float q410 = q310 * qx;
    const float q401 = q301 * qx;
    const float q320 = q220 * qx;
    const float q311 = q211 * qx;
    const float q302 = q202 * qx;
    const float q230 = q130 * qx;
    const float q221 = q121 * qx;
    const float q212 = q112 * qx;
    const float q203 = q103 * qx;
    const float q140 = q040 * qx;
    const float q131 = q031 * qx;
    const float q122 = q022 * qx;
    const float q113 = q013 * qx;
    const float q104 = q004 * qx;
    const float q050 = q040 * qy;
    const float q041 = q031 * qy;
    const float q032 = q022 * qy;
    const float q023 = q013 * qy;
    const float q014 = q004 * qy;
    const float q005 = q004 * qz;
    D[0] = 1.0f;
    D[1] = -1.0f * qx;
    D[2] = -1.0f * qy;
    D[3] = -1.0f * qz;
    D[4] = 3.0f * q200 + -1.0f;
    D[5] = 3.0f * q110;
    D[6] = 3.0f * q101;
    D[7] = 3.0f * q020 + -1.0f;
    D[8] = 3.0f * q011;
    D[9] = 3.0f * q002 + -1.0f;
    D[10] = -15.0f * q300 + 9.0f * qx;
    D[11] = -15.0f * q210 + 3.0f * qy;
    D[12] = -15.0f * q201 + 3.0f * qz;
    D[13] = -15.0f * q120 + 3.0f * qx;
    D[14] = -15.0f * q111;
    D[15] = -15.0f * q102 + 3.0f * qx;
    D[16] = -15.0f * q030 + 9.0f * qy;
    D[17] = -15.0f * q021 + 3.0f * qz;
    D[18] = -15.0f * q012 + 3.0f * qy;
    D[19] = -15.0f * q003 + 9.0f * qz;
    D[20] = 105.0f * q400 + -90.0f * q200 + 9.0f;
    D[21] = 105.0f * q310 + -45.0f * q110;
    D[22] = 105.0f * q301 + -45.0f * q101;
    D[23] = 105.0f * q220 + -15.0f * q200 + -15.0f * q020 + 3.0f;
    D[24] = 105.0f * q211 + -15.0f * q011;
    D[25] = 105.0f * q202 + -15.0f * q200 + -15.0f * q002 + 3.0f;
    D[26] = 105.0f * q130 + -45.0f * q110;
    D[27] = 105.0f * q121 + -15.0f * q101;
    D[28] = 105.0f * q112 + -15.0f * q110;
    D[29] = 105.0f * q103 + -45.0f * q101;
    D[30] = 105.0f * q040 + -90.0f * q020 + 9.0f;
    D[31] = 105.0f * q031 + -45.0f * q011;
    D[32] = 105.0f * q022 + -15.0f * q020 + -15.0f * q002 + 3.0f;
    D[33] = 105.0f * q013 + -45.0f * q011;
    D[34] = 105.0f * q004 + -90.0f * q002 + 9.0f;
    D[35] = -945.0f * q500 + 1050.0f * q300 + -225.0f * qx;
    D[36] = -945.0f * q410 + 630.0f * q210 + -45.0f * qy;
    D[37] = -945.0f * q401 + 630.0f * q201 + -45.0f * qz;
    D[38] = -945.0f * q320 + 105.0f * q300 + 315.0f * q120 + -45.0f * qx;
    D[39] = -945.0f * q311 + 315.0f * q111;
    D[40] = -945.0f * q302 + 105.0f * q300 + 315.0f * q102 + -45.0f * qx;
    D[41] = -945.0f * q230 + 315.0f * q210 + 105.0f * q030 + -45.0f * qy;
    D[42] = -945.0f * q221 + 105.0f * q201 + 105.0f * q021 + -15.0f * qz;
    D[43] = -945.0f * q212 + 105.0f * q210 + 105.0f * q012 + -15.0f * qy;
    D[44] = -945.0f * q203 + 315.0f * q201 + 105.0f * q003 + -45.0f * qz;
    D[45] = -945.0f * q140 + 630.0f * q120 + -45.0f * qx;
    D[46] = -945.0f * q131 + 315.0f * q111;
    D[47] = -945.0f * q122 + 105.0f * q120 + 105.0f * q102 + -15.0f * qx;
    D[48] = -945.0f * q113 + 315.0f * q111;
    D[49] = -945.0f * q104 + 630.0f * q102 + -45.0f * qx;
    D[50] = -945.0f * q050 + 1050.0f * q030 + -225.0f * qy;
    D[51] = -945.0f * q041 + 630.0f * q021 + -45.0f * qz;
    D[52] = -945.0f * q032 + 105.0f * q030 + 315.0f * q012 + -45.0f * qy;
    D[53] = -945.0f * q023 + 315.0f * q021 + 105.0f * q003 + -45.0f * qz;
    D[54] = -945.0f * q014 + 630.0f * q012 + -45.0f * qy;
    D[55] = -945.0f * q005 + 1050.0f * q003 + -225.0f * qz;
}

/* moments about the centre: M[slot(n)] += m y^n, orders 0, 2, 3, 4 */
__device__ __forceinline__ void fmm_p2m_acc(float m, float yx, float yy, float yz, float* __restrict__ M)
{
    const float y100 = yx;
    const float y010 = yy;
    const float y001 = yz;
    const float y200 = y100 * yx;
    const float y110 = y010 * yx;
    const float y101 = y001 * yx;
    const float y020 = y010 * yy;
    const float y011 = y001 * yy;
    const float y002 = y001 * yz;
    const float y300 = y200 * yx;
    const float y210 = y110 * yx;
    const float y201 = y101 * yx;
    const float y120 = y020 * yx;
    const float y111 = y011 * yx;
    const float y102 = y002 * yx;
    const float y030 = y020 * yy;
    const float y021 = y011 * yy;
    const float y012 = y002 * yy;
    const float y003 = y002 * yz;
    const float y400 = y300 * yx;
    const float y310 = y210 * yx;
    const float y301 = y201 * yx;
    const float y220 = y120 * yx;
    const float y211 = y111 * yx;
    const float y202 = y102 * yx;
    const float y130 = y030 * yx;
    const float y121 = y021 * yx;
    const float y112 = y012 * yx;
    const float y103 = y003 * yx;
    const float y040 = y030 * yy;
    const float y031 = y021 * yy;
    const float y022 = y012 * yy;
    const float y013 = y003 * yy;
    const float y004 = y003 * yz;
    M[0] += m;
    M[1] += m * y200;
    M[2] += m * y110;
    M[3] += m * y101;
    M[4] += m * y020;
    M[5] += m * y011;
    M[6] += m * y002;
    M[7] += m * y300;
    M[8] += m * y210;
    M[9] += m * y201;
    M[10] += m * y120;
    M[11] += m * y111;
    M[12] += m * y102;
    M[13] += m * y030;
    M[14] += m * y021;
    M[15] += m * y012;
    M[16] += m * y003;
    M[17] += m * y400;
    M[18] += m * y310;
    M[19] += m * y301;
    M[20] += m * y220;
    M[21] += m * y211;
    M[22] += m * y202;
    M[23] += m * y130;
    M[24] += m * y121;
    M[25] += m * y112;
    M[26] += m * y103;
    M[27] += m * y040;
    M[28] += m * y031;
    M[29] += m * y022;
    M[30] += m * y013;
    M[31] += m * y004;
}

/* child moments about its own centre -> parent centre, t = com_child - com_parent */
__device__ __forceinline__ void fmm_m2m_acc(const float* __restrict__ Mc, float tx, float ty, float tz,
                                            float* __restrict__ Mp)
{
    const float t100 = tx;
    const float t010 = ty;
    const float t001 = tz;
    const float t200 = t100 * tx;
    const float t110 = t010 * tx;
    const float t101 = t001 * tx;
    const float t020 = t010 * ty;
    const float t011 = t001 * ty;
    const float t002 = t001 * tz;
    const float t300 = t200 * tx;
    const float t210 = t110 * tx;
    const float t201 = t101 * tx;
    const float t120 = t020 * tx;
    const float t111 = t011 * tx;
    const float t102 = t002 * tx;
    const float t030 = t020 * ty;
    const float t021 = t011 * ty;
    const float t012 = t002 * ty;
    const float t003 = t002 * tz;
    const float t400 = t300 * tx;
    const float t310 = t210 * tx;
    const float t301 = t201 * tx;
    const float t220 = t120 * tx;
    const float t211 = t111 * tx;
    const float t202 = t102 * tx;
    const float t130 = t030 * tx;
    const float t121 = t021 * tx;
    const float t112 = t012 * tx;
    const float t103 = t003 * tx;
    const float t040 = t030 * ty;
    const float t031 = t021 * ty;
    const float t022 = t012 * ty;
    const float t013 = t003 * ty;
    const float t004 = t003 * tz;
    Mp[0] += Mc[0];
    Mp[1] += t200 * Mc[0] + Mc[1];
    Mp[2] += t110 * Mc[0] + Mc[2];
    Mp[3] += t101 * Mc[0] + Mc[3];
    Mp[4] += t020 * Mc[0] + Mc[4];
    Mp[5] += t011 * Mc[0] + Mc[5];
    Mp[6] += t002 * Mc[0] + Mc[6];
    Mp[7] += t300 * Mc[0] + 3.0f * tx * Mc[1] + Mc[7];
    Mp[8] += t210 * Mc[0] + ty * Mc[1] + 2.0f * tx * Mc[2] + Mc[8];
    Mp[9] += t201 * Mc[0] + tz * Mc[1] + 2.0f * tx * Mc[3] + Mc[9];
    Mp[10] += t120 * Mc[0] + 2.0f * ty * Mc[2] + tx * Mc[4] + Mc[10];
    Mp[11] += t111 * Mc[0] + tz * Mc[2] + ty * Mc[3] + tx * Mc[5] + Mc[11];
    Mp[12] += t102 * Mc[0] + 2.0f * tz * Mc[3] + tx * Mc[6] + Mc[12];
    Mp[13] += t030 * Mc[0] + 3.0f * ty * Mc[4] + Mc[13];
    Mp[14] += t021 * Mc[0] + tz * Mc[4] + 2.0f * ty * Mc[5] + Mc[14];
    Mp[15] += t012 * Mc[0] + 2.0f * tz * Mc[5] + ty * Mc[6] + Mc[15];
    Mp[16] += t003 * Mc[0] + 3.0f * tz * Mc[6] + Mc[16];
    Mp[17] += t400 * Mc[0] + 6.0f * t200 * Mc[1] + 4.0f * tx * Mc[7] + Mc[17];
    Mp[18] += t310 * Mc[0] + 3.0f * t110 * Mc[1] + 3.0f * t200 * Mc[2] + ty * Mc[7] + 3.0f * tx * Mc[8] + Mc[18];
    Mp[19] += t301 * Mc[0] + 3.0f * t101 * Mc[1] + 3.0f * t200 * Mc[3] + tz * Mc[7] + 3.0f * tx * Mc[9] + Mc[19];
    Mp[20] += t220 * Mc[0] + t020 * Mc[1] + 4.0f * t110 * Mc[2] + t200 * Mc[4] + 2.0f * ty * Mc[8] + 2.0f * tx * Mc[10] + Mc[20];
    Mp[21] += t211 * Mc[0] + t011 * Mc[1] + 2.0f * t101 * Mc[2] + 2.0f * t110 * Mc[3] + t200 * Mc[5] + tz * Mc[8] + ty * Mc[9] + 2.0f * tx * Mc[11] + Mc[21];
    Mp[22] += t202 * Mc[0] + t002 * Mc[1] + 4.0f * t101 * Mc[3] + t200 * Mc[6] + 2.0f * tz * Mc[9] + 2.0f * tx * Mc[12] + Mc[22];
    Mp[23] += t130 * Mc[0] + 3.0f * t020 * Mc[2] + 3.0f * t110 * Mc[4] + 3.0f * ty * Mc[10] + tx * Mc[13] + Mc[23];
    Mp[24] += t121 * Mc[0] + 2.0f * t011 * Mc[2] + t020 * Mc[3] + t101 * Mc[4] + 2.0f * t110 * Mc[5] + tz * Mc[10] + 2.0f * ty * Mc[11] + tx * Mc[14] + Mc[24];
    Mp[25] += t112 * Mc[0] + t002 * Mc[2] + 2.0f * t011 * Mc[3] + 2.0f * t101 * Mc[5] + t110 * Mc[6] + 2.0f * tz * Mc[11] + ty * Mc[12] + tx * Mc[15] + Mc[25];
    Mp[26] += t103 * Mc[0] + 3.0f * t002 * Mc[3] + 3.0f * t101 * Mc[6] + 3.0f * tz * Mc[12] + tx * Mc[16] + Mc[26];
    Mp[27] += t040 * Mc[0] + 6.0f * t020 * Mc[4] + 4.0f * ty * Mc[13] + Mc[27];
    Mp[28] += t031 * Mc[0] + 3.0f * t011 * Mc[4] + 3.0f * t020 * Mc[5] + tz * Mc[13] + 3.0f * ty * Mc[14] + Mc[28];
    Mp[29] += t022 * Mc[0] + t002 * Mc[4] + 4.0f * t011 * Mc[5] + t020 * Mc[6] + 2.0f * tz * Mc[14] + 2.0f * ty * Mc[15] + Mc[29];
    Mp[30] += t013 * Mc[0] + 3.0f * t002 * Mc[5] + 3.0f * t011 * Mc[6] + 3.0f * tz * Mc[15] + ty * Mc[16] + Mc[30];
    Mp[31] += t004 * Mc[0] + 6.0f * t002 * Mc[6] + 4.0f * tz * Mc[16] + Mc[31];
}

/* traces of the moment tensors for the particle-cell kernel */
__device__ __forceinline__ void fmm_moment_traces(float* __restrict__ R)
{
    R[32] = R[1] + R[4] + R[6];
    R[33] = R[7] + R[10] + R[12];
    R[34] = R[8] + R[13] + R[15];
    R[35] = R[9] + R[14] + R[16];
    R[36] = R[17] + R[20] + R[22];
    R[37] = R[18] + R[23] + R[25];
    R[38] = R[19] + R[24] + R[26];
    R[39] = R[20] + R[27] + R[29];
    R[40] = R[21] + R[28] + R[30];
    R[41] = R[22] + R[29] + R[31];
    R[42] = R[36] + R[39] + R[41];
    R[43] = 0.0f;
}

/* squared Frobenius norms of the order-2 and order-4 moment tensors of a record, each
   component scaled (by s2, s4) before it is squared so that small cells do not underflow */
__device__ __forceinline__ void fmm_moment_norms2(const float* __restrict__ R, float s2, float s4, float& n2,
                                                  float& n4)
{
    const float t1 = R[1] * s2;
    const float t2 = R[2] * s2;
    const float t3 = R[3] * s2;
    const float t4 = R[4] * s2;
    const float t5 = R[5] * s2;
    const float t6 = R[6] * s2;
    n2 = t1 * t1 + 2.0f * t2 * t2 + 2.0f * t3 * t3 + t4 * t4 + 2.0f * t5 * t5 + t6 * t6;
    const float t17 = R[17] * s4;
    const float t18 = R[18] * s4;
    const float t19 = R[19] * s4;
    const float t20 = R[20] * s4;
    const float t21 = R[21] * s4;
    const float t22 = R[22] * s4;
    const float t23 = R[23] * s4;
    const float t24 = R[24] * s4;
    const float t25 = R[25] * s4;
    const float t26 = R[26] * s4;
    const float t27 = R[27] * s4;
    const float t28 = R[28] * s4;
    const float t29 = R[29] * s4;
    const float t30 = R[30] * s4;
    const float t31 = R[31] * s4;
    n4 = t17 * t17 + 4.0f * t18 * t18 + 4.0f * t19 * t19 + 6.0f * t20 * t20 + 12.0f * t21 * t21 + 6.0f * t22 * t22 + 4.0f * t23 * t23 + 12.0f * t24 * t24 + 12.0f * t25 * t25 + 4.0f * t26 * t26 + t27 * t27 + 4.0f * t28 * t28 + 6.0f * t29 * t29 + 4.0f * t30 * t30 + t31 * t31;
}

/* multipole (moment record M about z) -> local coefficients about c; r = c - z */
__device__ __forceinline__ void fmm_m2l_acc(const float* __restrict__ M, float rx, float ry, float rz,
                                            float eps2, float* __restrict__ Lc)
{
    const float ir = fmm_rsqrt(fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, eps2))));
    float D[56];
    fmm_green_scaled(rx * ir, ry * ir, rz * ir, D);
    const float ir2 = ir * ir, ir3 = ir2 * ir, ir4 = ir2 * ir2;
    const float w000 = 1.0f * M[0];
    const float w200 = 0.5f * M[1] * ir2;
    const float w110 = 1.0f * M[2] * ir2;
    const float w101 = 1.0f * M[3] * ir2;
    const float w020 = 0.5f * M[4] * ir2;
    const float w011 = 1.0f * M[5] * ir2;
    const float w002 = 0.5f * M[6] * ir2;
    const float w300 = -0.16666666666666666f * M[7] * ir3;
    const float w210 = -0.5f * M[8] * ir3;
    const float w201 = -0.5f * M[9] * ir3;
    const float w120 = -0.5f * M[10] * ir3;
    const float w111 = -1.0f * M[11] * ir3;
    const float w102 = -0.5f * M[12] * ir3;
    const float w030 = -0.16666666666666666f * M[13] * ir3;
    const float w021 = -0.5f * M[14] * ir3;
    const float w012 = -0.5f * M[15] * ir3;
    const float w003 = -0.16666666666666666f * M[16] * ir3;
    const float w400 = 0.041666666666666664f * M[17] * ir4;
    const float w310 = 0.16666666666666666f * M[18] * ir4;
    const float w301 = 0.16666666666666666f * M[19] * ir4;
    const float w220 = 0.25f * M[20] * ir4;
    const float w211 = 0.5f * M[21] * ir4;
    const float w202 = 0.25f * M[22] * ir4;
    const float w130 = 0.16666666666666666f * M[23] * ir4;
    const float w121 = 0.5f * M[24] * ir4;
    const float w112 = 0.5f * M[25] * ir4;
    const float w103 = 0.16666666666666666f * M[26] * ir4;
    const float w040 = 0.041666666666666664f * M[27] * ir4;
    const float w031 = 0.16666666666666666f * M[28] * ir4;
    const float w022 = 0.25f * M[29] * ir4;
    const float w013 = 0.16666666666666666f * M[30] * ir4;
    const float w004 = 0.041666666666666664f * M[31] * ir4;
    float p = ir;
    Lc[0] += p * (w000 * D[0] + w200 * D[4] + w110 * D[5] + w101 * D[6] + w020 * D[7] + w011 * D[8] + w002 * D[9] + w300 * D[10] + w210 * D[11] + w201 * D[12] + w120 * D[13] + w111 * D[14] + w102 * D[15] + w030 * D[16] + w021 * D[17] + w012 * D[18] + w003 * D[19] + w400 * D[20] + w310 * D[21] + w301 * D[22] + w220 * D[23] + w211 * D[24] + w202 * D[25] + w130 * D[26] + w121 * D[27] + w112 * D[28] + w103 * D[29] + w040 * D[30] + w031 * D[31] + w022 * D[32] + w013 * D[33] + w004 * D[34]);
    p *= ir;
    Lc[1] += p * (w000 * D[1] + w200 * D[10] + w110 * D[11] + w101 * D[12] + w020 * D[13] + w011 * D[14] + w002 * D[15] + w300 * D[20] + w210 * D[21] + w201 * D[22] + w120 * D[23] + w111 * D[24] + w102 * D[25] + w030 * D[26] + w021 * D[27] + w012 * D[28] + w003 * D[29] + w400 * D[35] + w310 * D[36] + w301 * D[37] + w220 * D[38] + w211 * D[39] + w202 * D[40] + w130 * D[41] + w121 * D[42] + w112 * D[43] + w103 * D[44] + w040 * D[45] + w031 * D[46] + w022 * D[47] + w013 * D[48] + w004 * D[49]);
    Lc[2] += p * (w000 * D[2] + w200 * D[11] + w110 * D[13] + w101 * D[14] + w020 * D[16] + w011 * D[17] + w002 * D[18] + w300 * D[21] + w210 * D[23] + w201 * D[24] + w120 * D[26] + w111 * D[27] + w102 * D[28] + w030 * D[30] + w021 * D[31] + w012 * D[32] + w003 * D[33] + w400 * D[36] + w310 * D[38] + w301 * D[39] + w220 * D[41] + w211 * D[42] + w202 * D[43] + w130 * D[45] + w121 * D[46] + w112 * D[47] + w103 * D[48] + w040 * D[50] + w031 * D[51] + w022 * D[52] + w013 * D[53] + w004 * D[54]);
    Lc[3] += p * (w000 * D[3] + w200 * D[12] + w110 * D[14] + w101 * D[15] + w020 * D[17] + w011 * D[18] + w002 * D[19] + w300 * D[22] + w210 * D[24] + w201 * D[25] + w120 * D[27] + w111 * D[28] + w102 * D[29] + w030 * D[31] + w021 * D[32] + w012 * D[33] + w003 * D[34] + w400 * D[37] + w310 * D[39] + w301 * D[40] + w220 * D[42] + w211 * D[43] + w202 * D[44] + w130 * D[46] + w121 * D[47] + w112 * D[48] + w103 * D[49] + w040 * D[51] + w031 * D[52] + w022 * D[53] + w013 * D[54] + w004 * D[55]);
    p *= ir;
    Lc[4] += p * (w000 * D[4] + w200 * D[20] + w110 * D[21] + w101 * D[22] + w020 * D[23] + w011 * D[24] + w002 * D[25] + w300 * D[35] + w210 * D[36] + w201 * D[37] + w120 * D[38] + w111 * D[39] + w102 * D[40] + w030 * D[41] + w021 * D[42] + w012 * D[43] + w003 * D[44]);
    Lc[5] += p * (w000 * D[5] + w200 * D[21] + w110 * D[23] + w101 * D[24] + w020 * D[26] + w011 * D[27] + w002 * D[28] + w300 * D[36] + w210 * D[38] + w201 * D[39] + w120 * D[41] + w111 * D[42] + w102 * D[43] + w030 * D[45] + w021 * D[46] + w012 * D[47] + w003 * D[48]);
    Lc[6] += p * (w000 * D[6] + w200 * D[22] + w110 * D[24] + w101 * D[25] + w020 * D[27] + w011 * D[28] + w002 * D[29] + w300 * D[37] + w210 * D[39] + w201 * D[40] + w120 * D[42] + w111 * D[43] + w102 * D[44] + w030 * D[46] + w021 * D[47] + w012 * D[48] + w003 * D[49]);
    Lc[7] += p * (w000 * D[7] + w200 * D[23] + w110 * D[26] + w101 * D[27] + w020 * D[30] + w011 * D[31] + w002 * D[32] + w300 * D[38] + w210 * D[41] + w201 * D[42] + w120 * D[45] + w111 * D[46] + w102 * D[47] + w030 * D[50] + w021 * D[51] + w012 * D[52] + w003 * D[53]);
    Lc[8] += p * (w000 * D[8] + w200 * D[24] + w110 * D[27] + w101 * D[28] + w020 * D[31] + w011 * D[32] + w002 * D[33] + w300 * D[39] + w210 * D[42] + w201 * D[43] + w120 * D[46] + w111 * D[47] + w102 * D[48] + w030 * D[51] + w021 * D[52] + w012 * D[53] + w003 * D[54]);
    Lc[9] += p * (w000 * D[9] + w200 * D[25] + w110 * D[28] + w101 * D[29] + w020 * D[32] + w011 * D[33] + w002 * D[34] + w300 * D[40] + w210 * D[43] + w201 * D[44] + w120 * D[47] + w111 * D[48] + w102 * D[49] + w030 * D[52] + w021 * D[53] + w012 * D[54] + w003 * D[55]);
    p *= ir;
    Lc[10] += p * (w000 * D[10] + w200 * D[35] + w110 * D[36] + w101 * D[37] + w020 * D[38] + w011 * D[39] + w002 * D[40]);
    Lc[11] += p * (w000 * D[11] + w200 * D[36] + w110 * D[38] + w101 * D[39] + w020 * D[41] + w011 * D[42] + w002 * D[43]);
    Lc[12] += p * (w000 * D[12] + w200 * D[37] + w110 * D[39] + w101 * D[40] + w020 * D[42] + w011 * D[43] + w002 * D[44]);
    Lc[13] += p * (w000 * D[13] + w200 * D[38] + w110 * D[41] + w101 * D[42] + w020 * D[45] + w011 * D[46] + w002 * D[47]);
    Lc[14] += p * (w000 * D[14] + w200 * D[39] + w110 * D[42] + w101 * D[43] + w020 * D[46] + w011 * D[47] + w002 * D[48]);
    Lc[15] += p * (w000 * D[15] + w200 * D[40] + w110 * D[43] + w101 * D[44] + w020 * D[47] + w011 * D[48] + w002 * D[49]);
    Lc[16] += p * (w000 * D[16] + w200 * D[41] + w110 * D[45] + w101 * D[46] + w020 * D[50] + w011 * D[51] + w002 * D[52]);
    Lc[17] += p * (w000 * D[17] + w200 * D[42] + w110 * D[46] + w101 * D[47] + w020 * D[51] + w011 * D[52] + w002 * D[53]);
    Lc[18] += p * (w000 * D[18] + w200 * D[43] + w110 * D[47] + w101 * D[48] + w020 * D[52] + w011 * D[53] + w002 * D[54]);
    Lc[19] += p * (w000 * D[19] + w200 * D[44] + w110 * D[48] + w101 * D[49] + w020 * D[53] + w011 * D[54] + w002 * D[55]);
    p *= ir;
    Lc[20] += p * (w000 * D[20]);
    Lc[21] += p * (w000 * D[21]);
    Lc[22] += p * (w000 * D[22]);
    Lc[23] += p * (w000 * D[23]);
    Lc[24] += p * (w000 * D[24]);
    Lc[25] += p * (w000 * D[25]);
    Lc[26] += p * (w000 * D[26]);
    Lc[27] += p * (w000 * D[27]);
    Lc[28] += p * (w000 * D[28]);
    Lc[29] += p * (w000 * D[29]);
    Lc[30] += p * (w000 * D[30]);
    Lc[31] += p * (w000 * D[31]);
    Lc[32] += p * (w000 * D[32]);
    Lc[33] += p * (w000 * D[33]);
    Lc[34] += p * (w000 * D[34]);
    p *= ir;
    Lc[35] += p * (w000 * D[35]);
    Lc[36] += p * (w000 * D[36]);
    Lc[37] += p * (w000 * D[37]);
    Lc[38] += p * (w000 * D[38]);
    Lc[39] += p * (w000 * D[39]);
    Lc[40] += p * (w000 * D[40]);
    Lc[41] += p * (w000 * D[41]);
    Lc[42] += p * (w000 * D[42]);
    Lc[43] += p * (w000 * D[43]);
    Lc[44] += p * (w000 * D[44]);
    Lc[45] += p * (w000 * D[45]);
    Lc[46] += p * (w000 * D[46]);
    Lc[47] += p * (w000 * D[47]);
    Lc[48] += p * (w000 * D[48]);
    Lc[49] += p * (w000 * D[49]);
    Lc[50] += p * (w000 * D[50]);
    Lc[51] += p * (w000 * D[51]);
    Lc[52] += p * (w000 * D[52]);
    Lc[53] += p * (w000 * D[53]);
    Lc[54] += p * (w000 * D[54]);
    Lc[55] += p * (w000 * D[55]);
}

/* particle of mass m at z -> local coefficients about c; r = c - z */
__device__ __forceinline__ void fmm_p2l_acc(float m, float rx, float ry, float rz, float eps2,
                                            float* __restrict__ Lc)
{
    const float ir = fmm_rsqrt(fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, eps2))));
    float D[56];
    fmm_green_scaled(rx * ir, ry * ir, rz * ir, D);
    float p = m * ir;
    Lc[0] = fmaf(p, D[0], Lc[0]);
    p *= ir;
    Lc[1] = fmaf(p, D[1], Lc[1]);
    Lc[2] = fmaf(p, D[2], Lc[2]);
    Lc[3] = fmaf(p, D[3], Lc[3]);
    p *= ir;
    Lc[4] = fmaf(p, D[4], Lc[4]);
    Lc[5] = fmaf(p, D[5], Lc[5]);
    Lc[6] = fmaf(p, D[6], Lc[6]);
    Lc[7] = fmaf(p, D[7], Lc[7]);
    Lc[8] = fmaf(p, D[8], Lc[8]);
    Lc[9] = fmaf(p, D[9], Lc[9]);
    p *= ir;
    Lc[10] = fmaf(p, D[10], Lc[10]);
    Lc[11] = fmaf(p, D[11], Lc[11]);
    Lc[12] = fmaf(p, D[12], Lc[12]);
    Lc[13] = fmaf(p, D[13], Lc[13]);
    Lc[14] = fmaf(p, D[14], Lc[14]);
    Lc[15] = fmaf(p, D[15], Lc[15]);
    Lc[16] = fmaf(p, D[16], Lc[16]);
    Lc[17] = fmaf(p, D[17], Lc[17]);
    Lc[18] = fmaf(p, D[18], Lc[18]);
    Lc[19] = fmaf(p, D[19], Lc[19]);
    p *= ir;
    Lc[20] = fmaf(p, D[20], Lc[20]);
    Lc[21] = fmaf(p, D[21], Lc[21]);
    Lc[22] = fmaf(p, D[22], Lc[22]);
    Lc[23] = fmaf(p, D[23], Lc[23]);
    Lc[24] = fmaf(p, D[24], Lc[24]);
    Lc[25] = fmaf(p, D[25], Lc[25]);
    Lc[26] = fmaf(p, D[26], Lc[26]);
    Lc[27] = fmaf(p, D[27], Lc[27]);
    Lc[28] = fmaf(p, D[28], Lc[28]);
    Lc[29] = fmaf(p, D[29], Lc[29]);
    Lc[30] = fmaf(p, D[30], Lc[30]);
    Lc[31] = fmaf(p, D[31], Lc[31]);
    Lc[32] = fmaf(p, D[32], Lc[32]);
    Lc[33] = fmaf(p, D[33], Lc[33]);
    Lc[34] = fmaf(p, D[34], Lc[34]);
    p *= ir;
    Lc[35] = fmaf(p, D[35], Lc[35]);
    Lc[36] = fmaf(p, D[36], Lc[36]);
    Lc[37] = fmaf(p, D[37], Lc[37]);
    Lc[38] = fmaf(p, D[38], Lc[38]);
    Lc[39] = fmaf(p, D[39], Lc[39]);
    Lc[40] = fmaf(p, D[40], Lc[40]);
    Lc[41] = fmaf(p, D[41], Lc[41]);
    Lc[42] = fmaf(p, D[42], Lc[42]);
    Lc[43] = fmaf(p, D[43], Lc[43]);
    Lc[44] = fmaf(p, D[44], Lc[44]);
    Lc[45] = fmaf(p, D[45], Lc[45]);
    Lc[46] = fmaf(p, D[46], Lc[46]);
    Lc[47] = fmaf(p, D[47], Lc[47]);
    Lc[48] = fmaf(p, D[48], Lc[48]);
    Lc[49] = fmaf(p, D[49], Lc[49]);
    Lc[50] = fmaf(p, D[50], Lc[50]);
    Lc[51] = fmaf(p, D[51], Lc[51]);
    Lc[52] = fmaf(p, D[52], Lc[52]);
    Lc[53] = fmaf(p, D[53], Lc[53]);
    Lc[54] = fmaf(p, D[54], Lc[54]);
    Lc[55] = fmaf(p, D[55], Lc[55]);
}

/* re-expand local coefficients about c at c + t */
__device__ __forceinline__ void fmm_l2l(const float* __restrict__ Lp, float tx, float ty, float tz,
                                        float* __restrict__ Lo)
{
    const float t100 = tx;
    const float t010 = ty;
    const float t001 = tz;
    const float t200 = t100 * tx;
    const float t110 = t010 * tx;
    const float t101 = t001 * tx;
    const float t020 = t010 * ty;
    const float t011 = t001 * ty;
    const float t002 = t001 * tz;
    const float t300 = t200 * tx;
    const float t210 = t110 * tx;
    const float t201 = t101 * tx;
    const float t120 = t020 * tx;
    const float t111 = t011 * tx;
    const float t102 = t002 * tx;
    const float t030 = t020 * ty;
    const float t021 = t011 * ty;
    const float t012 = t002 * ty;
    const float t003 = t002 * tz;
    const float t400 = t300 * tx;
    const float t310 = t210 * tx;
    const float t301 = t201 * tx;
    const float t220 = t120 * tx;
    const float t211 = t111 * tx;
    const float t202 = t102 * tx;
    const float t130 = t030 * tx;
    const float t121 = t021 * tx;
    const float t112 = t012 * tx;
    const float t103 = t003 * tx;
    const float t040 = t030 * ty;
    const float t031 = t021 * ty;
    const float t022 = t012 * ty;
    const float t013 = t003 * ty;
    const float t004 = t003 * tz;
    const float t500 = t400 * tx;
    const float t410 = t310 * tx;
    const float t401 = t301 * tx;
    const float t320 = t220 * tx;
    const float t311 = t211 * tx;
    const float t302 = t202 * tx;
    const float t230 = t130 * tx;
    const float t221 = t121 * tx;
    const float t212 = t112 * tx;
    const float t203 = t103 * tx;
    const float t140 = t040 * tx;
    const float t131 = t031 * tx;
    const float t122 = t022 * tx;
    const float t113 = t013 * tx;
    const float t104 = t004 * tx;
    const float t050 = t040 * ty;
    const float t041 = t031 * ty;
    const float t032 = t022 * ty;
    const float t023 = t013 * ty;
    const float t014 = t004 * ty;
    const float t005 = t004 * tz;
    Lo[0] = Lp[0] + tx * Lp[1] + ty * Lp[2] + tz * Lp[3] + 0.5f * t200 * Lp[4] + t110 * Lp[5] + t101 * Lp[6] + 0.5f * t020 * Lp[7] + t011 * Lp[8] + 0.5f * t002 * Lp[9] + 0.16666666666666666f * t300 * Lp[10] + 0.5f * t210 * Lp[11] + 0.5f * t201 * Lp[12] + 0.5f * t120 * Lp[13] + t111 * Lp[14] + 0.5f * t102 * Lp[15] + 0.16666666666666666f * t030 * Lp[16] + 0.5f * t021 * Lp[17] + 0.5f * t012 * Lp[18] + 0.16666666666666666f * t003 * Lp[19] + 0.041666666666666664f * t400 * Lp[20] + 0.16666666666666666f * t310 * Lp[21] + 0.16666666666666666f * t301 * Lp[22] + 0.25f * t220 * Lp[23] + 0.5f * t211 * Lp[24] + 0.25f * t202 * Lp[25] + 0.16666666666666666f * t130 * Lp[26] + 0.5f * t121 * Lp[27] + 0.5f * t112 * Lp[28] + 0.16666666666666666f * t103 * Lp[29] + 0.041666666666666664f * t040 * Lp[30] + 0.16666666666666666f * t031 * Lp[31] + 0.25f * t022 * Lp[32] + 0.16666666666666666f * t013 * Lp[33] + 0.041666666666666664f * t004 * Lp[34] + 0.008333333333333333f * t500 * Lp[35] + 0.041666666666666664f * t410 * Lp[36] + 0.041666666666666664f * t401 * Lp[37] + 0.08333333333333333f * t320 * Lp[38] + 0.16666666666666666f * t311 * Lp[39] + 0.08333333333333333f * t302 * Lp[40] + 0.08333333333333333f * t230 * Lp[41] + 0.25f * t221 * Lp[42] + 0.25f * t212 * Lp[43] + 0.08333333333333333f * t203 * Lp[44] + 0.041666666666666664f * t140 * Lp[45] + 0.16666666666666666f * t131 * Lp[46] + 0.25f * t122 * Lp[47] + 0.16666666666666666f * t113 * Lp[48] + 0.041666666666666664f * t104 * Lp[49] + 0.008333333333333333f * t050 * Lp[50] + 0.041666666666666664f * t041 * Lp[51] + 0.08333333333333333f * t032 * Lp[52] + 0.08333333333333333f * t023 * Lp[53] + 0.041666666666666664f * t014 * Lp[54] + 0.008333333333333333f * t005 * Lp[55];
    Lo[1] = Lp[1] + tx * Lp[4] + ty * Lp[5] + tz * Lp[6] + 0.5f * t200 * Lp[10] + t110 * Lp[11] + t101 * Lp[12] + 0.5f * t020 * Lp[13] + t011 * Lp[14] + 0.5f * t002 * Lp[15] + 0.16666666666666666f * t300 * Lp[20] + 0.5f * t210 * Lp[21] + 0.5f * t201 * Lp[22] + 0.5f * t120 * Lp[23] + t111 * Lp[24] + 0.5f * t102 * Lp[25] + 0.16666666666666666f * t030 * Lp[26] + 0.5f * t021 * Lp[27] + 0.5f * t012 * Lp[28] + 0.16666666666666666f * t003 * Lp[29] + 0.041666666666666664f * t400 * Lp[35] + 0.16666666666666666f * t310 * Lp[36] + 0.16666666666666666f * t301 * Lp[37] + 0.25f * t220 * Lp[38] + 0.5f * t211 * Lp[39] + 0.25f * t202 * Lp[40] + 0.16666666666666666f * t130 * Lp[41] + 0.5f * t121 * Lp[42] + 0.5f * t112 * Lp[43] + 0.16666666666666666f * t103 * Lp[44] + 0.041666666666666664f * t040 * Lp[45] + 0.16666666666666666f * t031 * Lp[46] + 0.25f * t022 * Lp[47] + 0.16666666666666666f * t013 * Lp[48] + 0.041666666666666664f * t004 * Lp[49];
    Lo[2] = Lp[2] + tx * Lp[5] + ty * Lp[7] + tz * Lp[8] + 0.5f * t200 * Lp[11] + t110 * Lp[13] + t101 * Lp[14] + 0.5f * t020 * Lp[16] + t011 * Lp[17] + 0.5f * t002 * Lp[18] + 0.16666666666666666f * t300 * Lp[21] + 0.5f * t210 * Lp[23] + 0.5f * t201 * Lp[24] + 0.5f * t120 * Lp[26] + t111 * Lp[27] + 0.5f * t102 * Lp[28] + 0.16666666666666666f * t030 * Lp[30] + 0.5f * t021 * Lp[31] + 0.5f * t012 * Lp[32] + 0.16666666666666666f * t003 * Lp[33] + 0.041666666666666664f * t400 * Lp[36] + 0.16666666666666666f * t310 * Lp[38] + 0.16666666666666666f * t301 * Lp[39] + 0.25f * t220 * Lp[41] + 0.5f * t211 * Lp[42] + 0.25f * t202 * Lp[43] + 0.16666666666666666f * t130 * Lp[45] + 0.5f * t121 * Lp[46] + 0.5f * t112 * Lp[47] + 0.16666666666666666f * t103 * Lp[48] + 0.041666666666666664f * t040 * Lp[50] + 0.16666666666666666f * t031 * Lp[51] + 0.25f * t022 * Lp[52] + 0.16666666666666666f * t013 * Lp[53] + 0.041666666666666664f * t004 * Lp[54];
    Lo[3] = Lp[3] + tx * Lp[6] + ty * Lp[8] + tz * Lp[9] + 0.5f * t200 * Lp[12] + t110 * Lp[14] + t101 * Lp[15] + 0.5f * t020 * Lp[17] + t011 * Lp[18] + 0.5f * t002 * Lp[19] + 0.16666666666666666f * t300 * Lp[22] + 0.5f * t210 * Lp[24] + 0.5f * t201 * Lp[25] + 0.5f * t120 * Lp[27] + t111 * Lp[28] + 0.5f * t102 * Lp[29] + 0.16666666666666666f * t030 * Lp[31] + 0.5f * t021 * Lp[32] + 0.5f * t012 * Lp[33] + 0.16666666666666666f * t003 * Lp[34] + 0.041666666666666664f * t400 * Lp[37] + 0.16666666666666666f * t310 * Lp[39] + 0.16666666666666666f * t301 * Lp[40] + 0.25f * t220 * Lp[42] + 0.5f * t211 * Lp[43] + 0.25f * t202 * Lp[44] + 0.16666666666666666f * t130 * Lp[46] + 0.5f * t121 * Lp[47] + 0.5f * t112 * Lp[48] + 0.16666666666666666f * t103 * Lp[49] + 0.041666666666666664f * t040 * Lp[51] + 0.16666666666666666f * t031 * Lp[52] + 0.25f * t022 * Lp[53] + 0.16666666666666666f * t013 * Lp[54] + 0.041666666666666664f * t004 * Lp[55];
    Lo[4] = Lp[4] + tx * Lp[10] + ty * Lp[11] + tz * Lp[12] + 0.5f * t200 * Lp[20] + t110 * Lp[21] + t101 * Lp[22] + 0.5f * t020 * Lp[23] + t011 * Lp[24] + 0.5f * t002 * Lp[25] + 0.16666666666666666f * t300 * Lp[35] + 0.5f * t210 * Lp[36] + 0.5f * t201 * Lp[37] + 0.5f * t120 * Lp[38] + t111 * Lp[39] + 0.5f * t102 * Lp[40] + 0.16666666666666666f * t030 * Lp[41] + 0.5f * t021 * Lp[42] + 0.5f * t012 * Lp[43] + 0.16666666666666666f * t003 * Lp[44];
    Lo[5] = Lp[5] + tx * Lp[11] + ty * Lp[13] + tz * Lp[14] + 0.5f * t200 * Lp[21] + t110 * Lp[23] + t101 * Lp[24] + 0.5f * t020 * Lp[26] + t011 * Lp[27] + 0.5f * t002 * Lp[28] + 0.16666666666666666f * t300 * Lp[36] + 0.5f * t210 * Lp[38] + 0.5f * t201 * Lp[39] + 0.5f * t120 * Lp[41] + t111 * Lp[42] + 0.5f * t102 * Lp[43] + 0.16666666666666666f * t030 * Lp[45] + 0.5f * t021 * Lp[46] + 0.5f * t012 * Lp[47] + 0.16666666666666666f * t003 * Lp[48];
    Lo[6] = Lp[6] + tx * Lp[12] + ty * Lp[14] + tz * Lp[15] + 0.5f * t200 * Lp[22] + t110 * Lp[24] + t101 * Lp[25] + 0.5f * t020 * Lp[27] + t011 * Lp[28] + 0.5f * t002 * Lp[29] + 0.16666666666666666f * t300 * Lp[37] + 0.5f * t210 * Lp[39] + 0.5f * t201 * Lp[40] + 0.5f * t120 * Lp[42] + t111 * Lp[43] + 0.5f * t102 * Lp[44] + 0.16666666666666666f * t030 * Lp[46] + 0.5f * t021 * Lp[47] + 0.5f * t012 * Lp[48] + 0.16666666666666666f * t003 * Lp[49];
    Lo[7] = Lp[7] + tx * Lp[13] + ty * Lp[16] + tz * Lp[17] + 0.5f * t200 * Lp[23] + t110 * Lp[26] + t101 * Lp[27] + 0.5f * t020 * Lp[30] + t011 * Lp[31] + 0.5f * t002 * Lp[32] + 0.16666666666666666f * t300 * Lp[38] + 0.5f * t210 * Lp[41] + 0.5f * t201 * Lp[42] + 0.5f * t120 * Lp[45] + t111 * Lp[46] + 0.5f * t102 * Lp[47] + 0.16666666666666666f * t030 * Lp[50] + 0.5f * t021 * Lp[51] + 0.5f * t012 * Lp[52] + 0.16666666666666666f * t003 * Lp[53];
    Lo[8] = Lp[8] + tx * Lp[14] + ty * Lp[17] + tz * Lp[18] + 0.5f * t200 * Lp[24] + t110 * Lp[27] + t101 * Lp[28] + 0.5f * t020 * Lp[31] + t011 * Lp[32] + 0.5f * t002 * Lp[33] + 0.16666666666666666f * t300 * Lp[39] + 0.5f * t210 * Lp[42] + 0.5f * t201 * Lp[43] + 0.5f * t120 * Lp[46] + t111 * Lp[47] + 0.5f * t102 * Lp[48] + 0.16666666666666666f * t030 * Lp[51] + 0.5f * t021 * Lp[52] + 0.5f * t012 * Lp[53] + 0.16666666666666666f * t003 * Lp[54];
    Lo[9] = Lp[9] + tx * Lp[15] + ty * Lp[18] + tz * Lp[19] + 0.5f * t200 * Lp[25] + t110 * Lp[28] + t101 * Lp[29] + 0.5f * t020 * Lp[32] + t011 * Lp[33] + 0.5f * t002 * Lp[34] + 0.16666666666666666f * t300 * Lp[40] + 0.5f * t210 * Lp[43] + 0.5f * t201 * Lp[44] + 0.5f * t120 * Lp[47] + t111 * Lp[48] + 0.5f * t102 * Lp[49] + 0.16666666666666666f * t030 * Lp[52] + 0.5f * t021 * Lp[53] + 0.5f * t012 * Lp[54] + 0.16666666666666666f * t003 * Lp[55];
    Lo[10] = Lp[10] + tx * Lp[20] + ty * Lp[21] + tz * Lp[22] + 0.5f * t200 * Lp[35] + t110 * Lp[36] + t101 * Lp[37] + 0.5f * t020 * Lp[38] + t011 * Lp[39] + 0.5f * t002 * Lp[40];
    Lo[11] = Lp[11] + tx * Lp[21] + ty * Lp[23] + tz * Lp[24] + 0.5f * t200 * Lp[36] + t110 * Lp[38] + t101 * Lp[39] + 0.5f * t020 * Lp[41] + t011 * Lp[42] + 0.5f * t002 * Lp[43];
    Lo[12] = Lp[12] + tx * Lp[22] + ty * Lp[24] + tz * Lp[25] + 0.5f * t200 * Lp[37] + t110 * Lp[39] + t101 * Lp[40] + 0.5f * t020 * Lp[42] + t011 * Lp[43] + 0.5f * t002 * Lp[44];
    Lo[13] = Lp[13] + tx * Lp[23] + ty * Lp[26] + tz * Lp[27] + 0.5f * t200 * Lp[38] + t110 * Lp[41] + t101 * Lp[42] + 0.5f * t020 * Lp[45] + t011 * Lp[46] + 0.5f * t002 * Lp[47];
    Lo[14] = Lp[14] + tx * Lp[24] + ty * Lp[27] + tz * Lp[28] + 0.5f * t200 * Lp[39] + t110 * Lp[42] + t101 * Lp[43] + 0.5f * t020 * Lp[46] + t011 * Lp[47] + 0.5f * t002 * Lp[48];
    Lo[15] = Lp[15] + tx * Lp[25] + ty * Lp[28] + tz * Lp[29] + 0.5f * t200 * Lp[40] + t110 * Lp[43] + t101 * Lp[44] + 0.5f * t020 * Lp[47] + t011 * Lp[48] + 0.5f * t002 * Lp[49];
    Lo[16] = Lp[16] + tx * Lp[26] + ty * Lp[30] + tz * Lp[31] + 0.5f * t200 * Lp[41] + t110 * Lp[45] + t101 * Lp[46] + 0.5f * t020 * Lp[50] + t011 * Lp[51] + 0.5f * t002 * Lp[52];
    Lo[17] = Lp[17] + tx * Lp[27] + ty * Lp[31] + tz * Lp[32] + 0.5f * t200 * Lp[42] + t110 * Lp[46] + t101 * Lp[47] + 0.5f * t020 * Lp[51] + t011 * Lp[52] + 0.5f * t002 * Lp[53];
    Lo[18] = Lp[18] + tx * Lp[28] + ty * Lp[32] + tz * Lp[33] + 0.5f * t200 * Lp[43] + t110 * Lp[47] + t101 * Lp[48] + 0.5f * t020 * Lp[52] + t011 * Lp[53] + 0.5f * t002 * Lp[54];
    Lo[19] = Lp[19] + tx * Lp[29] + ty * Lp[33] + tz * Lp[34] + 0.5f * t200 * Lp[44] + t110 * Lp[48] + t101 * Lp[49] + 0.5f * t020 * Lp[53] + t011 * Lp[54] + 0.5f * t002 * Lp[55];
    Lo[20] = Lp[20] + tx * Lp[35] + ty * Lp[36] + tz * Lp[37];
    Lo[21] = Lp[21] + tx * Lp[36] + ty * Lp[38] + tz * Lp[39];
    Lo[22] = Lp[22] + tx * Lp[37] + ty * Lp[39] + tz * Lp[40];
    Lo[23] = Lp[23] + tx * Lp[38] + ty * Lp[41] + tz * Lp[42];
    Lo[24] = Lp[24] + tx * Lp[39] + ty * Lp[42] + tz * Lp[43];
    Lo[25] = Lp[25] + tx * Lp[40] + ty * Lp[43] + tz * Lp[44];
    Lo[26] = Lp[26] + tx * Lp[41] + ty * Lp[45] + tz * Lp[46];
    Lo[27] = Lp[27] + tx * Lp[42] + ty * Lp[46] + tz * Lp[47];
    Lo[28] = Lp[28] + tx * Lp[43] + ty * Lp[47] + tz * Lp[48];
    Lo[29] = Lp[29] + tx * Lp[44] + ty * Lp[48] + tz * Lp[49];
    Lo[30] = Lp[30] + tx * Lp[45] + ty * Lp[50] + tz * Lp[51];
    Lo[31] = Lp[31] + tx * Lp[46] + ty * Lp[51] + tz * Lp[52];
    Lo[32] = Lp[32] + tx * Lp[47] + ty * Lp[52] + tz * Lp[53];
    Lo[33] = Lp[33] + tx * Lp[48] + ty * Lp[53] + tz * Lp[54];
    Lo[34] = Lp[34] + tx * Lp[49] + ty * Lp[54] + tz * Lp[55];
    Lo[35] = Lp[35];
    Lo[36] = Lp[36];
    Lo[37] = Lp[37];
    Lo[38] = Lp[38];
    Lo[39] = Lp[39];
    Lo[40] = Lp[40];
    Lo[41] = Lp[41];
    Lo[42] = Lp[42];
    Lo[43] = Lp[43];
    Lo[44] = Lp[44];
    Lo[45] = Lp[45];
    Lo[46] = Lp[46];
    Lo[47] = Lp[47];
    Lo[48] = Lp[48];
    Lo[49] = Lp[49];
    Lo[50] = Lp[50];
    Lo[51] = Lp[51];
    Lo[52] = Lp[52];
    Lo[53] = Lp[53];
    Lo[54] = Lp[54];
    Lo[55] = Lp[55];
}

/* local coefficients about c, evaluated at c + u: acceleration += grad Phi, phi -= Phi */
__device__ __forceinline__ void fmm_l2p_acc(const float* __restrict__ Lc, float ux, float uy, float uz,
                                            float& ax, float& ay, float& az, float& phi)
{
    const float u100 = ux;
    const float u010 = uy;
    const float u001 = uz;
    const float u200 = u100 * ux;
    const float u110 = u010 * ux;
    const float u101 = u001 * ux;
    const float u020 = u010 * uy;
    const float u011 = u001 * uy;
    const float u002 = u001 * uz;
    const float u300 = u200 * ux;
    const float u210 = u110 * ux;
    const float u201 = u101 * ux;
    const float u120 = u020 * ux;
    const float u111 = u011 * ux;
    const float u102 = u002 * ux;
    const float u030 = u020 * uy;
    const float u021 = u011 * uy;
    const float u012 = u002 * uy;
    const float u003 = u002 * uz;
    const float u400 = u300 * ux;
    const float u310 = u210 * ux;
    const float u301 = u201 * ux;
    const float u220 = u120 * ux;
    const float u211 = u111 * ux;
    const float u202 = u102 * ux;
    const float u130 = u030 * ux;
    const float u121 = u021 * ux;
    const float u112 = u012 * ux;
    const float u103 = u003 * ux;
    const float u040 = u030 * uy;
    const float u031 = u021 * uy;
    const float u022 = u012 * uy;
    const float u013 = u003 * uy;
    const float u004 = u003 * uz;
    const float u500 = u400 * ux;
    const float u410 = u310 * ux;
    const float u401 = u301 * ux;
    const float u320 = u220 * ux;
    const float u311 = u211 * ux;
    const float u302 = u202 * ux;
    const float u230 = u130 * ux;
    const float u221 = u121 * ux;
    const float u212 = u112 * ux;
    const float u203 = u103 * ux;
    const float u140 = u040 * ux;
    const float u131 = u031 * ux;
    const float u122 = u022 * ux;
    const float u113 = u013 * ux;
    const float u104 = u004 * ux;
    const float u050 = u040 * uy;
    const float u041 = u031 * uy;
    const float u032 = u022 * uy;
    const float u023 = u013 * uy;
    const float u014 = u004 * uy;
    const float u005 = u004 * uz;
    ax += Lc[1] + ux * Lc[4] + uy * Lc[5] + uz * Lc[6] + 0.5f * u200 * Lc[10] + u110 * Lc[11] + u101 * Lc[12] + 0.5f * u020 * Lc[13] + u011 * Lc[14] + 0.5f * u002 * Lc[15] + 0.16666666666666666f * u300 * Lc[20] + 0.5f * u210 * Lc[21] + 0.5f * u201 * Lc[22] + 0.5f * u120 * Lc[23] + u111 * Lc[24] + 0.5f * u102 * Lc[25] + 0.16666666666666666f * u030 * Lc[26] + 0.5f * u021 * Lc[27] + 0.5f * u012 * Lc[28] + 0.16666666666666666f * u003 * Lc[29] + 0.041666666666666664f * u400 * Lc[35] + 0.16666666666666666f * u310 * Lc[36] + 0.16666666666666666f * u301 * Lc[37] + 0.25f * u220 * Lc[38] + 0.5f * u211 * Lc[39] + 0.25f * u202 * Lc[40] + 0.16666666666666666f * u130 * Lc[41] + 0.5f * u121 * Lc[42] + 0.5f * u112 * Lc[43] + 0.16666666666666666f * u103 * Lc[44] + 0.041666666666666664f * u040 * Lc[45] + 0.16666666666666666f * u031 * Lc[46] + 0.25f * u022 * Lc[47] + 0.16666666666666666f * u013 * Lc[48] + 0.041666666666666664f * u004 * Lc[49];
    ay += Lc[2] + ux * Lc[5] + uy * Lc[7] + uz * Lc[8] + 0.5f * u200 * Lc[11] + u110 * Lc[13] + u101 * Lc[14] + 0.5f * u020 * Lc[16] + u011 * Lc[17] + 0.5f * u002 * Lc[18] + 0.16666666666666666f * u300 * Lc[21] + 0.5f * u210 * Lc[23] + 0.5f * u201 * Lc[24] + 0.5f * u120 * Lc[26] + u111 * Lc[27] + 0.5f * u102 * Lc[28] + 0.16666666666666666f * u030 * Lc[30] + 0.5f * u021 * Lc[31] + 0.5f * u012 * Lc[32] + 0.16666666666666666f * u003 * Lc[33] + 0.041666666666666664f * u400 * Lc[36] + 0.16666666666666666f * u310 * Lc[38] + 0.16666666666666666f * u301 * Lc[39] + 0.25f * u220 * Lc[41] + 0.5f * u211 * Lc[42] + 0.25f * u202 * Lc[43] + 0.16666666666666666f * u130 * Lc[45] + 0.5f * u121 * Lc[46] + 0.5f * u112 * Lc[47] + 0.16666666666666666f * u103 * Lc[48] + 0.041666666666666664f * u040 * Lc[50] + 0.16666666666666666f * u031 * Lc[51] + 0.25f * u022 * Lc[52] + 0.16666666666666666f * u013 * Lc[53] + 0.041666666666666664f * u004 * Lc[54];
    az += Lc[3] + ux * Lc[6] + uy * Lc[8] + uz * Lc[9] + 0.5f * u200 * Lc[12] + u110 * Lc[14] + u101 * Lc[15] + 0.5f * u020 * Lc[17] + u011 * Lc[18] + 0.5f * u002 * Lc[19] + 0.16666666666666666f * u300 * Lc[22] + 0.5f * u210 * Lc[24] + 0.5f * u201 * Lc[25] + 0.5f * u120 * Lc[27] + u111 * Lc[28] + 0.5f * u102 * Lc[29] + 0.16666666666666666f * u030 * Lc[31] + 0.5f * u021 * Lc[32] + 0.5f * u012 * Lc[33] + 0.16666666666666666f * u003 * Lc[34] + 0.041666666666666664f * u400 * Lc[37] + 0.16666666666666666f * u310 * Lc[39] + 0.16666666666666666f * u301 * Lc[40] + 0.25f * u220 * Lc[42] + 0.5f * u211 * Lc[43] + 0.25f * u202 * Lc[44] + 0.16666666666666666f * u130 * Lc[46] + 0.5f * u121 * Lc[47] + 0.5f * u112 * Lc[48] + 0.16666666666666666f * u103 * Lc[49] + 0.041666666666666664f * u040 * Lc[51] + 0.16666666666666666f * u031 * Lc[52] + 0.25f * u022 * Lc[53] + 0.16666666666666666f * u013 * Lc[54] + 0.041666666666666664f * u004 * Lc[55];
    phi -= Lc[0] + ux * Lc[1] + uy * Lc[2] + uz * Lc[3] + 0.5f * u200 * Lc[4] + u110 * Lc[5] + u101 * Lc[6] + 0.5f * u020 * Lc[7] + u011 * Lc[8] + 0.5f * u002 * Lc[9] + 0.16666666666666666f * u300 * Lc[10] + 0.5f * u210 * Lc[11] + 0.5f * u201 * Lc[12] + 0.5f * u120 * Lc[13] + u111 * Lc[14] + 0.5f * u102 * Lc[15] + 0.16666666666666666f * u030 * Lc[16] + 0.5f * u021 * Lc[17] + 0.5f * u012 * Lc[18] + 0.16666666666666666f * u003 * Lc[19] + 0.041666666666666664f * u400 * Lc[20] + 0.16666666666666666f * u310 * Lc[21] + 0.16666666666666666f * u301 * Lc[22] + 0.25f * u220 * Lc[23] + 0.5f * u211 * Lc[24] + 0.25f * u202 * Lc[25] + 0.16666666666666666f * u130 * Lc[26] + 0.5f * u121 * Lc[27] + 0.5f * u112 * Lc[28] + 0.16666666666666666f * u103 * Lc[29] + 0.041666666666666664f * u040 * Lc[30] + 0.16666666666666666f * u031 * Lc[31] + 0.25f * u022 * Lc[32] + 0.16666666666666666f * u013 * Lc[33] + 0.041666666666666664f * u004 * Lc[34] + 0.008333333333333333f * u500 * Lc[35] + 0.041666666666666664f * u410 * Lc[36] + 0.041666666666666664f * u401 * Lc[37] + 0.08333333333333333f * u320 * Lc[38] + 0.16666666666666666f * u311 * Lc[39] + 0.08333333333333333f * u302 * Lc[40] + 0.08333333333333333f * u230 * Lc[41] + 0.25f * u221 * Lc[42] + 0.25f * u212 * Lc[43] + 0.08333333333333333f * u203 * Lc[44] + 0.041666666666666664f * u140 * Lc[45] + 0.16666666666666666f * u131 * Lc[46] + 0.25f * u122 * Lc[47] + 0.16666666666666666f * u113 * Lc[48] + 0.041666666666666664f * u104 * Lc[49] + 0.008333333333333333f * u050 * Lc[50] + 0.041666666666666664f * u041 * Lc[51] + 0.08333333333333333f * u032 * Lc[52] + 0.08333333333333333f * u023 * Lc[53] + 0.041666666666666664f * u014 * Lc[54] + 0.008333333333333333f * u005 * Lc[55];
}

/* particle-cell: acceleration and potential at r = x - z of the record R (44 floats, smem) */
__device__ __forceinline__ void fmm_pc_acc(const float* __restrict__ R, float rx, float ry, float rz,
                                           float eps2, float& ax, float& ay, float& az, float& phi)
{
    const float ir = fmm_rsqrt(fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, eps2))));
    const float qx = rx * ir, qy = ry * ir, qz = rz * ir;
    const float ir2 = ir * ir;
    const float A3_300 = R[17] * qx + R[18] * qy + R[19] * qz;
    const float A3_210 = R[18] * qx + R[20] * qy + R[21] * qz;
    const float A3_201 = R[19] * qx + R[21] * qy + R[22] * qz;
    const float A3_120 = R[20] * qx + R[23] * qy + R[24] * qz;
    const float A3_111 = R[21] * qx + R[24] * qy + R[25] * qz;
    const float A3_102 = R[22] * qx + R[25] * qy + R[26] * qz;
    const float A3_030 = R[23] * qx + R[27] * qy + R[28] * qz;
    const float A3_021 = R[24] * qx + R[28] * qy + R[29] * qz;
    const float A3_012 = R[25] * qx + R[29] * qy + R[30] * qz;
    const float A3_003 = R[26] * qx + R[30] * qy + R[31] * qz;
    const float A2_200 = A3_300 * qx + A3_210 * qy + A3_201 * qz;
    const float A2_110 = A3_210 * qx + A3_120 * qy + A3_111 * qz;
    const float A2_101 = A3_201 * qx + A3_111 * qy + A3_102 * qz;
    const float A2_020 = A3_120 * qx + A3_030 * qy + A3_021 * qz;
    const float A2_011 = A3_111 * qx + A3_021 * qy + A3_012 * qz;
    const float A2_002 = A3_102 * qx + A3_012 * qy + A3_003 * qz;
    const float A1_100 = A2_200 * qx + A2_110 * qy + A2_101 * qz;
    const float A1_010 = A2_110 * qx + A2_020 * qy + A2_011 * qz;
    const float A1_001 = A2_101 * qx + A2_011 * qy + A2_002 * qz;
    const float A0_000 = A1_100 * qx + A1_010 * qy + A1_001 * qz;
    const float B2_200 = R[7] * qx + R[8] * qy + R[9] * qz;
    const float B2_110 = R[8] * qx + R[10] * qy + R[11] * qz;
    const float B2_101 = R[9] * qx + R[11] * qy + R[12] * qz;
    const float B2_020 = R[10] * qx + R[13] * qy + R[14] * qz;
    const float B2_011 = R[11] * qx + R[14] * qy + R[15] * qz;
    const float B2_002 = R[12] * qx + R[15] * qy + R[16] * qz;
    const float B1_100 = B2_200 * qx + B2_110 * qy + B2_101 * qz;
    const float B1_010 = B2_110 * qx + B2_020 * qy + B2_011 * qz;
    const float B1_001 = B2_101 * qx + B2_011 * qy + B2_002 * qz;
    const float B0_000 = B1_100 * qx + B1_010 * qy + B1_001 * qz;
    const float C1_100 = R[1] * qx + R[2] * qy + R[3] * qz;
    const float C1_010 = R[2] * qx + R[4] * qy + R[5] * qz;
    const float C1_001 = R[3] * qx + R[5] * qy + R[6] * qz;
    const float C0_000 = C1_100 * qx + C1_010 * qy + C1_001 * qz;
    const float T1_100 = R[36] * qx + R[37] * qy + R[38] * qz;
    const float T1_010 = R[37] * qx + R[39] * qy + R[40] * qz;
    const float T1_001 = R[38] * qx + R[40] * qy + R[41] * qz;
    const float T0_000 = T1_100 * qx + T1_010 * qy + T1_001 * qz;
    const float U0_000 = R[33] * qx + R[34] * qy + R[35] * qz;
    const float p2 = 1.5f * C0_000 - 0.5f * R[32];
    const float p3 = 2.5f * B0_000 - 1.5f * U0_000;
    const float p4 = 4.375f * A0_000 - 3.75f * T0_000 + 0.375f * R[42];
    const float s2 = -7.5f * C0_000 + 1.5f * R[32];
    const float s3 = -17.5f * B0_000 + 7.5f * U0_000;
    const float s4 = -39.375f * A0_000 + 26.25f * T0_000 - 1.875f * R[42];
    const float S = -R[0] + ir2 * (s2 + ir * (s3 + ir * s4));
    phi -= ir * (R[0] + ir2 * (p2 + ir * (p3 + ir * p4)));
    const float vx = 3.0f * C1_100 + ir * ((7.5f * B1_100 - 1.5f * R[33]) + ir * (17.5f * A1_100 - 7.5f * T1_100));
    ax = fmaf(ir2, fmaf(S, qx, ir2 * vx), ax);
    const float vy = 3.0f * C1_010 + ir * ((7.5f * B1_010 - 1.5f * R[34]) + ir * (17.5f * A1_010 - 7.5f * T1_010));
    ay = fmaf(ir2, fmaf(S, qy, ir2 * vy), ay);
    const float vz = 3.0f * C1_001 + ir * ((7.5f * B1_001 - 1.5f * R[35]) + ir * (17.5f * A1_001 - 7.5f * T1_001));
    az = fmaf(ir2, fmaf(S, qz, ir2 * vz), az);
}

/* particle-cell for two sinks (FP32x2 lanes): field of the record R at r0 and r1; phip sums -phi */
__device__ __forceinline__ void fmm_pc_acc2(const float* __restrict__ R, float2 rx, float2 ry, float2 rz,
                                            float2 eps2, float2& ax, float2& ay, float2& az, float2& phip)
{
    const float2 r2 = __ffma2_rn(rx, rx, __ffma2_rn(ry, ry, __ffma2_rn(rz, rz, eps2)));
    const float2 ir = make_float2(fmm_rsqrt(r2.x), fmm_rsqrt(r2.y));
    const float2 qx = __fmul2_rn(rx, ir), qy = __fmul2_rn(ry, ir), qz = __fmul2_rn(rz, ir);
    const float2 ir2 = __fmul2_rn(ir, ir);
    const float2 A3_300 = __ffma2_rn(make_float2(R[19], R[19]), qz, __ffma2_rn(make_float2(R[18], R[18]), qy, __fmul2_rn(make_float2(R[17], R[17]), qx)));
    const float2 A3_210 = __ffma2_rn(make_float2(R[21], R[21]), qz, __ffma2_rn(make_float2(R[20], R[20]), qy, __fmul2_rn(make_float2(R[18], R[18]), qx)));
    const float2 A3_201 = __ffma2_rn(make_float2(R[22], R[22]), qz, __ffma2_rn(make_float2(R[21], R[21]), qy, __fmul2_rn(make_float2(R[19], R[19]), qx)));
    const float2 A3_120 = __ffma2_rn(make_float2(R[24], R[24]), qz, __ffma2_rn(make_float2(R[23], R[23]), qy, __fmul2_rn(make_float2(R[20], R[20]), qx)));
    const float2 A3_111 = __ffma2_rn(make_float2(R[25], R[25]), qz, __ffma2_rn(make_float2(R[24], R[24]), qy, __fmul2_rn(make_float2(R[21], R[21]), qx)));
    const float2 A3_102 = __ffma2_rn(make_float2(R[26], R[26]), qz, __ffma2_rn(make_float2(R[25], R[25]), qy, __fmul2_rn(make_float2(R[22], R[22]), qx)));
    const float2 A3_030 = __ffma2_rn(make_float2(R[28], R[28]), qz, __ffma2_rn(make_float2(R[27], R[27]), qy, __fmul2_rn(make_float2(R[23], R[23]), qx)));
    const float2 A3_021 = __ffma2_rn(make_float2(R[29], R[29]), qz, __ffma2_rn(make_float2(R[28], R[28]), qy, __fmul2_rn(make_float2(R[24], R[24]), qx)));
    const float2 A3_012 = __ffma2_rn(make_float2(R[30], R[30]), qz, __ffma2_rn(make_float2(R[29], R[29]), qy, __fmul2_rn(make_float2(R[25], R[25]), qx)));
    const float2 A3_003 = __ffma2_rn(make_float2(R[31], R[31]), qz, __ffma2_rn(make_float2(R[30], R[30]), qy, __fmul2_rn(make_float2(R[26], R[26]), qx)));
    const float2 A2_200 = __ffma2_rn(A3_201, qz, __ffma2_rn(A3_210, qy, __fmul2_rn(A3_300, qx)));
    const float2 A2_110 = __ffma2_rn(A3_111, qz, __ffma2_rn(A3_120, qy, __fmul2_rn(A3_210, qx)));
    const float2 A2_101 = __ffma2_rn(A3_102, qz, __ffma2_rn(A3_111, qy, __fmul2_rn(A3_201, qx)));
    const float2 A2_020 = __ffma2_rn(A3_021, qz, __ffma2_rn(A3_030, qy, __fmul2_rn(A3_120, qx)));
    const float2 A2_011 = __ffma2_rn(A3_012, qz, __ffma2_rn(A3_021, qy, __fmul2_rn(A3_111, qx)));
    const float2 A2_002 = __ffma2_rn(A3_003, qz, __ffma2_rn(A3_012, qy, __fmul2_rn(A3_102, qx)));
    const float2 A1_100 = __ffma2_rn(A2_101, qz, __ffma2_rn(A2_110, qy, __fmul2_rn(A2_200, qx)));
    const float2 A1_010 = __ffma2_rn(A2_011, qz, __ffma2_rn(A2_020, qy, __fmul2_rn(A2_110, qx)));
    const float2 A1_001 = __ffma2_rn(A2_002, qz, __ffma2_rn(A2_011, qy, __fmul2_rn(A2_101, qx)));
    const float2 A0_000 = __ffma2_rn(A1_001, qz, __ffma2_rn(A1_010, qy, __fmul2_rn(A1_100, qx)));
    const float2 B2_200 = __ffma2_rn(make_float2(R[9], R[9]), qz, __ffma2_rn(make_float2(R[8], R[8]), qy, __fmul2_rn(make_float2(R[7], R[7]), qx)));
    const float2 B2_110 = __ffma2_rn(make_float2(R[11], R[11]), qz, __ffma2_rn(make_float2(R[10], R[10]), qy, __fmul2_rn(make_float2(R[8], R[8]), qx)));
    const float2 B2_101 = __ffma2_rn(make_float2(R[12], R[12]), qz, __ffma2_rn(make_float2(R[11], R[11]), qy, __fmul2_rn(make_float2(R[9], R[9]), qx)));
    const float2 B2_020 = __ffma2_rn(make_float2(R[14], R[14]), qz, __ffma2_rn(make_float2(R[13], R[13]), qy, __fmul2_rn(make_float2(R[10], R[10]), qx)));
    const float2 B2_011 = __ffma2_rn(make_float2(R[15], R[15]), qz, __ffma2_rn(make_float2(R[14], R[14]), qy, __fmul2_rn(make_float2(R[11], R[11]), qx)));
    const float2 B2_002 = __ffma2_rn(make_float2(R[16], R[16]), qz, __ffma2_rn(make_float2(R[15], R[15]), qy, __fmul2_rn(make_float2(R[12], R[12]), qx)));
    const float2 B1_100 = __ffma2_rn(B2_101, qz, __ffma2_rn(B2_110, qy, __fmul2_rn(B2_200, qx)));
    const float2 B1_010 = __ffma2_rn(B2_011, qz, __ffma2_rn(B2_020, qy, __fmul2_rn(B2_110, qx)));
    const float2 B1_001 = __ffma2_rn(B2_002, qz, __ffma2_rn(B2_011, qy, __fmul2_rn(B2_101, qx)));
    const float2 B0_000 = __ffma2_rn(B1_001, qz, __ffma2_rn(B1_010, qy, __fmul2_rn(B1_100, qx)));
    const float2 C1_100 = __ffma2_rn(make_float2(R[3], R[3]), qz, __ffma2_rn(make_float2(R[2], R[2]), qy, __fmul2_rn(make_float2(R[1], R[1]), qx)));
    const float2 C1_010 = __ffma2_rn(make_float2(R[5], R[5]), qz, __ffma2_rn(make_float2(R[4], R[4]), qy, __fmul2_rn(make_float2(R[2], R[2]), qx)));
    const float2 C1_001 = __ffma2_rn(make_float2(R[6], R[6]), qz, __ffma2_rn(make_float2(R[5], R[5]), qy, __fmul2_rn(make_float2(R[3], R[3]), qx)));
    const float2 C0_000 = __ffma2_rn(C1_001, qz, __ffma2_rn(C1_010, qy, __fmul2_rn(C1_100, qx)));
    const float2 T1_100 = __ffma2_rn(make_float2(R[38], R[38]), qz, __ffma2_rn(make_float2(R[37], R[37]), qy, __fmul2_rn(make_float2(R[36], R[36]), qx)));
    const float2 T1_010 = __ffma2_rn(make_float2(R[40], R[40]), qz, __ffma2_rn(make_float2(R[39], R[39]), qy, __fmul2_rn(make_float2(R[37], R[37]), qx)));
    const float2 T1_001 = __ffma2_rn(make_float2(R[41], R[41]), qz, __ffma2_rn(make_float2(R[40], R[40]), qy, __fmul2_rn(make_float2(R[38], R[38]), qx)));
    const float2 T0_000 = __ffma2_rn(T1_001, qz, __ffma2_rn(T1_010, qy, __fmul2_rn(T1_100, qx)));
    const float2 U0_000 = __ffma2_rn(make_float2(R[35], R[35]), qz, __ffma2_rn(make_float2(R[34], R[34]), qy, __fmul2_rn(make_float2(R[33], R[33]), qx)));
    const float2 p2 = __ffma2_rn(make_float2(1.5f, 1.5f), C0_000, make_float2(-0.5f * R[32], -0.5f * R[32]));
    const float2 p3 = __ffma2_rn(make_float2(2.5f, 2.5f), B0_000, __fmul2_rn(make_float2(-1.5f, -1.5f), U0_000));
    const float2 p4 = __ffma2_rn(make_float2(4.375f, 4.375f), A0_000, __ffma2_rn(make_float2(-3.75f, -3.75f), T0_000, make_float2(0.375f * R[42], 0.375f * R[42])));
    const float2 s2 = __ffma2_rn(make_float2(-7.5f, -7.5f), C0_000, make_float2(1.5f * R[32], 1.5f * R[32]));
    const float2 s3 = __ffma2_rn(make_float2(-17.5f, -17.5f), B0_000, __fmul2_rn(make_float2(7.5f, 7.5f), U0_000));
    const float2 s4 = __ffma2_rn(make_float2(-39.375f, -39.375f), A0_000, __ffma2_rn(make_float2(26.25f, 26.25f), T0_000, make_float2(-1.875f * R[42], -1.875f * R[42])));
    const float2 S = __ffma2_rn(ir2, __ffma2_rn(ir, __ffma2_rn(ir, s4, s3), s2), make_float2(-R[0], -R[0]));
    phip = __ffma2_rn(ir, __ffma2_rn(ir2, __ffma2_rn(ir, __ffma2_rn(ir, p4, p3), p2), make_float2(R[0], R[0])), phip);
    const float2 wx = __ffma2_rn(make_float2(17.5f, 17.5f), A1_100, __fmul2_rn(make_float2(-7.5f, -7.5f), T1_100));
    const float2 vx = __ffma2_rn(make_float2(3.0f, 3.0f), C1_100, __fmul2_rn(ir, __ffma2_rn(ir, wx, __ffma2_rn(make_float2(7.5f, 7.5f), B1_100, make_float2(-1.5f * R[33], -1.5f * R[33])))));
    ax = __ffma2_rn(ir2, __ffma2_rn(S, qx, __fmul2_rn(ir2, vx)), ax);
    const float2 wy = __ffma2_rn(make_float2(17.5f, 17.5f), A1_010, __fmul2_rn(make_float2(-7.5f, -7.5f), T1_010));
    const float2 vy = __ffma2_rn(make_float2(3.0f, 3.0f), C1_010, __fmul2_rn(ir, __ffma2_rn(ir, wy, __ffma2_rn(make_float2(7.5f, 7.5f), B1_010, make_float2(-1.5f * R[34], -1.5f * R[34])))));
    ay = __ffma2_rn(ir2, __ffma2_rn(S, qy, __fmul2_rn(ir2, vy)), ay);
    const float2 wz = __ffma2_rn(make_float2(17.5f, 17.5f), A1_001, __fmul2_rn(make_float2(-7.5f, -7.5f), T1_001));
    const float2 vz = __ffma2_rn(make_float2(3.0f, 3.0f), C1_001, __fmul2_rn(ir, __ffma2_rn(ir, wz, __ffma2_rn(make_float2(7.5f, 7.5f), B1_001, make_float2(-1.5f * R[35], -1.5f * R[35])))));
    az = __ffma2_rn(ir2, __ffma2_rn(S, qz, __fmul2_rn(ir2, vz)), az);
}

/* FP32 flops of the generated bodies (fmaf = 2): green 300, p2m 94, m2m 344, traces 22, norms 76, m2l 810, p2l 119, l2l 1095, l2p 499, pc 293 */
#define FMM_FLOPS_PC 293
