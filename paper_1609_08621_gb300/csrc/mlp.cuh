// Learned opening criterion: network layout and the warp-level tensor-core forward pass.
//
// The network (not in the paper, whose criterion is the fixed-theta test of Sec. 3.1)
// predicts log10 of the force error of accepting a (sink cell, source cell) pair as a
// cell-cell interaction, from 8 features:
//   x (8) -> relu(W1 x + b1) (64) -> relu(W2 . + b2) (64) -> relu(W3 . + b3) (64) -> w4 . + b4
// Master weights are FP32 (flat layout MLP_* offsets below, followed by the feature
// normalisation mean[8], inv_std[8]); inference uses a BF16 copy with FP32 accumulation on the
// tensor cores (mma.sync m16n8k16, one warp evaluates 32 samples).
#pragma once

#include <cuda_bf16.h>

#include "fmm_internal.cuh"

#define MLP_F 8
#define MLP_H 64
// flat FP32 parameter layout
#define MLP_W1 0
#define MLP_B1 (MLP_W1 + MLP_H * MLP_F)
#define MLP_W2 (MLP_B1 + MLP_H)
#define MLP_B2 (MLP_W2 + MLP_H * MLP_H)
#define MLP_W3 (MLP_B2 + MLP_H)
#define MLP_B3 (MLP_W3 + MLP_H * MLP_H)
#define MLP_W4 (MLP_B3 + MLP_H)
#define MLP_B4 (MLP_W4 + MLP_H)
#define MLP_NW (MLP_B4 + 1)          // 8961 trainable weights
#define MLP_MEAN MLP_NW
#define MLP_ISTD (MLP_MEAN + MLP_F)
// surrogate bound of the network's output, set by training: alpha, beta, r_lo, r_hi, then the
// coefficients gamma[8] of the raw features (see mlp_surrogate); r_hi <= r_lo switches it off
#define MLP_NSUR 12
#define MLP_SUR (MLP_ISTD + MLP_F)
#define MLP_NP (MLP_SUR + MLP_NSUR)  // 8989 parameters in all

// packed inference layout (bytes), identical in global and shared memory; matrix rows are
// padded (24 / 72 BF16) so the fragment loads of the 8 row groups hit distinct banks
#define MLPP_W1 0        // [64][24] bf16, columns 8..23 zero
#define MLPP_W2 3072     // [64][72] bf16
#define MLPP_W3 12288    // [64][72] bf16
#define MLPP_W4 21504    // [8][72] bf16, row 0 = w4, rows 1..7 zero
#define MLPP_B1 22656    // [64] f32
#define MLPP_B2 22912
#define MLPP_B3 23168
#define MLPP_B4 23424    // f32 (16 bytes reserved)
#define MLPP_MEAN 23440  // [8] f32
#define MLPP_ISTD 23472  // [8] f32
#define MLPP_SUR 23504   // [12] f32
#define MLPP_SIZE 23552
// per-warp scratch of the forward pass: inputs [32][24] bf16 and predictions [32] f32
#define MLP_WARP_SCRATCH (32 * 24 * 2 + 32 * 4)

__device__ __forceinline__ unsigned int mlp_pack2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned int*>(&v);
}

__device__ __forceinline__ void mlp_mma(float* c, const unsigned int* a, unsigned int b0, unsigned int b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// copy the packed weights into shared memory (whole block)
__device__ __forceinline__ void mlp_load_smem(const unsigned char* __restrict__ g, unsigned char* s)
{
    const uint4* src = reinterpret_cast<const uint4*>(g);
    uint4* dst = reinterpret_cast<uint4*>(s);
    for (int i = threadIdx.x; i < MLPP_SIZE / 16; i += blockDim.x) dst[i] = src[i];
}

// one hidden layer for one m-tile (16 samples): in A fragments (4 k-tiles), out A fragments
__device__ __forceinline__ void mlp_hidden(const unsigned char* W, int wbyte, int bbyte, int ktiles, int wstride,
                                           const unsigned int (*ain)[4], unsigned int (*aout)[4], int g, int t)
{
    const __nv_bfloat16* w = reinterpret_cast<const __nv_bfloat16*>(W + wbyte);
    const float* b = reinterpret_cast<const float*>(W + bbyte);
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        acc[nt][0] = acc[nt][2] = b[nt * 8 + 2 * t];
        acc[nt][1] = acc[nt][3] = b[nt * 8 + 2 * t + 1];
    }
    for (int kt = 0; kt < ktiles; kt++) {
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const __nv_bfloat16* row = w + (nt * 8 + g) * wstride + kt * 16 + 2 * t;
            const unsigned int b0 = *reinterpret_cast<const unsigned int*>(row);
            const unsigned int b1 = *reinterpret_cast<const unsigned int*>(row + 8);
            mlp_mma(acc[nt], ain[kt], b0, b1);
        }
    }
#pragma unroll
    for (int kt = 0; kt < 4; kt++) {
        aout[kt][0] = mlp_pack2(fmaxf(acc[2 * kt][0], 0.f), fmaxf(acc[2 * kt][1], 0.f));
        aout[kt][1] = mlp_pack2(fmaxf(acc[2 * kt][2], 0.f), fmaxf(acc[2 * kt][3], 0.f));
        aout[kt][2] = mlp_pack2(fmaxf(acc[2 * kt + 1][0], 0.f), fmaxf(acc[2 * kt + 1][1], 0.f));
        aout[kt][3] = mlp_pack2(fmaxf(acc[2 * kt + 1][2], 0.f), fmaxf(acc[2 * kt + 1][3], 0.f));
    }
}

// Forward pass of the samples held by the lanes in mask (lane i: raw features f[8]).  The samples
// are packed into the first popc(mask) rows, so a warp with at most 16 of them runs one m-tile
// instead of two.  W: packed weights in shared memory; scratch: this warp's MLP_WARP_SCRATCH
// bytes.  All 32 lanes must call it (mma.sync is warp-wide); returns this lane's prediction
// (meaningful for lanes in mask).
__device__ __forceinline__ float mlp_predict_warp(const unsigned char* W, unsigned char* scratch, const float* f,
                                                  int lane, unsigned int mask)
{
    __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(scratch);
    float* ps = reinterpret_cast<float*>(scratch + 32 * 24 * 2);
    const float* mean = reinterpret_cast<const float*>(W + MLPP_MEAN);
    const float* istd = reinterpret_cast<const float*>(W + MLPP_ISTD);
    const unsigned int lt = (1u << lane) - 1u;
    const int cnt = __popc(mask);
    const int row = ((mask >> lane) & 1u) ? __popc(mask & lt) : cnt + __popc(~mask & lt);
#pragma unroll
    for (int k = 0; k < MLP_F; k++) xs[row * 24 + k] = __float2bfloat16_rn((f[k] - mean[k]) * istd[k]);
#pragma unroll
    for (int k = MLP_F; k < 16; k++) xs[row * 24 + k] = __float2bfloat16_rn(0.0f);
    __syncwarp();
    const int g = lane >> 2, t = lane & 3;
    const float b4 = *reinterpret_cast<const float*>(W + MLPP_B4);
    const int mtiles = (cnt + 15) >> 4;
    for (int mt = 0; mt < mtiles; mt++) {
        const int r0 = mt * 16 + g, r1 = r0 + 8;
        unsigned int a1[4][4], a2[4][4];
        a1[0][0] = *reinterpret_cast<const unsigned int*>(xs + r0 * 24 + 2 * t);
        a1[0][1] = *reinterpret_cast<const unsigned int*>(xs + r1 * 24 + 2 * t);
        a1[0][2] = *reinterpret_cast<const unsigned int*>(xs + r0 * 24 + 2 * t + 8);
        a1[0][3] = *reinterpret_cast<const unsigned int*>(xs + r1 * 24 + 2 * t + 8);
        mlp_hidden(W, MLPP_W1, MLPP_B1, 1, 24, a1, a2, g, t);
        mlp_hidden(W, MLPP_W2, MLPP_B2, 4, 72, a2, a1, g, t);
        mlp_hidden(W, MLPP_W3, MLPP_B3, 4, 72, a1, a2, g, t);
        float out[4] = {0.f, 0.f, 0.f, 0.f};
        const __nv_bfloat16* w4 = reinterpret_cast<const __nv_bfloat16*>(W + MLPP_W4);
#pragma unroll
        for (int kt = 0; kt < 4; kt++) {
            const __nv_bfloat16* row = w4 + g * 72 + kt * 16 + 2 * t;
            mlp_mma(out, a2[kt], *reinterpret_cast<const unsigned int*>(row),
                    *reinterpret_cast<const unsigned int*>(row + 8));
        }
        if (t == 0) {
            ps[r0] = out[0] + b4;
            ps[r1] = out[2] + b4;
        }
    }
    __syncwarp();
    const float p = ps[row];
    __syncwarp();
    return p;
}

// The band in which the network decides: theta_eff = (1.5 b_max(k) + b_max(s)) / d is the smallest
// opening angle at which the fixed criterion would accept the pair.  A hard guard applies first:
// never accept unless d > 1.1 (b_max(k) + b_max(s)) (the expansion converges) and the bounding
// boxes are >= 2 eps apart.  Returns 0 = guard fails (not accepted), 1 = accept without the
// network (theta_eff < band_lo), 2 = reject (theta_eff >= band_hi), 3 = the network decides;
// te = theta_eff.
__device__ __forceinline__ int mlp_band(const WalkNode& K, const WalkNode& S, float d2, float gap2, float four_eps2,
                                        float band_lo, float band_hi, float& te)
{
    const float d = sqrtf(d2), bk = K.b.w, bs = S.b.w;
    te = 0.0f;
    if (!(d > 1.1f * (bk + bs)) || !(gap2 >= four_eps2)) return 0;
    te = (1.5f * bk + bs) / d;
    if (te < band_lo) return 1;
    if (te >= band_hi) return 2;
    return 3;
}

// the 8 features of a (sink k, source s) pair: b_max(s)/d, b_max(k)/d, eps/d,
// log10(M_s / (d^2 a_k)) (the source's monopole field at the sink relative to the sink's smallest
// particle acceleration a_k), log2 N_s, log2 N_k, |M2|_F/(M b^2), |M4|_F/(M b^4) of the source.
// mn = (|M2| norm, |M4| norm, M_s, -) of the source; ak = a_k (clamped below at 1e-30).
__device__ __forceinline__ void mlp_pair_features(const WalkNode& K, const WalkNode& S, float4 mn, float ak, float eps,
                                                  float* f)
{
    const float dx = K.a.x - S.a.x, dy = K.a.y - S.a.y, dz = K.a.z - S.a.z;
    const float d2 = dx * dx + dy * dy + dz * dz;
    const float d = sqrtf(d2);
    const float id = 1.0f / d;
    f[0] = S.b.w * id;
    f[1] = K.b.w * id;
    f[2] = eps * id;
    f[3] = log10f(mn.z) - log10f(d2) - log10f(fmaxf(ak, 1e-30f));
    f[4] = log2f((float)S.d.w);
    f[5] = log2f((float)K.d.w);
    f[6] = mn.x;
    f[7] = mn.y;
}

// Surrogate of the network's output, linear in the raw features f[8] around the physical scaling of
// a truncated expansion's error (the source's monopole field relative to the sink's acceleration,
// f[3], times a power of the opening angle):
//   y_lin = f[3] + alpha log10(theta_eff) + beta + sum_i gamma_i f[i].
// Training fits it to the labels by least squares and records the range [r_lo, r_hi] of the
// network's residual y_net - y_lin over its training rows (0.05% quantiles).  With the margin m in
// [0, 1] (fmm_params.mlp_margin), a pair with y_lin + m r_hi < tau is accepted and one with
// y_lin + m r_lo >= tau rejected without running the network; the network decides the pairs in
// between, where the surrogate's prediction lies near the budget.  m = 1 leaves the network every
// pair the surrogate could get wrong on the training rows; m = 0 lets the surrogate decide alone.
// sur: the MLP_NSUR floats.  Returns 1 accept, 2 reject, 3 ask the network.
__device__ __forceinline__ int mlp_surrogate(const float* sur, const float* f, float te, float tau, float margin)
{
    const float r_lo = sur[2], r_hi = sur[3];
    if (!(r_hi > r_lo)) return 3;  // no surrogate fitted: the network decides every band pair
    float y = f[3] + sur[0] * log10f(te) + sur[1];
#pragma unroll
    for (int i = 0; i < MLP_F; i++) y = fmaf(sur[4 + i], f[i], y);
    if (y + margin * r_hi < tau) return 1;
    if (y + margin * r_lo >= tau) return 2;
    return 3;
}
