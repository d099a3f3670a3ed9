// Learned opening criterion: training (FP32), inference (BF16 tensor cores) and the audit that
// produces training labels from the plain method's own force errors.  Not in the paper, whose
// criterion is the fixed-theta test of Sec. 3.1; see mlp.cuh for the network.
#include <math.h>

#include "expansions.cuh"
#include "fmm_internal.cuh"
#include "mlp.cuh"

// ---------------------------------------------------------------- packing for inference

__global__ void k_mlp_pack(const float* __restrict__ p, unsigned char* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    __nv_bfloat16* w1 = reinterpret_cast<__nv_bfloat16*>(out + MLPP_W1);
    __nv_bfloat16* w2 = reinterpret_cast<__nv_bfloat16*>(out + MLPP_W2);
    __nv_bfloat16* w3 = reinterpret_cast<__nv_bfloat16*>(out + MLPP_W3);
    __nv_bfloat16* w4 = reinterpret_cast<__nv_bfloat16*>(out + MLPP_W4);
    if (i < 64 * 24) {
        const int r = i / 24, c = i % 24;
        w1[i] = __float2bfloat16_rn(c < MLP_F ? p[MLP_W1 + r * MLP_F + c] : 0.0f);
    }
    if (i < 64 * 72) {
        const int r = i / 72, c = i % 72;
        w2[i] = __float2bfloat16_rn(c < MLP_H ? p[MLP_W2 + r * MLP_H + c] : 0.0f);
        w3[i] = __float2bfloat16_rn(c < MLP_H ? p[MLP_W3 + r * MLP_H + c] : 0.0f);
    }
    if (i < 8 * 72) {
        const int r = i / 72, c = i % 72;
        w4[i] = __float2bfloat16_rn(r == 0 && c < MLP_H ? p[MLP_W4 + c] : 0.0f);
    }
    if (i < MLP_H) {
        reinterpret_cast<float*>(out + MLPP_B1)[i] = p[MLP_B1 + i];
        reinterpret_cast<float*>(out + MLPP_B2)[i] = p[MLP_B2 + i];
        reinterpret_cast<float*>(out + MLPP_B3)[i] = p[MLP_B3 + i];
    }
    if (i < 4) reinterpret_cast<float*>(out + MLPP_B4)[i] = i == 0 ? p[MLP_B4] : 0.0f;
    if (i < MLP_F) {
        reinterpret_cast<float*>(out + MLPP_MEAN)[i] = p[MLP_MEAN + i];
        reinterpret_cast<float*>(out + MLPP_ISTD)[i] = p[MLP_ISTD + i];
    }
    if (i < MLP_NSUR) reinterpret_cast<float*>(out + MLPP_SUR)[i] = p[MLP_SUR + i];
}

cudaError_t fmm_mlp_pack(const float* params, unsigned char* packed, cudaStream_t s)
{
    k_mlp_pack<<<(64 * 72 + 255) / 256, 256, 0, s>>>(params, packed);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- training (FP32)

// Gradient of 0.5 * mean((y - label)^2) over a minibatch, accumulated into grad with atomics.
// One block of 64 threads per 64 rows: thread j owns hidden unit j in the forward pass and
// row j of each weight gradient in the backward pass; activations live in shared memory.
#define TB_ROWS 64
#define TPAD 65
__global__ void __launch_bounds__(64) k_mlp_grad(const float* __restrict__ p, const float* __restrict__ feats,
                                                 const float* __restrict__ labels, const unsigned int* __restrict__ idx,
                                                 long long nrows, float inv_b, float loss_scale,
                                                 float* __restrict__ grad, float* __restrict__ loss)
{
    extern __shared__ float sm[];
    float* X = sm;                         // [64][8]
    float* H1 = X + TB_ROWS * MLP_F;       // [64][65]
    float* H2 = H1 + TB_ROWS * TPAD;
    float* H3 = H2 + TB_ROWS * TPAD;
    float* Da = H3 + TB_ROWS * TPAD;
    float* Db = Da + TB_ROWS * TPAD;
    float* dy = Db + TB_ROWS * TPAD;       // [64]
    const int j = threadIdx.x;
    const long long r0 = (long long)blockIdx.x * TB_ROWS;
    const int nr = (int)min((long long)TB_ROWS, nrows - r0);
    // inputs
    if (j < nr) {
        const unsigned int r = idx ? idx[r0 + j] : (unsigned int)(r0 + j);
        for (int k = 0; k < MLP_F; k++) X[j * MLP_F + k] = (feats[(long long)r * MLP_F + k] - p[MLP_MEAN + k]) * p[MLP_ISTD + k];
        dy[j] = labels[r];
    } else {
        for (int k = 0; k < MLP_F; k++) X[j * MLP_F + k] = 0.0f;
        dy[j] = 0.0f;
    }
    __syncthreads();
    // forward: unit j of each layer for all rows
    {
        float w[MLP_F];
        for (int k = 0; k < MLP_F; k++) w[k] = p[MLP_W1 + j * MLP_F + k];
        const float b = p[MLP_B1 + j];
        for (int s = 0; s < TB_ROWS; s++) {
            float z = b;
            for (int k = 0; k < MLP_F; k++) z = fmaf(w[k], X[s * MLP_F + k], z);
            H1[s * TPAD + j] = fmaxf(z, 0.0f);
        }
    }
    __syncthreads();
    const float* Ws[2] = {p + MLP_W2, p + MLP_W3};
    const float* Bs[2] = {p + MLP_B2, p + MLP_B3};
    float* Hin[2] = {H1, H2};
    float* Hout[2] = {H2, H3};
    for (int l = 0; l < 2; l++) {
        const float* W = Ws[l] + j * MLP_H;
        const float b = Bs[l][j];
        for (int s = 0; s < TB_ROWS; s++) {
            float z = b;
            for (int k = 0; k < MLP_H; k++) z = fmaf(__ldg(W + k), Hin[l][s * TPAD + k], z);
            Hout[l][s * TPAD + j] = fmaxf(z, 0.0f);
        }
        __syncthreads();
    }
    // output and its error (thread j = row j)
    {
        float y = p[MLP_B4];
        for (int k = 0; k < MLP_H; k++) y = fmaf(p[MLP_W4 + k], H3[j * TPAD + k], y);
        const float r = j < nr ? y - dy[j] : 0.0f;
        if (j < nr) atomicAdd(loss, 0.5f * r * r * loss_scale);
        __syncthreads();
        dy[j] = r * inv_b;
    }
    __syncthreads();
    // output layer gradient; delta of layer 3 into Da
    {
        float gw = 0.0f, gb = 0.0f;
        const float w4 = p[MLP_W4 + j];
        for (int s = 0; s < TB_ROWS; s++) {
            gw = fmaf(H3[s * TPAD + j], dy[s], gw);
            Da[s * TPAD + j] = H3[s * TPAD + j] > 0.0f ? dy[s] * w4 : 0.0f;
            gb += dy[s];
        }
        atomicAdd(grad + MLP_W4 + j, gw);
        if (j == 0) atomicAdd(grad + MLP_B4, gb);
    }
    __syncthreads();
    // hidden layers 3 and 2: dW[j][k] = sum_s D[s][j] Hin[s][k]; delta_in[s][j] = sum_i D[s][i] W[i][j] (Hin > 0)
    const int offW[2] = {MLP_W3, MLP_W2}, offB[2] = {MLP_B3, MLP_B2};
    float* Hprev[2] = {H2, H1};
    float* Din[2] = {Da, Db};
    float* Dout[2] = {Db, Da};
    for (int l = 0; l < 2; l++) {
        const float* D = Din[l];
        const float* Hp = Hprev[l];
        float gb = 0.0f;
        for (int s = 0; s < TB_ROWS; s++) gb += D[s * TPAD + j];
        atomicAdd(grad + offB[l] + j, gb);
        for (int k = 0; k < MLP_H; k++) {
            float gw = 0.0f;
            for (int s = 0; s < TB_ROWS; s++) gw = fmaf(D[s * TPAD + j], Hp[s * TPAD + k], gw);
            atomicAdd(grad + offW[l] + j * MLP_H + k, gw);
        }
        const float* W = p + offW[l];
        for (int s = 0; s < TB_ROWS; s++) {
            float a = 0.0f;
            for (int i = 0; i < MLP_H; i++) a = fmaf(D[s * TPAD + i], __ldg(W + i * MLP_H + j), a);
            Dout[l][s * TPAD + j] = Hp[s * TPAD + j] > 0.0f ? a : 0.0f;
        }
        __syncthreads();
    }
    // first layer: delta in Da (after two swaps)
    {
        const float* D = Da;
        float gb = 0.0f;
        for (int s = 0; s < TB_ROWS; s++) gb += D[s * TPAD + j];
        atomicAdd(grad + MLP_B1 + j, gb);
        for (int k = 0; k < MLP_F; k++) {
            float gw = 0.0f;
            for (int s = 0; s < TB_ROWS; s++) gw = fmaf(D[s * TPAD + j], X[s * MLP_F + k], gw);
            atomicAdd(grad + MLP_W1 + j * MLP_F + k, gw);
        }
    }
}

static size_t grad_smem() { return (size_t)(TB_ROWS * MLP_F + 5 * TB_ROWS * TPAD + TB_ROWS) * sizeof(float); }

cudaError_t fmm_mlp_grad(const float* params, const float* feats, const float* labels, const unsigned int* idx,
                         long long nrows, float inv_b, float loss_scale, float* grad, float* loss, cudaStream_t s)
{
    static std::atomic<unsigned long long> attr{0};
    cudaError_t e = fmm_smem_attr_once(k_mlp_grad, (int)grad_smem(), attr);
    if (e != cudaSuccess) return e;
    k_mlp_grad<<<(unsigned)fmm_ceil_div(nrows, TB_ROWS), 64, grad_smem(), s>>>(params, feats, labels, idx, nrows, inv_b,
                                                                             loss_scale, grad, loss);
    return cudaGetLastError();
}

// Adam step on the trainable weights (bias-corrected moments)
__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NW) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

cudaError_t fmm_mlp_adam(float* p, const float* g, float* m, float* v, float lr, int step, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_mlp_adam<<<(MLP_NW + 255) / 256, 256, 0, s>>>(p, g, m, v, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- inference (tensor cores)

__global__ void __launch_bounds__(128) k_mlp_predict(const unsigned char* __restrict__ packed,
                                                     const float* __restrict__ feats, long long n,
                                                     float* __restrict__ out)
{
    extern __shared__ __align__(16) unsigned char msm[];
    unsigned char* W = msm;
    unsigned char* scratch = msm + MLPP_SIZE + (threadIdx.x >> 5) * MLP_WARP_SCRATCH;
    mlp_load_smem(packed, W);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = gw * 32; base < n; base += nw * 32) {
        const long long r = base + lane;
        float f[MLP_F];
#pragma unroll
        for (int k = 0; k < MLP_F; k++) f[k] = r < n ? feats[r * MLP_F + k] : 0.0f;
        const float y = mlp_predict_warp(W, scratch, f, lane, __ballot_sync(FMM_FULL_MASK, r < n));
        if (r < n) out[r] = y;
    }
}

size_t fmm_mlp_predict_smem(int warps) { return MLPP_SIZE + (size_t)warps * MLP_WARP_SCRATCH; }

cudaError_t fmm_mlp_predict(const unsigned char* packed, const float* feats, long long n, float* out, cudaStream_t s)
{
    static std::atomic<unsigned long long> attr{0};
    cudaError_t e = fmm_smem_attr_once(k_mlp_predict, (int)fmm_mlp_predict_smem(4), attr);
    if (e != cudaSuccess) return e;
    long long blocks = fmm_ceil_div(n, 128);
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    if (blocks < 1) blocks = 1;
    k_mlp_predict<<<(unsigned)blocks, 128, fmm_mlp_predict_smem(4), s>>>(packed, feats, n, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- audit labels

// For every recorded (sink k, source s) pair: the 8 features and the label log10 of the largest
// relative force error, over up to 32 sink particles i of k, of accepting s for k as a
// cell-cell interaction (M2L about k's centre, then L2P at i) instead of summing s's particles
// directly: |a_expansion - a_direct| / |a_ref_i|, a_ref the particle's total acceleration from a
// reference solve.  One warp per pair, one sampled sink particle per lane.
__global__ void __launch_bounds__(128) k_audit_labels(
    const int2* __restrict__ pairs, long long npairs, const int* __restrict__ cfirst, const int* __restrict__ ccount,
    const Com4* __restrict__ com, const float* __restrict__ rec, const float4* __restrict__ mnorm,
    const float* __restrict__ amin,
    const WalkNode* __restrict__ node, const int* __restrict__ bucket_of, const int* __restrict__ bucket_cell,
    const float4* __restrict__ off, const unsigned int* __restrict__ perm, const float* __restrict__ acc_ref,
    long long n, float eps, float* __restrict__ feats, float* __restrict__ labels)
{
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const float eps2 = eps * eps;
    for (long long q = gw; q < npairs; q += nw) {
        const int k = pairs[q].x, s = pairs[q].y;
        const Com4 ck = com[k], cs = com[s];
        const int fk = cfirst[k], nk = ccount[k], fs = cfirst[s], ns = ccount[s];
        // local expansion of s about k's centre
        float L[FMM_NL];
#pragma unroll
        for (int i = 0; i < FMM_NL; i++) L[i] = 0.0f;
        {
            float M[FMM_NMOM];
            const float4* r4 = reinterpret_cast<const float4*>(rec + (long long)s * FMM_NREC);
#pragma unroll
            for (int i = 0; i < FMM_NMOM / 4; i++) {
                const float4 v = r4[i];
                M[4 * i] = v.x;
                M[4 * i + 1] = v.y;
                M[4 * i + 2] = v.z;
                M[4 * i + 3] = v.w;
            }
            fmm_m2l_acc(M, __double2float_rn(ck.x - cs.x), __double2float_rn(ck.y - cs.y),
                        __double2float_rn(ck.z - cs.z), eps2, L);
        }
        float err = 0.0f;
        const int ns_sample = nk < 32 ? nk : 32;
        if (lane < ns_sample) {
            const int i = fk + (int)(((long long)lane * nk) / ns_sample);
            const Com4 cb = com[bucket_cell[bucket_of[i]]];
            const float4 oi = off[i];
            const float ux = __double2float_rn(cb.x - ck.x) + oi.x, uy = __double2float_rn(cb.y - ck.y) + oi.y,
                        uz = __double2float_rn(cb.z - ck.z) + oi.z;
            float ax = 0.f, ay = 0.f, az = 0.f, ph = 0.f;
            fmm_l2p_acc(L, ux, uy, uz, ax, ay, az, ph);
            float ex = 0.f, ey = 0.f, ez = 0.f;
            int b = -1;
            float bx = 0.f, by = 0.f, bz = 0.f;
            for (int j = fs; j < fs + ns; j++) {
                const int bj = bucket_of[j];
                if (bj != b) {
                    b = bj;
                    const Com4 cj = com[bucket_cell[bj]];
                    bx = __double2float_rn(cj.x - ck.x);
                    by = __double2float_rn(cj.y - ck.y);
                    bz = __double2float_rn(cj.z - ck.z);
                }
                const float4 o = off[j];
                const float dx = bx + o.x - ux, dy = by + o.y - uy, dz = bz + o.z - uz;
                const float ir = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2))));
                const float w = o.w * ir * ir * ir;
                ex = fmaf(w, dx, ex);
                ey = fmaf(w, dy, ey);
                ez = fmaf(w, dz, ez);
            }
            const unsigned int pi = perm[i];
            const float rx = acc_ref[pi], ry = acc_ref[n + pi], rz = acc_ref[2 * n + pi];
            const float ref = sqrtf(rx * rx + ry * ry + rz * rz);
            const float dxe = ax - ex, dye = ay - ey, dze = az - ez;
            err = sqrtf(dxe * dxe + dye * dye + dze * dze) / fmaxf(ref, 1e-30f);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) err = fmaxf(err, __shfl_xor_sync(FMM_FULL_MASK, err, o));
        if (lane == 0) {
            labels[q] = log10f(err + 1e-12f);
            mlp_pair_features(node[k], node[s], mnorm[s], amin[k], eps, feats + q * MLP_F);
        }
    }
}

cudaError_t fmm_launch_audit_labels(DevTree& t, const int2* pairs, long long npairs, const float* acc_ref,
                                    long long n, float eps, float* feats, float* labels, cudaStream_t s)
{
    long long blocks = fmm_ceil_div(npairs, 4);
    if (blocks > 152LL * 32) blocks = 152LL * 32;
    if (blocks < 1) blocks = 1;
    k_audit_labels<<<(unsigned)blocks, 128, 0, s>>>(pairs, npairs, t.cfirst, t.ccount, t.com, t.rec, t.mnorm, t.amin, t.node,
                                                     t.bucket_of, t.bucket_cell, t.off, t.idx, acc_ref, n, eps, feats,
                                                     labels);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- sink acceleration scale

// Per cell, the smallest |a| of its particles from an acceleration estimate acc (3 x n SoA in
// input order, e.g. the previous step's forces): bucket cells scan their particles, and the
// second child to arrive at a parent takes the smaller of the two (arrive[] zeroed first).
__global__ void __launch_bounds__(128) k_cell_amin(const unsigned int* __restrict__ nbucket,
                                                   const int* __restrict__ bucket_cell,
                                                   const int* __restrict__ cfirst, const int* __restrict__ ccount,
                                                   const int* __restrict__ cparent, const int* __restrict__ cchild,
                                                   const unsigned int* __restrict__ perm,
                                                   const float* __restrict__ acc, long long n, float* amin,
                                                   unsigned int* arrive)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int)*nbucket) return;
    const int c = bucket_cell[b];
    float a = INFINITY;
    for (int j = cfirst[c], e = cfirst[c] + ccount[c]; j < e; j++) {
        const unsigned int p = perm[j];
        const float x = acc[p], y = acc[n + p], z = acc[2 * n + p];
        a = fminf(a, sqrtf(x * x + y * y + z * z));
    }
    amin[c] = a;
    int p = cparent[c];
    while (p >= 0) {
        __threadfence();
        if (atomicAdd(&arrive[p], 1u) == 0u) return;
        __threadfence();
        amin[p] = fminf(__ldcg(&amin[cchild[2 * p]]), __ldcg(&amin[cchild[2 * p + 1]]));
        p = cparent[p];
    }
}

cudaError_t fmm_launch_cell_amin(DevTree& t, const float* acc, long long n, cudaStream_t s)
{
    const long long nb = t.cap_grid ? t.cap_cells : t.n_buckets, nc = t.cap_grid ? t.cap_cells : t.n_cells;
    cudaError_t e = cudaMemsetAsync(t.arrive, 0, sizeof(unsigned int) * (size_t)nc, s);
    if (e != cudaSuccess) return e;
    k_cell_amin<<<(unsigned)fmm_ceil_div(nb, 128), 128, 0, s>>>(t.dcount + 1, t.bucket_cell, t.cfirst, t.ccount,
                                                                 t.cparent, t.cchild, t.idx, acc, n, t.amin, t.arrive);
    return cudaGetLastError();
}
