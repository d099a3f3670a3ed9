// Interaction evaluation per sink group (Sec. 3.1, Sec. 3.3): particle-particle (PP),
// particle-cell (PC) and the group's local expansion at its particles (L2P), then the
// results are written back in the caller's order.
//
// One warp per group; lane l holds sinks l and l + 32 (g <= 64) in registers.  All
// coordinates are single precision offsets from the group's centre of mass c_g
// (Sec. 3.1: interactions in single precision):
//   sink     u_i = fl(com_bucket(i) - c_g) + fl(x_i - com_bucket(i))
//   source   s_j = fl(com_bucket(j) - c_g) + fl(x_j - com_bucket(j))
//   cell     z_s = fl(com_s - c_g)
// where the differences of double-precision centres are formed in FP64 and rounded once
// per bucket or cell (never per interaction: FP64 issue is 1/64 of FP32 on this GPU),
// and fl(x - com_bucket) is stored per particle by the upward pass.
//
// PP: a_i += m_j (s_j - u_i) / (|s_j - u_i|^2 + eps^2)^(3/2), phi_i -= m_j / (...)^(1/2)
// over every particle of every PP source, the sink itself included: its force term is
// exactly zero (identical offsets) and its potential term m_i / eps is removed at the end
// by adding back the identically computed value.  Source particles are staged per warp in
// shared memory (32 list entries at a time, <= 16 particles each).
// PC: the order-4 moment record of each source cell evaluated at u_i - z_s
// (fmm_pc_acc, trace form).  Records of 32 cells are staged per warp in shared memory.
// L2P: the group's order-5 local coefficients evaluated at u_i.
#include "expansions.cuh"
#include "fmm_internal.cuh"

#define IW 4  // warps per block
#define ITHREADS (IW * 32)
#define PP_TILE 512

struct SinkPair {
    float ux0, uy0, uz0, ux1, uy1, uz1;
    float m0, m1;
    int s0, s1;
    bool v0, v1;
};

__device__ __forceinline__ void load_sinks(const Group& G, const Com4& ck, const int* __restrict__ bucket_of,
                                           const int* __restrict__ bucket_cell, const Com4* __restrict__ com,
                                           const float4* __restrict__ off, int lane, SinkPair& S)
{
    S.s0 = G.first + lane;
    S.s1 = G.first + lane + 32;
    S.v0 = lane < G.count;
    S.v1 = lane + 32 < G.count;
    S.ux0 = S.uy0 = S.uz0 = S.ux1 = S.uy1 = S.uz1 = 0.0f;
    S.m0 = S.m1 = 0.0f;
    if (S.v0) {
        Com4 cb = com[bucket_cell[bucket_of[S.s0]]];
        float4 o = off[S.s0];
        S.ux0 = __double2float_rn(cb.x - ck.x) + o.x;
        S.uy0 = __double2float_rn(cb.y - ck.y) + o.y;
        S.uz0 = __double2float_rn(cb.z - ck.z) + o.z;
        S.m0 = o.w;
    }
    if (S.v1) {
        Com4 cb = com[bucket_cell[bucket_of[S.s1]]];
        float4 o = off[S.s1];
        S.ux1 = __double2float_rn(cb.x - ck.x) + o.x;
        S.uy1 = __double2float_rn(cb.y - ck.y) + o.y;
        S.uz1 = __double2float_rn(cb.z - ck.z) + o.z;
        S.m1 = o.w;
    }
}

__device__ __forceinline__ void pp_pair(float ux, float uy, float uz, float4 s, float eps2, float& ax, float& ay,
                                        float& az, float& ph)
{
    const float dx = s.x - ux, dy = s.y - uy, dz = s.z - uz;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    const float ir = rsqrtf(r2);
    const float mir = s.w * ir;
    const float mir3 = mir * ir * ir;
    ax = fmaf(mir3, dx, ax);
    ay = fmaf(mir3, dy, ay);
    az = fmaf(mir3, dz, az);
    ph -= mir;
}

__global__ void __launch_bounds__(ITHREADS) k_pp(const Group* __restrict__ groups, long long n_groups,
                                                 const unsigned int* __restrict__ pp, const int* __restrict__ cfirst,
                                                 const int* __restrict__ ccount, const int* __restrict__ cnact,
                                                 const Com4* __restrict__ com, const int* __restrict__ bucket_of,
                                                 const int* __restrict__ bucket_cell, const float4* __restrict__ off,
                                                 float4* __restrict__ accs, float eps2, int enabled,
                                                 DevCounters* __restrict__ ctr)
{
    __shared__ float4 tile[IW][PP_TILE];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    float4* T = tile[wl];
    unsigned long long pairs = 0;
    for (long long gi = gw; gi < n_groups; gi += nw) {
        const Group G = groups[gi];
        const Com4 ck = com[G.cell];
        SinkPair S;
        load_sinks(G, ck, bucket_of, bucket_cell, com, off, lane, S);
        float ax0 = 0.f, ay0 = 0.f, az0 = 0.f, p0 = 0.f, ax1 = 0.f, ay1 = 0.f, az1 = 0.f, p1 = 0.f;
        long long nsrc = 0;
        if (enabled) {
            for (int base = 0; base < G.pp_len; base += 32) {
                const int ne = min(32, G.pp_len - base);
                int first = 0, cnt = 0;
                float dx = 0.f, dy = 0.f, dz = 0.f;
                if (lane < ne) {
                    unsigned int e = pp[G.pp_off + base + lane];
                    int bc;
                    if (e & FMM_PARTICLE_BIT) {
                        first = (int)(e & ~FMM_PARTICLE_BIT);
                        cnt = 1;
                        bc = bucket_cell[bucket_of[first]];
                    } else {
                        first = cfirst[e];
                        cnt = ccount[e];
                        bc = (int)e;
                    }
                    Com4 cb = com[bc];
                    dx = __double2float_rn(cb.x - ck.x);
                    dy = __double2float_rn(cb.y - ck.y);
                    dz = __double2float_rn(cb.z - ck.z);
                }
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int t = __shfl_up_sync(FMM_FULL_MASK, incl, o);
                    if (lane >= o) incl += t;
                }
                const int total = __shfl_sync(FMM_FULL_MASK, incl, 31);
                const int excl = incl - cnt;
                for (int j = 0; j < ne; j++) {
                    const int fj = __shfl_sync(FMM_FULL_MASK, first, j);
                    const int nj = __shfl_sync(FMM_FULL_MASK, cnt, j);
                    const int pj = __shfl_sync(FMM_FULL_MASK, excl, j);
                    const float ex = __shfl_sync(FMM_FULL_MASK, dx, j);
                    const float ey = __shfl_sync(FMM_FULL_MASK, dy, j);
                    const float ez = __shfl_sync(FMM_FULL_MASK, dz, j);
                    if (lane < nj) {
                        float4 o = off[fj + lane];
                        T[pj + lane] = make_float4(ex + o.x, ey + o.y, ez + o.z, o.w);
                    }
                }
                __syncwarp();
                for (int t = 0; t < total; t++) {
                    const float4 s = T[t];
                    pp_pair(S.ux0, S.uy0, S.uz0, s, eps2, ax0, ay0, az0, p0);
                    pp_pair(S.ux1, S.uy1, S.uz1, s, eps2, ax1, ay1, az1, p1);
                }
                nsrc += total;
                __syncwarp();
            }
            // remove the self term of the potential (the force term is exactly zero)
            const float ie = rsqrtf(eps2);
            p0 += S.m0 * ie;
            p1 += S.m1 * ie;
        }
        if (S.v0) accs[S.s0] = make_float4(ax0, ay0, az0, p0);
        if (S.v1) accs[S.s1] = make_float4(ax1, ay1, az1, p1);
        if (lane == 0) pairs += (unsigned long long)cnact[G.cell] * (unsigned long long)nsrc;
    }
    if (lane == 0 && pairs) atomicAdd(&ctr->n_pp_pairs, pairs);
}

#define PC_CHUNK 32

__global__ void __launch_bounds__(ITHREADS) k_pc(const Group* __restrict__ groups, long long n_groups,
                                                 const unsigned int* __restrict__ pc, const int* __restrict__ cnact,
                                                 const Com4* __restrict__ com, const int* __restrict__ bucket_of,
                                                 const int* __restrict__ bucket_cell, const float4* __restrict__ off,
                                                 const float* __restrict__ rec, float4* __restrict__ accs, float eps2,
                                                 DevCounters* __restrict__ ctr)
{
    __shared__ float4 R4[IW][PC_CHUNK * FMM_NREC / 4];
    __shared__ float4 Z[IW][PC_CHUNK];
    __shared__ int ids[IW][PC_CHUNK];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const float4* rec4 = reinterpret_cast<const float4*>(rec);
    unsigned long long pairs = 0;
    for (long long gi = gw; gi < n_groups; gi += nw) {
        const Group G = groups[gi];
        if (G.pc_len == 0) continue;
        const Com4 ck = com[G.cell];
        SinkPair S;
        load_sinks(G, ck, bucket_of, bucket_cell, com, off, lane, S);
        float ax0 = 0.f, ay0 = 0.f, az0 = 0.f, p0 = 0.f, ax1 = 0.f, ay1 = 0.f, az1 = 0.f, p1 = 0.f;
        for (int base = 0; base < G.pc_len; base += PC_CHUNK) {
            const int ne = min(PC_CHUNK, G.pc_len - base);
            if (lane < ne) {
                unsigned int c = pc[G.pc_off + base + lane];
                Com4 cs = com[c];
                ids[wl][lane] = (int)c;
                Z[wl][lane] = make_float4(__double2float_rn(cs.x - ck.x), __double2float_rn(cs.y - ck.y),
                                          __double2float_rn(cs.z - ck.z), 0.0f);
            }
            __syncwarp();
            const int nv = ne * (FMM_NREC / 4);
            for (int i = lane; i < nv; i += 32) {
                int cl = i / (FMM_NREC / 4), part = i - cl * (FMM_NREC / 4);
                R4[wl][i] = rec4[(long long)ids[wl][cl] * (FMM_NREC / 4) + part];
            }
            __syncwarp();
            for (int j = 0; j < ne; j++) {
                const float* Rj = reinterpret_cast<const float*>(&R4[wl][j * (FMM_NREC / 4)]);
                const float4 z = Z[wl][j];
                fmm_pc_acc(Rj, S.ux0 - z.x, S.uy0 - z.y, S.uz0 - z.z, eps2, ax0, ay0, az0, p0);
                fmm_pc_acc(Rj, S.ux1 - z.x, S.uy1 - z.y, S.uz1 - z.z, eps2, ax1, ay1, az1, p1);
            }
            __syncwarp();
        }
        if (S.v0) {
            float4 a = accs[S.s0];
            accs[S.s0] = make_float4(a.x + ax0, a.y + ay0, a.z + az0, a.w + p0);
        }
        if (S.v1) {
            float4 a = accs[S.s1];
            accs[S.s1] = make_float4(a.x + ax1, a.y + ay1, a.z + az1, a.w + p1);
        }
        if (lane == 0) pairs += (unsigned long long)cnact[G.cell] * (unsigned long long)G.pc_len;
    }
    if (lane == 0 && pairs) atomicAdd(&ctr->n_pc_pairs, pairs);
}

__global__ void __launch_bounds__(ITHREADS) k_l2p_out(const Group* __restrict__ groups, long long n_groups,
                                                      const Com4* __restrict__ com,
                                                      const int* __restrict__ bucket_of,
                                                      const int* __restrict__ bucket_cell,
                                                      const float4* __restrict__ off, const float* __restrict__ L,
                                                      const float4* __restrict__ accs,
                                                      const unsigned char* __restrict__ sact,
                                                      const unsigned int* __restrict__ perm, long long n,
                                                      float* __restrict__ acc, float* __restrict__ pot, int use_local)
{
    __shared__ float Ls[IW][FMM_NL];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long gi = gw; gi < n_groups; gi += nw) {
        const Group G = groups[gi];
        const Com4 ck = com[G.cell];
        SinkPair S;
        load_sinks(G, ck, bucket_of, bucket_cell, com, off, lane, S);
        for (int i = lane; i < FMM_NL; i += 32) Ls[wl][i] = L[(long long)G.cell * FMM_NL + i];
        __syncwarp();
        for (int h = 0; h < 2; h++) {
            const bool v = h ? S.v1 : S.v0;
            if (!v) continue;
            const int s = h ? S.s1 : S.s0;
            float4 a = accs[s];
            if (use_local) {
                if (h) fmm_l2p_acc(Ls[wl], S.ux1, S.uy1, S.uz1, a.x, a.y, a.z, a.w);
                else fmm_l2p_acc(Ls[wl], S.ux0, S.uy0, S.uz0, a.x, a.y, a.z, a.w);
            }
            if (sact[s]) {
                const unsigned int p = perm[s];
                acc[p] = a.x;
                acc[n + p] = a.y;
                acc[2 * n + p] = a.z;
                if (pot) pot[p] = a.w;
            }
        }
        __syncwarp();
    }
}

int fmm_interact_blocks(int device)
{
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms;
}

static unsigned grid_for(long long n_groups)
{
    long long b = fmm_ceil_div(n_groups, IW);
    if (b > 65535LL * 8) b = 65535LL * 8;
    return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t fmm_launch_pp(DevTree& t, DevWalk& w, DevCounters* ctr, const InteractArgs& a, cudaStream_t s)
{
    k_pp<<<grid_for(w.n_groups), ITHREADS, 0, s>>>(w.groups, w.n_groups, w.pp, t.cfirst, t.ccount, t.cnact, t.com,
                                                   t.bucket_of, t.bucket_cell, t.off, t.accs, a.eps2, a.terms & 1,
                                                   ctr);
    return cudaGetLastError();
}

cudaError_t fmm_launch_pc(DevTree& t, DevWalk& w, DevCounters* ctr, const InteractArgs& a, cudaStream_t s)
{
    if (!(a.terms & 2)) return cudaSuccess;
    k_pc<<<grid_for(w.n_groups), ITHREADS, 0, s>>>(w.groups, w.n_groups, w.pc, t.cnact, t.com, t.bucket_of,
                                                   t.bucket_cell, t.off, t.rec, t.accs, a.eps2, ctr);
    return cudaGetLastError();
}

cudaError_t fmm_launch_l2p_out(DevTree& t, DevWalk& w, DevCounters* ctr, const InteractArgs& a, float* acc,
                               float* pot, long long n, cudaStream_t s)
{
    (void)ctr;
    k_l2p_out<<<grid_for(w.n_groups), ITHREADS, 0, s>>>(w.groups, w.n_groups, t.com, t.bucket_of, t.bucket_cell,
                                                        t.off, t.L, t.accs, t.sact, t.idx, n, acc, pot,
                                                        (a.terms & 4) ? 1 : 0);
    return cudaGetLastError();
}
