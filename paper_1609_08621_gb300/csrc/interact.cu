// Interaction evaluation per sink group (Sec. 3.1, Sec. 3.3): particle-particle (PP),
// particle-cell (PC) and the group's local expansion at its particles (L2P), then the
// results are written back in the caller's order.
//
// All coordinates are single precision offsets from the group's centre of mass c_g
// (Sec. 3.1: interactions in single precision):
//   sink     u_i = fl(com_bucket(i) - c_g) + fl(x_i - com_bucket(i))
//   source   s_j = fl(com_bucket(j) - c_g) + fl(x_j - com_bucket(j))
//   cell     z_s = fl(com_s - c_g)
// where the differences of double-precision centres are formed in FP64 and rounded once
// per bucket or cell (never per interaction: FP64 issue is 1/64 of FP32 on this GPU),
// and fl(x - com_bucket) is stored per particle by the upward pass.
//
// Work items: each group's PP list is cut into chunks of `chunk` entries and its PC list into
// chunks of `chunk` cells (list_chunk, default 64); a persistent grid of warps takes items from an atomic
// counter, so a group with a very long list no longer sets the kernel's duration.  Each item
// writes one partial (ax, ay, az, phi) per sink slot; the output kernel adds a sink's
// partials in item order (deterministic), then the local expansion.
//
// One warp per item.  The warp's 32 lanes are laid out as Q list splits of 32/Q lanes,
// each lane holding R sinks (slots lane%S, +S, ...): a group of n <= R*32/Q sinks uses
// the (R, Q) of the smallest such slot count, so few lanes idle whatever the group size
// (groups hold <= g particles, typically 30-64).  Each split takes every Q-th source; the
// splits' partial sums are added with warp shuffles.
//
// PP: a_i += m_j (s_j - u_i) / (|s_j - u_i|^2 + eps^2)^(3/2), phi_i -= m_j / (...)^(1/2)
// over every particle of every PP source, the sink itself included: its force term is
// exactly zero (identical offsets) and its potential term m_i / eps is removed at the end
// by adding back the identically computed value.  Source particles are staged per warp in
// shared memory (32 list entries at a time, <= 16 particles each).
// PC: the order-4 moment record of each source cell evaluated at u_i - z_s
// (fmm_pc_acc, trace form).  Records of 32 cells are staged per warp in shared memory.
// L2P: the group's order-5 local coefficients evaluated at u_i.
#include <algorithm>

#include "expansions.cuh"
#include "fmm_internal.cuh"

#define IW 4  // warps per block
#define ITHREADS (IW * 32)
#define PP_TILE 512
#define PC_CHUNK 32

// one sink's offset from the group centre and its mass
__device__ __forceinline__ void load_sink(int s, const Com4& ck, const int* __restrict__ bucket_of,
                                          const int* __restrict__ bucket_cell, const Com4* __restrict__ com,
                                          const float4* __restrict__ off, float& ux, float& uy, float& uz, float& m)
{
    const Com4 cb = com[bucket_cell[bucket_of[s]]];
    const float4 o = off[s];
    ux = __double2float_rn(cb.x - ck.x) + o.x;
    uy = __double2float_rn(cb.y - ck.y) + o.y;
    uz = __double2float_rn(cb.z - ck.z) + o.z;
    m = o.w;
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

template <int R, int Q>
struct Sinks {
    static constexpr int S = 32 / Q;
    float ux[R], uy[R], uz[R], m[R];
    float ax[R], ay[R], az[R], ph[R];
    bool v[R];
    int split, slot;

    // sink slot i of the group is its i-th active particle act[G.first + i], i < nact
    __device__ __forceinline__ void load(const Group& G, int nact, const int* __restrict__ act, const Com4& ck,
                                         const int* __restrict__ bucket_of, const int* __restrict__ bucket_cell,
                                         const Com4* __restrict__ com, const float4* __restrict__ off, int lane)
    {
        split = lane / S;
        slot = lane % S;
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int i = slot + r * S;
            v[r] = i < nact;
            ux[r] = uy[r] = uz[r] = m[r] = 0.0f;
            ax[r] = ay[r] = az[r] = ph[r] = 0.0f;
            if (v[r]) load_sink(act[G.first + i], ck, bucket_of, bucket_cell, com, off, ux[r], uy[r], uz[r], m[r]);
        }
    }

    // add the partial sums of the Q splits (lanes l, l ^ S, l ^ 2S, ...)
    __device__ __forceinline__ void reduce()
    {
#pragma unroll
        for (int o = S; o < 32; o <<= 1)
#pragma unroll
            for (int r = 0; r < R; r++) {
                ax[r] += __shfl_xor_sync(FMM_FULL_MASK, ax[r], o);
                ay[r] += __shfl_xor_sync(FMM_FULL_MASK, ay[r], o);
                az[r] += __shfl_xor_sync(FMM_FULL_MASK, az[r], o);
                ph[r] += __shfl_xor_sync(FMM_FULL_MASK, ph[r], o);
            }
    }
};

// Source particles of 32 PP entries staged in shared memory: entry j contributes cnt_j
// particles at tile positions [excl_j, excl_j + cnt_j); each lane fills tile slots
// lane, lane + 32, ... independently (entry found by binary search over the prefix), so the
// particle loads of the whole chunk are in flight together.
struct PPChunk {
    int first[32], excl[33];
    float dx[32], dy[32], dz[32];
};

template <int R, int Q>
__device__ __forceinline__ long long pp_item(const Group& G, int nact, const int* __restrict__ act, int chunk,
                                             const Com4& ck,
                                             const unsigned int* __restrict__ pp, const int* __restrict__ cfirst,
                                             const int* __restrict__ ccount, const Com4* __restrict__ com,
                                             const int* __restrict__ bucket_of, const int* __restrict__ bucket_cell,
                                             const float4* __restrict__ off, float4* __restrict__ part, float4* T,
                                             PPChunk& E, float eps2, int lane, int csize)
{
    Sinks<R, Q> K;
    K.load(G, nact, act, ck, bucket_of, bucket_cell, com, off, lane);
    long long nsrc = 0;
    const int e0 = chunk * csize, e1 = min(e0 + csize, G.pp_len);
    {
        for (int base = e0; base < e1; base += 32) {
            const int ne = min(32, e1 - base);
            int first = 0, cnt = 0;
            float dx = 0.f, dy = 0.f, dz = 0.f;
            if (lane < ne) {
                const unsigned int e = pp[G.pp_off + base + lane];
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
                const Com4 cb = com[bc];
                dx = __double2float_rn(cb.x - ck.x);
                dy = __double2float_rn(cb.y - ck.y);
                dz = __double2float_rn(cb.z - ck.z);
            }
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FMM_FULL_MASK, incl, o);
                if (lane >= o) incl += t;
            }
            const int total = __shfl_sync(FMM_FULL_MASK, incl, 31);
            E.first[lane] = first;
            E.excl[lane] = incl - cnt;
            E.dx[lane] = dx;
            E.dy[lane] = dy;
            E.dz[lane] = dz;
            if (lane == 31) E.excl[32] = total;
            __syncwarp();
            for (int t = lane; t < total; t += 32) {
                // largest j with excl[j] <= t (entries with cnt 0 never occur)
                int lo = 0, hi = ne - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (E.excl[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                const float4 o = off[E.first[lo] + (t - E.excl[lo])];
                T[t] = make_float4(E.dx[lo] + o.x, E.dy[lo] + o.y, E.dz[lo] + o.z, o.w);
            }
            __syncwarp();
#pragma unroll 4
            for (int t = K.split; t < total; t += Q) {
                const float4 s = T[t];
#pragma unroll
                for (int r = 0; r < R; r++) pp_pair(K.ux[r], K.uy[r], K.uz[r], s, eps2, K.ax[r], K.ay[r], K.az[r], K.ph[r]);
            }
            nsrc += total;
            __syncwarp();
        }
        K.reduce();
        // remove the self term of the potential (the force term is exactly zero), once per sink
        if (chunk == 0) {
            const float ie = rsqrtf(eps2);
#pragma unroll
            for (int r = 0; r < R; r++) K.ph[r] += K.m[r] * ie;
        }
    }
    if (K.split == 0) {
#pragma unroll
        for (int r = 0; r < R; r++)
            if (K.v[r]) part[K.slot + r * K.S] = make_float4(K.ax[r], K.ay[r], K.az[r], K.ph[r]);
    }
    return nsrc;
}

// Persistent: each warp takes the next PP work item until none is left.
__global__ void __launch_bounds__(ITHREADS) k_pp(const Group* __restrict__ groups, const unsigned int* __restrict__ item_pp,
                                                 const unsigned int* __restrict__ base_pp,
                                                 const unsigned int* __restrict__ pp, const int* __restrict__ cfirst,
                                                 const int* __restrict__ ccount, const int* __restrict__ cnact,
                                                 const Com4* __restrict__ com, const int* __restrict__ bucket_of,
                                                 const int* __restrict__ bucket_cell, const float4* __restrict__ off,
                                                 float4* __restrict__ part_pp, const int* __restrict__ act,
                                                 float eps2, int csize, long long cap_items,
                                                 DevCounters* __restrict__ ctr)
{
    __shared__ float4 tile[IW][PP_TILE];
    __shared__ PPChunk chunk[IW];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    float4* T = tile[wl];
    const unsigned long long n_items =
        min((unsigned long long)*(volatile unsigned int*)&ctr->n_item_pp, (unsigned long long)cap_items);
    unsigned long long pairs = 0;
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0) i = atomicAdd(&ctr->pp_work, 1ull);
        i = __shfl_sync(FMM_FULL_MASK, i, 0);
        if (i >= n_items) break;
        const unsigned int gi = item_pp[i];
        const Group G = groups[gi];
        const int k = (int)(i - base_pp[gi]);
        const Com4 ck = com[G.cell];
        const int n = cnact[G.cell];  // active sinks of the group
        float4* part = part_pp + i * FMM_GMAX;
        long long nsrc;
#define PP_CALL(R, Q) pp_item<R, Q>(G, n, act, k, ck, pp, cfirst, ccount, com, bucket_of, bucket_cell, off, part, T, chunk[wl], eps2, lane, csize)
        if (n <= 8) nsrc = PP_CALL(1, 4);
        else if (n <= 16) nsrc = PP_CALL(1, 2);
        else if (n <= 24) nsrc = PP_CALL(3, 4);
        else if (n <= 32) nsrc = PP_CALL(1, 1);
        else if (n <= 48) nsrc = PP_CALL(3, 2);
        else nsrc = PP_CALL(2, 1);
#undef PP_CALL
        if (lane == 0) pairs += (unsigned long long)cnact[G.cell] * (unsigned long long)nsrc;
    }
    if (lane == 0 && pairs) atomicAdd(&ctr->n_pp_pairs, pairs);
}

// PC for one group with a runtime sink layout (R sinks per lane, Q list splits): the sinks
// are taken one after another against each staged chunk of cell records, so a single copy of
// the (large) particle-cell body serves every layout.
#define PC_RMAX 3
__device__ __forceinline__ void pc_item(const Group& G, int nact, const int* __restrict__ act, int chunk, int R,
                                        int Q, const Com4& ck,
                                        const unsigned int* __restrict__ pc, const Com4* __restrict__ com,
                                        const int* __restrict__ bucket_of, const int* __restrict__ bucket_cell,
                                        const float4* __restrict__ off, const float4* __restrict__ rec4,
                                        float4* __restrict__ part, float4* R4, float4* Z, int* ids, float eps2,
                                        int lane, int csize)
{
    const int S = 32 / Q, split = lane / S, slot = lane % S;
    float ux[PC_RMAX], uy[PC_RMAX], uz[PC_RMAX];
    float ax[PC_RMAX], ay[PC_RMAX], az[PC_RMAX], ph[PC_RMAX];
#pragma unroll
    for (int r = 0; r < PC_RMAX; r++) {
        ux[r] = uy[r] = uz[r] = 0.0f;
        ax[r] = ay[r] = az[r] = ph[r] = 0.0f;
        const int i = slot + r * S;
        if (r < R && i < nact) {
            float m;
            load_sink(act[G.first + i], ck, bucket_of, bucket_cell, com, off, ux[r], uy[r], uz[r], m);
        }
    }
    const int e0 = chunk * csize, e1 = min(e0 + csize, G.pc_len);
    for (int base = e0; base < e1; base += PC_CHUNK) {
        const int ne = min(PC_CHUNK, e1 - base);
        if (lane < ne) {
            const unsigned int c = pc[G.pc_off + base + lane];
            const Com4 cs = com[c];
            ids[lane] = (int)c;
            Z[lane] = make_float4(__double2float_rn(cs.x - ck.x), __double2float_rn(cs.y - ck.y),
                                  __double2float_rn(cs.z - ck.z), 0.0f);
        }
        __syncwarp();
        const int nv = ne * (FMM_NREC / 4);
        for (int i = lane; i < nv; i += 32) {
            const int cl = i / (FMM_NREC / 4), part = i - cl * (FMM_NREC / 4);
            R4[i] = rec4[(long long)ids[cl] * (FMM_NREC / 4) + part];
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < PC_RMAX; r++) {
            if (r >= R) break;
            float bx = 0.f, by = 0.f, bz = 0.f, bp = 0.f;
            const float sx = ux[r], sy = uy[r], sz = uz[r];
#pragma unroll 2
            for (int j = split; j < ne; j += Q) {
                const float4 z = Z[j];
                fmm_pc_acc(reinterpret_cast<const float*>(&R4[j * (FMM_NREC / 4)]), sx - z.x, sy - z.y, sz - z.z,
                           eps2, bx, by, bz, bp);
            }
            ax[r] += bx;
            ay[r] += by;
            az[r] += bz;
            ph[r] += bp;
        }
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < PC_RMAX; r++) {
        if (r >= R) break;
        for (int o = S; o < 32; o <<= 1) {
            ax[r] += __shfl_xor_sync(FMM_FULL_MASK, ax[r], o);
            ay[r] += __shfl_xor_sync(FMM_FULL_MASK, ay[r], o);
            az[r] += __shfl_xor_sync(FMM_FULL_MASK, az[r], o);
            ph[r] += __shfl_xor_sync(FMM_FULL_MASK, ph[r], o);
        }
        const int i = slot + r * S;
        if (split == 0 && i < nact) part[i] = make_float4(ax[r], ay[r], az[r], ph[r]);
    }
}

__global__ void __launch_bounds__(ITHREADS) k_pc(const Group* __restrict__ groups, const unsigned int* __restrict__ item_pc,
                                                 const unsigned int* __restrict__ base_pc,
                                                 const unsigned int* __restrict__ pc, const int* __restrict__ cnact,
                                                 const Com4* __restrict__ com, const int* __restrict__ bucket_of,
                                                 const int* __restrict__ bucket_cell, const float4* __restrict__ off,
                                                 const float* __restrict__ rec, float4* __restrict__ part_pc,
                                                 const int* __restrict__ act, float eps2, int csize, long long cap_items,
                                                 DevCounters* __restrict__ ctr)
{
    __shared__ float4 R4s[IW][PC_CHUNK * FMM_NREC / 4];
    __shared__ float4 Zs[IW][PC_CHUNK];
    __shared__ int idss[IW][PC_CHUNK];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const float4* rec4 = reinterpret_cast<const float4*>(rec);
    const unsigned long long n_items =
        min((unsigned long long)*(volatile unsigned int*)&ctr->n_item_pc, (unsigned long long)cap_items);
    unsigned long long pairs = 0;
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0) i = atomicAdd(&ctr->pc_work, 1ull);
        i = __shfl_sync(FMM_FULL_MASK, i, 0);
        if (i >= n_items) break;
        const unsigned int gi = item_pc[i];
        const Group G = groups[gi];
        const int k = (int)(i - base_pc[gi]);
        const Com4 ck = com[G.cell];
        const int n = cnact[G.cell];  // active sinks of the group
        int R, Q;
        if (n <= 8) { R = 1; Q = 4; }
        else if (n <= 16) { R = 1; Q = 2; }
        else if (n <= 24) { R = 3; Q = 4; }
        else if (n <= 32) { R = 1; Q = 1; }
        else if (n <= 48) { R = 3; Q = 2; }
        else { R = 2; Q = 1; }
        pc_item(G, n, act, k, R, Q, ck, pc, com, bucket_of, bucket_cell, off, rec4, part_pc + i * FMM_GMAX, R4s[wl], Zs[wl],
                idss[wl], eps2, lane, csize);
        if (lane == 0) {
            const int nc = min(csize, G.pc_len - k * csize);
            pairs += (unsigned long long)cnact[G.cell] * (unsigned long long)nc;
        }
    }
    if (lane == 0 && pairs) atomicAdd(&ctr->n_pc_pairs, pairs);
}

// Per group: each sink adds its PP partials and PC partials in item order, then the group's
// local expansion, and the result goes to the caller's order (active particles only).
// T = float: partial sums added in FP32; T = double: added in FP64 (accumulate = 1)
template <typename T>
__global__ void __launch_bounds__(ITHREADS) k_l2p_out(const Group* __restrict__ groups,
                                                      const unsigned long long* __restrict__ ngroups_dev, long long cap_groups,
                                                      long long cap_item_pp, long long cap_item_pc,
                                                      const Com4* __restrict__ com,
                                                      const int* __restrict__ bucket_of,
                                                      const int* __restrict__ bucket_cell,
                                                      const float4* __restrict__ off, const float* __restrict__ Lg,
                                                      const unsigned int* __restrict__ cnt_pp,
                                                      const unsigned int* __restrict__ base_pp,
                                                      const float4* __restrict__ part_pp,
                                                      const unsigned int* __restrict__ cnt_pc,
                                                      const unsigned int* __restrict__ base_pc,
                                                      const float4* __restrict__ part_pc,
                                                      const int* __restrict__ act, const int* __restrict__ cnact,
                                                      const unsigned int* __restrict__ perm, long long n,
                                                      float* __restrict__ acc, float* __restrict__ pot, int terms)
{
    __shared__ float Ls[IW][FMM_NL];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long n_groups = (long long)min(*ngroups_dev, (unsigned long long)cap_groups);
    for (long long gi = gw; gi < n_groups; gi += nw) {
        const Group G = groups[gi];
        const Com4 ck = com[G.cell];
        for (int i = lane; i < FMM_NL; i += 32) Ls[wl][i] = Lg[gi * FMM_NL + i];
        __syncwarp();
        // items beyond the buffers (an overflow the host then repairs) are skipped
        unsigned int npp = (terms & 1) ? cnt_pp[gi] : 0u, bpp = base_pp[gi];
        unsigned int npc = (terms & 2) ? cnt_pc[gi] : 0u, bpc = base_pc[gi];
        if ((long long)bpp + npp > cap_item_pp) npp = 0;
        if ((long long)bpc + npc > cap_item_pc) npc = 0;
        const int nact = cnact[G.cell];
        for (int i = lane; i < nact; i += 32) {
            const int s = act[G.first + i];
            T ax = 0, ay = 0, az = 0, aw = 0;
            for (unsigned int k = 0; k < npp; k++) {
                const float4 p = part_pp[(unsigned long long)(bpp + k) * FMM_GMAX + i];
                ax += p.x;
                ay += p.y;
                az += p.z;
                aw += p.w;
            }
            for (unsigned int k = 0; k < npc; k++) {
                const float4 p = part_pc[(unsigned long long)(bpc + k) * FMM_GMAX + i];
                ax += p.x;
                ay += p.y;
                az += p.z;
                aw += p.w;
            }
            if (terms & 4) {
                float ux, uy, uz, m;
                load_sink(s, ck, bucket_of, bucket_cell, com, off, ux, uy, uz, m);
                float lx = 0.f, ly = 0.f, lz = 0.f, lw = 0.f;
                fmm_l2p_acc(Ls[wl], ux, uy, uz, lx, ly, lz, lw);
                ax += lx;
                ay += ly;
                az += lz;
                aw += lw;
            }
            {
                const unsigned int p = perm[s];
                acc[p] = (float)ax;
                acc[n + p] = (float)ay;
                acc[2 * n + p] = (float)az;
                if (pot) pot[p] = (float)aw;
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

// resident blocks of a kernel on the whole GPU (persistent grids)
template <typename K>
static int persistent_blocks(K kernel)
{
    int per_sm = 1, sms = 152, device = 0;
    cudaGetDevice(&device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, ITHREADS, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return (per_sm < 1 ? 1 : per_sm) * sms;
}

// Active sinks of every group, compacted in particle order: act[G.first + i] = the group's i-th
// active particle (with no inactive particles, the identity).  One warp per group.
__global__ void k_group_active(const Group* __restrict__ groups, const unsigned long long* __restrict__ ngroups_dev,
                               long long cap_groups, const unsigned char* __restrict__ sact, int* __restrict__ act)
{
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long ng = (long long)min(*ngroups_dev, (unsigned long long)cap_groups);
    const unsigned int lt = fmm_lanemask_lt();
    for (long long gi = gw; gi < ng; gi += nw) {
        const Group G = groups[gi];
        int done = 0;
        for (int b = 0; b < G.count; b += 32) {
            const int i = b + lane;
            const bool a = i < G.count && sact[G.first + i] != 0;
            const unsigned int m = __ballot_sync(FMM_FULL_MASK, a);
            if (a) act[G.first + done + __popc(m & lt)] = G.first + i;
            done += __popc(m);
        }
    }
}

// Work items: per group ceil(pp_len / chunk) PP items and ceil(pc_len / chunk) PC items; exclusive scans give each group's first item, and every item learns its group.
__global__ void k_item_counts(const Group* __restrict__ groups, long long grid, const unsigned long long* __restrict__ ng,
                              unsigned int* __restrict__ cnt_pp, unsigned int* __restrict__ cnt_pc, int csize)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= grid) return;
    if (i >= (long long)*ng) {  // slots past the group count (capacity-sized launches) add nothing
        cnt_pp[i] = 0u;
        cnt_pc[i] = 0u;
        return;
    }
    const Group G = groups[i];
    cnt_pp[i] = (unsigned int)fmm_ceil_div(G.pp_len, csize);
    cnt_pc[i] = (unsigned int)fmm_ceil_div(G.pc_len, csize);
}

__global__ void k_item_expand(long long grid, const unsigned int* __restrict__ cnt_pp,
                              const unsigned int* __restrict__ base_pp, const unsigned int* __restrict__ cnt_pc,
                              const unsigned int* __restrict__ base_pc, unsigned int* __restrict__ item_pp,
                              unsigned int* __restrict__ item_pc, long long cap_pp, long long cap_pc,
                              unsigned int* __restrict__ overflow)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= grid) return;
    const long long bp = base_pp[i], np = cnt_pp[i], bc = base_pc[i], nc = cnt_pc[i];
    if (bp + np > cap_pp || bc + nc > cap_pc) {
        atomicOr(overflow, 1u);
        return;
    }
    for (long long k = 0; k < np; k++) item_pp[bp + k] = (unsigned int)i;
    for (long long k = 0; k < nc; k++) item_pc[bc + k] = (unsigned int)i;
}

cudaError_t fmm_launch_items(DevTree& t, DevWalk& w, DevCounters* ctr, int chunk, cudaStream_t s)
{
    // under graph capture the group count is known only on the device: cover the capacity
    const long long ng = t.cap_grid ? w.cap_groups : w.n_groups;
    const unsigned blocks = (unsigned)fmm_ceil_div(ng, 256);
    k_item_counts<<<blocks, 256, 0, s>>>(w.groups, ng, &ctr->n_groups, w.cnt_pp, w.cnt_pc, chunk);
    cudaError_t e = fmm_scan_exclusive(w.cnt_pp, w.base_pp, ng, &ctr->n_item_pp, t, s);
    if (e == cudaSuccess) e = fmm_scan_exclusive(w.cnt_pc, w.base_pc, ng, &ctr->n_item_pc, t, s);
    if (e != cudaSuccess) return e;
    k_item_expand<<<blocks, 256, 0, s>>>(ng, w.cnt_pp, w.base_pp, w.cnt_pc, w.base_pc, w.item_pp, w.item_pc,
                                         w.cap_item_pp, w.cap_item_pc, &ctr->overflow);
    k_group_active<<<(unsigned)std::max(1LL, std::min(fmm_ceil_div(ng, ITHREADS / 32), 152LL * 16)), ITHREADS, 0, s>>>(
        w.groups, &ctr->n_groups, w.cap_groups, t.sact, t.act);
    return cudaGetLastError();
}

cudaError_t fmm_launch_pp(DevTree& t, DevWalk& w, DevCounters* ctr, const InteractArgs& a, cudaStream_t s)
{
    if (!(a.terms & 1)) return cudaSuccess;
    static int blocks = 0;
    if (!blocks) blocks = persistent_blocks(k_pp);
    cudaMemsetAsync(&ctr->pp_work, 0, sizeof(unsigned long long), s);
    k_pp<<<blocks, ITHREADS, 0, s>>>(w.groups, w.item_pp, w.base_pp, w.pp, t.cfirst, t.ccount, t.cnact, t.com,
                                     t.bucket_of, t.bucket_cell, t.off, w.part_pp, t.act, a.eps2, a.chunk, w.cap_item_pp, ctr);
    return cudaGetLastError();
}

cudaError_t fmm_launch_pc(DevTree& t, DevWalk& w, DevCounters* ctr, const InteractArgs& a, cudaStream_t s)
{
    if (!(a.terms & 2)) return cudaSuccess;
    static int blocks = 0;
    if (!blocks) blocks = persistent_blocks(k_pc);
    cudaMemsetAsync(&ctr->pc_work, 0, sizeof(unsigned long long), s);
    k_pc<<<blocks, ITHREADS, 0, s>>>(w.groups, w.item_pc, w.base_pc, w.pc, t.cnact, t.com, t.bucket_of,
                                     t.bucket_cell, t.off, t.rec, w.part_pc, t.act, a.eps2, a.chunk, w.cap_item_pc, ctr);
    return cudaGetLastError();
}

cudaError_t fmm_launch_l2p_out(DevTree& t, DevWalk& w, DevCounters* ctr, const InteractArgs& a, float* acc,
                               float* pot, long long n, cudaStream_t s)
{
    const long long ng = t.cap_grid ? w.cap_groups : w.n_groups;
    if (a.accumulate == 1)
        k_l2p_out<double><<<grid_for(ng), ITHREADS, 0, s>>>(
            w.groups, &ctr->n_groups, w.cap_groups, w.cap_item_pp, w.cap_item_pc, t.com, t.bucket_of, t.bucket_cell,
            t.off, w.Lg, w.cnt_pp, w.base_pp, w.part_pp, w.cnt_pc, w.base_pc, w.part_pc, t.act, t.cnact, t.idx, n, acc, pot,
            a.terms);
    else
        k_l2p_out<float><<<grid_for(ng), ITHREADS, 0, s>>>(
            w.groups, &ctr->n_groups, w.cap_groups, w.cap_item_pp, w.cap_item_pc, t.com, t.bucket_of, t.bucket_cell,
            t.off, w.Lg, w.cnt_pp, w.base_pp, w.part_pp, w.cnt_pc, w.base_pc, w.part_pc, t.act, t.cnact, t.idx, n, acc, pot,
            a.terms);
    return cudaGetLastError();
}
