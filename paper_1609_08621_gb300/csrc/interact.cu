// Interaction evaluation per sink group (Sec. 3.1, Sec. 3.3): particle-particle (PP),
// particle-cell (PC) and the group's local expansion at its particles (L2P), then the
// results are written back in the caller's order.
//
// All coordinates are single precision offsets from the group's centre of mass c_g
// (Sec. 3.1: interactions in single precision):
//   sink     u_i = d(com_bucket(i), c_g) + fl(x_i - com_bucket(i))
//   source   s_j = d(com_bucket(j), c_g) + fl(x_j - com_bucket(j))
//   cell     z_s = d(com_s, c_g)
// where d(a, b) is the single-precision difference of two double-precision centres, taken from
// their float pairs (hi, lo) by cen_diff within about one unit in the last place of fl(a - b),
// without FP64 instructions (FP64 issues at 1/64 of the FP32 rate on this GPU), once per bucket
// or cell; fl(x - com_bucket) is stored per particle by the upward pass.
//
// Work items: each group's PP list is cut into chunks of `chunk` entries and its PC list into
// chunks of `chunk` cells (list_chunk, default 64); a persistent grid of warps takes items from an atomic
// counter, so a group with a very long list no longer sets the kernel's duration.  Each item
// writes one partial (ax, ay, az, phi) per sink slot; the output kernel adds a sink's
// partials in item order (deterministic), then the local expansion.
//
// One warp per item.  The warp's 32 lanes are laid out as Q list splits of S = 32/Q lanes,
// each lane holding R sinks (slots lane%S, +S, ...); each split takes every Q-th source and the
// splits' partial sums are added with warp shuffles.  Groups hold <= g particles (typically
// 30-64), and a layout with more slots than active sinks idles lanes, so the slot count follows
// the active count closely: PP uses one or two compile-time layouts in steps of 8 slots up to 48
// (e.g. 32 + 8 for 40 sinks), PC a runtime sequence of passes of 64, 32, 16 or 8 slots (at most 7
// idle).  In both, each lane holds its sinks in pairs that share FP32x2 instructions.
//
// PP: a_i += m_j (s_j - u_i) / (|s_j - u_i|^2 + eps^2)^(3/2), phi_i -= m_j / (...)^(1/2)
// over every particle of every PP source, the sink itself included: its force term is
// exactly zero (identical offsets) and its potential term m_i / eps is removed at the end
// by adding back the identically computed value.  Source particles are staged per warp in
// shared memory (32 list entries at a time, <= 16 particles each).
// PC: the order-4 moment record of each source cell evaluated at u_i - z_s
// (fmm_pc_acc2: the trace form of fmm_pc_acc for two sinks).  Records of 32 cells are staged
// per warp in shared memory.
// L2P: the group's order-5 local coefficients evaluated at u_i.
#include <algorithm>
#include <atomic>

#include "expansions.cuh"
#include "f64bits.cuh"
#include "fmm_internal.cuh"

#define IW 4  // warps per block
#define ITHREADS (IW * 32)
#define PP_TILE 512
#define PC_CHUNK 32

// one sink's offset from the group centre and its mass
__device__ __forceinline__ void load_sink(int s, const float4& hk, const float4& lk, const int* __restrict__ bucket_of,
                                          const int* __restrict__ bucket_cell, const float4* __restrict__ cen,
                                          const float4* __restrict__ off, float& ux, float& uy, float& uz, float& m)
{
    const int bc = bucket_cell[bucket_of[s]];
    const float4 hb = cen[2 * bc], lb = cen[2 * bc + 1];
    const float4 o = off[s];
    ux = __fadd_rn(cen_diff(hb.x, lb.x, hk.x, lk.x), o.x);
    uy = __fadd_rn(cen_diff(hb.y, lb.y, hk.y, lk.y), o.y);
    uz = __fadd_rn(cen_diff(hb.z, lb.z, hk.z, lk.z), o.z);
    m = o.w;
}

__device__ __forceinline__ void pp_pair(float ux, float uy, float uz, float4 s, float eps2, float& ax, float& ay,
                                        float& az, float& ph)
{
    const float dx = s.x - ux, dy = s.y - uy, dz = s.z - uz;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    const float ir = fmm_rsqrt(r2);
    const float mir = s.w * ir;
    const float mir3 = mir * ir * ir;
    ax = fmaf(mir3, dx, ax);
    ay = fmaf(mir3, dy, ay);
    az = fmaf(mir3, dz, az);
    ph -= mir;
}

// Two (sink, source) pairs in one set of FP32x2 instructions: the same operations, in the same
// order and rounding, as pp_pair for each component (fmaf / fadd / fmul round to nearest per
// component), so the sums are bit-identical, but half the FP32 instructions are issued.  The
// sink offsets come negated (s - u = s + (-u) exactly) and the potential is summed positively and
// negated at the end (rounding to nearest is symmetric), so no negation is issued per pair.
__device__ __forceinline__ void pp_pair2(float2 nux, float2 nuy, float2 nuz, float4 s, float2 eps2, float2& ax,
                                         float2& ay, float2& az, float2& pw)
{
    const float2 dx = __fadd2_rn(make_float2(s.x, s.x), nux);
    const float2 dy = __fadd2_rn(make_float2(s.y, s.y), nuy);
    const float2 dz = __fadd2_rn(make_float2(s.z, s.z), nuz);
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps2)));
    const float2 ir = make_float2(fmm_rsqrt(r2.x), fmm_rsqrt(r2.y));
    const float2 mir = __fmul2_rn(make_float2(s.w, s.w), ir);
    const float2 mir3 = __fmul2_rn(__fmul2_rn(mir, ir), ir);
    ax = __ffma2_rn(mir3, dx, ax);
    ay = __ffma2_rn(mir3, dy, ay);
    az = __ffma2_rn(mir3, dz, az);
    pw = __fadd2_rn(pw, mir);
}

// R (even) sinks per lane as R/2 pairs: slots base + slot + r*S, pair p holding r = 2p and 2p+1.
template <int R, int Q>
struct Sinks {
    static_assert(R % 2 == 0, "sinks are taken in pairs");
    static constexpr int S = 32 / Q, P = R / 2;
    float2 nux[P], nuy[P], nuz[P];
    float2 ax[P], ay[P], az[P], pw[P];
    int split, slot;

    // sink slot base + slot + r*S of the group is its active particle act[G.first + i], i < nact
    __device__ __forceinline__ void load(const Group& G, int nact, int base, const int* __restrict__ act,
                                         const float4& hk, const float4& lk, const int* __restrict__ bucket_of,
                                         const int* __restrict__ bucket_cell, const float4* __restrict__ cen,
                                         const float4* __restrict__ off, int lane)
    {
        split = lane / S;
        slot = lane % S;
#pragma unroll
        for (int p = 0; p < P; p++) {
            float ux0 = 0.f, uy0 = 0.f, uz0 = 0.f, ux1 = 0.f, uy1 = 0.f, uz1 = 0.f, m;
            const int i0 = base + slot + 2 * p * S, i1 = i0 + S;
            if (i0 < nact) load_sink(act[G.first + i0], hk, lk, bucket_of, bucket_cell, cen, off, ux0, uy0, uz0, m);
            if (i1 < nact) load_sink(act[G.first + i1], hk, lk, bucket_of, bucket_cell, cen, off, ux1, uy1, uz1, m);
            nux[p] = make_float2(-ux0, -ux1);
            nuy[p] = make_float2(-uy0, -uy1);
            nuz[p] = make_float2(-uz0, -uz1);
            ax[p] = ay[p] = az[p] = pw[p] = make_float2(0.f, 0.f);
        }
    }

    // every Q-th staged source from this lane's split, against the lane's R sinks
    __device__ __forceinline__ void sweep(const float4* T, int total, float eps2)
    {
        const float2 e2 = make_float2(eps2, eps2);
#pragma unroll 4
        for (int t = split; t < total; t += Q) {
            const float4 s = T[t];
#pragma unroll
            for (int p = 0; p < P; p++) pp_pair2(nux[p], nuy[p], nuz[p], s, e2, ax[p], ay[p], az[p], pw[p]);
        }
    }

    // add the partial sums of the Q splits (lanes l, l ^ S, l ^ 2S, ...)
    __device__ __forceinline__ void reduce()
    {
#pragma unroll
        for (int o = S; o < 32; o <<= 1)
#pragma unroll
            for (int p = 0; p < P; p++) {
                ax[p].x += __shfl_xor_sync(FMM_FULL_MASK, ax[p].x, o);
                ax[p].y += __shfl_xor_sync(FMM_FULL_MASK, ax[p].y, o);
                ay[p].x += __shfl_xor_sync(FMM_FULL_MASK, ay[p].x, o);
                ay[p].y += __shfl_xor_sync(FMM_FULL_MASK, ay[p].y, o);
                az[p].x += __shfl_xor_sync(FMM_FULL_MASK, az[p].x, o);
                az[p].y += __shfl_xor_sync(FMM_FULL_MASK, az[p].y, o);
                pw[p].x += __shfl_xor_sync(FMM_FULL_MASK, pw[p].x, o);
                pw[p].y += __shfl_xor_sync(FMM_FULL_MASK, pw[p].y, o);
            }
    }

    // split 0 writes the sums; with self_term the sink's own potential term m_i / eps, which the
    // sweep included through the identical pair computation, is added back first
    __device__ __forceinline__ void store(const Group& G, int nact, int base, const int* __restrict__ act,
                                          const float4* __restrict__ off, float4* __restrict__ part, bool self_term,
                                          float eps2)
    {
        if (split != 0) return;
        const float ie = fmm_rsqrt(eps2);
#pragma unroll
        for (int p = 0; p < P; p++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int i = base + slot + (2 * p + h) * S;
                if (i < nact) {
                    float ph = -(h ? pw[p].y : pw[p].x);
                    if (self_term) ph += off[act[G.first + i]].w * ie;
                    part[i] = make_float4(h ? ax[p].y : ax[p].x, h ? ay[p].y : ay[p].x, h ? az[p].y : az[p].x, ph);
                }
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

// One PP work item with the sink layout (R1, Q1) for slots [0, R1*32/Q1) and, when R2 > 0, a
// second layout (R2, Q2) for the slots from there on, both swept over each staged tile: a group of
// 24 or 40 sinks takes 16 + 8 or 32 + 8 slots instead of 32 or 48.
template <int R1, int Q1, int R2, int Q2>
__device__ __forceinline__ long long pp_item(const Group& G, int nact, const int* __restrict__ act, int chunk,
                                             const float4& hk, const float4& lk,
                                             const unsigned int* __restrict__ pp, const int* __restrict__ cfirst,
                                             const int* __restrict__ ccount, const float4* __restrict__ cen,
                                             const int* __restrict__ bucket_of, const int* __restrict__ bucket_cell,
                                             const float4* __restrict__ off, float4* __restrict__ part, float4* T,
                                             PPChunk& E, float eps2, int lane, int csize, int ib, int R)
{
    constexpr int B2 = R1 * (32 / Q1);
    Sinks<R1, Q1> K;
    Sinks<(R2 > 0 ? R2 : 2), (R2 > 0 ? Q2 : 1)> K2;
    K.load(G, nact, 0, act, hk, lk, bucket_of, bucket_cell, cen, off, lane);
    if (R2 > 0) K2.load(G, nact, B2, act, hk, lk, bucket_of, bucket_cell, cen, off, lane);
    long long nsrc = 0;
    const int e0 = chunk * csize, e1 = min(e0 + csize, G.pp_len);
    for (int base = e0; base < e1; base += 32) {
        const int ne = min(32, e1 - base);
        int first = 0, cnt = 0;
        float dx = 0.f, dy = 0.f, dz = 0.f;
        if (lane < ne) {
            const unsigned int e = pp[G.pp_off + base + lane];
            const unsigned int j = entry_index(e, ib);
            int bc;
            if (e & FMM_PARTICLE_BIT) {
                first = (int)j;
                cnt = 1;
                bc = bucket_cell[bucket_of[first]];
            } else {
                first = cfirst[j];
                cnt = ccount[j];
                bc = (int)j;
            }
            float4 hb = cen[2 * bc], lb = cen[2 * bc + 1];
            const unsigned int q = entry_copy(e, ib);
            if (q != copy_centre(R)) {  // a source in a periodic copy: its bucket's centre shifted
                int nx, ny, nz;
                copy_shift(q, R, nx, ny, nz);
                cen_shift(hb.x, lb.x, (float)nx);
                cen_shift(hb.y, lb.y, (float)ny);
                cen_shift(hb.z, lb.z, (float)nz);
            }
            dx = cen_diff(hb.x, lb.x, hk.x, lk.x);
            dy = cen_diff(hb.y, lb.y, hk.y, lk.y);
            dz = cen_diff(hb.z, lb.z, hk.z, lk.z);
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
        K.sweep(T, total, eps2);
        if (R2 > 0) K2.sweep(T, total, eps2);
        nsrc += total;
        __syncwarp();
    }
    // the self term of the potential is removed once per sink, by the group's first item
    K.reduce();
    K.store(G, nact, 0, act, off, part, chunk == 0, eps2);
    if (R2 > 0) {
        K2.reduce();
        K2.store(G, nact, B2, act, off, part, chunk == 0, eps2);
    }
    return nsrc;
}

// Persistent: each warp takes the next PP work item until none is left.
__global__ void __launch_bounds__(ITHREADS) k_pp(const Group* __restrict__ groups, const unsigned int* __restrict__ item_pp,
                                                 const unsigned int* __restrict__ base_pp,
                                                 const unsigned int* __restrict__ pp, const int* __restrict__ cfirst,
                                                 const int* __restrict__ ccount, const int* __restrict__ cnact,
                                                 const float4* __restrict__ cen, const int* __restrict__ bucket_of,
                                                 const int* __restrict__ bucket_cell, const float4* __restrict__ off,
                                                 float4* __restrict__ part_pp, const int* __restrict__ act,
                                                 float eps2, int csize, long long cap_items, int ib, int R,
                                                 DevCounters* __restrict__ ctr)
{
    __shared__ float4 tile[IW][PP_TILE];
    __shared__ PPChunk chunk[IW];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    float4* T = tile[wl];
    if (fmm_overflowed(ctr)) return;
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
        const float4 hk = cen[2 * G.cell], lk = cen[2 * G.cell + 1];
        const int n = cnact[G.cell];  // active sinks of the group
        float4* part = part_pp + i * FMM_GMAX;
        long long nsrc;
#define PP_CALL(R1, Q1, R2, Q2) \
    pp_item<R1, Q1, R2, Q2>(G, n, act, k, hk, lk, pp, cfirst, ccount, cen, bucket_of, bucket_cell, off, part, T, chunk[wl], eps2, lane, csize, ib, R)
        // sink slots in steps of 8 up to 48 sinks, in pairs per lane
        if (n <= 8) nsrc = PP_CALL(2, 8, 0, 0);
        else if (n <= 16) nsrc = PP_CALL(2, 4, 0, 0);
        else if (n <= 24) nsrc = PP_CALL(2, 4, 2, 8);
        else if (n <= 32) nsrc = PP_CALL(2, 2, 0, 0);
        else if (n <= 40) nsrc = PP_CALL(2, 2, 2, 8);
        else if (n <= 48) nsrc = PP_CALL(2, 2, 2, 4);
        else nsrc = PP_CALL(4, 2, 0, 0);
#undef PP_CALL
        if (lane == 0) pairs += (unsigned long long)cnact[G.cell] * (unsigned long long)nsrc;
    }
    if (lane == 0 && pairs) atomicAdd(&ctr->n_pp_pairs, pairs);
}

// PC sink passes: the group's active sinks [0, n) are covered by passes of 64, 32, 16 or 8 slots;
// in a pass of 2S slots (S = 32, 16, 8, 4 lanes per split) lane l holds the sink pair base + l % S
// and base + l % S + S, evaluated together in FP32x2 lanes, and takes every Q-th staged cell
// (Q = 32 / S, split l / S).  The remainder r after full passes of 64 goes to passes of 32
// (r > 24), 16 (r > 8) or 8, so a group idles at most 7 slots.
#define PC_PMAX 3  // passes for n <= 64: 32 + 16 + 8 at most
__device__ __forceinline__ int pc_pass_slots(int rem)
{
    return rem > 56 ? 64 : rem > 24 ? 32 : rem > 8 ? 16 : 8;
}

// PC for one work item: each pass sweeps every staged chunk of cell records.  The sinks' offsets
// (U, by slot) and each lane's running sums per pass (A: two float4 per lane and pass) stay in
// shared memory between chunks, so one copy of the particle-cell body serves every pass.  Cell
// centres are staged negated and duplicated ({-z, -z} per axis) for the FP32x2 differences.
__device__ __forceinline__ void pc_item(const Group& G, int nact, const int* __restrict__ act, int chunk,
                                        const float4& hk, const float4& lk,
                                        const unsigned int* __restrict__ pc, const float4* __restrict__ cen,
                                        const int* __restrict__ bucket_of, const int* __restrict__ bucket_cell,
                                        const float4* __restrict__ off, const float4* __restrict__ rec4,
                                        float4* __restrict__ part, float4* R4, float4* Zxy, float2* Zz, int* ids,
                                        float4* U, float4* A, float eps2, int lane, int csize, int ib, int R)
{
    for (int i = lane; i < FMM_GMAX; i += 32) {
        float ux = 0.f, uy = 0.f, uz = 0.f, m;
        if (i < nact) load_sink(act[G.first + i], hk, lk, bucket_of, bucket_cell, cen, off, ux, uy, uz, m);
        U[i] = make_float4(ux, uy, uz, 0.0f);
    }
    int npass = 0;
    for (int base = 0; base < nact; npass++) {
        A[(npass * 32 + lane) * 2] = make_float4(0.f, 0.f, 0.f, 0.f);
        A[(npass * 32 + lane) * 2 + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        base += pc_pass_slots(nact - base);
    }
    __syncwarp();
    const float2 e2 = make_float2(eps2, eps2);
    const int e0 = chunk * csize, e1 = min(e0 + csize, G.pc_len);
    for (int cbase = e0; cbase < e1; cbase += PC_CHUNK) {
        const int ne = min(PC_CHUNK, e1 - cbase);
        if (lane < ne) {
            const unsigned int e = pc[G.pc_off + cbase + lane];
            const unsigned int c = entry_index(e, ib);
            float4 hs = cen[2 * c], ls = cen[2 * c + 1];
            const unsigned int q = entry_copy(e, ib);
            if (q != copy_centre(R)) {  // a cell in a periodic copy: its centre shifted
                int nx, ny, nz;
                copy_shift(q, R, nx, ny, nz);
                cen_shift(hs.x, ls.x, (float)nx);
                cen_shift(hs.y, ls.y, (float)ny);
                cen_shift(hs.z, ls.z, (float)nz);
            }
            ids[lane] = (int)c;
            const float zx = cen_diff(hs.x, ls.x, hk.x, lk.x), zy = cen_diff(hs.y, ls.y, hk.y, lk.y),
                        zz = cen_diff(hs.z, ls.z, hk.z, lk.z);
            Zxy[lane] = make_float4(-zx, -zx, -zy, -zy);
            Zz[lane] = make_float2(-zz, -zz);
        }
        __syncwarp();
        const int nv = ne * (FMM_NREC / 4);
        for (int v = lane; v < nv; v += 32) {
            const int cl = v / (FMM_NREC / 4), q = v - cl * (FMM_NREC / 4);
            R4[v] = rec4[(long long)ids[cl] * (FMM_NREC / 4) + q];
        }
        __syncwarp();
        for (int p = 0, base = 0; p < npass; p++) {
            const int P2 = pc_pass_slots(nact - base), S = P2 / 2, Q = 32 / S, split = lane / S;
            const float4 u0 = U[base + lane % S], u1 = U[base + lane % S + S];
            const float2 ux = make_float2(u0.x, u1.x), uy = make_float2(u0.y, u1.y), uz = make_float2(u0.z, u1.z);
            float2 bx = make_float2(0.f, 0.f), by = bx, bz = bx, bp = bx;
#pragma unroll 2
            for (int j = split; j < ne; j += Q) {
                const float4 zxy = Zxy[j];
                const float2 zz = Zz[j];
                fmm_pc_acc2(reinterpret_cast<const float*>(&R4[j * (FMM_NREC / 4)]),
                            __fadd2_rn(ux, make_float2(zxy.x, zxy.y)), __fadd2_rn(uy, make_float2(zxy.z, zxy.w)),
                            __fadd2_rn(uz, zz), e2, bx, by, bz, bp);
            }
            float4 a0 = A[(p * 32 + lane) * 2], a1 = A[(p * 32 + lane) * 2 + 1];
            a0.x += bx.x;
            a0.y += bx.y;
            a0.z += by.x;
            a0.w += by.y;
            a1.x += bz.x;
            a1.y += bz.y;
            a1.z += bp.x;
            a1.w += bp.y;
            A[(p * 32 + lane) * 2] = a0;
            A[(p * 32 + lane) * 2 + 1] = a1;
            base += P2;
        }
        __syncwarp();
    }
    // add each pass's Q split sums (lanes l, l ^ S, l ^ 2S, ...) and write the sinks' partials
    for (int p = 0, base = 0; p < npass; p++) {
        const int P2 = pc_pass_slots(nact - base), S = P2 / 2;
        float4 a0 = A[(p * 32 + lane) * 2], a1 = A[(p * 32 + lane) * 2 + 1];
        for (int o = S; o < 32; o <<= 1) {
            a0.x += __shfl_xor_sync(FMM_FULL_MASK, a0.x, o);
            a0.y += __shfl_xor_sync(FMM_FULL_MASK, a0.y, o);
            a0.z += __shfl_xor_sync(FMM_FULL_MASK, a0.z, o);
            a0.w += __shfl_xor_sync(FMM_FULL_MASK, a0.w, o);
            a1.x += __shfl_xor_sync(FMM_FULL_MASK, a1.x, o);
            a1.y += __shfl_xor_sync(FMM_FULL_MASK, a1.y, o);
            a1.z += __shfl_xor_sync(FMM_FULL_MASK, a1.z, o);
            a1.w += __shfl_xor_sync(FMM_FULL_MASK, a1.w, o);
        }
        const int i0 = base + lane % S, i1 = i0 + S;
        if (lane < S && i0 < nact) part[i0] = make_float4(a0.x, a0.z, a1.x, -a1.z);
        if (lane < S && i1 < nact) part[i1] = make_float4(a0.y, a0.w, a1.y, -a1.w);
        base += P2;
    }
    __syncwarp();
}

// Persistent: each warp takes the next PC work item until none is left.
// at least 4 blocks per SM: up to 128 registers for the paired particle-cell body
__global__ void __launch_bounds__(ITHREADS, 4) k_pc(const Group* __restrict__ groups, const unsigned int* __restrict__ item_pc,
                                                 const unsigned int* __restrict__ base_pc,
                                                 const unsigned int* __restrict__ pc, const int* __restrict__ cnact,
                                                 const float4* __restrict__ cen, const int* __restrict__ bucket_of,
                                                 const int* __restrict__ bucket_cell, const float4* __restrict__ off,
                                                 const float* __restrict__ rec, float4* __restrict__ part_pc,
                                                 const int* __restrict__ act, float eps2, int csize, long long cap_items,
                                                 int ib, int R, DevCounters* __restrict__ ctr)
{
    __shared__ float4 R4s[IW][PC_CHUNK * FMM_NREC / 4];
    __shared__ float4 Zs[IW][PC_CHUNK];
    __shared__ float2 Zzs[IW][PC_CHUNK];
    __shared__ int idss[IW][PC_CHUNK];
    __shared__ float4 Us[IW][FMM_GMAX], As[IW][PC_PMAX * 32 * 2];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const float4* rec4 = reinterpret_cast<const float4*>(rec);
    if (fmm_overflowed(ctr)) return;
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
        const float4 hk = cen[2 * G.cell], lk = cen[2 * G.cell + 1];
        const int n = cnact[G.cell];  // active sinks of the group
        pc_item(G, n, act, k, hk, lk, pc, cen, bucket_of, bucket_cell, off, rec4, part_pc + i * FMM_GMAX, R4s[wl], Zs[wl],
                Zzs[wl], idss[wl], Us[wl], As[wl], eps2, lane, csize, ib, R);
        if (lane == 0) {
            const int nc = min(csize, G.pc_len - k * csize);
            pairs += (unsigned long long)cnact[G.cell] * (unsigned long long)nc;
        }
    }
    if (lane == 0 && pairs) atomicAdd(&ctr->n_pc_pairs, pairs);
}

// The partial sums as the accumulator type: FP64 values are formed from the FP32 encodings and
// rounded back the same way (f64bits.cuh), so the FP64 pipe, at 1/64 of the FP32 rate on this GPU,
// runs only the additions.
__device__ __forceinline__ float acc_widen(float x, float) { return x; }
__device__ __forceinline__ double acc_widen(float x, double) { return fmm_f2d(x); }
__device__ __forceinline__ float acc_round(float x) { return x; }
__device__ __forceinline__ float acc_round(double x) { return fmm_d2f_rn(x); }

// nk partials of slot i from item b on, added in item order; the loads of four items are issued
// before their additions
template <typename T>
__device__ __forceinline__ void sum_partials(const float4* __restrict__ part, unsigned int b, unsigned int nk, int i,
                                             T& ax, T& ay, T& az, T& aw)
{
    unsigned int k = 0;
    for (; k + 4 <= nk; k += 4) {
        float4 p[4];
#pragma unroll
        for (int u = 0; u < 4; u++) p[u] = part[(unsigned long long)(b + k + u) * FMM_GMAX + i];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            ax += acc_widen(p[u].x, ax);
            ay += acc_widen(p[u].y, ay);
            az += acc_widen(p[u].z, az);
            aw += acc_widen(p[u].w, aw);
        }
    }
    for (; k < nk; k++) {
        const float4 p = part[(unsigned long long)(b + k) * FMM_GMAX + i];
        ax += acc_widen(p.x, ax);
        ay += acc_widen(p.y, ay);
        az += acc_widen(p.z, az);
        aw += acc_widen(p.w, aw);
    }
}

// Per group: each sink adds its PP partials and PC partials in item order, then the group's
// local expansion, and the result goes to the caller's order (active particles only).
// T = float: partial sums added in FP32; T = double: added in FP64 (accumulate = 1)
template <typename T>
__global__ void __launch_bounds__(ITHREADS) k_l2p_out(const Group* __restrict__ groups,
                                                      const unsigned long long* __restrict__ ngroups_dev, long long cap_groups,
                                                      long long cap_item_pp, long long cap_item_pc,
                                                      const float4* __restrict__ cen,
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
                                                      float* __restrict__ acc, float* __restrict__ pot, int terms,
                                                      const DevCounters* __restrict__ ctr)
{
    __shared__ float Ls[IW][FMM_NL];
    if (fmm_overflowed(ctr)) return;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long n_groups = (long long)min(*ngroups_dev, (unsigned long long)cap_groups);
    for (long long gi = gw; gi < n_groups; gi += nw) {
        const Group G = groups[gi];
        const float4 hk = cen[2 * G.cell], lk = cen[2 * G.cell + 1];
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
            // the sink's geometry and output slot first, so their loads overlap the partials'
            const unsigned int po = perm[s];
            float ux = 0.f, uy = 0.f, uz = 0.f, m;
            if (terms & 4) load_sink(s, hk, lk, bucket_of, bucket_cell, cen, off, ux, uy, uz, m);
            T ax = 0, ay = 0, az = 0, aw = 0;
            // partials in item order, four loads in flight at a time
            sum_partials(part_pp, bpp, npp, i, ax, ay, az, aw);
            sum_partials(part_pc, bpc, npc, i, ax, ay, az, aw);
            if (terms & 4) {
                float lx = 0.f, ly = 0.f, lz = 0.f, lw = 0.f;
                fmm_l2p_acc(Ls[wl], ux, uy, uz, lx, ly, lz, lw);
                ax += acc_widen(lx, ax);
                ay += acc_widen(ly, ay);
                az += acc_widen(lz, az);
                aw += acc_widen(lw, aw);
            }
            acc[po] = acc_round(ax);
            acc[n + po] = acc_round(ay);
            acc[2 * n + po] = acc_round(az);
            if (pot) pot[po] = acc_round(aw);
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

// resident blocks of a kernel on the current device (persistent grids), looked up once per device
// and kernel: a table of atomics, 0 until the first launch on that device
template <typename K>
static int persistent_blocks(K kernel, std::atomic<int>* table)
{
    int device = 0;
    cudaGetDevice(&device);
    const bool cached = device >= 0 && device < 64;
    if (cached) {
        const int b = table[device].load(std::memory_order_relaxed);
        if (b > 0) return b;
    }
    int per_sm = 1, sms = 152;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, ITHREADS, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int b = (per_sm < 1 ? 1 : per_sm) * sms;
    if (cached) table[device].store(b, std::memory_order_relaxed);
    return b;
}
static std::atomic<int> g_pp_blocks[64], g_pc_blocks[64];

// Active sinks of every group, compacted in particle order: act[G.first + i] = the group's i-th
// active particle (with no inactive particles, the identity).  One warp per group.
__global__ void k_group_active(const Group* __restrict__ groups, const unsigned long long* __restrict__ ngroups_dev,
                               long long cap_groups, const unsigned char* __restrict__ sact, int* __restrict__ act,
                               const DevCounters* __restrict__ ctr)
{
    if (fmm_overflowed(ctr)) return;
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
                              unsigned int* __restrict__ cnt_pp, unsigned int* __restrict__ cnt_pc, int csize,
                              const DevCounters* __restrict__ ctr)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= grid) return;
    // slots past the group count (capacity-sized launches) add nothing, nor does a walk that overflowed
    if (i >= (long long)*ng || fmm_overflowed(ctr)) {
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
    k_item_counts<<<blocks, 256, 0, s>>>(w.groups, ng, &ctr->n_groups, w.cnt_pp, w.cnt_pc, chunk, ctr);
    cudaError_t e = fmm_scan_exclusive(w.cnt_pp, w.base_pp, ng, &ctr->n_item_pp, t, s);
    if (e == cudaSuccess) e = fmm_scan_exclusive(w.cnt_pc, w.base_pc, ng, &ctr->n_item_pc, t, s);
    if (e != cudaSuccess) return e;
    k_item_expand<<<blocks, 256, 0, s>>>(ng, w.cnt_pp, w.base_pp, w.cnt_pc, w.base_pc, w.item_pp, w.item_pc,
                                         w.cap_item_pp, w.cap_item_pc, &ctr->overflow);
    k_group_active<<<(unsigned)std::max(1LL, std::min(fmm_ceil_div(ng, ITHREADS / 32), 152LL * 16)), ITHREADS, 0, s>>>(
        w.groups, &ctr->n_groups, w.cap_groups, t.sact, t.act, ctr);
    return cudaGetLastError();
}

cudaError_t fmm_launch_pp(DevTree& t, DevWalk& w, DevCounters* ctr, const InteractArgs& a, cudaStream_t s)
{
    if (!(a.terms & 1)) return cudaSuccess;
    const int blocks = persistent_blocks(k_pp, g_pp_blocks);
    cudaMemsetAsync(&ctr->pp_work, 0, sizeof(unsigned long long), s);
    k_pp<<<blocks, ITHREADS, 0, s>>>(w.groups, w.item_pp, w.base_pp, w.pp, t.cfirst, t.ccount, t.cnact, t.cen,
                                     t.bucket_of, t.bucket_cell, t.off, w.part_pp, t.act, a.eps2, a.chunk, w.cap_item_pp,
                                     t.per_ib, t.per_R, ctr);
    return cudaGetLastError();
}

cudaError_t fmm_launch_pc(DevTree& t, DevWalk& w, DevCounters* ctr, const InteractArgs& a, cudaStream_t s)
{
    if (!(a.terms & 2)) return cudaSuccess;
    const int blocks = persistent_blocks(k_pc, g_pc_blocks);
    cudaMemsetAsync(&ctr->pc_work, 0, sizeof(unsigned long long), s);
    k_pc<<<blocks, ITHREADS, 0, s>>>(w.groups, w.item_pc, w.base_pc, w.pc, t.cnact, t.cen, t.bucket_of,
                                     t.bucket_cell, t.off, t.rec, w.part_pc, t.act, a.eps2, a.chunk, w.cap_item_pc,
                                     t.per_ib, t.per_R, ctr);
    return cudaGetLastError();
}

cudaError_t fmm_launch_l2p_out(DevTree& t, DevWalk& w, DevCounters* ctr, const InteractArgs& a, float* acc,
                               float* pot, long long n, cudaStream_t s, const unsigned int* perm)
{
    // the group expansions also carry the Ewald correction of a periodic box (terms & 8), so they
    // are evaluated when either part is asked for
    const int terms = (t.per_R > 0 && (a.terms & 8)) ? (a.terms | 4) : a.terms;
    if (!perm) perm = t.idx;
    const long long ng = t.cap_grid ? w.cap_groups : w.n_groups;
    if (a.accumulate == 1)
        k_l2p_out<double><<<grid_for(ng), ITHREADS, 0, s>>>(
            w.groups, &ctr->n_groups, w.cap_groups, w.cap_item_pp, w.cap_item_pc, t.cen, t.bucket_of, t.bucket_cell,
            t.off, w.Lg, w.cnt_pp, w.base_pp, w.part_pp, w.cnt_pc, w.base_pc, w.part_pc, t.act, t.cnact, perm, n, acc, pot,
            terms, ctr);
    else
        k_l2p_out<float><<<grid_for(ng), ITHREADS, 0, s>>>(
            w.groups, &ctr->n_groups, w.cap_groups, w.cap_item_pp, w.cap_item_pc, t.cen, t.bucket_of, t.bucket_cell,
            t.off, w.Lg, w.cnt_pp, w.base_pp, w.part_pp, w.cnt_pc, w.base_pc, w.part_pc, t.act, t.cnact, perm, n, acc, pot,
            terms, ctr);
    return cudaGetLastError();
}
