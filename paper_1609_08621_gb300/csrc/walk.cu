// Checklist walk and local expansions (Sec. 3.1).
//
// Sink cells are walked top-down, one tree level per launch.  A warp owns one sink cell k
// and its checklist: the sources its parent left on the checklist ("remain on the
// checklist for further consideration by the children of the sink cell") plus, for the
// root, the root itself.  Each lane takes one entry, evaluates the opening criterion and
// the warp appends the entry to one of five places with ballot/popc ranks:
//   accept  -> k's local-expansion list (CC for a cell, CP for a particle)
//   defer   -> the checklist handed to k's children
//   PC, PP  -> the group's interaction lists (k a group: <= g particles)
//   open    -> its two children, or for a bucket its particles with R_O = 0, are
//              appended to k's own queue and examined in turn.
// The criterion (single precision, fixed operation order, no fused multiply-add):
//   d = |com_k - com_s|, R_O = b_max / theta (0 for a particle or a one-particle cell)
//   accept if d > 1.5 R_O(k) + R_O(s) and the bounding boxes are >= 2 eps apart
//   k not a group: defer if s is point-like or R_O(s) <= R_O(k), else open
//   k a group:     PP if s is point-like; PC if d > R_O(s) + b_max(k); PP if s is a
//                  bucket; else open.
// Outputs are staged in per-warp scratch and copied to contiguous per-cell ranges, so each
// cell's lists are in a deterministic order whatever the scheduling.
//
// The local expansion of a walked cell is L_k = L2L(L_parent) + sum of M2L (CC) and P2L
// (CP) terms.  A level's local lists are complete when its walk kernel ends, so a large walk runs
// their M2L and P2L terms and the level's top-down pass on a side stream while the walk goes on
// below; a small one runs them after its last level.
#include <algorithm>

#include "expansions.cuh"
#include "fmm_internal.cuh"
#include "mlp.cuh"

#define WALK_WPB 4
#define WALK_THREADS (WALK_WPB * 32)

enum { OUT_NONE = 0, OUT_ACCEPT = 1, OUT_DEFER = 2, OUT_PC = 3, OUT_PP = 4, OUT_OPEN = 5 };

// Learned criterion (MODE 1): the pairs the network must decide are not evaluated one step at a
// time, where a step has a few of them and the tensor-core tile of 16 rows runs mostly empty.  They
// wait in a per-warp buffer (entry and features) until 32 of them fill two tiles, or the sink's
// queue runs dry; the evaluated entries return to the queue marked with their decision, and the
// next steps sort them like any other entry.  Marks: bit 30 accepted, bit 29 rejected (cell entries
// of an isolated box, whose indices stay below 2^29).
#define WALK_NET_ACC (1u << 30)
#define WALK_NET_REJ (1u << 29)
#define WALK_PEND 64  // pending pairs per warp: fewer than 32 left after a flush, plus one step's 32
#define WALK_PEND_BYTES (WALK_PEND * 4 + WALK_PEND * MLP_F * 4)

__device__ __forceinline__ float d2_ordered(float dx, float dy, float dz)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ float gap_axis(float lo_s, float hi_s, float lo_k, float hi_k)
{
    float g1 = __fsub_rn(lo_s, hi_k), g2 = __fsub_rn(lo_k, hi_s);
    float g = g1 > g2 ? g1 : g2;
    return g > 0.0f ? g : 0.0f;
}

// MODE 0: fixed-theta criterion.  MODE 1: learned criterion for source cells (the network
// decides inside the band, see mlp.cuh).  MODE 2: fixed criterion, and every (sink, source cell)
// pair of the band is recorded for labelling (audit).
//
// A warp examines up to E * 32 entries of its sink's queue per step: lane l takes entries
// base + s * 32 + l for slots s < E, the loads of every slot are in flight together, and the
// outcomes are ranked slot by slot, so each list comes out in queue order, exactly as with one
// entry per lane.  A sink's serial chain of steps (its checklist and what it opens, 32 entries
// at a time) set each level's duration; E entries per lane shorten it E-fold where the queue is
// long, and cost nothing extra where it is short (slots past the queue are skipped, warp-uniformly).
//
// Measured on the 128^3 NFW box: 2 to 4 entries per lane made the walk slower (3.93 ms with one,
// 4.09 with two, 4.41 with four), because the extra registers halve the resident warps and each
// entry's chain of dependent instructions does not shorten; one entry per lane is the default.
#ifndef FMM_WALK_SLOTS
#define FMM_WALK_SLOTS 1  // entries per lane and step
#endif
#ifndef FMM_WALK_MINB
#define FMM_WALK_MINB 5  // resident blocks per SM the fixed-theta walk is compiled for (96 registers, no spills)
#endif
template <int MODE>
struct WalkSlots {
    static constexpr int E = FMM_WALK_SLOTS;
};

// PER: a periodic box (list entries carry a copy code above their index bits); the isolated walk is
// compiled without the decoding.
template <int MODE, bool PER>
__global__ void __launch_bounds__(WALK_THREADS, MODE == 1 ? 4 : FMM_WALK_MINB) k_walk_level(
    const WalkNode* __restrict__ node, const float4* __restrict__ posf, const int* __restrict__ cnact,
    const int* __restrict__ f_cell, const unsigned long long* __restrict__ f_cloff, const int* __restrict__ f_cllen,
    int level, const unsigned int* __restrict__ cl_cur, int* __restrict__ f_cell_next,
    unsigned long long* __restrict__ f_cloff_next, int* __restrict__ f_cllen_next, long long cap_front,
    unsigned int* __restrict__ cl_next, long long cap_cl, unsigned long long* __restrict__ lcc_off,
    int* __restrict__ lcc_len, unsigned long long* __restrict__ lcp_off, int* __restrict__ lcp_len,
    int* __restrict__ wcells,
    unsigned int* __restrict__ pp, long long cap_pp, unsigned int* __restrict__ pc,
    long long cap_pc, unsigned int* __restrict__ cc, int* __restrict__ cc_sink, long long cap_cc,
    unsigned int* __restrict__ cp, int* __restrict__ cp_sink, long long cap_cp,
    Group* __restrict__ groups, long long cap_groups, unsigned int* __restrict__ scratch, long long cap_scr,
    DevCounters* __restrict__ ctr, int bucket, int group, float four_eps2, const float4* __restrict__ mnorm,
    const float* __restrict__ amin,
    float eps, float band_lo, float band_hi, float tau, float margin, const unsigned char* __restrict__ mlp_packed,
    int2* __restrict__ audit_pairs, long long audit_cap, const unsigned char* __restrict__ nogroup, PeriodicArgs pa)
{
    constexpr int E = WalkSlots<MODE>::E;
    const unsigned int q0 = PER ? copy_centre(pa.R) : 0u;
    const int ib = PER ? pa.ib : 31;  // index bits of a list entry
    extern __shared__ __align__(16) unsigned char walk_smem[];
    if (MODE == 1) {
        mlp_load_smem(mlp_packed, walk_smem);
        __syncthreads();
    }
    unsigned char* mlp_scratch = walk_smem + MLPP_SIZE + (threadIdx.x >> 5) * MLP_WARP_SCRATCH;
    unsigned int* pend_e = reinterpret_cast<unsigned int*>(walk_smem + MLPP_SIZE + WALK_WPB * MLP_WARP_SCRATCH +
                                                           (threadIdx.x >> 5) * WALK_PEND_BYTES);
    float* pend_f = reinterpret_cast<float*>(pend_e + WALK_PEND);
    static_assert(MODE != 1 || E == 1, "the learned walk takes one entry per lane and step");
    unsigned long long n_mlp = 0;
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    unsigned int* Q = scratch + gw * 5 * cap_scr;
    unsigned int* D = Q + cap_scr;
    unsigned int* A = Q + 2 * cap_scr;  // accepted: multipole sources from the front, point sources from the back
    unsigned int* P = Q + 3 * cap_scr;
    unsigned int* C = Q + 4 * cap_scr;
    const unsigned int lt = fmm_lanemask_lt();
    const unsigned long long n_front = *(volatile unsigned long long*)&ctr->lv_front[level];
    // this level's sinks go to the walked-cell list after the levels before it
    const unsigned long long wbase = *(volatile unsigned long long*)&ctr->lv_base[level];
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->lv_base[level + 1] = wbase + n_front;
    unsigned long long w_entries = 0, w_max = 0;  // this warp's statistics, added once at the end

    for (;;) {
        unsigned long long fi = 0;
        if (lane == 0) fi = atomicAdd(&ctr->lv_work[level], 1ull);
        fi = __shfl_sync(FMM_FULL_MASK, fi, 0);
        if (fi >= n_front) break;
        const int k = f_cell[fi];
        if (lane == 0 && (long long)(wbase + fi) < cap_front) wcells[wbase + fi] = k;
        const WalkNode K = node[k];
        // a group holds <= g particles; in a graded tree (dual trees) it is also no larger than the
        // fixed tree's groups around it
        const bool kg = K.d.w <= group && !(nogroup && nogroup[k]);
        const float rk = K.a.w, bk = K.b.w;
        const float ak = MODE == 1 ? amin[k] : 0.0f;
        const unsigned long long cl0 = f_cloff[fi];
        const long long ncl = f_cllen[fi];
        long long nq = 0, nd = 0, na = 0, nap = 0, npp = 0, npc = 0;
        int npend = 0;  // learned criterion: pairs waiting for the network
        int srcpp = 0;  // this lane's PP source particles
        bool overflow = false;
        long long base = 0;
        while (base < ncl + nq) {
            // entries appended while this step runs get indices >= ncl + nq (step start), so the
            // next step begins right after the entries that were actually available here
            const long long avail = ncl + nq - base;
            const int ns = avail >= 32 * E ? E : (int)((avail + 31) >> 5);  // slots in use (warp-uniform)
            unsigned int e[E];
            bool valid[E];
#pragma unroll
            for (int s = 0; s < E; s++) {
                const long long vi = base + s * 32 + lane;
                valid[s] = s < ns && s * 32 + lane < avail;
                e[s] = 0;
                if (valid[s]) e[s] = vi < ncl ? cl_cur[cl0 + vi] : Q[vi - ncl];
            }
            unsigned int decided = 0u;  // learned criterion: the network's decision carried by the entry
            if (MODE == 1 && valid[0] && !(e[0] & FMM_PARTICLE_BIT)) {
                decided = e[0] & (WALK_NET_ACC | WALK_NET_REJ);
                e[0] &= ~(WALK_NET_ACC | WALK_NET_REJ);
            }
            base += avail < 32 * E ? avail : 32 * E;
            WalkNode S[E];
#pragma unroll
            for (int s = 0; s < E; s++) {
                if (valid[s]) {
                    const unsigned int j = entry_index(e[s], ib);
                    if (e[s] & FMM_PARTICLE_BIT) S[s].a = posf[j];
                    else S[s] = node[j];
                }
            }
            // a source in a periodic copy: its centre and box shifted in FP64, then rounded, read from
            // the tables of those values (the axes with a non-zero shift)
#pragma unroll
            for (int s = 0; s < E; s++) {
                if (PER && valid[s] && entry_copy(e[s], ib) != q0) {
                    const unsigned int j = entry_index(e[s], ib);
                    int nv[3];
                    copy_shift(entry_copy(e[s], ib), pa.R, nv[0], nv[1], nv[2]);
                    const int w2 = 2 * pa.R;
#pragma unroll
                    for (int ax = 0; ax < 3; ax++) {
                        if (nv[ax] == 0) continue;
                        const long long slot = ((long long)j * 3 + ax) * w2 + shift_slot(nv[ax], pa.R);
                        if (e[s] & FMM_PARTICLE_BIT) {
                            const float x = pa.pshift[slot];
                            if (ax == 0) S[s].a.x = x;
                            else if (ax == 1) S[s].a.y = x;
                            else S[s].a.z = x;
                        } else {
                            const float4 g = pa.cshift[slot];
                            if (ax == 0) {
                                S[s].a.x = g.x;
                                S[s].b.x = g.y;
                                S[s].c.x = g.z;
                            } else if (ax == 1) {
                                S[s].a.y = g.x;
                                S[s].b.y = g.y;
                                S[s].c.y = g.z;
                            } else {
                                S[s].a.z = g.x;
                                S[s].b.z = g.y;
                                S[s].c.z = g.z;
                            }
                        }
                    }
                }
            }
            int out[E], nadd[E], sfirst[E], c0[E], c1[E], nsrc_cell[E];
            bool sleaf[E], ptl[E];
#pragma unroll
            for (int s = 0; s < E; s++) {
                out[s] = OUT_NONE;
                nadd[s] = 0;
                sfirst[s] = 0;
                c0[s] = c1[s] = -1;
                nsrc_cell[s] = 0;
                sleaf[s] = false;
                ptl[s] = false;
                if (s >= ns) continue;
                float f[MLP_F];  // learned criterion: the pair's features (set for band pairs)
                bool pointlike = false, acc = false, need = false;
                float d2 = 0.0f, ro = 0.0f;
                if (valid[s]) {
                    float cx, cy, cz, lox, loy, loz, hix, hiy, hiz;
                    if (e[s] & FMM_PARTICLE_BIT) {
                        const float4 p = S[s].a;
                        cx = lox = hix = p.x;
                        cy = loy = hiy = p.y;
                        cz = loz = hiz = p.z;
                        ro = 0.0f;
                        pointlike = true;
                    } else {
                        cx = S[s].a.x; cy = S[s].a.y; cz = S[s].a.z; ro = S[s].a.w;
                        lox = S[s].b.x; loy = S[s].b.y; loz = S[s].b.z;
                        hix = S[s].c.x; hiy = S[s].c.y; hiz = S[s].c.z;
                        pointlike = S[s].d.w == 1;
                        sleaf[s] = S[s].d.x < 0;  // a leaf (bucket) has no children
                        c0[s] = S[s].d.x;
                        c1[s] = S[s].d.y;
                        sfirst[s] = S[s].d.z;
                        nsrc_cell[s] = S[s].d.w;
                        nadd[s] = sleaf[s] ? S[s].d.w : 2;
                    }
                    d2 = d2_ordered(__fsub_rn(K.a.x, cx), __fsub_rn(K.a.y, cy), __fsub_rn(K.a.z, cz));
                    const float thr = __fadd_rn(__fmul_rn(1.5f, rk), ro);
                    const float gx = gap_axis(lox, hix, K.b.x, K.c.x);
                    const float gy = gap_axis(loy, hiy, K.b.y, K.c.y);
                    const float gz = gap_axis(loz, hiz, K.b.z, K.c.z);
                    const float gap2 = d2_ordered(gx, gy, gz);
                    acc = d2 > __fmul_rn(thr, thr) && gap2 >= four_eps2;
                    if (MODE != 0 && !pointlike) {
                        float te;
                        int band = mlp_band(K, S[s], d2, gap2, four_eps2, band_lo, band_hi, te);
                        if (MODE == 1) {
                            if (band == 3 && decided) {
                                band = decided == WALK_NET_ACC ? 1 : 2;  // the network has decided
                            } else if (band == 3 && !(ak > 0.0f)) {
                                band = acc ? 1 : 2;  // no acceleration estimate: the fixed criterion decides
                            } else if (band == 3) {
                                mlp_pair_features(K, S[s], mnorm[entry_index(e[s], ib)], ak, eps, f);
                                band = mlp_surrogate(reinterpret_cast<const float*>(walk_smem + MLPP_SUR), f, te, tau,
                                                     margin);
                            }
                            acc = band == 1;
                            need = band == 3;
                        } else if (band == 3) {
                            const unsigned long long q = atomicAdd(&ctr->n_audit, 1ull);
                            if ((long long)q < audit_cap) audit_pairs[q] = make_int2(k, (int)e[s]);
                        }
                    }
                }
                if (MODE == 1) {
                    // a pair for the network waits in the buffer and gives no output this step
                    const unsigned int nm = __ballot_sync(FMM_FULL_MASK, need);
                    if (need) {
                        const int slot = npend + __popc(nm & lt);
                        pend_e[slot] = e[s];
#pragma unroll
                        for (int q = 0; q < MLP_F; q++) pend_f[slot * MLP_F + q] = f[q];
                    }
                    npend += __popc(nm);
                    if (need) {
                        valid[s] = false;
                        nadd[s] = 0;
                    }
                }
                ptl[s] = pointlike;
                if (valid[s]) {
                    if (acc) {
                        out[s] = OUT_ACCEPT;
                    } else if (!kg) {
                        out[s] = (pointlike || ro <= rk) ? OUT_DEFER : OUT_OPEN;
                    } else if (pointlike) {
                        out[s] = OUT_PP;
                    } else {
                        const float u = __fadd_rn(ro, bk);
                        if (d2 > __fmul_rn(u, u)) out[s] = OUT_PC;
                        else out[s] = sleaf[s] ? OUT_PP : OUT_OPEN;
                    }
                    if (out[s] != OUT_OPEN) nadd[s] = 0;
                }
            }
            // ranks in queue order: slot by slot, lanes in order within a slot
            unsigned int mA[E], mAp[E], mD[E], mC[E], mP[E];
            int incl[E], tot[E];
            long long tA = 0, tAp = 0, tD = 0, tC = 0, tP = 0, tQ = 0;
#pragma unroll
            for (int s = 0; s < E; s++) {
                mA[s] = mAp[s] = mD[s] = mC[s] = mP[s] = 0u;
                incl[s] = tot[s] = 0;
                if (s >= ns) continue;
                mA[s] = __ballot_sync(FMM_FULL_MASK, out[s] == OUT_ACCEPT && !ptl[s]);
                mAp[s] = __ballot_sync(FMM_FULL_MASK, out[s] == OUT_ACCEPT && ptl[s]);
                mD[s] = __ballot_sync(FMM_FULL_MASK, out[s] == OUT_DEFER);
                mC[s] = __ballot_sync(FMM_FULL_MASK, out[s] == OUT_PC);
                mP[s] = __ballot_sync(FMM_FULL_MASK, out[s] == OUT_PP);
                int v = nadd[s];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(FMM_FULL_MASK, v, o);
                    if (lane >= o) v += t;
                }
                incl[s] = v;
                tot[s] = __shfl_sync(FMM_FULL_MASK, v, 31);
                tA += __popc(mA[s]);
                tAp += __popc(mAp[s]);
                tD += __popc(mD[s]);
                tC += __popc(mC[s]);
                tP += __popc(mP[s]);
                tQ += tot[s];
            }
            if (na + nap + tA + tAp > cap_scr || nd + tD > cap_scr || npc + tC > cap_scr || npp + tP > cap_scr ||
                nq + tQ > cap_scr) {
                overflow = true;
                break;
            }
#pragma unroll
            for (int s = 0; s < E; s++) {
                if (s >= ns) continue;
                if (out[s] == OUT_ACCEPT) {
                    if (ptl[s]) A[cap_scr - 1 - (nap + __popc(mAp[s] & lt))] = e[s];
                    else A[na + __popc(mA[s] & lt)] = e[s];
                }
                if (out[s] == OUT_DEFER) D[nd + __popc(mD[s] & lt)] = e[s];
                if (out[s] == OUT_PC) C[npc + __popc(mC[s] & lt)] = e[s];
                if (out[s] == OUT_PP) {
                    P[npp + __popc(mP[s] & lt)] = e[s];
                    srcpp += (e[s] & FMM_PARTICLE_BIT) ? 1 : nsrc_cell[s];
                }
                if (out[s] == OUT_OPEN) {
                    // the children, or a leaf's particles, stay in the source's copy
                    const long long pos = nq + incl[s] - nadd[s];
                    const unsigned int qb = PER ? entry_copy(e[s], ib) << ib : 0u;
                    if (sleaf[s]) {
                        for (int j = 0; j < nadd[s]; j++)
                            Q[pos + j] = ((unsigned int)(sfirst[s] + j) | qb) | FMM_PARTICLE_BIT;
                    } else {
                        Q[pos] = (unsigned int)c0[s] | qb;
                        Q[pos + 1] = (unsigned int)c1[s] | qb;
                    }
                }
                na += __popc(mA[s]);
                nap += __popc(mAp[s]);
                nd += __popc(mD[s]);
                npc += __popc(mC[s]);
                npp += __popc(mP[s]);
                nq += tot[s];
            }
            __syncwarp();
            if (MODE == 1) {
                // evaluate 32 waiting pairs (or the rest once the queue is dry) and return them
                // to the queue with their decisions
                while (npend >= 32 || (npend > 0 && base >= ncl + nq)) {
                    const int cnt = npend < 32 ? npend : 32;
                    if (nq + cnt > cap_scr) {
                        overflow = true;
                        break;
                    }
                    float f[MLP_F];
                    const bool have = lane < cnt;
#pragma unroll
                    for (int q = 0; q < MLP_F; q++) f[q] = have ? pend_f[lane * MLP_F + q] : 0.0f;
                    const unsigned int pe = have ? pend_e[lane] : 0u;
                    const float pred = mlp_predict_warp(walk_smem, mlp_scratch, f, lane,
                                                        cnt == 32 ? FMM_FULL_MASK : (1u << cnt) - 1u);
                    if (have) Q[nq + lane] = pe | (pred < tau ? WALK_NET_ACC : WALK_NET_REJ);
                    n_mlp += cnt;
                    nq += cnt;
                    // move the rest (fewer than 32) to the front of the buffer
                    const int rest = npend - cnt;
                    unsigned int me = 0u;
                    float mf[MLP_F];
                    if (lane < rest) {
                        me = pend_e[cnt + lane];
#pragma unroll
                        for (int q = 0; q < MLP_F; q++) mf[q] = pend_f[(cnt + lane) * MLP_F + q];
                    }
                    __syncwarp();
                    if (lane < rest) {
                        pend_e[lane] = me;
#pragma unroll
                        for (int q = 0; q < MLP_F; q++) pend_f[lane * MLP_F + q] = mf[q];
                    }
                    npend = rest;
                    __syncwarp();
                }
                if (overflow) break;
            }
        }
        if (overflow) {
            if (lane == 0) atomicOr(&ctr->overflow, 1u);
            continue;
        }
        w_entries += (unsigned long long)(ncl + nq);
        w_max = max(w_max, (unsigned long long)(ncl + nq));
        // local-expansion entries of this sink: multipole sources (M2L) and point sources (P2L) in
        // two lists, each in queue order
        unsigned long long off = 0, offp = 0;
        if (lane == 0) {
            if (na) {
                off = atomicAdd(&ctr->cc_len, (unsigned long long)na);
                atomicAdd(&ctr->lv_cc[level], (unsigned long long)na);
            }
            if (nap) {
                offp = atomicAdd(&ctr->cp_len, (unsigned long long)nap);
                atomicAdd(&ctr->lv_cp[level], (unsigned long long)nap);
            }
        }
        off = __shfl_sync(FMM_FULL_MASK, off, 0);
        offp = __shfl_sync(FMM_FULL_MASK, offp, 0);
        if ((long long)(off + na) > cap_cc || (long long)(offp + nap) > cap_cp) {
            if (lane == 0) atomicOr(&ctr->overflow, 1u);
            continue;
        }
        for (long long i = lane; i < na; i += 32) {
            cc[off + i] = A[i];
            cc_sink[off + i] = k;
        }
        for (long long i = lane; i < nap; i += 32) {
            cp[offp + i] = A[cap_scr - 1 - i];
            cp_sink[offp + i] = k;
        }
        if (lane == 0) {
            lcc_off[k] = off;
            lcc_len[k] = (int)na;
            lcp_off[k] = offp;
            lcp_len[k] = (int)nap;
        }
        if (kg) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) srcpp += __shfl_xor_sync(FMM_FULL_MASK, srcpp, o);
            unsigned long long po = 0, co = 0, gi = 0;
            if (lane == 0) {
                po = atomicAdd(&ctr->pp_len, (unsigned long long)npp);
                co = atomicAdd(&ctr->pc_len, (unsigned long long)npc);
                gi = atomicAdd(&ctr->n_groups, 1ull);
            }
            po = __shfl_sync(FMM_FULL_MASK, po, 0);
            co = __shfl_sync(FMM_FULL_MASK, co, 0);
            gi = __shfl_sync(FMM_FULL_MASK, gi, 0);
            if ((long long)(po + npp) > cap_pp || (long long)(co + npc) > cap_pc || (long long)gi >= cap_groups) {
                if (lane == 0) atomicOr(&ctr->overflow, 1u);
                continue;
            }
            for (long long i = lane; i < npp; i += 32) pp[po + i] = P[i];
            for (long long i = lane; i < npc; i += 32) pc[co + i] = C[i];
            if (lane == 0) {
                Group g;
                g.cell = k;
                g.first = K.d.z;
                g.count = K.d.w;
                g.pp_src = srcpp;
                g.pp_off = po;
                g.pc_off = co;
                g.pp_len = (int)npp;
                g.pc_len = (int)npc;
                groups[gi] = g;
            }
        } else {
            unsigned long long doff = 0;
            if (lane == 0) doff = atomicAdd(&ctr->lv_cl[level + 1], (unsigned long long)nd);
            doff = __shfl_sync(FMM_FULL_MASK, doff, 0);
            if ((long long)(doff + nd) > cap_cl) {
                if (lane == 0) atomicOr(&ctr->overflow, 1u);
                continue;
            }
            for (long long i = lane; i < nd; i += 32) cl_next[doff + i] = D[i];
            if (lane < 2) {
                int c = lane == 0 ? K.d.x : K.d.y;
                if (cnact[c] > 0) {
                    unsigned long long fj = atomicAdd(&ctr->lv_front[level + 1], 1ull);
                    if ((long long)fj < cap_front) {
                        f_cell_next[fj] = c;
                        f_cloff_next[fj] = doff;
                        f_cllen_next[fj] = (int)nd;
                    } else {
                        atomicOr(&ctr->overflow, 1u);
                    }
                }
            }
        }
    }
    if (MODE == 1 && lane == 0 && n_mlp) atomicAdd(&ctr->n_mlp, n_mlp);
    if (lane == 0 && w_entries) {
        atomicAdd(&ctr->lv_entries[level], w_entries);
        atomicMax(&ctr->lv_max_entries[level], w_max);
    }
}

#define LOCAL_WPB 2
#define LOCAL_THREADS (LOCAL_WPB * 32)

// Own local expansions over the flat list of all local entries (every walked sink's CC and CP
// entries, contiguous per sink).  A warp takes a range of about LF_ENTRIES entries, moved to the
// next sink boundaries so that no sink is split between warps, and walks it in chunks of 32, one
// entry per lane, so lanes stay busy whatever the list lengths.  Each sink's 56 coefficients are
// added strictly in list order (runs of equal sink along the lanes, a run that continues into
// the next chunk carried on): the result depends only on the sink's own list, not on where the
// list lies in the flat array or which warp took it.
#define LF_ENTRIES FMM_LOCAL_RANGE

// Centres enter as float pairs (cen_diff): the sink's (hk, lk), a cell's from cen, a particle's
// from posf (hi, and its mass) and plo (lo); a source in a periodic copy has its pair shifted
// (cen_shift) by the copy's integer offset.
// KIND 0: a cell of several particles (M2L); KIND 1: a particle, or a cell of one (P2L).
template <int KIND>
__device__ __forceinline__ void local_entry(unsigned int e, const float4& hk, const float4& lk,
                                            const float4* __restrict__ cen,
                                            const float4* __restrict__ posf, const float4* __restrict__ plo,
                                            const float* __restrict__ rec, float eps2, int ib, int R, float* acc)
{
    const unsigned int j = entry_index(e, ib);
    const unsigned int q = entry_copy(e, ib);
    const bool shifted = q != copy_centre(R);
    int nx = 0, ny = 0, nz = 0;
    if (shifted) copy_shift(q, R, nx, ny, nz);
    float4 hs, ls;
    if (e & FMM_PARTICLE_BIT) {
        hs = posf[j];
        ls = plo[j];
    } else {
        hs = cen[2 * j];
        ls = cen[2 * j + 1];
    }
    if (shifted) {
        cen_shift(hs.x, ls.x, (float)nx);
        cen_shift(hs.y, ls.y, (float)ny);
        cen_shift(hs.z, ls.z, (float)nz);
    }
    const float rx = cen_diff(hk.x, lk.x, hs.x, ls.x), ry = cen_diff(hk.y, lk.y, hs.y, ls.y),
                rz = cen_diff(hk.z, lk.z, hs.z, ls.z);
    if (KIND == 1) {
        // a one-particle cell: its particle (mass = moment M[0]) -> local expansion
        fmm_p2l_acc((e & FMM_PARTICLE_BIT) ? hs.w : rec[(long long)j * FMM_NREC], rx, ry, rz, eps2, acc);
    } else {
        float M[FMM_NMOM];
        const float4* r4 = reinterpret_cast<const float4*>(rec + (long long)j * FMM_NREC);
#pragma unroll
        for (int q4 = 0; q4 < FMM_NMOM / 4; q4++) {
            const float4 v = r4[q4];
            M[4 * q4] = v.x;
            M[4 * q4 + 1] = v.y;
            M[4 * q4 + 2] = v.z;
            M[4 * q4 + 3] = v.w;
        }
        fmm_m2l_acc(M, rx, ry, rz, eps2, acc);
    }
}

// first entry of the first sink that starts at or after position p of the flat list
__device__ __forceinline__ long long local_boundary(long long p, long long total, const int* __restrict__ cc_sink,
                                                    const unsigned long long* __restrict__ lcc_off,
                                                    const int* __restrict__ lcc_len)
{
    if (p >= total) return total;
    const int k = cc_sink[p];
    const long long f = (long long)lcc_off[k];
    return f == p ? p : f + lcc_len[k];
}

// Two launches, one per list: KIND 0 the multipole sources (M2L), which write each sink's sum;
// KIND 1 the point sources (P2L), which add theirs to it (or write it, for a sink with no
// multipole source).  Every warp of a launch runs one kind of interaction.
// One level's entries: those of the sinks of walk level `level`, [sum of the earlier levels' counts,
// plus this level's), all of them complete when the level's walk kernel has ended; level -1: all.
#ifndef FMM_LOCAL_MINB
#define FMM_LOCAL_MINB 8  // resident blocks per SM the local-expansion kernels are compiled for (128 registers)
#endif
template <int KIND>
__global__ void __launch_bounds__(LOCAL_THREADS, FMM_LOCAL_MINB) k_local_flat(
    const unsigned int* __restrict__ cc, const int* __restrict__ cc_sink, const unsigned long long* __restrict__ lcc_off,
    const int* __restrict__ lcc_len, const int* __restrict__ lm2l_len, const float4* __restrict__ cen,
    const float4* __restrict__ posf, const float4* __restrict__ plo,
    const float* __restrict__ rec, float* __restrict__ Lown, long long cap_cc,
    float eps2, int ib, int R, int level, DevCounters* __restrict__ ctr)
{
    __shared__ float red[LOCAL_WPB][32][FMM_NL + 1];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    if (fmm_overflowed(ctr)) return;
    long long start = 0, total;
    if (level < 0) {  // every level's entries
        total = min((long long)*(volatile unsigned long long*)(KIND == 0 ? &ctr->cc_len : &ctr->cp_len), cap_cc);
    } else {
        const unsigned long long* lv = KIND == 0 ? ctr->lv_cc : ctr->lv_cp;
        for (int l = 0; l < level; l++) start += (long long)__ldcg(lv + l);
        total = min(start + (long long)__ldcg(lv + level), cap_cc);
    }
    if (start >= total) return;
    const long long nranges = fmm_ceil_div(total - start, LF_ENTRIES);
    const int c0 = lane, c1 = lane + 32;  // this lane's coefficients in the reduction
    int nent = 0;
    for (long long r = gw; r < nranges; r += nw) {
        const long long r0 = local_boundary(start + r * LF_ENTRIES, total, cc_sink, lcc_off, lcc_len);
        const long long r1 = local_boundary(start + (r + 1) * LF_ENTRIES, total, cc_sink, lcc_off, lcc_len);
        float carry0 = 0.0f, carry1 = 0.0f;
        int carry_sink = -1;
        for (long long base = r0; base < r1; base += 32) {
            const long long idx = base + lane;
            const bool valid = idx < r1;
            int sink = -1;
            float acc[FMM_NL];
#pragma unroll
            for (int i = 0; i < FMM_NL; i++) acc[i] = 0.0f;
            if (valid) {
                sink = cc_sink[idx];
                local_entry<KIND>(cc[idx], cen[2 * sink], cen[2 * sink + 1], cen, posf, plo, rec, eps2, ib, R, acc);
                nent++;
            }
#pragma unroll
            for (int i = 0; i < FMM_NL; i++) red[wl][lane][i] = acc[i];
            const int prev = __shfl_up_sync(FMM_FULL_MASK, sink, 1);
            unsigned int heads = __ballot_sync(FMM_FULL_MASK, valid && (lane == 0 || sink != prev));
            __syncwarp();
            const int nvalid = (int)min(32LL, r1 - base);
            while (heads) {
                const int st = __ffs(heads) - 1;
                heads &= heads - 1;
                const int en = heads ? __ffs(heads) - 1 : nvalid;  // exclusive
                const int s_sink = __shfl_sync(FMM_FULL_MASK, sink, st);
                const bool cont = st == 0 && carry_sink == s_sink;
                float sum0 = cont ? carry0 : 0.0f, sum1 = cont ? carry1 : 0.0f;
                for (int row = st; row < en; row++) {
                    sum0 += red[wl][row][c0];
                    if (c1 < FMM_NL) sum1 += red[wl][row][c1];
                }
                carry_sink = -1;
                const long long se = (long long)lcc_off[s_sink] + lcc_len[s_sink];
                if (base + en < se) {  // the sink's list goes on in the next chunk
                    carry0 = sum0;
                    carry1 = sum1;
                    carry_sink = s_sink;
                    continue;
                }
                float* dst = Lown + (long long)s_sink * FMM_NL;
                if (KIND == 1 && lm2l_len[s_sink] > 0) {
                    sum0 = dst[c0] + sum0;
                    if (c1 < FMM_NL) sum1 = dst[c1] + sum1;
                }
                dst[c0] = sum0;
                if (c1 < FMM_NL) dst[c1] = sum1;
            }
            __syncwarp();
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nent += __shfl_xor_sync(FMM_FULL_MASK, nent, o);
    if (lane == 0 && nent) atomicAdd(KIND == 0 ? &ctr->n_cc : &ctr->n_cp, (unsigned long long)nent);
}

// The local expansion of every walked cell about its centre of mass, top-down one level per
// launch: L(c) = L2L(L(parent), com(c) - com(parent)) + L_own(c), with L_own the sum of c's own
// M2L and P2L terms (zero for a cell with empty lists) and a level-0 cell taking its own terms
// only.  Written in place over L_own.  A local expansion is a polynomial of degree 5, so the chain
// of re-expansions equals re-expanding every ancestor's own terms to the cell directly.  One
// thread per cell.
#define LD_THREADS 128
__global__ void __launch_bounds__(LD_THREADS) k_local_down(int level, const int* __restrict__ wcells, long long cap,
                                                          const int* __restrict__ cparent,
                                                          const int* __restrict__ lcc_len,
                                                          const int* __restrict__ lcp_len,
                                                          const Com4* __restrict__ com, float* __restrict__ L,
                                                          const DevCounters* __restrict__ ctr)
{
    if (fmm_overflowed(ctr)) return;
    const long long b0 = min((long long)ctr->lv_base[level], cap);
    const long long b1 = min((long long)ctr->lv_base[level + 1], cap);
    for (long long i = b0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < b1;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = wcells[i];
        float* Lc = L + (long long)c * FMM_NL;
        float acc[FMM_NL];
        if (lcc_len[c] > 0 || lcp_len[c] > 0) {
#pragma unroll
            for (int q = 0; q < FMM_NL; q++) acc[q] = Lc[q];
        } else {
#pragma unroll
            for (int q = 0; q < FMM_NL; q++) acc[q] = 0.0f;
        }
        if (level > 0) {
            const int p = cparent[c];
            const Com4 cc = com[c], cp = com[p];
            float Lo[FMM_NL];
            fmm_l2l(L + (long long)p * FMM_NL, __double2float_rn(cc.x - cp.x), __double2float_rn(cc.y - cp.y),
                    __double2float_rn(cc.z - cp.z), Lo);
#pragma unroll
            for (int q = 0; q < FMM_NL; q++) acc[q] = Lo[q] + acc[q];
        }
#pragma unroll
        for (int q = 0; q < FMM_NL; q++) Lc[q] = acc[q];
    }
}

// Each group's local expansion: its cell's, after the top-down pass.
__global__ void k_local_groups(const Group* __restrict__ groups, const float* __restrict__ L, float* __restrict__ Lg,
                               long long cap_groups, const DevCounters* __restrict__ ctr)
{
    if (fmm_overflowed(ctr)) return;
    const long long ng = min((long long)*(volatile const unsigned long long*)&ctr->n_groups, cap_groups);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ng * FMM_NL;
         i += (long long)gridDim.x * blockDim.x) {
        const long long gi = i / FMM_NL;
        Lg[i] = L[(long long)groups[gi].cell * FMM_NL + (i - gi * FMM_NL)];
    }
}

// The shifted geometry of a periodic box's copies (PeriodicArgs): per cell and particle, axis and
// non-zero shift v, the FP64 sum rounded once to FP32 -- the values the walk's decisions use.
__global__ void k_shift_tables(const unsigned int* __restrict__ ncell, long long n, int R, const Com4* __restrict__ com,
                               const double* __restrict__ clo, const double* __restrict__ chi,
                               const double* __restrict__ sx, const double* __restrict__ sy,
                               const double* __restrict__ sz, float4* __restrict__ cshift, float* __restrict__ pshift)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int w2 = 2 * R;
    if (i < (long long)*ncell) {
        const Com4 c = com[i];
        const double cc[3] = {c.x, c.y, c.z};
        for (int ax = 0; ax < 3; ax++)
            for (int v = -R; v <= R; v++) {
                if (v == 0) continue;
                cshift[(i * 3 + ax) * w2 + shift_slot(v, R)] =
                    make_float4(__double2float_rn(cc[ax] + v), __double2float_rn(clo[3 * i + ax] + v),
                                __double2float_rn(chi[3 * i + ax] + v), 0.0f);
            }
    }
    if (i < n) {
        const double x[3] = {sx[i], sy[i], sz[i]};
        for (int ax = 0; ax < 3; ax++)
            for (int v = -R; v <= R; v++) {
                if (v == 0) continue;
                pshift[(i * 3 + ax) * w2 + shift_slot(v, R)] = __double2float_rn(x[ax] + v);
            }
    }
}

cudaError_t fmm_launch_shift_tables(DevTree& t, cudaStream_t s)
{
    if (t.per_R <= 0) return cudaSuccess;
    if (!t.cshift || !t.pshift) return cudaErrorInvalidValue;
    const long long span = std::max(t.cap_grid ? t.cap_cells : t.n_cells, t.n);
    k_shift_tables<<<(unsigned)fmm_ceil_div(span, 256), 256, 0, s>>>(t.dcount, t.n, t.per_R, t.com, t.clo, t.chi, t.sx,
                                                                     t.sy, t.sz, t.cshift, t.pshift);
    return cudaGetLastError();
}

// level 0 of the walk: every box's root cell as a sink, with that root alone on its checklist
// (isolated boxes: sources of other boxes are never seen); boxes without an active particle
// are not walked
// Each box's root starts the walk with itself on its checklist.  With one box and second_root >= 0
// (the root of an appended fixed tree, dual.cu) the checklist holds both roots.
// In a periodic box (R > 0, one box) the checklist holds the root and its (2R + 1)^3 - 1 copies,
// in the order of their copy codes.
__global__ void k_walk_seed(int* f_cell, unsigned long long* f_cloff, int* f_cllen, unsigned int* cl,
                            const int* __restrict__ cnact, const int* __restrict__ box_root, int nbox,
                            int second_root, int R, int ib, DevCounters* ctr)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const int r = box_root ? box_root[b] : 0;
    if (r < 0 || cnact[r] <= 0) return;  // an empty box has no root cell
    const unsigned long long k = atomicAdd(&ctr->lv_front[0], 1ull);
    f_cell[k] = r;
    if (R > 0) {  // one box only
        const int W = 2 * R + 1, nc = W * W * W;
        f_cloff[k] = 0;
        f_cllen[k] = nc;
        for (int q = 0; q < nc; q++) cl[q] = ((unsigned int)q << ib) | (unsigned int)r;
        return;
    }
    if (second_root >= 0) {  // one box only: its entries are cl[0], cl[1]
        f_cloff[k] = 0;
        f_cllen[k] = 2;
        cl[0] = (unsigned int)r;
        cl[1] = (unsigned int)second_root;
        return;
    }
    f_cloff[k] = k;
    f_cllen[k] = 1;
    cl[k] = (unsigned int)r;
}

cudaError_t fmm_launch_walk_seed(DevTree& t, DevWalk& w, DevCounters* ctr, cudaStream_t s, int second_root)
{
    if (second_root >= 0 && t.nbox != 1) return cudaErrorInvalidValue;
    if (t.per_R > 0 && (t.nbox != 1 || second_root >= 0)) return cudaErrorInvalidValue;
    k_walk_seed<<<(unsigned)fmm_ceil_div(t.nbox, 128), 128, 0, s>>>(w.f_cell[0], w.f_cloff[0], w.f_cllen[0], w.cl[0],
                                                                     t.cnact, t.nbox > 1 ? t.box_root : nullptr,
                                                                     t.nbox, second_root, t.per_R, t.per_ib, ctr);
    return cudaGetLastError();
}

int fmm_walk_warps(int device)
{
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms * 24;  // warps per SM of the walk and local-expansion grids (measured better than 20 or 16)
}

cudaError_t fmm_launch_walk_level(DevTree& t, DevWalk& w, DevCounters* ctr, const WalkArgs& a, cudaStream_t s)
{
    const int cur = a.level_parity, nxt = cur ^ 1;
    // persistent grid: every warp owns a scratch slot; idle warps exit after one atomic
    const int blocks = w.n_warps / WALK_WPB;
#define WALK_ARGS                                                                                                   \
    t.node, t.posf, t.cnact, w.f_cell[cur], w.f_cloff[cur], w.f_cllen[cur], a.level, w.cl[cur], w.f_cell[nxt],      \
        w.f_cloff[nxt], w.f_cllen[nxt], w.cap_front, w.cl[nxt], w.cap_cl, w.lcc_off, w.lcc_len, w.lcp_off,          \
        w.lcp_len, w.wcells, w.pp, w.cap_pp, w.pc, w.cap_pc, w.cc, w.cc_sink, w.cap_cc, w.cp, w.cp_sink, w.cap_cp, w.groups, w.cap_groups, w.scratch, w.cap_scratch, ctr, \
        a.bucket, a.group, a.four_eps2, t.mnorm, t.amin, a.eps, a.band_lo, a.band_hi, a.tau, a.margin, a.mlp_packed, a.audit_pairs, \
        a.audit_cap, t.graded ? t.nogroup : nullptr, periodic_args(t)
    // the learned and audit walks take isolated boxes only (the host refuses the combinations)
    if (a.mode != 0 && t.per_R > 0) return cudaErrorInvalidValue;
    if (a.mode == 1) {
        const size_t smem = MLPP_SIZE + (size_t)WALK_WPB * (MLP_WARP_SCRATCH + WALK_PEND_BYTES);
        static std::atomic<unsigned long long> attr{0};
        cudaError_t e = fmm_smem_attr_once(k_walk_level<1, false>, (int)smem, attr);
        if (e != cudaSuccess) return e;
        k_walk_level<1, false><<<blocks, WALK_THREADS, smem, s>>>(WALK_ARGS);
    } else if (a.mode == 2) {
        k_walk_level<2, false><<<blocks, WALK_THREADS, 0, s>>>(WALK_ARGS);
    } else if (t.per_R > 0) {
        k_walk_level<0, true><<<blocks, WALK_THREADS, 0, s>>>(WALK_ARGS);
    } else {
        k_walk_level<0, false><<<blocks, WALK_THREADS, 0, s>>>(WALK_ARGS);
    }
#undef WALK_ARGS
    return cudaGetLastError();
}

// The local expansions of walk level `level` (-1: the whole lists, then every level's top-down
// pass): its own M2L terms, then its P2L terms, then the top-down pass of its cells (which reads the
// level above, done by an earlier call on the same stream).  The grids are the caller's: every
// kernel takes its work with grid-stride loops, so any size gives the same result.
cudaError_t fmm_launch_local_level(DevTree& t, DevWalk& w, DevCounters* ctr, float eps2, int level, int levels,
                                   const LocalGrids& g, cudaStream_t s)
{
    k_local_flat<0><<<g.cc, LOCAL_THREADS, 0, s>>>(w.cc, w.cc_sink, w.lcc_off, w.lcc_len, w.lcc_len, t.cen, t.posf,
                                                    t.plo, t.rec, t.L, w.cap_cc, eps2, t.per_ib, t.per_R, level, ctr);
    k_local_flat<1><<<g.cp, LOCAL_THREADS, 0, s>>>(w.cp, w.cp_sink, w.lcp_off, w.lcp_len, w.lcc_len, t.cen, t.posf,
                                                    t.plo, t.rec, t.L, w.cap_cp, eps2, t.per_ib, t.per_R, level, ctr);
    const int l0 = level < 0 ? 0 : level, l1 = level < 0 ? levels : level + 1;
    for (int l = l0; l < l1; l++)
        k_local_down<<<g.down, LD_THREADS, 0, s>>>(l, w.wcells, w.cap_front, t.cparent, w.lcc_len, w.lcp_len, t.com,
                                                   t.L, ctr);
    return cudaGetLastError();
}

// Grid sizes for a level with about n_cc / n_cp local entries and n_cells walked cells (counts of
// the context's previous walk; negative: unknown, the full persistent grids).  Never below two
// blocks per SM: counts that changed since cost a level at most a few-fold, not its parallelism.
LocalGrids fmm_local_grids(const DevWalk& w, long long n_cc, long long n_cp, long long n_cells)
{
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long full = w.n_warps / LOCAL_WPB, full_down = (long long)sms * 8, floor = 2LL * sms;
    auto flat = [&](long long e) {
        if (e < 0) return (unsigned)full;
        // a quarter more warps than ranges
        const long long warps = fmm_ceil_div(e, LF_ENTRIES) * 5 / 4 + 1;
        return (unsigned)std::max(std::min(floor, full), std::min(full, fmm_ceil_div(warps, LOCAL_WPB)));
    };
    LocalGrids g;
    g.cc = flat(n_cc);
    g.cp = flat(n_cp);
    g.down = n_cells < 0 ? (unsigned)full_down
                         : (unsigned)std::max(std::min(floor, full_down),
                                              std::min(full_down, fmm_ceil_div(n_cells * 5 / 4 + 1, LD_THREADS)));
    return g;
}

cudaError_t fmm_launch_local_groups(DevWalk& w, DevTree& t, DevCounters* ctr, cudaStream_t s)
{
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_local_groups<<<(unsigned)(sms * 8), 256, 0, s>>>(w.groups, t.L, w.Lg, w.cap_groups, ctr);
    return cudaGetLastError();
}
