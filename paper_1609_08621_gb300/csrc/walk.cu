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
// (CP) terms, computed by a second kernel per level after the walk kernel of that level.
#include "expansions.cuh"
#include "fmm_internal.cuh"
#include "mlp.cuh"

#define WALK_WPB 4
#define WALK_THREADS (WALK_WPB * 32)

enum { OUT_NONE = 0, OUT_ACCEPT = 1, OUT_DEFER = 2, OUT_PC = 3, OUT_PP = 4, OUT_OPEN = 5 };

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
template <int MODE>
__global__ void __launch_bounds__(WALK_THREADS, MODE == 1 ? 4 : 6) k_walk_level(
    const WalkNode* __restrict__ node, const float4* __restrict__ posf, const int* __restrict__ cnact,
    const int* __restrict__ f_cell, const unsigned long long* __restrict__ f_cloff, const int* __restrict__ f_cllen,
    int level, const unsigned int* __restrict__ cl_cur, int* __restrict__ f_cell_next,
    unsigned long long* __restrict__ f_cloff_next, int* __restrict__ f_cllen_next, long long cap_front,
    unsigned int* __restrict__ cl_next, long long cap_cl, unsigned long long* __restrict__ lcc_off,
    int* __restrict__ lcc_len, int* __restrict__ lcells, unsigned int* __restrict__ pp, long long cap_pp,
    unsigned int* __restrict__ pc,
    long long cap_pc, unsigned int* __restrict__ cc, int* __restrict__ cc_sink, long long cap_cc,
    Group* __restrict__ groups, long long cap_groups, unsigned int* __restrict__ scratch, long long cap_scr,
    DevCounters* __restrict__ ctr, int bucket, int group, float four_eps2, const float4* __restrict__ mnorm,
    const float* __restrict__ amin,
    float eps, float band_lo, float band_hi, float tau, const unsigned char* __restrict__ mlp_packed,
    int2* __restrict__ audit_pairs, long long audit_cap, const unsigned char* __restrict__ nogroup)
{
    extern __shared__ __align__(16) unsigned char walk_smem[];
    if (MODE == 1) {
        mlp_load_smem(mlp_packed, walk_smem);
        __syncthreads();
    }
    unsigned char* mlp_scratch = walk_smem + MLPP_SIZE + (threadIdx.x >> 5) * MLP_WARP_SCRATCH;
    unsigned long long n_mlp = 0;
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    unsigned int* Q = scratch + gw * 5 * cap_scr;
    unsigned int* D = Q + cap_scr;
    unsigned int* A = Q + 2 * cap_scr;
    unsigned int* P = Q + 3 * cap_scr;
    unsigned int* C = Q + 4 * cap_scr;
    const unsigned int lt = fmm_lanemask_lt();
    const unsigned long long n_front = *(volatile unsigned long long*)&ctr->lv_front[level];

    for (;;) {
        unsigned long long fi = 0;
        if (lane == 0) fi = atomicAdd(&ctr->lv_work[level], 1ull);
        fi = __shfl_sync(FMM_FULL_MASK, fi, 0);
        if (fi >= n_front) break;
        const int k = f_cell[fi];
        const WalkNode K = node[k];
        // a group holds <= g particles; in a graded tree (dual trees) it is also no larger than the
        // fixed tree's groups around it
        const bool kg = K.d.w <= group && !(nogroup && nogroup[k]);
        const float rk = K.a.w, bk = K.b.w;
        const float ak = MODE == 1 ? amin[k] : 0.0f;
        const unsigned long long cl0 = f_cloff[fi];
        const long long ncl = f_cllen[fi];
        long long nq = 0, nd = 0, na = 0, npp = 0, npc = 0;
        int srcpp = 0;  // this lane's PP source particles
        bool overflow = false;
        long long base = 0;
        while (base < ncl + nq) {
            // entries appended while this batch runs get indices >= ncl + nq (batch start), so the
            // next batch begins right after the entries that were actually available here
            const long long avail = ncl + nq - base;
            const long long vi = base + lane;
            const bool valid = lane < avail;
            base += avail < 32 ? avail : 32;
            unsigned int e = 0;
            if (valid) e = vi < ncl ? cl_cur[cl0 + vi] : Q[vi - ncl];
            int out = OUT_NONE, nadd = 0, sfirst = 0, c0 = -1, c1 = -1, nsrc_cell = 0;
            float f[MLP_F];  // learned criterion: the pair's features (set for band pairs)
            bool sleaf = false, pointlike = false, acc = false, need = false;
            float d2 = 0.0f, ro = 0.0f;
            WalkNode S;
            if (valid) {
                float cx, cy, cz, lox, loy, loz, hix, hiy, hiz;
                if (e & FMM_PARTICLE_BIT) {
                    float4 p = posf[e & ~FMM_PARTICLE_BIT];
                    cx = lox = hix = p.x;
                    cy = loy = hiy = p.y;
                    cz = loz = hiz = p.z;
                    ro = 0.0f;
                    pointlike = true;
                } else {
                    S = node[e];
                    cx = S.a.x; cy = S.a.y; cz = S.a.z; ro = S.a.w;
                    lox = S.b.x; loy = S.b.y; loz = S.b.z;
                    hix = S.c.x; hiy = S.c.y; hiz = S.c.z;
                    pointlike = S.d.w == 1;
                    sleaf = S.d.x < 0;  // a leaf (bucket) has no children
                    c0 = S.d.x;
                    c1 = S.d.y;
                    sfirst = S.d.z;
                    nsrc_cell = S.d.w;
                    nadd = sleaf ? S.d.w : 2;
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
                    int band = mlp_band(K, S, d2, gap2, four_eps2, band_lo, band_hi, te);
                    if (MODE == 1) {
                        if (band == 3 && !(ak > 0.0f)) {
                            band = acc ? 1 : 2;  // no acceleration estimate: the fixed criterion decides
                        } else if (band == 3) {
                            mlp_pair_features(K, S, mnorm[e], ak, eps, f);
                            band = mlp_surrogate(reinterpret_cast<const float*>(walk_smem + MLPP_SUR), f, te, tau);
                        }
                        acc = band == 1;
                        need = band == 3;
                    } else if (band == 3) {
                        const unsigned long long q = atomicAdd(&ctr->n_audit, 1ull);
                        if ((long long)q < audit_cap) audit_pairs[q] = make_int2(k, (int)e);
                    }
                }
            }
            if (MODE == 1) {
                const unsigned int nm = __ballot_sync(FMM_FULL_MASK, need);
                if (nm) {
                    if (!need) {
#pragma unroll
                        for (int q = 0; q < MLP_F; q++) f[q] = 0.0f;
                    }
                    const float pred = mlp_predict_warp(walk_smem, mlp_scratch, f, lane, nm);
                    if (need) acc = pred < tau;
                    n_mlp += __popc(nm);
                }
            }
            if (valid) {
                if (acc) {
                    out = OUT_ACCEPT;
                } else if (!kg) {
                    out = (pointlike || ro <= rk) ? OUT_DEFER : OUT_OPEN;
                } else if (pointlike) {
                    out = OUT_PP;
                } else {
                    const float u = __fadd_rn(ro, bk);
                    if (d2 > __fmul_rn(u, u)) out = OUT_PC;
                    else out = sleaf ? OUT_PP : OUT_OPEN;
                }
                if (out != OUT_OPEN) nadd = 0;
            }
            const unsigned int mA = __ballot_sync(FMM_FULL_MASK, out == OUT_ACCEPT);
            const unsigned int mD = __ballot_sync(FMM_FULL_MASK, out == OUT_DEFER);
            const unsigned int mC = __ballot_sync(FMM_FULL_MASK, out == OUT_PC);
            const unsigned int mP = __ballot_sync(FMM_FULL_MASK, out == OUT_PP);
            int incl = nadd;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(FMM_FULL_MASK, incl, o);
                if (lane >= o) incl += t;
            }
            const int tot = __shfl_sync(FMM_FULL_MASK, incl, 31);
            if (na + __popc(mA) > cap_scr || nd + __popc(mD) > cap_scr || npc + __popc(mC) > cap_scr ||
                npp + __popc(mP) > cap_scr || nq + tot > cap_scr) {
                overflow = true;
                break;
            }
            if (out == OUT_ACCEPT) A[na + __popc(mA & lt)] = e;
            if (out == OUT_DEFER) D[nd + __popc(mD & lt)] = e;
            if (out == OUT_PC) C[npc + __popc(mC & lt)] = e;
            if (out == OUT_PP) {
                P[npp + __popc(mP & lt)] = e;
                srcpp += (e & FMM_PARTICLE_BIT) ? 1 : nsrc_cell;
            }
            if (out == OUT_OPEN) {
                long long pos = nq + incl - nadd;
                if (sleaf) {
                    for (int j = 0; j < nadd; j++) Q[pos + j] = (unsigned int)(sfirst + j) | FMM_PARTICLE_BIT;
                } else {
                    Q[pos] = (unsigned int)c0;
                    Q[pos + 1] = (unsigned int)c1;
                }
            }
            na += __popc(mA);
            nd += __popc(mD);
            npc += __popc(mC);
            npp += __popc(mP);
            nq += tot;
            __syncwarp();
        }
        if (overflow) {
            if (lane == 0) atomicOr(&ctr->overflow, 1u);
            continue;
        }
        if (lane == 0) {
            atomicAdd(&ctr->lv_entries[level], (unsigned long long)(ncl + nq));
            atomicMax(&ctr->lv_max_entries[level], (unsigned long long)(ncl + nq));
        }
        __syncwarp();
        // local-expansion entries of this sink
        unsigned long long off = 0;
        if (lane == 0) off = atomicAdd(&ctr->cc_len, (unsigned long long)na);
        off = __shfl_sync(FMM_FULL_MASK, off, 0);
        if ((long long)(off + na) > cap_cc) {
            if (lane == 0) atomicOr(&ctr->overflow, 1u);
            continue;
        }
        for (long long i = lane; i < na; i += 32) {
            cc[off + i] = A[i];
            cc_sink[off + i] = k;
        }
        if (lane == 0) {
            lcc_off[k] = off;
            lcc_len[k] = (int)na;
            if (na > 0) lcells[atomicAdd(&ctr->n_lcells, 1ull)] = k;
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
// from posf (hi, and its mass) and plo (lo).
__device__ __forceinline__ void local_entry(unsigned int e, const float4& hk, const float4& lk,
                                            const int* __restrict__ ccount, const float4* __restrict__ cen,
                                            const float4* __restrict__ posf, const float4* __restrict__ plo,
                                            const float* __restrict__ rec, float eps2, float* acc, int& ncc, int& ncp)
{
    if (e & FMM_PARTICLE_BIT) {
        const unsigned int j = e & ~FMM_PARTICLE_BIT;
        const float4 hs = posf[j], ls = plo[j];
        fmm_p2l_acc(hs.w, cen_diff(hk.x, lk.x, hs.x, ls.x), cen_diff(hk.y, lk.y, hs.y, ls.y),
                    cen_diff(hk.z, lk.z, hs.z, ls.z), eps2, acc);
        ncp++;
    } else if (ccount[e] == 1) {  // a one-particle cell: its particle (mass = moment M[0]) -> local expansion
        const float4 hs = cen[2 * e], ls = cen[2 * e + 1];
        fmm_p2l_acc(rec[(long long)e * FMM_NREC], cen_diff(hk.x, lk.x, hs.x, ls.x), cen_diff(hk.y, lk.y, hs.y, ls.y),
                    cen_diff(hk.z, lk.z, hs.z, ls.z), eps2, acc);
        ncp++;
    } else {
        const float4 hs = cen[2 * e], ls = cen[2 * e + 1];
        float M[FMM_NMOM];
        const float4* r4 = reinterpret_cast<const float4*>(rec + (long long)e * FMM_NREC);
#pragma unroll
        for (int q = 0; q < FMM_NMOM / 4; q++) {
            const float4 v = r4[q];
            M[4 * q] = v.x;
            M[4 * q + 1] = v.y;
            M[4 * q + 2] = v.z;
            M[4 * q + 3] = v.w;
        }
        fmm_m2l_acc(M, cen_diff(hk.x, lk.x, hs.x, ls.x), cen_diff(hk.y, lk.y, hs.y, ls.y),
                    cen_diff(hk.z, lk.z, hs.z, ls.z), eps2, acc);
        ncc++;
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

__global__ void __launch_bounds__(LOCAL_THREADS) k_local_flat(
    const unsigned int* __restrict__ cc, const int* __restrict__ cc_sink, const unsigned long long* __restrict__ lcc_off,
    const int* __restrict__ lcc_len, const int* __restrict__ ccount, const float4* __restrict__ cen,
    const float4* __restrict__ posf, const float4* __restrict__ plo,
    const float* __restrict__ rec, float* __restrict__ Lown, long long cap_cc,
    float eps2, DevCounters* __restrict__ ctr)
{
    __shared__ float red[LOCAL_WPB][32][FMM_NL + 1];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long total = min((long long)*(volatile unsigned long long*)&ctr->cc_len, cap_cc);
    const long long nranges = fmm_ceil_div(total, LF_ENTRIES);
    const int c0 = lane, c1 = lane + 32;  // this lane's coefficients in the reduction
    int ncc = 0, ncp = 0;
    for (long long r = gw; r < nranges; r += nw) {
        const long long r0 = local_boundary(r * LF_ENTRIES, total, cc_sink, lcc_off, lcc_len);
        const long long r1 = local_boundary((r + 1) * LF_ENTRIES, total, cc_sink, lcc_off, lcc_len);
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
                local_entry(cc[idx], cen[2 * sink], cen[2 * sink + 1], ccount, cen, posf, plo, rec, eps2, acc, ncc, ncp);
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
                dst[c0] = sum0;
                if (c1 < FMM_NL) dst[c1] = sum1;
            }
            __syncwarp();
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ncc += __shfl_xor_sync(FMM_FULL_MASK, ncc, o);
        ncp += __shfl_xor_sync(FMM_FULL_MASK, ncp, o);
    }
    if (lane == 0) {
        if (ncc) atomicAdd(&ctr->n_cc, (unsigned long long)ncc);
        if (ncp) atomicAdd(&ctr->n_cp, (unsigned long long)ncp);
    }
}

// Local expansion of each group about its centre of mass: the own expansions of the group and
// of all its ancestors, each re-expanded (L2L) at the group's centre.  A local expansion is a
// polynomial of degree 5, so one re-expansion from an ancestor equals the chain of L2L steps
// down the tree.  One warp per group, lanes take ancestors.
#define LG_MAX_ANC FMM_MAX_LEVELS
__global__ void __launch_bounds__(LOCAL_THREADS) k_local_groups(
    const Group* __restrict__ groups, const int* __restrict__ cparent, const int* __restrict__ lcc_len,
    const Com4* __restrict__ com, const float* __restrict__ Lown, float* __restrict__ Lg,
    DevCounters* __restrict__ ctr)
{
    __shared__ float red[LOCAL_WPB][32][FMM_NL + 1];
    __shared__ int anc[LOCAL_WPB][LG_MAX_ANC];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long ng = (long long)*(volatile unsigned long long*)&ctr->n_groups;
    for (long long gi = gw; gi < ng; gi += nw) {
        const int g = groups[gi].cell;
        int na = 0;
        if (lane == 0) {
            for (int a = g; a >= 0 && na < LG_MAX_ANC; a = cparent[a])
                if (lcc_len[a] > 0) anc[wl][na++] = a;
        }
        na = __shfl_sync(FMM_FULL_MASK, na, 0);
        __syncwarp();
        const Com4 cg = com[g];
        float acc[FMM_NL];
#pragma unroll
        for (int i = 0; i < FMM_NL; i++) acc[i] = 0.0f;
        for (int i = lane; i < na; i += 32) {
            const int a = anc[wl][i];
            const float* La = Lown + (long long)a * FMM_NL;
            if (a == g) {
#pragma unroll
                for (int q = 0; q < FMM_NL; q++) acc[q] += La[q];
            } else {
                const Com4 ca = com[a];
                float Lo[FMM_NL];
                fmm_l2l(La, __double2float_rn(cg.x - ca.x), __double2float_rn(cg.y - ca.y),
                        __double2float_rn(cg.z - ca.z), Lo);
#pragma unroll
                for (int q = 0; q < FMM_NL; q++) acc[q] += Lo[q];
            }
        }
#pragma unroll
        for (int i = 0; i < FMM_NL; i++) red[wl][lane][i] = acc[i];
        __syncwarp();
        float* out = Lg + gi * FMM_NL;
        for (int c = lane; c < FMM_NL; c += 32) {
            float sum = 0.0f;
            for (int r = 0; r < 32; r++) sum += red[wl][r][c];
            out[c] = sum;
        }
        __syncwarp();
    }
}

// level 0 of the walk: every box's root cell as a sink, with that root alone on its checklist
// (isolated boxes: sources of other boxes are never seen); boxes without an active particle
// are not walked
// Each box's root starts the walk with itself on its checklist.  With one box and second_root >= 0
// (the root of an appended fixed tree, dual.cu) the checklist holds both roots.
__global__ void k_walk_seed(int* f_cell, unsigned long long* f_cloff, int* f_cllen, unsigned int* cl,
                            const int* __restrict__ cnact, const int* __restrict__ box_root, int nbox,
                            int second_root, DevCounters* ctr)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const int r = box_root ? box_root[b] : 0;
    if (r < 0 || cnact[r] <= 0) return;  // an empty box has no root cell
    const unsigned long long k = atomicAdd(&ctr->lv_front[0], 1ull);
    f_cell[k] = r;
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
    k_walk_seed<<<(unsigned)fmm_ceil_div(t.nbox, 128), 128, 0, s>>>(w.f_cell[0], w.f_cloff[0], w.f_cllen[0], w.cl[0],
                                                                     t.cnact, t.nbox > 1 ? t.box_root : nullptr,
                                                                     t.nbox, second_root, ctr);
    return cudaGetLastError();
}

int fmm_walk_warps(int device)
{
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms * 24;  // 6 resident blocks of 4 warps per SM
}

cudaError_t fmm_launch_walk_level(DevTree& t, DevWalk& w, DevCounters* ctr, const WalkArgs& a, cudaStream_t s)
{
    const int cur = a.level_parity, nxt = cur ^ 1;
    // persistent grid: every warp owns a scratch slot; idle warps exit after one atomic
    const int blocks = w.n_warps / WALK_WPB;
#define WALK_ARGS                                                                                                   \
    t.node, t.posf, t.cnact, w.f_cell[cur], w.f_cloff[cur], w.f_cllen[cur], a.level, w.cl[cur], w.f_cell[nxt],      \
        w.f_cloff[nxt], w.f_cllen[nxt], w.cap_front, w.cl[nxt], w.cap_cl, w.lcc_off, w.lcc_len, w.lcells, w.pp,     \
        w.cap_pp, w.pc, w.cap_pc, w.cc, w.cc_sink, w.cap_cc, w.groups, w.cap_groups, w.scratch, w.cap_scratch, ctr, \
        a.bucket, a.group, a.four_eps2, t.mnorm, t.amin, a.eps, a.band_lo, a.band_hi, a.tau, a.mlp_packed, a.audit_pairs,  \
        a.audit_cap, t.graded ? t.nogroup : nullptr
    if (a.mode == 1) {
        const size_t smem = MLPP_SIZE + (size_t)WALK_WPB * MLP_WARP_SCRATCH;
        static std::atomic<unsigned long long> attr{0};
        cudaError_t e = fmm_smem_attr_once(k_walk_level<1>, (int)smem, attr);
        if (e != cudaSuccess) return e;
        k_walk_level<1><<<blocks, WALK_THREADS, smem, s>>>(WALK_ARGS);
    } else if (a.mode == 2) {
        k_walk_level<2><<<blocks, WALK_THREADS, 0, s>>>(WALK_ARGS);
    } else {
        k_walk_level<0><<<blocks, WALK_THREADS, 0, s>>>(WALK_ARGS);
    }
#undef WALK_ARGS
    return cudaGetLastError();
}

cudaError_t fmm_launch_local(DevTree& t, DevWalk& w, DevCounters* ctr, float eps2, cudaStream_t s)
{
    const int blocks = w.n_warps / LOCAL_WPB;
    k_local_flat<<<blocks, LOCAL_THREADS, 0, s>>>(w.cc, w.cc_sink, w.lcc_off, w.lcc_len, t.ccount, t.cen, t.posf,
                                                   t.plo, t.rec, t.L, w.cap_cc, eps2, ctr);
    k_local_groups<<<blocks, LOCAL_THREADS, 0, s>>>(w.groups, t.cparent, w.lcc_len, t.com, t.L, w.Lg, ctr);
    return cudaGetLastError();
}
