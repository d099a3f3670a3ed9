// Tree build: Morton keys, sorted particle arrays, binary radix tree, bucket cells and the
// upward pass (Sec. 3.1).
//
// Geometry.  Level l of the tree bisects axis l mod 3 (x, y, z) of the unit box; on a cube
// this is the paper's longest-axis equal-volume bisection with ties broken x, y, z.  The
// tree is the binary radix tree of the sorted 63-bit keys (Karras 2012 construction):
// every internal node splits its range at the highest key bit in which its first and last
// keys differ (runs of identical keys split on the highest differing bit of the
// positions), so empty children never exist and one-child chains are collapsed.  Nodes
// holding <= b particles whose parent holds more become the buckets (Sec. 3.1, leaf cells
// of up to b particles); nodes below them are dropped.
//
// Upward pass.  Per cell: mass and centre of mass (FP64), bounding box (FP64),
// b_max = distance from the centre of mass to the farthest particle (Sec. 3.1), exact in
// FP64, and moments M_n = sum m y^n to order 4 about the centre of mass (FP32; Sec. 3.1
// "4th order moments").  Buckets take moments from FP64 offsets rounded to FP32; parents
// shift their children's moments (M2M).  A thread per bucket walks up with an arrival
// counter per cell; the second child to arrive computes the parent.
#include <math.h>

#include <algorithm>

#include "expansions.cuh"
#include "fmm_internal.cuh"
#include "morton.cuh"

#define TB 256

// ---------------------------------------------------------------- keys

// A position given as FP64 coordinates, or as 32-bit fixed-point ones (Sec. 3.4: x = u 2^-32, exact
// in FP64), component a of particle i of n.
__device__ __forceinline__ double pos_at(const double* __restrict__ pos, const unsigned int* __restrict__ ipos,
                                         long long n, int a, long long i)
{
    return ipos ? __dmul_rn(__uint2double_rn(ipos[a * n + i]), 0x1p-32) : pos[a * n + i];
}

__global__ void k_keys(const double* __restrict__ pos, const unsigned int* __restrict__ ipos,
                       const float* __restrict__ mass, const unsigned char* __restrict__ active, long long n,
                       unsigned long long* __restrict__ key, unsigned int* __restrict__ idx,
                       SrcRec* __restrict__ src, unsigned int* __restrict__ status)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = pos_at(pos, ipos, n, 0, i), y = pos_at(pos, ipos, n, 1, i), z = pos_at(pos, ipos, n, 2, i);
    float m = mass[i];
    SrcRec r;
    r.x = x;
    r.y = y;
    r.z = z;
    r.m = m;
    r.act = active ? (active[i] != 0 ? 1u : 0u) : 1u;
    src[i] = r;
    // 0 <= x < 1 per axis, tested on the encodings (FP64 comparisons issue at 1/64 of the FP32 rate)
    bool ok = (fmm_in_unit(x) && fmm_in_unit(y) && fmm_in_unit(z) && m > 0.0f && isfinite(m));
    if (!ok) atomicOr(status, FMM_DEV_ERR_ARG);
    // axis x owns the highest bit of each level triple: key bit 62 - l for level l
    key[i] = (spread3(quantise21(x)) << 2) | (spread3(quantise21(y)) << 1) | spread3(quantise21(z));
    idx[i] = (unsigned int)i;
}

cudaError_t fmm_launch_keys(DevTree& t, const double* pos, const float* mass, const unsigned char* active,
                            long long n, DevCounters* ctr, cudaStream_t s, const unsigned int* ipos)
{
    k_keys<<<(unsigned)fmm_ceil_div(n, TB), TB, 0, s>>>(pos, ipos, mass, active, n, t.key, t.idx, t.src,
                                                         &ctr->status);
    return cudaGetLastError();
}

__global__ void k_gather(const SrcRec* __restrict__ src, long long n, const unsigned int* __restrict__ idx,
                         double* __restrict__ sx, double* __restrict__ sy, double* __restrict__ sz,
                         float* __restrict__ sm, unsigned char* __restrict__ sact, float4* __restrict__ posf,
                         float4* __restrict__ plo, unsigned long long* __restrict__ n_active)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool act = false;
    if (i < n) {
        const SrcRec r = src[idx[i]];
        const double x = r.x, y = r.y, z = r.z;
        sx[i] = x;
        sy[i] = y;
        sz[i] = z;
        const float m = r.m;
        sm[i] = m;
        act = r.act != 0u;
        sact[i] = act ? 1 : 0;
        // (fl(x), fl(x - fl(x))) per axis, from the encodings
        float hx, hy, hz, lx, ly, lz;
        fmm_split_f32(x, hx, lx);
        fmm_split_f32(y, hy, ly);
        fmm_split_f32(z, hz, lz);
        posf[i] = make_float4(hx, hy, hz, m);
        plo[i] = make_float4(lx, ly, lz, 0.0f);
    }
    unsigned int b = __ballot_sync(FMM_FULL_MASK, act);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_active, (unsigned long long)__popc(b));
}

cudaError_t fmm_launch_gather(DevTree& t, long long n, DevCounters* ctr, cudaStream_t s)
{
    k_gather<<<(unsigned)fmm_ceil_div(n, TB), TB, 0, s>>>(t.src, n, t.idx, t.sx, t.sy, t.sz, t.sm, t.sact, t.posf,
                                                           t.plo, &ctr->n_active);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- radix tree

// length of the common prefix of the augmented keys (box, key, position); -1 outside [0, n).
// With several boxes the 8-bit box id is the most significant part, so every box is one
// subtree of the radix tree; with one box (box == NULL) it is absent.
__device__ __forceinline__ int delta(const unsigned long long* __restrict__ k, const unsigned long long* __restrict__ box,
                                     int n, int i, long long j)
{
    if (j < 0 || j >= n) return -1;
    int base = 0;
    if (box) {
        unsigned long long ba = box[i], bb = box[j];
        if (ba != bb) return __clzll(ba ^ bb) - 56;
        base = 8;
    }
    unsigned long long a = k[i], b = k[j];
    if (a != b) return base + __clzll(a ^ b);
    return base + 64 + __clz((unsigned int)(i ^ (int)j));
}

__global__ void k_radix_tree(const unsigned long long* __restrict__ key, const unsigned long long* __restrict__ box,
                             int n, int* __restrict__ ifirst,
                             int* __restrict__ ilast, int* __restrict__ ileft, int* __restrict__ iright,
                             int* __restrict__ nparent)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(key, box, n, i, i + 1) - delta(key, box, n, i, i - 1)) > 0 ? 1 : -1;
    int dmin = delta(key, box, n, i, i - d);
    long long lmax = 2;
    while (delta(key, box, n, i, i + lmax * d) > dmin) lmax <<= 1;
    long long l = 0;
    for (long long t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(key, box, n, i, i + (l + t) * d) > dmin) l += t;
    int j = (int)(i + l * d);
    int dnode = delta(key, box, n, i, j);
    long long s = 0;
    for (long long div = 2;; div <<= 1) {
        long long t = (l + div - 1) / div;
        if (delta(key, box, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
    }
    int gamma = (int)(i + s * d + (d < 0 ? -1 : 0));
    int first = min(i, j), last = max(i, j);
    // node ids: internal g -> g, leaf p -> n - 1 + p
    int left = (first == gamma) ? (n - 1 + gamma) : gamma;
    int right = (last == gamma + 1) ? (n - 1 + gamma + 1) : gamma + 1;
    ifirst[i] = first;
    ilast[i] = last;
    ileft[i] = left;
    iright[i] = right;
    nparent[left] = i;
    nparent[right] = i;
    if (i == 0) nparent[0] = -1;
}

__device__ __forceinline__ int node_count(const int* ifirst, const int* ilast, int n, int x)
{
    return x < n - 1 ? ilast[x] - ifirst[x] + 1 : 1;
}

// first index of a sorted key array k[0, n) that is >= v
__device__ __forceinline__ long long lower_bound_u64(const unsigned long long* __restrict__ k, long long n,
                                                     unsigned long long v)
{
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (k[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Graded split flags of the radix nodes (dual trees, Sec. 3.2: the active tree takes the fixed
// tree's geometric structure).  A node splits when it holds more than b particles, or more than
// one while the fixed tree holds more than b in the node's Morton box (the dyadic box of its
// keys' common prefix); it is no group when the fixed tree holds more than g there.  So the
// active tree's leaves and groups are no larger than the fixed tree's around them.
__global__ void k_split(const int* __restrict__ ifirst, const int* __restrict__ ilast,
                        const unsigned long long* __restrict__ key, int n, int bucket, int group,
                        const unsigned long long* __restrict__ fkey, long long nf, unsigned char* __restrict__ split)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= 2 * n - 1) return;
    const int count = node_count(ifirst, ilast, n, x);
    unsigned int f = count > bucket ? 1u : 0u;
    if (count > 1 && count <= max(bucket, group)) {
        const int first = x < n - 1 ? ifirst[x] : x - (n - 1);
        const unsigned long long a = key[first], b = key[first + count - 1];
        if (a != b) {  // equal keys are one point: no finer box exists
            const int d = __clzll(a ^ b);                   // common leading bits, >= 1 (bit 63 is 0)
            const unsigned long long span = 1ull << (64 - d);  // the box holds keys [lo, lo + span)
            const unsigned long long lo = a & ~(span - 1), hi = lo + span;
            // more than k fixed keys in [lo, hi) exactly when the k-th after the first one there
            // exists and is below hi (the keys are sorted): one search instead of two
            const long long p0 = lower_bound_u64(fkey, nf, lo);
            if (p0 + bucket < nf && fkey[p0 + bucket] < hi) f |= 1u;
            if (p0 + group < nf && fkey[p0 + group] < hi) f |= 2u;
        }
    }
    split[x] = (unsigned char)f;
}

// a node's children are cells when it splits: more than b particles, or the graded flag
__device__ __forceinline__ bool node_splits(const int* ifirst, const int* ilast, int n, int bucket,
                                            const unsigned char* split, int x)
{
    return split ? (split[x] & 1u) != 0u : node_count(ifirst, ilast, n, x) > bucket;
}

__global__ void k_keep(const int* __restrict__ ifirst, const int* __restrict__ ilast, const int* __restrict__ nparent,
                       int n, int bucket, const unsigned char* __restrict__ split, unsigned int* __restrict__ keep)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= 2 * n - 1) return;
    unsigned int k;
    if (n == 1) {
        k = 1;
    } else {
        int p = nparent[x];
        k = (p < 0) ? 1u : (node_splits(ifirst, ilast, n, bucket, split, p) ? 1u : 0u);
    }
    keep[x] = k;
}

// keep[] has been turned into exclusive cell ids in place; kept marks whether node x is kept
__global__ void k_cells(const int* __restrict__ ifirst, const int* __restrict__ ilast, const int* __restrict__ ileft,
                        const int* __restrict__ iright, const int* __restrict__ nparent,
                        const unsigned int* __restrict__ cid, int n, int bucket, const unsigned char* __restrict__ split,
                        int* __restrict__ cfirst, int* __restrict__ ccount, int* __restrict__ cparent,
                        int* __restrict__ cchild, unsigned int* __restrict__ bflag, unsigned char* __restrict__ nogroup,
                        long long cap)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= 2 * n - 1) return;
    bool kept;
    if (n == 1) {
        kept = true;
    } else {
        int p = nparent[x];
        kept = (p < 0) || node_splits(ifirst, ilast, n, bucket, split, p);
    }
    if (!kept) return;
    int c = (int)cid[x];
    if ((long long)c >= cap) return;  // never taken: the host sizes the cells from the count first
    int first = x < n - 1 ? ifirst[x] : x - (n - 1);
    int count = node_count(ifirst, ilast, n, x);
    cfirst[c] = first;
    ccount[c] = count;
    int p = n == 1 ? -1 : nparent[x];
    cparent[c] = p < 0 ? -1 : (int)cid[p];
    if (split) nogroup[c] = (unsigned char)((split[x] >> 1) & 1u);
    if (node_splits(ifirst, ilast, n, bucket, split, x)) {
        const long long l = cid[ileft[x]], r = cid[iright[x]];
        cchild[2 * c] = l < cap ? (int)l : -1;
        cchild[2 * c + 1] = r < cap ? (int)r : -1;
    } else {
        cchild[2 * c] = -1;
        cchild[2 * c + 1] = -1;
        bflag[first] = 1u;
    }
}

__global__ void k_bucket_index(const unsigned int* __restrict__ bscan, const unsigned int* __restrict__ bflag_raw,
                               long long n, int* __restrict__ bucket_of)
{
    // bscan is the exclusive scan of the start flags; bucket id of particle i is the
    // number of bucket starts at or before i, minus one
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bucket_of[i] = (int)(bscan[i] + bflag_raw[i]) - 1;
}

__global__ void k_bucket_cells(const int* __restrict__ cfirst, const int* __restrict__ cchild,
                               const unsigned int* __restrict__ ncell, const int* __restrict__ bucket_of,
                               int* __restrict__ bucket_cell)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (int)*ncell) return;
    if (cchild[2 * c] < 0) bucket_cell[bucket_of[cfirst[c]]] = c;
}

cudaError_t fmm_launch_bucket_index(DevTree& t, long long n, cudaStream_t s)
{
    k_bucket_index<<<(unsigned)fmm_ceil_div(n, TB), TB, 0, s>>>(t.keep, t.bflag, n, t.bucket_of);
    return cudaGetLastError();
}

cudaError_t fmm_launch_radix_tree(DevTree& t, long long n, int bucket, cudaStream_t s)
{
    int ni = (int)n;
    if (ni > 1)
        k_radix_tree<<<(unsigned)fmm_ceil_div(ni - 1, TB), TB, 0, s>>>(t.key, t.nbox > 1 ? t.sbox : nullptr, ni,
                                                                       t.ifirst, t.ilast, t.ileft,
                                                                       t.iright, t.nparent);
    const unsigned char* split = nullptr;
    if (t.grade_key && ni > 1) {
        k_split<<<(unsigned)fmm_ceil_div(2 * ni - 1, TB), TB, 0, s>>>(t.ifirst, t.ilast, t.key, ni, bucket,
                                                                      t.grade_group, t.grade_key, t.grade_n, t.split);
        split = t.split;
    }
    k_keep<<<(unsigned)fmm_ceil_div(2 * ni - 1, TB), TB, 0, s>>>(t.ifirst, t.ilast, t.nparent, ni, bucket, split, t.keep);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- upward pass

__device__ __forceinline__ Com4 ldcg_d4(const Com4* p)
{
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = __ldcg(q), b = __ldcg(q + 1);
    return make_com4(a.x, a.y, b.x, b.y);
}

__device__ void write_record(float* __restrict__ rec, const float* M)
{
    float R[FMM_NREC];
#pragma unroll
    for (int i = 0; i < FMM_NMOM; i++) R[i] = M[i];
    fmm_moment_traces(R);
    float4* dst = reinterpret_cast<float4*>(rec);
#pragma unroll
    for (int i = 0; i < FMM_NREC / 4; i++) dst[i] = make_float4(R[4 * i], R[4 * i + 1], R[4 * i + 2], R[4 * i + 3]);
}

__device__ __forceinline__ double dist2_ordered(double dx, double dy, double dz)
{
    // ((dx*dx + dy*dy) + dz*dz), correctly rounded step by step, no fused multiply-add
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// the FP32 squared distance, in a fixed order of roundings, and the distance
__device__ __forceinline__ float bm_d2_32(const float4 v, float px, float py, float pz)
{
    const float dx = __fsub_rn(v.x, px), dy = __fsub_rn(v.y, py), dz = __fsub_rn(v.z, pz);
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}
__device__ __forceinline__ float bm_d32(const float4 v, float px, float py, float pz)
{
    return sqrtf(bm_d2_32(v, px, py, pz));
}

// The FP32 distance of a particle from an FP32-rounded centre differs from the exact one by less
// than about 1.1e-7 + 1.3e-7 d (positions in [0, 1), one subtraction and the norm), so every particle
// within twice that margin of the largest FP32 distance is a candidate for the farthest one.
__device__ __forceinline__ float bm_threshold(float top) { return top - (4e-7f + 6e-7f * top); }

#ifndef FMM_UPWARD_MINB
#define FMM_UPWARD_MINB 5  // resident blocks per SM the upward pass is compiled for (96 registers; 4: 128)
#endif
__global__ void __launch_bounds__(128, FMM_UPWARD_MINB) k_upward(const unsigned int* __restrict__ nbucket, const int* __restrict__ bucket_cell,
                                                const int* __restrict__ cfirst, const int* __restrict__ ccount,
                                                const int* __restrict__ cparent, const int* __restrict__ cchild,
                                                const double* __restrict__ sx, const double* __restrict__ sy,
                                                const double* __restrict__ sz, const float* __restrict__ sm,
                                                const unsigned char* __restrict__ sact,
                                                const float4* __restrict__ posf, Com4* com, double* clo,
                                                double* chi, double* bmax, int* cnact, float* rec,
                                                float4* __restrict__ off, unsigned int* arrive)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int)*nbucket) return;
    int c = bucket_cell[b];
    int f = cfirst[c], cnt = ccount[c];
    // FP64 issues at 1/64 of the FP32 rate here: the sums stay FP64, while the box is a minimum and
    // maximum of the positions' order keys, the widening of the mass and the rounding of the offsets
    // work on the encodings (f64bits.cuh), and the exact squared distances are evaluated only for
    // the particles that can be the farthest
    double M = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    int na = 0;
    for (int j = f; j < f + cnt; j++) {
        double m = fmm_f2d(sm[j]), x = sx[j], y = sy[j], z = sz[j];
        M += m;
        mx += m * x;
        my += m * y;
        mz += m * z;
        const unsigned long long kx = fmm_nonneg_key(x), ky = fmm_nonneg_key(y), kz = fmm_nonneg_key(z);
        lo[0] = min(lo[0], kx);
        hi[0] = max(hi[0], kx);
        lo[1] = min(lo[1], ky);
        hi[1] = max(hi[1], ky);
        lo[2] = min(lo[2], kz);
        hi[2] = max(hi[2], kz);
        na += sact[j] ? 1 : 0;
    }
    const double iM = 1.0 / M;  // one FP64 division (a software sequence on this part) instead of three
    double cx = mx * iM, cy = my * iM, cz = mz * iM;
    float Mo[FMM_NMOM];
#pragma unroll
    for (int i = 0; i < FMM_NMOM; i++) Mo[i] = 0.0f;
    // the FP32 distances from the rounded centre single out the candidates for the farthest particle
    // (the margin of the exact b_max passes below), at most 32 of them in a bit mask
    const float pcx = fmm_d2f_rn(cx), pcy = fmm_d2f_rn(cy), pcz = fmm_d2f_rn(cz);
    float m2 = 0.0f;
    for (int j = f; j < f + cnt; j++) {
        double dx = sx[j] - cx, dy = sy[j] - cy, dz = sz[j] - cz;
        float m = sm[j];
        float fx = fmm_d2f_rn(dx), fy = fmm_d2f_rn(dy), fz = fmm_d2f_rn(dz);
        fmm_p2m_acc(m, fx, fy, fz, Mo);
        off[j] = make_float4(fx, fy, fz, m);
        m2 = fmaxf(m2, bm_d2_32(posf[j], pcx, pcy, pcz));
    }
    const float thr = bm_threshold(sqrtf(m2));
    double b2 = 0.0;
    for (int j0 = f; j0 < f + cnt; j0 += 32) {
        unsigned int cand = 0u;
        for (int t = 0; t < 32 && j0 + t < f + cnt; t++)
            if (bm_d32(posf[j0 + t], pcx, pcy, pcz) >= thr) cand |= 1u << t;
        while (cand) {
            const int j = j0 + __ffs(cand) - 1;
            cand &= cand - 1;
            b2 = fmax(b2, dist2_ordered(sx[j] - cx, sy[j] - cy, sz[j] - cz));
        }
    }
    com[c] = make_com4(cx, cy, cz, M);
    for (int a = 0; a < 3; a++) {
        clo[3 * c + a] = fmm_dfrom(lo[a]);
        chi[3 * c + a] = fmm_dfrom(hi[a]);
    }
    bmax[c] = __dsqrt_rn(b2);
    cnact[c] = na;
    write_record(rec + (long long)c * FMM_NREC, Mo);
    // climb: the second child to arrive at a parent computes it
    int p = cparent[c];
    while (p >= 0) {
        __threadfence();
        unsigned int old = atomicAdd(&arrive[p], 1u);
        if (old == 0u) return;
        __threadfence();
        int c0 = cchild[2 * p], c1 = cchild[2 * p + 1];
        Com4 a0 = ldcg_d4(&com[c0]), a1 = ldcg_d4(&com[c1]);
        double Mp = a0.w + a1.w;
        const double iMp = 1.0 / Mp;
        double px = (a0.w * a0.x + a1.w * a1.x) * iMp;
        double py = (a0.w * a0.y + a1.w * a1.y) * iMp;
        double pz = (a0.w * a0.z + a1.w * a1.z) * iMp;
        float Mq[FMM_NMOM];
#pragma unroll
        for (int i = 0; i < FMM_NMOM; i++) Mq[i] = 0.0f;
        for (int h = 0; h < 2; h++) {
            int ch = h ? c1 : c0;
            Com4 ac = h ? a1 : a0;
            float Mc[FMM_NMOM];
            const float* src = rec + (long long)ch * FMM_NREC;
#pragma unroll
            for (int i = 0; i < FMM_NMOM; i++) Mc[i] = __ldcg(src + i);
            double tx = ac.x - px, ty = ac.y - py, tz = ac.z - pz;
            fmm_m2m_acc(Mc, fmm_d2f_rn(tx), fmm_d2f_rn(ty), fmm_d2f_rn(tz), Mq);
        }
        com[p] = make_com4(px, py, pz, Mp);
        for (int a = 0; a < 3; a++) {
            clo[3 * p + a] = fmm_dfrom(min(fmm_nonneg_key(__ldcg(&clo[3 * c0 + a])), fmm_nonneg_key(__ldcg(&clo[3 * c1 + a]))));
            chi[3 * p + a] = fmm_dfrom(max(fmm_nonneg_key(__ldcg(&chi[3 * c0 + a])), fmm_nonneg_key(__ldcg(&chi[3 * c1 + a]))));
        }
        cnact[p] = __ldcg(&cnact[c0]) + __ldcg(&cnact[c1]);
        write_record(rec + (long long)p * FMM_NREC, Mq);
        p = cparent[p];
    }
}

// Exact b_max of every internal cell: the distance from its centre of mass p to the farthest of
// its particles, in FP64 with the same operations as a brute-force scan (so the value is the exact
// one).  Every (cell, chunk of BM_CHUNK of its particles) pair is a work item of one warp, so big
// cells are spread over many warps and every lane does the same work.  Two passes over the items:
//   1. the largest FP32 distance d32 = |fl(x) - fl(p)| of each cell (atomic max of its bits; a cell
//      of a single item finishes step 2 at once);
//   2. the FP64 squared distance, for the particles whose d32 is within the FP32 error margin
//      4e-7 + 6e-7 d of that maximum (atomic max of the bits of the non-negative double).
// The FP32 distance of a particle differs from the exact one by less than about 1.1e-7 + 1.3e-7 d
// (positions in [0, 1) and the centre rounded to FP32, one subtraction and the norm), so the
// margin, twice the sum of two such errors, keeps the farthest particle among the candidates.
#define BM_CHUNK 2048

// items of the b_max passes: at most one partial chunk per internal cell beyond the full chunks,
// and every particle is in at most depth + 1 cells
long long fmm_bmax_items_bound(long long n, int depth, long long n_cells)
{
    return fmm_ceil_div(n * (long long)(depth + 1), BM_CHUNK) + n_cells + 1;
}

// The passes take the items ordered by the particle they start at (counted per BM_CHUNK particles,
// then placed): the warps in flight then read the same particles for the cells of every level
// around them, from L2, instead of streaming all particles once per level.  Every item keeps its
// index (its FP32 maximum is stored under it), and the maxima are order-independent.
long long fmm_bmax_bins(long long n) { return fmm_ceil_div(n, BM_CHUNK) + 1; }

__device__ __forceinline__ unsigned int bm_bin_of(long long i, const int* __restrict__ item,
                                                  const unsigned int* __restrict__ ncell,
                                                  const unsigned int* __restrict__ base, const int* __restrict__ cfirst)
{
    const int c = item[i];
    if (c < 0 || c >= (int)*ncell) return 0u;  // an item the expansion could not write: skipped by the passes
    const long long k = i - (long long)base[c];
    return (unsigned int)(((long long)cfirst[c] + k * BM_CHUNK) / BM_CHUNK);
}

__global__ void k_bm_bin_count(const int* __restrict__ item, const unsigned int* __restrict__ n_items, long long cap,
                               const unsigned int* __restrict__ ncell, const unsigned int* __restrict__ base,
                               const int* __restrict__ cfirst, unsigned int* __restrict__ bin)
{
    const long long ni = min((long long)*n_items, cap);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += (long long)gridDim.x * blockDim.x)
        atomicAdd(bin + bm_bin_of(i, item, ncell, base, cfirst), 1u);
}

__global__ void k_bm_place(const int* __restrict__ item, const unsigned int* __restrict__ n_items, long long cap,
                           const unsigned int* __restrict__ ncell, const unsigned int* __restrict__ base,
                           const int* __restrict__ cfirst, unsigned int* __restrict__ cursor,
                           unsigned int* __restrict__ order)
{
    const long long ni = min((long long)*n_items, cap);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += (long long)gridDim.x * blockDim.x)
        order[atomicAdd(cursor + bm_bin_of(i, item, ncell, base, cfirst), 1u)] = (unsigned int)i;
}

__global__ void k_bm_count(const unsigned int* __restrict__ ncell, long long grid, const int* __restrict__ ccount,
                           const int* __restrict__ cchild, unsigned int* __restrict__ cnt, unsigned int* __restrict__ bm32,
                           unsigned long long* __restrict__ bm64)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= grid) return;
    unsigned int k = 0;
    if (c < (long long)*ncell && cchild[2 * c] >= 0) k = (unsigned int)fmm_ceil_div(ccount[c], BM_CHUNK);
    cnt[c] = k;
    bm32[c] = 0u;
    bm64[c] = 0ull;
}

__global__ void k_bm_expand(long long grid, const unsigned int* __restrict__ cnt, const unsigned int* __restrict__ base,
                            int* __restrict__ item, long long cap, unsigned int* __restrict__ overflow)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= grid) return;
    const long long b = base[c], k = cnt[c];
    if (b + k > cap) {
        if (k) atomicOr(overflow, 1u);
        return;
    }
    for (long long i = 0; i < k; i++) item[b + i] = (int)c;
}

// FP64 candidates: (cell, particle) pairs whose FP32 distance reaches the cell's threshold wait in
// a per-warp buffer and are evaluated 32 at a time, one per lane.  FP64 issues at 1/64 of the FP32
// rate and a warp instruction costs the same with one active lane as with 32, so evaluating the
// few candidates of each item as they are found kept the FP64 pipe busy on mostly idle lanes.
#define BM_PEND 64
struct BmPend {
    int c[BM_PEND];
    int j[BM_PEND];
};

// the exact squared distance of each of the first cnt waiting pairs, raised into its cell's maximum
// (the bits of non-negative doubles order as unsigned integers)
__device__ __forceinline__ void bm_eval(const BmPend& B, int cnt, const Com4* __restrict__ com,
                                        const double* __restrict__ sx, const double* __restrict__ sy,
                                        const double* __restrict__ sz, unsigned long long* __restrict__ bm64, int lane)
{
    if (lane < cnt) {
        const int c = B.c[lane], j = B.j[lane];
        const Com4 p = com[c];
        const double d2 = dist2_ordered(sx[j] - p.x, sy[j] - p.y, sz[j] - p.z);
        atomicMax(bm64 + c, (unsigned long long)__double_as_longlong(d2));
    }
}

// queue the particles [j0, j1) of cell c whose FP32 distance from (px, py, pz) reaches thr;
// evaluate whenever 32 wait
__device__ __forceinline__ void bm_candidates(int c, long long j0, long long j1, float px, float py, float pz, float thr,
                                              const float4* __restrict__ posf, BmPend& B, int& npend,
                                              const Com4* __restrict__ com, const double* __restrict__ sx,
                                              const double* __restrict__ sy, const double* __restrict__ sz,
                                              unsigned long long* __restrict__ bm64, int lane)
{
    const unsigned int lt = fmm_lanemask_lt();
    for (long long jb = j0; jb < j1; jb += 32) {
        const long long j = jb + lane;
        const bool cand = j < j1 && bm_d32(posf[j], px, py, pz) >= thr;
        const unsigned int m = __ballot_sync(FMM_FULL_MASK, cand);
        if (cand) {
            const int slot = npend + __popc(m & lt);
            B.c[slot] = c;
            B.j[slot] = (int)j;
        }
        npend += __popc(m);
        __syncwarp();
        if (npend >= 32) {
            bm_eval(B, 32, com, sx, sy, sz, bm64, lane);
            const int rest = npend - 32;
            int rc = 0, rj = 0;
            if (lane < rest) {
                rc = B.c[32 + lane];
                rj = B.j[32 + lane];
            }
            __syncwarp();
            if (lane < rest) {
                B.c[lane] = rc;
                B.j[lane] = rj;
            }
            npend = rest;
            __syncwarp();
        }
    }
}


// PASS 1: per item the FP32 maximum; a cell of one item finishes at once (its FP64 candidates),
// a cell of several items records the item's maximum and raises the cell's.  PASS 2: the items of
// multi-item cells whose maximum reaches the cell's threshold look for FP64 candidates.
template <int PASS>
__global__ void __launch_bounds__(256) k_bm_pass(const unsigned int* __restrict__ order,
                                                 const int* __restrict__ item, const unsigned int* __restrict__ n_items,
                                                 long long cap, const unsigned int* __restrict__ ncell,
                                                 const unsigned int* __restrict__ cnt, const unsigned int* __restrict__ base,
                                                 const int* __restrict__ cfirst, const int* __restrict__ ccount,
                                                 const Com4* __restrict__ com, const float4* __restrict__ posf,
                                                 const double* __restrict__ sx, const double* __restrict__ sy,
                                                 const double* __restrict__ sz, unsigned int* __restrict__ bm32,
                                                 unsigned long long* __restrict__ bm64, float* __restrict__ imax)
{
    __shared__ BmPend pend[8];
    const int lane = threadIdx.x & 31;
    BmPend& B = pend[threadIdx.x >> 5];
    int npend = 0;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long ni = min((long long)*n_items, cap);
    const int nc = (int)*ncell;
    // A warp takes 32 consecutive items at a time: lane q looks up item q's cell, chunk and centre
    // (one chain of dependent loads for all 32), then the warp runs the items one by one.
    for (long long ib = gw * 32; ib < ni; ib += nw * 32) {
        const long long ii = ib + lane;
        long long i = 0, j0 = 0, j1 = 0, nk = 0;
        int c = -1;
        float px = 0.0f, py = 0.0f, pz = 0.0f, thr = 0.0f;
        bool ok = false;
        if (ii < ni) {
            i = order[ii];
            // an item the expansion could not write (capacity overflow, reported to the host) is skipped
            c = item[i];
            if (c >= 0 && c < nc) {
                const long long k = i - (long long)base[c];
                nk = cnt[c];
                ok = k >= 0 && k < nk && !(PASS == 2 && nk == 1);
                if (ok) {
                    const long long f = cfirst[c], e = f + ccount[c];
                    j0 = f + k * BM_CHUNK;
                    j1 = min(j0 + BM_CHUNK, e);
                    const Com4 p = com[c];
                    px = fmm_d2f_rn(p.x);
                    py = fmm_d2f_rn(p.y);
                    pz = fmm_d2f_rn(p.z);
                    if (PASS == 2) {
                        thr = bm_threshold(__uint_as_float(bm32[c]));
                        ok = imax[i] >= thr;  // else no particle of this item can be the farthest
                    }
                }
            }
        }
        unsigned int todo = __ballot_sync(FMM_FULL_MASK, ok);
        while (todo) {
            const int q = __ffs(todo) - 1;
            todo &= todo - 1;
            const long long iq = __shfl_sync(FMM_FULL_MASK, i, q), a0 = __shfl_sync(FMM_FULL_MASK, j0, q),
                            a1 = __shfl_sync(FMM_FULL_MASK, j1, q), nkq = __shfl_sync(FMM_FULL_MASK, nk, q);
            const int cq = __shfl_sync(FMM_FULL_MASK, c, q);
            const float qx = __shfl_sync(FMM_FULL_MASK, px, q), qy = __shfl_sync(FMM_FULL_MASK, py, q),
                        qz = __shfl_sync(FMM_FULL_MASK, pz, q);
            if (PASS == 1) {
                // the largest FP32 distance, as the square root of the largest square (the same
                // value: the square root is monotonic and correctly rounded)
                float m2 = 0.0f;
                for (long long j = a0 + lane; j < a1; j += 32) m2 = fmaxf(m2, bm_d2_32(posf[j], qx, qy, qz));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m2 = fmaxf(m2, __shfl_xor_sync(FMM_FULL_MASK, m2, o));
                const float m = sqrtf(m2);
                if (nkq == 1) {
                    bm_candidates(cq, a0, a1, qx, qy, qz, bm_threshold(m), posf, B, npend, com, sx, sy, sz, bm64,
                                  lane);
                } else if (lane == 0) {
                    imax[iq] = m;
                    atomicMax(bm32 + cq, __float_as_uint(m));
                }
            } else {
                const float tq = __shfl_sync(FMM_FULL_MASK, thr, q);
                bm_candidates(cq, a0, a1, qx, qy, qz, tq, posf, B, npend, com, sx, sy, sz, bm64, lane);
            }
        }
    }
    bm_eval(B, npend, com, sx, sy, sz, bm64, lane);
}

__global__ void k_bm_final(const unsigned int* __restrict__ ncell, const int* __restrict__ cchild,
                           const unsigned long long* __restrict__ bm64, double* __restrict__ bmax)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (int)*ncell || cchild[2 * c] < 0) return;  // buckets are exact already
    bmax[c] = __dsqrt_rn(__longlong_as_double((long long)bm64[c]));
}

cudaError_t fmm_launch_cells(DevTree& t, long long n, int bucket, cudaStream_t s)
{
    int ni = (int)n;
    const unsigned char* split = (t.grade_key && ni > 1) ? t.split : nullptr;
    k_cells<<<(unsigned)fmm_ceil_div(2 * ni - 1, TB), TB, 0, s>>>(t.ifirst, t.ilast, t.ileft, t.iright, t.nparent,
                                                                  t.keep, ni, bucket, split, t.cfirst, t.ccount,
                                                                  t.cparent, t.cchild, t.bflag, t.nogroup,
                                                                  t.cap_cells);
    return cudaGetLastError();
}

// cells and buckets covered by a launch: the counts, or the capacity under graph capture
static long long grid_cells(const DevTree& t) { return t.cap_grid ? t.cap_cells : t.n_cells; }
static long long grid_buckets(const DevTree& t) { return t.cap_grid ? t.cap_cells : t.n_buckets; }

cudaError_t fmm_launch_upward(DevTree& t, long long n, int bucket, DevCounters* ctr, cudaStream_t s)
{
    (void)bucket;
    const long long nc = grid_cells(t), nb = grid_buckets(t);
    k_bucket_cells<<<(unsigned)fmm_ceil_div(nc, TB), TB, 0, s>>>(t.cfirst, t.cchild, t.dcount, t.bucket_of,
                                                                 t.bucket_cell);
    cudaMemsetAsync(t.arrive, 0, sizeof(unsigned int) * (size_t)nc, s);
    k_upward<<<(unsigned)fmm_ceil_div(nb, 128), 128, 0, s>>>(t.dcount + 1, t.bucket_cell, t.cfirst, t.ccount,
                                                              t.cparent, t.cchild, t.sx, t.sy, t.sz, t.sm, t.sact,
                                                              t.posf, t.com, t.clo, t.chi, t.bmax, t.cnact, t.rec, t.off,
                                                              t.arrive);
    // exact b_max of the internal cells: items, then the two passes
    const unsigned gb = (unsigned)fmm_ceil_div(nc, TB);
    k_bm_count<<<gb, TB, 0, s>>>(t.dcount, nc, t.ccount, t.cchild, t.bm_cnt, t.bm32, t.bm64);
    cudaError_t e = fmm_scan_exclusive(t.bm_cnt, t.bm_base, nc, &ctr->n_bm_items, t, s);
    if (e != cudaSuccess) return e;
    k_bm_expand<<<gb, TB, 0, s>>>(nc, t.bm_cnt, t.bm_base, t.bm_item, t.cap_bm_items, &ctr->overflow);
    {
        const long long nbins = fmm_bmax_bins(n);
        const unsigned ob = (unsigned)std::max(1LL, std::min(fmm_ceil_div(t.cap_bm_items, TB), 152LL * 32));
        cudaMemsetAsync(t.bm_bin, 0, sizeof(unsigned int) * (size_t)nbins, s);
        k_bm_bin_count<<<ob, TB, 0, s>>>(t.bm_item, &ctr->n_bm_items, t.cap_bm_items, t.dcount, t.bm_base, t.cfirst,
                                          t.bm_bin);
        e = fmm_scan_exclusive(t.bm_bin, t.bm_binbase, nbins, &ctr->pad1, t, s);
        if (e != cudaSuccess) return e;
        k_bm_place<<<ob, TB, 0, s>>>(t.bm_item, &ctr->n_bm_items, t.cap_bm_items, t.dcount, t.bm_base, t.cfirst,
                                      t.bm_binbase, t.bm_order);
    }
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = fmm_ceil_div(t.cap_bm_items, 8);
    const unsigned pb = (unsigned)std::max(1LL, std::min(want, (long long)sms * 8));
    k_bm_pass<1><<<pb, 256, 0, s>>>(t.bm_order, t.bm_item, &ctr->n_bm_items, t.cap_bm_items, t.dcount, t.bm_cnt, t.bm_base,
                                    t.cfirst, t.ccount,
                                    t.com, t.posf, t.sx, t.sy, t.sz, t.bm32, t.bm64, t.bm_imax);
    k_bm_pass<2><<<pb, 256, 0, s>>>(t.bm_order, t.bm_item, &ctr->n_bm_items, t.cap_bm_items, t.dcount, t.bm_cnt, t.bm_base,
                                    t.cfirst, t.ccount,
                                    t.com, t.posf, t.sx, t.sy, t.sz, t.bm32, t.bm64, t.bm_imax);
    k_bm_final<<<gb, TB, 0, s>>>(t.dcount, t.cchild, t.bm64, t.bmax);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- walk nodes (depend on theta)

__global__ void k_nodes(const unsigned int* __restrict__ ncell, float theta, const int* __restrict__ cfirst,
                        const int* __restrict__ ccount,
                        const int* __restrict__ cchild, const Com4* __restrict__ com, const double* __restrict__ clo,
                        const double* __restrict__ chi, const double* __restrict__ bmax, const float* __restrict__ rec,
                        WalkNode* __restrict__ node, float4* __restrict__ mnorm, float4* __restrict__ cen)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (int)*ncell) return;
    Com4 cm = com[c];
    // every rounding to single precision from the encodings (f64bits.cuh), no FP64 instruction
    float bm = fmm_d2f_rn(bmax[c]);
    int cnt = ccount[c];
    float ro = (cnt == 1) ? 0.0f : __fdiv_rn(bm, theta);
    WalkNode w;
    float hx, hy, hz, lx, ly, lz;
    fmm_split_f32(cm.x, hx, lx);
    fmm_split_f32(cm.y, hy, ly);
    fmm_split_f32(cm.z, hz, lz);
    w.a = make_float4(hx, hy, hz, ro);
    cen[2 * c] = make_float4(hx, hy, hz, 0.0f);
    cen[2 * c + 1] = make_float4(lx, ly, lz, 0.0f);
    w.b = make_float4(fmm_d2f_rn(clo[3 * c]), fmm_d2f_rn(clo[3 * c + 1]), fmm_d2f_rn(clo[3 * c + 2]), bm);
    w.c = make_float4(fmm_d2f_rn(chi[3 * c]), fmm_d2f_rn(chi[3 * c + 1]), fmm_d2f_rn(chi[3 * c + 2]), 0.0f);
    w.d = make_int4(cchild[2 * c], cchild[2 * c + 1], cfirst[c], cnt);
    node[c] = w;
    // multipole norms for the learned criterion: |M2|_F / (M b^2), |M4|_F / (M b^4), both in [0, 1];
    // cells smaller than 1e-7 of the box (coincident particles) report 0
    const float mass32 = fmm_d2f_rn(cm.w);
    float4 mn = make_float4(0.0f, 0.0f, mass32, 0.0f);
    if (bm > 1e-7f && cnt > 1) {
        const float b2 = bm * bm, s2 = 1.0f / (mass32 * b2), s4 = s2 / b2;
        float n2, n4;
        fmm_moment_norms2(rec + (long long)c * FMM_NREC, s2, s4, n2, n4);
        mn.x = fminf(sqrtf(n2), 1.0f);
        mn.y = fminf(sqrtf(n4), 1.0f);
    }
    mnorm[c] = mn;
}

cudaError_t fmm_launch_nodes(DevTree& t, double theta, cudaStream_t s)
{
    const long long nc = grid_cells(t);
    k_nodes<<<(unsigned)fmm_ceil_div(nc, TB), TB, 0, s>>>(t.dcount, (float)theta, t.cfirst, t.ccount, t.cchild,
                                                          t.com, t.clo, t.chi, t.bmax, t.rec, t.node, t.mnorm,
                                                          t.cen);
    return cudaGetLastError();
}

// deepest level of any cell (the walk needs at most depth + 1 levels)
__global__ void k_depth(const unsigned int* __restrict__ ncell, const int* __restrict__ cparent,
                        DevCounters* __restrict__ ctr)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (int)*ncell) return;
    unsigned int d = 0;
    for (int p = cparent[c]; p >= 0; p = cparent[p]) d++;
    atomicMax(&ctr->depth, d);
}

// ncell_dev: device copy of the cell count (the grid covers the cell capacity)
cudaError_t fmm_launch_depth(DevTree& t, const unsigned int* ncell_dev, DevCounters* ctr, cudaStream_t s)
{
    k_depth<<<(unsigned)fmm_ceil_div(t.cap_cells, TB), TB, 0, s>>>(ncell_dev, t.cparent, ctr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- several boxes

__device__ __forceinline__ int box_of(const long long* __restrict__ off, int nbox, long long i)
{
    int lo = 0, hi = nbox - 1;  // largest b with off[b] <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// after the Morton sort: box id of every sorted particle, as the key of a second stable sort
__global__ void k_box_keys(const long long* __restrict__ off, int nbox, const unsigned int* __restrict__ idx,
                           long long n, unsigned long long* __restrict__ bkey)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bkey[i] = (unsigned long long)box_of(off, nbox, idx[i]);
}

// final order is (box, key, input index): Morton keys follow the permutation
__global__ void k_regather_keys(const unsigned long long* __restrict__ korig, const unsigned int* __restrict__ idx,
                                long long n, unsigned long long* __restrict__ key)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = korig[idx[i]];
}

// the cell spanning exactly each box's particles (the box's own root)
__global__ void k_box_roots(const unsigned int* __restrict__ ncell, const int* __restrict__ cfirst,
                            const int* __restrict__ ccount, const long long* __restrict__ off, int nbox,
                            int* __restrict__ box_root)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (int)*ncell) return;
    const long long f = cfirst[c];
    const int b = box_of(off, nbox, f);
    if (off[b] == f && off[b + 1] - f == ccount[c]) box_root[b] = c;
}

// Stable sort of all boxes' particles by (box, Morton key): Morton keys first (8 passes), then
// the box ids (2 passes); t.key_orig keeps the keys in input order.
cudaError_t fmm_launch_box_sort(DevTree& t, long long n, cudaStream_t s)
{
    cudaError_t e = cudaMemcpyAsync(t.key_orig, t.key, sizeof(unsigned long long) * (size_t)n,
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    e = fmm_radix_sort(t, n, s);
    if (e != cudaSuccess) return e;
    k_box_keys<<<(unsigned)fmm_ceil_div(n, TB), TB, 0, s>>>(t.box_off, t.nbox, t.idx, n, t.sbox);
    e = fmm_radix_sort_kv(t.sbox, t.key_alt, t.idx, t.idx_alt, n, 2, t, s);
    if (e != cudaSuccess) return e;
    k_regather_keys<<<(unsigned)fmm_ceil_div(n, TB), TB, 0, s>>>(t.key_orig, t.idx, n, t.key);
    return cudaGetLastError();
}

cudaError_t fmm_launch_box_roots(DevTree& t, cudaStream_t s)
{
    const long long nc = grid_cells(t);
    k_box_roots<<<(unsigned)fmm_ceil_div(nc, TB), TB, 0, s>>>(t.dcount, t.cfirst, t.ccount, t.box_off, t.nbox,
                                                              t.box_root);
    return cudaGetLastError();
}
