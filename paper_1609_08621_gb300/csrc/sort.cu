// Device-wide exclusive scan and stable LSD radix sort of (63-bit Morton key, index) pairs.
//
// The sort produces the "hierarchically sorted order" of the particles (Sec. 3.1):
// particles ordered by Morton key, ties kept in input order (the sort is stable and
// starts from the identity permutation).  8 passes of 8-bit digits; each pass is a
// per-tile digit histogram, an exclusive scan of the (digit, tile) counts in
// digit-major order, and a stable scatter that ranks keys within the tile with
// warp match masks and stages the tile in shared memory so that global writes are
// runs of equal digits.
#include "fmm_internal.cuh"

#define SCAN_THREADS 1024
#define SCAN_ITEMS 4
#define SCAN_TILE (SCAN_THREADS * SCAN_ITEMS)

#define RS_THREADS 256
#define RS_WARPS (RS_THREADS / 32)
#define RS_ITEMS 16
#define RS_TILE (RS_THREADS * RS_ITEMS)

// inclusive block scan of one value per thread (blockDim.x multiple of 32, <= 1024)
__device__ __forceinline__ unsigned int block_inclusive_scan(unsigned int v, unsigned int* sh /* 32 */,
                                                             unsigned int* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned int t = __shfl_up_sync(FMM_FULL_MASK, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        unsigned int s = lane < nw ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned int t = __shfl_up_sync(FMM_FULL_MASK, s, o);
            if (lane >= o) s += t;
        }
        sh[lane] = s;
    }
    __syncthreads();
    unsigned int add = w > 0 ? sh[w - 1] : 0u;
    if (total) *total = sh[nw - 1];
    __syncthreads();
    return v + add;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const unsigned int* __restrict__ in, long long n,
                                                              unsigned int* __restrict__ part)
{
    __shared__ unsigned int sh[32];
    long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    unsigned int s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++)
        if (base + i < n) s += in[base + i];
    unsigned int tot;
    block_inclusive_scan(s, sh, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// exclusive scan of the per-tile sums in place, one block, any length
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_parts(unsigned int* __restrict__ part, long long np,
                                                             unsigned int* __restrict__ total)
{
    __shared__ unsigned int sh[32];
    long long per = fmm_ceil_div(np, SCAN_THREADS);
    long long b = (long long)threadIdx.x * per, e = b + per < np ? b + per : np;
    unsigned int s = 0;
    for (long long i = b; i < e; i++) s += part[i];
    unsigned int tot;
    unsigned int incl = block_inclusive_scan(s, sh, &tot);
    unsigned int run = incl - s;
    for (long long i = b; i < e; i++) {
        unsigned int v = part[i];
        part[i] = run;
        run += v;
    }
    if (threadIdx.x == 0 && total) *total = tot;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const unsigned int* __restrict__ in,
                                                            unsigned int* __restrict__ out, long long n,
                                                            const unsigned int* __restrict__ part)
{
    __shared__ unsigned int sh[32];
    long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    unsigned int v[SCAN_ITEMS];
    unsigned int s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        v[i] = base + i < n ? in[base + i] : 0u;
        s += v[i];
    }
    unsigned int incl = block_inclusive_scan(s, sh, nullptr);
    unsigned int run = incl - s + part[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

static cudaError_t ensure_u32(unsigned int** p, long long* cap, long long need)
{
    if (need <= *cap) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(p, (size_t)need * sizeof(unsigned int));
    if (e == cudaSuccess) *cap = need;
    return e;
}

// scratch of fmm_scan_exclusive for scans of up to n values, allocated ahead (graph capture)
cudaError_t fmm_scan_reserve(DevTree& t, long long n)
{
    return ensure_u32(&t.scan_part, &t.cap_scan_part, fmm_ceil_div(n, SCAN_TILE));
}

cudaError_t fmm_scan_exclusive(const unsigned int* in, unsigned int* out, long long n, unsigned int* total_dev,
                               DevTree& t, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long nb = fmm_ceil_div(n, SCAN_TILE);
    cudaError_t e = ensure_u32(&t.scan_part, &t.cap_scan_part, nb);
    if (e != cudaSuccess) return e;
    k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, t.scan_part);
    k_scan_parts<<<1, SCAN_THREADS, 0, s>>>(t.scan_part, nb, total_dev);
    k_scan_down<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, t.scan_part);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- radix sort

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const unsigned long long* __restrict__ kin, long long n,
                                                        int shift, unsigned int* __restrict__ hist, int nblk)
{
    __shared__ unsigned int c[RS_WARPS * 256];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    for (int i = tid; i < RS_WARPS * 256; i += RS_THREADS) c[i] = 0;
    __syncthreads();
    const long long t0 = (long long)blockIdx.x * RS_TILE + (long long)w * 32 * RS_ITEMS;
    const unsigned int lt = fmm_lanemask_lt();
#pragma unroll 4
    for (int r = 0; r < RS_ITEMS; r++) {
        long long i = t0 + r * 32 + lane;
        bool ok = i < n;
        unsigned int d = ok ? (unsigned int)((kin[i] >> shift) & 255u) : 256u;
        unsigned int peers = __match_any_sync(FMM_FULL_MASK, d);
        if (ok && (peers & lt) == 0) c[w * 256 + d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    unsigned int s = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ww++) s += c[ww * 256 + tid];
    hist[(long long)tid * nblk + blockIdx.x] = s;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const unsigned long long* __restrict__ kin,
                                                           const unsigned int* __restrict__ vin,
                                                           unsigned long long* __restrict__ kout,
                                                           unsigned int* __restrict__ vout, long long n, int shift,
                                                           const unsigned int* __restrict__ offs, int nblk)
{
    extern __shared__ __align__(16) unsigned char rs_smem[];
    unsigned long long* sk = reinterpret_cast<unsigned long long*>(rs_smem);
    unsigned int* sv = reinterpret_cast<unsigned int*>(sk + RS_TILE);
    unsigned int* wcnt = sv + RS_TILE;          // RS_WARPS * 256
    unsigned int* dstart = wcnt + RS_WARPS * 256;  // 256
    unsigned int* gbase = dstart + 256;         // 256
    unsigned int* sh = gbase + 256;             // 32
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const long long tile0 = (long long)blockIdx.x * RS_TILE;
    for (int i = tid; i < RS_WARPS * 256; i += RS_THREADS) wcnt[i] = 0;
    gbase[tid] = offs[(long long)tid * nblk + blockIdx.x];
    __syncthreads();
    unsigned long long k[RS_ITEMS];
    unsigned int v[RS_ITEMS], lp[RS_ITEMS];
    const unsigned int lt = fmm_lanemask_lt();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        long long i = tile0 + (long long)w * 32 * RS_ITEMS + r * 32 + lane;
        bool ok = i < n;
        k[r] = ok ? kin[i] : 0ull;
        v[r] = ok ? vin[i] : 0u;
        unsigned int d = ok ? (unsigned int)((k[r] >> shift) & 255u) : 256u;
        unsigned int peers = __match_any_sync(FMM_FULL_MASK, d);
        unsigned int rank = __popc(peers & lt);
        unsigned int before = ok ? wcnt[w * 256 + d] : 0u;
        __syncwarp();
        if (ok && rank == 0) wcnt[w * 256 + d] = before + __popc(peers);
        __syncwarp();
        lp[r] = before + rank;
    }
    __syncthreads();
    // per digit: exclusive scan over warps; block total
    unsigned int run = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ww++) {
        unsigned int c = wcnt[ww * 256 + tid];
        wcnt[ww * 256 + tid] = run;
        run += c;
    }
    unsigned int incl = block_inclusive_scan(run, sh, nullptr);
    dstart[tid] = incl - run;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        long long i = tile0 + (long long)w * 32 * RS_ITEMS + r * 32 + lane;
        if (i < n) {
            unsigned int d = (unsigned int)((k[r] >> shift) & 255u);
            unsigned int pos = dstart[d] + wcnt[w * 256 + d] + lp[r];
            sk[pos] = k[r];
            sv[pos] = v[r];
        }
    }
    __syncthreads();
    long long rem = n - tile0;
    int cnt = rem < RS_TILE ? (int)rem : RS_TILE;
    for (int i = tid; i < cnt; i += RS_THREADS) {
        unsigned long long kk = sk[i];
        unsigned int d = (unsigned int)((kk >> shift) & 255u);
        unsigned long long g = (unsigned long long)gbase[d] + (unsigned long long)(i - (int)dstart[d]);
        kout[g] = kk;
        vout[g] = sv[i];
    }
}

static size_t rs_smem_bytes()
{
    return (size_t)RS_TILE * 8 + (size_t)RS_TILE * 4 + (RS_WARPS * 256 + 256 + 256 + 32) * 4;
}

// Lets the scatter kernel use its shared-memory tile on the current device.
static std::atomic<unsigned long long> g_rs_attr{0};
cudaError_t fmm_sort_prepare() { return fmm_smem_attr_once(k_rs_scatter, (int)rs_smem_bytes(), g_rs_attr); }

cudaError_t fmm_sort_ensure(DevTree& t, long long n)
{
    long long nblk = fmm_ceil_div(n, RS_TILE);
    cudaError_t e = ensure_u32(&t.hist, &t.cap_hist, 256 * nblk);
    if (e != cudaSuccess) return e;
    return fmm_sort_prepare();
}

// Stable LSD sort of n (key, value) pairs on the low 8 * passes key bits (passes even): the
// result is back in ka / va; kb / vb are scratch of the same size.
cudaError_t fmm_radix_sort_kv(unsigned long long* ka, unsigned long long* kb, unsigned int* va, unsigned int* vb,
                              long long n, int passes, DevTree& t, cudaStream_t s)
{
    if (n <= 1) return cudaSuccess;
    cudaError_t e = fmm_sort_ensure(t, n);
    if (e != cudaSuccess) return e;
    int nblk = (int)fmm_ceil_div(n, RS_TILE);
    for (int pass = 0; pass < passes; pass++) {
        int shift = 8 * pass;
        k_rs_hist<<<nblk, RS_THREADS, 0, s>>>(ka, n, shift, t.hist, nblk);
        e = fmm_scan_exclusive(t.hist, t.hist, 256LL * nblk, nullptr, t, s);
        if (e != cudaSuccess) return e;
        k_rs_scatter<<<nblk, RS_THREADS, rs_smem_bytes(), s>>>(ka, va, kb, vb, n, shift, t.hist, nblk);
        unsigned long long* tk = ka;
        ka = kb;
        kb = tk;
        unsigned int* tv = va;
        va = vb;
        vb = tv;
    }
    return cudaGetLastError();
}

// sorts t.key / t.idx (n elements) on all 64 key bits
cudaError_t fmm_radix_sort(DevTree& t, long long n, cudaStream_t s)
{
    return fmm_radix_sort_kv(t.key, t.key_alt, t.idx, t.idx_alt, n, 8, t, s);
}

// ---------------------------------------------------------------- sort on caller scratch

// Scratch entries the sort below needs for n keys: digit counts (256 per tile) and the partial
// sums of their scan.
long long fmm_sort_hist_entries(long long n) { return 256LL * fmm_ceil_div(n, RS_TILE); }
long long fmm_sort_part_entries(long long n) { return fmm_ceil_div(fmm_sort_hist_entries(n), SCAN_TILE); }

// Lets the scatter kernel use its shared-memory tile on the current device.

// The same stable LSD sort as fmm_radix_sort_kv, with every scratch buffer supplied by the
// caller (hist, part of the sizes above; kb, vb of n entries) and nothing allocated here.
// fmm_sort_prepare must have run on the current device.
cudaError_t fmm_radix_sort_kv_scratch(unsigned long long* ka, unsigned long long* kb, unsigned int* va,
                                      unsigned int* vb, long long n, int passes, unsigned int* hist,
                                      unsigned int* part, cudaStream_t s)
{
    if (n <= 1) return cudaSuccess;
    const int nblk = (int)fmm_ceil_div(n, RS_TILE);
    const long long nh = 256LL * nblk, nb = fmm_ceil_div(nh, SCAN_TILE);
    for (int pass = 0; pass < passes; pass++) {
        const int shift = 8 * pass;
        k_rs_hist<<<nblk, RS_THREADS, 0, s>>>(ka, n, shift, hist, nblk);
        k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(hist, nh, part);
        k_scan_parts<<<1, SCAN_THREADS, 0, s>>>(part, nb, nullptr);
        k_scan_down<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(hist, hist, nh, part);
        k_rs_scatter<<<nblk, RS_THREADS, rs_smem_bytes(), s>>>(ka, va, kb, vb, n, shift, hist, nblk);
        unsigned long long* tk = ka;
        ka = kb;
        kb = tk;
        unsigned int* tv = va;
        va = vb;
        vb = tv;
    }
    return cudaGetLastError();
}
