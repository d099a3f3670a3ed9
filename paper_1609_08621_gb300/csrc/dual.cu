// Dual trees for multiple time steps (Sec. 3.2, multiple time stepping with dual trees).
//
// On the substeps between two kicks of the slower rungs, only the particles of the fast rungs
// need forces.  The particles of rungs <= r_fixed are not kicked there, so their velocity is
// constant over that interval.  They are drifted to the middle of the interval and a tree of
// them, the fixed tree, is built once.  Every substep inside the interval then builds a tree of
// the active particles only and walks its sinks against both trees, so the full tree build is
// not repeated on each substep.
//
// The two trees share one geometric structure as the paper requires: both are radix trees over
// Morton keys of the same unit box, so every cell of either tree is a dyadic box of the same
// bisection (level l splits axis l mod 3).
//
// The active tree holds every particle outside the fixed set (the fast rungs) at its current
// position; its sinks are the particles active on the substep.
//
// Layout: the active tree is built as usual into cells [0, C_a), buckets [0, B_a) and sorted
// particles [0, N_a).  The fixed tree, kept in a context-owned copy, is appended after it with
// every cell, bucket and particle index offset by (C_a, B_a, N_a), so every kernel of the solve
// reads the two trees as one array space.  The walk starts from the active root with both roots
// on its checklist.
#include "expansions.cuh"
#include "fmm_internal.cuh"

#define DT 256

// flag[i] = 1 for the particles of the subset: rung[i] <= r_max when rungs are given, else
// flag_not[i] == 0 when the complement of a flag array is asked for, else every particle
__global__ void k_subset_flags(const unsigned char* __restrict__ rung, int r_max, const unsigned int* __restrict__ flag_not,
                               long long n, unsigned int* __restrict__ flag)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned int f = 1u;
    if (rung) f = (int)rung[i] <= r_max ? 1u : 0u;
    else if (flag_not) f = flag_not[i] ? 0u : 1u;
    flag[i] = f;
}

// Compact the flagged particles (exclusive scan `at`) into SoA arrays of length m, drifting each
// position by vel * dt in double precision (x + v dt, rounded once per operation, no fused
// multiply-add); idx maps a subset slot back to the caller's index, and a byte mask (the sinks),
// when given, is compacted alongside.
__global__ void k_subset_gather(const unsigned int* __restrict__ flag, const unsigned int* __restrict__ at,
                                long long n, const double* __restrict__ pos, const double* __restrict__ vel, double dt,
                                const float* __restrict__ mass, const unsigned char* __restrict__ mask, long long m,
                                double* __restrict__ pos_out, float* __restrict__ mass_out,
                                unsigned char* __restrict__ mask_out, unsigned int* __restrict__ idx)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    const long long j = at[i];
    if (j >= m) return;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        double x = pos[d * n + i];
        if (vel) x = __dadd_rn(x, __dmul_rn(vel[d * n + i], dt));
        pos_out[d * m + j] = x;
    }
    mass_out[j] = mass[i];
    if (mask) mask_out[j] = mask[i];
    idx[j] = (unsigned int)i;
}

// Fixed-tree cells after the active tree's: first particle, children and parent move by
// (n_a, c_a); a fixed cell holds no sink (active count 0).
__global__ void k_append_cells(long long cf, int ca, int na, const int* __restrict__ f_cfirst,
                               const int* __restrict__ f_cchild, const int* __restrict__ f_cparent,
                               int* __restrict__ cfirst, int* __restrict__ cchild, int* __restrict__ cparent,
                               int* __restrict__ cnact)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cf) return;
    const long long d = ca + c;
    cfirst[d] = f_cfirst[c] + na;
    const int k0 = f_cchild[2 * c], k1 = f_cchild[2 * c + 1];
    cchild[2 * d] = k0 >= 0 ? k0 + ca : k0;
    cchild[2 * d + 1] = k1 >= 0 ? k1 + ca : k1;
    const int p = f_cparent[c];
    cparent[d] = p >= 0 ? p + ca : -1;
    cnact[d] = 0;
}

// Fixed-tree buckets (their cells move by c_a) and particles (their buckets move by b_a; none is
// a sink).
__global__ void k_append_buckets(long long bf, int ba, int ca, const int* __restrict__ f_bucket_cell,
                                 int* __restrict__ bucket_cell)
{
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= bf) return;
    bucket_cell[ba + b] = f_bucket_cell[b] + ca;
}

__global__ void k_append_particles(long long nf, int na, int ba, const int* __restrict__ f_bucket_of,
                                   int* __restrict__ bucket_of, unsigned char* __restrict__ sact)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nf) return;
    bucket_of[na + p] = f_bucket_of[p] + ba;
    sact[na + p] = 0;
}

// out[s] = sub[perm[s]]: a sorted active particle's index in the caller's arrays
__global__ void k_compose_perm(const unsigned int* __restrict__ perm, const unsigned int* __restrict__ sub,
                               long long n, unsigned int* __restrict__ out)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    out[s] = sub[perm[s]];
}

cudaError_t fmm_launch_subset_flags(const unsigned char* rung, int r_max, const unsigned int* flag_not, long long n,
                                    unsigned int* flag, cudaStream_t s)
{
    k_subset_flags<<<(unsigned)fmm_ceil_div(n, DT), DT, 0, s>>>(rung, r_max, flag_not, n, flag);
    return cudaGetLastError();
}

cudaError_t fmm_launch_subset_gather(const unsigned int* flag, const unsigned int* at, long long n, const double* pos,
                                     const double* vel, double dt, const float* mass, const unsigned char* mask,
                                     long long m, double* pos_out, float* mass_out, unsigned char* mask_out,
                                     unsigned int* idx, cudaStream_t s)
{
    k_subset_gather<<<(unsigned)fmm_ceil_div(n, DT), DT, 0, s>>>(flag, at, n, pos, vel, dt, mass, mask, m, pos_out,
                                                                 mass_out, mask_out, idx);
    return cudaGetLastError();
}

static cudaError_t copy_at(void* dst, const void* src, size_t bytes, cudaStream_t s)
{
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s) : cudaSuccess;
}

cudaError_t fmm_append_fixed(DevTree& t, const FixedTree& f, long long na, long long ca, long long ba, cudaStream_t s)
{
    const long long cf = f.n_cells, bf = f.n_buckets, nf = f.n;
    cudaError_t e = cudaSuccess;
    if (cf > 0)
        k_append_cells<<<(unsigned)fmm_ceil_div(cf, DT), DT, 0, s>>>(cf, (int)ca, (int)na, f.cfirst, f.cchild, f.cparent,
                                                                     t.cfirst, t.cchild, t.cparent, t.cnact);
    if (bf > 0)
        k_append_buckets<<<(unsigned)fmm_ceil_div(bf, DT), DT, 0, s>>>(bf, (int)ba, (int)ca, f.bucket_cell,
                                                                       t.bucket_cell);
    if (nf > 0)
        k_append_particles<<<(unsigned)fmm_ceil_div(nf, DT), DT, 0, s>>>(nf, (int)na, (int)ba, f.bucket_of,
                                                                         t.bucket_of, t.sact);
    e = cudaGetLastError();
    // arrays without indices are copied as they are
    if (e == cudaSuccess) e = copy_at(t.ccount + ca, f.ccount, sizeof(int) * cf, s);
    if (e == cudaSuccess) e = copy_at(t.com + ca, f.com, sizeof(Com4) * cf, s);
    if (e == cudaSuccess) e = copy_at(t.clo + 3 * ca, f.clo, sizeof(double) * 3 * cf, s);
    if (e == cudaSuccess) e = copy_at(t.chi + 3 * ca, f.chi, sizeof(double) * 3 * cf, s);
    if (e == cudaSuccess) e = copy_at(t.bmax + ca, f.bmax, sizeof(double) * cf, s);
    if (e == cudaSuccess) e = copy_at(t.rec + (long long)FMM_NREC * ca, f.rec, sizeof(float) * FMM_NREC * cf, s);
    if (e == cudaSuccess) e = copy_at(t.posf + na, f.posf, sizeof(float4) * nf, s);
    if (e == cudaSuccess) e = copy_at(t.plo + na, f.plo, sizeof(float4) * nf, s);
    if (e == cudaSuccess) e = copy_at(t.off + na, f.off, sizeof(float4) * nf, s);
    return e;
}

cudaError_t fmm_launch_compose_perm(const unsigned int* perm, const unsigned int* sub, long long n, unsigned int* out,
                                    cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_compose_perm<<<(unsigned)fmm_ceil_div(n, DT), DT, 0, s>>>(perm, sub, n, out);
    return cudaGetLastError();
}
