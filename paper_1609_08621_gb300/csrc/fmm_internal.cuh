// Internal definitions shared by the CUDA translation units of the FMM library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "fmm.h"

#define FMM_FULL_MASK 0xffffffffu
#define FMM_PARTICLE_BIT 0x80000000u  // checklist / list entry is a particle index

// device status word bits
#define FMM_DEV_ERR_ARG 1u        // invalid position or mass seen by a kernel
#define FMM_DEV_ERR_TIMEOUT 4u    // a bounded wait gave up
#define FMM_DEV_ERR_NUMERIC 8u    // non-finite output

// Centre of mass (x, y, z) and mass (w) of a cell, double precision, one 32-byte load.
struct __align__(32) Com4 {
    double x, y, z, w;
};
__host__ __device__ __forceinline__ Com4 make_com4(double x, double y, double z, double w)
{
    Com4 r;
    r.x = x;
    r.y = y;
    r.z = z;
    r.w = w;
    return r;
}

// One tree cell as the walk reads it: 64 bytes, four aligned 16-byte loads.
//   a = (centre of mass, single precision, and R_O = b_max / theta)
//   b = (bounding box lo, single precision, and b_max)
//   c = (bounding box hi, single precision, and unused)
//   d = (child0, child1, first, count); child0 = -1 for a bucket
struct __align__(16) WalkNode {
    float4 a, b, c;
    int4 d;
};

// Single-precision difference of two double-precision centres a - b without FP64 instructions
// (FP64 issues at 1/64 of the FP32 rate on this GPU).  Each centre is held as the float pair
// h = fl(c), l = fl(c - h), so c = h + l to about 2^-48 |c|, and the difference is formed as
// (h_a - h_b) + (l_a - l_b): within about one unit in the last place of fl(a - b), the rounded
// double difference it replaces.
__device__ __forceinline__ float cen_diff(float ha, float la, float hb, float lb)
{
    return __fadd_rn(__fsub_rn(ha, hb), __fsub_rn(la, lb));
}

// Periodic unit box (Sec. 3.1, periodic boundaries): the walk starts from the root and its copies
// shifted by n, |n|_inf <= R (R = nrep, 26 or 124 copies), and every checklist and list entry
// carries the copy its source lies in.  An entry is
//   bit 31: particle (else cell) | bits 30..ib: copy code q | bits ib-1..0: index,
// q = (n_x + R) W^2 + (n_y + R) W + (n_z + R) with W = 2R + 1, so the box itself is
// q0 = R (W^2 + W + 1).  An isolated box has R = 0 and ib = 31: q is always 0 and the index is
// the whole entry, as before.
//
// The walk decides on a copy's geometry shifted in FP64 and then rounded, fl(x + n_a) per axis, as
// for the box itself.  FP64 issues at 1/64 of the FP32 rate, so those values are tabulated once
// per solve (k_shift_tables) for every cell and particle, axis and non-zero shift value v in
// [-R, R]: slot (i * 3 + axis) * 2R + shift_slot(v).
struct PeriodicArgs {
    int ib;        // index bits
    int R;         // replica shell radius (0: isolated)
    const float4* cshift;  // per cell, axis and shift: (fl(com + v), fl(lo + v), fl(hi + v), 0)
    const float* pshift;   // per particle, axis and shift: fl(x + v)
};

__host__ __device__ __forceinline__ int shift_slot(int v, int R) { return v < 0 ? v + R : v + R - 1; }

__host__ __device__ __forceinline__ unsigned int entry_index(unsigned int e, int ib)
{
    return e & ((1u << ib) - 1u);
}
__host__ __device__ __forceinline__ unsigned int entry_copy(unsigned int e, int ib)
{
    return (e & ~FMM_PARTICLE_BIT) >> ib;
}
__host__ __device__ __forceinline__ unsigned int copy_centre(int R)
{
    const int W = 2 * R + 1;
    return (unsigned int)(R * (W * W + W + 1));
}
// the shift n of copy code q
__host__ __device__ __forceinline__ void copy_shift(unsigned int q, int R, int& nx, int& ny, int& nz)
{
    const int W = 2 * R + 1;
    nx = (int)q / (W * W) - R;
    ny = ((int)q / W) % W - R;
    nz = (int)q % W - R;
}

// Shift the float pair (h, l) of a centre c = h + l by an integer n (|n| <= 2, |h| < 1): the
// rounded sum t = fl(n + h) and its exact rounding error h - (t - n) (|n| >= |h|, so the error is
// representable and computed exactly), added into the low part.  n = 0 leaves the pair unchanged.
__device__ __forceinline__ void cen_shift(float& h, float& l, float n)
{
    const float t = __fadd_rn(n, h);
    const float err = __fsub_rn(h, __fsub_rn(t, n));
    h = t;
    l = __fadd_rn(l, err);
}

// A sink group after the walk.
struct __align__(16) Group {
    int cell;
    int first;
    int count;
    int pp_src;  // source particles in the PP list
    unsigned long long pp_off, pc_off;
    int pp_len, pc_len;
};

#define FMM_LIST_CHUNK 64  // default list entries per PP / PC work item
#define FMM_LOCAL_RANGE 512  // local entries per warp range of the own-expansion kernel
#define FMM_GMAX 64       // sink slots per group
#define FMM_MAX_LEVELS 192  // walk levels: tree depth + 1 (63 key bits + 31 position bits at most)

// Device-side counters and status, one per context.
struct DevCounters {
    unsigned int status;    // FMM_DEV_ERR_* bits of invalid input or failed waits
    unsigned int overflow;  // a walk list or scratch capacity was exceeded (host grows and retries)
    unsigned int depth;     // deepest cell level
    unsigned int kdk_status;  // FMM_DEV_ERR_ARG: a compressed kick-drift kept a particle from leaving the
                              // isolated box (kept across solves until a solve reports it)
    unsigned long long n_active;
    // walk totals
    unsigned long long n_groups, cp_len;  // cp_len: entries of the point-source local list
    unsigned long long pp_len, pc_len, cc_len;
    unsigned long long n_pp_pairs, n_pc_pairs, n_cc, n_cp;
    unsigned long long pp_work, pc_work;  // work counters of the persistent interaction kernels
    unsigned int n_item_pp, n_item_pc;    // work items of the interaction kernels
    unsigned int n_bm_items;              // (cell, particle chunk) items of the exact b_max
    unsigned int pad1;
    unsigned long long n_audit;           // (sink, source) pairs recorded by an audit walk
    unsigned long long n_mlp;             // learned decisions taken
    // per walk level: frontier size, work counters of the walk and local kernels, and the
    // number of checklist entries handed to that level
    unsigned long long lv_front[FMM_MAX_LEVELS];
    unsigned long long lv_work[FMM_MAX_LEVELS];
    unsigned long long lv_cl[FMM_MAX_LEVELS];
    unsigned long long lv_entries[FMM_MAX_LEVELS];      // checklist entries examined (incl. opened)
    unsigned long long lv_max_entries[FMM_MAX_LEVELS];  // largest per-sink count
    unsigned long long lv_base[FMM_MAX_LEVELS + 1];     // first walked cell of each level in DevWalk::wcells
    // local-list entries (multipole and point sources) of each level's sinks: a level's entries
    // follow those of the levels before it in the flat lists
    unsigned long long lv_cc[FMM_MAX_LEVELS];
    unsigned long long lv_cp[FMM_MAX_LEVELS];
};

// A walk (or the b_max items before it) that ran past a capacity left holes in the lists: the
// kernels after it read nothing and return, and the host grows the buffers and solves again.
__device__ __forceinline__ bool fmm_overflowed(const DevCounters* ctr)
{
    return *(const volatile unsigned int*)&ctr->overflow != 0u;
}

// One particle of the input as the key kernel copies it, in input order, for the gather after
// the sort: a single aligned 32-byte sector per particle instead of one per coordinate.
struct __align__(32) SrcRec {
    double x, y, z;
    float m;
    unsigned int act;
};
static_assert(sizeof(SrcRec) == 8 * sizeof(int), "an input record spans the 8 ints per particle of the radix block");

// Device buffers of a context.  Capacities are in elements.
struct DevTree {
    long long n = 0, cap_n = 0;
    long long n_cells = 0, cap_cells = 0, n_buckets = 0;
    int depth = 0;
    // device copies of the cell and bucket counts [n_cells, n_buckets]; kernels over cells or
    // buckets read their bound there, so a launch may cover the capacity (graph capture, where
    // the host does not know the counts) instead of the count
    const unsigned int* dcount = nullptr;
    bool cap_grid = false;
    // exact b_max of internal cells: per cell a count and first index of (cell, chunk) items, the
    // FP32 and FP64 running maxima (as ordered bit patterns), and the items' cells
    unsigned int *bm_cnt = nullptr, *bm_base = nullptr, *bm32 = nullptr;
    unsigned long long* bm64 = nullptr;
    int* bm_item = nullptr;
    unsigned int* bm_order = nullptr;  // the items by the particle they start at
    unsigned int *bm_bin = nullptr, *bm_binbase = nullptr;  // items per chunk of particles, and their scan
    float* bm_imax = nullptr;  // FP32 maximum of each item
    long long cap_bm_items = 0;
    // sorting
    unsigned long long *key = nullptr, *key_alt = nullptr;
    unsigned int *idx = nullptr, *idx_alt = nullptr;
    SrcRec *src = nullptr;  // the input particles in input order (key kernel to gather), a view of radix
    int *radix = nullptr;   // one block of 8 ints per particle: src, then the radix tree's arrays
    // sorted particles
    double *sx = nullptr, *sy = nullptr, *sz = nullptr;
    float *sm = nullptr;
    unsigned char *sact = nullptr;
    float4 *posf = nullptr;  // single-precision position for the walk's decisions
    float4 *plo = nullptr;   // per particle fl(x - fl(x)): with posf the centre pair of cen_diff
    float4 *off = nullptr;   // (x - com_bucket) in single precision, mass
    int *bucket_of = nullptr;
    int *act = nullptr;      // per group, its active particles compacted (see k_group_active)
    // radix tree (nodes 0..n-2 internal, leaf p is node n-1+p)
    int *ifirst = nullptr, *ilast = nullptr, *ileft = nullptr, *iright = nullptr;  // child node ids (views of radix)
    int *nparent = nullptr;  // parent internal node of every node (2n-1)
    unsigned int *keep = nullptr;  // 2n-1 flags, scanned to cell ids
    unsigned int *bflag = nullptr; // n flags, scanned to bucket ids
    // cells
    int *cfirst = nullptr, *ccount = nullptr, *cparent = nullptr, *cchild = nullptr, *cnact = nullptr;
    int *bucket_cell = nullptr;
    unsigned int *arrive = nullptr;
    Com4 *com = nullptr;      // centre of mass + mass
    float4 *cen = nullptr;    // per cell [2c] = fl(com), [2c + 1] = fl(com - fl(com)) (cen_diff)
    double *clo = nullptr, *chi = nullptr;  // 3 per cell
    double *bmax = nullptr;
    float *rec = nullptr;        // FMM_NREC per cell
    WalkNode *node = nullptr;
    float4 *mnorm = nullptr;     // per cell: |M2|/(M b^2), |M4|/(M b^4), M (float), 0
    float *amin = nullptr;       // per cell: smallest |a| estimate of its particles (learned criterion)
    float *L = nullptr;          // FMM_NL per cell: own local expansion of walked cells
    // several independent boxes: box b holds sorted particles [box_off[b], box_off[b+1])
    int nbox = 1;
    long long *box_off = nullptr;            // device, nbox + 1
    long long *box_off_h = nullptr;          // pinned copy
    int *box_root = nullptr;                 // device, nbox: the cell spanning the box
    long long cap_box = 0;
    unsigned long long *sbox = nullptr;      // sorted box id per particle (several boxes only)
    unsigned long long *key_orig = nullptr;  // Morton keys in input order (several boxes only)
    long long cap_box_n = 0;
    // graded build (dual trees): with grade_key set, a radix node also splits where the fixed
    // tree's sorted keys grade_key hold more than b particles in its Morton box, and a cell is no
    // group where they hold more than g (split: per node, bit 0 split, bit 1 no group; nogroup:
    // per cell, valid while graded)
    const unsigned long long* grade_key = nullptr;
    long long grade_n = 0;
    int grade_group = 0;
    bool graded = false;
    unsigned char *split = nullptr, *nogroup = nullptr;
    long long cap_split = 0, cap_nogroup = 0;
    // periodic box (nrep > 0): the replica shell radius and the index bits of list entries;
    // R = 0, ib = 31 for an isolated box
    int per_R = 0, per_ib = 31;
    float* ewald_L = nullptr;  // FP32 local coefficients of the Ewald correction per sub-cube
    float4* cshift = nullptr;  // shifted cell geometry (PeriodicArgs), 3 * 2R per cell
    float* pshift = nullptr;   // shifted particle positions, 3 * 2R per particle
    long long cap_cshift = 0, cap_pshift = 0;
    // scan scratch
    unsigned int *scan_part = nullptr;
    long long cap_scan_part = 0;
    unsigned int *hist = nullptr;
    long long cap_hist = 0;
};

__host__ __forceinline__ PeriodicArgs periodic_args(const DevTree& t)
{
    PeriodicArgs a;
    a.ib = t.per_ib;
    a.R = t.per_R;
    a.cshift = t.cshift;
    a.pshift = t.pshift;
    return a;
}

struct DevWalk {
    long long cap_front = 0, cap_cl = 0, cap_pp = 0, cap_pc = 0, cap_cc = 0, cap_cp = 0, cap_groups = 0;
    long long cap_scratch = 0;  // entries per list per warp
    int n_warps = 0;
    int *f_cell[2] = {nullptr, nullptr};
    unsigned long long *f_cloff[2] = {nullptr, nullptr};
    int *f_cllen[2] = {nullptr, nullptr};
    // per cell: its local-expansion entries, multipole sources (lcc, list cc) and point sources
    // (lcp, list cp: particles and one-particle cells)
    unsigned long long *lcc_off = nullptr, *lcp_off = nullptr;
    int *lcc_len = nullptr, *lcp_len = nullptr;
    int *wcells = nullptr;  // the walked cells in level order (level l at ctr->lv_base[l])
    float *Lg = nullptr;                    // FMM_NL per group: the group's local expansion
    // work items of the interaction kernels: group g's PP list is cut into chunks of list_chunk
    // entries (items base_pp[g] ..), its PC list into chunks of list_chunk cells;
    // every item writes one partial result per sink slot, summed per sink in item order
    unsigned int *cnt_pp = nullptr, *cnt_pc = nullptr, *base_pp = nullptr, *base_pc = nullptr;
    unsigned int *item_pp = nullptr, *item_pc = nullptr;
    float4 *part_pp = nullptr, *part_pc = nullptr;
    long long cap_item_pp = 0, cap_item_pc = 0;
    unsigned int *cl[2] = {nullptr, nullptr};
    unsigned int *pp = nullptr, *pc = nullptr, *cc = nullptr, *cp = nullptr;
    int *cc_sink = nullptr, *cp_sink = nullptr;  // sink cell of every local entry
    Group *groups = nullptr;
    unsigned int *scratch = nullptr;
    // levels kept for export of the local lists
    long long n_groups = 0, pp_len = 0, pc_len = 0, cc_len = 0, cp_len = 0, n_levels = 0;
};

// The fixed tree of the dual-tree scheme (dual.cu): a copy of the source-side arrays of a tree
// built from the particles of the slow rungs, in its own numbering (cells [0, n_cells), buckets
// [0, n_buckets), sorted particles [0, n)), appended after each active tree.
struct FixedTree {
    bool valid = false;        // set by fmm_set_fixed_sources
    int bucket = 0;            // bucket size it was built with (the active tree must use the same)
    long long n_all = 0;       // particle count of the caller's arrays it was selected from
    unsigned int* member = nullptr;  // n_all flags: 1 for the particles in the fixed set
    long long cap_member = 0;
    long long n = 0, n_cells = 0, n_buckets = 0;
    long long cap_n = 0, cap_cells = 0;
    int *cfirst = nullptr, *ccount = nullptr, *cchild = nullptr, *cparent = nullptr, *bucket_cell = nullptr;
    Com4 *com = nullptr;
    double *clo = nullptr, *chi = nullptr, *bmax = nullptr;
    float *rec = nullptr;
    float4 *posf = nullptr, *plo = nullptr, *off = nullptr;
    int *bucket_of = nullptr;
    unsigned long long *key = nullptr;  // its sorted Morton keys (the graded build of the active tree)
};

// ---------------------------------------------------------------- launchers (host)

// scan.cu / sort.cu
cudaError_t fmm_scan_exclusive(const unsigned int* in, unsigned int* out, long long n, unsigned int* total_dev,
                               DevTree& t, cudaStream_t s);
cudaError_t fmm_radix_sort(DevTree& t, long long n, cudaStream_t s);
cudaError_t fmm_radix_sort_kv(unsigned long long* ka, unsigned long long* kb, unsigned int* va, unsigned int* vb,
                              long long n, int passes, DevTree& t, cudaStream_t s);
cudaError_t fmm_sort_ensure(DevTree& t, long long n);
cudaError_t fmm_scan_reserve(DevTree& t, long long n);
long long fmm_sort_hist_entries(long long n);
long long fmm_sort_part_entries(long long n);
cudaError_t fmm_sort_prepare();
cudaError_t fmm_radix_sort_kv_scratch(unsigned long long* ka, unsigned long long* kb, unsigned int* va,
                                      unsigned int* vb, long long n, int passes, unsigned int* hist,
                                      unsigned int* part, cudaStream_t s);

// tree.cu
// positions: pos (FP64 SoA) or, when ipos is given, 32-bit fixed-point coordinates x = u 2^-32
cudaError_t fmm_launch_keys(DevTree& t, const double* pos, const float* mass, const unsigned char* active,
                            long long n, DevCounters* ctr,
                            cudaStream_t s, const unsigned int* ipos = nullptr);
cudaError_t fmm_launch_gather(DevTree& t, long long n, DevCounters* ctr, cudaStream_t s);
cudaError_t fmm_launch_bucket_index(DevTree& t, long long n, cudaStream_t s);
cudaError_t fmm_launch_radix_tree(DevTree& t, long long n, int bucket, cudaStream_t s);
cudaError_t fmm_launch_cells(DevTree& t, long long n, int bucket, cudaStream_t s);
cudaError_t fmm_launch_upward(DevTree& t, long long n, int bucket, DevCounters* ctr, cudaStream_t s);
long long fmm_bmax_items_bound(long long n, int depth, long long n_cells);
long long fmm_bmax_bins(long long n);
cudaError_t fmm_launch_nodes(DevTree& t, double theta, cudaStream_t s);
cudaError_t fmm_launch_depth(DevTree& t, const unsigned int* ncell_dev, DevCounters* ctr, cudaStream_t s);
cudaError_t fmm_launch_box_sort(DevTree& t, long long n, cudaStream_t s);
cudaError_t fmm_launch_box_roots(DevTree& t, cudaStream_t s);

// walk.cu
struct WalkArgs {
    int level;
    int level_parity;
    int bucket, group;
    float four_eps2;
    float eps2;
    float eps;
    // learned criterion (mode 1) and audit (mode 2); mode 0 is the fixed-theta criterion
    int mode;
    float band_lo, band_hi, tau, margin;
    const unsigned char* mlp_packed;
    int2* audit_pairs;
    long long audit_cap;
};
cudaError_t fmm_launch_walk_level(DevTree& t, DevWalk& w, DevCounters* ctr, const WalkArgs& a, cudaStream_t s);
struct LocalGrids {
    unsigned cc, cp, down;  // blocks of the M2L, P2L and top-down kernels
};
LocalGrids fmm_local_grids(const DevWalk& w, long long n_cc, long long n_cp, long long n_cells);
cudaError_t fmm_launch_local_level(DevTree& t, DevWalk& w, DevCounters* ctr, float eps2, int level, int levels,
                                   const LocalGrids& g, cudaStream_t s);
cudaError_t fmm_launch_local_groups(DevWalk& w, DevTree& t, DevCounters* ctr, cudaStream_t s);
cudaError_t fmm_launch_walk_seed(DevTree& t, DevWalk& w, DevCounters* ctr, cudaStream_t s, int second_root = -1);
cudaError_t fmm_launch_shift_tables(DevTree& t, cudaStream_t s);
int fmm_walk_warps(int device);

// interact.cu
struct InteractArgs {
    float eps2;
    int terms;
    int accumulate;
    int chunk;  // list entries per PP / PC work item (multiple of 32)
};
cudaError_t fmm_launch_items(DevTree& t, DevWalk& w, DevCounters* ctr, int chunk, cudaStream_t s);
cudaError_t fmm_launch_pp(DevTree& t, DevWalk& w, DevCounters* ctr, const InteractArgs& a, cudaStream_t s);
cudaError_t fmm_launch_pc(DevTree& t, DevWalk& w, DevCounters* ctr, const InteractArgs& a, cudaStream_t s);
// perm: sorted sink -> index in acc/pot (NULL: the tree's own order t.idx)
cudaError_t fmm_launch_l2p_out(DevTree& t, DevWalk& w, DevCounters* ctr, const InteractArgs& a, float* acc,
                               float* pot, long long n, cudaStream_t s, const unsigned int* perm = nullptr);
int fmm_interact_blocks(int device);

// dual.cu
cudaError_t fmm_launch_subset_flags(const unsigned char* rung, int r_max, const unsigned int* flag_not, long long n,
                                    unsigned int* flag, cudaStream_t s);
cudaError_t fmm_launch_subset_gather(const unsigned int* flag, const unsigned int* at, long long n, const double* pos,
                                     const double* vel, double dt, const float* mass, const unsigned char* mask,
                                     long long m, double* pos_out, float* mass_out, unsigned char* mask_out,
                                     unsigned int* idx, cudaStream_t s);
cudaError_t fmm_append_fixed(DevTree& t, const FixedTree& f, long long na, long long ca, long long ba, cudaStream_t s);
cudaError_t fmm_launch_compose_perm(const unsigned int* perm, const unsigned int* sub, long long n, unsigned int* out,
                                    cudaStream_t s);

// ewald.cu
long long fmm_ewald_floats();
cudaError_t fmm_launch_ewald_grid(DevTree& t, int terms, cudaStream_t s);
cudaError_t fmm_launch_ewald_groups(DevTree& t, DevWalk& w, DevCounters* ctr, int terms, cudaStream_t s);

// kdk.cu
cudaError_t fmm_launch_kick_drift(double* pos, double* vel, const float* acc, unsigned char* rung,
                                  unsigned char* active_next, long long n, double eps, double dt0, int max_rung,
                                  int substep, int closing, DevCounters* ctr, cudaStream_t s);
cudaError_t fmm_launch_assign_rungs(const float* acc, unsigned char* rung, long long n, double eps, double dt0,
                                    int max_rung, cudaStream_t s);
cudaError_t fmm_launch_kick_drift_i32(unsigned int* ipos, float* vel, const float* acc, unsigned char* rung,
                                      unsigned char* active_next, long long n, double eps, double dt0, int max_rung,
                                      int substep, int closing, int periodic, DevCounters* ctr, cudaStream_t s);

// Raises a kernel's dynamic shared-memory limit to `bytes` on the calling thread's current
// device, once per device.  Function attributes belong to each device's context, so a flag for
// the whole process would skip the call on the second device; `done` holds one bit per device
// (devices 0-63; others set the attribute on every call).  Setting it twice is harmless, so two
// threads that race on the first call only repeat the call.
template <typename F>
cudaError_t fmm_smem_attr_once(F* func, int bytes, std::atomic<unsigned long long>& done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ unsigned int fmm_lanemask_lt()
{
    unsigned int m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__host__ __device__ __forceinline__ long long fmm_ceil_div(long long a, long long b) { return (a + b - 1) / b; }
