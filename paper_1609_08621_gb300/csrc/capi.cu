// C ABI and host orchestration of the force solve (see include/fmm.h).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <mutex>
#include <unordered_map>
#include <vector>

#include <math.h>

#include "expansions.cuh"
#include "fmm_internal.cuh"
#include "mlp.cuh"

cudaError_t fmm_mlp_pack(const float* params, unsigned char* packed, cudaStream_t s);
cudaError_t fmm_mlp_grad(const float* params, const float* feats, const float* labels, const unsigned int* idx,
                         long long nrows, float inv_b, float loss_scale, float* grad, float* loss, cudaStream_t s);
cudaError_t fmm_mlp_adam(float* p, const float* g, float* m, float* v, float lr, int step, cudaStream_t s);
cudaError_t fmm_mlp_predict(const unsigned char* packed, const float* feats, long long n, float* out, cudaStream_t s);
cudaError_t fmm_launch_audit_labels(DevTree& t, const int2* pairs, long long npairs, const float* acc_ref,
                                    long long n, float eps, float* feats, float* labels, cudaStream_t s);
cudaError_t fmm_launch_cell_amin(DevTree& t, const float* acc, long long n, cudaStream_t s);

namespace {

thread_local std::string g_err;

fmm_status fail(fmm_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail(e_ == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                         \
    } while (0)

// Buffer growth.  A block that regrows a group of buffers first sets their capacity to 0, so an
// allocation that fails part-way (FMM_ERR_OOM) leaves every buffer of the group to be allocated
// again by the next call: the context stays usable.  fmm_debug_fail_allocations makes the calling
// thread's next allocations fail, to test exactly that.
thread_local long long g_fail_allocs_after = -1;  // < 0: off; else successful allocations left

// Sizes of the device buffers allocated here, by address (fmm_memory_info sums a context's).
std::mutex g_size_mutex;
std::unordered_map<void*, size_t> g_sizes;

void dev_free(void* p)
{
    if (!p) return;
    cudaFree(p);
    std::lock_guard<std::mutex> lock(g_size_mutex);
    g_sizes.erase(p);
}

size_t dev_size(const void* p)
{
    if (!p) return 0;
    std::lock_guard<std::mutex> lock(g_size_mutex);
    auto it = g_sizes.find(const_cast<void*>(p));
    return it == g_sizes.end() ? 0 : it->second;
}

template <typename T>
cudaError_t grow(T** p, long long* cap, long long need)
{
    if (need <= *cap && *p) return cudaSuccess;
    dev_free(*p);
    *p = nullptr;
    *cap = 0;
    if (need < 1) need = 1;
    if (g_fail_allocs_after == 0) return cudaErrorMemoryAllocation;
    if (g_fail_allocs_after > 0) g_fail_allocs_after--;
    const size_t bytes = (size_t)need * sizeof(T);
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e == cudaSuccess) {
        *cap = need;
        std::lock_guard<std::mutex> lock(g_size_mutex);
        g_sizes[(void*)*p] = bytes;
    }
    return e;
}

template <typename T>
cudaError_t alloc(T** p, long long need)
{
    long long cap = 0;
    dev_free(*p);
    *p = nullptr;
    return grow(p, &cap, need);
}

}  // namespace

// records the message returned by fmm_last_error for entry points of other translation units
fmm_status fmm_report_error(fmm_status st, const char* msg)
{
    g_err = msg;
    return st;
}

struct fmm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    fmm_params params;
    DevTree t;
    DevWalk w;
    DevCounters* ctr = nullptr;       // device
    DevCounters* ctr_h = nullptr;     // pinned mirror
    unsigned int* totals = nullptr;   // device: [cells, buckets]
    unsigned int* totals_h = nullptr; // pinned
    unsigned int* seed = nullptr;     // device: root frontier / checklist constants
    cudaEvent_t ev[8] = {};
    fmm_stats stats;
    bool have_tree = false, have_solve = false;
    // the per-level counts of the context's last completed walk (size the next walk's local grids);
    // kept apart from ctr_h, which later copies overwrite
    bool have_counts = false;
    long long prev_front[FMM_MAX_LEVELS] = {}, prev_cc[FMM_MAX_LEVELS] = {}, prev_cp[FMM_MAX_LEVELS] = {};
    long long prev_cc_len = 0, prev_cp_len = 0;
    int launches = 0;  // kernels launched by the current solve
    float theta_nodes = -1.0f;
    // dual trees: the fixed tree, the subset scratch (flags, their scan, subset -> caller index,
    // the subset's positions and masses, the composed output order) and the walk's second root
    FixedTree fx;
    unsigned int *d_flag = nullptr, *d_at = nullptr, *d_idx = nullptr, *d_perm = nullptr;
    unsigned char* d_act = nullptr;
    double* d_pos = nullptr;
    float* d_mass = nullptr;
    long long cap_d = 0;
    int second_root = -1;
    // learned criterion: FP32 master parameters, Adam state, packed BF16 copy
    float *mlp_p = nullptr, *mlp_g = nullptr, *mlp_m = nullptr, *mlp_v = nullptr, *mlp_loss = nullptr;
    unsigned char* mlp_packed = nullptr;
    bool mlp_ready = false;
    int2* audit_pairs = nullptr;
    long long audit_cap = 0;
    unsigned int* mlp_idx = nullptr;
    long long mlp_idx_cap = 0;
    float* mlp_pred = nullptr;  // predictions over the training rows (surrogate fit)
    long long mlp_pred_cap = 0;
    // CUDA graph of the whole solve (fmm_set_graphs): captured after an eager solve and replayed
    // while the call's inputs, buffers and parameters stay the same
    bool graphs = false;
    cudaGraphExec_t gexec_head = nullptr, gexec = nullptr;  // the solve's head and the rest
    cudaStream_t cap_stream = nullptr;  // capture needs a stream of its own (the caller's may be the legacy one)
    struct GraphKey {
        const void *pos, *mass, *active, *acc, *pot;
        bool i32;  // pos holds 32-bit fixed-point coordinates
        long long n;
        int nbox;
        std::vector<long long> off;
        fmm_params p;
        double eps, theta;
    } gkey;
    int graph_levels = 0, graph_launches = 0;
    std::vector<void*> graph_bufs;  // the context's buffer addresses when the graph was captured
    long long graph_replays = 0;
    // periodic box: the Ewald sub-cube expansions run on a side stream beside the walk (fork after
    // the tree, join before the groups add them)
    cudaStream_t ew_stream = nullptr;
    cudaEvent_t ew_fork = nullptr, ew_join = nullptr;
    // the local expansions of each walk level run on a side stream while the walk goes on (a fork
    // after every level, a join before the groups take their expansions)
    cudaStream_t loc_stream = nullptr;
    cudaEvent_t loc_fork = nullptr, loc_join = nullptr;
    // positions of the current call as 32-bit fixed-point coordinates (fmm_compute_forces_i32), else
    // NULL and the call's FP64 positions are used
    const unsigned int* cur_ipos = nullptr;
    // walks of at least this many sinks (previous solve) run the local expansions on a side stream
    // (fmm_debug_local_side; FMM_LOCAL_SIDE_SINKS by default)
    long long side_sinks = -1;
    // test hook (fmm_debug_walk_capacity): the walk's first per-warp scratch and list capacities
    long long dbg_scratch = 0, dbg_list_scale = 0;
    // staging for the host-buffer entry point
    double* hpos = nullptr;
    float *hmass = nullptr, *hacc = nullptr, *hpot = nullptr;
    unsigned char* hact = nullptr;
    long long hcap = 0;
};

static fmm_status check_params(const fmm_params* p)
{
    if (!p) return fail(FMM_ERR_ARG, "params is NULL");
    if (!(p->theta > 0.0 && p->theta <= 1.0)) return fail(FMM_ERR_ARG, "theta must be in (0, 1], got %g", p->theta);
    if (!(p->eps > 0.0) || !(p->eps < 1.0)) return fail(FMM_ERR_ARG, "eps must be in (0, 1), got %g", p->eps);
    if (p->bucket < 1 || p->bucket > 16) return fail(FMM_ERR_ARG, "bucket must be in [1, 16], got %d", p->bucket);
    if (p->group < p->bucket || p->group > 64)
        return fail(FMM_ERR_ARG, "group must be in [bucket, 64], got %d", p->group);
    if (p->criterion != 0 && p->criterion != 1) return fail(FMM_ERR_ARG, "criterion must be 0 or 1, got %d", p->criterion);
    if (!(p->band_lo > 0.0 && p->band_lo <= p->band_hi && p->band_hi <= 2.0))
        return fail(FMM_ERR_ARG, "band must satisfy 0 < band_lo <= band_hi <= 2");
    if (!isfinite(p->mlp_tau)) return fail(FMM_ERR_ARG, "mlp_tau must be finite");
    if (!(p->mlp_margin >= 0.0 && p->mlp_margin <= 1.0)) return fail(FMM_ERR_ARG, "mlp_margin must be in [0, 1]");
    if (p->accumulate != 0 && p->accumulate != 1) return fail(FMM_ERR_ARG, "accumulate must be 0 or 1, got %d", p->accumulate);
    if (p->terms < 0 || p->terms > 15) return fail(FMM_ERR_ARG, "terms must be a mask of 1|2|4|8, got %d", p->terms);
    if (p->nrep < 0 || p->nrep > 2) return fail(FMM_ERR_ARG, "nrep must be 0 (isolated), 1 or 2, got %d", p->nrep);
    if (p->list_chunk != 0 && (p->list_chunk < 32 || p->list_chunk > 1024 || p->list_chunk % 32 != 0))
        return fail(FMM_ERR_ARG, "list_chunk must be 0 or a multiple of 32 in [32, 1024], got %d", p->list_chunk);
    if (p->spin_limit < 1) return fail(FMM_ERR_ARG, "spin_limit must be >= 1");
    return FMM_OK;
}

extern "C" fmm_status fmm_default_params(fmm_params* p)
{
    if (!p) return fail(FMM_ERR_ARG, "params is NULL");
    memset(p, 0, sizeof *p);
    p->theta = 0.55;
    p->eps = 1e-3;
    p->bucket = 16;
    p->group = 64;
    p->criterion = 0;
    p->accumulate = 0;
    p->terms = 15;
    p->spin_limit = 1LL << 26;
    p->nrep = 0;
    p->mlp_tau = -3.5;
    p->band_lo = 0.35;
    p->band_hi = 1.0;
    p->mlp_margin = 0.1;
    return FMM_OK;
}

extern "C" const char* fmm_last_error(void) { return g_err.c_str(); }

extern "C" fmm_status fmm_debug_fail_allocations(long long after)
{
    g_fail_allocs_after = after < 0 ? -1 : after;
    return FMM_OK;
}

extern "C" fmm_status fmm_debug_local_side(fmm_ctx* c, long long min_sinks)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    c->side_sinks = min_sinks < 0 ? -1 : min_sinks;
    return FMM_OK;
}

extern "C" fmm_status fmm_debug_walk_capacity(fmm_ctx* c, long long scratch_entries, long long list_scale)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    if (scratch_entries < 0 || list_scale < 0) return fail(FMM_ERR_ARG, "capacities must be >= 0");
    c->dbg_scratch = scratch_entries;
    c->dbg_list_scale = list_scale;
    return FMM_OK;
}

extern "C" double fmm_flops_per_pc(void) { return (double)FMM_FLOPS_PC; }

// The device buffers of the tree, the walk, the fixed tree and the subset scratch.
static std::vector<void*> tree_walk_buffers(const fmm_ctx* c)
{
    const DevTree& t = c->t;
    const DevWalk& w = c->w;
    const FixedTree& f = c->fx;
    return {t.key, t.key_alt, t.idx, t.idx_alt, t.radix, t.sx, t.sy, t.sz, t.sm, t.sact, t.posf, t.plo, t.cen, t.off,
            t.bucket_of, t.act, t.bflag, t.cfirst,
            t.ccount, t.cparent, t.cchild, t.cnact, t.bucket_cell, t.arrive, t.com, t.clo, t.chi, t.bmax, t.rec,
            t.node, t.mnorm, t.amin, t.bm_cnt, t.bm_base, t.bm32, t.bm64, t.bm_item, t.bm_imax, t.bm_order, t.bm_bin, t.bm_binbase, t.L, t.scan_part,
            t.hist, t.box_off, t.box_root, t.sbox, t.key_orig, t.split, t.nogroup, t.ewald_L, t.cshift, t.pshift,
            w.f_cell[0], w.f_cell[1], w.f_cloff[0], w.f_cloff[1], w.f_cllen[0], w.f_cllen[1], w.lcc_off, w.lcc_len,
            w.lcp_off, w.lcp_len, w.wcells, w.cp, w.cp_sink, w.Lg, w.cnt_pp, w.cnt_pc, w.base_pp, w.base_pc, w.item_pp, w.item_pc, w.part_pp, w.part_pc,
            w.cl[0], w.cl[1], w.pp, w.pc, w.cc, w.cc_sink, w.groups, w.scratch,
            f.cfirst, f.ccount, f.cchild, f.cparent, f.bucket_cell, f.com, f.clo, f.chi, f.bmax, f.rec, f.posf, f.plo,
            f.off, f.bucket_of, f.key, f.member, c->d_flag, c->d_at, c->d_idx, c->d_perm, c->d_act, c->d_pos, c->d_mass};
}

static void free_all(fmm_ctx* c)
{
    DevTree& t = c->t;
    for (void* p : tree_walk_buffers(c)) dev_free(p);
    if (c->ctr) cudaFree(c->ctr);
    if (c->totals) cudaFree(c->totals);
    if (c->seed) cudaFree(c->seed);
    if (c->ctr_h) cudaFreeHost(c->ctr_h);
    if (t.box_off_h) cudaFreeHost(t.box_off_h);
    if (c->totals_h) cudaFreeHost(c->totals_h);
    void* hs[] = {c->hpos, c->hmass, c->hacc, c->hpot, c->hact, c->mlp_p, c->mlp_g, c->mlp_m, c->mlp_v, c->mlp_loss,
                  c->mlp_packed, c->audit_pairs, c->mlp_idx, c->mlp_pred};
    for (void* p : hs) dev_free(p);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->gexec_head) cudaGraphExecDestroy(c->gexec_head);
    c->gexec_head = nullptr;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    c->cap_stream = nullptr;
    if (c->loc_stream) cudaStreamDestroy(c->loc_stream);
    if (c->loc_fork) cudaEventDestroy(c->loc_fork);
    if (c->loc_join) cudaEventDestroy(c->loc_join);
    c->loc_stream = nullptr;
    c->loc_fork = c->loc_join = nullptr;
    if (c->ew_stream) cudaStreamDestroy(c->ew_stream);
    if (c->ew_fork) cudaEventDestroy(c->ew_fork);
    if (c->ew_join) cudaEventDestroy(c->ew_join);
    c->ew_stream = nullptr;
    c->ew_fork = c->ew_join = nullptr;
}

extern "C" fmm_status fmm_memory_info(const fmm_ctx* c, long long* device_bytes, long long* host_bytes)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    long long d = 0;
    for (void* p : tree_walk_buffers(c)) d += (long long)dev_size(p);
    const void* hs[] = {c->hpos, c->hmass, c->hacc, c->hpot, c->hact, c->mlp_p, c->mlp_g, c->mlp_m, c->mlp_v,
                        c->mlp_loss, c->mlp_packed, c->audit_pairs, c->mlp_idx, c->mlp_pred};
    for (const void* p : hs) d += (long long)dev_size(p);
    d += (long long)(sizeof(DevCounters) + 12 * sizeof(unsigned int));
    if (device_bytes) *device_bytes = d;
    if (host_bytes) *host_bytes = (long long)sizeof(DevCounters) + 2 * (long long)sizeof(unsigned int);
    return FMM_OK;
}

extern "C" fmm_status fmm_create(fmm_ctx** out, int device, void* cuda_stream)
{
    if (!out) return fail(FMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(FMM_ERR_ARG, "device %d out of range (%d devices)", device, ndev);
    CK(cudaSetDevice(device));
    fmm_ctx* c = new fmm_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    fmm_default_params(&c->params);
    memset(&c->stats, 0, sizeof c->stats);
    cudaError_t e = cudaMalloc(&c->ctr, sizeof(DevCounters));
    if (e == cudaSuccess) e = cudaMallocHost(&c->ctr_h, sizeof(DevCounters));
    if (e == cudaSuccess) e = cudaMalloc(&c->totals, 4 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMallocHost(&c->totals_h, 4 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&c->seed, 8 * sizeof(unsigned int));
    for (auto& ev : c->ev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e == cudaSuccess) e = cudaMemset(c->seed, 0, 8 * sizeof(unsigned int));
    // the side stream of the walk levels' local expansions, made here so that no capture creates it
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->loc_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->loc_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->loc_join, cudaEventDisableTiming);
    // every counter starts at zero, the compressed kick-drift's status word included (it is kept
    // across solves, so memory left by an earlier context must not read as a report)
    if (e == cudaSuccess) e = cudaMemset(c->ctr, 0, sizeof(DevCounters));
    if (e == cudaSuccess) memset(c->ctr_h, 0, sizeof(DevCounters));
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return fail(e == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA, "fmm_create: %s",
                    cudaGetErrorString(e));
    }
    c->w.n_warps = fmm_walk_warps(device);
    c->t.dcount = c->totals;
    *out = c;
    return FMM_OK;
}

extern "C" void fmm_destroy(fmm_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

extern "C" fmm_status fmm_set_params(fmm_ctx* c, const fmm_params* p)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    fmm_status st = check_params(p);
    if (st != FMM_OK) return st;
    c->params = *p;
    return FMM_OK;
}

extern "C" fmm_status fmm_get_params(const fmm_ctx* c, fmm_params* p)
{
    if (!c || !p) return fail(FMM_ERR_ARG, "NULL argument");
    *p = c->params;
    return FMM_OK;
}

static fmm_status ensure_cells(fmm_ctx* c, long long need_cells);

static fmm_status ensure_tree(fmm_ctx* c, long long n, int bucket, int nbox = 1, long long min_cells = 0)
{
    DevTree& t = c->t;
    if (n > t.cap_n) {
        t.cap_n = 0;
        long long cap = n;
        CK(alloc(&t.key, cap));
        CK(alloc(&t.key_alt, cap));
        CK(alloc(&t.idx, cap));
        CK(alloc(&t.idx_alt, cap));
        CK(alloc(&t.bm_bin, fmm_bmax_bins(cap)));
        CK(alloc(&t.bm_binbase, fmm_bmax_bins(cap)));
        CK(alloc(&t.sx, cap));
        CK(alloc(&t.sy, cap));
        CK(alloc(&t.sz, cap));
        CK(alloc(&t.sm, cap));
        CK(alloc(&t.sact, cap));
        CK(alloc(&t.posf, cap));
        CK(alloc(&t.plo, cap));
        CK(alloc(&t.off, cap));
        CK(alloc(&t.act, cap));
        CK(alloc(&t.bucket_of, cap));
        CK(alloc(&t.bflag, cap));
        // the radix tree's arrays share one block of 32 bytes per particle with the input records,
        // which the gather reads before the radix tree writes them
        CK(alloc(&t.radix, 8 * cap));
        t.ifirst = t.radix;
        t.ilast = t.radix + cap;
        t.ileft = t.radix + 2 * cap;
        t.iright = t.radix + 3 * cap;
        t.nparent = t.radix + 4 * cap;
        t.keep = reinterpret_cast<unsigned int*>(t.radix + 6 * cap);
        t.src = reinterpret_cast<SrcRec*>(t.radix);
        t.cap_n = cap;
    }
    // the cells themselves are sized by build_tree once the tree's cell count is known; callers
    // that append more cells (the dual trees' fixed tree) ask for min_cells here
    CK(fmm_sort_ensure(t, n));
    return ensure_cells(c, min_cells);
}

// Cell arrays for at least need cells.
static fmm_status ensure_cells(fmm_ctx* c, long long need_cells)
{
    DevTree& t = c->t;
    if (!t.ewald_L) CK(alloc(&t.ewald_L, fmm_ewald_floats()));
    if (need_cells > t.cap_cells) {
        t.cap_cells = 0;
        long long cap = need_cells;
        CK(alloc(&t.cfirst, cap));
        CK(alloc(&t.ccount, cap));
        CK(alloc(&t.cparent, cap));
        CK(alloc(&t.cchild, 2 * cap));
        CK(alloc(&t.cnact, cap));
        CK(alloc(&t.bucket_cell, cap));
        CK(alloc(&t.arrive, cap));
        CK(alloc(&t.com, cap));
        CK(alloc(&t.cen, 2 * cap));
        CK(alloc(&t.clo, 3 * cap));
        CK(alloc(&t.chi, 3 * cap));
        CK(alloc(&t.bmax, cap));
        CK(alloc(&t.rec, (long long)FMM_NREC * cap));
        CK(alloc(&t.node, cap));
        CK(alloc(&t.mnorm, cap));
        CK(alloc(&t.amin, cap));
        CK(alloc(&t.bm_cnt, cap));
        CK(alloc(&t.bm_base, cap));
        CK(alloc(&t.bm32, cap));
        CK(alloc(&t.bm64, cap));
        CK(alloc(&t.L, (long long)FMM_NL * cap));
        t.cap_cells = cap;
    }
    return FMM_OK;
}

// Every counter of a solve starts at zero, except the compressed kick-drift's status word, which
// waits for the next solve to report it.
static cudaError_t clear_counters(fmm_ctx* c, cudaStream_t s)
{
    const size_t k = offsetof(DevCounters, kdk_status);
    cudaError_t e = cudaMemsetAsync(c->ctr, 0, k, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(reinterpret_cast<char*>(c->ctr) + k + sizeof(unsigned int), 0,
                            sizeof(DevCounters) - k - sizeof(unsigned int), s);
    return e;
}

static fmm_status read_status(fmm_ctx* c, const char* where)
{
    if (c->ctr_h->kdk_status & FMM_DEV_ERR_ARG) {
        c->ctr_h->kdk_status = 0;
        CK(cudaMemsetAsync(&c->ctr->kdk_status, 0, sizeof(unsigned int), c->stream));
        return fail(FMM_ERR_ARG, "%s: the last fmm_kick_drift_i32 kept a particle from leaving the isolated box",
                    where);
    }
    unsigned int st = c->ctr_h->status;
    if (st & FMM_DEV_ERR_ARG)
        return fail(FMM_ERR_ARG, "%s: a position outside [0,1), or a mass that is not finite and > 0", where);
    if (st & FMM_DEV_ERR_TIMEOUT) return fail(FMM_ERR_TIMEOUT, "%s: a bounded device wait gave up", where);
    if (st & FMM_DEV_ERR_NUMERIC) return fail(FMM_ERR_NUMERIC, "%s: non-finite result", where);
    return FMM_OK;
}

static fmm_status set_boxes_check(long long n, const long long* off, int nbox)
{
    if (nbox < 1 || nbox > 256) return fail(FMM_ERR_ARG, "nbox must be in [1, 256], got %d", nbox);
    if (off) {
        if (off[0] != 0 || off[nbox] != n) return fail(FMM_ERR_ARG, "box offsets must start at 0 and end at n");
        for (int b = 0; b < nbox; b++)
            if (off[b + 1] < off[b]) return fail(FMM_ERR_ARG, "box offsets must not decrease");
    } else if (nbox != 1) {
        return fail(FMM_ERR_ARG, "box offsets are required for several boxes");
    }
    return FMM_OK;
}

static fmm_status set_boxes(fmm_ctx* c, long long n, const long long* off, int nbox)
{
    DevTree& t = c->t;
    fmm_status st = set_boxes_check(n, off, nbox);
    if (st != FMM_OK) return st;
    t.nbox = nbox;
    if (nbox == 1) return FMM_OK;
    if (nbox + 1 > t.cap_box) {
        t.cap_box = 0;
        CK(alloc(&t.box_off, nbox + 1));
        CK(alloc(&t.box_root, nbox + 1));
        if (t.box_off_h) cudaFreeHost(t.box_off_h);
        t.box_off_h = nullptr;
        CK(cudaMallocHost(&t.box_off_h, sizeof(long long) * (size_t)(nbox + 1)));
        t.cap_box = nbox + 1;
    }
    if (n > t.cap_box_n) {
        t.cap_box_n = 0;
        CK(alloc(&t.sbox, n));
        CK(alloc(&t.key_orig, n));
        t.cap_box_n = n;
    }
    memcpy(t.box_off_h, off, sizeof(long long) * (size_t)(nbox + 1));
    CK(cudaMemcpyAsync(t.box_off, t.box_off_h, sizeof(long long) * (size_t)(nbox + 1), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemsetAsync(t.box_root, 0xff, sizeof(int) * (size_t)nbox, c->stream));
    return FMM_OK;
}

static fmm_status build_tree(fmm_ctx* c, const double* pos, const float* mass, const unsigned char* active,
                             long long n, int bucket, const long long* box_off = nullptr, int nbox = 1)
{
    DevTree& t = c->t;
    cudaStream_t s = c->stream;
    fmm_status st = ensure_tree(c, n, bucket, nbox);
    if (st != FMM_OK) return st;
    st = set_boxes(c, n, box_off, nbox);
    if (st != FMM_OK) return st;
    c->have_tree = false;
    CK(clear_counters(c, s));
    CK(fmm_launch_keys(t, pos, mass, active, n, c->ctr, s, c->cur_ipos));
    if (nbox > 1) {
        CK(fmm_launch_box_sort(t, n, s));
        c->launches += 8 * 5 + 1 + 2 * 5 + 1;
    } else {
        CK(fmm_radix_sort(t, n, s));
        c->launches += 8 * 5;
    }
    CK(fmm_launch_gather(t, n, c->ctr, s));
    CK(fmm_launch_radix_tree(t, n, bucket, s));
    CK(fmm_scan_exclusive(t.keep, t.keep, 2 * n - 1, c->totals, t, s));
    // the cell count, then cell arrays for it (a small margin lets graph replays of a slowly
    // changing box keep their buffers; a replay with more cells than that is solved eagerly)
    CK(cudaMemcpyAsync(c->totals_h, c->totals, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    {
        const long long nc = c->totals_h[0];
        const fmm_status se = ensure_cells(c, nc + nc / 32 + 64);
        if (se != FMM_OK) return se;
        if (t.grade_key) CK(grow(&t.nogroup, &t.cap_nogroup, t.cap_cells));  // a graded build's per-cell flags
    }
    CK(cudaMemsetAsync(t.bflag, 0, sizeof(unsigned int) * (size_t)n, s));
    CK(fmm_launch_cells(t, n, bucket, s));
    // bucket ids: exclusive scan of the bucket start flags into keep[] (free after k_cells)
    CK(fmm_scan_exclusive(t.bflag, t.keep, n, c->totals + 1, t, s));
    CK(fmm_launch_bucket_index(t, n, s));
    CK(fmm_launch_depth(t, c->totals, c->ctr, s));
    CK(cudaMemcpyAsync(c->totals_h, c->totals, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->ctr_h, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    st = read_status(c, "fmm_build_tree");
    if (st != FMM_OK) return st;
    t.n = n;
    t.n_cells = c->totals_h[0];
    t.n_buckets = c->totals_h[1];
    if (t.n_cells > t.cap_cells) return fail(FMM_ERR_CUDA, "internal: %lld cells exceed capacity", t.n_cells);
    {
        const long long need = fmm_bmax_items_bound(n, (int)c->ctr_h->depth, t.n_cells);
        if (need > t.cap_bm_items) {
            t.cap_bm_items = 0;
            CK(alloc(&t.bm_item, need));
            CK(alloc(&t.bm_imax, need));
            CK(alloc(&t.bm_order, need));
            t.cap_bm_items = need;
        }
    }
    CK(fmm_launch_upward(t, n, bucket, c->ctr, s));
    if (nbox > 1) {
        CK(fmm_launch_box_roots(t, s));
        c->launches += 1;
    }
    // keys, gather, radix tree + keep, scan, cells, scan, bucket index, depth, bucket cells,
    // upward, exact b_max (count, scan, expand, item order: count, scan, place; two passes, final)
    c->launches += 1 + 1 + (n > 1 ? 2 : 1) + 3 + 1 + 3 + 1 + 1 + 2 + 13;
    t.depth = (int)c->ctr_h->depth;
    t.graded = t.grade_key != nullptr && n > 1;
    c->have_tree = true;
    c->theta_nodes = -1.0f;
    return FMM_OK;
}

static fmm_status check_common(fmm_ctx* c, const double* pos, const float* mass, long long n)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    if (!pos || !mass) return fail(FMM_ERR_ARG, "pos and mass must not be NULL");
    if (n < 1 || n >= (1LL << 31)) return fail(FMM_ERR_ARG, "n must be in [1, 2^31), got %lld", n);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(FMM_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return FMM_OK;
}

extern "C" fmm_status fmm_build_tree(fmm_ctx* c, const double* pos, const float* mass, const unsigned char* active,
                                     long long n, const fmm_params* p)
{
    fmm_status st = check_common(c, pos, mass, n);
    if (st != FMM_OK) return st;
    const fmm_params* q = p ? p : &c->params;
    st = check_params(q);
    if (st != FMM_OK) return st;
    c->have_solve = false;
    return build_tree(c, pos, mass, active, n, q->bucket);
}

// What a walk asks of its buffers beyond their starting sizes: per list a minimum capacity in
// entries (0: the starting size), and a factor on the per-warp scratch.
struct WalkNeed {
    long long cl = 0, pp = 0, pc = 0, cc = 0, cp = 0, groups = 0;
    long long scratch_scale = 1;
};

static fmm_status ensure_walk(fmm_ctx* c, long long n, int group, const WalkNeed& more)
{
    DevWalk& w = c->w;
    const long long cells = c->t.cap_cells;
    const long long need_front = cells;
    // Starting capacities per particle, from the NFW and clustered boxes measured here (per
    // particle: PP entries 1.8, PC 5.2; local entries 4.4 multipole and 3.4 point sources in the
    // NFW halo, 7.8 and none in the clustered 512^3 box; a level's checklists under 5):
    // checklists 8, PP 3, PC 8, local entries 8 multipole and 4 point sources, and 8192 scratch
    // entries per warp and list (fmm_debug_walk_capacity may start them smaller).  Groups: in a
    // plain tree they are one more than the cells with more than g particles, which no multiple of
    // n / (g + 1) bounds (a chain of such cells may shed a few particles per level); measured
    // 2.3 n / (g + 1) in a 20000-particle NFW halo and 1.7 in one of 2^21, so they start at
    // 4 n / (g + 1) (graded trees take the cell count).  A walk that overflows asks for what its
    // counters show it needed (run_walk).
    const long long ls = c->dbg_list_scale > 0 ? c->dbg_list_scale : 8;
    const long long floor = c->dbg_list_scale > 0 ? 4096 : 65536;  // small boxes have longer lists per particle
    long long need_cl = std::max(ls * n + floor, more.cl);
    long long need_pp = std::max((c->dbg_list_scale > 0 ? (ls + 1) / 2 : 3) * n + floor, more.pp);
    long long need_pc = std::max(ls * n + floor, more.pc);
    long long need_cc = std::max((c->dbg_list_scale > 0 ? ls : 8) * n + floor, more.cc);
    long long need_cp = std::max((c->dbg_list_scale > 0 ? ls : 4) * n + floor, more.cp);
    long long need_scr = (c->dbg_scratch > 0 ? c->dbg_scratch : 8192LL) * more.scratch_scale;
    long long need_groups =
        std::max(c->t.graded ? cells : 4 * n / (group + 1) + 64 + 2LL * c->t.nbox, more.groups);
    if (need_groups > cells) need_groups = cells;
    if (need_front > w.cap_front) {
        w.cap_front = 0;
        for (int i = 0; i < 2; i++) {
            CK(alloc(&w.f_cell[i], need_front));
            CK(alloc(&w.f_cloff[i], need_front));
            CK(alloc(&w.f_cllen[i], need_front));
        }
        CK(alloc(&w.lcc_off, need_front));
        CK(alloc(&w.lcc_len, need_front));
        CK(alloc(&w.lcp_off, need_front));
        CK(alloc(&w.lcp_len, need_front));
        CK(alloc(&w.wcells, need_front));
        w.cap_front = need_front;
    }
    if (need_groups > w.cap_groups) {
        w.cap_groups = 0;
        CK(alloc(&w.groups, need_groups));
        CK(alloc(&w.Lg, (long long)FMM_NL * need_groups));
        CK(alloc(&w.cnt_pp, need_groups));
        CK(alloc(&w.cnt_pc, need_groups));
        CK(alloc(&w.base_pp, need_groups));
        CK(alloc(&w.base_pc, need_groups));
        w.cap_groups = need_groups;
    }
    if (need_cl > w.cap_cl) {
        w.cap_cl = 0;
        CK(alloc(&w.cl[0], need_cl));
        CK(alloc(&w.cl[1], need_cl));
        w.cap_cl = need_cl;
    }
    if (need_pp > w.cap_pp) {
        w.cap_pp = 0;
        CK(alloc(&w.pp, need_pp));
        w.cap_pp = need_pp;
    }
    if (need_pc > w.cap_pc) {
        w.cap_pc = 0;
        CK(alloc(&w.pc, need_pc));
        w.cap_pc = need_pc;
    }
    if (need_cc > w.cap_cc) {
        w.cap_cc = 0;
        CK(alloc(&w.cc, need_cc));
        CK(alloc(&w.cc_sink, need_cc));
        w.cap_cc = need_cc;
    }
    if (need_cp > w.cap_cp) {
        w.cap_cp = 0;
        CK(alloc(&w.cp, need_cp));
        CK(alloc(&w.cp_sink, need_cp));
        w.cap_cp = need_cp;
    }
    if (need_scr > w.cap_scratch) {
        w.cap_scratch = 0;
        CK(alloc(&w.scratch, (long long)w.n_warps * 5 * need_scr));
        w.cap_scratch = need_scr;
    }
    return FMM_OK;
}

// The encoding of the coming walk's list entries: for a periodic box (Sec. 3.1, periodic
// boundaries) the replica shell and the index bits, which must leave room for the copy code above
// them; isolated solves reset it.
static fmm_status set_periodic(fmm_ctx* c, const fmm_params& q, long long n, int nbox)
{
    DevTree& t = c->t;
    t.per_R = 0;
    t.per_ib = 31;
    // the learned walk marks cell entries with the network's decision in bits 29 and 30
    if (q.criterion == 1 && t.cap_cells >= (1LL << 29))
        return fail(FMM_ERR_ARG, "the learned criterion holds at most 2^29 cells, the tree may have %lld", t.cap_cells);
    if (q.nrep == 0) return FMM_OK;
    if (nbox != 1) return fail(FMM_ERR_ARG, "a periodic solve (nrep %d) takes one box, got %d", q.nrep, nbox);
    if (q.criterion != 0) return fail(FMM_ERR_ARG, "a periodic solve (nrep %d) takes the fixed criterion", q.nrep);
    const long long W = 2 * q.nrep + 1, copies = W * W * W;
    const long long span = std::max(n, t.cap_cells);
    int ib = 1;
    while ((1LL << ib) < span) ib++;
    if (((copies - 1) << ib) >= (1LL << 31))
        return fail(FMM_ERR_ARG, "a periodic solve with nrep %d holds at most %lld particles and cells, got %lld", q.nrep,
                    (1LL << 31) / copies, span);
    t.per_R = q.nrep;
    t.per_ib = ib;
    return FMM_OK;
}

// The shifted-geometry tables of a periodic walk, sized for the tree's capacity (eager solves
// only: a captured graph reuses what the eager solve before it allocated).
static fmm_status ensure_periodic(fmm_ctx* c)
{
    DevTree& t = c->t;
    if (t.per_R <= 0) return FMM_OK;
    const long long w2 = 2 * t.per_R;
    CK(grow(&t.cshift, &t.cap_cshift, t.cap_cells * 3 * w2));
    CK(grow(&t.pshift, &t.cap_pshift, t.cap_n * 3 * w2));
    return FMM_OK;
}

// Fork the Ewald sub-cube expansions onto the side stream once the tree (the root's moments) is
// on the context's stream; ewald_join makes the context's stream wait for them.  Nothing to do for
// an isolated box or without the correction term.
static bool ewald_on(const fmm_ctx* c, int terms) { return c->t.per_R > 0 && (terms & 8); }

static fmm_status ewald_fork(fmm_ctx* c, int terms)
{
    if (!ewald_on(c, terms)) return FMM_OK;
    if (!c->ew_stream) CK(cudaStreamCreateWithFlags(&c->ew_stream, cudaStreamNonBlocking));
    if (!c->ew_fork) CK(cudaEventCreateWithFlags(&c->ew_fork, cudaEventDisableTiming));
    if (!c->ew_join) CK(cudaEventCreateWithFlags(&c->ew_join, cudaEventDisableTiming));
    CK(cudaEventRecord(c->ew_fork, c->stream));
    CK(cudaStreamWaitEvent(c->ew_stream, c->ew_fork, 0));
    CK(fmm_launch_ewald_grid(c->t, terms, c->ew_stream));
    CK(cudaEventRecord(c->ew_join, c->ew_stream));
    c->launches += 1;
    return FMM_OK;
}

static fmm_status ewald_join(fmm_ctx* c, int terms)
{
    if (!ewald_on(c, terms)) return FMM_OK;
    CK(cudaStreamWaitEvent(c->stream, c->ew_join, 0));
    CK(fmm_launch_ewald_groups(c->t, c->w, c->ctr, terms, c->stream));
    c->launches += 1;
    return FMM_OK;
}

// The walk's levels on the context's stream, and the local expansions of every level.
//
// A walk of many sinks (at least FMM_LOCAL_SIDE_SINKS in the context's previous walk) forks each level's
// expansions onto a side stream as soon as the level's walk kernel ends, to run beside the levels
// below; the context's stream joins the side stream before the groups take their expansions.
// There the walk warps leave the FMA pipes idle while they wait on loads.  A smaller walk is bound
// by its longest chains of dependent steps instead, and kernels running beside it lengthen them:
// measured on one GB300, the side stream took the 512^3 box's walk phase from 155.6 to 144.8 ms
// (6.8 M sinks) and the 128^3 NFW box's from 4.1 to 5.2 ms (0.1 M sinks), so a smaller walk runs
// the expansions after its last level.  Grids follow the previous walk's counts (full persistent
// grids for the context's first walk).
#ifndef FMM_LOCAL_SIDE_SINKS
#define FMM_LOCAL_SIDE_SINKS (1LL << 22)
#endif
static fmm_status walk_levels(fmm_ctx* c, WalkArgs& a, int levels)
{
    DevTree& t = c->t;
    DevWalk& w = c->w;
    cudaStream_t s = c->stream;
    const bool prev = c->have_counts;
    long long prev_sinks = 0;
    if (prev)
        for (int L = 0; L < FMM_MAX_LEVELS; L++) prev_sinks += c->prev_front[L];
    const long long side_from = c->side_sinks >= 0 ? c->side_sinks : FMM_LOCAL_SIDE_SINKS;
    if (!prev || prev_sinks < side_from) {
        for (int L = 0; L < levels; L++) {
            a.level = L;
            a.level_parity = L & 1;
            CK(fmm_launch_walk_level(t, w, c->ctr, a, s));
            c->launches += 1;
        }
        const LocalGrids g = fmm_local_grids(w, prev ? c->prev_cc_len : -1, prev ? c->prev_cp_len : -1, -1);
        CK(fmm_launch_local_level(t, w, c->ctr, a.eps2, -1, levels, g, s));
        c->launches += 2 + levels;
    } else {
        for (int L = 0; L < levels; L++) {
            a.level = L;
            a.level_parity = L & 1;
            CK(fmm_launch_walk_level(t, w, c->ctr, a, s));
            CK(cudaEventRecord(c->loc_fork, s));
            CK(cudaStreamWaitEvent(c->loc_stream, c->loc_fork, 0));
            const LocalGrids g = fmm_local_grids(w, c->prev_cc[L], c->prev_cp[L], c->prev_front[L]);
            CK(fmm_launch_local_level(t, w, c->ctr, a.eps2, L, levels, g, c->loc_stream));
            c->launches += 1 + 3;
        }
        CK(cudaEventRecord(c->loc_join, c->loc_stream));
        CK(cudaStreamWaitEvent(s, c->loc_join, 0));
    }
    CK(fmm_launch_local_groups(w, t, c->ctr, s));
    c->launches += 1;
    return FMM_OK;
}

static fmm_status run_walk(fmm_ctx* c, long long n, double eps, int bucket, int group, int mode = 0)
{
    DevTree& t = c->t;
    DevWalk& w = c->w;
    cudaStream_t s = c->stream;
    WalkArgs a;
    float e2 = (float)(2.0 * eps);
    a.four_eps2 = e2 * e2;
    a.eps2 = (float)(eps * eps);
    a.bucket = bucket;
    a.group = group;
    a.eps = (float)eps;
    a.mode = mode;
    a.band_lo = (float)c->params.band_lo;
    a.band_hi = (float)c->params.band_hi;
    a.tau = (float)c->params.mlp_tau;
    a.margin = (float)c->params.mlp_margin;
    a.mlp_packed = c->mlp_packed;
    a.audit_pairs = c->audit_pairs;
    a.audit_cap = c->audit_cap;
    // groups sit at most at the deepest cell level: depth + 1 levels, no host round trip between them
    const int levels = t.depth + 1;
    if (levels + 1 > FMM_MAX_LEVELS) return fail(FMM_ERR_STATE, "tree depth %d exceeds the walk's levels", t.depth);
    WalkNeed more;
    for (int attempt = 0;; attempt++) {
        fmm_status st = ensure_walk(c, n, group, more);
        if (st != FMM_OK) return st;
        CK(cudaMemsetAsync(&c->ctr->overflow, 0, sizeof(unsigned int), s));
        // cells above a box's root are never walked: their local lists must read as empty
        CK(cudaMemsetAsync(w.lcc_len, 0, sizeof(int) * (size_t)t.n_cells, s));
        CK(cudaMemsetAsync(w.lcp_len, 0, sizeof(int) * (size_t)t.n_cells, s));
        CK(cudaMemsetAsync(&c->ctr->n_groups, 0, sizeof(DevCounters) - offsetof(DevCounters, n_groups), s));
        CK(fmm_launch_walk_seed(t, w, c->ctr, s, c->second_root));
        c->launches += 1;
        {
            const fmm_status sw = walk_levels(c, a, levels);
            if (sw != FMM_OK) return sw;
        }
        {
            const fmm_status se = ewald_join(c, c->params.terms);
            if (se != FMM_OK) return se;
        }
        CK(cudaMemcpyAsync(c->ctr_h, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!c->ctr_h->overflow) {
            if (c->ctr_h->lv_front[levels] != 0) return fail(FMM_ERR_STATE, "walk went below the deepest cell");
            long long used = 0;
            while (used < levels && c->ctr_h->lv_front[used] > 0) used++;
            w.n_levels = used;
            w.n_groups = (long long)c->ctr_h->n_groups;
            w.pp_len = (long long)c->ctr_h->pp_len;
            w.pc_len = (long long)c->ctr_h->pc_len;
            w.cc_len = (long long)c->ctr_h->cc_len;
            w.cp_len = (long long)c->ctr_h->cp_len;
            c->stats.retries = attempt;
            for (int L = 0; L < FMM_MAX_LEVELS; L++) {
                c->prev_front[L] = (long long)c->ctr_h->lv_front[L];
                c->prev_cc[L] = (long long)c->ctr_h->lv_cc[L];
                c->prev_cp[L] = (long long)c->ctr_h->lv_cp[L];
            }
            c->prev_cc_len = w.cc_len;
            c->prev_cp_len = w.cp_len;
            c->have_counts = true;
            return FMM_OK;
        }
        if (attempt >= 8) return fail(FMM_ERR_OOM, "walk lists keep overflowing after %d grows", attempt);
        // The list counters kept counting past the capacities: a list that overflowed grows to what
        // this walk asked of it plus an eighth, and at least doubles (a checklist or scratch
        // overflow hides the sinks below it, so the next walk may ask for much more); the lists
        // that fitted keep their size.  An overflow that no counter shows was the per-warp scratch,
        // which doubles; scratch started below its default size (fmm_debug_walk_capacity) doubles
        // at every overflow.
        {
            const DevCounters& h = *c->ctr_h;
            bool seen = false;
            auto grow_to = [&](unsigned long long used, long long cap, long long& need) {
                if ((long long)used > cap) {
                    need = std::max(need, std::max((long long)used + (long long)used / 8 + 4096, 2 * cap));
                    seen = true;
                }
            };
            grow_to(h.pp_len, w.cap_pp, more.pp);
            grow_to(h.pc_len, w.cap_pc, more.pc);
            grow_to(h.cc_len, w.cap_cc, more.cc);
            grow_to(h.cp_len, w.cap_cp, more.cp);
            grow_to(h.n_groups, w.cap_groups, more.groups);
            for (int l = 0; l <= levels; l++) grow_to(h.lv_cl[l], w.cap_cl, more.cl);
            if (!seen || w.cap_scratch < 8192) more.scratch_scale *= 2;
        }
    }
}

static fmm_status finish_stats(fmm_ctx* c, long long n);
static fmm_status interact_and_finish(fmm_ctx* c, const fmm_params& q, double eps, float* acc, float* pot,
                                      long long n_out, long long n_stats, const unsigned int* perm);

static fmm_status solve_eager(fmm_ctx* c, const double* pos, const float* mass, const unsigned char* active, long long n,
                        double eps, double theta, float* acc, float* pot, const long long* box_off = nullptr,
                        int nbox = 1)
{
    fmm_params q = c->params;
    q.eps = eps;
    q.theta = theta;
    fmm_status st = check_params(&q);
    if (st != FMM_OK) return st;
    if (!acc) return fail(FMM_ERR_ARG, "acc must not be NULL");
    cudaStream_t s = c->stream;
    c->have_solve = false;
    memset(&c->stats, 0, sizeof c->stats);
    c->launches = 0;
    CK(cudaEventRecord(c->ev[0], s));
    st = build_tree(c, pos, mass, active, n, q.bucket, box_off, nbox);
    if (st != FMM_OK) return st;
    st = set_periodic(c, q, n, nbox);
    if (st == FMM_OK) st = ensure_periodic(c);
    if (st != FMM_OK) return st;
    c->stats.n_active = (long long)c->ctr_h->n_active;
    CK(fmm_launch_nodes(c->t, theta, s));
    c->launches += 1;
    if (c->t.per_R > 0) {
        CK(fmm_launch_shift_tables(c->t, s));
        c->launches += 1;
    }
    st = ewald_fork(c, q.terms);
    if (st != FMM_OK) return st;
    CK(cudaEventRecord(c->ev[1], s));
    if (q.criterion == 1) {
        if (!c->mlp_ready) return fail(FMM_ERR_STATE, "criterion 1 needs network parameters");
        // the acceleration estimate held by acc on entry sets each sink cell's error scale
        CK(fmm_launch_cell_amin(c->t, acc, n, s));
        c->launches += 1;
    }
    st = run_walk(c, n, eps, q.bucket, q.group, q.criterion);
    if (st != FMM_OK) return st;
    return interact_and_finish(c, q, eps, acc, pot, n, n, nullptr);
}

// After the walk: work items, PP, PC, and the sums plus local expansion written to acc/pot
// (n_out particles long, in the order perm gives; NULL: the tree's own order); then the counters
// and timing events are read back.
static fmm_status interact_and_finish(fmm_ctx* c, const fmm_params& q, double eps, float* acc, float* pot,
                                      long long n_out, long long n_stats, const unsigned int* perm)
{
    cudaStream_t s = c->stream;
    fmm_status st;
    CK(cudaEventRecord(c->ev[2], s));
    InteractArgs ia;
    ia.eps2 = (float)(eps * eps);
    ia.terms = q.terms;
    ia.accumulate = q.accumulate;
    ia.chunk = q.list_chunk ? q.list_chunk : FMM_LIST_CHUNK;
    if (c->w.n_groups > 0) {
        // work items: at most one partial chunk per group beyond the full chunks
        DevWalk& w = c->w;
        long long need_pp = w.pp_len / ia.chunk + w.n_groups + 1;
        long long need_pc = w.pc_len / ia.chunk + w.n_groups + 1;
        if (need_pp > w.cap_item_pp) {
            w.cap_item_pp = 0;
            CK(alloc(&w.item_pp, need_pp));
            CK(alloc(&w.part_pp, need_pp * FMM_GMAX));
            w.cap_item_pp = need_pp;
        }
        if (need_pc > w.cap_item_pc) {
            w.cap_item_pc = 0;
            CK(alloc(&w.item_pc, need_pc));
            CK(alloc(&w.part_pc, need_pc * FMM_GMAX));
            w.cap_item_pc = need_pc;
        }
        CK(fmm_launch_items(c->t, w, c->ctr, ia.chunk, s));
        c->launches += 3 + 2 * 3;
        CK(fmm_launch_pp(c->t, c->w, c->ctr, ia, s));
        CK(cudaEventRecord(c->ev[3], s));
        CK(fmm_launch_pc(c->t, c->w, c->ctr, ia, s));
        CK(cudaEventRecord(c->ev[4], s));
        CK(fmm_launch_l2p_out(c->t, c->w, c->ctr, ia, acc, pot, n_out, s, perm));
        c->launches += ((q.terms & 1) ? 1 : 0) + ((q.terms & 2) ? 1 : 0) + 1;
    } else {
        CK(cudaEventRecord(c->ev[3], s));
        CK(cudaEventRecord(c->ev[4], s));
    }
    CK(cudaEventRecord(c->ev[5], s));
    CK(cudaMemcpyAsync(c->ctr_h, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    st = read_status(c, "fmm_compute_forces");
    if (st != FMM_OK) return st;
    return finish_stats(c, n_stats);
}

static fmm_status finish_stats(fmm_ctx* c, long long n)
{
    fmm_stats& S = c->stats;
    S.n = n;
    S.n_cells = c->t.n_cells;
    S.n_buckets = c->t.n_buckets;
    S.n_groups = c->w.n_groups;
    S.n_levels = c->w.n_levels;
    S.n_pp_pairs = (long long)c->ctr_h->n_pp_pairs;
    S.n_pc_pairs = (long long)c->ctr_h->n_pc_pairs;
    S.n_cc = (long long)c->ctr_h->n_cc;
    S.n_cp = (long long)c->ctr_h->n_cp;
    S.n_pp_entries = c->w.pp_len;
    S.n_pc_entries = c->w.pc_len;
    float ms[6] = {};
    const int from[6] = {0, 1, 2, 3, 4, 0}, to[6] = {1, 2, 3, 4, 5, 5};
    for (int i = 0; i < 6; i++) CK(cudaEventElapsedTime(&ms[i], c->ev[from[i]], c->ev[to[i]]));
    S.ms_tree = ms[0];
    S.ms_walk = ms[1];
    S.ms_pp = ms[2];
    S.ms_pc = ms[3];
    S.ms_l2p = ms[4];
    S.ms_total = ms[5];
    S.paper_flops = 53.0 * S.n_pp_pairs + 215.0 * S.n_pc_pairs + 479.0 * S.n_cc + 213.0 * S.n_cp;
    S.kernel_flops_pp = 19.0 * S.n_pp_pairs;
    S.kernel_flops_pc = (double)FMM_FLOPS_PC * S.n_pc_pairs;
    S.n_launches = c->launches;
    S.n_learned = (long long)c->ctr_h->n_mlp;
    c->have_solve = true;
    return FMM_OK;
}

// ---------------------------------------------------------------- CUDA graph of a solve

// Enqueue the solve for capture in two parts.  The head (keys, sort, gather, radix tree and the
// scan of the kept nodes) ends with the cell count copied to the host: a replay checks it against
// the cell buffers before the rest runs, since every later kernel indexes cells by that count.  The
// rest makes the same launches as solve_eager, with every launch over cells, buckets or groups
// covering the capacity (kernels read the counts on the device) and the walk run for graph_levels
// levels (levels past the deepest cell find an empty front).  Used only inside stream capture,
// after an eager solve has sized every buffer.
static fmm_status enqueue_graph_head(fmm_ctx* c, const double* pos, const float* mass, const unsigned char* active,
                                     long long n, const fmm_params& q, const long long* box_off, int nbox)
{
    DevTree& t = c->t;
    cudaStream_t s = c->stream;
    c->launches = 0;
    CK(cudaEventRecordWithFlags(c->ev[0], s, cudaEventRecordExternal));
    fmm_status st = set_boxes(c, n, box_off, nbox);
    if (st != FMM_OK) return st;
    st = set_periodic(c, q, n, nbox);
    if (st != FMM_OK) return st;
    CK(clear_counters(c, s));
    CK(fmm_launch_keys(t, pos, mass, active, n, c->ctr, s, c->cur_ipos));
    if (nbox > 1) {
        CK(fmm_launch_box_sort(t, n, s));
        c->launches += 8 * 5 + 1 + 2 * 5 + 1;
    } else {
        CK(fmm_radix_sort(t, n, s));
        c->launches += 8 * 5;
    }
    CK(fmm_launch_gather(t, n, c->ctr, s));
    CK(fmm_launch_radix_tree(t, n, q.bucket, s));
    CK(fmm_scan_exclusive(t.keep, t.keep, 2 * n - 1, c->totals, t, s));
    CK(cudaMemcpyAsync(c->totals_h, c->totals, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    c->launches += 1 + 1 + (n > 1 ? 2 : 1) + 3;
    return FMM_OK;
}

static fmm_status enqueue_graph_rest(fmm_ctx* c, long long n, const fmm_params& q, float* acc, float* pot, int nbox)
{
    DevTree& t = c->t;
    DevWalk& w = c->w;
    cudaStream_t s = c->stream;
    t.cap_grid = true;
    struct Reset {
        DevTree& t;
        ~Reset() { t.cap_grid = false; }
    } reset{t};
    CK(cudaMemsetAsync(t.bflag, 0, sizeof(unsigned int) * (size_t)n, s));
    CK(fmm_launch_cells(t, n, q.bucket, s));
    CK(fmm_scan_exclusive(t.bflag, t.keep, n, c->totals + 1, t, s));
    CK(fmm_launch_bucket_index(t, n, s));
    CK(fmm_launch_depth(t, c->totals, c->ctr, s));
    CK(fmm_launch_upward(t, n, q.bucket, c->ctr, s));
    if (nbox > 1) {
        CK(fmm_launch_box_roots(t, s));
        c->launches += 1;
    }
    c->launches += 1 + 3 + 1 + 1 + 2 + 13;
    CK(fmm_launch_nodes(t, q.theta, s));
    c->launches += 1;
    if (t.per_R > 0) {
        if (!t.cshift || !t.pshift || t.cap_cshift < t.cap_cells * 3 * 2 * t.per_R ||
            t.cap_pshift < t.cap_n * 3 * 2 * t.per_R)
            return fail(FMM_ERR_STATE, "internal: periodic tables missing at capture");
        CK(fmm_launch_shift_tables(t, s));
        c->launches += 1;
    }
    fmm_status st = ewald_fork(c, q.terms);
    if (st != FMM_OK) return st;
    CK(cudaEventRecordWithFlags(c->ev[1], s, cudaEventRecordExternal));
    if (q.criterion == 1) {
        CK(fmm_launch_cell_amin(t, acc, n, s));
        c->launches += 1;
    }
    WalkArgs a;
    const float e2 = (float)(2.0 * q.eps);
    a.four_eps2 = e2 * e2;
    a.eps2 = (float)(q.eps * q.eps);
    a.bucket = q.bucket;
    a.group = q.group;
    a.eps = (float)q.eps;
    a.mode = q.criterion;
    a.band_lo = (float)q.band_lo;
    a.band_hi = (float)q.band_hi;
    a.tau = (float)q.mlp_tau;
    a.margin = (float)q.mlp_margin;
    a.mlp_packed = c->mlp_packed;
    a.audit_pairs = c->audit_pairs;
    a.audit_cap = c->audit_cap;
    // the overflow flag is not cleared here: the b_max items may have set it (the head cleared it)
    CK(cudaMemsetAsync(w.lcc_len, 0, sizeof(int) * (size_t)t.cap_cells, s));
    CK(cudaMemsetAsync(w.lcp_len, 0, sizeof(int) * (size_t)t.cap_cells, s));
    CK(cudaMemsetAsync(&c->ctr->n_groups, 0, sizeof(DevCounters) - offsetof(DevCounters, n_groups), s));
    CK(fmm_launch_walk_seed(t, w, c->ctr, s));
    c->launches += 1;
    st = walk_levels(c, a, c->graph_levels);
    if (st != FMM_OK) return st;
    st = ewald_join(c, q.terms);
    if (st != FMM_OK) return st;
    CK(cudaEventRecordWithFlags(c->ev[2], s, cudaEventRecordExternal));
    InteractArgs ia;
    ia.eps2 = (float)(q.eps * q.eps);
    ia.terms = q.terms;
    ia.accumulate = q.accumulate;
    ia.chunk = q.list_chunk ? q.list_chunk : FMM_LIST_CHUNK;
    CK(fmm_launch_items(t, w, c->ctr, ia.chunk, s));
    c->launches += 3 + 2 * 3;
    CK(fmm_launch_pp(t, w, c->ctr, ia, s));
    CK(cudaEventRecordWithFlags(c->ev[3], s, cudaEventRecordExternal));
    CK(fmm_launch_pc(t, w, c->ctr, ia, s));
    CK(cudaEventRecordWithFlags(c->ev[4], s, cudaEventRecordExternal));
    CK(fmm_launch_l2p_out(t, w, c->ctr, ia, acc, pot, n, s));
    c->launches += ((q.terms & 1) ? 1 : 0) + ((q.terms & 2) ? 1 : 0) + 1;
    CK(cudaEventRecordWithFlags(c->ev[5], s, cudaEventRecordExternal));
    CK(cudaMemcpyAsync(c->ctr_h, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->totals_h, c->totals, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    return FMM_OK;
}

static bool same_params(const fmm_params& a, const fmm_params& b)
{
    return a.theta == b.theta && a.eps == b.eps && a.bucket == b.bucket && a.group == b.group &&
           a.criterion == b.criterion && a.accumulate == b.accumulate && a.terms == b.terms &&
           a.list_chunk == b.list_chunk && a.spin_limit == b.spin_limit && a.mlp_tau == b.mlp_tau &&
           a.band_lo == b.band_lo && a.band_hi == b.band_hi && a.nrep == b.nrep && a.mlp_margin == b.mlp_margin;
}

static fmm_ctx::GraphKey make_key(const double* pos, const float* mass, const unsigned char* active, float* acc,
                                  float* pot, long long n, const long long* box_off, int nbox, const fmm_params& q,
                                  double eps, double theta)
{
    fmm_ctx::GraphKey k;
    k.pos = pos;
    k.i32 = false;
    k.mass = mass;
    k.active = active;
    k.acc = acc;
    k.pot = pot;
    k.n = n;
    k.nbox = nbox;
    if (box_off) k.off.assign(box_off, box_off + nbox + 1);
    k.p = q;
    k.eps = eps;
    k.theta = theta;
    return k;
}

static bool same_key(const fmm_ctx::GraphKey& a, const fmm_ctx::GraphKey& b)
{
    return a.pos == b.pos && a.i32 == b.i32 && a.mass == b.mass && a.active == b.active && a.acc == b.acc &&
           a.pot == b.pot &&
           a.n == b.n && a.nbox == b.nbox && a.off == b.off && same_params(a.p, b.p) && a.eps == b.eps &&
           a.theta == b.theta;
}

static void drop_graph(fmm_ctx* c)
{
    if (c->gexec_head) cudaGraphExecDestroy(c->gexec_head);
    c->gexec_head = nullptr;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
}

// One part of the solve captured on the context's capture stream and instantiated; null on any
// failure (the context then keeps solving eagerly).
template <class F>
static cudaGraphExec_t capture_part(fmm_ctx* c, F&& enqueue)
{
    if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    const fmm_status st = enqueue();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    c->stream = user;
    cudaGraphExec_t ge = nullptr;
    if (st != FMM_OK || e != cudaSuccess || !g || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) ge = nullptr;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return ge;
}

// Capture the solve just done eagerly (same arguments) into a graph; on any failure the context
// simply keeps solving eagerly.
static void capture_graph(fmm_ctx* c, const fmm_ctx::GraphKey& key, const double* pos, const float* mass,
                          const unsigned char* active, long long n, const fmm_params& q, float* acc, float* pot,
                          const long long* box_off, int nbox)
{
    drop_graph(c);
    if (c->w.n_groups < 1) return;
    // buffers the capacity-sized launches need, reserved now (no allocation may happen inside capture)
    if (fmm_scan_reserve(c->t, std::max(2 * n + 2, std::max(c->w.cap_groups, c->t.cap_cells))) != cudaSuccess) return;
    c->graph_levels = c->t.depth + 1 + 4;  // a few levels of slack for a slightly deeper tree
    if (c->graph_levels + 1 > FMM_MAX_LEVELS) return;
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        c->cap_stream = nullptr;
        cudaGetLastError();
        return;
    }
    // the work is recorded on the context's capture stream; replays launch on the caller's stream
    const int saved_launches = c->launches;
    cudaGraphExec_t head = capture_part(c, [&] { return enqueue_graph_head(c, pos, mass, active, n, q, box_off, nbox); });
    cudaGraphExec_t rest = head ? capture_part(c, [&] { return enqueue_graph_rest(c, n, q, acc, pot, nbox); }) : nullptr;
    c->graph_launches = c->launches;  // both parts
    c->launches = saved_launches;
    if (!head || !rest) {
        if (head) cudaGraphExecDestroy(head);
        if (rest) cudaGraphExecDestroy(rest);
        return;
    }
    c->gexec_head = head;
    c->gexec = rest;
    c->gkey = key;
    c->graph_bufs = tree_walk_buffers(c);
}

enum { GRAPH_DONE = 0, GRAPH_RETRY = 1 };

// Replay the captured solve; GRAPH_RETRY when a capacity or the level count was not enough (the
// eager path then repeats the solve, growing what it must).
static fmm_status replay_graph(fmm_ctx* c, long long n, int* outcome)
{
    *outcome = GRAPH_RETRY;
    cudaStream_t s = c->stream;
    DevTree& t = c->t;
    DevWalk& w = c->w;
    CK(cudaGraphLaunch(c->gexec_head, s));
    CK(cudaStreamSynchronize(s));
    if ((long long)c->totals_h[0] > t.cap_cells) return FMM_OK;  // more cells than the buffers hold
    CK(cudaGraphLaunch(c->gexec, s));
    CK(cudaStreamSynchronize(s));
    fmm_status st = read_status(c, "fmm_compute_forces");
    if (st != FMM_OK) return st;
    const DevCounters& h = *c->ctr_h;
    if (h.overflow || h.lv_front[c->graph_levels] != 0 || (long long)h.n_groups > w.cap_groups)
        return FMM_OK;
    t.n = n;
    t.n_cells = c->totals_h[0];
    t.n_buckets = c->totals_h[1];
    t.depth = (int)h.depth;
    long long used = 0;
    while (used < c->graph_levels && h.lv_front[used] > 0) used++;
    w.n_levels = used;
    w.n_groups = (long long)h.n_groups;
    w.pp_len = (long long)h.pp_len;
    w.pc_len = (long long)h.pc_len;
    w.cc_len = (long long)h.cc_len;
    w.cp_len = (long long)h.cp_len;
    c->have_tree = true;
    c->theta_nodes = -1.0f;
    memset(&c->stats, 0, sizeof c->stats);
    c->stats.n_active = (long long)h.n_active;
    c->launches = c->graph_launches;
    st = finish_stats(c, n);
    if (st != FMM_OK) return st;
    c->graph_replays++;
    *outcome = GRAPH_DONE;
    return FMM_OK;
}

static fmm_status solve(fmm_ctx* c, const double* pos, const float* mass, const unsigned char* active, long long n,
                        double eps, double theta, float* acc, float* pot, const long long* box_off = nullptr,
                        int nbox = 1)
{
    if (!c->graphs) return solve_eager(c, pos, mass, active, n, eps, theta, acc, pot, box_off, nbox);
    fmm_params q = c->params;
    q.eps = eps;
    q.theta = theta;
    fmm_status st = check_params(&q);
    if (st != FMM_OK) return st;
    if (!acc) return fail(FMM_ERR_ARG, "acc must not be NULL");
    if (q.criterion == 1 && !c->mlp_ready) return fail(FMM_ERR_STATE, "criterion 1 needs network parameters");
    st = set_boxes_check(n, box_off, nbox);
    if (st != FMM_OK) return st;
    fmm_ctx::GraphKey key = make_key(pos, mass, active, acc, pot, n, box_off, nbox, q, eps, theta);
    if (c->cur_ipos) {
        key.pos = c->cur_ipos;
        key.i32 = true;
    }
    // a graph holds the addresses of the context's buffers it was captured with: it replays only while
    // none of them was reallocated since (another call may have grown them)
    if (c->gexec && same_key(c->gkey, key) && c->graph_bufs == tree_walk_buffers(c)) {
        c->have_solve = false;
        int outcome = GRAPH_RETRY;
        st = replay_graph(c, n, &outcome);
        if (st != FMM_OK) {
            drop_graph(c);
            return st;
        }
        if (outcome == GRAPH_DONE) return FMM_OK;
        drop_graph(c);
    }
    st = solve_eager(c, pos, mass, active, n, eps, theta, acc, pot, box_off, nbox);
    if (st != FMM_OK) return st;
    const fmm_stats saved = c->stats;
    capture_graph(c, key, pos, mass, active, n, q, acc, pot, box_off, nbox);
    c->stats = saved;
    return FMM_OK;
}

extern "C" fmm_status fmm_set_graphs(fmm_ctx* c, int enable)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    if (enable != 0 && enable != 1) return fail(FMM_ERR_ARG, "enable must be 0 or 1");
    CK(cudaSetDevice(c->device));
    c->graphs = enable == 1;
    if (!c->graphs) drop_graph(c);
    return FMM_OK;
}

extern "C" fmm_status fmm_graph_info(const fmm_ctx* c, int* captured, long long* replays)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    if (captured) *captured = c->gexec ? 1 : 0;
    if (replays) *replays = c->graph_replays;
    return FMM_OK;
}

extern "C" fmm_status fmm_compute_forces(fmm_ctx* c, const double* pos, const float* mass,
                                         const unsigned char* active, long long n, double eps, double theta,
                                         float* acc, float* pot)
{
    fmm_status st = check_common(c, pos, mass, n);
    if (st != FMM_OK) return st;
    return solve(c, pos, mass, active, n, eps, theta, acc, pot);
}

extern "C" fmm_status fmm_autotune(fmm_ctx* c, const double* pos, const float* mass, long long n,
                                   const long long* box_offsets, int nbox, double eps, double theta,
                                   const fmm_params* candidates, int n_candidates, int reps, float* acc,
                                   fmm_params* best, float* best_ms)
{
    fmm_status st = check_common(c, pos, mass, n);
    if (st != FMM_OK) return st;
    if (!acc) return fail(FMM_ERR_ARG, "acc must not be NULL");
    if (reps < 1 || reps > 100) return fail(FMM_ERR_ARG, "reps must be in [1, 100]");
    if (candidates && (n_candidates < 1 || n_candidates > 4096)) return fail(FMM_ERR_ARG, "bad candidate count");
    // the built-in grid: bucket x group x list_chunk, group >= bucket
    std::vector<fmm_params> cand;
    const fmm_params base = c->params;
    if (candidates) {
        for (int i = 0; i < n_candidates; i++) {
            fmm_params p = base;
            p.bucket = candidates[i].bucket;
            p.group = candidates[i].group;
            p.list_chunk = candidates[i].list_chunk;
            st = check_params(&p);
            if (st != FMM_OK) return st;
            cand.push_back(p);
        }
    } else {
        for (int b : {8, 12, 16})
            for (int g : {32, 48, 64})
                for (int ch : {32, 64, 128}) {
                    fmm_params p = base;
                    p.bucket = b;
                    p.group = g;
                    p.list_chunk = ch;
                    cand.push_back(p);
                }
    }
    cudaStream_t s = c->stream;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_t = INFINITY;
    fmm_params best_p = base;
    for (const fmm_params& p : cand) {
        c->params = p;
        st = solve(c, pos, mass, nullptr, n, eps, theta, acc, nullptr, box_offsets, nbox);  // untimed
        float t = 0.0f;
        if (st == FMM_OK) {
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && st == FMM_OK; r++)
                st = solve(c, pos, mass, nullptr, n, eps, theta, acc, nullptr, box_offsets, nbox);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&t, e0, e1);
            t /= (float)reps;
        }
        if (st != FMM_OK) break;
        if (t < best_t) {
            best_t = t;
            best_p = p;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->params = st == FMM_OK ? best_p : base;
    if (st != FMM_OK) return st;
    if (best) *best = best_p;
    if (best_ms) *best_ms = best_t;
    return FMM_OK;
}

// ---------------------------------------------------------------- dual trees (Sec. 3.2)

static fmm_status ensure_subset(fmm_ctx* c, long long n)
{
    if (n <= c->cap_d) return FMM_OK;
    CK(alloc(&c->d_flag, n));
    CK(alloc(&c->d_at, n));
    CK(alloc(&c->d_idx, n));
    CK(alloc(&c->d_perm, n));
    CK(alloc(&c->d_act, n));
    CK(alloc(&c->d_pos, 3 * n));
    CK(alloc(&c->d_mass, n));
    c->cap_d = n;
    return FMM_OK;
}

// The particles with rung[i] <= r_max (with rungs), or outside the set flagged in flag_not (with
// that array), or all, in input order, into d_pos (SoA, drifted by vel * dt when vel is given),
// d_mass, d_idx (the caller's index) and, when sinks is given, d_act (their sink flags); *m is
// their count.
static fmm_status select_subset(fmm_ctx* c, const double* pos, const double* vel, double dt, const float* mass,
                                const unsigned char* rung, int r_max, const unsigned int* flag_not,
                                const unsigned char* sinks, long long n, long long* m)
{
    cudaStream_t s = c->stream;
    fmm_status st = ensure_subset(c, n);
    if (st != FMM_OK) return st;
    CK(fmm_launch_subset_flags(rung, r_max, flag_not, n, c->d_flag, s));
    CK(fmm_scan_exclusive(c->d_flag, c->d_at, n, c->totals + 2, c->t, s));
    CK(cudaMemcpyAsync(c->totals_h + 2, c->totals + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *m = (long long)c->totals_h[2];
    c->launches += 4;
    if (*m > 0) {
        CK(fmm_launch_subset_gather(c->d_flag, c->d_at, n, pos, vel, dt, mass, sinks, *m, c->d_pos, c->d_mass, c->d_act,
                                    c->d_idx, s));
        c->launches += 1;
    }
    return FMM_OK;
}

extern "C" fmm_status fmm_set_fixed_sources(fmm_ctx* c, const double* pos, const double* vel, const float* mass,
                                            const unsigned char* rung, long long n, int r_fixed, double dt)
{
    fmm_status st = check_common(c, pos, mass, n);
    if (st != FMM_OK) return st;
    if (!std::isfinite(dt)) return fail(FMM_ERR_ARG, "fmm_set_fixed_sources: dt must be finite");
    st = check_params(&c->params);
    if (st != FMM_OK) return st;
    FixedTree& f = c->fx;
    f.valid = false;
    c->have_solve = false;
    c->launches = 0;
    long long m = 0;
    st = select_subset(c, pos, vel, dt, mass, rung, r_fixed, nullptr, nullptr, n, &m);
    if (st != FMM_OK) return st;
    // membership of the fixed set, in the caller's order, for the dual solves
    if (n > f.cap_member) {
        f.cap_member = 0;
        CK(alloc(&f.member, n));
        f.cap_member = n;
    }
    CK(cudaMemcpyAsync(f.member, c->d_flag, sizeof(unsigned int) * n, cudaMemcpyDeviceToDevice, c->stream));
    f.n_all = n;
    f.bucket = c->params.bucket;
    f.n = m;
    f.n_cells = f.n_buckets = 0;
    if (m > 0) {
        st = build_tree(c, c->d_pos, c->d_mass, nullptr, m, c->params.bucket);
        if (st != FMM_OK) return st;
        const DevTree& t = c->t;
        cudaStream_t s = c->stream;
        const long long nc = t.n_cells, nb = t.n_buckets;
        if (nc > f.cap_cells) {
            f.cap_cells = 0;
            CK(alloc(&f.cfirst, nc));
            CK(alloc(&f.ccount, nc));
            CK(alloc(&f.cchild, 2 * nc));
            CK(alloc(&f.cparent, nc));
            CK(alloc(&f.bucket_cell, nc));
            CK(alloc(&f.com, nc));
            CK(alloc(&f.clo, 3 * nc));
            CK(alloc(&f.chi, 3 * nc));
            CK(alloc(&f.bmax, nc));
            CK(alloc(&f.rec, (long long)FMM_NREC * nc));
            f.cap_cells = nc;
        }
        if (m > f.cap_n) {
            f.cap_n = 0;
            CK(alloc(&f.posf, m));
            CK(alloc(&f.plo, m));
            CK(alloc(&f.off, m));
            CK(alloc(&f.bucket_of, m));
            CK(alloc(&f.key, m));
            f.cap_n = m;
        }
        auto cp = [&](void* dst, const void* src, size_t bytes) {
            return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
        };
        CK(cp(f.cfirst, t.cfirst, sizeof(int) * nc));
        CK(cp(f.ccount, t.ccount, sizeof(int) * nc));
        CK(cp(f.cchild, t.cchild, sizeof(int) * 2 * nc));
        CK(cp(f.cparent, t.cparent, sizeof(int) * nc));
        CK(cp(f.bucket_cell, t.bucket_cell, sizeof(int) * nb));
        CK(cp(f.com, t.com, sizeof(Com4) * nc));
        CK(cp(f.clo, t.clo, sizeof(double) * 3 * nc));
        CK(cp(f.chi, t.chi, sizeof(double) * 3 * nc));
        CK(cp(f.bmax, t.bmax, sizeof(double) * nc));
        CK(cp(f.rec, t.rec, sizeof(float) * FMM_NREC * nc));
        CK(cp(f.posf, t.posf, sizeof(float4) * m));
        CK(cp(f.plo, t.plo, sizeof(float4) * m));
        CK(cp(f.off, t.off, sizeof(float4) * m));
        CK(cp(f.bucket_of, t.bucket_of, sizeof(int) * m));
        CK(cp(f.key, t.key, sizeof(unsigned long long) * m));
        CK(cudaStreamSynchronize(s));
        f.n_cells = nc;
        f.n_buckets = nb;
    }
    f.valid = true;
    // fmm_get_stats reports this call's kernel launches and the fixed tree's size
    memset(&c->stats, 0, sizeof c->stats);
    c->stats.n = m;
    c->stats.n_cells = f.n_cells;
    c->stats.n_buckets = f.n_buckets;
    c->stats.n_launches = c->launches;
    return FMM_OK;
}

extern "C" fmm_status fmm_compute_forces_dual(fmm_ctx* c, const double* pos, const float* mass,
                                              const unsigned char* active, long long n, double eps, double theta,
                                              float* acc, float* pot)
{
    fmm_status st = check_common(c, pos, mass, n);
    if (st != FMM_OK) return st;
    if (!acc) return fail(FMM_ERR_ARG, "acc must not be NULL");
    const FixedTree& f = c->fx;
    if (!f.valid) return fail(FMM_ERR_STATE, "fmm_compute_forces_dual: no fixed sources (fmm_set_fixed_sources first)");
    fmm_params q = c->params;
    q.eps = eps;
    q.theta = theta;
    st = check_params(&q);
    if (st != FMM_OK) return st;
    if (q.criterion != 0) return fail(FMM_ERR_ARG, "fmm_compute_forces_dual: only the fixed criterion (criterion 0)");
    if (q.nrep != 0) return fail(FMM_ERR_ARG, "fmm_compute_forces_dual: isolated boxes only (nrep 0)");
    c->t.per_R = 0;
    c->t.per_ib = 31;
    if (q.bucket != f.bucket)
        return fail(FMM_ERR_ARG, "fmm_compute_forces_dual: bucket %d differs from the fixed tree's %d", q.bucket,
                    f.bucket);
    if (n != f.n_all)
        return fail(FMM_ERR_ARG, "fmm_compute_forces_dual: n = %lld, the fixed set was chosen from %lld particles", n,
                    f.n_all);
    cudaStream_t s = c->stream;
    c->have_solve = false;
    memset(&c->stats, 0, sizeof c->stats);
    c->launches = 0;
    CK(cudaEventRecord(c->ev[0], s));
    // the active tree: every particle outside the fixed set, at its current position
    long long na = 0;
    st = select_subset(c, pos, nullptr, 0.0, mass, nullptr, 0, f.member, active, n, &na);
    if (st != FMM_OK) return st;
    if (na == 0) return FMM_OK;  // no particle outside the fixed set: nothing is written
    // both trees' capacity before the active tree is built (buffers only grow); a graded active
    // tree may keep every radix node (2 n_a - 1 cells)
    DevTree& t = c->t;
    st = ensure_tree(c, na + f.n + 64, q.bucket, 1, 2 * na + f.n_cells + 16);
    if (st != FMM_OK) return st;
    if (f.n > 0) {
        CK(grow(&t.split, &t.cap_split, 2 * na));
        CK(grow(&t.nogroup, &t.cap_nogroup, t.cap_cells));
        t.grade_key = f.key;  // the active tree takes the fixed tree's geometric structure
        t.grade_n = f.n;
        t.grade_group = q.group;
    }
    st = build_tree(c, c->d_pos, c->d_mass, active ? c->d_act : nullptr, na, q.bucket);
    t.grade_key = nullptr;
    if (st != FMM_OK) return st;
    const long long ca = t.n_cells, ba = t.n_buckets;
    c->stats.n_active = (long long)c->ctr_h->n_active;
    if (ca + f.n_cells > t.cap_cells || na + f.n > t.cap_n)
        return fail(FMM_ERR_STATE, "internal: the two trees exceed the tree capacity");
    if (f.n > 0) {
        CK(fmm_append_fixed(t, f, na, ca, ba, s));
        c->launches += 3;
        t.n_cells = ca + f.n_cells;
        t.n_buckets = ba + f.n_buckets;
        c->totals_h[0] = (unsigned int)t.n_cells;
        c->totals_h[1] = (unsigned int)t.n_buckets;
        CK(cudaMemcpyAsync(c->totals, c->totals_h, 2 * sizeof(unsigned int), cudaMemcpyHostToDevice, s));
    }
    CK(fmm_launch_nodes(t, theta, s));
    c->launches += 1;
    CK(cudaEventRecord(c->ev[1], s));
    c->second_root = f.n > 0 ? (int)ca : -1;  // the fixed tree's root (its cell 0)
    // the walk's list capacities follow the sources of both trees (as a plain solve's follow all
    // its particles, sinks or not): sized for the active tree alone they overflow and re-run
    st = run_walk(c, na + f.n, eps, q.bucket, q.group, 0);
    c->second_root = -1;
    if (st != FMM_OK) return st;
    CK(fmm_launch_compose_perm(t.idx, c->d_idx, na, c->d_perm, s));
    c->launches += 1;
    return interact_and_finish(c, q, eps, acc, pot, n, na, c->d_perm);
}

extern "C" fmm_status fmm_compute_forces_batch(fmm_ctx* c, const double* pos, const float* mass,
                                               const unsigned char* active, long long n, const long long* box_offsets,
                                               int nbox, double eps, double theta, float* acc, float* pot)
{
    fmm_status st = check_common(c, pos, mass, n);
    if (st != FMM_OK) return st;
    if (!box_offsets) return fail(FMM_ERR_ARG, "box_offsets must not be NULL");
    return solve(c, pos, mass, active, n, eps, theta, acc, pot, box_offsets, nbox);
}

extern "C" fmm_status fmm_compute_forces_host(fmm_ctx* c, const double* pos, const float* mass,
                                              const unsigned char* active, long long n, double eps, double theta,
                                              float* acc, float* pot)
{
    fmm_status st = check_common(c, pos, mass, n);
    if (st != FMM_OK) return st;
    if (!acc) return fail(FMM_ERR_ARG, "acc must not be NULL");
    cudaStream_t s = c->stream;
    if (n > c->hcap) {
        c->hcap = 0;
        CK(alloc(&c->hpos, 3 * n));
        CK(alloc(&c->hmass, n));
        CK(alloc(&c->hacc, 3 * n));
        CK(alloc(&c->hpot, n));
        CK(alloc(&c->hact, n));
        c->hcap = n;
    }
    CK(cudaMemcpyAsync(c->hpos, pos, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->hmass, mass, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, s));
    if (active) CK(cudaMemcpyAsync(c->hact, active, (size_t)n, cudaMemcpyHostToDevice, s));
    if (active || c->params.criterion == 1) {
        // entries of inactive particles keep the caller's values; the learned criterion reads acc
        // on entry as its acceleration estimate
        CK(cudaMemcpyAsync(c->hacc, acc, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, s));
        if (pot) CK(cudaMemcpyAsync(c->hpot, pot, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, s));
    }
    st = solve(c, c->hpos, c->hmass, active ? c->hact : nullptr, n, eps, theta, c->hacc, pot ? c->hpot : nullptr);
    if (st != FMM_OK) return st;
    CK(cudaMemcpyAsync(acc, c->hacc, sizeof(float) * 3 * (size_t)n, cudaMemcpyDeviceToHost, s));
    if (pot) CK(cudaMemcpyAsync(pot, c->hpot, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return FMM_OK;
}

extern "C" fmm_status fmm_kick_drift(fmm_ctx* c, double* pos, double* vel, const float* acc, unsigned char* rung,
                                     unsigned char* active_next, long long n, double eps, double dt0, int max_rung,
                                     int substep, int closing)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    if (!pos || !vel || !acc || !rung || !active_next) return fail(FMM_ERR_ARG, "NULL array");
    if (n < 1 || n >= (1LL << 31)) return fail(FMM_ERR_ARG, "n must be in [1, 2^31)");
    if (!(eps > 0.0) || !(dt0 > 0.0)) return fail(FMM_ERR_ARG, "eps and dt0 must be > 0");
    if (max_rung < 0 || max_rung > 30) return fail(FMM_ERR_ARG, "max_rung must be in [0, 30]");
    if (substep < 0 || substep >= (1 << max_rung)) return fail(FMM_ERR_ARG, "substep out of range");
    CK(cudaSetDevice(c->device));
    CK(fmm_launch_kick_drift(pos, vel, acc, rung, active_next, n, eps, dt0, max_rung, substep, closing ? 1 : 0,
                             c->ctr, c->stream));
    return FMM_OK;
}

// Sec. 3.4, memory: the solve on positions stored as 32-bit fixed-point coordinates.
extern "C" fmm_status fmm_compute_forces_i32(fmm_ctx* c, const unsigned int* ipos, const float* mass,
                                             const unsigned char* active, long long n, double eps, double theta,
                                             float* acc, float* pot)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    if (!ipos || !mass) return fail(FMM_ERR_ARG, "ipos and mass must not be NULL");
    if (n < 1 || n >= (1LL << 31)) return fail(FMM_ERR_ARG, "n must be in [1, 2^31), got %lld", n);
    CK(cudaSetDevice(c->device));
    c->cur_ipos = ipos;
    const fmm_status st = solve(c, nullptr, mass, active, n, eps, theta, acc, pot);
    c->cur_ipos = nullptr;
    return st;
}

extern "C" fmm_status fmm_kick_drift_i32(fmm_ctx* c, unsigned int* ipos, float* vel, const float* acc,
                                         unsigned char* rung, unsigned char* active_next, long long n, double eps,
                                         double dt0, int max_rung, int substep, int closing)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    if (!ipos || !vel || !acc || !rung || !active_next) return fail(FMM_ERR_ARG, "NULL array");
    if (n < 1 || n >= (1LL << 31)) return fail(FMM_ERR_ARG, "n must be in [1, 2^31)");
    if (!(eps > 0.0) || !(dt0 > 0.0)) return fail(FMM_ERR_ARG, "eps and dt0 must be > 0");
    if (max_rung < 0 || max_rung > 30) return fail(FMM_ERR_ARG, "max_rung must be in [0, 30]");
    if (substep < 0 || substep >= (1 << max_rung)) return fail(FMM_ERR_ARG, "substep out of range");
    CK(cudaSetDevice(c->device));
    CK(fmm_launch_kick_drift_i32(ipos, vel, acc, rung, active_next, n, eps, dt0, max_rung, substep, closing ? 1 : 0,
                                 c->params.nrep > 0 ? 1 : 0, c->ctr, c->stream));
    return FMM_OK;
}

extern "C" fmm_status fmm_assign_rungs(fmm_ctx* c, const float* acc, unsigned char* rung, long long n, double eps,
                                       double dt0, int max_rung)
{
    if (!c || !acc || !rung) return fail(FMM_ERR_ARG, "NULL argument");
    if (n < 1 || n >= (1LL << 31)) return fail(FMM_ERR_ARG, "n must be in [1, 2^31)");
    if (!(eps > 0.0) || !(dt0 > 0.0)) return fail(FMM_ERR_ARG, "eps and dt0 must be > 0");
    if (max_rung < 0 || max_rung > 30) return fail(FMM_ERR_ARG, "max_rung must be in [0, 30]");
    CK(cudaSetDevice(c->device));
    CK(fmm_launch_assign_rungs(acc, rung, n, eps, dt0, max_rung, c->stream));
    return FMM_OK;
}

extern "C" fmm_status fmm_get_stats(const fmm_ctx* c, fmm_stats* out)
{
    if (!c || !out) return fail(FMM_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    *out = c->stats;
    return FMM_OK;
}

// ---------------------------------------------------------------- introspection

template <typename T>
static cudaError_t d2h(T* dst, const T* src, long long n, cudaStream_t s)
{
    if (!dst || n <= 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost, s);
}

extern "C" fmm_status fmm_tree_info(const fmm_ctx* c, long long* n_cells, long long* n_groups, long long* n_pp,
                                    long long* n_pc, long long* n_local)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    if (!c->have_tree) return fail(FMM_ERR_STATE, "no tree built yet");
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    if (n_cells) *n_cells = c->t.n_cells;
    if (n_groups) *n_groups = c->have_solve ? c->w.n_groups : 0;
    if (n_pp) *n_pp = c->have_solve ? c->w.pp_len : 0;
    if (n_pc) *n_pc = c->have_solve ? c->w.pc_len : 0;
    if (n_local) *n_local = c->have_solve ? c->w.cc_len + c->w.cp_len : 0;
    return FMM_OK;
}

extern "C" fmm_status fmm_export_order(const fmm_ctx* c, unsigned int* perm, unsigned long long* keys)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    if (!c->have_tree) return fail(FMM_ERR_STATE, "no tree built yet");
    CK(cudaSetDevice(c->device));
    CK(d2h(perm, c->t.idx, c->t.n, c->stream));
    CK(d2h(keys, c->t.key, c->t.n, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FMM_OK;
}

extern "C" fmm_status fmm_export_cells(const fmm_ctx* c, int* first, int* count, int* parent, int* child, int* nact,
                                       double* mass, double* com, double* lo, double* hi, double* bmax,
                                       float* moments)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    if (!c->have_tree) return fail(FMM_ERR_STATE, "no tree built yet");
    CK(cudaSetDevice(c->device));
    const DevTree& t = c->t;
    long long nc = t.n_cells;
    cudaStream_t s = c->stream;
    CK(d2h(first, t.cfirst, nc, s));
    CK(d2h(count, t.ccount, nc, s));
    CK(d2h(parent, t.cparent, nc, s));
    CK(d2h(child, t.cchild, 2 * nc, s));
    CK(d2h(nact, t.cnact, nc, s));
    CK(d2h(lo, t.clo, 3 * nc, s));
    CK(d2h(hi, t.chi, 3 * nc, s));
    CK(d2h(bmax, t.bmax, nc, s));
    CK(d2h(moments, t.rec, (long long)FMM_NREC * nc, s));
    std::vector<Com4> cm;
    if (mass || com) {
        cm.resize((size_t)nc);
        CK(d2h(cm.data(), t.com, nc, s));
    }
    CK(cudaStreamSynchronize(s));
    for (long long i = 0; i < (long long)cm.size(); i++) {
        if (mass) mass[i] = cm[i].w;
        if (com) {
            com[3 * i] = cm[i].x;
            com[3 * i + 1] = cm[i].y;
            com[3 * i + 2] = cm[i].z;
        }
    }
    return FMM_OK;
}

// The kind's list entries of the last solve (0 PP, 1 PC, 2 CC, 3 CP) as (sink cell, source first,
// source count, source copy n) in list order; n = 0 for an isolated box.
static fmm_status collect_lists(const fmm_ctx* c, int kind, std::vector<long long>& out_sink,
                                std::vector<long long>& out_first, std::vector<long long>& out_count,
                                std::vector<int>& out_shift)
{
    if (kind < 0 || kind > 3) return fail(FMM_ERR_ARG, "kind must be 0..3");
    if (!c->have_solve) return fail(FMM_ERR_STATE, "no solve yet");
    CK(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    const DevTree& t = c->t;
    const DevWalk& w = c->w;
    const int ib = t.per_ib, R = t.per_R;
    long long nc = t.n_cells;
    std::vector<int> cf((size_t)nc), cn((size_t)nc);
    CK(d2h(cf.data(), t.cfirst, nc, s));
    CK(d2h(cn.data(), t.ccount, nc, s));
    auto push = [&](int sk, unsigned int e) {
        const unsigned int j = entry_index(e, ib);
        int nx = 0, ny = 0, nz = 0;
        copy_shift(entry_copy(e, ib), R, nx, ny, nz);
        out_sink.push_back(sk);
        if (e & FMM_PARTICLE_BIT) {
            out_first.push_back((int)j);
            out_count.push_back(1);
        } else {
            out_first.push_back(cf[j]);
            out_count.push_back(cn[j]);
        }
        out_shift.push_back(nx);
        out_shift.push_back(ny);
        out_shift.push_back(nz);
    };
    if (kind <= 1) {
        std::vector<Group> g((size_t)w.n_groups);
        CK(d2h(g.data(), w.groups, w.n_groups, s));
        long long len = kind == 0 ? w.pp_len : w.pc_len;
        std::vector<unsigned int> L((size_t)len);
        CK(d2h(L.data(), kind == 0 ? w.pp : w.pc, len, s));
        CK(cudaStreamSynchronize(s));
        for (const Group& G : g) {
            unsigned long long o = kind == 0 ? G.pp_off : G.pc_off;
            int l = kind == 0 ? G.pp_len : G.pc_len;
            for (int i = 0; i < l; i++) push(G.cell, L[o + i]);
        }
    } else {
        // kind 2 (CC): the multipole-source list; kind 3 (CP): the point-source list
        const long long len = kind == 2 ? w.cc_len : w.cp_len;
        std::vector<unsigned int> L((size_t)len);
        std::vector<int> sk((size_t)len);
        CK(d2h(L.data(), kind == 2 ? w.cc : w.cp, len, s));
        CK(d2h(sk.data(), kind == 2 ? w.cc_sink : w.cp_sink, len, s));
        CK(cudaStreamSynchronize(s));
        for (long long i = 0; i < len; i++) push(sk[i], L[i]);
    }
    return FMM_OK;
}

extern "C" fmm_status fmm_export_lists(const fmm_ctx* c, int kind, long long* n_entries, int* sink, int* src_first,
                                       int* src_count, long long capacity)
{
    if (!c || !n_entries) return fail(FMM_ERR_ARG, "NULL argument");
    std::vector<long long> out_sink, out_first, out_count;
    std::vector<int> out_shift;
    fmm_status st = collect_lists(c, kind, out_sink, out_first, out_count, out_shift);
    if (st != FMM_OK) return st;
    *n_entries = (long long)out_sink.size();
    if (capacity < *n_entries) return FMM_OK;  // size query
    for (long long i = 0; i < *n_entries; i++) {
        if (sink) sink[i] = (int)out_sink[i];
        if (src_first) src_first[i] = (int)out_first[i];
        if (src_count) src_count[i] = (int)out_count[i];
    }
    return FMM_OK;
}

extern "C" fmm_status fmm_export_list_shifts(const fmm_ctx* c, int kind, long long* n_entries, int* shift,
                                             long long capacity)
{
    if (!c || !n_entries) return fail(FMM_ERR_ARG, "NULL argument");
    std::vector<long long> out_sink, out_first, out_count;
    std::vector<int> out_shift;
    fmm_status st = collect_lists(c, kind, out_sink, out_first, out_count, out_shift);
    if (st != FMM_OK) return st;
    *n_entries = (long long)out_sink.size();
    if (capacity < *n_entries || !shift) return FMM_OK;  // size query
    memcpy(shift, out_shift.data(), sizeof(int) * out_shift.size());
    return FMM_OK;
}

extern "C" fmm_status fmm_export_locals(const fmm_ctx* c, int* group_cell, float* L, long long capacity)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    if (!c->have_solve) return fail(FMM_ERR_STATE, "no solve yet");
    if (capacity < c->w.n_groups) return fail(FMM_ERR_ARG, "capacity %lld < %lld groups", capacity, c->w.n_groups);
    CK(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    std::vector<Group> g((size_t)c->w.n_groups);
    CK(d2h(g.data(), c->w.groups, c->w.n_groups, s));
    CK(d2h(L, c->w.Lg, c->w.n_groups * FMM_NL, s));
    CK(cudaStreamSynchronize(s));
    for (size_t i = 0; i < g.size(); i++)
        if (group_cell) group_cell[i] = g[i].cell;
    return FMM_OK;
}

extern "C" fmm_status fmm_export_walk_levels(const fmm_ctx* c, long long* counts, int capacity, int* n_levels)
{
    if (!c || !n_levels) return fail(FMM_ERR_ARG, "NULL argument");
    if (!c->have_solve) return fail(FMM_ERR_STATE, "no solve yet");
    *n_levels = (int)c->w.n_levels;
    for (int l = 0; l < capacity && l < (int)c->w.n_levels; l++) {
        counts[3 * l] = (long long)c->ctr_h->lv_front[l];
        counts[3 * l + 1] = (long long)c->ctr_h->lv_entries[l];
        counts[3 * l + 2] = (long long)c->ctr_h->lv_max_entries[l];
    }
    return FMM_OK;
}

extern "C" fmm_status fmm_multi_index(int* local_idx, int* moment_idx)
{
    if (local_idx) memcpy(local_idx, fmm_multi_index_table, sizeof(fmm_multi_index_table));
    if (moment_idx) memcpy(moment_idx, fmm_moment_index_table, sizeof(fmm_moment_index_table));
    return FMM_OK;
}

// ---------------------------------------------------------------- learned criterion

static_assert(FMM_MLP_NP == MLP_NP && FMM_MLP_NW == MLP_NW, "network sizes in fmm.h and mlp.cuh differ");

static fmm_status mlp_alloc(fmm_ctx* c)
{
    if (c->mlp_p) return FMM_OK;
    CK(alloc(&c->mlp_p, MLP_NP));
    CK(alloc(&c->mlp_g, MLP_NW));
    CK(alloc(&c->mlp_m, MLP_NW));
    CK(alloc(&c->mlp_v, MLP_NW));
    CK(alloc(&c->mlp_loss, 1));
    CK(alloc(&c->mlp_packed, MLPP_SIZE));
    return FMM_OK;
}

extern "C" fmm_status fmm_mlp_load(fmm_ctx* c, const float* params, long long n)
{
    if (!c || !params) return fail(FMM_ERR_ARG, "NULL argument");
    if (n != MLP_NP) return fail(FMM_ERR_ARG, "expected %d parameters, got %lld", MLP_NP, n);
    for (long long i = 0; i < n; i++)
        if (!isfinite(params[i])) return fail(FMM_ERR_NUMERIC, "parameter %lld is not finite", i);
    CK(cudaSetDevice(c->device));
    fmm_status st = mlp_alloc(c);
    if (st != FMM_OK) return st;
    CK(cudaMemcpyAsync(c->mlp_p, params, sizeof(float) * MLP_NP, cudaMemcpyHostToDevice, c->stream));
    CK(fmm_mlp_pack(c->mlp_p, c->mlp_packed, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->mlp_ready = true;
    return FMM_OK;
}

extern "C" fmm_status fmm_mlp_get(const fmm_ctx* c, float* params, long long n)
{
    if (!c || !params) return fail(FMM_ERR_ARG, "NULL argument");
    if (n < MLP_NP) return fail(FMM_ERR_ARG, "need room for %d parameters", MLP_NP);
    if (!c->mlp_ready) return fail(FMM_ERR_STATE, "no network parameters");
    CK(cudaSetDevice(c->device));
    CK(cudaMemcpyAsync(params, c->mlp_p, sizeof(float) * MLP_NP, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FMM_OK;
}

extern "C" fmm_status fmm_mlp_predict(fmm_ctx* c, const float* feats, long long n, float* out)
{
    if (!c || !feats || !out) return fail(FMM_ERR_ARG, "NULL argument");
    if (n < 0) return fail(FMM_ERR_ARG, "n must be >= 0");
    if (!c->mlp_ready) return fail(FMM_ERR_STATE, "no network parameters");
    if (n == 0) return FMM_OK;
    CK(cudaSetDevice(c->device));
    CK(fmm_mlp_predict(c->mlp_packed, feats, n, out, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FMM_OK;
}

extern "C" fmm_status fmm_mlp_gradient(fmm_ctx* c, const float* feats, const float* labels, long long n, float* grad,
                                       float* loss)
{
    if (!c || !feats || !labels || !grad) return fail(FMM_ERR_ARG, "NULL argument");
    if (n < 1) return fail(FMM_ERR_ARG, "n must be >= 1");
    if (!c->mlp_ready) return fail(FMM_ERR_STATE, "no network parameters");
    CK(cudaSetDevice(c->device));
    CK(cudaMemsetAsync(c->mlp_g, 0, sizeof(float) * MLP_NW, c->stream));
    CK(cudaMemsetAsync(c->mlp_loss, 0, sizeof(float), c->stream));
    CK(fmm_mlp_grad(c->mlp_p, feats, labels, nullptr, n, 1.0f / (float)n, 1.0f / (float)n, c->mlp_g, c->mlp_loss,
                    c->stream));
    CK(cudaMemcpyAsync(grad, c->mlp_g, sizeof(float) * MLP_NW, cudaMemcpyDeviceToHost, c->stream));
    if (loss) CK(cudaMemcpyAsync(loss, c->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return FMM_OK;
}

namespace {
// splitmix64: the seed of the weight initialisation and of the minibatch shuffles
unsigned long long splitmix(unsigned long long& s)
{
    unsigned long long z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
double uniform01(unsigned long long& s) { return (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }
}  // namespace

extern "C" fmm_status fmm_mlp_train(fmm_ctx* c, const float* feats, const float* labels, long long n, int epochs,
                                    int batch, float lr, unsigned int seed, float* final_loss)
{
    if (!c || !feats || !labels) return fail(FMM_ERR_ARG, "NULL argument");
    if (n < 2 || epochs < 1 || batch < 1 || !(lr > 0.0f)) return fail(FMM_ERR_ARG, "invalid training arguments");
    if (n >= (1LL << 32)) return fail(FMM_ERR_ARG, "too many rows");
    CK(cudaSetDevice(c->device));
    cudaStream_t s = c->stream;
    fmm_status st = mlp_alloc(c);
    if (st != FMM_OK) return st;
    // normalisation from the data, weights from the seed
    std::vector<float> hf((size_t)n * MLP_F), hl((size_t)n);
    CK(cudaMemcpyAsync(hf.data(), feats, sizeof(float) * hf.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hl.data(), labels, sizeof(float) * hl.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<float> p(MLP_NP, 0.0f);
    double lmean = 0.0;
    for (long long i = 0; i < n; i++) lmean += hl[i];
    lmean /= (double)n;
    for (int k = 0; k < MLP_F; k++) {
        double m = 0.0, v = 0.0;
        for (long long i = 0; i < n; i++) m += hf[i * MLP_F + k];
        m /= (double)n;
        for (long long i = 0; i < n; i++) v += (hf[i * MLP_F + k] - m) * (hf[i * MLP_F + k] - m);
        v /= (double)n;
        p[MLP_MEAN + k] = (float)m;
        p[MLP_ISTD + k] = (float)(v > 1e-20 ? 1.0 / sqrt(v) : 1.0);
    }
    unsigned long long rs = 0x5eedull ^ ((unsigned long long)seed << 17);
    auto init = [&](int off, int rows, int cols) {
        const double a = sqrt(6.0 / cols);
        for (int i = 0; i < rows * cols; i++) p[off + i] = (float)(a * (2.0 * uniform01(rs) - 1.0));
    };
    init(MLP_W1, MLP_H, MLP_F);
    init(MLP_W2, MLP_H, MLP_H);
    init(MLP_W3, MLP_H, MLP_H);
    init(MLP_W4, 1, MLP_H);
    for (int i = 0; i < MLP_H; i++) p[MLP_W4 + i] *= 0.1f;
    p[MLP_B4] = (float)lmean;
    CK(cudaMemcpyAsync(c->mlp_p, p.data(), sizeof(float) * MLP_NP, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(c->mlp_m, 0, sizeof(float) * MLP_NW, s));
    CK(cudaMemsetAsync(c->mlp_v, 0, sizeof(float) * MLP_NW, s));
    if (n > c->mlp_idx_cap) {
        c->mlp_idx_cap = 0;
        CK(alloc(&c->mlp_idx, n));
        c->mlp_idx_cap = n;
    }
    std::vector<unsigned int> perm((size_t)n);
    for (long long i = 0; i < n; i++) perm[i] = (unsigned int)i;
    int step = 0;
    float last = 0.0f;
    for (int ep = 0; ep < epochs; ep++) {
        for (long long i = n - 1; i > 0; i--) {  // Fisher-Yates
            long long j = (long long)(splitmix(rs) % (unsigned long long)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        CK(cudaMemcpyAsync(c->mlp_idx, perm.data(), sizeof(unsigned int) * (size_t)n, cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(c->mlp_loss, 0, sizeof(float), s));
        for (long long b = 0; b < n; b += batch) {
            const long long nr = std::min<long long>(batch, n - b);
            CK(cudaMemsetAsync(c->mlp_g, 0, sizeof(float) * MLP_NW, s));
            // minibatch-mean gradient; the loss is accumulated as the epoch mean
            CK(fmm_mlp_grad(c->mlp_p, feats, labels, c->mlp_idx + b, nr, 1.0f / (float)nr, 1.0f / (float)n, c->mlp_g,
                            c->mlp_loss, s));
            CK(fmm_mlp_adam(c->mlp_p, c->mlp_g, c->mlp_m, c->mlp_v, lr, ++step, s));
        }
        CK(cudaMemcpyAsync(&last, c->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!isfinite(last)) return fail(FMM_ERR_NUMERIC, "training diverged at epoch %d", ep);
    }
    CK(fmm_mlp_pack(c->mlp_p, c->mlp_packed, s));
    // surrogate bound: y_lin = f3 + alpha log10(theta_eff) + beta + sum_i gamma_i f_i fitted to the
    // labels by least squares (normal equations in FP64, columns scaled to unit RMS), then the
    // 0.05% and 99.95% quantiles of the network's residual y_net - y_lin
    if (n > c->mlp_pred_cap) {
        c->mlp_pred_cap = 0;
        CK(alloc(&c->mlp_pred, n));
        c->mlp_pred_cap = n;
    }
    CK(fmm_mlp_predict(c->mlp_packed, feats, n, c->mlp_pred, s));
    std::vector<float> pred((size_t)n);
    CK(cudaMemcpyAsync(pred.data(), c->mlp_pred, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int NC = 2 + MLP_F;  // columns: log10(theta_eff), 1, f_0..f_7
    auto columns = [&](long long i, double* x) -> bool {
        const double te = 1.5 * hf[i * MLP_F + 1] + hf[i * MLP_F + 0];
        if (!(te > 0)) return false;
        x[0] = log10(te);
        x[1] = 1.0;
        for (int k = 0; k < MLP_F; k++) x[2 + k] = hf[i * MLP_F + k];
        for (int k = 0; k < NC; k++)
            if (!isfinite(x[k])) return false;
        return isfinite((double)hl[i]) && isfinite((double)pred[i]);
    };
    std::vector<double> scale(NC, 0.0);
    double cnt = 0;
    {
        double x[2 + MLP_F];
        for (long long i = 0; i < n; i++) {
            if (!columns(i, x)) continue;
            for (int k = 0; k < NC; k++) scale[k] += x[k] * x[k];
            cnt += 1;
        }
    }
    float sur[MLP_NSUR] = {};  // off unless the fit is well posed
    if (cnt > 100) {
        for (int k = 0; k < NC; k++) scale[k] = scale[k] > 0 ? 1.0 / sqrt(scale[k] / cnt) : 1.0;
        std::vector<double> G((size_t)NC * NC, 0.0), rhs(NC, 0.0);
        double x[2 + MLP_F];
        for (long long i = 0; i < n; i++) {
            if (!columns(i, x)) continue;
            const double z = hl[i] - hf[i * MLP_F + 3];
            for (int a = 0; a < NC; a++) {
                const double xa = x[a] * scale[a];
                rhs[a] += xa * z;
                for (int b = 0; b <= a; b++) G[a * NC + b] += xa * x[b] * scale[b];
            }
        }
        for (int a = 0; a < NC; a++) {
            G[a * NC + a] += 1e-9 * cnt;  // ridge: keeps collinear columns solvable
            for (int b = a + 1; b < NC; b++) G[a * NC + b] = G[b * NC + a];
        }
        // Gauss-Jordan elimination with partial pivoting
        std::vector<double> coef(rhs);
        bool ok = true;
        for (int col = 0; col < NC && ok; col++) {
            int piv = col;
            for (int r = col + 1; r < NC; r++)
                if (fabs(G[r * NC + col]) > fabs(G[piv * NC + col])) piv = r;
            if (!(fabs(G[piv * NC + col]) > 0)) {
                ok = false;
                break;
            }
            if (piv != col) {
                for (int k = 0; k < NC; k++) std::swap(G[col * NC + k], G[piv * NC + k]);
                std::swap(coef[col], coef[piv]);
            }
            for (int r = 0; r < NC; r++) {
                if (r == col) continue;
                const double m = G[r * NC + col] / G[col * NC + col];
                for (int k = col; k < NC; k++) G[r * NC + k] -= m * G[col * NC + k];
                coef[r] -= m * coef[col];
            }
        }
        if (ok) {
            for (int a = 0; a < NC; a++) coef[a] = coef[a] / G[a * NC + a] * scale[a];
            std::vector<float> r;
            r.reserve((size_t)cnt);
            for (long long i = 0; i < n; i++) {
                if (!columns(i, x)) continue;
                double y = hf[i * MLP_F + 3];
                for (int a = 0; a < NC; a++) y += coef[a] * x[a];
                r.push_back((float)(pred[i] - y));
            }
            const size_t klo = r.size() / 2000, khi = r.size() - 1 - r.size() / 2000;
            std::nth_element(r.begin(), r.begin() + klo, r.end());
            const float rlo = r[klo];
            std::nth_element(r.begin(), r.begin() + khi, r.end());
            const float rhi = r[khi];
            sur[0] = (float)coef[0];
            sur[1] = (float)coef[1];
            sur[2] = rlo;
            sur[3] = rhi;
            for (int k = 0; k < MLP_F; k++) sur[4 + k] = (float)coef[2 + k];
        }
    }
    CK(cudaMemcpyAsync(c->mlp_p + MLP_SUR, sur, sizeof sur, cudaMemcpyHostToDevice, s));
    CK(fmm_mlp_pack(c->mlp_p, c->mlp_packed, s));
    CK(cudaStreamSynchronize(s));
    c->mlp_ready = true;
    if (final_loss) *final_loss = last;
    return FMM_OK;
}

extern "C" fmm_status fmm_mlp_audit(fmm_ctx* c, const double* pos, const float* mass, long long n, double eps,
                                    double theta, double band_lo, double band_hi, const float* acc_ref,
                                    long long max_pairs, float* feats, float* labels, long long* n_pairs)
{
    fmm_status st = check_common(c, pos, mass, n);
    if (st != FMM_OK) return st;
    if (!acc_ref || !feats || !labels || !n_pairs || max_pairs < 1) return fail(FMM_ERR_ARG, "invalid audit buffers");
    fmm_params q = c->params;
    q.eps = eps;
    q.theta = theta;
    q.band_lo = band_lo;
    q.band_hi = band_hi;
    q.criterion = 0;
    st = check_params(&q);
    if (st != FMM_OK) return st;
    if (q.nrep != 0) return fail(FMM_ERR_ARG, "fmm_mlp_audit: isolated boxes only (nrep 0)");
    c->t.per_R = 0;
    c->t.per_ib = 31;
    const fmm_params saved = c->params;
    c->params = q;
    cudaStream_t s = c->stream;
    if (max_pairs > c->audit_cap) {
        c->audit_cap = 0;
        CK(alloc(&c->audit_pairs, max_pairs));
        c->audit_cap = max_pairs;
    }
    c->launches = 0;
    st = build_tree(c, pos, mass, nullptr, n, q.bucket);
    if (st == FMM_OK) {
        cudaError_t e = fmm_launch_nodes(c->t, theta, s);
        if (e != cudaSuccess) st = fail(FMM_ERR_CUDA, "nodes: %s", cudaGetErrorString(e));
    }
    if (st == FMM_OK) {
        cudaError_t e = fmm_launch_cell_amin(c->t, acc_ref, n, s);
        if (e != cudaSuccess) st = fail(FMM_ERR_CUDA, "cell amin: %s", cudaGetErrorString(e));
    }
    if (st == FMM_OK) st = run_walk(c, n, eps, q.bucket, q.group, 2);
    c->params = saved;
    if (st != FMM_OK) return st;
    const long long np = std::min<long long>((long long)c->ctr_h->n_audit, max_pairs);
    if (np > 0) CK(fmm_launch_audit_labels(c->t, c->audit_pairs, np, acc_ref, n, (float)eps, feats, labels, s));
    CK(cudaStreamSynchronize(s));
    *n_pairs = np;
    c->have_solve = false;
    return FMM_OK;
}

extern "C" fmm_status fmm_mlp_audit_pairs(const fmm_ctx* c, int* sink_first, int* sink_count, int* src_first,
                                          int* src_count, long long n)
{
    if (!c) return fail(FMM_ERR_ARG, "ctx is NULL");
    if (n < 0 || n > c->audit_cap || n > (long long)c->ctr_h->n_audit) return fail(FMM_ERR_ARG, "bad pair count");
    CK(cudaSetDevice(c->device));
    std::vector<int2> pr((size_t)n);
    std::vector<int> cf((size_t)c->t.n_cells), cn((size_t)c->t.n_cells);
    CK(d2h(pr.data(), c->audit_pairs, n, c->stream));
    CK(d2h(cf.data(), c->t.cfirst, c->t.n_cells, c->stream));
    CK(d2h(cn.data(), c->t.ccount, c->t.n_cells, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (long long i = 0; i < n; i++) {
        if (sink_first) sink_first[i] = cf[pr[i].x];
        if (sink_count) sink_count[i] = cn[pr[i].x];
        if (src_first) src_first[i] = cf[pr[i].y];
        if (src_count) src_count[i] = cn[pr[i].y];
    }
    return FMM_OK;
}
