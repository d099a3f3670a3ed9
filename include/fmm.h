/*
 * fmm.h -- C ABI of the GB300 (sm_103a) FMM gravity force solve.
 *
 * The library computes softened gravitational accelerations and potentials of N
 * particles in the isolated unit box with the fast multipole method of PKDGRAV3
 * (Potter, Stadel & Teyssier, arXiv:1609.08621):
 *   - a Morton-ordered binary tree whose leaves ("buckets") hold at most b
 *     particles (Sec. 3.1, "Leaf cells of our tree contain up to b particles");
 *   - order-4 multipoles about each cell's centre of mass and the opening
 *     radius R_O = b_max / theta (Sec. 3.1);
 *   - a checklist walk that sorts each source into cell-cell / cell-particle
 *     (local expansion), particle-cell, particle-particle, "stay on the
 *     checklist" or "open" (Sec. 3.1), stopping at groups of at most g
 *     particles;
 *   - PP, PC and local-expansion (order 5) evaluation for each group (Sec. 3.1,
 *     Sec. 3.3);
 *   - kick-drift-kick on individual time-step rungs (Sec. 3.2), with dual trees
 *     for the substeps: a tree of the slow rungs kept over their interval and
 *     a tree of the other particles per substep (Sec. 3.2);
 *   - independent boxes solved together in one pass, CUDA-graph replay of the
 *     solve and an autotuner of bucket, group and work-item size;
 *   - an opening criterion learned by a small network trained on the GPU (not
 *     in the paper; it replaces the fixed-theta test of Sec. 3.1 inside a band);
 *   - the periodic unit box: the root's 26 or 124 copies on the checklist and the
 *     5th-order Ewald multipole correction for the copies beyond (Sec. 3.1, Sec. 3.3).
 *
 * Physics conventions (all entry points): G = 1, Plummer softening,
 *     a_i   =  sum_{j != i} m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2)
 *     phi_i = -sum_{j != i} m_j / (|x_j - x_i|^2 + eps^2)^(1/2)
 * which the method approximates in the isolated unit box.  With fmm_params.nrep > 0
 * the box is periodic (Sec. 3.1): the sum runs over every periodic copy of the sources,
 * softened within the replica shell |n|_inf <= nrep and Newtonian (Ewald, with a uniform
 * background of the mean density) beyond it.  Positions must lie in [0,1)^3, masses
 * must be finite and > 0, eps > 0, 0 < theta <= 1.
 *
 * Memory and ownership:
 *   - "device" arguments are CUDA device pointers on the context's device;
 *     "host" arguments are host pointers (pinned memory is faster, pageable
 *     works).  The caller owns every pointer it passes; the library never
 *     frees or retains them beyond the call.
 *   - Positions are structure-of-arrays doubles: x[0..N), then y, then z
 *     (3N values).  Accelerations likewise (3N floats).  Outputs are in the
 *     caller's particle order.
 *   - Everything behind an fmm_ctx (tree, lists, scratch, events) is owned by
 *     the library and released by fmm_destroy.
 *
 * Streams and synchronisation: all device work of a context runs on the CUDA
 * stream given to fmm_create (0 = the legacy default stream).  fmm_kick_drift and
 * fmm_assign_rungs are asynchronous with respect to the host.  fmm_build_tree and
 * fmm_compute_forces read sizes back to the host (cell counts, per-level frontier
 * sizes of the walk) and return after their work has completed on the stream.
 *
 * Errors: every entry point returns an fmm_status.  A message for the last
 * failure on the calling thread is returned by fmm_last_error().  Device-side
 * failures (a bounded wait that gave up, capacity exhausted, invalid input
 * detected by a kernel) are reported through a device status word that the
 * library reads at its next synchronisation point; kernels never trap.
 * After FMM_ERR_CUDA the context should be destroyed.
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_ctx fmm_ctx;

typedef enum {
    FMM_OK = 0,
    FMM_ERR_ARG = -1,     /* invalid argument (pointer, size, range, parameter) */
    FMM_ERR_OOM = -2,     /* device or host allocation failed */
    FMM_ERR_CUDA = -3,    /* a CUDA runtime call failed */
    FMM_ERR_TIMEOUT = -4, /* a bounded device-side wait gave up */
    FMM_ERR_STATE = -5,   /* call order violated (e.g. export before any solve) */
    FMM_ERR_NUMERIC = -6  /* non-finite input or output detected */
} fmm_status;

/* Solver parameters.  Obtain defaults from fmm_default_params. */
typedef struct fmm_params {
    double theta;          /* opening angle, 0 < theta <= 1 (Sec. 3.1; default 0.55, Sec. 4.2) */
    double eps;            /* Plummer softening length, > 0 (Sec. 3.1: 1/50 of the mean separation) */
    int bucket;            /* b: maximum particles per leaf, 1..16 (Sec. 3.1: ~16; default 16) */
    int group;             /* g: sink group size, bucket..64 (Sec. 3.1: 64 = 4 b; default 64) */
    int criterion;         /* 0: fixed theta (Sec. 3.1); 1: learned (MLP, requires fmm_mlp_load) */
    int accumulate;        /* 0: a particle's partial sums (one per list chunk of <= 64 entries, and the
                              local expansion) are added in FP32; 1: they are added in FP64 */
    int terms;             /* bit mask of evaluated terms: 1 PP, 2 PC, 4 local expansion of the walk,
                              8 Ewald correction (periodic box only); default 15 */
    int list_chunk;        /* list entries per PP / PC work item: 0 (default, 64) or a multiple of
                              32 in [32, 1024] */
    long long spin_limit;  /* iteration cap of any device-side wait (default 1<<26) */
    /* learned criterion (criterion = 1), not in the paper: for a source cell with
     * theta_eff = (1.5 b_max(sink) + b_max(source)) / d, the pair is accepted as a cell-cell
     * interaction when theta_eff < band_lo, rejected when theta_eff >= band_hi, and in between
     * accepted when the network's predicted log10 relative force error is < mlp_tau.  A guard
     * (d > 1.1 (b_max(sink) + b_max(source)), bounding boxes >= 2 eps apart) always applies.
     * Defaults: band 0.35 .. 1.0, mlp_tau = -3.5.  Inside the band a linear surrogate fitted
     * to the network at training time decides the pairs whose prediction lies clear of mlp_tau:
     * mlp_margin in [0, 1] scales the surrogate's residual range on the training rows (1: the
     * network decides every pair the surrogate could have got wrong there; 0: the surrogate
     * decides alone); default 0.1. */
    double mlp_tau;
    double band_lo;
    double band_hi;
    /* Periodic unit box (Sec. 3.1, periodic boundaries): 0 (default) for the isolated box; 1 or 2
     * for the periodic box, whose walk starts from the root and its copies shifted by the integer
     * vectors n with |n|_inf <= nrep (26 or 124 copies, softened like the box itself), and whose
     * copies beyond that shell enter as the 5th-order Ewald multipole correction (Sec. 3.1,
     * Sec. 3.3): the periodic Newtonian sum with a uniform background of the mean density, from the
     * root's moments, evaluated in FP64 once per solve as order-5 local expansions about the
     * centres of 4^3 sub-cubes.  Periodic solves take one box (not fmm_compute_forces_batch), the
     * fixed criterion only, no dual trees, and n <= 2^26 (nrep 1) or 2^24 (nrep 2): list entries
     * carry the copy in their upper bits. */
    int nrep;
    double mlp_margin;
} fmm_params;

/* Per-solve statistics of the last fmm_compute_forces on a context. */
typedef struct fmm_stats {
    long long n;            /* particles */
    long long n_active;     /* active particles (forces computed) */
    long long n_cells;      /* tree cells */
    long long n_buckets;    /* leaf buckets */
    long long n_groups;     /* sink groups walked to the end */
    long long n_levels;     /* walk levels (tree depth reached by the walk + 1) */
    long long n_pp_pairs;   /* particle-particle interactions (sink x source particle) */
    long long n_pc_pairs;   /* particle-cell interactions (sink x source cell) */
    long long n_cc;         /* cell-cell (multipole -> local) interactions */
    long long n_cp;         /* cell-particle (particle -> local) interactions */
    long long n_pp_entries; /* PP list entries (buckets or particles) */
    long long n_pc_entries; /* PC list entries (cells) */
    double ms_tree;         /* keys, sort, tree, upward pass (CUDA events) */
    double ms_walk;         /* checklist walk + local expansions */
    double ms_pp;           /* PP kernel */
    double ms_pc;           /* PC kernel */
    double ms_l2p;          /* local expansion at particles + output */
    double ms_total;        /* whole solve */
    double paper_flops;     /* paper-equivalent flops: 53 PP + 215 PC + 479 CC + 213 CP (Sec. 4.6) */
    double kernel_flops_pp; /* FP32 flops performed by the PP kernel (19 per pair) */
    double kernel_flops_pc; /* FP32 flops performed by the PC kernel (per pair count, see fmm_flops_per_pc) */
    int retries;            /* walk restarts after a capacity grow */
    int n_launches;         /* kernels launched by the solve */
    long long n_learned;    /* decisions taken by the learned criterion's network */
} fmm_stats;

/* Fill *p with the defaults: theta 0.55, eps 1e-3, bucket 16, group 64, criterion 0,
 * accumulate 0, terms 15, spin_limit 1<<26, nrep 0.  Returns FMM_ERR_ARG for p == NULL. */
fmm_status fmm_default_params(fmm_params *p);

/* Create a context on CUDA device `device`, enqueuing all work on `cuda_stream`
 * (a cudaStream_t, or NULL for the legacy default stream).  *out receives the
 * context.  FMM_ERR_CUDA if the device cannot be used, FMM_ERR_OOM on allocation
 * failure.  The context's parameters start at fmm_default_params. */
fmm_status fmm_create(fmm_ctx **out, int device, void *cuda_stream);

/* Release the context and all device memory it owns.  NULL is accepted. */
void fmm_destroy(fmm_ctx *ctx);

/* Replace the context's parameters (validated; FMM_ERR_ARG leaves them unchanged). */
fmm_status fmm_set_params(fmm_ctx *ctx, const fmm_params *p);
fmm_status fmm_get_params(const fmm_ctx *ctx, fmm_params *p);

/* Build the tree of N particles: Morton keys, radix sort, binary radix tree with
 * buckets of <= bucket particles, and the upward pass (mass, centre of mass,
 * bounding box, exact b_max, order-4 moments) -- Sec. 3.1.
 *   pos    device, 3N doubles, SoA x|y|z, each in [0,1)
 *   mass   device, N floats, > 0
 *   active device, N bytes (non-zero = active) or NULL for all active
 *   n      1 <= n < 2^31
 *   p      parameters (bucket is used) or NULL for the context's
 * Returns after the tree is built (the cell count is read back to size the upward
 * pass).  Invalid positions or masses are reported as FMM_ERR_ARG. */
fmm_status fmm_build_tree(fmm_ctx *ctx, const double *pos, const float *mass, const unsigned char *active,
                          long long n, const fmm_params *p);

/* Full force solve (Sec. 3.1): build the tree, walk it with the context's
 * criterion, evaluate PP, PC and local expansions for every group that holds an
 * active particle, and write the results in the caller's order.
 *   pos, mass, active, n   as for fmm_build_tree
 *   eps, theta             softening (> 0) and opening angle (0 < theta <= 1);
 *                          they override the context's parameters for this call
 *   acc    device, 3N floats SoA out (ax|ay|az); entries of inactive particles
 *          are left unchanged.  With criterion 1 it is also read on entry: an estimate of
 *          every particle's acceleration (e.g. the previous step's) that scales the learned
 *          criterion's error budget; sink cells whose smallest estimate is zero fall back to
 *          the fixed criterion
 *   pot    device, N floats out, or NULL
 * Returns after completion (see Streams).  Statistics via fmm_get_stats. */
fmm_status fmm_compute_forces(fmm_ctx *ctx, const double *pos, const float *mass, const unsigned char *active,
                              long long n, double eps, double theta, float *acc, float *pot);

/* Force solve of several independent isolated boxes in one pass (one tree build, one walk and
 * one launch of every interaction kernel for all boxes).  Box b holds the particles
 * [box_offsets[b], box_offsets[b+1]) of the concatenated SoA arrays; each box is its own unit
 * box [0,1)^3 and its particles feel only each other.  box_offsets: HOST array of nbox + 1
 * non-decreasing values from 0 to n; 1 <= nbox <= 256.  Other arguments, outputs and
 * semantics as for fmm_compute_forces; every box's results equal those of solving it alone. */
fmm_status fmm_compute_forces_batch(fmm_ctx *ctx, const double *pos, const float *mass,
                                    const unsigned char *active, long long n, const long long *box_offsets,
                                    int nbox, double eps, double theta, float *acc, float *pot);

/* CUDA graphs (not in the paper).  With enable = 1, a force solve (fmm_compute_forces, _batch,
 * _host, and the autotuner's solves) that repeats the previous call's buffers (pos, mass,
 * active, acc, pot pointers), n, box offsets, eps, theta and parameters replays the solve as two
 * CUDA graphs: the first builds the keys, the sorted particles and the radix tree and reads back
 * the tree's cell count; the host checks it against the cell buffers and launches the second
 * (everything else), then synchronises once at the end.  The first call of a new combination runs
 * eagerly and captures the graphs (on the context's stream, in thread-local capture mode) for the
 * next.  A replay that finds the cell buffers, another buffer or the walk's level count too small
 * repeats the solve eagerly, which grows what it must, and recaptures.  Results are identical to
 * eager solves.  enable = 0 (the default) drops the graph.  The contents of the buffers may change
 * between calls; their addresses may not (a new address means a new capture). */
fmm_status fmm_set_graphs(fmm_ctx *ctx, int enable);

/* Whether a graph is currently captured (*captured 0/1) and how many solves replayed one so far
 * (*replays); either pointer may be NULL. */
fmm_status fmm_graph_info(const fmm_ctx *ctx, int *captured, long long *replays);

/* Autotuner (not in the paper): times force solves of the given particles (device buffers, as
 * for fmm_compute_forces; box_offsets/nbox as for fmm_compute_forces_batch, or NULL/1 for one box)
 * for each candidate setting and leaves the fastest in the context's parameters.
 *   candidates   host array of n_candidates fmm_params of which bucket, group and list_chunk are
 *                tried (the other fields stay the context's), or NULL for the built-in grid:
 *                bucket {8, 12, 16} x group {32, 48, 64} x list_chunk {32, 64, 128}
 *   reps         timed solves per candidate after one untimed solve, 1..100
 *   acc          device scratch of 3N floats (overwritten)
 *   best, best_ms  HOST outputs (may be NULL): the chosen parameters and their mean time per
 *                solve in ms (CUDA events on the context's stream)
 * Every candidate is a valid FMM at the same theta; they differ in how work is cut (leaf and group
 * sizes, work-item size), so the force errors differ only slightly.  A failing candidate stops
 * the tuner with its error and restores the previous parameters. */
fmm_status fmm_autotune(fmm_ctx *ctx, const double *pos, const float *mass, long long n, const long long *box_offsets,
                        int nbox, double eps, double theta, const fmm_params *candidates, int n_candidates, int reps,
                        float *acc, fmm_params *best, float *best_ms);

/* Same as fmm_compute_forces with HOST buffers: pos (3N doubles), mass (N floats),
 * active (N bytes or NULL) are copied to device memory owned by the context, and
 * acc (3N floats) / pot (N floats or NULL) are copied back before returning (acc is also
 * copied in first when active is given or the criterion is 1). */
fmm_status fmm_compute_forces_host(fmm_ctx *ctx, const double *pos, const float *mass,
                                   const unsigned char *active, long long n, double eps, double theta, float *acc,
                                   float *pot);

/* One substep of the hierarchical kick-drift-kick leapfrog on time-step rungs
 * (Sec. 3.2, Fig. KDK).  The base step dt0 is cut into 2^max_rung substeps of
 * h = dt0 / 2^max_rung; particle i sits on rung r_i (step dt0 / 2^r_i) and is active at
 * substep s when s is a multiple of 2^(max_rung - r_i).  For substep s this call does,
 * for the particles active at s:
 *   1. if closing != 0, the closing half kick v += a dt0 / 2^(r_i + 1) of the step that
 *      ends at s (pass closing = 0 for the very first substep of a run),
 *   2. rung reassignment from Delta T = 0.2 sqrt(eps / |a|) (Sec. 3.2): the target rung
 *      is the smallest r in [0, max_rung] with dt0 / 2^r <= Delta T; a particle moves
 *      to a coarser rung only at a substep where that rung is synchronised,
 *   3. the opening half kick v += a dt0 / 2^(r_i + 1) with the new rung;
 * then drifts every particle, x += v h (FP64), and marks in active_next the particles
 * active at substep s + 1, whose forces the caller computes next (for example with
 * fmm_compute_forces(..., active_next, ...)).
 *   pos   device, 3N doubles SoA, updated in place (must stay in [0,1): a particle that
 *         leaves the box is reported as FMM_ERR_ARG by the next synchronising call)
 *   vel   device, 3N doubles SoA, updated in place
 *   acc   device, 3N floats SoA: accelerations at substep s of the active particles
 *   rung  device, N bytes in [0, max_rung], updated in place
 *   active_next  device, N bytes out
 *   eps > 0, dt0 > 0, 0 <= max_rung <= 30, 0 <= substep < 2^max_rung.
 * Asynchronous. */
fmm_status fmm_kick_drift(fmm_ctx *ctx, double *pos, double *vel, const float *acc, unsigned char *rung,
                          unsigned char *active_next, long long n, double eps, double dt0, int max_rung,
                          int substep, int closing);

/* ---------------------------------------------------------------- compressed storage (Sec. 3.4)
 *
 * The paper stores positions as 32-bit integer coordinates of the box (converted from and to
 * doubles, a resolution well below the softening length) and velocities as single-precision
 * floats.  These calls take that storage directly:
 *   ipos  device, 3N unsigned 32-bit SoA (x then y then z): the coordinate is u * 2^-32 of the
 *         unit box (exact in FP64), always inside [0, 1)
 *   vel   device, 3N floats SoA
 *
 * fmm_compute_forces_i32: fmm_compute_forces on those positions; the results are bit for bit those
 * of fmm_compute_forces on the FP64 positions u * 2^-32.  Graph replay, periodic boxes and the
 * learned criterion work as there; FMM_ERR_ARG for NULL ipos or mass or n out of range. */
fmm_status fmm_compute_forces_i32(fmm_ctx *ctx, const unsigned int *ipos, const float *mass,
                                  const unsigned char *active, long long n, double eps, double theta, float *acc,
                                  float *pot);

/* fmm_kick_drift_i32: the substep of fmm_kick_drift on compressed storage.  The kicks of a substep
 * are FP64 from the stored FP32 velocity (each product and sum rounded once), and the velocity is
 * stored rounded to FP32; the drift adds to u the nearest integer of v h 2^32 (FP64, ties to even).
 * In a periodic box (fmm_params.nrep > 0) u wraps modulo 2^32, the box's period; in the isolated box
 * a particle that would leave [0, 1) keeps its position and the next synchronising call reports
 * FMM_ERR_ARG.  Asynchronous; the other arguments as for fmm_kick_drift. */
fmm_status fmm_kick_drift_i32(fmm_ctx *ctx, unsigned int *ipos, float *vel, const float *acc, unsigned char *rung,
                              unsigned char *active_next, long long n, double eps, double dt0, int max_rung,
                              int substep, int closing);

/* Device memory the context holds: *device_bytes = its buffers (tree, lists, scratch, staging,
 * network) as allocated so far, *host_bytes = its pinned host mirrors; either may be NULL. */
fmm_status fmm_memory_info(const fmm_ctx *ctx, long long *device_bytes, long long *host_bytes);

/* Assign rungs from accelerations: the smallest r in [0, max_rung] with dt0 / 2^r <= Delta T,
 * Delta T = 0.2 sqrt(eps / |a|) (Sec. 3.2).  acc device 3N floats SoA, rung device N bytes out.
 * Asynchronous. */
fmm_status fmm_assign_rungs(fmm_ctx *ctx, const float *acc, unsigned char *rung, long long n, double eps,
                            double dt0, int max_rung);

/* ---------------- dual trees for multiple time steps (Sec. 3.2) ----------------
 * On the substeps between two kicks of the slower rungs only the fast rungs need forces.  The
 * particles of rungs <= r_fixed are not kicked there, so they move on straight lines; they are
 * drifted to the middle of the interval once and a "fixed" tree of them is kept, and each
 * substep builds a tree of the other (fast) particles and walks it against both trees.  Both
 * trees are radix trees over Morton keys of the same unit box, so their cells are the same
 * dyadic boxes; the active tree is moreover graded on the fixed one (the shared geometric
 * structure the method asks for): a node keeps splitting while the fixed tree holds more than
 * b particles in its box, and is no sink group while it holds more than g there, so active
 * leaves and groups are never larger than the fixed tree's around them. */

/* Build and keep the fixed tree: the particles i with rung[i] <= r_fixed (every particle when
 * rung is NULL), at positions pos_i + vel_i * dt (FP64; pos_i when vel is NULL).  Which particles
 * of the n are fixed is kept for the dual solves, which must pass the same n.
 *   pos, vel  device, 3N doubles SoA (vel may be NULL); the drifted positions must lie in [0,1)
 *   mass      device, N floats;  rung  device, N bytes or NULL
 *   dt        the drift to the middle of the interval (finite)
 * The tree uses the context's bucket size, which later dual solves must keep (FMM_ERR_ARG
 * otherwise).  It replaces any earlier fixed tree; zero selected particles give an empty one.
 * Uses the context's tree buffers (an earlier solve's exports are gone); afterwards fmm_get_stats
 * reports the fixed tree's particles, cells, buckets and this call's kernel launches.  Synchronous. */
fmm_status fmm_set_fixed_sources(fmm_ctx *ctx, const double *pos, const double *vel, const float *mass,
                                 const unsigned char *rung, long long n, int r_fixed, double dt);

/* Force solve on a substep inside the fixed tree's interval.  Every particle outside the fixed
 * set (the fast rungs) goes into an active tree at its current position, built on each call; the
 * fixed tree is appended to it and the walk starts with both roots on the checklist.  The sinks
 * are the particles marked in active.
 *   pos, mass  device, the caller's full arrays (3N doubles SoA, N floats), N as given to
 *              fmm_set_fixed_sources (FMM_ERR_ARG otherwise)
 *   active     device, N bytes: the sinks, particles outside the fixed set (NULL: all of them);
 *              flags on fixed particles are ignored (they are not kicked inside the interval)
 *   acc, pot   device, 3N / N floats (pot may be NULL): written for the sinks only
 * Criterion 0 only (FMM_ERR_ARG otherwise); FMM_ERR_STATE when no fixed tree was set.  With no
 * particle outside the fixed set nothing is written.  Statistics via fmm_get_stats (cells and
 * buckets count both trees).  Synchronous; no CUDA graph. */
fmm_status fmm_compute_forces_dual(fmm_ctx *ctx, const double *pos, const float *mass, const unsigned char *active,
                                   long long n, double eps, double theta, float *acc, float *pot);

/* ---------------- learned opening criterion (not in the paper; criterion = 1) ----------------
 * The network x (8) -> 64 -> 64 -> 64 -> 1 (ReLU) predicts log10 of the relative force error of
 * accepting a (sink cell, source cell) pair as a cell-cell interaction, from the features
 *   b_max(s)/d, b_max(k)/d, eps/d, log10(M_s / (d^2 a_k)), log2 N_s, log2 N_k,
 *   |M2|_F/(M_s b_s^2), |M4|_F/(M_s b_s^4)
 * (d distance of the centres of mass, M_s the source's mass, a_k the smallest acceleration
 * estimate of the sink's particles).  Parameters: FMM_MLP_NP
 * floats, W1 [64x8], b1 [64], W2 [64x64], b2 [64], W3 [64x64], b3 [64], w4 [64], b4 [1] (row-
 * major), then the feature normalisation mean [8] and inv_std [8], then a surrogate bound
 * [alpha, beta, r_lo, r_hi, gamma[8]]: pairs whose y_lin = f_3 + alpha log10(theta_eff) + beta +
 * sum_i gamma_i f_i (f the raw features) satisfies y_lin + r_hi < mlp_tau are accepted and those
 * with y_lin + r_lo >= mlp_tau are rejected without evaluating the network (training sets it from
 * the labels and the network's residuals; r_hi <= r_lo turns it off).  Inference runs on the tensor cores with BF16 weights and
 * FP32 accumulation; training in FP32 with Adam. */
#define FMM_MLP_NP 8989
#define FMM_MLP_NW 8961

/* Load (host, FMM_MLP_NP floats) or read back the context's network parameters. */
fmm_status fmm_mlp_load(fmm_ctx *ctx, const float *params, long long n);
fmm_status fmm_mlp_get(const fmm_ctx *ctx, float *params, long long n);

/* Predictions for n feature rows: feats device n x 8 floats (raw features), out device n floats. */
fmm_status fmm_mlp_predict(fmm_ctx *ctx, const float *feats, long long n, float *out);

/* Loss 0.5 mean((y - label)^2) and its gradient with respect to the FMM_MLP_NW weights over
 * the n rows (feats device n x 8, labels device n); grad and loss are HOST outputs. */
fmm_status fmm_mlp_gradient(fmm_ctx *ctx, const float *feats, const float *labels, long long n, float *grad,
                            float *loss);

/* Train the network on n labelled rows (device): feature normalisation from the data, weights
 * initialised from seed (He-uniform, output bias = mean label), then epochs of Adam on shuffled
 * minibatches of `batch` rows with learning rate lr; last, the surrogate bound is fitted to the
 * same rows.  *final_loss (host, may be NULL) gets the last epoch's mean training loss. */
fmm_status fmm_mlp_train(fmm_ctx *ctx, const float *feats, const float *labels, long long n, int epochs, int batch,
                         float lr, unsigned int seed, float *final_loss);

/* Audit: build the tree of N particles, walk it with the fixed criterion at theta, record every
 * (sink cell, source cell) pair with band_lo <= theta_eff < band_hi that passes the guard (at
 * most max_pairs), and write for each its 8 features (feats, device max_pairs x 8) and label
 * (labels, device max_pairs): log10 of the largest relative force error, over up to 32
 * particles of the sink, of the cell-cell expansion of the source against the direct sum of its
 * particles, relative to the particle's total acceleration acc_ref (device, 3N SoA, input order),
 * which also serves as the acceleration estimate of the features.
 * *n_pairs (host) = pairs written. */
fmm_status fmm_mlp_audit(fmm_ctx *ctx, const double *pos, const float *mass, long long n, double eps,
                         double theta, double band_lo, double band_hi, const float *acc_ref, long long max_pairs,
                         float *feats, float *labels, long long *n_pairs);

/* The (sink cell, source cell) pairs of the last audit as particle ranges in the sorted order
 * (HOST outputs of n entries, n <= the audit's *n_pairs; any pointer may be NULL). */
fmm_status fmm_mlp_audit_pairs(const fmm_ctx *ctx, int *sink_first, int *sink_count, int *src_first, int *src_count,
                               long long n);

/* Statistics of the last solve.  Synchronises the context's stream. */
fmm_status fmm_get_stats(const fmm_ctx *ctx, fmm_stats *out);

/* Message of the last error on the calling thread ("" if none). Never NULL. */
const char *fmm_last_error(void);

/* FP32 flops per particle-cell interaction performed by the PC kernel (a constant of the build). */
double fmm_flops_per_pc(void);

/* ---------------- introspection (stage-by-stage parity; synchronise the stream) ----------------
 * All outputs are HOST buffers sized from fmm_tree_info.  Valid after fmm_build_tree
 * (tree exports) or fmm_compute_forces (list and local exports); FMM_ERR_STATE otherwise.
 * Cells are numbered by the library; a cell is identified across implementations by its
 * particle range [first, first + count) in the sorted (Morton) order, which is the
 * stable sort of the keys by (key, input index). */
fmm_status fmm_tree_info(const fmm_ctx *ctx, long long *n_cells, long long *n_groups, long long *n_pp_entries,
                         long long *n_pc_entries, long long *n_local_entries);

/* perm[i] = input index of the i-th particle in sorted order; keys[i] its 63-bit Morton key
 * (level l of the tree bisects axis l mod 3 in the order x, y, z; 21 bits per axis). */
fmm_status fmm_export_order(const fmm_ctx *ctx, unsigned int *perm, unsigned long long *keys);

/* Per cell: first, count, parent (-1 for the root), child (2 per cell, -1 for leaves),
 * number of active particles, mass, centre of mass (3), bounding box lo (3) / hi (3),
 * b_max, and the moment record (44 floats: M, M2 (6), M3 (10), M4 (15) about the centre of
 * mass, then the traces trM2, trM3 (3), trM4 (6), trtrM4, 0).  Any pointer may be NULL. */
fmm_status fmm_export_cells(const fmm_ctx *ctx, int *first, int *count, int *parent, int *child, int *nact,
                            double *mass, double *com, double *lo, double *hi, double *bmax, float *moments);

/* Interaction lists of the last solve.  kind: 0 PP, 1 PC, 2 CC, 3 CP.  For every entry:
 * the sink cell and the source's particle range (a single particle has count 1).
 * PP and PC entries belong to groups; CC and CP entries to any walked sink cell. */
fmm_status fmm_export_lists(const fmm_ctx *ctx, int kind, long long *n_entries, int *sink, int *src_first,
                            int *src_count, long long capacity);

/* The periodic copy of each entry's source, in the order of fmm_export_lists for the same kind:
 * shift[3i..3i+2] = the integer vector n of the copy the source lies in (Sec. 3.1, periodic
 * boundaries; all zero for an isolated box).  *n_entries receives the entry count; with
 * capacity < *n_entries (or shift NULL) the call only reports it.  shift: host, 3 * capacity ints. */
fmm_status fmm_export_list_shifts(const fmm_ctx *ctx, int kind, long long *n_entries, int *shift, long long capacity);

/* Local expansions of the groups: group_cell[i] and 56 coefficients L_k = D^k Phi at the
 * group's centre of mass, in the order of fmm_multi_index. */
fmm_status fmm_export_locals(const fmm_ctx *ctx, int *group_cell, float *L, long long capacity);

/* Per walk level of the last solve (the root is level 0), for l < min(*n_levels, capacity):
 * counts[3l] = sink cells walked, counts[3l+1] = checklist entries they examined (opened
 * entries included), counts[3l+2] = the largest number examined by one sink.  Any of the
 * three may be used; counts must hold 3 * capacity values. */
fmm_status fmm_export_walk_levels(const fmm_ctx *ctx, long long *counts, int capacity, int *n_levels);

/* The 56 multi-indices (a, b, c) of the local coefficients in storage order (168 ints),
 * and the 32 multi-indices of the moment slots (96 ints).  Either may be NULL. */
fmm_status fmm_multi_index(int *local_idx, int *moment_idx);

/* ---------------------------------------------------------------- test hooks
 *
 * Not in the paper: they let tests drive the library's recovery paths from the host, with no GPU
 * fault.
 *
 * fmm_debug_fail_allocations: the calling thread's next `after` device allocations of any context
 * succeed and the ones after them fail as out of memory (FMM_ERR_OOM from the call that needed
 * them); after < 0 switches the hook off.  A context whose allocation failed stays usable: the
 * buffers involved are allocated again by its next call.
 *
 * fmm_debug_walk_capacity: the walk's first capacities for a context whose buffers have not been
 * sized yet: scratch_entries per warp and list (default 8192) and list_scale checklist, local and
 * PC entries per particle (defaults 8, 12 and 8; PP half of list_scale, rounded up, default 3);
 * 0 keeps the defaults.  Each overflow doubles them and repeats the walk, up to 8 times, so small
 * values exercise that path.  Returns FMM_ERR_ARG for ctx == NULL or negative values.
 *
 * fmm_debug_local_side: the walk size, in sinks of the context's previous walk, from which each
 * walk level's local expansions (M2L, P2L, L2L) run on a side stream beside the levels below
 * instead of after the last level (default 2^22; a context's first walk never uses it).  Both
 * orders give the same bits, since every sink's terms are added in its own list order; 0 takes the
 * side stream whenever the context has walked before, so tests can compare the two.  A negative
 * value restores the default.  Returns FMM_ERR_ARG for ctx == NULL. */
fmm_status fmm_debug_fail_allocations(long long after);
fmm_status fmm_debug_walk_capacity(fmm_ctx *ctx, long long scratch_entries, long long list_scale);
fmm_status fmm_debug_local_side(fmm_ctx *ctx, long long min_sinks);

/* ---------------------------------------------------------------- allocation-free Morton order
 *
 * The paper has no counterpart to this call: it exists for callers that cannot let a library
 * allocate device memory while they run, such as an application that has already given the
 * device's free memory to its own pool (cudaMalloc would fail there), or one whose loop cannot
 * take the device-wide synchronisation that cudaFree implies.  It computes the key and sort stage
 * of fmm_build_tree (Sec. 3.1, hierarchically sorted order) with no context, no cudaMalloc or
 * cudaFree and no other allocating routine: its scratch is a fixed ~13.6 MB array in the
 * library's device image, which bounds n by FMM_STATIC_ORDER_MAX_N.
 *
 *   pos   device, FP64, SoA [3][n] (x then y then z), read only; every coordinate in [0, 1)
 *   n     1 <= n <= FMM_STATIC_ORDER_MAX_N; larger n is rejected with FMM_ERR_ARG before any work
 *   keys  device, n values, written: the 63-bit Morton keys in ascending order
 *   order device, n values, written: order[i] = input index of the i-th particle in that order
 *         (ties in input order); keys and order equal fmm_export_order after fmm_build_tree
 *   cuda_stream  the cudaStream_t to run on (NULL: the legacy default stream), on the calling
 *         thread's current device; the call returns after that stream has finished the work.
 *
 * The first call on each device looks up the scratch array's device address (and sets a kernel
 * attribute) with that device current.
 * One scratch array serves all calls on a device: calls that overlap in time (from several
 * threads, or on several streams) race on it and must be serialised by the caller.
 * Errors: FMM_ERR_ARG for NULL pointers, n out of range or a position outside [0, 1) (keys and
 * order are then not valid), FMM_ERR_CUDA when a CUDA call fails. */
#define FMM_STATIC_ORDER_MAX_N 1048576
fmm_status fmm_morton_order_static(const double *pos, long long n, unsigned long long *keys, unsigned int *order,
                                   void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FMM_GB300_H */
