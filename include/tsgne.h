/*
 * tsgne.h -- C ABI of the GB300 t-SGNE layout library (libtsgne.so).
 *
 * t-SGNE (Li, Xiao, Zhou, "Efficiently Visualizing Large Graphs",
 * arXiv 2310.11186) places the nodes of an undirected graph G in 2-D: it runs
 * t-SNE (Sec. 2.1, Eqs. 2-5) with the neighbour graph taken from G instead of
 * from the embedding X (Sec. 2.2, Eq. 7).  This library implements the layout
 * loop on one GPU:
 *
 *   tsgne_build_P  neighbour structure (Eq. 7), conditional affinities with
 *                  the perplexity binary search (Eq. 2, Sec. 2.1) and the
 *                  joint affinities (Eq. 3);
 *   tsgne_step     one gradient-descent iteration on KL(P||Q) (Eq. 5): the
 *                  sparse attraction over P, the exact all-pairs Student-t
 *                  repulsion with its normaliser Z (Eq. 4), and the
 *                  gains / momentum / early-exaggeration update;
 *   tsgne_run      many iterations (CUDA-graph replay);
 *   tsgne_kl       the objective of Eq. 5 at the current layout.
 *
 * Conventions shared by every call:
 *   - Every call returns a tsgne_status; nothing aborts and no C++ exception
 *     crosses this boundary.  On error, tsgne_last_error(ctx) holds a message.
 *     TSGNE_ERR_CUDA leaves the context unusable (destroy it); every other
 *     error leaves it as it was before the call unless stated otherwise.
 *   - A context is bound to one CUDA device (the current one at creation) and
 *     one stream; it is not thread-safe.  Distinct contexts are independent.
 *   - Input pointers are borrowed for the duration of the call and copied.
 *     ptr_kind says where they live (TSGNE_PTR_HOST or TSGNE_PTR_DEVICE).
 *     Output buffers are owned by the caller and must have the stated size.
 *   - Calls that return results to the caller synchronise the context's
 *     stream; tsgne_step only enqueues work.
 *   - Layout Y is n x 2 row-major float (x0, y0, x1, y1, ...).  Coordinates
 *     must stay below 1e18 in magnitude (the repulsion pads ragged tiles with
 *     points at 1e30 whose kernel value underflows to exactly zero).
 */
#ifndef TSGNE_H
#define TSGNE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsgne_ctx tsgne_ctx;

typedef enum {
  TSGNE_OK = 0,
  TSGNE_ERR_INVALID_ARG = 1, /* bad size, NULL pointer, perplexity <= 1, n < 2, ... */
  TSGNE_ERR_BAD_CSR = 2,     /* row_ptr[0] != 0, decreasing row_ptr, column outside [0, n) */
  TSGNE_ERR_OOM = 3,         /* device allocation failed; ctx unchanged */
  TSGNE_ERR_CUDA = 4,        /* CUDA runtime error; ctx must be destroyed */
  TSGNE_ERR_NOT_BUILT = 5,   /* call needs P (tsgne_build_P / tsgne_set_P) or Y first */
  TSGNE_ERR_NONFINITE = 6,   /* NaN / Inf met in X, P or the layout */
  TSGNE_ERR_TIMEOUT = 7,     /* a bounded device-side wait ran out */
  TSGNE_ERR_CANCELLED = 8,   /* work cancelled by the caller */
  TSGNE_ERR_INDEX = 9        /* debug build (libtsgne_debug.so) only: an index check failed and its
                                access was skipped; the results of that pass are not valid */
} tsgne_status;

typedef enum { TSGNE_PTR_HOST = 0, TSGNE_PTR_DEVICE = 1 } tsgne_ptr_kind;

/*
 * Parameters.  Only the perplexity comes from the paper (Sec. 2.1: typically
 * 5-50, default 30); the paper gives no optimiser, so the published t-SNE
 * schedule is the default: early exaggeration 12 for 250 iterations,
 * momentum 0.5 then 0.8, learning rate max(n / early_exag / 4, 50), gains
 * +0.2 / x0.8 with a floor of 0.01.
 */
typedef struct {
  float perplexity;        /* target Perp(P_i) = 2^{H(P_i)} (Sec. 2.1); > 1 */
  int32_t k_nn;            /* 0: neighbours = graph edges; 1..256: the first k_nn nodes in
                              breadth-first order from each node (Eq. 7), ties by ascending
                              id, symmetrised by union */
  float early_exag;        /* alpha multiplying P in the gradient while t < ee_iters */
  int32_t ee_iters;        /* length of the early-exaggeration phase */
  float momentum0;         /* momentum while t < ee_iters */
  float momentum1;         /* momentum afterwards */
  float learning_rate;     /* <= 0: max(n / early_exag / 4, 50) */
  float min_gain;          /* floor of the per-coordinate gains */
  float bisect_tol;        /* |H_i - ln perp| tolerance of the bisection, nats */
  int32_t bisect_max_iter; /* max entropy evaluations per row */
  uint64_t seed;           /* seed of tsgne_init_Y(ctx, NULL, ...) */
  int32_t precision;       /* storage read by the force kernels (arithmetic is FP32, Z and KL
                              FP64 in both): 0 = FP32 P and Y; 1 = BF16 copies of P and of
                              the layout, rounded to nearest even from the FP32 values, which
                              stay the optimiser's master copy and what every getter returns.
                              Not an option of the paper; the batch API accepts 0 only. */
  int32_t profile;         /* 1: time every kernel with CUDA events (see tsgne_kernel_times) */
  int64_t spin_budget_cycles; /* > 0: SM clock cycles a device-side wait may last (the look-back
                                 of the tree code's sort); past it the pass gives up, its forces
                                 are zero and the next synchronising call returns
                                 TSGNE_ERR_TIMEOUT once (the context stays usable) */
  int32_t repulsion;       /* 0: exact all-pairs sums of Eq. 4 (default); 1: tree code, an
                              approximation the paper does not use: points sorted along a
                              Morton curve, binary radix tree, per group (a maximal subtree
                              of at most 32 points) a walk that takes a node with box side r
                              and centre at distance d from the group's box as one
                              interaction when r < theta * d; opened nodes of <= 4 points
                              are summed exactly.  Z and the forces are both approximated;
                              n must be below 2^30 (else INVALID_ARG when P is built).  The
                              exact sums take at most 2^24 - 2048 points (else INVALID_ARG
                              when P is built).  In the batch API it is the default of the
                              members (tsgne_batch_add_ex chooses per member) */
  float theta;             /* opening angle of the tree code, [0, 1] (default 0.5; 0 sums
                              every pair exactly through the tree) */
  int32_t p_walks;         /* 0: p_{j|i} by the perplexity bisection of Eq. 2 (default);
                              1..512: the random-walk estimate of Eq. 6 instead: p_walks
                              walks of p_walk_length steps from every node over the
                              neighbour graph, a step from u to v in N(u) with probability
                              proportional to exp(-||x_u - x_v||^2); p_{j|i} = (walks from
                              i ending at j) / p_walks, j != i; P then follows Eq. 3 on the
                              symmetrised set of walk pairs (tsgne_get_P returns that
                              structure).  Draws come from SplitMix64 seeded with
                              seed ^ 0xD1B54A32D192ED03, output 1 + (i p_walks + r)
                              p_walk_length + s for step s of walk r from node i. */
  int32_t p_walk_length;   /* steps per walk, 1..64 (default 3) */
} tsgne_config;

/* Fills *cfg with the defaults listed above (perplexity 30). */
void tsgne_config_default(tsgne_config* cfg);

/*
 * Creates a context on the current CUDA device.  cuda_stream is a
 * cudaStream_t the context will use for all of its work; NULL creates a
 * private non-blocking stream.  *out receives the context (NULL on error).
 */
tsgne_status tsgne_create(tsgne_ctx** out, const tsgne_config* cfg, void* cuda_stream);

/* Frees every device buffer of the context.  NULL is ignored. */
void tsgne_destroy(tsgne_ctx* ctx);

/* Message of the last failed call on ctx ("" if none).  Valid until the next
 * call.  With ctx = NULL: the message of the calling thread's last failed
 * call of an entry point that takes no context (tsgne_repulsion_noalloc,
 * tsgne_shortest_path_embedding), valid until that thread's next call. */
const char* tsgne_last_error(const tsgne_ctx* ctx);

/* Static name of a status code. */
const char* tsgne_status_string(tsgne_status s);

/*
 * Builds the joint affinities P from a graph and its high-dimensional
 * embedding (the t-SGNE input pair (G, X), Sec. 2.2):
 *   1. neighbour structure (Eq. 7): with cfg.k_nn = 0, N(i) = { j != i :
 *      (i,j) or (j,i) in G }; with k_nn = k > 0, the first k nodes of the
 *      breadth-first order from i on that graph (levels in order, each node's
 *      neighbours by ascending id), symmetrised by union; either way
 *      symmetric, sorted, unique, no self loops;
 *   2. p_{j|i} = exp(-beta_i ||x_i-x_j||^2) / sum_{k in N(i)} exp(...) (Eq. 2
 *      over N(i)), beta_i by bisection until |H_i - ln perplexity| <=
 *      bisect_tol (Sec. 2.1); rows with |N(i)| <= perplexity are uniform;
 *   3. p_ij = (p_{j|i} + p_{i|j}) / T, T the sum of all numerators (Eq. 3;
 *      T = 2n when no node is isolated), so sum P = 1.
 * With cfg.p_walks > 0 step 2 is the random-walk estimate of Eq. 6 over the
 * structure of step 1 (see tsgne_config.p_walks), and step 3 runs on the
 * symmetrised set of walk pairs, which becomes the structure of P.
 * n >= 2 nodes; row_ptr int64[n+1] with row_ptr[0] = 0, non-decreasing;
 * col_idx int32[row_ptr[n]] in [0, n) (any order, duplicates and self loops
 * allowed, either direction suffices); X float[n*d] row-major, d >= 1.
 * All three arrays live where ptr_kind says.  Resets the layout state
 * (tsgne_init_Y must follow).  Errors: INVALID_ARG, BAD_CSR, NONFINITE (X
 * produced a non-finite affinity), OOM.
 */
tsgne_status tsgne_build_P(tsgne_ctx* ctx, int32_t n, const int64_t* row_ptr, const int32_t* col_idx,
                           const float* X, int32_t d, int32_t ptr_kind);

/*
 * Installs a joint affinity matrix computed elsewhere.  The structure must
 * already be symmetric, sorted, unique and loop-free (else BAD_CSR); P float
 * [row_ptr[n]] holds p_ij per entry (not checked for symmetry or sum).
 * Resets the layout state like tsgne_build_P.
 */
tsgne_status tsgne_set_P(tsgne_ctx* ctx, int32_t n, const int64_t* row_ptr, const int32_t* col_idx,
                         const float* P, int32_t ptr_kind);

/* Number of nodes and of stored affinities (2|E| after symmetrisation). */
tsgne_status tsgne_get_sizes(tsgne_ctx* ctx, int32_t* n, int64_t* nnz);

/*
 * Copies the symmetric structure and P out: row_ptr int64[n+1], col int32[nnz],
 * val float[nnz]; any pointer may be NULL to skip it.
 */
tsgne_status tsgne_get_P(tsgne_ctx* ctx, int64_t* row_ptr, int32_t* col, float* val, int32_t ptr_kind);

/*
 * Sets the initial layout and resets the optimiser (updates 0, gains 1,
 * iteration 0).  Y0 float[n*2]; NULL draws Y0 ~ N(0, 1e-4^2) on the device
 * from cfg.seed with SplitMix64 in counter mode and Box-Muller.
 */
tsgne_status tsgne_init_Y(tsgne_ctx* ctx, const float* Y0, int32_t ptr_kind);

/*
 * One iteration, enqueued on the context's stream (no host synchronisation):
 * repulsion F^r_i = sum_{j != i} w_ij^2 (y_i - y_j) and Z = sum_{k != l} w_kl
 * (Eq. 4, w = (1 + ||y_k - y_l||^2)^-1, Z accumulated in FP64), attraction
 * F^a_i = sum_{j in N(i)} p_ij w_ij (y_i - y_j), gradient
 * g = 4 (alpha F^a - F^r / Z) of Eq. 5, then gains, momentum and y += update.
 * A non-finite layout is reported by the next synchronising call.
 */
tsgne_status tsgne_step(tsgne_ctx* ctx);

/* n_iter iterations by CUDA-graph replay; synchronises at the end. */
tsgne_status tsgne_run(tsgne_ctx* ctx, int32_t n_iter);

/* KL(P || Q) of Eq. 5 at the current layout (one repulsion pass for Z); synchronises. */
tsgne_status tsgne_kl(tsgne_ctx* ctx, double* kl_out);

/*
 * Gradient of Eq. 5 at the current layout with P multiplied by alpha
 * (alpha = 1: the plain KL gradient), without changing any state.
 * g_out float[n*2] where ptr_kind says; z_out (host, may be NULL) receives Z.
 */
tsgne_status tsgne_gradient(tsgne_ctx* ctx, float alpha, float* g_out, double* z_out, int32_t ptr_kind);

/* Current layout into Y_out float[n*2]. */
tsgne_status tsgne_get_Y(tsgne_ctx* ctx, float* Y_out, int32_t ptr_kind);

/*
 * Optimiser state for checkpoint / resume: layout, updates and gains
 * (float[n*2] each, any may be NULL) and the iteration counter (host).
 * set_state restores exactly what get_state returned, so a resumed run is
 * bit-identical to an uninterrupted one.
 */
tsgne_status tsgne_get_state(tsgne_ctx* ctx, float* Y, float* update, float* gains, int32_t* iter,
                             int32_t ptr_kind);
tsgne_status tsgne_set_state(tsgne_ctx* ctx, const float* Y, const float* update, const float* gains,
                             int32_t iter, int32_t ptr_kind);

/*
 * Profiling (cfg.profile = 1): cumulative device time in ms and launch count
 * of each kernel class since the last reset, measured with CUDA events on
 * the context's stream.  Classes: 0 repulsion (the tree walk when
 * cfg.repulsion = 1), 1 attraction+update (hub-row chunks included), 2
 * gradient export, 3 KL, 4 build, 5 repulsion force conversion, 6 hub-row
 * attraction chunks of the gradient export, 7 tree build
 * (bounding box, keys, sort, tree, summaries).  ms and launches hold n
 * entries (n <= 8).
 * reset != 0 clears the counters after reading.  Synchronises.
 */
tsgne_status tsgne_kernel_times(tsgne_ctx* ctx, double* ms, int64_t* launches, int32_t n, int32_t reset);

/*
 * Process-wide limit on the device bytes the library holds (contexts,
 * batches and servers together, the no-allocation entry point's static array
 * excepted); bytes <= 0 removes it.  An allocation that would pass the limit
 * fails with TSGNE_ERR_OOM before cudaMalloc is called; the object that
 * asked stays usable (a later call may retry).  The paper has no
 * counterpart: the limit serves hosts that share a GPU among tenants, and
 * tests of the out-of-memory paths.
 */
void tsgne_set_device_memory_limit(int64_t bytes);

/* Device bytes the library holds at the moment (same account). */
int64_t tsgne_device_memory_in_use(void);

/* Launch geometry of the exact repulsion pass (cfg.repulsion = 0; with the
 * tree code the layout buffers still use this padding): grid CTAs, threads
 * per CTA, i per thread, j-tile, j-chunks, pad length.  Any pointer may be
 * NULL. */
tsgne_status tsgne_repulsion_shape(tsgne_ctx* ctx, int32_t* grid, int32_t* block, int32_t* i_per_thread,
                                   int32_t* j_tile, int32_t* j_chunks, int32_t* n_pad);

/*
 * Shape of the exact repulsion pass (cfg.repulsion = 0), after P is built.
 * symmetric = 1: each unordered pair once, tile_warps 1 or 2 warps per CTA,
 * i_per_lane 8 or 16 i-points per lane (the default is chosen from n:
 * 16 i-points, 2 warps once the tile pairs fill four waves of the grid);
 * symmetric = 0: the ordered-pair kernel (every ordered pair, partial forces
 * per j-chunk; FP32 storage only; tile_warps / i_per_lane ignored).  Results
 * depend on the shape only through the order of FP32 partial sums.
 * tsgne_autotune times trial_passes repulsion passes of each shape (in the
 * order (2, 16, 1), (1, 16, 1), (2, 8, 1), (1, 8, 1), (-, -, 0); -1 in
 * ms_per_pass, 5 floats, for a shape that does not apply), keeps the
 * fastest and records it per (SM count, ceil log2 n, storage); the layout
 * and the iteration counter are unchanged.  Synchronises.
 */
tsgne_status tsgne_set_repulsion_shape(tsgne_ctx* ctx, int32_t tile_warps, int32_t i_per_lane, int32_t symmetric);
tsgne_status tsgne_autotune(tsgne_ctx* ctx, int32_t trial_passes, int32_t* tile_warps, int32_t* i_per_lane,
                            int32_t* symmetric, float* ms_per_pass);

/* Waits for all work of the context; reports a pending NONFINITE layout. */
tsgne_status tsgne_sync(tsgne_ctx* ctx);

/*
 * ---------------------------------------------------------------- batches
 * Many layouts advanced together: every iteration of every member runs in
 * four kernel launches (five when a member has rows of more than 32
 * entries; replayed as one CUDA graph per membership) instead of two
 * launches per member.  Each member keeps its own P, layout, optimiser
 * state and iteration counter on the device, may be added or removed between
 * runs (continuous batching), and evolves exactly as it would in a batch of
 * its own: the per-member arithmetic, including the order of every
 * reduction, does not depend on the other members.  The attraction sums
 * rows as the single-layout path does (rows above 32 entries in 1024-entry
 * warp chunks added in chunk order), so a batch of one equals tsgne_run at
 * the same repulsion tile.  cfg.repulsion = 1 makes every member a tree-code
 * member (see tsgne_batch_add_ex); precision must be 0.  All members share one
 * repulsion tile of 512 * tile_warps points (1, 2 or 4; smaller tiles pad
 * small graphs less, larger tiles amortise more per unit).  The same
 * conventions as the context API apply (status codes, one stream, not
 * thread-safe); the batch API has its own error string.
 */
typedef struct tsgne_batch tsgne_batch;

/* Creates an empty batch; tile_warps 0 means 1 until tsgne_batch_autotune runs. */
tsgne_status tsgne_batch_create(tsgne_batch** out, const tsgne_config* cfg, int32_t tile_warps, void* cuda_stream);
void tsgne_batch_destroy(tsgne_batch* b);
const char* tsgne_batch_last_error(const tsgne_batch* b);

/*
 * Adds a layout: builds its P exactly as tsgne_build_P does (same arguments)
 * and sets its initial layout Y0 (float[n*2]; NULL: N(0, 1e-4^2) from
 * cfg.seed), updates 0, gains 1, iteration 0.  *id_out receives the member id.
 */
tsgne_status tsgne_batch_add(tsgne_batch* b, int32_t n, const int64_t* row_ptr, const int32_t* col_idx, const float* X,
                             int32_t d, const float* Y0, int32_t ptr_kind, int32_t* id_out);

/* tsgne_batch_add with the member's repulsion chosen here (0: exact,
 * 1: tree code with the batch's theta) instead of by the batch's
 * cfg.repulsion.  A tree member takes no part in the shared exact pass: its
 * tree is built and walked by its own launches, on a branch of the
 * iteration that runs concurrently with the other members'; its layout is
 * the same as the single-layout tree code's for the same inputs. */
tsgne_status tsgne_batch_add_ex(tsgne_batch* b, int32_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                const float* X, int32_t d, const float* Y0, int32_t ptr_kind, int32_t repulsion,
                                int32_t* id_out);

/*
 * tsgne_batch_add_ex in two steps, so that a new member's build overlaps
 * with the batch's running iterations.  tsgne_batch_prepare builds the
 * member (structure, P, buffers, state; same arguments as
 * tsgne_batch_add_ex) on cuda_stream (not NULL, not the batch's stream)
 * without touching the batch's membership, so it may run on another thread
 * while tsgne_batch_run runs; its device memory is allocated stream-ordered
 * on cuda_stream (cudaMallocAsync), which must outlive the member.  It
 * synchronises cuda_stream; on error *out is NULL and tsgne_last_error(NULL)
 * on that thread says why.  tsgne_batch_attach adds a prepared member (it
 * joins at the next run) and consumes the handle; tsgne_batch_discard frees
 * one that will not be attached.  Calls on one batch other than prepare
 * stay single-threaded.
 */
typedef struct tsgne_member tsgne_member;
tsgne_status tsgne_batch_prepare(tsgne_batch* b, int32_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                 const float* X, int32_t d, const float* Y0, int32_t ptr_kind, int32_t repulsion,
                                 void* cuda_stream, tsgne_member** out);
tsgne_status tsgne_batch_attach(tsgne_batch* b, tsgne_member* m, int32_t* id_out);
void tsgne_batch_discard(tsgne_member* m);

/* Removes a member and frees its device memory. */
tsgne_status tsgne_batch_remove(tsgne_batch* b, int32_t id);

/* Members, tile warps and the repulsion work units of one iteration of the active members. */
tsgne_status tsgne_batch_size(tsgne_batch* b, int32_t* members, int32_t* tile_warps, int64_t* units);

/* n_iter iterations of every member; synchronises; NONFINITE if any layout diverged. */
tsgne_status tsgne_batch_run(tsgne_batch* b, int32_t n_iter);

/* Current layout of a member (float[n*2]) and its iteration count (host, may be NULL). */
tsgne_status tsgne_batch_get_Y(tsgne_batch* b, int32_t id, float* Y_out, int32_t* iter, int32_t ptr_kind);

/*
 * Marks a member active (default) or inactive.  tsgne_batch_run advances
 * only active members; inactive ones keep their state untouched (schedulers
 * use this to run short jobs first without evicting long ones).
 */
tsgne_status tsgne_batch_set_active(tsgne_batch* b, int32_t id, int32_t active);

/* Changes the repulsion tile of the batch (members' states are kept). */
tsgne_status tsgne_batch_set_tile(tsgne_batch* b, int32_t tile_warps);

/* Changes the shape of the batched exact pass: tile_warps 1, 2 or 4 warps
 * per CTA and i_per_lane 8 or 16 i-points per lane (the tile is 32 x
 * i_per_lane x tile_warps points; 8 i-points need half the registers, so
 * twice as many warps per SM are launched).  Members' states are kept; a
 * member's results depend on the shape (the order of its FP32 partial sums)
 * but not on the other members. */
tsgne_status tsgne_batch_set_shape(tsgne_batch* b, int32_t tile_warps, int32_t i_per_lane);
tsgne_status tsgne_batch_shape(tsgne_batch* b, int32_t* tile_warps, int32_t* i_per_lane);

/* Resets every member to its initial layout, updates 0, gains 1, iteration 0. */
tsgne_status tsgne_batch_reset(tsgne_batch* b);

/*
 * Tile autotuner: times trial_iters iterations of the current membership
 * with each tile (1, 2, 4 warps), keeps the fastest, records it in a
 * process-wide cache keyed by (SM count, log2 of the pair count, log2 of the
 * member count), and resets every member (tsgne_batch_reset).  *chosen gets
 * the tile; ms_per_iter (may be NULL) gets the 3 measured times.
 */
tsgne_status tsgne_batch_autotune(tsgne_batch* b, int32_t trial_iters, int32_t* chosen, float* ms_per_iter);

/* The autotuner over every compiled shape of the batched pass: (tile_warps,
 * i_per_lane) = (1, 16), (2, 16), (4, 16), (1, 8), (2, 8), (4, 8), in that
 * order in ms_per_iter (6 floats, may be NULL); keeps and caches the fastest
 * as tsgne_batch_autotune does and resets every member. */
tsgne_status tsgne_batch_autotune_shapes(tsgne_batch* b, int32_t trial_iters, int32_t* tile_warps,
                                         int32_t* i_per_lane, float* ms_per_iter);

/* Cached tile for the current membership's key, 0 if none was tuned yet. */
tsgne_status tsgne_batch_cached_tile(tsgne_batch* b, int32_t* tile_warps);

/*
 * ------------------------------------------------- ShortestPath embedding
 * The paper's graph embedding for t-SGNE (Sec. 2.3, Eq. 8): for d target
 * nodes (the paper draws them at random; the caller passes them, int32[d] in
 * [0, n), repeats allowed), X[i][t] = shortest-path length from node i to
 * target t when it is <= l0, else l0 + 1 (also when no path exists).  l0 <= 0
 * selects the paper's default floor(sqrt(|E|)), |E| the undirected edges after
 * symmetrisation.  The graph is read like tsgne_build_P reads it (any CSR,
 * symmetrised).  X_out float[n*d] row-major.  1 <= d <= 1024.  All pointers
 * live where ptr_kind says; work runs on cuda_stream (NULL: legacy default)
 * and the call synchronises.  Errors: INVALID_ARG (also a target outside
 * [0, n)), BAD_CSR, OOM.
 */
tsgne_status tsgne_shortest_path_embedding(int32_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                           const int32_t* targets, int32_t d, int32_t l0, float* X_out,
                                           int32_t ptr_kind, void* cuda_stream);

/*
 * The paper's full pipeline GD = DR o GE (Sec. 2, Eq. 1) for the context:
 * ShortestPath embedding of the graph (as tsgne_shortest_path_embedding, X
 * kept on the device) followed by tsgne_build_P on (G, X).
 */
tsgne_status tsgne_build_P_shortest_path(tsgne_ctx* ctx, int32_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                         const int32_t* targets, int32_t d, int32_t l0, int32_t ptr_kind);

/* Largest n accepted by tsgne_repulsion_noalloc. */
#define TSGNE_NOALLOC_MAX_N 65536

/*
 * ---------------------------------------------------------------- serving
 * Continuous-batching server over one batch (the paper has no serving
 * layer).  Requests wait in a FIFO queue; each tsgne_server_tick
 *   1. admits queued requests in order while the estimated device bytes of
 *      the resident layouts (tsgne_server_estimate_bytes) stay within
 *      budget_bytes and below the free device memory -- the first request is
 *      admitted whatever its size when nothing is resident;
 *   2. selects the resident layouts to advance: all (policy 0) or, policy 1,
 *      those with the least remaining iterations x n^2, in that order, until
 *      their pairs per iteration reach fill_pairs;
 *   3. runs tick_iters iterations of the selected layouts (tsgne_batch_run);
 *   4. retires the layouts that reached iters: the layout is copied to
 *      server-owned host memory and the member's device memory freed.
 * A request's layout equals the one it gets alone (members are independent,
 * see tsgne_batch_*).  Cancelling frees a queued or resident request; its
 * result then reports TSGNE_ERR_CANCELLED.  Not thread-safe.
 */
typedef struct tsgne_server tsgne_server;

typedef struct {
  int64_t budget_bytes; /* admission budget of the resident layouts (default 80 GiB) */
  int32_t iters;        /* iterations per request (default 500; a multiple of tick_iters) */
  int32_t tick_iters;   /* iterations per tick (default 10) */
  int32_t max_members;  /* resident layouts at most (default 256) */
  int32_t tile_warps;   /* repulsion tile of the batch: 1, 2 or 4 warps (default 2) */
  int32_t policy;       /* 0: advance every resident layout; 1: shortest remaining work first (default) */
  int32_t aging_ticks;  /* policy 1: a resident layout left out of this many ticks in a row is
                           chosen first, oldest first (default 20; 0: no aging) */
  double fill_pairs;    /* policy 1: pairs per iteration that fill the GPU (default 4e9) */
  int32_t tree_min_n;   /* requests of at least this many points run the tree code with cfg.theta
                           (tsgne_batch_add_ex); 0 (default): every request runs the exact pass */
} tsgne_server_config;

void tsgne_server_config_default(tsgne_server_config* cfg);

/* Device bytes a resident layout of n points and nnz affinities holds in a
 * batch with the given tile (P, layout, optimiser state, initial layout,
 * fixed-point repulsion accumulators, Z partials, an upper bound for the hub-row
 * chunk lists); -1 for invalid arguments.  A tree-code member holds about
 * 144 bytes per point more (its tree); the server adds them.  Host
 * arithmetic only (no GPU needed). */
int64_t tsgne_server_estimate_bytes(int32_t n, int64_t nnz, int32_t tile_warps);

/* cfg (may be NULL: defaults) configures every layout; cuda_stream as for
 * tsgne_batch_create.  Errors: INVALID_ARG (iters not a multiple of
 * tick_iters, policy not 0/1, ...), OOM, CUDA. */
tsgne_status tsgne_server_create(tsgne_server** out, const tsgne_server_config* scfg, const tsgne_config* cfg,
                                 void* cuda_stream);
void tsgne_server_destroy(tsgne_server* s);
const char* tsgne_server_last_error(const tsgne_server* s);

/* Queues a request (host arrays, copied): the graph's CSR (as for
 * tsgne_build_P), X float[n*d], Y0 float[n*2] or NULL (N(0, 1e-4^2) from the
 * seed).  *request_id receives its id (> 0).  Errors: INVALID_ARG, BAD_CSR,
 * OOM (host). */
tsgne_status tsgne_server_submit(tsgne_server* s, int32_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                 const float* X, int32_t d, const float* Y0, int64_t* request_id);

/* One scheduling round (admit, select, run, retire; see above).  Outputs
 * (may be NULL): resident layouts and queued requests after the round, and
 * how many were retired by it.  Synchronises. */
tsgne_status tsgne_server_tick(tsgne_server* s, int32_t* resident, int32_t* queued, int32_t* retired);

/* Pops up to capacity ids of requests retired since the last call, oldest first. */
tsgne_status tsgne_server_finished(tsgne_server* s, int64_t* ids, int32_t capacity, int32_t* count);

/* State of a request: 0 queued, 1 resident, 2 done, 3 cancelled; and its iterations. */
tsgne_status tsgne_server_status(tsgne_server* s, int64_t request_id, int32_t* state, int32_t* iterations);

/* Copies a finished layout into Y_out (host float[n*2]) and forgets the
 * request.  NOT_BUILT if it has not finished; CANCELLED (and forgets it) if
 * it was cancelled; INVALID_ARG for an unknown id. */
tsgne_status tsgne_server_result(tsgne_server* s, int64_t request_id, float* Y_out);

/* Cancels a queued or resident request (its device memory is freed at
 * once).  INVALID_ARG if it is unknown, finished or already cancelled. */
tsgne_status tsgne_server_cancel(tsgne_server* s, int64_t request_id);

/* Estimated device bytes held, resident layouts, queued requests. */
tsgne_status tsgne_server_usage(tsgne_server* s, int64_t* used_bytes, int32_t* resident, int32_t* queued);

/*
 * ---------------------------------------------------------------------------
 * One layout over several GPUs (one context per GPU, same P and layout on
 * every context).  The paper runs on one CPU and describes no distribution;
 * the split follows from the form of Eq. 4: the repulsive forces and Z are
 * sums over the unordered pairs, which the exact pass evaluates in tile
 * pairs ("units", nt (nt + 1) / 2 of them for nt tiles of the layout), so the
 * units can be divided among contexts and the sums added afterwards.  Each
 * context holds the whole (O(n + nnz)) state and updates every row itself;
 * only the O(n^2) repulsion is divided.
 *
 * An iteration on context r of w (rank and world set by tsgne_shard_set):
 *   1. tsgne_shard_repulsion: enqueues units [u0, u1) = [U r / w, U (r+1) / w)
 *      on the context's stream and returns two device buffers that the
 *      caller must sum element-wise over the w contexts, in place, after
 *      that work (an all-reduce on the same stream, or after synchronising
 *      it): acc, 2 n int64 fixed-point force accumulators (sum as int64:
 *      exact, wrapping), and zunit, U doubles with the unit partials of Z
 *      (units of other contexts hold 0 here, so the sum is exact too);
 *   2. tsgne_shard_step_finish: Z, the schedule, F^r and the attraction /
 *      update of every row.
 * Because both sums are exact, every context then holds the same bits as a
 * single context running tsgne_step (for any w).  tsgne_shard_gradient_finish
 * ends a pass without advancing and exports the gradient (parity hook).
 * Exact repulsion only (cfg.repulsion = 0); TSGNE_ERR_INVALID_ARG otherwise,
 * or when a share is enqueued before the previous one was finished.
 * tsgne_step / tsgne_run / tsgne_kl / tsgne_gradient keep computing every
 * unit locally.
 */
tsgne_status tsgne_shard_set(tsgne_ctx* ctx, int32_t rank, int32_t world);
/* units: U; [*u0, *u1): this context's units; *acc: device int64[*acc_count]
 * (2 n); *zunit: device double[U].  Both buffers belong to the context. */
tsgne_status tsgne_shard_repulsion(tsgne_ctx* ctx, int64_t* units, int32_t* u0, int32_t* u1, void** acc,
                                   int64_t* acc_count, void** zunit);
tsgne_status tsgne_shard_step_finish(tsgne_ctx* ctx);
/* g_out: float[n*2] (host or device per ptr_kind); z_out: may be NULL.  Synchronises. */
tsgne_status tsgne_shard_gradient_finish(tsgne_ctx* ctx, float alpha, float* g_out, double* z_out,
                                         int32_t ptr_kind);
/* The cudaStream_t the context runs on (its private stream if it was created
 * with NULL), for callers that order their own work or collectives on it. */
tsgne_status tsgne_stream(tsgne_ctx* ctx, void** cuda_stream);

/*
 * Repulsion pass that allocates no device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc, e.g. code running inside a framework or plugin host that owns
 * the device-memory budget, or code that must not trigger the device-wide
 * synchronisation an allocation or free can cause.
 *
 * Computes, for the layout Y (device float[n*2], row-major x, y), the
 * unnormalised repulsive sums F^r_i = sum_{j != i} w_ij^2 (y_i - y_j) into
 * frep_out (device float[n*2]) and Z = sum_{k != l} w_kl into z_out (one
 * device double), with w = (1 + ||y_k - y_l||^2)^-1 -- the same quantities as
 * the repulsion pass of tsgne_step.  Work is enqueued on cuda_stream (NULL =
 * the legacy default stream); nothing is synchronised.  No context is used.
 *
 * Temporaries live in one static device array of about 8.6 MiB that every GPU
 * loading the library holds until the process exits.  2 <= n <=
 * TSGNE_NOALLOC_MAX_N, and Y, frep_out and z_out 8-byte aligned, else
 * TSGNE_ERR_INVALID_ARG before any work; tsgne_last_error(NULL) then says
 * why.  The array's address is cached per device for the life of the
 * process and does not survive cudaDeviceReset.  The first
 * call on a device looks up that array's address with the device current:
 * make it before any stream capture.  All calls share the array (each call
 * clears what must start at zero and overwrites what it reads), so calls
 * that overlap on the GPU race; serialise them on one stream.
 */
tsgne_status tsgne_repulsion_noalloc(int32_t n, const float* Y, float* frep_out, double* z_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* TSGNE_H */
