/*
 * gempe.h -- C ABI of the GB300 GEMPE epoch engine.
 *
 * GEMPE (Graph Embedding by Minimizing the Predictive Entropy; Boehm & Plant,
 * "Massively Parallel Graph Drawing and Representation Learning", IEEE
 * BigData 2020, arXiv 2011.03479) places the n vertices of an undirected,
 * unweighted graph G = (V, E) at points x_i in R^d (Sec. II.A) so that the
 * predictive entropy PE of Eq. 2 is small.  One epoch (Fig. 4) fits, for
 * every edge and for randomly sampled non-edges, a parabola w (delta - d)^2
 * to the description length (Eq. 4, Eq. 5), accumulates the weighted-
 * majorization numerator y_i and denominator z_i (Eq. 3) per vertex, moves
 * every vertex to x_i = y_i / z_i and refits the sigmoid slope sigma on
 * distance histograms (Sec. III.F).
 *
 * Conventions shared by every call:
 *  - Every function returns a gempe_status and never throws or aborts.  On
 *    failure gempe_last_error() holds a message for the calling thread.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory of the current device.  The caller owns every array it
 *    passes; inputs are copied before the call returns unless stated.
 *  - Positions are FP32, row-major [n][d].  Graphs are int32 CSR matrices
 *    (row_ptr[n+1], col_idx[nnz]) that must be symmetric, with strictly
 *    increasing column indices per row and no self loops; nnz counts each
 *    undirected edge twice.
 *  - A context owns all device memory it allocates.  Work is ordered on the
 *    context's CUDA stream; calls that return data to the host synchronise
 *    that stream.  Device-side failures (non-finite positions) are recorded
 *    in a device status word and reported by the next synchronising call.
 *  - A context may be used from one host thread at a time.
 */
#ifndef GEMPE_H
#define GEMPE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gempe_status {
    GEMPE_OK = 0,
    GEMPE_E_INVALID_ARG = -1,    /* a null pointer, a size out of range, a wrong count */
    GEMPE_E_INVALID_GRAPH = -2,  /* CSR not symmetric / unsorted / self loop / duplicate / range */
    GEMPE_E_OOM = -3,            /* device allocation failed */
    GEMPE_E_CUDA = -4,           /* a CUDA runtime call failed (message has the CUDA error) */
    GEMPE_E_TIMEOUT = -5,        /* a bounded device wait gave up */
    GEMPE_E_NUMERIC = -6,        /* a position became non-finite; the vertex kept its old value */
    GEMPE_E_BUDGET = -7          /* request exceeds a memory budget */
} gempe_status;

/* Parameters of the method.  gempe_default_params() fills the paper's values. */
typedef struct gempe_params {
    float mu;               /* sigmoid position, fixed at 1.5 (Sec. III.F) */
    float sigma0;           /* initial slope, 1.0 (Fig. 4) */
    int32_t sigma_every;    /* refit sigma after every sigma_every-th epoch (Sec. III.F); 0 = fixed */
    int32_t neg_per_vertex; /* k: non-edges sampled per vertex per epoch (Sec. III.C), 0..32 */
    int32_t max_retries;    /* draws per sample before it is dropped (Fig. 2 retries without bound) */
    int32_t symmetric_neg;  /* 1: the sampled partner g also receives the pair's term (Fig. 4) */
    int32_t w_formula;      /* 0: w from second-derivative matching (Sec. II.C text);
                               1: Eq. 4 as printed (first term doubled) */
    int32_t clamp_neg_d;    /* 1: d := max(d, 0) */
    float z_min;            /* x_i is kept when z_i < z_min (1e-30) */
    float init_range;       /* initial x uniform in [-init_range, init_range) (Fig. 4) */
    uint64_t seed;          /* Philox4x32-10 key */
    int32_t hist_bins;      /* B distance-histogram bins on [0, hist_max) (Sec. III.F), 16..4096 */
    float hist_max;         /* 12.0 */
    int32_t precision;      /* 0: FP32 positions; 1: BF16 shadow positions feed the pair arithmetic
                               (FP32 master positions and sums), d >= 8 */
    int32_t block_partners; /* 0: k sampled non-edges per vertex; 64: block sampling -- every tile of
                               tile_vertices consecutive vertices shares 64 partners per epoch,
                               pairs with the vertex itself or a neighbour are masked; d >= 8.  With
                               precision 1 and d in {16, 32, 64} the tiles run on tensor cores */
    int32_t tile_vertices;  /* 128 (the only tile size) */
    int32_t sampling;       /* 0: neg_per_vertex samples per vertex; 1: Sec. III.C's policy, one sample
                               per CSR slot (every edge endpoint draws one non-edge partner, so
                               vertex i has deg(i) samples); not with block sampling.  The loss
                               estimator (gempe_loss) draws neg_per_vertex samples per vertex
                               either way */
    int32_t sigma_source;   /* 0: the slope fit bins the distances the sweep computes anyway (the
                               epoch's start positions, Sec. III.F's first way); 1: a separate pass
                               after the update bins all edges and neg_per_vertex fresh samples per
                               vertex at the new positions (Sec. III.F's second way) */
    int32_t autotune;       /* 1: time the sweep's launch shapes (units, lanes per pair, CTAs per
                               SM) on the graph at create and keep the fastest; 0: fixed defaults.
                               Only the launch shape changes, never the arithmetic of a pair */
    int32_t membership;     /* how the sampler tells edges from non-edges (Sec. III.C, Fig. 2):
                               0: the exact edge set; 1: the paper's byte map -- s = 2^bytemap_log2
                               bytes, edge (i, j) marks ((pi(i) n + pi(j)) * 1103515245) & (s - 1)
                               (32-bit wrap), a draw whose address is marked is redrawn, so
                               non-edges that collide with an edge are lost (counted in
                               gempe_stats_t.false_pos); not with block sampling.  The loss
                               estimator always uses the exact set */
    int32_t bytemap_log2;   /* log2 s, 6..32; 0: nnz rounded up to a power of two times 128,
                               clamped to [2^12, 2^30] */
    int32_t rename_every;   /* the random renaming pi(v) = (alpha v + beta) mod n (alpha coprime
                               to n, drawn from counter (period, 0, 0, 0x09000000)) is redrawn and
                               the map rebuilt every rename_every epochs (period = sample epoch /
                               rename_every); 0: one renaming for the whole run */
    int32_t rng;            /* random numbers of the sampled non-edges (k per vertex or per slot):
                               0: Philox4x32-10, attempt a of a slot from its own counter;
                               1: Sec. III.C's LCG (state := state * 1103515245 + 1 mod 2^32), one
                               state per sample slot seeded from Philox, advanced before every draw,
                               the vertex by Fig. 2's FP32 float trick (mantissa bits in [1, 2),
                               times n minus n, rounded to nearest; n wraps to vertex 0); not with
                               block sampling.  The loss estimator and the separate histogram pass
                               keep Philox */
    /* Optional device allocator (e.g. a framework's caching allocator).  When
     * dev_alloc is null the engine uses cudaMalloc / cudaFree. */
    void* (*dev_alloc)(size_t bytes, void* user);
    void (*dev_free)(void* ptr, void* user);
    void* alloc_user;
} gempe_params;

typedef struct gempe_stats_t {
    int32_t epoch;                 /* epochs completed */
    float sigma;                   /* current slope */
    uint64_t accepted;             /* sampled non-edges drawn (cumulative; the sampler runs */
    uint64_t rejected;             /*   one epoch ahead of the sweep): draws that hit an edge */
    uint64_t exhausted;            /*   or the anchor, samples dropped after max_retries, */
    uint64_t draws;                /*   accepted + rejected */
    uint64_t used;                 /* sampled non-edges the sweeps consumed (cumulative) */
    int64_t n_edges;               /* m, undirected */
    int32_t n, d, k;
    int32_t sigma_iters;           /* root-finding steps of the last slope fit */
    uint64_t false_pos;            /* byte-map membership: rejected draws that are not edges */
} gempe_stats_t;

typedef struct gempe_ctx gempe_ctx;

/* Fill *p with the defaults: mu 1.5, sigma0 1, sigma_every 1, k 5, max_retries
 * 32, symmetric 1, derived w, clamp 1, z_min 1e-30, init_range 1, seed
 * 0x6E6D7065, 1024 bins on [0, 12), FP32, per-vertex sampling (tile size
 * 128 for block sampling), no autotuning, the exact membership test, no
 * custom allocator. */
void gempe_default_params(gempe_params* p);

/* Check that a host CSR array describes the undirected simple graph of
 * Sec. II.A, on the host alone: row_ptr[0] = 0 and
 * non-decreasing, column indices in range, no self loops, rows strictly
 * increasing (no duplicates), and symmetric (every (i, j) has its (j, i)).
 * GEMPE_OK or GEMPE_E_INVALID_GRAPH with the lowest offending row in
 * gempe_last_error().  Needs no GPU. */
gempe_status gempe_validate_csr(const int32_t* row_ptr, const int32_t* col_idx, int32_t n);

/* Create an embedding context from a host CSR graph (Sec. II.A: G, n, d).
 * row_ptr: host int32[n+1]; col_idx: host int32[row_ptr[n]].  d must be one
 * of 1,2,3,4,8,16,32,64,128,256.  cuda_stream: a cudaStream_t for all work of
 * the context, or NULL for a stream the context creates.  Validates the
 * graph (GEMPE_E_INVALID_GRAPH: the row checks of gempe_validate_csr on the
 * host before any device work, the symmetry on the device against the edge
 * set), uploads it, builds the exact edge hash set, draws the initial
 * positions (Fig. 4: uniform random) and sets sigma = sigma0, epoch = 0.  On
 * success *out owns the context; on failure *out is NULL. */
gempe_status gempe_create(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int32_t d,
                          const gempe_params* p, void* cuda_stream, gempe_ctx** out);

/* Same as gempe_create (Sec. II.A) with the CSR arrays in device memory
 * (copied). */
gempe_status gempe_create_device(const int32_t* d_row_ptr, const int32_t* d_col_idx, int32_t n,
                                 int64_t nnz, int32_t d, const gempe_params* p, void* cuda_stream,
                                 gempe_ctx** out);

/* Release the context and all device memory it allocated (waits for its
 * queued work first; the paper has no counterpart).  NULL is ignored. */
void gempe_destroy(gempe_ctx* ctx);

/* Run `iters` full epochs (Fig. 4): sweep + position update + sigma refit.
 * Asynchronous on the context stream (replays a captured CUDA graph). */
gempe_status gempe_step(gempe_ctx* ctx, int32_t iters);

/* The first half of one epoch (the same kernel gempe_step runs): zeroed
 * accumulators receive the Eq. 3 terms of every edge slot and every accepted
 * sampled non-edge (Fig. 2), and the distance histograms are filled
 * (Sec. III.F).  Positions, sigma and the epoch counter are unchanged; the
 * sums stay for gempe_accumulators / gempe_histograms until gempe_update.
 * host_samples: NULL, or host int32[n*k] that receives the accepted partner
 * of each (vertex, sample slot), -1 if dropped (synchronises); with block
 * sampling int32[n*64]: partner p of the vertex's tile, -1 where masked.
 * gempe_step between gempe_sweep and gempe_update is GEMPE_E_INVALID_ARG. */
gempe_status gempe_sweep(gempe_ctx* ctx, int32_t* host_samples);

/* The second half: x_i := y_i / z_i for z_i >= z_min (Fig. 4), accumulators
 * and histograms cleared, sigma refit when due, epoch counter + 1. */
gempe_status gempe_update(gempe_ctx* ctx);

/* Per-kernel timing of the epochs run as gempe_sweep + gempe_update (not
 * gempe_step's graph replays; the paper has no counterpart).  enable = 1:
 * those calls record CUDA events on the context's stream before the pair
 * sweep and after it, before and after the tile kernel of the block form
 * (on its own stream when it runs beside the sweep), after their join and
 * after the position update (the event before the update keeps it from
 * starting while the previous kernel's last blocks run); enable = 0 stops
 * recording.  out_ms3 (may be NULL) receives the windows of the last epoch
 * recorded, in milliseconds: {sweep, tiles (0 without tiles), update}; all 0
 * when no epoch was recorded.  Synchronises on the last event when out_ms3 is set. */
gempe_status gempe_kernel_times(gempe_ctx* ctx, int32_t enable, float* out_ms3);

/* Copy the positions x_i (Sec. II.A, updated by Fig. 4's loop) to host
 * float[n*d] (synchronises).  count must be n*d. */
gempe_status gempe_positions(gempe_ctx* ctx, float* host_out, size_t count);

/* Borrow a device pointer to the FP32 positions [n][d]; valid until the next
 * call that changes them or gempe_destroy. */
gempe_status gempe_positions_device(gempe_ctx* ctx, const float** d_view);

/* Overwrite the positions from host float[n*d] (count must be n*d). */
gempe_status gempe_set_positions(gempe_ctx* ctx, const float* host_x, size_t count);

/* Set / read sigma (the sigmoid slope of Sec. II.B, refitted by Sec. III.F)
 * and the counter of Fig. 4's epoch loop (the epoch keys the sampler). */
gempe_status gempe_set_state(gempe_ctx* ctx, float sigma, int32_t epoch);
gempe_status gempe_get_state(gempe_ctx* ctx, float* sigma, int32_t* epoch);

/* Checkpoint of a context between epochs (not between gempe_sweep and
 * gempe_update), so that a run of Fig. 4 can stop and resume: the FP32
 * positions, sigma, the epoch counter and the sampler statistics, with the
 * graph's n, d and nnz and the parameters that key the draws (seed,
 * neg_per_vertex, max_retries, sampling, block_partners, tile_vertices,
 * membership, rng and, with the byte map, bytemap_log2 and rename_every) and the
 * parameters of the run's arithmetic (mu, hist_max, z_min, hist_bins,
 * sigma_every, sigma_source, precision, symmetric_neg, w_formula,
 * clamp_neg_d).  A context created from the same graph with those parameters
 * and loaded from the checkpoint continues as the saved one would: the same
 * samples, sigma and statistics, positions up to the order of FP32 atomic
 * additions.  The graph itself is checked only by n and nnz; the remaining
 * parameters (autotune, the allocator) do not change the run.
 * Plain little-endian bytes: a 184-byte header, then float[n*d].
 *
 * gempe_save: buf NULL -> *len = the bytes needed, GEMPE_OK.  Otherwise *len
 * must be at least that (else GEMPE_E_INVALID_ARG, *len set to the size
 * needed); writes the checkpoint and sets *len to its size.  Synchronises;
 * reports a pending device failure (GEMPE_E_NUMERIC) like gempe_positions.
 * gempe_load: GEMPE_E_INVALID_ARG when buf is not a checkpoint of this
 * format, is truncated, belongs to another graph size, other sampling
 * parameters or another run's arithmetic (the message says which), or holds a non-finite position or
 * sigma; the context is unchanged then.  On success it redraws the samples
 * of the saved epoch (they depend only on the graph and the epoch) and
 * restores the statistics as saved.  Synchronises. */
gempe_status gempe_save(gempe_ctx* ctx, void* buf, size_t* len);
gempe_status gempe_load(gempe_ctx* ctx, const void* buf, size_t len);

/* Copy the accumulators after gempe_sweep to host float[n*(d+1)]: for each
 * vertex d values of y_i - z_i x_i (the Eq. 3 numerator minus z_i x_i; the
 * update is x_i + that / z_i = y_i / z_i), then z_i.  Synchronises. */
gempe_status gempe_accumulators(gempe_ctx* ctx, float* host_out, size_t count);

/* Copy the distance histograms to host float[2*B]: B edge bins (counts),
 * then B non-edge bins (sums of sample weights, kept on the device in fixed
 * point with 2^-20 resolution) (Sec. III.F).  Synchronises. */
gempe_status gempe_histograms(gempe_ctx* ctx, float* host_out, size_t count);

/* Draw the sampled non-edges of the current epoch without using them:
 * host int32[n*k] partners or -1.  stream_id 0 = the epoch's sampler, 1 =
 * the loss estimator's sampler, 2 = the separate histogram pass's sampler.
 * Synchronises. */
gempe_status gempe_sample(gempe_ctx* ctx, int32_t stream_id, int32_t* host_out, size_t count);

/* Membership test against the device edge hash set (Sec. III.C, exact):
 * host int32 pairs[2*count] (i0,j0,i1,j1,...) -> host uint8 out[count],
 * 1 if (i,j) is an edge.  Pairs out of range give GEMPE_E_INVALID_ARG. */
gempe_status gempe_is_edge(gempe_ctx* ctx, const int32_t* host_pairs, size_t count, uint8_t* host_out);

/* Sampled predictive entropy (Eq. 2) at the current positions and sigma, mu
 * fixed: (sum over edges of dl+ + sum over k loss-stream samples per vertex
 * of (n-1-deg_i)/(2 k_i) dl-) / (n(n-1)/2).  Per-pair dl in FP32, sums in
 * FP64.  Synchronises. */
gempe_status gempe_loss(gempe_ctx* ctx, double* out_pe_bits, float* out_sigma);

/* Exact predictive entropy (Eq. 2) over all n(n-1)/2 pairs at the current
 * positions, mu fixed: with fit_sigma = 0 at the context's sigma; with
 * fit_sigma = 1 at the sigma that minimises it (Eq. 2's min over sigma),
 * found by Newton steps on the exact dPE/dsigma (safeguarded by bisection in
 * ln sigma on [1e-3, 1e3]), returned in *out_sigma (the context's sigma is
 * not changed).  Each evaluation is one pass over all pairs (O(n^2 d)), meant
 * for graphs up to ~10^5 vertices.  Per-pair terms in FP32, sums in FP64.
 * Synchronises. */
gempe_status gempe_loss_exact(gempe_ctx* ctx, int32_t fit_sigma, double* out_pe_bits, float* out_sigma);

/* Slope fit of Sec. III.F on a given histogram (host float[2*B], edge bins
 * then non-edge bins, B = bins in [16, 4096], values at the bin centres of
 * [0, hist_max)) on the GPU: the zero of dPE/dsigma in log sigma on
 * [1e-3, 1e3] that the paper's bisection finds, reached by Newton steps from
 * sigma = 1 with a bracketed search (Newton inside the bracket, else
 * Illinois regula falsi) as the fallback; without a sign change the bracket
 * end with the lower entropy.  cuda_stream may be NULL.  Synchronises.
 * GEMPE_E_INVALID_ARG for null pointers, bins out of range, hist_max <= 0
 * or a non-finite mu. */
gempe_status gempe_fit_sigma(const float* host_hist, int32_t bins, float hist_max, float mu,
                             void* cuda_stream, float* out_sigma);

/* gempe_fit_sigma without device allocation (the paper has no counterpart:
 * this is a convenience of the library).  For callers that must not allocate
 * device memory where they call it -- inside another allocator's callbacks,
 * in serving loops where cudaMalloc/cudaFree would synchronise the device, or
 * in a process whose device memory a framework has already reserved.  The
 * histogram is staged in a 32 KiB static device array (held by every GPU that
 * loads the library until exit), so bins is limited to 4096 per side
 * (GEMPE_E_INVALID_ARG beyond).  Arguments and result are those of
 * gempe_fit_sigma; synchronises cuda_stream.  The first call on a device
 * looks up the array's device address and should come before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race. */
gempe_status gempe_fit_sigma_static(const float* host_hist, int32_t bins, float hist_max, float mu,
                                    void* cuda_stream, float* out_sigma);

/* ------------------------------------------------------------------------
 * One graph over several GPUs: a vertex-range shard per rank (Sec. III.E's
 * parallel reduction of the numerators and denominators of Eq. 3, with the
 * ranks in place of the paper's threads).
 *
 * gempe_create_shard: a context holding the whole graph and every position
 * (the same seed gives every rank the same initial positions) whose epochs
 * evaluate the anchors v_begin <= i < v_end only: their edges (each
 * undirected edge once in the d <= 4 oriented form, at its endpoint of
 * larger degree), their sampled non-edges and, in the block form, their
 * tiles (the range then starts and ends on a tile of 128 vertices, or at n).
 * The sums of all vertices receive this shard's terms.  One epoch over R
 * ranks: gempe_sweep on every rank; the sums (what 0) and the four
 * histogram arrays (1-4) copied out, summed over the ranks and copied back;
 * gempe_update on every rank (its own rows, and the same sigma on every rank,
 * fitted on the summed histograms; the other rows' sums are cleared); the
 * positions (5) copied out, each rank's own rows gathered from every rank,
 * and copied back.  Arguments and errors as gempe_create, plus
 * GEMPE_E_INVALID_ARG for a range outside [0, n) or not on tiles.
 * gempe_stats counts this shard's samples; gempe_loss is this shard's part.
 *
 * gempe_shard_layout: out4 = {floats of the sums (n * stride), stride,
 * histogram bins, floats of the positions (n * d)}.
 * gempe_shard_copy: what 0 the sums (float [n][stride]: d values of
 * y - z x, then z, padded), 1 the edge counts (uint32 [bins]), 2 the sample
 * counts (uint32 [bins]), 3 the samples' anchor-degree sums (uint64 [bins]),
 * 4 the weight corrections (float [bins]), 5 the positions (float [n][d]);
 * direction 0 copies the context's array into device_buf, 1 device_buf
 * into the context (positions: the BF16 shadow is refreshed).  Sums and
 * histograms move between gempe_sweep and gempe_update, positions after
 * gempe_update.  Device-to-device copies ordered on the context's stream. */
gempe_status gempe_create_shard(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int32_t d,
                                int32_t v_begin, int32_t v_end, const gempe_params* p, void* cuda_stream,
                                gempe_ctx** out);
gempe_status gempe_shard_layout(gempe_ctx* ctx, int64_t* out4);
gempe_status gempe_shard_copy(gempe_ctx* ctx, int32_t what, int32_t direction, void* device_buf);

/* Test hook for the bounded device waits of the tensor-core tile kernel
 * (failure detection without a GPU fault; the paper has no counterpart).
 * Launches one CTA set up like a tile CTA (256 TMEM columns allocated, an
 * mbarrier initialised) that waits, with poll_limit polls (1 .. 2^22), for a
 * barrier phase nothing completes -- no MMA is issued -- and then takes the
 * tile kernel's give-up path.  *out_status receives the status it recorded
 * (GEMPE_E_TIMEOUT when the wait ran out), *out_freed 1 once it released its
 * TMEM.  Allocates 8 bytes of device memory; synchronises the device. */
gempe_status gempe_test_tile_wait(int32_t poll_limit, int32_t* out_status, int32_t* out_freed);

/* Counters and state of the context (gempe_stats_t), read from the device
 * after the context's queued work.  Synchronises. */
gempe_status gempe_stats(gempe_ctx* ctx, gempe_stats_t* out);

/* Launch shape of the context's pair sweep (what the autotuner chooses; a
 * GPU launch parameter with no counterpart in the paper):
 * shape5 = {unit pair budget of a packed unit (64 or 128, d <= 4), CSR
 * slots per work unit (8..1024, the per-unit kernel), lanes per pair (d >= 8:
 * d/8 or d/4; 0 = default), sweep CTAs per SM (0 = all that fit), kernel
 * (d <= 4: 0 packed units, 1 one lane per vertex; d >= 8 in the block form
 * with tiles: 0 the tiles after the sweep, 2 the sweep in 512-thread blocks,
 * one per SM, beside one tile CTA per SM on a second stream)}.  Only the launch shape
 * changes, never the arithmetic of a pair; not allowed between gempe_sweep
 * and gempe_update.  gempe_get_shape: the same five, then the sweep grid. */
gempe_status gempe_set_shape(gempe_ctx* ctx, const int32_t* shape5);
gempe_status gempe_get_shape(gempe_ctx* ctx, int32_t* out6);

/* ------------------------------------------------------------------------
 * Batched form: many independent graphs stepped together.
 *
 * The graphs of a batch are grouped by dimension; each group lives in one
 * set of device arrays (a "pack") and every kernel of an epoch runs once per
 * pack over the work units of all its graphs.  One gempe_batch_step epoch
 * is one CUDA-graph launch whose branches (one per pack) run concurrently.
 * Graph g of the batch uses the Philox key seed ^ g and keeps its own sigma,
 * epoch counter and histograms, so it draws the same samples as a context
 * created alone with that seed and reaches the same positions up to FP32
 * summation order.  precision 1 applies to the graphs with d >= 8 (the
 * others stay FP32), and so does block sampling.
 * ------------------------------------------------------------------------ */
typedef struct gempe_graph_desc {
    const int32_t* row_ptr;  /* host int32[n+1] */
    const int32_t* col_idx;  /* host int32[row_ptr[n]] */
    int32_t n;
    int32_t d;               /* one of the dimensions gempe_create accepts */
} gempe_graph_desc;

typedef struct gempe_batch gempe_batch;

/* Validate, upload and initialise n_graphs graphs (copied; the caller keeps
 * ownership of the arrays).  As in gempe_create, the rows are checked on
 * the host before any device work and the symmetry on the device; an error
 * names the graph by its index ("graph g: ...").  cuda_stream as in
 * gempe_create.  With p->autotune each pack's sweep shape is tuned before
 * the first epoch. */
gempe_status gempe_batch_create(int32_t n_graphs, const gempe_graph_desc* graphs, const gempe_params* p,
                                void* cuda_stream, gempe_batch** out);
void gempe_batch_destroy(gempe_batch* b);
/* `iters` epochs (Fig. 4) of every graph, asynchronous on the batch stream. */
gempe_status gempe_batch_step(gempe_batch* b, int32_t iters);
/* Positions of graph `graph` to host float[n*d] (synchronises). */
gempe_status gempe_batch_positions(gempe_batch* b, int32_t graph, float* host_out, size_t count);
/* Sampled predictive entropy (Eq. 2) of graph `graph` (as gempe_loss). */
gempe_status gempe_batch_loss(gempe_batch* b, int32_t graph, double* out_pe_bits, float* out_sigma);
/* Statistics of graph `graph` (as gempe_stats).  Synchronises. */
gempe_status gempe_batch_stats(gempe_batch* b, int32_t graph, gempe_stats_t* out);
/* Launch shape of the pack holding dimension d: out[0] unit pair budget
 * (packed units, d <= 4) or CSR slots per unit (one lane group per vertex),
 * out[1] lanes per pair, out[2] sweep CTAs per SM (0 = all that fit), out[3]
 * sweep grid, out[4] graphs in the pack, out[5] tuned sweep time in ns (0 if
 * not tuned), out[6] the sweep kernel (d <= 4: 0 packed units, 1 one lane per
 * vertex; 0 for d >= 8). */
gempe_status gempe_batch_shape(gempe_batch* b, int32_t d, int64_t* out7);

/* ------------------------------------------------------------------------
 * Serving form: embedding jobs admitted by device-memory budget and run with
 * continuous batching.
 *
 * A server owns max_jobs job slots (CUDA streams) and two host threads.  Jobs
 * are admitted in arrival order as soon as a slot is free and the job's
 * device bytes (gempe_job_bytes) fit in the budget next to the running jobs;
 * a running job keeps its CSR, edge set, positions and accumulators resident
 * on the device and runs its epochs on its slot's stream, so the kernels of
 * all running jobs overlap.  When its epochs are done its positions go to
 * pinned host memory and its device memory returns to the budget.  A job
 * computes what gempe_create + gempe_step(epochs) compute with params.seed =
 * the job's seed (up to the order of FP32 atomic additions).  The server's
 * params apply to every job (precision 1 and block sampling only for d >= 8).
 * ------------------------------------------------------------------------ */
typedef struct gempe_server gempe_server;

typedef struct gempe_job_desc {
    const int32_t* row_ptr;  /* host int32[n+1], copied at submit */
    const int32_t* col_idx;  /* host int32[row_ptr[n]], copied at submit */
    int32_t n;
    int32_t d;
    int32_t epochs;
    uint64_t seed;           /* Philox key of the job */
} gempe_job_desc;

typedef struct gempe_job_info {
    int32_t state;           /* 0 queued, 1 running, 2 done; a negative gempe_status if it failed */
    int32_t epochs, epochs_done;
    uint64_t submit_ns, admit_ns, done_ns;   /* steady clock, ns since the server was created */
    uint64_t device_bytes;   /* device bytes reserved for the job */
    uint64_t pairs;          /* pair-updates of the finished job: epochs * m + sampled non-edges used */
    float sigma;             /* final slope of the finished job */
} gempe_job_info;

/* Device bytes a job of n vertices and nnz CSR slots holds while it runs
 * (0 for invalid arguments).  Pure host arithmetic. */
size_t gempe_job_bytes(int32_t n, int64_t nnz, int32_t d, const gempe_params* p);
/* max_jobs in [1, 256]; p->dev_alloc must be NULL (jobs allocate stream-ordered). */
gempe_status gempe_server_create(size_t hbm_budget_bytes, int32_t max_jobs, const gempe_params* p,
                                 gempe_server** out);
/* Stops the threads; running jobs finish their enqueued work and are dropped. */
void gempe_server_destroy(gempe_server* s);
/* Queue a job (copies the CSR).  GEMPE_E_BUDGET if the job alone exceeds the
 * budget; invalid graphs are reported by poll / wait / result (rows checked
 * on the host before admission, the symmetry on the device when the job
 * starts). */
gempe_status gempe_server_submit(gempe_server* s, const gempe_job_desc* job, uint64_t* job_id);
/* State of a job without waiting.  GEMPE_E_INVALID_ARG for an unknown or
 * already released job id; for a failed job, *info is filled and its
 * gempe_status is returned (message in gempe_last_error). */
gempe_status gempe_server_poll(gempe_server* s, uint64_t job_id, gempe_job_info* info);
/* Block until the job is done or failed, at most timeout_ms (GEMPE_E_TIMEOUT). */
gempe_status gempe_server_wait(gempe_server* s, uint64_t job_id, int32_t timeout_ms, gempe_job_info* info);
/* Positions of a finished job to host float[n*d]; releases the job record. */
gempe_status gempe_server_result(gempe_server* s, uint64_t job_id, float* host_out, size_t count);
/* out6: queued, running, completed, failed, device bytes in use, peak bytes in use. */
gempe_status gempe_server_stats(gempe_server* s, int64_t* out6);

/* Message of the last failure on this thread ("" if none). */
const char* gempe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GEMPE_H */
