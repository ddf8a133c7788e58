/*
 * slim_gb300.h — C ABI of the GB300 scan-integration library for SLIM-VDB
 * style probabilistic semantic TSDF maps (arXiv 2512.12945).
 *
 * The library keeps one sparse voxel map per slim_map handle on one CUDA
 * device: 8^3-voxel blocks behind an open-addressing hash, each voxel holding
 * a truncated signed distance D, a weight W and its semantic state — Dirichlet
 * class counts (closed set, Sec. III-C) or the Normal-Inverse-Gamma mean m
 * and diagonal beta of an l-dimensional embedding (open set, Sec. III-D).
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are memory the GPU can address, owned by the
 *     caller: device memory, or pinned (page-locked) host memory, which the
 *     kernels then read in place over the host link. The library never frees
 *     them and never keeps them after the call returns (work it queued on
 *     `stream` may still read them until the stream reaches that point).
 *     Pointers named *_host are ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Work is queued asynchronously on it unless stated otherwise.
 *   - Arguments are checked on the host before anything is queued; a bad
 *     argument returns SLIM_ERR_ARG and queues nothing.
 *   - Faults found on the device (capacity exhausted, a bounded probe or wait
 *     that ran out) set a sticky status word in the map. The scan during
 *     which the fault happens may be partly applied; every later scan sees
 *     the status and leaves the voxel fields untouched. The status is
 *     returned by slim_map_sync and by the calls that synchronise (stats,
 *     extract, query); slim_map_reset clears it.
 *   - No exception or longjmp crosses this boundary. A map handle must not be
 *     used from two host threads at once.
 *   - slim_last_error() gives a human-readable message for the last failure
 *     on the calling thread.
 */
#ifndef SLIM_GB300_H
#define SLIM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SLIM_OK = 0,
  SLIM_ERR_ARG = 1,         /* invalid argument (nothing queued) */
  SLIM_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  SLIM_ERR_CAPACITY = 3,    /* block, voxel, hash or scratch capacity exhausted */
  SLIM_ERR_TIMEOUT = 4,     /* a bounded device-side probe or wait ran out */
  SLIM_ERR_NOMEM = 5,       /* device allocation failed at map creation */
  SLIM_ERR_UNSUPPORTED = 6, /* valid request this map's mode cannot serve */
  SLIM_ERR_INTERNAL = 7,    /* an internal device-side consistency check failed */
  SLIM_ERR_RANGE = 8        /* an input value outside its stated range (open set: an
                               embedding element beyond embed_bound); the
                               observations that carried it were not fused */
} slim_status;

/* Semantic fusion mode. */
typedef enum {
  /* Theorem 1 / Eq. (alpha_update): each observation adds 1 to the count of
   * its most probable class (argmax of the per-point probabilities, ties to
   * the lowest index). */
  SLIM_CLOSED_ONEHOT = 0,
  /* Soft-count reading of Eq. (alpha_update): each observation adds its whole
   * probability vector (the mode the adjoint differentiates). */
  SLIM_CLOSED_SOFT = 1,
  /* Theorem 2 / Eqs. (norm_update_1)-(norm_update_4) with lambda = 2 nu = W
   * (Sec. III-D): per-element NIG mean m and beta of l-dim embeddings. */
  SLIM_OPEN = 2,
  /* The non-Bayesian ablation of the evaluation (SLIM-VDB*, Sec. IV): the
   * voxel keeps the label (argmax) of its most recent observation — last in
   * scan, then point-index order; D and W as in the other modes. Direct
   * reductions only; extract writes the label as a one-hot row; no
   * uncertainty read-out, no adjoint. */
  SLIM_CLOSED_LATEST = 3
} slim_mode;

typedef enum { SLIM_STORE_F32 = 0, SLIM_STORE_BF16 = 1 } slim_storage;

/* How closed-set (voxel, point) pairs reach the records (all give the same
 * result up to FP32 summation order; Theorem 1 makes the grouping free):
 *   SLIM_AGG_SORT    a CTA tile of pairs is radix-sorted by voxel key, then a
 *                    warp segmented reduction sends one update per voxel;
 *   SLIM_AGG_HASH    one-hot only: a CTA tile adds each pair at once into a
 *                    shared-memory table keyed by (voxel, class), then sends
 *                    one vector red.add per table entry;
 *   SLIM_AGG_DIRECT  closed set: no grouping on chip, reductions per pair
 *                    resolved in L2 (one thread per point; soft counts send
 *                    2 + K 64-bit fixed-point reductions per pair);
 *   SLIM_AGG_AUTO    one-hot: direct, or hash when tile_points is set;
 *                    slim_autotune picks between direct and the hash tiles;
 *                    soft counts: sort (each voxel's pairs of a tile summed
 *                    on chip before its 2 + K 64-bit fixed-point reductions;
 *                    direct sends them per pair). */
typedef enum {
  SLIM_AGG_AUTO = 0,
  SLIM_AGG_SORT = 1,
  SLIM_AGG_HASH = 2,
  SLIM_AGG_DIRECT = 3
} slim_aggregation;

/* Per-observation weight w~ of the TSDF update (Sec. III-A: W_t = W_{t-1} +
 * w~, D_t = (W_{t-1} D_{t-1} + w~ d) / W_t; the paper uses w~ = 1):
 *   SLIM_WEIGHT_CONSTANT  w~ = 1 (default);
 *   SLIM_WEIGHT_LINEAR    the linear decay behind the surface of Bylow et
 *                         al. (RSS 2013): w~ = 1 for d >= -weight_eps,
 *                         (tau + d) / (tau - weight_eps) below, 0 at d = -tau
 *                         (d > 0 in front of the surface). The class counts
 *                         take the same weight (one-hot: c_z += w~; soft:
 *                         c += w~ p), so sum c = W still holds; an
 *                         observation of weight 0 changes nothing.
 * The linear weighting serves the closed-set modes with direct reductions
 * (aggregation AUTO or DIRECT); it has no adjoint (slim_backward returns
 * SLIM_ERR_UNSUPPORTED). */
typedef enum { SLIM_WEIGHT_CONSTANT = 0, SLIM_WEIGHT_LINEAR = 1 } slim_weighting;

typedef struct {
  float voxel_size;      /* metres, > 0 */
  float trunc;           /* truncation tau in metres, 0 < tau <= 4 voxel_size */
  float min_range;       /* valid sensor-frame range [min_range, max_range] */
  float max_range;
  int32_t mode;          /* slim_mode */
  int32_t num_classes;   /* K for the closed-set modes (1..64) */
  int32_t embed_dim;     /* l for SLIM_OPEN (multiple of 64, 64..1024) */
  int32_t embed_storage; /* slim_storage of m and beta (SLIM_OPEN) */
  double alpha0;         /* Dirichlet prior per class, >= 0 (read-out only) */
  double body_from_sensor[16]; /* row-major 4x4 extrinsic, FP64 */
  int64_t block_capacity;  /* maximum allocated 8^3 blocks, < 2^23 */
  int64_t hash_capacity;   /* hash entries (rounded up to 32 x power of 2) */
  int64_t voxel_capacity;  /* SLIM_OPEN: maximum allocated voxels */
  int64_t max_points;      /* largest scan passed to slim_integrate */
  int32_t aggregation;     /* slim_aggregation: how pairs reach the records */
  int32_t tile_points;     /* hash aggregation: points per CTA tile, 64, 128 or
                              256 (0 = 256); SLIM_OPEN with image_width > 0:
                              tile width in pixels, 8, 16 or 32 (0 = 16; tiles
                              hold 256 pixels); see slim_autotune */
  int32_t weighting;       /* slim_weighting (default SLIM_WEIGHT_CONSTANT) */
  float weight_eps;        /* SLIM_WEIGHT_LINEAR: metres, 0 <= eps < trunc */
  int32_t image_width;     /* SLIM_OPEN: the points of a scan are the pixels of a
                              row-major image of this many columns (an RGB-D
                              frame back-projected), so integration groups them
                              in 16 x 16 pixel tiles; 0 (default): unorganized,
                              tiles of 256 consecutive points. Results do not
                              depend on it. 0 .. 65536 */
  float embed_bound;       /* SLIM_OPEN: bound B on the magnitude of every
                              embedding element, |z_e| <= B (default 1: unit-norm
                              embeddings, as the paper's normalised features).
                              The per-call sums of each voxel's observations
                              about its stored mean are accumulated exactly, as
                              64-bit integers in units of B 2^-32 (first moments)
                              and B^2 2^-31 (second moments); an embedding beyond
                              B raises SLIM_ERR_RANGE. 2^-16 .. 2^16 */
} slim_map_params;

typedef struct slim_map slim_map;

typedef struct {
  int64_t blocks;        /* allocated blocks */
  int64_t voxels;        /* SLIM_OPEN: allocated voxel rows; closed: -1 */
  int64_t device_bytes;  /* device memory held by the map */
  int64_t scans;         /* scans integrated since creation / reset */
  uint32_t status;       /* sticky device status (slim_status value) */
} slim_stats;

/* Fill *p with defaults: 0.1 m voxels, tau = 0.3 m, closed one-hot with
 * K = 20, alpha0 = 1, identity extrinsic, capacities for ~1e5 blocks. */
slim_status slim_map_params_default(slim_map_params* p);

/* Create a map on the current CUDA device. The map allocates and owns its
 * hash, block pool, voxel storage and scratch (cudaMalloc, synchronous).
 * *out receives the handle. */
slim_status slim_map_create(const slim_map_params* p, slim_map** out);

/* Release everything the map owns (synchronises the device first). */
slim_status slim_map_destroy(slim_map* m);

/* Empty the map (all blocks and voxels gone, status cleared), keeping its
 * memory. Queued on `stream`. For closed-set maps it also re-zeroes the
 * records the integrations since the last reset wrote (one kernel,
 * SLIM_KERNEL_RESET):
 * the record pool is kept zero outside the 2 x 2 x 2 sub-blocks written since
 * the last reset (every block marks them), so integration never zeroes a
 * block it creates. */
slim_status slim_map_reset(slim_map* m, void* stream);

/* Integrate one scan (Sec. III-A to III-D). For each of the n points:
 *   p = pts_dev[3j .. 3j+2], the sensor-frame point (float32, AoS xyz);
 *   valid iff finite, min_range <= |p| <= max_range and within 2^19 voxels
 *   of the world origin; world point x = R p + t with
 *   [R t] = pose_host (row-major 4x4 world_from_body, FP64) composed with
 *   body_from_sensor in FP64 on the host, then rounded once to float32.
 *   The ray from o = t through x is marched over the band
 *   t in [max(0, r - tau), r + tau] (Amanatides & Woo); each voxel entered
 *   with along-ray SDF d = (x - c) . u >= -tau receives one observation
 *   min(d, tau) and the point's semantics:
 *     closed modes: sem_dev = n x K float32 class probabilities (row-major);
 *     SLIM_OPEN:    sem_dev = n x l float32 embeddings (row-major, 16-byte
 *                   aligned), every element within embed_bound in
 *                   magnitude (otherwise the observations that carry it
 *                   are not fused and the map's status becomes
 *                   SLIM_ERR_RANGE).
 * Fusion: W += 1, D running average (w~ = 1), then the mode's update.
 * n may be 0. n <= max_points; SLIM_OPEN: n <= 2^23 (SLIM_ERR_ARG beyond).
 * Asynchronous on `stream`. */
slim_status slim_integrate(slim_map* m, const float* pts_dev, int64_t n,
                           const double pose_host[16], const void* sem_dev,
                           void* stream);

/* RGB-D front end (no counterpart in the paper's code, which back-projects
 * depth frames on the CPU): integrate one row-major width x height z-depth
 * image (float32 metres along the optical axis, device memory) without
 * materialising points. Pixel (u, v) is the sensor-frame point
 * (((u + 0.5) - cx) / fx * z, ((v + 0.5) - cy) / fy * z, z), computed in
 * this FP32 op order inside the traversal kernels; non-finite or
 * non-positive depths are invalid; then everything is as in slim_integrate
 * (sem_dev: one row per pixel, width * height <= max_points). One-hot and
 * latest-label maps use the direct kernel, soft counts the sort tiles, the
 * open set its usual pipeline. Asynchronous on `stream`. */
slim_status slim_integrate_depth(slim_map* m, const float* depth_dev, int32_t width,
                                 int32_t height, float fx, float fy, float cx, float cy,
                                 const double pose_host[16], const void* sem_dev, void* stream);

/* As slim_integrate with pts_host / sem_host in host memory. The map keeps
 * two device staging buffers and its own copy stream: the call copies the
 * scan into the buffer the call before last used (once the integration that
 * read it has run), makes `stream` wait for the copies and queues the
 * integration there. Consecutive calls therefore overlap the copy of scan
 * k + 1 with the integration of scan k. Pinned host memory makes the copies
 * asynchronous; the host buffers must stay valid until the integration
 * queued on `stream` has run. */
slim_status slim_integrate_host(slim_map* m, const float* pts_host, int64_t n,
                                const double pose_host[16], const void* sem_host,
                                void* stream);

/* Wait for `stream` and return the map's sticky device status. */
slim_status slim_map_sync(slim_map* m, void* stream);

/* Host-side counters (synchronises `stream` to read device counters). */
slim_status slim_map_stats(slim_map* m, slim_stats* out, void* stream);

/* Extract flags. */
#define SLIM_EXTRACT_POSTERIOR 1 /* closed set: sem = Eq. (dir_to_cat)
                                    posterior (alpha0 + c_i)/(K alpha0 + sum c)
                                    instead of the raw counts c */

/* Export every allocated voxel (W > 0), ordered by block coordinates
 * (bx, by, bz) lexicographically, then by the local index
 * ((ix & 7) * 8 + (iy & 7)) * 8 + (iz & 7).
 * Two-call protocol: with cap == 0 only *n_out is written (the call
 * synchronises `stream`). With cap >= *n_out the outputs are written:
 *   ijk_dev   n x 3 int32 voxel indices (may be NULL)
 *   D_dev, W_dev  n float32 (may be NULL)
 *   sem_dev   closed: n x K float32 counts or posteriors; open: n x l float32
 *             NIG means m (may be NULL)
 *   beta_dev  open: n x l float32 NIG beta (may be NULL; ignored if closed)
 *   index_dev n int32 internal voxel index (closed: slot*512 + local; open:
 *             voxel row) as used by slim_backward (may be NULL).
 * The call synchronises `stream`. cap < *n_out returns SLIM_ERR_CAPACITY. */
slim_status slim_extract_tsdf(slim_map* m, int32_t* ijk_dev, float* D_dev, float* W_dev,
                              float* sem_dev, float* beta_dev, int32_t* index_dev,
                              int64_t cap, int64_t* n_out, int32_t flags, void* stream);

/* Ray-cast render of the map from a pinhole camera (Sec. III-E; the paper
 * renders its VDB grid from a camera viewpoint with NanoVDB). Camera: x
 * right, y down, looking along +z; pixel (px, py) looks along
 * ((px + 0.5 - cx) / fx, (py + 0.5 - cy) / fy, 1), normalised, rotated by
 * world_from_camera (row-major 4x4 FP64, rounded to FP32 like scan poses).
 * Pixels are row-major, width x height (1..16384 each). Along each ray the
 * voxels entered for t in [near_t, far_t] (0 <= near_t < far_t) are visited
 * by the integration DDA; the surface is the first pair of consecutive
 * visited voxels with positive weight and D_prev > 0 >= D, its depth the ray
 * distance interpolated linearly between the two voxel-centre projections.
 * Outputs (caller-owned device memory; all but depth_dev may be NULL):
 *   depth_dev  float32 per pixel, +inf where no surface was found;
 *   ijk_dev    int32 x 3 per pixel, the voxel after the crossing
 *              (INT32_MIN where none);
 *   label_dev  int32 per pixel: closed set, the largest count at that voxel
 *              (ties to the lowest class); open set and misses, -1;
 *   sim_dev    float32 per pixel: open set with q_dev (l float32, device):
 *              cosine of the voxel's NIG mean with q; else 0.
 * Asynchronous on `stream`. */
slim_status slim_render(slim_map* m, const double world_from_camera[16], float fx, float fy,
                        float cx, float cy, int32_t width, int32_t height, float near_t,
                        float far_t, const float* q_dev, float* depth_dev, int32_t* ijk_dev,
                        int32_t* label_dev, float* sim_dev, void* stream);

/* Uncertainty read-out of the fused semantics, one row per allocated voxel
 * in the order of slim_extract_tsdf, same two-call protocol (cap == 0 writes
 * only *n_out). No counterpart in the paper's code; the quantities are the
 * ones its Bayesian model defines:
 *   closed set (Sec. III-C; Dirichlet posterior Dir(a), a_i = alpha0 + c_i,
 *     A = sum a_i): unc_dev is n x (K + 1) float32: the variance of each
 *     class probability, a_i (A - a_i) / (A^2 (A + 1)), then the entropy
 *     -sum p_i ln p_i of the posterior predictive p_i = a_i / A
 *     (Eq. dir_to_cat);
 *   open set (Eq. student_t, with lambda = 2 nu = W): unc_dev is n x l
 *     float32: the variance of the Student-t predictive of each element,
 *     2 beta (W + 1) / (W (W - 2)), +inf where W <= 2 (the variance does
 *     not exist for 2 nu <= 2).
 * unc_dev is caller-owned device memory. The call synchronises `stream`.
 * cap < *n_out returns SLIM_ERR_CAPACITY. */
slim_status slim_extract_uncertainty(slim_map* m, float* unc_dev, int64_t cap, int64_t* n_out,
                                     void* stream);

/* Open-set read-out (end of Sec. III-D; Fig. "sit"): for every voxel row v
 * (0 .. voxels-1), cosine similarity s_vq = m_v . q_q / (|m_v| |q_q|) against
 * q queries (q_dev: q x l, bf16 bit patterns, row-major), softmax over the
 * queries of s / temperature, label_dev[v] = most probable query (ties to
 * the lowest index) if its probability >= tp, else -1; prob_dev[v] = that
 * probability. Rows with |m| = 0 get label -1, prob 0. scores_dev (voxels x q
 * float32 cosine similarities) may be NULL. The contraction runs on the
 * tcgen05 tensor cores in BF16 with FP32 accumulation. 1 <= q <= 256. */
slim_status slim_query(slim_map* m, const uint16_t* q_dev, int32_t q, float temperature,
                       float tp, int32_t* label_dev, float* prob_dev, float* scores_dev,
                       void* stream);

/* The open-set read-out of slim_query over rows the caller holds, for
 * callers that cannot allocate device memory (plug-ins whose host
 * application owns every device allocation, real-time loops whose memory
 * budget is fixed up front, hosts that only pass buffers they own). The
 * paper has no counterpart; this is an interface convenience.
 *   rows_dev  n_rows x l bf16 bit patterns (voxel means, row-major, 16-byte
 *             aligned); q_dev q x l bf16 queries (16-byte aligned);
 *   label_dev, prob_dev  n_rows outputs as in slim_query.
 * It calls no cudaMalloc / cudaFree and no allocating library routine: its
 * working memory (the inverse norms of up to 256 queries and a few status
 * words, about 1 KB) is one static array in device memory, present on every
 * GPU that loads the library until the process exits; the row norms are
 * computed inside the query kernel from the tiles it already loads. At most
 * 2^20 rows and 256 queries per call; larger requests return SLIM_ERR_ARG.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current) and opts the query kernel
 * into its shared memory; make that first call before any stream capture.
 * Every call shares the array and leaves its contents behind (the status
 * words are cleared at the start of each call); calls whose work overlaps on
 * the GPU (other streams, other threads) race on it, so serialise them.
 * The call queues its work on `stream`, then waits for it and returns
 * SLIM_ERR_TIMEOUT if a bounded wait inside the query kernel ran out (the
 * outputs are then incomplete). */
slim_status slim_query_rows_static(const uint16_t* rows_dev, int64_t n_rows, int32_t l,
                                   const uint16_t* q_dev, int32_t q, float temperature, float tp,
                                   int32_t* label_dev, float* prob_dev, void* stream);

/* Reverse mode of a map integrated from empty (zero priors, so the state is
 * the batch posterior of all observations, Theorems 1-2). Given loss
 * gradients per voxel (indexed like index_dev of slim_extract_tsdf, arrays
 * sized to cover the largest index + 1):
 *   gD_dev  dL/dD          (float32)
 *   gS_dev  closed SOFT: dL/dc (x K); open: dL/dm (x l)       (float32)
 *   gB_dev  open: dL/dbeta (x l) or NULL
 * writes, for one scan's n points (the same pts_dev, pose_host and sem_dev
 * that were integrated), gsem_dev = dL/dsem (n x K or n x l) and
 * gxyz_dev = dL/dp (n x 3, sensor frame); invalid points get zeros.
 * The (voxel, point) pairs are recomputed, not stored. */
slim_status slim_backward(slim_map* m, const float* pts_dev, int64_t n,
                          const double pose_host[16], const void* sem_dev,
                          const float* gD_dev, const float* gS_dev, const float* gB_dev,
                          float* gsem_dev, float* gxyz_dev, void* stream);

/* The stored-pair form of the reverse mode (closed set, one-hot and soft
 * counts): no counterpart in the paper, which has no reverse mode; it is the
 * alternative slim_backward avoids, kept to measure what storing the pairs
 * costs. slim_record_pairs writes, for one scan of a map that already holds
 * it (call after the forward integration, before the next reset), the
 * scan's (voxel, point) observations in point order and, within a point, in
 * ray order: offsets_dev (n + 1 uint32, caller-owned device memory)
 * receives the CSR offsets, vox_dev (cap uint32) each pair's voxel index
 * (slot * 512 + local, as index_dev of slim_extract_tsdf), *n_pairs the
 * total. cap = 0 is a size query (offsets_dev is still written); cap below
 * the total returns SLIM_ERR_CAPACITY. The first call allocates a count
 * buffer of max_points entries; the call synchronises `stream`.
 * slim_backward_pairs then gives the results of slim_backward for the same
 * scan (the same terms in the same order) from the stored list instead of
 * recomputing the band walk and the hash lookups. Latest-label maps and
 * weighted maps return SLIM_ERR_UNSUPPORTED. */
slim_status slim_record_pairs(slim_map* m, const float* pts_dev, int64_t n,
                              const double pose_host[16], uint32_t* offsets_dev,
                              uint32_t* vox_dev, int64_t cap, int64_t* n_pairs, void* stream);
slim_status slim_backward_pairs(slim_map* m, const float* pts_dev, int64_t n,
                                const double pose_host[16], const uint32_t* offsets_dev,
                                const uint32_t* vox_dev, const float* gD_dev,
                                const float* gS_dev, float* gsem_dev, float* gxyz_dev,
                                void* stream);

/* One work item of a batched integration: a scan for one map. */
typedef struct {
  slim_map* map;
  const float* pts_dev;
  int64_t n;
  double pose[16];
  const void* sem_dev;
} slim_batch_item;

/* Integrate n_items scans, possibly of different maps and sizes, in few
 * launches: closed-set items of maps with direct reductions share one grid
 * per mode and weighting and per 64 items (one CTA per 256 points of each
 * item); items of hash-tile maps share one persistent launch per 64 items
 * (CTAs take tiles of all items from a device counter); open-set items
 * share one tile grid per embedding storage and 48 items (one CTA per pixel
 * tile of each item) and one update launch per storage and 48 maps;
 * sort-aggregation items are integrated one by one by their own kernels.
 * Items of the same map are fused as one observation set (Theorems 1-2 make
 * the result independent of order and grouping; the latest-label mode keeps
 * scan order through its stamp). All maps must live on the current device.
 * Nothing is allocated or read back, so the call is capturable in a CUDA
 * graph when every map was created before capture. */
slim_status slim_integrate_batch(const slim_batch_item* items, int32_t n_items,
                                 void* stream);

/* Strategy autotuner (no counterpart in the paper). Times candidates on the
 * caller's scan (same arguments as slim_integrate) with CUDA events on
 * `stream`, keeps the fastest for this map and writes it to *best_tile (may
 * be NULL). The map is reset (emptied) before each trial and at the end.
 * Synchronous.
 *   closed-set one-hot maps (aggregation AUTO, HASH or DIRECT): 8 copies of
 *     the scan per launch with direct reductions (AUTO, DIRECT) and hash
 *     tiles of 64, 128 and 256 points (AUTO, HASH); *best_tile = 0 for
 *     direct, else the tile's points;
 *   open-set maps of organized frames (image_width > 0): tiles of 8 x 32,
 *     16 x 16 and 32 x 8 pixels; *best_tile = the tile width in pixels
 *     (unorganized open-set maps have one tiling: *best_tile = 0).
 * Soft-count, latest-label and sort-aggregation maps return
 * SLIM_ERR_UNSUPPORTED. */
slim_status slim_autotune(slim_map* m, const float* pts_dev, int64_t n,
                          const double pose_host[16], const void* sem_dev, void* stream,
                          int32_t* best_tile);

/* Kernel kinds reported by slim_profile_read. */
typedef enum {
  SLIM_KERNEL_TRAVERSE = 0,     /* band DDA + block allocation */
  SLIM_KERNEL_FUSE_CLOSED = 1,  /* closed-set tile sort + segmented reduce */
  SLIM_KERNEL_OPEN_TILE = 2,    /* open-set band DDA + on-chip aggregation per tile */
  SLIM_KERNEL_OPEN_APPLY = 3,   /* open-set NIG update of the touched voxels */
  SLIM_KERNEL_QUERY = 4,        /* tensor-core query GEMM + epilogue */
  SLIM_KERNEL_BACKWARD = 5,     /* adjoint gather */
  SLIM_KERNEL_BATCH = 6,        /* batched persistent integration */
  SLIM_KERNEL_RESET = 7,        /* slim_map_reset: re-zeroing of used closed-set blocks */
  SLIM_KERNEL_RENDER = 8,       /* slim_render ray casting */
  SLIM_KERNEL_KINDS = 16
} slim_kernel;

/* Measurement aid (no counterpart in the paper). With on != 0 every kernel
 * the map launches is bracketed by two CUDA events recorded on its launch
 * stream. slim_profile_read waits for those events and writes, per kernel
 * kind, the number of launches and their summed device time in ms since the
 * last read; it then clears the record. launches and ms each hold
 * SLIM_KERNEL_KINDS entries (caller-owned host arrays). */
slim_status slim_profile_enable(slim_map* m, int32_t on);
slim_status slim_profile_read(slim_map* m, int64_t* launches, double* ms);

/* Message for the last failure on this thread (never NULL). */
const char* slim_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SLIM_GB300_H */
