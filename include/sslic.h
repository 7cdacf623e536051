/*
 * sslic.h -- C ABI of the GB300 (sm_103a) Scalable SLIC library.
 *
 * Method: Lowekamp, Chen, Yaniv, Bernardini, "Scalable Simple Linear
 * Iterative Clustering (SSLIC) Using a Generic and Parallel Approach",
 * arXiv 1806.08741.  Section references below are to that paper.
 *
 * Conventions
 *  - Image layout: C-contiguous [N_{n-1}]...[N_1][N_0][C], dimension 0
 *    (x) fastest, channels interleaved (Sec. 3.3 keeps a pixel's components
 *    together).  Element type uint8, uint16 or float32.
 *  - Labels: int32, one per voxel, same raster order as the image.
 *  - Centres: float32 table K x (C + n): the C feature components followed
 *    by the n position components x_0..x_{n-1} (Sec. 3.3 stores all
 *    centres in one flat array of C + n values each).
 *  - K = prod_d ceil(N_d / S_d) clusters, seeded on a centred lattice.
 *  - Ownership: the caller owns every image / label / centre buffer and the
 *    stream; a context owns its device workspace (bins, sums, connectivity
 *    scratch), allocated by sslic_create and released by sslic_destroy.
 *  - Every call returns an int status: SSLIC_OK (0) or a negative code; no
 *    exception ever crosses the ABI.  sslic_strerror() names a code and
 *    sslic_last_error() gives detail for the last failure on a context.
 *  - Calls on one context must not overlap (the context's workspace is
 *    shared); calls on different contexts are independent.
 *  - Device-pointer entry points are stream ordered.  They return once the
 *    work is enqueued, except where noted (a positive convergence
 *    threshold and connectivity enforcement each need one host read-back,
 *    and `out` results are filled after a stream synchronisation).
 */
#ifndef SSLIC_H
#define SSLIC_H
#include <stdint.h>

#if defined(__GNUC__)
#define SSLIC_API __attribute__((visibility("default")))
#else
#define SSLIC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define SSLIC_OK 0
#define SSLIC_EINVAL (-1)   /* bad shape, grid, weight, dtype, channel count or pointer */
#define SSLIC_ENOMEM (-2)   /* a device or pinned-host allocation failed */
#define SSLIC_ECUDA (-3)    /* a CUDA launch or runtime call failed */
#define SSLIC_ETIMEOUT (-4) /* a bounded device-side wait expired */
#define SSLIC_EBUSY (-5)    /* the context is in use by another call */
#define SSLIC_EUNSUPPORTED (-6) /* valid request the library does not implement */

typedef enum { SSLIC_U8 = 0, SSLIC_U16 = 1, SSLIC_F32 = 2 } sslic_dtype;

/* The paper's filter parameters (Sec. 3.2): grid size per axis, spatial
 * weight m, iteration cap, monitored residual, connectivity on/off, plus
 * seed perturbation on/off (Sec. 3.1 step 1). */
typedef struct {
    int32_t ndim;           /* n: 1 to 4 (2-D and 3-D integer and 3-channel float images run
                             * the tile kernels; the rest the per-voxel kernel) */
    int64_t size[4];        /* N_d (d = 0 fastest); entries >= ndim ignored; 1 <= N_d <= 2^24 */
    int32_t channels;       /* C: 1 .. 256 */
    int32_t dtype;          /* sslic_dtype */
    int32_t grid[4];        /* S_d >= 1 in voxels, per axis (anisotropic grid, Sec. 3.2/3.3) */
    float   m;              /* spatial weight m > 0 (Sec. 2.1; 10 is the paper's default) */
    int32_t max_iter;       /* iteration cap >= 1 (Sec. 3.2: 10 for 2-D, 5 for n >= 3) */
    double  conv_threshold; /* stop once the centre residual drops below this; <= 0 disables (Sec. 3.1) */
    int32_t perturb;        /* 1: move seeds to the lowest gradient in the 3^n neighbourhood (Sec. 3.1) */
    int32_t enforce_connectivity; /* 1: run the connectivity enforcement of Sec. 3.1 stage 3 */
    int32_t precision;      /* 0: exact FP32 distances.  1: the feature term of float images with
                             * 32..128 channels (2-D / 3-D) from BF16 tensor-core dot products,
                             * with an exact FP32 recheck of every voxel whose candidates the
                             * error bound does not separate, so labels equal those of 0.
                             * SSLIC_EINVAL for C < 32, SSLIC_EUNSUPPORTED for other images.
                             * This form goes beyond the paper (Sec. 2.1 only defines D). */
} sslic_params;

typedef struct {
    int64_t num_clusters;   /* K */
    int64_t num_labels;     /* K + labels created by connectivity enforcement */
    int32_t iterations;     /* assign/update iterations performed */
    double  residual;       /* centre residual of the last iteration */
} sslic_result;

typedef struct sslic_ctx sslic_ctx;

/* Fill *p with the paper's defaults for an n-D image (grid 16, m 10,
 * 10 iterations for n = 2 and 5 for n >= 3, perturbation on, connectivity on). */
SSLIC_API int sslic_default_params(int32_t ndim, sslic_params* p);

/* Validate p and allocate the device workspace on the current CUDA device.
 * Errors: SSLIC_EINVAL, SSLIC_ENOMEM, SSLIC_ECUDA.  *out is NULL on error. */
SSLIC_API int sslic_create(const sslic_params* p, sslic_ctx** out);

/* K for the context's parameters. */
SSLIC_API int sslic_num_clusters(const sslic_ctx* c, int64_t* K);

/* The whole method (Sec. 3.1): seeding (+ perturbation), up to max_iter
 * assign/update iterations, optional connectivity enforcement.
 *   image_dev   device, read only, layout above
 *   labels_dev  device, V int32, written (-1 marks voxels no window reaches,
 *               possible only without connectivity enforcement)
 *   centres_dev device, K x (C+n) float32, written; may be NULL
 *   stream      cudaStream_t, or NULL for the legacy default stream
 *   out         host, may be NULL; filled after a stream synchronisation */
SSLIC_API int sslic_run(sslic_ctx* c, const void* image_dev, int32_t* labels_dev, float* centres_dev,
              void* stream, sslic_result* out);

/* As sslic_run, but starting from caller-given centres instead of seeding
 * (checkpoint / resume: the state after t iterations is the centre table).
 * init_centres_dev: device, K x (C+n) float32, read only. */
SSLIC_API int sslic_run_from(sslic_ctx* c, const void* image_dev, const float* init_centres_dev,
                   int32_t* labels_dev, float* centres_dev, void* stream, sslic_result* out);

/* As sslic_run with HOST buffers: the image is copied to the device, the
 * method runs, labels (and centres if non-NULL) are copied back, and the
 * call returns after the stream is synchronised.  Page-locked buffers give
 * the full copy bandwidth; pageable ones work but copy synchronously.  The
 * context allocates its device image/label buffers on first use.  For 2-D
 * and 3-D images (except float images with 16 or more channels) with a grid
 * of at least 8 along the last axis and at least 128 planes along it, the
 * upload runs on a copy stream of the context in pieces -- first the planes
 * seeding reads, then slabs of 64 planes -- and seeding and each slab's first
 * assignment start as soon as their planes are in; the results are those of
 * the single copy (bit for bit for integer images).  With connectivity
 * enforcement (2-D and 3-D), the final relabel pass runs in slabs of planes and
 * each slab's labels are copied to labels_host as soon as it is relabelled. */
SSLIC_API int sslic_run_host(sslic_ctx* c, const void* image_host, int32_t* labels_host,
                   float* centres_host, void* stream, sslic_result* out);

/* Step entry points (the rows of the method, for parity tests and callers
 * that drive the loop themselves).  All device pointers, stream ordered. */

/* Streamed form, for volumes larger than device memory (the paper's
 * motivating several-GB images, Sec. 1; its 53 GB Lab volume, Sec. 4.1):
 * the image stays in host memory and every iteration streams it through the
 * GPU in slabs of slab_planes planes along its last axis (z in 3-D, y in
 * 2-D), two slab buffers deep, so the upload of one slab overlaps the
 * assignment of the other.  Assignment is voxel-centric and needs only the
 * centres and their bins, which stay on the device, so slabs need no halo
 * (seeding reads two planes on either side); each slab adds its exact sums
 * to the centres' sums, so integer images give the labels and centres of
 * sslic_run bit for bit.  Device memory: the context's centres, sums and
 * bins plus two slabs (image planes + int32 labels).  With connectivity
 * enforcement (Sec. 3.1 stage 3) the labels then pass through the device
 * slab by slab twice more (see sslic_conn_slabs_*): the component records
 * and 16-bit component ids of the whole image stay on the device meanwhile
 * (2 bytes per voxel plus about 45 bytes per component).
 *   image_host   the whole image (layout as sslic_run), host memory;
 *                page-locked memory overlaps best
 *   labels_host  receives the final labels (host, V int32)
 *   centres_host receives the final centres (host, K x (C+n) float, may be NULL)
 *   slab_planes  planes per slab: a positive multiple of 32; with
 *                connectivity also of 64 in 2-D, and at least S along the
 *                last axis
 *   stream       cudaStream_t for the kernels (a copy stream of the context
 *                carries the transfers), or NULL for the legacy default stream
 * 2-D and 3-D images without the precision form (else SSLIC_EUNSUPPORTED);
 * float images with 16 or more channels take the per-voxel kernel here.
 * Synchronous: returns when the labels are in labels_host.  Errors:
 * SSLIC_EINVAL (pointers, slab_planes), SSLIC_ENOMEM, SSLIC_ECUDA,
 * SSLIC_EBUSY. */
SSLIC_API int sslic_run_streamed(sslic_ctx* c, const void* image_host, int32_t* labels_host, float* centres_host,
                                 int64_t slab_planes, void* stream, sslic_result* out);

/* Seeding on the lattice plus optional perturbation (Sec. 2.2 / 3.1 step 1).
 * centres_dev: K x (C+n) float32, written. */
SSLIC_API int sslic_seed(sslic_ctx* c, const void* image_dev, float* centres_dev, void* stream);

/* One iteration: assignment of every voxel to the argmin of D^2 over the
 * centres whose 2S window covers it, ties to the lowest index (Sec. 2.1,
 * 2.2, 3.1 step 2), then the centre update as the mean of [I(x), x] over
 * each label (Sec. 3.1 map-reduce).  centres_in and centres_out are
 * K x (C+n) float32 and may alias; empty clusters keep their centre.
 * residual_host (may be NULL): if non-NULL the call synchronises the stream
 * and stores the centre residual there. */
SSLIC_API int sslic_iterate(sslic_ctx* c, const void* image_dev, const float* centres_in_dev,
                  int32_t* labels_dev, float* centres_out_dev, void* stream,
                  double* residual_host);

/* Connectivity enforcement (Sec. 3.1 stage 3) of a label image produced
 * with the given centres.  labels_in_dev and labels_out_dev may alias.
 * num_labels_host (may be NULL) receives K + the number of new labels.
 * Synchronises the stream once (the component count sizes the scratch).
 * SSLIC_EUNSUPPORTED when more than 2^31 components or labels arise, or
 * when a voxel's coordinates packed in ceil(log2 N_d) bits per axis need
 * more than 63 bits (no image that fits in device memory does). */
SSLIC_API int sslic_connectivity(sslic_ctx* c, const float* centres_dev, const int32_t* labels_in_dev,
                       int32_t* labels_out_dev, void* stream, int64_t* num_labels_host);

/* ---- one image shared by several GPUs (slabs of planes) -------------------
 * The paper's map-reduce update (Sec. 3.1: non-overlapping regions map their
 * pixels into per-label sums, a reduce merges them) across GPUs: each rank
 * holds a slab of planes [lo, hi) along the last axis (z in 3-D, y in 2-D)
 * and a context created with the WHOLE image's parameters.  Assignment is
 * voxel-centric and needs only the centres (replicated), so a slab needs no
 * halo for it.  Per iteration a rank computes its slab's exact integer sums
 * (sslic_shard_map), the caller sums them over the ranks (one all-reduce of
 * K x (C + 4) int64, plus K x C double for float images), and every rank
 * divides identically (sslic_shard_finalize): integer images then get the
 * labels and centres of sslic_run bit for bit.  Slab bounds are multiples
 * of 8 planes (3-D) or 64 rows (2-D), the last ending at N_{n-1}; 2-D and
 * 3-D images, precision 0 (else SSLIC_EUNSUPPORTED).  The library does no
 * communication: the caller's collective library does (NCCL, gloo...). */

/* Seeds of the lattice planes in [lo, hi) (Sec. 3.1 step 1), perturbed by
 * gradients read from planes lo-2 .. hi+1.  image_dev holds planes
 * [a, b) of the image, a = max(0, lo - 2), b = min(N_{n-1}, hi + 2).  Writes
 * the whole K x (C+n) centre table, rows of seeds outside the slab zero, so
 * that a sum over the ranks gives every seed. */
SSLIC_API int sslic_shard_seed(sslic_ctx* c, const void* image_dev, int64_t lo, int64_t hi, float* centres_dev,
                               void* stream);

/* Element counts of one rank's sums: n_u64 uint64 (K x (C + 4): features,
 * three positions, count; sum them as int64) followed, for float images, by
 * n_f64 doubles (K x C feature sums). */
SSLIC_API int sslic_shard_sums_size(const sslic_ctx* c, int64_t* n_u64, int64_t* n_f64);

/* Assignment of the slab's voxels (Sec. 2.2 / 3.1 step 2) from centres_dev
 * (K x (C+n)) and the map of their [I(x), x] into sums_dev (the layout of
 * sslic_shard_sums_size, device memory).  image_dev / labels_dev hold
 * planes [lo, hi) only. */
SSLIC_API int sslic_shard_map(sslic_ctx* c, const void* image_dev, int32_t* labels_dev, int64_t lo, int64_t hi,
                              const float* centres_dev, void* sums_dev, void* stream);

/* The reduce: centres = member means of the summed sums_dev (every rank's
 * sums added), empty clusters keeping centres_prev_dev's rows; writes
 * centres_out_dev (may alias centres_prev_dev) and, if residual_host is
 * non-NULL, the centre residual (synchronises the stream). */
SSLIC_API int sslic_shard_finalize(sslic_ctx* c, const void* sums_dev, const float* centres_prev_dev,
                                   float* centres_out_dev, double* residual_host, void* stream);

/* Connectivity enforcement (Sec. 3.1 stage 3) of an image handed over slab
 * by slab, with the result of sslic_connectivity: begin (with the centres
 * the labels were assigned from), add every slab's labels in order of their
 * planes (slab bounds multiples of 8 planes in 3-D, 64 rows in 2-D; every
 * slab but the last at least S planes deep), finish (the component count:
 * one read-back), then relabel any slab.  The context keeps the component
 * records and the 16-bit component ids of the whole image on the device
 * (2 bytes per voxel plus about 45 bytes per component), and S planes of the
 * previous slab's labels; a slab's buffer is free again when its call
 * returns.  Used by sslic_run_streamed, and by a rank that collects the
 * slabs of an image shared by several GPUs. */
SSLIC_API int sslic_conn_slabs_begin(sslic_ctx* c, const float* centres_dev, void* stream);
SSLIC_API int sslic_conn_slabs_add(sslic_ctx* c, const int32_t* labels_dev, int64_t lo, int64_t hi, void* stream);
SSLIC_API int sslic_conn_slabs_finish(sslic_ctx* c, void* stream, int64_t* num_labels_host);
SSLIC_API int sslic_conn_slabs_relabel(sslic_ctx* c, int32_t* labels_out_dev, int64_t lo, int64_t hi,
                                       void* stream);

/* One assign + update iteration (the same step as sslic_iterate) that
 * allocates nothing.  The paper has no counterpart to this call.  It serves
 * callers that cannot call cudaMalloc: code running under an allocator or
 * memory pool that must not grow, plug-ins whose device memory is budgeted
 * up front, and latency-critical paths that cannot afford an allocation's
 * implicit device synchronisation.  Instead of a context it uses one
 * file-scope device array of about 3 MB, which every GPU that loads this
 * library holds until the process exits.  That array bounds the request:
 * K <= 16384 clusters, C <= 4 channels and at most 65536 assignment tiles
 * counted with the smallest tile (16x8x8 voxels in 3-D, 32x16 pixels in
 * 2-D), i.e. about 67M voxels or 33.5M pixels; larger requests return
 * SSLIC_EINVAL.  It always stages the image with plain loads (a TMA-staged
 * tile shape recorded by sslic_autotune or sslic_tune_record runs its
 * plain twin here).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current, so make
 * it before any stream capture.  All calls share the array and it keeps the
 * previous call's contents: the sums are cleared at the start of each call,
 * and calls whose work overlaps on the GPU (unordered streams) race on it.
 *   p                parameters, validated as for sslic_create
 *   image_dev, centres_in_dev, labels_dev, centres_out_dev: as sslic_iterate
 *   stream           cudaStream_t, or NULL for the legacy default stream */
SSLIC_API int sslic_iterate_static(const sslic_params* p, const void* image_dev, const float* centres_in_dev,
                                   int32_t* labels_dev, float* centres_out_dev, void* stream);

/* Colour input: 8-bit sRGB to CIE-Lab float, on the device.  SLIC clusters
 * colour pixels as [L, a, b, x, y] (Sec. 2, 2.1; its default m = 10 assumes
 * Lab ranges) and the paper converts its 8-bit RGB volume to CIE-Lab float
 * before segmenting (Sec. 4.1).  The colour space is sRGB (IEC 61966-2-1
 * transfer function and matrix) under the D65 white (0.95047, 1, 1.08883),
 * CIE 1976 L*a*b*: the reading whose extremes over the 8-bit cube match the
 * L, a, b ranges of Sec. 2.1.  Single precision; within 1e-3 of the exact
 * value in every component.
 *   rgb_dev  n interleaved (R, G, B) uint8 triples (device, read only)
 *   lab_dev  n interleaved (L, a, b) float32 triples (device, written); it
 *            may not overlap rgb_dev.  The result is an image for the float
 *            path of sslic_run (C = 3, dtype SSLIC_F32).
 *   n        voxels (>= 0; 0 is a no-op)
 *   stream   cudaStream_t, or NULL for the legacy default stream
 * The fast path wants rgb_dev 4-byte and lab_dev 16-byte aligned; other
 * pointers take a per-voxel path (same values).  Returns SSLIC_EINVAL for
 * n < 0, a NULL pointer with n > 0 or overlapping buffers, SSLIC_ECUDA if
 * the launch fails.  Stream ordered; needs no context. */
SSLIC_API int sslic_srgb_to_lab(const void* rgb_dev, void* lab_dev, int64_t n, void* stream);

/* Launch configuration of the assignment kernel.  The paper has no
 * counterpart: its multi-threaded filter splits the image into regions per
 * thread (Sec. 3.1), while here a tile shape fixes how voxels map to CUDA
 * blocks and lanes.  A shape is a tile extent, the voxels each lane handles
 * (2 or 4 consecutive voxels along x) and how a tile reaches shared memory
 * (plain loads, or a TMA copy of the next tile issued while the current one
 * is computed -- where image rows are 16-byte multiples, otherwise plain);
 * it changes speed only, never a label or a centre.  Shapes exist for 2-D and 3-D images of uint8 with 1
 * or 3 channels and uint16 with 1 channel; other images use the per-voxel
 * kernel and report shape -1.  Shape indices run over
 * [0, sslic_num_tile_shapes(ndim)); -1 selects the measured shape from
 * sslic_autotune if one was recorded for this (dtype, channels, dims, grid),
 * else the built-in rule (the large tile unless too many centres reach it). */
SSLIC_API int sslic_num_tile_shapes(int32_t ndim, int32_t* count);

/* dims (host, 3 int32): tile extent along x, y, z; voxels_per_lane and
 * tma_staged (1 = TMA-staged tiles) may be NULL.  SSLIC_EINVAL for an
 * unknown shape. */
SSLIC_API int sslic_tile_shape_info(int32_t ndim, int32_t shape, int32_t* dims, int32_t* voxels_per_lane,
                                    int32_t* tma_staged);

/* Fix the context's shape (-1: back to automatic).  SSLIC_EUNSUPPORTED if
 * the image type has no tile kernel. */
SSLIC_API int sslic_set_tile_shape(sslic_ctx* c, int32_t shape);

/* The shape the next run will use (host int32). */
SSLIC_API int sslic_get_tile_shape(const sslic_ctx* c, int32_t* shape);

/* Measure every shape on this image and keep the fastest.  Seeds the image,
 * then for each shape runs reps + 1 assign + update iterations from the
 * same seeded centres (the first one warms up) and takes the median time of
 * the rest, measured with CUDA events on `stream`.  The fastest shape is set
 * on the context and recorded in a process-wide table for the image's
 * (dtype, channels, dims, grid), which later contexts and servers use.
 * labels_dev (V int32, device) is overwritten as scratch; best (host, may be
 * NULL) receives the chosen index and ms_out (host, may be NULL, at least
 * sslic_num_tile_shapes entries) the median milliseconds per shape.  Blocks
 * until the measurements are done; allocates one centre table.  Returns
 * SSLIC_EUNSUPPORTED for image types without a tile kernel. */
SSLIC_API int sslic_autotune(sslic_ctx* c, const void* image_dev, int32_t* labels_dev, void* stream,
                             int32_t reps, int32_t* best, float* ms_out);

/* Diagnostic of the tensor-core form (precision = 1): runs its MMA on one
 * assignment tile of the image (128 voxels: 16x8 in 2-D, 8x4x4 in 3-D, tiles
 * numbered in raster order) with the given centres (device, K x (C+n)) and
 * returns what the tensor core computed, before any decision:
 *   dots_host  (host, 128 x 32 float): dots[v][j] = sum_c (xh xh' + xh xl' + xl xh')
 *              with xh = bf16(x_v,c - mu_c), xl = bf16(x_v,c - mu_c - xh) and
 *              xh', xl' the same split of C_j,c - mu_c; v = voxel of the tile in
 *              raster order (x fastest), j = candidate slot; empty slots hold 0
 *   cand_host  (host, 32 int32): cluster index per slot (ascending), -1 = empty
 *   mu_host    (host, C float): the shift mu (mean of the candidates' features)
 * SSLIC_EINVAL if the context is not of the tensor-core form or the tile is
 * out of range; SSLIC_EUNSUPPORTED if more than 32 centres reach the tile. */
SSLIC_API int sslic_precision_probe(sslic_ctx* c, const void* image_dev, const float* centres_dev, int64_t tile,
                                    float* dots_host, int32_t* cand_host, float* mu_host);

/* Clear the process-wide table of measured shapes. */
SSLIC_API int sslic_tune_forget(void);

/* Write (shape >= 0) or read an entry of that table for the (dtype,
 * channels, dims, grid) of p, e.g. to restore measurements saved by an
 * earlier process.  Lookup gives -1 when there is no entry.  SSLIC_EINVAL
 * for bad parameters or shape, SSLIC_EUNSUPPORTED for image types without a
 * tile kernel.  Host only. */
SSLIC_API int sslic_tune_record(const sslic_params* p, int32_t shape);
SSLIC_API int sslic_tune_lookup(const sslic_params* p, int32_t* shape);

/* Serving (continuous batching).  A server keeps requests on the device and
 * advances all admitted requests together, one assign/update iteration per
 * round, each round running one launch per phase over every request of the
 * batch (batched form of Sec. 3.1 step 2).  A round's kernels read their
 * request counts from device tables, so each form of round (which image
 * types and tile shapes, whether requests join or finish) is captured once
 * as a CUDA graph and replayed.  Requests that have done their
 * iterations leave after the round and queued requests are admitted, first
 * come first served, as soon as the HBM budget has room for their image,
 * labels, centres, bins and sums.  Each request's labels and centres are the
 * ones sslic_run gives for it alone.  Requests need enforce_connectivity = 0.  A request with
 * conv_threshold > 0 stops after the round whose centre residual (computed
 * as sslic_run computes it) falls below the threshold, as sslic_run would;
 * while such requests are on the device, each round waits for the previous
 * one to finish before it is formed. */
typedef struct sslic_server sslic_server;

typedef struct {
    int64_t submitted, completed, rejected;  /* rejected: larger than the whole budget */
    int64_t rounds;                          /* batched iterations run */
    int32_t max_active;                      /* most requests on the device at once */
    int32_t status;                          /* SSLIC_OK, or the first error of the worker */
    int64_t peak_bytes;                      /* most budget bytes in use */
    double  voxel_iters;                     /* sum of voxels x iterations of completed requests */
    double  busy_s;                          /* first admission to last completion, seconds */
    double  p50_ms, p99_ms, mean_ms;         /* latency: submission to result in host memory */
    int64_t graph_launches;                  /* rounds replayed from a captured CUDA graph */
    int64_t graph_captures;                  /* round forms captured (a form is captured when it recurs) */
    int64_t eager_rounds;                    /* rounds of a form met for the first time, launched directly */
} sslic_server_stats;

/* Start a server on the current device with a device-memory budget for
 * requests (allocated once, here) and a cap on requests on the device. */
SSLIC_API int sslic_server_create(int64_t hbm_budget_bytes, int32_t max_active, sslic_server** out);

/* Queue one request.  image_host (read), labels_host (V int32, written) and
 * centres_host (K x (C+n) float32, written, may be NULL) must stay valid
 * until sslic_server_wait returns for the ticket; page-locked buffers let the
 * copies overlap the computation.  A request with enforce_connectivity
 * leaves the batched rounds after its last iteration: a finisher thread of
 * the server runs connectivity enforcement (Sec. 3.1 stage 3) on it on a
 * stream of its own, one request at a time, while the rounds of the others
 * go on, and then copies its results back.  Its workspace (2 bytes per voxel
 * plus about 45 bytes per local component of the largest such request so
 * far) is allocated by the server on first use, outside the budget.
 * SSLIC_ENOMEM if the request alone exceeds the budget; SSLIC_EUNSUPPORTED
 * for images of more than three axes. */
SSLIC_API int sslic_server_submit(sslic_server* s, const sslic_params* p, const void* image_host,
                                  int32_t* labels_host, float* centres_host, int64_t* ticket);

/* Wait up to timeout_ms for a ticket; on success the results are in the
 * caller's buffers and latency_ms (may be NULL) holds submission-to-result
 * time.  SSLIC_ETIMEOUT if the ticket is still running (wait again).  A
 * ticket is released by its first successful wait. */
SSLIC_API int sslic_server_wait(sslic_server* s, int64_t ticket, int32_t timeout_ms, double* latency_ms);

SSLIC_API int sslic_server_stats_get(sslic_server* s, sslic_server_stats* out);

/* Finish every queued request, stop the worker and free the server. */
SSLIC_API void sslic_server_destroy(sslic_server* s);

/* Tracing.  When enabled, every phase of the method is bracketed by CUDA
 * events recorded on the launching stream; sslic_profile_read waits for the
 * recorded events and returns the summed device time per phase.  The
 * kernel-launch counter runs whether or not timing is enabled. */
#define SSLIC_PHASE_SEED 0          /* seeding + perturbation */
#define SSLIC_PHASE_BINS 1          /* bin grid of the centres */
#define SSLIC_PHASE_ASSIGN 2        /* fused assign + map-update tile kernel */
#define SSLIC_PHASE_ASSIGN_VOXEL 3  /* per-voxel assign + update (other shapes, crowded tiles) */
#define SSLIC_PHASE_FINALIZE 4      /* centre division, residual */
#define SSLIC_PHASE_CONNECTIVITY 5  /* the whole connectivity enforcement */
#define SSLIC_NPHASES 6

typedef struct {
    double ms[8];             /* device milliseconds per phase */
    int64_t calls[8];         /* timed executions per phase */
    int64_t kernel_launches;  /* kernels this context launched since the last enable */
    int64_t rechecks;         /* voxels the tensor-core form re-evaluated in exact FP32 */
} sslic_profile;

/* Turn phase timing on (1) or off (0); both reset the counters. */
SSLIC_API int sslic_profile_enable(sslic_ctx* c, int32_t on);

/* Replay of the iterated loop (Sec. 3.1, steps 2-3) from a CUDA graph: on (1,
 * the default) or off (0).  When it is on, phase timing is off, the run has
 * no convergence threshold and max_iter >= 2, sslic_run / sslic_run_from /
 * sslic_run_host run the first iteration eagerly, capture the next one
 * (bins, assignment + update, reduce) from a stream the context owns, and
 * replay that graph on the caller's stream for the remaining iterations.
 * Results are bit-identical either way; the graph only removes per-kernel
 * launch latency, which dominates on small images.  The executable graph is
 * cached in the context and updated in place on later runs.
 * Returns SSLIC_EINVAL for a null context. */
SSLIC_API int sslic_set_loop_graph(sslic_ctx* c, int32_t enable);

/* Read the counters (host struct).  Synchronises on the recorded events. */
SSLIC_API int sslic_profile_read(sslic_ctx* c, sslic_profile* out);

/* Release the context (NULL is a no-op).  Synchronises the device first. */
SSLIC_API void sslic_destroy(sslic_ctx* c);

/* Static text for a status code. */
SSLIC_API const char* sslic_strerror(int code);

/* Detail for the most recent failure on this context ("" if none). */
SSLIC_API const char* sslic_last_error(const sslic_ctx* c);

#ifdef __cplusplus
}
#endif
#endif
