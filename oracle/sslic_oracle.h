/*
 * sslic_oracle.h -- plain, slow, single-threaded CPU oracle for Scalable SLIC
 * (Lowekamp et al., "Scalable Simple Linear Iterative Clustering (SSLIC)
 * Using a Generic and Parallel Approach", arXiv 1806.08741).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * The oracle follows the paper's centre-centric formulation step by step:
 *   - seeding on a regular grid and gradient perturbation   (Sec. 2.2 and 3.1, "Initialization")
 *   - assignment by iterating over the centres, each one visiting its
 *     2S-per-side window and keeping the strictly smaller distance
 *                                                           (Sec. 2.2 "Update label and distance images")
 *   - the distance D^2 = d_c^2 + sum_i (d_i/S_i)^2 m^2      (Sec. 2.1, anisotropic form Sec. 3.3)
 *   - the centre update as the mean of [I(x), x]            (Sec. 2.2 "Update clusters", Sec. 3.1 map-reduce)
 *   - termination on the iteration cap or the centre residual
 *                                                           (Sec. 2.2 "Terminate iterations if", Sec. 3.2)
 *   - connectivity enforcement with a marker image          (Sec. 3.1, stage 3)
 *
 * Every place where the paper is silent is resolved by a stated reading; the
 * readings are listed next to the function that applies them.
 *
 * Two arithmetic modes:
 *   ORACLE_FP32 : "FP32 canonical".  Distances and float-image gradients are
 *                 evaluated in IEEE single precision, one rounding per
 *                 operation, in a fixed order and without fused multiply-add.
 *                 Centres are stored as float.  This is the mode that integer
 *                 images are compared against bit for bit.
 *   ORACLE_FP64 : the same formulas in double precision; centres kept in
 *                 double.  The reference for float images.
 *
 * Layout: image C-contiguous [N_{n-1}]...[N_0][C] (channels interleaved,
 * dimension 0 fastest); labels int32 [N_{n-1}]...[N_0]; centres a K x (C+n)
 * table of doubles (features first, then positions x_0..x_{n-1}).  In FP32
 * mode every stored centre value is exactly a float.
 */
#ifndef SSLIC_ORACLE_H
#define SSLIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_U8 = 0, ORACLE_U16 = 1, ORACLE_F32 = 2 };
enum { ORACLE_FP32 = 0, ORACLE_FP64 = 1 };

typedef struct {
    int32_t ndim;           /* 1..4 */
    int64_t size[4];        /* N_d, d = 0 fastest; unused dims ignored */
    int32_t channels;       /* C >= 1 */
    int32_t dtype;          /* ORACLE_U8 / ORACLE_U16 / ORACLE_F32 */
    int32_t grid[4];        /* S_d >= 1 */
    double  m;              /* proximity weight */
    int32_t max_iter;       /* >= 0 */
    double  conv_threshold; /* <= 0: always run max_iter iterations */
    int32_t perturb;        /* 0/1 */
    int32_t enforce_connectivity; /* 0/1 */
    int32_t mode;           /* ORACLE_FP32 / ORACLE_FP64 */
} oracle_params;

/* Number of clusters K = prod_d ceil(N_d / S_d).  Returns -1 on bad params. */
int64_t oracle_num_clusters(const oracle_params* p);

/* Seeding (+ perturbation if p->perturb).  centres: K x (C+n). */
int oracle_seed(const oracle_params* p, const void* image, double* centres);

/* Gradient magnitude^2 at voxel index q (Frobenius norm of the central
 * difference Jacobian, squared).  Returned as double; in FP32 mode for float
 * images it is the float value of the canonical single-precision sum. */
double oracle_gradient(const oracle_params* p, const void* image, int64_t q);

/* One assignment: labels (V) from centres (K x (C+n)).  Centre-centric. */
int oracle_assign(const oracle_params* p, const void* image,
                  const double* centres, int64_t K, int32_t* labels);

/* The labels oracle_assign would leave at the nq voxels q[i] (raster
 * indices), for images too large to assign whole.  The candidates of voxel
 * i are cand[cand_start[i] .. cand_start[i+1]) (cand_start has nq + 1
 * entries); they must include every centre whose window covers the voxel,
 * in any order (others fail the window test). */
int oracle_assign_voxels(const oracle_params* p, const void* image, const double* centres, int64_t K,
                         const int64_t* q, int64_t nq, const int64_t* cand_start, const int64_t* cand,
                         int32_t* labels_out);

/* One update: new centres from labels.  centres is read (previous values,
 * kept for empty clusters) and overwritten.  counts (K, may be NULL)
 * receives member counts; residual (may be NULL) receives the residual. */
int oracle_update(const oracle_params* p, const void* image,
                  const int32_t* labels, int64_t K, double* centres,
                  int64_t* counts, double* residual);

/* Distance D^2 between voxel feature/position and one centre, in the mode's
 * arithmetic (exposed for tests). */
double oracle_distance(const oracle_params* p, const double* feature,
                       const int64_t* pos, const double* centre);

/* Connectivity enforcement.  labels_in is the last assignment (read only),
 * labels_out receives the relabelled image; *num_labels = K + #new labels. */
int oracle_connectivity(const oracle_params* p, const double* centres,
                        int64_t K, const int32_t* labels_in,
                        int32_t* labels_out, int64_t* num_labels);

/* Whole method.  centres_out: K x (C+n) (may be NULL).  iters_done,
 * residual, num_labels may be NULL. */
int oracle_slic(const oracle_params* p, const void* image, int32_t* labels,
                double* centres_out, int32_t* iters_done, double* residual,
                int64_t* num_labels);

/* Same, starting from the given centres instead of seeding (resume). */
int oracle_slic_from(const oracle_params* p, const void* image,
                     const double* init_centres, int32_t* labels,
                     double* centres_out, int32_t* iters_done,
                     double* residual, int64_t* num_labels);

/* The whole method in the paper's multi-threaded form (Sec. 3.1): the
 * image split into non-overlapping regions (ranges of planes along the last
 * axis), each assigned and mapped by one thread, the per-region sums merged
 * per label.  Same results as oracle_slic, bit for bit (float images keep
 * the sequential map so that their double sums are added in raster order;
 * connectivity is sequential).  threads >= 1; the library built with
 * OpenMP runs the regions on that many threads, the plain build one after
 * another. */
int oracle_slic_regions(const oracle_params* p, const void* image, int32_t* labels,
                        double* centres_out, int32_t* iters_done, double* residual,
                        int64_t* num_labels, int threads);

/* Threads OpenMP would use by default (1 in the build without OpenMP). */
int oracle_threads_available(void);

/* 8-bit sRGB -> CIE-Lab in double precision (reading R16 in the source):
 * rgb holds n interleaved (R, G, B) triples, lab receives n (L, a, b). */
int oracle_srgb_to_lab(const uint8_t* rgb, int64_t n, double* lab);

#ifdef __cplusplus
}
#endif
#endif
