// common.cuh -- shared definitions of the sm_103a SSLIC kernels.
//
// Internal conventions (the C ABI in include/sslic.h converts to and from
// the public layout):
//  * every image is handled as 3-D: missing axes have N_d = 1 and S_d = 1,
//    which adds no term to the distance and no seed along that axis;
//  * centres are a K x CW float table with CW = C + 3: the C features, then
//    x_0, x_1, x_2 (padded axes hold 0);
//  * integer images accumulate exact uint64 sums (C features, 3 positions,
//    count) per cluster; float images add C double feature sums.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "sslic.h"

namespace sslic {

constexpr int kMaxChannels = 256;
constexpr uint8_t kNoSlot = 255;

constexpr int kMaxDims = 4;  // images of 1 to 4 dimensions (the paper's filter is n-dimensional, Sec. 3)

struct Geom {
    int n;                // real spatial dims (1..4)
    int64_t N[kMaxDims];  // sizes, padded with 1
    int S[kMaxDims];      // grid, padded with 1
    int64_t nb[kMaxDims]; // seeds (= bins) per axis: ceil(N_d / S_d)
    int64_t off[kMaxDims];// lattice offset o_d = floor((N_d - 1 - (nb_d - 1) S_d) / 2)
    int64_t V, K;
    int C;                // channels
    int dtype;            // SSLIC_U8 / SSLIC_U16 / SSLIC_F32
    int CW;               // internal centre row width C + P, P = max(3, n) position slots
    int AW;               // accumulator row width C + P + 1 (features, positions, count last)
    float w[kMaxDims];    // fl32(m^2 / S_d^2)
    double w64[kMaxDims]; // m^2 / S_d^2
    int64_t sprod;        // prod S_d over the real axes
};

// ---- packed FP32 pairs (sm_100 family .f32x2 arithmetic, round to nearest) --
__device__ __forceinline__ uint64_t pk2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(uint64_t v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// ---- geometry helpers ------------------------------------------------------
__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

__host__ __device__ __forceinline__ int64_t vidx(const Geom& g, int64_t x, int64_t y, int64_t z, int64_t w = 0)
{
    return x + g.N[0] * (y + g.N[1] * (z + g.N[2] * w));
}

// Covered range of a centre coordinate c along an axis of grid S: the voxels
// x with c - S <= x < c + S are exactly [ceil(c) - S, ceil(c) + S - 1]
// (S is an integer, so c - S <= x <=> x >= ceil(c) - S, and x < c + S <=>
// x <= ceil(c) + S - 1).  Sec. 2.2 "[2S x 2S] region around C_k".
__device__ __forceinline__ int64_t window_lo(float c, int S)
{
    return (int64_t)ceilf(c) - S;
}

// bin of a centre coordinate: floor(c) / S (exactly floor(c / S) for c >= 0)
__device__ __forceinline__ int64_t bin_of_coord(float c, int S, int64_t nb)
{
    int64_t b = (int64_t)floorf(c);
    b = b < 0 ? 0 : b / S;
    return b >= nb ? nb - 1 : b;
}

// one image's arguments of the assignment kernels (one entry per request in
// the batched form)
struct TileArgs {
    Geom g;
    const void* img;
    const float* ctr;
    const unsigned* bin_start;
    const int* bin_items;
    int32_t* labels;
    unsigned long long* acc;
    double* facc;
    int ntx, nty;     // tile grid of the tile shape in use
    int tx, ty, tz;   // that shape's tile dimensions
    const int* lists; // per-tile candidate records of that shape, or nullptr (gathered in the kernel)
    int64_t tile0;    // first tile of the launch (a slab of the streamed form), else 0
};

// Part of an image along its last axis (z in 3-D, y in 2-D) for the streamed
// form: the kernels read and write only the planes [lo, hi), through buffers
// whose pointers are set back by lo planes so that voxel indices stay global.
struct Slab {
    int64_t lo, hi;
};

// ---- context ---------------------------------------------------------------
struct Workspace {
    // centres and update sums
    float* ctr = nullptr;               // K x CW
    unsigned long long* acc = nullptr;  // K x AW
    double* facc = nullptr;             // K x C (float images)
    double* resid_k = nullptr;          // K: per-cluster residual terms
    unsigned* nonempty_k = nullptr;     // K
    double* resid_part = nullptr;       // reduction partials
    unsigned* resid_cnt_part = nullptr;
    double* resid_out = nullptr;        // [0] residual
    // bins
    unsigned* bin_count = nullptr;      // K + 1
    unsigned* bin_start = nullptr;      // K + 1
    unsigned* bin_cursor = nullptr;     // K
    int* bin_items = nullptr;           // K
    int* bin_of = nullptr;              // K
    unsigned* scan_tmp = nullptr;       // scan block sums (all levels)
    size_t scan_tmp_len = 0;
    // precision form: error flag of bounded waits, rechecked-voxel count
    unsigned* hc_err = nullptr;
    unsigned long long* hc_rechecks = nullptr;
    // assign tile overflow list
    int64_t n_assign_tiles = 0;
    int64_t* ovf_tiles = nullptr;
    unsigned* ovf_count = nullptr;
    int* tile_lists = nullptr;          // n_assign_tiles records of tile_list_stride() ints (tile kernel images)
    // connectivity
    uint16_t* lid = nullptr;            // V
    int64_t lid_cap = 0;                // voxels lid holds
    int64_t n_ccl_tiles = 0;
    int* tile_base = nullptr;           // n_ccl_tiles: first component record of each tile
    int* tile_cnt = nullptr;            // n_ccl_tiles: component records of each tile
    unsigned* counters = nullptr;       // [0] M, [1] overflow, [2] new count
    int64_t m_cap = 0;
    int* comp_label = nullptr;
    int* gparent = nullptr;
    // per record: its own size and first voxel as the tile pass leaves them;
    // after the flatten pass a root's entries hold its whole component's
    unsigned long long* root_size = nullptr;
    unsigned long long* root_first = nullptr;
    uint8_t* fin = nullptr;
    int* out_label = nullptr;
    int* link = nullptr;
    unsigned long long* new_key = nullptr;
    int* new_val = nullptr;
    unsigned long long* sort_key = nullptr;  // power-of-two scratch for large sorts
    int* sort_val = nullptr;
    int64_t sort_cap = 0;
    // host-buffer entry point
    void* img_dev = nullptr;
    int32_t* lab_dev = nullptr;
    float* cen_dev = nullptr;
    // streamed form (sslic_run_streamed): two slab buffers of image planes and
    // of labels, a copy stream and the events that order the two streams
    unsigned char* slab_img[2] = {nullptr, nullptr};
    int32_t* slab_lab[2] = {nullptr, nullptr};
    int64_t slab_planes = 0;            // planes each buffer holds (image: + 4 halo planes)
    cudaStream_t copy_stream = nullptr;  // uploads
    cudaStream_t down_stream = nullptr;  // label downloads (the other direction, concurrently)
    cudaEvent_t slab_ev[8] = {};        // img ready / img free / labels done / labels free, per buffer
    // connectivity in slabs (conn_slabs_*): the phase-1 seed voxel of every
    // centre, the labels of the last planes of the previous slab, and how far
    // the slabs have come
    long long* conn_seed = nullptr;     // K
    int32_t* conn_carry = nullptr;      // S_last planes
    int64_t conn_next = 0;              // first plane the next slab must start at
    int64_t conn_carried = 0;           // planes the carry holds (those just below conn_next)
};

}  // namespace sslic

namespace sslic {
struct ProfRec {
    int phase;
    cudaEvent_t start, stop;
};
}  // namespace sslic

struct sslic_ctx {
    sslic_params p;
    sslic::Geom g;
    sslic::Workspace ws;
    int device = 0;
    int sms = 148;
    int busy = 0;
    int tile_shape = -1;   // assignment tile shape index, -1 = chosen from the grid (assign_tile.cu)
    int status_pending = 0;  // a kernel with bounded waits ran: check the status flag
    char err[512] = {0};
    // the iterated loop of a run replayed from a CUDA graph (run_loop): the
    // private stream it is captured from and the cached executable graph
    int loop_graph = 1;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t loop_exec = nullptr;
    // sslic_run_host with connectivity: the relabel pass runs in slabs of
    // tile planes and each slab's final labels go to this host buffer on the
    // download stream right after it (relabel_sent records that it happened)
    int32_t* relabel_host = nullptr;
    int relabel_sent = 0;
    // tracing
    int prof_on = 0;
    int64_t launches = 0;
    std::vector<sslic::ProfRec> prof;       // recorded brackets (events owned by the pool)
    std::vector<cudaEvent_t> prof_pool;     // created events, reused
};

namespace sslic {
// kernels / launchers implemented in the .cu files
int launch_seed(sslic_ctx* c, const void* img, cudaStream_t st, const Slab* slab = nullptr);
int build_bins(sslic_ctx* c, cudaStream_t st);
int launch_assign_update(sslic_ctx* c, const void* img, int32_t* labels, cudaStream_t st, const Slab* slab = nullptr);
// residual: also reduce the per-cluster residual terms into resid_out (a
// run without a convergence threshold needs it only after its last iteration)
int launch_finalize(sslic_ctx* c, cudaStream_t st, bool residual = true);
int launch_residual(sslic_ctx* c, cudaStream_t st);
int launch_export_centres(sslic_ctx* c, float* out, cudaStream_t st);
int launch_import_centres(sslic_ctx* c, const float* in, cudaStream_t st);
int run_connectivity(sslic_ctx* c, const int32_t* labels_in, int32_t* labels_out, cudaStream_t st,
                     int64_t* num_labels);
// Connectivity for the batched server: one context that owns only the
// connectivity workspace, retargeted to each request's geometry (its
// buffers only grow) and given the request's centres (internal layout,
// K x CW) for the call; labels are relabelled in place on st.
sslic_ctx* conn_ctx_create(int device, int sms);
int conn_ctx_run(sslic_ctx* c, const sslic_params& p, const Geom& g, const float* ctr, int32_t* labels,
                 cudaStream_t st, int64_t* num_labels);
void conn_ctx_destroy(sslic_ctx* c);
int scan_exclusive_u32(sslic_ctx* c, const unsigned* in, unsigned* out, int64_t n, cudaStream_t st);
size_t scan_tmp_needed(int64_t n);
int64_t ccl_num_tiles(const Geom& g);
int64_t assign_num_tiles(const Geom& g);
int tile_list_stride();  // ints per per-tile candidate record
// the batched queue's per-tile records for the requests of one group (each
// request's TileArgs::lists holds its tiles' records); crowded tiles go to ovf
// as (request << 40 | tile)
cudaError_t launch_tile_lists_queue(int ndim, const TileArgs* reqs, const int64_t* tpre, const int* nR, int64_t* ovf,
                                    unsigned* ovf_count, int grid, cudaStream_t st);
constexpr int kTileListStride = 49;  // a record: count, then up to 48 centre indices in ascending order
// per-tile candidate records for tiles [tile0, tile0 + ntiles) of a tx x ty x tz
// tiling (ntx x nty tiles per plane of tiles), into the workspace's list buffer
int launch_tile_lists(sslic_ctx* c, int ndim, int tx, int ty, int tz, int ntx, int nty, int64_t tile0,
                      int64_t ntiles, cudaStream_t st);
bool has_tile_kernel(const Geom& g);  // integer images with a tile kernel (2-D, 3-D)
// TMA tensor map of an image as bytes [N_2][N_1][N_0 * C * esz] (tma.cu);
// map points at 128 bytes, 64-byte aligned
bool image_tma_ok(const Geom& g, const void* img, int esz);
int encode_image_map(void* map, const Geom& g, const void* img, int esz, int tx, int ty, int tz);
// high-channel float images (hc.cu)
bool hc_applies(const Geom& g);
int64_t hc_num_tiles(const Geom& g);
int launch_hc(sslic_ctx* c, const float* img, int32_t* labels, cudaStream_t st);
int launch_hc_probe(sslic_ctx* c, const float* img, int32_t* labels, int64_t tile, float* dots, int* cand,
                    float* mu, cudaStream_t st);
int default_tile_shape(const Geom& g);
int num_base_shapes(int ndim);
int num_tile_shapes(int ndim);
void tile_dims(int ndim, int shape, int* tx, int* ty, int* tz);
int tile_voxels_per_lane(int ndim, int shape);
template <typename T, int C, int NDIM>
cudaError_t launch_tile_queue(int shape, const TileArgs* reqs, const int64_t* tpre, const int* nR, int64_t* ovf,
                              unsigned* ovf_count, int grid, cudaStream_t st);
template <typename T, int C, int NDIM>
int launch_tile_impl(sslic_ctx* c, const T* img, int32_t* labels, cudaStream_t st, const Slab* slab = nullptr);
template <typename T>
int launch_voxel_tiles(sslic_ctx* c, const T* img, int32_t* labels, int tx, int ty, int tz, int ntx, int nty,
                       cudaStream_t st);
int ensure_ccl_capacity(sslic_ctx* c, int64_t m);
// grows the component records to m, keeping the first `keep` records the
// tile pass has written (the slab form grows between slabs)
int grow_ccl_records(sslic_ctx* c, int64_t m, int64_t keep, cudaStream_t st);
int ensure_conn_slab_scratch(sslic_ctx* c);
// connectivity of an image handed over slab by slab (ranges of planes along
// the last axis, in order): begin, add every slab, finish, then relabel
// each slab (ccl.cu)
int conn_slabs_begin(sslic_ctx* c, cudaStream_t st);
int conn_slabs_add(sslic_ctx* c, const int32_t* labels_slab, int64_t lo, int64_t hi, cudaStream_t st);
int conn_slabs_finish(sslic_ctx* c, cudaStream_t st, int64_t* num_labels);
int conn_slabs_relabel(sslic_ctx* c, int32_t* labels_out_slab, int64_t lo, int64_t hi, cudaStream_t st);
int set_error(sslic_ctx* c, int code, const char* fmt, ...);
int make_geom(const sslic_params* p, Geom* g);
// phase brackets: prof_begin returns a record index (or -1 when timing is off)
int prof_begin(sslic_ctx* c, int phase, cudaStream_t st);
void prof_end(sslic_ctx* c, int rec, cudaStream_t st);
inline void count_launch(sslic_ctx* c, int n = 1) { c->launches += n; }
// tile shape measured by sslic_autotune for this image type and grid, or -1
int tuned_tile_shape(const Geom& g);
// holds the context for one call; ok = false when another call holds it
struct Busy {
    sslic_ctx* c;
    bool ok;
    explicit Busy(sslic_ctx* c_) : c(c_) { ok = __sync_bool_compare_and_swap(&c->busy, 0, 1); }
    ~Busy() { if (ok) __sync_lock_release(&c->busy); }
};
int cuda_check(sslic_ctx* c, cudaError_t e, const char* what);
}  // namespace sslic
