// static_ws.cu -- one SSLIC iteration that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs while another
// component owns the device allocator (for example inside a memory-pool or
// arena that must not grow), plugins loaded into a host process whose device
// memory is budgeted in advance, and real-time paths where an allocation's
// latency or its implicit device synchronisation is not acceptable.  For
// them sslic_iterate_static performs the same step as sslic_iterate -- the
// assignment of every voxel and the centre update -- with all of its
// workspace taken from one file-scope device array instead of a context.
//
// The array is a static __device__ object, so every GPU that loads this
// library holds it (kStaticBytes) until the process exits.  In host code its
// name only stands for it and is not a device address: the device address
// is looked up once per device with cudaGetSymbolAddress, on the first call
// made on that device (with the device current), and cached.  That first
// call should therefore come before any stream capture.  Every call shares
// the one array, which keeps the previous call's contents: the sums that
// must start at zero are cleared at the start of every call, and calls whose
// work overlaps on the GPU (different streams, no ordering) race on it.
#include <cstring>

#include "common.cuh"

namespace sslic {
namespace stat {

constexpr int64_t kMaxK = 16384;          // clusters
constexpr int kMaxC = 4;                  // channels
// assignment tiles; the count is taken over every base tile shape, so the
// smallest tile sets it: 65536 tiles of 16x8x8 voxels (3-D) or 32x16
// pixels (2-D), i.e. about 67M voxels or 33.5M pixels
constexpr int64_t kMaxTiles = 65536;
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr int kCW = kMaxC + 3, kAW = kMaxC + 4;
constexpr size_t kScanTmp = 64;           // >= scan_tmp_needed(kMaxK + 1) entries
constexpr size_t kBytes =
    align256(kMaxK * kCW * sizeof(float)) +                 // centres
    align256(kMaxK * kAW * sizeof(unsigned long long)) +    // integer sums
    align256(kMaxK * kMaxC * sizeof(double)) +              // float feature sums
    align256(kMaxK * sizeof(double)) +                      // residual terms
    align256(kMaxK * sizeof(unsigned)) +                    // non-empty flags
    align256(256 * sizeof(double)) + align256(256 * sizeof(unsigned)) + align256(sizeof(double)) +
    2 * align256((kMaxK + 1) * sizeof(unsigned)) +          // bin counts, starts
    3 * align256(kMaxK * sizeof(int)) +                     // cursor, items, bin of
    align256(kScanTmp * sizeof(unsigned)) +
    align256(kMaxTiles * sizeof(int64_t)) + align256(sizeof(unsigned));

static __device__ __align__(256) unsigned char g_scratch[kBytes];

static void* g_scratch_addr[kMaxDevices];  // device address of g_scratch, per device

// carve the workspace out of the array (same layout as kBytes)
static void carve(Workspace& w, unsigned char* base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base + off;
        off += align256(bytes);
        return p;
    };
    w.ctr = (float*)take(kMaxK * kCW * sizeof(float));
    w.acc = (unsigned long long*)take(kMaxK * kAW * sizeof(unsigned long long));
    w.facc = (double*)take(kMaxK * kMaxC * sizeof(double));
    w.resid_k = (double*)take(kMaxK * sizeof(double));
    w.nonempty_k = (unsigned*)take(kMaxK * sizeof(unsigned));
    w.resid_part = (double*)take(256 * sizeof(double));
    w.resid_cnt_part = (unsigned*)take(256 * sizeof(unsigned));
    w.resid_out = (double*)take(sizeof(double));
    w.bin_count = (unsigned*)take((kMaxK + 1) * sizeof(unsigned));
    w.bin_start = (unsigned*)take((kMaxK + 1) * sizeof(unsigned));
    w.bin_cursor = (unsigned*)take(kMaxK * sizeof(unsigned));
    w.bin_items = (int*)take(kMaxK * sizeof(int));
    w.bin_of = (int*)take(kMaxK * sizeof(int));
    w.scan_tmp = (unsigned*)take(kScanTmp * sizeof(unsigned));
    w.scan_tmp_len = kScanTmp;
    w.ovf_tiles = (int64_t*)take(kMaxTiles * sizeof(int64_t));
    w.ovf_count = (unsigned*)take(sizeof(unsigned));
}

}  // namespace stat
}  // namespace sslic

using namespace sslic;

extern "C" int sslic_iterate_static(const sslic_params* p, const void* image_dev, const float* centres_in_dev,
                                    int32_t* labels_dev, float* centres_out_dev, void* stream)
{
    if (!p || !image_dev || !centres_in_dev || !labels_dev || !centres_out_dev) return SSLIC_EINVAL;
    Geom g;
    int rc = make_geom(p, &g);
    if (rc) return rc;
    if (g.n > 3) return SSLIC_EUNSUPPORTED;  // the array's centre rows hold three positions
    if (g.K > stat::kMaxK || g.C > stat::kMaxC || assign_num_tiles(g) > stat::kMaxTiles ||
        scan_tmp_needed(g.K + 1) > stat::kScanTmp)
        return SSLIC_EINVAL;  // beyond the array's stated maximum sizes
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= stat::kMaxDevices) return SSLIC_ECUDA;
    if (!stat::g_scratch_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, stat::g_scratch) != cudaSuccess || !ptr) return SSLIC_ECUDA;
        stat::g_scratch_addr[dev] = ptr;
    }
    // a context on the stack whose workspace points into the array; the
    // launchers below are the ones every other entry point uses
    sslic_ctx c;
    c.p = *p;
    c.g = g;
    c.device = dev;
    // the tile shape with plain-load staging: a TMA-staged shape recorded by
    // the autotuner would need a status word and its check, which the array
    // does not provide
    if (has_tile_kernel(g)) {
        int sh = tuned_tile_shape(g);
        if (sh < 0) sh = default_tile_shape(g);
        c.tile_shape = sh % num_base_shapes(g.n);
    }
    if (cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SSLIC_ECUDA;
    stat::carve(c.ws, (unsigned char*)stat::g_scratch_addr[dev]);
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = cuda_check(&c, cudaMemsetAsync(c.ws.acc, 0, g.K * g.AW * sizeof(unsigned long long), st),
                         "clear sums")))
        return rc;
    if (g.dtype == SSLIC_F32 &&
        (rc = cuda_check(&c, cudaMemsetAsync(c.ws.facc, 0, g.K * g.C * sizeof(double), st), "clear sums")))
        return rc;
    if ((rc = launch_import_centres(&c, centres_in_dev, st))) return rc;
    if ((rc = build_bins(&c, st))) return rc;
    if ((rc = launch_assign_update(&c, image_dev, labels_dev, st))) return rc;
    if ((rc = launch_finalize(&c, st))) return rc;
    return launch_export_centres(&c, centres_out_dev, st);
}
