// cube_counts_to_offsets_noalloc: the exclusive scan that turns per-cell
// particle counts into the cell-ordered store's offsets, for callers that
// cannot allocate device memory.
//
// Its only scratch is a fixed, file-scope device array (the scan's per-block
// sums).  Every GPU that loads libcube holds this array until the process
// exits.  The array's host-side name is not a device address, so the host
// code below asks the runtime for the device address once per device and
// passes that pointer to the kernels.
#include <mutex>
#include <string>

#include "cube.h"
#include "kernels.h"

namespace {

constexpr int kScanTile = 4096;                                  // cells per scan block
constexpr int64_t kMaxBlocks = 65536;                            // block sums the array holds
constexpr int64_t kMaxCells = kMaxBlocks * kScanTile;            // 268,435,456 cells

// block sums + the total: (kMaxBlocks + 1) words = 256 KiB + 4 bytes
static __device__ __align__(256) unsigned g_scan_scratch[kMaxBlocks + 1];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned* g_scratch_ptr[kMaxDevices] = {};

cube_status noalloc_fail(cube_status s, const std::string& m) {
    cube::set_last_error(m);        // reported by cube_last_error()
    return s;
}

}  // namespace

extern "C" cube_status cube_counts_to_offsets_noalloc(const uint32_t* counts, int64_t n_cells, uint32_t* offsets,
                                                      void* cuda_stream) {
    if (!counts || !offsets) return noalloc_fail(CUBE_E_ARG, "counts and offsets are required");
    if (n_cells < 1 || n_cells > kMaxCells)
        return noalloc_fail(CUBE_E_ARG, "n_cells must be in [1, 268435456] (the fixed scratch holds 65536 "
                                        "block sums of 4096 cells)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(CUBE_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(CUBE_E_ARG, "device index out of range");
    unsigned* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            // first call on this device, with it current: device address of the array
            e = cudaGetSymbolAddress((void**)&g_scratch_ptr[dev], g_scan_scratch);
            if (e != cudaSuccess) {
                g_scratch_ptr[dev] = nullptr;
                return noalloc_fail(CUBE_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
        }
        scratch = g_scratch_ptr[dev];
    }
    // every block sum and the total are written before they are read, so the
    // scratch needs no clearing between calls
    cube::exclusive_scan(counts, offsets, n_cells, scratch, (cudaStream_t)cuda_stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(CUBE_E_CUDA, std::string("scan launch: ") + cudaGetErrorString(e));
    return CUBE_OK;
}
