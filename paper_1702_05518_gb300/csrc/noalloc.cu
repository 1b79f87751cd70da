// noalloc.cu -- Jones-Plassmann colouring of a device-resident CSR graph that allocates no
// memory: its scratch is one file-scope device array of fixed size.
//
// Who needs it: callers that cannot let a library allocate device memory.  A process whose
// device memory is held by its own caching allocator (so a cudaMalloc inside the call can fail
// although the pool has room), and a serving loop that must not take the device-wide
// synchronisation that cudaFree implies, both call this instead of gmrf_color_graph.
//
// The colouring itself is the one of gmrf_color_graph (same kernels, same result); only where
// the scratch and the graph live differs.  Overlapping calls share the scratch and race.
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/gmrf.h"
#include "gmrf_internal.h"

using namespace gmrf;

namespace {

// Scratch: [0, 256) the CSR check flag, then the JP scratch (priorities [n] u32, round
// selection [n] u8, coloured-vertex counter and largest colour), laid out by jp_color.
constexpr size_t kFlagBytes = 256;
constexpr size_t kJpBytes = 4ull * GMRF_NOALLOC_MAX_VERTICES + 1ull * GMRF_NOALLOC_MAX_VERTICES + 256;
constexpr size_t kScratchBytes = kFlagBytes + kJpBytes;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
void *g_scratch_ptr[kMaxDevices] = {};

enum : int32_t { kBadFirst = 1, kBadLast = 2, kBadOrder = 4, kBadColumn = 8, kSelfLoop = 16 };

// row_ptr[0] == 0, non-decreasing, row_ptr[n] == nnz: afterwards every row's range lies in
// [0, nnz) and the column check may walk it.
__global__ void rows_check_kernel(int32_t n, int64_t nnz, const int32_t *rp, int32_t *flag)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i <= n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t a = rp[i];
        int32_t bad = 0;
        if (i == 0 && a != 0) bad |= kBadFirst;
        if (i == n && static_cast<int64_t>(a) != nnz) bad |= kBadLast;
        if (i < n && rp[i + 1] < a) bad |= kBadOrder;
        if (bad) atomicOr(flag, bad);
    }
}

// Every column index in [0, n) and no self-loop; skipped when the rows failed their check.
__global__ void cols_check_kernel(int32_t n, const int32_t *rp, const int32_t *ci, int32_t *flag)
{
    if (*reinterpret_cast<volatile int32_t *>(flag) != 0) return;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int32_t bad = 0;
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t j = ci[e];
            if (j < 0 || j >= n) bad |= kBadColumn;
            if (j == static_cast<int32_t>(i)) bad |= kSelfLoop;
        }
        if (bad) atomicOr(flag, bad);
    }
}

int grid_for(int64_t items)
{
    int64_t g = (items + 255) / 256;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return static_cast<int>(g);
}

gmrf_status cuda_fail(cudaError_t e, const char *where)
{
    std::string msg = std::string("CUDA error ") + cudaGetErrorString(e) + " in " + where;
    return static_cast<gmrf_status>(record_error(GMRF_E_CUDA, msg.c_str()));
}

}  // namespace

extern "C" gmrf_status gmrf_color_graph_noalloc(int32_t n, int64_t nnz, const int32_t *row_ptr,
                                                const int32_t *col_idx, const uint32_t *priorities,
                                                uint64_t seed, int32_t *colors, int32_t *num_colors,
                                                void *cuda_stream)
{
    record_error(GMRF_OK, "");
    if (n < 1) return static_cast<gmrf_status>(record_error(GMRF_E_INVALID, "CSR: n must be >= 1"));
    if (n > GMRF_NOALLOC_MAX_VERTICES) {
        std::string msg = "n = " + std::to_string(n) + " exceeds the static scratch of gmrf_color_graph_noalloc (" +
                          std::to_string(GMRF_NOALLOC_MAX_VERTICES) + " vertices); use gmrf_color_graph";
        return static_cast<gmrf_status>(record_error(GMRF_E_INVALID, msg.c_str()));
    }
    if (nnz < 0 || nnz > INT32_MAX)
        return static_cast<gmrf_status>(record_error(GMRF_E_INVALID, "CSR: nnz must lie in [0, 2^31)"));
    if (!row_ptr || (!col_idx && nnz > 0) || !colors || !num_colors)
        return static_cast<gmrf_status>(
            record_error(GMRF_E_INVALID, "row_ptr, col_idx (when nnz > 0), colors and num_colors are required"));
    if (jp_scratch_bytes(n) > kJpBytes)
        return static_cast<gmrf_status>(record_error(GMRF_E_INVALID, "JP scratch larger than the static array"));

    // Set-up, once per device with that device current: the address of the static scratch.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return static_cast<gmrf_status>(record_error(GMRF_E_UNSUPPORTED, "device ordinal beyond 63"));
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> guard(g_setup_lock);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
            g_scratch_ptr[dev] = p;
        }
        base = g_scratch_ptr[dev];
    }
    int32_t *flag = static_cast<int32_t *>(base);
    void *jp_scratch = static_cast<unsigned char *>(base) + kFlagBytes;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    // The flag must start at zero every call; the JP scratch is initialised by jp_color itself.
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int32_t), stream)) != cudaSuccess) return cuda_fail(e, "flag reset");
    rows_check_kernel<<<grid_for(static_cast<int64_t>(n) + 1), 256, 0, stream>>>(n, nnz, row_ptr, flag);
    cols_check_kernel<<<grid_for(n), 256, 0, stream>>>(n, row_ptr, col_idx, flag);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "CSR check launch");
    int32_t bad = 0;
    if ((e = cudaMemcpyAsync(&bad, flag, sizeof(bad), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_fail(e, "CSR check read-back");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "CSR check");
    if (bad) {
        const char *what = (bad & kBadFirst)    ? "CSR: row_ptr[0] must be 0"
                           : (bad & kBadLast)   ? "CSR: row_ptr[n] must equal nnz"
                           : (bad & kBadOrder)  ? "CSR: row_ptr must be non-decreasing"
                           : (bad & kBadColumn) ? "CSR: column index out of range"
                                                : "CSR: self-loop";
        return static_cast<gmrf_status>(record_error(GMRF_E_INVALID, what));
    }

    int32_t k = 0;
    if ((e = jp_color(n, row_ptr, col_idx, priorities, seed, colors, jp_scratch, &k, stream)) != cudaSuccess)
        return cuda_fail(e, "jp_color");
    *num_colors = k;
    return GMRF_OK;
}
