// spamm_multiply_noalloc: the SpAMM product for callers that must not
// allocate device memory.
//
// Some callers cannot let a library call cudaMalloc.  Examples: a host
// program that reserved all device memory up front and forbids allocation
// once it is running (real-time or fixed-budget services), and code that
// runs where an allocation would be unsafe or would break the caller's own
// memory accounting.  spamm_multiply keeps per-size scratch that it
// allocates on first use.  This variant keeps its scratch in one
// file-scope device array of fixed size instead, so it never allocates.
//
// The array lives on every GPU that loads the library, until the process
// exits.  Every call shares it, and a call leaves its contents behind, so
// two calls that overlap on the GPU (different streams, or different host
// threads) race; calls on one stream are ordered and safe.
#include <cmath>
#include <mutex>
#include <string>

#include "spamm.h"
#include "spamm_internal.cuh"

namespace spamm {
void set_error_message(const char* msg);  // spamm_api.cu: message for spamm_last_error()

namespace {

constexpr int kNoAllocMaxN = SPAMM_NOALLOC_MAX_N;
constexpr size_t kTileDoubles = (size_t)kNoAllocMaxN * kNoAllocMaxN;  // m*nb <= 512 for nb in {32, 64, 128}
constexpr size_t kTreeDoubles = 512;   // all quadtree levels for m <= 16 (341 nodes)
constexpr size_t kListDoubles = 4096;  // counts (m^2 <= 256 ints), task lists (m^3 <= 4096 ints), counters,
                                       // compacted output tiles (m^2 <= 256 ints)
constexpr size_t kScratchDoubles = 3 * kTileDoubles + 3 * kTreeDoubles + kListDoubles;

// The scratch itself: about 6.3 MB per GPU.  In host code this name is only
// a stand-in; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
int scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error_message((std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
        return SPAMM_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error_message("device ordinal out of range");
        return SPAMM_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error_message((std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
            return SPAMM_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return SPAMM_OK;
}

// Device memory of the current device, or managed memory.  Device memory of another GPU is refused: without
// peer access the kernels could not reach it.
bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    if (a.type != cudaMemoryTypeDevice) return false;
    int cur = -1;
    return cudaGetDevice(&cur) == cudaSuccess && a.device == cur;
}

}  // namespace
}  // namespace spamm

using namespace spamm;

extern "C" int spamm_multiply_noalloc(const double* A, const double* B, double* C, int n, double tau, int leaf,
                                      void* stream) {
    set_error_message("");
    if (leaf == 0) leaf = 64;
    if (n <= 0 || !(tau >= 0.0) || std::isinf(tau) || !(leaf == 32 || leaf == 64 || leaf == 128)) {
        set_error_message("n must be positive, tau finite and >= 0, leaf 32, 64 or 128");
        return SPAMM_ERR_ARG;
    }
    if (n > kNoAllocMaxN) {
        set_error_message("n exceeds SPAMM_NOALLOC_MAX_N (512), the size of the fixed scratch array");
        return SPAMM_ERR_UNSUPPORTED;
    }
    if (!A || !B || !C || !on_device(A) || !on_device(B) || !on_device(C)) {
        set_error_message("A, B and C must be device pointers of the current device");
        return SPAMM_ERR_ARG;
    }
    double* base = nullptr;
    int st = scratch_address(&base);
    if (st) return st;
    init_device_attributes();

    const Geometry g = make_geometry(n, leaf);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TileMat a{base, base + 3 * kTileDoubles};
    TileMat b{base + kTileDoubles, base + 3 * kTileDoubles + kTreeDoubles};
    TileMat c{base + 2 * kTileDoubles, base + 3 * kTileDoubles + 2 * kTreeDoubles};
    int* counts = reinterpret_cast<int*>(base + 3 * kTileDoubles + 3 * kTreeDoubles);
    int* jlist = counts + 256;
    unsigned long long* ctr = reinterpret_cast<unsigned long long*>(counts + 256 + 4096);
    int* tile_count = reinterpret_cast<int*>(ctr + 1);
    int* tile_list = tile_count + 2;

    // Only the task counter and the output-tile count must start from zero;
    // every other word the kernels read is written earlier in this same call.
    cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) + sizeof(int), s);
    if (e != cudaSuccess) {
        set_error_message((std::string("cudaMemsetAsync: ") + cudaGetErrorString(e)).c_str());
        return SPAMM_ERR_CUDA;
    }
    launch_pack(A, n, g, nullptr, nullptr, a, s);
    launch_tree(g, a.tree, nullptr, s);
    launch_pack(B, n, g, nullptr, nullptr, b, s);
    launch_tree(g, b.tree, nullptr, s);
    const CullOut co{counts, jlist, tile_list, tile_count, c.tree, 0};
    launch_cull(g, a.tree, b.tree, tau, co, ctr, nullptr, nullptr, s);
    launch_gemm_f64(g, a.t, b.t, c.t, a.tree, b.tree, c.tree, counts, jlist, tile_list, tile_count, 0, EPI_PLAIN,
                    nullptr, nullptr, s);
    launch_unpack(c.t, c.tree, g, C, nullptr, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error_message((std::string("kernel launch: ") + cudaGetErrorString(e)).c_str());
        return SPAMM_ERR_CUDA;
    }
    return SPAMM_OK;
}
