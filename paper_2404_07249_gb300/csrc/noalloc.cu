// Allocation-free variant of the triplet contraction, for callers that cannot allocate device memory: code
// running inside a caller-managed memory pool or arena, plugins whose host application owns every allocation,
// or threads that must not call cudaMalloc/cudaFree (which can synchronise the device).  It computes the same
// M[(j<=k)][i] = sum_x g_j(x) g_k(x) h_i(x) as polybin_contract with the FP32 SIMT kernel, but its per-CTA
// partial sums and its pair table live in file-scope __device__ arrays instead of context-owned allocations.
//
// The arrays occupy kScratchDoubles * 8 bytes (16 MiB) plus the pair tables of every n <= 64 maps (45,760 entries,
// 179 KiB) on every GPU that loads the library, until the process exits.  Host code must not pass the array names to a kernel (in host code they are stand-ins, not device
// addresses): their device addresses are looked up with cudaGetSymbolAddress once per device.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "polybin_internal.h"

namespace pb {
namespace noalloc {

constexpr long kScratchDoubles = 2L * 1024 * 1024;          // 16 MiB of FP64 partial sums
constexpr int kMaxMaps = 64;
// pair tables of every n = 1 .. 64 back to back, table n at pairs_offset(n): sum_{n <= 64} n (n + 1) / 2 entries
constexpr long kPairTables = (long)kMaxMaps * (kMaxMaps + 1) * (kMaxMaps + 2) / 6;

static __device__ __align__(256) double g_scratch[kScratchDoubles];
static __device__ __align__(256) short2 g_pairs[kPairTables];

static thread_local std::string g_error;

// Per device: the looked-up addresses of the two arrays; `ready` once the pair tables have been filled (the fill
// runs once, on the first call, and is complete before that call returns).
struct DeviceSlot {
    bool ready = false;
    double* scratch = nullptr;
    short2* pairs = nullptr;
};

static std::mutex g_mutex;
constexpr int kMaxDevices = 256;
static DeviceSlot g_slots[kMaxDevices];

// Entry p of the table of n maps (p < n (n + 1) / 2) is the p-th pair (j <= k) in lexicographic order.
static __global__ void k_fill_pair_tables(short2* pairs) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kPairTables) return;
    int n = 1;
    while (pairs_offset(n + 1) <= i) ++n;
    int rem = (int)(i - pairs_offset(n)), j = 0;
    while (rem >= n - j) { rem -= n - j; ++j; }
    pairs[i] = make_short2((short)j, (short)(j + rem));
}

static int set_error(int status, const std::string& msg) {
    g_error = msg;
    return status;
}

// True when p is device (or managed) memory of the current device's address space.
static bool device_pointer(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace noalloc
}  // namespace pb

using namespace pb;

extern "C" const char* polybin_contract_noalloc_error(void) { return noalloc::g_error.c_str(); }

extern "C" int polybin_contract_noalloc(const float* g, int n_g, const float* h, int n_h, long long ncell,
                                        double* m_out_dev, void* cuda_stream) {
    using namespace noalloc;
    if (!g || !m_out_dev || ncell < 1) return set_error(POLYBIN_EINVAL, "polybin_contract_noalloc: NULL or empty argument");
    if (!h) n_h = n_g;
    if (n_g < 1 || n_g > kMaxMaps || n_h < 1 || n_h > kMaxMaps)
        return set_error(POLYBIN_EINVAL, "polybin_contract_noalloc: 1 <= n_g, n_h <= 64");
    if (!device_pointer(g) || (h && !device_pointer(h)) || !device_pointer(m_out_dev))
        return set_error(POLYBIN_EINVAL, "polybin_contract_noalloc: g, h and m_out_dev must be device memory");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return set_error(POLYBIN_ECUDA, std::string("polybin_contract_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(POLYBIN_EINVAL, "polybin_contract_noalloc: device index " + std::to_string(dev) +
                                             " beyond the 256 devices this entry point keeps state for");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    ContractGeom G = contract_geom(n_g, n_h, (long)ncell);
    const long per_cb = (long)G.npairs * G.nh;
    if (per_cb > kScratchDoubles)
        return set_error(POLYBIN_EINVAL, "polybin_contract_noalloc: n_g (n_g + 1) / 2 * n_h exceeds the 2^21-double scratch");
    if ((long)G.ncb * per_cb > kScratchDoubles) {
        // fewer, longer cell blocks so that the partial sums fit the fixed scratch array
        const long ncb = std::max(1L, kScratchDoubles / per_cb);
        G.cells_cta = ((ncell + ncb - 1) / ncb + kCH - 1) / kCH * kCH;
        G.ncb = (int)((ncell + G.cells_cta - 1) / G.cells_cta);
    }
    DeviceSlot* slot = &g_slots[dev];
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!slot->ready) {
            e = cudaGetSymbolAddress((void**)&slot->scratch, g_scratch);
            if (e != cudaSuccess)
                return set_error(POLYBIN_ECUDA, std::string("polybin_contract_noalloc: cudaGetSymbolAddress(scratch): ") +
                                                    cudaGetErrorString(e));
            e = cudaGetSymbolAddress((void**)&slot->pairs, g_pairs);
            if (e != cudaSuccess)
                return set_error(POLYBIN_ECUDA, std::string("polybin_contract_noalloc: cudaGetSymbolAddress(pairs): ") +
                                                    cudaGetErrorString(e));
            // all 64 pair tables at once, finished before this first call goes on: later calls, on any stream,
            // read them without depending on anything the host remembers
            k_fill_pair_tables<<<(unsigned)((kPairTables + 255) / 256), 256, 0, st>>>(slot->pairs);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess)
                return set_error(POLYBIN_ECUDA, std::string("polybin_contract_noalloc: pair tables: ") + cudaGetErrorString(e));
            slot->ready = true;
        }
    }
    const size_t sm = ((size_t)kCH * G.rows_cta + (size_t)kCH * G.nhp + (size_t)n_g * (kCH + 1)) * sizeof(float) + 16;
    if (sm > 48 * 1024) {
        e = cudaFuncSetAttribute((const void*)k_contract<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return set_error(POLYBIN_ECUDA, std::string("polybin_contract_noalloc: ") + cudaGetErrorString(e));
    }
    k_contract<float><<<dim3(G.ngroups, G.ncb, 1), 256, sm, st>>>(g, h, (long)ncell, slot->pairs + pairs_offset(n_g), G,
                                                                 slot->scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(POLYBIN_ECUDA, std::string("polybin_contract_noalloc: ") + cudaGetErrorString(e));
    k_reduce_partials<<<(unsigned)((per_cb + 255) / 256), 256, 0, st>>>(slot->scratch, G.ncb, per_cb, m_out_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(POLYBIN_ECUDA, std::string("polybin_contract_noalloc: ") + cudaGetErrorString(e));
    return POLYBIN_OK;
}
