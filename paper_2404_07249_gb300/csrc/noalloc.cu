// Allocation-free variant of the triplet contraction, for callers that cannot allocate device memory: code
// running inside a caller-managed memory pool or arena, plugins whose host application owns every allocation,
// or threads that must not call cudaMalloc/cudaFree (which can synchronise the device).  It computes the same
// M[(j<=k)][i] = sum_x g_j(x) g_k(x) h_i(x) as polybin_contract with the FP32 SIMT kernel, but its per-CTA
// partial sums and its pair table live in file-scope __device__ arrays instead of context-owned allocations.
//
// The arrays occupy kScratchDoubles * 8 bytes (16 MiB) plus 8 KiB on every GPU that loads the library, until the
// process exits.  Host code must not pass the array names to a kernel (in host code they are stand-ins, not device
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
constexpr int kPairTable = kMaxMaps * (kMaxMaps + 1) / 2;   // pairs of up to 64 maps

static __device__ __align__(256) double g_scratch[kScratchDoubles];
static __device__ __align__(256) short2 g_pairs[kPairTable];

static thread_local std::string g_error;

struct DeviceSlot {
    bool ready = false;
    double* scratch = nullptr;
    short2* pairs = nullptr;
    int pairs_n = 0;          // the pair table currently holds the pairs of pairs_n maps
};

static std::mutex g_mutex;
static DeviceSlot g_slots[256];

static __global__ void k_fill_pairs(short2* pairs, int n) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int np = n * (n + 1) / 2;
    if (p >= np) return;
    int j = 0, rem = p;
    while (rem >= n - j) { rem -= n - j; ++j; }
    pairs[p] = make_short2((short)j, (short)(j + rem));
}

static int set_error(int status, const std::string& msg) {
    g_error = msg;
    return status;
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
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256)
        return set_error(POLYBIN_ECUDA, std::string("polybin_contract_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
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
            slot->ready = true;
        }
        if (slot->pairs_n != n_g) {
            const int np = n_g * (n_g + 1) / 2;
            k_fill_pairs<<<(np + 255) / 256, 256, 0, st>>>(slot->pairs, n_g);
            e = cudaGetLastError();
            if (e != cudaSuccess)
                return set_error(POLYBIN_ECUDA, std::string("polybin_contract_noalloc: pair table: ") + cudaGetErrorString(e));
            slot->pairs_n = n_g;
        }
    }
    const size_t sm = ((size_t)kCH * G.rows_cta + (size_t)kCH * G.nhp + (size_t)n_g * (kCH + 1)) * sizeof(float) + 16;
    if (sm > 48 * 1024) {
        e = cudaFuncSetAttribute((const void*)k_contract<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return set_error(POLYBIN_ECUDA, std::string("polybin_contract_noalloc: ") + cudaGetErrorString(e));
    }
    k_contract<float><<<dim3(G.ngroups, G.ncb, 1), 256, sm, st>>>(g, h, (long)ncell, slot->pairs, G, slot->scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(POLYBIN_ECUDA, std::string("polybin_contract_noalloc: ") + cudaGetErrorString(e));
    k_reduce_partials<<<(unsigned)((per_cb + 255) / 256), 256, 0, st>>>(slot->scratch, G.ncb, per_cb, m_out_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(POLYBIN_ECUDA, std::string("polybin_contract_noalloc: ") + cudaGetErrorString(e));
    return POLYBIN_OK;
}
