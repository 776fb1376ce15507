// Contraction dispatch and optional-state hooks of the context.
#include "polybin_internal.h"

namespace pb {

void destroy_extras(polybin_ctx* ctx) {
    destroy_unwindowed(ctx);
    destroy_multi(ctx);
    destroy_tc(ctx);
    if (ctx->d_err) cudaFree(ctx->d_err);
    ctx->d_err = nullptr;
    if (ctx->d_S) cudaFree(ctx->d_S);
    ctx->d_S = nullptr;
    if (ctx->d_trip_m) cudaFree(ctx->d_trip_m);
    ctx->d_trip_m = nullptr;
}

// POLYBIN_SPLIT_TF32X3 runs the tensor-core kernel whenever its shape limits hold (<= 512 pairs, <= 32 singles,
// aligned maps); other shapes and the FP32 mode run the SIMT kernel.
template <>
int run_contract_any<float>(polybin_ctx* ctx, const float* g, int ng, const float* h, int nh, double* part, size_t cap,
                            double* out) {
    const int nhh = h ? nh : ng;
    if (ctx->prec == POLYBIN_SPLIT_TF32X3 && tc_shape_ok(ctx, g, ng, h, nhh))
        return run_contract_tc(ctx, g, ng, h, nh, part, cap, out);
    return run_contract<float>(ctx, g, ng, h, nh, part, cap, out);
}

// S[t] = M[m[t]]: the closed-triplet entries of a pair-major contraction.
static __global__ void k_gather_triplets(const double* __restrict__ M, const int* __restrict__ m, int nt,
                                         double* __restrict__ S) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt) S[t] = M[m[t]];
}

template <typename T>
static int triplet_sums_from_pairs(polybin_ctx* ctx, const T* g, double* d_S) {
    const int nb = ctx->nb, nt = (int)ctx->Nabc.size();
    Work& w = ctx->w;
    int rc = run_contract_any<T>(ctx, g, nb, nullptr, nb, w.partial, w.partial_cap, w.mout);
    if (rc) return rc;
    k_gather_triplets<<<(nt + 255) / 256, 256, 0, ctx->stream>>>(w.mout, ctx->d_trip_m, nt, d_S);
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(ctx, e, "k_gather_triplets", __FILE__, __LINE__);
    return POLYBIN_OK;
}

// The split-TF32 mode contracts only the pairs and singles of closed triplets on the tensor cores.
template <>
int run_triplet_sums<float>(polybin_ctx* ctx, const float* g, double* d_S) {
    if (ctx->Nabc.empty()) return POLYBIN_OK;
    if (ctx->prec == POLYBIN_SPLIT_TF32X3 && tc_shape_ok(ctx, g, ctx->nb, nullptr, ctx->nb))
        return run_triplet_sums_tc(ctx, g, d_S);
    return triplet_sums_from_pairs<float>(ctx, g, d_S);
}

template <>
int run_triplet_sums<double>(polybin_ctx* ctx, const double* g, double* d_S) {
    if (ctx->Nabc.empty()) return POLYBIN_OK;
    return triplet_sums_from_pairs<double>(ctx, g, d_S);
}

}  // namespace pb
