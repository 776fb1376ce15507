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
    if (ctx->d_B) cudaFree(ctx->d_B);
    ctx->d_B = nullptr;
    if (ctx->d_T) cudaFree(ctx->d_T);
    ctx->d_T = nullptr;
    if (ctx->d_trip_m) cudaFree(ctx->d_trip_m);
    ctx->d_trip_m = nullptr;
}

// POLYBIN_SPLIT_TF32X3 runs the tensor-core kernel whenever its shape limits hold (<= 512 pairs, <= 32 singles,
// aligned maps); other shapes and the FP32 mode run the SIMT kernel.  The path taken is recorded in the context
// (polybin_last_path).
template <>
int run_contract_any<float>(polybin_ctx* ctx, const float* g, int ng, const float* h, int nh, double* part, size_t cap,
                            double* out, long ncell) {
    const int nhh = h ? nh : ng;
    if (ctx->prec == POLYBIN_SPLIT_TF32X3 && tc_shape_ok(ncell, g, ng, h, nhh)) {
        ctx->last_path = POLYBIN_PATH_TENSOR_SPLIT_TF32X3;
        return run_contract_tc(ctx, g, ng, h, nh, out, ncell);
    }
    ctx->last_path = POLYBIN_PATH_SIMT_FP32;
    return run_contract<float>(ctx, g, ng, h, nh, part, cap, out, ncell);
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
    int rc = run_contract_any<T>(ctx, g, nb, nullptr, nb, w.partial, w.partial_cap, w.mout, ctx->cg.ncell);
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
    if (ctx->prec == POLYBIN_SPLIT_TF32X3 && tc_shape_ok(ctx->cg.ncell, g, ctx->nb, nullptr, ctx->nb)) {
        ctx->last_path = POLYBIN_PATH_TENSOR_SPLIT_TF32X3;
        return run_triplet_sums_tc(ctx, g, d_S);
    }
    return triplet_sums_from_pairs<float>(ctx, g, d_S);
}

// S^ell' from pairs of the g maps and singles of the Legendre-weighted maps gl (M[(a <= b)][c], gathered).
template <typename T>
static int triplet_sums_ell_from_pairs(polybin_ctx* ctx, const T* g, const T* gl, double* d_S) {
    const int nb = ctx->nb, nt = (int)ctx->Nabc.size();
    Work& w = ctx->w;
    int rc = run_contract_any<T>(ctx, g, nb, gl, nb, w.partial, w.partial_cap, w.mout, ctx->cg.ncell);
    if (rc) return rc;
    k_gather_triplets<<<(nt + 255) / 256, 256, 0, ctx->stream>>>(w.mout, ctx->d_trip_m, nt, d_S);
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(ctx, e, "k_gather_triplets", __FILE__, __LINE__);
    return POLYBIN_OK;
}

template <>
int run_triplet_sums_ell<float>(polybin_ctx* ctx, const float* g, const float* gl, double* d_S) {
    if (ctx->Nabc.empty()) return POLYBIN_OK;
    if (ctx->prec == POLYBIN_SPLIT_TF32X3 && tc_shape_ok(ctx->cg.ncell, g, ctx->nb, gl, ctx->nb)) {
        ctx->last_path = POLYBIN_PATH_TENSOR_SPLIT_TF32X3;
        return run_triplet_sums_ell_tc(ctx, g, gl, d_S);
    }
    return triplet_sums_ell_from_pairs<float>(ctx, g, gl, d_S);
}

template <>
int run_triplet_sums_ell<double>(polybin_ctx* ctx, const double* g, const double* gl, double* d_S) {
    if (ctx->Nabc.empty()) return POLYBIN_OK;
    ctx->last_path = POLYBIN_PATH_SIMT_FP64;
    return triplet_sums_ell_from_pairs<double>(ctx, g, gl, d_S);
}

template <>
int run_triplet_sums<double>(polybin_ctx* ctx, const double* g, double* d_S) {
    if (ctx->Nabc.empty()) return POLYBIN_OK;
    ctx->last_path = POLYBIN_PATH_SIMT_FP64;
    return triplet_sums_from_pairs<double>(ctx, g, d_S);
}

// B[t] = scale S[t] / T[t] (FP64).
static __global__ void k_bk_normalise(const double* __restrict__ S, const double* __restrict__ T, int nt, double scale,
                                      double* __restrict__ B) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt) B[t] = scale * S[t] / T[t];
}

int run_bk_normalise(polybin_ctx* ctx, const double* d_S, double* d_B, double fac) {
    const int nt = (int)ctx->Nabc.size();
    if (nt == 0) return POLYBIN_OK;
    const double n = (double)ctx->ncell;
    const double scale = fac * (ctx->vol * ctx->vol / (n * n * n)) * ctx->cg_ratio;
    k_bk_normalise<<<(nt + 255) / 256, 256, 0, ctx->stream>>>(d_S, ctx->d_T, nt, scale, d_B);
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(ctx, e, "k_bk_normalise", __FILE__, __LINE__);
    return POLYBIN_OK;
}

// P[l][b] = (4 l + 1) scale sum_seg part[b][seg][l] / counts[b] (segments summed in order; NaN for an empty bin).
static __global__ void k_pk_normalise(const double* __restrict__ part, int nb, int nseg, int nell,
                                      const double* __restrict__ counts, double scale, double* __restrict__ P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * nell) return;
    const int l = i / nb, b = i - l * nb;
    double s = 0.0;
    for (int q = 0; q < nseg; ++q) s += part[((long)b * nseg + q) * nell + l];
    P[i] = counts[b] > 0 ? (4 * l + 1) * scale * s / counts[b] : __longlong_as_double(0x7ff8000000000000LL);
}

int run_pk_normalise(polybin_ctx* ctx, double* d_P) {
    const int n = ctx->nb * ctx->nell;
    const double N = (double)ctx->ncell;
    k_pk_normalise<<<(n + 127) / 128, 128, 0, ctx->stream>>>(ctx->d_pkpart, ctx->nb, ctx->pk_nseg, ctx->nell,
                                                             ctx->d_counts, ctx->vol / (N * N), d_P);
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(ctx, e, "k_pk_normalise", __FILE__, __LINE__);
    return POLYBIN_OK;
}

}  // namespace pb

extern "C" int polybin_last_path(const polybin_ctx* ctx, int* path) {
    if (!ctx || !path) return pb::fail(const_cast<polybin_ctx*>(ctx), POLYBIN_EINVAL, "polybin_last_path: NULL argument");
    *path = ctx->last_path;
    return POLYBIN_OK;
}

extern "C" int polybin_contraction_grid(const polybin_ctx* ctx, int dims[3]) {
    if (!ctx || !dims) return pb::fail(const_cast<polybin_ctx*>(ctx), POLYBIN_EINVAL, "polybin_contraction_grid: NULL argument");
    for (int a = 0; a < 3; ++a) dims[a] = ctx->cg.N[a];
    return POLYBIN_OK;
}
