// Contraction dispatch and optional-state hooks of the context.
#include "polybin_internal.h"

namespace pb {

void destroy_extras(polybin_ctx* ctx) {
    destroy_unwindowed(ctx);
    destroy_multi(ctx);
    if (ctx->d_err) cudaFree(ctx->d_err);
    ctx->d_err = nullptr;
}

// POLYBIN_SPLIT_TF32X3 runs the tensor-core kernel whenever its tile limits hold (<= 512 pairs, <= 32 singles);
// other shapes and the FP32 mode run the SIMT kernel.
template <>
int run_contract_any<float>(polybin_ctx* ctx, const float* g, int ng, const float* h, int nh, double* part, size_t cap,
                            double* out) {
    const int nhh = h ? nh : ng;
    if (ctx->prec == POLYBIN_SPLIT_TF32X3 && ng * (ng + 1) / 2 <= 512 && nhh <= 32)
        return run_contract_tc(ctx, g, ng, h, nh, part, cap, out);
    return run_contract<float>(ctx, g, ng, h, nh, part, cap, out);
}

}  // namespace pb
