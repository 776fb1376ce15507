// Contraction dispatch and optional-state hooks of the context.
#include "polybin_internal.h"

namespace pb {

bool split_tc_available() { return false; }

void destroy_extras(polybin_ctx*) {}

template <>
int run_contract_any<float>(polybin_ctx* ctx, const float* g, int ng, const float* h, int nh, double* part, size_t cap,
                            double* out) {
    return run_contract<float>(ctx, g, ng, h, nh, part, cap, out);
}

}  // namespace pb
