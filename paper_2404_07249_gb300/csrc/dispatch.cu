// Contraction dispatch and optional-state hooks of the context, and the closed-triplet (pruned) SIMT plans of the
// FP32 and FP64 modes.
#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "polybin_internal.h"

namespace pb {

// Pruned SIMT contraction of the closed triplets: the pair rows that some closed triplet needs, cut into groups of
// consecutive rows (sorted by their window of singles) by dynamic programming on rows x window width; group i runs
// the SIMT kernel on its own pair table against the singles [s0, s0 + W) only, and a gather picks every triplet's
// entry.  This is the same work the tensor-core plan does (pairs and windows of closed triplets), on the FP32/FP64
// pipes.
struct SimtGroup {
    int pair_off, npairs, s0, W;
    long out_off;
};
struct SimtPlan {
    std::vector<SimtGroup> groups;
    short2* d_pairs = nullptr;
    int* d_gidx = nullptr;      // triplet -> index into d_M
    double* d_M = nullptr;      // concatenated group outputs [npairs_i][W_i]
    long nM = 0;
};
struct SimtPlans {
    SimtPlan kind[2];           // 0: pair (b, c), single a (ell = 0); 1: pair (a, b), single c from the ell maps
};

static void free_simt(SimtPlans* sp) {
    if (!sp) return;
    for (SimtPlan& p : sp->kind) {
        if (p.d_pairs) cudaFree(p.d_pairs);
        if (p.d_gidx) cudaFree(p.d_gidx);
        if (p.d_M) cudaFree(p.d_M);
    }
    delete sp;
}

struct RowNeed {
    int j, k, lo, hi;
    std::vector<std::pair<int, int>> outs;   // (single, triplet)
};

static int build_simt_plan(polybin_ctx* ctx, int kind, SimtPlan& pl) {
    const int nt = (int)ctx->Nabc.size();
    std::map<std::pair<int, int>, RowNeed> m;
    for (int t = 0; t < nt; ++t) {
        const int a = ctx->trip[3 * t], b = ctx->trip[3 * t + 1], c = ctx->trip[3 * t + 2];
        const int j = kind == 0 ? b : a, k = kind == 0 ? c : b, sgl = kind == 0 ? a : c;
        auto f = m.find({j, k});
        if (f == m.end()) f = m.emplace(std::make_pair(j, k), RowNeed{j, k, sgl, sgl, {}}).first;
        f->second.lo = std::min(f->second.lo, sgl);
        f->second.hi = std::max(f->second.hi, sgl);
        f->second.outs.push_back({sgl, t});
    }
    std::vector<RowNeed> rows;
    for (auto& kv : m) rows.push_back(std::move(kv.second));
    std::stable_sort(rows.begin(), rows.end(),
                     [](const RowNeed& x, const RowNeed& y) { return std::tie(x.hi, x.lo) < std::tie(y.hi, y.lo); });
    // groups of <= 256 consecutive rows minimising sum rows x ceil8(W) + 1024: a group re-stages every map for each
    // chunk of cells, which costs about as much as 1024 row x single products (measured: 26 groups at a cost of 32
    // ran slower than the unpruned contraction; 2-3 groups at 1024 do 2.5x less work than it)
    const int n = (int)rows.size();
    std::vector<long> f(n + 1, (long)1 << 50);
    std::vector<int> arg(n + 1, 0);
    f[0] = 0;
    for (int i = 1; i <= n; ++i) {
        int lo = 1 << 30, hi = -1;
        for (int j = i - 1; j >= 0 && j >= i - 256; --j) {
            lo = std::min(lo, rows[j].lo);
            hi = std::max(hi, rows[j].hi);
            const long c = f[j] + (long)(i - j) * ((hi - lo + 1 + 7) / 8 * 8) + 1024;
            if (c < f[i]) { f[i] = c; arg[i] = j; }
        }
    }
    std::vector<std::pair<int, int>> seg;
    for (int i = n; i > 0; i = arg[i]) seg.push_back({arg[i], i});
    std::reverse(seg.begin(), seg.end());
    std::vector<short2> tab;
    std::vector<int> gidx(std::max(nt, 1), 0);
    long off = 0;
    for (auto& sg : seg) {
        SimtGroup G;
        int lo = 1 << 30, hi = -1;
        for (int i = sg.first; i < sg.second; ++i) { lo = std::min(lo, rows[i].lo); hi = std::max(hi, rows[i].hi); }
        G.pair_off = (int)tab.size();
        G.npairs = sg.second - sg.first;
        G.s0 = lo;
        G.W = hi - lo + 1;
        G.out_off = off;
        for (int i = sg.first; i < sg.second; ++i) {
            const int r = i - sg.first;
            tab.push_back(make_short2((short)rows[i].j, (short)rows[i].k));
            for (auto& so : rows[i].outs) gidx[so.second] = (int)(off + (long)r * G.W + (so.first - lo));
        }
        off += (long)G.npairs * G.W;
        pl.groups.push_back(G);
    }
    pl.nM = std::max(off, 1L);
    PB_CUDA_OK(cudaMalloc(&pl.d_pairs, sizeof(short2) * std::max<size_t>(tab.size(), 1)));
    PB_CUDA_OK(cudaMalloc(&pl.d_gidx, sizeof(int) * gidx.size()));
    PB_CUDA_OK(cudaMalloc(&pl.d_M, sizeof(double) * pl.nM));
    if (!tab.empty()) PB_CUDA_OK(cudaMemcpy(pl.d_pairs, tab.data(), sizeof(short2) * tab.size(), cudaMemcpyHostToDevice));
    PB_CUDA_OK(cudaMemcpy(pl.d_gidx, gidx.data(), sizeof(int) * gidx.size(), cudaMemcpyHostToDevice));
    return POLYBIN_OK;
}

// SIMT geometry for an explicit pair table of npairs rows against nh singles over ncell cells.
static ContractGeom geom_rows(int nb, int npairs, int nh, long ncell) {
    ContractGeom G;
    G.nb = nb; G.nh = nh; G.npairs = npairs;
    G.ct = (nh + kTN - 1) / kTN;
    G.rt = 256 / G.ct;
    const int need = (npairs + kTM - 1) / kTM * kTM;
    G.rows_cta = std::min(G.rt * kTM, need);
    G.nhp = G.ct * kTN;
    G.ngroups = (npairs + G.rows_cta - 1) / G.rows_cta;
    const long nchunks = (ncell + kCH - 1) / kCH;
    long ncb = std::max(1L, std::min(nchunks, (long)(4 * 152 / G.ngroups)));
    G.cells_cta = ((ncell + ncb - 1) / ncb + kCH - 1) / kCH * kCH;
    G.ncb = (int)((ncell + G.cells_cta - 1) / G.cells_cta);
    return G;
}

__global__ void k_gather_triplets(const double* __restrict__ M, const int* __restrict__ m, int nt,
                                  double* __restrict__ S);

// Closed-triplet sums with the SIMT kernel: kind 0 from g alone (S'_abc), kind 1 with the singles from h (S^ell').
template <typename T>
static int simt_triplet_sums(polybin_ctx* ctx, int kind, const T* g, const T* h, double* d_S) {
    SimtPlans*& sp = reinterpret_cast<SimtPlans*&>(ctx->simt);
    if (!sp) {
        sp = new (std::nothrow) SimtPlans();
        if (!sp) return fail(ctx, POLYBIN_ENOMEM, "simt plans: out of host memory");
    }
    SimtPlan& pl = sp->kind[kind];
    int rc;
    if (!pl.d_M && (rc = build_simt_plan(ctx, kind, pl))) return rc;
    const int nb = ctx->nb, nt = (int)ctx->Nabc.size();
    const long ncell = ctx->cg.ncell;
    Work& w = ctx->w;
    {
        StageTimer timer(ctx, kStageContract);
        for (const SimtGroup& Gp : pl.groups) {
            ContractGeom G = geom_rows(nb, Gp.npairs, Gp.W, ncell);
            if ((size_t)G.ncb * G.npairs * G.nh > w.partial_cap)
                return fail(ctx, POLYBIN_EINVAL, "contract: partial buffer too small");
            const size_t sm = ((size_t)kCH * G.rows_cta + (size_t)kCH * G.nhp + (size_t)nb * (kCH + 1)) * sizeof(T) + 16;
            if (sm > 48 * 1024) {
                cudaError_t e = cudaFuncSetAttribute((const void*)k_contract<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)sm);
                if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaFuncSetAttribute", __FILE__, __LINE__);
            }
            const T* hs = (kind == 0 ? g : h) + (size_t)Gp.s0 * ncell;
            k_contract<T><<<dim3(G.ngroups, G.ncb, 1), 256, sm, ctx->stream>>>(g, hs, ncell, pl.d_pairs + Gp.pair_off, G,
                                                                             w.partial);
            const long nout = (long)G.npairs * G.nh;
            k_reduce_partials<<<(unsigned)((nout + 255) / 256), 256, 0, ctx->stream>>>(w.partial, G.ncb, nout,
                                                                                       pl.d_M + Gp.out_off);
            ctx->launches += 2;
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return fail_cuda(ctx, e, "k_contract (pruned)", __FILE__, __LINE__);
        }
    }
    k_gather_triplets<<<(nt + 255) / 256, 256, 0, ctx->stream>>>(pl.d_M, pl.d_gidx, nt, d_S);
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(ctx, e, "k_gather_triplets", __FILE__, __LINE__);
    return POLYBIN_OK;
}

void destroy_extras(polybin_ctx* ctx) {
    free_simt(reinterpret_cast<SimtPlans*>(ctx->simt));
    ctx->simt = nullptr;
    destroy_unwindowed(ctx);
    destroy_optimal(ctx);
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
__global__ void k_gather_triplets(const double* __restrict__ M, const int* __restrict__ m, int nt,
                                         double* __restrict__ S) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt) S[t] = M[m[t]];
}

// The split-TF32 mode contracts only the pairs and singles of closed triplets on the tensor cores.
template <>
int run_triplet_sums<float>(polybin_ctx* ctx, const float* g, double* d_S) {
    if (ctx->Nabc.empty()) return POLYBIN_OK;
    if (ctx->prec == POLYBIN_SPLIT_TF32X3 && tc_shape_ok(ctx->cg.ncell, g, ctx->nb, nullptr, ctx->nb)) {
        ctx->last_path = POLYBIN_PATH_TENSOR_SPLIT_TF32X3;
        return run_triplet_sums_tc(ctx, g, d_S);
    }
    ctx->last_path = POLYBIN_PATH_SIMT_FP32;
    return simt_triplet_sums<float>(ctx, 0, g, nullptr, d_S);
}

template <>
int run_triplet_sums_ell<float>(polybin_ctx* ctx, const float* g, const float* gl, double* d_S) {
    if (ctx->Nabc.empty()) return POLYBIN_OK;
    if (ctx->prec == POLYBIN_SPLIT_TF32X3 && tc_shape_ok(ctx->cg.ncell, g, ctx->nb, gl, ctx->nb)) {
        ctx->last_path = POLYBIN_PATH_TENSOR_SPLIT_TF32X3;
        return run_triplet_sums_ell_tc(ctx, g, gl, d_S);
    }
    ctx->last_path = POLYBIN_PATH_SIMT_FP32;
    return simt_triplet_sums<float>(ctx, 1, g, gl, d_S);
}

template <>
int run_triplet_sums_ell<double>(polybin_ctx* ctx, const double* g, const double* gl, double* d_S) {
    if (ctx->Nabc.empty()) return POLYBIN_OK;
    ctx->last_path = POLYBIN_PATH_SIMT_FP64;
    return simt_triplet_sums<double>(ctx, 1, g, gl, d_S);
}

template <>
int run_triplet_sums<double>(polybin_ctx* ctx, const double* g, double* d_S) {
    if (ctx->Nabc.empty()) return POLYBIN_OK;
    ctx->last_path = POLYBIN_PATH_SIMT_FP64;
    return simt_triplet_sums<double>(ctx, 0, g, nullptr, d_S);
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
