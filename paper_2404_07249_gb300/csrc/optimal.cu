// Optimal weighting S^-1 by preconditioned conjugate gradients (Sec. 2.4, eq. cgd-operation-eqn and the transpose
// equation beside it; Sec. 3.3.3, eq. Sinv-optimal in the distant-observer limit).
//
// Data model d = n delta + eps with C = P xi P^T + N, P = diag(n), N = diag(n2), xi = IFT[P(k) FT[.]],
// P(k) = sum_ell P_ell(k) L_ell(mu) about the global line of sight.  On the cells with n_w > 0 (Phi = 1) the
// distant-observer equation n IFT[P FT[Phi S^-1 v]] + (n2 / n) Phi S^-1 v = v, divided by n, is A u = v / n with
//     A = Phi (K + D) Phi,   K = IFT[P FT[.]],   D = n2_w / n_w^2,
// symmetric positive definite on the subspace.  With G = A^-1 there (0 off it):
//     S^-1 v = G (v / n_w),     S^-T v = G (v) / n_w.
// Discretised, int dy int_k e^{ik(x-y)} P(k) u(y) is exactly IFT[P FT[u]] with the unnormalised forward DFT and the
// 1/N inverse, so n_w, n2_w are densities and P a power in the matching units (n P dimensionless).
//
// The fiducial P_ell are given on the integer shells |n|^2 = s < n_s <= smax + 1 (smax: the largest binned |n|^2) and
// vanish beyond, so K acts only on the box of wave numbers |n_i| <= m that the pruned transforms produce
// (run_forward / run_inverse_box).  Preconditioner: the ideal weighting of eq. Sinv-ideal, the exact inverse for a
// uniform density, with noise level sigma = mean of D over the cells with n_w > 0:
//     M^-1 r = Phi IFT[FT[Phi r] / (P + sigma)] = Phi (r / sigma + IFT_box[h FT_box[r]]),  h = 1/(P + sigma) - 1/sigma,
// h vanishing wherever P does, so this too needs the box only.
//
// One iteration: two pruned forward transforms, two pruned inverse transforms, two box multiplies and four map
// kernels.  Dot products are FP64: per-block partials summed in a fixed order by the last block to finish
// (deterministic, no extra launch).  Step lengths are read from device memory by the update kernels, so the loop has
// no host round trip; with tol > 0 the host reads ||r||^2 after each iteration to stop early.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "polybin_internal.h"

namespace pb {
namespace opt {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 152 * 8;
// device scalar slots
enum { kBB = 0, kPQ = 1, kRR = 2, kRZ0 = 3, kRZ1 = 4, kDsum = 5, kDcnt = 6, kSlots = 8 };

// Per-thread accumulator of a dot product: FP64 for FP64 maps; for FP32 maps compensated (Kahan) FP32 sums, which keep
// the per-thread error at the FP32 rounding of one term while staying off the FP64 pipe (a small fraction of the FP32
// rate on this part: an FP64 multiply-add plus two conversions per element made these kernels arithmetic-bound).
template <typename T>
struct Acc {
    double s = 0.0;
    __device__ __forceinline__ void add(T x) { s += (double)x; }
    __device__ __forceinline__ double get() const { return s; }
};
template <>
struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sums of NV values -> part[j * gridDim.x + block]; the last block to arrive sums the partials of each value
// in block order into dst[slot[j]] and re-arms the counter.
template <int NV>
__device__ void reduce_to(const double (&v)[NV], double* part, double* dst, const int (&slot)[NV], unsigned* counter) {
    __shared__ double sh[NV][kThreads / 32];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const double s = warp_sum(v[j]);
        if (lane == 0) sh[j][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double s = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) s += sh[j][w];
            part[(size_t)j * gridDim.x + blockIdx.x] = s;
        }
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        double s = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) s += __ldcg(part + (size_t)j * gridDim.x + b);
        s = warp_sum(s);
        __syncthreads();
        if (lane == 0) sh[j][warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += sh[j][w];
            dst[slot[j]] = t;
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// Dm = n2_w / n_w^2 on the cells with n_w > 0, -1 elsewhere (Phi = Dm >= 0); sums of D and of the cell count.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dmap(const float* __restrict__ nw, const float* __restrict__ n2w,
                                                   T* __restrict__ Dm, long N, double* part, double* sc,
                                                   unsigned* counter) {
    double v[2] = {0.0, 0.0};
    for (long i = (long)blockIdx.x * kThreads + threadIdx.x; i < N; i += (long)gridDim.x * kThreads) {
        const float n = nw[i];
        if (n > 0.f) {
            const double d = (double)n2w[i] / ((double)n * (double)n);
            Dm[i] = T(d);
            v[0] += d;
            v[1] += 1.0;
        } else {
            Dm[i] = T(-1);
        }
    }
    const int slot[2] = {kDsum, kDcnt};
    reduce_to<2>(v, part, sc, slot, counter);
}

// r = Phi pre v (/ n_w), x = 0; ||r||^2 -> sc[kBB].
template <typename T, typename TIN>
__global__ void __launch_bounds__(kThreads) k_init(const TIN* __restrict__ v, const float* __restrict__ pre, int pre_div,
                                                   const float* __restrict__ nw, const T* __restrict__ Dm,
                                                   T* __restrict__ r, T* __restrict__ x, long N, double* part, double* sc,
                                                   unsigned* counter) {
    Acc<T> acc;
    for (long i = (long)blockIdx.x * kThreads + threadIdx.x; i < N; i += (long)gridDim.x * kThreads) {
        T ri = T(0);
        if (Dm[i] >= T(0)) {
            ri = T(v[i]);
            if (pre) ri *= T(pre[i]);
            if (pre_div) ri /= T(nw[i]);
        }
        r[i] = ri;
        x[i] = T(0);
        acc.add(ri * ri);
    }
    const double v2[1] = {acc.get()};
    const int slot[1] = {kBB};
    reduce_to<1>(v2, part, sc, slot, counter);
}

template <typename T>
__global__ void k_box_mul(C<T>* __restrict__ box, const T* __restrict__ w, long nbox) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nbox; i += (long)gridDim.x * blockDim.x) {
        const T f = w[i];
        C<T> c = box[i];
        c.x *= f;
        c.y *= f;
        box[i] = c;
    }
}

// q = Phi (y + D p); p.q -> sc[kPQ].
template <typename T>
__global__ void __launch_bounds__(kThreads) k_op_post(const T* __restrict__ y, const T* __restrict__ p,
                                                      const T* __restrict__ Dm, T* __restrict__ q, long N,
                                                      double* part, double* sc, unsigned* counter) {
    Acc<T> acc;
    for (long i = (long)blockIdx.x * kThreads + threadIdx.x; i < N; i += (long)gridDim.x * kThreads) {
        const T d = Dm[i];
        const T pi = p[i];
        const T qi = d >= T(0) ? y[i] + d * pi : T(0);
        q[i] = qi;
        acc.add(pi * qi);
    }
    const double v[1] = {acc.get()};
    const int slot[1] = {kPQ};
    reduce_to<1>(v, part, sc, slot, counter);
}

// alpha = rz / pq; x += alpha p; r -= alpha q; ||r||^2 -> sc[kRR].
template <typename T>
__global__ void __launch_bounds__(kThreads) k_update(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                     const T* __restrict__ q, long N, int rz_slot, double* part,
                                                     double* sc, unsigned* counter) {
    const double pq = sc[kPQ];
    const T alpha = pq != 0.0 ? T(sc[rz_slot] / pq) : T(0);   // p = 0 only once r = 0 exactly
    Acc<T> acc;
    for (long i = (long)blockIdx.x * kThreads + threadIdx.x; i < N; i += (long)gridDim.x * kThreads) {
        x[i] += alpha * p[i];
        const T ri = r[i] - alpha * q[i];
        r[i] = ri;
        acc.add(ri * ri);
    }
    const double v[1] = {acc.get()};
    const int slot[1] = {kRR};
    reduce_to<1>(v, part, sc, slot, counter);
}

// z = Phi (r / sigma + y); r.z -> sc[rz_slot].
template <typename T>
__global__ void __launch_bounds__(kThreads) k_prec_post(const T* __restrict__ y, const T* __restrict__ r,
                                                        const T* __restrict__ Dm, T inv_sigma, T* __restrict__ z,
                                                        long N, int rz_slot, double* part, double* sc,
                                                        unsigned* counter) {
    Acc<T> acc;
    for (long i = (long)blockIdx.x * kThreads + threadIdx.x; i < N; i += (long)gridDim.x * kThreads) {
        const T ri = r[i];
        const T zi = Dm[i] >= T(0) ? ri * inv_sigma + y[i] : T(0);
        z[i] = zi;
        acc.add(ri * zi);
    }
    const double v[1] = {acc.get()};
    const int slot[1] = {rz_slot};
    reduce_to<1>(v, part, sc, slot, counter);
}

// p = z + beta p, beta = rz_new / rz_old (0 on the first direction).
template <typename T>
__global__ void k_dir(T* __restrict__ p, const T* __restrict__ z, long N, int first, int new_slot, int old_slot,
                      const double* __restrict__ sc) {
    const double rz_old = sc[old_slot];
    const T beta = (first || rz_old == 0.0) ? T(0) : T(sc[new_slot] / rz_old);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
        p[i] = first ? z[i] : z[i] + beta * p[i];
}

// out = post x (/ n_w), 0 off the mask.
template <typename T, typename TOUT>
__global__ void k_final(const T* __restrict__ x, const float* __restrict__ post, int post_div,
                        const float* __restrict__ nw, const T* __restrict__ Dm, TOUT* __restrict__ out, long N) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        T o = T(0);
        if (Dm[i] >= T(0)) {
            o = x[i];
            if (post) o *= T(post[i]);
            if (post_div) o /= T(nw[i]);
        }
        out[i] = TOUT(o);
    }
}

}  // namespace opt

// ---------------------------------------------------------------------------------------------- state

struct OptState {
    bool ready = false;
    size_t elem = 0;                 // sizeof(T) of the maps
    int nell_fid = 0, n_s = 0, max_iter = 0;
    double tol = 0.0, sigma = 0.0;
    uint64_t hash = 0;
    float* nw = nullptr;             // weighting density n_w [N]
    void* Dm = nullptr;              // n2_w / n_w^2, -1 off the mask [N], T
    void* wk = nullptr;              // box weights P(k) [nbox], T
    void* wm = nullptr;              // box weights 1/(P + sigma) - 1/sigma [nbox], T
    void* map[6] = {};               // x, r, z, p, q, y [N], T
    void* box = nullptr;             // box spectrum [nbox], C<T>
    void* f1 = nullptr;              // [N0][N1][Bz] C<T>: forward z-pass output / inverse y-pass output
    void* f2 = nullptr;              // [N0][By][Bz] C<T>: forward y-pass output / inverse x-pass output
    double* sc = nullptr;            // device scalars [kSlots]
    double* part = nullptr;          // block partials [2][kMaxBlocks]
    unsigned* counter = nullptr;
    double* hsc = nullptr;           // pinned host copy of the scalars
    // the two halves of an iteration with the r.z slots of parity 0 and 1, captured once per configuration:
    // half[par][0] = q = A p and the x, r update; half[par][1] = z = M^-1 r and the new direction
    cudaStream_t cap = nullptr;
    cudaGraphExec_t half[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    long half_launches[2] = {0, 0};
    int last_iters = 0;
    double last_relres = 0.0;
};

static void opt_drop_graphs(OptState* s) {
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            if (s->half[a][b]) { cudaGraphExecDestroy(s->half[a][b]); s->half[a][b] = nullptr; }
}

static void opt_free(OptState* s) {
    if (!s) return;
    opt_drop_graphs(s);
    if (s->cap) cudaStreamDestroy(s->cap);
    void* ptrs[] = {s->nw, s->Dm, s->wk, s->wm, s->map[0], s->map[1], s->map[2], s->map[3], s->map[4], s->map[5],
                    s->box, s->f1, s->f2, s->sc, s->part, s->counter};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (s->hsc) cudaFreeHost(s->hsc);
    delete s;
}

static unsigned opt_blocks(long n) {
    return (unsigned)std::max<long>(1, std::min<long>((n + opt::kThreads - 1) / opt::kThreads, opt::kMaxBlocks));
}

static uint64_t fnv(const void* p, size_t n, uint64_t h) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ULL; }
    return h;
}

template <typename T>
static int opt_configure_t(polybin_ctx* ctx, const float* nw, const float* n2w, const double* pfid, int nell_fid,
                           int n_s, int max_iter, double tol) {
    OptState* s = static_cast<OptState*>(ctx->opt);
    if (s && s->elem != sizeof(T)) { opt_free(s); s = nullptr; ctx->opt = nullptr; }
    if (!s) {
        s = new (std::nothrow) OptState();
        if (!s) return fail(ctx, POLYBIN_ENOMEM, "polybin_set_optimal: out of host memory");
        ctx->opt = s;
        s->elem = sizeof(T);
    }
    s->ready = false;
    opt_drop_graphs(s);   // the captured iterations carry 1 / sigma by value
    const long N = ctx->ncell;
    const long nbox = (long)ctx->gx.cnt * ctx->gy.cnt * ctx->gz.cnt;
    auto need = [&](void** p, size_t bytes) -> int {
        if (*p) return POLYBIN_OK;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) { *p = nullptr; return fail_cuda(ctx, e, "optimal weighting workspace", __FILE__, __LINE__); }
        return POLYBIN_OK;
    };
    int rc;
    if ((rc = need((void**)&s->nw, sizeof(float) * N))) return rc;
    if ((rc = need(&s->Dm, sizeof(T) * N))) return rc;
    if ((rc = need(&s->wk, sizeof(T) * nbox))) return rc;
    if ((rc = need(&s->wm, sizeof(T) * nbox))) return rc;
    for (int j = 0; j < 6; ++j)
        if ((rc = need(&s->map[j], sizeof(T) * N))) return rc;
    if ((rc = need(&s->box, sizeof(C<T>) * nbox))) return rc;
    if ((rc = need(&s->f1, sizeof(C<T>) * (size_t)ctx->N[0] * ctx->N[1] * ctx->gz.cnt))) return rc;
    if ((rc = need(&s->f2, sizeof(C<T>) * (size_t)ctx->N[0] * ctx->gy.cnt * ctx->gz.cnt))) return rc;
    if ((rc = need((void**)&s->sc, sizeof(double) * opt::kSlots))) return rc;
    if ((rc = need((void**)&s->part, sizeof(double) * 2 * opt::kMaxBlocks))) return rc;
    if (!s->counter) {
        if ((rc = need((void**)&s->counter, sizeof(unsigned)))) return rc;
        PB_CUDA_OK(cudaMemsetAsync(s->counter, 0, sizeof(unsigned), ctx->stream));
    }
    if (!s->hsc) {
        cudaError_t e = cudaMallocHost((void**)&s->hsc, sizeof(double) * opt::kSlots);
        if (e != cudaSuccess) { s->hsc = nullptr; return fail_cuda(ctx, e, "cudaMallocHost", __FILE__, __LINE__); }
    }
    // n_w, D and sigma
    PB_CUDA_OK(cudaMemcpyAsync(s->nw, nw, sizeof(float) * N, cudaMemcpyDeviceToDevice, ctx->stream));
    opt::k_dmap<T><<<opt_blocks(N), opt::kThreads, 0, ctx->stream>>>(nw, n2w, (T*)s->Dm, N, s->part, s->sc, s->counter);
    ctx->launches++;
    PB_CUDA_OK(cudaGetLastError());
    PB_CUDA_OK(cudaMemcpyAsync(s->hsc, s->sc, sizeof(double) * opt::kSlots, cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    const double cnt = s->hsc[opt::kDcnt];
    if (!(cnt > 0.0)) return fail(ctx, POLYBIN_EINVAL, "polybin_set_optimal: the weighting density n_w has no cell > 0");
    s->sigma = s->hsc[opt::kDsum] / cnt;
    if (!(s->sigma > 0.0) || !std::isfinite(s->sigma))
        return fail(ctx, POLYBIN_EINVAL, "polybin_set_optimal: mean n2_w / n_w^2 over the mask must be finite and > 0");
    // box weights: P(k) = sum_ell P_ell[s] L_ell(mu) for s < n_s, h = 1/(P + sigma) - 1/sigma
    const int Bx = ctx->gx.cnt, By = ctx->gy.cnt, Bz = ctx->gz.cnt;
    std::vector<T> hk(nbox), hm(nbox);
    for (int ix = 0; ix < Bx; ++ix)
        for (int iy = 0; iy < By; ++iy)
            for (int iz = 0; iz < Bz; ++iz) {
                const long fx = ctx->gx.lo + ix, fy = ctx->gy.lo + iy, fz = iz;
                const long sq = fx * fx + fy * fy + fz * fz;
                double P = 0.0;
                if (sq < n_s) {
                    const double mu2 = sq > 0 ? (double)(fz * fz) / (double)sq : 0.0;
                    for (int l = 0; l < nell_fid; ++l) {
                        const double L = l == 0 ? 1.0 : (l == 1 ? 0.5 * (3.0 * mu2 - 1.0)
                                                                : (35.0 * mu2 * mu2 - 30.0 * mu2 + 3.0) / 8.0);
                        P += pfid[(size_t)l * n_s + sq] * L;
                    }
                }
                if (!(P + s->sigma > 0.0))
                    return fail(ctx, POLYBIN_EINVAL, "polybin_set_optimal: P(k, mu) + sigma <= 0 at |n|^2 = %ld", sq);
                const long b = ((long)ix * By + iy) * Bz + iz;
                hk[b] = T(P);
                hm[b] = T(1.0 / (P + s->sigma) - 1.0 / s->sigma);
            }
    PB_CUDA_OK(cudaMemcpyAsync(s->wk, hk.data(), sizeof(T) * nbox, cudaMemcpyHostToDevice, ctx->stream));
    PB_CUDA_OK(cudaMemcpyAsync(s->wm, hm.data(), sizeof(T) * nbox, cudaMemcpyHostToDevice, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    s->nell_fid = nell_fid;
    s->n_s = n_s;
    s->max_iter = max_iter;
    s->tol = tol;
    // identity of the weighting (Fisher checkpoints and caches)
    std::vector<float> h1(N), h2(N);
    PB_CUDA_OK(cudaMemcpyAsync(h1.data(), nw, sizeof(float) * N, cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaMemcpyAsync(h2.data(), n2w, sizeof(float) * N, cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    uint64_t h = fnv(h1.data(), sizeof(float) * N, 1469598103934665603ULL);
    h = fnv(h2.data(), sizeof(float) * N, h);
    h = fnv(pfid, sizeof(double) * (size_t)nell_fid * n_s, h);
    h = fnv(&nell_fid, sizeof(int), h);
    h = fnv(&n_s, sizeof(int), h);
    h = fnv(&max_iter, sizeof(int), h);
    h = fnv(&tol, sizeof(double), h);
    s->hash = h;
    s->ready = true;
    return POLYBIN_OK;
}

static int opt_launched(polybin_ctx* ctx, const char* what) {
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(ctx, e, what, __FILE__, __LINE__);
    return POLYBIN_OK;
}

// z = M^-1 r = Phi (r / sigma + IFT_box[h FT_box[r]]) and r.z -> sc[slot].
template <typename T>
static int opt_precondition(polybin_ctx* ctx, OptState* s, int slot) {
    const long N = ctx->ncell;
    const long nbox = (long)ctx->gx.cnt * ctx->gy.cnt * ctx->gz.cnt;
    T* r = (T*)s->map[1];
    T* z = (T*)s->map[2];
    T* y = (T*)s->map[5];
    C<T>* box = (C<T>*)s->box;
    int rc;
    if ((rc = run_forward<T, T, T>(ctx, r, (const T*)nullptr, (const T*)nullptr, (C<T>*)s->f1, (C<T>*)s->f2, box))) return rc;
    opt::k_box_mul<T><<<opt_blocks(nbox), opt::kThreads, 0, ctx->stream>>>(box, (const T*)s->wm, nbox);
    if ((rc = opt_launched(ctx, "k_box_mul"))) return rc;
    if ((rc = run_inverse_box<T>(ctx, box, (C<T>*)s->f2, (C<T>*)s->f1, y, nullptr))) return rc;
    opt::k_prec_post<T><<<opt_blocks(N), opt::kThreads, 0, ctx->stream>>>(y, r, (const T*)s->Dm, T(1.0 / s->sigma), z, N,
                                                                           slot, s->part, s->sc, s->counter);
    return opt_launched(ctx, "k_prec_post");
}

// First half of iteration `par`: q = A p (pruned forward, times P on the box, pruned inverse, + D p on the mask),
// p.q, then x += alpha p, r -= alpha q with alpha = r.z / p.q (r.z in slot kRZ0 + par).
template <typename T>
static int opt_half_op(polybin_ctx* ctx, OptState* s, int par) {
    const long N = ctx->ncell;
    const long nbox = (long)ctx->gx.cnt * ctx->gy.cnt * ctx->gz.cnt;
    T* x = (T*)s->map[0];
    T* r = (T*)s->map[1];
    T* p = (T*)s->map[3];
    T* q = (T*)s->map[4];
    T* y = (T*)s->map[5];
    C<T>* box = (C<T>*)s->box;
    const unsigned nbk = opt_blocks(N);
    int rc;
    if ((rc = run_forward<T, T, T>(ctx, p, (const T*)nullptr, (const T*)nullptr, (C<T>*)s->f1, (C<T>*)s->f2, box)))
        return rc;
    opt::k_box_mul<T><<<opt_blocks(nbox), opt::kThreads, 0, ctx->stream>>>(box, (const T*)s->wk, nbox);
    if ((rc = opt_launched(ctx, "k_box_mul"))) return rc;
    if ((rc = run_inverse_box<T>(ctx, box, (C<T>*)s->f2, (C<T>*)s->f1, y, nullptr))) return rc;
    opt::k_op_post<T><<<nbk, opt::kThreads, 0, ctx->stream>>>(y, p, (const T*)s->Dm, q, N, s->part, s->sc, s->counter);
    if ((rc = opt_launched(ctx, "k_op_post"))) return rc;
    opt::k_update<T><<<nbk, opt::kThreads, 0, ctx->stream>>>(x, r, p, q, N, opt::kRZ0 + par, s->part, s->sc, s->counter);
    return opt_launched(ctx, "k_update");
}

// Second half of iteration `par`: z = M^-1 r with r.z into slot kRZ0 + (1 - par), p = z + beta p.
template <typename T>
static int opt_half_prec(polybin_ctx* ctx, OptState* s, int par) {
    const int cur = opt::kRZ0 + par, nxt = opt::kRZ0 + (1 - par);
    int rc;
    if ((rc = opt_precondition<T>(ctx, s, nxt))) return rc;
    opt::k_dir<T><<<opt_blocks(ctx->ncell), opt::kThreads, 0, ctx->stream>>>((T*)s->map[3], (const T*)s->map[2],
                                                                               ctx->ncell, 0, nxt, cur, s->sc);
    return opt_launched(ctx, "k_dir");
}

// Captures the four iteration halves into CUDA graphs (private capture stream; the graphs are launched on the
// context's stream).  They refer only to the configuration's own buffers, so they stay valid until it is replaced.
template <typename T>
static int opt_capture(polybin_ctx* ctx, OptState* s) {
    if (s->half[1][1]) return POLYBIN_OK;
    if (!s->cap) PB_CUDA_OK(cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking));
    for (int par = 0; par < 2; ++par)
        for (int h = 0; h < 2; ++h) {
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) { cudaGetLastError(); opt_drop_graphs(s); return fail_cuda(ctx, e, "cudaStreamBeginCapture", __FILE__, __LINE__); }
            cudaStream_t saved = ctx->stream;
            ctx->stream = s->cap;
            ctx->capturing = true;
            const long l0 = ctx->launches;
            int rc = h == 0 ? opt_half_op<T>(ctx, s, par) : opt_half_prec<T>(ctx, s, par);
            s->half_launches[h] = ctx->launches - l0;
            ctx->launches = l0;
            ctx->capturing = false;
            ctx->stream = saved;
            e = cudaStreamEndCapture(s->cap, &graph);
            if (rc || e != cudaSuccess) {
                cudaGetLastError();
                if (graph) cudaGraphDestroy(graph);
                opt_drop_graphs(s);
                return rc ? rc : fail_cuda(ctx, e, "cudaStreamEndCapture", __FILE__, __LINE__);
            }
            e = cudaGraphInstantiate(&s->half[par][h], graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) { s->half[par][h] = nullptr; opt_drop_graphs(s); return fail_cuda(ctx, e, "cudaGraphInstantiate", __FILE__, __LINE__); }
        }
    return POLYBIN_OK;
}

template <typename T, typename TIN, typename TOUT>
int opt_apply(polybin_ctx* ctx, const TIN* v, const float* pre, int pre_div, const float* post, int post_div, TOUT* out) {
    OptState* s = static_cast<OptState*>(ctx->opt);
    if (!s || !s->ready) return fail(ctx, POLYBIN_ENOTREADY, "optimal weighting: call polybin_set_optimal first");
    if (s->elem != sizeof(T)) return fail(ctx, POLYBIN_EINVAL, "optimal weighting: configured in another precision");
    const long N = ctx->ncell;
    T* x = (T*)s->map[0];
    T* r = (T*)s->map[1];
    T* z = (T*)s->map[2];
    T* p = (T*)s->map[3];
    const T* Dm = (const T*)s->Dm;
    const unsigned nbk = opt_blocks(N);
    int rc;
    opt::k_init<T, TIN><<<nbk, opt::kThreads, 0, ctx->stream>>>(v, pre, pre_div, s->nw, Dm, r, x, N, s->part, s->sc,
                                                                 s->counter);
    if ((rc = opt_launched(ctx, "k_init"))) return rc;
    PB_CUDA_OK(cudaMemcpyAsync(s->hsc, s->sc, sizeof(double) * opt::kSlots, cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    const double bb = s->hsc[opt::kBB];
    if (!std::isfinite(bb)) return fail(ctx, POLYBIN_EINVAL, "optimal weighting: the input map is not finite on the mask");
    int it = 0;
    if (bb > 0.0) {
        if ((rc = opt_precondition<T>(ctx, s, opt::kRZ0))) return rc;
        opt::k_dir<T><<<nbk, opt::kThreads, 0, ctx->stream>>>(p, z, N, 1, opt::kRZ0, opt::kRZ0, s->sc);
        if ((rc = opt_launched(ctx, "k_dir"))) return rc;
        const bool graphs = !ctx->capturing && opt_capture<T>(ctx, s) == POLYBIN_OK;
        if (!graphs) cudaGetLastError();
        auto half = [&](int par, int h) -> int {
            if (!graphs) return h == 0 ? opt_half_op<T>(ctx, s, par) : opt_half_prec<T>(ctx, s, par);
            cudaError_t e = cudaGraphLaunch(s->half[par][h], ctx->stream);
            if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaGraphLaunch", __FILE__, __LINE__);
            ctx->launches += s->half_launches[h];
            return POLYBIN_OK;
        };
        while (it < s->max_iter) {
            if ((rc = half(it & 1, 0))) return rc;
            ++it;
            if (it == s->max_iter) break;
            if (s->tol > 0.0) {
                PB_CUDA_OK(cudaMemcpyAsync(s->hsc, s->sc, sizeof(double) * opt::kSlots, cudaMemcpyDeviceToHost, ctx->stream));
                PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
                const double rel = std::sqrt(s->hsc[opt::kRR] / bb);
                if (!std::isfinite(rel))
                    return fail(ctx, POLYBIN_ETOL, "optimal weighting: conjugate gradients broke down (operator not positive definite?)");
                if (rel <= s->tol) break;
            }
            if ((rc = half((it - 1) & 1, 1))) return rc;
        }
    }
    opt::k_final<T, TOUT><<<nbk, opt::kThreads, 0, ctx->stream>>>(x, post, post_div, s->nw, Dm, out, N);
    if ((rc = opt_launched(ctx, "k_final"))) return rc;
    PB_CUDA_OK(cudaMemcpyAsync(s->hsc, s->sc, sizeof(double) * opt::kSlots, cudaMemcpyDeviceToHost, ctx->stream));
    PB_CUDA_OK(cudaStreamSynchronize(ctx->stream));
    s->last_iters = it;
    s->last_relres = bb > 0.0 ? std::sqrt(s->hsc[opt::kRR] / bb) : 0.0;
    if (!std::isfinite(s->last_relres))
        return fail(ctx, POLYBIN_ETOL, "optimal weighting: conjugate gradients broke down (operator not positive definite?)");
    return POLYBIN_OK;
}

template int opt_apply<float, float, float>(polybin_ctx*, const float*, const float*, int, const float*, int, float*);
template int opt_apply<double, double, double>(polybin_ctx*, const double*, const float*, int, const float*, int, double*);
template int opt_apply<double, float, double>(polybin_ctx*, const float*, const float*, int, const float*, int, double*);

uint64_t opt_hash(const polybin_ctx* ctx) {
    const OptState* s = static_cast<const OptState*>(ctx->opt);
    return s && s->ready ? s->hash : 0;
}

void opt_stats(const polybin_ctx* ctx, int* iters, double* relres) {
    const OptState* s = static_cast<const OptState*>(ctx->opt);
    if (iters) *iters = s ? s->last_iters : 0;
    if (relres) *relres = s ? s->last_relres : 0.0;
}

void destroy_optimal(polybin_ctx* ctx) {
    opt_free(static_cast<OptState*>(ctx->opt));
    ctx->opt = nullptr;
}

}  // namespace pb

using namespace pb;

static bool opt_is_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

extern "C" int polybin_max_shell(polybin_ctx* ctx, int* smax) {
    if (!ctx || !smax) return fail(ctx, POLYBIN_EINVAL, "polybin_max_shell: NULL argument");
    *smax = ctx->smax;
    return POLYBIN_OK;
}

extern "C" int polybin_set_optimal(polybin_ctx* ctx, const float* n_w_dev, const float* n2_w_dev, const double* pfid,
                                   int nell_fid, int n_s, int max_iter, double tol) {
    if (!ctx || !n_w_dev || !pfid) return fail(ctx, POLYBIN_EINVAL, "polybin_set_optimal: NULL argument");
    if (!opt_is_device(n_w_dev) || (n2_w_dev && !opt_is_device(n2_w_dev)))
        return fail(ctx, POLYBIN_EINVAL, "polybin_set_optimal: n_w and n2_w must be device memory");
    if (nell_fid < 1 || nell_fid > 3 || n_s < 1 || n_s > ctx->smax + 1 || max_iter < 1 || !(tol >= 0.0) || !std::isfinite(tol))
        return fail(ctx, POLYBIN_EINVAL,
                    "polybin_set_optimal: nell_fid in 1..3, 1 <= n_s <= %d (largest binned |n|^2 + 1), max_iter >= 1, tol >= 0",
                    ctx->smax + 1);
    for (size_t i = 0; i < (size_t)nell_fid * n_s; ++i)
        if (!std::isfinite(pfid[i])) return fail(ctx, POLYBIN_EINVAL, "polybin_set_optimal: fiducial table is not finite");
    const float* n2 = n2_w_dev ? n2_w_dev : n_w_dev;
    return ctx->prec == POLYBIN_FP64 ? opt_configure_t<double>(ctx, n_w_dev, n2, pfid, nell_fid, n_s, max_iter, tol)
                                     : opt_configure_t<float>(ctx, n_w_dev, n2, pfid, nell_fid, n_s, max_iter, tol);
}

extern "C" int polybin_sinv_optimal(polybin_ctx* ctx, const float* v_dev, int transpose, void* out_dev, int* iters_out,
                                    double* relres_out) {
    if (!ctx || !v_dev || !out_dev) return fail(ctx, POLYBIN_EINVAL, "polybin_sinv_optimal: NULL argument");
    if (!opt_is_device(v_dev) || !opt_is_device(out_dev))
        return fail(ctx, POLYBIN_EINVAL, "polybin_sinv_optimal: device pointers required");
    if (transpose != 0 && transpose != 1) return fail(ctx, POLYBIN_EINVAL, "polybin_sinv_optimal: transpose is 0 or 1");
    int rc = ctx->prec == POLYBIN_FP64
                 ? opt_apply<double, float, double>(ctx, v_dev, nullptr, !transpose, nullptr, transpose, (double*)out_dev)
                 : opt_apply<float, float, float>(ctx, v_dev, nullptr, !transpose, nullptr, transpose, (float*)out_dev);
    if (rc) return rc;
    opt_stats(ctx, iters_out, relres_out);
    return POLYBIN_OK;
}
